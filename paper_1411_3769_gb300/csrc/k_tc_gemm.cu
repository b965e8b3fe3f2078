// Tensor-core GEMM for sm_103a: TMA loads into a 128-byte-swizzled shared-memory
// ring, one thread issues tcgen05.mma into a TMEM accumulator, four warps drain
// it with tcgen05.ld.  Used for the FP32 (3xTF32) Schur contraction and the
// FP32 Cholesky trailing update of the mixed-precision path and for the BF16
// MLP layers.
//
//   D[m][n] = sum_k A[m][k] * B[n][k]      (A: M x Kd, B: N x Kd, both K-major)
//   C[n*ldc + m] = alpha * D[m][n] + beta * C[n*ldc + m]   (column-major store)
//
// kind::tf32 reads FP32 data and keeps 10 explicit mantissa bits.  With
// split = 3 the operands arrive as (hi, lo) pairs, hi = tf32(x), lo = x - hi,
// and D accumulates hi*hi + hi*lo + lo*hi (the 3xTF32 technique), which keeps
// close to FP32 accuracy.  kind::f16 with BF16 operands serves the MLP.
//
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the thread
// raises FL_TIMEOUT in *flag and the CTA unwinds, freeing its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "psdp_internal.h"
#include "tc_ptx.cuh"

namespace {

constexpr int BM = 128, BN = 128;
constexpr int ROW_BYTES = 128;                    // one swizzle row = BK elements
constexpr int TILE_A = BM * ROW_BYTES;            // 16 KB
constexpr int TILE_B = BN * ROW_BYTES;            // 16 KB

// shared-memory matrix descriptor: K-major, SWIZZLE_128B, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;               // descriptor version
    d |= (uint64_t)2 << 61;               // SWIZZLE_128B
    return d;
}
template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (BF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}
// instruction descriptor: F32 accumulate, A/B format (TF32 = 2, BF16 = 1), K-major, N = BN, M = BM
template <bool BF16>
__host__ __device__ constexpr uint32_t make_idesc() {
    return (1u << 4) | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

template <bool BF16, int SPLIT, int STAGES>
__global__ void __launch_bounds__(128, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
          const __grid_constant__ CUtensorMap mAlo, const __grid_constant__ CUtensorMap mBlo, int M, int N, int b0,
          const int32_t* __restrict__ kd, int kd_uniform, float* C, int64_t ldc, int64_t c_batch, float alpha,
          float beta, int tri, int* flag, float* aux_hi, float* aux_lo, int aux_ld, int aux_m0, int aux_n1) {
    constexpr int STAGE_BYTES = (SPLIT == 3) ? 2 * (TILE_A + TILE_B) : (TILE_A + TILE_B);
    constexpr int BK = BF16 ? 64 : 32;            // elements per 128-byte row
    constexpr int KSTEP_BYTES = 32;               // bytes of K consumed by one MMA (K = 8 tf32 / 16 bf16)
    extern __shared__ uint8_t smem_raw[];
    const int nt = blockIdx.x, mt = blockIdx.y, b = blockIdx.z;
    if (tri && mt < nt) return;
    const uint32_t base_raw = smem_u32(smem_raw);
    const uint32_t base = (base_raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - base_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + STAGES * STAGE_BYTES);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
    __shared__ int abort_flag;
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * STAGES, accb = full0 + 16 * STAGES;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Kd = kd ? kd[b] : kd_uniform;
    const int nk = (Kd + BK - 1) / BK;
    const int m0 = mt * BM, n0 = nt * BN;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;

    if (nk > 0) {
        if (warp == 0 && lane == 0) {
            // TMA producer
            for (int kt = 0; kt < nk; ++kt) {
                const int s = kt % STAGES;
                if (kt >= STAGES && !mbar_wait(empty0 + 8 * s, ((kt / STAGES) - 1) & 1, flag)) {
                    abort_flag = 1;
                    break;
                }
                const uint32_t st = base + s * STAGE_BYTES;
                const uint32_t fb = full0 + 8 * s;
                mbar_expect_tx(fb, STAGE_BYTES);
                tma_load_3d(st, &mA, fb, kt * BK, m0, b0 + b);
                tma_load_3d(st + TILE_A, &mB, fb, kt * BK, n0, b0 + b);
                if constexpr (SPLIT == 3) {
                    tma_load_3d(st + TILE_A + TILE_B, &mAlo, fb, kt * BK, m0, b0 + b);
                    tma_load_3d(st + 2 * TILE_A + TILE_B, &mBlo, fb, kt * BK, n0, b0 + b);
                }
            }
        } else if (warp == 1 && lane == 0) {
            // MMA issuer
            constexpr uint32_t idesc = make_idesc<BF16>();
            for (int kt = 0; kt < nk; ++kt) {
                const int s = kt % STAGES;
                if (!mbar_wait(full0 + 8 * s, (kt / STAGES) & 1, flag)) {
                    abort_flag = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t st = base + s * STAGE_BYTES;
                const uint32_t aH = st, bH = st + TILE_A;
#pragma unroll
                for (int kk = 0; kk < ROW_BYTES / KSTEP_BYTES; ++kk) {
                    const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                    mma<BF16>(tmem, sdesc(aH + kk * KSTEP_BYTES), sdesc(bH + kk * KSTEP_BYTES), idesc, acc);
                    if constexpr (SPLIT == 3) {
                        const uint32_t aL = st + TILE_A + TILE_B, bL = st + 2 * TILE_A + TILE_B;
                        mma<BF16>(tmem, sdesc(aH + kk * KSTEP_BYTES), sdesc(bL + kk * KSTEP_BYTES), idesc, 1u);
                        mma<BF16>(tmem, sdesc(aL + kk * KSTEP_BYTES), sdesc(bH + kk * KSTEP_BYTES), idesc, 1u);
                    }
                }
                mma_commit(empty0 + 8 * s);
            }
            mma_commit(accb);
        }
    }
    __syncwarp();
    // epilogue: every warp drains its 32 TMEM lanes (rows m0 + 32*warp + lane).
    // With beta != 0 the thread's 128 old C values are loaded before waiting for
    // the accumulator, so their latency overlaps the tail of the main loop
    // instead of being paid once per column.
    const int m = m0 + 32 * warp + lane;
    float* Cb = C + (int64_t)b * c_batch;
    float old[BN];
#pragma unroll
    for (int j = 0; j < BN; ++j) old[j] = 0.f;
    if (beta != 0.f && m < M) {
#pragma unroll
        for (int j = 0; j < BN; ++j) {
            const int n = n0 + j;
            if (n < N) old[j] = Cb[(int64_t)n * ldc + m];
        }
    }
    bool ok = true;
    if (nk > 0) ok = mbar_wait(accb, 0, flag);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            if (nk > 0) {
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, r);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) r[j] = 0u;
            }
            if (m < M) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    v[j] = alpha * __uint_as_float(r[j]) + beta * old[c0 + j];
                    if (n < N) Cb[(int64_t)n * ldc + m] = v[j];
                }
                if (aux_hi && m >= aux_m0) {
                    // the same values as (hi, lo) TF32 pairs, row-major [m - aux_m0][n] for
                    // n < aux_n1 (the K-major operand layout of a following product)
                    float* ph = aux_hi + (int64_t)(m - aux_m0) * aux_ld + n0 + c0;
                    float* pl = aux_lo + (int64_t)(m - aux_m0) * aux_ld + n0 + c0;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (n0 + c0 + j < N && n0 + c0 + j < aux_n1) {
                            uint32_t h;
                            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v[j]));
                            ph[j] = __uint_as_float(h);
                            pl[j] = v[j] - __uint_as_float(h);
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
    }
}

// Tiles of one (optionally lower-triangular, tiles mt >= nt) M x N update,
// column by column: nt ascending, mt ascending inside a column.
struct TileWalk {
    int MT, NT, tri, nt, off;
    __device__ TileWalk(int M, int N, int tri_, int start)
        : MT((M + BM - 1) / BM), NT((N + BN - 1) / BN), tri(tri_), nt(0), off(start) { settle(); }
    __device__ int len(int c) const { return tri ? (MT > c ? MT - c : 0) : MT; }
    __device__ void settle() {
        while (nt < NT && off >= len(nt)) {
            off -= len(nt);
            ++nt;
        }
    }
    __device__ bool valid() const { return nt < NT; }
    __device__ int mt() const { return tri ? nt + off : off; }
    __device__ void advance(int step) {
        off += step;
        settle();
    }
};

// Persistent form of k_tc_gemm for one large update (batch 1): one CTA per SM
// walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...  Warp 0 issues the
// TMA loads, warp 1 the MMAs (and owns TMEM), warps 2-9 drain the accumulators.
// Two TMEM accumulators of BN columns alternate between tiles and each has its
// own group of four epilogue warps, so the epilogues of two tiles (each reads
// and writes its C tile in HBM) run at once and under the MMAs and loads of
// the next.  Barriers: full/empty per stage (TMA <-> MMA), tfull/tempty per
// accumulator (MMA <-> epilogue, tempty counts the group's four warps).
constexpr int kPersistThreads = 320;
template <int SPLIT, int STAGES>
__global__ void __launch_bounds__(kPersistThreads, 1)
k_tc_gemm_persist(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                  const __grid_constant__ CUtensorMap mAlo, const __grid_constant__ CUtensorMap mBlo, int M, int N,
                  int Kd, float* C, int64_t ldc, float alpha, float beta, int tri, int* flag) {
    constexpr int STAGE_BYTES = (SPLIT == 3) ? 2 * (TILE_A + TILE_B) : (TILE_A + TILE_B);
    constexpr int BK = 32;                        // TF32 elements per 128-byte row
    constexpr int KSTEP_BYTES = 32;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t base_raw = smem_u32(smem_raw);
    const uint32_t base = (base_raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - base_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + STAGES * STAGE_BYTES);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
    __shared__ int abort_flag;
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * STAGES;
    const uint32_t tfull0 = full0 + 16 * STAGES, tempty0 = tfull0 + 16, drain = tfull0 + 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (Kd + BK - 1) / BK;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull0 + 8 * b, 1);
            mbar_init(tempty0 + 8 * b, 4);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(2 * BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;

    if (nk > 0 && warp == 0 && lane == 0) {
        // TMA producer
        int g = 0;
        for (TileWalk t(M, N, tri, blockIdx.x); t.valid() && !*(volatile int*)&abort_flag; t.advance(gridDim.x)) {
            const int m0 = t.mt() * BM, n0 = t.nt * BN;
            for (int kt = 0; kt < nk; ++kt, ++g) {
                const int s = g % STAGES;
                if (g >= STAGES && !mbar_wait(empty0 + 8 * s, ((g / STAGES) - 1) & 1, flag)) {
                    abort_flag = 1;
                    break;
                }
                const uint32_t st = base + s * STAGE_BYTES;
                const uint32_t fb = full0 + 8 * s;
                mbar_expect_tx(fb, STAGE_BYTES);
                tma_load_3d(st, &mA, fb, kt * BK, m0, 0);
                tma_load_3d(st + TILE_A, &mB, fb, kt * BK, n0, 0);
                if constexpr (SPLIT == 3) {
                    tma_load_3d(st + TILE_A + TILE_B, &mAlo, fb, kt * BK, m0, 0);
                    tma_load_3d(st + 2 * TILE_A + TILE_B, &mBlo, fb, kt * BK, n0, 0);
                }
            }
        }
        // every issued stage has landed before the CTA may exit
        for (int q = (g > STAGES ? g - STAGES : 0); q < g; ++q) mbar_wait(full0 + 8 * (q % STAGES), (q / STAGES) & 1, flag);
    } else if (nk > 0 && warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = make_idesc<false>();
        int g = 0, i = 0;
        bool issued = false;
        for (TileWalk t(M, N, tri, blockIdx.x); t.valid() && !*(volatile int*)&abort_flag; t.advance(gridDim.x), ++i) {
            const int b = i & 1;
            const uint32_t tacc = tmem + (uint32_t)(b * BN);
            if (i >= 2 && !mbar_wait(tempty0 + 8 * b, ((i >> 1) - 1) & 1, flag)) {
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int kt = 0; kt < nk; ++kt, ++g) {
                const int s = g % STAGES;
                if (!mbar_wait(full0 + 8 * s, (g / STAGES) & 1, flag)) {
                    abort_flag = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t st = base + s * STAGE_BYTES;
                const uint32_t aH = st, bH = st + TILE_A;
#pragma unroll
                for (int kk = 0; kk < ROW_BYTES / KSTEP_BYTES; ++kk) {
                    const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                    mma<false>(tacc, sdesc(aH + kk * KSTEP_BYTES), sdesc(bH + kk * KSTEP_BYTES), idesc, acc);
                    if constexpr (SPLIT == 3) {
                        const uint32_t aL = st + TILE_A + TILE_B, bL = st + 2 * TILE_A + TILE_B;
                        mma<false>(tacc, sdesc(aH + kk * KSTEP_BYTES), sdesc(bL + kk * KSTEP_BYTES), idesc, 1u);
                        mma<false>(tacc, sdesc(aL + kk * KSTEP_BYTES), sdesc(bH + kk * KSTEP_BYTES), idesc, 1u);
                    }
                }
                issued = true;
                mma_commit(empty0 + 8 * s);
            }
            if (*(volatile int*)&abort_flag) break;
            mma_commit(tfull0 + 8 * b);
        }
        // all MMAs complete before TMEM is released
        if (issued) {
            mma_commit(drain);
            mbar_wait(drain, 0, flag);
        }
    } else if (warp >= 2) {
        // epilogue: two groups of four warps, group g drains the tiles i = g
        // (mod 2), i.e. accumulator g, so two tiles' C traffic is in flight at
        // once; warp w reads TMEM lanes 32*(w%4) .. +31 (rows m0 + 32*(w%4) + lane)
        const int qd = warp & 3, grp = (warp - 2) >> 2;
        int i = 0;
        for (TileWalk t(M, N, tri, blockIdx.x); t.valid(); t.advance(gridDim.x), ++i) {
            if ((i & 1) != grp) continue;
            const int b = i & 1;
            const int m0 = t.mt() * BM, n0 = t.nt * BN;
            const int m = m0 + 32 * qd + lane;
            float old[BN];
#pragma unroll
            for (int j = 0; j < BN; ++j) old[j] = 0.f;
            if (beta != 0.f && m < M) {
#pragma unroll
                for (int j = 0; j < BN; ++j) {
                    const int n = n0 + j;
                    if (n < N) old[j] = C[(int64_t)n * ldc + m];
                }
            }
            // warp-uniform decision: the TMEM loads below are warp-collective
            const bool ok = __all_sync(0xffffffffu, nk > 0 && mbar_wait(tfull0 + 8 * b, (i >> 1) & 1, flag));
            if (!ok) {
                if (nk > 0) abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(b * BN + c0), r);
                if (m < M) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int n = n0 + c0 + j;
                        if (n < N) C[(int64_t)n * ldc + m] = alpha * __uint_as_float(r[j]) + beta * old[c0 + j];
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty0 + 8 * b);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    }
    return fn;
}

template <bool BF16, int SPLIT, int STAGES>
constexpr size_t smem_bytes() {
    return (size_t)STAGES * ((SPLIT == 3) ? 2 * (TILE_A + TILE_B) : (TILE_A + TILE_B)) + 1024 + 8 * (2 * STAGES + 1) + 16;
}

template <int SPLIT, int STAGES>
constexpr size_t smem_bytes_persist() {
    return (size_t)STAGES * ((SPLIT == 3) ? 2 * (TILE_A + TILE_B) : (TILE_A + TILE_B)) + 1024 +
           8 * (2 * STAGES + 5) + 16;
}

}  // namespace

// 3-D tensor map over a K-major operand: element (k, row, batch) at
// base + batch*batch_stride + row*row_stride + k (elements); box = 128 B of k x box_rows rows.
bool tc_make_map(CUtensorMap* map, const void* base, bool bf16, int64_t kdim, int64_t rows, int64_t batch,
                 int64_t row_stride, int64_t batch_stride, int box_rows) {
    auto enc = encoder();
    if (!enc) return false;
    const int es = bf16 ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)kdim, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)(row_stride * es), (cuuint64_t)(batch_stride * es)};
    cuuint32_t box[3] = {(cuuint32_t)(ROW_BYTES / es), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    if (batch == 1) strides[1] = (cuuint64_t)(rows * row_stride * es);
    CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                     const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The same with a chosen swizzle (32, 64 or 128 bytes) and a box of box_k
// elements along k (box_k * element size must not exceed the swizzle span).
bool tc_make_map_swz(CUtensorMap* map, const void* base, bool bf16, int64_t kdim, int64_t rows, int64_t batch,
                     int64_t row_stride, int64_t batch_stride, int box_k, int box_rows, int swizzle_bytes) {
    auto enc = encoder();
    if (!enc) return false;
    const int es = bf16 ? 2 : 4;
    if (box_k * es > swizzle_bytes) return false;
    const CUtensorMapSwizzle sw = swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                  : swizzle_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                                        : CU_TENSOR_MAP_SWIZZLE_NONE;
    cuuint64_t dims[3] = {(cuuint64_t)kdim, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)(row_stride * es), (cuuint64_t)(batch_stride * es)};
    cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    if (batch == 1) strides[1] = (cuuint64_t)(rows * row_stride * es);
    CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                     const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// D = A B^T over a batch; see the file header.  Returns false if a tensor map
// could not be encoded (nothing is launched then).
bool launch_tc_gemm(cudaStream_t st, bool bf16, int split, const CUtensorMap& A, const CUtensorMap& B,
                    const CUtensorMap* Alo, const CUtensorMap* Blo, int M, int N, int batch, int b0,
                    const int32_t* kd, int kd_uniform, float* C, int64_t ldc, int64_t c_batch, float alpha,
                    float beta, int tri, int* flag, float* aux_hi, float* aux_lo, int aux_ld, int aux_m0,
                    int aux_n1) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
    if (aux_n1 <= 0) aux_n1 = N;
    if (grid.x == 0 || grid.y == 0 || batch <= 0) return true;
    if (bf16) {
        k_tc_gemm<true, 1, 4><<<grid, 128, smem_bytes<true, 1, 4>(), st>>>(A, B, A, B, M, N, b0, kd, kd_uniform, C,
                                                                         ldc, c_batch, alpha, beta, tri, flag,
                                                                         aux_hi, aux_lo, aux_ld, aux_m0, aux_n1);
    } else if (split == 3) {
        k_tc_gemm<false, 3, 3><<<grid, 128, smem_bytes<false, 3, 3>(), st>>>(A, B, *Alo, *Blo, M, N, b0, kd,
                                                                           kd_uniform, C, ldc, c_batch, alpha, beta,
                                                                           tri, flag, aux_hi, aux_lo, aux_ld, aux_m0, aux_n1);
    } else {
        k_tc_gemm<false, 1, 4><<<grid, 128, smem_bytes<false, 1, 4>(), st>>>(A, B, A, B, M, N, b0, kd, kd_uniform, C,
                                                                           ldc, c_batch, alpha, beta, tri, flag,
                                                                           aux_hi, aux_lo, aux_ld, aux_m0, aux_n1);
    }
    return true;
}

// Persistent TF32 update of one M x N matrix (batch 1, maps with batch extent 1):
// C[n*ldc + m] = alpha * sum_k A[m][k] B[n][k] + beta * C, lower-triangular tiles
// only when tri.  ctas = number of persistent CTAs (at most the tile count).
bool launch_tc_gemm_persist(cudaStream_t st, int split, const CUtensorMap& A, const CUtensorMap& B,
                            const CUtensorMap* Alo, const CUtensorMap* Blo, int M, int N, int kd, float* C,
                            int64_t ldc, float alpha, float beta, int tri, int ctas, int* flag) {
    if (M <= 0 || N <= 0 || kd <= 0) return true;
    const int64_t MT = (M + BM - 1) / BM, NT = (N + BN - 1) / BN;
    int64_t tiles = 0;
    for (int64_t c = 0; c < NT; ++c) tiles += tri ? std::max<int64_t>(0, MT - c) : MT;
    if (tiles == 0) return true;
    const int grid = (int)std::min<int64_t>(tiles, std::max(1, ctas));
    if (split == 3)
        k_tc_gemm_persist<3, 3><<<grid, kPersistThreads, smem_bytes_persist<3, 3>(), st>>>(A, B, *Alo, *Blo, M, N, kd, C, ldc,
                                                                              alpha, beta, tri, flag);
    else
        k_tc_gemm_persist<1, 4><<<grid, kPersistThreads, smem_bytes_persist<1, 4>(), st>>>(A, B, A, B, M, N, kd, C, ldc, alpha,
                                                                              beta, tri, flag);
    return true;
}

void init_attrs_tc(int smem_optin) {
    set_max_dynamic_smem((const void*)k_tc_gemm_persist<3, 3>, smem_optin);
    set_max_dynamic_smem((const void*)k_tc_gemm_persist<1, 4>, smem_optin);
    set_max_dynamic_smem((const void*)k_tc_gemm<true, 1, 4>, smem_optin);
    set_max_dynamic_smem((const void*)k_tc_gemm<false, 3, 3>, smem_optin);
    set_max_dynamic_smem((const void*)k_tc_gemm<false, 1, 4>, smem_optin);
}

// The same limit for the two FP32 forms of k_tc_gemm only, reporting the first
// failing runtime call instead of clearing it.
cudaError_t set_attrs_tc_gemm_fp32(int smem_optin) {
    const void* fns[2] = {(const void*)k_tc_gemm<false, 3, 3>, (const void*)k_tc_gemm<false, 1, 4>};
    for (const void* f : fns) {
        cudaFuncAttributes a;
        cudaError_t e = cudaFuncGetAttributes(&a, f);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin - (int)a.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {
// hi = tf32(x) (round to nearest, ties away), lo = x - hi, both FP32
__global__ void k_split_tf32(int64_t n, const float* __restrict__ x, float* hi, float* lo) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[i];
        uint32_t h;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
        const float hf = __uint_as_float(h);
        hi[i] = hf;
        lo[i] = v - hf;
    }
}
}  // namespace

void launch_split_tf32(cudaStream_t st, int64_t n, const float* x, float* hi, float* lo) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks < 1) blocks = 1;
    k_split_tf32<<<(int)blocks, 256, 0, st>>>(n, x, hi, lo);
}

// Self-test of the tensor-core GEMM on host data: C (N x M, column-major D) =
// A (M x K) B^T (B: N x K).  dtype 0 = FP32 through kind::tf32 (split 1 or 3),
// 1 = BF16 (A, B given as uint16 bit patterns) through kind::f16.
extern "C" psdp_status psdp_tc_gemm_check(int M, int N, int K, int dtype, int split, const void* A, const void* B,
                                          float* C) {
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || (dtype != 0 && dtype != 1) || (split != 1 && split != 3) ||
        (dtype == 1 && split != 1))
        return PSDP_EINVAL;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    init_attrs_tc(optin);
    const int es = dtype ? 2 : 4;
    const int kpad = (K + 63) / 64 * 64;   // rows padded to a 16-byte-aligned stride
    void *dA = nullptr, *dB = nullptr, *dAl = nullptr, *dBl = nullptr, *dAh = nullptr, *dBh = nullptr;
    float* dC = nullptr;
    int* dflag = nullptr;
    psdp_status s = PSDP_OK;
    cudaStream_t st;
    cudaStreamCreate(&st);
    auto al = [&](void** p, size_t b) { if (cudaMalloc(p, b) != cudaSuccess) s = PSDP_ENOMEM; };
    al(&dA, (size_t)M * kpad * es);
    al(&dB, (size_t)N * kpad * es);
    al((void**)&dC, (size_t)M * N * 4);
    al((void**)&dflag, 4);
    if (split == 3) {
        al(&dAh, (size_t)M * kpad * 4); al(&dAl, (size_t)M * kpad * 4);
        al(&dBh, (size_t)N * kpad * 4); al(&dBl, (size_t)N * kpad * 4);
    }
    if (s == PSDP_OK) {
        cudaMemset(dA, 0, (size_t)M * kpad * es);
        cudaMemset(dB, 0, (size_t)N * kpad * es);
        cudaMemset(dflag, 0, 4);
        cudaMemcpy2D(dA, (size_t)kpad * es, A, (size_t)K * es, (size_t)K * es, M, cudaMemcpyHostToDevice);
        cudaMemcpy2D(dB, (size_t)kpad * es, B, (size_t)K * es, (size_t)K * es, N, cudaMemcpyHostToDevice);
        CUtensorMap mA, mB, mAl, mBl;
        bool ok;
        if (split == 3) {
            launch_split_tf32(st, (int64_t)M * kpad, (const float*)dA, (float*)dAh, (float*)dAl);
            launch_split_tf32(st, (int64_t)N * kpad, (const float*)dB, (float*)dBh, (float*)dBl);
            ok = tc_make_map(&mA, dAh, false, K, M, 1, kpad, 0, 128) && tc_make_map(&mB, dBh, false, K, N, 1, kpad, 0, 128) &&
                 tc_make_map(&mAl, dAl, false, K, M, 1, kpad, 0, 128) && tc_make_map(&mBl, dBl, false, K, N, 1, kpad, 0, 128);
            if (ok) launch_tc_gemm(st, false, 3, mA, mB, &mAl, &mBl, M, N, 1, 0, nullptr, K, dC, M, 0, 1.f, 0.f, 0, dflag);
        } else {
            ok = tc_make_map(&mA, dA, dtype == 1, K, M, 1, kpad, 0, 128) &&
                 tc_make_map(&mB, dB, dtype == 1, K, N, 1, kpad, 0, 128);
            if (ok) launch_tc_gemm(st, dtype == 1, 1, mA, mB, nullptr, nullptr, M, N, 1, 0, nullptr, K, dC, M, 0, 1.f, 0.f, 0, dflag);
        }
        if (!ok) s = PSDP_ECUDA;
        int flag = 0;
        if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) s = PSDP_ECUDA;
        cudaMemcpy(&flag, dflag, 4, cudaMemcpyDeviceToHost);
        if (flag) s = PSDP_ETIMEOUT;
        if (s == PSDP_OK) cudaMemcpy(C, dC, (size_t)M * N * 4, cudaMemcpyDeviceToHost);
    }
    for (void* p : {dA, dB, dAl, dBl, dAh, dBh, (void*)dC, (void*)dflag})
        if (p) cudaFree(p);
    cudaStreamDestroy(st);
    cudaGetLastError();
    return s;
}

extern "C" psdp_status psdp_tc_gemm_persist_check(int M, int N, int K, int split, int tri, int ctas, const float* A,
                                                  const float* B, float* C, float* ms) {
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || (split != 1 && split != 3) || ctas < 1) return PSDP_EINVAL;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    init_attrs_tc(optin);
    const int kpad = (K + 31) / 32 * 32;   // 128-byte rows
    float *dA = nullptr, *dB = nullptr, *dAl = nullptr, *dBl = nullptr, *dAh = nullptr, *dBh = nullptr, *dC = nullptr;
    int* dflag = nullptr;
    psdp_status s = PSDP_OK;
    cudaStream_t st;
    cudaStreamCreate(&st);
    auto al = [&](float** q, size_t n) { if (cudaMalloc((void**)q, n * 4) != cudaSuccess) s = PSDP_ENOMEM; };
    al(&dA, (size_t)M * kpad); al(&dB, (size_t)N * kpad); al(&dC, (size_t)M * N);
    al(&dAh, (size_t)M * kpad); al(&dAl, (size_t)M * kpad); al(&dBh, (size_t)N * kpad); al(&dBl, (size_t)N * kpad);
    if (cudaMalloc((void**)&dflag, 4) != cudaSuccess) s = PSDP_ENOMEM;
    if (s == PSDP_OK) {
        cudaMemset(dA, 0, (size_t)M * kpad * 4);
        cudaMemset(dB, 0, (size_t)N * kpad * 4);
        cudaMemset(dflag, 0, 4);
        cudaMemcpy2D(dA, (size_t)kpad * 4, A, (size_t)K * 4, (size_t)K * 4, M, cudaMemcpyHostToDevice);
        cudaMemcpy2D(dB, (size_t)kpad * 4, B, (size_t)K * 4, (size_t)K * 4, N, cudaMemcpyHostToDevice);
        cudaMemcpy(dC, C, (size_t)M * N * 4, cudaMemcpyHostToDevice);
        CUtensorMap mA, mB, mAl, mBl;
        bool ok;
        if (split == 3) {
            launch_split_tf32(st, (int64_t)M * kpad, dA, dAh, dAl);
            launch_split_tf32(st, (int64_t)N * kpad, dB, dBh, dBl);
            ok = tc_make_map(&mA, dAh, false, K, M, 1, kpad, 0, 128) && tc_make_map(&mB, dBh, false, K, N, 1, kpad, 0, 128) &&
                 tc_make_map(&mAl, dAl, false, K, M, 1, kpad, 0, 128) && tc_make_map(&mBl, dBl, false, K, N, 1, kpad, 0, 128);
        } else {
            ok = tc_make_map(&mA, dA, false, K, M, 1, kpad, 0, 128) && tc_make_map(&mB, dB, false, K, N, 1, kpad, 0, 128);
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
        if (ok && split == 3) launch_tc_gemm_persist(st, 3, mA, mB, &mAl, &mBl, M, N, K, dC, M, -1.f, 1.f, tri, ctas, dflag);
        if (ok && split == 1)
            launch_tc_gemm_persist(st, 1, mA, mB, nullptr, nullptr, M, N, K, dC, M, -1.f, 1.f, tri, ctas, dflag);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        if (ms) cudaEventElapsedTime(ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (!ok) s = PSDP_ECUDA;
        int flag = 0;
        if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) s = PSDP_ECUDA;
        cudaMemcpy(&flag, dflag, 4, cudaMemcpyDeviceToHost);
        if (flag) s = PSDP_ETIMEOUT;
        if (s == PSDP_OK) cudaMemcpy(C, dC, (size_t)M * N * 4, cudaMemcpyDeviceToHost);
    }
    for (float* q : {dA, dB, dAl, dBl, dAh, dBh, dC})
        if (q) cudaFree(q);
    if (dflag) cudaFree(dflag);
    cudaStreamDestroy(st);
    cudaGetLastError();
    return s;
}
