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

#include <cstring>

#include "psdp_internal.h"

namespace {

constexpr int BM = 128, BN = 128;
constexpr int ROW_BYTES = 128;                    // one swizzle row = BK elements
constexpr int TILE_A = BM * ROW_BYTES;            // 16 KB
constexpr int TILE_B = BN * ROW_BYTES;            // 16 KB
constexpr uint64_t kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// bounded wait on the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* flag) {
    const uint64_t t0 = gtimer();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (gtimer() - t0 > kWaitNs) {
            atomicOr(flag, (int)FL_TIMEOUT);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
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
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
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
          float beta, int tri, int* flag) {
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
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    if (n < N) Cb[(int64_t)n * ldc + m] = alpha * __uint_as_float(r[j]) + beta * old[c0 + j];
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

// D = A B^T over a batch; see the file header.  Returns false if a tensor map
// could not be encoded (nothing is launched then).
bool launch_tc_gemm(cudaStream_t st, bool bf16, int split, const CUtensorMap& A, const CUtensorMap& B,
                    const CUtensorMap* Alo, const CUtensorMap* Blo, int M, int N, int batch, int b0,
                    const int32_t* kd, int kd_uniform, float* C, int64_t ldc, int64_t c_batch, float alpha,
                    float beta, int tri, int* flag) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
    if (grid.x == 0 || grid.y == 0 || batch <= 0) return true;
    if (bf16) {
        k_tc_gemm<true, 1, 4><<<grid, 128, smem_bytes<true, 1, 4>(), st>>>(A, B, A, B, M, N, b0, kd, kd_uniform, C,
                                                                         ldc, c_batch, alpha, beta, tri, flag);
    } else if (split == 3) {
        k_tc_gemm<false, 3, 3><<<grid, 128, smem_bytes<false, 3, 3>(), st>>>(A, B, *Alo, *Blo, M, N, b0, kd,
                                                                           kd_uniform, C, ldc, c_batch, alpha, beta,
                                                                           tri, flag);
    } else {
        k_tc_gemm<false, 1, 4><<<grid, 128, smem_bytes<false, 1, 4>(), st>>>(A, B, A, B, M, N, b0, kd, kd_uniform, C,
                                                                           ldc, c_batch, alpha, beta, tri, flag);
    }
    return true;
}

void init_attrs_tc(int smem_optin) {
    set_max_dynamic_smem((const void*)k_tc_gemm<true, 1, 4>, smem_optin);
    set_max_dynamic_smem((const void*)k_tc_gemm<false, 3, 3>, smem_optin);
    set_max_dynamic_smem((const void*)k_tc_gemm<false, 1, 4>, smem_optin);
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
