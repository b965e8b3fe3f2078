// FP64 matrix products on the BF16 tensor cores by the Ozaki scheme (Ozaki,
// Ogita, Oishi & Rump, "Error-free transformations of matrix multiplication by
// using fast routines of matrix multiplication and its applications", Numer.
// Algorithms 59, 2012): the operands are split into slices whose products the
// tensor cores form without rounding error, and the exact slice products are
// summed in integer and FP64 arithmetic.  GB300's FP64 rate (~1.1 TFLOP/s) is
// about 1/1700 of its BF16 rate, so the two large FP64 contractions of a Newton
// step (the Schur complement and the trailing updates of its Cholesky factor)
// run here at FP64 accuracy.
//
// Split.  Row i of an operand (depth Kd <= 384) is scaled by 2^-e_i, where
// e_i is the exponent with max_k |a_ik| < 2^e_i, and rounded to the integer
// X = round(a_ik 2^(56 - e_i)), |X| < 2^56.  X is written in balanced base-128
// digits, X = sum_{p=1..8} s_p 128^(8-p): s_2..s_8 in [-64, 63] and s_1 in
// [-128, 128].  Every digit is an integer of at most 8 significant bits, so it
// is exact in BF16, and a_ik = 2^e_i sum_p s_p 2^(-7p) up to 2^(e_i - 57).
//
// Product.  sum_k a_ik b_jk = 2^(e_i + f_j) sum_{t=2..9} 2^(-7t) T_t with the
// level sums T_t = sum_{p+q=t} sum_k s_p(a_ik) s_q(b_jk); the levels t > 9 are
// left out: their pairs have digits of at most 64 in magnitude, so per k they
// carry at most 2^12 (7 2^-70 + 6 2^-77 + ...) < 7.1 2^-58 of the scale.  Per k a level adds at
// most 2 * 2^13 + (t - 3) * 2^12 <= 10 * 2^12 in magnitude, so over Kd <= 384
// every partial sum is an integer of at most 15,728,640 < 2^24 in magnitude: the FP32 accumulation of the
// tensor cores is exact.  Each level has its own TMEM accumulator (8 levels x
// 64 columns fill the 512 columns of TMEM).
//
// Combination (epilogue).  Va = T_2 128^3 + T_3 128^2 + T_4 128 + T_5 and
// Vb = T_6 128^3 + T_7 128^2 + T_8 128 + T_9 in int64 (exact, below 2^47 in
// magnitude); D_ij = 2^(e_i + f_j - 63) (Va 2^28 + Vb), rounded once by an FMA
// of the exactly converted Va and Vb.  With the split's own rounding (2^(e-57)
// an entry, so 2^(e_i + f_j - 56) a product) and the levels left out, the error
// of D_ij is at most Kd 2.8 2^(e_i + f_j - 56) + 2^-53 |D_ij|
// <= Kd 2^-52.5 max|a_i| max|b_j| + 2^-53 |D_ij|, the accuracy of an FP64 GEMM.
//
// Kernel: persistent, one CTA per SM walking 128 x 64 tiles (128 TMEM lanes;
// 8 levels x 64 columns fill the 512 TMEM columns); per stage 32 of k for all
// 8 slices of both operands (64-byte swizzled rows, 96 KB), two stages.  Warp
// 0 lane 0 issues the TMA loads, warp 1 lane 0 the 36 slice-pair MMAs per
// 16-deep k step, and sixteen epilogue warps drain TMEM, release it to the
// next tile's MMAs and then update C.  Measured rates that set this shape
// (GB300, one issuing thread, operands in shared memory): an M = 128, K = 16
// BF16 MMA takes about 44.5 cycles at N = 32 or 48, 48 at N = 64, 56 at N = 96
// and 64 at N = 128 (the tensor-core rate), so 64 columns keep 67 % of the
// tensor rate while the eight accumulators still fit in TMEM; more issuing
// threads make it slower.  Waits are bounded as in the other tcgen05 kernels.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "psdp_internal.h"
#include "tc_ptx.cuh"

namespace {

constexpr int OZ_S = 8;                         // slices per operand
constexpr int OZ_BM = 128, OZ_BK = 32;
constexpr int OZ_ROW = OZ_BK * 2;               // bytes of one slice row in a stage (64-byte swizzle)
constexpr int OZ_TA = OZ_BM * OZ_ROW;           // 8 KB
constexpr int OZ_STAGES = 2;
constexpr int OZ_SPLIT_THREADS = 256;


// shared-memory matrix descriptor: K-major, SWIZZLE_64B (8-row groups of 64-byte rows, 512 B apart)
__device__ __forceinline__ uint64_t sdesc64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;      // stride byte offset
    d |= (uint64_t)1 << 46;               // descriptor version
    d |= (uint64_t)4 << 61;               // SWIZZLE_64B
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// 8 columns of 32 lanes from TMEM, without the wait (the caller waits once)
__device__ __forceinline__ void tmem_ld8_nw(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// Depth of batch b in the window [k_off, k_off + kOzakiMaxDepth) of its full depth.
__device__ __forceinline__ int oz_depth(const int32_t* kdv, int kd_uniform, int b, int k_off) {
    const int kd = (kdv ? kdv[b] : kd_uniform) - k_off;
    return kd < 0 ? 0 : (kd > kOzakiMaxDepth ? kOzakiMaxDepth : kd);
}

// Exact FP64 value of an integer below 2^53 in magnitude, assembled from its
// bits by integer operations (the conversion instruction issues on GB300's
// scarce FP64 pipe).
__device__ __forceinline__ double oz_i2d(long long x) {
    if (x == 0) return 0.0;
    const unsigned long long sgn = x < 0 ? (1ull << 63) : 0ull;
    const unsigned long long u = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
    const int msb = 63 - __clzll((long long)u);                      // <= 52
    const unsigned long long m = u << (52 - msb);
    return __longlong_as_double((long long)(sgn | ((unsigned long long)(msb + 1023) << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// round-to-nearest-even of x 2^s for |x 2^s| < 2^62 by integer operations on
// x's bits: the same integer as __double2ll_rn(ldexp(x, s)), whose conversion and
// scaling issue on GB300's scarce FP64 pipe
__device__ __forceinline__ long long oz_round_scaled(double x, int s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (ex) m |= 1ull << 52;
    const int sh = (ex ? ex : 1) - 1075 + s;      // |x| 2^s = m 2^sh
    unsigned long long q;
    if (sh >= 0) {
        q = m << sh;
    } else if (sh < -63) {
        q = 0;
    } else {
        const int r = -sh;
        q = m >> r;
        const unsigned long long rem = m & ((1ull << r) - 1), half = 1ull << (r - 1);
        if (rem > half || (rem == half && (q & 1))) ++q;
    }
    return (b >> 63) ? -(long long)q : (long long)q;
}

// BF16 bits of an integer d with |d| <= 256 (exact: at most 8 significant bits)
__device__ __forceinline__ uint16_t oz_bf16_of_int(int d) {
    if (d == 0) return 0;
    const unsigned a = (unsigned)(d < 0 ? -d : d);
    const int msb = 31 - __clz((int)a);
    const unsigned bits = ((unsigned)(msb + 127) << 7) | ((a << (7 - msb)) & 0x7Fu);
    return (uint16_t)(bits | (d < 0 ? 0x8000u : 0u));
}

// Slices of one batch of operands.  Element (r, k) of batch b is
// src[off_b + (k_off + k) * ld + r], off_b = src_off[b] if given, else
// b * src_batch (rows contiguous: a column-major block, or the stacked n x n
// operand matrices of the Schur contraction); depth window oz_depth <=
// kOzakiMaxDepth, padded with zeros to dpad.
// out[(b * 8 + p) * rows * dpad + r * dpad + k] = digit p of (r, k) as BF16;
// ex[b * rows + r] = e_r.  One CTA per 32 rows: the block is staged in shared
// memory through coalesced row-contiguous loads, then every thread writes
// digits along k (contiguous in the output).
__global__ void __launch_bounds__(OZ_SPLIT_THREADS)
k_ozaki_split(const double* __restrict__ src, int64_t ld, int64_t src_batch, const int32_t* __restrict__ src_off,
              int rows, const int32_t* __restrict__ kdv, int kd_uniform, int k_off, int dpad,
              __nv_bfloat16* __restrict__ out, int32_t* __restrict__ ex) {
    extern __shared__ double tile[];            // [kd][33]
    __shared__ int es[32];
    const int b = blockIdx.y;
    const int r0 = blockIdx.x * 32;
    const int kd = min(oz_depth(kdv, kd_uniform, b, k_off), dpad);   // the staging holds dpad columns
    src += (src_off ? (int64_t)src_off[b] : (int64_t)b * src_batch) + (int64_t)k_off * ld;
    out += (int64_t)b * OZ_S * rows * dpad;
    ex += (int64_t)b * rows;
    for (int idx = threadIdx.x; idx < 32 * kd; idx += OZ_SPLIT_THREADS) {
        const int k = idx >> 5, rr = idx & 31, r = r0 + rr;
        tile[k * 33 + rr] = (r < rows) ? src[(int64_t)k * ld + r] : 0.0;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int rr = warp; rr < 32; rr += OZ_SPLIT_THREADS / 32) {
        double m = 0.0;
        for (int k = lane; k < kd; k += 32) m = fmax(m, fabs(tile[k * 33 + rr]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) {
            int e = 0;
            if (m > 0.0) frexp(m, &e);
            es[rr] = e;
            if (r0 + rr < rows) ex[r0 + rr] = e;
        }
    }
    __syncthreads();
    const int64_t slice = (int64_t)rows * dpad;
    for (int idx = threadIdx.x; idx < 32 * dpad; idx += OZ_SPLIT_THREADS) {
        const int rr = idx / dpad, k = idx - rr * dpad, r = r0 + rr;
        if (r >= rows) continue;
        const double x = (k < kd) ? tile[k * 33 + rr] : 0.0;
        long long X = oz_round_scaled(x, 56 - es[rr]);
        int dig[OZ_S];
#pragma unroll
        for (int p = OZ_S - 1; p >= 1; --p) {
            const int d = (int)((X + 64) & 127) - 64;
            dig[p] = d;
            X = (X - d) >> 7;
        }
        dig[0] = (int)X;
        uint16_t* o = reinterpret_cast<uint16_t*>(out) + (int64_t)r * dpad + k;
#pragma unroll
        for (int p = 0; p < OZ_S; ++p) o[p * slice] = oz_bf16_of_int(dig[p]);
    }
}

// Tiles of one Ozaki product in the order every role of the persistent kernel
// walks them: batch by batch, column tile by column tile (nt), row tiles (mt)
// inside a column; with lower only the row tiles that reach the diagonal,
// mt >= nt * BN / 128.
template <int BN>
struct OzWalk {
    int MT, NT, batch, lower, b, nt, off;
    __device__ OzWalk(int M, int N, int batch_, int lower_, int start)
        : MT((M + OZ_BM - 1) / OZ_BM), NT((N + BN - 1) / BN), batch(batch_), lower(lower_), b(0), nt(0),
          off(start) { settle(); }
    __device__ int first(int c) const { return lower ? (c * BN) / OZ_BM : 0; }
    __device__ int len(int c) const { return MT - first(c); }
    __device__ void settle() {
        while (b < batch && off >= len(nt)) {
            off -= len(nt);
            if (++nt == NT) {
                nt = 0;
                ++b;
            }
        }
    }
    __device__ bool valid() const { return b < batch; }
    __device__ int mt() const { return first(nt) + off; }
    __device__ void advance(int step) {
        off += step;
        settle();
    }
};

// Shape of the persistent kernel: tiles of 128 x BN, EPI epilogue warps.  A
// tile's eight level accumulators take 8 BN of the 512 TMEM columns, so NBUF =
// 512 / (8 BN) tiles fit at once (BN = 32: the MMAs fill one buffer while the
// epilogue drains the other; measured slower than BN = 64 with one buffer, as
// the MMAs cost as much at N = 32 as at 64).  EPI = 16 drains a 128 x 64 tile
// in about 9.7k cycles against 13.8k with 8 warps.
template <int BN, int EPI>
struct OzCfg {
    static constexpr int NBUF = 512 / (8 * BN);
    static constexpr int THREADS = 64 + 32 * EPI;     // warp 0 TMA, warp 1 MMA and TMEM, then the epilogue
    static constexpr int CW = BN * 4 / EPI;           // columns of one epilogue warp
    static constexpr int TB = BN * OZ_ROW;            // one B slice of a stage
    static constexpr int STAGE = OZ_S * (OZ_TA + TB);
    static constexpr int NBAR = 2 * OZ_STAGES + 2 * NBUF + 1;
    static constexpr size_t SMEM = (size_t)OZ_STAGES * STAGE + 1024 + 8 * NBAR + 16;
    // instruction descriptor: F32 accumulate, BF16 A and B, both K-major, N = BN, M = 128
    static constexpr uint32_t IDESC =
        (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(OZ_BM >> 4) << 24);
    static_assert(NBUF >= 1 && 8 * BN * NBUF == 512 && CW % 8 == 0 && EPI % 4 == 0, "tile shape");
};

// C_b = alpha * D_b + beta * C_b with D_b[i][j] = sum_k A_b[i][k] B_b[j][k] from
// the slices of A_b (rows a_row0 + i, i < M, of slice arrays of a_rows rows) and
// B_b (rows b_row0 + j, j < N, of b_rows) over the depth window
// oz_depth(kd, kd_uniform, b, k_off); C_b[j * ldc + i] (column-major in i).
// lower: only elements with i >= j, tiles wholly above the diagonal are skipped.
//
// Persistent: one CTA per SM (or fewer) walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...  Warp 0 lane 0 issues the TMA loads of every
// stage (running up to two stages ahead, across tiles), warp 1 lane 0 the 36
// slice-pair MMAs per 16-deep k step into the tile's TMEM buffer, and the
// epilogue warps drain a tile's eight level accumulators into registers,
// combined to one FP64 value per element, release the buffer (barrier tfree)
// and then read, update and write C while the MMAs run on.  Epilogue warp w
// takes TMEM lanes 32 (w % 4) .. +31 and CW columns.  Barriers: full/empty per
// stage, accb per buffer (MMA -> epilogue, one phase per tile), tfree per buffer
// (epilogue -> MMA, EPI arrivals per tile).  Every wait is bounded; after a
// timeout the roles stop walking and the CTA unwinds with FL_TIMEOUT raised.
template <int BN, int EPI>
__global__ void __launch_bounds__(OzCfg<BN, EPI>::THREADS, 1)
k_ozaki_gemm_persist(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                     const int32_t* __restrict__ eA, const int32_t* __restrict__ eB, int a_rows, int a_row0,
                     int b_rows, int b_row0, int M, int N, int batch, const int32_t* __restrict__ kd, int kd_uniform,
                     int k_off, double* C, int64_t ldc, int64_t c_batch, double alpha, double beta, int lower,
                     int* flag) {
    using Cfg = OzCfg<BN, EPI>;
    using Walk = OzWalk<BN>;
    constexpr int NBUF = Cfg::NBUF, CW = Cfg::CW;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t base_raw = smem_u32(smem_raw);
    const uint32_t base = (base_raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - base_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + OZ_STAGES * Cfg::STAGE);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + Cfg::NBAR);
    __shared__ int abort_flag;
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * OZ_STAGES;
    const uint32_t accb0 = full0 + 16 * OZ_STAGES, tfree0 = accb0 + 8 * NBUF, drain = tfree0 + 8 * NBUF;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < OZ_STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int u = 0; u < NBUF; ++u) {
            mbar_init(accb0 + 8 * u, 1);
            mbar_init(tfree0 + 8 * u, EPI);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;

    if (warp == 0 && lane == 0) {
        // TMA producer: every slice of both operands for 32 of k per stage, tile after tile
        int g = 0;
        for (Walk t(M, N, batch, lower, blockIdx.x); t.valid() && !*(volatile int*)&abort_flag;
             t.advance(gridDim.x)) {
            const int nk = (oz_depth(kd, kd_uniform, t.b, k_off) + OZ_BK - 1) / OZ_BK;
            const int m0 = t.mt() * OZ_BM, n0 = t.nt * BN;
            for (int kt = 0; kt < nk; ++kt, ++g) {
                const int s = g % OZ_STAGES;
                if (g >= OZ_STAGES && !mbar_wait(empty0 + 8 * s, ((g / OZ_STAGES) - 1) & 1, flag)) {
                    abort_flag = 1;
                    break;
                }
                const uint32_t st = base + s * Cfg::STAGE;
                const uint32_t fb = full0 + 8 * s;
                mbar_expect_tx(fb, Cfg::STAGE);
#pragma unroll
                for (int p = 0; p < OZ_S; ++p)
                    tma_load_3d(st + p * OZ_TA, &mA, fb, kt * OZ_BK, a_row0 + m0, t.b * OZ_S + p);
#pragma unroll
                for (int q = 0; q < OZ_S; ++q)
                    tma_load_3d(st + OZ_S * OZ_TA + q * Cfg::TB, &mB, fb, kt * OZ_BK, b_row0 + n0, t.b * OZ_S + q);
            }
        }
        // every issued stage has landed before the CTA may exit
        for (int q = (g > OZ_STAGES ? g - OZ_STAGES : 0); q < g; ++q)
            mbar_wait(full0 + 8 * (q % OZ_STAGES), (q / OZ_STAGES) & 1, flag);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: tile i goes to buffer i % NBUF once tile i - NBUF has been drained from it
        int g = 0, i = 0;
        bool issued = false;
        for (Walk t(M, N, batch, lower, blockIdx.x); t.valid() && !*(volatile int*)&abort_flag;
             t.advance(gridDim.x), ++i) {
            const int u = i % NBUF;
            if (i >= NBUF && !mbar_wait(tfree0 + 8 * u, ((i / NBUF) - 1) & 1, flag)) {
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t tbuf = tmem + (uint32_t)(u * 8 * BN);
            const int nk = (oz_depth(kd, kd_uniform, t.b, k_off) + OZ_BK - 1) / OZ_BK;
            for (int kt = 0; kt < nk; ++kt, ++g) {
                const int s = g % OZ_STAGES;
                if (!mbar_wait(full0 + 8 * s, (g / OZ_STAGES) & 1, flag)) {
                    abort_flag = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t st = base + s * Cfg::STAGE;
#pragma unroll
                for (int kk = 0; kk < OZ_ROW / 32; ++kk) {
#pragma unroll
                    for (int p = 0; p < OZ_S; ++p) {
#pragma unroll
                        for (int q = 0; q < OZ_S - p; ++q) {
                            const uint32_t acc = (kt > 0 || kk > 0 || p > 0) ? 1u : 0u;
                            mma_bf16(tbuf + (uint32_t)(BN * (p + q)), sdesc64(st + p * OZ_TA + kk * 32),
                                     sdesc64(st + OZ_S * OZ_TA + q * Cfg::TB + kk * 32), Cfg::IDESC, acc);
                        }
                    }
                }
                issued = true;
                mma_commit(empty0 + 8 * s);
            }
            if (*(volatile int*)&abort_flag) break;
            mma_commit(accb0 + 8 * u);   // a tile of depth 0 commits too: its epilogue reads zeros
        }
        // all MMAs complete before TMEM is released
        if (issued) {
            mma_commit(drain);
            mbar_wait(drain, 0, flag);
        }
    } else if (warp >= 2) {
        const int quad = warp & 3, grp = (warp - 2) >> 2;
        const int amode = (alpha == 1.0) ? 0 : (alpha == -1.0 ? 1 : 2);
        const int bmode = (beta == 0.0) ? 0 : (beta == 1.0 ? 1 : 2);
        int i = 0;
        for (Walk t(M, N, batch, lower, blockIdx.x); t.valid(); t.advance(gridDim.x), ++i) {
            const int u = i % NBUF;
            const int Kd = oz_depth(kd, kd_uniform, t.b, k_off);
            const int m0 = t.mt() * OZ_BM, n0 = t.nt * BN;
            const int row = m0 + 32 * quad + lane;
            const int jc = n0 + CW * grp;
            // warp-uniform decision: the TMEM loads below are warp-collective
            const bool ok = __all_sync(0xffffffffu, mbar_wait(accb0 + 8 * u, (i / NBUF) & 1, flag));
            if (!ok) {
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // drain: the eight levels of CW columns, combined exactly to (Va 2^28 + Vb)
            // in FP64 (one rounding); the 2^(e_i + f_j - 63) scale is applied below
            const uint32_t tl0 = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(u * 8 * BN + CW * grp);
            double w[CW];
#pragma unroll
            for (int c0 = 0; c0 < CW; c0 += 8) {
                uint32_t r[OZ_S][8];
                if (Kd > 0) {
#pragma unroll
                    for (int tl = 0; tl < OZ_S; ++tl) tmem_ld8_nw(tl0 + (uint32_t)(BN * tl + c0), r[tl]);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                } else {
#pragma unroll
                    for (int tl = 0; tl < OZ_S; ++tl)
#pragma unroll
                        for (int j = 0; j < 8; ++j) r[tl][j] = 0u;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    long long T[OZ_S];
#pragma unroll
                    for (int tl = 0; tl < OZ_S; ++tl) T[tl] = (long long)__float2int_rn(__uint_as_float(r[tl][j]));
                    const long long Va = ((T[0] * 128 + T[1]) * 128 + T[2]) * 128 + T[3];
                    const long long Vb = ((T[4] * 128 + T[5]) * 128 + T[6]) * 128 + T[7];
                    w[c0 + j] = fma(oz_i2d(Va), 268435456.0, oz_i2d(Vb));
                }
            }
            // the buffer is free for tile i + NBUF's MMAs
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(tfree0 + 8 * u);
            // C update under the next tiles' MMAs
            if (row < M) {
                const int ei = eA[(int64_t)t.b * a_rows + a_row0 + row];
                const int32_t* eBb = eB + (int64_t)t.b * b_rows + b_row0;
                double* Cb = C + (int64_t)t.b * c_batch;
#pragma unroll
                for (int c0 = 0; c0 < CW; c0 += 8) {
                    double cold[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int col = jc + c0 + j;
                        cold[j] =
                            (bmode != 0 && col < N && !(lower && row < col)) ? Cb[(int64_t)col * ldc + row] : 0.0;
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int col = jc + c0 + j;
                        if (col >= N || (lower && row < col)) continue;
                        double v = w[c0 + j];
                        const int E = ei + eBb[col] - 63;
                        if (v != 0.0) {
                            const long long bits = __double_as_longlong(v);
                            const int be = (int)((bits >> 52) & 0x7FF) + E;
                            v = (be <= 0 || be >= 2047) ? ldexp(v, E)
                                                        : __longlong_as_double(bits + ((long long)E << 52));
                        }
                        if (amode) v = (amode == 1) ? -v : alpha * v;
                        Cb[(int64_t)col * ldc + row] =
                            (bmode == 0) ? v : (bmode == 1 ? cold[j] + v : fma(beta, cold[j], v));
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

}  // namespace

void init_attrs_ozaki(int smem_optin) {
    set_max_dynamic_smem((const void*)k_ozaki_gemm_persist<64, 16>, smem_optin);
    set_max_dynamic_smem((const void*)k_ozaki_split, smem_optin);
}

size_t ozaki_slice_elems(int rows, int dpad, int batch) { return (size_t)batch * OZ_S * rows * dpad; }

void launch_ozaki_split(cudaStream_t st, const double* src, int64_t ld, int64_t src_batch, const int32_t* src_off,
                        int rows, const int32_t* kdv, int kd_uniform, int k_off, int dpad, int batch, uint16_t* out_bits,
                        int32_t* ex) {
    __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(out_bits);
    if (rows <= 0 || batch <= 0 || dpad <= 0 || dpad > kOzakiMaxDepth) return;
    dim3 grid((rows + 31) / 32, batch);
    // staging for the launch's own depth (at most dpad columns), not the largest window
    k_ozaki_split<<<grid, OZ_SPLIT_THREADS, (size_t)dpad * 33 * sizeof(double), st>>>(src, ld, src_batch, src_off, rows, kdv,
                                                                         kd_uniform, k_off, dpad, out, ex);
}

// Persistent grid: one CTA per SM (ctas <= 0) or ctas, and at most one per tile.
int persist_grid(int M, int N, int batch, int lower, int bn, int ctas) {
    const int64_t MT = (M + OZ_BM - 1) / OZ_BM, NT = (N + bn - 1) / bn;
    int64_t tiles = 0;
    for (int64_t c = 0; c < NT; ++c) tiles += lower ? MT - (c * bn) / OZ_BM : MT;
    tiles *= batch;
    if (tiles <= 0) return 0;
    if (ctas <= 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        ctas = sms > 0 ? sms : 1;
    }
    return (int)std::min<int64_t>(tiles, ctas);
}

template <int BN, int EPI>
bool launch_persist(cudaStream_t st, const uint16_t* As, int a_rows, int a_row0, const int32_t* eA,
                    const uint16_t* Bs, int b_rows, int b_row0, const int32_t* eB, int M, int N, int dpad, int batch,
                    const int32_t* kd, int kd_uniform, int k_off, double* C, int64_t ldc, int64_t c_batch,
                    double alpha, double beta, int lower, int* flag, int ctas) {
    using Cfg = OzCfg<BN, EPI>;
    CUtensorMap mA, mB;
    if (!tc_make_map_swz(&mA, As, true, dpad, a_rows, (int64_t)batch * OZ_S, dpad, (int64_t)a_rows * dpad, OZ_BK,
                         OZ_BM, 64) ||
        !tc_make_map_swz(&mB, Bs, true, dpad, b_rows, (int64_t)batch * OZ_S, dpad, (int64_t)b_rows * dpad, OZ_BK,
                         BN, 64))
        return false;
    const int grid = persist_grid(M, N, batch, lower, BN, ctas);
    if (grid <= 0) return true;
    k_ozaki_gemm_persist<BN, EPI><<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(mA, mB, eA, eB, a_rows, a_row0, b_rows,
                                                                         b_row0, M, N, batch, kd, kd_uniform, k_off,
                                                                         C, ldc, c_batch, alpha, beta, lower, flag);
    return true;
}

bool launch_ozaki_gemm(cudaStream_t st, const uint16_t* As, int a_rows, int a_row0, const int32_t* eA,
                       const uint16_t* Bs, int b_rows, int b_row0, const int32_t* eB, int M, int N, int dpad,
                       int batch, const int32_t* kd, int kd_uniform, int k_off, double* C, int64_t ldc,
                       int64_t c_batch, double alpha, double beta, int lower, int* flag, int ctas) {
    if (M <= 0 || N <= 0 || batch <= 0) return true;
    if (dpad % OZ_BK != 0 || dpad > kOzakiMaxDepth || a_row0 + M > a_rows || b_row0 + N > b_rows || a_row0 < 0 ||
        b_row0 < 0)
        return false;
    return launch_persist<64, 16>(st, As, a_rows, a_row0, eA, Bs, b_rows, b_row0, eB, M, N, dpad, batch, kd,
                                  kd_uniform, k_off, C, ldc, c_batch, alpha, beta, lower, flag, ctas);
}

// Self-test on host data: C (N x M column-major, C[j*M + i]) = alpha A B^T + beta C
// with A: M x K, B: N x K row-major FP64, K <= kOzakiMaxDepth.
extern "C" psdp_status psdp_ozaki_gemm_check(int M, int N, int K, const double* A, const double* B, double* C,
                                             double alpha, double beta, int lower) {
    if (M < 1 || N < 1 || K < 1 || K > 8 * kOzakiMaxDepth || !A || !B || !C) return PSDP_EINVAL;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PSDP_ECUDA;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    init_attrs_ozaki(optin);
    const int dpad = (std::min(K, kOzakiMaxDepth) + OZ_BK - 1) / OZ_BK * OZ_BK;
    // the split reads (row, k) at k * rows + row: transpose on the host
    std::vector<double> At((size_t)K * M), Bt((size_t)K * N);
    for (int i = 0; i < M; ++i)
        for (int k = 0; k < K; ++k) At[(size_t)k * M + i] = A[(size_t)i * K + k];
    for (int j = 0; j < N; ++j)
        for (int k = 0; k < K; ++k) Bt[(size_t)k * N + j] = B[(size_t)j * K + k];
    double *dA = nullptr, *dB = nullptr, *dC = nullptr;
    uint16_t *sA = nullptr, *sB = nullptr;
    int32_t *eA = nullptr, *eB = nullptr;
    int* dflag = nullptr;
    psdp_status s = PSDP_OK;
    auto al = [&](void** p, size_t bytes) { if (cudaMalloc(p, bytes) != cudaSuccess) s = PSDP_ENOMEM; };
    al((void**)&dA, At.size() * 8);
    al((void**)&dB, Bt.size() * 8);
    al((void**)&dC, (size_t)M * N * 8);
    al((void**)&sA, ozaki_slice_elems(M, dpad, 1) * 2);
    al((void**)&sB, ozaki_slice_elems(N, dpad, 1) * 2);
    al((void**)&eA, (size_t)M * 4);
    al((void**)&eB, (size_t)N * 4);
    al((void**)&dflag, 4);
    if (s == PSDP_OK) {
        cudaMemcpy(dA, At.data(), At.size() * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(dB, Bt.data(), Bt.size() * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(dC, C, (size_t)M * N * 8, cudaMemcpyHostToDevice);
        cudaMemset(dflag, 0, 4);
        // depth windows of kOzakiMaxDepth: each window's product is exact, the windows are summed in FP64
        for (int k0 = 0; k0 < K && s == PSDP_OK; k0 += kOzakiMaxDepth) {
            launch_ozaki_split(0, dA, M, 0, nullptr, M, nullptr, K, k0, dpad, 1, sA, eA);
            launch_ozaki_split(0, dB, N, 0, nullptr, N, nullptr, K, k0, dpad, 1, sB, eB);
            if (!launch_ozaki_gemm(0, sA, M, 0, eA, sB, N, 0, eB, M, N, dpad, 1, nullptr, K, k0, dC, M, 0, alpha,
                                   k0 == 0 ? beta : 1.0, lower, dflag))
                s = PSDP_ECUDA;
        }
        int hflag = 0;
        if (cudaDeviceSynchronize() != cudaSuccess) s = PSDP_ECUDA;
        cudaMemcpy(&hflag, dflag, 4, cudaMemcpyDeviceToHost);
        if (s == PSDP_OK && hflag) s = PSDP_ETIMEOUT;
        if (s == PSDP_OK) cudaMemcpy(C, dC, (size_t)M * N * 8, cudaMemcpyDeviceToHost);
    }
    cudaFree(dA); cudaFree(dB); cudaFree(dC); cudaFree(sA); cudaFree(sB); cudaFree(eA); cudaFree(eB); cudaFree(dflag);
    if (cudaGetLastError() != cudaSuccess && s == PSDP_OK) s = PSDP_ECUDA;
    return s;
}
