// Blocked triangular sweeps with the dense Cholesky factor of the Schur
// complement (Sec. IV-A, the two solves of every Newton step; with the FP32
// factor, the preconditioner of the mixed-precision path), one launch per sweep.
//
// Factor layout (both precisions): Omega is K x K row-major and the factor is
// kept in its upper triangle, A[j*K + i] = L(i, j) for i >= j, with the inverse
// of every W x W diagonal block in Linv[p][k*W + r] = Linv_p(r, k).
//
// One CTA per block row.  A CTA takes a ticket from an atomic counter and
// solves block row `ticket` (forward) or `npanel-1-ticket` (backward), so it
// only waits for CTAs that took earlier tickets, i.e. CTAs that are already
// running: the sweep cannot deadlock whatever the residency.  While it waits it
// applies every block that is already solved; each thread's running sum runs
// over a fixed index sequence however the solved blocks arrive, so the result
// is bit-reproducible.  A finished block is published with a release store of
// its ready flag; readers acquire the flag and read the solved values through
// L2.  Warp 0 polls, the CTA synchronises once per batch of newly solved
// blocks, and the tile of the last predecessor is loaded into registers before
// the wait, so the critical path per block is the flag latency, one W x W tile
// product from registers and the diagonal-block product.  Every wait is
// bounded (2 s without progress): the CTA sets FL_TIMEOUT and finishes with
// what it has, so its dependants finish too.
//
// sync: [0] forward ticket, [1] backward ticket, [2, 2+npanel) forward ready
// flags, [2+npanel, 2+2*npanel) backward ready flags; zeroed before each solve.
#include "psdp_internal.h"

namespace {

constexpr int TT = 256;
constexpr long long kWaitNs = 2000000000LL;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ long long gtimer() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

// V contiguous elements from a 16-byte aligned address (V = 1: one element)
template <typename T, int V>
__device__ __forceinline__ void load_vec(const T* p, T* o) {
    if constexpr (V == 1) {
        o[0] = *p;
    } else if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else {
        const double2 v = *reinterpret_cast<const double2*>(p);
        o[0] = v.x; o[1] = v.y;
    }
}

template <typename T, int V>
__device__ __forceinline__ void load_vec_cg(const T* p, T* o) {
    if constexpr (V == 1) {
        o[0] = __ldcg(p);
    } else if constexpr (sizeof(T) == 4) {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else {
        const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
        o[0] = v.x; o[1] = v.y;
    }
}

// values of the last predecessor's tile a thread keeps in registers
template <typename T>
constexpr int kPreVals = sizeof(T) == 4 ? 64 : 16;

// the backward sweep keeps the inverse transposed with padded rows, W (W + 1)
template <typename T>
size_t trsv_smem(int W) { return ((size_t)W * (W + 1) + (size_t)(TT / W) * W + W) * sizeof(T); }

// Pairwise sum of v[0], v[stride], ..., v[(G-1) stride] in a fixed order (G a power of two).
template <typename T, int G>
__device__ __forceinline__ T tree_sum(const T* v, int stride) {
    T b[G];
#pragma unroll
    for (int g = 0; g < G; ++g) b[g] = v[g * stride];
#pragma unroll
    for (int h = G / 2; h >= 1; h >>= 1)
#pragma unroll
        for (int i = 0; i < h; ++i) b[i] += b[i + h];
    return b[0];
}

// Warp 0 polls the ready flags; returns (to every thread) the first unsolved
// block at or after qd in [qd, p) (p if all are solved) once it is past qd, or
// -1 after 2 s without progress (FL_TIMEOUT raised).  slot alternates between
// calls so a slow warp still reading the previous answer is never overwritten.
__device__ __forceinline__ int wait_prefix(const unsigned* ready, int qd, int p, int* flag, int* s_q, int slot) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        long long t0 = 0;
        int qe;
        for (;;) {
            int first = p;
            for (int q = qd + lane; q < p; q += 32)
                if (ld_acquire(ready + q) == 0u) {
                    first = q;
                    break;
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
            if (first > qd) {
                qe = first;
                break;
            }
            int give_up = 0;
            if (lane == 0) {
                const long long now = gtimer();
                if (t0 == 0) t0 = now;
                if (now - t0 > kWaitNs) {
                    atomicOr(flag, (int)FL_TIMEOUT);
                    give_up = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, give_up, 0)) {
                qe = -1;
                break;
            }
            __nanosleep(64);
        }
        if (lane == 0) s_q[slot] = qe;
    }
    __syncthreads();
    return s_q[slot];
}

// Mirror image for the backward sweep: blocks (p, npanel) are solved from the
// top down; returns qe < qd such that blocks [qe, qd) are solved and qe-1 is p
// or unsolved, or -1 on timeout.
__device__ __forceinline__ int wait_suffix(const unsigned* ready, int qd, int p, int* flag, int* s_q, int slot) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        long long t0 = 0;
        int qe;
        for (;;) {
            int last = p;
            for (int q = qd - 1 - lane; q > p; q -= 32)
                if (ld_acquire(ready + q) == 0u) {
                    last = q;
                    break;
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
            if (last + 1 < qd) {
                qe = last + 1;
                break;
            }
            int give_up = 0;
            if (lane == 0) {
                const long long now = gtimer();
                if (t0 == 0) t0 = now;
                if (now - t0 > kWaitNs) {
                    atomicOr(flag, (int)FL_TIMEOUT);
                    give_up = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, give_up, 0)) {
                qe = -1;
                break;
            }
            __nanosleep(64);
        }
        if (lane == 0) s_q[slot] = qe;
    }
    __syncthreads();
    return s_q[slot];
}

// Forward sweep L z = b.  Block row p: z_p = Linv_p (b_p - sum_{q<p} L_pq z_q),
// L_pq(r, k) = A[(qW + k) K + pW + r].  b from bin (FP64) when given, else x.
// Off-diagonal part: thread (c, g) owns columns [cV, cV+V) of the block row and
// the rows j = qW + g + G t of every solved block q, U rows in flight.  The
// tile of block p-1, the last to be solved, is loaded before the first wait.
template <typename T, int W, int V>
__global__ void __launch_bounds__(TT, sizeof(T) == 4 ? 2 : 1)
k_trsv_fwd(const T* __restrict__ A, int K, const T* __restrict__ Linv, const double* __restrict__ bin, T* x,
           unsigned* sync, int* flag, const int* skip) {
    if (skip && *skip) return;
    // U independent running sums per column: FP32 keeps 8 for loads in flight;
    // FP64 keeps 2, because folding them costs FP64 adds on GB300's narrow pipe
    constexpr int UMAX = (sizeof(T) == 8) ? 2 : 8;
    constexpr int R = W / V, G = TT / R, RPB = W / G, U = RPB < UMAX ? RPB : UMAX;
    constexpr int G2 = TT / W;
    static_assert(TT % R == 0 && W % G == 0 && RPB % U == 0, "thread layout");
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Ls = reinterpret_cast<T*>(smraw);   // [W][W]  Ls[k*W + r] = Linv_p(r, k)
    T* red = Ls + W * W;                   // [G2][W]
    T* acc = red + G2 * W;                 // [W]
    __shared__ int s_ticket, s_q[2];
    __shared__ T s_off[G][W];
    unsigned* ready = sync + 2;
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(&sync[0], 1u);
    __syncthreads();
    const int p = s_ticket, j0 = p * W, w = min(W, K - j0);
    const T* Lp = Linv + (size_t)p * W * W;
#pragma unroll 8
    for (int i = threadIdx.x; i < W * W; i += TT) Ls[i] = Lp[i];
    // this block's right-hand side, read before any wait
    const T bown = (threadIdx.x < w) ? (T)(bin ? bin[j0 + threadIdx.x] : (double)ldcg(x + j0 + threadIdx.x)) : T(0);
    const int c = (threadIdx.x % R) * V, g = threadIdx.x / R;
    // the last predecessor's tile is held in registers before the wait: 16 values
    // a thread for FP64, 64 for the FP32 preconditioner's 128-row blocks (at
    // most 128 registers, so two CTAs still fit an SM)
    constexpr bool PRE = RPB * V <= kPreVals<T>;
    T last[PRE ? RPB : 1][V];
    if (PRE && p > 0 && c < w) {
#pragma unroll
        for (int t = 0; t < (PRE ? RPB : 1); ++t)
            load_vec<T, V>(A + (int64_t)((p - 1) * W + g + G * t) * K + j0 + c, last[t]);
    }
    T part[U][V];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < V; ++v) part[u][v] = T(0);
    int qd = 0, it = 0;         // blocks [0, qd) applied
    while (qd < p) {
        const int qe = wait_prefix(ready, qd, p, flag, s_q, it++ & 1);
        if (qe < 0) break;
        if (c < w) {
            for (int q = qd; q < qe; ++q) {
                const int jb = q * W + g;
                if (PRE && q == p - 1) {
#pragma unroll
                    for (int ta = 0; ta < RPB; ta += U) {
                        T xv[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) xv[u] = ldcg(x + jb + G * (ta + u));
#pragma unroll
                        for (int u = 0; u < U; ++u)
#pragma unroll
                            for (int v = 0; v < V; ++v)
                                part[u][v] = fma(last[PRE ? ta + u : 0][v], xv[u], part[u][v]);
                    }
                } else {
#pragma unroll
                    for (int ta = 0; ta < RPB; ta += U) {
                        T a[U][V], xv[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int j = jb + G * (ta + u);
                            load_vec<T, V>(A + (int64_t)j * K + j0 + c, a[u]);
                            xv[u] = ldcg(x + j);
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u)
#pragma unroll
                            for (int v = 0; v < V; ++v) part[u][v] = fma(a[u][v], xv[u], part[u][v]);
                    }
                }
            }
        }
        qd = qe;
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        T pu[U];
#pragma unroll
        for (int u = 0; u < U; ++u) pu[u] = part[u][v];
        s_off[g][c + v] = tree_sum<T, U>(pu, 1);
    }
    __syncthreads();
    if (threadIdx.x < W) {
        const int rr = threadIdx.x;
        const T sum = tree_sum<T, G>(&s_off[0][rr], W);
        acc[rr] = (rr < w) ? bown - sum : T(0);
    }
    __syncthreads();
    // z_p[r] = sum_{k <= r} Linv_p(r, k) acc[k], k = g2 (mod G2)
    const int r = threadIdx.x % W, g2 = threadIdx.x / W;
    T sum = T(0);
    if (r < w)
        for (int k = g2; k <= r; k += G2) sum = fma(Ls[k * W + r], acc[k], sum);
    red[g2 * W + r] = sum;
    __syncthreads();
    if (threadIdx.x < w) x[j0 + threadIdx.x] = tree_sum<T, G2>(red + threadIdx.x, W);
    __syncthreads();
    if (threadIdx.x == 0) st_release(ready + p, 1u);   // cumulative over the block's stores ordered by bar.sync
}

// Backward sweep L^T x = z.  Block row p: x_p = Linv_p^T (z_p - sum_{q>p} L_qp^T x_q),
// (L_qp^T x_q)[k] = sum_{i in block q} A[(pW + k) K + i] x_i.  x holds z on entry;
// the FP64 copy of the result also goes to xout when given.  Off-diagonal part:
// R threads share a row (V columns each, W / (R V) segments per block), thread
// row group g owns rows k = g + G t.  The tile of block p+1, the last to be
// solved, is loaded before the first wait.
template <typename T, int W, int V>
__global__ void __launch_bounds__(TT, sizeof(T) == 4 ? 2 : 1)
k_trsv_bwd(const T* __restrict__ A, int K, const T* __restrict__ Linv, T* x, double* xout, unsigned* sync, int* flag,
           const int* skip) {
    if (skip && *skip) return;
    // eight lanes share a row (fewer cross-lane adds: three shuffle levels), each
    // lane covering SEG segments of V columns per block
    constexpr int R = (W / V < 8) ? W / V : 8, G = TT / R, RPB = W / G, SEG = W / (R * V);
    constexpr int G2 = TT / W;
    static_assert(32 % R == 0 && W % G == 0 && W % (R * V) == 0, "thread layout");
    extern __shared__ __align__(16) unsigned char smraw[];
    // LsT[r (W + 1) + k] = Linv_p(r, k): the diagonal-block product runs threads
    // over k, so the row-major copy with a padded row keeps both this fill and
    // that product free of bank conflicts (the column-major copy put every
    // thread of a warp in one bank)
    T* LsT = reinterpret_cast<T*>(smraw);
    T* red = LsT + W * (W + 1);
    T* acc = red + G2 * W;
    __shared__ int s_ticket, s_q[2];
    const int npanel = (K + W - 1) / W;
    unsigned* ready = sync + 2 + npanel;
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(&sync[1], 1u);
    __syncthreads();
    const int p = npanel - 1 - s_ticket, j0 = p * W, w = min(W, K - j0);
    const T* Lp = Linv + (size_t)p * W * W;
#pragma unroll 8
    for (int i = threadIdx.x; i < W * W; i += TT) LsT[(i % W) * (W + 1) + i / W] = Lp[i];
    if (threadIdx.x < W) acc[threadIdx.x] = (threadIdx.x < w) ? ldcg(x + j0 + threadIdx.x) : T(0);   // z_p
    const int cl = (threadIdx.x % R) * V, g = threadIdx.x / R;
    constexpr bool PRE = SEG * RPB * V <= kPreVals<T>;   // as in the forward sweep
    T last[PRE ? SEG : 1][PRE ? RPB : 1][V];
    if (PRE && p + 1 < npanel) {
#pragma unroll
        for (int sg = 0; sg < (PRE ? SEG : 1); ++sg) {
            const int i = (p + 1) * W + sg * R * V + cl;
#pragma unroll
            for (int t = 0; t < (PRE ? RPB : 1); ++t) {
                const int k = g + G * t;
                if (i < K && k < w) load_vec<T, V>(A + (int64_t)(j0 + k) * K + i, last[sg][t]);
            }
        }
    }
    T part[RPB];
#pragma unroll
    for (int t = 0; t < RPB; ++t) part[t] = T(0);
    __syncthreads();            // z_p in acc before any thread may read it
    int qd = npanel, it = 0;    // blocks [qd, npanel) applied
    while (qd > p + 1) {
        const int qe = wait_suffix(ready, qd, p, flag, s_q, it++ & 1);
        if (qe < 0) break;
        // blocks in descending order, segments ascending inside a block
        for (int q = qd - 1; q >= qe; --q) {
#pragma unroll
            for (int sg = 0; sg < SEG; ++sg) {
                const int i = q * W + sg * R * V + cl;
                if (i < K) {           // K is a multiple of V: the whole vector is inside
                    T xv[V];
                    load_vec_cg<T, V>(x + i, xv);
#pragma unroll
                    for (int t = 0; t < RPB; ++t) {
                        const int k = g + G * t;
                        if (k < w) {
                            T a[V];
                            if (PRE && q == p + 1) {
#pragma unroll
                                for (int v = 0; v < V; ++v) a[v] = last[PRE ? sg : 0][PRE ? t : 0][v];
                            } else {
                                load_vec<T, V>(A + (int64_t)(j0 + k) * K + i, a);
                            }
#pragma unroll
                            for (int v = 0; v < V; ++v) part[t] = fma(a[v], xv[v], part[t]);
                        }
                    }
                }
            }
        }
        qd = qe;
    }
#pragma unroll
    for (int t = 0; t < RPB; ++t) {
        T v = part[t];
#pragma unroll
        for (int o = R / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int k = g + G * t;
        if ((threadIdx.x % R) == 0) acc[k] = (k < w) ? acc[k] - v : T(0);
    }
    __syncthreads();
    // x_p[k] = sum_{r >= k} Linv_p(r, k) acc[r], r = g2 (mod G2)
    const int k = threadIdx.x % W, g2 = threadIdx.x / W;
    T s = T(0);
    if (k < w)
        for (int rr = g2; rr < w; rr += G2)
            if (rr >= k) s = fma(LsT[rr * (W + 1) + k], acc[rr], s);
    red[g2 * W + k] = s;
    __syncthreads();
    if (threadIdx.x < w) {
        const T z = tree_sum<T, G2>(red + threadIdx.x, W);
        x[j0 + threadIdx.x] = z;
        if (xout) xout[j0 + threadIdx.x] = (double)z;
    }
    __syncthreads();
    if (threadIdx.x == 0) st_release(ready + p, 1u);   // cumulative over the block's stores ordered by bar.sync
}

template <typename T, int W>
void set_attrs(int smem_max) {
    const size_t need = trsv_smem<T>(W);
    if ((int)need > 40 * 1024 && (int)need + 16 * 1024 <= smem_max) {
        cudaFuncSetAttribute(k_trsv_fwd<T, W, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
        cudaFuncSetAttribute(k_trsv_bwd<T, W, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
        constexpr int V = 16 / sizeof(T);
        cudaFuncSetAttribute(k_trsv_fwd<T, W, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
        cudaFuncSetAttribute(k_trsv_bwd<T, W, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    }
}

// Both sweeps; 16-byte loads when every row of A starts on a 16-byte boundary.
template <typename T, int W>
void sweeps(cudaStream_t st, const T* A, int K, const T* Linv, const double* bin, T* x, double* xout,
            unsigned* sync, int* flag, const int* skip) {
    constexpr int V = 16 / sizeof(T);
    const int npanel = (K + W - 1) / W;
    const size_t sm = trsv_smem<T>(W);
    cudaMemsetAsync(sync, 0, (size_t)(2 + 2 * npanel) * sizeof(unsigned), st);
    const bool vec = (K % V == 0) && ((uintptr_t)A % 16 == 0) && ((uintptr_t)x % 16 == 0);
    if (vec) {
        k_trsv_fwd<T, W, V><<<npanel, TT, sm, st>>>(A, K, Linv, bin, x, sync, flag, skip);
        k_trsv_bwd<T, W, V><<<npanel, TT, sm, st>>>(A, K, Linv, x, xout, sync, flag, skip);
    } else {
        k_trsv_fwd<T, W, 1><<<npanel, TT, sm, st>>>(A, K, Linv, bin, x, sync, flag, skip);
        k_trsv_bwd<T, W, 1><<<npanel, TT, sm, st>>>(A, K, Linv, x, xout, sync, flag, skip);
    }
}

// 64 x 64 diagonal-block inverses from pairs of 32 x 32 ones, so the FP64
// sweeps take half as many dependent steps:
//   [X_a 0; -X_b L_ba X_a  X_b]  with L_ba(i, k) = L(j0b + i, j0a + k) = A[(j0a + k) K + j0b + i].
// One CTA per pair; T = L_ba X_a, then the lower-left block -X_b T.
__global__ void __launch_bounds__(256)
k_pair_inverse(const double* __restrict__ A, int K, const double* __restrict__ Linv32, double* Linv64) {
    __shared__ double Xa[32][33], Xb[32][33], Lba[32][33], T[32][33];
    const int t = blockIdx.x, tid = threadIdx.x;
    const int np32 = (K + 31) / 32;
    const int a = 2 * t, b = 2 * t + 1;
    const int j0a = 32 * a, j0b = 32 * b;
    const int wb = (b < np32) ? min(32, K - j0b) : 0;
    const double* Xa_g = Linv32 + (size_t)a * 1024;
    const double* Xb_g = Linv32 + (size_t)b * 1024;
#pragma unroll
    for (int idx = tid; idx < 1024; idx += 256) {
        const int c = idx >> 5, r = idx & 31;              // column-major element (r, c)
        Xa[r][c] = Xa_g[idx];
        Xb[r][c] = (wb > 0) ? Xb_g[idx] : 0.0;
        Lba[r][c] = (r < wb) ? A[(int64_t)(j0a + c) * K + j0b + r] : 0.0;
    }
    __syncthreads();
    // thread (r, c4): four outputs of a row, k in order
    const int r = tid >> 3, c4 = (tid & 7) * 4;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < 32; ++k) {
        const double l = Lba[r][k];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fma(l, Xa[k][c4 + u], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) T[r][c4 + u] = acc[u];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = 0.0;
    for (int k = 0; k < 32; ++k) {
        const double xb = Xb[r][k];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fma(xb, T[k][c4 + u], acc[u]);
    }
    double* X = Linv64 + (size_t)t * 4096;                 // X(r, c) at c*64 + r
    for (int idx = tid; idx < 1024; idx += 256) {
        const int c = idx >> 5, rr = idx & 31;
        X[c * 64 + rr] = Xa[rr][c];                         // upper-left
        X[(32 + c) * 64 + rr] = 0.0;                        // upper-right
        X[(32 + c) * 64 + 32 + rr] = Xb[rr][c];             // lower-right
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) X[(c4 + u) * 64 + 32 + r] = -acc[u];   // lower-left
}

}  // namespace

size_t trsv_sync_words(int K, int nb) { return (size_t)2 + 2 * (size_t)((K + nb - 1) / nb); }

void init_attrs_trsv(int smem_max) {
    set_attrs<double, 32>(smem_max);
    set_attrs<double, 64>(smem_max);
    set_attrs<float, 64>(smem_max);
    set_attrs<float, 128>(smem_max);
}

// 64 x 64 diagonal-block inverses (Linv64: [ceil(K/64)][64][64]) from the
// 32 x 32 ones of the FP64 factor.
void launch_pair_inverse(cudaStream_t st, const double* A, int K, const double* Linv32, double* Linv64) {
    k_pair_inverse<<<(K + 63) / 64, 256, 0, st>>>(A, K, Linv32, Linv64);
}

// x <- Omega^{-1} x with the FP64 factor; Linv holds nb x nb diagonal-block
// inverses (nb = 32, or 64 from launch_pair_inverse).
bool launch_solve_fp64(cudaStream_t st, const double* A, int K, int nb, const double* Linv, double* x,
                       unsigned* sync, int* flag) {
    if (nb == 32)
        sweeps<double, 32>(st, A, K, Linv, nullptr, x, nullptr, sync, flag, nullptr);
    else if (nb == 64)
        sweeps<double, 64>(st, A, K, Linv, nullptr, x, nullptr, sync, flag, nullptr);
    else
        return false;
    return true;
}

// z <- M^{-1} r with M = L L^T the FP32 factor (panel width 64 or 128); the
// sweeps run in FP32 in z32, r and z are FP64.  Nothing runs when *skip != 0.
bool launch_precond32(cudaStream_t st, const float* A, int K, int nb, const float* Linv, float* z32,
                           const double* r, double* z, unsigned* sync, int* flag, const int* skip) {
    if (nb == 128)
        sweeps<float, 128>(st, A, K, Linv, r, z32, z, sync, flag, skip);
    else if (nb == 64)
        sweeps<float, 64>(st, A, K, Linv, r, z32, z, sync, flag, skip);
    else
        return false;
    return true;
}

// Self-test of the bounded wait (no counterpart in the paper): a forward sweep
// whose block 0 is never solved.  Tickets start at 1, so every CTA waits for a
// ready flag that nothing sets; each gives up after 2 s, raises FL_TIMEOUT and
// finishes.  All indices stay inside the buffers (K = 256, eight blocks of 32,
// seven CTAs for blocks 1..7).
extern "C" psdp_status psdp_trsv_timeout_check(float* waited_ms) {
    constexpr int K = 256, W = 32, np = K / W;
    double *A = nullptr, *Li = nullptr, *x = nullptr;
    unsigned* sync = nullptr;
    int* flag = nullptr;
    psdp_status s = PSDP_OK;
    if (cudaMalloc((void**)&A, (size_t)K * K * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&Li, (size_t)np * W * W * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&x, (size_t)K * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&sync, (size_t)(2 + 2 * np) * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc((void**)&flag, sizeof(int)) != cudaSuccess)
        s = PSDP_ENOMEM;
    if (s == PSDP_OK) {
        cudaMemset(A, 0, (size_t)K * K * sizeof(double));
        cudaMemset(Li, 0, (size_t)np * W * W * sizeof(double));
        cudaMemset(x, 0, (size_t)K * sizeof(double));
        cudaMemset(sync, 0, (size_t)(2 + 2 * np) * sizeof(unsigned));
        cudaMemset(flag, 0, sizeof(int));
        const unsigned first = 1;
        cudaMemcpy(sync, &first, sizeof(unsigned), cudaMemcpyHostToDevice);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0);
        k_trsv_fwd<double, W, 2><<<np - 1, TT, trsv_smem<double>(W)>>>(A, K, Li, nullptr, x, sync, flag, nullptr);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) s = PSDP_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (waited_ms) *waited_ms = ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        int h = 0;
        cudaMemcpy(&h, flag, sizeof(int), cudaMemcpyDeviceToHost);
        if (s == PSDP_OK) s = (h & FL_TIMEOUT) ? PSDP_ETIMEOUT : PSDP_OK;
    }
    cudaFree(A);
    cudaFree(Li);
    cudaFree(x);
    cudaFree(sync);
    cudaFree(flag);
    cudaGetLastError();
    return s;
}
