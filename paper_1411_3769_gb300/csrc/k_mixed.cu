// Mixed-precision pieces: the Schur operands packed K-major as 3xTF32 (hi, lo)
// FP32 pairs for the tcgen05 contraction, the FP32 Cholesky panel steps
// (diagonal block factored in FP64 arithmetic, panel TRSM on CUDA cores that
// also packs the panel for the tensor-core trailing update), the FP32
// triangular solves used as the preconditioner, and the FP64 preconditioned
// conjugate-gradient vector kernels.  Every kernel taking `skip` does nothing
// while *skip != 0 (a converged PCG keeps its graph nodes but skips the work).
#include <cmath>

#include "psdp_internal.h"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void split_tf32(float v, float& hi, float& lo) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
    hi = __uint_as_float(h);
    lo = v - hi;
}

// ------------------------------------------------------------- operand packing
// op*[p][e][tl] (K-major, row length tpad) for pair p, element e of the n x n
// operand matrix, local term tl < term_cnt[p]; A side holds Psi (N operand of
// the GEMM), B side holds Phi^T (M operand).  Sources as in the FP64 path, with
// desc[6] / desc[7] the product index of a GEMM-built Psi / Phi^T.
__global__ void k_schur_pack32(int n, int tpad, const int32_t* __restrict__ term_off,
                               const int32_t* __restrict__ term_cnt, const int32_t* __restrict__ desc,
                               const double* __restrict__ w, const double* __restrict__ Y,
                               const double* __restrict__ X, const double* __restrict__ U,
                               const double* __restrict__ V, const double* __restrict__ prodA,
                               const double* __restrict__ prodB, float* aHi, float* aLo, float* bHi, float* bLo) {
    __shared__ float ta[32][33], tb[32][33];
    const int n2 = n * n;
    const int p = blockIdx.z;
    const int e0 = blockIdx.x * 32, t0 = blockIdx.y * 32;
    const int cnt = term_cnt[p], off = term_off[p];
    if (t0 >= cnt) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    const double* bufs[5] = {nullptr, Y, X, U, V};
    for (int tl = ty; tl < 32; tl += 8) {
        const int t = t0 + tl;
        const int e = e0 + tx;
        float va = 0.f, vb = 0.f;
        if (t < cnt && e < n2) {
            const int32_t* d = desc + 8 * (off + t);
            const int i = e / n, j = e % n;
            double a, b;
            if (d[0]) {
                const double* s = bufs[d[0]] + (int64_t)d[1] * n2;
                a = d[2] ? s[j * n + i] : s[e];
            } else {
                a = prodA[(int64_t)d[6] * n2 + e];
            }
            if (d[3]) {
                const double* s = bufs[d[3]] + (int64_t)d[4] * n2;
                b = d[5] ? s[j * n + i] : s[e];
            } else {
                b = prodB[(int64_t)d[7] * n2 + e];
            }
            va = (float)(w[off + t] * a);
            vb = (float)b;
        }
        ta[tl][tx] = va;
        tb[tl][tx] = vb;
    }
    __syncthreads();
    for (int el = ty; el < 32; el += 8) {
        const int e = e0 + el, t = t0 + tx;
        if (e < n2 && t < cnt) {
            const int64_t o = ((int64_t)p * n2 + e) * tpad + t;
            float h, l;
            split_tf32(ta[tx][el], h, l);
            aHi[o] = h;
            aLo[o] = l;
            split_tf32(tb[tx][el], h, l);
            bHi[o] = h;
            bLo[o] = l;
        }
    }
}

// ------------------------------------------------------------- FP32 Cholesky
// Diagonal w x w block (w <= 128) of the FP32 matrix (column-major lower view),
// factored in FP32 (it only seeds the preconditioner; FP64 PCG fixes the
// rest); writes L back, L^{-1} (column-major, ld nb) and L^{-1} row-major as
// TF32 (hi, lo) pairs.  The block is padded to Wp = 32 ceil(w/32) with an
// identity tail and processed in 32-column sub-panels:
//   (a) warp 0 factors the 32 x 32 diagonal sub-block in registers (a lane
//       per row, multipliers exchanged by shuffles);
//   (b) its inverse by forward substitution, a thread per column, the column
//       kept in registers;
//   (c) the rows below: S = B D^{-T} (a thread per row and four columns);
//   (d) the trailing update A22 -= S S^T on 4 x 4 register tiles, and S back
//       into the panel;
// then the off-diagonal blocks of L^{-1} level by level,
//   X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj,
// on 4 x 4 register tiles.  Five barriers per sub-panel instead of two per column.
constexpr int PB = 32;
constexpr int kPotrfThreads = 256;

// scratch after L and L^{-1}: the panel's solved rows k-major, [PB][kSLD]
// (float4-aligned rows of up to 96 solved rows), reused as [3][32][33] by the
// inverse's off-diagonal levels
constexpr int kSLD = 100;
size_t potrf32_smem(int w) {
    const int wp = (w + PB - 1) / PB * PB;
    return ((size_t)2 * wp * (wp + 1) + PB * kSLD) * sizeof(float);
}

// Column J of the in-register factor of a 32 x 32 block (lane = row), then
// the columns after it; compile-time recursion keeps d[] in registers.
template <int J>
__device__ __forceinline__ void chol_warp_step(float (&d)[PB], int lane, int c0, float* rinv, float* ldiag, int& badl) {
    if constexpr (J < PB) {
        float piv = __shfl_sync(0xffffffffu, d[J], J);
        if (!(piv > 0.f) || !isfinite(piv)) {
            badl = 1;
            piv = 1.f;
        }
        const float rj = rsqrtf(piv);
        if (lane == J) {
            d[J] = piv * rj;
            rinv[c0 + J] = rj;
            ldiag[c0 + J] = piv * rj;
        } else if (lane > J) {
            d[J] *= rj;
        }
#pragma unroll
        for (int c = J + 1; c < PB; ++c) {
            const float lc = __shfl_sync(0xffffffffu, d[J], c);
            if (lane >= c) d[c] = fmaf(-d[J], lc, d[c]);
        }
        chol_warp_step<J + 1>(d, lane, c0, rinv, ldiag, badl);
    }
}

__global__ void __launch_bounds__(kPotrfThreads)
k_potrf_diag32(float* A, int K, int j0, int w, int nb, float* Linv, float* LtHi, float* LtLo, int* flag) {
    extern __shared__ float smf[];
    const int wp = (w + PB - 1) / PB * PB, ld = wp + 1, nsub = wp / PB;
    float* L = smf;                        // [wp][ld] column-major: L(r, c) = L[c*ld + r]
    float* X = L + (size_t)wp * ld;        // L^{-1}, same layout
    float* S = X + (size_t)wp * ld;        // [PB][kSLD] scratch, S[k*kSLD + i] = row i of the solved panel
    __shared__ float rinv[128], ldiag[128];
    __shared__ int bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) bad = 0;
    if ((K & 3) == 0) {
        // 16-byte loads of four rows of a column, unrolled: loads in flight
        const int wp4 = wp / 4;
#pragma unroll 4
        for (int idx = tid; idx < wp * wp4; idx += kPotrfThreads) {
            const int c = idx / wp4, r0 = (idx - c * wp4) * 4;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c < w && r0 < w) q = *reinterpret_cast<const float4*>(A + (int64_t)(j0 + c) * K + j0 + r0);
            const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int r = r0 + u;
                float v = 0.f;
                if (r < w && c < w) {
                    if (r >= c) v = qv[u];
                } else if (r == c) {
                    v = 1.f;               // identity tail
                }
                L[c * ld + r] = v;
                X[c * ld + r] = 0.f;
            }
        }
    } else {
#pragma unroll 8
        for (int idx = tid; idx < wp * wp; idx += kPotrfThreads) {   // unrolled: loads in flight
            const int c = idx / wp, r = idx - c * wp;
            float v = 0.f;
            if (r < w && c < w) {
                if (r >= c) v = A[(int64_t)(j0 + c) * K + j0 + r];
            } else if (r == c) {
                v = 1.f;                   // identity tail
            }
            L[c * ld + r] = v;
            X[c * ld + r] = 0.f;
        }
    }
    __syncthreads();
    for (int kb = 0; kb < nsub; ++kb) {
        const int c0 = kb * PB, rest = wp - c0 - PB;
        // (a) factor the diagonal sub-block D
        if (warp == 0) {
            float d[PB];
#pragma unroll
            for (int c = 0; c < PB; ++c) d[c] = (c <= lane) ? L[(c0 + c) * ld + c0 + lane] : 0.f;
            int badl = 0;
            chol_warp_step<0>(d, lane, c0, rinv, ldiag, badl);
#pragma unroll
            for (int c = 0; c < PB; ++c)
                if (c <= lane) L[(c0 + c) * ld + c0 + lane] = d[c];
            if (lane == 0 && badl) bad = 1;
        }
        __syncthreads();
        // (b) D^{-1}: thread c solves D x = e_c, x kept in registers
        if (tid < PB) {
            const int c = tid;
            float xr[PB];
#pragma unroll
            for (int r = 0; r < PB; ++r) {
                float sacc = (r == c) ? 1.f : 0.f;
#pragma unroll
                for (int k = 0; k < r; ++k)
                    if (k >= c) sacc = fmaf(-L[(c0 + k) * ld + c0 + r], xr[k], sacc);
                xr[r] = (r >= c) ? sacc * rinv[c0 + r] : 0.f;
            }
#pragma unroll
            for (int r = 0; r < PB; ++r) X[(c0 + c) * ld + c0 + r] = xr[r];
        }
        __syncthreads();
        if (rest > 0) {
            // (c) S[i][j] = sum_k B(i, k) D^{-1}(j, k), B(i, k) = L(c0+32+i, c0+k)
            for (int idx = tid; idx < rest * 8; idx += kPotrfThreads) {
                const int i = idx % rest, jg = idx / rest;
                float acc4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
                for (int k = 0; k < PB; ++k) {
                    const float bik = L[(c0 + k) * ld + c0 + PB + i];
#pragma unroll
                    for (int t = 0; t < 4; ++t) acc4[t] = fmaf(bik, X[(c0 + k) * ld + c0 + jg + 8 * t], acc4[t]);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) S[(jg + 8 * t) * kSLD + i] = acc4[t];
            }
            __syncthreads();
            // (d) A22 -= S S^T on the lower 4 x 4 tiles; S back into the panel
            const int nt = rest / 4, ntiles = nt * (nt + 1) / 2;
            for (int q = tid; q < ntiles; q += kPotrfThreads) {
                // q -> (ti, tc), ti >= tc, row-major over the lower triangle of tiles
                int ti = (int)((sqrtf(8.f * q + 1.f) - 1.f) * 0.5f);
                while ((ti + 1) * (ti + 2) / 2 <= q) ++ti;
                while (ti * (ti + 1) / 2 > q) --ti;
                const int tc = q - ti * (ti + 1) / 2;
                float acc[4][4] = {};
#pragma unroll 4
                for (int k = 0; k < PB; ++k) {
                    // 16-byte reads of four consecutive rows: neighbouring tiles are
                    // 16 bytes apart, no bank conflict
                    const float4 a4 = *reinterpret_cast<const float4*>(S + k * kSLD + 4 * ti);
                    const float4 b4 = *reinterpret_cast<const float4*>(S + k * kSLD + 4 * tc);
                    const float a[4] = {a4.x, a4.y, a4.z, a4.w}, bb[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], bb[v], acc[u][v]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int i = 4 * ti + u, cc = 4 * tc + v;
                        if (i >= cc) L[(c0 + PB + cc) * ld + c0 + PB + i] -= acc[u][v];
                    }
            }
            for (int idx = tid; idx < rest * PB; idx += kPotrfThreads) {
                const int i = idx % rest, j = idx / rest;
                L[(c0 + j) * ld + c0 + PB + i] = S[j * kSLD + i];
            }
            __syncthreads();
        }
    }
    // off-diagonal blocks of L^{-1}, one block diagonal per level
    float* T = S;                          // [3][32][33]
    for (int lev = 1; lev < nsub; ++lev) {
        const int npair = nsub - lev;      // pairs (bi, bj) = (q + lev, q)
        // T_q = sum_{k=bj}^{bi-1} L_{bi,k} X_{k,bj}: 64 tiles of 4 x 4 per pair
        for (int idx = tid; idx < npair * 64; idx += kPotrfThreads) {
            const int q = idx >> 6, tt = idx & 63, tr = tt & 7, tcl = tt >> 3;
            const int bj = q, bi = q + lev;
            float acc[4][4] = {};
            for (int k = bj * PB; k < bi * PB; ++k) {
                float a[4], bb[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    a[u] = L[k * ld + bi * PB + 4 * tr + u];       // L(bi*32 + row, k)
                    bb[u] = X[(bj * PB + 4 * tcl + u) * ld + k];   // X(k, bj*32 + col)
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], bb[v], acc[u][v]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) T[q * PB * 33 + (4 * tr + u) * 33 + 4 * tcl + v] = acc[u][v];
        }
        __syncthreads();
        // X_{bi,bj} = -X_{bi,bi} T_q
        for (int idx = tid; idx < npair * 64; idx += kPotrfThreads) {
            const int q = idx >> 6, tt = idx & 63, tr = tt & 7, tcl = tt >> 3;
            const int bj = q, bi = q + lev;
            float acc[4][4] = {};
#pragma unroll 4
            for (int k = 0; k < PB; ++k) {
                float a[4], bb[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    a[u] = X[(bi * PB + k) * ld + bi * PB + 4 * tr + u];   // X(bi*32 + row, bi*32 + k)
                    bb[u] = T[q * PB * 33 + k * 33 + 4 * tcl + u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], bb[v], acc[u][v]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    X[(bj * PB + 4 * tcl + v) * ld + bi * PB + 4 * tr + u] = -acc[u][v];
        }
        __syncthreads();
    }
    for (int idx = tid; idx < w * w; idx += kPotrfThreads) {
        const int j = idx / w, i = idx - j * w;
        if (i >= j) A[(int64_t)(j0 + j) * K + j0 + i] = (i == j) ? ldiag[j] : L[j * ld + i];
    }
    for (int idx = tid; idx < nb * nb; idx += kPotrfThreads) {
        const int j = idx / nb, i = idx - j * nb;
        Linv[idx] = (j < w && i < w) ? X[j * ld + i] : 0.f;
        // row-major copy split into TF32 (hi, lo): LtHi[k*nb + m] ~ Linv(k, m),
        // the K-major right operand of the tensor-core panel solve
        const float v = (j < w && i < w) ? X[i * ld + j] : 0.f;    // Linv(j, i)
        uint32_t h;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
        LtHi[idx] = __uint_as_float(h);
        LtLo[idx] = v - __uint_as_float(h);
    }
    if (tid == 0 && bad) atomicOr(flag, (int)FL_CHOL_SCHUR);
}

// Unsolved panel rows packed K-major as TF32 (hi, lo) pairs:
// Pk[i][m] = P(i, m) = A[(j0 + m) K + j0 + w + i], i < rest, m < w (row length nb).
__global__ void __launch_bounds__(256)
k_pack_panel32(const float* __restrict__ A, int K, int j0, int w, int nb, float* PkHi, float* PkLo) {
    __shared__ float t[32][33];
    const int rest = K - j0 - w;
    const int i0 = blockIdx.x * 32, m0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 rows of 32
#pragma unroll
    for (int r = ty; r < 32; r += 8) {
        const int m = m0 + r, i = i0 + tx;
        t[r][tx] = (m < w && i < rest) ? A[(int64_t)(j0 + m) * K + j0 + w + i] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r, m = m0 + tx;
        if (i < rest && m < w) {
            const float v = t[tx][r];
            uint32_t h;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
            PkHi[(int64_t)i * nb + m] = __uint_as_float(h);
            PkLo[(int64_t)i * nb + m] = v - __uint_as_float(h);
        }
    }
}

// ------------------------------------------------------------------- PCG
// state: [0] rz, [1] ||b||^2, [2] ||r||^2, [3] alpha, [4] beta, [5] iterations, [6] relative residual
// done: 0 running, 1 converged, 2 breakdown
__device__ double cta_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

__global__ void k_pcg_init(int K, const double* __restrict__ b, double* x, double* r, double* st, int* done) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        const double v = b[i];
        x[i] = 0.0;
        r[i] = v;
        s = fma(v, v, s);
    }
    s = cta_sum(s, red);
    if (threadIdx.x == 0) {
        st[1] = s;
        st[2] = s;
        st[5] = 0.0;
        st[6] = 0.0;
        *done = (s == 0.0) ? 1 : 0;
    }
}

__global__ void k_pcg_start(int K, const double* __restrict__ r, const double* __restrict__ z, double* p, double* st,
                            const int* done) {
    if (*done) return;
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        s = fma(r[i], z[i], s);
        p[i] = z[i];
    }
    s = cta_sum(s, red);
    if (threadIdx.x == 0) st[0] = s;
}

__global__ void k_pcg_alpha(int K, const double* __restrict__ p, const double* __restrict__ q, double* x, double* r,
                            double* st, int* done, double tol) {
    if (*done) return;
    __shared__ double red[32];
    __shared__ double alpha_s;
    double s = 0.0;
    for (int i = threadIdx.x; i < K; i += blockDim.x) s = fma(p[i], q[i], s);
    s = cta_sum(s, red);
    if (threadIdx.x == 0) alpha_s = (s > 0.0 && st[0] > 0.0) ? st[0] / s : 0.0;
    __syncthreads();
    const double alpha = alpha_s;
    if (alpha == 0.0) {
        if (threadIdx.x == 0) *done = 2;
        return;
    }
    double rr = 0.0;
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double v = fma(-alpha, q[i], r[i]);
        r[i] = v;
        rr = fma(v, v, rr);
    }
    rr = cta_sum(rr, red);
    if (threadIdx.x == 0) {
        st[3] = alpha;
        st[2] = rr;
        st[5] += 1.0;
        if (rr <= tol * tol * st[1]) *done = 1;
    }
}

__global__ void k_pcg_beta(int K, const double* __restrict__ r, const double* __restrict__ z, double* p, double* st,
                           const int* done) {
    if (*done) return;
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < K; i += blockDim.x) s = fma(r[i], z[i], s);
    s = cta_sum(s, red);
    __shared__ double beta_s;
    if (threadIdx.x == 0) {
        beta_s = (st[0] > 0.0) ? s / st[0] : 0.0;
        st[4] = beta_s;
        st[0] = s;
    }
    __syncthreads();
    const double beta = beta_s;
    for (int i = threadIdx.x; i < K; i += blockDim.x) p[i] = fma(beta, p[i], z[i]);
}

__global__ void k_pcg_finish(int K, const double* __restrict__ x, double* out, double* st, const int* done, int* flag,
                             double tol_fail, double* info_slot) {
    for (int i = threadIdx.x; i < K; i += blockDim.x) out[i] = x[i];
    if (threadIdx.x == 0) {
        const double rel = st[1] > 0.0 ? sqrt(st[2] / st[1]) : 0.0;
        st[6] = rel;
        if (*done == 2 || !(rel <= tol_fail)) atomicOr(flag, (int)FL_MIXED);
        if (info_slot) *info_slot += st[5];
    }
}

}  // namespace

// ===================================================================== launchers
void launch_schur_pack32(cudaStream_t st, psdp_ctx* c) {
    const int tmax = c->tpad;
    dim3 g((c->n2 + 31) / 32, (tmax + 31) / 32, c->npairs);
    k_schur_pack32<<<g, kThreads, 0, st>>>(c->n, c->tpad, c->d_term_off_t, c->d_term_cnt, c->d_term_desc, c->d_term_w,
                                           c->d_Y, c->d_X, c->d_U, c->d_V, c->d_prodA, c->d_prodB, c->d_opA_hi,
                                           c->d_opA_lo, c->d_opB_hi, c->d_opB_lo);
}

void launch_potrf_diag32(cudaStream_t st, float* A, int K, int j0, int nb, float* Linv, float* LtHi, float* LtLo,
                         int* flag) {
    const int w = (K - j0 < nb) ? K - j0 : nb;
    k_potrf_diag32<<<1, kPotrfThreads, potrf32_smem(w), st>>>(A, K, j0, w, nb, Linv, LtHi, LtLo, flag);
}

void launch_pack_panel32(cudaStream_t st, const float* A, int K, int j0, int nb, float* PkHi, float* PkLo) {
    const int w = (K - j0 < nb) ? K - j0 : nb;
    const int rest = K - j0 - w;
    if (rest <= 0) return;
    dim3 grid((rest + 31) / 32, (w + 31) / 32);
    k_pack_panel32<<<grid, 256, 0, st>>>(A, K, j0, w, nb, PkHi, PkLo);
}

void launch_pcg_init(cudaStream_t st, int K, const double* b, double* x, double* r, double* s, int* done) {
    k_pcg_init<<<1, 1024, 0, st>>>(K, b, x, r, s, done);
}
void launch_pcg_start(cudaStream_t st, int K, const double* r, const double* z, double* p, double* s, const int* done) {
    k_pcg_start<<<1, 1024, 0, st>>>(K, r, z, p, s, done);
}
void launch_pcg_alpha(cudaStream_t st, int K, const double* p, const double* q, double* x, double* r, double* s,
                      int* done, double tol) {
    k_pcg_alpha<<<1, 1024, 0, st>>>(K, p, q, x, r, s, done, tol);
}
void launch_pcg_beta(cudaStream_t st, int K, const double* r, const double* z, double* p, double* s, const int* done) {
    k_pcg_beta<<<1, 1024, 0, st>>>(K, r, z, p, s, done);
}
void launch_pcg_finish(cudaStream_t st, int K, const double* x, double* out, double* s, const int* done, int* flag,
                       double tol_fail, double* info_slot) {
    k_pcg_finish<<<1, 1024, 0, st>>>(K, x, out, s, done, flag, tol_fail, info_slot);
}

void init_attrs_mixed(int smem_optin) {
    set_max_dynamic_smem((const void*)k_potrf_diag32, smem_optin);
}
