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
// rest); writes L back and L^{-1} (column-major, ld nb).
__global__ void __launch_bounds__(kThreads)
k_potrf_diag32(float* A, int K, int j0, int w, int nb, float* Linv, float* LtHi, float* LtLo, int* flag) {
    extern __shared__ float smf[];
    const int ld = w + 1;
    float* L = smf;
    float* I = smf + (size_t)w * ld;
    __shared__ float rinv[128], ldiag[128];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
        const int j = idx / w, i = idx % w;
        L[j * ld + i] = (i >= j) ? A[(int64_t)(j0 + j) * K + j0 + i] : 0.f;
    }
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        float piv = L[j * ld + j];
        if (!(piv > 0.f) || !isfinite(piv)) {
            if (threadIdx.x == 0) bad = 1;
            piv = 1.f;
        }
        const float ri = 1.f / sqrtf(piv);
        if (threadIdx.x == 0) {
            rinv[j] = ri;
            ldiag[j] = piv * ri;
        }
        for (int i = j + 1 + threadIdx.x; i < w; i += blockDim.x) L[j * ld + i] *= ri;
        __syncthreads();
        // trailing lower triangle: warps take columns, lanes take rows
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int c = j + 1 + wid; c < w; c += nw) {
            const float ljc = L[j * ld + c];
            for (int r = c + lane; r < w; r += 32) L[c * ld + r] = fmaf(-L[j * ld + r], ljc, L[c * ld + r]);
        }
        __syncthreads();
    }
    // L^{-1} by 32 x 32 blocks: diagonal blocks by forward substitution (one
    // thread per column, all blocks at once), then block row i of column j from
    // X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj, one block diagonal per level.
    for (int idx = threadIdx.x; idx < w * ld; idx += blockDim.x) I[idx] = 0.f;
    __syncthreads();
    const int nbk = (w + 31) / 32;
    if (threadIdx.x < nbk * 32) {
        const int d = threadIdx.x >> 5, c = threadIdx.x;
        const int hi = min(w, d * 32 + 32);
        if (c < w) {
            for (int r = c; r < hi; ++r) {
                float s = (r == c) ? 1.f : 0.f;
                for (int k = c; k < r; ++k) s = fmaf(-L[k * ld + r], I[c * ld + k], s);
                I[c * ld + r] = s * rinv[r];
            }
        }
    }
    __syncthreads();
    __shared__ float Tb[3][32][33];
    for (int lev = 1; lev < nbk; ++lev) {
        const int npair = nbk - lev;
        for (int idx = threadIdx.x; idx < npair * 1024; idx += blockDim.x) {
            const int q = idx >> 10, e = idx & 1023, rr = e >> 5, cc = e & 31;
            const int bj = q, bi = q + lev;
            const int r = bi * 32 + rr, c = bj * 32 + cc;
            float s = 0.f;
            if (r < w && c < w)
                for (int k = c; k < bi * 32; ++k) s = fmaf(L[k * ld + r], I[c * ld + k], s);
            Tb[q][rr][cc] = s;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < npair * 1024; idx += blockDim.x) {
            const int q = idx >> 10, e = idx & 1023, rr = e >> 5, cc = e & 31;
            const int bi = q + lev;
            const int r = bi * 32 + rr, c = q * 32 + cc;
            if (r < w && c < w) {
                float s = 0.f;
                for (int k = 0; k <= rr; ++k) s = fmaf(I[(bi * 32 + k) * ld + r], Tb[q][k][cc], s);
                I[c * ld + r] = -s;
            }
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
        const int j = idx / w, i = idx % w;
        if (i >= j) A[(int64_t)(j0 + j) * K + j0 + i] = (i == j) ? ldiag[j] : L[j * ld + i];
    }
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int j = idx / nb, i = idx % nb;
        Linv[idx] = (j < w && i < w) ? I[j * ld + i] : 0.f;
        // row-major copy split into TF32 (hi, lo): LtHi[k*nb + m] ~ Linv(k, m),
        // the K-major right operand of the tensor-core panel solve
        const float v = (j < w && i < w) ? I[i * ld + j] : 0.f;    // Linv(j, i)
        uint32_t h;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
        LtHi[idx] = __uint_as_float(h);
        LtLo[idx] = v - __uint_as_float(h);
    }
    if (threadIdx.x == 0 && bad) atomicOr(flag, (int)FL_CHOL_SCHUR);
}

// Unsolved panel rows packed K-major as TF32 (hi, lo) pairs:
// Pk[i][m] = P(i, m) = A[(j0 + m) K + j0 + w + i], i < rest, m < w (row length nb).
__global__ void __launch_bounds__(256)
k_pack_panel32(const float* __restrict__ A, int K, int j0, int w, int nb, float* PkHi, float* PkLo) {
    __shared__ float t[32][33];
    const int rest = K - j0 - w;
    const int i0 = blockIdx.x * 32, m0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 rows of 32
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

// Panel rows i in [j0+w, K): P'(i,k) = sum_{m<=k} P(i,m) Linv(k,m), written back
// column-major and packed K-major as (hi, lo) into Pt*[i - j0 - w][k] (row length nb).
constexpr int TR = 64;   // panel rows per CTA
__global__ void __launch_bounds__(kThreads)
k_trsm32_pack(float* A, int K, int j0, int w, int nb, const float* __restrict__ Linv, float* PtHi, float* PtLo) {
    extern __shared__ float smf[];
    float* Li = smf;                    // [w][w]  Li[k*w + m] = Linv(k, m)
    float* Ps = smf + w * w;            // [w][TR+1]  Ps[m*(TR+1) + r] = P(i0 + r, m)
    const int i0 = j0 + w + blockIdx.x * TR;
    const int rows = min(TR, K - i0);
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
        const int m = idx / w, k = idx % w;              // column-major source: Linv(k, m) at m*nb + k
        Li[k * w + m] = Linv[m * nb + k];
    }
    for (int idx = threadIdx.x; idx < w * TR; idx += blockDim.x) {
        const int m = idx / TR, r = idx % TR;
        Ps[m * (TR + 1) + r] = (r < rows) ? A[(int64_t)(j0 + m) * K + i0 + r] : 0.f;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * TR; idx += blockDim.x) {
        const int k = idx / TR, r = idx % TR;
        float s = 0.f;
        for (int m = 0; m <= k; ++m) s = fmaf(Ps[m * (TR + 1) + r], Li[k * w + m], s);
        if (r < rows) {
            A[(int64_t)(j0 + k) * K + i0 + r] = s;
            float h, l;
            split_tf32(s, h, l);
            const int64_t o = (int64_t)(i0 + r - j0 - w) * nb + k;
            PtHi[o] = h;
            PtLo[o] = l;
        }
    }
}

// ----------------------------------------------------------- FP32 solves
__global__ void k_trsv_fwd_diag32(const float* __restrict__ Linv, int nb, int w, int j0, float* b, const int* skip) {
    if (skip && *skip) return;
    __shared__ float z[128];
    for (int i = threadIdx.x; i < w; i += blockDim.x) z[i] = b[j0 + i];
    __syncthreads();
    for (int r = threadIdx.x; r < w; r += blockDim.x) {
        float s = 0.f;
        for (int k = 0; k <= r; ++k) s = fmaf(Linv[k * nb + r], z[k], s);
        b[j0 + r] = s;
    }
}

__global__ void k_gemv_fwd32(const float* __restrict__ A, int K, int j0, int w, float* b, const int* skip) {
    if (skip && *skip) return;
    __shared__ float z[128];
    for (int i = threadIdx.x; i < w; i += blockDim.x) z[i] = b[j0 + i];
    __syncthreads();
    for (int i = j0 + w + blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < w; ++k) s = fmaf(A[(int64_t)(j0 + k) * K + i], z[k], s);
        b[i] -= s;
    }
}

constexpr int kChunk = 2048;
__global__ void k_gemv_bwd_partial32(const float* __restrict__ A, int K, int j0, int w, const float* __restrict__ b,
                                     float* partial, int nchunk, const int* skip) {
    if (skip && *skip) return;
    __shared__ float red[32];
    const int k = blockIdx.x, ch = blockIdx.y;
    const int i0 = j0 + w + ch * kChunk, i1 = min(K, i0 + kChunk);
    float s = 0.f;
    const float* col = A + (int64_t)(j0 + k) * K;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) s = fmaf(col[i], b[i], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        partial[k * nchunk + ch] = t;
    }
}

__global__ void k_trsv_bwd_diag32(const float* __restrict__ Linv, int nb, int w, int j0, const float* partial,
                                  int nchunk, float* b, const int* skip) {
    if (skip && *skip) return;
    __shared__ float z[128];
    for (int r = threadIdx.x; r < w; r += blockDim.x) {
        float s = b[j0 + r];
        for (int ch = 0; ch < nchunk; ++ch) s -= partial[r * nchunk + ch];
        z[r] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < w; k += blockDim.x) {
        float s = 0.f;
        for (int r = k; r < w; ++r) s = fmaf(Linv[k * nb + r], z[r], s);
        b[j0 + k] = s;
    }
}

__global__ void k_cvt64to32(int K, const double* __restrict__ a, float* b, const int* skip) {
    if (skip && *skip) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) b[i] = (float)a[i];
}
__global__ void k_cvt32to64(int K, const float* __restrict__ a, double* b, const int* skip) {
    if (skip && *skip) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) b[i] = (double)a[i];
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
    const size_t sm = (size_t)2 * w * (w + 1) * sizeof(float);
    k_potrf_diag32<<<1, kThreads, sm, st>>>(A, K, j0, w, nb, Linv, LtHi, LtLo, flag);
}

void launch_pack_panel32(cudaStream_t st, const float* A, int K, int j0, int nb, float* PkHi, float* PkLo) {
    const int w = (K - j0 < nb) ? K - j0 : nb;
    const int rest = K - j0 - w;
    if (rest <= 0) return;
    dim3 grid((rest + 31) / 32, (w + 31) / 32);
    k_pack_panel32<<<grid, 256, 0, st>>>(A, K, j0, w, nb, PkHi, PkLo);
}

void launch_trsm32_pack(cudaStream_t st, float* A, int K, int j0, int nb, const float* Linv, float* PtHi,
                        float* PtLo) {
    const int w = (K - j0 < nb) ? K - j0 : nb;
    const int rest = K - j0 - w;
    if (rest <= 0) return;
    const size_t sm = ((size_t)w * w + (size_t)w * (TR + 1)) * sizeof(float);
    k_trsm32_pack<<<(rest + TR - 1) / TR, kThreads, sm, st>>>(A, K, j0, w, nb, Linv, PtHi, PtLo);
}

// z <- M^{-1} r with M = L L^T the FP32 factor (r, z FP64; work in FP32 in z32)
void launch_precond32(cudaStream_t st, const float* A, int K, int nb, const float* Linv, float* z32, float* partial,
                      const double* r, double* z, const int* skip) {
    int blocks = (K + kThreads - 1) / kThreads;
    if (blocks > 4096) blocks = 4096;
    k_cvt64to32<<<blocks, kThreads, 0, st>>>(K, r, z32, skip);
    const int npanel = (K + nb - 1) / nb;
    for (int p = 0; p < npanel; ++p) {
        const int j0 = p * nb, w = (K - j0 < nb) ? K - j0 : nb;
        k_trsv_fwd_diag32<<<1, 128, 0, st>>>(Linv + (size_t)p * nb * nb, nb, w, j0, z32, skip);
        const int rest = K - j0 - w;
        if (rest > 0) {
            int b = (rest + kThreads - 1) / kThreads;
            if (b > 1024) b = 1024;
            k_gemv_fwd32<<<b, kThreads, 0, st>>>(A, K, j0, w, z32, skip);
        }
    }
    for (int p = npanel - 1; p >= 0; --p) {
        const int j0 = p * nb, w = (K - j0 < nb) ? K - j0 : nb;
        const int rest = K - j0 - w;
        int nchunk = 0;
        if (rest > 0) {
            nchunk = (rest + kChunk - 1) / kChunk;
            dim3 g(w, nchunk);
            k_gemv_bwd_partial32<<<g, kThreads, 0, st>>>(A, K, j0, w, z32, partial, nchunk, skip);
        }
        k_trsv_bwd_diag32<<<1, 128, 0, st>>>(Linv + (size_t)p * nb * nb, nb, w, j0, partial, nchunk, z32, skip);
    }
    k_cvt32to64<<<blocks, kThreads, 0, st>>>(K, z32, z, skip);
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
    set_max_dynamic_smem((const void*)k_trsm32_pack, smem_optin);
}
