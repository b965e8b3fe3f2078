// Dense K x K Cholesky of the Schur complement: the diagonal-block factor.
//
// Omega is held row-major with its upper triangle filled, which is the same
// memory as a column-major matrix with its lower triangle filled: element
// (i, j), i >= j, of the column-major view sits at A[j*K + i].  The factor is
// L with Omega = L L^T, overwriting that lower triangle.  Right-looking blocked
// algorithm with panels of nb columns (orchestrated in api.cu): (1) factor the
// nb x nb diagonal block in shared memory and invert it (this file), (2) panel
// <- panel * L_jj^{-T} as a GEMM with the inverse, (3) symmetric rank-nb
// update of the trailing lower triangle with the FP64 TN GEMM.  The
// diagonal-block inverses are kept for the triangular sweeps (k_trsv.cu).
#include <cmath>

#include "psdp_internal.h"

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
k_potrf_diag(double* A, int K, int j0, int w, int nb, double* Linv, int* flag) {
    extern __shared__ double sm[];
    const int ld = w + 1;
    double* L = sm;
    double* I = sm + (size_t)w * ld;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
        const int j = idx / w, i = idx % w;
        L[j * ld + i] = (i >= j) ? A[(int64_t)(j0 + j) * K + j0 + i] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        if (threadIdx.x == 0) {
            double d = L[j * ld + j];
            if (!(d > 0.0) || !isfinite(d)) {
                bad = 1;
                d = 1.0;
            }
            L[j * ld + j] = sqrt(d);
        }
        __syncthreads();
        const double piv = L[j * ld + j];
        for (int i = j + 1 + threadIdx.x; i < w; i += blockDim.x) L[j * ld + i] /= piv;
        __syncthreads();
        const int m = w - j - 1;
        for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
            const int c = j + 1 + idx / m, r = j + 1 + idx % m;
            if (r >= c) L[c * ld + r] -= L[j * ld + r] * L[j * ld + c];
        }
        __syncthreads();
    }
    for (int c = threadIdx.x; c < w; c += blockDim.x) {
        for (int r = 0; r < c; ++r) I[c * ld + r] = 0.0;
        for (int r = c; r < w; ++r) {
            double s = (r == c) ? 1.0 : 0.0;
            for (int k = c; k < r; ++k) s -= L[k * ld + r] * I[c * ld + k];
            I[c * ld + r] = s / L[r * ld + r];
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
        const int j = idx / w, i = idx % w;
        if (i >= j) A[(int64_t)(j0 + j) * K + j0 + i] = L[j * ld + i];
    }
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int j = idx / nb, i = idx % nb;
        Linv[idx] = (j < w && i < w) ? I[j * ld + i] : 0.0;
    }
    if (threadIdx.x == 0 && bad) atomicOr(flag, (int)FL_CHOL_SCHUR);
}

// Diagonal block of at most 32 columns, four warps, factor and inverse in one
// sweep.  GB300's FP64 pipe is narrow, so the critical path is counted in
// dependent FP64 operations.  Column j needs 1/L_jj = rsqrt(piv_j) for the
// column scale and for row j of L^{-1}; then one rank-1 step updates the
// trailing lower triangle of L and, beside it, the running sums of L^{-1}:
// S(i, c) = -sum_{k<j} L(i, k) X(k, c), X(j, c) = S(j, c) / L_jj.  Row i of the
// combined update touches positions q <= i: S(i, q) for q <= j, L(i, q) for
// q > j (a lane per q).  Warp 0 updates only row j+1 and computes the next
// pivot's rsqrt at once, while warps 1-3 update the other rows, so the rsqrt
// overlaps the rank-1 step.  The block is padded to 32 with an identity tail.
__global__ void __launch_bounds__(128)
k_potrf_diag32x4(double* A, int K, int j0, int w, int nb, double* Linv, int* flag) {
    constexpr int LD = 33;
    __shared__ double L[32 * LD];   // column-major: L(r, c) = L[c*LD + r]
    __shared__ double X[32 * LD];   // S, then L^{-1}, column-major
    __shared__ double ldiag[32];
    __shared__ double s_piv, s_ri;
    __shared__ int bad;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) bad = 0;
#pragma unroll
    for (int idx = tid; idx < 32 * 32; idx += 128) {             // all eight loads in flight
        const int c = idx >> 5, r = idx & 31;
        double v = (r == c) ? 1.0 : 0.0;
        if (r < w && c < w && r >= c) v = A[(int64_t)(j0 + c) * K + j0 + r];
        L[c * LD + r] = v;
        X[c * LD + r] = 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        double piv = L[0];
        if (!(piv > 0.0) || !isfinite(piv)) {
            bad = 1;
            piv = 1.0;
        }
        s_piv = piv;
        s_ri = rsqrt(piv);
    }
    __syncthreads();
    const int q = lane;
    for (int j = 0; j < 32; ++j) {
        const double ri = s_ri, piv = s_piv;
        if (wid == 0) {
            if (lane > j) L[j * LD + lane] *= ri;                  // column j of L
        } else if (wid == 1) {
            if (lane < j) X[lane * LD + j] *= ri;                  // row j of L^{-1}
            else if (lane == j) X[j * LD + j] = ri;
        } else if (tid == 64) {
            ldiag[j] = piv * ri;
        }
        __syncthreads();
        const bool sx = q <= j;
        double* U = sx ? X : L;                                    // U(i, q) = U[q*LD + i]
        const double vq = sx ? X[q * LD + j] : L[j * LD + q];      // X(j, q) or L(q, j)
        if (wid == 0) {
            const int i = j + 1;
            if (i < 32 && (sx || q <= i)) {
                const double u = fma(-L[j * LD + i], vq, U[q * LD + i]);
                U[q * LD + i] = u;
                if (q == i) {                                      // next pivot, its rsqrt now
                    double p = u;
                    if (!(p > 0.0) || !isfinite(p)) {
                        bad = 1;
                        p = 1.0;
                    }
                    s_piv = p;
                    s_ri = rsqrt(p);
                }
            }
        } else {
#pragma unroll 4
            for (int i = j + 1 + wid; i < 32; i += 3) {
                if (sx || q <= i) U[q * LD + i] = fma(-L[j * LD + i], vq, U[q * LD + i]);
            }
        }
        __syncthreads();
    }
    for (int idx = tid; idx < 32 * 32; idx += 128) {
        const int c = idx >> 5, r = idx & 31;
        if (r < w && c < w && r >= c) A[(int64_t)(j0 + c) * K + j0 + r] = (r == c) ? ldiag[c] : L[c * LD + r];
    }
    for (int idx = tid; idx < nb * nb; idx += 128) {
        const int c = idx / nb, r = idx % nb;
        Linv[idx] = (r < w && c < w) ? X[c * LD + r] : 0.0;
    }
    if (tid == 0 && bad) atomicOr(flag, (int)FL_CHOL_SCHUR);
}

}  // namespace

void launch_potrf_diag(cudaStream_t st, double* A, int K, int j0, int nb, double* Linv, int* flag) {
    const int w = (K - j0 < nb) ? K - j0 : nb;
    if (w <= 32) {
        k_potrf_diag32x4<<<1, 128, 0, st>>>(A, K, j0, w, nb, Linv, flag);
        return;
    }
    const size_t sm = (size_t)2 * w * (w + 1) * sizeof(double);
    k_potrf_diag<<<1, kThreads, sm, st>>>(A, K, j0, w, nb, Linv, flag);
}

void init_attrs_dense(int smem_max) {
    set_max_dynamic_smem((const void*)k_potrf_diag, smem_max);
}
