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

// Diagonal block of at most 32 columns, four warps.  GB300's FP64 pipe is
// narrow, so the critical path is counted in dependent FP64 operations:
// column j needs one rsqrt (1/L_jj; L_jj = piv * rsqrt(piv)) shared by the
// column scale, then a rank-1 update spread over 128 threads.  L^{-1} is
// built by 2 x 2 block recursion: the 16 x 16 diagonal inverses by forward
// substitution in two warps at once, then -C^{-1} (B A^{-1}) as two small GEMMs.
__global__ void __launch_bounds__(128)
k_potrf_diag32x4(double* A, int K, int j0, int w, int nb, double* Linv, int* flag) {
    constexpr int LD = 33;
    __shared__ double L[32 * LD];   // column-major: L[c*LD + r]
    __shared__ double X[32 * LD];   // L^{-1}, column-major
    __shared__ double T[16 * 17];
    __shared__ double rinv[32], ldiag[32];
    __shared__ int bad;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    for (int idx = tid; idx < 32 * 32; idx += 128) {
        const int c = idx / 32, r = idx % 32;
        double v = (r == c) ? 1.0 : 0.0;
        if (r < w && c < w && r >= c) v = A[(int64_t)(j0 + c) * K + j0 + r];
        L[c * LD + r] = v;
        X[c * LD + r] = 0.0;
    }
    __syncthreads();
    for (int j = 0; j < 32; ++j) {
        double piv = L[j * LD + j];
        if (!(piv > 0.0) || !isfinite(piv)) {
            if (tid == 0) bad = 1;
            piv = 1.0;
        }
        const double ri = rsqrt(piv);
        if (tid == 0) {
            rinv[j] = ri;
            ldiag[j] = piv * ri;    // L_jj; the stored diagonal is read by no later step
        }
        if (tid > j && tid < 32) L[j * LD + tid] *= ri;
        __syncthreads();
        // trailing lower triangle: the four warps take columns, lanes take rows
        for (int c = j + 1 + (tid >> 5); c < 32; c += 4) {
            const double ljc = L[j * LD + c];
            const int r = tid & 31;
            if (r >= c) L[c * LD + r] = fma(-L[j * LD + r], ljc, L[c * LD + r]);
        }
        __syncthreads();
    }
    // diagonal 16 x 16 inverses: warp 0 -> rows/cols 0..15, warp 1 -> 16..31 (lane = column)
    if (tid < 64 && (tid & 31) < 16) {
        const int o = (tid >> 5) * 16, c = o + (tid & 31);
        for (int r = c; r < o + 16; ++r) {
            double s = (r == c) ? 1.0 : 0.0;
            for (int k = c; k < r; ++k) s = fma(-L[k * LD + r], X[c * LD + k], s);
            X[c * LD + r] = s * rinv[r];
        }
    }
    __syncthreads();
    // T = B A^{-1}   (B = L[16..31][0..15], A^{-1} = X[0..15][0..15])
    for (int idx = tid; idx < 256; idx += 128) {
        const int r = idx / 16, c = idx % 16;
        double s = 0.0;
        for (int k = c; k < 16; ++k) s = fma(L[k * LD + 16 + r], X[c * LD + k], s);
        T[r * 17 + c] = s;
    }
    __syncthreads();
    // X[16..31][0..15] = -C^{-1} T
    for (int idx = tid; idx < 256; idx += 128) {
        const int r = idx / 16, c = idx % 16;
        double s = 0.0;
        for (int k = 0; k <= r; ++k) s = fma(X[(16 + k) * LD + 16 + r], T[k * 17 + c], s);
        X[c * LD + 16 + r] = -s;
    }
    __syncthreads();
    for (int idx = tid; idx < 32 * 32; idx += 128) {
        const int c = idx / 32, r = idx % 32;
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
