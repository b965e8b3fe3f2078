// Dense K x K Cholesky of the Schur complement: the diagonal-block factor.
//
// Omega is held row-major with its upper triangle filled, which is the same
// memory as a column-major matrix with its lower triangle filled: element
// (i, j), i >= j, of the column-major view sits at A[j*K + i].  The factor is
// L with Omega = L L^T, overwriting that lower triangle.  Right-looking blocked
// algorithm with panels of nb = 32 columns (orchestrated in api.cu): (1) factor
// the diagonal block in shared memory and invert it (this file), (2) panel <-
// panel * L_jj^{-T} as a GEMM with the inverse, (3) symmetric rank-32 update of
// the trailing lower triangle (next panel's rows by the thin GEMM, the rest by
// the persistent update in k_linalg.cu).  The diagonal-block inverses are kept
// for the triangular sweeps (k_trsv.cu).
#include <cmath>

#include "psdp_internal.h"

namespace {

// Diagonal block of at most 32 columns, four warps, factor and inverse in one
// sweep with one CTA barrier per column.  On GB300 a dependent FP64 operation
// costs ~65 cycles and rsqrt ~375, and one warp issues DFMAs slowly, so the
// sweep is built around the chain pivot_j -> rsqrt -> pivot_{j+1}.  The
// columns stay unscaled during the sweep (A(i, j) instead of
// L(i, j) = A(i, j) r_j, r_j = 1/L_jj) and every rank-1 step uses r_j^2:
//   A(i, q) -= A(i, j) (A(q, j) r_j^2)          (trailing lower triangle, q > j)
//   S(i, q) -= A(i, j) (S(j, q) r_j^2)          (running sums of L^{-1}, q <= j)
// with S the identity at the start, so that L^{-1}(i, q) = S(i, q) r_i and
// L(i, j) = A(i, j) r_j are formed once at the end.  Warp 0 updates only row
// j+1, whose diagonal entry is the next pivot, and its lane j+1 takes the
// rsqrt at once while warps 1-3 update the other rows two at a time (lane =
// column q).  The block is padded to 32 with an identity tail.
__global__ void __launch_bounds__(128)
k_potrf_diag32x4(double* A, int K, int j0, int w, int nb, double* Linv, int* flag) {
    constexpr int LD = 33;
    __shared__ double L[32 * LD];   // A, column-major: A(r, c) = L[c*LD + r]
    __shared__ double X[32 * LD];   // S, column-major
    __shared__ double piv[32], rinv[32], rinv2[32];
    __shared__ int bad;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) bad = 0;
#pragma unroll
    for (int idx = tid; idx < 32 * 32; idx += 128) {             // all eight loads in flight
        const int c = idx >> 5, r = idx & 31;
        double v = (r == c) ? 1.0 : 0.0;
        if (r < w && c < w && r >= c) v = A[(int64_t)(j0 + c) * K + j0 + r];
        L[c * LD + r] = v;
        X[c * LD + r] = (r == c) ? 1.0 : 0.0;
    }
    // a pivot that is not positive and finite is flagged and replaced by 1
    auto take_pivot = [&](int j, double p) {
        const long long bits = __double_as_longlong(p);
        if (!(bits > 0 && bits < 0x7ff0000000000000LL)) {
            bad = 1;
            p = 1.0;
        }
        const double r = rsqrt(p);
        piv[j] = p;
        rinv[j] = r;
        rinv2[j] = r * r;
    };
    __syncthreads();
    if (tid == 0) take_pivot(0, L[0]);
    __syncthreads();
    const int q = lane;
    for (int j = 0; j < 32; ++j) {
        const double r2 = rinv2[j];
        const double vq = (q <= j ? X[q * LD + j] : L[j * LD + q]) * r2;   // S(j, q) or A(q, j), times r_j^2
        double* U = q <= j ? X : L;                                        // U(i, q) = U[q*LD + i]
        if (wid == 0) {
            const int i = j + 1;
            if (i < 32 && q <= i) {
                const double u = fma(-L[j * LD + i], vq, U[q * LD + i]);
                U[q * LD + i] = u;
                if (q == i) take_pivot(i, u);                               // next pivot, its rsqrt now
            }
        } else {
            // rows j+1+wid, j+4+wid, ... two per round: both loads, both DFMAs,
            // both stores, so the second row's DFMA does not wait for the first
            for (int i = j + 1 + wid; i < 32; i += 6) {
                const int ib = i + 3;
                const double la = L[j * LD + i], ua = q <= i ? U[q * LD + i] : 0.0;
                double lb = 0.0, ub = 0.0;
                if (ib < 32) {
                    lb = L[j * LD + ib];
                    ub = q <= ib ? U[q * LD + ib] : 0.0;
                }
                const double ra = fma(-la, vq, ua), rb = fma(-lb, vq, ub);
                if (q <= i) U[q * LD + i] = ra;
                if (ib < 32 && q <= ib) U[q * LD + ib] = rb;
            }
        }
        __syncthreads();
    }
    for (int idx = tid; idx < 32 * 32; idx += 128) {
        const int c = idx >> 5, r = idx & 31;
        if (r < w && c < w && r >= c)
            A[(int64_t)(j0 + c) * K + j0 + r] = (r == c ? piv[c] : L[c * LD + r]) * rinv[c];
    }
    for (int idx = tid; idx < nb * nb; idx += 128) {
        const int c = idx / nb, r = idx % nb;
        Linv[idx] = (r < w && c < w) ? X[c * LD + r] * rinv[r] : 0.0;
    }
    if (tid == 0 && bad) atomicOr(flag, (int)FL_CHOL_SCHUR);
}

}  // namespace

// nb is the Cholesky's panel width, 32 (the kernel's block size)
void launch_potrf_diag(cudaStream_t st, double* A, int K, int j0, int nb, double* Linv, int* flag) {
    const int w = (K - j0 < nb) ? K - j0 : nb;
    k_potrf_diag32x4<<<1, 128, 0, st>>>(A, K, j0, w, nb, Linv, flag);
}

void init_attrs_dense(int) {}
