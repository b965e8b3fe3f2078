// Kernels specific to the Polya SDP: integer tables, the operators B^T and B,
// the Schur-complement operand build and gather, and the elementwise pieces and
// reductions of one predictor-corrector step.
#include <cfloat>
#include <cmath>

#include <type_traits>

#include "psdp_internal.h"
#include "tc_ptx.cuh"

namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------------ tables
__device__ int64_t dbinom(int nn, int kk) {
    if (kk < 0 || nn < 0 || kk > nn) return 0;
    int64_t r = 1;
    for (int i = 1; i <= kk; ++i) r = r * (nn - kk + i) / i;
    return r;
}
__device__ int64_t dcard(int l, int d) { return (l <= 0 || d < 0) ? 0 : dbinom(l + d - 1, l - 1); }

// exponent vector of the rank-th monomial of W_d (0-based), (d,0,..,0) first
__device__ void unrank(int l, int d, int64_t rank, int* out) {
    int rem = d;
    for (int j = 0; j < l - 1; ++j) {
        int v = rem;
        while (v > 0) {
            const int64_t cnt = dcard(l - j - 1, rem - v);
            if (rank < cnt) break;
            rank -= cnt;
            --v;
        }
        out[j] = v;
        rem -= v;
    }
    out[l - 1] = rem;
}

// d! / prod mu_i! as a product of binomials; 0 if some mu_i < 0 or |mu| != d
__device__ int64_t dmultinomial(int d, const int* mu, int l) {
    int s = 0;
    int64_t r = 1;
    for (int i = 0; i < l; ++i) {
        if (mu[i] < 0) return 0;
        s += mu[i];
        r *= dbinom(s, mu[i]);
    }
    return s == d ? r : 0;
}

__global__ void k_tables(int l, int d_p, int d1, int d2, int d_a, int L0, int L, int M, int Na,
                         int32_t* beta, int32_t* cH, int32_t* W0, int32_t* Wa) {
    const int64_t nbeta = (int64_t)L0 * L, nc = (int64_t)L0 * M * Na;
    int h[PSDP_MAX_L], g[PSDP_MAX_L], lam[PSDP_MAX_L], mu[PSDP_MAX_L];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nbeta + nc + L0 + Na;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < nbeta) {
            // beta_{h,gamma} = coefficient of P_h in alpha^gamma of (sum alpha)^{d1} P(alpha)
            const int hi = (int)(t / L), gi = (int)(t % L);
            unrank(l, d_p, hi, h);
            unrank(l, d_p + d1, gi, g);
            for (int i = 0; i < l; ++i) mu[i] = g[i] - h[i];
            beta[t] = (int32_t)dmultinomial(d1, mu, l);
        } else if (t < nbeta + nc) {
            // H_{h,gamma} = sum_lambda multinomial(d2; gamma - h - lambda) A_lambda
            const int64_t u = t - nbeta;
            const int hi = (int)(u / ((int64_t)M * Na));
            const int gi = (int)((u / Na) % M);
            const int li = (int)(u % Na);
            unrank(l, d_p, hi, h);
            unrank(l, d_p + d_a + d2, gi, g);
            unrank(l, d_a, li, lam);
            for (int i = 0; i < l; ++i) mu[i] = g[i] - h[i] - lam[i];
            cH[u] = (int32_t)dmultinomial(d2, mu, l);
        } else if (t < nbeta + nc + L0) {
            const int hi = (int)(t - nbeta - nc);
            unrank(l, d_p, hi, h);
            for (int i = 0; i < l; ++i) W0[hi * l + i] = h[i];
        } else {
            const int li = (int)(t - nbeta - nc - L0);
            unrank(l, d_a, li, lam);
            for (int i = 0; i < l; ++i) Wa[li * l + i] = lam[i];
        }
    }
}

__global__ void k_hmat(int L0, int M, int Na, int n2, const int32_t* __restrict__ cH, const double* __restrict__ A,
                       double* __restrict__ H) {
    const int64_t total = (int64_t)L0 * M * n2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t hg = t / n2;
        const int e = (int)(t % n2);
        double s = 0.0;
        for (int li = 0; li < Na; ++li) {
            const int c = cH[hg * Na + li];
            if (c) s = fma((double)c, A[(int64_t)li * n2 + e], s);
        }
        H[t] = s;
    }
}

// C_gamma = delta * sum_h beta_{h,gamma} d_p!/h! on P-side blocks (Eq. Cj),
// delta_L * multinomial(gamma) on Lyapunov blocks (0 in the paper).
__global__ void k_cdiag(int l, int d_p, int d1, int d2, int d_a, int L0, int L, int M, const int32_t* beta,
                        double delta, double delta_L, double* cdiag) {
    int h[PSDP_MAX_L], g[PSDP_MAX_L];
    for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < L + M; gi += gridDim.x * blockDim.x) {
        if (gi < L) {
            int64_t s = 0;
            for (int hi = 0; hi < L0; ++hi) {
                unrank(l, d_p, hi, h);
                s += (int64_t)beta[(int64_t)hi * L + gi] * dmultinomial(d_p, h, l);
            }
            cdiag[gi] = delta * (double)s;
        } else {
            unrank(l, d_p + d_a + d2, gi - L, g);
            cdiag[gi] = delta_L * (double)dmultinomial(d_p + d_a + d2, g, l);
        }
    }
}

// --------------------------------------------------------------- svec helpers
__device__ __forceinline__ int svec_index(int i, int j, int n) {
    const int r = min(i, j), s = max(i, j), off = s - r;
    return off * n - (off * (off - 1)) / 2 + r;
}

// ------------------------------------------------------------------ B^T(v)
// targets t < L: out[t] = sum_h beta[h][t] smat(v_h)  (P-side blocks)
// targets t >= L: S[(t-L)] = sum_h c[h][gamma][lambda] smat(v_h), (gamma,lambda) = divmod(t-L, Na)
__global__ void k_bt_combine(int n, int Nt, int L0, int L, int M, int Na, const int32_t* __restrict__ beta,
                             const int32_t* __restrict__ cH, const double* __restrict__ v, double* out, double* S,
                             const int* skip) {
    if (skip && *skip) return;
    const int n2 = n * n;
    const int t = blockIdx.y;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += gridDim.x * blockDim.x) {
        const int i = e / n, j = e % n;
        const int q = svec_index(i, j, n);
        double s = 0.0;
        if (t < L) {
            for (int h = 0; h < L0; ++h) {
                const int b = beta[h * L + t];
                if (b) s = fma((double)b, v[(int64_t)h * Nt + q], s);
            }
            out[(int64_t)t * n2 + e] = s;
        } else {
            const int u = t - L, gi = u / Na, li = u % Na;
            for (int h = 0; h < L0; ++h) {
                const int c = cH[((int64_t)h * M + gi) * Na + li];
                if (c) s = fma((double)c, v[(int64_t)h * Nt + q], s);
            }
            S[(int64_t)u * n2 + e] = s;
        }
    }
}

// in place: out = -(N + N^T) on the Lyapunov blocks
__global__ void k_symneg(int nb, int n, double* N, const int* skip) {
    if (skip && *skip) return;
    const int g = blockIdx.y;
    double* Ng = N + (int64_t)g * n * n;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int i = e / n, j = e % n;
        if (i <= j) {
            const double a = Ng[i * n + j], b = Ng[j * n + i];
            Ng[i * n + j] = -(a + b);
            Ng[j * n + i] = -(a + b);
        }
    }
}

// ------------------------------------------------------------------ B(W)
// targets t = h*(Na+1) + lp: lp == Na -> Q_h = sum_{gamma in P} beta sym(W_gamma);
// else R_{h,lp} = sum_{gamma in Lyap} c[h][gamma][lp] sym(W_{L+gamma}).
constexpr int kAdjE = 64, kAdjG = 4;   // outputs per CTA pass, interleaved partial sums over blocks
__global__ void __launch_bounds__(kAdjE * kAdjG)
k_adj_combine(int n, int L0, int L, int M, int Na, const int32_t* __restrict__ beta,
              const int32_t* __restrict__ cH, const double* __restrict__ W, double* out, const int* skip) {
    if (skip && *skip) return;
    __shared__ double red[kAdjG][kAdjE];
    const int n2 = n * n;
    const int t = blockIdx.y;
    const int h = t / (Na + 1), lp = t % (Na + 1);
    const int tx = threadIdx.x % kAdjE, ty = threadIdx.x / kAdjE;
    for (int e0 = blockIdx.x * kAdjE; e0 < n2; e0 += gridDim.x * kAdjE) {
        const int e = e0 + tx;
        double s = 0.0;
        if (e < n2) {
            const int i = e / n, j = e % n;
            const int et = j * n + i;
            // thread row ty sums the blocks g = ty (mod kAdjG) in order
            if (lp == Na) {
                for (int g = ty; g < L; g += kAdjG) {
                    const int b = beta[h * L + g];
                    if (b) s = fma((double)b, 0.5 * (W[(int64_t)g * n2 + e] + W[(int64_t)g * n2 + et]), s);
                }
            } else {
                for (int g = ty; g < M; g += kAdjG) {
                    const int c = cH[((int64_t)h * M + g) * Na + lp];
                    if (c) {
                        const int64_t o = (int64_t)(L + g) * n2;
                        s = fma((double)c, 0.5 * (W[o + e] + W[o + et]), s);
                    }
                }
            }
        }
        red[ty][tx] = s;
        __syncthreads();
        if (ty == 0 && e < n2) out[(int64_t)t * n2 + e] = (red[0][tx] + red[1][tx]) + (red[2][tx] + red[3][tx]);
        __syncthreads();
    }
}

// out[h*Nt + q] = svec_adj(Q_h)_q - 2 sum_lambda svec_adj(A_lambda R_{h,lambda})_q - acoef
__global__ void k_adj_finish(int n, int Nt, int L0, int Na, const double* __restrict__ adj,
                             const double* __restrict__ adj2, const int32_t* __restrict__ svec, double acoef,
                             const double* __restrict__ avec, double* out, const int* skip) {
    if (skip && *skip) return;
    const int n2 = n * n;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L0 * Nt; t += gridDim.x * blockDim.x) {
        const int h = t / Nt, q = t % Nt;
        const int r = svec[2 * q], s = svec[2 * q + 1];
        const double* Q = adj + ((int64_t)h * (Na + 1) + Na) * n2;
        double val = (r == s) ? Q[r * n + r] : Q[r * n + s] + Q[s * n + r];
        double ly = 0.0;
        for (int li = 0; li < Na; ++li) {
            const double* N = adj2 + ((int64_t)h * Na + li) * n2;
            ly += (r == s) ? N[r * n + r] : N[r * n + s] + N[s * n + r];
        }
        out[t] = val - 2.0 * ly - (avec ? acoef * avec[t] : acoef);
    }
}

// ---------------------------------------------------------------- elementwise
// G = C - B^T(y) + Z; C = cdiag I on every block plus, when CR is given, the
// constant term's coefficients on the Lyapunov blocks g >= L (CR[(g - L) n^2 + e])
__global__ void k_ew_G(int nb, int n, int L, const double* __restrict__ cdiag, const double* __restrict__ CR,
                       const double* __restrict__ BTy, const double* __restrict__ Z, double* G) {
    const int64_t n2 = (int64_t)n * n, total = n2 * nb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(t / n2), e = (int)(t % n2);
        double c = (e / n == e % n) ? cdiag[g] : 0.0;
        if (CR && g >= L) c += CR[t - (int64_t)L * n2];
        G[t] = c - BTy[t] + Z[t];
    }
}

// M[g] -= CR[g - L] on the Lyapunov blocks (the constant term of the generalised form)
__global__ void k_sub_CR(int nb, int n, int L, const double* __restrict__ CR, double* Mb) {
    const int64_t n2 = (int64_t)n * n, off = (int64_t)L * n2, total = n2 * (nb - L);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        Mb[off + t] -= CR[t];
}

// Q[pt] += R(alpha_pt) = sum_rho R_rho alpha^rho on the simplex lattice points of k_grid_build
__global__ void k_grid_addR(int l, int n, int Nr, int N, int64_t first, const int32_t* __restrict__ Wr,
                            const double* __restrict__ R, double* Q);

__global__ void k_ew_pred(int64_t total, const double* __restrict__ G, const double* __restrict__ D, double* E,
                          double* dZh) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const double e = G[t] - D[t];
        E[t] = e;
        dZh[t] = -e;
    }
}

// out = sym(T) - X
__global__ void k_ew_symsub(int nb, int n, const double* __restrict__ T, const double* __restrict__ X, double* out) {
    const int64_t n2 = (int64_t)n * n, total = n2 * nb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = t / n2;
        const int e = (int)(t % n2), i = e / n, j = e % n;
        out[t] = 0.5 * (T[t] + T[g * n2 + j * n + i]) - X[t];
    }
}

// F = mu * Y - W2
__global__ void k_ew_muY(int64_t total, const double* __restrict__ Y, const double* __restrict__ W2,
                         const double* __restrict__ mu, double* F) {
    const double m = *mu;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        F[t] = m * Y[t] - W2[t];
}

// dX = dXh + sym(F - T);  dZ = dZh + dZb
__global__ void k_ew_corr(int nb, int n, const double* __restrict__ F, const double* __restrict__ T,
                          const double* __restrict__ dXh, const double* __restrict__ dZh,
                          const double* __restrict__ dZb, double* dX, double* dZ) {
    const int64_t n2 = (int64_t)n * n, total = n2 * nb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = t / n2;
        const int e = (int)(t % n2), i = e / n, j = e % n;
        const int64_t tt = g * n2 + j * n + i;
        dX[t] = dXh[t] + 0.5 * ((F[t] - T[t]) + (F[tt] - T[tt]));
        dZ[t] = dZh[t] + dZb[t];
    }
}

__global__ void k_update(int64_t total, int K, double* X, double* Z, double* y, const double* __restrict__ dX,
                         const double* __restrict__ dZ, const double* __restrict__ dyh,
                         const double* __restrict__ dyb, const double* __restrict__ scal, const int* flag) {
    if (*flag) return;   // a failed factorisation leaves the iterate untouched
    const double tp = scal[SC_TP], td = scal[SC_TD];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total + K;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < total) {
            X[t] += tp * dX[t];
            Z[t] += td * dZ[t];
        } else {
            const int64_t k = t - total;
            y[k] += td * (dyh[k] + dyb[k]);
        }
    }
}

__global__ void k_identity(int64_t total, int n, double* X) {
    const int64_t n2 = (int64_t)n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t % n2);
        X[t] = (e / n == e % n) ? 1.0 : 0.0;
    }
}

// ----------------------------------------------------------------- reductions
__device__ double block_sum(double v, double* red) {
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

// part[g] = (tr(Z_g X_g), tr(X_g), ||G_g||^2, cdiag_g tr(X_g)); part[nb] = (sum y, ||BX-1||^2, ||BX||^2, 0)
__global__ void k_partials(int nb, int n, int K, int L, const double* __restrict__ X, const double* __restrict__ Z,
                           const double* __restrict__ G, const double* __restrict__ cdiag,
                           const double* __restrict__ CR, const double* __restrict__ avec,
                           const double* __restrict__ y, const double* __restrict__ BX, double* part) {
    __shared__ double red[32];
    const int g = blockIdx.x;
    const int64_t n2 = (int64_t)n * n;
    if (g < nb) {
        double zx = 0.0, tx = 0.0, gg = 0.0, cx = 0.0;
        const double* Cg = (CR && g >= L) ? CR + (int64_t)(g - L) * n2 : nullptr;
        for (int e = threadIdx.x; e < n2; e += blockDim.x) {
            const double x = X[g * n2 + e];
            zx = fma(Z[g * n2 + e], x, zx);
            const double gv = G[g * n2 + e];
            gg = fma(gv, gv, gg);
            if (e / n == e % n) tx += x;
            if (Cg) cx = fma(Cg[e], x, cx);   // tr(C_g X_g), C_g symmetric
        }
        zx = block_sum(zx, red);
        tx = block_sum(tx, red);
        gg = block_sum(gg, red);
        if (Cg) cx = block_sum(cx, red);
        if (threadIdx.x == 0) {
            part[4 * g + 0] = zx;
            part[4 * g + 1] = tx;
            part[4 * g + 2] = gg;
            part[4 * g + 3] = cdiag[g] * tx + cx;
        }
    } else {
        double sy = 0.0, r2 = 0.0, b2 = 0.0;
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            const double ak = avec ? avec[k] : 1.0;
            sy = fma(ak, y[k], sy);
            const double b = BX[k];
            r2 = fma(b - ak, b - ak, r2);
            b2 = fma(b, b, b2);
        }
        sy = block_sum(sy, red);
        r2 = block_sum(r2, red);
        b2 = block_sum(b2, red);
        if (threadIdx.x == 0) {
            part[4 * nb + 0] = sy;
            part[4 * nb + 1] = r2;
            part[4 * nb + 2] = b2;
            part[4 * nb + 3] = 0.0;
        }
    }
}

__global__ void k_finalize(int nb, int n, int K, const double* __restrict__ part, const double* __restrict__ cdiag,
                           double c2_extra, double a_norm, double sigma, int iter, double* scal, double* info,
                           int* flag) {
    // lane t sums blocks g = t (mod 32) in order, then a fixed xor tree: the
    // same bit pattern on every replay, 32 short chains instead of one long one
    double zx = 0, tx = 0, gg = 0, phi = 0, c2 = 0;
    for (int g = threadIdx.x; g < nb; g += 32) {
        zx += part[4 * g + 0];
        tx += part[4 * g + 1];
        gg += part[4 * g + 2];
        phi += part[4 * g + 3];
        c2 += cdiag[g] * cdiag[g] * n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        zx += __shfl_xor_sync(0xffffffffu, zx, o);
        tx += __shfl_xor_sync(0xffffffffu, tx, o);
        gg += __shfl_xor_sync(0xffffffffu, gg, o);
        phi += __shfl_xor_sync(0xffffffffu, phi, o);
        c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    }
    if (threadIdx.x != 0) return;
    const double psi = part[4 * nb + 0];
    const double pres = sqrt(part[4 * nb + 1]) / (1.0 + a_norm);
    const double dres = sqrt(gg) / (1.0 + sqrt(c2 + c2_extra));
    const double relgap = fabs(psi - phi) / (1.0 + fabs(psi) + fabs(phi));
    const double mu = sigma * zx / ((double)nb * n);
    scal[SC_TRZX] = zx;
    scal[SC_MU] = mu;
    scal[SC_PHI] = phi;
    scal[SC_PSI] = psi;
    scal[SC_RELGAP] = relgap;
    scal[SC_PRES] = pres;
    scal[SC_DRES] = dres;
    scal[SC_TRX] = tx;
    scal[SC_BXN] = sqrt(part[4 * nb + 2]);
    if (!isfinite(zx) || !isfinite(phi) || !isfinite(psi) || !isfinite(pres) || !isfinite(dres))
        atomicOr(flag, (int)FL_NAN);
    info[0] = phi;
    info[1] = psi;
    info[2] = relgap;
    info[3] = pres;
    info[4] = dres;
    info[5] = mu;
    info[6] = scal[SC_TP];
    info[7] = scal[SC_TD];
    info[8] = zx;
    info[9] = tx;
    info[10] = scal[SC_BXN];
    info[11] = (double)iter;
}

__global__ void k_steplen(int nb, double tau, const double* __restrict__ tstep, double* scal) {
    __shared__ double red[2][32];
    double tp = 1e300, td = 1e300;
    for (int g = threadIdx.x; g < nb; g += blockDim.x) {
        tp = fmin(tp, tstep[g]);
        td = fmin(td, tstep[nb + g]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tp = fmin(tp, __shfl_xor_sync(0xffffffffu, tp, o));
        td = fmin(td, __shfl_xor_sync(0xffffffffu, td, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = tp;
        red[1][wid] = td;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            tp = fmin(tp, red[0][i]);
            td = fmin(td, red[1][i]);
        }
        tp = fmin(red[0][0], tp);
        td = fmin(red[1][0], td);
        scal[SC_TPMAX] = tp;
        scal[SC_TDMAX] = td;
        scal[SC_TP] = fmin(1.0, tau * tp);
        scal[SC_TD] = fmin(1.0, tau * td);
    }
}

// --------------------------------------------------------------- Schur pieces
// term descriptor: [a_src, a_idx, a_trans, b_src, b_idx, b_trans, 0, 0]
// src: 0 product (filled by a GEMM), 1 Y block, 2 X block, 3 U, 4 V
__global__ void k_schur_copy(int n, int nterms, const int32_t* __restrict__ desc, const double* __restrict__ w,
                             const double* __restrict__ Y, const double* __restrict__ X,
                             const double* __restrict__ U, const double* __restrict__ V, double* Aop, double* Bop) {
    const int n2 = n * n;
    const int t = blockIdx.y;
    const int32_t* d = desc + 8 * t;
    const double* bufs[5] = {nullptr, Y, X, U, V};
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += gridDim.x * blockDim.x) {
        const int i = e / n, j = e % n;
        if (d[0]) {
            const double* src = bufs[d[0]] + (int64_t)d[1] * n2;
            Aop[(int64_t)t * n2 + e] = w[t] * (d[2] ? src[j * n + i] : src[e]);
        }
        if (d[3]) {
            const double* src = bufs[d[3]] + (int64_t)d[4] * n2;
            Bop[(int64_t)t * n2 + e] = d[5] ? src[j * n + i] : src[e];
        }
    }
}

// One CTA per (pair, p): Omega[(a,p),(b,q)] for all q from the sub-blocks
// F_{iv}[j][u] = T'[(i n + j) n^2 + v n + u] of the pair's contraction T'.
template <class F>
__global__ void __launch_bounds__(kThreads)
k_schur_gather(int n, int Nt, int K, int p0, const int32_t* __restrict__ pa, const int32_t* __restrict__ pb,
               const int32_t* __restrict__ svec, const F* __restrict__ T, F* Om, int* flag) {
    extern __shared__ double smd[];
    __shared__ uint64_t bar;
    F* sm = reinterpret_cast<F*>(smd);
    const int n2 = n * n;
    const int p = blockIdx.x, pl = blockIdx.y, pair = p0 + pl;
    const int a = pa[pair], b = pb[pair];
    const int r = svec[2 * p], s = svec[2 * p + 1];
    const F* Tp = T + (int64_t)pl * n2 * n2;
    F* F1 = sm;                   // F_rs
    F* F2 = sm + n2;              // F_sr (only if r != s)
    constexpr int V = 16 / sizeof(F);
    if (n % V == 0) {
        // rows of 16-byte multiples: every row of both sub-blocks is an asynchronous
        // bulk copy issued at once, completing on one mbarrier, so the whole 2 n^2
        // staging is in flight together (one CTA an SM at n = 100 has nothing else
        // to overlap it with)
        const uint32_t mb = smem_u32(&bar);
        const int nrow = (r != s) ? 2 * n : n;
        const uint32_t rowb = (uint32_t)(n * sizeof(F));
        if (threadIdx.x == 0) {
            mbar_init(mb, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(mb, (uint32_t)nrow * rowb);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            for (int j = threadIdx.x; j < nrow; j += 32) {
                const bool second = j >= n;
                const int jj = second ? j - n : j;
                const F* src = Tp + ((int64_t)(second ? s : r) * n + jj) * n2 + (int64_t)(second ? r : s) * n;
                const uint32_t dst = smem_u32((second ? F2 : F1) + jj * n);
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                    "l"(src), "r"(rowb), "r"(mb)
                    : "memory");
            }
        }
        if (!__syncthreads_and(mbar_wait(mb, 0, flag) ? 1 : 0)) return;
    } else {
#pragma unroll 4
        for (int e = threadIdx.x; e < n2; e += blockDim.x) {
            const int j = e / n, u = e % n;
            F1[e] = Tp[((int64_t)r * n + j) * n2 + s * n + u];
            if (r != s) F2[e] = Tp[((int64_t)s * n + j) * n2 + r * n + u];
        }
    }
    __syncthreads();
    F* row = Om + (int64_t)(a * Nt + p) * K + (int64_t)b * Nt;
    for (int q = threadIdx.x; q < Nt; q += blockDim.x) {
        const int k = svec[2 * q], m = svec[2 * q + 1];
        F v = F1[k * n + m];
        if (k != m) v += F1[m * n + k];
        if (r != s) {
            v += F2[k * n + m];
            if (k != m) v += F2[m * n + k];
        }
        row[q] = v;
    }
}

// ---------------------------------------------------------------- certificate
__global__ void k_certify_finalize(int count, int n, const double* __restrict__ eig, int L, double* out) {
    if (threadIdx.x != 0) return;
    const double u = 1.1102230246251565e-16;   // 2^-53
    int ok = 1;
    double minP = 1e300, minL = 1e300;
    for (int g = 0; g < count; ++g) {
        const double lam = eig[2 * g], fro = eig[2 * g + 1];
        if (!(lam > 64.0 * n * u * fro)) ok = 0;
        if (g < L) minP = fmin(minP, lam);
        else minL = fmin(minL, lam);
    }
    out[0] = ok;
    out[1] = minP;
    out[2] = -minL;
}

// lattice points alpha = gamma / N, gamma in W_N ranks [first, first+cnt):
// P[pt] = sum_h alpha^h smat(y_h), Aal[pt] = sum_lambda alpha^lambda A_lambda
__global__ void k_grid_build(int l, int n, int Nt, int L0, int Na, int N, int64_t first, const int32_t* __restrict__ W0,
                             const int32_t* __restrict__ Wa, const double* __restrict__ y,
                             const double* __restrict__ A, double* P, double* Aal) {
    const int pt = blockIdx.y;
    int gam[PSDP_MAX_L];
    unrank(l, N, first + pt, gam);
    double al[PSDP_MAX_L];
    for (int i = 0; i < l; ++i) al[i] = (double)gam[i] / N;
    const int n2 = n * n;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += gridDim.x * blockDim.x) {
        const int i = e / n, j = e % n;
        const int q = svec_index(i, j, n);
        double sp = 0.0, sa = 0.0;
        for (int h = 0; h < L0; ++h) {
            double w = 1.0;
            for (int k = 0; k < l; ++k)
                for (int c = 0; c < W0[h * l + k]; ++c) w *= al[k];
            sp = fma(w, y[(int64_t)h * Nt + q], sp);
        }
        for (int li = 0; li < Na; ++li) {
            double w = 1.0;
            for (int k = 0; k < l; ++k)
                for (int c = 0; c < Wa[li * l + k]; ++c) w *= al[k];
            sa = fma(w, A[(int64_t)li * n2 + e], sa);
        }
        P[(int64_t)pt * n2 + e] = sp;
        Aal[(int64_t)pt * n2 + e] = sa;
    }
}

__global__ void k_grid_addR(int l, int n, int Nr, int N, int64_t first, const int32_t* __restrict__ Wr,
                            const double* __restrict__ R, double* Q) {
    const int pt = blockIdx.y;
    int gam[PSDP_MAX_L];
    unrank(l, N, first + pt, gam);
    double al[PSDP_MAX_L];
    for (int i = 0; i < l; ++i) al[i] = (double)gam[i] / N;
    const int n2 = n * n;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < Nr; ++r) {
            double w = 1.0;
            for (int k = 0; k < l; ++k)
                for (int c = 0; c < Wr[r * l + k]; ++c) w *= al[k];
            s = fma(w, R[(int64_t)r * n2 + e], s);
        }
        Q[(int64_t)pt * n2 + e] += s;
    }
}

// Warm start: Z_g = (B^T(y0) - C)_g + max(0, theta / x_g - lambda_min) I (the
// block's smallest eigenvalue is eig[2g]), X_g = x_g I.
__global__ void k_start_fix(int nb, int n, const double* __restrict__ cdiag, const double* __restrict__ BTy,
                            const double* __restrict__ eig, const double* __restrict__ xs, double theta, double* X,
                            double* Z) {
    const int64_t n2 = (int64_t)n * n, total = n2 * nb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(t / n2), e = (int)(t % n2);
        const bool diag = (e / n == e % n);
        const double x = xs ? xs[g] : 1.0;
        const double lam = eig[2 * g] - cdiag[g];
        const double shift = fmax(0.0, theta / x - lam);
        Z[t] = BTy[t] - (diag ? cdiag[g] - shift : 0.0);
        X[t] = diag ? x : 0.0;
    }
}

int grid_for(int64_t total) {
    int64_t b = (total + kThreads - 1) / kThreads;
    if (b > 65535 * 8) b = 65535 * 8;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

// ===================================================================== launchers
void launch_tables(cudaStream_t st, int l, int d_p, int d1, int d2, int d_a, int L0, int L, int M, int Na,
                   int32_t* beta, int32_t* cH, int32_t* W0, int32_t* Wa) {
    const int64_t total = (int64_t)L0 * L + (int64_t)L0 * M * Na + L0 + Na;
    k_tables<<<grid_for(total), kThreads, 0, st>>>(l, d_p, d1, d2, d_a, L0, L, M, Na, beta, cH, W0, Wa);
}

void launch_hmat(cudaStream_t st, int L0, int M, int Na, int n, const int32_t* cH, const double* A, double* H) {
    const int64_t total = (int64_t)L0 * M * n * n;
    k_hmat<<<grid_for(total), kThreads, 0, st>>>(L0, M, Na, n * n, cH, A, H);
}

void launch_cdiag(cudaStream_t st, psdp_ctx* c) {
    k_cdiag<<<grid_for(c->nblk), kThreads, 0, st>>>(c->l, c->d_p, c->d1, c->d2, c->d_a, c->L0, c->L, c->M, c->d_beta,
                                                    c->opt.delta, c->opt.delta_L, c->d_cdiag);
}

void launch_bt(cudaStream_t st, psdp_ctx* c, const double* v, double* out, const int* skip) {
    const int n = c->n, n2 = c->n2;
    dim3 g1((n2 + kThreads - 1) / kThreads, c->L + c->M * c->Na);
    k_bt_combine<<<g1, kThreads, 0, st>>>(n, c->Nt, c->L0, c->L, c->M, c->Na, c->d_beta, c->d_cH, v, out, c->d_S,
                                          skip);
    // N_gamma = sum_lambda S_{gamma,lambda} A_lambda  (written into the Lyapunov output blocks)
    double* outL = out + (int64_t)c->L * n2;
    launch_bgemm(st, n, c->M, c->d_S, nullptr, c->Na, 0, c->d_A, nullptr, 0, 0, outL, nullptr, 1, 0, 1.0, 0.0, skip,
                 c->Na, 1, 1);
    dim3 g2((n2 + kThreads - 1) / kThreads, c->M);
    k_symneg<<<g2, kThreads, 0, st>>>(c->M, n, outL, skip);
}

void launch_b(cudaStream_t st, psdp_ctx* c, const double* W, double* out, double acoef, const int* skip) {
    const int n = c->n, n2 = c->n2;
    dim3 g1((n2 + kAdjE - 1) / kAdjE, c->L0 * (c->Na + 1));
    k_adj_combine<<<g1, kAdjE * kAdjG, 0, st>>>(n, c->L0, c->L, c->M, c->Na, c->d_beta, c->d_cH, W, c->d_adj, skip);
    const int32_t* ix = c->d_adj_idx;
    const int np = c->L0 * c->Na;
    launch_bgemm(st, n, np, c->d_A, ix, 0, 0, c->d_adj, ix + np, 0, 0, c->d_adj2, ix + 2 * np, 0, 0, 1.0, 0.0, skip);
    k_adj_finish<<<grid_for((int64_t)c->L0 * c->Nt), kThreads, 0, st>>>(n, c->Nt, c->L0, c->Na, c->d_adj, c->d_adj2,
                                                                        c->d_svec, acoef, c->d_avec, out, skip);
}

void launch_ew_G(cudaStream_t st, psdp_ctx* c, const double* BTy, const double* Z, double* G) {
    k_ew_G<<<grid_for((int64_t)c->nblk * c->n2), kThreads, 0, st>>>(c->nblk, c->n, c->L, c->d_cdiag, c->d_CR, BTy, Z,
                                                                    G);
}
void launch_ew_pred(cudaStream_t st, psdp_ctx* c, const double* G, const double* D, double* E, double* dZh) {
    const int64_t total = (int64_t)c->nblk * c->n2;
    k_ew_pred<<<grid_for(total), kThreads, 0, st>>>(total, G, D, E, dZh);
}
void launch_ew_symsub(cudaStream_t st, psdp_ctx* c, const double* T, const double* X, double* out) {
    k_ew_symsub<<<grid_for((int64_t)c->nblk * c->n2), kThreads, 0, st>>>(c->nblk, c->n, T, X, out);
}
void launch_ew_muY(cudaStream_t st, psdp_ctx* c, const double* Y, const double* W2, const double* mu, double* F) {
    const int64_t total = (int64_t)c->nblk * c->n2;
    k_ew_muY<<<grid_for(total), kThreads, 0, st>>>(total, Y, W2, mu, F);
}
void launch_ew_corr(cudaStream_t st, psdp_ctx* c, const double* F, const double* T, const double* dXh,
                    const double* dZh, const double* dZb, double* dX, double* dZ) {
    k_ew_corr<<<grid_for((int64_t)c->nblk * c->n2), kThreads, 0, st>>>(c->nblk, c->n, F, T, dXh, dZh, dZb, dX, dZ);
}
void launch_update(cudaStream_t st, psdp_ctx* c) {
    const int64_t total = (int64_t)c->nblk * c->n2;
    k_update<<<grid_for(total + c->K), kThreads, 0, st>>>(total, c->K, c->d_X, c->d_Z, c->d_y, c->d_dX, c->d_dZ,
                                                          c->d_dyh, c->d_dyb, c->d_scal, c->d_flag);
}
void launch_identity(cudaStream_t st, int nb, int n, double* X) {
    const int64_t total = (int64_t)nb * n * n;
    k_identity<<<grid_for(total), kThreads, 0, st>>>(total, n, X);
}
void launch_partials(cudaStream_t st, psdp_ctx* c) {
    k_partials<<<c->nblk + 1, kThreads, 0, st>>>(c->nblk, c->n, c->K, c->L, c->d_X, c->d_Z, c->d_G, c->d_cdiag,
                                                 c->d_CR, c->d_avec, c->d_y, c->d_BX, c->d_part);
}
void launch_finalize(cudaStream_t st, psdp_ctx* c, int iter) {
    k_finalize<<<1, 32, 0, st>>>(c->nblk, c->n, c->K, c->d_part, c->d_cdiag, c->c2_extra,
                                 c->d_avec ? c->a_norm : sqrt((double)c->K), c->opt.sigma, iter, c->d_scal, c->d_info,
                                 c->d_flag);
}
void launch_steplen(cudaStream_t st, psdp_ctx* c) {
    k_steplen<<<1, kThreads, 0, st>>>(c->nblk, c->opt.tau, c->d_tstep, c->d_scal);
}

void launch_schur_operands(cudaStream_t st, psdp_ctx* c) {
    const int n = c->n, n2 = c->n2, LM = c->L0 * c->M;
    const int64_t Loff = (int64_t)c->L * n2;
    // U[h][g] = Y_{L+g} H_{h,g}^T,  V[h][g] = X_{L+g} H_{h,g}^T
    launch_bgemm(st, n, LM, c->d_Y + Loff, c->d_uv_idx, 0, 0, c->d_H, nullptr, 1, 1, c->d_U, nullptr, 1, 0, 1.0, 0.0);
    launch_bgemm(st, n, LM, c->d_X + Loff, c->d_uv_idx, 0, 0, c->d_H, nullptr, 1, 1, c->d_V, nullptr, 1, 0, 1.0, 0.0);
    dim3 g((n2 + kThreads - 1) / kThreads, c->nterms);
    k_schur_copy<<<g, kThreads, 0, st>>>(n, c->nterms, c->d_term_desc, c->d_term_w, c->d_Y, c->d_X, c->d_U, c->d_V,
                                         c->d_Aop, c->d_Bop);
    const int np = c->nlyap_prod;
    if (np > 0) {
        const int32_t* ix = c->d_prod_idx;
        // Phi^T of kind 2: H_a V_b  -> Bop[t]
        launch_bgemm(st, n, np, c->d_H, ix, 0, 0, c->d_V, ix + np, 0, 0, c->d_Bop, ix + 2 * np, 0, 0, 1.0, 0.0);
        // Psi of kind 3: H_a U_b -> Aop[t]
        launch_bgemm(st, n, np, c->d_H, ix + 3 * np, 0, 0, c->d_U, ix + 4 * np, 0, 0, c->d_Aop, ix + 5 * np, 0, 0, 1.0,
                     0.0);
    }
}

void launch_schur_gather(cudaStream_t st, psdp_ctx* c, int p0, int np) {
    const size_t sm = (size_t)2 * c->n2 * sizeof(double);
    dim3 g(c->Nt, np);
    k_schur_gather<double><<<g, kThreads, sm, st>>>(c->n, c->Nt, c->K, p0, c->d_pair_a, c->d_pair_b, c->d_svec,
                                                    c->d_Tbuf, c->d_Om, c->d_flag);
}

void launch_schur_gather32(cudaStream_t st, psdp_ctx* c, int p0, int np, const float* T, float* Om) {
    const size_t sm = (size_t)2 * c->n2 * sizeof(float);
    dim3 g(c->Nt, np);
    k_schur_gather<float><<<g, kThreads, sm, st>>>(c->n, c->Nt, c->K, p0, c->d_pair_a, c->d_pair_b, c->d_svec, T,
                                                   Om, c->d_flag);
}

void launch_start_fix(cudaStream_t st, psdp_ctx* c, const double* BTy, const double* eig, const double* xs,
                      double theta) {
    k_start_fix<<<grid_for((int64_t)c->nblk * c->n2), kThreads, 0, st>>>(c->nblk, c->n, c->d_cdiag, BTy, eig, xs,
                                                                        theta, c->d_X, c->d_Z);
}

void launch_sub_CR(cudaStream_t st, psdp_ctx* c, double* blocks) {
    if (!c->d_CR) return;
    k_sub_CR<<<grid_for((int64_t)c->M * c->n2), kThreads, 0, st>>>(c->nblk, c->n, c->L, c->d_CR, blocks);
}

void launch_grid_addR(cudaStream_t st, psdp_ctx* c, int N, int64_t first, int cnt, double* Q) {
    if (!c->d_R) return;
    dim3 g((c->n2 + kThreads - 1) / kThreads, cnt);
    k_grid_addR<<<g, kThreads, 0, st>>>(c->l, c->n, c->Nr, N, first, c->d_Wr, c->d_R, Q);
}

void launch_certify_finalize(cudaStream_t st, int count, int n, const double* eig, int L, double* out) {
    k_certify_finalize<<<1, 32, 0, st>>>(count, n, eig, L, out);
}

void launch_grid_build(cudaStream_t st, psdp_ctx* c, int N, int64_t first, int cnt, double* P, double* Aal) {
    dim3 g((c->n2 + kThreads - 1) / kThreads, cnt);
    k_grid_build<<<g, kThreads, 0, st>>>(c->l, c->n, c->Nt, c->L0, c->Na, N, first, c->d_W0, c->d_Wa, c->d_y, c->d_A,
                                         P, Aal);
}

void init_attrs_sdp(int smem_max) {
    set_max_dynamic_smem((const void*)k_schur_gather<double>, smem_max);
    set_max_dynamic_smem((const void*)k_schur_gather<float>, smem_max);
}
