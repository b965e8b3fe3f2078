// C ABI of the Polya/SDP library: context set-up, the Newton-step orchestration
// (one CUDA graph per step), solve / certify and the inspection hooks.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <new>

#include "psdp_internal.h"

void launch_cdiag(cudaStream_t st, psdp_ctx* c);
void init_attrs_linalg(int smem_max);
void init_attrs_sdp(int smem_max);
void init_attrs_dense(int smem_max);
void init_attrs_trsv(int smem_max);

namespace {

int64_t hbinom(int nn, int kk) {
    if (kk < 0 || nn < 0 || kk > nn) return 0;
    int64_t r = 1;
    for (int i = 1; i <= kk; ++i) r = r * (nn - kk + i) / i;
    return r;
}
int64_t hcard(int l, int d) { return (l <= 0 || d < 0) ? 0 : hbinom(l + d - 1, l - 1); }

template <class T>
psdp_status dalloc(T** p, size_t count) {
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return PSDP_ENOMEM;
    }
    return PSDP_OK;
}

#define TRY(x) do { psdp_status s__ = (x); if (s__ != PSDP_OK) return s__; } while (0)

// ------------------------------------------------------------------ profiling
int prof_name_id(psdp_ctx* c, const char* name) {
    for (size_t i = 0; i < c->prof_names.size(); ++i)
        if (c->prof_names[i] == name) return (int)i;
    c->prof_names.emplace_back(name);
    c->prof_launches.push_back(0);
    c->prof_ms.push_back(0.0);
    return (int)c->prof_names.size() - 1;
}

// Inside a stream capture an event record must be an external node to be
// timeable after each replay of the graph.
void record_event(cudaStream_t st, cudaEvent_t e) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
}

int prof_begin(psdp_ctx* c, const char* name, cudaStream_t st) {
    if (!c->prof_on || !c->prof_cur || c->prof_pool_used + 2 > c->prof_pool_limit) return -1;
    ProfSite s;
    s.name_id = prof_name_id(c, name);
    s.a = c->prof_pool[c->prof_pool_used++];
    s.b = c->prof_pool[c->prof_pool_used++];
    s.st = st;
    record_event(st, s.a);
    c->prof_cur->push_back(s);
    return (int)c->prof_cur->size() - 1;
}

void prof_end(psdp_ctx* c, int site) {
    if (site < 0) return;
    const ProfSite& s = (*c->prof_cur)[site];
    record_event(s.st, s.b);
}

void prof_collect(psdp_ctx* c, bool mixed) {
    if (!c->prof_on) return;
    const std::vector<ProfSite>& sites = mixed ? c->prof_sites32 : c->prof_sites;
    c->prof_tr_id.clear();
    c->prof_tr_crit.clear();
    c->prof_tr_t0.clear();
    c->prof_tr_t1.clear();
    for (const ProfSite& s : sites) {
        float ms = 0.f, t0 = 0.f, t1 = 0.f;
        if (cudaEventElapsedTime(&ms, s.a, s.b) == cudaSuccess) {
            c->prof_ms[s.name_id] += ms;
            c->prof_launches[s.name_id] += 1;
        }
        if (cudaEventElapsedTime(&t0, sites[0].a, s.a) == cudaSuccess &&
            cudaEventElapsedTime(&t1, sites[0].a, s.b) == cudaSuccess) {
            c->prof_tr_id.push_back(s.name_id);
            c->prof_tr_crit.push_back(s.st == c->crit ? 1 : 0);
            c->prof_tr_t0.push_back(t0);
            c->prof_tr_t1.push_back(t1);
        }
    }
    cudaGetLastError();
}

struct ProfScope {
    psdp_ctx* c;
    int site;
    ProfScope(psdp_ctx* cc, const char* name) : c(cc), site(prof_begin(cc, name, cc->stream)) {}
    ProfScope(psdp_ctx* cc, const char* name, cudaStream_t st) : c(cc), site(prof_begin(cc, name, st)) {}
    ~ProfScope() { prof_end(c, site); }
};

// ---------------------------------------------------------------- step pieces
void enqueue_schur(psdp_ctx* c) {
    cudaStream_t st = c->stream;
    {
        ProfScope p(c, "schur_operands");
        launch_schur_operands(st, c);
    }
    for (int p0 = 0; p0 < c->npairs; p0 += c->pairs_per_chunk) {
        const int np = std::min(c->pairs_per_chunk, c->npairs - p0);
        if (c->oz_schur) {
            // T_b[r][c] = sum_k Aop_b[k][r] Bop_b[k][c] by the Ozaki scheme: Bop's rows
            // are the tile rows (TMEM lanes), so the column-major store is T_b row-major;
            // depth windows of 256 terms summed in FP64
            const int dpad = std::min(c->tpad, kOzakiMaxDepth);
            for (int k0 = 0; k0 < c->tpad; k0 += kOzakiMaxDepth) {
                {
                    ProfScope p(c, "schur_oz_split");
                    launch_ozaki_split(st, c->d_Aop, c->n2, 0, c->d_term_off + p0, c->n2, c->d_term_cnt + p0, 0, k0,
                                       dpad, np, c->d_oz_sa, c->d_oz_ea);
                    launch_ozaki_split(st, c->d_Bop, c->n2, 0, c->d_term_off + p0, c->n2, c->d_term_cnt + p0, 0, k0,
                                       dpad, np, c->d_oz_sb, c->d_oz_eb);
                }
                ProfScope p(c, "schur_gemm");
                launch_ozaki_gemm(st, c->d_oz_sb, c->n2, 0, c->d_oz_eb, c->d_oz_sa, c->n2, 0, c->d_oz_ea, c->n2, c->n2,
                                  dpad, np, c->d_term_cnt + p0, 0, k0, c->d_Tbuf, c->n2, (int64_t)c->n2 * c->n2, 1.0,
                                  k0 == 0 ? 0.0 : 1.0, 0, c->d_flag);
            }
        } else {
            ProfScope p(c, "schur_gemm");
            launch_gemm_tn(st, c->n2, c->n2, np, c->d_Aop, c->n2, c->d_term_off + p0, 0, c->d_Bop, c->n2,
                           c->d_term_off + p0, 0, c->d_term_cnt + p0, 0, c->d_Tbuf, c->n2, (int64_t)c->n2 * c->n2,
                           1.0, 0.0, 0);
        }
        {
            ProfScope p(c, "schur_gather");
            launch_schur_gather(st, c, p0, np);
        }
    }
}

// `to` waits for the work enqueued on `from` so far (a graph edge under capture).
void stream_dep(cudaStream_t from, cudaStream_t to, cudaEvent_t e) {
    cudaEventRecord(e, from);
    cudaStreamWaitEvent(to, e, 0);
}

// Omega = L L^T in place (column-major lower view of the row-major upper
// triangle), right-looking with panels of nb_chol columns; the diagonal-block
// inverses are kept for the triangular solves.  Look-ahead of depth one: the
// panel factor, the panel solve and the update of the next panel's rows run on
// the high-priority stream `crit`, and the update of the rest of the trailing
// matrix on the main stream, so panel p+1 is factored while the bulk of
// update p is still running.  Per panel p (rows/columns >= j0 + w trailing):
//   crit: potrf(p), trsm(p) | wait bulk(p-1) | next-rows update(p)
//   main: wait trsm(p) | bulk update(p) of the rows below the next panel
// Both updates read only panel p; they write disjoint rows.
// SMs the persistent FP64 trailing update leaves to the look-ahead chain
// (psdp_opts.crit_sms overrides it); measured on the mid-size workload:
// 6.97 ms per step with 8 or 12, 7.02 with 16, 7.18 with 24.
constexpr int kCritSms64 = 8;
// trailing updates of more than this many waves of 32 x 32 tiles per SM take
// the one-shot kernel (large workload: 97 % FP64 pipe on 152 SMs against 92 %
// for the persistent one on 144)
constexpr int kOneShotWaves = 64;

// Omega = L L^T with the trailing updates by the Ozaki scheme: outer panels of
// kOzakiMaxDepth (384) columns (256 below K = 8192), each factored as 32-column inner panels (FP64
// diagonal factor and inverse, FP64 panel solve, update of the outer panel's
// remaining columns), then FP64-accurate updates of depth 256 from the outer
// panel's slices.  Look-ahead of depth one at the outer level:
//   crit: inner(P), split(P) | wait bulk(P-1) | next(P): the next outer panel's columns
//   main: wait split(P) | bulk(P): every column right of the next outer panel
// so outer panel P+1 is factored while bulk(P) runs.  bulk(P-1) and next(P)
// write the same columns and are ordered by the wait; split(P+1) reuses the
// slice buffer bulk(P-1) read, after the same wait.  Every element receives its
// updates in panel order, and the 32 x 32 diagonal inverses are those the
// triangular solves use.
constexpr int kOzakiInnerMinRows = 8192;
// the depth-128 block updates take the Ozaki product from this many rows (large
// step: 420 ms with FP64 FMA below 8192 rows, 414 with it below 2048)
constexpr int kOzakiBlockMinRows = 2048;
// SMs the persistent bulk update leaves to the look-ahead chain: its CTAs fill
// an SM (197 KB of shared memory, all of TMEM), so the chain's kernels run only
// on SMs it does not hold (large workload: 476.5 ms a step with all 152 SMs,
// 473.3 with 8 left, 469.2 with 16, 483.5 with 32).
constexpr int kCritSmsOzaki = 16;
// ... at least, and kCritSmsOzaki * kCritOzakiRows / rest for a trailing matrix
// of rest rows, at most kCritSmsOzakiMax (large step: 468 ms fixed at 16, 463 /
// 459 / 482 / 528 ms with 25000 / 35000 / 45000 / 60000 rows)
constexpr int kCritOzakiRows = 35000, kCritSmsOzakiMax = 64;
void enqueue_cholesky_ozaki(psdp_ctx* c) {
    cudaStream_t st = c->stream, cs = c->crit;
    // outer panels as deep as one exact Ozaki window where the factor is large: each
    // bulk tile drains its TMEM levels once per window (large step: 445 ms with
    // 384 columns, 455 with 256); 256 below, where the longer chain costs more
    // (mid step: 4.56 vs 4.34-4.51 ms)
    const int K = c->K, nb = c->nb_chol, OB = c->K >= kOzakiInnerMinRows ? kOzakiMaxDepth : 256;
    const int crit = c->opt.crit_sms > 0 ? c->opt.crit_sms : kCritSmsOzaki;
    // SMs left to the chain beside bulk(P): the bulk's work falls as rest^2 and the
    // chain's as rest, so the share grows as 1/rest (psdp_opts.crit_sms fixes it)
    auto crit_for = [&](int rest) {
        if (c->opt.crit_sms > 0) return crit;
        return std::min(kCritSmsOzakiMax, std::max(crit, (int)((int64_t)crit * kCritOzakiRows / std::max(rest, 1))));
    };
    double* A = c->d_Om;
    const size_t slice_elems = ozaki_slice_elems(K, OB, 1);
    stream_dep(st, cs, c->ev_fork);
    for (int J0 = 0, P = 0; J0 < K; J0 += OB, ++P) {
        const int wo = std::min(OB, K - J0);
        // blocks of 128 columns inside a large outer panel: an inner panel updates only
        // its own block's columns (depth 32), and each block then updates the outer
        // panel's columns right of it at depth 128, which drains rest x 1344 instead of
        // rest x 2496 Ozaki elements per outer panel (large step: 432 -> 420 ms; the mid
        // workload keeps the single block: 4.36 vs 4.41 ms)
        const int BW = K >= kOzakiInnerMinRows ? 128 : wo;
        for (int b0 = J0; b0 < J0 + wo; b0 += BW) {
            const int wb = std::min(BW, J0 + wo - b0);
            for (int j0 = b0; j0 < b0 + wb; j0 += nb) {
                const int w = std::min(nb, K - j0);
                double* Lp = c->d_Linv + (size_t)(j0 / nb) * nb * nb;
                {
                    ProfScope q(c, "chol_potrf_diag", cs);
                    launch_potrf_diag(cs, A, K, j0, nb, Lp, c->d_flag);
                }
                const int rest = K - j0 - w;
                if (rest <= 0) break;
                double* panel = A + (int64_t)j0 * K + j0 + w;
                {
                    ProfScope q(c, "chol_trsm_gemm", cs);
                    if (rest >= kOzakiInnerMinRows) {
                        // P <- P L_jj^{-T} by the Ozaki scheme (depth 32): the panel and L_jj^{-1}
                        // are split first, so the product may overwrite the panel.  On the FP64
                        // pipe the solve of a 25000-row panel is ~8 SM-ms of DFMAs, which the
                        // chain's SMs cannot finish under the bulk update (470 us against 55 on
                        // the whole GPU)
                        uint16_t* sl_l = c->d_oz_si + ozaki_slice_elems(K, 32, 1);
                        int32_t* ex_l = c->d_oz_ei + K;
                        launch_ozaki_split(cs, panel, K, 0, nullptr, rest, nullptr, w, 0, 32, 1, c->d_oz_si, c->d_oz_ei);
                        launch_ozaki_split(cs, Lp, nb, 0, nullptr, w, nullptr, w, 0, 32, 1, sl_l, ex_l);
                        launch_ozaki_gemm(cs, c->d_oz_si, rest, 0, c->d_oz_ei, sl_l, w, 0, ex_l, rest, w, 32, 1, nullptr,
                                          w, 0, panel, K, 0, 1.0, 0.0, 0, c->d_flag);
                    } else {
                        launch_gemm_tn(cs, w, rest, 1, Lp, nb, nullptr, 0, panel, K, nullptr, 0, nullptr, w, panel, K, 0,
                                       1.0, 0.0, 0);
                    }
                }
                const int nrem = b0 + wb - (j0 + w);      // block columns right of this inner panel
                if (nrem > 0) {
                    // the outer panel's remaining columns, all rows below (lower part): by the
                    // Ozaki scheme from the inner panel's own slices (depth w = 32) where the
                    // rows are many (large workload: 99 -> 55 ms a step), by FP64 FMA below
                    // (mid workload: 1.05 vs 1.84 ms)
                    ProfScope q(c, "chol_inner_update", cs);
                    if (rest >= kOzakiInnerMinRows) {
                        launch_ozaki_split(cs, panel, K, 0, nullptr, rest, nullptr, w, 0, 32, 1, c->d_oz_si, c->d_oz_ei);
                        launch_ozaki_gemm(cs, c->d_oz_si, rest, 0, c->d_oz_ei, c->d_oz_si, rest, 0, c->d_oz_ei, rest, nrem,
                                          32, 1, nullptr, w, 0, A + (int64_t)(j0 + w) * K + j0 + w, K, 0, -1.0, 1.0, 1,
                                          c->d_flag);
                    } else {
                        launch_gemm_tn(cs, nrem, rest, 1, panel, K, nullptr, 0, panel, K, nullptr, 0, nullptr, w,
                                       A + (int64_t)(j0 + w) * K + j0 + w, K, 0, -1.0, 1.0, 1);
                    }
                }
            }
            // the outer panel's columns right of this block, with the whole block (depth wb)
            const int nrem_o = J0 + wo - (b0 + wb), rest_b = K - (b0 + wb);
            if (nrem_o > 0 && rest_b > 0) {
                ProfScope q(c, "chol_block_update", cs);
                const double* Pb = A + (int64_t)b0 * K + b0 + wb;
                double* Cb = A + (int64_t)(b0 + wb) * K + b0 + wb;
                if (rest_b >= kOzakiBlockMinRows) {
                    const int dpb = (wb + 31) / 32 * 32;
                    launch_ozaki_split(cs, Pb, K, 0, nullptr, rest_b, nullptr, wb, 0, dpb, 1, c->d_oz_sm, c->d_oz_em);
                    launch_ozaki_gemm(cs, c->d_oz_sm, rest_b, 0, c->d_oz_em, c->d_oz_sm, rest_b, 0, c->d_oz_em, rest_b,
                                      nrem_o, dpb, 1, nullptr, wb, 0, Cb, K, 0, -1.0, 1.0, 1, c->d_flag);
                } else {
                    launch_gemm_tn(cs, nrem_o, rest_b, 1, Pb, K, nullptr, 0, Pb, K, nullptr, 0, nullptr, wb, Cb, K, 0,
                                   -1.0, 1.0, 1);
                }
            }
        }
        const int rest = K - (J0 + wo);
        if (rest <= 0) break;
        // L(J0+wo+r, J0+k) at Pp[k*K + r]: rows of the outer panel below it
        const double* Pp = A + (int64_t)J0 * K + J0 + wo;
        const int dpad = (wo + 31) / 32 * 32;
        uint16_t* sl = c->d_oz_sa + (size_t)(P & 1) * slice_elems;
        int32_t* ex = c->d_oz_ea + (size_t)(P & 1) * K;
        {
            ProfScope q(c, "chol_oz_split", cs);
            launch_ozaki_split(cs, Pp, K, 0, nullptr, rest, nullptr, wo, 0, dpad, 1, sl, ex);
        }
        stream_dep(cs, st, c->ev_join);                     // main: after split(P)
        stream_dep(st, cs, c->ev_fork);                     // crit: after bulk(P-1)
        double* T = A + (int64_t)(J0 + wo) * K + J0 + wo;   // trailing matrix
        const int wo2 = std::min(OB, rest);
        {
            // the next outer panel's columns [0, wo2) of T, all rows (lower part)
            ProfScope q(c, "chol_syrk_next", cs);
            launch_ozaki_gemm(cs, sl, rest, 0, ex, sl, rest, 0, ex, rest, wo2, dpad, 1, nullptr, wo, 0, T, K, 0,
                              -1.0, 1.0, 1, c->d_flag);
        }
        if (rest > wo2) {
            // columns [wo2, rest) of T, rows from wo2 (lower part)
            ProfScope q(c, "chol_syrk_gemm", st);
            launch_ozaki_gemm(st, sl, rest, wo2, ex, sl, rest, wo2, ex, rest - wo2, rest - wo2, dpad, 1, nullptr,
                              wo, 0, T + (int64_t)wo2 * K + wo2, K, 0, -1.0, 1.0, 1, c->d_flag,
                              std::max(1, c->num_sms - crit_for(rest)));
        }
    }
    stream_dep(cs, st, c->ev_join);
}

void enqueue_cholesky(psdp_ctx* c) {
    if (c->oz_chol) {
        enqueue_cholesky_ozaki(c);
        return;
    }
    cudaStream_t st = c->stream, cs = c->crit;
    const int K = c->K, nb = c->nb_chol;
    double* A = c->d_Om;
    const int npanel = (K + nb - 1) / nb;
    const int crit = c->opt.crit_sms > 0 ? c->opt.crit_sms : kCritSms64;
    cudaMemsetAsync(c->d_chol_ctr, 0, (size_t)npanel * sizeof(int), st);
    stream_dep(st, cs, c->ev_fork);
    for (int j0 = 0, p = 0; j0 < K; j0 += nb, ++p) {
        const int w = std::min(nb, K - j0);
        double* Lp = c->d_Linv + (size_t)p * nb * nb;
        {
            ProfScope q(c, "chol_potrf_diag", cs);
            launch_potrf_diag(cs, A, K, j0, nb, Lp, c->d_flag);
        }
        const int rest = K - j0 - w;
        if (rest <= 0) break;
        double* panel = A + (int64_t)j0 * K + j0 + w;
        {
            // panel <- panel L_jj^{-T}:  C[k][i] = sum_m Linv(k,m) P(i,m)
            ProfScope q(c, "chol_trsm_gemm", cs);
            launch_gemm_tn(cs, w, rest, 1, Lp, nb, nullptr, 0, panel, K, nullptr, 0, nullptr, w, panel, K, 0, 1.0,
                           0.0, 0);
        }
        const int w2 = std::min(nb, rest);
        double* T = A + (int64_t)(j0 + w) * K + j0 + w;     // trailing matrix, leading dimension K
        // the next-rows update and bulk(p) start together (measured faster than
        // holding bulk(p) until the next-rows update has finished)
        stream_dep(cs, st, c->ev_join);                     // main: after trsm(p)
        stream_dep(st, cs, c->ev_fork);                     // crit: after bulk(p-1)
        {
            // rows [0, w2) of the trailing upper triangle -= P[:, :w2]^T P
            ProfScope q(c, "chol_syrk_next", cs);
            launch_gemm_tn(cs, w2, rest, 1, panel, K, nullptr, 0, panel, K, nullptr, 0, nullptr, w, T, K, 0, -1.0,
                           1.0, 1);
        }
        if (rest > w2) {
            // rows [w2, rest) of the trailing upper triangle -= P[:, w2:]^T P[:, w2:].
            // Persistent on all but the SMs left to the look-ahead chain while the
            // chain can be the longer path; a trailing matrix of many waves of
            // tiles (the large workloads' early panels) takes the one-shot tiled
            // kernel on every SM, where the chain hides under the update anyway.
            ProfScope q(c, "chol_syrk_gemm", st);
            const int m = rest - w2, nt = (m + 31) / 32;
            const int64_t ntiles = (int64_t)nt * (nt + 1) / 2;
            double* C = T + (int64_t)w2 * K + w2;
            if (ntiles > (int64_t)kOneShotWaves * c->num_sms) {
                launch_gemm_tn(st, m, m, 1, panel + w2, K, nullptr, 0, panel + w2, K, nullptr, 0, nullptr, w, C, K, 0,
                               -1.0, 1.0, 1);
            } else {
                const int grid = (int)std::min<int64_t>(std::max(1, c->num_sms - crit), (ntiles + 1) / 2);
                launch_syrk_tri_persist(st, m, w, panel + w2, K, C, K, c->d_chol_ctr + p, grid);
            }
        }
    }
    stream_dep(cs, st, c->ev_join);
}

// ----------------------------------------------------------- mixed precision
// Omega in FP32 from the 3xTF32 tensor-core contraction: operands packed K-major
// (Phi^T as the M side, Psi as the N side), T' = sum_t Psi_t (x) Phi_t^T per pair
// in FP32, then the same sub-block gather as the FP64 path.
void enqueue_schur_mixed(psdp_ctx* c) {
    cudaStream_t st = c->stream;
    const int n = c->n, n2 = c->n2, LM = c->L0 * c->M;
    const int64_t Loff = (int64_t)c->L * n2;
    {
        ProfScope p(c, "schur_operands");
        launch_bgemm(st, n, LM, c->d_Y + Loff, c->d_uv_idx, 0, 0, c->d_H, nullptr, 1, 1, c->d_U, nullptr, 1, 0, 1.0, 0.0);
        launch_bgemm(st, n, LM, c->d_X + Loff, c->d_uv_idx, 0, 0, c->d_H, nullptr, 1, 1, c->d_V, nullptr, 1, 0, 1.0, 0.0);
        const int np = c->nlyap_prod;
        if (np > 0) {
            const int32_t* ix = c->d_prod_idx;
            launch_bgemm(st, n, np, c->d_H, ix, 0, 0, c->d_V, ix + np, 0, 0, c->d_prodB, nullptr, 1, 0, 1.0, 0.0);
            launch_bgemm(st, n, np, c->d_H, ix + 3 * np, 0, 0, c->d_U, ix + 4 * np, 0, 0, c->d_prodA, nullptr, 1, 0,
                         1.0, 0.0);
        }
        launch_schur_pack32(st, c);
    }
    for (int p0 = 0; p0 < c->npairs; p0 += c->pairs_per_chunk32) {
        const int np = std::min(c->pairs_per_chunk32, c->npairs - p0);
        {
            ProfScope p(c, "schur_tc_gemm");
            launch_tc_gemm(st, false, 3, c->map_opB_hi, c->map_opA_hi, &c->map_opB_lo, &c->map_opA_lo, n2, n2, np, p0,
                           c->d_term_cnt + p0, 0, c->d_T32, n2, (int64_t)n2 * n2, 1.f, 0.f, 0, c->d_flag);
        }
        {
            ProfScope p(c, "schur_gather");
            launch_schur_gather32(st, c, p0, np, c->d_T32, c->d_Om32);
        }
    }
}

// SMs the persistent trailing update leaves free for the panel factor, the
// panel solve and the next-rows update of the look-ahead (psdp_opts.crit_sms
// overrides it).
constexpr int kCritSms = 16;
// inner panels per outer panel of the FP32 Cholesky
constexpr int kOuterPanels = 4;

// FP32 Cholesky of Omega32 in outer panels of nbo = 4 nb32 columns, each
// factored as nb32-column inner panels:
//   inner panel (critical stream): diagonal factor and inverse (FP32 shared
//     memory), panel solve on the tensor cores (3xTF32; the epilogue writes
//     Omega's panel rows and the TF32 pairs into the outer panel's wide packed
//     buffer), then the update of the outer panel's remaining columns below
//     them (whose epilogue packs the next inner panel);
//   outer trailing update with the whole outer panel, depth nbo, by the
//     persistent tcgen05 kernel: the next outer panel's rows on the critical
//     stream's SMs (then its first inner panel is packed), the rest on the main
//     stream's.
// Depth-one look-ahead at the outer level: outer panel P+1 is factored while the
// bulk update of P runs.  The deep outer updates move each trailing element
// through HBM once per nbo columns instead of once per nb32, and give the tensor
// cores nbo-deep tiles.  The wide packed buffer is double-buffered by outer
// parity: P+1's panel solves write one copy while bulk(P) reads the other
// (bulk(P-1), the last reader of the copy P+1 overwrites, finished before
// P's next-rows update on the critical stream).
void enqueue_cholesky_mixed(psdp_ctx* c) {
    cudaStream_t st = c->stream, cs = c->crit;
    const int K = c->K, nb = c->nb32, OB = kOuterPanels * c->nb32;
    float* A = c->d_Om32;
    const int crit = c->opt.crit_sms > 0 ? c->opt.crit_sms : kCritSms;
    auto fail = [&]() {
        // cannot happen for the sizes setup accepts; report a failed factor
        // rather than leave a silently wrong one (low byte of the flag)
        cudaMemsetAsync(c->d_flag, FL_CHOL_SCHUR, 1, cs);
    };
    stream_dep(st, cs, c->ev_fork);
    bool done = false;
    for (int J0 = 0, P = 0; J0 < K && !done; J0 += OB, ++P) {
        const int wo = std::min(OB, K - J0);
        // wide packed panel: row r <-> factor row J0 + nb + r, column = index within the outer panel
        float* wh = c->d_Pt_hi + (size_t)(P & 1) * K * OB;
        float* wl = c->d_Pt_lo + (size_t)(P & 1) * K * OB;
        for (int j0 = J0; j0 < J0 + wo; j0 += nb) {
            const int w = std::min(nb, K - j0);
            float* Lp = c->d_Linv32 + (size_t)(j0 / nb) * nb * nb;
            {
                ProfScope q(c, "chol32_potrf_diag", cs);
                launch_potrf_diag32(cs, A, K, j0, nb, Lp, c->d_Lt_hi, c->d_Lt_lo, c->d_flag);
            }
            const int rest = K - j0 - w;
            if (rest <= 0) {
                done = true;
                break;
            }
            const int ri = j0 - J0;                              // this panel's offset in the outer panel
            float* ah = wh + (size_t)ri * OB + ri;
            float* al = wl + (size_t)ri * OB + ri;
            CUtensorMap pkh, pkl, lth, ltl;
            if (!(tc_make_map(&pkh, c->d_Pk_hi, false, w, rest, 1, nb, 0, 128) &&
                  tc_make_map(&pkl, c->d_Pk_lo, false, w, rest, 1, nb, 0, 128) &&
                  tc_make_map(&lth, c->d_Lt_hi, false, w, w, 1, nb, 0, 128) &&
                  tc_make_map(&ltl, c->d_Lt_lo, false, w, w, 1, nb, 0, 128))) {
                fail();
                done = true;
                break;
            }
            {
                // panel solve P L_jj^{-T}; an outer panel's first inner panel is packed
                // from Omega, every later one by the epilogue of the inner update
                // that finished its rows
                ProfScope q(c, "chol32_trsm", cs);
                if (j0 == 0) launch_pack_panel32(cs, A, K, j0, nb, c->d_Pk_hi, c->d_Pk_lo);
                launch_tc_gemm(cs, false, 3, pkh, lth, &pkl, &ltl, rest, w, 1, 0, nullptr, w,
                               A + (int64_t)j0 * K + j0 + w, K, 0, 1.f, 0.f, 0, c->d_flag, ah, al, OB, 0, w);
            }
            const int nrem = J0 + wo - (j0 + w);                 // outer-panel columns right of this panel
            if (nrem > 0) {
                CUtensorMap ph, pl, ph2, pl2;
                if (!(tc_make_map(&ph, ah, false, w, rest, 1, OB, 0, 128) &&
                      tc_make_map(&pl, al, false, w, rest, 1, OB, 0, 128) &&
                      tc_make_map(&ph2, ah, false, w, nrem, 1, OB, 0, 128) &&
                      tc_make_map(&pl2, al, false, w, nrem, 1, OB, 0, 128))) {
                    fail();
                    done = true;
                    break;
                }
                ProfScope q(c, "chol32_inner_update", cs);
                launch_tc_gemm(cs, false, 3, ph, ph2, &pl, &pl2, rest, nrem, 1, 0, nullptr, w,
                               A + (int64_t)(j0 + w) * K + j0 + w, K, 0, -1.f, 1.f, 1, c->d_flag, c->d_Pk_hi,
                               c->d_Pk_lo, nb, nb, nb);   // packs the next inner panel
            }
        }
        if (done) break;
        const int rest = K - (J0 + wo);
        if (rest <= 0) break;
        const int wo2 = std::min(OB, rest);                      // next outer panel
        float* oh = wh + (size_t)(wo - nb) * OB;                 // rows from factor row J0 + wo
        float* ol = wl + (size_t)(wo - nb) * OB;
        CUtensorMap qh, ql, qh2, ql2, qhb, qlb;
        bool ok = tc_make_map(&qh, oh, false, wo, rest, 1, OB, 0, 128) &&
                  tc_make_map(&ql, ol, false, wo, rest, 1, OB, 0, 128) &&
                  tc_make_map(&qh2, oh, false, wo, wo2, 1, OB, 0, 128) &&
                  tc_make_map(&ql2, ol, false, wo, wo2, 1, OB, 0, 128);
        if (rest > wo2)
            ok = ok && tc_make_map(&qhb, oh + (size_t)wo2 * OB, false, wo, rest - wo2, 1, OB, 0, 128) &&
                 tc_make_map(&qlb, ol + (size_t)wo2 * OB, false, wo, rest - wo2, 1, OB, 0, 128);
        if (!ok) {
            fail();
            break;
        }
        float* T = A + (int64_t)(J0 + wo) * K + J0 + wo;
        stream_dep(cs, st, c->ev_join);                     // main: after outer panel P
        stream_dep(st, cs, c->ev_fork);                     // crit: after bulk(P-1)
        {
            // the next outer panel's rows (persistent on the critical SMs), then
            // the pack of its first inner panel
            ProfScope q(c, "chol32_syrk_next", cs);
            launch_tc_gemm_persist(cs, 3, qh, qh2, &ql, &ql2, rest, wo2, wo, T, K, -1.f, 1.f, 1, crit, c->d_flag);
            launch_pack_panel32(cs, A, K, J0 + wo, nb, c->d_Pk_hi, c->d_Pk_lo);
        }
        if (rest > wo2) {
            // persistent CTAs leave a few SMs to the critical-path kernels
            ProfScope q(c, "chol32_syrk_tc", st);
            launch_tc_gemm_persist(st, 3, qhb, qhb, &qlb, &qlb, rest - wo2, rest - wo2, wo, T + (int64_t)wo2 * K + wo2,
                                   K, -1.f, 1.f, 1, std::max(1, c->num_sms - crit), c->d_flag);
        }
    }
    stream_dep(cs, st, c->ev_join);
}

// x <- Omega^{-1} b by conjugate gradients in FP64 with the matrix-free product
// Omega v = B(Z^{-1} B^T(v) X) and the FP32 factor as preconditioner; the
// iterations after convergence are skipped on the device.
void enqueue_pcg(psdp_ctx* c, double* b) {
    cudaStream_t st = c->stream;
    const int K = c->K, n = c->n, nb = c->nblk;
    const int* done = c->d_pcg_done;
    ProfScope p(c, "pcg_solve");
    launch_pcg_init(st, K, b, c->d_pcg_x, c->d_pcg_r, c->d_pcg_state, c->d_pcg_done);
    launch_precond32(st, c->d_Om32, K, c->nb32, c->d_Linv32, c->d_z32, c->d_pcg_r, c->d_pcg_z, c->d_trsv_sync,
                          c->d_flag, done);
    launch_pcg_start(st, K, c->d_pcg_r, c->d_pcg_z, c->d_pcg_p, c->d_pcg_state, done);
    for (int it = 0; it < c->pcg_max; ++it) {
        launch_bt(st, c, c->d_pcg_p, c->d_M1, done);
        launch_bgemm(st, n, nb, c->d_Y, nullptr, 1, 0, c->d_M1, nullptr, 1, 0, c->d_M2, nullptr, 1, 0, 1.0, 0.0, done);
        launch_bgemm(st, n, nb, c->d_M2, nullptr, 1, 0, c->d_X, nullptr, 1, 0, c->d_M1, nullptr, 1, 0, 1.0, 0.0, done);
        launch_b(st, c, c->d_M1, c->d_pcg_q, 0.0, done);
        launch_pcg_alpha(st, K, c->d_pcg_p, c->d_pcg_q, c->d_pcg_x, c->d_pcg_r, c->d_pcg_state, c->d_pcg_done,
                         c->pcg_tol);
        launch_precond32(st, c->d_Om32, K, c->nb32, c->d_Linv32, c->d_z32, c->d_pcg_r, c->d_pcg_z,
                              c->d_trsv_sync, c->d_flag, done);
        launch_pcg_beta(st, K, c->d_pcg_r, c->d_pcg_z, c->d_pcg_p, c->d_pcg_state, done);
    }
    launch_pcg_finish(st, K, c->d_pcg_x, b, c->d_pcg_state, done, c->d_flag, c->pcg_fail, c->d_info + 12);
}

void enqueue_refresh(psdp_ctx* c) {
    cudaStream_t st = c->stream;
    launch_bt(st, c, c->d_y, c->d_T1);
    launch_ew_G(st, c, c->d_T1, c->d_Z, c->d_G);
    launch_b(st, c, c->d_X, c->d_BX, 0.0);
    launch_partials(st, c);
    launch_finalize(st, c, 0);
}

// One predictor-corrector step.  mixed: Schur complement and its Cholesky in
// 3xTF32/FP32 on the tensor cores, both Newton systems solved by FP64 PCG;
// otherwise everything in FP64 with direct solves.
void enqueue_step(psdp_ctx* c, bool mixed) {
    cudaStream_t st = c->stream;
    const int n = c->n, nb = c->nblk;
    // each step graph owns half of the profiling event pool and its own site list
    c->prof_cur = mixed ? &c->prof_sites32 : &c->prof_sites;
    c->prof_cur->clear();
    c->prof_pool_used = mixed ? c->prof_pool.size() / 2 : 0;
    c->prof_pool_limit = mixed ? c->prof_pool.size() : c->prof_pool.size() / 2;
    cudaMemsetAsync(c->d_info + 12, 0, 2 * sizeof(double), st);
    {
        ProfScope p(c, "block_chol_inv");
        launch_block_chol_inv(st, nb, n, c->d_Z, c->d_Y, c->d_flag);
    }
    if (mixed)
        enqueue_schur_mixed(c);
    else
        enqueue_schur(c);
    // predictor right-hand side: B(Y G X) - a
    launch_bgemm(st, n, nb, c->d_Y, nullptr, 1, 0, c->d_G, nullptr, 1, 0, c->d_T1, nullptr, 1, 0, 1.0, 0.0);
    launch_bgemm(st, n, nb, c->d_T1, nullptr, 1, 0, c->d_X, nullptr, 1, 0, c->d_W, nullptr, 1, 0, 1.0, 0.0);
    launch_b(st, c, c->d_W, c->d_dyh, 1.0);
    if (mixed) {
        enqueue_cholesky_mixed(c);
        enqueue_pcg(c, c->d_dyh);
    } else {
        enqueue_cholesky(c);
        ProfScope p(c, "dense_solve");
        launch_pair_inverse(st, c->d_Om, c->K, c->d_Linv, c->d_Linv64);
        launch_solve_fp64(st, c->d_Om, c->K, 64, c->d_Linv64, c->d_dyh, c->d_trsv_sync, c->d_flag);
    }
    // predictor directions
    launch_bt(st, c, c->d_dyh, c->d_T2);
    launch_ew_pred(st, c, c->d_G, c->d_T2, c->d_T1, c->d_dZh);
    launch_bgemm(st, n, nb, c->d_Y, nullptr, 1, 0, c->d_T1, nullptr, 1, 0, c->d_W, nullptr, 1, 0, 1.0, 0.0);
    launch_bgemm(st, n, nb, c->d_W, nullptr, 1, 0, c->d_X, nullptr, 1, 0, c->d_T2, nullptr, 1, 0, 1.0, 0.0);
    launch_ew_symsub(st, c, c->d_T2, c->d_X, c->d_dXh);
    // corrector right-hand side: B(mu Y - Y dZh dXh)
    launch_bgemm(st, n, nb, c->d_Y, nullptr, 1, 0, c->d_dZh, nullptr, 1, 0, c->d_T1, nullptr, 1, 0, 1.0, 0.0);
    launch_bgemm(st, n, nb, c->d_T1, nullptr, 1, 0, c->d_dXh, nullptr, 1, 0, c->d_W, nullptr, 1, 0, 1.0, 0.0);
    launch_ew_muY(st, c, c->d_Y, c->d_W, c->d_scal + SC_MU, c->d_F);
    launch_b(st, c, c->d_F, c->d_dyb, 0.0);
    if (mixed) {
        enqueue_pcg(c, c->d_dyb);
    } else {
        ProfScope p(c, "dense_solve");
        launch_solve_fp64(st, c->d_Om, c->K, 64, c->d_Linv64, c->d_dyb, c->d_trsv_sync, c->d_flag);
    }
    // corrector directions and totals
    launch_bt(st, c, c->d_dyb, c->d_T2);
    launch_bgemm(st, n, nb, c->d_Y, nullptr, 1, 0, c->d_T2, nullptr, 1, 0, c->d_T1, nullptr, 1, 0, 1.0, 0.0);
    launch_bgemm(st, n, nb, c->d_T1, nullptr, 1, 0, c->d_X, nullptr, 1, 0, c->d_W, nullptr, 1, 0, 1.0, 0.0);
    launch_ew_corr(st, c, c->d_F, c->d_W, c->d_dXh, c->d_dZh, c->d_T2, c->d_dX, c->d_dZ);
    {
        ProfScope p(c, "block_maxstep");
        launch_block_maxstep(st, nb, n, c->d_X, c->d_dX, c->d_Z, c->d_dZ, c->d_tstep, c->d_flag);
    }
    launch_steplen(st, c);
    launch_update(st, c);
    enqueue_refresh(c);
    cudaMemcpyAsync(c->h_info, c->d_info, PSDP_INFO_LEN * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(c->h_flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
}

psdp_status cuda_fail(cudaError_t e, const char* where) {
    static const bool dbg = getenv("PSDP_DEBUG") != nullptr;
    if (dbg) fprintf(stderr, "[psdp] %s: %s (%s)\n", where, cudaGetErrorName(e), cudaGetErrorString(e));
    return PSDP_ECUDA;
}

psdp_status sync_check(psdp_ctx* c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch");
    return PSDP_OK;
}

psdp_status refresh(psdp_ctx* c) {
    enqueue_refresh(c);
    cudaMemcpyAsync(c->h_info, c->d_info, PSDP_INFO_LEN * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    return sync_check(c);
}

void free_ctx(psdp_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->graph_exec32) cudaGraphExecDestroy(c->graph_exec32);
    if (c->graph32) cudaGraphDestroy(c->graph32);
    void* ptrs[] = {c->d_beta, c->d_cH, c->d_W0, c->d_Wa, c->d_A, c->d_H, c->d_cdiag, c->d_X, c->d_Z, c->d_G,
                    c->d_Y, c->d_T1, c->d_T2, c->d_W, c->d_F, c->d_dXh, c->d_dZh, c->d_dX, c->d_dZ, c->d_S,
                    c->d_adj, c->d_adj2, c->d_adj_idx, c->d_y, c->d_dyh, c->d_dyb, c->d_BX, c->d_part, c->d_tstep,
                    c->d_scal, c->d_info, c->d_flag, c->d_pair_a, c->d_pair_b, c->d_term_off, c->d_term_cnt,
                    c->d_term_desc, c->d_term_w, c->d_uv_idx, c->d_prod_idx, c->d_U, c->d_V, c->d_Aop, c->d_Bop,
                    c->d_Tbuf, c->d_Om, c->d_Linv, c->d_Linv64, c->d_chol_ctr, c->d_grid, c->d_svec, c->d_cert, c->d_term_off_t,
                    c->d_opA_hi, c->d_opA_lo, c->d_opB_hi, c->d_opB_lo, c->d_prodA, c->d_prodB, c->d_T32,
                    c->d_Om32, c->d_Linv32, c->d_Pt_hi, c->d_Pt_lo, c->d_z32, c->d_trsv_sync, c->d_Pk_hi, c->d_Pk_lo, c->d_Lt_hi, c->d_Lt_lo, c->d_pcg_x, c->d_pcg_r,
                    c->d_pcg_z, c->d_pcg_p, c->d_pcg_q, c->d_pcg_state, c->d_pcg_done, c->d_M1, c->d_M2,
                    c->d_oz_sa, c->d_oz_sb, c->d_oz_ea, c->d_oz_eb, c->d_R, c->d_Wr, c->d_CR, c->d_avec,
                    c->d_oz_si, c->d_oz_ei, c->d_oz_sm, c->d_oz_em};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->h_info) cudaFreeHost(c->h_info);
    if (c->h_flag) cudaFreeHost(c->h_flag);
    for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->crit) cudaStreamDestroy(c->crit);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
}

psdp_status build_schur_lists(psdp_ctx* c) {
    const int L0 = c->L0, L = c->L, M = c->M, Na = c->Na;
    std::vector<char> hz((size_t)L0 * M, 0);
    for (int h = 0; h < L0; ++h)
        for (int g = 0; g < M; ++g)
            for (int li = 0; li < Na; ++li)
                if (c->cH[((size_t)h * M + g) * Na + li]) hz[(size_t)h * M + g] = 1;
    std::vector<int32_t> desc, prod_a2, prod_b2, prod_c2, prod_a3, prod_b3, prod_c3;
    std::vector<double> w;
    c->pair_a.clear();
    c->pair_b.clear();
    c->term_off.clear();
    c->term_cnt.clear();
    int t = 0;
    double dense_terms = 0;
    for (int a = 0; a < L0; ++a)
        for (int b = a; b < L0; ++b) {
            c->pair_a.push_back(a);
            c->pair_b.push_back(b);
            c->term_off.push_back(t);
            const int t0 = t;
            dense_terms += L + 4.0 * M;
            for (int g = 0; g < L; ++g) {
                const int wt = c->beta[(size_t)a * L + g] * c->beta[(size_t)b * L + g];
                if (!wt) continue;
                const int32_t d[8] = {1, g, 0, 2, g, 0, 0, 0};
                desc.insert(desc.end(), d, d + 8);
                w.push_back((double)wt);
                ++t;
            }
            for (int g = 0; g < M; ++g) {
                if (!hz[(size_t)a * M + g] || !hz[(size_t)b * M + g]) continue;
                const int blk = L + g, ia = a * M + g, ib = b * M + g;
                const int j = (int)prod_a2.size();                  // index of this (pair, block) product
                const int32_t d1[8] = {3, ib, 0, 4, ia, 1, 0, 0};   // (Y H_b^T, (X H_a^T)^T)
                const int32_t d2[8] = {1, blk, 0, 0, 0, 0, 0, j};   // (Y, H_a X H_b^T)
                const int32_t d3[8] = {0, 0, 0, 2, blk, 0, j, 0};   // (H_a Y H_b^T, X)
                const int32_t d4[8] = {3, ia, 1, 4, ib, 0, 0, 0};   // ((Y H_a^T)^T, X H_b^T)
                desc.insert(desc.end(), d1, d1 + 8);
                desc.insert(desc.end(), d2, d2 + 8);
                desc.insert(desc.end(), d3, d3 + 8);
                desc.insert(desc.end(), d4, d4 + 8);
                w.insert(w.end(), {1.0, 1.0, 1.0, 1.0});
                prod_a2.push_back(ia); prod_b2.push_back(ib); prod_c2.push_back(t + 1);
                prod_a3.push_back(ia); prod_b3.push_back(ib); prod_c3.push_back(t + 2);
                t += 4;
            }
            c->term_cnt.push_back(t - t0);
        }
    c->npairs = (int)c->pair_a.size();
    c->nterms = t;
    c->nlyap_prod = (int)prod_a2.size();
    if ((int64_t)c->nterms * c->n2 >= ((int64_t)1 << 31)) return PSDP_EINVAL;
    c->flops_schur_dense = 2.0 * c->n2 * (double)c->n2 * dense_terms;
    c->flops_schur = 2.0 * c->n2 * (double)c->n2 * (double)c->nterms;
    std::vector<int32_t> offs(c->npairs);
    for (int p = 0; p < c->npairs; ++p) offs[p] = c->term_off[p] * c->n2;
    TRY(dalloc(&c->d_pair_a, c->npairs));
    TRY(dalloc(&c->d_pair_b, c->npairs));
    TRY(dalloc(&c->d_term_off, c->npairs));
    TRY(dalloc(&c->d_term_cnt, c->npairs));
    TRY(dalloc(&c->d_term_desc, (size_t)8 * std::max(1, t)));
    TRY(dalloc(&c->d_term_w, std::max(1, t)));
    const int np = c->nlyap_prod;
    TRY(dalloc(&c->d_prod_idx, (size_t)6 * std::max(1, np)));
    cudaMemcpy(c->d_pair_a, c->pair_a.data(), c->npairs * sizeof(int32_t), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_pair_b, c->pair_b.data(), c->npairs * sizeof(int32_t), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_term_off, offs.data(), c->npairs * sizeof(int32_t), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_term_cnt, c->term_cnt.data(), c->npairs * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (t) {
        cudaMemcpy(c->d_term_desc, desc.data(), desc.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_term_w, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (np) {
        std::vector<int32_t> all;
        for (auto* v : {&prod_a2, &prod_b2, &prod_c2, &prod_a3, &prod_b3, &prod_c3}) all.insert(all.end(), v->begin(), v->end());
        cudaMemcpy(c->d_prod_idx, all.data(), all.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    }
    std::vector<int32_t> uv((size_t)L0 * M);
    for (int e = 0; e < L0 * M; ++e) uv[e] = e % M;
    TRY(dalloc(&c->d_uv_idx, uv.size()));
    cudaMemcpy(c->d_uv_idx, uv.data(), uv.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    TRY(dalloc(&c->d_U, (size_t)L0 * M * c->n2));
    TRY(dalloc(&c->d_V, (size_t)L0 * M * c->n2));
    std::vector<int32_t> toff_t(c->term_off.begin(), c->term_off.end());
    TRY(dalloc(&c->d_term_off_t, c->npairs));
    cudaMemcpy(c->d_term_off_t, toff_t.data(), c->npairs * sizeof(int32_t), cudaMemcpyHostToDevice);
    int tmax = 1;
    for (int p = 0; p < c->npairs; ++p) tmax = std::max(tmax, c->term_cnt[p]);
    c->tpad = (tmax + 31) / 32 * 32;
    return PSDP_OK;
}

psdp_status alloc_ozaki(psdp_ctx* c);

// Buffers of the FP64 Schur contraction and Cholesky (allocated at set-up in
// FP64 mode, on first need in mixed mode).
psdp_status alloc_fp64(psdp_ctx* c) {
    if (c->have_fp64) return PSDP_OK;
    const int t = std::max(1, c->nterms);
    TRY(dalloc(&c->d_Aop, (size_t)t * c->n2));
    TRY(dalloc(&c->d_Bop, (size_t)t * c->n2));
    // contraction output: as many pairs per launch as fit in ~2 GiB
    const size_t per_pair = (size_t)c->n2 * c->n2 * sizeof(double);
    c->pairs_per_chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)c->npairs, ((size_t)2 << 30) / per_pair));
    TRY(dalloc(&c->d_Tbuf, (size_t)c->pairs_per_chunk * c->n2 * c->n2));
    const int nbc = c->nb_chol;
    const int npanel = (c->K + nbc - 1) / nbc;
    TRY(dalloc(&c->d_Om, (size_t)c->K * c->K));
    TRY(dalloc(&c->d_Linv, (size_t)npanel * nbc * nbc));
    TRY(dalloc(&c->d_Linv64, (size_t)((c->K + 63) / 64) * 64 * 64));
    TRY(dalloc(&c->d_chol_ctr, (size_t)npanel));
    TRY(alloc_ozaki(c));
    c->have_fp64 = true;
    return PSDP_OK;
}

// The Ozaki slice buffers for the engines chosen now.
psdp_status alloc_ozaki(psdp_ctx* c) {
    // Ozaki slices: the Schur operands of one chunk of pairs (both sides), or one
    // outer Cholesky panel's rows, whichever is larger
    size_t sa = 0, sb = 0, ea = 0;
    if (c->oz_schur) {
        const int dpad = std::min(c->tpad, kOzakiMaxDepth);
        sa = sb = ozaki_slice_elems(c->n2, dpad, c->pairs_per_chunk);
        ea = (size_t)c->pairs_per_chunk * c->n2;
    }
    if (c->oz_chol) {
        // one outer panel's rows, double-buffered by panel parity (look-ahead),
        // and one inner panel's rows (depth 32) for the inner updates
        sa = std::max(sa, 2 * ozaki_slice_elems(c->K, kOzakiMaxDepth, 1));
        ea = std::max(ea, 2 * (size_t)c->K);
        // (and 32 more rows: L_jj^{-1} of the panel solve)
        if (!c->d_oz_si) TRY(dalloc(&c->d_oz_si, ozaki_slice_elems(c->K + 32, 32, 1)));
        if (!c->d_oz_ei) TRY(dalloc(&c->d_oz_ei, (size_t)c->K + 32));
        // and one 128-column block's rows (the block updates inside an outer panel)
        if (!c->d_oz_sm) TRY(dalloc(&c->d_oz_sm, ozaki_slice_elems(c->K, 128, 1)));
        if (!c->d_oz_em) TRY(dalloc(&c->d_oz_em, (size_t)c->K));
    }
    if (sa) {
        TRY(dalloc(&c->d_oz_sa, sa));
        TRY(dalloc(&c->d_oz_ea, ea));
    }
    if (sb) {
        TRY(dalloc(&c->d_oz_sb, sb));
        TRY(dalloc(&c->d_oz_eb, ea));
    }
    return PSDP_OK;
}

psdp_status realloc_ozaki(psdp_ctx* c) {
    if (!c->have_fp64) return PSDP_OK;     // alloc_fp64 sizes them when it runs
    cudaStreamSynchronize(c->stream);
    for (void* p : {(void*)c->d_oz_sa, (void*)c->d_oz_sb, (void*)c->d_oz_ea, (void*)c->d_oz_eb})
        if (p) cudaFree(p);
    c->d_oz_sa = c->d_oz_sb = nullptr;
    c->d_oz_ea = c->d_oz_eb = nullptr;
    return alloc_ozaki(c);
}

// Buffers of the mixed-precision step and the Schur operand tensor maps.
psdp_status alloc_mixed(psdp_ctx* c) {
    const size_t K = c->K, n2 = c->n2, np = std::max(1, c->nlyap_prod);
    const size_t opsz = (size_t)c->npairs * n2 * c->tpad;
    float** ops[] = {&c->d_opA_hi, &c->d_opA_lo, &c->d_opB_hi, &c->d_opB_lo};
    for (float** p : ops) {
        TRY(dalloc(p, opsz));
        cudaMemset(*p, 0, opsz * sizeof(float));   // padding terms stay zero
    }
    TRY(dalloc(&c->d_prodA, np * n2));
    TRY(dalloc(&c->d_prodB, np * n2));
    const size_t per_pair = n2 * n2 * sizeof(float);
    c->pairs_per_chunk32 = (int)std::max<size_t>(1, std::min<size_t>((size_t)c->npairs, ((size_t)2 << 30) / per_pair));
    TRY(dalloc(&c->d_T32, (size_t)c->pairs_per_chunk32 * n2 * n2));
    // sized for the widest panel the autotuner may pick (128), whatever nb32 is now
    const int nb = std::max(c->nb32, 128), npanel = (c->K + 63) / 64;
    TRY(dalloc(&c->d_Om32, K * K));
    TRY(dalloc(&c->d_Linv32, (size_t)npanel * 64 * 64 + (size_t)((c->K + 127) / 128) * 128 * 128));
    TRY(dalloc(&c->d_Pt_hi, 2 * K * kOuterPanels * nb));   // wide packed panel, double-buffered by outer parity
    TRY(dalloc(&c->d_Pt_lo, 2 * K * kOuterPanels * nb));
    TRY(dalloc(&c->d_Pk_hi, K * nb));
    TRY(dalloc(&c->d_Pk_lo, K * nb));
    TRY(dalloc(&c->d_Lt_hi, nb * nb));
    TRY(dalloc(&c->d_Lt_lo, nb * nb));
    TRY(dalloc(&c->d_z32, K));
    double** vecs[] = {&c->d_pcg_x, &c->d_pcg_r, &c->d_pcg_z, &c->d_pcg_p, &c->d_pcg_q};
    for (double** p : vecs) TRY(dalloc(p, K));
    TRY(dalloc(&c->d_pcg_state, 8));
    TRY(dalloc(&c->d_pcg_done, 1));
    TRY(dalloc(&c->d_M1, (size_t)c->nblk * n2));
    TRY(dalloc(&c->d_M2, (size_t)c->nblk * n2));
    // operands: element (t, e, pair) at pair*n2*tpad + e*tpad + t
    const bool ok = tc_make_map(&c->map_opA_hi, c->d_opA_hi, false, c->tpad, n2, c->npairs, c->tpad, n2 * c->tpad, 128) &&
                    tc_make_map(&c->map_opA_lo, c->d_opA_lo, false, c->tpad, n2, c->npairs, c->tpad, n2 * c->tpad, 128) &&
                    tc_make_map(&c->map_opB_hi, c->d_opB_hi, false, c->tpad, n2, c->npairs, c->tpad, n2 * c->tpad, 128) &&
                    tc_make_map(&c->map_opB_lo, c->d_opB_lo, false, c->tpad, n2, c->npairs, c->tpad, n2 * c->tpad, 128);
    return ok ? PSDP_OK : PSDP_ECUDA;
}

// Engines of the FP64 contractions.  Automatic: the Ozaki scheme where its
// 128 x 64 tiles are filled: the Cholesky from K >= kOzakiCholMinK (mid
// workload, K = 2100: 4.45 vs 6.64 ms a step), the Schur contraction from
// n >= 16 (n^2 >= 256 rows); DFMA below, where the step is latency-bound.
constexpr int kOzakiCholMinK = 1024;
bool choose_engine_chol(const psdp_ctx* c) {
    const int e = c->opt.fp64_gemm;
    return e == PSDP_GEMM_OZAKI || (e == PSDP_GEMM_AUTO && c->K >= kOzakiCholMinK);
}
bool choose_engine_schur(const psdp_ctx* c) {
    const int e = c->opt.fp64_gemm;
    return e == PSDP_GEMM_OZAKI || (e == PSDP_GEMM_AUTO && c->n2 >= 256);
}
void choose_fp64_engines(psdp_ctx* c) {
    c->oz_chol = choose_engine_chol(c);
    c->oz_schur = choose_engine_schur(c);
}

psdp_status setup_impl(int n, int l, int d_p, int d1, const double* A, const psdp_opts* o, psdp_ctx** out) {
    psdp_opts opt;
    psdp_default_opts(&opt);
    if (o) opt = *o;
    const int d2 = opt.d2 < 0 ? d1 : opt.d2;
    const int d_a = opt.d_a;
    if (n < 1 || n > PSDP_MAX_N || l < 1 || l > PSDP_MAX_L || d_p < 0 || d1 < 0 || d2 < 0 || d_a < 1 ||
        d_p > 12 || d1 > 12 || d2 > 12 || d_a > 12 || !A)
        return PSDP_EINVAL;
    if (!(opt.tau > 0 && opt.tau < 1) || !(opt.sigma >= 0 && opt.sigma < 1) || !(opt.eps > 0) || opt.max_iter < 1 ||
        !std::isfinite(opt.delta) || !std::isfinite(opt.delta_L) ||
        (opt.precision != PSDP_FP64 && opt.precision != PSDP_MIXED) || opt.crit_sms < 0 || opt.fp64_gemm < 0 ||
        opt.fp64_gemm > PSDP_GEMM_OZAKI)
        return PSDP_EINVAL;
    const int64_t Na = hcard(l, d_a), L0 = hcard(l, d_p), L = hcard(l, d_p + d1), M = hcard(l, d_p + d_a + d2);
    const int64_t Nt = (int64_t)n * (n + 1) / 2, K = L0 * Nt;
    if (K > 65536 || L + M > 100000 || L0 * M * Na > (1 << 26)) return PSDP_EINVAL;
    for (int64_t i = 0; i < Na * n * n; ++i)
        if (!std::isfinite(A[i])) return PSDP_EINVAL;
    if (cudaSetDevice(opt.device) != cudaSuccess) { cudaGetLastError(); return PSDP_ECUDA; }
    int smem_max = 0, num_sms = 0;
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, opt.device);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, opt.device);
    if ((size_t)2 * n * (n + 1) * sizeof(double) + 4 * n * sizeof(double) > (size_t)smem_max) return PSDP_EINVAL;
    init_attrs_linalg(smem_max);
    init_attrs_sdp(smem_max);
    init_attrs_dense(smem_max);
    init_attrs_tc(smem_max);
    init_attrs_mixed(smem_max);
    init_attrs_trsv(smem_max);
    init_attrs_ozaki(smem_max);
    cudaGetLastError();

    psdp_ctx* c = new (std::nothrow) psdp_ctx();
    if (!c) return PSDP_ENOMEM;
    c->n = n; c->l = l; c->d_p = d_p; c->d1 = d1; c->d2 = d2; c->d_a = d_a;
    c->L0 = (int)L0; c->L = (int)L; c->M = (int)M; c->Na = (int)Na; c->Nt = (int)Nt; c->K = (int)K;
    c->nblk = (int)(L + M); c->n2 = n * n;
    c->opt = opt;
    c->device = opt.device;
    c->num_sms = std::max(1, num_sms);
    c->mixed = opt.precision == PSDP_MIXED;
    c->flops_chol = (double)K * K * K / 3.0;
    if (opt.stream) {
        c->stream = (cudaStream_t)opt.stream;
        c->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { free_ctx(c); return PSDP_ECUDA; }
        c->own_stream = true;
    }
    {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (cudaStreamCreateWithPriority(&c->crit, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            free_ctx(c);
            return PSDP_ECUDA;
        }
    }
    psdp_status s = PSDP_OK;
    auto fail = [&](psdp_status e) { free_ctx(c); return e; };
    const size_t nbn2 = (size_t)c->nblk * c->n2;
    if ((s = dalloc(&c->d_beta, (size_t)L0 * L)) || (s = dalloc(&c->d_cH, (size_t)L0 * M * Na)) ||
        (s = dalloc(&c->d_W0, (size_t)L0 * l)) || (s = dalloc(&c->d_Wa, (size_t)Na * l)) ||
        (s = dalloc(&c->d_A, (size_t)Na * c->n2)) || (s = dalloc(&c->d_H, (size_t)L0 * M * c->n2)) ||
        (s = dalloc(&c->d_cdiag, c->nblk)))
        return fail(s);
    double** blocks[] = {&c->d_X, &c->d_Z, &c->d_G, &c->d_Y, &c->d_T1, &c->d_T2, &c->d_W, &c->d_F,
                         &c->d_dXh, &c->d_dZh, &c->d_dX, &c->d_dZ};
    for (double** p : blocks)
        if ((s = dalloc(p, nbn2))) return fail(s);
    if ((s = dalloc(&c->d_S, (size_t)M * Na * c->n2)) || (s = dalloc(&c->d_adj, (size_t)L0 * (Na + 1) * c->n2)) ||
        (s = dalloc(&c->d_adj2, (size_t)L0 * Na * c->n2)) || (s = dalloc(&c->d_adj_idx, (size_t)3 * L0 * Na)))
        return fail(s);
    {
        // product e = g Na + lambda of the adjoint: A_lambda x adj[g][lambda] -> adj2[g][lambda]
        std::vector<int32_t> ix((size_t)3 * L0 * Na);
        for (int g = 0; g < L0; ++g)
            for (int li = 0; li < Na; ++li) {
                const size_t e = (size_t)g * Na + li;
                ix[e] = li;
                ix[(size_t)L0 * Na + e] = g * (Na + 1) + li;
                ix[(size_t)2 * L0 * Na + e] = (int32_t)e;
            }
        cudaMemcpy(c->d_adj_idx, ix.data(), ix.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    }
    double** vecs[] = {&c->d_y, &c->d_dyh, &c->d_dyb, &c->d_BX};
    for (double** p : vecs)
        if ((s = dalloc(p, (size_t)K))) return fail(s);
    if ((s = dalloc(&c->d_part, (size_t)4 * (c->nblk + 1))) ||
        (s = dalloc(&c->d_tstep, (size_t)2 * c->nblk)) || (s = dalloc(&c->d_scal, SC_COUNT)) ||
        (s = dalloc(&c->d_info, PSDP_INFO_LEN)) || (s = dalloc(&c->d_flag, 1)) || (s = dalloc(&c->d_cert, 4)) ||
        (s = dalloc(&c->d_svec, (size_t)2 * Nt)) || (s = dalloc(&c->d_trsv_sync, trsv_sync_words((int)K, 32))))
        return fail(s);
    if (cudaMallocHost((void**)&c->h_info, PSDP_INFO_LEN * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_flag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(PSDP_ENOMEM);
    }
    cudaStream_t st = c->stream;
    cudaMemsetAsync(c->d_flag, 0, sizeof(int), st);
    cudaMemsetAsync(c->d_scal, 0, SC_COUNT * sizeof(double), st);
    cudaMemsetAsync(c->d_info, 0, PSDP_INFO_LEN * sizeof(double), st);
    cudaMemcpyAsync(c->d_A, A, (size_t)Na * c->n2 * sizeof(double), cudaMemcpyHostToDevice, st);
    launch_tables(st, l, d_p, d1, d2, d_a, c->L0, c->L, c->M, c->Na, c->d_beta, c->d_cH, c->d_W0, c->d_Wa);
    launch_cdiag(st, c);
    launch_hmat(st, c->L0, c->M, c->Na, n, c->d_cH, c->d_A, c->d_H);
    c->beta.resize((size_t)L0 * L);
    c->cH.resize((size_t)L0 * M * Na);
    c->cdiag.resize(c->nblk);
    cudaMemcpyAsync(c->beta.data(), c->d_beta, c->beta.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(c->cH.data(), c->d_cH, c->cH.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(c->cdiag.data(), c->d_cdiag, c->nblk * sizeof(double), cudaMemcpyDeviceToHost, st);
    if ((s = sync_check(c))) return fail(s);
    std::vector<int32_t> sv;
    for (int off = 0; off < n; ++off)
        for (int r = 0; r + off < n; ++r) { sv.push_back(r); sv.push_back(r + off); }
    cudaMemcpy(c->d_svec, sv.data(), sv.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if ((s = build_schur_lists(c))) return fail(s);
    choose_fp64_engines(c);
    if ((s = c->mixed ? alloc_mixed(c) : alloc_fp64(c))) return fail(s);
    launch_identity(st, c->nblk, n, c->d_X);
    launch_identity(st, c->nblk, n, c->d_Z);
    cudaMemsetAsync(c->d_y, 0, (size_t)K * sizeof(double), st);
    if ((s = refresh(c))) return fail(s);
    *out = c;
    return PSDP_OK;
}

// Capture (once) the Newton-step graph of the given precision.
psdp_status ensure_graph(psdp_ctx* c, bool mixed) {
    if (!mixed) TRY(alloc_fp64(c));
    cudaGraph_t& g = mixed ? c->graph32 : c->graph;
    cudaGraphExec_t& ge = mixed ? c->graph_exec32 : c->graph_exec;
    bool& have = mixed ? c->have_graph32 : c->have_graph;
    if (!have) {
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PSDP_ECUDA;
        enqueue_step(c, mixed);
        if (cudaStreamEndCapture(c->stream, &g) != cudaSuccess) { cudaGetLastError(); return PSDP_ECUDA; }
        if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) { cudaGetLastError(); return PSDP_ECUDA; }
        have = true;
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
        int nk = 0;
        for (size_t i = 0; i < nn; ++i) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++nk;
        }
        c->kernels_per_step = nk;
    }
    return PSDP_OK;
}

// Launch one Newton step of the given precision on the context's stream.
psdp_status launch_step(psdp_ctx* c, bool mixed) {
    if (!c->opt.use_graph) {
        if (!mixed) TRY(alloc_fp64(c));
        enqueue_step(c, mixed);
        return PSDP_OK;
    }
    TRY(ensure_graph(c, mixed));
    if (cudaGraphLaunch(mixed ? c->graph_exec32 : c->graph_exec, c->stream) != cudaSuccess) return PSDP_ECUDA;
    return PSDP_OK;
}

// After a step of the given precision completed: FP64 fallback of a missed
// mixed step, flag -> status, info for the caller.
psdp_status finish_step(psdp_ctx* c, bool mixed, double* info) {
    prof_collect(c, mixed);
    int flag = *c->h_flag;
    if (mixed && (flag & (FL_MIXED | FL_CHOL_SCHUR)) && !(flag & (FL_CHOL_BLOCK | FL_TIMEOUT))) {
        // The mixed-precision direction missed its residual target (the iterate
        // was left untouched): take this and all later steps in FP64.
        c->mixed_failed = true;
        cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream);
        TRY(launch_step(c, false));
        TRY(sync_check(c));
        prof_collect(c, false);
        flag = *c->h_flag;
    }
    c->h_info[11] = (double)(c->iters + 1);
    c->h_info[13] = (c->mixed && c->mixed_failed) ? 1.0 : 0.0;
    if (flag) {
        cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream);
        TRY(sync_check(c));
        if (info) memcpy(info, c->h_info, PSDP_INFO_LEN * sizeof(double));
        if (flag & FL_CHOL_BLOCK) return PSDP_ECHOL_BLOCK;
        if (flag & FL_CHOL_SCHUR) return PSDP_ECHOL_SCHUR;
        if (flag & FL_TIMEOUT) return PSDP_ETIMEOUT;
        return PSDP_ENAN;
    }
    c->iters += 1;
    if (info) memcpy(info, c->h_info, PSDP_INFO_LEN * sizeof(double));
    return PSDP_OK;
}

psdp_status step_impl(psdp_ctx* c, double* info) {
    cudaSetDevice(c->device);
    const bool mixed = c->mixed && !c->mixed_failed;
    TRY(launch_step(c, mixed));
    TRY(sync_check(c));
    return finish_step(c, mixed, info);
}

// Stopping rule after a successful step: PSDP_OK when the relative gap and both
// relative residuals are <= eps, PSDP_EUNBOUNDED on a primal ray, else
// PSDP_ESTATE meaning "keep iterating".
psdp_status converged(const psdp_ctx* c, const double* inf) {
    const double eps = c->opt.eps;
    if (inf[2] <= eps && inf[3] <= eps && inf[4] <= eps) return PSDP_OK;
    const double trX = inf[9];
    if (trX > 1e8 && inf[10] / trX < 1e-6 && inf[0] / trX > 1e-8) return PSDP_EUNBOUNDED;
    return PSDP_ESTATE;
}

void invalidate_graph(psdp_ctx* c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->graph_exec32) cudaGraphExecDestroy(c->graph_exec32);
    if (c->graph32) cudaGraphDestroy(c->graph32);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_exec32 = nullptr;
    c->graph32 = nullptr;
    c->have_graph = false;
    c->have_graph32 = false;
}

// The cold start X = Z = I, y = 0 (Algorithm 2) with the current problem data.
psdp_status reset_to_cold_start(psdp_ctx* c) {
    cudaStream_t st = c->stream;
    launch_identity(st, c->nblk, c->n, c->d_X);
    launch_identity(st, c->nblk, c->n, c->d_Z);
    cudaMemsetAsync(c->d_y, 0, (size_t)c->K * sizeof(double), st);
    cudaMemsetAsync(c->d_flag, 0, sizeof(int), st);
    c->iters = 0;
    c->mixed_failed = false;
    return refresh(c);
}

}  // namespace

// ======================================================================= ABI
extern "C" {

void psdp_default_opts(psdp_opts* o) {
    if (!o) return;
    o->delta = 1.0;
    o->delta_L = 0.0;
    o->eps = 1e-7;
    o->sigma = 1.0 / 3.0;
    o->tau = 0.95;
    o->max_iter = 100;
    o->d2 = -1;
    o->d_a = 1;
    o->precision = PSDP_FP64;
    o->use_graph = 1;
    o->stream = nullptr;
    o->device = 0;
    o->crit_sms = 0;
    o->fp64_gemm = PSDP_GEMM_AUTO;
}

psdp_status psdp_setup(int n, int l, int d_p, int d1, const double* A, const psdp_opts* o, psdp_ctx** out) {
    if (!out) return PSDP_EINVAL;
    *out = nullptr;
    try {
        return setup_impl(n, l, d_p, d1, A, o, out);
    } catch (...) {
        return PSDP_ENOMEM;
    }
}

psdp_status psdp_sizes(const psdp_ctx* c, int32_t* o) {
    if (!c || !o) return PSDP_EINVAL;
    const int32_t v[9] = {c->n, c->l, c->L0, c->L, c->M, c->Nt, c->K, c->nblk, c->Na};
    memcpy(o, v, sizeof(v));
    return PSDP_OK;
}

psdp_status psdp_step(psdp_ctx* c, double* info) {
    if (!c) return PSDP_EINVAL;
    try {
        return step_impl(c, info);
    } catch (...) {
        return PSDP_ENOMEM;
    }
}

psdp_status psdp_solve(psdp_ctx* c, int* iters, double* info) {
    if (!c) return PSDP_EINVAL;
    double inf[PSDP_INFO_LEN];
    psdp_status s = PSDP_EMAXITER;
    int it = 0;
    for (; it < c->opt.max_iter; ++it) {
        psdp_status r = psdp_step(c, inf);
        if (r == PSDP_OK) r = converged(c, inf);
        if (r != PSDP_ESTATE) {
            s = r;
            ++it;
            break;
        }
    }
    if (iters) *iters = it;
    if (info) memcpy(info, c->h_info, PSDP_INFO_LEN * sizeof(double));
    return s;
}

psdp_status psdp_solve_batch(psdp_ctx** v, int count, psdp_status* status, int* iters) {
    if (!v || count < 1) return PSDP_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!v[i] || v[i]->device != v[0]->device || !v[i]->opt.use_graph || v[i]->prof_on) return PSDP_EINVAL;
        for (int j = 0; j < i; ++j)
            if (v[j] == v[i]) return PSDP_EINVAL;
    }
    try {
        cudaSetDevice(v[0]->device);
        std::vector<psdp_status> st(count, PSDP_EMAXITER);
        std::vector<int> it(count, 0), built;
        std::vector<char> done(count, 0), frozen(count, 0);
        cudaStream_t bs;
        if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) return PSDP_ECUDA;
        cudaGraphExec_t exec = nullptr;
        const int frozen_flag = FL_FROZEN;
        psdp_status err = PSDP_OK;
        int remaining = count;
        bool rebuild = true;
        // a finished instance's branch keeps running (frozen) until the graph is
        // rebuilt: rebuild once the step work of the frozen branches, at the measured
        // time of an iteration, costs more than half a measured rebuild
        auto work = [&](int i) { return v[i]->flops_chol + v[i]->flops_schur + 1.0; };
        double t_build = 0.0, t_iter = 0.0;
        while (remaining > 0 && err == PSDP_OK) {
            if (rebuild) {
                const auto b0 = std::chrono::steady_clock::now();
                // one graph whose branches are the step graphs of all unfinished instances
                if (exec) cudaGraphExecDestroy(exec);
                exec = nullptr;
                built.clear();
                cudaGraph_t parent;
                cudaGraphCreate(&parent, 0);
                for (int i = 0; i < count && err == PSDP_OK; ++i) {
                    if (done[i]) continue;
                    psdp_ctx* c = v[i];
                    const bool mixed = c->mixed && !c->mixed_failed;
                    if ((err = ensure_graph(c, mixed)) != PSDP_OK) break;
                    cudaGraphNode_t node;
                    if (cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, mixed ? c->graph32 : c->graph) !=
                        cudaSuccess)
                        err = PSDP_ECUDA;
                    built.push_back(i);
                }
                if (err == PSDP_OK && cudaGraphInstantiate(&exec, parent, 0) != cudaSuccess) err = PSDP_ECUDA;
                cudaGraphDestroy(parent);
                if (err != PSDP_OK) break;
                for (int i : built) frozen[i] = 0;
                rebuild = false;
                t_build = std::chrono::duration<double>(std::chrono::steady_clock::now() - b0).count();
            }
            const auto l0 = std::chrono::steady_clock::now();
            if (cudaGraphLaunch(exec, bs) != cudaSuccess || cudaStreamSynchronize(bs) != cudaSuccess) {
                err = PSDP_ECUDA;
                break;
            }
            t_iter = std::chrono::duration<double>(std::chrono::steady_clock::now() - l0).count();
            for (int i : built) {
                if (frozen[i]) continue;
                psdp_ctx* c = v[i];
                const bool mixed = c->mixed && !c->mixed_failed;
                double inf[PSDP_INFO_LEN];
                psdp_status r = finish_step(c, mixed, inf);
                if (mixed && c->mixed_failed) rebuild = true;       // its graph branch changed precision
                ++it[i];
                if (r == PSDP_OK) r = converged(c, inf);
                if (r == PSDP_ESTATE && it[i] >= c->opt.max_iter) r = PSDP_EMAXITER;
                if (r != PSDP_ESTATE) {
                    st[i] = r;
                    done[i] = 1;
                    frozen[i] = 1;
                    --remaining;
                    // a frozen instance keeps running inside the graph until the next
                    // rebuild, but its update kernel sees the flag and leaves the iterate
                    cudaMemcpyAsync(c->d_flag, &frozen_flag, sizeof(int), cudaMemcpyHostToDevice, c->stream);
                    cudaStreamSynchronize(c->stream);
                }
            }
            double w_all = 0.0, w_frozen = 0.0;
            for (int i : built) {
                w_all += work(i);
                if (frozen[i]) w_frozen += work(i);
            }
            if (w_frozen / w_all * t_iter >= 0.5 * t_build) rebuild = true;
        }
        if (exec) cudaGraphExecDestroy(exec);
        for (int i = 0; i < count; ++i) {
            cudaMemsetAsync(v[i]->d_flag, 0, sizeof(int), v[i]->stream);
            cudaStreamSynchronize(v[i]->stream);
            if (status) status[i] = st[i];
            if (iters) iters[i] = it[i];
        }
        cudaStreamDestroy(bs);
        cudaGetLastError();
        return err;
    } catch (...) {
        return PSDP_ENOMEM;
    }
}

// Apply candidate `cand` of psdp_autotune_ex to the context (buffers allocated on first need).
psdp_status apply_tune_candidate(psdp_ctx* c, int cand) {
    const bool mixed = cand == 1 || cand == 2;
    if (mixed && !c->d_Om32) TRY(alloc_mixed(c));
    if (!mixed) {
        const bool oz_s = cand == 4 || cand == 5 || (cand == 0 && choose_engine_schur(c));
        const bool oz_c = cand == 4 || (cand == 0 && choose_engine_chol(c));
        if ((oz_s && !c->oz_schur) || (oz_c && !c->oz_chol)) {
            // the Ozaki slice buffers are sized at allocation: redo them for the new engines
            c->oz_schur = oz_s;
            c->oz_chol = oz_c;
            TRY(realloc_ozaki(c));
        }
        c->oz_schur = oz_s;
        c->oz_chol = oz_c;
        TRY(alloc_fp64(c));
    }
    c->mixed = mixed;
    c->mixed_failed = false;
    if (mixed) c->nb32 = (cand == 1) ? 64 : 128;
    invalidate_graph(c);
    return PSDP_OK;
}

psdp_status psdp_autotune_ex(psdp_ctx* c, const char* cache_path, unsigned mask, int* choice, double* ms_out) {
    if (!c || (mask & ((1u << PSDP_TUNE_CANDIDATES) - 1)) == 0) return PSDP_EINVAL;
    cudaSetDevice(c->device);
    mask &= (1u << PSDP_TUNE_CANDIDATES) - 1;
    char key[160];
    snprintf(key, sizeof key, "n=%d l=%d d_p=%d d1=%d d2=%d d_a=%d mask=%u", c->n, c->l, c->d_p, c->d1, c->d2, c->d_a,
             mask);
    int best = -1;
    double ms[PSDP_TUNE_CANDIDATES];
    for (double& m : ms) m = -1.0;
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            char line[512];
            while (fgets(line, sizeof line, f)) {
                int ch = -1;
                double t[PSDP_TUNE_CANDIDATES];
                char* bar = strchr(line, '|');
                if (bar && (size_t)(bar - line) == strlen(key) && strncmp(line, key, strlen(key)) == 0 &&
                    sscanf(bar + 1, "%d %lf %lf %lf %lf %lf %lf", &ch, &t[0], &t[1], &t[2], &t[3], &t[4], &t[5]) ==
                        1 + PSDP_TUNE_CANDIDATES &&
                    ch >= 0 && ch < PSDP_TUNE_CANDIDATES && ((mask >> ch) & 1u)) {
                    best = ch;
                    memcpy(ms, t, sizeof ms);
                }
            }
            fclose(f);
        }
    }
    if (best < 0) {
        // time one Newton step per candidate from the current iterate, which is restored after each
        const size_t nb = (size_t)c->nblk * c->n2;
        std::vector<double> X(nb), Z(nb), y(c->K);
        TRY(psdp_get_iterate(c, X.data(), Z.data(), y.data()));
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        for (int cand = 0; cand < PSDP_TUNE_CANDIDATES; ++cand) {
            if (!((mask >> cand) & 1u)) continue;
            TRY(apply_tune_candidate(c, cand));
            float total = 0.f;
            for (int rep = 0; rep < 2; ++rep) {
                TRY(psdp_load_iterate(c, X.data(), Z.data(), y.data()));
                cudaEventRecord(a, c->stream);
                TRY(launch_step(c, c->mixed));
                cudaEventRecord(b, c->stream);
                TRY(sync_check(c));
                cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream);
                float t = 0.f;
                cudaEventElapsedTime(&t, a, b);
                if (rep == 1) total = t;   // the first repetition captures the graph
            }
            ms[cand] = total;
            if (best < 0 || ms[cand] < ms[best]) best = cand;
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        TRY(psdp_load_iterate(c, X.data(), Z.data(), y.data()));
        if (cache_path) {
            if (FILE* f = fopen(cache_path, "a")) {
                fprintf(f, "%s|%d", key, best);
                for (double m : ms) fprintf(f, " %.4f", m);
                fprintf(f, "\n");
                fclose(f);
            }
        }
    }
    TRY(apply_tune_candidate(c, best));
    if (choice) *choice = best;
    if (ms_out) memcpy(ms_out, ms, sizeof ms);
    return PSDP_OK;
}

psdp_status psdp_autotune(psdp_ctx* c, const char* cache_path, int* choice, double* ms_out) {
    double ms[PSDP_TUNE_CANDIDATES];
    const psdp_status s = psdp_autotune_ex(c, cache_path, 7u, choice, ms);
    if (s == PSDP_OK && ms_out) memcpy(ms_out, ms, 3 * sizeof(double));
    return s;
}

psdp_status psdp_certify(psdp_ctx* c, int* verdict, double* minP, double* maxL) {
    if (!c) return PSDP_EINVAL;
    cudaSetDevice(c->device);
    cudaStream_t st = c->stream;
    launch_bt(st, c, c->d_y, c->d_T1);
    launch_sub_CR(st, c, c->d_T1);    // Lyapunov coefficients -(A^T P + P A + R)
    launch_block_mineig(st, c->nblk, c->n, c->d_T1, 1.0, c->d_tstep);
    launch_certify_finalize(st, c->nblk, c->n, c->d_tstep, c->L, c->d_cert);
    double h[3];
    cudaMemcpyAsync(h, c->d_cert, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
    TRY(sync_check(c));
    if (verdict) *verdict = (int)h[0];
    if (minP) *minP = h[1];
    if (maxL) *maxL = h[2];
    return PSDP_OK;
}

psdp_status psdp_grid_check(psdp_ctx* c, int N, double* minP, double* maxQ) {
    if (!c || N < 1 || N > 4096) return PSDP_EINVAL;
    cudaSetDevice(c->device);
    const int64_t total = hcard(c->l, N);
    const int chunk = (int)std::min<int64_t>(total, 2048);
    const size_t need = (size_t)3 * chunk * c->n2 + (size_t)4 * chunk;
    if (c->grid_cap < need) {
        if (c->d_grid) cudaFree(c->d_grid);
        c->d_grid = nullptr;
        c->grid_cap = 0;
        TRY(dalloc(&c->d_grid, need));
        c->grid_cap = need;
    }
    double* P = c->d_grid;
    double* Aal = P + (size_t)chunk * c->n2;
    double* Q = Aal + (size_t)chunk * c->n2;
    double* eig = Q + (size_t)chunk * c->n2;
    std::vector<double> h((size_t)4 * chunk);
    double mp = 1e300, mq = -1e300;
    cudaStream_t st = c->stream;
    for (int64_t first = 0; first < total; first += chunk) {
        const int cnt = (int)std::min<int64_t>(chunk, total - first);
        launch_grid_build(st, c, N, first, cnt, P, Aal);
        launch_bgemm(st, c->n, cnt, Aal, nullptr, 1, 1, P, nullptr, 1, 0, Q, nullptr, 1, 0, 1.0, 0.0);
        launch_bgemm(st, c->n, cnt, P, nullptr, 1, 0, Aal, nullptr, 1, 0, Q, nullptr, 1, 0, 1.0, 1.0);
        launch_grid_addR(st, c, N, first, cnt, Q);
        launch_block_mineig(st, cnt, c->n, P, 1.0, eig);
        launch_block_mineig(st, cnt, c->n, Q, -1.0, eig + 2 * chunk);
        cudaMemcpyAsync(h.data(), eig, (size_t)4 * chunk * sizeof(double), cudaMemcpyDeviceToHost, st);
        TRY(sync_check(c));
        for (int i = 0; i < cnt; ++i) {
            mp = std::min(mp, h[2 * i]);
            mq = std::max(mq, -h[2 * chunk + 2 * i]);
        }
    }
    if (minP) *minP = mp;
    if (maxQ) *maxQ = mq;
    return PSDP_OK;
}

psdp_status psdp_get_P(psdp_ctx* c, double* P) {
    if (!c || !P) return PSDP_EINVAL;
    std::vector<double> y(c->K);
    TRY(psdp_get_y(c, y.data()));
    const int n = c->n;
    for (int h = 0; h < c->L0; ++h) {
        int q = 0;
        for (int off = 0; off < n; ++off)
            for (int r = 0; r + off < n; ++r, ++q) {
                const double v = y[(size_t)h * c->Nt + q];
                P[((size_t)h * n + r) * n + r + off] = v;
                P[((size_t)h * n + r + off) * n + r] = v;
            }
    }
    return PSDP_OK;
}

psdp_status psdp_get_y(psdp_ctx* c, double* y) {
    if (!c || !y) return PSDP_EINVAL;
    cudaSetDevice(c->device);
    cudaMemcpyAsync(y, c->d_y, (size_t)c->K * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    return sync_check(c);
}

psdp_status psdp_get_tables(psdp_ctx* c, int32_t* beta, int32_t* cH) {
    if (!c) return PSDP_EINVAL;
    if (beta) memcpy(beta, c->beta.data(), c->beta.size() * sizeof(int32_t));
    if (cH) memcpy(cH, c->cH.data(), c->cH.size() * sizeof(int32_t));
    return PSDP_OK;
}

psdp_status psdp_load_iterate(psdp_ctx* c, const double* X, const double* Z, const double* y) {
    if (!c || !X || !Z || !y) return PSDP_EINVAL;
    cudaSetDevice(c->device);
    const size_t nb = (size_t)c->nblk * c->n2 * sizeof(double);
    cudaMemcpyAsync(c->d_X, X, nb, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_Z, Z, nb, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_y, y, (size_t)c->K * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    return refresh(c);
}

psdp_status psdp_set_start(psdp_ctx* c, const double* y0, const double* xscale, double theta) {
    if (!c || !y0 || !(theta > 0.0) || !std::isfinite(theta)) return PSDP_EINVAL;
    for (int k = 0; k < c->K; ++k)
        if (!std::isfinite(y0[k])) return PSDP_EINVAL;
    if (xscale)
        for (int g = 0; g < c->nblk; ++g)
            if (!(xscale[g] > 0.0) || !std::isfinite(xscale[g])) return PSDP_EINVAL;
    cudaSetDevice(c->device);
    cudaStream_t st = c->stream;
    cudaMemcpyAsync(c->d_y, y0, (size_t)c->K * sizeof(double), cudaMemcpyHostToDevice, st);
    if (xscale) cudaMemcpyAsync(c->d_tstep, xscale, (size_t)c->nblk * sizeof(double), cudaMemcpyHostToDevice, st);
    launch_bt(st, c, c->d_y, c->d_T1);
    launch_sub_CR(st, c, c->d_T1);    // B^T(y0) - C with the constant term's part of C
    launch_block_mineig(st, c->nblk, c->n, c->d_T1, 1.0, c->d_part);
    launch_start_fix(st, c, c->d_T1, c->d_part, xscale ? c->d_tstep : nullptr, theta);
    c->iters = 0;
    c->mixed_failed = false;
    return refresh(c);
}

psdp_status psdp_set_constant_term(psdp_ctx* c, int d_r, const double* R) {
    if (!c || !R || d_r < 0 || d_r > c->d_p + c->d_a + c->d2) return PSDP_EINVAL;
    const int l = c->l, n = c->n;
    const int64_t Nr = hcard(l, d_r);
    const size_t n2 = (size_t)c->n2;
    for (size_t i = 0; i < (size_t)Nr * n2; ++i)
        if (!std::isfinite(R[i])) return PSDP_EINVAL;
    for (int64_t r = 0; r < Nr; ++r)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < i; ++j)
                if (R[r * n2 + (size_t)i * n + j] != R[r * n2 + (size_t)j * n + i]) return PSDP_EINVAL;
    cudaSetDevice(c->device);
    // exponents of W_{d_r} (lexicographic, (d_r, 0, ..., 0) first) and the
    // Lyapunov blocks' coefficients sum_rho multinomial(e; gamma - rho) R_rho,
    // e = d_p + d_a + d2 - d_r, formed on the host once
    std::vector<std::vector<int>> Wr, Wg;
    auto enumerate = [&](int d, std::vector<std::vector<int>>& out) {
        std::vector<int> g(l, 0);
        std::function<void(int, int)> rec = [&](int pos, int left) {
            if (pos == l - 1) {
                g[pos] = left;
                out.push_back(g);
                return;
            }
            for (int v = left; v >= 0; --v) {
                g[pos] = v;
                rec(pos + 1, left - v);
            }
        };
        rec(0, d);
    };
    enumerate(d_r, Wr);
    enumerate(c->d_p + c->d_a + c->d2, Wg);
    if ((int64_t)Wr.size() != Nr || (int)Wg.size() != c->M) return PSDP_EINVAL;
    const int e = c->d_p + c->d_a + c->d2 - d_r;
    std::vector<double> lf(64, 0.0);
    for (int k = 1; k < 64; ++k) lf[k] = lf[k - 1] + std::log((double)k);
    std::vector<double> CR((size_t)c->M * n2, 0.0);
    double c2 = 0.0;
    for (int gi = 0; gi < c->M; ++gi) {
        double* Cg = CR.data() + (size_t)gi * n2;
        for (int64_t r = 0; r < Nr; ++r) {
            bool ok = true;
            double lm = lf[e];
            for (int k = 0; k < l; ++k) {
                const int dk = Wg[gi][k] - Wr[r][k];
                if (dk < 0) ok = false;
                else lm -= lf[dk];
            }
            if (!ok) continue;
            const double m = std::round(std::exp(lm));    // multinomial(e; gamma - rho), an integer
            for (size_t t = 0; t < n2; ++t) Cg[t] += m * R[r * n2 + t];
        }
        const double cd = c->cdiag[c->L + gi];
        for (size_t t = 0; t < n2; ++t) c2 += Cg[t] * Cg[t];
        for (int i = 0; i < n; ++i) c2 += 2.0 * cd * Cg[(size_t)i * n + i];
    }
    std::vector<int32_t> wr((size_t)Nr * l);
    for (int64_t r = 0; r < Nr; ++r)
        for (int k = 0; k < l; ++k) wr[(size_t)r * l + k] = Wr[r][k];
    if (!c->d_CR) TRY(dalloc(&c->d_CR, (size_t)c->M * n2));
    if (c->d_R) cudaFree(c->d_R);
    if (c->d_Wr) cudaFree(c->d_Wr);
    c->d_R = nullptr;
    c->d_Wr = nullptr;
    TRY(dalloc(&c->d_R, (size_t)Nr * n2));
    TRY(dalloc(&c->d_Wr, (size_t)Nr * l));
    cudaMemcpy(c->d_CR, CR.data(), CR.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_R, R, (size_t)Nr * n2 * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_Wr, wr.data(), wr.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    c->d_r = d_r;
    c->Nr = (int)Nr;
    c->c2_extra = c2;
    invalidate_graph(c);
    return reset_to_cold_start(c);
}

psdp_status psdp_set_objective(psdp_ctx* c, const double* a) {
    if (!c || !a) return PSDP_EINVAL;
    double s = 0.0;
    for (int k = 0; k < c->K; ++k) {
        if (!std::isfinite(a[k])) return PSDP_EINVAL;
        s += a[k] * a[k];
    }
    cudaSetDevice(c->device);
    if (!c->d_avec) TRY(dalloc(&c->d_avec, (size_t)c->K));
    cudaMemcpy(c->d_avec, a, (size_t)c->K * sizeof(double), cudaMemcpyHostToDevice);
    c->a_norm = std::sqrt(s);
    invalidate_graph(c);
    return reset_to_cold_start(c);
}

psdp_status psdp_get_iterate(psdp_ctx* c, double* X, double* Z, double* y) {
    if (!c) return PSDP_EINVAL;
    cudaSetDevice(c->device);
    const size_t nb = (size_t)c->nblk * c->n2 * sizeof(double);
    if (X) cudaMemcpyAsync(X, c->d_X, nb, cudaMemcpyDeviceToHost, c->stream);
    if (Z) cudaMemcpyAsync(Z, c->d_Z, nb, cudaMemcpyDeviceToHost, c->stream);
    if (y) cudaMemcpyAsync(y, c->d_y, (size_t)c->K * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    return sync_check(c);
}

psdp_status psdp_get_schur_mixed(psdp_ctx* c, float* Om) {
    if (!c || !Om) return PSDP_EINVAL;
    if (!c->mixed) return PSDP_ESTATE;
    cudaSetDevice(c->device);
    cudaStream_t st = c->stream;
    cudaMemsetAsync(c->d_flag, 0, sizeof(int), st);
    launch_block_chol_inv(st, c->nblk, c->n, c->d_Z, c->d_Y, c->d_flag);
    const bool on = c->prof_on;
    c->prof_on = false;
    enqueue_schur_mixed(c);
    c->prof_on = on;
    int flag = 0;
    cudaMemcpyAsync(Om, c->d_Om32, (size_t)c->K * c->K * sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    TRY(sync_check(c));
    if (flag) {
        cudaMemsetAsync(c->d_flag, 0, sizeof(int), st);
        sync_check(c);
        return (flag & FL_TIMEOUT) ? PSDP_ETIMEOUT : PSDP_ECHOL_BLOCK;
    }
    const size_t K = c->K;
    for (size_t i = 0; i < K; ++i)
        for (size_t j = 0; j < i; ++j) Om[i * K + j] = Om[j * K + i];
    return PSDP_OK;
}

psdp_status psdp_get_schur(psdp_ctx* c, double* Om) {
    if (!c || !Om) return PSDP_EINVAL;
    cudaSetDevice(c->device);
    TRY(alloc_fp64(c));
    cudaStream_t st = c->stream;
    cudaMemsetAsync(c->d_flag, 0, sizeof(int), st);
    launch_block_chol_inv(st, c->nblk, c->n, c->d_Z, c->d_Y, c->d_flag);
    const bool on = c->prof_on;
    c->prof_on = false;
    enqueue_schur(c);
    c->prof_on = on;
    int flag = 0;
    cudaMemcpyAsync(Om, c->d_Om, (size_t)c->K * c->K * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    TRY(sync_check(c));
    if (flag) {
        cudaMemsetAsync(c->d_flag, 0, sizeof(int), st);
        sync_check(c);
        return PSDP_ECHOL_BLOCK;
    }
    const size_t K = c->K;
    for (size_t i = 0; i < K; ++i)
        for (size_t j = 0; j < i; ++j) Om[i * K + j] = Om[j * K + i];
    return PSDP_OK;
}

psdp_status psdp_get_schur_cols(psdp_ctx* c, const int32_t* cols, int ncols, double* out) {
    if (!c || !cols || !out || ncols < 0) return PSDP_EINVAL;
    for (int q = 0; q < ncols; ++q)
        if (cols[q] < 0 || cols[q] >= c->K) return PSDP_EINVAL;
    cudaSetDevice(c->device);
    TRY(alloc_fp64(c));
    cudaStream_t st = c->stream;
    cudaMemsetAsync(c->d_flag, 0, sizeof(int), st);
    launch_block_chol_inv(st, c->nblk, c->n, c->d_Z, c->d_Y, c->d_flag);
    const bool on = c->prof_on;
    c->prof_on = false;
    enqueue_schur(c);
    c->prof_on = on;
    // Omega is row-major with its upper triangle filled: column j holds
    // Omega[i][j] (i < j) in rows above j and Omega[j][i] (i >= j) in row j
    const size_t K = c->K;
    for (int q = 0; q < ncols; ++q) {
        const size_t j = cols[q];
        double* o = out + (size_t)q * K;
        if (j > 0)
            cudaMemcpy2DAsync(o, sizeof(double), c->d_Om + j, K * sizeof(double), sizeof(double), j,
                              cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(o + j, c->d_Om + j * K + j, (K - j) * sizeof(double), cudaMemcpyDeviceToHost, st);
    }
    int flag = 0;
    cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    TRY(sync_check(c));
    if (flag) {
        cudaMemsetAsync(c->d_flag, 0, sizeof(int), st);
        sync_check(c);
        return PSDP_ECHOL_BLOCK;
    }
    return PSDP_OK;
}

psdp_status psdp_apply_BT(psdp_ctx* c, const double* v, double* out) {
    if (!c || !v || !out) return PSDP_EINVAL;
    cudaSetDevice(c->device);
    cudaStream_t st = c->stream;
    cudaMemcpyAsync(c->d_dyb, v, (size_t)c->K * sizeof(double), cudaMemcpyHostToDevice, st);
    launch_bt(st, c, c->d_dyb, c->d_T1);
    cudaMemcpyAsync(out, c->d_T1, (size_t)c->nblk * c->n2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    return sync_check(c);
}

psdp_status psdp_apply_B(psdp_ctx* c, const double* W, double* out) {
    if (!c || !W || !out) return PSDP_EINVAL;
    cudaSetDevice(c->device);
    cudaStream_t st = c->stream;
    cudaMemcpyAsync(c->d_T1, W, (size_t)c->nblk * c->n2 * sizeof(double), cudaMemcpyHostToDevice, st);
    launch_b(st, c, c->d_T1, c->d_dyb, 0.0);
    cudaMemcpyAsync(out, c->d_dyb, (size_t)c->K * sizeof(double), cudaMemcpyDeviceToHost, st);
    return sync_check(c);
}

psdp_status psdp_profile_enable(psdp_ctx* c, int on) {
    if (!c) return PSDP_EINVAL;
    cudaSetDevice(c->device);
    if (on && c->prof_pool.empty()) {
        // two halves (FP64 and mixed step graphs), each with an event pair for up
        // to four timed launches per 32-column panel plus the step's other sites
        const size_t sites = 4 * (size_t)((c->K + 31) / 32) + 512;
        c->prof_pool.resize(std::max<size_t>(8192, 4 * sites));
        for (auto& e : c->prof_pool)
            if (cudaEventCreate(&e) != cudaSuccess) return PSDP_ECUDA;
    }
    if ((bool)on != c->prof_on) invalidate_graph(c);
    c->prof_on = on != 0;
    return PSDP_OK;
}

psdp_status psdp_profile_reset(psdp_ctx* c) {
    if (!c) return PSDP_EINVAL;
    std::fill(c->prof_launches.begin(), c->prof_launches.end(), 0);
    std::fill(c->prof_ms.begin(), c->prof_ms.end(), 0.0);
    return PSDP_OK;
}

psdp_status psdp_profile_get(psdp_ctx* c, int max_entries, char* names, int64_t* launches, double* ms, int* count) {
    if (!c || !count) return PSDP_EINVAL;
    const int nn = std::min<int>(max_entries, (int)c->prof_names.size());
    for (int i = 0; i < nn; ++i) {
        if (names) {
            memset(names + 32 * i, 0, 32);
            strncpy(names + 32 * i, c->prof_names[i].c_str(), 31);
        }
        if (launches) launches[i] = c->prof_launches[i];
        if (ms) ms[i] = c->prof_ms[i];
    }
    *count = nn;
    return PSDP_OK;
}

psdp_status psdp_profile_trace(psdp_ctx* c, int max_entries, int* name_ids, double* t0_ms, double* t1_ms,
                               int* on_crit, int* count) {
    if (!c || !count || max_entries < 0) return PSDP_EINVAL;
    const int nn = std::min<int>(max_entries, (int)c->prof_tr_id.size());
    for (int i = 0; i < nn; ++i) {
        if (name_ids) name_ids[i] = c->prof_tr_id[i];
        if (t0_ms) t0_ms[i] = c->prof_tr_t0[i];
        if (t1_ms) t1_ms[i] = c->prof_tr_t1[i];
        if (on_crit) on_crit[i] = c->prof_tr_crit[i];
    }
    *count = nn;
    return PSDP_OK;
}

psdp_status psdp_work(const psdp_ctx* c, double* out) {
    if (!c || !out) return PSDP_EINVAL;
    out[0] = c->flops_schur;
    out[1] = c->flops_chol;
    out[2] = (double)c->nterms;
    out[3] = c->flops_schur_dense;
    out[4] = (double)c->kernels_per_step;
    out[5] = (double)c->nb_chol;
    out[6] = (double)c->nb32;
    return PSDP_OK;
}

void* psdp_stream(psdp_ctx* c) { return c ? (void*)c->stream : nullptr; }

psdp_status psdp_fp64_peak(int device, double* tflops) {
    if (!tflops) return PSDP_EINVAL;
    const double v = fp64_peak_probe(device);
    if (v <= 0) return PSDP_ECUDA;
    *tflops = v;
    return PSDP_OK;
}

psdp_status psdp_engines(const psdp_ctx* c, int32_t* out) {
    if (!c || !out) return PSDP_EINVAL;
    out[0] = c->oz_schur ? 1 : 0;
    out[1] = c->oz_chol ? 1 : 0;
    return PSDP_OK;
}

psdp_status psdp_fp64_peaks(int device, double* dfma_tflops, double* dmma_tflops) {
    if (!dfma_tflops || !dmma_tflops) return PSDP_EINVAL;
    const double v = fp64_peak_probe(device);
    const double w = dmma_peak_probe(device);
    if (v <= 0 || w <= 0) return PSDP_ECUDA;
    *dfma_tflops = v;
    *dmma_tflops = w;
    return PSDP_OK;
}

void psdp_destroy(psdp_ctx* c) { free_ctx(c); }

const char* psdp_strerror(psdp_status s) {
    switch (s) {
        case PSDP_OK: return "ok";
        case PSDP_EINVAL: return "invalid argument";
        case PSDP_ENOMEM: return "device allocation failed";
        case PSDP_ECUDA: return "CUDA error";
        case PSDP_ECHOL_BLOCK: return "a block of X or Z is not positive definite";
        case PSDP_ECHOL_SCHUR: return "Schur complement is not positive definite";
        case PSDP_EMAXITER: return "iteration limit reached";
        case PSDP_ESTEP: return "step length collapsed";
        case PSDP_EUNBOUNDED: return "primal ray found: LMIs infeasible at these degrees";
        case PSDP_ENAN: return "non-finite value";
        case PSDP_ETIMEOUT: return "bounded device wait gave up";
        case PSDP_ESTATE: return "call not valid in the current state";
    }
    return "unknown status";
}

}  // extern "C"
