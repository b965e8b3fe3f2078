// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/polya_sdp.h"

#define PSDP_MAX_N 112
#define PSDP_MAX_L 16

// Slots of the device scalar array ctx->d_scal.
enum ScalarSlot {
    SC_TRZX = 0,   // tr(ZX) at the current iterate
    SC_MU = 1,     // sigma * tr(ZX) / n_X for the next corrector
    SC_TP = 2,     // primal step of the last update
    SC_TD = 3,     // dual step of the last update
    SC_PHI = 4,    // tr(CX)
    SC_PSI = 5,    // a^T y
    SC_RELGAP = 6,
    SC_PRES = 7,
    SC_DRES = 8,
    SC_TRX = 9,
    SC_BXN = 10,   // ||B(X)||
    SC_TPMAX = 11, // raw max steps before tau
    SC_TDMAX = 12,
    SC_COUNT = 16
};

// Bits of the device failure flag ctx->d_flag.
enum FlagBits {
    FL_CHOL_BLOCK = 1,
    FL_CHOL_SCHUR = 2,
    FL_NAN = 4,
    FL_TIMEOUT = 8,
    FL_MIXED = 16,     // mixed-precision solve did not reach its residual target
    FL_FROZEN = 32,    // finished batch member: its graph branch runs but leaves the iterate
};

struct ProfSite {
    int name_id;
    cudaEvent_t a, b;
    cudaStream_t st;    // stream the two events are recorded on
};

struct psdp_ctx {
    // ----- sizes
    int n, l, d_p, d1, d2, d_a;
    int L0, L, M, Na, Nt, K, nblk, n2;
    psdp_opts opt;
    int device;
    int num_sms = 1;
    cudaStream_t stream;
    bool own_stream;
    // high-priority stream for the Cholesky critical path (panel factor, panel
    // solve, next-panel update) and the events that fork/join it with `stream`
    cudaStream_t crit = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    // ----- host copies of the tables
    std::vector<int32_t> beta;   // [L0][L]
    std::vector<int32_t> cH;     // [L0][M][Na]
    std::vector<double> cdiag;   // C_gamma = cdiag[gamma] * I  (all nblk blocks)

    // ----- device tables and data
    int32_t *d_beta = nullptr, *d_cH = nullptr;
    int32_t *d_W0 = nullptr, *d_Wa = nullptr;   // monomial exponents [L0][l], [Na][l]
    double *d_A = nullptr;                      // [Na][n][n]
    double *d_H = nullptr;                      // [L0][M][n][n]
    double *d_cdiag = nullptr;                  // [nblk]
    // generalised form (Sec. III-C): constant term R(alpha) and the dual objective a
    int d_r = -1, Nr = 0;                       // degree of R, card W_{d_r}
    double *d_R = nullptr;                      // R coefficients [Nr][n][n]
    int32_t *d_Wr = nullptr;                    // their exponents [Nr][l]
    double *d_CR = nullptr;                     // R's part of the Lyapunov blocks of C [M][n][n]
    double *d_avec = nullptr;                   // objective a [K]; null: all ones (Eq. a)
    double c2_extra = 0.0;                      // ||C||_F^2 beyond the cdiag part
    double a_norm = 0.0;                        // ||a|| when d_avec is set

    // ----- iterate and per-block work arrays, each [nblk][n][n]
    double *d_X = nullptr, *d_Z = nullptr, *d_G = nullptr, *d_Y = nullptr;
    double *d_T1 = nullptr, *d_T2 = nullptr, *d_W = nullptr, *d_F = nullptr;
    double *d_dXh = nullptr, *d_dZh = nullptr, *d_dX = nullptr, *d_dZ = nullptr;
    double *d_S = nullptr;      // [M][Na][n][n]   B^T scratch
    double *d_adj = nullptr;    // [L0][Na+1][n][n] adjoint scratch
    double *d_adj2 = nullptr;   // [L0][Na][n][n]
    int32_t *d_adj_idx = nullptr;   // operand indices of the adjoint's products [3][L0*Na]
    double *d_y = nullptr, *d_dyh = nullptr, *d_dyb = nullptr, *d_BX = nullptr;
    double *d_part = nullptr;   // per-block partial sums [2*nblk][4]
    double *d_tstep = nullptr;  // per-block max steps [2*nblk]
    double *d_scal = nullptr;   // [SC_COUNT]
    double *d_info = nullptr;   // [PSDP_INFO_LEN]
    int *d_flag = nullptr;
    double *h_info = nullptr;   // pinned host mirror of d_info
    int *h_flag = nullptr;

    // ----- Schur complement
    int npairs = 0, nterms = 0, nlyap_prod = 0;
    std::vector<int> pair_a, pair_b, term_off, term_cnt;
    int32_t *d_pair_a = nullptr, *d_pair_b = nullptr, *d_term_off = nullptr, *d_term_cnt = nullptr;
    int32_t *d_term_desc = nullptr;   // [nterms][8] operand sources
    double *d_term_w = nullptr;       // [nterms]
    int32_t *d_uv_idx = nullptr;      // index arrays for U/V GEMMs [3][L0*M]
    int32_t *d_prod_idx = nullptr;    // index arrays for pair products [3][nlyap_prod*2]
    double *d_U = nullptr, *d_V = nullptr;   // [L0][M][n][n]
    double *d_Aop = nullptr, *d_Bop = nullptr;  // [nterms][n][n]
    double *d_Tbuf = nullptr;         // [pairs_per_chunk][n2][n2]
    int pairs_per_chunk = 1;
    double *d_Om = nullptr;           // [K][K] row-major, upper triangle authoritative
    double *d_Linv = nullptr;         // diagonal-block inverses of the dense factor [npanel][nb][nb]
    double *d_Linv64 = nullptr;       // the same paired into 64 x 64 blocks for the sweeps [ceil(K/64)][64][64]
    unsigned *d_trsv_sync = nullptr;  // tickets and ready flags of the triangular sweeps
    int *d_chol_ctr = nullptr;        // tile counters of the persistent FP64 trailing updates, one per panel
    int nb_chol = 32;                 // FP64 Cholesky panel width (the diagonal factor's block size)
    // ----- Ozaki-scheme FP64 products (BF16 tensor-core slices)
    bool oz_chol = false, oz_schur = false;   // engines chosen at set-up
    uint16_t *d_oz_sa = nullptr, *d_oz_sb = nullptr;   // slices [batch][8][rows][dpad]
    int32_t *d_oz_ea = nullptr, *d_oz_eb = nullptr;    // row exponents [batch][rows]
    uint16_t *d_oz_si = nullptr;                        // an inner Cholesky panel's slices [8][K][32], then L_jj^{-1}'s [8][32][32]
    int32_t *d_oz_ei = nullptr;                         // and row exponents [K + 32]
    uint16_t *d_oz_sm = nullptr;                        // a 128-column block's rows [8][K][128]
    int32_t *d_oz_em = nullptr;                         // and row exponents [K]
    double flops_schur = 0, flops_chol = 0, flops_schur_dense = 0;

    // ----- misc
    double *d_grid = nullptr; size_t grid_cap = 0;   // grid-check scratch
    int32_t *d_svec = nullptr;        // (r, s) of each svec index [Nt][2]

    // ----- mixed precision (3xTF32 Schur and Cholesky, FP64 PCG)
    bool mixed = false;               // precision == PSDP_MIXED
    bool mixed_failed = false;        // sticky: fell back to the FP64 step
    bool have_fp64 = false;           // FP64 Schur / Cholesky buffers allocated
    int tpad = 0, nb32 = 128, pairs_per_chunk32 = 1;
    int pcg_max = 8;
    double pcg_tol = 1e-12, pcg_fail = 1e-9;
    int32_t *d_term_off_t = nullptr;  // first term of each pair [npairs]
    float *d_opA_hi = nullptr, *d_opA_lo = nullptr, *d_opB_hi = nullptr, *d_opB_lo = nullptr;
    double *d_prodA = nullptr, *d_prodB = nullptr;     // GEMM-built operand products [nlyap_prod][n][n]
    float *d_T32 = nullptr, *d_Om32 = nullptr, *d_Linv32 = nullptr, *d_Pt_hi = nullptr, *d_Pt_lo = nullptr;
    float *d_Pk_hi = nullptr, *d_Pk_lo = nullptr;   // unsolved panel, K-major TF32 pairs [K][nb32]
    float *d_Lt_hi = nullptr, *d_Lt_lo = nullptr;   // current diagonal-block inverse, row-major TF32 pairs
    float *d_z32 = nullptr;
    double *d_pcg_x = nullptr, *d_pcg_r = nullptr, *d_pcg_z = nullptr, *d_pcg_p = nullptr, *d_pcg_q = nullptr;
    double *d_pcg_state = nullptr;
    int *d_pcg_done = nullptr;
    double *d_M1 = nullptr, *d_M2 = nullptr;          // matrix-free Omega*v scratch blocks
    CUtensorMap map_opA_hi, map_opA_lo, map_opB_hi, map_opB_lo;
    bool have_graph32 = false;
    cudaGraphExec_t graph_exec32 = nullptr;
    cudaGraph_t graph32 = nullptr;
    double *d_cert = nullptr;         // certificate outputs [4]
    int iters = 0;
    int kernels_per_step = 0;   // kernel nodes in the captured Newton-step graph
    bool have_graph = false;
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraph_t graph = nullptr;

    // ----- profiling
    bool prof_on = false;
    std::vector<std::string> prof_names;
    std::vector<int64_t> prof_launches;
    std::vector<double> prof_ms;
    std::vector<ProfSite> prof_sites;     // sites of the FP64 step
    std::vector<ProfSite> prof_sites32;   // sites of the mixed-precision step
    std::vector<ProfSite>* prof_cur = nullptr;
    std::vector<cudaEvent_t> prof_pool;   // reusable events
    // trace of the last profiled step: per site, its name, start and end (ms
    // after the step's first site started) and whether it ran on the critical stream
    std::vector<int> prof_tr_id, prof_tr_crit;
    std::vector<double> prof_tr_t0, prof_tr_t1;
    size_t prof_pool_used = 0, prof_pool_limit = 0;
};

// ------------------------------------------------------------- launchers
// All launchers enqueue on `st` and never synchronise.

// tables: beta [L0][L], cH [L0][M][Na], monomial lists; closed-form multinomials
void launch_tables(cudaStream_t st, int l, int d_p, int d1, int d2, int d_a, int L0, int L, int M, int Na,
                   int32_t* beta, int32_t* cH, int32_t* W0, int32_t* Wa);
// H[h][g] = sum_lambda cH[h][g][lambda] A[lambda]
void launch_hmat(cudaStream_t st, int L0, int M, int Na, int n, const int32_t* cH, const double* A, double* H);

// batched n x n GEMM: C_e = alpha sum_{q < nsum} op(A_{e,q}) op(B_{e,q}) + beta C_e
// (or its transpose if tc); matrix index of operand X for element e and term q
// is (ix ? ix[e] : e * sx) + q * qx.
void launch_bgemm(cudaStream_t st, int n, int count,
                  const double* A, const int32_t* ia, int sa, int ta,
                  const double* B, const int32_t* ib, int sb, int tb,
                  double* C, const int32_t* ic, int sc, int tc, double alpha, double beta,
                  const int* skip = nullptr, int nsum = 1, int qa = 0, int qb = 0);

// batched TN GEMM: C_b[r][c] = alpha * sum_{k<kd_b} A_b[k*lda + r] * B_b[k*ldb + c] + beta * C_b[r*ldc + c]
// for r < m, c < ncol; per-batch offsets (elements) and contraction lengths from device arrays
// (or uniform when the arrays are null).  tri: only tiles with tile_c >= tile_r.
// Persistent FP64 Cholesky trailing update C[r][c] -= sum_k P[k*lda+r] P[k*lda+c]
// on the c >= r 32 x 32 tiles of the m x m matrix (depth kdep); grid CTAs of two
// 256-thread groups each reserve a whole SM; *ctr must be zero at launch.
void launch_syrk_tri_persist(cudaStream_t st, int m, int kdep, const double* P, int lda, double* C, int ldc, int* ctr,
                             int grid);
void launch_gemm_tn(cudaStream_t st, int m, int ncol, int batch,
                    const double* A, int lda, const int32_t* a_off, int64_t a_stride,
                    const double* B, int ldb, const int32_t* b_off, int64_t b_stride,
                    const int32_t* kd, int kd_uniform,
                    double* C, int ldc, int64_t c_stride, double alpha, double beta, int tri);

// per-block Cholesky of Z and inverse Y = Z^{-1}; flag |= FL_CHOL_BLOCK on failure
void launch_block_chol_inv(cudaStream_t st, int nb, int n, const double* Z, double* Y, int* flag);
// per-block max step sup{t: M + t D >= 0} for (X,dX) blocks [0,nb) and (Z,dZ) blocks [nb,2nb)
void launch_block_maxstep(cudaStream_t st, int nb, int n, const double* X, const double* dX,
                          const double* Z, const double* dZ, double* tstep, int* flag);
// per-matrix smallest eigenvalue of sign*M and Frobenius norm; out[2*i] = lambda_min, out[2*i+1] = ||M||
void launch_block_mineig(cudaStream_t st, int count, int n, const double* M, double sign, double* out);

// SDP operators
// out = B^T(v);  out = B(W) - acoef*1.  With skip non-null the kernels do nothing while *skip != 0.
void launch_bt(cudaStream_t st, psdp_ctx* c, const double* v, double* out_blocks, const int* skip = nullptr);
void launch_b(cudaStream_t st, psdp_ctx* c, const double* W, double* out, double acoef, const int* skip = nullptr);

// elementwise
void launch_ew_G(cudaStream_t st, psdp_ctx* c, const double* BTy, const double* Z, double* G);
void launch_ew_pred(cudaStream_t st, psdp_ctx* c, const double* G, const double* D, double* E, double* dZh);
void launch_ew_symsub(cudaStream_t st, psdp_ctx* c, const double* T, const double* X, double* out);
void launch_ew_muY(cudaStream_t st, psdp_ctx* c, const double* Y, const double* W2, const double* mu, double* F);
void launch_ew_corr(cudaStream_t st, psdp_ctx* c, const double* F, const double* T, const double* dXh,
                    const double* dZh, const double* dZb, double* dX, double* dZ);
void launch_update(cudaStream_t st, psdp_ctx* c);
void launch_identity(cudaStream_t st, int nb, int n, double* X);
void launch_partials(cudaStream_t st, psdp_ctx* c);
void launch_finalize(cudaStream_t st, psdp_ctx* c, int iter);  // iter unused on device
void launch_steplen(cudaStream_t st, psdp_ctx* c);

// Schur complement
void launch_schur_operands(cudaStream_t st, psdp_ctx* c);
void launch_schur_gather(cudaStream_t st, psdp_ctx* c, int p0, int np);

// dense Cholesky (Omega stored row-major with the upper triangle, i.e. column-major lower)
void launch_potrf_diag(cudaStream_t st, double* A, int K, int j0, int nb, double* Linv, int* flag);
void launch_cdiag(cudaStream_t st, psdp_ctx* c);

// raise the dynamic shared-memory limit of the shared-memory-heavy kernels once,
// outside any stream capture
void init_attrs_linalg(int smem_max);
void init_attrs_sdp(int smem_max);
void init_attrs_dense(int smem_max);

// warm start: X_g = xs_g I, Z_g = B^T(y0)_g - C_g lifted to lambda_min >= theta / xs_g
// (eig[2g] = lambda_min of B^T(y0)_g, computed beforehand)
void launch_start_fix(cudaStream_t st, psdp_ctx* c, const double* BTy, const double* eig, const double* xs,
                      double theta);

// certificate / grid
void launch_certify_finalize(cudaStream_t st, int count, int n, const double* eig, int L, double* out);
// blocks[g] -= CR[g - L] on the Lyapunov blocks (no-op without a constant term)
void launch_sub_CR(cudaStream_t st, psdp_ctx* c, double* blocks);
// Q[pt] += R(alpha_pt) on the lattice points of launch_grid_build (no-op without R)
void launch_grid_addR(cudaStream_t st, psdp_ctx* c, int N, int64_t first, int cnt, double* Q);
void launch_grid_build(cudaStream_t st, psdp_ctx* c, int N, int64_t first, int cnt, double* P, double* Aal);

// FP64 throughput probe
double fp64_peak_probe(int device);
double dmma_peak_probe(int device);

// tensor-core GEMM (k_tc_gemm.cu)
bool tc_make_map(CUtensorMap* map, const void* base, bool bf16, int64_t kdim, int64_t rows, int64_t batch,
                 int64_t row_stride, int64_t batch_stride, int box_rows);
bool tc_make_map_swz(CUtensorMap* map, const void* base, bool bf16, int64_t kdim, int64_t rows, int64_t batch,
                     int64_t row_stride, int64_t batch_stride, int box_k, int box_rows, int swizzle_bytes);
bool launch_tc_gemm(cudaStream_t st, bool bf16, int split, const CUtensorMap& A, const CUtensorMap& B,
                    const CUtensorMap* Alo, const CUtensorMap* Blo, int M, int N, int batch, int b0,
                    const int32_t* kd, int kd_uniform, float* C, int64_t ldc, int64_t c_batch, float alpha,
                    float beta, int tri, int* flag, float* aux_hi = nullptr, float* aux_lo = nullptr,
                    int aux_ld = 0, int aux_m0 = 0, int aux_n1 = 0);
void launch_split_tf32(cudaStream_t st, int64_t n, const float* x, float* hi, float* lo);
bool launch_tc_gemm_persist(cudaStream_t st, int split, const CUtensorMap& A, const CUtensorMap& B,
                            const CUtensorMap* Alo, const CUtensorMap* Blo, int M, int N, int kd, float* C,
                            int64_t ldc, float alpha, float beta, int tri, int ctas, int* flag);
void init_attrs_tc(int smem_optin);
cudaError_t set_attrs_tc_gemm_fp32(int smem_optin);

// FP64 products by the Ozaki scheme on the BF16 tensor cores (k_ozaki.cu).
// Slices: 8 BF16 digits per element, [batch][8][rows][dpad] (uint16 bit
// patterns), row exponents [batch][rows]; depth <= kOzakiMaxDepth, dpad a
// multiple of 32.
constexpr int kOzakiMaxDepth = 384;
void init_attrs_ozaki(int smem_optin);
size_t ozaki_slice_elems(int rows, int dpad, int batch);
// Each call covers the depth window [k_off, k_off + kOzakiMaxDepth) of every batch
// (depths per batch from kdv, else kd_uniform); deeper products sum the windows
// with beta = 1.  Split: element (r, k) of batch b at src[off_b + k * ld + r],
// off_b = src_off[b] (elements) if given, else b * src_batch.
void launch_ozaki_split(cudaStream_t st, const double* src, int64_t ld, int64_t src_batch, const int32_t* src_off,
                        int rows, const int32_t* kdv, int kd_uniform, int k_off, int dpad, int batch, uint16_t* out,
                        int32_t* ex);
// C_b[j * ldc + i] = alpha sum_k A_b[i][k] B_b[j][k] + beta C_b[...] (i >= j only when lower),
// A_b's rows a_row0 + i (i < M) of slice arrays of a_rows rows (exponents eA[b][a_rows]), B_b likewise;
// a persistent launch of min(tiles, ctas) CTAs (ctas <= 0: one per SM)
bool launch_ozaki_gemm(cudaStream_t st, const uint16_t* As, int a_rows, int a_row0, const int32_t* eA,
                       const uint16_t* Bs, int b_rows, int b_row0, const int32_t* eB, int M, int N, int dpad,
                       int batch, const int32_t* kd, int kd_uniform, int k_off, double* C, int64_t ldc,
                       int64_t c_batch, double alpha, double beta, int lower, int* flag, int ctas = 0);

// mixed precision (k_mixed.cu)
void launch_schur_pack32(cudaStream_t st, psdp_ctx* c);
void launch_schur_gather32(cudaStream_t st, psdp_ctx* c, int p0, int np, const float* T, float* Om);
void launch_potrf_diag32(cudaStream_t st, float* A, int K, int j0, int nb, float* Linv, float* LtHi, float* LtLo,
                         int* flag);
void launch_pack_panel32(cudaStream_t st, const float* A, int K, int j0, int nb, float* PkHi, float* PkLo);

// Triangular sweeps with the dense factor (one launch per sweep, flag-synchronised
// block rows).  sync needs trsv_sync_words(K, nb) words; false for an
// unsupported panel width (FP64: 32; FP32: 64, 128).
size_t trsv_sync_words(int K, int nb);
bool launch_solve_fp64(cudaStream_t st, const double* A, int K, int nb, const double* Linv, double* x,
                       unsigned* sync, int* flag);
void launch_pair_inverse(cudaStream_t st, const double* A, int K, const double* Linv32, double* Linv64);
bool launch_precond32(cudaStream_t st, const float* A, int K, int nb, const float* Linv, float* z32,
                           const double* r, double* z, unsigned* sync, int* flag, const int* skip);
void launch_pcg_init(cudaStream_t st, int K, const double* b, double* x, double* r, double* s, int* done);
void launch_pcg_start(cudaStream_t st, int K, const double* r, const double* z, double* p, double* s, const int* done);
void launch_pcg_alpha(cudaStream_t st, int K, const double* p, const double* q, double* x, double* r, double* s,
                      int* done, double tol);
void launch_pcg_beta(cudaStream_t st, int K, const double* r, const double* z, double* p, double* s, const int* done);
void launch_pcg_finish(cudaStream_t st, int K, const double* x, double* out, double* s, const int* done, int* flag,
                       double tol_fail, double* info_slot);
void init_attrs_mixed(int smem_optin);

// errors
#define CK(x) do { cudaError_t e__ = (x); if (e__ != cudaSuccess) return PSDP_ECUDA; } while (0)

// Allow `f` the largest dynamic shared memory the device permits next to its
// static shared memory; clears the error state either way.
inline void set_max_dynamic_smem(const void* f, int smem_optin) {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, f) == cudaSuccess)
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin - (int)a.sharedSizeBytes);
    cudaGetLastError();
}
