/*
 * polya_sdp.h -- C ABI of the GB300 (sm_103a) Polya/SDP robust-stability library.
 *
 * The library certifies that x' = A(alpha) x is stable for every alpha on the
 * unit simplex (Theorem 1 of Kamyar, Peet & Peet, "Solving Large-Scale Robust
 * Stability Problems by Exploiting the Parallel Structure of Polya's
 * Theorem", IEEE TAC 2013).  It builds the block-diagonal SDP that Polya's
 * theorem (Theorem 2) gives for a homogeneous Lyapunov matrix
 * P(alpha) = sum_h P_h alpha^h (Sec. III) and solves it with the primal-dual
 * predictor-corrector interior-point method of Sec. IV-A / Algorithm 2.  Every
 * numerical step runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions (all entry points):
 *  - Every pointer argument is a HOST pointer unless stated otherwise.  The
 *    library copies inputs; the caller keeps ownership of its buffers.  All
 *    device memory is owned by the context and freed by psdp_destroy.
 *  - Matrices are row-major float64: M[i*n + j] = M_ij.
 *  - Monomial sets W_d are in the paper's lexicographic order, (d,0,...,0)
 *    first (Sec. I, text and worked examples).
 *  - Symmetric-matrix variables use the basis E_k of S^n (Sec. I): the n
 *    diagonal entries first, then the first superdiagonal (r, r+1), then the
 *    second (r, r+2), and so on ("svec order"); each off-diagonal basis matrix
 *    has unit entries, so y_{q + Ntil*h} is the (r,s) entry of P_h (Eq. V_h).
 *  - Block-diagonal matrices X, Z (Eq. S) are stored as (L+M) consecutive
 *    n x n blocks: the L P-side blocks gamma in W_{d_p+d1}, then the M
 *    Lyapunov blocks gamma in W_{d_p+d_a+d2}.
 *  - No exception crosses the ABI; every call returns a psdp_status.  A NULL
 *    context or output pointer gives PSDP_EINVAL.  After PSDP_ECUDA the
 *    context must only be destroyed.
 */
#ifndef POLYA_SDP_H
#define POLYA_SDP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct psdp_ctx psdp_ctx;

typedef enum {
    PSDP_OK = 0,
    PSDP_EINVAL = 1,        /* bad argument (size, NULL pointer, non-finite A, ...) */
    PSDP_ENOMEM = 2,        /* device allocation failed */
    PSDP_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    PSDP_ECHOL_BLOCK = 4,   /* a block Z_gamma or X_gamma lost positive definiteness */
    PSDP_ECHOL_SCHUR = 5,   /* the Schur complement Omega was not positive definite */
    PSDP_EMAXITER = 6,      /* psdp_solve hit max_iter; the iterate stays valid */
    PSDP_ESTEP = 7,         /* step length collapsed to zero */
    PSDP_EUNBOUNDED = 8,    /* primal ray: the LMIs are infeasible at these degrees */
    PSDP_ENAN = 9,          /* a non-finite scalar appeared */
    PSDP_ETIMEOUT = 10,     /* a bounded device wait gave up */
    PSDP_ESTATE = 11        /* call not valid in the context's current state */
} psdp_status;

typedef enum { PSDP_FP64 = 0, PSDP_MIXED = 1 } psdp_precision;

typedef struct {
    double delta;       /* delta of Eq. (Cj): C_gamma = delta*multinomial(gamma)*I; default 1 */
    double delta_L;     /* optional strict margin on the Lyapunov blocks (paper: 0); default 0 */
    double eps;         /* stopping tolerance of the relative gap and residuals; default 1e-7 */
    double sigma;       /* centring parameter of mu = sigma*tr(ZX)/n_X; default 1/3 */
    double tau;         /* step = min(1, tau * max feasible step); default 0.95 */
    int    max_iter;    /* iteration cap of psdp_solve; default 100 */
    int    d2;          /* Polya exponent of the Lyapunov inequality; < 0 means d2 = d1 */
    int    d_a;         /* degree of the homogeneous A(alpha); default 1 (affine) */
    int    precision;   /* psdp_precision; default PSDP_FP64 */
    int    use_graph;   /* capture one Newton step in a CUDA graph and replay it; default 1 */
    void*  stream;      /* cudaStream_t to run on; NULL: the context creates its own */
    int    device;      /* CUDA device ordinal; default 0 */
    int    crit_sms;    /* SMs the persistent Cholesky trailing update leaves to the
                           critical path (panel factor, panel solve, next-rows
                           update); 0 = the default (8 with FP64 FMA, 16 with the
                           Ozaki scheme and in the mixed form) */
    int    fp64_gemm;   /* engine of the FP64 form's two large contractions, the Schur
                           complement and the Cholesky trailing updates:
                           PSDP_GEMM_AUTO (default: by size), PSDP_GEMM_DFMA (FP64 FMA),
                           PSDP_GEMM_OZAKI (FP64-accurate products from exact BF16
                           tensor-core slice products, Ozaki et al. 2012) */
} psdp_opts;

enum { PSDP_GEMM_AUTO = 0, PSDP_GEMM_DFMA = 1, PSDP_GEMM_OZAKI = 2 };

/* Number of doubles psdp_step / psdp_solve write to their info array. */
#define PSDP_INFO_LEN 16
/* info layout: 0 phi=tr(CX), 1 psi=a^T y, 2 relative gap, 3 relative primal residual,
 * 4 relative dual residual, 5 mu, 6 t_p, 7 t_d, 8 tr(ZX), 9 tr(X), 10 ||B(X)||,
 * 11 iterations done so far, 12 mixed-precision refinement sweeps of the last step,
 * 13 1 if the last step fell back from mixed to FP64, 14-15 reserved. */

/* Fill *o with the defaults listed above. */
void psdp_default_opts(psdp_opts* o);

/* Build the SDP of Sec. III for dx/dt = A(alpha) x and allocate a solver context.
 *  n   : states, 1 <= n <= 112
 *  l   : uncertain parameters (simplex dimension), 1 <= l <= 16
 *  d_p : degree of P(alpha), d_p >= 0;   d1 : Polya exponent of P (Eq. LMI_1), d1 >= 0
 *  A   : host, N_a * n * n doubles, N_a = card W_{d_a} = C(l+d_a-1, l-1): the
 *        coefficients A_lambda of the homogeneous A(alpha) (Eq. A_alpha), lambda in
 *        W_{d_a} in lexicographic order; for the affine case d_a = 1 these are A_1..A_l.
 *  o   : options (NULL = defaults);   out : receives the context.
 * The Polya tables beta (Eqs. beta_init/beta) and H (Eqs. H_init/H) are computed on
 * the device; the iterate is set to the cold start X = Z = I, y = 0 (Algorithm 2).
 * Errors: EINVAL for sizes outside the ranges or non-finite A; ENOMEM; ECUDA. */
psdp_status psdp_setup(int n, int l, int d_p, int d1, const double* A,
                       const psdp_opts* o, psdp_ctx** out);

/* Sizes of the SDP: out[0..8] = n, l, L0 = card W_{d_p}, L = card W_{d_p+d1},
 * M = card W_{d_p+d_a+d2}, Ntil = n(n+1)/2, K = L0*Ntil (Eq. K), L+M, N_a. */
psdp_status psdp_sizes(const psdp_ctx* c, int32_t* out9);

/* One predictor-corrector Newton step (Sec. IV-A, Processors/Root steps 1-4 of
 * Algorithm 2) entirely on the device; info (may be NULL) receives PSDP_INFO_LEN
 * doubles describing the new iterate.  ECHOL_BLOCK / ECHOL_SCHUR / ENAN leave the
 * iterate unchanged. */
psdp_status psdp_step(psdp_ctx* c, double* info);

/* Repeat psdp_step until the relative gap and both relative residuals are <= eps
 * (the paper's gap rule plus feasibility), a failure, a primal ray (EUNBOUNDED)
 * or max_iter (EMAXITER).  iters/info may be NULL. */
psdp_status psdp_solve(psdp_ctx* c, int* iters, double* info);

/* Solve many independent instances together (no counterpart in the paper, whose
 * parallelism is over the blocks of one instance).  Every unfinished instance's
 * captured Newton-step graph becomes one branch of a single batch graph, launched
 * once per interior-point iteration; instances that meet their stopping rule
 * drop out (the batch graph is rebuilt once a quarter of its branches are done).
 * All contexts must be distinct, on one device, with use_graph = 1 and profiling
 * off.  status[i] / iters[i] (may be NULL) receive what psdp_solve would return
 * for instance i.  The function's own result is PSDP_OK unless the batch itself
 * could not run (EINVAL, ECUDA, ENOMEM). */
psdp_status psdp_solve_batch(psdp_ctx** ctx, int count, psdp_status* status, int* iters);

/* Pick the fastest Newton-step configuration for this instance shape by timing
 * one step of each candidate from the current iterate (restored afterwards):
 * 0 = FP64, 1 = mixed precision with 64-column FP32 Cholesky panels (SYRK tiles
 * of depth 64), 2 = mixed with 128-column panels.  With cache_path non-NULL the
 * result is looked up in / appended to that text file, keyed by
 * (n, l, d_p, d1, d2, d_a).  The choice is applied to the context.
 * choice and ms3 (per-candidate step times in ms, -1 if read from the cache)
 * may be NULL. */
psdp_status psdp_autotune(psdp_ctx* c, const char* cache_path, int* choice, double* ms3);

/* The same over a chosen set of step configurations (no counterpart in the
 * paper): bit k of mask enables candidate k,
 *   0 FP64 with the automatic engines (psdp_opts.fp64_gemm),
 *   1 mixed precision, 64-column FP32 Cholesky panels,
 *   2 mixed precision, 128-column FP32 Cholesky panels,
 *   3 FP64 with FP64-FMA contractions (Schur tiles 80 x 80 or 64 x 64 by n^2,
 *     32 x 32 Cholesky bulk tiles, one-shot or persistent by the tile waves),
 *   4 FP64 with Ozaki-scheme contractions (128 x 64 tensor-core tiles, 256-column
 *     outer Cholesky panels),
 *   5 FP64 with the Ozaki Schur contraction and the FP64-FMA Cholesky.
 * The cache key is (n, l, d_p, d1, d2, d_a, mask); ms (may be NULL) receives
 * PSDP_TUNE_CANDIDATES per-candidate step times in ms (-1 if not timed).  The
 * fastest candidate is applied to the context.  psdp_autotune is mask 7. */
#define PSDP_TUNE_CANDIDATES 6
psdp_status psdp_autotune_ex(psdp_ctx* c, const char* cache_path, unsigned mask, int* choice, double* ms);

/* Certificate of Theorems 1-2 from the current y: P_h = smat(y_h) (Root step 4);
 * every P-side coefficient sum_h beta_{h,gamma} P_h (Eq. LMI_3) and every negated
 * Lyapunov coefficient -sum_h (H^T P_h + P_h H) (Eq. LMI_4) must have its smallest
 * FP64 eigenvalue above 64*n*2^-53*||.||_F.  verdict = 1 certified, 0 not.
 * minP_margin = smallest eigenvalue over the P-side coefficients; maxLyap_margin =
 * largest eigenvalue over the Lyapunov coefficients sum_h(H^T P_h + P_h H)
 * (negative when certified).  Any output pointer may be NULL. */
psdp_status psdp_certify(psdp_ctx* c, int* verdict, double* minP_margin, double* maxLyap_margin);

/* Theorem 1 on the simplex lattice {gamma/N : gamma in W_N}: minP = min over the
 * lattice of lambda_min(P(alpha)), maxQ = max of lambda_max(A^T P + P A). N >= 1. */
psdp_status psdp_grid_check(psdp_ctx* c, int N, double* minP, double* maxQ);

/* Copy out P_h (L0 * n * n doubles, full symmetric) or y (K doubles). */
psdp_status psdp_get_P(psdp_ctx* c, double* P);
psdp_status psdp_get_y(psdp_ctx* c, double* y);

/* Warm start (no counterpart in the paper, whose start is X = Z = I, y = 0):
 * y = y0 (K doubles), X_gamma = xscale[gamma] I ((L+M) positive doubles; NULL
 * means 1), and Z_gamma = B^T(y0)_gamma - C_gamma lifted by a multiple of I so
 * that its smallest eigenvalue is at least theta / xscale[gamma] (theta > 0),
 * which keeps the start strictly interior.  Resets the iteration count.
 * Errors: EINVAL for non-finite y0, non-positive scalings or theta. */
psdp_status psdp_set_start(psdp_ctx* c, const double* y0, const double* xscale, double theta);

/* The generalised inequality of Sec. III-C (Eq. LMI_general) with one term,
 * A~ = A(alpha)^T and B~ = I:  A(alpha)^T P(alpha) + P(alpha) A(alpha) + R(alpha) < 0
 * on the simplex, with the constant term R(alpha) = sum_rho R_rho alpha^rho
 * homogeneous of degree d_r, 0 <= d_r <= d_p + d_a + d2 (the Lyapunov
 * inequality's degree).  R: host, card(W_{d_r}) * n * n doubles, rho in W_{d_r}
 * in lexicographic order, each n x n coefficient row-major and symmetric
 * (else EINVAL).  R enters the SDP only through C: on Lyapunov block gamma,
 * C_gamma = sum_rho multinomial(e; gamma - rho) R_rho, e = d_p + d_a + d2 - d_r
 * (the coefficients of R(alpha) (sum alpha)^e); the certificate and the
 * lattice check include R.  Example: R = C^T C with the objective below gives
 * the robust H2 analysis LMI.  Resets the iterate to the cold start. */
psdp_status psdp_set_constant_term(psdp_ctx* c, int d_r, const double* R);

/* The dual objective a of min a^T y (Eq. a; the paper's all-ones vector by
 * default): host, K doubles, finite (else EINVAL).  With y_{q + Ntil h} the
 * (r, s) entry of P_h, a = the svec weights of a symmetric W (W_rr, 2 W_rs)
 * minimises sum_h tr(W P_h).  Resets the iterate to the cold start. */
psdp_status psdp_set_objective(psdp_ctx* c, const double* a);

/* The learned warm-start network (no counterpart in the paper): a three-layer
 * ReLU MLP n_in -> width -> width -> n_out whose products all run on the tensor
 * cores with BF16 operands and FP32 accumulation; Adam on FP32 master weights.
 * Host arrays are row-major float32 batches (one sample per row). */
typedef struct psdp_mlp psdp_mlp;
/* n_in, width, max_batch multiples of 8; He-normal weights from `seed`. */
psdp_status psdp_mlp_create(int n_in, int width, int n_out, int max_batch, uint64_t seed, int device, psdp_mlp** out);
void psdp_mlp_destroy(psdp_mlp* m);
/* Parameters as one float32 array W1 (width x n_in), b1, W2, b2, W3 (n_out x width), b3;
 * *count receives its length.  get / set may be NULL. */
psdp_status psdp_mlp_params(psdp_mlp* m, float* get, const float* set, int64_t* count);
/* Loss mean((Y - T)^2) and its gradients (layout of psdp_mlp_params) on one batch
 * of B <= max_batch raw (unstandardised) samples: the gradient-check hook. */
psdp_status psdp_mlp_grads(psdp_mlp* m, const float* X, const float* T, int B, float* loss, float* grads);
/* Adam training on n samples for `epochs` passes of batches of B (multiple of 8):
 * inputs and targets are standardised per feature with statistics of this set,
 * kept for psdp_mlp_predict; *final_loss = mean standardised loss of the last epoch. */
psdp_status psdp_mlp_train(psdp_mlp* m, const float* X, const float* T, int n, int epochs, int B, float lr,
                           uint64_t seed, float* final_loss);
/* Y (n x n_out) in target units. */
psdp_status psdp_mlp_predict(psdp_mlp* m, const float* X, int n, float* Y);

/* The integer Polya tables: beta (L0 x L, row h) and c (L0 x M x N_a) with
 * H_{h,gamma} = sum_lambda c[h][gamma][lambda] A_lambda. */
psdp_status psdp_get_tables(psdp_ctx* c, int32_t* beta, int32_t* cH);

/* Replace / read the iterate: X, Z as (L+M)*n*n doubles, y as K doubles.  X and Z
 * must be symmetric positive definite block by block (checked on the next step). */
psdp_status psdp_load_iterate(psdp_ctx* c, const double* X, const double* Z, const double* y);
psdp_status psdp_get_iterate(psdp_ctx* c, double* X, double* Z, double* y);

/* Schur complement Omega_ij = sum_k tr(B_i^k Z_k^{-1} B_j^k X_k) (Sec. IV-A,
 * Processors step 1) at the current iterate, as a full K x K matrix (lower triangle
 * authoritative; FP64 in both precision modes).  Test and inspection hook. */
psdp_status psdp_get_schur(psdp_ctx* c, double* Omega);

/* Selected columns of the same FP64 Omega (Sec. IV-A) at the current iterate,
 * for parity checks at sizes where the full K x K copy does not fit the host:
 * out[q*K + i] = Omega_{i, cols[q]} for q < ncols, i < K.  cols: host int32,
 * each in [0, K) (else EINVAL); out: host, ncols*K doubles, caller-owned.
 * Forms Omega on the device like psdp_get_schur (ECHOL_BLOCK if a block of Z is
 * not positive definite). */
psdp_status psdp_get_schur_cols(psdp_ctx* c, const int32_t* cols, int ncols, double* out);

/* The same Omega as computed by the mixed-precision path (PSDP_MIXED contexts only,
 * else ESTATE): operands rounded to FP32 and contracted on the tensor cores in
 * 3xTF32 with FP32 accumulation; K x K float32, full (upper triangle computed,
 * lower mirrored on the host).  Its error against psdp_get_schur is the stated
 * error of the mixed path's Schur complement. */
psdp_status psdp_get_schur_mixed(psdp_ctx* c, float* Omega);

/* Operator hooks for parity tests: out_blocks = B^T(v) (Eq. AT) and
 * out = B(W) = (tr(B_i W))_i for block-diagonal W ((L+M)*n*n doubles). */
psdp_status psdp_apply_BT(psdp_ctx* c, const double* v, double* out_blocks);
psdp_status psdp_apply_B(psdp_ctx* c, const double* W_blocks, double* out);

/* Per-kernel timing with CUDA events recorded on the context's stream around
 * each launch of the library's heavy kernels.  psdp_profile_get writes up to
 * max_entries records of (name[32], launches, total_ms) into names/launches/ms and
 * returns the count in *count. */
psdp_status psdp_profile_enable(psdp_ctx* c, int on);
psdp_status psdp_profile_reset(psdp_ctx* c);
psdp_status psdp_profile_get(psdp_ctx* c, int max_entries, char* names, int64_t* launches,
                             double* ms, int* count);

/* Timeline of the last profiled step (the paper has no counterpart: this is
 * instrumentation).  Entry i is one timed launch in issue order: name_ids[i]
 * indexes the names of psdp_profile_get, t0_ms[i] / t1_ms[i] are the times its
 * start and end events completed, in ms after the step's first timed launch
 * started, and on_crit[i] is 1 for launches on the look-ahead's critical stream.
 * Writes up to max_entries entries (any output pointer may be NULL) and the
 * count to *count; an empty trace when profiling is off.  Host arrays, owned by
 * the caller. */
psdp_status psdp_profile_trace(psdp_ctx* c, int max_entries, int* name_ids, double* t0_ms, double* t1_ms,
                               int* on_crit, int* count);

/* Algorithmic floating-point work of one Newton step: out[0] = Schur assembly
 * flops over the non-zero (pair, block) terms, out[1] = Cholesky flops K^3/3,
 * out[2] = Schur terms in the contraction (sum over block pairs), out[3] = dense
 * Schur flops (every block for every pair), out[4] = kernel launches in one
 * captured Newton step (0 before the first graph-mode step), out[5] = panel
 * width of the FP64 Cholesky, out[6] = panel width of the FP32 Cholesky of the
 * mixed-precision step. */
psdp_status psdp_work(const psdp_ctx* c, double* out7);

/* Engines the context chose for its FP64 contractions (psdp_opts.fp64_gemm):
 * out[0] = 1 if the Schur complement uses the Ozaki scheme, out[1] = 1 if the
 * Cholesky trailing updates do (0: FP64 FMA). */
psdp_status psdp_engines(const psdp_ctx* c, int32_t* out2);

/* The CUDA stream the context runs on (cudaStream_t as void*). */
void* psdp_stream(psdp_ctx* c);

/* Self-test of the library's tcgen05 tensor-core GEMM (no counterpart in the
 * paper; it is the contraction engine of the mixed-precision path and the MLP).
 * A: M x K, B: N x K, both row-major host arrays; C receives D = A B^T stored
 * column-major (C[n*M + m] = D[m][n]), float32, M*N values.
 * dtype 0: A, B float32, multiplied as TF32 (split 1) or as the 3xTF32 split
 * hi*hi + hi*lo + lo*hi (split 3); dtype 1: A, B bfloat16 bit patterns (uint16),
 * split must be 1.  Runs on the current device; allocates its own scratch.
 * Errors: EINVAL on bad sizes/flags, ETIMEOUT if a bounded device wait expired. */
psdp_status psdp_tc_gemm_check(int M, int N, int K, int dtype, int split, const void* A, const void* B, float* C);

/* Self-test of the bounded device waits (no counterpart in the paper): runs a
 * triangular sweep in which one block is never solved, so every waiting CTA
 * gives up after its 2 s limit.  Returns PSDP_ETIMEOUT when the wait gave up as
 * designed (the context stays usable), PSDP_OK if it did not; waited_ms (may be
 * NULL) receives the kernel's duration. */
psdp_status psdp_trsv_timeout_check(float* waited_ms);

/* Self-test of the persistent tcgen05 update used for the FP32 Cholesky trailing
 * update (no counterpart in the paper).  A: M x K, B: N x K row-major float32;
 * C: M x N column-major (C[n*M + m]), in/out.  On every 128 x 128 tile (mt, nt)
 * with mt >= nt when tri (all tiles otherwise): C <- C - A B^T, the product in
 * TF32 (split 1) or 3xTF32 (split 3); other tiles are left as they are.  ctas =
 * persistent CTAs (>= 1; fewer CTAs walk more tiles each).  ms (may be NULL)
 * receives the kernel's duration from CUDA events around the launch.  Allocates
 * its own scratch.  Errors: EINVAL on bad sizes, ETIMEOUT if a bounded wait expired. */
psdp_status psdp_tc_gemm_persist_check(int M, int N, int K, int split, int tri, int ctas, const float* A,
                                       const float* B, float* C, float* ms);

/* Allocation-free variant of psdp_tc_gemm_check (dtype 0); the paper has no
 * counterpart.  For callers that cannot allocate device memory where they need
 * the product: allocator or memory-pool callbacks (an allocation there would
 * re-enter the allocator) and hosts that give the library a fixed device budget.
 *  A: DEVICE pointer, M x K float32 row-major;  B: DEVICE pointer, N x K;
 *  C: DEVICE pointer receiving D = A B^T column-major (C[n*M + m]), M*N floats;
 *  split: 1 (TF32) or 3 (3xTF32);  stream: cudaStream_t (NULL = legacy stream).
 * The scratch (padded, TF32-split copies of A and B) is one static device array
 * of 8 MiB + 256 B that every GPU loading the library holds until exit, so
 * (M + N) * Kpad must not exceed 2^20, Kpad = K rounded up to 64: larger sizes
 * give EINVAL before any device work.  Nothing is allocated: no cudaMalloc or
 * cudaFree, no allocating library routine.  Every call looks up the array's
 * device address on the current device and sets the GEMM kernel's shared-memory
 * limit there.  The call is synchronous: it returns after the product is
 * complete on `stream` (it reads the kernel's timeout flag back and waits for
 * the stream).  Every call shares the array; calls that
 * overlap on the GPU (other host threads, other streams) race.  An unread CUDA
 * error left by earlier work gives ECUDA before anything is enqueued and stays
 * pending for its owner.  Errors: EINVAL, ECUDA, ETIMEOUT (bounded wait). */
psdp_status psdp_tc_gemm_noalloc(int M, int N, int K, int split, const float* A, const float* B, float* C,
                                 void* stream);

/* Measure this GPU's FP64 FMA throughput with a short dependent-chain kernel;
 * *tflops receives FP64 TFLOP/s (2 flops per FMA). */
psdp_status psdp_fp64_peak(int device, double* tflops);

/* FP64 throughput of this GPU by two short kernels: *dfma_tflops from
 * independent FMA chains on the FP64 pipe, *dmma_tflops from the FP64
 * tensor-core instruction (mma.sync m8n8k4 .f64, 512 flops a warp each).  The
 * FP64 roofline of the library's kernels takes the larger. */
psdp_status psdp_fp64_peaks(int device, double* dfma_tflops, double* dmma_tflops);

/* Self-test of the FP64 product by the Ozaki scheme on the BF16 tensor cores
 * (Ozaki, Ogita, Oishi & Rump 2012; the engine of the FP64 contractions of the
 * large workloads; no counterpart in the paper).  A: M x K, B: N x K row-major
 * float64 host arrays, K <= 2048; C: N x M column-major (C[j*M + i]), in/out:
 * C <- alpha A B^T + beta C, only the elements with i >= j when lower.  Each
 * row is split into eight BF16 digits of 7 bits below its own power-of-two
 * scale; the 36 digit-pair products are exact in the tensor cores' FP32
 * accumulation and are summed in int64 and FP64 (depth windows of 384, summed
 * in FP64): the error of each element is at most
 * K 2.8 2^(e_i + f_j - 56) + 2^-53 |(AB^T)_ij| per window, where 2^e_i is the
 * power of two just above max|A_i| (so at most K 2^-52.5 max|A_i| max|B_j|).  Allocates its
 * own scratch.  Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT (bounded wait). */
psdp_status psdp_ozaki_gemm_check(int M, int N, int K, const double* A, const double* B, double* C, double alpha,
                                  double beta, int lower);

void psdp_destroy(psdp_ctx* c);
const char* psdp_strerror(psdp_status s);

#ifdef __cplusplus
}
#endif
#endif /* POLYA_SDP_H */
