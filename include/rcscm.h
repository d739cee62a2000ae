/*
 * rcscm.h -- C ABI of the GB300 (sm_103a) library for rank-constrained spatial
 * covariance matrix (SCM) estimation, Kubo, Takamune, Kitamura, Saruwatari,
 * "Acceleration of rank-constrained spatial covariance matrix estimation for
 * blind speech extraction", APSIPA 2019.
 *
 * Model (Sec. II-B-1): x_ij = h_ij + u_ij, h_ij = a_i s_ij with
 * s_ij ~ N_c(0, r^(h)_ij), r^(h)_ij ~ IG(alpha, beta), and
 * u_ij ~ N_c(0, r^(u)_ij R_i), R_i = R'_i + lambda_i b_i b_i^H, where R'_i is the
 * rank-(M-1) noise SCM of Eq. (eq:rit) and b_i its unit null eigenvector.
 * The library estimates r^(h), r^(u), lambda by EM (Sec. II-B-2) with either
 * the second-stage accelerated rule (Algorithm 2, Sec. III-C-2) or the naive
 * rule (per-slot M x M inverse, Sec. II-B-2), then extracts the target with the
 * multichannel Wiener filter (Sec. II-A, Sec. IV-B).
 *
 * Conventions for every entry point:
 *  - Indices: i frequency bin (I), j frame (J), m microphone (M, 2 <= M <= 8).
 *  - "device" pointers are CUDA global-memory addresses on the current device;
 *    "host" pointers are ordinary CPU memory.  Complex numbers are interleaved
 *    (re, im) pairs: complex64 = 2 x float, complex128 = 2 x double.  All arrays
 *    are dense, row-major, without padding, in the index order given.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on it; calls return without synchronising unless stated.
 *  - The caller owns every buffer it passes.  A context owns its derived data
 *    (per-frequency constants, per-slot invariants, EM state, status word) and
 *    frees it in rcscm_destroy.
 *  - Every call returns an rcscm status code (RCSCM_OK = 0) and never aborts,
 *    traps or prints.  Errors detected on the device are collected in a status
 *    word that rcscm_status reads back.
 */
#ifndef RCSCM_H
#define RCSCM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define RCSCM_OK          0
#define RCSCM_EINVAL      1  /* bad shape, pointer, option or call order          */
#define RCSCM_ENULLSPACE  2  /* R'_i is not rank M-1 within options.null_tol, or a
                                caller-supplied b_i is not its null vector          */
#define RCSCM_ENONFINITE  3  /* a NaN/Inf or non-positive lambda_i was produced   */
#define RCSCM_ECLAMP      4  /* warning: some r^(u) reached options.ru_floor, or a
                                naive-rule r^(h) estimate fell below zero in FP32 and
                                was held at beta/(alpha+2)                         */
#define RCSCM_ECUDA       5  /* a CUDA runtime call failed                         */
#define RCSCM_ENOMEM      6  /* device allocation failed                           */
#define RCSCM_ETIMEOUT    7  /* reserved: a bounded device wait gave up            */
#define RCSCM_ECAPACITY   8  /* the problem does not fit the fixed scratch array of
                                rcscm_solve_noalloc (nothing was launched)         */
#define RCSCM_EBOUNDS     9  /* a row, slot or shape index check of the debug build
                                 (compiled with RCSCM_DEBUG) failed; the offending
                                 CTA skipped its work.  Never set by the normal build */

/* ---- update rules ------------------------------------------------------ */
#define RCSCM_RULE_ACCEL  0  /* second-stage accelerated rule, Algorithm 2         */
#define RCSCM_RULE_NAIVE  1  /* naive rule, Eqs. (eq:rijx)-(eq:M_ru), FP32 arithmetic per slot:
                                the explicit M x M inverse of every slot's model covariance
                                is taken in the whitened coordinates of R~_i (a per-row FP64
                                congruence with R~_i -> I), where the E-step and M-step
                                formulas are evaluated as printed                      */
#define RCSCM_RULE_NAIVE_F64 2 /* naive rule in FP64 arithmetic, printed coordinates (state
                                kept in FP32)                                           */
#define RCSCM_RULE_ACCEL1 3  /* first-stage accelerated rule, Algorithm 1: the per-slot
                                quadratic forms with the per-frequency inverses are
                                re-evaluated from x at every pass (O(M^2) per slot),
                                rows of up to 4096 frames                             */
#define RCSCM_RULE_NAIVE_PRINTED 4 /* naive rule in FP32 in the printed coordinates (the
                                per-slot inverse of R~^(x)_ij itself, then R~ P R~ etc.).
                                Kept to time the literal form: FP32 rounding in the
                                ill-conditioned R~ P R~ and r~_h^2 a^H P a terms costs it
                                1e-4 to 1e-2 relative error after one pass, and it relies
                                on the RCSCM_ECLAMP projections                         */

#define RCSCM_MAX_M       8  /* largest supported number of microphones          */
#define RCSCM_MAX_J_ACCEL 4096 /* longest row (frames) of the accelerated kernel  */

typedef struct rcscm_ctx rcscm_ctx;

/* One utterance.  The pointers are device pointers of the current device or
 * page-locked host memory (cudaHostAlloc / cudaHostRegister), which the kernels
 * then read in place over the host link; any other address (pageable host
 * memory, another device) makes rcscm_create return EINVAL.  They must stay
 * valid (and unchanged) from rcscm_create until rcscm_destroy; rcscm_setup reads
 * x, a, Rp, lambda0, rh0, ru0, rcscm_run reads x, rh0, ru0, and the naive and
 * first-stage rules re-read x at every iteration. */
typedef struct {
    int64_t I, J, M;
    const void*   x;        /* complex64  [I][J][M]  observed STFT x_ij                 */
    const void*   a;        /* complex128 [I][M]     steering vector a_i^(h)            */
    const void*   Rp;       /* complex128 [I][M][M]  R'_i^(u), Hermitian, rank M-1
                               (complex64 when rp_c64 = 1)                               */
    const double* lambda0;  /* [I] initial lambda_i, or NULL: the smallest nonzero
                               eigenvalue of R'_i (Sec. II-B-3)                          */
    const float*  rh0;      /* [I][J] initial r^(h)_ij (Eq. (eq:rhinit)), > 0            */
    const float*  ru0;      /* [I][J] initial r^(u)_ij (Eq. (eq:ruinit)), > 0            */
    const void*   b;        /* complex128 [I][M] the caller's unit null vector b_i of R'_i,
                               or NULL.  When given it is validated against the setup's
                               eigendecomposition (|R'_i b_i| <= 1e-6 |R'_i|_F |b_i| and
                               |b_i^H e_1| >= (1 - 1e-6) |b_i|, e_1 the eigenvector of the
                               smallest eigenvalue); a row that fails sets RCSCM_ENULLSPACE
                               in the status word.  The estimator uses e_1 either way, so
                               results do not depend on the phase the caller chose.      */
    int           rp_c64;   /* 0: Rp is complex128 (default); 1: Rp is complex64, read and
                               widened to FP64 by the setup                               */
} rcscm_problem;

typedef struct {
    int    rule;             /* RCSCM_RULE_ACCEL (default), RCSCM_RULE_NAIVE,
                                RCSCM_RULE_NAIVE_F64, RCSCM_RULE_ACCEL1 or
                                RCSCM_RULE_NAIVE_PRINTED                                */
    double alpha;            /* inverse-gamma shape, Table II: 1.1                      */
    double beta;             /* inverse-gamma scale, Table II: 1e-16                    */
    float  ru_floor;         /* lower bound applied to r^(u) (default FLT_MIN)          */
    double null_tol;         /* zero-eigenvalue test: mu_1 <= null_tol * mu_M (1e-6)   */
    int    block;            /* threads per row of the accelerated kernel: 0 = choose
                                by J, else 32, 64, 128, 256, 512 or 1024; rows may be
                                up to 8*block (block <= 512) or 4096 (1024) frames
                                long                                                   */
    int    iters_per_launch; /* 0: every iteration of one rcscm_iterate call in one
                                register-resident launch; k > 0: one launch per k
                                iterations, state streamed through HBM between them    */
    int    persistent;       /* 1: the accelerated kernel runs as a persistent grid of
                                resident CTAs that take rows (longest first) from an
                                atomic counter; 0 (default): one CTA per row            */
    int    ckpt_stride;      /* accelerated rule: k > 0 keeps the EM state entering every
                                k-th pass since the last rcscm_setup / rcscm_set_state
                                (a checkpoint) for rcscm_backward; 0 (default): none.
                                With k > 0, block 0 picks 128 (J <= 512) or 256 (J <=
                                2048), an explicit block must be 128 or 256, J <= 2048,
                                and rcscm_graph_create is not available                 */
    int    ckpt_max_iters;   /* with ckpt_stride > 0: most passes that may run between
                                two rcscm_setup / rcscm_set_state calls; sizes the
                                checkpoint memory, ceil(ckpt_max_iters / ckpt_stride)
                                states of 8 B per slot (plus the adjoint's scratch:
                                min(ckpt_stride, ckpt_max_iters) states, and 1.4 KB per
                                frequency row)                                           */
} rcscm_options;

/* Fill *opt with the defaults listed above. */
void rcscm_default_options(rcscm_options* opt);

/* Validate the shapes of n_probs utterances (uneven J and mixed M allowed),
 * allocate the context's device memory and upload its row tables on `stream`.
 * *ctx receives the new context (NULL on error).  No estimator work is done.
 * Errors: EINVAL (NULL pointer, M outside [2, 8], I or J < 1, J above
 * RCSCM_MAX_J_ACCEL for the accelerated rule, bad option), ENOMEM, ECUDA. */
int rcscm_create(rcscm_ctx** ctx, const rcscm_problem* probs, int n_probs,
                 const rcscm_options* opt, void* stream);

/* Per-frequency setup and per-slot invariants, then EM state initialisation.
 * Setup (FP64, Sec. II-B-1, Eq. (eq:riinv), (eq:taa), (eq:sap)): symmetrise R'_i,
 * Hermitian eigendecomposition, b_i = eigenvector of the smallest eigenvalue,
 * (R'_i)^+, lambda_i (Sec. II-B-3), tau^(aa)_i, sigma^(ab)_i.  Invariants (FP32,
 * Algorithm 2 before its loop; Eq. (eq:tax), (eq:txx), (eq:spx)): tau^(ax)_ij,
 * sigma^(bx)_ij and kappa_ij = tau^(xx)_ij - |tau^(ax)_ij|^2 / tau^(aa)_i >= 0.
 * State: r^(h) <- rh0, r^(u) <- ru0, lambda <- lambda0.  May be called again to
 * restart from the (possibly updated) input buffers.  A failed null-space test
 * is reported by rcscm_status as RCSCM_ENULLSPACE. */
int rcscm_setup(rcscm_ctx* ctx, void* stream);

/* Run n_iter EM passes (n_iter >= 0) of the context's rule on every utterance.
 * Accelerated rule: the repeat loop of Algorithm 2 (Sec. III-C-2) -- gamma~_ij
 * (eq:tal), r^(h) (eq:1st_rh), lambda_i (eq:1st_li, a mean over j), r^(u)
 * (eq:1st_ru with the new lambda_i).  Naive rule: E-step (eq:rijx)-(eq:E_hru)
 * with an explicit M x M inverse per slot, then M-step (eq:M_rh)-(eq:M_ru); in
 * FP32 its r_h estimate and b^H R^u b, non-negative in exact arithmetic, are held
 * at zero when rounding makes them negative (reported as RCSCM_ECLAMP).
 * First-stage rule: the repeat loop of Algorithm 1 (Sec. III-C-1), the same
 * updates with rho~_ax and the r^(u) numerator re-evaluated from x_ij at every
 * pass through the per-frequency inverses (Eq. (eq:riinv)). */
int rcscm_iterate(rcscm_ctx* ctx, int n_iter, void* stream);

/* Multichannel Wiener filter with the current state: the posterior mean
 * h_ij = r^(h) a a^H (R^(x)_ij)^{-1} x_ij = [r^(h) rho^(ax) / (r^(u) + r^(h) rho^(aa))] a_i.
 * h_out: complex64, the utterances concatenated in order, each [I][J][M]; device
 * memory or page-locked host memory (written in place), else EINVAL. */
int rcscm_extract(rcscm_ctx* ctx, void* h_out, void* stream);

/* The same work as rcscm_setup + rcscm_iterate(n_iter) + rcscm_extract(h_out),
 * in fewer launches.  rcscm_setup_freq runs the per-frequency part of
 * rcscm_setup alone (eigendecomposition, b, (R')^+, lambda_0, tau_aa, sigma_ab,
 * projection; Sec. II-B-1, Eq. (eq:riinv)).  rcscm_run then computes in ONE
 * kernel per row, from the initial state (rh0, ru0, lambda_0) whatever ran
 * before: the per-slot invariants from x (stored in the context, as rcscm_setup
 * does), n_iter passes of Algorithm 2 in registers, and the Wiener output h_out;
 * x is read once and the invariants and state are not re-read.  It needs the
 * accelerated rule, iters_per_launch = 0 and no checkpoints (else EINVAL), and
 * rcscm_setup_freq or rcscm_setup since the inputs last changed.  rcscm_solve =
 * rcscm_setup_freq + rcscm_run, or the three separate calls in any other
 * configuration.  Outputs, state and invariants are bitwise those of the
 * separate calls. */
int rcscm_setup_freq(rcscm_ctx* ctx, void* stream);
int rcscm_run(rcscm_ctx* ctx, int n_iter, void* h_out, void* stream);
int rcscm_solve(rcscm_ctx* ctx, int n_iter, void* h_out, void* stream);

/* Copy one utterance's state out of / into the context (device pointers:
 * rh, ru [I][J] float, lambda [I] float).  set_state accepts any of them NULL
 * (left unchanged).  Errors: EINVAL for a bad index. */
int rcscm_get_state(rcscm_ctx* ctx, int prob, float* rh, float* ru, float* lambda, void* stream);
int rcscm_set_state(rcscm_ctx* ctx, int prob, const float* rh, const float* ru,
                    const float* lambda, void* stream);

/* Setup results of one utterance (device pointers, any may be NULL):
 * b complex128 [I][M], lambda0 double [I], tau_aa double [I],
 * sigma_ab complex128 [I], mu double [I][M] (ascending eigenvalues of R'_i). */
int rcscm_get_setup(rcscm_ctx* ctx, int prob, void* b, double* lambda0, double* tau_aa,
                    void* sigma_ab, double* mu, void* stream);

/* Per-slot invariants of one utterance (device pointers, any may be NULL):
 * tau_ax complex64 [I][J], sigma_bx complex64 [I][J], kappa float [I][J]. */
int rcscm_get_invariants(rcscm_ctx* ctx, int prob, void* tau_ax, void* sigma_bx,
                         float* kappa, void* stream);

/* Synchronise `stream`, read and clear the device status word.  Returns the most
 * severe code seen since the last call (ENULLSPACE, ENONFINITE, then ECLAMP);
 * *flags (may be NULL) receives the raw bit set (bit k-1 for code k). */
int rcscm_status(rcscm_ctx* ctx, int* flags, void* stream);

/* Sizes: rows (sum of I), slots (sum of I*J), device bytes held by the context. */
int rcscm_info(const rcscm_ctx* ctx, int64_t* rows, int64_t* slots, int64_t* device_bytes);

/* Free the context (synchronises the device first).  NULL is accepted. */
void rcscm_destroy(rcscm_ctx* ctx);

/* Static, NUL-terminated description of a status code. */
const char* rcscm_strerror(int code);

/* Observed-data log posterior of the model of Sec. II-B-1 with the current state,
 * constants dropped: sum_ij [-log det R^(x) - x^H (R^(x))^{-1} x - (alpha+1) log r_h
 * - beta/r_h], one value per utterance into the host array value[n_probs].  Each
 * EM pass leaves it non-decreasing.  Synchronises `stream`. */
int rcscm_objective(rcscm_ctx* ctx, double* value, void* stream);

/* Autotuner of the accelerated kernel's launch shape: times n_iter_probe passes
 * for every valid (block in {32,...,1024}) x (persistent 0/1) on this context's
 * work list, restoring the EM state before each trial and at the end, and keeps
 * the fastest in the context's options (also returned through the non-NULL
 * pointers).  Results depend on the block size only through the order of the
 * lambda reduction.  Allocates temporary device memory; synchronises `stream`.
 * EINVAL for a naive-rule context. */
int rcscm_autotune(rcscm_ctx* ctx, int n_iter_probe, int* chosen_block, int* chosen_persistent, void* stream);

/* Capture one full solve step -- rcscm_solve(n_iter, h_out), i.e. setup,
 * n_iter passes and the Wiener filter -- as a CUDA graph owned by the context (replacing any
 * previous one); rcscm_graph_launch replays it on `stream`.  The graph keeps the
 * context's and h_out's device addresses; the problem buffers must keep them
 * too. */
int rcscm_graph_create(rcscm_ctx* ctx, int n_iter, void* h_out);
int rcscm_graph_launch(rcscm_ctx* ctx, void* stream);

/* Gradient of a real loss L of the Wiener estimate h (rcscm_extract with the
 * current state) with respect to x, a and R', through the K accelerated passes
 * run since the last rcscm_setup or rcscm_set_state, the Wiener filter, the
 * per-slot invariants and the per-frequency setup.  The paper defines no
 * gradient: this is reverse-mode differentiation of the computation of
 * Algorithm 2 (Sec. III-C-2), the posterior mean (Sec. II-A) and the setup of
 * Sec. II-B-1 / Eq. (eq:riinv).  Needs a context created with ckpt_stride > 0:
 * the state entering each pass is recomputed from the nearest checkpoint with
 * the forward kernel's code, bit for bit.  Per-slot adjoint arithmetic is FP32,
 * per-frequency FP64.  lambda0 and the initial variances are held constant (no
 * gradient flows into them, including the dependence of the default
 * lambda0 = mu_2 on R').  Device buffers, utterances concatenated in context
 * order:
 *   grad_h  complex64  like h_out ([I][J][M] each): dL/dRe h + i dL/dIm h;
 *   grad_x  complex64  like x ([I][J][M] each), same convention;
 *   grad_a  complex128 [I][M] each;
 *   grad_Rp complex128 [I][M][M] each: the gradient through the Hermitian part
 *           (R' + R'^H)/2 that the setup reads, itself Hermitian; it is the
 *           exact first-order gradient when the eigenvalues of R' are distinct.
 * Every output element is written.  Errors: EINVAL (NULL buffer, no checkpoints,
 * a block or row length the adjoint kernel does not support, passes run with a
 * different block since the last setup), ECUDA. */
int rcscm_backward(rcscm_ctx* ctx, const void* grad_h, void* grad_x, void* grad_a, void* grad_Rp, void* stream);

/* One-shot solve of a single utterance from HOST memory: copies x, a, Rp, rh0,
 * ru0 (same layouts as rcscm_problem, host pointers; lambda0 may be NULL) to the
 * device, runs setup, n_iter passes and the Wiener filter, and copies h_out
 * (complex64 [I][J][M]) and, when not NULL, rh, ru [I][J] and lambda [I] back to
 * host memory.  Allocates and frees its own device buffers; synchronous. */
int rcscm_solve_host(int64_t I, int64_t J, int64_t M, const void* x, const void* a,
                     const void* Rp, const double* lambda0, const float* rh0,
                     const float* ru0, const rcscm_options* opt, int n_iter,
                     void* h_out, float* rh, float* ru, float* lambda);

/* Solve one utterance without allocating any device memory.  (The paper has no
 * counterpart: this is a deployment variant of the accelerated solve.)
 *
 * For callers that cannot call cudaMalloc: a real-time audio thread, where an
 * allocation may synchronise the device and stall for an unbounded time, or a
 * host application that hands the library a fixed GPU memory budget and does
 * not let it allocate more.  The caller passes inputs (x, a, Rp, lambda0 (may
 * be NULL), rh0, ru0, same layouts as rcscm_problem, complex128 Rp) and
 * outputs: rh, ru [I][J] float (may alias rh0, ru0), lambda [I] float, h_out
 * complex64 [I][J][M], and status (an int that receives the status bits of
 * rcscm_status, or NULL).  Each is device memory of the current device or
 * page-locked host memory, as for rcscm_create; any other address (pageable
 * host memory, another device's memory) returns EINVAL before anything is
 * launched.  The work is the same as rcscm_create + rcscm_setup +
 * rcscm_iterate(n_iter) + rcscm_extract with opt->rule = RCSCM_RULE_ACCEL and
 * the options block and iters_per_launch; other rules, persistent != 0 and
 * ckpt_stride != 0 return EINVAL.  The work is enqueued on `stream`; the call
 * does not synchronise and never calls cudaMalloc, cudaFree or any allocating
 * routine.
 *
 * Working memory comes from one 32 MiB array in the library's device memory,
 * reserved on every GPU that loads the library's module until the process
 * exits.  With lazy module loading (the CUDA default) the module, and with it
 * the array, is loaded by the first call on each device; if the device has no
 * room for it that call returns RCSCM_ENOMEM.  A
 * problem needs about 1.5 KB per frequency bin plus 20 B per slot (I*J): for
 * example I = 1025, J = 1000 (about 22 MB) fits and I = 2049, J = 4000 does
 * not.  A problem that does not fit returns RCSCM_ECAPACITY before anything is
 * launched.  The first call on each device looks the array's address up (with
 * that device current) and caches it; make that first call before any stream
 * capture.  All calls on a device share the array: two calls whose GPU work
 * overlaps (for example on two streams) race and corrupt each other's results,
 * so serialise them.  Each call clears the parts of the array that must start
 * at zero and overwrites the rest. */
int rcscm_solve_noalloc(int64_t I, int64_t J, int64_t M, const void* x, const void* a, const void* Rp,
                        const double* lambda0, const float* rh0, const float* ru0,
                        const rcscm_options* opt, int n_iter, float* rh, float* ru, float* lambda,
                        void* h_out, int* status, void* stream);

/* Estimator inputs from the outputs of the ILRMA stage (Sec. II-A, Sec. II-B-1
 * Eq. (eq:rit), Sec. II-B-3 Eqs. (eq:rhinit), (eq:ruinit)).  ILRMA gives per
 * frequency i the demixing matrix W_i = (w_{i,1} ... w_{i,M})^H = A_i^{-1} and,
 * for the target source n_h, the NMF bases t_{ik} and activations v_{kj}.  For
 * each utterance this writes
 *   a    complex128 [I][M]     column n_h of W_i^{-1} (the target's steering vector),
 *   Rp   complex128 [I][M][M]  R'_i = (1/J) sum_j W_i^{-1} diag(|w_{i,n}^H x_ij|^2,
 *                              with 0 at n = n_h) W_i^{-H}, Eq. (eq:rit),
 *   rh0  float [I][J]          sum_k t_ik v_kj, Eq. (eq:rhinit),
 *   ru0  float [I][J]          (1/M) y^H (R'_i)^+ y with the back-projected noise
 *                              image y, Eq. (eq:ruinit), evaluated in its closed form
 *                              (1/M) sum_{n != n_h} |w_{i,n}^H x_ij|^2 / d_n, d_n the
 *                              mean power of output n,
 * in the layouts of rcscm_problem, so the buffers can be passed to rcscm_create
 * as they are (lambda_i then starts at the minimum nonzero eigenvalue of R'_i).
 * W_i^{-1} and R'_i are formed in FP64, the frame sums from FP32 products with
 * compensated accumulation.  Inputs and outputs are device memory or page-locked
 * host memory of the calling process; the caller owns them, and no output may
 * overlap an input.  The work of every utterance is enqueued on `stream` (one
 * launch per utterance) without synchronising.  Returns RCSCM_EINVAL, before anything is launched, for a bad
 * shape (M outside 2..RCSCM_MAX_M, K outside 1..256, n_h outside 0..M-1, I or J
 * below 1) or pointer.  `status` (a device int, or NULL) receives the status bits
 * of rcscm_status: RCSCM_ENULLSPACE's for a singular W_i or a noise output with
 * zero power (R'_i would not have rank M-1), RCSCM_ENONFINITE's for a non-finite
 * R'_i.  (The paper computes these inputs on the CPU before the iterations.) */
typedef struct {
    int64_t I, J, M, K;
    int64_t n_h;           /* index of the target source, 0 <= n_h < M */
    const void* x;         /* complex64 [I][J][M] observed STFT x_ij */
    const void* W;         /* complex128 [I][M][M] demixing matrices, row n = w_{i,n}^H */
    const float* T;        /* [I][K] NMF bases of the target source, t_{ik,n_h} */
    const float* V;        /* [K][J] NMF activations of the target source, v_{kj,n_h} */
    void* a;               /* out: complex128 [I][M] */
    void* Rp;              /* out: complex128 [I][M][M] */
    float* rh0;            /* out: [I][J] */
    float* ru0;            /* out: [I][J] */
} rcscm_ilrma;

int rcscm_ilrma_init(const rcscm_ilrma* u, int n_utt, int* status, void* stream);

/* Host-memory pipeline for utterances of one shape (I, J, M).  rcscm_host_create
 * allocates device buffers for one utterance and splits its frequency rows into
 * n_chunks contiguous ranges, each with its own context and stream (rows are
 * independent in every rule).  rcscm_host_run copies x, a, Rp, rh0, ru0 from host
 * memory (layouts of rcscm_problem), runs setup, n_iter passes of opt->rule and
 * the Wiener filter, and copies h_out (complex64 [I][J][M]) and, when not NULL,
 * rh, ru [I][J] and lambda [I] back; the copies of one chunk overlap the kernels
 * of another.  Host buffers should be page-locked for the copies to overlap.
 * lambda0 must be NULL (lambda_i starts at the smallest nonzero eigenvalue of
 * R'_i).  rcscm_host_run synchronises before returning and reports the most
 * severe status of the chunks.  Errors: EINVAL, ENOMEM, ECUDA, and the status
 * codes of rcscm_status. */
typedef struct rcscm_host rcscm_host;
int rcscm_host_create(rcscm_host** plan, int64_t I, int64_t J, int64_t M, const rcscm_options* opt, int n_chunks);
int rcscm_host_run(rcscm_host* plan, const void* x, const void* a, const void* Rp, const double* lambda0,
                   const float* rh0, const float* ru0, int n_iter, void* h_out, float* rh, float* ru,
                   float* lambda);
void rcscm_host_destroy(rcscm_host* plan);

#ifdef __cplusplus
}
#endif
#endif /* RCSCM_H */
