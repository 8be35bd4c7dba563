/*
 * xm.h - C ABI of libxm: the data-parallel hot path of XM (scaled bundle adjustment solved
 * as an SDP by Burer-Monteiro factorisation, a Riemannian trust-region method and a dual
 * certificate), for NVIDIA B300 (sm_103a).
 *
 * Notation follows the paper: N cameras, M landmarks, E observations (i, k, u_ik, w_ik),
 * n = 3N.  The BM factor U = [Rbar_1 ... Rbar_N] (r x 3N, Prop. 4) is exchanged as
 * Y = U^T, an n x r row-major array of doubles (camera i owns rows 3i..3i+2, the "world"
 * dimension r is fastest).  Camera 0 is the anchor (the paper's camera 1: R = I, s = 1).
 *
 * Conventions for every entry point
 *   - Array arguments are DEVICE pointers owned by the caller unless the name ends in
 *     _host; the library never frees them and never keeps them after the call returns.
 *   - Work is issued on the stream given to xm_create.  Calls that must read scalars
 *     back (solve, certify, build, the pipeline) synchronise that stream before returning;
 *     xm_qy is asynchronous.
 *   - Errors are returned as xm_status; xm_last_error() gives a message for the calling
 *     thread.  No call traps or aborts the device: device-side checks raise an error word
 *     that the host turns into a status.  On error, output arrays are unspecified.
 *   - Not thread-safe per context; distinct contexts may be used from distinct threads.
 */
#ifndef XM_H_
#define XM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XM_ABI_VERSION 3
#define XM_MAX_RANK 8   /* largest BM rank r the kernels handle (Alg. 1 stops there) */

typedef struct xm_ctx xm_ctx;   /* opaque: device, stream, workspaces */
typedef struct xm_qmat xm_qmat; /* opaque: the reduced data matrix Q on the device */

typedef enum xm_status {
  XM_OK = 0,
  XM_EINVAL = 1,        /* bad argument or observation (index range, w <= 0, NaN) */
  XM_EDISCONNECTED = 2, /* view graph not connected: Q_tp rank < N+M-1 (App. A lemma) */
  XM_ECUDA = 3,         /* CUDA runtime / library error */
  XM_ENOMEM = 4,        /* device allocation failed */
  XM_ENOCONV = 5,       /* iteration or time limit reached; best iterate returned */
  XM_ENUMERIC = 6,      /* NaN/Inf in the objective or gradient */
  XM_ETIMEOUT = 7,      /* a bounded device-side wait gave up (kernel pipeline stall) */
  XM_ENOTCERT = 8       /* lambda_min(Z) < -tau at r_max: results filled, not certified */
} xm_status;

/* Precision modes (arithmetic of the Q.Y sweeps).
 * XM_FP64:        every sweep, vector and scalar in FP64 (Q stored FP64).
 * XM_FP32_BULK:   RTR-tCG in FP32 (Q stored FP32), then an FP64 polish (FP64 gradient and
 *                 objective, FP32 Hessian-vector products) and the FP64 certificate.
 * XM_BF16Q_BULK:  as XM_FP32_BULK but the tCG Hessian-vector products read Q stored in
 *                 BF16 (FP32 accumulation); gradients and objectives use FP32/FP64 Q. */
typedef enum xm_prec { XM_FP64 = 0, XM_FP32_BULK = 1, XM_BF16Q_BULK = 2 } xm_prec;

/* Storage copies of Q that xm_build_Q keeps (bit mask). */
#define XM_STORE_FP64 1u   /* FP64 packed upper-triangle tiles (needed by XM_FP64, polish) */
#define XM_STORE_FP32 2u   /* FP32 packed tiles */
#define XM_STORE_BF16 4u   /* BF16 packed tiles */
#define XM_STORE_ALL  7u   /* the three dense copies */
#define XM_STORE_FACTORED 8u /* the factored operator (App. A in product form, see xm_qfact_create):
                                every FP64 product of a Q without XM_STORE_FP64 goes through it
                                (FP64-mode solves, the mixed modes' FP64 polish, certificates,
                                rounding).  With no dense bit set, Q itself is never formed (10155
                                cameras: 1.2 GB resident instead of 3.8 GB of FP64 tiles); solves
                                then run in XM_FP64 and the block-Jacobi preconditioners (precond,
                                the LOBPCG certificate) read the FP32 tiles when there are any */

typedef struct xm_opts {
  int r0;                  /* initial BM rank, 1 <= r0 <= XM_MAX_RANK (Alg. 1 uses 3);
                              default 4                                                     */
  int r_max;               /* staircase cap, r0 <= r_max <= XM_MAX_RANK (default XM_MAX_RANK) */
  int prec;                /* xm_prec (default XM_FP32_BULK)                                */
  double grad_tol_rel;     /* final stop: ||rgrad|| <= grad_tol_rel * ||rgrad(Y0)||
                              (default 1e-11)                                                */
  double bulk_tol_rel;     /* mixed modes: hand over to the FP64 polish at this tolerance
                              (default 1e-9)                                                 */
  double cert_tau_rel;     /* certified iff lambda_min(Z) >= -cert_tau_rel * lambda_max
                              (default 1e-6)                                                 */
  int max_outer;           /* RTR iterations per rank (per phase; default 300)             */
  int max_tcg;             /* tCG iterations per RTR step (default 200); steps of the FP32
                              bulk phase stop at min(max_tcg, 60)                          */
  int max_polish;          /* FP64 polish RTR iterations (mixed modes; default 20)         */
  int lanczos_max;         /* Krylov dimension cap of the certificate (default 800)        */
  double lanczos_tol;      /* Ritz residual / |theta_max| stop for lambda_min (default 1e-8) */
  double time_limit_s;     /* wall-clock cap of xm_solve (<= 0: none; default 0)           */
  uint64_t seed;           /* Lanczos start vector and init_jitter fill (default 12345)    */
  int verbose;             /* 0 silent (default), 1 per rank, 2 per RTR iteration (stderr)  */
  double init_jitter;      /* start = Alg. 1's [I_3, ..., I_3] padded to rank r0, plus this
                              amplitude times a seeded uniform(-1, 1) fill of the extra
                              columns (0: the padded start exactly; a zero column confines
                              rank-r0 RTR to the rank-3 subspace); default 0.1              */
  double scale_reg;        /* App. D scale regularisation: objective tr(QX) + scale_reg *
                              sum_{i>=2} (X_{3i,3i} - 1)^2 (the third diagonal entry of every
                              non-anchor block, paper's 1-based indexing); Z, the dual value
                              and the suboptimality bounds follow App. D / App. E.  0 (the
                              default): the plain objective of Eq. 17.  Must be >= 0.        */
  int precond;             /* tCG preconditioner: 0 plain Steihaug-Toint tCG (Sec. 3.2);
                              1: block Jacobi z_i = P(B_i^-1 r_i), B_i = 2 Q_ii (eigenvalues
                              clamped at 1e-6 of the largest), trust region in the B-norm
                              (halves the sweeps on the 1934-camera workload, slower on the
                              10155-camera one); 2 (default): adaptive, plain until three tCG
                              solves in a row stop at max_tcg, block Jacobi from then on     */
  int bulk_stall;          /* mixed modes, hand-over from the FP32 bulk phase to the FP64
                              polish before bulk_tol_rel when FP32 has stopped converging (both
                              rules only once ||rgrad|| <= 1e-6 ||rgrad(Y0)||; the polish starts
                              from the bulk's trust radius).  -1 (default): automatic, at the FP32 noise
                              floor: the running minimum of ||rgrad|| has not halved over 15
                              outer steps and the last three tCG solves stopped at max_tcg.
                              k > 0: when the best objective has not improved by
                              more than the ratio test's FP32 noise allowance over k outer steps.
                              0: run the bulk to bulk_tol_rel or max_outer.  Default -1.
                              -1 <= bulk_stall <= max_outer                                   */
  int cert_lobpcg;         /* certificates with FP32 Z products (mixed modes): 1 (default)
                              finds lambda_min(Z) on range(Y)^perp by block-Jacobi preconditioned
                              LOBPCG (blocks of 4, stop at a Ritz residual <= 1e-6 lambda_max,
                              lambda_max from 40 Lanczos steps; Lanczos if it does not converge
                              in 300 iterations); 0: Lanczos to lanczos_tol                     */
  double bf16_hvp_until;   /* XM_FP32_BULK with a BF16 copy of Q (XM_STORE_BF16): the bulk
                              phase's Hessian products read the BF16 tiles (the tensor-core
                              sweep, half the bytes) while ||rgrad|| > bf16_hvp_until *
                              ||rgrad(Y0)||, the FP32 tiles after; gradients, objective and
                              ratio test stay FP32.  0 (default): FP32 products throughout.
                              Must be >= 0; > 0 needs the BF16 copy (XM_EINVAL otherwise)    */
} xm_opts;

typedef struct xm_info {
  double f;                /* tr(Q Y^T Y) at the returned Y, FP64 (Eq. 17 objective)        */
  double grad_norm;        /* ||rgrad|| at the returned Y, FP64                              */
  double lambda_min;       /* lambda_min(Z), Z = Q - blockdiag(Lambda) (Thm. 1), FP64 Ritz  */
  double lambda_min_deflated; /* smallest Ritz value of Z on range(Y)^perp                  */
  double lambda_max;       /* largest Ritz value of Z (scale of the tolerance tau)           */
  double dual;             /* sum b_i y_i = tr(Lambda_0)                                     */
  double rho_hat;          /* objective of the rounded SO(3) solution (Eq. 5)                */
  double eta;              /* Eq. 18 relative suboptimality                                   */
  double eta_robust;       /* App. E bound with min(0, lambda_min) tr(X)                      */
  int rank;                /* BM rank r of the returned Y                                    */
  int certified;           /* 1 iff lambda_min >= -tau                                       */
  int n_sweeps;            /* Q.Y sweeps of every precision                                  */
  int n_sweeps_fp64;       /* of which FP64                                                  */
  int n_outer, n_tcg, n_lanczos, n_escapes;
  double t_solve_s, t_cert_s, t_build_s;
  double qy_ms_fp32, qy_ms_fp64; /* mean device time of one r-column sweep, when measured   */
  int lanczos_converged;   /* 1 iff the last certificate's Ritz residual met lanczos_tol (0: it
                              stopped at the Krylov cap lanczos_max; the decision then rests on an
                              unconverged Ritz value)                                           */
} xm_info;

/* ---- context ---------------------------------------------------------------------- */
int         xm_abi_version(void);
void        xm_default_opts(xm_opts* opts);
/* device: CUDA ordinal; stream: a cudaStream_t (NULL = legacy default stream). */
xm_status   xm_create(xm_ctx** out, int device, void* stream);
void        xm_destroy(xm_ctx* ctx);
const char* xm_last_error(void);
xm_status   xm_sync(xm_ctx* ctx);

/* Self-check of the failure path that every pipelined kernel shares (the paper has no
 * counterpart: its solver has no device-side waits).  Each wait of a CTA on its copy pipeline is
 * a bounded poll of an mbarrier; when the bound runs out the kernel raises a timeout flag in the
 * context's device error word, stops waiting and returns, and the calling entry point reports
 * XM_ETIMEOUT.  This call runs that wait in isolation: one CTA initialises an mbarrier for one
 * arrival and waits for its first phase with at most `polls` polls (1 <= polls <= 2^24, the
 * kernels' own bound).  arrive = 1: the CTA arrives first, the wait completes, XM_OK.
 * arrive = 0: nothing arrives, the wait gives up, XM_ETIMEOUT; no copy is in flight and the
 * context stays usable.  Synchronous; XM_EINVAL for polls out of range. */
xm_status   xm_selftest_wait(xm_ctx* ctx, long long polls, int arrive);

/* ---- Q construction (Prop. 1, App. A) ------------------------------------------------
 * Q = P - Bbar Sbar^{-1} Bbar^T with P = Q1 - V2 Q3^{-1} V2^T, B = V1 - V2 Q3^{-1} V3^T,
 * S = Q2 - V3 Q3^{-1} V3^T (landmarks eliminated, then translations with t_0 = 0); equal to
 * the printed A^T Q_tp A + V_tp A + A^T V_tp^T + Q1.  FP64 arithmetic throughout.
 * cam, lmk: int32[E]; ukp: double[E][3] (u_ik, camera frame); w: double[E] (> 0).
 * Observations may come in any order; landmarks with one observation contribute zero.
 * Fails with XM_EINVAL on out-of-range indices, w <= 0 or non-finite values, and with
 * XM_EDISCONNECTED when the view graph is not connected.  store_mask: XM_STORE_*.
 * The returned handle owns its device memory until xm_free_Q. */
xm_status xm_build_Q(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam,
                     const int32_t* lmk, const double* ukp, const double* w,
                     unsigned store_mask, xm_qmat** out);
/* Arithmetic of the translation elimination that ends xm_build_Q (App. A): the Cholesky factor
 * L of the anchored translation block (N^3 / 3 flops), C = L^{-1} Bbar^T (3 N^3 flops) and the
 * symmetric rank-(N-1) update Q = P - C^T C (9 N^3 flops; 9.4 TFLOP at N = 10155): the build's
 * dense contractions.
 * XM_BUILD_FP64:       the library's own FP64 kernels (blocked Cholesky, substitution, tiled
 *                      products) on the FP64 units.
 * XM_BUILD_SPLIT_BF16: the dense products on the BF16 tensor cores by error-free digit splitting
 *                      (Ozaki et al. 2012): each operand vector as 8 signed 7-bit digits scaled by
 *                      a power of two, exact FP32 accumulation of the digit products, int32 and
 *                      FP64 recombination; normwise as accurate as FP64 products (error below
 *                      2^-56 sqrt(K) |u| |v| per dot product).  The factorisation and the
 *                      triangular solve are blocked (256- and 1024-row diagonal blocks, panels by
 *                      the library's FP64 kernels, the trailing and block updates on the tensor
 *                      cores).  Needs N - 1 <= 16640.
 * XM_BUILD_AUTO:       XM_BUILD_SPLIT_BF16 when 512 <= N <= 16641, else XM_BUILD_FP64 (default).
 * The landmark elimination stays in FP64 either way. */
#define XM_BUILD_AUTO 0
#define XM_BUILD_FP64 1
#define XM_BUILD_SPLIT_BF16 2
/* Select the arithmetic for later xm_build_Q calls on ctx (XM_EINVAL for an unknown mode). */
xm_status xm_set_build_mode(xm_ctx* ctx, int mode);
/* Which arithmetic built q (XM_BUILD_FP64 or XM_BUILD_SPLIT_BF16; XM_BUILD_AUTO when N = 1 and
 * there was no translation elimination) and the device seconds of its Cholesky factor,
 * triangular solve, rank-(N-1) update and packing (either pointer may be NULL). */
xm_status xm_qmat_build_info(const xm_qmat* q, int* path, double* t_update_s);
/* Q from a dense symmetric n x n FP64 array (device, row-major); for tests. */
xm_status xm_qmat_from_dense(xm_ctx* ctx, int N, const double* Q, unsigned store_mask,
                             xm_qmat** out);
/* Copy Q back as a dense symmetric n x n FP64 row-major array (device); needs the FP64
 * copy. */
xm_status xm_qmat_to_dense(xm_ctx* ctx, const xm_qmat* q, double* Q_out);
xm_status xm_qmat_dims(const xm_qmat* q, int* N, int* n, unsigned* store_mask);
xm_status xm_free_Q(xm_ctx* ctx, xm_qmat* q);

/* ---- one sweep (Sec. 3.2, Euclidean Hessian-vector product) ---------------------------
 * W = Q Y for an n x r row-major Y, r in [1, XM_MAX_RANK].  prec picks the stored copy:
 * XM_FP64 reads FP64 Q with double Y/W; XM_FP32_BULK reads FP32 Q, XM_BF16Q_BULK BF16 Q,
 * both with float Y/W.  Asynchronous on the context stream. */
xm_status xm_qy(xm_ctx* ctx, const xm_qmat* q, int prec, int r, const void* Y, void* W);

/* The same sweep as xm_qy without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot let a library allocate device memory, such as
 * applications whose device memory is owned by their own pool allocator, or latency-bound
 * loops that cannot afford an allocation's implicit synchronisation.  The padded copies of Y
 * and W live in one fixed 4 MiB device array inside the library (held on every GPU that loads
 * it until the process exits); 2 * n_pad * R * sizeof(element) must fit, n_pad = n rounded up
 * to a multiple of 128 and R = 1, 4 or 8 the padded width of r (for example every precision and
 * r <= 8 at 10155 cameras).  Larger sizes are rejected with XM_EINVAL (use xm_qy).  The first
 * call on a device looks up the array's device address; make it before any stream capture.
 * The address is kept for the life of the process: after cudaDeviceReset on a device, do not
 * call this entry point on that device again.
 * All calls share the array: calls whose work overlaps on the GPU race.  Asynchronous on the
 * context stream. */
xm_status xm_qy_noalloc(xm_ctx* ctx, const xm_qmat* q, int prec, int r, const void* Y, void* W);

/* ---- factored Q operator (App. A's elimination kept in product form; Prop. 1) -------------
 * Q Y without forming Q: for observation e = (i, k) with a_e = u_e^T Y_i, landmark means
 * m_k = sum_{e in k} w_e a_e / d_k (d_k = sum_{e in k} w_e), camera sums b_j = sum_{e in j}
 * w_e (a_e - m_k) (= Bbar^T Y), the optimal translations t = -Sbar^{-1} bbar (t_0 = 0) and
 * their landmark means tb_k,
 *   (Q Y)_i = sum_{e in i} w_e u_e (a_e - m_k + t_i - tb_k),
 * the least-squares residual of Eq. 3 for the columns of Y weighted by the keypoints (the
 * envelope theorem applied to Prop. 1's minimisation over t and p).  Per product four passes
 * over the observations and one packed symmetric product with -Sbar^{-1} ((N-1)^2 entries,
 * against (3N)^2 for Q); FP64 throughout, deterministic.
 * xm_qfact_create: observations as for xm_build_Q (device pointers, copied); sets up the
 * landmark- and camera-major copies of (u, w), 1 / d_k and the FP64 tiles of -Sbar^{-1} (Cholesky
 * factor, triangular inverse and product by the build's FP64-accurate digit-split tensor-core
 * arithmetic).  XM_EINVAL on bad observations, XM_EDISCONNECTED when Sbar is singular.  The
 * handle owns its device memory until xm_qfact_free.
 * xm_qy_factored: W = Q Y for an n x r row-major FP64 Y (1 <= r <= XM_MAX_RANK); W (n x r) is
 * overwritten.  Asynchronous on the context stream; one product at a time per handle (it keeps
 * its intermediate vectors).
 * xm_qfact_info: sizes, resident device bytes and set-up seconds (any pointer may be NULL). */
typedef struct xm_qfact xm_qfact;
xm_status xm_qfact_create(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam,
                          const int32_t* lmk, const double* ukp, const double* w, xm_qfact** out);
xm_status xm_qy_factored(xm_ctx* ctx, const xm_qfact* f, int r, const double* Y, double* W);
xm_status xm_qfact_info(const xm_qfact* f, int* N, int* M, int64_t* E, size_t* bytes,
                        double* t_setup_s);
xm_status xm_qfact_free(xm_ctx* ctx, xm_qfact* f);

/* Device time of one sweep, measured with CUDA events on the context stream after three
 * warm-up sweeps (Y filled with a fixed pattern, W zeroed before each sweep outside the timed
 * interval).  ms_mean / ms_min may be NULL.  Synchronous. */
xm_status xm_bench_qy(xm_ctx* ctx, const xm_qmat* q, int prec, int r, int iters, double* ms_mean,
                      double* ms_min);
/* Kernel launches issued by the most recent xm_solve / xm_certify call of this process. */
long xm_last_launch_count(void);

/* ---- solve (Alg. 1 + RTR-tCG, Sec. 3) -------------------------------------------------
 * Y0: NULL for Alg. 1's [I_3, ..., I_3] start padded with zero columns to rank r0, else an
 * n x r_in row-major start (made feasible by the retraction).  Outputs (device, may be NULL):
 * Y_out n x XM_MAX_RANK (columns >= rank are zero), R_out N x 3 x 3 and s_out N of the
 * rounded solution (Sec. 2.2), G_out N x 3 x 3 the rounded anchored blocks G_i = s_i R_i (the
 * scaled rotations of Eq. 4, row-major; what xm_backward differentiates).  Synchronous.  Returns
 * XM_ENOTCERT if the staircase stops at r_max without a certificate, XM_ENOCONV on the time
 * limit. */
xm_status xm_solve(xm_ctx* ctx, const xm_qmat* q, const xm_opts* opts, int r_in,
                   const double* Y0, double* Y_out, double* R_out, double* s_out, double* G_out,
                   xm_info* info);

/* ---- certificate (Thm. 1) ---------------------------------------------------------------
 * For a rank-r Y (n x r row-major): Lambda_i = P_i(sym((QY)_i Y_i^T)) / alpha_i, Z = Q -
 * blockdiag(Lambda), lambda_min(Z) by Lanczos with full reorthogonalisation on range(Y)^perp
 * (FP64 vectors and Ritz values).  Lambda_out: N x 3 x 3 (may be NULL); v_out: n (the Ritz
 * vector of lambda_min, may be NULL).  Synchronous. */
xm_status xm_certify(xm_ctx* ctx, const xm_qmat* q, const xm_opts* opts, int r,
                     const double* Y, double* Lambda_out, double* v_out, xm_info* info);

/* ---- end-to-end from host arrays --------------------------------------------------------
 * Copies the observations to the device, builds Q, solves, certifies and rounds, and
 * copies R (N x 3 x 3) and s (N) back.  Every pointer here is a HOST pointer. */
xm_status xm_pipeline_host(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam_host,
                           const int32_t* lmk_host, const double* ukp_host,
                           const double* w_host, const xm_opts* opts, double* R_host,
                           double* s_host, xm_info* info);

/* ---- adjoint of the certified optimum (implicit differentiation of Sec. 3's first-order
 * condition through the Q of App. A) ---------------------------------------------------------
 * Loss L(G) of the anchored blocks G_i = Y_0 Y_i^T (i >= 1; equal to s_i R_i of Sec. 2.2 at a
 * tight optimum with R_0 = I, s_0 = 1).  Given dL/dG, returns dL/du_e (E x 3) and dL/dw_e (E)
 * for the lifted keypoints u_e = d_e * bearing_e and the weights of Eq. 1 (dL/dd_e follows as
 * <dL/du_e, bearing_e>).  Steps: lambda with Hess[lambda] = P_Y(dL/dY) (CG on the Riemannian
 * Hessian of Sec. 3; the operator is positive semi-definite at a certified optimum), then
 * dL/dQ = -(lambda Y^T + Y lambda^T) pulled back to the observations by the envelope theorem
 * at the optimal translations and landmarks of Prop. 1:
 *   dL/du_e = -2 w_e (Y_i e_lambda + lambda_i e_Y),   dL/dw_e = -2 <e_lambda, e_Y>,
 * e_a = U_i^T u_e + t_i - p_k the least-squares residual of column set a (t_0 = 0).
 * Arguments (device pointers unless stated): q from xm_build_Q on the same observations, with
 * an FP64 copy (and an FP32 copy unless opts->prec == XM_FP64); Y n x ldy row-major, the
 * first r columns used (the Y_out of xm_solve, r = info.rank); cam, lmk, ukp, w as for
 * xm_build_Q; dL_dG N x 3 x 3 row-major (entry 0 ignored).  Outputs dL_dukp (E x 3), dL_dw (E)
 * and, if not NULL, lam (n x r).  opts: prec XM_FP64 runs the CG on the FP64 operator; any
 * other value runs FP32 inner CG (at most max_tcg iterations per pass) inside FP64 residual
 * refinement (at most max_polish passes) until ||res|| <= grad_tol_rel ||P_Y(dL/dY)||, or
 * until a pass no longer halves ||res|| (the floor set by the stationarity of Y; XM_OK if
 * ||res|| <= 1e-6 ||P_Y(dL/dY)|| then, else XM_ENOCONV);
 * scale_reg must be the value the solve used (App. D's term enters the Hessian).
 * Allocates an N x N FP64 work matrix (the Cholesky factor of the anchored camera block) and
 * O(E + n) more, freed before return.  Synchronous.  Returns XM_ENOCONV (outputs written,
 * info->res_rel says how far) when the refinement cap is reached, XM_EDISCONNECTED if the
 * camera block is singular, XM_EINVAL on bad arguments. */
typedef struct xm_adj_info {
  double res_rel;          /* ||P_Y(dL/dY) - Hess[lambda]|| / ||P_Y(dL/dY)||, FP64 operator  */
  double g_norm;           /* ||P_Y(dL/dY)||                                                   */
  double grad_norm_Y;      /* ||rgrad|| at Y (the solve's stationarity, FP64)                  */
  int n_refine;            /* FP64 residual passes after the first                            */
  int n_cg;                /* inner CG iterations over all passes                             */
  int n_sweeps_fp32, n_sweeps_fp64;
  double t_lambda_s;       /* wall time of the adjoint solve                                   */
  double t_resid_s;        /* wall time of the residual pull-back (incl. the Cholesky)         */
  double t_total_s;
  long launches;           /* kernel launches of this call (library calls not counted)        */
  int dense_precond;       /* 1: CG preconditioned by the explicit FP32 inverse of the dense
                              Z + gamma Pi_Y (n <= 40000), packed like Q and applied by the
                              sweep; 0: by Z's 3 x 3 diagonal blocks                          */
  double gamma;            /* curvature given to range(Y) by the dense preconditioner          */
  double t_precond_s;      /* wall time of forming the preconditioner (part of t_lambda_s):
                              dense Z + gamma Pi_Y, its inverse (xm_spd_inverse), packing     */
} xm_adj_info;

xm_status xm_backward(xm_ctx* ctx, const xm_qmat* q, const xm_opts* opts, int r, const double* Y,
                      int ldy, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                      const double* ukp, const double* w, const double* dL_dG, double* dL_dukp,
                      double* dL_dw, double* lam, xm_adj_info* info);

/* In-place inverse of a dense symmetric positive definite FP32 matrix: the adjoint's
 * preconditioner (Z + gamma Pi_Y)^{-1} above (the paper has no adjoint; Z is the certificate
 * matrix of Sec. 3).  A: device, n x n column-major with leading dimension lda >= n, both
 * triangles set; overwritten by A^{-1} (both triangles).  Block inversion by Schur complements
 * (blocks split near n / 2 at multiples of 128; Gauss-Jordan below 129 rows); the
 * products, n^3 / 2 multiply-adds in all, run on the BF16 tensor cores with every FP32 operand
 * split into three BF16 digits and FP32 accumulation (the accuracy of FP32 products).  Allocates
 * about 1.1 n^2 floats of scratch, freed before return.  Synchronous.  XM_ENUMERIC when a pivot
 * is not positive (A not numerically positive definite; A is then undefined), XM_EINVAL on bad
 * arguments. */
xm_status xm_spd_inverse(xm_ctx* ctx, int n, float* A, int lda);

/* ---- translations and landmarks (Eq. 7), per-measurement residuals, XM^2 (Sec. 5) --------
 * xm_recover_tp: for rotations R (N x 3 x 3 row-major) and scales s (N), the least-squares
 * translations (t_0 = 0) and landmarks of Eq. 3, in FP64: t_out N x 3, p_out M x 3 (a landmark
 * without observations gets 0), res2_out E (w_e ||s_i R_i u_e + t_i - p_k||^2); any output may
 * be NULL.  Device pointers; synchronous.  XM_EDISCONNECTED if the anchored camera block is
 * singular. */
xm_status xm_recover_tp(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                        const double* ukp, const double* w, const double* R, const double* s,
                        double* t_out, double* p_out, double* res2_out);
/* xm_solve_xm2: XM^2 (running twice): build Q, solve, recover (t, p), drop the floor(drop_frac E)
 * measurements with the largest Eq. 3 terms (ties by the lower index), then build and solve
 * again on the rest.  The paper does not say what happens when the cut splits the view graph
 * (a camera, even the anchor, whose every measurement was dropped): the second solve then runs
 * on the connected component with the most cameras (ties: the one holding the lowest camera
 * index), re-indexed and anchored at its lowest-index camera (R = I, s = 1, t = 0 there);
 * cameras outside it get R = 0 and s = 0 (a solved camera always has s > 0), t = 0, and
 * landmarks outside it p = 0.  Outputs (device) of the second solve: R_out, s_out, t_out,
 * p_out (may be NULL); keep_out (E bytes, may be NULL): 1 for a measurement used by the second
 * solve.  info_first / info_second (host, may be NULL).  Returns the second solve's status;
 * XM_EDISCONNECTED only if the full view graph is disconnected. */
xm_status xm_solve_xm2(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                       const double* ukp, const double* w, const xm_opts* opts, double drop_frac,
                       double* R_out, double* s_out, double* t_out, double* p_out,
                       unsigned char* keep_out, xm_info* info_first, xm_info* info_second);

/* ---- batched solve of many independent scenes (serving-style batches) ------------------
 * Alg. 1 / Sec. 3.2 / Thm. 1 / Sec. 2.2 for every scene of a batch in one persistent launch:
 * each CTA takes the next scene of a work queue (descending size) and runs its whole
 * staircase with xm_solve's FP32-bulk schedule (FP32 RTR-tCG, quick certificate, FP64-gradient
 * polish, Lanczos certificate with FP64 vectors, FP64 stationarity check, rounding).  A scene
 * that needs rank > 4 is finished by a second (rank-8) persistent kernel in the same graph.
 *
 * xm_batch_create copies every scene's Q (each from xm_build_Q with an FP64 copy) into dense
 * full FP32 and FP64 row-major copies (rows padded to a multiple of 4 columns) owned by the
 * batch; the xm_qmat handles stay the caller's.  Scene size is limited by shared memory:
 * 2 * 8 * ldq_max * 8 bytes of sweep staging plus the Krylov work must fit the 227 KB of a CTA
 * (about 3N <= 1300; checked, XM_EINVAL otherwise).  The Krylov work is shared-memory resident,
 * so the batched certificate uses min(lanczos_max, 400) steps at most. */
typedef struct xm_batch xm_batch;

typedef struct xm_batch_info {
  double f, grad_norm, lambda_min, lambda_min_deflated, lambda_max, dual, rho_hat, eta, eta_robust;
  unsigned long long t_begin_ns, t_end_ns; /* device clock when the scene started / finished  */
  unsigned long long t_cert_ns, t_polish_ns; /* device time in the certificates / FP64 polish  */
  int N;                   /* cameras                                                          */
  int status;              /* xm_status of this scene (XM_OK, XM_ENOTCERT, XM_ENOCONV)         */
  int rank, certified, n_sweeps, n_sweeps_fp64, n_outer, n_tcg, n_lanczos, n_escapes;
} xm_batch_info;

xm_status xm_batch_create(xm_ctx* ctx, int S, const xm_qmat* const* qs, xm_batch** out);
xm_status xm_batch_free(xm_ctx* ctx, xm_batch* b);
/* Autotuner of the block-row tiling of the per-scene sweep: times `reps` FP32 sweeps of every
 * scene for each candidate (rows per warp, 16-byte column chunks per lane and step) in
 * {(2,4), (4,1), (4,2), (4,4), (8,1), (8,2)} and keeps, per scene-size class (3N <= 150, <= 450,
 * <= 900, larger), the fastest; tile_out (8 ints: rows, chunks per class; may be NULL)
 * receives the choice.  Run by xm_solve_batched on first use if not called before. */
xm_status xm_batch_autotune(xm_ctx* ctx, xm_batch* b, int reps, int* tile_out);
/* Teams for large scenes.  A scene with n = 3N >= n_min rows runs on a thread-block cluster of
 * cs CTAs that execute the same solve and split the rows of every Q product between them,
 * exchanging the results through distributed shared memory (results bit-identical to cs = 1);
 * the queue is ordered by size, and at the first smaller scene each cluster splits into single
 * CTAs for the rest of the batch.  cs in {1, 2, 4}, or 0 (the default): 2.  n_min >= 0, or 0
 * (the default): the smallest n with n^2 >= sum over scenes of n^2 / (SM count), i.e. the scenes
 * whose products alone outweigh one SM's share; no cluster launch when no scene reaches it.
 * With both automatic (cs = 0, n_min = 0), when at least two scenes reach 1.8 times that n, those
 * (at most one per 16 SMs) run on 4-CTA clusters in a launch beside the pairs, which then start at
 * 1.3 times it; both launches go on with single CTAs from one shared queue (still bit-identical).
 * XM_EINVAL for other values.  Takes effect at the next xm_solve_batched. */
xm_status xm_batch_cluster(xm_ctx* ctx, xm_batch* b, int cs, int n_min);
/* The CUDA graph that the last xm_solve_batched replayed: *launches (may be NULL) receives its
 * kernel launches per call (one rank-4 launch, or the 4-CTA and 2-CTA launches side by side; plus
 * the rank-8 launch when r_max > 4), *quad_scenes (may be NULL) the number of scenes it runs on
 * 4-CTA clusters beside the pairs.  XM_EINVAL before the first xm_solve_batched. */
xm_status xm_batch_launches(xm_ctx* ctx, const xm_batch* b, int* launches, int* quad_scenes);
/* Solves every scene.  opts: as xm_solve (r0 <= 4, r_max <= 8; prec is ignored: the FP32-bulk
 * schedule is used; time_limit_s applies per scene).  R_out (sum N x 3 x 3) and s_out (sum N),
 * device pointers, receive the rounded solutions scene after scene in the order of
 * xm_batch_create; info (host, S entries, may be NULL) the per-scene results.  The two
 * persistent launches are captured once in a CUDA graph (re-captured when opts or the output
 * pointers change) and replayed.  Synchronous.  Returns XM_ENOTCERT / XM_ENOCONV if any scene
 * ended so (see info[s].status). */
xm_status xm_solve_batched(xm_ctx* ctx, xm_batch* b, const xm_opts* opts, double* R_out,
                           double* s_out, xm_batch_info* info);

#ifdef __cplusplus
}
#endif
#endif /* XM_H_ */
