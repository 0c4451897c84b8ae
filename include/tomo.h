/*
 * tomo.h -- C ABI of the GB300 Toeplitz-structured spatio-angular MMSE
 * tomographic wave-front reconstructor (Ono et al., "Fast iterative
 * tomographic wave-front estimation with recursive Toeplitz reconstructor
 * structure for large scale systems").
 *
 * The library solves, per slope frame s (Eq. covIterative1 with the aperture
 * mask of Eq. SAap1),
 *
 *     W_s (Sigma_ss + Sigma_eta_eta) W_s^T zeta = s,
 *
 * by conjugate gradients whose every matrix-vector product applies Sigma_ss
 * through its two-level recursive block-Toeplitz (2RBT) structure (Sec. 2.D,
 * 2.E, Eq. mvm_ss): zero-pad -> 2-D FFT -> per-frequency (2 nGS) x (2 nGS)
 * block multiply -> inverse 2-D FFT -> crop and mask.  It then projects to
 * each target direction (Eq. covIterative2 / SAap2, Eqs. mvm_ps and
 * ToeplitzLGS):  phi_hat = W_phi Sigma_phi_beta_s zeta.
 *
 * Measurement model: Hudgin-like two-point slopes (Appendix A.2); slopes are
 * phase differences across a subaperture in radians at the wavelength of r0
 * (the paper's lambda/(2 pi d) factor is dropped; it cancels in the
 * reconstructor).  Turbulence: von Karman layers (Appendix A.2,
 * structure-function equation).  Laser guide stars see layer k through the
 * cone factor gamma = 1 - h_k / H (Sec. 2.D).
 *
 * Layouts (all row-major, C order):
 *   slope / zeta vector of one frame: guide stars in order, each
 *     [x-slopes over valid subapertures ; y-slopes over valid subapertures],
 *     valid subapertures listed row-major, k(i, j) = i*n + j (Sec. 2.E);
 *     N = 2 * n_gs * n_vs floats.  A batch is [batch][N].
 *   phase of one frame: [target][valid phase point, row-major over (n+1)^2];
 *     a batch is [batch][n_targets][n_vphi].
 *   masks returned by tomo_layout: n*n and (n+1)*(n+1) bytes, 1 = valid.
 *
 * Ownership: the caller owns every buffer passed in; the handle owns its
 * spectra, tables and workspaces.  Device-pointer entry points enqueue work on
 * the handle's stream and return without synchronising; *_host entry points
 * copy in, run and copy out, and return after the stream has finished.
 * Solves also synchronise their own private stream at each convergence check.
 * A handle keeps per-call workspaces: use it from one host thread at a time
 * (separate handles are independent, on one device or several). 
 *
 * Errors: every call returns a tomo_status; on failure nothing is written to
 * the outputs that the caller can rely on, except TOMO_ETIMEOUT from a solve
 * whose opts.deadline_ms ran out, which writes its outputs and per-frame
 * information as a normal return would.  A solve also returns TOMO_ETIMEOUT
 * when a bounded wait inside a kernel expired (a bulk copy that did not
 * complete; the kernel then returns early instead of hanging).  Per-frame
 * non-convergence is not an error: it is reported in tomo_frame_info.status.
 */
#ifndef TOMO_H
#define TOMO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TOMO_OK = 0,
    TOMO_EINVAL = 1,    /* bad argument or configuration                      */
    TOMO_ENOMEM = 2,    /* device or host allocation failed                   */
    TOMO_ECUDA = 3,     /* a CUDA runtime call failed                         */
    TOMO_ETIMEOUT = 4,  /* a bounded device wait expired                      */
    TOMO_ERANGE = 5     /* size beyond a compiled or configured maximum       */
} tomo_status;

/* Per-frame solver outcome (tomo_frame_info.status). */
enum {
    TOMO_FRAME_CONVERGED = 0,  /* FP64 true relative residual <= tol           */
    TOMO_FRAME_MAXIT = 1,      /* iteration limit (or opts.deadline_ms) first  */
    TOMO_FRAME_BREAKDOWN = 2,  /* p^T A p <= 0, or a NaN / infinity in the
                                  frame's slopes, warm start or iterates: the
                                  frame stops and returns its last iterate
                                  (the initial guess when its input is not
                                  finite); the other frames are not affected */
    TOMO_FRAME_FALLBACK_PLAIN_CG = 3 /* converged, after leaving the flexible
                                  iteration with the learned preconditioner
                                  (opts.precond = 2) for PCG with M alone     */
};

/* One guide star (Sec. 2 intro): direction alpha [rad] and altitude H [m];
 * H = 0 denotes a natural guide star at infinity.  noise_sigma [rad] is the
 * standard deviation of its slope noise: Sigma_eta_eta = sigma^2 I on its
 * slopes (Sec. 2.B, diagonal noise covariance). */
typedef struct {
    double alpha_x, alpha_y;
    double height;
    double noise_sigma;
} tomo_gs;

/* System description.  Arrays are read during tomo_create only. */
typedef struct {
    double D;              /* pupil diameter [m]                                 */
    double obstruction;    /* central obstruction, fraction of D (Sec. 2.F)       */
    int n;                 /* subapertures across, the same for every WFS         */
    int n_gs;              /* number of guide stars (>= 1)                        */
    const tomo_gs* gs;     /* [n_gs]                                              */
    int n_layers;          /* number of turbulent layers (>= 1)                   */
    const double* layer_h;     /* [n_layers] altitudes [m]                        */
    const double* layer_frac;  /* [n_layers] Cn^2 fractions, summing to 1         */
    double r0;             /* Fried parameter [m] at the slope wavelength         */
    double L0;             /* outer scale [m]                                     */
    int n_targets;         /* target directions (>= 1)                            */
    const double* target_x;    /* [n_targets] beta_x [rad]                        */
    const double* target_y;    /* [n_targets] beta_y [rad]                        */
    int fft_P;             /* padded FFT side for Sigma_ss, 0 = smallest valid,
                              < 0 = autotuned (see tomo_autotune_result)          */
    int fft_Pcos;          /* padded FFT side for Sigma_phi_s, 0 = smallest valid */
    int max_batch;         /* frames per call the workspaces are sized for        */
    int precond;           /* 1: also build the block-circulant preconditioner    */
    double precond_floor;  /* c of the preconditioner (see tomo_solve_opts), 0 = 3 */
    int mode_removal;      /* 1: remove tip, tilt and focus (Sec. 2.F, mode
                              removal; see tomo_solve)                           */
    int slope_model;       /* TOMO_SLOPE_HUDGIN (0) or TOMO_SLOPE_FRIED (1)         */
    const double* noise_cov;   /* NULL, or [n_gs][n][n][3] = s_xx, s_yy, s_xy:
                              per subaperture (row-major grid; entries outside
                              the pupil are ignored) the 2 x 2 covariance of its
                              x and y slope noise (elongated laser spots,
                              Sec. 2.F).  It replaces noise_sigma in
                              Sigma_eta_eta, and the preconditioner's floor
                              for a guide star becomes the mean of
                              (s_xx + s_yy) / 2 over its valid subapertures
                              (PCG needs 17-28 % fewer iterations than with
                              the blocks' smaller eigenvalue on the 16 x 16
                              system); noise_sigma is then not used.  Each
                              valid block must be
                              positive semidefinite (TOMO_EINVAL otherwise).
                              Read during tomo_create only. */
} tomo_config;

/* Slope model of the covariances (Appendix A; the paper compares both):
 * Hudgin-like, a slope is the phase difference between the midpoints of the
 * two subaperture edges across its direction; Fried, the mean of the
 * differences along the two edges parallel to it, i.e. over the four corners
 * with weights +-1/2 (it does not see the waffle mode of the corner grid).
 * The model changes the generators and spectra only; tip, tilt and focus
 * have the same slopes in both. */
enum { TOMO_SLOPE_HUDGIN = 0, TOMO_SLOPE_FRIED = 1 };

typedef struct {
    int n, n_gs, n_vs;     /* n_vs valid subapertures per WFS                     */
    int N;                 /* unknowns per frame = 2 n_gs n_vs                    */
    int n_vphi;            /* valid phase points                                  */
    int n_targets, n_layers;
    int P, Pcos;           /* padded FFT sides in use                             */
    int n_new;             /* n' of the new phase grid of the projection          */
    int max_batch;
} tomo_layout_info;

typedef struct {
    double tol;            /* target FP64 true relative residual ||s-A z||/||s||;
                              CG drives its recursive residual to 0.7 tol       */
    int max_iter;          /* CG iterations per call, over all refinement passes   */
    int max_refine;        /* FP64 true-residual restarts after the first pass    */
    int warm_start;        /* 1: zeta_dev holds the initial guess on entry;
                              2: the initial guess is the warm-start network's  */
    int check_every;       /* iterations between host convergence checks (>= 1)   */
    int precond;           /* 1: preconditioned CG with the block-circulant M;
                              2: flexible PCG with the learned preconditioner
                              z = pre_gain M r + out_scale N([r, M r]) (the
                              warm-start network initialised with
                              precond_input = 1, see tomo_ws_init), plain PCG
                              with M as its fallback (method CG only): a frame
                              falls back when r^T z <= 0 or when r^T r sets no
                              new minimum for 64 iterations                    */
    int method;            /* TOMO_METHOD_CG (0), _MINRES (1) or _BLOCK (2)        */
    int precision;         /* TOMO_PREC_FP32 (0), _FP64 (1) or _MIXED (2), below   */
    double inner_tol;      /* TOMO_PREC_MIXED: relative residual reduction asked
                              of each inner FP32 solve; 0 = automatic (the
                              remaining factor to tol, at least 2e-5)           */
    double deadline_ms;    /* > 0: wall-clock budget of the call, checked at
                              every convergence check; when it is spent the
                              frames still iterating stop (TOMO_FRAME_MAXIT),
                              the outputs are written as usual and the call
                              returns TOMO_ETIMEOUT                             */
    int host_loop;         /* 0 (default): the whole iteration loop of CG, PCG,
                              MINRES and FP64 CG is one CUDA graph launch with
                              conditional nodes: check_every iterations, a
                              device-side convergence and budget check, the FP64
                              true residual and its restarts, repeated while a
                              frame is active; the host waits only to read
                              info_host.  1: the host checks convergence every
                              check_every iterations.  Block CG always runs its
                              loop on the host.                                 */
} tomo_solve_opts;

/* Arithmetic of a solve (tomo_solve_opts.precision).
 * TOMO_PREC_FP32: FP32 vectors, FFTs and spectra, FP64 dot products and
 *   alpha/beta, FP64 true residual at exit with restarts from it (the
 *   default).  FP32 storage of zeta floors the relative residual near 1e-5.
 * TOMO_PREC_FP64: everything in FP64 (vectors, FFTs, spectra, scalars);
 *   tomo_solve_f64 only, method CG without preconditioner.
 * TOMO_PREC_MIXED: iterative refinement with an FP64 outer loop: zeta is
 *   accumulated in FP64, each pass computes the FP64 true residual
 *   r = s - A zeta with the FP64 operator and solves A d = r with the FP32
 *   machinery of TOMO_PREC_FP32 (any method and preconditioner) to
 *   inner_tol, then zeta += d in FP64; it reaches FP64-level residuals at
 *   FP32 speed per iteration.  tomo_frame_info.iters sums the inner
 *   iterations, refinements counts the outer passes after the first.
 *   With tomo_solve the FP64 zeta is rounded to FP32 on output (relres is
 *   that of the FP64 iterate); tomo_solve_f64 returns it in FP64. */
enum { TOMO_PREC_FP32 = 0, TOMO_PREC_FP64 = 1, TOMO_PREC_MIXED = 2 };

/* Krylov method of tomo_solve (tomo_solve_opts.method).  The paper tests CG
 * and MINRES, both unpreconditioned (Sec. 2.G).  MINRES runs in its
 * conjugate-residual form: for the symmetric positive (semi)definite systems
 * here each iterate minimises ||s - A zeta|| over the Krylov space, with one
 * operator product per iteration; it cannot be combined with precond = 1
 * (TOMO_EINVAL).  tomo_frame_info.iters counts operator products of the
 * iteration loop in both methods.
 * TOMO_METHOD_BLOCK: block conjugate gradients over the frames of each chunk
 * of at most 64 frames (O'Leary; with precond = 1 the block-circulant
 * preconditioner): every frame shares the operator, so one Krylov space,
 * grown by the whole chunk at each iteration, serves all of them.  Each
 * iteration applies the operator (and the preconditioner) to the chunk once,
 * as the other methods do, plus FP64-accumulated Gram products of the block
 * vectors and 64 x 64 FP64 algebra on the host; the search block is kept
 * orthonormal by Cholesky QR with numerically dependent columns dropped.
 * All frames of a chunk iterate until every one meets the tolerance; iters
 * counts block iterations.  Needs max_batch <= 64 and one operator for all
 * frames up to a factor per frame (see tomo_solve_r0). */
enum { TOMO_METHOD_CG = 0, TOMO_METHOD_MINRES = 1, TOMO_METHOD_BLOCK = 2 };

typedef struct {
    int iters;             /* CG iterations summed over refinement passes         */
    int refinements;       /* restarts from the FP64 true residual                */
    int status;            /* TOMO_FRAME_*                                        */
    int pad_;
    double relres;         /* FP64 true relative residual at exit                 */
} tomo_frame_info;

typedef struct tomo_handle tomo_handle;

/* Preconditioner (an addition to the paper, which runs its solvers without
 * one, Sec. 2.G): M^{-1} = W_s F^{-1} M(f) F W_s^T with, per frequency f of
 * the P x P torus, M(f) = (K_+(f) + c diag(sigma_g^2))^{-1}, K(f) the
 * (2 nGS) x (2 nGS) Hermitian block of the spectrum of Sigma_ss's covariance
 * evaluated at every lag of the torus (periodised), K_+ its eigenvalues
 * clamped at zero.  It is the block-circulant approximation of
 * (Sigma_ss + Sigma_eta_eta)^{-1} and costs one more FFT round trip per
 * iteration.  Used by tomo_solve when both cfg->precond and opts->precond are
 * set.
 *
 * Builds geometry, the Sigma_ss and Sigma_phi_s generator vectors (FP64, on
 * the device) and their spectra (Sec. 2.E: the FFT of the unique-element
 * vector is computed once, offline).  cuda_stream may be NULL (legacy default
 * stream).  Returns TOMO_EINVAL for an inconsistent configuration, e.g. a
 * layer at or above a laser guide star, guide stars at different finite
 * altitudes, fractions that are not positive, or an FFT side too small
 * (P >= 2n - 1, Pcos >= n' + n - 1) or with a prime factor above 7. */
tomo_status tomo_create(const tomo_config* cfg, void* cuda_stream, tomo_handle** out);

/* FFT-side autotuning (no counterpart in the paper, which takes any
 * P >= 2n - 1, Sec. 2.E).  With cfg.fft_P < 0, tomo_create times the FP32
 * Sigma_ss product (three passes, on min(max_batch, 64) frames) for every even
 * side P in [2n - 1, 1.25 (2n - 1)] whose prime factors are <= 7 (at most six
 * sides, smallest first) and keeps the fastest; the product is exact for any
 * such P, so the choice changes speed, not results.  This call returns the
 * sides tried and their mean times in ms (-1: the side could not run) into
 * sides[capacity] and ms[capacity] (either may be NULL); *count receives the
 * number of sides (0 when the handle was not autotuned). */
tomo_status tomo_autotune_result(const tomo_handle* h, int* sides, double* ms, int capacity, int* count);

/* Sizes and, if the pointers are non-NULL, host copies of the subaperture
 * mask (n*n bytes) and phase-point mask ((n+1)*(n+1) bytes). */
tomo_status tomo_layout(const tomo_handle* h, tomo_layout_info* info,
                        uint8_t* subap_mask, uint8_t* phase_mask);

/* y = W_s (Sigma_ss + Sigma_eta_eta) W_s^T x for `batch` frames, FP32 through
 * the 2RBT MVM (Eq. mvm_ss plus the noise term of Eq. SAap1: diagonal, or with
 * cfg.noise_cov the 2 x 2 per-subaperture blocks of Sec. 2.F, applied by a
 * separate pass over each guide star's slopes).
 * x_dev, y_dev: device [batch][N] floats, must not alias. */
tomo_status tomo_apply_css(tomo_handle* h, const float* x_dev, float* y_dev, int batch);

/* Allocation-free variant of tomo_apply_css (no counterpart in the paper).
 * For callers that must not allocate device memory once they are running: a
 * real-time reconstruction loop with a fixed frame deadline (cudaMalloc and
 * cudaFree synchronise the device and can take milliseconds), or a process
 * whose device memory is already handed out to another allocator.  The handle
 * is created beforehand (tomo_create allocates); this call itself allocates
 * nothing: the two intermediate half spectra of the product live in a 16 MiB
 * static device buffer of the library, which every GPU that loads the library
 * keeps until the process exits.  Frames are processed in chunks that fit the
 * buffer (at most 65535 frames per chunk); TOMO_ERANGE if a single frame does
 * not fit (2 * 2nGS * (P/2+1) * n complex floats must be <= 16 MiB; the
 * 74 x 74, 6-star system needs 1.08 MB, 15 frames per chunk).
 * Same arguments, result and stream as tomo_apply_css.  The first call on a
 * device looks up the buffer's device address, so make it before any stream
 * capture; the address is kept until the process exits, so do not call this
 * on a device after cudaDeviceReset (which also invalidates every handle).  All calls share the buffer and leave their intermediates in it
 * (nothing in it needs to start at zero: each call writes every element it
 * reads); calls that overlap on the GPU, on different streams or handles,
 * race on it. */
tomo_status tomo_apply_css_noalloc(tomo_handle* h, const float* x_dev, float* y_dev, int batch);

/* The same operator with FP64 vectors, FFTs and spectra (used for the true
 * residual of the solver). */
tomo_status tomo_apply_css_f64(tomo_handle* h, const double* x_dev, double* y_dev, int batch);

/* phi = W_phi Sigma_phi_beta_s W_s^T zeta for every target (Eq. SAap2), FP32.
 * Natural guide stars: the exact 2RBT form (Eq. mvm_ps).  Laser guide stars:
 * the per-layer new phase grid, bilinear interpolation and sum over layers
 * (Eq. interp, Eq. ToeplitzLGS).  zeta_dev [batch][N], phase_dev
 * [batch][n_targets][n_vphi] device floats. */
tomo_status tomo_apply_cos(tomo_handle* h, const float* zeta_dev, float* phase_dev, int batch);

/* The adjoint of tomo_apply_cos: zeta = sum_t W_s Sigma_s_phi_t W_phi^T phi_t,
 * the exact transpose of the same FP32 operator (for LGS the transposed
 * bilinear interpolation, then the conjugate-transposed per-frequency
 * blocks of Eq. ToeplitzLGS; for NGS the transposed Eq. mvm_ps).
 * phase_dev [batch][n_targets][n_vphi], zeta_dev [batch][N] device floats. */
tomo_status tomo_apply_cos_adjoint(tomo_handle* h, const float* phase_dev, float* zeta_dev, int batch);

/* The explicit reconstructor of one target (Eq. covBasedReconstructors1):
 *     R = W_phi Sigma_phi_s W_s^T (W_s (Sigma_ss + Sigma_eta_eta) W_s^T)^{-1},
 * the matrix a "direct MVM" reconstructor applies (the paper's comparison,
 * Sec. 4.B).  Row v of R solves the system with the right-hand side
 * W_s Sigma_s_phi W_phi^T e_v (tomo_apply_cos_adjoint of a unit phase), so
 * R is built by n_vphi solves, max_batch at a time, with the options in opts
 * (NULL: tomo_solve's defaults; warm_start must be 0).  R_dev: device
 * [n_vphi][N] floats, or NULL to keep only the error below; info_host: NULL
 * or [n_vphi] per-row solve outcomes.
 * wfe_host: NULL or [3] doubles, the analytic wave-front error of this
 * reconstructor for the target (Eq. analytical1, piston removed, mean over
 * the valid phase points, rad^2 at the r0 wavelength): [0] the rms error
 * sqrt([1] - [2]) [rad], [1] trace(P Sigma_phi_phi P) / n_vphi,
 * [2] trace(P R Sigma_s_phi P) / n_vphi, taking the reconstructor's own
 * covariance model as the truth (Hudgin slopes; for laser stars the
 * interpolated Sigma_phi_s of Eq. ToeplitzLGS) and R = F A^{-1} as solved.
 * R_dev and wfe_host cannot both be NULL.  TOMO_EINVAL with mode removal
 * (cfg.mode_removal).  Uses the handle's staging buffers of tomo_solve_host:
 * do not run both at the same time. */
tomo_status tomo_reconstructor(tomo_handle* h, int target, const tomo_solve_opts* opts, float* R_dev,
                               tomo_frame_info* info_host, double* wfe_host);

/* phase[b][v] = sum_j R[v][j] s[b][j]: the direct MVM with an explicit
 * reconstructor R_dev [rows][N] (e.g. from tomo_reconstructor), FP32,
 * hand-written tiled GEMM split over N with a fixed summation order.
 * slopes_dev [batch][N], phase_dev [batch][rows] device floats.  May
 * allocate a workspace on the first call with a larger batch x rows. */
tomo_status tomo_apply_reconstructor(tomo_handle* h, const float* R_dev, int rows, const float* slopes_dev,
                                     int batch, float* phase_dev);

/* Full reconstruction of `batch` frames: CG (FP32 vectors and MVMs, FP64
 * dot products and alpha/beta) on Eq. SAap1, FP64 true residual at exit and
 * restarts from it while it exceeds opts->tol, then the projection of
 * Eq. SAap2.  slopes_dev [batch][N]; zeta_dev [batch][N] (warm start in if
 * opts->warm_start); phase_dev [batch][n_targets][n_vphi] or NULL to skip the
 * projection; info_host [batch] host memory or NULL.  opts NULL = defaults
 * (tol 1e-4, max_iter 10000, max_refine 2, cold start, check_every 32, no
 * preconditioner, TOMO_PREC_FP32, no deadline).  opts->precision FP32 or
 * MIXED (FP64 is tomo_solve_f64's).
 * Synchronises the stream at each convergence check.  TOMO_ETIMEOUT when
 * opts->deadline_ms ran out (outputs and info are still written). */
tomo_status tomo_solve(tomo_handle* h, const float* slopes_dev, int batch,
                       const tomo_solve_opts* opts, float* zeta_dev, float* phase_dev,
                       tomo_frame_info* info_host);

/* tomo_solve with a Fried parameter per frame (Sec. 2.A: the von Karman
 * covariance of every layer is proportional to r0^{-5/3}, with the Cn^2
 * fractions fixed).  Frame f solves
 *     (c_f W_s Sigma_ss W_s^T + nu_f Sigma_eta_eta) zeta_f = s_f,
 *     phi_f = c_f W_phi Sigma_phi_s W_s^T zeta_f,
 * with c_f = (r0_host[f] / cfg.r0)^{-5/3} and nu_f = noise_scale_host[f]
 * (all 1 when noise_scale_host is NULL: the noise variance of the
 * configuration), so one batch can mix frames taken under different seeing.
 * r0_host [batch] metres at 500 nm, > 0; noise_scale_host [batch] >= 0 or
 * NULL; both host memory, read before the call returns.  The preconditioner,
 * if used, is the configuration's one scaled by 1 / c_f (exact when
 * nu_f = c_f).  Other arguments and results as tomo_solve; TOMO_EINVAL for a
 * non-positive or non-finite r0 or a negative noise scale.
 * With TOMO_METHOD_BLOCK the operators of all frames must be multiples of one
 * another, i.e. kappa = nu_f / c_f the same for every frame (as when the noise
 * variance follows the seeing); the library then solves the common system
 * (Sigma_ss + kappa Sigma_eta_eta) zeta~_f = s_f by block CG and returns
 * zeta_f = zeta~_f / c_f (and phi_f = c_f Cos zeta_f = Cos zeta~_f).  Other
 * mixes are TOMO_EINVAL. */
tomo_status tomo_solve_r0(tomo_handle* h, const float* slopes_dev, int batch,
                          const double* r0_host, const double* noise_scale_host,
                          const tomo_solve_opts* opts, float* zeta_dev, float* phase_dev,
                          tomo_frame_info* info_host);

/* With cfg.mode_removal = 1 (split tomography, Sec. 2.F "Mode removal"),
 * tomo_solve, tomo_solve_r0 and tomo_solve_host solve instead
 *     M_s W_s (Sigma_ss + Sigma_eta_eta) W_s^T M_s zeta = M_s s,
 *     phi = M_phi W_phi Sigma_phi_s W_s^T M_s zeta,
 * with M_s = I - Z_s Z_s^+ per WFS (Z_s: the 2 n_vs x 3 slopes of tip x,
 * tilt y and focus x^2 + y^2 on the valid subapertures) and M_phi the same on
 * the valid phase points (Z_phi: x, y, x^2 + y^2).  The returned zeta is
 * M_s zeta (the minimum-norm solution when the solve converges), relres is
 * ||M_s s - M_s A M_s zeta|| / ||M_s s||, and tomo_apply_css / tomo_apply_cos
 * keep applying the operators without the projections.  The paper applies
 * it to laser guide stars; here it applies to every WFS of the handle. */

/* The solve on FP64 slopes and solution (config of the 8 m system of Sec. 3,
 * stated in FP64): slopes_dev, zeta_dev [batch][N] device doubles (zeta_dev
 * holds the initial guess if opts->warm_start = 1; warm_start 2 is EINVAL).
 * opts->precision TOMO_PREC_FP64 runs textbook CG (Sec. 2.G) entirely in
 * FP64: the FP64 2RBT product of tomo_apply_css_f64, FP64 vectors, dot
 * products and alpha/beta (method CG and precond 0 only, EINVAL otherwise);
 * TOMO_PREC_MIXED the FP64-outer refinement described above (any method);
 * TOMO_PREC_FP32 is EINVAL here.  No projection (apply tomo_apply_cos to the
 * rounded zeta).  Synchronises like tomo_solve. */
tomo_status tomo_solve_f64(tomo_handle* h, const double* slopes_dev, int batch, const tomo_solve_opts* opts,
                           double* zeta_dev, tomo_frame_info* info_host);

/* tomo_solve on host buffers: copies slopes in and zeta / phase out around the
 * solve (phase_host may be NULL).  Returns after the stream has finished. */
tomo_status tomo_solve_host(tomo_handle* h, const float* slopes_host, int batch,
                            const tomo_solve_opts* opts, float* zeta_host, float* phase_host,
                            tomo_frame_info* info_host);

/* Number of kernel launches the handle has issued since creation (a counter
 * kept by the library, for launch accounting). */
long long tomo_launch_count(const tomo_handle* h);

/* Learned warm start (an addition to the paper, which starts its solvers from
 * zero or from the previous estimate, Sec. 5).  A convolutional network maps
 * the slope grids of one frame to an initial zeta for tomo_solve
 * (opts->warm_start = 2):
 *   input  [2 nGS][n][n]  slopes * in_scale on the subaperture grid, 0 off W_s;
 *   layers 3x3 convolutions 2nGS -> hidden -> hidden -> hidden -> 2nGS, zero
 *          padding, ReLU after the first three, FP32;
 *   output zeta_0 = out_scale * (last layer at the valid subapertures).
 * With precond_input (needs the preconditioner, cfg->precond) the input has
 * 4 nGS planes, [slopes * in_scale, M^{-1} slopes / out_scale], and the output
 * is zeta_0 = pre_gain M^{-1} slopes + out_scale * (last layer): the network learns a
 * local correction of the block-circulant estimate (whose errors sit at the
 * pupil edges and obstruction, where the circulant model misses the mask).
 * Parameters are one FP32 vector: per layer W [Cout][Cin][3][3] then b [Cout].
 * Training (tomo_ws_train_step, Adam) minimises ||zeta_0 - zeta*||^2 / ||zeta*||^2
 * over (slopes, zeta*) pairs, zeta* from tomo_solve.  Device buffers are
 * [batch][N] as elsewhere; batch <= max_batch for the gradient calls.
 * tomo_ws_init: once per handle (EINVAL on a second call, hidden > 32 or
 * 2 nGS > 32).  Parameters start at zero: set them with tomo_ws_set_params,
 * which also resets the optimiser state.  tomo_ws_gradient returns the
 * parameter gradient and the loss without updating (for checks). */
tomo_status tomo_ws_init(tomo_handle* h, int hidden, int max_batch, float in_scale, float out_scale,
                         int precond_input, float pre_gain);
tomo_status tomo_ws_param_count(const tomo_handle* h, int* count);
tomo_status tomo_ws_set_params(tomo_handle* h, const float* params_host, int count);
tomo_status tomo_ws_get_params(const tomo_handle* h, float* params_host, int count);
tomo_status tomo_ws_apply(tomo_handle* h, const float* slopes_dev, float* zeta_dev, int batch);
tomo_status tomo_ws_gradient(tomo_handle* h, const float* slopes_dev, const float* zeta_target_dev, int batch,
                             float* grad_host, double* loss_host);
tomo_status tomo_ws_train_step(tomo_handle* h, const float* slopes_dev, const float* zeta_target_dev, int batch,
                               float lr, double* loss_host);

/* y = M^{-1} x: the block-circulant preconditioner (see tomo_create) applied to
 * `batch` frames, FP32.  EINVAL if the handle was created without it. */
tomo_status tomo_apply_precond(tomo_handle* h, const float* x_dev, float* y_dev, int batch);

/* Kernel timing.  With timing enabled, tomo_solve launches its CG iterations
 * eagerly (no CUDA graph) with a CUDA event on the handle's stream before and
 * after each MVM pass, and accumulates the elapsed times per pass:
 *   [0] row-forward FFT pass, [1] column FFT + block-multiply pass,
 *   [2] row-inverse FFT + mask pass, [3] per-frame CG scalars.
 * Enabling or disabling resets the accumulators and the frame-iteration count
 * (sum over frames of the CG iterations of the solves since the reset). */
#define TOMO_NKERNELS 4
tomo_status tomo_set_kernel_timing(tomo_handle* h, int enable);
tomo_status tomo_get_kernel_timing(const tomo_handle* h, double* ms_total /*[TOMO_NKERNELS]*/,
                                   long long* launches /*[TOMO_NKERNELS]*/, long long* frame_iters);

void tomo_destroy(tomo_handle* h);

const char* tomo_strerror(tomo_status s);

#ifdef __cplusplus
}
#endif

#endif /* TOMO_H */
