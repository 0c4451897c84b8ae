// Internal interface between the host side of the library (capi.cu) and the
// device kernels (kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fft.cuh"

namespace tomo {

constexpr int kWarps = 8;              // warps per block in the FFT kernels
constexpr int kThreads = 32 * kWarps;
#ifndef TOMO_MIN_BLOCKS
#define TOMO_MIN_BLOCKS 3                  // resident blocks per SM the FFT kernels are compiled for
#endif

// Row passes: one block transforms the row pairs of one plane of one frame
// (one pair per sequence), or, for batches too small to fill the GPU, up to
// kRowPairsPerBlock of them (kFftGroup sequences per warp), so that a plane of
// n rows is split over row_groups(n) blocks.  Partial sums of the row passes
// are stored per (frame, plane, row group).
constexpr int kRowPairsPerBlock = 16;
__host__ __device__ constexpr int row_groups(int nrows) {
    return ((nrows + 1) / 2 + kRowPairsPerBlock - 1) / kRowPairsPerBlock;
}

// Geometry of one FFT-based 2RBT product y = T x (Sec. 2.E): inputs are NPin
// masked planes on an n x n grid, outputs NPout planes on an m x m grid, both
// embedded in a P x P periodic grid (P >= m + n - 1); half spectrum nh = P/2+1.
struct MvmGeom {
    int n, m, NPin, NPout, nh;
    FftPlan plan;
};

// Per-frame CG scalars (FP64), one per frame.
struct FrameState {
    double rr;       // r^T r of the current residual
    double alpha;    // alpha applied by the next row-forward pass (x += alpha p, r -= alpha Ap)
    double beta;     // beta applied by the next row-forward pass (p = r + beta p)
    double snorm2;   // ||s||^2
    double tol2;     // (tol ||s||)^2
    double relres;   // FP64 true relative residual (after a true-residual pass)
    int iters;       // iterations done (all passes)
    int active;      // 1 while CG runs on this frame
    int status;      // TOMO_FRAME_*
    int refinements; // restarts from the true residual
    double gamma;    // PCG: r^T M^{-1} r of the previous iteration; MINRES: r^T A r
    int fresh;       // PCG, MINRES, flexible PCG: 1 on the first iteration after a (re)start
    int pad_;
    double delta;    // MINRES: (Ap)^T (Ap) of the current direction
    // flexible (learned) PCG
    int fb;          // 1 once the frame has fallen back to PCG with M alone
    int ckpt_iter;   // iteration of the last progress checkpoint
    double rr_ckpt;  // r^T r at that checkpoint
};

// Masked-vector index tables: valid entries of row r are [rowstart[r], rowstart[r+1]),
// with column col[e]; the same tables serve input and output of Sigma_ss.
struct MaskTables {
    const int* rowstart;   // [n+1]
    const int* col;        // [n_vs]
    const int* rowcol;     // [n_vs]: row << 16 | col of each valid entry
    int n_vs;
};

struct Launch {
    cudaStream_t stream;
    long long* counter;    // incremented once per kernel launch
};

// Raises the dynamic shared-memory limit of every kernel to the device's
// opt-in maximum (once per process and device, before any launch or capture).
cudaError_t init_kernel_attributes();

// CG vectors of a batch, [B][N] each (FP32).
//   mode 1 (CG):  row-forward applies x += alpha p, r -= alpha Ap, p = r + beta p and transforms p;
//   mode 2 (PCG, Chronopoulos-Gear form): row-forward applies p = z + beta p,
//                 s = w + beta s, x += alpha p, r -= alpha s and transforms r;
//                 z = M^{-1} r and w = A z come from the two products of the iteration.
//   mode 3 (MINRES in conjugate-residual form): row-forward applies
//                 p = r + beta p, Ap = w + beta Ap, x += alpha p, r -= alpha Ap
//                 and transforms r; the product gives w = A r and the partial
//                 sums r^T w, Ap^T w, w^T w.
struct CgVecs {
    float* x;         // iterate (zeta)
    float* r;         // residual
    float* p;         // search direction
    float* Ap;        // CG: A p of the previous iteration; PCG: s, the recurrence for A p
    double* rr_part;  // [B][NP][row groups] partial sums of r^T r after the update
    double* dot_part; // [B][NP][row groups][3] partial sums xin^T y, r^T y, y^T y of the row-inverse pass
    int mode;
    float* z;         // PCG: M^{-1} r
    float* w;         // PCG: A z; MINRES: A r
};

// --- MVM passes ---------------------------------------------------------
// Row-forward pass: x [B][NPin][n_vs] (masked) -> X1T [B][NPin][nh][n].
// CG mode (cg != nullptr; x ignored): first applies the previous iteration's
// update x += alpha p, r -= alpha Ap, forms p = r + beta p, accumulates r^T r
// of the updated residual, and transforms p.
// rg: 1 (one block per plane) or row_groups(g.n) (one block per row group);
// the partial sums are stored per (frame, plane, row group) accordingly.
template <typename T, typename TIn>
cudaError_t rows_fwd(const Launch& L, const MvmGeom& g, const MaskTables& mt, int B,
                     const TIn* x, const CgVecs* cg, const FrameState* st,
                     cplx_t<T>* X1T, const cplx_t<T>* tw, int rg = 1);

// Column pass: forward column FFT of the NPin planes, per-frequency block
// multiply by K [nh][NPin][P][NPout] (herm = false) or by the Hermitian
// upper triangle [nh][P][e(p <= q)] (herm = true, NPin = NPout), inverse
// column FFT, keep rows < m: X1T [B][NPin][nh][n] -> Y1T [B][NPout][nh][m].
template <typename T>
cudaError_t cols_mul(const Launch& L, const MvmGeom& g, int B, const FrameState* st,
                     const cplx_t<T>* X1T, cplx_t<T>* Y1T, const cplx_t<T>* K, const cplx_t<T>* tw, bool herm);
// Full [nh][NP][P][NP] spectrum -> Hermitian upper-triangle layout [nh][P][e].
// Elements of the Hermitian-packed spectra of an NP x NP block operator on a
// P x P torus: (P/2 + 1) kx x P padded to a multiple of 8 (ky) x NP (NP + 1) / 2
// padded to an even count.
__host__ __device__ inline size_t herm_packed_elems(int P, int NP) {
    return (size_t)(P / 2 + 1) * ((P + 7) / 8 * 8) * ((NP * (NP + 1) / 2 + 1) / 2 * 2);
}
cudaError_t pack_hermitian(const Launch& L, int P, int NP, const float2* Kfull, float2* Kpacked);

// Row-inverse pass to masked output (Sigma_ss): y = c_f crop/mask(IFFT rows) +
// nu_f noise_var[plane] * xin, with (c_f, nu_f) = fscale[frame] ((1, 1) when
// fscale is null); xin may be null (no diagonal term) outside CG mode.  CG mode (cg != nullptr; xin = cg->p, y = cg->Ap): also the
// partial sums p^T Ap, r^T Ap, Ap^T Ap per (frame, plane).
template <typename T, typename TIn>
cudaError_t rows_inv_masked(const Launch& L, const MvmGeom& g, const MaskTables& mt, int B,
                            const FrameState* st, const cplx_t<T>* Y1T, const TIn* xin,
                            const double* noise_var, const double2* fscale, TIn* y, const CgVecs* cg,
                            const cplx_t<T>* tw, int rg = 1);

// Persistent, prefetching forms of the FP32 row passes (rows_pp.cu), used by
// rows_fwd / rows_inv_masked when they apply (fused FFT size, whole planes per
// block, 16-byte aligned slices, n_vs a multiple of 4; row-forward in plain or
// CG mode); *used reports whether they ran.
cudaError_t rows_inv_pp(const Launch& L, const MvmGeom& g, const MaskTables& mt, int B, const FrameState* st,
                        const float2* Y1T, const float* xin, const double* noise_var, const double2* fscale,
                        float* y, const CgVecs* cg, const float2* tw, int max_smem, bool* used);
cudaError_t rows_fwd_pp(const Launch& L, const MvmGeom& g, const MaskTables& mt, int B, const float* x,
                        const CgVecs* cg, const FrameState* st, float2* X1T, const float2* tw, int max_smem,
                        bool* used);
cudaError_t init_rows_pp_attributes(int dyn);
// Reads and clears the device's flag of bounded waits that expired (0: none).
cudaError_t take_wait_error(int* flag);

// Row-inverse pass to a dense m x m output per plane: Yd [B][NPout][m][m].
template <typename T>
cudaError_t rows_inv_dense(const Launch& L, const MvmGeom& g, int B, const cplx_t<T>* Y1T,
                           T* Yd, const cplx_t<T>* tw);

// --- CG ---------------------------------------------------------------------
cudaError_t cg_init(const Launch& L, int B, int N, int nparts, const float* s, const float* Ax0,
                    float* x, float* r, float* p, float* Ap, double* parts);
cudaError_t cg_init_scalars(const Launch& L, int B, int nparts, const double* parts, double tol,
                            int warm, FrameState* st);
// The scalar kernels take NP = the number of partial-sum entries per frame
// (planes x row groups).
// Per-frame scalars after an iteration: convergence test on the updated
// residual, alpha, and beta of the next iteration from
// r_new^T r_new = r^T r - 2 alpha r^T Ap + alpha^2 Ap^T Ap (Chronopoulos & Gear).
cudaError_t cg_scalars(const Launch& L, int B, int NP, const double* rr_part, const double* dot_part,
                       FrameState* st);
// PCG scalars (Chronopoulos & Gear): gamma = r^T z, delta = z^T A z,
// beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old);
// dot_M from the preconditioner pass (xin = r, y = z), dot_A from the
// operator pass (xin = z, y = w).
cudaError_t pcg_scalars(const Launch& L, int B, int NP, const double* rr_part, const double* dot_M,
                        const double* dot_A, FrameState* st);
// MINRES scalars (conjugate-residual recurrences): rho = r^T A r,
// beta = rho / rho_old, (Ap)^T(Ap) = w^T w + 2 beta Ap_old^T w + beta^2 (Ap_old)^T(Ap_old),
// alpha = rho / (Ap)^T(Ap); the convergence test uses r^T r of the row-forward pass.
cudaError_t mr_scalars(const Launch& L, int B, int NP, const double* rr_part, const double* dot_part,
                       FrameState* st);
// State of a solve's device-side loop (a CUDA graph with conditional nodes:
// WHILE {check_every iterations; loop_check; IF {true residual}; loop_next}).
struct LoopState {
    long long iters;            // iterations run in this solve (in chunks of `chunk`)
    long long max_iter;
    unsigned long long t0;      // GPU global timer at the start of the loop [ns]
    unsigned long long budget;  // time budget [ns] (0: none)
    double tol;
    int max_refine;
    int chunk;
    int stop;                   // the iteration or time budget is spent: the next true residual is final
    int timed_out;              // the time budget ran out
    int true_res_runs;          // true residuals computed (IF node bodies run)
};
// Initialises the loop state of a solve (before the graph launch).
cudaError_t loop_start(const Launch& L, LoopState* ls, long long max_iter, unsigned long long budget_ns, double tol,
                       int max_refine, int chunk);
// Adds a chunk to the iteration count, stops the active frames (TOMO_FRAME_MAXIT)
// once a budget is spent, and sets `need_true_res` to 1 when no frame is
// active or the budget is spent.
cudaError_t loop_check(const Launch& L, int B, FrameState* st, LoopState* ls, cudaGraphConditionalHandle need_true_res);
// Sets `more` to 1 while a frame is active (after the true residual's restarts).
cudaError_t loop_next(const Launch& L, int B, const FrameState* st, const LoopState* ls,
                      cudaGraphConditionalHandle more);
cudaError_t to_f64(const Launch& L, size_t n, const float* a, double* b);
cudaError_t true_residual(const Launch& L, int B, int N, int nparts, const float* s,
                          const double* Ax, float* r, double* parts);
// With ls (device loop), tol and max_refine are read from it (max_refine 0 once ls->stop is set).
cudaError_t true_residual_finalize(const Launch& L, int B, int nparts, const double* parts,
                                   double tol, int max_refine, FrameState* st, const LoopState* ls = nullptr);
cudaError_t count_active(const Launch& L, int B, const FrameState* st, int* n_active);
// v [B][N]: frames with status TOMO_FRAME_BREAKDOWN set to zero.
cudaError_t zero_broken(const Launch& L, int B, int N, const FrameState* st, float* v);

// --- flexible (learned) PCG (flex.cu) ----------------------------------------------
// Vectors [B][N] FP32; partial sums [B][nparts][5] / [B][nparts].
// flex_dots: r^T r, r^T zN, q^T zN, r^T zM, q^T zM (q = A p of the previous direction).
cudaError_t flex_dots(const Launch& L, int B, int N, int nparts, const FrameState* st, const float* r, const float* q,
                      const float* zN, const float* zM, double* parts);
// Convergence test, fallback decisions, beta (Polak-Ribiere in the form -alpha q^T z / r_old^T z_old).
cudaError_t flex_beta(const Launch& L, int B, int nparts, const double* parts, int window, FrameState* st);
// p = z + beta p with z = zM (fallen back) or zN (flexible), active frames.
cudaError_t flex_dir(const Launch& L, int B, int N, const FrameState* st, const float* zN, const float* zM, float* p);
cudaError_t flex_pq(const Launch& L, int B, int N, int nparts, const FrameState* st, const float* p, const float* q,
                    double* parts);
// alpha = r^T z / p^T q (breakdown when p^T q <= 0 or not finite); iters += 1.
cudaError_t flex_alpha(const Launch& L, int B, int nparts, const double* parts, FrameState* st);
// x += alpha p, r -= alpha q, active frames.
cudaError_t flex_update(const Launch& L, int B, int N, const FrameState* st, float* x, float* r, const float* p,
                        const float* q);

// --- FP64 solves and mixed-precision refinement (solve64.cu) --------------------
// FP64 CG vectors [B][N]; partial sums [B][nparts] (r^T r, s^T s: [B][2][nparts]
// for the init), dot_part [B][nparts][3] as the fused passes lay them out.
cudaError_t cg64_init(const Launch& L, int B, int N, int nparts, const double* s, const double* Ax0, double* x,
                      double* r, double* p, double* Ap, double* parts);
cudaError_t cg64_update(const Launch& L, int B, int N, int nparts, const FrameState* st, double* x, double* r,
                        double* p, const double* Ap, double* rr_part);
cudaError_t cg64_dots(const Launch& L, int B, int N, int nparts, const FrameState* st, const double* p,
                      const double* r, const double* Ap, double* dot_part);
// r = s - Ax (r may be null), parts [B][nparts] of r^T r
cudaError_t residual64(const Launch& L, int B, int N, int nparts, const double* s, const double* Ax, double* r,
                       double* parts);
// rhs [f] = (float) r[f] where rel[f] > tol, else 0
cudaError_t inner_rhs(const Launch& L, int B, int N, const double* rel, double tol, const double* r, float* rhs);
cudaError_t add_f32_to_f64(const Launch& L, size_t n, const float* d, double* x);
// out [f] = (float)(scale[f] x[f]) (scale may be null)
cudaError_t f64_to_f32(const Launch& L, int B, int N, const double* scale, const double* x, float* out);
cudaError_t relres64(const Launch& L, int B, int nparts, const double* parts, const double* snorm2, double* rel);
// out[f] = s[f]^T s[f] (parts: [B][nparts] scratch)
cudaError_t norm2_64(const Launch& L, int B, int N, int nparts, const double* s, double* parts, double* out);

// --- mode removal (modes.cu) -------------------------------------------------
// y [B][nblk][len] <- y - Q^T (Q y) per (frame, block), Q [3][len] orthonormal
// rows (FP64).  Slopes: nblk = n_gs blocks of len = 2 n_vs; phase: nblk =
// n_targets blocks of len = n_vphi.  With cg != nullptr (slopes, FP32): also
// the partial sums xin^T y, r^T y (Ap^T y in mode 3), y^T y of the projected y
// per plane into cg->dot_part, replacing those of the row-inverse pass that
// produced y.
// Frames with st[f].active == 0 are skipped when st is not null.
// rg: row groups per plane of the partial-sum layout.
template <typename TV>
cudaError_t mode_project(const Launch& L, int B, int len, int nblk, int rg, const double* Q, const FrameState* st,
                         TV* y, const float* xin, const CgVecs* cg);

// Elongated-spot noise (modes.cu): y += nu_f Sigma_eta_eta x with one 2 x 2
// block per subaperture (cov [n_gs][n_vs][3] = s_xx, s_yy, s_xy; nu_f =
// fscale[f].y or 1), x and y [B][n_gs][2][n_vs]; with cg the partial sums of
// the updated y replace those of the row-inverse pass (as mode_project).
template <typename TV>
cudaError_t noise_blocks(const Launch& L, int B, int n_vs, int n_gs, int rg, const double* cov, const double2* fscale,
                         const FrameState* st, TV* y, const TV* x, const float* xin, const CgVecs* cg);

// --- adjoint projection and explicit reconstructor (recon.cu) -----------------
// out [B][n_layers][m][m] = I'^T of phi[:, t, :] through the transposed
// bilinear table (ptr [n_layers][m*m + 1], vi / w entries: phase point, weight).
cudaError_t interp_adjoint(const Launch& L, int B, int T_all, int t, int n_layers, int m, int n_vphi,
                           const int* ptr, const int* vi, const float* w, const float* phi, float* out);
// Kadj [nh][np][P][nq] = conj(K [nh][nq][P][np]).
cudaError_t adjoint_spectra(const Launch& L, int nh, int P, int nq, int np, const float2* K, float2* Kadj);
// phi [B][T][n_vphi]: unit vector at (t, v0 + f) for frame f.
cudaError_t unit_phase(const Launch& L, int B, int T_all, int t, int n_vphi, int v0, float* phi);
// C [M][N] (row stride ldc) = A [M][K] (lda) * B [N][K]^T (ldb), FP32, split
// over K into `splits` partial tiles (part: gemm_nt_workspace floats) added
// in a fixed order.
// dots[b] = F[b] . X[b]; sumF += sum_b F[b], sumX += sum_b X[b] (FP64, fixed
// order): the terms of the analytic error of an explicit reconstructor.
cudaError_t wfe_accumulate(const Launch& L, int B, int N, const float* F, const float* X, double* dots, double* sumF,
                           double* sumX);
size_t gemm_nt_workspace(int M, int N, int splits);
// Block recurrences over the frames of a batch (B <= 64 vectors [B][N]):
// G [B][B] = U V^T (FP32 products, FP64 sums in a fixed order; part:
// gram_workspace(N) doubles); Y = Y0 + C^T U, i.e. Y_j = Y0_j + sum_i C[i][j] U_i
// (C [B][B] FP64, Y0 may be null, Y must not alias U); out [B][slices]: the
// squared norm of each of `slices` column ranges of X_j (sum them for |X_j|^2).
size_t gram_workspace(int N);
cudaError_t gram(const Launch& L, int B, int N, const float* U, const float* V, double* G, double* part);
cudaError_t block_combine(const Launch& L, int B, int N, const double* C, const float* U, const float* Y0, float* Y,
                          double scale = 1.0);
// Y = scale op(A) X for B x B FP64 matrices, op(A) = A or A^T (Y must not alias A or X).
// Y = scale T (T^T X), B x B row-major FP64 (T^T X is never stored)
cudaError_t gram_apply(const Launch& L, int B, const double* T, const double* X, double* Y, double scale);
cudaError_t row_norms(const Launch& L, int B, int N, const float* X, double* out, int slices);
// Y_j = f[j] X_j (device FP64 factors; Y may alias X).
cudaError_t scale_rows(const Launch& L, int B, int N, const double* f, const float* X, float* Y);
cudaError_t gemm_nt(const Launch& L, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                    int ldc, int splits, float* part);

// --- setup ------------------------------------------------------------------
struct VkParams {
    double L0;
    double norm;     // 2^{1/6} / Gamma(5/6)
    const double* cosh_t;    // quadrature table cosh(m h), m in [0, nq)
    const double* cosh_nu_t; // cosh(5/6 m h)
    int nq;
    double h;
};

struct LayerGeom {
    double h;        // altitude
    double amp;      // c_v (L0/r0)^{5/3} f_k : B_k(0)
    double gamma;    // cone factor shared by the guide stars
};

// Sigma_ss generators on the wrapped P x P grid: G[p*NP+q][P][P] (pre-zeroed).
// periodised = false: the exact 2RBT generator, lags [-(n-1), n-1];
// periodised = true: the covariance at every lag of the P-torus, [-P/2, P/2).
// model: slope model of the points (0 Hudgin-like, 1 Fried).
cudaError_t gen_css(const Launch& L, int n, int P, int NP, double d, int n_layers,
                    const LayerGeom* layers, const double* gs_alpha, VkParams vk, double* G, bool periodised,
                    int model);
// Block-circulant preconditioner spectra M(f) = (K_+(f) + c diag(sigma^2))^{-1} / P^2
// from the FP64 spectra of the periodised generator (both [nh][NP][P][NP]).
cudaError_t precond_spectra(const Launch& L, int P, int NP, const double2* K64, const double* noise_var,
                            double floor_c, float2* M32);
// Sigma_phi_s generators of one target: G[k*NP+q][P][P] for the m x n 2RBT blocks.
cudaError_t gen_cos(const Launch& L, int n, int m, int P, int NP, double d, int n_layers,
                    const LayerGeom* layers, const double* gs_alpha, double bx, double by,
                    VkParams vk, double* G, int model);
// Spectra: 2-D real FFT of each G plane, scaled by 1/P^2, into
// K [nh][NPin][P][NPout] (plane index p*NPin + q), FP64 and FP32 copies.
cudaError_t spectra(const Launch& L, int P, int npl, int NPin, const FftPlan& plan,
                    const double* G, double2* H, const double2* tw64, double2* K64, float2* K32);
// Bilinear interpolation of the projection: phi [B][T][n_vphi] (target t slot),
// times fscale[frame].x when fscale is not null.
cudaError_t interp(const Launch& L, int B, int T_all, int t, int n_layers, int m, int n_vphi,
                   const float* Yd, const int* idx, const float* w, const double2* fscale, float* phi);

}  // namespace tomo
