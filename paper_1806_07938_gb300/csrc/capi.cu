// Host side of the C ABI declared in include/tomo.h.
//
// Index mapping of the 2RBT MVM (Sec. 2.E).  The paper writes y = T x for an
// m^2 x n^2 two-level Toeplitz T as a 1-D FFT of length (m+n-1)^2 with the
// shuffles S_1 (x reversed into the padded vector) and S_2 (read back).  Here
// the same product is evaluated as the 2-D linear convolution
//     y(a) = sum_b t(a - b) x(b),   a in [0,m)^2, b in [0,n)^2,
// on a P x P periodic grid, P >= m + n - 1: x placed unreversed at its grid
// position, the generator t stored at the wrapped lag (a - b) mod P, and y read
// at a.  Both orderings give the same exact product (any P >= m + n - 1 avoids
// wrap-around); the 2-D form lets the x-FFTs act on the n non-zero rows only
// and lets the inverse keep only the m needed rows.
//
// Noise: Sigma_eta_eta = sigma_g^2 I per guide star (Sec. 2.B), applied as a
// diagonal term after the masked gather (Eq. SAap1).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/tomo.h"
#include "cnn.cuh"
#include "kernels.cuh"

using namespace tomo;

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int B = -1, iters = 0, mode = 0;
    long long nodes = 0;
};

// The device-side solve loop: one graph per (batch, chunk, kind) with a WHILE
// node around {chunk iterations; loop_check; IF {FP64 true residual}; loop_next}.
struct LoopGraph {
    cudaGraphExec_t exec = nullptr;
    int B = -1, chunk = 0, kind = -1;
    long long body_nodes = 0, if_nodes = 0;   // kernel launches per body pass / per true residual
};

// Warm-start network state (see tomo_ws_* in include/tomo.h).
struct WarmStartNet {
    bool ready = false;
    int layers = 4, maxB = 0, np = 0, step = 0;
    int ch[5] = {0, 0, 0, 0, 0};
    size_t offW[4] = {0, 0, 0, 0}, offb[4] = {0, 0, 0, 0};
    float in_scale = 1.f, out_scale = 1.f;
    bool dirty = true;                 // weight layouts need rebuilding
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    float *Wt[4] = {nullptr, nullptr, nullptr, nullptr}, *Wb[4] = {nullptr, nullptr, nullptr, nullptr};
    float* zero_bias = nullptr;
    float* act[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    float *d0 = nullptr, *d1 = nullptr, *gz = nullptr, *z = nullptr;
    float* wpart = nullptr;
    double *sums = nullptr, *loss = nullptr;
    bool hybrid = false;               // input channels [s, M^{-1} s], output M^{-1} s + correction
    float pre_scale = 1.f;             // scale of the M^{-1} s input channels
    float pre_gain = 1.f;              // zeta_0 = pre_gain M^{-1} s + out_scale * network
    float* zpre = nullptr;             // M^{-1} s of the current batch
};

struct tomo_handle {
    // configuration
    int n = 0, n_gs = 0, NP = 0, n_vs = 0, N = 0, n_vphi = 0, n_layers = 0, n_targets = 0;
    int P = 0, Pc = 0, m = 0, cos_layers = 0, max_batch = 0;
    int rg = 1;                        // row groups per plane of the row passes (partial-sum layout)
    int slope_model = TOMO_SLOPE_HUDGIN;
    double* d_ncov = nullptr;          // elongated-spot noise blocks [n_gs][n_vs][3] (nullptr: diagonal noise)
    double* d_rows_noise = nullptr;    // the diagonal the row-inverse pass adds (zero with d_ncov)
    int block_slots = 456;             // SMs x resident blocks of the row passes
    double D = 0, obstruction = 0, d = 0, r0 = 0, L0 = 0;
    bool all_ngs = true;
    std::vector<double> tx, ty;
    cudaStream_t stream = nullptr;     // the caller's stream
    cudaStream_t work = nullptr;       // private stream of the solver (graph capture needs a non-legacy stream)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    long long launches = 0;
    std::vector<uint8_t> subap_mask, phase_mask;
    std::vector<int> ph_i, ph_j;       // valid phase points (row, column), row-major
    double frac_sum = 1.0;             // sum of the Cn^2 fractions
    FftPlan plan{}, planc{};
    MvmGeom g_ss{}, g_os{};
    MaskTables mt{};
    // device tables
    int* d_rowstart = nullptr;
    int* d_col = nullptr;
    int* d_rowcol = nullptr;
    double* d_noise_var = nullptr;     // sigma_g^2 per plane: the diagonal noise, the preconditioner's floor
    float2* d_tw32 = nullptr;
    double2* d_tw64 = nullptr;
    float2* d_twc32 = nullptr;
    float2* d_K32 = nullptr;
    double2* d_K64 = nullptr;
    float2* d_Kc32 = nullptr;
    float2* d_M32 = nullptr;           // block-circulant preconditioner spectra (nullptr: not built)
    double* d_zero_var = nullptr;      // zero diagonal for the preconditioner pass
    // per-frame scales of the solve (tomo_solve_r0): (c_f, nu_f) of
    // A_f = c_f Sigma_ss + nu_f Sigma_eta_eta, and (1 / c_f, 0) for the preconditioner
    double2* d_fscale = nullptr;
    double2* d_fscale_pre = nullptr;
    bool fscale_unit = false;          // both hold the unit scales
    // tip/tilt/focus removal: orthonormal mode bases of one WFS's slopes
    // [3][2 n_vs] and of the phase points [3][n_vphi]
    bool modes = false;
    double* d_Qs = nullptr;
    double* d_Qp = nullptr;
    float* s_proj = nullptr;           // M_s s of the current chunk
    // adjoint of the projection (built on first use) and the explicit reconstructor
    int* d_aptr = nullptr;             // transposed bilinear table [layer][m*m + 1]
    int* d_avi = nullptr;
    float* d_aw = nullptr;
    int *d_rowstart_m = nullptr, *d_col_m = nullptr, *d_rowcol_m = nullptr;
    MaskTables mt_m{};                 // every node of the m x m layer grid
    MvmGeom g_adj{};
    bool adj_ready = false;
    float2* d_Kadj = nullptr;          // [target] conjugate-transposed projection spectra
    float2 *Xa = nullptr, *Ya = nullptr;
    float *Yda = nullptr, *za = nullptr;
    float* gemm_part = nullptr;
    size_t gemm_part_size = 0;
    // block CG: small FP64 matrices [5][64 x 64] and the Gram workspace
    double* d_small = nullptr;
    double* h_small = nullptr;         // pinned host mirror of d_small
    // block solves of proportional per-frame operators (tomo_solve_r0): 1 / c_f
    double* d_rhs_scale = nullptr;
    double* d_gram_part = nullptr;
    // FFT-side autotuning (cfg.fft_P < 0): candidate sides and their measured
    // Sigma_ss product times [ms] (negative: the side could not run)
    std::vector<int> tune_P;
    std::vector<double> tune_ms;
    int* d_iidx = nullptr;
    float* d_iw = nullptr;
    // workspaces
    float2 *X1 = nullptr, *Y1 = nullptr, *Xc = nullptr, *Yc = nullptr;
    double2 *X1d = nullptr, *Y1d = nullptr;
    float* Ydc = nullptr;
    float *x = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr, *z = nullptr, *w = nullptr;
    double *xd = nullptr, *yd = nullptr;
    FrameState* st = nullptr;
    double *dot_part = nullptr, *dot_part_M = nullptr, *rr_part = nullptr, *init_part = nullptr, *res_part = nullptr;
    int nparts = 0;
    int* d_nactive = nullptr;
    int* h_nactive = nullptr;
    float *s_stage = nullptr, *z_stage = nullptr, *phi_stage = nullptr;
    GraphCache graph;
    std::vector<void*> allocs;
    // kernel timing (tomo_set_kernel_timing): eager CG iterations with events
    WarmStartNet ws;
    bool timing = false;
    double kt_ms[TOMO_NKERNELS] = {0};
    long long kt_n[TOMO_NKERNELS] = {0};
    long long frame_iters = 0;   // sum over frames of CG iterations in solves since the last reset
    std::vector<cudaEvent_t> ev;
    // FP64 solves (tomo_solve_f64) and the FP64 outer loop of mixed precision,
    // allocated on first use: vectors [B][N], partial sums [B][nparts] (x3 for dots)
    double *x64 = nullptr, *r64 = nullptr, *p64 = nullptr, *Ap64 = nullptr, *s64 = nullptr;
    double *rr64_part = nullptr, *dot64_part = nullptr;
    double *rel64 = nullptr, *snorm64 = nullptr;     // per frame: outer relative residual, ||s||^2
    float *rhs32 = nullptr, *d32 = nullptr;          // inner right-hand side and correction
    double2* d_fs_outer = nullptr;                   // per-frame (c_f, nu_f) of the outer operator
    // device-side loop: its state on the device, a pinned copy read back after
    // the launch, the right-hand side it recomputes the true residual from
    double* flex_part = nullptr;                     // flexible PCG partial sums [B][nparts][5]
    LoopGraph loop;
    LoopState* d_loop = nullptr;
    LoopState* h_loop = nullptr;
    bool loop_pending = false;                       // h_loop holds a launch not yet accounted for
    float* s_loop = nullptr;
    // wall-clock budget of the current call (tomo_solve_opts.deadline_ms)
    bool has_deadline = false, timed_out = false;
    std::chrono::steady_clock::time_point deadline{};
};

namespace {

const double kPi = 3.14159265358979323846;

#define CK(call)                                                         \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) {                                         \
            std::fprintf(stderr, "tomo: %s failed: %s (%s:%d)\n", #call, \
                         cudaGetErrorString(e_), __FILE__, __LINE__);    \
            return TOMO_ECUDA;                                           \
        }                                                                \
    } while (0)

template <typename Tp>
tomo_status dalloc(tomo_handle* h, Tp** ptr, size_t count) {
    void* v = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(&v, count * sizeof(Tp)) != cudaSuccess) {
        cudaGetLastError();
        return TOMO_ENOMEM;
    }
    h->allocs.push_back(v);
    *ptr = static_cast<Tp*>(v);
    return TOMO_OK;
}

#define TRY(expr)                          \
    do {                                   \
        tomo_status s_ = (expr);           \
        if (s_ != TOMO_OK) return s_;      \
    } while (0)

// Orthonormal rows spanning the three columns of Z ([3][len], row-major),
// modified Gram-Schmidt applied twice (FP64); false if Z is rank deficient.
bool orthonormal_rows(std::vector<double>& Z, int len) {
    for (int k = 0; k < 3; ++k) {
        double* zk = Z.data() + (size_t)k * len;
        const double n0 = std::sqrt(std::inner_product(zk, zk + len, zk, 0.0));
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j < k; ++j) {
                const double* zj = Z.data() + (size_t)j * len;
                const double c = std::inner_product(zk, zk + len, zj, 0.0);
                for (int e = 0; e < len; ++e) zk[e] -= c * zj[e];
            }
        const double nk = std::sqrt(std::inner_product(zk, zk + len, zk, 0.0));
        if (!(nk > 1e-9 * n0)) return false;
        for (int e = 0; e < len; ++e) zk[e] /= nk;
    }
    return true;
}

// Radix plan for P (factors 2, 3, 4, 5, 7); false if P has another prime factor.
bool make_plan(int P, FftPlan* pl) {
    pl->P = P;
    pl->nst = 0;
    int r = P;
    const int order[] = {5, 4, 3, 2, 7};
    for (int rad : order) {
        while (r % rad == 0) {
            if (pl->nst >= 8) return false;
            pl->rad[pl->nst++] = rad;
            r /= rad;
        }
    }
    return r == 1 && pl->nst > 0;
}

int smallest_fft_side(int pmin) {
    for (int P = pmin + (pmin & 1); ; P += 2) {
        FftPlan pl;
        if (make_plan(P, &pl)) return P;
    }
}

template <typename C>
std::vector<C> twiddles(int P) {
    std::vector<C> t(P);
    for (int k = 0; k < P; ++k) {
        const double a = -2.0 * kPi * (double)k / (double)P;
        t[k].x = (decltype(t[k].x))std::cos(a);
        t[k].y = (decltype(t[k].y))std::sin(a);
    }
    return t;
}

// Host-to-device copy ordered on the caller's stream (which may be non-blocking).
tomo_status upload(tomo_handle* h, const void* host, void* dev, size_t bytes) {
    CK(cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return TOMO_OK;
}

Launch launch_of(tomo_handle* h) { return Launch{h->stream, &h->launches}; }

// Row groups of the row passes for a batch of B frames: one block per plane
// while the batch fills a wave of the GPU, one block per group of row pairs
// when it does not (small batches, single-frame latency).
int rg_for(const tomo_handle* h, int B) { return (long long)h->NP * B >= h->block_slots ? 1 : h->rg; }

// Sigma_ss + noise on FP32 vectors; with cg != nullptr, one CG product (see rows_fwd).
tomo_status apply_ss32(tomo_handle* h, const Launch& L, const float* x, float* y, int B, const FrameState* st,
                       const CgVecs* cg, const double2* fscale = nullptr) {
    const int rg = rg_for(h, B);
    CK((rows_fwd<float, float>(L, h->g_ss, h->mt, B, x, cg, st, h->X1, h->d_tw32, rg)));
    CK((cols_mul<float>(L, h->g_ss, B, st, h->X1, h->Y1, h->d_K32, h->d_tw32, true)));
    const float* xin = cg ? cg->p : x;
    float* yout = cg ? cg->Ap : y;
    CK((rows_inv_masked<float, float>(L, h->g_ss, h->mt, B, st, h->Y1, xin, h->d_rows_noise, fscale, yout, cg,
                                      h->d_tw32, rg)));
    if (h->d_ncov)
        CK(noise_blocks<float>(L, B, h->n_vs, h->n_gs, rg, h->d_ncov, fscale, st, yout, xin, xin, cg));
    return TOMO_OK;
}

CgVecs cg_vecs(tomo_handle* h, int mode, double* dots) {
    return CgVecs{h->x, h->r, h->p, h->Ap, h->rr_part, dots, mode, h->z, h->w};
}

// FP64 product; with st, frames that are not active are skipped (y keeps its values there).
tomo_status apply_ss64(tomo_handle* h, const Launch& L, const double* x, double* y, int B,
                       const double2* fscale = nullptr, const FrameState* st = nullptr) {
    const int rg = rg_for(h, B);
    CK((rows_fwd<double, double>(L, h->g_ss, h->mt, B, x, nullptr, st, h->X1d, h->d_tw64, rg)));
    CK((cols_mul<double>(L, h->g_ss, B, st, h->X1d, h->Y1d, h->d_K64, h->d_tw64, false)));
    CK((rows_inv_masked<double, double>(L, h->g_ss, h->mt, B, st, h->Y1d, x, h->d_rows_noise, fscale, y,
                                        nullptr, h->d_tw64, rg)));
    if (h->d_ncov)
        CK(noise_blocks<double>(L, B, h->n_vs, h->n_gs, rg, h->d_ncov, fscale, st, y, x, nullptr, nullptr));
    return TOMO_OK;
}

// A bounded wait of a kernel (a bulk copy's mbarrier) that expired since the
// last check is reported as TOMO_ETIMEOUT (the flag is per device).  Call after
// the work has been synchronised.
tomo_status check_wait_error() {
    int flag = 0;
    CK(take_wait_error(&flag));
    if (flag) {
        std::fprintf(stderr, "tomo: a bounded device wait expired (a bulk copy did not complete)\n");
        return TOMO_ETIMEOUT;
    }
    return TOMO_OK;
}

// Wall-clock budget of a solve call (tomo_solve_opts.deadline_ms).
void begin_call(tomo_handle* h, const tomo_solve_opts& o) {
    h->timed_out = false;
    h->has_deadline = o.deadline_ms > 0;
    if (h->has_deadline)
        h->deadline = std::chrono::steady_clock::now() +
                      std::chrono::microseconds((long long)std::ceil(o.deadline_ms * 1000.0));
}

bool past_deadline(tomo_handle* h) {
    if (!h->has_deadline || std::chrono::steady_clock::now() < h->deadline) return false;
    h->timed_out = true;
    return true;
}

// Buffers of the FP64 solves and of the mixed-precision outer loop (first use).
tomo_status ensure_f64(tomo_handle* h) {
    if (h->x64) return TOMO_OK;
    const size_t BN = (size_t)h->max_batch * h->N, B = h->max_batch;
    TRY(dalloc(h, &h->x64, BN));
    TRY(dalloc(h, &h->r64, BN));
    TRY(dalloc(h, &h->p64, BN));
    TRY(dalloc(h, &h->Ap64, BN));
    TRY(dalloc(h, &h->s64, BN));
    TRY(dalloc(h, &h->rr64_part, B * h->nparts));
    TRY(dalloc(h, &h->dot64_part, B * h->nparts * 3));
    TRY(dalloc(h, &h->rel64, B));
    TRY(dalloc(h, &h->snorm64, B));
    TRY(dalloc(h, &h->rhs32, BN));
    TRY(dalloc(h, &h->d32, BN));
    TRY(dalloc(h, &h->d_fs_outer, B));
    return TOMO_OK;
}

tomo_status apply_os(tomo_handle* h, const Launch& L, const float* z, float* phi, int B,
                     const double2* fscale = nullptr) {
    CK((rows_fwd<float, float>(L, h->g_os, h->mt, B, z, nullptr, nullptr, h->Xc, h->d_twc32, rg_for(h, B))));
    const size_t kc_stride = (size_t)h->g_os.nh * h->Pc * h->cos_layers * h->NP;
    for (int t = 0; t < h->n_targets; ++t) {
        CK((cols_mul<float>(L, h->g_os, B, nullptr, h->Xc, h->Yc, h->d_Kc32 + t * kc_stride, h->d_twc32, false)));
        CK((rows_inv_dense<float>(L, h->g_os, B, h->Yc, h->Ydc, h->d_twc32)));
        CK(interp(L, B, h->n_targets, t, h->cos_layers, h->m, h->n_vphi, h->Ydc, h->d_iidx, h->d_iw, fscale,
                  phi));
    }
    return TOMO_OK;
}

// One CG iteration on all active frames of the batch: the previous update and
// the new direction (row-forward pass), A p (column and row-inverse passes),
// and the per-frame scalars.
//
// One PCG iteration (Chronopoulos & Gear): the previous update and FFT of r
// (row-forward), z = M^{-1} r (column pass with M, row-inverse pass with
// r^T z), w = A z (three passes, z^T w), and the per-frame scalars.
//
// With marks != nullptr every kernel is bracketed by events (kernel timing).
//
// One MINRES iteration (conjugate-residual form): the previous update and FFT
// of r (row-forward), w = A r with r^T w, Ap^T w, w^T w (column and
// row-inverse passes), and the per-frame scalars.
//
// One FP64 CG iteration (tomo_solve_f64): the scheduled update and new
// direction (cg64_update), A p with the FP64 product, the partial sums, and
// the per-frame scalars.
//
// One flexible PCG iteration with the learned preconditioner (flex.cu): z from
// the network on [r, M r] (M r kept for the fallback), the per-frame
// convergence test, fallback decisions and beta, the new direction, q = A p,
// alpha and the update.
enum IterKind { kIterCG = 0, kIterPCG = 1, kIterMINRES = 2, kIterCG64 = 3, kIterFlex = 4 };

// Iterations without a new minimum of r^T r after which a flexible-PCG frame
// falls back to PCG with M.
constexpr int kFlexWindow = 64;

tomo_status ws_forward(tomo_handle* h, const Launch& L, const float* s, int B, float* zeta);

tomo_status iteration(tomo_handle* h, const Launch& L, int B, int kind, std::vector<std::pair<int, int>>* marks) {
    int last = -1;
    auto mark = [&](int slot) -> tomo_status {
        if (!marks) return TOMO_OK;
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return TOMO_ECUDA;
        h->ev.push_back(e);
        if (cudaEventRecord(e, L.stream) != cudaSuccess) return TOMO_ECUDA;
        const int id = (int)h->ev.size() - 1;
        if (last >= 0) marks->push_back({last * 8 + slot, id});
        last = id;
        return TOMO_OK;
    };
    // slot encoding: pair (start event * 8 + kernel class, end event)
    const int rg = rg_for(h, B);
    TRY(mark(0));
    if (kind == kIterFlex) {
        // z = pre_gain M r + out_scale N([r, M r]) (into z), M r (into w)
        const WarmStartNet& w = h->ws;
        for (int b0 = 0; b0 < B; b0 += w.maxB) {
            const int nb = std::min(w.maxB, B - b0);
            TRY(ws_forward(h, L, h->r + (size_t)b0 * h->N, nb, h->z + (size_t)b0 * h->N));
            CK(cudaMemcpyAsync(h->w + (size_t)b0 * h->N, w.zpre, sizeof(float) * nb * h->N, cudaMemcpyDeviceToDevice,
                               L.stream));
        }
        TRY(mark(1));
        CK(flex_dots(L, B, h->N, h->nparts, h->st, h->r, h->Ap, h->z, h->w, h->flex_part));
        CK(flex_beta(L, B, h->nparts, h->flex_part, kFlexWindow, h->st));
        CK(flex_dir(L, B, h->N, h->st, h->z, h->w, h->p));
        TRY(mark(3));
        TRY(apply_ss32(h, L, h->p, h->Ap, B, h->st, nullptr, h->d_fscale));
        TRY(mark(2));
        CK(flex_pq(L, B, h->N, h->nparts, h->st, h->p, h->Ap, h->flex_part));
        CK(flex_alpha(L, B, h->nparts, h->flex_part, h->st));
        CK(flex_update(L, B, h->N, h->st, h->x, h->r, h->p, h->Ap));
        TRY(mark(3));
        return TOMO_OK;
    }
    if (kind == kIterCG64) {
        CK(cg64_update(L, B, h->N, h->nparts, h->st, h->x64, h->r64, h->p64, h->Ap64, h->rr64_part));
        TRY(mark(0));
        TRY(apply_ss64(h, L, h->p64, h->Ap64, B, h->d_fscale, h->st));
        if (h->modes)
            CK(mode_project<double>(L, B, 2 * h->n_vs, h->n_gs, 1, h->d_Qs, h->st, h->Ap64, nullptr, nullptr));
        TRY(mark(2));
        CK(cg64_dots(L, B, h->N, h->nparts, h->st, h->p64, h->r64, h->Ap64, h->dot64_part));
        CK(cg_scalars(L, B, h->nparts, h->rr64_part, h->dot64_part, h->st));
        TRY(mark(3));
        return TOMO_OK;
    }
    if (kind == kIterMINRES) {
        const CgVecs cg = cg_vecs(h, 3, h->dot_part);
        CK((rows_fwd<float, float>(L, h->g_ss, h->mt, B, nullptr, &cg, h->st, h->X1, h->d_tw32, rg)));
        TRY(mark(0));
        CK((cols_mul<float>(L, h->g_ss, B, h->st, h->X1, h->Y1, h->d_K32, h->d_tw32, true)));
        TRY(mark(1));
        CK((rows_inv_masked<float, float>(L, h->g_ss, h->mt, B, h->st, h->Y1, h->r, h->d_rows_noise, h->d_fscale,
                                          h->w, &cg, h->d_tw32, rg)));
        if (h->d_ncov)
            CK(noise_blocks<float>(L, B, h->n_vs, h->n_gs, rg, h->d_ncov, h->d_fscale, h->st, h->w, h->r, h->r, &cg));
        if (h->modes) CK(mode_project<float>(L, B, 2 * h->n_vs, h->n_gs, rg, h->d_Qs, h->st, h->w, h->r, &cg));
        TRY(mark(2));
        CK(mr_scalars(L, B, h->NP * rg, h->rr_part, h->dot_part, h->st));
        TRY(mark(3));
        return TOMO_OK;
    }
    if (kind == kIterCG) {
        const CgVecs cg = cg_vecs(h, 1, h->dot_part);
        CK((rows_fwd<float, float>(L, h->g_ss, h->mt, B, nullptr, &cg, h->st, h->X1, h->d_tw32, rg)));
        TRY(mark(0));
        CK((cols_mul<float>(L, h->g_ss, B, h->st, h->X1, h->Y1, h->d_K32, h->d_tw32, true)));
        TRY(mark(1));
        CK((rows_inv_masked<float, float>(L, h->g_ss, h->mt, B, h->st, h->Y1, h->p, h->d_rows_noise, h->d_fscale,
                                          h->Ap, &cg, h->d_tw32, rg)));
        if (h->d_ncov)
            CK(noise_blocks<float>(L, B, h->n_vs, h->n_gs, rg, h->d_ncov, h->d_fscale, h->st, h->Ap, h->p, h->p, &cg));
        if (h->modes) CK(mode_project<float>(L, B, 2 * h->n_vs, h->n_gs, rg, h->d_Qs, h->st, h->Ap, h->p, &cg));
        TRY(mark(2));
        CK(cg_scalars(L, B, h->NP * rg, h->rr_part, h->dot_part, h->st));
        TRY(mark(3));
        return TOMO_OK;
    }
    const CgVecs cgM = cg_vecs(h, 2, h->dot_part_M);
    const CgVecs cgA = cg_vecs(h, 2, h->dot_part);
    CK((rows_fwd<float, float>(L, h->g_ss, h->mt, B, nullptr, &cgM, h->st, h->X1, h->d_tw32, rg)));
    TRY(mark(0));
    CK((cols_mul<float>(L, h->g_ss, B, h->st, h->X1, h->Y1, h->d_M32, h->d_tw32, true)));
    TRY(mark(1));
    CK((rows_inv_masked<float, float>(L, h->g_ss, h->mt, B, h->st, h->Y1, h->r, h->d_zero_var, h->d_fscale_pre,
                                      h->z, &cgM, h->d_tw32, rg)));
    if (h->modes) CK(mode_project<float>(L, B, 2 * h->n_vs, h->n_gs, rg, h->d_Qs, h->st, h->z, h->r, &cgM));
    TRY(mark(2));
    CK((rows_fwd<float, float>(L, h->g_ss, h->mt, B, h->z, nullptr, h->st, h->X1, h->d_tw32, rg)));
    TRY(mark(0));
    CK((cols_mul<float>(L, h->g_ss, B, h->st, h->X1, h->Y1, h->d_K32, h->d_tw32, true)));
    TRY(mark(1));
    CK((rows_inv_masked<float, float>(L, h->g_ss, h->mt, B, h->st, h->Y1, h->z, h->d_rows_noise, h->d_fscale,
                                      h->w, &cgA, h->d_tw32, rg)));
    if (h->d_ncov)
        CK(noise_blocks<float>(L, B, h->n_vs, h->n_gs, rg, h->d_ncov, h->d_fscale, h->st, h->w, h->z, h->z, &cgA));
    if (h->modes) CK(mode_project<float>(L, B, 2 * h->n_vs, h->n_gs, rg, h->d_Qs, h->st, h->w, h->z, &cgA));
    TRY(mark(2));
    CK(pcg_scalars(L, B, h->NP * rg, h->rr_part, h->dot_part_M, h->dot_part, h->st));
    TRY(mark(3));
    return TOMO_OK;
}

void collect_timing(tomo_handle* h, std::vector<std::pair<int, int>>& marks) {
    for (const auto& m : marks) {
        float ms = 0.f;
        const int start = m.first / 8, slot = m.first % 8;
        if (cudaEventElapsedTime(&ms, h->ev[start], h->ev[m.second]) == cudaSuccess) {
            h->kt_ms[slot] += ms;
            h->kt_n[slot] += 1;
        }
    }
    marks.clear();
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    h->ev.clear();
}

tomo_status build_graph(tomo_handle* h, int B, int iters, int kind) {
    if (h->graph.exec && h->graph.B == B && h->graph.iters == iters && h->graph.mode == kind) return TOMO_OK;
    if (h->graph.exec) {
        cudaGraphExecDestroy(h->graph.exec);
        h->graph.exec = nullptr;
    }
    long long before = h->launches;
    CK(cudaStreamBeginCapture(h->work, cudaStreamCaptureModeThreadLocal));
    Launch Lc{h->work, &h->launches};
    tomo_status s = TOMO_OK;
    for (int i = 0; i < iters && s == TOMO_OK; ++i) s = iteration(h, Lc, B, kind, nullptr);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->work, &graph);
    const long long nodes = h->launches - before;
    h->launches = before;
    if (s != TOMO_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return TOMO_ECUDA;
    e = cudaGraphInstantiate(&h->graph.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return TOMO_ECUDA;
    h->graph.B = B;
    h->graph.iters = iters;
    h->graph.mode = kind;
    h->graph.nodes = nodes;
    return TOMO_OK;
}

tomo_status validate(const tomo_config* c) {
    if (!c || !c->gs || !c->layer_h || !c->layer_frac || !c->target_x || !c->target_y) return TOMO_EINVAL;
    if (c->n < 2 || c->n > 1024 || c->n_gs < 1 || 2 * c->n_gs > 16 || c->n_layers < 1 || c->n_targets < 1)
        return TOMO_EINVAL;
    if (!(c->D > 0) || !(c->obstruction >= 0) || !(c->obstruction < 1) || !(c->r0 > 0) || !(c->L0 > 0))
        return TOMO_EINVAL;
    if (!(c->precond_floor >= 0)) return TOMO_EINVAL;
    if (c->mode_removal != 0 && c->mode_removal != 1) return TOMO_EINVAL;
    if (c->slope_model != TOMO_SLOPE_HUDGIN && c->slope_model != TOMO_SLOPE_FRIED) return TOMO_EINVAL;
    if (c->max_batch < 1 || c->max_batch > 4096) return TOMO_EINVAL;
    const double H = c->gs[0].height;
    for (int g = 0; g < c->n_gs; ++g) {
        if (c->gs[g].height != H) return TOMO_EINVAL;  // one altitude: every Theta_pq block stays 2RBT
        if (!(c->gs[g].height >= 0) || !(c->gs[g].noise_sigma >= 0)) return TOMO_EINVAL;
    }
    for (int k = 0; k < c->n_layers; ++k) {
        if (!(c->layer_frac[k] > 0) || !(c->layer_h[k] >= 0)) return TOMO_EINVAL;
        if (H > 0 && !(c->layer_h[k] < H)) return TOMO_EINVAL;
    }
    return TOMO_OK;
}

// Picks the Sigma_ss FFT side P by timing the FP32 product (three passes) on
// min(max_batch, 64) frames for every even P in [2n - 1, 1.25 (2n - 1)] with
// radices 2..7 (at most 6 sides).  The product's run time does not depend on
// the values, so the spectra are zeros here; the chosen side's real spectra
// are built afterwards.  Needs the mask tables and the noise variances.
tomo_status autotune_side(tomo_handle* h) {
    const int n = h->n, pmin = 2 * n - 1;
    const int pmax = (int)std::ceil(1.25 * pmin);
    h->tune_P.clear();
    h->tune_ms.clear();
    for (int P = pmin + (pmin & 1); P <= pmax && h->tune_P.size() < 6; P += 2) {
        FftPlan pl;
        if (make_plan(P, &pl)) h->tune_P.push_back(P);
    }
    if (h->tune_P.empty()) h->tune_P.push_back(smallest_fft_side(pmin));
    const int B = std::min(h->max_batch, 64);
    const int Pmax = *std::max_element(h->tune_P.begin(), h->tune_P.end());
    const size_t nhmax = Pmax / 2 + 1;
    float *x = nullptr, *y = nullptr;
    float2 *X1 = nullptr, *Y1 = nullptr, *K = nullptr, *tw = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        cudaFree(x); cudaFree(y); cudaFree(X1); cudaFree(Y1); cudaFree(K); cudaFree(tw);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    const size_t nK = herm_packed_elems(Pmax, h->NP);
    const size_t nX = (size_t)B * h->NP * nhmax * n;
    if (cudaMalloc(&x, sizeof(float) * B * h->N) != cudaSuccess || cudaMalloc(&y, sizeof(float) * B * h->N) ||
        cudaMalloc(&X1, sizeof(float2) * nX) || cudaMalloc(&Y1, sizeof(float2) * nX) ||
        cudaMalloc(&K, sizeof(float2) * nK) || cudaMalloc(&tw, sizeof(float2) * Pmax) ||
        cudaEventCreate(&e0) || cudaEventCreate(&e1)) {
        cleanup();
        cudaGetLastError();
        return TOMO_ENOMEM;
    }
    Launch L{h->stream, nullptr};
    double best = 0.0;
    int bestP = 0;
    cudaError_t err = cudaMemsetAsync(x, 0, sizeof(float) * B * h->N, h->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(K, 0, sizeof(float2) * nK, h->stream);
    for (int P : h->tune_P) {
        FftPlan pl;
        make_plan(P, &pl);
        const MvmGeom g{n, n, h->NP, h->NP, P / 2 + 1, pl};
        const auto t = twiddles<float2>(P);
        if (err == cudaSuccess) err = cudaMemcpyAsync(tw, t.data(), sizeof(float2) * P, cudaMemcpyHostToDevice, h->stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
        if (err != cudaSuccess) break;
        auto product = [&]() -> cudaError_t {
            cudaError_t e = rows_fwd<float, float>(L, g, h->mt, B, x, nullptr, nullptr, X1, tw);
            if (e == cudaSuccess) e = cols_mul<float>(L, g, B, nullptr, X1, Y1, K, tw, true);
            if (e == cudaSuccess)
                e = rows_inv_masked<float, float>(L, g, h->mt, B, nullptr, Y1, x, h->d_noise_var, nullptr, y, nullptr,
                                                  tw);
            return e;
        };
        double ms = -1.0;
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = product();
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
        for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = product();
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t_ms = 0.f;
        if (e == cudaSuccess && cudaEventElapsedTime(&t_ms, e0, e1) == cudaSuccess) ms = t_ms / 5.0;
        if (e == cudaErrorInvalidValue) {
            cudaGetLastError();       // a launch configuration this side cannot use: skip it
        } else if (e != cudaSuccess) {
            err = e;
            break;
        }
        h->tune_ms.push_back(ms);
        if (ms > 0 && (bestP == 0 || ms < best)) { best = ms; bestP = P; }
    }
    cleanup();
    if (err != cudaSuccess) {
        std::fprintf(stderr, "tomo: FFT-side autotuning failed: %s\n", cudaGetErrorString(err));
        return TOMO_ECUDA;
    }
    if (bestP == 0) return TOMO_EINVAL;
    h->P = bestP;
    return TOMO_OK;
}

tomo_status create_impl(const tomo_config* c, void* stream, tomo_handle* h) {
    h->stream = static_cast<cudaStream_t>(stream);
    CK(init_kernel_attributes());
    CK(cudaStreamCreateWithFlags(&h->work, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    h->n = c->n;
    h->n_gs = c->n_gs;
    h->NP = 2 * c->n_gs;
    h->n_layers = c->n_layers;
    h->n_targets = c->n_targets;
    h->D = c->D;
    h->obstruction = c->obstruction;
    h->d = c->D / c->n;
    h->r0 = c->r0;
    h->L0 = c->L0;
    h->max_batch = c->max_batch;
    h->slope_model = c->slope_model;
    h->all_ngs = c->gs[0].height == 0.0;
    const int n = h->n;

    // --- geometry (Sec. 2.F): centre-in-annulus rule, in integers ---------------
    h->subap_mask.assign((size_t)n * n, 0);
    const double thr = (c->obstruction * n) * (c->obstruction * n);
    std::vector<int> rowstart(n + 1, 0), col;
    for (int i = 0; i < n; ++i) {
        rowstart[i] = (int)col.size();
        for (int j = 0; j < n; ++j) {
            const long long a = 2LL * j + 1 - n, b = 2LL * i + 1 - n;
            const long long q = a * a + b * b;
            if (q <= (long long)n * n && (double)q >= thr) {
                h->subap_mask[(size_t)i * n + j] = 1;
                col.push_back(j);
            }
        }
    }
    rowstart[n] = (int)col.size();
    h->n_vs = (int)col.size();
    if (h->n_vs == 0) return TOMO_EINVAL;
    h->N = h->NP * h->n_vs;
    h->rg = row_groups(n);
    {
        int dev = 0, sms = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        h->block_slots = sms * TOMO_MIN_BLOCKS;
    }
    h->phase_mask.assign((size_t)(n + 1) * (n + 1), 0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (h->subap_mask[(size_t)i * n + j])
                for (int di = 0; di < 2; ++di)
                    for (int dj = 0; dj < 2; ++dj) h->phase_mask[(size_t)(i + di) * (n + 1) + j + dj] = 1;
    std::vector<int> pv_i, pv_j;
    for (int i = 0; i <= n; ++i)
        for (int j = 0; j <= n; ++j)
            if (h->phase_mask[(size_t)i * (n + 1) + j]) { pv_i.push_back(i); pv_j.push_back(j); }
    h->n_vphi = (int)pv_i.size();
    h->ph_i = pv_i;
    h->ph_j = pv_j;
    h->frac_sum = 0.0;
    for (int k = 0; k < c->n_layers; ++k) h->frac_sum += c->layer_frac[k];
    if (c->mode_removal) {
        // Z_s: slopes of tip x, tilt y and focus x^2 + y^2 on one WFS; the
        // two-point slopes (Appendix A.2) of these modes at the subaperture
        // centre (xc, yc) are (d, 0), (0, d) and (2 d xc, 2 d yc); the common
        // factor d does not change the span
        const int len = 2 * h->n_vs;
        std::vector<double> Zs((size_t)3 * len, 0.0);
        int e = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                if (h->subap_mask[(size_t)i * n + j]) {
                    const double xc = (j + 0.5 - 0.5 * n) * h->d, yc = (i + 0.5 - 0.5 * n) * h->d;
                    Zs[e] = 1.0;
                    Zs[(size_t)len + h->n_vs + e] = 1.0;
                    Zs[(size_t)2 * len + e] = 2.0 * xc;
                    Zs[(size_t)2 * len + h->n_vs + e] = 2.0 * yc;
                    ++e;
                }
        std::vector<double> Zp((size_t)3 * h->n_vphi);
        for (int v = 0; v < h->n_vphi; ++v) {
            const double x = (pv_j[v] - 0.5 * n) * h->d, y = (pv_i[v] - 0.5 * n) * h->d;
            Zp[v] = x;
            Zp[(size_t)h->n_vphi + v] = y;
            Zp[(size_t)2 * h->n_vphi + v] = x * x + y * y;
        }
        if (!orthonormal_rows(Zs, len) || !orthonormal_rows(Zp, h->n_vphi)) return TOMO_EINVAL;
        h->modes = true;
        TRY(dalloc(h, &h->d_Qs, Zs.size()));
        TRY(dalloc(h, &h->d_Qp, Zp.size()));
        TRY(upload(h, Zs.data(), h->d_Qs, sizeof(double) * Zs.size()));
        TRY(upload(h, Zp.data(), h->d_Qp, sizeof(double) * Zp.size()));
    }

    // --- layers: B_k(0) = c_v (L0/r0)^{5/3} f_k and cone factors ------------------
    const double cv = std::pow(24.0 / 5.0 * std::tgamma(6.0 / 5.0), 5.0 / 6.0) * std::tgamma(11.0 / 6.0) *
                      std::tgamma(5.0 / 6.0) / (2.0 * std::pow(kPi, 8.0 / 3.0));
    const double Hgs = c->gs[0].height;
    std::vector<LayerGeom> layers(h->n_layers);
    double gmin = 1.0;
    for (int k = 0; k < h->n_layers; ++k) {
        layers[k].h = c->layer_h[k];
        layers[k].amp = cv * std::pow(c->L0 / c->r0, 5.0 / 3.0) * c->layer_frac[k];
        layers[k].gamma = Hgs > 0 ? 1.0 - c->layer_h[k] / Hgs : 1.0;
        gmin = std::min(gmin, layers[k].gamma);
    }
    // n' of the new phase grid (Sec. 2.D): covers the n+1 phase points at spacing gamma_min d
    h->m = h->all_ngs ? n + 1 : (int)std::ceil((double)n / gmin - 1e-9) + 1;
    h->cos_layers = h->all_ngs ? 1 : h->n_layers;

    // --- device tables -------------------------------------------------------------
    TRY(dalloc(h, &h->d_rowstart, n + 1));
    TRY(dalloc(h, &h->d_col, h->n_vs));
    TRY(upload(h, rowstart.data(), h->d_rowstart, sizeof(int) * (n + 1)));
    TRY(upload(h, col.data(), h->d_col, sizeof(int) * h->n_vs));
    std::vector<int> rowcol(h->n_vs);
    for (int i = 0; i < n; ++i)
        for (int e = rowstart[i]; e < rowstart[i + 1]; ++e) rowcol[e] = (i << 16) | col[e];
    TRY(dalloc(h, &h->d_rowcol, h->n_vs));
    TRY(upload(h, rowcol.data(), h->d_rowcol, sizeof(int) * h->n_vs));
    h->mt = MaskTables{h->d_rowstart, h->d_col, h->d_rowcol, h->n_vs};
    std::vector<double> nvar(h->NP);
    for (int p = 0; p < h->NP; ++p) nvar[p] = c->gs[p / 2].noise_sigma * c->gs[p / 2].noise_sigma;
    TRY(dalloc(h, &h->d_noise_var, h->NP));
    TRY(upload(h, nvar.data(), h->d_noise_var, sizeof(double) * h->NP));
    h->d_rows_noise = h->d_noise_var;
    if (c->noise_cov) {
        // gather the valid subapertures' blocks: [n_gs][n][n][3] -> [n_gs][n_vs][3]
        const size_t nc = (size_t)h->n_gs * h->n_vs * 3;
        std::vector<double> blocks(nc);
        for (int g = 0; g < h->n_gs; ++g)
            for (int i = 0; i < n; ++i)
                for (int e = rowstart[i]; e < rowstart[i + 1]; ++e) {
                    const double* src = c->noise_cov + (((size_t)g * n + i) * n + col[e]) * 3;
                    const double a = src[0], b = src[1], x = src[2];
                    if (!(a >= 0) || !(b >= 0) || !std::isfinite(a) || !std::isfinite(b) || !std::isfinite(x) ||
                        !(a * b - x * x >= 0))
                        return TOMO_EINVAL;
                    std::memcpy(&blocks[((size_t)g * h->n_vs + e) * 3], src, 3 * sizeof(double));
                }
        TRY(dalloc(h, &h->d_ncov, nc));
        TRY(upload(h, blocks.data(), h->d_ncov, sizeof(double) * nc));
        // the preconditioner's noise floor of each guide star: the mean
        // eigenvalue (s_xx + s_yy) / 2 of its blocks
        if (h->n_vs > 0) {
            for (int g = 0; g < h->n_gs; ++g) {
                double t = 0.0;
                for (int e = 0; e < h->n_vs; ++e)
                    t += 0.5 * (blocks[((size_t)g * h->n_vs + e) * 3] + blocks[((size_t)g * h->n_vs + e) * 3 + 1]);
                nvar[2 * g] = nvar[2 * g + 1] = t / h->n_vs;
            }
            TRY(upload(h, nvar.data(), h->d_noise_var, sizeof(double) * h->NP));
        }
        const std::vector<double> zero(h->NP, 0.0);
        TRY(dalloc(h, &h->d_rows_noise, h->NP));
        TRY(upload(h, zero.data(), h->d_rows_noise, sizeof(double) * h->NP));
    }

    // --- FFT sides and plans ----------------------------------------------------------
    if (c->fft_P < 0) TRY(autotune_side(h));
    h->P = c->fft_P > 0 ? c->fft_P : (c->fft_P < 0 ? h->P : smallest_fft_side(2 * n - 1));
    h->Pc = c->fft_Pcos > 0 ? c->fft_Pcos : smallest_fft_side(h->m + n - 1);
    if (h->P < 2 * n - 1 || (h->P & 1) || h->Pc < h->m + n - 1 || (h->Pc & 1)) return TOMO_EINVAL;
    if (!make_plan(h->P, &h->plan) || !make_plan(h->Pc, &h->planc)) return TOMO_EINVAL;
    if (h->cos_layers > 16) return TOMO_ERANGE;
    h->g_ss = MvmGeom{n, n, h->NP, h->NP, h->P / 2 + 1, h->plan};
    h->g_os = MvmGeom{n, h->m, h->NP, h->cos_layers, h->Pc / 2 + 1, h->planc};
    auto tw32 = twiddles<float2>(h->P);
    auto tw64 = twiddles<double2>(h->P);
    auto twc32 = twiddles<float2>(h->Pc);
    auto twc64 = twiddles<double2>(h->Pc);
    double2* d_twc64 = nullptr;
    TRY(dalloc(h, &h->d_tw32, h->P));
    TRY(dalloc(h, &h->d_tw64, h->P));
    TRY(dalloc(h, &h->d_twc32, h->Pc));
    TRY(dalloc(h, &d_twc64, h->Pc));
    TRY(upload(h, tw32.data(), h->d_tw32, sizeof(float2) * h->P));
    TRY(upload(h, tw64.data(), h->d_tw64, sizeof(double2) * h->P));
    TRY(upload(h, twc32.data(), h->d_twc32, sizeof(float2) * h->Pc));
    TRY(upload(h, twc64.data(), d_twc64, sizeof(double2) * h->Pc));

    // quadrature tables for K_{5/6} (step 0.2, t up to 40)
    const int nq = 200;
    const double hq = 0.2;
    std::vector<double> ct(nq), cnt(nq);
    for (int i = 0; i < nq; ++i) {
        ct[i] = std::cosh(i * hq);
        cnt[i] = std::cosh(5.0 / 6.0 * i * hq);
    }
    double *d_ct = nullptr, *d_cnt = nullptr, *d_alpha = nullptr;
    LayerGeom* d_layers = nullptr;
    TRY(dalloc(h, &d_ct, nq));
    TRY(dalloc(h, &d_cnt, nq));
    TRY(upload(h, ct.data(), d_ct, sizeof(double) * nq));
    TRY(upload(h, cnt.data(), d_cnt, sizeof(double) * nq));
    VkParams vk{c->L0, std::pow(2.0, 1.0 / 6.0) / std::tgamma(5.0 / 6.0), d_ct, d_cnt, nq, hq};
    std::vector<double> alpha(2 * h->n_gs);
    for (int g = 0; g < h->n_gs; ++g) { alpha[2 * g] = c->gs[g].alpha_x; alpha[2 * g + 1] = c->gs[g].alpha_y; }
    TRY(dalloc(h, &d_alpha, 2 * h->n_gs));
    TRY(upload(h, alpha.data(), d_alpha, sizeof(double) * 2 * h->n_gs));
    TRY(dalloc(h, &d_layers, h->n_layers));
    TRY(upload(h, layers.data(), d_layers, sizeof(LayerGeom) * h->n_layers));

    Launch L = launch_of(h);
    // --- Sigma_ss generators and spectra (FP64 on the device) ------------------------
    {
        const int npl = h->NP * h->NP;
        const size_t Gsz = (size_t)npl * h->P * h->P;
        double* G = nullptr;
        double2* H = nullptr;
        CK(cudaMalloc(&G, sizeof(double) * Gsz));
        CK(cudaMalloc(&H, sizeof(double2) * (size_t)npl * (h->P / 2 + 1) * h->P));
        float2* Kfull = nullptr;
        CK(cudaMalloc(&Kfull, sizeof(float2) * (size_t)npl * (h->P / 2 + 1) * h->P));
        TRY(dalloc(h, &h->d_K64, (size_t)npl * (h->P / 2 + 1) * h->P));
        TRY(dalloc(h, &h->d_K32, herm_packed_elems(h->P, h->NP)));
        CK(cudaMemsetAsync(G, 0, sizeof(double) * Gsz, h->stream));
        CK(gen_css(L, n, h->P, h->NP, h->d, h->n_layers, d_layers, d_alpha, vk, G, false, h->slope_model));
        CK(spectra(L, h->P, npl, h->NP, h->plan, G, H, h->d_tw64, h->d_K64, Kfull));
        CK(pack_hermitian(L, h->P, h->NP, Kfull, h->d_K32));
        CK(cudaStreamSynchronize(h->stream));
        cudaFree(G);
        cudaFree(H);
        cudaFree(Kfull);
    }
    // --- block-circulant preconditioner on the same P x P torus ------------------------
    if (c->precond) {
        const int npl = h->NP * h->NP;
        const size_t Gsz = (size_t)npl * h->P * h->P;
        const size_t Ksz = (size_t)npl * (h->P / 2 + 1) * h->P;
        double* G = nullptr;
        double2 *H = nullptr, *K64 = nullptr;
        CK(cudaMalloc(&G, sizeof(double) * Gsz));
        CK(cudaMalloc(&H, sizeof(double2) * Ksz));
        CK(cudaMalloc(&K64, sizeof(double2) * Ksz));
        float2* Mfull = nullptr;
        CK(cudaMalloc(&Mfull, sizeof(float2) * Ksz));
        TRY(dalloc(h, &h->d_M32, herm_packed_elems(h->P, h->NP)));
        TRY(dalloc(h, &h->d_zero_var, h->NP));
        CK(cudaMemsetAsync(h->d_zero_var, 0, sizeof(double) * h->NP, h->stream));
        CK(cudaMemsetAsync(G, 0, sizeof(double) * Gsz, h->stream));
        CK(gen_css(L, n, h->P, h->NP, h->d, h->n_layers, d_layers, d_alpha, vk, G, true, h->slope_model));
        CK(spectra(L, h->P, npl, h->NP, h->plan, G, H, h->d_tw64, K64, nullptr));
        const double floor_c = c->precond_floor > 0 ? c->precond_floor : 3.0;
        CK(precond_spectra(L, h->P, h->NP, K64, h->d_noise_var, floor_c, Mfull));
        CK(pack_hermitian(L, h->P, h->NP, Mfull, h->d_M32));
        CK(cudaStreamSynchronize(h->stream));
        cudaFree(G);
        cudaFree(H);
        cudaFree(K64);
        cudaFree(Mfull);
    }
    // --- Sigma_phi_s generators and spectra, one set per target ------------------------
    {
        const int npl = h->cos_layers * h->NP;
        const size_t Gsz = (size_t)npl * h->Pc * h->Pc;
        const size_t kstride = (size_t)npl * (h->Pc / 2 + 1) * h->Pc;
        double* G = nullptr;
        double2* H = nullptr;
        CK(cudaMalloc(&G, sizeof(double) * Gsz));
        CK(cudaMalloc(&H, sizeof(double2) * (size_t)npl * (h->Pc / 2 + 1) * h->Pc));
        TRY(dalloc(h, &h->d_Kc32, kstride * h->n_targets));
        for (int t = 0; t < h->n_targets; ++t) {
            CK(cudaMemsetAsync(G, 0, sizeof(double) * Gsz, h->stream));
            CK(gen_cos(L, n, h->m, h->Pc, h->NP, h->d, h->all_ngs ? -h->n_layers : h->n_layers, d_layers, d_alpha,
                       c->target_x[t], c->target_y[t], vk, G, h->slope_model));
            CK(spectra(L, h->Pc, npl, h->NP, h->planc, G, H, d_twc64, nullptr, h->d_Kc32 + t * kstride));
        }
        CK(cudaStreamSynchronize(h->stream));
        cudaFree(G);
        cudaFree(H);
    }
    // --- bilinear interpolation I'_k (Eq. interp) from layer k's grid to the phase points ---
    {
        const int m = h->m, L_ = h->cos_layers;
        std::vector<int> idx((size_t)L_ * h->n_vphi * 4);
        std::vector<float> w((size_t)L_ * h->n_vphi * 4);
        for (int k = 0; k < L_; ++k) {
            const double dk = (h->all_ngs ? 1.0 : layers[k].gamma) * h->d;
            for (int v = 0; v < h->n_vphi; ++v) {
                const double x = (pv_j[v] - n / 2.0) * h->d, y = (pv_i[v] - n / 2.0) * h->d;
                const double tx = x / dk + (m - 1) / 2.0, ty = y / dk + (m - 1) / 2.0;
                const int ix = std::min(std::max((int)std::floor(tx), 0), m - 2);
                const int iy = std::min(std::max((int)std::floor(ty), 0), m - 2);
                const double fx = tx - ix, fy = ty - iy;
                const size_t o = ((size_t)k * h->n_vphi + v) * 4;
                idx[o + 0] = iy * m + ix;             w[o + 0] = (float)((1 - fx) * (1 - fy));
                idx[o + 1] = iy * m + ix + 1;         w[o + 1] = (float)(fx * (1 - fy));
                idx[o + 2] = (iy + 1) * m + ix;       w[o + 2] = (float)((1 - fx) * fy);
                idx[o + 3] = (iy + 1) * m + ix + 1;   w[o + 3] = (float)(fx * fy);
            }
        }
        TRY(dalloc(h, &h->d_iidx, idx.size()));
        TRY(dalloc(h, &h->d_iw, w.size()));
        TRY(upload(h, idx.data(), h->d_iidx, sizeof(int) * idx.size()));
        TRY(upload(h, w.data(), h->d_iw, sizeof(float) * w.size()));
        // transposed table for the adjoint: per layer and grid node, the
        // (phase point, weight) pairs that read it, in phase-point order
        const int m2 = m * m;
        std::vector<int> aptr((size_t)L_ * (m2 + 1), 0), avi(idx.size());
        std::vector<float> aw(idx.size());
        size_t off = 0;
        for (int k = 0; k < L_; ++k) {
            std::vector<int> cnt(m2 + 1, 0);
            for (int v = 0; v < h->n_vphi; ++v)
                for (int c = 0; c < 4; ++c) ++cnt[idx[((size_t)k * h->n_vphi + v) * 4 + c] + 1];
            int* pk = aptr.data() + (size_t)k * (m2 + 1);
            pk[0] = (int)off;
            for (int i = 0; i < m2; ++i) pk[i + 1] = pk[i] + cnt[i + 1];
            std::vector<int> fill(pk, pk + m2);
            for (int v = 0; v < h->n_vphi; ++v)
                for (int c = 0; c < 4; ++c) {
                    const size_t o = ((size_t)k * h->n_vphi + v) * 4 + c;
                    const int e = fill[idx[o]]++;
                    avi[e] = v;
                    aw[e] = w[o];
                }
            off = pk[m2];
        }
        TRY(dalloc(h, &h->d_aptr, aptr.size()));
        TRY(dalloc(h, &h->d_avi, avi.size()));
        TRY(dalloc(h, &h->d_aw, aw.size()));
        TRY(upload(h, aptr.data(), h->d_aptr, sizeof(int) * aptr.size()));
        TRY(upload(h, avi.data(), h->d_avi, sizeof(int) * avi.size()));
        TRY(upload(h, aw.data(), h->d_aw, sizeof(float) * aw.size()));
        // mask tables of the full m x m grid (input of the adjoint's row pass)
        std::vector<int> rs(m + 1), cl((size_t)m2), rc((size_t)m2);
        for (int i = 0; i <= m; ++i) rs[i] = i * m;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) { cl[(size_t)i * m + j] = j; rc[(size_t)i * m + j] = (i << 16) | j; }
        TRY(dalloc(h, &h->d_rowstart_m, m + 1));
        TRY(dalloc(h, &h->d_col_m, m2));
        TRY(dalloc(h, &h->d_rowcol_m, m2));
        TRY(upload(h, rs.data(), h->d_rowstart_m, sizeof(int) * (m + 1)));
        TRY(upload(h, cl.data(), h->d_col_m, sizeof(int) * m2));
        TRY(upload(h, rc.data(), h->d_rowcol_m, sizeof(int) * m2));
        h->mt_m = MaskTables{h->d_rowstart_m, h->d_col_m, h->d_rowcol_m, m2};
        h->g_adj = MvmGeom{m, n, h->cos_layers, h->NP, h->Pc / 2 + 1, h->planc};
    }

    // --- workspaces --------------------------------------------------------------
    const size_t B = h->max_batch;
    const size_t nh = h->P / 2 + 1, nhc = h->Pc / 2 + 1;
    TRY(dalloc(h, &h->X1, B * h->NP * nh * n));
    TRY(dalloc(h, &h->Y1, B * h->NP * nh * n));
    TRY(dalloc(h, &h->X1d, B * h->NP * nh * n));
    TRY(dalloc(h, &h->Y1d, B * h->NP * nh * n));
    TRY(dalloc(h, &h->Xc, B * h->NP * nhc * n));
    TRY(dalloc(h, &h->Yc, B * h->cos_layers * nhc * h->m));
    TRY(dalloc(h, &h->Ydc, B * h->cos_layers * h->m * h->m));
    TRY(dalloc(h, &h->x, B * h->N));
    TRY(dalloc(h, &h->r, B * h->N));
    TRY(dalloc(h, &h->p, B * h->N));
    TRY(dalloc(h, &h->Ap, B * h->N));
    TRY(dalloc(h, &h->xd, B * h->N));
    TRY(dalloc(h, &h->yd, B * h->N));
    TRY(dalloc(h, &h->st, B));
    h->nparts = std::max(1, std::min(64, (h->N + 4095) / 4096));
    TRY(dalloc(h, &h->dot_part, B * h->NP * h->rg * 3));
    TRY(dalloc(h, &h->dot_part_M, B * h->NP * h->rg * 3));
    TRY(dalloc(h, &h->z, B * h->N));
    TRY(dalloc(h, &h->w, B * h->N));
    TRY(dalloc(h, &h->rr_part, B * h->NP * h->rg));
    TRY(dalloc(h, &h->res_part, B * h->nparts));
    TRY(dalloc(h, &h->init_part, B * 2 * h->nparts));
    TRY(dalloc(h, &h->d_nactive, 1));
    TRY(dalloc(h, &h->s_stage, B * h->N));
    TRY(dalloc(h, &h->z_stage, B * h->N));
    TRY(dalloc(h, &h->phi_stage, B * h->n_targets * h->n_vphi));
    TRY(dalloc(h, &h->d_fscale, B));
    if (h->modes) TRY(dalloc(h, &h->s_proj, B * h->N));
    TRY(dalloc(h, &h->d_fscale_pre, B));
    CK(cudaMallocHost(&h->h_nactive, sizeof(int)));
    CK(cudaStreamSynchronize(h->stream));
    return TOMO_OK;
}

void release(tomo_handle* h) {
    if (!h) return;
    if (h->graph.exec) cudaGraphExecDestroy(h->graph.exec);
    if (h->loop.exec) cudaGraphExecDestroy(h->loop.exec);
    if (h->h_loop) cudaFreeHost(h->h_loop);
    if (h->work) cudaStreamSynchronize(h->work);
    for (void* p : h->allocs) cudaFree(p);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->work) cudaStreamDestroy(h->work);
    if (h->h_nactive) cudaFreeHost(h->h_nactive);
    if (h->h_small) cudaFreeHost(h->h_small);
    delete h;
}

// Conjugate-transposed projection spectra and workspaces of the adjoint, on
// first use.
tomo_status adjoint_init(tomo_handle* h) {
    if (h->adj_ready) return TOMO_OK;
    Launch L = launch_of(h);
    const size_t nhc = h->Pc / 2 + 1;
    const size_t kstride = (size_t)h->cos_layers * h->NP * nhc * h->Pc;
    const size_t B = h->max_batch;
    TRY(dalloc(h, &h->d_Kadj, kstride * h->n_targets));
    for (int t = 0; t < h->n_targets; ++t)
        CK(adjoint_spectra(L, (int)nhc, h->Pc, h->NP, h->cos_layers, h->d_Kc32 + t * kstride, h->d_Kadj + t * kstride));
    TRY(dalloc(h, &h->Xa, B * h->cos_layers * nhc * h->m));
    TRY(dalloc(h, &h->Ya, B * h->NP * nhc * h->n));
    TRY(dalloc(h, &h->Yda, B * h->cos_layers * h->m * h->m));
    TRY(dalloc(h, &h->za, B * h->N));
    CK(cudaStreamSynchronize(h->stream));
    h->adj_ready = true;
    return TOMO_OK;
}

// zeta = sum_{t in [t0, t1)} W_s Sigma_s_phi_t W_phi^T phi[:, t] (the adjoint of
// apply_os restricted to those targets), B <= max_batch frames.
tomo_status apply_os_adjoint(tomo_handle* h, const Launch& L, const float* phi, float* zeta, int B, int t0, int t1) {
    TRY(adjoint_init(h));
    const size_t nhc = h->Pc / 2 + 1;
    const size_t kstride = (size_t)h->cos_layers * h->NP * nhc * h->Pc;
    for (int t = t0; t < t1; ++t) {
        float* out = t == t0 ? zeta : h->za;
        CK(interp_adjoint(L, B, h->n_targets, t, h->cos_layers, h->m, h->n_vphi, h->d_aptr, h->d_avi, h->d_aw, phi,
                          h->Yda));
        CK((rows_fwd<float, float>(L, h->g_adj, h->mt_m, B, h->Yda, nullptr, nullptr, h->Xa, h->d_twc32)));
        CK((cols_mul<float>(L, h->g_adj, B, nullptr, h->Xa, h->Ya, h->d_Kadj + t * kstride, h->d_twc32, false)));
        CK((rows_inv_masked<float, float>(L, h->g_adj, h->mt, B, nullptr, h->Ya, nullptr, h->d_noise_var, nullptr,
                                          out, nullptr, h->d_twc32)));
        if (t != t0) CK(axpy_f32(L, (size_t)B * h->N, 1.f, h->za, zeta));
    }
    return TOMO_OK;
}

// y = W_s F^{-1} M(f) F W_s^T x (the block-circulant preconditioner), FP32
tomo_status apply_pre(tomo_handle* h, const Launch& L, const float* x, float* y, int B) {
    CK((rows_fwd<float, float>(L, h->g_ss, h->mt, B, x, nullptr, nullptr, h->X1, h->d_tw32)));
    CK((cols_mul<float>(L, h->g_ss, B, nullptr, h->X1, h->Y1, h->d_M32, h->d_tw32, true)));
    CK((rows_inv_masked<float, float>(L, h->g_ss, h->mt, B, nullptr, h->Y1, x, h->d_zero_var, nullptr, y,
                                      nullptr, h->d_tw32)));
    return TOMO_OK;
}

// --- warm-start network -------------------------------------------------------
tomo_status ws_layouts(tomo_handle* h, const Launch& L) {
    WarmStartNet& w = h->ws;
    if (!w.dirty) return TOMO_OK;
    for (int l = 0; l < w.layers; ++l)
        CK(weight_layouts(L, w.ch[l], w.ch[l + 1], w.params + w.offW[l], w.Wt[l], w.Wb[l]));
    w.dirty = false;
    return TOMO_OK;
}

// act[4] = network(slopes), zeta = gather(act[4]) * out_scale
tomo_status ws_forward(tomo_handle* h, const Launch& L, const float* s, int B, float* zeta) {
    WarmStartNet& w = h->ws;
    TRY(ws_layouts(h, L));
    CK(cnn_scatter(L, B, h->NP, h->n, h->n_vs, h->mt.rowcol, s, w.in_scale, w.act[0], w.ch[0]));
    if (w.hybrid) {
        TRY(apply_pre(h, L, s, w.zpre, B));
        // channels NP..2NP-1 of the input grid: M^{-1} s * in_scale / out_scale
        CK(cnn_scatter_planes(L, B, h->NP, 2 * h->NP, h->NP, h->n, h->n_vs, h->mt.rowcol, w.zpre,
                              w.pre_scale, w.act[0]));
    }
    for (int l = 0; l < w.layers; ++l)
        CK(conv_fwd(L, B, w.ch[l], w.ch[l + 1], h->n, w.act[l], w.Wt[l], w.params + w.offb[l], w.act[l + 1],
                    l + 1 < w.layers));
    if (zeta) {
        CK(cnn_gather(L, B, h->NP, h->n, h->n_vs, h->mt.rowcol, w.act[w.layers], w.out_scale, zeta));
        if (w.hybrid) CK(axpy_f32(L, (size_t)B * h->N, w.pre_gain, w.zpre, zeta));
    }
    return TOMO_OK;
}

// parameter gradient of loss(zeta) for dloss/dzeta = gz (valid entries), after ws_forward
tomo_status ws_backward(tomo_handle* h, const Launch& L, int B) {
    WarmStartNet& w = h->ws;
    const size_t plane = (size_t)h->n * h->n;
    CK(cnn_scatter(L, B, h->NP, h->n, h->n_vs, h->mt.rowcol, w.gz, w.out_scale, w.d0, h->NP));
    float* dy = w.d0;
    float* dx = w.d1;
    for (int l = w.layers - 1; l >= 0; --l) {
        if (l + 1 < w.layers) CK(relu_bwd(L, (size_t)B * w.ch[l + 1] * plane, w.act[l + 1], dy));
        CK(conv_wgrad(L, B, w.ch[l], w.ch[l + 1], h->n, w.act[l], dy, w.wpart, w.grad + w.offW[l]));
        if (l > 0) {
            CK(conv_fwd(L, B, w.ch[l + 1], w.ch[l], h->n, dy, w.Wb[l], w.zero_bias, dx, false));
            std::swap(dx, dy);
        }
    }
    return TOMO_OK;
}

// --- small dense FP64 algebra of block CG (B <= 64, row-major) -----------------
// Cholesky L L^T = A of a symmetric positive semi-definite A.  A pivot below
// rel_drop times its diagonal entry marks the column as dependent on the
// previous ones: it is dropped (flag set, row and column of L zero, L_jj = 1).
void chol_drop(const std::vector<double>& A, int B, double rel_drop, std::vector<double>& L,
               std::vector<char>& drop) {
    L.assign((size_t)B * B, 0.0);
    drop.assign(B, 0);
    for (int j = 0; j < B; ++j) {
        double d = A[(size_t)j * B + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * B + k] * L[(size_t)j * B + k];
        if (!(d > rel_drop * A[(size_t)j * B + j]) || !(A[(size_t)j * B + j] > 0) || !std::isfinite(d)) {
            drop[j] = 1;
            L[(size_t)j * B + j] = 1.0;
            continue;
        }
        const double ljj = std::sqrt(d);
        L[(size_t)j * B + j] = ljj;
        for (int i = j + 1; i < B; ++i) {
            double v = A[(size_t)i * B + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * B + k] * L[(size_t)j * B + k];
            L[(size_t)i * B + j] = v / ljj;
        }
    }
}

// y -= a x over n contiguous entries (vectorised).
inline void row_axpy(double* __restrict__ y, const double* __restrict__ x, double a, int n) {
    for (int c = 0; c < n; ++c) y[c] -= a * x[c];
}

// T = L^{-T} (upper triangular) with the dropped rows and columns of T zero,
// so that W T has orthonormal columns (Cholesky QR) and zero columns where W
// was dependent.  L^{-1} by row-oriented forward substitution on the identity.
void chol_inv_t(const std::vector<double>& L, const std::vector<char>& drop, int B, std::vector<double>& T) {
    std::vector<double> Li((size_t)B * B, 0.0);
    double* Ld = Li.data();
    for (int i = 0; i < B; ++i) {
        double* li = Ld + (size_t)i * B;
        li[i] = 1.0;
        for (int k = 0; k < i; ++k) row_axpy(li, Ld + (size_t)k * B, L[(size_t)i * B + k], i);
        const double inv = 1.0 / L[(size_t)i * B + i];
        for (int c = 0; c <= i; ++c) li[c] *= inv;
    }
    T.assign((size_t)B * B, 0.0);
    for (int j = 0; j < B; ++j) {
        if (drop[j]) continue;
        const double* lj = Ld + (size_t)j * B;
        for (int i = 0; i <= j; ++i) T[(size_t)i * B + j] = drop[i] ? 0.0 : lj[i];
    }
}

// Per-frame operator scales of the next B frames on the work stream:
// A_f = c_f Sigma_ss + nu_f Sigma_eta_eta (c, nu host arrays; null = all 1),
// and the preconditioner scale 1 / c_f.
tomo_status set_fscale(tomo_handle* h, int B, const double* c, const double* nu) {
    if (!c && !nu) {
        if (h->fscale_unit) return TOMO_OK;
        B = h->max_batch;
    }
    std::vector<double2> fs(B), fp(B);
    for (int f = 0; f < B; ++f) {
        const double cf = c ? c[f] : 1.0, nf = nu ? nu[f] : 1.0;
        fs[f] = make_double2(cf, nf);
        fp[f] = make_double2(1.0 / cf, 0.0);
    }
    CK(cudaMemcpyAsync(h->d_fscale, fs.data(), sizeof(double2) * B, cudaMemcpyHostToDevice, h->work));
    CK(cudaMemcpyAsync(h->d_fscale_pre, fp.data(), sizeof(double2) * B, cudaMemcpyHostToDevice, h->work));
    CK(cudaStreamSynchronize(h->work));
    h->fscale_unit = !c && !nu;
    return TOMO_OK;
}

// The host loop of the single-vector methods: graphs of check_every
// iterations, with a convergence check between them; when no frame is active
// the FP64 true residual (true_res) decides which frames restart.  Stops the
// frames still active when max_iter iterations are spent or the call's
// deadline has passed (TOMO_FRAME_MAXIT).
template <typename TrueRes>
tomo_status run_iterations(tomo_handle* h, const Launch& L, int B, const tomo_solve_opts& o, int kind,
                           TrueRes&& true_res) {
    const int chunk = std::max(1, o.check_every);
    if (!h->timing) TRY(build_graph(h, B, chunk, kind));
    long long total_iters = 0;
    std::vector<std::pair<int, int>> marks;
    for (;;) {
        CK(count_active(L, B, h->st, h->d_nactive));
        CK(cudaMemcpyAsync(h->h_nactive, h->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, h->work));
        CK(cudaStreamSynchronize(h->work));
        if (h->timing) collect_timing(h, marks);
        if (*h->h_nactive == 0) {
            // FP64 true residual s - A zeta and restart of the frames above tol
            TRY(true_res(o.max_refine));
            CK(count_active(L, B, h->st, h->d_nactive));
            CK(cudaMemcpyAsync(h->h_nactive, h->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, h->work));
            CK(cudaStreamSynchronize(h->work));
            if (*h->h_nactive == 0) break;
        }
        if (total_iters >= (long long)o.max_iter || past_deadline(h)) {
            // iteration budget or time spent: stop the remaining frames
            std::vector<FrameState> tmp(B);
            CK(cudaMemcpyAsync(tmp.data(), h->st, sizeof(FrameState) * B, cudaMemcpyDeviceToHost, h->work));
            CK(cudaStreamSynchronize(h->work));
            for (auto& f : tmp)
                if (f.active) { f.active = 0; f.status = TOMO_FRAME_MAXIT; }
            CK(cudaMemcpyAsync(h->st, tmp.data(), sizeof(FrameState) * B, cudaMemcpyHostToDevice, h->work));
            CK(cudaStreamSynchronize(h->work));
            TRY(true_res(0));
            break;
        }
        if (h->timing) {
            for (int i = 0; i < chunk; ++i) TRY(iteration(h, L, B, kind, &marks));
        } else {
            CK(cudaGraphLaunch(h->graph.exec, h->work));
            h->launches += h->graph.nodes;
        }
        total_iters += chunk;
    }
    return TOMO_OK;
}

// The FP64 true residual of the device loop (inside its IF node): reads the
// right-hand side from the handle's buffer (s_loop, or s64 for FP64 CG) and
// tol / max_refine from the loop state.
tomo_status true_res_device(tomo_handle* h, const Launch& L, int B, int kind) {
    const int ms_len = 2 * h->n_vs;
    if (kind == kIterCG64) {
        if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, 1, h->d_Qs, nullptr, h->x64, nullptr, nullptr));
        TRY(apply_ss64(h, L, h->x64, h->yd, B, h->d_fscale));
        if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, 1, h->d_Qs, nullptr, h->yd, nullptr, nullptr));
        CK(residual64(L, B, h->N, h->nparts, h->s64, h->yd, h->r64, h->res_part));
    } else {
        CK(to_f64(L, (size_t)B * h->N, h->x, h->xd));
        if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, h->rg, h->d_Qs, nullptr, h->xd, nullptr, nullptr));
        TRY(apply_ss64(h, L, h->xd, h->yd, B, h->d_fscale));
        if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, h->rg, h->d_Qs, nullptr, h->yd, nullptr, nullptr));
        CK(true_residual(L, B, h->N, h->nparts, h->s_loop, h->yd, h->r, h->res_part));
    }
    CK(true_residual_finalize(L, B, h->nparts, h->res_part, 0.0, 0, h->st, h->d_loop));
    return TOMO_OK;
}

// Builds (or reuses) the device-loop graph: WHILE (more) { chunk iterations;
// loop_check, which sets `need`; IF (need) { FP64 true residual }; loop_next,
// which sets `more` }.  The body is captured from the same launch code as the
// host loop; the IF node is spliced in through the capture's dependencies.
tomo_status build_loop_graph(tomo_handle* h, int B, int chunk, int kind) {
    LoopGraph& lg = h->loop;
    if (lg.exec && lg.B == B && lg.chunk == chunk && lg.kind == kind) return TOMO_OK;
    if (lg.exec) {
        cudaGraphExecDestroy(lg.exec);
        lg.exec = nullptr;
    }
    const long long before = h->launches;
    Launch Lc{h->work, &h->launches};
    cudaGraph_t g = nullptr;
    tomo_status st = TOMO_OK;
    bool capturing = false;
    auto bad = [&](cudaError_t e, const char* what) {
        std::fprintf(stderr, "tomo: device loop graph: %s failed: %s\n", what, cudaGetErrorString(e));
        st = TOMO_ECUDA;
    };
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) { bad(e, "cudaGraphCreate"); return st; }
    cudaGraphConditionalHandle more{}, need{};
    cudaGraphNodeParams wp{};
    cudaGraphNodeParams ip{};
    cudaGraphNode_t wnode = nullptr, inode = nullptr;
    long long body_nodes = 0, if_nodes = 0;
    do {
        if ((e = cudaGraphConditionalHandleCreate(&more, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) {
            bad(e, "cudaGraphConditionalHandleCreate");
            break;
        }
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = more;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        if ((e = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp)) != cudaSuccess) {
            bad(e, "cudaGraphAddNode (while)");
            break;
        }
        cudaGraph_t body = wp.conditional.phGraph_out[0];
        if ((e = cudaGraphConditionalHandleCreate(&need, body, 0, 0)) != cudaSuccess) {
            bad(e, "cudaGraphConditionalHandleCreate");
            break;
        }
        if ((e = cudaStreamBeginCaptureToGraph(h->work, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess) {
            bad(e, "cudaStreamBeginCaptureToGraph (body)");
            break;
        }
        capturing = true;
        const long long b0 = h->launches;
        for (int i = 0; i < chunk && st == TOMO_OK; ++i) st = iteration(h, Lc, B, kind, nullptr);
        if (st != TOMO_OK) break;
        if ((e = loop_check(Lc, B, h->st, h->d_loop, need)) != cudaSuccess) { bad(e, "loop_check"); break; }
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        if ((e = cudaStreamGetCaptureInfo(h->work, &cs, nullptr, nullptr, &deps, nullptr, &nd)) != cudaSuccess) {
            bad(e, "cudaStreamGetCaptureInfo");
            break;
        }
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = need;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        if ((e = cudaGraphAddNode(&inode, body, deps, nullptr, nd, &ip)) != cudaSuccess) {
            bad(e, "cudaGraphAddNode (if)");
            break;
        }
        if ((e = cudaStreamUpdateCaptureDependencies(h->work, &inode, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
            cudaSuccess) {
            bad(e, "cudaStreamUpdateCaptureDependencies");
            break;
        }
        if ((e = loop_next(Lc, B, h->st, h->d_loop, more)) != cudaSuccess) { bad(e, "loop_next"); break; }
        body_nodes = h->launches - b0;
        cudaGraph_t out = nullptr;
        capturing = false;
        if ((e = cudaStreamEndCapture(h->work, &out)) != cudaSuccess) { bad(e, "cudaStreamEndCapture (body)"); break; }
        cudaGraph_t ibody = ip.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(h->work, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess) {
            bad(e, "cudaStreamBeginCaptureToGraph (if)");
            break;
        }
        capturing = true;
        const long long i0 = h->launches;
        st = true_res_device(h, Lc, B, kind);
        if_nodes = h->launches - i0;
        capturing = false;
        if ((e = cudaStreamEndCapture(h->work, &out)) != cudaSuccess) { bad(e, "cudaStreamEndCapture (if)"); break; }
        if (st != TOMO_OK) break;
        if ((e = cudaGraphInstantiate(&lg.exec, g, 0)) != cudaSuccess) { bad(e, "cudaGraphInstantiate"); break; }
    } while (false);
    if (capturing) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(h->work, &junk);
        if (junk && junk != g) cudaGraphDestroy(junk);
        cudaGetLastError();
    }
    cudaGraphDestroy(g);
    h->launches = before;
    if (st != TOMO_OK || !lg.exec) {
        lg.exec = nullptr;
        return st == TOMO_OK ? TOMO_ECUDA : st;
    }
    lg.B = B;
    lg.chunk = chunk;
    lg.kind = kind;
    lg.body_nodes = body_nodes;
    lg.if_nodes = if_nodes;
    return TOMO_OK;
}

// The solve loop as one graph launch on the work stream (no host
// synchronisation); s: the right-hand side the true residual uses (copied to
// the handle's buffer; unused for FP64 CG, whose right-hand side is s64).
tomo_status run_device_loop(tomo_handle* h, const Launch& L, int B, const tomo_solve_opts& o, int kind,
                            const float* s) {
    if (!h->d_loop) {
        TRY(dalloc(h, &h->d_loop, 1));
        TRY(dalloc(h, &h->s_loop, (size_t)h->max_batch * h->N));
        CK(cudaMallocHost(&h->h_loop, sizeof(LoopState)));
    }
    const int chunk = std::max(1, o.check_every);
    if (kind != kIterCG64) CK(cudaMemcpyAsync(h->s_loop, s, sizeof(float) * B * h->N, cudaMemcpyDeviceToDevice, h->work));
    unsigned long long budget = 0;
    if (h->has_deadline) {
        const double ns =
            std::chrono::duration<double, std::nano>(h->deadline - std::chrono::steady_clock::now()).count();
        budget = (unsigned long long)std::max(1.0, ns);
    }
    TRY(build_loop_graph(h, B, chunk, kind));
    CK(loop_start(L, h->d_loop, o.max_iter, budget, o.tol, o.max_refine, chunk));
    CK(cudaGraphLaunch(h->loop.exec, h->work));
    CK(cudaMemcpyAsync(h->h_loop, h->d_loop, sizeof(LoopState), cudaMemcpyDeviceToHost, h->work));
    h->loop_pending = true;
    return TOMO_OK;
}

// After the work stream has been synchronised: the device loop's outcome
// (time budget, launch count: body passes and true residuals).
void account_loop(tomo_handle* h) {
    if (!h->loop_pending) return;
    h->loop_pending = false;
    const LoopState& ls = *h->h_loop;
    if (ls.timed_out) h->timed_out = true;
    const long long passes = ls.chunk > 0 ? ls.iters / ls.chunk : 0;
    h->launches += passes * h->loop.body_nodes + (long long)ls.true_res_runs * h->loop.if_nodes;
}

tomo_status solve_chunk(tomo_handle* h, const float* s, int B, const tomo_solve_opts& o, float* zeta, float* phase,
                        tomo_frame_info* info, const double* c_scale = nullptr, const double* nu_scale = nullptr,
                        const double* prop_c = nullptr) {
    // the solve runs on the private stream, ordered after the caller's stream
    // and before anything the caller enqueues next
    Launch L{h->work, &h->launches};
    TRY(set_fscale(h, B, c_scale, nu_scale));
    CK(cudaEventRecord(h->ev_in, h->stream));
    CK(cudaStreamWaitEvent(h->work, h->ev_in, 0));
    const int ms_len = 2 * h->n_vs;
    if (prop_c) {
        // proportional operators A_f = c_f A~ (the caller passes the common
        // A~ as c = 1, nu = kappa): solve A~ zeta~_f = s_f (same relative
        // residual), then zeta_f = zeta~_f / c_f and phi_f = c_f Cos zeta_f = Cos zeta~_f
        if (!h->d_rhs_scale) TRY(dalloc(h, &h->d_rhs_scale, h->max_batch));
        std::vector<double> inv(B);
        for (int f = 0; f < B; ++f) inv[f] = 1.0 / prop_c[f];
        CK(cudaMemcpyAsync(h->d_rhs_scale, inv.data(), sizeof(double) * B, cudaMemcpyHostToDevice, h->work));
        CK(cudaStreamSynchronize(h->work));
    }
    if (h->modes) {
        // right-hand side M_s s
        CK(cudaMemcpyAsync(h->s_proj, s, sizeof(float) * B * h->N, cudaMemcpyDeviceToDevice, h->work));
        CK(mode_project<float>(L, B, ms_len, h->n_gs, h->rg, h->d_Qs, nullptr, h->s_proj, nullptr, nullptr));
        s = h->s_proj;
    }
    // A x0 for a warm start x0 (projected first under mode removal)
    auto start_from_x = [&]() -> tomo_status {
        if (h->modes) CK(mode_project<float>(L, B, ms_len, h->n_gs, h->rg, h->d_Qs, nullptr, h->x, nullptr, nullptr));
        TRY(apply_ss32(h, L, h->x, h->Ap, B, nullptr, nullptr, h->d_fscale));
        if (h->modes) CK(mode_project<float>(L, B, ms_len, h->n_gs, h->rg, h->d_Qs, nullptr, h->Ap, nullptr, nullptr));
        CK(cg_init(L, B, h->N, h->nparts, s, h->Ap, h->x, h->r, h->p, h->Ap, h->init_part));
        return TOMO_OK;
    };
    // FP64 true residual r = s - A x (M_s s - M_s A M_s x under mode removal)
    auto true_res = [&](int max_refine) -> tomo_status {
        CK(to_f64(L, (size_t)B * h->N, h->x, h->xd));
        if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, h->rg, h->d_Qs, nullptr, h->xd, nullptr, nullptr));
        TRY(apply_ss64(h, L, h->xd, h->yd, B, h->d_fscale));
        if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, h->rg, h->d_Qs, nullptr, h->yd, nullptr, nullptr));
        CK(true_residual(L, B, h->N, h->nparts, s, h->yd, h->r, h->res_part));
        CK(true_residual_finalize(L, B, h->nparts, h->res_part, o.tol, max_refine, h->st));
        return TOMO_OK;
    };
    // the handle's x buffer holds zeta during the solve
    if (o.warm_start == 2) {
        if (!h->ws.ready) return TOMO_EINVAL;
        for (int b0 = 0; b0 < B; b0 += h->ws.maxB) {
            const int nb = std::min(h->ws.maxB, B - b0);
            TRY(ws_forward(h, L, s + (size_t)b0 * h->N, nb, h->x + (size_t)b0 * h->N));
        }
        TRY(start_from_x());
    } else if (o.warm_start) {
        CK(cudaMemcpyAsync(h->x, zeta, sizeof(float) * B * h->N, cudaMemcpyDeviceToDevice, h->work));
        TRY(start_from_x());
    } else {
        CK(cg_init(L, B, h->N, h->nparts, s, nullptr, h->x, h->r, h->p, h->Ap, h->init_part));
    }
    CK(cg_init_scalars(L, B, h->nparts, h->init_part, o.tol, o.warm_start, h->st));
    const bool pcg = o.precond && h->d_M32;
    const int kind = o.method == TOMO_METHOD_MINRES ? kIterMINRES
                     : o.precond == 2                ? kIterFlex
                     : (pcg ? kIterPCG : kIterCG);
    if (kind == kIterFlex) {
        // the learned preconditioner needs the network in its [r, M r] form and
        // M itself; it is not rescaled per frame (no tomo_solve_r0) nor projected
        if (!h->ws.ready || !h->ws.hybrid || !h->d_M32 || h->modes || c_scale || nu_scale) return TOMO_EINVAL;
        if (!h->flex_part) TRY(dalloc(h, &h->flex_part, (size_t)h->max_batch * h->nparts * 5));
        TRY(ws_layouts(h, L));     // the network's weight layouts, before any graph captures their use
    }
    if (kind != kIterCG) {
        // the first row-forward pass reads these with zero coefficients
        CK(cudaMemsetAsync(h->z, 0, sizeof(float) * B * h->N, h->work));
        CK(cudaMemsetAsync(h->w, 0, sizeof(float) * B * h->N, h->work));
    }
    long long block_iters = -1;
    if (o.method == TOMO_METHOD_BLOCK) {
        // Block (preconditioned) conjugate gradients over the B frames
        // (O'Leary): one Krylov space for all frames, the search block P kept
        // orthonormal in storage by Cholesky QR (numerically dependent
        // columns dropped).  Forming P explicitly keeps FP32 storage
        // well conditioned: folding the QR factor into the coefficients
        // instead measured 142 against 112 block iterations at ELT scale.
        if (!h->d_small) {
            TRY(dalloc(h, &h->d_small, 9 * 64 * 64));
            TRY(dalloc(h, &h->d_gram_part, gram_workspace(h->N)));
            CK(cudaMallocHost(&h->h_small, sizeof(double) * 9 * 64 * 64));
        }
        // small FP64 matrices, device and pinned host at the same offsets:
        // [G] [norms] [H] [E] [T_G] [T_W] [Gw] [alpha / beta]
        constexpr size_t kS = 4096;
        constexpr int kNormSlices = 16;
        double* dG = h->d_small;
        double* dRR = dG + kS;                           // [B][16] partial norms, right after G
        double* dH = dG + 2 * kS;
        double* dE = dG + 3 * kS;
        double* dTG = dG + 4 * kS;
        double* dTW = dG + 5 * kS;
        double* dGw = dG + 6 * kS;
        double* dAB = dG + 7 * kS;                       // alpha, then beta
        double* hs = h->h_small;
        const size_t BB = (size_t)B * B;
        std::vector<double> G(BB), Gw(BB), C, LG, LW, tol2(B);
        std::vector<char> dropG, dropW;
        auto d2h = [&](const double* d, size_t n) -> tomo_status {
            CK(cudaMemcpyAsync(hs + (d - h->d_small), d, sizeof(double) * n, cudaMemcpyDeviceToHost, h->work));
            return TOMO_OK;
        };
        auto h2d = [&](double* d, size_t n) -> tomo_status {
            CK(cudaMemcpyAsync(d, hs + (d - h->d_small), sizeof(double) * n, cudaMemcpyHostToDevice, h->work));
            return TOMO_OK;
        };
        auto hv = [&](const double* d) { return hs + (d - h->d_small); };
        auto apply_A = [&](const float* in, float* out) -> tomo_status {
            TRY(apply_ss32(h, L, in, out, B, nullptr, nullptr, h->d_fscale));
            if (h->modes) CK(mode_project<float>(L, B, ms_len, h->n_gs, h->rg, h->d_Qs, nullptr, out, nullptr, nullptr));
            return TOMO_OK;
        };
        auto apply_M = [&](const float* in, float* out) -> tomo_status {
            TRY(apply_pre(h, L, in, out, B));
            if (h->modes) CK(mode_project<float>(L, B, ms_len, h->n_gs, h->rg, h->d_Qs, nullptr, out, nullptr, nullptr));
            return TOMO_OK;
        };
        // T = L^{-T} of the Cholesky factor of the Gram matrix at d (host), to dT
        auto factor = [&](const double* dGram, std::vector<double>& Gh, double rel_drop, std::vector<double>& Lf,
                          std::vector<char>& drop, double* dT) -> tomo_status {
            std::copy(hv(dGram), hv(dGram) + BB, Gh.begin());
            chol_drop(Gh, B, rel_drop, Lf, drop);
            chol_inv_t(Lf, drop, B, C);
            std::copy(C.begin(), C.end(), hv(dT));
            TRY(h2d(dT, BB));
            return TOMO_OK;
        };
        // frames reported as breakdowns at the start (non-finite slopes or
        // warm start) take no part: their residual columns are zeroed, so the
        // Gram products drop them as dependent, and their result is the
        // initial guess
        std::vector<char> broken(B, 0);
        {
            std::vector<FrameState> tmp(B);
            CK(cudaMemcpyAsync(tmp.data(), h->st, sizeof(FrameState) * B, cudaMemcpyDeviceToHost, h->work));
            CK(cudaStreamSynchronize(h->work));
            for (int f = 0; f < B; ++f) {
                tol2[f] = tmp[f].tol2;
                broken[f] = tmp[f].status == TOMO_FRAME_BREAKDOWN;
            }
        }
        CK(zero_broken(L, B, h->N, h->st, h->r));
        block_iters = 0;
        bool done = false;
        while (!done) {
            // (re)start from the residual in r: W = M r (or r), P = W T_W
            const float* W = h->r;
            if (pcg) { TRY(apply_M(h->r, h->z)); W = h->z; }
            CK(gram(L, B, h->N, W, W, dGw, h->d_gram_part));
            TRY(d2h(dGw, BB));
            CK(cudaStreamSynchronize(h->work));
            TRY(factor(dGw, Gw, 1e-6, LW, dropW, dTW));
            bool converged = false;
            bool have_norms = false;
            while (!converged) {
                if (block_iters >= (long long)o.max_iter || past_deadline(h)) break;
                // P = W T_W (orthonormal columns), A P, and the Gram products with P
                CK(block_combine(L, B, h->N, dTW, W, nullptr, h->p));
                TRY(apply_A(h->p, h->Ap));
                CK(gram(L, B, h->N, h->p, h->Ap, dG, h->d_gram_part));
                CK(gram(L, B, h->N, h->p, h->r, dH, h->d_gram_part));
                // G and the residual norms of the previous update in one copy
                TRY(d2h(dG, kS + (size_t)B * kNormSlices));
                CK(cudaStreamSynchronize(h->work));
                if (have_norms) {
                    const double* rrs = hv(dRR);
                    converged = true;
                    for (int f = 0; f < B; ++f) {
                        if (broken[f]) continue;
                        double t = 0.0;
                        for (int q = 0; q < kNormSlices; ++q) t += rrs[(size_t)f * kNormSlices + q];
                        converged = converged && t <= tol2[f];
                    }
                    if (converged) break;
                }
                TRY(factor(dG, G, 1e-13, LG, dropG, dTG));
                // alpha = G^+ P^T r = T_G T_G^T H on the device; x += P alpha, r -= A P alpha
                CK(gram_apply(L, B, dTG, dH, dAB, 1.0));
                CK(block_combine(L, B, h->N, dAB, h->p, h->x, h->x));
                CK(block_combine(L, B, h->N, dAB, h->Ap, h->r, h->r, -1.0));
                ++block_iters;
                CK(row_norms(L, B, h->N, h->r, dRR, kNormSlices));
                have_norms = true;
                const float* Z = h->r;
                if (pcg) { TRY(apply_M(h->r, h->z)); Z = h->z; }
                // beta = -G^+ (A P)^T z; next W = z + P beta
                CK(gram(L, B, h->N, h->Ap, Z, dE, h->d_gram_part));
                CK(gram_apply(L, B, dTG, dE, dAB, -1.0));
                CK(block_combine(L, B, h->N, dAB, h->p, Z, h->w));
                W = h->w;
                CK(gram(L, B, h->N, W, W, dGw, h->d_gram_part));
                TRY(d2h(dGw, BB));
                CK(cudaStreamSynchronize(h->work));
                TRY(factor(dGw, Gw, 1e-6, LW, dropW, dTW));
            }
            if (!converged) {
                // iteration budget spent
                std::vector<FrameState> tmp(B);
                CK(cudaMemcpyAsync(tmp.data(), h->st, sizeof(FrameState) * B, cudaMemcpyDeviceToHost, h->work));
                CK(cudaStreamSynchronize(h->work));
                for (auto& f : tmp) f.active = 0;
                CK(cudaMemcpyAsync(h->st, tmp.data(), sizeof(FrameState) * B, cudaMemcpyHostToDevice, h->work));
                TRY(true_res(0));
                std::vector<FrameState> t2(B);
                CK(cudaMemcpyAsync(t2.data(), h->st, sizeof(FrameState) * B, cudaMemcpyDeviceToHost, h->work));
                CK(cudaStreamSynchronize(h->work));
                for (auto& f : t2)
                    if (f.relres > o.tol) f.status = TOMO_FRAME_MAXIT;
                CK(cudaMemcpyAsync(h->st, t2.data(), sizeof(FrameState) * B, cudaMemcpyHostToDevice, h->work));
                break;
            }
            // FP64 true residual; frames above tol restart the whole block
            std::vector<FrameState> tmp(B);
            CK(cudaMemcpyAsync(tmp.data(), h->st, sizeof(FrameState) * B, cudaMemcpyDeviceToHost, h->work));
            CK(cudaStreamSynchronize(h->work));
            for (auto& f : tmp) {
                f.active = 0;
                if (f.status != TOMO_FRAME_BREAKDOWN) f.status = 0;
            }
            CK(cudaMemcpyAsync(h->st, tmp.data(), sizeof(FrameState) * B, cudaMemcpyHostToDevice, h->work));
            TRY(true_res(o.max_refine));
            // a restart must not carry a non-finite residual column into the block
            CK(zero_broken(L, B, h->N, h->st, h->r));
            CK(count_active(L, B, h->st, h->d_nactive));
            CK(cudaMemcpyAsync(h->h_nactive, h->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, h->work));
            CK(cudaStreamSynchronize(h->work));
            done = *h->h_nactive == 0;
        }
    }
    if (block_iters < 0) {
        if (!o.host_loop && !h->timing) TRY(run_device_loop(h, L, B, o, kind, s));
        else TRY(run_iterations(h, L, B, o, kind, true_res));
    }
    if (h->modes) CK(mode_project<float>(L, B, ms_len, h->n_gs, h->rg, h->d_Qs, nullptr, h->x, nullptr, nullptr));
    if (prop_c) CK(scale_rows(L, B, h->N, h->d_rhs_scale, h->x, zeta));
    else CK(cudaMemcpyAsync(zeta, h->x, sizeof(float) * B * h->N, cudaMemcpyDeviceToDevice, h->work));
    if (phase) {
        TRY(apply_os(h, L, h->x, phase, B, h->d_fscale));
        if (h->modes)
            CK(mode_project<float>(L, B, h->n_vphi, h->n_targets, 1, h->d_Qp, nullptr, phase, nullptr, nullptr));
    }
    CK(cudaEventRecord(h->ev_out, h->work));
    CK(cudaStreamWaitEvent(h->stream, h->ev_out, 0));
    if (info) {
        std::vector<FrameState> tmp(B);
        CK(cudaMemcpyAsync(tmp.data(), h->st, sizeof(FrameState) * B, cudaMemcpyDeviceToHost, h->work));
        CK(cudaStreamSynchronize(h->work));
        account_loop(h);
        TRY(check_wait_error());
        for (int f = 0; f < B; ++f) {
            if (block_iters >= 0) tmp[f].iters = (int)block_iters;
            h->frame_iters += tmp[f].iters;
            info[f].iters = tmp[f].iters;
            info[f].refinements = tmp[f].refinements;
            info[f].status = (kind == kIterFlex && tmp[f].fb && tmp[f].status == TOMO_FRAME_CONVERGED)
                                 ? TOMO_FRAME_FALLBACK_PLAIN_CG
                                 : tmp[f].status;
            info[f].pad_ = 0;
            info[f].relres = tmp[f].relres;
        }
    }
    return TOMO_OK;
}

// Per-frame results of a solve into info_host (host array) from the FrameState.
tomo_status report(tomo_handle* h, int B, tomo_frame_info* info) {
    if (!info) return TOMO_OK;
    std::vector<FrameState> tmp(B);
    CK(cudaMemcpyAsync(tmp.data(), h->st, sizeof(FrameState) * B, cudaMemcpyDeviceToHost, h->work));
    CK(cudaStreamSynchronize(h->work));
    account_loop(h);
    TRY(check_wait_error());
    for (int f = 0; f < B; ++f) {
        h->frame_iters += tmp[f].iters;
        info[f].iters = tmp[f].iters;
        info[f].refinements = tmp[f].refinements;
        info[f].status = tmp[f].status;
        info[f].pad_ = 0;
        info[f].relres = tmp[f].relres;
    }
    return TOMO_OK;
}

// FP64 conjugate gradients (Sec. 2.G) on B <= max_batch frames: FP64 slopes
// s64 and solution zeta64 (device), the FP64 product of Eq. mvm_ss, FP64
// vectors and scalars, the FP64 true residual at exit with restarts from it.
tomo_status solve_chunk_f64(tomo_handle* h, const double* s64, int B, const tomo_solve_opts& o, double* zeta64,
                            tomo_frame_info* info, const double* c_scale = nullptr, const double* nu_scale = nullptr) {
    Launch L{h->work, &h->launches};
    TRY(ensure_f64(h));
    TRY(set_fscale(h, B, c_scale, nu_scale));
    CK(cudaEventRecord(h->ev_in, h->stream));
    CK(cudaStreamWaitEvent(h->work, h->ev_in, 0));
    const int ms_len = 2 * h->n_vs;
    const size_t BN = (size_t)B * h->N;
    // right-hand side (M_s s under mode removal) in the handle's own buffer
    CK(cudaMemcpyAsync(h->s64, s64, sizeof(double) * BN, cudaMemcpyDeviceToDevice, h->work));
    if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, 1, h->d_Qs, nullptr, h->s64, nullptr, nullptr));
    if (o.warm_start) {
        CK(cudaMemcpyAsync(h->x64, zeta64, sizeof(double) * BN, cudaMemcpyDeviceToDevice, h->work));
        if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, 1, h->d_Qs, nullptr, h->x64, nullptr, nullptr));
        TRY(apply_ss64(h, L, h->x64, h->Ap64, B, h->d_fscale));
        if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, 1, h->d_Qs, nullptr, h->Ap64, nullptr, nullptr));
        CK(cg64_init(L, B, h->N, h->nparts, h->s64, h->Ap64, h->x64, h->r64, h->p64, h->Ap64, h->init_part));
    } else {
        CK(cg64_init(L, B, h->N, h->nparts, h->s64, nullptr, h->x64, h->r64, h->p64, h->Ap64, h->init_part));
    }
    CK(cg_init_scalars(L, B, h->nparts, h->init_part, o.tol, o.warm_start, h->st));
    // FP64 true residual r = s - A x (the iterate is kept in range(M_s) under mode removal)
    auto true_res = [&](int max_refine) -> tomo_status {
        if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, 1, h->d_Qs, nullptr, h->x64, nullptr, nullptr));
        TRY(apply_ss64(h, L, h->x64, h->yd, B, h->d_fscale));
        if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, 1, h->d_Qs, nullptr, h->yd, nullptr, nullptr));
        CK(residual64(L, B, h->N, h->nparts, h->s64, h->yd, h->r64, h->res_part));
        CK(true_residual_finalize(L, B, h->nparts, h->res_part, o.tol, max_refine, h->st));
        return TOMO_OK;
    };
    if (!o.host_loop && !h->timing) TRY(run_device_loop(h, L, B, o, kIterCG64, nullptr));
    else TRY(run_iterations(h, L, B, o, kIterCG64, true_res));
    CK(cudaMemcpyAsync(zeta64, h->x64, sizeof(double) * BN, cudaMemcpyDeviceToDevice, h->work));
    CK(cudaEventRecord(h->ev_out, h->work));
    CK(cudaStreamWaitEvent(h->stream, h->ev_out, 0));
    return report(h, B, info);
}

// Mixed-precision iterative refinement (tomo_solve_opts.precision =
// TOMO_PREC_MIXED): zeta accumulated in FP64; each pass forms the FP64 true
// residual r = s - A zeta with the FP64 operator and solves A d = r with the
// FP32 solver of solve_chunk (any method) to a relative tolerance tau, then
// zeta += d in FP64.  tau = o.inner_tol, or automatically the factor still
// missing to tol (0.5 tol / max relres), at least 2e-5 (the floor FP32
// storage sets) and at most 0.5.  Frames that meet tol get a zero right-hand
// side in later passes (the inner solve then leaves them alone).  Slopes s32
// (FP32) or s64 (FP64), one of them; output zeta32 or zeta64 (one of them),
// phase as solve_chunk.  c_scale / nu_scale / prop_c as
// solve_chunk; the outer operator of frame f is A_f = c_f pc_f Sigma_ss +
// nu_f pc_f Sigma_eta_eta with pc_f = prop_c[f] (1 when null).
tomo_status solve_chunk_mixed(tomo_handle* h, const float* s32, const double* s64, int B, const tomo_solve_opts& o,
                              float* zeta32, double* zeta64, float* phase, tomo_frame_info* info,
                              const double* c_scale = nullptr, const double* nu_scale = nullptr,
                              const double* prop_c = nullptr) {
    Launch L{h->work, &h->launches};
    TRY(ensure_f64(h));
    const int ms_len = 2 * h->n_vs;
    const size_t BN = (size_t)B * h->N;
    {
        std::vector<double2> fs(B);
        for (int f = 0; f < B; ++f) {
            const double pc = prop_c ? prop_c[f] : 1.0;
            fs[f] = make_double2((c_scale ? c_scale[f] : 1.0) * pc, (nu_scale ? nu_scale[f] : 1.0) * pc);
        }
        CK(cudaMemcpyAsync(h->d_fs_outer, fs.data(), sizeof(double2) * B, cudaMemcpyHostToDevice, h->work));
        CK(cudaStreamSynchronize(h->work));
    }
    CK(cudaEventRecord(h->ev_in, h->stream));
    CK(cudaStreamWaitEvent(h->work, h->ev_in, 0));
    if (s64) CK(cudaMemcpyAsync(h->s64, s64, sizeof(double) * BN, cudaMemcpyDeviceToDevice, h->work));
    else CK(to_f64(L, BN, s32, h->s64));
    if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, 1, h->d_Qs, nullptr, h->s64, nullptr, nullptr));
    CK(norm2_64(L, B, h->N, h->nparts, h->s64, h->res_part, h->snorm64));
    // initial guess
    if (o.warm_start == 1) {
        if (zeta64) CK(cudaMemcpyAsync(h->x64, zeta64, sizeof(double) * BN, cudaMemcpyDeviceToDevice, h->work));
        else CK(to_f64(L, BN, zeta32, h->x64));
    } else if (o.warm_start == 2) {
        if (!h->ws.ready) return TOMO_EINVAL;
        CK(f64_to_f32(L, B, h->N, nullptr, h->s64, h->rhs32));
        for (int b0 = 0; b0 < B; b0 += h->ws.maxB) {
            const int nb = std::min(h->ws.maxB, B - b0);
            TRY(ws_forward(h, L, h->rhs32 + (size_t)b0 * h->N, nb, h->d32 + (size_t)b0 * h->N));
        }
        CK(to_f64(L, BN, h->d32, h->x64));
    } else {
        CK(cudaMemsetAsync(h->x64, 0, sizeof(double) * BN, h->work));
    }
    // the inner solves run under the call's deadline (h->deadline), which solve_chunk checks
    tomo_solve_opts in = o;
    in.precision = TOMO_PREC_FP32;
    in.warm_start = 0;
    std::vector<double> rel(B, 0.0);
    std::vector<int> iters(B, 0), status(B, TOMO_FRAME_MAXIT), passes(B, 0);
    std::vector<tomo_frame_info> inner(B);
    long long used = 0;
    for (int pass = 0;; ++pass) {
        // FP64 true residual of the current zeta
        if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, 1, h->d_Qs, nullptr, h->x64, nullptr, nullptr));
        TRY(apply_ss64(h, L, h->x64, h->yd, B, h->d_fs_outer));
        if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, 1, h->d_Qs, nullptr, h->yd, nullptr, nullptr));
        CK(residual64(L, B, h->N, h->nparts, h->s64, h->yd, h->r64, h->res_part));
        CK(relres64(L, B, h->nparts, h->res_part, h->snorm64, h->rel64));
        CK(cudaMemcpyAsync(rel.data(), h->rel64, sizeof(double) * B, cudaMemcpyDeviceToHost, h->work));
        CK(cudaStreamSynchronize(h->work));
        double worst = 0.0;
        int left = 0;
        for (int f = 0; f < B; ++f) {
            if (status[f] == TOMO_FRAME_BREAKDOWN) continue;
            if (!std::isfinite(rel[f])) { status[f] = TOMO_FRAME_BREAKDOWN; continue; }
            if (rel[f] <= o.tol) { status[f] = TOMO_FRAME_CONVERGED; continue; }
            status[f] = TOMO_FRAME_MAXIT;
            ++left;
            worst = std::max(worst, rel[f]);
        }
        if (left == 0 || pass > o.max_refine || used >= o.max_iter || past_deadline(h)) break;
        // the next correction: frames above tol only (broken and converged frames get zeros)
        for (int f = 0; f < B; ++f)
            if (status[f] != TOMO_FRAME_MAXIT) rel[f] = 0.0;
        CK(cudaMemcpyAsync(h->rel64, rel.data(), sizeof(double) * B, cudaMemcpyHostToDevice, h->work));
        CK(inner_rhs(L, B, h->N, h->rel64, o.tol, h->r64, h->rhs32));
        in.tol = o.inner_tol > 0 ? o.inner_tol : std::min(0.5, std::max(2e-5, 0.5 * o.tol / worst));
        in.max_iter = (int)std::max<long long>(1, o.max_iter - used);
        TRY(solve_chunk(h, h->rhs32, B, in, h->d32, nullptr, inner.data(), c_scale, nu_scale, prop_c));
        int most = 0;
        for (int f = 0; f < B; ++f) {
            if (status[f] != TOMO_FRAME_MAXIT) continue;
            iters[f] += inner[f].iters;
            passes[f] += 1;
            most = std::max(most, inner[f].iters);
            if (inner[f].status == TOMO_FRAME_BREAKDOWN) status[f] = TOMO_FRAME_BREAKDOWN;
        }
        used += most;
        CK(add_f32_to_f64(L, BN, h->d32, h->x64));
    }
    if (h->modes) CK(mode_project<double>(L, B, ms_len, h->n_gs, 1, h->d_Qs, nullptr, h->x64, nullptr, nullptr));
    if (zeta64) CK(cudaMemcpyAsync(zeta64, h->x64, sizeof(double) * BN, cudaMemcpyDeviceToDevice, h->work));
    float* z32 = zeta32 ? zeta32 : h->rhs32;
    if (zeta32 || phase) CK(f64_to_f32(L, B, h->N, nullptr, h->x64, z32));
    if (phase) {
        TRY(apply_os(h, L, z32, phase, B, h->d_fs_outer));
        if (h->modes)
            CK(mode_project<float>(L, B, h->n_vphi, h->n_targets, 1, h->d_Qp, nullptr, phase, nullptr, nullptr));
    }
    CK(cudaEventRecord(h->ev_out, h->work));
    CK(cudaStreamWaitEvent(h->stream, h->ev_out, 0));
    CK(cudaStreamSynchronize(h->work));
    if (info) {
        for (int f = 0; f < B; ++f) {
            info[f].iters = iters[f];
            info[f].refinements = std::max(0, passes[f] - 1);
            info[f].status = status[f];
            info[f].pad_ = 0;
            info[f].relres = rel[f];
        }
    }
    return TOMO_OK;
}

tomo_status check_opts(const tomo_solve_opts& o, int max_batch = 0) {
    if (!(o.tol > 0) || o.max_iter < 1 || o.max_refine < 0 || o.check_every < 1) return TOMO_EINVAL;
    if (o.precision != TOMO_PREC_FP32 && o.precision != TOMO_PREC_FP64 && o.precision != TOMO_PREC_MIXED)
        return TOMO_EINVAL;
    if (!(o.inner_tol >= 0) || !(o.inner_tol < 1) || !(o.deadline_ms >= 0)) return TOMO_EINVAL;
    if (o.host_loop != 0 && o.host_loop != 1) return TOMO_EINVAL;
    if (o.method != TOMO_METHOD_CG && o.method != TOMO_METHOD_MINRES && o.method != TOMO_METHOD_BLOCK)
        return TOMO_EINVAL;
    if (o.method == TOMO_METHOD_MINRES && o.precond) return TOMO_EINVAL;
    if (o.precond < 0 || o.precond > 2 || (o.precond == 2 && o.method != TOMO_METHOD_CG)) return TOMO_EINVAL;
    if (o.warm_start < 0 || o.warm_start > 2) return TOMO_EINVAL;
    if (o.method == TOMO_METHOD_BLOCK && max_batch > 64) return TOMO_EINVAL;
    return TOMO_OK;
}

tomo_solve_opts default_opts() {
    tomo_solve_opts o;
    o.tol = 1e-4;
    o.max_iter = 10000;
    o.max_refine = 2;
    o.warm_start = 0;
    o.check_every = 32;
    o.precond = 0;
    o.method = TOMO_METHOD_CG;
    o.precision = TOMO_PREC_FP32;
    o.inner_tol = 0.0;
    o.deadline_ms = 0.0;
    o.host_loop = 0;
    return o;
}

// tomo_solve's work, without the per-call set-up (deadline) and status.
tomo_status solve_impl(tomo_handle* h, const float* slopes, int batch, const tomo_solve_opts& o, float* zeta,
                       float* phase, tomo_frame_info* info) {
    for (int f0 = 0; f0 < batch; f0 += h->max_batch) {
        const int B = std::min(h->max_batch, batch - f0);
        const float* sb = slopes + (size_t)f0 * h->N;
        float* zb = zeta + (size_t)f0 * h->N;
        float* pb = phase ? phase + (size_t)f0 * h->n_targets * h->n_vphi : nullptr;
        tomo_frame_info* ib = info ? info + f0 : nullptr;
        if (o.precision == TOMO_PREC_MIXED) TRY(solve_chunk_mixed(h, sb, nullptr, B, o, zb, nullptr, pb, ib));
        else TRY(solve_chunk(h, sb, B, o, zb, pb, ib));
    }
    return TOMO_OK;
}

tomo_status end_call(tomo_handle* h, tomo_status s) {
    const bool late = h->timed_out;
    h->has_deadline = false;
    h->timed_out = false;
    return s == TOMO_OK && late ? TOMO_ETIMEOUT : s;
}

// ---------------------------------------------------------------------------
// Allocation-free Sigma_ss product (tomo_apply_css_noalloc).
// ---------------------------------------------------------------------------
// Room for the two half-spectrum intermediates of the product (the row-pass
// output and the column-pass output, NP * (P/2+1) * n complex floats each per
// frame).  It is a static device array: every GPU that loads this library
// holds these 16 MiB until the process exits, and every call of the entry
// point shares them.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
constexpr int kMaxGridY = 65535;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Host code may not use g_noalloc_scratch as a device address (on the host it
// is only a stand-in symbol); the device address is looked up once per device
// with that device current.  The address is kept for the life of the process:
// a cudaDeviceReset unloads the library's device code (and frees every
// handle's memory, so no handle survives it either), after which this entry
// point must not be called on that device again.
constexpr int kNoAllocMaxDevices = 64;
struct NoAllocDevice {
    std::once_flag once;
    void* ptr = nullptr;
    cudaError_t err = cudaSuccess;
};
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];

tomo_status noalloc_scratch(void** out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        std::fprintf(stderr, "tomo_apply_css_noalloc: device %d beyond the %d supported\n", dev, kNoAllocMaxDevices);
        return TOMO_ERANGE;
    }
    NoAllocDevice& d = g_noalloc_dev[dev];
    std::call_once(d.once, [&d] { d.err = cudaGetSymbolAddress(&d.ptr, g_noalloc_scratch); });
    if (d.err != cudaSuccess || d.ptr == nullptr) {
        std::fprintf(stderr, "tomo_apply_css_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(d.err));
        return TOMO_ECUDA;
    }
    *out = d.ptr;
    return TOMO_OK;
}

}  // namespace

extern "C" {

tomo_status tomo_apply_css_noalloc(tomo_handle* h, const float* x, float* y, int batch) {
    if (!h || !x || !y || batch < 0 || x == y) return TOMO_EINVAL;
    const size_t half = (size_t)h->NP * (h->P / 2 + 1) * h->n * sizeof(float2);
    const size_t per_frame = 2 * half;
    if (per_frame > kNoAllocScratchBytes) {
        std::fprintf(stderr,
                     "tomo_apply_css_noalloc: one frame needs %zu bytes of scratch, more than the %zu bytes of the "
                     "static buffer (use tomo_apply_css)\n",
                     per_frame, kNoAllocScratchBytes);
        return TOMO_ERANGE;
    }
    void* scratch = nullptr;
    TRY(noalloc_scratch(&scratch));
    // frames per chunk: as many as the buffer holds, at most kMaxGridY (every
    // pass puts the frames of a launch on gridDim.y, which is limited to 65535)
    const int chunk = (int)std::min<size_t>(kNoAllocScratchBytes / per_frame, (size_t)kMaxGridY);
    float2* X1 = static_cast<float2*>(scratch);
    float2* Y1 = X1 + (size_t)chunk * (half / sizeof(float2));
    Launch L = launch_of(h);
    for (int f0 = 0; f0 < batch; f0 += chunk) {
        const int B = std::min(chunk, batch - f0);
        const float* xb = x + (size_t)f0 * h->N;
        float* yb = y + (size_t)f0 * h->N;
        CK((rows_fwd<float, float>(L, h->g_ss, h->mt, B, xb, nullptr, nullptr, X1, h->d_tw32)));
        CK((cols_mul<float>(L, h->g_ss, B, nullptr, X1, Y1, h->d_K32, h->d_tw32, true)));
        CK((rows_inv_masked<float, float>(L, h->g_ss, h->mt, B, nullptr, Y1, xb, h->d_rows_noise, nullptr, yb,
                                          nullptr, h->d_tw32)));
        if (h->d_ncov)
            CK(noise_blocks<float>(L, B, h->n_vs, h->n_gs, 1, h->d_ncov, nullptr, nullptr, yb, xb, nullptr, nullptr));
    }
    return TOMO_OK;
}


tomo_status tomo_create(const tomo_config* cfg, void* cuda_stream, tomo_handle** out) {
    if (!out) return TOMO_EINVAL;
    *out = nullptr;
    tomo_status s = validate(cfg);
    if (s != TOMO_OK) return s;
    tomo_handle* h = new (std::nothrow) tomo_handle();
    if (!h) return TOMO_ENOMEM;
    s = create_impl(cfg, cuda_stream, h);
    if (s != TOMO_OK) {
        cudaStreamSynchronize(h->stream);
        release(h);
        return s;
    }
    *out = h;
    return TOMO_OK;
}

tomo_status tomo_autotune_result(const tomo_handle* h, int* sides, double* ms, int capacity, int* count) {
    if (!h || !count || capacity < 0) return TOMO_EINVAL;
    *count = (int)h->tune_P.size();
    for (int i = 0; i < *count && i < capacity; ++i) {
        if (sides) sides[i] = h->tune_P[i];
        if (ms) ms[i] = i < (int)h->tune_ms.size() ? h->tune_ms[i] : -1.0;
    }
    return TOMO_OK;
}

tomo_status tomo_layout(const tomo_handle* h, tomo_layout_info* info, uint8_t* subap_mask, uint8_t* phase_mask) {
    if (!h || !info) return TOMO_EINVAL;
    info->n = h->n;
    info->n_gs = h->n_gs;
    info->n_vs = h->n_vs;
    info->N = h->N;
    info->n_vphi = h->n_vphi;
    info->n_targets = h->n_targets;
    info->n_layers = h->n_layers;
    info->P = h->P;
    info->Pcos = h->Pc;
    info->n_new = h->m;
    info->max_batch = h->max_batch;
    if (subap_mask) std::memcpy(subap_mask, h->subap_mask.data(), h->subap_mask.size());
    if (phase_mask) std::memcpy(phase_mask, h->phase_mask.data(), h->phase_mask.size());
    return TOMO_OK;
}

tomo_status tomo_apply_css(tomo_handle* h, const float* x, float* y, int batch) {
    if (!h || !x || !y || batch < 0 || x == y) return TOMO_EINVAL;
    Launch L = launch_of(h);
    for (int f0 = 0; f0 < batch; f0 += h->max_batch) {
        const int B = std::min(h->max_batch, batch - f0);
        TRY(apply_ss32(h, L, x + (size_t)f0 * h->N, y + (size_t)f0 * h->N, B, nullptr, nullptr));
    }
    return TOMO_OK;
}

tomo_status tomo_apply_css_f64(tomo_handle* h, const double* x, double* y, int batch) {
    if (!h || !x || !y || batch < 0 || x == y) return TOMO_EINVAL;
    Launch L = launch_of(h);
    for (int f0 = 0; f0 < batch; f0 += h->max_batch) {
        const int B = std::min(h->max_batch, batch - f0);
        TRY(apply_ss64(h, L, x + (size_t)f0 * h->N, y + (size_t)f0 * h->N, B));
    }
    return TOMO_OK;
}

tomo_status tomo_apply_cos(tomo_handle* h, const float* z, float* phi, int batch) {
    if (!h || !z || !phi || batch < 0) return TOMO_EINVAL;
    Launch L = launch_of(h);
    for (int f0 = 0; f0 < batch; f0 += h->max_batch) {
        const int B = std::min(h->max_batch, batch - f0);
        TRY(apply_os(h, L, z + (size_t)f0 * h->N, phi + (size_t)f0 * h->n_targets * h->n_vphi, B));
    }
    return TOMO_OK;
}

tomo_status tomo_apply_cos_adjoint(tomo_handle* h, const float* phi, float* z, int batch) {
    if (!h || !phi || !z || batch < 0) return TOMO_EINVAL;
    Launch L = launch_of(h);
    for (int f0 = 0; f0 < batch; f0 += h->max_batch) {
        const int B = std::min(h->max_batch, batch - f0);
        TRY(apply_os_adjoint(h, L, phi + (size_t)f0 * h->n_targets * h->n_vphi, z + (size_t)f0 * h->N, B, 0,
                             h->n_targets));
    }
    return TOMO_OK;
}

tomo_status tomo_reconstructor(tomo_handle* h, int target, const tomo_solve_opts* opts, float* R,
                               tomo_frame_info* info, double* wfe) {
    if (!h || (!R && !wfe) || target < 0 || target >= h->n_targets) return TOMO_EINVAL;
    tomo_solve_opts o = opts ? *opts : default_opts();
    TRY(check_opts(o, h->max_batch));
    if (o.warm_start) return TOMO_EINVAL;
    if (h->modes || o.precision != TOMO_PREC_FP32) return TOMO_EINVAL;
    begin_call(h, o);
    Launch L = launch_of(h);
    const int nv = h->n_vphi;
    double *dots = nullptr, *sums = nullptr;
    if (wfe) {
        TRY(dalloc(h, &dots, nv));
        TRY(dalloc(h, &sums, 2 * (size_t)h->N));
        CK(cudaMemsetAsync(sums, 0, sizeof(double) * 2 * h->N, h->stream));
    }
    tomo_status st = TOMO_OK;
    for (int v0 = 0; v0 < nv && st == TOMO_OK; v0 += h->max_batch) {
        const int B = std::min(h->max_batch, nv - v0);
        float* rows = R ? R + (size_t)v0 * h->N : h->z_stage;
        // right-hand sides W_s Sigma_s_phi W_phi^T e_v: columns of R^T's system
        CK(unit_phase(L, B, h->n_targets, target, nv, v0, h->phi_stage));
        st = apply_os_adjoint(h, L, h->phi_stage, h->s_stage, B, target, target + 1);
        if (st == TOMO_OK) st = solve_chunk(h, h->s_stage, B, o, rows, nullptr, info ? info + v0 : nullptr);
        if (st == TOMO_OK && wfe) CK(wfe_accumulate(L, B, h->N, h->s_stage, rows, dots + v0, sums, sums + h->N));
    }
    if (st == TOMO_OK && wfe) {
        // Eq. analytical1 for R = F A^{-1} (F = W_phi Sigma_phi_s W_s^T): the error
        // covariance is Sigma_phi_phi - F A^{-1} F^T; piston removed (P = I - 1 1^T / n):
        //   trace(P F A^{-1} F^T P) = sum_v F_v . R_v - (sum_v F_v) . (sum_v R_v) / n
        //   trace(P S P) = n B(0) - sum_{u,v} B(|x_u - x_v|) / n
        std::vector<double> hd(nv), hs(2 * (size_t)h->N);
        CK(cudaMemcpyAsync(hd.data(), dots, sizeof(double) * nv, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(hs.data(), sums, sizeof(double) * 2 * h->N, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        double t2 = 0.0, cross = 0.0;
        for (int v = 0; v < nv; ++v) t2 += hd[v];
        for (int j = 0; j < h->N; ++j) cross += hs[j] * hs[(size_t)h->N + j];
        t2 -= cross / nv;
        // the target (at infinity) sees each layer through the pupil shifted by
        // h_k beta, so Sigma_phi_phi depends only on x_u - x_v: one von Karman
        // covariance with amplitude c_v (L0/r0)^{5/3} sum_k f_k, over the lags of
        // the phase-point lattice weighted by how often each occurs
        const int n = h->n, W = 2 * n + 1;
        std::vector<long long> cnt((size_t)W * W, 0);
        for (int u = 0; u < nv; ++u)
            for (int v = 0; v < nv; ++v)
                ++cnt[(size_t)(h->ph_i[u] - h->ph_i[v] + n) * W + (h->ph_j[u] - h->ph_j[v] + n)];
        const double cv = std::pow(24.0 / 5.0 * std::tgamma(6.0 / 5.0), 5.0 / 6.0) * std::tgamma(11.0 / 6.0) *
                          std::tgamma(5.0 / 6.0) / (2.0 * std::pow(kPi, 8.0 / 3.0));
        const double B0 = cv * std::pow(h->L0 / h->r0, 5.0 / 3.0) * h->frac_sum;
        const double norm = std::pow(2.0, 1.0 / 6.0) / std::tgamma(5.0 / 6.0);
        double pair_sum = 0.0;
        for (int di = -n; di <= n; ++di)
            for (int dj = -n; dj <= n; ++dj) {
                const long long c = cnt[(size_t)(di + n) * W + (dj + n)];
                if (!c) continue;
                const double rho = std::hypot((double)di, (double)dj) * h->d;
                const double x = 2.0 * kPi * rho / h->L0;
                const double b = rho == 0.0 ? B0 : B0 * norm * std::pow(x, 5.0 / 6.0) * std::cyl_bessel_k(5.0 / 6.0, x);
                pair_sum += (double)c * b;
            }
        const double t1 = nv * B0 - pair_sum / nv;
        wfe[1] = t1 / nv;
        wfe[2] = t2 / nv;
        wfe[0] = std::sqrt(std::max(0.0, (t1 - t2) / nv));
    }
    if (dots || sums) {
        cudaStreamSynchronize(h->stream);
        for (void* p : {(void*)dots, (void*)sums}) {
            if (!p) continue;
            cudaFree(p);
            h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), p), h->allocs.end());
        }
    }
    return end_call(h, st);
}

tomo_status tomo_apply_reconstructor(tomo_handle* h, const float* R, int rows, const float* slopes, int batch,
                                     float* phase) {
    if (!h || !R || !slopes || !phase || rows < 1 || batch < 0) return TOMO_EINVAL;
    if (batch == 0) return TOMO_OK;
    Launch L = launch_of(h);
    // enough K-splits that the grid covers the GPU several times, each split >= 256 columns
    const long long tiles = (long long)((rows + 63) / 64) * ((batch + 63) / 64);
    int splits = (int)std::min<long long>(32, std::max<long long>(1, (4LL * h->block_slots / 3 + tiles - 1) / tiles));
    splits = std::max(1, std::min(splits, h->N / 256));
    const size_t need = gemm_nt_workspace(batch, rows, splits);
    if (need > h->gemm_part_size) {
        if (h->gemm_part) {
            CK(cudaStreamSynchronize(h->stream));
            cudaFree(h->gemm_part);
            h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), (void*)h->gemm_part), h->allocs.end());
            h->gemm_part = nullptr;
        }
        TRY(dalloc(h, &h->gemm_part, need));
        h->gemm_part_size = need;
    }
    CK(gemm_nt(L, batch, rows, h->N, slopes, h->N, R, h->N, phase, rows, splits, h->gemm_part));
    return TOMO_OK;
}

tomo_status tomo_solve(tomo_handle* h, const float* slopes, int batch, const tomo_solve_opts* opts, float* zeta,
                       float* phase, tomo_frame_info* info) {
    if (!h || !slopes || !zeta || batch < 0) return TOMO_EINVAL;
    tomo_solve_opts o = opts ? *opts : default_opts();
    TRY(check_opts(o, h->max_batch));
    if (o.precision == TOMO_PREC_FP64) return TOMO_EINVAL;     // FP64 buffers: tomo_solve_f64
    begin_call(h, o);
    return end_call(h, solve_impl(h, slopes, batch, o, zeta, phase, info));
}

tomo_status tomo_solve_f64(tomo_handle* h, const double* slopes, int batch, const tomo_solve_opts* opts,
                           double* zeta, tomo_frame_info* info) {
    if (!h || !slopes || !zeta || batch < 0) return TOMO_EINVAL;
    tomo_solve_opts o = opts ? *opts : default_opts();
    if (!opts) o.precision = TOMO_PREC_FP64;
    TRY(check_opts(o, h->max_batch));
    if (o.precision == TOMO_PREC_FP32 || o.warm_start == 2) return TOMO_EINVAL;
    if (o.precision == TOMO_PREC_FP64 && (o.method != TOMO_METHOD_CG || o.precond)) return TOMO_EINVAL;
    begin_call(h, o);
    tomo_status st = TOMO_OK;
    for (int f0 = 0; f0 < batch && st == TOMO_OK; f0 += h->max_batch) {
        const int B = std::min(h->max_batch, batch - f0);
        const double* sb = slopes + (size_t)f0 * h->N;
        double* zb = zeta + (size_t)f0 * h->N;
        tomo_frame_info* ib = info ? info + f0 : nullptr;
        st = o.precision == TOMO_PREC_FP64 ? solve_chunk_f64(h, sb, B, o, zb, ib)
                                           : solve_chunk_mixed(h, nullptr, sb, B, o, nullptr, zb, nullptr, ib);
    }
    return end_call(h, st);
}

tomo_status solve_r0_impl(tomo_handle* h, const float* slopes, int batch, const double* r0, const double* noise_scale,
                          const tomo_solve_opts& o, float* zeta, float* phase, tomo_frame_info* info);

tomo_status tomo_solve_r0(tomo_handle* h, const float* slopes, int batch, const double* r0, const double* noise_scale,
                          const tomo_solve_opts* opts, float* zeta, float* phase, tomo_frame_info* info) {
    if (!h || !slopes || !zeta || !r0 || batch < 0) return TOMO_EINVAL;
    tomo_solve_opts o = opts ? *opts : default_opts();
    TRY(check_opts(o, h->max_batch));
    if (o.precision == TOMO_PREC_FP64) return TOMO_EINVAL;
    begin_call(h, o);
    return end_call(h, solve_r0_impl(h, slopes, batch, r0, noise_scale, o, zeta, phase, info));
}

tomo_status solve_r0_impl(tomo_handle* h, const float* slopes, int batch, const double* r0, const double* noise_scale,
                          const tomo_solve_opts& o, float* zeta, float* phase, tomo_frame_info* info) {
    const bool mixed = o.precision == TOMO_PREC_MIXED;
    // von Karman covariances scale as r0^{-5/3} (B(0) = c_v (L0 / r0)^{5/3})
    std::vector<double> c(batch);
    for (int f = 0; f < batch; ++f) {
        if (!(r0[f] > 0) || !std::isfinite(r0[f])) return TOMO_EINVAL;
        if (noise_scale && !(noise_scale[f] >= 0 && std::isfinite(noise_scale[f]))) return TOMO_EINVAL;
        c[f] = std::pow(r0[f] / h->r0, -5.0 / 3.0);
    }
    if (o.method == TOMO_METHOD_BLOCK) {
        // one Krylov space needs one operator up to a factor per frame:
        // A_f = c_f (Sigma_ss + kappa Sigma_eta_eta) with kappa = nu_f / c_f common
        const double kappa = (noise_scale ? noise_scale[0] : 1.0) / c[0];
        for (int f = 0; f < batch; ++f) {
            const double kf = (noise_scale ? noise_scale[f] : 1.0) / c[f];
            if (!(std::fabs(kf - kappa) <= 1e-9 * std::max(kappa, 1e-300))) return TOMO_EINVAL;
        }
        std::vector<double> one((size_t)h->max_batch, 1.0), kap((size_t)h->max_batch, kappa);
        for (int f0 = 0; f0 < batch; f0 += h->max_batch) {
            const int B = std::min(h->max_batch, batch - f0);
            const float* sb = slopes + (size_t)f0 * h->N;
            float* zb = zeta + (size_t)f0 * h->N;
            float* pb = phase ? phase + (size_t)f0 * h->n_targets * h->n_vphi : nullptr;
            tomo_frame_info* ib = info ? info + f0 : nullptr;
            if (mixed) TRY(solve_chunk_mixed(h, sb, nullptr, B, o, zb, nullptr, pb, ib, one.data(), kap.data(),
                                             c.data() + f0));
            else TRY(solve_chunk(h, sb, B, o, zb, pb, ib, one.data(), kap.data(), c.data() + f0));
        }
        return TOMO_OK;
    }
    for (int f0 = 0; f0 < batch; f0 += h->max_batch) {
        const int B = std::min(h->max_batch, batch - f0);
        const float* sb = slopes + (size_t)f0 * h->N;
        float* zb = zeta + (size_t)f0 * h->N;
        float* pb = phase ? phase + (size_t)f0 * h->n_targets * h->n_vphi : nullptr;
        tomo_frame_info* ib = info ? info + f0 : nullptr;
        const double* nb = noise_scale ? noise_scale + f0 : nullptr;
        if (mixed) TRY(solve_chunk_mixed(h, sb, nullptr, B, o, zb, nullptr, pb, ib, c.data() + f0, nb));
        else TRY(solve_chunk(h, sb, B, o, zb, pb, ib, c.data() + f0, nb));
    }
    return TOMO_OK;
}

tomo_status tomo_solve_host(tomo_handle* h, const float* slopes, int batch, const tomo_solve_opts* opts, float* zeta,
                            float* phase, tomo_frame_info* info) {
    if (!h || !slopes || !zeta || batch < 0) return TOMO_EINVAL;
    tomo_solve_opts o = opts ? *opts : default_opts();
    TRY(check_opts(o, h->max_batch));
    if (o.precision == TOMO_PREC_FP64) return TOMO_EINVAL;
    begin_call(h, o);
    tomo_status st = TOMO_OK;
    const size_t nphi = (size_t)h->n_targets * h->n_vphi;
    for (int f0 = 0; f0 < batch; f0 += h->max_batch) {
        const int B = std::min(h->max_batch, batch - f0);
        CK(cudaMemcpyAsync(h->s_stage, slopes + (size_t)f0 * h->N, sizeof(float) * B * h->N, cudaMemcpyHostToDevice,
                           h->stream));
        if (o.warm_start)
            CK(cudaMemcpyAsync(h->z_stage, zeta + (size_t)f0 * h->N, sizeof(float) * B * h->N,
                               cudaMemcpyHostToDevice, h->stream));
        st = solve_impl(h, h->s_stage, B, o, h->z_stage, phase ? h->phi_stage : nullptr, info ? info + f0 : nullptr);
        if (st != TOMO_OK) break;
        CK(cudaMemcpyAsync(zeta + (size_t)f0 * h->N, h->z_stage, sizeof(float) * B * h->N, cudaMemcpyDeviceToHost,
                           h->stream));
        if (phase)
            CK(cudaMemcpyAsync(phase + (size_t)f0 * nphi, h->phi_stage, sizeof(float) * B * nphi,
                               cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    if (st == TOMO_OK) st = check_wait_error();
    return end_call(h, st);
}

tomo_status tomo_ws_init(tomo_handle* h, int hidden, int max_batch, float in_scale, float out_scale,
                         int precond_input, float pre_gain) {
    if (!h || hidden < 1 || hidden > 32 || max_batch < 1 || !(in_scale > 0) || !(out_scale > 0)) return TOMO_EINVAL;
    if ((precond_input ? 2 : 1) * h->NP > 32 || (precond_input && !h->d_M32)) return TOMO_EINVAL;
    WarmStartNet& w = h->ws;
    if (w.ready) return TOMO_EINVAL;   // once per handle
    w.hybrid = precond_input != 0;
    const int ch[5] = {(w.hybrid ? 2 : 1) * h->NP, hidden, hidden, hidden, h->NP};
    size_t off = 0;
    for (int l = 0; l < 4; ++l) {
        w.ch[l] = ch[l];
        w.offW[l] = off;
        off += (size_t)ch[l + 1] * ch[l] * 9;
        w.offb[l] = off;
        off += ch[l + 1];
    }
    w.ch[4] = ch[4];
    w.np = (int)off;
    w.maxB = max_batch;
    w.in_scale = in_scale;
    w.out_scale = out_scale;
    w.pre_scale = 1.f / out_scale;
    w.pre_gain = pre_gain;
    TRY(dalloc(h, &w.params, off));
    TRY(dalloc(h, &w.grad, off));
    TRY(dalloc(h, &w.m, off));
    TRY(dalloc(h, &w.v, off));
    for (int l = 0; l < 4; ++l) {
        TRY(dalloc(h, &w.Wt[l], (size_t)ch[l + 1] * ch[l] * 9));
        TRY(dalloc(h, &w.Wb[l], (size_t)ch[l + 1] * ch[l] * 9));
    }
    TRY(dalloc(h, &w.zero_bias, 32));
    const size_t plane = (size_t)h->n * h->n;
    const int cmax = std::max(hidden, ch[0]);
    for (int l = 0; l < 5; ++l) TRY(dalloc(h, &w.act[l], (size_t)max_batch * ch[l] * plane));
    TRY(dalloc(h, &w.d0, (size_t)max_batch * cmax * plane));
    TRY(dalloc(h, &w.d1, (size_t)max_batch * cmax * plane));
    TRY(dalloc(h, &w.gz, (size_t)max_batch * h->N));
    TRY(dalloc(h, &w.z, (size_t)max_batch * h->N));
    TRY(dalloc(h, &w.zpre, (size_t)max_batch * h->N));
    TRY(dalloc(h, &w.wpart, conv_wgrad_parts(max_batch, cmax, cmax, h->n)));
    TRY(dalloc(h, &w.sums, 512));
    TRY(dalloc(h, &w.loss, 1));
    CK(cudaMemsetAsync(w.params, 0, sizeof(float) * off, h->stream));
    CK(cudaMemsetAsync(w.m, 0, sizeof(float) * off, h->stream));
    CK(cudaMemsetAsync(w.v, 0, sizeof(float) * off, h->stream));
    CK(cudaMemsetAsync(w.zero_bias, 0, sizeof(float) * 32, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    w.step = 0;
    w.dirty = true;
    w.ready = true;
    return TOMO_OK;
}

tomo_status tomo_ws_param_count(const tomo_handle* h, int* count) {
    if (!h || !count || !h->ws.ready) return TOMO_EINVAL;
    *count = h->ws.np;
    return TOMO_OK;
}

tomo_status tomo_ws_set_params(tomo_handle* h, const float* params, int count) {
    if (!h || !params || !h->ws.ready || count != h->ws.np) return TOMO_EINVAL;
    CK(cudaMemcpyAsync(h->ws.params, params, sizeof(float) * count, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(h->ws.m, 0, sizeof(float) * count, h->stream));
    CK(cudaMemsetAsync(h->ws.v, 0, sizeof(float) * count, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->ws.step = 0;
    h->ws.dirty = true;
    return TOMO_OK;
}

tomo_status tomo_ws_get_params(const tomo_handle* h, float* params, int count) {
    if (!h || !params || !h->ws.ready || count != h->ws.np) return TOMO_EINVAL;
    CK(cudaMemcpyAsync(params, h->ws.params, sizeof(float) * count, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return TOMO_OK;
}

tomo_status tomo_ws_apply(tomo_handle* h, const float* slopes, float* zeta, int batch) {
    if (!h || !slopes || !zeta || batch < 0 || !h->ws.ready) return TOMO_EINVAL;
    Launch L = launch_of(h);
    for (int b0 = 0; b0 < batch; b0 += h->ws.maxB) {
        const int nb = std::min(h->ws.maxB, batch - b0);
        TRY(ws_forward(h, L, slopes + (size_t)b0 * h->N, nb, zeta + (size_t)b0 * h->N));
    }
    return TOMO_OK;
}

tomo_status tomo_ws_gradient(tomo_handle* h, const float* slopes, const float* target, int batch, float* grad_host,
                             double* loss_host) {
    if (!h || !slopes || !target || !h->ws.ready || batch < 1 || batch > h->ws.maxB) return TOMO_EINVAL;
    Launch L = launch_of(h);
    WarmStartNet& w = h->ws;
    TRY(ws_forward(h, L, slopes, batch, w.z));
    CK(loss_grad(L, (size_t)batch * h->N, w.z, target, w.sums, w.gz, w.loss));
    TRY(ws_backward(h, L, batch));
    if (grad_host) CK(cudaMemcpyAsync(grad_host, w.grad, sizeof(float) * w.np, cudaMemcpyDeviceToHost, h->stream));
    if (loss_host) CK(cudaMemcpyAsync(loss_host, w.loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return TOMO_OK;
}

tomo_status tomo_ws_train_step(tomo_handle* h, const float* slopes, const float* target, int batch, float lr,
                               double* loss_host) {
    if (!(lr > 0)) return TOMO_EINVAL;
    TRY(tomo_ws_gradient(h, slopes, target, batch, nullptr, loss_host));
    Launch L = launch_of(h);
    WarmStartNet& w = h->ws;
    w.step += 1;
    CK(adam(L, w.np, w.params, w.grad, w.m, w.v, lr, w.step));
    w.dirty = true;
    return TOMO_OK;
}

tomo_status tomo_apply_precond(tomo_handle* h, const float* x, float* y, int batch) {
    if (!h || !x || !y || batch < 0 || x == y || !h->d_M32) return TOMO_EINVAL;
    Launch L = launch_of(h);
    for (int f0 = 0; f0 < batch; f0 += h->max_batch) {
        const int B = std::min(h->max_batch, batch - f0);
        TRY(apply_pre(h, L, x + (size_t)f0 * h->N, y + (size_t)f0 * h->N, B));
    }
    return TOMO_OK;
}

long long tomo_launch_count(const tomo_handle* h) { return h ? h->launches : 0; }

tomo_status tomo_set_kernel_timing(tomo_handle* h, int enable) {
    if (!h) return TOMO_EINVAL;
    h->timing = enable != 0;
    for (int k = 0; k < TOMO_NKERNELS; ++k) { h->kt_ms[k] = 0; h->kt_n[k] = 0; }
    h->frame_iters = 0;
    return TOMO_OK;
}

tomo_status tomo_get_kernel_timing(const tomo_handle* h, double* ms_total, long long* launches,
                                   long long* frame_iters) {
    if (!h || !ms_total || !launches) return TOMO_EINVAL;
    for (int k = 0; k < TOMO_NKERNELS; ++k) { ms_total[k] = h->kt_ms[k]; launches[k] = h->kt_n[k]; }
    if (frame_iters) *frame_iters = h->frame_iters;
    return TOMO_OK;
}

void tomo_destroy(tomo_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    release(h);
}

const char* tomo_strerror(tomo_status s) {
    switch (s) {
        case TOMO_OK: return "ok";
        case TOMO_EINVAL: return "invalid argument or configuration";
        case TOMO_ENOMEM: return "out of memory";
        case TOMO_ECUDA: return "CUDA runtime error";
        case TOMO_ETIMEOUT: return "bounded device wait expired";
        case TOMO_ERANGE: return "size beyond the supported maximum";
    }
    return "unknown status";
}

}  // extern "C"
