// Vector kernels of the FP64 solves (tomo_solve_f64) and of the FP64 outer
// loop of mixed-precision iterative refinement.
//
// FP64 conjugate gradients (Sec. 2.G) run unfused: the operator product is
// the FP64 three-pass 2RBT MVM of kernels.cu (Eq. mvm_ss), and these kernels
// do the vector updates and the partial sums the per-frame scalar kernel
// (k_cg_scalars, Chronopoulos & Gear's recurrence for r^T r) consumes.  One
// block row per frame (blockIdx.y), `nparts` blocks along x, each leaving one
// partial sum per quantity in a fixed order, so results do not depend on
// scheduling.
#include "kernels.cuh"

namespace tomo {

namespace {

constexpr int kThreads64 = 256;

inline void bump(const Launch& L) {
    if (L.counter) ++*L.counter;
}

__device__ __forceinline__ double block_total(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

}  // namespace

// r = s - A x0 (or s when Ax0 is null, with x = 0), p = Ap = 0; partial sums
// of r^T r and s^T s into parts [B][2][nparts].
__global__ void __launch_bounds__(kThreads64)
k64_cg_init(int N, int nparts, const double* __restrict__ s, const double* __restrict__ Ax0, double* __restrict__ x,
            double* __restrict__ r, double* __restrict__ p, double* __restrict__ Ap, double* __restrict__ parts) {
    __shared__ double red[kThreads64 / 32];
    const int f = blockIdx.y;
    const size_t base = (size_t)f * N;
    double rr = 0.0, ss = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double si = s[base + i];
        const double ri = Ax0 ? si - Ax0[base + i] : si;
        if (!Ax0) x[base + i] = 0.0;
        r[base + i] = ri;
        p[base + i] = 0.0;
        Ap[base + i] = 0.0;
        rr += ri * ri;
        ss += si * si;
    }
    const double a = block_total(rr, red);
    if (threadIdx.x == 0) parts[((size_t)f * 2 + 0) * nparts + blockIdx.x] = a;
    const double b = block_total(ss, red);
    if (threadIdx.x == 0) parts[((size_t)f * 2 + 1) * nparts + blockIdx.x] = b;
}

cudaError_t cg64_init(const Launch& L, int B, int N, int nparts, const double* s, const double* Ax0, double* x,
                      double* r, double* p, double* Ap, double* parts) {
    k64_cg_init<<<dim3(nparts, B), kThreads64, 0, L.stream>>>(N, nparts, s, Ax0, x, r, p, Ap, parts);
    bump(L);
    return cudaGetLastError();
}

// The update the scalar kernel scheduled (alpha, beta of the frame):
// x += alpha p, r -= alpha Ap (skipped while alpha = 0, i.e. on a (re)start),
// p = r + beta p; partial sums of r^T r of the updated residual into
// rr_part [B][nparts].  Frames that are not active are left as they are.
__global__ void __launch_bounds__(kThreads64)
k64_update(int N, int nparts, const FrameState* __restrict__ st, double* __restrict__ x, double* __restrict__ r,
           double* __restrict__ p, const double* __restrict__ Ap, double* __restrict__ rr_part) {
    __shared__ double red[kThreads64 / 32];
    const int f = blockIdx.y;
    if (!st[f].active) return;
    const double alpha = st[f].alpha, beta = st[f].beta;
    const size_t base = (size_t)f * N;
    double rr = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        double ri = r[base + i];
        const double pi = p[base + i];
        if (alpha != 0.0) {
            x[base + i] += alpha * pi;
            ri -= alpha * Ap[base + i];
            r[base + i] = ri;
        }
        p[base + i] = ri + beta * pi;
        rr += ri * ri;
    }
    const double t = block_total(rr, red);
    if (threadIdx.x == 0) rr_part[(size_t)f * nparts + blockIdx.x] = t;
}

cudaError_t cg64_update(const Launch& L, int B, int N, int nparts, const FrameState* st, double* x, double* r,
                        double* p, const double* Ap, double* rr_part) {
    k64_update<<<dim3(nparts, B), kThreads64, 0, L.stream>>>(N, nparts, st, x, r, p, Ap, rr_part);
    bump(L);
    return cudaGetLastError();
}

// Partial sums p^T Ap, r^T Ap, Ap^T Ap into dot_part [B][nparts][3] (the
// layout of the fused passes' sums, which k_cg_scalars reads).
__global__ void __launch_bounds__(kThreads64)
k64_dots(int N, int nparts, const FrameState* __restrict__ st, const double* __restrict__ p,
         const double* __restrict__ r, const double* __restrict__ Ap, double* __restrict__ dot_part) {
    __shared__ double red[kThreads64 / 32];
    const int f = blockIdx.y;
    if (!st[f].active) return;
    const size_t base = (size_t)f * N;
    double pa = 0.0, ra = 0.0, aa = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double a = Ap[base + i];
        pa += p[base + i] * a;
        ra += r[base + i] * a;
        aa += a * a;
    }
    double* d = dot_part + ((size_t)f * nparts + blockIdx.x) * 3;
    const double s0 = block_total(pa, red);
    if (threadIdx.x == 0) d[0] = s0;
    const double s1 = block_total(ra, red);
    if (threadIdx.x == 0) d[1] = s1;
    const double s2 = block_total(aa, red);
    if (threadIdx.x == 0) d[2] = s2;
}

cudaError_t cg64_dots(const Launch& L, int B, int N, int nparts, const FrameState* st, const double* p,
                      const double* r, const double* Ap, double* dot_part) {
    k64_dots<<<dim3(nparts, B), kThreads64, 0, L.stream>>>(N, nparts, st, p, r, Ap, dot_part);
    bump(L);
    return cudaGetLastError();
}

// r = s - Ax (written when r is not null), partial sums of r^T r into
// parts [B][nparts] (the layout k_true_residual_finalize reads).
__global__ void __launch_bounds__(kThreads64)
k64_residual(int N, int nparts, const double* __restrict__ s, const double* __restrict__ Ax, double* __restrict__ r,
             double* __restrict__ parts) {
    __shared__ double red[kThreads64 / 32];
    const int f = blockIdx.y;
    const size_t base = (size_t)f * N;
    double rr = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double ri = s[base + i] - Ax[base + i];
        if (r) r[base + i] = ri;
        rr += ri * ri;
    }
    const double t = block_total(rr, red);
    if (threadIdx.x == 0) parts[(size_t)f * nparts + blockIdx.x] = t;
}

cudaError_t residual64(const Launch& L, int B, int N, int nparts, const double* s, const double* Ax, double* r,
                       double* parts) {
    k64_residual<<<dim3(nparts, B), kThreads64, 0, L.stream>>>(N, nparts, s, Ax, r, parts);
    bump(L);
    return cudaGetLastError();
}

// Mixed precision: rhs32[f] = (float) r[f] for frames still above tol
// (rel[f] > tol) and 0 for the others, so that the inner FP32 solve leaves
// converged frames untouched; rel [B] is the frame's FP64 relative residual.
__global__ void k64_inner_rhs(int N, const double* __restrict__ rel, double tol, const double* __restrict__ r,
                              float* __restrict__ rhs) {
    const int f = blockIdx.y;
    const bool on = rel[f] > tol;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        rhs[(size_t)f * N + i] = on ? (float)r[(size_t)f * N + i] : 0.f;
}

cudaError_t inner_rhs(const Launch& L, int B, int N, const double* rel, double tol, const double* r, float* rhs) {
    k64_inner_rhs<<<dim3(16, B), kThreads64, 0, L.stream>>>(N, rel, tol, r, rhs);
    bump(L);
    return cudaGetLastError();
}

// x64 += d32 (the inner solve's correction, accumulated in FP64).
__global__ void k64_add_f32(size_t n, const float* __restrict__ d, double* __restrict__ x) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] += (double)d[i];
}

cudaError_t add_f32_to_f64(const Launch& L, size_t n, const float* d, double* x) {
    k64_add_f32<<<1216, kThreads64, 0, L.stream>>>(n, d, x);
    bump(L);
    return cudaGetLastError();
}

// out32 = (float)(scale[f] x64) per frame (scale null: 1).
__global__ void k64_to_f32(int N, const double* __restrict__ scale, const double* __restrict__ x,
                           float* __restrict__ out) {
    const int f = blockIdx.y;
    const double c = scale ? scale[f] : 1.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        out[(size_t)f * N + i] = (float)(c * x[(size_t)f * N + i]);
}

cudaError_t f64_to_f32(const Launch& L, int B, int N, const double* scale, const double* x, float* out) {
    k64_to_f32<<<dim3(16, B), kThreads64, 0, L.stream>>>(N, scale, x, out);
    bump(L);
    return cudaGetLastError();
}

// rel[f] = sqrt(sum of parts[f] / snorm2[f]) (FP64 relative residual of the
// outer loop; snorm2[f] = 0 gives 0, a non-finite sum NaN).
__global__ void k64_relres(int B, int nparts, const double* __restrict__ parts, const double* __restrict__ snorm2,
                           double* __restrict__ rel) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= B) return;
    double t = 0.0;
    for (int i = 0; i < nparts; ++i) t += parts[(size_t)f * nparts + i];
    const double s2 = snorm2[f];
    rel[f] = s2 > 0.0 ? sqrt(t / s2) : (isfinite(t) ? 0.0 : nan(""));
}

cudaError_t relres64(const Launch& L, int B, int nparts, const double* parts, const double* snorm2, double* rel) {
    k64_relres<<<(B + 127) / 128, 128, 0, L.stream>>>(B, nparts, parts, snorm2, rel);
    bump(L);
    return cudaGetLastError();
}

// snorm2[f] = s[f]^T s[f] in FP64, through per-block parts [B][nparts].
__global__ void __launch_bounds__(kThreads64)
k64_norm2_parts(int N, int nparts, const double* __restrict__ s, double* __restrict__ parts) {
    __shared__ double red[kThreads64 / 32];
    const int f = blockIdx.y;
    double t = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double v = s[(size_t)f * N + i];
        t += v * v;
    }
    const double a = block_total(t, red);
    if (threadIdx.x == 0) parts[(size_t)f * nparts + blockIdx.x] = a;
}

__global__ void k64_sum_parts(int B, int nparts, const double* __restrict__ parts, double* __restrict__ out) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= B) return;
    double t = 0.0;
    for (int i = 0; i < nparts; ++i) t += parts[(size_t)f * nparts + i];
    out[f] = t;
}

cudaError_t norm2_64(const Launch& L, int B, int N, int nparts, const double* s, double* parts, double* out) {
    k64_norm2_parts<<<dim3(nparts, B), kThreads64, 0, L.stream>>>(N, nparts, s, parts);
    bump(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k64_sum_parts<<<(B + 127) / 128, 128, 0, L.stream>>>(B, nparts, parts, out);
    bump(L);
    return cudaGetLastError();
}

}  // namespace tomo
