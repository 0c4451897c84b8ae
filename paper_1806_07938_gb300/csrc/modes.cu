// Tip/tilt/focus removal (Sec. 2.F, mode removal for laser guide stars).
//
// M_s,i = I - Z_s,i Z_s,i^+ removes from the 2 n_vs slopes of WFS i the
// slopes of tip, tilt and focus; with an orthonormal basis Q of the columns
// of Z_s,i (3 x 2 n_vs, the same for every WFS since all share one
// subaperture grid), M_s,i y = y - Q^T (Q y).  M_phi does the same on the
// valid phase points with the basis of x, y and x^2 + y^2.  Both are
// O(n_vs) per WFS: two passes over the block, three dot products.
#include "kernels.cuh"

namespace tomo {

namespace {

inline void count(const Launch& L) {
    if (L.counter) ++*L.counter;
}

constexpr int kModeThreads = 256;

// Block-wide sums of V doubles; the result is valid in every thread.
template <int V>
__device__ __forceinline__ void block_sums(double (&v)[V], double (*red)[kModeThreads / 32]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        double a = v[k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) red[k][warp] = a;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < V; ++k) {
        double s = 0.0;
        for (int w = 0; w < kModeThreads / 32; ++w) s += red[k][w];
        v[k] = s;
    }
    __syncthreads();
}

// One block per (block index, frame): y[blk] -= Q^T (Q y[blk]) over len
// entries.  With dots != nullptr (FP32 CG vectors) also the partial sums
// xin^T y, r^T y, y^T y of the projected y for the two halves of the block
// (the x- and y-slope planes), stored like the row-inverse pass stores them.
template <typename TV>
__global__ void __launch_bounds__(kModeThreads)
k_mode_project(int len, int nblk, int rg, const double* __restrict__ Q, const FrameState* st, TV* __restrict__ y,
               const float* __restrict__ xin, const float* __restrict__ r, double* __restrict__ dots) {
    __shared__ double red[6][kModeThreads / 32];
    const int blk = blockIdx.x, f = blockIdx.y;
    if (st && !st[f].active) return;
    TV* yb = y + ((size_t)f * nblk + blk) * len;
    double c[3] = {0.0, 0.0, 0.0};
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const double v = (double)yb[e];
        c[0] += Q[e] * v;
        c[1] += Q[len + e] * v;
        c[2] += Q[2 * len + e] * v;
    }
    block_sums<3>(c, red);
    const int half = len / 2;
    double d[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const size_t base = ((size_t)f * nblk + blk) * len;
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const double v = (double)yb[e] - (c[0] * Q[e] + c[1] * Q[len + e] + c[2] * Q[2 * len + e]);
        const TV out = (TV)v;
        yb[e] = out;
        if (dots) {
            const int h = e < half ? 0 : 3;
            const double o = (double)out;
            d[h + 0] += (double)xin[base + e] * o;
            d[h + 1] += (double)r[base + e] * o;
            d[h + 2] += o * o;
        }
    }
    if (dots) {
        // the row passes store partial sums per (plane, row group): the projected
        // sums go to row group 0, the other groups' entries are cleared
        block_sums<6>(d, red);
        for (int i = threadIdx.x; i < 6 * rg; i += blockDim.x) {
            const int plane = 2 * blk + i / (3 * rg), grp = (i / 3) % rg, c = i % 3;
            dots[(((size_t)f * 2 * nblk + plane) * rg + grp) * 3 + c] = grp == 0 ? d[(i / (3 * rg)) * 3 + c] : 0.0;
        }
    }
}

// Elongated-spot noise (Sec. 2.F): Sigma_eta_eta is block diagonal with one
// 2 x 2 block per subaperture, coupling its x and y slopes.  One block per
// (guide star, frame) adds y_x += nu_f (s_xx x_x + s_xy x_y) and
// y_y += nu_f (s_xy x_x + s_yy x_y) on the guide star's 2 n_vs entries
// (cov [n_gs][n_vs][3] = s_xx, s_yy, s_xy) and, with dots != nullptr,
// recomputes the CG partial sums of both planes like k_mode_project.
template <typename TV>
__global__ void __launch_bounds__(kModeThreads)
k_noise_blocks(int n_vs, int n_gs, int rg, const double* __restrict__ cov, const double2* __restrict__ fscale,
               const FrameState* st, TV* __restrict__ y, const TV* __restrict__ x, const float* __restrict__ xin,
               const float* __restrict__ r, double* __restrict__ dots) {
    __shared__ double red[6][kModeThreads / 32];
    const int g = blockIdx.x, f = blockIdx.y;
    if (st && !st[f].active) return;
    const double nu = fscale ? fscale[f].y : 1.0;
    const size_t base = ((size_t)f * n_gs + g) * 2 * n_vs;
    const double* c = cov + (size_t)g * n_vs * 3;
    double d[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int e = threadIdx.x; e < n_vs; e += blockDim.x) {
        const double xx = (double)x[base + e], xy = (double)x[base + n_vs + e];
        const double sxx = c[3 * e], syy = c[3 * e + 1], sxy = c[3 * e + 2];
        const TV ox = (TV)((double)y[base + e] + nu * (sxx * xx + sxy * xy));
        const TV oy = (TV)((double)y[base + n_vs + e] + nu * (sxy * xx + syy * xy));
        y[base + e] = ox;
        y[base + n_vs + e] = oy;
        if (dots) {
            const double a = (double)ox, b = (double)oy;
            d[0] += (double)xin[base + e] * a;
            d[1] += (double)r[base + e] * a;
            d[2] += a * a;
            d[3] += (double)xin[base + n_vs + e] * b;
            d[4] += (double)r[base + n_vs + e] * b;
            d[5] += b * b;
        }
    }
    if (dots) {
        block_sums<6>(d, red);
        for (int i = threadIdx.x; i < 6 * rg; i += blockDim.x) {
            const int plane = 2 * g + i / (3 * rg), grp = (i / 3) % rg, cc = i % 3;
            dots[(((size_t)f * 2 * n_gs + plane) * rg + grp) * 3 + cc] = grp == 0 ? d[(i / (3 * rg)) * 3 + cc] : 0.0;
        }
    }
}

}  // namespace

template <typename TV>
cudaError_t noise_blocks(const Launch& L, int B, int n_vs, int n_gs, int rg, const double* cov, const double2* fscale,
                         const FrameState* st, TV* y, const TV* x, const float* xin, const CgVecs* cg) {
    if (B <= 0) return cudaSuccess;
    if (cg && (!xin || rg < 1)) return cudaErrorInvalidValue;
    k_noise_blocks<TV><<<dim3(n_gs, B), kModeThreads, 0, L.stream>>>(
        n_vs, n_gs, rg, cov, fscale, st, y, x, cg ? xin : nullptr, cg ? (cg->mode == 3 ? cg->Ap : cg->r) : nullptr,
        cg ? cg->dot_part : nullptr);
    count(L);
    return cudaGetLastError();
}

template cudaError_t noise_blocks<float>(const Launch&, int, int, int, int, const double*, const double2*,
                                         const FrameState*, float*, const float*, const float*, const CgVecs*);
template cudaError_t noise_blocks<double>(const Launch&, int, int, int, int, const double*, const double2*,
                                          const FrameState*, double*, const double*, const float*, const CgVecs*);

template <typename TV>
cudaError_t mode_project(const Launch& L, int B, int len, int nblk, int rg, const double* Q, const FrameState* st,
                         TV* y, const float* xin, const CgVecs* cg) {
    if (B <= 0) return cudaSuccess;
    if (cg && (!xin || (len & 1) || rg < 1)) return cudaErrorInvalidValue;
    k_mode_project<TV><<<dim3(nblk, B), kModeThreads, 0, L.stream>>>(
        len, nblk, rg, Q, st, y, cg ? xin : nullptr, cg ? (cg->mode == 3 ? cg->Ap : cg->r) : nullptr,
        cg ? cg->dot_part : nullptr);
    count(L);
    return cudaGetLastError();
}

template cudaError_t mode_project<float>(const Launch&, int, int, int, int, const double*, const FrameState*,
                                         float*, const float*, const CgVecs*);
template cudaError_t mode_project<double>(const Launch&, int, int, int, int, const double*, const FrameState*,
                                          double*, const float*, const CgVecs*);

}  // namespace tomo
