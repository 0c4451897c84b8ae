// Flexible preconditioned conjugate gradients with a learned preconditioner
// (an addition to the paper, whose solvers run without a preconditioner and
// which names preconditioning the open problem, Sec. 6).
//
// The preconditioner is the block-circulant M plus the warm-start network's
// correction: z = pre_gain M r + out_scale N([r, M r]).  It changes from one
// iteration to the next (the network is not linear), so the direction update
// uses the flexible (Polak-Ribiere) form of Notay, "Flexible conjugate
// gradients", SIAM J. Sci. Comput. 22 (2000):
//     beta_k = z_k^T (r_k - r_{k-1}) / (r_{k-1}^T z_{k-1}) = -alpha_{k-1} z_k^T q_{k-1} / (r_{k-1}^T z_{k-1}),
// with q = A p (r_k - r_{k-1} = -alpha q), p_k = z_k + beta_k p_{k-1},
// alpha_k = r_k^T z_k / p_k^T q_k.  Plain PCG with M alone is the fallback
// and the judge: a frame leaves the flexible iteration for good (restarting
// its direction from M r) when r^T z <= 0 or when r^T r has set no new
// minimum for `window` iterations.  The solver reports such frames as
// TOMO_FRAME_FALLBACK_PLAIN_CG when they converge.
//
// Per-thread sums are FP32 (a few tens of products), FP64 across threads,
// blocks and frames' partials (GB300's FP64 rate is ~1/64 of its FP32 rate).
#include "kernels.cuh"

namespace tomo {

namespace {

constexpr int kT = 256;

inline void bump(const Launch& L) {
    if (L.counter) ++*L.counter;
}

template <int V>
__device__ __forceinline__ void block_sums(double (&v)[V], double (*red)[kT / 32]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        double x = v[j];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[j][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < V; ++j) {
            double t = 0.0;
            for (int w = 0; w < kT / 32; ++w) t += red[j][w];
            v[j] = t;
        }
    }
}

__device__ __forceinline__ double warp_total(double v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

}  // namespace

__global__ void __launch_bounds__(kT)
k_flex_dots(int N, int nparts, const FrameState* __restrict__ st, const float* __restrict__ r,
            const float* __restrict__ q, const float* __restrict__ zN, const float* __restrict__ zM,
            double* __restrict__ parts) {
    __shared__ double red[5][kT / 32];
    const int f = blockIdx.y;
    if (!st[f].active) return;
    const size_t b = (size_t)f * N;
    float a[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const float ri = r[b + i], qi = q[b + i], zn = zN[b + i], zm = zM[b + i];
        a[0] = fmaf(ri, ri, a[0]);
        a[1] = fmaf(ri, zn, a[1]);
        a[2] = fmaf(qi, zn, a[2]);
        a[3] = fmaf(ri, zm, a[3]);
        a[4] = fmaf(qi, zm, a[4]);
    }
    double v[5] = {a[0], a[1], a[2], a[3], a[4]};
    block_sums<5>(v, red);
    if (threadIdx.x == 0)
        for (int j = 0; j < 5; ++j) parts[((size_t)f * nparts + blockIdx.x) * 5 + j] = v[j];
}

cudaError_t flex_dots(const Launch& L, int B, int N, int nparts, const FrameState* st, const float* r, const float* q,
                      const float* zN, const float* zM, double* parts) {
    k_flex_dots<<<dim3(nparts, B), kT, 0, L.stream>>>(N, nparts, st, r, q, zN, zM, parts);
    bump(L);
    return cudaGetLastError();
}

// One warp per frame.
__global__ void k_flex_beta(int B, int nparts, const double* __restrict__ parts, int window, FrameState* st) {
    const int f = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (f >= B) return;
    double v[5] = {0, 0, 0, 0, 0};
    for (int i = lane; i < nparts; i += 32)
        for (int j = 0; j < 5; ++j) v[j] += parts[((size_t)f * nparts + i) * 5 + j];
    for (int j = 0; j < 5; ++j) v[j] = warp_total(v[j]);
    if (lane != 0 || !st[f].active) return;
    FrameState s = st[f];
    const double rr = v[0];
    s.rr = rr;
    s.relres = sqrt(rr / s.snorm2);
    if (rr <= s.tol2) {
        s.active = 0;
        s.status = 0;
        st[f] = s;
        return;
    }
    if (!isfinite(rr)) {
        s.active = 0;
        s.status = 2;  // TOMO_FRAME_BREAKDOWN
        st[f] = s;
        return;
    }
    const bool fresh = s.fresh != 0;
    bool fell = false;
    if (fresh) {
        s.ckpt_iter = s.iters;
        s.rr_ckpt = rr;
    } else if (!s.fb) {
        // rr_ckpt: the smallest r^T r so far; no new minimum within `window`
        // iterations leaves the flexible iteration (the residual norm of a
        // working preconditioner is not monotone, but its minimum keeps falling)
        if (rr < s.rr_ckpt) {
            s.rr_ckpt = rr;
            s.ckpt_iter = s.iters;
        } else if (s.iters - s.ckpt_iter >= window) {
            s.fb = 1;
            fell = true;
        }
    }
    double rz = v[1], qz = v[2];
    if (!s.fb && (!(rz > 0.0) || !isfinite(rz) || !isfinite(qz))) {
        s.fb = 1;                      // the learned step is not a descent direction
        fell = true;
    }
    if (s.fb) {
        rz = v[3];
        qz = v[4];
    }
    if (!(rz > 0.0) || !isfinite(rz) || !isfinite(qz)) {
        s.active = 0;
        s.status = 2;  // TOMO_FRAME_BREAKDOWN (M r not a descent direction)
        st[f] = s;
        return;
    }
    s.beta = (fresh || fell) ? 0.0 : -s.alpha * qz / s.gamma;
    s.gamma = rz;
    s.fresh = 0;
    st[f] = s;
}

cudaError_t flex_beta(const Launch& L, int B, int nparts, const double* parts, int window, FrameState* st) {
    k_flex_beta<<<(B + 3) / 4, 128, 0, L.stream>>>(B, nparts, parts, window, st);
    bump(L);
    return cudaGetLastError();
}

__global__ void k_flex_dir(int N, const FrameState* __restrict__ st, const float* __restrict__ zN,
                           const float* __restrict__ zM, float* __restrict__ p) {
    const int f = blockIdx.y;
    if (!st[f].active) return;
    const float beta = (float)st[f].beta;
    const float* z = st[f].fb ? zM : zN;
    const size_t b = (size_t)f * N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        p[b + i] = z[b + i] + beta * p[b + i];
}

cudaError_t flex_dir(const Launch& L, int B, int N, const FrameState* st, const float* zN, const float* zM, float* p) {
    k_flex_dir<<<dim3(32, B), kT, 0, L.stream>>>(N, st, zN, zM, p);
    bump(L);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kT)
k_flex_pq(int N, int nparts, const FrameState* __restrict__ st, const float* __restrict__ p,
          const float* __restrict__ q, double* __restrict__ parts) {
    __shared__ double red[1][kT / 32];
    const int f = blockIdx.y;
    if (!st[f].active) return;
    const size_t b = (size_t)f * N;
    float a = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        a = fmaf(p[b + i], q[b + i], a);
    double v[1] = {a};
    block_sums<1>(v, red);
    if (threadIdx.x == 0) parts[(size_t)f * nparts + blockIdx.x] = v[0];
}

cudaError_t flex_pq(const Launch& L, int B, int N, int nparts, const FrameState* st, const float* p, const float* q,
                    double* parts) {
    k_flex_pq<<<dim3(nparts, B), kT, 0, L.stream>>>(N, nparts, st, p, q, parts);
    bump(L);
    return cudaGetLastError();
}

__global__ void k_flex_alpha(int B, int nparts, const double* __restrict__ parts, FrameState* st) {
    const int f = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (f >= B) return;
    double pq = 0.0;
    for (int i = lane; i < nparts; i += 32) pq += parts[(size_t)f * nparts + i];
    pq = warp_total(pq);
    if (lane != 0 || !st[f].active) return;
    FrameState s = st[f];
    if (!(pq > 0.0) || !isfinite(pq)) {
        s.active = 0;
        s.status = 2;  // TOMO_FRAME_BREAKDOWN
        st[f] = s;
        return;
    }
    s.alpha = s.gamma / pq;
    s.iters += 1;
    st[f] = s;
}

cudaError_t flex_alpha(const Launch& L, int B, int nparts, const double* parts, FrameState* st) {
    k_flex_alpha<<<(B + 3) / 4, 128, 0, L.stream>>>(B, nparts, parts, st);
    bump(L);
    return cudaGetLastError();
}

__global__ void k_flex_update(int N, const FrameState* __restrict__ st, float* __restrict__ x, float* __restrict__ r,
                              const float* __restrict__ p, const float* __restrict__ q) {
    const int f = blockIdx.y;
    if (!st[f].active) return;
    const float alpha = (float)st[f].alpha;
    const size_t b = (size_t)f * N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        x[b + i] += alpha * p[b + i];
        r[b + i] -= alpha * q[b + i];
    }
}

cudaError_t flex_update(const Launch& L, int B, int N, const FrameState* st, float* x, float* r, const float* p,
                        const float* q) {
    k_flex_update<<<dim3(32, B), kT, 0, L.stream>>>(N, st, x, r, p, q);
    bump(L);
    return cudaGetLastError();
}

}  // namespace tomo
