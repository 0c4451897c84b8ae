// Learned warm start: a small convolutional network over the per-guide-star
// slope grids (an addition to the paper, which starts its iterative solvers
// from zero or from the previous frame, Sec. 5).
//
// Activations are [B][C][n][n] FP32 on the subaperture grid, zero outside the
// grid (3 x 3 kernels, zero padding).  Layer l: y = conv3x3(x, W_l) + b_l,
// ReLU on all but the last layer.  Weights W_l are [Cout][Cin][3][3].
#include <algorithm>

#include <cuda_runtime.h>

#include "cnn.cuh"

namespace tomo {

namespace {
inline void bump(const Launch& L) {
    if (L.counter) ++*L.counter;
}
constexpr int kTile = 16;          // output tile side of the convolution kernels
constexpr int kCog = 8;            // output channels per block
constexpr int kMaxC = 32;          // largest channel count supported
}  // namespace

// slopes [B][NP][n_vs] (valid subapertures) -> grid [B][NP][n][n] * scale, zero elsewhere
__global__ void k_scatter_grid(int B, int NP, int n, int n_vs, const int* __restrict__ rowcol,
                               const float* __restrict__ s, float scale, float* __restrict__ grid) {
    const size_t total = (size_t)B * NP * n * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        grid[i] = 0.f;
}

// grid [B][NP][n][n] -> valid entries [B][NP][n_vs] * scale
__global__ void k_gather_valid(int B, int NP, int n, int n_vs, const int* __restrict__ rowcol,
                               const float* __restrict__ grid, float scale, float* __restrict__ out) {
    const size_t total = (size_t)B * NP * n_vs;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(i % n_vs);
        const size_t plane = i / n_vs;
        const int rc = rowcol[e];
        out[i] = scale * grid[(plane * n + (rc >> 16)) * n + (rc & 0xffff)];
    }
}

// planes [B][np][n_vs] -> channels [c0, c0 + np) of a [B][ctot][n][n] grid (the grid is not cleared)
__global__ void k_scatter_planes(int B, int np, int ctot, int c0, int n, int n_vs, const int* __restrict__ rowcol,
                                 const float* __restrict__ s, float scale, float* __restrict__ grid) {
    const size_t total = (size_t)B * np * n_vs;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(i % n_vs);
        const size_t plane = i / n_vs;
        const size_t b = plane / np, c = plane % np;
        const int rc = rowcol[e];
        grid[((b * ctot + c0 + c) * n + (rc >> 16)) * n + (rc & 0xffff)] = scale * s[i];
    }
}

cudaError_t cnn_scatter_planes(const Launch& L, int B, int c0, int ctot, int np, int n, int n_vs, const int* rowcol,
                               const float* s, float scale, float* grid) {
    const size_t tv = (size_t)B * np * n_vs;
    k_scatter_planes<<<(unsigned)std::min((tv + 255) / 256, (size_t)4096), 256, 0, L.stream>>>(B, np, ctot, c0, n,
                                                                                           n_vs, rowcol, s, scale,
                                                                                           grid);
    bump(L);
    return cudaGetLastError();
}

__global__ void k_axpy(size_t total, float a, const float* __restrict__ x, float* __restrict__ y) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

cudaError_t axpy_f32(const Launch& L, size_t total, float a, const float* x, float* y) {
    k_axpy<<<(unsigned)std::min((total + 255) / 256, (size_t)4096), 256, 0, L.stream>>>(total, a, x, y);
    bump(L);
    return cudaGetLastError();
}

cudaError_t cnn_scatter(const Launch& L, int B, int NP, int n, int n_vs, const int* rowcol, const float* s,
                        float scale, float* grid, int ctot) {
    if (ctot < NP) ctot = NP;
    const size_t total = (size_t)B * ctot * n * n;
    k_scatter_grid<<<(unsigned)std::min((total + 255) / 256, (size_t)4096), 256, 0, L.stream>>>(B, ctot, n, n_vs,
                                                                                           rowcol, s, scale, grid);
    bump(L);
    const size_t tv = (size_t)B * NP * n_vs;
    k_scatter_planes<<<(unsigned)std::min((tv + 255) / 256, (size_t)4096), 256, 0, L.stream>>>(B, NP, ctot, 0, n,
                                                                                           n_vs, rowcol, s, scale,
                                                                                           grid);
    bump(L);
    return cudaGetLastError();
}

cudaError_t cnn_gather(const Launch& L, int B, int NP, int n, int n_vs, const int* rowcol, const float* grid,
                       float scale, float* out) {
    const size_t tv = (size_t)B * NP * n_vs;
    k_gather_valid<<<(unsigned)std::min((tv + 255) / 256, (size_t)4096), 256, 0, L.stream>>>(B, NP, n, n_vs, rowcol, grid,
                                                                                      scale, out);
    bump(L);
    return cudaGetLastError();
}

// y[b][co] = relu?(b[co] + sum_ci sum_taps Wt[ci][tap][co] x[b][ci][p + tap]),
// Wt the weights as [Cin][9][Cout].  Block: a 16 x 16 pixel tile, 8 output
// channels, one frame; the input tile with its halo and the block's weights
// sit in shared memory.
__global__ void __launch_bounds__(kTile * kTile)
k_conv_fwd(int Cin, int Cout, int n, const float* __restrict__ x, const float* __restrict__ Wt,
           const float* __restrict__ bias, float* __restrict__ y, int relu) {
    extern __shared__ __align__(16) float smf[];
    float (*xs)[kTile + 2][kTile + 2] = reinterpret_cast<float (*)[kTile + 2][kTile + 2]>(smf);
    float4 (*ws)[kCog / 4] = reinterpret_cast<float4 (*)[kCog / 4]>(smf + (size_t)Cin * (kTile + 2) * (kTile + 2));
    const int tiles = (n + kTile - 1) / kTile;
    const int tx0 = (blockIdx.x % tiles) * kTile, ty0 = (blockIdx.x / tiles) * kTile;
    const int co0 = blockIdx.y * kCog;
    const int b = blockIdx.z;
    const int tid = threadIdx.y * kTile + threadIdx.x;
    const float* xb = x + (size_t)b * Cin * n * n;
    for (int i = tid; i < Cin * (kTile + 2) * (kTile + 2); i += kTile * kTile) {
        const int ci = i / ((kTile + 2) * (kTile + 2));
        const int rem = i - ci * (kTile + 2) * (kTile + 2);
        const int yy = ty0 + rem / (kTile + 2) - 1, xx = tx0 + rem % (kTile + 2) - 1;
        xs[ci][rem / (kTile + 2)][rem % (kTile + 2)] =
            (yy >= 0 && yy < n && xx >= 0 && xx < n) ? __ldg(xb + ((size_t)ci * n + yy) * n + xx) : 0.f;
    }
    float* wsf = reinterpret_cast<float*>(ws);
    for (int i = tid; i < Cin * 9 * kCog; i += kTile * kTile) {
        const int c = i % kCog, k = i / kCog;     // k = ci * 9 + tap
        wsf[i] = co0 + c < Cout ? __ldg(Wt + (size_t)k * Cout + co0 + c) : 0.f;
    }
    __syncthreads();
    float acc[kCog];
#pragma unroll
    for (int c = 0; c < kCog; ++c) acc[c] = co0 + c < Cout ? __ldg(bias + co0 + c) : 0.f;
    const int py = threadIdx.y, px = threadIdx.x;
    for (int ci = 0; ci < Cin; ++ci) {
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const float v = xs[ci][py + tap / 3][px + tap % 3];
            const float4 w0 = ws[ci * 9 + tap][0], w1 = ws[ci * 9 + tap][1];
            acc[0] = fmaf(v, w0.x, acc[0]);
            acc[1] = fmaf(v, w0.y, acc[1]);
            acc[2] = fmaf(v, w0.z, acc[2]);
            acc[3] = fmaf(v, w0.w, acc[3]);
            acc[4] = fmaf(v, w1.x, acc[4]);
            acc[5] = fmaf(v, w1.y, acc[5]);
            acc[6] = fmaf(v, w1.z, acc[6]);
            acc[7] = fmaf(v, w1.w, acc[7]);
        }
    }
    const int oy = ty0 + py, ox = tx0 + px;
    if (oy < n && ox < n) {
#pragma unroll
        for (int c = 0; c < kCog; ++c)
            if (co0 + c < Cout) {
                const float v = relu ? fmaxf(acc[c], 0.f) : acc[c];
                y[(((size_t)b * Cout + co0 + c) * n + oy) * n + ox] = v;
            }
    }
}

cudaError_t conv_fwd(const Launch& L, int B, int Cin, int Cout, int n, const float* x, const float* Wt,
                     const float* bias, float* y, bool relu) {
    if (Cin > kMaxC || Cout < 1) return cudaErrorInvalidValue;
    const int tiles = (n + kTile - 1) / kTile;
    const size_t smem = sizeof(float) * ((size_t)Cin * (kTile + 2) * (kTile + 2) + (size_t)Cin * 9 * kCog);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_conv_fwd<<<dim3(tiles * tiles, (Cout + kCog - 1) / kCog, B), dim3(kTile, kTile), smem, L.stream>>>(
        Cin, Cout, n, x, Wt, bias, y, relu ? 1 : 0);
    bump(L);
    return cudaGetLastError();
}

// W [Cout][Cin][3][3] -> forward layout Wt[ci][tap][co] and data-gradient
// layout Wb[co][8 - tap][ci] (the transposed, flipped kernel: dX = conv(dY, Wb)).
__global__ void k_weight_layouts(int Cin, int Cout, const float* __restrict__ W, float* __restrict__ Wt,
                                 float* __restrict__ Wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Cout * Cin * 9) return;
    const int tap = i % 9, ci = (i / 9) % Cin, co = i / (9 * Cin);
    const float w = W[i];
    Wt[((size_t)ci * 9 + tap) * Cout + co] = w;
    if (Wb) Wb[((size_t)co * 9 + (8 - tap)) * Cin + ci] = w;
}

cudaError_t weight_layouts(const Launch& L, int Cin, int Cout, const float* W, float* Wt, float* Wb) {
    const int total = Cout * Cin * 9;
    k_weight_layouts<<<(total + 255) / 256, 256, 0, L.stream>>>(Cin, Cout, W, Wt, Wb);
    bump(L);
    return cudaGetLastError();
}

// dY <- dY * (Y > 0)   (ReLU backward through the stored post-activation)
__global__ void k_relu_bwd(size_t total, const float* __restrict__ yact, float* __restrict__ dy) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        if (!(yact[i] > 0.f)) dy[i] = 0.f;
}

cudaError_t relu_bwd(const Launch& L, size_t total, const float* yact, float* dy) {
    k_relu_bwd<<<(unsigned)std::min((total + 255) / 256, (size_t)4096), 256, 0, L.stream>>>(total, yact, dy);
    bump(L);
    return cudaGetLastError();
}

// Partial weight and bias gradients of one frame and one 16 x 16 tile:
//   dW[co][ci][tap] += sum_p dY[b][co][p] x[b][ci][p + tap],  db[co] += sum_p dY[b][co][p].
// Thread t owns the (co, ci) pairs t, t + 256, ...; partial sums go to
// part[block][Cout * Cin * 9 + Cout] and are reduced in a fixed order later.
__global__ void __launch_bounds__(kTile * kTile)
k_conv_wgrad(int Cin, int Cout, int n, const float* __restrict__ x, const float* __restrict__ dy,
             float* __restrict__ part) {
    extern __shared__ float sm[];
    float* xs = sm;                                         // [Cin][18][18]
    float* ds = sm + Cin * (kTile + 2) * (kTile + 2);       // [Cout][16][16]
    const int tiles = (n + kTile - 1) / kTile;
    const int tx0 = (blockIdx.x % tiles) * kTile, ty0 = (blockIdx.x / tiles) * kTile;
    const int b = blockIdx.y;
    const int tid = threadIdx.y * kTile + threadIdx.x;
    const float* xb = x + (size_t)b * Cin * n * n;
    const float* db = dy + (size_t)b * Cout * n * n;
    for (int i = tid; i < Cin * (kTile + 2) * (kTile + 2); i += kTile * kTile) {
        const int ci = i / ((kTile + 2) * (kTile + 2));
        const int rem = i - ci * (kTile + 2) * (kTile + 2);
        const int yy = ty0 + rem / (kTile + 2) - 1, xx = tx0 + rem % (kTile + 2) - 1;
        xs[i] = (yy >= 0 && yy < n && xx >= 0 && xx < n) ? __ldg(xb + ((size_t)ci * n + yy) * n + xx) : 0.f;
    }
    for (int i = tid; i < Cout * kTile * kTile; i += kTile * kTile) {
        const int co = i / (kTile * kTile), rem = i % (kTile * kTile);
        const int yy = ty0 + rem / kTile, xx = tx0 + rem % kTile;
        ds[i] = (yy < n && xx < n) ? __ldg(db + ((size_t)co * n + yy) * n + xx) : 0.f;
    }
    __syncthreads();
    const size_t stride = (size_t)Cout * Cin * 9 + Cout;
    float* out = part + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * stride;
    for (int pair = tid; pair < Cout * Cin; pair += kTile * kTile) {
        const int co = pair / Cin, ci = pair % Cin;
        float acc[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[t] = 0.f;
        const float* d = ds + co * kTile * kTile;
        const float* xc = xs + ci * (kTile + 2) * (kTile + 2);
        for (int py = 0; py < kTile; ++py)
            for (int px = 0; px < kTile; ++px) {
                const float g = d[py * kTile + px];
#pragma unroll
                for (int t = 0; t < 9; ++t) acc[t] = fmaf(g, xc[(py + t / 3) * (kTile + 2) + px + t % 3], acc[t]);
            }
#pragma unroll
        for (int t = 0; t < 9; ++t) out[((size_t)co * Cin + ci) * 9 + t] = acc[t];
    }
    for (int co = tid; co < Cout; co += kTile * kTile) {
        float a = 0.f;
        for (int i = 0; i < kTile * kTile; ++i) a += ds[co * kTile * kTile + i];
        out[(size_t)Cout * Cin * 9 + co] = a;
    }
}

// grad[j] = sum over blocks of part[block][j], in block order (deterministic)
__global__ void k_reduce_parts(int nblocks, int len, const float* __restrict__ part, float* __restrict__ grad) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= len) return;
    double a = 0.0;
    for (int k = 0; k < nblocks; ++k) a += part[(size_t)k * len + j];
    grad[j] = (float)a;
}

size_t conv_wgrad_parts(int B, int Cin, int Cout, int n) {
    const int tiles = (n + kTile - 1) / kTile;
    return (size_t)B * tiles * tiles * ((size_t)Cout * Cin * 9 + Cout);
}

cudaError_t conv_wgrad(const Launch& L, int B, int Cin, int Cout, int n, const float* x, const float* dy,
                       float* part, float* dW_db) {
    const int tiles = (n + kTile - 1) / kTile;
    const size_t smem = sizeof(float) * ((size_t)Cin * (kTile + 2) * (kTile + 2) + (size_t)Cout * kTile * kTile);
    if (Cin > kMaxC || Cout > kMaxC) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_conv_wgrad<<<dim3(tiles * tiles, B), dim3(kTile, kTile), smem, L.stream>>>(Cin, Cout, n, x, dy, part);
    bump(L);
    const int len = Cout * Cin * 9 + Cout;
    k_reduce_parts<<<(len + 255) / 256, 256, 0, L.stream>>>(B * tiles * tiles, len, part, dW_db);
    bump(L);
    return cudaGetLastError();
}

// Supervised loss on valid entries: L = sum (z - t)^2 / sum t^2 (per batch),
// dL/dz = 2 (z - t) / sum t^2.  Two passes: sums, then the gradient.
__global__ void k_loss_sums(size_t total, const float* __restrict__ z, const float* __restrict__ t,
                            double* __restrict__ sums) {
    __shared__ double r0[256], r1[256];
    double a = 0.0, c = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const double d = (double)z[i] - (double)t[i];
        a += d * d;
        c += (double)t[i] * t[i];
    }
    r0[threadIdx.x] = a;
    r1[threadIdx.x] = c;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            r0[threadIdx.x] += r0[threadIdx.x + s];
            r1[threadIdx.x] += r1[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sums[2 * blockIdx.x] = r0[0];
        sums[2 * blockIdx.x + 1] = r1[0];
    }
}

__global__ void k_loss_grad(size_t total, int nparts, const double* __restrict__ sums, const float* __restrict__ z,
                            const float* __restrict__ t, float* __restrict__ g, double* __restrict__ loss) {
    double den = 0.0, num = 0.0;
    for (int k = 0; k < nparts; ++k) {
        num += sums[2 * k];
        den += sums[2 * k + 1];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *loss = den > 0 ? num / den : 0.0;
    const float sc = den > 0 ? (float)(2.0 / den) : 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        g[i] = sc * (z[i] - t[i]);
}

cudaError_t loss_grad(const Launch& L, size_t total, const float* z, const float* t, double* sums, float* g,
                      double* loss) {
    const int nparts = 256;
    k_loss_sums<<<nparts, 256, 0, L.stream>>>(total, z, t, sums);
    bump(L);
    k_loss_grad<<<(unsigned)std::min((total + 255) / 256, (size_t)4096), 256, 0, L.stream>>>(total, nparts, sums, z, t, g,
                                                                                       loss);
    bump(L);
    return cudaGetLastError();
}

// Adam (Kingma & Ba, 2015) on the flat parameter vector.
__global__ void k_adam(int np, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

cudaError_t adam(const Launch& L, int np, float* w, const float* g, float* m, float* v, float lr, int step) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(np + 255) / 256, 256, 0, L.stream>>>(np, w, g, m, v, lr, b1, b2, 1e-8f, c1, c2);
    bump(L);
    return cudaGetLastError();
}

}  // namespace tomo
