// Adjoint of the projection and the explicit reconstructor (kernels).
//
// The projection of Eq. SAap2 (with Eqs. mvm_ps / ToeplitzLGS and Eq. interp)
// is phi = sum_k I'_k Xi'_k zeta.  Its adjoint zeta' = sum_k Xi'_k^T I'_k^T phi
// runs the same FFT passes with the roles of input and output exchanged: the
// bilinear weights scatter phi back to the layer grids (I'_k^T, here a
// gather over a transposed table, so the sums have a fixed order), and the
// per-frequency blocks are the conjugate transposes of the projection's
// (a real generator's correlation is the conjugate spectrum of its
// convolution).
//
// The explicit reconstructor R = W_phi Sigma_phi_s (Sigma_ss + Sigma_eta_eta)^{-1}
// (Eq. covBasedReconstructors1, the "direct MVM" the paper compares the
// iterative method with, Sec. 4.B) is applied to slopes by an FP32 GEMM,
// phi[b][v] = sum_j R[v][j] s[b][j]: 64 x 64 output tiles, split over the
// reduction dimension into a fixed number of partial tiles that a second
// kernel adds in a fixed order (deterministic).
#include <algorithm>
#include <cstdint>

#include "kernels.cuh"

namespace tomo {

namespace {

inline void count(const Launch& L) {
    if (L.counter) ++*L.counter;
}

// out[f][k][node] = sum_{c in [ptr[k][node], ptr[k][node+1])} w[c] * phi[f][t][v[c]]
__global__ void k_interp_adjoint(int T_all, int t, int n_layers, int m2, int n_vphi, const int* __restrict__ ptr,
                                 const int* __restrict__ vi, const float* __restrict__ w,
                                 const float* __restrict__ phi, float* __restrict__ out) {
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y, f = blockIdx.z;
    if (node >= m2) return;
    const int* p = ptr + (size_t)k * (m2 + 1);
    const float* ph = phi + ((size_t)f * T_all + t) * n_vphi;
    float acc = 0.f;
    for (int c = p[node]; c < p[node + 1]; ++c) acc += w[c] * ph[vi[c]];
    out[((size_t)f * n_layers + k) * m2 + node] = acc;
}

// Kadj[kx][p][ky][q] = conj(K[kx][q][ky][p]), K with NPin = nq, NPout = np planes
__global__ void k_adjoint_spectra(int nh, int P, int nq, int np, const float2* __restrict__ K,
                                  float2* __restrict__ Kadj) {
    const size_t total = (size_t)nh * nq * P * np;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        size_t r = i;
        const int p = (int)(r % np); r /= np;
        const int ky = (int)(r % P); r /= P;
        const int q = (int)(r % nq); r /= nq;
        const int kx = (int)r;
        const float2 v = K[i];
        Kadj[(((size_t)kx * np + p) * P + ky) * nq + q] = make_float2(v.x, -v.y);
    }
}

// phi[f][t][v] = 1 if v == v0 + f, else 0 (f < B), for the columns of R^T
__global__ void k_unit_phase(int B, int T_all, int t, int n_vphi, int v0, float* __restrict__ phi) {
    const size_t total = (size_t)B * T_all * n_vphi;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int v = (int)(i % n_vphi);
        const size_t ft = i / n_vphi;
        const int tt = (int)(ft % T_all), f = (int)(ft / T_all);
        phi[i] = (tt == t && v == v0 + f) ? 1.f : 0.f;
    }
}

constexpr int kTile = 64, kKStep = 16, kGemmThreads = 256;

// Partial tile of C = A B^T over the reduction range of this split:
// A [M][K] row-major (lda), B [N][K] row-major (ldb); part [split][M][N].
__global__ void __launch_bounds__(kGemmThreads)
k_gemm_nt_part(int M, int N, int K, int kchunk, const float* __restrict__ A, int lda, const float* __restrict__ Bm,
               int ldb, float* __restrict__ part) {
    __shared__ __align__(16) float As[kKStep][kTile + 4];   // row of 68 floats: 16-byte aligned rows
    __shared__ __align__(16) float Bs[kKStep][kTile + 4];
    const int n0 = blockIdx.x * kTile, m0 = blockIdx.y * kTile;
    const int k_begin = blockIdx.z * kchunk;
    const int k_end = min(K, k_begin + kchunk);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;    // 16 x 16 threads, 4 x 4 outputs each
    float acc[4][4] = {};
    // loader: each thread moves 4 consecutive k of one row of each tile
    const int lr = threadIdx.x / 4, lk = (threadIdx.x % 4) * 4;
    for (int k0 = k_begin; k0 < k_end; k0 += kKStep) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = k0 + lk + u;
            const int am = m0 + lr, bn = n0 + lr;
            As[lk + u][lr] = (am < M && k < k_end) ? A[(size_t)am * lda + k] : 0.f;
            Bs[lk + u][lr] = (bn < N && k < k_end) ? Bm[(size_t)bn * ldb + k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kKStep; ++kk) {
            const float4 av = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
            const float4 bv = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
            const float a[4] = {av.x, av.y, av.z, av.w};
            const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float* out = part + (size_t)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n < N) out[(size_t)m * N + n] = acc[i][j];
        }
    }
}

// C[m][n] (row stride ldc) = sum over the splits in order
__global__ void k_gemm_reduce(int M, int N, int splits, const float* __restrict__ part, float* __restrict__ C,
                              int ldc) {
    const size_t total = (size_t)M * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[(size_t)z * total + i];
        C[(i / N) * (size_t)ldc + i % N] = s;
    }
}

// sumF[j] += sum_b F[b][j], sumX[j] += sum_b X[b][j] (FP64, rows in order)
__global__ void k_col_sums(int B, int N, const float* __restrict__ F, const float* __restrict__ X,
                           double* __restrict__ sumF, double* __restrict__ sumX) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        double a = sumF[j], b = sumX[j];
        for (int r = 0; r < B; ++r) {
            a += (double)F[(size_t)r * N + j];
            b += (double)X[(size_t)r * N + j];
        }
        sumF[j] = a;
        sumX[j] = b;
    }
}

// dots[b] = sum_j F[b][j] X[b][j] (FP64), one block per row
__global__ void k_row_dots(int N, const float* __restrict__ F, const float* __restrict__ X, double* __restrict__ dots) {
    __shared__ double red[8];
    const int b = blockIdx.x;
    double acc = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) acc += (double)F[(size_t)b * N + j] * (double)X[(size_t)b * N + j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        dots[b] = t;
    }
}

}  // namespace

cudaError_t wfe_accumulate(const Launch& L, int B, int N, const float* F, const float* X, double* dots, double* sumF,
                           double* sumX) {
    if (B <= 0) return cudaSuccess;
    k_row_dots<<<B, 256, 0, L.stream>>>(N, F, X, dots);
    count(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_col_sums<<<(N + 255) / 256, 256, 0, L.stream>>>(B, N, F, X, sumF, sumX);
    count(L);
    return cudaGetLastError();
}

cudaError_t interp_adjoint(const Launch& L, int B, int T_all, int t, int n_layers, int m, int n_vphi,
                           const int* ptr, const int* vi, const float* w, const float* phi, float* out) {
    if (B <= 0) return cudaSuccess;
    const int m2 = m * m;
    k_interp_adjoint<<<dim3((m2 + 255) / 256, n_layers, B), 256, 0, L.stream>>>(T_all, t, n_layers, m2, n_vphi, ptr,
                                                                              vi, w, phi, out);
    count(L);
    return cudaGetLastError();
}

cudaError_t adjoint_spectra(const Launch& L, int nh, int P, int nq, int np, const float2* K, float2* Kadj) {
    k_adjoint_spectra<<<1216, 256, 0, L.stream>>>(nh, P, nq, np, K, Kadj);
    count(L);
    return cudaGetLastError();
}

cudaError_t unit_phase(const Launch& L, int B, int T_all, int t, int n_vphi, int v0, float* phi) {
    k_unit_phase<<<1216, 256, 0, L.stream>>>(B, T_all, t, n_vphi, v0, phi);
    count(L);
    return cudaGetLastError();
}

size_t gemm_nt_workspace(int M, int N, int splits) { return (size_t)splits * M * N; }

cudaError_t gemm_nt(const Launch& L, int M, int N, int K, const float* A, int lda, const float* Bm, int ldb, float* C,
                    int ldc, int splits, float* part) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (splits < 1 || K < 1) return cudaErrorInvalidValue;
    int kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + kKStep - 1) / kKStep * kKStep;
    const dim3 grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile, splits);
    k_gemm_nt_part<<<grid, kGemmThreads, 0, L.stream>>>(M, N, K, kchunk, A, lda, Bm, ldb, part);
    count(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gemm_reduce<<<1216, 256, 0, L.stream>>>(M, N, splits, part, C, ldc);
    count(L);
    return cudaGetLastError();
}

}  // namespace tomo

// ---------------------------------------------------------------------------
// Block conjugate gradients over the frames of a batch (all frames share the
// operator, so one Krylov space serves them all): the tall-skinny products
// of the block recurrences.  Vectors are [B][N] (frame-major), B <= 64.
// ---------------------------------------------------------------------------
namespace tomo {

namespace {

constexpr int kBlockMax = 64;

// Partial Gram tiles out[block][i][j] = sum over the block's columns of
// U[i][k] V[j][k]: the block walks chunks of 64 columns (grid-strided), loads
// each chunk of U and V with coalesced row reads into shared memory
// (transposed), sums the chunk's 64 products in FP32 and adds them to FP64
// accumulators, 4 x 4 outputs per thread.
constexpr int kGramChunk = 64;

__global__ void __launch_bounds__(256)
k_gram_part(int B, int N, const float* __restrict__ U, const float* __restrict__ V, double* __restrict__ part) {
    __shared__ __align__(16) float Us[kGramChunk][kBlockMax + 4];
    __shared__ __align__(16) float Vs[kGramChunk][kBlockMax + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    const int nchunks = (N + kGramChunk - 1) / kGramChunk;
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int k0 = ch * kGramChunk;
        for (int idx = threadIdx.x; idx < kBlockMax * kGramChunk; idx += blockDim.x) {
            const int row = idx / kGramChunk, col = idx % kGramChunk, k = k0 + col;
            const bool ok = row < B && k < N;
            Us[col][row] = ok ? U[(size_t)row * N + k] : 0.f;
            Vs[col][row] = ok ? V[(size_t)row * N + k] : 0.f;
        }
        __syncthreads();
        float a32[4][4] = {};
#pragma unroll 8
        for (int kk = 0; kk < kGramChunk; ++kk) {
            const float4 av = *reinterpret_cast<const float4*>(&Us[kk][ty * 4]);
            const float4 bv = *reinterpret_cast<const float4*>(&Vs[kk][tx * 4]);
            const float a[4] = {av.x, av.y, av.z, av.w};
            const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) a32[i][j] = fmaf(a[i], b[j], a32[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += (double)a32[i][j];
        __syncthreads();
    }
    double* out = part + (size_t)blockIdx.x * kBlockMax * kBlockMax;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * kBlockMax + tx * 4 + j] = acc[i][j];
}

// G[i][j] = sum over the partial tiles: a block of 256 threads serves 32
// entries; warp t sums tiles t, t + 8, t + 16, ... of its lane's entry
// (coalesced across the warp), and all sums are added in a fixed order.
__global__ void __launch_bounds__(256)
k_gram_reduce(int B, int splits, const double* __restrict__ part, double* __restrict__ G) {
    __shared__ double red[8][32];
    const int t = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int e = blockIdx.x * 32 + lane;
    // four independent running sums (tiles t, t + 8, t + 16, t + 24 of each
    // group of 32), so that four loads are in flight per thread
    double s4[4] = {0.0, 0.0, 0.0, 0.0};
    int z = t;
    for (; z + 24 < splits; z += 32)
#pragma unroll
        for (int u = 0; u < 4; ++u) s4[u] += part[(size_t)(z + 8 * u) * kBlockMax * kBlockMax + e];
#pragma unroll
    for (int u = 0; u < 3; ++u)
        if (z + 8 * u < splits) s4[u] += part[(size_t)(z + 8 * u) * kBlockMax * kBlockMax + e];
    red[t][lane] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    __syncthreads();
    if (t == 0) {
        const double v = ((red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane])) +
                         ((red[4][lane] + red[5][lane]) + (red[6][lane] + red[7][lane]));
        const int i = e / kBlockMax, j = e % kBlockMax;
        if (i < B && j < B) G[i * B + j] = v;
    }
}

// Y[j][k] = (Y0 ? Y0[j][k] : 0) + sum_i C[i][j] U[i][k], one thread per column
// k, four outputs at a time (independent sums).
__global__ void __launch_bounds__(128)
k_block_combine(int B, int N, const double* __restrict__ C, double scale, const float* __restrict__ U,
                const float* Y0, float* Y) {
    // C padded to 64 x 64 with zeros, so that the unrolled sums below add
    // exact zeros for i >= B
    __shared__ __align__(16) float Cs[kBlockMax * kBlockMax];   // read as float4
    for (int t = threadIdx.x; t < kBlockMax * kBlockMax; t += blockDim.x) {
        const int i = t / kBlockMax, j = t % kBlockMax;
        Cs[t] = (i < B && j < B) ? (float)(scale * C[i * B + j]) : 0.f;
    }
    __syncthreads();
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        float u[kBlockMax];
#pragma unroll
        for (int i = 0; i < kBlockMax; ++i) u[i] = i < B ? U[(size_t)i * N + k] : 0.f;
        for (int j0 = 0; j0 < B; j0 += 4) {
            float y[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) y[q] = (Y0 && j0 + q < B) ? Y0[(size_t)(j0 + q) * N + k] : 0.f;
#pragma unroll
            for (int i = 0; i < kBlockMax; ++i) {
                const float4 c = *reinterpret_cast<const float4*>(&Cs[i * kBlockMax + j0]);
                y[0] = fmaf(c.x, u[i], y[0]);
                y[1] = fmaf(c.y, u[i], y[1]);
                y[2] = fmaf(c.z, u[i], y[2]);
                y[3] = fmaf(c.w, u[i], y[3]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j0 + q < B) Y[(size_t)(j0 + q) * N + k] = y[q];
        }
    }
}

// Y = scale * T (T^T X) for B x B FP64 matrices (row-major): one block per
// column j of Y, one thread per row.  The inner product T^T X[:, j] is kept
// in shared memory; both sums run over k in ascending order.
__global__ void k_gram_apply(int B, const double* __restrict__ T, const double* __restrict__ X,
                             double* __restrict__ Y, double scale) {
    __shared__ double w[kBlockMax];
    const int j = blockIdx.x, i = threadIdx.x;
    if (i < B) {
        double acc = 0.0;
#pragma unroll 8
        for (int k = 0; k < B; ++k) acc += T[k * B + i] * X[k * B + j];
        w[i] = acc;
    }
    __syncthreads();
    if (i < B) {
        double acc = 0.0;
#pragma unroll 8
        for (int k = 0; k < B; ++k) acc += T[i * B + k] * w[k];
        Y[i * B + j] = scale * acc;
    }
}

// Y[j][k] = f[j] X[j][k] (per-row scale; Y may alias X)
__global__ void k_scale_rows(int B, int N, const double* __restrict__ f, const float* X, float* Y) {
    const int j = blockIdx.y;
    const float a = (float)f[j];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x)
        Y[(size_t)j * N + k] = a * X[(size_t)j * N + k];
}

// out[j][s] = sum over the s-th of S column slices of X[j][k]^2
__global__ void k_row_norms(int N, int S, const float* __restrict__ X, double* __restrict__ out) {
    __shared__ double red[8];
    const int b = blockIdx.x, sl = blockIdx.y;
    const int k0 = (int)((long long)N * sl / S), k1 = (int)((long long)N * (sl + 1) / S);
    // FP32 per-thread partials (a few tens of squares), FP64 from the warp sums
    // on (GB300's FP64 rate is ~1/64 of its FP32 rate)
    float a32 = 0.f;
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const float v = X[(size_t)b * N + k];
        a32 = fmaf(v, v, a32);
    }
    double acc = a32;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[(size_t)b * S + sl] = t;
    }
}

inline void count2(const Launch& L) {
    if (L.counter) ++*L.counter;
}

// --- register-tiled forms (N a multiple of 4, 16-byte aligned rows) ---------------
// Partial Gram tiles as k_gram_part, with the block's column range walked in
// sub-chunks of 32 columns: the next sub-chunk is loaded into registers (two
// float4 per matrix and thread) while the current one is multiplied; the
// transposed shared-memory tiles use an XOR swizzle of the float4 index (gswz)
// so that the transposed stores are free of bank conflicts and the reads stay
// float4;
// each output's per-sub-chunk FP32 sums (32 products) are accumulated with
// Knuth's TwoSum (error-free) instead of FP64 additions (GB300's FP64 rate is
// ~1/64 of its FP32 rate), and converted to FP64 once.
constexpr int kSub = 32;

// Float4 slot of row group g (rows 4g .. 4g + 3) in column col of a
// transposed tile: g XOR a key of the column.  The loader of a warp writes,
// per store, 8 rows x 4 columns 8 apart; the key takes 4 distinct even values
// mod 8 over those columns, so the 32 stores hit 32 distinct banks.
__device__ __forceinline__ int gkey(int col) { return (col & 7) ^ ((col >> 3) << 1); }
__device__ __forceinline__ int gswz(int col, int row) { return (((row >> 2) ^ gkey(col)) << 2) | (row & 3); }

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
    const float u = hi + x;
    const float bp = u - hi;
    lo += (hi - (u - bp)) + (x - bp);
    hi = u;
}

__global__ void __launch_bounds__(256, 2)
k_gram_part4(int B, int N, const float* __restrict__ U, const float* __restrict__ V, double* __restrict__ part) {
    __shared__ __align__(16) float Us[2][kSub][kBlockMax];
    __shared__ __align__(16) float Vs[2][kSub][kBlockMax];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    // this block's column range, in whole sub-chunks
    const int nsub = (N + kSub - 1) / kSub;
    const int s0 = (int)((long long)nsub * blockIdx.x / gridDim.x);
    const int s1 = (int)((long long)nsub * (blockIdx.x + 1) / gridDim.x);
    // loader: row lr, columns lc .. lc + 7 of a sub-chunk
    const int lr = threadIdx.x / 4, lc = (threadIdx.x % 4) * 8;
    float4 ua[2], va[2];
    auto load = [&](int sc) {
        const int k = sc * kSub + lc;
        const bool okr = lr < B;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int kk = k + 4 * h;
            if (okr && kk + 3 < N) {
                ua[h] = __ldg(reinterpret_cast<const float4*>(U + (size_t)lr * N + kk));
                va[h] = __ldg(reinterpret_cast<const float4*>(V + (size_t)lr * N + kk));
            } else {
                float a[4], b[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    a[c] = okr && kk + c < N ? U[(size_t)lr * N + kk + c] : 0.f;
                    b[c] = okr && kk + c < N ? V[(size_t)lr * N + kk + c] : 0.f;
                }
                ua[h] = make_float4(a[0], a[1], a[2], a[3]);
                va[h] = make_float4(b[0], b[1], b[2], b[3]);
            }
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float a[4] = {ua[h].x, ua[h].y, ua[h].z, ua[h].w};
            const float b[4] = {va[h].x, va[h].y, va[h].z, va[h].w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int col = lc + 4 * h + c;
                Us[buf][col][gswz(col, lr)] = a[c];
                Vs[buf][col][gswz(col, lr)] = b[c];
            }
        }
    };
    float hi[4][4] = {}, lo[4][4] = {};
    if (s0 < s1) {
        load(s0);
        store(0);
    }
    __syncthreads();
    for (int sc = s0; sc < s1; ++sc) {
        const int buf = (sc - s0) & 1;
        if (sc + 1 < s1) load(sc + 1);
        float a32[4][4] = {};
#pragma unroll 8
        for (int kk = 0; kk < kSub; ++kk) {
            const float4 av = *reinterpret_cast<const float4*>(&Us[buf][kk][(ty ^ gkey(kk)) << 2]);
            const float4 bv = *reinterpret_cast<const float4*>(&Vs[buf][kk][(tx ^ gkey(kk)) << 2]);
            const float a[4] = {av.x, av.y, av.z, av.w};
            const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) a32[i][j] = fmaf(a[i], b[j], a32[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) two_sum_acc(hi[i][j], lo[i][j], a32[i][j]);
        if (sc + 1 < s1) store(buf ^ 1);
        __syncthreads();
    }
    double* out = part + (size_t)blockIdx.x * kBlockMax * kBlockMax;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            out[(ty * 4 + i) * kBlockMax + tx * 4 + j] = (double)hi[i][j] + (double)lo[i][j];
}

// Y[j][k] = Y0[j][k] + sum_i C[i][j] U[i][k] as a tiled product: a block owns
// 128 columns k and all 64 j; thread (tk, tj) computes k = 4 tk .. 4 tk + 3 and
// j = 8 tj .. 8 tj + 7; per i one float4 of U (the warp reads 512 contiguous
// bytes) and two float4 broadcasts of C feed 32 FMAs.
constexpr int kCombK = 128;

__global__ void __launch_bounds__(256)
k_block_combine4(int B, int N, const double* __restrict__ C, double scale, const float* __restrict__ U,
                 const float* Y0, float* Y) {
    __shared__ __align__(16) float Us[kBlockMax][kCombK];
    __shared__ __align__(16) float Cs[kBlockMax][kBlockMax];
    const int k0 = blockIdx.x * kCombK;
    for (int t = threadIdx.x; t < kBlockMax * kBlockMax; t += blockDim.x) {
        const int i = t / kBlockMax, j = t % kBlockMax;
        Cs[i][j] = (i < B && j < B) ? (float)(scale * C[i * B + j]) : 0.f;
    }
    for (int t = threadIdx.x; t < kBlockMax * (kCombK / 4); t += blockDim.x) {
        const int i = t / (kCombK / 4), c4 = t % (kCombK / 4), k = k0 + 4 * c4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < B) {
            if (k + 3 < N) {
                v = __ldg(reinterpret_cast<const float4*>(U + (size_t)i * N + k));
            } else {
                float a[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) a[c] = k + c < N ? U[(size_t)i * N + k + c] : 0.f;
                v = make_float4(a[0], a[1], a[2], a[3]);
            }
        }
        *reinterpret_cast<float4*>(&Us[i][4 * c4]) = v;
    }
    __syncthreads();
    const int tk = threadIdx.x % 32, tj = threadIdx.x / 32;
    float acc[8][4] = {};
    const int ib = B < kBlockMax ? B : kBlockMax;
#pragma unroll 4
    for (int i = 0; i < ib; ++i) {
        const float4 u = *reinterpret_cast<const float4*>(&Us[i][4 * tk]);
        const float4 c0 = *reinterpret_cast<const float4*>(&Cs[i][8 * tj]);
        const float4 c1 = *reinterpret_cast<const float4*>(&Cs[i][8 * tj + 4]);
        const float cc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
        const float uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[jj][q] = fmaf(cc[jj], uu[q], acc[jj][q]);
    }
    const int k = k0 + 4 * tk;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        const int j = 8 * tj + jj;
        if (j >= B) continue;
        float o[4] = {acc[jj][0], acc[jj][1], acc[jj][2], acc[jj][3]};
        if (k + 3 < N) {
            if (Y0) {
                const float4 y0 = *reinterpret_cast<const float4*>(Y0 + (size_t)j * N + k);
                o[0] += y0.x;
                o[1] += y0.y;
                o[2] += y0.z;
                o[3] += y0.w;
            }
            *reinterpret_cast<float4*>(Y + (size_t)j * N + k) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
            for (int q = 0; q < 4; ++q)
                if (k + q < N) Y[(size_t)j * N + k + q] = o[q] + (Y0 ? Y0[(size_t)j * N + k + q] : 0.f);
        }
    }
}

bool tiled_ok(int N, const void* a, const void* b, const void* c) {
    auto al = [](const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    return (N & 3) == 0 && al(a) && al(b) && al(c);
}

}  // namespace

constexpr int kGramBlocks = 2 * 152;

size_t gram_workspace(int /*N*/) { return (size_t)kGramBlocks * kBlockMax * kBlockMax; }

cudaError_t gram(const Launch& L, int B, int N, const float* U, const float* V, double* G, double* part) {
    if (B < 1 || B > kBlockMax || N < 1) return cudaErrorInvalidValue;
    const int nchunks = (N + kGramChunk - 1) / kGramChunk;
    const int blocks = std::min(kGramBlocks, nchunks);
    if (tiled_ok(N, U, V, nullptr)) k_gram_part4<<<blocks, 256, 0, L.stream>>>(B, N, U, V, part);
    else k_gram_part<<<blocks, 256, 0, L.stream>>>(B, N, U, V, part);
    count2(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gram_reduce<<<kBlockMax * kBlockMax / 32, 256, 0, L.stream>>>(B, blocks, part, G);
    count2(L);
    return cudaGetLastError();
}

cudaError_t block_combine(const Launch& L, int B, int N, const double* C, const float* U, const float* Y0, float* Y,
                          double scale) {
    if (B < 1 || B > kBlockMax) return cudaErrorInvalidValue;
    if (tiled_ok(N, U, Y0, Y)) {
        // the tiled form reads Y0 and writes Y per element: they may alias (x += P alpha)
        k_block_combine4<<<(N + kCombK - 1) / kCombK, 256, 0, L.stream>>>(B, N, C, scale, U, Y0, Y);
        count2(L);
        return cudaGetLastError();
    }
    const int blocks = (N + 127) / 128;
    k_block_combine<<<blocks, 128, 0, L.stream>>>(B, N, C, scale, U, Y0, Y);
    count2(L);
    return cudaGetLastError();
}

cudaError_t gram_apply(const Launch& L, int B, const double* T, const double* X, double* Y, double scale) {
    if (B < 1 || B > kBlockMax) return cudaErrorInvalidValue;
    k_gram_apply<<<B, kBlockMax, 0, L.stream>>>(B, T, X, Y, scale);
    count2(L);
    return cudaGetLastError();
}

cudaError_t scale_rows(const Launch& L, int B, int N, const double* f, const float* X, float* Y) {
    if (B <= 0) return cudaSuccess;
    k_scale_rows<<<dim3((N + 1023) / 1024, B), 256, 0, L.stream>>>(B, N, f, X, Y);
    count2(L);
    return cudaGetLastError();
}

cudaError_t row_norms(const Launch& L, int B, int N, const float* X, double* out, int slices) {
    if (B <= 0) return cudaSuccess;
    if (slices < 1) return cudaErrorInvalidValue;
    k_row_norms<<<dim3(B, slices), 256, 0, L.stream>>>(N, slices, X, out);
    count2(L);
    return cudaGetLastError();
}

}  // namespace tomo
