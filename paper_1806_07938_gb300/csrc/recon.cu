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
