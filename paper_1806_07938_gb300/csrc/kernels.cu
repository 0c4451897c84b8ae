// Device kernels of the Toeplitz-structured tomographic reconstructor.
//
// Sigma_ss zeta (Eq. mvm_ss) and Sigma_phi_s zeta (Eqs. mvm_ps, ToeplitzLGS)
// are evaluated as 2-D periodic convolutions on a P x P grid (the 2-D form of
// the 2RBT MVM of Sec. 2.E; see the host file for the index mapping).  Three
// passes per product:
//   rows_fwd : scatter the valid entries of each input plane into its rows
//              (W_s^T), real FFT of the non-zero rows, two rows per complex
//              FFT, result stored column-major [plane][kx][row];
//   cols_mul : per frequency column kx, forward FFT along y of every input
//              plane, the (NPout x NPin) complex block multiply
//              y~_p = sum_q K_pq x~_q (the element-wise products of Eq. mvm_ss
//              summed before the inverse transform), inverse FFT along y,
//              keep the rows that survive the crop;
//   rows_inv : inverse real FFT of the kept rows, crop, gather the valid
//              outputs (W_s), add the diagonal noise term of Eq. SAap1.
// The 1/P^2 of the inverse transform is folded into the spectra K.
#include <cfloat>
#include <cmath>

#include "kernels.cuh"

namespace tomo {

namespace {

inline void count(const Launch& L) {
    if (L.counter) ++*L.counter;
}

int g_max_smem = 48 * 1024;   // raised by init_kernel_attributes()

template <typename T>
__device__ __forceinline__ double block_sum(double v, double* red) {
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

// ---------------------------------------------------------------------------
// Row-forward pass
// ---------------------------------------------------------------------------
template <typename T, typename TIn>
__global__ void __launch_bounds__(kThreads)
k_rows_fwd(MvmGeom g, MaskTables mt, const TIn* __restrict__ x, TIn* p, const FrameState* st,
           cplx_t<T>* __restrict__ X1T, const cplx_t<T>* __restrict__ twg) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = g.plan.P, n = g.n, nh = g.nh;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* wbuf = tw + P;
    C* S = wbuf + kWarps * 2 * P;
    const int q = blockIdx.x, f = blockIdx.y;
    if (st && !st[f].active) return;
    for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t vbase = ((size_t)f * g.NPin + q) * mt.n_vs;
    const TIn* xv = x + vbase;
    TIn* pv = p ? p + vbase : nullptr;
    const TIn beta = (p && st) ? (TIn)st[f].beta : (TIn)0;
    __syncthreads();
    C* buf = wbuf + warp * 2 * P;
    C* scr = buf + P;
    for (int r = 2 * warp; r < n; r += 2 * kWarps) {
        for (int j = lane; j < P; j += 32) buf[j] = cmk<C>(0, 0);
        __syncwarp();
        for (int h = 0; h < 2 && r + h < n; ++h) {
            const int e0 = mt.rowstart[r + h], e1 = mt.rowstart[r + h + 1];
            for (int e = e0 + lane; e < e1; e += 32) {
                T v;
                if (pv) {
                    const TIn pn = xv[e] + beta * pv[e];
                    pv[e] = pn;
                    v = (T)pn;
                } else {
                    v = (T)xv[e];
                }
                const int c = mt.col[e];
                if (h == 0) buf[c].x = v; else buf[c].y = v;
            }
        }
        __syncwarp();
        fft_warp<C>(buf, scr, g.plan, tw, true, lane, 32);
        // two real spectra from one complex one: A = (Z_k + conj Z_{P-k})/2, B = (Z_k - conj Z_{P-k})/(2i)
        for (int k = lane; k < nh; k += 32) {
            const C zk = buf[k];
            const C zc = cconj(buf[k == 0 ? 0 : P - k]);
            const C a = cscale(cadd(zk, zc), (T)0.5);
            const C dd = csub(zk, zc);
            S[k * n + r] = a;
            if (r + 1 < n) S[k * n + r + 1] = cmk<C>((T)0.5 * dd.y, (T)-0.5 * dd.x);
        }
        __syncwarp();
    }
    __syncthreads();
    C* out = X1T + ((size_t)f * g.NPin + q) * nh * n;
    for (int i = threadIdx.x; i < nh * n; i += blockDim.x) out[i] = S[i];
}

template <typename T, typename TIn>
cudaError_t rows_fwd(const Launch& L, const MvmGeom& g, const MaskTables& mt, int B, const TIn* x, TIn* p,
                     const FrameState* st, cplx_t<T>* X1T, const cplx_t<T>* tw) {
    using C = cplx_t<T>;
    const size_t smem = sizeof(C) * ((size_t)g.plan.P * (1 + 2 * kWarps) + (size_t)g.nh * g.n);
    auto kern = k_rows_fwd<T, TIn>;
    if (smem > (size_t)g_max_smem) return cudaErrorInvalidValue;
    kern<<<dim3(g.NPin, B), kThreads, smem, L.stream>>>(g, mt, x, p, st, X1T, tw);
    count(L);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Column pass with the per-frequency block multiply
// ---------------------------------------------------------------------------
// Per-frequency block product of Eq. mvm_ss for one column kx:
//   y_p(ky) = sum_q K_pq(kx, ky) x_q(ky)   for every frame of the block,
// in place in the column buffer D [frame][plane][ky].  K is stored
// [kx][q][ky][p], so the threads of a round, one per (ky, p), read it fully
// coalesced; each holds its row K_p.(ky) in registers and reads the x_q(ky)
// as shared-memory broadcasts.  Results are held in registers until every
// thread of the round has read its inputs.
constexpr int kMaxFramesPerBlock = 8;

template <typename C, int NPI, int NPO>
__device__ __forceinline__ void block_mul(C* D, int NPmax, int P, int nf, const int* act, const C* __restrict__ Kc) {
    using T = decltype(C::x);
    const int kyr = blockDim.x / NPO;                 // ky values per round
    const int kyl = threadIdx.x / NPO, pp = threadIdx.x % NPO;
    for (int ky0 = 0; ky0 < P; ky0 += kyr) {
        const int ky = ky0 + kyl;
        const bool on = kyl < kyr && ky < P;
        C k[NPI];
        C y[kMaxFramesPerBlock];
        if (on) {
#pragma unroll
            for (int q = 0; q < NPI; ++q) k[q] = __ldg(&Kc[((size_t)q * P + ky) * NPO + pp]);
#pragma unroll
            for (int fl = 0; fl < kMaxFramesPerBlock; ++fl) {
                if (fl < nf && act[fl]) {
                    const C* col = D + (size_t)fl * NPmax * P + ky;
                    T ar = 0, ai = 0;
#pragma unroll
                    for (int q = 0; q < NPI; ++q) {
                        const C x = col[q * P];
                        ar = fma(k[q].x, x.x, ar);
                        ar = fma(-k[q].y, x.y, ar);
                        ai = fma(k[q].x, x.y, ai);
                        ai = fma(k[q].y, x.x, ai);
                    }
                    y[fl] = cmk<C>(ar, ai);
                }
            }
        }
        __syncthreads();
        if (on) {
#pragma unroll
            for (int fl = 0; fl < kMaxFramesPerBlock; ++fl)
                if (fl < nf && act[fl]) D[((size_t)fl * NPmax + pp) * P + ky] = y[fl];
        }
        __syncthreads();
    }
}

template <typename C>
__device__ void block_mul_rt(C* D, int NPmax, int P, int nf, const int* act, const C* __restrict__ Kc, int NPin,
                             int NPout) {
    using T = decltype(C::x);
    const int kyr = blockDim.x / NPout;
    const int kyl = threadIdx.x / NPout, pp = threadIdx.x % NPout;
    for (int ky0 = 0; ky0 < P; ky0 += kyr) {
        const int ky = ky0 + kyl;
        const bool on = kyl < kyr && ky < P;
        C y[kMaxFramesPerBlock];
        if (on) {
            for (int fl = 0; fl < nf; ++fl) {
                if (!act[fl]) continue;
                const C* col = D + (size_t)fl * NPmax * P + ky;
                T ar = 0, ai = 0;
                for (int q = 0; q < NPin; ++q) {
                    const C kq = Kc[((size_t)q * P + ky) * NPout + pp];
                    const C x = col[q * P];
                    ar += kq.x * x.x - kq.y * x.y;
                    ai += kq.x * x.y + kq.y * x.x;
                }
                y[fl] = cmk<C>(ar, ai);
            }
        }
        __syncthreads();
        if (on)
            for (int fl = 0; fl < nf; ++fl)
                if (act[fl]) D[((size_t)fl * NPmax + pp) * P + ky] = y[fl];
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_cols_mul(MvmGeom g, int B, int Bc, const FrameState* st, const cplx_t<T>* __restrict__ X1T,
           cplx_t<T>* __restrict__ Y1T, const cplx_t<T>* __restrict__ K, const cplx_t<T>* __restrict__ twg) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = g.plan.P, n = g.n, m = g.m, nh = g.nh, NPin = g.NPin, NPout = g.NPout;
    const int NPmax = NPin > NPout ? NPin : NPout;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* scr = tw + P;
    C* D = scr + kWarps * P;                       // [Bc][NPmax][P]
    __shared__ int act[kMaxFramesPerBlock];
    const int kx = blockIdx.x;
    const int f0 = blockIdx.y * Bc;
    const int nf = min(Bc, B - f0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) act[i] = st ? st[f0 + i].active : 1;
    __syncthreads();
    // load the columns (rows >= n are the zero padding)
    for (int i = threadIdx.x; i < nf * NPin * P; i += blockDim.x) {
        const int r = i % P, t = i / P, q = t % NPin, fl = t / NPin;
        C v = cmk<C>(0, 0);
        if (r < n && act[fl]) v = X1T[(((size_t)(f0 + fl) * NPin + q) * nh + kx) * n + r];
        D[((size_t)fl * NPmax + q) * P + r] = v;
    }
    __syncthreads();
    for (int t = warp; t < nf * NPin; t += kWarps) {
        const int fl = t / NPin, q = t % NPin;
        if (act[fl]) fft_warp<C>(D + ((size_t)fl * NPmax + q) * P, scr + warp * P, g.plan, tw, true, lane, 32);
    }
    __syncthreads();
    // block multiply: one thread per (ky, frame), frames fastest so K loads broadcast
    const C* Kc = K + (size_t)kx * NPin * P * NPout;
    if (NPin == 12 && NPout == 12) block_mul<C, 12, 12>(D, NPmax, P, nf, act, Kc);
    else if (NPin == 6 && NPout == 6) block_mul<C, 6, 6>(D, NPmax, P, nf, act, Kc);
    else if (NPin == 4 && NPout == 4) block_mul<C, 4, 4>(D, NPmax, P, nf, act, Kc);
    else if (NPin == 2 && NPout == 2) block_mul<C, 2, 2>(D, NPmax, P, nf, act, Kc);
    else block_mul_rt<C>(D, NPmax, P, nf, act, Kc, NPin, NPout);
    for (int t = warp; t < nf * NPout; t += kWarps) {
        const int fl = t / NPout, pp = t % NPout;
        if (act[fl]) fft_warp<C>(D + ((size_t)fl * NPmax + pp) * P, scr + warp * P, g.plan, tw, false, lane, 32);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nf * NPout * m; i += blockDim.x) {
        const int r = i % m, t = i / m, pp = t % NPout, fl = t / NPout;
        if (act[fl]) Y1T[(((size_t)(f0 + fl) * NPout + pp) * nh + kx) * m + r] = D[((size_t)fl * NPmax + pp) * P + r];
    }
}

template <typename T>
cudaError_t cols_mul(const Launch& L, const MvmGeom& g, int B, const FrameState* st, const cplx_t<T>* X1T,
                     cplx_t<T>* Y1T, const cplx_t<T>* K, const cplx_t<T>* tw) {
    using C = cplx_t<T>;
    if (g.NPin > 16) return cudaErrorInvalidValue;
    const int NPmax = g.NPin > g.NPout ? g.NPin : g.NPout;
    const size_t fixed = sizeof(C) * (size_t)g.plan.P * (1 + kWarps);
    const size_t per_frame = sizeof(C) * (size_t)NPmax * g.plan.P;
    const size_t budget = 72 * 1024;
    int Bc = (int)((budget > fixed ? budget - fixed : 0) / per_frame);
    if (Bc < 1) Bc = 1;
    if (Bc > kMaxFramesPerBlock) Bc = kMaxFramesPerBlock;
    if (Bc > B) Bc = B;
    const size_t smem = fixed + per_frame * Bc;
    auto kern = k_cols_mul<T>;
    if (smem > (size_t)g_max_smem) return cudaErrorInvalidValue;
    kern<<<dim3(g.nh, (B + Bc - 1) / Bc), kThreads, smem, L.stream>>>(g, B, Bc, st, X1T, Y1T, K, tw);
    count(L);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Row-inverse passes
// ---------------------------------------------------------------------------
// Builds, in buf, the full spectrum z_k = A_k + i B_k of the row pair (r, r+1)
// from their half spectra (Hermitian extension), so that one inverse complex
// FFT returns row r in .x and row r+1 in .y.
template <typename C>
__device__ __forceinline__ void pack_row_pair(const C* S, int m, int r, int P, int nh, C* buf, int lane) {
    const bool two = r + 1 < m;
    for (int k = lane; k < P; k += 32) {
        const int kk = k < nh ? k : P - k;
        C a = S[kk * m + r];
        C b = two ? S[kk * m + r + 1] : cmk<C>(0, 0);
        if (kk == 0 || 2 * kk == P) { a.y = 0; b.y = 0; }
        if (k >= nh) { a = cconj(a); b = cconj(b); }
        buf[k] = cmk<C>(a.x - b.y, a.y + b.x);
    }
}

template <typename T, typename TIn>
__global__ void __launch_bounds__(kThreads)
k_rows_inv_masked(MvmGeom g, MaskTables mt, const FrameState* st, const cplx_t<T>* __restrict__ Y1T,
                  const TIn* __restrict__ xin, const double* __restrict__ noise_var, TIn* __restrict__ y,
                  double* part, const cplx_t<T>* __restrict__ twg) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kWarps];
    const int P = g.plan.P, m = g.m, nh = g.nh;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* wbuf = tw + P;
    C* S = wbuf + kWarps * 2 * P;
    const int pp = blockIdx.x, f = blockIdx.y;
    if (st && !st[f].active) return;
    for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
    const C* src = Y1T + ((size_t)f * g.NPout + pp) * nh * m;
    for (int i = threadIdx.x; i < nh * m; i += blockDim.x) S[i] = src[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C* buf = wbuf + warp * 2 * P;
    const size_t vbase = ((size_t)f * g.NPout + pp) * mt.n_vs;
    const TIn nv = (TIn)noise_var[pp];
    double acc = 0.0;
    for (int r = 2 * warp; r < m; r += 2 * kWarps) {
        pack_row_pair<C>(S, m, r, P, nh, buf, lane);
        __syncwarp();
        fft_warp<C>(buf, buf + P, g.plan, tw, false, lane, 32);
        for (int h = 0; h < 2 && r + h < m; ++h) {
            const int e0 = mt.rowstart[r + h], e1 = mt.rowstart[r + h + 1];
            for (int e = e0 + lane; e < e1; e += 32) {
                const C z = buf[mt.col[e]];
                const TIn xi = xin[vbase + e];
                const TIn out = (TIn)(h == 0 ? z.x : z.y) + nv * xi;
                y[vbase + e] = out;
                acc += (double)xi * (double)out;
            }
        }
        __syncwarp();
    }
    if (part) {
        const double s = block_sum<T>(acc, red);
        if (threadIdx.x == 0) part[(size_t)f * g.NPout + pp] = s;
    }
}

template <typename T, typename TIn>
cudaError_t rows_inv_masked(const Launch& L, const MvmGeom& g, const MaskTables& mt, int B, const FrameState* st,
                            const cplx_t<T>* Y1T, const TIn* xin, const double* noise_var, TIn* y, double* part,
                            const cplx_t<T>* tw) {
    using C = cplx_t<T>;
    const size_t smem = sizeof(C) * ((size_t)g.plan.P * (1 + 2 * kWarps) + (size_t)g.nh * g.m);
    auto kern = k_rows_inv_masked<T, TIn>;
    if (smem > (size_t)g_max_smem) return cudaErrorInvalidValue;
    kern<<<dim3(g.NPout, B), kThreads, smem, L.stream>>>(g, mt, st, Y1T, xin, noise_var, y, part, tw);
    count(L);
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_rows_inv_dense(MvmGeom g, const cplx_t<T>* __restrict__ Y1T, T* __restrict__ Yd, const cplx_t<T>* __restrict__ twg) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = g.plan.P, m = g.m, nh = g.nh;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* wbuf = tw + P;
    C* S = wbuf + kWarps * 2 * P;
    const int pp = blockIdx.x, f = blockIdx.y;
    for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
    const C* src = Y1T + ((size_t)f * g.NPout + pp) * nh * m;
    for (int i = threadIdx.x; i < nh * m; i += blockDim.x) S[i] = src[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C* buf = wbuf + warp * 2 * P;
    T* out = Yd + ((size_t)f * g.NPout + pp) * m * m;
    for (int r = 2 * warp; r < m; r += 2 * kWarps) {
        pack_row_pair<C>(S, m, r, P, nh, buf, lane);
        __syncwarp();
        fft_warp<C>(buf, buf + P, g.plan, tw, false, lane, 32);
        for (int c = lane; c < m; c += 32) {
            out[(size_t)r * m + c] = buf[c].x;
            if (r + 1 < m) out[(size_t)(r + 1) * m + c] = buf[c].y;
        }
        __syncwarp();
    }
}

template <typename T>
cudaError_t rows_inv_dense(const Launch& L, const MvmGeom& g, int B, const cplx_t<T>* Y1T, T* Yd, const cplx_t<T>* tw) {
    using C = cplx_t<T>;
    const size_t smem = sizeof(C) * ((size_t)g.plan.P * (1 + 2 * kWarps) + (size_t)g.nh * g.m);
    auto kern = k_rows_inv_dense<T>;
    if (smem > (size_t)g_max_smem) return cudaErrorInvalidValue;
    kern<<<dim3(g.NPout, B), kThreads, smem, L.stream>>>(g, Y1T, Yd, tw);
    count(L);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Conjugate gradients (FP32 vectors, FP64 reductions and scalars)
// ---------------------------------------------------------------------------
constexpr int kVecThreads = 256;

__global__ void __launch_bounds__(kVecThreads)
k_cg_init(int N, int nparts, const float* __restrict__ s, const float* __restrict__ Ax0, float* __restrict__ x,
          float* __restrict__ r, float* __restrict__ p, double* __restrict__ parts) {
    __shared__ double red[kVecThreads / 32];
    const int f = blockIdx.y;
    const size_t base = (size_t)f * N;
    double rr = 0.0, ss = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const float si = s[base + i];
        const float ri = Ax0 ? si - Ax0[base + i] : si;
        if (!Ax0) x[base + i] = 0.f;
        r[base + i] = ri;
        p[base + i] = 0.f;
        rr += (double)ri * ri;
        ss += (double)si * si;
    }
    double a = block_sum<float>(rr, red);
    if (threadIdx.x == 0) parts[((size_t)f * 2 + 0) * nparts + blockIdx.x] = a;
    double b = block_sum<float>(ss, red);
    if (threadIdx.x == 0) parts[((size_t)f * 2 + 1) * nparts + blockIdx.x] = b;
}

cudaError_t cg_init(const Launch& L, int B, int N, int nparts, const float* s, const float* Ax0, float* x, float* r,
                    float* p, double* parts) {
    k_cg_init<<<dim3(nparts, B), kVecThreads, 0, L.stream>>>(N, nparts, s, Ax0, x, r, p, parts);
    count(L);
    return cudaGetLastError();
}

__global__ void k_cg_init_scalars(int B, int nparts, const double* __restrict__ parts, double tol, FrameState* st) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= B) return;
    double rr = 0.0, ss = 0.0;
    for (int i = 0; i < nparts; ++i) {
        rr += parts[((size_t)f * 2 + 0) * nparts + i];
        ss += parts[((size_t)f * 2 + 1) * nparts + i];
    }
    FrameState s;
    s.rr = rr;
    s.beta = 0.0;
    s.snorm2 = ss;
    s.tol2 = tol * tol * ss;
    s.relres = ss > 0.0 ? sqrt(rr / ss) : 0.0;
    s.iters = 0;
    s.active = (ss > 0.0 && rr > s.tol2) ? 1 : 0;
    s.status = 0;
    s.refinements = 0;
    st[f] = s;
}

cudaError_t cg_init_scalars(const Launch& L, int B, int nparts, const double* parts, double tol, int /*warm*/,
                            FrameState* st) {
    k_cg_init_scalars<<<(B + 127) / 128, 128, 0, L.stream>>>(B, nparts, parts, tol, st);
    count(L);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kVecThreads)
k_cg_update(int N, int NP, int nparts, const float* __restrict__ p, const float* __restrict__ Ap,
            float* __restrict__ x, float* __restrict__ r, const double* __restrict__ pAp_part,
            double* __restrict__ rr_part, const FrameState* __restrict__ st) {
    __shared__ double red[kVecThreads / 32];
    const int f = blockIdx.y;
    if (!st[f].active) return;
    double pAp = 0.0;
    for (int i = 0; i < NP; ++i) pAp += pAp_part[(size_t)f * NP + i];
    const bool ok = pAp > 0.0 && isfinite(pAp);
    const float alpha = ok ? (float)(st[f].rr / pAp) : 0.f;
    const size_t base = (size_t)f * N;
    double rr = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        float ri = r[base + i];
        if (ok) {
            x[base + i] += alpha * p[base + i];
            ri -= alpha * Ap[base + i];
            r[base + i] = ri;
        }
        rr += (double)ri * ri;
    }
    const double s = block_sum<float>(rr, red);
    if (threadIdx.x == 0) rr_part[(size_t)f * nparts + blockIdx.x] = s;
}

cudaError_t cg_update(const Launch& L, int B, int N, int NP, int nparts, const float* p, const float* Ap, float* x,
                      float* r, const double* pAp_part, double* rr_part, const FrameState* st) {
    k_cg_update<<<dim3(nparts, B), kVecThreads, 0, L.stream>>>(N, NP, nparts, p, Ap, x, r, pAp_part, rr_part, st);
    count(L);
    return cudaGetLastError();
}

__global__ void k_cg_scalars(int B, int NP, int nparts, const double* __restrict__ pAp_part,
                             const double* __restrict__ rr_part, int maxit, FrameState* st) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= B || !st[f].active) return;
    double pAp = 0.0, rr = 0.0;
    for (int i = 0; i < NP; ++i) pAp += pAp_part[(size_t)f * NP + i];
    for (int i = 0; i < nparts; ++i) rr += rr_part[(size_t)f * nparts + i];
    FrameState s = st[f];
    if (!(pAp > 0.0) || !isfinite(pAp) || !isfinite(rr)) {
        s.active = 0;
        s.status = 2;  // TOMO_FRAME_BREAKDOWN
        st[f] = s;
        return;
    }
    s.iters += 1;
    s.beta = rr / s.rr;
    s.rr = rr;
    s.relres = sqrt(rr / s.snorm2);
    if (rr <= s.tol2) {
        s.active = 0;
        s.status = 0;
    } else if (s.iters >= maxit) {
        s.active = 0;
        s.status = 1;  // TOMO_FRAME_MAXIT
    }
    st[f] = s;
}

cudaError_t cg_scalars(const Launch& L, int B, int NP, int nparts, const double* pAp_part, const double* rr_part,
                       int maxit, FrameState* st) {
    k_cg_scalars<<<(B + 127) / 128, 128, 0, L.stream>>>(B, NP, nparts, pAp_part, rr_part, maxit, st);
    count(L);
    return cudaGetLastError();
}

__global__ void k_to_f64(size_t n, const float* __restrict__ a, double* __restrict__ b) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

cudaError_t to_f64(const Launch& L, size_t n, const float* a, double* b) {
    k_to_f64<<<1216, 256, 0, L.stream>>>(n, a, b);
    count(L);
    return cudaGetLastError();
}

// r64 = s - A zeta (FP64), stored rounded into the FP32 residual r for a restart.
__global__ void __launch_bounds__(kVecThreads)
k_true_residual(int N, int nparts, const float* __restrict__ s, const double* __restrict__ Ax, float* __restrict__ r,
                double* __restrict__ parts) {
    __shared__ double red[kVecThreads / 32];
    const int f = blockIdx.y;
    const size_t base = (size_t)f * N;
    double rr = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double ri = (double)s[base + i] - Ax[base + i];
        r[base + i] = (float)ri;
        rr += ri * ri;
    }
    const double t = block_sum<float>(rr, red);
    if (threadIdx.x == 0) parts[(size_t)f * nparts + blockIdx.x] = t;
}

cudaError_t true_residual(const Launch& L, int B, int N, int nparts, const float* s, const double* Ax, float* r,
                          double* parts) {
    k_true_residual<<<dim3(nparts, B), kVecThreads, 0, L.stream>>>(N, nparts, s, Ax, r, parts);
    count(L);
    return cudaGetLastError();
}

__global__ void k_true_residual_finalize(int B, int nparts, const double* __restrict__ parts, double tol,
                                         int max_refine, FrameState* st) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= B) return;
    FrameState s = st[f];
    if (s.snorm2 <= 0.0) { s.relres = 0.0; s.status = 0; s.active = 0; st[f] = s; return; }
    double rr = 0.0;
    for (int i = 0; i < nparts; ++i) rr += parts[(size_t)f * nparts + i];
    s.relres = sqrt(rr / s.snorm2);
    s.active = 0;
    if (s.relres > tol && s.status == 0) {
        if (s.refinements < max_refine) {
            s.refinements += 1;
            s.active = 1;
            s.rr = rr;
            s.beta = 0.0;
        } else {
            s.status = 1;  // could not reach tol: reported as MAXIT
        }
    }
    st[f] = s;
}

cudaError_t true_residual_finalize(const Launch& L, int B, int nparts, const double* parts, double tol, int max_refine,
                                   FrameState* st) {
    k_true_residual_finalize<<<(B + 127) / 128, 128, 0, L.stream>>>(B, nparts, parts, tol, max_refine, st);
    count(L);
    return cudaGetLastError();
}

__global__ void k_count_active(int B, const FrameState* st, int* n_active) {
    __shared__ int c;
    if (threadIdx.x == 0) c = 0;
    __syncthreads();
    for (int f = threadIdx.x; f < B; f += blockDim.x)
        if (st[f].active) atomicAdd(&c, 1);
    __syncthreads();
    if (threadIdx.x == 0) *n_active = c;
}

cudaError_t count_active(const Launch& L, int B, const FrameState* st, int* n_active) {
    k_count_active<<<1, 256, 0, L.stream>>>(B, st, n_active);
    count(L);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Setup: covariance generators and their spectra
// ---------------------------------------------------------------------------
// 2^{1/6}/Gamma(5/6) x^{5/6} K_{5/6}(x), which is 1 at x = 0: the von Karman
// covariance B(rho) = B(0) * shape(2 pi rho / L0).  K_nu is evaluated from its
// integral representation K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
// (Watson, "A treatise on the theory of Bessel functions", 6.22) by the
// trapezoidal rule with step h; the integrand is analytic in |Im t| < pi/2, so
// the discretisation error is of order exp(-pi^2 / h) (Trefethen & Weideman,
// SIAM Review 56, 2014).  Terms are summed until x cosh t - x > 45.
__device__ double vk_shape(double x, const VkParams& vk) {
    if (x < 1e-12) return 1.0;
    double s = 0.5 * exp(-x);
    for (int m = 1; m < vk.nq; ++m) {
        const double a = x * vk.cosh_t[m];
        if (a - x > 45.0) break;
        s += exp(-a) * vk.cosh_nu_t[m];
    }
    return vk.norm * pow(x, 5.0 / 6.0) * (s * vk.h);
}

// Theta_pq generator: t(di, dj) = cov(slope p at lag (di, dj), slope q at 0) =
//   sum_k sum_{u, v = +-1} u v B_k(| gamma_k ((dj d, di d) + u o_p - v o_q) + h_k (alpha_gp - alpha_gq) |)
// with o_p = (d/2) e_x for x-slopes and (d/2) e_y for y-slopes (Hudgin-like
// model, Appendix A.2; cone factor per layer, Sec. 2.D).  Stored at the
// wrapped lag (di mod P, dj mod P) so that y = IFFT(FFT(t) FFT(x)) is the
// linear convolution y(a) = sum_b t(a - b) x(b) on the n x n grid.
__global__ void k_gen_css(int n, int P, int NP, double d, int n_layers, const LayerGeom* __restrict__ layers,
                          const double* __restrict__ alpha, VkParams vk, double* __restrict__ G) {
    const int span = 2 * n - 1;
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= span * span) return;
    const int pair = blockIdx.y;
    const int p = pair / NP, q = pair % NP;
    const int gp = p >> 1, cp = p & 1, gq = q >> 1, cq = q & 1;
    const int di = li / span - (n - 1), dj = li % span - (n - 1);
    const double opx = cp == 0 ? 0.5 * d : 0.0, opy = cp == 1 ? 0.5 * d : 0.0;
    const double oqx = cq == 0 ? 0.5 * d : 0.0, oqy = cq == 1 ? 0.5 * d : 0.0;
    const double dax = alpha[2 * gp] - alpha[2 * gq], day = alpha[2 * gp + 1] - alpha[2 * gq + 1];
    const double k2pi = 2.0 * 3.14159265358979323846 / vk.L0;
    double t = 0.0;
    for (int k = 0; k < n_layers; ++k) {
        const LayerGeom lg = layers[k];
        double acc = 0.0;
        for (int u = -1; u <= 1; u += 2)
            for (int v = -1; v <= 1; v += 2) {
                const double sx = lg.gamma * (dj * d + u * opx - v * oqx) + lg.h * dax;
                const double sy = lg.gamma * (di * d + u * opy - v * oqy) + lg.h * day;
                acc += (double)(u * v) * vk_shape(k2pi * sqrt(sx * sx + sy * sy), vk);
            }
        t += lg.amp * acc;
    }
    const int wi = (di + P) % P, wj = (dj + P) % P;
    G[((size_t)pair * P + wi) * P + wj] = t;
}

cudaError_t gen_css(const Launch& L, int n, int P, int NP, double d, int n_layers, const LayerGeom* layers,
                    const double* gs_alpha, VkParams vk, double* G) {
    const int span = 2 * n - 1;
    k_gen_css<<<dim3((span * span + 127) / 128, NP * NP), 128, 0, L.stream>>>(n, P, NP, d, n_layers, layers, gs_alpha,
                                                                            vk, G);
    count(L);
    return cudaGetLastError();
}

// Xi'_{q,k} generator of the projection (Sec. 2.D, new phase grid; Eq. ToeplitzLGS):
// output node a of the m x m grid of layer k (pupil spacing gamma_k d, centred),
// input slope b of plane q; lag (di, dj) = a - b in [-(n-1), m-1]^2:
//   t = sum_{v=+-1} v B_k(| gamma_k d ((dj, di) + (n-m)/2) - v gamma_k o_q + h_k (beta - alpha_gq) |).
// With fold != 0 all layers are summed into slot 0 (natural guide stars:
// gamma = 1 for every layer and the interpolation is the identity).
__global__ void k_gen_cos(int n, int m, int P, int NP, double d, int n_layers, int fold,
                          const LayerGeom* __restrict__ layers, const double* __restrict__ alpha, double bx, double by,
                          VkParams vk, double* __restrict__ G) {
    const int span = m + n - 1;
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= span * span) return;
    const int slot = blockIdx.y;
    const int kk = slot / NP, q = slot % NP;
    const int gq = q >> 1, cq = q & 1;
    const int di = li / span - (n - 1), dj = li % span - (n - 1);
    const double oqx = cq == 0 ? 0.5 * d : 0.0, oqy = cq == 1 ? 0.5 * d : 0.0;
    const double k2pi = 2.0 * 3.14159265358979323846 / vk.L0;
    const double half = 0.5 * (double)(n - m);
    double t = 0.0;
    const int k0 = fold ? 0 : kk, k1 = fold ? n_layers : kk + 1;
    for (int k = k0; k < k1; ++k) {
        const LayerGeom lg = layers[k];
        double acc = 0.0;
        for (int v = -1; v <= 1; v += 2) {
            const double sx = lg.gamma * d * (dj + half) - v * lg.gamma * oqx + lg.h * (bx - alpha[2 * gq]);
            const double sy = lg.gamma * d * (di + half) - v * lg.gamma * oqy + lg.h * (by - alpha[2 * gq + 1]);
            acc += (double)v * vk_shape(k2pi * sqrt(sx * sx + sy * sy), vk);
        }
        t += lg.amp * acc;
    }
    const int wi = (di + P) % P, wj = (dj + P) % P;
    G[((size_t)slot * P + wi) * P + wj] = t;
}

cudaError_t gen_cos(const Launch& L, int n, int m, int P, int NP, double d, int n_layers, const LayerGeom* layers,
                    const double* gs_alpha, double bx, double by, VkParams vk, double* G) {
    // n_layers < 0 requests the folded (single-slot) form
    const int fold = n_layers < 0 ? 1 : 0;
    const int nl = fold ? -n_layers : n_layers;
    const int span = m + n - 1;
    k_gen_cos<<<dim3((span * span + 127) / 128, (fold ? 1 : nl) * NP), 128, 0, L.stream>>>(
        n, m, P, NP, d, nl, fold, layers, gs_alpha, bx, by, vk, G);
    count(L);
    return cudaGetLastError();
}

// Setup 2-D real FFT, rows: H[pl][kx][row] from G[pl][row][col].
__global__ void __launch_bounds__(kThreads)
k_setup_rows(FftPlan plan, const double* __restrict__ G, double2* __restrict__ H, const double2* __restrict__ twg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = plan.P, nh = P / 2 + 1;
    double2* tw = reinterpret_cast<double2*>(smem_raw);
    double2* wbuf = tw + P;
    const int pl = blockIdx.x;
    for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double2* buf = wbuf + warp * 2 * P;
    const double* g = G + (size_t)pl * P * P;
    for (int r = 2 * warp; r < P; r += 2 * kWarps) {
        for (int j = lane; j < P; j += 32) buf[j] = make_double2(g[(size_t)r * P + j], g[(size_t)(r + 1) * P + j]);
        __syncwarp();
        fft_warp<double2>(buf, buf + P, plan, tw, true, lane, 32);
        for (int k = lane; k < nh; k += 32) {
            const double2 zk = buf[k];
            const double2 zc = cconj(buf[k == 0 ? 0 : P - k]);
            H[((size_t)pl * nh + k) * P + r] = make_double2(0.5 * (zk.x + zc.x), 0.5 * (zk.y + zc.y));
            H[((size_t)pl * nh + k) * P + r + 1] = make_double2(0.5 * (zk.y - zc.y), -0.5 * (zk.x - zc.x));
        }
        __syncwarp();
    }
}

// Setup 2-D real FFT, columns, scaled by 1/P^2 into K [kx][ky][p][q].
__global__ void __launch_bounds__(kThreads)
k_setup_cols(FftPlan plan, int NPin, int npl, const double2* __restrict__ H, const double2* __restrict__ twg,
             double2* __restrict__ K64, float2* __restrict__ K32) {
    const int NPout = npl / NPin;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = plan.P, nh = P / 2 + 1;
    double2* tw = reinterpret_cast<double2*>(smem_raw);
    double2* wbuf = tw + P;
    const int pl = blockIdx.x;
    const int pp = pl / NPin, q = pl % NPin;
    for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double2* buf = wbuf + warp * 2 * P;
    const double sc = 1.0 / ((double)P * (double)P);
    for (int kx = warp; kx < nh; kx += kWarps) {
        for (int j = lane; j < P; j += 32) buf[j] = H[((size_t)pl * nh + kx) * P + j];
        __syncwarp();
        fft_warp<double2>(buf, buf + P, plan, tw, true, lane, 32);
        for (int ky = lane; ky < P; ky += 32) {
            const size_t o = (((size_t)kx * NPin + q) * P + ky) * NPout + pp;
            const double2 v = make_double2(buf[ky].x * sc, buf[ky].y * sc);
            if (K64) K64[o] = v;
            if (K32) K32[o] = make_float2((float)v.x, (float)v.y);
        }
        __syncwarp();
    }
}

cudaError_t spectra(const Launch& L, int P, int npl, int NPin, const FftPlan& plan, const double* G, double2* H,
                    const double2* tw64, double2* K64, float2* K32) {
    const size_t smem = sizeof(double2) * (size_t)P * (1 + 2 * kWarps);
    if (smem > (size_t)g_max_smem) return cudaErrorInvalidValue;
    cudaError_t e;
    k_setup_rows<<<npl, kThreads, smem, L.stream>>>(plan, G, H, tw64);
    count(L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_setup_cols<<<npl, kThreads, smem, L.stream>>>(plan, NPin, npl, H, tw64, K64, K32);
    count(L);
    return cudaGetLastError();
}

// phi[f][t][v] = sum_k sum_c w[k][v][c] Yd[f][k][idx[k][v][c]]  (Eq. interp, sum over layers)
__global__ void k_interp(int B, int T_all, int t, int n_layers, int m, int n_vphi, const float* __restrict__ Yd,
                         const int* __restrict__ idx, const float* __restrict__ w, float* __restrict__ phi) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const int f = blockIdx.y;
    if (v >= n_vphi) return;
    float acc = 0.f;
    for (int k = 0; k < n_layers; ++k) {
        const float* Y = Yd + ((size_t)f * n_layers + k) * m * m;
        const size_t o = ((size_t)k * n_vphi + v) * 4;
#pragma unroll
        for (int c = 0; c < 4; ++c) acc += w[o + c] * Y[idx[o + c]];
    }
    phi[((size_t)f * T_all + t) * n_vphi + v] = acc;
}

cudaError_t interp(const Launch& L, int B, int T_all, int t, int n_layers, int m, int n_vphi, const float* Yd,
                   const int* idx, const float* w, float* phi) {
    k_interp<<<dim3((n_vphi + 127) / 128, B), 128, 0, L.stream>>>(B, T_all, t, n_layers, m, n_vphi, Yd, idx, w, phi);
    count(L);
    return cudaGetLastError();
}

template <typename K>
cudaError_t allow_smem(K kern, int bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t init_kernel_attributes() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    // the kernels also use a little static shared memory
    const int dyn = optin - 1024;
    if ((e = allow_smem(k_rows_fwd<float, float>, dyn)) != cudaSuccess) return e;
    if ((e = allow_smem(k_rows_fwd<double, double>, dyn)) != cudaSuccess) return e;
    if ((e = allow_smem(k_cols_mul<float>, dyn)) != cudaSuccess) return e;
    if ((e = allow_smem(k_cols_mul<double>, dyn)) != cudaSuccess) return e;
    if ((e = allow_smem(k_rows_inv_masked<float, float>, dyn)) != cudaSuccess) return e;
    if ((e = allow_smem(k_rows_inv_masked<double, double>, dyn)) != cudaSuccess) return e;
    if ((e = allow_smem(k_rows_inv_dense<float>, dyn)) != cudaSuccess) return e;
    if ((e = allow_smem(k_setup_rows, dyn)) != cudaSuccess) return e;
    if ((e = allow_smem(k_setup_cols, dyn)) != cudaSuccess) return e;
    g_max_smem = dyn;
    return cudaSuccess;
}

// explicit instantiations
template cudaError_t rows_fwd<float, float>(const Launch&, const MvmGeom&, const MaskTables&, int, const float*,
                                            float*, const FrameState*, float2*, const float2*);
template cudaError_t rows_fwd<double, double>(const Launch&, const MvmGeom&, const MaskTables&, int, const double*,
                                              double*, const FrameState*, double2*, const double2*);
template cudaError_t cols_mul<float>(const Launch&, const MvmGeom&, int, const FrameState*, const float2*, float2*,
                                     const float2*, const float2*);
template cudaError_t cols_mul<double>(const Launch&, const MvmGeom&, int, const FrameState*, const double2*, double2*,
                                      const double2*, const double2*);
template cudaError_t rows_inv_masked<float, float>(const Launch&, const MvmGeom&, const MaskTables&, int,
                                                   const FrameState*, const float2*, const float*, const double*,
                                                   float*, double*, const float2*);
template cudaError_t rows_inv_masked<double, double>(const Launch&, const MvmGeom&, const MaskTables&, int,
                                                     const FrameState*, const double2*, const double*, const double*,
                                                     double*, double*, const double2*);
template cudaError_t rows_inv_dense<float>(const Launch&, const MvmGeom&, int, const float2*, float*, const float2*);

}  // namespace tomo
