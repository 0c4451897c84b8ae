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
#include <type_traits>

#include "fft_group.cuh"
#include "kernels.cuh"
#include "rowpass.cuh"

namespace tomo {

namespace {

inline void count(const Launch& L) {
    if (L.counter) ++*L.counter;
}

static_assert(kRowPairsPerBlock == kWarps * kFftGroup, "a row group is one round of the block's warps");

// Sequences per warp call of fft_rounds (rounds of whole sequences).  Six fill
// 30 of 32 lanes in both stages of 150 = 15 x 10 (rounds of three sequences at
// radix 15, of two at radix 10; a call of two leaves 12 lanes idle at radix
// 15).  The column pass uses it throughout; the row passes use it when one
// block holds a whole plane (37 row pairs: 7 calls on 8 warps, five round
// trips each, instead of up to three calls of two round trips), in FP32.
constexpr int kRoundGroup = 6;

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
// Row pair (2j, 2j+1) of a plane is packed as one complex sequence
// z = row_2j + i row_2j+1 in F[j][0..P) (row_stride, rowpass.cuh).

template <typename T, typename TIn, int PC>
__global__ void __launch_bounds__(kThreads, TOMO_MIN_BLOCKS)
k_rows_fwd(MvmGeom g, MaskTables mt, const TIn* __restrict__ x, CgVecs cg, const FrameState* st,
           cplx_t<T>* __restrict__ X1T, const cplx_t<T>* __restrict__ twg) {
    using C = cplx_t<T>;
    constexpr int G = kFftGroup;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kWarps];
    const int P = g.plan.P, n = g.n, nh = g.nh, RS = row_stride(P);
    // this block's row group: row pairs [pb, pb + npl) of the plane (all of
    // them when the plane is one block)
    const int ppb = gridDim.z == 1 ? (n + 1) / 2 : kRowPairsPerBlock;
    const int pb = blockIdx.z * ppb;
    const int npl = min(ppb, (n + 1) / 2 - pb);
    const int ngrp = (npl + G - 1) / G;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* scr = tw + P;                                // generic-path scratch, one per warp
    C* F = scr + (Fused<PC>::ok ? 0 : kWarps * P);  // [ngrp * G][RS]
    const int q = blockIdx.x, f = blockIdx.y;
    if (st && !st[f].active) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
    for (int i = threadIdx.x; i < ngrp * G * RS; i += blockDim.x) F[i] = cmk<C>(0, 0);
    // valid entries of rows [2 pb, 2 (pb + npl)) (row-major: a contiguous range)
    const int e0 = mt.rowstart[2 * pb], e1 = mt.rowstart[min(2 * (pb + npl), n)];
    __syncthreads();
    // sweep over the plane's valid entries (W_s^T scatter), with the CG update
    const size_t vbase = ((size_t)f * g.NPin + q) * mt.n_vs;
    const bool cgm = cg.p != nullptr;
    // r^T r: each thread's ~16 products summed in the vector type (FP32 in the
    // solver: GB300's FP64 rate is ~1/64 of its FP32 rate), FP64 across threads
    T rr = 0;
    float* __restrict__ vx = cg.x;
    float* __restrict__ vr = cg.r;
    float* __restrict__ vp = cg.p;
    float* __restrict__ vAp = cg.Ap;
    const float* __restrict__ vz = cg.z;
    const float* __restrict__ vw = cg.w;
    const int* __restrict__ rowcol = mt.rowcol;
    if (cgm && cg.mode == 1) {
        const float alpha = (float)st[f].alpha, beta = (float)st[f].beta;
#pragma unroll 4
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const size_t i = vbase + e;
            const int rc = rowcol[e];
            const float pe = vp[i];
            float re = vr[i];
            if (alpha != 0.f) {
                const float ape = vAp[i];
                vx[i] += alpha * pe;
                re -= alpha * ape;
                vr[i] = re;
            }
            const float pn = re + beta * pe;
            vp[i] = pn;
            rr = fma((T)re, (T)re, rr);
            const int row = rc >> 16, col = rc & 0xffff;
            T* dst = reinterpret_cast<T*>(F + ((row >> 1) - pb) * RS + col) + (row & 1);
            *dst = (T)pn;
        }
    } else if (cgm && cg.mode == 3) {
        const float alpha = (float)st[f].alpha, beta = (float)st[f].beta;
#pragma unroll 4
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const size_t i = vbase + e;
            const int rc = rowcol[e];
            float re = vr[i];
            const float pn = re + beta * vp[i];
            const float apn = vw[i] + beta * vAp[i];
            if (alpha != 0.f) {
                vx[i] += alpha * pn;
                re -= alpha * apn;
                vr[i] = re;
            }
            vp[i] = pn;
            vAp[i] = apn;
            rr = fma((T)re, (T)re, rr);
            const int row = rc >> 16, col = rc & 0xffff;
            T* dst = reinterpret_cast<T*>(F + ((row >> 1) - pb) * RS + col) + (row & 1);
            *dst = (T)re;
        }
    } else if (cgm) {
        const float alpha = (float)st[f].alpha, beta = (float)st[f].beta;
#pragma unroll 4
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const size_t i = vbase + e;
            const int rc = rowcol[e];
            const float pn = vz[i] + beta * vp[i];
            const float sn = vw[i] + beta * vAp[i];
            float re = vr[i];
            if (alpha != 0.f) {
                vx[i] += alpha * pn;
                re -= alpha * sn;
                vr[i] = re;
            }
            vp[i] = pn;
            vAp[i] = sn;
            rr = fma((T)re, (T)re, rr);
            const int row = rc >> 16, col = rc & 0xffff;
            T* dst = reinterpret_cast<T*>(F + ((row >> 1) - pb) * RS + col) + (row & 1);
            *dst = (T)re;
        }
    } else {
#pragma unroll 4
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const int rc = rowcol[e];
            const int row = rc >> 16, col = rc & 0xffff;
            T* dst = reinterpret_cast<T*>(F + ((row >> 1) - pb) * RS + col) + (row & 1);
            *dst = (T)__ldg(x + vbase + e);
        }
    }
    __syncthreads();
    bool rounds = false;
    if constexpr (sizeof(T) == 4) {                 // FP64 would spill
        rounds = gridDim.z == 1;
        if (rounds)
            for (int g0 = warp * kRoundGroup; g0 < npl; g0 += kWarps * kRoundGroup)
                fft_rounds<PC, C, true, kRoundGroup>(F + g0 * RS, RS, min(kRoundGroup, npl - g0), g.plan, tw,
                                                     scr + warp * P, lane, n, P);
    }
    if (!rounds)
        for (int gi = warp; gi < ngrp; gi += kWarps)
            fft_g<PC, C, true>(F + gi * G * RS, RS, G, g.plan, tw, scr + warp * P, lane, n, P);
    if (cgm) {
        const double t = block_sum<T>((double)rr, red);
        if (threadIdx.x == 0) cg.rr_part[((size_t)f * g.NPin + q) * gridDim.z + blockIdx.z] = t;
    }
    __syncthreads();
    // unpack the two real spectra of each pair, A = (Z_k + conj Z_{P-k})/2,
    // B = (Z_k - conj Z_{P-k})/(2i), and write them column-major [kx][row]
    C* out = X1T + ((size_t)f * g.NPin + q) * nh * n;
    for (int k = warp; k < nh; k += kWarps) {
        const int kc = k == 0 ? 0 : P - k;
        for (int jl = lane; jl < npl; jl += 32) {
            const int j = pb + jl;
            const C zk = F[jl * RS + k];
            const C zc = cconj(F[jl * RS + kc]);
            const C dd = csub(zk, zc);
            out[(size_t)k * n + 2 * j] = cscale(cadd(zk, zc), (T)0.5);
            if (2 * j + 1 < n) out[(size_t)k * n + 2 * j + 1] = cmk<C>((T)0.5 * dd.y, (T)-0.5 * dd.x);
        }
    }
}

template <typename T>
size_t rows_smem(const MvmGeom& g, int nrows) {
    const int G = kFftGroup;
    const int npair = (nrows + 1) / 2, ngrp = (npair + G - 1) / G;
    const int scratch = has_fused_plan(g.plan.P) ? 0 : kWarps;
    return sizeof(cplx_t<T>) * ((size_t)g.plan.P * (1 + scratch) + (size_t)ngrp * G * row_stride(g.plan.P));
}

template <typename T, typename TIn>
cudaError_t rows_fwd(const Launch& L, const MvmGeom& g, const MaskTables& mt, int B, const TIn* x, const CgVecs* cg,
                     const FrameState* st, cplx_t<T>* X1T, const cplx_t<T>* tw, int rg) {
    const CgVecs cgv = cg ? *cg : CgVecs{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr};
    if (rg != 1 && rg != row_groups(g.n)) return cudaErrorInvalidValue;
    if constexpr (std::is_same<T, float>::value && std::is_same<TIn, float>::value) {
        if (rg == 1) {
            bool used = false;
            const cudaError_t e = rows_fwd_pp(L, g, mt, B, x, cg, st, X1T, tw, g_max_smem, &used);
            if (e != cudaSuccess || used) return e;
        }
    }
    const size_t smem = rows_smem<T>(g, rg == 1 ? g.n : 2 * kRowPairsPerBlock);
    if (smem > (size_t)g_max_smem) return cudaErrorInvalidValue;
#define TOMO_L(PC)                                                                                      \
    k_rows_fwd<T, TIn, PC><<<dim3(g.NPin, B, rg), kThreads, smem, L.stream>>>(g, mt, x, cgv, st, X1T, tw)
    TOMO_DISPATCH_P(g.plan.P, TOMO_L)
#undef TOMO_L
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

// Sequences per warp call of the column transforms: a 12-plane frame is two calls.
constexpr int kColGroup = kRoundGroup;

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

// Hermitian variant for Sigma_ss (NP x NP blocks with K_qp = conj K_pq): only
// the upper triangle is stored, entry e(p, q) = herm_index(NP, p, q) for
// p <= q, in pairs of consecutive entries with the frequencies ky interleaved
// in groups of eight: [kx][ky / 8][e / 2][ky % 8][e % 2] (herm_offset; ky
// padded to a multiple of 8, e to an even count), so that one 16-byte load
// gives a thread two entries and the eight ky of a warp read one contiguous
// 128-byte segment.
//
// One thread per (ky, frame): it reads its x_q(ky) once, streams the packed
// entries of K(kx, ky) from global memory (L2; the frames of a ky share them
// through the same requests), applies each off-diagonal entry twice (K_pq to
// y_p, conj K_pq to y_q) and writes y back over x.  A thread touches only its
// own column entries, so the product needs no block barrier until its end.
// Each y_p is accumulated over q in ascending order.
__host__ __device__ constexpr int herm_index(int NP, int p, int q) { return p * NP - p * (p - 1) / 2 + (q - p); }

__host__ __device__ constexpr int herm_pairs(int NP) { return (NP * (NP + 1) / 2 + 1) / 2; }

__host__ __device__ inline size_t herm_offset(int NP, int P, int kx, int ky, int e) {
    const int P8 = (P + 7) / 8;
    return ((((size_t)kx * P8 + (ky >> 3)) * herm_pairs(NP) + (e >> 1)) * 8 + (ky & 7)) * 2 + (e & 1);
}

// Two consecutive complex values (16-byte aligned) in one load where they fit.
__device__ __forceinline__ void load_pair(const float2* src, float2 (&v)[2]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(src));
    v[0] = make_float2(t.x, t.y);
    v[1] = make_float2(t.z, t.w);
}
__device__ __forceinline__ void load_pair(const double2* src, double2 (&v)[2]) {
    v[0] = __ldg(src);
    v[1] = __ldg(src + 1);
}

template <typename C, int NP, int PS, int NPM>
__device__ __forceinline__ void block_mul_herm(C* D, int NPmax_rt, int P_rt, int nf, unsigned am,
                                               const C* __restrict__ Kc) {
    using T = decltype(C::x);
    const int P = PS ? PS : P_rt;
    const int NPmax = PS ? NPM : NPmax_rt;
    const int items = P * nf;
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
        const int ky = w / nf, fl = w - ky * nf;
        if (!((am >> fl) & 1u)) continue;
        C* col = D + (size_t)fl * NPmax * P + ky;
        const C* Kr = Kc + herm_offset(NP, P, 0, ky, 0);
        C x[NP];
        T yr[NP], yi[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            x[q] = col[q * P];
            yr[q] = 0;
            yi[q] = 0;
        }
        C kpair[2];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
#pragma unroll
            for (int q = p; q < NP; ++q) {
                const int e = herm_index(NP, p, q);
                if ((e & 1) == 0) load_pair(Kr + (e >> 1) * 16, kpair);
                const C k = kpair[e & 1];
                yr[p] = fma(k.x, x[q].x, yr[p]);           // y_p += K_pq x_q
                yr[p] = fma(-k.y, x[q].y, yr[p]);
                yi[p] = fma(k.x, x[q].y, yi[p]);
                yi[p] = fma(k.y, x[q].x, yi[p]);
                if (q != p) {                              // y_q += conj(K_pq) x_p
                    yr[q] = fma(k.x, x[p].x, yr[q]);
                    yr[q] = fma(k.y, x[p].y, yr[q]);
                    yi[q] = fma(k.x, x[p].y, yi[q]);
                    yi[q] = fma(-k.y, x[p].x, yi[q]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) col[p * P] = cmk<C>(yr[p], yi[p]);
    }
    __syncthreads();                               // the inverse transforms read other threads' columns
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

template <typename T, int PC>
__global__ void __launch_bounds__(kThreads, TOMO_MIN_BLOCKS)
k_cols_mul(MvmGeom g, int B, int Bc, const FrameState* st, const cplx_t<T>* __restrict__ X1T,
           cplx_t<T>* __restrict__ Y1T, const cplx_t<T>* __restrict__ K, const cplx_t<T>* __restrict__ twg,
           int herm) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = g.plan.P, n = g.n, m = g.m, nh = g.nh, NPin = g.NPin, NPout = g.NPout;
    constexpr int G = kColGroup;
    const int NPmax = NPin > NPout ? NPin : NPout;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* scr = tw + P;
    C* D = scr + (Fused<PC>::ok ? 0 : kWarps * P); // [Bc][NPmax][P]
    __shared__ int act[kMaxFramesPerBlock];
    const int kx = blockIdx.x;
    const int f0 = blockIdx.y * Bc;
    const int nf = min(Bc, B - f0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) act[i] = st ? st[f0 + i].active : 1;
    __syncthreads();
    unsigned am = 0;                               // active frames of the block, one bit each
    for (int i = 0; i < nf; ++i) am |= (act[i] ? 1u : 0u) << i;
    // load the columns, one warp per (frame, plane); rows >= n are the zero
    // padding, which the pruned forward transform never reads.  All loads of a
    // warp's two columns are issued before the first store (latency hiding).
    for (int t0 = warp * 2; t0 < nf * NPin; t0 += kWarps * 2) {
        C v[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int t = t0 + u;
            const int fl = t / NPin, q = t - fl * NPin;
            const bool ok = t < nf * NPin && act[fl < nf ? fl : 0];
            const C* src = X1T + (((size_t)(f0 + (ok ? fl : 0)) * NPin + (ok ? q : 0)) * nh + kx) * n;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = lane + 32 * i;
                if (ok && r < n) v[u][i] = __ldg(src + r);
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int t = t0 + u;
            const int fl = t / NPin, q = t - fl * NPin;
            if (t >= nf * NPin || !act[fl]) continue;
            C* dst = D + ((size_t)fl * NPmax + q) * P;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = lane + 32 * i;
                if (r < n) dst[r] = v[u][i];
            }
            if (!Fused<PC>::ok)
                for (int r = n + lane; r < P; r += 32) dst[r] = cmk<C>(0, 0);
        }
    }
    // rows beyond 128 (n > 128) are loaded here
    if (n > 128) {
        for (int t = warp; t < nf * NPin; t += kWarps) {
            const int fl = t / NPin, q = t - fl * NPin;
            if (!act[fl]) continue;
            const C* src = X1T + (((size_t)(f0 + fl) * NPin + q) * nh + kx) * n;
            C* dst = D + ((size_t)fl * NPmax + q) * P;
            for (int r = 128 + lane; r < n; r += 32) dst[r] = src[r];
        }
    }
    __syncthreads();
    {
        const int gpf = (NPin + G - 1) / G;        // the last group of a frame may be partial
        for (int t = warp; t < nf * gpf; t += kWarps) {
            const int fl = t / gpf, q0 = (t % gpf) * G;
            if (!act[fl]) continue;
            C* base = D + ((size_t)fl * NPmax + q0) * P;
            fft_rounds<PC, C, true, G>(base, P, min(G, NPin - q0), g.plan, tw, scr + warp * P, lane, n, P);
        }
    }
    __syncthreads();
    // block multiply: one thread per (ky, p), frames looped
    const C* Kc = K + (size_t)kx * NPin * P * NPout;
    const C* Kh = K + herm_offset(NPin, P, kx, 0, 0);
    if (herm) {
#define TOMO_BMH(NP_) block_mul_herm<C, NP_, PC, NP_>(D, NPmax, P, nf, am, Kh)
        switch (NPin) {
            case 2: TOMO_BMH(2); break;
            case 4: TOMO_BMH(4); break;
            case 6: TOMO_BMH(6); break;
            case 8: TOMO_BMH(8); break;
            case 10: TOMO_BMH(10); break;
            case 12: TOMO_BMH(12); break;
            case 14: TOMO_BMH(14); break;
            default: TOMO_BMH(16); break;
        }
#undef TOMO_BMH
    } else if (NPin == 12 && NPout == 12) block_mul<C, 12, 12>(D, NPmax, P, nf, act, Kc);
    else if (NPin == 6 && NPout == 6) block_mul<C, 6, 6>(D, NPmax, P, nf, act, Kc);
    else if (NPin == 4 && NPout == 4) block_mul<C, 4, 4>(D, NPmax, P, nf, act, Kc);
    else if (NPin == 2 && NPout == 2) block_mul<C, 2, 2>(D, NPmax, P, nf, act, Kc);
    else block_mul_rt<C>(D, NPmax, P, nf, act, Kc, NPin, NPout);
    {
        const int gpf = (NPout + G - 1) / G;       // the last group of a frame may be partial
        for (int t = warp; t < nf * gpf; t += kWarps) {
            const int fl = t / gpf, p0 = (t % gpf) * G;
            if (!act[fl]) continue;
            C* base = D + ((size_t)fl * NPmax + p0) * P;
            fft_rounds<PC, C, false, G>(base, P, min(G, NPout - p0), g.plan, tw, scr + warp * P, lane, P, m);
        }
    }
    __syncthreads();
    for (int t = warp; t < nf * NPout; t += kWarps) {
        const int fl = t / NPout, pp = t - fl * NPout;
        if (!act[fl]) continue;
        const C* src = D + ((size_t)fl * NPmax + pp) * P;
        C* dst = Y1T + (((size_t)(f0 + fl) * NPout + pp) * nh + kx) * m;
        for (int r = lane; r < m; r += 32) dst[r] = src[r];
    }
}

template <typename T>
cudaError_t cols_mul(const Launch& L, const MvmGeom& g, int B, const FrameState* st, const cplx_t<T>* X1T,
                     cplx_t<T>* Y1T, const cplx_t<T>* K, const cplx_t<T>* tw, bool herm) {
    using C = cplx_t<T>;
    if (g.NPin > 16) return cudaErrorInvalidValue;
    const int NPmax = g.NPin > g.NPout ? g.NPin : g.NPout;
    if (herm && (g.NPin != g.NPout || (g.NPin & 1) || g.NPin < 2 || g.NPin > 16)) return cudaErrorInvalidValue;
    const size_t fixed = sizeof(C) * (size_t)g.plan.P * (1 + (has_fused_plan(g.plan.P) ? 0 : kWarps));
    const size_t per_frame = sizeof(C) * (size_t)NPmax * g.plan.P;
#ifndef TOMO_COLS_BUDGET_KB
#define TOMO_COLS_BUDGET_KB 72
#endif
    const size_t budget = TOMO_COLS_BUDGET_KB * 1024;   // shared memory per block of the column pass
    int Bc = (int)((budget > fixed ? budget - fixed : 0) / per_frame);
    // no more frames than make one transform call per warp (kColGroup columns
    // each): with 12 planes that is 4 frames, 48 columns for 8 warps.  A fifth
    // frame fits the budget but takes a second round of calls in two warps and
    // leaves the launch's last wave mostly empty (ELT, 64 frames: 988 blocks
    // for 456 resident, 143.9 us per product against 139.2 us with 4 frames)
    const int Bround = (kWarps * kColGroup) / NPmax;
    if (Bround >= 1 && Bc > Bround) Bc = Bround;
    if (Bc < 1) Bc = 1;
    if (Bc > kMaxFramesPerBlock) Bc = kMaxFramesPerBlock;
    if (Bc > B) Bc = B;
    const size_t smem = fixed + per_frame * Bc;
    if (smem > (size_t)g_max_smem) return cudaErrorInvalidValue;
#define TOMO_L(PC) \
    k_cols_mul<T, PC><<<dim3(g.nh, (B + Bc - 1) / Bc), kThreads, smem, L.stream>>>(g, B, Bc, st, X1T, Y1T, K, tw, \
                                                                                  (int)herm)
    TOMO_DISPATCH_P(g.plan.P, TOMO_L)
#undef TOMO_L
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

// Loads the half spectra [kx][row] of the m kept rows of one plane into F as
// packed row pairs z_k = A_k + i B_k over the full k range (put_row_pair,
// rowpass.cuh), so that one inverse complex FFT per pair returns row 2j in .x
// and row 2j+1 in .y.  Pairs [pb, pb + npair) of the plane go to F rows
// [0, npair).
template <typename C>
__device__ __forceinline__ void load_row_pairs(const C* __restrict__ src, int m, int P, int nh, int RS, C* F,
                                               int pb, int npair) {
    const int total = nh * npair;
    constexpr int U = 4;
    for (int i0 = threadIdx.x; i0 < total; i0 += U * blockDim.x) {
        C a[U], b[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < total) {
                const int k = i / npair, j = i - k * npair, r = 2 * (pb + j);
                a[u] = __ldg(src + (size_t)k * m + r);
                b[u] = r + 1 < m ? __ldg(src + (size_t)k * m + r + 1) : cmk<C>(0, 0);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < total) {
                const int k = i / npair, j = i - k * npair;
                put_row_pair<C>(F, RS, P, j, k, a[u], b[u]);
            }
        }
    }
}

template <typename T, typename TIn, int PC>
__global__ void __launch_bounds__(kThreads, TOMO_MIN_BLOCKS)
k_rows_inv_masked(MvmGeom g, MaskTables mt, const FrameState* st, const cplx_t<T>* __restrict__ Y1T,
                  const TIn* __restrict__ xin, const double* __restrict__ noise_var,
                  const double2* __restrict__ fscale, TIn* __restrict__ y,
                  CgVecs cg, const cplx_t<T>* __restrict__ twg) {
    using C = cplx_t<T>;
    constexpr int G = kFftGroup;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kWarps];
    const int P = g.plan.P, m = g.m, nh = g.nh, RS = row_stride(P);
    // this block's row group: output row pairs [pb, pb + npair) of the plane
    // (all of them when the plane is one block)
    const int ppb = gridDim.z == 1 ? (m + 1) / 2 : kRowPairsPerBlock;
    const int pb = blockIdx.z * ppb;
    const int npair = min(ppb, (m + 1) / 2 - pb);
    const int ngrp = (npair + G - 1) / G;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* scr = tw + P;
    C* F = scr + (Fused<PC>::ok ? 0 : kWarps * P);
    const int pp = blockIdx.x, f = blockIdx.y;
    if (st && !st[f].active) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
    if (npair < ngrp * G)
        for (int i = threadIdx.x; i < (ngrp * G - npair) * RS; i += blockDim.x) F[npair * RS + i] = cmk<C>(0, 0);
    load_row_pairs<C>(Y1T + ((size_t)f * g.NPout + pp) * nh * m, m, P, nh, RS, F, pb, npair);
    __syncthreads();
    bool rounds = false;
    if constexpr (sizeof(T) == 4) {                 // FP64 would spill
        rounds = gridDim.z == 1;
        if (rounds)
            for (int g0 = warp * kRoundGroup; g0 < npair; g0 += kWarps * kRoundGroup)
                fft_rounds<PC, C, false, kRoundGroup>(F + g0 * RS, RS, min(kRoundGroup, npair - g0), g.plan, tw,
                                                      scr + warp * P, lane, P, m);
    }
    if (!rounds)
        for (int gi = warp; gi < ngrp; gi += kWarps)
            fft_g<PC, C, false>(F + gi * G * RS, RS, G, g.plan, tw, scr + warp * P, lane, P, m);
    __syncthreads();
    // gather the valid outputs (W_s), add the noise term, CG dot products
    const size_t vbase = ((size_t)f * g.NPout + pp) * mt.n_vs;
    const double2 fs = fscale ? fscale[f] : make_double2(1.0, 1.0);
    const TIn cs = (TIn)fs.x;
    const TIn nv = (TIn)(noise_var[pp] * fs.y);
    const bool cgm = cg.p != nullptr;
    // second partner of the partial sums: r (CG, PCG) or the direction's A p (MINRES)
    const float* __restrict__ vr = cg.mode == 3 ? cg.Ap : cg.r;
    const int* __restrict__ rowcol = mt.rowcol;
    // partial sums: each thread's ~16 products in the vector type (FP32 in the
    // solver), FP64 across threads, blocks and planes
    TIn acc = 0, acc_r = 0, acc_a = 0;
    const int e0 = mt.rowstart[2 * pb], e1 = mt.rowstart[min(2 * (pb + npair), m)];
#pragma unroll 4
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int rc = rowcol[e];
        const int row = rc >> 16, col = rc & 0xffff;
        const TIn xi = xin ? __ldg(xin + vbase + e) : (TIn)0;
        const float ri = cgm ? __ldg(vr + vbase + e) : 0.f;
        const T v = reinterpret_cast<const T*>(F + ((row >> 1) - pb) * RS + col)[row & 1];
        const TIn out = cs * (TIn)v + nv * xi;
        y[vbase + e] = out;
        if (cgm) {
            acc = fma(xi, out, acc);
            acc_r = fma((TIn)ri, out, acc_r);
            acc_a = fma(out, out, acc_a);
        }
    }
    if (cgm) {
        double* dp = cg.dot_part + (((size_t)f * g.NPout + pp) * gridDim.z + blockIdx.z) * 3;
        const double s0 = block_sum<T>((double)acc, red);
        if (threadIdx.x == 0) dp[0] = s0;
        const double s1 = block_sum<T>((double)acc_r, red);
        if (threadIdx.x == 0) dp[1] = s1;
        const double s2 = block_sum<T>((double)acc_a, red);
        if (threadIdx.x == 0) dp[2] = s2;
    }
}

template <typename T, typename TIn>
cudaError_t rows_inv_masked(const Launch& L, const MvmGeom& g, const MaskTables& mt, int B, const FrameState* st,
                            const cplx_t<T>* Y1T, const TIn* xin, const double* noise_var, const double2* fscale,
                            TIn* y, const CgVecs* cg, const cplx_t<T>* tw, int rg) {
    const CgVecs cgv = cg ? *cg : CgVecs{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr};
    if (rg != 1 && rg != row_groups(g.m)) return cudaErrorInvalidValue;
    if constexpr (std::is_same<T, float>::value && std::is_same<TIn, float>::value) {
        if (rg == 1) {
            bool used = false;
            const cudaError_t e =
                rows_inv_pp(L, g, mt, B, st, Y1T, xin, noise_var, fscale, y, cg, tw, g_max_smem, &used);
            if (e != cudaSuccess || used) return e;
        }
    }
    const size_t smem = rows_smem<T>(g, rg == 1 ? g.m : 2 * kRowPairsPerBlock);
    if (smem > (size_t)g_max_smem) return cudaErrorInvalidValue;
#define TOMO_L(PC)                                                                                \
    k_rows_inv_masked<T, TIn, PC><<<dim3(g.NPout, B, rg), kThreads, smem, L.stream>>>(               \
        g, mt, st, Y1T, xin, noise_var, fscale, y, cgv, tw)
    TOMO_DISPATCH_P(g.plan.P, TOMO_L)
#undef TOMO_L
    count(L);
    return cudaGetLastError();
}

template <typename T, int PC>
__global__ void __launch_bounds__(kThreads, TOMO_MIN_BLOCKS)
k_rows_inv_dense(MvmGeom g, const cplx_t<T>* __restrict__ Y1T, T* __restrict__ Yd, const cplx_t<T>* __restrict__ twg) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = g.plan.P, m = g.m, nh = g.nh;
    constexpr int G = kFftGroup;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* wbuf = tw + P;
    C* S = wbuf + kWarps * (G + 1) * P;
    const int pp = blockIdx.x, f = blockIdx.y;
    for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
    const C* src = Y1T + ((size_t)f * g.NPout + pp) * nh * m;
    for (int i = threadIdx.x; i < nh * m; i += blockDim.x) S[i] = src[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C* wb = wbuf + warp * (G + 1) * P;
    T* out = Yd + ((size_t)f * g.NPout + pp) * m * m;
    for (int r0 = 2 * G * warp; r0 < m; r0 += 2 * G * kWarps) {
        for (int gi = 0; gi < G; ++gi) {
            const int r = r0 + 2 * gi;
            if (r < m) pack_row_pair<C>(S, m, r, P, nh, wb + gi * P, lane);
            else for (int k = lane; k < P; k += 32) wb[gi * P + k] = cmk<C>(0, 0);
        }
        __syncwarp();
        fft_g<PC, C, false>(wb, P, G, g.plan, tw, wb + G * P, lane, P, m);
        for (int gi = 0; gi < G; ++gi) {
            const int r = r0 + 2 * gi;
            if (r >= m) break;
            const C* buf = wb + gi * P;
            for (int c = lane; c < m; c += 32) {
                out[(size_t)r * m + c] = buf[c].x;
                if (r + 1 < m) out[(size_t)(r + 1) * m + c] = buf[c].y;
            }
        }
        __syncwarp();
    }
}

template <typename T>
cudaError_t rows_inv_dense(const Launch& L, const MvmGeom& g, int B, const cplx_t<T>* Y1T, T* Yd, const cplx_t<T>* tw) {
    using C = cplx_t<T>;
    const size_t smem = sizeof(C) * ((size_t)g.plan.P * (1 + (kFftGroup + 1) * kWarps) + (size_t)g.nh * g.m);
    if (smem > (size_t)g_max_smem) return cudaErrorInvalidValue;
#define TOMO_L(PC) k_rows_inv_dense<T, PC><<<dim3(g.NPout, B), kThreads, smem, L.stream>>>(g, Y1T, Yd, tw)
    TOMO_DISPATCH_P(g.plan.P, TOMO_L)
#undef TOMO_L
    count(L);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Conjugate gradients (FP32 vectors, FP64 reductions and scalars)
// ---------------------------------------------------------------------------
constexpr int kVecThreads = 256;

__global__ void __launch_bounds__(kVecThreads)
k_cg_init(int N, int nparts, const float* __restrict__ s, const float* __restrict__ Ax0, float* __restrict__ x,
          float* __restrict__ r, float* __restrict__ p, float* __restrict__ Ap, double* __restrict__ parts) {
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
        Ap[base + i] = 0.f;
        rr += (double)ri * ri;
        ss += (double)si * si;
    }
    double a = block_sum<float>(rr, red);
    if (threadIdx.x == 0) parts[((size_t)f * 2 + 0) * nparts + blockIdx.x] = a;
    double b = block_sum<float>(ss, red);
    if (threadIdx.x == 0) parts[((size_t)f * 2 + 1) * nparts + blockIdx.x] = b;
}

cudaError_t cg_init(const Launch& L, int B, int N, int nparts, const float* s, const float* Ax0, float* x, float* r,
                    float* p, float* Ap, double* parts) {
    k_cg_init<<<dim3(nparts, B), kVecThreads, 0, L.stream>>>(N, nparts, s, Ax0, x, r, p, Ap, parts);
    count(L);
    return cudaGetLastError();
}

constexpr double kInnerTol = 0.7;

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
    s.alpha = 0.0;
    s.beta = 0.0;
    s.snorm2 = ss;
    // the recursive (FP32) residual is driven below kInnerTol * tol so that the
    // FP64 true residual normally clears tol without a restart
    s.tol2 = (kInnerTol * tol) * (kInnerTol * tol) * ss;
    // a frame whose slopes (or warm start) hold a NaN or an infinity never
    // iterates: it is reported as a breakdown, with the initial guess as result
    const bool finite = isfinite(rr) && isfinite(ss);
    s.relres = !finite ? nan("") : (ss > 0.0 ? sqrt(rr / ss) : 0.0);
    s.iters = 0;
    s.active = (finite && ss > 0.0 && rr > s.tol2) ? 1 : 0;
    s.status = finite ? 0 : 2;  // TOMO_FRAME_BREAKDOWN
    s.refinements = 0;
    s.gamma = 0.0;
    s.fresh = 1;
    s.pad_ = 0;
    s.delta = 0.0;
    s.fb = 0;
    s.ckpt_iter = 0;
    s.rr_ckpt = rr;
    st[f] = s;
}

cudaError_t cg_init_scalars(const Launch& L, int B, int nparts, const double* parts, double tol, int /*warm*/,
                            FrameState* st) {
    k_cg_init_scalars<<<(B + 127) / 128, 128, 0, L.stream>>>(B, nparts, parts, tol, st);
    count(L);
    return cudaGetLastError();
}

// The per-iteration scalar kernels run one warp per frame: lane i loads the
// partial sums i, i + 32, ... (all loads in flight at once; a serial loop over
// them was bound by one L2 round trip per partial) and an xor butterfly
// combines the lanes.  Floating-point addition is commutative, so every lane
// ends with bitwise the same totals; lane 0 then updates the frame's state.
constexpr int kScalarWarps = 4;

__device__ __forceinline__ double warp_total(double v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// rr_part holds r^T r of the residual that the row-forward pass of this
// iteration produced (r_k), dot_part the sums p^T Ap, r^T Ap, Ap^T Ap of this
// iteration's product.  Stops the frame when r_k is small enough (x_k is then
// final); otherwise alpha_k = r_k^T r_k / p^T Ap and
// beta_{k+1} = r_{k+1}^T r_{k+1} / r_k^T r_k with the recurrence value
// r_{k+1}^T r_{k+1} = r_k^T r_k - 2 alpha r_k^T Ap + alpha^2 Ap^T Ap.
__global__ void __launch_bounds__(kScalarWarps * 32)
k_cg_scalars(int B, int NP, const double* __restrict__ rr_part, const double* __restrict__ dot_part,
             FrameState* st) {
    const int f = blockIdx.x * kScalarWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (f >= B) return;
    const int active = st[f].active;
    double rr = 0.0, pAp = 0.0, rAp = 0.0, ApAp = 0.0;
    for (int i = lane; i < NP; i += 32) {
        rr += rr_part[(size_t)f * NP + i];
        const double* d = dot_part + ((size_t)f * NP + i) * 3;
        pAp += d[0];
        rAp += d[1];
        ApAp += d[2];
    }
    rr = warp_total(rr);
    pAp = warp_total(pAp);
    rAp = warp_total(rAp);
    ApAp = warp_total(ApAp);
    if (!active || lane != 0) return;
    FrameState s = st[f];
    s.rr = rr;
    s.relres = sqrt(rr / s.snorm2);
    if (rr <= s.tol2) {
        s.active = 0;
        s.status = 0;
        st[f] = s;
        return;
    }
    if (!(pAp > 0.0) || !isfinite(pAp) || !isfinite(rr)) {
        s.active = 0;
        s.status = 2;  // TOMO_FRAME_BREAKDOWN
        st[f] = s;
        return;
    }
    const double alpha = rr / pAp;
    double rr_next = rr - 2.0 * alpha * rAp + alpha * alpha * ApAp;
    if (!(rr_next > 0.0)) rr_next = 0.0;
    s.alpha = alpha;
    s.beta = rr_next / rr;
    s.iters += 1;
    st[f] = s;
}

cudaError_t cg_scalars(const Launch& L, int B, int NP, const double* rr_part, const double* dot_part, FrameState* st) {
    k_cg_scalars<<<(B + kScalarWarps - 1) / kScalarWarps, kScalarWarps * 32, 0, L.stream>>>(B, NP, rr_part, dot_part,
                                                                                           st);
    count(L);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kScalarWarps * 32)
k_pcg_scalars(int B, int NP, const double* __restrict__ rr_part, const double* __restrict__ dot_M,
              const double* __restrict__ dot_A, FrameState* st) {
    const int f = blockIdx.x * kScalarWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (f >= B) return;
    const int active = st[f].active;
    double rr = 0.0, gamma = 0.0, delta = 0.0;
    for (int i = lane; i < NP; i += 32) {
        rr += rr_part[(size_t)f * NP + i];
        gamma += dot_M[((size_t)f * NP + i) * 3];
        delta += dot_A[((size_t)f * NP + i) * 3];
    }
    rr = warp_total(rr);
    gamma = warp_total(gamma);
    delta = warp_total(delta);
    if (!active || lane != 0) return;
    FrameState s = st[f];
    s.rr = rr;
    s.relres = sqrt(rr / s.snorm2);
    if (rr <= s.tol2) {
        s.active = 0;
        s.status = 0;
        st[f] = s;
        return;
    }
    double beta = 0.0, den = delta;
    if (!s.fresh) {
        beta = gamma / s.gamma;
        den = delta - beta * gamma / s.alpha;
    }
    if (!(gamma > 0.0) || !(den > 0.0) || !isfinite(gamma) || !isfinite(den)) {
        s.active = 0;
        s.status = 2;  // TOMO_FRAME_BREAKDOWN
        st[f] = s;
        return;
    }
    s.alpha = gamma / den;
    s.beta = beta;
    s.gamma = gamma;
    s.fresh = 0;
    s.iters += 1;
    st[f] = s;
}

cudaError_t pcg_scalars(const Launch& L, int B, int NP, const double* rr_part, const double* dot_M,
                        const double* dot_A, FrameState* st) {
    k_pcg_scalars<<<(B + kScalarWarps - 1) / kScalarWarps, kScalarWarps * 32, 0, L.stream>>>(B, NP, rr_part, dot_M,
                                                                                            dot_A, st);
    count(L);
    return cudaGetLastError();
}

// rr_part: r^T r of the residual the row-forward pass produced (r_{k+1});
// dot_part: r^T w, Ap^T w, w^T w with w = A r_{k+1} and Ap the direction's
// product used in that update.  Conjugate residuals:
// p_{k+1} = r_{k+1} + beta p_k, A p_{k+1} = w + beta A p_k, alpha = r^T A r / |A p|^2;
// for symmetric positive (semi)definite A these are the MINRES iterates
// (each x_k minimises the residual norm over the Krylov space).
__global__ void __launch_bounds__(kScalarWarps * 32)
k_mr_scalars(int B, int NP, const double* __restrict__ rr_part, const double* __restrict__ dot_part,
             FrameState* st) {
    const int f = blockIdx.x * kScalarWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (f >= B) return;
    const int active = st[f].active;
    double rr = 0.0, rho = 0.0, apw = 0.0, ww = 0.0;
    for (int i = lane; i < NP; i += 32) {
        rr += rr_part[(size_t)f * NP + i];
        const double* d = dot_part + ((size_t)f * NP + i) * 3;
        rho += d[0];
        apw += d[1];
        ww += d[2];
    }
    rr = warp_total(rr);
    rho = warp_total(rho);
    apw = warp_total(apw);
    ww = warp_total(ww);
    if (!active || lane != 0) return;
    FrameState s = st[f];
    s.rr = rr;
    s.relres = sqrt(rr / s.snorm2);
    if (rr <= s.tol2) {
        s.active = 0;
        s.status = 0;
        st[f] = s;
        return;
    }
    double beta = 0.0, apap = ww;
    if (!s.fresh) {
        beta = rho / s.gamma;
        apap = ww + 2.0 * beta * apw + beta * beta * s.delta;
    }
    if (!(rho > 0.0) || !(apap > 0.0) || !isfinite(rho) || !isfinite(apap) || !isfinite(rr)) {
        s.active = 0;
        s.status = 2;  // TOMO_FRAME_BREAKDOWN
        st[f] = s;
        return;
    }
    s.alpha = rho / apap;
    s.beta = beta;
    s.gamma = rho;
    s.delta = apap;
    s.fresh = 0;
    s.iters += 1;
    st[f] = s;
}

cudaError_t mr_scalars(const Launch& L, int B, int NP, const double* rr_part, const double* dot_part, FrameState* st) {
    k_mr_scalars<<<(B + kScalarWarps - 1) / kScalarWarps, kScalarWarps * 32, 0, L.stream>>>(B, NP, rr_part, dot_part,
                                                                                           st);
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
                                         int max_refine, FrameState* st, const LoopState* __restrict__ ls) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= B) return;
    if (ls) {
        tol = ls->tol;
        max_refine = ls->stop ? 0 : ls->max_refine;
    }
    FrameState s = st[f];
    if (s.snorm2 <= 0.0) { s.relres = 0.0; s.status = 0; s.active = 0; st[f] = s; return; }
    double rr = 0.0;
    for (int i = 0; i < nparts; ++i) rr += parts[(size_t)f * nparts + i];
    s.relres = sqrt(rr / s.snorm2);
    s.active = 0;
    if (!isfinite(s.relres)) {
        s.status = 2;  // TOMO_FRAME_BREAKDOWN: non-finite input or iterate
        st[f] = s;
        return;
    }
    if (s.relres > tol && s.status == 0) {
        if (s.refinements < max_refine) {
            s.refinements += 1;
            s.active = 1;
            s.rr = rr;
            s.alpha = 0.0;
            s.beta = 0.0;
            s.fresh = 1;
        } else {
            s.status = 1;  // could not reach tol: reported as MAXIT
        }
    }
    st[f] = s;
}

cudaError_t true_residual_finalize(const Launch& L, int B, int nparts, const double* parts, double tol, int max_refine,
                                   FrameState* st, const LoopState* ls) {
    k_true_residual_finalize<<<(B + 127) / 128, 128, 0, L.stream>>>(B, nparts, parts, tol, max_refine, st, ls);
    count(L);
    return cudaGetLastError();
}

// --- device-side loop control (conditional graph nodes) ---------------------
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void k_loop_start(LoopState* ls, long long max_iter, unsigned long long budget, double tol, int max_refine,
                             int chunk) {
    ls->iters = 0;
    ls->max_iter = max_iter;
    ls->budget = budget;
    ls->tol = tol;
    ls->max_refine = max_refine;
    ls->chunk = chunk;
    ls->stop = 0;
    ls->timed_out = 0;
    ls->true_res_runs = 0;
    ls->t0 = global_ns();
}

cudaError_t loop_start(const Launch& L, LoopState* ls, long long max_iter, unsigned long long budget_ns, double tol,
                       int max_refine, int chunk) {
    k_loop_start<<<1, 1, 0, L.stream>>>(ls, max_iter, budget_ns, tol, max_refine, chunk);
    count(L);
    return cudaGetLastError();
}

__global__ void k_loop_check(int B, FrameState* st, LoopState* ls, cudaGraphConditionalHandle need) {
    __shared__ int active, stop;
    if (threadIdx.x == 0) {
        active = 0;
        ls->iters += ls->chunk;
        const bool late = ls->budget != 0 && global_ns() - ls->t0 > ls->budget;
        if (late) ls->timed_out = 1;
        stop = (ls->iters >= ls->max_iter || late) ? 1 : 0;
        if (stop) ls->stop = 1;
    }
    __syncthreads();
    for (int f = threadIdx.x; f < B; f += blockDim.x) {
        if (!st[f].active) continue;
        if (stop) {
            st[f].active = 0;
            st[f].status = 1;  // TOMO_FRAME_MAXIT
        } else {
            atomicAdd(&active, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool run = active == 0 || stop;
        if (run) ls->true_res_runs += 1;
        cudaGraphSetConditional(need, run ? 1u : 0u);
    }
}

cudaError_t loop_check(const Launch& L, int B, FrameState* st, LoopState* ls, cudaGraphConditionalHandle need) {
    k_loop_check<<<1, 256, 0, L.stream>>>(B, st, ls, need);
    count(L);
    return cudaGetLastError();
}

__global__ void k_loop_next(int B, const FrameState* st, const LoopState* ls, cudaGraphConditionalHandle more) {
    __shared__ int active;
    if (threadIdx.x == 0) active = 0;
    __syncthreads();
    for (int f = threadIdx.x; f < B; f += blockDim.x)
        if (st[f].active) atomicAdd(&active, 1);
    __syncthreads();
    if (threadIdx.x == 0) cudaGraphSetConditional(more, (active > 0 && !ls->stop) ? 1u : 0u);
}

cudaError_t loop_next(const Launch& L, int B, const FrameState* st, const LoopState* ls,
                      cudaGraphConditionalHandle more) {
    k_loop_next<<<1, 256, 0, L.stream>>>(B, st, ls, more);
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

// v[f] = 0 for the frames reported as breakdowns (keeps a non-finite frame out
// of the block recurrences, whose Gram products mix every frame).
__global__ void k_zero_broken(int N, const FrameState* __restrict__ st, float* __restrict__ v) {
    const int f = blockIdx.y;
    if (st[f].status != 2) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) v[(size_t)f * N + i] = 0.f;
}

cudaError_t zero_broken(const Launch& L, int B, int N, const FrameState* st, float* v) {
    k_zero_broken<<<dim3(16, B), 256, 0, L.stream>>>(N, st, v);
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
// Points of one slope component (0 = x, 1 = y) relative to the subaperture
// centre, and their weights, in the slope model (Appendix A): 0 Hudgin-like,
// the midpoints of the two edges across the component, weights +1 / -1;
// 1 Fried, the four corners, weights +-1/2 (the mean of the differences
// along the two edges parallel to the component).
struct Stencil {
    int n;
    double ox[4], oy[4], w[4];
};

__device__ __forceinline__ Stencil slope_stencil(int model, int comp, double d) {
    const double h = 0.5 * d;
    const double ex = comp == 0 ? h : 0.0, ey = comp == 1 ? h : 0.0;   // along the component
    const double fx = comp == 0 ? 0.0 : h, fy = comp == 0 ? h : 0.0;   // across it
    Stencil st;
    if (model == 1) {
        st.n = 4;
        st.ox[0] = ex + fx;  st.oy[0] = ey + fy;  st.w[0] = 0.5;
        st.ox[1] = -ex + fx; st.oy[1] = -ey + fy; st.w[1] = -0.5;
        st.ox[2] = ex - fx;  st.oy[2] = ey - fy;  st.w[2] = 0.5;
        st.ox[3] = -ex - fx; st.oy[3] = -ey - fy; st.w[3] = -0.5;
    } else {
        st.n = 2;
        st.ox[0] = ex;  st.oy[0] = ey;  st.w[0] = 1.0;
        st.ox[1] = -ex; st.oy[1] = -ey; st.w[1] = -1.0;
        st.ox[2] = st.oy[2] = st.w[2] = st.ox[3] = st.oy[3] = st.w[3] = 0.0;
    }
    return st;
}

__global__ void k_gen_css(int lo, int span, int P, int NP, double d, int n_layers, const LayerGeom* __restrict__ layers,
                          const double* __restrict__ alpha, VkParams vk, int model, double* __restrict__ G) {
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= span * span) return;
    const int pair = blockIdx.y;
    const int p = pair / NP, q = pair % NP;
    const int gp = p >> 1, cp = p & 1, gq = q >> 1, cq = q & 1;
    const int di = li / span + lo, dj = li % span + lo;
    const Stencil sp = slope_stencil(model, cp, d), sq = slope_stencil(model, cq, d);
    const double dax = alpha[2 * gp] - alpha[2 * gq], day = alpha[2 * gp + 1] - alpha[2 * gq + 1];
    const double k2pi = 2.0 * 3.14159265358979323846 / vk.L0;
    double t = 0.0;
    for (int k = 0; k < n_layers; ++k) {
        const LayerGeom lg = layers[k];
        double acc = 0.0;
        for (int u = 0; u < sp.n; ++u)
            for (int v = 0; v < sq.n; ++v) {
                const double sx = lg.gamma * (dj * d + sp.ox[u] - sq.ox[v]) + lg.h * dax;
                const double sy = lg.gamma * (di * d + sp.oy[u] - sq.oy[v]) + lg.h * day;
                acc += sp.w[u] * sq.w[v] * vk_shape(k2pi * sqrt(sx * sx + sy * sy), vk);
            }
        t += lg.amp * acc;
    }
    const int wi = (di + P) % P, wj = (dj + P) % P;
    G[((size_t)pair * P + wi) * P + wj] = t;
}

cudaError_t gen_css(const Launch& L, int n, int P, int NP, double d, int n_layers, const LayerGeom* layers,
                    const double* gs_alpha, VkParams vk, double* G, bool periodised, int model) {
    // exact 2RBT generator: lags [-(n-1), n-1]; periodised: every lag of the P-torus, [-P/2, P/2)
    const int lo = periodised ? -(P / 2) : -(n - 1);
    const int span = periodised ? P : 2 * n - 1;
    k_gen_css<<<dim3((span * span + 127) / 128, NP * NP), 128, 0, L.stream>>>(lo, span, P, NP, d, n_layers, layers,
                                                                            gs_alpha, vk, model, G);
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
                          VkParams vk, int model, double* __restrict__ G) {
    const int span = m + n - 1;
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= span * span) return;
    const int slot = blockIdx.y;
    const int kk = slot / NP, q = slot % NP;
    const int gq = q >> 1, cq = q & 1;
    const int di = li / span - (n - 1), dj = li % span - (n - 1);
    const Stencil sq = slope_stencil(model, cq, d);
    const double k2pi = 2.0 * 3.14159265358979323846 / vk.L0;
    const double half = 0.5 * (double)(n - m);
    double t = 0.0;
    const int k0 = fold ? 0 : kk, k1 = fold ? n_layers : kk + 1;
    for (int k = k0; k < k1; ++k) {
        const LayerGeom lg = layers[k];
        double acc = 0.0;
        for (int v = 0; v < sq.n; ++v) {
            const double sx = lg.gamma * (d * (dj + half) - sq.ox[v]) + lg.h * (bx - alpha[2 * gq]);
            const double sy = lg.gamma * (d * (di + half) - sq.oy[v]) + lg.h * (by - alpha[2 * gq + 1]);
            acc += sq.w[v] * vk_shape(k2pi * sqrt(sx * sx + sy * sy), vk);
        }
        t += lg.amp * acc;
    }
    const int wi = (di + P) % P, wj = (dj + P) % P;
    G[((size_t)slot * P + wi) * P + wj] = t;
}

cudaError_t gen_cos(const Launch& L, int n, int m, int P, int NP, double d, int n_layers, const LayerGeom* layers,
                    const double* gs_alpha, double bx, double by, VkParams vk, double* G, int model) {
    // n_layers < 0 requests the folded (single-slot) form
    const int fold = n_layers < 0 ? 1 : 0;
    const int nl = fold ? -n_layers : n_layers;
    const int span = m + n - 1;
    k_gen_cos<<<dim3((span * span + 127) / 128, (fold ? 1 : nl) * NP), 128, 0, L.stream>>>(
        n, m, P, NP, d, nl, fold, layers, gs_alpha, bx, by, vk, model, G);
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

// Block-circulant preconditioner (per frequency f of the P x P torus):
//   M(f) = (K_+(f) + c Sigma)^{-1} / P^2,
// K(f) the 12 x 12 (NP x NP) Hermitian block of the periodised generator's
// spectrum, K_+ its eigenvalues clamped at zero (the periodised kernel is not
// exactly positive semi-definite), Sigma = diag(sigma_p^2).  One thread per
// frequency, FP64: cyclic Jacobi (Golub & Van Loan, Matrix Computations, 8.5)
// on the real symmetric embedding [[Re K, -Im K], [Im K, Re K]], then a
// Cholesky inverse of the clamped, shifted embedding.  M is written in the
// layout of the spectra, [kx][q][ky][p].
constexpr int kMaxNP = 16;
__global__ void k_precond(int P, int NP, const double2* __restrict__ K64, const double* __restrict__ noise_var,
                          double floor_c, double scale, float2* __restrict__ M32) {
    // K64 holds FFT(t) / P^2 (the inverse-transform normalisation folded in); undo it here
    const double kscale = (double)P * (double)P;
    const int nh = P / 2 + 1;
    const int fi = blockIdx.x * blockDim.x + threadIdx.x;
    if (fi >= nh * P) return;
    const int kx = fi / P, ky = fi % P;
    const int n2 = 2 * NP;
    double R[2 * kMaxNP][2 * kMaxNP], V[2 * kMaxNP][2 * kMaxNP];
    for (int p = 0; p < NP; ++p)
        for (int q = 0; q < NP; ++q) {
            const double2 a = K64[(((size_t)kx * NP + q) * P + ky) * NP + p];
            const double2 b = K64[(((size_t)kx * NP + p) * P + ky) * NP + q];
            const double re = 0.5 * kscale * (a.x + b.x), im = 0.5 * kscale * (a.y - b.y);   // (K + K^H) / 2
            R[p][q] = re;
            R[p + NP][q + NP] = re;
            R[p + NP][q] = im;
            R[p][q + NP] = -im;
        }
    for (int i = 0; i < n2; ++i)
        for (int j = 0; j < n2; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n2; ++i)
            for (int j = 0; j < n2; ++j) {
                tot += R[i][j] * R[i][j];
                if (i != j) off += R[i][j] * R[i][j];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n2 - 1; ++p)
            for (int q = p + 1; q < n2; ++q) {
                const double apq = R[p][q];
                if (fabs(apq) <= 1e-300) continue;
                const double theta = (R[q][q] - R[p][p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n2; ++k) {        // columns p, q of R
                    const double rkp = R[k][p], rkq = R[k][q];
                    R[k][p] = c * rkp - s * rkq;
                    R[k][q] = s * rkp + c * rkq;
                }
                for (int k = 0; k < n2; ++k) {        // rows p, q of R
                    const double rpk = R[p][k], rqk = R[q][k];
                    R[p][k] = c * rpk - s * rqk;
                    R[q][k] = s * rpk + c * rqk;
                }
                for (int k = 0; k < n2; ++k) {        // eigenvectors
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    // R <- V max(Lambda, 0) V^T + c Sigma
    double lam[2 * kMaxNP];
    for (int i = 0; i < n2; ++i) lam[i] = R[i][i] > 0.0 ? R[i][i] : 0.0;
    for (int i = 0; i < n2; ++i)
        for (int j = 0; j <= i; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n2; ++k) acc += V[i][k] * lam[k] * V[j][k];
            R[i][j] = acc;
        }
    for (int i = 0; i < n2; ++i) R[i][i] += floor_c * noise_var[i % NP];
    // Cholesky R = L L^T in the lower triangle, then R^{-1} = L^{-T} L^{-1} into V
    for (int j = 0; j < n2; ++j) {
        double dsum = R[j][j];
        for (int k = 0; k < j; ++k) dsum -= R[j][k] * R[j][k];
        const double ljj = sqrt(dsum > 0.0 ? dsum : 1e-300);
        R[j][j] = ljj;
        for (int i = j + 1; i < n2; ++i) {
            double acc = R[i][j];
            for (int k = 0; k < j; ++k) acc -= R[i][k] * R[j][k];
            R[i][j] = acc / ljj;
        }
    }
    for (int col = 0; col < n2; ++col) {
        double y[2 * kMaxNP];
        for (int i = 0; i < n2; ++i) {            // L y = e_col
            double acc = i == col ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) acc -= R[i][k] * y[k];
            y[i] = acc / R[i][i];
        }
        for (int i = n2 - 1; i >= 0; --i) {       // L^T x = y
            double acc = y[i];
            for (int k = i + 1; k < n2; ++k) acc -= R[k][i] * V[k][col];
            V[i][col] = acc / R[i][i];
        }
    }
    for (int p = 0; p < NP; ++p)
        for (int q = 0; q < NP; ++q)
            M32[(((size_t)kx * NP + q) * P + ky) * NP + p] =
                make_float2((float)(V[p][q] * scale), (float)(V[p + NP][q] * scale));
}

cudaError_t precond_spectra(const Launch& L, int P, int NP, const double2* K64, const double* noise_var,
                            double floor_c, float2* M32) {
    if (NP > kMaxNP) return cudaErrorInvalidValue;
    const int nf = (P / 2 + 1) * P;
    k_precond<<<(nf + 63) / 64, 64, 0, L.stream>>>(P, NP, K64, noise_var, floor_c, 1.0 / ((double)P * P), M32);
    count(L);
    return cudaGetLastError();
}

// Packs a full NP x NP spectrum [nh][NP(q)][P][NP(p)] into the Hermitian
// upper-triangle layout of block_mul_herm (herm_offset), storing
// (K_pq + conj K_qp) / 2; the padding frequencies ky >= P are zero.
__global__ void k_pack_hermitian(int P, int NP, const float2* __restrict__ Kf, float2* __restrict__ Kp) {
    const int nh = P / 2 + 1, NE = NP * (NP + 1) / 2, P8 = (P + 7) / 8, NE2 = herm_pairs(NP);
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= herm_packed_elems(P, NP)) return;
    // i = (((kx P8 + ky / 8) NE2 + e / 2) 8 + ky % 8) 2 + e % 2
    const int e = 2 * (int)((i / 16) % NE2) + (int)(i % 2);
    const int ky = (int)((i / 2) % 8) + 8 * (int)((i / ((size_t)16 * NE2)) % P8);
    const int kx = (int)(i / ((size_t)16 * NE2 * P8));
    if (ky >= P || kx >= nh || e >= NE) {
        Kp[i] = make_float2(0.f, 0.f);
        return;
    }
    int p = 0;
    while (herm_index(NP, p + 1, p + 1) <= e && p + 1 < NP) ++p;
    const int q = p + (e - herm_index(NP, p, p));
    const float2 a = Kf[(((size_t)kx * NP + q) * P + ky) * NP + p];
    const float2 b = Kf[(((size_t)kx * NP + p) * P + ky) * NP + q];
    Kp[i] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
}

cudaError_t pack_hermitian(const Launch& L, int P, int NP, const float2* Kfull, float2* Kpacked) {
    const size_t total = herm_packed_elems(P, NP);
    k_pack_hermitian<<<(unsigned)((total + 255) / 256), 256, 0, L.stream>>>(P, NP, Kfull, Kpacked);
    count(L);
    return cudaGetLastError();
}

// phi[f][t][v] = sum_k sum_c w[k][v][c] Yd[f][k][idx[k][v][c]]  (Eq. interp, sum over layers)
__global__ void k_interp(int B, int T_all, int t, int n_layers, int m, int n_vphi, const float* __restrict__ Yd,
                         const int* __restrict__ idx, const float* __restrict__ w, const double2* __restrict__ fscale,
                         float* __restrict__ phi) {
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
    if (fscale) acc *= (float)fscale[f].x;
    phi[((size_t)f * T_all + t) * n_vphi + v] = acc;
}

cudaError_t interp(const Launch& L, int B, int T_all, int t, int n_layers, int m, int n_vphi, const float* Yd,
                   const int* idx, const float* w, const double2* fscale, float* phi) {
    k_interp<<<dim3((n_vphi + 127) / 128, B), 128, 0, L.stream>>>(B, T_all, t, n_layers, m, n_vphi, Yd, idx, w,
                                                                     fscale, phi);
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
#define TOMO_A(PC)                                                                         \
    if (e == cudaSuccess) e = allow_smem(k_rows_fwd<float, float, PC>, dyn);               \
    if (e == cudaSuccess) e = allow_smem(k_rows_fwd<double, double, PC>, dyn);             \
    if (e == cudaSuccess) e = allow_smem(k_cols_mul<float, PC>, dyn);                      \
    if (e == cudaSuccess) e = allow_smem(k_cols_mul<double, PC>, dyn);                     \
    if (e == cudaSuccess) e = allow_smem(k_rows_inv_masked<float, float, PC>, dyn);        \
    if (e == cudaSuccess) e = allow_smem(k_rows_inv_masked<double, double, PC>, dyn);      \
    if (e == cudaSuccess) e = allow_smem(k_rows_inv_dense<float, PC>, dyn);
    TOMO_A(150)
    TOMO_A(180)
    TOMO_A(160)
    TOMO_A(40)
    TOMO_A(32)
    TOMO_A(0)
#undef TOMO_A
    if (e != cudaSuccess) return e;
    if ((e = allow_smem(k_setup_rows, dyn)) != cudaSuccess) return e;
    if ((e = allow_smem(k_setup_cols, dyn)) != cudaSuccess) return e;
    if ((e = init_fft_constants()) != cudaSuccess) return e;
    if ((e = init_rows_pp_attributes(dyn)) != cudaSuccess) return e;
    g_max_smem = dyn;
    return cudaSuccess;
}

// explicit instantiations
template cudaError_t rows_fwd<float, float>(const Launch&, const MvmGeom&, const MaskTables&, int, const float*,
                                            const CgVecs*, const FrameState*, float2*, const float2*, int);
template cudaError_t rows_fwd<double, double>(const Launch&, const MvmGeom&, const MaskTables&, int, const double*,
                                              const CgVecs*, const FrameState*, double2*, const double2*, int);
template cudaError_t cols_mul<float>(const Launch&, const MvmGeom&, int, const FrameState*, const float2*, float2*,
                                     const float2*, const float2*, bool);
template cudaError_t cols_mul<double>(const Launch&, const MvmGeom&, int, const FrameState*, const double2*, double2*,
                                      const double2*, const double2*, bool);
template cudaError_t rows_inv_masked<float, float>(const Launch&, const MvmGeom&, const MaskTables&, int,
                                                   const FrameState*, const float2*, const float*, const double*,
                                                   const double2*, float*, const CgVecs*, const float2*, int);
template cudaError_t rows_inv_masked<double, double>(const Launch&, const MvmGeom&, const MaskTables&, int,
                                                     const FrameState*, const double2*, const double*, const double*,
                                                     const double2*, double*, const CgVecs*, const double2*, int);
template cudaError_t rows_inv_dense<float>(const Launch&, const MvmGeom&, int, const float2*, float*, const float2*);

}  // namespace tomo
