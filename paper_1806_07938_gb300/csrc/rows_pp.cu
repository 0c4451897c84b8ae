// Persistent, prefetching forms of the FP32 row passes of the Sigma_ss product
// (Sec. 2.E, steps 1-2 and 4-5 of the 2RBT MVM as 2-D real FFTs: the W_s^T
// scatter with the row FFTs, and the inverse row FFTs with the crop and the
// W_s gather).  kernels.cu has the plain forms and the shared-memory layout;
// these do the same arithmetic in the same order, and differ in how the work
// reaches the SMs:
//   * a fixed grid of blocks (as many as the SMs hold) walks the (frame,
//     plane) items of the batch, so no launch wave is left partly empty;
//   * one thread of each block fetches the next item's inputs with a bulk
//     asynchronous copy (cp.async.bulk, completion counted on an mbarrier)
//     while the block transforms the current one, so the loads are in flight
//     during the FFTs instead of before them.  Row-inverse: the plane's half
//     spectra [kx][row] (45 KB at P = 150), and its slices of the input and
//     of r fetched into L2 (cp.async.bulk.prefetch.L2) for the gather.
//     Row-forward in CG mode: the plane's slices of p, r, A p and x
//     (4 x 15.9 KB).
//   * the vector scatter and gather read four entries per load.
// Every wait on a copy is bounded (kMaxWaitPolls); on expiry the block sets
// g_wait_error, waits (again bounded) for its copy and returns.
#include <cstdio>
#include <cstdlib>

#include "fft_group.cuh"
#include "kernels.cuh"
#include "rowpass.cuh"

namespace tomo {

namespace {

__device__ int g_wait_error = 0;

constexpr int kPPRound = 6;            // sequences per warp call of the transforms (as the plain passes)

inline void bump(const Launch& L) {
    if (L.counter) ++*L.counter;
}

// Block sum of FP32 per-thread partials: within each warp in FP32 with an
// error-free transformation (Knuth's TwoSum: the rounding error of every
// addition is carried along, so the warp's sum is exact to about FP32
// precision squared), then the eight warp sums in FP64 by thread 0 (GB300's
// FP64 rate is ~1/64 of its FP32 rate, so FP64 shuffles cost more than the
// rest of the reduction).
__device__ __forceinline__ double bsum32(float v, double* red) {
    float s = v, c = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float t = __shfl_down_sync(0xffffffffu, s, o);
        const float tc = __shfl_down_sync(0xffffffffu, c, o);
        const float u = s + t;
        const float bp = u - s;
        const float err = (s - (u - bp)) + (t - bp);
        s = u;
        c += tc + err;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = (double)s + (double)c;
    __syncthreads();
    double out = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) out += red[w];
    return out;
}

// bsum32 for three values at once (one pair of block barriers); red holds
// 3 x (warps) doubles.  Thread 0 returns the sums in out.
__device__ __forceinline__ void bsum32x3(float v0, float v1, float v2, double* red, double (&out)[3]) {
    float s[3] = {v0, v1, v2}, c[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float t = __shfl_down_sync(0xffffffffu, s[q], o);
            const float tc = __shfl_down_sync(0xffffffffu, c[q], o);
            const float u = s[q] + t;
            const float bp = u - s[q];
            const float err = (s[q] - (u - bp)) + (t - bp);
            s[q] = u;
            c[q] += tc + err;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 3; ++q) red[q * nw + warp] = (double)s[q] + (double)c[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 3; ++q) out[q] = 0.0;
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 3; ++q)
            for (int w = 0; w < nw; ++w) out[q] += red[q * nw + w];
}

// Thread 0 waits for the barrier phase (bounded), the block learns the
// outcome through shared memory; then every thread observes the completed
// phase itself (immediate), which makes the copied bytes visible to it.
// Returns false (the block must return) if the copy did not land in time.
__device__ __forceinline__ bool block_wait(uint64_t* bar, uint32_t parity, int* ok) {
    if (threadIdx.x == 0) *ok = mbar_wait(bar, parity) ? 1 : 0;
    __syncthreads();
    if (!*ok) {
        if (threadIdx.x == 0) {
            atomicExch(&g_wait_error, 1);
            mbar_wait(bar, parity);        // the copy may still land: do not leave it writing into freed memory
        }
        return false;
    }
    mbar_wait(bar, parity);
    return true;
}

__device__ __forceinline__ bool item_active(const FrameState* st, int t, int planes) {
    return st == nullptr || st[t / planes].active;
}

// ---------------------------------------------------------------------------
// Row-inverse pass: y = c_f crop/mask(IFFT rows) + nu_f sigma^2 xin (and the
// CG partial sums), as k_rows_inv_masked with one block per whole plane.
// Shared memory: S [nh][m] (staged half spectra) | tw [P] | F [npair][RS].
template <int PC>
__global__ void __launch_bounds__(kThreads, 2)
k_rows_inv_pp(MvmGeom g, MaskTables mt, int items, const FrameState* __restrict__ st, const float2* __restrict__ Y1T,
              const float* __restrict__ xin, const double* __restrict__ noise_var, const double2* __restrict__ fscale,
              float* __restrict__ y, CgVecs cg, const float2* __restrict__ twg) {
    using C = float2;
    constexpr int P = PC, RS = P | 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[3 * kWarps];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int ok;
    const int m = g.m, nh = g.nh, NPo = g.NPout;
    const int npair = (m + 1) / 2;
    const int slab = nh * m;
    C* S = reinterpret_cast<C*>(smem_raw);
    C* tw = S + slab;
    C* F = tw + P;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int t = blockIdx.x;
    while (t < items && !item_active(st, t, NPo)) t += gridDim.x;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
    __syncthreads();
    if (t >= items) return;
    const bool cgm = cg.p != nullptr;
    // second partner of the partial sums: r (CG, PCG) or the direction's A p (MINRES)
    const float* __restrict__ vr = cg.mode == 3 ? cg.Ap : cg.r;
    // the vector slices the gather of item it reads, fetched into L2 with its
    // half spectra (they are read from DRAM otherwise: the column pass between
    // the two row passes evicts them)
    const uint32_t vbytes = (uint32_t)(mt.n_vs * sizeof(float));
    auto prefetch_vectors = [&](int it) {
        const size_t o = (size_t)it * mt.n_vs;
        if (xin) bulk_prefetch_l2(xin + o, vbytes);
        if (cgm) bulk_prefetch_l2(vr + o, vbytes);
    };
    if (threadIdx.x == 0) {
        bulk_load(S, Y1T + (size_t)t * slab, (uint32_t)(slab * sizeof(C)), &bar);
        prefetch_vectors(t);
    }
    const int n4 = mt.n_vs >> 2;
    uint32_t parity = 0;
    while (t < items) {
        if (!block_wait(&bar, parity, &ok)) return;
        parity ^= 1u;
        const int f = t / NPo, pp = t - f * NPo;
        for (int i = threadIdx.x; i < nh * npair; i += blockDim.x) {
            const int k = i / npair, j = i - k * npair, r = 2 * j;
            const C a = S[k * m + r];
            const C b = r + 1 < m ? S[k * m + r + 1] : make_float2(0.f, 0.f);
            put_row_pair<C>(F, RS, P, j, k, a, b);
        }
        __syncthreads();
        // the next active plane streams in while this one is transformed
        int tn = t + gridDim.x;
        while (tn < items && !item_active(st, tn, NPo)) tn += gridDim.x;
        if (threadIdx.x == 0 && tn < items) {
            fence_async_shared();
            bulk_load(S, Y1T + (size_t)tn * slab, (uint32_t)(slab * sizeof(C)), &bar);
            prefetch_vectors(tn);
        }
        for (int g0 = warp * kPPRound; g0 < npair; g0 += kWarps * kPPRound)
            fft_rounds<PC, C, false, kPPRound>(F + g0 * RS, RS, min(kPPRound, npair - g0), g.plan, tw, nullptr, lane,
                                               P, m);
        __syncthreads();
        // gather the valid outputs (W_s), add the noise term, CG partial sums;
        // four consecutive entries per load (the plane's entries are contiguous)
        const size_t vbase = (size_t)t * mt.n_vs;
        const double2 fs = fscale ? fscale[f] : make_double2(1.0, 1.0);
        const float cs = (float)fs.x;
        const float nv = (float)(noise_var[pp] * fs.y);
        const float4* __restrict__ x4 = xin ? reinterpret_cast<const float4*>(xin + vbase) : nullptr;
        const float4* __restrict__ r4 = cgm ? reinterpret_cast<const float4*>(vr + vbase) : nullptr;
        float4* __restrict__ y4 = reinterpret_cast<float4*>(y + vbase);
        const int4* __restrict__ rc4 = reinterpret_cast<const int4*>(mt.rowcol);
        float acc = 0.f, acc_r = 0.f, acc_a = 0.f;       // per thread FP32 (<= 16 products), FP64 across
        constexpr int U = 4;
        for (int i0 = threadIdx.x; i0 < n4; i0 += U * blockDim.x) {
            float4 xv[U], rv[U];
            int4 cv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * blockDim.x;
                if (i < n4) {
                    cv[u] = __ldg(rc4 + i);
                    xv[u] = x4 ? __ldg(x4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
                    rv[u] = r4 ? __ldg(r4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * blockDim.x;
                if (i >= n4) continue;
                const float* xs = &xv[u].x;
                const float* rs = &rv[u].x;
                const int* cs4 = &cv[u].x;
                float o[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int row = cs4[c] >> 16, col = cs4[c] & 0xffff;
                    const float v = reinterpret_cast<const float*>(F + (row >> 1) * RS + col)[row & 1];
                    o[c] = cs * v + nv * xs[c];
                    if (cgm) {
                        acc = fmaf(xs[c], o[c], acc);
                        acc_r = fmaf(rs[c], o[c], acc_r);
                        acc_a = fmaf(o[c], o[c], acc_a);
                    }
                }
                y4[i] = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
        if (cgm) {
            double sums[3];
            bsum32x3(acc, acc_r, acc_a, red, sums);
            if (threadIdx.x == 0) {
                double* dp = cg.dot_part + (size_t)t * 3;
                dp[0] = sums[0];
                dp[1] = sums[1];
                dp[2] = sums[2];
            }
        }
        __syncthreads();                       // F is rebuilt for the next plane
        t = tn;
    }
}

// ---------------------------------------------------------------------------
// Row-forward pass, as k_rows_fwd with one block per whole plane.  MODE 0:
// the input x is scattered (W_s^T) and transformed; MODE 1 (CG): the
// scheduled update x += alpha p, r -= alpha Ap, p = r + beta p is applied,
// r^T r of the updated residual summed, and p transformed.
// Shared memory: V [nvec][n_vs] (staged vector slices) | tw [P] | F [npl][RS].
template <int PC, int MODE>
__global__ void __launch_bounds__(kThreads, 2)
k_rows_fwd_pp(MvmGeom g, MaskTables mt, int items, const float* __restrict__ x, CgVecs cg,
              const FrameState* __restrict__ st, float2* __restrict__ X1T, const float2* __restrict__ twg) {
    using C = float2;
    constexpr int P = PC, RS = P | 1;
    constexpr int NVEC = MODE == 1 ? 4 : 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[kWarps];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int ok;
    const int n = g.n, nh = g.nh, NPi = g.NPin, nvs = mt.n_vs;
    const int npl = (n + 1) / 2;
    float* V = reinterpret_cast<float*>(smem_raw);     // MODE 1: p | r | Ap | x; MODE 0: x
    C* tw = reinterpret_cast<C*>(V + NVEC * nvs);
    C* F = tw + P;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t vbytes = (uint32_t)(nvs * sizeof(float));
    auto fetch = [&](int item) {
        const size_t o = (size_t)item * nvs;
        if (MODE == 1) {
            bulk_load(V, cg.p + o, vbytes, &bar);
            bulk_load_more(V + nvs, cg.r + o, vbytes, &bar);
            bulk_load_more(V + 2 * nvs, cg.Ap + o, vbytes, &bar);
            bulk_load_more(V + 3 * nvs, cg.x + o, vbytes, &bar);
        } else {
            bulk_load(V, x + o, vbytes, &bar);
        }
    };
    int t = blockIdx.x;
    while (t < items && !item_active(st, t, NPi)) t += gridDim.x;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = twg[i];
    __syncthreads();
    if (t >= items) return;
    if (threadIdx.x == 0) fetch(t);
    uint32_t parity = 0;
    const int n4 = nvs >> 2;
    const int4* __restrict__ rc4 = reinterpret_cast<const int4*>(mt.rowcol);
    auto put = [&](int rc, float v) {
        const int row = rc >> 16, col = rc & 0xffff;
        reinterpret_cast<float*>(F + (row >> 1) * RS + col)[row & 1] = v;
    };
    while (t < items) {
        const int f = t / NPi;
        // only the first n columns are read by the pruned row transforms
        for (int j = warp; j < npl; j += kWarps)
            for (int c = lane; c < n; c += 32) F[j * RS + c] = make_float2(0.f, 0.f);
        if (!block_wait(&bar, parity, &ok)) return;    // (includes the barrier that orders the zeroing)
        parity ^= 1u;
        const size_t vb = (size_t)t * nvs;
        float rr = 0.f;                                   // per thread FP32 (~16 products), FP64 across
        // four consecutive entries per thread and step, the mask entries of
        // two steps loaded ahead (the vector stores below may alias nothing
        // the loads read, but the compiler cannot know that)
        constexpr int U = 2;
        if (MODE == 1) {
            const float alpha = (float)st[f].alpha, beta = (float)st[f].beta;
            const float4* Vp = reinterpret_cast<const float4*>(V);
            const float4* Vr = Vp + n4;
            const float4* VAp = Vp + 2 * n4;
            const float4* Vx = Vp + 3 * n4;
            float4* x4 = reinterpret_cast<float4*>(cg.x + vb);
            float4* r4 = reinterpret_cast<float4*>(cg.r + vb);
            float4* p4 = reinterpret_cast<float4*>(cg.p + vb);
            for (int i0 = threadIdx.x; i0 < n4; i0 += U * blockDim.x) {
                int4 rc[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (i0 + u * (int)blockDim.x < n4) rc[u] = __ldg(rc4 + i0 + u * blockDim.x);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * blockDim.x;
                    if (i >= n4) continue;
                    const float4 pe = Vp[i];
                    float4 re = Vr[i];
                    if (alpha != 0.f) {
                        const float4 ap = VAp[i], xv = Vx[i];
                        x4[i] = make_float4(xv.x + alpha * pe.x, xv.y + alpha * pe.y, xv.z + alpha * pe.z,
                                            xv.w + alpha * pe.w);
                        re.x -= alpha * ap.x;
                        re.y -= alpha * ap.y;
                        re.z -= alpha * ap.z;
                        re.w -= alpha * ap.w;
                        r4[i] = re;
                    }
                    const float4 pn = make_float4(re.x + beta * pe.x, re.y + beta * pe.y, re.z + beta * pe.z,
                                                  re.w + beta * pe.w);
                    p4[i] = pn;
                    rr = fmaf(re.x, re.x, rr);
                    rr = fmaf(re.y, re.y, rr);
                    rr = fmaf(re.z, re.z, rr);
                    rr = fmaf(re.w, re.w, rr);
                    put(rc[u].x, pn.x);
                    put(rc[u].y, pn.y);
                    put(rc[u].z, pn.z);
                    put(rc[u].w, pn.w);
                }
            }
        } else {
            const float4* V4 = reinterpret_cast<const float4*>(V);
            for (int i0 = threadIdx.x; i0 < n4; i0 += U * blockDim.x) {
                int4 rc[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (i0 + u * (int)blockDim.x < n4) rc[u] = __ldg(rc4 + i0 + u * blockDim.x);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * blockDim.x;
                    if (i >= n4) continue;
                    const float4 v = V4[i];
                    put(rc[u].x, v.x);
                    put(rc[u].y, v.y);
                    put(rc[u].z, v.z);
                    put(rc[u].w, v.w);
                }
            }
        }
        __syncthreads();
        // the next active plane's vectors stream in while this one is transformed
        int tn = t + gridDim.x;
        while (tn < items && !item_active(st, tn, NPi)) tn += gridDim.x;
        if (threadIdx.x == 0 && tn < items) {
            fence_async_shared();
            fetch(tn);
        }
        for (int g0 = warp * kPPRound; g0 < npl; g0 += kWarps * kPPRound)
            fft_rounds<PC, C, true, kPPRound>(F + g0 * RS, RS, min(kPPRound, npl - g0), g.plan, tw, nullptr, lane, n,
                                              P);
        if (MODE == 1) {
            const double s = bsum32(rr, red);
            if (threadIdx.x == 0) cg.rr_part[t] = s;
        }
        __syncthreads();
        // unpack the two real spectra of each pair, A = (Z_k + conj Z_{P-k})/2,
        // B = (Z_k - conj Z_{P-k})/(2i), and write them column-major [kx][row]
        C* out = X1T + (size_t)t * nh * n;
        for (int k = warp; k < nh; k += kWarps) {
            const int kc = k == 0 ? 0 : P - k;
            for (int j = lane; j < npl; j += 32) {
                const C zk = F[j * RS + k];
                const C zc = cconj(F[j * RS + kc]);
                const C dd = csub(zk, zc);
                out[(size_t)k * n + 2 * j] = cscale(cadd(zk, zc), 0.5f);
                if (2 * j + 1 < n) out[(size_t)k * n + 2 * j + 1] = make_float2(0.5f * dd.y, -0.5f * dd.x);
            }
        }
        __syncthreads();                       // F is cleared for the next plane
        t = tn;
    }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// TOMO_ROWS_PP selects the persistent forms: unset or 3 both, 1 the row-inverse
// pass only, 2 the row-forward pass only, 0 neither (the plain kernels).
int pp_mask() {
    static const int mask = [] {
        const char* e = std::getenv("TOMO_ROWS_PP");
        return e == nullptr ? 3 : (std::atoi(e) & 3);
    }();
    return mask;
}

template <typename K>
int grid_for(K kern, size_t smem, int items) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem) != cudaSuccess || per < 1)
        return 0;
    return std::min(items, sms * per);
}

size_t inv_smem(const MvmGeom& g) {
    const int P = g.plan.P;
    return sizeof(float2) * ((size_t)g.nh * g.m + P + (size_t)((g.m + 1) / 2) * (P | 1));
}

size_t fwd_smem(const MvmGeom& g, int nvs, int nvec) {
    const int P = g.plan.P;
    return sizeof(float) * (size_t)nvec * nvs + sizeof(float2) * ((size_t)P + (size_t)((g.n + 1) / 2) * (P | 1));
}

}  // namespace

cudaError_t rows_inv_pp(const Launch& L, const MvmGeom& g, const MaskTables& mt, int B, const FrameState* st,
                        const float2* Y1T, const float* xin, const double* noise_var, const double2* fscale,
                        float* y, const CgVecs* cg, const float2* tw, int max_smem, bool* used) {
    *used = false;
    const int P = g.plan.P;
    if (!(pp_mask() & 1) || B < 1 || !has_fused_plan(P)) return cudaSuccess;
    const size_t slab_bytes = sizeof(float2) * (size_t)g.nh * g.m;
    if (slab_bytes % 16 != 0 || (mt.n_vs & 3) != 0 || !aligned16(Y1T) || !aligned16(y) || !aligned16(mt.rowcol))
        return cudaSuccess;
    if (xin && !aligned16(xin)) return cudaSuccess;
    if (cg && !aligned16(cg->mode == 3 ? cg->Ap : cg->r)) return cudaSuccess;
    const size_t smem = inv_smem(g);
    if (smem > (size_t)max_smem) return cudaSuccess;
    const CgVecs cgv = cg ? *cg : CgVecs{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr};
    const int items = B * g.NPout;
    int grid = 0;
#define TOMO_L(PC)                                                                                          \
    {                                                                                                       \
        grid = grid_for(k_rows_inv_pp<PC>, smem, items);                                                    \
        if (grid > 0)                                                                                       \
            k_rows_inv_pp<PC><<<grid, kThreads, smem, L.stream>>>(g, mt, items, st, Y1T, xin, noise_var, fscale, \
                                                                   y, cgv, tw);                             \
    }
    switch (P) {
        case 150: TOMO_L(150); break;
        case 180: TOMO_L(180); break;
        case 160: TOMO_L(160); break;
        case 40: TOMO_L(40); break;
        case 32: TOMO_L(32); break;
        default: return cudaSuccess;
    }
#undef TOMO_L
    if (grid == 0) return cudaSuccess;
    bump(L);
    *used = true;
    return cudaGetLastError();
}

cudaError_t rows_fwd_pp(const Launch& L, const MvmGeom& g, const MaskTables& mt, int B, const float* x,
                        const CgVecs* cg, const FrameState* st, float2* X1T, const float2* tw, int max_smem,
                        bool* used) {
    *used = false;
    const int P = g.plan.P;
    if (!(pp_mask() & 2) || B < 1 || !has_fused_plan(P) || (mt.n_vs & 3) != 0 || !aligned16(X1T) ||
        !aligned16(mt.rowcol))
        return cudaSuccess;
    const int mode = cg && cg->p ? cg->mode : 0;
    if (mode != 0 && mode != 1) return cudaSuccess;
    if (mode == 1 && !(aligned16(cg->p) && aligned16(cg->r) && aligned16(cg->Ap) && aligned16(cg->x)))
        return cudaSuccess;
    if (mode == 0 && !aligned16(x)) return cudaSuccess;
    const size_t smem = fwd_smem(g, mt.n_vs, mode == 1 ? 4 : 1);
    if (smem > (size_t)max_smem) return cudaSuccess;
    const CgVecs cgv = cg ? *cg : CgVecs{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr};
    const int items = B * g.NPin;
    int grid = 0;
#define TOMO_L(PC)                                                                                         \
    {                                                                                                      \
        if (mode == 1) {                                                                                   \
            grid = grid_for(k_rows_fwd_pp<PC, 1>, smem, items);                                            \
            if (grid > 0)                                                                                  \
                k_rows_fwd_pp<PC, 1><<<grid, kThreads, smem, L.stream>>>(g, mt, items, x, cgv, st, X1T, tw); \
        } else {                                                                                           \
            grid = grid_for(k_rows_fwd_pp<PC, 0>, smem, items);                                            \
            if (grid > 0)                                                                                  \
                k_rows_fwd_pp<PC, 0><<<grid, kThreads, smem, L.stream>>>(g, mt, items, x, cgv, st, X1T, tw); \
        }                                                                                                  \
    }
    switch (P) {
        case 150: TOMO_L(150); break;
        case 180: TOMO_L(180); break;
        case 160: TOMO_L(160); break;
        case 40: TOMO_L(40); break;
        case 32: TOMO_L(32); break;
        default: return cudaSuccess;
    }
#undef TOMO_L
    if (grid == 0) return cudaSuccess;
    bump(L);
    *used = true;
    return cudaGetLastError();
}

cudaError_t init_rows_pp_attributes(int dyn) {
    // the composite radices' twiddle tables are __constant__ data of each
    // translation unit that includes fft_group.cuh: fill this unit's copy
    cudaError_t e = init_fft_constants();
#define TOMO_A(PC)                                                                                              \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rows_inv_pp<PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn); \
    if (e == cudaSuccess)                                                                                       \
        e = cudaFuncSetAttribute(k_rows_fwd_pp<PC, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);        \
    if (e == cudaSuccess)                                                                                       \
        e = cudaFuncSetAttribute(k_rows_fwd_pp<PC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    TOMO_A(150)
    TOMO_A(180)
    TOMO_A(160)
    TOMO_A(40)
    TOMO_A(32)
#undef TOMO_A
    return e;
}

cudaError_t take_wait_error(int* flag) {
    *flag = 0;
    cudaError_t e = cudaMemcpyFromSymbol(flag, g_wait_error, sizeof(int));
    if (e != cudaSuccess || *flag == 0) return e;
    const int zero = 0;
    return cudaMemcpyToSymbol(g_wait_error, &zero, sizeof(int));
}

}  // namespace tomo
