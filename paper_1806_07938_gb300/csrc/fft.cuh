// Shared-memory mixed-radix Stockham FFT used by every kernel of the library.
//
// One warp transforms one complex sequence of length P = r_1 r_2 ... r_s
// (radices 2, 3, 4, 5, 7), ping-ponging between two shared-memory buffers.
// Stage with radix R after Ns = r_1...r_{t-1}: for j in [0, P/R), k = j mod Ns,
// the R inputs in[j + r P/R] are multiplied by w_P^{r k P/(Ns R)}, pass through
// an R-point DFT, and land at out[(j/Ns) Ns R + k + r Ns] (the self-sorting
// Stockham ordering; Govindaraju et al., "High performance discrete Fourier
// transforms on graphics processors", SC 2008).
//
// Sign convention: forward = exp(-2 pi i k m / P), inverse = exp(+...),
// both unnormalised.  Twiddles come from a per-block table tw[k] =
// exp(-2 pi i k / P) that the host computes in FP64.
#pragma once

#include <cuda_runtime.h>

namespace tomo {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx_t = typename cplx_of<T>::type;

template <typename C> __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) { C c; c.x = a; c.y = b; return c; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmk<C>(a.x * s, a.y * s); }
// multiply by -i (fwd = true) or +i (fwd = false)
template <typename C> __device__ __forceinline__ C cmul_mi(C a, bool fwd) { return fwd ? cmk<C>(a.y, -a.x) : cmk<C>(-a.y, a.x); }

struct FftPlan {
    int P;        // transform length
    int nst;      // number of stages
    int rad[8];   // radices, in order of application
};

// R-point DFT in registers; fwd selects exp(-2 pi i ...) vs exp(+2 pi i ...).
template <typename C, int R> struct SmallDft;

template <typename C> struct SmallDft<C, 2> {
    __device__ __forceinline__ static void run(C* v, bool) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b); v[1] = csub(a, b);
    }
};

template <typename C> struct SmallDft<C, 3> {
    __device__ __forceinline__ static void run(C* v, bool fwd) {
        using T = decltype(C::x);
        const T s3 = (T)0.86602540378443864676;  // sin(2 pi / 3)
        C t1 = cadd(v[1], v[2]);
        C t2 = cmk<C>(v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y);
        C d = cscale(csub(v[1], v[2]), s3);
        C md = cmul_mi(d, fwd);
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, md);
        v[2] = csub(t2, md);
    }
};

template <typename C> struct SmallDft<C, 4> {
    __device__ __forceinline__ static void run(C* v, bool fwd) {
        C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        C c = cadd(v[1], v[3]), d = cmul_mi(csub(v[1], v[3]), fwd);
        v[0] = cadd(a, c); v[2] = csub(a, c);
        v[1] = cadd(b, d); v[3] = csub(b, d);
    }
};

template <typename C> struct SmallDft<C, 5> {
    __device__ __forceinline__ static void run(C* v, bool fwd) {
        using T = decltype(C::x);
        const T c1 = (T)0.30901699437494742410;   // cos(2 pi / 5)
        const T c2 = (T)-0.80901699437494742410;  // cos(4 pi / 5)
        const T s1 = (T)0.95105651629515357212;   // sin(2 pi / 5)
        const T s2 = (T)0.58778525229247312917;   // sin(4 pi / 5)
        C a1 = cadd(v[1], v[4]), a2 = cadd(v[2], v[3]);
        C b1 = csub(v[1], v[4]), b2 = csub(v[2], v[3]);
        C t1 = cmk<C>(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
        C t2 = cmk<C>(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
        C u1 = cmk<C>(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);
        C u2 = cmk<C>(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);
        C m1 = cmul_mi(u1, fwd), m2 = cmul_mi(u2, fwd);
        v[0] = cadd(v[0], cadd(a1, a2));
        v[1] = cadd(t1, m1); v[4] = csub(t1, m1);
        v[2] = cadd(t2, m2); v[3] = csub(t2, m2);
    }
};

template <typename C> struct SmallDft<C, 7> {
    __device__ __forceinline__ static void run(C* v, bool fwd) {
        using T = decltype(C::x);
        const T cs[3] = {(T)0.62348980185873353053, (T)-0.22252093395631440429, (T)-0.90096886790241912624};
        const T sn[3] = {(T)0.78183148246802980871, (T)0.97492791218182360702, (T)0.43388373911755812048};
        C a[3], b[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) { a[m] = cadd(v[1 + m], v[6 - m]); b[m] = csub(v[1 + m], v[6 - m]); }
        C y0 = cadd(v[0], cadd(a[0], cadd(a[1], a[2])));
        C out[7];
#pragma unroll
        for (int k = 1; k <= 3; ++k) {
            C t = v[0], u = cmk<C>(0, 0);
#pragma unroll
            for (int m = 1; m <= 3; ++m) {
                int km = (k * m) % 7;            // cos(2 pi km/7), sin(2 pi km/7)
                T c = km <= 3 ? cs[km - 1] : cs[7 - km - 1];
                T s = km <= 3 ? sn[km - 1] : -sn[7 - km - 1];
                t.x += c * a[m - 1].x; t.y += c * a[m - 1].y;
                u.x += s * b[m - 1].x; u.y += s * b[m - 1].y;
            }
            C mu = cmul_mi(u, fwd);
            out[k] = cadd(t, mu); out[7 - k] = csub(t, mu);
        }
        v[0] = y0;
#pragma unroll
        for (int k = 1; k < 7; ++k) v[k] = out[k];
    }
};

template <typename C, int R>
__device__ __forceinline__ void stockham_stage(const C* __restrict__ in, C* __restrict__ out, int P, int Ns,
                                               const C* __restrict__ tw, bool fwd, int lane, int nl) {
    const int PR = P / R;
    const int tstep = P / (Ns * R);
    for (int j = lane; j < PR; j += nl) {
        const int k = j % Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[j + r * PR];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[r * k * tstep];
                if (!fwd) w = cconj(w);
                v[r] = cmul(v[r], w);
            }
        }
        SmallDft<C, R>::run(v, fwd);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[base + r * Ns] = v[r];
    }
}

// Transforms buf[0..P) in place (through scratch[0..P)) with the threads of one
// warp (lane in [0, nl)).  Callers must __syncwarp() before (data written) and
// may read buf after this returns (it ends with __syncwarp()).
template <typename C>
__device__ void fft_warp(C* buf, C* scratch, const FftPlan& pl, const C* tw, bool fwd, int lane, int nl) {
    C* src = buf;
    C* dst = scratch;
    int Ns = 1;
    for (int s = 0; s < pl.nst; ++s) {
        const int R = pl.rad[s];
        switch (R) {
            case 2: stockham_stage<C, 2>(src, dst, pl.P, Ns, tw, fwd, lane, nl); break;
            case 3: stockham_stage<C, 3>(src, dst, pl.P, Ns, tw, fwd, lane, nl); break;
            case 4: stockham_stage<C, 4>(src, dst, pl.P, Ns, tw, fwd, lane, nl); break;
            case 5: stockham_stage<C, 5>(src, dst, pl.P, Ns, tw, fwd, lane, nl); break;
            default: stockham_stage<C, 7>(src, dst, pl.P, Ns, tw, fwd, lane, nl); break;
        }
        __syncwarp();
        Ns *= R;
        C* t = src; src = dst; dst = t;
    }
    if (src != buf) {
        for (int j = lane; j < pl.P; j += nl) buf[j] = src[j];
        __syncwarp();
    }
}

}  // namespace tomo
