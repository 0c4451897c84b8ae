// Radix-fused, in-place FFTs of several sequences per warp (included by
// kernels.cu only).
//
// A length-P transform is factored into few composite radices (150 = 15 x 10,
// 180 = 12 x 15, 160 = 10 x 16, 40 = 8 x 5, 32 = 4 x 8).  Each Stockham stage
// (same ordering as fft.cuh) reads its inputs into registers, synchronises the
// warp, and writes the outputs back in place, so a 150-point transform costs
// two shared-memory round trips instead of four and needs no scratch buffer.
// gstage does this for G sequences at once; cstage in rounds of whole
// sequences, which lets one call take more sequences than the lanes of one
// round hold.  A composite radix R = R1 R2 is itself evaluated in
// registers as two small DFTs with the inner twiddles w_R^{b s} (the same
// two-factor decomposition, Cooley & Tukey 1965), read from __constant__
// tables that init_fft_constants() fills once.
#pragma once

#include "fft.cuh"

namespace tomo {

// exp(-2 pi i m / R), m in [0, R), for the composite radices
#define TOMO_TW_TABLE(R)                 \
    __constant__ float2 c_twf##R[R];     \
    __constant__ double2 c_twd##R[R];
TOMO_TW_TABLE(6)
TOMO_TW_TABLE(8)
TOMO_TW_TABLE(9)
TOMO_TW_TABLE(10)
TOMO_TW_TABLE(12)
TOMO_TW_TABLE(15)
TOMO_TW_TABLE(16)
#undef TOMO_TW_TABLE

template <typename C, int R> struct CTw;
#define TOMO_TW_ACCESS(R)                                                                    \
    template <> struct CTw<float2, R> {                                                      \
        __device__ __forceinline__ static float2 get(int m) { return c_twf##R[m]; }          \
    };                                                                                       \
    template <> struct CTw<double2, R> {                                                     \
        __device__ __forceinline__ static double2 get(int m) { return c_twd##R[m]; }         \
    };
TOMO_TW_ACCESS(6)
TOMO_TW_ACCESS(8)
TOMO_TW_ACCESS(9)
TOMO_TW_ACCESS(10)
TOMO_TW_ACCESS(12)
TOMO_TW_ACCESS(15)
TOMO_TW_ACCESS(16)
#undef TOMO_TW_ACCESS

// DFT of size R1*R2 in registers: DFTs of size R1 over the stride-R2
// subsequences, inner twiddles, DFTs of size R2; output index s + t R1.
template <typename C, int R1, int R2, bool FWD>
__device__ __forceinline__ void dft_composite(C* v) {
    constexpr int R = R1 * R2;
    C w[R];
#pragma unroll
    for (int b = 0; b < R2; ++b) {
        C u[R1];
#pragma unroll
        for (int a = 0; a < R1; ++a) u[a] = v[b + a * R2];
        SmallDft<C, R1>::run(u, FWD);
#pragma unroll
        for (int s = 0; s < R1; ++s) w[b * R1 + s] = u[s];
    }
#pragma unroll
    for (int b = 1; b < R2; ++b)
#pragma unroll
        for (int s = 1; s < R1; ++s) {
            C t = CTw<C, R>::get((b * s) % R);
            if (!FWD) t = cconj(t);
            w[b * R1 + s] = cmul(w[b * R1 + s], t);
        }
#pragma unroll
    for (int s = 0; s < R1; ++s) {
        C u[R2];
#pragma unroll
        for (int b = 0; b < R2; ++b) u[b] = w[b * R1 + s];
        SmallDft<C, R2>::run(u, FWD);
#pragma unroll
        for (int t = 0; t < R2; ++t) v[s + t * R1] = u[t];
    }
}

template <typename C, int R, bool FWD> struct Dft {
    __device__ __forceinline__ static void run(C* v) { SmallDft<C, R>::run(v, FWD); }
};
template <typename C, bool FWD> struct Dft<C, 6, FWD> {
    __device__ __forceinline__ static void run(C* v) { dft_composite<C, 3, 2, FWD>(v); }
};
template <typename C, bool FWD> struct Dft<C, 8, FWD> {
    __device__ __forceinline__ static void run(C* v) { dft_composite<C, 4, 2, FWD>(v); }
};
template <typename C, bool FWD> struct Dft<C, 9, FWD> {
    __device__ __forceinline__ static void run(C* v) { dft_composite<C, 3, 3, FWD>(v); }
};
template <typename C, bool FWD> struct Dft<C, 10, FWD> {
    __device__ __forceinline__ static void run(C* v) { dft_composite<C, 5, 2, FWD>(v); }
};
template <typename C, bool FWD> struct Dft<C, 12, FWD> {
    __device__ __forceinline__ static void run(C* v) { dft_composite<C, 4, 3, FWD>(v); }
};
template <typename C, bool FWD> struct Dft<C, 15, FWD> {
    __device__ __forceinline__ static void run(C* v) { dft_composite<C, 5, 3, FWD>(v); }
};
template <typename C, bool FWD> struct Dft<C, 16, FWD> {
    __device__ __forceinline__ static void run(C* v) { dft_composite<C, 4, 4, FWD>(v); }
};

// One in-place Stockham stage over G sequences at base + g * gstride.  In the
// first stage (Ns = 1) only inputs with index < nin are read (the rest are
// known zeros: the transforms here zero-pad an n-point grid to P); in the last
// stage (LAST) only outputs with index < nout are written back.
template <typename C, int P, int G, int Ns, int R, bool FWD, bool LAST>
__device__ __forceinline__ void gstage(C* base, int gstride, const C* __restrict__ tw, int lane, int nin, int nout) {
    constexpr int PR = P / R;
    constexpr int TT = G * PR;
    constexpr int RD = (TT + 31) / 32;
    constexpr int tstep = P / (Ns * R);
    C v[RD][R];
#pragma unroll
    for (int rd = 0; rd < RD; ++rd) {
        const int t = lane + 32 * rd;
        if (t < TT) {
            const int g = t / PR, j = t - g * PR, k = j % Ns;
            const C* b = base + g * gstride;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (Ns == 1) v[rd][r] = j + r * PR < nin ? b[j + r * PR] : cmk<C>(0, 0);
                else v[rd][r] = b[j + r * PR];
            }
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C w = tw[r * k * tstep];
                    if (!FWD) w = cconj(w);
                    v[rd][r] = cmul(v[rd][r], w);
                }
            }
            Dft<C, R, FWD>::run(v[rd]);
        }
    }
    __syncwarp();
#pragma unroll
    for (int rd = 0; rd < RD; ++rd) {
        const int t = lane + 32 * rd;
        if (t < TT) {
            const int g = t / PR, j = t - g * PR, k = j % Ns;
            const int o = (j / Ns) * Ns * R + k;
            C* b = base + g * gstride + o;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (!LAST || o + r * Ns < nout) b[r * Ns] = v[rd][r];
        }
    }
    __syncwarp();
}

// The same stage over count <= GG sequences, one round of whole sequences at a
// time: a round gives SPR = floor(32 / (P / R)) sequences one lane per
// butterfly, reads, synchronises the warp and writes back.  As no sequence
// spans two rounds, only one round's data is held in registers (the stage
// above keeps all of them across its single synchronisation), so large groups
// cost no registers; for 150 = 15 x 10 a group of six fills 30 of 32 lanes in
// both stages (rounds of three and of two sequences).  Sequences >= count are
// skipped.
template <typename C, int P, int GG, int Ns, int R, bool FWD, bool LAST>
__device__ __forceinline__ void cstage(C* base, int gstride, int count, const C* __restrict__ tw, int lane, int nin,
                                       int nout) {
    constexpr int PR = P / R;
    static_assert(PR <= 32, "one sequence's butterflies must fit a warp");
    constexpr int SPR = 32 / PR;
    constexpr int tstep = P / (Ns * R);
    const int gl = lane / PR, j = lane - gl * PR, k = j % Ns;
    const int o = (j / Ns) * Ns * R + k;
#pragma unroll 1
    for (int g0 = 0; g0 < GG; g0 += SPR) {
        if (g0 >= count) break;                    // warp-uniform
        const int g = g0 + gl;
        const bool on = gl < SPR && g < count;
        C v[R];
        if (on) {
            const C* b = base + g * gstride;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (Ns == 1) v[r] = j + r * PR < nin ? b[j + r * PR] : cmk<C>(0, 0);
                else v[r] = b[j + r * PR];
            }
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C w = tw[r * k * tstep];
                    if (!FWD) w = cconj(w);
                    v[r] = cmul(v[r], w);
                }
            }
            Dft<C, R, FWD>::run(v);
        }
        __syncwarp();
        if (on) {
            C* b = base + g * gstride + o;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (!LAST || o + r * Ns < nout) b[r * Ns] = v[r];
        }
        __syncwarp();
    }
}

template <typename C, int P, int GG, int Ns, bool FWD, int... Rs> struct CStages;
template <typename C, int P, int GG, int Ns, bool FWD> struct CStages<C, P, GG, Ns, FWD> {
    __device__ __forceinline__ static void run(C*, int, int, const C*, int, int, int) {}
};
template <typename C, int P, int GG, int Ns, bool FWD, int R, int... Rest>
struct CStages<C, P, GG, Ns, FWD, R, Rest...> {
    __device__ __forceinline__ static void run(C* base, int gstride, int count, const C* tw, int lane, int nin,
                                               int nout) {
        cstage<C, P, GG, Ns, R, FWD, sizeof...(Rest) == 0>(base, gstride, count, tw, lane, nin, nout);
        CStages<C, P, GG, Ns * R, FWD, Rest...>::run(base, gstride, count, tw, lane, nin, nout);
    }
};

template <typename C, int P, int G, int Ns, bool FWD, int... Rs> struct GStages;
template <typename C, int P, int G, int Ns, bool FWD> struct GStages<C, P, G, Ns, FWD> {
    __device__ __forceinline__ static void run(C*, int, const C*, int, int, int) {}
};
template <typename C, int P, int G, int Ns, bool FWD, int R, int... Rest> struct GStages<C, P, G, Ns, FWD, R, Rest...> {
    __device__ __forceinline__ static void run(C* base, int gstride, const C* tw, int lane, int nin, int nout) {
        gstage<C, P, G, Ns, R, FWD, sizeof...(Rest) == 0>(base, gstride, tw, lane, nin, nout);
        GStages<C, P, G, Ns * R, FWD, Rest...>::run(base, gstride, tw, lane, nin, nout);
    }
};

#ifndef TOMO_FFT_GROUP
#define TOMO_FFT_GROUP 2
#endif
constexpr int kFftGroup = TOMO_FFT_GROUP;   // sequences per warp and call

// Fused plans for the transform sizes of the workloads; other sizes use the
// generic Stockham path of fft.cuh, one sequence at a time.
template <int P> struct Fused { static constexpr bool ok = false; };
#define TOMO_FUSED(P_, ...)                                                                   \
    template <> struct Fused<P_> {                                                            \
        static constexpr bool ok = true;                                                      \
        template <typename C, bool FWD, int GG>                                               \
        __device__ __forceinline__ static void run(C* base, int gstride, const C* tw, int lane, int nin, \
                                                   int nout) {                                \
            GStages<C, P_, GG, 1, FWD, __VA_ARGS__>::run(base, gstride, tw, lane, nin, nout);   \
        }                                                                                     \
        template <typename C, bool FWD, int GG>                                               \
        __device__ __forceinline__ static void run_rounds(C* base, int gstride, int count, const C* tw, int lane, \
                                                          int nin, int nout) {                \
            CStages<C, P_, GG, 1, FWD, __VA_ARGS__>::run(base, gstride, count, tw, lane, nin, nout); \
        }                                                                                     \
    };
#ifndef TOMO_PLAN_150_ID
#define TOMO_PLAN_150_ID 3
#endif
#if TOMO_PLAN_150_ID == 1
#define TOMO_PLAN_150 5, 5, 3, 2
#elif TOMO_PLAN_150_ID == 2
#define TOMO_PLAN_150 5, 5, 6
#elif TOMO_PLAN_150_ID == 3
#define TOMO_PLAN_150 15, 10
#elif TOMO_PLAN_150_ID == 4
#define TOMO_PLAN_150 10, 5, 3
#else
#define TOMO_PLAN_150 10, 15
#endif
#ifndef TOMO_PLAN_180
#define TOMO_PLAN_180 12, 15
#endif
TOMO_FUSED(150, TOMO_PLAN_150)
TOMO_FUSED(180, TOMO_PLAN_180)
TOMO_FUSED(160, 10, 16)
TOMO_FUSED(40, 8, 5)
TOMO_FUSED(32, 4, 8)
#undef TOMO_FUSED

// Launch-side dispatch on the transform size: F(PC) is expanded with the
// compile-time size, or 0 for the generic path.
#define TOMO_DISPATCH_P(P, F) \
    switch (P) {              \
        case 150: F(150); break; \
        case 180: F(180); break; \
        case 160: F(160); break; \
        case 40: F(40); break;   \
        case 32: F(32); break;   \
        default: F(0); break;    \
    }

// Host side: true if P has a fused plan (then the generic scratch is unused).
inline bool has_fused_plan(int P) { return P == 150 || P == 180 || P == 160 || P == 40 || P == 32; }

// Transforms GG sequences base[g * gstride + 0..P) in place with one warp
// (the fused plans transform all GG; the generic path only the first count);
// PC is the compile-time size (0: generic, through scratch[0..P)).  Only the
// first nin inputs may be non-zero (the others are not read) and only the
// first nout outputs are needed (the others may be left unwritten) -- the
// generic path reads and writes everything.  The warp must be converged and
// the data visible on entry; ends with __syncwarp().  More sequences per call
// fill more lanes: a stage of radix R runs GG P / R butterflies over 32 lanes.
template <int PC, typename C, bool FWD, int GG = kFftGroup>
__device__ __forceinline__ void fft_g(C* base, int gstride, int count, const FftPlan& pl, const C* tw, C* scratch,
                                      int lane, int nin, int nout) {
    if constexpr (Fused<PC>::ok) {
        Fused<PC>::template run<C, FWD, GG>(base, gstride, tw, lane, nin, nout);
    } else {
        for (int gi = 0; gi < GG && gi < count; ++gi)
            fft_warp<C>(base + gi * gstride, scratch, pl, tw, FWD, lane, 32);
    }
}

// As fft_g, for up to GG sequences (count <= GG of them) in rounds of whole
// sequences (cstage): any group size at the registers of one round.
template <int PC, typename C, bool FWD, int GG>
__device__ __forceinline__ void fft_rounds(C* base, int gstride, int count, const FftPlan& pl, const C* tw,
                                           C* scratch, int lane, int nin, int nout) {
    if constexpr (Fused<PC>::ok) {
        Fused<PC>::template run_rounds<C, FWD, GG>(base, gstride, count, tw, lane, nin, nout);
    } else {
        for (int gi = 0; gi < GG && gi < count; ++gi)
            fft_warp<C>(base + gi * gstride, scratch, pl, tw, FWD, lane, 32);
    }
}

// Fills the __constant__ twiddle tables (host side, once per device).  The
// library is compiled without relocatable device code, so every translation
// unit that includes this header has its own tables and must call this; the
// function is static so that each unit's call fills that unit's tables (an
// inline function would be merged into one definition by the linker).
static cudaError_t init_fft_constants() {
    const double pi = 3.14159265358979323846;
    cudaError_t e = cudaSuccess;
#define TOMO_TW_FILL(R)                                                                  \
    {                                                                                    \
        float2 f[R];                                                                     \
        double2 d[R];                                                                    \
        for (int m = 0; m < R; ++m) {                                                    \
            const double a = -2.0 * pi * m / R;                                          \
            d[m] = make_double2(std::cos(a), std::sin(a));                               \
            f[m] = make_float2((float)d[m].x, (float)d[m].y);                            \
        }                                                                                \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_twf##R, f, sizeof(f));            \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_twd##R, d, sizeof(d));            \
    }
    TOMO_TW_FILL(6)
    TOMO_TW_FILL(8)
    TOMO_TW_FILL(9)
    TOMO_TW_FILL(10)
    TOMO_TW_FILL(12)
    TOMO_TW_FILL(15)
    TOMO_TW_FILL(16)
#undef TOMO_TW_FILL
    return e;
}

}  // namespace tomo
