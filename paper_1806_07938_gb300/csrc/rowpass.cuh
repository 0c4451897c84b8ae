// Pieces shared by the row passes of kernels.cu and their persistent,
// bulk-prefetching forms in rows_pp.cu (included by those two files only).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fft.cuh"

namespace tomo {

// Row pair (2j, 2j+1) of a plane is held as one complex sequence
// z = row_2j + i row_2j+1 in F[j][0..P); rows are padded to an odd stride so
// that the column-wise accesses of the transposed write are conflict-free.
__host__ __device__ constexpr int row_stride(int P) { return P | 1; }

// Stores the full-spectrum entries k and P - k of packed row pair j from the
// half-spectrum values a = A_k, b = B_k of its two rows (Hermitian extension;
// DC and Nyquist taken real), so that one inverse complex FFT returns row 2j
// in .x and row 2j+1 in .y.
template <typename C>
__device__ __forceinline__ void put_row_pair(C* F, int RS, int P, int j, int k, C a, C b) {
    if (k == 0 || 2 * k == P) { a.y = 0; b.y = 0; }
    F[j * RS + k] = cmk<C>(a.x - b.y, a.y + b.x);
    if (k != 0 && 2 * k != P) {
        const C ac = cconj(a), bc = cconj(b);
        F[j * RS + P - k] = cmk<C>(ac.x - bc.y, ac.y + bc.x);
    }
}

// --- bulk asynchronous copies global -> shared with an mbarrier -------------
// (PTX ISA: cp.async.bulk, mbarrier).  One thread arms the barrier with the
// byte count and issues the copy; every thread that needs the data waits on
// the barrier's phase.  Waits are bounded: a copy that has not landed after
// kMaxWaitPolls polls (seconds) is reported through the error flag instead of
// hanging the GPU.
constexpr long long kMaxWaitPolls = 1LL << 24;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses (after a block barrier:
// every thread's) before the asynchronous copies it issues next.
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Arms the barrier for `bytes` more bytes and copies them (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Adds more bytes to the current phase (after bulk_load armed it): for a
// phase fed by several copies, each extra copy goes through bulk_load_more.
__device__ __forceinline__ void bulk_load_more(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Starts fetching `bytes` of global memory into L2 (no shared memory, no
// completion to wait for; 16-byte aligned address, size a multiple of 16).
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Waits for the barrier phase with the given parity; false after kMaxWaitPolls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_addr(bar);
    for (long long i = 0; i < kMaxWaitPolls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace tomo
