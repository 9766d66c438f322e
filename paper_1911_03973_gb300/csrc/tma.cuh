// TMA bulk copies, mbarriers, grid barriers and block reductions used by the
// persistent kernels of libebe.so (sm_103a, inline PTX).
#pragma once

#include <cstdint>

namespace ebe {
namespace tma {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One arrival that also announces `bytes` of asynchronous copies.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait on an mbarrier phase: gives up after 2^24 polls (each poll may
// suspend the thread for a hardware-chosen time) and sets *err.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase, int32_t* err) {
    for (int it = 0; it < (1 << 24); ++it)
        if (mbar_try_wait(bar, phase)) return true;
    if (err != nullptr) atomicExch(err, 1);
    return false;
}
// L2 policy for data read once per pass: evict first.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// 1D bulk copy global -> shared on the TMA engine, completing on an mbarrier.
// dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(pol)
        : "memory");
}

// Bulk prefetch of global memory into L2 (no completion to wait for).
// src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Atomic add with acquire-release semantics at GPU scope: publishes the
// calling thread's earlier writes (and, through a preceding __syncthreads,
// its CTA's) to whoever later acquires this location, and makes visible to
// the caller everything published by earlier arrivals.
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch: bar[0] counts arrivals, bar[1]
// is the generation.  After a __syncthreads, thread 0 of each CTA arrives
// with an acquire-release atomic (publishing the CTA's writes) and waits
// with acquire loads for the generation to move on; the last CTA to arrive
// resets the count and releases the next generation.  The wait is bounded:
// after limit_ns of global time, or as soon as *err is nonzero, the CTA
// stops waiting and sets *err (2 = barrier timeout).  Returns false in every thread of a CTA that must
// stop (a timeout or an error raised anywhere); every CTA that gets past the
// barrier sees the same *err, so the decision is uniform.
__device__ __forceinline__ bool grid_sync(uint32_t* bar, uint32_t nblocks, int32_t* err, volatile int* sflag,
                                          uint64_t limit_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint32_t gen = ld_acquire(bar + 1);
        const uint32_t arrived = atom_add_acq_rel(bar, 1u);
        if (arrived == nblocks - 1) {
            st_relaxed(bar, 0u);
            st_release(bar + 1, gen + 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            uint32_t polls = 0;
            while (ld_acquire(bar + 1) == gen) {
                if ((++polls & 31u) == 0u) {
                    if (*reinterpret_cast<volatile int32_t*>(err) != 0) { ok = 0; break; }
                    if (globaltimer_ns() - t0 > limit_ns) { atomicExch(err, 2); ok = 0; break; }
                }
            }
        }
        if (ok && *reinterpret_cast<volatile int32_t*>(err) != 0) ok = 0;
        *sflag = ok;
    }
    __syncthreads();
    return *sflag != 0;
}

// Sum over a CTA of NT threads in a fixed order (warp butterflies, then warp
// 0 over the per-warp sums).  Every thread must call it; the result is valid
// in thread 0.  red: NT / 32 doubles of shared memory.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (w == 0) {
        s = lane < NT / 32 ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

// Two sums at once; red: 2 NT / 32 doubles.
template <int NT>
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) { red[w] = a; red[NT / 32 + w] = b; }
    __syncthreads();
    if (w == 0) {
        a = lane < NT / 32 ? red[lane] : 0.0;
        b = lane < NT / 32 ? red[NT / 32 + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
    }
}

}  // namespace tma
}  // namespace ebe
