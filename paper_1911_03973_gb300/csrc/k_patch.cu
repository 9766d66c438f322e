// Patch passes of the element-by-element operator (sm_103a).
//
// A patch is a run of kPatch elements (see plan.cpp); one CTA handles one
// patch and several CTAs share an SM, so that one CTA's copies overlap
// another's arithmetic:
//   * the TMA engine bulk-copies the patch's element matrices (structure of
//     arrays: packed symmetric entry t of the patch's 1024 slots is one
//     contiguous run, n_b(n_b+1)/2 runs) and
//     16-bit local connectivity into shared memory, evict-first in L2; while
//     they are in flight the threads gather the patch's node table, x and b
//     at the patch nodes -- the restriction x_e = R_e x of Algorithm 1,
//     shared by neighbouring elements;
//   * the threads add A_e x_e into per-node shared-memory sums colour by
//     colour: within a colour no two elements share a node, so there are no
//     atomics and the order of the additions is fixed (bitwise reproducible);
//     meshes with many colours per patch (tetrahedra) give each warp its own
//     copy of the sums instead, merged in warp order after one barrier;
//   * they write the result of every owned node (all of its elements are in
//     this patch) and the partial sum of every shared node to its halo slot.
// The fix-up pass adds the halo partials of each shared node in patch order.
#include <algorithm>
#include <cstdint>

#include "device_util.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace ebe {
namespace {

// Dot-product accumulator of a pass: FP64 products for FP64 data; for FP32
// data, FP32 products in a compensated FP32 sum (no FP64 work per node).
template <typename T>
struct DotAcc {
    double d = 0.0;
    __device__ __forceinline__ void add(T a, T b) { d = fmadd(double(a), double(b), d); }
    __device__ __forceinline__ double value() const { return d; }
};
template <>
struct DotAcc<float> {
    CompSum c;
    __device__ __forceinline__ void add(float a, float b) { c.add(a * b); }
    __device__ __forceinline__ double value() const { return c.value(); }
};

// Block total of a pass's dot product, valid in thread 0: FP64 butterflies
// for FP64 data; for FP32 data compensated FP32 butterflies and one FP64
// conversion per warp (per-thread FP64 work would load the FP64 pipe, which
// GB300 runs at 1/64 of the FP32 rate, with millions of operations a pass).
template <int NT>
__device__ __forceinline__ double block_total(const DotAcc<double>& d, double* red) {
    return tma::block_sum<NT>(d.value(), red);
}
template <int NT>
__device__ __forceinline__ double block_total(const DotAcc<float>& d, double* red) {
    CompSum v[1] = {d.c};
    double out[1];
    block_sums_comp<1, NT>(v, out, red);
    return out[0];
}

using tma::block_sum;
using tma::bulk_load;
using tma::bulk_prefetch_l2;
using tma::mbar_expect_tx;
using tma::mbar_init;
using tma::mbar_try_wait;
using tma::mbar_wait_bounded;
using tma::policy_evict_first;
using tma::smem_addr;

// Shared-memory layout of a patch pass.  One patch per CTA: its element
// matrices (n_b(n_b+1)/2 runs of 1024 values) and local connectivity (n_b runs) come
// in by TMA bulk copies; the node table, x and b at the patch nodes by plain
// loads issued while the bulk copies are in flight.
struct PatchSmem {
    uint32_t bar, flag, red, co, A, L, G, xs, bs, acc, total;
};
constexpr int kWarpCopies = 8;   // node-sum copies of the per-warp scheme (one per warp)
template <typename T, int NB, bool WARPS>
__host__ __device__ constexpr PatchSmem patch_layout(int max_nodes) {
    PatchSmem s{};
    const uint32_t gcap = uint32_t((max_nodes + 3) / 4 * 4);
    s.bar = 0;                                          // u64 mbarrier
    s.flag = 8;                                         // int
    s.red = 16;                                         // 32 doubles
    s.co = s.red + 32 * 8;                              // kMaxColours + 1 ints
    s.A = (s.co + (kMaxColours + 1) * 4 + 127) / 128 * 128;
    s.L = s.A + uint32_t(sym_count(NB) * kPatch * sizeof(T));
    s.G = s.L + uint32_t(NB * kPatch * 2);
    s.xs = s.G + gcap * 4;
    s.bs = (s.xs + gcap * uint32_t(sizeof(T)) + 15) / 16 * 16;
    s.acc = (s.bs + gcap * uint32_t(sizeof(T)) + 15) / 16 * 16;
    s.total = (s.acc + (WARPS ? kWarpCopies : 1) * gcap * uint32_t(sizeof(T)) + 127) / 128 * 128;
    return s;
}

constexpr int kPatchThreads = 256;
static_assert(kPatchThreads / 32 == kWarpCopies, "one node-sum copy per warp");

constexpr int kEPT = kPatch / kPatchThreads;     // elements owned by a thread

// The element products A_e x_e of one patch added into the per-node sums acc
// (shared memory) in a fixed order: colour rounds for few colours per patch,
// per-warp copies merged in warp order for many.  xs holds the operand at
// the patch nodes; with colour rounds the caller has zeroed acc[0, n_nodes)
// and synchronised the CTA.  On return acc[l] is node l's sum and the CTA is
// synchronised.
template <typename T, int NB, bool WARPS>
__device__ __forceinline__ void patch_sums(const PatchMeta& m, int max_nodes, const T* __restrict__ As,
                                           const uint16_t* __restrict__ Ls, const T* __restrict__ xs,
                                           T* __restrict__ acc, const int* __restrict__ co, int tid) {
    constexpr int NT = kPatchThreads;
    if constexpr (WARPS) {
        // Many colours (tetrahedra: about 30 per patch) would mean as many
        // block barriers with little work between them.  Instead warp w adds
        // the elements of colours w, w + 8, ... into its own copy of the node
        // sums (a colour's elements share no node; a warp sync separates its
        // colours); after one barrier the node value is the sum of the 8 copies
        // in warp order (a fixed order: bitwise reproducible).
        const int gcap = (max_nodes + 3) / 4 * 4;
        const int warp = tid >> 5, lane = tid & 31;
        T* accw = acc + warp * gcap;
        for (int l = lane; l < m.n_nodes; l += 32) accw[l] = T(0);
        __syncwarp();
        for (int c = warp; c < m.n_col; c += kWarpCopies) {
            const int lo = co[c], hi = co[c + 1];
            for (int s = lo + lane; s < hi; s += 32) {
                int ln[NB];
                T xe[NB];
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    ln[i] = int(Ls[i * kPatch + s]);
                    xe[i] = xs[ln[i]];
                }
                // difference form: the diagonal slot holds the row sum s_r,
                // y_r = s_r x_r + sum_{j != r} a_rj (x_j - x_r)
#pragma unroll
                for (int r = 0; r < NB; ++r) {
                    T v = As[sym_index(NB, r, r) * kPatch + s] * xe[r];
#pragma unroll
                    for (int j = 0; j < NB; ++j)
                        if (j != r) v = fmadd(As[sym_index(NB, r, j) * kPatch + s], xe[j] - xe[r], v);
                    accw[ln[r]] += v;
                }
            }
            __syncwarp();
        }
        __syncthreads();
        for (int l = tid; l < m.n_nodes; l += NT) {
            T v = acc[l];
#pragma unroll
            for (int w = 1; w < kWarpCopies; ++w) v += acc[w * gcap + l];
            acc[l] = v;
        }
        __syncthreads();
    } else {
        // my slots: local node ids and x values in registers
        int ln[kEPT][NB];
        T xe[kEPT][NB];
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            const int s = tid + k * NT;
            const bool ok = s < m.n_el;
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                ln[k][i] = ok ? int(Ls[i * kPatch + s]) : 0;
                xe[k][i] = xs[ln[k][i]];
            }
        }
        // FP32: every thread forms the products of its slots at once, then the
        // colour rounds only add them into the node sums (short rounds).
        // Difference form: the diagonal slot holds the row sum s_r,
        // y_r = s_r x_r + sum_{j != r} a_rj (x_j - x_r); for a smooth x the
        // difference is exact in FP32 and no accuracy is lost to cancellation.
        T y[kEPT][NB];
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            const int s = tid + k * NT;
            const bool ok = s < m.n_el;
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                T v = ok ? As[sym_index(NB, r, r) * kPatch + s] * xe[k][r] : T(0);
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    if (j != r) v = ok ? fmadd(As[sym_index(NB, r, j) * kPatch + s], xe[k][j] - xe[k][r], v) : v;
                y[k][r] = v;
            }
        }
        for (int c = 0; c < m.n_col; ++c) {
            const int lo = co[c], hi = co[c + 1];
#pragma unroll
            for (int k = 0; k < kEPT; ++k) {
                const int s = tid + k * NT;
                if (s >= lo && s < hi) {
#pragma unroll
                    for (int r = 0; r < NB; ++r) acc[ln[k][r]] += y[k][r];
                }
            }
            __syncthreads();
        }
    }

}

// One patch per CTA, several CTAs per SM so that one CTA's copies overlap
// another's arithmetic.  Thread 0 starts the bulk copies; meanwhile all
// threads gather the node table, x and b.  Each thread owns the slots
// tid + 256 k and keeps their local node ids and x values in registers, so a
// colour round only reads the element matrix entries from shared memory and
// updates the node sums.
template <typename T, int NB, int MODE, bool WARPS>
__global__ void __launch_bounds__(kPatchThreads)
k_patch(const PlanDev pd, const T* __restrict__ A, const T* __restrict__ x, const T* __restrict__ b,
        T* __restrict__ out, T* __restrict__ halo, double* __restrict__ part, const int32_t* __restrict__ stop) {
    static_assert(sizeof(T) == 4, "FP64 patch passes use k_patch64d");
    constexpr int NT = kPatchThreads;
    constexpr bool kRes = (MODE == kResidual || MODE == kResidualNorm);
    extern __shared__ __align__(128) unsigned char smem[];
    const PatchSmem L = patch_layout<T, NB, WARPS>(pd.max_nodes);
    volatile int* flag = reinterpret_cast<volatile int*>(smem + L.flag);
    double* red = reinterpret_cast<double*>(smem + L.red);
    int* co = reinterpret_cast<int*>(smem + L.co);
    const T* As = reinterpret_cast<const T*>(smem + L.A);
    const uint16_t* Ls = reinterpret_cast<const uint16_t*>(smem + L.L);
    int32_t* Gs = reinterpret_cast<int32_t*>(smem + L.G);
    T* xs = reinterpret_cast<T*>(smem + L.xs);
    T* bs = reinterpret_cast<T*>(smem + L.bs);
    T* acc = reinterpret_cast<T*>(smem + L.acc);
    const uint32_t bar = smem_addr(smem + L.bar);

    pdl_trigger();
    const int p = blockIdx.x;
    const PatchMeta m = pd.meta[p];
    const int tid = threadIdx.x;
    const int64_t ns = pd.n_slots;
    const int64_t slot0 = int64_t(p) * kPatch;

    // The element matrices, connectivity and partition are constant while a
    // solver iterates, so their copies start before waiting for the previous
    // kernel of the stream (programmatic dependent launch); x, b and the stop
    // flag are read after the wait.
    if (tid == 0) {
        mbar_init(bar, 1);
        const uint64_t pol = policy_evict_first();
        mbar_expect_tx(bar, uint32_t(sym_count(NB) * kPatch * sizeof(T)) + uint32_t(NB * kPatch * 2));
#pragma unroll
        for (int t = 0; t < sym_count(NB); ++t)
            bulk_load(smem_addr(As + t * kPatch), A + t * ns + slot0, uint32_t(kPatch * sizeof(T)), bar, pol);
#pragma unroll
        for (int i = 0; i < NB; ++i)
            bulk_load(smem_addr(Ls + i * kPatch), pd.lconn + i * ns + slot0, uint32_t(kPatch * 2), bar, pol);
    }
    for (int c = tid; c <= m.n_col; c += NT) co[c] = __ldg(pd.col_ptr + m.col_off + c);
    pdl_wait();
    if (stop != nullptr && *stop) {                // uniform: the solver has stopped
        if (tid == 0) mbar_wait_bounded(bar, 0, nullptr);   // let the copies land before the CTA exits
        return;
    }
    // restriction x_e = R_e x, shared by the patch: node table, x (and b)
    const int32_t* pn = pd.pnode + m.node_off;
    for (int l0 = 0; l0 < m.n_nodes; l0 += 2 * NT) {
        int32_t gr[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int l = l0 + u * NT + tid;
            gr[u] = l < m.n_nodes ? __ldg(pn + l) : 0;
        }
        T xv[2], bv[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int l = l0 + u * NT + tid;
            const int g = gr[u] & kNodeMask;
            xv[u] = l < m.n_nodes ? __ldg(x + g) : T(0);
            bv[u] = (kRes && l < m.n_owned) ? __ldg(b + g) : T(0);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int l = l0 + u * NT + tid;
            if (l < m.n_nodes) {
                Gs[l] = gr[u];
                xs[l] = xv[u];
                if (!WARPS) acc[l] = T(0);
                if (kRes) bs[l] = bv[u];
            }
        }
    }
    // one thread waits (bounded) for the bulk copies and shares the outcome
    if (tid == 0) *flag = mbar_wait_bounded(bar, 0, pd.err) ? 1 : 0;
    __syncthreads();
    if (*flag == 0) {                             // error flag set: give the copies a last
        if (tid == 0) mbar_wait_bounded(bar, 0, nullptr);   // bounded chance to land, then leave
        return;
    }
    while (!mbar_try_wait(bar, 0)) {
    }                                             // completed already: acquire for this thread

    patch_sums<T, NB, WARPS>(m, pd.max_nodes, As, Ls, xs, acc, co, tid);

    // owned nodes: final value; shared nodes: halo partial
    DotAcc<T> dot;
    for (int l = tid; l < m.n_nodes; l += NT) {
        const int32_t graw = Gs[l];
        const int g = graw & kNodeMask;
        const bool dir = graw < 0;
        const T v = acc[l];
        if (l < m.n_owned) {
            T o;
            if (kRes) o = dir ? T(0) : T(bs[l] - v);
            else o = dir ? T(0) : v;
            out[g] = o;
            if (MODE == kResidualNorm) dot.add(o, o);
            if (MODE == kApplyDot) dot.add(xs[l], o);
        } else {
            halo[m.halo_off + (l - m.n_owned)] = v;
        }
    }
    if (MODE == kResidualNorm || MODE == kApplyDot) {
        const double dsum = block_total<NT>(dot, red);
        if (tid == 0) part[p] = dsum;
    }
}

constexpr int kFixThreads = 256;

// Shared nodes: add the halo partials in patch order, then finish like the
// owned nodes.  With a norm/dot mode the last CTA to finish adds all partial
// sums (patch passes first, then fix-up CTAs) in index order.
template <typename T, int MODE, int ROWS>
__global__ void __launch_bounds__(kFixThreads)
k_fixup(const PlanDev pd, const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ out,
        const T* __restrict__ halo, double* __restrict__ part, const int32_t* __restrict__ stop,
        Scalars* __restrict__ sc) {
    __shared__ double red[32];
    __shared__ bool last;
    pdl_trigger();
    pdl_wait();
    if (stop != nullptr && *stop) return;
    DotAcc<T> dot;
    // ROWS shared rows per thread at a time, their index and halo loads
    // interleaved; each row's partials are added in patch order
    const int st = int(gridDim.x) * kFixThreads;
    for (int k = blockIdx.x * kFixThreads + threadIdx.x; k < pd.n_shared; k += ROWS * st) {
        int32_t graw[ROWS];
        int s0[ROWS], cnt[ROWS];
        int nmax = 0;
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const int kk = k + u * st;
            const bool ok = kk < pd.n_shared;
            graw[u] = ok ? __ldg(pd.sh_node + kk) : 0;
            s0[u] = ok ? __ldg(pd.sh_ptr + kk) : 0;
            cnt[u] = ok ? __ldg(pd.sh_ptr + kk + 1) - s0[u] : 0;
            nmax = cnt[u] > nmax ? cnt[u] : nmax;
        }
        T v[ROWS];
#pragma unroll
        for (int u = 0; u < ROWS; ++u) v[u] = T(0);
        for (int t = 0; t < nmax; ++t)
#pragma unroll
            for (int u = 0; u < ROWS; ++u)
                if (t < cnt[u]) v[u] += halo[__ldg(pd.sh_slot + s0[u] + t)];
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            if (k + u * st >= pd.n_shared) break;
            const int g = graw[u] & kNodeMask;
            const bool dir = graw[u] < 0;
            T o;
            if (MODE == kResidual || MODE == kResidualNorm) o = dir ? T(0) : T(__ldg(b + g) - v[u]);
            else o = dir ? T(0) : v[u];
            out[g] = o;
            if (MODE == kResidualNorm) dot.add(o, o);
            if (MODE == kApplyDot) dot.add(__ldg(x + g), o);
        }
    }
    if (MODE == kResidualNorm || MODE == kApplyDot) {
        // this block also adds a contiguous chunk of the patch partials (one per
        // patch, written by the patch pass), so the last block has few to add
        const int np = pd.n_patches;
        const int chunk = (np + int(gridDim.x) - 1) / int(gridDim.x);
        const int p1 = min(np, (int(blockIdx.x) + 1) * chunk);
        double dsum = block_total<kFixThreads>(dot, red);
        if (threadIdx.x == 0)
            for (int i = int(blockIdx.x) * chunk; i < p1; ++i) dsum += part[i];
        if (threadIdx.x == 0) {
            part[np + blockIdx.x] = dsum;
            __threadfence();
            last = atomicAdd(&sc->ctr_fix, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (last) {
            __threadfence();
            double s = 0.0;
            for (int i = threadIdx.x; i < int(gridDim.x); i += kFixThreads) s += __ldcg(part + np + i);
            s = block_sum<kFixThreads>(s, red);
            if (threadIdx.x == 0) {
                sc->ctr_fix = 0;
                if (MODE == kResidualNorm) {
                    sc->rrt = s;
                } else {
                    sc->pq = s;
                    if (!(s > 0.0) || !isfinite(s)) { sc->done = 1; sc->reason = kBreakdown; }
                    else sc->alpha = sc->rho / s;
                }
            }
        }
    }
}

// FP64 variant: each thread reads the element matrices of its slots straight
// from global memory (coalesced slot-major runs) and forms their products
// A_e x_e; the colour rounds then add them into the node sums.  GB300 runs
// FP64 at 1/64 of the FP32 rate, so this pass is bound by FP64 issue rather
// than by bytes; without a matrix tile in shared memory four CTAs (three for
// tetrahedra) share an SM and hide the latency of the FMA chains.
struct Patch64Smem {
    uint32_t red, co, G, xs, bs, acc, total;
};
__host__ __device__ constexpr Patch64Smem patch64_layout(int max_nodes) {
    Patch64Smem s{};
    const uint32_t gcap = uint32_t((max_nodes + 3) / 4 * 4);
    s.red = 0;
    s.co = 32 * 8;
    s.G = (s.co + (kMaxColours + 1) * 4 + 15) / 16 * 16;
    s.xs = (s.G + gcap * 4 + 15) / 16 * 16;
    s.bs = s.xs + gcap * 8;
    s.acc = s.bs + gcap * 8;
    s.total = (s.acc + gcap * 8 + 127) / 128 * 128;
    return s;
}

template <int NB, int MODE>
__global__ void __launch_bounds__(kPatchThreads, NB == 3 ? 4 : 3)
k_patch64d(const PlanDev pd, const double* __restrict__ A, const double* __restrict__ x, const double* __restrict__ b,
           double* __restrict__ out, double* __restrict__ halo, double* __restrict__ part,
           const int32_t* __restrict__ stop) {
    constexpr int NT = kPatchThreads;
    constexpr bool kRes = (MODE == kResidual || MODE == kResidualNorm);
    extern __shared__ __align__(128) unsigned char smem[];
    const Patch64Smem L = patch64_layout(pd.max_nodes);
    double* red = reinterpret_cast<double*>(smem + L.red);
    int* co = reinterpret_cast<int*>(smem + L.co);
    int32_t* Gs = reinterpret_cast<int32_t*>(smem + L.G);
    double* xs = reinterpret_cast<double*>(smem + L.xs);
    double* bs = reinterpret_cast<double*>(smem + L.bs);
    double* acc = reinterpret_cast<double*>(smem + L.acc);

    pdl_trigger();
    const int p = blockIdx.x;
    const PatchMeta m = pd.meta[p];
    const int tid = threadIdx.x;
    const int64_t ns = pd.n_slots;
    const int64_t slot0 = int64_t(p) * kPatch;
    for (int c = tid; c <= m.n_col; c += NT) co[c] = __ldg(pd.col_ptr + m.col_off + c);
    // this thread's slots: local node ids (constant data, before the wait)
    int ln[kEPT][NB];
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
        const int s = tid + k * NT;
        const bool ok = s < m.n_el;
#pragma unroll
        for (int i = 0; i < NB; ++i) ln[k][i] = ok ? int(__ldg(pd.lconn + i * ns + slot0 + s)) : 0;
    }
    pdl_wait();
    if (stop != nullptr && *stop) return;
    const int32_t* pn = pd.pnode + m.node_off;
    for (int l0 = 0; l0 < m.n_nodes; l0 += 2 * NT) {
        const int la = l0 + tid, lb = l0 + NT + tid;
        const int32_t ga = la < m.n_nodes ? __ldg(pn + la) : 0, gb = lb < m.n_nodes ? __ldg(pn + lb) : 0;
        const double xa = la < m.n_nodes ? __ldg(x + (ga & kNodeMask)) : 0.0;
        const double xb = lb < m.n_nodes ? __ldg(x + (gb & kNodeMask)) : 0.0;
        const double ba = (kRes && la < m.n_owned) ? __ldg(b + (ga & kNodeMask)) : 0.0;
        const double bb = (kRes && lb < m.n_owned) ? __ldg(b + (gb & kNodeMask)) : 0.0;
        if (la < m.n_nodes) { Gs[la] = ga; xs[la] = xa; acc[la] = 0.0; if (kRes) bs[la] = ba; }
        if (lb < m.n_nodes) { Gs[lb] = gb; xs[lb] = xb; acc[lb] = 0.0; if (kRes) bs[lb] = bb; }
    }
    __syncthreads();
    // products of all slots first, while every thread is busy (a colour round
    // keeps about one thread in eight at work); the rounds only add them
    double y[kEPT][NB];
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
        const int s = tid + k * NT;
        const bool ok = s < m.n_el;
        double a[sym_count(NB)];
#pragma unroll
        for (int t = 0; t < sym_count(NB); ++t) a[t] = ok ? __ldg(A + t * ns + slot0 + s) : 0.0;
        double xe[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) xe[j] = xs[ln[k][j]];
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            double v = a[sym_index(NB, r, 0)] * xe[0];
#pragma unroll
            for (int j = 1; j < NB; ++j) v = fmadd(a[sym_index(NB, r, j)], xe[j], v);
            y[k][r] = v;
        }
    }
    for (int c = 0; c < m.n_col; ++c) {
        const int lo = co[c], hi = co[c + 1];
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            const int s = tid + k * NT;
            if (s >= lo && s < hi) {
#pragma unroll
                for (int r = 0; r < NB; ++r) acc[ln[k][r]] += y[k][r];
            }
        }
        __syncthreads();
    }
    DotAcc<double> dot;
    for (int l = tid; l < m.n_nodes; l += NT) {
        const int32_t graw = Gs[l];
        const int g = graw & kNodeMask;
        const bool dir = graw < 0;
        const double v = acc[l];
        if (l < m.n_owned) {
            const double o = kRes ? (dir ? 0.0 : bs[l] - v) : (dir ? 0.0 : v);
            out[g] = o;
            if (MODE == kResidualNorm) dot.add(o, o);
            if (MODE == kApplyDot) dot.add(xs[l], o);
        } else {
            halo[m.halo_off + (l - m.n_owned)] = v;
        }
    }
    if (MODE == kResidualNorm || MODE == kApplyDot) {
        const double dsum = block_sum<NT>(dot.value(), red);
        if (tid == 0) part[p] = dsum;
    }
}

// ---------------------------------------------------------------- double-word FP64 residual
// The FP64 residual with its arithmetic on the FP32 pipe: every stored FP64
// entry a of A_e is kept as the pair a = hi + lo of FP32 values (the same 8
// bytes), x is split into such a pair per patch node on the integer pipe, and
// the element products and node sums run in double-word arithmetic (exact
// FP32 products by FMA, TwoSum additions; about 48 significant bits, Dekker
// 1971).  Only r = b - (s + c) and the conversions at the end are FP64, two
// operations per node instead of n_b^2 + n_b per element.  The pair
// representation of A_e and x is exact to 2^-48 relative, so r differs from
// the FP64 residual by about 2^-48 |A| |x| per node.
// Two forms, by element type (dw_pairs), each measured best for its type.
// Triangles (8 colours a patch) keep hi and lo in separate runs and x and the
// node sums in separate FP32 arrays, and form each slot's products in its
// colour's round, from matrix runs the L2 prefetch below has made resident:
// no product array, the slots' local ids in shared memory, 40 registers and
// six CTAs per SM.  Tetrahedra (about 30 colours) form all four slots'
// products first, every pair (matrix entry, x, node sum) side by side as one
// 8-byte access, and the products wait for their round in shared memory (y:
// NB runs of kPatch float2).
struct PatchDwSmem {
    uint32_t red, co, G, xh, xl, bs, as, ac, y, total;
};
// xh, xl (and as, ac) are adjacent runs of gcap floats: the paired form uses
// the span from xh (as) as gcap float2.
template <int NB>
__host__ __device__ constexpr PatchDwSmem patch_dw_layout(int max_nodes) {
    PatchDwSmem s{};
    const uint32_t gcap = uint32_t((max_nodes + 3) / 4 * 4);
    s.red = 0;
    s.co = 32 * 8;
    s.G = (s.co + (kMaxColours + 1) * 4 + 15) / 16 * 16;
    s.xh = s.G + gcap * 4;
    s.xl = s.xh + gcap * 4;
    s.bs = (s.xl + gcap * 4 + 15) / 16 * 16;
    s.as = s.bs + gcap * 8;
    s.ac = s.as + gcap * 4;
    s.y = (s.ac + gcap * 4 + 15) / 16 * 16;   // products (paired form) or local ids (separate form)
    s.total = (s.y + (dw_pairs(NB) ? uint32_t(NB * kPatch * 8) : uint32_t(NB * kPatch * 2)) + 127) / 128 * 128;
    return s;
}

template <int NB, int MODE>
__global__ void __launch_bounds__(kPatchThreads, NB == 3 ? 6 : 4)
k_patch_dw(const PlanDev pd, const float* __restrict__ Adw, const float* __restrict__ Alo, const double* __restrict__ x,
           const double* __restrict__ b, double* __restrict__ out, float2* __restrict__ halo, double* __restrict__ part,
           const int32_t* __restrict__ stop) {
    constexpr int NT = kPatchThreads;
    constexpr bool kRes = (MODE == kResidual || MODE == kResidualNorm);
    constexpr bool kPairs = dw_pairs(NB);
    extern __shared__ __align__(128) unsigned char smem[];
    const PatchDwSmem L = patch_dw_layout<NB>(pd.max_nodes);
    double* red = reinterpret_cast<double*>(smem + L.red);
    float2* ysm = reinterpret_cast<float2*>(smem + L.y);
    int* co = reinterpret_cast<int*>(smem + L.co);
    int32_t* Gs = reinterpret_cast<int32_t*>(smem + L.G);
    float* xh = reinterpret_cast<float*>(smem + L.xh);    // separate form
    float* xl = reinterpret_cast<float*>(smem + L.xl);
    float2* xp = reinterpret_cast<float2*>(smem + L.xh);  // paired form
    double* bs = reinterpret_cast<double*>(smem + L.bs);
    float* as = reinterpret_cast<float*>(smem + L.as);
    float* ac = reinterpret_cast<float*>(smem + L.ac);
    float2* ap = reinterpret_cast<float2*>(smem + L.as);

    pdl_trigger();
    const int p = blockIdx.x;
    const PatchMeta m = pd.meta[p];
    const int tid = threadIdx.x;
    const int64_t ns = pd.n_slots;
    const int64_t slot0 = int64_t(p) * kPatch;
    // the patch's element matrices start moving into L2 now, so their DRAM
    // reads overlap the node gather below (they are constant: before the wait)
    if (m.n_el > 0) {
        if (kPairs) {
            if (tid < sym_count(NB))
                bulk_prefetch_l2(Adw + 2 * (tid * ns + slot0), uint32_t((m.n_el + 1) / 2 * 16));
        } else if (tid < 2 * sym_count(NB)) {
            bulk_prefetch_l2((tid & 1 ? Alo : Adw) + (tid >> 1) * ns + slot0, uint32_t((m.n_el + 3) / 4 * 16));
        }
    }
    for (int c = tid; c <= m.n_col; c += NT) co[c] = __ldg(pd.col_ptr + m.col_off + c);
    // the slots' 16-bit local ids, two to a register
    constexpr int NP = (NB + 1) / 2;
    uint32_t lp[kEPT][NP];
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
        const int s = tid + k * NT;
        const bool ok = s < m.n_el;
#pragma unroll
        for (int w = 0; w < NP; ++w) {
            const uint32_t lo = ok ? uint32_t(__ldg(pd.lconn + (2 * w) * ns + slot0 + s)) : 0u;
            const uint32_t hi = (ok && 2 * w + 1 < NB) ? uint32_t(__ldg(pd.lconn + (2 * w + 1) * ns + slot0 + s)) : 0u;
            lp[k][w] = lo | (hi << 16);
        }
    }
    auto ln = [&](int k, int i) { return int((lp[k][i >> 1] >> (16 * (i & 1))) & 0xffffu); };
    pdl_wait();
    if (stop != nullptr && *stop) return;
    const int32_t* pn = pd.pnode + m.node_off;
    for (int l = tid; l < m.n_nodes; l += NT) {
        const int32_t g = __ldg(pn + l);
        const double xv = __ldg(x + (g & kNodeMask));
        const double bv = (kRes && l < m.n_owned) ? __ldg(b + (g & kNodeMask)) : 0.0;
        float h, lo;
        split_dw(xv, h, lo);
        Gs[l] = g;
        if (kPairs) {
            xp[l] = make_float2(h, lo);
            ap[l] = make_float2(0.0f, 0.0f);
        } else {
            xh[l] = h;
            xl[l] = lo;
            as[l] = 0.0f;
            ac[l] = 0.0f;
        }
        if (kRes) bs[l] = bv;
    }
    __syncthreads();
    if constexpr (kPairs) {
        // products of all slots first (every thread busy), then colour rounds
        // add them; a thread reads back only its own slots' products
        const float2* A2 = reinterpret_cast<const float2*>(Adw) + slot0 + tid;
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            const int s = tid + k * NT;
            const bool ok = s < m.n_el;
            float2 a[sym_count(NB)];
#pragma unroll
            for (int t = 0; t < sym_count(NB); ++t) a[t] = ok ? __ldg(A2 + t * ns + k * NT) : make_float2(0.0f, 0.0f);
            float2 e[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) e[j] = xp[ln(k, j)];
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                float sv, cv;
                const float2 a0 = a[sym_index(NB, r, 0)];
                dw_mul(a0.x, a0.y, e[0].x, e[0].y, sv, cv);
#pragma unroll
                for (int j = 1; j < NB; ++j) {
                    const float2 aj = a[sym_index(NB, r, j)];
                    dw_fma(aj.x, aj.y, e[j].x, e[j].y, sv, cv);
                }
                ysm[r * kPatch + s] = make_float2(sv, cv);
            }
        }
        for (int c = 0; c < m.n_col; ++c) {
            const int lo = co[c], hi = co[c + 1];
#pragma unroll
            for (int k = 0; k < kEPT; ++k) {
                const int s = tid + k * NT;
                if (s >= lo && s < hi) {
#pragma unroll
                    for (int r = 0; r < NB; ++r) {
                        const int n = ln(k, r);
                        const float2 y = ysm[r * kPatch + s];
                        float2 t = ap[n];
                        dw_add(t.x, t.y, y.x, y.y);
                        ap[n] = t;
                    }
                }
            }
            __syncthreads();
        }
    } else {
        // each slot's products in its colour's round; the local ids move to
        // shared memory (this thread reads back only its own slots')
        uint16_t* Ls = reinterpret_cast<uint16_t*>(smem + L.y);
#pragma unroll
        for (int k = 0; k < kEPT; ++k)
#pragma unroll
            for (int i = 0; i < NB; ++i) Ls[i * kPatch + tid + k * NT] = uint16_t(ln(k, i));
        for (int c = 0; c < m.n_col; ++c) {
            const int lo = co[c], hi = co[c + 1];
#pragma unroll
            for (int k = 0; k < kEPT; ++k) {
                const int s = tid + k * NT;
                if (s >= lo && s < hi) {
                    float ah[sym_count(NB)], al[sym_count(NB)];
#pragma unroll
                    for (int t = 0; t < sym_count(NB); ++t) {
                        ah[t] = __ldg(Adw + t * ns + slot0 + s);
                        al[t] = __ldg(Alo + t * ns + slot0 + s);
                    }
                    int nn[NB];
                    float eh[NB], el[NB];
#pragma unroll
                    for (int j = 0; j < NB; ++j) {
                        nn[j] = Ls[j * kPatch + s];
                        eh[j] = xh[nn[j]];
                        el[j] = xl[nn[j]];
                    }
#pragma unroll
                    for (int r = 0; r < NB; ++r) {
                        float sv, cv;
                        dw_mul(ah[sym_index(NB, r, 0)], al[sym_index(NB, r, 0)], eh[0], el[0], sv, cv);
#pragma unroll
                        for (int j = 1; j < NB; ++j)
                            dw_fma(ah[sym_index(NB, r, j)], al[sym_index(NB, r, j)], eh[j], el[j], sv, cv);
                        float s2 = as[nn[r]], c2 = ac[nn[r]];
                        dw_add(s2, c2, sv, cv);
                        as[nn[r]] = s2;
                        ac[nn[r]] = c2;
                    }
                }
            }
            __syncthreads();
        }
    }
    DotAcc<float> dot;
    for (int l = tid; l < m.n_nodes; l += NT) {
        const int32_t graw = Gs[l];
        const int g = graw & kNodeMask;
        const bool dir = graw < 0;
        const float2 t = kPairs ? ap[l] : make_float2(as[l], ac[l]);
        if (l < m.n_owned) {
            const double v = f2d(t.x) + f2d(t.y);
            const double o = dir ? 0.0 : (kRes ? bs[l] - v : v);
            out[g] = o;
            if (MODE == kResidualNorm) {
                const float of = d2f(o);
                dot.add(of, of);
            }
        } else {
            halo[m.halo_off + (l - m.n_owned)] = t;
        }
    }
    if (MODE == kResidualNorm) {
        const double dsum = block_total<NT>(dot, red);
        if (tid == 0) part[p] = dsum;
    }
}

// Shared nodes of the double-word residual: the halo pairs added in patch
// order (double-word), then r = b - (s + c) in FP64; with the norm mode the
// last block adds all partial sums in index order.
template <int MODE, int ROWS>
__global__ void __launch_bounds__(kFixThreads)
k_fixup_dw(const PlanDev pd, const double* __restrict__ b, double* __restrict__ out, const float2* __restrict__ halo,
           double* __restrict__ part, const int32_t* __restrict__ stop, Scalars* __restrict__ sc) {
    __shared__ double red[32];
    __shared__ bool last;
    pdl_trigger();
    pdl_wait();
    if (stop != nullptr && *stop) return;
    DotAcc<float> dot;
    // ROWS shared rows per thread at a time, their loads interleaved; each
    // row's partials added in patch order
    const int st = int(gridDim.x) * kFixThreads;
    for (int k = blockIdx.x * kFixThreads + threadIdx.x; k < pd.n_shared; k += ROWS * st) {
        int32_t graw[ROWS];
        int s0[ROWS], cnt[ROWS];
        int nmax = 0;
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const int kk = k + u * st;
            const bool ok = kk < pd.n_shared;
            graw[u] = ok ? __ldg(pd.sh_node + kk) : 0;
            s0[u] = ok ? __ldg(pd.sh_ptr + kk) : 0;
            cnt[u] = ok ? __ldg(pd.sh_ptr + kk + 1) - s0[u] : 0;
            nmax = cnt[u] > nmax ? cnt[u] : nmax;
        }
        float sv[ROWS], cv[ROWS];
#pragma unroll
        for (int u = 0; u < ROWS; ++u) { sv[u] = 0.0f; cv[u] = 0.0f; }
        for (int t = 0; t < nmax; ++t)
#pragma unroll
            for (int u = 0; u < ROWS; ++u)
                if (t < cnt[u]) {
                    const float2 h = halo[__ldg(pd.sh_slot + s0[u] + t)];
                    dw_add(sv[u], cv[u], h.x, h.y);
                }
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            if (k + u * st >= pd.n_shared) break;
            const int g = graw[u] & kNodeMask;
            const double v = f2d(sv[u]) + f2d(cv[u]);
            const double o = graw[u] < 0 ? 0.0 : ((MODE == kResidual || MODE == kResidualNorm) ? __ldg(b + g) - v : v);
            out[g] = o;
            if (MODE == kResidualNorm) {
                const float of = d2f(o);
                dot.add(of, of);
            }
        }
    }
    if (MODE == kResidualNorm) {
        const int np = pd.n_patches;
        const int chunk = (np + int(gridDim.x) - 1) / int(gridDim.x);
        const int p1 = min(np, (int(blockIdx.x) + 1) * chunk);
        double dsum = block_total<kFixThreads>(dot, red);
        if (threadIdx.x == 0) {
            for (int i = int(blockIdx.x) * chunk; i < p1; ++i) dsum += part[i];
            part[np + blockIdx.x] = dsum;
            __threadfence();
            last = atomicAdd(&sc->ctr_fix, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (last) {
            __threadfence();
            double s = 0.0;
            for (int i = threadIdx.x; i < int(gridDim.x); i += kFixThreads) s += __ldcg(part + np + i);
            s = block_sum<kFixThreads>(s, red);
            if (threadIdx.x == 0) {
                sc->ctr_fix = 0;
                sc->rrt = s;
            }
        }
    }
}

template <int NB, int MODE>
cudaError_t run_patch_dw(const PlanDev& pd, const float* Adw, const double* x, const double* b,
                         double* out, float2* halo, double* part, const int32_t* stop, Scalars* sc, cudaStream_t st,
                         int* launches, cudaEvent_t* ev) {
    const size_t sm = patch_dw_layout<NB>(pd.max_nodes).total;
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    auto kern = k_patch_dw<NB, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[0], st);
    // the separate form's lo runs follow all hi runs
    const float* Alo = dw_pairs(NB) ? nullptr : Adw + int64_t(sym_count(NB)) * pd.n_slots;
    kern<<<pd.n_patches, kPatchThreads, sm, st>>>(pd, Adw, Alo, x, b, out, halo, part, stop);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    if (fix_rows(pd) == 2)
        k_fixup_dw<MODE, 2><<<fix_grid(pd.n_shared, 2), kFixThreads, 0, st>>>(pd, b, out, halo, part, stop, sc);
    else
        k_fixup_dw<MODE, 1><<<fix_grid(pd.n_shared, 1), kFixThreads, 0, st>>>(pd, b, out, halo, part, stop, sc);
    if (ev) cudaEventRecord(ev[2], st);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_split_dw(int64_t n, const double* __restrict__ a, float* __restrict__ out,
                                                  int pairs) {
    for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < n; i += int64_t(gridDim.x) * 256) {
        float h, l;
        split_dw(a[i], h, l);
        if (pairs) {
            reinterpret_cast<float2*>(out)[i] = make_float2(h, l);
        } else {
            out[i] = h;
            out[n + i] = l;
        }
    }
}

template <int NB, int MODE>
cudaError_t run_patch64(const PlanDev& pd, const double* A, const double* x, const double* b, double* out, double* halo,
                        double* part, const int32_t* stop, Scalars* sc, cudaStream_t st, int* launches, cudaEvent_t* ev,
                        bool pdl) {
    const size_t sm = patch64_layout(pd.max_nodes).total;
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    auto kern = k_patch64d<NB, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[0], st);
    if (pdl) {
        e = launch_pdl(kern, dim3(pd.n_patches), dim3(kPatchThreads), sm, st, pd, A, x, b, out, halo, part, stop);
        if (e != cudaSuccess) return e;
    } else {
        kern<<<pd.n_patches, kPatchThreads, sm, st>>>(pd, A, x, b, out, halo, part, stop);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    if (fix_rows(pd) == 2)
        k_fixup<double, MODE, 2><<<fix_grid(pd.n_shared, 2), kFixThreads, 0, st>>>(pd, x, b, out, halo, part, stop, sc);
    else
        k_fixup<double, MODE, 1><<<fix_grid(pd.n_shared, 1), kFixThreads, 0, st>>>(pd, x, b, out, halo, part, stop, sc);
    if (ev) cudaEventRecord(ev[2], st);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

template <typename T, int NB, int MODE, bool WARPS>
cudaError_t run_patch_as(const PlanDev& pd, const T* A, const T* x, const T* b, T* out, T* halo, double* part,
                         const int32_t* stop, Scalars* sc, cudaStream_t st, int* launches, cudaEvent_t* ev,
                         bool pdl) {
    const size_t sm = patch_layout<T, NB, WARPS>(pd.max_nodes).total;
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;   // a patch does not fit in shared memory
    auto kern = k_patch<T, NB, MODE, WARPS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[0], st);
    if (pdl) {
        e = launch_pdl(kern, dim3(pd.n_patches), dim3(kPatchThreads), sm, st, pd, A, x, b, out, halo, part, stop);
        if (e != cudaSuccess) return e;
    } else {
        kern<<<pd.n_patches, kPatchThreads, sm, st>>>(pd, A, x, b, out, halo, part, stop);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    if (fix_rows(pd) == 2)
        k_fixup<T, MODE, 2><<<fix_grid(pd.n_shared, 2), kFixThreads, 0, st>>>(pd, x, b, out, halo, part, stop, sc);
    else
        k_fixup<T, MODE, 1><<<fix_grid(pd.n_shared, 1), kFixThreads, 0, st>>>(pd, x, b, out, halo, part, stop, sc);
    if (ev) cudaEventRecord(ev[2], st);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

// Colour rounds for meshes with few colours per patch (triangles: 8; measured
// 66.5 against 75.5 us per 2049^2 application), per-warp node-sum copies for
// many (Kuhn tetrahedra: about 30; 142 against 205 us per 129^3 application).
template <typename T, int NB, int MODE>
cudaError_t run_patch(const PlanDev& pd, const T* A, const T* x, const T* b, T* out, T* halo, double* part,
                      const int32_t* stop, Scalars* sc, cudaStream_t st, int* launches, cudaEvent_t* ev, bool pdl) {
    if (pd.max_col > kWarpSchemeColours)
        return run_patch_as<T, NB, MODE, true>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
    return run_patch_as<T, NB, MODE, false>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
}

template <typename T, int NB>
cudaError_t run_patch_mode(const PlanDev& pd, int mode, const T* A, const T* x, const T* b, T* out, T* halo,
                           double* part, const int32_t* stop, Scalars* sc, cudaStream_t st, int* launches,
                           cudaEvent_t* ev, bool pdl) {
    if constexpr (sizeof(T) == 8) {
        switch (mode) {
            case kResidual: return run_patch64<NB, kResidual>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
            case kResidualNorm:
                return run_patch64<NB, kResidualNorm>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
            case kApply: return run_patch64<NB, kApply>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
            case kApplyDot: return run_patch64<NB, kApplyDot>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (mode) {
            case kResidual: return run_patch<T, NB, kResidual>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
            case kResidualNorm:
                return run_patch<T, NB, kResidualNorm>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
            case kApply: return run_patch<T, NB, kApply>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
            case kApplyDot: return run_patch<T, NB, kApplyDot>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
            default: return cudaErrorInvalidValue;
        }
    }
}


// ---------------------------------------------------------------- single-sync CG pass
// One Jacobi-PCG iteration in two launches (see launch_cg_pass): the node
// work of the textbook update and direction steps is done where the operator
// pass gathers its operand, and the next step's r.z comes from the expansion
// r'.(dinv r') = r.z - 2 alpha q.z + alpha^2 q.(dinv q) of the sums the pass
// forms anyway, so one grid-wide reduction per iteration remains.  Vectors are
// in the solver numbering: a patch's owned nodes are one contiguous run
// (coalesced loads and stores, no node-table reads), shared nodes are read
// through the node table and updated by the fix-up, which owns them.

constexpr int kCgSums = 5;   // r.z, r.r, p.q, q.z, q.(dinv q)

struct CgSmem {
    uint32_t bar, flag, red, co, A, L, xs, acc, total;
};
template <int NB, bool WARPS>
__host__ __device__ constexpr CgSmem cg_layout(int max_nodes) {
    CgSmem s{};
    const uint32_t gcap = uint32_t((max_nodes + 3) / 4 * 4);
    s.bar = 0;                                          // u64 mbarrier
    s.flag = 8;                                         // int
    s.red = 16;                                         // kCgSums x 8 doubles
    s.co = s.red + kCgSums * 8 * 8;                     // kMaxColours + 1 ints
    s.A = (s.co + (kMaxColours + 1) * 4 + 127) / 128 * 128;
    s.L = s.A + (WARPS ? uint32_t(sym_count(NB) * kPatch * 4) : 0u);   // matrices in shared memory: per-warp form only
    s.xs = s.L + uint32_t(NB * kPatch * 2);             // p_new at the patch nodes
    s.acc = s.xs + gcap * 4;
    s.total = (s.acc + (WARPS ? kWarpCopies : 1) * gcap * 4 + 127) / 128 * 128;
    return s;
}

// kCgSums block sums in a fixed order (warp butterflies, then warp 0 over the
// per-warp sums); valid in thread 0.  red: kCgSums x 8 doubles.
__device__ __forceinline__ void block_sums5(double (&v)[kCgSums], double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < kCgSums; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < kCgSums; ++k) red[k * 8 + w] = v[k];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < kCgSums; ++k) v[k] = lane < int(blockDim.x >> 5) ? red[k * 8 + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < kCgSums; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
}

// The node step of one iteration at one node, as the textbook update and
// direction kernels compute it: r' = r - alpha q (FP32), z = dinv r',
// p' = z + beta p (FP32), x' = x + alpha p (FP64, p widened exactly).
struct CgNode {
    float rn, z, pn;
};
__device__ __forceinline__ CgNode cg_node(float r, float q, float p, float d, float alf, float bef) {
    CgNode o;
    o.rn = __fmaf_rn(-alf, q, r);
    o.z = d * o.rn;
    o.pn = __fmaf_rn(bef, p, o.z);
    return o;
}

template <int NB, bool WARPS>
__global__ void __launch_bounds__(kPatchThreads, NB == 3 ? 6 : 3)
k_cg_patch(const PlanDev pd, const float* __restrict__ A, float* __restrict__ r, float* __restrict__ q,
           const float* __restrict__ p_old, float* __restrict__ p_new, const float* __restrict__ dinv,
           double* __restrict__ x, float* __restrict__ halo, double* __restrict__ part, const Scalars* __restrict__ sc) {
    constexpr int NT = kPatchThreads;
    extern __shared__ __align__(128) unsigned char smem[];
    const CgSmem L = cg_layout<NB, WARPS>(pd.max_nodes);
    volatile int* flag = reinterpret_cast<volatile int*>(smem + L.flag);
    double* red = reinterpret_cast<double*>(smem + L.red);
    int* co = reinterpret_cast<int*>(smem + L.co);
    const float* As = reinterpret_cast<const float*>(smem + L.A);
    const uint16_t* Ls = reinterpret_cast<const uint16_t*>(smem + L.L);
    float* xs = reinterpret_cast<float*>(smem + L.xs);
    float* acc = reinterpret_cast<float*>(smem + L.acc);
    const uint32_t bar = smem_addr(smem + L.bar);

    pdl_trigger();
    const int p = blockIdx.x;
    const PatchMeta m = pd.meta[p];
    const int tid = threadIdx.x;
    const int64_t ns = pd.n_slots;
    const int64_t slot0 = int64_t(p) * kPatch;
    // element matrices and connectivity are constant: copy before the wait
    if (tid == 0) {
        mbar_init(bar, 1);
        const uint64_t pol = policy_evict_first();
        mbar_expect_tx(bar, (WARPS ? uint32_t(sym_count(NB) * kPatch * 4) : 0u) + uint32_t(NB * kPatch * 2));
        if (WARPS) {
#pragma unroll
            for (int t = 0; t < sym_count(NB); ++t)
                bulk_load(smem_addr(As + t * kPatch), A + t * ns + slot0, uint32_t(kPatch * 4), bar, pol);
        } else if (m.n_el > 0) {
            // the colour rounds read each slot's entries from L2
#pragma unroll
            for (int t = 0; t < sym_count(NB); ++t) bulk_prefetch_l2(A + t * ns + slot0, uint32_t((m.n_el + 3) / 4 * 16));
        }
#pragma unroll
        for (int i = 0; i < NB; ++i)
            bulk_load(smem_addr(Ls + i * kPatch), pd.lconn + i * ns + slot0, uint32_t(kPatch * 2), bar, pol);
    }
    for (int c = tid; c <= m.n_col; c += NT) co[c] = __ldg(pd.col_ptr + m.col_off + c);
    // Node step at every patch node.  Owned nodes come in groups of four
    // consecutive solver numbers (a patch's run starts on a multiple of 4 and
    // is padded to one; padding entries are zero in every vector and stay
    // zero): 16-byte loads and stores, written back here.  Shared nodes come
    // one by one through the node table; the fix-up writes them.
    const int own0 = __ldg(pd.own_off + p);
    const int32_t* pn = pd.pnode + m.node_off;
    const int n_own4 = (m.n_owned + 3) >> 2;
    const int n_items = n_own4 + (m.n_nodes - m.n_owned);
    // The owned entries were written by the previous patch pass, which had
    // completed before the fix-up launched, so this thread's first item is
    // loaded before waiting for the fix-up (the node table is constant);
    // shared-node entries and the scalars only after the wait.
    float4 rv0, qv0, pv0, dv0;
    double2 xa0, xb0;
    int sid0 = -1, hpos0 = 0;
    if (tid < n_own4) {
        const int id0 = own0 + 4 * tid;
        rv0 = *reinterpret_cast<const float4*>(r + id0);
        qv0 = *reinterpret_cast<const float4*>(q + id0);
        pv0 = __ldg(reinterpret_cast<const float4*>(p_old + id0));
        dv0 = __ldg(reinterpret_cast<const float4*>(dinv + id0));
        xa0 = *reinterpret_cast<const double2*>(x + id0);
        xb0 = *reinterpret_cast<const double2*>(x + id0 + 2);
    } else if (tid < n_items) {
        sid0 = __ldg(pn + m.n_owned + (tid - n_own4)) & kNodeMask;
        hpos0 = __ldg(pd.halo_pos + m.halo_off + (tid - n_own4));   // where its halo partial goes
    }
    pdl_wait();
    if (sc->done) {                                  // uniform: the solver has stopped
        if (tid == 0) mbar_wait_bounded(bar, 0, nullptr);
        return;
    }
    const double al = sc->alpha;
    const float alf = d2f(al), bef = d2f(sc->beta);
    // the node sums zeroed per group of four (16-byte shared-memory stores)
    if (!WARPS)
        for (int g = tid; g < (m.n_nodes + 3) >> 2; g += NT) reinterpret_cast<float4*>(acc)[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    // per-thread sums of at most four terms in plain FP32: the warp butterflies
    // below add 32 of them in plain FP32 as well, so a compensated sum here
    // would not change the accuracy of the totals
    float srz = 0.0f, srr = 0.0f;
    auto owned_group = [&](int g, const float4& rv, const float4& qv, const float4& pv, const float4& dv,
                           const double2& xa, const double2& xb) {
        const int l0 = 4 * g, id0 = own0 + l0;
        const float rr4[4] = {rv.x, rv.y, rv.z, rv.w}, qq4[4] = {qv.x, qv.y, qv.z, qv.w};
        const float pp4[4] = {pv.x, pv.y, pv.z, pv.w}, dd4[4] = {dv.x, dv.y, dv.z, dv.w};
        const double xx4[4] = {xa.x, xa.y, xb.x, xb.y};
        float rn4[4], pn4[4];
        double xn4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const CgNode c = cg_node(rr4[u], qq4[u], pp4[u], dd4[u], alf, bef);
            rn4[u] = c.rn;
            pn4[u] = c.pn;
            xn4[u] = fmadd(al, f2d(pp4[u]), xx4[u]);
            if (l0 + u < m.n_owned) {
                srz = __fmaf_rn(c.rn, c.z, srz);
                srr = __fmaf_rn(c.rn, c.rn, srr);
            }
        }
        if (l0 + 4 <= m.n_owned) {
            reinterpret_cast<float4*>(xs)[g] = make_float4(pn4[0], pn4[1], pn4[2], pn4[3]);
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (l0 + u < m.n_owned) xs[l0 + u] = pn4[u];   // the entries after belong to shared nodes
        }
        *reinterpret_cast<float4*>(r + id0) = make_float4(rn4[0], rn4[1], rn4[2], rn4[3]);
        *reinterpret_cast<float4*>(p_new + id0) = make_float4(pn4[0], pn4[1], pn4[2], pn4[3]);
        *reinterpret_cast<double2*>(x + id0) = make_double2(xn4[0], xn4[1]);
        *reinterpret_cast<double2*>(x + id0 + 2) = make_double2(xn4[2], xn4[3]);
    };
    auto shared_node = [&](int g, int id) {
        const CgNode c = cg_node(r[id], q[id], __ldg(p_old + id), __ldg(dinv + id), alf, bef);
        xs[m.n_owned + (g - n_own4)] = c.pn;
    };
    if (tid < n_own4) owned_group(tid, rv0, qv0, pv0, dv0, xa0, xb0);
    else if (tid < n_items) shared_node(tid, sid0);
    for (int g = tid + NT; g < n_items; g += NT) {   // patches with more than NT items
        if (g < n_own4) {
            const int id0 = own0 + 4 * g;
            owned_group(g, *reinterpret_cast<const float4*>(r + id0), *reinterpret_cast<const float4*>(q + id0),
                        __ldg(reinterpret_cast<const float4*>(p_old + id0)),
                        __ldg(reinterpret_cast<const float4*>(dinv + id0)), *reinterpret_cast<const double2*>(x + id0),
                        *reinterpret_cast<const double2*>(x + id0 + 2));
        } else {
            shared_node(g, __ldg(pn + m.n_owned + (g - n_own4)) & kNodeMask);
        }
    }
    if (tid == 0) *flag = mbar_wait_bounded(bar, 0, pd.err) ? 1 : 0;
    __syncthreads();
    if (*flag == 0) {
        if (tid == 0) mbar_wait_bounded(bar, 0, nullptr);
        return;
    }
    while (!mbar_try_wait(bar, 0)) {
    }
    if (WARPS) {
        patch_sums<float, NB, WARPS>(m, pd.max_nodes, As, Ls, xs, acc, co, tid);
    } else {
        // each slot's products in its colour's round, its matrix entries read
        // from the L2-resident runs: no matrix tile in shared memory and no
        // product registers (2049^2: 96.0 against 101.0 us per pass with the
        // tile copied in and the products formed first); the same rows, added
        // in the same colour order
        for (int c = 0; c < m.n_col; ++c) {
            const int lo = co[c], hi = co[c + 1];
#pragma unroll
            for (int k = 0; k < kEPT; ++k) {
                const int s = tid + k * NT;
                if (s >= lo && s < hi) {
                    float a[sym_count(NB)];
#pragma unroll
                    for (int t = 0; t < sym_count(NB); ++t) a[t] = __ldg(A + t * ns + slot0 + s);
                    int nn[NB];
                    float xe[NB];
#pragma unroll
                    for (int i = 0; i < NB; ++i) {
                        nn[i] = Ls[i * kPatch + s];
                        xe[i] = xs[nn[i]];
                    }
#pragma unroll
                    for (int r = 0; r < NB; ++r) {
                        float v = a[sym_index(NB, r, r)] * xe[r];
#pragma unroll
                        for (int j = 0; j < NB; ++j)
                            if (j != r) v = fmadd(a[sym_index(NB, r, j)], xe[j] - xe[r], v);
                        acc[nn[r]] += v;
                    }
                }
            }
            __syncthreads();
        }
    }
    // q = mask(A p_new): owned nodes final (Dirichlet rows: dinv = 0), shared
    // nodes to their halo slots
    float spq = 0.0f, sqz = 0.0f, sqdq = 0.0f;
    for (int g = tid; g < n_items; g += NT) {
        if (g < n_own4) {
            const int l0 = 4 * g;
            // z = dinv r of the owned nodes again from the r this thread stored
            // in the node step (the same product; shared memory then fits six
            // CTAs per SM); 16-byte loads; entries past n_owned (shared nodes'
            // sums) are not used
            const float4 r4 = *reinterpret_cast<const float4*>(r + own0 + l0);
            const float4 d4 = __ldg(reinterpret_cast<const float4*>(dinv + own0 + l0));
            const float4 a4 = reinterpret_cast<const float4*>(acc)[g], x4 = reinterpret_cast<const float4*>(xs)[g];
            const float av[4] = {a4.x, a4.y, a4.z, a4.w}, xv[4] = {x4.x, x4.y, x4.z, x4.w};
            const float dv[4] = {d4.x, d4.y, d4.z, d4.w};
            const float zv[4] = {d4.x * r4.x, d4.y * r4.y, d4.z * r4.z, d4.w * r4.w};
            float qn4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                qn4[u] = 0.0f;                      // padding entries stay zero
                if (l0 + u < m.n_owned) {
                    const float qn = dv[u] == 0.0f ? 0.0f : av[u];
                    qn4[u] = qn;
                    spq = __fmaf_rn(xv[u], qn, spq);
                    sqz = __fmaf_rn(qn, zv[u], sqz);
                    sqdq = __fmaf_rn(qn, dv[u] * qn, sqdq);
                }
            }
            *reinterpret_cast<float4*>(q + own0 + l0) = make_float4(qn4[0], qn4[1], qn4[2], qn4[3]);
        } else {
            const int l = m.n_owned + (g - n_own4);
            const int hp = g == tid ? hpos0 : __ldg(pd.halo_pos + m.halo_off + (g - n_own4));
            halo[hp] = acc[l];   // CSR order
        }
    }
    // The sums stay compensated FP32 pairs up to the last fix-up block (every
    // FP64 instruction of a CTA costs 16 cycles of its SM's FP64 pipe): warp
    // butterflies, then warp 0 adds the 8 warp totals of sums 0-3 at once
    // (lane 8k + w holds warp w's total of sum k) and of sum 4.
    CompSum cs[kCgSums];
    {
        const float tv[kCgSums] = {srz, srr, spq, sqz, sqdq};
#pragma unroll
        for (int k = 0; k < kCgSums; ++k) cs[k].s = tv[k];
    }
#pragma unroll
    for (int k = 0; k < kCgSums; ++k) warp_sum_plain(cs[k]);
    float2* red2 = reinterpret_cast<float2*>(red);
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < kCgSums; ++k) red2[k * 8 + warp] = make_float2(cs[k].s, cs[k].c);
    __syncthreads();
    if (warp == 0) {
        float2* part2 = reinterpret_cast<float2*>(part);
        const int64_t stride = int64_t(pd.n_patches) + kFixGridMax;
        CompSum a = comp_of(red2[lane]);                         // sums 0-3
        group8_sum(a);
        if ((lane & 7) == 0) part2[(lane >> 3) * stride + p] = make_float2(a.s, a.c);
        CompSum b = lane < 8 ? comp_of(red2[32 + lane]) : CompSum{};   // sum 4
        group8_sum(b);
        if (lane == 0) part2[4 * stride + p] = make_float2(b.s, b.c);
    }
}

// Shared nodes of a single-sync pass: the node step (the fix-up owns them),
// q from the halo partials in patch order, the sums; the last block adds all
// partials in index order and takes the iteration's scalar decisions.
template <int ROWS>
__global__ void __launch_bounds__(kFixThreads, 6)
k_cg_fixup(const PlanDev pd, float* __restrict__ r, float* __restrict__ q, const float* __restrict__ p_old,
           float* __restrict__ p_new, const float* __restrict__ dinv, double* __restrict__ x,
           const float* __restrict__ halo, double* __restrict__ part, Scalars* __restrict__ sc) {
    __shared__ double red[kCgSums * 8];
    __shared__ bool last;
    pdl_trigger();
    pdl_wait();
    if (sc->done) return;
    const double al = sc->alpha;
    const float alf = d2f(al), bef = d2f(sc->beta);
    CompSum s5[kCgSums];
    const int st = int(gridDim.x) * kFixThreads;
    for (int k = blockIdx.x * kFixThreads + threadIdx.x; k < pd.n_shared; k += ROWS * st) {
        int s0[ROWS], cnt[ROWS];
        int nmax = 0;
        float rv[ROWS], qv[ROWS], pv[ROWS], dv[ROWS];
        double xv[ROWS];
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const int kk = k + u * st;
            const bool ok = kk < pd.n_shared;
            s0[u] = ok ? __ldg(pd.sh_ptr + kk) : 0;
            cnt[u] = ok ? __ldg(pd.sh_ptr + kk + 1) - s0[u] : 0;
            nmax = cnt[u] > nmax ? cnt[u] : nmax;
            const int id = pd.sh_base + kk;
            rv[u] = ok ? r[id] : 0.0f;
            qv[u] = ok ? q[id] : 0.0f;
            pv[u] = ok ? __ldg(p_old + id) : 0.0f;
            dv[u] = ok ? __ldg(dinv + id) : 0.0f;
            xv[u] = ok ? x[id] : 0.0;
        }
        float hv[ROWS];
#pragma unroll
        for (int u = 0; u < ROWS; ++u) hv[u] = 0.0f;
        // the patch pass wrote the row's partials contiguously (CSR order), in patch order
        for (int t = 0; t < nmax; ++t)
#pragma unroll
            for (int u = 0; u < ROWS; ++u)
                if (t < cnt[u]) hv[u] += halo[s0[u] + t];
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const int kk = k + u * st;
            if (kk >= pd.n_shared) break;
            const int id = pd.sh_base + kk;
            const CgNode c = cg_node(rv[u], qv[u], pv[u], dv[u], alf, bef);
            const float qn = dv[u] == 0.0f ? 0.0f : hv[u];
            x[id] = fmadd(al, f2d(pv[u]), xv[u]);
            r[id] = c.rn;
            p_new[id] = c.pn;
            q[id] = qn;
            s5[0].add(c.rn * c.z);
            s5[1].add(c.rn * c.rn);
            s5[2].add(c.pn * qn);
            s5[3].add(qn * c.z);
            s5[4].add(qn * (dv[u] * qn));
        }
    }
    // Compensated FP32 pairs (no FP64 work per block): warp butterflies over
    // the block's rows; then warp 0 adds, per sum, the 8 warp totals (lanes
    // 0-7) and a contiguous chunk of the per-patch partials (lane l takes
    // partials l, l + 32, ... of the chunk, after its warp total) with one more
    // butterfly: a fixed order, and short chains.
    float2* red2 = reinterpret_cast<float2*>(red);
    float2* part2 = reinterpret_cast<float2*>(part);
    const int np = pd.n_patches;
    const int64_t stride = int64_t(np) + kFixGridMax;
    const int chunk = (np + int(gridDim.x) - 1) / int(gridDim.x);
    const int p0 = min(np, int(blockIdx.x) * chunk), p1 = min(np, (int(blockIdx.x) + 1) * chunk);
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
        for (int j = 0; j < kCgSums; ++j) warp_sum_plain(s5[j]);
        if (lane == 0)
#pragma unroll
            for (int j = 0; j < kCgSums; ++j) red2[j * 8 + warp] = make_float2(s5[j].s, s5[j].c);
        __syncthreads();
        if (warp < kCgSums) {                       // warp j adds sum j
            const int j = warp;
            CompSum a = lane < kFixThreads / 32 ? comp_of(red2[j * 8 + lane]) : CompSum{};
            for (int i = p0 + lane; i < p1; i += 32) merge(a, comp_of(part2[j * stride + i]));
            warp_sum(a);
            if (lane == 0) part2[j * stride + np + blockIdx.x] = make_float2(a.s, a.c);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            last = atomicAdd(&sc->ctr_fix, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last block: every block's pair, added in compensated FP32 in a fixed
    // order; only the five totals are formed in FP64
    // (warp j merges the block pairs of sum j, lane by lane, then across the warp)
    __shared__ double tot[kCgSums];
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (warp < kCgSums) {
            CompSum a;
            for (int i = lane; i < int(gridDim.x); i += 32) merge(a, comp_of(__ldcg(part2 + warp * stride + np + i)));
            warp_sum(a);
            if (lane == 0) tot[warp] = a.value();
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double v[kCgSums];
#pragma unroll
    for (int j = 0; j < kCgSums; ++j) v[j] = tot[j];
    sc->ctr_fix = 0;
    const double rho = v[0], rr = v[1], pq = v[2], qz = v[3], qdq = v[4];
    const bool fresh = sc->fresh != 0;
    sc->fresh = 0;
    sc->passes += 1;
    if (!fresh) sc->iter += 1;
    sc->rz = rho;
    sc->rr = rr;
    sc->pq = pq;
    sc->qz = qz;
    sc->qdq = qdq;
    if (!isfinite(rho) || !isfinite(rr) || !isfinite(pq) || !isfinite(qz) || !isfinite(qdq) || rho < 0.0) {
        sc->done = 1;
        sc->reason = kBreakdown;
    } else if (!fresh && rr <= sc->thr2) {
        sc->done = 1;            // rho keeps the previous direction's r.z for the replacement
        sc->reason = kTrigger;
    } else if (!fresh && sc->iter >= sc->maxit) {
        sc->done = 1;
        sc->reason = kMaxit;
    } else if (!(pq > 0.0)) {
        sc->done = 1;
        sc->reason = kBreakdown;
    } else {
        const double a = rho / pq;
        const double rho_next = fmadd(a * a, qdq, fmadd(-2.0 * a, qz, rho));
        sc->alpha = a;
        sc->beta = rho_next > 0.0 ? rho_next / rho : 0.0;   // < 0 only through cancellation: restart the direction
        sc->rho = rho;
    }
}

template <int NB, bool WARPS>
cudaError_t run_cg_pass(const PlanDev& pd, const float* A, float* r, float* q, const float* p_old, float* p_new,
                        const float* dinv, double* x, float* halo, double* part, Scalars* sc, cudaStream_t st,
                        int* launches, bool pdl, cudaEvent_t* ev) {
    const size_t sm = cg_layout<NB, WARPS>(pd.max_nodes).total;
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    auto kern = k_cg_patch<NB, WARPS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[0], st);
    if (pdl) {
        e = launch_pdl(kern, dim3(pd.n_patches), dim3(kPatchThreads), sm, st, pd, A, r, q, p_old, p_new, dinv, x, halo,
                       part, sc);
        if (e != cudaSuccess) return e;
    } else {
        kern<<<pd.n_patches, kPatchThreads, sm, st>>>(pd, A, r, q, p_old, p_new, dinv, x, halo, part, sc);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    // one row per thread at a time (each row has five vector loads in flight
    // already), one wave of six 256-thread blocks per SM
    const int fg = std::min(fix_grid(pd.n_shared, 1), 6 * std::max(pd.num_sms, 1));
    k_cg_fixup<1><<<fg, kFixThreads, 0, st>>>(pd, r, q, p_old, p_new, dinv, x, halo, part, sc);
    if (ev) cudaEventRecord(ev[2], st);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

__global__ void k_cg_arm(Scalars* sc) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        sc->alpha = 0.0;
        sc->fresh = 1;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_permute(int64_t n, const int32_t* __restrict__ map, const T* __restrict__ src,
                                                 T* __restrict__ dst, int to_solver) {
    for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < n; i += int64_t(gridDim.x) * 256) {
        if (to_solver) dst[map[i]] = src[i];
        else dst[i] = src[map[i]];
    }
}

__global__ void __launch_bounds__(256) k_copy_dirichlet_bit(int32_t* __restrict__ dst, const int32_t* __restrict__ src,
                                                            int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < n; i += int64_t(gridDim.x) * 256)
        dst[i] = int32_t((uint32_t(dst[i]) & uint32_t(kNodeMask)) | (uint32_t(src[i]) & kDirichletBit));
}
}  // namespace

int fix_grid(int n_shared, int rows) {
    int g = (n_shared + rows * kFixThreads - 1) / (rows * kFixThreads);
    return g < 1 ? 1 : (g > kFixGridMax ? kFixGridMax : g);
}

int fix_rows(const PlanDev& pd) {
    // 2049^2 triangles: 2.04 slots per shared node, 10.5 -> 9.0 us per fix-up with
    // two rows; 129^3 tetrahedra (more slots per node): 16.0 -> 18.5 us, one row
    return 2 * pd.n_halo <= 5 * int64_t(pd.n_shared) ? 2 : 1;
}

cudaError_t launch_patch_pass_dw(const PlanDev& pd, int mode, const float* Adw, const double* x,
                                 const double* b, double* out, double* halo, double* part, const int32_t* stop,
                                 Scalars* sc, cudaStream_t st, int* launches, cudaEvent_t* ev) {
    float2* h = reinterpret_cast<float2*>(halo);
    if (pd.nb == 3) {
        switch (mode) {
            case kResidual: return run_patch_dw<3, kResidual>(pd, Adw, x, b, out, h, part, stop, sc, st, launches, ev);
            case kResidualNorm:
                return run_patch_dw<3, kResidualNorm>(pd, Adw, x, b, out, h, part, stop, sc, st, launches, ev);
            case kApply: return run_patch_dw<3, kApply>(pd, Adw, x, b, out, h, part, stop, sc, st, launches, ev);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (mode) {
        case kResidual: return run_patch_dw<4, kResidual>(pd, Adw, x, b, out, h, part, stop, sc, st, launches, ev);
        case kResidualNorm:
            return run_patch_dw<4, kResidualNorm>(pd, Adw, x, b, out, h, part, stop, sc, st, launches, ev);
        case kApply: return run_patch_dw<4, kApply>(pd, Adw, x, b, out, h, part, stop, sc, st, launches, ev);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_split_dw(int64_t n, const double* a, float* out, int nb, cudaStream_t st, int* launches) {
    if (n <= 0) return cudaSuccess;
    k_split_dw<<<int(std::min<int64_t>((n + 255) / 256, 8192)), 256, 0, st>>>(n, a, out, dw_pairs(nb) ? 1 : 0);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_cg_pass(const PlanDev& pd, const float* A, float* r, float* q, const float* p_old, float* p_new,
                           const float* dinv, double* x, float* halo, double* part, Scalars* sc, cudaStream_t st,
                           int* launches, bool pdl, cudaEvent_t* ev) {
    if (pd.own_off == nullptr) return cudaErrorInvalidValue;
    const bool warps = pd.max_col > kWarpSchemeColours;
    if (pd.nb == 3)
        return warps ? run_cg_pass<3, true>(pd, A, r, q, p_old, p_new, dinv, x, halo, part, sc, st, launches, pdl, ev)
                     : run_cg_pass<3, false>(pd, A, r, q, p_old, p_new, dinv, x, halo, part, sc, st, launches, pdl, ev);
    return warps ? run_cg_pass<4, true>(pd, A, r, q, p_old, p_new, dinv, x, halo, part, sc, st, launches, pdl, ev)
                 : run_cg_pass<4, false>(pd, A, r, q, p_old, p_new, dinv, x, halo, part, sc, st, launches, pdl, ev);
}

cudaError_t launch_cg_arm(Scalars* sc, cudaStream_t st, int* launches) {
    k_cg_arm<<<1, 32, 0, st>>>(sc);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_permute(int dtype, int to_solver, int64_t n, const int32_t* map, const void* src, void* dst,
                           cudaStream_t st, int* launches) {
    if (n <= 0) return cudaSuccess;
    const int g = int(std::min<int64_t>((n + 255) / 256, 4096));
    if (dtype == 0)
        k_permute<double><<<g, 256, 0, st>>>(n, map, static_cast<const double*>(src), static_cast<double*>(dst), to_solver);
    else
        k_permute<float><<<g, 256, 0, st>>>(n, map, static_cast<const float*>(src), static_cast<float*>(dst), to_solver);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_copy_dirichlet_bit(int32_t* dst, const int32_t* src, int64_t n, cudaStream_t st, int* launches) {
    if (n <= 0) return cudaSuccess;
    const int g = int(std::min<int64_t>((n + 255) / 256, 4096));
    k_copy_dirichlet_bit<<<g, 256, 0, st>>>(dst, src, n);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_patch_pass(const PlanDev& pd, int dtype, int mode, const void* A, const void* x, const void* b,
                              void* out, void* halo, double* part, const int32_t* stop, Scalars* sc, cudaStream_t st,
                              int* launches, cudaEvent_t* ev, bool pdl) {
    if (dtype == 0) {
        auto a = static_cast<const double*>(A);
        auto xx = static_cast<const double*>(x);
        auto bb = static_cast<const double*>(b);
        auto o = static_cast<double*>(out);
        auto h = static_cast<double*>(halo);
        return pd.nb == 3 ? run_patch_mode<double, 3>(pd, mode, a, xx, bb, o, h, part, stop, sc, st, launches, ev, pdl)
                          : run_patch_mode<double, 4>(pd, mode, a, xx, bb, o, h, part, stop, sc, st, launches, ev, pdl);
    }
    auto a = static_cast<const float*>(A);
    auto xx = static_cast<const float*>(x);
    auto bb = static_cast<const float*>(b);
    auto o = static_cast<float*>(out);
    auto h = static_cast<float*>(halo);
    return pd.nb == 3 ? run_patch_mode<float, 3>(pd, mode, a, xx, bb, o, h, part, stop, sc, st, launches, ev, pdl)
                      : run_patch_mode<float, 4>(pd, mode, a, xx, bb, o, h, part, stop, sc, st, launches, ev, pdl);
}

}  // namespace ebe
