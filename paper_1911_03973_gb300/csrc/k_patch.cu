// Patch passes of the element-by-element operator (sm_103a).
//
// A patch is a run of kPatch elements (see plan.cpp); one CTA handles one
// patch and several CTAs share an SM, so that one CTA's copies overlap
// another's arithmetic:
//   * the TMA engine bulk-copies the patch's element matrices (structure of
//     arrays: entry t of the patch's 1024 slots is one contiguous run) and
//     16-bit local connectivity into shared memory, evict-first in L2; while
//     they are in flight the threads gather the patch's node table, x and b
//     at the patch nodes -- the restriction x_e = R_e x of Algorithm 1,
//     shared by neighbouring elements;
//   * the threads add A_e x_e into per-node shared-memory sums colour by
//     colour: within a colour no two elements share a node, so there are no
//     atomics and the order of the additions is fixed (bitwise reproducible).
//     The product is folded into the sum (sum = fma(a_ij, x_j, sum)), so the
//     FP64 pipe does exactly n_b^2 FMAs per element;
//   * they write the result of every owned node (all of its elements are in
//     this patch) and the partial sum of every shared node to its halo slot.
// The fix-up pass adds the halo partials of each shared node in patch order.
#include <cstdint>

#include "device_util.cuh"
#include "kernels.h"

namespace ebe {
namespace {

constexpr int kHead = 32 * 8 + ((kMaxColours + 1) * 4 + 15) / 16 * 16;  // reduction + colour offsets

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

// Sum over the block in a fixed order: warp butterflies, then warp 0 over the
// per-warp sums.  Every thread must call it; the result is valid in thread 0.
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

// ---------------------------------------------------------------- TMA / mbarrier helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
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
// L2 policy for data read exactly once per pass (element matrices, local
// connectivity): evict first, so that the node vectors stay in L2.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// 1D bulk copy global -> shared on the TMA engine, completing on an mbarrier.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(pol)
        : "memory");
}

// Bounded wait on an mbarrier phase: gives up after `limit` polls (each poll
// may suspend the thread for a hardware-chosen time) and reports it.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase, int32_t* err) {
    for (int it = 0; it < (1 << 24); ++it)
        if (mbar_try_wait(bar, phase)) return true;
    if (err != nullptr) atomicExch(err, 1);
    return false;
}

// Shared-memory layout of a patch pass.  One patch per CTA: its element
// matrices (n_b^2 runs of 1024 values) and local connectivity (n_b runs) come
// in by TMA bulk copies; the node table, x and b at the patch nodes by plain
// loads issued while the bulk copies are in flight.
struct PatchSmem {
    uint32_t bar, flag, red, co, A, L, G, xs, bs, acc, total;
};
template <typename T, int NB>
__host__ __device__ constexpr PatchSmem patch_layout(int max_nodes) {
    PatchSmem s{};
    const uint32_t gcap = uint32_t((max_nodes + 3) / 4 * 4);
    s.bar = 0;                                          // u64 mbarrier
    s.flag = 8;                                         // int
    s.red = 16;                                         // 32 doubles
    s.co = s.red + 32 * 8;                              // kMaxColours + 1 ints
    s.A = (s.co + (kMaxColours + 1) * 4 + 127) / 128 * 128;
    s.L = s.A + uint32_t(NB * NB * kPatch * sizeof(T));
    s.G = s.L + uint32_t(NB * kPatch * 2);
    s.xs = s.G + gcap * 4;
    s.bs = (s.xs + gcap * uint32_t(sizeof(T)) + 15) / 16 * 16;
    s.acc = (s.bs + gcap * uint32_t(sizeof(T)) + 15) / 16 * 16;
    s.total = (s.acc + gcap * uint32_t(sizeof(T)) + 127) / 128 * 128;
    return s;
}

constexpr int kPatchThreads = 256;
constexpr int kEPT = kPatch / kPatchThreads;     // elements owned by a thread

// One patch per CTA, several CTAs per SM so that one CTA's copies overlap
// another's arithmetic.  Thread 0 starts the bulk copies; meanwhile all
// threads gather the node table, x and b.  Each thread owns the slots
// tid + 256 k and keeps their local node ids and x values in registers, so a
// colour round only reads the element matrix entries from shared memory and
// updates the node sums.
template <typename T, int NB, int MODE>
__global__ void __launch_bounds__(kPatchThreads)
k_patch(const PlanDev pd, const T* __restrict__ A, const T* __restrict__ x, const T* __restrict__ b,
        T* __restrict__ out, T* __restrict__ halo, double* __restrict__ part, const int32_t* __restrict__ stop) {
    constexpr int NT = kPatchThreads;
    constexpr bool kRes = (MODE == kResidual || MODE == kResidualNorm);
    extern __shared__ __align__(128) unsigned char smem[];
    const PatchSmem L = patch_layout<T, NB>(pd.max_nodes);
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
        mbar_expect_tx(bar, uint32_t(NB * NB * kPatch * sizeof(T)) + uint32_t(NB * kPatch * 2));
#pragma unroll
        for (int t = 0; t < NB * NB; ++t)
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
                acc[l] = T(0);
                if (kRes) bs[l] = bv[u];
            }
        }
    }
    // one thread waits (bounded) for the bulk copies and shares the outcome
    if (tid == 0) *flag = mbar_wait_bounded(bar, 0, pd.err) ? 1 : 0;
    __syncthreads();
    if (*flag == 0) return;
    while (!mbar_try_wait(bar, 0)) {
    }                                             // completed already: acquire for this thread

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
    if constexpr (sizeof(T) == 8) {
        // FP64: the product is folded into the node sum inside the colour
        // rounds (acc = fma(a_rj, x_j, acc)), the minimum of n_b^2 FP64 FMAs
        // per element -- the FP64 pipe, not DRAM, bounds this pass
        for (int c = 0; c < m.n_col; ++c) {
            const int lo = co[c], hi = co[c + 1];
#pragma unroll
            for (int k = 0; k < kEPT; ++k) {
                const int s = tid + k * NT;
                if (s >= lo && s < hi) {
#pragma unroll
                    for (int r = 0; r < NB; ++r) {
                        T v = acc[ln[k][r]];
#pragma unroll
                        for (int j = 0; j < NB; ++j) v = fmadd(As[(r * NB + j) * kPatch + s], xe[k][j], v);
                        acc[ln[k][r]] = v;
                    }
                }
            }
            __syncthreads();
        }
    } else {
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
                T v = ok ? As[(r * NB + r) * kPatch + s] * xe[k][r] : T(0);
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    if (j != r) v = ok ? fmadd(As[(r * NB + j) * kPatch + s], xe[k][j] - xe[k][r], v) : v;
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
        const double dsum = block_sum<NT>(dot.value(), red);
        if (tid == 0) part[p] = dsum;
    }
}

constexpr int kFixThreads = 256;

// Shared nodes: add the halo partials in patch order, then finish like the
// owned nodes.  With a norm/dot mode the last CTA to finish adds all partial
// sums (patch passes first, then fix-up CTAs) in index order.
template <typename T, int MODE>
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
    for (int k = blockIdx.x * kFixThreads + threadIdx.x; k < pd.n_shared; k += gridDim.x * kFixThreads) {
        const int32_t graw = __ldg(pd.sh_node + k);
        const int g = graw & kNodeMask;
        const bool dir = graw < 0;
        T v = T(0);
        const int s1 = __ldg(pd.sh_ptr + k + 1);
        for (int s = __ldg(pd.sh_ptr + k); s < s1; ++s) v += halo[__ldg(pd.sh_slot + s)];
        T o;
        if (MODE == kResidual || MODE == kResidualNorm) o = dir ? T(0) : T(__ldg(b + g) - v);
        else o = dir ? T(0) : v;
        out[g] = o;
        if (MODE == kResidualNorm) dot.add(o, o);
        if (MODE == kApplyDot) dot.add(__ldg(x + g), o);
    }
    if (MODE == kResidualNorm || MODE == kApplyDot) {
        double dsum = dot.value();
        // this block also adds a contiguous chunk of the patch partials (one per
        // patch, written by the patch pass), so the last block has few to add
        const int np = pd.n_patches;
        const int chunk = (np + int(gridDim.x) - 1) / int(gridDim.x);
        const int p1 = min(np, (int(blockIdx.x) + 1) * chunk);
        for (int i = int(blockIdx.x) * chunk + threadIdx.x; i < p1; i += kFixThreads) dsum += part[i];
        dsum = block_sum<kFixThreads>(dsum, red);
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

// ---------------------------------------------------------------- P1 element matrices
// K_ij = int grad(l_i).grad(l_j) and M_ij = int l_i l_j on one simplex
// (Eq. matrices_K_M), closed form.  2D: with the edge vectors opposite each
// vertex e_0 = v2-v1, e_1 = v0-v2, e_2 = v1-v0 and D = (v1-v0) x (v2-v0),
// grad(l_i) = rot(e_i)/D, so K_ij = e_i.e_j / (2|D|), |T| = |D|/2.  3D: with
// d_k = v_k - v0 and J = [d1 d2 d3], grad(l_1..3) are the rows of inv(J):
// c_1 = d2 x d3, c_2 = d3 x d1, c_3 = d1 x d2 over det J, c_0 = -(c_1+c_2+c_3),
// so K_ij = c_i.c_j / (6|det J|), |T| = |det J|/6.  M_ij = |T|(1+delta_ij)/12
// (2D) or /20 (3D).  Returns |T| (0 for a degenerate simplex).
template <int NB>
__device__ __forceinline__ double p1_element(const double (&v)[NB][NB - 1], double (&K)[NB][NB], double& mdiag,
                                             double& moff) {
    if constexpr (NB == 3) {
        const double e[3][2] = {{v[2][0] - v[1][0], v[2][1] - v[1][1]},
                                {v[0][0] - v[2][0], v[0][1] - v[2][1]},
                                {v[1][0] - v[0][0], v[1][1] - v[0][1]}};
        const double D = e[2][0] * (v[2][1] - v[0][1]) - e[2][1] * (v[2][0] - v[0][0]);
        const double aD = fabs(D);
        const double w = aD > 0.0 ? 1.0 / (2.0 * aD) : 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) K[i][j] = w * (e[i][0] * e[j][0] + e[i][1] * e[j][1]);
        const double area = 0.5 * aD;
        moff = area / 12.0;
        mdiag = 2.0 * moff;
        return area;
    } else {
        double d[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) d[k][c] = v[k + 1][c] - v[0][c];
        double cr[4][3];
        auto cross = [](const double* u, const double* w, double* o) {
            o[0] = u[1] * w[2] - u[2] * w[1];
            o[1] = u[2] * w[0] - u[0] * w[2];
            o[2] = u[0] * w[1] - u[1] * w[0];
        };
        cross(d[1], d[2], cr[1]);
        cross(d[2], d[0], cr[2]);
        cross(d[0], d[1], cr[3]);
#pragma unroll
        for (int c = 0; c < 3; ++c) cr[0][c] = -(cr[1][c] + cr[2][c] + cr[3][c]);
        const double det = d[0][0] * cr[1][0] + d[0][1] * cr[1][1] + d[0][2] * cr[1][2];
        const double ad = fabs(det);
        const double w = ad > 0.0 ? 1.0 / (6.0 * ad) : 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                K[i][j] = w * (cr[i][0] * cr[j][0] + cr[i][1] * cr[j][1] + cr[i][2] * cr[j][2]);
        const double vol = ad / 6.0;
        moff = vol / 20.0;
        mdiag = 2.0 * moff;
        return vol;
    }
}

// Element matrices of every slot, A_e = K_e + nu M_e stored FP64 (and FP32),
// with the load vector b = sum_e C_e^T M_e f_e and d = sum_e C_e^T diag(A_e)
// accumulated per node like the residual (colour order, halo for shared).
template <int NB>
__global__ void __launch_bounds__(256, 2)
k_assemble(const PlanDev pd, const double* __restrict__ coords, const double* __restrict__ f, double nu,
           double* __restrict__ A64, float* __restrict__ A32, double* __restrict__ b, double* __restrict__ d,
           double* __restrict__ dinv, float* __restrict__ b32, float* __restrict__ dinv32,
           double* __restrict__ halo2, unsigned long long* __restrict__ bad) {
    constexpr int DIM = NB - 1, NT = 256, EPT = kPatch / NT;
    extern __shared__ __align__(128) unsigned char smem[];
    int* co = reinterpret_cast<int*>(smem + 32 * 8);
    double* cs = reinterpret_cast<double*>(smem + kHead);   // [max_nodes][DIM]
    double* fs = cs + pd.max_nodes * DIM;
    double* bacc = fs + pd.max_nodes;
    double* dacc = bacc + pd.max_nodes;

    const int p = blockIdx.x;
    const PatchMeta m = pd.meta[p];
    const int tid = threadIdx.x;
    const int64_t ns = pd.n_slots;
    const int64_t slot0 = int64_t(p) * kPatch;
    const int32_t* gid = pd.pnode + m.node_off;
    for (int l = tid; l < m.n_nodes; l += NT) {
        const int g = __ldg(gid + l) & kNodeMask;
#pragma unroll
        for (int c = 0; c < DIM; ++c) cs[l * DIM + c] = __ldg(coords + int64_t(g) * DIM + c);
        fs[l] = __ldg(f + g);
        bacc[l] = 0.0;
        dacc[l] = 0.0;
    }
    for (int c = tid; c <= m.n_col; c += NT) co[c] = __ldg(pd.col_ptr + m.col_off + c);
    __syncthreads();

    double be[EPT][NB], di[EPT][NB];
    int ln[EPT][NB];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const int s = tid + k * NT;
        const bool ok = s < m.n_el;
        double v[NB][DIM];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            ln[k][i] = ok ? int(pd.lconn[i * ns + slot0 + s]) : 0;
#pragma unroll
            for (int c = 0; c < DIM; ++c) v[i][c] = cs[ln[k][i] * DIM + c];
        }
        double K[NB][NB], md, mo;
        const double meas = p1_element<NB>(v, K, md, mo);
        double fsum = 0.0;
#pragma unroll
        for (int j = 0; j < NB; ++j) fsum += fs[ln[k][j]];
        // row sum of A_e: K_e rows sum to zero, M_e rows to |T|/3 (2D) or |T|/4 (3D)
        const double rowsum = nu * (md + (NB - 1) * mo);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                const double aij = K[i][j] + nu * (i == j ? md : mo);
                if (ok) {
                    A64[(i * NB + j) * ns + slot0 + s] = aij;
                    // FP32 copy in difference form: row sums on the diagonal slots
                    if (A32 != nullptr) A32[(i * NB + j) * ns + slot0 + s] = float(i == j ? rowsum : aij);
                }
                if (i == j) di[k][i] = aij;
            }
            // (M_e f_e)_i = m (f_i + sum_j f_j) with m = |T|/12 (2D) or |T|/20 (3D)
            be[k][i] = mo * (fs[ln[k][i]] + fsum);
        }
        if (ok && !(meas > 0.0)) atomicMin(bad, (unsigned long long)(unsigned)__ldg(pd.slot_elem + slot0 + s));
    }
    for (int c = 0; c < m.n_col; ++c) {
        const int lo = co[c], hi = co[c + 1];
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const int s = tid + k * NT;
            if (s >= lo && s < hi) {
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    bacc[ln[k][i]] += be[k][i];
                    dacc[ln[k][i]] += di[k][i];
                }
            }
        }
        __syncthreads();
    }
    for (int l = tid; l < m.n_nodes; l += NT) {
        const int32_t graw = __ldg(gid + l);
        const int g = graw & kNodeMask;
        const bool dir = graw < 0;
        if (l < m.n_owned) {
            b[g] = bacc[l];
            d[g] = dacc[l];
            const double iv = dir ? 0.0 : 1.0 / dacc[l];
            dinv[g] = iv;
            if (b32 != nullptr) { b32[g] = float(bacc[l]); dinv32[g] = float(iv); }
        } else {
            const int64_t h = m.halo_off + (l - m.n_owned);
            halo2[2 * h] = bacc[l];
            halo2[2 * h + 1] = dacc[l];
        }
    }
}

__global__ void __launch_bounds__(kFixThreads)
k_fixup_assemble(const PlanDev pd, const double* __restrict__ halo2, double* __restrict__ b, double* __restrict__ d,
                 double* __restrict__ dinv, float* __restrict__ b32, float* __restrict__ dinv32) {
    for (int k = blockIdx.x * kFixThreads + threadIdx.x; k < pd.n_shared; k += gridDim.x * kFixThreads) {
        const int32_t graw = pd.sh_node[k];
        const int g = graw & kNodeMask;
        double bv = 0.0, dv = 0.0;
        for (int s = pd.sh_ptr[k]; s < pd.sh_ptr[k + 1]; ++s) {
            const int64_t h = pd.sh_slot[s];
            bv += halo2[2 * h];
            dv += halo2[2 * h + 1];
        }
        b[g] = bv;
        d[g] = dv;
        const double iv = graw < 0 ? 0.0 : 1.0 / dv;
        dinv[g] = iv;
        if (b32 != nullptr) { b32[g] = float(bv); dinv32[g] = float(iv); }
    }
}

// K_e, M_e of every element in the paper's layout, caller's element order.
template <int NB>
__global__ void k_export_km(const PlanDev pd, const double* __restrict__ coords, double* __restrict__ Kout,
                            double* __restrict__ Mout) {
    constexpr int DIM = NB - 1;
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= pd.n_slots) return;
    const int32_t e = pd.slot_elem[s];
    if (e < 0) return;
    const PatchMeta m = pd.meta[s / kPatch];
    double v[NB][DIM];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int g = pd.pnode[m.node_off + pd.lconn[i * pd.n_slots + s]] & kNodeMask;
#pragma unroll
        for (int c = 0; c < DIM; ++c) v[i][c] = coords[int64_t(g) * DIM + c];
    }
    double K[NB][NB], md, mo;
    p1_element<NB>(v, K, md, mo);
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const int64_t o = int64_t(e) * NB * NB + j * NB + i;
            if (Kout) Kout[o] = K[i][j];
            if (Mout) Mout[o] = i == j ? md : mo;
        }
}

template <typename T>
__global__ void k_export_A(const PlanDev pd, const T* __restrict__ A, T* __restrict__ out) {
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= pd.n_slots) return;
    const int32_t e = pd.slot_elem[s];
    if (e < 0) return;
    const int nb = pd.nb;
    for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j) out[int64_t(e) * nb * nb + j * nb + i] = A[(i * nb + j) * pd.n_slots + s];
}

__global__ void k_mark(int32_t* __restrict__ ids, int64_t n, const uint8_t* __restrict__ mask) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int g = ids[k] & kNodeMask;
        ids[k] = mask[g] ? int32_t(uint32_t(g) | kDirichletBit) : g;
    }
}


template <typename T, int NB, int MODE>
cudaError_t run_patch(const PlanDev& pd, const T* A, const T* x, const T* b, T* out, T* halo, double* part,
                      const int32_t* stop, Scalars* sc, cudaStream_t st, int* launches, cudaEvent_t* ev, bool pdl) {
    const size_t sm = patch_layout<T, NB>(pd.max_nodes).total;
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;   // a patch does not fit in shared memory
    auto kern = k_patch<T, NB, MODE>;
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
    k_fixup<T, MODE><<<fix_grid(pd.n_shared), kFixThreads, 0, st>>>(pd, x, b, out, halo, part, stop, sc);
    if (ev) cudaEventRecord(ev[2], st);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

template <typename T, int NB>
cudaError_t run_patch_mode(const PlanDev& pd, int mode, const T* A, const T* x, const T* b, T* out, T* halo,
                           double* part, const int32_t* stop, Scalars* sc, cudaStream_t st, int* launches,
                           cudaEvent_t* ev, bool pdl) {
    switch (mode) {
        case kResidual: return run_patch<T, NB, kResidual>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
        case kResidualNorm:
            return run_patch<T, NB, kResidualNorm>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
        case kApply: return run_patch<T, NB, kApply>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
        case kApplyDot: return run_patch<T, NB, kApplyDot>(pd, A, x, b, out, halo, part, stop, sc, st, launches, ev, pdl);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int fix_grid(int n_shared) {
    int g = (n_shared + kFixThreads - 1) / kFixThreads;
    return g < 1 ? 1 : (g > 1216 ? 1216 : g);
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

cudaError_t launch_assemble(const PlanDev& pd, const double* coords, const double* f, double nu, double* A64,
                            float* A32, double* b, double* d, double* dinv, float* b32, float* dinv32,
                            double* halo2, unsigned long long* bad, cudaStream_t st, int* launches) {
    const size_t sm = kHead + size_t(pd.max_nodes) * sizeof(double) * (pd.dim + 3);
    cudaError_t e;
    if (pd.nb == 3) {
        if (sm > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k_assemble<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm))) != cudaSuccess)
            return e;
        k_assemble<3><<<pd.n_patches, 256, sm, st>>>(pd, coords, f, nu, A64, A32, b, d, dinv, b32, dinv32, halo2, bad);
    } else {
        if (sm > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k_assemble<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm))) != cudaSuccess)
            return e;
        k_assemble<4><<<pd.n_patches, 256, sm, st>>>(pd, coords, f, nu, A64, A32, b, d, dinv, b32, dinv32, halo2, bad);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_fixup_assemble<<<fix_grid(pd.n_shared), kFixThreads, 0, st>>>(pd, halo2, b, d, dinv, b32, dinv32);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_export_km(const PlanDev& pd, const double* coords, double* K, double* M, cudaStream_t st,
                             int* launches) {
    const int nt = 256;
    const int64_t g = (pd.n_slots + nt - 1) / nt;
    if (pd.nb == 3) k_export_km<3><<<unsigned(g), nt, 0, st>>>(pd, coords, K, M);
    else k_export_km<4><<<unsigned(g), nt, 0, st>>>(pd, coords, K, M);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_export_A(const PlanDev& pd, int dtype, const void* A, void* out, cudaStream_t st, int* launches) {
    const int nt = 256;
    const int64_t g = (pd.n_slots + nt - 1) / nt;
    if (dtype == 0) k_export_A<double><<<unsigned(g), nt, 0, st>>>(pd, static_cast<const double*>(A), static_cast<double*>(out));
    else k_export_A<float><<<unsigned(g), nt, 0, st>>>(pd, static_cast<const float*>(A), static_cast<float*>(out));
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_mark_dirichlet(const PlanDev& pd, int32_t* pnode, int64_t n_pnode, int32_t* sh_node,
                                  const uint8_t* mask, cudaStream_t st, int* launches) {
    k_mark<<<1216, 256, 0, st>>>(pnode, n_pnode, mask);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (pd.n_shared > 0) {
        k_mark<<<1216, 256, 0, st>>>(sh_node, pd.n_shared, mask);
        if (launches) *launches += 1;
    }
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace ebe
