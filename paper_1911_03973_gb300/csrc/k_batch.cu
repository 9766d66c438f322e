// Persistent Jacobi-PCG over a batch of independent problems (sm_103a).
//
// The batch is one partition of the disjoint union of the meshes in which no
// patch, fix-up item or node tile mixes two problems, so every dot product
// of Algorithm 2 (Jacobi-PCG) is a sum over the items of one problem.  One
// cooperative launch of a few CTAs per SM runs the whole solve; each loop
// iteration has four phases separated by grid barriers:
//   P  patch pass over the patches of live problems: q = A p (inner type)
//      for a problem in kBNormal, the FP64 true residual r = b - A x for a
//      problem in kBReplace (its first one gives |r0|); partial dots;
//   F  shared nodes: halo partials in patch order, finish q (or r); the last
//      fix-up item of a problem to finish sums the problem's partials in
//      index order: alpha = rho / p.Ap, or the true r.r;
//   U  node tiles: x += alpha p, r -= alpha q (or, after a replacement, only
//      the sums); the last tile of a problem sums r.z and r.r and takes the
//      problem's decisions (beta, replacement, convergence, breakdown, stall);
//   D  node tiles: p = z + beta p for the problems still iterating.
// (Forming p inside the next patch pass instead, which saves D's pass and a
// barrier, measured slower: the extra gathers of r and dinv lengthen the
// patch pass's latency-bound critical path by more than D costs.)
// Scheduling: every CTA keeps in shared memory the list of the problems still
// running with prefix sums of their patch, fix-up and tile counts, rebuilt
// (block-wide scan) whenever a problem finishes; item i of a phase belongs to
// CTA i mod gridDim, so the live work is spread evenly however many problems
// have finished.
// The per-problem decisions follow the single-problem solver: mixed
// precision keeps x in FP64 and the recurrence residual in FP32, and replaces
// it by the FP64 true residual whenever it has dropped by delta; a problem is done
// when its true relative residual reaches rtol.  Problems that are done cost
// nothing but a shared-memory lookup per item.  Every sum is taken in a fixed
// order, so a solve is bitwise reproducible (for any launch shape with the
// same tile size: the sums do not depend on which CTA runs an item).
#include <cstdint>

#include "device_util.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace ebe {
namespace {

constexpr int NT = 256;
constexpr int kEPT = kPatch / NT;

using tma::block_sum;
using tma::block_sum2;

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

// Block total, valid in thread 0: FP64 butterflies for FP64 data; for FP32
// data compensated FP32 butterflies and one FP64 conversion per warp (the FP64
// pipe runs at 1/64 of the FP32 rate on GB300).
__device__ __forceinline__ double block_total(const DotAcc<double>& d, double* red) {
    return block_sum<NT>(d.value(), red);
}
__device__ __forceinline__ double block_total(const DotAcc<float>& d, double* red) {
    CompSum v[1] = {d.c};
    double out[1];
    block_sums_comp<1, NT>(v, out, red);
    return out[0];
}

// Data written during the launch by other CTAs is read through L2 only.
template <typename V>
__device__ __forceinline__ V ld_l2(const V* p) { return __ldcg(p); }

// ---------------------------------------------------------------- shared memory
struct BatchSmem {
    uint32_t bar, flag, broken, live, last, nl, ver, timer, red, co, mode, list, pre;
    uint32_t A, L, G, xs, acc;        // inner-operator patch pass
    uint32_t G2, xs2, bs2, acc2;      // FP64 true-residual patch pass (same region)
    uint32_t total;
};
__host__ __device__ constexpr uint32_t up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

template <typename T, int NB>
__host__ __device__ constexpr BatchSmem batch_layout(int max_nodes, int n_prob) {
    BatchSmem s{};
    const uint32_t gcap = uint32_t((max_nodes + 3) / 4 * 4);
    s.bar = 0;
    s.flag = 8;
    s.broken = 12;
    s.live = 16;
    s.last = 20;
    s.nl = 24;
    s.ver = 28;
    s.timer = 32;                                    // 5 u64
    s.red = 80;                                      // 2 * NT / 32 doubles (also the scan's scratch)
    s.co = s.red + 2 * (NT / 32) * 8;
    s.mode = up(s.co + (kMaxColours + 1) * 4, 16);   // int8 per problem
    s.list = up(s.mode + uint32_t(n_prob), 16);      // live problems
    s.pre = s.list + uint32_t(n_prob) * 4;           // prefix sums: patches, fix-up items, tiles [3][n_prob + 1]
    s.A = up(s.pre + 3u * uint32_t(n_prob + 1) * 4, 128);
    s.L = s.A + uint32_t(sym_count(NB) * kPatch * sizeof(T));
    s.G = s.L + uint32_t(NB * kPatch * 2);
    s.xs = up(s.G + gcap * 4, 16);
    s.acc = up(s.xs + gcap * uint32_t(sizeof(T)), 16);
    const uint32_t end1 = s.acc + gcap * uint32_t(sizeof(T));
    s.G2 = s.A;
    s.xs2 = up(s.G2 + gcap * 4, 16);
    s.bs2 = s.xs2 + gcap * 8;
    s.acc2 = s.bs2 + gcap * 8;
    const uint32_t end2 = s.acc2 + gcap * 8;
    s.total = up(end1 > end2 ? end1 : end2, 128);
    return s;
}

// The shared-memory layout is recomputed where it is used (a few integer
// operations on kernel parameters) rather than carried in registers.
template <typename T, int NB>
__device__ __forceinline__ BatchSmem layout_of(const BatchDev& bd) {
    return batch_layout<T, NB>(bd.pd.max_nodes, bd.n_prob);
}

struct Ctx {
    const BatchDev* bd;
    unsigned char* smem;
    uint32_t mph;      // parity of the CTA's mbarrier phase
};

// ---------------------------------------------------------------- phase P
// Bulk copies of one patch's element matrices and local connectivity into
// the CTA's buffers (thread 0; completes on the CTA's mbarrier).
template <typename T, int NB>
__device__ __forceinline__ void issue_patch_copies(const BatchDev& bd, unsigned char* smem, int p) {
    const BatchSmem Lo = layout_of<T, NB>(bd);
    const T* A = static_cast<const T*>(bd.A);
    const int64_t ns = bd.pd.n_slots;
    const int64_t slot0 = int64_t(p) * kPatch;
    const uint32_t mbar = tma::smem_addr(smem + Lo.bar);
    const uint64_t pol = tma::policy_evict_first();
    tma::mbar_expect_tx(mbar, uint32_t(sym_count(NB) * kPatch * sizeof(T)) + uint32_t(NB * kPatch * 2));
#pragma unroll
    for (int t = 0; t < sym_count(NB); ++t)
        tma::bulk_load(tma::smem_addr(smem + Lo.A + t * kPatch * sizeof(T)), A + t * ns + slot0,
                       uint32_t(kPatch * sizeof(T)), mbar, pol);
#pragma unroll
    for (int i = 0; i < NB; ++i)
        tma::bulk_load(tma::smem_addr(smem + Lo.L + i * kPatch * 2), bd.pd.lconn + i * ns + slot0, uint32_t(kPatch * 2),
                       mbar, pol);
}

// q = A p on one patch (inner type T): the element matrices and local
// connectivity come in by TMA bulk copies while the threads gather the node
// table and p; products first, then colour rounds add them into the node
// sums (FP32: difference form, the diagonal slot holds the row sum).
// have: the copies of p were issued already (prefetch).  next_p >= 0: issue
// the copies of the CTA's next patch as soon as this patch's products are
// formed, so that they land during this patch's colour rounds and the next
// patch's gathers.  Returns false in every thread if the copies did not
// arrive in time (the device error flag is set; the CTA stops its patch work).
template <typename T, int NB>
__device__ __forceinline__ bool apply_patch(Ctx& c, int p, bool have, int next_p) {
    const BatchDev& bd = *c.bd;
    const PlanDev& pd = bd.pd;
    unsigned char* smem = c.smem;
    const BatchSmem Lo = layout_of<T, NB>(bd);
    volatile int* flag = reinterpret_cast<volatile int*>(smem + Lo.broken);
    double* red = reinterpret_cast<double*>(smem + Lo.red);
    int* co = reinterpret_cast<int*>(smem + Lo.co);
    const T* As = reinterpret_cast<const T*>(smem + Lo.A);
    const uint16_t* Ls = reinterpret_cast<const uint16_t*>(smem + Lo.L);
    int32_t* Gs = reinterpret_cast<int32_t*>(smem + Lo.G);
    T* xs = reinterpret_cast<T*>(smem + Lo.xs);
    T* acc = reinterpret_cast<T*>(smem + Lo.acc);
    const uint32_t mbar = tma::smem_addr(smem + Lo.bar);
    const T* pv = static_cast<const T*>(bd.p);
    T* q = static_cast<T*>(bd.q);
    T* halo = static_cast<T*>(bd.halo);
    const int tid = threadIdx.x;
    const PatchMeta m = pd.meta[p];

    // (the previous item's reads of these buffers ended before its block
    // reduction's barriers)
    if (!have && tid == 0) issue_patch_copies<T, NB>(bd, smem, p);
    for (int k = tid; k <= m.n_col; k += NT) co[k] = __ldg(pd.col_ptr + m.col_off + k);
    const int32_t* pn = pd.pnode + m.node_off;
    // two nodes per thread per round: both table loads, then both value loads, in flight
    for (int l0 = 0; l0 < m.n_nodes; l0 += 2 * NT) {
        const int la = l0 + tid, lb = l0 + NT + tid;
        const int32_t ga = la < m.n_nodes ? __ldg(pn + la) : 0, gb = lb < m.n_nodes ? __ldg(pn + lb) : 0;
        const T xa = la < m.n_nodes ? ld_l2(pv + (ga & kNodeMask)) : T(0);
        const T xb = lb < m.n_nodes ? ld_l2(pv + (gb & kNodeMask)) : T(0);
        if (la < m.n_nodes) { Gs[la] = ga; xs[la] = xa; acc[la] = T(0); }
        if (lb < m.n_nodes) { Gs[lb] = gb; xs[lb] = xb; acc[lb] = T(0); }
    }
    // *flag (the CTA's "broken" word) stays 1 from here on if the copies are lost:
    // this CTA does no more patch work and the next grid barrier ends the launch
    if (tid == 0 && !tma::mbar_wait_bounded(mbar, c.mph, pd.err)) *flag = 1;
    __syncthreads();
    const uint32_t ph = c.mph;
    c.mph ^= 1u;
    if (*flag != 0) return false;
    while (!tma::mbar_try_wait(mbar, ph)) {
    }

    int ln[kEPT][NB];
    T y[kEPT][NB];
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
        const int s = tid + k * NT;
        const bool ok = s < m.n_el;
        T xe[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            ln[k][i] = ok ? int(Ls[i * kPatch + s]) : 0;
            xe[i] = xs[ln[k][i]];
        }
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            T v;
            if constexpr (sizeof(T) == 4) {
                v = ok ? As[sym_index(NB, r, r) * kPatch + s] * xe[r] : T(0);
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    if (j != r) v = ok ? fmadd(As[sym_index(NB, r, j) * kPatch + s], xe[j] - xe[r], v) : v;
            } else {
                v = T(0);
#pragma unroll
                for (int j = 0; j < NB; ++j) v = ok ? fmadd(As[sym_index(NB, r, j) * kPatch + s], xe[j], v) : v;
            }
            y[k][r] = v;
        }
    }
    if (next_p >= 0) {
        __syncthreads();   // every thread is done with As, Ls
        if (tid == 0) issue_patch_copies<T, NB>(bd, smem, next_p);
    }
    for (int cc = 0; cc < m.n_col; ++cc) {
        const int lo = co[cc], hi = co[cc + 1];
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
    DotAcc<T> dot;
    for (int l = tid; l < m.n_nodes; l += NT) {
        const int32_t graw = Gs[l];
        const T v = acc[l];
        if (l < m.n_owned) {
            const T o = graw < 0 ? T(0) : v;
            q[graw & kNodeMask] = o;
            dot.add(xs[l], o);
        } else {
            halo[m.halo_off + (l - m.n_owned)] = v;
        }
    }
    const double dsum = block_total(dot, red);
    if (tid == 0) bd.part_p[p] = dsum;
    return true;
}

// The true residual r = mask(b - A x) on one patch, FP64 vectors.  A
// replacement happens a few times per problem and solve, so this pass
// favours few registers over speed: element matrices are read straight from
// global memory (coalesced slot-major runs) inside the colour rounds.  The
// FP64 solver forms it in FP64; the mixed solver in double-word FP32
// arithmetic (A_e and x as pairs of FP32, exact products and TwoSum
// additions: Dekker 1971), which keeps FP64's accuracy to about 2^-48 |A||x|
// and stays off the FP64 pipe.  The halo partials are then FP32 pairs.
template <int NB>
__device__ __forceinline__ void residual_patch_dw(Ctx& c, int p, const BatchSmem& Lo) {
    const BatchDev& bd = *c.bd;
    const PlanDev& pd = bd.pd;
    unsigned char* smem = c.smem;
    double* red = reinterpret_cast<double*>(smem + Lo.red);
    int* co = reinterpret_cast<int*>(smem + Lo.co);
    int32_t* Gs = reinterpret_cast<int32_t*>(smem + Lo.G2);
    float2* xw = reinterpret_cast<float2*>(smem + Lo.xs2);
    double* bs = reinterpret_cast<double*>(smem + Lo.bs2);
    float2* aw = reinterpret_cast<float2*>(smem + Lo.acc2);
    const int tid = threadIdx.x;
    const int64_t ns = pd.n_slots;
    const int64_t n_dw = int64_t(sym_count(NB)) * ns;   // the lo runs start here when the pairs are not side by side
    const int64_t slot0 = int64_t(p) * kPatch;
    const PatchMeta m = pd.meta[p];

    __syncthreads();
    for (int k = tid; k <= m.n_col; k += NT) co[k] = __ldg(pd.col_ptr + m.col_off + k);
    const int32_t* pn = pd.pnode + m.node_off;
    for (int l0 = 0; l0 < m.n_nodes; l0 += 2 * NT) {
        const int la = l0 + tid, lb = l0 + NT + tid;
        const int32_t ga = la < m.n_nodes ? __ldg(pn + la) : 0, gb = lb < m.n_nodes ? __ldg(pn + lb) : 0;
        const double xa = la < m.n_nodes ? ld_l2(bd.x + (ga & kNodeMask)) : 0.0;
        const double xb = lb < m.n_nodes ? ld_l2(bd.x + (gb & kNodeMask)) : 0.0;
        const double ba = la < m.n_owned ? __ldg(bd.b + (ga & kNodeMask)) : 0.0;
        const double bb = lb < m.n_owned ? __ldg(bd.b + (gb & kNodeMask)) : 0.0;
        float h, lo;
        if (la < m.n_nodes) { split_dw(xa, h, lo); Gs[la] = ga; xw[la] = make_float2(h, lo); bs[la] = ba; aw[la] = make_float2(0.f, 0.f); }
        if (lb < m.n_nodes) { split_dw(xb, h, lo); Gs[lb] = gb; xw[lb] = make_float2(h, lo); bs[lb] = bb; aw[lb] = make_float2(0.f, 0.f); }
    }
    __syncthreads();
    for (int cc = 0; cc < m.n_col; ++cc) {
        const int lo = co[cc], hi = co[cc + 1];
        for (int s = lo + tid; s < hi; s += NT) {
            int ln[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) ln[i] = int(__ldg(pd.lconn + i * ns + slot0 + s));
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                float sv = 0.0f, cv = 0.0f;
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    const int64_t e = sym_index(NB, r, j) * ns + slot0 + s;
                    const float2 xv = xw[ln[j]];
                    const float2 a = dw_pairs(NB) ? __ldg(reinterpret_cast<const float2*>(bd.Adw) + e)
                                                  : make_float2(__ldg(bd.Adw + e), __ldg(bd.Adw + n_dw + e));
                    if (j == 0) dw_mul(a.x, a.y, xv.x, xv.y, sv, cv);
                    else dw_fma(a.x, a.y, xv.x, xv.y, sv, cv);
                }
                float2 t = aw[ln[r]];
                dw_add(t.x, t.y, sv, cv);
                aw[ln[r]] = t;
            }
        }
        __syncthreads();
    }
    double dot = 0.0;
    float2* halo2 = reinterpret_cast<float2*>(bd.halo64);
    for (int l = tid; l < m.n_nodes; l += NT) {
        const int32_t graw = Gs[l];
        const float2 t = aw[l];
        if (l < m.n_owned) {
            const double o = graw < 0 ? 0.0 : bs[l] - (f2d(t.x) + f2d(t.y));
            bd.r[graw & kNodeMask] = o;
            dot = fmadd(o, o, dot);
        } else {
            halo2[m.halo_off + (l - m.n_owned)] = t;
        }
    }
    const double dsum = block_sum<NT>(dot, red);
    if (tid == 0) bd.part_p[p] = dsum;
}

template <typename T, int NB>
__device__ __forceinline__ void residual_patch(Ctx& c, int p, bool exact) {
    if constexpr (sizeof(T) == 4) {
        if (!exact) {
            residual_patch_dw<NB>(c, p, layout_of<T, NB>(*c.bd));
            return;
        }
    }
    const BatchDev& bd = *c.bd;
    const PlanDev& pd = bd.pd;
    unsigned char* smem = c.smem;
    const BatchSmem Lo = layout_of<T, NB>(bd);
    double* red = reinterpret_cast<double*>(smem + Lo.red);
    int* co = reinterpret_cast<int*>(smem + Lo.co);
    int32_t* Gs = reinterpret_cast<int32_t*>(smem + Lo.G2);
    double* xs = reinterpret_cast<double*>(smem + Lo.xs2);
    double* bs = reinterpret_cast<double*>(smem + Lo.bs2);
    double* acc = reinterpret_cast<double*>(smem + Lo.acc2);
    const int tid = threadIdx.x;
    const int64_t ns = pd.n_slots;
    const int64_t n_dw = int64_t(sym_count(NB)) * ns;   // the lo runs start here when the pairs are not side by side
    const int64_t slot0 = int64_t(p) * kPatch;
    const PatchMeta m = pd.meta[p];

    __syncthreads();
    for (int k = tid; k <= m.n_col; k += NT) co[k] = __ldg(pd.col_ptr + m.col_off + k);
    const int32_t* pn = pd.pnode + m.node_off;
    for (int l0 = 0; l0 < m.n_nodes; l0 += 2 * NT) {
        const int la = l0 + tid, lb = l0 + NT + tid;
        const int32_t ga = la < m.n_nodes ? __ldg(pn + la) : 0, gb = lb < m.n_nodes ? __ldg(pn + lb) : 0;
        const double xa = la < m.n_nodes ? ld_l2(bd.x + (ga & kNodeMask)) : 0.0;
        const double xb = lb < m.n_nodes ? ld_l2(bd.x + (gb & kNodeMask)) : 0.0;
        const double ba = la < m.n_owned ? __ldg(bd.b + (ga & kNodeMask)) : 0.0;
        const double bb = lb < m.n_owned ? __ldg(bd.b + (gb & kNodeMask)) : 0.0;
        if (la < m.n_nodes) { Gs[la] = ga; xs[la] = xa; bs[la] = ba; acc[la] = 0.0; }
        if (lb < m.n_nodes) { Gs[lb] = gb; xs[lb] = xb; bs[lb] = bb; acc[lb] = 0.0; }
    }
    __syncthreads();
    for (int cc = 0; cc < m.n_col; ++cc) {
        const int lo = co[cc], hi = co[cc + 1];
        for (int s = lo + tid; s < hi; s += NT) {
            int ln[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) ln[i] = int(__ldg(pd.lconn + i * ns + slot0 + s));
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                double v = acc[ln[r]];
#pragma unroll
                for (int j = 0; j < NB; ++j) v = fmadd(__ldg(bd.A64 + sym_index(NB, r, j) * ns + slot0 + s), xs[ln[j]], v);
                acc[ln[r]] = v;
            }
        }
        __syncthreads();
    }
    double dot = 0.0;
    for (int l = tid; l < m.n_nodes; l += NT) {
        const int32_t graw = Gs[l];
        if (l < m.n_owned) {
            const double o = graw < 0 ? 0.0 : bs[l] - acc[l];
            bd.r[graw & kNodeMask] = o;
            dot = fmadd(o, o, dot);
        } else {
            bd.halo64[m.halo_off + (l - m.n_owned)] = acc[l];
        }
    }
    const double dsum = block_sum<NT>(dot, red);
    if (tid == 0) bd.part_p[p] = dsum;
}

// ---------------------------------------------------------------- phase F
template <typename T, int NB>
__device__ __forceinline__ void fix_item(Ctx& c, int ci, int md) {
    const BatchDev& bd = *c.bd;
    const PlanDev& pd = bd.pd;
    unsigned char* smem = c.smem;
    const BatchSmem Lo = layout_of<T, NB>(bd);
    double* red = reinterpret_cast<double*>(smem + Lo.red);
    volatile int* last = reinterpret_cast<volatile int*>(smem + Lo.last);
    const int tid = threadIdx.x;
    const BatchItem it = bd.fix[ci];
    // two shared rows per thread, their index and halo loads interleaved
    double dsum;
    {
        const T* halo = static_cast<const T*>(bd.halo);
        const T* pv = static_cast<const T*>(bd.p);
        T* q = static_cast<T*>(bd.q);
        DotAcc<T> dot;
        double dot64 = 0.0;
        for (int r0 = it.lo + tid; r0 < it.hi; r0 += 2 * NT) {
            const int r1 = r0 + NT;
            const bool two = r1 < it.hi;
            const int32_t g0 = __ldg(pd.sh_node + r0), g1 = two ? __ldg(pd.sh_node + r1) : 0;
            const int a0 = __ldg(pd.sh_ptr + r0), a1 = __ldg(pd.sh_ptr + r0 + 1);
            const int b0 = two ? __ldg(pd.sh_ptr + r1) : 0, b1 = two ? __ldg(pd.sh_ptr + r1 + 1) : 0;
            const int na = a1 - a0, nb = b1 - b0, nmax = na > nb ? na : nb;
            if (md == kBNormal) {
                T v0 = T(0), v1 = T(0);
                for (int t = 0; t < nmax; ++t) {
                    if (t < na) v0 += ld_l2(halo + __ldg(pd.sh_slot + a0 + t));
                    if (t < nb) v1 += ld_l2(halo + __ldg(pd.sh_slot + b0 + t));
                }
                const int h0 = g0 & kNodeMask, h1 = g1 & kNodeMask;
                const T o0 = g0 < 0 ? T(0) : v0;
                q[h0] = o0;
                dot.add(ld_l2(pv + h0), o0);
                if (two) {
                    const T o1 = g1 < 0 ? T(0) : v1;
                    q[h1] = o1;
                    dot.add(ld_l2(pv + h1), o1);
                }
            } else {
                double v0 = 0.0, v1 = 0.0;
                if (sizeof(T) == 4 && ld_l2(&bd.prob[it.k].exact) == 0) {
                    // double-word halo partials (FP32 pairs) of the mixed solver
                    const float2* halo2 = reinterpret_cast<const float2*>(bd.halo64);
                    float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
                    for (int t = 0; t < nmax; ++t) {
                        if (t < na) { const float2 h = ld_l2(halo2 + __ldg(pd.sh_slot + a0 + t)); dw_add(s0, c0, h.x, h.y); }
                        if (t < nb) { const float2 h = ld_l2(halo2 + __ldg(pd.sh_slot + b0 + t)); dw_add(s1, c1, h.x, h.y); }
                    }
                    v0 = f2d(s0) + f2d(c0);
                    v1 = f2d(s1) + f2d(c1);
                } else {
                    for (int t = 0; t < nmax; ++t) {
                        if (t < na) v0 += ld_l2(bd.halo64 + __ldg(pd.sh_slot + a0 + t));
                        if (t < nb) v1 += ld_l2(bd.halo64 + __ldg(pd.sh_slot + b0 + t));
                    }
                }
                const double o0 = g0 < 0 ? 0.0 : __ldg(bd.b + (g0 & kNodeMask)) - v0;
                bd.r[g0 & kNodeMask] = o0;
                dot64 = fmadd(o0, o0, dot64);
                if (two) {
                    const double o1 = g1 < 0 ? 0.0 : __ldg(bd.b + (g1 & kNodeMask)) - v1;
                    bd.r[g1 & kNodeMask] = o1;
                    dot64 = fmadd(o1, o1, dot64);
                }
            }
        }
        dsum = md == kBNormal ? block_total(dot, red) : block_sum<NT>(dot64, red);
    }
    if (tid == 0)
        for (int i = it.plo; i < it.phi; ++i) dsum += ld_l2(bd.part_p + i);
    // last item of the problem to finish: the acquire-release arrival makes
    // every earlier item's partial visible to it
    if (tid == 0) {
        bd.part_f[ci] = dsum;
        *last = tma::atom_add_acq_rel(bd.ctr + it.k, 1u) == uint32_t(it.count - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!*last) return;
    double s = 0.0;
    for (int i = tid; i < it.count; i += NT) s += ld_l2(bd.part_f + it.first + i);
    s = block_sum<NT>(s, red);
    if (tid == 0) {
        bd.ctr[it.k] = 0u;
        volatile BatchProblem* P = bd.prob + it.k;
        if (md == kBNormal) {
            if (!(s > 0.0) || !isfinite(s)) P->bd = 1;
            else P->alpha = P->rho / s;
        } else {
            P->rrt = s;
        }
    }
}

// ---------------------------------------------------------------- decisions
// Thread 0 of the last node tile of problem k.
template <bool MIXED>
__device__ __forceinline__ void decide(const BatchDev& bd, int k, int md, double rz, double rr) {
    volatile BatchProblem* P = bd.prob + k;
    auto finish = [&](int status) {
        P->mode = kBDone;
        P->status = status;
        atomicSub(bd.live, 1);
    };
    if (md == kBNormal) {
        const int64_t it = P->iter + 1;
        P->iter = it;
        if (P->bd || !isfinite(rz) || !isfinite(rr) || rz < 0.0) {
            P->bd = 1;
            P->exact = 1;
            P->mode = kBReplace;                // a last true residual, then done
        } else if (rr <= P->thr2 || it >= bd.maxit) {
            // the replacement in double-word form while the threshold is large
            // against its error, else in FP64
            const double lim = kDwReplaceRel * P->r0;
            P->exact = (P->thr2 >= lim * lim && it < bd.maxit) ? 0 : 1;
            P->mode = kBReplace;                // rho stays: the replacement recomputes r.z
        } else {
            P->beta = rz / P->rho;
            P->rho = rz;
            P->dir_init = 0;
        }
        return;
    }
    // after a true residual (rrt from the fix-up phase)
    const double rrt = P->rrt;
    P->n_true = P->n_true + 1;
    if (P->init) {
        P->init = 0;
        const double r0 = sqrt(rrt);
        P->r0 = r0;
        if (!isfinite(r0)) { P->rel = r0; finish(EBE_BREAKDOWN); return; }
        if (!(r0 > 0.0)) { P->rel = 0.0; finish(EBE_OK); return; }
        P->rel = 1.0;
        P->best = 1.0;
        P->rho = rz;
        P->beta = 0.0;
        P->dir_init = 1;
        const double fin = bd.rtol * r0;
        P->fin = fin;
        const double thr = MIXED ? fmax(bd.delta * r0, fin) : fin;
        P->thr2 = thr * thr;
        P->mode = kBNormal;
        return;
    }
    const double rel = sqrt(rrt) / P->r0;
    P->rel = rel;
    if (!isfinite(rel)) { finish(EBE_BREAKDOWN); return; }
    if (rel <= bd.rtol) { finish(EBE_OK); return; }
    if (P->bd) { finish(EBE_BREAKDOWN); return; }
    if (P->iter >= bd.maxit) { finish(EBE_MAXIT); return; }
    if (rel < 0.9 * P->best) {
        P->best = rel;
        P->no_progress = 0;
    } else {
        const int np = P->no_progress + 1;
        P->no_progress = np;
        if (np >= bd.stall_updates) { finish(EBE_STALL); return; }
    }
    // mixed precision: a failed check at the final threshold tightens it
    // (the FP32 recurrence residual drifted below the true one)
    double fin = P->fin;
    if (MIXED && P->thr2 <= fin * fin) {
        fin *= bd.margin;
        P->fin = fin;
    }
    // residual replacement: continue CG from the true residual, same direction
    const double rho = P->rho;
    P->beta = rho != 0.0 ? rz / rho : 0.0;
    P->rho = rz;
    P->dir_init = 0;
    const double thr = MIXED ? fmax(bd.delta * sqrt(rrt), fin) : fin;
    P->thr2 = thr * thr;
    P->mode = kBNormal;
}

// ---------------------------------------------------------------- phase U
template <typename T, int NB>
__device__ __forceinline__ void update_item(Ctx& c, int ti, int md) {
    constexpr bool MIXED = sizeof(T) == 4;
    const BatchDev& bd = *c.bd;
    unsigned char* smem = c.smem;
    const BatchSmem Lo = layout_of<T, NB>(bd);
    double* red = reinterpret_cast<double*>(smem + Lo.red);
    volatile int* last = reinterpret_cast<volatile int*>(smem + Lo.last);
    const int tid = threadIdx.x;
    const BatchItem it = bd.tile[ti];
    const T* pv = static_cast<const T*>(bd.p);
    const T* q = static_cast<const T*>(bd.q);
    const T* dinv = static_cast<const T*>(bd.dinv);
    double* x = bd.x;
    double* r = bd.r;
    T* ri_v = static_cast<T*>(bd.rin);   // recurrence residual (FP32 when mixed)
    double a = 0.0, b = 0.0;       // per-thread sums of the FP64 solver
    CompSum ca, cb;                // per-thread sums of the mixed solver (compensated FP32)
    const BatchProblem* P = bd.prob + it.k;
    if (md == kBNormal) {
        const double al = ld_l2(&P->alpha);
        const int brk = ld_l2(&P->bd);
        if (!brk) {
            if constexpr (MIXED) {
                // x += alpha p in FP64; r -= alpha q and z = dinv r in FP32
                const float alf = d2f(al);
                CompSum rz, rr;
                int i = it.lo + tid;
                for (; i + 3 * NT < it.hi; i += 4 * NT) {
                    float pq[4], qq[4], dv[4], rv[4];
                    double xv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = i + u * NT;
                        pq[u] = ld_l2(pv + j); qq[u] = ld_l2(q + j); dv[u] = __ldg(dinv + j);
                        xv[u] = ld_l2(x + j); rv[u] = ld_l2(ri_v + j);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = i + u * NT;
                        x[j] = fmadd(al, f2d(pq[u]), xv[u]);
                        const float rf = __fmaf_rn(-alf, qq[u], rv[u]);
                        ri_v[j] = rf;
                        rz.add(rf * (dv[u] * rf));
                        rr.add(rf * rf);
                    }
                }
                for (; i < it.hi; i += NT) {
                    x[i] = fmadd(al, f2d(ld_l2(pv + i)), ld_l2(x + i));
                    const float rf = __fmaf_rn(-alf, ld_l2(q + i), ld_l2(ri_v + i));
                    ri_v[i] = rf;
                    rz.add(rf * (__ldg(dinv + i) * rf));
                    rr.add(rf * rf);
                }
                ca = rz;
                cb = rr;
            } else {
                int i = it.lo + tid;
                for (; i + 3 * NT < it.hi; i += 4 * NT) {
                    double pq[4], qq[4], dv[4], xv[4], rv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = i + u * NT;
                        pq[u] = ld_l2(pv + j); qq[u] = ld_l2(q + j); dv[u] = __ldg(dinv + j);
                        xv[u] = ld_l2(x + j); rv[u] = ld_l2(r + j);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = i + u * NT;
                        x[j] = fmadd(al, pq[u], xv[u]);
                        const double ri = fmadd(-al, qq[u], rv[u]);
                        r[j] = ri;
                        a = fmadd(ri, dv[u] * ri, a);
                        b = fmadd(ri, ri, b);
                    }
                }
                for (; i < it.hi; i += NT) {
                    x[i] = fmadd(al, ld_l2(pv + i), ld_l2(x + i));
                    const double ri = fmadd(-al, ld_l2(q + i), ld_l2(r + i));
                    r[i] = ri;
                    a = fmadd(ri, __ldg(dinv + i) * ri, a);
                    b = fmadd(ri, ri, b);
                }
            }
        }
    } else {
        // after a replacement: the sums of the restart, z formed as in the
        // update; mixed: the FP32 recurrence residual restarts from the true one
        if constexpr (MIXED) {
            CompSum rz, rr;
            for (int i = it.lo + tid; i < it.hi; i += NT) {
                const float rf = d2f(ld_l2(r + i));
                ri_v[i] = rf;
                rz.add(rf * (__ldg(dinv + i) * rf));
                rr.add(rf * rf);
            }
            ca = rz;
            cb = rr;
        } else {
            for (int i = it.lo + tid; i < it.hi; i += NT) {
                const double ri = ld_l2(r + i);
                a = fmadd(ri, __ldg(dinv + i) * ri, a);
                b = fmadd(ri, ri, b);
            }
        }
    }
    if constexpr (MIXED) {
        CompSum v[2] = {ca, cb};
        double t[2];
        block_sums_comp<2, NT>(v, t, red);
        a = t[0];
        b = t[1];
    } else {
        block_sum2<NT>(a, b, red);
    }
    if (tid == 0) {
        bd.part_u[2 * ti] = a;
        bd.part_u[2 * ti + 1] = b;
        *last = tma::atom_add_acq_rel(bd.ctr + bd.n_prob + it.k, 1u) == uint32_t(it.count - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!*last) return;
    double sa = 0.0, sb = 0.0;
    for (int i = tid; i < it.count; i += NT) {
        sa += ld_l2(bd.part_u + 2 * (it.first + i));
        sb += ld_l2(bd.part_u + 2 * (it.first + i) + 1);
    }
    block_sum2<NT>(sa, sb, red);
    if (tid == 0) {
        bd.ctr[bd.n_prob + it.k] = 0u;
        decide<MIXED>(bd, it.k, md, sa, sb);
    }
}

// ---------------------------------------------------------------- phase D
template <typename T>
__device__ __forceinline__ void direction_item(Ctx& c, int ti) {
    const BatchDev& bd = *c.bd;
    const BatchItem it = bd.tile[ti];
    const BatchProblem* P = bd.prob + it.k;
    const int init = ld_l2(&P->dir_init);
    const T be = T(ld_l2(&P->beta));
    T* pv = static_cast<T*>(bd.p);
    const T* dinv = static_cast<const T*>(bd.dinv);
    const T* r = static_cast<const T*>(bd.rin);
    int i = it.lo + int(threadIdx.x);
    for (; i + 3 * NT < it.hi; i += 4 * NT) {
        T rv[4], dv[4], pq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = i + u * NT;
            rv[u] = ld_l2(r + j); dv[u] = __ldg(dinv + j); pq[u] = init ? T(0) : ld_l2(pv + j);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const T zi = dv[u] * rv[u];
            pv[i + u * NT] = init ? zi : fmadd(be, pq[u], zi);
        }
    }
    for (; i < it.hi; i += NT) {
        const T zi = __ldg(dinv + i) * ld_l2(r + i);
        pv[i] = init ? zi : fmadd(be, ld_l2(pv + i), zi);
    }
}

// ---------------------------------------------------------------- scheduling
// Exclusive block scan of four counters; scratch: 8 int4 (NT = 256).
__device__ __forceinline__ int4 block_exscan4(int4 v, int4* scratch, int4& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int4 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, inc.x, o), b = __shfl_up_sync(0xffffffffu, inc.y, o);
        const int c = __shfl_up_sync(0xffffffffu, inc.z, o), d = __shfl_up_sync(0xffffffffu, inc.w, o);
        if (lane >= o) { inc.x += a; inc.y += b; inc.z += c; inc.w += d; }
    }
    __syncthreads();
    if (lane == 31) scratch[w] = inc;
    __syncthreads();
    int4 base = make_int4(0, 0, 0, 0);
    total = make_int4(0, 0, 0, 0);
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) {
        const int4 t = scratch[i];
        if (i < w) { base.x += t.x; base.y += t.y; base.z += t.z; base.w += t.w; }
        total.x += t.x; total.y += t.y; total.z += t.z; total.w += t.w;
    }
    return make_int4(base.x + inc.x - v.x, base.y + inc.y - v.y, base.z + inc.z - v.z, base.w + inc.w - v.w);
}

// The live-problem list and the prefix sums of their item counts (all threads).
__device__ __forceinline__ void rebuild_lists(const BatchDev& bd, const int8_t* smode, int32_t* list, int32_t* pre,
                                              volatile int* snl, int4* scratch) {
    const int n = bd.n_prob;
    const int per = (n + NT - 1) / NT;
    const int k0 = min(n, int(threadIdx.x) * per), k1 = min(n, k0 + per);
    int4 c = make_int4(0, 0, 0, 0);
    for (int k = k0; k < k1; ++k) {
        if (smode[k] == kBDone) continue;
        const BatchProbInfo pi = bd.pinfo[k];
        c.x += 1; c.y += pi.patch_count; c.z += pi.fix_count; c.w += pi.tile_count;
    }
    int4 tot;
    int4 o = block_exscan4(c, scratch, tot);
    int32_t* pp = pre;
    int32_t* pf = pre + (n + 1);
    int32_t* pt = pre + 2 * (n + 1);
    for (int k = k0; k < k1; ++k) {
        if (smode[k] == kBDone) continue;
        const BatchProbInfo pi = bd.pinfo[k];
        list[o.x] = k;
        pp[o.x] = o.y;
        pf[o.x] = o.z;
        pt[o.x] = o.w;
        o.x += 1; o.y += pi.patch_count; o.z += pi.fix_count; o.w += pi.tile_count;
    }
    if (threadIdx.x == 0) {
        pp[tot.x] = tot.y;
        pf[tot.x] = tot.z;
        pt[tot.x] = tot.w;
        *snl = tot.x;
    }
    __syncthreads();
}

// Position j of the live list whose items contain item i: pre[j] <= i < pre[j + 1].
__device__ __forceinline__ int find_item(const int32_t* pre, int nl, int i) {
    int lo = 0, hi = nl;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- the persistent kernel
template <typename T, int NB>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && NB == 3) ? 4 : 2)
k_batch_pcg(const __grid_constant__ BatchDev bd) {
    extern __shared__ __align__(128) unsigned char smem[];
    Ctx c;
    c.bd = &bd;
    c.smem = smem;
    c.mph = 0;
    const BatchSmem Lo = layout_of<T, NB>(bd);
    volatile int* sflag = reinterpret_cast<volatile int*>(smem + Lo.flag);
    volatile int* broken = reinterpret_cast<volatile int*>(smem + Lo.broken);
    volatile int* slive = reinterpret_cast<volatile int*>(smem + Lo.live);
    volatile int* snl = reinterpret_cast<volatile int*>(smem + Lo.nl);
    volatile int* sver = reinterpret_cast<volatile int*>(smem + Lo.ver);
    int8_t* smode = reinterpret_cast<int8_t*>(smem + Lo.mode);
    int32_t* list = reinterpret_cast<int32_t*>(smem + Lo.list);
    int32_t* pre = reinterpret_cast<int32_t*>(smem + Lo.pre);
    const int32_t* pre_p = pre;
    const int32_t* pre_f = pre + (bd.n_prob + 1);
    const int32_t* pre_t = pre + 2 * (bd.n_prob + 1);
    int4* scratch = reinterpret_cast<int4*>(smem + Lo.red);
    uint64_t* tph = reinterpret_cast<uint64_t*>(smem + Lo.timer);   // [5]: phase times, last lap
    const int tid = threadIdx.x;
    const uint32_t G = gridDim.x;

    // problem modes and, when a problem has finished since the last look,
    // the live list (every CTA sees the same state after a grid barrier)
    auto refresh = [&]() {
        for (int k = tid; k < bd.n_prob; k += NT) smode[k] = int8_t(ld_l2(&bd.prob[k].mode));
        if (tid == 0) *slive = ld_l2(bd.live);
        __syncthreads();
        if (*slive != *sver) {
            rebuild_lists(bd, smode, list, pre, snl, scratch);
            if (tid == 0) *sver = *slive;
            __syncthreads();
        }
    };
    // phase times (thread 0 of CTA 0, in shared memory): from one barrier exit to the next
    const bool timer = blockIdx.x == 0 && tid == 0;
    if (tid == 0) {
        tma::mbar_init(tma::smem_addr(smem + Lo.bar), 1);
        *broken = 0;
        *sver = -1;
        for (int ph = 0; ph < 4; ++ph) tph[ph] = 0;
        tph[4] = tma::globaltimer_ns();
    }
    __syncthreads();
    refresh();
    const uint64_t lim = bd.barrier_ns;
    auto lap = [&](int ph) {
        if (timer) {
            const uint64_t t = tma::globaltimer_ns();
            tph[ph] += t - tph[4];
            tph[4] = t;
        }
    };
    auto flush = [&]() {
        if (timer)
            for (int ph = 0; ph < 4; ++ph) atomicAdd(bd.phase_ns + ph, (unsigned long long)tph[ph]);
    };

    // patch whose bulk copies are in flight for this CTA's next apply (-1: none)
    int pf = -1;
    const uint32_t mbar = tma::smem_addr(smem + Lo.bar);
    // the patch of item i if it is an operator application, else -1
    auto next_apply = [&](int i, int nlv) {
        if (i >= pre_p[nlv]) return -1;
        const int j = find_item(pre_p, nlv, i);
        const int k = list[j];
        return smode[k] == kBNormal ? __ldg(&bd.pinfo[k].patch_first) + (i - pre_p[j]) : -1;
    };
    // copies still in flight when the CTA leaves: wait for them (bounded)
    auto drain = [&]() {
        if (pf >= 0 && tid == 0) tma::mbar_wait_bounded(mbar, c.mph, nullptr);
    };

    for (int64_t loop = 0; loop < bd.iter_budget; ++loop) {
        if (*slive <= 0) break;
        const int nl = *snl;
        // P
        if (!*broken)
            for (int i = int(blockIdx.x); i < pre_p[nl]; i += int(G)) {
                const int j = find_item(pre_p, nl, i);
                const int k = list[j];
                const int p = __ldg(&bd.pinfo[k].patch_first) + (i - pre_p[j]);
                if (smode[k] == kBNormal) {
                    const int nxt = next_apply(i + int(G), nl);
                    if (!apply_patch<T, NB>(c, p, pf == p, nxt)) {
                        pf = -1;
                        break;
                    }
                    pf = nxt;
                } else {
                    residual_patch<T, NB>(c, p, ld_l2(&bd.prob[k].exact) != 0);
                }
            }
        if (!tma::grid_sync(bd.bar, G, bd.pd.err, sflag, lim)) { drain(); return; }
        lap(0);
        // The element matrices are constant: the copies of this CTA's first
        // patch of the next loop start now and land during F, U and D (if U
        // changes which patch that is, they are waited for and dropped).
        if (!*broken && pf < 0 && loop + 1 < bd.iter_budget) {
            pf = next_apply(int(blockIdx.x), nl);
            if (pf >= 0 && tid == 0) issue_patch_copies<T, NB>(bd, smem, pf);
        }
        // F
        for (int i = int(blockIdx.x); i < pre_f[nl]; i += int(G)) {
            const int j = find_item(pre_f, nl, i);
            const int k = list[j];
            fix_item<T, NB>(c, __ldg(&bd.pinfo[k].fix_first) + (i - pre_f[j]), smode[k]);
        }
        if (!tma::grid_sync(bd.bar, G, bd.pd.err, sflag, lim)) { drain(); return; }
        lap(1);
        // U
        for (int i = int(blockIdx.x); i < pre_t[nl]; i += int(G)) {
            const int j = find_item(pre_t, nl, i);
            const int k = list[j];
            update_item<T, NB>(c, __ldg(&bd.pinfo[k].tile_first) + (i - pre_t[j]), smode[k]);
        }
        if (!tma::grid_sync(bd.bar, G, bd.pd.err, sflag, lim)) { drain(); return; }
        refresh();
        if (pf >= 0 && pf != next_apply(int(blockIdx.x), *snl)) {
            if (tid == 0 && !tma::mbar_wait_bounded(mbar, c.mph, bd.pd.err)) *broken = 1;
            c.mph ^= 1u;
            pf = -1;
            __syncthreads();
        }
        lap(2);
        // D (the list may have shrunk: problems finished in U are gone)
        const int nl2 = *snl;
        for (int i = int(blockIdx.x); i < pre_t[nl2]; i += int(G)) {
            const int j = find_item(pre_t, nl2, i);
            const int k = list[j];
            if (smode[k] != kBNormal) continue;
            direction_item<T>(c, __ldg(&bd.pinfo[k].tile_first) + (i - pre_t[j]));
        }
        if (blockIdx.x == 0 && tid == 0) *bd.loops += 1;
        if (!tma::grid_sync(bd.bar, G, bd.pd.err, sflag, lim)) { drain(); return; }
        lap(3);
    }
    drain();
    flush();
}

__global__ void k_batch_init(BatchProblem* prob, int n_prob, uint32_t* ctr, uint32_t* bar, int32_t* live,
                             int64_t* loops, unsigned long long* phase_ns) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n_prob) {
        BatchProblem P{};
        P.mode = kBReplace;
        P.status = EBE_OK;
        P.init = 1;
        prob[k] = P;
        ctr[k] = 0u;
        ctr[n_prob + k] = 0u;
    }
    if (k == 0) {
        bar[0] = 0u;
        bar[1] = 0u;
        *live = n_prob;
        *loops = 0;
        for (int ph = 0; ph < 4; ++ph) phase_ns[ph] = 0ull;
    }
}

template <typename T, int NB>
int smem_for(const BatchDev& bd) {
    return int(batch_layout<T, NB>(bd.pd.max_nodes, bd.n_prob).total);
}

template <typename T, int NB>
int max_ctas(const BatchDev& bd, int* smem_bytes) {
    auto kern = k_batch_pcg<T, NB>;
    int best = 0;
    for (int c = 1; c <= 8; ++c) {
        const int sm = smem_for<T, NB>(bd);
        if (sm > 227 * 1024) break;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) break;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, size_t(sm)) != cudaSuccess) break;
        if (occ >= c) {
            best = c;
            if (smem_bytes) *smem_bytes = sm;
        }
    }
    return best;
}

template <typename T, int NB>
cudaError_t run_batch(const BatchDev& bd, int ctas_per_sm, cudaStream_t st) {
    auto kern = k_batch_pcg<T, NB>;
    const int grid = ctas_per_sm * bd.pd.num_sms;
    const int sm = smem_for<T, NB>(bd);
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = size_t(sm);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, bd);
}

}  // namespace

cudaError_t launch_batch_init(const BatchDev& bd, cudaStream_t st, int* launches) {
    const int nt = 256;
    k_batch_init<<<(bd.n_prob + nt - 1) / nt, nt, 0, st>>>(bd.prob, bd.n_prob, bd.ctr, bd.bar, bd.live, bd.loops,
                                                                bd.phase_ns);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

int batch_max_ctas_per_sm(const BatchDev& bd, bool mixed, int* smem_bytes) {
    if (mixed) return bd.pd.nb == 3 ? max_ctas<float, 3>(bd, smem_bytes) : max_ctas<float, 4>(bd, smem_bytes);
    return bd.pd.nb == 3 ? max_ctas<double, 3>(bd, smem_bytes) : max_ctas<double, 4>(bd, smem_bytes);
}

cudaError_t launch_batch_solve(const BatchDev& bd, bool mixed, int ctas_per_sm, cudaStream_t st, int* launches) {
    if (ctas_per_sm < 1) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    if (mixed) e = bd.pd.nb == 3 ? run_batch<float, 3>(bd, ctas_per_sm, st) : run_batch<float, 4>(bd, ctas_per_sm, st);
    else e = bd.pd.nb == 3 ? run_batch<double, 3>(bd, ctas_per_sm, st) : run_batch<double, 4>(bd, ctas_per_sm, st);
    if (launches) *launches += 1;
    return e;
}

}  // namespace ebe
