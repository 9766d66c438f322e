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
// The per-problem decisions follow the single-problem solver: mixed
// precision keeps x and r in FP64 and replaces the recurrence residual by
// the FP64 true residual whenever it has dropped by delta; a problem is done
// when its true relative residual reaches rtol.  Problems that are done cost
// nothing but a shared-memory lookup per item.  Every sum is taken in a fixed
// order, so a solve is bitwise reproducible for a given launch shape.
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

// Data written during the launch by other CTAs is read through L2 only.
template <typename V>
__device__ __forceinline__ V ld_l2(const V* p) { return __ldcg(p); }

// ---------------------------------------------------------------- shared memory
struct BatchSmem {
    uint32_t bar, flag, broken, live, last, red, co, mode, sp, sf, st;
    uint32_t A, L, G, xs, acc;        // inner-operator patch pass
    uint32_t G2, xs2, bs2, acc2;      // FP64 true-residual patch pass (same region)
    uint32_t total;
};
__host__ __device__ constexpr uint32_t up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

template <typename T, int NB>
__host__ __device__ constexpr BatchSmem batch_layout(int max_nodes, int n_prob, int cap_p, int cap_f, int cap_t) {
    BatchSmem s{};
    const uint32_t gcap = uint32_t((max_nodes + 3) / 4 * 4);
    s.bar = 0;
    s.flag = 8;
    s.broken = 12;
    s.live = 16;
    s.last = 20;
    s.red = 32;                                      // 2 * NT / 32 doubles
    s.co = s.red + 2 * (NT / 32) * 8;
    s.mode = up(s.co + (kMaxColours + 1) * 4, 16);   // int8 per problem
    s.sp = up(s.mode + uint32_t(n_prob), 16);
    s.sf = s.sp + uint32_t(cap_p) * 4;
    s.st = s.sf + uint32_t(cap_f) * 4;
    s.A = up(s.st + uint32_t(cap_t) * 4, 128);
    s.L = s.A + uint32_t(NB * NB * kPatch * sizeof(T));
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

struct Ctx {
    const BatchDev* bd;
    unsigned char* smem;
    BatchSmem L;
    uint32_t mbar;
    uint32_t mph;
};

// ---------------------------------------------------------------- phase P
// q = A p on one patch (inner type T): the element matrices and local
// connectivity come in by TMA bulk copies while the threads gather the node
// table and p; products first, then colour rounds add them into the node
// sums (FP32: difference form, the diagonal slot holds the row sum).
// Returns false in every thread if the bulk copies did not arrive in time
// (the device error flag is set; the CTA stops its patch work).
template <typename T, int NB>
__device__ __forceinline__ bool apply_patch(Ctx& c, int p) {
    const BatchDev& bd = *c.bd;
    const PlanDev& pd = bd.pd;
    unsigned char* smem = c.smem;
    volatile int* flag = reinterpret_cast<volatile int*>(smem + c.L.broken);
    double* red = reinterpret_cast<double*>(smem + c.L.red);
    int* co = reinterpret_cast<int*>(smem + c.L.co);
    T* As = reinterpret_cast<T*>(smem + c.L.A);
    uint16_t* Ls = reinterpret_cast<uint16_t*>(smem + c.L.L);
    int32_t* Gs = reinterpret_cast<int32_t*>(smem + c.L.G);
    T* xs = reinterpret_cast<T*>(smem + c.L.xs);
    T* acc = reinterpret_cast<T*>(smem + c.L.acc);
    const T* A = static_cast<const T*>(bd.A);
    const T* pv = static_cast<const T*>(bd.p);
    T* q = static_cast<T*>(bd.q);
    T* halo = static_cast<T*>(bd.halo);
    const int tid = threadIdx.x;
    const int64_t ns = pd.n_slots;
    const int64_t slot0 = int64_t(p) * kPatch;
    const PatchMeta m = pd.meta[p];

    __syncthreads();   // the previous item's reads of shared memory are done
    if (tid == 0) {
        const uint64_t pol = tma::policy_evict_first();
        tma::mbar_expect_tx(c.mbar, uint32_t(NB * NB * kPatch * sizeof(T)) + uint32_t(NB * kPatch * 2));
#pragma unroll
        for (int t = 0; t < NB * NB; ++t)
            tma::bulk_load(tma::smem_addr(As + t * kPatch), A + t * ns + slot0, uint32_t(kPatch * sizeof(T)), c.mbar, pol);
#pragma unroll
        for (int i = 0; i < NB; ++i)
            tma::bulk_load(tma::smem_addr(Ls + i * kPatch), pd.lconn + i * ns + slot0, uint32_t(kPatch * 2), c.mbar, pol);
    }
    for (int k = tid; k <= m.n_col; k += NT) co[k] = __ldg(pd.col_ptr + m.col_off + k);
    const int32_t* pn = pd.pnode + m.node_off;
    for (int l = tid; l < m.n_nodes; l += NT) {
        const int32_t gr = __ldg(pn + l);
        Gs[l] = gr;
        xs[l] = ld_l2(pv + (gr & kNodeMask));
        acc[l] = T(0);
    }
    // *flag (the CTA's "broken" word) stays 1 from here on if the copies are lost:
    // this CTA does no more patch work and the next grid barrier ends the launch
    if (tid == 0 && !tma::mbar_wait_bounded(c.mbar, c.mph, pd.err)) *flag = 1;
    __syncthreads();
    const uint32_t ph = c.mph;
    c.mph ^= 1u;
    if (*flag != 0) return false;
    while (!tma::mbar_try_wait(c.mbar, ph)) {
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
                v = ok ? As[(r * NB + r) * kPatch + s] * xe[r] : T(0);
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    if (j != r) v = ok ? fmadd(As[(r * NB + j) * kPatch + s], xe[j] - xe[r], v) : v;
            } else {
                v = T(0);
#pragma unroll
                for (int j = 0; j < NB; ++j) v = ok ? fmadd(As[(r * NB + j) * kPatch + s], xe[j], v) : v;
            }
            y[k][r] = v;
        }
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
    const double dsum = block_sum<NT>(dot.value(), red);
    if (tid == 0) bd.part_p[p] = dsum;
    return true;
}

// FP64 true residual r = mask(b - A x) on one patch; element matrices read
// straight from global memory (coalesced: slot-major runs), products first.
template <int NB>
__device__ __forceinline__ void residual_patch(Ctx& c, int p) {
    const BatchDev& bd = *c.bd;
    const PlanDev& pd = bd.pd;
    unsigned char* smem = c.smem;
    double* red = reinterpret_cast<double*>(smem + c.L.red);
    int* co = reinterpret_cast<int*>(smem + c.L.co);
    int32_t* Gs = reinterpret_cast<int32_t*>(smem + c.L.G2);
    double* xs = reinterpret_cast<double*>(smem + c.L.xs2);
    double* bs = reinterpret_cast<double*>(smem + c.L.bs2);
    double* acc = reinterpret_cast<double*>(smem + c.L.acc2);
    const int tid = threadIdx.x;
    const int64_t ns = pd.n_slots;
    const int64_t slot0 = int64_t(p) * kPatch;
    const PatchMeta m = pd.meta[p];

    __syncthreads();
    for (int k = tid; k <= m.n_col; k += NT) co[k] = __ldg(pd.col_ptr + m.col_off + k);
    const int32_t* pn = pd.pnode + m.node_off;
    for (int l = tid; l < m.n_nodes; l += NT) {
        const int32_t gr = __ldg(pn + l);
        const int g = gr & kNodeMask;
        Gs[l] = gr;
        xs[l] = ld_l2(bd.x + g);
        bs[l] = l < m.n_owned ? __ldg(bd.b + g) : 0.0;
        acc[l] = 0.0;
    }
    __syncthreads();
    int ln[kEPT][NB];
    double y[kEPT][NB];
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
        const int s = tid + k * NT;
        const bool ok = s < m.n_el;
        double xe[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            ln[k][i] = ok ? int(__ldg(pd.lconn + i * ns + slot0 + s)) : 0;
            xe[i] = xs[ln[k][i]];
        }
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            double v = 0.0;
#pragma unroll
            for (int j = 0; j < NB; ++j) v = ok ? fmadd(__ldg(bd.A64 + (r * NB + j) * ns + slot0 + s), xe[j], v) : v;
            y[k][r] = v;
        }
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
template <typename T>
__device__ __forceinline__ void fix_item(Ctx& c, int ci, int md) {
    const BatchDev& bd = *c.bd;
    const PlanDev& pd = bd.pd;
    unsigned char* smem = c.smem;
    double* red = reinterpret_cast<double*>(smem + c.L.red);
    volatile int* last = reinterpret_cast<volatile int*>(smem + c.L.last);
    const int tid = threadIdx.x;
    const BatchItem it = bd.fix[ci];
    double dsum;
    if (md == kBNormal) {
        const T* halo = static_cast<const T*>(bd.halo);
        const T* pv = static_cast<const T*>(bd.p);
        T* q = static_cast<T*>(bd.q);
        DotAcc<T> dot;
        for (int row = it.lo + tid; row < it.hi; row += NT) {
            const int32_t graw = __ldg(pd.sh_node + row);
            const int g = graw & kNodeMask;
            T v = T(0);
            const int s1 = __ldg(pd.sh_ptr + row + 1);
            for (int s = __ldg(pd.sh_ptr + row); s < s1; ++s) v += ld_l2(halo + __ldg(pd.sh_slot + s));
            const T o = graw < 0 ? T(0) : v;
            q[g] = o;
            dot.add(ld_l2(pv + g), o);
        }
        dsum = dot.value();
    } else {
        double dot = 0.0;
        for (int row = it.lo + tid; row < it.hi; row += NT) {
            const int32_t graw = __ldg(pd.sh_node + row);
            const int g = graw & kNodeMask;
            double v = 0.0;
            const int s1 = __ldg(pd.sh_ptr + row + 1);
            for (int s = __ldg(pd.sh_ptr + row); s < s1; ++s) v += ld_l2(bd.halo64 + __ldg(pd.sh_slot + s));
            const double o = graw < 0 ? 0.0 : __ldg(bd.b + g) - v;
            bd.r[g] = o;
            dot = fmadd(o, o, dot);
        }
        dsum = dot;
    }
    for (int i = it.plo + tid; i < it.phi; i += NT) dsum += ld_l2(bd.part_p + i);
    dsum = block_sum<NT>(dsum, red);
    if (tid == 0) {
        bd.part_f[ci] = dsum;
        __threadfence();
        *last = atomicAdd(bd.ctr + it.k, 1u) == uint32_t(it.count - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!*last) return;
    __threadfence();
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
            P->mode = kBReplace;                // a last true residual, then done
        } else if (rr <= P->thr2 || it >= bd.maxit) {
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
        const double fin = (MIXED ? bd.margin : 1.0) * bd.rtol * r0;
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
    // residual replacement: continue CG from the true residual, same direction
    const double rho = P->rho;
    P->beta = rho != 0.0 ? rz / rho : 0.0;
    P->rho = rz;
    P->dir_init = 0;
    const double fin = (MIXED ? bd.margin : 1.0) * bd.rtol * P->r0;
    const double thr = MIXED ? fmax(bd.delta * sqrt(rrt), fin) : fin;
    P->thr2 = thr * thr;
    P->mode = kBNormal;
}

// ---------------------------------------------------------------- phase U
template <typename T>
__device__ __forceinline__ void update_item(Ctx& c, int ti, int md) {
    constexpr bool MIXED = sizeof(T) == 4;
    const BatchDev& bd = *c.bd;
    unsigned char* smem = c.smem;
    double* red = reinterpret_cast<double*>(smem + c.L.red);
    volatile int* last = reinterpret_cast<volatile int*>(smem + c.L.last);
    const int tid = threadIdx.x;
    const BatchItem it = bd.tile[ti];
    const T* pv = static_cast<const T*>(bd.p);
    const T* q = static_cast<const T*>(bd.q);
    const T* dinv = static_cast<const T*>(bd.dinv);
    double* x = bd.x;
    double* r = bd.r;
    double a = 0.0, b = 0.0;
    const BatchProblem* P = bd.prob + it.k;
    if (md == kBNormal) {
        const double al = ld_l2(&P->alpha);
        const int brk = ld_l2(&P->bd);
        if (!brk) {
            if constexpr (MIXED) {
                CompSum rz, rr;
                int i = it.lo + tid;
                for (; i + 3 * NT < it.hi; i += 4 * NT) {
                    float pq[4], qq[4], dv[4];
                    double xv[4], rv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = i + u * NT;
                        pq[u] = ld_l2(pv + j); qq[u] = ld_l2(q + j); dv[u] = __ldg(dinv + j);
                        xv[u] = ld_l2(x + j); rv[u] = ld_l2(r + j);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = i + u * NT;
                        x[j] = fmadd(al, f2d(pq[u]), xv[u]);
                        const double ri = fmadd(-al, f2d(qq[u]), rv[u]);
                        r[j] = ri;
                        const float rf = d2f(ri);
                        rz.add(rf * (dv[u] * rf));
                        rr.add(rf * rf);
                    }
                }
                for (; i < it.hi; i += NT) {
                    x[i] = fmadd(al, f2d(ld_l2(pv + i)), ld_l2(x + i));
                    const double ri = fmadd(-al, f2d(ld_l2(q + i)), ld_l2(r + i));
                    r[i] = ri;
                    const float rf = d2f(ri);
                    rz.add(rf * (__ldg(dinv + i) * rf));
                    rr.add(rf * rf);
                }
                a = rz.value();
                b = rr.value();
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
        // after a replacement: the sums of the restart, z formed as in the update
        if constexpr (MIXED) {
            CompSum rz, rr;
            for (int i = it.lo + tid; i < it.hi; i += NT) {
                const float rf = d2f(ld_l2(r + i));
                rz.add(rf * (__ldg(dinv + i) * rf));
                rr.add(rf * rf);
            }
            a = rz.value();
            b = rr.value();
        } else {
            for (int i = it.lo + tid; i < it.hi; i += NT) {
                const double ri = ld_l2(r + i);
                a = fmadd(ri, __ldg(dinv + i) * ri, a);
                b = fmadd(ri, ri, b);
            }
        }
    }
    block_sum2<NT>(a, b, red);
    if (tid == 0) {
        bd.part_u[2 * ti] = a;
        bd.part_u[2 * ti + 1] = b;
        __threadfence();
        *last = atomicAdd(bd.ctr + bd.n_prob + it.k, 1u) == uint32_t(it.count - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!*last) return;
    __threadfence();
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
    const double* r = bd.r;
    int i = it.lo + int(threadIdx.x);
    for (; i + 3 * NT < it.hi; i += 4 * NT) {
        double rv[4];
        T dv[4], pq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = i + u * NT;
            rv[u] = ld_l2(r + j); dv[u] = __ldg(dinv + j); pq[u] = init ? T(0) : ld_l2(pv + j);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            T zi;
            if constexpr (sizeof(T) == 4) zi = dv[u] * d2f(rv[u]);
            else zi = dv[u] * rv[u];
            pv[i + u * NT] = init ? zi : fmadd(be, pq[u], zi);
        }
    }
    for (; i < it.hi; i += NT) {
        T zi;
        if constexpr (sizeof(T) == 4) zi = __ldg(dinv + i) * d2f(ld_l2(r + i));
        else zi = __ldg(dinv + i) * ld_l2(r + i);
        pv[i] = init ? zi : fmadd(be, ld_l2(pv + i), zi);
    }
}

// ---------------------------------------------------------------- the persistent kernel
template <typename T, int NB>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && NB == 3) ? 4 : 2)
k_batch_pcg(const __grid_constant__ BatchDev bd, int cap_p, int cap_f, int cap_t) {
    constexpr bool MIXED = sizeof(T) == 4;
    extern __shared__ __align__(128) unsigned char smem[];
    Ctx c;
    c.bd = &bd;
    c.smem = smem;
    c.L = batch_layout<T, NB>(bd.pd.max_nodes, bd.n_prob, cap_p, cap_f, cap_t);
    c.mbar = tma::smem_addr(smem + c.L.bar);
    c.mph = 0;
    volatile int* sflag = reinterpret_cast<volatile int*>(smem + c.L.flag);
    volatile int* broken = reinterpret_cast<volatile int*>(smem + c.L.broken);
    volatile int* slive = reinterpret_cast<volatile int*>(smem + c.L.live);
    int8_t* smode = reinterpret_cast<int8_t*>(smem + c.L.mode);
    int32_t* sp = reinterpret_cast<int32_t*>(smem + c.L.sp);
    int32_t* sf = reinterpret_cast<int32_t*>(smem + c.L.sf);
    int32_t* stl = reinterpret_cast<int32_t*>(smem + c.L.st);
    const int tid = threadIdx.x;
    const uint32_t G = gridDim.x;
    const int np = bd.pd.n_patches;

    // this CTA's items (static: item blockIdx.x + j G) and their problems
    for (int j = tid; j < cap_p; j += NT) {
        const int64_t p = int64_t(blockIdx.x) + int64_t(j) * G;
        sp[j] = p < np ? __ldg(bd.patch_prob + p) : -1;
    }
    for (int j = tid; j < cap_f; j += NT) {
        const int64_t i = int64_t(blockIdx.x) + int64_t(j) * G;
        sf[j] = i < bd.n_fix ? __ldg(&bd.fix[i].k) : -1;
    }
    for (int j = tid; j < cap_t; j += NT) {
        const int64_t i = int64_t(blockIdx.x) + int64_t(j) * G;
        stl[j] = i < bd.n_tile ? __ldg(&bd.tile[i].k) : -1;
    }
    auto refresh = [&]() {
        for (int k = tid; k < bd.n_prob; k += NT) smode[k] = int8_t(ld_l2(&bd.prob[k].mode));
        if (tid == 0) *slive = ld_l2(bd.live);
        __syncthreads();
    };
    if (tid == 0) {
        tma::mbar_init(c.mbar, 1);
        *broken = 0;
    }
    refresh();
    const uint64_t lim = bd.barrier_ns;

    for (int64_t loop = 0; loop < bd.iter_budget; ++loop) {
        if (*slive <= 0) break;
        // P
        if (!*broken)
            for (int j = 0; j < cap_p; ++j) {
                const int k = sp[j];
                if (k < 0) break;
                const int md = smode[k];
                if (md == kBDone) continue;
                const int p = int(blockIdx.x + uint32_t(j) * G);
                if (md == kBNormal) {
                    if (!apply_patch<T, NB>(c, p)) break;
                } else {
                    residual_patch<NB>(c, p);
                }
            }
        if (!tma::grid_sync(bd.bar, G, bd.pd.err, sflag, lim)) return;
        // F
        for (int j = 0; j < cap_f; ++j) {
            const int k = sf[j];
            if (k < 0) break;
            const int md = smode[k];
            if (md == kBDone) continue;
            fix_item<T>(c, int(blockIdx.x + uint32_t(j) * G), md);
        }
        if (!tma::grid_sync(bd.bar, G, bd.pd.err, sflag, lim)) return;
        // U
        for (int j = 0; j < cap_t; ++j) {
            const int k = stl[j];
            if (k < 0) break;
            const int md = smode[k];
            if (md == kBDone) continue;
            update_item<T>(c, int(blockIdx.x + uint32_t(j) * G), md);
        }
        if (!tma::grid_sync(bd.bar, G, bd.pd.err, sflag, lim)) return;
        refresh();
        // D
        for (int j = 0; j < cap_t; ++j) {
            const int k = stl[j];
            if (k < 0) break;
            if (smode[k] != kBNormal) continue;
            direction_item<T>(c, int(blockIdx.x + uint32_t(j) * G));
        }
        if (blockIdx.x == 0 && tid == 0) *bd.loops += 1;
        if (!tma::grid_sync(bd.bar, G, bd.pd.err, sflag, lim)) return;
    }
}

__global__ void k_batch_init(BatchProblem* prob, int n_prob, uint32_t* ctr, uint32_t* bar, int32_t* live,
                             int64_t* loops) {
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
    }
}

int caps(const BatchDev& bd, int grid, int* cp, int* cf, int* ct) {
    *cp = (bd.pd.n_patches + grid - 1) / grid;
    *cf = (bd.n_fix + grid - 1) / grid;
    *ct = (bd.n_tile + grid - 1) / grid;
    return 0;
}

template <typename T, int NB>
int smem_for(const BatchDev& bd, int grid) {
    int cp, cf, ct;
    caps(bd, grid, &cp, &cf, &ct);
    return int(batch_layout<T, NB>(bd.pd.max_nodes, bd.n_prob, cp, cf, ct).total);
}

template <typename T, int NB>
int max_ctas(const BatchDev& bd, int* smem_bytes) {
    auto kern = k_batch_pcg<T, NB>;
    int best = 0;
    for (int c = 1; c <= 8; ++c) {
        const int sm = smem_for<T, NB>(bd, c * bd.pd.num_sms);
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
    int cp, cf, ct;
    caps(bd, grid, &cp, &cf, &ct);
    const int sm = smem_for<T, NB>(bd, grid);
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
    return cudaLaunchKernelEx(&cfg, kern, bd, cp, cf, ct);
}

}  // namespace

cudaError_t launch_batch_init(const BatchDev& bd, cudaStream_t st, int* launches) {
    const int nt = 256;
    k_batch_init<<<(bd.n_prob + nt - 1) / nt, nt, 0, st>>>(bd.prob, bd.n_prob, bd.ctr, bd.bar, bd.live, bd.loops);
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
