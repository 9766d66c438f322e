// Mixed-precision Jacobi-PCG of a small mesh in one CTA (sm_103a).
//
// A mesh of a few patches leaves the grid-wide solver latency-bound: each
// iteration is two or four launches whose CTAs mostly wait (33^2 triangles:
// about 29 us per iteration).  Here one CTA of 1024 threads runs the whole
// solve, with every node vector in shared memory and block barriers in place
// of launches.  The arithmetic is the textbook mixed form of the library
// (EBE_PREC_MIXED_TEXTBOOK): the FP32 difference-form operator on the FP32
// direction, FP32 recurrence residual, FP64 solution, and the FP64 true
// residual b - A x (FP64 element matrices) at every replacement and for the
// stopping test.  The elements are taken in the order of a colouring of the
// whole mesh (no two elements of a colour share a node).  The FP64 true
// residual adds each element's products into the node sums in one round per
// colour; the FP32 operator of every iteration instead has each node's thread
// gather its element rows in that same order (no barrier per colour).  The
// decisions (alpha, beta, replacement, convergence, stall, breakdown, maxit)
// follow the host loop of the grid-wide solver, taken by thread 0.  Every sum
// has a fixed order: bitwise reproducible.
#include <cstdint>

#include "device_util.cuh"
#include "kernels.h"

namespace ebe {
namespace {

constexpr int NT = kPatch;   // one thread per slot of a patch

struct SmallSmem {
    uint32_t red, cols, x, acc64, r, p, acc, dinv, lid, incp, inc, a32, total;
};
// Node vectors, then the elements' node ids (16-bit, the caller's numbering)
// and FP32 matrices in the order of a colouring of the whole mesh, copied
// once: an iteration then reads only shared memory.
__host__ __device__ constexpr SmallSmem small_layout(int64_t n_n, int64_t n_e, int nb, bool gather) {
    SmallSmem s{};
    const uint32_t n = uint32_t((n_n + 3) / 4 * 4);
    const uint32_t ne = uint32_t((n_e + 3) / 4 * 4);
    s.red = 0;                                   // block-reduction scratch, 2 x 32 doubles
    s.cols = 64 * 8;                             // colour classes: kSmallMaxColours + 1 offsets
    s.x = s.cols + 80 * 4;                       // FP64 solution
    s.acc64 = s.x + n * 8;                       // FP64 node sums / true residual
    s.r = s.acc64 + n * 8;                       // FP32 recurrence residual
    s.p = s.r + n * 4;                           // FP32 direction
    s.acc = s.p + n * 4;                         // FP32 node sums / q = A p
    s.dinv = s.acc + n * 4;                      // FP32 inverse Jacobi diagonal (0: Dirichlet)
    s.lid = s.dinv + n * 4;                      // [nb][n_e] uint16 node ids, colour order
    s.incp = s.lid + uint32_t(nb) * ne * 2;      // gather form: [n_n + 1] uint16 incidence offsets
    s.inc = (s.incp + (gather ? (uint32_t(n_n) + 1) * 2 : 0u) + 3) / 4 * 4;   // [nb * n_e] uint16 incidences
    s.a32 = (s.inc + (gather ? uint32_t(nb) * ne * 2 : 0u) + 15) / 16 * 16;   // [nb(nb+1)/2][n_e] FP32, colour order
    s.total = s.a32 + uint32_t(nb * (nb + 1) / 2) * ne * 4;
    return s;
}

constexpr int kSmallEPT = 4;   // elements per thread: at most 4 * 1024 elements

// Two compensated FP32 sums over the block, totals in FP64 valid in thread 0
// (the caller broadcasts what it derives from them): warp butterflies, then
// warp 0 adds the 32 warp totals with another butterfly, all in FP32; one
// FP64 conversion at the end.
__device__ __forceinline__ void block_sums2(CompSum a, CompSum b, double& ta, double& tb, double* red) {
    static_assert(NT == 1024, "32 warps");
    warp_sum(a);
    warp_sum(b);
    float2* red2 = reinterpret_cast<float2*>(red);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        red2[w] = make_float2(a.s, a.c);
        red2[32 + w] = make_float2(b.s, b.c);
    }
    __syncthreads();
    ta = tb = 0.0;
    if (w == 0) {
        CompSum x = comp_of(red2[lane]), y = comp_of(red2[32 + lane]);
        warp_sum(x);
        warp_sum(y);
        ta = x.value();
        tb = y.value();
    }
}

// One FP64 sum over the block, valid in thread 0.
__device__ __forceinline__ double block_sum64(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = red[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

// acc = sum over the elements of A_e p_e at the nodes (FP32 difference-form
// matrices in shared memory): products of a thread's elements first, then one
// round per colour of the whole mesh (a colour's elements share no node).
// Ends synchronised.
template <int NB>
__device__ __forceinline__ void operator32(const float* __restrict__ a32, const float* __restrict__ v,
                                           float* __restrict__ acc, int64_t n_n, const uint16_t* __restrict__ lid,
                                           int n_e, const int* __restrict__ cols, int n_col) {
    const int tid = threadIdx.x;
    for (int64_t i = tid; i < n_n; i += NT) acc[i] = 0.0f;
    int g[kSmallEPT][NB];
    float y[kSmallEPT][NB];
#pragma unroll
    for (int j = 0; j < kSmallEPT; ++j) {
        const int k = tid + j * NT;
        const bool ok = k < n_e;
        float ve[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            g[j][i] = ok ? int(lid[i * n_e + k]) : 0;
            ve[i] = ok ? v[g[j][i]] : 0.0f;
        }
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            // difference form: the diagonal slot holds the row sum
            float a = ok ? a32[sym_index(NB, r, r) * n_e + k] * ve[r] : 0.0f;
#pragma unroll
            for (int jj = 0; jj < NB; ++jj)
                if (jj != r) a = ok ? fmadd(a32[sym_index(NB, r, jj) * n_e + k], ve[jj] - ve[r], a) : a;
            y[j][r] = a;
        }
    }
    __syncthreads();
    for (int c = 0; c < n_col; ++c) {
        const int lo = cols[c], hi = cols[c + 1];
#pragma unroll
        for (int j = 0; j < kSmallEPT; ++j) {
            const int k = tid + j * NT;
            if (k >= lo && k < hi) {
#pragma unroll
                for (int r = 0; r < NB; ++r) acc[g[j][r]] += y[j][r];
            }
        }
        __syncthreads();
    }
}

// Node v's entry of sum_e A_e p_e (FP32 difference-form matrices in shared
// memory), gathered by v's own thread from its (element, row) incidences: each
// row as the element-wise form computes it (the diagonal slot holds the row
// sum: y = s_r p_r + sum_{j != r} a_rj (p_j - p_r)), added from 0 in the
// colour order of the elements, the order of colour rounds over the whole
// mesh, without the rounds' block barriers.
template <int NB>
__device__ __forceinline__ float gather_row_sums(const float* __restrict__ a32, const float* __restrict__ p,
                                                 const uint16_t* __restrict__ lid, int n_e,
                                                 const uint16_t* __restrict__ incp, const uint16_t* __restrict__ inc,
                                                 int v, float pv) {
    float acc = 0.0f;
    const int t1 = incp[v + 1];
#pragma unroll 2
    for (int t = incp[v]; t < t1; ++t) {
        const uint32_t e = inc[t];
        const int k = int(e & 0xfffu), r = int(e >> 12);
        float pe[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) pe[i] = p[lid[i * n_e + k]];
        float y = a32[sym_index(NB, r, r) * n_e + k] * pv;   // p_r = p_v
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (j != r) y = fmadd(a32[sym_index(NB, r, j) * n_e + k], pe[j] - pv, y);
        acc += y;
    }
    return acc;
}

// acc64 = sum over the elements of A_e x_e (FP64 matrices from global memory,
// element k of the colour order is slot order[k]), the products formed in
// each colour's round (few registers: this runs once per replacement).
template <int NB>
__device__ __forceinline__ void operator64(const double* __restrict__ A64, int64_t n_slots,
                                           const int32_t* __restrict__ order, const double* __restrict__ x,
                                           double* __restrict__ acc, int64_t n_n, const uint16_t* __restrict__ lid,
                                           int n_e, const int* __restrict__ cols, int n_col) {
    const int tid = threadIdx.x;
    for (int64_t i = tid; i < n_n; i += NT) acc[i] = 0.0;
    __syncthreads();
    for (int c = 0; c < n_col; ++c) {
        for (int k = cols[c] + tid; k < cols[c + 1]; k += NT) {
            const int64_t s = __ldg(order + k);
            int g[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) g[i] = int(lid[i * n_e + k]);
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                double a = acc[g[r]];
#pragma unroll
                for (int j = 0; j < NB; ++j) a = fmadd(__ldg(A64 + sym_index(NB, r, j) * n_slots + s), x[g[j]], a);
                acc[g[r]] = a;
            }
        }
        __syncthreads();
    }
}

template <int NB>
__global__ void __launch_bounds__(NT, 1)
k_cg_small(const PlanDev pd, int64_t n_n, const float* __restrict__ A32, const double* __restrict__ A64,
           const double* __restrict__ b, const float* __restrict__ dinv_g, double* __restrict__ x_g,
           SmallColouring sc, SmallOpts o, SmallInfo* __restrict__ info) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n_e = sc.n_e, n_col = sc.n_col;
    const bool gather = sc.gather != 0;
    const SmallSmem L = small_layout(n_n, n_e, NB, gather);
    int* cols = reinterpret_cast<int*>(smem + L.cols);
    double* red = reinterpret_cast<double*>(smem + L.red);
    double* x = reinterpret_cast<double*>(smem + L.x);
    double* acc64 = reinterpret_cast<double*>(smem + L.acc64);
    float* r = reinterpret_cast<float*>(smem + L.r);
    float* p = reinterpret_cast<float*>(smem + L.p);
    float* acc = reinterpret_cast<float*>(smem + L.acc);
    float* dinv = reinterpret_cast<float*>(smem + L.dinv);
    uint16_t* lid = reinterpret_cast<uint16_t*>(smem + L.lid);
    uint16_t* incp = reinterpret_cast<uint16_t*>(smem + L.incp);
    uint16_t* inc = reinterpret_cast<uint16_t*>(smem + L.inc);
    float* a32 = reinterpret_cast<float*>(smem + L.a32);
    const int tid = threadIdx.x;
    // Thread 0 forms the iteration's scalars and takes its decisions (GB300's
    // FP64 pipe issues two lanes per SM and clock: a division or square root
    // in every thread would cost more than the iteration's vector work) and
    // hands them to the block through shared memory.
    struct Ctl {
        double rho, beta, al, r0, rel, fin, thr, thr2, best, rrt;
        int64_t iters;
        int32_t n_true, status, reason, no_progress, init_dir, pad;
    };
    __shared__ Ctl C;

    for (int64_t i = tid; i < n_n; i += NT) {
        x[i] = x_g[i];
        dinv[i] = dinv_g[i];
    }
    {
        const int64_t ns = pd.n_slots;
        for (int k = tid; k < n_e; k += NT) {
            const int64_t s = __ldg(sc.order + k);
#pragma unroll
            for (int i = 0; i < NB; ++i) lid[i * n_e + k] = uint16_t(__ldg(sc.gconn + i * ns + s));
#pragma unroll
            for (int t = 0; t < sym_count(NB); ++t) a32[t * n_e + k] = __ldg(A32 + t * ns + s);
        }
        for (int c = tid; c <= n_col; c += NT) cols[c] = __ldg(sc.col + c);
        if (gather) {
            for (int64_t v = tid; v <= n_n; v += NT) incp[v] = __ldg(sc.inc_ptr + v);
            for (int t = tid; t < NB * n_e; t += NT) inc[t] = __ldg(sc.inc + t);
        }
    }
    if (tid == 0) {
        C.rho = C.beta = 0.0;
        C.iters = 0;
        C.n_true = 0;
        C.status = EBE_OK;
        C.init_dir = 1;
    }
    __syncthreads();

    // r64 = mask(b - A64 x) into acc64; its r.r in thread 0
    auto true_residual = [&]() -> double {
        operator64<NB>(A64, pd.n_slots, sc.order, x, acc64, n_n, lid, n_e, cols, n_col);
        double rr = 0.0;
        for (int64_t i = tid; i < n_n; i += NT) {
            const double v = dinv[i] == 0.0f ? 0.0 : __ldg(b + i) - acc64[i];
            acc64[i] = v;
            rr = fmadd(v, v, rr);
        }
        return block_sum64(rr, red);
    };
    // the recurrence restarted from the true residual in acc64: r = fp32(r64);
    // beta = r.z / rho (0 at the start), rho = r.z
    auto restart = [&](bool init) {
        CompSum rz, rr;
        for (int64_t i = tid; i < n_n; i += NT) {
            const float rf = d2f(acc64[i]);
            r[i] = rf;
            rz.add(rf * (dinv[i] * rf));
            rr.add(rf * rf);
        }
        double trz, trr;
        block_sums2(rz, rr, trz, trr, red);
        if (tid == 0) {
            C.beta = (init || !(C.rho != 0.0)) ? 0.0 : trz / C.rho;
            C.rho = trz;
            C.init_dir = init ? 1 : 0;
        }
        __syncthreads();
    };
    // p = z + beta p (p = z at the start)
    auto direction = [&]() {
        const float be = float(C.beta);
        const bool init = C.init_dir != 0;
        for (int64_t i = tid; i < n_n; i += NT) {
            const float z = dinv[i] * r[i];
            p[i] = init ? z : fmaf(be, p[i], z);
        }
        __syncthreads();
        if (tid == 0) C.init_dir = 0;
    };

    {
        const double rr0 = true_residual();
        if (tid == 0) {
            C.n_true = 1;
            C.r0 = sqrt(rr0);
            C.rel = C.r0 > 0.0 ? 1.0 : 0.0;
            C.status = isfinite(C.r0) ? EBE_OK : EBE_BREAKDOWN;
            C.fin = o.rtol * C.r0;
            C.best = 1.0;
            C.thr = fmax(o.delta * C.r0, C.fin);
            C.thr2 = C.thr * C.thr;
            C.no_progress = 0;
            C.reason = kRunning;
        }
        __syncthreads();
    }
    if (C.r0 > 0.0 && isfinite(C.r0)) {
        restart(true);
        direction();
        for (;;) {
            if (C.reason == kRunning) {
                // one CG iteration: q = mask(A p), alpha, x and r updated, r.z and r.r;
                // a node's q stays with its thread (no barrier before the update)
                CompSum pq, none;
                if (gather) {
                    for (int64_t i = tid; i < n_n; i += NT) {
                        const float pv = p[i];
                        const float qv =
                            dinv[i] == 0.0f ? 0.0f : gather_row_sums<NB>(a32, p, lid, n_e, incp, inc, int(i), pv);
                        acc[i] = qv;
                        pq.add(pv * qv);
                    }
                } else {
                    operator32<NB>(a32, p, acc, n_n, lid, n_e, cols, n_col);
                    for (int64_t i = tid; i < n_n; i += NT) {
                        const float qv = dinv[i] == 0.0f ? 0.0f : acc[i];
                        acc[i] = qv;
                        pq.add(p[i] * qv);
                    }
                }
                double tpq, tnone;
                block_sums2(pq, none, tpq, tnone, red);
                if (tid == 0) {
                    if (!(tpq > 0.0) || !isfinite(tpq)) C.reason = kBreakdown;
                    else C.al = C.rho / tpq;
                }
                __syncthreads();
                if (C.reason != kRunning) continue;
                const double al = C.al;
                const float alf = d2f(al);
                CompSum rz, rr;
                for (int64_t i = tid; i < n_n; i += NT) {
                    x[i] = fmadd(al, f2d(p[i]), x[i]);
                    const float rf = fmaf(-alf, acc[i], r[i]);
                    r[i] = rf;
                    rz.add(rf * (dinv[i] * rf));
                    rr.add(rf * rf);
                }
                double trz, trr;
                block_sums2(rz, rr, trz, trr, red);
                if (tid == 0) {
                    C.iters += 1;
                    if (!isfinite(trz) || !isfinite(trr) || trz < 0.0) C.reason = kBreakdown;
                    else if (trr <= C.thr2) C.reason = kTrigger;       // rho stays for the replacement
                    else if (C.iters >= o.maxit) C.reason = kMaxit;
                    else {
                        C.beta = trz / C.rho;
                        C.rho = trz;
                    }
                }
                __syncthreads();
                if (C.reason == kRunning) direction();
                continue;
            }
            if (C.reason == kBreakdown) {
                if (tid == 0) C.status = EBE_BREAKDOWN;
                break;
            }
            const double rrt = true_residual();
            // thread 0: the checks of the grid-wide solver's host loop
            if (tid == 0) {
                C.n_true += 1;
                C.rrt = rrt;
                const double rel = sqrt(rrt) / C.r0;
                C.rel = rel;
                int st = -1;
                if (!isfinite(rel)) st = EBE_BREAKDOWN;
                else if (rel <= o.rtol) st = EBE_OK;
                else if (C.reason == kMaxit) st = EBE_MAXIT;
                else if (rel < 0.9 * C.best) { C.best = rel; C.no_progress = 0; }
                else if (++C.no_progress >= o.stall_updates) st = EBE_STALL;
                if (st >= 0) {
                    C.status = st;
                    C.reason = -1;          // done
                } else {
                    // a failed check at the final threshold tightens it (the FP32
                    // recurrence drifted below the true residual)
                    if (C.reason == kTrigger && C.thr <= C.fin) C.fin *= kFinalMargin;
                    C.thr = fmax(o.delta * sqrt(rrt), C.fin);
                    C.thr2 = C.thr * C.thr;
                }
            }
            __syncthreads();
            if (C.reason == -1) break;
            // residual replacement: continue CG from the true residual, same direction
            restart(false);
            direction();
            if (tid == 0) C.reason = kRunning;
            __syncthreads();
        }
        __syncthreads();   // the status thread 0 set before the loop ended
        if (C.status == EBE_BREAKDOWN) {
            const double rrt = true_residual();
            if (tid == 0) C.rel = sqrt(rrt) / C.r0;
        }
    }
    __syncthreads();
    for (int64_t i = tid; i < n_n; i += NT) x_g[i] = x[i];
    if (tid == 0) {
        info->iterations = C.iters;
        info->true_residuals = C.n_true;
        info->status = C.status;
        info->r0 = C.r0;
        info->rel = C.rel;
    }
}

}  // namespace

size_t small_solver_smem(int64_t n_n, int64_t n_e, int nb) {
    return (n_n > 65536 || n_e > int64_t(kSmallEPT) * NT) ? size_t(1) << 40 : small_layout(n_n, n_e, nb, false).total;
}

bool small_solver_gather(int64_t n_n, int64_t n_e, int nb) {
    return n_n <= kSmallGatherNodes && n_e <= int64_t(kSmallEPT) * NT &&
           small_layout(n_n, n_e, nb, true).total <= size_t(kSmallGatherSmem);
}

cudaError_t launch_cg_small(const PlanDev& pd, int64_t n_n, const float* A32, const double* A64, const double* b,
                            const float* dinv, double* x, const SmallColouring& sc, const SmallOpts& o,
                            SmallInfo* info, cudaStream_t st, int* launches) {
    if (sc.gather && (sc.inc_ptr == nullptr || sc.inc == nullptr)) return cudaErrorInvalidValue;
    const size_t base = small_solver_smem(n_n, sc.n_e, pd.nb);   // 2^40 beyond the solver's limits
    const size_t sm = (base >> 40) ? base : small_layout(n_n, sc.n_e, pd.nb, sc.gather != 0).total;
    if (sm > 227 * 1024 || sc.n_col < 1 || sc.n_col > kSmallMaxColours) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    if (pd.nb == 3) {
        e = cudaFuncSetAttribute(k_cg_small<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
        k_cg_small<3><<<1, NT, sm, st>>>(pd, n_n, A32, A64, b, dinv, x, sc, o, info);
    } else {
        e = cudaFuncSetAttribute(k_cg_small<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
        k_cg_small<4><<<1, NT, sm, st>>>(pd, n_n, A32, A64, b, dinv, x, sc, o, info);
    }
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace ebe
