// Node-vector kernels of the Jacobi-PCG iteration and of the paper's
// stationary iterations (sm_103a).
//
// All dot products end in FP64: per thread in a fixed index order, then over
// the block by fixed-pattern warp butterflies, then over a fixed grid by the
// last block to arrive, which adds the per-block partials in index order.  The
// results are therefore bitwise reproducible for a given problem size.  The
// last block also takes the iteration's scalar decisions (beta, stop) so that
// the host never reads anything inside a graph chunk.
//
// GB300 runs FP64 at 1/64 of the FP32 rate (two FP64 operations per SM and
// clock), so the mixed-precision kernels keep only the solution x in FP64:
// FP32 rounding of x would reach the residual amplified by the condition
// number.  The recurrence residual r, z = dinv r, the direction p and q = A p
// are FP32 (r's own rounding drift is not amplified and is removed at every
// replacement by the FP64 true residual); the per-thread dot sums use
// compensated FP32 (Neumaier) before the FP64 block reduction.
#include <atomic>
#include <cstdint>
#include <tuple>

#include "device_util.cuh"
#include "kernels.h"

namespace ebe {
namespace {

constexpr int NT = kVecThreads;

__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) { red[w] = a; red[32 + w] = b; }
    __syncthreads();
    if (w == 0) {
        a = lane < NT / 32 ? red[lane] : 0.0;
        b = lane < NT / 32 ? red[32 + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
    }
}

// Publish the block totals (a, b) (valid in thread 0); returns true in every
// thread of the last block, which then holds the grid totals in (a, b)
// (thread 0).
__device__ __forceinline__ bool grid_publish2(double& a, double& b, double* part, uint32_t* ctr, double* red) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
        __threadfence();
        last = atomicAdd(ctr, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    a = 0.0;
    b = 0.0;
    for (int i = threadIdx.x; i < int(gridDim.x); i += NT) {
        a += __ldcg(part + 2 * i);
        b += __ldcg(part + 2 * i + 1);
    }
    block_sum2(a, b, red);
    if (threadIdx.x == 0) *ctr = 0;
    return true;
}

// Block sums of per-thread (a, b), then grid_publish2.
__device__ __forceinline__ bool grid_sum2(double& a, double& b, double* part, uint32_t* ctr, double* red) {
    block_sum2(a, b, red);
    return grid_publish2(a, b, part, ctr, red);
}

// The same for compensated FP32 per-thread sums: block totals by FP32
// butterflies (one FP64 conversion per warp), then grid_publish2.
__device__ __forceinline__ bool grid_sum2(CompSum a, CompSum b, double& ta, double& tb, double* part, uint32_t* ctr,
                                          double* red) {
    CompSum v[2] = {a, b};
    double t[2];
    block_sums_comp<2, NT>(v, t, red);
    ta = t[0];
    tb = t[1];
    return grid_publish2(ta, tb, part, ctr, red);
}

// Stop tests and beta of one CG iteration (last block, thread 0).
__device__ __forceinline__ void decide(Scalars* sc, double rz, double rr) {
    sc->iter += 1;
    sc->rz = rz;
    sc->rr = rr;
    if (!isfinite(rz) || !isfinite(rr) || rz < 0.0) {
        sc->done = 1;
        sc->reason = kBreakdown;
    } else if (rr <= sc->thr2) {
        sc->done = 1;            // rho stays: the host recomputes r.z after the replacement
        sc->reason = kTrigger;
    } else if (sc->iter >= sc->maxit) {
        sc->done = 1;
        sc->reason = kMaxit;
    } else {
        sc->beta = rz / sc->rho;
        sc->rho = rz;
    }
}

// ------------------------------------------------------------------ FP64
// The update and direction kernels contain pdl_trigger / pdl_wait
// (programmatic dependent launch; no-ops unless launched with it).

// Four consecutive nodes per vector access (16-byte loads and stores: float4,
// or two double2); every array is a library buffer (cudaMalloc, 256-byte
// aligned), grid-stride over the groups (the direction kernels take two
// groups per step); the n mod 4 tail nodes go one per thread.  Per-thread
// sums run in node order.
struct D4 {
    double v[4];
};
__device__ __forceinline__ D4 ld4(const double* p, int64_t g) {
    const double2 a = reinterpret_cast<const double2*>(p)[2 * g], b = reinterpret_cast<const double2*>(p)[2 * g + 1];
    return D4{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(double* p, int64_t g, const D4& d) {
    reinterpret_cast<double2*>(p)[2 * g] = make_double2(d.v[0], d.v[1]);
    reinterpret_cast<double2*>(p)[2 * g + 1] = make_double2(d.v[2], d.v[3]);
}
__device__ __forceinline__ float4 ldf4(const float* p, int64_t g) { return reinterpret_cast<const float4*>(p)[g]; }
__device__ __forceinline__ float at(const float4& f, int u) { return u == 0 ? f.x : u == 1 ? f.y : u == 2 ? f.z : f.w; }

// x += alpha p;  r -= alpha q;  z = dinv r;  sums r.z, r.r (all FP64).
__global__ void __launch_bounds__(NT, 4)
k_update64(int64_t n, double* __restrict__ x, const double* __restrict__ p, double* __restrict__ r,
           const double* __restrict__ q, const double* __restrict__ dinv, double* __restrict__ part,
           Scalars* __restrict__ sc) {
    __shared__ double red[64];
    pdl_trigger();
    pdl_wait();
    if (sc->done) return;
    const double al = sc->alpha;
    double rz = 0.0, rr = 0.0;
    const int64_t st = int64_t(gridDim.x) * NT, n4 = n >> 2;
    for (int64_t g = int64_t(blockIdx.x) * NT + threadIdx.x; g < n4; g += st) {
        const D4 pv = ld4(p, g), qv = ld4(q, g), xv = ld4(x, g), rv = ld4(r, g), dv = ld4(dinv, g);
        D4 xo, ro;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            xo.v[u] = fmadd(al, pv.v[u], xv.v[u]);
            const double ri = fmadd(-al, qv.v[u], rv.v[u]);
            ro.v[u] = ri;
            rz = fmadd(ri, dv.v[u] * ri, rz);
            rr = fmadd(ri, ri, rr);
        }
        st4(x, g, xo);
        st4(r, g, ro);
    }
    for (int64_t i = 4 * n4 + int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += st) {
        x[i] = fmadd(al, p[i], x[i]);
        const double ri = fmadd(-al, q[i], r[i]);
        r[i] = ri;
        rz = fmadd(ri, dinv[i] * ri, rz);
        rr = fmadd(ri, ri, rr);
    }
    if (grid_sum2(rz, rr, part, &sc->ctr_vec, red) && threadIdx.x == 0) decide(sc, rz, rr);
}

// p = dinv r + beta p  (init: p = dinv r), FP64.
__global__ void __launch_bounds__(NT, 4)
k_direction64(int64_t n, double* __restrict__ p, const double* __restrict__ r, const double* __restrict__ dinv,
              int init, const Scalars* __restrict__ sc) {
    pdl_trigger();
    pdl_wait();
    if (sc->done) return;
    const double be = init ? 0.0 : sc->beta;
    const int64_t st = int64_t(gridDim.x) * NT, n4 = n >> 2;
    for (int64_t g = int64_t(blockIdx.x) * NT + threadIdx.x; g < n4; g += 2 * st) {
        const bool two = g + st < n4;
        D4 rv[2], dv[2], pv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !two) break;
            const int64_t k = g + h * st;
            rv[h] = ld4(r, k); dv[h] = ld4(dinv, k);
            if (!init) pv[h] = ld4(p, k);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !two) break;
            D4 po;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double zi = dv[h].v[u] * rv[h].v[u];
                po.v[u] = init ? zi : fmadd(be, pv[h].v[u], zi);
            }
            st4(p, g + h * st, po);
        }
    }
    for (int64_t i = 4 * n4 + int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += st) {
        const double zi = dinv[i] * r[i];
        p[i] = init ? zi : fmadd(be, p[i], zi);
    }
}

// ------------------------------------------------------------------ mixed
// x += alpha p in FP64 (p FP32); r -= alpha q, z = dinv r in FP32; sums r.z,
// r.r per thread in compensated FP32.  Two FP64 operations per node (the
// widening of p and the FMA).
__global__ void __launch_bounds__(NT, 4)
k_update_mixed(int64_t n, double* __restrict__ x, const float* __restrict__ p, float* __restrict__ r,
               const float* __restrict__ q, const float* __restrict__ dinv, double* __restrict__ part,
               Scalars* __restrict__ sc) {
    __shared__ double red[64];
    pdl_trigger();
    pdl_wait();
    if (sc->done) return;
    const double al = sc->alpha;
    const float alf = d2f(al);
    CompSum rz, rr;
    const int64_t st = int64_t(gridDim.x) * NT, n4 = n >> 2;
    for (int64_t g = int64_t(blockIdx.x) * NT + threadIdx.x; g < n4; g += st) {
        const float4 pv = ldf4(p, g), qv = ldf4(q, g), dv = ldf4(dinv, g), rv = ldf4(r, g);
        const D4 xv = ld4(x, g);
        D4 xo;
        float ro[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            xo.v[u] = fmadd(al, f2d(at(pv, u)), xv.v[u]);
            const float rf = __fmaf_rn(-alf, at(qv, u), at(rv, u));
            ro[u] = rf;
            rz.add(rf * (at(dv, u) * rf));
            rr.add(rf * rf);
        }
        st4(x, g, xo);
        reinterpret_cast<float4*>(r)[g] = make_float4(ro[0], ro[1], ro[2], ro[3]);
    }
    for (int64_t i = 4 * n4 + int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += st) {
        x[i] = fmadd(al, f2d(p[i]), x[i]);
        const float rf = __fmaf_rn(-alf, q[i], r[i]);
        r[i] = rf;
        rz.add(rf * (dinv[i] * rf));
        rr.add(rf * rf);
    }
    double a = 0.0, b = 0.0;
    if (grid_sum2(rz, rr, a, b, part, &sc->ctr_vec, red) && threadIdx.x == 0) decide(sc, a, b);
}

// p = dinv r + beta p  (init: p = dinv r), FP32.
__global__ void __launch_bounds__(NT, 4)
k_direction_mixed(int64_t n, float* __restrict__ p, const float* __restrict__ r, const float* __restrict__ dinv,
                  int init, const Scalars* __restrict__ sc) {
    pdl_trigger();
    pdl_wait();
    if (sc->done) return;
    const float be = init ? 0.0f : d2f(sc->beta);
    const int64_t st = int64_t(gridDim.x) * NT, n4 = n >> 2;
    for (int64_t g = int64_t(blockIdx.x) * NT + threadIdx.x; g < n4; g += 2 * st) {
        const bool two = g + st < n4;
        float4 rv[2], dv[2], pv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !two) break;
            const int64_t k = g + h * st;
            rv[h] = ldf4(r, k); dv[h] = ldf4(dinv, k);
            pv[h] = init ? make_float4(0.f, 0.f, 0.f, 0.f) : ldf4(p, k);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !two) break;
            float o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float zi = at(dv[h], u) * at(rv[h], u);
                o[u] = init ? zi : __fmaf_rn(be, at(pv[h], u), zi);
            }
            reinterpret_cast<float4*>(p)[g + h * st] = make_float4(o[0], o[1], o[2], o[3]);
        }
    }
    for (int64_t i = 4 * n4 + int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += st) {
        const float zi = dinv[i] * r[i];
        p[i] = init ? zi : __fmaf_rn(be, p[i], zi);
    }
}

// After a true-residual replacement: sums r.z, r.r with z as the update
// kernel of the same precision forms it; beta = r.z / rho, rho = r.z
// (init: rho = r.z, beta = 0).  Mixed: also r32 = (float) r, the start of
// the FP32 recurrence residual.
template <bool MIXED>
__global__ void __launch_bounds__(NT)
k_restart(int64_t n, const double* __restrict__ r, const void* __restrict__ dinv_v, int init,
          double* __restrict__ part, Scalars* __restrict__ sc, float* __restrict__ r32) {
    __shared__ double red[64];
    double a = 0.0, b = 0.0;
    bool last;
    if (MIXED) {
        const float* dinv = static_cast<const float*>(dinv_v);
        CompSum rz, rr;
        for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) {
            const float rf = d2f(r[i]);
            if (r32 != nullptr) r32[i] = rf;
            rz.add(rf * (dinv[i] * rf));
            rr.add(rf * rf);
        }
        last = grid_sum2(rz, rr, a, b, part, &sc->ctr_vec, red);
    } else {
        const double* dinv = static_cast<const double*>(dinv_v);
        a = 0.0;
        b = 0.0;
        for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) {
            const double ri = r[i];
            a = fmadd(ri, dinv[i] * ri, a);
            b = fmadd(ri, ri, b);
        }
        last = grid_sum2(a, b, part, &sc->ctr_vec, red);
    }
    if (last && threadIdx.x == 0) {
        sc->rz = a;
        sc->rr = b;
        if (init || !(sc->rho != 0.0)) sc->beta = 0.0;
        else sc->beta = a / sc->rho;
        sc->rho = a;
        sc->done = 0;
        sc->reason = kRunning;
    }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_fill(int64_t n, T* __restrict__ v, T value) {
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) v[i] = value;
}

__global__ void __launch_bounds__(NT)
k_set_dirichlet(double* __restrict__ x, const int32_t* __restrict__ nd, const double* __restrict__ g, int64_t n_d) {
    for (int64_t k = int64_t(blockIdx.x) * NT + threadIdx.x; k < n_d; k += int64_t(gridDim.x) * NT)
        x[nd[k]] = g ? g[k] : 0.0;
}

// Stationary steps of Sec. 2.  kind 0: x += w r (Richardson, two-level
// Chebyshev with w = 1/alpha_k); kind 1: p = r + beta p, x += alpha p (the
// three-level Chebyshev iteration in its direction form; beta = 0 starts it).
__global__ void __launch_bounds__(NT)
k_stationary(int64_t n, double* __restrict__ x, const double* __restrict__ r, double* __restrict__ p, int kind,
             double w, double beta) {
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) {
        if (kind == 0) {
            x[i] = fmadd(w, r[i], x[i]);
        } else {
            const double pi = beta == 0.0 ? r[i] : fmadd(beta, p[i], r[i]);
            p[i] = pi;
            x[i] = fmadd(w, pi, x[i]);
        }
    }
}

// Host-chosen controls of a solve: stop threshold, iteration cap, counters.
__global__ void k_control(Scalars* sc, double thr2, int64_t maxit, int reset_iter) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (thr2 >= 0.0) sc->thr2 = thr2;
    if (maxit >= 0) sc->maxit = maxit;
    if (reset_iter) { sc->iter = 0; sc->ctr_fix = 0; sc->ctr_vec = 0; }
    sc->done = 0;
    sc->reason = kRunning;
}

}  // namespace

// One wave of CTAs: the update and direction kernels hold 64 registers per
// thread (4 CTAs of 256 threads per SM), and a second wave would only add a
// tail and more block partials.  Capped at the 1216 partials the reductions
// have room for.
int vec_grid(int64_t n) {
    constexpr int kDevices = 64;
    static std::atomic<int> caps[kDevices];   // per device, 0 = not yet queried
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    int cap = dev < kDevices ? caps[dev].load(std::memory_order_relaxed) : 0;
    if (cap == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
        cap = sms * 4 > 1216 ? 1216 : sms * 4;
        if (dev < kDevices) caps[dev].store(cap, std::memory_order_relaxed);
    }
    const int64_t g = (n + NT - 1) / NT;
    return int(g < 1 ? 1 : (g > cap ? cap : g));
}

cudaError_t launch_update(int vt, int64_t n, void* x, const void* p, void* r, const void* q, const void* dinv,
                          double* part, Scalars* sc, cudaStream_t st, int* launches, bool pdl) {
    cudaError_t e;
    if (vt == 0) {
        auto kern = k_update64;
        auto args = std::make_tuple(n, static_cast<double*>(x), static_cast<const double*>(p), static_cast<double*>(r),
                                    static_cast<const double*>(q), static_cast<const double*>(dinv), part, sc);
        e = pdl ? std::apply([&](auto... a) { return launch_pdl(kern, dim3(vec_grid(n)), dim3(NT), 0, st, a...); }, args)
                : (std::apply([&](auto... a) { kern<<<vec_grid(n), NT, 0, st>>>(a...); }, args), cudaGetLastError());
    } else {
        auto kern = k_update_mixed;
        auto args = std::make_tuple(n, static_cast<double*>(x), static_cast<const float*>(p), static_cast<float*>(r),
                                    static_cast<const float*>(q), static_cast<const float*>(dinv), part, sc);
        e = pdl ? std::apply([&](auto... a) { return launch_pdl(kern, dim3(vec_grid(n)), dim3(NT), 0, st, a...); }, args)
                : (std::apply([&](auto... a) { kern<<<vec_grid(n), NT, 0, st>>>(a...); }, args), cudaGetLastError());
    }
    if (launches) *launches += 1;
    return e;
}

cudaError_t launch_direction(int vt, int64_t n, void* p, const void* r, const void* dinv, int init, Scalars* sc,
                             cudaStream_t st, int* launches, bool pdl) {
    cudaError_t e;
    if (vt == 0) {
        auto kern = k_direction64;
        auto args = std::make_tuple(n, static_cast<double*>(p), static_cast<const double*>(r),
                                    static_cast<const double*>(dinv), init, static_cast<const Scalars*>(sc));
        e = pdl ? std::apply([&](auto... a) { return launch_pdl(kern, dim3(vec_grid(n)), dim3(NT), 0, st, a...); }, args)
                : (std::apply([&](auto... a) { kern<<<vec_grid(n), NT, 0, st>>>(a...); }, args), cudaGetLastError());
    } else {
        auto kern = k_direction_mixed;
        auto args = std::make_tuple(n, static_cast<float*>(p), static_cast<const float*>(r),
                                    static_cast<const float*>(dinv), init, static_cast<const Scalars*>(sc));
        e = pdl ? std::apply([&](auto... a) { return launch_pdl(kern, dim3(vec_grid(n)), dim3(NT), 0, st, a...); }, args)
                : (std::apply([&](auto... a) { kern<<<vec_grid(n), NT, 0, st>>>(a...); }, args), cudaGetLastError());
    }
    if (launches) *launches += 1;
    return e;
}

cudaError_t launch_restart(int vt, int64_t n, const double* r, const void* dinv, int init, double* part, Scalars* sc,
                           cudaStream_t st, int* launches, float* r32) {
    if (vt == 0) k_restart<false><<<vec_grid(n), NT, 0, st>>>(n, r, dinv, init, part, sc, nullptr);
    else k_restart<true><<<vec_grid(n), NT, 0, st>>>(n, r, dinv, init, part, sc, r32);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_control(Scalars* sc, double thr2, int64_t maxit, int reset_iter, cudaStream_t st, int* launches) {
    k_control<<<1, 32, 0, st>>>(sc, thr2, maxit, reset_iter);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_fill(int dtype, int64_t n, void* v, double value, cudaStream_t st, int* launches) {
    if (dtype == 0) k_fill<double><<<vec_grid(n), NT, 0, st>>>(n, static_cast<double*>(v), value);
    else k_fill<float><<<vec_grid(n), NT, 0, st>>>(n, static_cast<float*>(v), float(value));
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_set_dirichlet(double* x, const int32_t* nd, const double* g, int64_t n_d, cudaStream_t st,
                                 int* launches) {
    if (n_d <= 0) return cudaSuccess;
    k_set_dirichlet<<<vec_grid(n_d), NT, 0, st>>>(x, nd, g, n_d);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_stationary(int64_t n, double* x, const double* r, double* p, int kind, double w, double beta,
                              cudaStream_t st, int* launches) {
    k_stationary<<<vec_grid(n), NT, 0, st>>>(n, x, r, p, kind, w, beta);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace ebe
