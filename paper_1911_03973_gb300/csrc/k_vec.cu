// Node-vector kernels of the Jacobi-PCG iteration (sm_103a).
//
// All dot products are accumulated in FP64 whatever the vector type, per
// thread in a fixed index order, then over the block by fixed-pattern warp
// butterflies, then over a fixed grid by the last block to arrive, which adds
// the per-block partials in index order.  The results are therefore bitwise
// reproducible for a given problem size.  The last block also takes the
// iteration's scalar decisions (alpha, beta, stop) so that the host never has
// to read anything inside a graph chunk.
#include <cstdint>

#include "kernels.h"

namespace ebe {
namespace {

constexpr int NT = kVecThreads;

__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }

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

// Publish (a, b) for this block; returns true in every thread of the last
// block, which then holds the grid totals in (a, b) (thread 0).
__device__ __forceinline__ bool grid_sum2(double& a, double& b, double* part, uint32_t* ctr, double* red) {
    __shared__ bool last;
    block_sum2(a, b, red);
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

// x += alpha p;  r -= alpha q;  z = dinv r;  sums r.z, r.r.
// TX: type of x, r, dinv (the recurrences); TP: type of p, q (the direction
// and its product, which the operator pass reads and writes).
// Last block: iteration count, stop tests, beta = r.z / rho, rho = r.z.
template <typename TX, typename TP>
__global__ void __launch_bounds__(NT)
k_update(int64_t n, TX* __restrict__ x, const TP* __restrict__ p, TX* __restrict__ r, const TP* __restrict__ q,
         const TX* __restrict__ dinv, double* __restrict__ part, Scalars* __restrict__ sc) {
    __shared__ double red[64];
    if (sc->done) return;
    const TX al = TX(sc->alpha);
    double rz = 0.0, rr = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) {
        x[i] = fmadd(al, TX(p[i]), x[i]);
        const TX ri = fmadd(-al, TX(q[i]), r[i]);
        r[i] = ri;
        const TX zi = dinv[i] * ri;
        rz = fmadd(double(ri), double(zi), rz);
        rr = fmadd(double(ri), double(ri), rr);
    }
    if (grid_sum2(rz, rr, part, &sc->ctr_vec, red) && threadIdx.x == 0) {
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
}

// p = dinv r + beta p   (init: p = dinv r), evaluated in TX, stored as TP.
template <typename TX, typename TP>
__global__ void __launch_bounds__(NT)
k_direction(int64_t n, TP* __restrict__ p, const TX* __restrict__ r, const TX* __restrict__ dinv, int init,
            const Scalars* __restrict__ sc) {
    if (sc->done) return;
    const TX be = init ? TX(0) : TX(sc->beta);
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) {
        const TX zi = dinv[i] * r[i];
        p[i] = TP(init ? zi : fmadd(be, TX(p[i]), zi));
    }
}

// After a true-residual replacement: sums r.z, r.r; beta = r.z / rho,
// rho = r.z (init: rho = r.z, beta = 0).
__global__ void __launch_bounds__(NT)
k_restart(int64_t n, const double* __restrict__ r, const double* __restrict__ dinv, int init,
          double* __restrict__ part, Scalars* __restrict__ sc) {
    __shared__ double red[64];
    double rz = 0.0, rr = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) {
        const double ri = r[i];
        const double zi = dinv[i] * ri;
        rz = fmadd(ri, zi, rz);
        rr = fmadd(ri, ri, rr);
    }
    if (grid_sum2(rz, rr, part, &sc->ctr_vec, red) && threadIdx.x == 0) {
        sc->rz = rz;
        sc->rr = rr;
        if (init || !(sc->rho != 0.0)) sc->beta = 0.0;
        else sc->beta = rz / sc->rho;
        sc->rho = rz;
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

cudaError_t launch_control(Scalars* sc, double thr2, int64_t maxit, int reset_iter, cudaStream_t st, int* launches) {
    k_control<<<1, 32, 0, st>>>(sc, thr2, maxit, reset_iter);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

int vec_grid(int64_t n) {
    int64_t g = (n + NT - 1) / NT;
    return int(g < 1 ? 1 : (g > 1216 ? 1216 : g));
}

// vt: 0 = all FP64; 1 = x, r, dinv FP64 with p, q FP32.
cudaError_t launch_update(int vt, int64_t n, void* x, const void* p, void* r, const void* q, const void* dinv,
                          double* part, Scalars* sc, cudaStream_t st, int* launches) {
    if (vt == 0)
        k_update<double, double><<<vec_grid(n), NT, 0, st>>>(n, static_cast<double*>(x), static_cast<const double*>(p),
                                                             static_cast<double*>(r), static_cast<const double*>(q),
                                                             static_cast<const double*>(dinv), part, sc);
    else
        k_update<double, float><<<vec_grid(n), NT, 0, st>>>(n, static_cast<double*>(x), static_cast<const float*>(p),
                                                            static_cast<double*>(r), static_cast<const float*>(q),
                                                            static_cast<const double*>(dinv), part, sc);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_direction(int vt, int64_t n, void* p, const void* r, const void* dinv, int init, Scalars* sc,
                             cudaStream_t st, int* launches) {
    if (vt == 0)
        k_direction<double, double><<<vec_grid(n), NT, 0, st>>>(n, static_cast<double*>(p), static_cast<const double*>(r),
                                                                static_cast<const double*>(dinv), init, sc);
    else
        k_direction<double, float><<<vec_grid(n), NT, 0, st>>>(n, static_cast<float*>(p), static_cast<const double*>(r),
                                                               static_cast<const double*>(dinv), init, sc);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_restart(int64_t n, const double* r, const double* dinv, int init, double* part, Scalars* sc,
                           cudaStream_t st, int* launches) {
    k_restart<<<vec_grid(n), NT, 0, st>>>(n, r, dinv, init, part, sc);
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

}  // namespace ebe
