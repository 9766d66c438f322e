// Comparison scatters of the FP64 residual r = mask(b - sum_e C_e^T A_e C_e x).
//
// They exist to measure the patch pass against the usual alternatives:
//   colour  - all elements greedily coloured; one pass per colour adds A_e x_e
//             into r with plain read-modify-write (deterministic);
//   node    - phase 1 writes A_e x_e per element to Y, phase 2 gathers, per
//             node, its entries of Y over the inverse connectivity in a fixed
//             order (deterministic);
//   atomic  - FP64 atomic adds into r (order and result vary run to run).
// Each reads the same element matrices as the patch pass (slot layout).
#include <cstdint>

#include "kernels.h"

namespace ebe {
namespace {

constexpr int NT = 256;

__global__ void k_build_gconn(const PlanDev pd, int32_t* __restrict__ gconn) {
    const int64_t s = int64_t(blockIdx.x) * NT + threadIdx.x;
    if (s >= pd.n_slots) return;
    const PatchMeta m = pd.meta[s / kPatch];
    const bool ok = pd.slot_elem[s] >= 0;
    for (int i = 0; i < pd.nb; ++i)
        gconn[i * pd.n_slots + s] = ok ? (pd.pnode[m.node_off + pd.lconn[i * pd.n_slots + s]] & kNodeMask) : 0;
}

__global__ void k_permute(int nb, int64_t n_slots, int64_t n, const int32_t* __restrict__ order,
                          const double* __restrict__ A, const int32_t* __restrict__ gconn, double* __restrict__ Ao,
                          int32_t* __restrict__ go) {
    const int64_t k = int64_t(blockIdx.x) * NT + threadIdx.x;
    if (k >= n) return;
    const int64_t s = order[k];
    for (int t = 0; t < sym_count(nb); ++t) Ao[t * n + k] = A[t * n_slots + s];
    for (int i = 0; i < nb; ++i) go[i * n + k] = gconn[i * n_slots + s];
}

template <int NB>
__global__ void k_colour_pass(int64_t lo, int64_t hi, int64_t n, const double* __restrict__ Ac,
                              const int32_t* __restrict__ gc, const double* __restrict__ x, double* __restrict__ r) {
    const int64_t k = lo + int64_t(blockIdx.x) * NT + threadIdx.x;
    if (k >= hi) return;
    int g[NB];
    double xe[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) { g[i] = gc[i * n + k]; xe[i] = __ldg(x + g[i]); }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        double v = r[g[i]];
#pragma unroll
        for (int j = 0; j < NB; ++j) v = __fma_rn(__ldcs(Ac + sym_index(NB, i, j) * n + k), xe[j], v);
        r[g[i]] = v;
    }
}

template <int NB>
__global__ void k_atomic_pass(const PlanDev pd, const double* __restrict__ A, const int32_t* __restrict__ gconn,
                              const double* __restrict__ x, double* __restrict__ r) {
    const int64_t s = int64_t(blockIdx.x) * NT + threadIdx.x;
    if (s >= pd.n_slots || pd.slot_elem[s] < 0) return;
    const int64_t ns = pd.n_slots;
    int g[NB];
    double xe[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) { g[i] = gconn[i * ns + s]; xe[i] = __ldg(x + g[i]); }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < NB; ++j) v = __fma_rn(__ldcs(A + sym_index(NB, i, j) * ns + s), xe[j], v);
        atomicAdd(r + g[i], v);
    }
}

template <int NB>
__global__ void k_element_products(const PlanDev pd, const double* __restrict__ A, const int32_t* __restrict__ gconn,
                                   const double* __restrict__ x, double* __restrict__ Y) {
    const int64_t s = int64_t(blockIdx.x) * NT + threadIdx.x;
    if (s >= pd.n_slots || pd.slot_elem[s] < 0) return;
    const int64_t ns = pd.n_slots;
    double xe[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) xe[i] = __ldg(x + gconn[i * ns + s]);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < NB; ++j) v = __fma_rn(__ldcs(A + sym_index(NB, i, j) * ns + s), xe[j], v);
        Y[i * ns + s] = v;
    }
}

__global__ void k_node_gather(int64_t n_n, const int32_t* __restrict__ node_ptr, const int32_t* __restrict__ node_ent,
                              const double* __restrict__ Y, const double* __restrict__ b,
                              const uint8_t* __restrict__ dmask, double* __restrict__ r) {
    const int64_t g = int64_t(blockIdx.x) * NT + threadIdx.x;
    if (g >= n_n) return;
    double v = 0.0;
    for (int k = node_ptr[g]; k < node_ptr[g + 1]; ++k) v += Y[node_ent[k]];
    r[g] = dmask[g] ? 0.0 : b[g] - v;
}

// r = mask(b - r): finish of the colour and atomic scatters.
__global__ void k_finish(int64_t n_n, const double* __restrict__ b, const uint8_t* __restrict__ dmask,
                         double* __restrict__ r) {
    const int64_t g = int64_t(blockIdx.x) * NT + threadIdx.x;
    if (g >= n_n) return;
    r[g] = dmask[g] ? 0.0 : b[g] - r[g];
}

unsigned blocks(int64_t n) { return unsigned((n + NT - 1) / NT); }

}  // namespace

cudaError_t launch_build_gconn(const PlanDev& pd, int32_t* gconn, cudaStream_t st, int* launches) {
    k_build_gconn<<<blocks(pd.n_slots), NT, 0, st>>>(pd, gconn);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_permute_slots(int nb, int64_t n_slots, int64_t n, const int32_t* order, const double* A,
                                 const int32_t* gconn, double* A_out, int32_t* gconn_out, cudaStream_t st,
                                 int* launches) {
    k_permute<<<blocks(n), NT, 0, st>>>(nb, n_slots, n, order, A, gconn, A_out, gconn_out);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_residual_colour(int nb, int n_col, const int64_t* col_ptr_host, int64_t n_el, const double* Ac,
                                   const int32_t* gc, const double* x, const double* b, const uint8_t* dmask,
                                   int64_t n_n, double* r, cudaStream_t st, int* launches) {
    cudaError_t e = cudaMemsetAsync(r, 0, sizeof(double) * size_t(n_n), st);
    if (e != cudaSuccess) return e;
    for (int c = 0; c < n_col; ++c) {
        const int64_t lo = col_ptr_host[c], hi = col_ptr_host[c + 1];
        if (hi <= lo) continue;
        if (nb == 3) k_colour_pass<3><<<blocks(hi - lo), NT, 0, st>>>(lo, hi, n_el, Ac, gc, x, r);
        else k_colour_pass<4><<<blocks(hi - lo), NT, 0, st>>>(lo, hi, n_el, Ac, gc, x, r);
        if (launches) *launches += 1;
    }
    k_finish<<<blocks(n_n), NT, 0, st>>>(n_n, b, dmask, r);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_residual_atomic(const PlanDev& pd, const double* A, const int32_t* gconn, const double* x,
                                   const double* b, const uint8_t* dmask, int64_t n_n, double* r, cudaStream_t st,
                                   int* launches) {
    cudaError_t e = cudaMemsetAsync(r, 0, sizeof(double) * size_t(n_n), st);
    if (e != cudaSuccess) return e;
    if (pd.nb == 3) k_atomic_pass<3><<<blocks(pd.n_slots), NT, 0, st>>>(pd, A, gconn, x, r);
    else k_atomic_pass<4><<<blocks(pd.n_slots), NT, 0, st>>>(pd, A, gconn, x, r);
    k_finish<<<blocks(n_n), NT, 0, st>>>(n_n, b, dmask, r);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_residual_node(const PlanDev& pd, const double* A, const int32_t* gconn, const int32_t* node_ptr,
                                 const int32_t* node_ent, const double* x, const double* b, const uint8_t* dmask,
                                 int64_t n_n, double* Y, double* r, cudaStream_t st, int* launches) {
    if (pd.nb == 3) k_element_products<3><<<blocks(pd.n_slots), NT, 0, st>>>(pd, A, gconn, x, Y);
    else k_element_products<4><<<blocks(pd.n_slots), NT, 0, st>>>(pd, A, gconn, x, Y);
    k_node_gather<<<blocks(n_n), NT, 0, st>>>(n_n, node_ptr, node_ent, Y, b, dmask, r);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

}  // namespace ebe
