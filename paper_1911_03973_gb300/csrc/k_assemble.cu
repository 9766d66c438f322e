// Element matrices, load vector and Jacobi diagonal, and exports of the
// element data (sm_103a).
//
// The P1 element matrices of Eq. matrices_K_M are formed in closed form per
// element; the load vector b = sum_e C_e^T M_e f_e and the Jacobi diagonal
// d = sum_e C_e^T diag(A_e) are summed per node like the residual: one patch
// per CTA, colour rounds in shared memory, halo partials for shared nodes
// added in patch order by a fix-up pass (bitwise reproducible).
#include <cstdint>

#include "device_util.cuh"
#include "kernels.h"

namespace ebe {
namespace {

constexpr int kHead = 32 * 8 + ((kMaxColours + 1) * 4 + 15) / 16 * 16;  // reduction + colour offsets
constexpr int kFixThreads = 256;

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
// packed symmetric (sym_index),
// with the load vector b = sum_e C_e^T M_e f_e and d = sum_e C_e^T diag(A_e)
// accumulated per node like the residual (colour order, halo for shared).
template <int NB>
__global__ void __launch_bounds__(256, 2)
k_assemble(const PlanDev pd, const double* __restrict__ coords, const double* __restrict__ f, double nu_all,
           const double* __restrict__ nu_patch, double* __restrict__ A64, float* __restrict__ A32, double* __restrict__ b, double* __restrict__ d,
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
    const double nu = nu_patch != nullptr ? __ldg(nu_patch + p) : nu_all;   // batches: nu of the patch's problem
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
                if (ok && i <= j) {   // packed symmetric storage
                    A64[sym_index(NB, i, j) * ns + slot0 + s] = aij;
                    // FP32 copy in difference form: row sums on the diagonal slots
                    if (A32 != nullptr) A32[sym_index(NB, i, j) * ns + slot0 + s] = float(i == j ? rowsum : aij);
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
        for (int j = 0; j < nb; ++j) out[int64_t(e) * nb * nb + j * nb + i] = A[sym_index(nb, i, j) * pd.n_slots + s];
}

__global__ void k_mark(int32_t* __restrict__ ids, int64_t n, const uint8_t* __restrict__ mask) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int g = ids[k] & kNodeMask;
        ids[k] = mask[g] ? int32_t(uint32_t(g) | kDirichletBit) : g;
    }
}

}  // namespace

cudaError_t launch_assemble(const PlanDev& pd, const double* coords, const double* f, double nu, const double* nu_patch,
                            double* A64,
                            float* A32, double* b, double* d, double* dinv, float* b32, float* dinv32,
                            double* halo2, unsigned long long* bad, cudaStream_t st, int* launches) {
    const size_t sm = kHead + size_t(pd.max_nodes) * sizeof(double) * (pd.dim + 3);
    cudaError_t e;
    if (pd.nb == 3) {
        if (sm > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k_assemble<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm))) != cudaSuccess)
            return e;
        k_assemble<3><<<pd.n_patches, 256, sm, st>>>(pd, coords, f, nu, nu_patch, A64, A32, b, d, dinv, b32, dinv32, halo2, bad);
    } else {
        if (sm > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k_assemble<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm))) != cudaSuccess)
            return e;
        k_assemble<4><<<pd.n_patches, 256, sm, st>>>(pd, coords, f, nu, nu_patch, A64, A32, b, d, dinv, b32, dinv32, halo2, bad);
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
