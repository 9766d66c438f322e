// Learned message-passing preconditioner and flexible CG (sm_103a).
//
// The network (definition in include/ebe.h): 2 input features per node, an
// encoder to 32 features, 4 message-passing layers (mean over mesh
// neighbours minus self, then a per-node 64 -> 32 layer with a residual
// ReLU), and a decoder to a correction of the Jacobi step.  Hidden features
// and weights are BF16 (round to nearest even), accumulation FP32.
//
// Each message-passing layer is one kernel: a CTA of 128 threads takes tiles
// of 128 nodes; every thread gathers its node's neighbour features, forms
// u = [h; a] as BF16 directly in shared memory in the canonical no-swizzle
// K-major layout of the tensor cores, and thread 0 issues four
// tcgen05.mma.kind::f16 (M = 128, N = 32, K = 16) with the FP32 accumulator
// in tensor memory; tcgen05.ld brings row t back to thread t for the bias,
// ReLU and residual.  The backward pass (training only, on small meshes)
// runs on the CUDA cores in FP32 with deterministic block partials.
#include <cstdint>
#include <cuda_bf16.h>

#include "device_util.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace ebe {
namespace {

constexpr int H = kMpnnHidden;        // 32
constexpr int K2 = 2 * kMpnnHidden;   // 64
constexpr int L = kMpnnLayers;        // 4
constexpr int NT = 256;

// ---------------------------------------------------------------- tcgen05 helpers
// Shared-memory matrix descriptor, canonical K-major layout without swizzle:
// 8 x 16-byte core matrices; lbo = byte distance of core matrices adjacent in
// K, sbo = in M (or N).  Bits 46-47 hold the descriptor version (1).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: D FP32 (bit 4), A and B BF16 (bits 7,
// 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(H >> 3) << 17) | (uint32_t(128 >> 4) << 24);

// byte offset of element (row, k) of a K-major operand with K = 64
__host__ __device__ constexpr uint32_t core_off(int row, int k) {
    return uint32_t((row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 BF16 features of a node (64 bytes) <-> FP32.
__device__ __forceinline__ void load_h(const __nv_bfloat16* h, int64_t i, float (&v)[H]) {
    const uint4* p = reinterpret_cast<const uint4*>(h + i * H);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const uint4 w = __ldg(p + c);
        const uint32_t q[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            v[c * 8 + 2 * t] = __uint_as_float(q[t] << 16);
            v[c * 8 + 2 * t + 1] = __uint_as_float(q[t] & 0xffff0000u);
        }
    }
}
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
    return uint32_t(__bfloat16_as_ushort(x)) | (uint32_t(__bfloat16_as_ushort(y)) << 16);
}
__device__ __forceinline__ float bf(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }

// Sum over the block in a fixed order; result valid in thread 0.
template <int NTH>
__device__ __forceinline__ double bsum(double v, double* red) {
    return tma::block_sum<NTH>(v, red);
}

// ---------------------------------------------------------------- forward
// s = rms(r), sz = rms(dinv r) over free nodes (dinv != 0); last block writes
// sc[0] = s, sc[1] = sz.
__global__ void __launch_bounds__(NT) k_mpnn_norms(int64_t n, const double* __restrict__ r, const double* __restrict__ dinv,
                                                   double* __restrict__ part, uint32_t* __restrict__ ctr,
                                                   double* __restrict__ sc) {
    __shared__ double red[64];
    __shared__ bool last;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) {
        const double d = dinv[i];
        if (d != 0.0) {
            const double ri = r[i], zi = d * ri;
            a = fmadd(ri, ri, a);
            b = fmadd(zi, zi, b);
            c += 1.0;
        }
    }
    tma::block_sum2<NT>(a, b, red);
    c = bsum<NT>(c, red);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = a;
        part[3 * blockIdx.x + 1] = b;
        part[3 * blockIdx.x + 2] = c;
        last = tma::atom_add_acq_rel(ctr, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    double sa = 0.0, sb = 0.0, scn = 0.0;
    for (int i = threadIdx.x; i < int(gridDim.x); i += NT) {
        sa += __ldcg(part + 3 * i);
        sb += __ldcg(part + 3 * i + 1);
        scn += __ldcg(part + 3 * i + 2);
    }
    tma::block_sum2<NT>(sa, sb, red);
    scn = bsum<NT>(scn, red);
    if (threadIdx.x == 0) {
        const double nf = scn > 0.0 ? scn : 1.0;
        sc[0] = sqrt(sa / nf);
        sc[1] = sqrt(sb / nf);
        *ctr = 0u;
    }
}

// h = bf16(W_in x + b_in), x = [r / s, dinv r / sz] (FP32).
__global__ void __launch_bounds__(NT) k_mpnn_encode(int64_t n, const double* __restrict__ r, const double* __restrict__ dinv,
                                                    const double* __restrict__ sc, const float* __restrict__ wsm,
                                                    __nv_bfloat16* __restrict__ h, float* __restrict__ save_x) {
    const double s = sc[0], sz = sc[1];
    const bool ok = s > 0.0 && sz > 0.0;
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) {
        const double ri = r[i];
        const float x0 = ok ? float(ri / s) : 0.0f, x1 = ok ? float(dinv[i] * ri / sz) : 0.0f;
        if (save_x) { save_x[2 * i] = x0; save_x[2 * i + 1] = x1; }
        uint32_t w[H / 2];
#pragma unroll
        for (int o = 0; o < H; o += 2) {
            const float a = fmaf(wsm[kMpnnWin + 2 * o + 1], x1, fmaf(wsm[kMpnnWin + 2 * o], x0, wsm[kMpnnBin + o]));
            const float b = fmaf(wsm[kMpnnWin + 2 * o + 3], x1, fmaf(wsm[kMpnnWin + 2 * o + 2], x0, wsm[kMpnnBin + o + 1]));
            w[o / 2] = pack2(a, b);
        }
        uint4* dst = reinterpret_cast<uint4*>(h + i * H);
#pragma unroll
        for (int c = 0; c < 4; ++c) dst[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
    }
}

// One message-passing layer on the tensor cores (see the file comment).
// wl: this layer's 32 x 64 BF16 weights in the core-matrix layout (4 KB);
// bias: FP32 (BF16-rounded) [32].  save_u (bf16 [n][64]) and save_v (fp32
// [n][32]) are kept for training (nullable).
struct LayerSmem {
    static constexpr uint32_t B = 0, A = 4096, bar = 4096 + 16384, taddr = bar + 8, total = taddr + 8;
};

__global__ void __launch_bounds__(128) k_mpnn_layer(int64_t n, const int32_t* __restrict__ nbr_ptr,
                                                    const int32_t* __restrict__ nbr, const float* __restrict__ inv_deg,
                                                    const __nv_bfloat16* __restrict__ h_in, __nv_bfloat16* __restrict__ h_out,
                                                    const uint4* __restrict__ wl, const float* __restrict__ bias,
                                                    __nv_bfloat16* __restrict__ save_u, float* __restrict__ save_v,
                                                    int32_t* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t sB = tma::smem_addr(smem + LayerSmem::B), sA = tma::smem_addr(smem + LayerSmem::A);
    const uint32_t mbar = tma::smem_addr(smem + LayerSmem::bar);
    uint32_t* taddr_s = reinterpret_cast<uint32_t*>(smem + LayerSmem::taddr);
    __shared__ int sflag;

    // weights into shared memory (already in the core-matrix layout)
    for (int c = tid; c < 4096 / 16; c += 128) reinterpret_cast<uint4*>(smem + LayerSmem::B)[c] = __ldg(wl + c);
    if (tid == 0) {
        tma::mbar_init(mbar, 1);
        sflag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(
                         tma::smem_addr(taddr_s))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *taddr_s;
    float b[H];
#pragma unroll
    for (int o = 0; o < H; ++o) b[o] = __ldg(bias + o);

    const int64_t ntiles = (n + 127) / 128;
    uint32_t phase = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t i = tile * 128 + tid;
        const bool valid = i < n;
        float hi[H], a[H];
#pragma unroll
        for (int o = 0; o < H; ++o) { hi[o] = 0.0f; a[o] = 0.0f; }
        if (valid) {
            load_h(h_in, i, hi);
            const int j0 = __ldg(nbr_ptr + i), j1 = __ldg(nbr_ptr + i + 1);
            for (int j = j0; j < j1; ++j) {
                float hj[H];
                load_h(h_in, __ldg(nbr + j), hj);
#pragma unroll
                for (int o = 0; o < H; ++o) a[o] += hj[o];
            }
            const float w = __ldg(inv_deg + i);
#pragma unroll
            for (int o = 0; o < H; ++o) a[o] = fmaf(a[o], w, -hi[o]);
        }
        // u = [h; a] (BF16) into the A tile, row tid: 8 chunks of 8 values
        uint32_t u[K2 / 2];
#pragma unroll
        for (int o = 0; o < H; o += 2) { u[o / 2] = pack2(hi[o], hi[o + 1]); u[H / 2 + o / 2] = pack2(a[o], a[o + 1]); }
#pragma unroll
        for (int c = 0; c < 8; ++c)
            *reinterpret_cast<uint4*>(smem + LayerSmem::A + core_off(tid, 8 * c)) =
                make_uint4(u[4 * c], u[4 * c + 1], u[4 * c + 2], u[4 * c + 3]);
        if (save_u != nullptr && valid) {
            uint4* dst = reinterpret_cast<uint4*>(save_u + i * K2);
#pragma unroll
            for (int c = 0; c < 8; ++c) dst[c] = make_uint4(u[4 * c], u[4 * c + 1], u[4 * c + 2], u[4 * c + 3]);
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < K2 / 16; ++kk)
                tc_mma(tmem, umma_desc(sA + kk * 256, 128, 1024), umma_desc(sB + kk * 256, 128, 1024), kIdesc, kk > 0);
            tc_commit(mbar);
        }
        if (tid == 0 && !tma::mbar_wait_bounded(mbar, phase, err)) sflag = 1;
        __syncthreads();
        if (sflag) {                        // uniform: the accumulator did not arrive in time
            // the committed MMA may still be writing TMEM: wait once more
            // (bounded) before the accumulator is freed below
            if (tid == 0) tma::mbar_wait_bounded(mbar, phase, nullptr);
            break;
        }
        phase ^= 1u;
        while (!tma::mbar_try_wait(mbar, phase ^ 1u)) {
        }
        tc_fence_after();
        float v[H];
        tc_ld32(tmem + (uint32_t(warp * 32) << 16), v);
        if (valid) {
            uint32_t w[H / 2];
#pragma unroll
            for (int o = 0; o < H; o += 2) {
                const float v0 = v[o] + b[o], v1 = v[o + 1] + b[o + 1];
                if (save_v != nullptr) { save_v[i * H + o] = v0; save_v[i * H + o + 1] = v1; }
                w[o / 2] = pack2(hi[o] + fmaxf(v0, 0.0f), hi[o + 1] + fmaxf(v1, 0.0f));
            }
            uint4* dst = reinterpret_cast<uint4*>(h_out + i * H);
#pragma unroll
            for (int c = 0; c < 4; ++c) dst[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
        }
        tc_fence_before();
        __syncthreads();                    // TMEM and the A tile are free for the next tile
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

// z = zj + sz * (w_out . h + b_out) on free nodes, 0 on Dirichlet nodes.
__global__ void __launch_bounds__(NT) k_mpnn_decode(int64_t n, const double* __restrict__ r, const double* __restrict__ dinv,
                                                    const double* __restrict__ sc, const float* __restrict__ wsm,
                                                    const __nv_bfloat16* __restrict__ h, double* __restrict__ z) {
    const double sz = sc[1];
    const bool ok = sc[0] > 0.0 && sz > 0.0;
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) {
        const double d = dinv[i];
        if (!ok || d == 0.0) { z[i] = 0.0; continue; }
        float hv[H];
        load_h(h, i, hv);
        float o = wsm[kMpnnBout];
#pragma unroll
        for (int c = 0; c < H; ++c) o = fmaf(wsm[kMpnnWout + c], hv[c], o);
        z[i] = fmadd(sz, double(o), d * r[i]);
    }
}

// ---------------------------------------------------------------- backward (CUDA cores, FP32)
// go = gz * sz on free nodes; gh = go * w_out; partials of dL/dw_out, dL/db_out.
__global__ void __launch_bounds__(NT) k_mpnn_bwd_out(int64_t n, const double* __restrict__ gz, const double* __restrict__ dinv,
                                                     const double* __restrict__ sc, const float* __restrict__ wsm,
                                                     const __nv_bfloat16* __restrict__ h4, float* __restrict__ gh,
                                                     double* __restrict__ part) {
    __shared__ double red[32];
    const double sz = sc[1];
    double gw[H + 1];
#pragma unroll
    for (int c = 0; c <= H; ++c) gw[c] = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) {
        const float go = dinv[i] != 0.0 ? float(gz[i] * sz) : 0.0f;
        float hv[H];
        load_h(h4, i, hv);
#pragma unroll
        for (int c = 0; c < H; ++c) {
            gh[i * H + c] = go * wsm[kMpnnWout + c];
            gw[c] += double(go) * double(hv[c]);
        }
        gw[H] += double(go);
    }
    for (int c = 0; c <= H; ++c) {
        const double s = bsum<NT>(gw[c], red);
        if (threadIdx.x == 0) part[int64_t(blockIdx.x) * (H + 1) + c] = s;
    }
}

// Layer backward, first half: gv = gh * [v > 0]; gu = W^T gv; the node's own
// part gh' = gh + gu_h - gu_a and ga = gu_a / deg (spread to neighbours by
// k_mpnn_bwd_gather); block partials of dL/dW (32 x 64) and dL/db (32).
// A block takes 64 nodes at a time: gv and u staged in shared memory, each
// thread then owns 8 of the 2048 weight entries (and thread o < 32 the bias o).
constexpr int kBwdNodes = 64;
__global__ void __launch_bounds__(NT) k_mpnn_bwd_layer(int64_t n, const float* __restrict__ inv_deg,
                                                       const float* __restrict__ gh, const float* __restrict__ v,
                                                       const __nv_bfloat16* __restrict__ u, const float* __restrict__ wT,
                                                       float* __restrict__ ghp, float* __restrict__ ga,
                                                       double* __restrict__ part) {
    __shared__ float gvs[kBwdNodes][H];
    __shared__ float us[kBwdNodes][K2];
    double acc[8];
    double accb = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    const int tid = threadIdx.x;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = int64_t(blockIdx.x) * chunk, c1 = min(n, c0 + chunk);
    for (int64_t base = c0; base < c1; base += kBwdNodes) {
        // stage gv and u for 64 nodes; 4 threads per node
        for (int t = tid; t < kBwdNodes * 4; t += NT) {
            const int ln = t >> 2, part4 = t & 3;
            const int64_t i = base + ln;
            const bool ok = i < c1;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int o = part4 * 8 + q;
                gvs[ln][o] = ok && v[i * H + o] > 0.0f ? gh[i * H + o] : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int k = part4 * 16 + q;
                us[ln][k] = ok ? __bfloat162float(u[i * K2 + k]) : 0.0f;
            }
        }
        __syncthreads();
        // per node (one thread per node for the first 64 threads): gu = W^T gv
        if (tid < kBwdNodes && base + tid < c1) {
            const int64_t i = base + tid;
            float gu[K2];
#pragma unroll
            for (int k = 0; k < K2; ++k) gu[k] = 0.0f;
            for (int o = 0; o < H; ++o) {
                const float g = gvs[tid][o];
#pragma unroll
                for (int k = 0; k < K2; ++k) gu[k] = fmaf(wT[k * H + o], g, gu[k]);
            }
            const float w = inv_deg[i];
#pragma unroll
            for (int c = 0; c < H; ++c) {
                ghp[i * H + c] = gh[i * H + c] + gu[c] - gu[H + c];
                ga[i * H + c] = gu[H + c] * w;
            }
        }
        // weight gradient partials: entry e = tid + 256 q of the 32 x 64 matrix
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = tid + NT * q, o = e >> 6, k = e & 63;
            float s = 0.0f;
            for (int ln = 0; ln < kBwdNodes; ++ln) s = fmaf(gvs[ln][o], us[ln][k], s);
            acc[q] += double(s);
        }
        if (tid < H) {
            float s = 0.0f;
            for (int ln = 0; ln < kBwdNodes; ++ln) s += gvs[ln][tid];
            accb += double(s);
        }
        __syncthreads();
    }
    double* p = part + int64_t(blockIdx.x) * (H * K2 + H);
#pragma unroll
    for (int q = 0; q < 8; ++q) p[tid + NT * q] = acc[q];
    if (tid < H) p[H * K2 + tid] = accb;
}

// gh_prev[j] = ghp[j] + sum over neighbours i of j of ga[i] (the mesh graph is symmetric).
__global__ void __launch_bounds__(NT) k_mpnn_bwd_gather(int64_t n, const int32_t* __restrict__ nbr_ptr,
                                                        const int32_t* __restrict__ nbr, const float* __restrict__ ghp,
                                                        const float* __restrict__ ga, float* __restrict__ gh) {
    for (int64_t t = int64_t(blockIdx.x) * NT + threadIdx.x; t < n * H; t += int64_t(gridDim.x) * NT) {
        const int64_t j = t / H;
        const int c = int(t % H);
        float s = ghp[t];
        const int i1 = nbr_ptr[j + 1];
        for (int q = nbr_ptr[j]; q < i1; ++q) s += ga[int64_t(nbr[q]) * H + c];
        gh[t] = s;
    }
}

// Encoder backward: block partials of dL/dW_in (32 x 2) and dL/db_in (32),
// in parameter order (W_in[o][c] at 2 o + c, b_in[o] at 64 + o).
__global__ void __launch_bounds__(NT) k_mpnn_bwd_in(int64_t n, const float* __restrict__ gh, const float* __restrict__ x,
                                                    double* __restrict__ part) {
    __shared__ double red[32];
    for (int o0 = 0; o0 < H; o0 += 8) {
        double s[8][3];
#pragma unroll
        for (int q = 0; q < 8; ++q) s[q][0] = s[q][1] = s[q][2] = 0.0;
        for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) {
            const double x0 = x[2 * i], x1 = x[2 * i + 1];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const double g = gh[i * H + o0 + q];
                s[q][0] = fmadd(g, x0, s[q][0]);
                s[q][1] = fmadd(g, x1, s[q][1]);
                s[q][2] += g;
            }
        }
        for (int q = 0; q < 8; ++q) {
            const int o = o0 + q;
            const double t0 = bsum<NT>(s[q][0], red);
            const double t1 = bsum<NT>(s[q][1], red);
            const double t2 = bsum<NT>(s[q][2], red);
            if (threadIdx.x == 0) {
                double* p = part + int64_t(blockIdx.x) * (3 * H);
                p[2 * o] = t0;
                p[2 * o + 1] = t1;
                p[2 * H + o] = t2;
            }
        }
    }
}

// Sum of block partials in index order: out[k] = sum_b part[b * stride + k].
__global__ void k_mpnn_reduce(int nblocks, int stride, int count, const double* __restrict__ part, double* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[int64_t(b) * stride + k];
    out[k] = s;
}

// Adam on the FP32 master parameters, then the BF16 copies the forward
// pass reads (core-matrix layout for the layer weights, rounded FP32 values
// for the encoder, biases and decoder).
__global__ void k_mpnn_adam(int np, float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const double* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const float gk = float(g[k]);
    const float mk = b1 * m[k] + (1.0f - b1) * gk, vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    theta[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

__global__ void k_mpnn_pack(const float* __restrict__ theta, uint16_t* __restrict__ wl, float* __restrict__ wsm,
                            float* __restrict__ wT) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < kMpnnParams) {
        // small parameters: encoder, biases, decoder (BF16-rounded values as FP32)
        if (k < kMpnnW0) {
            wsm[k] = bf(theta[k]);
        } else {
            const int rel = k - kMpnnW0, l = rel / kMpnnLayerParams, q = rel % kMpnnLayerParams;
            if (l < L && q < H * K2) {
                const int o = q / K2, kk = q % K2;
                const __nv_bfloat16 w = __float2bfloat16_rn(theta[k]);
                wl[l * (H * K2) + core_off(o, kk) / 2] = __bfloat16_as_ushort(w);
                wT[l * (H * K2) + kk * H + o] = __bfloat162float(w);
            } else if (l < L) {
                wsm[kMpnnBl + l * H + (q - H * K2)] = bf(theta[k]);
            } else {
                wsm[kMpnnWout + (k - kMpnnThWout)] = bf(theta[k]);   // w_out, then b_out at kMpnnBout
            }
        }
    }
}

// ---------------------------------------------------------------- energy loss and flexible CG vectors
// w = e - z (into w), and grad = -2 Aw / eAe after the operator pass (second kernel).
__global__ void __launch_bounds__(NT) k_sub(int64_t n, const double* __restrict__ e, const double* __restrict__ z,
                                            double* __restrict__ w) {
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) w[i] = e[i] - z[i];
}
__global__ void __launch_bounds__(NT) k_dot2(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                             const double* __restrict__ c, double* __restrict__ part,
                                             uint32_t* __restrict__ ctr, double* __restrict__ out) {
    // out[0] = a.b, out[1] = a.c (c nullable)
    __shared__ double red[64];
    __shared__ bool last;
    double s0 = 0.0, s1 = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) {
        s0 = fmadd(a[i], b[i], s0);
        if (c) s1 = fmadd(a[i], c[i], s1);
    }
    tma::block_sum2<NT>(s0, s1, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s0;
        part[2 * blockIdx.x + 1] = s1;
        last = tma::atom_add_acq_rel(ctr, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    double t0 = 0.0, t1 = 0.0;
    for (int i = threadIdx.x; i < int(gridDim.x); i += NT) { t0 += __ldcg(part + 2 * i); t1 += __ldcg(part + 2 * i + 1); }
    tma::block_sum2<NT>(t0, t1, red);
    if (threadIdx.x == 0) { out[0] = t0; out[1] = t1; *ctr = 0u; }
}
__global__ void __launch_bounds__(NT) k_scale(int64_t n, const double* __restrict__ a, const double* __restrict__ num,
                                              double factor, double* __restrict__ out) {
    // out = factor * a / num[0]
    const double f = factor / num[0];
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) out[i] = f * a[i];
}

// FCG step 1: dots z.q_prev, z.r, p_prev.r (last block): beta = -z.q/p.q_prev
// (0 on the first step), and sc->rho = p.r for the operator pass's alpha.
__global__ void __launch_bounds__(NT) k_fcg_dots(int64_t n, const double* __restrict__ z, const double* __restrict__ r,
                                                 const double* __restrict__ p, const double* __restrict__ q, int first,
                                                 double* __restrict__ part, Scalars* __restrict__ sc) {
    __shared__ double red[64];
    __shared__ bool last;
    if (sc->done) return;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) {
        const double zi = z[i], ri = r[i];
        b = fmadd(zi, ri, b);
        if (!first) {
            a = fmadd(zi, q[i], a);
            c = fmadd(p[i], ri, c);
        }
    }
    tma::block_sum2<NT>(a, b, red);
    c = bsum<NT>(c, red);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = a;
        part[3 * blockIdx.x + 1] = b;
        part[3 * blockIdx.x + 2] = c;
        last = tma::atom_add_acq_rel(&sc->ctr_vec, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    double sa = 0.0, sb = 0.0, scc = 0.0;
    for (int i = threadIdx.x; i < int(gridDim.x); i += NT) {
        sa += __ldcg(part + 3 * i);
        sb += __ldcg(part + 3 * i + 1);
        scc += __ldcg(part + 3 * i + 2);
    }
    tma::block_sum2<NT>(sa, sb, red);
    scc = bsum<NT>(scc, red);
    if (threadIdx.x == 0) {
        sc->ctr_vec = 0u;
        const double beta = first ? 0.0 : -sa / sc->pq;
        sc->beta = beta;
        sc->rho = sb + beta * scc;        // p.r with p = z + beta p_prev
        if (!isfinite(beta) || !isfinite(sc->rho)) { sc->done = 1; sc->reason = kBreakdown; }
    }
}
// p = z + beta p (first: p = z).
__global__ void __launch_bounds__(NT) k_fcg_dir(int64_t n, const double* __restrict__ z, double* __restrict__ p, int first,
                                                const Scalars* __restrict__ sc) {
    if (sc->done) return;
    const double be = first ? 0.0 : sc->beta;
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT)
        p[i] = first ? z[i] : fmadd(be, p[i], z[i]);
}
// z = dinv r (the Jacobi preconditioner of the fallback and of the comparison).
__global__ void __launch_bounds__(NT) k_jacobi(int64_t n, const double* __restrict__ r, const double* __restrict__ dinv,
                                               double* __restrict__ z, const int32_t* __restrict__ stop) {
    if (stop && *stop) return;
    for (int64_t i = int64_t(blockIdx.x) * NT + threadIdx.x; i < n; i += int64_t(gridDim.x) * NT) z[i] = dinv[i] * r[i];
}

int grid_for(int64_t n) {
    int64_t g = (n + NT - 1) / NT;
    return int(g < 1 ? 1 : (g > 1216 ? 1216 : g));
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_mpnn_forward(const MpnnDev& m, int64_t n, const double* r, const double* dinv, double* z, bool save,
                                cudaStream_t st, int* launches) {
    const int g = grid_for(n);
    k_mpnn_norms<<<g, NT, 0, st>>>(n, r, dinv, m.part, m.ctr, m.sc);
    auto B = [](uint16_t* p) { return reinterpret_cast<__nv_bfloat16*>(p); };
    k_mpnn_encode<<<g, NT, 0, st>>>(n, r, dinv, m.sc, m.wsm, B(m.h[0]), save ? m.save_x : nullptr);
    cudaError_t e = cudaFuncSetAttribute(k_mpnn_layer, cudaFuncAttributeMaxDynamicSharedMemorySize, int(LayerSmem::total));
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + 127) / 128;
    const int lg = int(tiles < int64_t(m.num_sms) * 8 ? tiles : int64_t(m.num_sms) * 8);
    for (int l = 0; l < L; ++l) {
        const __nv_bfloat16* hin = B(save ? m.h[l] : m.h[l & 1]);
        __nv_bfloat16* hout = B(save ? m.h[l + 1] : m.h[(l + 1) & 1]);
        k_mpnn_layer<<<lg > 0 ? lg : 1, 128, LayerSmem::total, st>>>(
            n, m.nbr_ptr, m.nbr, m.inv_deg, hin, hout, reinterpret_cast<const uint4*>(m.wl + l * (H * K2)),
            m.wsm + kMpnnBl + l * H, save ? B(m.save_u) + int64_t(l) * n * K2 : nullptr,
            save ? m.save_v + int64_t(l) * n * H : nullptr, m.err);
    }
    k_mpnn_decode<<<g, NT, 0, st>>>(n, r, dinv, m.sc, m.wsm, B(save ? m.h[L] : m.h[L & 1]), z);
    if (launches) *launches += 3 + L;
    return cudaGetLastError();
}

cudaError_t launch_mpnn_backward(const MpnnDev& m, int64_t n, const double* gz, const double* dinv, double* grad,
                                 cudaStream_t st, int* launches) {
    const int g = grid_for(n);
    const int gb = int(g < 152 ? g : 152);
    auto B = [](uint16_t* p) { return reinterpret_cast<const __nv_bfloat16*>(p); };
    // decoder
    k_mpnn_bwd_out<<<gb, NT, 0, st>>>(n, gz, dinv, m.sc, m.wsm, B(m.h[L]), m.gh, m.part);
    k_mpnn_reduce<<<1, 64, 0, st>>>(gb, H + 1, H + 1, m.part, grad + kMpnnThWout);
    for (int l = L - 1; l >= 0; --l) {
        k_mpnn_bwd_layer<<<gb, NT, 0, st>>>(n, m.inv_deg, m.gh, m.save_v + int64_t(l) * n * H,
                                            B(m.save_u) + int64_t(l) * n * K2, m.wT + l * (H * K2), m.ghp, m.ga, m.part);
        k_mpnn_reduce<<<(H * K2 + H + 255) / 256, 256, 0, st>>>(gb, H * K2 + H, H * K2 + H, m.part,
                                                                grad + kMpnnW0 + l * kMpnnLayerParams);
        k_mpnn_bwd_gather<<<g, NT, 0, st>>>(n, m.nbr_ptr, m.nbr, m.ghp, m.ga, m.gh);
    }
    // encoder: partials already in parameter order (W_in [32][2], b_in [32])
    k_mpnn_bwd_in<<<gb, NT, 0, st>>>(n, m.gh, m.save_x, m.part);
    k_mpnn_reduce<<<1, 128, 0, st>>>(gb, 3 * H, 3 * H, m.part, grad);
    if (launches) *launches += 5 + 3 * L;
    return cudaGetLastError();
}

cudaError_t launch_mpnn_pack(const MpnnDev& m, cudaStream_t st, int* launches) {
    k_mpnn_pack<<<(kMpnnParams + 255) / 256, 256, 0, st>>>(m.theta, m.wl, m.wsm, m.wT);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_mpnn_adam(const MpnnDev& m, const double* grad, float lr, int step, cudaStream_t st, int* launches) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, float(step)), c2 = 1.0f - powf(b2, float(step));
    k_mpnn_adam<<<(kMpnnParams + 255) / 256, 256, 0, st>>>(kMpnnParams, m.theta, m.adam_m, m.adam_v, grad, lr, b1, b2,
                                                            1e-8f, c1, c2);
    if (launches) *launches += 1;
    return launch_mpnn_pack(m, st, launches);
}

cudaError_t launch_sub(int64_t n, const double* e, const double* z, double* w, cudaStream_t st, int* launches) {
    k_sub<<<grid_for(n), NT, 0, st>>>(n, e, z, w);
    if (launches) *launches += 1;
    return cudaGetLastError();
}
cudaError_t launch_dot2(int64_t n, const double* a, const double* b, const double* c, double* part, uint32_t* ctr,
                        double* out, cudaStream_t st, int* launches) {
    k_dot2<<<grid_for(n), NT, 0, st>>>(n, a, b, c, part, ctr, out);
    if (launches) *launches += 1;
    return cudaGetLastError();
}
cudaError_t launch_scale(int64_t n, const double* a, const double* num, double factor, double* out, cudaStream_t st,
                         int* launches) {
    k_scale<<<grid_for(n), NT, 0, st>>>(n, a, num, factor, out);
    if (launches) *launches += 1;
    return cudaGetLastError();
}
cudaError_t launch_fcg_dots(int64_t n, const double* z, const double* r, const double* p, const double* q, int first,
                            double* part, Scalars* sc, cudaStream_t st, int* launches) {
    k_fcg_dots<<<grid_for(n), NT, 0, st>>>(n, z, r, p, q, first, part, sc);
    if (launches) *launches += 1;
    return cudaGetLastError();
}
cudaError_t launch_fcg_dir(int64_t n, const double* z, double* p, int first, const Scalars* sc, cudaStream_t st,
                           int* launches) {
    k_fcg_dir<<<grid_for(n), NT, 0, st>>>(n, z, p, first, sc);
    if (launches) *launches += 1;
    return cudaGetLastError();
}
cudaError_t launch_jacobi(int64_t n, const double* r, const double* dinv, double* z, const int32_t* stop, cudaStream_t st,
                          int* launches) {
    k_jacobi<<<grid_for(n), NT, 0, st>>>(n, r, dinv, z, stop);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace ebe
