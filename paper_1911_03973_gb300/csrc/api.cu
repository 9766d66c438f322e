// C ABI of libebe.so (declared in include/ebe.h).
//
// The handle owns the element partition, the element matrices and all solver
// workspaces on one device.  Every call validates its arguments on the host
// before it enqueues anything, and reports failures as an ebe_status plus a
// message; nothing is thrown across the ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "ebe.h"
#include "ebe_internal.h"
#include "kernels.h"

using namespace ebe;

struct ebe_handle {
    int device = 0;
    cudaStream_t st = nullptr;      // stream all work is ordered on
    bool own_stream = false;
    cudaStream_t user = nullptr;    // the caller's stream when it is the legacy stream
    cudaEvent_t ev_join = nullptr;
    HostPlan plan;
    PlanDev pd;
    std::vector<void*> allocs;
    int64_t bytes = 0;
    int64_t launches = 0;
    std::string err;

    // mesh and partition on the device
    double* coords = nullptr;
    int32_t* pnode = nullptr;
    int32_t* sh_node = nullptr;
    int64_t n_pnode = 0;

    // problem
    bool problem_set = false;
    double nu = 0.0;
    int64_t n_d = 0;
    double* f = nullptr;
    int32_t* nd = nullptr;
    double* g = nullptr;
    uint8_t* dmask = nullptr;

    // assembled operator
    bool assembled = false;
    int store = EBE_STORE_FP64;
    double *A64 = nullptr, *b = nullptr, *d = nullptr, *dinv = nullptr;
    float *A32 = nullptr, *b32 = nullptr, *dinv32 = nullptr;
    float* Adw = nullptr;           // A64 as FP32 pairs, the dw_pairs layout (made on first use)
    bool dw_ready = false;

    // scratch of the patch passes
    double* halo64 = nullptr;
    float* halo32 = nullptr;
    SmallInfo* small_info = nullptr;  // outcome of the one-CTA solver
    int32_t* small_order = nullptr;   // its colouring of the whole mesh
    int32_t* small_col = nullptr;
    uint16_t* small_inc_ptr = nullptr;   // node -> (element, row) incidences in colour order
    uint16_t* small_inc = nullptr;
    int small_ncol = 0;
    double* halo2 = nullptr;
    double* part_patch = nullptr;   // n_patches + fix_grid(n_shared)
    double* part_vec = nullptr;     // 3 * 1216
    Scalars* sc = nullptr;
    Scalars* sc_host = nullptr;     // pinned
    unsigned long long* bad = nullptr;
    int32_t* dev_err = nullptr;     // set by a device wait that gave up

    // solver vectors
    double *x64w = nullptr, *r64 = nullptr, *p64 = nullptr, *q64 = nullptr;
    float *p32 = nullptr, *q32 = nullptr, *r32 = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_chunk[2] = {0, 0};
    int graph_nodes[2] = {0, 0};

    // solver numbering of the single-sync mixed solver (see create_device)
    PlanDev pd_int;                 // pd with the node tables in the solver numbering
    int64_t n_int = 0;              // nodes of the solver numbering (with padding)
    int32_t* int_of_user = nullptr; // [n_n] solver number of each node
    int32_t* pnode_int = nullptr;
    int32_t* sh_node_int = nullptr;
    bool int_ready = false;         // bi, dinvi32 built from the current assembly
    double *xi = nullptr, *ri64 = nullptr, *bi = nullptr;
    float *dinvi32 = nullptr, *ri32 = nullptr, *qi32 = nullptr, *pi32[2] = {nullptr, nullptr};
    double* part5 = nullptr;
    cudaGraphExec_t cg_graph[2] = {nullptr, nullptr};   // chunk of passes per starting direction buffer
    int cg_chunk = 0;
    int cg_nodes = 0;

    // batches (ebe_create makes a batch of one)
    int n_prob = 1;
    BatchLayout lay;
    double* nu_patch = nullptr;          // [n_patches] nu of each patch's problem (batches of > 1)
    BatchItem* bfix = nullptr;           // fix-up items
    int n_bfix = 0;
    BatchItem* btile[3] = {nullptr, nullptr, nullptr};   // node tiles of 1024, 2048, 4096 nodes
    int n_btile[3] = {0, 0, 0};
    BatchProbInfo* bpinfo[3] = {nullptr, nullptr, nullptr};   // per problem item ranges, per tile size
    double* bpart_f = nullptr;
    double* bpart_u = nullptr;
    BatchProblem* bprob = nullptr;
    BatchProblem* bprob_host = nullptr;  // pinned [n_prob]
    uint32_t* bctr = nullptr;
    uint32_t* bbar = nullptr;
    int32_t* blive = nullptr;
    int64_t* bloops = nullptr;
    unsigned long long* bphase = nullptr;   // [4] phase times of the persistent kernel
    int64_t* bcount_host = nullptr;      // pinned: loops, live, phase times [4]
    ebe_batch_config bcfg[2] = {{0, 0, 0}, {0, 0, 0}};   // launch shape per precision (FP64, mixed)
    cudaGraphExec_t bgraph = nullptr;
    std::vector<double> bgraph_key;

    // mesh graph (learned preconditioner) and flexible-CG vectors
    int32_t* g_ptr = nullptr;
    int32_t* g_nbr = nullptr;
    float* g_invdeg = nullptr;
    double* z64 = nullptr;
    double *xsave0 = nullptr, *xsave1 = nullptr;   // iterates of the learned solver's race

    // comparison scatters
    int32_t* gconn = nullptr;
    std::vector<int32_t> gconn_host;   // [n_slots][nb]
    double* Acol = nullptr;
    int32_t* gcol = nullptr;
    std::vector<int64_t> col_ptr;
    int n_gcol = 0;
    int32_t* node_ptr = nullptr;
    int32_t* node_ent = nullptr;
    double* Y = nullptr;
};

namespace {

thread_local std::string g_create_error;

struct CudaFail {
    cudaError_t e;
    const char* what;
};

int fail(ebe_handle* h, int status, const std::string& msg) {
    if (h) h->err = msg;
    return status;
}

int cuda_fail(ebe_handle* h, cudaError_t e, const char* what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, e == cudaErrorMemoryAllocation ? EBE_OOM : EBE_CUDA_ERROR, msg);
}

#define CK(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return ebe_status(cuda_fail(h, e_, what)); \
    } while (0)

template <typename T>
int dalloc(ebe_handle* h, T** p, int64_t count, bool zero = false) {
    if (*p) return EBE_OK;
    void* v = nullptr;
    size_t bytes = size_t(std::max<int64_t>(count, 1)) * sizeof(T);
    cudaError_t e = cudaMalloc(&v, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(h, e, "cudaMalloc"); }
    h->allocs.push_back(v);
    h->bytes += int64_t(bytes);
    if (zero) {
        e = cudaMemsetAsync(v, 0, bytes, h->st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
    }
    *p = static_cast<T*>(v);
    return EBE_OK;
}

#define TRY(call)                    \
    do {                             \
        int s_ = (call);             \
        if (s_ != EBE_OK) return ebe_status(s_); \
    } while (0)

template <typename T>
int upload(ebe_handle* h, T** dst, const T* src, int64_t count) {
    TRY(dalloc(h, dst, count));
    if (count > 0) CK(cudaMemcpyAsync(*dst, src, sizeof(T) * size_t(count), cudaMemcpyHostToDevice, h->st), "upload");
    return EBE_OK;
}

// Order the handle's stream after the caller's legacy stream (and back).
void enter(ebe_handle* h) {
    if (h->own_stream) {
        cudaEventRecord(h->ev_join, h->user);
        cudaStreamWaitEvent(h->st, h->ev_join, 0);
    }
}
void leave(ebe_handle* h) {
    if (h->own_stream) {
        cudaEventRecord(h->ev_join, h->st);
        cudaStreamWaitEvent(h->user, h->ev_join, 0);
    }
}

// Makes `device` current for the lifetime of the guard and gives the caller
// back the device that was current before, so that a host program driving
// several GPUs keeps its own current device across library calls.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); prev = -1; }
        if (prev != device) cudaSetDevice(device);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

struct Scope {
    ebe_handle* h;
    DeviceGuard dev;
    explicit Scope(ebe_handle* hh) : h(hh), dev(hh->device) { enter(h); }
    ~Scope() { leave(h); }
};

int add_launches(ebe_handle* h, int n) {
    h->launches += n;
    return EBE_OK;
}

int check_ready(ebe_handle* h, bool need_assembled) {
    if (!h) return EBE_INVALID_ARG;
    if (!h->problem_set) return fail(h, EBE_NOT_READY, "ebe_set_problem has not been called");
    if (need_assembled && !h->assembled) return fail(h, EBE_NOT_READY, "ebe_assemble has not been called");
    return EBE_OK;
}

// Reads the device error word on the handle's stream (synchronises it).  A
// wait that gave up is reported once: the word is cleared again, so the
// handle can run the next call (the results of this one are invalid).
int check_device(ebe_handle* h) {
    int32_t e = 0;
    CK(cudaMemcpyAsync(&e, h->dev_err, sizeof(e), cudaMemcpyDeviceToHost, h->st), "read device flag");
    CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    if (e != 0) {
        CK(cudaMemsetAsync(h->dev_err, 0, sizeof(int32_t), h->st), "clear device flag");
        CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
        return fail(h, EBE_CUDA_ERROR, e == 2 ? "a grid-wide barrier wait of the batched solver timed out"
                                              : "a device-side wait timed out (bulk copy did not complete)");
    }
    return EBE_OK;
}

int sync_scalars(ebe_handle* h) {
    CK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->st), "read scalars");
    return check_device(h);
}

}  // namespace

extern "C" {

const char* ebe_status_string(int s) {
    switch (s) {
        case EBE_OK: return "EBE_OK";
        case EBE_INVALID_ARG: return "EBE_INVALID_ARG";
        case EBE_INDEX_RANGE: return "EBE_INDEX_RANGE";
        case EBE_DEGENERATE_ELEMENT: return "EBE_DEGENERATE_ELEMENT";
        case EBE_SINGULAR: return "EBE_SINGULAR";
        case EBE_CUDA_ERROR: return "EBE_CUDA_ERROR";
        case EBE_OOM: return "EBE_OOM";
        case EBE_MAXIT: return "EBE_MAXIT";
        case EBE_BREAKDOWN: return "EBE_BREAKDOWN";
        case EBE_STALL: return "EBE_STALL";
        case EBE_NOT_READY: return "EBE_NOT_READY";
        default: return "EBE_UNKNOWN";
    }
}

const char* ebe_last_error(const ebe_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void ebe_solve_opts_default(ebe_solve_opts* o) {
    if (!o) return;
    o->rtol = 1e-8;
    o->maxit = 200000;
    o->precision = EBE_PREC_FP64;
    o->chunk = 32;
    o->delta = 0.1;
    o->stall_updates = 8;
    o->use_graph = 1;
    o->race_iters = -1;
}

void ebe_destroy(ebe_handle* h) {
    if (!h) return;
    DeviceGuard dev(h->device);
    if (h->st) cudaStreamSynchronize(h->st);
    for (int k = 0; k < 2; ++k) {
        if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
        if (h->cg_graph[k]) cudaGraphExecDestroy(h->cg_graph[k]);
    }
    if (h->bgraph) cudaGraphExecDestroy(h->bgraph);
    for (void* p : h->allocs) cudaFree(p);
    if (h->sc_host) cudaFreeHost(h->sc_host);
    if (h->bprob_host) cudaFreeHost(h->bprob_host);
    if (h->bcount_host) cudaFreeHost(h->bcount_host);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->own_stream && h->st) cudaStreamDestroy(h->st);
    delete h;
}

// Device side of ebe_create / ebe_create_batch, once h->plan and h->lay hold
// the partition.  coords: host [n_n][dim] in the union numbering.
static int create_device(ebe_handle* h, const double* coords_host) {
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (h->device < 0 || h->device >= ndev) return fail(h, EBE_INVALID_ARG, "no such CUDA device");
    DeviceGuard dev(h->device);
    CK(cudaDeviceGetAttribute(&h->pd.num_sms, cudaDevAttrMultiProcessorCount, h->device), "cudaDeviceGetAttribute");
    if (h->own_stream) CK(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking), "cudaStreamCreate");
    CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming), "cudaEventCreate");
    enter(h);
    HostPlan& P = h->plan;
    PlanDev& pd = h->pd;
    pd.nb = P.nb;
    pd.dim = P.dim;
    pd.n_slots = P.n_slots;
    pd.n_patches = int(P.n_patches);
    pd.n_shared = int(P.sh_node.size());
    pd.n_halo = P.n_halo;
    pd.max_nodes = P.max_nodes;
    pd.max_col = P.max_col;
    int32_t* col_ptr = nullptr;
    int32_t* sh_ptr = nullptr;
    int32_t* sh_slot = nullptr;
    int32_t* slot_elem = nullptr;
    uint16_t* lconn = nullptr;
    PatchMeta* meta = nullptr;
    TRY(upload(h, &h->coords, coords_host, P.n_n * P.dim));
    TRY(upload(h, &meta, P.meta.data(), int64_t(P.meta.size())));
    TRY(upload(h, &h->pnode, P.pnode.data(), int64_t(P.pnode.size())));
    TRY(upload(h, &lconn, P.lconn.data(), int64_t(P.lconn.size())));
    TRY(upload(h, &col_ptr, P.col_ptr.data(), int64_t(P.col_ptr.size())));
    TRY(upload(h, &h->sh_node, P.sh_node.data(), int64_t(P.sh_node.size())));
    TRY(upload(h, &sh_ptr, P.sh_ptr.data(), int64_t(P.sh_ptr.size())));
    TRY(upload(h, &sh_slot, P.sh_slot.data(), int64_t(P.sh_slot.size())));
    TRY(upload(h, &slot_elem, P.slot_elem.data(), int64_t(P.slot_elem.size())));
    h->n_pnode = int64_t(P.pnode.size());
    pd.meta = meta;
    pd.pnode = h->pnode;
    pd.lconn = lconn;
    pd.col_ptr = col_ptr;
    pd.sh_node = h->sh_node;
    pd.sh_ptr = sh_ptr;
    pd.sh_slot = sh_slot;
    pd.slot_elem = slot_elem;
    // Solver numbering for the single-sync mixed solver: the owned nodes of
    // each patch as one contiguous run in patch order (each run padded to a
    // multiple of 4 nodes), then the shared nodes in the order of the fix-up
    // rows.  The patch pass then reads and writes its owned nodes' vector
    // entries with coalesced accesses and the fix-up its shared rows.
    {
        const int64_t np = P.n_patches, nsh = int64_t(P.sh_node.size());
        std::vector<int32_t> own_off(size_t(np) + 1);
        int64_t off = 0;
        for (int64_t p = 0; p < np; ++p) {
            own_off[size_t(p)] = int32_t(off);
            off += (P.meta[size_t(p)].n_owned + 3) / 4 * 4;
        }
        own_off[size_t(np)] = int32_t(off);
        h->n_int = (off + nsh + 3) / 4 * 4;
        if (h->n_int >= (int64_t(1) << 31)) return fail(h, EBE_INVALID_ARG, "mesh too large for the solver numbering");
        std::vector<int32_t> iou(static_cast<size_t>(P.n_n), -1), pint(P.pnode.size()), shint(static_cast<size_t>(nsh));
        for (int64_t p = 0; p < np; ++p) {
            const PatchMeta& m = P.meta[size_t(p)];
            for (int l = 0; l < m.n_owned; ++l) iou[size_t(P.pnode[size_t(m.node_off + l)] & kNodeMask)] = own_off[size_t(p)] + l;
        }
        for (int64_t k = 0; k < nsh; ++k) {
            shint[size_t(k)] = int32_t(off + k);
            iou[size_t(P.sh_node[size_t(k)] & kNodeMask)] = int32_t(off + k);
        }
        for (size_t i = 0; i < pint.size(); ++i) pint[i] = iou[size_t(P.pnode[i] & kNodeMask)];
        int32_t* own_off_d = nullptr;
        TRY(upload(h, &own_off_d, own_off.data(), int64_t(own_off.size())));
        TRY(upload(h, &h->int_of_user, iou.data(), int64_t(iou.size())));
        TRY(upload(h, &h->pnode_int, pint.data(), int64_t(pint.size())));
        TRY(upload(h, &h->sh_node_int, shint.data(), int64_t(shint.size())));
        std::vector<int32_t> hpos(static_cast<size_t>(std::max<int64_t>(P.n_halo, 1)), 0);
        for (int64_t j = 0; j < P.n_halo; ++j) hpos[size_t(P.sh_slot[size_t(j)])] = int32_t(j);
        int32_t* hpos_d = nullptr;
        TRY(upload(h, &hpos_d, hpos.data(), int64_t(hpos.size())));
        h->pd_int = pd;
        h->pd_int.halo_pos = hpos_d;
        h->pd_int.pnode = h->pnode_int;
        h->pd_int.sh_node = h->sh_node_int;
        h->pd_int.own_off = own_off_d;
        h->pd_int.sh_base = int32_t(off);
        CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");   // the host tables go away
    }
    TRY(dalloc(h, &h->part_patch, P.n_patches + 1216));
    TRY(dalloc(h, &h->part_vec, 3 * 1216));   // up to three partial sums per block
    TRY(dalloc(h, &h->sc, 1, true));
    TRY(dalloc(h, &h->bad, 1));
    TRY(dalloc(h, &h->dev_err, 1, true));
    pd.err = h->dev_err;
    h->pd_int.err = h->dev_err;
    h->pd_int.num_sms = pd.num_sms;
    CK(cudaMallocHost(&h->sc_host, sizeof(Scalars)), "cudaMallocHost");
    std::memset(h->sc_host, 0, sizeof(Scalars));
    CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");  // host arrays may go away now
    leave(h);
    return EBE_OK;
}

static int check_create_opts(ebe_handle* h, const ebe_create_opts* opts) {
    if (opts && opts->patch_elems != 0 && opts->patch_elems != kPatch)
        return fail(h, EBE_INVALID_ARG, "patch_elems must be 0 or 1024");
    return EBE_OK;
}

static int create_impl(ebe_handle* h, const ebe_mesh* m, const ebe_create_opts* opts) {
    TRY(check_create_opts(h, opts));
    // host-side validation and partition first: no device work for a bad mesh
    std::string err;
    int s = build_plan(*m, h->plan, err);
    if (s != EBE_OK) return fail(h, s, err);
    h->n_prob = 1;
    h->lay.node_off = {0, h->plan.n_n};
    h->lay.elem_off = {0, h->plan.n_e};
    h->lay.patch_off = {0, int32_t(h->plan.n_patches)};
    h->lay.shared_off = {0, int32_t(h->plan.sh_node.size())};
    return create_device(h, m->coords);
}

static int create_batch_impl(ebe_handle* h, const ebe_mesh* meshes, int n_prob, const ebe_create_opts* opts) {
    TRY(check_create_opts(h, opts));
    if (n_prob < 1 || n_prob > kBatchMaxProblems)
        return fail(h, EBE_INVALID_ARG, "n_problems must be in [1, " + std::to_string(kBatchMaxProblems) + "]");
    for (int k = 0; k < n_prob; ++k)
        if (!meshes[k].coords || !meshes[k].elems)
            return fail(h, EBE_INVALID_ARG, "problem " + std::to_string(k) + ": coords and elems must be non-NULL");
    std::string err;
    const int threads = host_threads(32);
    int s = build_batch_plan(meshes, n_prob, threads, h->plan, h->lay, err);
    if (s != EBE_OK) return fail(h, s, err);
    h->n_prob = n_prob;
    const int dim = h->plan.dim;
    std::vector<double> coords(size_t(h->plan.n_n) * size_t(dim));
    for (int k = 0; k < n_prob; ++k)
        std::copy(meshes[k].coords, meshes[k].coords + meshes[k].n_n * dim, coords.begin() + h->lay.node_off[k] * dim);
    return create_device(h, coords.data());
}

ebe_status ebe_create(ebe_handle** out, const ebe_mesh* m, const ebe_create_opts* opts, void* cuda_stream) {
    if (!out || !m) { g_create_error = "out and mesh must be non-NULL"; return EBE_INVALID_ARG; }
    *out = nullptr;
    ebe_handle* h = new (std::nothrow) ebe_handle();
    if (!h) { g_create_error = "host allocation failed"; return EBE_OOM; }
    h->device = opts ? opts->device : 0;
    h->user = static_cast<cudaStream_t>(cuda_stream);
    if (cuda_stream == nullptr) h->own_stream = true;   // legacy default stream: work on a private stream
    else h->st = static_cast<cudaStream_t>(cuda_stream);
    int s = create_impl(h, m, opts);
    if (s != EBE_OK) {
        g_create_error = h->err;
        ebe_destroy(h);
        return ebe_status(s);
    }
    *out = h;
    return EBE_OK;
}

ebe_status ebe_create_batch(ebe_handle** out, const ebe_mesh* meshes, int32_t n_problems, const ebe_create_opts* opts,
                            void* cuda_stream) {
    if (!out || !meshes) { g_create_error = "out and meshes must be non-NULL"; return EBE_INVALID_ARG; }
    *out = nullptr;
    ebe_handle* h = new (std::nothrow) ebe_handle();
    if (!h) { g_create_error = "host allocation failed"; return EBE_OOM; }
    h->device = opts ? opts->device : 0;
    h->user = static_cast<cudaStream_t>(cuda_stream);
    if (cuda_stream == nullptr) h->own_stream = true;
    else h->st = static_cast<cudaStream_t>(cuda_stream);
    int s = create_batch_impl(h, meshes, n_problems, opts);
    if (s != EBE_OK) {
        g_create_error = h->err;
        ebe_destroy(h);
        return ebe_status(s);
    }
    *out = h;
    return EBE_OK;
}

ebe_status ebe_batch_layout(const ebe_handle* h, int32_t* n_problems, int64_t* node_off, int64_t* elem_off) {
    if (!h) return EBE_INVALID_ARG;
    if (n_problems) *n_problems = h->n_prob;
    if (node_off) std::copy(h->lay.node_off.begin(), h->lay.node_off.end(), node_off);
    if (elem_off) std::copy(h->lay.elem_off.begin(), h->lay.elem_off.end(), elem_off);
    return EBE_OK;
}

// nu: one value per problem.
static int set_problem_impl(ebe_handle* h, const double* nu, const double* f_nodal, const int32_t* dirichlet,
                            int64_t n_d, const double* g, const int32_t* neumann, int64_t n_neu) {
    const int64_t n_n = h->plan.n_n;
    for (int k = 0; k < h->n_prob; ++k)
        if (!std::isfinite(nu[k]) || nu[k] < 0.0)
            return fail(h, EBE_INVALID_ARG, h->n_prob == 1 ? std::string("nu must be finite and >= 0")
                                                           : "nu of problem " + std::to_string(k) + " must be finite and >= 0");
    if (!f_nodal) return fail(h, EBE_INVALID_ARG, "f_nodal must be non-NULL");
    if (n_d < 0 || n_neu < 0 || (n_d > 0 && !dirichlet) || (n_neu > 0 && !neumann))
        return fail(h, EBE_INVALID_ARG, "bad boundary node set");
    for (int64_t k = 0; k < n_n; ++k)
        if (!std::isfinite(f_nodal[k])) return fail(h, EBE_INVALID_ARG, "f is not finite at node " + std::to_string(k));
    std::vector<uint8_t> mask(n_n, 0);
    for (int64_t k = 0; k < n_d; ++k) {
        int32_t v = dirichlet[k];
        if (v < 0 || v >= n_n) return fail(h, EBE_INDEX_RANGE, "Dirichlet node id out of range");
        if (mask[v]) return fail(h, EBE_INVALID_ARG, "Dirichlet node listed twice: " + std::to_string(v));
        mask[v] = 1;
        if (g && !std::isfinite(g[k])) return fail(h, EBE_INVALID_ARG, "g is not finite");
    }
    for (int64_t k = 0; k < n_neu; ++k) {
        int32_t v = neumann[k];
        if (v < 0 || v >= n_n) return fail(h, EBE_INDEX_RANGE, "Neumann node id out of range");
        if (mask[v]) return fail(h, EBE_INVALID_ARG, "node in both the Dirichlet and the Neumann set: " + std::to_string(v));
    }
    for (int k = 0; k < h->n_prob; ++k) {
        if (nu[k] != 0.0) continue;
        const auto lo = mask.begin() + h->lay.node_off[k], hi = mask.begin() + h->lay.node_off[k + 1];
        if (std::find(lo, hi, uint8_t(1)) == hi)
            return fail(h, EBE_SINGULAR, std::string("nu = 0 needs a Dirichlet boundary of positive measure (Sec. 1)") +
                                             (h->n_prob > 1 ? ": problem " + std::to_string(k) : std::string()));
    }
    Scope scp(h);
    std::vector<double> gv(n_d, 0.0);
    if (g) std::copy(g, g + n_d, gv.begin());
    if (h->nd && h->n_d < n_d) { /* grow: old buffer stays allocated until destroy */ h->nd = nullptr; h->g = nullptr; }
    TRY(upload(h, &h->f, f_nodal, n_n));
    TRY(dalloc(h, &h->nd, std::max<int64_t>(n_d, 1)));
    TRY(dalloc(h, &h->g, std::max<int64_t>(n_d, 1)));
    if (n_d > 0) {
        CK(cudaMemcpyAsync(h->nd, dirichlet, sizeof(int32_t) * n_d, cudaMemcpyHostToDevice, h->st), "upload");
        CK(cudaMemcpyAsync(h->g, gv.data(), sizeof(double) * n_d, cudaMemcpyHostToDevice, h->st), "upload");
    }
    TRY(upload(h, &h->dmask, mask.data(), n_n));
    std::vector<double> nup;
    if (h->n_prob > 1) {
        nup.resize(size_t(h->plan.n_patches));
        for (int k = 0; k < h->n_prob; ++k)
            std::fill(nup.begin() + h->lay.patch_off[k], nup.begin() + h->lay.patch_off[k + 1], nu[k]);
        TRY(dalloc(h, &h->nu_patch, int64_t(nup.size())));
        CK(cudaMemcpyAsync(h->nu_patch, nup.data(), sizeof(double) * nup.size(), cudaMemcpyHostToDevice, h->st), "upload");
    }
    int l = 0;
    CK(launch_mark_dirichlet(h->pd, h->pnode, h->n_pnode, h->sh_node, h->dmask, h->st, &l), "mark Dirichlet");
    CK(launch_copy_dirichlet_bit(h->pnode_int, h->pnode, h->n_pnode, h->st, &l), "mark Dirichlet");
    CK(launch_copy_dirichlet_bit(h->sh_node_int, h->sh_node, h->pd.n_shared, h->st, &l), "mark Dirichlet");
    add_launches(h, l);
    CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    h->nu = nu[0];
    h->n_d = n_d;
    h->problem_set = true;
    h->assembled = false;
    return EBE_OK;
}

ebe_status ebe_set_problem(ebe_handle* h, double nu, const double* f_nodal, const int32_t* dirichlet, int64_t n_d,
                           const double* g, const int32_t* neumann, int64_t n_neu) {
    if (!h) return EBE_INVALID_ARG;
    const std::vector<double> nus(size_t(h->n_prob), nu);
    return ebe_status(set_problem_impl(h, nus.data(), f_nodal, dirichlet, n_d, g, neumann, n_neu));
}

ebe_status ebe_set_problem_batch(ebe_handle* h, const double* nu, const double* f_nodal, const int32_t* dirichlet,
                                 int64_t n_d, const double* g, const int32_t* neumann, int64_t n_neu) {
    if (!h) return EBE_INVALID_ARG;
    if (!nu) return ebe_status(fail(h, EBE_INVALID_ARG, "nu must be non-NULL (one value per problem)"));
    return ebe_status(set_problem_impl(h, nu, f_nodal, dirichlet, n_d, g, neumann, n_neu));
}

ebe_status ebe_assemble(ebe_handle* h, int32_t store) {
    TRY(check_ready(h, false));
    if (store != EBE_STORE_FP64 && store != EBE_STORE_MIXED) return ebe_status(fail(h, EBE_INVALID_ARG, "bad store"));
    Scope scp(h);
    const int64_t n_n = h->plan.n_n, nbb = sym_count(h->pd.nb);
    TRY(dalloc(h, &h->A64, nbb * h->pd.n_slots, true));
    TRY(dalloc(h, &h->b, n_n));
    TRY(dalloc(h, &h->d, n_n));
    TRY(dalloc(h, &h->dinv, n_n));
    TRY(dalloc(h, &h->halo2, 2 * std::max<int64_t>(h->plan.n_halo, 1)));
    float *A32 = nullptr, *b32 = nullptr, *dinv32 = nullptr;
    if (store == EBE_STORE_MIXED) {
        TRY(dalloc(h, &h->A32, nbb * h->pd.n_slots, true));
        TRY(dalloc(h, &h->b32, n_n));
        TRY(dalloc(h, &h->dinv32, n_n));
        A32 = h->A32; b32 = h->b32; dinv32 = h->dinv32;
    }
    CK(cudaMemsetAsync(h->bad, 0xff, sizeof(unsigned long long), h->st), "memset");
    int l = 0;
    CK(launch_assemble(h->pd, h->coords, h->f, h->nu, h->nu_patch, h->A64, A32, h->b, h->d, h->dinv, b32, dinv32, h->halo2,
                       h->bad, h->st, &l), "assemble");
    add_launches(h, l);
    unsigned long long bad = 0;
    CK(cudaMemcpyAsync(&bad, h->bad, sizeof(bad), cudaMemcpyDeviceToHost, h->st), "read flag");
    CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    if (bad != ~0ull) {
        h->assembled = false;
        return ebe_status(fail(h, EBE_DEGENERATE_ELEMENT, "element " + std::to_string(bad) + " has zero measure"));
    }
    h->store = store;
    h->assembled = true;
    h->int_ready = false;
    h->dw_ready = false;
    return EBE_OK;
}

ebe_status ebe_element_matrices(ebe_handle* h, double* K, double* M) {
    if (!h) return EBE_INVALID_ARG;
    Scope scp(h);
    int l = 0;
    CK(launch_export_km(h->pd, h->coords, K, M, h->st, &l), "export K_e, M_e");
    add_launches(h, l);
    return EBE_OK;
}

ebe_status ebe_get_local_matrices(ebe_handle* h, void* A, int32_t dtype) {
    TRY(check_ready(h, true));
    if (!A || (dtype != EBE_F64 && dtype != EBE_F32)) return ebe_status(fail(h, EBE_INVALID_ARG, "bad arguments"));
    if (dtype == EBE_F32 && h->store != EBE_STORE_MIXED) return ebe_status(fail(h, EBE_NOT_READY, "FP32 matrices need EBE_STORE_MIXED"));
    Scope scp(h);
    int l = 0;
    CK(launch_export_A(h->pd, dtype, dtype == EBE_F64 ? static_cast<const void*>(h->A64) : h->A32, A, h->st, &l),
       "export A_e");
    add_launches(h, l);
    return EBE_OK;
}

ebe_status ebe_get_rhs(ebe_handle* h, double* b) {
    TRY(check_ready(h, true));
    if (!b) return ebe_status(fail(h, EBE_INVALID_ARG, "b is NULL"));
    Scope scp(h);
    CK(cudaMemcpyAsync(b, h->b, sizeof(double) * h->plan.n_n, cudaMemcpyDeviceToDevice, h->st), "copy b");
    return EBE_OK;
}

ebe_status ebe_jacobi_diag(ebe_handle* h, double* d) {
    TRY(check_ready(h, true));
    if (!d) return ebe_status(fail(h, EBE_INVALID_ARG, "d is NULL"));
    Scope scp(h);
    CK(cudaMemcpyAsync(d, h->d, sizeof(double) * h->plan.n_n, cudaMemcpyDeviceToDevice, h->st), "copy d");
    return EBE_OK;
}

// The element matrices as FP32 pairs (the double-word residual), once per assembly.
static int ensure_dw(ebe_handle* h) {
    const int64_t n = int64_t(sym_count(h->pd.nb)) * h->pd.n_slots;
    TRY(dalloc(h, &h->Adw, 2 * n));
    if (h->dw_ready) return EBE_OK;
    int l = 0;
    CK(launch_split_dw(n, h->A64, h->Adw, h->pd.nb, h->st, &l), "split A_e");
    add_launches(h, l);
    h->dw_ready = true;
    return EBE_OK;
}

static int patch_call(ebe_handle* h, const void* x, void* y, int32_t dtype, int mode) {
    TRY(check_ready(h, true));
    if (!x || !y || x == y) return fail(h, EBE_INVALID_ARG, "x and y must be distinct non-NULL device buffers");
    if (dtype != EBE_F64 && dtype != EBE_F32 && dtype != EBE_F64_DW)
        return fail(h, EBE_INVALID_ARG, "dtype must be EBE_F64, EBE_F32 or EBE_F64_DW");
    if (dtype == EBE_F32 && h->store != EBE_STORE_MIXED) return fail(h, EBE_NOT_READY, "EBE_F32 needs ebe_assemble(EBE_STORE_MIXED)");
    Scope scp(h);
    if (dtype == EBE_F64_DW) {
        TRY(dalloc(h, &h->halo64, std::max<int64_t>(h->plan.n_halo, 1)));
        TRY(ensure_dw(h));
        int l = 0;
        CK(launch_patch_pass_dw(h->pd, mode, h->Adw, static_cast<const double*>(x), h->b,
                                static_cast<double*>(y), h->halo64, h->part_patch, nullptr, h->sc, h->st, &l),
           "double-word patch pass");
        add_launches(h, l);
        return EBE_OK;
    }
    void* halo;
    if (dtype == EBE_F64) {
        TRY(dalloc(h, &h->halo64, std::max<int64_t>(h->plan.n_halo, 1)));
        halo = h->halo64;
    } else {
        TRY(dalloc(h, &h->halo32, std::max<int64_t>(h->plan.n_halo, 1)));
        halo = h->halo32;
    }
    const void* A = dtype == EBE_F64 ? static_cast<const void*>(h->A64) : h->A32;
    const void* b = dtype == EBE_F64 ? static_cast<const void*>(h->b) : h->b32;
    int l = 0;
    CK(launch_patch_pass(h->pd, dtype, mode, A, x, b, y, halo, h->part_patch, nullptr, h->sc, h->st, &l), "patch pass");
    add_launches(h, l);
    return EBE_OK;
}

ebe_status ebe_residual(ebe_handle* h, const void* x, void* r, int32_t dtype) {
    return ebe_status(patch_call(h, x, r, dtype, kResidual));
}

ebe_status ebe_apply(ebe_handle* h, const void* x, void* y, int32_t dtype) {
    return ebe_status(patch_call(h, x, y, dtype, kApply));
}

ebe_status ebe_time_operator(ebe_handle* h, const void* x, void* y, int32_t dtype, int32_t apply, int32_t reps,
                             double* ms) {
    if (!ms || reps < 1 || reps > 100000) return ebe_status(fail(h, EBE_INVALID_ARG, "ms must be non-NULL, 1 <= reps <= 100000"));
    // argument checks and scratch allocation as a plain call; also a warm-up launch
    TRY(patch_call(h, x, y, dtype, apply ? kApply : kResidual));
    Scope scp(h);
    std::vector<cudaEvent_t> ev(size_t(3) * reps, nullptr);
    for (auto& e : ev) CK(cudaEventCreate(&e), "cudaEventCreate");
    const void* A = dtype == EBE_F64 ? static_cast<const void*>(h->A64) : h->A32;
    const void* b = dtype == EBE_F64 ? static_cast<const void*>(h->b) : h->b32;
    void* halo = dtype == EBE_F64 ? static_cast<void*>(h->halo64) : h->halo32;
    int l = 0;
    int status = EBE_OK;
    for (int r = 0; r < reps && status == EBE_OK; ++r) {
        cudaError_t e =
            dtype == EBE_F64_DW
                ? launch_patch_pass_dw(h->pd, apply ? kApply : kResidual, h->Adw,
                                       static_cast<const double*>(x), h->b, static_cast<double*>(y), h->halo64,
                                       h->part_patch, nullptr, h->sc, h->st, &l, &ev[size_t(3) * r])
                : launch_patch_pass(h->pd, dtype, apply ? kApply : kResidual, A, x, b, y, halo, h->part_patch, nullptr,
                                    h->sc, h->st, &l, &ev[size_t(3) * r]);
        if (e != cudaSuccess) status = cuda_fail(h, e, "timed patch pass");
    }
    add_launches(h, l);
    double t_patch = 0.0, t_fix = 0.0;
    if (status == EBE_OK) {
        cudaError_t e = cudaEventSynchronize(ev.back());
        if (e != cudaSuccess) status = cuda_fail(h, e, "cudaEventSynchronize");
        for (int r = 0; r < reps && status == EBE_OK; ++r) {
            float a = 0.f, c = 0.f;
            cudaEventElapsedTime(&a, ev[3 * r], ev[3 * r + 1]);
            cudaEventElapsedTime(&c, ev[3 * r + 1], ev[3 * r + 2]);
            t_patch += a;
            t_fix += c;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (status != EBE_OK) return ebe_status(status);
    ms[0] = t_patch / reps;
    ms[1] = t_fix / reps;
    return EBE_OK;
}

static int ensure_gconn(ebe_handle* h) {
    if (h->gconn) return EBE_OK;
    TRY(dalloc(h, &h->gconn, int64_t(h->pd.nb) * h->pd.n_slots));
    int l = 0;
    CK(launch_build_gconn(h->pd, h->gconn, h->st, &l), "build connectivity");
    add_launches(h, l);
    const HostPlan& P = h->plan;
    h->gconn_host.assign(size_t(P.n_slots) * P.nb, 0);
    for (int64_t s = 0; s < P.n_slots; ++s) {
        if (P.slot_elem[s] < 0) continue;
        const PatchMeta& m = P.meta[s / kPatch];
        for (int i = 0; i < P.nb; ++i) h->gconn_host[s * P.nb + i] = P.pnode[m.node_off + P.lconn[size_t(i) * P.n_slots + s]];
    }
    return EBE_OK;
}

ebe_status ebe_residual_variant(ebe_handle* h, const double* x, double* r, int32_t scatter) {
    if (scatter == EBE_SCATTER_PATCH) return ebe_residual(h, x, r, EBE_F64);
    TRY(check_ready(h, true));
    if (!x || !r || x == r) return ebe_status(fail(h, EBE_INVALID_ARG, "x and r must be distinct non-NULL device buffers"));
    Scope scp(h);
    TRY(ensure_gconn(h));
    const HostPlan& P = h->plan;
    int l = 0;
    if (scatter == EBE_SCATTER_ATOMIC) {
        CK(launch_residual_atomic(h->pd, h->A64, h->gconn, x, h->b, h->dmask, P.n_n, r, h->st, &l), "atomic residual");
    } else if (scatter == EBE_SCATTER_NODE) {
        if (!h->node_ptr) {
            std::vector<int32_t> ptr(P.n_n + 1, 0), ent(size_t(P.n_e) * P.nb);
            for (int64_t s = 0; s < P.n_slots; ++s)
                if (P.slot_elem[s] >= 0)
                    for (int i = 0; i < P.nb; ++i) ++ptr[h->gconn_host[s * P.nb + i] + 1];
            for (int64_t k = 0; k < P.n_n; ++k) ptr[k + 1] += ptr[k];
            std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
            for (int64_t s = 0; s < P.n_slots; ++s)
                if (P.slot_elem[s] >= 0)
                    for (int i = 0; i < P.nb; ++i)
                        ent[fill[h->gconn_host[s * P.nb + i]]++] = int32_t(int64_t(i) * P.n_slots + s);
            TRY(upload(h, &h->node_ptr, ptr.data(), int64_t(ptr.size())));
            TRY(upload(h, &h->node_ent, ent.data(), int64_t(ent.size())));
            TRY(dalloc(h, &h->Y, int64_t(P.nb) * P.n_slots));
            CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
        }
        CK(launch_residual_node(h->pd, h->A64, h->gconn, h->node_ptr, h->node_ent, x, h->b, h->dmask, P.n_n, h->Y, r,
                                h->st, &l), "node residual");
    } else if (scatter == EBE_SCATTER_COLOUR) {
        if (!h->Acol) {
            std::vector<int32_t> order;
            std::string err;
            int nc = global_colouring(P, h->gconn_host, order, h->col_ptr, err);
            if (nc < 0) return ebe_status(fail(h, EBE_INVALID_ARG, err));
            h->n_gcol = nc;
            int32_t* order_d = nullptr;
            TRY(upload(h, &order_d, order.data(), int64_t(order.size())));
            TRY(dalloc(h, &h->Acol, int64_t(sym_count(P.nb)) * P.n_e));
            TRY(dalloc(h, &h->gcol, int64_t(P.nb) * P.n_e));
            CK(launch_permute_slots(P.nb, P.n_slots, P.n_e, order_d, h->A64, h->gconn, h->Acol, h->gcol, h->st, &l),
               "permute");
            CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
        }
        CK(launch_residual_colour(P.nb, h->n_gcol, h->col_ptr.data(), P.n_e, h->Acol, h->gcol, x, h->b, h->dmask, P.n_n,
                                  r, h->st, &l), "colour residual");
    } else {
        return ebe_status(fail(h, EBE_INVALID_ARG, "unknown scatter"));
    }
    add_launches(h, l);
    return EBE_OK;
}

// ---------------------------------------------------------------- solver

namespace {

struct SolveBufs {
    int dt;        // type of A, p, q and the recurrence residual r: 0 = FP64, 1 = FP32
    void* p;
    void* q;
    void* r;       // recurrence residual (r64 itself for FP64)
    const void* A;
    const void* dinv;  // FP64 (plain) or FP32 (mixed) inverse Jacobi diagonal
    void* halo;
};

SolveBufs bufs_for(ebe_handle* h, bool mixed) {
    SolveBufs s;
    s.dt = mixed ? 1 : 0;
    if (mixed) {
        s.p = h->p32; s.q = h->q32; s.r = h->r32; s.A = h->A32; s.dinv = h->dinv32; s.halo = h->halo32;
    } else {
        s.p = h->p64; s.q = h->q64; s.r = h->r64; s.A = h->A64; s.dinv = h->dinv; s.halo = h->halo64;
    }
    return s;
}

// One CG iteration: q = mask(A p) and p.q (alpha), update (stop test), direction.
// x is FP64 in both precisions.
int enqueue_iteration(ebe_handle* h, const SolveBufs& s, int* l) {
    const int64_t n = h->plan.n_n;
    CK(launch_patch_pass(h->pd, s.dt, kApplyDot, s.A, s.p, nullptr, s.q, s.halo, h->part_patch, &h->sc->done, h->sc,
                         h->st, l, nullptr, true),
       "apply");
    CK(launch_update(s.dt, n, h->x64w, s.p, s.r, s.q, s.dinv, h->part_vec, h->sc, h->st, l), "update");
    CK(launch_direction(s.dt, n, s.p, s.r, s.dinv, 0, h->sc, h->st, l), "direction");
    return EBE_OK;
}

int ensure_graph(ebe_handle* h, bool mixed, int chunk) {
    const int k = mixed ? 1 : 0;
    if (h->graph[k] && h->graph_chunk[k] == chunk) return EBE_OK;
    if (h->graph[k]) { cudaGraphExecDestroy(h->graph[k]); h->graph[k] = nullptr; }
    const SolveBufs s = bufs_for(h, mixed);
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    int l = 0, st = EBE_OK;
    for (int it = 0; it < chunk && st == EBE_OK; ++it) st = enqueue_iteration(h, s, &l);
    cudaError_t e = cudaStreamEndCapture(h->st, &g);
    if (st != EBE_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph[k], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { h->graph[k] = nullptr; return cuda_fail(h, e, "cudaGraphInstantiate"); }
    h->graph_chunk[k] = chunk;
    h->graph_nodes[k] = l;
    return EBE_OK;
}

// r64 = mask(b - A64 x64w) and its squared norm (FP64 element matrices).
int true_residual(ebe_handle* h, double& rr) {
    int l = 0;
    CK(launch_patch_pass(h->pd, 0, kResidualNorm, h->A64, h->x64w, h->b, h->r64, h->halo64, h->part_patch, nullptr, h->sc,
                         h->st, &l), "true residual");
    add_launches(h, l);
    TRY(sync_scalars(h));
    rr = h->sc_host->rrt;
    return EBE_OK;
}

// Jacobi-PCG in the textbook form (four launches per iteration: operator
// pass, fix-up, update, direction).  The solution x is FP64 in both
// precisions.  EBE_PREC_MIXED_TEXTBOOK
// keeps the recurrence residual r, z = dinv r, the search direction p,
// q = A p and the element matrices in FP32 (difference form), so the passes
// stream about half the bytes and the FP64 pipe only updates x; FP32
// rounding makes the recurrence residual drift from the true one, so
// whenever the recurrence residual has dropped by `delta` since the last
// FP64 true residual, r is replaced by a fresh FP64 true residual (FP64
// element matrices) and CG continues with the same direction.
int solve_impl(ebe_handle* h, double* x, bool x_on_host, const ebe_solve_opts& o, ebe_solve_info& info) {
    const auto t0 = std::chrono::steady_clock::now();
    const bool mixed = o.precision == EBE_PREC_MIXED_TEXTBOOK;
    if (mixed && h->store != EBE_STORE_MIXED) return fail(h, EBE_NOT_READY, "mixed precision needs ebe_assemble(EBE_STORE_MIXED)");
    const int64_t n = h->plan.n_n;
    const int64_t nh = std::max<int64_t>(h->plan.n_halo, 1);
    TRY(dalloc(h, &h->x64w, n));
    TRY(dalloc(h, &h->r64, n));
    TRY(dalloc(h, &h->halo64, nh));
    if (mixed) {
        TRY(dalloc(h, &h->p32, n));
        TRY(dalloc(h, &h->q32, n));
        TRY(dalloc(h, &h->r32, n));
        TRY(dalloc(h, &h->halo32, nh));
    } else {
        TRY(dalloc(h, &h->p64, n));
        TRY(dalloc(h, &h->q64, n));
    }
    const SolveBufs s = bufs_for(h, mixed);
    int l = 0;
    CK(cudaMemcpyAsync(h->x64w, x, sizeof(double) * n, x_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       h->st), "copy x0");
    CK(launch_set_dirichlet(h->x64w, h->nd, h->g, h->n_d, h->st, &l), "x(nd) = g");
    CK(launch_control(h->sc, 0.0, o.maxit, 1, h->st, &l), "control");
    add_launches(h, l);
    double rr = 0.0;
    TRY(true_residual(h, rr));
    info.true_residuals = 1;
    const double r0 = std::sqrt(rr);
    info.r0_norm = r0;
    info.iterations = 0;
    info.rel_residual = r0 > 0.0 ? 1.0 : 0.0;
    int status = EBE_OK;
    if (!std::isfinite(r0)) status = EBE_BREAKDOWN;
    if (r0 > 0.0 && std::isfinite(r0)) {
        const double target = o.rtol * r0;
        // The true residual is checked once the recurrence residual reaches
        // rtol (a textbook stopping test); mixed precision also replaces r
        // whenever the recurrence has dropped by delta.  In mixed precision a
        // failed check at the final threshold (the FP32 recurrence drifted
        // below the true residual) tightens that threshold by kFinalMargin;
        // the 2-norm residual of CG falls in steps, so a fixed margin below
        // rtol from the start would cost whole steps of iterations.  The
        // FP64 recurrence tracks the true residual, and its threshold stays.
        double fin = target;
        l = 0;
        CK(launch_restart(s.dt, n, h->r64, s.dinv, 1, h->part_vec, h->sc, h->st, &l, h->r32), "restart");
        CK(launch_direction(s.dt, n, s.p, s.r, s.dinv, 1, h->sc, h->st, &l), "direction");
        double thr = mixed ? std::max(o.delta * r0, fin) : fin;
        CK(launch_control(h->sc, thr * thr, -1, 0, h->st, &l), "control");
        add_launches(h, l);
        if (o.use_graph) TRY(ensure_graph(h, mixed, o.chunk));
        double best = 1.0;
        int no_progress = 0;
        for (;;) {
            if (o.use_graph) {
                CK(cudaGraphLaunch(h->graph[mixed ? 1 : 0], h->st), "cudaGraphLaunch");
                add_launches(h, h->graph_nodes[mixed ? 1 : 0]);
            } else {
                l = 0;
                for (int it = 0; it < o.chunk; ++it) TRY(enqueue_iteration(h, s, &l));
                add_launches(h, l);
            }
            const int64_t before = info.iterations;
            TRY(sync_scalars(h));
            const Scalars sh = *h->sc_host;
            info.iterations = sh.iter;
            if (sh.reason == kRunning) {
                if (sh.iter == before) return fail(h, EBE_CUDA_ERROR, "solver chunk made no progress");
                continue;
            }
            if (sh.reason == kBreakdown) { status = EBE_BREAKDOWN; break; }
            TRY(true_residual(h, rr));
            info.true_residuals += 1;
            const double rel = std::sqrt(rr) / r0;
            info.rel_residual = rel;
            if (!std::isfinite(rel)) { status = EBE_BREAKDOWN; break; }
            if (rel <= o.rtol) { status = EBE_OK; break; }
            if (sh.reason == kMaxit) { status = EBE_MAXIT; break; }
            if (rel < 0.9 * best) { best = rel; no_progress = 0; }
            else if (++no_progress >= o.stall_updates) { status = EBE_STALL; break; }
            if (mixed && sh.reason == kTrigger && thr <= fin) fin *= kFinalMargin;
            // residual replacement: r64 already holds the FP64 true residual;
            // continue CG from it with the same direction
            l = 0;
            CK(launch_restart(s.dt, n, h->r64, s.dinv, 0, h->part_vec, h->sc, h->st, &l, h->r32), "restart");
            CK(launch_direction(s.dt, n, s.p, s.r, s.dinv, 0, h->sc, h->st, &l), "direction");
            thr = mixed ? std::max(o.delta * std::sqrt(rr), fin) : fin;
            CK(launch_control(h->sc, thr * thr, -1, 0, h->st, &l), "control");
            add_launches(h, l);
        }
        if (status == EBE_BREAKDOWN) {
            // report the true residual of the iterate reached
            if (true_residual(h, rr) == EBE_OK) info.rel_residual = std::sqrt(rr) / r0;
        }
    }
    CK(cudaMemcpyAsync(x, h->x64w, sizeof(double) * n, x_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                       h->st), "copy x");
    CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    info.status = status;
    info.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (status != EBE_OK) {
        const char* why = status == EBE_MAXIT ? "maxit reached" : status == EBE_STALL ? "true residual stalled"
                                                                                        : "breakdown (p.Ap <= 0 or non-finite)";
        h->err = std::string("solve stopped: ") + why;
    }
    return status;
}

// ------------------------------------------------ single-synchronisation mixed solver
// Jacobi-PCG with the search direction, q = A p, the recurrence residual and
// the FP32 element matrices as in the textbook mixed solver, but one
// iteration is one launch_cg_pass (patch pass + fix-up): the x, r updates and
// the new direction are formed where the next operator pass gathers its
// operand, and beta comes from the expansion of r'.(dinv r') in sums that
// pass forms, so each iteration has one grid-wide reduction.  Vectors live
// in the solver numbering (owned nodes of a patch contiguous); x is permuted
// in and out once per solve.  The direction alternates between two buffers
// (a pass reads one and writes the other), so that after a residual
// replacement CG continues from the previous direction exactly as the
// textbook solver does.

// b and dinv in the solver numbering, once per assembly.
int ensure_solver_vectors(ebe_handle* h) {
    const int64_t n = h->plan.n_n, ni = h->n_int;
    TRY(dalloc(h, &h->bi, ni, true));
    TRY(dalloc(h, &h->dinvi32, ni, true));
    if (h->int_ready) return EBE_OK;
    int l = 0;
    CK(launch_permute(0, 1, n, h->int_of_user, h->b, h->bi, h->st, &l), "b to the solver numbering");
    CK(launch_permute(1, 1, n, h->int_of_user, h->dinv32, h->dinvi32, h->st, &l), "dinv to the solver numbering");
    add_launches(h, l);
    h->int_ready = true;
    return EBE_OK;
}

int ensure_cg_graphs(ebe_handle* h, int chunk) {
    if (h->cg_graph[0] && h->cg_graph[1] && h->cg_chunk == chunk) return EBE_OK;
    for (int k = 0; k < 2; ++k)
        if (h->cg_graph[k]) { cudaGraphExecDestroy(h->cg_graph[k]); h->cg_graph[k] = nullptr; }
    for (int par = 0; par < 2; ++par) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        int l = 0;
        cudaError_t e = cudaSuccess;
        for (int it = 0; it < chunk && e == cudaSuccess; ++it)
            e = launch_cg_pass(h->pd_int, h->A32, h->ri32, h->qi32, h->pi32[(par + it) & 1], h->pi32[(par + it + 1) & 1],
                               h->dinvi32, h->xi, h->halo32, h->part5, h->sc, h->st, &l, true);
        cudaError_t e2 = cudaStreamEndCapture(h->st, &g);
        if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(h, e, "single-sync pass"); }
        if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&h->cg_graph[par], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { h->cg_graph[par] = nullptr; return cuda_fail(h, e, "cudaGraphInstantiate"); }
        h->cg_nodes = l;
    }
    h->cg_chunk = chunk;
    return EBE_OK;
}

// r = mask(b - A64 x) in the solver numbering and its squared norm: the FP64
// pass, or (dw) the same residual in double-word arithmetic on the FP32 pipe.
int true_residual_int(ebe_handle* h, double& rr, bool dw = false) {
    int l = 0;
    if (dw) {
        TRY(ensure_dw(h));
        CK(launch_patch_pass_dw(h->pd_int, kResidualNorm, h->Adw, h->xi, h->bi, h->ri64, h->halo64,
                                h->part_patch, nullptr, h->sc, h->st, &l), "double-word true residual");
    } else {
        CK(launch_patch_pass(h->pd_int, 0, kResidualNorm, h->A64, h->xi, h->bi, h->ri64, h->halo64, h->part_patch,
                             nullptr, h->sc, h->st, &l), "true residual");
    }
    add_launches(h, l);
    TRY(sync_scalars(h));
    rr = h->sc_host->rrt;
    return EBE_OK;
}

// Work vectors of the single-sync solver (solver numbering).
int cg1_buffers(ebe_handle* h) {
    if (h->store != EBE_STORE_MIXED) return fail(h, EBE_NOT_READY, "EBE_PREC_MIXED needs ebe_assemble(EBE_STORE_MIXED)");
    const int64_t n = h->plan.n_n, ni = h->n_int;
    const int64_t nh = std::max<int64_t>(h->plan.n_halo, 1);
    TRY(dalloc(h, &h->x64w, n));
    TRY(dalloc(h, &h->xi, ni));
    TRY(dalloc(h, &h->ri64, ni, true));       // padding entries stay zero
    TRY(dalloc(h, &h->ri32, ni));
    TRY(dalloc(h, &h->qi32, ni));
    TRY(dalloc(h, &h->pi32[0], ni));
    TRY(dalloc(h, &h->pi32[1], ni));
    TRY(dalloc(h, &h->halo64, nh));
    TRY(dalloc(h, &h->halo32, nh));
    TRY(dalloc(h, &h->part5, 5 * (int64_t(h->pd.n_patches) + kFixGridMax)));
    return ensure_solver_vectors(h);
}

// The recurrence started from the FP64 true residual in ri64: p = q = 0,
// r32, r.z, beta = 0, alpha = 0 and the fresh flag (first pass: no update).
int cg1_start(ebe_handle* h, double thr2) {
    const int64_t ni = h->n_int;
    int l = 0;
    CK(cudaMemsetAsync(h->pi32[0], 0, sizeof(float) * size_t(ni), h->st), "memset");
    CK(cudaMemsetAsync(h->pi32[1], 0, sizeof(float) * size_t(ni), h->st), "memset");
    CK(cudaMemsetAsync(h->qi32, 0, sizeof(float) * size_t(ni), h->st), "memset");
    CK(launch_restart(1, ni, h->ri64, h->dinvi32, 1, h->part_vec, h->sc, h->st, &l, h->ri32), "restart");
    CK(launch_cg_arm(h->sc, h->st, &l), "arm");
    CK(launch_control(h->sc, thr2, -1, 0, h->st, &l), "control");
    add_launches(h, l);
    return EBE_OK;
}

int solve_cg1_impl(ebe_handle* h, double* x, bool x_on_host, const ebe_solve_opts& o, ebe_solve_info& info) {
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t n = h->plan.n_n, ni = h->n_int;
    TRY(cg1_buffers(h));
    int l = 0;
    CK(cudaMemcpyAsync(h->x64w, x, sizeof(double) * n, x_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       h->st), "copy x0");
    CK(launch_set_dirichlet(h->x64w, h->nd, h->g, h->n_d, h->st, &l), "x(nd) = g");
    CK(cudaMemsetAsync(h->xi, 0, sizeof(double) * size_t(ni), h->st), "memset");
    CK(launch_permute(0, 1, n, h->int_of_user, h->x64w, h->xi, h->st, &l), "x0 to the solver numbering");
    CK(launch_control(h->sc, 0.0, o.maxit, 1, h->st, &l), "control");
    add_launches(h, l);
    double rr = 0.0;
    TRY(true_residual_int(h, rr));
    info.true_residuals = 1;
    const double r0 = std::sqrt(rr);
    info.r0_norm = r0;
    info.iterations = 0;
    info.rel_residual = r0 > 0.0 ? 1.0 : 0.0;
    int status = EBE_OK;
    if (!std::isfinite(r0)) status = EBE_BREAKDOWN;
    if (r0 > 0.0 && std::isfinite(r0)) {
        const double target = o.rtol * r0;
        double fin = target;
        double thr = std::max(o.delta * r0, fin);
        TRY(cg1_start(h, thr * thr));
        if (o.use_graph) TRY(ensure_cg_graphs(h, o.chunk));
        int par = 0;                   // buffer of the current direction (read by the next pass)
        int64_t passes = h->sc_host->passes;
        double best = 1.0;
        int no_progress = 0;
        for (;;) {
            if (o.use_graph) {
                CK(cudaGraphLaunch(h->cg_graph[par], h->st), "cudaGraphLaunch");
                add_launches(h, h->cg_nodes);
            } else {
                l = 0;
                for (int it = 0; it < o.chunk; ++it)
                    CK(launch_cg_pass(h->pd_int, h->A32, h->ri32, h->qi32, h->pi32[(par + it) & 1],
                                      h->pi32[(par + it + 1) & 1], h->dinvi32, h->xi, h->halo32, h->part5, h->sc, h->st,
                                      &l, false), "single-sync pass");
                add_launches(h, l);
            }
            TRY(sync_scalars(h));
            const Scalars sh = *h->sc_host;
            const int64_t ran = sh.passes - passes;   // the first pass after a start counts no iteration
            par = int((par + ran) & 1);
            passes = sh.passes;
            info.iterations = sh.iter;
            if (sh.reason == kRunning) {
                if (ran == 0) return fail(h, EBE_CUDA_ERROR, "solver chunk made no progress");
                continue;
            }
            if (sh.reason == kBreakdown) { status = EBE_BREAKDOWN; break; }
            // the replacement residual in double-word form while the threshold
            // is large against its error, else in FP64; convergence is always
            // confirmed by the FP64 pass
            const bool dw = sh.reason == kTrigger && thr >= kDwReplaceRel * r0;
            TRY(true_residual_int(h, rr, dw));
            info.true_residuals += 1;
            double rel = std::sqrt(rr) / r0;
            if (dw && rel <= o.rtol) {
                TRY(true_residual_int(h, rr));
                info.true_residuals += 1;
                rel = std::sqrt(rr) / r0;
            }
            info.rel_residual = rel;
            if (!std::isfinite(rel)) { status = EBE_BREAKDOWN; break; }
            if (rel <= o.rtol) { status = EBE_OK; break; }
            if (sh.reason == kMaxit) { status = EBE_MAXIT; break; }
            if (rel < 0.9 * best) { best = rel; no_progress = 0; }
            else if (++no_progress >= o.stall_updates) { status = EBE_STALL; break; }
            if (sh.reason == kTrigger && thr <= fin) fin *= kFinalMargin;
            // residual replacement: continue CG from the FP64 true residual with
            // the direction that preceded the triggering pass (the pass that
            // triggered formed the next direction in the other buffer)
            par ^= 1;
            l = 0;
            CK(launch_restart(1, ni, h->ri64, h->dinvi32, 0, h->part_vec, h->sc, h->st, &l, h->ri32), "restart");
            CK(launch_cg_arm(h->sc, h->st, &l), "arm");
            thr = std::max(o.delta * std::sqrt(rr), fin);
            CK(launch_control(h->sc, thr * thr, -1, 0, h->st, &l), "control");
            add_launches(h, l);
        }
        if (status == EBE_BREAKDOWN && true_residual_int(h, rr) == EBE_OK) info.rel_residual = std::sqrt(rr) / r0;
    }
    l = 0;
    CK(launch_permute(0, 0, n, h->int_of_user, h->xi, h->x64w, h->st, &l), "x to the caller's numbering");
    add_launches(h, l);
    CK(cudaMemcpyAsync(x, h->x64w, sizeof(double) * n, x_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                       h->st), "copy x");
    CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    info.status = status;
    info.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (status != EBE_OK) {
        const char* why = status == EBE_MAXIT ? "maxit reached" : status == EBE_STALL ? "true residual stalled"
                                                                                        : "breakdown (p.Ap <= 0 or non-finite)";
        h->err = std::string("solve stopped: ") + why;
    }
    return status;
}

// The whole mixed-precision solve of a mesh of at most kSmallPatches
// patches in one CTA (k_cg_small): such a mesh leaves the grid-wide
// iteration bound by launch and barrier latency.
constexpr int kSmallPatches = 4;

bool small_eligible(const ebe_handle* h, const ebe_solve_opts& o) {
    return o.precision == EBE_PREC_MIXED && o.use_graph != 0 && h->store == EBE_STORE_MIXED &&
           h->pd.n_patches <= kSmallPatches &&
           small_solver_smem(h->plan.n_n, h->plan.n_e, h->pd.nb) <= size_t(200) * 1024;
}

// A colouring of the whole mesh for the one-CTA solver (once per handle).
int ensure_small_tables(ebe_handle* h) {
    if (h->small_order) return EBE_OK;
    TRY(ensure_gconn(h));
    std::vector<int32_t> order;
    std::vector<int64_t> col;
    std::string err;
    const int nc = global_colouring(h->plan, h->gconn_host, order, col, err);
    if (nc < 1 || nc > kSmallMaxColours) return fail(h, EBE_INVALID_ARG, nc < 1 ? err : "too many colours for the one-CTA solver");
    std::vector<int32_t> col32(col.begin(), col.end());
    // each node's (element, row) incidences, elements in colour order
    const HostPlan& P = h->plan;
    const int nb = P.nb;
    const int64_t n_e = int64_t(order.size());
    if (n_e > 4096 || nb * n_e > 65535 || P.n_n > 65535) return fail(h, EBE_INVALID_ARG, "mesh too large for the one-CTA solver");
    std::vector<uint16_t> iptr(size_t(P.n_n) + 1, 0), inc(size_t(nb * n_e), 0);
    for (int64_t k = 0; k < n_e; ++k)
        for (int r = 0; r < nb; ++r) ++iptr[size_t(h->gconn_host[size_t(order[size_t(k)]) * nb + r] & kNodeMask) + 1];
    for (int64_t v = 0; v < P.n_n; ++v) iptr[size_t(v) + 1] = uint16_t(iptr[size_t(v) + 1] + iptr[size_t(v)]);
    std::vector<uint16_t> fill(iptr.begin(), iptr.end() - 1);
    for (int64_t k = 0; k < n_e; ++k)
        for (int r = 0; r < nb; ++r) {
            const int64_t v = h->gconn_host[size_t(order[size_t(k)]) * nb + r] & kNodeMask;
            inc[fill[size_t(v)]++] = uint16_t(k | (int64_t(r) << 12));
        }
    TRY(upload(h, &h->small_order, order.data(), int64_t(order.size())));
    TRY(upload(h, &h->small_col, col32.data(), int64_t(col32.size())));
    TRY(upload(h, &h->small_inc_ptr, iptr.data(), int64_t(iptr.size())));
    TRY(upload(h, &h->small_inc, inc.data(), int64_t(inc.size())));
    h->small_ncol = nc;
    CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");   // the host tables go away
    return EBE_OK;
}

int solve_small_impl(ebe_handle* h, double* x, bool x_on_host, const ebe_solve_opts& o, ebe_solve_info& info) {
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t n = h->plan.n_n;
    TRY(dalloc(h, &h->x64w, n));
    TRY(dalloc(h, &h->small_info, 1));
    int l = 0;
    CK(cudaMemcpyAsync(h->x64w, x, sizeof(double) * n, x_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       h->st), "copy x0");
    CK(launch_set_dirichlet(h->x64w, h->nd, h->g, h->n_d, h->st, &l), "x(nd) = g");
    SmallOpts so;
    so.rtol = o.rtol;
    so.delta = o.delta;
    so.maxit = o.maxit;
    so.stall_updates = o.stall_updates;
    SmallColouring sc;
    sc.order = h->small_order;
    sc.col = h->small_col;
    sc.inc_ptr = h->small_inc_ptr;
    sc.inc = h->small_inc;
    sc.gather = small_solver_gather(n, h->plan.n_e, h->pd.nb) ? 1 : 0;
    sc.gconn = h->gconn;
    sc.n_e = int32_t(h->plan.n_e);
    sc.n_col = h->small_ncol;
    CK(launch_cg_small(h->pd, n, h->A32, h->A64, h->b, h->dinv32, h->x64w, sc, so, h->small_info, h->st, &l),
       "one-CTA solver");
    add_launches(h, l);
    SmallInfo si{};
    CK(cudaMemcpyAsync(&si, h->small_info, sizeof(SmallInfo), cudaMemcpyDeviceToHost, h->st), "read solver outcome");
    CK(cudaMemcpyAsync(x, h->x64w, sizeof(double) * n, x_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                       h->st), "copy x");
    CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    info.status = si.status;
    info.iterations = si.iterations;
    info.true_residuals = si.true_residuals;
    info.rel_residual = si.rel;
    info.r0_norm = si.r0;
    info.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (si.status != EBE_OK) {
        const char* why = si.status == EBE_MAXIT ? "maxit reached" : si.status == EBE_STALL ? "true residual stalled"
                                                                                             : "breakdown (p.Ap <= 0 or non-finite)";
        h->err = std::string("solve stopped: ") + why;
    }
    return si.status;
}

int solve_entry(ebe_handle* h, double* x, bool host, const ebe_solve_opts* opts, ebe_solve_info* info) {
    TRY(check_ready(h, true));
    if (!x) return fail(h, EBE_INVALID_ARG, "x is NULL");
    ebe_solve_opts o;
    ebe_solve_opts_default(&o);
    if (opts) o = *opts;
    if (!(o.rtol > 0.0) || o.maxit < 1 || o.chunk < 1 || o.chunk > 4096 || !(o.delta > 0.0 && o.delta < 1.0) ||
        o.stall_updates < 1 ||
        (o.precision != EBE_PREC_FP64 && o.precision != EBE_PREC_MIXED && o.precision != EBE_PREC_MIXED_TEXTBOOK))
        return fail(h, EBE_INVALID_ARG, "bad solve options");
    ebe_solve_info local{};
    Scope scp(h);
    // a small mesh whose colouring needs more colours than the one-CTA solver
    // takes runs the grid-wide iteration
    const bool small = small_eligible(h, o) && ensure_small_tables(h) == EBE_OK;
    if (!small) h->err.clear();
    int s = o.precision != EBE_PREC_MIXED ? solve_impl(h, x, host, o, local)
            : small                      ? solve_small_impl(h, x, host, o, local)
                                         : solve_cg1_impl(h, x, host, o, local);
    if (info) *info = local;
    return s;
}

}  // namespace

ebe_status ebe_time_cg_pass(ebe_handle* h, int32_t reps, double* ms) {
    TRY(check_ready(h, true));
    if (!ms || reps < 1 || reps > 100000) return ebe_status(fail(h, EBE_INVALID_ARG, "ms must be non-NULL, 1 <= reps <= 100000"));
    Scope scp(h);
    TRY(cg1_buffers(h));
    int l = 0;
    CK(cudaMemsetAsync(h->xi, 0, sizeof(double) * size_t(h->n_int), h->st), "memset");
    CK(launch_control(h->sc, 0.0, int64_t(1) << 62, 1, h->st, &l), "control");
    add_launches(h, l);
    double rr = 0.0;
    TRY(true_residual_int(h, rr));
    TRY(cg1_start(h, -1.0));                       // threshold 0: no stop inside the timed passes
    std::vector<cudaEvent_t> ev(size_t(3) * size_t(reps + 1), nullptr);
    int status = EBE_OK;
    for (auto& e : ev) {
        const cudaError_t c = cudaEventCreate(&e);
        if (c != cudaSuccess && status == EBE_OK) status = cuda_fail(h, c, "cudaEventCreate");
    }
    l = 0;
    for (int r = 0; r <= reps && status == EBE_OK; ++r) {   // pass 0 is the fresh (untimed) pass
        const cudaError_t e = launch_cg_pass(h->pd_int, h->A32, h->ri32, h->qi32, h->pi32[r & 1], h->pi32[(r + 1) & 1],
                                             h->dinvi32, h->xi, h->halo32, h->part5, h->sc, h->st, &l, true,
                                             &ev[size_t(3) * size_t(r)]);
        if (e != cudaSuccess) status = cuda_fail(h, e, "single-sync pass");
    }
    add_launches(h, l);
    double t_patch = 0.0, t_fix = 0.0;
    if (status == EBE_OK) {
        const cudaError_t e = cudaEventSynchronize(ev.back());
        if (e != cudaSuccess) status = cuda_fail(h, e, "cudaEventSynchronize");
        for (int r = 1; r <= reps && status == EBE_OK; ++r) {
            float a = 0.f, c = 0.f;
            cudaEventElapsedTime(&a, ev[size_t(3) * r], ev[size_t(3) * r + 1]);
            cudaEventElapsedTime(&c, ev[size_t(3) * r + 1], ev[size_t(3) * r + 2]);
            t_patch += a;
            t_fix += c;
        }
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (status == EBE_OK) status = sync_scalars(h);
    if (status == EBE_OK && h->sc_host->reason != kRunning)
        status = fail(h, EBE_BREAKDOWN, "the timed passes stopped (breakdown)");
    if (status != EBE_OK) return ebe_status(status);
    ms[0] = t_patch / reps;
    ms[1] = t_fix / reps;
    return EBE_OK;
}

ebe_status ebe_solve(ebe_handle* h, double* x, const ebe_solve_opts* opts, ebe_solve_info* info) {
    return ebe_status(solve_entry(h, x, false, opts, info));
}

ebe_status ebe_solve_host(ebe_handle* h, double* x, const ebe_solve_opts* opts, ebe_solve_info* info) {
    return ebe_status(solve_entry(h, x, true, opts, info));
}

// Stationary iterations of Sec. 2 on a device x: method 0 Richardson
// (Eq. richardson), 1 two-level Chebyshev (Eq. Czebyshev2lev), 2 three-level
// Chebyshev (Eq. Czebyshev3lev) in its direction form: with d = (l1+l2)/2,
// c = (l2-l1)/2, step 0 takes p = r, alpha = 1/d; step k > 0 takes
// beta = (c alpha / 2)^2, p = r + beta p, alpha = 1/(d - beta/alpha); then
// x += alpha p.  Every step starts from the residual r = mask(b - A x).
static int stationary_impl(ebe_handle* h, double* x, int64_t iters, int method, const double* prm, int64_t np) {
    TRY(check_ready(h, true));
    if (!x || iters < 0) return fail(h, EBE_INVALID_ARG, "x must be non-NULL and iters >= 0");
    if (method == 1) {
        if (!prm || np < 1) return fail(h, EBE_INVALID_ARG, "alphas must hold N >= 1 roots");
        for (int64_t k = 0; k < np; ++k)
            if (!std::isfinite(prm[k]) || prm[k] == 0.0) return fail(h, EBE_INVALID_ARG, "roots must be finite and nonzero");
    }
    if (method == 2 && !(prm[0] > 0.0 && prm[1] > prm[0] && std::isfinite(prm[1])))
        return fail(h, EBE_INVALID_ARG, "need 0 < lam1 < lam2");
    if (method == 0 && !std::isfinite(prm[0])) return fail(h, EBE_INVALID_ARG, "omega must be finite");
    Scope scp(h);
    const int64_t n = h->plan.n_n;
    TRY(dalloc(h, &h->r64, n));
    TRY(dalloc(h, &h->halo64, std::max<int64_t>(h->plan.n_halo, 1)));
    if (method == 2) TRY(dalloc(h, &h->p64, n));
    int l = 0;
    CK(launch_set_dirichlet(x, h->nd, h->g, h->n_d, h->st, &l), "x(nd) = g");
    const double d = method == 2 ? 0.5 * (prm[0] + prm[1]) : 0.0, c = method == 2 ? 0.5 * (prm[1] - prm[0]) : 0.0;
    double alpha = 0.0;
    for (int64_t k = 0; k < iters; ++k) {
        CK(launch_patch_pass(h->pd, 0, kResidual, h->A64, x, h->b, h->r64, h->halo64, h->part_patch, nullptr, h->sc, h->st,
                             &l), "residual");
        if (method == 0) {
            CK(launch_stationary(n, x, h->r64, nullptr, 0, prm[0], 0.0, h->st, &l), "update");
        } else if (method == 1) {
            CK(launch_stationary(n, x, h->r64, nullptr, 0, 1.0 / prm[k % np], 0.0, h->st, &l), "update");
        } else {
            // From Eq. Czebyshev3lev: alpha_k = 2 C_k / (c C_{k+1}) and
            // beta_k = (C_{k-1} / C_k)^2 = (c alpha_{k-1} / 2)^2 for k >= 2; the
            // special first step x^1 = x^0 + r_0 / d makes beta_1 = (c alpha_0)^2 / 2.
            double beta = 0.0;
            if (k == 0) {
                alpha = 1.0 / d;
            } else {
                beta = k == 1 ? 0.5 * (c * alpha) * (c * alpha) : (c * alpha / 2.0) * (c * alpha / 2.0);
                alpha = 1.0 / (d - beta / alpha);
            }
            CK(launch_stationary(n, x, h->r64, h->p64, 1, alpha, beta, h->st, &l), "update");
        }
    }
    add_launches(h, l);
    return check_device(h);
}

ebe_status ebe_richardson(ebe_handle* h, double* x, int64_t iters, double omega) {
    return ebe_status(stationary_impl(h, x, iters, 0, &omega, 1));
}

ebe_status ebe_chebyshev2(ebe_handle* h, double* x, int64_t iters, const double* alphas, int64_t N) {
    return ebe_status(stationary_impl(h, x, iters, 1, alphas, N));
}

// The roots of P_N (Sec. 2.2) for the spectrum bounds lam1 < lam2, in the
// order the paper's two-level listing cycles through them:
// alpha_k = (lam1 + lam2)/2 + (lam2 - lam1)/2 cos(pi (k + 1/2) / N),
// k = 0..N-1, largest first.  The order matters in floating point: it decides
// how far the partial products of (I - A / alpha_k) grow within a cycle.
ebe_status ebe_chebyshev2_bounds(ebe_handle* h, double* x, int64_t iters, double lam1, double lam2, int64_t N) {
    if (!h) return EBE_INVALID_ARG;
    if (!(lam1 > 0.0 && lam2 > lam1 && std::isfinite(lam2)) || N < 1 || N > (int64_t(1) << 20))
        return ebe_status(fail(h, EBE_INVALID_ARG, "need 0 < lam1 < lam2 and 1 <= N <= 2^20"));
    const double d = 0.5 * (lam1 + lam2), c = 0.5 * (lam2 - lam1);
    std::vector<double> alphas(static_cast<size_t>(N));
    for (int64_t k = 0; k < N; ++k) alphas[size_t(k)] = d + c * std::cos(M_PI * (double(k) + 0.5) / double(N));
    return ebe_status(stationary_impl(h, x, iters, 1, alphas.data(), N));
}

ebe_status ebe_chebyshev3(ebe_handle* h, double* x, int64_t iters, double lam1, double lam2) {
    const double prm[2] = {lam1, lam2};
    return ebe_status(stationary_impl(h, x, iters, 2, prm, 2));
}

// ---------------------------------------------------------------- batched solver

namespace {

constexpr int kFixRows = 512;                         // shared-node rows per fix-up item (2 per thread)
constexpr int kTileSizes[3] = {1024, 2048, 4096};     // node-tile sizes of the vector phases

int tile_index(int tile_nodes) {
    for (int i = 0; i < 3; ++i)
        if (kTileSizes[i] == tile_nodes) return i;
    return -1;
}

// Work items of the batched solver (host-built once per handle and tile size)
// and its per-problem state.
int ensure_batch_tables(ebe_handle* h, int ti) {
    const BatchLayout& L = h->lay;
    if (!h->bfix) {
        std::vector<BatchItem> fx;
        for (int k = 0; k < h->n_prob; ++k) {
            const int r0 = L.shared_off[k], r1 = L.shared_off[k + 1];
            const int p0 = L.patch_off[k], p1 = L.patch_off[k + 1];
            const int cnt = std::max(1, (r1 - r0 + kFixRows - 1) / kFixRows);
            const int pch = (p1 - p0 + cnt - 1) / cnt;
            const int first = int(fx.size());
            for (int c = 0; c < cnt; ++c) {
                BatchItem it{};
                it.k = k;
                it.lo = std::min(r1, r0 + c * kFixRows);
                it.hi = std::min(r1, r0 + (c + 1) * kFixRows);
                it.plo = std::min(p1, p0 + c * pch);
                it.phi = std::min(p1, p0 + (c + 1) * pch);
                it.first = first;
                it.count = cnt;
                fx.push_back(it);
            }
        }
        TRY(upload(h, &h->bfix, fx.data(), int64_t(fx.size())));
        h->n_bfix = int(fx.size());
        TRY(dalloc(h, &h->bpart_f, h->n_bfix));
    }
    auto tiles = [&](int tn, std::vector<BatchItem>* out) {
        int64_t n = 0;
        for (int k = 0; k < h->n_prob; ++k) {
            const int64_t n0 = L.node_off[k], n1 = L.node_off[k + 1];
            const int cnt = int(std::max<int64_t>(1, (n1 - n0 + tn - 1) / tn));
            if (out) {
                const int first = int(out->size());
                for (int c = 0; c < cnt; ++c) {
                    BatchItem it{};
                    it.k = k;
                    it.lo = int32_t(std::min(n1, n0 + int64_t(c) * tn));
                    it.hi = int32_t(std::min(n1, n0 + int64_t(c + 1) * tn));
                    it.first = first;
                    it.count = cnt;
                    out->push_back(it);
                }
            }
            n += cnt;
        }
        return n;
    };
    if (!h->btile[ti]) {
        std::vector<BatchItem> tl;
        tiles(kTileSizes[ti], &tl);
        TRY(upload(h, &h->btile[ti], tl.data(), int64_t(tl.size())));
        h->n_btile[ti] = int(tl.size());
        std::vector<BatchProbInfo> pi(size_t(h->n_prob));
        std::vector<BatchItem> fx(size_t(h->n_bfix));
        CK(cudaMemcpyAsync(fx.data(), h->bfix, sizeof(BatchItem) * fx.size(), cudaMemcpyDeviceToHost, h->st), "read items");
        CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
        for (const BatchItem& it : fx)
            if (it.first == int(&it - fx.data())) { pi[it.k].fix_first = it.first; pi[it.k].fix_count = it.count; }
        for (size_t t = 0; t < tl.size(); ++t)
            if (tl[t].first == int(t)) { pi[tl[t].k].tile_first = tl[t].first; pi[tl[t].k].tile_count = tl[t].count; }
        for (int k = 0; k < h->n_prob; ++k) {
            pi[k].patch_first = L.patch_off[k];
            pi[k].patch_count = L.patch_off[k + 1] - L.patch_off[k];
        }
        TRY(upload(h, &h->bpinfo[ti], pi.data(), int64_t(pi.size())));
    }
    if (!h->bpart_u) TRY(dalloc(h, &h->bpart_u, 2 * tiles(kTileSizes[0], nullptr)));   // the most tiles
    if (!h->bprob) {
        TRY(dalloc(h, &h->bprob, h->n_prob, true));
        TRY(dalloc(h, &h->bctr, 2 * h->n_prob, true));
        TRY(dalloc(h, &h->bbar, 2, true));
        TRY(dalloc(h, &h->blive, 1, true));
        TRY(dalloc(h, &h->bloops, 1, true));
        TRY(dalloc(h, &h->bphase, 4, true));
        CK(cudaMallocHost(&h->bprob_host, sizeof(BatchProblem) * size_t(h->n_prob)), "cudaMallocHost");
        CK(cudaMallocHost(&h->bcount_host, 6 * sizeof(int64_t)), "cudaMallocHost");
    }
    return EBE_OK;
}

int batch_buffers(ebe_handle* h, bool mixed) {
    const int64_t n = h->plan.n_n;
    const int64_t nh = std::max<int64_t>(h->plan.n_halo, 1);
    TRY(dalloc(h, &h->x64w, n));
    TRY(dalloc(h, &h->r64, n));
    TRY(dalloc(h, &h->halo64, nh));
    if (mixed) {
        TRY(dalloc(h, &h->p32, n));
        TRY(dalloc(h, &h->q32, n));
        TRY(dalloc(h, &h->r32, n));
        TRY(dalloc(h, &h->halo32, nh));
    } else {
        TRY(dalloc(h, &h->p64, n));
        TRY(dalloc(h, &h->q64, n));
    }
    return EBE_OK;
}

BatchDev make_batch_dev(ebe_handle* h, bool mixed, int ti, const ebe_solve_opts& o, int64_t budget) {
    BatchDev bd;
    bd.pd = h->pd;
    bd.n_prob = h->n_prob;
    bd.n_fix = h->n_bfix;
    bd.n_tile = h->n_btile[ti];
    bd.pinfo = h->bpinfo[ti];
    bd.fix = h->bfix;
    bd.tile = h->btile[ti];
    bd.A = mixed ? static_cast<const void*>(h->A32) : h->A64;
    bd.A64 = h->A64;
    bd.Adw = mixed ? h->Adw : nullptr;
    bd.b = h->b;
    bd.dinv = mixed ? static_cast<const void*>(h->dinv32) : h->dinv;
    bd.x = h->x64w;
    bd.r = h->r64;
    bd.rin = mixed ? static_cast<void*>(h->r32) : h->r64;
    bd.p = mixed ? static_cast<void*>(h->p32) : h->p64;
    bd.q = mixed ? static_cast<void*>(h->q32) : h->q64;
    bd.halo = mixed ? static_cast<void*>(h->halo32) : h->halo64;
    bd.halo64 = h->halo64;
    bd.part_p = h->part_patch;
    bd.part_f = h->bpart_f;
    bd.part_u = h->bpart_u;
    bd.prob = h->bprob;
    bd.ctr = h->bctr;
    bd.bar = h->bbar;
    bd.live = h->blive;
    bd.loops = h->bloops;
    bd.phase_ns = h->bphase;
    bd.rtol = o.rtol;
    bd.delta = o.delta;
    bd.margin = kFinalMargin;
    bd.maxit = o.maxit;
    bd.stall_updates = o.stall_updates;
    bd.iter_budget = budget;
    return bd;
}

// The launch shape to use: cfg's fields, 0 = default; checked against what fits.
int resolve_shape(ebe_handle* h, const BatchDev& bd, bool mixed, const ebe_batch_config& cfg, int& ctas) {
    const int maxc = batch_max_ctas_per_sm(bd, mixed, nullptr);
    if (maxc < 1) return fail(h, EBE_INVALID_ARG, "the batched solver's shared memory does not fit on an SM");
    ctas = cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : maxc;
    if (ctas > maxc) return fail(h, EBE_INVALID_ARG, "ctas_per_sm = " + std::to_string(ctas) + " does not fit (at most " +
                                                         std::to_string(maxc) + ")");
    return EBE_OK;
}

int enqueue_batch(ebe_handle* h, const BatchDev& bd, bool mixed, int ctas, int* l) {
    CK(launch_set_dirichlet(h->x64w, h->nd, h->g, h->n_d, h->st, l), "x(nd) = g");
    CK(launch_batch_init(bd, h->st, l), "batch init");
    CK(launch_batch_solve(bd, mixed, ctas, h->st, l), "batched solver");
    return EBE_OK;
}

// Reads the problems' state and the loop counters (synchronises the stream).
int read_batch_state(ebe_handle* h, int64_t& loops, int32_t& live) {
    CK(cudaMemcpyAsync(h->bprob_host, h->bprob, sizeof(BatchProblem) * size_t(h->n_prob), cudaMemcpyDeviceToHost, h->st),
       "read batch state");
    CK(cudaMemcpyAsync(h->bcount_host, h->bloops, sizeof(int64_t), cudaMemcpyDeviceToHost, h->st), "read loops");
    CK(cudaMemcpyAsync(h->bcount_host + 1, h->blive, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st), "read live");
    CK(cudaMemcpyAsync(h->bcount_host + 2, h->bphase, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, h->st),
       "read phase times");
    TRY(check_device(h));
    loops = h->bcount_host[0];
    live = *reinterpret_cast<const int32_t*>(h->bcount_host + 1);
    return EBE_OK;
}

int solve_batch_impl(ebe_handle* h, double* x, bool x_on_host, const ebe_solve_opts& o, ebe_solve_info* info,
                     ebe_batch_info* summary) {
    const auto t0 = std::chrono::steady_clock::now();
    const bool mixed = o.precision == EBE_PREC_MIXED;
    if (mixed && h->store != EBE_STORE_MIXED) return fail(h, EBE_NOT_READY, "EBE_PREC_MIXED needs ebe_assemble(EBE_STORE_MIXED)");
    const ebe_batch_config& cfg = h->bcfg[mixed ? 1 : 0];
    const int tile = cfg.tile_nodes > 0 ? cfg.tile_nodes : 2048;
    const int ti = tile_index(tile);
    TRY(batch_buffers(h, mixed));
    TRY(ensure_batch_tables(h, ti));
    if (mixed) TRY(ensure_dw(h));
    // one launch runs up to maxit CG steps plus the true residuals of every
    // problem; a launch that ends with problems left is followed by another
    const int64_t budget = o.maxit + 65536;
    BatchDev bd = make_batch_dev(h, mixed, ti, o, budget);
    if (cfg.barrier_ns > 0) bd.barrier_ns = uint64_t(cfg.barrier_ns);
    int ctas = 0;
    TRY(resolve_shape(h, bd, mixed, cfg, ctas));
    const int64_t n = h->plan.n_n;
    CK(cudaMemcpyAsync(h->x64w, x, sizeof(double) * n, x_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->st),
       "copy x0");
    int l = 0;
    if (o.use_graph) {
        const std::vector<double> key = {double(mixed), double(ctas), double(tile), o.rtol, o.delta, double(o.maxit),
                                         double(o.stall_updates), double(bd.barrier_ns)};
        if (!h->bgraph || h->bgraph_key != key) {
            if (h->bgraph) { cudaGraphExecDestroy(h->bgraph); h->bgraph = nullptr; }
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
            int lc = 0;
            const int st = enqueue_batch(h, bd, mixed, ctas, &lc);
            cudaError_t e = cudaStreamEndCapture(h->st, &g);
            if (st != EBE_OK) { if (g) cudaGraphDestroy(g); return st; }
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture (batched solver)");
            e = cudaGraphInstantiate(&h->bgraph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { h->bgraph = nullptr; return cuda_fail(h, e, "cudaGraphInstantiate (batched solver)"); }
            h->bgraph_key = key;
        }
        CK(cudaGraphLaunch(h->bgraph, h->st), "cudaGraphLaunch");
        l += 2 + (h->n_d > 0 ? 1 : 0);
    } else {
        TRY(enqueue_batch(h, bd, mixed, ctas, &l));
    }
    int launches = 1;
    int64_t loops = 0, prev = -1;
    int32_t live = 0;
    for (;;) {
        TRY(read_batch_state(h, loops, live));
        if (live <= 0) break;
        if (loops == prev) return fail(h, EBE_CUDA_ERROR, "batched solver made no progress");
        prev = loops;
        CK(launch_batch_solve(bd, mixed, ctas, h->st, &l), "batched solver");
        ++launches;
    }
    add_launches(h, l);
    CK(cudaMemcpyAsync(x, h->x64w, sizeof(double) * n, x_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->st),
       "copy x");
    CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    int status = EBE_OK, n_ok = 0;
    for (int k = 0; k < h->n_prob; ++k) {
        const BatchProblem& P = h->bprob_host[k];
        if (P.status == EBE_OK) ++n_ok;
        else if (status == EBE_OK) status = P.status;
        if (info) {
            info[k].status = P.status;
            info[k].iterations = P.iter;
            info[k].true_residuals = P.n_true;
            info[k].rel_residual = P.rel;
            info[k].r0_norm = P.r0;
            info[k].solve_ms = ms;
        }
    }
    if (summary) {
        summary->loops = loops;
        summary->launches = launches;
        summary->n_converged = n_ok;
        summary->solve_ms = ms;
        summary->config.ctas_per_sm = ctas;
        summary->config.tile_nodes = tile;
        summary->config.barrier_ns = int64_t(bd.barrier_ns);
        for (int ph = 0; ph < 4; ++ph) summary->phase_ms[ph] = double(h->bcount_host[2 + ph]) * 1e-6;
    }
    if (status != EBE_OK)
        h->err = std::to_string(h->n_prob - n_ok) + " of " + std::to_string(h->n_prob) + " problems did not reach rtol (" +
                 ebe_status_string(status) + " first)";
    return status;
}

int solve_batch_entry(ebe_handle* h, double* x, bool host, const ebe_solve_opts* opts, ebe_solve_info* info,
                      ebe_batch_info* summary) {
    TRY(check_ready(h, true));
    if (!x) return fail(h, EBE_INVALID_ARG, "x is NULL");
    ebe_solve_opts o;
    ebe_solve_opts_default(&o);
    if (opts) o = *opts;
    if (!(o.rtol > 0.0) || o.maxit < 1 || !(o.delta > 0.0 && o.delta < 1.0) || o.stall_updates < 1 ||
        (o.precision != EBE_PREC_FP64 && o.precision != EBE_PREC_MIXED))
        return fail(h, EBE_INVALID_ARG, "bad solve options");
    Scope scp(h);
    return solve_batch_impl(h, x, host, o, info, summary);
}

}  // namespace

ebe_status ebe_solve_batch(ebe_handle* h, double* x, const ebe_solve_opts* opts, ebe_solve_info* info,
                           ebe_batch_info* summary) {
    return ebe_status(solve_batch_entry(h, x, false, opts, info, summary));
}

ebe_status ebe_solve_batch_host(ebe_handle* h, double* x, const ebe_solve_opts* opts, ebe_solve_info* info,
                                ebe_batch_info* summary) {
    return ebe_status(solve_batch_entry(h, x, true, opts, info, summary));
}

ebe_status ebe_set_batch_config(ebe_handle* h, const ebe_batch_config* cfg) {
    if (!h) return EBE_INVALID_ARG;
    if (!cfg) { h->bcfg[0] = h->bcfg[1] = ebe_batch_config{0, 0, 0}; return EBE_OK; }
    if (cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > 8 || (cfg->tile_nodes != 0 && tile_index(cfg->tile_nodes) < 0) ||
        cfg->barrier_ns < 0)
        return ebe_status(fail(h, EBE_INVALID_ARG,
                               "ctas_per_sm must be in [0, 8], tile_nodes 0, 1024, 2048 or 4096, barrier_ns >= 0"));
    h->bcfg[0] = h->bcfg[1] = *cfg;
    return EBE_OK;
}

ebe_status ebe_batch_tune(ebe_handle* h, int32_t precision, int32_t loops, ebe_batch_config* best,
                          ebe_batch_config* shapes, double* ms_out, int32_t capacity, int32_t* n_written) {
    TRY(check_ready(h, true));
    if (loops < 0 || (precision != EBE_PREC_FP64 && precision != EBE_PREC_MIXED) || capacity < 0)
        return ebe_status(fail(h, EBE_INVALID_ARG, "bad tuning arguments"));
    const bool mixed = precision == EBE_PREC_MIXED;
    if (mixed && h->store != EBE_STORE_MIXED) return ebe_status(fail(h, EBE_NOT_READY, "EBE_PREC_MIXED needs EBE_STORE_MIXED"));
    Scope scp(h);
    TRY(batch_buffers(h, mixed));
    if (mixed) TRY(ensure_dw(h));
    ebe_solve_opts o;
    ebe_solve_opts_default(&o);
    o.precision = precision;
    cudaEvent_t ev[2];
    CK(cudaEventCreate(&ev[0]), "cudaEventCreate");
    CK(cudaEventCreate(&ev[1]), "cudaEventCreate");
    struct Cand { ebe_batch_config c; double ms; };
    std::vector<Cand> cands;
    int status = EBE_OK;
    for (int ti = 0; ti < 3 && status == EBE_OK; ++ti) {
        status = ensure_batch_tables(h, ti);
        if (status != EBE_OK) break;
        const BatchDev bd = make_batch_dev(h, mixed, ti, o, loops > 0 ? loops : o.maxit + 65536);
        const int maxc = batch_max_ctas_per_sm(bd, mixed, nullptr);
        for (int c = 1; c <= maxc && status == EBE_OK; ++c) {
            // one untimed run for the first candidate (module load, attributes)
            for (int rep = cands.empty() ? 0 : 1; rep < 2 && status == EBE_OK; ++rep) {
                int l = 0;
                cudaError_t e = cudaMemsetAsync(h->x64w, 0, sizeof(double) * size_t(h->plan.n_n), h->st);
                if (e != cudaSuccess) { status = cuda_fail(h, e, "cudaMemsetAsync"); break; }
                cudaEventRecord(ev[0], h->st);
                status = enqueue_batch(h, bd, mixed, c, &l);
                cudaEventRecord(ev[1], h->st);
                add_launches(h, l);
                int64_t done_loops = 0;
                int32_t live = 0;
                if (status == EBE_OK) status = read_batch_state(h, done_loops, live);
                if (status != EBE_OK || rep == 0) continue;
                float t = 0.f;
                cudaEventElapsedTime(&t, ev[0], ev[1]);
                const double per = loops > 0 ? double(t) / double(std::max<int64_t>(done_loops, 1)) : double(t);
                cands.push_back({ebe_batch_config{c, kTileSizes[ti], h->bcfg[mixed ? 1 : 0].barrier_ns}, per});
            }
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (status != EBE_OK) return ebe_status(status);
    if (cands.empty()) return ebe_status(fail(h, EBE_INVALID_ARG, "no launch shape of the batched solver fits"));
    size_t bi = 0;
    for (size_t i = 1; i < cands.size(); ++i)
        if (cands[i].ms < cands[bi].ms) bi = i;
    h->bcfg[mixed ? 1 : 0] = cands[bi].c;
    if (best) *best = cands[bi].c;
    int nw = 0;
    for (size_t i = 0; i < cands.size() && nw < capacity; ++i, ++nw) {
        if (shapes) shapes[nw] = cands[i].c;
        if (ms_out) ms_out[nw] = cands[i].ms;
    }
    if (n_written) *n_written = nw;
    return EBE_OK;
}

static void export_plan(const HostPlan& P, ebe_partition_sizes* sz, int32_t* slot_elem, uint16_t* lconn,
                        int32_t* patch_meta, int32_t* pnode, int32_t* col_ptr, int32_t* sh_node, int32_t* sh_ptr,
                        int32_t* sh_slot) {
    sz->n_patches = P.n_patches;
    sz->n_slots = P.n_slots;
    sz->n_pnode = int64_t(P.pnode.size());
    sz->n_colptr = int64_t(P.col_ptr.size());
    sz->n_shared = int64_t(P.sh_node.size());
    sz->n_halo = P.n_halo;
    sz->max_nodes = P.max_nodes;
    sz->max_colours = P.max_col;
    sz->patch_elems = kPatch;
    auto put = [](auto* dst, const auto& v) { if (dst) std::copy(v.begin(), v.end(), dst); };
    put(slot_elem, P.slot_elem);
    put(lconn, P.lconn);
    put(pnode, P.pnode);
    put(col_ptr, P.col_ptr);
    put(sh_node, P.sh_node);
    put(sh_ptr, P.sh_ptr);
    put(sh_slot, P.sh_slot);
    if (patch_meta)
        for (int64_t p = 0; p < P.n_patches; ++p) std::memcpy(patch_meta + 8 * p, &P.meta[p], sizeof(PatchMeta));
}

ebe_status ebe_partition_export(const ebe_mesh* m, ebe_partition_sizes* sz, int32_t* slot_elem, uint16_t* lconn,
                                int32_t* patch_meta, int32_t* pnode, int32_t* col_ptr, int32_t* sh_node,
                                int32_t* sh_ptr, int32_t* sh_slot) {
    if (!m || !sz) { g_create_error = "mesh and sizes must be non-NULL"; return EBE_INVALID_ARG; }
    HostPlan P;
    std::string err;
    int s = build_plan(*m, P, err);
    if (s != EBE_OK) { g_create_error = err; return ebe_status(s); }
    export_plan(P, sz, slot_elem, lconn, patch_meta, pnode, col_ptr, sh_node, sh_ptr, sh_slot);
    return EBE_OK;
}

ebe_status ebe_partition_export_batch(const ebe_mesh* meshes, int32_t n_problems, ebe_partition_sizes* sz,
                                      int32_t* patch_off, int32_t* slot_elem, uint16_t* lconn, int32_t* patch_meta,
                                      int32_t* pnode, int32_t* col_ptr, int32_t* sh_node, int32_t* sh_ptr,
                                      int32_t* sh_slot) {
    if (!meshes || !sz || n_problems < 1 || n_problems > kBatchMaxProblems) {
        g_create_error = "meshes and sizes must be non-NULL, 1 <= n_problems <= " + std::to_string(kBatchMaxProblems);
        return EBE_INVALID_ARG;
    }
    HostPlan P;
    BatchLayout L;
    std::string err;
    const int threads = host_threads(32);
    int s = build_batch_plan(meshes, n_problems, threads, P, L, err);
    if (s != EBE_OK) { g_create_error = err; return ebe_status(s); }
    export_plan(P, sz, slot_elem, lconn, patch_meta, pnode, col_ptr, sh_node, sh_ptr, sh_slot);
    if (patch_off) std::copy(L.patch_off.begin(), L.patch_off.end(), patch_off);
    return EBE_OK;
}

// ---------------------------------------------------------------- learned preconditioner

struct ebe_mpnn {
    int device = 0;
    std::vector<void*> allocs;
    MpnnDev md;
    double* grad = nullptr;          // [kMpnnParams]
    int64_t cap_inf = 0, cap_train = 0, cap_vec = 0;
    double *z = nullptr, *w = nullptr, *aw = nullptr, *ae = nullptr, *gz = nullptr;
    int32_t* err = nullptr;
    int step = 0;
    std::string msg;
};

extern "C++" {
namespace {

int mfail(ebe_mpnn* m, int status, const std::string& msg) {
    if (m) m->msg = msg;
    return status;
}

template <typename T>
int malloc_net(ebe_mpnn* m, T** p, int64_t count, bool zero = false) {
    void* v = nullptr;
    const size_t bytes = size_t(std::max<int64_t>(count, 1)) * sizeof(T);
    cudaError_t e = cudaMalloc(&v, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return mfail(m, EBE_OOM, "cudaMalloc failed"); }
    m->allocs.push_back(v);
    if (zero && cudaMemset(v, 0, bytes) != cudaSuccess) return mfail(m, EBE_CUDA_ERROR, "cudaMemset failed");
    *p = static_cast<T*>(v);
    return EBE_OK;
}

#define MTRY(call)                        \
    do {                                  \
        int s_ = (call);                  \
        if (s_ != EBE_OK) return s_;      \
    } while (0)

// Mesh graph of the handle: every node's neighbours (nodes sharing an element),
// ascending, from the partition's element lists; built once per handle.
int ensure_mesh_graph(ebe_handle* h) {
    if (h->g_ptr) return EBE_OK;
    const HostPlan& P = h->plan;
    const int64_t n = P.n_n;
    const int nb = P.nb;
    std::vector<int32_t> el(size_t(P.n_e) * nb);
    int64_t e = 0;
    for (int64_t p = 0; p < P.n_patches; ++p) {
        const PatchMeta& m = P.meta[p];
        for (int s = 0; s < m.n_el; ++s, ++e)
            for (int i = 0; i < nb; ++i)
                el[size_t(e) * nb + i] =
                    P.pnode[m.node_off + P.lconn[size_t(i) * P.n_slots + size_t(p) * kPatch + s]] & kNodeMask;
    }
    std::vector<int64_t> cnt(n + 1, 0);
    for (int32_t v : el) ++cnt[v + 1];
    for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    std::vector<int32_t> inc(el.size());
    {
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
        for (size_t k = 0; k < el.size(); ++k) inc[fill[el[k]]++] = int32_t(k / nb);
    }
    std::vector<int32_t> ptr(n + 1, 0), nbr;
    std::vector<float> invdeg(n);
    nbr.reserve(size_t(n) * 7);
    std::vector<int32_t> tmp;
    for (int64_t v = 0; v < n; ++v) {
        tmp.clear();
        for (int64_t k = cnt[v]; k < cnt[v + 1]; ++k)
            for (int i = 0; i < nb; ++i) {
                const int32_t u = el[size_t(inc[k]) * nb + i];
                if (u != v) tmp.push_back(u);
            }
        std::sort(tmp.begin(), tmp.end());
        tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
        nbr.insert(nbr.end(), tmp.begin(), tmp.end());
        if (nbr.size() > size_t(INT32_MAX)) return fail(h, EBE_INVALID_ARG, "mesh graph exceeds 2^31 entries");
        ptr[v + 1] = int32_t(nbr.size());
        invdeg[v] = tmp.empty() ? 0.0f : 1.0f / float(tmp.size());
    }
    TRY(upload(h, &h->g_ptr, ptr.data(), int64_t(ptr.size())));
    TRY(upload(h, &h->g_nbr, nbr.data(), int64_t(nbr.size())));
    TRY(upload(h, &h->g_invdeg, invdeg.data(), int64_t(invdeg.size())));
    CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    return EBE_OK;
}

int net_buffers(ebe_mpnn* m, int64_t n, bool train) {
    MpnnDev& d = m->md;
    if (n > m->cap_inf) {
        MTRY(malloc_net(m, &d.h[0], n * kMpnnHidden));
        MTRY(malloc_net(m, &d.h[1], n * kMpnnHidden));
        m->cap_inf = n;
        m->cap_train = 0;   // training layers reuse h[0], h[1]
    }
    if (train && n > m->cap_train) {
        for (int l = 2; l <= kMpnnLayers; ++l) MTRY(malloc_net(m, &d.h[l], n * kMpnnHidden));
        if (n > m->cap_inf) return EBE_INVALID_ARG;
        MTRY(malloc_net(m, &d.save_u, int64_t(kMpnnLayers) * n * 2 * kMpnnHidden));
        MTRY(malloc_net(m, &d.save_v, int64_t(kMpnnLayers) * n * kMpnnHidden));
        MTRY(malloc_net(m, &d.save_x, 2 * n));
        MTRY(malloc_net(m, &d.gh, n * kMpnnHidden));
        MTRY(malloc_net(m, &d.ghp, n * kMpnnHidden));
        MTRY(malloc_net(m, &d.ga, n * kMpnnHidden));
        m->cap_train = n;
    }
    if (n > m->cap_vec) {
        MTRY(malloc_net(m, &m->z, n));
        MTRY(malloc_net(m, &m->w, n));
        MTRY(malloc_net(m, &m->aw, n));
        MTRY(malloc_net(m, &m->ae, n));
        MTRY(malloc_net(m, &m->gz, n));
        m->cap_vec = n;
    }
    return EBE_OK;
}

// Bind the network to the handle's mesh for the next launches.
int net_bind(ebe_mpnn* m, ebe_handle* h, bool train) {
    if (!m || !h) return EBE_INVALID_ARG;
    if (m->device != h->device) return fail(h, EBE_INVALID_ARG, "network and handle are on different devices");
    TRY(check_ready(h, true));
    DeviceGuard dev(h->device);
    TRY(ensure_mesh_graph(h));
    const int s = net_buffers(m, h->plan.n_n, train);
    if (s != EBE_OK) return fail(h, s, "network buffers: " + m->msg);
    m->md.nbr_ptr = h->g_ptr;
    m->md.nbr = h->g_nbr;
    m->md.inv_deg = h->g_invdeg;
    m->md.num_sms = h->pd.num_sms;
    return EBE_OK;
}

int net_check_device(ebe_handle* h, ebe_mpnn* m) {
    int32_t e = 0;
    CK(cudaMemcpyAsync(&e, m->err, sizeof(e), cudaMemcpyDeviceToHost, h->st), "read device flag");
    CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    if (e != 0) return fail(h, EBE_CUDA_ERROR, "a device-side wait timed out in the network (tensor-core result missing)");
    return EBE_OK;
}

}  // namespace
}  // extern "C++"

int64_t ebe_mpnn_n_params(void) { return kMpnnParams; }

ebe_status ebe_mpnn_create(ebe_mpnn** out, int32_t device, const double* theta) {
    if (!out) return EBE_INVALID_ARG;
    *out = nullptr;
    ebe_mpnn* m = new (std::nothrow) ebe_mpnn();
    if (!m) return EBE_OOM;
    m->device = device;
    auto bail = [&](int s) {
        g_create_error = m->msg;
        ebe_mpnn_destroy(m);
        return ebe_status(s);
    };
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        m->msg = "no such CUDA device";
        return bail(EBE_INVALID_ARG);
    }
    DeviceGuard dev(device);
    MpnnDev& d = m->md;
    int s = EBE_OK;
    if ((s = malloc_net(m, &d.theta, kMpnnParams)) || (s = malloc_net(m, &d.adam_m, kMpnnParams, true)) ||
        (s = malloc_net(m, &d.adam_v, kMpnnParams, true)) || (s = malloc_net(m, &d.wl, kMpnnLayers * 2 * kMpnnHidden * kMpnnHidden, true)) ||
        (s = malloc_net(m, &d.wT, kMpnnLayers * 2 * kMpnnHidden * kMpnnHidden)) || (s = malloc_net(m, &d.wsm, kMpnnSmall)) ||
        (s = malloc_net(m, &m->grad, kMpnnParams, true)) || (s = malloc_net(m, &d.part, 256 * (2 * kMpnnHidden * kMpnnHidden + kMpnnHidden))) ||
        (s = malloc_net(m, &d.ctr, 1, true)) || (s = malloc_net(m, &d.sc, 8, true)) || (s = malloc_net(m, &m->err, 1, true)))
        return bail(s);
    d.err = m->err;
    s = int(ebe_mpnn_set_params(m, theta));
    if (s != EBE_OK) return bail(s);
    *out = m;
    return EBE_OK;
}

void ebe_mpnn_destroy(ebe_mpnn* m) {
    if (!m) return;
    DeviceGuard dev(m->device);
    cudaDeviceSynchronize();
    for (void* p : m->allocs) cudaFree(p);
    delete m;
}

ebe_status ebe_mpnn_set_params(ebe_mpnn* m, const double* theta) {
    if (!m) return EBE_INVALID_ARG;
    std::vector<float> t(kMpnnParams, 0.0f);
    if (theta) {
        for (int k = 0; k < kMpnnParams; ++k) {
            if (!std::isfinite(theta[k])) return ebe_status(mfail(m, EBE_INVALID_ARG, "parameters must be finite"));
            t[k] = float(theta[k]);
        }
    } else {
        // seeded default: uniform +-1/sqrt(fan_in) layers, zero decoder (the Jacobi preconditioner)
        uint64_t st = 0x9E3779B97F4A7C15ull;
        auto uni = [&]() {
            st ^= st << 13; st ^= st >> 7; st ^= st << 17;
            return double(st >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
        };
        for (int k = 0; k < 2 * kMpnnHidden; ++k) t[k] = float(uni() / std::sqrt(2.0));
        for (int l = 0; l < kMpnnLayers; ++l)
            for (int k = 0; k < 2 * kMpnnHidden * kMpnnHidden; ++k)
                t[kMpnnW0 + l * kMpnnLayerParams + k] = float(uni() / std::sqrt(2.0 * kMpnnHidden));
    }
    DeviceGuard dev(m->device);
    if (cudaMemcpy(m->md.theta, t.data(), sizeof(float) * kMpnnParams, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->md.adam_m, 0, sizeof(float) * kMpnnParams) != cudaSuccess ||
        cudaMemset(m->md.adam_v, 0, sizeof(float) * kMpnnParams) != cudaSuccess)
        return ebe_status(mfail(m, EBE_CUDA_ERROR, "upload of the parameters failed"));
    m->step = 0;
    if (launch_mpnn_pack(m->md, nullptr, nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return ebe_status(mfail(m, EBE_CUDA_ERROR, "packing the parameters failed"));
    return EBE_OK;
}

ebe_status ebe_mpnn_get_params(const ebe_mpnn* m, double* theta) {
    if (!m || !theta) return EBE_INVALID_ARG;
    std::vector<float> t(kMpnnParams);
    DeviceGuard dev(m->device);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(t.data(), m->md.theta, sizeof(float) * kMpnnParams, cudaMemcpyDeviceToHost) != cudaSuccess)
        return EBE_CUDA_ERROR;
    std::copy(t.begin(), t.end(), theta);
    return EBE_OK;
}

ebe_status ebe_mpnn_apply(ebe_mpnn* m, ebe_handle* h, const double* r, double* z) {
    if (!r || !z) return EBE_INVALID_ARG;
    TRY(net_bind(m, h, false));
    Scope scp(h);
    int l = 0;
    CK(launch_mpnn_forward(m->md, h->plan.n_n, r, h->dinv, z, false, h->st, &l), "network forward");
    add_launches(h, l);
    return ebe_status(net_check_device(h, m));
}

ebe_status ebe_mpnn_grad(ebe_mpnn* m, ebe_handle* h, const double* r, const double* gz, double* z_out, double* grad) {
    if (!r || !gz || !grad) return EBE_INVALID_ARG;
    TRY(net_bind(m, h, true));
    Scope scp(h);
    const int64_t n = h->plan.n_n;
    int l = 0;
    CK(launch_mpnn_forward(m->md, n, r, h->dinv, m->z, true, h->st, &l), "network forward");
    CK(launch_mpnn_backward(m->md, n, gz, h->dinv, m->grad, h->st, &l), "network backward");
    add_launches(h, l);
    if (z_out) CK(cudaMemcpyAsync(z_out, m->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st), "copy z");
    CK(cudaMemcpyAsync(grad, m->grad, sizeof(double) * kMpnnParams, cudaMemcpyDeviceToHost, h->st), "copy gradient");
    return ebe_status(net_check_device(h, m));
}

ebe_status ebe_mpnn_train_step(ebe_mpnn* m, ebe_handle* h, const double* r, const double* e, double lr, double* loss) {
    if (!r || !e || !(lr > 0.0) || !std::isfinite(lr)) return EBE_INVALID_ARG;
    TRY(net_bind(m, h, true));
    Scope scp(h);
    const int64_t n = h->plan.n_n;
    TRY(dalloc(h, &h->halo64, std::max<int64_t>(h->plan.n_halo, 1)));
    int l = 0;
    double* sc = m->md.sc;
    CK(launch_mpnn_forward(m->md, n, r, h->dinv, m->z, true, h->st, &l), "network forward");
    CK(launch_sub(n, e, m->z, m->w, h->st, &l), "e - z");
    CK(launch_patch_pass(h->pd, 0, kApply, h->A64, m->w, nullptr, m->aw, h->halo64, h->part_patch, nullptr, h->sc, h->st,
                         &l), "A (e - z)");
    CK(launch_patch_pass(h->pd, 0, kApply, h->A64, e, nullptr, m->ae, h->halo64, h->part_patch, nullptr, h->sc, h->st, &l),
       "A e");
    CK(launch_dot2(n, m->w, m->aw, nullptr, m->md.part, m->md.ctr, sc + 2, h->st, &l), "w'Aw");
    CK(launch_dot2(n, e, m->ae, nullptr, m->md.part, m->md.ctr, sc + 4, h->st, &l), "e'Ae");
    CK(launch_scale(n, m->aw, sc + 4, -2.0, m->gz, h->st, &l), "dL/dz");
    CK(launch_mpnn_backward(m->md, n, m->gz, h->dinv, m->grad, h->st, &l), "network backward");
    m->step += 1;
    CK(launch_mpnn_adam(m->md, m->grad, float(lr), m->step, h->st, &l), "Adam");
    add_launches(h, l);
    double v[6];
    CK(cudaMemcpyAsync(v, sc, sizeof(v), cudaMemcpyDeviceToHost, h->st), "read loss");
    TRY(net_check_device(h, m));
    if (loss) *loss = v[4] > 0.0 ? v[2] / v[4] : 0.0;
    return EBE_OK;
}

const char* ebe_mpnn_last_error(const ebe_mpnn* m) { return m ? m->msg.c_str() : g_create_error.c_str(); }

namespace {

// Flexible CG (one stored direction) with the network (or Jacobi) as the
// preconditioner, FP64 vectors and FP64 element matrices.  On a breakdown or
// when the residual stops decreasing, the solve falls back to Jacobi from the
// current iterate.
int learned_impl(ebe_handle* h, ebe_mpnn* net, double* x, bool x_on_host, const ebe_solve_opts& o, ebe_solve_info& info,
                 int32_t* fell_back) {
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t n = h->plan.n_n;
    const int64_t nh = std::max<int64_t>(h->plan.n_halo, 1);
    TRY(dalloc(h, &h->x64w, n));
    TRY(dalloc(h, &h->r64, n));
    TRY(dalloc(h, &h->p64, n));
    TRY(dalloc(h, &h->q64, n));
    TRY(dalloc(h, &h->z64, n));
    TRY(dalloc(h, &h->halo64, nh));
    if (net) TRY(net_bind(net, h, false));
    bool use_net = net != nullptr;
    if (fell_back) *fell_back = 0;
    int l = 0;
    CK(cudaMemcpyAsync(h->x64w, x, sizeof(double) * n, x_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       h->st), "copy x0");
    CK(launch_set_dirichlet(h->x64w, h->nd, h->g, h->n_d, h->st, &l), "x(nd) = g");
    CK(launch_control(h->sc, 0.0, o.maxit, 1, h->st, &l), "control");
    add_launches(h, l);
    double rr = 0.0;
    TRY(true_residual(h, rr));
    info.true_residuals = 1;
    const double r0 = std::sqrt(rr);
    info.r0_norm = r0;
    info.iterations = 0;
    info.rel_residual = r0 > 0.0 ? 1.0 : 0.0;
    int status = EBE_OK;
    if (!std::isfinite(r0)) status = EBE_BREAKDOWN;
    if (r0 > 0.0 && std::isfinite(r0)) {
        const double target = o.rtol * r0;
        l = 0;
        CK(launch_control(h->sc, target * target, -1, 0, h->st, &l), "control");
        add_launches(h, l);
        int first = 1;
        double best = 1.0, best_rr = rr;
        int no_progress = 0, flat_chunks = 0;
        // giving up on the network: the solve is finished by the library's
        // Jacobi-PCG (the plain FP64 solver) from the current iterate
        bool to_pcg = false;
        auto fallback = [&]() -> int {
            use_net = false;
            to_pcg = true;
            if (fell_back) *fell_back = 1;
            return EBE_OK;
        };
        // `iters` FCG iterations with the current preconditioner, enqueued
        auto enqueue = [&](int iters) -> int {
            int ll = 0;
            for (int it = 0; it < iters; ++it) {
                if (use_net) CK(launch_mpnn_forward(net->md, n, h->r64, h->dinv, h->z64, false, h->st, &ll), "network");
                else CK(launch_jacobi(n, h->r64, h->dinv, h->z64, &h->sc->done, h->st, &ll), "Jacobi");
                CK(launch_fcg_dots(n, h->z64, h->r64, h->p64, h->q64, first, h->part_vec, h->sc, h->st, &ll), "FCG dots");
                CK(launch_fcg_dir(n, h->z64, h->p64, first, h->sc, h->st, &ll), "FCG direction");
                CK(launch_patch_pass(h->pd, 0, kApplyDot, h->A64, h->p64, nullptr, h->q64, h->halo64, h->part_patch,
                                     &h->sc->done, h->sc, h->st, &ll), "apply");
                CK(launch_update(0, n, h->x64w, h->p64, h->r64, h->q64, h->dinv, h->part_vec, h->sc, h->st, &ll),
                   "update");
                first = 0;
            }
            add_launches(h, ll);
            return EBE_OK;
        };
        // With a network, a race first decides whether to use it: from x0,
        // kRace iterations of Jacobi-FCG and then, again from x0, kRace
        // iterations with the network, each timed with CUDA events on the
        // stream; the preconditioner with the larger reduction of the
        // residual norm per unit time continues (the network from its own
        // iterate, Jacobi from its saved one).  A network that loses costs
        // its kRace timed iterations and one restart.  A network that wins
        // must keep Jacobi's early rate over every window of kWindow chunks
        // (CG's rate falls as it proceeds, so this errs towards Jacobi).
        bool pending = false;          // scalars already read: process them before launching
        // Jacobi's rate in the race (log of the residual-norm reduction per ms);
        // the network keeps it up, measured over windows of kWindow chunks, or
        // the solve falls back to Jacobi
        double rate_jac = 0.0;
        constexpr int kWindow = 2;            // chunks per check of the network's rate
        constexpr int kRaceDefault = 16;      // iterations of each leg of the race
        constexpr double kRaceMargin = 1.5;   // the network must beat Jacobi's early rate by this factor
        struct Events {
            cudaEvent_t e[2] = {nullptr, nullptr};
            ~Events() { for (auto& v : e) if (v) cudaEventDestroy(v); }
        } evs;
        CK(cudaEventCreate(&evs.e[0]), "cudaEventCreate");
        CK(cudaEventCreate(&evs.e[1]), "cudaEventCreate");
        if (use_net && o.race_iters != 0) {
            const int kRace = o.race_iters > 0 ? o.race_iters : kRaceDefault;
            TRY(dalloc(h, &h->xsave0, n));
            TRY(dalloc(h, &h->xsave1, n));
            cudaEvent_t* ev = evs.e;
            auto timed = [&](double& ms) -> int {
                CK(cudaEventRecord(ev[0], h->st), "cudaEventRecord");
                TRY(enqueue(kRace));
                CK(cudaEventRecord(ev[1], h->st), "cudaEventRecord");
                TRY(sync_scalars(h));
                float t = 0.f;
                CK(cudaEventElapsedTime(&t, ev[0], ev[1]), "cudaEventElapsedTime");
                ms = double(t);
                return EBE_OK;
            };
            int rs = EBE_OK;
            double t_jac = 0.0, t_net = 0.0, rr_jac = rr, rr_net = rr;
            CK(cudaMemcpyAsync(h->xsave0, h->x64w, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st), "save x0");
            use_net = false;
            first = 1;
            rs = timed(t_jac);
            if (rs == EBE_OK && h->sc_host->reason != kRunning) {
                pending = true;        // Jacobi alone already reached rtol |r0| (or stopped): no race
                if (fell_back) *fell_back = 1;
            } else if (rs == EBE_OK) {
                rr_jac = h->sc_host->rr;
                CK(cudaMemcpyAsync(h->xsave1, h->x64w, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st), "save");
                CK(cudaMemcpyAsync(h->x64w, h->xsave0, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st), "x0");
                double t = 0.0;
                rs = true_residual(h, t);
                info.true_residuals += 1;
                use_net = true;
                first = 1;
                if (rs == EBE_OK) rs = timed(t_net);
                if (rs == EBE_OK) rs = net_check_device(h, net);
                if (rs == EBE_OK && h->sc_host->reason != kRunning) {
                    pending = true;
                } else if (rs == EBE_OK) {
                    rr_net = h->sc_host->rr;
                    rate_jac = std::log(rr / rr_jac) / t_jac;
                    const double rate_net = std::log(rr / rr_net) / t_net;
                    // CG's residual norm need not fall in its first iterations:
                    // a race in which Jacobi's did not fall decides nothing, and
                    // Jacobi-PCG continues
                    if (!(rate_jac > 0.0) || !(rate_net > kRaceMargin * rate_jac)) {
                        // Jacobi-PCG continues from the Jacobi leg's iterate
                        CK(cudaMemcpyAsync(h->x64w, h->xsave1, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st),
                           "restore");
                        rs = fallback();
                    } else {
                        best_rr = rr_net;
                    }
                }
            }
            TRY(rs);
        }
        double win_ms = 0.0, win_rr = h->sc_host->rr;
        int win_chunks = 0;
        for (;;) {
            if (to_pcg) break;
            const bool watch = use_net && rate_jac > 0.0 && !pending;
            if (watch) CK(cudaEventRecord(evs.e[0], h->st), "cudaEventRecord");
            if (!pending) TRY(enqueue(o.chunk));
            if (watch) CK(cudaEventRecord(evs.e[1], h->st), "cudaEventRecord");
            pending = false;
            const int64_t before = info.iterations;
            TRY(sync_scalars(h));
            if (use_net) TRY(net_check_device(h, net));
            const Scalars sh = *h->sc_host;
            info.iterations = sh.iter;
            if (sh.reason == kRunning) {
                if (sh.iter == before) return fail(h, EBE_CUDA_ERROR, "solver chunk made no progress");
                if (watch) {
                    float t = 0.f;
                    CK(cudaEventElapsedTime(&t, evs.e[0], evs.e[1]), "cudaEventElapsedTime");
                    win_ms += double(t);
                    if (++win_chunks == kWindow) {
                        const double rate = std::log(win_rr / sh.rr) / win_ms;
                        win_ms = 0.0;
                        win_chunks = 0;
                        win_rr = sh.rr;
                        if (!(rate >= rate_jac)) { TRY(fallback()); continue; }
                    }
                }
                if (use_net) {
                    // the learned step must keep reducing the residual: at least
                    // a halving every 16 chunks (Jacobi-CG halves it about every
                    // 0.1 sqrt(n_n) iterations on the 2D model problems)
                    if (!(sh.rr < 0.25 * best_rr)) {
                        if (++flat_chunks >= 16) TRY(fallback());
                    } else {
                        best_rr = sh.rr;
                        flat_chunks = 0;
                    }
                }
                continue;
            }
            if (sh.reason == kBreakdown) {
                if (use_net) { TRY(fallback()); continue; }
                status = EBE_BREAKDOWN;
                break;
            }
            TRY(true_residual(h, rr));
            info.true_residuals += 1;
            const double rel = std::sqrt(rr) / r0;
            info.rel_residual = rel;
            if (!std::isfinite(rel)) {
                if (use_net) { TRY(fallback()); continue; }
                status = EBE_BREAKDOWN;
                break;
            }
            if (rel <= o.rtol) { status = EBE_OK; break; }
            if (sh.reason == kMaxit) { status = EBE_MAXIT; break; }
            if (rel < 0.9 * best) { best = rel; no_progress = 0; }
            else if (++no_progress >= o.stall_updates) {
                if (use_net) { TRY(fallback()); no_progress = 0; continue; }
                status = EBE_STALL;
                break;
            }
            // residual replacement: restart the flexible recurrence from the true residual
            first = 1;
            l = 0;
            CK(launch_control(h->sc, -1.0, -1, 0, h->st, &l), "control");
            add_launches(h, l);
        }
        if (to_pcg) {
            // Jacobi-PCG from the current iterate, to the same target rtol |r0|
            // of the original start: the single-sync mixed solver when the FP32
            // element matrices are stored, else the FP64 one
            TRY(dalloc(h, &h->xsave1, n));
            double rr_now = 0.0;
            TRY(true_residual(h, rr_now));
            info.true_residuals += 1;
            const double r_now = std::sqrt(rr_now);
            if (!std::isfinite(r_now)) {
                status = EBE_BREAKDOWN;
            } else if (r_now <= o.rtol * r0) {
                info.rel_residual = r_now / r0;
                status = EBE_OK;
            } else {
                CK(cudaMemcpyAsync(h->xsave1, h->x64w, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st), "save x");
                ebe_solve_opts po = o;
                po.precision = h->store == EBE_STORE_MIXED ? EBE_PREC_MIXED : EBE_PREC_FP64;
                po.rtol = o.rtol * r0 / r_now;
                po.maxit = std::max<int64_t>(1, o.maxit - info.iterations);
                po.use_graph = 1;
                ebe_solve_info pi{};
                status = po.precision == EBE_PREC_MIXED ? solve_cg1_impl(h, h->xsave1, false, po, pi)
                                                        : solve_impl(h, h->xsave1, false, po, pi);
                if (status != EBE_OK && status != EBE_MAXIT && status != EBE_STALL && status != EBE_BREAKDOWN)
                    return status;
                CK(cudaMemcpyAsync(h->x64w, h->xsave1, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st), "x");
                info.iterations += pi.iterations;
                info.true_residuals += pi.true_residuals;
                info.rel_residual = pi.rel_residual * r_now / r0;
            }
        }
    }
    CK(cudaMemcpyAsync(x, h->x64w, sizeof(double) * n, x_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                       h->st), "copy x");
    CK(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    info.status = status;
    info.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return status;
}

}  // namespace

ebe_status ebe_solve_learned(ebe_handle* h, ebe_mpnn* net, double* x, const ebe_solve_opts* opts, ebe_solve_info* info,
                             int32_t* fell_back) {
    TRY(check_ready(h, true));
    if (!x) return ebe_status(fail(h, EBE_INVALID_ARG, "x is NULL"));
    ebe_solve_opts o;
    ebe_solve_opts_default(&o);
    if (opts) o = *opts;
    if (!(o.rtol > 0.0) || o.maxit < 1 || o.chunk < 1 || o.chunk > 4096 || o.stall_updates < 1)
        return ebe_status(fail(h, EBE_INVALID_ARG, "bad solve options"));
    ebe_solve_info local{};
    Scope scp(h);
    const int s = learned_impl(h, net, x, false, o, local, fell_back);
    if (info) *info = local;
    return ebe_status(s);
}

ebe_status ebe_get_stats(const ebe_handle* h, ebe_stats* s) {
    if (!h || !s) return EBE_INVALID_ARG;
    s->kernel_launches = h->launches;
    s->n_patches = h->plan.n_patches;
    s->patch_elems = kPatch;
    s->n_shared_nodes = int64_t(h->plan.sh_node.size());
    s->n_halo = h->plan.n_halo;
    s->max_colours = h->plan.max_col;
    s->n_global_colours = h->n_gcol;
    s->device_bytes = h->bytes;
    s->device_error = 0;
    if (h->dev_err) {
        int32_t e = 0;
        DeviceGuard dev(h->device);
        if (cudaMemcpyAsync(&e, h->dev_err, sizeof(e), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
            cudaStreamSynchronize(h->st) != cudaSuccess)
            return EBE_CUDA_ERROR;
        s->device_error = e;
    }
    return EBE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free residual
// Some callers cannot call cudaMalloc at the point where they need a
// residual: a process whose device memory is handed out by another allocator
// (a framework's caching allocator or a fixed pool that owns the device), or
// a real-time loop that must not take the allocator's locks or risk the
// implicit device synchronisation of cudaMalloc.  ebe_residual allocates its halo scratch on first use;
// ebe_residual_noalloc takes it from a fixed file-scope device array
// instead: kNoAllocHaloMax doubles (32 MiB), present on every device that
// loads the library for the life of the process.  Every call shares the
// array, so calls whose kernels overlap on the GPU (several streams or
// handles at once) race on it.  Each halo slot is written by the patch pass
// before the fix-up pass reads it, so nothing in the array needs clearing.
namespace {

constexpr int64_t kNoAllocHaloMax = int64_t(1) << 22;
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) double g_noalloc_halo[kNoAllocHaloMax];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the handle's device (in host code
// the array's name is only a stand-in).  Looked up once per device; the
// caller has made the handle's device current.
int noalloc_scratch(ebe_handle* h, double** out) {
    if (h->device < 0 || h->device >= kNoAllocMaxDevices) return fail(h, EBE_INVALID_ARG, "device ordinal too large");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[h->device]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_noalloc_halo), "cudaGetSymbolAddress");
        g_noalloc_addr[h->device] = p;
    }
    *out = static_cast<double*>(g_noalloc_addr[h->device]);
    return EBE_OK;
}

}  // namespace

extern "C" ebe_status ebe_residual_noalloc(ebe_handle* h, const double* x, double* r) {
    TRY(check_ready(h, true));
    if (!x || !r || x == r) return ebe_status(fail(h, EBE_INVALID_ARG, "x and r must be distinct non-NULL device buffers"));
    if (h->plan.n_halo > kNoAllocHaloMax)
        return ebe_status(fail(h, EBE_INVALID_ARG,
                               "mesh needs " + std::to_string(h->plan.n_halo) + " halo slots; ebe_residual_noalloc holds " +
                                   std::to_string(kNoAllocHaloMax) + " (use ebe_residual)"));
    Scope scp(h);
    double* halo = nullptr;
    TRY(noalloc_scratch(h, &halo));
    int l = 0;
    CK(launch_patch_pass(h->pd, 0, kResidual, h->A64, x, h->b, r, halo, h->part_patch, nullptr, h->sc, h->st, &l),
       "patch pass");
    add_launches(h, l);
    return EBE_OK;
}
