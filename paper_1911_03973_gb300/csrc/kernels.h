// Device-side views, solver scalars and kernel launchers of libebe.so.
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#include "ebe_internal.h"

namespace ebe {

// Read-only view of the element partition on the device.
struct PlanDev {
    int nb = 0;
    int dim = 0;
    int64_t n_slots = 0;
    int n_patches = 0;
    int n_shared = 0;
    int64_t n_halo = 0;                 // halo slots (sh_ptr[n_shared])
    int max_nodes = 0;
    int max_col = 0;
    const PatchMeta* meta = nullptr;
    const int32_t* pnode = nullptr;     // local-node tables, bit 31 = Dirichlet
    const uint16_t* lconn = nullptr;    // [nb][n_slots]
    const int32_t* col_ptr = nullptr;
    const int32_t* sh_node = nullptr;   // bit 31 = Dirichlet
    const int32_t* sh_ptr = nullptr;
    const int32_t* sh_slot = nullptr;
    const int32_t* slot_elem = nullptr; // [n_slots], -1 = padding
    int32_t* err = nullptr;             // set to 1 when a bounded device wait gives up
    int num_sms = 1;                    // persistent grid size of the patch pass
    // Solver numbering (set in the view of the single-sync solver only): the
    // owned nodes of patch p are nodes own_off[p] + l, l < n_owned (one
    // contiguous run per patch, padded to a multiple of 4), and shared row k
    // of the fix-up is node sh_base + k.
    const int32_t* own_off = nullptr;   // [n_patches + 1]
    int sh_base = 0;
    // [n_halo] position of each halo slot in the shared rows' CSR order
    // (halo_pos[sh_slot[j]] = j), so that the single-sync fix-up reads a row's
    // partials contiguously
    const int32_t* halo_pos = nullptr;
};

// Element matrices are symmetric (K_e and M_e of Eq. matrices_K_M; the
// closed forms give a_ij and a_ji from the same products, so they are equal
// bit for bit) and are stored packed: sym_count(nb) slot-major runs of
// n_slots values, the nb diagonal entries first, then the pairs i < j in the
// order (0,1), (0,2), (1,2), (0,3), (1,3), (2,3).
__host__ __device__ constexpr int sym_count(int nb) { return nb * (nb + 1) / 2; }
// Layout of the FP32-pair copy of A_e (the double-word residual): tetrahedra
// keep each entry's hi and lo side by side (one 8-byte load), triangles keep
// all hi runs and then all lo runs.  Measured on GB300 (warm, per residual,
// with the products formed before the colour rounds): 129^3 tetrahedra 365 us
// side by side against 397 us separate; 2049^2 triangles 162 us separate
// against 170 us side by side.
__host__ __device__ constexpr bool dw_pairs(int nb) { return nb == 4; }
__host__ __device__ constexpr int sym_index(int nb, int i, int j) {
    return i == j ? i : nb + (i < j ? j * (j - 1) / 2 + i : i * (i - 1) / 2 + j);
}

// What a patch pass produces at the nodes.
enum PatchMode : int {
    kResidual = 0,      // out = mask(b - A x)
    kResidualNorm = 1,  // same, and sum of out^2 -> Scalars::rrt
    kApply = 2,         // out = mask(A x)
    kApplyDot = 3       // same, and sum of x.out -> Scalars::pq, alpha = rho / pq
};

// Why a solver graph stopped (Scalars::reason).
enum StopReason : int { kRunning = 0, kTrigger = 1, kBreakdown = 2, kMaxit = 3 };

// Factor by which a mixed-precision solver's final recurrence threshold
// (first rtol |r0|) tightens after an FP64 true-residual check at that
// threshold has failed.
constexpr double kFinalMargin = 0.7;

// Solver scalars, kept on the device between kernels of an iteration.
struct Scalars {
    double rho;      // r.z of the current direction
    double alpha;    // rho / p.Ap
    double beta;     // rho_new / rho
    double pq;       // p.Ap
    double rr;       // recurrence r.r after the last update
    double rz;       // recurrence r.z after the last update
    double rrt;      // last true-residual r.r (kResidualNorm)
    double thr2;     // stop the graph once rr <= thr2
    int64_t iter;    // CG iterations done
    int64_t maxit;
    int32_t done;    // nonzero: every solver kernel returns at once
    int32_t reason;  // StopReason
    uint32_t ctr_fix;   // arrival counters of the last-block reductions
    uint32_t ctr_vec;
    // single-sync iteration (launch_cg_pass)
    double qz;       // q.z of the last pass (z = dinv r)
    double qdq;      // q.(dinv q) of the last pass
    int64_t passes;  // passes that ran to completion (parity of the two direction buffers)
    int32_t fresh;   // the next pass starts from a new residual: no update, no iteration counted
    int32_t pad;
};

// Launch with programmatic stream serialisation: the kernel may start while
// the previous kernel in the stream drains; it synchronises with
// griddepcontrol.wait before reading that kernel's results.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Fixed grid of the node-vector kernels for n nodes (deterministic partials).
int vec_grid(int64_t n);
// Fix-up grid: `rows` shared rows per thread at a time (1 or 2), at most
// kFixGridMax blocks.
constexpr int kFixGridMax = 1216;
int fix_grid(int n_shared, int rows = 1);
// Rows per fix-up thread for this partition: 2 (their loads interleaved) when
// a shared node has at most 2.5 halo slots on average, else 1.
int fix_rows(const PlanDev& pd);
constexpr int kVecThreads = 256;

// ---- patch passes (k_patch.cu) -------------------------------------------
// dtype 0 = double (FP64 A_e), 1 = float (FP32 A_e).  part must hold
// n_patches + fix_grid(n_shared) doubles; halo n_halo values of the dtype.
// stop (nullable): the pass does nothing when *stop != 0 (solver graphs).
// sc: receives the norm / dot of kResidualNorm / kApplyDot.
// ev (nullable): three events recorded before the patch kernel, between it
// and the fix-up kernel, and after the fix-up.  pdl: launch both kernels with
// programmatic dependent launch (only where the element matrices cannot have
// been written by the preceding kernel, i.e. inside a solver iteration).
cudaError_t launch_patch_pass(const PlanDev& pd, int dtype, int mode, const void* A, const void* x,
                              const void* b, void* out, void* halo, double* part, const int32_t* stop,
                              Scalars* sc, cudaStream_t st, int* launches, cudaEvent_t* ev = nullptr,
                              bool pdl = false);

// ---- double-word FP64 residual (k_patch.cu) -----------------------------
// The FP64 residual / operator (modes kResidual, kResidualNorm, kApply) with
// A_e stored as FP32 pairs a = hi + lo in Adw (2 * n entries of FP32, n =
// sym_count(nb) * n_slots, in the FP64 layout's entry runs of n_slots): with
// dw_pairs(nb) each entry is one float2 (hi, lo); otherwise all hi runs come
// first and the lo runs follow at Adw + n.  The arithmetic is double-word
// FP32; x, b, out FP64; halo: n_halo pairs (the FP64 halo buffer
// reinterpreted).
cudaError_t launch_patch_pass_dw(const PlanDev& pd, int mode, const float* Adw, const double* x,
                                 const double* b, double* out, double* halo, double* part, const int32_t* stop,
                                 Scalars* sc, cudaStream_t st, int* launches, cudaEvent_t* ev = nullptr);
// Fills Adw from a (n FP64 entries) in the layout above for element type nb:
// hi + lo = a[i] to 48 bits.
cudaError_t launch_split_dw(int64_t n, const double* a, float* out, int nb, cudaStream_t st, int* launches);

// ---- single-synchronisation mixed-precision CG (k_patch.cu) ---------------
// One pass = one CG iteration in two launches (patch pass + shared-node
// fix-up), all node vectors in the solver numbering (pd.own_off set), FP32
// except x:
//   r <- r - alpha q;  x <- x + alpha p_old;  z = dinv r;  p_new = z + beta p_old;
//   q <- mask(A p_new) (FP32 difference-form element matrices A);
//   sums r.z, r.r, p_new.q, q.z, q.(dinv q) -> the last fix-up block sets
//   alpha = r.z / p.q, beta = rho_next / r.z with
//   rho_next = r.z - 2 alpha q.z + alpha^2 q.(dinv q) (= r'.(dinv r') of the
//   next residual r' = r - alpha q), counts the iteration and takes the stop
//   decisions of the textbook update step (trigger on r.r <= thr2, maxit,
//   breakdown).  sc->fresh: alpha = 0 and no iteration (first pass after a
//   (re)start).  Dirichlet rows are those with dinv = 0.  part: 5 x
//   (n_patches + fix_grid(n_shared)) doubles.
// ev (nullable): three events around the two kernels, as launch_patch_pass.
cudaError_t launch_cg_pass(const PlanDev& pd, const float* A, float* r, float* q, const float* p_old, float* p_new,
                           const float* dinv, double* x, float* halo, double* part, Scalars* sc, cudaStream_t st,
                           int* launches, bool pdl = false, cudaEvent_t* ev = nullptr);
// alpha = 0, fresh = 1 (after a restart of the recurrence).
cudaError_t launch_cg_arm(Scalars* sc, cudaStream_t st, int* launches);
// dst[map[i]] = src[i] (to the solver numbering) or dst[i] = src[map[i]] (back), i < n.
cudaError_t launch_permute(int dtype, int to_solver, int64_t n, const int32_t* map, const void* src, void* dst,
                           cudaStream_t st, int* launches);
// dst[i] = (dst[i] & node mask) | (src[i] & Dirichlet bit), i < n.
cudaError_t launch_copy_dirichlet_bit(int32_t* dst, const int32_t* src, int64_t n, cudaStream_t st, int* launches);

// ---- element data (k_assemble.cu) -----------------------------------------
// Element matrices, load vector and Jacobi diagonal (FP64), Eq. matrices_K_M.
// nu_patch (nullable): nu of every patch (batches of problems); else nu.
cudaError_t launch_assemble(const PlanDev& pd, const double* coords, const double* f, double nu,
                            const double* nu_patch, double* A64, float* A32, double* b, double* d, double* dinv, float* b32,
                            float* dinv32, double* halo2, unsigned long long* bad, cudaStream_t st,
                            int* launches);
// K_e, M_e (or A_e) in the caller's element order, paper layout [e][j][i].
cudaError_t launch_export_km(const PlanDev& pd, const double* coords, double* K, double* M,
                             cudaStream_t st, int* launches);
cudaError_t launch_export_A(const PlanDev& pd, int dtype, const void* A, void* out, cudaStream_t st,
                            int* launches);
// Set / clear the Dirichlet bit of the node tables from a byte mask [n_n].
cudaError_t launch_mark_dirichlet(const PlanDev& pd, int32_t* pnode, int64_t n_pnode, int32_t* sh_node,
                                  const uint8_t* mask, cudaStream_t st, int* launches);

// ---- node-vector kernels (k_vec.cu) ---------------------------------------
cudaError_t launch_set_dirichlet(double* x, const int32_t* nd, const double* g, int64_t n_d,
                                 cudaStream_t st, int* launches);
// x += alpha p; r -= alpha q; sums r.(dinv r), r.r; stop test (last block).
// vt 0: x, r, dinv, p, q FP64.  vt 1: x FP64; r, p, q, dinv FP32.
cudaError_t launch_update(int vt, int64_t n, void* x, const void* p, void* r, const void* q,
                          const void* dinv, double* part, Scalars* sc, cudaStream_t st, int* launches,
                          bool pdl = false);
// p = dinv r + beta p  (init: p = dinv r); vt as launch_update (r FP32 for vt 1).
cudaError_t launch_direction(int vt, int64_t n, void* p, const void* r, const void* dinv, int init,
                             Scalars* sc, cudaStream_t st, int* launches, bool pdl = false);
// After a residual replacement: sums r.(dinv r) and r.r; beta = rz/rho, rho = rz
// (init: rho = rz, beta = 0).  FP64 r; dinv FP64 (vt 0) or FP32 (vt 1); for
// vt 1, r32 (if not NULL) receives (float) r.
cudaError_t launch_restart(int vt, int64_t n, const double* r, const void* dinv, int init, double* part,
                           Scalars* sc, cudaStream_t st, int* launches, float* r32 = nullptr);
// thr2 >= 0: new stop threshold; maxit >= 0: new cap; reset_iter: iter = 0.
// Always clears done / reason.
cudaError_t launch_control(Scalars* sc, double thr2, int64_t maxit, int reset_iter, cudaStream_t st, int* launches);
cudaError_t launch_fill(int dtype, int64_t n, void* v, double value, cudaStream_t st, int* launches);
// kind 0: x += w r; kind 1: p = r + beta p (beta = 0: p = r), x += w p.
cudaError_t launch_stationary(int64_t n, double* x, const double* r, double* p, int kind, double w, double beta,
                              cudaStream_t st, int* launches);

// ---- batched solver (k_batch.cu) ------------------------------------------
constexpr int kBatchMaxProblems = 4096;   // problems of one batch (a mode byte each in shared memory)

// Phase of one problem of a batch inside the persistent solver.
enum BatchMode : int32_t {
    kBNormal = 0,    // next iteration: q = A p, x and r updates, new direction
    kBReplace = 1,   // next iteration: FP64 true residual r = b - A x replaces r
    kBDone = 2       // finished (status set)
};

// Per-problem solver state of a batch, on the device (64-bit fields first).
struct BatchProblem {
    double rho;        // r.z of the current direction
    double alpha;      // rho / p.Ap
    double beta;       // direction factor of the next direction step
    double thr2;       // replacement threshold on the recurrence r.r
    double r0;         // |r0|, FP64 true residual of x0
    double rrt;        // last true-residual r.r
    double rel;        // last true relative residual
    double best;       // best true relative residual so far (stall test)
    double fin;        // final recurrence threshold: rtol r0 (mixed: times bd.margin per failed check at it)
    int64_t iter;      // CG iterations done
    int32_t mode;      // BatchMode
    int32_t status;    // ebe_status once done
    int32_t n_true;    // true residuals evaluated
    int32_t no_progress;
    int32_t init;      // the pending replacement is the initial residual
    int32_t bd;        // breakdown seen: finish after a last true residual
    int32_t dir_init;  // the pending direction step starts from p = z
    int32_t exact;     // mixed: the pending true residual in FP64, not in double-word form
};

// The mixed solvers take a residual replacement in double-word arithmetic
// while its threshold is at least kDwReplaceRel |r0|, and in FP64 below.  The
// double-word residual errs by about 2^-48 |A||x|, which near a solution is
// of the order of 1e-9 |r0| on the 2049^2 square (|A||x| / |b| grows like
// 1 / h^2): negligible against residuals of 1e-6 |r0| and above, not against
// the last checks before rtol.
constexpr double kDwReplaceRel = 1e-6;

// A work item of the fix-up or node phases: one problem's shared-node rows
// [lo, hi) (fix-up) or nodes [lo, hi) (node phases).  A fix-up item also
// adds the patch partials [plo, phi) of its problem.  The items of problem
// k are [first, first + count).
struct BatchItem {
    int32_t k, lo, hi, plo, phi, first, count, pad;
};

// Where the work items of one problem of a batch are: patches
// [patch_first, +patch_count), fix-up items [fix_first, +fix_count), node
// tiles [tile_first, +tile_count) (of the launch's tile size); all counts >= 1.
struct BatchProbInfo {
    int32_t patch_first, patch_count, fix_first, fix_count, tile_first, tile_count, pad0, pad1;
};

// Everything the persistent batched solver reads and writes.
struct BatchDev {
    PlanDev pd;
    int32_t n_prob = 0;
    int32_t n_fix = 0, n_tile = 0;
    const BatchProbInfo* pinfo = nullptr;  // [n_prob]
    const BatchItem* fix = nullptr;        // [n_fix]
    const BatchItem* tile = nullptr;       // [n_tile]
    const void* A = nullptr;               // element matrices of the inner operator (FP32 difference form or FP64)
    const double* A64 = nullptr;           // FP64 element matrices (true residuals, FP64 solver)
    const float* Adw = nullptr;            // mixed solver: A64 as FP32 pairs (double-word true residuals), dw_pairs layout
    const double* b = nullptr;             // FP64 load vector
    const void* dinv = nullptr;            // inverse Jacobi diagonal, inner type
    double* x = nullptr;
    double* r = nullptr;                   // FP64 true residual
    void* rin = nullptr;                   // recurrence residual, inner type (r itself for FP64)
    void* p = nullptr;                     // direction, inner type
    void* q = nullptr;                     // A p, inner type
    void* halo = nullptr;                  // halo partials, inner type
    double* halo64 = nullptr;
    double* part_p = nullptr;              // [n_patches]
    double* part_f = nullptr;              // [n_fix]
    double* part_u = nullptr;              // [2 n_tile]
    BatchProblem* prob = nullptr;          // [n_prob]
    uint32_t* ctr = nullptr;               // [2 n_prob] arrival counters: fix-up, node phase
    uint32_t* bar = nullptr;               // [2] grid barrier
    int32_t* live = nullptr;               // problems not done
    int64_t* loops = nullptr;              // iterations (of any kind) run by the persistent kernel
    unsigned long long* phase_ns = nullptr;   // [4] time of the phases P, F, U, D (barrier to barrier, CTA 0)
    double rtol = 1e-8, delta = 0.1, margin = kFinalMargin;
    int64_t maxit = 0;
    int32_t stall_updates = 8;
    int64_t iter_budget = 0;               // loop iterations of one launch
    uint64_t barrier_ns = 2000000000ull;   // bound of one grid-barrier wait
};

// Options and outcome of the one-CTA mixed-precision solver of small meshes.
struct SmallOpts {
    double rtol = 1e-8, delta = 0.1;
    int64_t maxit = 0;
    int32_t stall_updates = 8;
    int32_t pad = 0;
};
struct SmallInfo {
    int64_t iterations;
    int32_t true_residuals;
    int32_t status;        // ebe_status
    double r0;             // |r(x0)|, FP64
    double rel;            // last true relative residual
};
// A colouring of all elements of a small mesh (device arrays): element k of
// the colour order is slot order[k]; colour c holds elements [col[c], col[c+1]).
// Node v's incidences inc[inc_ptr[v] .. inc_ptr[v+1]) list its (element k,
// row r) pairs as k | r << 12, k ascending: the order in which the colour
// rounds add the element rows into the node.
constexpr int kSmallMaxColours = 64;
struct SmallColouring {
    const int32_t* order = nullptr;    // [n_e]
    const int32_t* col = nullptr;      // [n_col + 1]
    const int32_t* gconn = nullptr;    // [nb][n_slots] global node ids per slot
    const uint16_t* inc_ptr = nullptr; // [n_n + 1]
    const uint16_t* inc = nullptr;     // [nb * n_e]
    int32_t n_e = 0, n_col = 0;
    int32_t gather = 0;                // 1: the operator gathers per node (small_solver_gather)
};
// Shared memory the one-CTA solver needs (node ids are 16-bit: n_n <= 65536;
// at most 4096 elements).
size_t small_solver_smem(int64_t n_n, int64_t n_e, int nb);
// Whether the FP32 operator of the one-CTA solver gathers each node's element
// rows (no barrier per colour) instead of adding them in colour rounds: at
// most 1.5 nodes per thread, and the incidence tables fitting next to the
// rest.  Beyond 1.5 nodes per thread a thread's serial gathers cost more than
// the rounds' barriers (GB300, per iteration against the rounds: 1,089 nodes
// 15 % faster, 1,444 nodes 5 % faster, 1,764 nodes 2 % and 2,116 nodes 11 %
// slower; 125 and 729 tetrahedral nodes 28 and 14 % faster).
constexpr int kSmallGatherNodes = 1536;
constexpr size_t kSmallGatherSmem = size_t(224) * 1024;
bool small_solver_gather(int64_t n_n, int64_t n_e, int nb);
// Jacobi-PCG (textbook mixed form) of the whole mesh in one CTA: x (device,
// FP64, Dirichlet values set) in and out; pd in the caller's numbering.
cudaError_t launch_cg_small(const PlanDev& pd, int64_t n_n, const float* A32, const double* A64, const double* b,
                            const float* dinv, double* x, const SmallColouring& sc, const SmallOpts& o,
                            SmallInfo* info, cudaStream_t st, int* launches);

// Per-problem state reset: every problem starts with the true residual of x0.
cudaError_t launch_batch_init(const BatchDev& bd, cudaStream_t st, int* launches);
// CTAs per SM that fit for the persistent kernel of this batch (0: none).
int batch_max_ctas_per_sm(const BatchDev& bd, bool mixed, int* smem_bytes);
// The persistent solver: one cooperative launch of ctas_per_sm x SM CTAs that
// iterates until every problem is done or iter_budget loops have run.
cudaError_t launch_batch_solve(const BatchDev& bd, bool mixed, int ctas_per_sm, cudaStream_t st, int* launches);

// ---- learned preconditioner (k_mpnn.cu) -----------------------------------
constexpr int kMpnnHidden = 32;
constexpr int kMpnnLayers = 4;
constexpr int kMpnnLayerParams = 2 * kMpnnHidden * kMpnnHidden + kMpnnHidden;   // W_l [32][64], b_l [32]
// parameter vector: W_in [32][2], b_in [32], per layer W_l, b_l, w_out [32], b_out
constexpr int kMpnnW0 = 3 * kMpnnHidden;                                        // first layer's W_l
constexpr int kMpnnThWout = kMpnnW0 + kMpnnLayers * kMpnnLayerParams;           // w_out
constexpr int kMpnnParams = kMpnnThWout + kMpnnHidden + 1;                       // 8449
// small-weight array of the forward pass (BF16-rounded values as FP32):
// W_in, b_in, the layer biases, w_out, b_out
constexpr int kMpnnWin = 0, kMpnnBin = 64, kMpnnBl = 96, kMpnnWout = kMpnnBl + kMpnnLayers * kMpnnHidden,
              kMpnnBout = kMpnnWout + kMpnnHidden, kMpnnSmall = kMpnnBout + 1;

// Network state and work buffers on the device (BF16 data as uint16_t).
struct MpnnDev {
    int num_sms = 1;
    const int32_t* nbr_ptr = nullptr;   // mesh graph of the current handle (CSR, no self loops)
    const int32_t* nbr = nullptr;
    const float* inv_deg = nullptr;
    float* theta = nullptr;             // [kMpnnParams] FP32 master parameters
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    uint16_t* wl = nullptr;             // [layers][32 * 64] BF16 layer weights, tensor-core layout
    float* wT = nullptr;                // [layers][64][32] the same values transposed (backward)
    float* wsm = nullptr;               // [kMpnnSmall]
    uint16_t* h[kMpnnLayers + 1] = {};  // node features [n][32]; inference uses h[0], h[1] only
    uint16_t* save_u = nullptr;         // training: [layers][n][64] layer inputs
    float* save_v = nullptr;            // training: [layers][n][32] pre-activations
    float* save_x = nullptr;            // training: [n][2] input features
    float* gh = nullptr;                // backward work [n][32] x 3
    float* ghp = nullptr;
    float* ga = nullptr;
    double* part = nullptr;             // block partials
    uint32_t* ctr = nullptr;
    double* sc = nullptr;               // sc[0] = rms(r), sc[1] = rms(dinv r); sc[2..3] dot results
    int32_t* err = nullptr;
};

// z = B(r) on n nodes (save: keep what backward needs).
cudaError_t launch_mpnn_forward(const MpnnDev& m, int64_t n, const double* r, const double* dinv, double* z, bool save,
                                cudaStream_t st, int* launches);
// grad [kMpnnParams] = dL/dtheta for gz = dL/dz, after a forward with save.
cudaError_t launch_mpnn_backward(const MpnnDev& m, int64_t n, const double* gz, const double* dinv, double* grad,
                                 cudaStream_t st, int* launches);
// Refresh the BF16 / FP32 copies the forward pass reads from theta.
cudaError_t launch_mpnn_pack(const MpnnDev& m, cudaStream_t st, int* launches);
// One Adam step on theta (step >= 1), then pack.
cudaError_t launch_mpnn_adam(const MpnnDev& m, const double* grad, float lr, int step, cudaStream_t st, int* launches);
// w = e - z;  out[0] = a.b, out[1] = a.c (c nullable);  out = factor * a / num[0].
cudaError_t launch_sub(int64_t n, const double* e, const double* z, double* w, cudaStream_t st, int* launches);
cudaError_t launch_dot2(int64_t n, const double* a, const double* b, const double* c, double* part, uint32_t* ctr,
                        double* out, cudaStream_t st, int* launches);
cudaError_t launch_scale(int64_t n, const double* a, const double* num, double factor, double* out, cudaStream_t st,
                         int* launches);
// Flexible CG: dots z.q_prev, z.r, p_prev.r -> sc->beta, sc->rho = p.r; p = z + beta p; Jacobi z = dinv r.
cudaError_t launch_fcg_dots(int64_t n, const double* z, const double* r, const double* p, const double* q, int first,
                            double* part, Scalars* sc, cudaStream_t st, int* launches);
cudaError_t launch_fcg_dir(int64_t n, const double* z, double* p, int first, const Scalars* sc, cudaStream_t st,
                           int* launches);
cudaError_t launch_jacobi(int64_t n, const double* r, const double* dinv, double* z, const int32_t* stop, cudaStream_t st,
                          int* launches);

// ---- comparison scatters (k_alt.cu) ---------------------------------------
cudaError_t launch_build_gconn(const PlanDev& pd, int32_t* gconn, cudaStream_t st, int* launches);
cudaError_t launch_permute_slots(int nb, int64_t n_slots, int64_t n, const int32_t* order,
                                 const double* A, const int32_t* gconn, double* A_out,
                                 int32_t* gconn_out, cudaStream_t st, int* launches);
cudaError_t launch_residual_colour(int nb, int n_col, const int64_t* col_ptr_host, int64_t n_el,
                                   const double* Ac, const int32_t* gc, const double* x,
                                   const double* b, const uint8_t* dmask, int64_t n_n, double* r,
                                   cudaStream_t st, int* launches);
cudaError_t launch_residual_atomic(const PlanDev& pd, const double* A, const int32_t* gconn,
                                   const double* x, const double* b, const uint8_t* dmask,
                                   int64_t n_n, double* r, cudaStream_t st, int* launches);
cudaError_t launch_residual_node(const PlanDev& pd, const double* A, const int32_t* gconn,
                                 const int32_t* node_ptr, const int32_t* node_ent, const double* x,
                                 const double* b, const uint8_t* dmask, int64_t n_n, double* Y,
                                 double* r, cudaStream_t st, int* launches);

}  // namespace ebe
