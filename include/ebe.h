/*
 * ebe.h -- C ABI of the GB300 element-by-element (EbE) finite-element library.
 *
 * The library evaluates the element-based residual of Marcinkowski & Valdman,
 * "MATLAB Implementation of Element-based Solvers" (Sec. 2, Eq. residual and
 * Algorithm 1),
 *
 *     r = b - A x = sum_e C_e^T (b_e - A_e C_e x),   A_e = K_e + nu M_e,
 *
 * directly from per-element matrices, never assembling the sparse A, and
 * drives Jacobi-preconditioned conjugate gradients with it.  The calls follow
 * the paper's problem statement (Sec. 1): a mesh (nodal coordinates and the
 * element-to-node connectivity that replaces the Boolean matrices C_e), a
 * parameter nu >= 0, nodal values of f, and Dirichlet / Neumann node sets.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns an ebe_status; nothing is thrown or aborted across the
 *   ABI.  On failure ebe_last_error(h) holds a one-line message.
 * - Host pointers ("host") are read during the call only; the caller keeps
 *   ownership and may free them afterwards.  Device pointers ("device") are
 *   caller-owned CUDA global-memory buffers on the handle's device (for
 *   example torch.Tensor.data_ptr()); they must stay valid until the work
 *   enqueued by the call has finished on the handle's stream.
 * - All device work of a handle is ordered on the CUDA stream given to
 *   ebe_create (NULL means the legacy default stream).  Calls that return
 *   host results (ebe_solve, ebe_get_*) synchronise that stream.
 * - Node and element numbering is the caller's, 0-based, everywhere.  The
 *   library reorders elements internally for locality; this never shows.
 * - Vectors are dense arrays of length n_n indexed by node id.  The Dirichlet
 *   rows of a residual or an operator application are set to zero, as in the
 *   paper's listings (r(nd) = 0 after every residual, Sec. 2.1).
 * - A handle is not thread-safe: one host thread at a time per handle.
 *
 * Call sequence: ebe_create (mesh) -> ebe_set_problem (nu, f, boundary sets)
 * -> ebe_assemble (element matrices, b, Jacobi diagonal) -> any number of
 * ebe_residual / ebe_apply / ebe_solve / ebe_richardson / ebe_chebyshev* ->
 * ebe_destroy.  ebe_set_problem may be called again (then ebe_assemble
 * again); batches use ebe_create_batch / ebe_set_problem_batch /
 * ebe_solve_batch in the same order.
 */
#ifndef EBE_H
#define EBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EBE_OK = 0,
    EBE_INVALID_ARG = 1,        /* NULL pointer, bad size, dim/n_b mismatch, unused node, ... */
    EBE_INDEX_RANGE = 2,        /* a node id outside [0, n_n) or repeated within an element   */
    EBE_DEGENERATE_ELEMENT = 3, /* an element with zero area / volume                          */
    EBE_SINGULAR = 4,           /* nu == 0 and no Dirichlet node (Sec. 1 requires a positive
                                   Dirichlet measure when nu = 0)                             */
    EBE_CUDA_ERROR = 5,         /* a CUDA runtime call failed                                  */
    EBE_OOM = 6,                /* device allocation failed                                    */
    EBE_MAXIT = 7,              /* solver stopped at maxit before reaching rtol                */
    EBE_BREAKDOWN = 8,          /* p.Ap <= 0 or a non-finite value in the solver               */
    EBE_STALL = 9,              /* the FP64 true residual stopped decreasing                   */
    EBE_NOT_READY = 10          /* call order: ebe_set_problem / ebe_assemble not done yet     */
} ebe_status;

/* Arithmetic types for ebe_residual / ebe_apply. */
enum {
    EBE_F64 = 0,      /* FP64 vectors, FP64 element matrices and arithmetic             */
    EBE_F32 = 1,      /* FP32 vectors and element matrices (EBE_STORE_MIXED)            */
    EBE_F64_DW = 2    /* FP64 vectors; the FP64 element matrices split into pairs of
                         FP32 (hi + lo, made on first use after each ebe_assemble: 8
                         bytes per stored entry, like the FP64 copy) and the products
                         and sums in double-word FP32 arithmetic (exact FMA products,
                         TwoSum additions, about 48 significant bits); r = b - A x is
                         formed in FP64 per node.  It agrees with EBE_F64 to about
                         2^-48 |A| |x| per node and runs on the FP32 pipe: GB300's
                         FP64 pipe bounds the EBE_F64 residual                     */
};

/* Storage of the element matrices made by ebe_assemble. */
enum {
    EBE_STORE_FP64 = 0,   /* A_e in FP64 only                                               */
    EBE_STORE_MIXED = 1   /* A_e in FP64 and an FP32 copy in difference form: the
                             off-diagonal entries a_ij (i != j) rounded to nearest, and on
                             the diagonal slots the row sums s_i = sum_j a_ij rounded to
                             nearest.  The FP32 operator evaluates
                             y_i = s_i x_i + sum_{j != i} a_ij (x_j - x_i), which keeps FP32
                             relative accuracy for smooth x (K_e rows sum to zero).     */
};

/* Solver precision for ebe_solve. */
enum {
    EBE_PREC_FP64 = 0,    /* plain FP64 Jacobi-PCG (textbook: four launches per iteration) */
    EBE_PREC_MIXED = 1,   /* the operator pass runs on FP32 A_e (difference form) with the
                             search direction p, q = A p, the recurrence residual r and
                             z = dinv r in FP32; the solution x stays FP64; dot products
                             add in FP32 within a warp and in compensated FP32 across
                             warps and blocks, the last block in FP64; r is replaced by
                             the true residual whenever the recurrence residual has
                             dropped by the factor `delta` since the last replacement
                             (the double-word residual of EBE_F64_DW while the threshold
                             is at least 1e-6 |r0|, the FP64 one below; convergence is
                             confirmed by the FP64 residual; needs EBE_STORE_MIXED).
                             One iteration is two launches with one grid-wide reduction:
                             the x and r updates and the new direction are formed where
                             the operator pass gathers its operand, and the next r.z
                             comes from r'.(dinv r') = r.z - 2 alpha q.z + alpha^2
                             q.(dinv q) (the same iterates as the textbook form in exact
                             arithmetic).  A mesh of at most 4 patches (4096 elements)
                             with use_graph = 1 is solved instead by one CTA that runs
                             every iteration of the textbook mixed form (with FP64
                             replacement residuals) with block barriers in place of
                             launches: such a mesh leaves the grid-wide iteration bound by
                             launch latency; use_graph = 0 keeps the grid-wide one    */
    EBE_PREC_MIXED_TEXTBOOK = 2   /* EBE_PREC_MIXED arithmetic in the textbook four-launch
                             iteration (operator, update, direction; two reductions), for
                             comparison; ebe_solve only                               */
};

/* Scatter strategies of the residual (ebe_residual_variant). */
enum {
    EBE_SCATTER_PATCH = 0,  /* default: patch-local colour-ordered accumulation in shared
                               memory + fixed-order halo sum (deterministic)                */
    EBE_SCATTER_COLOUR = 1, /* global element colouring, one pass per colour, plain
                               read-modify-write of r (deterministic)                       */
    EBE_SCATTER_NODE = 2,   /* two-phase: per-element A_e x_e to a buffer, then a node-
                               centric gather over the inverse connectivity (deterministic) */
    EBE_SCATTER_ATOMIC = 3  /* FP64 atomic adds (NOT deterministic; for measurement only)   */
};

typedef struct ebe_handle ebe_handle;

/* Mesh description (Sec. 1).  P1 simplices: dim = 2 -> triangles, n_b = 3;
 * dim = 3 -> tetrahedra, n_b = 4. */
typedef struct {
    int32_t dim;             /* 2 or 3                                                   */
    int32_t n_b;             /* dim + 1                                                  */
    int64_t n_n;             /* number of nodes, 1 <= n_n < 2^31                         */
    int64_t n_e;             /* number of elements, 1 <= n_e < 2^31 / n_b                */
    const double* coords;    /* host, [n_n][dim] row-major                               */
    const int32_t* elems;    /* host, [n_e][n_b] row-major node ids (the index arrays
                                ind_e / indt of Sec. 2 in one array)                     */
} ebe_mesh;

/* Options of ebe_create; pass NULL for the defaults. */
typedef struct {
    int32_t device;          /* CUDA device ordinal (default 0)                          */
    int32_t patch_elems;     /* elements per patch, 0 = default (1024); must be 1024 in
                                this version                                             */
} ebe_create_opts;

typedef struct {
    double rtol;             /* target FP64 true relative residual
                                |mask(b - A x)|_2 / |mask(b - A x0)|_2, default 1e-8     */
    int64_t maxit;           /* CG iteration cap, default 200000                         */
    int32_t precision;       /* EBE_PREC_FP64 (default) or EBE_PREC_MIXED                */
    int32_t chunk;           /* CG iterations per CUDA-graph launch, default 32          */
    double delta;            /* reliable-update factor for EBE_PREC_MIXED, default 0.1   */
    int32_t stall_updates;   /* true-residual checks without progress before EBE_STALL,
                                default 8                                                */
    int32_t use_graph;       /* 1 (default): iterations run as captured CUDA graphs      */
    int32_t race_iters;      /* ebe_solve_learned only: iterations of each leg of the race
                                between Jacobi and the network; 0 = no race (the network
                                from the start, with the fallback rules only); default -1
                                = 16                                                     */
} ebe_solve_opts;

typedef struct {
    int32_t status;          /* ebe_status of the solve                                  */
    int64_t iterations;      /* CG iterations                                            */
    int64_t true_residuals;  /* FP64 true-residual evaluations (incl. the initial one)    */
    double rel_residual;     /* final FP64 true relative residual                        */
    double r0_norm;          /* |mask(b - A x0)|_2                                        */
    double solve_ms;         /* wall time of the solve on the host clock                 */
} ebe_solve_info;

typedef struct {
    int64_t kernel_launches;   /* kernels launched by this handle so far (graph nodes count
                                  once per graph launch)                                 */
    int64_t n_patches;         /* patches of the element partition                         */
    int64_t patch_elems;       /* elements per patch                                       */
    int64_t n_shared_nodes;    /* nodes touched by more than one patch                    */
    int64_t n_halo;            /* halo partial sums per residual (sum over patches of
                                  their shared nodes)                                    */
    int64_t max_colours;       /* largest colour count of a patch                         */
    int64_t n_global_colours;  /* colours of the global colouring (0 until first used)    */
    int64_t device_bytes;      /* device memory held by the handle                        */
    int64_t device_error;      /* nonzero if a bounded device-side wait gave up (the
                                  affected results are invalid); reading it synchronises
                                  the handle's stream                                    */
} ebe_stats;

/* ---------------------------------------------------------------- lifetime */

/* Validate the mesh on the host, copy it to the device and build the element
 * partition (patches, local connectivity, halo lists).  Sec. 1 / Sec. 2: the
 * connectivity plays the role of C_e and R_e, which are never stored.
 * The partition is built on up to 16 host threads (32 problems at a time for
 * a batch); the environment variable EBE_HOST_THREADS (an integer >= 1) caps
 * them.  The partition does not depend on the thread count.
 * Errors: EBE_INVALID_ARG, EBE_INDEX_RANGE, EBE_CUDA_ERROR, EBE_OOM.
 * On error *h is NULL. */
ebe_status ebe_create(ebe_handle** h, const ebe_mesh* mesh, const ebe_create_opts* opts,
                      void* cuda_stream);

/* Free every device and host resource of the handle (NULL is ignored). */
void ebe_destroy(ebe_handle* h);

/* Message of the last failed call on h (never NULL; "" if none).  With h NULL,
 * the message of the last failed ebe_create in this thread. */
const char* ebe_last_error(const ebe_handle* h);

/* Static name of a status code. */
const char* ebe_status_string(int status);

/* Defaults for ebe_solve_opts. */
void ebe_solve_opts_default(ebe_solve_opts* opts);

/* ---------------------------------------------------------------- problem data */

/* Set nu, f and the boundary node sets of the problem -Lap u + nu u = f
 * (Sec. 1).  f_nodal: host [n_n], nodal values of f (b_j = int f Phi_j is
 * evaluated as b = M f_I, f interpolated at the nodes).  dirichlet: host
 * [n_d] node ids with prescribed values g (host [n_d], NULL = 0).  neumann:
 * host [n_neu] node ids with homogeneous Neumann data; they add nothing to
 * the system and are only validated.  A node may not be in both sets.
 * Errors: EBE_INVALID_ARG (nu < 0 or not finite, bad sizes, overlap),
 * EBE_INDEX_RANGE, EBE_SINGULAR (nu == 0 and n_d == 0). */
ebe_status ebe_set_problem(ebe_handle* h, double nu, const double* f_nodal,
                           const int32_t* dirichlet, int64_t n_d, const double* g,
                           const int32_t* neumann, int64_t n_neu);

/* Generate on the device, for every element, the P1 matrices of
 * Eq. matrices_K_M, A_e = K_e + nu M_e (Sec. 2), the assembled load vector
 * b = sum_e C_e^T M_e f_e and the inverse Jacobi diagonal
 * dinv = 1 / sum_e C_e^T diag(A_e) (0 on Dirichlet nodes).  store:
 * EBE_STORE_FP64 or EBE_STORE_MIXED.  A_e is symmetric, so the handle keeps
 * its n_b(n_b+1)/2 distinct entries per element (6 for triangles, 10 for
 * tetrahedra; FP64, plus FP32 for MIXED).  Enqueued on the handle's stream;
 * the degenerate-element check synchronises it.
 * Errors: EBE_NOT_READY, EBE_DEGENERATE_ELEMENT, EBE_CUDA_ERROR, EBE_OOM. */
ebe_status ebe_assemble(ebe_handle* h, int32_t store);

/* Write K_e and M_e of every element (Eq. matrices_K_M) to device buffers in
 * the paper's n_b x n_b x n_e layout (Fig. 2; entry (i,j) of element e at
 * [e*n_b*n_b + j*n_b + i], element order = caller's).  Either may be NULL.
 * Needs ebe_create only.  Errors: EBE_INVALID_ARG, EBE_CUDA_ERROR. */
ebe_status ebe_element_matrices(ebe_handle* h, double* K_dev, double* M_dev);

/* Copy the element matrices A_e held by the handle to a device buffer in the
 * same layout (full n_b x n_b, both triangles written).  dtype EBE_F64 (double*) or EBE_F32 (float*, MIXED storage; the
 * stored difference form: diagonal entries hold the row sums s_i).
 * Errors: EBE_NOT_READY, EBE_INVALID_ARG, EBE_CUDA_ERROR. */
ebe_status ebe_get_local_matrices(ebe_handle* h, void* A_dev, int32_t dtype);

/* Copy b (device [n_n] double; Dirichlet rows not masked). */
ebe_status ebe_get_rhs(ebe_handle* h, double* b_dev);

/* Write the Jacobi diagonal d = sum_e C_e^T diag(A_e) (device [n_n] double,
 * Dirichlet rows not masked). */
ebe_status ebe_jacobi_diag(ebe_handle* h, double* d_dev);

/* ---------------------------------------------------------------- operator */

/* r = mask(b - A x) by the element-based residual (Eq. residual, Algorithm 1;
 * mask = zero Dirichlet rows).  x_dev, r_dev: device [n_n] of double
 * (dtype EBE_F64, FP64 A_e; dtype EBE_F64_DW, the double-word form) or float
 * (dtype EBE_F32, FP32 A_e; needs EBE_STORE_MIXED).  x and r must not
 * overlap.  Deterministic.
 * Errors: EBE_NOT_READY, EBE_INVALID_ARG, EBE_CUDA_ERROR. */
ebe_status ebe_residual(ebe_handle* h, const void* x_dev, void* r_dev, int32_t dtype);

/* y = mask(A x) = mask(sum_e C_e^T A_e C_e x).  Same arguments as ebe_residual. */
ebe_status ebe_apply(ebe_handle* h, const void* x_dev, void* y_dev, int32_t dtype);

/* Measure the operator: run `reps` passes of ebe_residual (apply = 0) or
 * ebe_apply (apply = 1) on the handle's stream, after one untimed pass, with
 * CUDA events recorded on that stream around each of the pass's two kernels
 * (the patch kernel and the halo fix-up kernel).  ms: host [2], receives the
 * mean milliseconds per launch of the patch kernel and of the fix-up kernel.
 * Synchronises the stream.  Arguments and errors as ebe_residual. */
ebe_status ebe_time_operator(ebe_handle* h, const void* x_dev, void* y_dev, int32_t dtype, int32_t apply,
                             int32_t reps, double* ms);

/* Measure one iteration of the EBE_PREC_MIXED solver (the single-sync pass:
 * patch kernel and fix-up kernel): from x0 = 0 on the handle's problem, one
 * untimed first pass and then `reps` CG iterations without a stopping test,
 * with CUDA events recorded on the handle's stream around each of the two
 * kernels.  ms: host [2], receives the mean milliseconds per launch of the
 * patch kernel and of the fix-up kernel.  Uses the solver's own work vectors
 * (no caller data).  Needs EBE_STORE_MIXED.  Synchronises the stream.
 * Errors: EBE_NOT_READY, EBE_INVALID_ARG, EBE_BREAKDOWN, EBE_CUDA_ERROR. */
ebe_status ebe_time_cg_pass(ebe_handle* h, int32_t reps, double* ms);

/* FP64 residual r = mask(b - A x) with a chosen scatter strategy
 * (EBE_SCATTER_*), for comparing them.  Builds the strategy's data on first
 * use.  Errors as ebe_residual. */
ebe_status ebe_residual_variant(ebe_handle* h, const double* x_dev, double* r_dev, int32_t scatter);

/* ---------------------------------------------------------------- solvers */

/* Jacobi-PCG on A x = b with x(nd) = g, stopping when the FP64 true relative
 * residual |mask(b - A x)| / |mask(b - A x0)| <= rtol (x0 = the given x with
 * x(nd) = g).  The true residual is evaluated (FP64 element matrices) each
 * time the recurrence residual reaches rtol |r0| (and, in mixed precision, at
 * every replacement); in mixed precision a failed check at that final
 * threshold tightens it by the factor 0.7.  x_dev: device [n_n] double, in: x0, out:
 * solution.  opts NULL = defaults.  info may be NULL.  Synchronises the
 * stream once at the end.  Returns EBE_OK, EBE_MAXIT, EBE_BREAKDOWN,
 * EBE_STALL or an error. */
ebe_status ebe_solve(ebe_handle* h, double* x_dev, const ebe_solve_opts* opts, ebe_solve_info* info);

/* ebe_solve with a HOST x (host [n_n] double, in: x0, out: solution); the
 * host<->device copies are part of the call. */
ebe_status ebe_solve_host(ebe_handle* h, double* x_host, const ebe_solve_opts* opts,
                          ebe_solve_info* info);

/* The paper's stationary iterations (Sec. 2), each step starting from the
 * element-based residual r = mask(b - A x) (FP64).  x_dev: device [n_n]
 * double, in: x0, out: x after `iters` steps; x(nd) = g is set first.  No
 * stopping test: exactly `iters` steps, as in the paper's experiment.
 * Synchronises the stream.  Errors: EBE_NOT_READY, EBE_INVALID_ARG,
 * EBE_CUDA_ERROR. */
/* Eq. richardson: x += omega r (the optimum is 2 / (lambda_1 + lambda_2)). */
ebe_status ebe_richardson(ebe_handle* h, double* x_dev, int64_t iters, double omega);
/* Eq. Czebyshev2lev: step k uses x += r / alphas[k mod N]; alphas host [N],
 * the roots of the shifted and scaled Chebyshev polynomial in the order the
 * caller chooses. */
ebe_status ebe_chebyshev2(ebe_handle* h, double* x_dev, int64_t iters, const double* alphas, int64_t N);
/* Eq. Czebyshev2lev in the paper's form: the library builds the N roots of
 * the shifted and scaled Chebyshev polynomial P_N for the spectrum bounds
 * 0 < lam1 < lam2 (Sec. 2.2), alpha_k = (lam1 + lam2)/2 + (lam2 - lam1)/2
 * cos(pi (k + 1/2) / N), k = 0..N-1, and cycles through them in that order
 * (the order of the paper's listing; with N = 32 on the Sec. 3 problem the
 * partial products of a cycle amplify rounding errors, the instability the
 * paper reports).  Errors: EBE_INVALID_ARG (bounds, 1 <= N <= 2^20), and as
 * ebe_chebyshev2. */
ebe_status ebe_chebyshev2_bounds(ebe_handle* h, double* x_dev, int64_t iters, double lam1, double lam2, int64_t N);
/* Eq. Czebyshev3lev (the three-term recurrence with the scaling factors of
 * Eq. recrCk) for spectrum bounds 0 < lam1 < lam2, evaluated in the
 * equivalent direction form p = r + beta p, x += alpha p. */
ebe_status ebe_chebyshev3(ebe_handle* h, double* x_dev, int64_t iters, double lam1, double lam2);

/* Counters of the handle (see ebe_stats). */
ebe_status ebe_get_stats(const ebe_handle* h, ebe_stats* stats);

/* ---------------------------------------------------------------- batches of problems */

/* A batch handle holds n_problems independent meshes of the same dim as one
 * disjoint union: node i of problem k is node node_off[k] + i of the union and
 * element e of problem k is element elem_off[k] + e (ebe_batch_layout), in
 * the order given.  Each mesh is partitioned exactly as ebe_create would
 * partition it, so no patch mixes two problems; ebe_create is the batch of
 * one.  Every call above works on a batch handle and acts on the union (the
 * residual of the union is every problem's residual at once; ebe_solve solves
 * the union as one system with global dot products).  ebe_solve_batch solves
 * the problems independently.  meshes: host [n_problems], each validated as
 * by ebe_create.  1 <= n_problems <= 4096, total nodes < 2^31.
 * Errors as ebe_create; the message names the failing problem. */
ebe_status ebe_create_batch(ebe_handle** h, const ebe_mesh* meshes, int32_t n_problems,
                            const ebe_create_opts* opts, void* cuda_stream);

/* Problem count and offsets of the union numbering.  node_off, elem_off: host
 * [n_problems + 1] or NULL. */
ebe_status ebe_batch_layout(const ebe_handle* h, int32_t* n_problems, int64_t* node_off, int64_t* elem_off);

/* ebe_set_problem with one nu per problem (Sec. 1 for each problem):
 * nu host [n_problems]; f_nodal, dirichlet, g, neumann as for
 * ebe_set_problem, in the union numbering.  A problem with nu = 0 needs at
 * least one Dirichlet node.  Errors as ebe_set_problem. */
ebe_status ebe_set_problem_batch(ebe_handle* h, const double* nu, const double* f_nodal,
                                 const int32_t* dirichlet, int64_t n_d, const double* g,
                                 const int32_t* neumann, int64_t n_neu);

/* Launch shape of the batched solver. */
typedef struct {
    int32_t ctas_per_sm;     /* CTAs per SM of the persistent kernel; 0 = as many as fit */
    int32_t tile_nodes;      /* nodes per work item of the vector phases: 1024, 2048 or 4096;
                                0 = 2048                                                 */
    int64_t barrier_ns;      /* bound of one grid-barrier wait in nanoseconds, 0 = 2 s.  A
                                wait that runs out ends the launch: ebe_solve_batch returns
                                EBE_CUDA_ERROR, the solution is invalid, and the handle
                                stays usable for the next call                           */
} ebe_batch_config;

typedef struct {
    int64_t loops;           /* iterations of the persistent loop (each is a CG step or a
                                true residual for every problem still running)           */
    int32_t launches;        /* persistent-kernel launches                               */
    int32_t n_converged;     /* problems that reached rtol                               */
    double solve_ms;         /* wall time of the call on the host clock                  */
    ebe_batch_config config; /* launch shape used                                        */
    double phase_ms[4];      /* device time of the loop's four phases summed over the
                                loops: patch pass, halo fix-up, update, direction (each
                                from one grid barrier to the next, seen by CTA 0)        */
} ebe_batch_info;

/* Jacobi-PCG on every problem of the batch at once, each stopping on its own
 * FP64 true relative residual |mask(b_k - A_k x_k)| / |mask(b_k - A_k x0_k)|
 * <= rtol, with the per-problem rules of ebe_solve (precision, delta,
 * maxit, stall_updates; chunk is not used).  The batched iteration is the
 * textbook four-phase form; in mixed precision a replacement residual is the
 * double-word one while the problem's threshold is at least 1e-6 |r0|, the
 * FP64 one below (so the last checks before rtol are FP64).  All iterations of all problems
 * run in one persistent cooperative kernel with grid-wide barriers (each
 * wait bounded in time); problems that have finished drop out of the work.
 * With use_graph = 1 the solve (x0 Dirichlet values, state reset, the
 * persistent kernel) is replayed from a CUDA graph captured once per handle,
 * launch shape and options.  x_dev: device [n_n] double (union numbering),
 * in: x0, out: solutions.  info: host [n_problems] or NULL; summary: NULL
 * allowed.  Launch shape: the handle's (ebe_set_batch_config,
 * ebe_batch_tune), else the defaults.  Synchronises the stream.
 * Returns EBE_OK when every problem reached rtol, otherwise the status of the
 * first problem that did not (every problem's status is in info). */
ebe_status ebe_solve_batch(ebe_handle* h, double* x_dev, const ebe_solve_opts* opts, ebe_solve_info* info,
                           ebe_batch_info* summary);

/* ebe_solve_batch with a HOST x; the host<->device copies are part of the call. */
ebe_status ebe_solve_batch_host(ebe_handle* h, double* x_host, const ebe_solve_opts* opts,
                                ebe_solve_info* info, ebe_batch_info* summary);

/* Set the launch shape of ebe_solve_batch for both precisions (NULL: back to
 * the defaults).  Errors: EBE_INVALID_ARG (tile_nodes not 0/1024/2048/4096,
 * ctas_per_sm outside [0, 8], barrier_ns < 0); a ctas_per_sm that does not fit on an SM for
 * the precision of a later ebe_solve_batch makes that call fail with
 * EBE_INVALID_ARG. */
ebe_status ebe_set_batch_config(ebe_handle* h, const ebe_batch_config* cfg);

/* Autotuner of the batched solver: for every launch shape (ctas_per_sm from
 * 1 to the most that fit, tile_nodes 1024, 2048, 4096) run the solver on the
 * handle's own problems from x0 = 0 -- `loops` persistent-loop iterations, or
 * complete solves with loops = 0 -- timed with CUDA events, and keep the
 * fastest shape as the handle's launch shape.  Caller data is not touched.
 * precision: as in ebe_solve_opts.  best: the chosen shape (NULL allowed).
 * shapes, ms: host [capacity] or NULL; receive each candidate and its time
 * (ms per loop iteration with loops > 0, ms per solve with loops = 0);
 * n_written: candidates written.  The chosen shape is kept for ebe_solve_batch
 * calls of this precision only.  Errors: EBE_NOT_READY, EBE_INVALID_ARG,
 * EBE_CUDA_ERROR. */
ebe_status ebe_batch_tune(ebe_handle* h, int32_t precision, int32_t loops, ebe_batch_config* best,
                          ebe_batch_config* shapes, double* ms, int32_t capacity, int32_t* n_written);

/* ---------------------------------------------------------------- learned preconditioner */

/* A small message-passing network in the preconditioner slot of the solver
 * loop (the paper's listings apply z = r where a preconditioner would act,
 * Sec. 2; the network is this library's own addition).  For a residual r on
 * the mesh of a handle, with dinv the inverse Jacobi diagonal (0 on
 * Dirichlet nodes) and rms taken over the free nodes:
 *   x_i = [r_i / rms(r), (dinv r)_i / rms(dinv r)]                (2 features)
 *   h_i = W_in x_i + b_in                                         (32)
 *   4 layers: a_i = mean_{j in N(i)} h_j - h_i, h_i += relu(W_l [h_i; a_i] + b_l)
 *   z_i = (dinv r)_i + rms(dinv r) (w_out . h_i + b_out),  z_i = 0 on Dirichlet nodes
 * N(i): the nodes sharing an element with node i.  z is homogeneous of degree
 * one in r, and a zero decoder gives the Jacobi step.  Weights and hidden
 * features are BF16 (round to nearest even), sums FP32; the per-node layers
 * run on the tensor cores (tcgen05).  Parameter vector (ebe_mpnn_n_params()
 * doubles): W_in [32][2], b_in [32], then per layer W_l [32][64], b_l [32],
 * then w_out [32], b_out.  A network object holds FP32 master parameters,
 * Adam moments and work buffers on one device and can be used with any
 * handle on that device (train on one mesh, use on another). */
typedef struct ebe_mpnn ebe_mpnn;

int64_t ebe_mpnn_n_params(void);
/* theta: host [n_params] or NULL for the library's seeded initial weights
 * (zero decoder).  Errors: EBE_INVALID_ARG (no such device, non-finite
 * theta), EBE_OOM, EBE_CUDA_ERROR (message: ebe_mpnn_last_error(NULL)). */
ebe_status ebe_mpnn_create(ebe_mpnn** net, int32_t device, const double* theta);
void ebe_mpnn_destroy(ebe_mpnn* net);
const char* ebe_mpnn_last_error(const ebe_mpnn* net);
/* Replace the parameters (host [n_params], NULL = initial weights) and reset
 * the optimiser; get: host [n_params] (FP32 masters as doubles). */
ebe_status ebe_mpnn_set_params(ebe_mpnn* net, const double* theta);
ebe_status ebe_mpnn_get_params(const ebe_mpnn* net, double* theta);

/* z = B(r) on the mesh of h (assembled).  r_dev, z_dev: device [n_n] double.
 * Builds the handle's mesh graph on first use.  Synchronises the stream.
 * Errors: EBE_NOT_READY, EBE_INVALID_ARG, EBE_CUDA_ERROR. */
ebe_status ebe_mpnn_apply(ebe_mpnn* net, ebe_handle* h, const double* r_dev, double* z_dev);

/* Gradient of a loss L(z) with respect to the parameters for
 * gz_dev = dL/dz (device [n_n] double): forward pass at r_dev (z written to
 * z_dev if not NULL), then the backward pass.  grad: host [n_params].  The
 * BF16 roundings of the forward pass count as the identity. */
ebe_status ebe_mpnn_grad(ebe_mpnn* net, ebe_handle* h, const double* r_dev, const double* gz_dev, double* z_dev,
                         double* grad);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step size lr) on the
 * energy-norm loss L = (e - z)' A (e - z) / e' A e of one sample: a residual
 * r_dev and the error e_dev = x* - x that it belongs to (device [n_n]
 * double, zero on Dirichlet nodes), A the FP64 operator of h.  loss: host,
 * the loss before the step (NULL allowed).  Synchronises the stream. */
ebe_status ebe_mpnn_train_step(ebe_mpnn* net, ebe_handle* h, const double* r_dev, const double* e_dev, double lr,
                               double* loss);

/* Flexible CG (one stored direction: p = z - (z.q_prev / p_prev.q_prev) p_prev,
 * alpha = p.r / p.q) with z = B(r) from net, or the Jacobi step with net NULL,
 * FP64 vectors and element matrices, stopping on the FP64 true relative
 * residual as ebe_solve.  With a network the solve starts with a race: from
 * x0, race_iters iterations of Jacobi-FCG, then, again from x0, race_iters
 * iterations with the network, each timed with CUDA events; the network
 * continues only if Jacobi's leg reduced the residual norm and the network's
 * leg reduced it at least 1.5 times faster per unit time (early rates favour
 * a smoother), and then only while every
 * window of 2 chunks keeps at least Jacobi's race rate, the residual norm
 * halves within 16 chunks, no breakdown occurs and the true residual does not
 * stall (stall_updates checks).  Otherwise the library's Jacobi-PCG (ebe_solve
 * with EBE_PREC_MIXED after ebe_assemble(EBE_STORE_MIXED), else with
 * EBE_PREC_FP64) finishes the solve from the current iterate (from
 * the Jacobi leg's iterate when the race is lost), to the same target
 * rtol |r0|, so a network that does not pay off costs its race leg and a
 * restart of CG; *fell_back (may be NULL) is 1 when that happened.  opts:
 * rtol, maxit, chunk (iterations between host checks), stall_updates,
 * race_iters (default 16).  iterations counts every iteration of the call.
 * Returns EBE_OK, EBE_MAXIT, EBE_BREAKDOWN, EBE_STALL or an error. */
ebe_status ebe_solve_learned(ebe_handle* h, ebe_mpnn* net, double* x_dev, const ebe_solve_opts* opts,
                             ebe_solve_info* info, int32_t* fell_back);

/* ---------------------------------------------------------------- allocation-free residual */

/* ebe_residual (FP64) for callers that cannot call cudaMalloc when they need
 * a residual: a process whose device memory is handed out by another
 * allocator (a framework's caching allocator, or a fixed pool that owns the
 * whole device), or a real-time loop that must not take the allocator's
 * locks or risk the implicit device synchronisation of cudaMalloc.
 * ebe_residual allocates its scratch on first use; this call takes it from a
 * fixed device array compiled into the library (32 MiB: 4,194,304 doubles,
 * held on every device that loads the library until the process exits) and
 * calls no allocator.  The paper has no counterpart: this is an interface
 * feature of the library.
 * x_dev, r_dev: device [n_n] double (caller-owned), as for ebe_residual.
 * The first call on a device looks up the array's device address and keeps it
 * for the life of the process; make that first call before any stream
 * capture.  A device reset (cudaDeviceReset) invalidates every handle on the
 * device and that address: do not call the library on a device after
 * resetting it.  All calls share the array, so calls whose kernels overlap on
 * the GPU (several streams or handles at once) race.
 * Errors: EBE_NOT_READY, EBE_INVALID_ARG (also when the mesh needs more than
 * 4,194,304 halo slots, see ebe_stats.n_halo), EBE_CUDA_ERROR. */
ebe_status ebe_residual_noalloc(ebe_handle* h, const double* x_dev, double* r_dev);

/* ---------------------------------------------------------------- inspection */

typedef struct {
    int64_t n_patches;       /* patches                                                  */
    int64_t n_slots;         /* n_patches * patch_elems (slots past an element are padding) */
    int64_t n_pnode;         /* entries of the local-node tables of all patches          */
    int64_t n_colptr;        /* entries of the colour-offset tables                      */
    int64_t n_shared;        /* nodes touched by more than one patch                     */
    int64_t n_halo;          /* halo slots                                               */
    int32_t max_nodes;       /* largest local-node count of a patch                      */
    int32_t max_colours;     /* largest colour count of a patch                          */
    int32_t patch_elems;     /* elements per patch                                       */
} ebe_partition_sizes;

/* Host only, no device needed: validate the mesh and build the element
 * partition that ebe_create uses, then copy it out (the data that replaces
 * the index arrays ind_e / indt of Sec. 2 on the device).  With all arrays
 * NULL only sizes is filled; otherwise each non-NULL array must hold:
 *   slot_elem  [n_slots]          caller's element id per slot, -1 = padding
 *   lconn      [n_b][n_slots]     local node id of vertex i of each slot
 *   patch_meta [n_patches][8]     node_off, n_nodes, n_owned, halo_off, n_el,
 *                                 col_off, n_col, 0
 *   pnode      [n_pnode]          global node ids of each patch's local nodes
 *                                 (owned nodes first, then shared nodes)
 *   col_ptr    [n_colptr]         per patch n_col + 1 slot offsets (colour classes)
 *   sh_node    [n_shared]         shared nodes
 *   sh_ptr     [n_shared + 1]     CSR offsets into sh_slot
 *   sh_slot    [n_halo]           halo slots of each shared node, in patch order
 * Errors as ebe_create's validation (message: ebe_last_error(NULL)). */
ebe_status ebe_partition_export(const ebe_mesh* mesh, ebe_partition_sizes* sizes, int32_t* slot_elem,
                                uint16_t* lconn, int32_t* patch_meta, int32_t* pnode, int32_t* col_ptr,
                                int32_t* sh_node, int32_t* sh_ptr, int32_t* sh_slot);

/* ebe_partition_export for the union of a batch (the partition that
 * ebe_create_batch uses): every array in the union numbering, plus
 * patch_off host [n_problems + 1] (problem k owns patches
 * [patch_off[k], patch_off[k+1])) or NULL. */
ebe_status ebe_partition_export_batch(const ebe_mesh* meshes, int32_t n_problems, ebe_partition_sizes* sizes,
                                      int32_t* patch_off, int32_t* slot_elem, uint16_t* lconn,
                                      int32_t* patch_meta, int32_t* pnode, int32_t* col_ptr, int32_t* sh_node,
                                      int32_t* sh_ptr, int32_t* sh_slot);

#ifdef __cplusplus
}
#endif

#endif /* EBE_H */
