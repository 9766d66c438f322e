// Internal declarations shared by the translation units of libebe.so.
// Not part of the public ABI (include/ebe.h is).
#pragma once

#include <cstdint>
#include <memory>
#include <new>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "ebe.h"

namespace ebe {

// Elements per patch.  A patch is a run of elements that one CTA processes:
// it gathers the patch's nodes into shared memory, applies every element
// matrix and sums the contributions per node in shared memory.
constexpr int kPatch = 1024;
// Bit 31 of a stored node id marks a Dirichlet node (its rows are zeroed).
constexpr uint32_t kDirichletBit = 0x80000000u;
constexpr int32_t kNodeMask = 0x7fffffff;
constexpr int kMaxColours = 64;
// Meshes whose patches need more colours than this (tetrahedra) have the FP32
// patch pass add element products through per-warp copies of the node sums:
// a warp walks each of its colours from the colour's first slot, 32 slots at a
// time.  With fewer colours it runs colour rounds, a warp holding 32
// consecutive slots counted from the patch's first slot.  The planner numbers
// local nodes for the shared-memory banks of the same access groups.
constexpr int kWarpSchemeColours = 16;

// Per-patch metadata (32 bytes).
struct PatchMeta {
    int32_t node_off;   // first entry of this patch in the local-node table
    int32_t n_nodes;    // local nodes: owned ones first, then shared ones
    int32_t n_owned;    // nodes all of whose elements lie in this patch
    int32_t halo_off;   // first halo slot of this patch (one per shared node)
    int32_t n_el;       // elements in the patch (<= kPatch; slots beyond are padding)
    int32_t col_off;    // first entry of this patch's colour offsets
    int32_t n_col;      // colours used inside the patch
    int32_t pad;
};

// Host-side element partition, built once per mesh.
// A std::vector whose resize() leaves new elements of trivial types
// uninitialised: the partition's large tables are written in full by host
// threads, so the first touch of their pages happens there, in parallel,
// instead of in a serial zero fill.
template <typename T>
struct NoInitAlloc : std::allocator<T> {
    template <typename U>
    struct rebind {
        using other = NoInitAlloc<U>;
    };
    NoInitAlloc() = default;
    template <typename U>
    NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
    template <typename U>
    void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
        ::new (static_cast<void*>(p)) U;
    }
    template <typename U, typename... A>
    void construct(U* p, A&&... a) {
        ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
    }
};
template <typename T>
using HostVec = std::vector<T, NoInitAlloc<T>>;

struct HostPlan {
    int dim = 0, nb = 0;
    int64_t n_n = 0, n_e = 0;
    int64_t n_patches = 0, n_slots = 0;
    HostVec<int32_t> slot_elem;   // [n_slots] caller's element id of each slot, -1 = padding
    HostVec<uint16_t> lconn;      // [nb][n_slots] local node id of vertex i of each slot
    HostVec<PatchMeta> meta;      // [n_patches]
    HostVec<int32_t> pnode;       // local-node tables of all patches (global node ids)
    HostVec<int32_t> col_ptr;     // colour offsets (n_col + 1 per patch), slot-relative
    HostVec<int32_t> sh_node;     // [n_shared] nodes touched by >= 2 patches
    HostVec<int32_t> sh_ptr;      // [n_shared + 1] CSR into sh_slot
    HostVec<int32_t> sh_slot;     // [n_halo] halo slots of each shared node, patch order
    int64_t n_halo = 0;
    int max_nodes = 0;
    int max_col = 0;
};

// Host threads for the partition build: EBE_HOST_THREADS if set (>= 1),
// else the hardware's, at most `cap`.
int host_threads(int cap);

// Validate the mesh and build the partition.  Returns an ebe_status.
int build_plan(const ebe_mesh& m, HostPlan& plan, std::string& err);

// Where each problem of a batch sits in the concatenated numbering:
// problem k owns nodes [node_off[k], node_off[k+1]), elements
// [elem_off[k], elem_off[k+1]), patches [patch_off[k], patch_off[k+1]) and
// shared-node rows [shared_off[k], shared_off[k+1]).  A single mesh is a
// batch of one.
struct BatchLayout {
    std::vector<int64_t> node_off, elem_off;
    std::vector<int32_t> patch_off, shared_off;
};

// Partition every mesh of a batch on its own (exactly as build_plan would,
// on up to `threads` host threads) and concatenate the partitions: node and
// element ids, local-node tables, halo slots and colour offsets are shifted
// by the sizes of the problems before.  No patch mixes two problems.
// All meshes must have the same dim.  Returns an ebe_status; err names the
// failing problem.
int build_batch_plan(const ebe_mesh* meshes, int n_prob, int threads, HostPlan& plan, BatchLayout& lay,
                     std::string& err);

// Greedy colouring of all elements (no two elements of a colour share a
// node), elements of each colour listed in the given slot order.
// Returns the colour count; order receives the slots grouped by colour and
// col_ptr the colour offsets.
int global_colouring(const HostPlan& plan, const std::vector<int32_t>& gconn_slot_major,
                     std::vector<int32_t>& order, std::vector<int64_t>& col_ptr, std::string& err);

}  // namespace ebe
