// Host-side element partition of the EbE operator.
//
// The paper replaces the Boolean matrices C_e, R_e by index arrays (Sec. 2,
// ind_e / indt).  On the GPU the same information is regrouped once per mesh
// so that the residual sum_e C_e^T A_e C_e x can be formed deterministically
// without atomics:
//   1. elements are sorted along a Morton (Z-order) curve of their centroids
//      and cut into patches of kPatch consecutive elements;
//   2. each patch lists its distinct nodes ("local nodes"); a node all of
//      whose elements lie in the patch is "owned", the others are "shared";
//   3. inside a patch the elements are greedily coloured so that no two
//      elements of one colour share a node, and stored colour by colour;
//   4. the local node ids of a patch are chosen so that the 32 nodes one
//      warp touches in a colour round fall in distinct shared-memory banks
//      where possible (owned ids first, then shared);
//   5. every shared local node gets a halo slot; for every shared node the
//      halo slots are listed in patch order (a CSR), which fixes the order in
//      which its partial sums are added.
// Validation, Morton keys, the sort, the patches and the halo CSR run on up to
// 16 host threads; the result does not depend on the thread count.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <thread>

#include "ebe_internal.h"

namespace ebe {
namespace {

// Spread the low 32 bits of v so that bit k moves to bit 2k.
uint64_t spread2(uint64_t v) {
    v &= 0xffffffffull;
    v = (v | (v << 16)) & 0x0000ffff0000ffffull;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

// Spread the low 21 bits of v so that bit k moves to bit 3k.
uint64_t spread3(uint64_t v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x001f00000000ffffull;
    v = (v | (v << 16)) & 0x001f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Run f(t, begin, end) on `threads` host threads over [0, n) in contiguous
// blocks of at least `grain` items.
template <typename F>
void parallel_blocks(int64_t n, int threads, F f, int64_t grain = 65536) {
    const int nt = int(std::max<int64_t>(1, std::min<int64_t>(threads, n / grain + 1)));
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(f, t, n * t / nt, n * (t + 1) / nt);
    f(0, 0, n / nt);
    for (auto& th : pool) th.join();
}

// Lowest i in [0, n) with bad(i), or n if none: each host thread scans a
// contiguous block up to its first failure; the lowest block result wins.
template <typename F>
int64_t first_failing(int64_t n, int threads, F bad) {
    std::vector<int64_t> first(size_t(std::max(threads, 1)), n);
    parallel_blocks(n, threads, [&](int t, int64_t b, int64_t e) {
        for (int64_t i = b; i < e; ++i)
            if (bad(i)) { first[size_t(t)] = i; return; }
    });
    return *std::min_element(first.begin(), first.end());
}

// Stable LSD radix sort of 64-bit values by their bits [lo_bit, 64) (the
// bits below keep their input order), 10-bit digits, the histogram and the
// scatter of each pass split over host threads in contiguous blocks.
void radix_sort_u64(HostVec<uint64_t>& a, int lo_bit, int threads) {
    constexpr int kBits = 10, kBuckets = 1 << kBits;
    const int64_t n = int64_t(a.size());
    HostVec<uint64_t> tmp(a.size());   // every entry is written by each pass's scatter
    uint64_t any = 0;
    for (uint64_t v : a) any |= v;
    const int nt = int(std::max<int64_t>(1, std::min<int64_t>(threads, n / 65536 + 1)));
    std::vector<int64_t> count(size_t(nt) * kBuckets);
    for (int shift = lo_bit; shift < 64; shift += kBits) {
        const uint64_t mask = (shift + kBits >= 64) ? (~0ull >> shift) : uint64_t(kBuckets - 1);
        if (((any >> shift) & mask) == 0) continue;        // digit is zero everywhere
        std::fill(count.begin(), count.end(), 0);
        parallel_blocks(n, nt, [&](int t, int64_t b, int64_t e) {
            int64_t* c = count.data() + size_t(t) * kBuckets;
            for (int64_t i = b; i < e; ++i) ++c[(a[i] >> shift) & mask];
        });
        int64_t sum = 0;                                    // bucket-major, then block order: stable
        for (int d = 0; d < kBuckets; ++d)
            for (int t = 0; t < nt; ++t) {
                int64_t& c = count[size_t(t) * kBuckets + d];
                const int64_t v = c;
                c = sum;
                sum += v;
            }
        parallel_blocks(n, nt, [&](int t, int64_t b, int64_t e) {
            int64_t* c = count.data() + size_t(t) * kBuckets;
            for (int64_t i = b; i < e; ++i) tmp[c[(a[i] >> shift) & mask]++] = a[i];
        });
        a.swap(tmp);
    }
}

// Ascending sort of distinct 64-bit values: one bucket pass on the 12 highest
// occupied bits (histogram and scatter split over host threads in contiguous
// blocks), then every bucket sorted on its own by the threads, in cache.
// Distinct values have one sorted order, so the result equals any other
// sort's.  Buckets above 2^20 values (a strongly clustered input) fall back
// to the LSD radix sort of the whole array.
void sort_distinct_u64(HostVec<uint64_t>& a, int threads) {
    constexpr int kBits = 12, kBuckets = 1 << kBits;
    constexpr int64_t kMaxBucket = int64_t(1) << 20;
    const int64_t n = int64_t(a.size());
    if (n < 2) return;
    uint64_t any = 0;
    for (uint64_t v : a) any |= v;
    if (any == 0) return;
    const int hb = 63 - __builtin_clzll(any);
    const int shift = std::max(0, hb + 1 - kBits);
    const int nt = int(std::max<int64_t>(1, std::min<int64_t>(threads, n / 65536 + 1)));
    std::vector<int64_t> count(size_t(nt) * kBuckets, 0);
    parallel_blocks(n, nt, [&](int t, int64_t b, int64_t e) {
        int64_t* c = count.data() + size_t(t) * kBuckets;
        for (int64_t i = b; i < e; ++i) ++c[a[i] >> shift];
    });
    std::vector<int64_t> start(kBuckets + 1, 0);
    int64_t sum = 0, biggest = 0;
    for (int d = 0; d < kBuckets; ++d) {
        start[d] = sum;
        for (int t = 0; t < nt; ++t) {
            int64_t& c = count[size_t(t) * kBuckets + d];
            const int64_t v = c;
            c = sum;
            sum += v;
        }
        biggest = std::max(biggest, sum - start[d]);
    }
    start[kBuckets] = sum;
    if (biggest > kMaxBucket) { radix_sort_u64(a, 0, threads); return; }
    HostVec<uint64_t> tmp(a.size());   // every entry is written by the scatter
    parallel_blocks(n, nt, [&](int t, int64_t b, int64_t e) {
        int64_t* c = count.data() + size_t(t) * kBuckets;
        for (int64_t i = b; i < e; ++i) tmp[c[a[i] >> shift]++] = a[i];
    });
    std::atomic<int> next{0};
    auto work = [&]() {
        for (int d = next++; d < kBuckets; d = next++) std::sort(tmp.begin() + start[d], tmp.begin() + start[d + 1]);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (auto& th : pool) th.join();
    a.swap(tmp);
}

}  // namespace

int host_threads(int cap) {
    if (const char* env = std::getenv("EBE_HOST_THREADS")) {   // a user's cap, 1..64
        const int v = std::atoi(env);
        if (v >= 1) return std::min(v, std::min(cap, 64));
    }
    const unsigned h = std::thread::hardware_concurrency();
    return int(std::max(1u, std::min(unsigned(cap), h)));
}

namespace {

int bits_for(uint64_t n) {  // smallest b with n <= 2^b
    int b = 0;
    while (b < 64 && (uint64_t(1) << b) < n) ++b;
    return b;
}

}  // namespace

int build_plan(const ebe_mesh& m, HostPlan& P, std::string& err) {
    if (m.dim != 2 && m.dim != 3) { err = "dim must be 2 or 3"; return EBE_INVALID_ARG; }
    if (m.n_b != m.dim + 1) { err = "n_b must be dim + 1 (P1 simplices)"; return EBE_INVALID_ARG; }
    if (m.n_n < 1 || m.n_n > int64_t(kNodeMask)) { err = "n_n out of range"; return EBE_INVALID_ARG; }
    if (m.n_e < 1 || m.n_e * m.n_b > int64_t(kNodeMask)) { err = "n_e out of range"; return EBE_INVALID_ARG; }
    if (!m.coords || !m.elems) { err = "coords and elems must be non-NULL"; return EBE_INVALID_ARG; }
    const int dim = m.dim, nb = m.n_b;
    const int64_t n_n = m.n_n, n_e = m.n_e;
    P = HostPlan();
    P.dim = dim; P.nb = nb; P.n_n = n_n; P.n_e = n_e;

    // ---- validation: finite coords, ids in range, distinct within an element,
    // every node in some element.  Each check runs over host threads in
    // blocks; the lowest failing index is reported, as a serial scan would.
    const int threads = host_threads(16);
    {
        const int64_t nc = n_n * dim;
        const int64_t bad = first_failing(nc, threads, [&](int64_t k) { return !std::isfinite(m.coords[k]); });
        if (bad < nc) { err = "non-finite coordinate at node " + std::to_string(bad / dim); return EBE_INVALID_ARG; }
    }
    auto element_fault = [&](int64_t e) {
        const int32_t* v = m.elems + e * nb;
        for (int i = 0; i < nb; ++i) {
            if (v[i] < 0 || v[i] >= n_n) return true;
            for (int j = 0; j < i; ++j) if (v[j] == v[i]) return true;
        }
        return false;
    };
    const int64_t bad_e = first_failing(n_e, threads, element_fault);
    if (bad_e < n_e) {
        const int32_t* v = m.elems + bad_e * nb;
        for (int i = 0; i < nb; ++i) {
            if (v[i] < 0 || v[i] >= n_n) {
                err = "element " + std::to_string(bad_e) + " has node id " + std::to_string(v[i]) + " outside [0, n_n)";
                return EBE_INDEX_RANGE;
            }
            for (int j = 0; j < i; ++j)
                if (v[j] == v[i]) { err = "element " + std::to_string(bad_e) + " repeats node " + std::to_string(v[i]); return EBE_INDEX_RANGE; }
        }
    }
    HostVec<int32_t> inc(n_n);  // elements per node (ids are valid now)
    parallel_blocks(n_n, threads, [&](int, int64_t g0, int64_t g1) { std::fill(inc.begin() + g0, inc.begin() + g1, 0); });
    parallel_blocks(n_e * nb, threads, [&](int, int64_t k0, int64_t k1) {
        for (int64_t k = k0; k < k1; ++k) __atomic_fetch_add(&inc[m.elems[k]], 1, __ATOMIC_RELAXED);
    });
    {
        const int64_t bad = first_failing(n_n, threads, [&](int64_t g) { return inc[g] == 0; });
        if (bad < n_n) { err = "node " + std::to_string(bad) + " belongs to no element"; return EBE_INVALID_ARG; }
    }

    // ---- Morton order of element centroids
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) { lo[d] = std::numeric_limits<double>::max(); hi[d] = -lo[d]; }
    {
        // per-thread bounds, then combined (min and max are exact in any order)
        std::vector<double> tb(size_t(threads) * 6);
        for (int t = 0; t < threads; ++t)
            for (int d = 0; d < 3; ++d) { tb[t * 6 + d] = lo[d]; tb[t * 6 + 3 + d] = hi[d]; }
        parallel_blocks(n_n, threads, [&](int t, int64_t k0, int64_t k1) {
            double* b = tb.data() + size_t(t) * 6;
            for (int64_t k = k0; k < k1; ++k)
                for (int d = 0; d < dim; ++d) {
                    b[d] = std::min(b[d], m.coords[k * dim + d]);
                    b[3 + d] = std::max(b[3 + d], m.coords[k * dim + d]);
                }
        });
        for (int t = 0; t < threads; ++t)
            for (int d = 0; d < dim; ++d) { lo[d] = std::min(lo[d], tb[t * 6 + d]); hi[d] = std::max(hi[d], tb[t * 6 + 3 + d]); }
    }
    const int ebits = bits_for(uint64_t(n_e));
    const int kbits_axis = std::min((64 - ebits) / dim, dim == 2 ? 32 : 21);
    const double qmax = double((uint64_t(1) << kbits_axis) - 1);
    HostVec<uint64_t> keys(n_e);
    parallel_blocks(n_e, threads, [&](int, int64_t e0, int64_t e1) {
        for (int64_t e = e0; e < e1; ++e) {
            const int32_t* v = m.elems + e * nb;
            uint64_t q[3] = {0, 0, 0};
            for (int d = 0; d < dim; ++d) {
                double c = 0;
                for (int i = 0; i < nb; ++i) c += m.coords[int64_t(v[i]) * dim + d];
                c /= nb;
                double span = hi[d] - lo[d];
                double t = span > 0 ? (c - lo[d]) / span : 0.0;
                q[d] = uint64_t(std::min(qmax, std::max(0.0, std::floor(t * qmax + 0.5))));
            }
            uint64_t key = dim == 2 ? (spread2(q[0]) | (spread2(q[1]) << 1))
                                    : (spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2));
            keys[e] = (key << ebits) | uint64_t(e);
        }
    });
    // the low ebits hold the element id, so the keys are distinct and their
    // sorted order is the Morton order with ties kept in element order
    sort_distinct_u64(keys, threads);
    const uint64_t emask = ebits >= 64 ? ~0ull : ((uint64_t(1) << ebits) - 1);

    // ---- patches, built independently on host threads (scratch per thread:
    // an open-addressing table from global node id to local index), then
    // concatenated in patch order
    P.n_patches = (n_e + kPatch - 1) / kPatch;
    P.n_slots = P.n_patches * kPatch;
    // slots of elements are written by their patch below; the padding slots
    // of the last patch are element -1 with local ids 0
    P.slot_elem.resize(size_t(P.n_slots));
    P.lconn.resize(size_t(nb) * P.n_slots);
    for (int64_t s = n_e; s < P.n_slots; ++s) {
        P.slot_elem[s] = -1;
        for (int i = 0; i < nb; ++i) P.lconn[size_t(i) * P.n_slots + s] = 0;
    }
    P.meta.resize(P.n_patches);

    struct PatchOut {
        std::vector<int32_t> lnodes;    // local nodes (owned first), padded to a multiple of 4
        std::vector<int32_t> col_ptr;   // n_col + 1 slot offsets
        int n_nodes = 0, n_owned = 0, n_col = 0;
        int status = EBE_OK;
        const char* msg = nullptr;
    };
    std::vector<PatchOut> outs(size_t(P.n_patches));
    parallel_blocks(P.n_patches, threads, [&](int, int64_t p0, int64_t p1) {
        constexpr int kTable = 1 << 13;   // twice the 4 * kPatch local nodes a patch can have
        static_assert(kTable >= 8 * kPatch, "hash table too small");
        std::vector<int32_t> tkey(kTable, -1), tval(kTable), tcnt(kTable);
        std::vector<int32_t> el(kPatch), first_touch;
        std::vector<int> lid(size_t(kPatch) * 4);
        std::vector<int32_t> gv(size_t(kPatch) * 4);
        std::vector<uint32_t> filled;   // table slots in use, cleared slot by slot after each patch
        std::vector<uint64_t> used;
        std::vector<int> colour(kPatch);
        std::vector<int> cstart, order, gidx, first_set, set_list, set_fill, perm, bank, visit;
        std::vector<int32_t> renum;
        std::vector<uint32_t> set_used;
        auto slot_of = [&](int32_t g) {
            uint32_t hsh = (uint32_t(g) * 2654435761u) >> 19;   // 13 bits
            while (tkey[hsh] != g && tkey[hsh] != -1) hsh = (hsh + 1) & (kTable - 1);
            return hsh;
        };
        for (int64_t p = p0; p < p1; ++p) {
            PatchOut& out = outs[size_t(p)];
            const int64_t e0 = p * kPatch;
            const int n_el = int(std::min<int64_t>(kPatch, n_e - e0));
            // the patch's elements and their global node ids, gathered once
            for (int s = 0; s < n_el; ++s) {
                el[s] = int32_t(keys[e0 + s] & emask);
                const int32_t* v = m.elems + int64_t(el[s]) * nb;
                for (int i = 0; i < nb; ++i) gv[s * nb + i] = v[i];
            }
            // local nodes in first-touch order, with their counts in the patch
            first_touch.clear();
            for (int s = 0; s < n_el; ++s) {
                const int32_t* v = gv.data() + s * nb;
                for (int i = 0; i < nb; ++i) {
                    const uint32_t t = slot_of(v[i]);
                    if (tkey[t] == -1) { tkey[t] = v[i]; tcnt[t] = 0; first_touch.push_back(v[i]); filled.push_back(t); }
                    ++tcnt[t];
                }
            }
            // owned first, then shared, each in first-touch order
            std::vector<int32_t>& lnodes = out.lnodes;
            int n_owned = 0;
            for (int32_t g : first_touch) if (tcnt[slot_of(g)] == inc[g]) { lnodes.push_back(g); ++n_owned; }
            for (int32_t g : first_touch) if (tcnt[slot_of(g)] != inc[g]) lnodes.push_back(g);
            const int n_nodes = int(lnodes.size());
            out.n_nodes = n_nodes;
            out.n_owned = n_owned;
            // (clearing by key would cut probe chains of keys not yet cleared)
            auto reset = [&]() { for (uint32_t t : filled) tkey[t] = -1; filled.clear(); };
            if (n_nodes > 65535) {
                out.status = EBE_INVALID_ARG;
                out.msg = "patch with more than 65535 nodes";
                reset();
                return;
            }
            for (int l = 0; l < n_nodes; ++l) tval[slot_of(lnodes[l])] = l;
            // local ids of the patch's elements, looked up once: lid[s * nb + i]
            for (int s = 0; s < n_el * nb; ++s) lid[s] = tval[slot_of(gv[s])];
            // greedy colouring in Morton order
            used.assign(n_nodes, 0);
            int n_col = 0;
            for (int s = 0; s < n_el; ++s) {
                const int* v = lid.data() + s * nb;
                uint64_t busy = 0;
                for (int i = 0; i < nb; ++i) busy |= used[v[i]];
                if (busy == ~0ull) {
                    out.status = EBE_INVALID_ARG;
                    out.msg = "patch needs more than 64 colours";
                    reset();
                    return;
                }
                const int c = __builtin_ctzll(~busy);   // lowest free colour (busy != ~0 here)
                colour[s] = c;
                n_col = std::max(n_col, c + 1);
                for (int i = 0; i < nb; ++i) used[v[i]] |= (1ull << c);
            }
            out.n_col = n_col;
            // slots: elements grouped by colour, Morton order within a colour
            // (a counting sort by colour: stable, so Morton order is kept)
            cstart.assign(n_col + 1, 0);
            for (int s = 0; s < n_el; ++s) ++cstart[colour[s] + 1];
            for (int c = 0; c < n_col; ++c) cstart[c + 1] += cstart[c];
            out.col_ptr.assign(cstart.begin(), cstart.end());
            order.resize(n_el);
            for (int s = 0; s < n_el; ++s) order[cstart[colour[s]]++] = s;
            // Local numbering for the shared-memory banks.  The patch kernel
            // gives 32 consecutive slots to a warp; in a colour round its
            // lanes read-modify-write the node sums of vertex r of their
            // elements, and they gather x the same way.  Those 32 nodes are
            // distinct, and the accesses take one shared-memory cycle when
            // their local ids are distinct modulo 32 (the bank), more
            // otherwise.  Greedily, in order of first appearance, each node
            // takes a bank that none of its access sets (warp group x colour
            // x vertex) holds yet, among the banks with free ids in its block
            // (owned or shared); the ids then follow the banks.  Sums are taken
            // in colour order whatever the numbering, so results do not change.
            {
                const int ns = int(order.size());
                gidx.assign(ns, 0);
                int n_grp = 0;
                const bool per_warp = n_col > kWarpSchemeColours;   // groups as the kernel's warps walk them
                for (int q = 0, c0 = 0; q < ns; ++q) {
                    const bool new_colour = q > 0 && colour[order[q]] != colour[order[q - 1]];
                    if (new_colour) c0 = q;
                    if (q > 0 && (new_colour || (per_warp ? (q - c0) % 32 == 0 : q % 32 == 0))) ++n_grp;
                    gidx[q] = n_grp;
                }
                ++n_grp;
                const int n_set = n_grp * nb;
                // node -> access sets (CSR)
                first_set.assign(n_nodes + 1, 0);
                for (int q = 0; q < ns; ++q) {
                    const int* v = lid.data() + order[q] * nb;
                    for (int i = 0; i < nb; ++i) ++first_set[v[i] + 1];
                }
                for (int l = 0; l < n_nodes; ++l) first_set[l + 1] += first_set[l];
                set_list.assign(first_set[n_nodes], 0);
                set_fill.assign(first_set.begin(), first_set.end() - 1);
                visit.clear();
                for (int q = 0; q < ns; ++q) {
                    const int* v = lid.data() + order[q] * nb;
                    for (int i = 0; i < nb; ++i) {
                        const int l = v[i];
                        if (set_fill[l] == first_set[l]) visit.push_back(l);   // first appearance
                        set_list[set_fill[l]++] = gidx[q] * nb + i;
                    }
                }
                set_used.assign(n_set, 0u);
                int cap[2][32] = {};
                for (int l = 0; l < n_nodes; ++l) ++cap[l < n_owned ? 0 : 1][l % 32];
                uint32_t open_banks[2] = {0u, 0u};   // bit b: bank b still has a free id in the block
                for (int blk = 0; blk < 2; ++blk)
                    for (int b = 0; b < 32; ++b) open_banks[blk] |= (cap[blk][b] > 0 ? 1u : 0u) << b;
                bank.assign(n_nodes, 0);
                for (int l : visit) {
                    const int blk = l < n_owned ? 0 : 1;
                    uint32_t busy = 0;
                    for (int k = first_set[l]; k < first_set[l + 1]; ++k) busy |= set_used[set_list[k]];
                    const uint32_t open = open_banks[blk];
                    int best;
                    if (open & ~busy) {
                        best = __builtin_ctz(open & ~busy);
                    } else {   // every open bank conflicts somewhere: fewest conflicting sets, lowest bank on ties
                        // the 32 banks' counts as bit planes (plane j holds bit j of every count),
                        // each set added with a ripple carry
                        uint32_t plane[32];
                        int np = 0;
                        for (int k = first_set[l]; k < first_set[l + 1]; ++k) {
                            uint32_t carry = set_used[set_list[k]];
                            for (int j = 0; carry != 0; ++j) {
                                if (j == np) plane[np++] = 0u;
                                const uint32_t t = plane[j] & carry;
                                plane[j] ^= carry;
                                carry = t;
                            }
                        }
                        // the open banks of least count: from the highest plane down, keep those
                        // with a zero bit whenever any has one
                        uint32_t cand = open;
                        for (int j = np - 1; j >= 0; --j) {
                            const uint32_t z = cand & ~plane[j];
                            if (z) cand = z;
                        }
                        best = __builtin_ctz(cand);
                    }
                    bank[l] = best;
                    if (--cap[blk][best] == 0) open_banks[blk] &= ~(1u << best);
                    for (int k = first_set[l]; k < first_set[l + 1]; ++k) set_used[set_list[k]] |= 1u << best;
                }
                // ids by bank, in each block in order of first appearance
                int next[2][32];
                for (int b = 0; b < 32; ++b) {
                    next[0][b] = b;
                    next[1][b] = n_owned + ((b - n_owned % 32) % 32 + 32) % 32;
                }
                perm.assign(n_nodes, 0);
                for (int l : visit) {
                    const int blk = l < n_owned ? 0 : 1;
                    perm[l] = next[blk][bank[l]];
                    next[blk][bank[l]] += 32;
                }
                renum.resize(n_nodes);
                for (int l = 0; l < n_nodes; ++l) renum[perm[l]] = lnodes[l];
                for (int l = 0; l < n_nodes; ++l) lnodes[l] = renum[l];
            }
            for (int q = 0; q < int(order.size()); ++q) {
                const int64_t gs = e0 + q;
                P.slot_elem[gs] = el[order[q]];
                const int* v = lid.data() + order[q] * nb;
                for (int i = 0; i < nb; ++i) P.lconn[size_t(i) * P.n_slots + gs] = uint16_t(perm[v[i]]);
            }
            // each table starts on a 16-byte boundary (bulk copies need it)
            while (lnodes.size() % 4 != 0) lnodes.push_back(lnodes[0]);
            reset();
        }
    }, 16);
    // offsets in patch order; the first failing patch reports
    int64_t n_pnode = 0, n_colptr = 0, halo_count = 0;
    for (int64_t p = 0; p < P.n_patches; ++p) {
        const PatchOut& o = outs[size_t(p)];
        if (o.status != EBE_OK) { err = o.msg; return o.status; }
        PatchMeta& mt = P.meta[p];
        mt.node_off = int32_t(n_pnode);
        mt.n_nodes = o.n_nodes;
        mt.n_owned = o.n_owned;
        mt.halo_off = int32_t(halo_count);
        mt.n_el = int32_t(std::min<int64_t>(kPatch, n_e - p * kPatch));
        mt.col_off = int32_t(n_colptr);
        mt.n_col = o.n_col;
        mt.pad = 0;
        n_pnode += int64_t(o.lnodes.size());
        n_colptr += int64_t(o.col_ptr.size());
        halo_count += o.n_nodes - o.n_owned;
        P.max_nodes = std::max(P.max_nodes, o.n_nodes);
        P.max_col = std::max(P.max_col, o.n_col);
        if (n_pnode > int64_t(kNodeMask) || halo_count > int64_t(kNodeMask)) {
            err = "partition tables exceed 2^31 entries";
            return EBE_INVALID_ARG;
        }
    }
    P.pnode.resize(size_t(n_pnode));
    P.col_ptr.resize(size_t(n_colptr));
    HostVec<int32_t> halo_node(static_cast<size_t>(halo_count));   // halo slot -> global node
    parallel_blocks(P.n_patches, threads, [&](int, int64_t p0, int64_t p1) {
        for (int64_t p = p0; p < p1; ++p) {
            const PatchOut& o = outs[size_t(p)];
            const PatchMeta& mt = P.meta[p];
            std::copy(o.lnodes.begin(), o.lnodes.end(), P.pnode.begin() + mt.node_off);
            std::copy(o.col_ptr.begin(), o.col_ptr.end(), P.col_ptr.begin() + mt.col_off);
            std::copy(o.lnodes.begin() + o.n_owned, o.lnodes.begin() + o.n_nodes, halo_node.begin() + mt.halo_off);
        }
    }, 64);
    outs.clear();
    outs.shrink_to_fit();
    P.n_halo = halo_count;

    // ---- shared nodes: CSR of halo slots in patch order (slots are numbered
    // patch by patch, so ascending slot order is ascending patch order)
    HostVec<int32_t> cnt(n_n);
    parallel_blocks(n_n, threads, [&](int, int64_t g0, int64_t g1) { std::fill(cnt.begin() + g0, cnt.begin() + g1, 0); });
    parallel_blocks(halo_count, threads, [&](int, int64_t s0, int64_t s1) {
        for (int64_t s = s0; s < s1; ++s) __atomic_fetch_add(&cnt[halo_node[s]], 1, __ATOMIC_RELAXED);
    });
    // rows of the shared nodes in ascending node order: per-block counts, then
    // each block numbers its nodes from its prefix
    HostVec<int32_t> node_row(n_n);   // written for every shared node, read only there
    std::vector<int64_t> blk_rows(size_t(threads) + 1, 0);
    parallel_blocks(n_n, threads, [&](int t, int64_t g0, int64_t g1) {
        int64_t c = 0;
        for (int64_t g = g0; g < g1; ++g) c += cnt[g] > 0;
        blk_rows[size_t(t) + 1] = c;
    });
    for (int t = 0; t < threads; ++t) blk_rows[size_t(t) + 1] += blk_rows[size_t(t)];
    const int64_t n_shared = blk_rows[size_t(threads)];
    P.sh_node.resize(n_shared);
    P.sh_ptr.assign(n_shared + 1, 0);
    parallel_blocks(n_n, threads, [&](int t, int64_t g0, int64_t g1) {
        int64_t row = blk_rows[size_t(t)];
        for (int64_t g = g0; g < g1; ++g)
            if (cnt[g] > 0) {
                node_row[g] = int32_t(row);
                P.sh_node[row] = int32_t(g);
                P.sh_ptr[row + 1] = cnt[g];
                ++row;
            }
    });
    for (int64_t k = 0; k < n_shared; ++k) P.sh_ptr[k + 1] += P.sh_ptr[k];
    P.sh_slot.resize(halo_count);
    std::vector<int32_t> fill(P.sh_ptr.begin(), P.sh_ptr.end() - 1);
    for (int64_t s = 0; s < halo_count; ++s) P.sh_slot[fill[node_row[halo_node[s]]]++] = int32_t(s);
    return EBE_OK;
}

int global_colouring(const HostPlan& P, const std::vector<int32_t>& gconn, std::vector<int32_t>& order,
                     std::vector<int64_t>& col_ptr, std::string& err) {
    // gconn: [n_slots][nb] global node ids per slot (padding slots ignored)
    const int nb = P.nb;
    std::vector<uint64_t> used(P.n_n, 0);
    std::vector<uint8_t> colour(P.n_slots, 0xff);
    int n_col = 0;
    for (int64_t s = 0; s < P.n_slots; ++s) {
        if (P.slot_elem[s] < 0) continue;
        uint64_t busy = 0;
        for (int i = 0; i < nb; ++i) busy |= used[gconn[s * nb + i]];
        if (busy == ~0ull) { err = "global colouring needs more than 64 colours"; return -1; }
        int c = 0;
        while (busy & (1ull << c)) ++c;
        colour[s] = uint8_t(c);
        n_col = std::max(n_col, c + 1);
        for (int i = 0; i < nb; ++i) used[gconn[s * nb + i]] |= (1ull << c);
    }
    std::vector<int64_t> cnt(n_col + 1, 0);
    for (int64_t s = 0; s < P.n_slots; ++s) if (colour[s] != 0xff) ++cnt[colour[s] + 1];
    for (int c = 0; c < n_col; ++c) cnt[c + 1] += cnt[c];
    col_ptr = cnt;
    order.assign(size_t(cnt[n_col]), 0);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t s = 0; s < P.n_slots; ++s) if (colour[s] != 0xff) order[fill[colour[s]]++] = int32_t(s);
    return n_col;
}

int build_batch_plan(const ebe_mesh* meshes, int n_prob, int threads, HostPlan& P, BatchLayout& L, std::string& err) {
    if (!meshes || n_prob < 1) { err = "a batch needs at least one mesh"; return EBE_INVALID_ARG; }
    for (int k = 0; k < n_prob; ++k)
        if (meshes[k].dim != meshes[0].dim) { err = "all meshes of a batch must have the same dim"; return EBE_INVALID_ARG; }
    // 1. every problem on its own, in parallel (each plan is independent)
    std::vector<HostPlan> parts(n_prob);
    std::vector<int> status(n_prob, EBE_OK);
    std::vector<std::string> errs(n_prob);
    std::atomic<int> next{0};
    auto work = [&]() {
        for (int k = next++; k < n_prob; k = next++) status[k] = build_plan(meshes[k], parts[k], errs[k]);
    };
    const int nt = std::max(1, std::min(threads, n_prob));
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
    for (int k = 0; k < n_prob; ++k)
        if (status[k] != EBE_OK) { err = "problem " + std::to_string(k) + ": " + errs[k]; return status[k]; }

    // 2. sizes and offsets
    L = BatchLayout();
    L.node_off.assign(n_prob + 1, 0);
    L.elem_off.assign(n_prob + 1, 0);
    L.patch_off.assign(n_prob + 1, 0);
    L.shared_off.assign(n_prob + 1, 0);
    int64_t n_pnode = 0, n_col = 0, n_halo = 0, n_patch = 0, n_sh = 0;
    for (int k = 0; k < n_prob; ++k) {
        const HostPlan& Q = parts[k];
        L.node_off[k + 1] = L.node_off[k] + Q.n_n;
        L.elem_off[k + 1] = L.elem_off[k] + Q.n_e;
        n_patch += Q.n_patches;
        n_sh += int64_t(Q.sh_node.size());
        n_pnode += int64_t(Q.pnode.size());
        n_col += int64_t(Q.col_ptr.size());
        n_halo += Q.n_halo;
        const int64_t lim = int64_t(kNodeMask);
        if (L.node_off[k + 1] > lim || L.elem_off[k + 1] * Q.nb > lim || n_patch > lim || n_pnode > lim ||
            n_halo > lim || n_col > lim) {
            err = "batch exceeds 2^31 nodes, element entries or table entries";
            return EBE_INVALID_ARG;
        }
        L.patch_off[k + 1] = int32_t(n_patch);
        L.shared_off[k + 1] = int32_t(n_sh);
    }

    // 3. concatenation
    P = HostPlan();
    P.dim = parts[0].dim;
    P.nb = parts[0].nb;
    P.n_n = L.node_off[n_prob];
    P.n_e = L.elem_off[n_prob];
    P.n_patches = n_patch;
    P.n_slots = n_patch * kPatch;
    P.n_halo = n_halo;
    P.slot_elem.resize(size_t(P.n_slots));
    P.lconn.resize(size_t(P.nb) * size_t(P.n_slots));
    P.meta.resize(size_t(n_patch));
    P.pnode.resize(size_t(n_pnode));
    P.col_ptr.resize(size_t(n_col));
    P.sh_node.resize(size_t(n_sh));
    P.sh_ptr.assign(size_t(n_sh) + 1, 0);
    P.sh_slot.resize(size_t(n_halo));
    int64_t o_pnode = 0, o_col = 0, o_halo = 0;
    for (int k = 0; k < n_prob; ++k) {
        const HostPlan& Q = parts[k];
        const int32_t nbase = int32_t(L.node_off[k]), ebase = int32_t(L.elem_off[k]);
        const int64_t sbase = int64_t(L.patch_off[k]) * kPatch, shbase = L.shared_off[k];
        for (int64_t s = 0; s < Q.n_slots; ++s) P.slot_elem[sbase + s] = Q.slot_elem[s] < 0 ? -1 : Q.slot_elem[s] + ebase;
        for (int i = 0; i < P.nb; ++i)
            std::copy(Q.lconn.begin() + size_t(i) * Q.n_slots, Q.lconn.begin() + size_t(i + 1) * Q.n_slots,
                      P.lconn.begin() + size_t(i) * P.n_slots + sbase);
        for (int64_t p = 0; p < Q.n_patches; ++p) {
            PatchMeta m = Q.meta[p];
            m.node_off += int32_t(o_pnode);
            m.halo_off += int32_t(o_halo);
            m.col_off += int32_t(o_col);
            P.meta[L.patch_off[k] + p] = m;
        }
        // tables stay 16-byte aligned: every part's node table is a multiple of 4 entries
        for (size_t j = 0; j < Q.pnode.size(); ++j) P.pnode[o_pnode + j] = Q.pnode[j] + nbase;
        std::copy(Q.col_ptr.begin(), Q.col_ptr.end(), P.col_ptr.begin() + o_col);
        for (size_t j = 0; j < Q.sh_node.size(); ++j) {
            P.sh_node[shbase + j] = Q.sh_node[j] + nbase;
            P.sh_ptr[shbase + j + 1] = Q.sh_ptr[j + 1] + int32_t(o_halo);
        }
        for (int64_t j = 0; j < Q.n_halo; ++j) P.sh_slot[o_halo + j] = Q.sh_slot[j] + int32_t(o_halo);
        o_pnode += int64_t(Q.pnode.size());
        o_col += int64_t(Q.col_ptr.size());
        o_halo += Q.n_halo;
        P.max_nodes = std::max(P.max_nodes, Q.max_nodes);
        P.max_col = std::max(P.max_col, Q.max_col);
        parts[k] = HostPlan();   // release this part early
    }
    return EBE_OK;
}

}  // namespace ebe
