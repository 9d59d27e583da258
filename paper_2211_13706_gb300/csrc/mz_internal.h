// Internal plan layout shared by the host build (mz_host.cpp) and the CUDA
// side (mz_abi.cu, mz_kernels.cu). Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/mz.h"

namespace mz {

// Rows of the niv map are stored in *slot order*: chain 0 bottom -> top, then
// chain 1, and so on. The prefix array y' has n + k slots: chain c owns slots
// [base_c, base_c + len_c], where base_c = sum_{c' < c} len_{c'} + c holds a
// constant 0 (it stands for niv_c(x) = infinity), and the element at chain
// position p (0 = bottom) sits at slot base_c + 1 + p. Row r of the map is the
// element at slot r + c + 1. Every map entry is a slot index, so the gather
// needs no branch for infinity.
constexpr int kTileRows = 32;  // rows per tile of the tiled (column-major within a tile) map
constexpr int64_t kDenseMaxChains = 512;  // above this many chains the niv map is kept sparse

struct HostSide {
    int64_t n = 0;
    int32_t k = 0;
    int64_t edges = 0;          // distinct edges
    int64_t nnz = 0;            // finite niv entries (self entries included)
    int32_t nlevels = 0;        // antichain levels (heights)
    int32_t nulevels = 0;       // levels of U's dependency graph
    int32_t max_chain = 0;
    std::vector<int32_t> topo;       // [n] topological order, a largest element first
    std::vector<int32_t> chain_id;   // [n]
    std::vector<int32_t> chain_pos;  // [n] 0 = bottom
    std::vector<int64_t> chain_base; // [k + 1], chain_base[k] = n + k
    std::vector<int32_t> node_slot;  // [n]
    std::vector<int32_t> slot_node;  // [n + k], -1 at zero slots
    std::vector<int32_t> row_node;   // [n] node of row r
    bool sparse = false;             // niv map stored as finite entries only
    std::vector<int32_t> N;          // dense: [n][k] by row, slot indices
    std::vector<int64_t> row_beg;    // sparse: first entry of row r
    std::vector<int32_t> row_len;    // sparse: number of entries of row r (own chain included)
    std::vector<int32_t> ent_chain;  // sparse: chain of each entry, sorted within a row
    std::vector<int32_t> ent_slot;   // sparse: slot of each entry

    // Calls f(chain, slot) for every finite entry of row r (the own chain included).
    template <class F>
    void for_row(int64_t r, F f) const {
        if (sparse) {
            for (int64_t q = row_beg[r], e = q + row_len[r]; q < e; ++q) f(ent_chain[q], ent_slot[q]);
        } else {
            const int32_t *row = &N[(size_t)r * k];
            for (int64_t c = 0; c < k; ++c)
                if (row[c] != (int32_t)chain_base[c]) f((int32_t)c, row[c]);
        }
    }
    // Number of finite entries of row r.
    int64_t row_count(int64_t r) const {
        if (sparse) return row_len[r];
        int64_t cnt = 0;
        for_row(r, [&](int32_t, int32_t) { ++cnt; });
        return cnt;
    }
    std::vector<int32_t> level;      // [n] heights, 1 = minimal
    std::vector<int32_t> ulevel;     // [n] 0 = no dependency on another chain
    // Device build: the niv map exists only on the device (N stays empty, for_row and
    // row_count must not be called); the children lists are kept until the upload.
    bool niv_on_device = false;
    std::vector<int64_t> csr_ptr;    // [n + 1]
    std::vector<int32_t> csr_adj;    // children of each node, ascending ids
};

// Device copies of one side (primal or dual) for all components of the plan. The
// components' slot spaces are concatenated (component p's slot s is global slot
// slot_off[p] + s) and so are their node ids (node_off[p] + x).
struct DeviceSide {
    int64_t n = 0;                 // nodes of all components
    int64_t nslots = 0;            // n + total number of chains
    int32_t *slot_node = nullptr;  // [nslots] global node or -1 (zero slot), padded to 64 entries
    int32_t *Nt = nullptr;         // tiles of 32 rows, column-major in a tile, concatenated
    int64_t *tile_off = nullptr;   // [ntiles] start of each tile in Nt
    int32_t *tile_k = nullptr;     // [ntiles] row length (k of the tile's component)
    int32_t *row_node = nullptr;   // [ntiles * 32] global node of each tile row, -1 for padding
    int64_t ntiles = 0;
    int32_t *Nm = nullptr;         // Moebius rows in processing order, concatenated
    int64_t *mob_off = nullptr;    // [n] start of the i-th processed row in Nm
    int32_t *mob_kp = nullptr;     // [n] its length: k of its component rounded up to 16
    int32_t *mob_node = nullptr;   // [n] global node of the i-th processed row
    int32_t *mob_slot = nullptr;   // [n] its global slot
    int32_t *mob_level = nullptr;  // [n] its level in the schedule
    int32_t kpad_max = 0;
    int32_t k_max = 0;
    int64_t nmob = 0;              // rows of the Moebius schedule (U-level: the referenced rows only)
    int32_t mob_kp_max = 0;        // longest row of the Moebius schedule (padded length)
    int64_t nmob_entries = 0;      // their finite entries on other chains
    uint8_t *slot_ref = nullptr;   // U-level schedule: [nslots] 1 = a slot another row reads
    int32_t *row_leaf = nullptr;   // U-level schedule: [ntiles * 32] slot of a tile row no other row
                                   // reads (computed by the leaf gather), -1 otherwise
};

}  // namespace mz

struct mz_plan {
    std::vector<mz::HostSide> host[2];   // per component: primal, dual
    std::vector<int64_t> node_off;       // [components + 1]
    std::vector<int64_t> slot_off;       // [components + 1] (same for both sides)
    std::vector<int64_t> chain_off;      // [components + 1]
    mz::DeviceSide dev[2];
    bool has_dual = false;
    bool host_only = false;
    int32_t schedule = MZ_SCHED_ULEVEL;
    int64_t spin_limit = 1ll << 22;
    int64_t withhold = -1;          // test hook (see mz_build_opts::debug_withhold)
    uint32_t *d_status = nullptr;   // device status word (MZ_OK / MZ_ERR_TIMEOUT)
    int device = -1;
    int num_sms = 0;
    int32_t mob_blocks_per_sm = 2;  // wavefront: resident blocks of 128 threads per SM (per lane group)
    int32_t mob_pace_ns = 600;      // wavefront pacing per level of distance (0: none)
    int32_t gather_blocks_per_sm = 32;
    int32_t mob_lanes = 32;         // batch-1 wavefront: lanes per row (1, 2, 4, 8, 16, 32)
    int64_t device_bytes = 0;
    std::vector<void *> allocations;
    void *(*dev_alloc)(size_t, void *) = nullptr;
    void (*dev_free)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;

    int64_t n_total() const { return node_off.back(); }
    int64_t slots_total() const { return slot_off.back(); }
    size_t components() const { return host[0].size(); }
};

namespace mz {

// Host build of one side: validates, orders, decomposes into chains, builds
// the niv map (Thm. 4) and both level structures. chain_in may be null.
// niv_format: 0 = dense unless k > kDenseMaxChains, 1 = dense, 2 = sparse.
// device_niv: stop after the slot layout and the heights (the device build does the rest).
// matcher: computes Alg. 1's matching when chain_in is null (null: the host's).
// A maximum matching of Alg. 1's bipartite graph over the children lists (ptr, adj):
// next[u] = the node matched below u, or -1.
using Matcher = std::function<mz_status(int64_t n, const std::vector<int64_t> &ptr, const std::vector<int32_t> &adj,
                                        std::vector<int32_t> &next, std::string &err)>;

mz_status build_host_side(int64_t n, const std::vector<int32_t> &src, const std::vector<int32_t> &dst,
                          const int32_t *chain_in, int niv_format, bool device_niv, HostSide &H, std::string &err,
                          const Matcher *matcher = nullptr);

void set_last_error(const std::string &s);

// Plan files (mz_plan_io.cpp): the host sides of every poset (the dual included) and the
// plan's flags. load_host_sides fills p->host, p->has_dual and the offsets of the union,
// after checking every length and index; the device part is built from them afterwards.
mz_status save_host_sides(const mz_plan *p, const char *path, std::string &err);
mz_status load_host_sides(mz_plan *p, const char *path, std::string &err);

// Caps the host threads build_host_side uses on the calling thread (0: no cap); set to 1
// where several posets are built at once, one per thread.
void set_host_threads_cap(int cap);

}  // namespace mz
