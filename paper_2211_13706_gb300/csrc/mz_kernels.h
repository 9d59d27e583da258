// Launch interface of the CUDA kernels (host side of mz_kernels.cu and mz_build.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "mz_internal.h"

namespace mz {

struct ScanShape {
    int32_t BW = 1;          // batch columns per tile
    int32_t R = 256;         // threads per column
    int32_t groups = 1;      // column groups (grid.y)
    int64_t tile_slots = 0;  // slots per tile
    int64_t ntiles = 0;      // tiles per column group
};

struct ScanArgs {
    const int32_t *slot_node;
    int64_t nslots;
    int32_t B, BW, R;
    int64_t ntiles;          // per column group
    const void *f;
    int64_t nB;              // n * B (F32C: offset of the lo plane)
    void *P;                 // [nslots][B] prefix array
    uint32_t *counters;      // [groups] dynamic tile ids (zeroed before the launch)
    uint32_t *flags;         // [groups * ntiles] look-back status (zeroed before the launch)
    void *agg, *inc;         // [groups * ntiles * BW] tile aggregates / inclusive prefixes
    uint32_t *status;
    int64_t spin_limit;
    int64_t withhold;        // test hook: tile whose look-back flag is never published (-1: none)
    int32_t pair_words;      // set by the launcher: F32C prefixes stored in column pairs (f32c_pair_words)
};

// F32C with B a power of two >= 32: the chain scan stores the prefixes of columns b, b + 1
// (b even) of a slot as one 16-byte group hi_b, hi_b+1, lo_b, lo_b+1, which the batched
// gather reads as packed fp32 pairs; the Moebius double-word copies Q are kept the same
// way for the leaf gather. Other batch sizes keep one (hi, lo) word per column.
inline bool f32c_pair_words(int64_t B) { return B >= 32 && (B & (B - 1)) == 0; }

struct GatherArgs {
    int32_t blocks_per_sm;    // grid size: resident 256-thread blocks per SM
    const int32_t *Nt;
    const int64_t *tile_off;  // [ntiles] start of each tile in Nt
    const int32_t *tile_k;    // [ntiles] row length of each tile
    const int32_t *row_node;
    int64_t ntiles;
    int32_t B;
    const void *P;
    void *g;
    int64_t nB;
    int64_t nslots;           // rows of P; nslots * B < 2^32 lets the batched gather index in 32 bits
    uint32_t *status;         // MZ_DEBUG builds: where a failed bounds check is reported
};

struct MobArgs {
    const int32_t *Nm;          // rows in processing order, concatenated
    const int64_t *mob_off;     // [n] start of each row in Nm
    const int32_t *mob_kp;      // [n] its length (a multiple of 16)
    int32_t kpad_max;           // longest row
    int32_t blocks_per_sm;      // one-thread-per-row kernel: resident blocks of 128 per SM
    const int32_t *mob_node;
    const int32_t *mob_slot;
    const int32_t *mob_level;   // level of each processed row
    int32_t pace_ns;            // sleep per level of distance before polling (0: none)
    int64_t n;                  // rows of the forward substitution's schedule
    int64_t nslots;             // slots of the prefix array (bound of every map entry)
    int32_t B;
    const void *g;
    void *f;
    int64_t nB;                 // (all nodes) * B: offset of the lo plane of F32C values
    unsigned long long *P;
    uint32_t *status;
    int64_t spin_limit;
    int64_t withhold;        // test hook: processing index whose y' is never published (-1: none)
    unsigned char *esc;      // int64: [nslots][B] escape flags of words equal to the sentinel (else null)
    float2 *Q;               // F32C, U-level schedule: [nslots][B] double-word copies of y' (else null)
    const uint8_t *slot_ref; // U-level schedule: 1 at the slots the forward substitution computes
                             // (read by another row); null: every slot (antichain schedule)
    // leaf gather (U-level schedule): the zeta gather's tiles, and per tile row the slot
    // of a row no other row reads (-1: a row of the forward substitution, or padding)
    const int32_t *Nt;
    const int64_t *tile_off;
    const int32_t *tile_k;
    const int32_t *row_node;
    const int32_t *row_leaf;
    int64_t ntiles;
    int32_t gather_blocks_per_sm;
    int32_t lanes;           // batch 1: lanes per row of the forward substitution (1, 2, 4, 8, 16 or 32)
    int32_t tree_w;          // batch 1: smallest power of two >= the longest row's chunks of 16 entries
    int32_t pair_q;              // set by the launcher: Q in column pairs (F32C, f32c_pair_words)
};

// Device build (mz_build.cu).
struct BuildNivArgs {
    const int64_t *ptr;         // [n + 1] children lists (CSR)
    const int32_t *adj;         // children
    const int32_t *order;       // [n] nodes bottom-up (ascending height)
    const int32_t *node_slot;   // [n]
    const int32_t *chain_id;    // [n]
    const int32_t *base;        // [k] zero slot of each chain
    const int32_t *topo_pos;    // [n] position in the host's topological order
    int64_t n;
    int32_t k;
    int32_t *N;                 // [n][k] out: the map, row r = slot - chain - 1
    int32_t *uslot;             // [n + k] out: U level by slot; -1 preset (stays -1 at zero slots)
    int32_t *rowcnt;            // [n] out: finite entries of each row, own chain included
    uint32_t *ready;            // [n] 0 until the node's row is published (zeroed before the launch)
    uint32_t *ticket;           // claim counter (zeroed)
    int32_t *bad;               // largest topo_pos of a node whose chain check fails (-1 preset)
    unsigned long long *nnz;    // total finite entries (zeroed)
    uint32_t *status;           // MZ_ERR_TIMEOUT after a wait ran out (zeroed)
    int64_t spin_limit;
    // Plans of several posets (null for one): every node's poset, and per poset its
    // number of chains, first chain, first row and the start of its rows in N (a poset's
    // rows are as wide as its own number of chains). Rows, slots, chains and nodes are
    // numbered over the union; k is then the widest poset's number of chains.
    const int32_t *comp;        // [n]
    const int32_t *comp_k;
    const int32_t *comp_koff;
    const int64_t *comp_roff;
    const int64_t *comp_moff;
};

struct BuildMobArgs {
    const int32_t *N;           // [n][k] row-major map
    int32_t k;
    const int32_t *mrow;        // [n] row of the i-th row of the schedule
    const int64_t *moff;        // [n] its start in Nm
    const int32_t *mkp;         // [n] its padded length
    const int32_t *mslot;       // [n] slot of its element (the own chain's entry)
    const int32_t *key_slot;    // [n + k] sort key of the element in each slot, -1 at zero slots
    int64_t n;
    int32_t *Nm;                // out, zeroed before the launch
    const int64_t *row_moff;    // plans of several posets: start of each schedule row's map row in N
    const int32_t *row_k;       // and its width (null for one poset: mrow[i] * k, width k)
};

// Sparse map, one height level [lo, lo + cnt) of `order` per launch pair.
struct SparseLevelArgs {
    const int64_t *ptr;
    const int32_t *adj;
    const int32_t *order;
    int64_t lo, cnt;
    const int32_t *node_slot;
    const int32_t *chain_id;
    const int32_t *slot_chain;  // [n + k] chain of each slot
    const int32_t *base;        // [k] zero slot of each chain
    const int32_t *topo_pos;
    int64_t *row_beg;           // [n] out: start of row r in pool
    int32_t *row_len;           // [n] out: its length (finite entries, own chain included)
    int32_t *pool;              // rows, appended in any order
    unsigned long long *pool_top;
    int64_t pool_cap;           // entries the pool holds
    int64_t *cand_off;          // [cnt + 1] candidate-list offsets (written by launch_sparse_bounds)
    unsigned long long *cand;   // candidate lists (scratch)
    int32_t *uslot;
    int32_t *bad;
    uint32_t *status;
};

struct BuildMobSparseArgs {
    const int64_t *row_beg;
    const int32_t *row_len;
    const int32_t *pool;
    const int32_t *mrow;
    const int64_t *moff;
    const int32_t *mkp;
    const int32_t *mslot;
    const int32_t *key_slot;
    int64_t n;
    int32_t *Nm;
};

cudaError_t launch_sparse_bounds(const SparseLevelArgs &a, int num_sms, cudaStream_t st);
cudaError_t launch_sparse_merge(const SparseLevelArgs &a, int num_sms, cudaStream_t st);
cudaError_t launch_build_tiles_sparse(const int64_t *row_beg, const int32_t *row_len, const int32_t *pool,
                                      const int32_t *order, int64_t n, int64_t ntiles, const int64_t *tile_off,
                                      const int32_t *tile_k, int32_t *Nt, int num_sms, cudaStream_t st);
cudaError_t launch_build_mob_rows_sparse(const BuildMobSparseArgs &a, int num_sms, cudaStream_t st);
cudaError_t launch_build_niv(const BuildNivArgs &a, int num_sms, cudaStream_t st);
cudaError_t launch_build_tiles(const int32_t *N, int64_t n, int32_t k, int32_t *Nt, int num_sms, cudaStream_t st);
// Tiles of a plan of several posets: tile t holds tile_rows[t] rows of width tile_k[t] that
// start at N + tile_moff[t], and goes to Nt + tile_off[t] (padding rows read slot 0).
cudaError_t launch_build_tiles_var(const int32_t *N, int64_t ntiles, const int64_t *tile_moff, const int32_t *tile_k,
                                   const int32_t *tile_rows, const int64_t *tile_off, int32_t *Nt, int num_sms,
                                   cudaStream_t st);
cudaError_t launch_build_mob_rows(const BuildMobArgs &a, int num_sms, cudaStream_t st);
// Alg. 1 on the device (maximum matching for a minimum path cover), see mz_build.cu.
cudaError_t launch_match_greedy(const int64_t *ptr, const int32_t *adj, int64_t n, int32_t *match_u,
                                int32_t *match_v, uint32_t *changed, int num_sms, cudaStream_t st);
cudaError_t launch_match_roots(const int64_t *ptr, int64_t n, const int32_t *match_u, int32_t *root,
                               int32_t *frontier, unsigned long long *count, int num_sms, cudaStream_t st);
cudaError_t launch_match_expand(const int64_t *ptr, const int32_t *adj, const int32_t *frontier, int64_t fcount,
                                int32_t *next, unsigned long long *ncount, const int32_t *match_u,
                                const int32_t *match_v, int32_t *parent_v, int32_t *root, uint32_t *root_done,
                                int32_t *ends, unsigned long long *ecount, int num_sms, cudaStream_t st);
cudaError_t launch_match_augment(const int32_t *ends, int64_t ecount, int64_t n, const int32_t *parent_v,
                                 int32_t *match_u, int32_t *match_v, uint32_t *status, int num_sms,
                                 cudaStream_t st);
// Marks (slot_ref[s] = 1) every slot that some tile row holds as an entry of another
// chain: the rows of the forward substitution. slot_ref is zeroed before the launch.
cudaError_t launch_mark_referenced(const int32_t *Nt, const int64_t *tile_off, const int32_t *tile_k,
                                   const int32_t *row_node, int64_t ntiles, const int32_t *node_slot,
                                   const int32_t *slot_node, uint8_t *slot_ref, int num_sms, cudaStream_t st);

ScanShape scan_shape(int64_t nslots, int32_t B);
void mark_event(int i, cudaStream_t s);   // profiling hook of mz_set_launch_events
cudaError_t launch_scan(int dtype, const ScanArgs &a, const ScanShape &sh, cudaStream_t st);
cudaError_t launch_gather(int dtype, const GatherArgs &a, int num_sms, cudaStream_t st);
cudaError_t launch_mobius(int dtype, const MobArgs &a, const int32_t *slot_node, int64_t nslots, bool anti,
                          int num_sms, cudaStream_t st, int *launches);

}  // namespace mz
