// Launch interface of the CUDA kernels (host side of mz_kernels.cu).
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
};

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
    int64_t n;
    int32_t B;
    const void *g;
    void *f;
    int64_t nB;
    unsigned long long *P;
    uint32_t *status;
    int64_t spin_limit;
    int64_t withhold;        // test hook: processing index whose y' is never published (-1: none)
};

ScanShape scan_shape(int64_t nslots, int32_t B);
void mark_event(int i, cudaStream_t s);   // profiling hook of mz_set_launch_events
cudaError_t launch_scan(int dtype, const ScanArgs &a, const ScanShape &sh, cudaStream_t st);
cudaError_t launch_gather(int dtype, const GatherArgs &a, int num_sms, cudaStream_t st);
cudaError_t launch_mobius(int dtype, const MobArgs &a, const int32_t *slot_node, int64_t nslots, bool anti,
                          int num_sms, cudaStream_t st, int *launches);

}  // namespace mz
