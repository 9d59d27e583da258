/*
 * mz.h - fast zeta and Moebius transforms on a finite poset (C ABI).
 *
 * Implements, on one NVIDIA GB300 GPU (sm_103a), the O(n k) transforms of
 * "Fast Moebius and Zeta Transforms" (Pegolotti, Seifert, Pueschel,
 * arxiv 2211.13706):
 *
 *   zeta    g(x) = sum_{y <= x} f(y)               (Thm. 1 left, Cor. 1: g = Z f)
 *   Moebius f(x) = sum_{y <= x} mu(y, x) g(y)      (Thm. 1 right, Cor. 1: f = M g = Z^-1 g)
 *
 * computed through the factorisation Z = U V of Sec. 3 (Eq. zfac): V is a
 * per-chain prefix sum (Eq. zeta_cache) and U sums one entry per chain
 * selected by the reachability map niv (Sec. 2.4, Eq. zeta-fast). The
 * Moebius transform solves U y' = g by forward substitution and then applies
 * V^-1 (Sec. 3 "Fast Moebius transform", Alg. 4). The transposes Z^T and M^T
 * are the same transforms on the dual poset (all edges flipped, Sec. 2.1).
 *
 * A plan (mz_build) holds the one-time precomputation: topological order,
 * chain decomposition, niv map and the processing schedule (Sec. 4). It is
 * built on the host and uploaded to the current CUDA device once. Every
 * transform call is then asynchronous on the caller's stream and runs only
 * hand-written CUDA kernels.
 *
 * Conventions shared by every call
 *  - Nodes are 0 .. n-1 (the caller's ids). An edge src[i] -> dst[i] means
 *    dst[i] <= src[i] (dst is a successor of src, Sec. 2.1). Duplicate and
 *    transitive edges are allowed; they define the same poset.
 *  - A poset function with `batch` columns is a row-major [n][batch] array:
 *    element (x, b) at index x * batch + b.
 *  - MZ_I64 and MZ_F64 values are int64_t / double. MZ_F32C values are
 *    double-word fp32 pairs stored as two planes: the hi plane ([n][batch]
 *    floats) followed directly by the lo plane; the value is hi + lo.
 *    Inputs with plain fp32 data pass a zero lo plane.
 *  - int64 arithmetic wraps on overflow: results are exact modulo 2^64.
 *  - f, g and ws are device pointers the caller owns. Input and output must
 *    not overlap. Calls on one workspace must not overlap in time.
 *  - Errors found on the host are returned directly and nothing is launched.
 *    Errors found on the device (a bounded wait that ran out; in the MZ_DEBUG
 *    build also an index outside its array) are recorded in the plan and
 *    returned by mz_check. Outputs are undefined after an error.
 *
 * Debug build: the same sources compiled with MZ_DEBUG (libmz_debug.so) check
 * every index a transform kernel takes from the niv map or a plan table before
 * using it (MZ_ERR_BOUNDS through mz_check, the access skipped, never a trap)
 * and fill the workspace and the output with a poison pattern (all bytes 0xFF)
 * before each transform, so that a word left unwritten shows in the result.
 */
#ifndef MZ_H
#define MZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *mz_stream; /* a cudaStream_t; NULL = the legacy default stream */

typedef enum {
    MZ_OK = 0,
    MZ_ERR_INVALID_ARG = 1, /* bad size, pointer, id out of range, overlapping buffers, small workspace */
    MZ_ERR_CYCLE = 2,       /* the edges contain a cycle or a self-loop: not a DAG (Sec. 2.1) */
    MZ_ERR_BAD_CHAINS = 3,  /* chain_id does not partition the nodes into chains (Def. 1) */
    MZ_ERR_OOM = 4,         /* host or device allocation failed */
    MZ_ERR_CUDA = 5,        /* a CUDA runtime call failed (mz_last_error() has the text) */
    MZ_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out (reported by mz_check) */
    MZ_ERR_UNSUPPORTED = 7, /* e.g. a transpose call on a plan built without the dual */
    MZ_ERR_NO_DEVICE = 8,   /* the plan was built host-only; transforms need a device plan */
    MZ_ERR_BOUNDS = 9       /* MZ_DEBUG builds only: a kernel read an index from a plan table or the
                               niv map that lies outside its array (reported by mz_check; the
                               access was skipped) */
} mz_status;

typedef enum {
    MZ_I64 = 0,  /* int64 values, exact (wrapping) arithmetic */
    MZ_F64 = 1,  /* fp64 values, plain fp64 arithmetic */
    MZ_F32C = 2  /* fp32 double-word pairs in and out; compensated fp32 scan and gather for
                    zeta, fp64 chain prefixes in the Moebius forward substitution */
} mz_dtype;

typedef enum {
    /* Moebius schedule: levels of U's own dependency graph. Alg. 4 solves U y' = g and
       then applies V^-1; y'(x) depends only on y' at niv_j(x) for the other chains j,
       so x can run as soon as those are done. Default. */
    MZ_SCHED_ULEVEL = 0,
    /* Moebius schedule of Alg. 5 / Alg. 6: antichain levels (heights), one level after
       the other, each x computing f(x) = g(x) - sum_j y'[niv^-_j(x)] directly. */
    MZ_SCHED_ANTICHAIN = 1
} mz_schedule;

typedef struct mz_plan mz_plan;

typedef struct {
    int32_t build_transpose;  /* nonzero: also build the dual poset's plan for mz_zeta_T / mz_mobius_T */
    int32_t host_only;        /* nonzero: build host structures only (no device use at all) */
    int32_t mobius_schedule;  /* an mz_schedule value */
    int32_t mobius_blocks_per_sm; /* resident 128-thread blocks per SM of the Moebius forward
                                     substitution, per lane of a row; 0 = default (2) */
    int32_t mobius_pace_ns;   /* Moebius forward substitution: before polling for a row that is
                                 d levels above the row it just finished, a thread sleeps about
                                 (d - 2) * pace ns, so rows far from the frontier do not load L2
                                 with polls. 0 = default (500); negative = no pacing */
    int32_t niv_format;       /* 0: dense niv map (k entries per node) unless k > 512, then sparse
                                 (only the finite entries, nnz(N) of Sec. 2.4); 1: dense; 2: sparse */
    int64_t spin_limit;       /* bound on polling iterations of every device-side wait; 0 = default (2^22) */
    /* Test hook, 0 = off. v > 0 makes every transform of this plan skip one publication:
       the look-back flag of scan tile v-1 and the y' word of the (v-1)-th row of the
       Moebius schedule, so the waits on it run out and mz_check reports MZ_ERR_TIMEOUT. */
    int64_t debug_withhold;
    /* Optional allocator for the plan's device buffers (both or neither). alloc returns
       device memory of at least `bytes` bytes, 256-byte aligned, or NULL. */
    void *(*dev_alloc)(size_t bytes, void *ctx);
    void (*dev_free)(void *ptr, void *ctx);
    void *alloc_ctx;
    /* Nonzero: build the niv map on the device. The host still checks the edges, orders
       the nodes, finds the chains (Alg. 1), lays out the slots and computes the heights;
       the recurrence of Thm. 4 (Alg. 2), the levels of U's dependency graph, the tiled
       map of the zeta gather and the rows of the Moebius schedule are then computed by
       kernels: for a dense map every node as soon as its children are done, for a sparse
       map one height level after the other. The plan is the one the host build makes,
       entry for entry. A dense map only with k <= 512 (niv_format 1 with more chains:
       MZ_ERR_UNSUPPORTED). mz_build_batch builds all its posets in one dataflow launch
       when every one of them keeps a dense map (else MZ_ERR_UNSUPPORTED). Not with
       host_only (MZ_ERR_INVALID_ARG). A bounded wait that runs out fails the build with
       MZ_ERR_TIMEOUT. 2: as 1, and for a single poset given without chains (chain_id
       NULL) Alg. 1's maximum matching runs on the device too (a greedy maximal matching,
       then phases of augmenting paths, each found by a breadth-first search from every
       free node at once). Its chains come from another maximum matching than the host's:
       the same number k of chains, but the plan may then differ from the host build's.
       Other values: MZ_ERR_INVALID_ARG. */
    int32_t device_build;
} mz_build_opts;

typedef struct {
    int64_t n;             /* number of elements */
    int32_t k;             /* number of chains in the decomposition used */
    int32_t has_transpose; /* the dual plan exists */
    int64_t nnz;           /* nnz(N): finite entries of the niv map, self entries included (Sec. 2.4) */
    int64_t edges;         /* distinct edges after removing duplicates */
    int32_t levels;        /* number of antichain levels = length of the longest chain (Thm. 5) */
    int32_t ulevels;       /* number of levels of U's dependency graph (schedule MZ_SCHED_ULEVEL) */
    int32_t schedule;      /* the mz_schedule the plan was built for */
    int32_t levels_T;      /* the same two numbers for the dual plan (0 without it) */
    int32_t ulevels_T;
    int32_t max_chain;     /* longest chain of the decomposition (q in Sec. 4) */
    int64_t device_bytes;  /* device memory held by the plan (dual included) */
    int32_t components;    /* posets in the plan (1 for mz_build) */
    int32_t sparse;        /* how many of them keep a sparse niv map */
    int64_t wave_rows;     /* rows of the Moebius forward substitution (0 for a host-only plan):
                              with MZ_SCHED_ULEVEL only the elements some row of another chain
                              reads (niv_j(x) = y for an x not on y's chain); the others are
                              computed afterwards by a gather. All n with MZ_SCHED_ANTICHAIN */
    int64_t wave_entries;  /* their finite niv entries on other chains */
} mz_plan_info_t;
/* For a plan of several posets (mz_build_batch) n, k, nnz and edges are totals over
   them and levels, ulevels, levels_T, ulevels_T and max_chain are maxima. */

/* Arrays mz_plan_export can copy out (host memory; no device work, except that the
   niv map of a plan built with device_build is copied back from the device). */
typedef enum {
    MZ_EXPORT_CHAIN_ID = 0, /* int32[n]: chain of each node, 0 .. k-1 */
    MZ_EXPORT_CHAIN_POS = 1,/* int32[n]: position on its chain, 0 = bottom (smallest element) */
    MZ_EXPORT_NIV = 2,      /* int32[n*k]: niv_j(x) as a node id, -1 for infinity, row x col j */
    MZ_EXPORT_LEVEL = 3,    /* int32[n]: antichain level (height), 1 = minimal elements */
    MZ_EXPORT_ULEVEL = 4,   /* int32[n]: level in U's dependency graph, 0 = no dependency */
    MZ_EXPORT_TOPO = 5      /* int32[n]: a topological order, a largest element first */
} mz_export;

/*
 * mz_build - the one-time precomputation for a poset (Sec. 4: Alg. 1 chain
 * decomposition, Alg. 2 niv map via Thm. 4, Alg. 6 levels).
 *   n         number of nodes, 1 <= n <= 2^30
 *   m         number of edges, m >= 0
 *   src, dst  host arrays of m node ids; edge src[i] -> dst[i] means dst[i] <= src[i]
 *   chain_id  optional host array of n values: the caller's chain decomposition
 *             (ids need not be dense). Each class must be totally ordered in the poset,
 *             else MZ_ERR_BAD_CHAINS. NULL: the build computes a minimum path cover of
 *             the DAG by maximum bipartite matching (Alg. 1). That is a chain
 *             decomposition, but it reaches the width only when the edge set is
 *             transitively closed.
 *   opts      optional (NULL = defaults)
 *   out       receives the plan; NULL on error
 * The host arrays are only read during the call. The plan's device buffers are
 * allocated on the current CUDA device (skipped with opts->host_only). Returns
 * MZ_ERR_INVALID_ARG (sizes, ids out of range), MZ_ERR_CYCLE, MZ_ERR_BAD_CHAINS,
 * MZ_ERR_OOM or MZ_ERR_CUDA (with opts->device_build also MZ_ERR_UNSUPPORTED or
 * MZ_ERR_TIMEOUT); nothing leaks on error.
 */
mz_status mz_build(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                   const int32_t *chain_id, const mz_build_opts *opts, mz_plan **out);

/*
 * mz_build_batch - one plan for `count` independent posets, so that one launch of each
 * kernel transforms all of them (many posets of uneven n and k). The plan is the
 * plan of their disjoint union: poset p's node x is node off_p + x of the union,
 * off_p = n[0] + ... + n[p-1], and every transform takes and returns [sum n][batch]
 * arrays in that order. The zeta and Moebius transforms of a disjoint union act on
 * each poset separately (no element of one is comparable with an element of another).
 *   count     number of posets, >= 1; the union may hold at most 2^30 nodes
 *   n, m      count sizes each; src[p], dst[p] the m[p] edges of poset p (local ids)
 *   chain_id  NULL, or count pointers, each NULL or n[p] chain ids of poset p
 *   opts, out as for mz_build
 * Errors as for mz_build; the message of mz_last_error names the failing poset.
 */
mz_status mz_build_batch(int32_t count, const int64_t *n, const int64_t *m, const int32_t *const *src,
                         const int32_t *const *dst, const int32_t *const *chain_id, const mz_build_opts *opts,
                         mz_plan **out);

/* Frees the plan and its device buffers (synchronises the device first). NULL is a no-op. */
void mz_destroy(mz_plan *plan);

/*
 * mz_workspace_size - bytes of device scratch every transform of this plan needs
 * for `dtype` and `batch` (transposes included). The workspace holds the chain
 * prefix array y' (Sec. 3, x' of Alg. 3 / y' of Alg. 4) and the scan's look-back state; it
 * needs 256-byte alignment and no initialisation.
 */
mz_status mz_workspace_size(const mz_plan *plan, mz_dtype dtype, int32_t batch, size_t *bytes);

/*
 * mz_zeta - g = Z f (Thm. 1 left). Two kernels: the per-chain prefix scan
 * c = V f (Eq. zeta_cache; decoupled look-back across tiles) and the gather
 * g(x) = sum_j c[niv_j(x)] (Eq. zeta-fast).
 *   f   device, [n][batch] input (F32C: 2 planes)
 *   g   device, [n][batch] output (F32C: 2 planes)
 *   ws  device workspace of ws_bytes >= mz_workspace_size(plan, dtype, batch)
 * Asynchronous on `stream`. batch >= 1.
 */
mz_status mz_zeta(const mz_plan *plan, mz_dtype dtype, const void *f, void *g, int32_t batch,
                  void *ws, size_t ws_bytes, mz_stream stream);

/*
 * mz_mobius - f = M g (Thm. 1 right) by the fast Moebius transform of Sec. 3:
 * forward substitution y'(x) = g(x) - sum_{j != id(x)} y'(niv_j(x)) (Alg. 4), then
 * f(x) = y'(x) - y'(next(x)) (V^-1). Arguments as for mz_zeta (g in, f out).
 * With MZ_SCHED_ULEVEL a persistent kernel substitutes, in the order of U's
 * dependency levels, only the rows some row of another chain reads; the remaining
 * rows (on the planted and random posets most of them) read only finished values
 * and are computed next by a gather over the zeta map, then V^-1 runs (4 launches).
 * MZ_SCHED_ANTICHAIN substitutes every row by antichain levels (Alg. 5) and writes
 * f directly (2 launches). MZ_F32C keeps y' in fp64 in the forward substitution; the
 * gather and V^-1 then run in compensated fp32 on double-word copies of y'. int64
 * results are exact modulo 2^64 for every input.
 */
mz_status mz_mobius(const mz_plan *plan, mz_dtype dtype, const void *g, void *f, int32_t batch,
                    void *ws, size_t ws_bytes, mz_stream stream);

/*
 * mz_zeta_noalloc - the same zeta transform as mz_zeta, for callers that cannot
 * allocate device memory at the time of the call: code running where cudaMalloc is
 * forbidden or unsafe (inside another allocator's callbacks, in a host-side
 * real-time loop that must not block on the driver's allocator, or under a memory
 * pool policy that reserves all device memory at start-up). The paper has no
 * counterpart; this is a service of the library.
 *
 * The scratch lives in a fixed array inside the library (MZ_NOALLOC_SCRATCH_BYTES,
 * 16 MiB), which every GPU that loads the library holds until the process exits.
 * The call allocates nothing: it needs no workspace argument, and the plan must
 * already exist (mz_build can route its own buffers through opts->dev_alloc).
 * The first call in each CUDA context looks up the array's device address
 * (cudaGetSymbolAddress) and caches it for that context, so make that first call
 * before any stream capture. A context that is destroyed and created again (for
 * example after cudaDeviceReset) is a new context: its first call looks the address
 * up again, and its array starts with undefined contents.
 *   f, g, batch, stream  as for mz_zeta
 * Returns MZ_ERR_INVALID_ARG when the transform needs more scratch than the fixed
 * array holds (the needed bytes are mz_workspace_size(plan, dtype, batch)), and the
 * errors of mz_zeta otherwise. All calls share the one array, which keeps the last
 * call's contents: calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it and give wrong results; order them on one stream or
 * synchronise between them.
 */
#define MZ_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
mz_status mz_zeta_noalloc(const mz_plan *plan, mz_dtype dtype, const void *f, void *g, int32_t batch,
                          mz_stream stream);

/* mz_zeta_T - r = Z^T h: r(y) = sum_{x : y <= x} h(x), the zeta transform of the dual
   poset. Needs a plan built with build_transpose, else MZ_ERR_UNSUPPORTED. */
mz_status mz_zeta_T(const mz_plan *plan, mz_dtype dtype, const void *h, void *r, int32_t batch,
                    void *ws, size_t ws_bytes, mz_stream stream);

/* mz_mobius_T - r = M^T h, the Moebius transform of the dual poset. As mz_zeta_T. */
mz_status mz_mobius_T(const mz_plan *plan, mz_dtype dtype, const void *h, void *r, int32_t batch,
                      void *ws, size_t ws_bytes, mz_stream stream);

/*
 * mz_check - synchronises `stream`, then returns and clears the plan's device-side
 * status word, which every transform of the plan sets when one of its bounded waits
 * runs out (MZ_OK or MZ_ERR_TIMEOUT, and MZ_ERR_BOUNDS in the MZ_DEBUG build; the word
 * is shared by all calls of the plan).
 * MZ_ERR_CUDA if the stream reports an error.
 */
mz_status mz_check(const mz_plan *plan, mz_stream stream);

/* Launch shapes a plan uses; mz_plan_tune changes them after the build (0 keeps a
   value). An autotuner times transforms under candidate shapes and keeps the best. */
typedef struct {
    int32_t mobius_blocks_per_sm; /* as mz_build_opts::mobius_blocks_per_sm (default 2) */
    int32_t mobius_pace_ns;       /* as mz_build_opts::mobius_pace_ns (default 600; < 0 = none) */
    int32_t gather_blocks_per_sm; /* resident 256-thread blocks per SM of the zeta gather (default 32) */
    int32_t mobius_lanes;         /* forward substitution of one function (batch 1): lanes sharing one
                                     row, a power of two up to 32 (default 32, or 1 when no row has
                                     more than 16 entries on other chains). The row's entries are
                                     dealt to the lanes 16 at a time, each lane polls and sums its
                                     own, the lanes' sums meet in a shuffle tree and the row's first
                                     lane publishes it; 0 keeps the current value */
} mz_tuning;

/* Sets the plan's launch shapes (results are unaffected); fills *current if non-NULL. */
mz_status mz_plan_tune(mz_plan *plan, const mz_tuning *set, mz_tuning *current);

/* Fills *info (host data only). */
mz_status mz_plan_info(const mz_plan *plan, mz_plan_info_t *info);

/* Copies one host-side array of the plan (mz_export) into `out` (`bytes` long).
   `dual` nonzero selects the dual plan. MZ_ERR_INVALID_ARG if `bytes` is too small.
   Plans of several posets export per-node arrays in union order (chain ids and topo
   entries offset to the union); their niv map is not exported (MZ_ERR_UNSUPPORTED). */
mz_status mz_plan_export(const mz_plan *plan, int32_t what, int32_t dual, void *out, size_t bytes);

/*
 * mz_plan_save - writes the plan's one-time precomputation (for every poset and the
 * dual: order, chains, slot layout, niv map, heights and U levels) to the file `path`,
 * so that mz_plan_load can rebuild the plan without computing it again. The format
 * is this library's (magic, version, checksum; the byte order and type sizes of the
 * writing machine). A plan whose niv map was built with device_build keeps the map
 * only on the device: MZ_ERR_UNSUPPORTED (build it with device_build = 0 to save it).
 * MZ_ERR_INVALID_ARG if the file cannot be written.
 */
mz_status mz_plan_save(const mz_plan *plan, const char *path);

/*
 * mz_plan_load - a plan from a file written by mz_plan_save. From `opts` (NULL: the
 * defaults) it takes what concerns the device part: host_only, mobius_schedule,
 * mobius_blocks_per_sm, mobius_pace_ns, spin_limit, debug_withhold and the allocator
 * callbacks; build_transpose, niv_format and device_build are the saved plan's. The
 * file is checked before anything is uploaded (magic, version, checksum, every array
 * length and every index against its range): MZ_ERR_INVALID_ARG names what failed, and
 * no file can make a kernel read outside an array. MZ_ERR_OOM, MZ_ERR_CUDA as mz_build;
 * *out is NULL on any error.
 */
mz_status mz_plan_load(const char *path, const mz_build_opts *opts, mz_plan **out);

/* Kernel launches issued by the last transform call on this thread (memsets excluded). */
int32_t mz_last_launch_count(void);

/*
 * Profiling hook. While `events` is non-NULL, every transform call on this thread
 * records events[0] on its stream before its first device operation and events[i]
 * right after its i-th kernel launch (i = 1 .. launches), skipping indices at or
 * beyond `capacity`. The events are the caller's cudaEvent_t handles (created with
 * timing enabled); the library never creates, waits on or destroys them. NULL (or
 * capacity 0) turns the hook off. Timing only: results are unaffected.
 */
void mz_set_launch_events(void *const *events, int32_t capacity);

/* Static text for a status code. */
const char *mz_status_string(mz_status s);

/* Detail of the last error on this thread (empty string if none). */
const char *mz_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MZ_H */
