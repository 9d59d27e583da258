// Device build of a plan's niv map and of the layouts derived from it (sm_103a).
//
//   k_build_niv       the recurrence of Thm. 4 (Alg. 2): niv_j(x) is the largest
//                     niv_j(z) over the children z of x, except on x's own chain,
//                     where it is x itself. One warp per node, k entries per row
//                     spread over the lanes. Nodes are claimed in a bottom-up order
//                     (by height) from a global ticket; a node waits, with bounded
//                     polls, until its children have published their rows. The same
//                     warp checks the chain (the element below x on its chain must be
//                     the largest element of that chain reachable through a child),
//                     counts the row's finite entries and computes x's level in U's
//                     dependency graph: one more than the largest level among the
//                     other chains' entries.
//   k_build_tiles     the row-major map into tiles of 32 rows, column-major inside a
//                     tile, the layout k_niv_gather streams.
//   k_build_mob_rows  the rows of the Moebius schedule: each row's finite entries of
//                     the other chains, ordered by (level of the element in the slot,
//                     chain), packed at the end of the row's padded extent.
//
// Every entry is an integer decided by comparisons only, so the map equals the host
// build's entry for entry.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <type_traits>

#include "mz_kernels.h"

namespace mz {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBuildThreads = 256;

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Waits until *flag != 0 with at most `limit` polls, sleeping longer between polls
// the longer it waits (up to 2 us), so that warps far ahead of the frontier do not
// load L2. Returns false after a timeout, or early once another wait has failed.
__device__ bool wait_ready(const uint32_t *flag, uint32_t *status, int64_t limit) {
    unsigned sleep = 32;
    for (int64_t it = 0;; ++it) {
        if (ld_acquire(flag)) return true;
        if ((it & 63) == 63 && ld_relaxed(status)) return false;
        if (it >= limit) {
            atomicCAS(status, 0u, (uint32_t)MZ_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(sleep);
        if (sleep < 2048) sleep *= 2;
    }
}

template <int KJ>
__global__ void __launch_bounds__(kBuildThreads) k_build_niv(BuildNivArgs a) {
    const int lane = threadIdx.x & 31;
    int32_t k = a.k;
    int32_t base[KJ];
#pragma unroll
    for (int j = 0; j < KJ; ++j) {
        const int c = lane + 32 * j;
        base[j] = c < k ? a.base[c] : 0;
    }
    unsigned long long my_nnz = 0;
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(a.ticket, 1u);
        t = __shfl_sync(kFull, t, 0);
        if ((int64_t)t >= a.n) break;
        const int32_t x = a.order[t];
        int32_t cx = a.chain_id[x];
        const int32_t sx = a.node_slot[x];
        // the map of x's poset: rows of width k from N + moff on (row roff first)
        int64_t roff = 0, moff = 0;
        if (a.comp) {
            const int32_t c = a.comp[x];
            const int32_t koff = a.comp_koff[c];
            k = a.comp_k[c];
            roff = a.comp_roff[c];
            moff = a.comp_moff[c];
            cx -= koff;   // x's chain within its poset
#pragma unroll
            for (int j = 0; j < KJ; ++j) {
                const int q = lane + 32 * j;
                base[j] = q < k ? a.base[koff + q] : 0;
            }
        }
        int32_t cur[KJ];
#pragma unroll
        for (int j = 0; j < KJ; ++j) cur[j] = base[j];
        const int64_t e0 = a.ptr[x], e1 = a.ptr[x + 1];
        for (int64_t e = e0; e < e1; e += 32) {
            // up to 32 children at once: lane q waits for child q and finds its row
            int64_t rz = 0;
            bool ok = true;
            if (e + lane < e1) {
                const int32_t z = a.adj[e + lane];
                rz = (int64_t)a.node_slot[z] - a.chain_id[z] - 1;   // over the union: the poset's rows are contiguous
                ok = wait_ready(&a.ready[z], a.status, a.spin_limit);
            }
            // after a failed wait the rows are not read (the build reports the timeout)
            if (!__all_sync(kFull, ok)) break;
            __syncwarp();   // orders every lane's acquire before every lane's row loads
            const int cnt = e1 - e < 32 ? (int)(e1 - e) : 32;
#pragma unroll 2
            for (int q = 0; q < cnt; ++q) {
                const int32_t *row = a.N + moff + (__shfl_sync(kFull, rz, q) - roff) * k;
#pragma unroll
                for (int j = 0; j < KJ; ++j) {
                    const int c = lane + 32 * j;
                    if (c < k) cur[j] = max(cur[j], __ldcg(row + c));
                }
            }
        }
        // the own chain: the children must reach exactly the element below x on it
        bool bad = false;
#pragma unroll
        for (int j = 0; j < KJ; ++j)
            if (lane + 32 * j == cx) {
                bad = cur[j] != sx - 1;
                cur[j] = sx;
            }
        if (bad) atomicMax(a.bad, a.topo_pos[x]);
        // level in U's dependency graph; zero slots hold -1 and add nothing
        int32_t u = 0, finite = 0;
#pragma unroll
        for (int j = 0; j < KJ; ++j) {
            const int c = lane + 32 * j;
            if (c < k) {
                finite += cur[j] != base[j];
                if (c != cx) u = max(u, __ldcg(a.uslot + cur[j]) + 1);
            }
        }
        u = __reduce_max_sync(kFull, u);
        finite = __reduce_add_sync(kFull, finite);
        const int64_t r = (int64_t)sx - a.chain_id[x] - 1;   // row over the union
        int32_t *out = a.N + moff + (r - roff) * k;
#pragma unroll
        for (int j = 0; j < KJ; ++j) {
            const int c = lane + 32 * j;
            if (c < k) out[c] = cur[j];
        }
        if (lane == 0) {
            a.uslot[sx] = u;
            a.rowcnt[r] = finite;
            my_nnz += (unsigned long long)finite;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(&a.ready[x], 1u);
    }
    if (lane == 0 && my_nnz) atomicAdd(a.nnz, my_nnz);
}

// One 32 x 32 block of the map at a time through shared memory; rows past n are 0
// (slot 0, a zero slot), as the gather's padding rows expect.
__global__ void __launch_bounds__(kBuildThreads) k_build_tiles(const int32_t *N, int64_t n, int32_t k,
                                                              int64_t ntiles, int32_t *Nt) {
    __shared__ int32_t s[32][33];
    const int tx = threadIdx.x & 31, ty0 = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        for (int32_t q0 = 0; q0 < k; q0 += 32) {
            for (int ty = ty0; ty < 32; ty += kBuildThreads / 32) {
                const int64_t r = t * 32 + ty;
                const int32_t q = q0 + tx;
                s[ty][tx] = (r < n && q < k) ? N[r * k + q] : 0;
            }
            __syncthreads();
            for (int ty = ty0; ty < 32; ty += kBuildThreads / 32) {
                const int32_t q = q0 + ty;
                if (q < k) Nt[t * (int64_t)k * 32 + (int64_t)q * 32 + tx] = s[tx][ty];
            }
            __syncthreads();
        }
    }
}

// The same transpose for plans of several posets: per tile its rows' start in N, width
// and number of rows.
__global__ void __launch_bounds__(kBuildThreads) k_build_tiles_var(const int32_t *N, int64_t ntiles,
                                                                  const int64_t *tile_moff, const int32_t *tile_k,
                                                                  const int32_t *tile_rows, const int64_t *tile_off,
                                                                  int32_t *Nt) {
    __shared__ int32_t s[32][33];
    const int tx = threadIdx.x & 31, ty0 = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int32_t k = tile_k[t], rows = tile_rows[t];
        const int32_t *src = N + tile_moff[t];
        int32_t *dst = Nt + tile_off[t];
        for (int32_t q0 = 0; q0 < k; q0 += 32) {
            for (int ty = ty0; ty < 32; ty += kBuildThreads / 32) {
                const int32_t q = q0 + tx;
                s[ty][tx] = (ty < rows && q < k) ? src[(int64_t)ty * k + q] : 0;
            }
            __syncthreads();
            for (int ty = ty0; ty < 32; ty += kBuildThreads / 32) {
                const int32_t q = q0 + ty;
                if (q < k) dst[(int64_t)q * 32 + tx] = s[tx][ty];
            }
            __syncthreads();
        }
    }
}

// One warp per row of the schedule. An entry's place is its rank under the order
// (key, chain), the key being the level of the element in its slot; the host build
// sorts by key stably over ascending chains, which is the same order.
template <int KJ>
__global__ void __launch_bounds__(kBuildThreads) k_build_mob_rows(BuildMobArgs a) {
    __shared__ int32_t s_key[kBuildThreads / 32][32 * KJ];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * (kBuildThreads / 32);
    for (int64_t i = (int64_t)blockIdx.x * (kBuildThreads / 32) + w; i < a.n; i += nwarps) {
        const int32_t k = a.row_k ? a.row_k[i] : a.k;
        const int32_t *rowp = a.row_moff ? a.N + a.row_moff[i] : a.N + (int64_t)a.mrow[i] * k;
        const int32_t sx = a.mslot[i];
        int32_t slot[KJ], key[KJ];
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < KJ; ++j) {
            const int c = lane + 32 * j;
            slot[j] = c < k ? rowp[c] : sx;
            key[j] = INT_MAX;
            if (c < k && slot[j] != sx) {
                const int32_t kv = a.key_slot[slot[j]];
                if (kv >= 0) {
                    key[j] = kv;
                    ++cnt;
                }
            }
            s_key[w][c] = key[j];
        }
        cnt = __reduce_add_sync(kFull, cnt);
        __syncwarp();
        if (cnt > a.mkp[i]) continue;   // cannot happen for a map built by k_build_niv; keeps writes in the row
        int32_t rank[KJ];
#pragma unroll
        for (int j = 0; j < KJ; ++j) rank[j] = 0;
        for (int c2 = 0; c2 < k; ++c2) {
            const int32_t kv = s_key[w][c2];
#pragma unroll
            for (int j = 0; j < KJ; ++j) rank[j] += (kv < key[j]) | ((kv == key[j]) & (c2 < lane + 32 * j));
        }
        int32_t *dst = a.Nm + a.moff[i] + a.mkp[i] - cnt;
#pragma unroll
        for (int j = 0; j < KJ; ++j)
            if (key[j] != INT_MAX) dst[rank[j]] = slot[j];
        __syncwarp();   // s_key is rewritten by the next row
    }
}

// ---------------------------------------------------------------- sparse map (k > 512)
// The same recurrence on rows that hold only their finite entries, as ascending slot
// lists (slots are numbered chain after chain, so slot order is chain order). One height
// level per launch: every child of a node sits on a lower level, so a kernel boundary
// separates a row from the rows it reads and there are no waits at all.

// Ascending bitonic sort of p keys (p a power of two) by the calling warp, in global memory.
__device__ void warp_bitonic_sort(unsigned long long *v, int64_t p) {
    const int lane = threadIdx.x & 31;
    for (int64_t kk = 2; kk <= p; kk <<= 1) {
        for (int64_t j = kk >> 1; j > 0; j >>= 1) {
            for (int64_t i = lane; i < p; i += 32) {
                const int64_t l = i ^ j;
                if (l > i) {
                    const unsigned long long x = v[i], y = v[l];
                    if ((x > y) == ((i & kk) == 0)) {
                        v[i] = y;
                        v[l] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
}

__device__ __forceinline__ int64_t row_of(const SparseLevelArgs &a, int32_t z) {
    return (int64_t)a.node_slot[z] - a.chain_id[z] - 1;
}

// Candidate-list sizes of the level's nodes: the children's rows plus the own entry,
// rounded up to a power of two for the sort. cand_off[1 + i] = size of node lo + i.
__global__ void __launch_bounds__(kBuildThreads) k_sparse_bounds(SparseLevelArgs a) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = a.order[a.lo + i];
        int64_t b = 1;
        for (int64_t e = a.ptr[x]; e < a.ptr[x + 1]; ++e) b += a.row_len[row_of(a, a.adj[e])];
        int64_t p = 1;
        while (p < b) p <<= 1;
        a.cand_off[1 + i] = p;
        if (i == 0) a.cand_off[0] = 0;
    }
}

// In-place inclusive scan of v[1 .. count] by one block (v[0] stays as it is).
__global__ void __launch_bounds__(1024) k_scan_i64(int64_t *v, int64_t count) {
    __shared__ int64_t s[1024];
    const int t = threadIdx.x;
    const int64_t per = (count + 1023) / 1024;
    const int64_t b = 1 + (int64_t)t * per, e = min(count + 1, b + per);
    int64_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += v[i];
    s[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int64_t add = t >= off ? s[t - off] : 0;
        __syncthreads();
        s[t] += add;
        __syncthreads();
    }
    int64_t run = t ? s[t - 1] : 0;
    for (int64_t i = b; i < e; ++i) {
        run += v[i];
        v[i] = run;
    }
}

// One warp per node of the level: gather the children's entries and the own one, sort
// them by slot, keep the last (largest) slot of every chain's run, append the row to the
// pool. The chain check, the U level and the row's length come out of the same passes.
__global__ void __launch_bounds__(kBuildThreads) k_sparse_merge(SparseLevelArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (kBuildThreads / 32);
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < a.cnt; i += nwarps) {
        const int32_t x = a.order[a.lo + i];
        const int32_t cx = a.chain_id[x], sx = a.node_slot[x];
        const int64_t r = (int64_t)sx - cx - 1;
        const int64_t off = a.cand_off[i], p = a.cand_off[i + 1] - off;
        unsigned long long *v = a.cand + off;
        int64_t L = 0;
        int32_t m = a.base[cx];   // largest slot of x's own chain the children reach
        for (int64_t e = a.ptr[x]; e < a.ptr[x + 1]; ++e) {
            const int64_t rz = row_of(a, a.adj[e]);
            const int64_t b = a.row_beg[rz];
            const int32_t len = a.row_len[rz];
            if (L + len + 1 > p) break;   // cannot happen: p covers every child's row
            for (int32_t q = lane; q < len; q += 32) {
                const int32_t s2 = a.pool[b + q];
                v[L + q] = (unsigned long long)(uint32_t)s2;
                if (a.slot_chain[s2] == cx) m = max(m, s2);
            }
            L += len;
        }
        if (lane == 0) v[L] = (unsigned long long)(uint32_t)sx;
        ++L;
        for (int64_t q = L + lane; q < p; q += 32) v[q] = ~0ull;
        m = __reduce_max_sync(kFull, m);
        if (lane == 0 && m != sx - 1) atomicMax(a.bad, a.topo_pos[x]);
        __syncwarp();
        warp_bitonic_sort(v, p);
        // pass 1: count the kept entries, U level over the other chains
        int32_t nk = 0, u = 0;
        for (int64_t q0 = 0; q0 < L; q0 += 32) {
            const int64_t q = q0 + lane;
            bool keep = false;
            if (q < L) {
                const int32_t s2 = (int32_t)v[q];
                const int32_t c = a.slot_chain[s2];
                keep = q == L - 1 || a.slot_chain[(int32_t)v[q + 1]] != c;
                if (keep && c != cx) u = max(u, a.uslot[s2] + 1);
            }
            nk += __popc(__ballot_sync(kFull, keep));
        }
        u = __reduce_max_sync(kFull, u);
        unsigned long long beg = 0;
        if (lane == 0) beg = atomicAdd(a.pool_top, (unsigned long long)nk);
        beg = __shfl_sync(kFull, beg, 0);
        if ((int64_t)(beg + nk) > a.pool_cap) {   // cannot happen: the host sized the pool
            if (lane == 0) atomicCAS(a.status, 0u, (uint32_t)MZ_ERR_OOM);
            continue;
        }
        // pass 2: write the kept entries in slot order
        int32_t run = 0;
        for (int64_t q0 = 0; q0 < L; q0 += 32) {
            const int64_t q = q0 + lane;
            bool keep = false;
            int32_t s2 = 0;
            if (q < L) {
                s2 = (int32_t)v[q];
                keep = q == L - 1 || a.slot_chain[(int32_t)v[q + 1]] != a.slot_chain[s2];
            }
            const unsigned mask = __ballot_sync(kFull, keep);
            if (keep) a.pool[beg + run + __popc(mask & lt)] = s2;
            run += __popc(mask);
        }
        if (lane == 0) {
            a.row_beg[r] = (int64_t)beg;
            a.row_len[r] = nk;
            a.uslot[sx] = u;
        }
    }
}

// Sparse tiles: one warp per tile of 32 positions, lane = position, order[position] =
// its row; entries in slot order, then 0 (slot 0, a zero slot) up to the tile's width.
__global__ void __launch_bounds__(kBuildThreads) k_build_tiles_sparse(const int64_t *row_beg, const int32_t *row_len,
                                                                     const int32_t *pool, const int32_t *order,
                                                                     int64_t n, int64_t ntiles,
                                                                     const int64_t *tile_off, const int32_t *tile_k,
                                                                     int32_t *Nt) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (kBuildThreads / 32);
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntiles; t += nwarps) {
        const int64_t q = t * 32 + lane;
        const int64_t r = q < n ? order[q] : 0;
        const int64_t b = q < n ? row_beg[r] : 0;
        const int32_t len = q < n ? row_len[r] : 0;
        int32_t *dst = Nt + tile_off[t] + lane;
        for (int32_t q = 0; q < tile_k[t]; ++q) dst[(int64_t)q * 32] = q < len ? pool[b + q] : 0;
    }
}

// Moebius rows from sparse rows: one warp per row of the schedule; entries ranked by
// (key of the element in the slot, slot), the other chains only. Keys go through
// shared memory 256 at a time, so rows of any length work.
constexpr int kRankTile = 256;
__global__ void __launch_bounds__(kBuildThreads) k_build_mob_rows_sparse(BuildMobSparseArgs a) {
    __shared__ unsigned long long s_key[kBuildThreads / 32][kRankTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * (kBuildThreads / 32);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < a.n; i += nwarps) {
        const int64_t r = a.mrow[i];
        const int32_t sx = a.mslot[i];
        const int64_t b = a.row_beg[r];
        const int32_t len = a.row_len[r];
        const int32_t cnt = len - 1;   // the own chain's entry is left out
        if (cnt > a.mkp[i] || cnt < 0) continue;   // cannot happen for rows built by k_sparse_merge
        int32_t *dst = a.Nm + a.moff[i] + a.mkp[i] - cnt;
        for (int32_t q0 = 0; q0 < len; q0 += 32) {
            const int32_t q = q0 + lane;
            unsigned long long key = ~0ull;
            int32_t s2 = sx;
            if (q < len) {
                s2 = a.pool[b + q];
                if (s2 != sx) key = ((unsigned long long)(uint32_t)a.key_slot[s2] << 32) | (uint32_t)s2;
            }
            int32_t rank = 0;
            for (int32_t t0 = 0; t0 < len; t0 += kRankTile) {
                __syncwarp();
                for (int32_t t = lane; t < kRankTile && t0 + t < len; t += 32) {
                    const int32_t s3 = a.pool[b + t0 + t];
                    s_key[w][t] = s3 == sx ? ~0ull : ((unsigned long long)(uint32_t)a.key_slot[s3] << 32) | (uint32_t)s3;
                }
                __syncwarp();
                const int32_t tn = min(kRankTile, len - t0);
                for (int32_t t = 0; t < tn; ++t) rank += s_key[w][t] < key;
            }
            if (key != ~0ull) dst[rank] = s2;
        }
    }
}

int kj_for(int32_t k) {
    int kj = 1;
    while (32 * kj < k) kj *= 2;
    return kj;
}

template <class F>
cudaError_t dispatch_kj(int32_t k, F f) {
    switch (kj_for(k)) {
        case 1: return f(std::integral_constant<int, 1>());
        case 2: return f(std::integral_constant<int, 2>());
        case 4: return f(std::integral_constant<int, 4>());
        case 8: return f(std::integral_constant<int, 8>());
        case 16: return f(std::integral_constant<int, 16>());
        default: return cudaErrorInvalidValue;
    }
}

// ---- Alg. 1 on the device: a maximum matching between the edge sources ("upper" copies)
// and edge targets ("lower" copies) of the nodes, for a minimum path cover. A greedy
// maximal matching first, then phases of augmenting paths: a breadth-first search over
// alternating paths from every free upper node at once (one launch per level; each lower
// node is claimed by one search tree, and each tree augments along the first free lower
// node it reaches), then every found path is flipped. A phase that finds no path ends it:
// the trees then covered every alternating path from a free upper node (Berge's theorem).
// match_u[u] = lower node matched to u (-1 free), match_v[v] = upper node matched to v.

// Each free upper node takes its first free child, if it wins the claim.
__global__ void __launch_bounds__(kBuildThreads) k_match_greedy(const int64_t *ptr, const int32_t *adj, int64_t n,
                                                                int32_t *match_u, int32_t *match_v,
                                                                uint32_t *changed) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        if (match_u[u] >= 0) continue;
        for (int64_t e = ptr[u]; e < ptr[u + 1]; ++e) {
            const int32_t v = adj[e];
            if (match_v[v] < 0 && atomicCAS(&match_v[v], -1, (int32_t)u) == -1) {
                match_u[u] = v;
                *changed = 1u;
                break;
            }
        }
    }
}

// The roots of a phase: every free upper node with a child.
__global__ void __launch_bounds__(kBuildThreads) k_match_roots(const int64_t *ptr, int64_t n, const int32_t *match_u,
                                                               int32_t *root, int32_t *frontier,
                                                               unsigned long long *count) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        if (match_u[u] < 0 && ptr[u + 1] > ptr[u]) {
            root[u] = (int32_t)u;
            frontier[atomicAdd(count, 1ull)] = (int32_t)u;
        }
}

// One level: each upper node of the frontier tries its children over unmatched edges. A
// child claimed first here (parent_v) is either free (the tree's path ends there, once per
// tree) or leads on to its mate, which joins the next frontier in the same tree.
__global__ void __launch_bounds__(kBuildThreads) k_match_expand(const int64_t *ptr, const int32_t *adj,
                                                                const int32_t *frontier, int64_t fcount,
                                                                int32_t *next, unsigned long long *ncount,
                                                                const int32_t *match_u, const int32_t *match_v,
                                                                int32_t *parent_v, int32_t *root,
                                                                uint32_t *root_done, int32_t *ends,
                                                                unsigned long long *ecount) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < fcount; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = frontier[i];
        const int32_t r = root[u];
        if (ld_relaxed(&root_done[r])) continue;
        for (int64_t e = ptr[u]; e < ptr[u + 1]; ++e) {
            const int32_t v = adj[e];
            if (v == match_u[u]) continue;
            if (atomicCAS(&parent_v[v], -1, u) != -1) continue;
            const int32_t w = match_v[v];
            if (w < 0) {
                if (atomicCAS(&root_done[r], 0u, 1u) == 0u) ends[atomicAdd(ecount, 1ull)] = v;
                break;
            }
            root[w] = r;
            next[atomicAdd(ncount, 1ull)] = w;
        }
    }
}

// Flips each found path, from its free lower end up to its root: every upper node on it
// takes the lower node below it on the path. The paths share no node. A walk longer than
// n steps (impossible for a path of a tree) stops and reports MZ_ERR_TIMEOUT.
__global__ void __launch_bounds__(kBuildThreads) k_match_augment(const int32_t *ends, int64_t ecount, int64_t n,
                                                                 const int32_t *parent_v, int32_t *match_u,
                                                                 int32_t *match_v, uint32_t *status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ecount; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = ends[i];
        for (int64_t step = 0;; ++step) {
            if (step > n) {
                atomicCAS(status, 0u, (uint32_t)MZ_ERR_TIMEOUT);
                break;
            }
            const int32_t u = parent_v[v];
            const int32_t prev = match_u[u];
            match_u[u] = v;
            match_v[v] = u;
            if (prev < 0) break;   // u is the root
            v = prev;
        }
    }
}

}  // namespace

cudaError_t launch_build_niv(const BuildNivArgs &a, int num_sms, cudaStream_t st) {
    return dispatch_kj(a.k, [&](auto kj) {
        constexpr int KJ = decltype(kj)::value;
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_niv<KJ>, kBuildThreads, 0);
        if (e != cudaSuccess) return e;
        // Claimed nodes are always running, so any grid size is safe; 4 blocks per SM
        // keep enough nodes in flight without flooding L2 with polls.
        const int64_t blocks = (int64_t)std::max(1, std::min(per_sm, 4)) * num_sms;
        k_build_niv<KJ><<<(unsigned)blocks, kBuildThreads, 0, st>>>(a);
        return cudaGetLastError();
    });
}

cudaError_t launch_build_tiles_var(const int32_t *N, int64_t ntiles, const int64_t *tile_moff, const int32_t *tile_k,
                                   const int32_t *tile_rows, const int64_t *tile_off, int32_t *Nt, int num_sms,
                                   cudaStream_t st) {
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)num_sms * 8));
    k_build_tiles_var<<<(unsigned)blocks, kBuildThreads, 0, st>>>(N, ntiles, tile_moff, tile_k, tile_rows, tile_off, Nt);
    return cudaGetLastError();
}

cudaError_t launch_build_tiles(const int32_t *N, int64_t n, int32_t k, int32_t *Nt, int num_sms, cudaStream_t st) {
    const int64_t ntiles = (n + 31) / 32;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)num_sms * 8));
    k_build_tiles<<<(unsigned)blocks, kBuildThreads, 0, st>>>(N, n, k, ntiles, Nt);
    return cudaGetLastError();
}

// Blocks of one thread per item, at most 16 resident blocks per SM (grid-stride loops).
static int64_t grid_for(int64_t items, int num_sms) {
    return std::max<int64_t>(1, std::min<int64_t>((items + kBuildThreads - 1) / kBuildThreads, (int64_t)num_sms * 16));
}

static int64_t warp_blocks(int64_t items, int num_sms) {
    return std::max<int64_t>(1, std::min<int64_t>((items + kBuildThreads / 32 - 1) / (kBuildThreads / 32),
                                                  (int64_t)num_sms * 8));
}

cudaError_t launch_sparse_bounds(const SparseLevelArgs &a, int num_sms, cudaStream_t st) {
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((a.cnt + kBuildThreads - 1) / kBuildThreads,
                                                                  (int64_t)num_sms * 8));
    k_sparse_bounds<<<(unsigned)blocks, kBuildThreads, 0, st>>>(a);
    if (cudaError_t e = cudaGetLastError()) return e;
    k_scan_i64<<<1, 1024, 0, st>>>(a.cand_off, a.cnt);
    return cudaGetLastError();
}

cudaError_t launch_sparse_merge(const SparseLevelArgs &a, int num_sms, cudaStream_t st) {
    k_sparse_merge<<<(unsigned)warp_blocks(a.cnt, num_sms), kBuildThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_build_tiles_sparse(const int64_t *row_beg, const int32_t *row_len, const int32_t *pool,
                                      const int32_t *order, int64_t n, int64_t ntiles, const int64_t *tile_off,
                                      const int32_t *tile_k, int32_t *Nt, int num_sms, cudaStream_t st) {
    k_build_tiles_sparse<<<(unsigned)warp_blocks(ntiles, num_sms), kBuildThreads, 0, st>>>(
        row_beg, row_len, pool, order, n, ntiles, tile_off, tile_k, Nt);
    return cudaGetLastError();
}

cudaError_t launch_build_mob_rows_sparse(const BuildMobSparseArgs &a, int num_sms, cudaStream_t st) {
    k_build_mob_rows_sparse<<<(unsigned)warp_blocks(a.n, num_sms), kBuildThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_build_mob_rows(const BuildMobArgs &a, int num_sms, cudaStream_t st) {
    return dispatch_kj(a.k, [&](auto kj) {
        constexpr int KJ = decltype(kj)::value;
        const int64_t blocks =
            std::max<int64_t>(1, std::min<int64_t>((a.n + kBuildThreads / 32 - 1) / (kBuildThreads / 32),
                                                   (int64_t)num_sms * 8));
        k_build_mob_rows<KJ><<<(unsigned)blocks, kBuildThreads, 0, st>>>(a);
        return cudaGetLastError();
    });
}

cudaError_t launch_match_greedy(const int64_t *ptr, const int32_t *adj, int64_t n, int32_t *match_u,
                                int32_t *match_v, uint32_t *changed, int num_sms, cudaStream_t st) {
    k_match_greedy<<<(unsigned)grid_for(n, num_sms), kBuildThreads, 0, st>>>(ptr, adj, n, match_u, match_v, changed);
    return cudaGetLastError();
}

cudaError_t launch_match_roots(const int64_t *ptr, int64_t n, const int32_t *match_u, int32_t *root,
                               int32_t *frontier, unsigned long long *count, int num_sms, cudaStream_t st) {
    k_match_roots<<<(unsigned)grid_for(n, num_sms), kBuildThreads, 0, st>>>(ptr, n, match_u, root, frontier, count);
    return cudaGetLastError();
}

cudaError_t launch_match_expand(const int64_t *ptr, const int32_t *adj, const int32_t *frontier, int64_t fcount,
                                int32_t *next, unsigned long long *ncount, const int32_t *match_u,
                                const int32_t *match_v, int32_t *parent_v, int32_t *root, uint32_t *root_done,
                                int32_t *ends, unsigned long long *ecount, int num_sms, cudaStream_t st) {
    k_match_expand<<<(unsigned)grid_for(fcount, num_sms), kBuildThreads, 0, st>>>(
        ptr, adj, frontier, fcount, next, ncount, match_u, match_v, parent_v, root, root_done, ends, ecount);
    return cudaGetLastError();
}

cudaError_t launch_match_augment(const int32_t *ends, int64_t ecount, int64_t n, const int32_t *parent_v,
                                 int32_t *match_u, int32_t *match_v, uint32_t *status, int num_sms,
                                 cudaStream_t st) {
    k_match_augment<<<(unsigned)grid_for(ecount, num_sms), kBuildThreads, 0, st>>>(ends, ecount, n, parent_v,
                                                                                    match_u, match_v, status);
    return cudaGetLastError();
}

}  // namespace mz
