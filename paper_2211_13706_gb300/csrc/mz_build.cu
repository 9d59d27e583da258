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
    const int32_t k = a.k;
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
        const int32_t cx = a.chain_id[x], sx = a.node_slot[x];
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
                rz = (int64_t)a.node_slot[z] - a.chain_id[z] - 1;
                ok = wait_ready(&a.ready[z], a.status, a.spin_limit);
            }
            // after a failed wait the rows are not read (the build reports the timeout)
            if (!__all_sync(kFull, ok)) break;
            __syncwarp();   // orders every lane's acquire before every lane's row loads
            const int cnt = e1 - e < 32 ? (int)(e1 - e) : 32;
#pragma unroll 2
            for (int q = 0; q < cnt; ++q) {
                const int32_t *row = a.N + __shfl_sync(kFull, rz, q) * k;
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
        const int64_t r = (int64_t)sx - cx - 1;
        int32_t *out = a.N + r * k;
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

// One warp per row of the schedule. An entry's place is its rank under the order
// (key, chain), the key being the level of the element in its slot; the host build
// sorts by key stably over ascending chains, which is the same order.
template <int KJ>
__global__ void __launch_bounds__(kBuildThreads) k_build_mob_rows(BuildMobArgs a) {
    __shared__ int32_t s_key[kBuildThreads / 32][32 * KJ];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t k = a.k;
    const int64_t nwarps = (int64_t)gridDim.x * (kBuildThreads / 32);
    for (int64_t i = (int64_t)blockIdx.x * (kBuildThreads / 32) + w; i < a.n; i += nwarps) {
        const int64_t r = a.mrow[i];
        const int32_t sx = a.mslot[i];
        int32_t slot[KJ], key[KJ];
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < KJ; ++j) {
            const int c = lane + 32 * j;
            slot[j] = c < k ? a.N[r * k + c] : sx;
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

cudaError_t launch_build_tiles(const int32_t *N, int64_t n, int32_t k, int32_t *Nt, int num_sms, cudaStream_t st) {
    const int64_t ntiles = (n + 31) / 32;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)num_sms * 8));
    k_build_tiles<<<(unsigned)blocks, kBuildThreads, 0, st>>>(N, n, k, ntiles, Nt);
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

}  // namespace mz
