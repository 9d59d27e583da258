// CUDA kernels of the transforms (sm_103a) and their launchers.
//
//   k_chain_scan   c = V f, the per-chain prefix sums of Eq. (zeta_cache), as one
//                  segmented inclusive scan over the slot array with a zero slot
//                  in front of every chain; single pass, decoupled look-back
//                  between tiles (Merrill & Garland, "Single-pass parallel prefix
//                  scan with decoupled look-back", 2016).
//   k_niv_gather   g(x) = sum_j c[niv_j(x)], Eq. (zeta-fast) = U c. One warp per
//                  tile of 32 consecutive rows (one row per lane), the tiled map
//                  streamed with coalesced loads, each group of 8 entries requested
//                  while the previous group's values are gathered; along a chain
//                  niv_j is monotone, so a warp's 32 gathers of one column hit a
//                  narrow window of c.
//   k_mob_init     fills y' with the "not ready" sentinel (0 at zero slots).
//   k_mob_wave     forward substitution of Alg. 4, U y' = g:
//                  y'(x) = g(x) - sum_{j != id(x)} y'(niv_j(x)),
//                  persistent (cooperative launch), one warp per row in the
//                  schedule's order; every read of y' polls until the word is
//                  no longer the sentinel, with a bounded number of polls.
//                  Antichain schedule (Alg. 5/6): f(x) = g(x) - sum_j y'[niv^-_j(x)]
//                  and y'(x) = y'(next(x)) + f(x) (Sec. 3, V^-1 folded in).
//   k_mob_diff     f(x) = y'(x) - y'(next(x)): V^-1 (Sec. 3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "mz_arith.cuh"
#include "mz_kernels.h"

namespace mz {

// ---------------------------------------------------------------- memory-model helpers
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_u8(unsigned char *p, unsigned short v) {
    asm volatile("st.relaxed.gpu.global.u8 [%0], %1;" ::"l"(p), "h"(v) : "memory");
}
__device__ __forceinline__ unsigned short ld_relaxed_u8(const unsigned char *p) {
    unsigned short v;
    asm volatile("ld.relaxed.gpu.global.u8 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void report(uint32_t *status, uint32_t code) { atomicCAS(status, 0u, code); }

// Double-word copies of y' (F32C): word i = s * B + b as one float2, or, in column pairs
// (pair: B even), hi at float 2 (i - (i & 1)) + (i & 1) and lo two floats further.
__device__ __forceinline__ void dwq_store(float2 *Q, int64_t i, bool pair, float2 v) {
    if (pair) {
        float *q = reinterpret_cast<float *>(Q) + 2 * (i & ~1ll) + (i & 1);
        q[0] = v.x;
        q[2] = v.y;
    } else {
        Q[i] = v;
    }
}
// MZ_DEBUG builds check every index a kernel takes from the niv map or a plan table before
// using it: outside its range the status word gets MZ_ERR_BOUNDS and the index becomes a
// safe one (slot 0, a zero slot; node -1, nothing written). Release builds compile the
// checks away.
__device__ __forceinline__ int32_t chk(int32_t v, int64_t lo, int64_t hi, int32_t safe, uint32_t *status) {
#ifdef MZ_DEBUG
    if (v < lo || v >= hi) {
        report(status, MZ_ERR_BOUNDS);
        return safe;
    }
#endif
    return v;
}
// a niv map entry: a slot index in [0, nslots)
__device__ __forceinline__ int32_t map_ldg(const int32_t *p, int64_t nslots, uint32_t *status) {
    return chk(__ldg(p), 0, nslots, 0, status);
}
__device__ __forceinline__ int32_t map_ldcs(const int32_t *p, int64_t nslots, uint32_t *status) {
    return chk(__ldcs(p), 0, nslots, 0, status);
}

__device__ __forceinline__ float2 dwq_load(const float2 *Q, int64_t i, bool pair) {
    if (pair) {
        const float *q = reinterpret_cast<const float *>(Q) + 2 * (i & ~1ll) + (i & 1);
        return make_float2(q[0], q[2]);
    }
    return Q[i];
}

// Publishes y' word w (esc: its escape flag). A value whose bits equal the sentinel
// (possible for int64 only) goes out as kSentinel + 1 after its escape flag is set
// and fenced, so a reader that sees kSentinel + 1 and then fences sees the flag.
template <class M>
__device__ __forceinline__ void publish(unsigned long long *w, unsigned char *esc, typename M::T v) {
    unsigned long long b = M::to_bits(v);
    if constexpr (M::kEscapes) {
        if (b == M::kSentinel) {
            st_relaxed_u8(esc, 1);
            __threadfence();
            b = M::kSentinel + 1;
        }
    }
    st_relaxed_u64(w, b);
}

// The value of a published y' word (esc: its escape flag).
template <class M>
__device__ __forceinline__ typename M::T decode(unsigned long long b, const unsigned char *esc) {
    if constexpr (M::kEscapes) {
        if (b == M::kSentinel + 1) {
            __threadfence();
            if (ld_relaxed_u8(esc)) return M::from_bits(M::kSentinel);
        }
    }
    return M::from_bits(b);
}

// Wait until *flag != 0 (acquire). Gives up after `limit` polls, or early once
// another wait has recorded an error; returns 0 then.
__device__ uint32_t wait_flag(const uint32_t *flag, uint32_t *status, int64_t limit) {
    for (int64_t it = 0;; ++it) {
        uint32_t v = ld_acquire_u32(flag);
        if (v) return v;
        if ((it & 255) == 255 && ld_relaxed_u32(status)) return 0;
        if (it >= limit) {
            report(status, MZ_ERR_TIMEOUT);
            return 0;
        }
        __nanosleep(32);
    }
}

// Wait until *p != sentinel; returns the word (0 after a timeout or an abort).
__device__ __forceinline__ unsigned long long wait_value(const unsigned long long *p, unsigned long long sentinel,
                                                         uint32_t *status, int64_t limit) {
    unsigned long long v = ld_relaxed_u64(p);
    if (v != sentinel) return v;
    for (int64_t it = 0;; ++it) {
        v = ld_relaxed_u64(p);
        if (v != sentinel) return v;
        if ((it & 255) == 255 && ld_relaxed_u32(status)) return 0;
        if (it >= limit) {
            report(status, MZ_ERR_TIMEOUT);
            return 0;
        }
        if (it > 256) __nanosleep(32);
    }
}

// ---------------------------------------------------------------- chain scan (V f)
constexpr int kScanThreads = 256;
constexpr int kScanSeg = 16;  // slots per thread

template <class Pol>
__global__ void __launch_bounds__(kScanThreads) k_chain_scan(ScanArgs a) {
    using P_t = typename Pol::P_t;
    __shared__ uint32_t s_tile;
    __shared__ int s_has_reset;
    __shared__ unsigned char s_flag[kScanThreads];
    __shared__ P_t s_val[kScanThreads];
    __shared__ P_t s_excl[32];

    const int t = threadIdx.x;
    const int group = blockIdx.y;
    if (t == 0) {
        s_tile = atomicAdd(&a.counters[group], 1u);   // tiles start in order: look-back never waits on an unstarted tile
        s_has_reset = 0;
    }
    __syncthreads();
    const int64_t tile = s_tile;
    const int BW = a.BW, R = a.R;
    const int col = t % BW, r = t / BW;
    const bool active = r < R;
    const int64_t b = (int64_t)group * BW + col;
    const bool colok = active && b < a.B;
    const int64_t slot0 = tile * (int64_t)R * kScanSeg + (int64_t)r * kScanSeg;

    // all loads first (slot map as 16-byte vectors, then the f gathers), arithmetic after
    int32_t sn[kScanSeg];
    if (colok && slot0 < a.nslots) {
        const int4 *sv = reinterpret_cast<const int4 *>(a.slot_node + slot0);   // padded to 64 entries
#pragma unroll
        for (int q = 0; q < kScanSeg / 4; ++q) {
            const int4 w = sv[q];
            sn[4 * q] = w.x; sn[4 * q + 1] = w.y; sn[4 * q + 2] = w.z; sn[4 * q + 3] = w.w;
        }
#pragma unroll
        for (int j = 0; j < kScanSeg; ++j) sn[j] = chk(sn[j], -1, a.nB / a.B, -1, a.status);
    } else {
#pragma unroll
        for (int j = 0; j < kScanSeg; ++j) sn[j] = -1;
    }
    P_t vals[kScanSeg];
#pragma unroll
    for (int j = 0; j < kScanSeg; ++j)
        vals[j] = (sn[j] >= 0 && slot0 + j < a.nslots) ? Pol::load_in(a.f, (int64_t)sn[j] * a.B + b, a.nB) : Pol::zero();
    P_t acc = Pol::zero();
    int first_reset = kScanSeg;
#pragma unroll
    for (int j = 0; j < kScanSeg; ++j) {
        if (colok && slot0 + j < a.nslots) {
            if (sn[j] < 0) {                       // zero slot: a chain starts here
                acc = Pol::zero();
                if (first_reset == kScanSeg) first_reset = j;
            } else {
                acc = Pol::scan_add(acc, vals[j]);
            }
        }
        vals[j] = acc;
    }
    const bool seg_reset = first_reset < kScanSeg;
    if (seg_reset) s_has_reset = 1;
    s_flag[t] = seg_reset;
    s_val[t] = acc;
    __syncthreads();
    // inclusive segmented scan over the R sub-threads of each column (Hillis-Steele)
    for (int d = 1; d < R; d <<= 1) {
        const bool take = active && r >= d;
        unsigned char of = 0;
        P_t ov = Pol::zero();
        if (take) {
            of = s_flag[t - d * BW];
            ov = s_val[t - d * BW];
        }
        __syncthreads();
        if (take && !s_flag[t]) {
            s_val[t] = Pol::scan_add(ov, s_val[t]);
            s_flag[t] = of;
        }
        __syncthreads();
    }
    unsigned char ef = 0;
    P_t ev = Pol::zero();
    if (active && r > 0) {
        ef = s_flag[t - BW];
        ev = s_val[t - BW];
    }

    if (t < 32) {
        const int lane = t;
        const int64_t me = (int64_t)group * a.ntiles + tile;
        const bool has_reset = s_has_reset != 0;   // same for every column: resets sit at zero slots
        P_t tagg = Pol::zero();
        if (lane < BW) tagg = s_val[(R - 1) * BW + lane];
        P_t *agg = reinterpret_cast<P_t *>(a.agg);
        P_t *inc = reinterpret_cast<P_t *>(a.inc);
        const bool withhold = (me == a.withhold);
        // publish the tile aggregate, or directly its inclusive value when it holds a chain start
        if (lane < BW) {
            (has_reset ? inc : agg)[me * BW + lane] = tagg;
            __threadfence();
        }
        __syncwarp();
        if (lane == 0 && !withhold) st_release_u32(&a.flags[me], has_reset ? 2u : 1u);
        // look-back over the predecessors of this tile in the same column group
        P_t excl = Pol::zero();
        if (tile > 0) {
            int64_t pred = tile - 1;
            while (true) {
                const int64_t pid = (int64_t)group * a.ntiles + pred;
                const uint32_t fl = wait_flag(&a.flags[pid], a.status, a.spin_limit);
                if (fl == 2u) {
                    if (lane < BW) excl = Pol::scan_add(inc[pid * BW + lane], excl);
                    break;
                }
                if (fl == 1u) {
                    if (lane < BW) excl = Pol::scan_add(agg[pid * BW + lane], excl);
                    if (pred == 0) break;
                    --pred;
                    continue;
                }
                break;   // timed out or aborted
            }
        }
        if (!has_reset) {
            if (lane < BW) {
                inc[me * BW + lane] = Pol::scan_add(excl, tagg);
                __threadfence();
            }
            __syncwarp();
            if (lane == 0 && !withhold) st_release_u32(&a.flags[me], 2u);
        }
        if (lane < BW) s_excl[lane] = excl;
    }
    __syncthreads();

    if (colok) {
        const P_t pre = ef ? ev : Pol::scan_add(s_excl[col], ev);
        P_t *P = reinterpret_cast<P_t *>(a.P);
#pragma unroll
        for (int j = 0; j < kScanSeg; ++j) {
            const int64_t s = slot0 + j;
            if (s < a.nslots) {
                const P_t v = (j < first_reset) ? Pol::scan_add(pre, vals[j]) : vals[j];
                if constexpr (std::is_same<Pol, PolF32C>::value) {
                    if (a.pair_words) {   // hi of columns b, b ^ 1 side by side, then their lo
                        float *q = reinterpret_cast<float *>(a.P) + 2 * (s * a.B + (b & ~1ll)) + (b & 1);
                        q[0] = v.x;
                        q[2] = v.y;
                        continue;
                    }
                }
                P[s * a.B + b] = v;
            }
        }
    }
}

// ---------------------------------------------------------------- niv gather (U c)
constexpr int kGatherThreads = 256;

template <class Pol, int BT>
__global__ void __launch_bounds__(kGatherThreads) k_niv_gather(GatherArgs a) {
    using P_t = typename Pol::P_t;
    using Acc = typename Pol::Acc;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t b0 = (int64_t)blockIdx.y * BT;
    const P_t *__restrict__ P = reinterpret_cast<const P_t *>(a.P);
    for (int64_t tile = warp; tile < a.ntiles; tile += nwarps) {
        const int k = a.tile_k[tile];
        const int32_t *__restrict__ np = a.Nt + a.tile_off[tile] + lane;
        Acc acc[BT];
#pragma unroll
        for (int u = 0; u < BT; ++u) acc[u] = Pol::acc_zero();
        int c = 0;
        int32_t s[8];
        if (k >= 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) s[u] = map_ldcs(np + (int64_t)u * kTileRows, a.nslots, a.status);
        }
        for (; c + 8 <= k; c += 8) {
            // the next 8 map entries are requested before this group's values are gathered
            int32_t sn[8];
            const bool more = c + 16 <= k;
#pragma unroll
            for (int u = 0; u < 8; ++u) sn[u] = more ? map_ldcs(np + (int64_t)(c + 8 + u) * kTileRows, a.nslots, a.status) : 0;
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int q = 0; q < BT; ++q)
                    if (BT == 1 || b0 + q < a.B) Pol::acc_add(acc[q], __ldg(P + (int64_t)s[u] * a.B + b0 + q));
#pragma unroll
            for (int u = 0; u < 8; ++u) s[u] = sn[u];
        }
        for (; c < k; ++c) {
            const int32_t s = map_ldcs(np + (int64_t)c * kTileRows, a.nslots, a.status);
#pragma unroll
            for (int q = 0; q < BT; ++q)
                if (BT == 1 || b0 + q < a.B) Pol::acc_add(acc[q], __ldg(P + (int64_t)s * a.B + b0 + q));
        }
        const int32_t node = chk(a.row_node[tile * kTileRows + lane], -1, a.nB / a.B, -1, a.status);
        if (node >= 0) {
#pragma unroll
            for (int q = 0; q < BT; ++q)
                if (BT == 1 || b0 + q < a.B) Pol::store_out(a.g, (int64_t)node * a.B + b0 + q, a.nB, acc[q]);
        }
    }
}

// Batched gather (B > 1, B a power of two): one warp per tile of 32 rows, G = min(B, 32)
// lanes per row (lane b0 owns the columns b0 + G t), 32 / G row pairs at a time (rows r and
// r + 16: two independent sums, twice the loads in flight). Within a row group the map
// entry is a broadcast and the G loads of y' are contiguous. NARROW (nslots * B < 2^32):
// y' offsets in 32-bit arithmetic, one instruction per address instead of a 64-bit multiply.
template <class Pol, int G, bool NARROW>
__global__ void __launch_bounds__(kGatherThreads, 3) k_niv_gather_b(GatherArgs a) {
    using P_t = typename Pol::P_t;
    using Acc = typename Pol::Acc;
    constexpr int R = 32 / G;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, b0 = lane % G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const P_t *__restrict__ P = reinterpret_cast<const P_t *>(a.P);
    const int64_t B = a.B;
    const uint32_t Bu = (uint32_t)a.B;
    for (int64_t tile = warp; tile < a.ntiles; tile += nwarps) {
        const int k = a.tile_k[tile];
        const int32_t *__restrict__ nt = a.Nt + a.tile_off[tile];
        for (int r = sub; r < kTileRows / 2; r += R) {
            const int r2 = r + kTileRows / 2;
            const int32_t node = chk(a.row_node[tile * kTileRows + r], -1, a.nB / a.B, -1, a.status);
            const int32_t node2 = chk(a.row_node[tile * kTileRows + r2], -1, a.nB / a.B, -1, a.status);
            for (int64_t b = b0; b < B; b += G) {
                const P_t *__restrict__ Pb = P + b;
                Acc acc = Pol::acc_zero(), acc2 = Pol::acc_zero();
                int c = 0;
                for (; c + 8 <= k; c += 8) {
                    int32_t sl[8], sl2[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        sl[u] = map_ldg(nt + (int64_t)(c + u) * kTileRows + r, a.nslots, a.status);
                        sl2[u] = map_ldg(nt + (int64_t)(c + u) * kTileRows + r2, a.nslots, a.status);
                    }
                    P_t v[8], v2[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (NARROW) {
                            v[u] = __ldg(Pb + (uint32_t)sl[u] * Bu);
                            v2[u] = __ldg(Pb + (uint32_t)sl2[u] * Bu);
                        } else {
                            v[u] = __ldg(Pb + (int64_t)sl[u] * B);
                            v2[u] = __ldg(Pb + (int64_t)sl2[u] * B);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        Pol::acc_add(acc, v[u]);
                        Pol::acc_add(acc2, v2[u]);
                    }
                }
                for (; c < k; ++c) {
                    Pol::acc_add(acc, __ldg(P + (int64_t)map_ldg(nt + (int64_t)c * kTileRows + r, a.nslots, a.status) * B + b));
                    Pol::acc_add(acc2, __ldg(P + (int64_t)map_ldg(nt + (int64_t)c * kTileRows + r2, a.nslots, a.status) * B + b));
                }
                if (node >= 0) Pol::store_out(a.g, (int64_t)node * B + b, a.nB, acc);
                if (node2 >= 0) Pol::store_out(a.g, (int64_t)node2 * B + b, a.nB, acc2);
            }
        }
    }
}

// Batched zeta gather for B a multiple of 32: a half-warp per row and two adjacent
// columns per lane, so that one 16-byte load of y' serves two terms and one map entry and
// one address serve both (rows r and r + 8 in half 0, r + 16 and r + 24 in half 1). The
// compensated form runs 12-14 % faster than with k_niv_gather_b (256 posets, B = 32); the
// same layout for the Moebius leaf gather was not faster (it holds more live registers,
// so fewer warps fit), which keeps k_mob_leaf_b.
template <class T>
__device__ __forceinline__ T word_as(long long w) {
    T v;
    memcpy(&v, &w, sizeof(T));
    return v;
}

template <class Pol, bool NARROW>
__global__ void __launch_bounds__(kGatherThreads, 2) k_niv_gather_h(GatherArgs a) {
    using P_t = typename Pol::P_t;
    using Acc = typename Pol::Acc;
    static_assert(sizeof(P_t) == 8, "8-byte prefix words");
    const int lane = threadIdx.x & 31;
    const int half = lane >> 4, cp = lane & 15;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const P_t *__restrict__ P = reinterpret_cast<const P_t *>(a.P);
    const int64_t B = a.B;
    const uint32_t Bu = (uint32_t)a.B;
    for (int64_t tile = warp; tile < a.ntiles; tile += nwarps) {
        const int k = a.tile_k[tile];
        const int32_t *__restrict__ nt = a.Nt + a.tile_off[tile];
        for (int r0 = 0; r0 < 8; ++r0) {
            const int ra = r0 + 16 * half, rb = ra + 8;
            const int32_t na = chk(a.row_node[tile * kTileRows + ra], -1, a.nB / a.B, -1, a.status);
            const int32_t nb = chk(a.row_node[tile * kTileRows + rb], -1, a.nB / a.B, -1, a.status);
            for (int64_t b = 2 * cp; b < B; b += 32) {
                const P_t *__restrict__ Pb = P + b;
                Acc a0 = Pol::acc_zero(), a1 = Pol::acc_zero(), b0 = Pol::acc_zero(), b1 = Pol::acc_zero();
                int c = 0;
                for (; c + 8 <= k; c += 8) {
                    int32_t sa[8], sb[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        sa[u] = map_ldg(nt + (int64_t)(c + u) * kTileRows + ra, a.nslots, a.status);
                        sb[u] = map_ldg(nt + (int64_t)(c + u) * kTileRows + rb, a.nslots, a.status);
                    }
                    longlong2 va[8], vb[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const P_t *pa = NARROW ? Pb + (uint32_t)sa[u] * Bu : Pb + (int64_t)sa[u] * B;
                        const P_t *pb = NARROW ? Pb + (uint32_t)sb[u] * Bu : Pb + (int64_t)sb[u] * B;
                        va[u] = __ldg(reinterpret_cast<const longlong2 *>(pa));
                        vb[u] = __ldg(reinterpret_cast<const longlong2 *>(pb));
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        Pol::acc_add(a0, word_as<P_t>(va[u].x));
                        Pol::acc_add(a1, word_as<P_t>(va[u].y));
                        Pol::acc_add(b0, word_as<P_t>(vb[u].x));
                        Pol::acc_add(b1, word_as<P_t>(vb[u].y));
                    }
                }
                for (; c < k; ++c) {
                    const P_t *pa = P + (int64_t)map_ldg(nt + (int64_t)c * kTileRows + ra, a.nslots, a.status) * B + b;
                    const P_t *pb = P + (int64_t)map_ldg(nt + (int64_t)c * kTileRows + rb, a.nslots, a.status) * B + b;
                    Pol::acc_add(a0, __ldg(pa));
                    Pol::acc_add(a1, __ldg(pa + 1));
                    Pol::acc_add(b0, __ldg(pb));
                    Pol::acc_add(b1, __ldg(pb + 1));
                }
                if (na >= 0) {
                    Pol::store_out(a.g, (int64_t)na * B + b, a.nB, a0);
                    Pol::store_out(a.g, (int64_t)na * B + b + 1, a.nB, a1);
                }
                if (nb >= 0) {
                    Pol::store_out(a.g, (int64_t)nb * B + b, a.nB, b0);
                    Pol::store_out(a.g, (int64_t)nb * B + b + 1, a.nB, b1);
                }
            }
        }
    }
}

// Sum2 of one pair of tile rows (ra, rb) over one column pair of the packed F32C words, in
// groups of 8 entries: a group's words are requested together, and the map entries of the
// next group load while they arrive. Entries are added in map order. (Measured on 256
// posets, B = 32: 2.70 ms per zeta gather; two groups of 4 in flight 3.10 ms, of 8 with
// the same scheme 6.8 ms.)
template <bool NARROW>
__device__ __forceinline__ void pair_rows_sum2(const int32_t *__restrict__ nt, int ra, int rb, int k,
                                               const ulonglong2 *__restrict__ Pb, int64_t B2, uint32_t B2u,
                                               int64_t nslots, uint32_t *status, Acc2 &x, Acc2 &y) {
    int32_t sa[8], sb[8];
    if (k >= 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            sa[u] = map_ldg(nt + (int64_t)u * kTileRows + ra, nslots, status);
            sb[u] = map_ldg(nt + (int64_t)u * kTileRows + rb, nslots, status);
        }
    }
    int c = 0;
    for (; c + 8 <= k; c += 8) {
        ulonglong2 va[8], vb[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            va[u] = __ldg(NARROW ? Pb + (uint32_t)sa[u] * B2u : Pb + (int64_t)sa[u] * B2);
            vb[u] = __ldg(NARROW ? Pb + (uint32_t)sb[u] * B2u : Pb + (int64_t)sb[u] * B2);
        }
        if (c + 16 <= k) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                sa[u] = map_ldg(nt + (int64_t)(c + 8 + u) * kTileRows + ra, nslots, status);
                sb[u] = map_ldg(nt + (int64_t)(c + 8 + u) * kTileRows + rb, nslots, status);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            acc2_add(x, va[u].x, va[u].y);
            acc2_add(y, vb[u].x, vb[u].y);
        }
    }
    for (; c < k; ++c) {
        const ulonglong2 va = __ldg(Pb + (int64_t)map_ldg(nt + (int64_t)c * kTileRows + ra, nslots, status) * B2);
        const ulonglong2 vb = __ldg(Pb + (int64_t)map_ldg(nt + (int64_t)c * kTileRows + rb, nslots, status) * B2);
        acc2_add(x, va.x, va.y);
        acc2_add(y, vb.x, vb.y);
    }
}

// The compensated gather of k_niv_gather_h on packed fp32 pairs: the chain scan stores
// the prefixes of columns b and b + 1 (b even) as hi_b, hi_b+1, lo_b, lo_b+1, so one
// 16-byte load gives the pair of hi parts and the pair of lo parts, and every step of
// Sum2 runs once for both columns (sums bit-identical to k_niv_gather_h, in half the fp32
// instructions).
template <bool NARROW>
__global__ void __launch_bounds__(kGatherThreads, 2) k_niv_gather_h2(GatherArgs a) {
    const int lane = threadIdx.x & 31;
    const int half = lane >> 4, cp = lane & 15;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const ulonglong2 *__restrict__ P = reinterpret_cast<const ulonglong2 *>(a.P);   // one per column pair
    const int64_t B = a.B, B2 = a.B / 2;
    const uint32_t B2u = (uint32_t)(a.B / 2);
    float *g = reinterpret_cast<float *>(a.g);
    for (int64_t tile = warp; tile < a.ntiles; tile += nwarps) {
        const int k = a.tile_k[tile];
        const int32_t *__restrict__ nt = a.Nt + a.tile_off[tile];
        for (int r0 = 0; r0 < 8; ++r0) {
            const int ra = r0 + 16 * half, rb = ra + 8;
            const int32_t na = chk(a.row_node[tile * kTileRows + ra], -1, a.nB / a.B, -1, a.status);
            const int32_t nb = chk(a.row_node[tile * kTileRows + rb], -1, a.nB / a.B, -1, a.status);
            for (int64_t bp = cp; bp < B2; bp += 16) {        // column pair bp: columns 2 bp, 2 bp + 1
                const ulonglong2 *__restrict__ Pb = P + bp;
                Acc2 x{0ull, 0ull}, y{0ull, 0ull};
                pair_rows_sum2<NARROW>(nt, ra, rb, k, Pb, B2, B2u, a.nslots, a.status, x, y);
                // normalise once, as PolF32C::store_out: hi and lo planes, both columns at once
                f32x2 hi, lo;
                if (na >= 0) {
                    two_sum2(x.s, x.e, hi, lo);
                    const int64_t i = (int64_t)na * B + 2 * bp;
                    *reinterpret_cast<f32x2 *>(g + i) = hi;
                    *reinterpret_cast<f32x2 *>(g + a.nB + i) = lo;
                }
                if (nb >= 0) {
                    two_sum2(y.s, y.e, hi, lo);
                    const int64_t i = (int64_t)nb * B + 2 * bp;
                    *reinterpret_cast<f32x2 *>(g + i) = hi;
                    *reinterpret_cast<f32x2 *>(g + a.nB + i) = lo;
                }
            }
        }
    }
}

// ---------------------------------------------------------------- Moebius
// y' init: the sentinel ("not yet published") at every slot the forward substitution
// computes, 0 at zero slots and at the rows no other row reads (the leaf gather adds
// the own-chain entry of such a row, its own slot, and it must add nothing); escape
// flags and double-word copies cleared.
template <class M>
__global__ void k_mob_init(const int32_t *__restrict__ slot_node, const uint8_t *__restrict__ slot_ref,
                           int64_t nslots, int32_t B, unsigned long long *__restrict__ P,
                           unsigned char *__restrict__ esc, float2 *__restrict__ Q) {
    const int64_t total = nslots * B;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / B;
        const bool live = slot_node[s] >= 0 && (slot_ref == nullptr || slot_ref[s] != 0);
        P[i] = live ? M::kSentinel : 0ull;
        if (esc) esc[i] = 0;
        if (Q) Q[i] = make_float2(0.f, 0.f);
    }
}

template <class T>
__device__ __forceinline__ T shfl_xor_t(T v, int off) {
    return __shfl_xor_sync(0xffffffffu, v, off);
}

// x + 0 for a value type without the arithmetic pipe: -0 becomes +0 and every other value
// stays what an IEEE add of +0 gives (a sum is never a signalling NaN, and a NaN ends up
// as the final subtraction makes it either way); integers are unchanged. It stands for
// the levels of a 32-lane shuffle tree that only add the zeros of lanes holding no chunk.
template <class M>
__device__ __forceinline__ typename M::T plus_zero(typename M::T x) {
    if constexpr (std::is_same<typename M::T, double>::value) {
        return __double_as_longlong(x) == (long long)0x8000000000000000ull ? 0.0 : x;
    } else {
        return x;
    }
}

// Sleeps about ns nanoseconds. __nanosleep may sleep up to twice what it is asked, so a
// long wait is a deadline on the SM clock (about 2 cycles per ns) checked between naps of
// a quarter microsecond: a thread sleeping through many levels wakes on time.
__device__ __forceinline__ void pace_until(int64_t ns) {
    if (ns <= 0) return;
    const long long end = clock64() + 2 * ns;
    while (clock64() < end) __nanosleep(256);
}

// Sums the NV words v[j] = P[id[j]] into acc (or subtracts them, SUB) in column order, adding each one as
// soon as it and all before it are present: columns are sorted by dependency
// level, so words land roughly in order and when the last one lands only one
// addition is left. The first missing word is polled, one request per round;
// once it lands every later missing word is requested again in one round.
// E: the escape flags aligned with P (int64 only).
template <class M, int NV, bool SUB>
__device__ __forceinline__ void sum_in_order(unsigned long long *v, const int32_t *id, const unsigned long long *P,
                                             const unsigned char *E, typename M::T &acc, uint32_t *status,
                                             int64_t limit, int start) {
    const unsigned long long S = M::kSentinel;
    int next = start;   // words before `start` are the row's padding (slot 0, the value 0)
    auto advance = [&]() {
#pragma unroll
        for (int j = 0; j < NV; ++j)
            if (j == next && v[j] != S) {
                const typename M::T x = decode<M>(v[j], E + id[j]);
                acc = SUB ? M::sub(acc, x) : M::add(acc, x);
                next = j + 1;
            }
    };
    advance();
    for (int64_t it = 0; next < NV; ++it) {
        const unsigned long long *addr = P;
#pragma unroll
        for (int j = 0; j < NV; ++j)
            if (j == next) addr = P + id[j];
        // no pause between rounds: a sleep, however short, costs a round trip per level
        const unsigned long long got = ld_relaxed_u64(addr);
        if (got != S) {
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                if (j == next) v[j] = got;
                else if (j > next && v[j] == S) v[j] = ld_relaxed_u64(P + id[j]);
            }
        } else if ((it & 127) == 127 && (ld_relaxed_u32(status) || it >= limit)) {
            if (it >= limit) report(status, MZ_ERR_TIMEOUT);
#pragma unroll
            for (int j = 0; j < NV; ++j)
                if (v[j] == S) v[j] = 0ull;
        }
        advance();
    }
}

// One thread per row, B == 1. Rows have kpad columns (a multiple of 16; the
// padding entries come first and point at slot 0, a zero slot), sorted by the
// level of their dependency, so the last chunk of 16 holds the ones that finish
// last. A thread never waits for another thread's columns: once its last
// dependency lands, one poll round, a few additions and the store remain.
// The ids of the next chunk load while the current chunk is awaited, and the
// thread's next row is prefetched into L1 at the start of each row.
constexpr int kChunk = 16;

__device__ __forceinline__ void load_ids(const int32_t *p, int32_t *id, int64_t nslots, uint32_t *status) {
    const int4 *q = reinterpret_cast<const int4 *>(p);
#pragma unroll
    for (int t = 0; t < kChunk / 4; ++t) {
        const int4 w = __ldg(q + t);
        id[4 * t] = w.x; id[4 * t + 1] = w.y; id[4 * t + 2] = w.z; id[4 * t + 3] = w.w;
    }
#pragma unroll
    for (int j = 0; j < kChunk; ++j) id[j] = chk(id[j], 0, nslots, 0, status);
}

// G lanes per row (G = 1 for one function, G = min(B, 32) for B functions, B a
// power of two): lane b0 of a row group owns the columns b = b0 + G t, t < B / G,
// and waits only for its own words, so no lane ever waits for another lane.
template <class M, bool ANTI, int G>
__global__ void __launch_bounds__(128) k_mob_wave_t(MobArgs a) {
    using T = typename M::T;
    // Warps are numbered across blocks first (warp w of block b is warp b + w * gridDim.x),
    // so consecutive groups of rows, which share a level, go to different SMs; inside a
    // warp the rows stay consecutive. G lanes per row.
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = gwarp * 32 + lane;
    const int64_t grp = tid / G, ngrp = nthreads / G;
    const int b0 = (int)(tid % G);
    const int64_t B = (G == 1) ? 1 : a.B;
    unsigned long long *P = a.P;
    const unsigned long long SENT = M::kSentinel;
    int32_t done_level = 0;   // level of the row this group finished last (the frontier was there)
    for (int64_t i = grp; i < a.n; i += ngrp) {
        const int32_t *row = a.Nm + a.mob_off[i];
        const int kp = a.mob_kp[i];
        const int32_t level = a.mob_level[i];
        // The dependencies of this row sit at least one level lower; levels finish one
        // after the other, so sleep through the ones that must come first.
        if (a.pace_ns > 0) pace_until((int64_t)(level - done_level - 2) * a.pace_ns);
        if (b0 == 0 && i + ngrp < a.n) {
            const char *nxt = reinterpret_cast<const char *>(a.Nm + a.mob_off[i + ngrp]);
            const int nkp = a.mob_kp[i + ngrp];
            for (int c = 0; c < nkp * 4; c += 128) asm volatile("prefetch.global.L1 [%0];" ::"l"(nxt + c));
        }
        const int64_t node = chk(a.mob_node[i], 0, a.nB / a.B, 0, a.status);
        const int64_t sout = chk(a.mob_slot[i], 0, a.nslots, 0, a.status);
        const bool publish_row = (i != a.withhold);
        for (int64_t b = b0; b < B; b += G) {
            unsigned long long *Pb = P + b;           // column b of every slot: Pb[s * B]
            unsigned char *Eb = M::kEscapes ? a.esc + b : nullptr;
            const T gx = M::load_in(a.g, node * B + b, a.nB);
            unsigned long long vprev = ANTI ? ld_relaxed_u64(Pb + (sout - 1) * B) : 0ull;
            int32_t id[kChunk], nid[kChunk];
            load_ids(row, id, a.nslots, a.status);
            // The row's padding: slot 0 (a zero slot, never an element) in front of its entries.
            // Its words are 0, and subtracting or adding them (from g(x), or from a sum that
            // starts at +0) leaves every bit as it is, so they are skipped: fp64 adds are what
            // bounds this kernel on GB300, and rows of posets with few chains are mostly padding.
            int lead = 0;
#pragma unroll
            for (int j = 0; j < kChunk; ++j) lead += id[j] == 0;
            // U form: acc runs as g(x) - (sum of the values so far), so that once the last
            // value lands one subtraction is left; the antichain form sums, as it needs
            // y'(next(x)) apart.
            T acc = ANTI ? T(0) : gx;
            // all chunks but the last: in column order
            for (int c0 = 0; c0 + kChunk < kp; c0 += kChunk) {
                unsigned long long v[kChunk];
                int32_t sid[kChunk];
                const int start = c0 == 0 ? lead : 0;
#pragma unroll
                for (int j = 0; j < kChunk; ++j) sid[j] = (int32_t)((int64_t)id[j] * B);
#pragma unroll
                for (int j = 0; j < kChunk; ++j) v[j] = j < start ? 0ull : ld_relaxed_u64(Pb + sid[j]);
                load_ids(row + c0 + kChunk, nid, a.nslots, a.status);
                sum_in_order<M, kChunk, !ANTI>(v, sid, Pb, Eb, acc, a.status, a.spin_limit, start);
#pragma unroll
                for (int j = 0; j < kChunk; ++j) id[j] = nid[j];
            }
            // The last chunk holds the latest dependencies. The row is finished and
            // published inside the waiting loop itself, the moment its last value is
            // in: a lane never waits for the other lanes of its warp to publish.
            {
                const unsigned long long S = SENT;
                unsigned long long v[kChunk];
                int64_t sid[kChunk];
                const int start = kp == kChunk ? lead : 0;   // the row's only chunk holds its padding
#pragma unroll
                for (int j = 0; j < kChunk; ++j) sid[j] = (int64_t)id[j] * B;
#pragma unroll
                for (int j = 0; j < kChunk; ++j) v[j] = j < start ? 0ull : ld_relaxed_u64(Pb + sid[j]);
                int next = start;
                for (int64_t it = 0;; ++it) {
#pragma unroll
                    for (int j = 0; j < kChunk; ++j)
                        if (j == next && v[j] != S) {
                            const T x = decode<M>(v[j], Eb + sid[j]);
                            acc = ANTI ? M::add(acc, x) : M::sub(acc, x);
                            next = j + 1;
                        }
                    if (ANTI && next == kChunk && vprev == S) vprev = ld_relaxed_u64(Pb + (sout - 1) * B);
                    if (next == kChunk && (!ANTI || vprev != S)) {
                        if (ANTI) {
                            const T prev = decode<M>(vprev, Eb + (sout - 1) * B);
                            const T fx = M::sub(gx, M::add(acc, prev));
                            if (publish_row) publish<M>(Pb + sout * B, Eb + sout * B, M::add(prev, fx));
                            M::store_out(a.f, node * B + b, a.nB, fx);
                        } else if (publish_row) {
                            if constexpr (M::kDW) {
                                if (a.Q) dwq_store(a.Q, sout * B + b, a.pair_q, M::to_dw(acc));   // read after this kernel ends
                            }
                            publish<M>(Pb + sout * B, Eb + sout * B, acc);
                        }
                        break;
                    }
                    if ((it & 127) == 127 && (ld_relaxed_u32(a.status) || it >= a.spin_limit)) {
                        if (it >= a.spin_limit) report(a.status, MZ_ERR_TIMEOUT);
#pragma unroll
                        for (int j = 0; j < kChunk; ++j)
                            if (v[j] == S) v[j] = 0ull;
                        if (vprev == S) vprev = 0ull;
                        continue;
                    }
                    // one round: ask again for every missing word at once
#pragma unroll
                    for (int j = 0; j < kChunk; ++j)
                        if (j >= next && v[j] == S) v[j] = ld_relaxed_u64(Pb + sid[j]);
                }
            }
        }
        done_level = level;
    }
}

// One function, U-level schedule, LR lanes per row: the row's chunks of 16 entries are
// dealt to its lanes (chunk c to lane c mod LR), so all of a row's values are requested in
// one round trip however late the row starts. Each lane adds its values as they land
// (re-asking every missing one each round, bounded); the lanes' sums meet by shuffles and
// the row's first lane publishes y'(x) = g(x) - sum. The row's own data (node, slot, g(x))
// is requested before the waiting starts, so that only the shuffles, one subtraction and
// the store follow the last value. (Measured on GB300, n = 2^20, k = 64: the full shuffle
// tree after a warp barrier beat a tree over only the lanes holding chunks, a publishing
// lane that waits on the last chunk itself, and partial sums met in shared memory.)
template <class M, int LR>
__global__ void __launch_bounds__(128) k_mob_wave_lr(MobArgs a) {
    using T = typename M::T;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int64_t tid = gwarp * 32 + lane;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t grp = tid / LR, ngrp = nthreads / LR;
    const int sub = lane & (LR - 1);
    const unsigned gmask = LR == 32 ? 0xffffffffu : (((1u << LR) - 1u) << (lane & ~(LR - 1)));
    unsigned long long *P = a.P;
    unsigned char *E = a.esc;
    const unsigned long long S = M::kSentinel;
    int32_t done_level = 0;
    for (int64_t i = grp; i < a.n; i += ngrp) {
        const int32_t *row = a.Nm + a.mob_off[i];
        const int nch = a.mob_kp[i] / kChunk;
        const int32_t level = a.mob_level[i];
        if (a.pace_ns > 0) pace_until((int64_t)(level - done_level - 2) * a.pace_ns);
        if (sub == 0 && i + ngrp < a.n) {
            const char *nxt = reinterpret_cast<const char *>(a.Nm + a.mob_off[i + ngrp]);
            const int nkp = a.mob_kp[i + ngrp];
            for (int c = 0; c < nkp * 4; c += 128) asm volatile("prefetch.global.L1 [%0];" ::"l"(nxt + c));
        }
        int64_t sout = 0;
        T gx = T(0);
        if (sub == 0) {
            const int64_t node = chk(a.mob_node[i], 0, a.nB, 0, a.status);   // B == 1
            sout = chk(a.mob_slot[i], 0, a.nslots, 0, a.status);
            gx = M::load_in(a.g, node, a.nB);
        }
        T acc = T(0);
        for (int c = sub; c < nch; c += LR) {
            int32_t id[kChunk];
            load_ids(row + c * kChunk, id, a.nslots, a.status);
            unsigned long long v[kChunk];
#pragma unroll
            for (int j = 0; j < kChunk; ++j) v[j] = ld_relaxed_u64(P + id[j]);
            int next = 0;
            for (int64_t it = 0;; ++it) {
#pragma unroll
                for (int j = 0; j < kChunk; ++j)
                    if (j == next && v[j] != S) {
                        acc = M::add(acc, decode<M>(v[j], E + id[j]));
                        next = j + 1;
                    }
                if (next == kChunk) break;
                if ((it & 127) == 127 && (ld_relaxed_u32(a.status) || it >= a.spin_limit)) {
                    if (it >= a.spin_limit) report(a.status, MZ_ERR_TIMEOUT);
#pragma unroll
                    for (int j = 0; j < kChunk; ++j)
                        if (v[j] == S) v[j] = 0ull;
                    continue;
                }
                // no pause between rounds: a sleep, however short, costs a round trip per level
                // (and additions only when a word has landed were slower: 0.65 -> 0.75 ms)
#pragma unroll
                for (int j = 0; j < kChunk; ++j)
                    if (j >= next && v[j] == S) v[j] = ld_relaxed_u64(P + id[j]);
            }
        }
        if (LR > 1) {
            // The LR-lane butterfly; its levels above the plan's tree width only add the zeros
            // of lanes without a chunk, one plus_zero in their place (same bits). Each fp64 add
            // on this path costs latency on GB300's narrow FP64 pipe: dropping the three
            // all-zero levels at k = 64 took the wavefront from 0.75 to 0.65 ms.
            __syncwarp(gmask);
            const int tw = a.tree_w < LR ? a.tree_w : LR;
            if (tw < LR) acc = plus_zero<M>(acc);
            for (int off = tw / 2; off >= 1; off >>= 1) acc = M::add(acc, __shfl_xor_sync(gmask, acc, off));
        }
        if (sub == 0 && i != a.withhold) {
            const T y = M::sub(gx, acc);
            if constexpr (M::kDW) {
                if (a.Q) a.Q[sout] = M::to_dw(y);   // read after this kernel ends
            }
            publish<M>(P + sout, E + sout, y);
        }
        done_level = level;
    }
}

template <class M, bool ANTI>
__global__ void __launch_bounds__(256) k_mob_wave(MobArgs a) {
    using T = typename M::T;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t B = a.B;
    unsigned long long *P = a.P;
    unsigned char *E = a.esc;
    const unsigned long long SENT = M::kSentinel;
    auto get = [&](int64_t w) { return decode<M>(wait_value(P + w, SENT, a.status, a.spin_limit), E + w); };
    auto put = [&](int64_t w, T v) {
        if constexpr (M::kDW) {
            if (!ANTI && a.Q) dwq_store(a.Q, w, a.pair_q, M::to_dw(v));
        }
        publish<M>(P + w, E + w, v);
    };
    for (int64_t i = warp; i < a.n; i += nwarps) {
        const int32_t *__restrict__ row = a.Nm + a.mob_off[i];
        const int k = a.mob_kp[i];
        const int64_t node = chk(a.mob_node[i], 0, a.nB / a.B, 0, a.status);
        const int64_t sout = chk(a.mob_slot[i], 0, a.nslots, 0, a.status);
        const bool publish_row = (i != a.withhold);
        auto ent = [&](int c) { return (int64_t)chk(row[c], 0, a.nslots, 0, a.status); };
        if (B == 1) {
            T acc = T(0);
            for (int c = lane; c < k; c += 32) acc = M::add(acc, get(ent(c)));
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) acc = M::add(acc, shfl_xor_t(acc, off));
            if (lane == 0) {
                const T gx = M::load_in(a.g, node, a.nB);
                if (ANTI) {
                    const T prev = get(sout - 1);
                    const T fx = M::sub(gx, M::add(acc, prev));
                    if (publish_row) put(sout, M::add(prev, fx));
                    M::store_out(a.f, node, a.nB, fx);
                } else if (publish_row) {
                    put(sout, M::sub(gx, acc));
                }
            }
        } else if (B <= 32 && (B & (B - 1)) == 0) {
            const int bl = lane & (B - 1);
            const int cstep = 32 / B;
            T acc = T(0);
            for (int c = lane / B; c < k; c += cstep) acc = M::add(acc, get(ent(c) * B + bl));
            for (int off = 16; off >= B; off >>= 1) acc = M::add(acc, shfl_xor_t(acc, off));
            if (lane < B) {
                const T gx = M::load_in(a.g, node * B + bl, a.nB);
                if (ANTI) {
                    const T prev = get((sout - 1) * B + bl);
                    const T fx = M::sub(gx, M::add(acc, prev));
                    if (publish_row) put(sout * B + bl, M::add(prev, fx));
                    M::store_out(a.f, node * B + bl, a.nB, fx);
                } else if (publish_row) {
                    put(sout * B + bl, M::sub(gx, acc));
                }
            }
        } else {
            for (int64_t bl = lane; bl < B; bl += 32) {
                T acc = T(0);
                for (int c = 0; c < k; ++c) acc = M::add(acc, get(ent(c) * B + bl));
                const T gx = M::load_in(a.g, node * B + bl, a.nB);
                if (ANTI) {
                    const T prev = get((sout - 1) * B + bl);
                    const T fx = M::sub(gx, M::add(acc, prev));
                    if (publish_row) put(sout * B + bl, M::add(prev, fx));
                    M::store_out(a.f, node * B + bl, a.nB, fx);
                } else if (publish_row) {
                    put(sout * B + bl, M::sub(gx, acc));
                }
            }
        }
    }
}

// ---- leaf gather (U-level schedule): the rows no other row reads, after the forward
// substitution has finished every row they read: y'(x) = g(x) - sum over x's tile row of
// the gather's map (own slot included, zeroed by the init). The same tiles and lane
// layouts as the zeta gather.
template <class L, class M>
__device__ __forceinline__ typename L::W leaf_load(const MobArgs &a, const typename L::W *Pw, int64_t idx) {
    typename L::W v = __ldg(Pw + idx);
    if constexpr (M::kEscapes) {   // int64: a word of kSentinel + 1 with its escape flag set holds kSentinel
        if ((unsigned long long)v == M::kSentinel + 1 && a.esc[idx]) v = (typename L::W)M::kSentinel;
    }
    return v;
}

template <class L, class M>
__device__ __forceinline__ const typename L::W *leaf_words(const MobArgs &a) {
    if constexpr (M::kDW) return reinterpret_cast<const typename L::W *>(a.Q);
    else return reinterpret_cast<const typename L::W *>(a.P);
}

template <class L, class M>
__device__ __forceinline__ void leaf_store(const MobArgs &a, int64_t idx, typename L::W v) {
    if constexpr (M::kDW) a.Q[idx] = v;
    else reinterpret_cast<typename L::W *>(a.P)[idx] = v;
}

template <class L, class M, int BT>
__global__ void __launch_bounds__(kGatherThreads) k_mob_leaf(MobArgs a) {
    using W = typename L::W;
    using Acc = typename L::Acc;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t b0 = (int64_t)blockIdx.y * BT;
    const int64_t B = a.B;
    const W *__restrict__ Pw = leaf_words<L, M>(a);
    for (int64_t tile = warp; tile < a.ntiles; tile += nwarps) {
        const int32_t lslot = chk(a.row_leaf[tile * kTileRows + lane], -1, a.nslots, -1, a.status);
        if (__all_sync(0xffffffffu, lslot < 0)) continue;   // no leaf row in this tile
        const int k = a.tile_k[tile];
        const int32_t *__restrict__ np = a.Nt + a.tile_off[tile] + lane;
        Acc acc[BT];
#pragma unroll
        for (int u = 0; u < BT; ++u) acc[u] = L::acc_zero();
        int c = 0;
        for (; c + 8 <= k; c += 8) {
            int32_t s[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) s[u] = map_ldcs(np + (int64_t)(c + u) * kTileRows, a.nslots, a.status);
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int q = 0; q < BT; ++q)
                    if (BT == 1 || b0 + q < B) L::acc_add(acc[q], leaf_load<L, M>(a, Pw, (int64_t)s[u] * B + b0 + q));
        }
        for (; c < k; ++c) {
            const int32_t s = map_ldcs(np + (int64_t)c * kTileRows, a.nslots, a.status);
#pragma unroll
            for (int q = 0; q < BT; ++q)
                if (BT == 1 || b0 + q < B) L::acc_add(acc[q], leaf_load<L, M>(a, Pw, (int64_t)s * B + b0 + q));
        }
        if (lslot >= 0) {
            const int64_t node = chk(a.row_node[tile * kTileRows + lane], 0, a.nB / a.B, 0, a.status);
#pragma unroll
            for (int q = 0; q < BT; ++q)
                if (BT == 1 || b0 + q < B)
                    leaf_store<L, M>(a, (int64_t)lslot * B + b0 + q, L::result(a.g, node * B + b0 + q, a.nB, acc[q]));
        }
    }
}

// Batched leaf gather (B > 1 a power of two): the lane layout of k_niv_gather_b.
template <class L, class M, int G, bool NARROW>
__global__ void __launch_bounds__(kGatherThreads, 3) k_mob_leaf_b(MobArgs a) {
    using W = typename L::W;
    using Acc = typename L::Acc;
    constexpr int R = 32 / G;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, b0 = lane % G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const W *__restrict__ Pw = leaf_words<L, M>(a);
    const int64_t B = a.B;
    const uint32_t Bu = (uint32_t)a.B;
    for (int64_t tile = warp; tile < a.ntiles; tile += nwarps) {
        const int32_t *rl = a.row_leaf + tile * kTileRows;
        if (__all_sync(0xffffffffu, rl[lane] < 0)) continue;   // no leaf row in this tile
        const int k = a.tile_k[tile];
        const int32_t *__restrict__ nt = a.Nt + a.tile_off[tile];
        for (int r = sub; r < kTileRows / 2; r += R) {
            const int r2 = r + kTileRows / 2;
            const int32_t ls = chk(rl[r], -1, a.nslots, -1, a.status), ls2 = chk(rl[r2], -1, a.nslots, -1, a.status);
            if (ls < 0 && ls2 < 0) continue;                    // the whole lane group agrees
            const int64_t node = chk(a.row_node[tile * kTileRows + r], -1, a.nB / a.B, 0, a.status);
            const int64_t node2 = chk(a.row_node[tile * kTileRows + r2], -1, a.nB / a.B, 0, a.status);
            for (int64_t b = b0; b < B; b += G) {
                Acc acc = L::acc_zero(), acc2 = L::acc_zero();
                int c = 0;
                for (; c + 8 <= k; c += 8) {
                    int32_t sl[8], sl2[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        sl[u] = map_ldg(nt + (int64_t)(c + u) * kTileRows + r, a.nslots, a.status);
                        sl2[u] = map_ldg(nt + (int64_t)(c + u) * kTileRows + r2, a.nslots, a.status);
                    }
                    W v[8], v2[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (NARROW) {
                            v[u] = leaf_load<L, M>(a, Pw, (int64_t)((uint32_t)sl[u] * Bu + (uint32_t)b));
                            v2[u] = leaf_load<L, M>(a, Pw, (int64_t)((uint32_t)sl2[u] * Bu + (uint32_t)b));
                        } else {
                            v[u] = leaf_load<L, M>(a, Pw, (int64_t)sl[u] * B + b);
                            v2[u] = leaf_load<L, M>(a, Pw, (int64_t)sl2[u] * B + b);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        L::acc_add(acc, v[u]);
                        L::acc_add(acc2, v2[u]);
                    }
                }
                for (; c < k; ++c) {
                    L::acc_add(acc, leaf_load<L, M>(a, Pw, (int64_t)map_ldg(nt + (int64_t)c * kTileRows + r, a.nslots, a.status) * B + b));
                    L::acc_add(acc2, leaf_load<L, M>(a, Pw, (int64_t)map_ldg(nt + (int64_t)c * kTileRows + r2, a.nslots, a.status) * B + b));
                }
                if (ls >= 0) leaf_store<L, M>(a, (int64_t)ls * B + b, L::result(a.g, node * B + b, a.nB, acc));
                if (ls2 >= 0) leaf_store<L, M>(a, (int64_t)ls2 * B + b, L::result(a.g, node2 * B + b, a.nB, acc2));
            }
        }
    }
}

// The F32C leaf gather on packed fp32 pairs (B a power of two >= 32, Q in column pairs):
// the lane layout of k_niv_gather_h2, Sum2 over the double-word copies of both columns
// at once, then g(x) minus the sum in double-word arithmetic (LeafF32C::result on both
// halves), written back as one 16-byte group. Bit-identical to k_mob_leaf_b.
template <bool NARROW>
__global__ void __launch_bounds__(kGatherThreads, 2) k_mob_leaf_h2(MobArgs a) {
    const int lane = threadIdx.x & 31;
    const int half = lane >> 4, cp = lane & 15;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    ulonglong2 *__restrict__ Q = reinterpret_cast<ulonglong2 *>(a.Q);   // one per column pair
    const int64_t B = a.B, B2 = a.B / 2;
    const uint32_t B2u = (uint32_t)(a.B / 2);
    const float *g = reinterpret_cast<const float *>(a.g);
    for (int64_t tile = warp; tile < a.ntiles; tile += nwarps) {
        const int32_t *rl = a.row_leaf + tile * kTileRows;
        if (__all_sync(0xffffffffu, rl[lane] < 0)) continue;   // no leaf row in this tile
        const int k = a.tile_k[tile];
        const int32_t *__restrict__ nt = a.Nt + a.tile_off[tile];
        for (int r0 = 0; r0 < 8; ++r0) {
            const int ra = r0 + 16 * half, rb = ra + 8;
            const int32_t la = chk(rl[ra], -1, a.nslots, -1, a.status), lb = chk(rl[rb], -1, a.nslots, -1, a.status);
            if (la < 0 && lb < 0) continue;                     // the whole half-warp agrees
            const int64_t na = chk(a.row_node[tile * kTileRows + ra], -1, a.nB / a.B, 0, a.status);
            const int64_t nb = chk(a.row_node[tile * kTileRows + rb], -1, a.nB / a.B, 0, a.status);
            for (int64_t bp = cp; bp < B2; bp += 16) {
                const ulonglong2 *__restrict__ Qb = Q + bp;
                Acc2 x{0ull, 0ull}, y{0ull, 0ull};
                pair_rows_sum2<NARROW>(nt, ra, rb, k, Qb, B2, B2u, a.nslots, a.status, x, y);
                f32x2 sh, sl;
                ulonglong2 r;
                if (la >= 0) {
                    two_sum2(x.s, x.e, sh, sl);
                    const int64_t i = na * B + 2 * bp;
                    dw_add2(*reinterpret_cast<const f32x2 *>(g + i), *reinterpret_cast<const f32x2 *>(g + a.nB + i),
                            f2_neg(sh), f2_neg(sl), r.x, r.y);
                    Q[(int64_t)la * B2 + bp] = r;
                }
                if (lb >= 0) {
                    two_sum2(y.s, y.e, sh, sl);
                    const int64_t i = nb * B + 2 * bp;
                    dw_add2(*reinterpret_cast<const f32x2 *>(g + i), *reinterpret_cast<const f32x2 *>(g + a.nB + i),
                            f2_neg(sh), f2_neg(sl), r.x, r.y);
                    Q[(int64_t)lb * B2 + bp] = r;
                }
            }
        }
    }
}

// V^-1 (Sec. 3): f(x) = y'(x) - y'(next(x)), slot s - 1 being next(x) on the same
// chain or the chain's zero slot. DWQ: from the double-word copies (F32C, U-level
// schedule), in double-word arithmetic.
template <class M, bool DWQ>
__global__ void k_mob_diff(const int32_t *__restrict__ slot_node, int64_t nslots, int32_t B,
                           const unsigned long long *__restrict__ P, const unsigned char *__restrict__ esc,
                           const float2 *__restrict__ Q, bool pair_q, void *f, int64_t nB, uint32_t *status) {
    const int64_t total = nslots * B;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / B;
        const int32_t node = chk(slot_node[s], -1, nB / B, -1, status);
        if (node < 0) continue;
        const int64_t bl = i - s * B;
        const int64_t o = (int64_t)node * B + bl;
        if constexpr (DWQ) {
            const float2 y = dwq_load(Q, i, pair_q), yp = dwq_load(Q, i - B, pair_q);
            const DW r = dw_add({y.x, y.y}, {-yp.x, -yp.y});
            float *q = reinterpret_cast<float *>(f);
            q[o] = r.hi;
            q[nB + o] = r.lo;
        } else {
            const typename M::T y = decode<M>(P[i], esc + i);
            const typename M::T yp = decode<M>(P[i - B], esc + i - B);
            M::store_out(f, o, nB, M::sub(y, yp));
        }
    }
}

// Marks the slots read by a row of another chain: the rows of the forward substitution.
__global__ void k_mark_referenced(const int32_t *__restrict__ Nt, const int64_t *__restrict__ tile_off,
                                  const int32_t *__restrict__ tile_k, const int32_t *__restrict__ row_node,
                                  int64_t ntiles, const int32_t *__restrict__ node_slot,
                                  const int32_t *__restrict__ slot_node, uint8_t *__restrict__ slot_ref) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t tile = warp; tile < ntiles; tile += nwarps) {
        const int32_t x = row_node[tile * kTileRows + lane];
        if (x < 0) continue;
        const int32_t own = node_slot[x];
        const int32_t *np = Nt + tile_off[tile] + lane;
        for (int c = 0, k = tile_k[tile]; c < k; ++c) {
            const int32_t s = np[(int64_t)c * kTileRows];
            if (s != own && slot_node[s] >= 0) slot_ref[s] = 1;
        }
    }
}

// ---------------------------------------------------------------- launchers
ScanShape scan_shape(int64_t nslots, int32_t B) {
    ScanShape sh;
    sh.BW = B < 32 ? B : 32;
    sh.R = kScanThreads / sh.BW;
    sh.groups = (B + sh.BW - 1) / sh.BW;
    sh.tile_slots = (int64_t)sh.R * kScanSeg;
    sh.ntiles = (nslots + sh.tile_slots - 1) / sh.tile_slots;
    return sh;
}

template <class Pol>
static cudaError_t launch_scan_t(const ScanArgs &a, const ScanShape &sh, cudaStream_t st) {
    dim3 grid((unsigned)sh.ntiles, (unsigned)sh.groups);
    ScanArgs args = a;
    args.pair_words = std::is_same<Pol, PolF32C>::value && f32c_pair_words(a.B);
    k_chain_scan<Pol><<<grid, kScanThreads, 0, st>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_scan(int dtype, const ScanArgs &a, const ScanShape &sh, cudaStream_t st) {
    switch (dtype) {
        case MZ_I64: return launch_scan_t<PolI64>(a, sh, st);
        case MZ_F64: return launch_scan_t<PolF64>(a, sh, st);
        default: return launch_scan_t<PolF32C>(a, sh, st);
    }
}

template <class Pol>
static cudaError_t launch_gather_t(const GatherArgs &a, int num_sms, cudaStream_t st) {
    const int warps_per_block = kGatherThreads / 32;
    int64_t blocks = (a.ntiles + warps_per_block - 1) / warps_per_block;
    blocks = std::min<int64_t>(blocks, (int64_t)num_sms * std::max(1, a.blocks_per_sm));
    if (a.B == 1) {
        k_niv_gather<Pol, 1><<<dim3((unsigned)blocks, 1), kGatherThreads, 0, st>>>(a);
    } else if ((a.B & (a.B - 1)) == 0) {
        const int G = a.B < 32 ? a.B : 32;
        const dim3 grid((unsigned)blocks, 1);
        const bool narrow = a.nslots * (int64_t)a.B <= (int64_t)0xffffffffll;
#define MZ_GATHER_B(g)                                                                   \
    (narrow ? k_niv_gather_b<Pol, g, true><<<grid, kGatherThreads, 0, st>>>(a)             \
            : k_niv_gather_b<Pol, g, false><<<grid, kGatherThreads, 0, st>>>(a))
        if (G == 32) {               // B a multiple of 32: two columns per lane
            if constexpr (std::is_same<Pol, PolF32C>::value) {   // prefixes in column pairs (f32c_pair_words)
                if (narrow) k_niv_gather_h2<true><<<grid, kGatherThreads, 0, st>>>(a);
                else k_niv_gather_h2<false><<<grid, kGatherThreads, 0, st>>>(a);
            } else {
                if (narrow) k_niv_gather_h<Pol, true><<<grid, kGatherThreads, 0, st>>>(a);
                else k_niv_gather_h<Pol, false><<<grid, kGatherThreads, 0, st>>>(a);
            }
            return cudaGetLastError();
        }
        switch (G) {
            case 2: MZ_GATHER_B(2); break;
            case 4: MZ_GATHER_B(4); break;
            case 8: MZ_GATHER_B(8); break;
            case 16: MZ_GATHER_B(16); break;
            default: MZ_GATHER_B(32); break;
        }
#undef MZ_GATHER_B
    } else {
        const unsigned gy = (unsigned)((a.B + 3) / 4);
        k_niv_gather<Pol, 4><<<dim3((unsigned)blocks, gy), kGatherThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(int dtype, const GatherArgs &a, int num_sms, cudaStream_t st) {
    switch (dtype) {
        case MZ_I64: return launch_gather_t<PolI64>(a, num_sms, st);
        case MZ_F64: return launch_gather_t<PolF64>(a, num_sms, st);
        default: return launch_gather_t<PolF32C>(a, num_sms, st);
    }
}

template <class L, class M>
static cudaError_t launch_leaf_t(const MobArgs &a, int64_t nslots, int num_sms, cudaStream_t st) {
    const int warps_per_block = kGatherThreads / 32;
    int64_t blocks = (a.ntiles + warps_per_block - 1) / warps_per_block;
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms * std::max(1, a.gather_blocks_per_sm)));
    if (a.B == 1) {
        k_mob_leaf<L, M, 1><<<dim3((unsigned)blocks, 1), kGatherThreads, 0, st>>>(a);
    } else if ((a.B & (a.B - 1)) == 0) {
        const int G = a.B < 32 ? a.B : 32;
        const dim3 grid((unsigned)blocks, 1);
        const bool narrow = nslots * (int64_t)a.B <= (int64_t)0xffffffffll;
#define MZ_LEAF_B(g)                                                                     \
    (narrow ? k_mob_leaf_b<L, M, g, true><<<grid, kGatherThreads, 0, st>>>(a)              \
            : k_mob_leaf_b<L, M, g, false><<<grid, kGatherThreads, 0, st>>>(a))
        if constexpr (M::kDW) {
            if (a.pair_q) {         // Q in column pairs: the packed compensated gather
                if (narrow) k_mob_leaf_h2<true><<<grid, kGatherThreads, 0, st>>>(a);
                else k_mob_leaf_h2<false><<<grid, kGatherThreads, 0, st>>>(a);
                return cudaGetLastError();
            }
        }
        switch (G) {
            case 2: MZ_LEAF_B(2); break;
            case 4: MZ_LEAF_B(4); break;
            case 8: MZ_LEAF_B(8); break;
            case 16: MZ_LEAF_B(16); break;
            default: MZ_LEAF_B(32); break;
        }
#undef MZ_LEAF_B
    } else {
        const unsigned gy = (unsigned)((a.B + 3) / 4);
        k_mob_leaf<L, M, 4><<<dim3((unsigned)blocks, gy), kGatherThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

// Moebius launches. U-level schedule: init, forward substitution over the referenced
// rows, leaf gather over the others, V^-1 (4 launches). Antichain schedule: init and
// the forward substitution, which writes f itself (2 launches).
template <class M, class L>
static cudaError_t launch_mobius_t(const MobArgs &a, const int32_t *slot_node, int64_t nslots, bool anti,
                                   int num_sms, cudaStream_t st, int *launches) {
    const int64_t total = nslots * a.B;
    const unsigned eblocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 16));
    const bool dwq = M::kDW && !anti;      // F32C, U-level schedule: double-word copies for the later stages
    float2 *Q = dwq ? a.Q : nullptr;
    k_mob_init<M><<<eblocks, 256, 0, st>>>(slot_node, anti ? nullptr : a.slot_ref, nslots, a.B, a.P, a.esc, Q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mark_event(++*launches, st);
    // persistent wavefront: every block resident (cooperative launch)
    void *fn;
    int threads = 256;
    // rows per thread group: G = 1 for one function, G = min(B, 32) for a power-of-two batch
    const bool pow2 = (a.B & (a.B - 1)) == 0;
    const bool per_thread = pow2 && (int64_t)a.B * nslots < ((int64_t)1 << 31);
    int G = 1;
    const bool lanes = per_thread && a.B == 1 && !anti;   // one function: LR lanes per row
    if (lanes) {
        threads = 128;
        G = a.lanes;
        switch (G) {
            case 1: fn = (void *)k_mob_wave_lr<M, 1>; break;
            case 2: fn = (void *)k_mob_wave_lr<M, 2>; break;
            case 8: fn = (void *)k_mob_wave_lr<M, 8>; break;
            case 16: fn = (void *)k_mob_wave_lr<M, 16>; break;
            case 32: fn = (void *)k_mob_wave_lr<M, 32>; break;
            default: G = 4; fn = (void *)k_mob_wave_lr<M, 4>; break;
        }
    } else if (per_thread) {
        threads = 128;
        G = a.B < 32 ? a.B : 32;
#define MZ_WAVE_G(g) (anti ? (void *)k_mob_wave_t<M, true, g> : (void *)k_mob_wave_t<M, false, g>)
        switch (G) {
            case 1: fn = MZ_WAVE_G(1); break;
            case 2: fn = MZ_WAVE_G(2); break;
            case 4: fn = MZ_WAVE_G(4); break;
            case 8: fn = MZ_WAVE_G(8); break;
            case 16: fn = MZ_WAVE_G(16); break;
            default: fn = MZ_WAVE_G(32); break;
        }
#undef MZ_WAVE_G
    } else {
        fn = anti ? (void *)k_mob_wave<M, true> : (void *)k_mob_wave<M, false>;
    }
    MobArgs args = a;
    args.Q = Q;
    args.pair_q = dwq && f32c_pair_words(a.B);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
    if (e != cudaSuccess) return e;
    // One thread per row: enough resident threads for several levels of rows in
    // flight, few enough that the threads waiting ahead of the frontier do not
    // flood L2 with polls.
    int64_t blocks = (int64_t)std::max(1, per_sm) * num_sms;
    if (per_thread) blocks = std::min<int64_t>(blocks, (int64_t)std::max(1, a.blocks_per_sm) * G * num_sms);
    const int64_t rows_per_block = per_thread ? threads / G : threads / 32;
    blocks = std::min<int64_t>(blocks, (a.n + rows_per_block - 1) / rows_per_block);
    blocks = std::max<int64_t>(blocks, 1);
    void *params[] = {&args};
    e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)blocks), dim3(threads), params, 0, st);
    if (e != cudaSuccess) return e;
    mark_event(++*launches, st);
    if (!anti) {
        if ((e = launch_leaf_t<L, M>(args, nslots, num_sms, st)) != cudaSuccess) return e;
        mark_event(++*launches, st);
        if (dwq)
            k_mob_diff<M, true><<<eblocks, 256, 0, st>>>(slot_node, nslots, a.B, a.P, a.esc, Q, args.pair_q != 0,
                                                        a.f, a.nB, a.status);
        else
            k_mob_diff<M, false><<<eblocks, 256, 0, st>>>(slot_node, nslots, a.B, a.P, a.esc, nullptr, false, a.f,
                                                         a.nB, a.status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        mark_event(++*launches, st);
    }
    return cudaSuccess;
}

cudaError_t launch_mobius(int dtype, const MobArgs &a, const int32_t *slot_node, int64_t nslots, bool anti,
                          int num_sms, cudaStream_t st, int *launches) {
    switch (dtype) {
        case MZ_I64: return launch_mobius_t<MobI64, LeafI64>(a, slot_node, nslots, anti, num_sms, st, launches);
        case MZ_F64: return launch_mobius_t<MobF64, LeafF64>(a, slot_node, nslots, anti, num_sms, st, launches);
        default: return launch_mobius_t<MobF32C, LeafF32C>(a, slot_node, nslots, anti, num_sms, st, launches);
    }
}

cudaError_t launch_mark_referenced(const int32_t *Nt, const int64_t *tile_off, const int32_t *tile_k,
                                   const int32_t *row_node, int64_t ntiles, const int32_t *node_slot,
                                   const int32_t *slot_node, uint8_t *slot_ref, int num_sms, cudaStream_t st) {
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((ntiles + 7) / 8, (int64_t)num_sms * 16));
    k_mark_referenced<<<(unsigned)blocks, 256, 0, st>>>(Nt, tile_off, tile_k, row_node, ntiles, node_slot, slot_node,
                                                        slot_ref);
    return cudaGetLastError();
}

}  // namespace mz
