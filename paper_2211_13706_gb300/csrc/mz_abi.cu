// The C ABI of include/mz.h: plan build and upload, workspace layout, and the
// transform entry points (argument checks, then kernel launches on the
// caller's stream). Every transform runs on the GPU; there is no host path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <atomic>
#include <mutex>
#include <thread>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>   // header-only; the ranges cost nothing unless a profiler is attached

#include "mz_internal.h"
#include "mz_kernels.h"

namespace mz {

static thread_local std::string g_last_error;
static thread_local int g_last_launches = 0;
static thread_local void *const *g_events = nullptr;
static thread_local int32_t g_event_cap = 0;

// profiling hook: events[i] after the i-th launch of the current call (events[0] before it)
void mark_event(int i, cudaStream_t s) {
    if (g_events && i < g_event_cap && g_events[i]) cudaEventRecord((cudaEvent_t)g_events[i], s);
}

void set_last_error(const std::string &s) { g_last_error = s; }

static mz_status cuda_fail(cudaError_t e, const char *what) {
    set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    return MZ_ERR_CUDA;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// An NVTX range over a scope: the build's phases and every transform call show up by
// name on a profiler's host timeline (Nsight Systems, ncu --nvtx).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---------------------------------------------------------------- device memory of a plan
static void *plan_alloc(mz_plan *p, size_t bytes) {
    void *ptr = nullptr;
    bytes = align256(std::max<size_t>(bytes, 256));
    if (p->dev_alloc) {
        ptr = p->dev_alloc(bytes, p->alloc_ctx);
    } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr) {
        p->allocations.push_back(ptr);
        p->device_bytes += (int64_t)bytes;
    }
    return ptr;
}

static void plan_free_all(mz_plan *p) {
    if (!p->allocations.empty()) cudaDeviceSynchronize();
    for (void *ptr : p->allocations) {
        if (p->dev_free) p->dev_free(ptr, p->alloc_ctx);
        else cudaFree(ptr);
    }
    p->allocations.clear();
}

template <class T>
static mz_status upload(mz_plan *p, T **dst, const T *src, size_t count) {
    *dst = (T *)plan_alloc(p, sizeof(T) * count);
    if (!*dst) {
        set_last_error("device allocation failed");
        return MZ_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    return MZ_OK;
}

// Runs fn(begin, end) over [0, count) split into contiguous pieces on the host's threads.
template <class F>
static void parallel_for(int64_t count, F fn) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int64_t pieces = std::min<int64_t>(hw, std::max<int64_t>(1, count / 4096));
    if (pieces <= 1) {
        fn((int64_t)0, count);
        return;
    }
    std::vector<std::thread> pool;
    for (int64_t t = 0; t < pieces; ++t)
        pool.emplace_back([&, t]() { fn(count * t / pieces, count * (t + 1) / pieces); });
    for (auto &th : pool) th.join();
}

// Row order of the gather's tiles for a sparse map: rows by length, longest first (ties
// in row order), so that a tile is about as wide as each of its rows. In slot order the
// rows of the paper's random DAGs differ so much in length that padding the tiles to
// their longest row reads 7-8 times nnz(N). The dense map keeps slot order.
static std::vector<int32_t> sparse_tile_order(const int32_t *len, int64_t n) {
    int32_t maxlen = 0;
    for (int64_t r = 0; r < n; ++r) maxlen = std::max(maxlen, len[r]);
    std::vector<int64_t> start((size_t)maxlen + 2, 0);
    for (int64_t r = 0; r < n; ++r) start[(size_t)(maxlen - len[r]) + 1]++;
    for (size_t l = 1; l < start.size(); ++l) start[l] += start[l - 1];
    std::vector<int32_t> order((size_t)n);
    for (int64_t r = 0; r < n; ++r) order[(size_t)start[(size_t)(maxlen - len[r])]++] = (int32_t)r;
    return order;
}

// Device layouts of one side (all components): the concatenated slot map, the
// tiled niv map for the zeta gather, and the map in Moebius processing order.
static mz_status upload_side(mz_plan *p, int side) {
    const std::vector<HostSide> &Hs = p->host[side];
    DeviceSide &D = p->dev[side];
    const size_t C = Hs.size();
    D.n = p->n_total();
    D.nslots = p->slots_total();
    D.k_max = 0;
    D.kpad_max = 0;
    for (const HostSide &H : Hs) {
        D.k_max = std::max(D.k_max, H.k);
        D.kpad_max = std::max<int32_t>(D.kpad_max, (H.k + 15) / 16 * 16);
    }
    mz_status st;
    {   // slot map, padded with -1 to a multiple of 64 entries (the scan reads 16-byte vectors)
        std::vector<int32_t> sn(((size_t)D.nslots + 63) / 64 * 64, -1);
        for (size_t c = 0; c < C; ++c)
            for (size_t q = 0; q < Hs[c].slot_node.size(); ++q) {
                const int32_t v = Hs[c].slot_node[q];
                sn[p->slot_off[c] + q] = v < 0 ? -1 : (int32_t)(v + p->node_off[c]);
            }
        if ((st = upload(p, &D.slot_node, sn.data(), sn.size()))) return st;
    }
    // U-level schedule: the slots some row of another chain reads (an entry of another
    // chain in its niv row). Only their rows go through the forward substitution; every
    // other row is read by no row and is computed afterwards by the leaf gather.
    const bool anti = (p->schedule == MZ_SCHED_ANTICHAIN);
    std::vector<uint8_t> ref;
    if (!anti) {
        std::unique_ptr<std::atomic<uint8_t>[]> refa(new std::atomic<uint8_t>[(size_t)D.nslots]());
        parallel_for((int64_t)C == 1 ? Hs[0].n : (int64_t)C, [&](int64_t lo, int64_t hi) {
            const bool rows = (C == 1);
            for (int64_t u = lo; u < hi; ++u) {
                const size_t c = rows ? 0 : (size_t)u;
                const HostSide &H = Hs[c];
                const int64_t so = p->slot_off[c];
                for (int64_t r = rows ? u : 0, r1 = rows ? u + 1 : H.n; r < r1; ++r) {
                    const int32_t cx = H.chain_id[H.row_node[r]];
                    H.for_row(r, [&](int32_t ch, int32_t slot) {
                        if (ch != cx) refa[(size_t)(so + slot)].store(1, std::memory_order_relaxed);
                    });
                }
            }
        });
        ref.resize((size_t)D.nslots);
        for (size_t q = 0; q < ref.size(); ++q) ref[q] = refa[q].load(std::memory_order_relaxed);
        if ((st = upload(p, &D.slot_ref, ref.data(), ref.size()))) return st;
    }
    {   // tiles of 32 rows per component, column-major inside a tile
        std::vector<int64_t> toff;
        std::vector<int32_t> tk;
        // rows at the tile positions of each sparse component (dense: position = row)
        std::vector<std::vector<int32_t>> order(C);
        for (size_t c = 0; c < C; ++c)
            if (Hs[c].sparse) order[c] = sparse_tile_order(Hs[c].row_len.data(), Hs[c].n);
        size_t total = 0;
        for (size_t c = 0; c < C; ++c) {
            const HostSide &H = Hs[c];
            const int64_t nt = (H.n + kTileRows - 1) / kTileRows;
            for (int64_t t = 0; t < nt; ++t) {
                // dense: all k columns; sparse: as many as the tile's longest row, padded
                int32_t kt = H.k;
                if (H.sparse) {
                    kt = 1;
                    for (int64_t q = t * kTileRows; q < std::min<int64_t>(H.n, (t + 1) * kTileRows); ++q)
                        kt = std::max(kt, H.row_len[order[c][q]]);
                }
                toff.push_back((int64_t)total);
                tk.push_back(kt);
                total += (size_t)kt * kTileRows;
            }
        }
        D.ntiles = (int64_t)toff.size();
        std::vector<int32_t> tiled, rn((size_t)D.ntiles * kTileRows, -1), rl;
        if (!anti) rl.assign((size_t)D.ntiles * kTileRows, -1);
        try {
            tiled.assign(total, 0);   // padding rows read slot 0, a zero slot
        } catch (...) {
            set_last_error("host allocation failed");
            return MZ_ERR_OOM;
        }
        std::vector<int64_t> tile0(C + 1, 0);   // first tile of each component
        for (size_t c = 0; c < C; ++c) tile0[c + 1] = tile0[c] + (Hs[c].n + kTileRows - 1) / kTileRows;
        parallel_for((int64_t)C == 1 ? Hs[0].n : (int64_t)C, [&](int64_t lo, int64_t hi) {
            // one poset: split its rows; many posets: split the posets
            const bool rows = (C == 1);
            for (int64_t u = lo; u < hi; ++u) {
                const size_t c = rows ? 0 : (size_t)u;
                const HostSide &H = Hs[c];
                const int64_t k = H.k;
                const int32_t so = (int32_t)p->slot_off[c];
                const int64_t q0 = rows ? u : 0, q1 = rows ? u + 1 : H.n;
                for (int64_t q0i = q0; q0i < q1; ++q0i) {
                    const int64_t r = H.sparse ? order[c][q0i] : q0i;    // the row at tile position q0i
                    const int64_t t = tile0[c] + q0i / kTileRows, lane = q0i % kTileRows;
                    int32_t *dst = &tiled[(size_t)toff[t] + lane];
                    if (H.sparse) {           // finite entries only; the rest stay slot 0 (a zero slot)
                        int64_t q = 0;
                        H.for_row(r, [&](int32_t, int32_t slot) { dst[(q++) * kTileRows] = slot + so; });
                    } else {
                        const int32_t *row = &H.N[(size_t)r * k];
                        for (int64_t q = 0; q < k; ++q) dst[q * kTileRows] = row[q] + so;
                    }
                    rn[(size_t)t * kTileRows + lane] = (int32_t)(H.row_node[r] + p->node_off[c]);
                    if (!anti) {
                        const int32_t gs = H.node_slot[H.row_node[r]] + so;
                        rl[(size_t)t * kTileRows + lane] = ref[(size_t)gs] ? -1 : gs;
                    }
                }
            }
        });
        if ((st = upload(p, &D.Nt, tiled.data(), tiled.size()))) return st;
        if (!anti && (st = upload(p, &D.row_leaf, rl.data(), rl.size()))) return st;
        if ((st = upload(p, &D.tile_off, toff.data(), toff.size()))) return st;
        if ((st = upload(p, &D.tile_k, tk.data(), tk.size()))) return st;
        if ((st = upload(p, &D.row_node, rn.data(), rn.size()))) return st;
    }
    {   // Moebius rows: all components in one order, by level, then component, then row;
        // the U-level schedule keeps only the referenced rows
        int32_t maxlvl = 0;
        for (const HostSide &H : Hs) maxlvl = std::max(maxlvl, anti ? H.nlevels : H.nulevels);
        auto in_schedule = [&](size_t c, int64_t r) {
            return anti || ref[(size_t)(Hs[c].node_slot[Hs[c].row_node[r]] + p->slot_off[c])] != 0;
        };
        std::vector<int64_t> cnt((size_t)maxlvl + 2, 0);
        for (size_t c = 0; c < C; ++c) {
            const HostSide &H = Hs[c];
            for (int64_t r = 0; r < H.n; ++r)
                if (in_schedule(c, r)) cnt[(anti ? H.level : H.ulevel)[H.row_node[r]] + 1]++;
        }
        for (size_t l = 1; l < cnt.size(); ++l) cnt[l] += cnt[l - 1];
        D.nmob = cnt.back();
        std::vector<std::pair<int32_t, int32_t>> order((size_t)D.nmob);   // (component, row)
        for (size_t c = 0; c < C; ++c) {
            const HostSide &H = Hs[c];
            const std::vector<int32_t> &lvl = anti ? H.level : H.ulevel;
            for (int64_t r = 0; r < H.n; ++r)
                if (in_schedule(c, r)) order[(size_t)cnt[lvl[H.row_node[r]]]++] = {(int32_t)c, (int32_t)r};
        }
        std::vector<int64_t> moff((size_t)D.nmob);
        std::vector<int32_t> mkp((size_t)D.nmob), mnode((size_t)D.nmob), mslot((size_t)D.nmob), mlevel((size_t)D.nmob);
        std::vector<int64_t> ment((size_t)D.nmob);
        // A row holds the finite entries of the other chains (the own chain and the
        // infinite entries add nothing), padded in front to a multiple of 16, at least 16.
        parallel_for((int64_t)order.size(), [&](int64_t lo, int64_t hi) {
            for (int64_t i = lo; i < hi; ++i) {
                const HostSide &H = Hs[order[i].first];
                const int64_t cnt = H.row_count(order[i].second) - 1;   // minus the own chain
                mkp[i] = (int32_t)std::max<int64_t>(16, (cnt + 15) / 16 * 16);
                ment[i] = cnt;
            }
        });
        size_t total = 0;
        D.nmob_entries = 0;
        D.mob_kp_max = 0;
        for (size_t i = 0; i < order.size(); ++i) {
            moff[i] = (int64_t)total;
            total += (size_t)mkp[i];
            D.nmob_entries += ment[i];
            D.mob_kp_max = std::max(D.mob_kp_max, mkp[i]);
        }
        std::vector<int32_t> Nm;
        try {
            Nm.assign(total, 0);      // padding in front of each row reads slot 0, a zero slot
        } catch (...) {
            set_last_error("host allocation failed");
            return MZ_ERR_OOM;
        }
        // Each row lists its slots ordered by the level of the element in them (zero
        // slots first): the kernel adds the latest-finishing ones last.
        parallel_for((int64_t)order.size(), [&](int64_t lo, int64_t hi) {
            std::vector<std::pair<int32_t, int32_t>> cols;
            for (int64_t i = lo; i < hi; ++i) {
                const size_t c = (size_t)order[i].first;
                const int64_t r = order[i].second;
                const HostSide &H = Hs[c];
                const std::vector<int32_t> &lvl = anti ? H.level : H.ulevel;
                const int32_t x = H.row_node[r];
                const int32_t cx = H.chain_id[x];
                cols.clear();
                H.for_row(r, [&](int32_t ch, int32_t slot) {
                    if (ch != cx) cols.push_back({lvl[H.slot_node[slot]], slot + (int32_t)p->slot_off[c]});
                });
                std::stable_sort(cols.begin(), cols.end(),
                                 [](const std::pair<int32_t, int32_t> &a, const std::pair<int32_t, int32_t> &b) {
                                     return a.first < b.first;
                                 });
                int32_t *dst = &Nm[(size_t)moff[i] + (mkp[i] - (int64_t)cols.size())];
                for (size_t q = 0; q < cols.size(); ++q) dst[q] = cols[q].second;
                mnode[i] = (int32_t)(x + p->node_off[c]);
                mslot[i] = (int32_t)(H.node_slot[x] + p->slot_off[c]);
                mlevel[i] = lvl[x];
            }
        });
        if ((st = upload(p, &D.Nm, Nm.data(), Nm.size()))) return st;
        if ((st = upload(p, &D.mob_off, moff.data(), moff.size()))) return st;
        if ((st = upload(p, &D.mob_kp, mkp.data(), mkp.size()))) return st;
        if ((st = upload(p, &D.mob_node, mnode.data(), mnode.size()))) return st;
        if ((st = upload(p, &D.mob_slot, mslot.data(), mslot.size()))) return st;
        if ((st = upload(p, &D.mob_level, mlevel.data(), mlevel.size()))) return st;
    }
    return MZ_OK;
}

// Device memory held only while a plan is built; freed (after the device is idle)
// when the build returns, through the caller's allocator if it gave one.
class BuildScratch {
  public:
    explicit BuildScratch(mz_plan *p) : p_(p) {}
    BuildScratch(const BuildScratch &) = delete;
    BuildScratch &operator=(const BuildScratch &) = delete;
    ~BuildScratch() {
        if (!bufs_.empty()) cudaDeviceSynchronize();
        for (void *q : bufs_) {
            if (p_->dev_free) p_->dev_free(q, p_->alloc_ctx);
            else cudaFree(q);
        }
    }
    template <class T>
    T *get(size_t count) {
        void *q = nullptr;
        const size_t bytes = align256(std::max<size_t>(sizeof(T) * count, 256));
        if (p_->dev_alloc) {
            q = p_->dev_alloc(bytes, p_->alloc_ctx);
        } else if (cudaMalloc(&q, bytes) != cudaSuccess) {
            cudaGetLastError();
            q = nullptr;
        }
        if (q) bufs_.push_back(q);
        return (T *)q;
    }
    // Frees one buffer before the build ends (after the device is idle).
    void release(void *q) {
        auto it = std::find(bufs_.begin(), bufs_.end(), q);
        if (it == bufs_.end()) return;
        cudaDeviceSynchronize();
        if (p_->dev_free) p_->dev_free(q, p_->alloc_ctx);
        else cudaFree(q);
        bufs_.erase(it);
    }
    template <class T>
    mz_status put(T **dst, const T *src, size_t count) {
        *dst = get<T>(count);
        if (!*dst) {
            set_last_error("device allocation failed");
            return MZ_ERR_OOM;
        }
        if (count == 0) return MZ_OK;
        cudaError_t e = cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice);
        return e == cudaSuccess ? MZ_OK : cuda_fail(e, "cudaMemcpy");
    }

  private:
    mz_plan *p_;
    std::vector<void *> bufs_;
};

// Alg. 1's maximum matching on the device (mz_build_opts::device_build = 2, no chains
// given): next[u] = the node matched below u, or -1. The kernels of mz_build.cu do the
// work; the host only sequences the launches and reads the counters between levels.
// The result is checked on the host (every matched pair is an edge, no node matched
// twice) before it is used.
static mz_status device_matching(mz_plan *p, int64_t n, const std::vector<int64_t> &ptr,
                                 const std::vector<int32_t> &adj, std::vector<int32_t> &next, std::string &err) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        err = std::string("device matching: ") + cudaGetErrorString(e);
        return MZ_ERR_CUDA;
    }
    BuildScratch tmp(p);
    int64_t *d_ptr;
    int32_t *d_adj;
    mz_status st;
    if ((st = tmp.put(&d_ptr, ptr.data(), ptr.size())) || (st = tmp.put(&d_adj, adj.data(), adj.size()))) {
        err = "device matching: " + std::string(mz_last_error());
        return st;
    }
    int32_t *mu = tmp.get<int32_t>(n), *mv = tmp.get<int32_t>(n), *parent = tmp.get<int32_t>(n);
    int32_t *root = tmp.get<int32_t>(n), *fa = tmp.get<int32_t>(n), *fb = tmp.get<int32_t>(n);
    int32_t *ends = tmp.get<int32_t>(n);
    uint32_t *done = tmp.get<uint32_t>(n), *flags = tmp.get<uint32_t>(4);
    unsigned long long *counts = tmp.get<unsigned long long>(4);
    if (!mu || !mv || !parent || !root || !fa || !fb || !ends || !done || !flags || !counts) {
        err = "device allocation failed";
        return MZ_ERR_OOM;
    }
    auto fail = [&](cudaError_t ce, const char *what) {
        err = std::string("device matching: ") + what + ": " + cudaGetErrorString(ce);
        return MZ_ERR_CUDA;
    };
    const size_t nb = sizeof(int32_t) * (size_t)n;
    if ((e = cudaMemset(mu, 0xff, nb)) != cudaSuccess || (e = cudaMemset(mv, 0xff, nb)) != cudaSuccess ||
        (e = cudaMemset(flags, 0, 16)) != cudaSuccess)
        return fail(e, "cudaMemset");
    // greedy start: rounds until no free upper node wins a free child (bounded)
    for (int round = 0; round < 64; ++round) {
        uint32_t changed = 0;
        if ((e = cudaMemset(flags, 0, 4)) != cudaSuccess) return fail(e, "cudaMemset");
        if ((e = launch_match_greedy(d_ptr, d_adj, n, mu, mv, flags, sms, 0)) != cudaSuccess)
            return fail(e, "greedy launch");
        if ((e = cudaMemcpy(&changed, flags, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return fail(e, "cudaMemcpy");
        if (!changed) break;
    }
    // phases of augmenting paths; each flips at least one path, so at most n phases
    for (int64_t phase = 0; phase <= n; ++phase) {
        if ((e = cudaMemset(parent, 0xff, nb)) != cudaSuccess || (e = cudaMemset(done, 0, nb)) != cudaSuccess ||
            (e = cudaMemset(counts, 0, 32)) != cudaSuccess)
            return fail(e, "cudaMemset");
        if ((e = launch_match_roots(d_ptr, n, mu, root, fa, counts, sms, 0)) != cudaSuccess)
            return fail(e, "roots launch");
        unsigned long long c[4];
        if ((e = cudaMemcpy(c, counts, 32, cudaMemcpyDeviceToHost)) != cudaSuccess) return fail(e, "cudaMemcpy");
        int64_t fcount = (int64_t)c[0];
        int32_t *cur = fa, *nxt = fb;
        while (fcount > 0) {                 // one launch per level of the search forest
            if ((e = cudaMemset(counts + 1, 0, 8)) != cudaSuccess) return fail(e, "cudaMemset");
            if ((e = launch_match_expand(d_ptr, d_adj, cur, fcount, nxt, counts + 1, mu, mv, parent, root, done, ends,
                                         counts + 2, sms, 0)) != cudaSuccess)
                return fail(e, "search launch");
            if ((e = cudaMemcpy(c, counts, 32, cudaMemcpyDeviceToHost)) != cudaSuccess)
                return fail(e, "cudaMemcpy");
            fcount = (int64_t)c[1];
            std::swap(cur, nxt);
        }
        const int64_t found = (int64_t)c[2];
        if (found == 0) break;               // no augmenting path: the matching is maximum
        if ((e = launch_match_augment(ends, found, n, parent, mu, mv, flags + 1, sms, 0)) != cudaSuccess)
            return fail(e, "augment launch");
    }
    uint32_t status = 0;
    if ((e = cudaMemcpy(&status, flags + 1, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return fail(e, "cudaMemcpy");
    next.assign((size_t)n, -1);
    if ((e = cudaMemcpy(next.data(), mu, nb, cudaMemcpyDeviceToHost)) != cudaSuccess) return fail(e, "cudaMemcpy");
    // check: a matching of edges
    std::vector<char> below((size_t)n, 0);
    for (int64_t u = 0; u < n && status == 0; ++u) {
        const int32_t v = next[(size_t)u];
        if (v < 0) continue;
        if (v >= n || below[(size_t)v] || !std::binary_search(adj.begin() + ptr[u], adj.begin() + ptr[u + 1], v))
            status = MZ_ERR_CUDA;
        else
            below[(size_t)v] = 1;
    }
    if (status) {
        err = "device matching produced an invalid matching";
        return MZ_ERR_CUDA;
    }
    return MZ_OK;
}

// The same layouts as upload_side for a single poset whose niv map is built on the
// device (mz_build_opts::device_build): the host sends the children lists and the
// slot layout, the kernels of mz_build.cu build the map, the U levels, the tiles and
// the Moebius rows, and the host fills in the per-node arrays it keeps (U levels,
// nnz) and the O(n) orderings in between. Dense map: one dataflow launch over all
// nodes. Sparse map: one launch pair per height level.
static mz_status upload_side_device(mz_plan *p, int side) {
    HostSide &H = p->host[side][0];
    DeviceSide &D = p->dev[side];
    const int64_t n = H.n, k = H.k, nslots = n + k;
    const std::string who = side ? "dual: " : "";
    D.n = n;
    D.nslots = nslots;
    D.k_max = H.k;
    D.kpad_max = (H.k + 15) / 16 * 16;
    mz_status st;
    cudaError_t e;
    {   // slot map, padded with -1 to a multiple of 64 entries
        std::vector<int32_t> sn(((size_t)nslots + 63) / 64 * 64, -1);
        std::copy(H.slot_node.begin(), H.slot_node.end(), sn.begin());
        if ((st = upload(p, &D.slot_node, sn.data(), sn.size()))) return st;
    }
    BuildScratch tmp(p);
    // ---- inputs of the recurrence: nodes bottom-up by height
    std::vector<int32_t> order(n), topo_pos(n), base(k);
    std::vector<int64_t> level_start((size_t)H.nlevels + 2, 0);
    {
        for (int64_t x = 0; x < n; ++x) level_start[H.level[x]]++;
        for (size_t l = 1; l < level_start.size(); ++l) level_start[l] += level_start[l - 1];
        std::vector<int64_t> fill(level_start);
        for (int64_t i = n - 1; i >= 0; --i) order[(size_t)fill[H.level[H.topo[i]] - 1]++] = H.topo[i];
        for (int64_t i = 0; i < n; ++i) topo_pos[H.topo[i]] = (int32_t)i;
        for (int64_t c = 0; c < k; ++c) base[c] = (int32_t)H.chain_base[c];
    }
    int64_t *d_ptr;
    int32_t *d_adj, *d_order, *d_node_slot, *d_chain, *d_base, *d_pos;
    if ((st = tmp.put(&d_ptr, H.csr_ptr.data(), H.csr_ptr.size()))) return st;
    if ((st = tmp.put(&d_adj, H.csr_adj.data(), H.csr_adj.size()))) return st;
    if ((st = tmp.put(&d_order, order.data(), order.size()))) return st;
    if ((st = tmp.put(&d_node_slot, H.node_slot.data(), H.node_slot.size()))) return st;
    if ((st = tmp.put(&d_chain, H.chain_id.data(), H.chain_id.size()))) return st;
    if ((st = tmp.put(&d_base, base.data(), base.size()))) return st;
    if ((st = tmp.put(&d_pos, topo_pos.data(), topo_pos.size()))) return st;
    int32_t *d_uslot = tmp.get<int32_t>((size_t)nslots);
    int32_t *d_rowcnt = tmp.get<int32_t>((size_t)n);
    uint32_t *d_small = tmp.get<uint32_t>(64);   // ticket, status, bad, -, nnz / pool top (u64 at word 4)
    if (!d_uslot || !d_rowcnt || !d_small) {
        set_last_error("device allocation failed");
        return MZ_ERR_OOM;
    }
    const uint32_t small_init[6] = {0u, 0u, 0xffffffffu, 0u, 0u, 0u};
    if ((e = cudaMemset(d_uslot, 0xff, sizeof(int32_t) * nslots)) != cudaSuccess ||
        (e = cudaMemcpy(d_small, small_init, sizeof(small_init), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "build setup");
    unsigned long long *d_top = (unsigned long long *)(d_small + 4);
    auto read_small = [&](uint32_t *out6) -> mz_status {
        cudaError_t e2 = cudaMemcpy(out6, d_small, 6 * sizeof(uint32_t), cudaMemcpyDeviceToHost);
        return e2 == cudaSuccess ? MZ_OK : cuda_fail(e2, "niv build");
    };
    auto check_small = [&](const uint32_t *sm) -> mz_status {
        if (sm[1] == MZ_ERR_OOM) {
            set_last_error(who + "device build: the row pool overflowed");
            return MZ_ERR_OOM;
        }
        if (sm[1]) {
            set_last_error(who + "device build: a bounded wait ran out");
            return MZ_ERR_TIMEOUT;
        }
        if ((int32_t)sm[2] >= 0) {
            const int32_t x = H.topo[(int32_t)sm[2]];
            set_last_error(who + "chain " + std::to_string(H.chain_id[x]) + " is not totally ordered at node " +
                           std::to_string(x));
            return MZ_ERR_BAD_CHAINS;
        }
        return MZ_OK;
    };
    uint32_t small[6];
    int32_t *d_N = nullptr;                 // dense: [n][k]
    int64_t *d_row_beg = nullptr;           // sparse: rows in the pool
    int32_t *d_pool = nullptr;
    if (!H.sparse) {
        // ---- dense map: Thm. 4 as a dataflow over all nodes
        d_N = tmp.get<int32_t>((size_t)n * (size_t)k);
        uint32_t *d_ready = tmp.get<uint32_t>((size_t)n);
        if (!d_N || !d_ready) {
            set_last_error("device allocation failed");
            return MZ_ERR_OOM;
        }
        // the map starts at slot 0 everywhere, so that no read can leave the slot range
        if ((e = cudaMemset(d_N, 0, sizeof(int32_t) * (size_t)n * (size_t)k)) != cudaSuccess ||
            (e = cudaMemset(d_ready, 0, sizeof(uint32_t) * n)) != cudaSuccess)
            return cuda_fail(e, "build setup");
        BuildNivArgs a;
        std::memset(&a, 0, sizeof(a));
        a.ptr = d_ptr;
        a.adj = d_adj;
        a.order = d_order;
        a.node_slot = d_node_slot;
        a.chain_id = d_chain;
        a.base = d_base;
        a.topo_pos = d_pos;
        a.n = n;
        a.k = (int32_t)k;
        a.N = d_N;
        a.uslot = d_uslot;
        a.rowcnt = d_rowcnt;
        a.ready = d_ready;
        a.ticket = d_small;
        a.status = d_small + 1;
        a.bad = (int32_t *)(d_small + 2);
        a.nnz = d_top;
        a.spin_limit = p->spin_limit;
        if ((e = launch_build_niv(a, p->num_sms, 0)) != cudaSuccess) return cuda_fail(e, "niv build launch");
        if ((st = read_small(small)) || (st = check_small(small))) return st;
    } else {
        // ---- sparse map: one height level per launch pair
        std::vector<int32_t> slot_chain((size_t)nslots);
        for (int64_t c = 0; c < k; ++c)
            for (int64_t q = H.chain_base[c]; q < H.chain_base[c + 1]; ++q) slot_chain[q] = (int32_t)c;
        int32_t *d_slot_chain;
        if ((st = tmp.put(&d_slot_chain, slot_chain.data(), slot_chain.size()))) return st;
        d_row_beg = tmp.get<int64_t>((size_t)n);
        int64_t *d_cand_off = tmp.get<int64_t>((size_t)n + 1);
        if (!d_row_beg || !d_cand_off) {
            set_last_error("device allocation failed");
            return MZ_ERR_OOM;
        }
        int64_t pool_cap = 0, cand_cap = 0;
        unsigned long long *d_cand = nullptr;
        // grows a scratch buffer of the build; `keep` entries of the old one are copied over
        auto grow = [&](auto *&buf, int64_t &cap, int64_t need, int64_t keep) -> mz_status {
            if (need <= cap) return MZ_OK;
            using T = std::remove_reference_t<decltype(*buf)>;
            const int64_t ncap = std::max<int64_t>(need, cap + cap / 2);
            T *nb = tmp.get<T>((size_t)ncap);
            if (!nb) {
                set_last_error("device allocation failed");
                return MZ_ERR_OOM;
            }
            if (keep > 0) {
                cudaError_t e2 = cudaMemcpy(nb, buf, sizeof(T) * (size_t)keep, cudaMemcpyDeviceToDevice);
                if (e2 != cudaSuccess) return cuda_fail(e2, "cudaMemcpy");
            }
            if (buf) tmp.release(buf);
            buf = nb;
            cap = ncap;
            return MZ_OK;
        };
        if ((st = grow(d_pool, pool_cap, 4 * n + 1024, 0))) return st;
        SparseLevelArgs a;
        std::memset(&a, 0, sizeof(a));
        a.ptr = d_ptr;
        a.adj = d_adj;
        a.order = d_order;
        a.node_slot = d_node_slot;
        a.chain_id = d_chain;
        a.slot_chain = d_slot_chain;
        a.base = d_base;
        a.topo_pos = d_pos;
        a.row_beg = d_row_beg;
        a.row_len = d_rowcnt;
        a.pool_top = d_top;
        a.cand_off = d_cand_off;
        a.uslot = d_uslot;
        a.bad = (int32_t *)(d_small + 2);
        a.status = d_small + 1;
        for (int32_t h = 1; h <= H.nlevels; ++h) {
            a.lo = level_start[h - 1];
            a.cnt = level_start[h] - a.lo;
            if (a.cnt == 0) continue;
            if ((e = launch_sparse_bounds(a, p->num_sms, 0)) != cudaSuccess) return cuda_fail(e, "sparse build launch");
            int64_t total = 0;
            if ((e = cudaMemcpy(&total, d_cand_off + a.cnt, sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
                return cuda_fail(e, "sparse build");
            if ((st = read_small(small))) return st;
            const int64_t top = (int64_t)(small[4] | ((uint64_t)small[5] << 32));
            // every kept entry comes from a candidate: the level adds at most `total` entries
            if ((st = grow(d_cand, cand_cap, total, 0))) return st;
            if ((st = grow(d_pool, pool_cap, top + total, top))) return st;
            a.cand = d_cand;
            a.pool = d_pool;
            a.pool_cap = pool_cap;
            if ((e = launch_sparse_merge(a, p->num_sms, 0)) != cudaSuccess) return cuda_fail(e, "sparse build launch");
        }
        if ((st = read_small(small)) || (st = check_small(small))) return st;
    }
    H.nnz = (int64_t)(small[4] | ((uint64_t)small[5] << 32));
    std::vector<int32_t> uslot((size_t)nslots), rowcnt((size_t)n);
    if ((e = cudaMemcpy(uslot.data(), d_uslot, sizeof(int32_t) * nslots, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(rowcnt.data(), d_rowcnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy");
    H.ulevel.assign(n, 0);
    for (int64_t x = 0; x < n; ++x) H.ulevel[x] = uslot[H.node_slot[x]];
    H.nulevels = *std::max_element(H.ulevel.begin(), H.ulevel.end()) + 1;
    // ---- tiles of 32 rows for the gather
    std::vector<int32_t> rn_host;   // node of each tile row (-1: padding)
    {
        D.ntiles = (n + kTileRows - 1) / kTileRows;
        std::vector<int64_t> toff((size_t)D.ntiles);
        std::vector<int32_t> tk((size_t)D.ntiles, (int32_t)k), rn((size_t)D.ntiles * kTileRows, -1);
        std::vector<int32_t> order;   // sparse: the row at each tile position (as upload_side)
        if (H.sparse) order = sparse_tile_order(rowcnt.data(), n);
        int64_t total = 0;
        for (int64_t t = 0; t < D.ntiles; ++t) {
            if (H.sparse) {   // as many columns as the tile's longest row
                int32_t kt = 1;
                for (int64_t q = t * kTileRows; q < std::min<int64_t>(n, (t + 1) * kTileRows); ++q)
                    kt = std::max(kt, rowcnt[order[q]]);
                tk[t] = kt;
            }
            toff[t] = total;
            total += (int64_t)tk[t] * kTileRows;
        }
        for (int64_t q = 0; q < n; ++q) rn[q] = H.row_node[H.sparse ? order[q] : q];
        int32_t *d_order = nullptr;
        if (H.sparse && (st = tmp.put(&d_order, order.data(), order.size()))) return st;
        D.Nt = (int32_t *)plan_alloc(p, sizeof(int32_t) * (size_t)total);
        if (!D.Nt) {
            set_last_error("device allocation failed");
            return MZ_ERR_OOM;
        }
        if ((st = upload(p, &D.tile_off, toff.data(), toff.size()))) return st;
        if ((st = upload(p, &D.tile_k, tk.data(), tk.size()))) return st;
        if ((st = upload(p, &D.row_node, rn.data(), rn.size()))) return st;
        e = H.sparse ? launch_build_tiles_sparse(d_row_beg, d_rowcnt, d_pool, d_order, n, D.ntiles, D.tile_off,
                                                 D.tile_k, D.Nt, p->num_sms, 0)
                     : launch_build_tiles(d_N, n, (int32_t)k, D.Nt, p->num_sms, 0);
        if (e != cudaSuccess) return cuda_fail(e, "tile build launch");
        rn_host.swap(rn);
    }
    // ---- U-level schedule: the slots another chain's row reads (marked from the tiles);
    // only their rows go through the forward substitution, the others through the leaf gather
    const bool anti = (p->schedule == MZ_SCHED_ANTICHAIN);
    std::vector<uint8_t> ref;
    if (!anti) {
        D.slot_ref = (uint8_t *)plan_alloc(p, (size_t)nslots);
        if (!D.slot_ref) {
            set_last_error("device allocation failed");
            return MZ_ERR_OOM;
        }
        if ((e = cudaMemset(D.slot_ref, 0, (size_t)nslots)) != cudaSuccess) return cuda_fail(e, "cudaMemset");
        if ((e = launch_mark_referenced(D.Nt, D.tile_off, D.tile_k, D.row_node, D.ntiles, d_node_slot, D.slot_node,
                                        D.slot_ref, p->num_sms, 0)) != cudaSuccess)
            return cuda_fail(e, "reference marking launch");
        ref.resize((size_t)nslots);
        if ((e = cudaMemcpy(ref.data(), D.slot_ref, (size_t)nslots, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpy");
        std::vector<int32_t> rl(rn_host.size(), -1);
        for (size_t q = 0; q < rn_host.size(); ++q)
            if (rn_host[q] >= 0) {
                const int32_t gs = H.node_slot[rn_host[q]];
                rl[q] = ref[(size_t)gs] ? -1 : gs;
            }
        if ((st = upload(p, &D.row_leaf, rl.data(), rl.size()))) return st;
    }
    // ---- Moebius rows, by level of the schedule and then by row
    {
        const std::vector<int32_t> &lvl = anti ? H.level : H.ulevel;
        const int32_t maxlvl = anti ? H.nlevels : H.nulevels;
        auto in_schedule = [&](int64_t r) { return anti || ref[(size_t)H.node_slot[H.row_node[r]]] != 0; };
        std::vector<int64_t> cnt((size_t)maxlvl + 2, 0);
        for (int64_t r = 0; r < n; ++r)
            if (in_schedule(r)) cnt[lvl[H.row_node[r]] + 1]++;
        for (size_t l = 1; l < cnt.size(); ++l) cnt[l] += cnt[l - 1];
        const int64_t nm = cnt.back();
        D.nmob = nm;
        std::vector<int32_t> mrow((size_t)nm), mkp((size_t)nm), mnode((size_t)nm), mslot((size_t)nm),
            mlevel((size_t)nm);
        std::vector<int64_t> moff((size_t)nm);
        for (int64_t r = 0; r < n; ++r)
            if (in_schedule(r)) mrow[(size_t)cnt[lvl[H.row_node[r]]]++] = (int32_t)r;
        int64_t total = 0;
        D.nmob_entries = 0;
        D.mob_kp_max = 0;
        for (int64_t i = 0; i < nm; ++i) {
            const int32_t r = mrow[i], x = H.row_node[r];
            mkp[i] = std::max<int32_t>(16, (rowcnt[r] - 1 + 15) / 16 * 16);
            D.mob_kp_max = std::max(D.mob_kp_max, mkp[i]);
            moff[i] = total;
            total += mkp[i];
            D.nmob_entries += rowcnt[r] - 1;
            mnode[i] = x;
            mslot[i] = H.node_slot[x];
            mlevel[i] = lvl[x];
        }
        const int32_t *key_slot = d_uslot;   // U levels by slot, -1 at zero slots
        if (anti) {
            std::vector<int32_t> ks((size_t)nslots);
            for (int64_t s2 = 0; s2 < nslots; ++s2) ks[s2] = H.slot_node[s2] < 0 ? -1 : H.level[H.slot_node[s2]];
            int32_t *d_ks;
            if ((st = tmp.put(&d_ks, ks.data(), ks.size()))) return st;
            key_slot = d_ks;
        }
        D.Nm = (int32_t *)plan_alloc(p, sizeof(int32_t) * (size_t)total);
        if (!D.Nm) {
            set_last_error("device allocation failed");
            return MZ_ERR_OOM;
        }
        if ((e = cudaMemset(D.Nm, 0, sizeof(int32_t) * (size_t)total)) != cudaSuccess)
            return cuda_fail(e, "cudaMemset");
        if ((st = upload(p, &D.mob_off, moff.data(), moff.size()))) return st;
        if ((st = upload(p, &D.mob_kp, mkp.data(), mkp.size()))) return st;
        if ((st = upload(p, &D.mob_node, mnode.data(), mnode.size()))) return st;
        if ((st = upload(p, &D.mob_slot, mslot.data(), mslot.size()))) return st;
        if ((st = upload(p, &D.mob_level, mlevel.data(), mlevel.size()))) return st;
        int32_t *d_mrow;
        if ((st = tmp.put(&d_mrow, mrow.data(), mrow.size()))) return st;
        if (!H.sparse) {
            BuildMobArgs b;
            std::memset(&b, 0, sizeof(b));
            b.N = d_N;
            b.k = (int32_t)k;
            b.mrow = d_mrow;
            b.moff = D.mob_off;
            b.mkp = D.mob_kp;
            b.mslot = D.mob_slot;
            b.key_slot = key_slot;
            b.n = nm;
            b.Nm = D.Nm;
            e = launch_build_mob_rows(b, p->num_sms, 0);
        } else {
            BuildMobSparseArgs b;
            b.row_beg = d_row_beg;
            b.row_len = d_rowcnt;
            b.pool = d_pool;
            b.mrow = d_mrow;
            b.moff = D.mob_off;
            b.mkp = D.mob_kp;
            b.mslot = D.mob_slot;
            b.key_slot = key_slot;
            b.n = nm;
            b.Nm = D.Nm;
            e = launch_build_mob_rows_sparse(b, p->num_sms, 0);
        }
        if (e != cudaSuccess) return cuda_fail(e, "row build launch");
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "device build");
    H.csr_ptr = std::vector<int64_t>();
    H.csr_adj = std::vector<int32_t>();
    return MZ_OK;
}

// Device build of a plan of several posets with dense maps: the recurrence of Thm. 4 for
// all posets in one dataflow launch over the union (a poset's rows are as wide as its own
// number of chains), then the layouts of upload_side: tiles of 32 rows per poset, the
// Moebius rows of all posets in one order (level, then poset, then row). Every entry is
// decided by comparisons, so the plan equals the host build's entry for entry.
static mz_status upload_batch_device(mz_plan *p, int side) {
    std::vector<HostSide> &Hs = p->host[side];
    DeviceSide &D = p->dev[side];
    const size_t C = Hs.size();
    const int64_t n = p->n_total(), nslots = p->slots_total(), K = p->chain_off.back();
    const std::string who = side ? "dual: " : "";
    const bool anti = (p->schedule == MZ_SCHED_ANTICHAIN);
    D.n = n;
    D.nslots = nslots;
    D.k_max = 0;
    D.kpad_max = 0;
    int32_t maxh = 0;
    for (const HostSide &H : Hs) {
        D.k_max = std::max(D.k_max, H.k);
        D.kpad_max = std::max<int32_t>(D.kpad_max, (H.k + 15) / 16 * 16);
        maxh = std::max(maxh, H.nlevels);
    }
    mz_status st;
    cudaError_t e;
    {   // slot map, padded with -1 to a multiple of 64 entries
        std::vector<int32_t> sn(((size_t)nslots + 63) / 64 * 64, -1);
        for (size_t c = 0; c < C; ++c)
            for (size_t q = 0; q < Hs[c].slot_node.size(); ++q) {
                const int32_t v = Hs[c].slot_node[q];
                sn[p->slot_off[c] + q] = v < 0 ? -1 : (int32_t)(v + p->node_off[c]);
            }
        if ((st = upload(p, &D.slot_node, sn.data(), sn.size()))) return st;
    }
    BuildScratch tmp(p);
    // ---- the union's inputs of the recurrence
    int64_t edges = 0, entries = 0;
    for (const HostSide &H : Hs) {
        edges += H.csr_ptr[(size_t)H.n];
        entries += H.n * (int64_t)H.k;
    }
    std::vector<int64_t> ptr((size_t)n + 1), croff(C), cmoff(C);
    std::vector<int32_t> adj((size_t)edges), node_slot((size_t)n), chain((size_t)n), comp((size_t)n),
        topo_pos((size_t)n), base((size_t)K), ck(C), ckoff(C);
    {
        int64_t eo = 0, mo = 0;
        for (size_t c = 0; c < C; ++c) {
            const HostSide &H = Hs[c];
            const int64_t no = p->node_off[c], so = p->slot_off[c], ko = p->chain_off[c];
            ck[c] = H.k;
            ckoff[c] = (int32_t)ko;
            croff[c] = no;
            cmoff[c] = mo;
            mo += H.n * (int64_t)H.k;
            for (int64_t x = 0; x < H.n; ++x) {
                ptr[(size_t)(no + x)] = eo + H.csr_ptr[(size_t)x];
                node_slot[(size_t)(no + x)] = (int32_t)(H.node_slot[(size_t)x] + so);
                chain[(size_t)(no + x)] = (int32_t)(H.chain_id[(size_t)x] + ko);
                comp[(size_t)(no + x)] = (int32_t)c;
                topo_pos[(size_t)(no + H.topo[(size_t)x])] = (int32_t)(no + x);
            }
            const int64_t ne = H.csr_ptr[(size_t)H.n];
            for (int64_t q = 0; q < ne; ++q) adj[(size_t)(eo + q)] = (int32_t)(H.csr_adj[(size_t)q] + no);
            eo += ne;
            for (int32_t j = 0; j < H.k; ++j) base[(size_t)(ko + j)] = (int32_t)(H.chain_base[(size_t)j] + so);
        }
        ptr[(size_t)n] = eo;
    }
    // nodes bottom-up by height over all posets
    std::vector<int32_t> order((size_t)n);
    {
        std::vector<int64_t> fill((size_t)maxh + 2, 0);
        for (size_t c = 0; c < C; ++c)
            for (int64_t x = 0; x < Hs[c].n; ++x) fill[(size_t)Hs[c].level[(size_t)x]]++;
        for (size_t l = 1; l < fill.size(); ++l) fill[l] += fill[l - 1];
        for (size_t c = 0; c < C; ++c) {
            const HostSide &H = Hs[c];
            for (int64_t i = H.n - 1; i >= 0; --i) {
                const int32_t x = H.topo[(size_t)i];
                order[(size_t)fill[(size_t)H.level[(size_t)x] - 1]++] = (int32_t)(x + p->node_off[c]);
            }
        }
    }
    int64_t *d_ptr, *d_croff, *d_cmoff;
    int32_t *d_adj, *d_order, *d_node_slot, *d_chain, *d_base, *d_pos, *d_comp, *d_ck, *d_ckoff;
    if ((st = tmp.put(&d_ptr, ptr.data(), ptr.size())) || (st = tmp.put(&d_adj, adj.data(), adj.size())) ||
        (st = tmp.put(&d_order, order.data(), order.size())) ||
        (st = tmp.put(&d_node_slot, node_slot.data(), node_slot.size())) ||
        (st = tmp.put(&d_chain, chain.data(), chain.size())) || (st = tmp.put(&d_base, base.data(), base.size())) ||
        (st = tmp.put(&d_pos, topo_pos.data(), topo_pos.size())) || (st = tmp.put(&d_comp, comp.data(), comp.size())) ||
        (st = tmp.put(&d_ck, ck.data(), ck.size())) || (st = tmp.put(&d_ckoff, ckoff.data(), ckoff.size())) ||
        (st = tmp.put(&d_croff, croff.data(), croff.size())) || (st = tmp.put(&d_cmoff, cmoff.data(), cmoff.size())))
        return st;
    adj = std::vector<int32_t>();
    int32_t *d_uslot = tmp.get<int32_t>((size_t)nslots);
    int32_t *d_rowcnt = tmp.get<int32_t>((size_t)n);
    uint32_t *d_small = tmp.get<uint32_t>(64);   // ticket, status, bad, -, nnz (u64 at word 4)
    int32_t *d_N = tmp.get<int32_t>((size_t)entries);
    uint32_t *d_ready = tmp.get<uint32_t>((size_t)n);
    if (!d_uslot || !d_rowcnt || !d_small || !d_N || !d_ready) {
        set_last_error("device allocation failed");
        return MZ_ERR_OOM;
    }
    const uint32_t small_init[6] = {0u, 0u, 0xffffffffu, 0u, 0u, 0u};
    // the map starts at slot 0 everywhere, so that no read can leave the slot range
    if ((e = cudaMemset(d_uslot, 0xff, sizeof(int32_t) * nslots)) != cudaSuccess ||
        (e = cudaMemcpy(d_small, small_init, sizeof(small_init), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(d_N, 0, sizeof(int32_t) * (size_t)entries)) != cudaSuccess ||
        (e = cudaMemset(d_ready, 0, sizeof(uint32_t) * (size_t)n)) != cudaSuccess)
        return cuda_fail(e, "build setup");
    {
        BuildNivArgs a;
        std::memset(&a, 0, sizeof(a));
        a.ptr = d_ptr;
        a.adj = d_adj;
        a.order = d_order;
        a.node_slot = d_node_slot;
        a.chain_id = d_chain;
        a.base = d_base;
        a.topo_pos = d_pos;
        a.n = n;
        a.k = D.k_max;
        a.N = d_N;
        a.uslot = d_uslot;
        a.rowcnt = d_rowcnt;
        a.ready = d_ready;
        a.ticket = d_small;
        a.status = d_small + 1;
        a.bad = (int32_t *)(d_small + 2);
        a.nnz = (unsigned long long *)(d_small + 4);
        a.spin_limit = p->spin_limit;
        a.comp = d_comp;
        a.comp_k = d_ck;
        a.comp_koff = d_ckoff;
        a.comp_roff = d_croff;
        a.comp_moff = d_cmoff;
        if ((e = launch_build_niv(a, p->num_sms, 0)) != cudaSuccess) return cuda_fail(e, "niv build launch");
    }
    uint32_t small[6];
    if ((e = cudaMemcpy(small, d_small, sizeof(small), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "niv build");
    if (small[1]) {
        set_last_error(who + "device build: a bounded wait ran out");
        return MZ_ERR_TIMEOUT;
    }
    if ((int32_t)small[2] >= 0) {   // the largest topological position (over the union) of a failing node
        const int64_t g = (int32_t)small[2];
        const size_t c = (size_t)(std::upper_bound(p->node_off.begin(), p->node_off.end(), g) - p->node_off.begin() - 1);
        const HostSide &H = Hs[c];
        const int32_t x = H.topo[(size_t)(g - p->node_off[c])];
        set_last_error(who + "poset " + std::to_string(c) + ": chain " + std::to_string(H.chain_id[(size_t)x]) +
                       " is not totally ordered at node " + std::to_string(x));
        return MZ_ERR_BAD_CHAINS;
    }
    std::vector<int32_t> uslot((size_t)nslots), rowcnt((size_t)n);
    if ((e = cudaMemcpy(uslot.data(), d_uslot, sizeof(int32_t) * nslots, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(rowcnt.data(), d_rowcnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy");
    for (size_t c = 0; c < C; ++c) {   // per poset: U levels, nnz (rows of poset c are global rows node_off[c] ..)
        HostSide &H = Hs[c];
        H.ulevel.assign((size_t)H.n, 0);
        int64_t nnz = 0;
        for (int64_t x = 0; x < H.n; ++x) {
            H.ulevel[(size_t)x] = uslot[(size_t)(H.node_slot[(size_t)x] + p->slot_off[c])];
            nnz += rowcnt[(size_t)(p->node_off[c] + x)];
        }
        H.nulevels = H.n ? *std::max_element(H.ulevel.begin(), H.ulevel.end()) + 1 : 0;
        H.nnz = nnz;
    }
    // ---- tiles of 32 rows per poset (rows in slot order), as upload_side lays them out
    std::vector<int32_t> rn_host;
    {
        int64_t nt = 0;
        for (const HostSide &H : Hs) nt += (H.n + kTileRows - 1) / kTileRows;
        D.ntiles = nt;
        std::vector<int64_t> toff((size_t)nt), tmoff((size_t)nt);
        std::vector<int32_t> tk((size_t)nt), trows((size_t)nt);
        rn_host.assign((size_t)nt * kTileRows, -1);
        int64_t t = 0, total = 0;
        for (size_t c = 0; c < C; ++c) {
            const HostSide &H = Hs[c];
            for (int64_t t0 = 0; t0 * kTileRows < H.n; ++t0, ++t) {
                toff[(size_t)t] = total;
                tk[(size_t)t] = H.k;
                trows[(size_t)t] = (int32_t)std::min<int64_t>(kTileRows, H.n - t0 * kTileRows);
                tmoff[(size_t)t] = cmoff[c] + t0 * kTileRows * (int64_t)H.k;
                total += (int64_t)H.k * kTileRows;
                for (int32_t q = 0; q < trows[(size_t)t]; ++q)
                    rn_host[(size_t)(t * kTileRows + q)] =
                        (int32_t)(H.row_node[(size_t)(t0 * kTileRows + q)] + p->node_off[c]);
            }
        }
        D.Nt = (int32_t *)plan_alloc(p, sizeof(int32_t) * (size_t)std::max<int64_t>(total, 1));
        if (!D.Nt) {
            set_last_error("device allocation failed");
            return MZ_ERR_OOM;
        }
        int64_t *d_tmoff;
        int32_t *d_trows;
        if ((st = upload(p, &D.tile_off, toff.data(), toff.size())) ||
            (st = upload(p, &D.tile_k, tk.data(), tk.size())) ||
            (st = upload(p, &D.row_node, rn_host.data(), rn_host.size())) ||
            (st = tmp.put(&d_tmoff, tmoff.data(), tmoff.size())) || (st = tmp.put(&d_trows, trows.data(), trows.size())))
            return st;
        if ((e = launch_build_tiles_var(d_N, nt, d_tmoff, D.tile_k, d_trows, D.tile_off, D.Nt, p->num_sms, 0)) !=
            cudaSuccess)
            return cuda_fail(e, "tile build launch");
    }
    // ---- U-level schedule: the slots another chain's row reads
    std::vector<uint8_t> ref;
    if (!anti) {
        D.slot_ref = (uint8_t *)plan_alloc(p, (size_t)nslots);
        if (!D.slot_ref) {
            set_last_error("device allocation failed");
            return MZ_ERR_OOM;
        }
        if ((e = cudaMemset(D.slot_ref, 0, (size_t)nslots)) != cudaSuccess) return cuda_fail(e, "cudaMemset");
        if ((e = launch_mark_referenced(D.Nt, D.tile_off, D.tile_k, D.row_node, D.ntiles, d_node_slot, D.slot_node,
                                        D.slot_ref, p->num_sms, 0)) != cudaSuccess)
            return cuda_fail(e, "reference marking launch");
        ref.resize((size_t)nslots);
        if ((e = cudaMemcpy(ref.data(), D.slot_ref, (size_t)nslots, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpy");
        std::vector<int32_t> rl(rn_host.size(), -1);
        for (size_t q = 0; q < rn_host.size(); ++q)
            if (rn_host[q] >= 0) {
                const int32_t gs = node_slot[(size_t)rn_host[q]];
                rl[q] = ref[(size_t)gs] ? -1 : gs;
            }
        if ((st = upload(p, &D.row_leaf, rl.data(), rl.size()))) return st;
    }
    // ---- Moebius rows: all posets in one order, by level, then poset, then row
    {
        auto in_schedule = [&](size_t c, int64_t r) {
            return anti || ref[(size_t)(Hs[c].node_slot[(size_t)Hs[c].row_node[(size_t)r]] + p->slot_off[c])] != 0;
        };
        int32_t maxlvl = 0;
        for (const HostSide &H : Hs) maxlvl = std::max(maxlvl, anti ? H.nlevels : H.nulevels);
        std::vector<int64_t> cnt((size_t)maxlvl + 2, 0);
        for (size_t c = 0; c < C; ++c) {
            const HostSide &H = Hs[c];
            const std::vector<int32_t> &lvl = anti ? H.level : H.ulevel;
            for (int64_t r = 0; r < H.n; ++r)
                if (in_schedule(c, r)) cnt[(size_t)lvl[(size_t)H.row_node[(size_t)r]] + 1]++;
        }
        for (size_t l = 1; l < cnt.size(); ++l) cnt[l] += cnt[l - 1];
        const int64_t nm = cnt.back();
        D.nmob = nm;
        std::vector<std::pair<int32_t, int32_t>> ord((size_t)nm);
        for (size_t c = 0; c < C; ++c) {
            const HostSide &H = Hs[c];
            const std::vector<int32_t> &lvl = anti ? H.level : H.ulevel;
            for (int64_t r = 0; r < H.n; ++r)
                if (in_schedule(c, r)) ord[(size_t)cnt[(size_t)lvl[(size_t)H.row_node[(size_t)r]]]++] = {(int32_t)c, (int32_t)r};
        }
        std::vector<int64_t> moff((size_t)nm), rmoff((size_t)nm);
        std::vector<int32_t> mkp((size_t)nm), mnode((size_t)nm), mslot((size_t)nm), mlevel((size_t)nm), rk((size_t)nm);
        int64_t total = 0;
        D.nmob_entries = 0;
        D.mob_kp_max = 0;
        for (int64_t i = 0; i < nm; ++i) {
            const size_t c = (size_t)ord[(size_t)i].first;
            const int64_t r = ord[(size_t)i].second;
            const HostSide &H = Hs[c];
            const std::vector<int32_t> &lvl = anti ? H.level : H.ulevel;
            const int32_t x = H.row_node[(size_t)r];
            const int32_t cntr = rowcnt[(size_t)(p->node_off[c] + r)];
            mkp[(size_t)i] = std::max<int32_t>(16, (cntr - 1 + 15) / 16 * 16);
            moff[(size_t)i] = total;
            total += mkp[(size_t)i];
            D.nmob_entries += cntr - 1;
            D.mob_kp_max = std::max(D.mob_kp_max, mkp[(size_t)i]);
            mnode[(size_t)i] = (int32_t)(x + p->node_off[c]);
            mslot[(size_t)i] = (int32_t)(H.node_slot[(size_t)x] + p->slot_off[c]);
            mlevel[(size_t)i] = lvl[(size_t)x];
            rmoff[(size_t)i] = cmoff[c] + r * (int64_t)H.k;
            rk[(size_t)i] = H.k;
        }
        const int32_t *key_slot = d_uslot;   // U levels by slot, -1 at zero slots
        if (anti) {
            std::vector<int32_t> ks((size_t)nslots, -1);
            for (size_t c = 0; c < C; ++c)
                for (int64_t x = 0; x < Hs[c].n; ++x)
                    ks[(size_t)(Hs[c].node_slot[(size_t)x] + p->slot_off[c])] = Hs[c].level[(size_t)x];
            int32_t *d_ks;
            if ((st = tmp.put(&d_ks, ks.data(), ks.size()))) return st;
            key_slot = d_ks;
        }
        D.Nm = (int32_t *)plan_alloc(p, sizeof(int32_t) * (size_t)std::max<int64_t>(total, 1));
        if (!D.Nm) {
            set_last_error("device allocation failed");
            return MZ_ERR_OOM;
        }
        if ((e = cudaMemset(D.Nm, 0, sizeof(int32_t) * (size_t)std::max<int64_t>(total, 1))) != cudaSuccess)
            return cuda_fail(e, "cudaMemset");
        int64_t *d_rmoff;
        int32_t *d_rk;
        if ((st = upload(p, &D.mob_off, moff.data(), moff.size())) || (st = upload(p, &D.mob_kp, mkp.data(), mkp.size())) ||
            (st = upload(p, &D.mob_node, mnode.data(), mnode.size())) ||
            (st = upload(p, &D.mob_slot, mslot.data(), mslot.size())) ||
            (st = upload(p, &D.mob_level, mlevel.data(), mlevel.size())) ||
            (st = tmp.put(&d_rmoff, rmoff.data(), rmoff.size())) || (st = tmp.put(&d_rk, rk.data(), rk.size())))
            return st;
        BuildMobArgs b;
        std::memset(&b, 0, sizeof(b));
        b.N = d_N;
        b.k = D.k_max;
        b.mrow = nullptr;
        b.moff = D.mob_off;
        b.mkp = D.mob_kp;
        b.mslot = D.mob_slot;
        b.key_slot = key_slot;
        b.n = nm;
        b.Nm = D.Nm;
        b.row_moff = d_rmoff;
        b.row_k = d_rk;
        if ((e = launch_build_mob_rows(b, p->num_sms, 0)) != cudaSuccess) return cuda_fail(e, "row build launch");
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "device build");
    for (HostSide &H : Hs) {
        H.csr_ptr = std::vector<int64_t>();
        H.csr_adj = std::vector<int32_t>();
    }
    return MZ_OK;
}

// ---------------------------------------------------------------- workspace
struct WsLayout {
    ScanShape sh;
    size_t counters = 0, flags = 0, agg = 0, inc = 0, P = 0, esc = 0, Q = 0, memset_bytes = 0, total = 0;
};

// Workspace: the scan's look-back state, the prefix array y' ([nslots][B] 8-byte words),
// and for the Moebius transform the escape flags of int64 words ([nslots][B] bytes) or
// the double-word copies of y' for F32C ([nslots][B] float pairs).
static WsLayout ws_layout(const mz_plan *p, int32_t B, int dtype) {
    WsLayout L;
    const int64_t nslots = p->slots_total();
    L.sh = scan_shape(nslots, B);
    const size_t tiles = (size_t)L.sh.groups * (size_t)L.sh.ntiles;
    const size_t words = (size_t)nslots * (size_t)B;
    L.counters = 0;
    L.flags = align256(sizeof(uint32_t) * L.sh.groups);
    L.agg = L.flags + align256(sizeof(uint32_t) * tiles);
    L.memset_bytes = L.agg;
    L.inc = L.agg + align256(8 * tiles * L.sh.BW);
    L.P = L.inc + align256(8 * tiles * L.sh.BW);
    size_t end = L.P + align256(8 * words);
    if (dtype == MZ_I64) {
        L.esc = end;
        end += align256(words);
    } else if (dtype == MZ_F32C) {
        L.Q = end;
        end += align256(8 * words);
    }
    L.total = end;
    return L;
}

static bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + nb && y < x + na;
}

static mz_status check_call(const mz_plan *p, int dtype, const void *in, const void *out, int32_t B, void *ws,
                            size_t ws_bytes, int side, WsLayout *L) {
    if (!p || !in || !out || !ws) {
        set_last_error("null argument");
        return MZ_ERR_INVALID_ARG;
    }
    if (p->host_only) {
        set_last_error("plan was built host-only");
        return MZ_ERR_NO_DEVICE;
    }
    if (side == 1 && !p->has_dual) {
        set_last_error("plan was built without the dual (build_transpose = 0)");
        return MZ_ERR_UNSUPPORTED;
    }
    if (dtype != MZ_I64 && dtype != MZ_F64 && dtype != MZ_F32C) {
        set_last_error("unknown dtype");
        return MZ_ERR_INVALID_ARG;
    }
    if (B < 1) {
        set_last_error("batch must be >= 1");
        return MZ_ERR_INVALID_ARG;
    }
    *L = ws_layout(p, B, dtype);
    if (ws_bytes < L->total || ((uintptr_t)ws & 255)) {
        set_last_error("workspace too small or not 256-byte aligned");
        return MZ_ERR_INVALID_ARG;
    }
    const size_t vb = (size_t)p->n_total() * (size_t)B * 8;   // every dtype: 8 bytes per element
    if (overlaps(in, vb, out, vb) || overlaps(in, vb, ws, ws_bytes) || overlaps(out, vb, ws, ws_bytes)) {
        set_last_error("input, output and workspace must not overlap");
        return MZ_ERR_INVALID_ARG;
    }
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->device) {
        set_last_error("the current CUDA device is not the plan's device");
        return MZ_ERR_INVALID_ARG;
    }
    return MZ_OK;
}

// MZ_DEBUG builds fill the workspace and the output with a poison pattern (every byte
// 0xFF: int64 -1, a NaN in fp64 and fp32) before a transform, so that a word the kernels
// fail to write shows up in the result. Release builds do nothing here.
static mz_status debug_poison(const mz_plan *p, int side, void *ws, size_t ws_bytes, void *out, int32_t B,
                              cudaStream_t s) {
#ifdef MZ_DEBUG
    cudaError_t e = cudaMemsetAsync(ws, 0xFF, ws_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0xFF, (size_t)p->dev[side].n * (size_t)B * 8, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
#else
    (void)p, (void)side, (void)ws, (void)ws_bytes, (void)out, (void)B, (void)s;
#endif
    return MZ_OK;
}

static mz_status run_zeta(const mz_plan *p, int side, mz_dtype dtype, const void *f, void *g, int32_t B, void *ws,
                          size_t ws_bytes, mz_stream stream) {
    NvtxRange range(side ? "mz_zeta_T" : "mz_zeta");
    g_last_launches = 0;
    WsLayout L;
    mz_status st = check_call(p, dtype, f, g, B, ws, ws_bytes, side, &L);
    if (st) return st;
    const DeviceSide &D = p->dev[side];
    cudaStream_t s = (cudaStream_t)stream;
    char *w = (char *)ws;
    mark_event(0, s);
    if ((st = debug_poison(p, side, ws, ws_bytes, g, B, s))) return st;
    cudaError_t e = cudaMemsetAsync(w, 0, L.memset_bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    ScanArgs sa;
    sa.slot_node = D.slot_node;
    sa.nslots = D.nslots;
    sa.B = B;
    sa.BW = L.sh.BW;
    sa.R = L.sh.R;
    sa.ntiles = L.sh.ntiles;
    sa.f = f;
    sa.nB = D.n * (int64_t)B;
    sa.P = w + L.P;
    sa.counters = (uint32_t *)(w + L.counters);
    sa.flags = (uint32_t *)(w + L.flags);
    sa.agg = w + L.agg;
    sa.inc = w + L.inc;
    sa.status = p->d_status;
    sa.spin_limit = p->spin_limit;
    sa.withhold = p->withhold;
    if ((e = launch_scan(dtype, sa, L.sh, s)) != cudaSuccess) return cuda_fail(e, "chain scan launch");
    mark_event(++g_last_launches, s);
    GatherArgs ga;
    ga.blocks_per_sm = p->gather_blocks_per_sm;
    ga.Nt = D.Nt;
    ga.tile_off = D.tile_off;
    ga.tile_k = D.tile_k;
    ga.row_node = D.row_node;
    ga.ntiles = D.ntiles;
    ga.B = B;
    ga.P = w + L.P;
    ga.g = g;
    ga.nB = D.n * (int64_t)B;
    ga.nslots = D.nslots;
    ga.status = p->d_status;
    if ((e = launch_gather(dtype, ga, p->num_sms, s)) != cudaSuccess) return cuda_fail(e, "niv gather launch");
    mark_event(++g_last_launches, s);
    return MZ_OK;
}

static mz_status run_mobius(const mz_plan *p, int side, mz_dtype dtype, const void *g, void *f, int32_t B, void *ws,
                            size_t ws_bytes, mz_stream stream) {
    NvtxRange range(side ? "mz_mobius_T" : "mz_mobius");
    g_last_launches = 0;
    WsLayout L;
    mz_status st = check_call(p, dtype, g, f, B, ws, ws_bytes, side, &L);
    if (st) return st;
    const DeviceSide &D = p->dev[side];
    if ((st = debug_poison(p, side, ws, ws_bytes, f, B, (cudaStream_t)stream))) return st;
    MobArgs ma;
    ma.Nm = D.Nm;
    ma.mob_off = D.mob_off;
    ma.mob_kp = D.mob_kp;
    ma.kpad_max = D.kpad_max;
    ma.blocks_per_sm = p->mob_blocks_per_sm;
    ma.mob_node = D.mob_node;
    ma.mob_slot = D.mob_slot;
    ma.mob_level = D.mob_level;
    ma.pace_ns = p->mob_pace_ns;
    ma.B = B;
    ma.g = g;
    ma.f = f;
    ma.nB = D.n * (int64_t)B;
    ma.P = (unsigned long long *)((char *)ws + L.P);
    ma.status = p->d_status;
    ma.spin_limit = p->spin_limit;
    ma.withhold = p->withhold;
    ma.n = D.nmob;
    ma.nslots = D.nslots;
    ma.esc = dtype == MZ_I64 ? (unsigned char *)ws + L.esc : nullptr;
    ma.Q = dtype == MZ_F32C ? (float2 *)((char *)ws + L.Q) : nullptr;
    ma.slot_ref = D.slot_ref;
    ma.Nt = D.Nt;
    ma.tile_off = D.tile_off;
    ma.tile_k = D.tile_k;
    ma.row_node = D.row_node;
    ma.row_leaf = D.row_leaf;
    ma.ntiles = D.ntiles;
    ma.gather_blocks_per_sm = p->gather_blocks_per_sm;
    ma.lanes = p->mob_lanes;
    ma.tree_w = 1;
    while (ma.tree_w * 16 < D.mob_kp_max && ma.tree_w < 32) ma.tree_w *= 2;
    int launches = 0;
    mark_event(0, (cudaStream_t)stream);
    cudaError_t e = launch_mobius(dtype, ma, D.slot_node, D.nslots, p->schedule == MZ_SCHED_ANTICHAIN, p->num_sms,
                                  (cudaStream_t)stream, &launches);
    g_last_launches = launches;
    if (e != cudaSuccess) return cuda_fail(e, "moebius launch");
    return MZ_OK;
}

// Builds the host side of every component (in parallel for many components) and
// the offsets of the union.
static mz_status build_components(mz_plan *p, int32_t count, const int64_t *n, const int64_t *m,
                                  const int32_t *const *src, const int32_t *const *dst,
                                  const int32_t *const *chain_id, bool dual, int niv_format, bool device_niv,
                                  bool device_chains) {
    // Alg. 1 on the device for a single poset given without chains (device_build = 2)
    Matcher matcher;
    if (device_chains && count == 1)
        matcher = [p](int64_t nn, const std::vector<int64_t> &ptr, const std::vector<int32_t> &adj,
                      std::vector<int32_t> &next, std::string &err) {
            return device_matching(p, nn, ptr, adj, next, err);
        };
    p->host[0].resize(count);
    if (dual) p->host[1].resize(count);
    std::vector<mz_status> sts(count, MZ_OK);
    std::vector<std::string> errs(count);
    auto work = [&](int32_t c) {
        try {
            std::vector<int32_t> s(src[c], src[c] + m[c]), d(dst[c], dst[c] + m[c]);
            const int32_t *cid = chain_id ? chain_id[c] : nullptr;
            sts[c] = build_host_side(n[c], s, d, cid, niv_format, device_niv, p->host[0][c], errs[c],
                                     matcher ? &matcher : nullptr);
            if (sts[c] == MZ_OK && dual) {
                // the dual poset: every edge flipped, the same chains (a chain of P is a chain of its dual)
                sts[c] = build_host_side(n[c], d, s, p->host[0][c].chain_id.data(), niv_format, device_niv,
                                         p->host[1][c], errs[c]);
                if (sts[c]) errs[c] = "dual: " + errs[c];
            }
        } catch (const std::bad_alloc &) {
            sts[c] = MZ_ERR_OOM;
            errs[c] = "host allocation failed";
        }
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int32_t nthreads = (int32_t)std::min<int64_t>(count, hw);
    if (nthreads <= 1) {
        for (int32_t c = 0; c < count; ++c) work(c);
    } else {
        std::atomic<int32_t> next{0};
        std::vector<std::thread> pool;
        for (int32_t t = 0; t < nthreads; ++t)
            pool.emplace_back([&]() {
                set_host_threads_cap(1);   // the posets already share the host's threads
                for (int32_t c = next++; c < count; c = next++) work(c);
            });
        for (auto &th : pool) th.join();
    }
    for (int32_t c = 0; c < count; ++c)
        if (sts[c]) {
            set_last_error(count > 1 ? "poset " + std::to_string(c) + ": " + errs[c] : errs[c]);
            return sts[c];
        }
    p->node_off.assign(count + 1, 0);
    p->slot_off.assign(count + 1, 0);
    p->chain_off.assign(count + 1, 0);
    for (int32_t c = 0; c < count; ++c) {
        const HostSide &H = p->host[0][c];
        p->node_off[c + 1] = p->node_off[c] + H.n;
        p->chain_off[c + 1] = p->chain_off[c] + H.k;
        p->slot_off[c + 1] = p->slot_off[c] + H.n + H.k;
    }
    if (p->slot_off[count] >= (int64_t)INT32_MAX) {
        set_last_error("too many nodes plus chains for 32-bit slot indices");
        return MZ_ERR_INVALID_ARG;
    }
    p->has_dual = dual;
    return MZ_OK;
}

static mz_status finish_plan(std::unique_ptr<mz_plan> &p, const mz_build_opts &o, mz_plan **out);

static mz_status build_plan(int32_t count, const int64_t *n, const int64_t *m, const int32_t *const *src,
                            const int32_t *const *dst, const int32_t *const *chain_id, const mz_build_opts *opts,
                            mz_plan **out) {
    if (out) *out = nullptr;
    if (!out || count < 1 || !n || !m || !src || !dst) {
        set_last_error("invalid sizes or null pointers");
        return MZ_ERR_INVALID_ARG;
    }
    int64_t total = 0;
    for (int32_t c = 0; c < count; ++c) {
        if (n[c] < 1 || n[c] > (int64_t(1) << 30) || m[c] < 0 || (m[c] > 0 && (!src[c] || !dst[c]))) {
            set_last_error("invalid sizes or null pointers" + (count > 1 ? " for poset " + std::to_string(c) : ""));
            return MZ_ERR_INVALID_ARG;
        }
        total += n[c];
    }
    if (total > (int64_t(1) << 30)) {
        set_last_error("more than 2^30 nodes in one plan");
        return MZ_ERR_INVALID_ARG;
    }
    mz_build_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if ((o.dev_alloc == nullptr) != (o.dev_free == nullptr)) {
        set_last_error("dev_alloc and dev_free must be given together");
        return MZ_ERR_INVALID_ARG;
    }
    if (o.mobius_schedule != MZ_SCHED_ULEVEL && o.mobius_schedule != MZ_SCHED_ANTICHAIN) {
        set_last_error("unknown mobius_schedule");
        return MZ_ERR_INVALID_ARG;
    }
    std::unique_ptr<mz_plan> p;
    try {
        p.reset(new mz_plan());
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return MZ_ERR_OOM;
    }
    if (o.niv_format < 0 || o.niv_format > 2) {
        set_last_error("unknown niv_format");
        return MZ_ERR_INVALID_ARG;
    }
    if (o.device_build && o.host_only) {
        set_last_error("device_build needs a device plan (host_only is set)");
        return MZ_ERR_INVALID_ARG;
    }

    if (o.device_build < 0 || o.device_build > 2) {
        set_last_error("device_build is 0, 1 or 2");
        return MZ_ERR_INVALID_ARG;
    }
    mz_status st;
    {
        NvtxRange range("mz_build: host sides (order, chains, slots, levels)");
        st = build_components(p.get(), count, n, m, src, dst, chain_id, o.build_transpose != 0, o.niv_format,
                              o.device_build != 0, o.device_build == 2);
    }
    if (st) return st;
    if (o.device_build && count > 1)
        for (int side = 0; side < (p->has_dual ? 2 : 1); ++side)
            for (const HostSide &H : p->host[side])
                if (H.sparse) {
                    set_last_error("device_build of several posets needs dense niv maps (k <= 512 chains each)");
                    return MZ_ERR_UNSUPPORTED;
                }
    return finish_plan(p, o, out);
}

// The device part of a plan whose host sides are complete (a build or a plan file): the
// settings of the options, then the upload of every side; *out gets the plan.
static mz_status finish_plan(std::unique_ptr<mz_plan> &p, const mz_build_opts &o, mz_plan **out) {
    mz_status st = MZ_OK;
    p->schedule = o.mobius_schedule;
    p->host_only = o.host_only != 0;
    if (o.spin_limit > 0) p->spin_limit = o.spin_limit;
    if (o.mobius_blocks_per_sm > 0) p->mob_blocks_per_sm = o.mobius_blocks_per_sm;
    if (o.mobius_pace_ns != 0) p->mob_pace_ns = o.mobius_pace_ns < 0 ? 0 : o.mobius_pace_ns;
    p->withhold = o.debug_withhold > 0 ? o.debug_withhold - 1 : -1;
    p->dev_alloc = o.dev_alloc;
    p->dev_free = o.dev_free;
    p->alloc_ctx = o.alloc_ctx;
    if (!p->host_only) {
        cudaError_t e = cudaGetDevice(&p->device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
        e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        p->d_status = (uint32_t *)plan_alloc(p.get(), 256);
        if (!p->d_status) {
            set_last_error("device allocation failed");
            st = MZ_ERR_OOM;
        } else if ((e = cudaMemset(p->d_status, 0, 256)) != cudaSuccess) {
            st = cuda_fail(e, "cudaMemset");
        }
        NvtxRange range("mz_build: device part (uploads, device build)");
        for (int side = 0; side < (p->has_dual ? 2 : 1) && st == MZ_OK; ++side)
            st = !p->host[side][0].niv_on_device ? upload_side(p.get(), side)
                 : p->components() > 1            ? upload_batch_device(p.get(), side)
                                                  : upload_side_device(p.get(), side);
        if (st) {
            plan_free_all(p.get());
            return st;
        }
        // rows of one chunk (16 entries or fewer, as on the sparse random DAGs) leave nothing
        // to share between lanes: one lane per row; longer rows: a warp per row
        p->mob_lanes = p->dev[0].mob_kp_max <= 16 ? 1 : 32;
    }
    *out = p.release();
    return MZ_OK;
}

}  // namespace mz

using namespace mz;

extern "C" {

mz_status mz_build(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *chain_id,
                   const mz_build_opts *opts, mz_plan **out) {
    if (m > 0 && (!src || !dst)) {
        if (out) *out = nullptr;
        set_last_error("invalid sizes or null pointers");
        return MZ_ERR_INVALID_ARG;
    }
    const int32_t *const cids[1] = {chain_id};
    return build_plan(1, &n, &m, &src, &dst, chain_id ? cids : nullptr, opts, out);
}

mz_status mz_build_batch(int32_t count, const int64_t *n, const int64_t *m, const int32_t *const *src,
                         const int32_t *const *dst, const int32_t *const *chain_id, const mz_build_opts *opts,
                         mz_plan **out) {
    return build_plan(count, n, m, src, dst, chain_id, opts, out);
}

void mz_destroy(mz_plan *plan) {
    if (!plan) return;
    plan_free_all(plan);
    delete plan;
}

mz_status mz_workspace_size(const mz_plan *plan, mz_dtype dtype, int32_t batch, size_t *bytes) {
    if (!plan || !bytes || batch < 1 || (dtype != MZ_I64 && dtype != MZ_F64 && dtype != MZ_F32C)) {
        set_last_error("invalid argument");
        return MZ_ERR_INVALID_ARG;
    }
    *bytes = ws_layout(plan, batch, dtype).total;   // primal and dual share the slot count
    return MZ_OK;
}

mz_status mz_zeta(const mz_plan *plan, mz_dtype dtype, const void *f, void *g, int32_t batch, void *ws,
                  size_t ws_bytes, mz_stream stream) {
    return run_zeta(plan, 0, dtype, f, g, batch, ws, ws_bytes, stream);
}

// ---------------------------------------------------------------- zeta without allocation
// Scratch for mz_zeta_noalloc: a fixed device array owned by the library. Its
// name is only a host-side handle; the device address comes from
// cudaGetSymbolAddress in the context that is current at the call. The address
// is cached per CUDA context, keyed by the context's process-unique id
// (cuCtxGetId, reached through the runtime's driver entry points so that the
// library needs no link against the driver), so a context that was destroyed
// and created again (cudaDeviceReset) gets a fresh lookup instead of a stale
// address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MZ_NOALLOC_SCRATCH_BYTES];
struct NoallocEntry {
    unsigned long long ctx_id;
    void *addr;
};
static NoallocEntry g_noalloc_cache[64];
static int g_noalloc_used = 0, g_noalloc_next = 0;
static std::mutex g_noalloc_mutex;
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);
static CtxGetCurrentFn g_ctx_get_current = nullptr;
static CtxGetIdFn g_ctx_get_id = nullptr;
static bool g_ctx_fns_tried = false;

// Id of the context current on this thread; false if it cannot be had.
static bool current_context_id(unsigned long long *id) {
    if (!g_ctx_fns_tried) {
        g_ctx_fns_tried = true;
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess && qb == cudaDriverEntryPointSuccess) {
            g_ctx_get_current = (CtxGetCurrentFn)a;
            g_ctx_get_id = (CtxGetIdFn)b;
        }
        cudaGetLastError();
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return false;
    void *ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0 || !ctx) return false;
    return g_ctx_get_id(ctx, id) == 0;
}

// Device address of the scratch array in the current context.
static mz_status noalloc_address(void **out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);
    if (have_id)
        for (int i = 0; i < g_noalloc_used; ++i)
            if (g_noalloc_cache[i].ctx_id == id) {
                *out = g_noalloc_cache[i].addr;
                return MZ_OK;
            }
    void *addr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);   // also makes the context current
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    if (!have_id) have_id = current_context_id(&id);
    if (have_id) {   // no id (no driver entry points): look the address up on every call
        const int slot = g_noalloc_used < 64 ? g_noalloc_used++ : (g_noalloc_next++ & 63);
        g_noalloc_cache[slot] = {id, addr};
    }
    *out = addr;
    return MZ_OK;
}

mz_status mz_zeta_noalloc(const mz_plan *plan, mz_dtype dtype, const void *f, void *g, int32_t batch,
                          mz_stream stream) {
    if (!plan || batch < 1 || (dtype != MZ_I64 && dtype != MZ_F64 && dtype != MZ_F32C)) {
        set_last_error("invalid argument");
        return MZ_ERR_INVALID_ARG;
    }
    if (plan->host_only) {
        set_last_error("plan was built host-only");
        return MZ_ERR_NO_DEVICE;
    }
    const size_t need = ws_layout(plan, batch, dtype).total;
    if (need > MZ_NOALLOC_SCRATCH_BYTES) {
        set_last_error("mz_zeta_noalloc: this plan and batch need " + std::to_string(need) +
                       " bytes of scratch; the fixed scratch array holds " +
                       std::to_string((size_t)MZ_NOALLOC_SCRATCH_BYTES) + " (use mz_zeta with a workspace)");
        return MZ_ERR_INVALID_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != plan->device) {
        set_last_error("the current CUDA device is not the plan's device");
        return MZ_ERR_INVALID_ARG;
    }
    void *ws = nullptr;
    mz_status st = noalloc_address(&ws);
    if (st) return st;
    return run_zeta(plan, 0, dtype, f, g, batch, ws, MZ_NOALLOC_SCRATCH_BYTES, stream);
}

mz_status mz_mobius(const mz_plan *plan, mz_dtype dtype, const void *g, void *f, int32_t batch, void *ws,
                    size_t ws_bytes, mz_stream stream) {
    return run_mobius(plan, 0, dtype, g, f, batch, ws, ws_bytes, stream);
}

mz_status mz_zeta_T(const mz_plan *plan, mz_dtype dtype, const void *h, void *r, int32_t batch, void *ws,
                    size_t ws_bytes, mz_stream stream) {
    return run_zeta(plan, 1, dtype, h, r, batch, ws, ws_bytes, stream);
}

mz_status mz_mobius_T(const mz_plan *plan, mz_dtype dtype, const void *h, void *r, int32_t batch, void *ws,
                      size_t ws_bytes, mz_stream stream) {
    return run_mobius(plan, 1, dtype, h, r, batch, ws, ws_bytes, stream);
}

mz_status mz_check(const mz_plan *plan, mz_stream stream) {
    if (!plan) {
        set_last_error("null plan");
        return MZ_ERR_INVALID_ARG;
    }
    if (plan->host_only) return MZ_ERR_NO_DEVICE;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    uint32_t word = 0;
    e = cudaMemcpyAsync(&word, plan->d_status, sizeof(word), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (word) {
        e = cudaMemsetAsync(plan->d_status, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "status reset");
        set_last_error("a bounded device-side wait ran out");
        return (mz_status)word;
    }
    return MZ_OK;
}

mz_status mz_plan_tune(mz_plan *plan, const mz_tuning *set, mz_tuning *current) {
    if (!plan) {
        set_last_error("null plan");
        return MZ_ERR_INVALID_ARG;
    }
    if (set) {
        if (set->mobius_blocks_per_sm < 0 || set->mobius_blocks_per_sm > 64 || set->gather_blocks_per_sm < 0 ||
            set->gather_blocks_per_sm > 256 || set->mobius_lanes < 0 || set->mobius_lanes > 32 ||
            (set->mobius_lanes & (set->mobius_lanes - 1)) != 0) {
            set_last_error("tuning value out of range");
            return MZ_ERR_INVALID_ARG;
        }
        if (set->mobius_blocks_per_sm) plan->mob_blocks_per_sm = set->mobius_blocks_per_sm;
        if (set->mobius_pace_ns) plan->mob_pace_ns = set->mobius_pace_ns < 0 ? 0 : set->mobius_pace_ns;
        if (set->gather_blocks_per_sm) plan->gather_blocks_per_sm = set->gather_blocks_per_sm;
        if (set->mobius_lanes) plan->mob_lanes = set->mobius_lanes;
    }
    if (current) {
        std::memset(current, 0, sizeof(*current));
        current->mobius_blocks_per_sm = plan->mob_blocks_per_sm;
        current->mobius_pace_ns = plan->mob_pace_ns ? plan->mob_pace_ns : -1;
        current->gather_blocks_per_sm = plan->gather_blocks_per_sm;
        current->mobius_lanes = plan->mob_lanes;
    }
    return MZ_OK;
}

mz_status mz_plan_info(const mz_plan *plan, mz_plan_info_t *info) {
    if (!plan || !info) return MZ_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n = plan->n_total();
    info->k = (int32_t)plan->chain_off.back();
    info->has_transpose = plan->has_dual;
    info->schedule = plan->schedule;
    info->components = (int32_t)plan->components();
    for (const HostSide &H : plan->host[0]) {
        info->sparse += H.sparse ? 1 : 0;
        info->nnz += H.nnz;
        info->edges += H.edges;
        info->levels = std::max(info->levels, H.nlevels);
        info->ulevels = std::max(info->ulevels, H.nulevels);
        info->max_chain = std::max(info->max_chain, H.max_chain);
    }
    for (const HostSide &H : plan->host[1]) {
        info->levels_T = std::max(info->levels_T, H.nlevels);
        info->ulevels_T = std::max(info->ulevels_T, H.nulevels);
    }
    info->device_bytes = plan->device_bytes;
    if (!plan->host_only) {
        info->wave_rows = plan->dev[0].nmob;
        info->wave_entries = plan->dev[0].nmob_entries;
    }
    return MZ_OK;
}

mz_status mz_plan_save(const mz_plan *plan, const char *path) {
    if (!plan || !path) {
        set_last_error("null plan or path");
        return MZ_ERR_INVALID_ARG;
    }
    for (int side = 0; side < (plan->has_dual ? 2 : 1); ++side)
        for (const HostSide &H : plan->host[side])
            if (H.niv_on_device) {
                set_last_error("the niv map of a plan built with device_build exists only on the device; "
                               "a plan built with device_build = 0 can be saved");
                return MZ_ERR_UNSUPPORTED;
            }
    NvtxRange range("mz_plan_save");
    std::string err;
    const mz_status st = save_host_sides(plan, path, err);
    if (st) set_last_error(err);
    return st;
}

mz_status mz_plan_load(const char *path, const mz_build_opts *opts, mz_plan **out) {
    if (out) *out = nullptr;
    if (!path || !out) {
        set_last_error("null path or out");
        return MZ_ERR_INVALID_ARG;
    }
    mz_build_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if ((o.dev_alloc == nullptr) != (o.dev_free == nullptr)) {
        set_last_error("dev_alloc and dev_free must be given together");
        return MZ_ERR_INVALID_ARG;
    }
    if (o.mobius_schedule != MZ_SCHED_ULEVEL && o.mobius_schedule != MZ_SCHED_ANTICHAIN) {
        set_last_error("unknown mobius_schedule");
        return MZ_ERR_INVALID_ARG;
    }
    std::unique_ptr<mz_plan> p;
    try {
        p.reset(new mz_plan());
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return MZ_ERR_OOM;
    }
    NvtxRange range("mz_plan_load");
    std::string err;
    const mz_status st = load_host_sides(p.get(), path, err);
    if (st) {
        set_last_error(err);
        return st;
    }
    return finish_plan(p, o, out);
}

mz_status mz_plan_export(const mz_plan *plan, int32_t what, int32_t dual, void *out, size_t bytes) {
    if (!plan || !out || (dual && !plan->has_dual)) {
        set_last_error("invalid argument");
        return MZ_ERR_INVALID_ARG;
    }
    const std::vector<HostSide> &Hs = plan->host[dual ? 1 : 0];
    const int64_t n = plan->n_total();
    if (what < MZ_EXPORT_CHAIN_ID || what > MZ_EXPORT_TOPO) {
        set_last_error("unknown export");
        return MZ_ERR_INVALID_ARG;
    }
    if (what == MZ_EXPORT_NIV) {
        if (Hs.size() != 1) {
            set_last_error("the niv map is exported for single-poset plans only");
            return MZ_ERR_UNSUPPORTED;
        }
        const HostSide &H = Hs[0];
        const int64_t k = H.k;
        if (bytes < (size_t)n * (size_t)k * sizeof(int32_t)) {
            set_last_error("output buffer too small");
            return MZ_ERR_INVALID_ARG;
        }
        int32_t *o = (int32_t *)out;
        std::fill(o, o + (size_t)n * (size_t)k, -1);
        if (H.niv_on_device) {   // the map exists only on the device: read the gather's tiles back
            const DeviceSide &D = plan->dev[dual ? 1 : 0];
            std::vector<int64_t> toff((size_t)D.ntiles);
            std::vector<int32_t> tk((size_t)D.ntiles);
            cudaError_t e = cudaMemcpy(toff.data(), D.tile_off, sizeof(int64_t) * toff.size(), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess)
                e = cudaMemcpy(tk.data(), D.tile_k, sizeof(int32_t) * tk.size(), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
            const size_t total = D.ntiles ? (size_t)toff.back() + (size_t)tk.back() * kTileRows : 0;
            std::vector<int32_t> t(total), rn((size_t)D.ntiles * kTileRows);
            if ((e = cudaMemcpy(t.data(), D.Nt, sizeof(int32_t) * total, cudaMemcpyDeviceToHost)) != cudaSuccess ||
                (e = cudaMemcpy(rn.data(), D.row_node, sizeof(int32_t) * rn.size(), cudaMemcpyDeviceToHost)) !=
                    cudaSuccess)
                return cuda_fail(e, "cudaMemcpy");
            // a tile row lists slots (every chain in order for a dense map, the finite
            // entries for a sparse one); zero slots stand for infinity
            for (int64_t r = 0; r < n; ++r) {   // r: tile position, rn[r] its node
                const int64_t x = rn[r], tt = r / kTileRows;
                const int32_t *col = &t[(size_t)toff[tt] + r % kTileRows];
                for (int64_t q = 0; q < tk[tt]; ++q) {
                    const int32_t y = H.slot_node[col[q * kTileRows]];
                    if (y >= 0) o[x * k + H.chain_id[y]] = y;
                }
            }
            return MZ_OK;
        }
        for (int64_t x = 0; x < n; ++x) {
            const int64_t cx = H.chain_id[x];
            H.for_row(H.node_slot[x] - cx - 1, [&](int32_t c, int32_t slot) { o[x * k + c] = H.slot_node[slot]; });
        }
        return MZ_OK;
    }
    if (bytes < (size_t)n * sizeof(int32_t)) {
        set_last_error("output buffer too small");
        return MZ_ERR_INVALID_ARG;
    }
    int32_t *o = (int32_t *)out;
    for (size_t c = 0; c < Hs.size(); ++c) {
        const HostSide &H = Hs[c];
        int32_t *dst = o + plan->node_off[c];
        for (int64_t x = 0; x < H.n; ++x) {
            switch (what) {
                case MZ_EXPORT_CHAIN_ID: dst[x] = H.chain_id[x] + (int32_t)plan->chain_off[c]; break;
                case MZ_EXPORT_CHAIN_POS: dst[x] = H.chain_pos[x]; break;
                case MZ_EXPORT_LEVEL: dst[x] = H.level[x]; break;
                case MZ_EXPORT_ULEVEL: dst[x] = H.ulevel[x]; break;
                default: dst[x] = H.topo[x] + (int32_t)plan->node_off[c]; break;   // MZ_EXPORT_TOPO
            }
        }
    }
    return MZ_OK;
}

int32_t mz_last_launch_count(void) { return g_last_launches; }

void mz_set_launch_events(void *const *events, int32_t capacity) {
    g_events = capacity > 0 ? events : nullptr;
    g_event_cap = capacity > 0 ? capacity : 0;
}

const char *mz_status_string(mz_status s) {
    switch (s) {
        case MZ_OK: return "MZ_OK";
        case MZ_ERR_INVALID_ARG: return "MZ_ERR_INVALID_ARG";
        case MZ_ERR_CYCLE: return "MZ_ERR_CYCLE";
        case MZ_ERR_BAD_CHAINS: return "MZ_ERR_BAD_CHAINS";
        case MZ_ERR_OOM: return "MZ_ERR_OOM";
        case MZ_ERR_CUDA: return "MZ_ERR_CUDA";
        case MZ_ERR_TIMEOUT: return "MZ_ERR_TIMEOUT";
        case MZ_ERR_UNSUPPORTED: return "MZ_ERR_UNSUPPORTED";
        case MZ_ERR_NO_DEVICE: return "MZ_ERR_NO_DEVICE";
        case MZ_ERR_BOUNDS: return "MZ_ERR_BOUNDS";
    }
    return "unknown status";
}

const char *mz_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
