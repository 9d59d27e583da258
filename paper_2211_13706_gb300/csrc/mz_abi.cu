// The C ABI of include/mz.h: plan build and upload, workspace layout, and the
// transform entry points (argument checks, then kernel launches on the
// caller's stream). Every transform runs on the GPU; there is no host path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

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

// Device layouts of one side: the tiled map for the zeta gather and the map in
// Moebius processing order.
static mz_status upload_side(mz_plan *p, int side) {
    const HostSide &H = p->host[side];
    DeviceSide &D = p->dev[side];
    const int64_t n = H.n, k = H.k;
    // padded with -1 to a multiple of 64 entries: the scan reads it as 16-byte vectors
    std::vector<int32_t> sn(H.slot_node);
    sn.resize(((size_t)(n + k) + 63) / 64 * 64, -1);
    mz_status st = upload(p, &D.slot_node, sn.data(), sn.size());
    if (st) return st;
    D.ntiles = (n + kTileRows - 1) / kTileRows;
    {
        std::vector<int32_t> tiled, rn(D.ntiles * kTileRows, -1);
        try {
            tiled.resize((size_t)D.ntiles * k * kTileRows);
        } catch (...) {
            set_last_error("host allocation failed");
            return MZ_ERR_OOM;
        }
        for (int64_t r = 0; r < D.ntiles * kTileRows; ++r) {
            const int64_t tile = r / kTileRows, lane = r % kTileRows;
            int32_t *dst = &tiled[(size_t)tile * k * kTileRows + lane];
            if (r < n) {
                const int32_t *row = &H.N[(size_t)r * k];
                for (int64_t c = 0; c < k; ++c) dst[c * kTileRows] = row[c];
                rn[r] = H.row_node[r];
            } else {
                for (int64_t c = 0; c < k; ++c) dst[c * kTileRows] = 0;  // slot 0 is a zero slot
            }
        }
        if ((st = upload(p, &D.Nt, tiled.data(), tiled.size()))) return st;
        if ((st = upload(p, &D.row_node, rn.data(), rn.size()))) return st;
    }
    {
        const std::vector<int32_t> &lvl = (p->schedule == MZ_SCHED_ANTICHAIN) ? H.level : H.ulevel;
        std::vector<int64_t> order(n);
        for (int64_t r = 0; r < n; ++r) order[r] = r;
        std::stable_sort(order.begin(), order.end(),
                         [&](int64_t a, int64_t b) { return lvl[H.row_node[a]] < lvl[H.row_node[b]]; });
        std::vector<int32_t> Nm, mnode(n), mslot(n), mlevel(n);
        const int64_t kp = (k + 15) / 16 * 16;   // rows padded with slot 0 (a zero slot) in front
        D.kpad = (int32_t)kp;
        try {
            Nm.assign((size_t)n * kp, 0);
        } catch (...) {
            set_last_error("host allocation failed");
            return MZ_ERR_OOM;
        }
        // Each row lists its k slots ordered by the level of the element in them
        // (zero slots first): the kernel adds the latest-finishing ones last.
        std::vector<std::pair<int32_t, int32_t>> cols(k);
        for (int64_t i = 0; i < n; ++i) {
            const int64_t r = order[i];
            const int32_t x = H.row_node[r];
            const int32_t cx = H.chain_id[x];
            const int32_t *src = &H.N[(size_t)r * k];
            for (int64_t c = 0; c < k; ++c) {
                const int32_t slot = (c == cx) ? (int32_t)H.chain_base[cx] : src[c];   // own chain: handled apart
                const int32_t y = H.slot_node[slot];
                cols[c] = {y < 0 ? -1 : lvl[y], slot};
            }
            std::stable_sort(cols.begin(), cols.end(),
                             [](const std::pair<int32_t, int32_t> &a, const std::pair<int32_t, int32_t> &b) {
                                 return a.first < b.first;
                             });
            for (int64_t c = 0; c < k; ++c) Nm[(size_t)i * kp + (kp - k) + c] = cols[c].second;
            mnode[i] = x;
            mslot[i] = H.node_slot[x];
            mlevel[i] = lvl[x];
        }
        if ((st = upload(p, &D.Nm, Nm.data(), Nm.size()))) return st;
        if ((st = upload(p, &D.mob_node, mnode.data(), mnode.size()))) return st;
        if ((st = upload(p, &D.mob_slot, mslot.data(), mslot.size()))) return st;
        if ((st = upload(p, &D.mob_level, mlevel.data(), mlevel.size()))) return st;
    }
    return MZ_OK;
}

// ---------------------------------------------------------------- workspace
struct WsLayout {
    ScanShape sh;
    size_t counters = 0, flags = 0, agg = 0, inc = 0, P = 0, memset_bytes = 0, total = 0;
};

static WsLayout ws_layout(const HostSide &H, int32_t B) {
    WsLayout L;
    const int64_t nslots = H.n + H.k;
    L.sh = scan_shape(nslots, B);
    const size_t tiles = (size_t)L.sh.groups * (size_t)L.sh.ntiles;
    L.counters = 0;
    L.flags = align256(sizeof(uint32_t) * L.sh.groups);
    L.agg = L.flags + align256(sizeof(uint32_t) * tiles);
    L.memset_bytes = L.agg;
    L.inc = L.agg + align256(8 * tiles * L.sh.BW);
    L.P = L.inc + align256(8 * tiles * L.sh.BW);
    L.total = L.P + align256((size_t)8 * (size_t)nslots * (size_t)B);
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
    const HostSide &H = p->host[side];
    *L = ws_layout(H, B);
    if (ws_bytes < L->total || ((uintptr_t)ws & 255)) {
        set_last_error("workspace too small or not 256-byte aligned");
        return MZ_ERR_INVALID_ARG;
    }
    const size_t vb = (size_t)H.n * (size_t)B * 8;   // every dtype: 8 bytes per element
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

static mz_status run_zeta(const mz_plan *p, int side, mz_dtype dtype, const void *f, void *g, int32_t B, void *ws,
                          size_t ws_bytes, mz_stream stream) {
    g_last_launches = 0;
    WsLayout L;
    mz_status st = check_call(p, dtype, f, g, B, ws, ws_bytes, side, &L);
    if (st) return st;
    const HostSide &H = p->host[side];
    const DeviceSide &D = p->dev[side];
    cudaStream_t s = (cudaStream_t)stream;
    char *w = (char *)ws;
    mark_event(0, s);
    cudaError_t e = cudaMemsetAsync(w, 0, L.memset_bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    ScanArgs sa;
    sa.slot_node = D.slot_node;
    sa.nslots = H.n + H.k;
    sa.B = B;
    sa.BW = L.sh.BW;
    sa.R = L.sh.R;
    sa.ntiles = L.sh.ntiles;
    sa.f = f;
    sa.nB = H.n * (int64_t)B;
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
    ga.Nt = D.Nt;
    ga.row_node = D.row_node;
    ga.ntiles = D.ntiles;
    ga.k = H.k;
    ga.B = B;
    ga.P = w + L.P;
    ga.g = g;
    ga.nB = H.n * (int64_t)B;
    if ((e = launch_gather(dtype, ga, p->num_sms, s)) != cudaSuccess) return cuda_fail(e, "niv gather launch");
    mark_event(++g_last_launches, s);
    return MZ_OK;
}

static mz_status run_mobius(const mz_plan *p, int side, mz_dtype dtype, const void *g, void *f, int32_t B, void *ws,
                            size_t ws_bytes, mz_stream stream) {
    g_last_launches = 0;
    WsLayout L;
    mz_status st = check_call(p, dtype, g, f, B, ws, ws_bytes, side, &L);
    if (st) return st;
    const HostSide &H = p->host[side];
    const DeviceSide &D = p->dev[side];
    MobArgs ma;
    ma.Nm = D.Nm;
    ma.kpad = D.kpad;
    ma.blocks_per_sm = p->mob_blocks_per_sm;
    ma.mob_node = D.mob_node;
    ma.mob_slot = D.mob_slot;
    ma.mob_level = D.mob_level;
    ma.pace_ns = p->mob_pace_ns;
    ma.n = H.n;
    ma.k = D.kpad;   // the Moebius kernels walk whole padded rows
    ma.B = B;
    ma.g = g;
    ma.f = f;
    ma.nB = H.n * (int64_t)B;
    ma.P = (unsigned long long *)((char *)ws + L.P);
    ma.status = p->d_status;
    ma.spin_limit = p->spin_limit;
    ma.withhold = p->withhold;
    int launches = 0;
    mark_event(0, (cudaStream_t)stream);
    cudaError_t e = launch_mobius(dtype, ma, D.slot_node, H.n + H.k, p->schedule == MZ_SCHED_ANTICHAIN, p->num_sms,
                                  (cudaStream_t)stream, &launches);
    g_last_launches = launches;
    if (e != cudaSuccess) return cuda_fail(e, "moebius launch");
    return MZ_OK;
}

}  // namespace mz

using namespace mz;

extern "C" {

mz_status mz_build(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *chain_id,
                   const mz_build_opts *opts, mz_plan **out) {
    if (out) *out = nullptr;
    if (!out || n < 1 || n > (int64_t(1) << 30) || m < 0 || (m > 0 && (!src || !dst))) {
        set_last_error("invalid sizes or null pointers");
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
        std::vector<int32_t> s(src, src + m), d(dst, dst + m);
        std::string err;
        mz_status st = build_host_side(n, s, d, chain_id, p->host[0], err);
        if (st) {
            set_last_error(err);
            return st;
        }
        if (o.build_transpose) {
            // the dual poset: every edge flipped, the same chains (a chain of P is a chain of its dual)
            st = build_host_side(n, d, s, p->host[0].chain_id.data(), p->host[1], err);
            if (st) {
                set_last_error("dual: " + err);
                return st;
            }
            p->has_dual = true;
        }
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return MZ_ERR_OOM;
    }
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
        mz_status st = MZ_OK;
        p->d_status = (uint32_t *)plan_alloc(p.get(), 256);
        if (!p->d_status) st = MZ_ERR_OOM;
        else if ((e = cudaMemset(p->d_status, 0, 256)) != cudaSuccess) st = cuda_fail(e, "cudaMemset");
        for (int side = 0; side < (p->has_dual ? 2 : 1) && st == MZ_OK; ++side) st = upload_side(p.get(), side);
        if (st) {
            if (st == MZ_ERR_OOM) set_last_error("device allocation failed");
            plan_free_all(p.get());
            return st;
        }
    }
    *out = p.release();
    return MZ_OK;
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
    size_t b = ws_layout(plan->host[0], batch).total;
    if (plan->has_dual) b = std::max(b, ws_layout(plan->host[1], batch).total);
    *bytes = b;
    return MZ_OK;
}

mz_status mz_zeta(const mz_plan *plan, mz_dtype dtype, const void *f, void *g, int32_t batch, void *ws,
                  size_t ws_bytes, mz_stream stream) {
    return run_zeta(plan, 0, dtype, f, g, batch, ws, ws_bytes, stream);
}

// ---------------------------------------------------------------- zeta without allocation
// Scratch for mz_zeta_noalloc: a fixed device array owned by the library. Its
// name is only a host-side handle; the device address comes from
// cudaGetSymbolAddress, looked up once per device on the first call there.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MZ_NOALLOC_SCRATCH_BYTES];
static void *g_noalloc_addr[128];
static std::mutex g_noalloc_mutex;

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
    const size_t need = ws_layout(plan->host[0], batch).total;
    if (need > MZ_NOALLOC_SCRATCH_BYTES) {
        set_last_error("mz_zeta_noalloc: this plan and batch need " + std::to_string(need) +
                       " bytes of scratch; the fixed scratch array holds " +
                       std::to_string((size_t)MZ_NOALLOC_SCRATCH_BYTES) + " (use mz_zeta with a workspace)");
        return MZ_ERR_INVALID_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 128) {
        set_last_error("device index out of range");
        return MZ_ERR_INVALID_ARG;
    }
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_addr[dev]) {
            e = cudaGetSymbolAddress(&g_noalloc_addr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_noalloc_addr[dev] = nullptr;
                return cuda_fail(e, "cudaGetSymbolAddress");
            }
        }
        ws = g_noalloc_addr[dev];
    }
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

mz_status mz_plan_info(const mz_plan *plan, mz_plan_info_t *info) {
    if (!plan || !info) return MZ_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    const HostSide &H = plan->host[0];
    info->n = H.n;
    info->k = H.k;
    info->has_transpose = plan->has_dual;
    info->nnz = H.nnz;
    info->edges = H.edges;
    info->levels = H.nlevels;
    info->ulevels = H.nulevels;
    info->schedule = plan->schedule;
    if (plan->has_dual) {
        info->levels_T = plan->host[1].nlevels;
        info->ulevels_T = plan->host[1].nulevels;
    }
    info->max_chain = H.max_chain;
    info->device_bytes = plan->device_bytes;
    return MZ_OK;
}

mz_status mz_plan_export(const mz_plan *plan, int32_t what, int32_t dual, void *out, size_t bytes) {
    if (!plan || !out || (dual && !plan->has_dual)) {
        set_last_error("invalid argument");
        return MZ_ERR_INVALID_ARG;
    }
    const HostSide &H = plan->host[dual ? 1 : 0];
    const int64_t n = H.n, k = H.k;
    std::vector<int32_t> tmp;
    const int32_t *src = nullptr;
    size_t count = (size_t)n;
    switch (what) {
        case MZ_EXPORT_CHAIN_ID: src = H.chain_id.data(); break;
        case MZ_EXPORT_CHAIN_POS: src = H.chain_pos.data(); break;
        case MZ_EXPORT_LEVEL: src = H.level.data(); break;
        case MZ_EXPORT_ULEVEL: src = H.ulevel.data(); break;
        case MZ_EXPORT_TOPO: src = H.topo.data(); break;
        case MZ_EXPORT_NIV: {
            count = (size_t)n * (size_t)k;
            if (bytes < count * sizeof(int32_t)) break;
            int32_t *o = (int32_t *)out;
            for (int64_t x = 0; x < n; ++x) {
                const int64_t cx = H.chain_id[x];
                const int32_t *row = &H.N[(size_t)(H.node_slot[x] - cx - 1) * k];
                for (int64_t c = 0; c < k; ++c)
                    o[x * k + c] = row[c] == (int32_t)H.chain_base[c] ? -1 : H.slot_node[row[c]];
            }
            return MZ_OK;
        }
        default:
            set_last_error("unknown export");
            return MZ_ERR_INVALID_ARG;
    }
    if (bytes < count * sizeof(int32_t)) {
        set_last_error("output buffer too small");
        return MZ_ERR_INVALID_ARG;
    }
    if (src) std::memcpy(out, src, count * sizeof(int32_t));
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
    }
    return "unknown status";
}

const char *mz_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
