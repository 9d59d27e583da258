// Plan files: the host side of a plan (every poset, the dual included) written to a
// file and read back, so that the one-time precomputation (chains by Alg. 1, the niv
// map by Thm. 4, heights and U levels) is done once and reused.
//
// Layout (little-endian, the sizes of the writing machine's types): an 8-byte magic
// and a version, the plan's flags and its number of posets, then per side and poset
// the scalars and arrays of its HostSide, each array as a 64-bit count and its
// elements, and last a 64-bit FNV-1a hash of all bytes before it. Reading checks the
// magic, the version, the hash, every array length against n and k, and every index
// against its range (slots, nodes, chains, levels, the chain layout), so that no file
// can make a kernel read outside an array; a file that passes the checks but was not
// written by mz_plan_save gives wrong transforms, not faults.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mz_internal.h"

namespace mz {

namespace {

constexpr char kMagic[8] = {'M', 'Z', 'P', 'L', 'A', 'N', '\0', '\1'};
constexpr uint32_t kVersion = 1;

uint64_t fnv1a(const std::vector<unsigned char> &b, size_t len) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < len; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct Writer {
    std::vector<unsigned char> buf;
    template <class T>
    void put(const T &v) {
        const unsigned char *p = reinterpret_cast<const unsigned char *>(&v);
        buf.insert(buf.end(), p, p + sizeof(T));
    }
    template <class T>
    void vec(const std::vector<T> &v) {
        put<uint64_t>((uint64_t)v.size());
        const unsigned char *p = reinterpret_cast<const unsigned char *>(v.data());
        buf.insert(buf.end(), p, p + sizeof(T) * v.size());
    }
};

struct Reader {
    const std::vector<unsigned char> &buf;
    size_t pos, end;
    bool ok = true;
    template <class T>
    T get() {
        T v{};
        if (!ok || end - pos < sizeof(T)) {
            ok = false;
            return v;
        }
        std::memcpy(&v, buf.data() + pos, sizeof(T));
        pos += sizeof(T);
        return v;
    }
    template <class T>
    void vec(std::vector<T> &v, uint64_t max_count) {
        const uint64_t count = get<uint64_t>();
        if (!ok || count > max_count || (end - pos) / sizeof(T) < count) {
            ok = false;
            return;
        }
        v.resize((size_t)count);
        std::memcpy(v.data(), buf.data() + pos, sizeof(T) * (size_t)count);
        pos += sizeof(T) * (size_t)count;
    }
};

void write_side(Writer &w, const HostSide &H) {
    w.put<int64_t>(H.n);
    w.put<int32_t>(H.k);
    w.put<int64_t>(H.edges);
    w.put<int64_t>(H.nnz);
    w.put<int32_t>(H.nlevels);
    w.put<int32_t>(H.nulevels);
    w.put<int32_t>(H.max_chain);
    w.put<int32_t>(H.sparse ? 1 : 0);
    w.vec(H.topo);
    w.vec(H.chain_id);
    w.vec(H.chain_pos);
    w.vec(H.chain_base);
    w.vec(H.node_slot);
    w.vec(H.slot_node);
    w.vec(H.row_node);
    w.vec(H.N);
    w.vec(H.row_beg);
    w.vec(H.row_len);
    w.vec(H.ent_chain);
    w.vec(H.ent_slot);
    w.vec(H.level);
    w.vec(H.ulevel);
}

// Every length and index of one side, as the kernels and the uploads rely on them.
bool check_side(const HostSide &H, std::string &why) {
    const int64_t n = H.n, k = H.k, ns = n + k;
    auto bad = [&](const char *what) {
        why = what;
        return false;
    };
    if (n < 1 || k < 1 || k > n || ns >= (int64_t)INT32_MAX) return bad("sizes");
    if ((int64_t)H.topo.size() != n || (int64_t)H.chain_id.size() != n || (int64_t)H.chain_pos.size() != n ||
        (int64_t)H.chain_base.size() != k + 1 || (int64_t)H.node_slot.size() != n ||
        (int64_t)H.slot_node.size() != ns || (int64_t)H.row_node.size() != n || (int64_t)H.level.size() != n ||
        (int64_t)H.ulevel.size() != n)
        return bad("array lengths");
    if (H.nlevels < 1 || H.nulevels < 1 || H.max_chain < 1 || H.max_chain > n) return bad("level counts");
    std::vector<char> seen((size_t)n, 0);
    for (int32_t x : H.topo) {
        if (x < 0 || x >= n || seen[(size_t)x]) return bad("topological order");
        seen[(size_t)x] = 1;
    }
    if (H.chain_base[0] != 0 || H.chain_base[(size_t)k] != ns) return bad("chain layout");
    for (int64_t c = 0; c < k; ++c)
        if (H.chain_base[(size_t)c + 1] <= H.chain_base[(size_t)c] ||
            H.chain_base[(size_t)c + 1] - H.chain_base[(size_t)c] - 1 > H.max_chain)
            return bad("chain layout");
    for (int64_t s = 0; s < ns; ++s)
        if (H.slot_node[(size_t)s] < -1 || H.slot_node[(size_t)s] >= n) return bad("slot map");
    for (int64_t c = 0; c < k; ++c)
        if (H.slot_node[(size_t)H.chain_base[(size_t)c]] != -1) return bad("zero slots");
    for (int64_t x = 0; x < n; ++x) {
        const int64_t c = H.chain_id[(size_t)x], p = H.chain_pos[(size_t)x];
        if (c < 0 || c >= k || p < 0) return bad("chains");
        const int64_t s = H.chain_base[(size_t)c] + 1 + p;
        if (s >= H.chain_base[(size_t)c + 1] || H.node_slot[(size_t)x] != s || H.slot_node[(size_t)s] != x)
            return bad("slots");
        if (H.level[(size_t)x] < 1 || H.level[(size_t)x] > H.nlevels || H.ulevel[(size_t)x] < 0 ||
            H.ulevel[(size_t)x] >= H.nulevels)
            return bad("levels");
    }
    for (int64_t r = 0; r < n; ++r) {
        const int32_t x = H.row_node[(size_t)r];
        if (x < 0 || x >= n || H.node_slot[(size_t)x] - H.chain_id[(size_t)x] - 1 != r) return bad("rows");
    }
    if (!H.sparse) {
        if ((int64_t)H.N.size() != n * k || !H.row_beg.empty() || !H.ent_slot.empty()) return bad("dense map");
        for (int32_t s : H.N)
            if (s < 0 || s >= ns) return bad("dense map entries");
    } else {
        if (!H.N.empty() || (int64_t)H.row_beg.size() != n || (int64_t)H.row_len.size() != n ||
            H.ent_chain.size() != H.ent_slot.size())
            return bad("sparse map");
        const int64_t ne = (int64_t)H.ent_slot.size();
        for (int64_t r = 0; r < n; ++r) {
            const int64_t b = H.row_beg[(size_t)r], l = H.row_len[(size_t)r];
            if (b < 0 || l < 1 || l > k || b > ne - l) return bad("sparse rows");
        }
        for (int64_t q = 0; q < ne; ++q)
            if (H.ent_slot[(size_t)q] < 0 || H.ent_slot[(size_t)q] >= ns || H.ent_chain[(size_t)q] < 0 ||
                H.ent_chain[(size_t)q] >= k)
                return bad("sparse map entries");
    }
    return true;
}

bool read_side(Reader &r, HostSide &H, std::string &why) {
    H = HostSide();
    H.n = r.get<int64_t>();
    H.k = r.get<int32_t>();
    H.edges = r.get<int64_t>();
    H.nnz = r.get<int64_t>();
    H.nlevels = r.get<int32_t>();
    H.nulevels = r.get<int32_t>();
    H.max_chain = r.get<int32_t>();
    H.sparse = r.get<int32_t>() != 0;
    if (!r.ok || H.n < 1 || H.n > ((int64_t)1 << 30) || H.k < 1 || H.k > H.n) {
        why = "sizes";
        return false;
    }
    const uint64_t n = (uint64_t)H.n, k = (uint64_t)H.k;
    r.vec(H.topo, n);
    r.vec(H.chain_id, n);
    r.vec(H.chain_pos, n);
    r.vec(H.chain_base, k + 1);
    r.vec(H.node_slot, n);
    r.vec(H.slot_node, n + k);
    r.vec(H.row_node, n);
    r.vec(H.N, n * k);
    r.vec(H.row_beg, n);
    r.vec(H.row_len, n);
    r.vec(H.ent_chain, n * k);
    r.vec(H.ent_slot, n * k);
    r.vec(H.level, n);
    r.vec(H.ulevel, n);
    if (!r.ok) {
        why = "truncated or oversized array";
        return false;
    }
    return check_side(H, why);
}

}  // namespace

mz_status save_host_sides(const mz_plan *p, const char *path, std::string &err) {
    Writer w;
    try {
        w.buf.insert(w.buf.end(), kMagic, kMagic + 8);
        w.put<uint32_t>(kVersion);
        w.put<uint32_t>(p->has_dual ? 1u : 0u);
        w.put<int32_t>((int32_t)p->components());
        w.put<int32_t>(0);
        for (int side = 0; side < (p->has_dual ? 2 : 1); ++side)
            for (const HostSide &H : p->host[side]) write_side(w, H);
        w.put<uint64_t>(fnv1a(w.buf, w.buf.size()));
    } catch (const std::bad_alloc &) {
        err = "host allocation failed";
        return MZ_ERR_OOM;
    }
    FILE *f = std::fopen(path, "wb");
    if (!f) {
        err = std::string("cannot open ") + path + " for writing";
        return MZ_ERR_INVALID_ARG;
    }
    const bool ok = std::fwrite(w.buf.data(), 1, w.buf.size(), f) == w.buf.size();
    if (std::fclose(f) != 0 || !ok) {
        err = std::string("cannot write ") + path;
        return MZ_ERR_INVALID_ARG;
    }
    return MZ_OK;
}

mz_status load_host_sides(mz_plan *p, const char *path, std::string &err) {
    FILE *f = std::fopen(path, "rb");
    if (!f) {
        err = std::string("cannot open ") + path;
        return MZ_ERR_INVALID_ARG;
    }
    std::vector<unsigned char> buf;
    try {
        unsigned char chunk[1 << 16];
        size_t got;
        while ((got = std::fread(chunk, 1, sizeof(chunk), f)) > 0) buf.insert(buf.end(), chunk, chunk + got);
    } catch (const std::bad_alloc &) {
        std::fclose(f);
        err = "host allocation failed";
        return MZ_ERR_OOM;
    }
    std::fclose(f);
    auto bad = [&](const std::string &why) {
        err = std::string("not a valid plan file (") + why + "): " + path;
        return MZ_ERR_INVALID_ARG;
    };
    if (buf.size() < 8 + 4 + 4 + 4 + 4 + 8 || std::memcmp(buf.data(), kMagic, 8) != 0) return bad("magic");
    uint64_t stored;
    std::memcpy(&stored, buf.data() + buf.size() - 8, 8);
    if (stored != fnv1a(buf, buf.size() - 8)) return bad("checksum");
    Reader r{buf, 8, buf.size() - 8};
    const uint32_t version = r.get<uint32_t>(), flags = r.get<uint32_t>();
    const int32_t count = r.get<int32_t>();
    r.get<int32_t>();
    if (version != kVersion) return bad("version");
    if (flags > 1 || count < 1 || count > (1 << 24)) return bad("header");
    try {
        p->has_dual = flags == 1;
        for (int side = 0; side < (p->has_dual ? 2 : 1); ++side) {
            p->host[side].resize((size_t)count);
            for (int32_t c = 0; c < count; ++c) {
                std::string why;
                if (!read_side(r, p->host[side][(size_t)c], why))
                    return bad((count > 1 ? "poset " + std::to_string(c) + ": " : std::string()) +
                               (side ? "dual: " : "") + why);
            }
        }
    } catch (const std::bad_alloc &) {
        err = "host allocation failed";
        return MZ_ERR_OOM;
    }
    if (r.pos != r.end) return bad("trailing bytes");
    if (p->has_dual)
        for (int32_t c = 0; c < count; ++c)
            if (p->host[1][(size_t)c].n != p->host[0][(size_t)c].n || p->host[1][(size_t)c].k != p->host[0][(size_t)c].k)
                return bad("dual sizes");
    int64_t total = 0, slots = 0;
    p->node_off.assign((size_t)count + 1, 0);
    p->slot_off.assign((size_t)count + 1, 0);
    p->chain_off.assign((size_t)count + 1, 0);
    for (int32_t c = 0; c < count; ++c) {
        const HostSide &H = p->host[0][(size_t)c];
        p->node_off[(size_t)c + 1] = p->node_off[(size_t)c] + H.n;
        p->chain_off[(size_t)c + 1] = p->chain_off[(size_t)c] + H.k;
        p->slot_off[(size_t)c + 1] = p->slot_off[(size_t)c] + H.n + H.k;
        total += H.n;
        slots += H.n + H.k;
    }
    if (total > ((int64_t)1 << 30) || slots >= (int64_t)INT32_MAX) return bad("plan too large");
    return MZ_OK;
}

}  // namespace mz
