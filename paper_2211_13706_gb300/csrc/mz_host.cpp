// Host-side precomputation of a plan (arxiv 2211.13706, Sec. 2.3, 2.4, 4).
//
//   1. validate the edge list and remove duplicates;
//   2. topological order by Kahn's algorithm (Sec. 2.1: x < y puts x after y);
//   3. a chain decomposition (Def. 1): the caller's, or a minimum path cover
//      of the DAG by maximum bipartite matching (Alg. 1, Hopcroft-Karp);
//   4. the slot layout of the chain prefix array (see mz_internal.h);
//   5. the niv map by Thm. 4 (Alg. 2), bottom-up, with the caller's chains
//      checked on the way;
//   6. antichain levels (Alg. 6, heights) and the levels of U's dependency
//      graph (the schedule of the forward substitution of Alg. 4).
// With the device build only steps 1-4 and the heights run here; mz_build.cu
// has the rest.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "mz_internal.h"

namespace mz {

namespace {

thread_local int t_threads_cap = 0;   // set by callers that already run builds in parallel

// Host threads for the parallel parts of the build: MZ_HOST_THREADS if set (tests use 1
// to compare with the one-thread order), else the hardware's, at most 64; 1 inside a
// build that already runs on one of several threads (many posets at once).
int host_threads() {
    const char *e = std::getenv("MZ_HOST_THREADS");
    int t = e ? std::atoi(e) : (int)std::thread::hardware_concurrency();
    if (t_threads_cap > 0) t = std::min(t, t_threads_cap);
    return std::max(1, std::min(64, t));
}

// Runs fn(thread, begin, end) over [0, count) in contiguous pieces, one per host
// thread, when the range is large enough to pay for the threads; else inline.
template <class F>
void for_pieces(int64_t count, int nthreads, F fn) {
    if (nthreads <= 1 || count < 4096) {
        fn(0, (int64_t)0, count);
        return;
    }
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t)
        pool.emplace_back([&, t]() { fn(t, count * t / nthreads, count * (t + 1) / nthreads); });
    for (auto &th : pool) th.join();
}

// Maximum matching between "upper" copies (edge sources) and "lower" copies (edge
// targets) of the nodes (Alg. 1's bipartite graph G'): a Karp-Sipser start (Karp and
// Sipser 1981), then Hopcroft-Karp phases (Hopcroft and Karp 1973) until no augmenting
// path is left. On the paper's random DAGs the start is already maximum.
// Returns next_of[u] = the node matched below u, or -1.
std::vector<int32_t> max_matching(int64_t n, const std::vector<int64_t> &ptr, const std::vector<int32_t> &adj) {
    const int32_t NIL = -1;
    std::vector<int32_t> mate_u(n, NIL), mate_v(n, NIL), dist(n), queue(n);
    std::vector<int64_t> it(n);
    std::vector<int32_t> stack;
    // Karp-Sipser start: match vertices left with one free neighbour first (such an edge is in
    // some maximum matching), else any free edge; the phases below then finish the job.
    {
        std::vector<int64_t> pptr(n + 1, 0);
        for (int64_t e = 0; e < (int64_t)adj.size(); ++e) pptr[adj[e] + 1]++;
        for (int64_t v = 0; v < n; ++v) pptr[v + 1] += pptr[v];
        std::vector<int32_t> padj(adj.size());
        {
            std::vector<int64_t> fill(pptr.begin(), pptr.end() - 1);
            for (int64_t u = 0; u < n; ++u)
                for (int64_t e = ptr[u]; e < ptr[u + 1]; ++e) padj[fill[adj[e]]++] = (int32_t)u;
        }
        std::vector<int32_t> deg_u(n), deg_v(n);
        for (int64_t u = 0; u < n; ++u) deg_u[u] = (int32_t)(ptr[u + 1] - ptr[u]);
        for (int64_t v = 0; v < n; ++v) deg_v[v] = (int32_t)(pptr[v + 1] - pptr[v]);
        std::vector<int64_t> one;   // degree-1 vertices: u as u, v as -(v + 1)
        for (int64_t u = 0; u < n; ++u) if (deg_u[u] == 1) one.push_back(u);
        for (int64_t v = 0; v < n; ++v) if (deg_v[v] == 1) one.push_back(-(v + 1));
        auto take = [&](int32_t u, int32_t v) {   // match u-v, remove both, update degrees
            mate_u[u] = v;
            mate_v[v] = u;
            for (int64_t e = ptr[u]; e < ptr[u + 1]; ++e) {
                const int32_t w = adj[e];
                if (mate_v[w] == NIL && --deg_v[w] == 1) one.push_back(-(int64_t)w - 1);
            }
            for (int64_t e = pptr[v]; e < pptr[v + 1]; ++e) {
                const int32_t w = padj[e];
                if (mate_u[w] == NIL && --deg_u[w] == 1) one.push_back(w);
            }
        };
        int64_t next_u = 0;
        while (true) {
            while (!one.empty()) {
                const int64_t t = one.back();
                one.pop_back();
                if (t >= 0) {
                    const int32_t u = (int32_t)t;
                    if (mate_u[u] != NIL || deg_u[u] != 1) continue;
                    for (int64_t e = ptr[u]; e < ptr[u + 1]; ++e)
                        if (mate_v[adj[e]] == NIL) { take(u, adj[e]); break; }
                } else {
                    const int32_t v = (int32_t)(-t - 1);
                    if (mate_v[v] != NIL || deg_v[v] != 1) continue;
                    for (int64_t e = pptr[v]; e < pptr[v + 1]; ++e)
                        if (mate_u[padj[e]] == NIL) { take(padj[e], v); break; }
                }
            }
            // no degree-1 vertex left: one greedy edge, then look again
            while (next_u < n && (mate_u[next_u] != NIL || deg_u[next_u] == 0)) ++next_u;
            if (next_u >= n) break;
            bool any = false;
            for (int64_t e = ptr[next_u]; e < ptr[next_u + 1]; ++e)
                if (mate_v[adj[e]] == NIL) { take((int32_t)next_u, adj[e]); any = true; break; }
            if (!any) deg_u[next_u] = 0;
        }
    }
    const int32_t INF = INT32_MAX;
    while (true) {
        // BFS from free upper nodes over alternating paths
        int64_t qh = 0, qt = 0;
        bool found = false;
        for (int64_t u = 0; u < n; ++u) {
            if (mate_u[u] == NIL) { dist[u] = 0; queue[qt++] = (int32_t)u; }
            else dist[u] = INF;
        }
        while (qh < qt) {
            int32_t u = queue[qh++];
            for (int64_t e = ptr[u]; e < ptr[u + 1]; ++e) {
                int32_t w = mate_v[adj[e]];
                if (w == NIL) found = true;
                else if (dist[w] == INF) { dist[w] = dist[u] + 1; queue[qt++] = w; }
            }
        }
        if (!found) break;
        // iterative DFS along the layered graph
        for (int64_t u = 0; u < n; ++u) it[u] = ptr[u];
        for (int64_t s = 0; s < n; ++s) {
            if (mate_u[s] != NIL) continue;
            stack.clear();
            stack.push_back((int32_t)s);
            while (!stack.empty()) {
                int32_t u = stack.back();
                bool advanced = false;
                while (it[u] < ptr[u + 1]) {
                    int32_t v = adj[it[u]];
                    int32_t w = mate_v[v];
                    if (w == NIL) {
                        // augment along the stack: each stacked node takes the edge it[] points at
                        for (size_t i = stack.size(); i-- > 0;) {
                            int32_t a = stack[i];
                            int32_t b = adj[it[a]];
                            mate_u[a] = b;
                            mate_v[b] = a;
                        }
                        stack.clear();
                        advanced = true;
                        break;
                    }
                    if (dist[w] == dist[u] + 1) { stack.push_back(w); advanced = true; break; }
                    ++it[u];
                }
                if (!advanced) {           // dead end: drop u from the layered graph
                    dist[u] = INF;
                    stack.pop_back();
                    if (!stack.empty()) ++it[stack.back()];
                }
            }
        }
    }
    return mate_u;
}

}  // namespace

void set_host_threads_cap(int cap) { t_threads_cap = cap; }

mz_status build_host_side(int64_t n, const std::vector<int32_t> &src_in, const std::vector<int32_t> &dst_in,
                          const int32_t *chain_in, int niv_format, bool device_niv, HostSide &H, std::string &err,
                          const Matcher *matcher) {
    H = HostSide();
    H.n = n;
    const int64_t m = (int64_t)src_in.size();
    // ---- 1. validate, dedupe, CSR of children
    for (int64_t i = 0; i < m; ++i) {
        if (src_in[i] < 0 || src_in[i] >= n || dst_in[i] < 0 || dst_in[i] >= n) {
            err = "edge " + std::to_string(i) + " has a node id outside [0, n)";
            return MZ_ERR_INVALID_ARG;
        }
        if (src_in[i] == dst_in[i]) {
            err = "edge " + std::to_string(i) + " is a self-loop";
            return MZ_ERR_CYCLE;
        }
    }
    std::vector<int64_t> ptr(n + 1, 0);
    for (int64_t i = 0; i < m; ++i) ptr[src_in[i] + 1]++;
    for (int64_t x = 0; x < n; ++x) ptr[x + 1] += ptr[x];
    std::vector<int32_t> adj(m);
    {
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t i = 0; i < m; ++i) adj[fill[src_in[i]]++] = dst_in[i];
    }
    {   // sort each child list and count its distinct children (in parallel over nodes),
        // then compact
        std::vector<int64_t> uptr(n + 1, 0);
        for_pieces(n, host_threads(), [&](int, int64_t x0, int64_t x1) {
            for (int64_t x = x0; x < x1; ++x) {
                const int64_t b = ptr[x], e = ptr[x + 1];
                std::sort(adj.begin() + b, adj.begin() + e);
                int64_t u = 0;
                for (int64_t i = b; i < e; ++i) u += (i == b || adj[i] != adj[i - 1]);
                uptr[x + 1] = u;
            }
        });
        for (int64_t x = 0; x < n; ++x) uptr[x + 1] += uptr[x];
        std::vector<int32_t> uadj((size_t)uptr[n]);
        for_pieces(n, host_threads(), [&](int, int64_t x0, int64_t x1) {
            for (int64_t x = x0; x < x1; ++x) {
                int64_t w = uptr[x];
                for (int64_t i = ptr[x]; i < ptr[x + 1]; ++i)
                    if (i == ptr[x] || adj[i] != adj[i - 1]) uadj[(size_t)w++] = adj[i];
            }
        });
        ptr.swap(uptr);
        adj.swap(uadj);
    }
    H.edges = (int64_t)adj.size();

    // ---- 2. Kahn's algorithm from the maximal elements
    std::vector<int32_t> indeg(n, 0);
    for (int32_t v : adj) indeg[v]++;
    H.topo.resize(n);
    int64_t head = 0, tail = 0;
    for (int64_t x = 0; x < n; ++x)
        if (indeg[x] == 0) H.topo[tail++] = (int32_t)x;
    while (head < tail) {
        int32_t x = H.topo[head++];
        for (int64_t e = ptr[x]; e < ptr[x + 1]; ++e)
            if (--indeg[adj[e]] == 0) H.topo[tail++] = adj[e];
    }
    if (tail != n) {
        err = "the edges contain a cycle";
        return MZ_ERR_CYCLE;
    }
    std::vector<int32_t> pos(n);
    for (int64_t i = 0; i < n; ++i) pos[H.topo[i]] = (int32_t)i;

    // ---- 3. chain decomposition
    H.chain_id.assign(n, -1);
    std::vector<std::vector<int32_t>> chains;  // members, bottom first
    if (chain_in) {
        std::vector<int32_t> ids(chain_in, chain_in + n);
        std::vector<int32_t> uniq(ids);
        std::sort(uniq.begin(), uniq.end());
        uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
        chains.resize(uniq.size());
        for (int64_t x = 0; x < n; ++x) {
            int32_t c = (int32_t)(std::lower_bound(uniq.begin(), uniq.end(), ids[x]) - uniq.begin());
            H.chain_id[x] = c;
        }
        // members in topological order, reversed (bottom first)
        for (int64_t i = n - 1; i >= 0; --i) chains[H.chain_id[H.topo[i]]].push_back(H.topo[i]);
    } else {
        std::vector<int32_t> next;
        if (matcher) {
            const mz_status st = (*matcher)(n, ptr, adj, next, err);
            if (st) return st;
        } else {
            next = max_matching(n, ptr, adj);
        }
        std::vector<char> has_pred(n, 0);
        for (int64_t u = 0; u < n; ++u)
            if (next[u] >= 0) has_pred[next[u]] = 1;
        for (int64_t i = 0; i < n; ++i) {       // chain heads in topological order
            int32_t x = H.topo[i];
            if (has_pred[x]) continue;
            std::vector<int32_t> members;
            for (int32_t y = x; y >= 0; y = next[y]) members.push_back(y);
            std::reverse(members.begin(), members.end());
            for (int32_t y : members) H.chain_id[y] = (int32_t)chains.size();
            chains.push_back(std::move(members));
        }
    }
    const int64_t k = (int64_t)chains.size();
    if (k < 1 || n + k > (int64_t)INT32_MAX) {
        err = "too many nodes plus chains for 32-bit slot indices";
        return MZ_ERR_INVALID_ARG;
    }
    H.k = (int32_t)k;

    // ---- 4. slot layout
    H.chain_base.assign(k + 1, 0);
    H.chain_pos.assign(n, 0);
    H.node_slot.assign(n, 0);
    H.slot_node.assign(n + k, -1);
    H.row_node.assign(n, 0);
    {
        int64_t base = 0, row = 0;
        for (int64_t c = 0; c < k; ++c) {
            H.chain_base[c] = base;
            H.max_chain = std::max<int32_t>(H.max_chain, (int32_t)chains[c].size());
            for (size_t p = 0; p < chains[c].size(); ++p) {
                int32_t x = chains[c][p];
                H.chain_pos[x] = (int32_t)p;
                H.node_slot[x] = (int32_t)(base + 1 + (int64_t)p);
                H.slot_node[base + 1 + p] = x;
                H.row_node[row++] = x;
            }
            base += (int64_t)chains[c].size() + 1;
        }
        H.chain_base[k] = base;
    }

    if (device_niv) {
        // Steps 5 and the U levels of step 6 run on the device (dense or sparse map, as
        // below); the host keeps the children lists for the upload and computes the
        // heights (one pass over the edges).
        H.sparse = niv_format == 2 || (niv_format == 0 && k > kDenseMaxChains);
        if (!H.sparse && k > kDenseMaxChains) {
            err = "the device build keeps a dense niv map for k <= " + std::to_string(kDenseMaxChains) +
                  " chains only (this poset has " + std::to_string(k) + "); use niv_format 0 or 2";
            return MZ_ERR_UNSUPPORTED;
        }
        H.niv_on_device = true;
        H.level.assign(n, 1);
        for (int64_t i = n - 1; i >= 0; --i) {
            const int32_t x = H.topo[i];
            int32_t h = 0;
            for (int64_t e = ptr[x]; e < ptr[x + 1]; ++e) h = std::max(h, H.level[adj[e]]);
            H.level[x] = h + 1;
        }
        H.nlevels = *std::max_element(H.level.begin(), H.level.end());
        H.csr_ptr = std::move(ptr);
        H.csr_adj = std::move(adj);
        return MZ_OK;
    }

    // ---- 5. niv map by Thm. 4, bottom-up. Entry (x, c) = slot of niv_c(x), or base_c.
    // The caller's chains are checked here: the element below x on its chain, or the
    // chain's zero slot when x is the bottom, must be exactly the highest element of
    // x's chain reachable through x's children.
    // Dense form: one k-wide row per node. Sparse form (Sec. 2.4's nnz(N)): only the
    // finite entries, as (chain, slot) pairs sorted by chain; chosen when k is large.
    H.sparse = niv_format == 2 || (niv_format == 0 && k > kDenseMaxChains);
    std::vector<int32_t> base32(k);
    for (int64_t c = 0; c < k; ++c) base32[c] = (int32_t)H.chain_base[c];
    std::vector<int32_t> kids;
    auto bad_chain = [&](int32_t cx, int32_t x) {
        err = "chain " + std::to_string(cx) + " is not totally ordered at node " + std::to_string(x);
        return MZ_ERR_BAD_CHAINS;
    };
    if (!H.sparse) {
        try {
            H.N.assign((size_t)n * (size_t)k, 0);
        } catch (...) {
            err = "host allocation of the niv map failed";
            return MZ_ERR_OOM;
        }
        std::vector<int32_t> cur(k);
        for (int64_t i = n - 1; i >= 0; --i) {
            int32_t x = H.topo[i];
            std::memcpy(cur.data(), base32.data(), sizeof(int32_t) * k);
            kids.assign(adj.begin() + ptr[x], adj.begin() + ptr[x + 1]);
            // highest children first: a child already covered adds nothing (G3 pruning)
            std::sort(kids.begin(), kids.end(), [&](int32_t a, int32_t b) { return pos[a] < pos[b]; });
            for (int32_t z : kids) {
                const int32_t cz = H.chain_id[z];
                if (cur[cz] >= H.node_slot[z]) continue;
                const int32_t *row = &H.N[(size_t)(H.node_slot[z] - cz - 1) * k];
                for (int64_t c = 0; c < k; ++c) cur[c] = std::max(cur[c], row[c]);
            }
            const int32_t cx = H.chain_id[x];
            const int32_t sx = H.node_slot[x];
            if (cur[cx] != sx - 1) return bad_chain(cx, x);
            cur[cx] = sx;
            std::memcpy(&H.N[(size_t)(sx - cx - 1) * k], cur.data(), sizeof(int32_t) * k);
        }
        H.nnz = 0;
        for (int64_t r = 0; r < n; ++r) {
            const int32_t *row = &H.N[(size_t)r * k];
            for (int64_t c = 0; c < k; ++c) H.nnz += row[c] != base32[c];
        }
    } else {
        // Level by level (heights): every child of a node sits on a lower level, so the
        // nodes of one level merge their children's finished rows independently, on all
        // host threads. Each thread keeps a scratch row (the merged row of the node it
        // builds; `touched` lists its chains) and appends to its own entry buffers, which
        // are concatenated after the level. A node that breaks its chain is recorded and
        // the build goes on; the one reported is the one the sequential order (topological
        // position, highest first) would meet first, whose descendants all passed.
        std::vector<int32_t> height(n, 1);
        for (int64_t i = n - 1; i >= 0; --i) {
            const int32_t x = H.topo[i];
            int32_t h = 0;
            for (int64_t e = ptr[x]; e < ptr[x + 1]; ++e) h = std::max(h, height[adj[e]]);
            height[x] = h + 1;
        }
        const int32_t nh = *std::max_element(height.begin(), height.end());
        std::vector<int64_t> lstart((size_t)nh + 2, 0);
        for (int64_t x = 0; x < n; ++x) lstart[height[x]]++;
        for (size_t l = 1; l < lstart.size(); ++l) lstart[l] += lstart[l - 1];
        std::vector<int32_t> by_level((size_t)n);
        {
            std::vector<int64_t> fill(lstart);
            for (int64_t i = n - 1; i >= 0; --i) by_level[(size_t)fill[height[H.topo[i]] - 1]++] = H.topo[i];
        }
        H.row_beg.assign(n, 0);
        H.row_len.assign(n, 0);
        H.ent_chain.clear();
        H.ent_slot.clear();
        const int T = host_threads();
        struct Local {
            std::vector<int32_t> scratch, touched, kids, chain, slot;
            std::vector<int64_t> rows;   // (row, first local entry, length) triples
            int64_t bad = -1;            // largest topological position of a failing node
        };
        std::vector<Local> loc((size_t)T);
        for (Local &L : loc) L.scratch = base32;
        for (int32_t lv = 0; lv < nh; ++lv) {
            const int64_t lo = lstart[lv], cnt = lstart[lv + 1] - lo;
            for_pieces(cnt, T, [&](int t, int64_t b0, int64_t b1) {
                Local &L = loc[(size_t)t];
                L.chain.clear();
                L.slot.clear();
                L.rows.clear();
                for (int64_t j = lo + b0; j < lo + b1; ++j) {
                    const int32_t x = by_level[(size_t)j];
                    L.touched.clear();
                    L.kids.assign(adj.begin() + ptr[x], adj.begin() + ptr[x + 1]);
                    std::sort(L.kids.begin(), L.kids.end(), [&](int32_t a, int32_t b) { return pos[a] < pos[b]; });
                    for (int32_t z : L.kids) {
                        const int32_t cz = H.chain_id[z];
                        if (L.scratch[cz] >= H.node_slot[z]) continue;
                        const int64_t rz = H.node_slot[z] - cz - 1;
                        const int64_t b = H.row_beg[rz], e = b + H.row_len[rz];
                        for (int64_t q = b; q < e; ++q) {
                            const int32_t c = H.ent_chain[q];
                            if (L.scratch[c] == base32[c]) L.touched.push_back(c);
                            L.scratch[c] = std::max(L.scratch[c], H.ent_slot[q]);
                        }
                    }
                    const int32_t cx = H.chain_id[x];
                    const int32_t sx = H.node_slot[x];
                    if (L.scratch[cx] != sx - 1) L.bad = std::max<int64_t>(L.bad, pos[x]);
                    if (L.scratch[cx] == base32[cx]) L.touched.push_back(cx);
                    L.scratch[cx] = sx;
                    std::sort(L.touched.begin(), L.touched.end());
                    L.rows.push_back(sx - cx - 1);
                    L.rows.push_back((int64_t)L.chain.size());
                    L.rows.push_back((int64_t)L.touched.size());
                    for (int32_t c : L.touched) {
                        L.chain.push_back(c);
                        L.slot.push_back(L.scratch[c]);
                        L.scratch[c] = base32[c];
                    }
                }
            });
            for (Local &L : loc) {   // append the level's rows in thread order
                const int64_t off = (int64_t)H.ent_chain.size();
                H.ent_chain.insert(H.ent_chain.end(), L.chain.begin(), L.chain.end());
                H.ent_slot.insert(H.ent_slot.end(), L.slot.begin(), L.slot.end());
                for (size_t q = 0; q < L.rows.size(); q += 3) {
                    H.row_beg[L.rows[q]] = off + L.rows[q + 1];
                    H.row_len[L.rows[q]] = (int32_t)L.rows[q + 2];
                }
                L.chain.clear();
                L.slot.clear();
                L.rows.clear();
            }
        }
        int64_t bad = -1;
        for (const Local &L : loc) bad = std::max(bad, L.bad);
        if (bad >= 0) {
            const int32_t x = H.topo[bad];
            return bad_chain(H.chain_id[x], x);
        }
        H.nnz = (int64_t)H.ent_chain.size();
    }

    // ---- 6. levels
    H.level.assign(n, 1);
    H.ulevel.assign(n, 0);
    for (int64_t i = n - 1; i >= 0; --i) {
        int32_t x = H.topo[i];
        int32_t h = 0;
        for (int64_t e = ptr[x]; e < ptr[x + 1]; ++e) h = std::max(h, H.level[adj[e]]);
        H.level[x] = h + 1;
    }
    // U levels: one more than the largest U level among the other chains' entries, which
    // all sit on lower heights; a sparse map's few, wide heights run on all host threads
    {
        auto ulevel_of = [&](int32_t x) {
            const int32_t cx = H.chain_id[x];
            int32_t u = 0;
            H.for_row(H.node_slot[x] - cx - 1, [&](int32_t c, int32_t slot) {
                if (c != cx) u = std::max(u, H.ulevel[H.slot_node[slot]] + 1);
            });
            H.ulevel[x] = u;
        };
        if (!H.sparse) {
            for (int64_t i = n - 1; i >= 0; --i) ulevel_of(H.topo[i]);
        } else {
            const int32_t nh = *std::max_element(H.level.begin(), H.level.end());
            std::vector<int64_t> lstart((size_t)nh + 2, 0);
            for (int64_t x = 0; x < n; ++x) lstart[H.level[x]]++;
            for (size_t l = 1; l < lstart.size(); ++l) lstart[l] += lstart[l - 1];
            std::vector<int32_t> by_level((size_t)n);
            std::vector<int64_t> fill(lstart);
            for (int64_t x = 0; x < n; ++x) by_level[(size_t)fill[H.level[x] - 1]++] = (int32_t)x;
            const int T = host_threads();
            for (int32_t lv = 0; lv < nh; ++lv)
                for_pieces(lstart[lv + 1] - lstart[lv], T, [&](int, int64_t b0, int64_t b1) {
                    for (int64_t j = lstart[lv] + b0; j < lstart[lv] + b1; ++j) ulevel_of(by_level[(size_t)j]);
                });
        }
    }
    H.nlevels = *std::max_element(H.level.begin(), H.level.end());
    H.nulevels = *std::max_element(H.ulevel.begin(), H.ulevel.end()) + 1;
    return MZ_OK;
}

}  // namespace mz
