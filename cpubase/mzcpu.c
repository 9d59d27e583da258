/*
 * The paper's fast transforms on the CPU, a timing baseline for the GPU path
 * (arxiv 2211.13706, Sec. 3; Alg. 3 for zeta, Alg. 4 for Moebius in the antichain
 * order of Alg. 5 / Alg. 6). OpenMP threads when compiled with -fopenmp.
 *
 * Layout (the library's slot layout): chain c owns slots [base_c, base_c + len_c];
 * slot base_c stands for "no element" and holds 0; the element at chain position p
 * (0 = bottom) sits at slot base_c + 1 + p.
 *   node_slot[n]     slot of each node
 *   slot_node[S]     node of each slot, -1 at the zero slots (S = n + k)
 *   chain_base[k+1]  first slot (the zero slot) of each chain, chain_base[k] = S
 *   N[n * k]         N[x * k + c] = slot of niv_c(x), or base_c when there is none
 *   chain_of[n]      chain of each node
 *   lvl_ptr[L + 1], lvl_nodes[n]   antichain levels from the bottom (heights)
 *
 * zeta (Alg. 3): P = per-chain prefix sums of f (Eq. zeta_cache), then
 *   g(x) = sum_c P[N(x, c)] (Eq. zeta-fast).
 * Moebius (Alg. 4 in the order of Alg. 5): level by level from the bottom, all x of
 *   a level in parallel: f(x) = g(x) - P[slot(x) - 1] - sum_{c != chain(x)} P[N(x, c)],
 *   then P[slot(x)] = P[slot(x) - 1] + f(x). A level is an antichain, and every slot
 *   x reads belongs to a lower level.
 * mzcpu_mobius_u_* runs Alg. 4's two loops instead, the first in the order of the levels
 * of U's dependency graph (the library's default schedule, with barriers between levels).
 * The int64 variant computes modulo 2^64 (unsigned arithmetic on the same bits).
 */
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int mzcpu_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void mzcpu_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

#define MZCPU_DEFINE(T, SUF)                                                                            \
    void mzcpu_zeta_##SUF(int64_t n, int32_t k, const int64_t *chain_base, const int32_t *slot_node,     \
                          const int32_t *N, const T *f, T *g, T *P) {                                   \
        int64_t x;                                                                                      \
        int32_t c;                                                                                      \
        /* one task per chain: its zero slot, then the running sum over its slots */                   \
        _Pragma("omp parallel for schedule(dynamic, 1)") for (c = 0; c < k; ++c) {                     \
            T run = 0;                                                                                  \
            P[chain_base[c]] = 0;                                                                       \
            for (int64_t q = chain_base[c] + 1; q < chain_base[c + 1]; ++q) {                           \
                run += f[slot_node[q]];                                                                 \
                P[q] = run;                                                                             \
            }                                                                                           \
        }                                                                                               \
        _Pragma("omp parallel for schedule(static)") for (x = 0; x < n; ++x) {                          \
            const int32_t *row = N + x * (int64_t)k;                                                    \
            T acc = 0;                                                                                  \
            for (int32_t j = 0; j < k; ++j) acc += P[row[j]];                                           \
            g[x] = acc;                                                                                 \
        }                                                                                               \
    }                                                                                                   \
                                                                                                        \
    void mzcpu_mobius_##SUF(int64_t S, int32_t k, const int32_t *node_slot, const int32_t *chain_of,    \
                            const int32_t *N, const int64_t *lvl_ptr, int32_t nlevels,                  \
                            const int32_t *lvl_nodes, const T *g, T *f, T *P) {                         \
        int64_t s;                                                                                      \
        _Pragma("omp parallel for schedule(static)") for (s = 0; s < S; ++s) P[s] = 0;                 \
        _Pragma("omp parallel") for (int32_t l = 0; l < nlevels; ++l) {                                \
            int64_t i;                                                                                  \
            /* the implicit barrier at the end of each level is Alg. 5's */                            \
            _Pragma("omp for schedule(static)") for (i = lvl_ptr[l]; i < lvl_ptr[l + 1]; ++i) {         \
                const int32_t x = lvl_nodes[i];                                                         \
                const int32_t sx = node_slot[x], cx = chain_of[x];                                      \
                const int32_t *row = N + (int64_t)x * k;                                                \
                const T below = P[sx - 1];                                                              \
                T acc = g[x] - below;                                                                   \
                for (int32_t j = 0; j < k; ++j)                                                         \
                    if (j != cx) acc -= P[row[j]];                                                      \
                f[x] = acc;                                                                             \
                P[sx] = below + acc;                                                                    \
            }                                                                                           \
        }                                                                                               \
    }

/* Moebius in the order of U's own dependency levels (fewer levels than antichains):
 * level by level, y'(x) = g(x) - sum_{c != chain(x)} P[N(x, c)] into P[slot(x)] (the
 * first loop of Alg. 4), then f(x) = P[slot(x)] - P[slot(x) - 1] for all x (V^-1). */
#define MZCPU_DEFINE_U(T, SUF)                                                                          \
    void mzcpu_mobius_u_##SUF(int64_t n, int64_t S, int32_t k, const int32_t *node_slot,               \
                              const int32_t *chain_of, const int32_t *N, const int64_t *lvl_ptr,        \
                              int32_t nlevels, const int32_t *lvl_nodes, const T *g, T *f, T *P) {      \
        int64_t s, x;                                                                                   \
        _Pragma("omp parallel for schedule(static)") for (s = 0; s < S; ++s) P[s] = 0;                 \
        _Pragma("omp parallel") for (int32_t l = 0; l < nlevels; ++l) {                                \
            int64_t i;                                                                                  \
            _Pragma("omp for schedule(static)") for (i = lvl_ptr[l]; i < lvl_ptr[l + 1]; ++i) {         \
                const int32_t y = lvl_nodes[i];                                                         \
                const int32_t cy = chain_of[y];                                                         \
                const int32_t *row = N + (int64_t)y * k;                                                \
                T acc = g[y];                                                                           \
                for (int32_t j = 0; j < k; ++j)                                                         \
                    if (j != cy) acc -= P[row[j]];                                                      \
                P[node_slot[y]] = acc;                                                                  \
            }                                                                                           \
        }                                                                                               \
        _Pragma("omp parallel for schedule(static)") for (x = 0; x < n; ++x)                           \
            f[x] = P[node_slot[x]] - P[node_slot[x] - 1];                                               \
    }

MZCPU_DEFINE(double, f64)
MZCPU_DEFINE(uint64_t, i64)
MZCPU_DEFINE_U(double, f64)
MZCPU_DEFINE_U(uint64_t, i64)
