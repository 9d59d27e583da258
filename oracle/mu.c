/*
 * Oracle helper: the Moebius function of a finite poset by its defining
 * recursion (Thm. 1 of arxiv 2211.13706, Sec. 2.2):
 *
 *     mu(y, y) = 1,
 *     mu(y, x) = - sum_{y <= z < x} mu(y, z)      for y != x,
 *     mu(y, x) = 0                                when y is not below x.
 *
 * TEST INFRASTRUCTURE ONLY. This file belongs to the CPU oracle: only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it. The GPU library never links or calls it, and it shares no code with it.
 *
 * Inputs
 *   n      number of elements
 *   Z      n*n bytes, Z[x*n + y] = 1 iff y <= x (the zeta matrix of Cor. 1,
 *          i.e. the reflexive transitive closure)
 *   order  a topological order, order[0] a largest element (x comes after
 *          every element above it), so walking it backwards visits every
 *          z < x before x
 * Output
 *   mu     n*n int64, mu[y*n + x] = mu(y, x)
 * Returns 0, or -1 if some partial sum overflows int64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int orc_mobius_function(int64_t n, const uint8_t *Z, const int64_t *order, int64_t *mu)
{
    int64_t *up = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!up) return -2;
    memset(mu, 0, sizeof(int64_t) * (size_t)n * (size_t)n);
    for (int64_t y = 0; y < n; ++y) {
        int64_t *row = mu + y * n;
        /* the up-set of y in bottom-up order: y first, every z < x before x */
        int64_t cnt = 0;
        for (int64_t t = n - 1; t >= 0; --t) {
            int64_t x = order[t];
            if (Z[x * n + y]) up[cnt++] = x;
        }
        for (int64_t a = 0; a < cnt; ++a) {
            int64_t x = up[a];
            if (x == y) { row[x] = 1; continue; }
            int64_t s = 0;
            /* z ranges over y <= z < x: z in the up-set of y, below x, not x */
            for (int64_t b = 0; b < a; ++b) {
                int64_t z = up[b];
                if (Z[x * n + z]) {
                    if (__builtin_add_overflow(s, row[z], &s)) { free(up); return -1; }
                }
            }
            if (s == INT64_MIN) { free(up); return -1; }
            row[x] = -s;
        }
    }
    free(up);
    return 0;
}
