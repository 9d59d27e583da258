/* A C99 program against include/mz.h and libmz.so, without a GPU: a host-only plan of the
 * paper's 12-element example (Sec. 2), its exports, a plan file written and read back, and
 * the documented errors. Prints "c abi ok" and exits 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "mz.h"

#define CHECK(cond)                                                        \
    do {                                                                   \
        if (!(cond)) {                                                     \
            fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
            return 1;                                                      \
        }                                                                  \
    } while (0)

int main(int argc, char **argv) {
    const char *path = argc > 1 ? argv[1] : "c_abi_example.mzplan";
    /* edges u -> v mean v <= u: the Hasse diagram of the example */
    const int32_t src[17] = {0, 0, 0, 1, 1, 2, 2, 3, 3, 4, 5, 5, 6, 7, 8, 9, 9};
    const int32_t dst[17] = {2, 3, 5, 3, 4, 6, 7, 6, 8, 9, 7, 8, 9, 10, 11, 10, 11};
    mz_build_opts opts;
    memset(&opts, 0, sizeof(opts));
    opts.host_only = 1;
    opts.build_transpose = 1;
    mz_plan *plan = NULL;
    CHECK(mz_build(12, 17, src, dst, NULL, &opts, &plan) == MZ_OK && plan != NULL);

    mz_plan_info_t info;
    CHECK(mz_plan_info(plan, &info) == MZ_OK);
    CHECK(info.n == 12 && info.k == 4 && info.has_transpose == 1 && info.components == 1);
    CHECK(info.levels == 5);            /* the example's longest chain has 5 elements */

    int32_t cid[12], pos[12], topo[12], niv[12 * 4];
    CHECK(mz_plan_export(plan, MZ_EXPORT_CHAIN_ID, 0, cid, sizeof(cid)) == MZ_OK);
    CHECK(mz_plan_export(plan, MZ_EXPORT_CHAIN_POS, 0, pos, sizeof(pos)) == MZ_OK);
    CHECK(mz_plan_export(plan, MZ_EXPORT_TOPO, 0, topo, sizeof(topo)) == MZ_OK);
    CHECK(mz_plan_export(plan, MZ_EXPORT_NIV, 0, niv, sizeof(niv)) == MZ_OK);
    for (int x = 0; x < 12; ++x) {
        CHECK(cid[x] >= 0 && cid[x] < 4);
        CHECK(niv[x * 4 + cid[x]] == x);   /* niv on its own chain is the element itself */
    }
    CHECK(mz_plan_export(plan, MZ_EXPORT_NIV, 0, niv, 8) == MZ_ERR_INVALID_ARG);   /* buffer too small */

    /* a plan file, read back host-only: the same exports */
    CHECK(mz_plan_save(plan, path) == MZ_OK);
    mz_plan *back = NULL;
    CHECK(mz_plan_load(path, &opts, &back) == MZ_OK && back != NULL);
    int32_t cid2[12], niv2[12 * 4];
    CHECK(mz_plan_export(back, MZ_EXPORT_CHAIN_ID, 0, cid2, sizeof(cid2)) == MZ_OK);
    CHECK(mz_plan_export(back, MZ_EXPORT_NIV, 1, niv2, sizeof(niv2)) == MZ_OK);   /* the dual's map */
    CHECK(memcmp(cid, cid2, sizeof(cid)) == 0);
    mz_destroy(back);

    /* errors: a cycle, an id out of range, a missing file; *out stays NULL */
    const int32_t csrc[3] = {0, 1, 2}, cdst[3] = {1, 2, 0};
    mz_plan *bad = (mz_plan *)&opts;
    CHECK(mz_build(3, 3, csrc, cdst, NULL, &opts, &bad) == MZ_ERR_CYCLE && bad == NULL);
    const int32_t osrc[1] = {0}, odst[1] = {7};
    CHECK(mz_build(3, 1, osrc, odst, NULL, &opts, &bad) == MZ_ERR_INVALID_ARG && bad == NULL);
    CHECK(mz_plan_load("/nonexistent/plan.mzplan", &opts, &bad) == MZ_ERR_INVALID_ARG && bad == NULL);
    CHECK(strcmp(mz_status_string(MZ_ERR_CYCLE), "MZ_ERR_CYCLE") == 0);
    CHECK(strlen(mz_last_error()) > 0);

    mz_destroy(plan);
    printf("c abi ok\n");
    return 0;
}
