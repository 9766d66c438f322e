/* The C ABI used from C (no GPU needed): status strings, solver defaults and
 * the host-only partition of the two-triangle mesh of Fig. 1.  Prints
 * "ok" and exits 0 when every check holds. */
#include <stdio.h>
#include <stdlib.h>

#include "ebe.h"

#define CHECK(c)                                              \
    do {                                                      \
        if (!(c)) {                                           \
            fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); \
            return 1;                                         \
        }                                                     \
    } while (0)

int main(void) {
    CHECK(ebe_status_string(EBE_OK) != NULL);

    ebe_solve_opts o;
    ebe_solve_opts_default(&o);
    CHECK(o.rtol == 1e-8 && o.precision == EBE_PREC_FP64 && o.chunk == 32);

    /* nodes 0=(0,0), 1=(1,0), 2=(0,1), 3=(1,1); triangles (0,1,3), (0,3,2) */
    const double coords[8] = {0, 0, 1, 0, 0, 1, 1, 1};
    const int32_t elems[6] = {0, 1, 3, 0, 3, 2};
    ebe_mesh m = {2, 3, 4, 2, coords, elems};
    ebe_partition_sizes sz;
    CHECK(ebe_partition_export(&m, &sz, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL) == EBE_OK);
    CHECK(sz.n_patches == 1 && sz.n_shared == 0 && sz.n_halo == 0 && sz.patch_elems == 1024);

    int32_t* slot_elem = malloc(sizeof(int32_t) * (size_t)sz.n_slots);
    uint16_t* lconn = malloc(sizeof(uint16_t) * 3 * (size_t)sz.n_slots);
    int32_t* meta = malloc(sizeof(int32_t) * 8 * (size_t)sz.n_patches);
    int32_t* pnode = malloc(sizeof(int32_t) * (size_t)sz.n_pnode);
    int32_t* col_ptr = malloc(sizeof(int32_t) * (size_t)sz.n_colptr);
    CHECK(slot_elem && lconn && meta && pnode && col_ptr);
    CHECK(ebe_partition_export(&m, &sz, slot_elem, lconn, meta, pnode, col_ptr, NULL, NULL, NULL) == EBE_OK);
    /* one patch: both elements, all 4 nodes owned; the two triangles share
     * nodes 0 and 3, so they fall into two colour classes */
    CHECK(meta[1] == 4 && meta[2] == 4 && meta[4] == 2 && meta[6] == 2);
    CHECK((slot_elem[0] == 0 && slot_elem[1] == 1) || (slot_elem[0] == 1 && slot_elem[1] == 0));
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < 3; ++i) CHECK(pnode[lconn[i * sz.n_slots + s]] == elems[slot_elem[s] * 3 + i]);

    /* a node id outside [0, n_n) is rejected before any device work */
    const int32_t bad[3] = {0, 1, 7};
    ebe_mesh mb = {2, 3, 4, 1, coords, bad};
    CHECK(ebe_partition_export(&mb, &sz, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL) == EBE_INDEX_RANGE);
    CHECK(ebe_last_error(NULL) != NULL);

    free(slot_elem); free(lconn); free(meta); free(pnode); free(col_ptr);
    printf("ok\n");
    return 0;
}
