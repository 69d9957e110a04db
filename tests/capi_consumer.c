/* A plain C99 consumer of the C-ABI: includes include/trids.h, links libtrids.so and
 * calls the entry points that need no GPU (argument checks fail before any CUDA call).
 * Built and run by tests/test_capi_c_consumer.py. */
#include <stdio.h>
#include <string.h>

#include "trids.h"

int main(void) {
    int bad = 0;
    if (trids_version() <= 0) { printf("version %d\n", trids_version()); bad = 1; }
    trids_pocket* pk = NULL;
    const float c[3] = {0.f, 0.f, 0.f}, s[3] = {22.5f, 22.5f, 22.5f};
    int rc = trids_make_pocket(NULL, NULL, 10, c, s, 0.f, NULL, &pk);
    if (rc != TRIDS_EINVAL || pk != NULL) { printf("make_pocket rc %d\n", rc); bad = 1; }
    if (strlen(trids_last_error()) == 0) { printf("empty error message\n"); bad = 1; }
    trids_batch* b = NULL;
    rc = trids_pack_ligands(NULL, 1, NULL, NULL, NULL, NULL, NULL, NULL, &b);
    if (rc != TRIDS_EINVAL || b != NULL) { printf("pack_ligands rc %d\n", rc); bad = 1; }
    rc = trids_topk(NULL, 1, NULL, NULL, 1, 1.f, NULL, NULL, NULL);
    if (rc != TRIDS_EINVAL) { printf("topk rc %d\n", rc); bad = 1; }
    rc = trids_screen_energy(NULL, NULL, 1, 1, NULL, NULL, NULL, NULL);
    if (rc != TRIDS_EINVAL) { printf("screen_energy rc %d\n", rc); bad = 1; }
    printf(bad ? "FAIL\n" : "OK %d\n", trids_version());
    return bad;
}
