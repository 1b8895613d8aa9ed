/* A plain C client of libkpp: includes only include/kpp.h, links the shared library, and calls the
 * entry points that need no GPU.  It shows that the boundary is a C ABI usable without Python:
 * partition handles, parameter defaults, status strings, the last-error message and the memo block
 * sequence.  Prints one "key value" line per check; the test that builds it compares them. */
#include <stdio.h>
#include <string.h>

#include "kpp.h"

int main(void) {
    kpp_partition_t P = NULL;
    kpp_status rc = kpp_partition(103, 10, &P);
    printf("partition_rc %d\n", (int)rc);
    printf("partition_blocks %lld\n", (long long)kpp_partition_blocks(P));
    kpp_partition_destroy(P);

    rc = kpp_partition(0, 10, &P);
    printf("bad_partition_rc %d\n", (int)rc);
    printf("last_error_mentions_call %d\n", strstr(kpp_last_error(), "kpp_partition") != NULL);

    kpp_params p = kpp_params_default();
    printf("default_tol %.1e\n", p.tol);
    printf("default_max_outer %d\n", p.max_outer);
    printf("status_string %s\n", kpp_status_string(KPP_ERR_NOT_SPD));

    int64_t blocks[64], subsets[64 * 16], nb = 0; /* subsets_cap x s entries */
    rc = kpp_memo_sequence(11, 0, 1, 256, 256, 16, 0, 64, 0, blocks, subsets, 64, &nb);
    printf("memo_rc %d\n", (int)rc);
    printf("memo_first_block %lld\n", (long long)blocks[0]);
    printf("memo_blocks %lld\n", (long long)nb);
    return 0;
}
