/* A plain C99 caller of the library: the header must compile as C (no C++ types or default
 * arguments), and the host-only entry points must link and answer without a GPU.  Prints
 * "ok" and exits 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "fc.h"

/* a separable cost with its minimum at gemm_cover 2, workers 24, order 1 */
static double cost(const fc_schedule* s, void* ctx) {
    int* calls = (int*)ctx;
    ++*calls;
    return 1.0 + (s->gemm_cover != 2) + (s->workers != 24) + (s->order != 1);
}

int main(void) {
    fc_handle h = NULL;
    int bad = 0;
    /* argument checks run before any CUDA call: d = 4, alpha = 1.5, n = 0 */
    if (fc_setup(63, 4, 0.5, 1.0, 1e-2, 1e-8, NULL, &h) != FC_EINVAL) bad |= 1;
    if (fc_setup(63, 2, 1.5, 1.0, 1e-2, 1e-8, NULL, &h) != FC_EINVAL) bad |= 2;
    if (fc_setup(0, 2, 0.5, 1.0, 1e-2, 1e-8, NULL, &h) != FC_EINVAL) bad |= 4;
    if (h != NULL) bad |= 8;
    if (strcmp(fc_strerror(FC_ERANK), "rank capacity exceeded") != 0) bad |= 16;
    if (strcmp(fc_strerror(12345), "unknown error") != 0) bad |= 32;
    if (fc_solve_batched(-1, NULL, NULL, NULL, NULL, NULL, NULL) != FC_EINVAL) bad |= 64;
    /* the schedule and its autotuner are host code */
    {
        fc_schedule s0, s1, best;
        int calls = 0, evals = 0;
        double c = 0.0;
        if (fc_get_schedule(&s0) != FC_OK || s0.workers != 16 || s0.tc_min_log2 != 22) bad |= 128;
        s1 = s0;
        s1.workers = 0;
        if (fc_set_schedule(&s1) != FC_EINVAL) bad |= 256;
        if (fc_autotune(NULL, 2, 0.0, cost, &calls, &best, &c, &evals) != FC_OK) bad |= 512;
        if (best.gemm_cover != 2 || best.workers != 24 || best.order != 1 || c != 1.0 ||
            evals != calls)
            bad |= 1024;
        if (fc_get_schedule(&s1) != FC_OK || memcmp(&s0, &s1, sizeof s0) != 0) bad |= 2048;
    }
    if (bad) {
        printf("failed checks: %d\n", bad);
        return 1;
    }
    printf("ok\n");
    return 0;
}
