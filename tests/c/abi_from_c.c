/* A plain C99 caller of the library: the header must compile as C (no C++ types or default
 * arguments), and the host-only entry points must link and answer without a GPU.  Prints
 * "ok" and exits 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "fc.h"

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
    if (bad) {
        printf("failed checks: %d\n", bad);
        return 1;
    }
    printf("ok\n");
    return 0;
}
