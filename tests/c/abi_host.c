/* A plain C caller of libafqmc.so: compiled with gcc against include/afqmc.h
 * only (no CUDA headers, no Python), it exercises the host-side parts of the
 * ABI that need no GPU: parameter checks, error messages and the twist
 * sequence.  Exit status 0 on success; the failing check is printed. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "afqmc.h"

static int fails = 0;
#define CHECK(c)                                                  \
    do {                                                          \
        if (!(c)) {                                               \
            fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); \
            ++fails;                                              \
        }                                                         \
    } while (0)

static afqmc_params base(void) {
    afqmc_params p;
    memset(&p, 0, sizeof p);
    p.L1 = 3; p.L2 = 3; p.t = 1.0; p.U = 3.73; p.beta = 3.0; p.dtau = 0.1;
    p.n_delay = 4; p.n_stab = 10; p.seed = 1;
    return p;
}

int main(void) {
    /* the Halton (2,3) points 1..6 */
    const double want[12] = {1.0 / 2, 1.0 / 3, 1.0 / 4, 2.0 / 3, 3.0 / 4, 1.0 / 9,
                             1.0 / 8, 4.0 / 9, 5.0 / 8, 7.0 / 9, 3.0 / 8, 2.0 / 9};
    double th[12];
    CHECK(afqmc_quasirandom_twists(6, 1, th) == AFQMC_OK);
    for (int i = 0; i < 12; ++i) CHECK(th[i] == want[i]);
    CHECK(afqmc_quasirandom_twists(-1, 1, th) == AFQMC_E_INVALID);
    CHECK(afqmc_quasirandom_twists(3, 1, NULL) == AFQMC_E_INVALID);
    CHECK(strstr(afqmc_last_error(NULL), "quasirandom") != NULL);
    CHECK(afqmc_quasirandom_twists(0, 0, NULL) == AFQMC_OK);

    /* parameters are checked before any device work */
    afqmc_handle* h = (afqmc_handle*)0x1;
    afqmc_params p = base();
    p.hs_channel = 2;
    CHECK(afqmc_create(&p, NULL, &h) == AFQMC_E_INVALID);
    CHECK(h == NULL);
    CHECK(strstr(afqmc_last_error(NULL), "hs_channel") != NULL);
    p = base();
    p.n_stab = 7;                       /* M = 30 is not a multiple of 7 */
    CHECK(afqmc_create(&p, NULL, &h) == AFQMC_E_INVALID);
    CHECK(strstr(afqmc_last_error(NULL), "n_stab") != NULL);
    p = base();
    p.theta1 = 1.0;
    CHECK(afqmc_create(&p, NULL, &h) == AFQMC_E_INVALID);
    CHECK(afqmc_create(NULL, NULL, &h) == AFQMC_E_INVALID);
    CHECK(afqmc_destroy(NULL) == AFQMC_OK);
    CHECK(afqmc_dims(NULL, NULL, NULL, NULL) == AFQMC_E_INVALID);

    if (fails) return 1;
    printf("c abi ok\n");
    return 0;
}
