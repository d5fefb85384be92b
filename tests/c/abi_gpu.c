/* A plain C caller of the GPU path of libafqmc.so: compiled with gcc against
 * include/afqmc.h only, it creates a chain (L = 3, beta t = 3, dtau = 0.1,
 * U/t = 3.73, n_d = 4, recomputation every 10 slices, seed 2024), runs two
 * sweeps, reads back the field, G at slice 0 and the observables of that G, and
 * writes them to the file named by argv[1]:
 *
 *   int32 N, int32 M, uint64 proposed, uint64 accepted,
 *   int8 field[M*N] (slice-major), double G[N*N] (row-major),
 *   double obs[10] (energy, double_occ, ekin, density, m2, S_af, S_af_dk,
 *                   R_m2, Czz_half, chi_e)
 *
 * so that a test can hold them to the oracle.  Error paths that need no
 * device fault are checked on the way.  Exit status 0 on success. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "afqmc.h"

static int fails = 0;
#define CHECK(c)                                                           \
    do {                                                                   \
        if (!(c)) {                                                        \
            fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); \
            ++fails;                                                       \
        }                                                                  \
    } while (0)

int main(int argc, char** argv) {
    if (argc != 2) {
        fprintf(stderr, "usage: %s OUTFILE\n", argv[0]);
        return 2;
    }
    afqmc_params p;
    memset(&p, 0, sizeof p);
    p.L1 = 3; p.L2 = 3; p.t = 1.0; p.U = 3.73; p.beta = 3.0; p.dtau = 0.1;
    p.n_delay = 4; p.n_stab = 10; p.seed = 2024;

    afqmc_handle* h = NULL;
    afqmc_status st = afqmc_create(&p, NULL, &h);
    if (st != AFQMC_OK) {
        fprintf(stderr, "afqmc_create: %d %s\n", (int)st, afqmc_last_error(NULL));
        return 1;
    }
    int32_t N = 0, M = 0, Nc = 0;
    CHECK(afqmc_dims(h, &N, &M, &Nc) == AFQMC_OK);
    CHECK(N == 18 && M == 30 && Nc == 9);

    afqmc_sweep_stats s;
    memset(&s, 0, sizeof s);
    CHECK(afqmc_sweep(h, 2, &s) == AFQMC_OK);
    CHECK(s.proposed == (uint64_t)2 * 2 * N * M);
    CHECK(s.accepted > 0 && s.accepted < s.proposed);
    CHECK(s.launches > 0);

    int8_t* field = (int8_t*)malloc((size_t)M * N);
    double* G = (double*)malloc(sizeof(double) * N * N);
    double* Czz = (double*)malloc(sizeof(double) * Nc);
    CHECK(afqmc_get_field(h, field) == AFQMC_OK);
    for (int i = 0; i < M * N; ++i) CHECK(field[i] == 1 || field[i] == -1);
    CHECK(afqmc_get_G(h, 0, G) == AFQMC_OK);
    afqmc_obs o;
    CHECK(afqmc_measure(h, &o, Czz, NULL) == AFQMC_OK);
    CHECK(o.n_samples == 1);

    /* rejected arguments leave the handle usable */
    CHECK(afqmc_get_G(h, M + 1, G + 0) == AFQMC_E_INVALID);
    CHECK(strstr(afqmc_last_error(h), "slice") != NULL);
    double r[3];
    CHECK(afqmc_det_ratio(h, 1, N, r) == AFQMC_E_INVALID);
    CHECK(afqmc_det_ratio(h, 1, 0, r) == AFQMC_OK);
    CHECK(r[0] > 0.0 && r[2] == 0.0);

    FILE* f = fopen(argv[1], "wb");
    if (!f) {
        fprintf(stderr, "cannot open %s\n", argv[1]);
        return 1;
    }
    const double obs[10] = {o.energy, o.double_occ, o.ekin, o.density, o.m2,
                            o.S_af, o.S_af_dk, o.R_m2, o.Czz_half, o.chi_e};
    fwrite(&N, sizeof N, 1, f);
    fwrite(&M, sizeof M, 1, f);
    fwrite(&s.proposed, sizeof s.proposed, 1, f);
    fwrite(&s.accepted, sizeof s.accepted, 1, f);
    fwrite(field, 1, (size_t)M * N, f);
    fwrite(G, sizeof(double), (size_t)N * N, f);
    fwrite(obs, sizeof(double), 10, f);
    fclose(f);

    CHECK(afqmc_destroy(h) == AFQMC_OK);
    free(field);
    free(G);
    free(Czz);
    if (fails) return 1;
    printf("c gpu abi ok\n");
    return 0;
}
