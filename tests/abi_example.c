/* A plain C program on the library's C ABI (include/spkmc.h): create a
 * lattice with a hot start, run spkMC cycles (Sec. 3.1 steps 1-6 with the
 * rotating colours of Sec. 3.2 step 4a), read the observables and the final
 * spins, destroy the handle.
 *
 *   gcc -I include tests/abi_example.c -L paper_1005_4713_gb300 -lspkmc \
 *       -Wl,-rpath,paper_1005_4713_gb300 -o abi_example
 *   ./abi_example [L d J H T seed cycles]        (default 128 8 1 0 4.5115 2 800)
 *
 * It prints one line of key=value pairs (the clock as a C99 hex float, so
 * that a reader gets its exact bits) and exits 0, or prints the library's
 * message on stderr and exits 1. */
#include <stdio.h>
#include <stdlib.h>

#include "spkmc.h"

static int fail(const char *what, spkmc_t *h)
{
    fprintf(stderr, "%s: %s\n", what, spkmc_last_error());
    spkmc_destroy(h); /* NULL-safe */
    return 1;
}

int main(int argc, char **argv)
{
    int32_t L = 128, d = 8;
    double J = 1.0, H = 0.0, T = 4.5115;
    unsigned long long seed = 2;
    long long cycles = 800;
    if (argc == 8) {
        L = (int32_t)atoi(argv[1]);
        d = (int32_t)atoi(argv[2]);
        J = atof(argv[3]);
        H = atof(argv[4]);
        T = atof(argv[5]);
        seed = strtoull(argv[6], NULL, 10);
        cycles = atoll(argv[7]);
    } else if (argc != 1) {
        fprintf(stderr, "usage: %s [L d J H T seed cycles]\n", argv[0]);
        return 2;
    }

    spkmc_t *h = NULL;
    if (spkmc_create(L, d, J, H, T, (uint64_t)seed, &h) != SPKMC_OK) return fail("spkmc_create", h);
    if (spkmc_run_cycles(h, cycles) != SPKMC_OK) return fail("spkmc_run_cycles", h);
    spkmc_obs o;
    if (spkmc_observables(h, &o) != SPKMC_OK) return fail("spkmc_observables", h);

    /* the final spins, one int8 per site in x-fastest global order */
    const size_t n = (size_t)L * (size_t)L * (size_t)L;
    int8_t *s = (int8_t *)malloc(n);
    if (!s) {
        spkmc_destroy(h);
        return 1;
    }
    if (spkmc_get_spins(h, s, n) != SPKMC_OK) {
        free(s);
        return fail("spkmc_get_spins", h);
    }
    long long up = 0;
    for (size_t i = 0; i < n; ++i) up += s[i] > 0;
    free(s);

    printf("cycle=%lld M=%lld B=%lld n_flip=%lld n_null=%lld null_fx_lo=%llu null_fx_hi=%llu up=%lld clock=%a\n",
           (long long)o.cycle, (long long)o.M, (long long)o.B, (long long)o.n_flip, (long long)o.n_null,
           (unsigned long long)o.sum_null_rate_fx[0], (unsigned long long)o.sum_null_rate_fx[1], up, o.clock);
    spkmc_destroy(h);
    return 0;
}
