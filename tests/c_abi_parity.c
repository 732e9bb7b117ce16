/* The C ABI used from plain C (no Python): an expanding two-field lattice in
 * FP64 stepped by libtl on the GPU and, from the same input, by the oracle's C
 * entry points (test infrastructure, oracle/tlo.c) on the CPU; fields, a and a'
 * must agree to 1e-12 relative (normwise for fields), the energies to 1e-12 of
 * K+G+V.  Also checks argument errors and tl_last_error.  Exit status 0 on
 * success; prints one line with the errors. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "tl.h"

/* the oracle's entry points, as oracle/tlo.c defines them */
typedef struct {
    int N, nf, expanding, pad_;
    double kIR, alpha, mu2, lambda, q, m2[3];
} tlo_params;
int tlo_run(const tlo_params *p, double *phi, double *pi, double *ab, double dt, int nsteps, int integrator);
void tlo_energies(const tlo_params *p, const double *phi, const double *pi, double a, double *out);

/* seeded input: splitmix64 -> uniform in [-1, 1) (no arithmetic of the method) */
static uint64_t rng_state = 0x5eed;
static double uniform_pm1(void)
{
    uint64_t z = (rng_state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

static int check(int rc, const char *what)
{
    if (rc != TL_OK) {
        fprintf(stderr, "%s failed: %d (%s)\n", what, rc, tl_last_error());
        exit(2);
    }
    return rc;
}

int main(void)
{
    const int N = 24, nf = 2, steps = 20;
    const double kIR = 0.5, dt = 0.005;
    const size_t n3 = (size_t)N * N * N;
    double *phi = malloc(nf * n3 * sizeof(double)), *pi = malloc(nf * n3 * sizeof(double));
    double *gphi = malloc(nf * n3 * sizeof(double)), *gpi = malloc(nf * n3 * sizeof(double));
    if (!phi || !pi || !gphi || !gpi) return 3;
    for (int f = 0; f < nf; ++f)
        for (size_t s = 0; s < n3; ++s) {
            phi[f * n3 + s] = (f == 0 ? 1.0 : 0.0) + 1e-3 * uniform_pm1();
            pi[f * n3 + s] = 1e-3 * uniform_pm1();
        }

    /* argument errors come back as codes with a message */
    tl_lattice *bad = NULL;
    if (tl_lattice_create(&bad, 7, kIR, nf, TL_F64, NULL, NULL) != TL_EINVAL || tl_last_error()[0] == '\0') {
        fprintf(stderr, "N = 7 was not refused with a message\n");
        return 4;
    }

    /* GPU */
    tl_lattice *L = NULL;
    const tl_expansion ex = {1, 1.0, 1.0, 1.0};
    const tl_potential pot = {1.0, 100.0, {0.0, 0.0, 0.0}};
    check(tl_lattice_create(&L, N, kIR, nf, TL_F64, &ex, NULL), "tl_lattice_create");
    check(tl_set_potential(L, &pot), "tl_set_potential");
    for (int f = 0; f < nf; ++f) {
        check(tl_set_state(L, f, 0, phi + f * n3, n3 * sizeof(double)), "tl_set_state phi");
        check(tl_set_state(L, f, 1, pi + f * n3, n3 * sizeof(double)), "tl_set_state pi");
    }
    check(tl_set_background(L, 1.0, 0.0, 1), "tl_set_background");
    check(tl_step(L, steps, dt, TL_YOSHIDA4), "tl_step");
    tl_energies_t E;
    check(tl_energies(L, &E), "tl_energies");
    for (int f = 0; f < nf; ++f) {
        check(tl_get_state(L, f, 0, gphi + f * n3, n3 * sizeof(double)), "tl_get_state phi");
        check(tl_get_state(L, f, 1, gpi + f * n3, n3 * sizeof(double)), "tl_get_state pi");
    }
    tl_lattice_destroy(L);

    /* oracle: b0 from the constraint of the same state, then the same steps */
    tlo_params p = {N, nf, 1, 0, kIR, 1.0, 1.0, 1.0, 100.0, {0.0, 0.0, 0.0}};
    double E0[7], Eo[7];
    tlo_energies(&p, phi, pi, 1.0, E0);
    double rho0 = 0.0;
    for (int i = 0; i < 2 * nf + 1; ++i) rho0 += E0[i];
    double ab[2] = {1.0, sqrt(rho0 / 3.0)};
    if (tlo_run(&p, phi, pi, ab, dt, steps, 2) != 0) return 5;
    tlo_energies(&p, phi, pi, ab[0], Eo);

    double dphi = 0, mphi = 0, dpi = 0, mpi = 0, rho = 0, dE = 0;
    for (size_t s = 0; s < nf * n3; ++s) {
        dphi = fmax(dphi, fabs(gphi[s] - phi[s]));
        mphi = fmax(mphi, fabs(phi[s]));
        dpi = fmax(dpi, fabs(gpi[s] - pi[s]));
        mpi = fmax(mpi, fabs(pi[s]));
    }
    const double gE[7] = {E.K[0], E.K[1], E.G[0], E.G[1], E.V, 0, 0};
    for (int i = 0; i < 2 * nf + 1; ++i) {
        rho += Eo[i];
        dE = fmax(dE, fabs(gE[i] - Eo[i]));
    }
    const double err_phi = dphi / mphi, err_pi = dpi / mpi, err_E = dE / rho;
    const double err_a = fabs(E.a - ab[0]) / ab[0], err_b = fabs(E.b - ab[1]) / fabs(ab[1]);
    printf("c-abi parity: phi %.3e pi %.3e energies %.3e a %.3e b %.3e (step %lld)\n", err_phi, err_pi, err_E, err_a,
           err_b, (long long)E.step);
    const int ok = err_phi < 1e-12 && err_pi < 1e-12 && err_E < 1e-12 && err_a < 1e-12 && err_b < 1e-12 &&
                   E.step == steps;
    free(phi);
    free(pi);
    free(gphi);
    free(gpi);
    return ok ? 0 : 1;
}
