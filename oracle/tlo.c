/*
 * Oracle for the scalar-field lattice stepper: a plain, slow, double-precision
 * CPU implementation written straight from the equations.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path (the
 * CUDA library) shares no code, header, table or helper with it.
 *
 * What it computes (program variables, tildes dropped):
 *   - lattice: N^3 sites, periodic, x fastest, dx = 2*pi/(kIR*N);
 *     7-point Laplacian  Lap phi = sum_i (phi(x+i) + phi(x-i) - 2 phi(x))/dx^2
 *     (the paper's LatLapl / "7-point stencil", Sec. 2 and Sec. 4).
 *   - potential  V = sum_f m_f^2 phi_f^2/2 + lambda phi_0^4/4
 *                    + (q/2) phi_0^2 sum_{f>=1} phi_f^2.
 *     With one field, m = 0: the phi^4 benchmark of Sec. 4; the kick there,
 *     pi+ = pi + dt (Lap phi - m^2 phi - lambda phi^3), is this model with
 *     a == 1 and the quartic written as lambda phi^4/4.
 *   - field equations with the alpha time variable, pi = a^(3-alpha) phi':
 *         phi' = a^(alpha-3) pi,
 *         pi'  = F(phi, a) = a^(1+alpha) Lap phi - a^(3+alpha) dV/dphi.
 *   - volume averages  K_f = a^-6 <pi_f^2>/2,
 *                      G_f = a^-2 <sum_i (phi(x+i)-phi(x))^2/dx^2>/2,
 *                      V   = <V(phi)>.
 *   - scale factor (Friedmann, mu2 = (fstar/m_p)^2):
 *         a'' = F_b = a^(2 alpha+1) (mu2/3) [(alpha-2) K + alpha G + (alpha+1) V],
 *         Hubble constraint (a'/a)^2 = a^(2 alpha) mu2 (K+G+V)/3.
 *   The paper prints only the static phi^4 kick/drift (Sec. 4); everything
 *   about expansion is the standard scalar field in an FLRW background,
 *   written in the alpha-time program variables the paper's CosmoLattice
 *   lineage uses.  These readings are listed with the design notes.
 *
 * Integrators (each is the literal operator sequence, no fusion):
 *   - velocity Verlet substep of size s (palindrome):
 *       b += s/2 F_b(E(phi,pi,a));  pi += s/2 F(phi,a);
 *       a_old = a; a += s b;  phi += s ((a_old+a)/2)^(alpha-3) pi;
 *       pi += s/2 F(phi,a);  b += s/2 F_b(E(phi,pi,a)).
 *   - leapfrog: the kick-then-drift of Sec. 4 with pi at half steps, started
 *     by a half kick; the momentum reported at integer time n is
 *     (pi_{n-1/2} + pi_{n+1/2})/2.
 *   - 4th-order Yoshida: VV(w1 h) VV(w0 h) VV(w1 h),
 *       w1 = 1/(2 - 2^(1/3)),  w0 = -2^(1/3)/(2 - 2^(1/3)).
 *   In a static background (expanding == 0) a == 1, b == 0 and the b-kicks
 *   and a-drift are skipped.
 *
 * Random numbers: Philox-2x64 with 10 rounds (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11), the generator the
 * paper names for its Gaussian random fields (Sec. 2).  Pinned to the
 * published known-answer vectors of Philox-2x64-10 (the Random123
 * distribution's kat_vectors rows), to the round structure by exact
 * inversion, and statistically.
 *
 * Compiled with -O2 -ffp-contract=off so every product and sum is rounded as
 * written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TLO_MAX_FIELDS 3

typedef struct {
    int N;          /* sites per side */
    int nf;         /* number of fields, 1..3 */
    int expanding;  /* 0: static background a == 1 */
    int pad_;
    double kIR;     /* infrared momentum, L = 2 pi / kIR */
    double alpha;   /* time variable d eta = a^-alpha dt */
    double mu2;     /* (fstar/m_p)^2 */
    double lambda;  /* quartic self-coupling of field 0 */
    double q;       /* field-0 / field-f coupling */
    double m2[TLO_MAX_FIELDS];
} tlo_params;

enum { TLO_LEAPFROG = 0, TLO_VERLET = 1, TLO_YOSHIDA4 = 2 };

static double tlo_dx(const tlo_params *p) { return 2.0 * M_PI / (p->kIR * (double)p->N); }

static size_t site(int N, int x, int y, int z)
{
    x = (x % N + N) % N;
    y = (y % N + N) % N;
    z = (z % N + N) % N;
    return ((size_t)z * (size_t)N + (size_t)y) * (size_t)N + (size_t)x;
}

/* dV/dphi_f at one site, given the values of all fields there. */
static double dV(const tlo_params *p, int f, const double *v)
{
    if (f == 0) {
        double others = 0.0;
        for (int g = 1; g < p->nf; ++g) others += v[g] * v[g];
        return p->m2[0] * v[0] + p->lambda * v[0] * v[0] * v[0] + p->q * v[0] * others;
    }
    return p->m2[f] * v[f] + p->q * v[0] * v[0] * v[f];
}

/* V at one site. */
static double Vsite(const tlo_params *p, const double *v)
{
    double s = 0.0;
    for (int f = 0; f < p->nf; ++f) s += 0.5 * p->m2[f] * v[f] * v[f];
    s += 0.25 * p->lambda * v[0] * v[0] * v[0] * v[0];
    double others = 0.0;
    for (int g = 1; g < p->nf; ++g) others += v[g] * v[g];
    s += 0.5 * p->q * v[0] * v[0] * others;
    return s;
}

/* F_f(x) = a^(1+alpha) Lap phi_f - a^(3+alpha) dV/dphi_f, all fields. */
void tlo_force(const tlo_params *p, const double *phi, double a, double *F)
{
    const int N = p->N, nf = p->nf;
    const size_t n3 = (size_t)N * N * N;
    const double dx = tlo_dx(p);
    const double inv_dx2 = 1.0 / (dx * dx);
    const double wl = p->expanding ? pow(a, 1.0 + p->alpha) : 1.0;
    const double wv = p->expanding ? pow(a, 3.0 + p->alpha) : 1.0;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < N; ++z)
        for (int y = 0; y < N; ++y)
            for (int x = 0; x < N; ++x) {
                size_t s = site(N, x, y, z);
                double v[TLO_MAX_FIELDS];
                for (int f = 0; f < nf; ++f) v[f] = phi[(size_t)f * n3 + s];
                for (int f = 0; f < nf; ++f) {
                    const double *ph = phi + (size_t)f * n3;
                    double lap = (ph[site(N, x + 1, y, z)] + ph[site(N, x - 1, y, z)] - 2.0 * ph[s])
                               + (ph[site(N, x, y + 1, z)] + ph[site(N, x, y - 1, z)] - 2.0 * ph[s])
                               + (ph[site(N, x, y, z + 1)] + ph[site(N, x, y, z - 1)] - 2.0 * ph[s]);
                    lap *= inv_dx2;
                    F[(size_t)f * n3 + s] = wl * lap - wv * dV(p, f, v);
                }
            }
}

/* Volume averages: out[f] = K_f, out[nf+f] = G_f, out[2 nf] = V.
 * Each z-plane is summed in order into its own slot, then the planes are
 * summed in order, so the result does not depend on the thread count. */
void tlo_energies(const tlo_params *p, const double *phi, const double *pi, double a, double *out)
{
    const int N = p->N, nf = p->nf;
    const size_t n3 = (size_t)N * N * N;
    const int nq = 2 * nf + 1;
    const double dx = tlo_dx(p);
    double *plane = (double *)calloc((size_t)N * nq, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int z = 0; z < N; ++z) {
        double *acc = plane + (size_t)z * nq;
        for (int y = 0; y < N; ++y)
            for (int x = 0; x < N; ++x) {
                size_t s = site(N, x, y, z);
                double v[TLO_MAX_FIELDS];
                for (int f = 0; f < nf; ++f) {
                    const double *ph = phi + (size_t)f * n3;
                    const double *pp = pi + (size_t)f * n3;
                    v[f] = ph[s];
                    double gx = (ph[site(N, x + 1, y, z)] - ph[s]) / dx;
                    double gy = (ph[site(N, x, y + 1, z)] - ph[s]) / dx;
                    double gz = (ph[site(N, x, y, z + 1)] - ph[s]) / dx;
                    acc[f] += pp[s] * pp[s];
                    acc[nf + f] += gx * gx + gy * gy + gz * gz;
                }
                acc[2 * nf] += Vsite(p, v);
            }
    }
    double tot[2 * TLO_MAX_FIELDS + 1] = {0};
    for (int z = 0; z < N; ++z)
        for (int i = 0; i < nq; ++i) tot[i] += plane[(size_t)z * nq + i];
    free(plane);
    const double inv_n3 = 1.0 / (double)n3;
    const double ak = p->expanding ? pow(a, -6.0) : 1.0;
    const double ag = p->expanding ? pow(a, -2.0) : 1.0;
    for (int f = 0; f < nf; ++f) {
        out[f] = 0.5 * ak * tot[f] * inv_n3;
        out[nf + f] = 0.5 * ag * tot[nf + f] * inv_n3;
    }
    out[2 * nf] = tot[2 * nf] * inv_n3;
}

/* a'' from the energies at scale factor a. */
double tlo_fb(const tlo_params *p, const double *E, double a)
{
    double K = 0.0, G = 0.0;
    for (int f = 0; f < p->nf; ++f) { K += E[f]; G += E[p->nf + f]; }
    double V = E[2 * p->nf];
    return pow(a, 2.0 * p->alpha + 1.0) * (p->mu2 / 3.0)
         * ((p->alpha - 2.0) * K + p->alpha * G + (p->alpha + 1.0) * V);
}

/* |(b/a)^2 - a^(2 alpha) mu2 rho/3| / (b/a)^2; 0 in a static background. */
double tlo_hubble_residual(const tlo_params *p, const double *E, double a, double b)
{
    if (!p->expanding) return 0.0;
    double rho = 0.0;
    for (int i = 0; i < 2 * p->nf + 1; ++i) rho += E[i];
    double H2 = (b / a) * (b / a);
    double rhs = pow(a, 2.0 * p->alpha) * p->mu2 * rho / 3.0;
    return fabs(H2 - rhs) / H2;
}

/* ---- integrators -------------------------------------------------------- */

static void axpy(size_t n, double s, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < n; ++i) y[i] = y[i] + s * x[i];
}

static void b_kick(const tlo_params *p, const double *phi, const double *pi, double a, double *b, double s)
{
    double E[2 * TLO_MAX_FIELDS + 1];
    tlo_energies(p, phi, pi, a, E);
    *b = *b + s * tlo_fb(p, E, a);
}

/* One velocity-Verlet substep of size s, operators in palindromic order. */
static void vv_substep(const tlo_params *p, double *phi, double *pi, double *a, double *b, double s, double *F)
{
    const size_t n = (size_t)p->nf * p->N * p->N * p->N;
    if (p->expanding) b_kick(p, phi, pi, *a, b, 0.5 * s);
    tlo_force(p, phi, *a, F);
    axpy(n, 0.5 * s, F, pi);
    double c = 1.0;
    if (p->expanding) {
        double a_old = *a;
        *a = *a + s * *b;
        c = pow(0.5 * (a_old + *a), p->alpha - 3.0);
    }
    axpy(n, s * c, pi, phi);
    tlo_force(p, phi, *a, F);
    axpy(n, 0.5 * s, F, pi);
    if (p->expanding) b_kick(p, phi, pi, *a, b, 0.5 * s);
}

/* Leapfrog with half-step momenta.  On entry pi holds pi_0, on exit pi_n
 * = (pi_{n-1/2} + pi_{n+1/2})/2, written as pi_{n-1/2} + dt/2 F(phi_n). */
static void leapfrog(const tlo_params *p, double *phi, double *pi, double *a, double *b, double dt, int nsteps,
                     double *F, double *pih)
{
    const size_t n = (size_t)p->nf * p->N * p->N * p->N;
    if (nsteps <= 0) return;
    /* start: half kick of pi and b */
    if (p->expanding) b_kick(p, phi, pi, *a, b, 0.5 * dt);
    tlo_force(p, phi, *a, F);
    memcpy(pih, pi, n * sizeof(double));
    axpy(n, 0.5 * dt, F, pih); /* pi_{1/2} */
    for (int it = 0; it < nsteps; ++it) {
        /* drift */
        double c = 1.0;
        if (p->expanding) {
            double a_old = *a;
            *a = *a + dt * *b;
            c = pow(0.5 * (a_old + *a), p->alpha - 3.0);
        }
        axpy(n, dt * c, pih, phi);
        /* kick at the new positions */
        tlo_force(p, phi, *a, F);
        memcpy(pi, pih, n * sizeof(double));
        axpy(n, 0.5 * dt, F, pi); /* integer-time momentum */
        if (it + 1 < nsteps) {
            if (p->expanding) b_kick(p, phi, pi, *a, b, dt);
            axpy(n, dt, F, pih); /* pi_{n+1/2} */
        } else if (p->expanding) {
            b_kick(p, phi, pi, *a, b, 0.5 * dt);
        }
    }
}

/* Advance (phi, pi, a, b) by nsteps steps of size dt.  phi and pi hold nf
 * arrays of N^3 values each, back to back; ab = {a, b}.  Returns 0, or -1 on
 * an unknown integrator. */
int tlo_run(const tlo_params *p, double *phi, double *pi, double *ab, double dt, int nsteps, int integrator)
{
    const size_t n = (size_t)p->nf * p->N * p->N * p->N;
    double a = p->expanding ? ab[0] : 1.0;
    double b = p->expanding ? ab[1] : 0.0;
    double *F = (double *)malloc(n * sizeof(double));
    int rc = 0;
    if (integrator == TLO_VERLET) {
        for (int it = 0; it < nsteps; ++it) vv_substep(p, phi, pi, &a, &b, dt, F);
    } else if (integrator == TLO_LEAPFROG) {
        double *pih = (double *)malloc(n * sizeof(double));
        leapfrog(p, phi, pi, &a, &b, dt, nsteps, F, pih);
        free(pih);
    } else if (integrator == TLO_YOSHIDA4) {
        const double cr = cbrt(2.0);
        const double w1 = 1.0 / (2.0 - cr);
        const double w0 = -cr / (2.0 - cr);
        for (int it = 0; it < nsteps; ++it) {
            vv_substep(p, phi, pi, &a, &b, w1 * dt, F);
            vv_substep(p, phi, pi, &a, &b, w0 * dt, F);
            vv_substep(p, phi, pi, &a, &b, w1 * dt, F);
        }
    } else {
        rc = -1;
    }
    free(F);
    if (p->expanding) { ab[0] = a; ab[1] = b; }
    return rc;
}

/* ---- Philox-2x64-10 ---------------------------------------------------- */
/* Salmon et al., SC'11: each round maps (L, R) with key k to
 *   L' = hi(M R) xor k xor L,  R' = lo(M R)  (in their 2-word notation the
 * product word is the first input word), and the key is bumped by the Weyl
 * constant between rounds.  Multiplier and Weyl constant as published. */
static void philox2x64_10(const uint64_t ctr[2], uint64_t key, uint64_t out[2])
{
    const uint64_t M = 0xD2B74407B1CE6E93ULL;
    const uint64_t W = 0x9E3779B97F4A7C15ULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], k = key;
    for (int r = 0; r < 10; ++r) {
        unsigned __int128 prod = (unsigned __int128)M * (unsigned __int128)x0;
        uint64_t hi = (uint64_t)(prod >> 64);
        uint64_t lo = (uint64_t)prod;
        uint64_t nx0 = hi ^ k ^ x1;
        uint64_t nx1 = lo;
        x0 = nx0;
        x1 = nx1;
        k += W;
    }
    out[0] = x0;
    out[1] = x1;
}

void tlo_philox2x64(size_t n, const uint64_t *c0, uint64_t c1, uint64_t key, uint64_t *out)
{
    for (size_t i = 0; i < n; ++i) {
        uint64_t c[2] = {c0[i], c1};
        philox2x64_10(c, key, out + 2 * i);
    }
}
