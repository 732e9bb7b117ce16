/*
 * tl.h -- C ABI of the GB300 lattice stepper for interacting scalar fields on
 * a periodic 3D lattice in an expanding (FLRW) background.
 *
 * Model (program variables, tildes dropped; the paper prints the static phi^4
 * kick/drift of Sec. 4, the rest is the standard scalar field in FLRW written
 * in the alpha time variable):
 *   - N^3 sites, periodic, spacing dx = 2 pi/(kIR N), row-major with x
 *     fastest (the paper keeps row-major layout on every device, Sec. 3.3);
 *     host arrays are dense [z][y][x], device arrays carry one-site ghost
 *     copies like the paper's single ghost layer (tl_array_layout);
 *   - fields phi_f (f < n_fields <= 3) with momenta pi_f = a^(3-alpha) phi_f';
 *   - phi' = a^(alpha-3) pi,  pi' = a^(1+alpha) Lap phi - a^(3+alpha) dV/dphi,
 *     Lap the 7-point lattice Laplacian (Sec. 2 "LatLapl", Sec. 4);
 *   - V = sum_f m_f^2 phi_f^2/2 + lambda phi_0^4/4 + (q/2) phi_0^2 sum_{f>0} phi_f^2;
 *   - a'' = a^(2 alpha+1) (mu2/3) [(alpha-2) K + alpha G + (alpha+1) V],
 *     mu2 = (fstar/m_p)^2, with the volume averages
 *     K_f = a^-6 <pi_f^2>/2,  G_f = a^-2 <sum_i (forward difference)^2>/2,
 *     V = <V(phi)> (the paper's "average", Sec. 2 and Sec. 3.2);
 *   - Hubble constraint (a'/a)^2 = a^(2 alpha) mu2 (K+G+V)/3.
 *
 * Conventions (every function):
 *   - returns TL_OK (0) or a negative TL_E* code; tl_last_error() then gives
 *     a message (thread-local, valid until the next call on that thread);
 *   - host pointers are borrowed for the duration of the call;
 *   - device memory is owned by the lattice (tl_lattice_create) or by the
 *     caller (tl_lattice_create_with_buffers, which must keep it alive);
 *   - all device work is ordered on the lattice's CUDA stream; calls that
 *     return host data (tl_energies, tl_spectrum, tl_get_state) synchronise
 *     that stream, the others only enqueue work;
 *   - one lattice must not be used from two threads at once; distinct
 *     lattices are independent.
 */
#ifndef TL_H
#define TL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TL_MAX_FIELDS 3

/* Error codes. */
#define TL_OK 0
#define TL_EINVAL (-1)    /* bad argument (size, enum, pointer, field index) */
#define TL_ENOMEM (-2)    /* device allocation failed or would exceed the budget */
#define TL_ECUDA (-3)     /* a CUDA or cuFFT call failed */
#define TL_EUNSTABLE (-4) /* a reduced energy became non-finite (reported at the next sync) */
#define TL_ETIMEOUT (-5)  /* a bounded device wait expired */
#define TL_ESTATE (-6)    /* call out of order (e.g. stepping before a potential and a state exist) */

typedef struct tl_lattice tl_lattice; /* opaque, owned by the library */

typedef enum { TL_F32 = 0, TL_F64 = 1 } tl_dtype;

/* TL_LEAPFROG is the paper's kick-then-drift with half-step momenta (Sec. 4);
 * TL_VERLET the palindromic velocity Verlet; both advance phi identically and
 * run one fused pass per step.  TL_YOSHIDA4 composes three Verlet substeps
 * with weights w1, w0, w1 (w1 = 1/(2-2^(1/3)), w0 = -2^(1/3) w1): three
 * passes per step. */
typedef enum { TL_LEAPFROG = 0, TL_VERLET = 1, TL_YOSHIDA4 = 2 } tl_integrator;

/* Background.  expanding = 0: static box, a = 1, b = a' = 0, alpha unused. */
typedef struct {
    int expanding;
    double alpha;         /* d eta = a^-alpha dt */
    double fstar_over_mp; /* sets mu2 = fstar_over_mp^2 */
    double a0;            /* scale factor at initialisation (tl_init_fluctuations) */
} tl_expansion;

/* Potential family above.  Fields beyond n_fields are ignored. */
typedef struct {
    double lambda;
    double q;
    double m2[TL_MAX_FIELDS];
} tl_potential;

/* Initial state for tl_init_fluctuations: homogeneous values plus a Gaussian
 * random field per field f.  Every mode n (k = kIR n) with 0 < |n| < N/2 gets
 * <|d(n)|^2> = P(k)/L^3, P(k) = A/(2 omega_k), omega_k^2 = k^2 + meff2[f]:
 * Rayleigh modulus, uniform phase, Hermitian pairs, drawn with Philox-2x64-10
 * (the paper's generator, Sec. 2) from counter (mode index, f) and key seed.
 * fluct_pi != 0 adds an independent draw with P = A omega_k/2 to pi_f
 * (counter (mode index, 8+f)), scaled by a0^(3-alpha).  fixed_modulus != 0
 * gives every mode the modulus sqrt(P(k)/L^3) exactly (random phase only)
 * instead of the Rayleigh modulus; both have <|d(n)|^2> = P(k)/L^3. */
typedef struct {
    double A;
    double meff2[TL_MAX_FIELDS];
    double phi0[TL_MAX_FIELDS];
    double pi0[TL_MAX_FIELDS];
    int fluct_pi;
    int fixed_modulus;
} tl_init_spec;

/* Volume averages and background at the last integer time. */
typedef struct {
    int64_t step;       /* completed time steps since the last init/set_state */
    double time;        /* program time eta since then */
    double a, b;        /* scale factor and a' */
    double K[TL_MAX_FIELDS], G[TL_MAX_FIELDS], V;
    double hubble_resid; /* |(b/a)^2 - a^(2 alpha) mu2 (K+G+V)/3| / (b/a)^2; 0 if static */
} tl_energies_t;

/* Create a lattice and allocate its device state (4 n_fields arrays of N^3
 * elements: phi and pi, ping-pong, plus O(grid) scratch for the fused
 * reductions).  Passage: Sec. 2, the memory toolbox of an N^3 box with one
 * ghost layer (MemoryToolBox::makeShared) and the scalar fields living on it
 * (Field<T, 3>, float or double); here phi and pi of every field are one
 * device allocation owned by the lattice.  N >= 8 and N % 4 == 0; 1 <= n_fields <= 3; kIR > 0;
 * expansion may be NULL (static).  cuda_stream is a cudaStream_t (NULL: the
 * legacy default stream).  The lattice needs a potential
 * (tl_set_potential) and a state (tl_init_fluctuations or tl_set_state)
 * before tl_step.  Errors: TL_EINVAL, TL_ENOMEM, TL_ECUDA. */
int tl_lattice_create(tl_lattice **out, int N, double kIR, int n_fields, tl_dtype dtype,
                      const tl_expansion *expansion, void *cuda_stream);

/* As tl_lattice_create (Sec. 2, toolbox and fields), but the 4 n_fields
 * field arrays live in caller-owned device memory: dev_ptrs[4 f + 0] phi_f (A), [4 f + 1] pi_f (A),
 * [4 f + 2] phi_f (B), [4 f + 3] pi_f (B); each holds the `elems` elements of
 * dtype that tl_array_layout gives (the padded layout), 16-byte aligned;
 * n_ptrs == 4 n_fields. */
int tl_lattice_create_with_buffers(tl_lattice **out, int N, double kIR, int n_fields, tl_dtype dtype,
                                   const tl_expansion *expansion, void *cuda_stream,
                                   void *const *dev_ptrs, size_t n_ptrs);

/* Device bytes tl_lattice_create would allocate for the field arrays (the
 * padded layout of tl_array_layout; no counterpart in the paper). */
size_t tl_state_bytes(int N, int n_fields, tl_dtype dtype);

/* Device layout of one field array of a lattice (Sec. 3.3: row-major on
 * every device; Sec. 3.1 and Sec. 4: one ghost layer).  Every z-plane carries
 * one ghost row above and below (copies of rows N - 1 and 0, kept current by
 * every pass), so that a tile's rows plus the rows around it are one in-bounds
 * box; every row has W = 16/sizeof reserved elements on each side (x in
 * [-W, 0) and [N, N + W)), which the library does not keep (at the x-edges the
 * pass reads the periodic image itself).  Element (x, y, z) is at
 * origin + z plane_pitch + y row_pitch + x; rows start x = 0 on a 128-byte
 * boundary (a left pad of 128 bytes) and row_pitch is a multiple of 128
 * bytes; plane_pitch = (N + 2) row_pitch, origin = row_pitch + 128/sizeof,
 * elems = N plane_pitch elements per array.  Any output may be NULL. */
int tl_array_layout(int N, tl_dtype dtype, size_t *elems, size_t *row_pitch, size_t *plane_pitch, size_t *origin);

/* Free a lattice and the device memory it owns (caller-owned buffers of
 * tl_lattice_create_with_buffers are left alone) after synchronising its
 * stream; NULL is a no-op, and so is a lattice still held by a tl_batch
 * (destroy the batch first).  No counterpart in the paper (its toolbox is
 * reference-counted). */
void tl_lattice_destroy(tl_lattice *lat);

/* Set the potential (may be changed between steps).  Passage: Sec. 4, the
 * quartic self-interaction (and mass term) in the kick of the phi^4
 * benchmark; the two-field coupling q phi_0^2 phi_f^2/2 is the family the
 * workloads need.  Errors: TL_EINVAL (NULL, non-finite coefficients). */
int tl_set_potential(tl_lattice *lat, const tl_potential *pot);

/* Passage: Sec. 2, Gaussian random fields drawn from Random123's counter-based
 * Philox 2x64 in Fourier space (the field's Fourier view, Sec. 2 and
 * Sec. 3.5); the spectrum A/(2 omega_k) is the workloads' vacuum spectrum.
 * Draw the initial state (see tl_init_spec), set a = a0 and, when expanding,
 * b = a0^(1+alpha) sqrt(mu2 rho0/3) with rho0 the lattice-averaged K+G+V of
 * that state.  Uses cuFFT (c2r, FP64) and temporary device memory of about
 * 16 N^3 bytes.  Resets step and time to 0. */
int tl_init_fluctuations(tl_lattice *lat, uint64_t seed, const tl_init_spec *spec);

/* Passage: Sec. 4, the kick-drift leapfrog of the phi^4 benchmark (kick
 * pi += dt (Lap phi - dV/dphi), drift phi += dt pi, 7-point stencil), here
 * with the expansion weights of the model above.
 * Advance n >= 0 steps of size dt (negative dt runs backwards).  The state
 * stays resident; the call only enqueues work: n P + 1 fused passes (P = 1
 * for leapfrog/Verlet, 3 for Yoshida), each one kernel that drifts phi,
 * applies the Laplacian, dV/dphi and the expansion-weighted kick, and reduces
 * K, G, V, followed in-kernel by the FP64 scale-factor update.  A non-finite
 * energy is reported by the next tl_energies / tl_get_state as TL_EUNSTABLE.
 * Errors: TL_EINVAL, TL_ESTATE, TL_ECUDA. */
int tl_step(tl_lattice *lat, int n, double dt, tl_integrator integrator);

/* Passage: Sec. 2.1, the volume average of an expression (average(...));
 * Sec. 3.2, the device reduction over a lattice (device::iteration::reduce).
 * Synchronise the lattice stream and return the energies at the current
 * integer time (measured on the device if the state was set since the last
 * step).  Errors: TL_EINVAL (NULL), TL_ESTATE (no state), TL_EUNSTABLE,
 * TL_ETIMEOUT, TL_ECUDA. */
int tl_energies(tl_lattice *lat, tl_energies_t *out);

/* Number of spectrum bins for size N: ceil(sqrt(3) N/2) + 1 (the shells of
 * tl_spectrum). */
int tl_spectrum_bins(int N);

/* Passage: Sec. 2, a field's Fourier-space view (inFourierSpace), and
 * Sec. 3.5, DFTs used for measurements such as power spectra.
 * Binned power spectrum of phi_field (which = 0) or pi_field (which = 1):
 * d(n) = N^-3 sum_x f(x) exp(-i k.x), bin b = floor(|n| + 1/2),
 * P_b = L^3 mean_{n in b} |d(n)|^2, k_b = kIR mean_{n in b} |n|, count_b =
 * modes in the bin (all N^3 modes, both members of each pair).  Host arrays
 * of nbins >= tl_spectrum_bins(N) entries; any may be NULL.  Bin sums use
 * FP64 atomics (reproducible to rounding, not bitwise).  Synchronises. */
int tl_spectrum(tl_lattice *lat, int field, int which, int nbins, double *k, double *P, int64_t *count);

/* Passage: Sec. 3.3, the row-major layout of a field ([z][y][x], x fastest,
 * ghosts stripped); used for checkpoints and tests.
 * Copy phi_field (which = 0) or pi_field (which = 1) at the current integer
 * time to host memory of bytes = N^3 * element size ([z][y][x], x fastest).
 * Synchronises.  TL_EUNSTABLE if the evolution went non-finite. */
int tl_get_state(tl_lattice *lat, int field, int which, void *host, size_t bytes);

/* Passage: Sec. 3.3, as tl_get_state (assignment of a field from host data;
 * the ghost copies are refilled on the device).
 * Overwrite phi_field or pi_field from host memory (same layout and size as
 * tl_get_state).  Resets step and time to 0; the energies are re-measured
 * on demand.  Call tl_set_background afterwards when expanding. */
int tl_set_state(tl_lattice *lat, int field, int which, const void *host, size_t bytes);

/* No counterpart in the paper (its benchmarks run in a static box): the
 * background of the FLRW model above.
 * Set the scale factor a and a' = b; from_constraint != 0 ignores b and sets
 * b = a^(1+alpha) sqrt(mu2 rho/3) from the current state's energies. */
int tl_set_background(tl_lattice *lat, double a, double b, int from_constraint);

/* No counterpart in the paper (checkpoint and resume of a run).
 * The lattice's counters: completed time steps and program time eta since the
 * last tl_init_fluctuations / tl_set_state / tl_commit_state, and the Langevin
 * steps taken since then (the noise counter of tl_langevin_step). */
typedef struct {
    int64_t step;
    double time;
    int64_t langevin_steps;
} tl_clock;

/* Read the counters.  Synchronises the lattice stream.
 * Errors: TL_EINVAL (NULL), TL_ECUDA. */
int tl_get_clock(tl_lattice *lat, tl_clock *out);

/* Restore the counters of a checkpoint: after tl_set_state of every array and
 * tl_set_background(a, b, 0) with a, b of tl_energies, a lattice of the same
 * size, fields, precision, potential and pass shape then continues bitwise as
 * the one the checkpoint was taken from, under the same tl_step calls.  Call it
 * last (tl_set_state and tl_set_background reset the counters).
 * Synchronises.  Errors: TL_EINVAL (NULL, negative counts, non-finite time),
 * TL_ESTATE (no state, or in a batch), TL_ECUDA. */
int tl_set_clock(tl_lattice *lat, const tl_clock *clock);

/* No counterpart in the paper (zero-copy access for callers on the device).
 * Device address of element (0, 0, 0) of phi_field / pi_field of the current
 * state (padded layout, see tl_array_layout; valid until the next tl_step). */
int tl_state_device_ptr(tl_lattice *lat, int field, int which, void **dev_ptr);

/* No counterpart in the paper (pairs with tl_state_device_ptr).
 * The caller has written every phi_f and pi_f of the current state directly on
 * the device (through tl_state_device_ptr or its own buffers of
 * tl_lattice_create_with_buffers, interior sites in the padded layout): refresh
 * their ghost rows and take them as the state, like tl_set_state of every
 * array without a host copy (step and time reset to 0, a = a0, b = 0; call
 * tl_set_background afterwards when expanding).  Synchronises the lattice
 * stream (the caller's writes must be ordered before the call on that stream
 * or complete).  Errors: TL_EINVAL (NULL), TL_ESTATE (in a batch), TL_ECUDA. */
int tl_commit_state(tl_lattice *lat);

/* Energies of a caller-owned device state, allocating no device memory.
 * No counterpart in the paper: this serves callers that cannot call
 * cudaMalloc (a host framework that owns all device memory, or code that must
 * not trigger the device synchronisation an allocation can cause).
 * phi[f], pi[f] (f < n_fields): device arrays of N^3 elements of dtype,
 * 16-byte aligned, laid out as in tl_get_state; pot: the potential;
 * expansion: NULL or static for a = 1 weights, else the scale factor a
 * weighs K by a^-6 and G by a^-2.  out: host array of 2 n_fields + 1
 * doubles, K_0.., G_0.., V.  The pass runs on cuda_stream and the call
 * synchronises it.
 * Scratch: a fixed 917,760-byte array inside the library (static device memory that
 * every GPU loading the library holds until exit) with room for 16384 CTA
 * partial sums, enough for N <= 1024 in both precisions; larger lattices get
 * TL_EINVAL.  The first call on each device looks up the array's address
 * (cudaGetSymbolAddress) and keeps it for the life of the process, so make
 * that call before any stream capture; a device reset (cudaDeviceReset, or a
 * reset of the primary context) invalidates the kept address, and later calls
 * on that device are then invalid.  All calls
 * share the array: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.
 * Errors: TL_EINVAL, TL_ECUDA, TL_EUNSTABLE (non-finite energies). */
int tl_energies_noalloc(int N, double kIR, int n_fields, tl_dtype dtype, const tl_potential *pot,
                        const tl_expansion *expansion, double a, const void *const *phi, const void *const *pi,
                        void *cuda_stream, double *out);

/* Page-locked host memory for the state copies (tl_get_state, tl_set_state,
 * tl_su2_get/set and any cudaMemcpy of the caller): anonymous memory with
 * transparent huge pages requested (start and length aligned to the huge
 * page size for buffers of at least one), every page faulted in, and the
 * range registered with CUDA (cudaHostRegister): one address translation per
 * huge page instead of per base page for the copies (their measured rates
 * against cudaHostAlloc memory varied between hosts).  *out receives a pointer to `bytes` writable bytes
 * (zero-filled), owned by the caller until tl_host_free.  No counterpart in
 * the paper.  Errors: TL_EINVAL (NULL out, bytes 0), TL_ENOMEM (the mapping
 * failed), TL_ECUDA (registration failed; nothing is left allocated). */
int tl_host_alloc(size_t bytes, void **out);

/* Unregister and unmap memory from tl_host_alloc; NULL is a no-op.  The
 * caller must have no copy in flight on it.  Errors: TL_EINVAL (a pointer
 * tl_host_alloc did not return, or one already freed), TL_ECUDA. */
int tl_host_free(void *ptr);

/* ---- Langevin evolution (Sec. 2, Eq. 1: the paper's interface example) ---- */

typedef struct {
    double lambda; /* the drift is Lap phi - m2 phi - (lambda/2) phi^3 */
    double m2;
    double noise;  /* amplitude of eta: <eta eta> = noise^2 delta(t-t') per site */
} tl_langevin_params;

/* n Euler-Maruyama steps of phi_0:  phi <- phi + dt (Lap phi - m2 phi -
 * lambda/2 phi^3) + noise sqrt(dt) xi, xi a unit Gaussian per site and step:
 * the sites of dense index s = [z][y][x] = 2k and 2k + 1 share Philox-2x64-10
 * of counter (k, 2^63 + step) under key seed; Box-Muller on the two words
 * (u1 = (w0 >> 11 + 1) 2^-53, u2 = (w1 >> 11) 2^-53, r = sqrt(-2 ln u1))
 * gives xi(2k) = r cos(2 pi u2) and xi(2k + 1) = r sin(2 pi u2).  Steps are counted
 * from the last tl_set_state / tl_init_fluctuations.  Only phi_0 evolves (the
 * momenta are untouched); the energies are re-measured on demand.  Enqueues
 * only.  Errors: TL_EINVAL, TL_ESTATE (phi_0 not set, or in a batch), TL_ECUDA. */
int tl_langevin_step(tl_lattice *lat, int n, double dt, const tl_langevin_params *p, uint64_t seed);

/* ---- SU(2) Yang-Mills in temporal gauge (Sec. 4 benchmark workload) ----
 * Links U_i(x) in SU(2) as unit quaternions (u0, u1, u2, u3) meaning
 * u0 + i (u1 s1 + u2 s2 + u3 s3); electric fields E_i(x) = i e_i.s as 3-vectors.
 * Host layout, component-major: U[i][c][z][y][x] (3 x 4 arrays of N^3) and
 * E[i][c][z][y][x] (3 x 3 arrays), elements of dtype.  On the device the
 * links are quaternion records U[i][z][y][x][c] (one vector load per link)
 * and E keeps the host layout.  Lattice units
 * (dx = 1).  One step is the paper's leapfrog: kick
 * e_i(x) <- e_i(x) - 2 dt sum_{j != i} Im[U_i(x) S_ij(x)] with the staples
 * S_ij(x) = U_j(x+i) U_i(x+j)^+ U_j(x)^+ + U_j(x+i-j)^+ U_i(x-j)^+ U_j(x-j)
 * (the paper's E+ = E - dt sum_j (P_ij - P_ij^+)), then drift
 * U_i(x) <- exp(dt E_i(x)) U_i(x) (closed-form exponential map), fused in one
 * pass per step.  FP32 links are renormalised to unit length after each drift.
 * The kick evaluates the staple sum through plaquettes, an identity that holds
 * for unit quaternions: links given to tl_su2_set_state must be normalised
 * (to the precision of dtype); a deviation d of |U|^2 from 1 enters the force
 * at relative order d. */

typedef struct tl_su2 tl_su2; /* opaque */

/* Allocate the links (two copies), the fields and measurement scratch:
 * 33 N^3 elements.  4 <= N <= 1290.  Errors: TL_EINVAL, TL_ENOMEM, TL_ECUDA. */
int tl_su2_create(tl_su2 **out, int N, tl_dtype dtype, void *cuda_stream);
void tl_su2_destroy(tl_su2 *lat);
/* Copy the whole state from / to host memory (layout above); synchronises. */
int tl_su2_set_state(tl_su2 *lat, const void *U, const void *E);
int tl_su2_get_state(tl_su2 *lat, void *U, void *E);
/* Random links q/|q|, q = (1, amp g1, amp g2, amp g3), g standard normal from
 * Philox-2x64-10 (counter (3 site + i, 2^62 + h), key seed, Box-Muller), and
 * E = 0 (so Gauss's law holds exactly).  Enqueues only. */
int tl_su2_init_random(tl_su2 *lat, uint64_t seed, double amp);
/* n leapfrog steps of size dt (kick then drift).  Enqueues only. */
int tl_su2_step(tl_su2 *lat, int n, double dt);
/* out4 = {<sum_i |e_i|^2/2>, <sum_{i<j} 2 (1 - Re P_ij)>, max_x |G(x)|,
 * sqrt(<|G|^2>)} with G(x) = sum_i [E_i(x) - U_i(x-i)^+ E_i(x-i) U_i(x-i)]
 * (Gauss's law), averages over sites; fixed-order FP64 sums.  Synchronises. */
int tl_su2_measure(tl_su2 *lat, double *out4);

/* Launch shape of the fused pass (the one kernel a step launches per
 * (sub)step, Sec. 4's kick and drift with the energy sums of Sec. 3.2).
 * Both kinds compute every site with the same operations in the same order,
 * so fields agree bitwise between them; only the energy sums, whose order
 * follows the CTA tiles, differ by rounding (and through a'' the fields of an
 * expanding run).
 *   TL_PASS_STREAM  each thread streams its column of sites through z-planes
 *                   in registers, neighbour rows from L1/L2 (the shape the
 *                   batched launch runs);
 *   TL_PASS_TMA     a producer warp stages tile-plus-halo boxes of each plane
 *                   in shared memory with tensor copies (cp.async.bulk.tensor)
 *                   through a ring of mbarrier-guarded stages; compute warps
 *                   read neighbours from the stage. */
typedef enum { TL_PASS_STREAM = 0, TL_PASS_TMA = 1 } tl_pass_kind;

typedef struct {
    int kind;    /* tl_pass_kind */
    int warps;   /* TMA: compute warps per CTA, 7 (two CTAs per SM) or 15 (one); 0 = 7 */
    int stages;  /* TMA: ring depth 3..8; 0 = as deep as the shared memory allows */
    int z_chunk; /* z-planes per CTA, 1..N; 0 = automatic (at least ~8 CTAs per SM) */
    int tile_x;  /* STREAM: threads along a tile row, 8, 16 or 32; 0 = 32 */
    int threads; /* STREAM: threads per CTA, 256 or 512; 0 = 256 */
} tl_pass_config;

/* ---- batched ensembles and launch tuning (beyond the paper's single
 * lattice: many independent small lattices advanced together) ---- */

typedef struct tl_batch tl_batch; /* opaque */

/* Group n existing lattices (same dtype; any N, n_fields, potential,
 * background) into a batch that tl_batch_step advances together (a lattice
 * belongs to at most one batch at a time).  Each lattice is moved to the
 * batch launch shape of its size (tl_batch_pass_config) if it is not on it,
 * and keeps it afterwards; a batch step is bitwise tl_step of the lattice
 * alone on that shape.  The batch's launch options are those
 * tl_batch_autotune found for the same composition (multiset of N, fields,
 * dtype) earlier in the process or in TL_TUNE_FILE, else the defaults.  The
 * lattices stay owned by the caller and cannot be destroyed or autotuned
 * while the batch exists; their own calls (tl_energies, tl_get_state,
 * tl_spectrum ...) keep working between batch steps.  cuda_stream: the
 * stream the batch runs on.  No counterpart in the paper (Sec. 3.2's foreach
 * over one lattice, here over many).  Errors: TL_EINVAL, TL_ENOMEM, TL_ECUDA. */
int tl_batch_create(tl_batch **out, tl_lattice *const *lats, int n, void *cuda_stream);

/* The launch shape tl_batch_create gives a lattice of this size on the
 * current device: the TL_PASS_STREAM kernel with 256-thread CTAs, with the
 * z-chunk and tile row width tl_batch_autotune measured for (N, n_fields,
 * dtype, SM count) if it has, else z-chunks of min(N, 32) planes.  Set it
 * with tl_set_pass_config on a lattice that should step alone bitwise like
 * its batched twin.  Errors: TL_EINVAL. */
int tl_batch_pass_config(int N, int n_fields, tl_dtype dtype, tl_pass_config *out);

/* Advance every lattice of the batch by n steps of size dt, as tl_step
 * would, with one persistent launch per pass and per field count (each
 * launch walks all lattices' CTA tiles), the whole pass sequence captured
 * once as a CUDA graph per (n, dt, integrator) and replayed; with the
 * "split" option the field-count groups are independent branches of that
 * graph, so their launches overlap on the device.  Each lattice keeps its
 * own launch geometry and reduction order, so its results are bitwise those
 * of tl_step on it alone.  Enqueues only. */
int tl_batch_step(tl_batch *batch, int n, double dt, tl_integrator integrator);

/* Choose the batch's launch shapes by measurement: for each class of members
 * (same N and n_fields), largest total work first, time the z-chunks 4 ... N
 * and tile row widths of the streaming kernel with the other classes held,
 * keep the fastest (one coordinate-descent sweep); then the batch-level
 * options (per-thread prefetch ring, field-count groups as graph branches,
 * persistent grid split by work).  Each candidate is timed as CUDA-graph
 * replays of the whole batch's grouped passes with zero kick and drift
 * coefficients, which rewrite every state unchanged.  The members keep the
 * chosen shapes; the shapes (per N, n_fields, dtype, SM count) and the
 * options (per composition) are cached for later tl_batch_create calls in
 * the process and appended to TL_TUNE_FILE when that names a file.
 * best_ms_per_pass (may be NULL): the winner's time per grouped pass.
 * Synchronises.  No counterpart in the paper.  Errors: TL_EINVAL, TL_ESTATE,
 * TL_ECUDA. */
int tl_batch_autotune(tl_batch *batch, double *best_ms_per_pass);

/* The batch's launch options: prefetch (0 or 3 planes), split (field-count
 * groups as independent graph branches, 0/1), share (persistent grid split
 * among the groups by work, 0/1); any output may be NULL. */
int tl_batch_get_options(const tl_batch *batch, int *prefetch, int *split, int *share);

void tl_batch_destroy(tl_batch *batch);

/* Time candidate launch shapes of the fused pass on this lattice (both
 * kinds of tl_pass_config: z-planes per CTA from 4 to the whole lattice, the
 * tile rows and CTA size of the streaming kernel, the warps of the TMA kernel) with
 * passes whose kick and drift coefficients are zero, which rewrite the state
 * unchanged, and keep the fastest.  Results are cached per (N, n_fields,
 * dtype, SM count) for the process and, if the environment variable
 * TL_TUNE_FILE names a file, appended there as one JSON object per line and
 * reused by later processes.  best_ms_per_pass (may be NULL) receives the winner's time.
 * Synchronises the lattice stream.  Errors: TL_ESTATE (in a batch), TL_ECUDA. */
int tl_autotune(tl_lattice *lat, double *best_ms_per_pass);

/* Set the launch shape of lat's fused pass (takes effect at the next launch;
 * the lattice's state is untouched).  tl_pass_config fields: tile_x 0, 8, 16
 * or 32 (threads along x of the streaming kernel's tiles; a lattice whose rows
 * need fewer threads, N/4 FP32 or N/2 FP64 below 32, also takes that count,
 * as tl_get_pass_config reports it), threads 0, 256 or 512, TMA warps 0, 7 or
 * 15, stages 0 or 3..8, z_chunk 0..N (0: automatic), so every shape
 * tl_get_pass_config returns can be set again.  Values out of range are TL_EINVAL;
 * TL_ESTATE while the lattice is in a batch.  May synchronise the lattice
 * stream (to grow its reduction slots).  A new lattice starts on TL_PASS_TMA
 * when it is FP32 and N >= 192 (z-chunks of 48 planes at N = 192, 64 up to
 * N = 319, then 56, 80, 160 (one field) or 96, 104, 72 and 76 planes around
 * N = 384, 448, 512, 576 ... 768, 896 and 1024, where they measured fastest;
 * 15 compute warps from N = 416, else 7), on
 * TL_PASS_STREAM otherwise (where those measured faster; FP64 from N = 128
 * with z-chunks of 32 planes, 64 from N = 512); the environment
 * variable TL_PASS_VARIANT=tma|ldg overrides that default at creation. */
int tl_set_pass_config(tl_lattice *lat, const tl_pass_config *cfg);

/* The launch shape lat runs now, with automatic values resolved. */
int tl_get_pass_config(const tl_lattice *lat, tl_pass_config *cfg);

/* Diagnostic (no counterpart in the paper): the device's FP64 and FP32 FMA
 * issue rates in FMA operations per second, measured by timing a kernel of
 * independent FMA chains over 8 CTAs of 256 threads per SM.  They are the
 * arithmetic roofline of passes bound by the FP64 pipe.  Synchronises
 * cuda_stream.  Errors: TL_EINVAL (NULL), TL_ENOMEM, TL_ECUDA. */
int tl_probe_fma_rates(double *fp64_fma_per_s, double *fp32_fma_per_s, void *cuda_stream);

/* Message for the last error on this thread ("" if none); no counterpart in
 * the paper. */
const char *tl_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TL_H */
