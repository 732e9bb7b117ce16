// Fused lattice pass: deferred drift + 7-point Laplacian + dV/dphi + kick +
// K/G/V reductions + (last CTA) FP64 scale-factor update, in one kernel.
//
// The paper's step (Sec. 4) is a kick pi+ = pi + dt (Lap phi - dV/dphi) and a
// drift phi+ = phi + dt pi+, each its own bandwidth-bound sweep.  Here the
// drift of step n is deferred into the pass of step n+1: a pass reads the
// stored (phi_s, pi_s), forms phi = phi_s + drift pi_s for each site and its
// six neighbours (one fma, bitwise the same wherever it is recomputed),
// evaluates F = a^(1+alpha) Lap phi - a^(3+alpha) dV/dphi, and writes phi and
// pi_s + kdt F to the other ping-pong buffer.  With expansion the drift
// coefficient depends on the scale factor after the b-kick, which needs the
// energies of this same pass; the last CTA to finish computes it and leaves
// it in device memory for the next pass, so the host never waits.
//
// Layout and traffic: each thread owns W = 16/sizeof(T) consecutive x-sites
// (one 128-bit word per array) of one y-row and marches a chunk of z-planes,
// keeping phi at z-1, z, z+1 in registers; the neighbour rows and edge sites
// come through L1/L2 (fused_pass_ldg).  HBM sees each array read once and
// written once per pass: 4 sizeof(T) bytes per site per field.
#pragma once
#include <cuda.h>
#include <math.h>

#include <atomic>

#include "tl_internal.cuh"

namespace tl {

template <typename T>
struct Vec;
template <>
struct Vec<float> {
    static constexpr int W = 4;
    typedef float4 type;
};
template <>
struct Vec<double> {
    static constexpr int W = 2;
    typedef double2 type;
};

__device__ __forceinline__ void load_vec(const float *p, float (&o)[4])
{
    float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void load_vec(const double *p, double (&o)[2])
{
    double2 t = __ldg(reinterpret_cast<const double2 *>(p));
    o[0] = t.x; o[1] = t.y;
}
__device__ __forceinline__ void store_vec(float *p, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store_vec(double *p, const double (&v)[2])
{
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}
__device__ __forceinline__ void load_vec_s(const float *p, float (&o)[4])
{
    float4 t = *reinterpret_cast<const float4 *>(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void load_vec_s(const double *p, double (&o)[2])
{
    double2 t = *reinterpret_cast<const double2 *>(p);
    o[0] = t.x; o[1] = t.y;
}
// streaming (evict-first) stores: the outputs are read again only by the next pass
__device__ __forceinline__ void store_vec_cs(float *p, const float (&v)[4])
{
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
}
__device__ __forceinline__ void store_vec_cs(double *p, const double (&v)[2])
{
    __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
}
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// x^e: integer exponents up to 16 in magnitude by repeated squaring (a few
// multiplications instead of a pow() on the FP64 unit, which this last-CTA
// tail would otherwise serialise every pass); other exponents by pow().
__device__ __forceinline__ double powe(double x, double e)
{
    const double r = rint(e);
    if (r == e && fabs(r) <= 16.0) {
        int n = (int)fabs(r);
        double acc = 1.0, b = x;
        while (n) {
            if (n & 1) acc *= b;
            b *= b;
            n >>= 1;
        }
        return r < 0.0 ? 1.0 / acc : acc;
    }
    return pow(x, e);
}

// Scale-factor update and next-pass coefficients (one thread of the last CTA).
// tot: raw lattice sums  [sum pi_int_f^2, sum |grad+ phi_f|^2 dx^2, sum V].
static __device__ void finalize(const Model &m, const PassCoef &c, Scalars *sc, const double *tot)
{
    const int nf = m.nf;
    const double n3 = (double)m.N * (double)m.N * (double)m.N;
    const double a = sc->a;
    double E[kMaxQ];
    double K = 0.0, G = 0.0;
    bool finite = true;
    for (int f = 0; f < nf; ++f) {
        E[f] = 0.5 * sc->wk * (tot[f] / n3);
        E[nf + f] = 0.5 * sc->wg * m.inv_dx2 * (tot[nf + f] / n3);
        K += E[f];
        G += E[nf + f];
    }
    const double V = tot[2 * nf] / n3;
    E[2 * nf] = V;
    for (int i = 0; i < 2 * nf + 1; ++i) {
        finite = finite && isfinite(E[i]);
        if (c.integer_time) sc->E[i] = E[i];
    }
    if (!finite && sc->status == TL_OK) sc->status = TL_EUNSTABLE;
    sc->time += sc->pending_dt;
    if (m.expanding) {
        const double al = m.alpha;
        const double rho = K + G + V;
        double b = sc->b, b_eval;
        if (c.set_b_from_constraint) {
            b = powe(a, 1.0 + al) * sqrt(m.mu2 * rho / 3.0);
            b_eval = b;
        } else {
            const double fb = powe(a, 2.0 * al + 1.0) * (m.mu2 / 3.0) * ((al - 2.0) * K + al * G + (al + 1.0) * V);
            b_eval = b + c.hb_dt * fb;
            b = b + c.edt * fb;
        }
        if (c.integer_time) {
            const double H2 = (b_eval / a) * (b_eval / a);
            sc->hubble = fabs(H2 - powe(a, 2.0 * al) * m.mu2 * rho / 3.0) / H2;
        }
        const double an = a + c.dnext_dt * b;
        sc->drift = c.dnext_dt * powe(0.5 * (a + an), al - 3.0);
        sc->a = an;
        sc->b = b;
        sc->wl = powe(an, 1.0 + al);
        sc->wv = powe(an, 3.0 + al);
        sc->wk = powe(an, -6.0);
        sc->wg = powe(an, -2.0);
    } else {
        sc->drift = c.dnext_dt;
        sc->hubble = 0.0;
    }
    sc->pending_dt = c.dnext_dt;
}

// ---- pieces shared by both pass variants ------------------------------------

// Per-pass constants in the storage precision.
template <typename T, int NF>
struct Coefs {
    T drift, wlx, wv, kdt, hdt, lam, q;
    T m2[NF];
    T qlam, hq;  // lambda/4, q/2 (the potential's own coefficients, FP64 form)
    T hm2[NF];   // m2/2
    T wlam, wq;  // a^(3+alpha) lambda, a^(3+alpha) q (the force's weight folded in, FP64 form)
    T wm2[NF];   // a^(3+alpha) m2
};

template <typename T, int NF>
__device__ __forceinline__ Coefs<T, NF> make_coefs(const Model &m, const PassCoef &c, const Scalars *sc)
{
    Coefs<T, NF> k;
    k.drift = (T)sc->drift;
    k.wlx = (T)(sc->wl * m.inv_dx2);
    k.wv = (T)sc->wv;
    k.kdt = (T)c.kdt;
    k.hdt = (T)c.hdt;
    k.lam = (T)m.lambda;
    k.q = (T)m.q;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        k.m2[f] = (T)m.m2[f];
        k.hm2[f] = (T)(0.5 * m.m2[f]);
    }
    k.qlam = (T)(0.25 * m.lambda);
    k.hq = (T)(0.5 * m.q);
    k.wlam = (T)(sc->wv * m.lambda);
    k.wq = (T)(sc->wv * m.q);
#pragma unroll
    for (int f = 0; f < NF; ++f) k.wm2[f] = (T)(sc->wv * m.m2[f]);
    return k;
}



// Update W consecutive sites of one row of plane z, all fields: Laplacian from
// the six neighbours (differences first, so FP32 keeps the small gradients
// exact), dV/dphi, the kick, and the K/G/V sums at the evaluation time.
// cu/zm/zp: phi at z, z-1, z+1; ym/yp: rows y-1, y+1; xl/xr: the sites left of
// element 0 and right of element W-1; pc: stored pi at z.
//
// FP64 (bound by the FP64 pipe) takes the same quantities with fewer FP64
// operations: the Laplacian as the neighbour sum minus 6 phi; the potential and
// its derivative in factored form, phi^2 (m2/2 + lambda phi^2/4) accumulated
// straight into the sum, and a^(3+alpha) dV/dphi = phi (a^(3+alpha) m2 +
// a^(3+alpha) lambda phi^2) with the force's weight folded into the
// coefficients; and the gradient energy by summation by parts, which on a
// periodic lattice is exact: sum_x sum_i (phi(x+i) - phi(x))^2
// = -sum_x phi(x) (sum_i [phi(x+i) + phi(x-i)] - 6 phi(x)), so each site adds
// -phi times the Laplacian it has already formed (one fma instead of three
// differences and three squares).  The lattice-wide sums are the same
// numbers up to rounding; per site the terms differ.
template <typename T, int NF, int W>
__device__ __forceinline__ void site_update(const Coefs<T, NF> &k, const T (&cu)[NF][W], const T (&zm)[NF][W],
                                            const T (&zp)[NF][W], const T (&ym)[NF][W], const T (&yp)[NF][W],
                                            const T (&xl)[NF], const T (&xr)[NF], const T (&pc)[NF][W],
                                            T (&pnew)[NF][W], T (&acc)[2 * NF + 1])
{
    if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            T v[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) v[f] = cu[f][j];
            const T v02 = v[0] * v[0];
            T dvw[NF];  // a^(3+alpha) dV/dphi_f
            if constexpr (NF > 1) {
                // sum_{f>0} phi_f^2, and the potential sum plus sum_{f>0} m2_f phi_f^2/2
                T others = (T)0, vsum = acc[2 * NF];
#pragma unroll
                for (int f = 1; f < NF; ++f) {
                    const T vf2 = v[f] * v[f];
                    others += vf2;
                    vsum = fma_t(k.hm2[f], vf2, vsum);
                    dvw[f] = v[f] * fma_t(k.wq, v02, k.wm2[f]);
                }
                dvw[0] = v[0] * fma_t(k.wq, others, fma_t(k.wlam, v02, k.wm2[0]));
                acc[2 * NF] = fma_t(k.hq * v02, others, fma_t(v02, fma_t(k.qlam, v02, k.hm2[0]), vsum));
            } else {
                dvw[0] = v[0] * fma_t(k.wlam, v02, k.wm2[0]);
                acc[2 * NF] = fma_t(v02, fma_t(k.qlam, v02, k.hm2[0]), acc[2 * NF]);
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const T cc = v[f];
                const T left = (j == 0) ? xl[f] : cu[f][j - 1];
                const T right = (j == W - 1) ? xr[f] : cu[f][j + 1];
                const T lap = fma_t((T)-6, cc, ((left + right) + (ym[f][j] + yp[f][j])) + (zm[f][j] + zp[f][j]));
                const T F = fma_t(k.wlx, lap, -dvw[f]);
                const T pint = fma_t(k.hdt, F, pc[f][j]);
                pnew[f][j] = fma_t(k.kdt, F, pc[f][j]);
                acc[f] = fma_t(pint, pint, acc[f]);
                acc[NF + f] = fma_t(-cc, lap, acc[NF + f]);
            }
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < W; ++j) {
        T v[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) v[f] = cu[f][j];
        const T v02 = v[0] * v[0];
        T dv[NF];
        dv[0] = k.m2[0] * v[0] + k.lam * v02 * v[0];
        T Vs = (T)0.5 * k.m2[0] * v02 + (T)0.25 * k.lam * v02 * v02;
        if constexpr (NF > 1) {  // the coupling terms (with one field they are zero: skip them)
            T others = (T)0;
#pragma unroll
            for (int f = 1; f < NF; ++f) others += v[f] * v[f];
            dv[0] += k.q * v[0] * others;
            Vs += (T)0.5 * k.q * v02 * others;
#pragma unroll
            for (int f = 1; f < NF; ++f) {
                dv[f] = k.m2[f] * v[f] + k.q * v02 * v[f];
                Vs += (T)0.5 * k.m2[f] * v[f] * v[f];
            }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const T cc = v[f];
            const T left = (j == 0) ? xl[f] : cu[f][j - 1];
            const T right = (j == W - 1) ? xr[f] : cu[f][j + 1];
            const T dxp = right - cc, dyp = yp[f][j] - cc, dzp = zp[f][j] - cc;
            // FP32: differences first, so the small gradients stay exact
            const T dxm = left - cc, dym = ym[f][j] - cc, dzm = zm[f][j] - cc;
            const T lap = ((dxm + dxp) + (dym + dyp)) + (dzm + dzp);
            const T F = k.wlx * lap - k.wv * dv[f];
            const T pint = fma_t(k.hdt, F, pc[f][j]);
            pnew[f][j] = fma_t(k.kdt, F, pc[f][j]);
            acc[f] += pint * pint;
            acc[NF + f] += dxp * dxp + dyp * dyp + dzp * dzp;
        }
        acc[2 * NF] += Vs;
    }
}

// CTA sum in a fixed order (warp trees, then warps in index order) into this
// CTA's slot; the last CTA to arrive sums all slots in index order and runs
// finalize().  Deterministic for a given launch geometry.
// F32TREE (FP32 lattices): the warp tree runs in FP32 and each warp adds its
// sum to the CTA's FP64 total -- thread sums (FP32 in-thread, promoted to FP64
// every 16 planes), FP32 warp tree, FP64 from there on; FP64 lattices keep the
// whole tree in FP64.
template <int NQ, bool F32TREE = false>
__device__ __forceinline__ void cta_reduce_finalize(const double (&accd)[NQ], const Model &m, const PassCoef &c,
                                                    Scalars *sc, double *slots, unsigned bid, unsigned nblocks)
{
    __shared__ double red[32][NQ];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        double v;
        if constexpr (F32TREE) {
            float w = (float)accd[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
            v = (double)w;
        } else {
            v = warp_sum(accd[i]);
        }
        if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    if (tid < NQ) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += red[w][tid];
        slots[(size_t)bid * NQ + tid] = s;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(&sc->ticket, 1u) == nblocks - 1);
    __syncthreads();
    if (last) {
        __threadfence();
        double part[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) part[i] = 0.0;
        for (unsigned b = tid; b < nblocks; b += blockDim.x)
#pragma unroll
            for (int i = 0; i < NQ; ++i) part[i] += __ldcg(slots + (size_t)b * NQ + i);
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            double v = warp_sum(part[i]);
            if (lane == 0) red[warp][i] = v;
        }
        __syncthreads();
        if (tid == 0) {
            double tot[kMaxQ];
            for (int i = 0; i < NQ; ++i) {
                double s = 0.0;
                for (int w = 0; w < nwarps; ++w) s += red[w][i];
                tot[i] = s;
            }
            finalize(m, c, sc, tot);
            sc->ticket = 0u;
            __threadfence();
        }
    }
    __syncthreads();  // red[] and last may be reused by the next tile of a persistent CTA
}

__device__ __forceinline__ unsigned grid_bid() { return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z); }
__device__ __forceinline__ unsigned grid_nblocks() { return gridDim.x * gridDim.y * gridDim.z; }

// Ghost rows of this thread's W output sites: a site in the first or last row
// also goes to the ghost row below or above the plane (the x-edges need no
// copies: the TMA pass reads the periodic image there).
template <typename T, int NF, int W>
__device__ __forceinline__ void store_ghosts(T *const (&pho)[NF], T *const (&pio)[NF], const T (&ph)[NF][W],
                                             const T (&pp)[NF][W], size_t pz, int x0, int y, int N, long long P)
{
    long long dy = 0;
    if (y == 0) dy = (long long)N * P;  // ghost row after the last row
    else if (y == N - 1) dy = -(long long)N * P;
    if (dy == 0) return;
    const size_t base = pz + (size_t)y * P + x0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        store_vec_cs(pho[f] + base + dy, ph[f]);
        store_vec_cs(pio[f] + base + dy, pp[f]);
    }
}

// ---- variant 1: register streaming with a per-thread prefetch ring -------------
// Each thread owns its 128-bit words.  The HBM stream (the stored phi and pi
// of its own sites, plane after plane) is prefetched D planes ahead with
// cp.async into a private shared-memory ring (no CTA barrier: a thread only
// waits for its own copies); the neighbour rows and edge sites of plane z are
// other threads' words of the same plane and come from L1/L2 with ld.global.
// D = 0 loads the next plane directly, without the ring.

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int Npending>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(Npending) : "memory"); }

// One CTA tile (bx, by, bz) of the register-streaming pass; bid/nblocks
// index the tile among the lattice's tiles for the reduction.
template <typename T, int NF, bool MEASURE, int D>
__device__ __forceinline__ void ldg_tile(const Model &m, const FieldPtrs &fp, const PassCoef &c, int txt, int ty,
                                         int zc, int bx, int by, int bz, unsigned bid, unsigned nblocks, Scalars *sc,
                                         double *slots, unsigned char *ring_raw)
{
    constexpr int W = Vec<T>::W;
    constexpr int NQ = 2 * NF + 1;
    const int N = m.N;
    const int tid = threadIdx.x;
    const int tx = tid % txt, tyi = tid / txt;
    const int x0 = (bx * txt + tx) * W;
    const int y = by * ty + tyi;
    const int z0 = bz * zc;
    const int z1 = min(z0 + zc, N);
    const bool active = (tyi < ty) && (x0 < N) && (y < N);
    // ring slot (plane d, field f, array a) of this thread
    auto slot = [&](int d, int f, int a) -> T * {
        return reinterpret_cast<T *>(ring_raw) + ((size_t)((d * NF + f) * 2 + a) * blockDim.x + tid) * W;
    };

    double accd[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) accd[i] = 0.0;

    if (active) {
        const Coefs<T, NF> k = make_coefs<T, NF>(m, c, sc);
        const T *phs[NF], *pis[NF];
        T *pho[NF], *pio[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            phs[f] = static_cast<const T *>(fp.phi_in[f]);
            pis[f] = static_cast<const T *>(fp.pi_in[f]);
            pho[f] = static_cast<T *>(fp.phi_out[f]);
            pio[f] = static_cast<T *>(fp.pi_out[f]);
        }
        const size_t NN = (size_t)m.pplane;
        const size_t P = (size_t)m.pitch;
        const int xl = (x0 == 0) ? N - 1 : x0 - 1;
        const int xr = (x0 + W == N) ? 0 : x0 + W;
        const size_t row = (size_t)y * P;
        const size_t rowm = (size_t)((y == 0) ? N - 1 : y - 1) * P;
        const size_t rowp = (size_t)((y + 1 == N) ? 0 : y + 1) * P;
        auto cur_vec = [&](int f, size_t off, T (&o)[W]) {
            T a[W], b[W];
            load_vec(phs[f] + off, a);
            load_vec(pis[f] + off, b);
#pragma unroll
            for (int j = 0; j < W; ++j) o[j] = fma_t(k.drift, b[j], a[j]);
        };
        auto cur_one = [&](int f, size_t off) -> T {
            return fma_t(k.drift, __ldg(pis[f] + off), __ldg(phs[f] + off));
        };
        auto plane_off = [&](int zz) -> size_t { return (size_t)(zz >= N ? zz - N : zz) * NN + row + x0; };
        // prefetch this thread's words of plane zz (<= z1) into ring slot d
        auto prefetch = [&](int zz, int d) {
            if (zz <= z1) {
                const size_t off = plane_off(zz);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    cp_async16(slot(d, f, 0), phs[f] + off);
                    cp_async16(slot(d, f, 1), pis[f] + off);
                }
            }
            cp_async_commit();
        };

        T zm[NF][W], cu[NF][W], zp[NF][W], pc[NF][W];
        {
            const size_t pm = (size_t)((z0 == 0) ? N - 1 : z0 - 1) * NN;
            const size_t p0 = (size_t)z0 * NN;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                cur_vec(f, pm + row + x0, zm[f]);
                T a[W];
                load_vec(phs[f] + p0 + row + x0, a);
                load_vec(pis[f] + p0 + row + x0, pc[f]);
#pragma unroll
                for (int j = 0; j < W; ++j) cu[f][j] = fma_t(k.drift, pc[f][j], a[j]);
            }
        }
        if (D > 0) {
#pragma unroll
            for (int d = 0; d < D; ++d) prefetch(z0 + 1 + d, d);
        }
        T acc[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) acc[i] = (T)0;

        int d = 0;  // ring slot holding plane z+1
        for (int z = z0; z < z1; ++z) {
            const size_t pz = (size_t)z * NN;
            T pnext[NF][W];
            if (D > 0) {
                cp_async_wait<(D > 0 ? D - 1 : 0)>();
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    T a[W];
                    load_vec_s(slot(d, f, 0), a);
                    load_vec_s(slot(d, f, 1), pnext[f]);
#pragma unroll
                    for (int j = 0; j < W; ++j) zp[f][j] = fma_t(k.drift, pnext[f][j], a[j]);
                }
                prefetch(z + 1 + D, d);
                d = (d + 1 == D) ? 0 : d + 1;
            } else {
                const size_t pn = plane_off(z + 1);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    T a[W];
                    load_vec(phs[f] + pn, a);
                    load_vec(pis[f] + pn, pnext[f]);
#pragma unroll
                    for (int j = 0; j < W; ++j) zp[f][j] = fma_t(k.drift, pnext[f][j], a[j]);
                }
            }
            T ym[NF][W], yp[NF][W], xlv[NF], xrv[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                cur_vec(f, pz + rowm + x0, ym[f]);
                cur_vec(f, pz + rowp + x0, yp[f]);
                xlv[f] = cur_one(f, pz + row + xl);
                xrv[f] = cur_one(f, pz + row + xr);
            }
            T pnew[NF][W];
            site_update<T, NF, W>(k, cu, zm, zp, ym, yp, xlv, xrv, pc, pnew, acc);
            if (!MEASURE) {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    store_vec_cs(pho[f] + pz + row + x0, cu[f]);
                    store_vec_cs(pio[f] + pz + row + x0, pnew[f]);
                }
                if (m.ghosts) store_ghosts<T, NF, W>(pho, pio, cu, pnew, pz, x0, y, N, (long long)P);
            }
            if (((z - z0) & 15) == 15) {
#pragma unroll
                for (int i = 0; i < NQ; ++i) {
                    accd[i] += (double)acc[i];
                    acc[i] = (T)0;
                }
            }
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    zm[f][j] = cu[f][j];
                    cu[f][j] = zp[f][j];
                    pc[f][j] = pnext[f][j];
                }
        }
        if (D > 0) cp_async_wait<0>();
#pragma unroll
        for (int i = 0; i < NQ; ++i) accd[i] += (double)acc[i];
    }
    cta_reduce_finalize<NQ, sizeof(T) == 4>(accd, m, c, sc, slots, bid, nblocks);
}

template <typename T, int NF, bool MEASURE, int D, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) fused_pass_ldg(Model m, FieldPtrs fp, PassCoef c, int txt, int ty, int zc,
                                                            Scalars *sc, double *slots)
{
    extern __shared__ __align__(16) unsigned char ring_raw[];
    ldg_tile<T, NF, MEASURE, D>(m, fp, c, txt, ty, zc, blockIdx.x, blockIdx.y, blockIdx.z, grid_bid(), grid_nblocks(),
                                sc, slots, ring_raw);
}

// ---- batched form: many lattices in one persistent launch ------------------------
// Each job is one lattice with its own model, fields, scalars, reduction slots
// and launch geometry (the geometry it would use alone, so its sums and thus
// its results are bitwise the same alone and in a batch).  The CTAs of the
// launch walk the flattened list of (job, tile) items.

// The job table (first item of each job) is staged in shared memory once per
// CTA when it fits (kGroupStagedJobs entries), so locating an item's job is a
// binary search in shared memory rather than a chain of dependent global loads.
// D > 0: each thread prefetches its words D planes ahead with cp.async into a
// per-thread ring placed after the staged table (group_smem_bytes).
constexpr int kGroupStagedJobs = 8192;

__host__ __device__ constexpr size_t group_table_bytes(int njobs)
{
    return njobs <= kGroupStagedJobs ? ((size_t)njobs * sizeof(unsigned) + 15) / 16 * 16 : 0;
}
__host__ __device__ constexpr size_t group_smem_bytes(int njobs, int nf, int D)
{
    return group_table_bytes(njobs) + (size_t)D * nf * 2 * 256 * 16;
}

template <typename T, int NF, int D>
__global__ void __launch_bounds__(256, 2) fused_pass_group(const BatchJob *__restrict__ jobs,
                                                           const unsigned *__restrict__ first_item, int njobs,
                                                           unsigned total, PassCoef c)
{
    extern __shared__ __align__(16) unsigned char g_smem[];
    unsigned *s_first = reinterpret_cast<unsigned *>(g_smem);
    unsigned char *ring = g_smem + group_table_bytes(njobs);
    const bool staged = njobs <= kGroupStagedJobs;
    if (staged) {
        for (int i = threadIdx.x; i < njobs; i += blockDim.x) s_first[i] = __ldg(first_item + i);
        __syncthreads();
    }
    const unsigned *first = staged ? s_first : first_item;
    for (unsigned item = blockIdx.x; item < total; item += gridDim.x) {
        int lo = 0, hi = njobs - 1;  // last job whose first item <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const BatchJob &j = jobs[lo];
        const unsigned local = item - first[lo];
        const int bx = (int)(local % (unsigned)j.gx);
        const int by = (int)((local / (unsigned)j.gx) % (unsigned)j.gy);
        const int bz = (int)(local / ((unsigned)j.gx * (unsigned)j.gy));
        ldg_tile<T, NF, false, D>(j.m, j.fp, c, j.txt, j.ty, j.zc, bx, by, bz, local, j.nblocks, j.sc, j.slots, ring);
    }
}

// Enqueue one grouped pass (see launch_group).
template <typename T, int NF>
static cudaError_t launch_group_t(int prefetch, const BatchJob *jobs, const unsigned *first_item, int njobs,
                                  unsigned total, const PassCoef &c, int grid, cudaStream_t s)
{
    const int D = prefetch > 0 ? 3 : 0;
    const size_t smem = group_smem_bytes(njobs, NF, D);
    auto kern = D ? fused_pass_group<T, NF, 3> : fused_pass_group<T, NF, 0>;
    if (smem > 48 * 1024) {
        // the opt-in limit for this kernel (per device, set once; an equal or smaller request needs nothing)
        static std::atomic<size_t> configured[64][2];
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        std::atomic<size_t> &done = configured[dev][D ? 1 : 0];
        if (smem > done.load(std::memory_order_acquire)) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            size_t cur = done.load(std::memory_order_relaxed);
            while (smem > cur && !done.compare_exchange_weak(cur, smem, std::memory_order_release)) {
            }
        }
    }
    kern<<<grid, 256, smem, s>>>(jobs, first_item, njobs, total, c);
    return cudaGetLastError();
}

// ---- PTX helpers for asynchronous copies ---------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for a plane with a time limit (about one second); on expiry record
// TL_ETIMEOUT in the lattice status and return false.
constexpr uint64_t kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, Scalars *sc)
{
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 256; ++i)
            if (mbar_test(bar, parity)) return true;
        if (global_ns() - t0 > kWaitLimitNs) {
            atomicCAS(&sc->status, TL_OK, TL_ETIMEOUT);
            return false;
        }
    }
}


// ---- variant 2: tiled TMA staging on the ghost-padded layout ---------------------
// Warps 0..CW-1 compute, warp CW produces.  A CTA owns a tile of txt W x ty
// sites and a chunk of z-planes.  For every plane its producer lane issues, per
// array, 3-D tensor copies (cp.async.bulk.tensor) of ty + 2 rows (the tile's
// rows and the rows above and below it; the ghost rows make this in-bounds at
// the y-edges) into a ring of S stages, completing on the stage's "full"
// mbarrier: a tile inside the lattice takes one box txt W + 2W sites wide (the
// tile and its x-halo); a tile at an x-edge takes its body (txt W wide) and
// the two W-wide columns that hold its left and right halo sites, the one on
// the far side of the edge from the periodic image (x = N - W or 0), so no
// copy reads past the lattice's rows.  Consumers release a stage on its
// "empty" mbarrier once they are done with it; they read the centre of plane
// z+1 and the halo of plane z from shared memory and run the same per-site
// update as the register-streaming variant.

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

constexpr int kMaxStages = 8;

// The fixed-order sum of cta_reduce_finalize for the compute warps of a TMA
// CTA alone (threads 0 .. nthr-1, named barrier 1), so that the producer warp
// can go on loading the next tile's planes meanwhile.  The same numbers as the
// whole-CTA form: the producer warp's share was zero.  The last tile to arrive
// sums all slots with a fixed stride of 128 threads.
template <int NQ, bool F32TREE>
__device__ __forceinline__ void consumer_reduce_finalize(const double (&accd)[NQ], const Model &m, const PassCoef &c,
                                                         Scalars *sc, double *slots, unsigned bid, unsigned nblocks,
                                                         unsigned nthr)
{
    __shared__ double red[32][NQ];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (int)(nthr >> 5);
    auto sync = [&] { asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory"); };
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        double v;
        if constexpr (F32TREE) {
            float w = (float)accd[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
            v = (double)w;
        } else {
            v = warp_sum(accd[i]);
        }
        if (lane == 0) red[warp][i] = v;
    }
    sync();
    if (tid < NQ) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += red[w][tid];
        slots[(size_t)bid * NQ + tid] = s;
    }
    __threadfence();
    sync();
    if (tid == 0) last = (atomicAdd(&sc->ticket, 1u) == nblocks - 1);
    sync();
    if (last) {
        __threadfence();
        double part[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) part[i] = 0.0;
        if (tid < 128)
            for (unsigned b = tid; b < nblocks; b += 128)
#pragma unroll
                for (int i = 0; i < NQ; ++i) part[i] += __ldcg(slots + (size_t)b * NQ + i);
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            double v = warp_sum(part[i]);
            if (lane == 0 && warp < 4) red[warp][i] = v;
        }
        sync();
        if (tid == 0) {
            double tot[kMaxQ];
            for (int i = 0; i < NQ; ++i) tot[i] = ((red[0][i] + red[1][i]) + red[2][i]) + red[3][i];
            finalize(m, c, sc, tot);
            sc->ticket = 0u;
            __threadfence();
        }
    }
    sync();  // red[] and last are reused by the next tile
}

// One CTA tile (bx, by, bz) of the TMA pass; bid/nblocks index the tile among
// the lattice's tiles for the reduction; maps points to the tensor maps of the
// lattice's input arrays (a kernel parameter or a copy in global memory).
// GLOBAL_MAPS: the maps live in global memory, written by the host; the
// producer makes them visible to the tensor-map proxy before their first use.
template <typename T, int NF, bool MEASURE, bool GLOBAL_MAPS = false>
__device__ __forceinline__ void tma_tile(const Model &m, const FieldPtrs &fp, const PassCoef &c, int txt, int ty,
                                         int zc, int S, int lpad, const TmaMaps *maps, Scalars *sc, double *slots,
                                         int bx, int by, int bz, unsigned bid, unsigned nblocks)
{
    constexpr int W = Vec<T>::W;
    constexpr int NQ = 2 * NF + 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
    __shared__ volatile int s_failed;
    __shared__ int s_warps;

    const int N = m.N;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int CW = (blockDim.x >> 5) - 1;
    const bool producer = (tid >> 5) == CW;
    const int x_tile = bx * txt * W, y_tile = by * ty;
    const int tx = tid % txt, tyi = tid / txt;
    const int x0 = x_tile + tx * W;
    const int y = y_tile + tyi;
    const bool active = !producer && (tyi < ty) && (x0 < N) && (y < N);
    // Compute warps without an active lane (rows past the lattice edge in the
    // last tile row) stay out of the ring: the "empty" barriers count only the
    // others, so no warp can release a stage ahead of the ones still reading it.
    const bool warp_active = __any_sync(0xffffffffu, active);
    if (tid == 0) s_warps = 0;
    __syncthreads();
    if (lane == 0 && warp_active) atomicAdd(&s_warps, 1);
    __syncthreads();
    const int z0 = bz * zc;
    const int z1 = min(z0 + zc, N);
    const int K = (z1 - z0) + 2;  // planes z0-1 .. z1
    // tile at an x-edge of the lattice: body box plus two halo columns, else
    // one tile-plus-halo box; either way (ty + 2) (txt + 2) 16-byte words per
    // array and plane
    const bool edge = x_tile == 0 || x_tile + txt * W >= N;
    const int rowe = edge ? txt * W : txt * W + 2 * W;  // row pitch of the staged body
    const uint32_t box_bytes = (uint32_t)((ty + 2) * (txt + 2) * 16);
    const uint32_t region = (uint32_t)tma_slot_bytes(txt, ty);  // one array's slot in a stage
    const int side_l = (int)(tma_side_offset(txt, ty, 0) / sizeof(T));
    const int side_r = (int)(tma_side_offset(txt, ty, 1) / sizeof(T));
    auto arr = [&](int s, int f, int a) -> T * {
        return reinterpret_cast<T *>(smem_raw + (size_t)((s * NF + f) * 2 + a) * region);
    };

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], s_warps);
        }
        s_failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    double accd[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) accd[i] = 0.0;
    int issued = 0;

    if (producer) {
        if ((tid & 31) == 0) {
            if constexpr (GLOBAL_MAPS) {
#pragma unroll
                for (int kk = 0; kk < 3; ++kk)
#pragma unroll
                    for (int i = 0; i < 2 * NF; ++i)
                        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&maps->map[kk][i])
                                     : "memory");
            }
            // source columns of the halo columns of an edge tile (16-byte aligned:
            // W divides N and the tile offsets)
            const int xl_src = x_tile == 0 ? N - W : x_tile - W;
            const int xr_src = x_tile + txt * W >= N ? 0 : x_tile + txt * W;
            int ps = 0;
            unsigned pph = 0;
            for (int k = 0; k < K; ++k) {
                const int s = ps;
                if (k >= S && !mbar_wait_bounded(&empty[s], pph ^ 1u, sc)) {
                    s_failed = 1;
                    break;
                }
                if (s_failed) break;
                int zg = z0 - 1 + k;
                if (zg < 0) zg += N;
                else if (zg >= N) zg -= N;
                if (++ps == S) {
                    ps = 0;
                    pph ^= 1u;
                }
                mbar_arrive_expect_tx(&full[s], (uint32_t)(NF * 2) * box_bytes);
#pragma unroll
                for (int f = 0; f < NF; ++f)
#pragma unroll
                    for (int a = 0; a < 2; ++a) {
                        T *dst = arr(s, f, a);
                        if (!edge) {
                            tma_load_3d(dst, &maps->map[kMapTile][2 * f + a], lpad + x_tile - W, y_tile, zg, &full[s]);
                        } else {
                            tma_load_3d(dst, &maps->map[kMapBody][2 * f + a], lpad + x_tile, y_tile, zg, &full[s]);
                            tma_load_3d(dst + side_l, &maps->map[kMapSide][2 * f + a], lpad + xl_src, y_tile, zg,
                                        &full[s]);
                            tma_load_3d(dst + side_r, &maps->map[kMapSide][2 * f + a], lpad + xr_src, y_tile, zg,
                                        &full[s]);
                        }
                    }
                issued = k + 1;
            }
        }
    } else if (warp_active) {
        // x-neighbours: the left site is the last one of the thread to the left
        // in the same row and warp, the right site the first one of the thread
        // to the right (warp shuffles, no shared-memory bank conflicts);
        // threads at a row end or a warp edge read theirs from the stage.
        const unsigned amask = __ballot_sync(0xffffffffu, active);
        const bool own_l = tx == 0 || lane == 0;
        const bool own_r = tx == txt - 1 || x0 + W >= N || lane == 31;
        // at an x-edge tile the sites beyond the tile come from the halo columns
        const bool col_l = edge && tx == 0;
        const bool col_r = edge && (tx == txt - 1 || x0 + W >= N);
        const int col = (tyi + 1) * W;  // this thread's row in a halo column
        const int src_l = own_l ? lane : lane - 1, src_r = own_r ? lane : lane + 1;
        const Coefs<T, NF> k = make_coefs<T, NF>(m, c, sc);
        const int ctr = (tyi + 1) * rowe + (edge ? 0 : W) + tx * W;
        const size_t P = (size_t)m.pitch, PP = (size_t)m.pplane;
        T *pho[NF], *pio[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            pho[f] = static_cast<T *>(fp.phi_out[f]);
            pio[f] = static_cast<T *>(fp.pi_out[f]);
        }
        T zm[NF][W], cu[NF][W], zp[NF][W], pc[NF][W], pn[NF][W];
        T acc[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) acc[i] = (T)0;
        auto centre = [&](int s, T (&ph)[NF][W], T (&pp)[NF][W]) {
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                T a[W];
                load_vec_s(arr(s, f, 0) + ctr, a);
                load_vec_s(arr(s, f, 1) + ctr, pp[f]);
#pragma unroll
                for (int j = 0; j < W; ++j) ph[f][j] = fma_t(k.drift, pp[f][j], a[j]);
            }
        };
        int ws = 0, rs = 0;
        unsigned wph = 0;
        auto adv_w = [&] {
            if (++ws == S) {
                ws = 0;
                wph ^= 1u;
            }
        };
        auto release = [&](int) {
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&empty[rs])) : "memory");
            if (++rs == S) rs = 0;
        };
        bool ok = true;
        if (active) {
            ok = mbar_wait_bounded(&full[ws], wph, sc);
            centre(ws, zm, pn);
        }
        adv_w();
        if (active) {
            ok = ok && mbar_wait_bounded(&full[ws], wph, sc);
            centre(ws, cu, pc);
        }
        adv_w();
        if (!ok) s_failed = 1;
        release(0);
        // blocks of 16 planes: after each, the FP32 energy sums go into FP64
        bool stop = false;
        for (int zb = z0; zb < z1 && !stop; zb += 16) {
        const int ze = min(zb + 16, z1);
        for (int z = zb; z < ze; ++z) {
            if (__any_sync(0xffffffffu, s_failed != 0)) {  // warp-uniform exit
                stop = true;
                break;
            }
            const int kz = z - z0 + 1;
            if (active) {
                if (!mbar_wait_bounded(&full[ws], wph, sc)) s_failed = 1;
                centre(ws, zp, pn);
                const int s0 = rs;
                T ym[NF][W], yp[NF][W], xlv[NF], xrv[NF];
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const T *ph = arr(s0, f, 0), *pp = arr(s0, f, 1);
                    T a[W], b[W];
                    load_vec_s(ph + ctr - rowe, a);
                    load_vec_s(pp + ctr - rowe, b);
#pragma unroll
                    for (int j = 0; j < W; ++j) ym[f][j] = fma_t(k.drift, b[j], a[j]);
                    load_vec_s(ph + ctr + rowe, a);
                    load_vec_s(pp + ctr + rowe, b);
#pragma unroll
                    for (int j = 0; j < W; ++j) yp[f][j] = fma_t(k.drift, b[j], a[j]);
                    const T l = __shfl_sync(amask, cu[f][W - 1], src_l);
                    const T r = __shfl_sync(amask, cu[f][0], src_r);
                    const int il = col_l ? side_l + col + W - 1 : ctr - 1;
                    const int ir = col_r ? side_r + col : ctr + W;
                    xlv[f] = own_l ? fma_t(k.drift, pp[il], ph[il]) : l;
                    xrv[f] = own_r ? fma_t(k.drift, pp[ir], ph[ir]) : r;
                }
                T pnew[NF][W];
                site_update<T, NF, W>(k, cu, zm, zp, ym, yp, xlv, xrv, pc, pnew, acc);
                if (!MEASURE) {
                    const size_t pz = (size_t)z * PP;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        store_vec_cs(pho[f] + pz + (size_t)y * P + x0, cu[f]);
                        store_vec_cs(pio[f] + pz + (size_t)y * P + x0, pnew[f]);
                    }
                    if (m.ghosts) store_ghosts<T, NF, W>(pho, pio, cu, pnew, pz, x0, y, N, (long long)P);
                }
#pragma unroll
                for (int f = 0; f < NF; ++f)
#pragma unroll
                    for (int j = 0; j < W; ++j) {
                        zm[f][j] = cu[f][j];
                        cu[f][j] = zp[f][j];
                        pc[f][j] = pn[f][j];
                    }
            }
            adv_w();
            release(kz);
        }
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            accd[i] += (double)acc[i];
            acc[i] = (T)0;
        }
        }
#pragma unroll
        for (int i = 0; i < NQ; ++i) accd[i] += (double)acc[i];
    }
    if (producer) {
        // After a timeout, wait (bounded) for the copies still in flight before the
        // CTA's shared memory goes away.
        if (s_failed && (tid & 31) == 0)
            for (int kk = (issued > S ? issued - S : 0); kk < issued; ++kk)
                mbar_wait_bounded(&full[kk % S], (kk / S) & 1u, sc);
        return;
    }
    consumer_reduce_finalize<NQ, sizeof(T) == 4>(accd, m, c, sc, slots, bid, nblocks, (unsigned)CW * 32u);
}

// Tiles first, first + stride, ... (< nitems) of the TMA pass, in a CTA whose
// stage ring carries on from tile to tile: the producer warp streams the
// planes of all its tiles through the ring (a global plane count gives each
// plane its stage and barrier phase), so it loads the next tile's first
// planes while the compute warps finish a tile and sum its energies.  Tile
// `item` is (bx, by, bz) = (item % gx, item / gx % gy, item / (gx gy)) and owns
// reduction slot `item` of nitems.  maps points to the tensor maps of the
// lattice's input arrays (a kernel parameter or a copy in global memory);
// GLOBAL_MAPS: the maps live in global memory, written by the host, and the
// producer makes them visible to the tensor-map proxy before their first use.
// Every compute warp takes part in every tile's ring traffic (a warp without
// sites only waits and releases), so the "empty" barriers count all of them.
template <typename T, int NF, bool MEASURE, bool GLOBAL_MAPS = false>
__device__ __forceinline__ void tma_items(const Model &m, const FieldPtrs &fp, const PassCoef &c, int txt, int ty,
                                          int zc, int S, int lpad, const TmaMaps *maps, Scalars *sc, double *slots,
                                          unsigned first, unsigned stride, unsigned nitems, int gx, int gy)
{
    constexpr int W = Vec<T>::W;
    constexpr int NQ = 2 * NF + 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
    __shared__ volatile int s_failed;
    __shared__ int s_stop;

    const int N = m.N;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int CW = (blockDim.x >> 5) - 1;
    const bool producer = (tid >> 5) == CW;
    const int tx = tid % txt, tyi = tid / txt;
    // (ty + 2) (txt + 2) 16-byte words per array and plane for every tile (a
    // tile-plus-halo box, or at an x-edge the body box and two halo columns)
    const uint32_t box_bytes = (uint32_t)((ty + 2) * (txt + 2) * 16);
    const uint32_t region = (uint32_t)tma_slot_bytes(txt, ty);  // one array's slot in a stage
    const int side_l = (int)(tma_side_offset(txt, ty, 0) / sizeof(T));
    const int side_r = (int)(tma_side_offset(txt, ty, 1) / sizeof(T));
    auto arr = [&](int s, int f, int a) -> T * {
        return reinterpret_cast<T *>(smem_raw + (size_t)((s * NF + f) * 2 + a) * region);
    };

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CW);
        }
        s_failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (producer) {
        if (lane == 0) {
            if constexpr (GLOBAL_MAPS) {
#pragma unroll
                for (int kk = 0; kk < 3; ++kk)
#pragma unroll
                    for (int i = 0; i < 2 * NF; ++i)
                        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&maps->map[kk][i])
                                     : "memory");
            }
            // plane count g and its ring stage ps and phase pph, advanced
            // incrementally (no division in the loop)
            unsigned g = 0, issued = 0, pph = 0;
            int ps = 0;
            bool stop = false;
            for (unsigned item = first; item < nitems && !stop; item += stride) {
                const int bx = (int)(item % (unsigned)gx), by = (int)((item / (unsigned)gx) % (unsigned)gy);
                const int bz = (int)(item / ((unsigned)gx * (unsigned)gy));
                const int x_tile = bx * txt * W, y_tile = by * ty;
                const int z0 = bz * zc, z1 = min(z0 + zc, N), K = z1 - z0 + 2;
                const bool edge = x_tile == 0 || x_tile + txt * W >= N;
                // source columns of the halo columns of an edge tile (16-byte
                // aligned: W divides N and the tile offsets)
                const int xl_src = x_tile == 0 ? N - W : x_tile - W;
                const int xr_src = x_tile + txt * W >= N ? 0 : x_tile + txt * W;
                for (int k = 0; k < K; ++k) {
                    const int s = ps;
                    // the stage's previous plane (g - S) completed phase pph ^ 1
                    if (g >= (unsigned)S && !mbar_wait_bounded(&empty[s], pph ^ 1u, sc)) {
                        s_failed = 1;
                        stop = true;
                        break;
                    }
                    if (s_failed) {
                        stop = true;
                        break;
                    }
                    int zg = z0 - 1 + k;
                    if (zg < 0) zg += N;
                    else if (zg >= N) zg -= N;
                    mbar_arrive_expect_tx(&full[s], (uint32_t)(NF * 2) * box_bytes);
#pragma unroll
                    for (int f = 0; f < NF; ++f)
#pragma unroll
                        for (int a = 0; a < 2; ++a) {
                            T *dst = arr(s, f, a);
                            if (!edge) {
                                tma_load_3d(dst, &maps->map[kMapTile][2 * f + a], lpad + x_tile - W, y_tile, zg,
                                            &full[s]);
                            } else {
                                tma_load_3d(dst, &maps->map[kMapBody][2 * f + a], lpad + x_tile, y_tile, zg, &full[s]);
                                tma_load_3d(dst + side_l, &maps->map[kMapSide][2 * f + a], lpad + xl_src, y_tile, zg,
                                            &full[s]);
                                tma_load_3d(dst + side_r, &maps->map[kMapSide][2 * f + a], lpad + xr_src, y_tile, zg,
                                            &full[s]);
                            }
                        }
                    issued = g + 1;
                    ++g;
                    if (++ps == S) {
                        ps = 0;
                        pph ^= 1u;
                    }
                }
            }
            // After a timeout, wait (bounded) for the copies still in flight
            // before the CTA's shared memory can go away.
            if (s_failed)
                for (unsigned gg = (issued > (unsigned)S ? issued - S : 0); gg < issued; ++gg)
                    mbar_wait_bounded(&full[gg % S], (gg / S) & 1u, sc);
        }
        return;  // the producer warp takes no part in the tiles' sums
    }

    const unsigned nthr = (unsigned)CW * 32u;
    const size_t P = (size_t)m.pitch, PP = (size_t)m.pplane;
    T *pho[NF], *pio[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        pho[f] = static_cast<T *>(fp.phi_out[f]);
        pio[f] = static_cast<T *>(fp.pi_out[f]);
    }
    // Two ring pointers, carried from tile to tile: the next plane to wait for
    // (stage ws, phase wph) and the next plane to release (stage rs).
    int ws = 0, rs = 0;
    unsigned wph = 0;
    auto wait_next = [&]() -> bool { return mbar_wait_bounded(&full[ws], wph, sc); };
    auto advance_wait = [&] {
        if (++ws == S) {
            ws = 0;
            wph ^= 1u;
        }
    };
    auto release_next = [&] {
        __syncwarp();
        if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&empty[rs])) : "memory");
        if (++rs == S) rs = 0;
    };

    for (unsigned item = first; item < nitems; item += stride) {
        const int bx = (int)(item % (unsigned)gx), by = (int)((item / (unsigned)gx) % (unsigned)gy);
        const int bz = (int)(item / ((unsigned)gx * (unsigned)gy));
        const int x_tile = bx * txt * W, y_tile = by * ty;
        const int z0 = bz * zc, z1 = min(z0 + zc, N), K = z1 - z0 + 2;
        const bool edge = x_tile == 0 || x_tile + txt * W >= N;
        const int rowe = edge ? txt * W : txt * W + 2 * W;  // row pitch of the staged body
        const int x0 = x_tile + tx * W;
        const int y = y_tile + tyi;
        const bool active = (tyi < ty) && (x0 < N) && (y < N);
        const bool warp_active = __any_sync(0xffffffffu, active);
        double accd[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) accd[i] = 0.0;
        if (warp_active) {
            // x-neighbours: the left site is the last one of the thread to the
            // left in the same row and warp, the right site the first one of the
            // thread to the right (warp shuffles, no shared-memory bank
            // conflicts); threads at a row end or a warp edge read theirs from
            // the stage, at a lattice x-edge from the halo columns.
            const unsigned amask = __ballot_sync(0xffffffffu, active);
            const bool own_l = tx == 0 || lane == 0;
            const bool own_r = tx == txt - 1 || x0 + W >= N || lane == 31;
            const bool col_l = edge && tx == 0;
            const bool col_r = edge && (tx == txt - 1 || x0 + W >= N);
            const int col = (tyi + 1) * W;  // this thread's row in a halo column
            const int src_l = own_l ? lane : lane - 1, src_r = own_r ? lane : lane + 1;
            const Coefs<T, NF> k = make_coefs<T, NF>(m, c, sc);
            const int ctr = (tyi + 1) * rowe + (edge ? 0 : W) + tx * W;
            T zm[NF][W], cu[NF][W], zp[NF][W], pc[NF][W], pn[NF][W];
            T acc[NQ];
#pragma unroll
            for (int i = 0; i < NQ; ++i) acc[i] = (T)0;
            auto centre = [&](int s, T (&ph)[NF][W], T (&pp)[NF][W]) {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    T a[W];
                    load_vec_s(arr(s, f, 0) + ctr, a);
                    load_vec_s(arr(s, f, 1) + ctr, pp[f]);
#pragma unroll
                    for (int j = 0; j < W; ++j) ph[f][j] = fma_t(k.drift, pp[f][j], a[j]);
                }
            };
            bool ok = true;
            if (active) {
                ok = wait_next();
                centre(ws, zm, pn);
            }
            advance_wait();
            if (active) {
                ok = ok && wait_next();
                centre(ws, cu, pc);
            }
            advance_wait();
            if (!ok) s_failed = 1;
            release_next();  // plane 0 (z0 - 1)
            int kz_done = 0;  // planes 0 .. kz_done of the tile released
            for (int z = z0; z < z1; ++z) {
                if (__any_sync(0xffffffffu, s_failed != 0)) break;  // warp-uniform exit
                const int kz = z - z0 + 1;
                if (active) {
                    if (!wait_next()) s_failed = 1;
                    centre(ws, zp, pn);
                    const int s0 = rs;  // plane kz, the next to release
                    T ym[NF][W], yp[NF][W], xlv[NF], xrv[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const T *ph = arr(s0, f, 0), *pp = arr(s0, f, 1);
                        T a[W], b[W];
                        load_vec_s(ph + ctr - rowe, a);
                        load_vec_s(pp + ctr - rowe, b);
#pragma unroll
                        for (int j = 0; j < W; ++j) ym[f][j] = fma_t(k.drift, b[j], a[j]);
                        load_vec_s(ph + ctr + rowe, a);
                        load_vec_s(pp + ctr + rowe, b);
#pragma unroll
                        for (int j = 0; j < W; ++j) yp[f][j] = fma_t(k.drift, b[j], a[j]);
                        const T l = __shfl_sync(amask, cu[f][W - 1], src_l);
                        const T r = __shfl_sync(amask, cu[f][0], src_r);
                        const int il = col_l ? side_l + col + W - 1 : ctr - 1;
                        const int ir = col_r ? side_r + col : ctr + W;
                        xlv[f] = own_l ? fma_t(k.drift, pp[il], ph[il]) : l;
                        xrv[f] = own_r ? fma_t(k.drift, pp[ir], ph[ir]) : r;
                    }
                    T pnew[NF][W];
                    site_update<T, NF, W>(k, cu, zm, zp, ym, yp, xlv, xrv, pc, pnew, acc);
                    if (!MEASURE) {
                        const size_t pz = (size_t)z * PP;
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            store_vec_cs(pho[f] + pz + (size_t)y * P + x0, cu[f]);
                            store_vec_cs(pio[f] + pz + (size_t)y * P + x0, pnew[f]);
                        }
                        if (m.ghosts) store_ghosts<T, NF, W>(pho, pio, cu, pnew, pz, x0, y, N, (long long)P);
                    }
                    if (((z - z0) & 15) == 15) {
#pragma unroll
                        for (int i = 0; i < NQ; ++i) {
                            accd[i] += (double)acc[i];
                            acc[i] = (T)0;
                        }
                    }
#pragma unroll
                    for (int f = 0; f < NF; ++f)
#pragma unroll
                        for (int j = 0; j < W; ++j) {
                            zm[f][j] = cu[f][j];
                            cu[f][j] = zp[f][j];
                            pc[f][j] = pn[f][j];
                        }
                }
                advance_wait();
                release_next();  // plane kz
                kz_done = kz;
            }
            if (kz_done == K - 2) release_next();  // the top halo plane, read as z + 1 of the last plane
#pragma unroll
            for (int i = 0; i < NQ; ++i) accd[i] += (double)acc[i];
        } else {
            // no sites in this tile: keep the ring's count, plane by plane
            for (int kk = 0; kk < K; ++kk) {
                if (__any_sync(0xffffffffu, s_failed != 0)) break;
                if (!wait_next()) s_failed = 1;
                advance_wait();
                release_next();
            }
        }
        consumer_reduce_finalize<NQ, sizeof(T) == 4>(accd, m, c, sc, slots, item, nitems, nthr);
        if (tid == 0) s_stop = s_failed;
        asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
        if (s_stop) break;
    }
}

// The TMA pass for one tile per CTA (tile blockIdx.x of nitems), in one of two
// code forms: tma_items (ITEMS) or tma_tile.  They process the same tile with
// the same arithmetic in the same order (the same numbers), but compile
// differently and measured faster in different cases: one field 256^3 ...
// 512^3 0.069 / 0.205 / 0.418 ms in tma_tile against 0.103 / 0.322 / 0.673;
// two fields 256^3, 640^3 and 1024^3 0.106, 1.329 and 5.397 ms in tma_items
// against 0.111, 1.332 and 5.453, 320^3, 384^3 and 512^3 0.219, 0.309 and
// 0.691 in tma_tile against 0.244, 0.325 and 0.705; three fields spill less
// in tma_tile.
template <typename T, int NF, bool MEASURE, bool ITEMS, bool GLOBAL_MAPS = false>
__device__ __forceinline__ void tma_one_tile(const Model &m, const FieldPtrs &fp, const PassCoef &c, int txt, int ty,
                                             int zc, int S, int lpad, const TmaMaps *maps, Scalars *sc, double *slots,
                                             unsigned item, unsigned nitems, int gx, int gy)
{
    if constexpr (!ITEMS) {
        const int bx = (int)(item % (unsigned)gx), by = (int)((item / (unsigned)gx) % (unsigned)gy);
        const int bz = (int)(item / ((unsigned)gx * (unsigned)gy));
        tma_tile<T, NF, MEASURE, GLOBAL_MAPS>(m, fp, c, txt, ty, zc, S, lpad, maps, sc, slots, bx, by, bz, item, nitems);
    } else {
        tma_items<T, NF, MEASURE, GLOBAL_MAPS>(m, fp, c, txt, ty, zc, S, lpad, maps, sc, slots, item, nitems, nitems, gx,
                                               gy);
    }
}

// The code form a lattice's TMA pass takes (see tma_one_tile).
__host__ __device__ constexpr bool tma_items_form(int nf, int N) { return nf == 2 && (N <= 256 || N >= 640); }

template <typename T, int NF, bool MEASURE, int NTHR, bool ITEMS>
__global__ void __launch_bounds__(NTHR, (NTHR <= 256 ? 2 : 1)) fused_pass_tma(Model m, FieldPtrs fp, PassCoef c, int txt, int ty, int zc,
                                                         int S, int lpad, const __grid_constant__ TmaMaps maps,
                                                         Scalars *sc, double *slots, int gx, int gy, unsigned nitems)
{
    tma_one_tile<T, NF, MEASURE, ITEMS>(m, fp, c, txt, ty, zc, S, lpad, &maps, sc, slots, blockIdx.x, nitems, gx, gy);
}

// Batched form of the TMA pass: one CTA per (job, tile) item of all jobs of a
// group (same precision and field count, 7 + 1 warps), each job with its own
// model, fields, scalars, reduction slots, tile geometry and tensor maps (in
// global memory), so every job's results are bitwise those of fused_pass_tma on
// it alone with the same geometry.  S stages of at most `region` bytes per box.
template <typename T, int NF>
__global__ void __launch_bounds__(256, 2) fused_pass_tma_group(const BatchJob *__restrict__ jobs,
                                                               const unsigned *__restrict__ first_item, int njobs,
                                                               PassCoef c, int S)
{
    __shared__ int s_job;
    if (threadIdx.x == 0) {
        int lo = 0, hi = njobs - 1;  // last job whose first item <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(first_item + mid) <= blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        s_job = lo;
    }
    __syncthreads();
    const BatchJob &j = jobs[s_job];
    const unsigned local = blockIdx.x - __ldg(first_item + s_job);
    // two fields in the multi-tile code form, as for the small lattices batches
    // hold (either form gives the same numbers)
    tma_one_tile<T, NF, false, NF == 2, true>(j.m, j.fp, c, j.txt, j.ty, j.zc, S, j.lpad, j.maps, j.sc, j.slots, local,
                                              j.nblocks, j.gx, j.gy);
}

// The dynamic shared-memory limit of a kernel is a per-device attribute: raise
// it once per device and kernel (thread-safe; a lower request needs no call).
constexpr int kMaxDevices = 64;

template <typename K, int SLOTS>
static cudaError_t ensure_smem_attribute(K kern, size_t smem, std::atomic<size_t> (*configured)[SLOTS], int slot)
{
    if (smem == 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::atomic<size_t> &done = configured[dev][slot];
    if (smem <= done.load(std::memory_order_acquire)) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    size_t cur = done.load(std::memory_order_relaxed);
    while (smem > cur && !done.compare_exchange_weak(cur, smem, std::memory_order_release)) {
    }
    return cudaSuccess;
}

template <typename T, int NF, bool MEASURE>
static cudaError_t launch_tma(const Model &m, const FieldPtrs &fp, const PassCoef &c, const PassGeom &g,
                              const TmaMaps &maps, Scalars *sc, double *slots, cudaStream_t s)
{
    // 7 + 1 warps (two CTAs per SM) or 15 + 1 warps (one CTA per SM): 16
    // warps per SM, at most 4 per SM sub-partition, so 128 registers a thread
    static std::atomic<size_t> configured[kMaxDevices][4];
    const int big = g.cwarps > 7 ? 1 : 0;
    const bool items = tma_items_form(NF, m.N);
    const int threads = 32 * (g.cwarps + 1);
    auto kern = big ? (items ? fused_pass_tma<T, NF, MEASURE, 512, true> : fused_pass_tma<T, NF, MEASURE, 512, false>)
                    : (items ? fused_pass_tma<T, NF, MEASURE, 256, true> : fused_pass_tma<T, NF, MEASURE, 256, false>);
    cudaError_t e = ensure_smem_attribute(kern, g.smem, configured, big + (items ? 2 : 0));
    if (e != cudaSuccess) return e;
    // one CTA per tile, in tile order: the hardware starts each CTA as an SM
    // frees up, which keeps the CTAs in flight a compact band of neighbouring
    // tiles (their halo rows meet in L2).  A persistent grid walking tiles b,
    // b + grid, ... measured 11-25% slower: its CTAs drift apart.
    kern<<<g.nblocks, threads, g.smem, s>>>(m, fp, c, g.txt, g.ty, g.zc, g.stages, g.lpad, maps, sc, slots,
                                            (int)g.grid.x, (int)g.grid.y, g.nblocks);
    return cudaGetLastError();
}

template <typename T, int NF>
static cudaError_t launch_tma_group_t(int stages, size_t smem, const BatchJob *jobs, const unsigned *first_item,
                                      int njobs, unsigned total, const PassCoef &c, cudaStream_t s)
{
    static std::atomic<size_t> configured[kMaxDevices][2];
    auto kern = fused_pass_tma_group<T, NF>;
    cudaError_t e = ensure_smem_attribute(kern, smem, configured, 0);
    if (e != cudaSuccess) return e;
    if (total == 0) return cudaSuccess;
    kern<<<total, 256, smem, s>>>(jobs, first_item, njobs, c, stages);
    return cudaGetLastError();
}

template <typename T, int NF, bool MEASURE, int D, int NT>
static cudaError_t launch_ldg(const Model &m, const FieldPtrs &fp, const PassCoef &c, const PassGeom &g, Scalars *sc,
                              double *slots, cudaStream_t s)
{
    static std::atomic<size_t> configured[kMaxDevices][2];
    auto kern = fused_pass_ldg<T, NF, MEASURE, D, NT>;
    cudaError_t e = ensure_smem_attribute(kern, g.smem, configured, 0);
    if (e != cudaSuccess) return e;
    kern<<<g.grid, NT, g.smem, s>>>(m, fp, c, g.txt, g.ty, g.zc, sc, slots);
    return cudaGetLastError();
}

template <typename T, int NF>
static cudaError_t launch_t(const Model &m, const FieldPtrs &fp, const PassCoef &c, const PassGeom &g, Scalars *sc,
                            double *slots, bool measure_only, cudaStream_t s, const TmaMaps *maps)
{
    if (g.variant == kVariantTma) {
        if (!maps || !m.ghosts) return cudaErrorInvalidValue;
        return measure_only ? launch_tma<T, NF, true>(m, fp, c, g, *maps, sc, slots, s)
                            : launch_tma<T, NF, false>(m, fp, c, g, *maps, sc, slots, s);
    }
    const bool big = g.threads == 512;
    if (g.prefetch == 0) {
        if (big)
            return measure_only ? launch_ldg<T, NF, true, 0, 512>(m, fp, c, g, sc, slots, s)
                                : launch_ldg<T, NF, false, 0, 512>(m, fp, c, g, sc, slots, s);
        return measure_only ? launch_ldg<T, NF, true, 0, 256>(m, fp, c, g, sc, slots, s)
                            : launch_ldg<T, NF, false, 0, 256>(m, fp, c, g, sc, slots, s);
    }
    return measure_only ? launch_ldg<T, NF, true, 3, 256>(m, fp, c, g, sc, slots, s)
                        : launch_ldg<T, NF, false, 3, 256>(m, fp, c, g, sc, slots, s);
}

}  // namespace tl
