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
// keeping phi at z-1, z, z+1 in registers.  y-neighbour rows and the two
// x-edge sites come through L1/L2 (they are other threads' centre loads), so
// HBM sees each array read once and written once per pass:
// 4 sizeof(T) bytes per site per field.
#include <math.h>

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
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Scale-factor update and next-pass coefficients (one thread of the last CTA).
// tot: raw lattice sums  [sum pi_int_f^2, sum |grad+ phi_f|^2 dx^2, sum V].
__device__ void finalize(const Model &m, const PassCoef &c, Scalars *sc, const double *tot)
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
    if (!finite) sc->status = TL_EUNSTABLE;
    sc->time += sc->pending_dt;
    if (m.expanding) {
        const double al = m.alpha;
        const double rho = K + G + V;
        double b = sc->b, b_eval;
        if (c.set_b_from_constraint) {
            b = pow(a, 1.0 + al) * sqrt(m.mu2 * rho / 3.0);
            b_eval = b;
        } else {
            const double fb = pow(a, 2.0 * al + 1.0) * (m.mu2 / 3.0) * ((al - 2.0) * K + al * G + (al + 1.0) * V);
            b_eval = b + c.hb_dt * fb;
            b = b + c.edt * fb;
        }
        if (c.integer_time) {
            const double H2 = (b_eval / a) * (b_eval / a);
            sc->hubble = fabs(H2 - pow(a, 2.0 * al) * m.mu2 * rho / 3.0) / H2;
        }
        const double an = a + c.dnext_dt * b;
        sc->drift = c.dnext_dt * pow(0.5 * (a + an), al - 3.0);
        sc->a = an;
        sc->b = b;
        sc->wl = pow(an, 1.0 + al);
        sc->wv = pow(an, 3.0 + al);
        sc->wk = pow(an, -6.0);
        sc->wg = pow(an, -2.0);
    } else {
        sc->drift = c.dnext_dt;
        sc->hubble = 0.0;
    }
    sc->pending_dt = c.dnext_dt;
}

template <typename T, int NF, bool MEASURE>
__global__ void __launch_bounds__(256) fused_pass(Model m, FieldPtrs fp, PassCoef c, int txt, int ty, int zc,
                                                  Scalars *sc, double *slots)
{
    constexpr int W = Vec<T>::W;
    constexpr int NQ = 2 * NF + 1;
    const int N = m.N;
    const int tx = threadIdx.x % txt, tyi = threadIdx.x / txt;
    const int x0 = (blockIdx.x * txt + tx) * W;
    const int y = blockIdx.y * ty + tyi;
    const int z0 = blockIdx.z * zc;
    const int z1 = min(z0 + zc, N);
    const bool active = (tyi < ty) && (x0 < N) && (y < N);

    double accd[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) accd[i] = 0.0;

    if (active) {
        const T drift = (T)sc->drift;
        const T wlx = (T)(sc->wl * m.inv_dx2);
        const T wv = (T)sc->wv;
        const T kdt = (T)c.kdt, hdt = (T)c.hdt;
        const T lam = (T)m.lambda, q = (T)m.q;
        T m2[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) m2[f] = (T)m.m2[f];

        const T *phs[NF], *pis[NF];
        T *pho[NF], *pio[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            phs[f] = static_cast<const T *>(fp.phi_in[f]);
            pis[f] = static_cast<const T *>(fp.pi_in[f]);
            pho[f] = static_cast<T *>(fp.phi_out[f]);
            pio[f] = static_cast<T *>(fp.pi_out[f]);
        }
        const size_t NN = (size_t)N * (size_t)N;
        const int xl = (x0 == 0) ? N - 1 : x0 - 1;
        const int xr = (x0 + W == N) ? 0 : x0 + W;
        const size_t row = (size_t)y * N;
        const size_t rowm = (size_t)((y == 0) ? N - 1 : y - 1) * N;
        const size_t rowp = (size_t)((y + 1 == N) ? 0 : y + 1) * N;

        // phi at the evaluation time for the W sites of one row of one plane
        auto cur_vec = [&](int f, size_t off, T (&o)[W]) {
            T a[W], b[W];
            load_vec(phs[f] + off, a);
            load_vec(pis[f] + off, b);
#pragma unroll
            for (int j = 0; j < W; ++j) o[j] = fma_t(drift, b[j], a[j]);
        };
        auto cur_one = [&](int f, size_t off) -> T { return fma_t(drift, __ldg(pis[f] + off), __ldg(phs[f] + off)); };

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
                for (int j = 0; j < W; ++j) cu[f][j] = fma_t(drift, pc[f][j], a[j]);
            }
        }
        T acc[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) acc[i] = (T)0;

        for (int z = z0; z < z1; ++z) {
            const size_t pz = (size_t)z * NN;
            const size_t pn = (size_t)((z + 1 == N) ? 0 : z + 1) * NN;
            T pnext[NF][W];
            T ym[NF][W], yp[NF][W], xlv[NF], xrv[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                T a[W];
                load_vec(phs[f] + pn + row + x0, a);
                load_vec(pis[f] + pn + row + x0, pnext[f]);
#pragma unroll
                for (int j = 0; j < W; ++j) zp[f][j] = fma_t(drift, pnext[f][j], a[j]);
                cur_vec(f, pz + rowm + x0, ym[f]);
                cur_vec(f, pz + rowp + x0, yp[f]);
                xlv[f] = cur_one(f, pz + row + xl);
                xrv[f] = cur_one(f, pz + row + xr);
            }
            T pnew[NF][W];
#pragma unroll
            for (int j = 0; j < W; ++j) {
                T v[NF];
#pragma unroll
                for (int f = 0; f < NF; ++f) v[f] = cu[f][j];
                T others = (T)0;
#pragma unroll
                for (int f = 1; f < NF; ++f) others += v[f] * v[f];
                const T v02 = v[0] * v[0];
                T dv[NF];
                dv[0] = m2[0] * v[0] + lam * v02 * v[0] + q * v[0] * others;
                T Vs = (T)0.5 * m2[0] * v02 + (T)0.25 * lam * v02 * v02 + (T)0.5 * q * v02 * others;
#pragma unroll
                for (int f = 1; f < NF; ++f) {
                    dv[f] = m2[f] * v[f] + q * v02 * v[f];
                    Vs += (T)0.5 * m2[f] * v[f] * v[f];
                }
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const T cc = v[f];
                    const T left = (j == 0) ? xlv[f] : cu[f][j - 1];
                    const T right = (j == W - 1) ? xrv[f] : cu[f][j + 1];
                    const T dxm = left - cc, dxp = right - cc;
                    const T dym = ym[f][j] - cc, dyp = yp[f][j] - cc;
                    const T dzm = zm[f][j] - cc, dzp = zp[f][j] - cc;
                    const T lap = ((dxm + dxp) + (dym + dyp)) + (dzm + dzp);
                    const T F = wlx * lap - wv * dv[f];
                    const T pint = fma_t(hdt, F, pc[f][j]);
                    pnew[f][j] = fma_t(kdt, F, pc[f][j]);
                    acc[f] += pint * pint;
                    acc[NF + f] += dxp * dxp + dyp * dyp + dzp * dzp;
                }
                acc[2 * NF] += Vs;
            }
            if (!MEASURE) {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    store_vec(pho[f] + pz + row + x0, cu[f]);
                    store_vec(pio[f] + pz + row + x0, pnew[f]);
                }
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
#pragma unroll
        for (int i = 0; i < NQ; ++i) accd[i] += (double)acc[i];
    }

    // CTA reduction in a fixed order: warp tree, then warps in index order.
    __shared__ double red[32][NQ];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        double v = warp_sum(accd[i]);
        if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (tid < NQ) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += red[w][tid];
        slots[(size_t)bid * NQ + tid] = s;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(&sc->ticket, 1u) == nblocks - 1);
    __syncthreads();
    if (!last) return;

    // Last CTA: sum the slots in a fixed order (thread t takes slots t, t+nt, ...).
    __threadfence();
    const int nt = blockDim.x;
    double part[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) part[i] = 0.0;
    for (unsigned b = tid; b < nblocks; b += nt)
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

__global__ void set_background_kernel(Model m, Scalars *sc, double a, double b)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (m.expanding) {
        const double al = m.alpha;
        sc->a = a;
        sc->b = b;
        sc->wl = pow(a, 1.0 + al);
        sc->wv = pow(a, 3.0 + al);
        sc->wk = pow(a, -6.0);
        sc->wg = pow(a, -2.0);
    } else {
        sc->a = 1.0;
        sc->b = 0.0;
        sc->wl = sc->wv = sc->wk = sc->wg = 1.0;
    }
    sc->drift = 0.0;
    sc->pending_dt = 0.0;
    sc->time = 0.0;
    sc->hubble = 0.0;
    sc->status = TL_OK;
    sc->ticket = 0u;
    for (int i = 0; i < kMaxQ; ++i) sc->E[i] = 0.0;
}

PassGeom pass_geometry(int N, int elem_bytes, int sm_count)
{
    const int W = 16 / elem_bytes;
    PassGeom g;
    int per_row = N / W;  // N % 4 == 0 is required, so W | N
    // 1-D CTAs of 256 threads (whole warps, as the CTA reduction needs) laid
    // over a tile of txt x ty threads; leftover threads idle.
    g.txt = per_row < 32 ? per_row : 32;
    g.ty = 256 / g.txt;
    if (g.ty > N) g.ty = N;
    const int gx = (per_row + g.txt - 1) / g.txt;
    const int gy = (N + g.ty - 1) / g.ty;
    // z-chunk: long enough to amortise the two extra planes, short enough
    // for several waves of CTAs over the GPU.
    const long target = 8L * (sm_count > 0 ? sm_count : 152);
    int zc = N < 128 ? N : 128;
    while (zc > 4 && (long)gx * gy * ((N + zc - 1) / zc) < target) zc /= 2;
    g.zc = zc;
    g.grid = dim3(gx, gy, (N + zc - 1) / zc);
    g.nblocks = g.grid.x * g.grid.y * g.grid.z;
    return g;
}

template <typename T, int NF>
static cudaError_t launch_t(const Model &m, const FieldPtrs &fp, const PassCoef &c, const PassGeom &g, Scalars *sc,
                            double *slots, bool measure_only, cudaStream_t s)
{
    if (measure_only)
        fused_pass<T, NF, true><<<g.grid, 256, 0, s>>>(m, fp, c, g.txt, g.ty, g.zc, sc, slots);
    else
        fused_pass<T, NF, false><<<g.grid, 256, 0, s>>>(m, fp, c, g.txt, g.ty, g.zc, sc, slots);
    return cudaGetLastError();
}

cudaError_t launch_pass(int dtype, const Model &m, const FieldPtrs &fp, const PassCoef &c, const PassGeom &g,
                        Scalars *sc, double *slots, bool measure_only, cudaStream_t s)
{
    if (dtype == TL_F32) {
        switch (m.nf) {
        case 1: return launch_t<float, 1>(m, fp, c, g, sc, slots, measure_only, s);
        case 2: return launch_t<float, 2>(m, fp, c, g, sc, slots, measure_only, s);
        case 3: return launch_t<float, 3>(m, fp, c, g, sc, slots, measure_only, s);
        }
    } else {
        switch (m.nf) {
        case 1: return launch_t<double, 1>(m, fp, c, g, sc, slots, measure_only, s);
        case 2: return launch_t<double, 2>(m, fp, c, g, sc, slots, measure_only, s);
        case 3: return launch_t<double, 3>(m, fp, c, g, sc, slots, measure_only, s);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_set_background(const Model &m, Scalars *sc, double a, double b, cudaStream_t s)
{
    set_background_kernel<<<1, 32, 0, s>>>(m, sc, a, b);
    return cudaGetLastError();
}

}  // namespace tl
