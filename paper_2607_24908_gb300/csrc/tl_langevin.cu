// Langevin evolution of a scalar phi^4 field (the paper's interface example,
// Sec. 2, Eq. 1): Euler-Maruyama steps
//     phi <- phi + dt (Lap phi - m^2 phi - (lambda/2) phi^3) + noise sqrt(dt) xi,
// with xi a unit Gaussian per site and step (the paper's field-valued random
// number generator rescaled by 1/sqrt(dt)).  The sites with dense indices 2k
// and 2k + 1 share one Philox-2x64-10 draw of counter (k, 2^63 + step) under
// key seed; Box-Muller on its two words gives two independent Gaussians, the
// cosine one for site 2k and the sine one for site 2k + 1 (half the generator
// work of one draw per site, which bounds this kernel).
//
// One kernel per step, marching z-planes like the fused pass: phi at z-1, z,
// z+1 in registers, the y-neighbour rows and edge sites through L1/L2; HBM
// sees one read and one write of phi per site.  The field ping-pongs between
// the lattice's two phi_0 buffers; momenta are not used.
#include <math.h>
#include <stdint.h>

#include "tl_internal.cuh"
#include "tl_lattice.cuh"
#include "tl_philox.cuh"

namespace {

using tl::philox2x64_10;  // the initial-state draw's generator

// The two Gaussians of draw k: (cos, sin) halves of Box-Muller.
template <typename T>
__device__ __forceinline__ void gauss2(uint64_t k, uint64_t ctr1, uint64_t seed, T &gc, T &gs);

template <>
__device__ __forceinline__ void gauss2<double>(uint64_t k, uint64_t ctr1, uint64_t seed, double &gc, double &gs)
{
    uint64_t w0, w1;
    philox2x64_10(k, ctr1, seed, w0, w1);
    const double two53 = 9007199254740992.0;
    const double u1 = ((double)(w0 >> 11) + 1.0) / two53;
    const double u2 = (double)(w1 >> 11) / two53;
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    gc = r * c;
    gs = r * s;
}

// x 2^-53 for an integer 0 <= x <= 2^53, formed in FP32 without FP64
// arithmetic (GB300's FP64 pipe is slow): x = hi 2^29 + lo, hi <= 2^24 exact,
// lo < 2^29 rounded once on conversion, one more rounding in the fma; the
// result keeps a relative precision of about 2^-24 at any magnitude, so small
// u1 (the Gaussian tail) stays as accurate as in a correctly rounded FP64->FP32
// conversion.
__device__ __forceinline__ float u53_f32(uint64_t x)
{
    const uint32_t hi = (uint32_t)(x >> 29), lo = (uint32_t)(x & 0x1FFFFFFFu);
    return fmaf((float)hi, 0x1p-24f, (float)lo * 0x1p-53f);
}

template <>
__device__ __forceinline__ void gauss2<float>(uint64_t k, uint64_t ctr1, uint64_t seed, float &gc, float &gs)
{
    uint64_t w0, w1;
    philox2x64_10(k, ctr1, seed, w0, w1);
    // the same 53-bit uniforms, Box-Muller in FP32 (the field is stored in FP32)
    const float u1 = u53_f32((w0 >> 11) + 1);
    const float u2 = u53_f32(w1 >> 11);
    const float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    gc = r * c;
    gs = r * s;
}

template <typename T>
struct V16;
template <>
struct V16<float> {
    static constexpr int W = 4;
};
template <>
struct V16<double> {
    static constexpr int W = 2;
};

template <typename T>
__device__ __forceinline__ void ld(const T *p, T (&o)[V16<T>::W])
{
#pragma unroll
    for (int j = 0; j < V16<T>::W; ++j) o[j] = __ldg(p + j);
}

template <typename T>
__global__ void __launch_bounds__(256) langevin_pass(const T *__restrict__ in, T *__restrict__ out, int N, int txt,
                                                     int ty, int zc, long long P, long long PP, T inv_dx2, T dt, T m2,
                                                     T half_lam, T amp, uint64_t seed, uint64_t ctr1)
{
    constexpr int W = V16<T>::W;
    const int tx = threadIdx.x % txt, tyi = threadIdx.x / txt;
    const int x0 = (blockIdx.x * txt + tx) * W;
    const int y = blockIdx.y * ty + tyi;
    const int z0 = blockIdx.z * zc;
    const int z1 = min(z0 + zc, N);
    if (!(tyi < ty && x0 < N && y < N)) return;
    const size_t NN = (size_t)PP;
    const size_t row = (size_t)y * P, rowm = (size_t)(y == 0 ? N - 1 : y - 1) * P,
                 rowp = (size_t)(y + 1 == N ? 0 : y + 1) * P;
    // ghost rows of this thread's sites (padded arrays carry one ghost row on
    // each side of a plane; the x-edges need no copies)
    const long long gy = y == 0 ? (long long)N * P : (y == N - 1 ? -(long long)N * P : 0);
    const int xl = x0 == 0 ? N - 1 : x0 - 1, xr = x0 + W == N ? 0 : x0 + W;
    T zm[W], cu[W], zp[W];
    ld(in + (size_t)(z0 == 0 ? N - 1 : z0 - 1) * NN + row + x0, zm);
    ld(in + (size_t)z0 * NN + row + x0, cu);
    for (int z = z0; z < z1; ++z) {
        const size_t pz = (size_t)z * NN;
        T ym[W], yp[W];
        ld(in + (size_t)(z + 1 == N ? 0 : z + 1) * NN + row + x0, zp);
        ld(in + pz + rowm + x0, ym);
        ld(in + pz + rowp + x0, yp);
        const T a = __ldg(in + pz + row + xl), b = __ldg(in + pz + row + xr);
        T xi[W];  // x0 and W are even: the thread's sites form whole pairs
        const uint64_t k0 = (((uint64_t)z * N + y) * N + x0) >> 1;
#pragma unroll
        for (int j = 0; j < W; j += 2) gauss2<T>(k0 + j / 2, ctr1, seed, xi[j], xi[j + 1]);
        T o[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const T c = cu[j];
            const T left = j == 0 ? a : cu[j - 1];
            const T right = j == W - 1 ? b : cu[j + 1];
            const T lap = (((left - c) + (right - c)) + ((ym[j] - c) + (yp[j] - c))) + ((zm[j] - c) + (zp[j] - c));
            const T drift = lap * inv_dx2 - m2 * c - half_lam * c * c * c;
            o[j] = (c + dt * drift) + amp * xi[j];
        }
#pragma unroll
        for (int j = 0; j < W; ++j) {
            out[pz + row + x0 + j] = o[j];
            if (gy) out[pz + row + x0 + j + gy] = o[j];
        }
#pragma unroll
        for (int j = 0; j < W; ++j) {
            zm[j] = cu[j];
            cu[j] = zp[j];
        }
    }
}

}  // namespace

extern "C" int tl_langevin_step(tl_lattice *L, int n, double dt, const tl_langevin_params *p, uint64_t seed)
{
    tl::NvtxScope nvtx_range("tl_langevin_step");
    tl::set_error(TL_OK, "", "");
    if (!L || !p) return tl::fail(TL_EINVAL, "NULL argument");
    if (n < 0 || !(dt > 0.0) || !isfinite(dt)) return tl::fail(TL_EINVAL, "n >= 0 and a positive finite dt needed");
    if (!isfinite(p->lambda) || !isfinite(p->m2) || !isfinite(p->noise)) return tl::fail(TL_EINVAL, "non-finite parameter");
    if (!(L->state_mask & 1u)) return tl::fail(TL_ESTATE, "phi_0 has not been set");
    if (L->batch_refs > 0) return tl::fail(TL_ESTATE, "lattice is part of a batch");
    tl::PassTuning t{tl::kVariantLdg, 8, 0, 0, 0, 256, 0};
    const tl::PassGeom g = tl::pass_geometry(L->N, (int)L->esz, L->sm_count, 1, t);
    const double inv_dx2 = 1.0 / (L->dx * L->dx);
    const double amp = p->noise * sqrt(dt);
    for (int s = 0; s < n; ++s) {
        void *in = L->buf[L->cur][0][0];
        void *out = L->buf[L->cur ^ 1][0][0];
        const uint64_t ctr1 = (1ull << 63) + (uint64_t)(L->langevin_steps + s);
        if (L->dtype == TL_F32)
            langevin_pass<float><<<g.grid, 256, 0, L->stream>>>(
                static_cast<const float *>(in), static_cast<float *>(out), L->N, g.txt, g.ty, g.zc, L->model.pitch,
                L->model.pplane, (float)inv_dx2,
                (float)dt, (float)p->m2, (float)(0.5 * p->lambda), (float)amp, seed, ctr1);
        else
            langevin_pass<double><<<g.grid, 256, 0, L->stream>>>(
                static_cast<const double *>(in), static_cast<double *>(out), L->N, g.txt, g.ty, g.zc, L->model.pitch,
                L->model.pplane, inv_dx2, dt,
                p->m2, 0.5 * p->lambda, amp, seed, ctr1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return tl::fail(TL_ECUDA, "langevin_pass: %s", cudaGetErrorString(e));
        // phi_0 ping-pongs; the momenta stay where they are
        L->buf[L->cur][0][0] = out;
        L->buf[L->cur ^ 1][0][0] = in;
    }
    L->langevin_steps += n;
    L->energies_valid = false;
    if (n & 1) tl::invalidate_launches(L);  // phi_0's buffers traded places: tensor maps and graphs are stale
    return TL_OK;
}
