// Classical SU(2) Yang-Mills in temporal gauge: the paper's benchmark
// workload (Sec. 4), each step a kick of the electric fields by the plaquette
// staples and a drift of the links by the closed-form SU(2) exponential map.
//
// Links are unit quaternions U = u0 + i u.s, stored on the device as
// quaternion records [direction][site][4] (one 16-byte load per link in FP32,
// two in FP64; consecutive threads read consecutive records); electric fields
// su(2) vectors E = i e.s, component-major [direction][component][site] (only
// a site's own fields are read).  The host layout of both is component-major;
// tl_su2_set_state / tl_su2_get_state transpose the links through the spare
// link buffer.
// One fused pass per step: e_i(x) <- e_i(x) - 2 dt sum_{j != i} Im[U_i S_ij]
// with the old links, then U_i(x) <- exp(dt E_i(x)) U_i(x) written to the
// other link buffer (ping-pong), so the neighbours' staples always see the old
// links.  HBM per site and step: read 12 link + 9 field values, write 9 + 12.
// A separate measurement kernel reduces the electric and plaquette energies
// and the Gauss-law violation in a fixed order (per-CTA slots, one summing CTA).
#include <math.h>
#include <stdint.h>

#include <new>

#include "tl_internal.cuh"
#include "tl_lattice.cuh"
#include "tl_philox.cuh"

namespace {

template <typename T>
struct Q {
    T w, x, y, z;
};

template <typename T>
__device__ __forceinline__ Q<T> qmul(const Q<T> &a, const Q<T> &b)
{
    // (a0 + i a.s)(b0 + i b.s) = a0 b0 - a.b + i (a0 b + b0 a - a x b).s
    Q<T> r;
    r.w = a.w * b.w - (a.x * b.x + a.y * b.y + a.z * b.z);
    r.x = a.w * b.x + b.w * a.x - (a.y * b.z - a.z * b.y);
    r.y = a.w * b.y + b.w * a.y - (a.z * b.x - a.x * b.z);
    r.z = a.w * b.z + b.w * a.z - (a.x * b.y - a.y * b.x);
    return r;
}
template <typename T>
__device__ __forceinline__ Q<T> qadj(const Q<T> &a)
{
    return Q<T>{a.w, -a.x, -a.y, -a.z};
}
template <typename T>
__device__ __forceinline__ Q<T> qadd(const Q<T> &a, const Q<T> &b)
{
    return Q<T>{a.w + b.w, a.x + b.x, a.y + b.y, a.z + b.z};
}

__device__ __forceinline__ size_t sidx(int N, int x, int y, int z)
{
    x = x < 0 ? x + N : (x >= N ? x - N : x);
    y = y < 0 ? y + N : (y >= N ? y - N : y);
    z = z < 0 ? z + N : (z >= N ? z - N : z);
    return ((size_t)z * N + y) * N + x;
}

// Link record of direction i at site s (records are 16- or 32-byte aligned).
__device__ __forceinline__ Q<float> ldU(const float *U, size_t n3, int i, size_t s)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(U + ((size_t)i * n3 + s) * 4));
    return Q<float>{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Q<double> ldU(const double *U, size_t n3, int i, size_t s)
{
    const double2 *b = reinterpret_cast<const double2 *>(U + ((size_t)i * n3 + s) * 4);
    const double2 a = __ldg(b), c = __ldg(b + 1);
    return Q<double>{a.x, a.y, c.x, c.y};
}
__device__ __forceinline__ void stU(float *U, size_t n3, int i, size_t s, const Q<float> &q)
{
    *reinterpret_cast<float4 *>(U + ((size_t)i * n3 + s) * 4) = make_float4(q.w, q.x, q.y, q.z);
}
__device__ __forceinline__ void stU(double *U, size_t n3, int i, size_t s, const Q<double> &q)
{
    double2 *b = reinterpret_cast<double2 *>(U + ((size_t)i * n3 + s) * 4);
    b[0] = make_double2(q.w, q.x);
    b[1] = make_double2(q.y, q.z);
}

template <typename T>
__device__ __forceinline__ void sincos_t(T a, T *s, T *c);
template <>
__device__ __forceinline__ void sincos_t<float>(float a, float *s, float *c) { sincosf(a, s, c); }
template <>
__device__ __forceinline__ void sincos_t<double>(double a, double *s, double *c) { sincos(a, s, c); }

// The rotation of the drift, exp(i dt e.s) = cos(theta) + i f e.s with
// theta = dt |e| and f = sin(theta) / |e| = dt sin(theta) / theta, from
// q2 = |e|^2.  Small angles (theta^2 below kSmallTheta2, the common case: the
// per-step angle is tiny) use the Taylor series of sin(theta)/theta and
// cos(theta) in theta^2, truncated where the first omitted term is below half
// an ulp of the result (FP32: theta < 1/2, terms to theta^8, first omitted
// term < 3e-10; FP64: theta < 1/4, terms to theta^10 / theta^12, < 1e-17): no
// square root, no division, no trigonometric call.  Larger angles take
// sincos of theta.
template <typename T>
constexpr T kSmallTheta2 = sizeof(T) == 4 ? (T)0.25 : (T)0.0625;

template <typename T>
__device__ __forceinline__ void drift_rotation(T q2, T dt, T *f, T *cs)
{
    const T t2 = dt * dt * q2;
    if (t2 < kSmallTheta2<T>) {
        T sc, cc;
        if (sizeof(T) == 4) {
            // sin(t)/t = sum_k (-t^2)^k / (2k+1)!,  cos(t) = sum_k (-t^2)^k / (2k)!
            sc = (T)(1.0 / 362880.0);
            sc = sc * t2 - (T)(1.0 / 5040.0);
            sc = sc * t2 + (T)(1.0 / 120.0);
            sc = sc * t2 - (T)(1.0 / 6.0);
            cc = (T)(1.0 / 40320.0);
            cc = cc * t2 - (T)(1.0 / 720.0);
            cc = cc * t2 + (T)(1.0 / 24.0);
            cc = cc * t2 - (T)(1.0 / 2.0);
        } else {
            sc = (T)(-1.0 / 39916800.0);
            sc = sc * t2 + (T)(1.0 / 362880.0);
            sc = sc * t2 - (T)(1.0 / 5040.0);
            sc = sc * t2 + (T)(1.0 / 120.0);
            sc = sc * t2 - (T)(1.0 / 6.0);
            cc = (T)(1.0 / 479001600.0);
            cc = cc * t2 - (T)(1.0 / 3628800.0);
            cc = cc * t2 + (T)(1.0 / 40320.0);
            cc = cc * t2 - (T)(1.0 / 720.0);
            cc = cc * t2 + (T)(1.0 / 24.0);
            cc = cc * t2 - (T)(1.0 / 2.0);
        }
        *f = dt * (sc * t2 + (T)1);
        *cs = cc * t2 + (T)1;
    } else {
        const T nrm = sqrt(q2);
        T sn;
        sincos_t<T>(dt * nrm, &sn, cs);
        *f = sn / nrm;
    }
}

template <typename T>
struct alignas(4 * sizeof(T)) Rec {
    T w, x, y, z;
};

__device__ __forceinline__ float fma_su(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_su(double a, double b, double c) { return fma(a, b, c); }

// F += sg (V - R(W^+) v), with R(W^+) v = Im(W^+ (0, v) W) the vector v rotated
// by the adjoint action of W^+.  For W = w + i u.s,
//   R(W^+) v = (w^2 - |u|^2) v + 2 (u.v) u + 2 w (u x v),
// which for a unit W is v + 2 w (u x v) + 2 u x (u x v); that form is
// accumulated here (two cross products and fused multiply-adds).  Links are
// unit quaternions anyway: the plaquette form of the backward staple itself
// uses W^+ W = 1.
template <typename T>
__device__ __forceinline__ void add_force(const Q<T> &W, const Rec<T> &V, const Rec<T> &v, T sg, T &Fx, T &Fy, T &Fz)
{
    const T cx = W.y * v.z - W.z * v.y, cy = W.z * v.x - W.x * v.z, cz = W.x * v.y - W.y * v.x;
    const T dx = W.y * cz - W.z * cy, dy = W.z * cx - W.x * cz, dz = W.x * cy - W.y * cx;
    const T a = (T)-2 * sg * W.w, b = (T)-2 * sg;
    Fx = fma_su(b, dx, fma_su(a, cx, Fx + sg * (V.x - v.x)));
    Fy = fma_su(b, dy, fma_su(a, cy, Fy + sg * (V.y - v.y)));
    Fz = fma_su(b, dz, fma_su(a, cz, Fz + sg * (V.z - v.z)));
}

// One pass per step over CTAs of 32 x 8 site columns, each marching a chunk of
// z-planes.  The force on U_i(x) is Im[U_i(x) S_i(x)] with the staples S of
// Sec. 4; in terms of the plaquettes
//   P_ij(x) = U_i(x) U_j(x+i) U_i(x+j)^+ U_j(x)^+,   V_ij = Im P_ij = -V_ji,
// U_i f_ij(x) = P_ij(x) and, for unit links, U_i b_ij(x) = W^+ P_ij(x-j)^+ W
// with W = U_j(x-j), so
//   Im[U_i S_i](x) = sum_{j != i} V_ij(x) - R(W^+) V_ij(x-j),
// R(W^+) the rotation of add_force.  Each plaquette is then formed once per site
// (three per site, instead of four staples per link) and shared through shared
// memory: V_xy, V_xz, V_yz of the CTA's tile plus the -x / -y halo it needs,
// in three buffers (planes z-1, z, and z+1 being formed).
//
// The link records of a plane's tile with a one-site halo, (kSu2Ty + 2) x
// (kSu2Tx + 2) sites x 3 directions, are copied into a ring of shared-memory
// stages with cp.async (16-byte chunks, addresses wrapped periodically by the
// copying thread) one plane ahead of their first use.  Stage s holds the
// plane with relative index (z - z0 + 1) % 4 == s.
constexpr int kSu2Tx = 32, kSu2Ty = 8;
constexpr int kSu2Hx = kSu2Tx + 2, kSu2Hy = kSu2Ty + 2;  // link tile with its one-site halo
constexpr int kSu2StageRecs = 3 * kSu2Hy * kSu2Hx;     // 1020 link records per plane
constexpr int kSu2Stages = 4;
constexpr int kSu2Px = kSu2Tx + 1, kSu2Py = kSu2Ty + 1;  // plaquette tile with the -x / -y halo
constexpr int kSu2PlaqRecs = 3 * kSu2Py * kSu2Px;      // 891 per buffer (V_xy, V_xz, V_yz)
constexpr int kSu2PlaqBufs = 3;                        // planes z-1 (read), z (read), z+1 (written)
constexpr int kSu2HaloJobs = 2 * kSu2Tx + 2 * kSu2Ty;   // row y0-1: V_xy, V_yz; column x0-1: V_xy, V_xz

template <typename T>
constexpr size_t su2_tiled_smem()
{
    return (size_t)(kSu2Stages * kSu2StageRecs + kSu2PlaqBufs * kSu2PlaqRecs) * sizeof(Rec<T>);
}

__device__ __forceinline__ void cp_async_cg16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1)
    su2_pass(const T *__restrict__ U, T *__restrict__ Uout, T *__restrict__ E, int N, int zc, T dt)
{
    extern __shared__ __align__(16) unsigned char su2_raw[];
    Rec<T> *ring = reinterpret_cast<Rec<T> *>(su2_raw);
    Rec<T> *plaq = ring + kSu2Stages * kSu2StageRecs;
    const int tid = threadIdx.x;
    const int tx = tid % kSu2Tx, ty = tid / kSu2Tx;
    const int x0 = blockIdx.x * kSu2Tx, y0 = blockIdx.y * kSu2Ty;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < N && y < N;
    const size_t n3 = (size_t)N * N * N;
    const size_t NN = (size_t)N * N;
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, N);

    // this thread's copy chunks: chunk r of a stage is half (r % C) of record
    // r / C = (i * Hy + ry) * Hx + rx; its source packed as wx | wy << 11 |
    // i << 22 | half << 24 (N <= 1290 < 2^11)
    constexpr int C = (int)sizeof(T) / 4;
    constexpr int kChunks = kSu2StageRecs * C;
    constexpr int kSlots = (kChunks + 255) / 256;
    unsigned src[kSlots];
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
        const int r = tid + 256 * k;
        const int rec = r / C, half = r % C;
        const int i = rec / (kSu2Hy * kSu2Hx), q = rec % (kSu2Hy * kSu2Hx);
        const int wx = (x0 - 1 + q % kSu2Hx + N) % N, wy = (y0 - 1 + q / kSu2Hx + N) % N;
        src[k] = (unsigned)wx | (unsigned)wy << 11 | (unsigned)(i & 3) << 22 | (unsigned)half << 24;
    }
    auto copy_plane = [&](int z) {
        const int zz = z < 0 ? z + N : (z >= N ? z - N : z);
        unsigned char *st = reinterpret_cast<unsigned char *>(ring + ((z - z0 + 1) & (kSu2Stages - 1)) * kSu2StageRecs);
        const T *Uz = U + (size_t)zz * NN * 4;
#pragma unroll
        for (int k = 0; k < kSlots; ++k) {
            const int r = tid + 256 * k;
            const unsigned v = src[k];
            const size_t rec = (size_t)((v >> 22) & 3u) * n3 + (size_t)((v >> 11) & 2047u) * N + (v & 2047u);
            if (r < kChunks) cp_async_cg16(st + (size_t)r * 16, Uz + rec * 4 + (v >> 24) * (16 / sizeof(T)));
        }
        cp_async_commit();
    };
    // link i at tile position (rx, ry) of the plane with relative index zr = z - z0 + 1
    auto link = [&](int i, int rx, int ry, int zr) -> Q<T> {
        const Rec<T> v = ring[(zr & (kSu2Stages - 1)) * kSu2StageRecs + (i * kSu2Hy + ry) * kSu2Hx + rx];
        return Q<T>{v.w, v.x, v.y, v.z};
    };
    // V_ij at tile position (rx, ry) of plane zr (i < j; reads planes zr and zr + 1)
    auto plaq_im = [&](int i, int j, int rx, int ry, int zr) -> Rec<T> {
        const Q<T> a = link(i, rx, ry, zr);
        const Q<T> b = link(j, rx + (i == 0), ry + (i == 1), zr + (i == 2));
        const Q<T> c = link(i, rx + (j == 0), ry + (j == 1), zr + (j == 2));
        const Q<T> d = link(j, rx, ry, zr);
        const Q<T> p = qmul(qmul(a, b), qmul(qadj(c), qadj(d)));
        return Rec<T>{(T)0, p.x, p.y, p.z};
    };
    auto pidx = [](int buf, int k, int rx, int ry) { return buf * kSu2PlaqRecs + (k * kSu2Py + ry) * kSu2Px + rx; };
    const int rx = tx + 1, ry = ty + 1;
    // plaquettes of plane zr (own site and the -x / -y halo) into buffer zr % 3
    auto form_plaquettes = [&](int zr) {
        const int b = zr % kSu2PlaqBufs;
        if (active) {
            plaq[pidx(b, 0, rx, ry)] = plaq_im(0, 1, rx, ry, zr);
            plaq[pidx(b, 1, rx, ry)] = plaq_im(0, 2, rx, ry, zr);
            plaq[pidx(b, 2, rx, ry)] = plaq_im(1, 2, rx, ry, zr);
        }
        if (tid < kSu2HaloJobs) {  // row y0-1 (V_xy, V_yz), column x0-1 (V_xy, V_xz)
            const bool row = tid < 2 * kSu2Tx;
            const int hx = row ? 1 + tid % kSu2Tx : 0;
            const int hy = row ? 0 : 1 + (tid - 2 * kSu2Tx) % kSu2Ty;
            const int k = row ? (tid < kSu2Tx ? 0 : 2) : (tid < 2 * kSu2Tx + kSu2Ty ? 0 : 1);
            plaq[pidx(b, k, hx, hy)] = k == 0   ? plaq_im(0, 1, hx, hy, zr)
                                       : k == 1 ? plaq_im(0, 2, hx, hy, zr)
                                                : plaq_im(1, 2, hx, hy, zr);
        }
    };

    // Software pipeline, one barrier per plane: the interval of plane z forms
    // the plaquettes of plane z+1 and then updates the links of plane z from
    // the plaquettes of planes z and z-1 (formed in earlier intervals).  Ring
    // stages hold planes z..z+2 while z+3 lands; U_z(x - z) is carried in
    // registers from the previous plane, whose stage is being refilled.
    copy_plane(z0 - 1);
    copy_plane(z0);
    copy_plane(z0 + 1);
    copy_plane(z0 + 2);
    cp_async_wait_all();
    __syncthreads();
    Q<T> uz_prev{0, 0, 0, 0};
    if (active) {  // V_xz, V_yz of plane z0 - 1 (relative index 0) for the first plane's -z terms
        plaq[pidx(0, 1, rx, ry)] = plaq_im(0, 2, rx, ry, 0);
        plaq[pidx(0, 2, rx, ry)] = plaq_im(1, 2, rx, ry, 0);
        uz_prev = link(2, rx, ry, 0);
    }
    form_plaquettes(1);
    // the electric fields of a plane are loaded one plane ahead of their update
    T eo[9], en[9];
    const size_t s0 = (size_t)z0 * NN + (size_t)y * N + x;
    if (active) {
#pragma unroll
        for (int c = 0; c < 9; ++c) eo[c] = E[(size_t)c * n3 + s0];
    }
    for (int z = z0; z < z1; ++z) {
        const int zr = z - z0 + 1;
        const int cur = zr % kSu2PlaqBufs, prev = (zr + kSu2PlaqBufs - 1) % kSu2PlaqBufs;
        cp_async_wait_all();
        __syncthreads();  // plaquettes of plane z complete, plane z+2 landed; the stage of z-1 and buffer (z+1) % 3 are free
        if (z + 3 <= z1) copy_plane(z + 3);
        const size_t s = (size_t)z * NN + (size_t)y * N + x;
        if (active && z + 1 < z1) {
#pragma unroll
            for (int c = 0; c < 9; ++c) en[c] = E[(size_t)c * n3 + s + NN];
        }
        if (z + 1 < z1) form_plaquettes(zr + 1);
        if (!active) continue;
        Rec<T> V[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) V[k] = plaq[pidx(cur, k, rx, ry)];
        const Q<T> uz = link(2, rx, ry, zr);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T Fx = 0, Fy = 0, Fz = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (j == i) continue;
                const int k = i + j - 1;  // (0,1) -> 0, (0,2) -> 1, (1,2) -> 2
                const T sg = i < j ? (T)1 : (T)-1;
                // V_ij(x - j) and W = U_j(x - j)
                const Rec<T> vn = j == 0   ? plaq[pidx(cur, k, rx - 1, ry)]
                                  : j == 1 ? plaq[pidx(cur, k, rx, ry - 1)]
                                           : plaq[pidx(prev, k, rx, ry)];
                const Q<T> W = j == 0 ? link(0, rx - 1, ry, zr) : j == 1 ? link(1, rx, ry - 1, zr) : uz_prev;
                add_force(W, V[k], vn, sg, Fx, Fy, Fz);
            }
            const T e1 = eo[3 * i] - (T)2 * dt * Fx;
            const T e2 = eo[3 * i + 1] - (T)2 * dt * Fy;
            const T e3 = eo[3 * i + 2] - (T)2 * dt * Fz;
            T *ei = E + (size_t)(3 * i) * n3 + s;
            ei[0] = e1;
            ei[n3] = e2;
            ei[2 * n3] = e3;
            // drift: exp(i dt e.s) = cos(dt|e|) + i sin(dt|e|) e/|e|
            T f, cs;
            drift_rotation<T>(e1 * e1 + e2 * e2 + e3 * e3, dt, &f, &cs);
            Q<T> u = qmul(Q<T>{cs, f * e1, f * e2, f * e3}, i == 2 ? uz : link(i, rx, ry, zr));
            if (sizeof(T) == 4) {  // FP32 storage: keep the link on the unit sphere
                const T r = rsqrt(u.w * u.w + u.x * u.x + u.y * u.y + u.z * u.z);
                u = Q<T>{u.w * r, u.x * r, u.y * r, u.z * r};
            }
            stU(Uout, n3, i, s, u);
        }
        uz_prev = uz;
#pragma unroll
        for (int c = 0; c < 9; ++c) eo[c] = en[c];
    }
    cp_async_wait_all();
}

// Per-CTA partial sums of |e|^2/2, 2(1 - Re P_ij) and |G|^2, and the CTA's
// max |G|, into slots[4 * cta + q].
template <typename T>
__global__ void __launch_bounds__(256) su2_measure(const T *__restrict__ U, const T *__restrict__ E, int N,
                                                   double *slots)
{
    const size_t n3 = (size_t)N * N * N;
    double el = 0.0, mag = 0.0, g2 = 0.0, gmax = 0.0;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n3; s += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % N), y = (int)((s / N) % N), z = (int)(s / ((size_t)N * N));
        const int d[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        double G[3] = {0, 0, 0};
        for (int i = 0; i < 3; ++i) {
            const T *e = E + (size_t)(3 * i) * n3;
            const double a = e[s], b = e[s + n3], c = e[s + 2 * n3];
            el += 0.5 * (a * a + b * b + c * c);
            // Gauss: E_i(x) - U_i(x-i)^+ E_i(x-i) U_i(x-i)
            const size_t xm = sidx(N, x - d[i][0], y - d[i][1], z - d[i][2]);
            auto ld = [&](int k, size_t site) {
                const Q<T> q = ldU(U, n3, k, site);
                return Q<double>{(double)q.w, (double)q.x, (double)q.y, (double)q.z};
            };
            const Q<double> Um = ld(i, xm);
            const Q<double> Em{0.0, (double)e[xm], (double)e[xm + n3], (double)e[xm + 2 * n3]};
            const Q<double> t = qmul(qmul(qadj(Um), Em), Um);
            G[0] += a - t.x;
            G[1] += b - t.y;
            G[2] += c - t.z;
            for (int j = i + 1; j < 3; ++j) {
                const size_t xpi = sidx(N, x + d[i][0], y + d[i][1], z + d[i][2]);
                const size_t xpj = sidx(N, x + d[j][0], y + d[j][1], z + d[j][2]);
                const Q<double> P = qmul(qmul(qmul(ld(i, s), ld(j, xpi)), qadj(ld(i, xpj))), qadj(ld(j, s)));
                mag += 2.0 * (1.0 - P.w);
            }
        }
        const double gg = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
        g2 += gg;
        gmax = fmax(gmax, sqrt(gg));
    }
    __shared__ double red[8][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double v[4] = {el, mag, g2, gmax};
    for (int q = 0; q < 4; ++q) {
        double w = v[q];
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_xor_sync(0xffffffffu, w, o);
            w = q == 3 ? fmax(w, u) : w + u;
        }
        if (lane == 0) red[warp][q] = w;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double w = red[0][threadIdx.x];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
            w = threadIdx.x == 3 ? fmax(w, red[k][threadIdx.x]) : w + red[k][threadIdx.x];
        slots[4 * blockIdx.x + threadIdx.x] = w;
    }
}

__global__ void su2_sum_slots(const double *slots, int nblocks, double inv_n3, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double el = 0, mag = 0, g2 = 0, gmax = 0;
    for (int b = 0; b < nblocks; ++b) {
        el += slots[4 * b];
        mag += slots[4 * b + 1];
        g2 += slots[4 * b + 2];
        gmax = fmax(gmax, slots[4 * b + 3]);
    }
    out[0] = el * inv_n3;
    out[1] = mag * inv_n3;
    out[2] = gmax;
    out[3] = sqrt(g2 * inv_n3);
}


template <typename T>
__global__ void su2_init(T *U, T *E, int N, uint64_t seed, double amp)
{
    const size_t n3 = (size_t)N * N * N;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n3; s += (size_t)gridDim.x * blockDim.x) {
        for (int i = 0; i < 3; ++i) {
            double g[4];
            for (int h = 0; h < 2; ++h) {
                uint64_t w0, w1;
                tl::philox2x64_10(3 * s + i, (1ull << 62) + h, seed, w0, w1);  // random initial links
                const double u1 = ((double)(w0 >> 11) + 1.0) / 9007199254740992.0;
                const double u2 = (double)(w1 >> 11) / 9007199254740992.0;
                const double r = sqrt(-2.0 * log(u1));
                double sn, cs;
                sincospi(2.0 * u2, &sn, &cs);
                g[2 * h] = r * cs;
                g[2 * h + 1] = r * sn;
            }
            const double q1 = amp * g[0], q2 = amp * g[1], q3 = amp * g[2];
            const double inv = 1.0 / sqrt(1.0 + q1 * q1 + q2 * q2 + q3 * q3);
            stU(U, n3, i, s, Q<T>{(T)inv, (T)(q1 * inv), (T)(q2 * inv), (T)(q3 * inv)});
            for (int c = 0; c < 3; ++c) E[(3 * i + c) * n3 + s] = (T)0;
        }
    }
}

// Host layout U[i][c][site] <-> device records U[i][site][c].
template <typename T>
__global__ void su2_to_records(const T *__restrict__ cm, T *__restrict__ rec, size_t n3)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < 3 * n3; k += (size_t)gridDim.x * blockDim.x) {
        const size_t i = k / n3, s = k - i * n3;
        stU(rec, n3, (int)i, s, Q<T>{cm[(4 * i) * n3 + s], cm[(4 * i + 1) * n3 + s], cm[(4 * i + 2) * n3 + s],
                                    cm[(4 * i + 3) * n3 + s]});
    }
}
template <typename T>
__global__ void su2_from_records(const T *__restrict__ rec, T *__restrict__ cm, size_t n3)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < 3 * n3; k += (size_t)gridDim.x * blockDim.x) {
        const size_t i = k / n3, s = k - i * n3;
        const Q<T> q = ldU(rec, n3, (int)i, s);
        cm[(4 * i) * n3 + s] = q.w;
        cm[(4 * i + 1) * n3 + s] = q.x;
        cm[(4 * i + 2) * n3 + s] = q.y;
        cm[(4 * i + 3) * n3 + s] = q.z;
    }
}

}  // namespace

struct tl_su2 {
    int N = 0;
    tl_dtype dtype = TL_F64;
    size_t esz = 8;
    cudaStream_t stream = nullptr;
    void *U[2] = {nullptr, nullptr};
    void *E = nullptr;
    int cur = 0;
    double *slots = nullptr;
    double *out = nullptr;
    int mblocks = 0;
    int sm_count = 0;
    bool has_state = false;
};

#define SU_CK(call)                                                                                         \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess)                                                                              \
            return tl::fail(e_ == cudaErrorMemoryAllocation ? TL_ENOMEM : TL_ECUDA, "%s: %s", #call,        \
                            cudaGetErrorString(e_));                                                        \
    } while (0)

extern "C" {

void tl_su2_destroy(tl_su2 *Y)
{
    if (!Y) return;
    cudaStreamSynchronize(Y->stream);
    cudaFree(Y->U[0]);
    cudaFree(Y->U[1]);
    cudaFree(Y->E);
    cudaFree(Y->slots);
    cudaFree(Y->out);
    delete Y;
}

int tl_su2_create(tl_su2 **out, int N, tl_dtype dtype, void *cuda_stream)
{
    tl::set_error(TL_OK, "", "");
    if (!out) return tl::fail(TL_EINVAL, "NULL out");
    *out = nullptr;
    if (N < 4 || N > 1290) return tl::fail(TL_EINVAL, "N must be in [4, 1290]");
    if (dtype != TL_F32 && dtype != TL_F64) return tl::fail(TL_EINVAL, "unknown dtype");
    tl_su2 *Y = new (std::nothrow) tl_su2();
    if (!Y) return tl::fail(TL_ENOMEM, "host allocation failed");
    Y->N = N;
    Y->dtype = dtype;
    Y->esz = dtype == TL_F32 ? 4 : 8;
    Y->stream = static_cast<cudaStream_t>(cuda_stream);
    const size_t n3 = (size_t)N * N * N;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete Y;
        return tl::fail(TL_ECUDA, "cudaMemGetInfo failed (no CUDA device?)");
    }
    const size_t need = 33 * n3 * Y->esz;  // two link buffers (12 values a site each) and the fields (9)
    if (need + (64u << 20) > free_b) {
        delete Y;
        return tl::fail(TL_ENOMEM, "SU(2) lattice needs %zu bytes", need);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&Y->sm_count, cudaDevAttrMultiProcessorCount, dev);
    Y->mblocks = 4 * (Y->sm_count > 0 ? Y->sm_count : 152);
    cudaError_t e = cudaMalloc(&Y->U[0], 12 * n3 * Y->esz);
    if (e == cudaSuccess) e = cudaMalloc(&Y->U[1], 12 * n3 * Y->esz);
    if (e == cudaSuccess) e = cudaMalloc(&Y->E, 9 * n3 * Y->esz);
    if (e == cudaSuccess) e = cudaMalloc(&Y->slots, sizeof(double) * 4 * Y->mblocks);
    if (e == cudaSuccess) e = cudaMalloc(&Y->out, sizeof(double) * 4);
    if (e != cudaSuccess) {
        tl_su2_destroy(Y);
        return tl::fail(TL_ENOMEM, "SU(2) allocation: %s", cudaGetErrorString(e));
    }
    *out = Y;
    return TL_OK;
}

int tl_su2_set_state(tl_su2 *Y, const void *U, const void *E)
{
    tl::set_error(TL_OK, "", "");
    if (!Y || !U || !E) return tl::fail(TL_EINVAL, "NULL argument");
    const size_t n3 = (size_t)Y->N * Y->N * Y->N;
    // host links into the spare buffer, then transposed into records
    SU_CK(cudaMemcpyAsync(Y->U[Y->cur ^ 1], U, 12 * n3 * Y->esz, cudaMemcpyHostToDevice, Y->stream));
    if (Y->dtype == TL_F32)
        su2_to_records<float><<<Y->mblocks, 256, 0, Y->stream>>>(static_cast<const float *>(Y->U[Y->cur ^ 1]),
                                                                 static_cast<float *>(Y->U[Y->cur]), n3);
    else
        su2_to_records<double><<<Y->mblocks, 256, 0, Y->stream>>>(static_cast<const double *>(Y->U[Y->cur ^ 1]),
                                                                  static_cast<double *>(Y->U[Y->cur]), n3);
    SU_CK(cudaGetLastError());
    SU_CK(cudaMemcpyAsync(Y->E, E, 9 * n3 * Y->esz, cudaMemcpyHostToDevice, Y->stream));
    SU_CK(cudaStreamSynchronize(Y->stream));
    Y->has_state = true;
    return TL_OK;
}

int tl_su2_get_state(tl_su2 *Y, void *U, void *E)
{
    tl::set_error(TL_OK, "", "");
    if (!Y || (!U && !E)) return tl::fail(TL_EINVAL, "NULL argument");
    const size_t n3 = (size_t)Y->N * Y->N * Y->N;
    if (U) {  // records transposed into the spare buffer, then copied out
        if (Y->dtype == TL_F32)
            su2_from_records<float><<<Y->mblocks, 256, 0, Y->stream>>>(static_cast<const float *>(Y->U[Y->cur]),
                                                                       static_cast<float *>(Y->U[Y->cur ^ 1]), n3);
        else
            su2_from_records<double><<<Y->mblocks, 256, 0, Y->stream>>>(static_cast<const double *>(Y->U[Y->cur]),
                                                                        static_cast<double *>(Y->U[Y->cur ^ 1]), n3);
        SU_CK(cudaGetLastError());
        SU_CK(cudaMemcpyAsync(U, Y->U[Y->cur ^ 1], 12 * n3 * Y->esz, cudaMemcpyDeviceToHost, Y->stream));
    }
    if (E) SU_CK(cudaMemcpyAsync(E, Y->E, 9 * n3 * Y->esz, cudaMemcpyDeviceToHost, Y->stream));
    SU_CK(cudaStreamSynchronize(Y->stream));
    return TL_OK;
}

int tl_su2_init_random(tl_su2 *Y, uint64_t seed, double amp)
{
    tl::set_error(TL_OK, "", "");
    if (!Y || !(amp >= 0.0)) return tl::fail(TL_EINVAL, "bad argument");
    if (Y->dtype == TL_F32)
        su2_init<float><<<Y->mblocks, 256, 0, Y->stream>>>(static_cast<float *>(Y->U[Y->cur]),
                                                           static_cast<float *>(Y->E), Y->N, seed, amp);
    else
        su2_init<double><<<Y->mblocks, 256, 0, Y->stream>>>(static_cast<double *>(Y->U[Y->cur]),
                                                            static_cast<double *>(Y->E), Y->N, seed, amp);
    SU_CK(cudaGetLastError());
    Y->has_state = true;
    return TL_OK;
}

int tl_su2_step(tl_su2 *Y, int n, double dt)
{
    tl::NvtxScope nvtx_range("tl_su2_step");
    tl::set_error(TL_OK, "", "");
    if (!Y) return tl::fail(TL_EINVAL, "NULL lattice");
    if (n < 0 || !isfinite(dt) || dt == 0.0) return tl::fail(TL_EINVAL, "n >= 0 and a finite nonzero dt needed");
    if (!Y->has_state) return tl::fail(TL_ESTATE, "no state");
    const int N = Y->N;
    const int gx = (N + kSu2Tx - 1) / kSu2Tx, gy = (N + kSu2Ty - 1) / kSu2Ty;
    const size_t smem = Y->dtype == TL_F32 ? su2_tiled_smem<float>() : su2_tiled_smem<double>();
    int per_sm = 0;
    if (Y->dtype == TL_F32) {
        SU_CK(cudaFuncSetAttribute(su2_pass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        SU_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, su2_pass<float>, 256, smem));
    } else {
        SU_CK(cudaFuncSetAttribute(su2_pass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        SU_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, su2_pass<double>, 256, smem));
    }
    // z-chunk: minimise (waves of CTAs) x (planes per CTA + the ~3 planes of
    // halo copies and the first plane's extra plaquettes), i.e. long chunks
    // without a ragged last wave
    const long slots = (long)(Y->sm_count > 0 ? Y->sm_count : 152) * (per_sm > 0 ? per_sm : 1);
    int zc = N;
    long best = -1;
    for (int c = N; c >= 1; --c) {
        const long ctas = (long)gx * gy * ((N + c - 1) / c);
        const long cost = (ctas + slots - 1) / slots * (long)(c + 3);
        if (best < 0 || cost < best) best = cost, zc = c;
    }
    const dim3 grid(gx, gy, (N + zc - 1) / zc);
    for (int k = 0; k < n; ++k) {
        if (Y->dtype == TL_F32)
            su2_pass<float><<<grid, 256, smem, Y->stream>>>(static_cast<const float *>(Y->U[Y->cur]),
                                                            static_cast<float *>(Y->U[Y->cur ^ 1]),
                                                            static_cast<float *>(Y->E), N, zc, (float)dt);
        else
            su2_pass<double><<<grid, 256, smem, Y->stream>>>(static_cast<const double *>(Y->U[Y->cur]),
                                                             static_cast<double *>(Y->U[Y->cur ^ 1]),
                                                             static_cast<double *>(Y->E), N, zc, dt);
        SU_CK(cudaGetLastError());
        Y->cur ^= 1;
    }
    return TL_OK;
}

int tl_su2_measure(tl_su2 *Y, double *out4)
{
    tl::NvtxScope nvtx_range("tl_su2_measure");
    tl::set_error(TL_OK, "", "");
    if (!Y || !out4) return tl::fail(TL_EINVAL, "NULL argument");
    const size_t n3 = (size_t)Y->N * Y->N * Y->N;
    if (Y->dtype == TL_F32)
        su2_measure<float><<<Y->mblocks, 256, 0, Y->stream>>>(static_cast<const float *>(Y->U[Y->cur]),
                                                              static_cast<const float *>(Y->E), Y->N, Y->slots);
    else
        su2_measure<double><<<Y->mblocks, 256, 0, Y->stream>>>(static_cast<const double *>(Y->U[Y->cur]),
                                                               static_cast<const double *>(Y->E), Y->N, Y->slots);
    SU_CK(cudaGetLastError());
    su2_sum_slots<<<1, 32, 0, Y->stream>>>(Y->slots, Y->mblocks, 1.0 / (double)n3, Y->out);
    SU_CK(cudaGetLastError());
    SU_CK(cudaMemcpyAsync(out4, Y->out, 4 * sizeof(double), cudaMemcpyDeviceToHost, Y->stream));
    SU_CK(cudaStreamSynchronize(Y->stream));
    return TL_OK;
}

}  // extern "C"
