// Launch geometry, variant dispatch and the background-reset kernel of the
// fused pass (the kernels themselves are in tl_pass_impl.cuh, instantiated
// per precision in tl_pass_f32.cu and tl_pass_f64.cu).
#include <math.h>

#include "tl_internal.cuh"

namespace tl {

// x^e with integer exponents by repeated squaring (as the pass's finalize does)
__device__ double powe_h(double x, double e)
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

__global__ void set_background_kernel(Model m, Scalars *sc, double a, double b)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (m.expanding) {
        const double al = m.alpha;
        sc->a = a;
        sc->b = b;
        sc->wl = powe_h(a, 1.0 + al);
        sc->wv = powe_h(a, 3.0 + al);
        sc->wk = powe_h(a, -6.0);
        sc->wg = powe_h(a, -2.0);
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

PassGeom pass_geometry(int N, int elem_bytes, int sm_count, int nf, const PassTuning &t)
{
    const int W = 16 / elem_bytes;
    PassGeom g;
    const int per_row = N / W;  // N % 4 == 0 is required, so W | N
    g.variant = t.variant;
    g.cwarps = (t.variant == kVariantTma) ? (t.cwarps == 15 ? 15 : 7) : 8;
    // CTAs of whole warps (the CTA reduction needs them) whose compute threads
    // are laid over a tile of txt x ty threads; leftover threads idle.
    g.threads = (t.variant == kVariantLdg && t.threads == 512) ? 512 : 256;
    const int threads = t.variant == kVariantTma ? 32 * g.cwarps : g.threads;
    const int txt_max = (t.variant == kVariantLdg && (t.txt == 8 || t.txt == 16)) ? t.txt : 32;
    g.txt = per_row < txt_max ? per_row : txt_max;
    g.ty = threads / g.txt;
    if (g.ty > N) g.ty = N;
    const int gx = (per_row + g.txt - 1) / g.txt;
    const int gy = (N + g.ty - 1) / g.ty;
    // z-chunk: long enough to amortise the two extra planes, short enough
    // for several waves of CTAs over the GPU.  FP64 passes are bound by the
    // FP64 pipe, so a small lattice spreads down to one plane per CTA to reach
    // more SMs (the extra halo planes cost loads, not FP64 work); FP32 passes
    // keep at least 4 planes, since for them the halo planes are traffic.
    int zc = t.zc > 0 ? t.zc : (N < 128 ? N : 128);
    if (t.zc <= 0) {
        const long target = 8L * (sm_count > 0 ? sm_count : 152);
        const int zmin = elem_bytes == 8 ? 1 : 4;
        while (zc > zmin && (long)gx * gy * ((N + zc - 1) / zc) < target) zc /= 2;
    }
    if (zc > N) zc = N;
    g.zc = zc;
    g.grid = dim3(gx, gy, (N + zc - 1) / zc);
    g.nblocks = g.grid.x * g.grid.y * g.grid.z;
    g.stages = 0;
    g.smem = 0;
    g.prefetch = 0;
    if (g.variant == kVariantLdg) {
        g.prefetch = (t.prefetch > 0 && g.threads == 256) ? 3 : 0;
        g.smem = (size_t)g.prefetch * nf * 2 * 256 * 16;
    }
    g.lpad = 128 / elem_bytes;
    if (g.variant == kVariantTma) {
        // ring depth: as deep as fits two CTAs per SM (<= 113 KB each), at
        // least 3 (two planes read + one in flight), at most 8; each stage
        // holds 2 nf slots of tma_slot_bytes.
        const size_t per_stage = (size_t)nf * 2 * tma_slot_bytes(g.txt, g.ty);
        int S = t.stages > 0 ? t.stages : 8;
        if (S > 8) S = 8;
        // two CTAs per SM for 7 compute warps, one for 15
        const size_t cap = (t.stages > 0 || g.cwarps > 7 ? 227u : 113u) * 1024u;
        while (S > 3 && per_stage * S > cap) --S;
        g.stages = S;
        g.smem = per_stage * S;
    }
    return g;
}

cudaError_t launch_pass_f32(const Model &m, const FieldPtrs &fp, const PassCoef &c, const PassGeom &g, Scalars *sc,
                            double *slots, bool measure_only, cudaStream_t s, const TmaMaps *maps);
cudaError_t launch_pass_f64(const Model &m, const FieldPtrs &fp, const PassCoef &c, const PassGeom &g, Scalars *sc,
                            double *slots, bool measure_only, cudaStream_t s, const TmaMaps *maps);

cudaError_t launch_pass(int dtype, const Model &m, const FieldPtrs &fp, const PassCoef &c, const PassGeom &g,
                        Scalars *sc, double *slots, bool measure_only, cudaStream_t s, const TmaMaps *maps)
{
    if (m.nf < 1 || m.nf > kMaxFields) return cudaErrorInvalidValue;
    return dtype == TL_F32 ? launch_pass_f32(m, fp, c, g, sc, slots, measure_only, s, maps)
                           : launch_pass_f64(m, fp, c, g, sc, slots, measure_only, s, maps);
}

cudaError_t launch_group_f32(int nf, int variant, int prefetch, int stages, size_t smem, const BatchJob *jobs,
                             const unsigned *first_item, int njobs, unsigned total, const PassCoef &c, int grid,
                             cudaStream_t s);
cudaError_t launch_group_f64(int nf, int variant, int prefetch, int stages, size_t smem, const BatchJob *jobs,
                             const unsigned *first_item, int njobs, unsigned total, const PassCoef &c, int grid,
                             cudaStream_t s);

cudaError_t launch_group(int dtype, int nf, int variant, int prefetch, int stages, size_t smem, const BatchJob *jobs,
                         const unsigned *first_item, int njobs, unsigned total, const PassCoef &c, int grid,
                         cudaStream_t s)
{
    return dtype == TL_F32
               ? launch_group_f32(nf, variant, prefetch, stages, smem, jobs, first_item, njobs, total, c, grid, s)
               : launch_group_f64(nf, variant, prefetch, stages, smem, jobs, first_item, njobs, total, c, grid, s);
}

size_t tma_group_smem(int nf, int stages, int max_txt, int max_ty)
{
    return (size_t)stages * nf * 2 * tma_slot_bytes(max_txt, max_ty);
}

// Refresh the ghost rows of one array (layout in tl_internal.cuh): the rows
// above and below every plane, copies of rows N - 1 and 0.
template <typename T>
__global__ void fill_ghosts_y(T *a, int N, long long P, long long PP)
{
    const long long n = (long long)N * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        T *plane = a + (i / N) * PP;
        const long long x = i % N;
        plane[-P + x] = plane[(long long)(N - 1) * P + x];
        plane[(long long)N * P + x] = plane[x];
    }
}

cudaError_t launch_fill_ghosts(int dtype, void *origin, int N, long long P, long long PP, cudaStream_t s)
{
    const long long n = (long long)N * N;
    const unsigned grid = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    if (dtype == TL_F32)
        fill_ghosts_y<float><<<grid, 256, 0, s>>>(static_cast<float *>(origin), N, P, PP);
    else
        fill_ghosts_y<double><<<grid, 256, 0, s>>>(static_cast<double *>(origin), N, P, PP);
    return cudaGetLastError();
}

cudaError_t launch_set_background(const Model &m, Scalars *sc, double a, double b, cudaStream_t s)
{
    set_background_kernel<<<1, 32, 0, s>>>(m, sc, a, b);
    return cudaGetLastError();
}

}  // namespace tl
