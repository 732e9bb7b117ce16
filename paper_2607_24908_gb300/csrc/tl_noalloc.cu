// tl_energies_noalloc: volume-averaged energies of a caller-owned device
// state with no device allocation at all.
//
// Some callers cannot call cudaMalloc: code embedded in a host framework that
// reserves all device memory up front and hands out only its own buffers,
// and code that must not allocate because cudaMalloc/cudaFree may
// synchronise the device and stall other work in flight.  For them this
// entry point runs the fused pass in measurement mode with its reduction
// scratch (per-CTA partial sums, the arrival ticket and the scalar block) in
// a fixed static device array that every GPU loading this library holds
// until the process exits.
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "tl_internal.cuh"

namespace {

// Scratch capacity: the scalar block plus kMaxSlotBlocks CTA slots of
// kMaxQ doubles.
constexpr size_t kMaxSlotBlocks = 16384;
constexpr size_t kScalarsBytes = (sizeof(tl::Scalars) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kScalarsBytes + kMaxSlotBlocks * tl::kMaxQ * sizeof(double);

// The pass shape of this entry point, fixed here so that its CTA count does
// not follow the library's default shapes: the register-streaming kernel with
// 256-thread CTAs and 32 threads along x (tiles of 32 W x 8 sites, W = 4 FP32
// or 2 FP64 sites per thread), z-chunks of 256 planes from N = 512 up and the
// automatic z-chunk below (at most 128 planes, so at most
// ceil(N/(32 W)) ceil(N/8) ceil(N/128) <= 2048 CTAs for N < 512).
constexpr int kZChunkLarge = 256;

tl::PassTuning noalloc_tuning(int N)
{
    return tl::PassTuning{tl::kVariantLdg, 7, 0, N >= 512 ? kZChunkLarge : 0, 0, 256, 32};
}

constexpr size_t large_blocks(int N, int W)
{
    return (size_t)((N / W + 31) / 32) * (size_t)((N + 7) / 8) * (size_t)((N + kZChunkLarge - 1) / kZChunkLarge);
}
// every lattice up to 1024^3 fits the scratch in both precisions (4096 and 8192 CTAs)
static_assert(large_blocks(1024, 4) <= kMaxSlotBlocks && large_blocks(1024, 2) <= kMaxSlotBlocks,
              "the static scratch must hold the CTA slots of a 1024^3 lattice");

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

int fail(int code, const char *msg, const char *detail = "") { return tl::set_error(code, msg, detail); }

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
int scratch_ptr(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(TL_ECUDA, "cudaGetDevice: ", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(TL_ECUDA, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return fail(TL_ECUDA, "cudaGetSymbolAddress: ", cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return TL_OK;
}

}  // namespace

extern "C" int tl_energies_noalloc(int N, double kIR, int n_fields, tl_dtype dtype, const tl_potential *pot,
                                   const tl_expansion *expansion, double a, const void *const *phi,
                                   const void *const *pi, void *cuda_stream, double *out)
{
    tl::NvtxScope nvtx_range("tl_energies_noalloc");
    tl::set_error(TL_OK, "", "");
    if (N < 8 || N % 4 != 0 || N > 2048) return fail(TL_EINVAL, "N must be a multiple of 4 in [8, 2048]");
    if (!(kIR > 0.0)) return fail(TL_EINVAL, "kIR must be positive");
    if (n_fields < 1 || n_fields > TL_MAX_FIELDS) return fail(TL_EINVAL, "n_fields must be 1..3");
    if (dtype != TL_F32 && dtype != TL_F64) return fail(TL_EINVAL, "unknown dtype");
    if (!pot || !phi || !pi || !out) return fail(TL_EINVAL, "NULL argument");
    if (!(a > 0.0)) return fail(TL_EINVAL, "a must be positive");
    for (int f = 0; f < n_fields; ++f)
        if (!phi[f] || !pi[f] || ((uintptr_t)phi[f] & 15u) || ((uintptr_t)pi[f] & 15u))
            return fail(TL_EINVAL, "field pointers must be non-NULL and 16-byte aligned");

    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(TL_ECUDA, "device query: ", cudaGetErrorString(e));
    // dense caller arrays have no ghost layer for tiled copies: the streaming kernel
    const tl::PassGeom g = tl::pass_geometry(N, dtype == TL_F32 ? 4 : 8, sms, n_fields, noalloc_tuning(N));
    if (g.nblocks > kMaxSlotBlocks)
        return fail(TL_EINVAL, "lattice needs more reduction slots than the static scratch holds (max 16384 CTAs)");

    void *base = nullptr;
    int rc = scratch_ptr(&base);
    if (rc) return rc;
    tl::Scalars *sc = static_cast<tl::Scalars *>(base);
    double *slots = reinterpret_cast<double *>(static_cast<unsigned char *>(base) + kScalarsBytes);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    tl::Model m{};
    m.N = N;
    m.nf = n_fields;
    m.ghosts = 0;  // caller arrays are dense: pitch N, plane N^2
    m.pitch = N;
    m.pplane = (long long)N * N;
    m.expanding = (expansion && expansion->expanding) ? 1 : 0;
    m.alpha = m.expanding ? expansion->alpha : 0.0;
    m.mu2 = m.expanding ? expansion->fstar_over_mp * expansion->fstar_over_mp : 1.0;
    const double dx = 2.0 * M_PI / (kIR * N);
    m.inv_dx2 = 1.0 / (dx * dx);
    m.lambda = pot->lambda;
    m.q = pot->q;
    for (int f = 0; f < TL_MAX_FIELDS; ++f) m.m2[f] = pot->m2[f];

    // The scratch keeps the previous call's contents: reset the scalar block
    // (ticket, status, weights for a) before the pass.
    e = cudaMemsetAsync(sc, 0, sizeof(tl::Scalars), s);
    if (e == cudaSuccess) e = tl::launch_set_background(m, sc, a, 0.0, s);
    tl::FieldPtrs fp{};
    for (int f = 0; f < n_fields; ++f) {
        fp.phi_in[f] = phi[f];
        fp.pi_in[f] = pi[f];
    }
    tl::PassCoef c{};
    c.integer_time = 1;
    if (e == cudaSuccess) e = tl::launch_pass((int)dtype, m, fp, c, g, sc, slots, true, s);
    tl::Scalars h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(TL_ECUDA, "energy pass: ", cudaGetErrorString(e));
    for (int i = 0; i < 2 * n_fields + 1; ++i) out[i] = h.E[i];
    if (h.status == TL_ETIMEOUT) return fail(TL_ETIMEOUT, "a bounded device wait expired");
    if (h.status != TL_OK) return fail(TL_EUNSTABLE, "energies are not finite");
    return TL_OK;
}
