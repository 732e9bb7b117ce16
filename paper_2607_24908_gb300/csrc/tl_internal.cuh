// Internal declarations shared by the CUDA translation units of libtl.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/tl.h"

namespace tl {

// A named NVTX range over a scope: the library's public calls show on a
// profiler's timeline (nvtx3 is header-only; with no tool attached a push or
// pop is a test of one function pointer).
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};

constexpr int kMaxFields = TL_MAX_FIELDS;
constexpr int kMaxQ = 2 * kMaxFields + 1;  // K_f, G_f, V

// Device-resident scalars of one lattice (always FP64).  The fused pass reads
// the coefficients for its own evaluation time (a, drift, weights) and its
// last CTA writes those of the next pass.
struct Scalars {
    double a;          // scale factor at the time of the next field evaluation
    double b;          // a'
    double drift;      // the next pass's drift: d dt ((a_prev + a)/2)^(alpha-3)
    double pending_dt; // program time the next pass's drift advances
    double wl, wv;     // a^(1+alpha), a^(3+alpha)
    double wk, wg;     // a^-6, a^-2
    double E[kMaxQ];   // K_f, G_f, V at the last evaluated time
    double hubble;     // Hubble residual at the last integer time
    double time;       // program time of the last evaluation
    int status;        // TL_OK or TL_EUNSTABLE
    unsigned ticket;   // CTAs of the current pass that finished their slot
};

// Scalar constants of a lattice/model passed by value to every pass.
// Field arrays are addressed from their element (0, 0, 0) as
// z * pplane + y * pitch + x.  A dense array has pitch = N, pplane = N^2;
// the lattice's own arrays carry ghost rows (ghosts = 1): one row above and
// below every z-plane, copies of rows N - 1 and 0 that every pass keeps
// current for the sites it writes, and W = 16/sizeof(T) reserved elements
// left and right of every row (x in [-W, 0) and [N, N + W); not kept: the TMA
// pass takes the x-halo at the lattice's x-edges from the periodic image);
// rows are padded to a multiple of 128 bytes with x = 0 on a 128-byte
// boundary, pplane = (N + 2) pitch.
struct Model {
    int N;
    int nf;
    int expanding;
    int ghosts;
    long long pitch;
    long long pplane;
    double alpha;
    double mu2;
    double inv_dx2;
    double lambda, q;
    double m2[kMaxFields];
};

// Coefficients of one fused pass, in units of dt already multiplied in.
struct PassCoef {
    double kdt;       // pi_new = pi_s + kdt F
    double hdt;       // pi_int = pi_s + hdt F (momentum at the evaluation time, for K)
    double edt;       // b += edt a''
    double hb_dt;     // b at the evaluation time: b_old + hb_dt a'' (Hubble residual)
    double dnext_dt;  // drift of the following pass (and a += dnext_dt b)
    int integer_time; // the evaluation time is a whole step: record the Hubble residual
    int set_b_from_constraint; // measurement pass after a new state: b from the constraint
};

struct FieldPtrs {
    const void *phi_in[kMaxFields];
    const void *pi_in[kMaxFields];
    void *phi_out[kMaxFields];
    void *pi_out[kMaxFields];
};

// Fused-pass variants: per-thread loads through L1/L2, or z-planes of a
// ghost-padded tile staged in shared memory by tiled TMA copies.
constexpr int kVariantLdg = 0;
constexpr int kVariantTma = 1;

// Tunable launch parameters of the fused pass (0 = choose automatically).
struct PassTuning {
    int variant;  // kVariantLdg or kVariantTma
    int cwarps;   // tma: compute warps per CTA (7 or 15; one producer warp is added)
    int stages;   // bulk: shared-memory ring depth in z-planes (3..8)
    int zc;       // z-planes per CTA
    int prefetch; // ldg: planes prefetched per thread with cp.async (0 or 3)
    int threads;  // ldg: threads per CTA, 256 (default) or 512
    int txt;      // ldg: threads along x per tile row, 32 (default), 16 or 8
};

// Tensor maps of the input arrays of a TMA pass: map[k][2 f + a], a = 0 phi,
// 1 pi, each 3-D over the padded array (x incl. pads, rows incl. ghost rows,
// planes), one plane deep and ty + 2 rows high, txt W + 2W sites wide for
// k = kMapTile (a tile with its x-halo: tiles inside the lattice), txt W for
// kMapBody (the tile alone) and W for kMapSide (one halo column: tiles at an
// x-edge of the lattice, whose halo on the far side of the edge is the
// periodic image).
constexpr int kMapTile = 0, kMapBody = 1, kMapSide = 2;
struct TmaMaps {
    CUtensorMap map[3][2 * kMaxFields];
};

// Bytes of one array's slot in a stage of the TMA ring (128-byte aligned
// parts; W sizeof(T) = 16 bytes in both precisions): a tile-plus-halo box
// ((ty + 2) x (txt + 2) 16-byte words), or at an x-edge the body box
// ((ty + 2) x txt words) followed by the left and right halo columns
// ((ty + 2) words each) at tma_side_offset(.., 0) and (.., 1).
__host__ __device__ constexpr size_t tma_r128(size_t b) { return (b + 127) / 128 * 128; }
__host__ __device__ constexpr size_t tma_side_offset(int txt, int ty, int side)
{
    return side == 0 ? tma_r128((size_t)(ty + 2) * txt * 16)
                     : tma_r128(tma_r128((size_t)(ty + 2) * txt * 16) + (size_t)(ty + 2) * 16);
}
__host__ __device__ constexpr size_t tma_slot_bytes(int txt, int ty)
{
    return tma_r128((size_t)(ty + 2) * (txt + 2) * 16 > tma_side_offset(txt, ty, 1) + (size_t)(ty + 2) * 16
                        ? (size_t)(ty + 2) * (txt + 2) * 16
                        : tma_side_offset(txt, ty, 1) + (size_t)(ty + 2) * 16);
}
// The slot layout, checked for every tile the pass can have (txt up to 32
// threads along x, ty up to 64 rows): the tile-plus-halo box fits the slot,
// and so do the body and the two halo columns after it, each part on a
// 128-byte boundary and the columns clear of the body and of each other.
constexpr bool tma_slot_layout_holds()
{
    for (int txt = 1; txt <= 32; ++txt)
        for (int ty = 1; ty <= 64; ++ty) {
            const size_t slot = tma_slot_bytes(txt, ty), l = tma_side_offset(txt, ty, 0),
                         r = tma_side_offset(txt, ty, 1), col = (size_t)(ty + 2) * 16;
            if (slot % 128 || l % 128 || r % 128) return false;
            if ((size_t)(ty + 2) * (txt + 2) * 16 > slot) return false;
            if ((size_t)(ty + 2) * txt * 16 > l || l + col > r || r + col > slot) return false;
        }
    return true;
}
static_assert(tma_slot_layout_holds(), "TMA stage slots must hold every tile's copies on 128-byte boundaries");
static_assert(tma_slot_bytes(32, 15) == 9472 && tma_slot_bytes(32, 7) == 5120,
              "slot sizes of the default tiles (two-field ring: 6 x 37.9 KB and 5 x 20.5 KB)");

// Launch geometry of the fused pass.
struct PassGeom {
    int txt;  // threads along x (each owns VEC consecutive sites)
    int ty;   // threads along y (one row each)
    int zc;   // z-planes per CTA
    dim3 grid;
    unsigned nblocks;
    int variant;   // kVariantLdg or kVariantTma
    int cwarps;    // compute warps per CTA
    int stages;    // shared-memory ring depth (TMA variant)
    int prefetch;  // per-thread prefetch depth (ldg variant)
    int lpad;      // TMA variant: padded-row index of x = 0 (128 bytes / element size)
    int threads;   // threads per CTA (ldg variant)
    size_t smem;   // dynamic shared memory per CTA
};

PassGeom pass_geometry(int N, int elem_bytes, int sm_count, int nf, const PassTuning &t);

// Tuning from the environment (TL_PASS_VARIANT=ldg|bulk, TL_PREFETCH, TL_LDG_THREADS, TL_LDG_TXT,
// TL_BULK_WARPS, TL_BULK_STAGES, TL_PASS_ZC), else the built-in defaults.
// Launch shape a new lattice starts with: the TMA pass for FP32 from N = 192
// up (z-chunks of 16 planes at 192, 64 above; 15 + 1 warps from N = 768),
// where it measured faster; the streaming pass otherwise (FP64 is bound by
// FP64 arithmetic, small lattices by latency).
PassTuning default_tuning(int N, int nf, int elem_bytes);

// One lattice of a batched (grouped) launch: its model, fields for this pass,
// scalars, reduction slots and its own launch geometry.
struct BatchJob {
    Model m;
    FieldPtrs fp;
    Scalars *sc;
    double *slots;
    int txt, ty, zc, gx, gy;
    unsigned nblocks;
    int lpad;              // TMA variant: padded-row index of x = 0
    const TmaMaps *maps;   // TMA variant: tensor maps of this pass's input arrays (global memory)
};

// Enqueue one grouped pass over every job (all with n_fields == nf).
// variant kVariantLdg: a persistent launch of `grid` CTAs of 256 threads
// walking the (job, tile) items of the register-streaming pass; prefetch > 0
// runs the variant whose threads prefetch their words three planes ahead
// (cp.async), the same arithmetic.  variant kVariantTma: one CTA of 7 + 1 warps
// per item (`total` CTAs) of the TMA pass, `stages` ring stages in `smem`
// bytes of dynamic shared memory.
cudaError_t launch_group(int dtype, int nf, int variant, int prefetch, int stages, size_t smem, const BatchJob *jobs,
                         const unsigned *first_item, int njobs, unsigned total, const PassCoef &c, int grid,
                         cudaStream_t s);

// Shared memory a TMA group launch needs: `stages` stages of 2 nf slots
// (tma_slot_bytes) for the largest txt and ty among its jobs.
size_t tma_group_smem(int nf, int stages, int max_txt, int max_ty);

// Enqueue one fused pass (measure_only: energies of the stored state, no writes).
cudaError_t launch_pass(int dtype, const Model &m, const FieldPtrs &fp, const PassCoef &c, const PassGeom &g,
                        Scalars *sc, double *slots, bool measure_only, cudaStream_t s,
                        const TmaMaps *maps = nullptr);

// Record msg+detail as this thread's tl_last_error() text; returns code.
int set_error(int code, const char *msg, const char *detail);

// Refresh the ghost rows of one padded array from its interior.
cudaError_t launch_fill_ghosts(int dtype, void *origin, int N, long long P, long long PP, cudaStream_t s);

// Set a, b (and the derived weights) on the device; drift = 0.
cudaError_t launch_set_background(const Model &m, Scalars *sc, double a, double b, cudaStream_t s);

}  // namespace tl
