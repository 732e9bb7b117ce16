// The lattice object behind the opaque tl_lattice handle (host side).
#pragma once

#include <cufft.h>
#include <stdint.h>

#include <vector>

#include "tl_internal.cuh"

struct tl_lattice {
    int N = 0, nf = 0;
    double kIR = 0.0, dx = 0.0;
    tl_dtype dtype = TL_F32;
    size_t esz = 0;
    tl_expansion ex{};
    tl_potential pot{};
    bool has_pot = false;
    unsigned state_mask = 0;  // bit 2 f + which: that array was set
    bool has_state = false;
    cudaStream_t stream = nullptr;
    bool own = false;
    void *base = nullptr;           // owned field memory
    void *buf[2][2][TL_MAX_FIELDS]; // [parity][phi, pi][field]
    int cur = 0;
    tl::Scalars *d_sc = nullptr;
    double *d_slots = nullptr;
    unsigned slots_cap = 0;       // CTA slots d_slots holds
    tl::PassTuning tuning{};      // launch parameters in use
    tl::TmaMaps maps[2];          // tensor maps of the arrays of parity 0 / 1 (TMA variant)
    int maps_txt = -1, maps_ty = -1;  // tile shape the maps were encoded for
    tl::PassGeom geom{};
    tl::Model model{};
    int sm_count = 0;
    int64_t step = 0;
    int64_t langevin_steps = 0;  // Langevin steps since the last state reset (noise counters)
    bool energies_valid = false;
    int batch_refs = 0;  // tl_batch objects that hold this lattice
    // Bumped whenever something a captured pass sequence bakes in changes: the
    // launch shape, the model (potential, expansion), the buffer assignment.
    unsigned version = 0;
    // tl_step's replayable pass sequences (see tl_step), newest last.
    struct StepGraph {
        int n, integrator, cur;
        double dt;
        unsigned version;
        cudaGraphExec_t exec;  // null until the key repeats
    };
    std::vector<StepGraph> graphs;
    cudaStream_t capture = nullptr;  // private stream the sequences are captured on
};

namespace tl {
// Padded array layout (see tl_internal.cuh): W = 16/esz ghost elements on
// each side of a row (the left ones inside a 128-byte pad so that x = 0 of
// every row starts a 128-byte line), rows padded to a multiple of 128 bytes,
// one ghost row on each side of a plane, no z ghosts.
struct Layout {
    long long W, lpad, pitch, pplane;
    size_t elems, origin;
};
inline Layout layout_of(int N, size_t esz)
{
    Layout l;
    const long long line = (long long)(128 / esz);
    l.W = (long long)(16 / esz);
    l.lpad = line;
    l.pitch = (l.lpad + N + l.W + line - 1) / line * line;
    l.pplane = (long long)(N + 2) * l.pitch;
    l.elems = (size_t)N * (size_t)l.pplane;
    l.origin = (size_t)(l.pitch + l.lpad);
    return l;
}


// Launch one fused pass of a lattice on its stream and flip its buffers.
int lattice_launch(tl_lattice *L, const PassCoef &c, bool measure_only);
// Record an error message for tl_last_error(); returns code.
int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
// Coefficients of the n P + 1 passes of n steps (false: unknown integrator).
bool pass_schedule(int n, double dt, int integrator, std::vector<PassCoef> &out);
// Drop tl_step's captured pass sequences and bump the lattice version (call
// after any change to what a pass launch bakes in).
void invalidate_launches(tl_lattice *L);
// Switch a lattice to launch shape t (grows its reduction slots if needed and
// re-encodes tensor maps at the next TMA launch).
int set_geometry(tl_lattice *L, const PassTuning &t);
// Encode (if needed) the tensor maps of L's arrays for its current tile shape;
// L->maps[p] then holds those of the arrays of buffer parity p.
int lattice_tma_maps(tl_lattice *L);
}  // namespace tl
