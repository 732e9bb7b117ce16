// Host runtime behind include/tl.h: lattice objects, the integrator schedule
// (pass list), launches, state transfer, initial fields and spectra.
#include <cufft.h>
#include <math.h>
#include <stddef.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <tuple>
#include <mutex>
#include <new>
#include <vector>

#include "tl_fourier.cuh"
#include "tl_internal.cuh"
#include "tl_lattice.cuh"

using tl::FieldPtrs;
using tl::Model;
using tl::PassCoef;
using tl::PassGeom;
using tl::Scalars;

using tl::fail;

namespace {

thread_local char g_err[512] = "";

#define TL_CK(call)                                                                                 \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(e_ == cudaErrorMemoryAllocation ? TL_ENOMEM : TL_ECUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                \
    } while (0)

#define TL_CKFFT(call)                                                                              \
    do {                                                                                            \
        cufftResult r_ = (call);                                                                    \
        if (r_ != CUFFT_SUCCESS) return fail(TL_ECUDA, "%s: cufft error %d", #call, (int)r_);      \
    } while (0)

}  // namespace

tl::PassTuning tl::default_tuning(int N, int nf, int elem_bytes)
{
    tl::PassTuning t{elem_bytes == 4 && N >= 192 ? tl::kVariantTma : tl::kVariantLdg, 7, 0, 0, 0, 256, 0};
    // environment overrides (tuning experiments)
    const char *v = getenv("TL_PASS_VARIANT");
    if (v && strcmp(v, "tma") == 0) t.variant = tl::kVariantTma;
    if (v && strcmp(v, "ldg") == 0) t.variant = tl::kVariantLdg;
    const char *cw = getenv("TL_BULK_WARPS"), *zc = getenv("TL_PASS_ZC");
    if (t.variant == tl::kVariantTma) {  // measured: long z-chunks for the ring, 15 + 1 warps from 416
        // warps x z-chunk sweeps of the current kernel (FP32, ms per pass, one / two fields):
        // 192^3 48 planes 0.083 two fields (16: 0.091); 384^3 7 + 1 warps, 56 planes 0.205 /
        // 0.325; 448^3 15 + 1, 80 planes 0.524 two fields (96: 0.531); 512^3 15 + 1, 160
        // planes 0.417 one field, 96 planes 0.705 two (160: 0.714); 576^3 ... 768^3 104
        // planes (640^3 1.330, 768^3 2.297 two fields); 896^3 72 planes 3.623 (92: 3.634);
        // 1024^3 76 planes 5.380 (92: 5.391).  The optimum is jagged in the chunk count, so
        // each measured size sets the value for the sizes around it.
        if (N <= 192) t.zc = 48;
        else if (N < 320) t.zc = 64;
        else if (N < 416) t.zc = 56;
        else if (N < 480) t.zc = 80;
        else if (N < 544) t.zc = nf == 1 ? 160 : 96;
        else if (N < 832) t.zc = 104;
        else if (N < 960) t.zc = 72;
        else t.zc = 76;
        t.cwarps = N >= 416 ? 15 : 7;
    } else if (elem_bytes == 8 && N >= 128) {
        // FP64 streaming pass (bound by the FP64 pipe): 32-plane chunks from 128^3 (one and two
        // fields, 128^3 ... 384^3: 0.7316 ms at 256^3 against 0.7465 with the 16 of the automatic
        // rule), 64 from 512^3 (5.465 vs 5.525 ms); tile row widths 8, 16, 32 measured alike.
        // Smaller FP64 lattices keep the automatic rule, which spreads them over more SMs.
        t.zc = N >= 512 ? 64 : 32;
    }
    if ((v = getenv("TL_PREFETCH"))) t.prefetch = atoi(v);
    if ((v = getenv("TL_LDG_THREADS"))) t.threads = atoi(v);
    if ((v = getenv("TL_LDG_TXT"))) t.txt = atoi(v);
    if (cw) t.cwarps = atoi(cw);
    if ((v = getenv("TL_BULK_STAGES"))) t.stages = atoi(v);
    if (zc) t.zc = atoi(zc);
    return t;
}

// Pass list of n steps from a synchronised state (phi_n, pi_n, a_n, b_n):
// substep sizes s_1..s_M (M = n P) in units of dt; pass 0 half-kicks with
// s_1, pass j (0 < j < M) closes substep j and opens j+1 (merged kicks
// (s_j + s_{j+1})/2), pass M closes substep M with a half kick.  Each pass
// evaluates at the boundary after its deferred drift; hdt/hb_dt bring pi and
// b to that boundary for the energies and the Hubble residual.
bool tl::pass_schedule(int n, double dt, int integrator, std::vector<PassCoef> &out)
{
    double w[3];
    int P;
    if (integrator == TL_LEAPFROG || integrator == TL_VERLET) {
        w[0] = 1.0;
        P = 1;
    } else if (integrator == TL_YOSHIDA4) {
        const double cr = cbrt(2.0);
        w[0] = w[2] = 1.0 / (2.0 - cr);
        w[1] = -cr / (2.0 - cr);
        P = 3;
    } else {
        return false;
    }
    const long M = (long)n * P;
    out.clear();
    out.reserve(M + 1);
    for (long j = 0; j <= M; ++j) {
        const double s_prev = j > 0 ? w[(j - 1) % P] : 0.0;
        const double s_next = j < M ? w[j % P] : 0.0;
        PassCoef c{};
        c.kdt = 0.5 * (s_prev + s_next) * dt;
        c.hdt = 0.5 * s_prev * dt;
        c.edt = 0.5 * (s_prev + s_next) * dt;
        c.hb_dt = 0.5 * s_prev * dt;
        c.dnext_dt = s_next * dt;
        c.integer_time = (j % P == 0) ? 1 : 0;
        out.push_back(c);
    }
    return true;
}

int tl::fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int tl::set_error(int code, const char *msg, const char *detail)
{
    snprintf(g_err, sizeof g_err, "%s%s", msg, detail);
    return code;
}


namespace {

size_t n3_of(int N) { return (size_t)N * (size_t)N * (size_t)N; }

// Bytes between consecutive field arrays beyond their size (TL_ARRAY_STAGGER,
// rounded to 256 bytes; default 0).
size_t array_stagger()
{
    const char *v = getenv("TL_ARRAY_STAGGER");
    long b = v ? atol(v) : 0;
    if (b < 0) b = 0;
    return (size_t)((b + 255) / 256 * 256);
}

int check_dims(int N, double kIR, int n_fields, tl_dtype dtype, const tl_expansion *ex)
{
    if (N < 8 || N % 4 != 0 || N > 2048) return fail(TL_EINVAL, "N must be a multiple of 4 in [8, 2048], got %d", N);
    if (!(kIR > 0.0) || !isfinite(kIR)) return fail(TL_EINVAL, "kIR must be positive and finite");
    if (n_fields < 1 || n_fields > TL_MAX_FIELDS) return fail(TL_EINVAL, "n_fields must be 1..%d", TL_MAX_FIELDS);
    if (dtype != TL_F32 && dtype != TL_F64) return fail(TL_EINVAL, "unknown dtype %d", (int)dtype);
    if (ex && ex->expanding) {
        if (!isfinite(ex->alpha)) return fail(TL_EINVAL, "alpha must be finite");
        if (!(ex->a0 > 0.0)) return fail(TL_EINVAL, "a0 must be positive");
        if (!(ex->fstar_over_mp > 0.0)) return fail(TL_EINVAL, "fstar_over_mp must be positive");
    }
    return TL_OK;
}

void refresh_model(tl_lattice *L)
{
    Model &m = L->model;
    const tl::Layout lay = tl::layout_of(L->N, L->esz);
    m.N = L->N;
    m.nf = L->nf;
    m.ghosts = 1;
    m.pitch = lay.pitch;
    m.pplane = lay.pplane;
    m.expanding = L->ex.expanding ? 1 : 0;
    m.alpha = L->ex.alpha;
    m.mu2 = L->ex.fstar_over_mp * L->ex.fstar_over_mp;
    m.inv_dx2 = 1.0 / (L->dx * L->dx);
    m.lambda = L->pot.lambda;
    m.q = L->pot.q;
    for (int f = 0; f < TL_MAX_FIELDS; ++f) m.m2[f] = L->pot.m2[f];
    tl::invalidate_launches(L);
}

int finish_create(tl_lattice *L, int N, double kIR, int nf, tl_dtype dtype, const tl_expansion *ex, void *stream)
{
    L->N = N;
    L->nf = nf;
    L->kIR = kIR;
    L->dx = 2.0 * M_PI / (kIR * N);
    L->dtype = dtype;
    L->esz = dtype == TL_F32 ? 4 : 8;
    if (ex) L->ex = *ex;
    if (!L->ex.expanding) {
        L->ex.alpha = 0.0;
        L->ex.a0 = 1.0;
        L->ex.fstar_over_mp = L->ex.fstar_over_mp > 0 ? L->ex.fstar_over_mp : 1.0;
    }
    L->stream = static_cast<cudaStream_t>(stream);
    int dev = 0;
    TL_CK(cudaGetDevice(&dev));
    TL_CK(cudaDeviceGetAttribute(&L->sm_count, cudaDevAttrMultiProcessorCount, dev));
    L->tuning = tl::default_tuning(N, nf, (int)L->esz);
    L->geom = tl::pass_geometry(N, (int)L->esz, L->sm_count, nf, L->tuning);
    TL_CK(cudaMalloc(&L->d_sc, sizeof(Scalars)));
    TL_CK(cudaMemsetAsync(L->d_sc, 0, sizeof(Scalars), L->stream));
    TL_CK(cudaMalloc(&L->d_slots, sizeof(double) * tl::kMaxQ * L->geom.nblocks));
    L->slots_cap = L->geom.nblocks;
    refresh_model(L);
    TL_CK(tl::launch_set_background(L->model, L->d_sc, L->ex.a0, 0.0, L->stream));
    return TL_OK;
}

int launch(tl_lattice *L, const PassCoef &c, bool measure_only, cudaStream_t stream);
int launch(tl_lattice *L, const PassCoef &c, bool measure_only) { return launch(L, c, measure_only, L->stream); }
int launch(tl_lattice *L, const PassCoef &c, bool measure_only, cudaStream_t stream)
{
    const tl::TmaMaps *maps = nullptr;
    if (L->geom.variant == tl::kVariantTma) {
        int rc = tl::lattice_tma_maps(L);
        if (rc) return rc;
        maps = &L->maps[L->cur];
    }
    FieldPtrs fp;
    for (int f = 0; f < TL_MAX_FIELDS; ++f) {
        fp.phi_in[f] = L->buf[L->cur][0][f];
        fp.pi_in[f] = L->buf[L->cur][1][f];
        fp.phi_out[f] = L->buf[L->cur ^ 1][0][f];
        fp.pi_out[f] = L->buf[L->cur ^ 1][1][f];
    }
    TL_CK(tl::launch_pass((int)L->dtype, L->model, fp, c, L->geom, L->d_sc, L->d_slots, measure_only, stream, maps));
    if (!measure_only) L->cur ^= 1;
    return TL_OK;
}

int measure(tl_lattice *L, bool b_from_constraint)
{
    PassCoef c{};
    c.integer_time = 1;
    c.set_b_from_constraint = b_from_constraint ? 1 : 0;
    int rc = launch(L, c, true);
    if (rc) return rc;
    L->energies_valid = true;
    return TL_OK;
}

int read_scalars(tl_lattice *L, Scalars *h)
{
    TL_CK(cudaMemcpyAsync(h, L->d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, L->stream));
    TL_CK(cudaStreamSynchronize(L->stream));
    return TL_OK;
}

// Dense host array [z][y][x] <-> padded device array: one 3-D copy (rows of
// N elements; device rows `pitch` apart, planes N + 2 rows apart).
int copy_planes(tl_lattice *L, void *host, void *dev, bool to_device)
{
    const size_t N = (size_t)L->N, esz = L->esz;
    const size_t dpitch = (size_t)L->model.pitch * esz;
    const size_t rows_per_plane = (size_t)L->model.pplane / (size_t)L->model.pitch;  // N + 2
    cudaMemcpy3DParms p = {};
    p.extent = make_cudaExtent(N * esz, N, N);
    const cudaPitchedPtr h = make_cudaPitchedPtr(host, N * esz, N * esz, N);
    const cudaPitchedPtr d = make_cudaPitchedPtr(dev, dpitch, N * esz, rows_per_plane);
    p.srcPtr = to_device ? h : d;
    p.dstPtr = to_device ? d : h;
    p.kind = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    TL_CK(cudaMemcpy3DAsync(&p, L->stream));
    return TL_OK;
}

int check_field(const tl_lattice *L, int field, int which)
{
    if (!L) return fail(TL_EINVAL, "NULL lattice");
    if (field < 0 || field >= L->nf) return fail(TL_EINVAL, "field %d out of range (n_fields %d)", field, L->nf);
    if (which != 0 && which != 1) return fail(TL_EINVAL, "which must be 0 (phi) or 1 (pi)");
    return TL_OK;
}

// cuFFT plans shared by all lattices of a size on a device (planning costs
// milliseconds and a workspace per plan).  Under this mutex a plan is bound
// to the caller's stream, which first waits for the plan's previous
// executions (on whatever stream they were enqueued) through the plan's
// event; the caller records that event after its last execution.  Calls that
// use a plan therefore only enqueue work: no host wait guards the workspace.
struct SharedPlan {
    cufftHandle h;
    cudaEvent_t done;  // recorded after the latest enqueued execution
};
std::mutex g_plan_mu;
std::map<std::tuple<int, int, int>, SharedPlan> g_plans;  // (device, N, cufftType) -> plan

int shared_plan(int N, cufftType type, cudaStream_t s, SharedPlan **out)
{
    int dev = 0;
    TL_CK(cudaGetDevice(&dev));
    auto key = std::make_tuple(dev, N, (int)type);
    auto it = g_plans.find(key);
    if (it == g_plans.end()) {
        SharedPlan p{};
        cufftResult r = cufftPlan3d(&p.h, N, N, N, type);
        if (r != CUFFT_SUCCESS) return fail(TL_ECUDA, "cufftPlan3d(%d) failed (%d)", N, (int)r);
        cudaError_t e = cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cufftDestroy(p.h);
            return fail(TL_ECUDA, "cudaEventCreateWithFlags: %s", cudaGetErrorString(e));
        }
        it = g_plans.emplace(key, p).first;
    }
    TL_CKFFT(cufftSetStream(it->second.h, s));
    TL_CK(cudaStreamWaitEvent(s, it->second.done, 0));  // a never-recorded event: no wait
    *out = &it->second;
    return TL_OK;
}

}  // namespace

int tl::lattice_launch(tl_lattice *L, const PassCoef &c, bool measure_only) { return launch(L, c, measure_only); }

int tl::set_geometry(tl_lattice *L, const PassTuning &t)
{
    const PassGeom g = pass_geometry(L->N, (int)L->esz, L->sm_count, L->nf, t);
    if (g.nblocks > L->slots_cap) {
        double *p = nullptr;
        TL_CK(cudaStreamSynchronize(L->stream));
        TL_CK(cudaMalloc(&p, sizeof(double) * kMaxQ * g.nblocks));
        cudaFree(L->d_slots);
        L->d_slots = p;
        L->slots_cap = g.nblocks;
    }
    L->geom = g;
    L->tuning = t;
    invalidate_launches(L);  // re-encodes tensor maps for the new tile shape too
    return TL_OK;
}

void tl::invalidate_launches(tl_lattice *L)
{
    for (auto &g : L->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    L->graphs.clear();
    L->maps_txt = L->maps_ty = -1;
    ++L->version;
}

extern "C" {

const char *tl_last_error(void) { return g_err; }

size_t tl_state_bytes(int N, int n_fields, tl_dtype dtype)
{
    if (N <= 0 || n_fields <= 0) return 0;
    const size_t esz = dtype == TL_F64 ? 8 : 4;
    return 4 * (size_t)n_fields * tl::layout_of(N, esz).elems * esz;
}

int tl_array_layout(int N, tl_dtype dtype, size_t *elems, size_t *row_pitch, size_t *plane_pitch, size_t *origin)
{
    if (N < 8 || N % 4 != 0 || (dtype != TL_F32 && dtype != TL_F64)) return fail(TL_EINVAL, "bad N or dtype");
    const tl::Layout l = tl::layout_of(N, dtype == TL_F64 ? 8 : 4);
    if (elems) *elems = l.elems;
    if (row_pitch) *row_pitch = (size_t)l.pitch;
    if (plane_pitch) *plane_pitch = (size_t)l.pplane;
    if (origin) *origin = l.origin;
    return TL_OK;
}

int tl_lattice_create(tl_lattice **out, int N, double kIR, int n_fields, tl_dtype dtype,
                      const tl_expansion *expansion, void *cuda_stream)
{
    g_err[0] = 0;
    if (!out) return fail(TL_EINVAL, "NULL out");
    *out = nullptr;
    int rc = check_dims(N, kIR, n_fields, dtype, expansion);
    if (rc) return rc;
    tl_lattice *L = new (std::nothrow) tl_lattice();
    if (!L) return fail(TL_ENOMEM, "host allocation failed");
    // Arrays are staggered by a few KiB so that the 4 n_fields streams of a
    // pass do not sit at identical offsets modulo large powers of two.
    const size_t stagger = array_stagger();
    const size_t bytes = tl_state_bytes(N, n_fields, dtype) + 4 * (size_t)n_fields * stagger;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete L;
        return fail(TL_ECUDA, "cudaMemGetInfo failed (no CUDA device?)");
    }
    if (bytes + (64u << 20) > free_b) {
        delete L;
        return fail(TL_ENOMEM, "lattice needs %zu bytes, %zu free on the device", bytes, free_b);
    }
    if (cudaMalloc(&L->base, bytes) != cudaSuccess) {
        delete L;
        return fail(TL_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
    }
    L->own = true;
    const size_t esz = dtype == TL_F64 ? 8 : 4;
    const tl::Layout lay = tl::layout_of(N, esz);
    const size_t arr = lay.elems * esz;
    char *p = static_cast<char *>(L->base);
    memset(L->buf, 0, sizeof L->buf);
    for (int f = 0; f < n_fields; ++f)
        for (int par = 0; par < 2; ++par)
            for (int w = 0; w < 2; ++w) {
                const size_t k = (size_t)(4 * f + 2 * par + w);
                L->buf[par][w][f] = p + k * (arr + stagger) + lay.origin * esz;
            }
    rc = finish_create(L, N, kIR, n_fields, dtype, expansion, cuda_stream);
    if (rc) {
        tl_lattice_destroy(L);
        return rc;
    }
    *out = L;
    return TL_OK;
}

int tl_lattice_create_with_buffers(tl_lattice **out, int N, double kIR, int n_fields, tl_dtype dtype,
                                   const tl_expansion *expansion, void *cuda_stream, void *const *dev_ptrs,
                                   size_t n_ptrs)
{
    g_err[0] = 0;
    if (!out) return fail(TL_EINVAL, "NULL out");
    *out = nullptr;
    int rc = check_dims(N, kIR, n_fields, dtype, expansion);
    if (rc) return rc;
    if (!dev_ptrs || n_ptrs != (size_t)(4 * n_fields)) return fail(TL_EINVAL, "need exactly 4*n_fields device pointers");
    for (size_t i = 0; i < n_ptrs; ++i)
        if (!dev_ptrs[i] || ((uintptr_t)dev_ptrs[i] & 15u)) return fail(TL_EINVAL, "device pointer %zu is NULL or not 16-byte aligned", i);
    tl_lattice *L = new (std::nothrow) tl_lattice();
    if (!L) return fail(TL_ENOMEM, "host allocation failed");
    memset(L->buf, 0, sizeof L->buf);
    const size_t esz = dtype == TL_F64 ? 8 : 4;
    const size_t org = tl::layout_of(N, esz).origin * esz;
    for (int f = 0; f < n_fields; ++f) {
        L->buf[0][0][f] = static_cast<char *>(dev_ptrs[4 * f + 0]) + org;
        L->buf[0][1][f] = static_cast<char *>(dev_ptrs[4 * f + 1]) + org;
        L->buf[1][0][f] = static_cast<char *>(dev_ptrs[4 * f + 2]) + org;
        L->buf[1][1][f] = static_cast<char *>(dev_ptrs[4 * f + 3]) + org;
    }
    rc = finish_create(L, N, kIR, n_fields, dtype, expansion, cuda_stream);
    if (rc) {
        tl_lattice_destroy(L);
        return rc;
    }
    *out = L;
    return TL_OK;
}

void tl_lattice_destroy(tl_lattice *L)
{
    if (!L || L->batch_refs > 0) return;  // still held by a tl_batch: destroy the batch first
    cudaStreamSynchronize(L->stream);
    for (auto &g : L->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (L->capture) cudaStreamDestroy(L->capture);
    if (L->own && L->base) cudaFree(L->base);
    if (L->d_sc) cudaFree(L->d_sc);
    if (L->d_slots) cudaFree(L->d_slots);
    delete L;
}

int tl_set_potential(tl_lattice *L, const tl_potential *pot)
{
    g_err[0] = 0;
    if (!L || !pot) return fail(TL_EINVAL, "NULL argument");
    if (!isfinite(pot->lambda) || !isfinite(pot->q)) return fail(TL_EINVAL, "non-finite coupling");
    for (int f = 0; f < TL_MAX_FIELDS; ++f)
        if (!isfinite(pot->m2[f])) return fail(TL_EINVAL, "non-finite mass");
    L->pot = *pot;
    L->has_pot = true;
    refresh_model(L);
    L->energies_valid = false;
    return TL_OK;
}

}  // extern "C"

namespace {

// Launch a pass list on the lattice's stream.
int run_passes(tl_lattice *L, const std::vector<PassCoef> &passes)
{
    for (const PassCoef &c : passes) {
        int rc = launch(L, c, false);
        if (rc) return rc;
    }
    return TL_OK;
}

// The pass list of tl_step as a CUDA graph: captured on the lattice's private
// stream (nothing runs during capture), instantiated, replayed on its stream.
// Returns false if the capture could not be made (the caller then launches
// directly); L->cur is left as it was.
bool capture_passes(tl_lattice *L, const std::vector<PassCoef> &passes, cudaGraphExec_t *exec)
{
    *exec = nullptr;
    if (!L->capture && cudaStreamCreateWithFlags(&L->capture, cudaStreamNonBlocking) != cudaSuccess) {
        L->capture = nullptr;
        return false;
    }
    if (cudaStreamBeginCapture(L->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    const int cur = L->cur;
    int rc = TL_OK;
    for (const PassCoef &c : passes)
        if ((rc = launch(L, c, false, L->capture))) break;
    L->cur = cur;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(L->capture, &graph);
    if (rc || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return false;
    }
    const cudaError_t ei = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        *exec = nullptr;
        cudaGetLastError();
        return false;
    }
    return true;
}

// tl_step's launches: the first call with a given (n, dt, integrator, buffer
// parity) on the current lattice version launches the passes directly and
// remembers the key; a repeat captures them once and from then on replays the
// graph (one launch per call instead of n P + 1).  TL_STEP_GRAPHS=0 in the
// environment turns this off.
constexpr size_t kMaxStepGraphs = 8;

int step_passes(tl_lattice *L, int n, double dt, int integrator, const std::vector<PassCoef> &passes)
{
    const char *env = getenv("TL_STEP_GRAPHS");
    if (env && strcmp(env, "0") == 0) return run_passes(L, passes);
    auto it = L->graphs.begin();
    for (; it != L->graphs.end(); ++it)
        if (it->n == n && it->dt == dt && it->integrator == integrator && it->cur == L->cur &&
            it->version == L->version)
            break;
    if (it == L->graphs.end()) {  // first sight: direct launches, remember the key
        if (L->graphs.size() >= kMaxStepGraphs) {
            if (L->graphs.front().exec) cudaGraphExecDestroy(L->graphs.front().exec);
            L->graphs.erase(L->graphs.begin());
        }
        L->graphs.push_back(tl_lattice::StepGraph{n, integrator, L->cur, dt, L->version, nullptr});
        return run_passes(L, passes);
    }
    if (!it->exec && !capture_passes(L, passes, &it->exec)) return run_passes(L, passes);
    TL_CK(cudaGraphLaunch(it->exec, L->stream));
    if (passes.size() & 1) L->cur ^= 1;
    return TL_OK;
}

}  // namespace

extern "C" {

int tl_step(tl_lattice *L, int n, double dt, tl_integrator integrator)
{
    tl::NvtxScope nvtx_range("tl_step");
    g_err[0] = 0;
    if (!L) return fail(TL_EINVAL, "NULL lattice");
    if (n < 0) return fail(TL_EINVAL, "n must be >= 0");
    if (!isfinite(dt) || dt == 0.0) return fail(TL_EINVAL, "dt must be finite and nonzero");
    if (!L->has_pot) return fail(TL_ESTATE, "tl_set_potential has not been called");
    if (!L->has_state) return fail(TL_ESTATE, "no state: call tl_init_fluctuations or tl_set_state for every array");
    if (n == 0) return TL_OK;
    std::vector<PassCoef> passes;
    if (!tl::pass_schedule(n, dt, (int)integrator, passes)) return fail(TL_EINVAL, "unknown integrator %d", (int)integrator);
    int rc = step_passes(L, n, dt, (int)integrator, passes);
    if (rc) return rc;
    L->step += n;
    L->energies_valid = true;
    return TL_OK;
}

int tl_energies(tl_lattice *L, tl_energies_t *out)
{
    tl::NvtxScope nvtx_range("tl_energies");
    g_err[0] = 0;
    if (!L || !out) return fail(TL_EINVAL, "NULL argument");
    if (!L->has_state || !L->has_pot) return fail(TL_ESTATE, "no state or potential");
    if (!L->energies_valid) {
        int rc = measure(L, false);
        if (rc) return rc;
    }
    Scalars h;
    int rc = read_scalars(L, &h);
    if (rc) return rc;
    memset(out, 0, sizeof *out);
    out->step = L->step;
    out->time = h.time;
    out->a = L->ex.expanding ? h.a : 1.0;
    out->b = L->ex.expanding ? h.b : 0.0;
    for (int f = 0; f < L->nf; ++f) {
        out->K[f] = h.E[f];
        out->G[f] = h.E[L->nf + f];
    }
    out->V = h.E[2 * L->nf];
    out->hubble_resid = h.hubble;
    if (h.status == TL_ETIMEOUT) return fail(TL_ETIMEOUT, "a bounded device wait expired during a pass");
    if (h.status != TL_OK) return fail(TL_EUNSTABLE, "energies became non-finite");
    return TL_OK;
}

int tl_get_state(tl_lattice *L, int field, int which, void *host, size_t bytes)
{
    g_err[0] = 0;
    int rc = check_field(L, field, which);
    if (rc) return rc;
    if (!host || bytes != n3_of(L->N) * L->esz) return fail(TL_EINVAL, "host buffer must hold N^3 elements");
    rc = copy_planes(L, host, L->buf[L->cur][which][field], false);
    if (rc) return rc;
    Scalars h;
    rc = read_scalars(L, &h);
    if (rc) return rc;
    if (h.status == TL_ETIMEOUT) return fail(TL_ETIMEOUT, "a bounded device wait expired during a pass");
    if (h.status != TL_OK) return fail(TL_EUNSTABLE, "evolution became non-finite");
    return TL_OK;
}

int tl_set_state(tl_lattice *L, int field, int which, const void *host, size_t bytes)
{
    g_err[0] = 0;
    int rc = check_field(L, field, which);
    if (rc) return rc;
    if (!host || bytes != n3_of(L->N) * L->esz) return fail(TL_EINVAL, "host buffer must hold N^3 elements");
    rc = copy_planes(L, const_cast<void *>(host), L->buf[L->cur][which][field], true);
    if (rc) return rc;
    TL_CK(tl::launch_fill_ghosts((int)L->dtype, L->buf[L->cur][which][field], L->N, L->model.pitch, L->model.pplane,
                                 L->stream));
    TL_CK(tl::launch_set_background(L->model, L->d_sc, L->ex.a0, 0.0, L->stream));
    TL_CK(cudaStreamSynchronize(L->stream));
    L->state_mask |= 1u << (2 * field + which);
    L->has_state = L->state_mask == (1u << (2 * L->nf)) - 1u;
    L->step = 0;
    L->langevin_steps = 0;
    L->energies_valid = false;
    return TL_OK;
}

int tl_commit_state(tl_lattice *L)
{
    g_err[0] = 0;
    if (!L) return fail(TL_EINVAL, "NULL lattice");
    if (L->batch_refs > 0) return fail(TL_ESTATE, "lattice is part of a batch");
    for (int f = 0; f < L->nf; ++f)
        for (int which = 0; which < 2; ++which)
            TL_CK(tl::launch_fill_ghosts((int)L->dtype, L->buf[L->cur][which][f], L->N, L->model.pitch,
                                         L->model.pplane, L->stream));
    TL_CK(tl::launch_set_background(L->model, L->d_sc, L->ex.a0, 0.0, L->stream));
    TL_CK(cudaStreamSynchronize(L->stream));
    L->state_mask = (1u << (2 * L->nf)) - 1u;
    L->has_state = true;
    L->step = 0;
    L->langevin_steps = 0;
    L->energies_valid = false;
    return TL_OK;
}

int tl_set_background(tl_lattice *L, double a, double b, int from_constraint)
{
    g_err[0] = 0;
    if (!L) return fail(TL_EINVAL, "NULL lattice");
    if (!(a > 0.0) || !isfinite(a) || !isfinite(b)) return fail(TL_EINVAL, "a must be positive, a and b finite");
    TL_CK(tl::launch_set_background(L->model, L->d_sc, a, b, L->stream));
    L->energies_valid = false;
    if (from_constraint && L->ex.expanding) {
        if (!L->has_state || !L->has_pot) return fail(TL_ESTATE, "from_constraint needs a state and a potential");
        return measure(L, true);
    }
    return TL_OK;
}

int tl_get_clock(tl_lattice *L, tl_clock *out)
{
    g_err[0] = 0;
    if (!L || !out) return fail(TL_EINVAL, "NULL argument");
    Scalars h;
    int rc = read_scalars(L, &h);
    if (rc) return rc;
    out->step = L->step;
    out->time = h.time;
    out->langevin_steps = L->langevin_steps;
    return TL_OK;
}

int tl_set_clock(tl_lattice *L, const tl_clock *c)
{
    g_err[0] = 0;
    if (!L || !c) return fail(TL_EINVAL, "NULL argument");
    if (c->step < 0 || c->langevin_steps < 0 || !isfinite(c->time))
        return fail(TL_EINVAL, "step counts must be >= 0 and time finite");
    if (!L->has_state) return fail(TL_ESTATE, "no state: set every array first");
    if (L->batch_refs > 0) return fail(TL_ESTATE, "lattice is part of a batch");
    const double t = c->time;
    TL_CK(cudaMemcpyAsync(reinterpret_cast<char *>(L->d_sc) + offsetof(Scalars, time), &t, sizeof t,
                          cudaMemcpyHostToDevice, L->stream));
    TL_CK(cudaStreamSynchronize(L->stream));
    L->step = c->step;
    L->langevin_steps = c->langevin_steps;
    return TL_OK;
}

int tl_state_device_ptr(tl_lattice *L, int field, int which, void **dev_ptr)
{
    g_err[0] = 0;
    int rc = check_field(L, field, which);
    if (rc) return rc;
    if (!dev_ptr) return fail(TL_EINVAL, "NULL dev_ptr");
    *dev_ptr = L->buf[L->cur][which][field];
    return TL_OK;
}

int tl_set_pass_config(tl_lattice *L, const tl_pass_config *cfg)
{
    g_err[0] = 0;
    if (!L || !cfg) return fail(TL_EINVAL, "NULL argument");
    if (L->batch_refs > 0) return fail(TL_ESTATE, "lattice is part of a batch");
    if (cfg->kind != TL_PASS_STREAM && cfg->kind != TL_PASS_TMA) return fail(TL_EINVAL, "unknown pass kind %d", cfg->kind);
    if (cfg->z_chunk < 0 || cfg->z_chunk > L->N) return fail(TL_EINVAL, "z_chunk must be in 0..N");
    tl::PassTuning t{tl::kVariantLdg, 7, 0, cfg->z_chunk, 0, 256, 0};
    if (cfg->kind == TL_PASS_TMA) {
        if (cfg->warps != 0 && cfg->warps != 7 && cfg->warps != 15) return fail(TL_EINVAL, "TMA warps must be 0, 7 or 15");
        if (cfg->stages != 0 && (cfg->stages < 3 || cfg->stages > 8))
            return fail(TL_EINVAL, "TMA stages must be 0 or 3..8");
        if (cfg->tile_x != 0 || cfg->threads != 0) return fail(TL_EINVAL, "tile_x and threads apply to TL_PASS_STREAM");
        t.variant = tl::kVariantTma;
        t.cwarps = cfg->warps ? cfg->warps : 7;
        t.stages = cfg->stages;
    } else {
        // a row narrower than 32 threads: its own width is what
        // tl_get_pass_config reports for the widths above it, and means the same
        const int per_row = L->N / (int)(16 / L->esz);
        const bool own_row = per_row < 32 && cfg->tile_x == per_row;
        if (cfg->tile_x != 0 && cfg->tile_x != 8 && cfg->tile_x != 16 && cfg->tile_x != 32 && !own_row)
            return fail(TL_EINVAL, "tile_x must be 0, 8, 16, 32 or the lattice's row width in threads (N/4 FP32, N/2 FP64) below 32");
        if (cfg->threads != 0 && cfg->threads != 256 && cfg->threads != 512)
            return fail(TL_EINVAL, "threads must be 0, 256 or 512");
        if (cfg->warps != 0 || cfg->stages != 0) return fail(TL_EINVAL, "warps and stages apply to TL_PASS_TMA");
        t.txt = own_row ? 0 : cfg->tile_x;
        t.threads = cfg->threads ? cfg->threads : 256;
    }
    return tl::set_geometry(L, t);
}

int tl_get_pass_config(const tl_lattice *L, tl_pass_config *cfg)
{
    g_err[0] = 0;
    if (!L || !cfg) return fail(TL_EINVAL, "NULL argument");
    const tl::PassGeom &g = L->geom;
    const bool tma = g.variant == tl::kVariantTma;
    cfg->kind = tma ? TL_PASS_TMA : TL_PASS_STREAM;
    cfg->warps = tma ? g.cwarps : 0;
    cfg->stages = tma ? g.stages : 0;
    cfg->z_chunk = g.zc;
    cfg->tile_x = tma ? 0 : g.txt;
    cfg->threads = tma ? 0 : g.threads;
    return TL_OK;
}

int tl_spectrum_bins(int N)
{
    if (N <= 0) return 0;
    return (int)ceil(sqrt(3.0) * N / 2.0) + 1;
}

int tl_init_fluctuations(tl_lattice *L, uint64_t seed, const tl_init_spec *spec)
{
    tl::NvtxScope nvtx_range("tl_init_fluctuations");
    g_err[0] = 0;
    if (!L || !spec) return fail(TL_EINVAL, "NULL argument");
    if (!L->has_pot) return fail(TL_ESTATE, "tl_set_potential must come first (b0 needs the potential)");
    if (!(spec->A >= 0.0) || !isfinite(spec->A)) return fail(TL_EINVAL, "A must be finite and >= 0");
    const int N = L->N;
    const size_t n3 = n3_of(N);
    const size_t nh = (size_t)N * N * (N / 2 + 1);
    std::lock_guard<std::mutex> plan_lock(g_plan_mu);
    SharedPlan *sp = nullptr;
    {
        int prc = shared_plan(N, CUFFT_Z2D, L->stream, &sp);
        if (prc) return prc;
    }
    const cufftHandle plan = sp->h;
    double2 *modes = nullptr;
    double *real = nullptr;
    TL_CK(cudaMallocAsync((void **)&modes, nh * sizeof(double2), L->stream));
    cudaError_t e = cudaMallocAsync((void **)&real, n3 * sizeof(double), L->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(modes, L->stream);
        return fail(TL_ENOMEM, "scratch allocation for the initial field failed");
    }
    int rc = TL_OK;
    const bool expanding = L->ex.expanding != 0;
    const double pscale = expanding ? pow(L->ex.a0, 3.0 - L->ex.alpha) : 1.0;
    for (int f = 0; f < L->nf && rc == TL_OK; ++f) {
        for (int which = 0; which < 2 && rc == TL_OK; ++which) {
            const double base = which == 0 ? spec->phi0[f] : spec->pi0[f];
            const bool fluct = which == 0 || spec->fluct_pi;
            void *dst = L->buf[L->cur][which][f];
            if (fluct && spec->A > 0.0) {
                cudaError_t ce = tl::launch_fill_modes(modes, N, L->kIR, spec->A, spec->meff2[f], which,
                                                       spec->fixed_modulus ? 1 : 0, seed, which == 0 ? (uint64_t)f : (uint64_t)(8 + f),
                                                       L->sm_count, L->stream);
                if (ce != cudaSuccess) { rc = fail(TL_ECUDA, "fill_modes: %s", cudaGetErrorString(ce)); break; }
                cufftResult fr = cufftExecZ2D(plan, reinterpret_cast<cufftDoubleComplex *>(modes), real);
                if (fr != CUFFT_SUCCESS) { rc = fail(TL_ECUDA, "cufftExecZ2D failed (%d)", (int)fr); break; }
                ce = tl::launch_assemble((int)L->dtype, dst, real, n3, base, which == 0 ? 1.0 : pscale, N,
                                         L->model.pitch, L->model.pplane, L->sm_count, L->stream);
                if (ce != cudaSuccess) { rc = fail(TL_ECUDA, "assemble: %s", cudaGetErrorString(ce)); break; }
            } else {
                cudaError_t ce = tl::launch_assemble((int)L->dtype, dst, nullptr, n3, base, 0.0, N, L->model.pitch,
                                                     L->model.pplane, L->sm_count, L->stream);
                if (ce != cudaSuccess) { rc = fail(TL_ECUDA, "assemble: %s", cudaGetErrorString(ce)); break; }
            }
        }
    }
    {
        const cudaError_t re = cudaEventRecord(sp->done, L->stream);  // after this call's executions
        if (re != cudaSuccess && rc == TL_OK) rc = fail(TL_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(re));
    }
    cudaFreeAsync(modes, L->stream);
    cudaFreeAsync(real, L->stream);
    if (rc) return rc;
    for (int f = 0; f < L->nf; ++f)
        for (int which = 0; which < 2; ++which)
            TL_CK(tl::launch_fill_ghosts((int)L->dtype, L->buf[L->cur][which][f], N, L->model.pitch, L->model.pplane,
                                         L->stream));
    L->state_mask = (1u << (2 * L->nf)) - 1u;
    L->has_state = true;
    L->step = 0;
    L->langevin_steps = 0;
    TL_CK(tl::launch_set_background(L->model, L->d_sc, L->ex.a0, 0.0, L->stream));
    return measure(L, expanding);
}

int tl_spectrum(tl_lattice *L, int field, int which, int nbins, double *k, double *P, int64_t *count)
{
    tl::NvtxScope nvtx_range("tl_spectrum");
    g_err[0] = 0;
    int rc = check_field(L, field, which);
    if (rc) return rc;
    const int N = L->N;
    const int nb = tl_spectrum_bins(N);
    if (nbins < nb) return fail(TL_EINVAL, "nbins must be >= %d", nb);
    const size_t n3 = n3_of(N);
    const size_t nh = (size_t)N * N * (N / 2 + 1);
    std::lock_guard<std::mutex> plan_lock(g_plan_mu);
    SharedPlan *sp = nullptr;
    {
        int prc = shared_plan(N, CUFFT_D2Z, L->stream, &sp);
        if (prc) return prc;
    }
    const cufftHandle plan = sp->h;
    double2 *modes = nullptr;
    double *real = nullptr, *acc = nullptr;
    TL_CK(cudaMallocAsync((void **)&modes, nh * sizeof(double2), L->stream));
    TL_CK(cudaMallocAsync((void **)&real, n3 * sizeof(double), L->stream));
    TL_CK(cudaMallocAsync((void **)&acc, (size_t)nb * 3 * sizeof(double), L->stream));
    TL_CK(cudaMemsetAsync(acc, 0, (size_t)nb * 3 * sizeof(double), L->stream));
    TL_CK(tl::launch_widen((int)L->dtype, real, L->buf[L->cur][which][field], n3, N, L->model.pitch, L->model.pplane,
                           L->sm_count, L->stream));
    cufftResult fr = cufftExecD2Z(plan, real, reinterpret_cast<cufftDoubleComplex *>(modes));
    if (fr != CUFFT_SUCCESS) return fail(TL_ECUDA, "cufftExecD2Z failed (%d)", (int)fr);
    TL_CK(cudaEventRecord(sp->done, L->stream));
    TL_CK(tl::launch_bin(modes, N, nb, acc, acc + nb, reinterpret_cast<unsigned long long *>(acc + 2 * nb),
                         L->sm_count, L->stream));
    std::vector<double> h((size_t)nb * 3);
    TL_CK(cudaMemcpyAsync(h.data(), acc, h.size() * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    cudaFreeAsync(modes, L->stream);
    cudaFreeAsync(real, L->stream);
    cudaFreeAsync(acc, L->stream);
    TL_CK(cudaStreamSynchronize(L->stream));
    const double Lbox = 2.0 * M_PI / L->kIR;
    const double V = Lbox * Lbox * Lbox;
    for (int b = 0; b < nbins; ++b) {
        unsigned long long c = 0;
        double ps = 0.0, rs = 0.0;
        if (b < nb) {
            memcpy(&c, &h[2 * (size_t)nb + b], sizeof c);
            ps = h[b];
            rs = h[(size_t)nb + b];
        }
        if (count) count[b] = (int64_t)c;
        if (P) P[b] = c ? V * ps / (double)c : 0.0;
        if (k) k[b] = c ? L->kIR * rs / (double)c : 0.0;
    }
    return TL_OK;
}

}  // extern "C"
