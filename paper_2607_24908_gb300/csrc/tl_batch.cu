// Batched ensembles and the launch-geometry autotuner.
//
// tl_batch advances many independent lattices (uneven N, 1-3 fields, their
// own potentials, backgrounds and seeds) with one persistent grouped launch
// per pass and per field count, the whole pass sequence of a tl_batch_step
// call captured once as a CUDA graph and replayed.  Each job keeps the launch
// geometry it has alone, so its per-CTA sums, and hence its results, are
// bitwise the same alone and in the batch.
//
// tl_autotune times candidate geometries (z-chunk, variant) of one lattice
// with identity passes (kick and drift coefficients zero, so the state is
// unchanged) and keeps the fastest; results are cached per (N, fields, dtype,
// SM count) in memory and, if TL_TUNE_FILE names a file, on disk.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "tl_internal.cuh"
#include "tl_lattice.cuh"

using tl::BatchJob;
using tl::PassCoef;

#define TB_CK(call)                                                                                         \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return tl::fail(TL_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));          \
    } while (0)

struct tl_batch {
    struct Group {
        int nf = 0;
        std::vector<int> idx;                 // lattices of this group
        BatchJob *d_jobs[2] = {nullptr, nullptr}; // even / odd passes of a call
        unsigned *d_first = nullptr;          // first item of each job
        unsigned total = 0;                   // items (CTA tiles) over all jobs
        int grid = 0;                         // persistent CTAs
    };
    std::vector<tl_lattice *> lats;
    std::vector<Group> groups;
    int dtype = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;
    // graph of the last (n, dt, integrator)
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    int g_n = -1, g_integ = -1;
    double g_dt = 0.0;
    std::vector<BatchJob> h_jobs;
};

namespace {

int upload_jobs(tl_batch *B)
{
    for (auto &g : B->groups) {
        for (int parity = 0; parity < 2; ++parity) {
            B->h_jobs.clear();
            for (int i : g.idx) {
                tl_lattice *L = B->lats[i];
                const int in = L->cur ^ parity;
                BatchJob j{};
                j.m = L->model;
                for (int f = 0; f < TL_MAX_FIELDS; ++f) {
                    j.fp.phi_in[f] = L->buf[in][0][f];
                    j.fp.pi_in[f] = L->buf[in][1][f];
                    j.fp.phi_out[f] = L->buf[in ^ 1][0][f];
                    j.fp.pi_out[f] = L->buf[in ^ 1][1][f];
                }
                j.sc = L->d_sc;
                j.slots = L->d_slots;
                j.txt = L->geom.txt;
                j.ty = L->geom.ty;
                j.zc = L->geom.zc;
                j.gx = (int)L->geom.grid.x;
                j.gy = (int)L->geom.grid.y;
                j.nblocks = L->geom.nblocks;
                B->h_jobs.push_back(j);
            }
            TB_CK(cudaMemcpyAsync(g.d_jobs[parity], B->h_jobs.data(), B->h_jobs.size() * sizeof(BatchJob),
                                  cudaMemcpyHostToDevice, B->stream));
        }
    }
    // h_jobs is pageable memory: each cudaMemcpyAsync has staged it before
    // returning, so the vector can be refilled at once without a sync.
    return TL_OK;
}

int build_graph(tl_batch *B, int n, double dt, int integrator)
{
    std::vector<PassCoef> passes;
    if (!tl::pass_schedule(n, dt, integrator, passes)) return tl::fail(TL_EINVAL, "unknown integrator %d", integrator);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
    TB_CK(cudaStreamBeginCapture(B->capture, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (size_t p = 0; p < passes.size() && e == cudaSuccess; ++p)
        for (auto &g : B->groups) {
            e = tl::launch_group(B->dtype, g.nf, g.d_jobs[p & 1], g.d_first, (int)g.idx.size(), g.total, passes[p],
                                 g.grid, B->capture);
            if (e != cudaSuccess) break;
        }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(B->capture, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return tl::fail(TL_ECUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return tl::fail(TL_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    B->graph = graph;
    B->exec = exec;
    B->g_n = n;
    B->g_dt = dt;
    B->g_integ = integrator;
    return TL_OK;
}

}  // namespace

namespace {

// The launch shape of batch members: the register-streaming tiles with
// 256-thread CTAs (what the grouped kernel runs) and z-chunks of 32 planes
// (the whole lattice below that), so that each (lattice, tile) item of the
// grouped launch carries enough planes to amortise its fixed costs (locating
// the job, the coefficient set-up, the FP64 reduction of its sums).
tl::PassTuning batch_tuning(int N) { return tl::PassTuning{tl::kVariantLdg, 7, 0, N < 32 ? N : 32, 0, 256, 0}; }

}  // namespace

extern "C" {

int tl_batch_pass_config(int N, int n_fields, tl_dtype dtype, tl_pass_config *out)
{
    tl::set_error(TL_OK, "", "");
    if (!out) return tl::fail(TL_EINVAL, "NULL out");
    if (N < 8 || N % 4 != 0 || N > 2048 || n_fields < 1 || n_fields > TL_MAX_FIELDS ||
        (dtype != TL_F32 && dtype != TL_F64))
        return tl::fail(TL_EINVAL, "bad lattice shape");
    const tl::PassTuning t = batch_tuning(N);
    *out = tl_pass_config{TL_PASS_STREAM, 0, 0, t.zc, 0, t.threads};
    return TL_OK;
}

int tl_batch_create(tl_batch **out, tl_lattice *const *lats, int n, void *cuda_stream)
{
    tl::set_error(TL_OK, "", "");
    if (!out || !lats || n <= 0) return tl::fail(TL_EINVAL, "need a non-empty list of lattices");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!lats[i]) return tl::fail(TL_EINVAL, "lattice %d is NULL", i);
        if (lats[i]->dtype != lats[0]->dtype) return tl::fail(TL_EINVAL, "all lattices of a batch share one dtype");
        for (int k = 0; k < i; ++k)
            if (lats[k] == lats[i]) return tl::fail(TL_EINVAL, "lattice %d appears twice", i);
    }
    // members move to the batch shape (and keep it afterwards)
    for (int i = 0; i < n; ++i) {
        tl_lattice *L = lats[i];
        const tl::PassTuning t = batch_tuning(L->N);
        if (L->tuning.variant != t.variant || L->tuning.threads != t.threads || L->tuning.zc != t.zc ||
            L->tuning.txt != t.txt || L->tuning.prefetch != t.prefetch) {
            int rc = tl::set_geometry(L, t);
            if (rc) return rc;
        }
    }
    tl_batch *B = new (std::nothrow) tl_batch();
    if (!B) return tl::fail(TL_ENOMEM, "host allocation failed");
    B->lats.assign(lats, lats + n);
    B->dtype = (int)lats[0]->dtype;
    B->stream = static_cast<cudaStream_t>(cuda_stream);
    B->sm_count = lats[0]->sm_count;
    int rc = TL_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&B->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = tl::fail(TL_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    for (int nf = 1; nf <= TL_MAX_FIELDS && rc == TL_OK; ++nf) {
        tl_batch::Group g;
        g.nf = nf;
        std::vector<unsigned> first;
        for (int i = 0; i < n; ++i)
            if (lats[i]->nf == nf) {
                g.idx.push_back(i);
                first.push_back(g.total);
                g.total += lats[i]->geom.nblocks;
            }
        if (g.idx.empty()) continue;
        const int per_sm = 2;  // the grouped kernel's register budget allows two CTAs per SM
        const long want = (long)B->sm_count * per_sm;
        g.grid = (int)((long)g.total < want ? (long)g.total : want);
        const size_t jb = g.idx.size() * sizeof(BatchJob);
        if ((e = cudaMalloc(&g.d_jobs[0], jb)) != cudaSuccess || (e = cudaMalloc(&g.d_jobs[1], jb)) != cudaSuccess ||
            (e = cudaMalloc(&g.d_first, first.size() * sizeof(unsigned))) != cudaSuccess ||
            (e = cudaMemcpy(g.d_first, first.data(), first.size() * sizeof(unsigned), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
            rc = tl::fail(TL_ENOMEM, "batch descriptors: %s", cudaGetErrorString(e));
        B->groups.push_back(g);
    }
    if (rc) {
        tl_batch_destroy(B);
        return rc;
    }
    for (tl_lattice *L : B->lats) L->batch_refs++;
    *out = B;
    return TL_OK;
}

void tl_batch_destroy(tl_batch *B)
{
    if (!B) return;
    cudaStreamSynchronize(B->stream);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    for (auto &g : B->groups) {
        cudaFree(g.d_jobs[0]);
        cudaFree(g.d_jobs[1]);
        cudaFree(g.d_first);
    }
    if (B->capture) cudaStreamDestroy(B->capture);
    for (tl_lattice *L : B->lats)
        if (L->batch_refs > 0) L->batch_refs--;
    delete B;
}

int tl_batch_step(tl_batch *B, int n, double dt, tl_integrator integrator)
{
    tl::set_error(TL_OK, "", "");
    if (!B) return tl::fail(TL_EINVAL, "NULL batch");
    if (n < 0) return tl::fail(TL_EINVAL, "n must be >= 0");
    if (!isfinite(dt) || dt == 0.0) return tl::fail(TL_EINVAL, "dt must be finite and nonzero");
    for (tl_lattice *L : B->lats) {
        if (!L->has_pot || !L->has_state) return tl::fail(TL_ESTATE, "every lattice needs a potential and a state");
        if (L->dtype != (tl_dtype)B->dtype) return tl::fail(TL_EINVAL, "dtype changed");
    }
    if (n == 0) return TL_OK;
    // the lattices' own streams must be done with earlier work before the batch stream runs
    for (tl_lattice *L : B->lats)
        if (L->stream != B->stream) TB_CK(cudaStreamSynchronize(L->stream));
    int rc = upload_jobs(B);
    if (rc) return rc;
    if (!(B->exec && B->g_n == n && B->g_dt == dt && B->g_integ == (int)integrator)) {
        rc = build_graph(B, n, dt, (int)integrator);
        if (rc) return rc;
    }
    TB_CK(cudaGraphLaunch(B->exec, B->stream));
    const long passes = (long)n * (integrator == TL_YOSHIDA4 ? 3 : 1) + 1;
    for (tl_lattice *L : B->lats) {
        if (passes & 1) L->cur ^= 1;
        L->step += n;
        L->energies_valid = true;
        if (L->stream != B->stream) {
            // later work on the lattice's own stream must wait for the batch
            cudaEvent_t ev;
            TB_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            TB_CK(cudaEventRecord(ev, B->stream));
            TB_CK(cudaStreamWaitEvent(L->stream, ev, 0));
            TB_CK(cudaEventDestroy(ev));
        }
    }
    return TL_OK;
}

}  // extern "C"

// ---- autotuner ------------------------------------------------------------------

namespace {

typedef std::tuple<int, int, int, int> TuneKey;  // N, fields, dtype, SMs
struct TuneVal {
    tl::PassTuning t;
    double ms;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
bool g_tune_loaded = false;

// TL_TUNE_FILE holds JSON lines, one object per tuned shape, keys in the order
// written below; lines that do not parse as such (or carry out-of-range
// values) are skipped.
const char *const kTuneFmt =
    "{\"N\": %d, \"fields\": %d, \"dtype\": %d, \"sms\": %d, \"variant\": %d, \"warps\": %d, "
    "\"stages\": %d, \"z_chunk\": %d, \"prefetch\": %d, \"threads\": %d, \"tile_x\": %d, \"ms\": %lf}";

void load_tune_file()
{
    g_tune_loaded = true;
    const char *path = getenv("TL_TUNE_FILE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        int N, nf, dt, sms, var, cw, st, zc, pf, th, txt;
        double ms;
        if (sscanf(line, kTuneFmt, &N, &nf, &dt, &sms, &var, &cw, &st, &zc, &pf, &th, &txt, &ms) != 12) continue;
        const bool ok = (var == tl::kVariantLdg || var == tl::kVariantTma) && (cw == 7 || cw == 15) &&
                        (st == 0 || (st >= 3 && st <= 8)) && zc >= 0 && zc <= N && (pf == 0 || pf == 3) &&
                        (th == 256 || th == 512) && (txt == 0 || txt == 8 || txt == 16 || txt == 32);
        if (!ok) continue;
        tl::PassTuning t{var, cw, st, zc, pf, th, txt};
        g_tune[TuneKey(N, nf, dt, sms)] = TuneVal{t, ms};
    }
    fclose(f);
}

void save_tune_entry(const TuneKey &k, const TuneVal &v)
{
    const char *path = getenv("TL_TUNE_FILE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    char buf[512];
    // the same format prints the value as %f (the scan reads it as %lf)
    snprintf(buf, sizeof buf,
             "{\"N\": %d, \"fields\": %d, \"dtype\": %d, \"sms\": %d, \"variant\": %d, \"warps\": %d, "
             "\"stages\": %d, \"z_chunk\": %d, \"prefetch\": %d, \"threads\": %d, \"tile_x\": %d, \"ms\": %.6f}\n",
             std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k), v.t.variant, v.t.cwarps, v.t.stages,
             v.t.zc, v.t.prefetch, v.t.threads, v.t.txt, v.ms);
    fputs(buf, f);
    fclose(f);
}

}  // namespace

extern "C" int tl_autotune(tl_lattice *L, double *best_ms_per_pass)
{
    tl::set_error(TL_OK, "", "");
    if (!L) return tl::fail(TL_EINVAL, "NULL lattice");
    if (L->batch_refs > 0) return tl::fail(TL_ESTATE, "lattice is part of a batch");
    const TuneKey key(L->N, L->nf, (int)L->dtype, L->sm_count);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (!g_tune_loaded) load_tune_file();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            if (best_ms_per_pass) *best_ms_per_pass = it->second.ms;
            return tl::set_geometry(L, it->second.t);
        }
    }
    // candidates: the register-streaming pass with 256- or 512-thread CTAs
    // (two or one per SM), tile rows of 32, 16 or 8 threads, and z-chunks from
    // 4 planes to the whole lattice, plus the automatic choice; the TMA pass
    // with 7 or 15 compute warps, the deepest ring that fits and the same
    // z-chunks
    std::vector<tl::PassTuning> cands;
    cands.push_back(tl::PassTuning{tl::kVariantLdg, 7, 0, 0, 0, 256, 0});
    for (int threads : {256, 512})  // two or one CTAs per SM
        for (int txt : {32, 16, 8})
            for (int zc = 4; zc <= L->N && zc <= 256; zc *= 2)
                cands.push_back(tl::PassTuning{tl::kVariantLdg, 7, 0, zc, 0, threads, txt});
    for (int cw : {7, 15}) {
        cands.push_back(tl::PassTuning{tl::kVariantTma, cw, 0, 0, 0, 256, 0});
        for (int zc = 4; zc <= L->N && zc <= 256; zc *= 2)
            cands.push_back(tl::PassTuning{tl::kVariantTma, cw, 0, zc, 0, 256, 0});
    }
    const tl::PassTuning saved = L->tuning;
    cudaEvent_t e0, e1;
    TB_CK(cudaEventCreate(&e0));
    TB_CK(cudaEventCreate(&e1));
    PassCoef ident{};  // zero kick and drift: the pass rewrites the state unchanged
    const int reps = 4;  // even: the buffers end where they started
    double best = 1e300;
    tl::PassTuning best_t = saved;
    int rc = TL_OK;
    for (const auto &t : cands) {
        if ((rc = tl::set_geometry(L, t))) break;
        for (int i = 0; i < 2 && rc == TL_OK; ++i) rc = tl::lattice_launch(L, ident, false);
        if (rc) break;
        cudaEventRecord(e0, L->stream);
        for (int i = 0; i < reps && rc == TL_OK; ++i) rc = tl::lattice_launch(L, ident, false);
        if (rc) break;
        cudaEventRecord(e1, L->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = tl::fail(TL_ECUDA, "autotune: %s", cudaGetErrorString(e));
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / reps < best) {
            best = ms / reps;
            best_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        tl::set_geometry(L, saved);
        return rc;
    }
    rc = tl::set_geometry(L, best_t);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = TuneVal{best_t, best};
        save_tune_entry(key, TuneVal{best_t, best});
    }
    if (best_ms_per_pass) *best_ms_per_pass = best;
    return TL_OK;
}
