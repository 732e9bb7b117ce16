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

#include <algorithm>
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

namespace {

// Launch options of a batch's grouped passes (the same for every member).
struct BatchOpts {
    int prefetch = 0;  // 0: plain streaming tiles; 3: per-thread cp.async ring three planes ahead
    int split = 1;     // field-count groups as independent branches of the graph (else one chain)
    int share = 0;     // 0: each group's persistent grid is 2 CTAs x SMs; 1: that grid split by work
};

}  // namespace

struct tl_batch {
    // Lattices of one field count and one kernel variant, advanced by one
    // grouped launch per pass.
    struct Group {
        int nf = 0;
        int variant = tl::kVariantLdg;        // the members' kernel: register streaming or TMA
        std::vector<int> idx;                 // lattices of this group
        BatchJob *d_jobs[2] = {nullptr, nullptr}; // even / odd passes of a call
        unsigned *d_first = nullptr;          // first item of each job
        tl::TmaMaps *d_maps = nullptr;        // TMA: tensor maps of each member, both buffer parities
        unsigned total = 0;                   // items (CTA tiles) over all jobs
        double work = 0.0;                    // sites x fields of its lattices
        int grid = 0;                         // CTAs (persistent for streaming, one per item for TMA)
        int stages = 0;                       // TMA: ring stages
        size_t smem = 0;                      // TMA: dynamic shared memory per CTA
        cudaStream_t branch = nullptr;        // capture stream of its graph branch (group 0: the capture stream)
        cudaEvent_t done = nullptr;           // end of its branch
    };
    std::vector<tl_lattice *> lats;
    std::vector<Group> groups;
    std::vector<cudaStream_t> branch_pool;    // branch streams and join events, reused by group rebuilds
    std::vector<cudaEvent_t> event_pool;
    int dtype = 0;
    int sm_count = 0;
    BatchOpts opts;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;
    cudaEvent_t fork = nullptr;
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
            for (const int &i : g.idx) {
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
                j.lpad = L->geom.lpad;
                j.maps = g.d_maps ? g.d_maps + 2 * (&i - g.idx.data()) + in : nullptr;
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

// Item layout of every group from its members' current launch geometry, and
// the persistent grid of each group's launch under the batch's options.
int refresh_groups(tl_batch *B)
{
    const int per_sm = 2;  // the grouped kernel's register budget allows two CTAs per SM
    const long full = (long)B->sm_count * per_sm;
    double all = 0.0;
    for (auto &g : B->groups) all += g.work;
    std::vector<unsigned> first;
    for (auto &g : B->groups) {
        first.clear();
        g.total = 0;
        for (int i : g.idx) {
            first.push_back(g.total);
            g.total += B->lats[i]->geom.nblocks;
        }
        if (g.variant == tl::kVariantTma) {
            // one CTA per item; the ring as deep as two CTAs per SM allow for the
            // largest box among the members; each member's tensor maps (both
            // buffer parities) copied to device memory for the kernel to read
            int txt_max = 0, ty_max = 0;
            std::vector<tl::TmaMaps> maps;
            for (int i : g.idx) {
                tl_lattice *L = B->lats[i];
                txt_max = std::max(txt_max, L->geom.txt);
                ty_max = std::max(ty_max, L->geom.ty);
                int rc = tl::lattice_tma_maps(L);
                if (rc) return rc;
                maps.push_back(L->maps[0]);
                maps.push_back(L->maps[1]);
            }
            int S = 8;
            while (S > 3 && tl::tma_group_smem(g.nf, S, txt_max, ty_max) > 113u * 1024u) --S;
            g.stages = S;
            g.smem = tl::tma_group_smem(g.nf, S, txt_max, ty_max);
            g.grid = (int)g.total;
            TB_CK(cudaMemcpyAsync(g.d_maps, maps.data(), maps.size() * sizeof(tl::TmaMaps), cudaMemcpyHostToDevice,
                                  B->stream));
        } else {
            long want = full;
            if (B->opts.share && B->groups.size() > 1 && all > 0.0) {
                want = (long)(full * (g.work / all) + 0.5);
                if (want < B->sm_count / 4) want = B->sm_count / 4 > 0 ? B->sm_count / 4 : 1;
            }
            g.grid = (int)((long)g.total < want ? (long)g.total : want);
            if (g.grid < 1) g.grid = 1;
        }
        TB_CK(cudaMemcpyAsync(g.d_first, first.data(), first.size() * sizeof(unsigned), cudaMemcpyHostToDevice,
                              B->stream));
        TB_CK(cudaStreamSynchronize(B->stream));  // `first` and `maps` are reused for the next group
    }
    return TL_OK;
}

void free_groups(tl_batch *B)
{
    for (auto &g : B->groups) {
        cudaFree(g.d_jobs[0]);
        cudaFree(g.d_jobs[1]);
        cudaFree(g.d_first);
        cudaFree(g.d_maps);
    }
    B->groups.clear();
}

// Partition the members into groups by field count and kernel variant (the
// variant each member's launch shape names) and allocate their descriptors;
// branch streams and join events come from the batch's pools.
int build_groups(tl_batch *B)
{
    free_groups(B);
    const int n = (int)B->lats.size();
    for (int nf = 1; nf <= TL_MAX_FIELDS; ++nf)
        for (int variant : {tl::kVariantLdg, tl::kVariantTma}) {
            tl_batch::Group g;
            g.nf = nf;
            g.variant = variant;
            for (int i = 0; i < n; ++i)
                if (B->lats[i]->nf == nf && B->lats[i]->tuning.variant == variant) {
                    g.idx.push_back(i);
                    g.work += (double)B->lats[i]->N * B->lats[i]->N * B->lats[i]->N * nf;
                }
            if (g.idx.empty()) continue;
            B->groups.push_back(g);
        }
    cudaError_t e = cudaSuccess;
    for (size_t gi = 0; gi < B->groups.size(); ++gi) {
        auto &g = B->groups[gi];
        const size_t jb = g.idx.size() * sizeof(BatchJob);
        if ((e = cudaMalloc(&g.d_jobs[0], jb)) != cudaSuccess || (e = cudaMalloc(&g.d_jobs[1], jb)) != cudaSuccess ||
            (e = cudaMalloc(&g.d_first, g.idx.size() * sizeof(unsigned))) != cudaSuccess ||
            (g.variant == tl::kVariantTma &&
             (e = cudaMalloc(&g.d_maps, 2 * g.idx.size() * sizeof(tl::TmaMaps))) != cudaSuccess))
            return tl::fail(TL_ENOMEM, "batch descriptors: %s", cudaGetErrorString(e));
        while (B->branch_pool.size() <= gi) {
            cudaStream_t st = nullptr;
            cudaEvent_t ev = nullptr;
            if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
                if (st) cudaStreamDestroy(st);
                return tl::fail(TL_ECUDA, "stream/event creation: %s", cudaGetErrorString(e));
            }
            B->branch_pool.push_back(st);
            B->event_pool.push_back(ev);
        }
        g.branch = B->branch_pool[gi];
        g.done = B->event_pool[gi];
    }
    return refresh_groups(B);
}

// Capture `passes` over every group into an executable graph: each group's
// passes form one chain on its own capture stream (a branch forked from and
// joined back into the batch's capture stream) when opts.split is set, so the
// groups' launches overlap on the device; else one chain of all groups.
int capture_passes(tl_batch *B, const std::vector<PassCoef> &passes, cudaGraph_t *graph_out,
                   cudaGraphExec_t *exec_out)
{
    *graph_out = nullptr;
    *exec_out = nullptr;
    TB_CK(cudaStreamBeginCapture(B->capture, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    const bool split = B->opts.split && B->groups.size() > 1;
    if (split) {
        e = cudaEventRecord(B->fork, B->capture);
        for (size_t gi = 1; gi < B->groups.size() && e == cudaSuccess; ++gi)
            e = cudaStreamWaitEvent(B->groups[gi].branch, B->fork, 0);
    }
    if (split) {
        for (size_t gi = 0; gi < B->groups.size() && e == cudaSuccess; ++gi) {
            auto &g = B->groups[gi];
            cudaStream_t s = gi == 0 ? B->capture : g.branch;
            for (size_t p = 0; p < passes.size() && e == cudaSuccess; ++p)
                e = tl::launch_group(B->dtype, g.nf, g.variant, B->opts.prefetch, g.stages, g.smem, g.d_jobs[p & 1],
                                     g.d_first, (int)g.idx.size(), g.total, passes[p], g.grid, s);
            if (gi > 0 && e == cudaSuccess) e = cudaEventRecord(g.done, s);
        }
        for (size_t gi = 1; gi < B->groups.size() && e == cudaSuccess; ++gi)
            e = cudaStreamWaitEvent(B->capture, B->groups[gi].done, 0);
    } else {
        for (size_t p = 0; p < passes.size() && e == cudaSuccess; ++p)
            for (auto &g : B->groups) {
                e = tl::launch_group(B->dtype, g.nf, g.variant, B->opts.prefetch, g.stages, g.smem, g.d_jobs[p & 1],
                                     g.d_first, (int)g.idx.size(), g.total, passes[p], g.grid, B->capture);
                if (e != cudaSuccess) break;
            }
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
    *graph_out = graph;
    *exec_out = exec;
    return TL_OK;
}

void drop_graph(tl_batch *B)
{
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
    B->g_n = -1;
}

int build_graph(tl_batch *B, int n, double dt, int integrator)
{
    std::vector<PassCoef> passes;
    if (!tl::pass_schedule(n, dt, integrator, passes)) return tl::fail(TL_EINVAL, "unknown integrator %d", integrator);
    drop_graph(B);
    int rc = capture_passes(B, passes, &B->graph, &B->exec);
    if (rc) return rc;
    B->g_n = n;
    B->g_dt = dt;
    B->g_integ = integrator;
    return TL_OK;
}

// ---- batch launch shapes ------------------------------------------------------
// A member's shape in a batch: the register-streaming tiles with 256-thread
// CTAs (what the grouped kernel runs).  Untuned, z-chunks of 32 planes (the
// whole lattice below that), so that each (lattice, tile) item of the grouped
// launch carries enough planes to amortise its fixed costs (locating the job,
// the coefficient set-up, the FP64 reduction of its sums); tl_batch_autotune
// replaces this rule by measured shapes per (N, fields, dtype, SMs), and the
// batch-level options per batch composition.

typedef std::tuple<int, int, int, int> ClassKey;  // N, fields, dtype, SMs
std::mutex g_batch_mu;
std::map<ClassKey, tl::PassTuning> g_batch_shapes;
std::map<std::string, BatchOpts> g_batch_opts;  // composition signature -> options

tl::PassTuning batch_rule(int N) { return tl::PassTuning{tl::kVariantLdg, 7, 0, N < 32 ? N : 32, 0, 256, 0}; }

void ensure_tune_loaded();  // TL_TUNE_FILE, read once (autotuner section below)

tl::PassTuning batch_tuning(int N, int nf, int dtype, int sms)
{
    ensure_tune_loaded();
    std::lock_guard<std::mutex> lk(g_batch_mu);
    auto it = g_batch_shapes.find(ClassKey(N, nf, dtype, sms));
    return it != g_batch_shapes.end() ? it->second : batch_rule(N);
}

std::string composition(const std::vector<tl_lattice *> &lats)
{
    std::map<std::tuple<int, int, int>, int> cnt;
    for (tl_lattice *L : lats) cnt[std::make_tuple(L->N, L->nf, (int)L->dtype)]++;
    std::string s = std::to_string(lats.empty() ? 0 : lats[0]->sm_count);
    for (auto &kv : cnt)
        s += ":" + std::to_string(std::get<0>(kv.first)) + "x" + std::to_string(std::get<1>(kv.first)) + "x" +
             std::to_string(std::get<2>(kv.first)) + "=" + std::to_string(kv.second);
    return s;
}

bool same_shape(const tl::PassTuning &a, const tl::PassTuning &b)
{
    if (a.variant != b.variant || a.zc != b.zc) return false;
    if (a.variant == tl::kVariantTma) return a.cwarps == b.cwarps;
    return a.threads == b.threads && a.txt == b.txt && a.prefetch == b.prefetch;
}

}  // namespace

extern "C" {

int tl_batch_pass_config(int N, int n_fields, tl_dtype dtype, tl_pass_config *out)
{
    tl::set_error(TL_OK, "", "");
    if (!out) return tl::fail(TL_EINVAL, "NULL out");
    if (N < 8 || N % 4 != 0 || N > 2048 || n_fields < 1 || n_fields > TL_MAX_FIELDS ||
        (dtype != TL_F32 && dtype != TL_F64))
        return tl::fail(TL_EINVAL, "bad lattice shape");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        sms = 0;
    const tl::PassTuning t = batch_tuning(N, n_fields, (int)dtype, sms);
    if (t.variant == tl::kVariantTma)
        *out = tl_pass_config{TL_PASS_TMA, t.cwarps, 0, t.zc, 0, 0};
    else
        *out = tl_pass_config{TL_PASS_STREAM, 0, 0, t.zc, t.txt, t.threads};
    return TL_OK;
}

int tl_batch_create(tl_batch **out, tl_lattice *const *lats, int n, void *cuda_stream)
{
    tl::NvtxScope nvtx_range("tl_batch_create");
    tl::set_error(TL_OK, "", "");
    if (!out || !lats || n <= 0) return tl::fail(TL_EINVAL, "need a non-empty list of lattices");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!lats[i]) return tl::fail(TL_EINVAL, "lattice %d is NULL", i);
        if (lats[i]->dtype != lats[0]->dtype) return tl::fail(TL_EINVAL, "all lattices of a batch share one dtype");
        if (lats[i]->batch_refs > 0) return tl::fail(TL_EINVAL, "lattice %d is already in a batch", i);
        for (int k = 0; k < i; ++k)
            if (lats[k] == lats[i]) return tl::fail(TL_EINVAL, "lattice %d appears twice", i);
    }
    tl_batch *B = new (std::nothrow) tl_batch();
    if (!B) return tl::fail(TL_ENOMEM, "host allocation failed");
    B->lats.assign(lats, lats + n);
    B->dtype = (int)lats[0]->dtype;
    B->stream = static_cast<cudaStream_t>(cuda_stream);
    B->sm_count = lats[0]->sm_count;
    ensure_tune_loaded();
    {
        std::lock_guard<std::mutex> lk(g_batch_mu);
        auto it = g_batch_opts.find(composition(B->lats));
        if (it != g_batch_opts.end()) B->opts = it->second;
    }
    // environment override of the options (tuning experiments): "prefetch,split,share"
    if (const char *v = getenv("TL_BATCH_OPTIONS")) {
        int pf = 0, sp = 1, sh = 0;
        if (sscanf(v, "%d,%d,%d", &pf, &sp, &sh) == 3 && (pf == 0 || pf == 3) && (sp == 0 || sp == 1) &&
            (sh == 0 || sh == 1))
            B->opts = BatchOpts{pf, sp, sh};
    }
    // members move to the batch shape (and keep it afterwards); every member
    // of a batch runs with the batch's prefetch option
    for (int i = 0; i < n; ++i) {
        tl_lattice *L = lats[i];
        tl::PassTuning t = batch_tuning(L->N, L->nf, (int)L->dtype, L->sm_count);
        if (t.variant == tl::kVariantLdg) t.prefetch = B->opts.prefetch;
        if (!same_shape(L->tuning, t)) {
            int rc = tl::set_geometry(L, t);
            if (rc) {
                delete B;
                return rc;
            }
        }
    }
    int rc = TL_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&B->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) rc = tl::fail(TL_ECUDA, "stream/event creation: %s", cudaGetErrorString(e));
    if (rc == TL_OK) rc = build_groups(B);
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
    drop_graph(B);
    free_groups(B);
    for (cudaStream_t st : B->branch_pool) cudaStreamDestroy(st);
    for (cudaEvent_t ev : B->event_pool) cudaEventDestroy(ev);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->capture) cudaStreamDestroy(B->capture);
    for (tl_lattice *L : B->lats)
        if (L->batch_refs > 0) L->batch_refs--;
    delete B;
}

namespace {

int check_members(tl_batch *B)
{
    for (tl_lattice *L : B->lats) {
        if (!L->has_pot || !L->has_state) return tl::fail(TL_ESTATE, "every lattice needs a potential and a state");
        if (L->dtype != (tl_dtype)B->dtype) return tl::fail(TL_EINVAL, "dtype changed");
    }
    // the lattices' own streams must be done with earlier work before the batch stream runs
    for (tl_lattice *L : B->lats)
        if (L->stream != B->stream) TB_CK(cudaStreamSynchronize(L->stream));
    return TL_OK;
}

}  // namespace

int tl_batch_step(tl_batch *B, int n, double dt, tl_integrator integrator)
{
    tl::NvtxScope nvtx_range("tl_batch_step");
    tl::set_error(TL_OK, "", "");
    if (!B) return tl::fail(TL_EINVAL, "NULL batch");
    if (n < 0) return tl::fail(TL_EINVAL, "n must be >= 0");
    if (!isfinite(dt) || dt == 0.0) return tl::fail(TL_EINVAL, "dt must be finite and nonzero");
    int rc = check_members(B);
    if (rc) return rc;
    if (n == 0) return TL_OK;
    rc = upload_jobs(B);
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

// Batch entries (tl_batch_autotune): one member shape per (N, fields, dtype,
// SMs), and the launch options of one batch composition.
const char *const kBatchShapeFmt =
    "{\"batch_shape\": {\"N\": %d, \"fields\": %d, \"dtype\": %d, \"sms\": %d, \"variant\": %d, "
    "\"z_chunk\": %d, \"tile_x\": %d, \"prefetch\": %d}}";
const char *const kBatchOptsFmt = "{\"batch_options\": {\"prefetch\": %d, \"split\": %d, \"share\": %d, "
                                  "\"composition\": \"%255[^\"]\"}}";

void load_tune_file()
{
    g_tune_loaded = true;
    const char *path = getenv("TL_TUNE_FILE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        {
            int N, nf, dt, sms, var, zc, txt, pf, sp, sh;
            char comp[256];
            if (sscanf(line, kBatchShapeFmt, &N, &nf, &dt, &sms, &var, &zc, &txt, &pf) == 8) {
                if (N >= 8 && nf >= 1 && nf <= TL_MAX_FIELDS && (dt == 0 || dt == 1) && zc >= 1 && zc <= N &&
                    (var == tl::kVariantLdg || var == tl::kVariantTma) &&
                    (txt == 0 || txt == 8 || txt == 16 || txt == 32) && (pf == 0 || pf == 3)) {
                    std::lock_guard<std::mutex> lk(g_batch_mu);
                    g_batch_shapes[ClassKey(N, nf, dt, sms)] =
                        var == tl::kVariantTma ? tl::PassTuning{tl::kVariantTma, 7, 0, zc, 0, 256, 0}
                                               : tl::PassTuning{tl::kVariantLdg, 7, 0, zc, pf, 256, txt};
                }
                continue;
            }
            if (sscanf(line, kBatchOptsFmt, &pf, &sp, &sh, comp) == 4) {
                if ((pf == 0 || pf == 3) && (sp == 0 || sp == 1) && (sh == 0 || sh == 1)) {
                    std::lock_guard<std::mutex> lk(g_batch_mu);
                    g_batch_opts[comp] = BatchOpts{pf, sp, sh};
                }
                continue;
            }
        }
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

void ensure_tune_loaded()
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_tune_loaded) load_tune_file();
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
    tl::NvtxScope nvtx_range("tl_autotune");
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

// ---- batch autotuner ------------------------------------------------------------

namespace {

void append_tune_line(const char *line)
{
    const char *path = getenv("TL_TUNE_FILE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fputs(line, f);
    fputs("\n", f);
    fclose(f);
}

// Average time of one grouped identity pass over the whole batch (ms): passes
// with zero kick and drift coefficients rewrite every state unchanged; an
// even number of them leaves each lattice's buffers where they started.
int time_identity(tl_batch *B, cudaEvent_t e0, cudaEvent_t e1, double *ms_out)
{
    int rc = build_groups(B);  // members may have changed kernel variant
    if (rc) return rc;
    rc = upload_jobs(B);
    if (rc) return rc;
    const int reps = 6;
    std::vector<PassCoef> passes(reps, PassCoef{});
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    rc = capture_passes(B, passes, &graph, &exec);
    if (rc) return rc;
    // warm-up, then the best of three timings of two replays each (single
    // timings of sub-millisecond replays vary by several percent)
    cudaError_t e = cudaGraphLaunch(exec, B->stream);
    float best = 0.f;
    for (int t = 0; t < 3 && e == cudaSuccess; ++t) {
        if (e == cudaSuccess) e = cudaEventRecord(e0, B->stream);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaGraphLaunch(exec, B->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, B->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (t == 0 || ms < best)) best = ms;
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return tl::fail(TL_ECUDA, "batch autotune: %s", cudaGetErrorString(e));
    *ms_out = best / (2.0 * reps);
    return TL_OK;
}

}  // namespace

extern "C" int tl_batch_autotune(tl_batch *B, double *best_ms_per_pass)
{
    tl::NvtxScope nvtx_range("tl_batch_autotune");
    tl::set_error(TL_OK, "", "");
    if (!B) return tl::fail(TL_EINVAL, "NULL batch");
    int rc = check_members(B);
    if (rc) return rc;
    ensure_tune_loaded();
    drop_graph(B);
    // classes of members: (N, fields), largest total work first
    struct Cls {
        int N, nf;
        double work;
        std::vector<tl_lattice *> members;
        tl::PassTuning t;
    };
    std::vector<Cls> cls;
    for (tl_lattice *L : B->lats) {
        Cls *c = nullptr;
        for (auto &k : cls)
            if (k.N == L->N && k.nf == L->nf) c = &k;
        if (!c) {
            cls.push_back(Cls{L->N, L->nf, 0.0, {}, L->tuning});
            c = &cls.back();
        }
        c->members.push_back(L);
        c->work += (double)L->N * L->N * L->N * L->nf;
    }
    std::sort(cls.begin(), cls.end(), [](const Cls &a, const Cls &b) { return a.work > b.work; });
    auto apply = [&](Cls &c, const tl::PassTuning &t) -> int {
        for (tl_lattice *L : c.members) {
            int r = tl::set_geometry(L, t);
            if (r) return r;
        }
        return TL_OK;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TB_CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return tl::fail(TL_ECUDA, "cudaEventCreate failed");
    }
    double best = 0.0;
    rc = time_identity(B, e0, e1, &best);
    // coordinate descent, one sweep: each class's z-chunk and tile row width
    // with the others held at their current best
    for (size_t ci = 0; ci < cls.size() && rc == TL_OK; ++ci) {
        Cls &c = cls[ci];
        const int per_row = c.N / (B->dtype == TL_F64 ? 2 : 4);
        std::vector<tl::PassTuning> cands;
        for (int txt : {0, 16, 8}) {
            if (txt && txt >= per_row) continue;  // the same tile as txt = 0
            for (int zc : {4, 8, 16, 32, 64, 128, c.N}) {
                if (zc > c.N) continue;
                tl::PassTuning t{tl::kVariantLdg, 7, 0, zc, B->opts.prefetch, 256, txt};
                bool dup = same_shape(t, c.t);
                for (auto &o : cands) dup = dup || same_shape(o, t);
                if (!dup) cands.push_back(t);
            }
        }
        // the TMA pass (7 + 1 warps, one CTA per item of the grouped launch)
        for (int zc : {8, 16, 32, 64, c.N}) {
            if (zc > c.N) continue;
            tl::PassTuning t{tl::kVariantTma, 7, 0, zc, 0, 256, 0};
            bool dup = same_shape(t, c.t);
            for (auto &o : cands) dup = dup || same_shape(o, t);
            if (!dup) cands.push_back(t);
        }
        for (const auto &t : cands) {
            const tl::PassTuning keep = c.t;
            if ((rc = apply(c, t))) break;
            double ms = 0.0;
            if ((rc = time_identity(B, e0, e1, &ms))) break;
            if (ms < best) {
                best = ms;
                c.t = t;
            } else if ((rc = apply(c, keep))) {
                break;
            }
        }
    }
    // batch-level options: prefetch ring, independent branches, grid split
    if (rc == TL_OK) {
        const BatchOpts start = B->opts;
        BatchOpts best_o = start;
        for (int pf : {0, 3})
            for (int sp : {1, 0})
                for (int sh : {0, 1}) {
                    if (rc) break;
                    BatchOpts o{pf, sp, sh};
                    if (o.prefetch == start.prefetch && o.split == start.split && o.share == start.share) continue;
                    if (B->groups.size() < 2 && (sp == 0 || sh == 1)) continue;  // no effect with one group
                    B->opts = o;
                    for (auto &c : cls) {
                        if (c.t.variant == tl::kVariantLdg) c.t.prefetch = pf;
                        if ((rc = apply(c, c.t))) break;
                    }
                    if (rc) break;
                    double ms = 0.0;
                    if ((rc = time_identity(B, e0, e1, &ms))) break;
                    if (ms < best) {
                        best = ms;
                        best_o = o;
                    }
                }
        if (rc == TL_OK) {
            B->opts = best_o;
            for (auto &c : cls) {
                if (c.t.variant == tl::kVariantLdg) c.t.prefetch = best_o.prefetch;
                if ((rc = apply(c, c.t))) break;
            }
        }
        if (rc == TL_OK) rc = build_groups(B);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_batch_mu);
        for (auto &c : cls) g_batch_shapes[ClassKey(c.N, c.nf, B->dtype, B->sm_count)] = c.t;
        g_batch_opts[composition(B->lats)] = B->opts;
    }
    char buf[512];
    for (auto &c : cls) {
        snprintf(buf, sizeof buf, kBatchShapeFmt, c.N, c.nf, B->dtype, B->sm_count, c.t.variant, c.t.zc, c.t.txt,
                 c.t.prefetch);
        append_tune_line(buf);
    }
    const std::string comp = composition(B->lats);
    if (comp.size() < 255) {
        snprintf(buf, sizeof buf, "{\"batch_options\": {\"prefetch\": %d, \"split\": %d, \"share\": %d, "
                                  "\"composition\": \"%s\"}}",
                 B->opts.prefetch, B->opts.split, B->opts.share, comp.c_str());
        append_tune_line(buf);
    }
    if (best_ms_per_pass) *best_ms_per_pass = best;
    return TL_OK;
}

extern "C" int tl_batch_get_options(const tl_batch *B, int *prefetch, int *split, int *share)
{
    tl::set_error(TL_OK, "", "");
    if (!B) return tl::fail(TL_EINVAL, "NULL batch");
    if (prefetch) *prefetch = B->opts.prefetch;
    if (split) *split = B->opts.split;
    if (share) *share = B->opts.share;
    return TL_OK;
}
