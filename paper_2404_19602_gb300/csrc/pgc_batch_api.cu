// pgc_batch_api.cu -- C ABI of the batched sweep (pgc_batch_*): many single-case contexts stepped
// together by one persistent launch sequence per time step, optionally replayed from a CUDA graph,
// with the tile size chosen by timing candidate tiles on the running simulation.
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "pgc.h"
#include "pgc_batch.cuh"
#include "pgc_ctx.h"

namespace pgc {

BatchRunner *make_batch_runner_1x1(int, const std::vector<BatchCase> &, const BatchScratch &, int);
BatchRunner *make_batch_runner_6x6(int, const std::vector<BatchCase> &, const BatchScratch &, int);
BatchRunner *make_batch_runner_21x36(int, const std::vector<BatchCase> &, const BatchScratch &, int);
size_t case_dev_size_1x1(int);
size_t case_dev_size_6x6(int);
size_t case_dev_size_21x36(int);

BatchRunner *make_batch_runner(int P, int Q, int precision, const std::vector<BatchCase> &cases, const BatchScratch &sc,
                               int num_sms)
{
    if (P == 1 && Q == 1) return make_batch_runner_1x1(precision, cases, sc, num_sms);
    if (P == 6 && Q == 6) return make_batch_runner_6x6(precision, cases, sc, num_sms);
    if (P == 21 && Q == 36) return make_batch_runner_21x36(precision, cases, sc, num_sms);
    return nullptr;
}

size_t case_dev_size(int P, int Q, int precision)
{
    if (P == 1 && Q == 1) return case_dev_size_1x1(precision);
    if (P == 6 && Q == 6) return case_dev_size_6x6(precision);
    if (P == 21 && Q == 36) return case_dev_size_21x36(precision);
    return 0;
}

}  // namespace pgc

using namespace pgc;

struct pgc_batch {
    std::vector<pgc_ctx *> ctxs;
    BatchRunner *run = nullptr;
    BatchScratch sc;
    cudaStream_t stream = nullptr;
    int every = -1;                 // moments_every the graph was captured with
    int graph_steps = 0;
    cudaGraphExec_t gexec = nullptr;
    std::string err;
};

static thread_local std::string g_batch_err;

// Launch configurations chosen by pgc_batch_autotune, per (P, Q, precision, floor(log2(total
// particles))): a batch created later with tile_particles = 0 starts from the cached choice.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, BatchLaunch> g_tune_cache;

static std::tuple<int, int, int, int> tune_key(const std::vector<pgc_ctx *> &ctxs)
{
    int64_t n = 0;
    for (const pgc_ctx *c : ctxs) n += c->b.N;
    int bucket = 0;
    while ((int64_t)1 << (bucket + 1) <= n) ++bucket;
    return std::make_tuple(ctxs[0]->t.P, ctxs[0]->t.Q, ctxs[0]->cfg.precision, bucket);
}

namespace {

struct BatchLayout {
    size_t cases = 0, tile0s = 0, bases = 0, queue = 0, qcount = 0, done = 0, d_step = 0, t_out = 0, part_tiles = 0,
           part2c = 0, total = 0;
    int64_t max_tiles = 0;
};

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// checks that the contexts can be stepped together; fills the layout for the smallest tile
pgc_status check_batch(pgc_ctx *const *ctxs, int32_t n, BatchLayout *L, std::string *msg)
{
    if (!ctxs || n < 1) { *msg = "need at least one context"; return PGC_EINVAL; }
    if (n > kBatchMaxCases) { *msg = "at most " + std::to_string(kBatchMaxCases) + " cases per batch"; return PGC_EINVAL; }
    const pgc_ctx *c0 = ctxs[0];
    if (!c0) { *msg = "NULL context"; return PGC_EINVAL; }
    int64_t ntot = 0, tiles = 0;
    const int pass = 256 * ((c0->t.P <= 8) ? 4 : 1);
    for (int i = 0; i < n; ++i) {
        const pgc_ctx *c = ctxs[i];
        if (!c || c->failed) { *msg = "context " + std::to_string(i) + " is NULL or failed"; return PGC_EINVAL; }
        const pgc_config &a = c->cfg, &b = c0->cfg;
        if (c->t.P != c0->t.P || c->t.Q != c0->t.Q || a.precision != b.precision || a.T_K != b.T_K ||
            a.mech_mask != b.mech_mask || a.alpha != b.alpha || a.Nk != b.Nk || a.Lk_hvF_eV != b.Lk_hvF_eV ||
            a.dt_fs != b.dt_fs || a.final_state != b.final_state || a.n_theta_edge != b.n_theta_edge ||
            a.max_collisions != b.max_collisions || a.pauli_norm != b.pauli_norm || a.degree_M != b.degree_M ||
            a.quad_per_dim != b.quad_per_dim) {
            *msg = "context " + std::to_string(i) + " differs from context 0 in shape, precision or physics";
            return PGC_EINVAL;
        }
        if (c->step != c0->step) { *msg = "all contexts must be at the same step"; return PGC_EINVAL; }
        if (a.splitting != PGC_SPLIT_LIE) { *msg = "the batched kernels run the Lie splitting (PGC_SPLIT_LIE)"; return PGC_EUNSUPPORTED; }
        if (a.tc_proj != PGC_TC_OFF) { *msg = "the batched kernels reconstruct on the FMA pipes (tc_proj must be PGC_TC_OFF)"; return PGC_EUNSUPPORTED; }
        if (c->stream != c0->stream) { *msg = "all contexts must use the same stream"; return PGC_EINVAL; }
        ntot += c->b.N;
        tiles += (c->b.N + pass - 1) / pass;
    }
    if (c0->cfg.pauli_norm == PGC_PAULI_CURRENT_MAX) { *msg = "batches support the initial-maximum and off Pauli modes"; return PGC_EUNSUPPORTED; }
    if (ntot >= (int64_t)0xffffffffLL) { *msg = "total particles of a batch must be < 2^32"; return PGC_EINVAL; }
    const int Q = c0->t.Q;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = (size_t)rup((int64_t)(off + bytes), 256); return o; };
    L->cases = take((size_t)n * case_dev_size(c0->t.P, Q, c0->cfg.precision));
    L->tile0s = take((size_t)(n + 1) * 8);
    L->bases = take((size_t)(n + 1) * 8);
    L->queue = take((size_t)ntot * 4);
    L->qcount = take(2 * 4);
    L->done = take(4);
    L->d_step = take(8);
    L->t_out = take((size_t)n * 8);
    L->part_tiles = take((size_t)tiles * Q * 3 * 8);
    L->part2c = take((size_t)n * Q * 3 * 8);
    L->total = off;
    L->max_tiles = tiles;
    return PGC_OK;
}

}  // namespace

extern "C" {

pgc_status pgc_batch_query_sizes(pgc_ctx *const *ctxs, int32_t n_cases, size_t *scratch_bytes)
{
    BatchLayout L;
    std::string msg;
    pgc_status s = check_batch(ctxs, n_cases, &L, &msg);
    if (s != PGC_OK) { g_batch_err = msg; return s; }
    if (scratch_bytes) *scratch_bytes = L.total;
    return PGC_OK;
}

pgc_status pgc_batch_create(pgc_ctx *const *ctxs, int32_t n_cases, void *d_scratch, int32_t tile_particles,
                            pgc_batch **out)
{
    if (!out) { g_batch_err = "out is NULL"; return PGC_EINVAL; }
    *out = nullptr;
    BatchLayout L;
    std::string msg;
    pgc_status s = check_batch(ctxs, n_cases, &L, &msg);
    if (s != PGC_OK) { g_batch_err = msg; return s; }
    if (!d_scratch || ((uintptr_t)d_scratch & 255)) { g_batch_err = "scratch must be non-NULL and 256-byte aligned"; return PGC_EINVAL; }
    const pgc_ctx *c0 = ctxs[0];
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { g_batch_err = cudaGetErrorString(e); return PGC_ECUDA; }
    pgc_batch *b = new pgc_batch();
    b->ctxs.assign(ctxs, ctxs + n_cases);
    b->stream = c0->stream;
    char *base = (char *)d_scratch;
    b->sc.cases = base + L.cases;
    b->sc.tile0s = (int64_t *)(base + L.tile0s);
    b->sc.bases = (int64_t *)(base + L.bases);
    b->sc.queue = (uint32_t *)(base + L.queue);
    b->sc.qcount = (uint32_t *)(base + L.qcount);
    b->sc.done = (uint32_t *)(base + L.done);
    b->sc.d_step = (int64_t *)(base + L.d_step);
    b->sc.t_out = (int64_t *)(base + L.t_out);
    b->sc.part_tiles = (double *)(base + L.part_tiles);
    b->sc.part2c = (double *)(base + L.part2c);
    b->sc.max_tiles = L.max_tiles;
    std::vector<BatchCase> cases(n_cases);
    std::vector<int64_t> tout(n_cases);
    for (int i = 0; i < n_cases; ++i) {
        cases[i].t = &ctxs[i]->t;
        cases[i].b = ctxs[i]->b;
        cases[i].series = ctxs[i]->series;
        tout[i] = ctxs[i]->T_out;
    }
    b->run = make_batch_runner(c0->t.P, c0->t.Q, c0->cfg.precision, cases, b->sc, sms);
    if (!b->run) { delete b; g_batch_err = "no batch kernel for this shape"; return PGC_EUNSUPPORTED; }
    int tile = tile_particles;
    if (tile_particles == 0) {   // the cached autotuner choice for this kind of batch, if any
        BatchLaunch lc;
        bool have = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(tune_key(b->ctxs));
            if (it != g_tune_cache.end()) { lc = it->second; have = true; }
        }
        if (have && b->run->set_launch(lc.block, lc.ppt, lc.g1_per_sm, lc.g2_per_sm) == cudaSuccess && lc.tile % b->run->pass() == 0)
            tile = lc.tile;
        else
            tile = 8 * b->run->pass();
    }
    const int pass = b->run->pass();
    if (tile % pass || tile > 65535) { delete b->run; delete b; g_batch_err = "tile must be a multiple of " + std::to_string(pass) + " and < 65536"; return PGC_EINVAL; }
    const int64_t step0 = c0->step;
    e = cudaMemsetAsync(d_scratch, 0, L.total, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->sc.d_step, &step0, 8, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->sc.t_out, tout.data(), tout.size() * 8, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = b->run->set_tile(tile, b->stream);  // synchronizes
    if (e != cudaSuccess) { delete b->run; delete b; g_batch_err = cudaGetErrorString(e); return PGC_ECUDA; }
    *out = b;
    return PGC_OK;
}

static pgc_status batch_fail(pgc_batch *b, pgc_status s, const std::string &m)
{
    b->err = m;
    return s;
}

static void drop_graph(pgc_batch *b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->graph_steps = 0;
}

pgc_status pgc_batch_step(pgc_batch *b, int64_t n_steps, int32_t moments_every, int32_t use_graph)
{
    if (!b) { g_batch_err = "batch is NULL"; return PGC_EINVAL; }
    if (n_steps < 0 || moments_every < 0) return batch_fail(b, PGC_EINVAL, "negative argument");
    const int64_t s0 = b->ctxs[0]->step;
    for (pgc_ctx *c : b->ctxs) {
        if (c->failed) return batch_fail(b, PGC_ESTATE, "a context failed earlier");
        if (c->step != s0) return batch_fail(b, PGC_ESTATE, "contexts were stepped outside the batch");
    }
    const int64_t outs = moments_every > 0 ? (s0 + n_steps) / moments_every - s0 / moments_every : 0;
    for (pgc_ctx *c : b->ctxs)
        if (c->T_out + outs > c->cfg.max_outputs) return batch_fail(b, PGC_ENOMEM, "moment series would exceed max_outputs");
    cudaStream_t s = b->stream;
    cudaError_t e = cudaSuccess;
    if (moments_every != b->every) {
        drop_graph(b);
        b->every = moments_every;
        b->run->set_moments_every(moments_every);
    }
    int64_t done = 0;
    const int K = 10;  // time steps per captured graph
    if (use_graph && n_steps >= K) {
        if (!b->gexec) {
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                for (int k = 0; k < K && e == cudaSuccess; ++k) e = b->run->step(s);
                cudaError_t e2 = cudaStreamEndCapture(s, &g);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) { cudaGetLastError(); drop_graph(b); return batch_fail(b, PGC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e)); }
            b->graph_steps = K;
        }
        for (; done + K <= n_steps && e == cudaSuccess; done += K) {
            e = cudaGraphLaunch(b->gexec, s);
            count_launch(3 * K);
        }
    }
    for (; done < n_steps && e == cudaSuccess; ++done) e = b->run->step(s);
    // the single-case collider counters must start at zero if a context is stepped alone later
    for (pgc_ctx *c : b->ctxs)
        if (e == cudaSuccess) e = cudaMemsetAsync(c->b.qcount, 0, 8 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return batch_fail(b, PGC_ECUDA, std::string("batch step: ") + cudaGetErrorString(e));
    for (pgc_ctx *c : b->ctxs) {
        c->step += n_steps;
        c->T_out += outs;
    }
    return PGC_OK;
}

// Time steps_per_candidate steps (no moments) under one launch configuration; +inf if the
// configuration cannot run (tile not a multiple of the pass, more tiles than the scratch holds).
static float time_launch(pgc_batch *b, const BatchLaunch &lc, int steps, pgc_status *st, cudaEvent_t e0, cudaEvent_t e1)
{
    if (b->run->set_launch(lc.block, lc.ppt, lc.g1_per_sm, lc.g2_per_sm) != cudaSuccess) return 1e30f;
    if (lc.tile % b->run->pass() || lc.tile > 65535) return 1e30f;
    if (b->run->set_tile(lc.tile, b->stream) != cudaSuccess) { cudaGetLastError(); return 1e30f; }
    drop_graph(b);
    cudaEventRecord(e0, b->stream);
    *st = pgc_batch_step(b, steps, 0, 0);
    cudaEventRecord(e1, b->stream);
    if (*st != PGC_OK) return 1e30f;
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
}

pgc_status pgc_batch_autotune(pgc_batch *b, int32_t steps_per_candidate, int32_t *chosen_tile, double *ms_per_step)
{
    if (!b) { g_batch_err = "batch is NULL"; return PGC_EINVAL; }
    if (steps_per_candidate < 1) return batch_fail(b, PGC_EINVAL, "steps_per_candidate < 1");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // coordinate descent over the tile, the streaming block size, the particles per thread and
    // the streaming and collider blocks per SM, from the current configuration, two rounds; the
    // timed steps are part of the run (no configuration changes a trajectory)
    BatchLaunch best = b->run->launch();
    pgc_status st = PGC_OK;
    float best_ms = time_launch(b, best, steps_per_candidate, &st, e0, e1);
    const int min_tile = (b->ctxs[0]->t.P <= 8) ? 1024 : 256;   // the scratch holds the tiles of this size
    for (int round = 0; round < 2 && st == PGC_OK; ++round) {
        for (int dim = 0; dim < 5 && st == PGC_OK; ++dim) {
            std::vector<BatchLaunch> cand;
            BatchLaunch c = best;
            if (dim == 0) for (int t = min_tile; t <= 32768; t *= 2) { c.tile = t; cand.push_back(c); }
            if (dim == 1) for (int blk : {128, 256}) { c.block = blk; c.g1_per_sm = std::max(1, b->run->max_g1(blk, c.ppt)); cand.push_back(c); }
            if (dim == 2) for (int ppt : b->run->ppts()) { c.ppt = ppt; c.g1_per_sm = std::max(1, b->run->max_g1(c.block, ppt)); cand.push_back(c); }
            if (dim == 3) for (int g = 1; g <= b->run->max_g1(c.block, c.ppt); ++g) { c.g1_per_sm = g; cand.push_back(c); }
            if (dim == 4) for (int g = 2; g <= b->run->max_g2(); ++g) { c.g2_per_sm = g; cand.push_back(c); }
            for (const BatchLaunch &x : cand) {
                if (x.tile == best.tile && x.block == best.block && x.ppt == best.ppt && x.g1_per_sm == best.g1_per_sm &&
                    x.g2_per_sm == best.g2_per_sm)
                    continue;
                const float ms = time_launch(b, x, steps_per_candidate, &st, e0, e1);
                if (st != PGC_OK) break;
                if (ms < best_ms) { best_ms = ms; best = x; }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PGC_OK) return st;
    drop_graph(b);
    b->every = -1;
    if (b->run->set_launch(best.block, best.ppt, best.g1_per_sm, best.g2_per_sm) != cudaSuccess ||
        b->run->set_tile(best.tile, b->stream) != cudaSuccess)
        return batch_fail(b, PGC_ECUDA, "applying the chosen launch configuration");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[tune_key(b->ctxs)] = best;
    }
    if (chosen_tile) *chosen_tile = best.tile;
    if (ms_per_step) *ms_per_step = best_ms / steps_per_candidate;
    return PGC_OK;
}

pgc_status pgc_batch_launch_config(const pgc_batch *b, int32_t *cfg5)
{
    if (!b || !cfg5) { g_batch_err = "NULL argument"; return PGC_EINVAL; }
    const BatchLaunch l = b->run->launch();
    cfg5[0] = l.tile;
    cfg5[1] = l.block;
    cfg5[2] = l.ppt;
    cfg5[3] = l.g1_per_sm;
    cfg5[4] = l.g2_per_sm;
    return PGC_OK;
}

void pgc_batch_destroy(pgc_batch *b)
{
    if (!b) return;
    drop_graph(b);
    delete b->run;
    delete b;
}

const char *pgc_batch_last_error(const pgc_batch *b)
{
    return b ? b->err.c_str() : g_batch_err.c_str();
}

}  // extern "C"
