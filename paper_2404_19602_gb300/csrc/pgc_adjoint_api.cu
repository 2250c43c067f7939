// pgc_adjoint_api.cu -- C ABI of the adjoint (pgc_adjoint_*): forward run with checkpoints, then
// the reverse sweep segment by segment (replay with the forward kernels, backward kernels of
// pgc_adjoint.cuh), returning the window-averaged mean and variance of J_x and their pathwise
// gradient with respect to the field and band-minimum interval endpoints.
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "pgc.h"
#include "pgc_adjoint.cuh"
#include "pgc_ctx.h"

namespace pgc {

AdjRunner *make_adj_runner_1x1(int, const HostTables &, const DevBuffers &, const AdjBuffers &, int);
AdjRunner *make_adj_runner_6x6(int, const HostTables &, const DevBuffers &, const AdjBuffers &, int);
AdjRunner *make_adj_runner_21x36(int, const HostTables &, const DevBuffers &, const AdjBuffers &, int);

AdjRunner *make_adj_runner(int P, int Q, int precision, const HostTables &t, const DevBuffers &b, const AdjBuffers &ab,
                           int num_sms)
{
    if (P == 1 && Q == 1) return make_adj_runner_1x1(precision, t, b, ab, num_sms);
    if (P == 6 && Q == 6) return make_adj_runner_6x6(precision, t, b, ab, num_sms);
    if (P == 21 && Q == 36) return make_adj_runner_21x36(precision, t, b, ab, num_sms);
    return nullptr;
}

}  // namespace pgc

using namespace pgc;

namespace {

struct AdjLayout {
    int64_t nseg = 0;
    size_t state = 0, hist1 = 0;
    size_t ckpt_state = 0, ckpt_hist = 0, replay_state = 0, replay_hist = 0, stack_state = 0, stack_hist = 0, lam = 0,
           queue = 0, qcount = 0, counters = 0, part1 = 0, part2 = 0, aqueue = 0, aqcount = 0, grad = 0, total = 0;
};

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

pgc_status adj_layout(const pgc_ctx *ctx, int64_t n_steps, int32_t K, AdjLayout *L, std::string *msg)
{
    if (!ctx) { *msg = "ctx is NULL"; return PGC_EINVAL; }
    if (n_steps < 1 || K < 1) { *msg = "n_steps and ckpt_every must be >= 1"; return PGC_EINVAL; }
    const int Q = ctx->t.Q, P = ctx->t.P;
    const size_t esz = ctx->cfg.precision == PGC_FP64 ? 8 : 4;
    L->nseg = (n_steps + K - 1) / K;
    L->state = (size_t)rup((int64_t)(2 * P * ctx->b.ld * esz), 256);
    L->hist1 = (size_t)rup((int64_t)Q * ctx->t.Nk * ctx->t.Nk * 4, 256);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = (size_t)rup((int64_t)(off + bytes), 256); return o; };
    L->ckpt_state = take((size_t)L->nseg * L->state);
    L->ckpt_hist = take((size_t)L->nseg * L->hist1);
    L->replay_state = take(L->state);
    L->replay_hist = take((size_t)kHistBufs * ctx->b.hist_stride * 4);
    L->stack_state = take((size_t)(K + 1) * L->state);
    L->stack_hist = take((size_t)K * L->hist1);
    L->lam = take(L->state);
    L->queue = take((size_t)ctx->b.N * 4);
    L->qcount = take(8 * 4);
    L->counters = take(8 * 8);
    L->part1 = take((size_t)kMaxGrid1 * Q * 3 * 8);
    L->part2 = take((size_t)kGrid2Max * Q * 3 * 8);   // the replay runs the forward phase-2 grid
    L->aqueue = take((size_t)ctx->b.N * 4);
    L->aqcount = take(4 * 4);
    L->grad = take(NTH * 8);
    L->total = off;
    return PGC_OK;
}

pgc_status afail(pgc_ctx *ctx, pgc_status s, const std::string &m)
{
    ctx->err = m;
    if (s == PGC_ECUDA) ctx->failed = true;
    return s;
}

}  // namespace

extern "C" {

pgc_status pgc_adjoint_query_sizes(pgc_ctx *ctx, int64_t n_steps, int32_t ckpt_every, size_t *work_bytes)
{
    AdjLayout L;
    std::string msg;
    pgc_status s = adj_layout(ctx, n_steps, ckpt_every, &L, &msg);
    if (s != PGC_OK) {
        if (ctx) ctx->err = msg;
        return s;
    }
    if (work_bytes) *work_bytes = L.total;
    return PGC_OK;
}

// (Jbar, Vbar): averages over the moment records T0.. of the context whose step n (counted from
// step cur0) lies in (n_steps - window_steps, n_steps] of the z-mean and z-variance of J_x; nout
// receives the number of such records.
static cudaError_t window_values(pgc_ctx *ctx, int64_t T0, int64_t cur0, int64_t n_steps, int64_t window_steps,
                                 std::vector<double> *rec, double value[2], int64_t *nout)
{
    const int RL = ctx->rec_len, Q = ctx->t.Q;
    rec->assign((size_t)(ctx->T_out - T0) * RL, 0.0);
    cudaError_t e = cudaSuccess;
    if (!rec->empty()) e = cudaMemcpyAsync(rec->data(), ctx->series + T0 * RL, rec->size() * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return e;
    double accJ = 0.0, accV = 0.0;
    *nout = 0;
    for (size_t r = 0; r < rec->size() / RL; ++r) {
        const double *R_ = &(*rec)[r * RL];
        const int64_t n = (int64_t)llround(R_[0] / ctx->t.dt) - cur0;
        if (!(n > n_steps - window_steps && n <= n_steps)) continue;
        accJ += R_[1 + Q * 4 + 3];
        accV += R_[1 + Q * 4 + 4 + 3];
        ++*nout;
    }
    if (*nout > 0) { value[0] = accJ / *nout; value[1] = accV / *nout; }
    return cudaSuccess;
}

pgc_status pgc_window_objective(pgc_ctx *ctx, int64_t n_steps, int32_t moments_every, int64_t window_steps, double *h_value)
{
    if (!ctx) return PGC_EINVAL;
    if (ctx->failed) return afail(ctx, PGC_ESTATE, "context failed earlier");
    if (!h_value || n_steps < 1 || moments_every < 1 || window_steps < 1 || window_steps > n_steps)
        return afail(ctx, PGC_EINVAL, "need h_value, n_steps >= 1, moments_every >= 1 and 1 <= window_steps <= n_steps");
    const int64_t T0 = ctx->T_out, cur0 = ctx->step;
    pgc_status st = pgc_step(ctx, n_steps, moments_every);
    if (st != PGC_OK) return st;
    std::vector<double> rec;
    int64_t nout = 0;
    cudaError_t e = window_values(ctx, T0, cur0, n_steps, window_steps, &rec, h_value, &nout);
    if (e != cudaSuccess) return afail(ctx, PGC_ECUDA, std::string("moments: ") + cudaGetErrorString(e));
    if (nout == 0) return afail(ctx, PGC_EINVAL, "no moment output inside the window");
    return PGC_OK;
}

pgc_status pgc_adjoint(pgc_ctx *ctx, int64_t n_steps, int32_t ckpt_every, int32_t moments_every, int64_t window_steps,
                       const double *h_weights, void *d_work, double *h_value, double *h_grad)
{
    AdjLayout L;
    std::string msg;
    pgc_status st = adj_layout(ctx, n_steps, ckpt_every, &L, &msg);
    if (st != PGC_OK) { if (ctx) ctx->err = msg; return st; }
    if (ctx->failed) return afail(ctx, PGC_ESTATE, "context failed earlier");
    if (!ctx->sampled || ctx->step != 0) return afail(ctx, PGC_EINVAL, "the adjoint starts from the sampled initial state (step 0, no state upload)");
    if (ctx->cfg.eps0_law != PGC_EPS0_AFFINE)
        return afail(ctx, PGC_EUNSUPPORTED, "the adjoint differentiates the affine band-minimum endpoints (PGC_EPS0_AFFINE)");
    if (ctx->cfg.splitting != PGC_SPLIT_LIE)
        return afail(ctx, PGC_EUNSUPPORTED, "the adjoint differentiates the Lie splitting (PGC_SPLIT_LIE)");
    if (ctx->cfg.tc_proj != PGC_TC_OFF)
        return afail(ctx, PGC_EUNSUPPORTED, "the adjoint replays the FMA reconstruction of the streaming kernel (tc_proj must be PGC_TC_OFF)");
    if (ctx->t.final_state != PGC_FS_PAPER || ctx->t.pauli_mode == PGC_PAULI_CURRENT_MAX)
        return afail(ctx, PGC_EUNSUPPORTED, "the adjoint supports the paper's final states and the initial-maximum or off Pauli modes");
    if (moments_every < 1 || window_steps < 1 || window_steps > n_steps) return afail(ctx, PGC_EINVAL, "need moments_every >= 1 and 1 <= window_steps <= n_steps");
    if (!h_weights || !d_work || ((uintptr_t)d_work & 255)) return afail(ctx, PGC_EINVAL, "weights and a 256-byte aligned work buffer are required");
    const int64_t outs = n_steps / moments_every;
    if (ctx->T_out + outs > ctx->cfg.max_outputs) return afail(ctx, PGC_ENOMEM, "moment series would exceed max_outputs");
    const int Q = ctx->t.Q, K = ckpt_every;
    cudaStream_t s = ctx->stream;
    char *w = (char *)d_work;
    const int64_t cur0 = ctx->step;  // 0
    cudaError_t e = cudaSuccess;
    const size_t stbytes = (size_t)2 * ctx->t.P * ctx->b.ld * (ctx->cfg.precision == PGC_FP64 ? 8 : 4);
    const size_t hbytes = (size_t)Q * ctx->t.Nk * ctx->t.Nk * 4;

    // ---- forward with checkpoints (state and f^n at every segment start) ----
    const int64_t T0 = ctx->T_out;
    for (int64_t sgi = 0; sgi < L.nseg; ++sgi) {
        const int64_t n0 = sgi * K, n1 = std::min<int64_t>(n_steps, n0 + K);
        e = cudaMemcpyAsync(w + L.ckpt_state + sgi * L.state, ctx->b.state, stbytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(w + L.ckpt_hist + sgi * L.hist1, ctx->b.hist + (int64_t)(ctx->step % kHistBufs) * ctx->b.hist_stride,
                                hbytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return afail(ctx, PGC_ECUDA, std::string("checkpoint: ") + cudaGetErrorString(e));
        st = pgc_step(ctx, n1 - n0, moments_every);
        if (st != PGC_OK) return st;
    }
    // ---- objective from the recorded moments ----
    const int RL = ctx->rec_len;
    std::vector<double> rec;
    double value[2] = {0.0, 0.0};
    int64_t nout = 0;
    e = window_values(ctx, T0, cur0, n_steps, window_steps, &rec, value, &nout);
    if (e != cudaSuccess) return afail(ctx, PGC_ECUDA, std::string("moments: ") + cudaGetErrorString(e));
    if (nout == 0) return afail(ctx, PGC_EINVAL, "no moment output inside the window");
    std::vector<std::vector<double>> dLdJ(n_steps + 1);
    for (size_t r = 0; r < rec.size() / RL; ++r) {
        const double *R_ = &rec[r * RL];
        const int64_t n = (int64_t)llround(R_[0] / ctx->t.dt) - cur0;
        if (!(n > n_steps - window_steps && n <= n_steps)) continue;
        const double mean = R_[1 + Q * 4 + 3];
        dLdJ[n].assign(Q, 0.0);
        for (int q = 0; q < Q; ++q) {
            const double Jq = R_[1 + q * 4 + 3], wq = ctx->t.w[q];
            dLdJ[n][q] = (h_weights[0] * wq + h_weights[1] * 2.0 * wq * (Jq - mean)) / (double)nout;
        }
    }
    if (h_value) { h_value[0] = value[0]; h_value[1] = value[1]; }

    // ---- reverse sweep ----
    DevBuffers rb = ctx->b;  // the replay runs the forward kernels on the work buffers
    rb.state = w + L.replay_state;
    rb.hist = (uint32_t *)(w + L.replay_hist);
    rb.queue = (uint32_t *)(w + L.queue);
    rb.queue_stride = 0;   // one queue: the replay runs the two-launch form of the step
    rb.qcount = (uint32_t *)(w + L.qcount);
    rb.counters = (unsigned long long *)(w + L.counters);
    rb.part1 = (double *)(w + L.part1);
    rb.part1_stride = 0;
    rb.part2 = (double *)(w + L.part2);
    rb.partN = nullptr;
    rb.marks = nullptr;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    Runner *replay = make_runner(ctx->t.P, Q, ctx->cfg.precision, ctx->t, rb, sms);
    AdjBuffers ab;
    ab.lam = w + L.lam;
    ab.queue = (uint32_t *)(w + L.aqueue);
    ab.qcount = (uint32_t *)(w + L.aqcount);
    ab.grad = (double *)(w + L.grad);
    AdjRunner *adj = make_adj_runner(ctx->t.P, Q, ctx->cfg.precision, ctx->t, ctx->b, ab, sms);
    if (!replay || !adj) { delete replay; delete adj; return afail(ctx, PGC_EUNSUPPORTED, "no adjoint kernel for this shape"); }
    e = cudaMemsetAsync(w + L.lam, 0, L.state, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ab.grad, 0, NTH * 8, s);
    for (int64_t sgi = L.nseg - 1; sgi >= 0 && e == cudaSuccess; --sgi) {
        const int64_t n0 = sgi * K, n1 = std::min<int64_t>(n_steps, n0 + K);
        e = cudaMemcpyAsync(rb.state, w + L.ckpt_state + sgi * L.state, stbytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(rb.hist, 0, (size_t)kHistBufs * rb.hist_stride * 4, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(rb.hist + (int64_t)(n0 % kHistBufs) * rb.hist_stride, w + L.ckpt_hist + sgi * L.hist1, hbytes,
                                cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(rb.qcount, 0, 8 * 4, s);
        for (int64_t n = n0; n < n1 && e == cudaSuccess; ++n) {
            e = cudaMemcpyAsync(w + L.stack_state + (n - n0) * L.state, rb.state, stbytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(w + L.stack_hist + (n - n0) * L.hist1, rb.hist + (int64_t)(n % kHistBufs) * rb.hist_stride, hbytes,
                                    cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = replay->step(n, false, s);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(w + L.stack_state + (n1 - n0) * L.state, rb.state, stbytes, cudaMemcpyDeviceToDevice, s);
        for (int64_t n = n1 - 1; n >= n0 && e == cudaSuccess; --n) {
            const bool inj = !dLdJ[n + 1].empty();
            e = adj->backward_step(w + L.stack_state + (n - n0) * L.state, w + L.stack_state + (n + 1 - n0) * L.state,
                                   (const uint32_t *)(w + L.stack_hist + (n - n0) * L.hist1), n, inj,
                                   inj ? dLdJ[n + 1].data() : nullptr, s);
        }
    }
    if (e == cudaSuccess) e = adj->init_term(s);
    double g[NTH] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(g, ab.grad, NTH * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    delete replay;
    delete adj;
    if (e != cudaSuccess) return afail(ctx, PGC_ECUDA, std::string("adjoint: ") + cudaGetErrorString(e));
    if (h_grad)
        for (int k = 0; k < NTH; ++k) h_grad[k] = g[k];
    return PGC_OK;
}

}  // extern "C"
