// pgc_batch.cuh -- many ensembles ("cases": different fields and band-minimum intervals, uneven
// particle counts, the same basis and physics) advanced together by one persistent launch
// sequence per time step.
//
// The particles of all cases are cut into tiles of `tile` consecutive particles of one case; a
// persistent phase-1 grid walks the tile list (the case of a tile is found by binary search in
// a shared-memory prefix table, and its node tables are staged in shared memory).  The collider
// queue and the phase-2 kernel are shared by all cases; a queue entry is a global particle index
// whose case is again found by binary search.  The step index lives in device memory: phase 1
// and phase 2 read it, the last phase-2 block advances it, and a per-case finalize writes the
// moment record on moment steps.  No kernel argument depends on the step, so one time step is a
// fixed sequence of three launches that a CUDA graph can capture once and replay.
#pragma once

#include <algorithm>
#include <vector>

#include "pgc_runner_impl.cuh"

namespace pgc {

constexpr int kBatchMaxCases = 256;

template <int P, int Q, typename R>
struct CaseDev {
    Nodes<P, Q, R> nd;         // the case's tables (basis tables are identical across cases)
    R *khat;
    int64_t N, ld;
    uint32_t *hist;            // kHistBufs rotating buffers of the case
    int64_t hist_stride;
    const uint32_t *nmax;
    unsigned long long *counters;
    double *series;            // moment records of the case's context
    int64_t *t_out;            // device count of records (mirrors the context)
    double nq[Q], w[Q];
    uint32_t key0, key1, stream_id;
    int64_t tile0, ntiles;     // the case's tiles in the global tile list
    int64_t base;              // first global particle index of the case
};

template <int P, int Q, typename R>
struct BatchArgs {
    Phys<R> ph;
    CaseDev<P, Q, R> *cases;
    const int64_t *tile0s;     // [ncases + 1] tile prefix
    const int64_t *bases;      // [ncases + 1] particle prefix
    int32_t ncases;
    int64_t ntiles;
    int32_t tile;              // particles per tile (multiple of the phase-1 block pass)
    uint32_t *queue;           // [sum N]
    uint32_t *qcount;          // [2]
    double *part_tiles;        // [ntiles][Q*3]
    double *part2c;            // [ncases][Q*3]
    int64_t *d_step;
    uint32_t *done;            // phase-2 block completion counter
    int32_t moments_every;
    int32_t win_r0, use_win;
    int32_t rec_len;
    double vF_ms;
};

__device__ __forceinline__ int find_case(const int64_t *prefix, int n, int64_t x)
{
    int lo = 0, hi = n;  // prefix[lo] <= x < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// Particles per thread of the batched streaming kernel: the autotuner's choices for a shape
// (four, two or one for the small bases; one for P = 21).
template <int P> struct BatchPPTs { static constexpr int n = (P <= 8) ? 3 : 1; static constexpr int v[3] = {Phase1PPT<P>::value, 2, 1}; };

// Any block size up to kPhase1Threads that is a multiple of 32 (the autotuner uses 128 and 256).
template <int P, int Q, typename R, int PPT>
__global__ void __launch_bounds__(kPhase1Threads)
k_phase1_batch(const __grid_constant__ BatchArgs<P, Q, R> a)
{
    constexpr int NW = kPhase1Threads / 32;
    __shared__ typename MomAcc<R>::T smom[NW][Q * 3];
    __shared__ int64_t stile[kBatchMaxCases + 1];
    __shared__ __align__(16) uint32_t snd[(sizeof(Nodes<P, Q, R>) + 3) / 4];
    extern __shared__ uint32_t swin[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t step = *a.d_step;
    const int nxt = (int)((step + 1) % kHistBufs), clr = (int)((step + 2) % kHistBufs);
    const bool out = a.moments_every > 0 && ((step + 1) % a.moments_every == 0);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.qcount[(step + 1) & 1] = 0u;
    for (int j = threadIdx.x; j <= a.ncases; j += blockDim.x) stile[j] = a.tile0s[j];
    __syncthreads();
    const int64_t NN = (int64_t)a.ph.Nk * a.ph.Nk;
    const int64_t helems = (int64_t)Q * NN;
    int cur = -1;
    unsigned int oog = 0u;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int c = find_case(stile, a.ncases + 1, tile);
        const CaseDev<P, Q, R> &cd = a.cases[c];
        __syncthreads();  // previous tile done with the window and the staged tables
        if (c != cur) {
            stage(snd, cd.nd);
            cur = c;
        }
        if (a.use_win)
            for (int j = threadIdx.x; j < Q * kWinWords; j += blockDim.x) swin[j] = 0u;
        if (out)
            for (int j = lane; j < Q * 3; j += 32) acc_zero(smom[warp][j]);
        // this tile's share of clearing the case's buffer of step n+2
        {
            const int64_t t = tile - cd.tile0;
            const int64_t chunk = ((helems + cd.ntiles - 1) / cd.ntiles + 3) & ~(int64_t)3;
            uint32_t *Hc = cd.hist + (int64_t)clr * cd.hist_stride;
            const int64_t lo = t * chunk, hi = min(helems, lo + chunk);
            for (int64_t j = lo + 4 * (int64_t)threadIdx.x; j < hi; j += 4 * (int64_t)blockDim.x) {
                if (j + 4 <= hi) *reinterpret_cast<uint4 *>(Hc + j) = make_uint4(0u, 0u, 0u, 0u);
                else for (int64_t k = j; k < hi; ++k) Hc[k] = 0u;
            }
        }
        __syncthreads();
        const Nodes<P, Q, R> &nd = *reinterpret_cast<const Nodes<P, Q, R> *>(snd);
        P1Target<R> t;
        t.khat = cd.khat; t.N = cd.N; t.ld = cd.ld;
        t.Hnext = cd.hist + (int64_t)nxt * cd.hist_stride;
        t.qcount = a.qcount + (step & 1); t.queue = a.queue; t.qoffset = (uint32_t)cd.base;
        t.key0 = cd.key0; t.key1 = cd.key1; t.stream_id = cd.stream_id; t.step = (uint32_t)step;
        const int64_t p0 = (tile - cd.tile0) * a.tile;
        const int64_t p1 = min(cd.N, p0 + a.tile);
        for (int64_t base = p0; base < p1; base += (int64_t)blockDim.x * PPT)
            phase1_pass<P, Q, R, PPT>(a.ph, nd, t, base + (int64_t)threadIdx.x * PPT, swin, a.win_r0, a.use_win != 0,
                                      out, smom[warp], oog);
        __syncthreads();
        if (a.use_win) flush_window<Q>(swin, t.Hnext, a.ph.Nk, a.win_r0);
        if (out)
            for (int j = threadIdx.x; j < Q * 3; j += blockDim.x) {
                double s = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += acc_value(smom[w][j]);   // fixed order
                a.part_tiles[tile * (Q * 3) + j] = s;
            }
        oog = warp_sum(oog);
        if (lane == 0 && oog) atomicAdd(&cd.counters[4], (unsigned long long)oog);
        oog = 0u;
    }
}

template <int P, int Q, typename R>
__global__ void __launch_bounds__(kPhase2Threads)
k_phase2_batch(const __grid_constant__ BatchArgs<P, Q, R> a)
{
    constexpr int G = GroupOf<Q>::G;
    __shared__ int64_t sbase[kBatchMaxCases + 1];
    __shared__ uint32_t scnt[kBatchMaxCases][5];   // per-case counters of this block
    __shared__ R sred[ProjRed<P, Q, R>::value ? (kPhase2Threads / 32) * ProjRed<P, Q, R>::warp_elems : 1];
    for (int j = threadIdx.x; j <= a.ncases; j += blockDim.x) sbase[j] = a.bases[j];
    for (int j = threadIdx.x; j < a.ncases * 5; j += blockDim.x) (&scnt[0][0])[j] = 0u;
    __syncthreads();
    const Phys<R> &ph = a.ph;   // read alike by all lanes: stays in the parameter bank
    const int64_t step = *a.d_step;
    const int cur = (int)(step % kHistBufs), nxt = (int)((step + 1) % kHistBufs);
    const bool out = a.moments_every > 0 && ((step + 1) % a.moments_every == 0);
    const uint32_t count = a.qcount[step & 1];

    const int lane = threadIdx.x & 31;
    const int r = lane % G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane - r));
    const uint32_t gid = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    const uint32_t ngroups = gridDim.x * blockDim.x / G;
    for (uint32_t j = gid; j < count; j += ngroups) {
        const int64_t g = a.queue[j];
        const int c = find_case(sbase, a.ncases + 1, g);
        const CaseDev<P, Q, R> &cd = a.cases[c];
        P2Target<R> t;
        t.khat = cd.khat; t.ld = cd.ld;
        t.Hcur = cd.hist + (int64_t)cur * cd.hist_stride;
        t.Hnext = cd.hist + (int64_t)nxt * cd.hist_stride;
        t.nmax = cd.nmax;
        t.mom = a.part2c + (int64_t)c * (Q * 3);
        t.key0 = cd.key0; t.key1 = cd.key1; t.stream_id = cd.stream_id; t.step = (uint32_t)step;
        t.out_step = out;
        t.red = sred;
        P2Counts cnt;
        collide_particle<P, Q, R>(ph, cd.nd, t, g - sbase[c], r, gmask, cnt);
        if (cnt.att) atomicAdd(&scnt[c][0], (uint32_t)cnt.att);
        if (cnt.chg) atomicAdd(&scnt[c][1], (uint32_t)cnt.chg);
        if (cnt.rej) atomicAdd(&scnt[c][2], (uint32_t)cnt.rej);
        if (cnt.cap) atomicAdd(&scnt[c][3], (uint32_t)cnt.cap);
        if (cnt.oog) atomicAdd(&scnt[c][4], (uint32_t)cnt.oog);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < a.ncases * 5; j += blockDim.x) {
        const uint32_t v = (&scnt[0][0])[j];
        if (v) atomicAdd(&a.cases[j / 5].counters[j % 5], (unsigned long long)v);
    }
    // the last block to finish advances the step index (no block waits for another)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t prev = atomicAdd(a.done, 1u);
        if (prev == gridDim.x - 1) {
            *a.done = 0u;
            *a.d_step = step + 1;
            __threadfence();
        }
    }
}

// Per-case moment record on moment steps (one block per case, fixed-order sums).
template <int P, int Q, typename R>
__global__ void __launch_bounds__(256)
k_finalize_batch(const __grid_constant__ BatchArgs<P, Q, R> a)
{
    __shared__ double red[256];
    __shared__ double S[Q * 3];
    const int64_t step = *a.d_step;  // already advanced: the post-step index
    if (!(a.moments_every > 0 && step % a.moments_every == 0)) return;
    const int c = blockIdx.x;
    CaseDev<P, Q, R> &cd = a.cases[c];
    constexpr int n3 = Q * 3;
    const int nslot = 256 / n3;
    const int t = threadIdx.x, col = t % n3, slot = t / n3;
    double s = 0.0;
    if (slot < nslot) s = strided_sum(a.part_tiles, cd.tile0 + slot, cd.tile0 + cd.ntiles, nslot, n3, col, s);
    red[t] = s;
    __syncthreads();
    if (t < n3) {
        double acc = 0.0;
        for (int k = 0; k < nslot; ++k) acc += red[k * n3 + t];
        acc += a.part2c[(int64_t)c * n3 + t];
        a.part2c[(int64_t)c * n3 + t] = 0.0;
        S[t] = acc;
    }
    __syncthreads();
    // node values, one thread per node, then the mean and variance by one thread in node order
    __shared__ double V[Q * 4];
    double *rec = cd.series + (*cd.t_out) * a.rec_len;
    if (t < Q) {
        const double qe = 1.602176634e-19;
        const int q = t;
        const double vx = S[q * 3 + 0] / (double)cd.N * a.vF_ms, vy = S[q * 3 + 1] / (double)cd.N * a.vF_ms;
        const double en = S[q * 3 + 2] / (double)cd.N, jx = -qe * cd.nq[q] * vx;
        const double v[4] = {vx, vy, en, jx};
        for (int o = 0; o < 4; ++o) {
            V[q * 4 + o] = v[o];
            rec[1 + q * 4 + o] = v[o];
        }
    }
    __syncthreads();
    if (t == 0) {
        rec[0] = (double)step * (double)a.ph.dt;
        double m[4] = {0, 0, 0, 0}, m2[4] = {0, 0, 0, 0};
        for (int q = 0; q < Q; ++q)
            for (int o = 0; o < 4; ++o) {
                const double v = V[q * 4 + o];
                m[o] += cd.w[q] * v;
                m2[o] += cd.w[q] * v * v;
            }
        for (int o = 0; o < 4; ++o) {
            rec[1 + Q * 4 + o] = m[o];
            rec[1 + Q * 4 + 4 + o] = m2[o] - m[o] * m[o];
        }
        *cd.t_out += 1;
    }
}

// ------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------
struct BatchCase {
    const HostTables *t;
    DevBuffers b;
    double *series;
};

struct BatchScratch {
    void *cases = nullptr;     // [n] CaseDev
    int64_t *tile0s = nullptr, *bases = nullptr;
    uint32_t *queue = nullptr, *qcount = nullptr, *done = nullptr;
    int64_t *d_step = nullptr, *t_out = nullptr;
    double *part_tiles = nullptr, *part2c = nullptr;
    int64_t max_tiles = 0;
};

// Launch configuration of a batch: particles per tile, threads per streaming block, particles
// per thread, streaming and collider blocks per SM.  None of it changes a trajectory (only the
// grouping of the FP32 warp sums of the moments).
struct BatchLaunch {
    int tile = 0, block = kPhase1Threads, ppt = 1, g1_per_sm = 1, g2_per_sm = 4;
};

class BatchRunner {
public:
    virtual ~BatchRunner() {}
    // set the tile size (particles, a multiple of pass()) and upload the case table
    virtual cudaError_t set_tile(int tile, cudaStream_t s) = 0;
    virtual int tile() const = 0;
    virtual int pass() const = 0;
    // block size, particles per thread and the two grids (not the tile: call set_tile after);
    // cudaErrorInvalidValue for a configuration this shape cannot run
    virtual cudaError_t set_launch(int block, int ppt, int g1_per_sm, int g2_per_sm) = 0;
    virtual BatchLaunch launch() const = 0;
    // the choices: particles per thread, and the most blocks per SM of each kernel
    virtual std::vector<int> ppts() const = 0;
    virtual int max_g1(int block, int ppt) const = 0;
    virtual int max_g2() const = 0;
    virtual void set_moments_every(int every) = 0;
    // one time step: phase 1, phase 2, finalize (3 launches, step index on the device)
    virtual cudaError_t step(cudaStream_t s) = 0;
};

template <int P, int Q, typename R>
class BatchRunnerT final : public BatchRunner {
public:
    BatchRunnerT(const std::vector<BatchCase> &cases, const BatchScratch &sc, int num_sms) : cases_(cases), sc_(sc)
    {
        const HostTables &t0 = *cases[0].t;
        // physics shared by all cases: take it from a single-case runner's argument block
        RunnerT<P, Q, R> proto(t0, cases[0].b, num_sms);
        a_.ph = proto.args().ph;
        a_.cases = static_cast<CaseDev<P, Q, R> *>(sc.cases);
        a_.tile0s = sc.tile0s;
        a_.bases = sc.bases;
        a_.ncases = (int)cases.size();
        a_.queue = sc.queue;
        a_.qcount = sc.qcount;
        a_.part_tiles = sc.part_tiles;
        a_.part2c = sc.part2c;
        a_.d_step = sc.d_step;
        a_.done = sc.done;
        a_.moments_every = 0;
        a_.win_r0 = proto.args().win_r0;
        a_.use_win = proto.args().use_win;
        a_.rec_len = 1 + 4 * Q + 8;
        a_.vF_ms = t0.vF_ms;
        win_bytes_ = a_.use_win ? (size_t)Q * kWinWords * 4 : 0;
        num_sms_ = num_sms;
        for (int j = 0; j < BatchPPTs<P>::n; ++j)
            if (win_bytes_) cudaFuncSetAttribute(kernel1(BatchPPTs<P>::v[j]), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)win_bytes_);
        // defaults: 256 threads, the shape's particles per thread, all resident streaming blocks,
        // four collider blocks per SM
        set_launch(kPhase1Threads, Phase1PPT<P>::value, max_g1(kPhase1Threads, Phase1PPT<P>::value), 4);
        host_.resize(cases.size());
        for (size_t c = 0; c < cases.size(); ++c) {
            RunnerT<P, Q, R> rc(*cases[c].t, cases[c].b, num_sms);
            CaseDev<P, Q, R> &d = host_[c];
            d.nd = rc.args().nd;
            d.khat = static_cast<R *>(cases[c].b.state);
            d.N = cases[c].b.N;
            d.ld = cases[c].b.ld;
            d.hist = cases[c].b.hist;
            d.hist_stride = cases[c].b.hist_stride;
            d.nmax = cases[c].b.nmax;
            d.counters = cases[c].b.counters;
            d.series = cases[c].series;
            d.t_out = sc.t_out + c;
            for (int q = 0; q < Q; ++q) { d.nq[q] = cases[c].t->nq[q]; d.w[q] = cases[c].t->w[q]; }
            d.key0 = cases[c].b.key0;
            d.key1 = cases[c].b.key1;
            d.stream_id = cases[c].b.stream_id;
        }
    }

    int pass() const override { return lc_.block * lc_.ppt; }
    int tile() const override { return a_.tile; }
    BatchLaunch launch() const override { BatchLaunch l = lc_; l.tile = a_.tile; return l; }
    std::vector<int> ppts() const override { return std::vector<int>(BatchPPTs<P>::v, BatchPPTs<P>::v + BatchPPTs<P>::n); }

    int max_g1(int block, int ppt) const override
    {
        const void *k = kernel1(ppt);
        int per_sm = 0;
        if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, win_bytes_) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return per_sm;
    }
    int max_g2() const override
    {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_phase2_batch<P, Q, R>, kPhase2Threads, 0) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return per_sm;
    }

    cudaError_t set_launch(int block, int ppt, int g1_per_sm, int g2_per_sm) override
    {
        if ((block != 128 && block != 256) || !kernel1(ppt)) return cudaErrorInvalidValue;
        if (g1_per_sm < 1 || g1_per_sm > max_g1(block, ppt) || g2_per_sm < 1 || g2_per_sm > max_g2())
            return cudaErrorInvalidValue;
        lc_.block = block;
        lc_.ppt = ppt;
        lc_.g1_per_sm = g1_per_sm;
        lc_.g2_per_sm = g2_per_sm;
        return cudaSuccess;
    }
    void set_moments_every(int every) override { a_.moments_every = every; }

    cudaError_t set_tile(int tile, cudaStream_t s) override
    {
        std::vector<int64_t> t0(cases_.size() + 1), b0(cases_.size() + 1);
        int64_t nt = 0, nb = 0;
        for (size_t c = 0; c < cases_.size(); ++c) {
            const int64_t n = cases_[c].b.N;
            host_[c].tile0 = nt;
            host_[c].ntiles = (n + tile - 1) / tile;
            host_[c].base = nb;
            t0[c] = nt;
            b0[c] = nb;
            nt += host_[c].ntiles;
            nb += n;
        }
        t0[cases_.size()] = nt;
        b0[cases_.size()] = nb;
        if (nt > sc_.max_tiles) return cudaErrorInvalidValue;
        a_.tile = tile;
        a_.ntiles = nt;
        cudaError_t e = cudaMemcpyAsync(sc_.cases, host_.data(), host_.size() * sizeof(CaseDev<P, Q, R>), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sc_.tile0s, t0.data(), t0.size() * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sc_.bases, b0.data(), b0.size() * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host_ and the prefix vectors are reused
        return e;
    }

    cudaError_t step(cudaStream_t s) override
    {
        const int g1 = num_sms_ * lc_.g1_per_sm, g2 = num_sms_ * lc_.g2_per_sm;
        switch (lc_.ppt) {
        case 4: if constexpr (BatchPPTs<P>::n == 3) k_phase1_batch<P, Q, R, 4><<<g1, lc_.block, win_bytes_, s>>>(a_); break;
        case 2: if constexpr (BatchPPTs<P>::n == 3) k_phase1_batch<P, Q, R, 2><<<g1, lc_.block, win_bytes_, s>>>(a_); break;
        default: k_phase1_batch<P, Q, R, 1><<<g1, lc_.block, win_bytes_, s>>>(a_); break;
        }
        k_phase2_batch<P, Q, R><<<g2, kPhase2Threads, 0, s>>>(a_);
        k_finalize_batch<P, Q, R><<<a_.ncases, 256, 0, s>>>(a_);
        count_launch(3);
        return cudaGetLastError();
    }

private:
    // the streaming kernel for ppt particles per thread (nullptr if not compiled for this shape)
    static const void *kernel1(int ppt)
    {
        if constexpr (BatchPPTs<P>::n == 3) {
            if (ppt == 4) return (const void *)k_phase1_batch<P, Q, R, 4>;
            if (ppt == 2) return (const void *)k_phase1_batch<P, Q, R, 2>;
        }
        if (ppt == 1) return (const void *)k_phase1_batch<P, Q, R, 1>;
        return nullptr;
    }

    std::vector<BatchCase> cases_;
    BatchScratch sc_;
    BatchArgs<P, Q, R> a_{};
    std::vector<CaseDev<P, Q, R>> host_;
    size_t win_bytes_ = 0;
    int num_sms_ = 1;
    BatchLaunch lc_;
};

template <int P, int Q>
BatchRunner *make_batch_runner_shape(int precision, const std::vector<BatchCase> &cases, const BatchScratch &sc, int num_sms)
{
    if (precision == 1) return new BatchRunnerT<P, Q, double>(cases, sc, num_sms);
    return new BatchRunnerT<P, Q, float>(cases, sc, num_sms);
}

template <int P, int Q>
size_t case_dev_bytes(int precision)
{
    return precision == 1 ? sizeof(CaseDev<P, Q, double>) : sizeof(CaseDev<P, Q, float>);
}

}  // namespace pgc
