// pgc_runner_impl.cuh -- the templated Runner: fills the kernel argument blocks from the host
// tables and launches the kernels of pgc_kernels.cuh.  Included by the per-shape instantiation
// units so that the shapes compile in parallel.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>

#include "pgc_kernels.cuh"
#include "pgc_kernels_tc.cuh"
#include "pgc_runner.h"

namespace pgc {

template <int P, int Q, typename R>
class RunnerT final : public Runner {
public:
    RunnerT(const HostTables &t, const DevBuffers &b, int num_sms) : t_(t), b_(b), num_sms_(num_sms)
    {
        fill_phys(t);
        auto &nd = args_.nd;
        for (int i = 0; i < Q * P; ++i) { nd.psi[i] = (R)t.psi[i]; nd.wpsi[i] = (R)t.wpsi[i]; }
        for (int h = 0; h < P; ++h) nd.dhat[h] = (R)t.dhat[h];
        for (int q = 0; q < Q; ++q) {
            nd.eps0[q] = (R)t.eps0[q];
            nd.dq[q] = (R)t.dq[q];
            nd.lkx[q] = (R)(t.Lk - t.xs[q]);   // Lie: the grid's Lk itself
            nd.xs[q] = (R)t.xs[q];
        }
        nd.eps0_max = (R)t.eps0_max;
        if constexpr (TensorShape<P, Q>::value) {
            // psi(q1,q2) = a_h1(z1_q1) b_h2(z2_q2) with a_0 = b_0 = 1
            for (int q = 0; q < 6; ++q)
                for (int h = 0; h < 6; ++h) {
                    nd.a1[q * 6 + h] = (R)t.psi[(size_t)(q * 6) * P + hidx2(h, 0)];
                    nd.b2[q * 6 + h] = (R)t.psi[(size_t)q * P + hidx2(0, h)];
                }
        }
        nd.drift_mask = t.drift_mask;
        // (w, w) pairs of the FP32 weights for the two-lane FMA
        auto pair = [](double w) {
            const float f = (float)w;
            uint32_t u;
            std::memcpy(&u, &f, 4);
            return ((unsigned long long)u << 32) | u;
        };
        if constexpr (!TensorShape<P, Q>::value && sizeof(R) == 4)
            for (int i = 0; i < Q * P; ++i) { nd.psi2[i] = pair(t.psi[i]); nd.wpsi2[i] = pair(t.wpsi[i]); }
        for (int i = 0; i < 36; ++i) { nd.a1_2[i] = pair((double)nd.a1[i]); nd.b2_2[i] = pair((double)nd.b2[i]); }
        args_.khat = static_cast<R *>(b.state);
        args_.N = b.N;
        args_.ld = b.ld;
        args_.hist_elems = (int64_t)Q * t.Nk * t.Nk;
        args_.nmax = b.nmax;
        args_.queue = b.queue;
        args_.part1 = b.part1;
        args_.part2 = b.part2;
        args_.mark_words = b.mark_words;
        static_assert(sizeof(Nodes<P, Q, R>) <= kTableBytes, "node tables exceed their device region");
        args_.nd_dev = b.tables ? static_cast<const Nodes<P, Q, R> *>(b.tables) : nullptr;
        args_.counters = b.counters;
        args_.key0 = b.key0;
        args_.key1 = b.key1;
        args_.stream_id = b.stream_id;
        for (int i = 0; i < Q * P; ++i) init_.wpsi[i] = t.wpsi[i];
        for (int q = 0; q < Q; ++q) init_.eps0[q] = t.eps0[q];
        init_.mu = t.mu;
        init_.kT = t.kT;
        init_.hvF = t.hvF;
        for (int h = 0; h < P; ++h) init_.dhalf[h] = t.dhalf[h];
        init_.strang = t.strang ? 1 : 0;
        init_.N = b.N;
        init_.ld = b.ld;
        init_.key0 = b.key0;
        init_.key1 = b.key1;
        init_.stream_id = b.stream_id;
        // phase-1 grid: enough resident blocks to fill the GPU, PPT particles per thread; the
        // shared-memory histogram window lies inside the grid (its 16-bit cells are flushed by
        // the block before they could overflow, at any N)
        constexpr int PPT = Phase1PPT<P>::value;
        win_bytes_ = (size_t)Q * kWinWords * 4;
        args_.win_r0 = std::max(0, t.Nk / 2 - kWin / 2);
        bool win = t.Nk >= kWin && win_bytes_ <= 160 * 1024;
        if (win && (cudaFuncSetAttribute(k_phase1<P, Q, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)win_bytes_) != cudaSuccess ||
                    !fused_attr())) {
            cudaGetLastError();
            win = false;
        }
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_phase1<P, Q, R>, kPhase1Threads, win ? win_bytes_ : 0);
        per_sm = std::max(per_sm, 1);
        const int64_t need = (b.N + (int64_t)kPhase1Threads * PPT - 1) / ((int64_t)kPhase1Threads * PPT);
        grid1_ = (int)std::max<int64_t>(1, std::min<int64_t>({need, (int64_t)num_sms * per_sm, (int64_t)kMaxGrid1}));
        args_.use_win = win ? 1 : 0;
        if (!win) win_bytes_ = 0;
        // phase 2: one resident wave (its work is one latency-bound collision chain per group)
        int per_sm2 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_phase2<P, Q, R, true>, kPhase2Threads, 0);
        grid2_ = std::max(1, std::min(P * Q > 64 ? kGrid2Max : kGrid2, num_sms * std::max(per_sm2, 1)));
        // the fused step kernel: as many collider groups as grid2_ blocks of phase 2 carry
        grid2f_ = std::max(1, grid2_ * kPhase2Threads / kPhase1Threads);
    }

    int grid1() const override { return grid1_; }
    int grid2() const override { return grid2_; }
    int grid2f() const override { return grid2f_; }
    const StepArgs<P, Q, R> &args() const { return args_; }

    cudaError_t init_sample(cudaStream_t s) override
    {
        int blocks = (int)std::min<int64_t>((b_.N + 127) / 128, 8192);
        k_init<P, Q, R><<<blocks, 128, 0, s>>>(init_, args_.khat);
        count_launch();
        return cudaGetLastError();
    }

    cudaError_t observe(int buf, cudaStream_t s) override
    {
        StepArgs<P, Q, R> a = args_;
        a.Hnext = b_.hist + (int64_t)buf * b_.hist_stride;
        a.out_step = 1;
        k_observe<P, Q, R><<<grid1_, kPhase1Threads, 0, s>>>(a);
        count_launch();
        return cudaGetLastError();
    }

    cudaError_t observe_into(uint32_t *hist, double *part, cudaStream_t s) override
    {
        StepArgs<P, Q, R> a = args_;
        a.Hnext = hist;
        a.part1 = part;
        a.out_step = 1;
        k_observe<P, Q, R><<<grid1_, kPhase1Threads, 0, s>>>(a);
        count_launch();
        return cudaGetLastError();
    }

    // arguments of step n: buffer rotation (kHistBufs histograms, kQSlots counters, two queues
    // and moment slots, kMarkSlots bitmaps)
    StepArgs<P, Q, R> args_at(int64_t n) const
    {
        StepArgs<P, Q, R> a = args_;
        auto H = [&](int64_t m) { return b_.hist + (int64_t)(m % kHistBufs) * b_.hist_stride; };
        auto M = [&](int64_t m) { return b_.marks ? b_.marks + (int64_t)(m % kMarkSlots) * b_.mark_words : nullptr; };
        a.Hcur = H(n);
        a.Hnext = H(n + 1);
        a.Hnext2 = H(n + 2);
        a.Hclear = H(n + 2);
        a.qcount = b_.qcount + (int)(n % kQSlots);
        a.qcount_next = b_.qcount + (int)((n + 1) % kQSlots);
        a.tilectr = nullptr;
        a.tilectr_next = b_.qcount + 4 + (int)((n + 1) % kQSlots);
        a.queue = b_.queue + (n & 1) * b_.queue_stride;
        a.queue_next = b_.queue + ((n + 1) & 1) * b_.queue_stride;
        a.mark = M(n);
        a.mark_next = M(n + 1);
        a.mark_clear = M(n + 1);
        a.skip = nullptr;
        a.part1 = b_.part1 + (n % kPartSlots) * b_.part1_stride;
        a.part2 = b_.part2 + (n % kPartSlots) * b_.part2_stride;
        a.partN = b_.partN ? b_.partN + ((n + 1) % kPartSlots) * (int64_t)kGrid2Max * Q * 3 : nullptr;
        a.step = (uint32_t)n;
        return a;
    }

    cudaError_t phase1(int64_t n, bool out_step, cudaStream_t s) override
    {
        StepArgs<P, Q, R> a = args_at(n);
        a.out_step = out_step ? 1 : 0;
        if constexpr (TensorShape<P, Q>::value && sizeof(R) == 4) {
            if (tc_mode_) {
                k_phase1_tc<P, Q><<<grid1_, kTcThreads, TcSmem<Q>::bytes, s>>>(a, tc_mode_);
                count_launch();
                return cudaGetLastError();
            }
        }
        k_phase1<P, Q, R><<<grid1_, kPhase1Threads, win_bytes_, s>>>(a);
        count_launch();
        return cudaGetLastError();
    }

    // The tensor-core streaming kernel: one CTA per SM (its shared memory admits no second
    // one, which also keeps its 512 TMEM columns to itself), 4 tiles of 128 particles per CTA
    // and iteration.  The phase-1 grid (and with it the moment partials of k_observe and
    // k_finalize) becomes that kernel's grid.
    cudaError_t set_tc(int mode) override
    {
        if constexpr (TensorShape<P, Q>::value && sizeof(R) == 4) {
            if (mode == 0) return cudaSuccess;
            if (mode != 1 && mode != 2) return cudaErrorInvalidValue;
            cudaError_t e = cudaFuncSetAttribute(k_phase1_tc<P, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)TcSmem<Q>::bytes);
            if (e != cudaSuccess) return e;
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_phase1_tc<P, Q>, kTcThreads, TcSmem<Q>::bytes);
            if (e != cudaSuccess) return e;
            if (per_sm != 1) return cudaErrorNotSupported;   // TMEM is sized for one CTA per SM
            const int64_t tiles = (b_.N + 127) / 128;
            grid1_ = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + kTcWG - 1) / kTcWG, num_sms_));
            tc_mode_ = mode;
            return cudaSuccess;
        } else {
            (void)mode;
            return cudaErrorNotSupported;
        }
    }

    cudaError_t phase2(int64_t n, bool out_step, cudaStream_t s) override
    {
        StepArgs<P, Q, R> a = args_at(n);
        a.out_step = out_step ? 1 : 0;
        k_phase2<P, Q, R, false><<<grid2_, kPhase2Threads, 0, s>>>(a);
        count_launch();
        return cudaGetLastError();
    }

    // the fused kernel takes two argument blocks: compiled where both fit the kernel-parameter
    // space (32764 bytes; all shapes but the 36-node FP64 one)
    static constexpr bool kFused = 2 * sizeof(StepArgs<P, Q, R>) + sizeof(int) <= 32764;
    bool fused() const override { return kFused && tc_mode_ == 0; }   // the fused kernel reconstructs on the FMA pipes

    // dynamic shared memory of the fused kernel: the phase-1 window, or the projection area of
    // its phase-2 blocks (ProjRed shapes), whichever is larger
    size_t fused_smem() const
    {
        const size_t red = ProjRed<P, Q, R>::value ? (size_t)(kPhase1Threads / 32) * ProjRed<P, Q, R>::warp_elems * sizeof(R) : 0;
        return std::max(win_bytes_, red);
    }

    bool fused_attr()
    {
        if constexpr (kFused)
            return cudaFuncSetAttribute(k_step<P, Q, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem()) == cudaSuccess;
        return true;
    }

    cudaError_t step_fused(int64_t n, bool out_n, bool out_prev, cudaStream_t s) override
    {
        if constexpr (!kFused) {
            (void)n; (void)out_n; (void)out_prev; (void)s;
            return cudaErrorNotSupported;
        } else {
        if (!(b_.marks && b_.partN)) return cudaErrorInvalidValue;
        StepArgs<P, Q, R> a1 = args_at(n), a2 = args_at(n - 1);
        a1.out_step = out_n ? 1 : 0;
        a1.skip = b_.marks + (int64_t)((n - 1) % kMarkSlots) * b_.mark_words;
        a1.tilectr = b_.qcount + 4 + (int)(n % kQSlots);
        a2.out_step = out_prev ? 1 : 0;
        a2.out_next = out_n ? 1 : 0;
        k_step<P, Q, R><<<grid2f_ + grid1_, kPhase1Threads, fused_smem(), s>>>(a1, a2, grid2f_);
        count_launch();
        return cudaGetLastError();
        }
    }

    cudaError_t upload_tables(cudaStream_t s) override
    {
        if (!b_.tables) return cudaSuccess;
        return cudaMemcpyAsync(b_.tables, &args_.nd, sizeof(Nodes<P, Q, R>), cudaMemcpyHostToDevice, s);
    }

    cudaError_t step(int64_t step, bool out_step, cudaStream_t s, cudaEvent_t *ev) override
    {
        if (ev) cudaEventRecord(ev[0], s);
        cudaError_t e = phase1(step, out_step, s);
        if (ev) { cudaEventRecord(ev[1], s); cudaEventRecord(ev[2], s); }
        if (e == cudaSuccess) e = phase2(step, out_step, s);
        if (ev) cudaEventRecord(ev[3], s);
        return e;
    }

    cudaError_t hist_at(const double *psi, double xs, uint32_t *out, cudaStream_t s) override
    {
        ReconArgs<P, Q, R> z;
        for (int h = 0; h < P; ++h) z.psi[h] = psi[h];
        z.lkx = (R)(t_.Lk - xs);
        int blocks = (int)std::min<int64_t>((b_.N + 255) / 256, 4096);
        k_hist_at<P, Q, R><<<blocks, 256, 0, s>>>(args_, z, out);
        count_launch();
        return cudaGetLastError();
    }

    cudaError_t obs_at(const double *psi, const double *eps0, const double *xs, int nzc, double *part, int *blocks,
                       cudaStream_t s) override
    {
        ObsArgs<P, R> o;
        o.khat = args_.khat;
        o.ld = b_.ld;
        o.N = b_.N;
        o.hvF2 = args_.ph.hvF2;
        for (int l = 0; l < kObsZ; ++l) {
            for (int h = 0; h < P; ++h) o.psi[l * P + h] = (l < nzc) ? (R)psi[(size_t)l * P + h] : (R)0;
            const R e = (l < nzc) ? (R)eps0[l] : (R)1;
            o.e0sq[l] = e * e;   // as the node observables square the band minimum
            o.xs[l] = (l < nzc) ? (R)xs[l] : (R)0;
        }
        constexpr int T = ObsTile<P, R>::value;
        const int g = (int)std::min<int64_t>((b_.N + T - 1) / T, kObsGrid);
        *blocks = g;
        k_obs_at<P, R><<<g, kObsThreads, 0, s>>>(o, part);
        count_launch();
        return cudaGetLastError();
    }

private:
    void fill_phys(const HostTables &t)
    {
        Phys<R> &p = args_.ph;
        p.hvF = (R)t.hvF;
        p.hvF2 = (R)(t.hvF * t.hvF);
        p.Lk = (R)t.Lk;
        p.dk = (R)t.dk;
        p.inv_dk = (R)(1.0 / t.dk);
        p.alpha1 = (R)(1.0 + t.alpha);
        p.dt = (R)t.dt;
        p.Cac = (R)t.Cac;
        p.COm = (R)(t.CO * (t.nO + 1.0));
        p.COp = (R)(t.CO * t.nO);
        p.CKm = (R)(t.CK * (t.nK + 1.0));
        p.CKp = (R)(t.CK * t.nK);
        p.hwO = (R)t.hwO;
        p.hwK = (R)t.hwK;
        p.wOk = (R)(t.hwO / t.hvF);
        p.wKk = (R)(t.hwK / t.hvF);
        p.Cedg = (R)t.Cedg;
        p.two_a2 = (R)(2.0 * t.a_nm * t.a_nm);
        p.edge_h = (R)(2.0 * kPi / t.n_theta);
        p.bound_edge = (R)(2.0 * kPi * (1.0 + 1e-5));
        p.vF_ms = (R)t.vF_ms;
        const double h = 2.0 * kPi / t.n_theta;
        for (int j = 0; j <= kMaxTheta; ++j) p.cosj[j] = (R)((j <= t.n_theta) ? std::cos(j * h) : 1.0);
        // edge-integral series: a[j][m] = (-1)^j / j! C(2j,2m) C(2m,m) 4^-m
        p.J = (sizeof(R) == 8) ? 16 : 10;
        p.beta_ser = (R)((t.n_theta >= 32) ? 0.25 : 0.0);
        auto binom = [](int n, int k) { double r = 1.0; for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i; return r; };
        for (int j = 0; j < kSerMax; ++j) {
            double fact = 1.0;
            for (int i = 2; i <= j; ++i) fact *= i;
            for (int m = 0; m < kSerMax; ++m)
                p.tser[j * kSerMax + m] = (R)((m <= j) ? ((j & 1) ? -1.0 : 1.0) / fact * binom(2 * j, 2 * m) * binom(2 * m, m) / std::pow(4.0, m) : 0.0);
        }
        p.mech = t.mech;
        p.n_theta = t.n_theta;
        p.pauli_mode = t.pauli_mode;
        p.final_state = t.final_state;
        p.max_coll = t.max_coll;
        p.Nk = t.Nk;
    }

    HostTables t_;
    DevBuffers b_;
    StepArgs<P, Q, R> args_{};
    InitArgs<P, Q> init_{};
    int grid1_ = 1;
    size_t win_bytes_ = 0;
    int grid2_ = 1;
    int grid2f_ = 1;
    int num_sms_ = 1;
    int tc_mode_ = 0;
};

template <int P, int Q>
Runner *make_runner_shape(int precision, const HostTables &t, const DevBuffers &b, int num_sms)
{
    if (precision == 1) return new RunnerT<P, Q, double>(t, b, num_sms);
    return new RunnerT<P, Q, float>(t, b, num_sms);
}

}  // namespace pgc
