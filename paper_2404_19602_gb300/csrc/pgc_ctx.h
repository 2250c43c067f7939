// pgc_ctx.h -- the context behind the opaque pgc_ctx handle of include/pgc.h.  Internal.
#pragma once

#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "pgc.h"
#include "pgc_runner.h"

struct pgc_ctx {
    pgc_config cfg{};
    pgc::HostTables t;
    pgc::DevBuffers b;
    pgc::Runner *run = nullptr;
    cudaStream_t stream = nullptr;
    int64_t step = 0;
    int64_t T_out = 0;
    int rec_len = 0;
    double *series = nullptr;
    uint32_t *tmp_max = nullptr;
    double *colsum = nullptr;    // [64 * 3] column sums of k_finalize_cols
    // records of pipelined steps: reduced on a second stream (created on first use)
    cudaStream_t fin_stream = nullptr;
    cudaEvent_t fin_ready = nullptr;
    cudaEvent_t fin_done[3] = {nullptr, nullptr, nullptr};   // by partial-sum slot
    double *obs_part = nullptr;  // [kObsGrid][kObsZ][3] block partials of pgc_observe_at
    double *obs_out = nullptr;   // [kObsZ][4]
    bool failed = false;
    bool sampled = false;  // state comes from the initial Fermi-Dirac sampling (no upload since)
    std::string err;
    int pipeline = 1;  // pipelined (fused) form of multi-step pgc_step calls (pgc_set_pipeline)
    // kernel timing samples (pgc_profile): events around phase 1 / phase 2 of sampled steps
    int prof_every = 0;
    std::vector<cudaEvent_t> prof_ev;  // 4 per sample
    int prof_used = 0;
    double prof_ms[2] = {0.0, 0.0};
    int64_t prof_samples = 0;
    cudaEvent_t prof_ref = nullptr;    // recorded before the first sampled step
    bool prof_ref_set = false;
    std::vector<double> prof_tl;       // [sample][4] ms after prof_ref: phase-1 start/end, phase-2 start/end
    // pinned host staging buffer of the state transfers (allocated on first use)
    void *pinned = nullptr;
    size_t pinned_bytes = 0;
};


namespace pgc {
cudaError_t launch_finalize(const pgc_ctx *ctx, const double *part, int g1, double t_fs, double *rec,
                            cudaStream_t s);
}  // namespace pgc
