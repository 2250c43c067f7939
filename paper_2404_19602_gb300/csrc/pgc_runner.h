// pgc_runner.h -- host-side interface between the C ABI (pgc_api.cu) and the kernels that are
// instantiated per basis size (pgc_inst_*.cu).  Internal to the library.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace pgc {

// Every FP64 table a context needs, built on the host (pgc_tables.cpp).
struct HostTables {
    int d = 0, P = 1, Q = 1;
    bool eps_random = false, field_random = false;
    std::vector<double> z;      // [Q][d] nodes in [-1,1]^d
    std::vector<double> w;      // [Q]
    std::vector<double> psi;    // [Q][P]
    std::vector<double> wpsi;   // [Q][P]
    std::vector<double> eps0;   // [Q]
    std::vector<double> Ex;     // [Q]
    std::vector<double> dq;     // [Q] (e/hbar) E dt, nm^-1
    std::vector<double> nq;     // [Q] electron density, m^-2
    std::vector<double> dhat;   // [P]
    double eps0_max = 0.0;
    uint32_t drift_mask = 0;
    // physics in eV, fs, nm
    double hvF = 0, hbar_fs = 0, kT = 0, Cac = 0, CO = 0, CK = 0, nO = 0, nK = 0, hwO = 0, hwK = 0;
    double Cedg = 0, a_nm = 0, Lk = 0, dk = 0, vF_ms = 0;
    double mu = 0, alpha = 0, dt = 0;
    uint32_t mech = 63;
    int n_theta = 64, pauli_mode = 0, final_state = 0, max_coll = 32, Nk = 240;
};

// Device buffers of one context (all owned by the caller, carved by pgc_api.cu).
struct DevBuffers {
    void *state = nullptr;          // R [2][P][ld]
    int64_t N = 0, ld = 0;
    uint32_t *hist = nullptr;       // [3][hist_stride]
    int64_t hist_stride = 0;        // elements per buffer (>= Q*Nk*Nk, multiple of 64)
    uint32_t *queue = nullptr;      // [N]
    uint32_t *qcount = nullptr;     // [4]
    unsigned long long *counters = nullptr;  // [8]
    uint32_t *nmax = nullptr;       // [Q]
    double *part1 = nullptr;        // [kMaxGrid1][Q*3]
    double *part2 = nullptr;        // [kGrid2][Q*3]
    uint32_t *recon_hist = nullptr; // [Nk*Nk]
    uint32_t key0 = 0, key1 = 0, stream_id = 0;
};

class Runner {
public:
    virtual ~Runner() {}
    virtual int grid1() const = 0;
    virtual int grid2() const = 0;
    // sample the Fermi-Dirac initial state into the state buffer
    virtual cudaError_t init_sample(cudaStream_t s) = 0;
    // histogram of the current state into hist buffer `buf` and moment partials into part1
    virtual cudaError_t observe(int buf, cudaStream_t s) = 0;
    // histogram of the current state into `hist` ([Q][Nk*Nk], zeroed by the caller) and moment
    // partials into `part` ([grid1()][Q*3]); touches no context buffer
    virtual cudaError_t observe_into(uint32_t *hist, double *part, cudaStream_t s) = 0;
    // time step number `step` (histograms rotate over the three buffers); if ev is non-NULL,
    // ev[0..2] are recorded before phase 1, between the phases and after phase 2
    virtual cudaError_t step(int64_t step, bool out_step, cudaStream_t s, cudaEvent_t *ev = nullptr) = 0;
    // histogram at one arbitrary z (psi of length P, FP64) into out [Nk*Nk]
    virtual cudaError_t hist_at(const double *psi, uint32_t *out, cudaStream_t s) = 0;
};

// Factories, one per compiled (P, Q) shape; precision 0 = FP32, 1 = FP64.  nullptr if the
// shape is not compiled.
Runner *make_runner(int P, int Q, int precision, const HostTables &t, const DevBuffers &b, int num_sms);
Runner *make_runner_1x1(int precision, const HostTables &t, const DevBuffers &b, int num_sms);
Runner *make_runner_6x6(int precision, const HostTables &t, const DevBuffers &b, int num_sms);
Runner *make_runner_21x36(int precision, const HostTables &t, const DevBuffers &b, int num_sms);

struct BatchCase;
struct BatchScratch;
class BatchRunner;
BatchRunner *make_batch_runner(int P, int Q, int precision, const std::vector<BatchCase> &cases,
                               const BatchScratch &sc, int num_sms);
size_t case_dev_size(int P, int Q, int precision);

struct AdjBuffers;
class AdjRunner;
AdjRunner *make_adj_runner(int P, int Q, int precision, const HostTables &t, const DevBuffers &b, const AdjBuffers &ab,
                           int num_sms);

// Launch accounting (every kernel launch of the library increments it).
void count_launch(uint64_t n = 1);

}  // namespace pgc
