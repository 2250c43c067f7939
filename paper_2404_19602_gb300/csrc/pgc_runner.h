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
    // Strang splitting: the stored state leads the state at the step boundary by half a drift;
    // xs[q] = dq[q] / 2 is subtracted from node x values before cells and observables, and
    // dhalf[h] = dhat[h] / 2 from the x coefficients on the way out (all zero for Lie)
    bool strang = false;
    std::vector<double> xs;     // [Q]
    std::vector<double> dhalf;  // [P]
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
    uint32_t *hist = nullptr;       // [kHistBufs][hist_stride]
    int64_t hist_stride = 0;        // elements per buffer (>= Q*Nk*Nk, multiple of 64)
    uint32_t *queue = nullptr;      // [2][queue_stride] (queue_stride 0: one queue for both slots)
    int64_t queue_stride = 0;
    uint32_t *qcount = nullptr;     // [8]: collider counters n % 3 in [0, 3), phase-1 tile counters n % 3 in [4, 7),
                                    // [3] the ticket counter of k_finalize_cols
    unsigned long long *counters = nullptr;  // [8]
    uint32_t *nmax = nullptr;       // [Q]
    double *part1 = nullptr;        // [kPartSlots][kMaxGrid1][Q*3] (part1_stride 0: one slot)
    int64_t part1_stride = 0;
    double *part2 = nullptr;        // [kPartSlots][kGrid2Max][Q*3] (part2_stride 0: one slot)
    int64_t part2_stride = 0;
    double *partN = nullptr;        // [kPartSlots][kGrid2Max][Q*3] or nullptr (pipelined steps only)
    uint32_t *marks = nullptr;      // [kMarkSlots][mark_words] collider bitmaps or nullptr (pipelined steps only)
    int64_t mark_words = 0;
    void *tables = nullptr;         // device copy of the node tables (kTableBytes) or nullptr
    uint32_t *recon_hist = nullptr; // [Nk*Nk]
    uint32_t key0 = 0, key1 = 0, stream_id = 0;
};

class Runner {
public:
    virtual ~Runner() {}
    virtual int grid1() const = 0;
    virtual int grid2() const = 0;
    virtual int grid2f() const = 0;   // phase-2 blocks of the fused step kernel
    // sample the Fermi-Dirac initial state into the state buffer
    virtual cudaError_t init_sample(cudaStream_t s) = 0;
    // histogram of the current state into hist buffer `buf` and moment partials into part1
    virtual cudaError_t observe(int buf, cudaStream_t s) = 0;
    // histogram of the current state into `hist` ([Q][Nk*Nk], zeroed by the caller) and moment
    // partials into `part` ([grid1()][Q*3]); touches no context buffer
    virtual cudaError_t observe_into(uint32_t *hist, double *part, cudaStream_t s) = 0;
    // time step number `step` as two launches on one stream; if ev is non-NULL, ev[0..3] are
    // recorded before phase 1, after it, before phase 2 and after it
    virtual cudaError_t step(int64_t step, bool out_step, cudaStream_t s, cudaEvent_t *ev = nullptr) = 0;
    // the two launches of a step separately (phase 1 with a static tile assignment)
    virtual cudaError_t phase1(int64_t n, bool out_step, cudaStream_t s) = 0;
    virtual cudaError_t phase2(int64_t n, bool out_step, cudaStream_t s) = 0;
    // pipelined form: one launch doing phase 1 of step n and phase 2 of step n - 1 with the
    // continuation of its particles into step n (after phase1(n0) or a previous fused step)
    virtual cudaError_t step_fused(int64_t n, bool out_n, bool out_prev, cudaStream_t s) = 0;
    virtual bool fused() const = 0;   // step_fused is available for this shape
    // copy the node tables to DevBuffers::tables (after the scratch buffer was cleared)
    virtual cudaError_t upload_tables(cudaStream_t s) = 0;
    // histogram at one arbitrary z (psi of length P, FP64; xs: x shift of the state at z, nonzero
    // for the Strang splitting) into out [Nk*Nk]
    virtual cudaError_t hist_at(const double *psi, double xs, uint32_t *out, cudaStream_t s) = 0;
    // block partials of the observables at nzc <= 32 arbitrary points (psi [nzc][P], the band
    // minima eps0 [nzc] and the x shifts xs [nzc], FP64) into part [blocks][32][3]; *blocks
    // receives the block count
    virtual cudaError_t obs_at(const double *psi, const double *eps0, const double *xs, int nzc, double *part,
                               int *blocks, cudaStream_t s) = 0;
    // reconstruction of the streaming kernel on the tensor cores (mode 1: FP16 hi/lo, three
    // products; 2: one FP16 product); cudaErrorNotSupported where it is not compiled
    virtual cudaError_t set_tc(int mode) { (void)mode; return cudaErrorNotSupported; }
};

// Factories, one per compiled (P, Q) shape; precision 0 = FP32, 1 = FP64.  nullptr if the
// shape is not compiled.
Runner *make_runner(int P, int Q, int precision, const HostTables &t, const DevBuffers &b, int num_sms);
Runner *make_runner_1x1(int precision, const HostTables &t, const DevBuffers &b, int num_sms);
Runner *make_runner_6x6(int precision, const HostTables &t, const DevBuffers &b, int num_sms);
Runner *make_runner_21x36(int precision, const HostTables &t, const DevBuffers &b, int num_sms);
// One-dimensional shapes P = Q = M + 1 beyond the default M = 5 (degrees M = 1..30 of the
// stochastic-Galerkin error study, Test 3 of Sec. 5): time-step kernels only, no batch or
// adjoint kernels.  pgc_inst_1d.cu is compiled once per entry with -DPGC_1D_P=<P>.
#define PGC_SHAPES_1D(X) X(2) X(3) X(4) X(5) X(7) X(9) X(11) X(13) X(16) X(21) X(26) X(31)
#define PGC_DECL_RUNNER_1D(n) Runner *make_runner_1d_##n(int precision, const HostTables &t, const DevBuffers &b, int num_sms);
PGC_SHAPES_1D(PGC_DECL_RUNNER_1D)
#undef PGC_DECL_RUNNER_1D

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

// Bytes reserved for the device copy of the node tables (the largest compiled shape fits).
constexpr size_t kTableBytes = 32768;

// Launch accounting (every kernel launch of the library increments it).
void count_launch(uint64_t n = 1);

}  // namespace pgc
