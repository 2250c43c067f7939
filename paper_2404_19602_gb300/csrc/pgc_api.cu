// pgc_api.cu -- the C ABI of include/pgc.h: configuration checks, the FP64 host tables
// (physical constants of Table 1 / Appendix A, Gauss-Legendre quadrature, Legendre basis,
// densities), the device buffer carving, and the per-step launch sequence.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "pgc.h"
#include "pgc_device.cuh"
#include "pgc_kernels.cuh"
#include "pgc_runner.h"
#include "pgc_ctx.h"

namespace pgc {

static std::atomic<uint64_t> g_launches{0};
void count_launch(uint64_t n) { g_launches += n; }

Runner *make_runner(int P, int Q, int precision, const HostTables &t, const DevBuffers &b, int num_sms)
{
    if (P == 1 && Q == 1) return make_runner_1x1(precision, t, b, num_sms);
    if (P == 6 && Q == 6) return make_runner_6x6(precision, t, b, num_sms);
    if (P == 21 && Q == 36) return make_runner_21x36(precision, t, b, num_sms);
#define PGC_CASE_1D(n) if (P == n && Q == n) return make_runner_1d_##n(precision, t, b, num_sms);
    PGC_SHAPES_1D(PGC_CASE_1D)
#undef PGC_CASE_1D
    return nullptr;
}

static bool shape_compiled(int d, int P, int Q)
{
    if ((P == 1 && Q == 1) || (P == 6 && Q == 6) || (P == 21 && Q == 36)) return true;
    bool one_d = false;
#define PGC_IS_1D(n) one_d = one_d || (P == n && Q == n);
    PGC_SHAPES_1D(PGC_IS_1D)
#undef PGC_IS_1D
    return d == 1 && one_d;
}

// ------------------------------------------------------------------------------------------
// Gauss-Legendre rule for the uniform density on [-1,1] by the Golub-Welsch method: the nodes
// are the eigenvalues of the symmetric Jacobi matrix of the orthonormal Legendre recurrence,
// the weights the squared first components of its normalised eigenvectors (total mass 1).
// The eigenproblem is solved with cyclic Jacobi rotations.
// ------------------------------------------------------------------------------------------
static void golub_welsch(int n, std::vector<double> &x, std::vector<double> &w)
{
    std::vector<double> A(n * n, 0.0), V(n * n, 0.0);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int k = 1; k < n; ++k) {
        const double b = k / std::sqrt(4.0 * k * k - 1.0);
        A[(k - 1) * n + k] = A[k * n + k - 1] = b;
    }
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
        if (off < 1e-34) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // A <- A J  (columns p, q)
                    const double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // A <- J^T A  (rows p, q)
                    const double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {  // V <- V J
                    const double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return A[a * n + a] < A[b * n + b]; });
    x.resize(n);
    w.resize(n);
    for (int j = 0; j < n; ++j) {
        const int e = idx[j];
        x[j] = A[e * n + e];
        w[j] = V[0 * n + e] * V[0 * n + e];
    }
    // symmetric rule: enforce exact symmetry of nodes and weights
    for (int j = 0; j < n / 2; ++j) {
        const double xm = 0.5 * (x[n - 1 - j] - x[j]), wm = 0.5 * (w[j] + w[n - 1 - j]);
        x[j] = -xm; x[n - 1 - j] = xm;
        w[j] = wm; w[n - 1 - j] = wm;
    }
    if (n % 2) x[n / 2] = 0.0;
}

// orthonormal Legendre values psi_0..psi_M at z from the orthonormal three-term recurrence
// z psi_n = b_{n+1} psi_{n+1} + b_n psi_{n-1},  b_n = n / sqrt(4 n^2 - 1)
static void onb_legendre(int M, double z, double *out)
{
    out[0] = 1.0;
    if (M == 0) return;
    out[1] = z / (1.0 / std::sqrt(3.0));
    for (int n = 1; n < M; ++n) {
        const double bn = n / std::sqrt(4.0 * n * n - 1.0);
        const double bn1 = (n + 1) / std::sqrt(4.0 * (n + 1) * (n + 1) - 1.0);
        out[n + 1] = (z * out[n] - bn * out[n - 1]) / bn1;
    }
}

// basis at a point z (d components), 2-D total degree in graded order (t - j, j)
static void basis_at(int d, int M, const double *z, double *psi)
{
    if (d == 0) { psi[0] = 1.0; return; }
    if (d == 1) { onb_legendre(M, z[0], psi); return; }
    std::vector<double> a(M + 1), b(M + 1);
    onb_legendre(M, z[0], a.data());
    onb_legendre(M, z[1], b.data());
    int h = 0;
    for (int t = 0; t <= M; ++t)
        for (int j = 0; j <= t; ++j) psi[h++] = a[t - j] * b[j];
}

// Is the band minimum a random input (per its law)?
static bool eps_random_of(const pgc_config &c)
{
    return c.eps0_law == PGC_EPS0_WIDTH ? c.width_nm.lo != c.width_nm.hi : c.eps0_eV.lo != c.eps0_eV.hi;
}

// Band minimum at the band-minimum variable z in [-1,1] (eps0 = hbar vF pi / W, Sec. 2).
static double eps0_at(const pgc_config &c, double hvF, double z)
{
    const bool er = eps_random_of(c);
    if (c.eps0_law == PGC_EPS0_WIDTH) {
        const double W = er ? c.width_nm.lo + 0.5 * (c.width_nm.hi - c.width_nm.lo) * (z + 1.0) : c.width_nm.lo;
        return kPi * hvF / W;
    }
    return er ? c.eps0_eV.lo + 0.5 * (c.eps0_eV.hi - c.eps0_eV.lo) * (z + 1.0) : c.eps0_eV.lo;
}

static int dims_of(const pgc_config &c, int *P, int *Q)
{
    const bool er = eps_random_of(c), fr = c.Ex_Vcm.lo != c.Ex_Vcm.hi;
    const int d = (int)er + (int)fr;
    if (d == 0) { *P = 1; *Q = 1; }
    else if (d == 1) { *P = c.degree_M + 1; *Q = c.quad_per_dim; }
    else { *P = (c.degree_M + 1) * (c.degree_M + 2) / 2; *Q = c.quad_per_dim * c.quad_per_dim; }
    return d;
}

// Physical constants of Table 1 (Sec. 5) and the closed-form rate prefactors of Appendix A.
static void build_tables(const pgc_config &c, HostTables &t)
{
    const double e = 1.602176634e-19, hbar_eVs = 6.582119569e-16, kB = 8.617333262e-5;
    const double hbar = hbar_eVs * e;            // J s
    const double vF = 1.0e6;                     // 1e8 cm/s
    const double sigma = 7.6e-8 * 10.0;          // 7.6e-8 g/cm^2 -> kg/m^2
    const double vp = 2.0e4;                     // 2e6 cm/s
    const double Dac = 6.8 * e;                  // J
    const double DO = 1.0e9 * e * 100.0;         // eV/cm -> J/m
    const double DK = 3.5e8 * e * 100.0;
    const double hwO = 0.1646, hwK = 0.124;      // eV
    const double Ni = 1.0e4 * 100.0;             // 1/m
    const double V0 = 4.56e-14 * e * 1.0e-4;     // J m^2
    const double a = 1.0e-8 * 1.0e-2;            // m
    const double kT = kB * c.T_K;                // eV
    const double kTJ = kT * e;
    t.hbar_fs = hbar_eVs * 1.0e15;
    t.hvF = hbar_eVs * vF * 1.0e9;               // eV nm
    t.kT = kT;
    t.hwO = hwO;
    t.hwK = hwK;
    t.nO = 1.0 / std::expm1(hwO / kT);
    t.nK = 1.0 / std::expm1(hwK / kT);
    const double hvFJ = hbar * vF;
    // Gamma_ac / eps  [1/s per J] -> [1/fs per eV]
    t.Cac = Dac * Dac * kTJ / (4.0 * hbar * hbar * hbar * vF * vF * sigma * vp * vp) * e * 1e-15;
    t.CO = DO * DO / (hbar * hbar * vF * vF * sigma * (hwO / hbar_eVs)) * e * 1e-15;
    t.CK = DK * DK / (hbar * hbar * vF * vF * sigma * (hwK / hbar_eVs)) * e * 1e-15;
    // Gamma_edg = Ni V0^2 /(2 pi hbar W (hbar vF)^2) eps T, 1/W = eps0/(pi hbar vF)
    t.Cedg = Ni * V0 * V0 / (2.0 * kPi * kPi * hbar * hvFJ * hvFJ * hvFJ) * e * e * 1e-15;
    t.a_nm = a * 1e9;
    t.Lk = c.Lk_hvF_eV / t.hvF;
    t.dk = 2.0 * t.Lk / c.Nk;
    t.vF_ms = vF;
    t.mu = c.eps_F_eV;
    t.alpha = c.alpha;
    t.dt = c.dt_fs;
    t.mech = c.mech_mask;
    t.n_theta = c.n_theta_edge;
    t.pauli_mode = c.pauli_norm;
    t.final_state = c.final_state;
    t.max_coll = c.max_collisions;
    t.Nk = c.Nk;

    int P, Q;
    const int d = dims_of(c, &P, &Q);
    t.d = d; t.P = P; t.Q = Q;
    std::vector<double> x1, w1;
    t.z.assign((size_t)Q * std::max(d, 1), 0.0);
    t.w.assign(Q, 0.0);
    if (d == 0) t.w[0] = 1.0;
    else {
        golub_welsch(c.quad_per_dim, x1, w1);
        if (d == 1) for (int q = 0; q < Q; ++q) { t.z[q] = x1[q]; t.w[q] = w1[q]; }
        else
            for (int q1 = 0; q1 < c.quad_per_dim; ++q1)
                for (int q2 = 0; q2 < c.quad_per_dim; ++q2) {
                    const int q = q1 * c.quad_per_dim + q2;
                    t.z[2 * q] = x1[q1]; t.z[2 * q + 1] = x1[q2];
                    t.w[q] = w1[q1] * w1[q2];
                }
    }
    const bool er = eps_random_of(c), fr = c.Ex_Vcm.lo != c.Ex_Vcm.hi;
    t.eps_random = er;
    t.field_random = fr;
    t.psi.assign((size_t)Q * P, 0.0);
    t.wpsi.assign((size_t)Q * P, 0.0);
    t.eps0.assign(Q, 0.0); t.Ex.assign(Q, 0.0); t.dq.assign(Q, 0.0); t.nq.assign(Q, 0.0);
    t.eps0_max = 0.0;
    for (int q = 0; q < Q; ++q) {
        double ze = 0.0, zf = 0.0;
        if (d == 1) { if (er) ze = t.z[q]; else zf = t.z[q]; }
        if (d == 2) { ze = t.z[2 * q]; zf = t.z[2 * q + 1]; }
        t.eps0[q] = eps0_at(c, t.hvF, ze);
        t.Ex[q] = fr ? c.Ex_Vcm.lo + 0.5 * (c.Ex_Vcm.hi - c.Ex_Vcm.lo) * (zf + 1.0) : c.Ex_Vcm.lo;
        t.dq[q] = t.Ex[q] * 1.0e-7 * c.dt_fs / t.hbar_fs;
        t.nq[q] = 2.0 / (kPi * t.hvF * t.hvF) * fd_upper<double>(t.eps0[q], c.eps_F_eV, kT) * 1.0e18;
        t.eps0_max = std::max(t.eps0_max, t.eps0[q]);
        basis_at(d, c.degree_M, d ? &t.z[(size_t)q * d] : nullptr, &t.psi[(size_t)q * P]);
        for (int h = 0; h < P; ++h) t.wpsi[(size_t)q * P + h] = t.w[q] * t.psi[(size_t)q * P + h];
    }
    t.dhat.assign(P, 0.0);
    t.drift_mask = 0;
    double dmax = 0.0;
    for (int h = 0; h < P; ++h) {
        double s = 0.0;
        for (int q = 0; q < Q; ++q) s += t.wpsi[(size_t)q * P + h] * t.dq[q];
        t.dhat[h] = s;
        dmax = std::max(dmax, std::fabs(s));
    }
    // the field is affine in z: only the constant and the linear field mode are non-zero;
    // quadrature round-off in the other entries is dropped
    for (int h = 0; h < P; ++h) {
        if (std::fabs(t.dhat[h]) <= 1e-13 * dmax) t.dhat[h] = 0.0;
        if (t.dhat[h] != 0.0) t.drift_mask |= (1u << h);
    }
    t.strang = c.splitting == PGC_SPLIT_STRANG;
    t.xs.assign(Q, 0.0);
    t.dhalf.assign(P, 0.0);
    if (t.strang) {
        for (int q = 0; q < Q; ++q) t.xs[q] = 0.5 * t.dq[q];
        for (int h = 0; h < P; ++h) t.dhalf[h] = 0.5 * t.dhat[h];
    }
}

// ------------------------------------------------------------------------------------------
// small kernels shared by all shapes
// ------------------------------------------------------------------------------------------
struct FinArgs {
    double nq[64], w[64];
    double N, vF_ms, t_fs;
    int Q, g1, g2, g3;
};

// fixed-order reduction of the block partials, node values, mean and variance (Sec. 4.2);
// record = [t, nodes[Q][4] (Vx, Vy, E, Jx), mean[4], var[4]].  Thread t sums column t % n3 over
// the blocks congruent to t / n3 (coalesced reads), then one thread per column adds the slots.
constexpr int kFinThreads = 1024;
__global__ void __launch_bounds__(kFinThreads)
k_finalize(const double *part1, const double *part2, const double *part3, const __grid_constant__ FinArgs f, double *rec)
{
    __shared__ double red[kFinThreads];
    __shared__ double S[64 * 3];
    const int n3 = f.Q * 3;
    const int nslot = kFinThreads / n3;
    const int t = threadIdx.x, col = t % n3, slot = t / n3;
    double s = 0.0;
    if (slot < nslot) {
        s = strided_sum(part1, slot, f.g1, nslot, n3, col, s);
        s = strided_sum(part2, slot, f.g2, nslot, n3, col, s);
        s = strided_sum(part3, slot, f.g3, nslot, n3, col, s);
    }
    red[t] = s;
    __syncthreads();
    if (t < n3) {
        double acc = 0.0;
        for (int k = 0; k < nslot; ++k) acc += red[k * n3 + t];
        S[t] = acc;
    }
    __syncthreads();
    // node values, one thread per node (FP64 divisions are slow on this part: in parallel), then
    // the mean and variance over the nodes by one thread in node order
    __shared__ double V[64 * 4];
    if (t < f.Q) {
        const double qe = 1.602176634e-19;
        const int q = t;
        const double vx = S[q * 3 + 0] / f.N * f.vF_ms, vy = S[q * 3 + 1] / f.N * f.vF_ms;
        const double en = S[q * 3 + 2] / f.N, jx = -qe * f.nq[q] * vx;
        const double v[4] = {vx, vy, en, jx};
        for (int o = 0; o < 4; ++o) {
            V[q * 4 + o] = v[o];
            rec[1 + q * 4 + o] = v[o];
        }
    }
    __syncthreads();
    if (t == 0) {
        rec[0] = f.t_fs;
        double m[4] = {0, 0, 0, 0}, m2[4] = {0, 0, 0, 0};
        for (int q = 0; q < f.Q; ++q)
            for (int o = 0; o < 4; ++o) {
                const double v = V[q * 4 + o];
                m[o] += f.w[q] * v;
                m2[o] += f.w[q] * v * v;
            }
        for (int o = 0; o < 4; ++o) {
            rec[1 + f.Q * 4 + o] = m[o];
            rec[1 + f.Q * 4 + 4 + o] = m2[o] - m[o] * m[o];
        }
    }
}

// The record of a moment step over several SMs (the reduction is FP64, which this part issues at a
// small fraction of its FP32 rate: one block would spend most of a step on it).  Block c sums
// column c of the block partials (part1: g1 rows, part2: g2 rows, part3: g3 rows) with a
// fixed-order tree and stores it in colsum[c]; the block that finishes last (its ticket from an
// atomic counter is the last one; nothing waits) forms the record from the column sums as
// k_finalize does and re-arms the counter.
constexpr int kFinColThreads = 256;
__global__ void __launch_bounds__(kFinColThreads)
k_finalize_cols(const double *part1, const double *part2, const double *part3, const __grid_constant__ FinArgs f,
                double *colsum, unsigned int *ticket, double *rec)
{
    __shared__ double red[kFinColThreads];
    __shared__ double S[64 * 3];
    __shared__ double V[64 * 4];
    __shared__ bool last;
    const int n3 = f.Q * 3, c = blockIdx.x, t = threadIdx.x;
    double s = 0.0;
    s = strided_sum(part1, t, f.g1, kFinColThreads, n3, c, s);
    s = strided_sum(part2, t, f.g2, kFinColThreads, n3, c, s);
    s = strided_sum(part3, t, f.g3, kFinColThreads, n3, c, s);
    red[t] = s;
    __syncthreads();
    for (int w = kFinColThreads / 2; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    if (t == 0) {
        colsum[c] = red[0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == (unsigned int)(n3 - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int j = t; j < n3; j += kFinColThreads) S[j] = __ldcg(colsum + j);
    __syncthreads();
    if (t < f.Q) {
        const double qe = 1.602176634e-19;
        const int q = t;
        const double vx = S[q * 3 + 0] / f.N * f.vF_ms, vy = S[q * 3 + 1] / f.N * f.vF_ms;
        const double en = S[q * 3 + 2] / f.N, jx = -qe * f.nq[q] * vx;
        const double v[4] = {vx, vy, en, jx};
        for (int o = 0; o < 4; ++o) {
            V[q * 4 + o] = v[o];
            rec[1 + q * 4 + o] = v[o];
        }
    }
    __syncthreads();
    if (t == 0) {
        rec[0] = f.t_fs;
        double m[4] = {0, 0, 0, 0}, m2[4] = {0, 0, 0, 0};
        for (int q = 0; q < f.Q; ++q)
            for (int o = 0; o < 4; ++o) {
                const double v = V[q * 4 + o];
                m[o] += f.w[q] * v;
                m2[o] += f.w[q] * v * v;
            }
        for (int o = 0; o < 4; ++o) {
            rec[1 + f.Q * 4 + o] = m[o];
            rec[1 + f.Q * 4 + 4 + o] = m2[o] - m[o] * m[o];
        }
        *ticket = 0u;
    }
}

// Observables at arbitrary points from the block partials of k_obs_at (fixed order over the
// blocks): out[z] = (V_x, V_y, energy, J_x) as in the records of k_finalize.
struct ObsFin {
    double n[kObsZ];   // density n(eps0(z)) (m^-2)
    double scale_v;    // hbar vF * vF / N: sum of kx/eps -> V_x in m/s
    double inv_N;
    int nz, g;
};

__global__ void __launch_bounds__(128)
k_obs_fin(const double *part, const __grid_constant__ ObsFin f, double *out)
{
    __shared__ double S[kObsZ * 3];
    const int t = threadIdx.x;
    if (t < kObsZ * 3) {
        double s = 0.0;
        s = strided_sum(part, 0, f.g, 1, kObsZ * 3, t, s);
        S[t] = s;
    }
    __syncthreads();
    if (t < f.nz) {
        const double qe = 1.602176634e-19;
        const double vx = S[t * 3 + 0] * f.scale_v, vy = S[t * 3 + 1] * f.scale_v;
        out[t * 4 + 0] = vx;
        out[t * 4 + 1] = vy;
        out[t * 4 + 2] = S[t * 3 + 2] * f.inv_N;
        out[t * 4 + 3] = -qe * f.n[t] * vx;
    }
}

// maximum over the cells of each node's histogram
__global__ void k_hist_max(const uint32_t *H, int64_t cells, uint32_t *out)
{
    __shared__ uint32_t sm[32];
    const uint32_t *h = H + (int64_t)blockIdx.x * cells;
    uint32_t m = 0;
    for (int64_t j = threadIdx.x; j < cells; j += blockDim.x) m = max(m, h[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = (threadIdx.x < (blockDim.x >> 5)) ? sm[threadIdx.x] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) out[blockIdx.x] = m;
    }
}

// Fixed-order reduction of g1 block partials (no second set) into one moment record of ctx's
// layout; used by entry points that keep their partial sums outside the context scratch.
cudaError_t launch_finalize(const pgc_ctx *ctx, const double *part, int g1, double t_fs, double *rec,
                            cudaStream_t s)
{
    FinArgs f{};
    for (int q = 0; q < ctx->t.Q; ++q) { f.nq[q] = ctx->t.nq[q]; f.w[q] = ctx->t.w[q]; }
    f.N = (double)ctx->b.N;
    f.vF_ms = ctx->t.vF_ms;
    f.t_fs = t_fs;
    f.Q = ctx->t.Q;
    f.g1 = g1;
    f.g2 = 0;
    f.g3 = 0;
    k_finalize<<<1, kFinThreads, 0, s>>>(part, nullptr, nullptr, f, rec);
    count_launch();
    return cudaGetLastError();
}

}  // namespace pgc

using namespace pgc;

// Runs fn(lo, hi) over [0, n) on up to 16 host threads (one for small n): the layout conversions
// of the state transfers touch every coefficient of the ensemble.
template <typename F>
static void host_parallel(int64_t n, F &&fn)
{
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int64_t nt = std::min<int64_t>({(int64_t)std::min(hw, 16u), std::max<int64_t>(1, n / (1 << 18)), n});
    if (nt <= 1) { fn((int64_t)0, n); return; }
    std::vector<std::thread> th;
    const int64_t chunk = (n + nt - 1) / nt;
    for (int64_t t = 1; t < nt; ++t) {
        const int64_t lo = t * chunk, hi = std::min(n, lo + chunk);
        if (lo < hi) th.emplace_back([&fn, lo, hi] { fn(lo, hi); });
    }
    fn((int64_t)0, std::min(n, chunk));
    for (auto &x : th) x.join();
}

static void *staging(pgc_ctx *ctx, size_t bytes)
{
    if (ctx->pinned_bytes >= bytes) return ctx->pinned;
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    ctx->pinned_bytes = 0;
    if (cudaMallocHost(&ctx->pinned, bytes) != cudaSuccess) { ctx->pinned = nullptr; return nullptr; }
    ctx->pinned_bytes = bytes;
    return ctx->pinned;
}

static constexpr size_t kMaxTimeline = 4096;  // samples kept for pgc_profile_timeline

static void prof_collect(pgc_ctx *ctx)
{
    for (int k = 0; k < ctx->prof_used; ++k) {
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, ctx->prof_ev[4 * k], ctx->prof_ev[4 * k + 1]) == cudaSuccess &&
            cudaEventElapsedTime(&b, ctx->prof_ev[4 * k + 2], ctx->prof_ev[4 * k + 3]) == cudaSuccess) {
            ctx->prof_ms[0] += a;
            ctx->prof_ms[1] += b;
            ctx->prof_samples++;
            if (ctx->prof_ref_set && ctx->prof_tl.size() < 4 * kMaxTimeline) {
                float t[4];
                bool ok = true;
                for (int j = 0; j < 4 && ok; ++j) ok = cudaEventElapsedTime(&t[j], ctx->prof_ref, ctx->prof_ev[4 * k + j]) == cudaSuccess;
                if (ok)
                    for (int j = 0; j < 4; ++j) ctx->prof_tl.push_back(t[j]);
            }
        }
    }
    ctx->prof_used = 0;
}

static std::mutex g_err_mu;
static std::string g_err;

static pgc_status fail(pgc_ctx *ctx, pgc_status s, const std::string &msg)
{
    if (ctx) {
        ctx->err = msg;
        if (s == PGC_ECUDA) ctx->failed = true;
    } else {
        std::lock_guard<std::mutex> lk(g_err_mu);
        g_err = msg;
    }
    return s;
}

static pgc_status cuda_fail(pgc_ctx *ctx, cudaError_t e, const char *where)
{
    return fail(ctx, PGC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

namespace {
struct Layout {
    int P = 1, Q = 1, d = 0;
    int64_t ld = 0, hist_stride = 0, queue_stride = 0, mark_words = 0;
    size_t state = 0, hist = 0, scratch = 0;
    size_t off_queue = 0, off_qcount = 0, off_counters = 0, off_nmax = 0, off_part1 = 0, off_part2 = 0,
           off_partN = 0, off_marks = 0, off_tables = 0, off_series = 0, off_recon = 0, off_tmpmax = 0,
           off_obs = 0, off_colsum = 0;
    int rec_len = 0;
};
}  // namespace

static pgc_status check_config(const pgc_config *c, Layout *L, std::string *msg)
{
    if (!c) { *msg = "cfg is NULL"; return PGC_EINVAL; }
    auto bad = [&](const char *m) { *msg = m; return PGC_EINVAL; };
    if (!(c->T_K > 0.0)) return bad("T_K must be > 0");
    if (c->eps0_law != PGC_EPS0_AFFINE && c->eps0_law != PGC_EPS0_WIDTH) return bad("eps0_law must be PGC_EPS0_AFFINE or PGC_EPS0_WIDTH");
    if (c->splitting != PGC_SPLIT_LIE && c->splitting != PGC_SPLIT_STRANG) return bad("splitting must be PGC_SPLIT_LIE or PGC_SPLIT_STRANG");
    if (c->eps0_law == PGC_EPS0_AFFINE && (!(c->eps0_eV.lo > 0.0) || !(c->eps0_eV.hi >= c->eps0_eV.lo)))
        return bad("eps0 interval must satisfy 0 < lo <= hi");
    if (c->eps0_law == PGC_EPS0_WIDTH && (!(c->width_nm.lo > 0.0) || !(c->width_nm.hi >= c->width_nm.lo) || !std::isfinite(c->width_nm.hi)))
        return bad("width interval must satisfy 0 < lo <= hi (finite)");
    if (!(c->Ex_Vcm.hi >= c->Ex_Vcm.lo) || !std::isfinite(c->Ex_Vcm.lo) || !std::isfinite(c->Ex_Vcm.hi))
        return bad("Ex interval must satisfy lo <= hi (finite)");
    if (c->mech_mask > 63u) return bad("mech_mask has unknown bits");
    if (!(c->alpha >= 0.0) || !(c->alpha < 10.0)) return bad("alpha must be in [0, 10)");
    if (c->Nk < 2 || c->Nk > 4096) return bad("Nk must be in [2, 4096]");
    if (!(c->Lk_hvF_eV > 0.0)) return bad("Lk_hvF_eV must be > 0");
    if (c->degree_M < 0 || c->degree_M > 30) return bad("degree_M must be in [0, 30]");
    if (c->quad_per_dim < 1 || c->quad_per_dim > 32) return bad("quad_per_dim must be in [1, 32]");
    if (c->n_particles < 1 || c->n_particles > 2000000000LL) return bad("n_particles must be in [1, 2e9]");
    if (!(c->dt_fs > 0.0)) return bad("dt_fs must be > 0");
    if (c->precision != PGC_FP32 && c->precision != PGC_FP64) return bad("precision must be PGC_FP32 or PGC_FP64");
    if (c->pauli_norm < 0 || c->pauli_norm > 2) return bad("pauli_norm must be 0, 1 or 2");
    if (c->final_state < 0 || c->final_state > 1) return bad("final_state must be 0 or 1");
    if (c->n_theta_edge < 4 || c->n_theta_edge > kMaxTheta || (c->n_theta_edge & 1)) return bad("n_theta_edge must be even in [4, 256]");
    if (c->max_collisions < 1 || c->max_collisions > 65535) return bad("max_collisions must be in [1, 65535]");
    if (c->max_outputs < 1) return bad("max_outputs must be >= 1");
    if (c->tc_proj != PGC_TC_OFF && c->tc_proj != PGC_TC_F16X3 && c->tc_proj != PGC_TC_F16)
        return bad("tc_proj must be PGC_TC_OFF, PGC_TC_F16X3 or PGC_TC_F16");
    L->d = dims_of(*c, &L->P, &L->Q);
    if (L->d > 0 && c->quad_per_dim < c->degree_M + 1) return bad("quad_per_dim must be >= degree_M + 1 (exact projection)");
    if (!shape_compiled(L->d, L->P, L->Q)) {
        *msg = "compiled (P,Q) shapes are (1,1), (6,6), (21,36) and, with one random input, (M+1,M+1) for "
               "M = 1, 2, 3, 4, 6, 8, 10, 12, 15, 20, 25, 30; got (" + std::to_string(L->P) + "," + std::to_string(L->Q) + ")";
        return PGC_EUNSUPPORTED;
    }
    if (c->tc_proj != PGC_TC_OFF && !(L->P == 21 && L->Q == 36 && c->precision == PGC_FP32)) {
        *msg = "tc_proj (the tensor-core reconstruction) is compiled for the FP32 21 x 36 shape only";
        return PGC_EUNSUPPORTED;
    }
    const int64_t N = c->n_particles;
    const size_t R = (c->precision == PGC_FP64) ? 8 : 4;
    L->ld = round_up(N, 64);
    L->state = (size_t)2 * L->P * L->ld * R;
    L->hist_stride = round_up((int64_t)L->Q * c->Nk * c->Nk, 64);
    L->hist = (size_t)kHistBufs * L->hist_stride * 4;
    L->rec_len = 1 + 4 * L->Q + 8;
    L->queue_stride = round_up(N, 64);
    L->mark_words = round_up((N + 31) / 32, 64);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = (size_t)round_up((int64_t)(off + bytes), 256); return o; };
    L->off_queue = take((size_t)2 * L->queue_stride * 4);
    L->off_qcount = take(8 * 4);
    L->off_counters = take(8 * 8);
    L->off_nmax = take((size_t)L->Q * 4);
    L->off_part1 = take((size_t)kPartSlots * kMaxGrid1 * L->Q * 3 * 8);
    L->off_part2 = take((size_t)kPartSlots * kGrid2Max * L->Q * 3 * 8);
    L->off_partN = take((size_t)kPartSlots * kGrid2Max * L->Q * 3 * 8);
    L->off_marks = take((size_t)kMarkSlots * L->mark_words * 4);
    L->off_tables = take(kTableBytes);
    L->off_series = take((size_t)c->max_outputs * L->rec_len * 8);
    L->off_recon = take((size_t)c->Nk * c->Nk * 4);
    L->off_tmpmax = take(4);
    L->off_obs = take((size_t)(kObsGrid * kObsZ * 3 + kObsZ * 4) * 8);
    L->off_colsum = take((size_t)64 * 3 * 8);
    L->scratch = off;
    return PGC_OK;
}

extern "C" {

void pgc_config_default(pgc_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->T_K = 300.0;
    c->eps_F_eV = 0.4;
    c->eps0_eV.lo = c->eps0_eV.hi = 0.1;
    c->Ex_Vcm.lo = c->Ex_Vcm.hi = 5000.0;
    c->mech_mask = PGC_MECH_ALL;
    c->alpha = 0.1;
    c->Nk = 240;
    c->Lk_hvF_eV = 5.0;
    c->degree_M = 5;
    c->quad_per_dim = 6;
    c->n_particles = 10000;
    c->dt_fs = 1.0;
    c->seed = 1;
    c->stream_id = 0;
    c->precision = PGC_FP32;
    c->pauli_norm = PGC_PAULI_INITIAL_MAX;
    c->final_state = PGC_FS_PAPER;
    c->n_theta_edge = 64;
    c->max_collisions = 32;
    c->max_outputs = 1024;
    c->eps0_law = PGC_EPS0_AFFINE;
    c->width_nm.lo = c->width_nm.hi = 0.0;
    c->splitting = PGC_SPLIT_LIE;
}

pgc_status pgc_query_sizes(const pgc_config *cfg, size_t *state_bytes, size_t *hist_bytes,
                           size_t *scratch_bytes, int32_t *P, int32_t *Q)
{
    Layout L;
    std::string msg;
    pgc_status s = check_config(cfg, &L, &msg);
    if (s != PGC_OK) return fail(nullptr, s, msg);
    if (state_bytes) *state_bytes = L.state;
    if (hist_bytes) *hist_bytes = L.hist;
    if (scratch_bytes) *scratch_bytes = L.scratch;
    if (P) *P = L.P;
    if (Q) *Q = L.Q;
    return PGC_OK;
}

static pgc_status observe_current(pgc_ctx *ctx, bool record, bool set_nmax)
{
    cudaStream_t s = ctx->stream;
    cudaError_t e;
    const int cur = (int)(ctx->step % kHistBufs);
    if ((e = cudaMemsetAsync(ctx->b.hist, 0, (size_t)kHistBufs * ctx->b.hist_stride * 4, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "memset hist");
    if ((e = ctx->run->observe(cur, s)) != cudaSuccess) return cuda_fail(ctx, e, "observe");
    const int64_t cells = (int64_t)ctx->t.Nk * ctx->t.Nk;
    if (set_nmax) {
        k_hist_max<<<ctx->t.Q, 256, 0, s>>>(ctx->b.hist + (int64_t)cur * ctx->b.hist_stride, cells, ctx->b.nmax);
        count_launch();
    }
    if (record) {
        if (ctx->T_out >= ctx->cfg.max_outputs) return fail(ctx, PGC_ENOMEM, "moment series full (max_outputs)");
        FinArgs f{};
        for (int q = 0; q < ctx->t.Q; ++q) { f.nq[q] = ctx->t.nq[q]; f.w[q] = ctx->t.w[q]; }
        f.N = (double)ctx->b.N;
        f.vF_ms = ctx->t.vF_ms;
        f.t_fs = ctx->step * ctx->t.dt;
        f.Q = ctx->t.Q;
        f.g1 = ctx->run->grid1();
        f.g2 = 0;
        f.g3 = 0;
        k_finalize<<<1, kFinThreads, 0, s>>>(ctx->b.part1, nullptr, nullptr, f, ctx->series + ctx->T_out * ctx->rec_len);
        count_launch();
        ctx->T_out++;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "observe launch");
    return PGC_OK;
}

pgc_status pgc_init(const pgc_config *cfg, void *d_state, void *d_hist, void *d_scratch,
                    const double *h_init_khat, void *stream, pgc_ctx **out)
{
    if (!out) return fail(nullptr, PGC_EINVAL, "out is NULL");
    *out = nullptr;
    Layout L;
    std::string msg;
    pgc_status st = check_config(cfg, &L, &msg);
    if (st != PGC_OK) return fail(nullptr, st, msg);
    if (!d_state || !d_hist || !d_scratch) return fail(nullptr, PGC_EINVAL, "device buffers must be non-NULL");
    if (((uintptr_t)d_state & 255) || ((uintptr_t)d_hist & 255) || ((uintptr_t)d_scratch & 255))
        return fail(nullptr, PGC_EINVAL, "device buffers must be 256-byte aligned");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, PGC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(nullptr, PGC_ECUDA, std::string("attribute: ") + cudaGetErrorString(e));

    pgc_ctx *ctx = new (std::nothrow) pgc_ctx();
    if (!ctx) return fail(nullptr, PGC_ENOMEM, "context allocation");
    ctx->cfg = *cfg;
    ctx->stream = (cudaStream_t)stream;
    build_tables(*cfg, ctx->t);
    char *scr = (char *)d_scratch;
    DevBuffers &b = ctx->b;
    b.state = d_state;
    b.N = cfg->n_particles;
    b.ld = L.ld;
    b.hist = (uint32_t *)d_hist;
    b.hist_stride = L.hist_stride;
    b.queue = (uint32_t *)(scr + L.off_queue);
    b.queue_stride = L.queue_stride;
    b.qcount = (uint32_t *)(scr + L.off_qcount);
    b.counters = (unsigned long long *)(scr + L.off_counters);
    b.nmax = (uint32_t *)(scr + L.off_nmax);
    b.part1 = (double *)(scr + L.off_part1);
    b.part1_stride = (int64_t)kMaxGrid1 * L.Q * 3;
    b.part2 = (double *)(scr + L.off_part2);
    b.part2_stride = (int64_t)kGrid2Max * L.Q * 3;
    b.partN = (double *)(scr + L.off_partN);
    b.marks = (uint32_t *)(scr + L.off_marks);
    b.mark_words = L.mark_words;
    b.tables = scr + L.off_tables;
    b.recon_hist = (uint32_t *)(scr + L.off_recon);
    b.key0 = (uint32_t)cfg->seed;
    b.key1 = (uint32_t)(cfg->seed >> 32);
    b.stream_id = cfg->stream_id;
    ctx->series = (double *)(scr + L.off_series);
    ctx->tmp_max = (uint32_t *)(scr + L.off_tmpmax);
    ctx->obs_part = (double *)(scr + L.off_obs);
    ctx->obs_out = ctx->obs_part + (size_t)kObsGrid * kObsZ * 3;
    ctx->colsum = (double *)(scr + L.off_colsum);
    ctx->rec_len = L.rec_len;
    ctx->run = make_runner(L.P, L.Q, cfg->precision, ctx->t, b, sms);
    if (!ctx->run) { delete ctx; return fail(nullptr, PGC_EUNSUPPORTED, "no kernel for this shape"); }
    // the fused step overlaps the collider work with the streaming work.  For 36 nodes the
    // collider work is itself throughput-bound (many chains per lane group) and, fused, holds
    // most resident blocks for the whole launch: measured slower, so off by default there
    ctx->pipeline = (ctx->run->fused() && L.P * L.Q <= 64) ? 1 : 0;
    if (cfg->tc_proj != PGC_TC_OFF) {
        if ((e = ctx->run->set_tc(cfg->tc_proj)) != cudaSuccess) {
            delete ctx->run; delete ctx;
            return fail(nullptr, PGC_EUNSUPPORTED, std::string("tensor-core streaming kernel unavailable: ") + cudaGetErrorString(e));
        }
        ctx->pipeline = 0;
    }

    cudaStream_t s = ctx->stream;
    if ((e = cudaMemsetAsync(d_scratch, 0, L.scratch, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(d_state, 0, L.state, s)) != cudaSuccess ||
        (e = ctx->run->upload_tables(s)) != cudaSuccess) {
        delete ctx->run; delete ctx;
        return fail(nullptr, PGC_ECUDA, std::string("memset: ") + cudaGetErrorString(e));
    }
    if (h_init_khat) {
        st = pgc_set_state(ctx, h_init_khat);
        if (st == PGC_OK) st = observe_current(ctx, true, true);
    } else {
        if ((e = ctx->run->init_sample(s)) != cudaSuccess) st = cuda_fail(ctx, e, "init kernel");
        else st = observe_current(ctx, true, true);
        ctx->sampled = true;
    }
    if (st != PGC_OK) {
        std::string m = ctx->err;
        delete ctx->run; delete ctx;
        return fail(nullptr, st, m);
    }
    *out = ctx;
    return PGC_OK;
}

static_assert(sizeof(pgc_ctx::fin_done) / sizeof(cudaEvent_t) == pgc::kPartSlots, "one event per partial-sum slot");

// The second stream (highest priority) and events of the pipelined records, created on first use.
static cudaError_t fin_stream_of(pgc_ctx *ctx)
{
    if (ctx->fin_stream) return cudaSuccess;
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->fin_ready, cudaEventDisableTiming);
    for (int k = 0; k < pgc::kPartSlots && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&ctx->fin_done[k], cudaEventDisableTiming);
    cudaStream_t fs = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&fs, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) ctx->fin_stream = fs;
    return e;
}

pgc_status pgc_step(pgc_ctx *ctx, int64_t n_steps, int32_t moments_every)
{
    if (!ctx) return fail(nullptr, PGC_EINVAL, "ctx is NULL");
    if (ctx->failed) return fail(ctx, PGC_ESTATE, "context failed earlier: " + ctx->err);
    if (n_steps < 0) return fail(ctx, PGC_EINVAL, "n_steps < 0");
    int64_t outs = 0;
    if (moments_every > 0) outs = (ctx->step + n_steps) / moments_every - ctx->step / moments_every;
    if (ctx->T_out + outs > ctx->cfg.max_outputs) return fail(ctx, PGC_ENOMEM, "moment series would exceed max_outputs");
    cudaStream_t s = ctx->stream;
    const int64_t cells = (int64_t)ctx->t.Nk * ctx->t.Nk;
    const int Q3 = ctx->t.Q * 3;
    FinArgs f{};
    for (int q = 0; q < ctx->t.Q; ++q) { f.nq[q] = ctx->t.nq[q]; f.w[q] = ctx->t.w[q]; }
    f.N = (double)ctx->b.N;
    f.vF_ms = ctx->t.vF_ms;
    f.Q = ctx->t.Q;
    f.g1 = ctx->run->grid1();
    f.g2 = ctx->run->grid2();
    auto is_out = [&](int64_t n) { return moments_every > 0 && ((n + 1) % moments_every == 0); };
    auto hist_max = [&](int64_t n) {
        if (ctx->t.pauli_mode != PGC_PAULI_CURRENT_MAX) return;
        k_hist_max<<<ctx->t.Q, 256, 0, s>>>(ctx->b.hist + (int64_t)(n % kHistBufs) * ctx->b.hist_stride, cells, ctx->b.nmax);
        count_launch();
    };
    // record of step n: phase-1 partials of step n (g1 blocks), phase-2 partials of step n (g2
    // blocks) and, when phase 2 of step n - 1 carried particles into step n, its partials of step
    // n (g3 blocks)
    // the record of step n from the partials of its slot, on stream fs
    auto finalize = [&](int64_t n, int g2, int g3, cudaStream_t fs) {
        f.t_fs = (n + 1) * ctx->t.dt;
        f.g2 = g2;
        f.g3 = g3;
        const int64_t slot = n % kPartSlots;
        const double *p3 = g3 > 0 ? ctx->b.partN + slot * (int64_t)kGrid2Max * Q3 : nullptr;
        k_finalize_cols<<<Q3, kFinColThreads, 0, fs>>>(ctx->b.part1 + slot * ctx->b.part1_stride,
                                                       ctx->b.part2 + slot * ctx->b.part2_stride, p3, f, ctx->colsum,
                                                       ctx->b.qcount + 3, ctx->series + ctx->T_out * ctx->rec_len);
        count_launch();
        ctx->T_out++;
    };
    // kernel timing events of step n (4 per sample), or nullptr
    auto prof_slot = [&](int64_t n, cudaEvent_t **out) -> cudaError_t {
        *out = nullptr;
        if (!(ctx->prof_every > 0 && (n % ctx->prof_every) == 0)) return cudaSuccess;
        if (ctx->prof_used * 4 + 4 > (int)ctx->prof_ev.size()) {
            cudaError_t se = cudaStreamSynchronize(s);
            if (se != cudaSuccess) return se;
            prof_collect(ctx);
        }
        if (!ctx->prof_ref_set) {
            cudaError_t re = cudaEventRecord(ctx->prof_ref, s);
            if (re != cudaSuccess) return re;
            ctx->prof_ref_set = true;
        }
        *out = &ctx->prof_ev[(size_t)4 * ctx->prof_used++];
        return cudaSuccess;
    };
    const int64_t n0 = ctx->step;
    const int g2 = ctx->run->grid2(), g2f = ctx->run->grid2f();
    cudaError_t e = cudaSuccess;
    // The records are reduced on a second stream of the highest priority, beside the next step
    // launches: the record of step m (slot m % kPartSlots) is queued there behind the launch that
    // completes it, and the first launch that overwrites that slot (step m + 3) waits for it.  The
    // call ends by joining that stream, so that the caller's stream orders everything it did.
    bool pending[kPartSlots] = {false, false, false};
    if (moments_every > 0 && n_steps > 0) e = fin_stream_of(ctx);
    const cudaStream_t fs = ctx->fin_stream;
    auto finalize_async = [&](int64_t m, int g2v, int g3v) {
        cudaError_t r = cudaEventRecord(ctx->fin_ready, s);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(fs, ctx->fin_ready, 0);
        if (r != cudaSuccess) return r;
        finalize(m, g2v, g3v, fs);
        pending[m % kPartSlots] = true;
        return cudaEventRecord(ctx->fin_done[m % kPartSlots], fs);
    };
    auto before_writing = [&](int64_t k) {   // a launch that overwrites the partials of slot k % kPartSlots
        const int sl = (int)(k % kPartSlots);
        if (!pending[sl]) return cudaSuccess;
        pending[sl] = false;
        return cudaStreamWaitEvent(s, ctx->fin_done[sl], 0);
    };
    if (e == cudaSuccess && (!ctx->pipeline || n_steps < 2)) {
        for (int64_t k = 0; k < n_steps && e == cudaSuccess; ++k) {
            const int64_t n = n0 + k;
            hist_max(n);
            cudaEvent_t *ev = nullptr;
            if ((e = prof_slot(n, &ev)) != cudaSuccess) break;
            if ((e = before_writing(n)) != cudaSuccess) break;
            e = ctx->run->step(n, is_out(n), s, ev);
            if (e == cudaSuccess && is_out(n)) e = finalize_async(n, g2, 0);
        }
    } else if (e == cudaSuccess) {
        // Pipelined form: phase 1 of step n0, then one fused launch per step n (phase 1 of n
        // beside phase 2 of n - 1, which carries its particles into step n), then phase 2 of the
        // last step, so that the call ends on a step boundary.  The record of step n - 1 is
        // complete after the fused launch of step n.
        const int64_t n1 = n0 + n_steps - 1;
        // the bitmap of step n0 may hold bits left by steps taken outside this context's kernels
        e = cudaMemsetAsync(ctx->b.marks + (n0 % kMarkSlots) * ctx->b.mark_words, 0, (size_t)ctx->b.mark_words * 4, s);
        if (e == cudaSuccess) {
            hist_max(n0);
            e = ctx->run->phase1(n0, is_out(n0), s);
        }
        for (int64_t n = n0 + 1; n <= n1 && e == cudaSuccess; ++n) {
            hist_max(n - 1);
            cudaEvent_t *ev = nullptr;
            if ((e = prof_slot(n, &ev)) != cudaSuccess) break;
            if ((e = before_writing(n)) != cudaSuccess) break;
            if (ev) cudaEventRecord(ev[0], s);
            e = ctx->run->step_fused(n, is_out(n), is_out(n - 1), s);
            if (ev) for (int j = 1; j < 4; ++j) cudaEventRecord(ev[j], s);
            if (e == cudaSuccess && is_out(n - 1)) e = finalize_async(n - 1, g2f, n - 1 > n0 ? g2f : 0);
        }
        if (e == cudaSuccess) {
            hist_max(n1);
            e = before_writing(n1);
            if (e == cudaSuccess) e = ctx->run->phase2(n1, is_out(n1), s);
            if (e == cudaSuccess && is_out(n1)) e = finalize_async(n1, g2, n1 > n0 ? g2f : 0);
        }
    }
    for (int sl = 0; sl < kPartSlots; ++sl)
        if (pending[sl]) {
            cudaError_t r = cudaStreamWaitEvent(s, ctx->fin_done[sl], 0);
            if (e == cudaSuccess) e = r;
        }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "step");
    ctx->step = n0 + n_steps;
    return PGC_OK;
}

pgc_status pgc_set_pipeline(pgc_ctx *ctx, int32_t on)
{
    if (!ctx) return fail(nullptr, PGC_EINVAL, "ctx is NULL");
    if (on != 0 && on != 1) return fail(ctx, PGC_EINVAL, "on must be 0 or 1");
    if (on && !ctx->run->fused()) return fail(ctx, PGC_EUNSUPPORTED, "no pipelined step kernel for this shape (P * Q > 64)");
    ctx->pipeline = on;
    return PGC_OK;
}

pgc_status pgc_moments(pgc_ctx *ctx, double *h_t_fs, double *h_mean, double *h_var, double *h_nodes, int64_t *T_out)
{
    if (!ctx) return fail(nullptr, PGC_EINVAL, "ctx is NULL");
    if (ctx->failed) return fail(ctx, PGC_ESTATE, "context failed earlier: " + ctx->err);
    const int64_t T = ctx->T_out;
    const int Q = ctx->t.Q, RL = ctx->rec_len;
    std::vector<double> buf((size_t)T * RL);
    unsigned long long dev_err = 0;
    cudaError_t e = cudaSuccess;
    if (T > 0) e = cudaMemcpyAsync(buf.data(), ctx->series, buf.size() * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&dev_err, ctx->b.counters + PGC_CNT_ERROR, sizeof(dev_err), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "moments copy");
    if (dev_err & 1ull) return fail(ctx, PGC_ETIMEOUT, "a bounded wait for the tensor cores gave up in a step; the results are not valid");
    for (int64_t t = 0; t < T; ++t) {
        const double *r = &buf[(size_t)t * RL];
        if (h_t_fs) h_t_fs[t] = r[0];
        if (h_nodes) std::memcpy(h_nodes + (size_t)t * Q * 4, r + 1, sizeof(double) * Q * 4);
        if (h_mean) std::memcpy(h_mean + (size_t)t * 4, r + 1 + Q * 4, sizeof(double) * 4);
        if (h_var) std::memcpy(h_var + (size_t)t * 4, r + 1 + Q * 4 + 4, sizeof(double) * 4);
    }
    if (T_out) *T_out = T;
    return PGC_OK;
}

pgc_status pgc_get_state(pgc_ctx *ctx, double *h_khat)
{
    if (!ctx || !h_khat) return fail(ctx, PGC_EINVAL, "NULL argument");
    if (ctx->failed) return fail(ctx, PGC_ESTATE, "context failed earlier: " + ctx->err);
    const int P = ctx->t.P;
    const int64_t N = ctx->b.N, ld = ctx->b.ld;
    const bool f64 = ctx->cfg.precision == PGC_FP64;
    const size_t esz = f64 ? 8 : 4;
    const size_t bytes = (size_t)2 * P * ld * esz;
    char *tmp = (char *)staging(ctx, bytes);
    if (!tmp) return fail(ctx, PGC_ENOMEM, "pinned staging buffer");
    cudaError_t e = cudaMemcpyAsync(tmp, ctx->b.state, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "state copy");
    for (int p = 0; p < 2 * P; ++p) {
        const double sh = (p < P) ? ctx->t.dhalf[p] : 0.0;   // Strang: back to the step boundary
        host_parallel(N, [&](int64_t lo, int64_t hi) {
            for (int64_t i = lo; i < hi; ++i) {
                const double v = f64 ? ((const double *)tmp)[(size_t)p * ld + i]
                                     : (double)((const float *)tmp)[(size_t)p * ld + i];
                h_khat[(size_t)p * N + i] = (sh != 0.0) ? v - sh : v;
            }
        });
    }
    return PGC_OK;
}

pgc_status pgc_set_state(pgc_ctx *ctx, const double *h_khat)
{
    if (!ctx || !h_khat) return fail(ctx, PGC_EINVAL, "NULL argument");
    if (ctx->failed) return fail(ctx, PGC_ESTATE, "context failed earlier: " + ctx->err);
    const int P = ctx->t.P;
    const int64_t N = ctx->b.N, ld = ctx->b.ld;
    const bool f64 = ctx->cfg.precision == PGC_FP64;
    const size_t esz = f64 ? 8 : 4;
    const size_t bytes = (size_t)2 * P * ld * esz;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);  // the staging buffer may still be in use
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sync");
    char *tmp = (char *)staging(ctx, bytes);
    if (!tmp) return fail(ctx, PGC_ENOMEM, "pinned staging buffer");
    for (int p = 0; p < 2 * P; ++p) {
        const double sh = (p < P) ? ctx->t.dhalf[p] : 0.0;   // Strang: half a drift ahead
        host_parallel(N, [&](int64_t lo, int64_t hi) {
            for (int64_t i = lo; i < hi; ++i) {
                const double v = (sh != 0.0) ? h_khat[(size_t)p * N + i] + sh : h_khat[(size_t)p * N + i];
                if (f64) ((double *)tmp)[(size_t)p * ld + i] = v;
                else ((float *)tmp)[(size_t)p * ld + i] = (float)v;
            }
        });
        for (int64_t i = N; i < ld; ++i) {
            if (f64) ((double *)tmp)[(size_t)p * ld + i] = 0.0;
            else ((float *)tmp)[(size_t)p * ld + i] = 0.0f;
        }
    }
    ctx->sampled = false;
    e = cudaMemcpyAsync(ctx->b.state, tmp, bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "state upload");
    // the histogram of the uploaded state becomes f^n (the Pauli normaliser is kept)
    if (ctx->T_out > 0) return observe_current(ctx, false, false);
    return PGC_OK;
}

pgc_status pgc_get_state_native(pgc_ctx *ctx, void *h_state)
{
    if (!ctx || !h_state) return fail(ctx, PGC_EINVAL, "NULL argument");
    if (ctx->failed) return fail(ctx, PGC_ESTATE, "context failed earlier: " + ctx->err);
    const size_t bytes = (size_t)2 * ctx->t.P * ctx->b.ld * (ctx->cfg.precision == PGC_FP64 ? 8 : 4);
    cudaError_t e = cudaMemcpyAsync(h_state, ctx->b.state, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "state copy");
    return PGC_OK;
}

pgc_status pgc_set_state_native(pgc_ctx *ctx, const void *h_state)
{
    if (!ctx || !h_state) return fail(ctx, PGC_EINVAL, "NULL argument");
    if (ctx->failed) return fail(ctx, PGC_ESTATE, "context failed earlier: " + ctx->err);
    const size_t bytes = (size_t)2 * ctx->t.P * ctx->b.ld * (ctx->cfg.precision == PGC_FP64 ? 8 : 4);
    ctx->sampled = false;
    cudaError_t e = cudaMemcpyAsync(ctx->b.state, h_state, bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "state upload");
    // the histogram of the uploaded state becomes f^n (the Pauli normaliser is kept)
    if (ctx->T_out > 0) return observe_current(ctx, false, false);
    return PGC_OK;
}

pgc_status pgc_counters(pgc_ctx *ctx, uint64_t *h)
{
    if (!ctx || !h) return fail(ctx, PGC_EINVAL, "NULL argument");
    if (ctx->failed) return fail(ctx, PGC_ESTATE, "context failed earlier: " + ctx->err);
    unsigned long long c[8];
    cudaError_t e = cudaMemcpyAsync(c, ctx->b.counters, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "counters copy");
    for (int k = 0; k < 8; ++k) h[k] = c[k];
    h[PGC_CNT_STEPS] = (uint64_t)ctx->step;
    return PGC_OK;
}

pgc_status pgc_get_hist(pgc_ctx *ctx, uint32_t *h_hist, uint32_t *h_nmax)
{
    if (!ctx) return fail(nullptr, PGC_EINVAL, "ctx is NULL");
    if (ctx->failed) return fail(ctx, PGC_ESTATE, "context failed earlier: " + ctx->err);
    const int cur = (int)(ctx->step % kHistBufs);
    cudaError_t e = cudaSuccess;
    if (h_hist)
        e = cudaMemcpyAsync(h_hist, ctx->b.hist + (int64_t)cur * ctx->b.hist_stride,
                            (size_t)ctx->t.Q * ctx->t.Nk * ctx->t.Nk * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && h_nmax)
        e = cudaMemcpyAsync(h_nmax, ctx->b.nmax, (size_t)ctx->t.Q * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hist copy");
    return PGC_OK;
}

pgc_status pgc_reconstruct_f(pgc_ctx *ctx, const double *h_z, int32_t nz, uint32_t *h_hist, uint32_t *h_max)
{
    if (!ctx) return fail(nullptr, PGC_EINVAL, "ctx is NULL");
    if (ctx->failed) return fail(ctx, PGC_ESTATE, "context failed earlier: " + ctx->err);
    if (nz < 0 || (nz > 0 && ((!h_z && ctx->t.d > 0) || !h_hist || !h_max))) return fail(ctx, PGC_EINVAL, "bad arguments");
    const int d = ctx->t.d, P = ctx->t.P;
    const int64_t cells = (int64_t)ctx->t.Nk * ctx->t.Nk;
    std::vector<double> psi(P);
    for (int j = 0; j < nz; ++j) {
        if (d > 0)
            for (int k = 0; k < d; ++k)
                if (!(h_z[(size_t)j * d + k] >= -1.0 && h_z[(size_t)j * d + k] <= 1.0))
                    return fail(ctx, PGC_EINVAL, "z outside [-1,1]");
        basis_at(d, ctx->cfg.degree_M, d ? &h_z[(size_t)j * d] : nullptr, psi.data());
        double xs = 0.0;   // Strang: half the drift at z
        for (int h = 0; h < P; ++h) xs += ctx->t.dhalf[h] * psi[h];
        cudaError_t e = cudaMemsetAsync(ctx->b.recon_hist, 0, cells * 4, ctx->stream);
        if (e == cudaSuccess) e = ctx->run->hist_at(psi.data(), xs, ctx->b.recon_hist, ctx->stream);
        if (e == cudaSuccess) {
            k_hist_max<<<1, 256, 0, ctx->stream>>>(ctx->b.recon_hist, cells, ctx->tmp_max);
            count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_hist + (size_t)j * cells, ctx->b.recon_hist, cells * 4, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_max + j, ctx->tmp_max, 4, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "reconstruct_f");
    }
    return PGC_OK;
}

pgc_status pgc_observe_at(pgc_ctx *ctx, const double *h_z, int32_t nz, double *h_out)
{
    if (!ctx) return fail(nullptr, PGC_EINVAL, "ctx is NULL");
    if (ctx->failed) return fail(ctx, PGC_ESTATE, "context failed earlier: " + ctx->err);
    const int d = ctx->t.d, P = ctx->t.P;
    if (nz < 0 || (nz > 0 && (!h_out || (!h_z && d > 0)))) return fail(ctx, PGC_EINVAL, "bad arguments");
    for (int64_t j = 0; j < (int64_t)nz * d; ++j)
        if (!(h_z[j] >= -1.0 && h_z[j] <= 1.0)) return fail(ctx, PGC_EINVAL, "z outside [-1,1]");
    const HostTables &t = ctx->t;
    std::vector<double> psi((size_t)kObsZ * P), e0(kObsZ), xs(kObsZ);
    for (int j0 = 0; j0 < nz; j0 += kObsZ) {
        const int nzc = std::min(kObsZ, nz - j0);
        ObsFin f{};
        for (int l = 0; l < nzc; ++l) {
            const double *z = d ? &h_z[(size_t)(j0 + l) * d] : nullptr;
            basis_at(d, ctx->cfg.degree_M, z, &psi[(size_t)l * P]);
            // z1 is the band-minimum variable when the band minimum is random
            const double ze = ((d == 1 && t.eps_random) || d == 2) ? z[0] : 0.0;
            e0[l] = eps0_at(ctx->cfg, t.hvF, ze);
            xs[l] = 0.0;   // Strang: half the drift at z
            for (int h = 0; h < P; ++h) xs[l] += t.dhalf[h] * psi[(size_t)l * P + h];
            f.n[l] = 2.0 / (kPi * t.hvF * t.hvF) * fd_upper<double>(e0[l], ctx->cfg.eps_F_eV, t.kT) * 1.0e18;
        }
        int g = 0;
        cudaError_t e = ctx->run->obs_at(psi.data(), e0.data(), xs.data(), nzc, ctx->obs_part, &g, ctx->stream);
        if (e == cudaSuccess) {
            f.scale_v = t.hvF * t.vF_ms / (double)ctx->b.N;
            f.inv_N = 1.0 / (double)ctx->b.N;
            f.nz = nzc;
            f.g = g;
            k_obs_fin<<<1, 128, 0, ctx->stream>>>(ctx->obs_part, f, ctx->obs_out);
            count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_out + (size_t)j0 * 4, ctx->obs_out, (size_t)nzc * 4 * 8, cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "observe_at");
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "observe_at");
    return PGC_OK;
}

pgc_status pgc_profile(pgc_ctx *ctx, int32_t every)
{
    if (!ctx) return fail(nullptr, PGC_EINVAL, "ctx is NULL");
    if (every < 0) return fail(ctx, PGC_EINVAL, "every < 0");
    if (every > 0 && ctx->prof_ev.empty()) {
        ctx->prof_ev.resize(4 * 256);
        for (auto &ev : ctx->prof_ev) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "event create");
        }
        cudaError_t e = cudaEventCreate(&ctx->prof_ref);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "event create");
    }
    ctx->prof_every = every;
    ctx->prof_used = 0;
    ctx->prof_ms[0] = ctx->prof_ms[1] = 0.0;
    ctx->prof_samples = 0;
    ctx->prof_ref_set = false;
    ctx->prof_tl.clear();
    return PGC_OK;
}

pgc_status pgc_profile_timeline(pgc_ctx *ctx, double *h_t, int64_t max_samples, int64_t *n_samples)
{
    if (!ctx || !n_samples || max_samples < 0 || (max_samples > 0 && !h_t)) return fail(ctx, PGC_EINVAL, "bad arguments");
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "profile sync");
    prof_collect(ctx);
    const int64_t n = std::min<int64_t>(max_samples, (int64_t)(ctx->prof_tl.size() / 4));
    for (int64_t k = 0; k < 4 * n; ++k) h_t[k] = ctx->prof_tl[(size_t)k];
    *n_samples = (int64_t)(ctx->prof_tl.size() / 4);
    return PGC_OK;
}

pgc_status pgc_profile_read(pgc_ctx *ctx, double *ms_phase1, double *ms_phase2, int64_t *samples)
{
    if (!ctx) return fail(nullptr, PGC_EINVAL, "ctx is NULL");
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "profile sync");
    prof_collect(ctx);
    const double n = ctx->prof_samples > 0 ? (double)ctx->prof_samples : 1.0;
    if (ms_phase1) *ms_phase1 = ctx->prof_ms[0] / n;
    if (ms_phase2) *ms_phase2 = ctx->prof_ms[1] / n;
    if (samples) *samples = ctx->prof_samples;
    return PGC_OK;
}

void pgc_destroy(pgc_ctx *ctx)
{
    if (!ctx) return;
    for (auto &ev : ctx->prof_ev) cudaEventDestroy(ev);
    if (ctx->prof_ref) cudaEventDestroy(ctx->prof_ref);
    if (ctx->fin_stream) cudaStreamDestroy(ctx->fin_stream);
    if (ctx->fin_ready) cudaEventDestroy(ctx->fin_ready);
    for (auto &ev : ctx->fin_done)
        if (ev) cudaEventDestroy(ev);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    delete ctx->run;
    delete ctx;
}

const char *pgc_last_error(const pgc_ctx *ctx)
{
    if (ctx) return ctx->err.c_str();
    static thread_local std::string copy;
    std::lock_guard<std::mutex> lk(g_err_mu);
    copy = g_err;
    return copy.c_str();
}

const char *pgc_status_string(pgc_status s)
{
    switch (s) {
    case PGC_OK: return "PGC_OK";
    case PGC_EINVAL: return "PGC_EINVAL";
    case PGC_ENOMEM: return "PGC_ENOMEM";
    case PGC_ECUDA: return "PGC_ECUDA";
    case PGC_ESTATE: return "PGC_ESTATE";
    case PGC_ETIMEOUT: return "PGC_ETIMEOUT";
    case PGC_EUNSUPPORTED: return "PGC_EUNSUPPORTED";
    }
    return "unknown status";
}

uint64_t pgc_launch_count(void) { return g_launches.load(); }

}  // extern "C"
