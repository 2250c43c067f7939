// pgc_kernels.cuh -- the time-step kernels of the particle stochastic-Galerkin scheme
// (arXiv:2404.19602, Algorithm 1 for P = Q = 1, Algorithm 2 otherwise), templated on the gPC
// basis size P, the number of quadrature nodes Q and the arithmetic type R.
//
// One time step n is two launches:
//   k_phase1 (every particle, streaming): drift of the coefficients (Eq. (17), Sec. 4.1),
//       reconstruction at the Q nodes (Eq. (23)), first flight-time draw, and a conservative
//       rate bound that proves "no collision in this step" for most particles; those are
//       finished here (histogram f^{n+1} of Eq. (24), moments).  The rest are appended to a
//       collider queue.  It also clears the histogram buffer of step n+2 and the next queue
//       counter, so that no separate memset is needed.
//   k_phase2 (queued particles only): the exact collision loop of Algorithm 1 / 2 with the
//       Pauli test against f^n, then the histogram f^{n+1} and moments of the final state.
// On moment steps a one-block k_finalize reduces the block partial sums in a fixed order and
// writes the node values, mean and variance of the record (Sec. 4.2).
//
// Pipelined form (several steps per call): k_phase2<EXT = true> of step n, after the collision
// loop of a queued particle, carries that particle on through the drift and the flight-time
// screen of step n + 1 (finishing it there, or queueing it for step n + 1), and k_phase1 of step
// n + 1 skips the particles queued at step n (a bitmap).  The two kernels then touch disjoint
// particles and buffers and run concurrently on two streams; every particle undergoes the same
// arithmetic as in the two-launch form, so the trajectories are identical.
#pragma once

#include "pgc_device.cuh"

namespace pgc {

constexpr int kPhase1Threads = 256;
constexpr int kPhase2Threads = 128;
constexpr int kMaxGrid1 = 4096;   // block partials sized for at most this many phase-1 blocks
constexpr int kGrid2 = 608;       // phase-2 blocks (grid-stride over the queue)
// Phase-2 blocks per SM the collider kernel is compiled for (four: no spills at 36 nodes; five
// were measured 1 % slower with the collider's rolled slot loops, six slower still).
template <int P, int Q> struct Phase2Blocks { static constexpr int per_sm = 4; };
constexpr int kGrid2Max = 5 * 152; // phase-2 partial sums are sized for this many blocks
// Block-private histogram window of phase 1: kWin x kWin cells per node around the grid centre,
// 16-bit counts packed two per 32-bit word in shared memory, flushed to the global histogram once
// per block.  Cells outside the window go straight to the global histogram.
constexpr int kWin = 32;
constexpr int kWinWords = kWin * kWin / 2;
// Rotating buffers.  Histogram f^n lives in buffer n % kHistBufs: while phase 2 of step n - 1
// (reading f^{n-1}, writing f^n and f^{n+1}) runs beside phase 1 of step n (writing f^{n+1},
// clearing f^{n+2}), four buffers are in use.  Collider counters: n % 3; queues and moment
// partials: n % 2; collider bitmaps: n % 3.
constexpr int kHistBufs = 4;
constexpr int kQSlots = 3;
// Moment partial sums of step n (streaming part1, collider part2, carried partN) live in slot
// n % kPartSlots: the record of step m is reduced beside the launches of steps m + 1 and m + 2,
// and step m + 3 is the first to overwrite its slot.
constexpr int kPartSlots = 3;
constexpr int kMarkSlots = 3;

// Basis of total degree <= 5 in two variables on 6 x 6 tensor nodes (the compiled 2-D shape):
// coefficient (h1, h2) sits at index t(t+1)/2 + h2 with t = h1 + h2.
template <int P, int Q> struct TensorShape { static constexpr bool value = (P == 21 && Q == 36); };
__host__ __device__ constexpr int hidx2(int h1, int h2) { return (h1 + h2) * (h1 + h2 + 1) / 2 + h2; }

// Quadrature / basis tables of one context (Sec. 4.1).
template <int P, int Q, typename R>
struct Nodes {
    R psi[Q * P];    // Psi_h(z_q), [q][h]
    R wpsi[Q * P];   // w_q Psi_h(z_q)
    R dhat[P];       // per-step drift of the x coefficients
    R eps0[Q];       // band minimum at the node
    R dq[Q];         // per-step drift (e/hbar) E(z_q) dt at the node
    R lkx[Q];        // x offset of the grid at the node: Lk, or Lk - dq/2 (Strang)
    R xs[Q];         // x shift from the stored state to the state at the step boundary: 0, or dq/2 (Strang)
    R eps0_max;
    uint32_t drift_mask;  // coefficients h with dhat[h] != 0
    // 2-D tensor nodes (P = 21, Q = 36): one-dimensional basis values for sum factorisation,
    // a1[q1][h1] = psi_h1(z1_q1), b2[q2][h2] = psi_h2(z2_q2)
    R a1[36], b2[36];
    // FP32: the same weights as pairs (w, w), the operand of the two-lane FMA that reconstructs
    // the x and y components together (one unused entry in FP64)
    unsigned long long psi2[(TensorShape<P, Q>::value || sizeof(R) == 8) ? 1 : Q * P];
    unsigned long long wpsi2[(TensorShape<P, Q>::value || sizeof(R) == 8) ? 1 : Q * P];
    unsigned long long a1_2[36], b2_2[36];
};

template <int P, int Q, typename R>
struct StepArgs {
    Phys<R> ph;
    Nodes<P, Q, R> nd;
    R *khat;                 // [2][P][ld]
    int64_t N, ld;
    const uint32_t *Hcur;    // f^n   [Q][Nk*Nk]
    uint32_t *Hnext;         // f^{n+1}
    uint32_t *Hclear;        // buffer of step n+2, cleared by phase 1
    int64_t hist_elems;      // Q*Nk*Nk
    const uint32_t *nmax;    // [Q]
    uint32_t *queue;         // [N]
    uint32_t *qcount;        // collider count of this step
    uint32_t *qcount_next;   // counter of the next step (zeroed by phase 1)
    uint32_t *tilectr;       // phase-1 tile counter of this step (nullptr: static tile assignment)
    uint32_t *tilectr_next;  // tile counter of the next step (zeroed by phase 1)
    double *part1;           // [gridDim(phase1)][Q*3]
    double *part2;           // [kGrid2Max][Q*3]
    unsigned long long *counters;
    uint32_t key0, key1, stream_id, step;
    int32_t out_step;        // 1: accumulate the moments of the post-step state
    int32_t win_r0;          // first row / column of the shared-memory window
    int32_t use_win;         // 1: phase 1 counts into the shared-memory window
    // collider bitmaps (bit i of word i / 32), all optional (nullptr)
    const uint32_t *skip;    // phase 1: particles queued at step n - 1, owned by a concurrent phase 2
    uint32_t *mark;          // phase 1: set for every particle queued at step n
    uint32_t *mark_clear;    // phase 1: bitmap of step n + 1, cleared
    int64_t mark_words;      // words per bitmap (multiple of 4)
    // phase 2 continuation into step n + 1 (k_phase2<EXT = true>)
    uint32_t *Hnext2;        // f^{n+2}
    uint32_t *queue_next;    // collider queue of step n + 1 (its counter is qcount_next)
    uint32_t *mark_next;     // bitmap of step n + 1
    double *partN;           // [kGrid2Max][Q*3] moments of step n + 1 of the particles finished here
    int32_t out_next;        // 1: step n + 1 is a moment step
    const Nodes<P, Q, R> *nd_dev;  // device copy of nd (phase 2 stages it into shared memory)
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-warp moment accumulators of the streaming kernels.  FP64 in the FP64 mode.  In the FP32
// mode a float-float pair (hi, lo) advanced by the error-free transformation TwoSum (Knuth,
// TAOCP vol. 2, 4.2.2): hi + lo carries ~48 significant bits, and no operation runs on the FP64
// pipe, which on this part issues a small fraction of the FP32 rate.  The block's partial sum
// is then formed in FP64 from hi + lo, in a fixed warp order.
template <typename R> struct MomAcc;
template <> struct MomAcc<double> { using T = double; };
template <> struct MomAcc<float> { using T = float2; };
__device__ __forceinline__ void acc_zero(double &a) { a = 0.0; }
__device__ __forceinline__ void acc_zero(float2 &a) { a = make_float2(0.0f, 0.0f); }
__device__ __forceinline__ void acc_add(double &a, double x) { a += x; }
__device__ __forceinline__ void acc_add(float2 &a, float x)
{
    const float s = a.x + x;
    const float bp = s - a.x;
    const float err = (a.x - (s - bp)) + (x - bp);
    a.x = s;
    a.y += err;
}
__device__ __forceinline__ double acc_value(double a) { return a; }
__device__ __forceinline__ double acc_value(float2 a) { return (double)a.x + (double)a.y; }

// Warp sums of 16 values at once (a reduce-scatter): lane l ends with the sum over the 32 lanes
// of v[(l >> 1) & 15] (lanes l and l ^ 1 hold the same sum), after 16 shuffles instead of the
// 80 of 16 separate butterflies.  The lanes with l even add their sum to the accumulator
// dst[(l >> 1)] when that index is below count.
__device__ __forceinline__ void warp_scatter16_add(const float v[16], float2 *dst, int count, int lane)
{
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const bool up = lane & 16;
        const float send = up ? v[j] : v[j + 8], keep = up ? v[j + 8] : v[j];
        a[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool up = lane & 8;
        const float send = up ? a[j] : a[j + 4], keep = up ? a[j + 4] : a[j];
        a[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const bool up = lane & 4;
        const float send = up ? a[j] : a[j + 2], keep = up ? a[j + 2] : a[j];
        a[j] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool up = lane & 2;
        const float send = up ? a[0] : a[1], keep = up ? a[1] : a[0];
        a[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
    const int idx = (lane >> 1) & 15;
    if (!(lane & 1) && idx < count) acc_add(dst[idx], a[0]);
}

// s + p[b * n3 + col] summed over b = b0, b0 + step, ... < b1 in that order (the fixed-order
// reductions of the block partials).  The loads are issued eight at a time ahead of their adds,
// so a thread waits for one memory round trip per eight rows instead of one per row; the sum is
// the plain loop's, bit for bit.
__device__ __forceinline__ double strided_sum(const double *p, int64_t b0, int64_t b1, int step, int n3, int col, double s)
{
    for (int64_t b = b0; b < b1; b += 8 * (int64_t)step) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t bb = b + (int64_t)k * step;
            v[k] = bb < b1 ? p[bb * n3 + col] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (b + (int64_t)k * step < b1) s += v[k];
    }
    return s;
}

// The same for 4 values: lane l ends with the sum over the 32 lanes of v[(l >> 3) & 3]; lanes
// 0, 8, 16, 24 add their sum to the accumulator dst[l >> 3] when that index is below count.
__device__ __forceinline__ void warp_scatter4_add(const float v[4], float2 *dst, int count, int lane)
{
    float a[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const bool up = lane & 16;
        const float send = up ? v[j] : v[j + 2], keep = up ? v[j + 2] : v[j];
        a[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    {
        const bool up = lane & 8;
        const float send = up ? a[0] : a[1], keep = up ? a[1] : a[0];
        a[0] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) a[0] += __shfl_xor_sync(0xffffffffu, a[0], o);
    const int idx = (lane >> 3) & 3;
    if (!(lane & 7) && idx < count) acc_add(dst[idx], a[0]);
}

// |k|^2 and the screen of the first flight time with an explicit operation order, so that
// phase 1 and the continuation in phase 2 take bit-identical decisions.
template <typename R>
__device__ __forceinline__ R knorm2(R kx, R ky)
{
    if constexpr (sizeof(R) == 8) return __fma_rn(kx, kx, __dmul_rn(ky, ky));
    else return __fmaf_rn(kx, kx, __fmul_rn(ky, ky));
}

template <int P, int Q, typename R>
__device__ __forceinline__ bool screen_maybe(const Phys<R> &ph, const Nodes<P, Q, R> &nd, R kkmax, uint32_t xi_bits)
{
    const R lnxi = -rlog<R>(u01<R>(xi_bits));
    const R emax = rsqrt_<R>(ph.hvF2 * kkmax + nd.eps0_max * nd.eps0_max);
    const R gub = ph.alpha1 * rate_bound(ph, emax, nd.eps0_max) * (R)1.0001;
    return lnxi < gub * ph.dt;
}

template <int P, int Q, typename R>
__device__ __forceinline__ void load_coeffs(const StepArgs<P, Q, R> &a, int64_t i, R cx[P], R cy[P])
{
#pragma unroll
    for (int h = 0; h < P; ++h) {
        cx[h] = a.khat[(int64_t)h * a.ld + i];
        cy[h] = a.khat[(int64_t)(P + h) * a.ld + i];
    }
}

// Two FP32 fused multiply-adds in one instruction (packed f32x2 of sm_100+; each lane rounds as
// a scalar fmaf, so results are those of the scalar code): (x, y) pairs share a weight (w, w).
struct F2 { unsigned long long v; };
__device__ __forceinline__ F2 f2_pack(float a, float b)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(F2 p, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(p.v)); }
__device__ __forceinline__ F2 f2_fma(F2 a, unsigned long long w2, F2 c)
{
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(w2), "l"(c.v));
    return r;
}

template <int P, int Q, typename R>
__device__ __forceinline__ void recon_node(const Nodes<P, Q, R> &nd, int q, const R cx[P], const R cy[P],
                                           R &kx, R &ky)
{
    if constexpr (sizeof(R) == 4 && !TensorShape<P, Q>::value) {
        F2 s = f2_pack(0.f, 0.f);
#pragma unroll
        for (int h = 0; h < P; ++h) s = f2_fma(f2_pack(cx[h], cy[h]), nd.psi2[q * P + h], s);
        f2_unpack(s, kx, ky);
    } else {
        R sx = (R)0, sy = (R)0;
#pragma unroll
        for (int h = 0; h < P; ++h) {
            sx += cx[h] * nd.psi[q * P + h];
            sy += cy[h] * nd.psi[q * P + h];
        }
        kx = sx;
        ky = sy;
    }
}

// Reconstruction at every node (Eq. 23), calling f(q, kx, ky) per node.  For the 2-D tensor
// shape the sum is factorised: t(q1, h2) = sum_h1 c(h1,h2) a_h1(q1), k(q1,q2) = sum_h2 t b_h2(q2)
// (2 x 342 instead of 2 x 756 multiply-adds per particle).
template <int P, int Q, typename R, typename F>
__device__ __forceinline__ void recon_all(const Nodes<P, Q, R> &nd, const R cx[P], const R cy[P], F &&f)
{
    if constexpr (TensorShape<P, Q>::value && sizeof(R) == 4) {
        F2 c2[P];
#pragma unroll
        for (int h = 0; h < P; ++h) c2[h] = f2_pack(cx[h], cy[h]);
#pragma unroll
        for (int q1 = 0; q1 < 6; ++q1) {
            F2 t2[6];
#pragma unroll
            for (int h2 = 0; h2 < 6; ++h2) {
                F2 s2 = f2_pack(0.f, 0.f);
#pragma unroll
                for (int h1 = 0; h1 + h2 <= 5; ++h1) s2 = f2_fma(c2[hidx2(h1, h2)], nd.a1_2[q1 * 6 + h1], s2);
                t2[h2] = s2;
            }
#pragma unroll
            for (int q2 = 0; q2 < 6; ++q2) {
                F2 k2 = f2_pack(0.f, 0.f);
#pragma unroll
                for (int h2 = 0; h2 < 6; ++h2) k2 = f2_fma(t2[h2], nd.b2_2[q2 * 6 + h2], k2);
                R kx, ky;
                f2_unpack(k2, kx, ky);
                f(q1 * 6 + q2, kx, ky);
            }
        }
    } else if constexpr (TensorShape<P, Q>::value) {
#pragma unroll
        for (int q1 = 0; q1 < 6; ++q1) {
            R tx[6], ty[6];
#pragma unroll
            for (int h2 = 0; h2 < 6; ++h2) {
                R sx = (R)0, sy = (R)0;
#pragma unroll
                for (int h1 = 0; h1 + h2 <= 5; ++h1) {
                    sx += cx[hidx2(h1, h2)] * nd.a1[q1 * 6 + h1];
                    sy += cy[hidx2(h1, h2)] * nd.a1[q1 * 6 + h1];
                }
                tx[h2] = sx;
                ty[h2] = sy;
            }
#pragma unroll
            for (int q2 = 0; q2 < 6; ++q2) {
                R kx = (R)0, ky = (R)0;
#pragma unroll
                for (int h2 = 0; h2 < 6; ++h2) {
                    kx += tx[h2] * nd.b2[q2 * 6 + h2];
                    ky += ty[h2] * nd.b2[q2 * 6 + h2];
                }
                f(q1 * 6 + q2, kx, ky);
            }
        }
    } else {
        // (large one-dimensional shapes: a rolled node loop keeps the code size in check)
#pragma unroll (P * Q <= 64 ? Q : 1)
        for (int q = 0; q < Q; ++q) {
            R kx, ky;
            recon_node(nd, q, cx, cy, kx, ky);
            f(q, kx, ky);
        }
    }
}

// The value recon_all produces at node q (same operations in the same order).
template <int P, int Q, typename R>
__device__ __forceinline__ void recon_at(const Nodes<P, Q, R> &nd, int q, const R cx[P], const R cy[P], R &kx, R &ky)
{
    if constexpr (TensorShape<P, Q>::value) {
        const int q1 = q / 6, q2 = q - 6 * (q / 6);
        R sx2 = (R)0, sy2 = (R)0;
#pragma unroll
        for (int h2 = 0; h2 < 6; ++h2) {
            R sx = (R)0, sy = (R)0;
#pragma unroll
            for (int h1 = 0; h1 + h2 <= 5; ++h1) {
                sx += cx[hidx2(h1, h2)] * nd.a1[q1 * 6 + h1];
                sy += cy[hidx2(h1, h2)] * nd.a1[q1 * 6 + h1];
            }
            sx2 += sx * nd.b2[q2 * 6 + h2];
            sy2 += sy * nd.b2[q2 * 6 + h2];
        }
        kx = sx2;
        ky = sy2;
    } else {
        recon_node(nd, q, cx, cy, kx, ky);
    }
}

// group velocity (units of vF) and energy at one node (Sec. 2).  The warp partial sums are
// taken in R (FP32 in the production mode, FP64 in the FP64 mode) and accumulated in FP64.
template <typename R>
__device__ __forceinline__ void observe(const Phys<R> &ph, R kx, R ky, R eps0, R &vx, R &vy, R &e)
{
    const R eps = rsqrt_<R>(ph.hvF2 * (kx * kx + ky * ky) + eps0 * eps0);
    vx = ph.hvF * kx / eps;
    vy = ph.hvF * ky / eps;
    e = eps;
}

// The same observables in FP32 from one reciprocal square root (rsqrtf, 2 ulp): 1/eps, eps and
// both velocity components (the 36-node moment steps, where the divisions were the cost).
__device__ __forceinline__ void observe_fast(const Phys<float> &ph, float kx, float ky, float eps0, float &vx, float &vy,
                                             float &e)
{
    const float s2 = ph.hvF2 * (kx * kx + ky * ky) + eps0 * eps0;
    const float inv = rsqrtf(s2);
    vx = ph.hvF * kx * inv;
    vy = ph.hvF * ky * inv;
    e = s2 * inv;
}

// ------------------------------------------------------------------------------------------
// Phase 1: every particle.  Each thread takes PPT consecutive particles and reads each
// coefficient plane with one 16-byte load (float4 / 2 x double2); the ensemble is streamed once.
// ------------------------------------------------------------------------------------------
template <int P> struct Phase1PPT { static constexpr int value = (P <= 8) ? 4 : 1; };
// resident blocks per SM the streaming kernels are compiled for: three for the small FP32
// shapes, two (more registers, no spills) for 36 nodes and for FP64
template <int P, int Q, typename R> struct kPhase1MinBlocks {
    static constexpr int value = (P * Q > 64 || sizeof(R) == 8) ? 2 : 3;
};

template <typename R, int PPT>
__device__ __forceinline__ void load_vec(const R *p, R v[PPT])
{
    if constexpr (PPT == 4 && sizeof(R) == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (PPT == 4 && sizeof(R) == 8) {
        const double2 a = reinterpret_cast<const double2 *>(p)[0];
        const double2 b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else if constexpr (PPT == 2 && sizeof(R) == 4) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x; v[1] = t.y;
    } else if constexpr (PPT == 2 && sizeof(R) == 8) {
        const double2 t = *reinterpret_cast<const double2 *>(p);
        v[0] = t.x; v[1] = t.y;
    } else {
#pragma unroll
        for (int e = 0; e < PPT; ++e) v[e] = p[e];
    }
}

template <typename R, int PPT>
__device__ __forceinline__ void store_vec(R *p, const R v[PPT])
{
    if constexpr (PPT == 4 && sizeof(R) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (PPT == 4 && sizeof(R) == 8) {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    } else if constexpr (PPT == 2 && sizeof(R) == 4) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else if constexpr (PPT == 2 && sizeof(R) == 8) {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    } else {
#pragma unroll
        for (int e = 0; e < PPT; ++e) p[e] = v[e];
    }
}

// Everything phase 1 needs about one ensemble (one case of a batch).
template <typename R>
struct P1Target {
    R *khat;
    int64_t N, ld;
    uint32_t *Hnext;          // f^{n+1} [Q][Nk*Nk]
    uint32_t *qcount;         // collider counter of this step
    uint32_t *queue;          // collider queue
    uint32_t qoffset;         // added to the particle index in queue entries
    uint32_t key0, key1, stream_id, step;
    const uint32_t *skip = nullptr;  // optional: particles left to a concurrent phase 2 (not touched here)
    uint32_t *mark = nullptr;        // optional: bitmap of the particles queued here
};

// One pass of a block over blockDim * PPT consecutive particles starting at i0 + threadIdx*PPT:
// drift, reconstruction, flight-time screen, histogram (window or global), queue, moments.
// (PPT particles per thread; i0 a multiple of PPT.)
template <int P, int Q, typename R, int PPT = Phase1PPT<P>::value>
__device__ __forceinline__ void phase1_pass(const Phys<R> &ph, const Nodes<P, Q, R> &nd, const P1Target<R> &t,
                                            int64_t i0, uint32_t *swin, int win_r0, bool use_win, bool out_step,
                                            typename MomAcc<R>::T *smom_warp, unsigned int &oog)
{
    const int lane = threadIdx.x & 31;
    const int64_t NN = (int64_t)ph.Nk * ph.Nk;
    R cx[PPT][P], cy[PPT][P];
    bool finished[PPT];
    const bool any = i0 < t.N;
    // i0 is a multiple of PPT, so its PPT bits lie in one word
    const uint32_t skipbits = (t.skip && any) ? (t.skip[i0 >> 5] >> (i0 & 31)) & ((1u << PPT) - 1u) : 0u;
    if (any) {
#pragma unroll
        for (int h = 0; h < P; ++h) {
            R vx[PPT], vy[PPT];
            load_vec<R, PPT>(t.khat + (int64_t)h * t.ld + i0, vx);
            load_vec<R, PPT>(t.khat + (int64_t)(P + h) * t.ld + i0, vy);
#pragma unroll
            for (int e = 0; e < PPT; ++e) { cx[e][h] = vx[e]; cy[e][h] = vy[e]; }
        }
        // drift (Eq. (17) / sG forcing term); the padding beyond N is left untouched
#pragma unroll
        for (int h = 0; h < P; ++h)
            if (nd.drift_mask & (1u << h)) {
                R v[PPT];
#pragma unroll
                for (int e = 0; e < PPT; ++e) {
                    if (i0 + e < t.N) cx[e][h] -= nd.dhat[h];
                    v[e] = cx[e][h];
                }
                if (skipbits == 0u) {
                    store_vec<R, PPT>(t.khat + (int64_t)h * t.ld + i0, v);
                } else {
                    // a skipped particle is being written by phase 2: element-wise stores
#pragma unroll
                    for (int e = 0; e < PPT; ++e)
                        if (!((skipbits >> e) & 1u) && i0 + e < t.N) t.khat[(int64_t)h * t.ld + i0 + e] = v[e];
                }
            }
    }
    constexpr bool kUnrollQ = P * Q <= 64 || TensorShape<P, Q>::value;
#pragma unroll
    for (int e = 0; e < PPT; ++e) {
        const int64_t i = i0 + e;
        finished[e] = false;
        bool maybe = false;
        if (any && i < t.N && !((skipbits >> e) & 1u)) {
            // reconstruction, cells and the bound on the majorant
            int rl[Q];   // cell (row << 16) | column; -1 outside the grid
            R kkmax = (R)0;
            recon_all(nd, cx[e], cy[e], [&](int q, R kx, R ky) {
                int r, l;
                rl[q] = cell_rl(ph, nd.lkx[q], kx, ky, r, l) ? ((r << 16) | l) : -1;
                kkmax = fmax(kkmax, knorm2(kx, ky));
            });
            const U4 r = philox4x32_10((uint32_t)i, t.stream_id, t.step, 0u, t.key0, t.key1);
            maybe = screen_maybe(ph, nd, kkmax, r.x);
            if (!maybe) {
                finished[e] = true;
#pragma unroll (kUnrollQ ? Q : 1)
                for (int q = 0; q < Q; ++q) {
                    if (rl[q] < 0) { ++oog; continue; }
                    const int r = rl[q] >> 16, l = rl[q] & 0xffff;
                    const int rr = r - win_r0, ll = l - win_r0;
                    if (use_win && (unsigned)rr < (unsigned)kWin && (unsigned)ll < (unsigned)kWin)
                        atomicAdd(&swin[q * kWinWords + rr * (kWin / 2) + (ll >> 1)], 1u << ((ll & 1) << 4));
                    else
                        atomicAdd(&t.Hnext[(int64_t)q * NN + r * ph.Nk + l], 1u);
                }
            }
        }
        // colliders go to the queue (warp-aggregated append)
        const unsigned int mask = __ballot_sync(0xffffffffu, maybe);
        if (mask) {
            const int leader = __ffs(mask) - 1;
            uint32_t basepos = 0;
            if (lane == leader) basepos = atomicAdd(t.qcount, (uint32_t)__popc(mask));
            basepos = __shfl_sync(0xffffffffu, basepos, leader);
            if (maybe) {
                t.queue[basepos + __popc(mask & ((1u << lane) - 1u))] = t.qoffset + (uint32_t)i;
                if (t.mark) atomicOr(&t.mark[i >> 5], 1u << (i & 31));
            }
        }
    }
    if (out_step) {
        if constexpr (TensorShape<P, Q>::value && sizeof(R) == 4 && PPT == 1) {
            // one particle per thread: the node values again by the (unrolled) sum factorisation,
            // their observables streamed 16 at a time into warp reduce-scatters (node q,
            // quantity j is value 3 q + j)
            float buf[16];
            const bool fin = finished[0];
            recon_all(nd, cx[0], cy[0], [&](int q, R kx, R ky) {
                float o[3] = {0.0f, 0.0f, 0.0f};
                if (fin) observe_fast(ph, kx - nd.xs[q], ky, nd.eps0[q], o[0], o[1], o[2]);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int idx = 3 * q + j;
                    buf[idx & 15] = o[j];
                    if ((idx & 15) == 15 || idx == 3 * Q - 1) {
                        for (int z = (idx & 15) + 1; z < 16; ++z) buf[z] = 0.0f;
                        warp_scatter16_add(buf, smom_warp + (idx & ~15), (idx & 15) + 1, lane);
                    }
                }
            });
        } else if constexpr (sizeof(R) == 4) {
            // per node: the three observables summed over the thread's particles, then one 4-value
            // warp reduce-scatter (6 shuffles instead of the 15 of three butterflies)
#pragma unroll 1
            for (int q = 0; q < Q; ++q) {
                float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int e = 0; e < PPT; ++e)
                    if (finished[e]) {
                        float kx, ky, a1, a2, a3;
                        recon_node(nd, q, cx[e], cy[e], kx, ky);
                        observe(ph, kx - nd.xs[q], ky, nd.eps0[q], a1, a2, a3);
                        s[0] += a1; s[1] += a2; s[2] += a3;
                    }
                warp_scatter4_add(s, smom_warp + q * 3, 3, lane);
            }
        } else {
#pragma unroll 1
            for (int q = 0; q < Q; ++q) {
                R vx = (R)0, vy = (R)0, en = (R)0;
#pragma unroll
                for (int e = 0; e < PPT; ++e)
                    if (finished[e]) {
                        R kx, ky, a1, a2, a3;
                        recon_node(nd, q, cx[e], cy[e], kx, ky);
                        observe(ph, kx - nd.xs[q], ky, nd.eps0[q], a1, a2, a3);
                        vx += a1; vy += a2; en += a3;
                    }
                vx = warp_sum(vx);
                vy = warp_sum(vy);
                en = warp_sum(en);
                if (lane == 0) {
                    acc_add(smom_warp[q * 3 + 0], vx);
                    acc_add(smom_warp[q * 3 + 1], vy);
                    acc_add(smom_warp[q * 3 + 2], en);
                }
            }
        }
    }
}

// Add a block's shared-memory window to the global histogram: one add per non-empty cell.
template <int Q>
__device__ __forceinline__ void flush_window(const uint32_t *swin, uint32_t *Hnext, int Nk, int win_r0)
{
    const int64_t NN = (int64_t)Nk * Nk;
    for (int j = threadIdx.x; j < Q * kWinWords; j += blockDim.x) {
        const uint32_t v = swin[j];
        if (!v) continue;
        const int q = j / kWinWords, w = j % kWinWords;
        const int rr = w / (kWin / 2) + win_r0, ll = 2 * (w % (kWin / 2)) + win_r0;
        uint32_t *base = Hnext + (int64_t)q * NN + (int64_t)rr * Nk + ll;
        if (v & 0xffffu) atomicAdd(base, v & 0xffffu);
        if (v >> 16) atomicAdd(base + 1, v >> 16);
    }
}

// Phase 1 of one block, block bid of the nb blocks doing phase 1.  Tiles of blockDim * PPT
// particles: taken from the step's tile counter when there is one (blocks that start late take
// fewer), else every nb-th tile.  swin: dynamic shared memory of the histogram window.
template <int P, int Q, typename R>
__device__ __forceinline__ void phase1_block(const StepArgs<P, Q, R> &a, int bid, int nb, uint32_t *swin)
{
    constexpr int PPT = Phase1PPT<P>::value;
    constexpr int NW = kPhase1Threads / 32;
    __shared__ typename MomAcc<R>::T smom[NW][Q * 3];
    __shared__ uint32_t s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (a.use_win)
        for (int j = threadIdx.x; j < Q * kWinWords; j += blockDim.x) swin[j] = 0u;
    if (a.out_step)
        for (int j = lane; j < Q * 3; j += 32) acc_zero(smom[warp][j]);
    __syncthreads();

    // housekeeping for the next steps
    if (bid == 0 && threadIdx.x == 0) {
        *a.qcount_next = 0u;
        if (a.tilectr_next) *a.tilectr_next = 0u;
    }
    {
        uint4 *hc = reinterpret_cast<uint4 *>(a.Hclear);
        const int64_t n4 = a.hist_elems >> 2;
        for (int64_t j = (int64_t)bid * blockDim.x + threadIdx.x; j < n4; j += (int64_t)nb * blockDim.x)
            hc[j] = make_uint4(0u, 0u, 0u, 0u);
        if (bid == 0)
            for (int64_t j = (n4 << 2) + threadIdx.x; j < a.hist_elems; j += blockDim.x) a.Hclear[j] = 0u;
        if (a.mark_clear) {
            uint4 *mc = reinterpret_cast<uint4 *>(a.mark_clear);
            for (int64_t j = (int64_t)bid * blockDim.x + threadIdx.x; j < (a.mark_words >> 2); j += (int64_t)nb * blockDim.x)
                mc[j] = make_uint4(0u, 0u, 0u, 0u);
        }
    }

    P1Target<R> t;
    t.khat = a.khat; t.N = a.N; t.ld = a.ld; t.Hnext = a.Hnext; t.qcount = a.qcount; t.queue = a.queue;
    t.qoffset = 0u; t.key0 = a.key0; t.key1 = a.key1; t.stream_id = a.stream_id; t.step = a.step;
    t.skip = a.skip; t.mark = a.mark;
    unsigned int oog = 0u;
    const int64_t tile = (int64_t)blockDim.x * PPT;
    // A window cell holds 16 bits and a particle adds at most one count to a cell per node, so the
    // window is flushed to f^{n+1} before the block has counted 65535 particles since the last
    // flush (block-uniform; with the tile counter a block may take any number of tiles).
    int64_t since_flush = 0;
    auto guard_window = [&]() {
        if (a.use_win && since_flush + tile > 65535) {
            __syncthreads();
            flush_window<Q>(swin, a.Hnext, a.ph.Nk, a.win_r0);
            __syncthreads();
            for (int j = threadIdx.x; j < Q * kWinWords; j += blockDim.x) swin[j] = 0u;
            __syncthreads();
            since_flush = 0;
        }
        since_flush += tile;
    };
    if (a.tilectr) {
        const int64_t ntiles = (a.N + tile - 1) / tile;
        for (;;) {
            if (threadIdx.x == 0) s_tile = atomicAdd(a.tilectr, 1u);
            __syncthreads();
            const int64_t tl = s_tile;
            __syncthreads();   // every thread has read s_tile before it is overwritten
            if (tl >= ntiles) break;
            guard_window();
            phase1_pass<P, Q, R>(a.ph, a.nd, t, tl * tile + (int64_t)threadIdx.x * PPT, swin, a.win_r0,
                                 a.use_win != 0, a.out_step != 0, smom[warp], oog);
        }
    } else {
        for (int64_t base = (int64_t)bid * tile; base < a.N; base += (int64_t)nb * tile) {
            guard_window();
            phase1_pass<P, Q, R>(a.ph, a.nd, t, base + (int64_t)threadIdx.x * PPT, swin, a.win_r0, a.use_win != 0,
                                 a.out_step != 0, smom[warp], oog);
        }
    }
    oog = warp_sum(oog);
    if (lane == 0 && oog) atomicAdd(&a.counters[4], (unsigned long long)oog);
    __syncthreads();
    if (a.use_win) flush_window<Q>(swin, a.Hnext, a.ph.Nk, a.win_r0);
    if (a.out_step) {
        for (int j = threadIdx.x; j < Q * 3; j += blockDim.x) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w) s += acc_value(smom[w][j]);
            a.part1[(int64_t)bid * (Q * 3) + j] = s;
        }
    }
}

template <int P, int Q, typename R>
__global__ void __launch_bounds__(kPhase1Threads, kPhase1MinBlocks<P, Q, R>::value)
k_phase1(const __grid_constant__ StepArgs<P, Q, R> a)
{
    extern __shared__ uint32_t swin[];   // [Q][kWinWords] when a.use_win
    phase1_block<P, Q, R>(a, blockIdx.x, gridDim.x, swin);
}

// ------------------------------------------------------------------------------------------
// Phase 2: the collision loop of Algorithm 1 / 2 for the queued particles.  A group of G
// lanes carries one particle, lane r owning the nodes q = r, r + G, ... (lanes <-> quadrature
// nodes): the rates, the mechanism selection, the final states and the Pauli look-ups of the Q
// nodes run in parallel, and the projection of Eqs. (28)-(30) and the majorant of Eq. (25) are
// group reductions by shuffles.
// ------------------------------------------------------------------------------------------
#ifndef PGC_GROUP36
#define PGC_GROUP36 32
#endif
#ifndef PGC_GROUP8
#define PGC_GROUP8 8
#endif

template <int Q> struct GroupOf {
    static constexpr int G = (Q == 36) ? PGC_GROUP36
                           : (Q >= 32) ? 32 : (Q > 16 ? 32 : (Q > 8 ? 16 : (Q > 4 ? PGC_GROUP8 : (Q > 2 ? 4 : (Q > 1 ? 2 : 1)))));
    static constexpr int NPL = (Q + G - 1) / G;  // nodes per lane
};

// Node slots of a lane (s = 0 .. NPL - 1) read and written with a runtime slot index by selects,
// so that a rolled loop over the slots keeps the per-slot arrays in registers: the per-node code
// of the collision loop is emitted once instead of NPL times (instruction-cache footprint).
template <int N, typename T>
__device__ __forceinline__ T slot_get(const T (&a)[N], int s)
{
    T v = a[0];
#pragma unroll
    for (int k = 1; k < N; ++k)
        if (s == k) v = a[k];
    return v;
}
template <int N, typename T>
__device__ __forceinline__ void slot_set(T (&a)[N], int s, T v)
{
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (s == k) a[k] = v;
}

template <int G, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
}

template <int G, typename T>
__device__ __forceinline__ T group_max(T v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(mask, v, o, G));
    return v;
}

template <int G>
__device__ __forceinline__ bool group_any(bool b, unsigned mask)
{
    return (__ballot_sync(mask, b) & mask) != 0u;
}

// Shared-memory transpose reduction of the projection for groups of a whole warp: per warp, 32
// rows of 2P partial sums (row stride 2P + 1, odd, so that the column reads are conflict-free)
// and the 2P totals.
template <int P, int Q, typename R> struct ProjRed {   // (its area fits the static shared memory up to P = 21)
    static constexpr bool value = GroupOf<Q>::G == 32 && sizeof(R) == 4 && P <= 21;
    static constexpr int stride = 2 * P + 1;
    static constexpr int warp_elems = 32 * stride + 2 * P;
};

// Projection of the node values onto the basis (the collisional matrices K1 + K2 of Eqs.
// (28)-(30)): cx_h = sum_q w_q Psi_h(z_q) kx_q, summed over the G lanes of the group (lane r holds
// nodes r, r + G, ...); every lane receives all 2P coefficients.  FP32 whole-warp groups: each
// lane writes its 2P partial sums to shared memory (red: this block's ProjRed area, one per warp),
// lane j adds column j over the 32 lanes in a fixed order, and every lane reads the 2P totals back
// (~2P shared stores and loads per lane instead of 2P five-level shuffle butterflies).  Otherwise
// butterfly shuffles.
template <int P, int Q, typename R>
__device__ __forceinline__ void project_group(const Nodes<P, Q, R> &nd, const R kx[GroupOf<Q>::NPL],
                                              const R ky[GroupOf<Q>::NPL], int r, unsigned gmask, R cx[P], R cy[P],
                                              R *red)
{
    constexpr int G = GroupOf<Q>::G, NPL = GroupOf<Q>::NPL;
    constexpr int S = ProjRed<P, Q, R>::stride;
    R *w = red + (threadIdx.x >> 5) * ProjRed<P, Q, R>::warp_elems;   // used by ProjRed shapes only
#pragma unroll (P * Q <= 64 ? P : 1)
    for (int h = 0; h < P; ++h) {
        R sx = (R)0, sy = (R)0;
        if constexpr (sizeof(R) == 4 && !TensorShape<P, Q>::value) {
            F2 s2 = f2_pack(0.f, 0.f);
#pragma unroll
            for (int s = 0; s < NPL; ++s) {
                const int q = r + s * G;
                if (q < Q) s2 = f2_fma(f2_pack(kx[s], ky[s]), nd.wpsi2[q * P + h], s2);
            }
            f2_unpack(s2, sx, sy);
        } else {
#pragma unroll
            for (int s = 0; s < NPL; ++s) {
                const int q = r + s * G;
                if (q < Q) {
                    sx += nd.wpsi[q * P + h] * kx[s];
                    sy += nd.wpsi[q * P + h] * ky[s];
                }
            }
        }
        if constexpr (ProjRed<P, Q, R>::value) {
            w[r * S + h] = sx;
            w[r * S + P + h] = sy;
        } else {
            cx[h] = group_sum<G>(sx, gmask);
            cy[h] = group_sum<G>(sy, gmask);
        }
    }
    if constexpr (ProjRed<P, Q, R>::value) {
        R *tot = w + 32 * S;
        __syncwarp(gmask);
        for (int v = r; v < 2 * P; v += 32) {
            R acc = (R)0;
#pragma unroll 8
            for (int l = 0; l < 32; ++l) acc += w[l * S + v];
            tot[v] = acc;
        }
        __syncwarp(gmask);
#pragma unroll
        for (int h = 0; h < P; ++h) {
            cx[h] = tot[h];
            cy[h] = tot[P + h];
        }
        __syncwarp(gmask);   // all lanes have read the totals before the next projection writes
    }
}

// Everything the collision loop of one particle needs about its ensemble.
template <typename R>
struct P2Target {
    R *khat;
    int64_t ld;
    const uint32_t *Hcur;     // f^n
    uint32_t *Hnext;          // f^{n+1}
    const uint32_t *nmax;
    double *mom;              // [Q*3] moment accumulators (shared or global), on moment steps
    uint32_t key0, key1, stream_id, step;
    bool out_step;
    // continuation into step n + 1 (EXT)
    uint32_t *Hnext2 = nullptr;      // f^{n+2}
    uint32_t *queue_next = nullptr, *qcount_next = nullptr, *mark_next = nullptr;
    double *momN = nullptr;          // [Q*3] moments of step n + 1
    bool out_next = false;
    R *red = nullptr;                // shared-memory area of project_group (ProjRed shapes)
};

struct P2Counts { unsigned long long att = 0, chg = 0, rej = 0, cap = 0, oog = 0; };

// The collision loop of Algorithm 1 / 2 for particle i, carried by the G lanes of a group (lane r
// owns nodes r, r + G, ...), then the histogram f^{n+1} and moments of its final state.  With
// EXT, the particle then goes through step n + 1 as far as phase 1 would take it: drift,
// reconstruction, flight-time screen, and either the histogram f^{n+2} and moments of step n + 1
// or a place in the collider queue of step n + 1.
template <int P, int Q, typename R, bool EXT = false>
__device__ __forceinline__ void collide_particle(const Phys<R> &ph, const Nodes<P, Q, R> &nd, const P2Target<R> &t,
                                                 int64_t i, int r, unsigned gmask, P2Counts &cnt)
{
    constexpr int G = GroupOf<Q>::G, NPL = GroupOf<Q>::NPL;
    const int64_t NN = (int64_t)ph.Nk * ph.Nk;
    R cx[P], cy[P], kx[NPL], ky[NPL];
#pragma unroll
    for (int h = 0; h < P; ++h) {
        cx[h] = t.khat[(int64_t)h * t.ld + i];
        cy[h] = t.khat[(int64_t)(P + h) * t.ld + i];
    }
    // the node values of the lane's slots from the coefficients
    // (NPL > 1: loops over the slots are rolled, see slot_get)
    auto recon_slots = [&](const R (&ccx)[P], const R (&ccy)[P], R (&x)[NPL], R (&y)[NPL]) {
        if constexpr (NPL > 1) {
#pragma unroll 1
            for (int s = 0; s < NPL; ++s) {
                const int q = r + s * G;
                if (q >= Q) break;
                R a, b;
                recon_node(nd, q, ccx, ccy, a, b);
                slot_set(x, s, a);
                slot_set(y, s, b);
            }
        } else {
            recon_node(nd, r, ccx, ccy, x[0], y[0]);
        }
    };
    recon_slots(cx, cy, kx, ky);
    R gc[NPL][6];  // rates of the current state at the lane's nodes (reused by the selection)
    R tc = (R)0, Gt = (R)0;
    uint32_t c = 0;
    bool touched = false, fresh = true;
    // One pass per free flight: majorant of the current state (Eq. (25)), flight time, and, if
    // the flight ends inside the step, a collision.  The rates and the random draw have one
    // call site each (instruction-cache footprint).  An event that changes no node (self
    // scattering or Pauli rejection everywhere) leaves the state, its rates and the majorant
    // as they were: the projection of unchanged node values returns the same coefficients, so
    // it, the reconstruction and the rates are not redone (fresh = false).
    for (;;) {
        if (fresh) {
            R gm = (R)0;
            if constexpr (NPL > 1) {
#pragma unroll 1
                for (int s = 0; s < NPL; ++s) {
                    const int q = r + s * G;
                    if (q >= Q) break;
                    R g[6];
                    gm = fmax(gm, rates6(ph, slot_get(kx, s), slot_get(ky, s), nd.eps0[q], g));
#pragma unroll
                    for (int m = 0; m < 6; ++m)
#pragma unroll
                        for (int k = 0; k < NPL; ++k)
                            if (s == k) gc[k][m] = g[m];
                }
            } else {
#pragma unroll
                for (int s = 0; s < NPL; ++s) {
                    const int q = r + s * G;
                    if (q < Q) gm = fmax(gm, rates6(ph, kx[s], ky[s], nd.eps0[q], gc[s]));
                }
            }
            Gt = ph.alpha1 * group_max<G>(gm, gmask);
        }
        const U4 rr = philox4x32_10((uint32_t)i, t.stream_id, t.step, c, t.key0, t.key1);
        const R dtc = (Gt > (R)0) ? -rlog<R>(u01<R>(rr.x)) / Gt : (R)INFINITY;
        if (!(tc + dtc < ph.dt)) break;             // group-uniform condition
        if ((int)c >= ph.max_coll) { if (r == 0) ++cnt.cap; break; }
        if (r == 0) ++cnt.att;
        EventAngles<R> ang;
        ang.reset(u01<R>(rr.w));
        const R target = u01<R>(rr.y) * Gt;
        bool changed = false;
        if constexpr (NPL > 1) {
#pragma unroll 1
            for (int s = 0; s < NPL; ++s) {
                const int q = r + s * G;
                if (q >= Q) break;
                int l = 6;
                R cum = (R)0;
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    R gsm = gc[0][m];
#pragma unroll
                    for (int k = 1; k < NPL; ++k)
                        if (s == k) gsm = gc[k][m];
                    cum += gsm;
                    if (l == 6 && target < cum) l = m;
                }
                if (l == 6) continue;  // self scattering: h^7 = identity
                R nkx, nky;
                final_state(ph, l, slot_get(kx, s), slot_get(ky, s), nd.eps0[q], ang, &nkx, &nky);
                bool accept = true;
                if (ph.pauli_mode != 2) {
                    const int cl = cell_of(ph, nd.lkx[q], nkx + nd.dq[q], nky);
                    if (cl >= 0) accept = pauli_accept(t.Hcur[(int64_t)q * NN + cl], t.nmax[q], rr.z);
                }
                if (accept) {
                    slot_set(kx, s, nkx);
                    slot_set(ky, s, nky);
                    changed = true;
                } else {
                    ++cnt.rej;
                }
            }
        } else {
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
            const int q = r + s * G;
            if (q >= Q) continue;
            int l = 6;
            R cum = (R)0;
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                cum += gc[s][m];
                if (l == 6 && target < cum) l = m;
            }
            if (l == 6) continue;  // self scattering: h^7 = identity
            R nkx, nky;
            final_state(ph, l, kx[s], ky[s], nd.eps0[q], ang, &nkx, &nky);
            bool accept = true;
            if (ph.pauli_mode != 2) {
                const int cl = cell_of(ph, nd.lkx[q], nkx + nd.dq[q], nky);
                if (cl >= 0) accept = pauli_accept(t.Hcur[(int64_t)q * NN + cl], t.nmax[q], rr.z);
            }
            if (accept) { kx[s] = nkx; ky[s] = nky; changed = true; }
            else ++cnt.rej;
        }
        }
        fresh = group_any<G>(changed, gmask);
        if (fresh && r == 0) ++cnt.chg;
        if (fresh) {
            touched = true;
            // collisional matrices K1 + K2 (Eqs. (28)-(30)): project the node values
            project_group<P, Q, R>(nd, kx, ky, r, gmask, cx, cy, t.red);
            recon_slots(cx, cy, kx, ky);
        }
        tc += dtc;
        ++c;
    }
    if constexpr (EXT) {
        // drift of step n + 1 (before the store: the stored state is the post-drift one, as phase 1 leaves it)
#pragma unroll
        for (int h = 0; h < P; ++h)
            if (nd.drift_mask & (1u << h)) cx[h] -= nd.dhat[h];
    }
    if (touched || (EXT && nd.drift_mask != 0u)) {
        // lane h of the group writes coefficient h (x and y planes)
        for (int h = r; h < P; h += G) {
            R vx = cx[0], vy = cy[0];
#pragma unroll
            for (int hh = 0; hh < P; ++hh) if (hh == h) { vx = cx[hh]; vy = cy[hh]; }
            t.khat[(int64_t)h * t.ld + i] = vx;
            t.khat[(int64_t)(P + h) * t.ld + i] = vy;
        }
    }
    auto finish_node = [&](int q, R x, R y) {
        const int cl = cell_of(ph, nd.lkx[q], x, y);
        if (cl >= 0) atomicAdd(&t.Hnext[(int64_t)q * NN + cl], 1u);
        else ++cnt.oog;
        if (t.out_step) {
            R vx, vy, e;
            observe(ph, x - nd.xs[q], y, nd.eps0[q], vx, vy, e);
            atomicAdd(&t.mom[q * 3 + 0], (double)vx);
            atomicAdd(&t.mom[q * 3 + 1], (double)vy);
            atomicAdd(&t.mom[q * 3 + 2], (double)e);
        }
    };
    if constexpr (NPL > 1) {
#pragma unroll 1
        for (int s = 0; s < NPL; ++s) {
            const int q = r + s * G;
            if (q >= Q) break;
            finish_node(q, slot_get(kx, s), slot_get(ky, s));
        }
    } else {
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
            const int q = r + s * G;
            if (q < Q) finish_node(q, kx[s], ky[s]);
        }
    }
    if constexpr (EXT) {
        // step n + 1 up to the flight-time screen, with the operations of phase 1
        int cl2[NPL];
        R kk = (R)0;
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
            const int q = r + s * G;
            cl2[s] = -1;
            if (q < Q) {
                R x, y;
                recon_at(nd, q, cx, cy, x, y);
                cl2[s] = cell_of(ph, nd.lkx[q], x, y);
                kk = fmax(kk, knorm2(x, y));
            }
        }
        const R kkmax = group_max<G>(kk, gmask);
        const U4 r1 = philox4x32_10((uint32_t)i, t.stream_id, t.step + 1u, 0u, t.key0, t.key1);
        if (!screen_maybe(ph, nd, kkmax, r1.x)) {
#pragma unroll
            for (int s = 0; s < NPL; ++s) {
                const int q = r + s * G;
                if (q >= Q) continue;
                if (cl2[s] >= 0) atomicAdd(&t.Hnext2[(int64_t)q * NN + cl2[s]], 1u);
                else ++cnt.oog;
                if (t.out_next) {
                    R x, y, vx, vy, e;
                    recon_node(nd, q, cx, cy, x, y);
                    observe(ph, x - nd.xs[q], y, nd.eps0[q], vx, vy, e);
                    atomicAdd(&t.momN[q * 3 + 0], (double)vx);
                    atomicAdd(&t.momN[q * 3 + 1], (double)vy);
                    atomicAdd(&t.momN[q * 3 + 2], (double)e);
                }
            }
        } else if (r == 0) {
            const uint32_t pos = atomicAdd(t.qcount_next, 1u);
            t.queue_next[pos] = (uint32_t)i;
            atomicOr(&t.mark_next[i >> 5], 1u << (i & 31));
        }
    }
}

// Copy a trivially-copyable table into shared memory (all threads; caller synchronises).
template <typename T>
__device__ __forceinline__ void stage(uint32_t *dst, const T &src)
{
    const uint32_t *s = reinterpret_cast<const uint32_t *>(&src);
    for (int j = threadIdx.x; j < (int)(sizeof(T) / 4); j += blockDim.x) dst[j] = s[j];
}

// Phase 2 of one block, block bid of the nb blocks doing phase 2 (any block size that is a
// multiple of the group size).
template <int P, int Q, typename R, bool EXT>
__device__ __forceinline__ void phase2_block(const StepArgs<P, Q, R> &a, int bid, int nb, R *red)
{
    constexpr int G = GroupOf<Q>::G;
    __shared__ double smom[Q * 3];
    __shared__ double smomN[EXT ? Q * 3 : 1];
    __shared__ unsigned long long scnt[5];
    // The lanes of a group read different nodes' entries of the node tables: staged in shared
    // memory from their device copy (divergent reads of the parameter bank serialise).  The
    // physics constants are read by all lanes alike and stay in the parameter bank.
    __shared__ __align__(16) uint32_t snd[(sizeof(Nodes<P, Q, R>) + 3) / 4];
    if (threadIdx.x < 5) scnt[threadIdx.x] = 0ull;
    for (int j = threadIdx.x; j < Q * 3; j += blockDim.x) smom[j] = 0.0;
    if constexpr (EXT)
        for (int j = threadIdx.x; j < Q * 3; j += blockDim.x) smomN[j] = 0.0;
    if (a.nd_dev) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(a.nd_dev);
        for (int j = threadIdx.x; j < (int)(sizeof(Nodes<P, Q, R>) / 4); j += blockDim.x) snd[j] = src[j];
    } else {
        stage(snd, a.nd);
    }
    __syncthreads();

    const Phys<R> &ph = a.ph;
    const Nodes<P, Q, R> &nd = *reinterpret_cast<const Nodes<P, Q, R> *>(snd);
    const uint32_t count = *a.qcount;
    P2Counts cnt;
    P2Target<R> t;
    t.khat = a.khat; t.ld = a.ld; t.Hcur = a.Hcur; t.Hnext = a.Hnext; t.nmax = a.nmax; t.mom = smom;
    t.key0 = a.key0; t.key1 = a.key1; t.stream_id = a.stream_id; t.step = a.step; t.out_step = a.out_step != 0;
    t.red = red;
    if constexpr (EXT) {
        t.Hnext2 = a.Hnext2; t.queue_next = a.queue_next; t.qcount_next = a.qcount_next; t.mark_next = a.mark_next;
        t.momN = smomN; t.out_next = a.out_next != 0;
    }

    const int lane = threadIdx.x & 31;
    const int r = lane % G;                                  // lane in the group
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane - r));
    const uint32_t gid = ((uint32_t)bid * blockDim.x + threadIdx.x) / G;
    const uint32_t ngroups = (uint32_t)nb * blockDim.x / G;
    for (uint32_t j = gid; j < count; j += ngroups) collide_particle<P, Q, R, EXT>(ph, nd, t, a.queue[j], r, gmask, cnt);

    if (cnt.att) atomicAdd(&scnt[0], cnt.att);
    if (cnt.chg) atomicAdd(&scnt[1], cnt.chg);
    if (cnt.rej) atomicAdd(&scnt[2], cnt.rej);
    if (cnt.cap) atomicAdd(&scnt[3], cnt.cap);
    if (cnt.oog) atomicAdd(&scnt[4], cnt.oog);
    __syncthreads();
    if (threadIdx.x < 5 && scnt[threadIdx.x]) atomicAdd(&a.counters[threadIdx.x], scnt[threadIdx.x]);
    if (threadIdx.x == 0 && bid == 0) atomicAdd(&a.counters[5], (unsigned long long)count);
    if (a.out_step)
        for (int j = threadIdx.x; j < Q * 3; j += blockDim.x) a.part2[(int64_t)bid * (Q * 3) + j] = smom[j];
    if constexpr (EXT)
        if (a.out_next)
            for (int j = threadIdx.x; j < Q * 3; j += blockDim.x) a.partN[(int64_t)bid * (Q * 3) + j] = smomN[j];
}

template <int P, int Q, typename R, bool EXT>
__global__ void __launch_bounds__(kPhase2Threads, Phase2Blocks<P, Q>::per_sm)
k_phase2(const __grid_constant__ StepArgs<P, Q, R> a)
{
    __shared__ R sred[ProjRed<P, Q, R>::value ? (kPhase2Threads / 32) * ProjRed<P, Q, R>::warp_elems : 1];
    phase2_block<P, Q, R, EXT>(a, blockIdx.x, gridDim.x, sred);
}

// One launch per time step in the pipelined form: blocks [0, nb2) run phase 2 of step n - 1 with
// the continuation into step n (a2), the others phase 1 of step n (a1, tiles from the tile
// counter, skipping the particles queued at step n - 1).  The two roles touch disjoint particles;
// shared buffers are only added to (histograms, queue of step n, bitmap of step n).
template <int P, int Q, typename R>
__global__ void __launch_bounds__(kPhase1Threads, kPhase1MinBlocks<P, Q, R>::value)
k_step(const __grid_constant__ StepArgs<P, Q, R> a1, const __grid_constant__ StepArgs<P, Q, R> a2, int nb2)
{
    extern __shared__ uint32_t swin[];   // phase 1: histogram window; phase 2: projection area
    if ((int)blockIdx.x < nb2) phase2_block<P, Q, R, true>(a2, blockIdx.x, nb2, reinterpret_cast<R *>(swin));
    else phase1_block<P, Q, R>(a1, blockIdx.x - nb2, gridDim.x - nb2, swin);
}

// ------------------------------------------------------------------------------------------
// Observation of a whole state: histogram into H and (optionally) moment partials into part1.
// Used after the initial sampling and after a state upload.
// ------------------------------------------------------------------------------------------
template <int P, int Q, typename R>
__global__ void __launch_bounds__(kPhase1Threads)
k_observe(const __grid_constant__ StepArgs<P, Q, R> a)
{
    constexpr int NW = kPhase1Threads / 32;
    __shared__ double smom[NW][Q * 3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = lane; j < Q * 3; j += 32) smom[warp][j] = 0.0;
    const Phys<R> &ph = a.ph;
    const Nodes<P, Q, R> &nd = a.nd;
    const int64_t NN = (int64_t)ph.Nk * ph.Nk;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.N; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < a.N;
        R cx[P], cy[P];
        if (valid) load_coeffs(a, i, cx, cy);
#pragma unroll 1
        for (int q = 0; q < Q; ++q) {
            R vx = (R)0, vy = (R)0, e = (R)0;
            if (valid) {
                R kx, ky;
                recon_node(nd, q, cx, cy, kx, ky);
                const int cl = cell_of(ph, nd.lkx[q], kx, ky);
                if (cl >= 0) atomicAdd(&a.Hnext[(int64_t)q * NN + cl], 1u);
                observe(ph, kx - nd.xs[q], ky, nd.eps0[q], vx, vy, e);
            }
            vx = warp_sum(vx);
            vy = warp_sum(vy);
            e = warp_sum(e);
            if (lane == 0) {
                smom[warp][q * 3 + 0] += (double)vx;
                smom[warp][q * 3 + 1] += (double)vy;
                smom[warp][q * 3 + 2] += (double)e;
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < Q * 3; j += blockDim.x) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += smom[w][j];
        a.part1[(int64_t)blockIdx.x * (Q * 3) + j] = s;
    }
}

// ------------------------------------------------------------------------------------------
// Initial state: Fermi-Dirac sampling at every node with shared uniforms, projection (FP64).
// ------------------------------------------------------------------------------------------
template <int P, int Q>
struct InitArgs {
    double wpsi[Q * P];
    double eps0[Q];
    double mu, kT, hvF;
    double dhalf[P];   // Strang: the stored state leads by half a drift (x coefficients)
    int32_t strang;
    int64_t N, ld;
    uint32_t key0, key1, stream_id;
};

template <int P, int Q, typename R>
__global__ void __launch_bounds__(128)
k_init(const __grid_constant__ InitArgs<P, Q> ia, R *khat)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ia.N; i += (int64_t)gridDim.x * blockDim.x) {
        const U4 r = philox4x32_10((uint32_t)i, ia.stream_id, 0u, 0x10000u, ia.key0, ia.key1);
        const double ue = u01<double>(r.x), uth = u01<double>(r.y);
        double s, c;
        sincos(2.0 * kPi * uth, &s, &c);
        double hx[P], hy[P];
#pragma unroll
        for (int h = 0; h < P; ++h) { hx[h] = 0.0; hy[h] = 0.0; }
#pragma unroll 1
        for (int q = 0; q < Q; ++q) {
            const double e0 = ia.eps0[q];
            const double eps = fd_inverse(e0, ia.mu, ia.kT, ue);
            const double rr = eps * eps - e0 * e0;
            const double km = (rr > 0.0) ? sqrt(rr) / ia.hvF : 0.0;
            const double kx = km * c, ky = km * s;
#pragma unroll
            for (int h = 0; h < P; ++h) {
                hx[h] += ia.wpsi[q * P + h] * kx;
                hy[h] += ia.wpsi[q * P + h] * ky;
            }
        }
#pragma unroll
        for (int h = 0; h < P; ++h) {
            khat[(int64_t)h * ia.ld + i] = (R)(ia.strang ? hx[h] + ia.dhalf[h] : hx[h]);
            khat[(int64_t)(P + h) * ia.ld + i] = (R)hy[h];
        }
    }
}

// Histogram of the particles reconstructed at one arbitrary z (Eq. (24)); psi given in FP64.
template <int P, int Q, typename R>
struct ReconArgs {
    double psi[P];
    R lkx;   // x offset of the grid at z (Lk, or Lk minus half the drift at z under Strang)
};

template <int P, int Q, typename R>
__global__ void __launch_bounds__(256)
k_hist_at(const __grid_constant__ StepArgs<P, Q, R> a, const __grid_constant__ ReconArgs<P, Q, R> z,
          uint32_t *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * blockDim.x) {
        R kx = (R)0, ky = (R)0;
#pragma unroll
        for (int h = 0; h < P; ++h) {
            kx += a.khat[(int64_t)h * a.ld + i] * (R)z.psi[h];
            ky += a.khat[(int64_t)(P + h) * a.ld + i] * (R)z.psi[h];
        }
        const int cl = cell_of(a.ph, z.lkx, kx, ky);
        if (cl >= 0) atomicAdd(&out[cl], 1u);
    }
}

// ------------------------------------------------------------------------------------------
// Observables at arbitrary points z (Eqs. (35)-(37) of the state reconstructed by Eq. (23) off
// the nodes).  Lane l of every warp evaluates point z_l; a block stages a tile of particles in
// shared memory as (x, y) coefficient pairs and each warp walks a share of the tile, every lane
// reading the same particle (broadcast).  Sums: in R over the particles of one tile, then FP64;
// block partials [kObsGrid][kObsZ][3] = (sum kx/eps, sum ky/eps, sum eps), reduced over the
// blocks in a fixed order by k_obs_fin.
// ------------------------------------------------------------------------------------------
constexpr int kObsZ = 32;        // points per pass over the state (one per lane)
constexpr int kObsGrid = 304;    // blocks of one pass (2 per SM)
constexpr int kObsThreads = 256;

template <int P, typename R>
struct ObsTile {   // particles per tile: the staged pairs take at most 32 KB
    static constexpr int value = (2 * P * (int)sizeof(R) * 256 <= 32768) ? 256
                               : (2 * P * (int)sizeof(R) * 128 <= 32768) ? 128 : 64;
};

template <int P, typename R>
struct ObsArgs {
    const R *khat;
    int64_t ld, N;
    R hvF2;
    R psi[kObsZ * P];   // basis at each point; zero rows for unused lanes
    R e0sq[kObsZ];      // eps0(z)^2; 1 for unused lanes
    R xs[kObsZ];        // x shift of the state at the point (Strang; else 0)
};

template <typename R> struct Pair;
template <> struct Pair<float> { using T = float2; };
template <> struct Pair<double> { using T = double2; };

template <int P, typename R>
__global__ void __launch_bounds__(kObsThreads)
k_obs_at(const __grid_constant__ ObsArgs<P, R> a, double *part)
{
    constexpr int T = ObsTile<P, R>::value;
    constexpr int kWarps = kObsThreads / 32;
    using R2 = typename Pair<R>::T;
    __shared__ R2 tile[P * T];
    __shared__ double red[kWarps][kObsZ * 3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    R ps[P];
#pragma unroll
    for (int h = 0; h < P; ++h) ps[h] = a.psi[lane * P + h];
    const R e0sq = a.e0sq[lane];
    const R xs = a.xs[lane];
    double ax = 0.0, ay = 0.0, ae = 0.0;
    const int64_t ntiles = (a.N + T - 1) / T;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t base = t * T;
        const int nv = (a.N - base < (int64_t)T) ? (int)(a.N - base) : T;
        __syncthreads();   // the previous tile is consumed
        for (int idx = threadIdx.x; idx < P * T; idx += kObsThreads) {
            const int h = idx / T, j = idx - h * T;
            R2 v;
            v.x = (j < nv) ? a.khat[(int64_t)h * a.ld + base + j] : (R)0;
            v.y = (j < nv) ? a.khat[(int64_t)(P + h) * a.ld + base + j] : (R)0;
            tile[h * T + j] = v;
        }
        __syncthreads();
        R sx = (R)0, sy = (R)0, se = (R)0;
        for (int j = warp; j < nv; j += kWarps) {   // uniform over the warp
            R kx, ky;
            if constexpr (sizeof(R) == 4) {
                F2 s = f2_pack(0.f, 0.f);
#pragma unroll
                for (int h = 0; h < P; ++h) {
                    const float2 c = tile[h * T + j];
                    F2 w;
                    asm("mov.b64 %0, {%1, %1};" : "=l"(w.v) : "f"(ps[h]));
                    s = f2_fma(f2_pack(c.x, c.y), w.v, s);
                }
                f2_unpack(s, kx, ky);
                kx -= xs;
            } else {
                kx = (R)0;
                ky = (R)0;
#pragma unroll
                for (int h = 0; h < P; ++h) {
                    const R2 c = tile[h * T + j];
                    kx += c.x * ps[h];
                    ky += c.y * ps[h];
                }
                kx -= xs;
            }
            const R eps = rsqrt_<R>(a.hvF2 * (kx * kx + ky * ky) + e0sq);
            const R ie = (R)1 / eps;
            sx += kx * ie;
            sy += ky * ie;
            se += eps;
        }
        ax += (double)sx;
        ay += (double)sy;
        ae += (double)se;
    }
    red[warp][lane * 3 + 0] = ax;
    red[warp][lane * 3 + 1] = ay;
    red[warp][lane * 3 + 2] = ae;
    __syncthreads();
    if (threadIdx.x < kObsZ * 3) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
        part[(int64_t)blockIdx.x * kObsZ * 3 + threadIdx.x] = s;
    }
}

}  // namespace pgc
