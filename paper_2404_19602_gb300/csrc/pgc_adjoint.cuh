// pgc_adjoint.cuh -- reverse-mode (adjoint) pathwise sensitivities of the time-averaged mean and
// variance over z of the current J_x with respect to theta = (E_lo, E_hi, eps0_lo, eps0_hi).
//
// Discrete events are frozen at those of the forward run: collision times, mechanisms, Pauli
// outcomes, the trapezoid segment of the edge angle and all histogram cells; the random numbers
// are the forward run's (Philox counters are recomputed, nothing is stored).  The forward run
// keeps a checkpoint (state + histogram f^n) every K steps; the backward pass replays each
// segment with the forward kernels, keeping the K states and histograms of the segment, then
// walks the segment backwards:
//   k_adj_screen  (every particle): adds the moment term of time n+1 to lambda, redoes the
//                 phase-1 flight-time screen of step n (same code, same decision), and for the
//                 particles that cannot have collided adds the drift term -d(dhat)/d(theta).lambda;
//                 the others are queued;
//   k_adj_collide (queued, lanes <-> nodes as in the forward collider kernel): replays the event
//                 chain of step n bit for bit, then applies the transposed Jacobians of the
//                 projection, the final-state maps h^l and the reconstruction, event by event from
//                 the last (each event's input state is recomputed by replaying from the start),
//                 and adds the drift term.
// After step 0, k_adj_init adds lambda^0 . d khat^0/d theta through the Fermi-Dirac sampling
// (implicit derivative of the inverse CDF).
#pragma once

#include <algorithm>
#include <cmath>

#include "pgc_runner_impl.cuh"

namespace pgc {

constexpr int NTH = 4;  // E_lo, E_hi, eps0_lo, eps0_hi

template <int P, int Q, typename R>
struct AdjArgs {
    Phys<R> ph;
    Nodes<P, Q, R> nd;
    const R *khat_n;          // state before step n (pre-drift), [2][P][ld]
    const R *khat_n1;         // state after step n (moment term of time n+1)
    R *lam;                   // adjoint of the state, [2][P][ld]
    const uint32_t *Hn;       // f^n
    const uint32_t *nmax;
    uint32_t *queue, *qcount;
    double *grad;             // [NTH], accumulated
    int64_t N, ld;
    uint32_t key0, key1, stream_id, step;
    int32_t inject;           // time n+1 is an output in the window
    double dLdJ[Q];           // dL/dJ_q at time n+1 (objective weights / number of outputs included)
    double ddhat[NTH][P];     // d dhat_h / d theta_t (per step)
    double de0[Q][NTH];       // d eps0_q / d theta_t
    double nq[Q], dnq[Q];     // density and d n / d eps0 at the nodes (m^-2)
    double cJ;                // -e vF / N : J_q = cJ n_q sum_i vhat
};

template <int P, int Q, typename R>
__device__ __forceinline__ void block_add_grad(double *grad, double g[NTH])
{
    __shared__ double sg[NTH][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < NTH; ++t) {
        double v = g[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sg[t][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < NTH) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sg[threadIdx.x][w];
        if (s != 0.0) atomicAdd(&grad[threadIdx.x], s);
    }
}

// ------------------------------------------------------------------------------------------
// All particles: moment term, screen, drift term of the non-colliders.
// ------------------------------------------------------------------------------------------
template <int P, int Q, typename R>
__global__ void __launch_bounds__(256)
k_adj_screen(const __grid_constant__ AdjArgs<P, Q, R> a)
{
    const Phys<R> &ph = a.ph;
    const Nodes<P, Q, R> &nd = a.nd;
    double g[NTH] = {0.0, 0.0, 0.0, 0.0};
    // The drift and moment terms of the gradient are linear in per-particle quantities: for the
    // small shapes each thread sums those over its particles (in R) and applies the FP64
    // coefficients once at the end, instead of FP64 multiply-adds per particle (FP64 throughput
    // is low on this GPU).
    constexpr bool kSums = P * Q <= 64;
    constexpr int SP = kSums ? P : 1, SQ = kSums ? Q : 1;
    R slx[SP], svh[SQ], sdve[SQ];
#pragma unroll
    for (int h = 0; h < SP; ++h) slx[h] = (R)0;
#pragma unroll
    for (int q = 0; q < SQ; ++q) { svh[q] = (R)0; sdve[q] = (R)0; }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.N; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool maybe = false;
        if (i < a.N) {
            R lx[P], ly[P];
#pragma unroll
            for (int h = 0; h < P; ++h) {
                lx[h] = a.lam[(int64_t)h * a.ld + i];
                ly[h] = a.lam[(int64_t)(P + h) * a.ld + i];
            }
            if (a.inject) {
                // dL/dk(z_q) = dL/dJ_q cJ n_q d vhat/dk,  vhat = hvF kx / eps(k, eps0_q)  (in R)
                R cx[P], cy[P];
#pragma unroll
                for (int h = 0; h < P; ++h) {
                    cx[h] = a.khat_n1[(int64_t)h * a.ld + i];
                    cy[h] = a.khat_n1[(int64_t)(P + h) * a.ld + i];
                }
#pragma unroll 1
                for (int q = 0; q < Q; ++q) {
                    R kx, ky;
                    recon_node(nd, q, cx, cy, kx, ky);
                    const R e0 = nd.eps0[q], hv = ph.hvF;
                    const R eps = rsqrt_<R>(ph.hvF2 * (kx * kx + ky * ky) + e0 * e0);
                    const R ie = (R)1 / eps, ie3 = ie * ie * ie;
                    const R vhat = hv * kx * ie;
                    const R dvx = hv * ie - hv * ph.hvF2 * kx * kx * ie3;
                    const R dvy = -hv * ph.hvF2 * kx * ky * ie3;
                    const R dve = -hv * kx * e0 * ie3;
                    const double s = a.dLdJ[q] * a.cJ;
                    const R gx = (R)(s * a.nq[q]) * dvx, gy = (R)(s * a.nq[q]) * dvy;
#pragma unroll
                    for (int h = 0; h < P; ++h) {
                        lx[h] += gx * nd.psi[q * P + h];
                        ly[h] += gy * nd.psi[q * P + h];
                    }
                    if constexpr (kSums) {
                        svh[q] += vhat;
                        sdve[q] += dve;
                    } else {
#pragma unroll
                        for (int t = 0; t < NTH; ++t)
                            g[t] += s * (a.dnq[q] * a.de0[q][t] * (double)vhat + a.nq[q] * (double)dve * a.de0[q][t]);
                    }
                }
#pragma unroll
                for (int h = 0; h < P; ++h) {
                    a.lam[(int64_t)h * a.ld + i] = lx[h];
                    a.lam[(int64_t)(P + h) * a.ld + i] = ly[h];
                }
            }
            // the flight-time screen of phase 1 at step n (identical arithmetic)
            R cx[P], cy[P];
#pragma unroll
            for (int h = 0; h < P; ++h) {
                cx[h] = a.khat_n[(int64_t)h * a.ld + i];
                cy[h] = a.khat_n[(int64_t)(P + h) * a.ld + i];
                if (nd.drift_mask & (1u << h)) cx[h] -= nd.dhat[h];
            }
            R kkmax = (R)0;
            recon_all(nd, cx, cy, [&](int, R kx, R ky) { kkmax = fmax(kkmax, kx * kx + ky * ky); });
            const U4 r = philox4x32_10((uint32_t)i, a.stream_id, a.step, 0u, a.key0, a.key1);
            const R lnxi = -rlog<R>(u01<R>(r.x));
            const R emax = rsqrt_<R>(ph.hvF2 * kkmax + nd.eps0_max * nd.eps0_max);
            const R gub = ph.alpha1 * rate_bound(ph, emax, nd.eps0_max) * (R)1.0001;
            maybe = lnxi < gub * ph.dt;
            if (!maybe) {  // lambda* = lambda: drift term -sum_h d dhat_h/d theta lambda_x,h
                if constexpr (kSums) {
#pragma unroll
                    for (int h = 0; h < P; ++h) slx[h] += lx[h];
                } else {
#pragma unroll
                    for (int t = 0; t < NTH; ++t) {
                        double s = 0.0;
#pragma unroll
                        for (int h = 0; h < P; ++h) s += a.ddhat[t][h] * (double)lx[h];
                        g[t] -= s;
                    }
                }
            }
        }
        const unsigned int mask = __ballot_sync(0xffffffffu, maybe);
        if (mask) {
            const int leader = __ffs(mask) - 1;
            uint32_t basepos = 0;
            if (lane == leader) basepos = atomicAdd(a.qcount, (uint32_t)__popc(mask));
            basepos = __shfl_sync(0xffffffffu, basepos, leader);
            if (maybe) a.queue[basepos + __popc(mask & ((1u << lane) - 1u))] = (uint32_t)i;
        }
    }
    if constexpr (kSums) {
#pragma unroll
        for (int t = 0; t < NTH; ++t) {
            double s = 0.0;
#pragma unroll
            for (int h = 0; h < P; ++h) s += a.ddhat[t][h] * (double)slx[h];
            g[t] -= s;
        }
        if (a.inject)
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const double s = a.dLdJ[q] * a.cJ;
#pragma unroll
                for (int t = 0; t < NTH; ++t)
                    g[t] += s * (a.dnq[q] * a.de0[q][t] * (double)svh[q] + a.nq[q] * (double)sdve[q] * a.de0[q][t]);
            }
    }
    block_add_grad<P, Q, R>(a.grad, g);
}

// ------------------------------------------------------------------------------------------
// Jacobians of the final-state maps (Sec. 3) with the random numbers fixed, row-major 2x2.
// ------------------------------------------------------------------------------------------
template <typename R>
__device__ R edge_angle_grad(const Phys<R> &ph, R beta, R c, R u, R *dbeta, R *dc)
{
    const int n = ph.n_theta;
    R x = ph.cosj[0] - c;
    R g = rexp<R>(-beta * x * x);
    R gp = g, gbp = -x * x * g, gcp = (R)2 * beta * x * g;
    R total = (R)0, tb = (R)0, tcn = (R)0;
    for (int j = 1; j <= n; ++j) {
        x = ph.cosj[j] - c;
        g = rexp<R>(-beta * x * x);
        const R gb = -x * x * g, gc = (R)2 * beta * x * g;
        total += (R)0.5 * ph.edge_h * (gp + g);
        tb += (R)0.5 * ph.edge_h * (gbp + gb);
        tcn += (R)0.5 * ph.edge_h * (gcp + gc);
        gp = g; gbp = gb; gcp = gc;
    }
    const R target = u * total;
    x = ph.cosj[0] - c;
    gp = rexp<R>(-beta * x * x);
    gbp = -x * x * gp;
    gcp = (R)2 * beta * x * gp;
    R C = (R)0, Cb = (R)0, Cc = (R)0;
    for (int j = 1; j <= n; ++j) {
        x = ph.cosj[j] - c;
        g = rexp<R>(-beta * x * x);
        const R gb = -x * x * g, gc = (R)2 * beta * x * g;
        const R Cn = C + (R)0.5 * ph.edge_h * (gp + g);
        const R Cbn = Cb + (R)0.5 * ph.edge_h * (gbp + gb);
        const R Ccn = Cc + (R)0.5 * ph.edge_h * (gcp + gc);
        if (Cn > target || j == n) {
            const R D = Cn - C, Db = Cbn - Cb, Dc = Ccn - Cc;
            const R f = (target - C) / D;
            *dbeta = ((u * tb - Cb) * D - (target - C) * Db) / (D * D) * ph.edge_h;
            *dc = ((u * tcn - Cc) * D - (target - C) * Dc) / (D * D) * ph.edge_h;
            return ((R)(j - 1) + f) * ph.edge_h;
        }
        C = Cn; Cb = Cbn; Cc = Ccn;
        gp = g; gbp = gb; gcp = gc;
    }
    *dbeta = (R)0;
    *dc = (R)0;
    return (R)0;
}

template <typename R>
__device__ void fs_jacobian(const Phys<R> &ph, int l, R kx, R ky, EventAngles<R> &ang, R J[4])
{
    const R kk = kx * kx + ky * ky;
    const R km = rsqrt_<R>(kk);
    if (l == 5) {
        const R c = (km > (R)0) ? kx / km : (R)1;
        R db, dc;
        const R th = edge_angle_grad(ph, ph.two_a2 * kk, c, ang.u, &db, &dc);
        R st, ct;
        rsincos<R>(th, &st, &ct);
        const R nx = (km > (R)0) ? kx / km : (R)1, ny = (km > (R)0) ? ky / km : (R)0;
        const R gbx = (R)2 * ph.two_a2 * kx, gby = (R)2 * ph.two_a2 * ky;  // d beta / dk
        R gcx = (R)0, gcy = (R)0;                                           // d c / dk
        if (km > (R)0) { gcx = ky * ky / (km * kk); gcy = -kx * ky / (km * kk); }
        const R tx = db * gbx + dc * gcx, ty = db * gby + dc * gcy;
        J[0] = ct * nx - km * st * tx; J[1] = ct * ny - km * st * ty;
        J[2] = st * nx + km * ct * tx; J[3] = st * ny + km * ct * ty;
        return;
    }
    if (!(km > (R)0)) {  // |k| = 0 (measure zero): keep the identity
        J[0] = (R)1; J[1] = (R)0; J[2] = (R)0; J[3] = (R)1;
        return;
    }
    R th, s = (R)0, dlt = (R)0;
    if (l == 0) th = ang.ac();
    else if (l == 1 || l == 2) { th = (R)(2.0 * kPi) * ang.u; dlt = ph.wOk; s = (l == 1) ? (R)-1 : (R)1; }
    else { th = ang.kk(); dlt = ph.wKk; s = (l == 3) ? (R)-1 : (R)1; }
    R st, ct;
    rsincos<R>(th, &st, &ct);
    // k' = R(th) k (1 + s dlt/|k|):  dk'/dk = R(th) [ (1 + s dlt/|k|) I - (s dlt/|k|) n n^T ]
    const R aa = (R)1 + s * dlt / km, bb = s * dlt / km;
    const R nx = kx / km, ny = ky / km;
    const R M0 = aa - bb * nx * nx, M1 = -bb * nx * ny, M2 = -bb * ny * nx, M3 = aa - bb * ny * ny;
    J[0] = ct * M0 - st * M2; J[1] = ct * M1 - st * M3;
    J[2] = st * M0 + ct * M2; J[3] = st * M1 + ct * M3;
}

// Replays the collision loop of collide_particle for particle i (same operations, same group
// layout; an event that changes no node leaves the coefficients, rates and majorant untouched)
// for at most `stop` events; on return cx/cy/kx/ky hold the state before event `stop` (or the
// final state), and *nev the number of events the loop would run.  The mechanism of every node
// at event `stop` is returned in l_out[] (6 = unchanged).
template <int P, int Q, typename R>
__device__ __forceinline__ void replay_events(const Phys<R> &ph, const Nodes<P, Q, R> &nd, const AdjArgs<P, Q, R> &a,
                                              int64_t i, int r, unsigned gmask, int stop, R cx[P], R cy[P],
                                              R kx[GroupOf<Q>::NPL], R ky[GroupOf<Q>::NPL], int *nev,
                                              int l_out[GroupOf<Q>::NPL], U4 *r_out, R *red)
{
    constexpr int G = GroupOf<Q>::G, NPL = GroupOf<Q>::NPL;
    const int64_t NN = (int64_t)ph.Nk * ph.Nk;
#pragma unroll
    for (int h = 0; h < P; ++h) {
        cx[h] = a.khat_n[(int64_t)h * a.ld + i];
        cy[h] = a.khat_n[(int64_t)(P + h) * a.ld + i];
        if (nd.drift_mask & (1u << h)) cx[h] -= nd.dhat[h];
    }
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
        const int q = r + s * G;
        if (q < Q) recon_node(nd, q, cx, cy, kx[s], ky[s]);
    }
    auto majorant = [&]() {
        R gm = (R)0;
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
            const int q = r + s * G;
            if (q < Q) {
                R g[6];
                gm = fmax(gm, rates6(ph, kx[s], ky[s], nd.eps0[q], g));
            }
        }
        return ph.alpha1 * group_max<G>(gm, gmask);
    };
    R Gt = majorant();
    R tc = (R)0;
    uint32_t c = 0;
    U4 rr = philox4x32_10((uint32_t)i, a.stream_id, a.step, c, a.key0, a.key1);
    R dtc = (Gt > (R)0) ? -rlog<R>(u01<R>(rr.x)) / Gt : (R)INFINITY;
    int e = 0;
    while (tc + dtc < ph.dt) {
        if ((int)c >= ph.max_coll) break;
        if (e == stop) {  // report the decisions of this event without applying it
            *r_out = rr;
            const R target = u01<R>(rr.y) * Gt;
            EventAngles<R> ang;
            ang.reset(u01<R>(rr.w));
#pragma unroll
            for (int s = 0; s < NPL; ++s) {
                const int q = r + s * G;
                l_out[s] = 6;
                if (q >= Q) continue;
                R g[6];
                rates6(ph, kx[s], ky[s], nd.eps0[q], g);
                int l = 6;
                R cum = (R)0;
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    cum += g[m];
                    if (l == 6 && target < cum) l = m;
                }
                if (l == 6) continue;
                R nkx, nky;
                final_state(ph, l, kx[s], ky[s], nd.eps0[q], ang, &nkx, &nky);
                bool accept = true;
                if (ph.pauli_mode != 2) {
                    const int cl = cell_of(ph, nd.lkx[q], nkx + nd.dq[q], nky);
                    if (cl >= 0) accept = pauli_accept(a.Hn[(int64_t)q * NN + cl], a.nmax[q], rr.z);
                }
                if (accept) l_out[s] = l;
            }
            *nev = -1;
            return;
        }
        EventAngles<R> ang;
        ang.reset(u01<R>(rr.w));
        const R target = u01<R>(rr.y) * Gt;
        bool changed = false;
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
            const int q = r + s * G;
            if (q >= Q) continue;
            R g[6];
            rates6(ph, kx[s], ky[s], nd.eps0[q], g);
            int l = 6;
            R cum = (R)0;
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                cum += g[m];
                if (l == 6 && target < cum) l = m;
            }
            if (l == 6) continue;
            R nkx, nky;
            final_state(ph, l, kx[s], ky[s], nd.eps0[q], ang, &nkx, &nky);
            bool accept = true;
            if (ph.pauli_mode != 2) {
                const int cl = cell_of(ph, nd.lkx[q], nkx + nd.dq[q], nky);
                if (cl >= 0) accept = pauli_accept(a.Hn[(int64_t)q * NN + cl], a.nmax[q], rr.z);
            }
            if (accept) { kx[s] = nkx; ky[s] = nky; changed = true; }
        }
        if (group_any<G>(changed, gmask)) {   // the forward's projection, reconstruction and majorant
            project_group<P, Q, R>(nd, kx, ky, r, gmask, cx, cy, red);
#pragma unroll
            for (int s = 0; s < NPL; ++s) {
                const int q = r + s * G;
                if (q < Q) recon_node(nd, q, cx, cy, kx[s], ky[s]);
            }
            Gt = majorant();
        }
        tc += dtc;
        ++c;
        ++e;
        rr = philox4x32_10((uint32_t)i, a.stream_id, a.step, c, a.key0, a.key1);
        dtc = (Gt > (R)0) ? -rlog<R>(u01<R>(rr.x)) / Gt : (R)INFINITY;
    }
    *nev = e;
}

template <int P, int Q, typename R>
__global__ void __launch_bounds__(kPhase2Threads)
k_adj_collide(const __grid_constant__ AdjArgs<P, Q, R> a)
{
    constexpr int G = GroupOf<Q>::G, NPL = GroupOf<Q>::NPL;
    __shared__ __align__(16) uint32_t sph[(sizeof(Phys<R>) + 3) / 4];
    __shared__ __align__(16) uint32_t snd[(sizeof(Nodes<P, Q, R>) + 3) / 4];
    __shared__ R sred[ProjRed<P, Q, R>::value ? (kPhase2Threads / 32) * ProjRed<P, Q, R>::warp_elems : 1];
    stage(sph, a.ph);
    stage(snd, a.nd);
    __syncthreads();
    const Phys<R> &ph = *reinterpret_cast<const Phys<R> *>(sph);
    const Nodes<P, Q, R> &nd = *reinterpret_cast<const Nodes<P, Q, R> *>(snd);
    const uint32_t count = *a.qcount;
    const int lane = threadIdx.x & 31;
    const int r = lane % G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane - r));
    const uint32_t gid = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    const uint32_t ngroups = gridDim.x * blockDim.x / G;
    double g[NTH] = {0.0, 0.0, 0.0, 0.0};
    for (uint32_t j = gid; j < count; j += ngroups) {
        const int64_t i = a.queue[j];
        R lx[P], ly[P];
#pragma unroll
        for (int h = 0; h < P; ++h) {
            lx[h] = a.lam[(int64_t)h * a.ld + i];
            ly[h] = a.lam[(int64_t)(P + h) * a.ld + i];
        }
        R cx[P], cy[P], kx[NPL], ky[NPL];
        int nev = 0, lsel[NPL];
        U4 rr;
        replay_events(ph, nd, a, i, r, gmask, 1 << 30, cx, cy, kx, ky, &nev, lsel, &rr, sred);
        for (int e = nev - 1; e >= 0; --e) {
            int dummy;
            replay_events(ph, nd, a, i, r, gmask, e, cx, cy, kx, ky, &dummy, lsel, &rr, sred);
            bool any = false;
#pragma unroll
            for (int s = 0; s < NPL; ++s) any |= lsel[s] < 6;
            if (!group_any<G>(any, gmask)) continue;   // an event that changed no node is the identity
            EventAngles<R> ang;
            ang.reset(u01<R>(rr.w));
            // lambda_e = sum_q Psi_q^T J_q^T (W_q^T lambda_{e+1})
            R nx[NPL], ny[NPL];
#pragma unroll
            for (int s = 0; s < NPL; ++s) {
                const int q = r + s * G;
                nx[s] = (R)0; ny[s] = (R)0;
                if (q >= Q) continue;
                R mx = (R)0, my = (R)0;
#pragma unroll
                for (int h = 0; h < P; ++h) {
                    mx += nd.wpsi[q * P + h] * lx[h];
                    my += nd.wpsi[q * P + h] * ly[h];
                }
                if (lsel[s] < 6) {
                    R J[4];
                    fs_jacobian(ph, lsel[s], kx[s], ky[s], ang, J);
                    nx[s] = J[0] * mx + J[2] * my;
                    ny[s] = J[1] * mx + J[3] * my;
                } else {
                    nx[s] = mx;
                    ny[s] = my;
                }
            }
#pragma unroll
            for (int h = 0; h < P; ++h) {
                R sx = (R)0, sy = (R)0;
#pragma unroll
                for (int s = 0; s < NPL; ++s) {
                    const int q = r + s * G;
                    if (q < Q) {
                        sx += nd.psi[q * P + h] * nx[s];
                        sy += nd.psi[q * P + h] * ny[s];
                    }
                }
                lx[h] = group_sum<G>(sx, gmask);
                ly[h] = group_sum<G>(sy, gmask);
            }
        }
        if (r == 0) {
#pragma unroll
            for (int t = 0; t < NTH; ++t) {
                double s = 0.0;
#pragma unroll
                for (int h = 0; h < P; ++h) s += a.ddhat[t][h] * (double)lx[h];
                g[t] -= s;
            }
        }
        for (int h = r; h < P; h += G) {
            R vx = lx[0], vy = ly[0];
#pragma unroll
            for (int hh = 0; hh < P; ++hh) if (hh == h) { vx = lx[hh]; vy = ly[hh]; }
            a.lam[(int64_t)h * a.ld + i] = vx;
            a.lam[(int64_t)(P + h) * a.ld + i] = vy;
        }
    }
    block_add_grad<P, Q, R>(a.grad, g);
}

// ------------------------------------------------------------------------------------------
// lambda^0 . d khat^0 / d theta through the Fermi-Dirac sampling (FP64).
// ------------------------------------------------------------------------------------------
template <int P, int Q>
struct AdjInitArgs {
    double wpsi[Q * P];
    double eps0[Q];
    double de0[Q][NTH];
    double mu, kT, hvF;
};

template <int P, int Q, typename R>
__global__ void __launch_bounds__(128)
k_adj_init(const __grid_constant__ AdjArgs<P, Q, R> a, const __grid_constant__ AdjInitArgs<P, Q> ia)
{
    double g[NTH] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.N; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        if (i >= a.N) continue;
        const U4 rr = philox4x32_10((uint32_t)i, a.stream_id, 0u, 0x10000u, a.key0, a.key1);
        const double ue = u01<double>(rr.x), uth = u01<double>(rr.y);
        double sn, cs;
        sincos(2.0 * kPi * uth, &sn, &cs);
        double lx[P], ly[P];
#pragma unroll
        for (int h = 0; h < P; ++h) {
            lx[h] = (double)a.lam[(int64_t)h * a.ld + i];
            ly[h] = (double)a.lam[(int64_t)(P + h) * a.ld + i];
        }
        for (int q = 0; q < Q; ++q) {
            const double e0 = ia.eps0[q];
            const double eps = fd_inverse(e0, ia.mu, ia.kT, ue);
            const double rr2 = eps * eps - e0 * e0;
            if (!(rr2 > 0.0)) continue;
            const double km = sqrt(rr2) / ia.hvF;
            auto rho = [&](double e) { return e / (1.0 + exp(fmin((e - ia.mu) / ia.kT, 700.0))); };
            const double deps = rho(e0) * (1.0 - ue) / rho(eps);
            const double dkm = (eps * deps - e0) / (ia.hvF * ia.hvF * km);
            double mx = 0.0, my = 0.0;
#pragma unroll
            for (int h = 0; h < P; ++h) { mx += ia.wpsi[q * P + h] * lx[h]; my += ia.wpsi[q * P + h] * ly[h]; }
            const double proj = dkm * (mx * cs + my * sn);
#pragma unroll
            for (int t = 0; t < NTH; ++t) g[t] += proj * ia.de0[q][t];
        }
    }
    block_add_grad<P, Q, R>(a.grad, g);
}

// ------------------------------------------------------------------------------------------
// Host side: the argument blocks and launches of one backward step.
// ------------------------------------------------------------------------------------------
struct AdjBuffers {
    void *lam = nullptr;
    uint32_t *queue = nullptr, *qcount = nullptr;
    double *grad = nullptr;
};

class AdjRunner {
public:
    virtual ~AdjRunner() {}
    // backward step n: moment term of time n+1 (if inject), then the map of step n
    virtual cudaError_t backward_step(const void *khat_n, const void *khat_n1, const uint32_t *Hn, int64_t n,
                                      bool inject, const double *dLdJ, cudaStream_t s) = 0;
    virtual cudaError_t init_term(cudaStream_t s) = 0;
};

template <int P, int Q, typename R>
class AdjRunnerT final : public AdjRunner {
public:
    AdjRunnerT(const HostTables &t, const DevBuffers &b, const AdjBuffers &ab, int num_sms) : ab_(ab)
    {
        RunnerT<P, Q, R> proto(t, b, num_sms);
        a_.ph = proto.args().ph;
        a_.nd = proto.args().nd;
        a_.lam = static_cast<R *>(ab.lam);
        a_.nmax = b.nmax;
        a_.queue = ab.queue;
        a_.qcount = ab.qcount;
        a_.grad = ab.grad;
        a_.N = b.N;
        a_.ld = b.ld;
        a_.key0 = b.key0;
        a_.key1 = b.key1;
        a_.stream_id = b.stream_id;
        const double c = 1.602176634e-19 * t.vF_ms / (double)b.N;
        a_.cJ = -c;
        // parameter derivatives of the nodes (affine maps; z = 0 for a deterministic input)
        for (int q = 0; q < Q; ++q) {
            double z1 = 0.0, z2 = 0.0;
            if (t.d == 1) { if (t.eps_random) z1 = t.z[q]; else z2 = t.z[q]; }
            if (t.d == 2) { z1 = t.z[2 * q]; z2 = t.z[2 * q + 1]; }
            double dE[NTH] = {0.5 * (1.0 - z2), 0.5 * (1.0 + z2), 0.0, 0.0};
            double de0[NTH] = {0.0, 0.0, 0.5 * (1.0 - z1), 0.5 * (1.0 + z1)};
            for (int k = 0; k < NTH; ++k) { a_.de0[q][k] = de0[k]; dEq_[q][k] = dE[k]; }
            a_.nq[q] = t.nq[q];
            const double e0 = t.eps0[q];
            const double rho = e0 / (1.0 + std::exp(std::fmin((e0 - t.mu) / t.kT, 700.0)));
            a_.dnq[q] = -2.0 / (kPi * t.hvF * t.hvF) * rho * 1.0e18;
        }
        for (int k = 0; k < NTH; ++k)
            for (int h = 0; h < P; ++h) {
                double sacc = 0.0;
                for (int q = 0; q < Q; ++q) sacc += t.wpsi[(size_t)q * P + h] * dEq_[q][k] * 1.0e-7 * t.dt / t.hbar_fs;
                a_.ddhat[k][h] = sacc;
            }
        for (int i = 0; i < Q * P; ++i) ia_.wpsi[i] = t.wpsi[i];
        for (int q = 0; q < Q; ++q) {
            ia_.eps0[q] = t.eps0[q];
            for (int k = 0; k < NTH; ++k) ia_.de0[q][k] = a_.de0[q][k];
        }
        ia_.mu = t.mu;
        ia_.kT = t.kT;
        ia_.hvF = t.hvF;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_screen<P, Q, R>, 256, 0);
        grid_ = (int)std::max<int64_t>(1, std::min<int64_t>((b.N + 255) / 256, (int64_t)num_sms * std::max(per_sm, 1)));
    }

    cudaError_t backward_step(const void *khat_n, const void *khat_n1, const uint32_t *Hn, int64_t n, bool inject,
                              const double *dLdJ, cudaStream_t s) override
    {
        AdjArgs<P, Q, R> a = a_;
        a.khat_n = static_cast<const R *>(khat_n);
        a.khat_n1 = static_cast<const R *>(khat_n1);
        a.Hn = Hn;
        a.step = (uint32_t)n;
        a.inject = inject ? 1 : 0;
        for (int q = 0; q < Q; ++q) a.dLdJ[q] = inject ? dLdJ[q] : 0.0;
        cudaError_t e = cudaMemsetAsync(ab_.qcount, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
        k_adj_screen<P, Q, R><<<grid_, 256, 0, s>>>(a);
        k_adj_collide<P, Q, R><<<kGrid2, kPhase2Threads, 0, s>>>(a);
        count_launch(2);
        return cudaGetLastError();
    }

    cudaError_t init_term(cudaStream_t s) override
    {
        int blocks = (int)std::min<int64_t>((a_.N + 127) / 128, 8192);
        k_adj_init<P, Q, R><<<blocks, 128, 0, s>>>(a_, ia_);
        count_launch();
        return cudaGetLastError();
    }

private:
    AdjBuffers ab_;
    AdjArgs<P, Q, R> a_{};
    AdjInitArgs<P, Q> ia_{};
    double dEq_[Q][NTH];
    int grid_ = 1;
};

template <int P, int Q>
AdjRunner *make_adj_runner_shape(int precision, const HostTables &t, const DevBuffers &b, const AdjBuffers &ab, int num_sms)
{
    if (precision == 1) return new AdjRunnerT<P, Q, double>(t, b, ab, num_sms);
    return new AdjRunnerT<P, Q, float>(t, b, ab, num_sms);
}

}  // namespace pgc
