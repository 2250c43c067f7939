// pgc_device.cuh -- device building blocks of the particle stochastic-Galerkin step
// (arXiv:2404.19602): counter-based random numbers, the closed-form scattering rates of
// Appendix A, the final-state maps h^1..h^7 of Sec. 3, the grid of the Pauli test, and the
// Fermi-Dirac sampler of the initial state.  Everything is templated on the arithmetic type R
// (float for the production path, double for the FP64 mode).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pgc {

constexpr int kMaxTheta = 256;   // upper bound of the edge trapezoid points
constexpr int kSerMax = 17;      // maximum order + 1 of the edge-integral series
constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------------------------------------------------
// Physical constants of one context, prepared on the host in FP64 and stored in R.
// Rates are in 1/fs; energies eV; wave-vectors nm^-1.
// ------------------------------------------------------------------------------------------
template <typename R>
struct Phys {
    R hvF, hvF2;          // hbar vF (eV nm) and its square
    R Lk, dk, inv_dk;     // grid half-width, cell size, 1/cell size
    R alpha1;             // 1 + alpha
    R dt;                 // fs
    R Cac;                // Gamma_ac = Cac * eps
    R COm, COp, CKm, CKp; // Gamma_O- = COm (eps - hwO) H(..), Gamma_O+ = COp (eps + hwO) ...
    R hwO, hwK;           // phonon energies, eV
    R wOk, wKk;           // hbar omega / (hbar vF): |k| change of the paper's final states
    R Cedg;               // Gamma_edg = Cedg * eps0 * eps * T(|k|, cos th)
    R two_a2;             // 2 a^2 (nm^2)
    R edge_h;             // 2 pi / n_theta
    R bound_edge;         // 2 pi * (1 + 1e-5): upper bound of the trapezoid T
    R vF_ms;              // vF in m/s
    R cosj[kMaxTheta + 1];// cos(2 pi j / n_theta), j = 0..n_theta
    // power series of T in beta (see edge_T): coefficient (j, m) of beta^j (c^2)^(j-m)
    R tser[kSerMax * kSerMax];
    R beta_ser;           // the series is used for beta <= beta_ser
    int32_t J;            // series order
    uint32_t mech;
    int32_t n_theta;
    int32_t pauli_mode;   // 0 initial max, 1 current max, 2 off
    int32_t final_state;  // 0 paper, 1 exact energy
    int32_t max_coll;
    int32_t Nk;
};

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, two multipliers, Weyl keys.
// ------------------------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// odd multiples of 2^-24 in (0,1): identical values in FP32 and FP64
template <typename R> __device__ __forceinline__ R u01(uint32_t x)
{
    return (R)((x >> 8) | 1u) * (R)5.9604644775390625e-8;
}

template <typename R> __device__ __forceinline__ R rlog(R x);
template <> __device__ __forceinline__ float rlog<float>(float x) { return logf(x); }
template <> __device__ __forceinline__ double rlog<double>(double x) { return log(x); }
template <typename R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return sqrt(x); }
template <typename R> __device__ __forceinline__ R rexp(R x);
template <> __device__ __forceinline__ float rexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double rexp<double>(double x) { return exp(x); }
template <typename R> __device__ __forceinline__ void rsincos(R x, R *s, R *c);
template <> __device__ __forceinline__ void rsincos<float>(float x, float *s, float *c) { sincosf(x, s, c); }
template <> __device__ __forceinline__ void rsincos<double>(double x, double *s, double *c) { sincos(x, s, c); }
template <typename R> __device__ __forceinline__ R rsin(R x);
template <> __device__ __forceinline__ float rsin<float>(float x) { return sinf(x); }
template <> __device__ __forceinline__ double rsin<double>(double x) { return sin(x); }
template <typename R> __device__ __forceinline__ R rfloor(R x);
template <> __device__ __forceinline__ float rfloor<float>(float x) { return floorf(x); }
template <> __device__ __forceinline__ double rfloor<double>(double x) { return floor(x); }

// ------------------------------------------------------------------------------------------
// Cell of a wave-vector on the fixed grid [-Lk, Lk]^2 (Sec. 3); -1 outside.  The FP64 mode
// gives the cell of the division (as the definition reads, floor_div_f64); the FP32 mode
// multiplies by the reciprocal.
// ------------------------------------------------------------------------------------------
// floor(fl(x / dk)) in FP64 with the division taken only where it can matter: x * fl(1/dk) lies
// within 2 ulps of fl(x / dk), so their floors differ only if an integer lies within 2 ulps of
// the product; there (8 ulps, to spare) the quotient is formed by the division itself.  The FP64
// divide is a long sequence on the FP64 pipe, which this part issues at a small fraction of the
// FP32 rate; the cell is the same as the division's in every case.
__device__ __forceinline__ int floor_div_f64(double x, double dk, double inv_dk)
{
    const double y = x * inv_dk;
    if (fabs(y - rint(y)) <= fabs(y) * 0x1p-49) return __double2int_rd(x / dk);
    return __double2int_rd(y);
}

template <typename R>
__device__ __forceinline__ bool cell_rl(const Phys<R> &ph, R kx, R ky, int &r, int &l)
{
    // floor and conversion in one rounding-down conversion; outside the grid (including the
    // saturated conversions of huge values) fails the unsigned comparison
    if constexpr (sizeof(R) == 8) {
        r = floor_div_f64(kx + ph.Lk, ph.dk, ph.inv_dk);
        l = floor_div_f64(ky + ph.Lk, ph.dk, ph.inv_dk);
    } else {
        r = __float2int_rd((kx + ph.Lk) * ph.inv_dk);
        l = __float2int_rd((ky + ph.Lk) * ph.inv_dk);
    }
    return (unsigned)r < (unsigned)ph.Nk && (unsigned)l < (unsigned)ph.Nk;
}

template <typename R>
__device__ __forceinline__ int cell_of(const Phys<R> &ph, R kx, R ky)
{
    int r, l;
    return cell_rl(ph, kx, ky, r, l) ? r * ph.Nk + l : -1;
}

// The same cells with the x offset of the grid given per node: lkx = Lk - s counts k on the grid
// moved by s along x (s = half a step's drift under the Strang splitting; lkx = Lk otherwise,
// which is the arithmetic of cell_rl).
template <typename R>
__device__ __forceinline__ bool cell_rl(const Phys<R> &ph, R lkx, R kx, R ky, int &r, int &l)
{
    if constexpr (sizeof(R) == 8) {
        r = floor_div_f64(kx + lkx, ph.dk, ph.inv_dk);
        l = floor_div_f64(ky + ph.Lk, ph.dk, ph.inv_dk);
    } else {
        r = __float2int_rd((kx + lkx) * ph.inv_dk);
        l = __float2int_rd((ky + ph.Lk) * ph.inv_dk);
    }
    return (unsigned)r < (unsigned)ph.Nk && (unsigned)l < (unsigned)ph.Nk;
}

template <typename R>
__device__ __forceinline__ int cell_of(const Phys<R> &ph, R lkx, R kx, R ky)
{
    int r, l;
    return cell_rl(ph, lkx, kx, ky, r, l) ? r * ph.Nk + l : -1;
}

// ------------------------------------------------------------------------------------------
// Edge integral T(|k|, c) = int_0^{2pi} exp(-beta (cos th' - c)^2) d th' (Appendix A).
// The paper evaluates it by the trapezoid rule.  For a periodic analytic integrand the
// n_theta-point rule is exact up to the Fourier modes of order >= n_theta, whose weight is
// ~beta^(n_theta/2)/(n_theta/2)!: for beta <= beta_ser the rule equals the integral to working
// precision, and the integral is summed from its power series
//   T/(2 pi) = sum_j (-beta)^j / j! E[(cos th' - c)^{2j}],
//   E[(cos th' - c)^{2j}] = sum_m C(2j,2m) C(2m,m) 4^-m c^{2(j-m)}
// (J + 1 terms, Horner in c^2 and beta).  Otherwise: the trapezoid rule itself, using the
// mirror symmetry th' -> 2pi - th'.
// ------------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R edge_T(const Phys<R> &ph, R beta, R c)
{
    if (beta <= ph.beta_ser) {
        constexpr int J = (sizeof(R) == 8) ? 16 : 10;
        const R x = c * c;
        R acc = (R)0;
#pragma unroll
        for (int j = J; j >= 0; --j) {
            const R *a = &ph.tser[j * kSerMax];
            R p = a[0];
#pragma unroll
            for (int m = 1; m <= j; ++m) p = p * x + a[m];
            acc = acc * beta + p;
        }
        return (R)(2.0 * kPi) * acc;
    }
    const int half = ph.n_theta >> 1;
    R x0 = ph.cosj[0] - c, xh = ph.cosj[half] - c;
    R s = rexp<R>(-beta * x0 * x0) + rexp<R>(-beta * xh * xh);
    R inner = (R)0;
    for (int j = 1; j < half; ++j) {
        const R x = ph.cosj[j] - c;
        inner += rexp<R>(-beta * x * x);
    }
    return ph.edge_h * (s + (R)2 * inner);
}

// Rates of the six mechanisms of Eq. (20) at one state (Appendix A closed forms).  Returns the sum.
template <typename R>
__device__ __forceinline__ R rates6(const Phys<R> &ph, R kx, R ky, R eps0, R g[6])
{
    const R kk = kx * kx + ky * ky;
    const R eps = rsqrt_<R>(ph.hvF2 * kk + eps0 * eps0);
    const uint32_t m = ph.mech;
    g[0] = (m & 1u) ? ph.Cac * eps : (R)0;
    g[1] = ((m & 2u) && (eps - ph.hwO - eps0 > (R)0)) ? ph.COm * (eps - ph.hwO) : (R)0;
    g[2] = ((m & 4u) && (eps + ph.hwO - eps0 > (R)0)) ? ph.COp * (eps + ph.hwO) : (R)0;
    g[3] = ((m & 8u) && (eps - ph.hwK - eps0 > (R)0)) ? ph.CKm * (eps - ph.hwK) : (R)0;
    g[4] = ((m & 16u) && (eps + ph.hwK - eps0 > (R)0)) ? ph.CKp * (eps + ph.hwK) : (R)0;
    if (m & 32u) {
        const R km = rsqrt_<R>(kk);
        const R c = (km > (R)0) ? kx / km : (R)1;
        g[5] = ph.Cedg * eps0 * eps * edge_T<R>(ph, ph.two_a2 * kk, c);
    } else {
        g[5] = (R)0;
    }
    return ((((g[0] + g[1]) + g[2]) + g[3]) + g[4]) + g[5];  // the order of Eq. (20)
}

// Upper bound of sum_nu Gamma_nu over all states with energy <= eps and band minimum <= eps0max:
// every closed form is non-decreasing in eps, the Heaviside factors are dropped, T <= 2pi.
template <typename R>
__device__ __forceinline__ R rate_bound(const Phys<R> &ph, R eps, R eps0max)
{
    const uint32_t m = ph.mech;
    R s = (R)0;
    if (m & 1u) s += ph.Cac * eps;
    if (m & 2u) s += ph.COm * fmax(eps - ph.hwO, (R)0);
    if (m & 4u) s += ph.COp * (eps + ph.hwO);
    if (m & 8u) s += ph.CKm * fmax(eps - ph.hwK, (R)0);
    if (m & 16u) s += ph.CKp * (eps + ph.hwK);
    if (m & 32u) s += ph.Cedg * eps0max * eps * ph.bound_edge;
    return s;
}

// ------------------------------------------------------------------------------------------
// Angle laws of the final states (Sec. 3).  One uniform u per collision, shared by all nodes.
// (1 + cos th) on [0, 2pi): solve th + sin th = 2 pi u ; (1 - cos th): th - sin th = 2 pi u.
// Both maps are monotone; safeguarded Newton iteration to the working precision.
// ------------------------------------------------------------------------------------------
template <typename R>
__device__ __noinline__ R solve_angle(R u, R sgn)
{
    // f(th) = th + sgn sin th - 2 pi u is non-decreasing on [0, 2pi]; safeguarded Newton from a
    // start that captures the cubic behaviour at the stationary point (th = pi for sgn = +1,
    // th = 0 or 2pi for sgn = -1).
    const R twopi = (R)(2.0 * kPi), t = twopi * u;
    R lo = (R)0, hi = twopi, th;
    if (sgn > (R)0) th = (R)kPi + cbrt((R)6 * (t - (R)kPi));
    else th = (t < (R)kPi) ? cbrt((R)6 * t) : twopi - cbrt((R)6 * (twopi - t));
    th = fmin(fmax(th, (R)0), twopi);
    const int iters = (sizeof(R) == 8) ? 60 : 30;
    const R tol = (sizeof(R) == 8) ? (R)1e-15 : (R)2e-7;
    for (int it = 0; it < iters; ++it) {
        R s, c;
        rsincos<R>(th, &s, &c);
        const R f = th + sgn * s - t, df = (R)1 + sgn * c;
        if (f == (R)0) break;  // exact root
        if (f < (R)0) lo = th; else hi = th;
        R tn = (df > (R)0) ? th - f / df : (R)0.5 * (lo + hi);
        if (!(tn >= lo && tn <= hi)) tn = (R)0.5 * (lo + hi);  // keep the iterate in the bracket
        const R d = fabs(tn - th);
        th = tn;
        if (d <= tol * twopi || hi - lo <= tol * twopi) break;
    }
    return th;
}

// Edge final angle: absolute angle with density exp(-beta (c - cos th')^2), inverted through
// the trapezoid CDF on the n_theta grid, linear between grid points.  The total of the CDF is
// T(beta, c) (edge_T); one pass up to the target's segment.
template <typename R>
__device__ R edge_angle(const Phys<R> &ph, R beta, R c, R u)
{
    const int n = ph.n_theta;
    const R target = u * edge_T<R>(ph, beta, c);
    R C = (R)0;
    R prev = rexp<R>(-beta * (ph.cosj[0] - c) * (ph.cosj[0] - c));
    for (int j = 1; j <= n; ++j) {
        const R x = ph.cosj[j] - c;
        const R g = rexp<R>(-beta * x * x);
        const R Cn = C + (R)0.5 * ph.edge_h * (prev + g);
        if (Cn > target || j == n) {
            const R frac = fmin(fmax((target - C) / (Cn - C), (R)0), (R)1);
            return ((R)(j - 1) + frac) * ph.edge_h;
        }
        C = Cn;
        prev = g;
    }
    return (R)0;
}

// Lazily computed angles of one collision event (common to every node)
template <typename R>
struct EventAngles {
    R u;
    R th_ac, th_k;
    bool have_ac, have_k;
    __device__ void reset(R uu) { u = uu; have_ac = have_k = false; }
    __device__ R ac() { if (!have_ac) { th_ac = solve_angle<R>(u, (R)1); have_ac = true; } return th_ac; }
    __device__ R kk() { if (!have_k) { th_k = solve_angle<R>(u, (R)-1); have_k = true; } return th_k; }
};

// Final state h^l(k) of mechanism l (0..5) at one node (Sec. 3).  Self scattering (l = 6) is
// handled by the caller.
template <typename R>
__device__ __forceinline__ void final_state(const Phys<R> &ph, int l, R kx, R ky, R eps0,
                                            EventAngles<R> &ang, R *nkx, R *nky)
{
    const R kk = kx * kx + ky * ky;
    const R km = rsqrt_<R>(kk);
    if (l == 5) {  // edge: absolute final angle, |k'| = |k|
        const R c = (km > (R)0) ? kx / km : (R)1;
        const R th = edge_angle<R>(ph, ph.two_a2 * kk, c, ang.u);
        R s, co;
        rsincos<R>(th, &s, &co);
        *nkx = km * co;
        *nky = km * s;
        return;
    }
    const R ci = (km > (R)0) ? kx / km : (R)1;
    const R si = (km > (R)0) ? ky / km : (R)0;
    R th, kn;
    if (l == 0) {
        th = ang.ac();
        kn = km;
    } else {
        const bool emit = (l == 1 || l == 3);
        const bool opt = (l == 1 || l == 2);
        th = opt ? (R)(2.0 * kPi) * ang.u : ang.kk();
        const R hw = opt ? ph.hwO : ph.hwK;
        if (ph.final_state == 1) {
            const R eps = rsqrt_<R>(ph.hvF2 * kk + eps0 * eps0);
            const R ep = emit ? eps - hw : eps + hw;
            kn = rsqrt_<R>(ep * ep - eps0 * eps0) / ph.hvF;
        } else {
            const R dk = opt ? ph.wOk : ph.wKk;
            kn = emit ? km - dk : km + dk;
        }
    }
    R st, ct;
    rsincos<R>(th, &st, &ct);
    *nkx = kn * (ct * ci - st * si);
    *nky = kn * (st * ci + ct * si);
}

// Pauli acceptance of a candidate in a cell: f = H / Nmax < eta with eta = m 2^-24 (m odd),
// decided exactly in integers: H 2^24 < m Nmax.  Outside the grid or Nmax = 0: f = 0, accept.
__device__ __forceinline__ bool pauli_accept(uint32_t H, uint32_t nmax, uint32_t eta_bits)
{
    if (nmax == 0u) return true;
    const uint64_t m = (uint64_t)((eta_bits >> 8) | 1u);
    return ((uint64_t)H << 24) < m * (uint64_t)nmax;
}

// ------------------------------------------------------------------------------------------
// Fermi-Dirac initial state (Sec. 2): energy density eps * FD(eps) on [eps0, inf).
// int_e^inf x/(1+exp((x-mu)/kT)) dx = kT [ mu ln(1+e^-b) + kT (b ln(1+e^-b) - Li2(-e^-b)) ],
// b = (e - mu)/kT.  Li2 for negative arguments: Bernoulli series in t = -ln(1 - x) on
// [-1, 0], inversion formula below -1.
// ------------------------------------------------------------------------------------------
template <typename T>
__host__ __device__ inline T li2_bern(T x)
{
    // x in [-1, 0]:  Li2(x) = sum_n B_n t^{n+1}/(n+1)!,  t = -ln(1 - x),  |t| <= ln 2;
    // B_0 t + B_1 t^2/2 + t^3 sum_k c_k (t^2)^k with c_k = B_{2k+2} / (2k+3)!, by Horner (no
    // divisions: on this GPU FP64 division is the dominant cost of the Fermi-Dirac inversion)
    const T t = -log1p(-x);
    constexpr double c[12] = {(1.0 / 6.0) / 6.0, (-1.0 / 30.0) / 120.0, (1.0 / 42.0) / 5040.0,
                              (-1.0 / 30.0) / 362880.0, (5.0 / 66.0) / 39916800.0,
                              (-691.0 / 2730.0) / 6227020800.0, (7.0 / 6.0) / 1307674368000.0,
                              (-3617.0 / 510.0) / 355687428096000.0, (43867.0 / 798.0) / 121645100408832000.0,
                              (-174611.0 / 330.0) / 51090942171709440000.0,
                              (854513.0 / 138.0) / 25852016738884976640000.0,
                              (-236364091.0 / 2730.0) / 15511210043330985984000000.0};
    constexpr int nterms = (sizeof(T) == 8) ? 12 : 5;
    const T t2 = t * t;
    T poly = (T)c[nterms - 1];
#pragma unroll
    for (int k = nterms - 2; k >= 0; --k) poly = poly * t2 + (T)c[k];
    return t - (T)0.25 * t2 + t * t2 * poly;
}

template <typename T>
__host__ __device__ inline T li2_negative(T x)
{
    if (x >= (T)-1) return li2_bern<T>(x);
    const T l = log(-x);
    return (T)(-kPi * kPi / 6.0) - (T)0.5 * l * l - li2_bern<T>((T)1 / x);
}

template <typename T>
__host__ __device__ inline T fd_upper(T e, T mu, T kT)
{
    const T b = (e - mu) / kT;
    const T l = (b > (T)0) ? log1p(exp(-b)) : -b + log1p(exp(b));
    const T big = (sizeof(T) == 8) ? (T)700 : (T)80;
    T li;
    if (b > big) li = (T)0;
    else if (b < -big) li = (T)(-kPi * kPi / 6.0) - (T)0.5 * b * b;
    else li = li2_negative<T>(-exp(-b));
    return kT * (mu * l + kT * (b * l - li));
}

// eps with F(eps) = u for the density eps*FD on [eps0, inf): an FP32 bisection gives a bracket,
// checked in FP64, then safeguarded Newton in FP64 (plain FP64 bisection if the check fails).
__host__ __device__ inline double fd_inverse(double eps0, double mu, double kT, double u)
{
    const double tot = fd_upper<double>(eps0, mu, kT), itot = 1.0 / tot;
    auto resid = [&](double e) {  // F(e) - u  (upper-tail form for u >= 1/2)
        return (u < 0.5) ? (tot - fd_upper<double>(e, mu, kT)) * itot - u : (1.0 - u) - fd_upper<double>(e, mu, kT) * itot;
    };
    const double top = fmax(mu, eps0) + 80.0 * kT;
    double lo = eps0, hi = top;
    {
        const float e0f = (float)eps0, muf = (float)mu, kTf = (float)kT, uf = (float)u;
        const float totf = fd_upper<float>(e0f, muf, kTf);
        float lf = e0f, hf = (float)top;
        for (int it = 0; it < 30; ++it) {
            const float mid = 0.5f * (lf + hf);
            if (!(mid > lf && mid < hf)) break;
            const float rf = (uf < 0.5f) ? (totf - fd_upper<float>(mid, muf, kTf)) / totf - uf
                                         : (1.0f - uf) - fd_upper<float>(mid, muf, kTf) / totf;
            if (rf < 0.0f) lf = mid; else hf = mid;
        }
        const double w = 1e-4 * ((double)hf - (double)lf) + 1e-6 * (double)hf;
        const double l2 = fmax(eps0, (double)lf - w), h2 = fmin(top, (double)hf + w);
        if (resid(l2) <= 0.0 && resid(h2) >= 0.0) { lo = l2; hi = h2; }
    }
    if (hi - lo > 1e-3 * hi)  // bracket check failed: FP64 bisection from the full range
        for (int it = 0; it < 40; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (resid(mid) < 0.0) lo = mid; else hi = mid;
        }
    // Newton from the bracket midpoint; quadratic convergence from the FP32 bracket reaches
    // rounding level in 2-3 steps, so stop once a step is below a few ulps (Newton iterates can
    // oscillate by an ulp and never meet a tighter test).
    double e = 0.5 * (lo + hi);
    for (int it = 0; it < 16; ++it) {
        const double r = resid(e);
        if (r == 0.0) break;  // exact root
        if (r < 0.0) lo = e; else hi = e;
        const double dens = e / (1.0 + exp(fmin((e - mu) / kT, 700.0))) * itot;
        double en = (dens > 0.0) ? e - r / dens : 0.5 * (lo + hi);
        if (!(en >= lo && en <= hi)) en = 0.5 * (lo + hi);  // keep the iterate in the bracket
        const double step = fabs(en - e);
        e = en;
        if (step <= 4e-16 * e) break;
    }
    return e;
}

}  // namespace pgc
