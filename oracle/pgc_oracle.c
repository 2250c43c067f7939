/*
 * pgc_oracle.c -- plain FP64 CPU oracle of the particle (stochastic-Galerkin) scheme for the
 * space-homogeneous semiclassical Boltzmann equation of electrons in a graphene nanoribbon
 * (Medaglia, Nastasi, Romano, Zanella, arXiv:2404.19602).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that the CUDA
 * path is checked against.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline /
 * reference leg may load it.  It shares no code, header or table with the CUDA library.
 *
 * Everything is FP64.  Every function cites the passage of the paper it follows.  Where the
 * paper is silent or ambiguous, the reading taken is stated next to the code (and collected in
 * the design notes of the repository).
 *
 * Units: energy eV, time fs, wave-vector nm^-1, field V/cm.  Velocities are reported in m/s,
 * densities in m^-2, the sheet current J = -e n V_x in A/m.
 *
 * Parity status of the functions (what pins each one, see tests/test_oracle_*.py):
 *   philox / uniform ........ published Random123 known-answer vectors
 *   li2 ..................... scipy spence, closed values Li2(-1), Li2(1/2)
 *   gauss_legendre / psi .... polynomial exactness, orthonormality, numpy leggauss (up to 31
 *                             nodes and degree 30, the stochastic-Galerkin error study)
 *   observe_at .............. Galerkin mean/variance vs brute-force z sampling (tiny ensembles)
 *   rates ................... 2-D quadrature of the transition rates S, detailed balance
 *   edge_T / edge angle ..... T(0,c)=2pi, Bessel closed form, KS vs the density
 *   AC / K / OP angles ...... KS vs the CDFs (th +- sin th)/2pi, uniform
 *   fd sampling, density .... numerical quadrature of eps*FD(eps), T->0 limit
 *   drift ................... closed form k(t) = k(0) - (e/hbar) E t (mechanisms off)
 *   histogram / Nmax ........ numpy histogram of floor((k + Lk)/dk) of the node values
 *                             reconstructed with numpy's Legendre basis; its maximum
 *   Pauli test .............. planted histograms: saturated (every in-grid candidate rejected,
 *                             the particles only drift), empty (= the run without the test,
 *                             bit for bit), uniform f (rejected share = f, binomial), the
 *                             current-maximum normaliser, a half-plane histogram under a strong
 *                             field (accepted states end left of -(e/hbar) E dt: the look-up
 *                             moves with the drift, Lie and Strang), zero outside the grid
 *   full step ............... conservation, positivity, zero-field symmetry, stationarity of the
 *                             Maxwellian, collision-count statistics, brute-force z sampling of
 *                             the Galerkin mean/variance, degenerate interval = deterministic run.
 *   Strang splitting ........ without the Pauli test: the Lie run from the initial state moved by
 *                             half a drift, moved back by half a drift (the two schemes differ by
 *                             that conjugation); ballistic closed form; second-order agreement
 *                             of the drift-only observables.
 *                             Beyond these properties, the scattering trajectory itself is
 *                             "parity unpinned" (no published trajectory exists).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------------ */
/* Physical constants (CODATA 2018) and Table 1 of the paper (Sec. 5).                         */
/* ------------------------------------------------------------------------------------------ */
#define HBAR_EVS 6.582119569e-16   /* eV s   */
#define Q_E 1.602176634e-19        /* C      */
#define KB_EVK 8.617333262e-5      /* eV / K */

/* Table 1 (Sec. 5), cgs units as printed */
#define T1_VF_CMS 1.0e8            /* Fermi velocity, cm/s            */
#define T1_SIGMA_GCM2 7.6e-8       /* areal density, g/cm^2           */
#define T1_HW_O_EV 0.1646          /* optical phonon energy, eV        */
#define T1_HW_K_EV 0.124           /* K phonon energy, eV              */
#define T1_VP_CMS 2.0e6            /* sound speed, cm/s                */
#define T1_DAC_EV 6.8              /* acoustic deformation potential   */
#define T1_DO_EVCM 1.0e9           /* optical coupling, eV/cm          */
#define T1_DK_EVCM 3.5e8           /* K-phonon coupling, eV/cm         */
#define T1_NI_CM 1.0e4             /* edge defect density, 1/cm        */
#define T1_V0_EVCM2 4.56e-14       /* edge potential, eV cm^2          */
#define T1_A_CM 1.0e-8             /* edge range, cm                   */

/* mechanism bits, in the order of the rate vector Lambda of Eq. (20) */
#define ORC_AC 1u
#define ORC_OPM 2u
#define ORC_OPP 4u
#define ORC_KM 8u
#define ORC_KP 16u
#define ORC_EDGE 32u

/* Pauli normalisation readings */
#define ORC_PAULI_INITIAL_MAX 0
#define ORC_PAULI_CURRENT_MAX 1
#define ORC_PAULI_OFF 2
/* final-state readings for OP/K */
#define ORC_FS_PAPER 0
#define ORC_FS_EXACT_ENERGY 1
/* how the band minimum depends on z: directly (an interval of eps0), or through the ribbon
   width, eps0 = pi hbar vF / W (Sec. 2), with W spread over an interval (Test 2) */
#define ORC_EPS0_AFFINE 0
#define ORC_EPS0_WIDTH 1
/* Time splitting of Sec. 3: Lie, f^{n+1} = C_dt(T_dt(f^n)) (the paper's scheme), or Strang,
 * f^{n+1} = T_{dt/2}(C_dt(T_{dt/2}(f^n))), the second-order splitting the paper names as possible. */
#define ORC_SPLIT_LIE 0
#define ORC_SPLIT_STRANG 1

typedef struct {
    double T_K;               /* lattice = initial Fermi-Dirac temperature */
    double eps_F;             /* Fermi level, eV */
    double eps0_lo, eps0_hi;  /* conduction-band minimum hbar vF pi / W, eV (lo==hi: deterministic) */
    double Ex_lo, Ex_hi;      /* field along x, V/cm (lo==hi: deterministic) */
    uint32_t mech_mask;       /* ORC_AC | ... ; 0 = ballistic */
    double alpha;             /* self-scattering tuning, Eq. (19) */
    int32_t Nk;               /* cells per direction of the k grid */
    double Lk_hvF;            /* L_k * hbar vF, eV */
    int32_t M;                /* gPC degree (total degree in 2-D) */
    int32_t Q1;               /* Gauss-Legendre nodes per random dimension */
    int64_t N;                /* particles */
    double dt_fs;             /* time step */
    uint64_t seed;            /* Philox key */
    uint32_t stream_id;       /* second Philox counter word (ensemble id) */
    int32_t pauli_norm;       /* ORC_PAULI_* */
    int32_t final_state;      /* ORC_FS_* */
    int32_t n_theta;          /* trapezoid points of the edge integral (Appendix A) */
    int32_t max_coll;         /* safety cap of collisions per particle and step */
    int32_t eps0_law;         /* ORC_EPS0_AFFINE or ORC_EPS0_WIDTH */
    double W_lo, W_hi;        /* ribbon width interval, nm (ORC_EPS0_WIDTH) */
    int32_t splitting;        /* ORC_SPLIT_LIE (the paper's scheme) or ORC_SPLIT_STRANG */
} orc_cfg;

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",  */
/* SC'11).  Written from the published definition: ten rounds of two 32x32->64 multiplies    */
/* with a Weyl-sequence key schedule.                                                         */
/* ------------------------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1): odd multiples of 2^-24.  Exactly representable in FP32 and FP64. */
double orc_u01(uint32_t x)
{
    return (double)((x >> 8) | 1u) * (1.0 / 16777216.0);
}

/* The four uniforms (xi, s, eta, u_theta) of collision attempt c of particle i in step n. */
static void orc_draw(const orc_cfg *cfg, int64_t i, int64_t n, uint32_t c, double u[4])
{
    uint32_t ctr[4] = {(uint32_t)i, cfg->stream_id, (uint32_t)n, c};
    uint32_t key[2] = {(uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32)};
    uint32_t o[4];
    orc_philox(ctr, key, o);
    for (int j = 0; j < 4; ++j) u[j] = orc_u01(o[j]);
}

#define ORC_INIT_PURPOSE 0x10000u

/* ------------------------------------------------------------------------------------------ */
/* Dilogarithm Li2(x) for x <= 0, used by the closed-form Fermi-Dirac integrals.              */
/* Series for 0 <= y <= 1/2, Landen's identity for -1 <= x < 0, inversion for x < -1.         */
/* ------------------------------------------------------------------------------------------ */
static double li2_series(double y)
{
    double s = 0.0, p = 1.0;
    for (int k = 1; k < 200; ++k) {
        p *= y;
        double t = p / ((double)k * (double)k);
        s += t;
        if (t < 1e-18 * fabs(s)) break;
    }
    return s;
}

double orc_li2_neg(double x)
{
    if (x == 0.0) return 0.0;
    if (x < -1.0) {
        double l = log(-x);
        return -ORC_PI * ORC_PI / 6.0 - 0.5 * l * l - orc_li2_neg(1.0 / x);
    }
    double y = x / (x - 1.0);
    double l = log1p(-x);
    return -li2_series(y) - 0.5 * l * l;
}

/* ln(1 + e^{-t}), without overflow */
static double ln1pexpm(double t)
{
    if (t > 0) return log1p(exp(-t));
    return -t + log1p(exp(t));
}

/* ------------------------------------------------------------------------------------------ */
/* Fermi-Dirac initial state (Sec. 2).  In polar coordinates the particle density in energy   */
/* is proportional to eps * FD(eps) on [eps0, inf) (Jacobian eps/(hbar vF)^2, Appendix A),    */
/* with a uniform angle.                                                                      */
/*   G(a,b) = int_a^b x/(1+exp((x-mu)/kT)) dx in closed form with                              */
/*   int 1/(1+e^t) dt = -ln(1+e^-t),  int t/(1+e^t) dt = -t ln(1+e^-t) + Li2(-e^-t).           */
/* ------------------------------------------------------------------------------------------ */
static double fd_A(double t) { return -ln1pexpm(t); }
static double fd_B(double t)
{
    double l = ln1pexpm(t);
    double li = (t > -700.0) ? orc_li2_neg(-exp(-t)) : -ORC_PI * ORC_PI / 6.0 - 0.5 * t * t;
    return -t * l + li;
}

/* upper tail int_e^inf x FD(x) dx */
static double fd_tail(double e, double mu, double kT)
{
    double b = (e - mu) / kT;
    return -kT * (mu * fd_A(b) + kT * fd_B(b));
}

/* int_{eps0}^{inf} x FD(x) dx */
double orc_fd_total(double eps0, double mu, double kT) { return fd_tail(eps0, mu, kT); }

/* inverse CDF of eps*FD(eps) on [eps0, inf) by bisection (reading: the paper does not say how
 * the initial particles are sampled; the inverse CDF with one uniform shared by all z keeps
 * k_i(z) continuous in z). */
double orc_fd_sample(double eps0, double mu, double kT, double u)
{
    double tot = orc_fd_total(eps0, mu, kT);
    double lo = eps0, hi = (mu > eps0 ? mu : eps0) + 80.0 * kT;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        int below; /* F(mid) < u ? */
        if (u < 0.5) {
            double g = tot - fd_tail(mid, mu, kT); /* int_eps0^mid */
            below = (g < u * tot);
        } else {
            double gc = fd_tail(mid, mu, kT);
            below = (gc > (1.0 - u) * tot);
        }
        if (below) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------------------------ */
/* gPC tables (Sec. 4.1, Eq. (23)): orthonormal Legendre polynomials for uniform z, Gauss     */
/* quadrature for the integrals over I_z (Eqs. (29),(30), the forcing term, the QoI).         */
/* ------------------------------------------------------------------------------------------ */

/* Legendre P_n(z) and P_{n-1}(z) by the three-term recurrence */
static void leg_pn(int n, double z, double *pn, double *pnm1)
{
    double p0 = 1.0, p1 = z;
    if (n == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
    }
    *pn = p1; *pnm1 = p0;
}

/* Gauss-Legendre nodes on [-1,1] (ascending) by Newton on P_n; weights 2/((1-z^2) P_n'^2)
 * divided by 2 so that they sum to 1 (uniform density p(z) = 1/2). */
void orc_gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5)), pn, pm1, dp;
        for (int it = 0; it < 100; ++it) {
            leg_pn(n, z, &pn, &pm1);
            dp = n * (z * pn - pm1) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        leg_pn(n, z, &pn, &pm1);
        dp = n * (z * pn - pm1) / (z * z - 1.0);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* orthonormal Legendre sqrt(2h+1) P_h(z), h = 0..M */
static void legendre_on(int M, double z, double *out)
{
    double p0 = 1.0, p1 = z;
    out[0] = 1.0;
    if (M >= 1) out[1] = sqrt(3.0) * z;
    for (int h = 2; h <= M; ++h) {
        double p2 = ((2.0 * h - 1.0) * z * p1 - (h - 1.0) * p0) / h;
        p0 = p1; p1 = p2;
        out[h] = sqrt(2.0 * h + 1.0) * p2;
    }
}

/* is the band minimum uncertain? (its own interval, or the width's) */
static int orc_eps_random(const orc_cfg *c)
{
    if (c->eps0_law == ORC_EPS0_WIDTH) return c->W_lo != c->W_hi;
    return c->eps0_lo != c->eps0_hi;
}

/* band minimum for the band-minimum variable z1 in [-1,1] (z ~ U maps affinely onto the
   interval of the uncertain quantity); with the width law the affine quantity is W and
   eps0 = pi hbar vF / W, the lowest transverse subband of a ribbon of width W (Sec. 2) */
static double orc_band_min(const orc_cfg *c, double hvF, double z1)
{
    int rnd = orc_eps_random(c);
    if (c->eps0_law == ORC_EPS0_WIDTH) {
        double W = rnd ? c->W_lo + 0.5 * (c->W_hi - c->W_lo) * (z1 + 1.0) : c->W_lo;
        return ORC_PI * hvF / W;
    }
    return rnd ? c->eps0_lo + 0.5 * (c->eps0_hi - c->eps0_lo) * (z1 + 1.0) : c->eps0_lo;
}

/* number of random dimensions, basis size P, node count Q */
static int orc_dims(const orc_cfg *c, int *P, int *Q)
{
    int d = orc_eps_random(c) + (c->Ex_lo != c->Ex_hi);
    if (d == 0) { *P = 1; *Q = 1; }
    else if (d == 1) { *P = c->M + 1; *Q = c->Q1; }
    else { *P = (c->M + 1) * (c->M + 2) / 2; *Q = c->Q1 * c->Q1; }
    return d;
}

/* Basis functions at a point z (d components in [-1,1]).  2-D basis: total degree <= M in
 * graded order: for t = 0..M, for j = 0..t: (deg in z_1, deg in z_2) = (t-j, j).  z_1 is the
 * band-minimum variable, z_2 the field variable; in 1-D the single z is whichever is random. */
void orc_psi_at(const orc_cfg *c, const double *z, double *psi)
{
    int P, Q;
    int d = orc_dims(c, &P, &Q);
    if (d == 0) { psi[0] = 1.0; return; }
    double a[64], b[64];
    if (d == 1) { legendre_on(c->M, z[0], psi); return; }
    legendre_on(c->M, z[0], a);
    legendre_on(c->M, z[1], b);
    int h = 0;
    for (int t = 0; t <= c->M; ++t)
        for (int j = 0; j <= t; ++j) psi[h++] = a[t - j] * b[j];
}

/* ------------------------------------------------------------------------------------------ */
/* Oracle state                                                                               */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    orc_cfg cfg;
    int d, P, Q;
    /* constants in eV, fs, nm */
    double hvF;        /* hbar vF, eV nm */
    double hbar_fs;    /* hbar, eV fs */
    double kT;
    double Cac, CO, CK, nO, nK, hwO, hwK, Cedg; /* rates in 1/fs */
    double a_nm;
    double Lk, dk;
    /* tables */
    double *zq;        /* [Q][d] nodes in [-1,1]^d */
    double *wq;        /* [Q] */
    double *psi;       /* [Q][P] */
    double *eps0q, *Exq, *dq, *nq; /* per node: band minimum, field, drift per step (nm^-1), density m^-2 */
    double *dhat;      /* [P] drift of the x coefficients per step (sG forcing term, Sec. 4.1) */
    /* particles */
    double *khat;      /* [2][P][N] */
    uint32_t *H;       /* [Q][Nk*Nk] histogram of the current state (Eqs. (24)) */
    uint32_t *Nmax;    /* [Q] normaliser of the Pauli test */
    int64_t *cellbuf;  /* [N][Q] scratch */
    int64_t step;
    int sampled;       /* 1 if the state came from the Fermi-Dirac sampling of orc_init */
    /* counters */
    int64_t n_coll_attempts, n_real, n_rejected, n_capped, n_out_of_grid;
    /* time series */
    int64_t T_out, T_cap;
    double *t_fs;      /* [T] */
    double *nodes;     /* [T][Q][4]: Vx, Vy, E, Jx */
    double *mean;      /* [T][4] */
    double *var;       /* [T][4] */
} orc_state;

/* ------------------------------------------------------------------------------------------ */
/* Scattering rates, Appendix A (final closed forms).  Returns the six rates of Eq. (20)     */
/* (without the self-scattering entry) in 1/fs.                                               */
/* ------------------------------------------------------------------------------------------ */

/* T(|k|, cos th) = int_0^{2pi} exp(-2 |k|^2 a^2 (cos th' - cos th)^2) d th' by the trapezoid  */
/* rule with n points (Appendix A: "computed numerically by the trapezoidal rule").           */
double orc_edge_T(double beta, double c, int n)
{
    double h = 2.0 * ORC_PI / n, s = 0.0;
    for (int j = 0; j < n; ++j) {
        double x = cos(j * h) - c;
        s += exp(-beta * x * x);
    }
    return h * s;
}

static void orc_rates_node(const orc_state *S, double kx, double ky, double eps0, double *g)
{
    const orc_cfg *c = &S->cfg;
    double kk = kx * kx + ky * ky;
    double km = sqrt(kk);
    double eps = sqrt(S->hvF * S->hvF * kk + eps0 * eps0); /* dispersion, Sec. 2 */
    for (int m = 0; m < 6; ++m) g[m] = 0.0;
    /* H(eps - eps0) of the AC and edge rates is 1 for every state (eps >= eps0). */
    if (c->mech_mask & ORC_AC) g[0] = S->Cac * eps;
    if ((c->mech_mask & ORC_OPM) && (eps - S->hwO - eps0 > 0.0)) g[1] = S->CO * (S->nO + 1.0) * (eps - S->hwO);
    if ((c->mech_mask & ORC_OPP) && (eps + S->hwO - eps0 > 0.0)) g[2] = S->CO * S->nO * (eps + S->hwO);
    if ((c->mech_mask & ORC_KM) && (eps - S->hwK - eps0 > 0.0)) g[3] = S->CK * (S->nK + 1.0) * (eps - S->hwK);
    if ((c->mech_mask & ORC_KP) && (eps + S->hwK - eps0 > 0.0)) g[4] = S->CK * S->nK * (eps + S->hwK);
    if (c->mech_mask & ORC_EDGE) {
        double cth = (km > 0.0) ? kx / km : 1.0;
        double beta = 2.0 * kk * S->a_nm * S->a_nm;
        /* 1/W = eps0 / (pi hbar vF) */
        g[5] = S->Cedg * eps0 * eps * orc_edge_T(beta, cth, c->n_theta);
    }
}

/* public wrapper for tests: rates at one state, 1/fs */
void orc_rates(const void *st, double kx, double ky, double eps0, double *g6)
{
    orc_rates_node((const orc_state *)st, kx, ky, eps0, g6);
}

/* ------------------------------------------------------------------------------------------ */
/* Angle samplers (Sec. 3, final states h^1..h^6).  One uniform u per collision, shared by     */
/* every node z (Sec. 4.1: the AC, OP and K angles have deterministic distributions).         */
/* ------------------------------------------------------------------------------------------ */

/* theta ~ (1 + cos th) on [0, 2pi): CDF (th + sin th)/(2pi) = u, solved by bisection */
double orc_angle_ac(double u)
{
    double lo = 0.0, hi = 2.0 * ORC_PI, t = 2.0 * ORC_PI * u;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (mid + sin(mid) < t) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* theta ~ (1 - cos th) on [0, 2pi): CDF (th - sin th)/(2pi) = u */
double orc_angle_k(double u)
{
    double lo = 0.0, hi = 2.0 * ORC_PI, t = 2.0 * ORC_PI * u;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (mid - sin(mid) < t) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Edge final angle (absolute): density exp(-beta (cos th_in - cos th')^2) on [0,2pi).
 * Reading: the density is written in the absolute final angle th' (it is the matrix element
 * of Eq. (9) as a function of k_x - k_x'), so th' is used as the absolute angle.  Sampled by
 * inverting the trapezoid CDF on the same n-point grid that gives T, linear between points. */
double orc_angle_edge(double beta, double cth, double u, int n)
{
    double h = 2.0 * ORC_PI / n;
    double *C = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double gprev = exp(-beta * (1.0 - cth) * (1.0 - cth));
    C[0] = 0.0;
    for (int j = 1; j <= n; ++j) {
        double x = cos(j * h) - cth;
        double g = exp(-beta * x * x);
        C[j] = C[j - 1] + 0.5 * h * (gprev + g);
        gprev = g;
    }
    double target = u * C[n];
    int j = 0;
    while (j < n - 1 && C[j + 1] <= target) ++j;
    double th = (j + (target - C[j]) / (C[j + 1] - C[j])) * h;
    free(C);
    return th;
}

/* ------------------------------------------------------------------------------------------ */
/* Creation: constants, tables.                                                               */
/* ------------------------------------------------------------------------------------------ */
void *orc_create(const orc_cfg *cfg)
{
    orc_state *S = (orc_state *)calloc(1, sizeof(orc_state));
    S->cfg = *cfg;
    S->d = orc_dims(cfg, &S->P, &S->Q);
    int P = S->P, Q = S->Q, d = S->d;

    /* --- constants (SI first, then eV / fs / nm) --- */
    double hbar = HBAR_EVS * Q_E;                    /* J s */
    double vF = T1_VF_CMS * 1e-2;                    /* m/s */
    double sig = T1_SIGMA_GCM2 * 1e-3 / 1e-4;        /* kg/m^2 */
    double vp = T1_VP_CMS * 1e-2;
    double kT_eV = KB_EVK * cfg->T_K;
    double kT = kT_eV * Q_E;
    double Dac = T1_DAC_EV * Q_E;
    double DO = T1_DO_EVCM * Q_E * 1e2;              /* J/m */
    double DK = T1_DK_EVCM * Q_E * 1e2;
    double wO = T1_HW_O_EV / HBAR_EVS, wK = T1_HW_K_EV / HBAR_EVS;
    double Ni = T1_NI_CM * 1e2;                      /* 1/m */
    double V0 = T1_V0_EVCM2 * Q_E * 1e-4;            /* J m^2 */
    S->hbar_fs = HBAR_EVS * 1e15;
    S->hvF = HBAR_EVS * (T1_VF_CMS * 1e7);           /* eV nm (vF in nm/s) */
    S->kT = kT_eV;
    S->hwO = T1_HW_O_EV;
    S->hwK = T1_HW_K_EV;
    /* Bose-Einstein occupations at T_L (Sec. 2) */
    S->nO = 1.0 / (exp(T1_HW_O_EV / kT_eV) - 1.0);
    S->nK = 1.0 / (exp(T1_HW_K_EV / kT_eV) - 1.0);
    /* Appendix A: Gamma_ac = Dac^2 kB T / (4 hbar^3 vF^2 sigma vp^2) eps  -> [1/s per J] */
    double Cac_SI = Dac * Dac * kT / (4.0 * hbar * hbar * hbar * vF * vF * sig * vp * vp);
    /* Gamma_O = DO^2/(hbar^2 vF^2 sigma wO) [...]  (energies in J) */
    double CO_SI = DO * DO / (hbar * hbar * vF * vF * sig * wO);
    double CK_SI = DK * DK / (hbar * hbar * vF * vF * sig * wK);
    /* Gamma_edg = 1/(hbar vF)^2 * Ni V0^2/(2 pi hbar W) * eps * T, with 1/W = eps0/(pi hbar vF) */
    double hvF_SI = hbar * vF;
    double Cedg_SI = Ni * V0 * V0 / (2.0 * ORC_PI * ORC_PI * hbar * hvF_SI * hvF_SI * hvF_SI);
    /* to 1/fs per eV (and per eV^2 for the edge constant) */
    S->Cac = Cac_SI * Q_E * 1e-15;
    S->CO = CO_SI * Q_E * 1e-15;
    S->CK = CK_SI * Q_E * 1e-15;
    S->Cedg = Cedg_SI * Q_E * Q_E * 1e-15;
    S->a_nm = T1_A_CM * 1e7;
    S->Lk = cfg->Lk_hvF / S->hvF;
    S->dk = 2.0 * S->Lk / cfg->Nk;

    /* --- quadrature nodes (tensor Gauss-Legendre), basis values --- */
    S->zq = (double *)calloc((size_t)Q * (d > 0 ? d : 1), sizeof(double));
    S->wq = (double *)calloc((size_t)Q, sizeof(double));
    S->psi = (double *)calloc((size_t)Q * P, sizeof(double));
    S->eps0q = (double *)calloc((size_t)Q, sizeof(double));
    S->Exq = (double *)calloc((size_t)Q, sizeof(double));
    S->dq = (double *)calloc((size_t)Q, sizeof(double));
    S->nq = (double *)calloc((size_t)Q, sizeof(double));
    S->dhat = (double *)calloc((size_t)P, sizeof(double));
    double x1[64], w1[64];
    if (d == 0) { S->wq[0] = 1.0; }
    else {
        orc_gauss_legendre(cfg->Q1, x1, w1);
        if (d == 1) {
            for (int q = 0; q < Q; ++q) { S->zq[q] = x1[q]; S->wq[q] = w1[q]; }
        } else {
            for (int q1 = 0; q1 < cfg->Q1; ++q1)
                for (int q2 = 0; q2 < cfg->Q1; ++q2) {
                    int q = q1 * cfg->Q1 + q2;
                    S->zq[2 * q] = x1[q1]; S->zq[2 * q + 1] = x1[q2];
                    S->wq[q] = w1[q1] * w1[q2];
                }
        }
    }
    for (int q = 0; q < Q; ++q) {
        double z1 = 0.0, z2 = 0.0;
        int eps_random = orc_eps_random(cfg), E_random = (cfg->Ex_lo != cfg->Ex_hi);
        if (d == 1) { if (eps_random) z1 = S->zq[q]; else z2 = S->zq[q]; }
        if (d == 2) { z1 = S->zq[2 * q]; z2 = S->zq[2 * q + 1]; }
        /* maps of z in [-1,1] onto the parameters (z ~ U) */
        S->eps0q[q] = orc_band_min(cfg, S->hvF, z1);
        S->Exq[q] = E_random ? cfg->Ex_lo + 0.5 * (cfg->Ex_hi - cfg->Ex_lo) * (z2 + 1.0) : cfg->Ex_lo;
        /* drift of Eq. (17): (e/hbar) E dt, E in V/cm -> eV/nm is 1e-7 */
        S->dq[q] = S->Exq[q] * 1e-7 * cfg->dt_fs / S->hbar_fs;
        /* density, Eq. (13)/(31): gs gv/(2pi)^2 * 2pi/(hbar vF)^2 * int eps FD(eps) deps */
        double nn = 2.0 / (ORC_PI * S->hvF * S->hvF) * orc_fd_total(S->eps0q[q], cfg->eps_F, kT_eV);
        S->nq[q] = nn * 1e18;
        orc_psi_at(cfg, (d > 0) ? &S->zq[q * d] : NULL, &S->psi[q * P]);
    }
    /* sG forcing term (Sec. 4.1): dhat_h = int (e/hbar) E(z) dt Psi_h(z) p(z) dz, by quadrature */
    for (int h = 0; h < P; ++h) {
        double s = 0.0;
        for (int q = 0; q < Q; ++q) s += S->wq[q] * S->dq[q] * S->psi[q * P + h];
        S->dhat[h] = s;
    }

    S->khat = (double *)calloc((size_t)2 * P * cfg->N, sizeof(double));
    S->H = (uint32_t *)calloc((size_t)Q * cfg->Nk * cfg->Nk, sizeof(uint32_t));
    S->Nmax = (uint32_t *)calloc((size_t)Q, sizeof(uint32_t));
    S->cellbuf = (int64_t *)calloc((size_t)cfg->N * Q + 1, sizeof(int64_t));
    S->T_cap = 16;
    S->t_fs = (double *)calloc((size_t)S->T_cap, sizeof(double));
    S->nodes = (double *)calloc((size_t)S->T_cap * Q * 4, sizeof(double));
    S->mean = (double *)calloc((size_t)S->T_cap * 4, sizeof(double));
    S->var = (double *)calloc((size_t)S->T_cap * 4, sizeof(double));
    return S;
}

void orc_destroy(void *st)
{
    orc_state *S = (orc_state *)st;
    if (!S) return;
    free(S->zq); free(S->wq); free(S->psi); free(S->eps0q); free(S->Exq); free(S->dq); free(S->nq);
    free(S->dhat); free(S->khat); free(S->H); free(S->Nmax); free(S->cellbuf);
    free(S->t_fs); free(S->nodes); free(S->mean); free(S->var);
    free(S);
}

/* ------------------------------------------------------------------------------------------ */
/* Reconstruction and projection (Eq. (23) and the sG projection of Sec. 4.1).               */
/* ------------------------------------------------------------------------------------------ */
static inline double khat_at(const orc_state *S, int c, int h, int64_t i)
{
    return S->khat[((size_t)c * S->P + h) * S->cfg.N + i];
}

static void recon_particle(const orc_state *S, int64_t i, double *kx, double *ky)
{
    for (int q = 0; q < S->Q; ++q) {
        double sx = 0.0, sy = 0.0;
        for (int h = 0; h < S->P; ++h) {
            sx += khat_at(S, 0, h, i) * S->psi[q * S->P + h];
            sy += khat_at(S, 1, h, i) * S->psi[q * S->P + h];
        }
        kx[q] = sx; ky[q] = sy;
    }
}

static void project_particle(orc_state *S, int64_t i, const double *kx, const double *ky)
{
    for (int h = 0; h < S->P; ++h) {
        double sx = 0.0, sy = 0.0;
        for (int q = 0; q < S->Q; ++q) {
            double wp = S->wq[q] * S->psi[q * S->P + h];
            sx += wp * kx[q];
            sy += wp * ky[q];
        }
        S->khat[((size_t)0 * S->P + h) * S->cfg.N + i] = sx;
        S->khat[((size_t)1 * S->P + h) * S->cfg.N + i] = sy;
    }
}

/* cell index of a wave-vector on the fixed grid [-Lk,Lk]^2 (Sec. 3), -1 outside */
static int64_t cell_of(const orc_state *S, double kx, double ky)
{
    double fr = floor((kx + S->Lk) / S->dk);
    double fl = floor((ky + S->Lk) / S->dk);
    int Nk = S->cfg.Nk;
    if (fr < 0.0 || fl < 0.0 || fr >= Nk || fl >= Nk) return -1;
    return (int64_t)fr * Nk + (int64_t)fl;
}

/* Histogram N_rl(z_q) of the reconstructed particles, Eq. (24); returns out-of-grid count. */
static int64_t build_hist(orc_state *S)
{
    int Q = S->Q;
    int64_t N = S->cfg.N, cells = (int64_t)S->cfg.Nk * S->cfg.Nk;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double kx[1296], ky[1296];
        recon_particle(S, i, kx, ky);
        for (int q = 0; q < Q; ++q) S->cellbuf[i * Q + q] = cell_of(S, kx[q], ky[q]);
    }
    memset(S->H, 0, sizeof(uint32_t) * (size_t)Q * cells);
    int64_t out = 0;
    for (int64_t i = 0; i < N; ++i)
        for (int q = 0; q < Q; ++q) {
            int64_t c = S->cellbuf[i * Q + q];
            if (c < 0) { ++out; continue; }
            S->H[(size_t)q * cells + c] += 1;
        }
    return out;
}

static void hist_max(const orc_state *S, uint32_t *mx)
{
    int64_t cells = (int64_t)S->cfg.Nk * S->cfg.Nk;
    for (int q = 0; q < S->Q; ++q) {
        uint32_t m = 0;
        for (int64_t c = 0; c < cells; ++c) if (S->H[(size_t)q * cells + c] > m) m = S->H[(size_t)q * cells + c];
        mx[q] = m;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Observables (Eqs. (13)-(16), per node Eqs. (35)-(37)) and QoI (Sec. 4.2).                  */
/* Reading for the variance (the paper defines only the expectation): Var = E[O^2] - E[O]^2   */
/* with the same quadrature.                                                                  */
/* ------------------------------------------------------------------------------------------ */
static void record_moments(orc_state *S)
{
    int Q = S->Q;
    int64_t N = S->cfg.N;
    if (S->T_out == S->T_cap) {
        S->T_cap *= 2;
        S->t_fs = (double *)realloc(S->t_fs, sizeof(double) * S->T_cap);
        S->nodes = (double *)realloc(S->nodes, sizeof(double) * S->T_cap * Q * 4);
        S->mean = (double *)realloc(S->mean, sizeof(double) * S->T_cap * 4);
        S->var = (double *)realloc(S->var, sizeof(double) * S->T_cap * 4);
    }
    int64_t t = S->T_out;
    double *nd = &S->nodes[(size_t)t * Q * 4];
    for (int q = 0; q < Q; ++q) {
        double svx = 0.0, svy = 0.0, se = 0.0;
        double e0 = S->eps0q[q];
        for (int64_t i = 0; i < N; ++i) {
            double kx = 0.0, ky = 0.0;
            for (int h = 0; h < S->P; ++h) {
                kx += khat_at(S, 0, h, i) * S->psi[q * S->P + h];
                ky += khat_at(S, 1, h, i) * S->psi[q * S->P + h];
            }
            double eps = sqrt(S->hvF * S->hvF * (kx * kx + ky * ky) + e0 * e0);
            /* group velocity v = (1/hbar) grad eps = vF (hbar vF k)/eps, in units of vF */
            svx += S->hvF * kx / eps;
            svy += S->hvF * ky / eps;
            se += eps;
        }
        double vF_ms = T1_VF_CMS * 1e-2;
        double Vx = svx / (double)N * vF_ms, Vy = svy / (double)N * vF_ms, E = se / (double)N;
        nd[q * 4 + 0] = Vx;
        nd[q * 4 + 1] = Vy;
        nd[q * 4 + 2] = E;
        nd[q * 4 + 3] = -Q_E * S->nq[q] * Vx; /* J = -e n V */
    }
    for (int o = 0; o < 4; ++o) {
        double m = 0.0, m2 = 0.0;
        for (int q = 0; q < Q; ++q) { m += S->wq[q] * nd[q * 4 + o]; m2 += S->wq[q] * nd[q * 4 + o] * nd[q * 4 + o]; }
        S->mean[t * 4 + o] = m;
        S->var[t * 4 + o] = m2 - m * m;
    }
    S->t_fs[t] = S->step * S->cfg.dt_fs;
    S->T_out++;
}

/* ------------------------------------------------------------------------------------------ */
/* Initial state: Fermi-Dirac sampling per node with shared uniforms, then projection.        */
/* h_khat (nullable) injects a given state [2][P][N] instead.                                  */
/* ------------------------------------------------------------------------------------------ */
int orc_init(void *st, const double *h_khat)
{
    orc_state *S = (orc_state *)st;
    const orc_cfg *c = &S->cfg;
    int P = S->P, Q = S->Q;
    int64_t N = c->N;
    S->sampled = (h_khat == NULL);
    if (h_khat) memcpy(S->khat, h_khat, sizeof(double) * 2 * (size_t)P * N);
    else {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            uint32_t ctr[4] = {(uint32_t)i, c->stream_id, 0u, ORC_INIT_PURPOSE};
            uint32_t key[2] = {(uint32_t)c->seed, (uint32_t)(c->seed >> 32)};
            uint32_t o[4];
            orc_philox(ctr, key, o);
            double ue = orc_u01(o[0]), uth = orc_u01(o[1]);
            double kx[1296], ky[1296];
            double th = 2.0 * ORC_PI * uth;
            for (int q = 0; q < Q; ++q) {
                double e0 = S->eps0q[q];
                double eps = orc_fd_sample(e0, c->eps_F, S->kT, ue);
                double r = eps * eps - e0 * e0;
                double km = (r > 0.0) ? sqrt(r) / S->hvF : 0.0;
                kx[q] = km * cos(th);
                ky[q] = km * sin(th);
            }
            project_particle(S, i, kx, ky);
        }
    }
    S->step = 0;
    S->T_out = 0;
    S->n_coll_attempts = S->n_real = S->n_rejected = S->n_capped = 0;
    S->n_out_of_grid = build_hist(S);
    hist_max(S, S->Nmax);
    record_moments(S);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* One collision event of one particle at one node: Eqs. (21),(22) for Q = 1, Eqs. (26),(27)   */
/* for the node z_q.  Selection by s against the cumulative rates normalised by Gt (reading:   */
/* Gt = max_z Gamma_tot(z); the self-scattering entry is Gt - sum Gamma(z_q), which keeps the */
/* sum of the entries equal to Gt at every node; half-open intervals [G^{l-1}, G^l)).          */
/* Returns 1 if the state changed.                                                            */
/* ------------------------------------------------------------------------------------------ */
static int collide_node(const orc_state *S, int q, double Gt, const double *g, double s, double eta,
                        double uth, const uint32_t *Hn, const uint32_t *Nmax, double shift, double *kx,
                        double *ky, int64_t *rej)
{
    const orc_cfg *c = &S->cfg;
    double target = s * Gt;
    double cum = 0.0;
    int l = 6; /* self scattering unless a real mechanism is hit */
    for (int m = 0; m < 6; ++m) {
        cum += g[m];
        if (target < cum) { l = m; break; }
    }
    if (l == 6) return 0; /* h^7 = identity */
    double k0x = *kx, k0y = *ky;
    double km = sqrt(k0x * k0x + k0y * k0y);
    double ci = (km > 0.0) ? k0x / km : 1.0, si = (km > 0.0) ? k0y / km : 0.0; /* theta_in; 0 if |k| = 0 */
    double e0 = S->eps0q[q];
    double nkx, nky;
    if (l == 5) {
        /* h^6: edge, absolute final angle, |k'| = |k| */
        double beta = 2.0 * km * km * S->a_nm * S->a_nm;
        double th = orc_angle_edge(beta, ci, uth, c->n_theta);
        nkx = km * cos(th);
        nky = km * sin(th);
    } else {
        double th, kn;
        if (l == 0) { th = orc_angle_ac(uth); kn = km; }
        else if (l == 1 || l == 2) {
            th = 2.0 * ORC_PI * uth;
            if (c->final_state == ORC_FS_EXACT_ENERGY) {
                double eps = sqrt(S->hvF * S->hvF * km * km + e0 * e0);
                double ep = (l == 1) ? eps - S->hwO : eps + S->hwO;
                kn = sqrt(ep * ep - e0 * e0) / S->hvF;
            } else kn = (l == 1) ? km - S->hwO / S->hvF : km + S->hwO / S->hvF; /* |k| -+ omega/vF */
        } else {
            th = orc_angle_k(uth);
            if (c->final_state == ORC_FS_EXACT_ENERGY) {
                double eps = sqrt(S->hvF * S->hvF * km * km + e0 * e0);
                double ep = (l == 3) ? eps - S->hwK : eps + S->hwK;
                kn = sqrt(ep * ep - e0 * e0) / S->hvF;
            } else kn = (l == 3) ? km - S->hwK / S->hvF : km + S->hwK / S->hvF;
        }
        /* rotation of the incoming direction by th (the matrices of h^1..h^5) */
        double ct = cos(th), st = sin(th);
        nkx = kn * (ct * ci - st * si);
        nky = kn * (st * ci + ct * si);
    }
    /* Pauli test against the previous-step distribution (Eq. (22)/(27)).  Reading: H^n was
     * counted on the fixed grid before the drift; the grid moves with the drift (Lagrangian,
     * Sec. 3), so the post-drift candidate k' is looked up at cell(k' + shift) with shift the
     * drift applied since H^n was counted: (e/hbar) E dt (Lie), half of it (Strang).  Cells
     * outside [-Lk,Lk]^2 have f = 0 (zero boundary condition). */
    if (c->pauli_norm != ORC_PAULI_OFF) {
        int64_t cell = cell_of(S, nkx + shift, nky);
        double f = 0.0;
        if (cell >= 0 && Nmax[q] > 0)
            f = (double)Hn[(size_t)q * c->Nk * c->Nk + cell] / (double)Nmax[q];
        if (f >= eta) { ++*rej; return 0; }
    }
    *kx = nkx; *ky = nky;
    return 1;
}

/* ------------------------------------------------------------------------------------------ */
/* One time step n -> n+1 for every particle: drift (Eq. (17) / sG forcing), then the          */
/* collision loop of Algorithm 1 / Algorithm 2 with the Pauli test against f^n.               */
/* Reading of the free flight: after every (real or self) collision the flight time is drawn  */
/* again from the current state (standard DSMC; a single draw per step would give an         */
/* unbounded number of collisions, since E[1/dt] diverges for exponential dt).                */
/* ------------------------------------------------------------------------------------------ */
/* One time step of particle i (drift, then the collision loop) against f^n = Hn. */
static void step_particle(orc_state *S, int64_t i, int64_t n, const uint32_t *Hn, const uint32_t *Nmx,
                          int64_t *att_, int64_t *real_, int64_t *rej_, int64_t *cap_)
{
    const orc_cfg *c = &S->cfg;
    int P = S->P, Q = S->Q;
    int64_t N = c->N;
    double kx[1296], ky[1296], g[1296 * 6];
    int64_t att = 0, real = 0, rej = 0, cap = 0;
    const int strang = (c->splitting == ORC_SPLIT_STRANG);
    /* drift of the coefficients: T_dt, or T_{dt/2} before the collisions (Strang) */
    for (int h = 0; h < P; ++h) S->khat[((size_t)0 * P + h) * N + i] -= strang ? 0.5 * S->dhat[h] : S->dhat[h];
    recon_particle(S, i, kx, ky);
    /* majorant: Gt = (1+alpha) max_q sum_nu Gamma_nu(k(z_q))  (Eq. (19), Eq. (25)) */
    double Gt = 0.0;
    for (int q = 0; q < Q; ++q) {
        orc_rates_node(S, kx[q], ky[q], S->eps0q[q], &g[q * 6]);
        double sg = 0.0;
        for (int m = 0; m < 6; ++m) sg += g[q * 6 + m];
        if (sg > Gt) Gt = sg;
    }
    Gt *= (1.0 + c->alpha);
    double tc = 0.0;
    uint32_t cc = 0;
    double u[4];
    orc_draw(c, i, n, cc, u);
    double dtc = (Gt > 0.0) ? -log(u[0]) / Gt : INFINITY; /* Eq. (18) / (25) */
    while (tc + dtc < c->dt_fs) {
        if ((int)cc >= c->max_coll) { ++cap; break; }
        ++att;
        int changed = 0;
        for (int q = 0; q < Q; ++q)
            changed |= collide_node(S, q, Gt, &g[q * 6], u[1], u[2], u[3], Hn, Nmx,
                                    strang ? 0.5 * S->dq[q] : S->dq[q], &kx[q], &ky[q], &rej);
        if (changed) ++real;
        /* collisional matrices K1 + K2 (Eqs. (28)-(30)): project the per-node result */
        project_particle(S, i, kx, ky);
        recon_particle(S, i, kx, ky);
        Gt = 0.0;
        for (int q = 0; q < Q; ++q) {
            orc_rates_node(S, kx[q], ky[q], S->eps0q[q], &g[q * 6]);
            double sg = 0.0;
            for (int m = 0; m < 6; ++m) sg += g[q * 6 + m];
            if (sg > Gt) Gt = sg;
        }
        Gt *= (1.0 + c->alpha);
        tc += dtc;
        ++cc;
        orc_draw(c, i, n, cc, u);
        dtc = (Gt > 0.0) ? -log(u[0]) / Gt : INFINITY;
    }
    /* Strang: the second half of the drift, T_{dt/2} after the collisions */
    if (strang)
        for (int h = 0; h < P; ++h) S->khat[((size_t)0 * P + h) * N + i] -= 0.5 * S->dhat[h];
    *att_ += att; *real_ += real; *rej_ += rej; *cap_ += cap;
}

static void step_once(orc_state *S)
{
    const orc_cfg *c = &S->cfg;
    int Q = S->Q;
    int64_t N = c->N;
    int64_t n = S->step;
    const uint32_t *Hn = S->H;
    uint32_t Nmx[1296];
    if (c->pauli_norm == ORC_PAULI_CURRENT_MAX) hist_max(S, Nmx);
    else memcpy(Nmx, S->Nmax, sizeof(uint32_t) * Q);
    int64_t att = 0, real = 0, rej = 0, cap = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : att, real, rej, cap)
    for (int64_t i = 0; i < N; ++i) step_particle(S, i, n, Hn, Nmx, &att, &real, &rej, &cap);
    S->n_coll_attempts += att;
    S->n_real += real;
    S->n_rejected += rej;
    S->n_capped += cap;
    S->step = n + 1;
    S->n_out_of_grid = build_hist(S); /* f^{n+1} for the next step */
}

/* Test hook: advance only the listed particles by one time step (index S->step) against the
 * current histogram; neither the step counter nor the histogram change.  The event counters
 * (attempts, real, rejected, capped) are added to. */
void orc_step_particles(void *st, const int64_t *idx, int64_t n)
{
    orc_state *S = (orc_state *)st;
    const orc_cfg *c = &S->cfg;
    uint32_t Nmx[1296];
    if (c->pauli_norm == ORC_PAULI_CURRENT_MAX) hist_max(S, Nmx);
    else memcpy(Nmx, S->Nmax, sizeof(uint32_t) * S->Q);
    int64_t att = 0, real = 0, rej = 0, cap = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : att, real, rej, cap)
    for (int64_t j = 0; j < n; ++j) step_particle(S, idx[j], S->step, S->H, Nmx, &att, &real, &rej, &cap);
    S->n_coll_attempts += att;
    S->n_real += real;
    S->n_rejected += rej;
    S->n_capped += cap;
}

/* Test hook: replace the histogram f^n [Q][Nk][Nk] that the next step's Pauli test reads. */
void orc_set_hist(void *st, const uint32_t *H)
{
    orc_state *S = (orc_state *)st;
    memcpy(S->H, H, sizeof(uint32_t) * (size_t)S->Q * S->cfg.Nk * S->cfg.Nk);
}

/* Test hook: set the step counter (the Philox counter word of the next step). */
void orc_set_step(void *st, int64_t step) { ((orc_state *)st)->step = step; }

/* Test hook: set the Pauli normaliser (e.g. that of another implementation's initial state). */
void orc_set_nmax(void *st, const uint32_t *nmax) { memcpy(((orc_state *)st)->Nmax, nmax, sizeof(uint32_t) * ((orc_state *)st)->Q); }

int orc_step(void *st, int64_t nsteps, int64_t moments_every)
{
    orc_state *S = (orc_state *)st;
    for (int64_t s = 0; s < nsteps; ++s) {
        step_once(S);
        if (moments_every > 0 && S->step % moments_every == 0) record_moments(S);
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Accessors                                                                                  */
/* ------------------------------------------------------------------------------------------ */
void orc_sizes(const void *st, int *d, int *P, int *Q)
{
    const orc_state *S = (const orc_state *)st;
    *d = S->d; *P = S->P; *Q = S->Q;
}

void orc_get_state(const void *st, double *khat)
{
    const orc_state *S = (const orc_state *)st;
    memcpy(khat, S->khat, sizeof(double) * 2 * (size_t)S->P * S->cfg.N);
}

void orc_set_state(void *st, const double *khat)
{
    orc_state *S = (orc_state *)st;
    memcpy(S->khat, khat, sizeof(double) * 2 * (size_t)S->P * S->cfg.N);
    S->n_out_of_grid = build_hist(S);
}

void orc_get_hist(const void *st, uint32_t *H, uint32_t *Nmax)
{
    const orc_state *S = (const orc_state *)st;
    memcpy(H, S->H, sizeof(uint32_t) * (size_t)S->Q * S->cfg.Nk * S->cfg.Nk);
    if (Nmax) memcpy(Nmax, S->Nmax, sizeof(uint32_t) * S->Q);
}

/* tables: zq [Q*d], wq [Q], psi [Q*P], eps0q, Exq, dq, nq [Q], dhat [P] */
void orc_get_tables(const void *st, double *zq, double *wq, double *psi, double *eps0q, double *Exq,
                    double *dq, double *nq, double *dhat)
{
    const orc_state *S = (const orc_state *)st;
    int Q = S->Q, P = S->P, d = S->d;
    if (zq && d > 0) memcpy(zq, S->zq, sizeof(double) * Q * d);
    if (wq) memcpy(wq, S->wq, sizeof(double) * Q);
    if (psi) memcpy(psi, S->psi, sizeof(double) * Q * P);
    if (eps0q) memcpy(eps0q, S->eps0q, sizeof(double) * Q);
    if (Exq) memcpy(Exq, S->Exq, sizeof(double) * Q);
    if (dq) memcpy(dq, S->dq, sizeof(double) * Q);
    if (nq) memcpy(nq, S->nq, sizeof(double) * Q);
    if (dhat) memcpy(dhat, S->dhat, sizeof(double) * P);
}

/* constants: [hvF, hbar_fs, kT, Cac, CO, CK, nO, nK, hwO, hwK, Cedg, a_nm, Lk, dk] */
void orc_get_constants(const void *st, double *out14)
{
    const orc_state *S = (const orc_state *)st;
    double v[14] = {S->hvF, S->hbar_fs, S->kT, S->Cac, S->CO, S->CK, S->nO, S->nK,
                    S->hwO, S->hwK, S->Cedg, S->a_nm, S->Lk, S->dk};
    memcpy(out14, v, sizeof(v));
}

/* counters: [attempts, real, rejected, capped, out_of_grid, step] */
void orc_get_counters(const void *st, int64_t *out6)
{
    const orc_state *S = (const orc_state *)st;
    out6[0] = S->n_coll_attempts; out6[1] = S->n_real; out6[2] = S->n_rejected;
    out6[3] = S->n_capped; out6[4] = S->n_out_of_grid; out6[5] = S->step;
}

int64_t orc_num_outputs(const void *st) { return ((const orc_state *)st)->T_out; }

void orc_get_moments(const void *st, double *t_fs, double *nodes, double *mean, double *var)
{
    const orc_state *S = (const orc_state *)st;
    int64_t T = S->T_out;
    if (t_fs) memcpy(t_fs, S->t_fs, sizeof(double) * T);
    if (nodes) memcpy(nodes, S->nodes, sizeof(double) * T * S->Q * 4);
    if (mean) memcpy(mean, S->mean, sizeof(double) * T * 4);
    if (var) memcpy(var, S->var, sizeof(double) * T * 4);
}

/* Distribution reconstructed at arbitrary z, Eq. (24): counts [nz][Nk*Nk] and max [nz].
 * z is [nz][d] in [-1,1]^d. */
void orc_reconstruct_f(const void *st, const double *z, int nz, uint32_t *hist, uint32_t *hmax)
{
    const orc_state *S = (const orc_state *)st;
    int P = S->P;
    int64_t N = S->cfg.N, cells = (int64_t)S->cfg.Nk * S->cfg.Nk;
    double psi[1296];
    for (int j = 0; j < nz; ++j) {
        orc_psi_at(&S->cfg, (S->d > 0) ? &z[j * S->d] : NULL, psi);
        uint32_t *Hj = &hist[(size_t)j * cells];
        memset(Hj, 0, sizeof(uint32_t) * cells);
        for (int64_t i = 0; i < N; ++i) {
            double kx = 0.0, ky = 0.0;
            for (int h = 0; h < P; ++h) { kx += khat_at(S, 0, h, i) * psi[h]; ky += khat_at(S, 1, h, i) * psi[h]; }
            int64_t c = cell_of(S, kx, ky);
            if (c >= 0) Hj[c] += 1;
        }
        uint32_t m = 0;
        for (int64_t c = 0; c < cells; ++c) if (Hj[c] > m) m = Hj[c];
        hmax[j] = m;
    }
}

/* Test hooks for the projection pins: project node values [Q] onto coefficients [P] and
 * reconstruct node values from coefficients, with the oracle's own tables. */
void orc_project_nodes(const void *st, const double *vq, double *vhat)
{
    const orc_state *S = (const orc_state *)st;
    for (int h = 0; h < S->P; ++h) {
        double s = 0.0;
        for (int q = 0; q < S->Q; ++q) s += S->wq[q] * S->psi[q * S->P + h] * vq[q];
        vhat[h] = s;
    }
}

void orc_recon_nodes(const void *st, const double *vhat, double *vq)
{
    const orc_state *S = (const orc_state *)st;
    for (int q = 0; q < S->Q; ++q) {
        double s = 0.0;
        for (int h = 0; h < S->P; ++h) s += vhat[h] * S->psi[q * S->P + h];
        vq[q] = s;
    }
}

/* Observables of the current state at one arbitrary z (d components): out = [Vx, Vy, E, Jx]. */
void orc_observe_at(const void *st, const double *z, double *out4)
{
    const orc_state *S = (const orc_state *)st;
    const orc_cfg *c = &S->cfg;
    int P = S->P;
    int64_t N = c->N;
    double psi[1296];
    orc_psi_at(c, (S->d > 0) ? z : NULL, psi);
    double z1 = 0.0;
    if (S->d == 1 && orc_eps_random(c)) z1 = z[0];
    if (S->d == 2) z1 = z[0];
    double e0 = orc_band_min(c, S->hvF, z1);
    double svx = 0.0, svy = 0.0, se = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double kx = 0.0, ky = 0.0;
        for (int h = 0; h < P; ++h) { kx += khat_at(S, 0, h, i) * psi[h]; ky += khat_at(S, 1, h, i) * psi[h]; }
        double eps = sqrt(S->hvF * S->hvF * (kx * kx + ky * ky) + e0 * e0);
        svx += S->hvF * kx / eps;
        svy += S->hvF * ky / eps;
        se += eps;
    }
    double vF_ms = T1_VF_CMS * 1e-2;
    double n = 2.0 / (ORC_PI * S->hvF * S->hvF) * orc_fd_total(e0, c->eps_F, S->kT) * 1e18;
    out4[0] = svx / N * vF_ms;
    out4[1] = svy / N * vF_ms;
    out4[2] = se / N;
    out4[3] = -Q_E * n * out4[0];
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the following parallel loops (n <= 0: all host cores); for timing the oracle */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* Pathwise sensitivities by forward-mode tangents (test reference for the adjoint).          */
/*                                                                                            */
/* theta = (E_lo, E_hi, eps0_lo, eps0_hi): the endpoints of the field and band-minimum         */
/* intervals; for a deterministic input the two endpoint derivatives are each half of the      */
/* derivative with respect to the common value (the affine map at z = 0).  Discrete events     */
/* (collision times, mechanisms, Pauli outcomes, the trapezoid segment of the edge angle, the   */
/* histogram cells) are frozen at those of the primal run; the random numbers are common.      */
/* Derivatives are propagated through: the Fermi-Dirac sampling (implicit derivative of the    */
/* inverse CDF), the drift (Eq. 17 / Sec. 4.1), the final-state maps h^1..h^6 of Sec. 3, the   */
/* projections (Eqs. 28-30) and the observables (Eqs. 35-37, with n(eps0) of Eq. 31).          */
/* ------------------------------------------------------------------------------------------ */
#define NTH 4

/* parameter derivatives of the node's band minimum and field */
static void node_param_derivs(const orc_state *S, int q, double de0[NTH], double dE[NTH])
{
    const orc_cfg *c = &S->cfg;
    int eps_random = orc_eps_random(c), E_random = (c->Ex_lo != c->Ex_hi);
    double z1 = 0.0, z2 = 0.0;
    if (S->d == 1) { if (eps_random) z1 = S->zq[q]; else z2 = S->zq[q]; }
    if (S->d == 2) { z1 = S->zq[2 * q]; z2 = S->zq[2 * q + 1]; }
    (void)E_random;
    for (int t = 0; t < NTH; ++t) { de0[t] = 0.0; dE[t] = 0.0; }
    dE[0] = 0.5 * (1.0 - z2);
    dE[1] = 0.5 * (1.0 + z2);
    de0[2] = 0.5 * (1.0 - z1);
    de0[3] = 0.5 * (1.0 + z1);
}

static double rho_fd(double e, double mu, double kT) { return e / (1.0 + exp(fmin((e - mu) / kT, 700.0))); }

/* edge angle (same operations as orc_angle_edge) and its derivatives in beta and c */
static double edge_angle_grad(double beta, double cth, double u, int n, double *dth_db, double *dth_dc)
{
    double h = 2.0 * ORC_PI / n;
    double *C = (double *)malloc(sizeof(double) * 3 * (size_t)(n + 1));
    double *Cb = C + (n + 1), *Cc = Cb + (n + 1);
    double x0 = 1.0 - cth;
    double gprev = exp(-beta * x0 * x0), gbp = -x0 * x0 * gprev, gcp = 2.0 * beta * x0 * gprev;
    C[0] = Cb[0] = Cc[0] = 0.0;
    for (int j = 1; j <= n; ++j) {
        double x = cos(j * h) - cth;
        double g = exp(-beta * x * x), gb = -x * x * g, gc = 2.0 * beta * x * g;
        C[j] = C[j - 1] + 0.5 * h * (gprev + g);
        Cb[j] = Cb[j - 1] + 0.5 * h * (gbp + gb);
        Cc[j] = Cc[j - 1] + 0.5 * h * (gcp + gc);
        gprev = g; gbp = gb; gcp = gc;
    }
    double target = u * C[n];
    int j = 0;
    while (j < n - 1 && C[j + 1] <= target) ++j;
    double D = C[j + 1] - C[j], f = (target - C[j]) / D;
    double Db = Cb[j + 1] - Cb[j], Dc = Cc[j + 1] - Cc[j];
    double fb = ((u * Cb[n] - Cb[j]) * D - (target - C[j]) * Db) / (D * D);
    double fc = ((u * Cc[n] - Cc[j]) * D - (target - C[j]) * Dc) / (D * D);
    free(C);
    *dth_db = fb * h;
    *dth_dc = fc * h;
    return (j + f) * h;
}

/* Jacobian dk'/dk (row-major 2x2) of the final-state map of mechanism l (0..5), random numbers
 * fixed, paper final states. */
static void fs_jacobian(const orc_state *S, int l, double kx, double ky, double uth, double J[4])
{
    double km = sqrt(kx * kx + ky * ky);
    if (l == 5) {
        double cth = (km > 0.0) ? kx / km : 1.0;
        double beta = 2.0 * km * km * S->a_nm * S->a_nm;
        double db, dc;
        double th = edge_angle_grad(beta, cth, uth, S->cfg.n_theta, &db, &dc);
        double ct = cos(th), st = sin(th);
        double nx = (km > 0.0) ? kx / km : 1.0, ny = (km > 0.0) ? ky / km : 0.0;
        double gbx = 4.0 * S->a_nm * S->a_nm * kx, gby = 4.0 * S->a_nm * S->a_nm * ky; /* d beta / dk */
        double gcx = 0.0, gcy = 0.0;                                                    /* d c / dk */
        if (km > 0.0) { gcx = ky * ky / (km * km * km); gcy = -kx * ky / (km * km * km); }
        double tx = db * gbx + dc * gcx, ty = db * gby + dc * gcy;                      /* d th / dk */
        J[0] = ct * nx - km * st * tx; J[1] = ct * ny - km * st * ty;
        J[2] = st * nx + km * ct * tx; J[3] = st * ny + km * ct * ty;
        return;
    }
    double th, s = 0.0, dlt = 0.0;
    if (l == 0) th = orc_angle_ac(uth);
    else if (l == 1 || l == 2) { th = 2.0 * ORC_PI * uth; dlt = S->hwO / S->hvF; s = (l == 1) ? -1.0 : 1.0; }
    else { th = orc_angle_k(uth); dlt = S->hwK / S->hvF; s = (l == 3) ? -1.0 : 1.0; }
    double ct = cos(th), st = sin(th);
    /* k' = R k (1 + s dlt/|k|):  dk'/dk = R [ (1 + s dlt/|k|) I - (s dlt/|k|) n n^T ] */
    double a = 1.0 + s * dlt / km, b = s * dlt / km;
    double nx = kx / km, ny = ky / km;
    double M0 = a - b * nx * nx, M1 = -b * nx * ny, M2 = -b * ny * nx, M3 = a - b * ny * ny;
    J[0] = ct * M0 - st * M2; J[1] = ct * M1 - st * M3;
    J[2] = st * M0 + ct * M2; J[3] = st * M1 + ct * M3;
}

/* node observables and their tangents at the current state: J[q], dJ[q][t] */
static void tangent_observe(const orc_state *S, const double *dk, double *Jq, double *dJq)
{
    int P = S->P, Q = S->Q;
    int64_t N = S->cfg.N;
    double vF_ms = T1_VF_CMS * 1e-2;
    for (int q = 0; q < Q; ++q) {
        double e0 = S->eps0q[q], de0[NTH], dE[NTH];
        node_param_derivs(S, q, de0, dE);
        double sv = 0.0, sdv[NTH] = {0, 0, 0, 0};
        for (int64_t i = 0; i < N; ++i) {
            double kx = 0.0, ky = 0.0;
            for (int h = 0; h < P; ++h) { kx += khat_at(S, 0, h, i) * S->psi[q * P + h]; ky += khat_at(S, 1, h, i) * S->psi[q * P + h]; }
            double eps = sqrt(S->hvF * S->hvF * (kx * kx + ky * ky) + e0 * e0);
            double v = S->hvF * kx / eps;
            double e3 = eps * eps * eps;
            double dvdkx = S->hvF / eps - S->hvF * S->hvF * S->hvF * kx * kx / e3;
            double dvdky = -S->hvF * S->hvF * S->hvF * kx * ky / e3;
            double dvde0 = -S->hvF * kx * e0 / e3;
            sv += v;
            for (int t = 0; t < NTH; ++t) {
                double dkx = 0.0, dky = 0.0;
                for (int h = 0; h < P; ++h) {
                    dkx += dk[(((size_t)t * 2 + 0) * P + h) * N + i] * S->psi[q * P + h];
                    dky += dk[(((size_t)t * 2 + 1) * P + h) * N + i] * S->psi[q * P + h];
                }
                sdv[t] += dvdkx * dkx + dvdky * dky + dvde0 * de0[t];
            }
        }
        double nq = S->nq[q];
        double dn = -2.0 / (ORC_PI * S->hvF * S->hvF) * rho_fd(e0, S->cfg.eps_F, S->kT) * 1e18;
        Jq[q] = -Q_E * nq * vF_ms * sv / (double)N;
        for (int t = 0; t < NTH; ++t)
            dJq[q * NTH + t] = -Q_E * vF_ms / (double)N * (dn * de0[t] * sv + nq * sdv[t]);
    }
}

int orc_tangent_run(void *st, int64_t nsteps, int64_t every, int64_t window, double *val2, double *grad8)
{
    orc_state *S = (orc_state *)st;
    const orc_cfg *c = &S->cfg;
    if (!S->sampled || S->step != 0 || c->final_state != ORC_FS_PAPER || every < 1 ||
        c->splitting != ORC_SPLIT_LIE)
        return -1;
    int P = S->P, Q = S->Q;
    int64_t N = c->N;
    double *dk = (double *)calloc((size_t)NTH * 2 * P * N, sizeof(double));
    /* initial tangents: k_q = |k|(cos th, sin th), |k| = sqrt(eps^2 - e0^2)/hvF, eps = F^-1(u; e0) */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        uint32_t ctr[4] = {(uint32_t)i, c->stream_id, 0u, ORC_INIT_PURPOSE};
        uint32_t key[2] = {(uint32_t)c->seed, (uint32_t)(c->seed >> 32)};
        uint32_t o[4];
        orc_philox(ctr, key, o);
        double ue = orc_u01(o[0]), th = 2.0 * ORC_PI * orc_u01(o[1]);
        for (int q = 0; q < Q; ++q) {
            double e0 = S->eps0q[q], de0[NTH], dE[NTH];
            node_param_derivs(S, q, de0, dE);
            double eps = orc_fd_sample(e0, c->eps_F, S->kT, ue);
            double r = eps * eps - e0 * e0;
            if (r <= 0.0) continue;
            double km = sqrt(r) / S->hvF;
            double deps = rho_fd(e0, c->eps_F, S->kT) * (1.0 - ue) / rho_fd(eps, c->eps_F, S->kT);
            double dkm = (eps * deps - e0) / (S->hvF * S->hvF * km);
            for (int t = 0; t < NTH; ++t)
                for (int h = 0; h < P; ++h) {
                    double wp = S->wq[q] * S->psi[q * P + h];
                    dk[(((size_t)t * 2 + 0) * P + h) * N + i] += wp * dkm * de0[t] * cos(th);
                    dk[(((size_t)t * 2 + 1) * P + h) * N + i] += wp * dkm * de0[t] * sin(th);
                }
        }
    }
    /* per-step drift derivative of the x coefficients: d dhat_h / d theta */
    double ddhat[NTH * 64];
    for (int t = 0; t < NTH; ++t)
        for (int h = 0; h < P; ++h) {
            double sacc = 0.0;
            for (int q = 0; q < Q; ++q) {
                double de0[NTH], dE[NTH];
                node_param_derivs(S, q, de0, dE);
                sacc += S->wq[q] * S->psi[q * P + h] * dE[t] * 1e-7 * c->dt_fs / S->hbar_fs;
            }
            ddhat[t * 64 + h] = sacc;
        }
    double accJ = 0.0, accV = 0.0, accdJ[NTH] = {0, 0, 0, 0}, accdV[NTH] = {0, 0, 0, 0};
    int64_t nout = 0;
    double *Jq = (double *)calloc((size_t)Q, sizeof(double)), *dJq = (double *)calloc((size_t)Q * NTH, sizeof(double));
    for (int64_t n = 0; n < nsteps; ++n) {
        const uint32_t *Hn = S->H;
        uint32_t Nmx[1296];
        if (c->pauli_norm == ORC_PAULI_CURRENT_MAX) hist_max(S, Nmx);
        else memcpy(Nmx, S->Nmax, sizeof(uint32_t) * Q);
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < N; ++i) {
            double kx[1296], ky[1296], g[1296 * 6];
            double *tk = (double *)malloc(sizeof(double) * NTH * 2 * (size_t)Q);  /* node tangents */
            int64_t rej = 0;
            for (int h = 0; h < P; ++h) {
                S->khat[((size_t)0 * P + h) * N + i] -= S->dhat[h];
                for (int t = 0; t < NTH; ++t) dk[(((size_t)t * 2 + 0) * P + h) * N + i] -= ddhat[t * 64 + h];
            }
            recon_particle(S, i, kx, ky);
            double Gt = 0.0;
            for (int q = 0; q < Q; ++q) {
                orc_rates_node(S, kx[q], ky[q], S->eps0q[q], &g[q * 6]);
                double sg = 0.0;
                for (int m = 0; m < 6; ++m) sg += g[q * 6 + m];
                if (sg > Gt) Gt = sg;
            }
            Gt *= (1.0 + c->alpha);
            double tc = 0.0, u[4];
            uint32_t cc = 0;
            orc_draw(c, i, n, cc, u);
            double dtc = (Gt > 0.0) ? -log(u[0]) / Gt : INFINITY;
            while (tc + dtc < c->dt_fs) {
                if ((int)cc >= c->max_coll) break;
                /* node tangents of the current state */
                for (int q = 0; q < Q; ++q)
                    for (int t = 0; t < NTH; ++t) {
                        double ax = 0.0, ay = 0.0;
                        for (int h = 0; h < P; ++h) {
                            ax += dk[(((size_t)t * 2 + 0) * P + h) * N + i] * S->psi[q * P + h];
                            ay += dk[(((size_t)t * 2 + 1) * P + h) * N + i] * S->psi[q * P + h];
                        }
                        tk[(q * NTH + t) * 2 + 0] = ax;
                        tk[(q * NTH + t) * 2 + 1] = ay;
                    }
                for (int q = 0; q < Q; ++q) {
                    double k0x = kx[q], k0y = ky[q];
                    /* the selected mechanism, as in collide_node */
                    double target = u[1] * Gt, cum = 0.0;
                    int l = 6;
                    for (int m = 0; m < 6; ++m) { cum += g[q * 6 + m]; if (target < cum) { l = m; break; } }
                    int changed = collide_node(S, q, Gt, &g[q * 6], u[1], u[2], u[3], Hn, Nmx, S->dq[q], &kx[q],
                                               &ky[q], &rej);
                    if (changed) {
                        double J[4];
                        fs_jacobian(S, l, k0x, k0y, u[3], J);
                        for (int t = 0; t < NTH; ++t) {
                            double ax = tk[(q * NTH + t) * 2 + 0], ay = tk[(q * NTH + t) * 2 + 1];
                            tk[(q * NTH + t) * 2 + 0] = J[0] * ax + J[1] * ay;
                            tk[(q * NTH + t) * 2 + 1] = J[2] * ax + J[3] * ay;
                        }
                    }
                }
                project_particle(S, i, kx, ky);
                for (int t = 0; t < NTH; ++t)
                    for (int h = 0; h < P; ++h) {
                        double ax = 0.0, ay = 0.0;
                        for (int q = 0; q < Q; ++q) {
                            double wp = S->wq[q] * S->psi[q * P + h];
                            ax += wp * tk[(q * NTH + t) * 2 + 0];
                            ay += wp * tk[(q * NTH + t) * 2 + 1];
                        }
                        dk[(((size_t)t * 2 + 0) * P + h) * N + i] = ax;
                        dk[(((size_t)t * 2 + 1) * P + h) * N + i] = ay;
                    }
                recon_particle(S, i, kx, ky);
                Gt = 0.0;
                for (int q = 0; q < Q; ++q) {
                    orc_rates_node(S, kx[q], ky[q], S->eps0q[q], &g[q * 6]);
                    double sg = 0.0;
                    for (int m = 0; m < 6; ++m) sg += g[q * 6 + m];
                    if (sg > Gt) Gt = sg;
                }
                Gt *= (1.0 + c->alpha);
                tc += dtc;
                ++cc;
                orc_draw(c, i, n, cc, u);
                dtc = (Gt > 0.0) ? -log(u[0]) / Gt : INFINITY;
            }
            free(tk);
        }
        S->step = n + 1;
        S->n_out_of_grid = build_hist(S);
        if (S->step % every == 0 && S->step > nsteps - window) {
            tangent_observe(S, dk, Jq, dJq);
            double m = 0.0, m2 = 0.0, dm[NTH] = {0, 0, 0, 0}, dm2[NTH] = {0, 0, 0, 0};
            for (int q = 0; q < Q; ++q) {
                m += S->wq[q] * Jq[q];
                m2 += S->wq[q] * Jq[q] * Jq[q];
                for (int t = 0; t < NTH; ++t) {
                    dm[t] += S->wq[q] * dJq[q * NTH + t];
                    dm2[t] += 2.0 * S->wq[q] * Jq[q] * dJq[q * NTH + t];
                }
            }
            accJ += m;
            accV += m2 - m * m;
            for (int t = 0; t < NTH; ++t) { accdJ[t] += dm[t]; accdV[t] += dm2[t] - 2.0 * m * dm[t]; }
            ++nout;
        }
    }
    free(Jq); free(dJq); free(dk);
    if (nout == 0) return -2;
    val2[0] = accJ / nout;
    val2[1] = accV / nout;
    for (int t = 0; t < NTH; ++t) { grad8[t] = accdJ[t] / nout; grad8[NTH + t] = accdV[t] / nout; }
    return 0;
}

/* Window averages of mean_z J_x and var_z J_x of an ordinary run (no tangents): the same
 * objective as orc_tangent_run, for finite-difference checks. */
int orc_window_objective(void *st, int64_t nsteps, int64_t every, int64_t window, double *val2)
{
    orc_state *S = (orc_state *)st;
    double accJ = 0.0, accV = 0.0;
    int64_t nout = 0;
    int64_t s0 = S->step;
    for (int64_t n = 0; n < nsteps; ++n) {
        step_once(S);
        if ((S->step - s0) % every == 0 && (S->step - s0) > nsteps - window) {
            record_moments(S);
            accJ += S->mean[(S->T_out - 1) * 4 + 3];
            accV += S->var[(S->T_out - 1) * 4 + 3];
            ++nout;
        }
    }
    if (nout == 0) return -2;
    val2[0] = accJ / nout;
    val2[1] = accV / nout;
    return 0;
}
