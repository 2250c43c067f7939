/*
 * pgc.h -- C ABI of the GB300 (sm_103a) particle stochastic-Galerkin solver for the
 * space-homogeneous semiclassical Boltzmann equation of electrons in a graphene nanoribbon
 * (Medaglia, Nastasi, Romano, Zanella, "Uncertainty quantification for charge transport in GNRs
 * through particle Galerkin methods for the semiclassical Boltzmann equation", arXiv:2404.19602).
 *
 * What one call computes
 * ----------------------
 * The ensemble is N particles.  Particle i carries its wave-vector as gPC coefficients
 * khat_{i,h}, h = 0..P-1 (Eq. (23)); with deterministic inputs P = 1 and khat is k itself.
 * pgc_step advances every particle by n_steps time steps of the Lie splitting of Sec. 3:
 *   1. field drift khat_{x,h} -= (e/hbar) dt int E(z) Psi_h p dz  (Eq. (17), Sec. 4.1);
 *   2. DSMC collision loop of Algorithm 1 (deterministic) / Algorithm 2 (stochastic Galerkin):
 *      free flight dt = -ln(xi) / max_z Gamma_tot(z) (Eqs. (18),(19),(25)), mechanism
 *      selection over the rate vector of Eq. (20), final states h^1..h^7 of Sec. 3, Pauli
 *      acceptance against the previous-step histogram (Eqs. (22),(27)), projection onto the
 *      gPC basis (Eqs. (28)-(30));
 *   3. the histogram f^{n+1}_{N,rl}(z_q) of Eq. (24) at the quadrature nodes, and, every
 *      moments_every steps, the observables of Eqs. (35)-(37) at the nodes and their mean and
 *      variance over z (Sec. 4.2).
 * Random numbers are Philox4x32-10 (Salmon et al., SC'11) with key = seed and counter
 * (i, stream_id, step, attempt); the same counters drive the FP64 CPU oracle of the tests.
 *
 * Readings of points the paper leaves open (the design notes list them with reasons):
 *   - Gauss-Legendre quadrature with quad_per_dim nodes per random dimension for every z-integral;
 *   - orthonormal Legendre basis sqrt(2h+1) P_h; in 2-D total degree <= M, graded order
 *     h -> (degree in z1, degree in z2) = (t-j, j) for t = 0..M, j = 0..t;
 *     z1 is the band-minimum variable, z2 the field variable; node q = q1 * quad_per_dim + q2;
 *   - the majorant is the maximum over the nodes; the self-scattering entry of node q is
 *     Gamma_tilde - sum_nu Gamma_nu(z_q);
 *   - the flight time is drawn again after every collision; at most max_collisions per step;
 *   - Pauli: f = N_rl / Nmax with Nmax the maximum of the initial histogram (default), the
 *     histogram counted on the fixed grid before the drift and looked up at cell(k' + (e/hbar)E dt);
 *   - the edge final angle is absolute; its CDF is the trapezoid CDF on n_theta_edge points.
 *
 * Units: energy eV, time fs, field V/cm, wave-vector nm^-1.  Velocities m/s, density m^-2,
 * sheet current J = -e n V_x in A/m.
 *
 * Memory and ownership
 * --------------------
 * The caller owns every device buffer: it asks pgc_query_sizes for the byte counts, allocates
 * them (e.g. as torch tensors), and passes the device pointers to pgc_init; they must stay valid
 * until pgc_destroy.  The context owns only host-side tables.  Device layouts:
 *   state   : R khat[2][P][ld], R = float (PGC_FP32) or double (PGC_FP64), c = x,y outermost,
 *             ld = N rounded up to a multiple of 64; 256-byte aligned base required;
 *   hist    : uint32 H[4][Q][Nk][Nk] (four rotating buffers, f^n in buffer n % 4; cell (r,l)
 *             of k is r = floor((kx+Lk)/dk), l = floor((ky+Lk)/dk));
 *   scratch : work space (two collider queues, collider bitmaps, block partial sums, time
 *             series, counters, a device copy of the node tables).
 * All calls on a context are ordered on the CUDA stream given to pgc_init; calls that return
 * host data (pgc_moments, pgc_get_state, pgc_counters, pgc_reconstruct_f) synchronize it.
 * The buffers are read and written by work queued on that stream: a caller that frees or reuses
 * them must do so behind that work (with a stream-ordered allocator, allocate them on that
 * stream); pgc_init's own initialisation of the buffers is queued on that stream too.
 *
 * Errors
 * ------
 * Every call returns a pgc_status and never throws across the ABI.  pgc_last_error(ctx) gives a
 * message for the last failing call on ctx (pgc_last_error(NULL) for failures before a context
 * exists).  A device-side error flag (e.g. a collision cap) is read back by pgc_counters.
 * After PGC_ECUDA the context is unusable (PGC_ESTATE) and must be destroyed.
 */
#ifndef PGC_H
#define PGC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PGC_OK = 0,
    PGC_EINVAL = 1,          /* invalid argument or configuration */
    PGC_ENOMEM = 2,          /* host allocation failed / buffer too small */
    PGC_ECUDA = 3,           /* a CUDA runtime call failed */
    PGC_ESTATE = 4,          /* context in a failed state */
    PGC_ETIMEOUT = 5,        /* a bounded device wait gave up */
    PGC_EUNSUPPORTED = 6     /* valid but not compiled (e.g. basis size without a kernel) */
} pgc_status;

/* mechanism bits, in the order of the rate vector Lambda of Eq. (20) */
enum {
    PGC_MECH_AC = 1, PGC_MECH_OPM = 2, PGC_MECH_OPP = 4, PGC_MECH_KM = 8, PGC_MECH_KP = 16,
    PGC_MECH_EDGE = 32, PGC_MECH_ALL = 63
};
enum { PGC_FP32 = 0, PGC_FP64 = 1 };
enum { PGC_PAULI_INITIAL_MAX = 0, PGC_PAULI_CURRENT_MAX = 1, PGC_PAULI_OFF = 2 };
enum { PGC_FS_PAPER = 0, PGC_FS_EXACT_ENERGY = 1 };
/* How the band minimum depends on z (Sec. 2: eps0 = hbar vF pi / W, W the ribbon width):
 * AFFINE: eps0(z) affine between eps0_eV.lo and .hi; WIDTH: the width is the input, W(z) affine
 * between width_nm.lo and .hi and eps0(z) = hbar vF pi / W(z) (not a polynomial in z; the
 * scenario of Test 2, W = (6.5 + z) nm). */
enum { PGC_EPS0_AFFINE = 0, PGC_EPS0_WIDTH = 1 };
/* Time splitting of the field drift T and the collisions C (Sec. 3): LIE, one step is
 * C_dt(T_dt(f)) (the paper's scheme); STRANG, T_{dt/2}(C_dt(T_{dt/2}(f))), the second-order
 * splitting the paper names as possible.  In the Strang form the Pauli look-up of a candidate
 * k' is at cell(k' + (e/hbar) E dt / 2) of f^n, and every histogram and observable is that of
 * the state at the step boundary.  The device state buffer then holds the coefficients of the
 * state at the step boundary plus half a step's drift (k^n + (e/hbar) E dt / 2, x coefficients);
 * pgc_get_state / pgc_set_state convert, and the batch and adjoint entry points return
 * PGC_EUNSUPPORTED for it. */
enum { PGC_SPLIT_LIE = 0, PGC_SPLIT_STRANG = 1 };
/* Where the streaming kernel reconstructs the node values k(z_q) = sum_h khat_h Psi_h(z_q)
 * (Eq. (23)), a dense [particles x P] x [P x Q] contraction: OFF, the FP32 FMA pipes (default);
 * F16X3, the tensor cores (tcgen05, FP32 accumulation) with every FP32 operand split into two
 * FP16 parts and three products (~22 significant bits, the precision class of the FMA path);
 * F16, the tensor cores with one FP16 product (FP16 inputs, ~11 bits; node values off by ~1e-3
 * relative).  Compiled for the FP32 21 x 36 shape (two random inputs, total degree 5); other
 * shapes return PGC_EUNSUPPORTED.  A context with tc_proj set steps in the two-launch form
 * (pgc_set_pipeline(ctx, 1) returns PGC_EUNSUPPORTED), and the batch and adjoint entry points
 * refuse it (their kernels reconstruct on the FMA pipes).  Collisions (phase 2) always
 * reconstruct on the FMA pipes.  Bit 0 of PGC_CNT_ERROR is set if a wait for the tensor cores
 * gave up (the step's results are then not valid). */
enum { PGC_TC_OFF = 0, PGC_TC_F16X3 = 1, PGC_TC_F16 = 2 };

/* counters returned by pgc_counters */
enum {
    PGC_CNT_ATTEMPTS = 0,     /* collision events (real or self) */
    PGC_CNT_CHANGED = 1,      /* events that changed the state at >= 1 node */
    PGC_CNT_REJECTED = 2,     /* node-level Pauli rejections */
    PGC_CNT_CAPPED = 3,       /* particle-steps that hit max_collisions */
    PGC_CNT_OUT_OF_GRID = 4,  /* node values outside [-Lk,Lk]^2 in the last histogram */
    PGC_CNT_QUEUED = 5,       /* particle-steps sent to the collider kernel */
    PGC_CNT_ERROR = 6,        /* device error flags (0 = none; bit 0: a tensor-core wait gave up) */
    PGC_CNT_STEPS = 7,        /* time steps done */
    PGC_NUM_COUNTERS = 8
};

typedef struct { double lo, hi; } pgc_interval;  /* lo == hi: deterministic input */

typedef struct {
    double T_K;              /* lattice and initial Fermi-Dirac temperature (300) */
    double eps_F_eV;         /* Fermi level of the initial state (0.4) */
    pgc_interval eps0_eV;    /* conduction-band minimum hbar vF pi / W; band gap E_g = 2 eps0 (AFFINE law) */
    pgc_interval Ex_Vcm;     /* field along x; E_y = 0 */
    uint32_t mech_mask;      /* PGC_MECH_*; 0 = ballistic */
    double alpha;            /* self-scattering tuning of Eq. (19) (0.1) */
    int32_t Nk;              /* grid cells per direction (240) */
    double Lk_hvF_eV;        /* L_k * hbar vF (5) */
    int32_t degree_M;        /* gPC degree (total degree in 2-D) */
    int32_t quad_per_dim;    /* Gauss-Legendre nodes per random dimension (M + 1) */
    int64_t n_particles;     /* N >= 1 */
    double dt_fs;            /* time step (1) */
    uint64_t seed;           /* Philox key */
    uint32_t stream_id;      /* second Philox counter word (case / ensemble id) */
    int32_t precision;       /* PGC_FP32 (state FP32, reductions FP64) or PGC_FP64 */
    int32_t pauli_norm;      /* PGC_PAULI_* */
    int32_t final_state;     /* PGC_FS_* */
    int32_t n_theta_edge;    /* trapezoid points of the edge integral (64; even, 4..256) */
    int32_t max_collisions;  /* per particle and step (32) */
    int32_t max_outputs;     /* capacity of the moment time series */
    int32_t eps0_law;        /* PGC_EPS0_AFFINE (default) or PGC_EPS0_WIDTH */
    pgc_interval width_nm;   /* ribbon width, nm (WIDTH law; lo > 0) */
    int32_t splitting;       /* PGC_SPLIT_LIE (default) or PGC_SPLIT_STRANG */
    int32_t tc_proj;         /* PGC_TC_OFF (default), PGC_TC_F16X3 or PGC_TC_F16 */
} pgc_config;

typedef struct pgc_ctx pgc_ctx;

/* Fill cfg with the defaults of Sec. 5 (300 K, eps_F 0.4 eV, eps0 0.1 eV, 5 kV/cm, all
 * mechanisms, alpha 0.1, Nk 240, Lk hbar vF 5 eV, M 5, 6 nodes, N 1e4, 1 fs, seed 1, FP32). */
void pgc_config_default(pgc_config *cfg);

/* Validate cfg and report the device buffer sizes (bytes) and the basis / node counts.
 * Any out pointer may be NULL.  Returns PGC_EINVAL / PGC_EUNSUPPORTED for a bad cfg. */
pgc_status pgc_query_sizes(const pgc_config *cfg, size_t *state_bytes, size_t *hist_bytes,
                           size_t *scratch_bytes, int32_t *P, int32_t *Q);

/* Create a context on the current CUDA device and set up the initial state:
 * if h_init_khat is NULL, particles are sampled on the device from the Fermi-Dirac state
 * (Sec. 2) by the inverse CDF of eps*FD(eps) with one uniform shared by all z, and projected
 * (Eq. (23)); otherwise h_init_khat (host, FP64, [2][P][N]) is uploaded.  Then the histogram
 * f^0 and the moments at t = 0 are computed.  stream is a cudaStream_t (NULL = default).
 * d_state / d_hist / d_scratch: caller-owned device buffers of the queried sizes. */
pgc_status pgc_init(const pgc_config *cfg, void *d_state, void *d_hist, void *d_scratch,
                    const double *h_init_khat, void *stream, pgc_ctx **out);

/* Advance n_steps time steps (>= 0).  If moments_every > 0, the moments are recorded after
 * every step whose index is a multiple of moments_every (until max_outputs is reached, then
 * PGC_ENOMEM).  Asynchronous on the context's stream.
 * A step is two kernels: the streaming kernel (drift, reconstruction, flight-time screen and
 * histogram of every particle that provably does not collide) and the collider kernel (the
 * collision loop of Algorithms 1/2 for the rest).  In the pipelined form (n_steps >= 2,
 * pgc_set_pipeline) one launch per step n runs the streaming work of step n beside the collider
 * work of step n - 1, whose particles are carried on through the drift and screen of step n
 * (the streaming work skips them).  Trajectories, histograms and counters are the same in both
 * forms; moment sums may differ in the last bits (FP32 summation order).
 * With moments_every > 0 the moment records (Sec. 4.2) are reduced on a second stream of the
 * highest priority, beside the following step launches; the context creates it on the first
 * such call and pgc_destroy releases it.  Before it returns, the call makes the context's stream
 * wait for that stream (event waits, no host synchronisation), so work queued on the context's
 * stream after the call is ordered after everything the call did. */
pgc_status pgc_step(pgc_ctx *ctx, int64_t n_steps, int32_t moments_every);

/* Switch the pipelined form of pgc_step on (1) or off (0).  Available for every compiled shape
 * and precision except P = 21, Q = 36 in FP64 (PGC_EUNSUPPORTED: the fused kernel's two argument
 * blocks exceed the kernel-parameter space).  On by default when P * Q <= 64. */
pgc_status pgc_set_pipeline(pgc_ctx *ctx, int32_t on);

/* Copy the recorded time series to the host (synchronizes).  Any pointer may be NULL.
 * h_t_fs[T]; h_mean[T][4], h_var[T][4] with columns (V_x m/s, V_y m/s, energy eV, J_x A/m);
 * h_nodes[T][Q][4] per-node values.  *T_out = number of records (t = 0 included).
 * Returns PGC_ETIMEOUT (the series is not copied) if bit 0 of the device error counter is set:
 * a bounded wait for the tensor cores (tc_proj) gave up in some step. */
pgc_status pgc_moments(pgc_ctx *ctx, double *h_t_fs, double *h_mean, double *h_var,
                       double *h_nodes, int64_t *T_out);

/* Distribution of Eq. (24) reconstructed at nz arbitrary points h_z[nz][d] in [-1,1]^d
 * (d = number of random inputs): counts h_hist[nz][Nk][Nk] and their maxima h_max[nz].
 * Counts are non-negative; counts plus particles outside the grid equal N. */
pgc_status pgc_reconstruct_f(pgc_ctx *ctx, const double *h_z, int32_t nz, uint32_t *h_hist,
                             uint32_t *h_max);

/* Observables of the current state at nz arbitrary points h_z[nz][d] in [-1,1]^d (d = number of
 * random inputs; h_z may be NULL when d = 0): every particle is reconstructed at z by Eq. (23),
 * and h_out[nz][4] receives the ensemble averages of Eqs. (35)-(37) at that z: V_x, V_y (m/s), the
 * mean energy (eV) and J_x = -e n(z) V_x (A/m, n of Eq. (31) at the band minimum eps0(z)).
 * At a quadrature node this is the node value pgc_moments reports.  Evaluated at many z drawn
 * from the input distribution, the values give the distribution of an observable over z, e.g.
 * the central 80 % band of Test 2 (Sec. 5) as its 10 % and 90 % quantiles.
 * Arithmetic: reconstruction, velocity and energy in the state precision, sums over groups of
 * particles in that precision, then FP64 in a fixed order (results are reproducible run to run).
 * Cost: one pass over the state per 32 points.  Synchronizes the context stream.
 * Errors: PGC_EINVAL for nz < 0, a NULL h_out (nz > 0), a NULL h_z (nz > 0, d > 0) or a
 * coordinate outside [-1,1]. */
pgc_status pgc_observe_at(pgc_ctx *ctx, const double *h_z, int32_t nz, double *h_out);

/* State as FP64 on the host, layout [2][P][N] (synchronizes), and the reverse upload (the
 * histogram of the uploaded state becomes f^n for the next step). */
pgc_status pgc_get_state(pgc_ctx *ctx, double *h_khat);
pgc_status pgc_set_state(pgc_ctx *ctx, const double *h_khat);

/* The state in the device layout and precision (R khat[2][P][ld], the state_bytes of
 * pgc_query_sizes; under the Strang splitting the stored, half-drift-ahead coefficients, so that
 * a get/set pair round-trips exactly), copied to or from host memory without conversion: for
 * checkpoints, and for feeding an ensemble from page-locked host memory at copy speed.
 * pgc_get_state_native synchronizes.  pgc_set_state_native only queues the copy and the
 * histogram of the new state (which becomes f^n for the next step, as in pgc_set_state) on the
 * context stream: from page-locked memory the copy is asynchronous, and h_state must stay valid
 * and unchanged until the stream has passed it (e.g. until the next synchronizing call).
 * Errors: PGC_EINVAL for a NULL argument; PGC_ECUDA if the copy fails. */
pgc_status pgc_get_state_native(pgc_ctx *ctx, void *h_state);
pgc_status pgc_set_state_native(pgc_ctx *ctx, const void *h_state);

/* Counters PGC_CNT_* (uint64 [PGC_NUM_COUNTERS]); synchronizes. */
pgc_status pgc_counters(pgc_ctx *ctx, uint64_t *h_counters);

/* Current histogram f^n: h_hist[Q][Nk][Nk] and the normaliser Nmax[Q] of the Pauli test. */
pgc_status pgc_get_hist(pgc_ctx *ctx, uint32_t *h_hist, uint32_t *h_nmax);

/* Kernel timing samples (tracing): with every > 0, CUDA events are recorded on the context
 * stream around the two kernels of every `every`-th step; every = 0 switches it off and
 * clears the samples.  pgc_profile_read (synchronizes) returns the mean duration in ms of the
 * streaming kernel (phase 1: drift, reconstruction, flight-time screen, histogram) and of the
 * collider kernel (phase 2: collision loop of Algorithms 1/2) over the samples.  In the
 * pipelined form the sampled steps are fused launches: ms_phase1 is the fused launch (the
 * whole step) and ms_phase2 is 0. */
pgc_status pgc_profile(pgc_ctx *ctx, int32_t every);
pgc_status pgc_profile_read(pgc_ctx *ctx, double *ms_phase1, double *ms_phase2, int64_t *samples);

/* Timeline of the sampled steps (synchronizes): h_t[k][4] = start and end of the streaming
 * kernel, start and end of the collider kernel of the k-th sampled step, in ms after an event
 * recorded before the first sampled step since pgc_profile (at most 4096 samples are kept).
 * In the pipelined form a sampled step is its fused launch: the streaming interval is that
 * launch and the collider interval is empty.  Copies min(max_samples, kept) samples;
 * *n_samples = samples kept. */
pgc_status pgc_profile_timeline(pgc_ctx *ctx, double *h_t, int64_t max_samples, int64_t *n_samples);

/* Release the context (does not free the caller's buffers). NULL is a no-op. */
void pgc_destroy(pgc_ctx *ctx);

/* Message of the last failing call on ctx; ctx == NULL gives the last failure of a call that
 * had no context (pgc_query_sizes, pgc_init). */
const char *pgc_last_error(const pgc_ctx *ctx);
const char *pgc_status_string(pgc_status s);

/* Observation of the current state that allocates nothing (the paper has no counterpart; this
 * is a service for callers that may not allocate device memory while they run, e.g. because a
 * framework's pool owns all device memory, or because cudaMalloc / cudaFree could synchronize the
 * device under queued work).  Writes the histogram of the current state at the quadrature nodes
 * to d_hist_out (device, uint32 [Q][Nk][Nk], cleared by the call) and one moment record to
 * d_record_out (device, double [1 + 4Q + 8]: t_fs, nodes[Q][4], mean[4], var[4], the layout of
 * pgc_moments).  Its block-partial scratch is a fixed 4 MiB device array inside the library
 * (held by every GPU that loads the library until exit): configurations whose partial sums need
 * more are rejected with PGC_EINVAL and a message.  No cudaMalloc/cudaFree or other allocating
 * call is made.  The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream capture.  All calls
 * share the array: calls whose work overlaps on the GPU (unordered streams) race.  Runs on
 * `stream`, which must be ordered after the context's pending work. */
pgc_status pgc_observe_static(pgc_ctx *ctx, uint32_t *d_hist_out, double *d_record_out, void *stream);

/* ---------------------------------------------------------------------------------------- */
/* Batched sweep: many contexts ("cases" with different fields, band-minimum intervals and    */
/* particle counts, the same basis, precision and physics) advanced together.  Each time step */
/* is one persistent phase-1 launch over a tile list of all cases, one collider launch and one */
/* finalize launch; the step index lives in device memory, so the sequence is captured once   */
/* into a CUDA graph and replayed.  Every case follows exactly the trajectory its context      */
/* would follow alone (same Philox streams, same arithmetic; only the grouping of the FP64      */
/* moment partial sums differs).  The contexts keep their buffers and moment series; after     */
/* pgc_batch_step their step counters and series have advanced as by pgc_step.                */
/* ---------------------------------------------------------------------------------------- */
typedef struct pgc_batch pgc_batch;

/* Check that the contexts can be batched (same shape, precision and physics, same step and
 * stream, Pauli mode initial-max or off, < 2^32 particles in total) and report the bytes of the
 * caller-owned device scratch the batch needs (case table, collider queue, partial sums). */
pgc_status pgc_batch_query_sizes(pgc_ctx *const *ctxs, int32_t n_cases, size_t *scratch_bytes);

/* Create a batch over ctxs[0..n_cases) (the contexts must outlive it) with caller scratch of the
 * queried size (256-byte aligned).  tile_particles: particles per tile of the phase-1 work list
 * (a multiple of the block pass, 1024 for P <= 8 and 256 otherwise); 0 = the launch
 * configuration pgc_batch_autotune chose earlier in this process for a batch of the same basis,
 * precision and total particle count (within a factor 2), else 8 passes with the default
 * launch configuration. */
pgc_status pgc_batch_create(pgc_ctx *const *ctxs, int32_t n_cases, void *d_scratch, int32_t tile_particles,
                            pgc_batch **out);

/* Advance every case by n_steps; moments as in pgc_step.  use_graph != 0 replays a captured
 * graph of 10 time steps (the stream must not be the legacy default stream). */
pgc_status pgc_batch_step(pgc_batch *b, int64_t n_steps, int32_t moments_every, int32_t use_graph);

/* Autotuner of the batch's launch configuration: the tile size (from the minimum tile to 32768
 * particles), the threads per streaming block (128, 256), the particles per thread of the
 * streaming kernel (4, 2, 1 for the small bases; 1 for P = 21), the streaming blocks per SM
 * (1 .. resident) and the collider blocks per SM (2 .. resident), by coordinate descent from the
 * current configuration, two rounds, each candidate timed over steps_per_candidate time steps
 * (no moments) with CUDA events.  The fastest is applied and cached for later batches of the
 * same kind (pgc_batch_create with tile_particles = 0); *chosen_tile and *ms_per_step (either
 * may be NULL) report it.  The timed steps advance the simulation (no launch configuration
 * changes a trajectory; only the grouping of the FP32 warp sums of the moments differs). */
pgc_status pgc_batch_autotune(pgc_batch *b, int32_t steps_per_candidate, int32_t *chosen_tile, double *ms_per_step);

/* The batch's launch configuration: cfg5 = {tile, threads per streaming block, particles per
 * thread, streaming blocks per SM, collider blocks per SM}. */
pgc_status pgc_batch_launch_config(const pgc_batch *b, int32_t *cfg5);

void pgc_batch_destroy(pgc_batch *b);
const char *pgc_batch_last_error(const pgc_batch *b);

/* ---------------------------------------------------------------------------------------- */
/* Adjoint: pathwise sensitivities (discrete events frozen) of the time-averaged mean and      */
/* variance over z of the current J_x.                                                        */
/*   Jbar = average over the moment records n in (n_steps - window_steps, n_steps] of mean_z J_x,*/
/*   Vbar = the same average of var_z J_x;  L = w[0] Jbar + w[1] Vbar.                        */
/* Gradient of L with respect to theta = (E_lo, E_hi, eps0_lo, eps0_hi), the endpoints of the   */
/* field and band-minimum intervals (for a deterministic input each endpoint derivative is half */
/* of the derivative with respect to the common value).  The context must be at step 0 with its */
/* sampled initial state.  pgc_adjoint runs the forward n_steps exactly as pgc_step (the context */
/* and its moment series advance), keeping a checkpoint (state + histogram) every ckpt_every   */
/* steps, then the reverse sweep: each segment is replayed with the forward kernels and walked  */
/* backwards (transposed Jacobians of drift, reconstruction, final-state maps and projection,  */
/* moment terms), ending with the sensitivity of the Fermi-Dirac sampling.                     */
/* Work memory (caller-owned device buffer) from pgc_adjoint_query_sizes.                      */
/* PGC_EUNSUPPORTED for the WIDTH band-minimum law, the exact-energy final states and the      */
/* current-maximum Pauli normalisation.                                                       */
/* Supported: the paper's final states; Pauli initial-maximum or off.                          */
/* ---------------------------------------------------------------------------------------- */
pgc_status pgc_adjoint_query_sizes(pgc_ctx *ctx, int64_t n_steps, int32_t ckpt_every, size_t *work_bytes);
pgc_status pgc_adjoint(pgc_ctx *ctx, int64_t n_steps, int32_t ckpt_every, int32_t moments_every, int64_t window_steps,
                       const double *h_weights, void *d_work, double *h_value, double *h_grad);

/* The objective of pgc_adjoint without the gradient: advances the context by n_steps as
 * pgc_step (moments every moments_every steps) and writes h_value = (Jbar, Vbar) over the records
 * of those steps in (n_steps - window_steps, n_steps] (synchronizes).  Any starting step; no work
 * memory. */
pgc_status pgc_window_objective(pgc_ctx *ctx, int64_t n_steps, int32_t moments_every, int64_t window_steps,
                                double *h_value);

/* Number of kernel launches issued by the library since load (for launch accounting). */
uint64_t pgc_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* PGC_H */
