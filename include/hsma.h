/*
 * hsma.h -- C ABI of the GB300-native harmonic surface mapping algorithm
 * (HSMA; Zhao, Liang & Xu, "Harmonic surface mapping algorithm for fast
 * electrostatic sums", arXiv:1806.04801).
 *
 * The library computes the electrostatic energy and forces of N point charges
 * in a box whose boundary condition is represented by infinitely many image
 * charges (Sec. II, Eq. "sum"): periodic copies, or the sign-alternating
 * reflections of a grounded (perfectly conducting) box (Eq. "diel" at
 * gamma = -1).  The method (Sec. II.A-C):
 *   (a) sums the N sources and their images inside an auxiliary sphere of
 *       radius Rs directly (Phi_in) at the particles and at monitoring points;
 *   (b) evaluates the harmonic basis r^n Y_n^m (Eq. "harmonic");
 *   (c) fits the coefficients A_nm of the far-image potential Phi_out by least
 *       squares to the boundary condition at the monitoring points;
 *   (d) maps Phi_out onto point charges and dipole pairs on the sphere by
 *       Green's second identity and Fibonacci integration (Eqs. "green",
 *       "cd", "integrals"), and sums their potential and field at the
 *       particles.
 * Every step runs in CUDA kernels on the device.
 *
 * Conventions.  Gaussian units: potential q/r, energy
 * U = 1/2 sum_i q_i phi'(r_i) where phi' omits only the particle's own
 * singular term, force F_i = q_i E'(r_i).  Positions are given in the box
 * frame [0, L_x) x [0, L_y) x [0, L_z), row-major n x 3, FP64.  Periodic
 * inputs are wrapped into the box; grounded inputs must lie strictly inside.
 *
 * Errors.  Every function returns HSMA_OK (0) or a negative code; no
 * exception crosses the ABI.  hsma_strerror() names a code.  After an error
 * the output buffers are unspecified; the plan stays usable unless the code
 * is HSMA_E_CUDA.
 *
 * Ownership.  The caller owns particles and output buffers.  A plan owns its
 * device-resident matrices and its workspace; it is not thread-safe (use one
 * plan per host thread, or the serving API).  All device work of a plan runs
 * on the stream given in hsma_opts (NULL = the legacy default stream).
 */
#ifndef HSMA_H
#define HSMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define HSMA_OK 0
#define HSMA_E_ARG (-1)          /* invalid argument (size, NULL, range)            */
#define HSMA_E_NONNEUTRAL (-2)   /* periodic system with |sum q| > 1e-12 sum |q|     */
#define HSMA_E_OUT_OF_BOX (-3)   /* grounded box: particle on/outside a wall, or NaN */
#define HSMA_E_COINCIDENT (-4)   /* two charges at one point: non-finite result      */
#define HSMA_E_OOM (-5)          /* device or pinned host allocation failed          */
#define HSMA_E_TIMEOUT (-6)      /* a bounded device-side wait ran out               */
#define HSMA_E_CUDA (-7)         /* CUDA runtime error (context may be unusable)     */
#define HSMA_E_ILLCOND (-8)      /* fitting matrix numerically rank deficient        */
#define HSMA_E_NOT_FOUND (-9)    /* unknown ticket / item                            */
#define HSMA_E_AGAIN (-10)       /* serving: result not ready yet                    */
#define HSMA_E_CAPACITY (-11)    /* request larger than the serving memory budget or
                                    the static scratch array                       */
#define HSMA_E_CANCELLED (-12)   /* serving: request cancelled before it ran          */

/* ------------------------------------------------------------ parameters */
typedef struct hsma_plan_s *hsma_plan_t;

typedef enum { HSMA_BC_PERIODIC = 0, HSMA_BC_GROUNDED = 1 } hsma_bc;

/* Arithmetic of the update step.
 *  HSMA_FP64          everything in FP64 (parity form).
 *  HSMA_FP32_ACC64    pair sums with FP32 differences (positions split into
 *                     two FP32 words), FP32 rsqrt and FP32 partial sums folded
 *                     into double-float accumulators; fit, mapping and energy
 *                     in FP64.
 *  HSMA_FP32_TC_FIT   as HSMA_FP32_ACC64, but the fit A = M+ b runs on the
 *                     tensor cores (tcgen05) as a split-BF16 product with
 *                     FP32 accumulation in tensor memory, plus one
 *                     refinement step (residual b - M A in double-float
 *                     arithmetic on the FP32 pipe, correction again on the
 *                     tensor cores). */
typedef enum { HSMA_FP64 = 0, HSMA_FP32_ACC64 = 1, HSMA_FP32_TC_FIT = 2 } hsma_precision;

typedef struct {
    int precision;      /* hsma_precision                         (default 1) */
    double dr_rel;      /* Delta r / Rs of Eq. "cd"; <= 0: 1e-5 periodic,
                           1e-4 grounded (Sec. III)                         */
    int fib_F2;         /* > 0: Fibonacci number F2 of the surface quadrature;
                           0: chosen from Q as the F2 whose 6(F2+1) is nearest
                           to Q (ties to the larger)                         */
    int far_field;      /* how Phi_out reaches the particles: 0 = the point
                           and dipole images on the auxiliary sphere (Sec.
                           II.B, the paper's method); 1 = direct evaluation
                           of the fitted series sum A_nm B_nm(r) and its
                           gradient at each particle (FP64)                 */
    void *stream;       /* cudaStream_t for all device work; NULL = default  */
    int use_graphs;     /* 1 = capture the update step in a CUDA graph (default) */
    int profile;        /* 1 = record per-phase CUDA-event timings           */
} hsma_opts;

/* Fill *opts with the defaults above.  Returns HSMA_OK or HSMA_E_ARG. */
int hsma_opts_default(hsma_opts *opts);

/* ------------------------------------------------------------------ plan */
/* Preparation step (Sec. II.C; Table I, upper half): monitoring points
 * (Fibonacci grid on the circumsphere of the box for periodic boxes, Sec.
 * II.A; a near-uniform lattice on the walls otherwise), the fitting matrix
 * M of basis values at the monitoring points (periodic: B(x_i) - B(x~_i),
 * with the constant column dropped), its pseudo-inverse by FP64 Householder
 * QR, and the basis at the 2(F2+1) Fibonacci integration directions on the
 * sphere Rs (Sec. II.B).  All of it stays resident on the device.
 *
 *   box   [L_x, L_y, L_z] > 0 (host pointer)
 *   bc    hsma_bc
 *   p     harmonic order P, 1 <= p <= 40; N_b = (p+1)^2 basis functions
 *   R     auxiliary sphere radius Rs; must exceed the circumradius of the box,
 *         and the image shifts k with |k_a| <= K_a, (K_a - 1/2) L_a < Rs <=
 *         (K_a + 1/2) L_a, must number at most 65535
 *   Q     requested number of surface points (used when opts->fib_F2 == 0)
 *   Kmon  number of monitoring points, Kmon >= N_b, Kmon <= 16384
 *   opts  NULL for defaults
 * On success *out receives a new plan (destroy with hsma_plan_destroy).
 * Errors: HSMA_E_ARG, HSMA_E_OOM, HSMA_E_ILLCOND, HSMA_E_CUDA. */
int hsma_plan(hsma_plan_t *out, const double box[3], int bc, int p, double R, int Q, int Kmon,
              const hsma_opts *opts);

void hsma_plan_destroy(hsma_plan_t plan);

typedef struct {
    int bc, p, n_basis, n_cols;  /* n_cols: fitted columns (N_b - 1 periodic)       */
    int Kmon, n_mon_targets;     /* monitoring points; targets (2 Kmon periodic)    */
    int F2, F1, n_images;        /* quadrature; N_o = 6(F2+1) images                */
    int n_shifts;                /* image shifts k tested when building the in-set  */
    double Rs, R0, alpha, dr;    /* sphere, circumradius, Rs/R0, Delta r            */
    double cond_estimate;        /* max|R_jj| / min|R_jj| of the QR factor          */
    int precision;
} hsma_plan_info_t;

int hsma_plan_get_info(hsma_plan_t plan, hsma_plan_info_t *info);

/* The dimensions hsma_plan would give a plan with these arguments, computed
 * on the host alone (no device, no allocation): N_b = (p+1)^2 and the fitted
 * columns (Sec. II.A), monitoring targets, F2, F1 and N_o = 6(F2+1) of the
 * Fibonacci integration (Sec. II.B), the image shifts tested for the in-set,
 * R0, alpha = Rs/R0 and Delta r (Eq. "cd").  cond_estimate is 0 (it needs
 * the QR).  Argument checks and errors as hsma_plan's host-side ones
 * (HSMA_E_ARG); for sizing plans before any device exists. */
int hsma_plan_dims(const double box[3], int bc, int p, double R, int Q, int Kmon, const hsma_opts *opts,
                   hsma_plan_info_t *info);

/* Change the stream a plan works on (NULL = legacy default stream). */
int hsma_plan_set_stream(hsma_plan_t plan, void *stream);

/* Change the arithmetic of later update steps (hsma_precision). */
int hsma_plan_set_precision(hsma_plan_t plan, int precision);

/* In-set reuse for repeated steps of one moving system (molecular dynamics;
 * the paper's stated application, Sec. III timing study and Sec. IV).  With
 * skin > 0, a single-system update step also records the candidate images
 * within Rs + skin of the sphere's centre (over the image shifts that sphere
 * needs), the particles' spatial order and their positions.  Later calls
 * with the same n and precision skip the sort and the in-set generation: one
 * kernel places every candidate at its particle's current position (a
 * particle that crossed a periodic wall keeps its unwrapped position: its
 * images are the same points) and gives the candidates outside Rs charge 0,
 * so the near-field sums still run over exactly the images inside Rs (Sec.
 * II.A).  This holds while every particle is within the skin of its recorded
 * position: an image moves as its particle does, so one that was farther
 * than Rs + skin from the centre is still outside Rs.  A call where some
 * particle has moved by the skin or more, or a charge changed, is detected on
 * the device and redone with a new list (hsma_plan_inset_stats counts such
 * calls).  Results equal those of a fresh in-set up to the order of the
 * floating-point sums.  skin = 0 (the default) switches reuse off.  Requires
 * skin < Rs - R0 and 2 skin < min L_a; else HSMA_E_ARG.  Costs device
 * memory for n x (shifts of Rs + skin) candidate entries. */
int hsma_plan_set_inset_skin(hsma_plan_t plan, double skin);

/* Launch the near-field pair work of later steps as one CTA per work item
 * (on = 1) instead of a persistent grid that pulls items until none are
 * left (on = 0, the default, faster alone).  CTAs that finish their item
 * free their SM, so work on a stream of higher priority (another plan, a
 * serving lane) starts between items instead of after the whole step; the
 * items are cut 8x finer than the tuned granularity, so an SM frees up
 * sooner, at the cost of more partial records in the workspace; the
 * tensor-core fit then also uses a quarter of the SMs.  Results are the
 * same up to the grouping of the sums.  No counterpart in the paper. */
int hsma_plan_set_preemptible(hsma_plan_t plan, int on);

/* Counts of the plan's single-system steps since creation: in-set lists
 * built, steps that reused a list, and steps redone because the list was
 * stale.  Any pointer may be NULL. */
int hsma_plan_inset_stats(hsma_plan_t plan, int64_t *builds, int64_t *reuses, int64_t *stale);

/* Device bytes the plan's workspace needs for a system of n particles
 * (for admission control).  *bytes is an upper bound. */
int hsma_plan_footprint(hsma_plan_t plan, int64_t n, size_t *bytes);

/* Copy a plan matrix to host memory (FP64, row-major), for inspection and
 * tests.  which: 0 = monitoring points (n_mon_targets x 3, periodic: the
 * Kmon points x_i followed by their partners x~_i), 1 = fitting matrix M
 * (Kmon x n_cols), 2 = pseudo-inverse M+ (n_cols x Kmon), 3 = integration
 * directions (2(F2+1) x 3 unit vectors), 4 = integration weights
 * (2(F2+1)), 5 = basis at the integration points (2(F2+1) x N_b).
 * count is the capacity of host_out in doubles. */
int hsma_plan_get_matrix(hsma_plan_t plan, int which, double *host_out, int64_t count);

/* ---------------------------------------------------------------- update */
typedef struct {
    int64_t n;          /* number of particles N >= 1                     */
    const double *xyz;  /* n x 3, box frame (see top)                     */
    const double *q;    /* n charges                                      */
    int on_device;      /* 1: xyz, q and the output arrays are device
                           pointers; 0: host pointers (copied in and out) */
} hsma_particles;

typedef struct {
    double energy;      /* U (Gaussian units)                                */
    double *forces;     /* n x 3 caller-owned, or NULL                       */
    double *potentials; /* n caller-owned, or NULL: phi'(r_i)                */
    int64_t n_inset;    /* N_s: sources and images inside the sphere          */
    int n_images;       /* N_o surface images                                */
} hsma_out;

/* Update step (Sec. II.C; Table I, lower half) for one configuration:
 * in-set generation, the near-field sums Phi_in and E_in at the particles
 * and at the monitoring points (Sec. II.A), the right-hand side and the fit
 * A = M+ b, the surface images Q_j (Sec. II.B) and their potential and field
 * at the particles, energy and forces.  Returns after the energy is on the
 * host; forces/potentials are complete on return.
 * Size limit: n * n_shifts < 2^31 (the in-set capacity of a system is
 * 32-bit; n < 7.9e7 for the usual 27 shifts); larger n is HSMA_E_ARG.
 * Errors: HSMA_E_ARG, HSMA_E_NONNEUTRAL, HSMA_E_OUT_OF_BOX,
 * HSMA_E_COINCIDENT, HSMA_E_OOM, HSMA_E_TIMEOUT, HSMA_E_CUDA. */
int hsma_energy_forces(hsma_plan_t plan, const hsma_particles *x_q, hsma_out *out);

/* Many independent systems that share one plan, in one persistent pass of
 * device work.  System s holds particles offsets[s] .. offsets[s+1]-1 of the
 * concatenated arrays in *all (offsets: host array of nsys+1 increasing
 * values, offsets[0] = 0).  energies: host array of nsys.  forces /
 * potentials: concatenated (offsets[nsys] x 3 / offsets[nsys]) in the same
 * memory space as *all, or NULL.  An error in one system fails the call;
 * status (host array of nsys, or NULL) receives each system's code.
 * Size limits: nsys <= 65528 and, per system, those of hsma_energy_forces;
 * beyond them HSMA_E_ARG. */
int hsma_energy_forces_batched(hsma_plan_t plan, int nsys, const int64_t *offsets,
                               const hsma_particles *all, double *energies, double *forces,
                               double *potentials, int *status);

/* ------------------------------------------------------- target sharding */
/* The update step split so that one system can be shared by several GPUs
 * (one process per GPU, each with a plan of the same parameters and all n
 * particles).  Part `part` of `nparts` owns a contiguous slice of the
 * particles in the plan's spatial (Morton) order -- whole blocks of the pair
 * kernel -- and a slice of the monitoring targets.
 *
 *   1. hsma_shard_near: Phi_in and E_in at the owned particles (Sec. II.A
 *      near-field sums over the whole in-set), and Phi_in at the owned
 *      monitoring targets, written into phi_mon (host, n_mon_targets, in the
 *      order of hsma_plan_get_matrix(0); zero outside the owned slice).
 *      Outputs (host arrays of capacity n): index[j] is the caller's index of
 *      the j-th owned particle, phi[j] its Phi_in and field[3j..3j+2] its
 *      E_in; *count receives the number of owned particles.
 *   2. The caller sums phi_mon over the parts (an all-reduce of
 *      n_mon_targets doubles).
 *   3. hsma_shard_far: the fit from the full phi_mon (the same on every
 *      part), the surface images (or series), Phi_out and E_out at the owned
 *      particles, and -- on the device, from phi_in / field_in, the near
 *      stage's phi / field of this part (host, count_in = the near stage's
 *      *count entries, owned order; another count_in is HSMA_E_ARG) -- the
 *      owned particles' potentials pot[j] = Phi_in + Phi_out, forces
 *      forces[3j..3j+2] = q (E_in + E_out), and the part's energy
 *      *energy = 1/2 sum_j q_j pot[j] (FP64, fixed summation order).  index
 *      and count as in stage 1 (the same slice).
 *   4. The caller sums *energy over the parts (an all-reduce of one double):
 *      U of Sec. II.C.  Forces stay with the part that owns the particle.
 *
 * x_q may be host or device; every other array is host memory.  Errors as
 * hsma_energy_forces. */
int hsma_shard_near(hsma_plan_t plan, const hsma_particles *x_q, int part, int nparts, int64_t *index,
                    double *phi, double *field, int64_t *count, double *phi_mon);
int hsma_shard_far(hsma_plan_t plan, const hsma_particles *x_q, const double *phi_mon, const double *phi_in,
                   const double *field_in, int64_t count_in, int part, int nparts, int64_t *index, double *pot,
                   double *forces, int64_t *count, double *energy);

/* ----------------------------------------------------------------- tuning */
/* Work decomposition of the near-field pair kernel (no counterpart in the
 * paper; it changes speed, not results beyond rounding of the chunk
 * grouping):
 *   pair_variant    FP32 kernel blocking: 4 = four targets per thread
 *                   (blocks and source tiles of 512) at 4 CTAs per SM;
 *                   5 = the same at 5 CTAs per SM (fewer registers);
 *                   2 = two targets per thread (blocks and tiles of 256) at
 *                   6 CTAs per SM; 12, 13 = two targets per thread with
 *                   packed FP32 pairs (two sources per f32x2 instruction)
 *                   at 6 and 5 CTAs per SM; 14 = four targets per thread,
 *                   packed, at 3 CTAs per SM; 15, 16 = four / two targets
 *                   per thread, packed, tile interleaved in place and the
 *                   double-float sums in shared memory, at 4 / 6 CTAs per
 *                   SM; 17 = three targets per thread (blocks and tiles of
 *                   384), packed, at 4 CTAs per SM; ignored in FP64.  Any
 *                   other value is HSMA_E_ARG in hsma_plan_set_tuning
 *   items_per_slot  work items per resident CTA slot (source chunks are sized
 *                   so that a call has about this many items per slot)
 *   ms              time measured by hsma_autotune (0 otherwise)
 * Defaults (no tuning entry for the call's work size): variant 14 for one
 * system, 17 for a batch, 48 items per slot (FP64: 24 items). */
typedef struct {
    int pair_variant;
    int items_per_slot;
    double ms;
} hsma_tuning;

/* Use *t for every later call (NULL: choose per call from the entries that
 * hsma_autotune / hsma_plan_load_tuning gave the plan for the call's work
 * size, else the defaults). */
int hsma_plan_set_tuning(hsma_plan_t plan, const hsma_tuning *t);

/* The tuning a call with this batch shape (offsets as in
 * hsma_energy_forces_batched, host array) would use. */
int hsma_plan_get_tuning(hsma_plan_t plan, int nsys, const int64_t *offsets, hsma_tuning *out);

/* Autotuner: runs the update step on this batch for each candidate
 * (pair_variant 14, 17, 12, 13, 2 x items_per_slot 8, 16, 24, 48; FP64:
 * items only), keeps the fastest as
 * the plan's entry for this work size, returns it in *best, and appends it as
 * one JSON line to cache_path (if not NULL).  Device inputs are recommended
 * (host inputs add their copies to every timing). */
int hsma_autotune(hsma_plan_t plan, int nsys, const int64_t *offsets, const hsma_particles *all,
                  const char *cache_path, hsma_tuning *best);

/* Loads the entries of a cache written by hsma_autotune that match this plan
 * (device name, boundary, p, Kmon, F2, precision).  Returns how many were
 * loaded (0 if the file does not exist), or a negative code. */
int hsma_plan_load_tuning(hsma_plan_t plan, const char *cache_path);

/* --------------------------------------------------------------- serving */
/* A request loop with continuous batching (a deployment layer over the
 * update step; the paper has no serving component).  The server keeps
 * `lanes` plans with the given parameters resident (matrices and
 * pseudo-inverse on the device), each with its own stream and workspace.  A
 * free lane takes the oldest waiting requests -- at most max_batch systems and
 * at most hbm_budget_bytes of device work in flight over all lanes, by
 * hsma_plan_footprint -- and runs them as one batched update step.  Requests
 * that arrive while other lanes are busy are admitted by the next free lane,
 * so their device work overlaps.  A request larger than the whole budget
 * fails with HSMA_E_CAPACITY.  Small requests (see express_lanes) queue
 * apart and have lanes of their own on a high-priority stream, while the
 * bulk lanes' pair work is preemptible (hsma_plan_set_preemptible), so a
 * small request waits for work items of a large batch, not for the whole
 * batch.  Optional medium lanes (mid_lanes) do the same one level down:
 * medium requests wait for work items of large batches, small ones for work
 * items of medium and large ones.  A batch holds the oldest waiting request
 * of its class and the waiting ones within a factor 4 of its size.
 * Thread-safe: submit and result may be called from any host thread. */
typedef struct hsma_server_s *hsma_server_t;

typedef struct {
    size_t hbm_budget_bytes;  /* device bytes of work in flight; 0 = half the free memory */
    int max_batch;            /* systems per batched pass, 1..65528 (default 64)          */
    int lanes;                /* concurrent batched passes, 1..16 (default 2)            */
    int precision;            /* hsma_precision of served requests (default 1)           */
    int express_lanes;        /* lanes that serve only small requests, on the stream of
                                 highest priority, 0..lanes-1 (default 1); the others
                                 (bulk) serve the large ones (all, if 0), on the
                                 stream of lowest priority, with preemptible pair
                                 work; an express lane's workspace is allocated at
                                 creation for max_batch requests of express_max_n   */
    int64_t express_max_n;    /* requests with n <= this are small (default 20000)     */
    int mid_lanes;            /* lanes that serve only medium requests (express_max_n <
                                 n <= mid_max_n), on a stream of middle priority, with
                                 preemptible pair work and a workspace allocated at
                                 creation for max_batch requests of mid_max_n;
                                 express_lanes + mid_lanes < lanes (default 0: medium
                                 requests are large ones)                            */
    int64_t mid_max_n;        /* upper size of a medium request (>= express_max_n)    */
} hsma_server_opts;

typedef struct {
    int64_t n;                /* particles of the request                                */
    double latency_ms;        /* submit -> result ready                                  */
    double queue_ms;          /* submit -> its batch started                             */
    int batch_size;           /* systems in the batched pass that served it              */
    int status;               /* its code                                                */
} hsma_request_info;

typedef struct {
    int64_t completed, failed, cancelled, queued, batches;
    double mean_batch;        /* systems per batched pass                                */
    double elapsed_s;         /* first submit -> last completion                         */
    size_t hbm_held_bytes, hbm_budget_bytes;
} hsma_server_stats_t;

int hsma_server_opts_default(hsma_server_opts *opts);

/* Plan parameters as in hsma_plan.  Errors as hsma_plan. */
int hsma_server_create(hsma_server_t *out, const double box[3], int bc, int p, double R, int Q, int Kmon,
                       const hsma_server_opts *opts);

/* Queue one configuration (host arrays, copied before return: xyz n x 3 in
 * the box frame, q n).  *ticket identifies it. */
int hsma_server_submit(hsma_server_t srv, int64_t n, const double *xyz, const double *q, int64_t *ticket);

/* Result of a ticket: with wait = 0 returns HSMA_E_AGAIN while it is not
 * ready; otherwise blocks.  energy, forces (host n x 3) and info may be NULL.
 * Returns the request's code; a ticket can be collected once
 * (HSMA_E_NOT_FOUND afterwards). */
int hsma_server_result(hsma_server_t srv, int64_t ticket, int wait, double *energy, double *forces,
                       hsma_request_info *info);

/* Withdraw a queued request: HSMA_OK (its result then reports
 * HSMA_E_CANCELLED), HSMA_E_AGAIN if it already runs or ran, HSMA_E_NOT_FOUND
 * for an unknown or collected ticket. */
int hsma_server_cancel(hsma_server_t srv, int64_t ticket);

int hsma_server_stats(hsma_server_t srv, hsma_server_stats_t *stats);

/* Finishes queued requests, then frees everything. */
void hsma_server_destroy(hsma_server_t srv);

/* ------------------------------------------------------- direct sums */
/* Coulomb sums of Sec. II.A (Phi_in) on their own:
 *   pot[t]   = sum_s q_s / |x_t - y_s|
 *   field[t] = sum_s q_s (x_t - y_s) / |x_t - y_s|^3
 * over ns sources (src: ns x 4 doubles x, y, z, q) and nt targets (tgt:
 * nt x 3), all device pointers.  A pair at distance exactly 0 is skipped.
 * field may be NULL.  precision as in hsma_precision (0 or 1).
 * stream: cudaStream_t or NULL.  Errors: HSMA_E_ARG, HSMA_E_OOM,
 * HSMA_E_CUDA. */
int hsma_coulomb_sum(int64_t ns, const double *src, int64_t nt, const double *tgt, double *pot,
                     double *field, int precision, void *stream);

/* Size of the device array hsma_coulomb_sum_static works in (32 MiB). */
#define HSMA_STATIC_SCRATCH_BYTES (32u << 20)

/* The sums of hsma_coulomb_sum, for callers that cannot allocate device
 * memory while they run -- for example a host application whose own memory
 * manager owns the whole device and forbids outside allocations after
 * start-up, or a time-critical loop that cannot afford the device-wide
 * synchronisation cudaFree implies.  The paper has no counterpart; this is a
 * deployment variant of the direct sum.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine: all working
 * memory is one static device array of HSMA_STATIC_SCRATCH_BYTES inside the
 * library, which every GPU that loads this part of the library keeps until
 * the process exits.  Arguments, layout and results are those of
 * hsma_coulomb_sum.  A call must fit in the array, roughly
 * 32 ns + 128 nt bytes (sources as two 16-byte words or one 32-byte FP64
 * record, targets with one partial-sum chunk); a larger call returns
 * HSMA_E_CAPACITY and does no work.  The array is shared by all calls on a
 * device and keeps what the last call left in it (each call first clears its
 * counters); calls whose device work overlaps -- two streams, two host
 * threads -- race on it and give wrong results, so serialise them.  The first
 * call on each device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The address is looked up again whenever the current context is a new one
 * (after a cudaDeviceReset, say), so the entry point stays usable then.
 * Returns once pot/field hold the results.
 * Errors: HSMA_E_ARG, HSMA_E_CAPACITY, HSMA_E_TIMEOUT, HSMA_E_CUDA. */
int hsma_coulomb_sum_static(int64_t ns, const double *src, int64_t nt, const double *tgt, double *pot,
                            double *field, int precision, void *stream);

/* Harmonic basis of Eq. "harmonic" at np points (device pointers; pts
 * np x 3, out np x (p+1)^2 row-major, FP64): the orthonormal real solid
 * harmonics (|x|/Rs)^n Y_nm, index k = n^2 + n + m, m > 0 the cosine and
 * m < 0 the sine part, without the Condon-Shortley phase; 0 <= p <= 40.
 * precision HSMA_FP64: the fully normalised recurrence in FP64 (relative
 * error ~1e-16 of the row's scale (|x|/Rs)^n); HSMA_FP32_ACC64: the same
 * recurrence in double-float arithmetic (pairs of FP32 words) on the FP32
 * pipe, faster on this part (whose FP64 issue rate is low) and accurate to
 * ~1e-14 of that scale; it scales each point by a power of two first, so it
 * does not underflow for points near the origin.  A point with a non-finite
 * coordinate gets non-finite values (NaN or infinity) wherever they depend
 * on it.  Allocates no device memory.  Returns once out holds the basis.
 * Errors: HSMA_E_ARG (p, Rs, np, null pointers, precision), HSMA_E_CUDA. */
int hsma_basis(int p, double Rs, int64_t np, const double *pts, double *out, int precision, void *stream);

/* ------------------------------------------------------ device peaks */
/* Measured FP32 throughput of the current device (no counterpart in the
 * paper): independent register-only FMA chains, scalar (fmaf) and packed
 * (fma.rn.f32x2, two lanes per instruction), 16 CTAs of 128 threads per SM,
 * best of three timed launches on a private stream.  Outputs: lane FMAs per
 * second (one FMA of one lane = 1).  Synchronous; takes ~10 ms.  Errors:
 * HSMA_E_ARG (NULL output), HSMA_E_CUDA. */
int hsma_fp32_peak(double *scalar_lane_ops_per_s, double *packed_lane_ops_per_s);

/* --------------------------------------------------------- inspection */
const char *hsma_strerror(int code);
const char *hsma_version(void);

/* Number of kernel launches this library has issued (all plans, all
 * threads) since it was loaded; graph replays count each kernel node. */
int64_t hsma_kernel_launches(void);

/* Number of device and pinned-host allocation and free calls (cudaMalloc,
 * cudaFree, cudaMallocHost, cudaFreeHost) this library has made since it was
 * loaded, over all plans and threads: a caller can check with it that a call
 * allocated nothing (no counterpart in the paper). */
int64_t hsma_allocation_calls(void);

/* Per-phase device times (milliseconds) of the plan's last update step,
 * when opts.profile was set: [0] in-set, [1] near-field pair sums,
 * [2] chunk reduction, [3] fit, [4] surface images, [5] surface pair sums,
 * [6] energy/forces, [7] total.  n: capacity of ms.  Returns the number of
 * entries written, or a negative code. */
int hsma_last_timings(hsma_plan_t plan, double *ms, int n);

/* Intermediates of the plan's last single-system update, copied to host
 * (FP64): which 0 = coefficients A (N_b, A_00 = 0 periodic), 1 = right-hand
 * side b (Kmon), 2 = Phi_in at the monitoring targets (n_mon_targets),
 * 3 = Phi_in at the particles (n), 4 = Phi_out at the particles (n).
 * Returns the number of values written or a negative code. */
int64_t hsma_last_get(hsma_plan_t plan, int which, double *host_out, int64_t count);

#ifdef __cplusplus
}
#endif

#endif /* HSMA_H */
