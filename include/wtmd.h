/*
 * wtmd.h -- C ABI of the B300 (sm_103a) well-tempered metadynamics
 * bias-force library (libwtmd.so).
 *
 * The calls follow the problem statement of the PySAGES paper
 * (arXiv 2301.04835):
 *   - a sampling method has an initialize step that allocates its state and an
 *     update step that advances it from the simulation's current snapshot
 *     (Sec. 2.1, SamplingMethod.build -> initialize/update): wtmd_create,
 *     cv_define, wtmd_bind, step_n;
 *   - the method's update runs inside the engine's time step as a force-like
 *     object whose biasing forces are added to the engine's net forces, with
 *     device-resident particle data and no host copies (Sec. 2, Snapshot and
 *     DLPack; Sec. 3.2.1 steps (a)-(f)): bias_eval, step_n;
 *   - metadynamics deposits Gaussian hills of width sigma at user-defined
 *     intervals, with fixed height (standard) or height scaled by a bias
 *     factor (well-tempered), optionally storing the bias on a grid
 *     (Sec. 2.1.5): hills_eval, wtmd_hills_load, wtmd_hills_read;
 *   - analyze turns the method's state into a free energy
 *     (Sec. 2, analyze; Sec. 2.1, Eq. (free-energy)): fes_grid;
 *   - CV gradients, obtained in the paper by automatic differentiation
 *     (Sec. 2, jax.grad), are a hand-written Jacobian and adjoint here:
 *     wtmd_cv_forward, wtmd_cv_adjoint.
 *
 * Conventions
 *   - Every call returns an int status: WTMD_OK (0) or a negative WTMD_E*
 *     code; wtmd_last_error() gives a message for the last failing call on a
 *     handle.  Calls are not thread-safe on one handle.
 *   - Precision is fixed per handle (WTMD_F32 or WTMD_F64).  "Real" below is
 *     float for WTMD_F32 and double for WTMD_F64.
 *   - Particle arrays (positions, velocities, forces) are DEVICE pointers to
 *     [n_atoms][4] Real (x, y, z, unused), 16-byte (F32) or 32-byte (F64)
 *     aligned.  They are borrowed: the caller owns them and keeps them alive
 *     while they are bound.  Walkers are contiguous, in walker order.
 *   - Every kernel is enqueued on the handle's stream (wtmd_set_stream;
 *     default: the legacy default stream).  Calls return after enqueueing;
 *     wtmd_check() synchronizes the stream and reports any error a kernel
 *     recorded (hill capacity, non-finite values, cell overflow, timeout).
 *   - Device memory of the handle (hills, grid, scratch, graphs) is owned by
 *     the handle and released by wtmd_destroy.
 */
#ifndef WTMD_H
#define WTMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define WTMD_OK 0
#define WTMD_EINVAL (-1)    /* bad argument, size, index or state */
#define WTMD_ENOMEM (-2)    /* device allocation failed */
#define WTMD_ECAPACITY (-3) /* hill list full: the deposit was skipped */
#define WTMD_ENUMERIC (-4)  /* a kernel saw a non-finite CV, bias or force */
#define WTMD_ETIMEOUT (-5)  /* a bounded device wait gave up */
#define WTMD_ECUDA (-6)     /* a CUDA runtime call failed */
#define WTMD_ECELL (-7)     /* a cell of the LJ cell list overflowed */

/* ---- enumerations ---- */
#define WTMD_F32 0
#define WTMD_F64 1

#define WTMD_ENGINE_NONE 0  /* no engine force (bias only) */
#define WTMD_ENGINE_MB 1    /* Mueller-Brown 2-D potential on (x, y); z frozen */
#define WTMD_ENGINE_LJ 2    /* 12-6 Lennard-Jones, cut and shifted at lj_rc */
#define WTMD_ENGINE_CHAIN 3 /* bead chain: harmonic bonds/angles, k(1+cos 3 phi) torsions */
#define WTMD_ENGINE_WELLS3 5 /* 3-D test landscape per particle: three Gaussian wells, depths
                              * (8, 6, 7), widths (0.45, 0.40, 0.50), centres (-1,0,0),
                              * (1,0.2,-0.3), (0.1,1.3,0.6), in a harmonic confinement
                              * (1.5/2)|r|^2 (a synthetic free-energy surface for CV-space
                              * runs that generate long hill lists) */

#define WTMD_CV_COMPONENT 1    /* one coordinate of one atom (Sec. 2.2, AxisCV Component) */
#define WTMD_CV_DIHEDRAL 2     /* IUPAC dihedral of 4 atoms (Sec. 2.2, FourPointCV DihedralAngle) */
#define WTMD_CV_COORDINATION 3 /* sum_{i in A} sum_{j in B, j != i} 1/(1+(r_ij/r0)^n) (rational switch, m = 2n) */
#define WTMD_CV_RG 4           /* radius of gyration of a group (Sec. 2.2, RadiusofGyration) */
#define WTMD_CV_QPAIRS 5       /* mean switching function over a fixed list of pairs */
#define WTMD_CV_DISTANCE 6     /* distance between the equal-mass centres of groups A and B (Sec. 2.2,
                                * TwoPointCV Distance); each group unwrapped by the minimum image
                                * relative to its first member, the centre difference by the minimum
                                * image; A and B non-empty and disjoint */
#define WTMD_CV_ANGLE 7        /* angle at a[1] between a[0] - a[1] and a[2] - a[1], in [0, pi]
                                * (Sec. 2.2, ThreePointCV Angle); gradient 0 at 0 and pi */
#define WTMD_CV_GYRATION 8     /* gyration tensor of group A (all atoms if n_a = -1), equal masses,
                                * unwrapped as for RG; eigenvalues l1 <= l2 <= l3; `axis` selects
                                * (Sec. 2.2, PrincipalMoment, Asphericity, Acylindricity,
                                * ShapeAnisotropy): */
#define WTMD_GY_L1 0           /*   smallest principal moment */
#define WTMD_GY_L2 1
#define WTMD_GY_L3 2           /*   largest */
#define WTMD_GY_ASPHERICITY 3  /*   l3 - (l1 + l2)/2 */
#define WTMD_GY_ACYLINDRICITY 4 /*  l2 - l1 */
#define WTMD_GY_ANISOTROPY 5   /*   3/2 (l1^2 + l2^2 + l3^2)/(l1 + l2 + l3)^2 - 1/2 */

#define WTMD_CV_INTENSIVE 1 /* RG only: divide by (group size)^(1/3) */

/* ---- configuration (copied by wtmd_create) ---- */
typedef struct wtmd_config {
    int32_t precision;      /* WTMD_F32 or WTMD_F64 */
    int32_t n_cv;           /* number of CVs d, 1..3 */
    double sigma[3];        /* Gaussian widths per CV (Sec. 2.1.5) */
    double w0;              /* initial hill height */
    double gamma;           /* bias factor; 0 selects standard metadynamics (fixed heights) */
    double kT;              /* thermal energy k_B T */
    int64_t stride;         /* deposit one hill per walker every `stride` steps; 0 = never */
    int64_t hill_capacity;  /* maximum number of hills */
    uint64_t seed;          /* Philox key of the thermostat noise */
    int32_t grid_bins[3];   /* cells per CV of the FP64 bias grid; all 0 = no grid */
    int32_t engine;         /* WTMD_ENGINE_* */
    double grid_lo[3];      /* grid range per CV (cell-centred cells) */
    double grid_hi[3];
    int32_t dims;           /* integrated spatial dimensions (2 or 3); 0 = 3 (2 for MB) */
    int32_t n_walkers;      /* number of walkers W (>= 1) */
    const int64_t* walker_size; /* host [W] atoms per walker (required; copied) */
    double dt, friction, mass;  /* BAOAB time step, friction (1/time), particle mass */
    double box[3];          /* periodic box edges; 0 = open in that direction */
    double lj_eps, lj_sigma, lj_rc;
    double bond_k, bond_r0, angle_k, angle_theta0, torsion_k;
} wtmd_config;

/* ---- one collective variable; indices are walker-local and host-side ---- */
typedef struct wtmd_cv_desc {
    int32_t kind;       /* WTMD_CV_* */
    int32_t axis;       /* COMPONENT: 0, 1 or 2; GYRATION: WTMD_GY_* */
    int64_t n_a;        /* group A size; -1 = all atoms of the walker (COORDINATION, RG) */
    const int32_t* a;   /* COMPONENT: 1 index; ANGLE: 3; DIHEDRAL: 4; COORDINATION/RG/GYRATION/DISTANCE: group A;
                           QPAIRS: 2*npairs indices (i0, j0, i1, j1, ...) */
    int64_t n_b;        /* COORDINATION partner group B size (-1 = all atoms); DISTANCE group B */
    const int32_t* b;
    double r0;          /* switching distance */
    int32_t nn, mm;     /* switching exponents; mm must equal 2*nn, nn even, 2..16 */
    double scale;       /* CV multiplier; 0 = default (COORDINATION 1/|A|, QPAIRS 1/npairs, else 1) */
    int32_t flags;      /* WTMD_CV_INTENSIVE */
    int32_t reserved;
    double period;      /* > 0: periodic CV (e.g. 2 pi for a dihedral); hill distances use the minimum image */
} wtmd_cv_desc;

typedef struct wtmd_t wtmd_t;

/* Create a handle: allocates the hill list (hill_capacity), the bias grid,
 * counters and per-walker scratch on the current CUDA device.
 * Errors: WTMD_EINVAL (bad config), WTMD_ENOMEM, WTMD_ECUDA. */
int wtmd_create(const wtmd_config* cfg, wtmd_t** out);

/* Release everything the handle owns (not the bound particle arrays). */
int wtmd_destroy(wtmd_t* h);

/* Message of the last error on this handle (never NULL). */
const char* wtmd_last_error(const wtmd_t* h);

/* Enqueue subsequent work on `stream` (a cudaStream_t; NULL = default). */
int wtmd_set_stream(wtmd_t* h, void* stream);

/* Define the next CV (ids 0..n_cv-1 in call order).  Index lists are copied
 * to the device.  Errors: WTMD_EINVAL (kind, index out of the walker, wrong
 * count, duplicate atoms, overlapping DISTANCE groups, GYRATION quantity
 * outside 0..5, mm != 2 nn, more than n_cv CVs). */
int cv_define(wtmd_t* h, const wtmd_cv_desc* desc, int32_t* cv_id);

/* Bind the engine's particle arrays (device, [n_atoms][4] Real).  n_atoms
 * must equal the sum of walker sizes.  Marks forces stale: the next step_n
 * first computes the total force at the bound positions. */
int wtmd_bind(wtmd_t* h, void* pos, void* vel, void* force, int64_t n_atoms);

/* Advance the bound system n_steps BAOAB steps: engine force, CVs, hills
 * sum, bias-force scatter into the force array, integration, and deposition
 * every `stride` steps (one hill per walker, well-tempered height).  Runs as
 * replays of a captured CUDA graph; no host synchronization inside.  Errors
 * recorded by kernels surface at wtmd_check(). */
int step_n(wtmd_t* h, int64_t n_steps);

/* Steps with the state in host memory (the paper keeps particle data on the
 * device, Sec. 2, Snapshot; this is the call for callers whose state lives
 * on the host).  in_host and out_host: [3][n_atoms][4] Real = positions,
 * velocities, forces (the forces must be those at the positions, as a
 * previous call returned them); out_host may equal in_host.  The state is
 * copied into the bound arrays, n_steps steps run, and the state is copied
 * back, all on the handle's stream.  When the bound arrays are one packed
 * [3][n_atoms][4] block, both buffers are pinned (page-locked) and
 * n_steps == 1, the copies and the step run as one captured CUDA graph
 * (captured on the first call with those buffers).  wait != 0 synchronizes
 * before returning; with wait == 0 the call returns after enqueueing and the
 * buffers must stay valid (and out_host unread) until the stream reaches
 * the copies.  Errors: WTMD_EINVAL (n_steps < 1, null buffers, arrays not
 * bound, CVs not all defined), those of step_n, WTMD_ECUDA. */
int wtmd_step_host(wtmd_t* h, const void* in_host, void* out_host, int64_t n_steps, int32_t wait);

/* Synchronize the handle's stream and return the first error a kernel
 * recorded since the last check (WTMD_ECAPACITY, WTMD_ENUMERIC, WTMD_ECELL,
 * WTMD_ETIMEOUT), or a CUDA error; clears the recorded status. */
int wtmd_check(wtmd_t* h);

/* One bias evaluation at `pos` (device [n_atoms][4] Real): CVs, hills sum over
 * the current hills, and force_inout -= J^T dV/dxi for every walker (force
 * may be NULL: nothing is scattered).  Outputs (device, may be NULL):
 * V_out [W] Real, xi_out [W][n_cv] Real, dV_out [W][n_cv] Real.  Does not
 * deposit and does not touch the bound arrays. */
int bias_eval(wtmd_t* h, const void* pos, void* force_inout, void* V_out, void* xi_out, void* dV_out);

/* CV values and Jacobians at `pos` (device [n_atoms][4] Real) for every
 * walker: xi_out (device [W][n_cv] Real).  The Jacobians are kept in the
 * handle for wtmd_cv_adjoint.  The paper obtains CV gradients with jax.grad
 * (Sec. 2); here they are written by hand. */
int wtmd_cv_forward(wtmd_t* h, const void* pos, void* xi_out);

/* Adjoint (vector-Jacobian product) of the CV map of the most recent
 * wtmd_cv_forward or bias_eval on this handle: grad_pos[i] =
 * sum_c grad_xi[w(i)][c] d xi_c / d r_i.  grad_xi: device [W][n_cv] Real;
 * grad_pos: device [n_atoms][4] Real, overwritten (w = 0).  With grad_xi =
 * -dV/dxi this is the bias force. */
int wtmd_cv_adjoint(wtmd_t* h, const void* grad_xi, void* grad_pos);

/* Hills sum alone at P points: xi (device [P][n_cv] Real) ->
 * V_out [P] Real, dV_out [P][n_cv] Real (device). */
int hills_eval(wtmd_t* h, const void* xi, int64_t P, void* V_out, void* dV_out);

/* Free-energy estimate on the grid: out (device, [prod grid_bins] double,
 * C order, last CV fastest) = -(gamma/(gamma-1)) V_grid (standard
 * metadynamics: -V_grid), shifted so that its minimum is 0.
 * Errors: WTMD_EINVAL (no grid, n_out too small). */
int fes_grid(wtmd_t* h, double* out, int64_t n_out);

/* ---- bias read from the grid ----------------------------------------------
 * The paper offers to keep the bias on a pre-defined grid to trade accuracy
 * for speed (Sec. 2.1.5); it stores the potential only.  Forces are taken
 * from it here as follows: the FP64 grid holds V at the cell centres
 * lo_i + (k + 1/2)(hi_i - lo_i)/bins_i; the gradient at a centre along axis
 * i is the central difference of its two neighbours (one-sided at the ends
 * of a non-periodic axis; a periodic axis wraps, and its grid must span
 * exactly one period); V and dV/dxi at a point are the multilinear
 * interpolations of the 2^d surrounding centres' values.  A non-periodic
 * coordinate outside the outermost centres is clamped to them (the edge
 * values hold).  The cost per point is fixed (2^d (2d + 1) grid reads)
 * instead of one Gaussian per hill; the error falls with the square of the
 * cell size relative to sigma. */
#define WTMD_BIAS_HILLS 0    /* exact sum over the hill list (default) */
#define WTMD_BIAS_GRID 1     /* read from the grid */
#define WTMD_BIAS_HARMONIC 2 /* harmonic windows (wtmd_harmonic) */

/* The grid-read bias at P points: xi (device [P][n_cv] Real) ->
 * V_out [P] Real, dV_out [P][n_cv] Real (device; either may be NULL).
 * Computed in FP64, rounded to Real.  Errors: WTMD_EINVAL (no grid, an axis
 * with fewer than 2 cells, bad sizes). */
int wtmd_grid_eval(wtmd_t* h, const void* xi, int64_t P, void* V_out, void* dV_out);

/* Select where step_n and bias_eval take V and dV/dxi from: WTMD_BIAS_HILLS,
 * WTMD_BIAS_GRID, or WTMD_BIAS_HARMONIC (after wtmd_harmonic).  With the grid, the well-tempered height of each new
 * hill also uses the grid's V, and hills are still appended to the list and
 * added to the grid.  Errors: WTMD_EINVAL (unknown source; for the grid: no
 * grid, an axis with fewer than 2 cells, a periodic CV whose grid does not
 * span one period, CVs not all defined, or the surrogate on).  Drops
 * captured step graphs; the persistent walker step follows the new source. */
int wtmd_bias_source(wtmd_t* h, int32_t source);

/* ---- harmonic bias and umbrella windows ------------------------------------
 * Harmonic biasing adds k/2 (xi - xi0)^2 to the Hamiltonian (Sec. 2.1.1);
 * umbrella sampling runs one such biased simulation per point of a path and
 * umbrella integration turns their statistics into a free-energy profile
 * (Sec. 2.1.2).  Here each walker is one window: V = sum_c k_c/2 (xi_c -
 * xi0_{w,c})^2, dV/dxi_c = k_c (xi_c - xi0_{w,c}) (minimum image on
 * periodic CVs), evaluated on the device in FP64 and rounded to Real; no
 * hills are deposited while it is on.  Every step adds each walker's CVs to
 * FP64 window sums on the device (bias_eval does not). */

/* Set the spring constants k (host [n_cv], > 0) and the window centres
 * (host [W][n_cv]), clear the window statistics and make the harmonic bias
 * the bias source.  Drops captured step graphs.  Errors: WTMD_EINVAL (CVs
 * not all defined, k <= 0, non-finite centres, surrogate on). */
int wtmd_harmonic(wtmd_t* h, const double* k, const double* centres);

/* Mean CVs of every window over the steps run since the last reset: mean_out
 * (host [W][n_cv], may be NULL), *n_samples (may be NULL) = steps counted;
 * reset != 0 clears the sums afterwards.  Synchronizes.  Errors: WTMD_EINVAL
 * (no windows set). */
int wtmd_umbrella_stats(wtmd_t* h, double* mean_out, int64_t* n_samples, int32_t reset);

/* Umbrella integration (Sec. 2.1.2) in its lowest order: the mean force of
 * window w is dA/dxi at its mean CV xi_bar_w, -k (xi_bar_w - xi0_w)
 * (minimum image on periodic CVs) -> mean_force_out (host [W][n_cv], may be
 * NULL); A along the path of the xi_bar_w in walker order is the
 * trapezoidal integral A_0 = 0, A_{w+1} = A_w + (g_w + g_{w+1})/2 .
 * (xi_bar_{w+1} - xi_bar_w) -> A_out (host [W], may be NULL).  Synchronizes.
 * Errors: WTMD_EINVAL (no windows, no samples). */
int wtmd_umbrella_integrate(wtmd_t* h, double* mean_force_out, double* A_out);

/* Replace the hill list by `count` hills from host memory [count][4] double
 * (s0, s1, s2, w); the grid is rebuilt from them.  Errors: WTMD_EINVAL
 * (count > capacity, w <= 0 or non-finite). */
int wtmd_hills_load(wtmd_t* h, const double* hills_host, int64_t count);

/* Copy the hill list to host memory [capacity_out][4] double; *count gets
 * the number of hills (synchronizes the stream). */
int wtmd_hills_read(wtmd_t* h, double* hills_host, int64_t capacity_out, int64_t* count);

/* Read the step counter and the hill count (synchronizes the stream). */
int wtmd_counters(wtmd_t* h, int64_t* step, int64_t* n_hills);

/* ---- checkpoint / restart --------------------------------------------------
 * The paper lists restarts as a capability still to be added to PySAGES
 * (Conclusion).  A checkpoint here is a host byte blob holding the
 * raw state a step reads: hill count, step counter, both hill layouts, the
 * FP64 grid, and the bound positions, velocities and forces.  The thermostat
 * noise is keyed by (seed, step, particle), so loading a checkpoint into a
 * handle made with the same configuration and CVs resumes the run bitwise.
 * The surrogate's network is not included (refused while it is on; its
 * weights are saved with wtmd_mlp_params), nor are umbrella-window sums.  The blob is in the byte order of
 * the machine that wrote it. */

/* Bytes needed by wtmd_checkpoint_save now (depends on the hill count).
 * Errors: WTMD_EINVAL (particle arrays not bound, surrogate on). */
int wtmd_checkpoint_size(wtmd_t* h, int64_t* bytes);

/* Write the checkpoint into host memory out[cap_bytes].  Synchronizes.
 * Errors: WTMD_EINVAL (cap_bytes too small, arrays not bound, surrogate on). */
int wtmd_checkpoint_save(wtmd_t* h, void* out, int64_t cap_bytes);

/* Restore a checkpoint (host memory in[n_bytes]) into this handle and its
 * bound arrays; the next step rebuilds the neighbour lists.  Synchronizes.
 * Errors: WTMD_EINVAL (not a checkpoint, truncated, or written by a handle
 * with another precision, CV count, walker count, atom count, hill capacity
 * or grid size; arrays not bound; surrogate on). */
int wtmd_checkpoint_load(wtmd_t* h, const void* in, int64_t n_bytes);

/* Copy the FP64 bias grid (device) to host memory [n_out] double. */
int wtmd_grid_read(wtmd_t* h, double* out_host, int64_t n_out);

/* Philox4x32-10 (Salmon et al., SC'11) on the device for n blocks: in_host
 * [n][6] uint32 (ctr0..3, key0..1) -> out_host [n][4] uint32.  Exposes the
 * generator behind the thermostat noise for bitwise checks. */
int wtmd_philox(const uint32_t* in_host, uint32_t* out_host, int64_t n);

/* Run n_steps eager (non-graph) MD steps with a CUDA event recorded on the
 * handle's stream after every kernel; return the mean time per kernel:
 * names [cap][32] (NUL-terminated) and ms [cap]; *n_marks = kernels per step.
 * Used to time kernels live for roofline reporting.  Synchronizes. */
int wtmd_profile_step(wtmd_t* h, int64_t n_steps, char* names, double* ms, int32_t cap, int32_t* n_marks);

/* Throughput probe of one SM pipe on the current device (not part of the
 * method): kind 0 = MUFU ex2.approx per second, kind 1 = FP32 FMA lane
 * operations per second (packed FFMA2 counted as two FMAs).  Gives the
 * measured denominators of the hills-sum roofline; *ms = kernel time. */
int wtmd_probe_peak(int32_t kind, double* ops_per_s, double* ms);

/* Check of the bounded device waits (failure detection without a fault): a
 * cooperative launch of `blocks` CTAs (1 per SM at most) in which CTA
 * `absent` leaves before the grid barrier (absent < 0: none leaves); the
 * others wait for its arrival, give up after limit_cycles SM cycles (1 ...
 * 2^31) and record the timeout.  *timed_out (host) receives 1 if the wait
 * gave up, else 0.  The device stays usable.  Errors: WTMD_EINVAL for bad
 * sizes, WTMD_ENOMEM, WTMD_ECUDA. */
int wtmd_barrier_probe(int32_t blocks, int32_t absent, int64_t limit_cycles, int32_t* timed_out);

/* Run each MD step of a multi-walker handle as one persistent (cooperative)
 * kernel launch: BAOAB, all-pairs LJ, coordination and Rg CVs, the bias at
 * every walker's CVs, bias force and deposition for every walker, with
 * bounded grid barriers between the phases.  The bias follows the handle's
 * source (wtmd_bias_source): the hills sum over the shared hill list, the
 * FP64 grid read (Sec. 2.1.5), or harmonic windows (wtmd_harmonic, Sec.
 * 2.1.1; one umbrella window per walker, Sec. 2.1.2, with the window sums
 * that wtmd_umbrella_stats reads).  The paper runs replicas as separate
 * simulations (Sec. 2, concurrent.futures / MPI); here walkers of uneven
 * size share one GPU launch and one hill list.  Each walker is either an
 * open cluster or, when the configured box has edges > 0, in its own
 * periodic box of that size (minimum-image pairs; Rg members unwrapped
 * relative to the walker's first atom).  Requirements: FP32, LJ engine, 1-2
 * CVs among COORDINATION (A = B = all) and RG (all atoms), walkers of at
 * most 8192 atoms, surrogate off; else WTMD_EINVAL.  enable = 0 returns to
 * the per-kernel step. */
int wtmd_walkers_persistent(wtmd_t* h, int32_t enable);

/* Bound of the grid-barrier waits of this handle's persistent launches (the
 * multi-walker step and the single-system step), in SM cycles: 0 restores
 * the default 2^31 (about a second at the maximum clock).  A wait that runs
 * out records a timeout that the next wtmd_check (or step_n with checking)
 * returns as WTMD_ETIMEOUT; every CTA then leaves the launch, the step's
 * results are not valid, and the handle stays usable (restore a checkpoint
 * to continue).  A short limit lets a test see that path.  Drops captured
 * step graphs when the limit changes.  Errors: WTMD_EINVAL outside
 * [0, 2^31]. */
int wtmd_wait_limit(wtmd_t* h, int64_t cycles);

/* The MD step of a single periodic system as one persistent (cooperative)
 * kernel launch per step (Sec. 3.2.1 steps (a)-(f) with the metadynamics
 * update of Sec. 2.1.5 inside): the first half of BAOAB, the LJ forces from
 * the Verlet lists (rebuilt in the same launch when an atom moved past half
 * the skin), the CVs, the hills sum, deposition, bias force and closing kick,
 * with bounded grid barriers between the phases and one CTA per SM.  Off by
 * default (the per-kernel step graph is faster at the sizes measured);
 * enable = 1 lets step_n and wtmd_step_host use it whenever the handle has
 * this form: FP32, one walker, LJ engine on the periodic cell lists, every
 * CV an FP32 tile coordination number (explicit list A) or a radius of
 * gyration (at most 1024 members), the bias summed from the hills (no
 * surrogate, grid or harmonic bias, no FP64 bias grid); other handles keep
 * the per-kernel sequence.  enable = 0 returns to the per-kernel sequence,
 * any other value leaves the setting; *active (host, may be NULL) receives 1
 * when the next step runs as one persistent launch, else 0.  Drops captured
 * step graphs when the setting changes.  Errors: WTMD_EINVAL for a null
 * handle. */
int wtmd_fused_step(wtmd_t* h, int32_t enable, int32_t* active);

/* Small FP64 systems in one CTA (Sec. 3.2.1 steps (a)-(f) with the
 * metadynamics update of Sec. 2.1.5): when the handle is FP64, its engine is
 * Mueller-Brown or the three wells, every CV is a COMPONENT, it has at most
 * 512 particles and 256 walkers (with the bias from the hills: at most 16
 * walkers and a hill capacity of at most 2048)
 * and the surrogate and the persistent walker step are off, step_n runs up
 * to 65536 steps per launch of one CTA that loops over the steps (the same
 * operations and Philox stream as the per-kernel step; the hills sum is
 * added in another fixed order).  On by default.  enable = 1 allows it,
 * 0 returns to the per-kernel step, -1 only queries; *active (host, may be
 * NULL) receives 1 when the next step runs that way.  Drops captured step
 * graphs when the setting changes.  Errors: WTMD_EINVAL for another enable. */
int wtmd_small_step(wtmd_t* h, int32_t enable, int32_t* active);

/* Autotuner of the persistent walker step: times every candidate (targets
 * per pair task 32/64/128/256, CTAs per SM 1/2/4, hill splits per CTA 1/2)
 * over `steps` steps from the same saved state, keeps the fastest, and
 * restores the state (positions, velocities, forces, hill count, step, grid),
 * so tuning does not advance the run.  choice (host [3], may be NULL)
 * receives the chosen (T, CTAs per SM, split factor).  Synchronizes. */
int wtmd_autotune(wtmd_t* h, int64_t steps, int32_t* choice);

/* Autotuner of the hills-sum launch plan (Sec. 2.1.5 sum; the plan splits the
 * hill list over CTAs and sets the hill lanes per point) for P evaluation
 * points: times every (lanes per point 1/4/32/256, splits 1 ... 1184)
 * candidate of the copy-ring kernel and, on FP32 handles with P <= 8, of
 * the few-points kernel (lanes per point reported as 0: every thread takes
 * whole hill pairs from global memory for all P points) and of the cluster
 * kernel (lanes per point reported as -1: one thread-block cluster of
 * `splits` = 8 or 16 CTAs whose split sums meet in distributed shared
 * memory) on the handle's current hills at P points placed at the CV
 * centre, and keeps the fastest for later sums with P points (step_n with
 * W = P walkers, bias_eval, hills_eval).  choice (host [2], may be NULL)
 * receives (lanes per point, splits); ms (host, may be NULL) the time of one
 * sum.  Synchronizes; drops captured step graphs.  Without tuning, FP32 sums
 * of P <= 8 points use the few-points kernel. */
int wtmd_hills_tune(wtmd_t* h, int64_t P, int32_t* choice, double* ms);

/* Set the hills-sum launch plan for P points instead of tuning it (the same
 * plans wtmd_hills_tune chooses from): lanes = hill lanes per point (1, 4,
 * 32 or 256: the copy-ring kernel), 0 (the few-points kernel) or -1 (the
 * cluster kernel; splits 8, or 16 where the device runs clusters of 16),
 * splits = CTAs the hill list is split over (1 ... 65535).  Lanes 0 and -1
 * need an FP32 handle and P <= 8.  Drops captured step graphs.  Errors:
 * WTMD_EINVAL for other values. */
int wtmd_hills_plan(wtmd_t* h, int64_t P, int32_t lanes, int32_t splits);

/* Hills sum for callers that cannot allocate device memory (the paper has no
 * counterpart: it is an interface for hosts such as an engine plugin that may
 * only touch the buffers it is given, or a caller whose memory footprint
 * must stay fixed after start-up).  Same quantity as hills_eval on a WTMD_F64
 * handle, without a handle: V_out[p] and dV_out[p][i] for P points xi
 * (device [P][n_cv] double) over n_hills hills (device [n_hills][4] double =
 * (s0, s1, s2, w), 32-byte aligned), widths sigma and periods period (host
 * [n_cv] double; period NULL or 0 = not periodic).  Calls no cudaMalloc,
 * cudaFree or other allocating routine: its partial sums use a fixed
 * library-owned device array of WTMD_STATIC_MAX_POINTS x 32 bytes (1 MiB)
 * that every GPU loading the library keeps until exit.  The first call in
 * each CUDA context (for most callers: the first call on each device, in its
 * primary context) looks the array's address up (cudaGetSymbolAddress) and
 * keeps it for that context; make that first call before any stream capture.
 * All calls share the array: calls whose kernels overlap on the GPU race, so
 * serialize them.  Work is enqueued on
 * `stream` (cudaStream_t, NULL = default).  Errors: WTMD_EINVAL when
 * P > WTMD_STATIC_MAX_POINTS, for bad sizes, sigma <= 0, negative periods,
 * null or misaligned pointers; WTMD_ECUDA if a CUDA call fails. */
#define WTMD_STATIC_MAX_POINTS 32768
int wtmd_hills_eval_static(int32_t n_cv, const double* sigma, const double* period, const double* hills,
                           int64_t n_hills, const double* xi, int64_t P, double* V_out, double* dV_out,
                           void* stream);

/* ---- MLP surrogate of the hills sum ----------------------------------------
 * The paper represents biases by neural networks in its ANN and FUNN methods
 * (Secs. 2.1.7 and 2.1.8); for metadynamics the hills sum (Sec. 2.1.5) is kept and a
 * network V_nn stands in for its older part only:
 *     V(xi) = V_nn(xi) + sum_{k >= K} w_k exp(-sum_i (xi_i - s_ki)^2 / (2 sigma_i^2)),
 * where V_nn approximates the sum over hills [0, K), K a multiple of 256.
 * V_nn(xi) = Vs * y((xi - mu) * inv_s) + Vm, y a 3 -> 64 -> 64 -> 1
 * perceptron with SiLU activations (z * sigmoid(z)); unused inputs (n_cv < 3)
 * are 0.  Parameters: 4481 FP32 numbers in the order W1 [64][3] (row j =
 * hidden unit j), b1 [64], W2 [64][64] (row i = output unit i), b2 [64],
 * w3 [64], b3; the kernels use them rounded to bfloat16 (nearest, ties to
 * even) with FP32 arithmetic.  Normalisation: norm[8] = mu[3], inv_s[3],
 * Vm, Vs.  FP32 handles only (else WTMD_EINVAL); not with the persistent
 * walker step. */
#define WTMD_MLP_PARAMS 4481

/* Enable (1) or disable (0) the surrogate in step_n and bias_eval.  When on,
 * the network is fitted at the next step_n (and again every `retrain_every`
 * new hills; 0 = only when asked by wtmd_surrogate_fit) on samples the run
 * generates: jittered copies (one sigma) of the most recent hill centres,
 * labelled by the exact FP32 hills sum over [0, K) (V and dV/dxi).  A tenth
 * of the samples is held out; the network part is used while the held-out
 * RMS error of V, after removing the mean offset, is <= tol_kT * kT, else the
 * exact sum over all hills is used (the fallback).  Synchronizes. */
int wtmd_surrogate(wtmd_t* h, int32_t enable, double tol_kT, int64_t retrain_every);

/* Training settings of later fits: samples per fit (rounded up to a multiple
 * of 10, >= 20), Adam iterations, batch size, learning rate (cosine decay to
 * lr/100 over the iterations of a fit) and the weight lambda of
 * the gradient term of the Sobolev loss
 *     L = mean_b (y_b - V_b)^2 + lambda * mean_b |grad_x y_b - G_b|^2
 * (targets scaled into the network's units). */
int wtmd_surrogate_config(wtmd_t* h, int64_t n_samples, int64_t iters, int64_t batch, double lr, double lambda);

/* Fit now (synchronous).  stats (host [8], may be NULL): K, held-out RMS
 * error of V in kT (after offset removal), its maximum in kT, relative RMS
 * error of dV/dxi, last training loss, 1 if the network part is in use,
 * number of fits so far, total Adam iterations.  With fewer than 512 hills
 * nothing is fitted and the exact sum stays in use. */
int wtmd_surrogate_fit(wtmd_t* h, double* stats);

/* The statistics of the last fit (host [8], as wtmd_surrogate_fit). */
int wtmd_surrogate_status(wtmd_t* h, double* stats);

/* Use the current network for hills [0, k0) (k0 a multiple of 256, within
 * capacity) without fitting, active = 1; active = 0 returns to the exact sum.
 * Turns the surrogate on with refits disabled. */
int wtmd_surrogate_set(wtmd_t* h, int64_t k0, int32_t active);

/* Load and/or read the network: in (host [4481] FP32, may be NULL) replaces
 * the master weights and resets the Adam state; norm_in (host [8], may be
 * NULL; Vs != 0) replaces the normalisation; out / norm_out (host, may be
 * NULL) receive the current master weights / normalisation.  Synchronizes. */
int wtmd_mlp_params(wtmd_t* h, const float* in, float* out, const double* norm_in, double* norm_out);

/* The network alone at P points: xi device [P][n_cv] double; V device [P]
 * float and dV device [P][n_cv] float (either may be NULL) receive V_nn and
 * dV_nn/dxi. */
int wtmd_mlp_eval(wtmd_t* h, const double* xi, int64_t P, float* V, float* dV);

/* Gradient of the Sobolev loss (wtmd_surrogate_config) over one batch of B
 * samples with respect to the 4481 parameters, at the bfloat16-rounded
 * weights: xi device [B][3] double (unused CVs 0), V device [B] float, dV
 * device [B][3] float (in CV units, unused 0); grad_out device [4482] float:
 * the gradient, then the loss.  Deterministic for a given GPU. */
int wtmd_mlp_grad(wtmd_t* h, const double* xi, const float* V, const float* dV, int64_t B, double lambda,
                  float* grad_out);

/* `iters` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on
 * the master weights; step t uses the batch of samples (t*B + b) mod n,
 * b < B, of the device arrays (layout as wtmd_mlp_grad).  loss_out (device
 * float, may be NULL) receives the last step's loss. */
int wtmd_mlp_train(wtmd_t* h, const double* xi, const float* V, const float* dV, int64_t n, int64_t B,
                   int64_t iters, double lr, double lambda, float* loss_out);

#ifdef __cplusplus
}
#endif

#endif /* WTMD_H */
