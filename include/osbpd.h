/*
 * osbpd.h -- C ABI of the GB300 (sm_103a) library for the per-time-step hot path of linearized
 * ordinary state-based peridynamics (OSB-PD), after T. Ni, M. Zaccariotto, Q. Zhu, U. Galvanetto,
 * "Matrix-based implementation and GPU acceleration of linearized ordinary state-based peridynamic
 * models in MATLAB", arXiv 2309.11273.
 *
 * One time step of the library evaluates, over every bond of every particle:
 *   - the bond-status update of the critical-stretch criterion (Eqs 1.17, 1.30);
 *   - the dilatation theta_i (Eq 1.6, discretized as the bond sum of Eq 2.3);
 *   - the linearized bond force of Eq 2.2 summed over the family (Eq 2.1);
 *   - the explicit update of Eq 2.11 with the diagonal mass rho V_i (Eq 2.12) and the boundary
 *     conditions of the solver loop (Appendix B).
 * The weighted volume m_i (Eq 1.9) and the damage denominator of Eq 1.31 are computed once when the
 * family is built.
 *
 * Conventions shared by every entry point:
 *   - Units are SI.  The influence function is w = 1 (Section 2.3).
 *   - Particle arrays are in the caller's particle order; internally the library reorders particles
 *     along a Morton curve and never exposes that order.
 *   - Vector fields are passed as "SoA" host arrays of dim * n doubles: first the n x-components, then
 *     the n y-components, then (3D only) the n z-components.
 *   - Every pointer argument is a HOST pointer unless its name ends in _dev.  Host arrays are owned
 *     by the caller, are read (or written) only during the call, and are never retained.
 *   - The library owns all device memory of a context (allocated with cudaMalloc on the context's
 *     device at creation / neighbour build, released by pd_destroy).
 *   - Every call returns a pd_status; on failure pd_last_error() describes it.  No C++ exception
 *     crosses the ABI.  A context must be used by one host thread at a time.
 *   - Asynchrony: calls that return data to host memory synchronize the context's stream before
 *     returning; pd_step only enqueues work (call pd_sync to wait).
 */
#ifndef OSBPD_H
#define OSBPD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pd_ctx pd_ctx;

typedef enum {
  PD_OK = 0,
  PD_ERR_ARG = -1,      /* invalid argument (null pointer, bad size, non-finite value, ...) */
  PD_ERR_STATE = -2,    /* call out of order (e.g. pd_step before pd_build_neighbors) */
  PD_ERR_OOM = -3,      /* a device or host allocation failed */
  PD_ERR_CUDA = -4,     /* a CUDA runtime call failed */
  PD_ERR_NUMERIC = -5,  /* the state became non-finite or exceeded the divergence guard */
  PD_ERR_TIMEOUT = -6   /* reserved for bounded device waits */
} pd_status;

/* Eq 1.8 / 1.15 / 1.16 rows. */
typedef enum { PD_3D = 0, PD_PLANE_STRESS = 1, PD_PLANE_STRAIN = 2 } pd_model;

/* PD_FP64: every operation in double precision (the paper computes in double precision, Section 4).
 * PD_MIXED: bond arithmetic (extension, stretch, dilatation and force sums) in FP32 with FP32
 *   accumulation; displacement and velocity integration in FP64; any bond whose FP32 stretch lies
 *   within a rigorous rounding bound of s0 is re-decided in FP64 from the FP64 displacement, so its
 *   status equals the FP64 decision on the run's own state. */
typedef enum { PD_FP64 = 0, PD_MIXED = 1 } pd_precision;

/* Bond kinematics.
 * PD_LINEARIZED: the paper's linearized model (Section 3, Eqs 2.2-2.4): extension e = M . (u_j - u_i)
 *   along the reference direction M = xi / |xi|, the small-deformation approximation of Eq 1.13.
 * PD_NONLINEAR: the state-based model of Section 2 without that approximation: Y = xi + u_j - u_i,
 *   e = |Y| - |xi| (Eq 1.10) and the force along the deformed bond M = Y / |Y| (Eq 1.13), with the
 *   force state of Eq 1.14 (as in the loop scheme of Appendix C).  Stretch for Eq 1.30: e / |xi|.
 *   With PD_MIXED the bond arithmetic is FP32 (fixed-point xi and the FP32 shadow of u in units of
 *   the quantum Q), the break test carries its own rounding band with the FP64 re-decision of
 *   PD_MIXED, and the staged kernels always run (PD_OPT_SPLIT and PD_OPT_STAGE are ignored). */
typedef enum { PD_LINEARIZED = 0, PD_NONLINEAR = 1 } pd_kinematics;

/* Influence function w(|xi|) of the weighted volume (Eq 1.9), the dilatation (Eq 1.6), the force
 * state (Eq 1.14, so the bond force of Eq 2.2) and the damage (Eq 1.31).
 * PD_W_ONE: w = 1, the paper's choice (Section 2.3).
 * PD_W_INV: w = delta / |xi|, a form of the published catalogue the paper refers to at Eq 1.9.
 *   Supported with linearized bonds and the explicit solver: in FP64 with the bond cache on (the
 *   default; w is folded into the per-slot tables) and in PD_MIXED on the lattice layout
 *   (PD_OPT_LATTICE; w is a per-direction factor).  Other combinations return PD_ERR_ARG.  The
 *   critical stretch of Eqs 1.26-1.29 (pd_critical_stretch) is derived for w = 1; s0 remains an
 *   input. */
typedef enum { PD_W_ONE = 0, PD_W_INV = 1 } pd_influence;

/* Internal particle order (results do not depend on it beyond rounding).
 * PD_ORDER_BRICKS: bricks of 32 x 4 x 4 (3D) or 32 x 8 (2D) points of the typical spacing
 *   (mean V)^(1/dim), x fastest inside a brick, bricks along a Morton curve: a warp's 32 particles
 *   form one row, so its neighbour gathers are contiguous on lattices.
 * PD_ORDER_MORTON: a Morton curve of the coordinates. */
typedef enum { PD_ORDER_BRICKS = 0, PD_ORDER_MORTON = 1 } pd_ordering;

typedef struct {
  int32_t model;       /* pd_model */
  int32_t precision;   /* pd_precision */
  double E;            /* Young's modulus [Pa] */
  double nu;           /* Poisson's ratio */
  double rho;          /* mass density [kg/m^3] */
  double horizon;      /* delta [m]; family = closed ball |xi| <= delta (Section 2.1) */
  double s0;           /* critical stretch s_c (Eq 1.30); <= 0 disables bond breaking */
  double dt;           /* time step [s] (Eq 2.11) */
  double band_safety;  /* PD_MIXED only: safety factor on the FP32 rounding bound; <= 0 -> 4 */
  int32_t device;      /* CUDA device ordinal */
  int32_t ordering;    /* internal particle order: PD_ORDER_BRICKS (0, default) or PD_ORDER_MORTON */
  void* stream;        /* cudaStream_t to run on, or NULL for a library-owned stream */
  int32_t kinematics;  /* pd_kinematics; every body of a batch takes the same */
  int32_t influence;   /* pd_influence (0: w = 1); every body of a batch takes the same */
} pd_params;

/* A pre-crack / notch: bonds whose segment crosses it are never created (Section 4.2 / 4.4).
 * 2D: the segment p0-p1 (p2 ignored).  3D: the parallelogram p0 + a (p1-p0) + b (p2-p0), a,b in
 * [0,1].  A bond i-j is cut iff x_i and x_j lie strictly on opposite sides of the crack's line /
 * plane and the crossing point lies on the closed segment / parallelogram.  body: in a batched
 * context the body it applies to (-1: all bodies); ignored otherwise. */
typedef struct {
  double p0[3], p1[3], p2[3];
  int32_t body;
  int32_t reserved;
} pd_crack;

typedef struct {
  int64_t steps;          /* time steps taken since creation */
  int64_t bonds;          /* directed bonds in the built family */
  int64_t broken_bonds;   /* directed bonds broken so far */
  int64_t band_rechecks;  /* PD_MIXED: bonds re-decided in FP64 (cumulative) */
  int64_t validate_mismatches; /* PD_MIXED with PD_OPT_VALIDATE: FP32+band vs pure FP64 decisions */
  double max_abs_u;       /* max |u| component at the last refresh */
  /* Diagnostics of the current state, evaluated in FP64 by pd_get_stats (two extra passes over the
   * bonds): */
  double min_rel_margin;  /* min |s - s0| / s0 over the intact breakable bonds (Eq 1.30; 1e300 if
                             none): how close the nearest bond is to its failure decision */
  double strain_energy;   /* sum_i V_i [(K - G/3)/(2A) theta_i^2 + G/(2 m_i) sum_j e_ij^2 V_j] over the
                             intact bonds (the energy whose derivative is the force of Eq 1.14) */
  double shadow_energy;   /* strain_energy + 1/2 sum_i rho V_i v_i^n . v_i^{n+1}, v^{n+1} the next
                             velocity of Eq 2.11 (free particles); for the linearized model without
                             loads, constraints or breaking it is conserved by the integrator */
} pd_stats;

/* Options for pd_set_option / pd_get_option. */
typedef enum {
  PD_OPT_GRAPH_CHUNK = 1,  /* steps captured per CUDA graph launch (0: no graphs). Default 100. */
  PD_OPT_PROFILE = 2,      /* 1: time every kernel launch with CUDA events (forces eager launches) */
  PD_OPT_VALIDATE = 3,     /* PD_MIXED: 1 = also decide every bond in FP64 and count mismatches */
  PD_OPT_BLOCK = 4,        /* threads per block of the step kernels (multiple of 32, <= 512) */
  PD_OPT_SPLIT = 5,        /* warps cooperating on one 32-particle slice: 1, 2 or 4 */
  PD_OPT_BOND_CACHE = 6,   /* PD_FP64: 1 (default) = keep per-bond tables of the reference
                              geometry and bond coefficients (xi, s0 |xi|^2, V_j xi,
                              G (1/m_i + 1/m_j) / |xi|^2, and the step's xi.(u_j - u_i); 72 bytes per
                              bond slot, plus a per-particle sum of V_j xi over the intact bonds) so
                              each step evaluates only displacement-dependent FP64 terms; 0 =
                              recompute the geometry from the coordinates every step.  With the
                              pair form, the first failure check before a read also keeps FP32
                              copies of xi and s0 |xi|^2 (16 bytes per slot) and of u (16 bytes
                              per particle) for its FP32 screen */
  PD_OPT_STAGE = 7,        /* PD_MIXED with split 1: 1 (default) = stream each warp's neighbour
                              indices and status words into shared memory with bulk asynchronous
                              copies (bounded waits; an expired wait makes the next pd_sync /
                              pd_get_* return PD_ERR_TIMEOUT); 0 = direct loads */
  PD_OPT_EXPIRE_WAITS = 8, /* testing the failure path: 1 = the staged kernels (PD_MIXED, split 1)
                              do not issue each warp's first index copy, so its bounded wait (1 s
                              of the GPU's global timer) expires; the warps skip their outputs
                              and the next pd_sync / pd_get_* returns PD_ERR_TIMEOUT.  Default 0. */
  PD_OPT_SOLVER = 9,       /* pd_solver: PD_SOLVER_EXPLICIT (0, default) or PD_SOLVER_ADR (1) */
  PD_OPT_PAIRS = 10,       /* PD_FP64 with the bond cache on: 1 (default) = form each bond's
                              extension (linearized: xi.(u_j - u_i); nonlinear: e and 1/|Y|) and
                              failure test once for its two directed entries (the failure check and
                              dilatation pass then runs as two kernels); 0 = once per entry.
                              Linearized results are bitwise the same, also when the option is
                              switched between steps; nonlinear theta sums differ in rounding
                              order only.  Has no effect when the build could not pair
                              every entry (pd_get_option then reports 0). */
  PD_OPT_LATTICE = 11,     /* PD_MIXED (linearized or nonlinear bonds): 1 (default) = when every
                              body's particles lie on a regular lattice (bond vectors h n with
                              integer n to within 2^-30 h, uniform volumes, a family |n|^2 <= m^2 for
                              an integer m from 3 to 5 in 3D or 8 in 2D: horizons from 3 h up to just
                              below sqrt(m^2 + 1) h), pd_build_neighbors lays the family out by
                              lattice direction (slot k of every slice = direction k for every lane)
                              and the step kernels take each slot's bond vector from a table instead
                              of gathering coordinates; 0 = the general layout and kernels.  Set before
                              pd_build_neighbors; after it, pd_get_option reports whether the built
                              layout is the lattice one. */
  PD_OPT_LAT_STAGE = 12,   /* lattice kernels: shared-memory ring of each warp's index and status
                              stream, 0 (default) = 3 chunks of 16 slots, 1 = 2 x 16, 2 = 3 x 8,
                              3 = 2 x 8 (smaller rings leave more of the SM's combined L1 / shared
                              memory to the displacement gathers); pd_autotune chooses it */
  PD_OPT_SHADOW_LO = 13    /* lattice kernels: 1 = carry each particle's FP32 displacement copy
                              (u / h) as two FP32 words hi + lo (lo the rounding remainder of hi,
                              16 more bytes per particle and per step gathered per bond in both
                              passes; linearized and nonlinear bonds), so that a bond's
                              u_j - u_i is rounded relative to
                              the difference rather than to |u| (bodies whose displacement is
                              large next to its variation over a horizon: rotations, rigid drift);
                              0 (default) = one word.  Decisions stay exact either way (the same
                              rounding band covers both).  May be set at any time; pd_get_option
                              reports 1 only while the built layout is the lattice one. */
} pd_option;

/* Solvers (PD_OPT_SOLVER).
 * PD_SOLVER_EXPLICIT: the dynamics of Eq 2.11 with time step pd_params.dt.
 * PD_SOLVER_ADR: adaptive dynamic relaxation for quasi-static solutions (the solver of the paper's
 *   Section 4.4, which cites it from the literature): every pd_step iteration solves
 *   L u'' + c L u' = f(u) + b with fictitious time step 1, a diagonal fictitious density
 *   lambda_i = R_i / 4 (R_i an upper bound of the absolute row sums of the force-density stiffness,
 *   so the unit step is stable) and the damping c = 2 sqrt(u.(k u) / u.u) over the free particles'
 *   components, k_ia = -(g_ia^n - g_ia^{n-1}) / (lambda_i v_ia^{n-1/2}) (g = f + b).  The first
 *   iteration after selecting the solver or pd_set_state starts from rest (v^{1/2} = g / (2 lambda)).
 *   pd_params.dt then only advances the boundary-condition clock (t_n = n dt), so a prescribed
 *   rotation grows by rate * dt per iteration (load stepping); a particle without bonds is held in
 *   place.  Bond failure is checked after every iteration as in the explicit solver.  With PD_MIXED
 *   the forces come from the FP32 bond arithmetic and the relaxation runs in FP64.  Single-body
 *   contexts only (PD_ERR_ARG otherwise).  With PD_OPT_PROFILE, the reduction and update
 *   kernels of an iteration are counted with PD_K_PASS2. */
typedef enum { PD_SOLVER_EXPLICIT = 0, PD_SOLVER_ADR = 1 } pd_solver;

/* Kernel identifiers for pd_get_profile.  With the FP64 pair form (PD_OPT_PAIRS) pass 1 is two
 * kernels: PD_K_PASS1 times the first (extension and failure check per pair), PD_K_PASS1B the
 * second (dilatation sum); otherwise PD_K_PASS1B records nothing. */
typedef enum { PD_K_PASS1 = 0, PD_K_PASS2 = 1, PD_K_PASS1B = 2, PD_K_COUNT = 3 } pd_kernel;

/* Critical stretch s_c from the critical energy release rate Gc [J/m^2] and the horizon (w = 1).
 *   3D: Eq 1.26 with beta = 125 delta / 1848 and beta' = 5 delta / 24.  Eq 1.27 prints
 *       beta' = 5 delta / (24 pi); integrating Eq 1.25 over the unit-weight sphere gives 5 delta / 24,
 *       which is the value used here.
 *   2D: Eq 1.28 with beta, beta' of Eq 1.29, as printed.
 * Returns a negative value for invalid arguments. */
double pd_critical_stretch(int32_t model, double E, double nu, double Gc, double delta);

/* Material constants of the model: A (Eq 1.8), K (Eq 1.15) and G (Eq 1.16) with the bulk and shear
 * moduli kappa = E / (3 (1 - 2 nu)), mu = E / (2 (1 + nu)).  Host helper (no context, no device).
 * PD_ERR_ARG for an unknown model, E <= 0, nu outside (-1, 0.5) or a NULL output. */
pd_status pd_material_constants(int32_t model, double E, double nu, double* A, double* K, double* G);

/* Creates a context for one body of n >= 1 particles (n <= 2^31 - 65).
 * x, y, z: reference coordinates (z must be NULL for 2D models and non-NULL for PD_3D).
 * vol: particle volumes V_i > 0 (required).  In 2D, V_i is the area times the thickness; the
 *      thickness cancels from u, v and damage.
 * Copies coordinates to the device; allocation failure -> PD_ERR_OOM. */
pd_status pd_create_particles(pd_ctx** out, const pd_params* prm, int64_t n, const double* x,
                              const double* y, const double* z, const double* vol);

/* Creates one context holding nbodies independent bodies that step together in the same kernels
 * (no bond ever joins two bodies).  Body b owns particles [body_offsets[b], body_offsets[b+1]) of
 * the concatenated arrays; per_body[b] gives its material, horizon, s0 and dt.  All bodies must
 * share model, precision, device and stream.  vol must be non-NULL. */
pd_status pd_create_batch(pd_ctx** out, int32_t nbodies, const pd_params* per_body,
                          const int64_t* body_offsets, const double* x, const double* y,
                          const double* z, const double* vol);

/* Builds the family of every particle on the device: closed horizon |xi| <= delta, minus the bonds
 * cut by the cracks; then m_i (Eq 1.9) and D_i = sum_j V_j (Eq 1.31 denominator) in FP64 over the
 * built family; every built bond starts intact.  Resets the state to u = v = 0.  May be called
 * again (rebuilds from scratch). */
pd_status pd_build_neighbors(pd_ctx* c, const pd_crack* cracks, int32_t ncracks);

/* Boundary conditions and loads (Appendix B applies the constraints at the top of every iteration).
 * flag[n]: 0 free, 1 fixed (u = v = 0), 2 prescribed rigid rotation: u = rate * t * a x (p - c),
 *          v = rate * a x (p - c), with c = axis_point, a = axis_dir (unit), t = step * dt.
 *          NULL: every particle free.
 * b: body-force density [N/m^3] as dim * n SoA, or NULL (zero).  axis_point / axis_dir may be NULL
 * when no particle is prescribed.  The constraints are applied to the current state at once. */
pd_status pd_set_bc(pd_ctx* c, const uint8_t* flag, const double* b, const double* axis_point,
                    const double* axis_dir, double rate);

/* Prescribed velocity field: every particle with flag 2 (pd_set_bc) then moves as u = t vp_i,
 * v = vp_i (t = step * dt) instead of the rotation of pd_set_bc: a constant velocity applied to
 * impacted nodes (Section 4.3).  vp: dim * n SoA in caller order (entries of other particles are
 * ignored).  PD_ERR_ARG for NULL or non-finite vp, PD_ERR_STATE before pd_set_bc marked prescribed
 * particles. */
pd_status pd_set_prescribed_velocity(pd_ctx* c, const double* vp);

/* Sets the displacement u (dim * n SoA, required) and velocity v (dim * n SoA, NULL: zero) and
 * applies the boundary conditions at the current time.  The next step does not apply the failure
 * criterion before its force evaluation (the paper applies it after each update, Appendix B).
 * PD_ERR_ARG (state unchanged) if u or v holds a non-finite value.  The new state replaces the old
 * after all work enqueued before the call; u and v may be reused when the call returns. */
pd_status pd_set_state(pd_ctx* c, const double* u, const double* v);

/* Advances nsteps >= 0 explicit time steps.  Per step: bond-status update on u^n (the failure block
 * that follows the previous update in Appendix B), dilatation, force, velocity / displacement
 * update with boundary conditions at t_{n+1}.  Runs as CUDA-graph chunks of PD_OPT_GRAPH_CHUNK
 * steps when graphs are enabled.  Enqueue only: returns before the GPU finishes.  A state that
 * became non-finite is reported by the next pd_sync / pd_get_* as PD_ERR_NUMERIC (a one-pass check
 * over the particles is enqueued after the steps). */
pd_status pd_step(pd_ctx* c, int64_t nsteps);

/* Waits for all work of the context. */
pd_status pd_sync(pd_ctx* c);

/* Applies the pending failure check to the current state (if a step ran since the last check) and
 * writes phi_i of Eq 1.31 in caller order (n doubles).  A particle without bonds gets 0. */
pd_status pd_get_damage(pd_ctx* c, double* phi);

/* Copies the state in caller order: u and v as dim * n SoA (FP64 master copies in PD_MIXED),
 * theta (n) = the dilatation evaluated by the last step.  Any of the three may be NULL.  Also
 * enqueues the pending failure check of the current state (none of the three depends on it); the
 * call returns when the copies are done, and later calls are ordered after the check. */
pd_status pd_get_state(pd_ctx* c, double* u, double* v, double* theta);

/* Number of directed bonds of the built family. */
pd_status pd_num_bonds(pd_ctx* c, int64_t* nbonds);

/* The built family in caller order as CSR (row_ptr: n + 1 int64, col: nbonds int32, neighbours in
 * ascending caller index) and, if intact != NULL, the bond status (1 intact, 0 broken) after the
 * pending failure check.  Inspection / testing aid; not on the hot path. */
pd_status pd_get_neighbors(pd_ctx* c, int64_t* row_ptr, int32_t* col, uint8_t* intact);

/* Counters (see pd_stats); synchronizes. */
pd_status pd_get_stats(pd_ctx* c, pd_stats* s);

/* Divergence guard: returns PD_ERR_NUMERIC if any displacement component is non-finite or larger
 * in magnitude than max_abs_u (> 0), PD_OK otherwise.  Synchronizes. */
pd_status pd_check_state(pd_ctx* c, double max_abs_u);

/* Picks the launch mapping (threads per block, warps per 32-particle slice) of the step kernels by
 * timing trial_steps steps of every candidate on the context's own data, keeps the fastest, and
 * restores the state, bond status and step count afterwards.  PD_FP64 contexts with the bond cache
 * also try both settings of PD_OPT_PAIRS for every mapping and keep the faster (read it back with
 * pd_get_option).  If the environment variable PD_AUTOTUNE_CACHE names a file, results are looked
 * up / appended there under a key made of the problem sizes, precision and device name.
 * *block / *split (may be NULL) receive the choice. */
pd_status pd_autotune(pd_ctx* c, int32_t trial_steps, int32_t* block, int32_t* split);

pd_status pd_set_option(pd_ctx* c, int32_t option, int64_t value);
pd_status pd_get_option(pd_ctx* c, int32_t option, int64_t* value);

/* With PD_OPT_PROFILE on: total device milliseconds and launch count of kernel `kernel` (pd_kernel)
 * since profiling was switched on or reset.  reset != 0 clears the counters after reading. */
pd_status pd_get_profile(pd_ctx* c, int32_t kernel, double* total_ms, int64_t* launches,
                         int32_t reset);

/* Measured FP64 fused multiply-add throughput of device `device` (not part of the method: the
 * denominator of the FP64 kernels' arithmetic roofline).  Runs `repeats` launches of a register-only
 * kernel (8 independent FMA chains per thread, 2048 threads per SM) and returns the rate in flop/s
 * (FMA = 2 flop) in *flops_per_s and the mean launch time in *ms_per_launch (may be NULL).  It
 * synchronizes, and allocates and frees 8 bytes of device memory.  Errors: PD_ERR_ARG, PD_ERR_CUDA. */
pd_status pd_probe_fp64(int32_t device, int32_t repeats, double* flops_per_s, double* ms_per_launch);

/* Number of particles, dimension and storage of the context (for sizing host buffers). */
pd_status pd_get_info(pd_ctx* c, int64_t* n, int32_t* dim, int64_t* device_bytes);

/* Checkpoint / resume (the paper has no counterpart; a library convenience for long runs).
 * pd_save_state writes the dynamic state -- u, v, the bond status, the step count and whether the
 * failure check on the current state is still pending -- to the file `path` (created or truncated),
 * with a header identifying the problem (a hash of the parameters, the particle positions and the
 * built family) and a checksum.  pd_load_state reads such a file into a context built the same way
 * (same particles, parameters and cracks; it may be a different context or process) and continues
 * exactly: N steps equal k steps, save, load, N - k steps, bit for bit.  The relaxation solver
 * restarts from rest after a load, as after pd_set_state.  Errors: PD_ERR_ARG for a path that cannot
 * be opened, a file that is not a checkpoint, a checksum mismatch or a problem that differs (the
 * context is then unchanged); PD_ERR_CUDA for device failures.  Both synchronize. */
pd_status pd_save_state(pd_ctx* c, const char* path);
pd_status pd_load_state(pd_ctx* c, const char* path);

/* pd_step_noalloc -- one explicit time step that allocates no memory at all.
 *
 * The paper has no counterpart; this is a library convenience for callers that cannot allocate
 * device memory: code inside a host framework whose allocator owns the whole device and hands out
 * fixed buffers, real-time loops that must never enter the allocator, or callers recording work
 * while allocation is forbidden.  Such callers cannot create a pd_ctx (which cudaMallocs its arrays).
 *
 * What it computes (on the calling thread's current device, on `stream`, enqueue only), for a body
 * with no constraints, no body force and no bond breaking: each particle's weighted volume over the
 * given family, its dilatation over the intact bonds, the linearized bond forces summed over the
 * intact bonds, and one explicit update of velocity then displacement:
 * v_out = v + dt F / (rho V), u_out = u + dt v_out.  Same model constants as pd_params.
 * Arguments (all arrays DEVICE memory of the current device, owned by the caller, in the caller's
 * particle order):
 *   x_dev, y_dev, z_dev (NULL unless PD_3D), vol_dev: n doubles each;
 *   row_ptr_dev (n + 1 int64), col_dev (row_ptr[n] int32): the family as CSR (e.g. from
 *   pd_get_neighbors); intact_dev: one byte per CSR entry (1 intact), or NULL for all intact;
 *   u_dev, v_dev -> u_out_dev, v_out_dev: dim * n SoA doubles; theta_dev: n doubles or NULL.
 *   No output (u_out, v_out, theta) may overlap another output or an input.
 *   stream: cudaStream_t or NULL (legacy default stream).
 * Limits: n <= 1,048,576.  Larger n returns PD_ERR_ARG with a message; so do NULL pointers, host
 * pointers, pointers to another GPU's memory and overlapping outputs (col and intact, whose length
 * the call does not read on the host, are checked at their first entry only).
 * Scratch: its one intermediate (2 doubles per particle) lives in a fixed 16 MiB device array that
 * every GPU loading the library holds until the process exits.  All calls share it and it keeps
 * the last call's contents (each call rewrites every entry it reads); calls that overlap on the GPU
 * race on it and must be serialized by the caller.  The first call on each device looks up that
 * array's device address (a runtime query, once per device): make that first call before any
 * stream capture.  Errors: PD_ERR_ARG, PD_ERR_CUDA (launch failure). */
pd_status pd_step_noalloc(int32_t model, double E, double nu, double rho, double dt, int64_t n,
                          const double* x_dev, const double* y_dev, const double* z_dev,
                          const double* vol_dev, const int64_t* row_ptr_dev, const int32_t* col_dev,
                          const uint8_t* intact_dev, const double* u_dev, const double* v_dev,
                          double* u_out_dev, double* v_out_dev, double* theta_dev, void* stream);

/* Thread-local description of the last failure on this host thread ("" if none). */
const char* pd_last_error(void);

/* Releases every resource of the context (NULL is ignored). */
void pd_destroy(pd_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* OSBPD_H */
