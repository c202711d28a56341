/*
 * osmpm.h - C ABI of the GB300 OS-MPM hot path.
 *
 * The library advances material-point domains with the implicit MPM step of
 * arxiv 2605.09097 Sec. 2.2 (APIC particle-to-grid transfer, backward-Euler
 * incremental potential minimised by Newton's method with a halving line
 * search, APIC grid-to-particle transfer with the deformation-gradient update
 * and advection) and couples a coarse and a fine domain with the overlapping
 * Schwarz alternating method of Sec. 3 and Alg. 1.  Every step runs in
 * hand-written CUDA kernels for sm_103a; nothing runs on the host but loop
 * control.
 *
 * Conventions (all entry points):
 *  - Every call returns an osmpm_status and never throws.  On failure the
 *    message is available from osmpm_last_error().
 *  - Domains are opaque and owned by the library.  Their device memory comes
 *    from the caller's allocator (or cudaMallocAsync when it is NULL) on the
 *    caller's CUDA stream, which every kernel of the domain is launched on.
 *  - Host arrays passed in are read during the call and not kept.  Output
 *    host arrays are caller-owned and written during the call.
 *  - Per-particle arrays are in the caller's particle order (the "id" order:
 *    index k of the input is particle id k).  The library keeps its
 *    particles sorted by the Morton code of their base grid node internally;
 *    every per-particle output is returned in id order.
 *  - Array layouts: x, v are n*dim doubles, particle-major (x[p*dim + a]);
 *    B, F are n*dim*dim doubles, particle-major then row-major
 *    (F[p*dim*dim + a*dim + b] = F_ab).  Grid fields are node-major with the
 *    node index i + res0*(j + res1*k) (x fastest), components innermost.
 *  - A failed osmpm_step or osmpm_schwarz_couple leaves the particles at the
 *    state they had at the start of the call, except for
 *    OSMPM_W_SCHWARZ_MAXITER, which commits the last Schwarz iterate.
 *  - Calls on one domain are not thread-safe.  To advance several domains
 *    concurrently, use osmpm_schwarz_couple_batch, which sizes the
 *    persistent PCG grids so that they can run side by side.
 */
#ifndef OSMPM_H
#define OSMPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum osmpm_status {
  OSMPM_OK = 0,
  OSMPM_E_INVALID = 1,         /* bad argument or descriptor */
  OSMPM_E_NOMEM = 2,           /* the allocator returned NULL */
  OSMPM_E_CUDA = 3,            /* a CUDA runtime call failed */
  OSMPM_E_NONFINITE = 4,       /* NaN/inf in inputs, or J <= 0 at an accepted iterate */
  OSMPM_E_NEWTON_MAXITER = 5,  /* Newton did not reach newton_tol in newton_max iterations */
  OSMPM_E_LINESEARCH = 6,      /* no energy decrease after ls_max halvings */
  OSMPM_E_OUT_OF_GRID = 7,     /* a particle's 3^dim support left the grid box */
  OSMPM_E_TIMEOUT = 8,         /* a device-side wait gave up (the kernel returned early) */
  OSMPM_E_UNSUPPORTED = 9,     /* a valid request the library does not serve */
  OSMPM_W_SCHWARZ_MAXITER = 100 /* Schwarz hit k_max; the last iterate was committed */
} osmpm_status;

/* Caller-supplied device allocator; alloc returns NULL on failure.  The
 * stream argument is the domain's cudaStream_t. */
typedef struct osmpm_allocator {
  void* (*alloc)(size_t bytes, void* ctx, void* stream);
  void (*free)(void* ptr, size_t bytes, void* ctx, void* stream);
  void* ctx;
} osmpm_allocator;

/* Description of one domain: its background grid (Sec. 2.2.2; node
 * (i,j,k) sits at origin + dx*(i,j,k), res nodes per axis), body force and
 * solver controls (Sec. 2.2.5). */
typedef struct osmpm_domain_desc {
  int32_t dim;              /* 2 or 3 */
  int32_t precision;        /* 0: FP64 throughout; 1: mixed - particle v, B, F stored in
                               FP32, the PCG's Hessian-vector product (per-particle Hessian
                               blocks, grad N, arithmetic) in FP32; positions, grid vectors,
                               the Newton residual, line-search energy change, PCG dot
                               products and Schwarz residuals stay FP64 */
  double origin[3];
  double dx;
  int32_t res[3];           /* nodes per axis; each >= 4 */
  double gravity[3];        /* body-force acceleration g (f_ext = m_i g) */
  double newton_tol;        /* stop when max |delta x_hat| / dt <= newton_tol */
  int32_t newton_max;       /* Newton iteration cap */
  double cg_rtol;           /* PCG stops when |r| <= cg_rtol |r_0| */
  int32_t cg_max;           /* PCG iteration cap per Newton iteration */
  int32_t ls_max;           /* line search tries alpha = 1, 1/2, ..., 2^-ls_max */
  double mass_eps;          /* active nodes (the set N of Sec. 3.2.1): m_i > mass_eps >= 0 */
  double cg_eta_max;        /* inexact Newton: PCG stops at eta |r_0|, eta = |g_k|/|g_0|
                               clamped to [cg_rtol, cg_eta_max]; 0 means 1e-3; < 1 */
  int32_t pcg_mode;         /* 0: automatic (the persistent single-launch PCG when one
                               co-resident pass covers the problem, else the streaming
                               PCG of three kernels per iteration); 1: persistent;
                               2: streaming */
  int32_t launch_mode;      /* 0: each Newton iteration's device work (gradient, Jacobi
                               diagonal, persistent PCG, max |delta|, scalar read-back) is
                               captured once per (dt, iteration kind, PCG shape) as a CUDA
                               graph and replayed; 1: plain stream launches.  Streaming PCG
                               solves, domains on the legacy default stream (which
                               cannot be captured) and the worker threads of
                               osmpm_schwarz_couple_batch always launch directly.
                               Results do not depend on it */
  int32_t hvp_mode;         /* Hessian-vector product of the streaming PCG in mixed
                               precision: 0 automatic (= 2); 1: lane groups over the
                               stencil gradients cached at P2G and the Hessian blocks
                               cached by the gradient kernel; 2: block tiles - each block
                               stages the grid nodes its Morton-sorted particles touch in
                               shared memory (gathers and a shared scatter, one global
                               atomic per tile node and component) and recomputes the
                               particle Hessian from the Newton iterate.  FP64 domains
                               always use 1 */
  int32_t reserved[3];      /* must be zero */
} osmpm_domain_desc;

/* Initial particle state, host arrays in id order (layouts above).  flags
 * bit 0 marks the boundary particle layer P_alpha^partial of Sec. 3.2.1. */
typedef struct osmpm_particles_in {
  int64_t n;
  const double* x;
  const double* v;
  const double* B;          /* APIC affine matrix B_p */
  const double* F;          /* deformation gradient F_p */
  const double* vol0;       /* V_p^0 */
  const double* mass;       /* m_p */
  const double* E;          /* Young's modulus */
  const double* nu;         /* Poisson's ratio, < 0.5 */
  const uint8_t* flags;
} osmpm_particles_in;

/* Prescribed grid-node velocity (Dirichlet data of Eqs. implicit_solve_coarse
 * and implicit_solve_fine) on the nodes whose position lies in the closed box
 * [lo, hi].  kind 0: velocity vel on the components set in comp_mask.
 * kind 1: all components follow the rigid rotation by omega*dt about the
 * axis through center along axis (in 2D: about z), v = (R - I)(x - c)/dt.
 * Later rules override earlier ones on the components they set. */
typedef struct osmpm_dirichlet {
  int32_t kind;
  uint32_t comp_mask;
  double lo[3], hi[3];
  double vel[3];
  double center[3];
  double axis[3];
  double omega;
} osmpm_dirichlet;

/* Schwarz controls (Sec. 3): sub-cycling ratio M = dT/dt, iteration cap
 * k_max (Alg. 1 runs k = 0..k_max), interface tolerance eps_conv (Eq.
 * convergence_criterion), boundary-node mass thresholds tau_Gamma per grid
 * (Eq. boundary_grid_set) and the projection regulariser eps_tol (Eq.
 * spatial_projection).  pi_source picks the fine state v_S^(k) that Pi_{S->B}
 * projects for the coarse solve of iteration k >= 1 (Eq.
 * implicit_solve_coarse; k = 0 always projects the fine P2G at t_n):
 *   OSMPM_PI_STEP_AVERAGE (0): the solved fine grid velocities of the M
 *     sub-steps averaged over the coarse step, mass- and momentum-weighted,
 *     (1/M) sum_m m^(m) v^(m) over (1/M) sum_m m^(m); the coarse boundary
 *     then moves with the fine material over the same dT;
 *   OSMPM_PI_LAST_SUBSTEP (1): the fine P2G grid that ends sub-step M (the
 *     velocity of the last dt only; with M > 1 the two grids drift apart
 *     during transients, see the validation tests). */
enum { OSMPM_PI_STEP_AVERAGE = 0, OSMPM_PI_LAST_SUBSTEP = 1 };
typedef struct osmpm_schwarz_desc {
  int32_t M;
  int32_t k_max;
  double eps_conv;
  double tau_B;
  double tau_S;
  double eps_tol;
  int32_t pi_source;        /* OSMPM_PI_STEP_AVERAGE or OSMPM_PI_LAST_SUBSTEP */
  int32_t reserved[7];      /* must be zero */
} osmpm_schwarz_desc;

typedef struct osmpm_stats {
  int32_t newton_iters;     /* summed over every solve of the call */
  int32_t cg_iters;         /* summed over every PCG of the call */
  int32_t ls_halvings;
  int32_t schwarz_iters;    /* k* + 1, 0 for osmpm_step */
  int32_t solves;           /* implicit solves performed */
  int32_t converged;        /* Schwarz converged (1) or hit k_max (0) */
  double r_B, r_S;          /* last interface residuals */
  double last_dx_inf;       /* max |delta x_hat| of the last Newton iteration */
  int32_t contact_sets;     /* active sets of the rigid-plane contact (0 without a plane) */
  int32_t pad;
  double reserved[5];
} osmpm_stats;

typedef struct osmpm_domain osmpm_domain;

/* Creates a domain: validates the descriptor and particles, copies the
 * particles to the device (allocator, stream), sorts them by the Morton code
 * of their base node (ties keep id order) and computes the Lame parameters
 * mu = E/(2(1+nu)), lam = E nu/((1+nu)(1-2nu)).  Errors: OSMPM_E_INVALID
 * (among others a particle count outside [1, 2^31 - 1], nu outside (-1, 0.5),
 * a non-positive mass or volume), OSMPM_E_NONFINITE, OSMPM_E_OUT_OF_GRID,
 * OSMPM_E_NOMEM, OSMPM_E_CUDA. */
osmpm_status osmpm_create_domain(const osmpm_domain_desc* desc,
                                 const osmpm_particles_in* particles,
                                 const osmpm_allocator* allocator,
                                 void* cuda_stream,
                                 osmpm_domain** out);

/* Frees the domain's device memory (through its allocator, on its stream). */
osmpm_status osmpm_destroy_domain(osmpm_domain* dom);

/* Replaces the domain's physical Dirichlet rules (n_rules may be 0). */
osmpm_status osmpm_set_dirichlet(osmpm_domain* dom, const osmpm_dirichlet* rules,
                                 int32_t n_rules);

/* Rigid frictionless plane y = level under a 2D domain (the rigid plane of
 * Sec. 4.2; the paper gives no contact treatment).  Reading: a unilateral,
 * gap-aware Signorini condition on the normal motion of the candidate grid
 * nodes (y_i <= cand_hi, active, no physical rule on y, some particle within
 * `spacing` of the node's column in x): over one step u_iy >= -gap_i, where
 * gap_i = max(0, (lowest such particle's y - spacing/2) - level); the
 * tangential motion stays free.  osmpm_step then solves the contact by a
 * primal-dual active set: Newton with u_iy = -gap_i held on the active
 * nodes, multipliers lambda_i = dE_h/du_iy (the plane's force on node i)
 * from the gradient with every active DOF free, release of held nodes with
 * lambda_i < 0 and holding of free candidates with u_iy < -gap_i, until the
 * set stops changing (at most max_sets solves; 0 means 50; then
 * OSMPM_E_NEWTON_MAXITER).  The first set holds the nodes whose gap is
 * closed.  enabled = 0 removes the plane.  Errors: OSMPM_E_UNSUPPORTED in
 * 3D; osmpm_schwarz_couple refuses a domain with a plane.  The reverse mode
 * holds the last active set fixed, like the Dirichlet DOFs. */
typedef struct osmpm_plane {
  int32_t enabled;
  int32_t max_sets;
  double level;      /* the plane y = level; the body lies above it */
  double cand_hi;    /* candidate nodes: y_i <= cand_hi */
  double spacing;    /* particle spacing: column width and gap offset */
} osmpm_plane;
osmpm_status osmpm_set_plane(osmpm_domain* dom, const osmpm_plane* plane);

/* One backward-Euler MPM step of a single domain (Sec. 2.2): P2G (Eq.
 * p2g_transfer), Newton with line search on E_h (Eq. discrete_energy,
 * Sec. 2.2.5) with a Jacobi-preconditioned matrix-free CG whose
 * Hessian-vector product is a particle gather-scatter, then G2P, F update
 * and advection (Eqs. g2p_v, g2p_B, F_update, advection).  stats may be
 * NULL. */
osmpm_status osmpm_step(osmpm_domain* dom, double dt, osmpm_stats* stats);

/* One global step dT of the overlapping Schwarz method, Alg. 1: coarse
 * domain solved over dT with Pi_{S->B} data on its receiver nodes, fine
 * domain reset and sub-cycled M times with T_m(I_{B->S}) data, until both
 * interface residuals are <= eps_conv (k >= 1) or k = k_max; then the coarse
 * particles take one G2P (Sec. 3.5).  Both domains must have the same dim
 * and stream; coarse dx >= fine dx.  Returns OSMPM_W_SCHWARZ_MAXITER when
 * k_max was reached (state committed).  stats may be NULL. */
osmpm_status osmpm_schwarz_couple(osmpm_domain* coarse, osmpm_domain* fine, double dT,
                                  const osmpm_schwarz_desc* sdesc, osmpm_stats* stats);

/* Batched global steps (not in the paper; a service for running many
 * independent OS-MPM instances): advances the n coupled pairs (coarse[i],
 * fine[i]) by one global step dT each with its Schwarz controls sdesc[i]
 * (n descriptors), as osmpm_schwarz_couple does, with
 * up to n_threads host worker threads (0: 8) driving the pairs
 * concurrently; each pair must own its two domains and should have its own
 * stream, so that kernels of different pairs overlap on the GPU.  While the
 * call runs, each pair's persistent PCG grid is limited to 3/4 of
 * 1/n_threads of the device's co-resident capacity, so that the concurrent
 * cooperative grids can all be resident together with room to spare for
 * the other pairs' ordinary kernels (their grid barriers never wait on a
 * block another grid keeps out).  The worker threads launch directly
 * (launch_mode 0 graphs are built and replayed only by calls made from the
 * caller's thread).  A pair whose PCG reports OSMPM_E_TIMEOUT (a grid
 * barrier gave up waiting) is back at t_n and runs its step once more on
 * half that grid.  Calls that drive domains concurrently
 * from several host threads must go through this entry point.  stats and
 * status (either may be NULL) receive n entries.  Returns OSMPM_OK, or the
 * status of the first failing pair (message names the pair), or
 * OSMPM_W_SCHWARZ_MAXITER when some pair hit k_max and none failed. */
osmpm_status osmpm_schwarz_couple_batch(osmpm_domain* const* coarse, osmpm_domain* const* fine,
                                        int32_t n, double dT, const osmpm_schwarz_desc* sdesc,
                                        int32_t n_threads, osmpm_stats* stats,
                                        osmpm_status* status);

/* A new non-blocking CUDA stream on the current device, for callers without
 * a stream factory of their own (every pair of osmpm_schwarz_couple_batch
 * wants its own stream).  *out receives the cudaStream_t; release it with
 * osmpm_destroy_stream after the domains that use it are destroyed.  Errors:
 * OSMPM_E_INVALID (null out), OSMPM_E_CUDA. */
osmpm_status osmpm_create_stream(void** out);
osmpm_status osmpm_destroy_stream(void* stream);

/* Launch-shape autotuner of the batched path (not in the paper): picks the
 * host concurrency of osmpm_schwarz_couple_batch for these pairs, which
 * also sets each pair's persistent PCG grid (1/n_threads of the device's
 * co-resident blocks).  It runs one untimed batched step with candidates[0]
 * and then one timed batched step per candidate (host wall clock, the
 * device synchronised on both sides); these are real global steps, so the
 * pairs advance by n_candidates + 1 steps.  A step's cost varies with the
 * Schwarz, Newton and PCG iterations it needs, so each candidate is scored
 * by wall time per PCG iteration summed over the pairs; *best receives the
 * candidate with the lowest score, us_per_cg_iter (may be NULL) the
 * n_candidates scores in microseconds.  candidates must be >= 1.  Errors:
 * OSMPM_E_INVALID for bad arguments, else the first failing step's status
 * (a pair reaching k_max is not a failure). */
osmpm_status osmpm_autotune_batch(osmpm_domain* const* coarse, osmpm_domain* const* fine,
                                  int32_t n, double dT, const osmpm_schwarz_desc* sdesc,
                                  const int32_t* candidates, int32_t n_candidates,
                                  int32_t* best, double* us_per_cg_iter);

/* Batched OS-MPM with one PCG service (the project's batching line, not a
 * passage of the paper; mixed-precision domains).  Advances n independent
 * pairs by one global step each, like osmpm_schwarz_couple_batch (host
 * threads drive the pairs' Alg. 1 and Newton loops on their own streams),
 * but no pair launches a PCG of its own: each Newton system goes to a
 * service thread, which solves every system handed in meanwhile with one
 * batched Jacobi PCG (the streaming PCG with the block-tiled
 * Hessian-vector product) over a work list of (pair's domain, particle
 * tile) and (pair's domain, DOF tile), each system with its own scalars
 * and stopping test; the iterations run in chunks (one CUDA graph reads
 * the work list from device memory), with a look at the stop flags after
 * each: converged systems leave and systems handed in meanwhile join
 * between chunks.  Results per pair are those of osmpm_schwarz_couple
 * within the solver tolerances.
 *  - desc: n_threads host threads (0: 32), dof_tile DOFs per DOF tile
 *    (0: 2048), chunk iterations per graph replay (0: 16), slot_tiles
 *    slot tiles (128 particle slots each) per work item of the
 *    Hessian-vector product (0: 1).
 *  - stats / status per pair as for osmpm_schwarz_couple_batch; ms (may be
 *    NULL) receives the service's counters.
 * Errors: OSMPM_E_UNSUPPORTED unless every domain is mixed precision (1)
 * and all share one dimension; OSMPM_E_INVALID for bad arguments. */
typedef struct osmpm_multi_desc {
  int32_t n_threads;
  int32_t dof_tile;
  int32_t chunk;
  int32_t slot_tiles;
} osmpm_multi_desc;

typedef struct osmpm_multi_stats {
  int64_t batches;     /* compositions of the running set: each time systems
                          join or leave, its tables are rebuilt */
  int64_t instances;   /* Newton systems solved */
  int64_t chunks;      /* chunks of iterations (graph replays) */
  int64_t max_batch;   /* most systems iterating together */
  int64_t particles;   /* particles of the systems solved, summed */
  int64_t dofs;        /* grid DOFs of the systems solved, summed */
  int64_t iterations;  /* PCG iterations, summed over the systems */
  int64_t particle_iterations;  /* sum over the systems of iterations x particles */
  int64_t dof_iterations;       /* sum over the systems of iterations x grid DOFs */
  double device_ms;    /* device time of the batched PCGs (CUDA events) */
  double hvp_ms;       /* durations of the timed batched Hessian-vector product */
  int64_t hvp_launches;  /* launches (k_m_hvp; those of every 8th chunk are timed) */
  int64_t hvp_particle_iterations;  /* particle-iterations of the timed launches */
} osmpm_multi_stats;

osmpm_status osmpm_schwarz_couple_multi(osmpm_domain* const* coarse, osmpm_domain* const* fine,
                                        int32_t n, double dT, const osmpm_schwarz_desc* sdesc,
                                        const osmpm_multi_desc* desc, osmpm_stats* stats,
                                        osmpm_status* status, osmpm_multi_stats* ms);

/* Launch-shape autotuner of osmpm_schwarz_couple_multi: runs one untimed
 * and then one timed multi step per candidate descriptor (host threads, DOF
 * tile, iterations per graph replay, slot tiles per product work item);
 * these are real global steps, so the
 * pairs advance by n_candidates + 1 steps.  Scored by wall time per PCG
 * iteration summed over the pairs; *best receives the index of the best
 * candidate, us_per_cg_iter (may be NULL) the n_candidates scores. */
osmpm_status osmpm_autotune_multi(osmpm_domain* const* coarse, osmpm_domain* const* fine,
                                  int32_t n, double dT, const osmpm_schwarz_desc* sdesc,
                                  const osmpm_multi_desc* candidates, int32_t n_candidates,
                                  int32_t* best, double* us_per_cg_iter);

/* Reverse mode, recording.  enable = 1 discards any earlier record and
 * makes every later osmpm_step of dom keep, in device memory from the
 * domain's allocator, its input particle state (x, v, B, F), its converged
 * grid displacement u* and its free-DOF mask (about 12 doubles per particle
 * and 2-3 per grid node and step, in 2D); enable = 0 stops and frees the
 * record.  When both domains of osmpm_schwarz_couple record, the coupled
 * step is recorded on the coarse domain instead (its start states, every
 * coarse solve and fine sub-step it ran, the projection sums).  A record
 * holds single-domain steps or coupled steps of one pair, not both;
 * mixing them, osmpm_set_particles, a mixed-precision domain or the
 * last-sub-step projection interrupts it, and osmpm_adjoint refuses an
 * interrupted record.
 *
 * Step checkpointing: enable = K >= 2 records only the particle state at
 * the start of every K-th step (for coupled steps both domains', on the
 * coarse domain, whose K counts) and every step's controls (dt or dT, the
 * Schwarz descriptor, the Dirichlet rule sets in force).  osmpm_adjoint then
 * works through the record one segment of K steps at a time, last segment
 * first: it re-runs the segment's steps from its checkpoint with the full
 * record, reverses them and frees that record.  Memory: the N/K checkpoints
 * plus one segment's full record, for about one extra forward pass.  The
 * re-run steps repeat the recorded ones up to the rounding order of the
 * atomic sums (the gradient is that of the re-run trajectory).
 * Errors: OSMPM_E_UNSUPPORTED for a mixed-precision domain (the adjoint
 * differentiates the FP64 trajectory); OSMPM_E_INVALID for enable < 0. */
osmpm_status osmpm_record(osmpm_domain* dom, int32_t enable);

/* Outputs of osmpm_adjoint: device arrays of the caller, in particle-id
 * order, particle-major (entry (p, a) at p*dim + a; (p, a, b) at
 * (p*dim + a)*dim + b).  dJ_dE is required; the adjoints of the state at the
 * start of the record may be NULL. */
typedef struct osmpm_adjoint_out {
  double* dJ_dE;    /* n: dJ / dE_p (Young's modulus of particle p) */
  double* dJ_dx0;   /* n*dim or NULL */
  double* dJ_dv0;   /* n*dim or NULL */
  double* dJ_dB0;   /* n*dim*dim or NULL */
  double* dJ_dF0;   /* n*dim*dim or NULL */
} osmpm_adjoint_out;

/* Reverse-mode gradient of an objective J of the particle positions after
 * the recorded steps (dJ_dx: device, n*dim, id order, particle-major) with
 * respect to every particle's Young's modulus, through the recorded
 * backward-Euler steps (Sec. 2.2).  Per step, last to first: the transposed
 * G2P, F update and advection (Eqs. g2p_v, g2p_B, F_update, advection), one
 * adjoint PCG K lam = u_bar on the free DOFs with the step's own symmetric
 * Hessian-vector product (the implicit function theorem at the converged
 * Newton solve, Sec. 2.2.5; stopped at cg_rtol |u_bar|), the lam-weighted
 * derivatives of the Newton residual (Eq. grid_residual) with respect to
 * F_p, the moduli, x_p, the nodal mass and velocity, and the transposed APIC
 * P2G (Eq. p2g_transfer).  The active node set and the Dirichlet DOFs of each
 * step are held fixed.  The domains' states are unchanged and the record kept
 * (several objectives may be differentiated).
 *
 * fine == NULL: coarse is a domain whose osmpm_step calls were recorded.
 * fine != NULL: the pair's recorded osmpm_schwarz_couple steps (both domains
 * recording, step-average projection), differentiated through the Schwarz
 * iterations each step ran (their number and the receiver sets held fixed):
 * per step the post-convergence coarse G2P, then for every iteration from
 * the last to the first the fine sub-steps in reverse (including the adjoint
 * of their receiver data, u_bar_D - (K lam)_D, through T_m), the transposed
 * I_{B->S} into the coarse solve of that iteration, its adjoint, and its
 * receiver data back through the transposed Pi_{S->B} (Eqs. interp_BtoS,
 * spatial_projection, temporal_interp).  Then every array holds the coarse
 * particles' entries followed by the fine ones: dJ_dx has (n_coarse +
 * n_fine) * dim entries, dJ_dE n_coarse + n_fine, and so on.
 *
 * stats: cg_iters and solves of the adjoint PCGs.  Errors: OSMPM_E_INVALID
 * (null arguments, no or interrupted record, a single-domain call on a
 * coupled record), OSMPM_E_UNSUPPORTED (mixed precision), OSMPM_E_NONFINITE,
 * OSMPM_E_CUDA, OSMPM_E_TIMEOUT. */
osmpm_status osmpm_adjoint(osmpm_domain* coarse, osmpm_domain* fine, const double* dJ_dx,
                           const osmpm_adjoint_out* out, osmpm_stats* stats);

/* Particle count and dimension of a domain. */
osmpm_status osmpm_get_info(const osmpm_domain* dom, int64_t* n_particles, int32_t* dim);

/* Copies the particle state to host arrays in id order; any pointer may be
 * NULL to skip that field. */
osmpm_status osmpm_get_particles(const osmpm_domain* dom, double* x, double* v, double* B,
                                 double* F);

/* Overwrites the particle state from host arrays in id order (x, v, B, F;
 * none may be NULL) and re-sorts the particles by Morton code. */
osmpm_status osmpm_set_particles(osmpm_domain* dom, const double* x, const double* v,
                                 const double* B, const double* F);

/* Writes the particle id held by each internal (Morton-sorted) slot:
 * ids[s] = id of the particle in slot s, n entries. */
osmpm_status osmpm_get_order(const osmpm_domain* dom, uint32_t* ids);

/* Grid fields copied to a host array (doubles).  Fields with one value
 * per node: OSMPM_FIELD_MASS (m_i of the last P2G), OSMPM_FIELD_BMASS
 * (boundary-particle mass, Eq. boundary_grid_set), OSMPM_FIELD_RECEIVER
 * (1.0 on Schwarz receiver nodes Gamma_hat, else 0.0).  Fields with dim
 * values per node: OSMPM_FIELD_VN (v^n = (mv)/m of the last P2G, 0 on
 * inactive nodes), OSMPM_FIELD_U (x_hat - x^n of the last solve),
 * OSMPM_FIELD_BC (Schwarz boundary values last applied). */
enum {
  OSMPM_FIELD_MASS = 0,
  OSMPM_FIELD_VN = 1,
  OSMPM_FIELD_U = 2,
  OSMPM_FIELD_BMASS = 3,
  OSMPM_FIELD_RECEIVER = 4,
  OSMPM_FIELD_BC = 5,
  OSMPM_FIELD_PLANE_FORCE = 6,   /* rigid plane: multiplier lambda_i per node (0 if not held) */
  OSMPM_FIELD_PLANE_GAP = 7,     /* rigid plane: gap_i per node (+inf off the candidates) */
  OSMPM_FIELD_PLANE_ACTIVE = 8   /* rigid plane: 1.0 on the held nodes of the last step */
};
osmpm_status osmpm_get_grid(const osmpm_domain* dom, int32_t field, double* out);

/* Probes of the discrete operators at the current particle state (one P2G
 * for step size dt first; no state change).  u, d and the outputs are host
 * arrays of n_nodes*dim doubles (node-major, components innermost); entries
 * on inactive nodes are ignored (read) or 0 (written).
 *  osmpm_probe_gradient: dE_h/du (Eq. grid_residual with the energy-
 *    consistent internal force) at u = x_hat - x^n, all active DOFs.
 *  osmpm_probe_hvp: (M/dt^2 + K(u)) d, all active DOFs.  With pcg_mode 2
 *    the particle part comes from the streaming PCG's own product (lane
 *    groups or, in mixed precision, block tiles per hvp_mode); otherwise
 *    from a one-thread-per-particle product over the cached Hessian blocks.
 *  osmpm_probe_energy_change: E_h(u + alpha d) - E_h(u), +inf if a trial
 *    inverts an element. */
osmpm_status osmpm_probe_gradient(osmpm_domain* dom, double dt, const double* u, double* grad);
osmpm_status osmpm_probe_hvp(osmpm_domain* dom, double dt, const double* u, const double* d,
                             double* hd);
osmpm_status osmpm_probe_energy_change(osmpm_domain* dom, double dt, const double* u,
                                       const double* d, double alpha, double* dE);

/* Counters for measurement.  launches: kernels this library has launched in
 * the process.  pcg_*: when timing is enabled on the domain, the number of
 * persistent PCG launches (one per Newton iteration), their summed
 * duration from CUDA events recorded on the domain's stream around each
 * launch, and the PCG iterations they ran; particles and dofs are the
 * per-iteration work units of the domain (n and n_nodes * dim);
 * graph_replays: Newton iterations of the domain that ran as a replay of a
 * captured CUDA graph (launch_mode 0), graphs: graphs it holds,
 * graph_error: the cudaError_t of a capture that failed (the domain then
 * launches directly), 0 if none. */
typedef struct osmpm_counters {
  int64_t launches;
  int64_t pcg_launches;
  double pcg_ms;
  int64_t pcg_iters;
  int64_t particles;
  int64_t dofs;
  int64_t graph_replays;
  int32_t graphs;
  int32_t graph_error;
  double hvp_ms;        /* streaming PCG: summed durations of its Hessian-vector */
  int64_t hvp_launches; /* product launches that iterated (CUDA events) */
} osmpm_counters;

/* Enables (1) or disables (0) CUDA-event timing of this domain's PCG
 * launches and resets its counters; read them with osmpm_get_counters. */
osmpm_status osmpm_set_profiling(osmpm_domain* dom, int32_t enable);

/* Diagnostic of the device-side waits: launches the PCG kernel's grid
 * barrier so that it waits for a block that does not exist; its bounded
 * spin gives up after about two seconds and the kernel returns.  Returns
 * OSMPM_E_TIMEOUT when the kernel reported the timeout (the expected
 * result; the CUDA context stays usable), OSMPM_E_CUDA otherwise. */
osmpm_status osmpm_check_wait_timeout(void* cuda_stream);

/* Reads the counters; dom may be NULL (process-wide launch count only). */
osmpm_status osmpm_get_counters(const osmpm_domain* dom, osmpm_counters* out);

/* ---------------------------------------------------------------------------
 * Energy change without device allocation.
 *
 * The paper has no counterpart to this entry point; it is a service for
 * callers that may not allocate device memory (a sandbox with a memory cap,
 * a host application whose own allocator owns the GPU, a caller that must
 * not allocate inside a latency budget).  It computes the line-search
 * quantity E_h(u + alpha s) - E_h(u) of osmpm_probe_energy_change from
 * caller-owned DEVICE arrays and calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its reduction scratch is a fixed file-scope device
 * array of 4128 doubles (33 KB) that every GPU loading the library holds
 * until the process exits.
 *  - Layouts (device): particle fields component-major (x[a*n + p],
 *    F[e*n + p] with e = a*dim + b); grid fields over the dense node box,
 *    component-major (vn[a*n_nodes + i]); m has one value per node.
 *  - mu, lam are the Lame parameters E/(2(1+nu)), E nu/((1+nu)(1-2nu)).
 *  - The result (one double, +inf if a trial inverts an element) is
 *    written to the device pointer dE on the given stream.  The call then
 *    waits for that stream: a particle whose B-spline support leaves the
 *    grid box makes dE NaN and the call return OSMPM_E_OUT_OF_GRID.
 *  - Size limit: max(n_particles, n_nodes * dim) <= 1,048,576; larger
 *    problems are rejected with OSMPM_E_INVALID before any device work.
 *  - The first call on each device looks up the scratch array's device
 *    address (cudaGetSymbolAddress with that device current); make that
 *    first call before any stream capture.  The address is kept for the
 *    life of the process (a cudaDeviceReset would make it stale).  All
 *    calls share the scratch, which keeps the last call's contents: calls
 *    that overlap on the GPU (other streams, other threads) race.
 * ------------------------------------------------------------------------- */
typedef struct osmpm_noalloc_grid {
  int32_t dim;
  double origin[3];
  double dx;
  int32_t res[3];
  double mass_eps;          /* active nodes: m_i > mass_eps */
  double gravity[3];
  const double* m;          /* n_nodes nodal masses */
  const double* vn;         /* dim * n_nodes, v^n */
  const double* u;          /* dim * n_nodes, x_hat - x^n */
  const double* s;          /* dim * n_nodes, step direction */
} osmpm_noalloc_grid;

typedef struct osmpm_noalloc_particles {
  int64_t n;
  const double* x;          /* dim * n */
  const double* F;          /* dim * dim * n, F^n */
  const double* vol0;       /* n */
  const double* mu;         /* n */
  const double* lam;        /* n */
} osmpm_noalloc_particles;

osmpm_status osmpm_energy_change_noalloc(const osmpm_noalloc_grid* grid,
                                         const osmpm_noalloc_particles* particles,
                                         double dt, double alpha, double* dE,
                                         void* cuda_stream);

/* Message of the last failure on this thread (never NULL). */
const char* osmpm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OSMPM_H */
