/*
 * sacra2d.h - C ABI of the GB300 (sm_103a) implementation of the SACRA-2D hot
 * path: one Runge-Kutta stage of BSSN-Z4c + HLLC general-relativistic
 * hydrodynamics on an axisymmetric (cartoon) fixed-mesh-refinement grid
 * (Lam & Shibata, "SACRA-2D", arXiv:2502.03223).
 *
 * Every entry point returns a sacra_status and never aborts; on failure
 * sacra_last_error() describes the cause.  Physics failures inside cells
 * (non-converged primitive recovery, atmosphere resets, HLLC -> TVDLF
 * fallbacks) are counted, not fatal (see sacra_diag).
 *
 * Memory and streams.  The library does all arithmetic in its own CUDA
 * kernels.  Device memory is one arena owned by the context: the caller may
 * pass a device buffer of at least sacra_arena_bytes() bytes (for instance a
 * torch uint8 tensor) or NULL, in which case the library allocates it with
 * cudaMalloc and frees it in sacra_destroy.  All work is issued on the CUDA
 * stream given to sacra_init_grid (NULL = legacy default stream).  Host
 * buffers passed to the library stay owned by the caller; copies to and from
 * them are complete when the call returns.
 *
 * Grid layout (Sec. II.A, Eqs. for Delta x^(l) and x_j^(l)).  L levels of
 * nx x nz cells; level l has spacing dx0 / 2^l; cell (j, k), j in [1, nx],
 * k in [1, nz], has centre x_j = (j - 1/2) dx, z_k = (k - 1/2) dz.  Each level
 * is stored padded with 8 cells on every side (the (4+4) buffer zone of
 * Sec. II.A): a field plane has pz = nz + 16 rows of px = nx + 16 doubles,
 * cell (j, k) at index (k + 7) * px + (j + 7), row-major with x fastest.
 * Level l (l >= 1) covers the parent cells [1, N/2]^2 (box-in-box, anchored
 * at the axis and the equator, Sec. II.D).
 *
 * Field numbering (state planes):
 *   0 W, 1-6 h_ij (xx,xy,xz,yy,yz,zz; gt_ij = delta_ij + h_ij), 7-12 At_ij,
 *   13 Khat, 14-16 Gt^i, 17 Theta, 18 alpha, 19-21 beta^i, 22-24 B^i
 *   (Sec. II.B.1, Eq. bssn and Eq. moving_puncture);
 *   25 q_D, 26 q_Sx, 27 q_Sy (cylindrical: q_Sphi = x q_Sy), 28 q_Sz, 29 q_E
 *   (Eq. cons_var, q = psi^6 (D, S_i, E), psi^6 = W^-3).
 * Primitive planes: 0 rho, 1 u_x, 2 u_y, 3 u_z (covariant), 4 P, 5 eps.
 */
#ifndef SACRA2D_H
#define SACRA2D_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sacra_ctx sacra_ctx;
typedef struct sacra_batch sacra_batch;

typedef enum {
  SACRA_OK = 0,
  SACRA_ERR_ARG = -1,      /* invalid argument or configuration */
  SACRA_ERR_CUDA = -2,     /* a CUDA call failed; the message names it */
  SACRA_ERR_OOM = -3,      /* arena too small or allocation failed */
  SACRA_ERR_STATE = -4     /* call out of sequence (e.g. no initial data) */
} sacra_status;

enum { SACRA_PLANAR = 0, SACRA_CYLINDRICAL = 1 };
enum { SACRA_HLLC = 0, SACRA_TVDLF = 1 };
enum { SACRA_RK4 = 0, SACRA_SSPRK3 = 1 };
/* precision: FP64 everywhere, or an OR of the parts whose arithmetic runs in FP32 */
enum {
  SACRA_FP64 = 0,
  SACRA_MIXED_FLUX = 1,      /* PPM reconstruction, face metric, tetrad HLLC / TVDLF flux */
  SACRA_MIXED_SOURCES = 2,   /* geometric and gravitational hydro sources (the divergence stays FP64) */
  SACRA_MIXED_Z4C = 4,       /* cartoon planes, weighted stencil sums and the pointwise Z4c right-hand side */
  SACRA_MIXED = 7
};
enum { SACRA_PRIM_METRIC = 0, SACRA_RAW = 1 };
enum { SACRA_FILL = 0, SACRA_RESTRICT_REFLUX = 1 };
enum { SACRA_STATE_STEP = 0, SACRA_STATE_STAGE = 1, SACRA_PRIMS = 2, SACRA_RHS = 3, SACRA_STATUS = 4 };

/* Run configuration.  Parameters the paper fixes: kappa = 5e-3/M (Sec. II.B.1),
   eps_ko = 0.5, eta_B ~ 1/M, r_z4 <= L_max/6 (Sec. II.B.3), w_max = 100 and
   rho_atm = f_atm rho_max(t=0) (Sec. II.C.4). */
typedef struct {
  int n_levels;          /* L >= 1; L > 1 needs nx == nz, even, >= 16, cylindrical */
  int nx, nz;            /* cells per level */
  int geometry;          /* SACRA_PLANAR (Cartesian slab, outflow boundaries) or SACRA_CYLINDRICAL
                            (x = varpi, axis and equatorial symmetry, outgoing outer boundary) */
  int evolve_spacetime;  /* 0: metric frozen */
  int solver;            /* SACRA_HLLC (with TVDLF fallback) or SACRA_TVDLF */
  int rk;                /* SACRA_RK4 (the paper's integrator) or SACRA_SSPRK3 */
  int c2p_maxit;         /* iteration cap of the primitive recovery */
  int precision;         /* SACRA_FP64, or an OR of SACRA_MIXED_* bits (SACRA_MIXED: all of them); every finite
                            difference of the state, the primitive recovery, the algebraic constraints, the flux
                            divergence, the RK combination and the flux registers stay FP64 in every mode */
  int subcycle_from;     /* Berger-Oliger sub-cycling (Sec. II.D): 0 = every level takes the step dt given to
                            sacra_step (lockstep); K >= 1 = levels >= K take half their parent's step
                            (the paper's l_fix = K - 1), dt being the step of the levels below K.
                            K >= n_levels is lockstep too.  Single contexts only (a batch star with
                            1 <= K < n_levels: SACRA_ERR_ARG); on a sub-cycled context the stage-wise
                            calls (sacra_regrid_ghosts, sacra_rk_stage) return SACRA_ERR_STATE.  Each
                            parent of a sub-cycled level keeps 2 x 25 metric and 3 x 6 primitive
                            planes more (its t^{n-1} and t^n slices and their interpolant) */
  int hydro_outer;       /* hydro at level 0's outer boundary: 0 = zero-gradient copy of the primitives,
                            1 = held at the initial data given to sacra_set_initial_data (an inflow
                            boundary with a known solution, e.g. Bondi accretion) */
  int eos_adiabatic;     /* 0: cold part + thermal Gamma_th law (Sec. II.C.3); 1: the "adiabatic" EOS of the
                            migration test (Sec. III): zero temperature, P = P_cold, eps = eps_cold everywhere,
                            the energy equation discarded (the recovery uses D and S_i only and rebuilds E);
                            needs K > 0 */
  int n_pieces;          /* cold part: 0 or 1 = the single polytrope (K, Gamma); 2..8 = piecewise polytropic
                            (Sec. II.C.3) with piece 1 = (K, Gamma) and the others from pwp_rho, pwp_Gamma.
                            Not accepted by sacra_hydro_rhs_noalloc (SACRA_ERR_ARG) */
  int bssn;              /* 0: Z4c (Sec. II.B.1); 1: the BSSN formulation the paper switches to for a cleaner
                            waveform (Sec. III): Theta held at zero (its right-hand side is zero; give Theta = 0
                            in the initial data) and no constraint damping (kappa taken as 0) */
  double dx0, dz0;       /* spacing of level 0 */
  double kappa, eta_B, eps_ko, r_z4;
  double K, Gamma, Gamma_th;   /* cold polytrope P = K rho^Gamma plus thermal Gamma_th law (Sec. II.C.3) */
  double rho_atm, w_max, c2p_tol;
  double r_hold;         /* > 0: the hydro of every cell with x^2 + z^2 < r_hold^2 is held at its state at the
                            start of the step (an excised inner boundary, e.g. inside a black hole: the
                            stage update keeps U^n and the recovery is skipped there); 0 = off */
  double pwp_rho[7];     /* transition densities rho_1 < rho_2 < ... < rho_(n_pieces-1), all > 0 */
  double pwp_Gamma[7];   /* Gamma_2 .. Gamma_(n_pieces), each > 1; K_i and Delta eps_i follow from the
                            continuity of P_cold and eps_cold at the transitions */
} sacra_params;

/* Global diagnostics (Sec. II.F.1) over the cells not covered by a finer
   level, volume element 2 pi x dx dz (cylindrical) or dx dz (planar),
   integrated over the computational domain. */
typedef struct {
  double H_L2;           /* sqrt(sum H^2 dV / sum dV) */
  double M_L2[3];        /* same for M_x, M_y (= M_phi / x), M_z */
  double Mb;             /* rest mass  sum q_D dV */
  double J;              /* angular momentum sum q_Sphi dV (cylindrical) */
  double rho_max;
  double n_c2p_fail;     /* cells whose last recovery did not converge or was invalid */
  double n_fallback;     /* HLLC -> TVDLF fallbacks since creation */
} sacra_diag;

/* Bytes of device memory the configuration needs (one arena). */
sacra_status sacra_arena_bytes(const sacra_params *p, size_t *bytes);

/* Create a context.  stream: a cudaStream_t (NULL = default stream);
   arena: device buffer of at least sacra_arena_bytes() bytes, 256-byte
   aligned, or NULL to let the library allocate one.  The arena must outlive
   the context.  *out receives the context (NULL on failure). */
sacra_status sacra_init_grid(const sacra_params *p, void *cuda_stream, void *arena, size_t arena_bytes,
                             sacra_ctx **out);

/* Initial data of one level from HOST memory (copied before returning).
   kind SACRA_PRIM_METRIC: n_fields = 30 padded planes, 25 metric fields then
   (rho, u_x, u_y, u_z, P); eps follows from the EOS and the conserved
   variables from Eq. cons_var, on every cell including the padding.
   kind SACRA_RAW: n_fields = 30 padded state planes (metric + conserved);
   the primitives are recovered on every cell (which may reset a cell to the
   atmosphere or the cold curve and rewrite its conserved variables, as any
   recovery does).  The RAW copy runs in row chunks on a stream of the
   context's own, each chunk's recovery on the context's stream once the chunk
   has arrived; the call returns when the host buffer has been copied, and the
   recovery is ordered before every later call's work on the context.
   host_planes: n_fields * pz * px doubles (pinned memory lets the copy run at
   the link's rate). */
sacra_status sacra_set_initial_data(sacra_ctx *c, int level, int kind, const double *host_planes, int n_fields);

/* Ghost and buffer fill (what = SACRA_FILL) for RK stage `stage` of a step of
   size dt: axis/equator parity, the outgoing condition of Sec. II.B.3 on the
   coarsest level's outer cells (tau = c_stage dt), and prolongation into the
   buffer zone of each finer level (Sec. II.D: [N+1, N+8] at stage 0,
   [N+5, N+8] afterwards).  what = SACRA_RESTRICT_REFLUX ends a step:
   conservative restriction of q and 8th-order restriction of the metric onto
   the parent, reflux of the coarse cells next to each refinement boundary,
   primitive recovery there (stage and dt are ignored). */
sacra_status sacra_regrid_ghosts(sacra_ctx *c, int what, int stage, double dt);

/* RK stage `stage` (0-based) on all levels: hydro RHS (PPM, tetrad HLLC/TVDLF,
   cylindrical finite-volume update with sources), Z4c RHS with cartoon terms
   and KO dissipation, RK combination, algebraic constraints, primitive
   recovery with atmosphere.  Requires the ghosts filled for this stage. */
sacra_status sacra_rk_stage(sacra_ctx *c, int stage, double dt);

/* n_steps full steps (fill + stage for every stage, then restrict/reflux).
   use_graph != 0 captures one step in a CUDA graph on first use and replays it. */
sacra_status sacra_step(sacra_ctx *c, double dt, int n_steps, int use_graph);

/* n_steps steps as sacra_step, with the diagnostics (Sec. II.F.1) of the
   state at the START of step i written to out[i], i < n_steps.  They are
   formed inside the step's first RK stage from the derivatives its Z4c pass
   has just computed, after the same ghost fill sacra_constraints does, so
   out[i] equals sacra_constraints called just before step i, without a second
   cartoon and derivative pass (n_fallback: the counter after step i).  The
   host waits for the stream after each step.  out: host array of n_steps
   entries (NULL with n_steps > 0: SACRA_ERR_ARG).  Lockstep contexts only
   (sub-cycled: SACRA_ERR_STATE). */
sacra_status sacra_step_constraints(sacra_ctx *c, double dt, int n_steps, int use_graph, sacra_diag *out);

/* Copy one plane to HOST memory.  which: SACRA_STATE_STEP (state at the start
   of the step, i.e. the current state between steps), SACRA_STATE_STAGE,
   SACRA_PRIMS, SACRA_RHS or SACRA_STATUS (per-cell recovery flags as
   doubles).  n = nx*nz copies the interior (row-major, x fastest), n = px*pz
   the padded plane. */
sacra_status sacra_read_state(sacra_ctx *c, int level, int which, int field, double *host_out, size_t n);

/* Copy all n_fields = 30 padded planes of one level (metric + conserved,
   which = SACRA_STATE_STEP, SACRA_STATE_STAGE or SACRA_RHS) to HOST memory:
   host_planes holds n_fields * pz * px doubles, packed plane after plane in
   field order, the layout sacra_set_initial_data(kind = SACRA_RAW) takes, so
   the pair saves and restores a level (e.g. a checkpoint).  One pitched
   device-to-host copy on the context's stream; waits for it.  Pinned host
   memory lets the copy run at the link's rate.  Errors: SACRA_ERR_ARG for a
   bad level, which, n_fields or a NULL buffer. */
sacra_status sacra_read_level(sacra_ctx *c, int level, int which, double *host_planes, int n_fields);

/* Diagnostics of the current state (a stage-0 ghost fill is done first). */
sacra_status sacra_constraints(sacra_ctx *c, sacra_diag *out);

/* Wait for all work of the context. */
sacra_status sacra_sync(sacra_ctx *c);

/* Number of kernels the library has launched since creation (graph replays
   count their kernels). */
long long sacra_launch_count(const sacra_ctx *c);

/* Optional per-kernel device timing for measurement.  enable != 0 starts (and
   resets) recording: every kernel launched outside a CUDA graph is bracketed
   by CUDA events on the context's stream.  sacra_profile_get reports kernel
   kind idx (0-based; SACRA_ERR_ARG past the last kind): its name (written to
   name, at most name_len bytes), the summed device time in ms, the number of
   launches and the cells (threads' units of work) they processed.  Waits for
   the stream. */
sacra_status sacra_profile(sacra_ctx *c, int enable);
sacra_status sacra_profile_get(sacra_ctx *c, int idx, char *name, size_t name_len, double *total_ms,
                               long long *launches, long long *cells);

/* Hydro right-hand side of one level without allocating anything (the paper
   has no counterpart: this serves callers that cannot call cudaMalloc, e.g.
   when a host framework's memory pool already owns the device or allocation
   is not allowed where the call is made).  Same arithmetic as the hydro part
   of sacra_rk_stage on the region [1, nx] x [1, nz]: face fluxes (PPM,
   tetrad HLLC/TVDLF), flux divergence and sources; no flux registers.
   state: DEVICE, 30 padded planes of px*pz doubles (plane stride exactly
   px*pz), ghosts filled; prims: DEVICE, 6 planes; rhs_out: DEVICE, 5 planes
   (d_t q_D, q_Sx, q_Sy, q_Sz, q_E), written on the region.  Work is queued on
   cuda_stream.  px*pz must not exceed SACRA_NOALLOC_MAX_PLANE (up to 256 x 256
   interior cells), else SACRA_ERR_ARG.  The face-flux scratch is one
   file-scope device array per GPU (about 5.9 MB, held until the process
   exits); its device address is looked up on every call (no allocation),
   and the first call on a device loads the library's device code, so make
   that first call before any stream capture.  Every call shares the array:
   calls that overlap on the GPU race (serialize them).  precision may carry
   SACRA_MIXED_FLUX / SACRA_MIXED_SOURCES (the FP32 flux and source kernels).
   The HLLC -> TVDLF fallback count is not reported by this entry point.
   Returns SACRA_ERR_CUDA without launching anything if the calling thread
   already holds an unread CUDA error (left by earlier work), and
   SACRA_ERR_CUDA if a launch fails. */
#define SACRA_NOALLOC_MAX_PLANE 73984
sacra_status sacra_hydro_rhs_noalloc(const sacra_params *p, int level, const double *state, const double *prims,
                                     double *rhs_out, void *cuda_stream);

/* Autotuner (no counterpart in the paper).  Every RK stage runs as one
   persistent launch per kernel kind over the tiles of all levels; for each
   kind this times every tile shape the kernel allows and every persistent
   grid size (blocks per SM) on the current state (reps launches each, CUDA
   events on the context's stream) and keeps the fastest.  The state is not
   changed.  Needs initial data on every level.  sacra_get_tuning reports the
   choice for kernel kind `kind` (0 x-fluxes, 1 z-fluxes, 2 hydro divergence
   and sources, 3 cartoon planes, 4 Z4c derivatives, 5 Z4c pointwise, 6 stage
   update); SACRA_ERR_ARG past the last kind. */
sacra_status sacra_tune(sacra_ctx *c, int reps);
sacra_status sacra_get_tuning(const sacra_ctx *c, int kind, int *tile_x, int *tile_y, int *blocks_per_sm);
/* Pins kind `kind`'s launch configuration instead of tuning it: the tile
   shape tile_x x tile_y, one of the autotuner's candidates (32x4, 64x2, 16x8,
   128x1 for kinds 0-3, 5 and 6; 32x8 and 64x4 also for kinds 0-2, whose
   kernels take 256 threads; kind 4, the derivative pass, accepts only its
   fixed shape: 16x8 in FP64, 32x8 in the mixed form), and the persistent
   grid size blocks_per_sm,
   one of 1, 2, 3, 4, 6, 8, 12.  A step's results do not depend on these
   choices.  Drops the context's captured CUDA graphs (the next graph step
   captures anew).  Errors: SACRA_ERR_ARG for a kind, shape or grid size
   outside those lists. */
sacra_status sacra_set_tuning(sacra_ctx *c, int kind, int tile_x, int tile_y, int blocks_per_sm);

/* ---- Learned seed of the primitive recovery (no counterpart in the paper).
   A 9 -> 64 -> 64 -> 1 tanh network (BF16 weights, FP32 arithmetic) predicts
   log10(P / D) from the conserved variables and metric invariants; the
   predicted pressure gives a first value z0 of the recovery's unknown, the
   FP64 Illinois iteration runs on the bracket z0 (1 -+ delta) and, whenever
   that bracket does not enclose the root or the iteration reaches its cap,
   on the plain bracket.  Converged primitives therefore equal those of the
   unseeded recovery to its tolerance (c2p_tol).

   sacra_mlp_bytes: size of the packed network (a device buffer the caller owns).
   sacra_mlp_collect: write tuples (9 features, then log10(P / D); 10 floats
   each) of every interior cell of every level whose recovery is non-trivial
   (moving fluid above the atmosphere, no cold or atmosphere branch) into
   DEVICE buffer dev_tuples (capacity tuples); *n = tuples written.
   sacra_mlp_train: train a fresh network (Glorot-uniform start from `seed`)
   on DEVICE tuples (every fifth tuple, index % 5 == 4, is held out) with Adam
   for `steps` minibatches of batch_blocks x 128 tuples, lr decaying by a
   cosine to lr / 100; writes the packed network to DEVICE dev_net.  The
   seed is tried only where k = r / (1 + q) >= kmin (slow flows, where the
   plain bracket already converges in 2-3 evaluations, can skip it).
   host_loss: NULL or `steps` floats (minibatch loss per step); host_report:
   NULL or 3 floats (held-out RMS error of log10(P / D), 99.9th percentile of
   the seed's relative z error, the bracket half-width delta chosen as four
   times that percentile, in [1e-5, 0.05]).  Runs on cuda_stream; allocates
   its scratch with cudaMalloc and frees it before returning.
   sacra_mlp_grad: the gradient (flat order w1 64x9, b1, w2 64x64, b2, w3, b3;
   MLP_NPARAM = 4865 floats to host_grad) of the mean squared error over all
   n DEVICE tuples at the network dev_net, and that loss (host_loss).
   sacra_set_mlp: use network dev_net (DEVICE, must outlive its use) in every
   later recovery of the context; NULL restores the plain bracket.
   sacra_c2p_counting / sacra_c2p_counts: count, from now on, Illinois
   function evaluations, recoveries where a seed was tried, seeded brackets
   that held, and recoveries; out4 receives the four counts (reset != 0
   zeroes them). */
size_t sacra_mlp_bytes(void);
sacra_status sacra_mlp_collect(sacra_ctx *c, float *dev_tuples, long long capacity, long long *n);
sacra_status sacra_mlp_train(const float *dev_tuples, long long n, int steps, int batch_blocks, float lr,
                             unsigned long long seed, float kmin, void *dev_net, float *host_loss, float *host_report,
                             void *cuda_stream);
sacra_status sacra_mlp_grad(const float *dev_tuples, long long n, const void *dev_net, float *host_grad,
                            float *host_loss, void *cuda_stream);
sacra_status sacra_set_mlp(sacra_ctx *c, const void *dev_net);
sacra_status sacra_c2p_counting(sacra_ctx *c, int enable);
sacra_status sacra_c2p_counts(sacra_ctx *c, long long *out4, int reset);

void sacra_destroy(sacra_ctx *c);
const char *sacra_last_error(const sacra_ctx *c);

/* ---- Batches of independent stars (no counterpart in the paper: many
   hierarchies advanced together).  Each star has its own sacra_params; the
   stars must agree in the choices that select kernels (geometry,
   evolve_spacetime, solver, rk, precision; else SACRA_ERR_ARG) and may differ
   in everything else (grid, EOS, gauge, atmosphere, recovery, bssn), which
   each launch reads per star.  All stars take the same dt.  Every
   RK stage is one persistent launch per kernel kind over the tiles of every
   level of every star (ghost fill, restriction and reflux stay per level);
   sacra_batch_step with use_graph != 0 replays whole steps of all stars as
   one CUDA graph.  Arena, stream, error and ownership rules are those of the
   single-star calls; `star` is 0-based. */
sacra_status sacra_batch_arena_bytes(const sacra_params *per_star, int n_stars, size_t *bytes);
sacra_status sacra_init_batch(const sacra_params *per_star, int n_stars, void *cuda_stream, void *arena,
                              size_t arena_bytes, sacra_batch **out);
sacra_status sacra_batch_set_initial_data(sacra_batch *b, int star, int level, int kind, const double *host_planes,
                                          int n_fields);
sacra_status sacra_batch_step(sacra_batch *b, double dt, int n_steps, int use_graph);
sacra_status sacra_batch_read_state(sacra_batch *b, int star, int level, int which, int field, double *host_out,
                                    size_t n);
sacra_status sacra_batch_constraints(sacra_batch *b, int star, sacra_diag *out);
sacra_status sacra_batch_tune(sacra_batch *b, int reps);
sacra_status sacra_batch_get_tuning(const sacra_batch *b, int kind, int *tile_x, int *tile_y, int *blocks_per_sm);
sacra_status sacra_batch_set_tuning(sacra_batch *b, int kind, int tile_x, int tile_y, int blocks_per_sm);
sacra_status sacra_batch_sync(sacra_batch *b);
long long sacra_batch_launch_count(const sacra_batch *b);
sacra_status sacra_batch_profile(sacra_batch *b, int enable);
sacra_status sacra_batch_profile_get(sacra_batch *b, int idx, char *name, size_t name_len, double *total_ms,
                                     long long *launches, long long *cells);
sacra_status sacra_batch_set_mlp(sacra_batch *b, const void *dev_net);
sacra_status sacra_batch_mlp_collect(sacra_batch *b, float *dev_tuples, long long capacity, long long *n);
void sacra_batch_destroy(sacra_batch *b);
const char *sacra_batch_last_error(const sacra_batch *b);

#ifdef __cplusplus
}
#endif

#endif
