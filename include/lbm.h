/*
 * lbm.h -- C ABI of the GB300 lattice Boltzmann hot path of arXiv 2512.12213
 * ("Shear Stress and Fluid-Wall Interaction Force in LBM Simulations of
 * Hydrodynamic and MHD Flows").
 *
 * What the library computes (all of it in CUDA kernels on the caller's stream):
 *   - the BGK relaxation-propagation step of Eq. (2) on D2Q9 / D3Q19 with the
 *     equilibrium of Eq. (1) (plus the Maxwell term of Eq. (10) on request),
 *     one of the five force models of Sec. 2 ([a] He, [b] Martys/Luo,
 *     [c] Shan-Chen reformulated, [d] exact difference reformulated, [e] Guo),
 *     a uniform body force and/or an imposed-field low-Rm Lorentz force,
 *     optional Smagorinsky relaxation time, halfway bounce-back with Ladd's
 *     moving-wall term;
 *   - the stress and strain-rate tensors of Eqs. (8)-(9) with or without the
 *     artefact term E_ij, and from the half-step distribution of Eqs. (27)-(30);
 *   - the momentum-exchange wall force of Eq. (25) with the moving-wall and
 *     Maxwell-stress corrections discussed in Sec. 5, accumulated in FP64;
 *   - global FP64 sums for the balance of Eq. (32);
 *   - one reverse step of the discrete adjoint of the above, for gradients of
 *     time-averaged wall drag.
 *
 * Conventions
 *   Memory   : every large device buffer is allocated by the caller and bound
 *              at lbm_create (sizes from lbm_buffer_sizes).  The library keeps
 *              pointers to them and allocates no device memory itself.
 *              Device pointers must be 256-byte aligned.
 *   Streams  : `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *              default stream).  Device work is asynchronous on it; a call that
 *              writes a host buffer synchronises that stream before returning,
 *              except a reduction asked for LBM_OUT_HOST_ASYNC output.
 *   Outputs  : the reductions (wall force, balance, adjoint gradient) take
 *              `out_on_host`: LBM_OUT_DEVICE (0) device memory written in
 *              stream order; LBM_OUT_HOST (1) any host memory, the call
 *              synchronises; LBM_OUT_HOST_ASYNC (2) page-locked host memory
 *              written by a copy in stream order, valid once the stream has
 *              been synchronised (LBM_ERR_ARG for pageable memory or with
 *              LBM_ACCUMULATE).  Reductions of one context share its scratch,
 *              so they must not be in flight on two streams at once.
 *   Units    : physical (dx, dt, c = dx/dt); forces are per unit depth in 2-D.
 *   Layout   : canonical arrays exchanged with the caller are dense C arrays,
 *              node index n = (z*ny + y)*nx + x; populations f[a][n] (a the
 *              velocity index), vectors v[k][n] (k = 0,1,2), tensors s[c][n]
 *              with components xx yy xy (2-D) or xx yy zz xy xz yz (3-D).
 *              Velocity order:
 *                D2Q9 : 0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1)
 *                       5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
 *                D3Q19: 0 rest, 1/2 +-x, 3/4 +-y, 5/6 +-z, 7/8 +-(1,1,0),
 *                       9/10 +-(1,-1,0), 11/12 +-(1,0,1), 13/14 +-(1,0,-1),
 *                       15/16 +-(0,1,1), 17/18 +-(0,1,-1)
 *   Geometry : wall_id[n] = 0 for a fluid node, k in 1..n_walls for a solid
 *              node of wall k.  A non-periodic axis is closed on both faces by
 *              halfway bounce-back walls with ids face_wall[2*axis + side].
 *              A link leaving the box through several closed faces at once
 *              takes the wall of the first such axis in the order x, y, z.
 *   Time     : the context holds the state at time T (steps taken since the
 *              last init/import).  Internally it stores the post-collision
 *              populations f^rel(T-1); the canonical f(T) (post-propagation,
 *              pre-collision) is what export returns.
 *   Errors   : every call returns an lbm_status; nothing aborts or throws
 *              across the ABI.  lbm_last_error() gives a message.  A context
 *              is not thread safe.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum lbm_status {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,          /* invalid argument, configuration or buffer */
    LBM_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    LBM_ERR_OOM = 3,          /* a host allocation failed */
    LBM_ERR_UNSUPPORTED = 4,  /* valid request that this build does not implement */
    LBM_ERR_NAN = 5,          /* a reduction read back to the host is not finite (the
                                 values are still written); device and asynchronous
                                 outputs are not checked */
    LBM_ERR_STATE = 6,        /* call not valid in the context's current state */
    LBM_ERR_NOT_CONVERGED = 7 /* lbm_run_steady reached its step limit first */
} lbm_status;

enum { LBM_D2Q9 = 9, LBM_D3Q19 = 19 };

/* force models of Sec. 2 (C, u^F, u^eq):
 * [a] He 1997 (1, -, u)  [b] Martys/Luo (1, u, u)  [c] Shan-Chen (1, u + tau dt a/2, u)
 * [d] exact difference (1, v, u)  [e] Guo 2002 (1 - 1/(2 tau), v, v), v = u + dt a/2 */
enum { LBM_FORCE_A = 0, LBM_FORCE_B = 1, LBM_FORCE_C = 2, LBM_FORCE_D = 3, LBM_FORCE_E = 4 };

/* population storage.  F64 computes in FP64; the others compute in FP32.
 * All modes store the shifted deviation f_a - w_a rho0; F16S stores it scaled
 * by 2^12 in IEEE binary16, BF16S unscaled in bfloat16. */
enum { LBM_STORE_F64 = 0, LBM_STORE_F32 = 1, LBM_STORE_F16S = 2, LBM_STORE_BF16S = 3 };

/* stress variants:
 * S1 sigma = -(1 - 1/(2 tau)) [Pi^neq + E_ij]   (Eq. 9 with the artefact term)
 * S2 sigma = -(1 - 1/(2 tau)) Pi^neq            (E_ij neglected, after Eq. 23)
 * S3 sigma = -sum e e (fbar - f^eq(rhobar, ubar)), fbar of Eq. (27)
 * S4 S3 + Theta/2                               (Eq. 30)
 * with Pi^neq = sum e e f - (p delta + rho u^eq u^eq + L); S = sigma/(2 rho nu). */
enum { LBM_S1 = 1, LBM_S2 = 2, LBM_S3 = 3, LBM_S4 = 4 };

/* wall-force options (Sec. 5) */
enum {
    LBM_MOVING_CORR = 1,      /* add u_w (fbar_a - fbar_a') per link (Galilean correction) */
    LBM_MAXWELL_REMOVE = 2,   /* subtract 2 e_a' Delta_a' per link (Maxwell stress) */
    LBM_ACCUMULATE = 4        /* out += weight * F instead of out = weight * F */
};

/* where the `out` argument of a reduction lives (see Outputs above) */
enum { LBM_OUT_DEVICE = 0, LBM_OUT_HOST = 1, LBM_OUT_HOST_ASYNC = 2 };

/* caller-allocated device buffers, indexed by kind */
enum {
    LBM_BUF_POP_A = 0,        /* populations, ping       (required) */
    LBM_BUF_POP_B = 1,        /* populations, pong       (required) */
    LBM_BUF_NODE = 2,         /* node classes            (required) */
    LBM_BUF_LINKS = 3,        /* boundary-link list      (required if any link exists) */
    LBM_BUF_SCRATCH = 4,      /* FP64 reduction partials (required) */
    LBM_BUF_STAGE = 5,        /* canonical staging for host import/export (optional) */
    LBM_BUF_PHI = 6,          /* signed wall distance per node, float (required if curved) */
    LBM_BUF_MAG_A = 7,        /* induced-field distributions, ping (required if induced):
                                 [3][5 or 7][padded node], FP64 for FP64 storage, else FP32 */
    LBM_BUF_MAG_B = 8,        /* induced-field distributions, pong (required if induced) */
    LBM_NUM_BUFFERS = 9
};

#define LBM_MAX_WALLS 16

typedef struct lbm_config {
    int32_t lattice;                 /* LBM_D2Q9 or LBM_D3Q19 */
    int32_t nx, ny, nz;              /* nz = 1 for D2Q9; 1 <= n, nx*ny*nz < 2^31 */
    int32_t periodic[3];             /* per axis; closed axes get face walls */
    double dx, dt;                   /* lattice spacing and time step, c = dx/dt */
    double tau;                      /* relaxation time, > 1/2; nu = dt c^2 (tau - 1/2)/3 */
    double rho0;                     /* reference density (shift of the storage, wall density) */
    int32_t force_model;             /* LBM_FORCE_* */
    double g[3];                     /* uniform body acceleration */
    int32_t lorentz;                 /* 1: add (sigma_e/rho)(E + v x B) x B at the flow velocity v */
    double B[3], E[3];               /* imposed magnetic and electric field */
    double sigma_e;                  /* electrical conductivity */
    double mu;                       /* magnetic permeability (Maxwell equilibrium) */
    int32_t maxwell;                 /* 1: Maxwell term of Eq. (10) with B in the equilibrium */
    int32_t les;                     /* 1: Smagorinsky relaxation time */
    double cs;                       /* Smagorinsky constant */
    int32_t storage;                 /* LBM_STORE_* */
    int32_t n_walls;                 /* wall ids 1..n_walls, n_walls <= LBM_MAX_WALLS */
    double wall_u[LBM_MAX_WALLS][3]; /* velocity of wall k at index k-1 */
    int32_t face_wall[6];            /* wall id of each closed face: -x +x -y +y -z +z */
    int32_t rounding;                /* LBM_ROUND_NEAREST, or LBM_ROUND_STOCHASTIC (16-bit storage only) */
    uint32_t seed;                   /* stream of the stochastic rounding */
    int32_t insulating;              /* 1 (needs lorentz): insulating walls, see below */
    int32_t curved;                  /* 1: walls off the half-grid from a signed distance, see below */
    int32_t stokes;                  /* 1: linear equilibrium rho w (1 + 3 e.u^eq/c^2), see below */
    double darcy;                    /* >= 0: porous resistance, a += -darcy v (Brinkman), see below */
    int32_t induced;                 /* 1: induced magnetic field (needs maxwell = 1), see below */
    double eta;                      /* magnetic diffusivity of the induced field, > 0 */
    int32_t mag_conducting;          /* induced field at walls: 0 insulating, 1 perfectly conducting */
    int32_t step_kernel;             /* LBM_STEP_*: which kernel runs the step (see below) */
} lbm_config;

/* Kernel of the fused step.  Both compute the same arithmetic and store the
 * same bits; they differ in how the pull sources reach the registers.
 * LBM_STEP_AUTO (0) picks the staged kernel for 16-bit storage wherever it
 * applies, enough shared memory holds its pipeline and at most 2% of the
 * 4-node chunks touch a solid or padding; else the register-tiled one.  LBM_STEP_REGISTER (1): every thread loads its vectors straight from
 * HBM.  LBM_STEP_STAGED (2): a persistent kernel stages each tile's source
 * rows in shared memory with bulk asynchronous copies; it serves FP32 and
 * 16-bit storage with closed or periodic faces and every node code except
 * curved walls, insulating walls and the induced field (those: LBM_ERR_ARG);
 * where its pipeline does not fit in shared memory (rows of more than about
 * 1,100 16-bit or 550 FP32 nodes) the register-tiled kernel runs instead. */
enum { LBM_STEP_AUTO = 0, LBM_STEP_REGISTER = 1, LBM_STEP_STAGED = 2 };

/* Induced magnetic field (Sec. 4 cites Dellar's vector lattice Boltzmann
 * model for the induction equation dB/dt + div(v B - B v) = eta lap B).
 * With induced = 1 the field B(x, t) is carried by distributions g_ik
 * (k = x, y, z) on the axis velocities of the fluid lattice (D2Q5 weights
 * 1/3, 1/6 with theta = 1/3; D3Q7 1/4, 1/8 with theta = 1/4), relaxed with
 * tau_m = 1/2 + eta/(theta c^2 dt) to g^eq_ik = W_i [B_k + e_ij (v_j B_k -
 * B_j v_k)/(theta c)] (e_i the integer lattice vectors) with the node's flow
 * velocity v, and propagated; a
 * field link into a wall or a closed face returns as -g'_i + 2 W_i B (B the
 * configured external field: insulating walls) or g'_i (conducting walls).
 * The fluid relaxes with the Maxwell term of Eq. (10) at the local field
 * (maxwell = 1 is required; lorentz, les, curved and insulating must be 0);
 * B above is the external field.  Both fields step from the same time
 * level.  Create / init / import / load set the field distributions to rest
 * in the external field, W_i B; lbm_step_from, the adjoint and the half-step
 * stress variants S3 / S4 are refused.  S1 / S2 take the Maxwell stress at
 * the node's field B(x, T); LBM_MAXWELL_REMOVE of the wall force takes it at
 * B(x_f, T-1), the field of the collision that produced f^rel(x_f, T-1).
 * lbm_export_field reads B(x, T). */

/* Stokes and Brinkman flow (the note after Eq. 11).  stokes = 1 replaces the
 * equilibrium of Eq. (1) by its linear part (plus the Maxwell term), whose
 * second moment c^2 rho delta/3 carries no rho u u: the recovered equation is
 * the Stokes equation.  darcy > 0 adds the resistance of a porous medium,
 * a += -darcy v at the flow velocity v (solved exactly with v = u + dt a/2,
 * together with the Lorentz force), which with stokes = 1 gives the Brinkman
 * equation.  Stress variant S1 (the artefact term of the full equilibrium) is
 * refused with stokes = 1, the adjoint with stokes = 1 or darcy > 0. */

/* Walls off the half-grid (discussion after Eq. 25, end of Sec. 6).  With
 * curved = 1 the context holds a signed wall distance phi per node (buffer
 * LBM_BUF_PHI; lattice units, > 0 at fluid nodes, < 0 at solid nodes; set
 * with lbm_set_wall_distance, +-1/2 until then).  A link from fluid node x_f
 * along a into a solid node x_s crosses the wall at x_f + q e_a with
 * q = phi_f / (phi_f - phi_s), and the population b = opp(a) entering x_f is
 * interpolated from the stored post-collision values (L the moving-wall term
 * of halfway bounce-back):
 *   q <  1/2: f_b(x_f) = 2q f^rel_a(x_f) + (1 - 2q) f^rel_a(x_f + e_b) + L
 *   q >= 1/2: f_b(x_f) = (f^rel_a(x_f) + L)/(2q) + (1 - 1/(2q)) f^rel_b(x_f)
 * (halfway bounce-back when q < 1/2 and x_f + e_b is not a fluid node; closed
 * box faces are always halfway).  q = 1/2 is halfway bounce-back.  The wall
 * force (Eq. 25) uses these values; it then refers to the imaginary points
 * x_f + e_a/2, and at steady state equals the body force on the fluid nodes'
 * volume units.  The adjoint step does not support curved walls. */

/* Insulating walls (Sec. 6, Eq. 36).  No current leaves the fluid, so the
 * electric field is the one that makes the net current sigma_e sum(E + v x B)
 * over fluid nodes vanish: E = -<v> x B, <v> the mean flow velocity of the
 * fluid nodes.  The library keeps E on the device and sets it after every
 * step from that step's mean flow velocity, so step t uses E = -<v(t-1)> x B
 * (a one-step lag; exact zero total Lorentz force at steady state).  The
 * first step after lbm_create, lbm_init_equilibrium, lbm_import_f or
 * lbm_load_state uses the configured E.  E is state that a population
 * checkpoint does not hold, so lbm_step_from returns LBM_ERR_UNSUPPORTED, and
 * the reductions of the step run on the stepping stream.  Costs a scratch
 * row of 3 doubles per step thread (see lbm_buffer_sizes). */

/* rounding of the populations stored by a step.  Stochastic rounding rounds
 * a value up with probability equal to its distance from the value below, so
 * that increments smaller than half a unit in the last place of the storage
 * format accumulate in expectation instead of being lost.  The random bits
 * are a counter-based function of (seed, step index, node, direction), so a
 * step recomputed from a checkpoint (lbm_step_from with the same index)
 * reproduces the original bit for bit. */
enum { LBM_ROUND_NEAREST = 0, LBM_ROUND_STOCHASTIC = 1 };

/* Required bytes of each buffer kind for this configuration and geometry.
 * host_wall_id: nx*ny*nz bytes (layout above), host memory.
 * sizes[LBM_NUM_BUFFERS] receives the byte counts (0 where not needed).
 * Errors: LBM_ERR_ARG for an invalid configuration (message via
 * lbm_config_error). */
lbm_status lbm_buffer_sizes(const lbm_config* cfg, const uint8_t* host_wall_id,
                            size_t sizes[LBM_NUM_BUFFERS]);

/* Message for the last lbm_buffer_sizes / lbm_create failure on this thread. */
const char* lbm_config_error(void);

/* Create a context on the current CUDA device.  buffers/sizes are indexed by
 * LBM_BUF_*; each buffer must be 256-byte aligned and at least the size from
 * lbm_buffer_sizes (STAGE may be NULL with size 0).  Uploads the node classes
 * and the link list with copies on `stream` and waits for them.  Populations
 * are left undefined until lbm_init_equilibrium or lbm_import_f. */
lbm_status lbm_create(const lbm_config* cfg, const uint8_t* host_wall_id,
                      void* const buffers[LBM_NUM_BUFFERS], const size_t sizes[LBM_NUM_BUFFERS],
                      void* stream, lbm_ctx** out);

/* Free the context (host memory only; the caller's buffers are untouched). */
lbm_status lbm_destroy(lbm_ctx* ctx);

const char* lbm_last_error(const lbm_ctx* ctx);

/* Number of boundary links of wall `wall` (all walls if wall < 0). */
lbm_status lbm_link_count(const lbm_ctx* ctx, int wall, int64_t* count);

/* Change the uniform body force / one wall's velocity (takes effect at the
 * next launch; used by the adjoint driver to set parameters). */
lbm_status lbm_set_body_force(lbm_ctx* ctx, const double g[3]);
lbm_status lbm_set_wall_velocity(lbm_ctx* ctx, int wall, const double u[3]);

/* Initialise f(0) = f^eq(rho, u) (1 + xi) at fluid nodes (Eq. 1, or Eq. 10
 * with the Maxwell term).  rho: N doubles; u: 3*N doubles (canonical layout);
 * xi: Q*N doubles or NULL.  Arrays are on the host if on_host, else on the
 * device.  Host arrays need the STAGE buffer.  Sets T = 0. */
lbm_status lbm_init_equilibrium(lbm_ctx* ctx, const double* rho, const double* u,
                                const double* xi, int on_host, void* stream);

/* Import / export the canonical populations f(T) (dense, Q*N values).
 * dtype: 0 = double, 1 = float.  Solid nodes export as 0 and are ignored on
 * import.  Host arrays need the STAGE buffer; export to host synchronises.
 * Import sets T = 0. */
lbm_status lbm_import_f(lbm_ctx* ctx, const void* src, int dtype, int on_host, void* stream);
lbm_status lbm_export_f(lbm_ctx* ctx, void* dst, int dtype, int on_host, void* stream);

/* Advance nsteps steps of Eq. (2) (fused relaxation, force and propagation). */
lbm_status lbm_step(lbm_ctx* ctx, int nsteps, void* stream);

/* One step from a stored state `src` into `dst` (raw post-collision buffers
 * laid out like LBM_BUF_POP_*, e.g. checkpoints); does not touch the
 * context's own populations or time.  `t` is the index of the step (the time
 * of the canonical state f(t) that src propagates to); with stochastic
 * rounding it selects the same random bits lbm_step used at time t. */
lbm_status lbm_step_from(lbm_ctx* ctx, const void* src, void* dst, int64_t t, void* stream);

/* Copy the current raw stored state out / back in (checkpointing).  Loading
 * sets T to `t` and marks the previous state as unavailable. */
lbm_status lbm_save_state(lbm_ctx* ctx, void* dst, void* stream);
lbm_status lbm_load_state(lbm_ctx* ctx, const void* src, int64_t t, void* stream);

/* Signed wall distance of a curved-wall context (see above): phi_host holds
 * nx*ny*nz floats in the canonical node order, host memory, > 0 exactly at the
 * fluid nodes and < 0 exactly at the solid nodes of the geometry the context
 * was created with (else LBM_ERR_ARG); NULL restores +-1/2 (halfway).  Takes
 * effect for the next step and every later call; synchronises the stream. */
lbm_status lbm_set_wall_distance(lbm_ctx* ctx, const float* phi_host, void* stream);

/* The induced field B(x, T) of an induced-field context (the sums of the
 * field distributions pulled to each node, Sec. 4): B[3][N] doubles owned by
 * the caller, canonical node order (zero at solid nodes), device memory or,
 * with on_host != 0, host memory through the STAGE buffer (synchronises).
 * LBM_ERR_ARG if B is NULL, the context was created without induced = 1, or
 * host output lacks the STAGE buffer. */
lbm_status lbm_export_field(lbm_ctx* ctx, double* B, int on_host, void* stream);

/* Current time T. */
lbm_status lbm_time(const lbm_ctx* ctx, int64_t* t);

/* The kernel that runs this context's step: LBM_STEP_REGISTER or
 * LBM_STEP_STAGED (the automatic choice resolved at lbm_create). */
lbm_status lbm_step_kernel(const lbm_ctx* ctx, int32_t* kind);

/* The imposed electric field that the next step uses (3 doubles, host
 * memory; synchronises the stream): the configured E, or with insulating
 * walls the field set by the last step. */
lbm_status lbm_electric_field(lbm_ctx* ctx, double* E, void* stream);

/* Error flags raised by kernels since the last clear (synchronises the
 * stream): bit 0 = a bounded wait of the staged step kernel expired (about a
 * second without progress; the step was not completed and the state is
 * invalid); bit 1 = the staged step was launched with a pipeline shape it
 * refuses (nothing was computed).  clear != 0 resets them. */
#define LBM_DEVICE_WAIT_TIMEOUT 1u
#define LBM_DEVICE_BAD_LAUNCH 2u
lbm_status lbm_device_status(lbm_ctx* ctx, uint32_t* flags, int clear, void* stream);

/* Stress tensor (Eqs. 8-9, 27-30).  Outputs are dense device arrays in the
 * compute precision (double for F64 storage, else float); any may be NULL:
 * sigma[ncomp][N], S[ncomp][N], rho[N], v[3][N].  S1/S2 use f(T) and report
 * the node's rho and flow velocity v; S3/S4 use the half step between T-1
 * and T (fbar of Eq. 27) and report rho-bar and u-bar; they need T >= 1
 * (LBM_ERR_STATE otherwise).  Solid nodes get zeros. */
lbm_status lbm_stress(lbm_ctx* ctx, int variant, void* sigma, void* S, void* rho, void* v,
                      void* stream);

/* Momentum-exchange force of Eq. (25) exerted during the last step (T-1 -> T)
 * on wall `wall` (every wall if wall < 0), times `weight`; flags
 * LBM_MOVING_CORR | LBM_MAXWELL_REMOVE | LBM_ACCUMULATE.  out: 3 doubles,
 * placed as out_on_host says.  Needs T >= 1.  Reduction: per-link FP64 terms,
 * warp shuffle, block, then a fixed-order pass (deterministic).  It reads the
 * stored state only, so it may run beside the lbm_step that advances from
 * the same state (on another stream, ordered after the previous step). */
lbm_status lbm_wall_force(lbm_ctx* ctx, int wall, unsigned flags, double weight, double* out,
                          int out_on_host, void* stream);

/* lbm_wall_force_noalloc -- the paper has no counterpart; this is a service
 * of the library.  It returns exactly what lbm_wall_force returns (same
 * arguments; the same launch shape and reduction order, so the results are
 * bit-identical at every link count), but it asks for no device memory: its
 * block partial sums and its result slot live in a fixed static device array
 * inside the library (24,640 bytes, held by every GPU that loads the library
 * until the process exits), not in the context's scratch buffer.
 * It is for callers that cannot allocate device memory when they need a
 * force -- their memory is fully committed to population arrays, or is owned
 * by a host application or another runtime that hands out no more -- while
 * the context's scratch buffer is taken by another reduction of the same
 * context queued on a different stream.
 * Limits and caveats:
 *   - at most 1,048,576 links per call (wall < 0 counts every link); larger
 *     requests return LBM_ERR_ARG with a message naming the limit;
 *   - the first call on a device looks up the array's device address (once
 *     per device) and keeps it for the life of the process; make that first
 *     call before any stream capture.  A device reset (cudaDeviceReset, or
 *     the primary context destroyed and created again) invalidates the kept
 *     address: after one, do not call this entry point again in the process;
 *   - all calls share the one array, which keeps the last call's contents
 *     (each call overwrites what it reads, so nothing needs clearing): calls
 *     that overlap on the GPU -- on different streams, from different
 *     contexts or threads on the same device -- race; serialise them. */
lbm_status lbm_wall_force_noalloc(lbm_ctx* ctx, int wall, unsigned flags, double weight, double* out,
                                  int out_on_host, void* stream);

/* One step of Eq. (2) with the wall force of lbm_wall_force fused in: the
 * momentum exchange of Eq. (25) on `wall` during the step T-1 -> T that
 * produced the stored state (what lbm_wall_force returns just before this
 * call), then T -> T+1.  Arguments, flags and outputs as for lbm_wall_force
 * (LBM_MAXWELL_REMOVE adds nothing: the kernel that fuses the force serves
 * contexts without the Maxwell term).  Needs T >= 1.  With the staged step
 * kernel in a box periodic on every axis with the plain node code the links
 * are summed inside the step kernel (FP64 per link and
 * lane, a fixed shuffle tree, one row per block, then the fixed-order pass
 * over the rows by the block that finishes last: deterministic, but in
 * another order than lbm_wall_force, so the two agree to rounding, not bit
 * for bit); otherwise the call is lbm_wall_force then lbm_step. */
lbm_status lbm_step_force(lbm_ctx* ctx, int wall, unsigned flags, double weight, double* out, int out_on_host,
                          void* stream);

/* FP64 sums over fluid nodes of the canonical state f(T), times dx^D:
 * out[0] mass, out[1..3] momentum sum e f, out[4..6] body force sum rho a. */
lbm_status lbm_balance(lbm_ctx* ctx, double* out, int out_on_host, void* stream);

/* Steady-state residual.  Sec. 6 balances the wall force against the body
 * force on the fluid (Eq. 32); the steady form holds once the flow stops
 * changing, which this measures.  With v(x) = u + dt a/2 the flow velocity of
 * the canonical state f(T) at each fluid node (text after Eq. 1; moments
 * summed in FP64 from the stored populations) and v_ref the velocity field of
 * an earlier time:
 *   out[0] = sum |v - v_ref|, out[1] = sum |v|, out[2] = out[0]/out[1]
 * (Euclidean norms, fluid nodes, FP64 block sums in a fixed order; out[2] = 0
 * if out[1] = 0).  v_ref: caller-owned device array of 3*nx*ny*nz doubles,
 * canonical layout v[k][n], 8-byte aligned; with update != 0 each node's
 * v(T) replaces its entries after they are read (solid nodes get 0), so
 * consecutive calls measure the change between them.  out: 3 doubles placed
 * as out_on_host says; LBM_OUT_HOST returns LBM_ERR_NAN for a non-finite
 * result. */
lbm_status lbm_residual(lbm_ctx* ctx, double* v_ref, int update, double* out, int out_on_host, void* stream);

/* Advance until steady: take the residual of the current state into v_ref,
 * then repeat { lbm_step(every); lbm_residual(update) } until the residual
 * over `every` steps is <= tol (LBM_OK) or max_steps steps have been taken
 * (LBM_ERR_NOT_CONVERGED); a non-finite residual stops with LBM_ERR_NAN.
 * v_ref as for lbm_residual; *r_out (may be NULL) receives the last residual
 * and *steps_out (may be NULL) the steps taken.  Synchronises the stream once
 * per `every` steps. */
lbm_status lbm_run_steady(lbm_ctx* ctx, int every, double tol, int64_t max_steps, double* v_ref, double* r_out,
                          int64_t* steps_out, void* stream);

/* Discrete adjoint of J = (1/T) sum_{t<T} d . F_wall(t) (uncorrected momentum
 * exchange on `wall`) for theta = (g, u_w of `wall`), one reverse step t:
 *   phi_t = (dC/df)^T [ S^T phi_{t+1} + dF_t/dfrel seeds ],
 * where C is the node collision at f(t) = propagation of state_prev (the
 * stored post-collision state P_{t-1}, laid out like LBM_BUF_POP_*) and S the
 * propagation with bounce-back.  phi_next (NULL for t = T-1) and phi_out are
 * device arrays laid out like populations but in the compute precision
 * (size from lbm_adjoint_buffer_bytes).  seed_weight = 1/T; dir = d (host, 3
 * doubles).  The u_w gradient collects the Ladd terms of f(t+1) (through
 * phi_next) and of F_t; f(0) is a fixed initial state.  Gradient
 * contributions accumulate in FP64 per-block slots of the scratch buffer;
 * read them with lbm_adjoint_gradient, clear them with lbm_adjoint_reset.
 * Supported: uniform body force, every force model, Maxwell equilibrium;
 * LBM_ERR_UNSUPPORTED with the Lorentz force or LES. */
lbm_status lbm_adjoint_buffer_bytes(const lbm_ctx* ctx, size_t* bytes);
lbm_status lbm_adjoint_reset(lbm_ctx* ctx, void* stream);
lbm_status lbm_adjoint_step(lbm_ctx* ctx, const void* state_prev, const void* phi_next,
                            void* phi_out, int wall, const double* dir, double seed_weight,
                            void* stream);
/* out[0..2] = dJ/dg, out[3..5] = dJ/du_w (host or device). */
lbm_status lbm_adjoint_gradient(lbm_ctx* ctx, double* out, int out_on_host, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
