/*
 * lbm_oracle.h -- plain FP64 CPU oracle of the lattice Boltzmann hot path
 * analysed in arXiv 2512.12213 (Li, "Shear Stress and Fluid-Wall Interaction
 * Force in LBM Simulations of Hydrodynamic and MHD Flows").
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against the paper.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no source, header,
 * table or helper with the CUDA library under paper_2512_12213_gb300/.
 *
 * Everything is double precision, single threaded, node by node, in the order
 * the paper states the algorithm (collide every node, then propagate).
 *
 * Data layout (an interchange format shared with the library's canonical
 * export, written independently on each side):
 *   populations f[a][z][y][x], index a*N + (z*ny + y)*nx + x, N = nx*ny*nz;
 *   per-node scalars s[(z*ny + y)*nx + x]; per-node vectors v[k*N + node].
 * Velocity ordering:
 *   D2Q9 : 0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
 *   D3Q19: 0 rest, 1/2 +-x, 3/4 +-y, 5/6 +-z, 7/8 +-(1,1,0), 9/10 +-(1,-1,0),
 *          11/12 +-(1,0,1), 13/14 +-(1,0,-1), 15/16 +-(0,1,1), 17/18 +-(0,1,-1)
 * Geometry: wall_id[node] = 0 for fluid, k > 0 for a solid node of wall k.
 * A non-periodic axis is closed by a halfway bounce-back wall outside the box
 * on each of its two faces, whose wall id is face_wall[2*axis + (0 low|1 high)].
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_WALLS 16

/* force models of Sec. 2: [a] He, [b] Martys/Luo, [c] Shan-Chen (reformulated),
 * [d] exact difference method (reformulated), [e] Guo */
enum { ORC_FORCE_A = 0, ORC_FORCE_B = 1, ORC_FORCE_C = 2, ORC_FORCE_D = 3, ORC_FORCE_E = 4 };

/* stress variants: 1 = from f^neq with the artefact term E_ij (Eq. 9),
 * 2 = without it (the simplification after Eq. 23), 3 = from the half-step
 * distribution (Eqs. 27-28), 4 = variant 3 plus Theta_ij/2 (Eq. 30) */
enum { ORC_S1 = 1, ORC_S2 = 2, ORC_S3 = 3, ORC_S4 = 4 };

/* wall-force corrections of Sec. 5 */
enum { ORC_MOVING_CORR = 1, ORC_MAXWELL_REMOVE = 2 };

typedef struct orc_cfg {
    int q;                 /* 9 (D2Q9) or 19 (D3Q19) */
    int nx, ny, nz;        /* nz = 1 for D2Q9 */
    int periodic[3];
    double dx, dt, tau, rho0;
    int force_model;       /* ORC_FORCE_* */
    double g[3];           /* uniform body acceleration */
    int lorentz;           /* 1: a = g + (sigma_e/rho) (E + v x B) x B, imposed B, E */
    double B[3], E[3], sigma_e, mu;
    int maxwell;           /* 1: equilibrium of Eq. (10) with the imposed B (in 2-D
                              the field must lie in the plane, B[2] = 0, for the
                              term to carry no mass and the Maxwell stress) */
    int les;               /* 1: Smagorinsky relaxation time from f^neq */
    double cs;             /* Smagorinsky constant */
    int n_walls;           /* wall ids 1..n_walls */
    double wall_u[ORC_MAX_WALLS][3];   /* velocity of wall k at index k-1 */
    int face_wall[6];
    const float* phi;      /* NULL: halfway bounce-back on every solid link.  Else the
                              signed wall distance per node (N floats, > 0 in fluid,
                              < 0 in solid, in lattice units): a solid link from x_f
                              to x_s crosses the wall at x_f + q e with
                              q = phi_f / (phi_f - phi_s), and the incoming population
                              is interpolated (see orc_step).  Closed box faces stay
                              halfway. */
    int insulating;        /* 1 (with lorentz): insulating walls, no net current.  The
                              field E of step t is -<v> x B with <v> the mean flow
                              velocity over fluid nodes of step t-1 (the first step
                              uses E as given); see orc_step_e / orc_run_e */
    int stokes;            /* 1: the linear equilibrium rho w (1 + 3 e.u^eq/c^2) (+ Maxwell
                              term), whose second moment is c^2 rho delta/3 (Stokes
                              equation, the note after Eq. 11) */
    double darcy;          /* >= 0: resistance of a porous medium, a += -darcy v at the
                              flow velocity v (Brinkman equation with stokes = 1) */
    int induced;           /* 1: the field is induced, B(x, t) carried by a vector lattice
                              Boltzmann model (see orc_run_mhd); the fluid sees it through
                              the Maxwell equilibrium of Eq. (10) at the local B (needs
                              maxwell = 1, lorentz = 0); B above is the external field */
    double eta;            /* magnetic diffusivity of the induced field */
    int mag_conducting;    /* walls for the field: 0 insulating (B = B_ext at the wall),
                              1 perfectly conducting (no normal gradient) */
    const double* Bfield;  /* NULL, or the local field B[3][N] that orc_stress and
                              orc_wall_force use instead of B (induced runs) */
} orc_cfg;

/* threads of the node loops: 1 for the parity build, the OpenMP thread count
 * for the timing build (the same source compiled with -fopenmp) */
int orc_threads(void);

/* lattice tables: e (unit-speed integers, Q*3), w (Q), opposite index (Q) */
int orc_lattice(int q, int* e, double* w, int* opp);

/* equilibrium of Eq. (1), plus the Maxwell term of Eq. (10) if cfg->maxwell */
void orc_feq(const orc_cfg* c, double rho, const double* u, double* out);

/* per-node macroscopic quantities for pre-collision populations f[Q]:
 * out[0] rho, out[1..3] u, out[4..6] v, out[7..9] a, out[10..12] u^eq,
 * out[13..15] u^F, out[16] C, out[17] tau_eff */
void orc_node_macro(const orc_cfg* c, const double* f, double* out);

/* force term F_alpha of the configured model at a node (Sec. 2) */
void orc_force_term(const orc_cfg* c, const double* f, double* F);

/* relaxation of Eq. (2): frel = f + (f^eq - f)/tau + F at one node */
void orc_collide_node(const orc_cfg* c, const double* f, double* frel);

/* canonical initial state f = f^eq(rho(x), u(x)) * (1 + xi) at fluid nodes,
 * 0 at solid nodes; u is [3][N]; xi may be NULL */
void orc_init(const orc_cfg* c, const unsigned char* wall_id, const double* rho,
              const double* u, const double* xi, double* f);

/* one step of Eq. (2): f (in: f(t), out: f(t+dt)); frel (N*Q) receives
 * f^rel(t) if not NULL.  A population f^rel_a(x_f) leaving a fluid node into
 * a solid node returns as f_b(x_f, t+dt), b = opp(a), by halfway bounce-back
 * f_b = f^rel_a(x_f) - L (L the moving-wall term) or, with cfg->phi, by linear
 * interpolation at the wall point x_f + q e_a:
 *   q <  1/2: f_b = 2q f^rel_a(x_f) + (1 - 2q) f^rel_a(x_f + e_b) - L
 *   q >= 1/2: f_b = (f^rel_a(x_f) - L)/(2q) + (1 - 1/(2q)) f^rel_b(x_f)
 * (halfway when q < 1/2 and x_f + e_b is not a fluid node).  The momentum
 * exchange of Eq. (25) with these values refers to the imaginary point
 * x_f + e_a/2 (discussion after Eq. 25). */
void orc_step(const orc_cfg* c, const unsigned char* wall_id, double* f, double* frel);

/* run n steps in place (with cfg->insulating, E starts at cfg->E and is
 * updated from step to step) */
void orc_run(const orc_cfg* c, const unsigned char* wall_id, double* f, int n);

/* the same with the field as explicit state: E[3] is the field of the first
 * step on entry and, with cfg->insulating, the field of the next step on exit
 * (-<v> x B of the last step, Eq. 36); frel as in orc_step (last step) */
void orc_step_e(const orc_cfg* c, const unsigned char* wall_id, double* f, double* frel, double* E);
void orc_run_e(const orc_cfg* c, const unsigned char* wall_id, double* f, int n, double* E);

/* Induced field (Sec. 4 cites Dellar's vector lattice Boltzmann model for
 * the induction equation dB/dt + div(v B - B v) = eta lap B): components
 * g[k][i][N] (k = x, y, z) on D2Q5 (weights 1/3, 1/6; theta = 1/3) or D3Q7
 * (1/4, 1/8; theta = 1/4) with the axis velocities of the fluid lattice.
 * Per step, from the fluid state f(t) and g(t): B = sum_i g_i at each fluid
 * node; the fluid relaxes with the Maxwell equilibrium at that B; the field
 * relaxes to g^eq_ik = W_i [B_k + e_ij (v_j B_k - B_j v_k)/(theta c)] with the
 * node's flow velocity v and tau_m = 1/2 + eta/(theta c^2 dt); both
 * propagate.  A field link into a wall returns anti-bounced,
 * -g'_i + 2 W_i B_ext (insulating) or bounced, g'_i (conducting).
 * orc_mag_init sets g = W_i B_ext at fluid nodes (0 at solids);
 * orc_mag_field gives B[3][N] = sum_i g (0 at solids). */
int orc_mag_q(int q);
void orc_mag_init(const orc_cfg* c, const unsigned char* wall_id, double* g);
void orc_mag_field(const orc_cfg* c, const unsigned char* wall_id, const double* g, double* B);
/* n coupled steps; frel (N*Q, may be NULL) receives f^rel of the last step */
void orc_run_mhd(const orc_cfg* c, const unsigned char* wall_id, double* f, double* g, int n, double* frel);

/* momentum-exchange force of Eq. (25) on wall `wall` (or every wall if
 * wall < 0) during the step t -> t+dt, from frel = f^rel(t) and
 * fnext = f(t+dt); flags ORC_MOVING_CORR | ORC_MAXWELL_REMOVE; out[3] */
void orc_wall_force(const orc_cfg* c, const unsigned char* wall_id, const double* frel,
                    const double* fnext, int wall, int flags, double* out);

/* number of boundary links of wall `wall` (or all walls if < 0) */
long orc_count_links(const orc_cfg* c, const unsigned char* wall_id, int wall);

/* stress tensor per node.  Variants 1, 2 use f = f(t); variants 3, 4 use
 * frel = f^rel(t) and fnext = f(t+dt).  sigma, S: ncomp*N (ncomp 3 in 2-D:
 * xx yy xy; 6 in 3-D: xx yy zz xy xz yz); rho: N; v: 3*N (for variants 1-2 the
 * node's rho and flow velocity v, for 3-4 the half-step rho-bar and u-bar).
 * Solid nodes get zeros. */
void orc_stress(const orc_cfg* c, const unsigned char* wall_id, const double* f,
                const double* frel, const double* fnext, int variant,
                double* sigma, double* S, double* rho, double* v);

/* global sums of the canonical state f(t) over fluid nodes, times dx^D:
 * out[0] mass, out[1..3] momentum sum_x sum_a e f, out[4..6] sum rho a */
void orc_balance(const orc_cfg* c, const unsigned char* wall_id, const double* f, double* out);

/* steady-state residual (Sec. 6): with v the flow velocity v = u + dt a/2 of
 * the canonical state f at each fluid node and vref [3][N] the velocity of an
 * earlier time (NULL: zero), out[0] = sum |v - vref|, out[1] = sum |v|,
 * out[2] = out[0]/out[1] (0 if out[1] = 0), Euclidean norms, fluid nodes
 * only; v [3][N] (may be NULL) receives the velocity, 0 at solid nodes */
void orc_residual(const orc_cfg* c, const unsigned char* wall_id, const double* f,
                  const double* vref, double* v, double* out);

/* time-averaged drag J = (1/T) sum_{t=0}^{T-1} d . F_wall(t) (uncorrected
 * momentum exchange on wall `wall`) from the canonical initial state f0, and
 * its gradient with respect to theta = (g[0..2], u_w[0..2] of `wall`), by the
 * discrete adjoint with complex-step collision Jacobians.  grad[6].  Returns
 * -2 with cfg->phi (interpolated walls have no transpose here). */
int orc_adjoint_drag(const orc_cfg* c, const unsigned char* wall_id, const double* f0, int T,
                     int wall, const double* d, double* J, double* grad);

/* J alone (forward only), for finite differences */
double orc_drag_average(const orc_cfg* c, const unsigned char* wall_id, const double* f0, int T,
                        int wall, const double* d);

#ifdef __cplusplus
}
#endif
#endif
