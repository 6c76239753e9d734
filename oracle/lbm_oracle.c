/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the lattice Boltzmann hot path of
 * arXiv 2512.12213.  TEST INFRASTRUCTURE ONLY: see lbm_oracle.h.
 *
 * The algorithm is taken in the paper's order: at every fluid node the
 * populations are relaxed with the force term (Eq. 2), then every relaxed
 * population is propagated to x + dt e_a; a population whose destination is
 * solid returns to its origin reversed (halfway bounce-back), with Ladd's
 * moving-wall term 6 w_a rho_w (e_a . u_w)/c^2 taken off, rho_w = rho0.
 * The wall force is the momentum exchange of Eq. (25) summed over boundary
 * links.  The adjoint is the transpose of this same recursion, with each
 * node's collision Jacobian obtained by complex-step differentiation of the
 * collision formulas of oracle_node.inc.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "lbm_oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

/* threads the node loops of a step use: 1 in the parity build */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

typedef struct {
    int q, d;
    int e[19][3];
    double w[19];
    int opp[19];
} lat_t;

/* D2Q9 and D3Q19 velocity sets (Qian et al., cited in Sec. 2), unit speed */
static const int E9[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const int E19[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static int get_lat(int q, lat_t* L)
{
    if (q != 9 && q != 19) return -1;
    L->q = q;
    L->d = (q == 9) ? 2 : 3;
    for (int a = 0; a < q; ++a) {
        int n2 = 0;
        for (int k = 0; k < 3; ++k) {
            L->e[a][k] = (q == 9) ? E9[a][k] : E19[a][k];
            n2 += L->e[a][k] * L->e[a][k];
        }
        /* weights by speed class: D2Q9 4/9, 1/9, 1/36; D3Q19 1/3, 1/18, 1/36 */
        if (q == 9) L->w[a] = (n2 == 0) ? 4.0 / 9.0 : (n2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
        else        L->w[a] = (n2 == 0) ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b)
            if (L->e[b][0] == -L->e[a][0] && L->e[b][1] == -L->e[a][1] && L->e[b][2] == -L->e[a][2])
                L->opp[a] = b;
    return 0;
}

/* Maxwell-stress part of the MHD equilibrium, Eq. (10), for direction a */
static double maxwell_delta(const orc_cfg* c, const lat_t* L, int a)
{
    const double cc = c->dx / c->dt;
    double ee = 0, eB = 0, B2 = 0;
    for (int k = 0; k < 3; ++k) {
        ee += (cc * L->e[a][k]) * (cc * L->e[a][k]);
        eB += (cc * L->e[a][k]) * c->B[k];
        B2 += c->B[k] * c->B[k];
    }
    double m = 0.5 * B2 * ee - eB * eB;
    if (L->d == 3) m -= cc * cc * B2 / 6.0;
    return 9.0 * L->w[a] / (2.0 * cc * cc * cc * cc * c->mu) * m;
}

/* ---- per-node formulas, real and complex instances ---- */
#define R double
#define SQRT sqrt
#define FN(n) n##_r
#include "oracle_node.inc"
#undef R
#undef SQRT
#undef FN

#define R double complex
#define SQRT csqrt
#define FN(n) n##_c
#include "oracle_node.inc"
#undef R
#undef SQRT
#undef FN

/* ---- geometry ---- */

static long nnodes(const orc_cfg* c) { return (long)c->nx * c->ny * c->nz; }

/* Destination of the link leaving node (x, y, z) along direction a.
 * Returns the destination node index if it is a fluid node; otherwise -1 and
 * the wall id of the solid it hits in *wall.  Periodic axes wrap.  A link
 * that leaves the box through several closed faces at once takes the wall of
 * the first such axis in the order x, y, z. */
static long link_dest(const orc_cfg* c, const lat_t* L, const unsigned char* wid,
                      int x, int y, int z, int a, int* wall)
{
    int p[3] = {x + L->e[a][0], y + L->e[a][1], z + L->e[a][2]};
    const int n[3] = {c->nx, c->ny, c->nz};
    for (int k = 0; k < 3; ++k) {
        if (p[k] >= 0 && p[k] < n[k]) continue;
        if (c->periodic[k]) {
            p[k] = (p[k] + n[k]) % n[k];
        } else {
            *wall = c->face_wall[2 * k + (p[k] < 0 ? 0 : 1)];
            return -1;
        }
    }
    long d = ((long)p[2] * c->ny + p[1]) * c->nx + p[0];
    if (wid[d] != 0) {
        *wall = wid[d];
        return -1;
    }
    return d;
}

/* index of the node one link away along a (periodic axes wrap), or -1 when
 * the link leaves the box through a closed face */
static long neighbour(const orc_cfg* c, const lat_t* L, int x, int y, int z, int a)
{
    int p[3] = {x + L->e[a][0], y + L->e[a][1], z + L->e[a][2]};
    const int n[3] = {c->nx, c->ny, c->nz};
    for (int k = 0; k < 3; ++k) {
        if (p[k] >= 0 && p[k] < n[k]) continue;
        if (!c->periodic[k]) return -1;
        p[k] = (p[k] + n[k]) % n[k];
    }
    return ((long)p[2] * c->ny + p[1]) * c->nx + p[0];
}

static const double* wall_velocity(const orc_cfg* c, int wall)
{
    static const double zero[3] = {0, 0, 0};
    if (wall < 1 || wall > c->n_walls) return zero;
    return c->wall_u[wall - 1];
}

/* the configuration at node n: with a local field (induced runs) B is that
 * node's field */
static const orc_cfg* node_cfg(const orc_cfg* c, long n, orc_cfg* tmp)
{
    if (!c->Bfield) return c;
    *tmp = *c;
    const long N = (long)c->nx * c->ny * c->nz;
    for (int k = 0; k < 3; ++k) tmp->B[k] = c->Bfield[k * N + n];
    return tmp;
}

/* Ladd's moving-wall term for a population leaving along a into a wall */
static double ladd(const orc_cfg* c, const lat_t* L, int a, int wall)
{
    const double cc = c->dx / c->dt;
    const double* uw = wall_velocity(c, wall);
    double eu = 0;
    for (int k = 0; k < 3; ++k) eu += (cc * L->e[a][k]) * uw[k];
    return 6.0 * L->w[a] * c->rho0 * eu / (cc * cc);
}

static double cell_volume(const orc_cfg* c, const lat_t* L)
{
    return (L->d == 3) ? c->dx * c->dx * c->dx : c->dx * c->dx;
}

/* ---- public API ---- */

int orc_lattice(int q, int* e, double* w, int* opp)
{
    lat_t L;
    if (get_lat(q, &L)) return -1;
    for (int a = 0; a < q; ++a) {
        for (int k = 0; k < 3; ++k) e[3 * a + k] = L.e[a][k];
        w[a] = L.w[a];
        opp[a] = L.opp[a];
    }
    return 0;
}

void orc_feq(const orc_cfg* c, double rho, const double* u, double* out)
{
    lat_t L;
    get_lat(c->q, &L);
    feq_r(c, &L, rho, u, out);
}

void orc_node_macro(const orc_cfg* c, const double* f, double* out)
{
    lat_t L;
    get_lat(c->q, &L);
    macro_t_r m;
    macro_r(c, &L, f, c->g, &m);
    out[0] = m.rho;
    for (int k = 0; k < 3; ++k) {
        out[1 + k] = m.u[k];
        out[4 + k] = m.v[k];
        out[7 + k] = m.a[k];
        out[10 + k] = m.ueq[k];
        out[13 + k] = m.uF[k];
    }
    out[16] = m.C;
    out[17] = m.tau;
}

void orc_force_term(const orc_cfg* c, const double* f, double* F)
{
    lat_t L;
    get_lat(c->q, &L);
    macro_t_r m;
    macro_r(c, &L, f, c->g, &m);
    force_r(c, &L, &m, F);
}

void orc_collide_node(const orc_cfg* c, const double* f, double* frel)
{
    lat_t L;
    get_lat(c->q, &L);
    collide_r(c, &L, f, c->g, frel);
}

void orc_init(const orc_cfg* c, const unsigned char* wid, const double* rho,
              const double* u, const double* xi, double* f)
{
    lat_t L;
    get_lat(c->q, &L);
    const long N = nnodes(c);
    for (long n = 0; n < N; ++n) {
        double fe[19], un[3] = {u[n], u[N + n], u[2 * N + n]};
        if (wid[n] != 0) {
            for (int a = 0; a < L.q; ++a) f[a * N + n] = 0.0;
            continue;
        }
        feq_r(c, &L, rho[n], un, fe);
        for (int a = 0; a < L.q; ++a) f[a * N + n] = fe[a] * (1.0 + (xi ? xi[a * N + n] : 0.0));
    }
}

/* propagation of f^rel to x + dt e_a, halfway or interpolated bounce-back at
 * solids (see orc_step) */
static void propagate(const orc_cfg* c, const lat_t* L, const unsigned char* wid, const double* frel, double* fnew)
{
    const long N = nnodes(c);
    const int Q = L->q;
    memset(fnew, 0, sizeof(double) * N * Q);
    /* every destination entry is written by exactly one (node, direction), so
     * the planes are independent; the pragma only acts in the OpenMP timing
     * build (the parity build is compiled without -fopenmp) */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                long n = ((long)z * c->ny + y) * c->nx + x;
                if (wid[n] != 0) continue;
                for (int a = 0; a < Q; ++a) {
                    int wall = 0;
                    long d = link_dest(c, L, wid, x, y, z, a, &wall);
                    if (d >= 0) {
                        fnew[a * N + d] = frel[a * N + n];
                        continue;
                    }
                    const int b = L->opp[a];
                    const double out = frel[a * N + n] - ladd(c, L, a, wall);
                    const long s = c->phi ? neighbour(c, L, x, y, z, a) : -1;
                    if (s < 0 || wid[s] == 0) {            /* box face, or no wall distance */
                        fnew[b * N + n] = out;
                        continue;
                    }
                    const double q = (double)c->phi[n] / ((double)c->phi[n] - (double)c->phi[s]);
                    if (q >= 0.5) {
                        fnew[b * N + n] = out / (2.0 * q) + (1.0 - 1.0 / (2.0 * q)) * frel[b * N + n];
                    } else {
                        int w2 = 0;
                        const long ff = link_dest(c, L, wid, x, y, z, b, &w2);
                        fnew[b * N + n] = (ff < 0) ? out
                                                   : 2.0 * q * frel[a * N + n] + (1.0 - 2.0 * q) * frel[a * N + ff] -
                                                         ladd(c, L, a, wall);
                    }
                }
            }
}

/* one step with caller work arrays frel (N*Q) and fnew (N*Q); vmean (if not
 * NULL) receives the mean flow velocity v over the fluid nodes */
static void step_work(const orc_cfg* c, const lat_t* L, const unsigned char* wid,
                      double* f, double* frel, double* fnew, double* vmean)
{
    const long N = nnodes(c);
    const int Q = L->q;
    /* relaxation with the force term at every fluid node, Eq. (2) (nodes
     * independent: parallel in the OpenMP timing build only) */
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (wid[n] != 0) {
            for (int a = 0; a < Q; ++a) frel[a * N + n] = 0.0;
            continue;
        }
        double fl[19], out[19];
        for (int a = 0; a < Q; ++a) fl[a] = f[a * N + n];
        collide_r(c, L, fl, c->g, out);
        for (int a = 0; a < Q; ++a) frel[a * N + n] = out[a];
    }
    /* the mean flow velocity of the pre-collision state, summed in node order */
    if (vmean) {
        double vs[3] = {0.0, 0.0, 0.0};
        long nf = 0;
        for (long n = 0; n < N; ++n) {
            if (wid[n] != 0) continue;
            double fl[19];
            for (int a = 0; a < Q; ++a) fl[a] = f[a * N + n];
            macro_t_r m;
            macro_r(c, L, fl, c->g, &m);
            for (int k = 0; k < 3; ++k) vs[k] += m.v[k];
            ++nf;
        }
        for (int k = 0; k < 3; ++k) vmean[k] = nf ? vs[k] / (double)nf : 0.0;
    }
    propagate(c, L, wid, frel, fnew);
    memcpy(f, fnew, sizeof(double) * N * Q);
}

/* insulating walls (Eq. 36): the field that makes the net current
 * sigma_e sum (E + v x B) over fluid nodes vanish, E = -<v> x B */
static void insulating_field(const orc_cfg* c, const double* vmean, double* E)
{
    E[0] = -(vmean[1] * c->B[2] - vmean[2] * c->B[1]);
    E[1] = -(vmean[2] * c->B[0] - vmean[0] * c->B[2]);
    E[2] = -(vmean[0] * c->B[1] - vmean[1] * c->B[0]);
}

void orc_run_e(const orc_cfg* c, const unsigned char* wid, double* f, int nsteps, double* E)
{
    lat_t L;
    get_lat(c->q, &L);
    const long N = nnodes(c);
    double* frel = (double*)malloc(sizeof(double) * N * L.q);
    double* fnew = (double*)malloc(sizeof(double) * N * L.q);
    orc_cfg cc = *c;
    for (int k = 0; k < 3; ++k) cc.E[k] = E[k];
    const int ins = c->insulating && c->lorentz;
    for (int s = 0; s < nsteps; ++s) {
        double vm[3];
        step_work(&cc, &L, wid, f, frel, fnew, ins ? vm : NULL);
        if (ins) insulating_field(c, vm, cc.E);
    }
    for (int k = 0; k < 3; ++k) E[k] = cc.E[k];
    free(frel);
    free(fnew);
}

void orc_step_e(const orc_cfg* c, const unsigned char* wid, double* f, double* frel_out, double* E)
{
    lat_t L;
    get_lat(c->q, &L);
    const long N = nnodes(c);
    double* frel = (double*)malloc(sizeof(double) * N * L.q);
    double* fnew = (double*)malloc(sizeof(double) * N * L.q);
    orc_cfg cc = *c;
    for (int k = 0; k < 3; ++k) cc.E[k] = E[k];
    double vm[3];
    step_work(&cc, &L, wid, f, frel, fnew, vm);
    if (c->insulating && c->lorentz) insulating_field(c, vm, E);
    if (frel_out) memcpy(frel_out, frel, sizeof(double) * N * L.q);
    free(frel);
    free(fnew);
}

void orc_step(const orc_cfg* c, const unsigned char* wid, double* f, double* frel_out)
{
    double E[3] = {c->E[0], c->E[1], c->E[2]};
    orc_step_e(c, wid, f, frel_out, E);
}

void orc_run(const orc_cfg* c, const unsigned char* wid, double* f, int nsteps)
{
    double E[3] = {c->E[0], c->E[1], c->E[2]};
    orc_run_e(c, wid, f, nsteps, E);
}

/* ---- induced field ---- */

typedef struct {
    int q;
    int e[7][3];
    double w[7], theta;
    int opp[7];
} mlat_t;

static void get_mlat(int fq, mlat_t* M)
{
    static const int e7[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    static const int e5[5][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}};
    M->q = (fq == 9) ? 5 : 7;
    M->theta = (fq == 9) ? 1.0 / 3.0 : 0.25;
    for (int i = 0; i < M->q; ++i) {
        for (int k = 0; k < 3; ++k) M->e[i][k] = (fq == 9) ? e5[i][k] : e7[i][k];
        M->w[i] = (i == 0) ? ((fq == 9) ? 1.0 / 3.0 : 0.25) : ((fq == 9) ? 1.0 / 6.0 : 0.125);
    }
    for (int i = 0; i < M->q; ++i)
        for (int j = 0; j < M->q; ++j)
            if (M->e[j][0] == -M->e[i][0] && M->e[j][1] == -M->e[i][1] && M->e[j][2] == -M->e[i][2]) M->opp[i] = j;
}

int orc_mag_q(int q) { return q == 9 ? 5 : 7; }

void orc_mag_init(const orc_cfg* c, const unsigned char* wid, double* g)
{
    mlat_t M;
    get_mlat(c->q, &M);
    const long N = nnodes(c);
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < M.q; ++i)
            for (long n = 0; n < N; ++n) g[((long)k * M.q + i) * N + n] = wid[n] ? 0.0 : M.w[i] * c->B[k];
}

void orc_mag_field(const orc_cfg* c, const unsigned char* wid, const double* g, double* B)
{
    mlat_t M;
    get_mlat(c->q, &M);
    const long N = nnodes(c);
    for (int k = 0; k < 3; ++k)
        for (long n = 0; n < N; ++n) {
            double s = 0.0;
            if (!wid[n])
                for (int i = 0; i < M.q; ++i) s += g[((long)k * M.q + i) * N + n];
            B[k * N + n] = s;
        }
}

/* node one step along the field-lattice velocity e (periodic wrap); -1 with
 * the wall id when it is solid or outside a closed face */
static long mlink_dest(const orc_cfg* c, const unsigned char* wid, int x, int y, int z, const int* e)
{
    int p[3] = {x + e[0], y + e[1], z + e[2]};
    const int n[3] = {c->nx, c->ny, c->nz};
    for (int k = 0; k < 3; ++k) {
        if (p[k] >= 0 && p[k] < n[k]) continue;
        if (!c->periodic[k]) return -1;
        p[k] = (p[k] + n[k]) % n[k];
    }
    long d = ((long)p[2] * c->ny + p[1]) * c->nx + p[0];
    return wid[d] ? -1 : d;
}

void orc_run_mhd(const orc_cfg* c, const unsigned char* wid, double* f, double* g, int nsteps, double* frel_out)
{
    lat_t L;
    mlat_t M;
    get_lat(c->q, &L);
    get_mlat(c->q, &M);
    const long N = nnodes(c);
    const int Q = L.q, Qm = M.q;
    const double cc = c->dx / c->dt;
    const double taum = 0.5 + c->eta / (M.theta * cc * cc * c->dt);
    double* frel = (double*)malloc(sizeof(double) * N * Q);
    double* fnew = (double*)malloc(sizeof(double) * N * Q);
    double* grel = (double*)malloc(sizeof(double) * 3 * Qm * N);
    for (int s = 0; s < nsteps; ++s) {
        memset(grel, 0, sizeof(double) * 3 * Qm * N);
        for (long n = 0; n < N; ++n) {
            if (wid[n] != 0) {
                for (int a = 0; a < Q; ++a) frel[a * N + n] = 0.0;
                continue;
            }
            /* the node's field, and the fluid relaxation with the Maxwell
             * equilibrium of Eq. (10) at that field */
            orc_cfg cn = *c;
            for (int k = 0; k < 3; ++k) {
                double b = 0.0;
                for (int i = 0; i < Qm; ++i) b += g[((long)k * Qm + i) * N + n];
                cn.B[k] = b;
            }
            double fl[19], out[19];
            for (int a = 0; a < Q; ++a) fl[a] = f[a * N + n];
            collide_r(&cn, &L, fl, c->g, out);
            for (int a = 0; a < Q; ++a) frel[a * N + n] = out[a];
            macro_t_r m;
            macro_r(&cn, &L, fl, c->g, &m);
            /* the field relaxation: Lambda_jk = v_j B_k - B_j v_k */
            double Lam[3][3];
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) Lam[j][k] = m.v[j] * cn.B[k] - cn.B[j] * m.v[k];
            for (int k = 0; k < 3; ++k)
                for (int i = 0; i < Qm; ++i) {
                    double el = 0.0;
                    for (int j = 0; j < 3; ++j) el += M.e[i][j] * Lam[j][k];
                    const double geq = M.w[i] * (cn.B[k] + el / (M.theta * cc));
                    const double gi = g[((long)k * Qm + i) * N + n];
                    grel[((long)k * Qm + i) * N + n] = gi - (gi - geq) / taum;
                }
        }
        propagate(c, &L, wid, frel, fnew);
        memcpy(f, fnew, sizeof(double) * N * Q);
        memset(g, 0, sizeof(double) * 3 * Qm * N);
        for (int z = 0; z < c->nz; ++z)
            for (int y = 0; y < c->ny; ++y)
                for (int x = 0; x < c->nx; ++x) {
                    const long n = ((long)z * c->ny + y) * c->nx + x;
                    if (wid[n] != 0) continue;
                    for (int i = 0; i < Qm; ++i) {
                        const long d = mlink_dest(c, wid, x, y, z, M.e[i]);
                        for (int k = 0; k < 3; ++k) {
                            const double gr = grel[((long)k * Qm + i) * N + n];
                            if (d >= 0) g[((long)k * Qm + i) * N + d] = gr;
                            else g[((long)k * Qm + M.opp[i]) * N + n] =
                                     c->mag_conducting ? gr : -gr + 2.0 * M.w[i] * c->B[k];
                        }
                    }
                }
        if (frel_out && s == nsteps - 1) memcpy(frel_out, frel, sizeof(double) * N * Q);
    }
    free(frel);
    free(fnew);
    free(grel);
}

void orc_wall_force(const orc_cfg* c, const unsigned char* wid, const double* frel,
                    const double* fnext, int wall, int flags, double* out)
{
    lat_t L;
    get_lat(c->q, &L);
    const long N = nnodes(c);
    const double cc = c->dx / c->dt, s = cell_volume(c, &L) / c->dt;
    out[0] = out[1] = out[2] = 0.0;
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                long n = ((long)z * c->ny + y) * c->nx + x;
                if (wid[n] != 0) continue;
                orc_cfg tmp;
                const orc_cfg* cn = node_cfg(c, n, &tmp);
                for (int a = 0; a < L.q; ++a) {
                    int lw = 0;
                    if (link_dest(c, &L, wid, x, y, z, a, &lw) >= 0) continue;
                    if (wall >= 0 && lw != wall) continue;
                    /* outgoing f-bar_{a'} = f^rel(x_f, t); bounced
                     * f-bar_a = f(x_f, t + dt) in the reversed direction */
                    double fo = frel[a * N + n], fi = fnext[L.opp[a] * N + n];
                    const double* uw = wall_velocity(c, lw);
                    for (int k = 0; k < 3; ++k) {
                        double ek = cc * L.e[a][k];
                        double d = ek * (fo + fi);
                        if (flags & ORC_MOVING_CORR) d += uw[k] * (fi - fo);
                        if ((flags & ORC_MAXWELL_REMOVE) && c->maxwell)
                            d -= 2.0 * ek * maxwell_delta(cn, &L, a);
                        out[k] += s * d;
                    }
                }
            }
}

long orc_count_links(const orc_cfg* c, const unsigned char* wid, int wall)
{
    lat_t L;
    get_lat(c->q, &L);
    long cnt = 0;
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                long n = ((long)z * c->ny + y) * c->nx + x;
                if (wid[n] != 0) continue;
                orc_cfg tmp;
                const orc_cfg* cn = node_cfg(c, n, &tmp);
                for (int a = 0; a < L.q; ++a) {
                    int lw = 0;
                    if (link_dest(c, &L, wid, x, y, z, a, &lw) >= 0) continue;
                    if (wall < 0 || lw == wall) ++cnt;
                }
            }
    return cnt;
}

/* Theta_ij of Eq. (4) for models [b]-[e]; zero for [a] */
static void theta_of(const orc_cfg* c, const macro_t_r* m, double T[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            T[i][j] = (c->force_model == ORC_FORCE_A)
                          ? 0.0
                          : m->C * c->dt * m->rho * (m->uF[i] * m->a[j] + m->uF[j] * m->a[i]);
}

void orc_stress(const orc_cfg* c0, const unsigned char* wid, const double* f,
                const double* frel, const double* fnext, int variant,
                double* sigma, double* S, double* rho_out, double* v_out)
{
    const orc_cfg* c = c0;
    lat_t L;
    get_lat(c->q, &L);
    const long N = nnodes(c);
    const int Q = L.q, D = L.d, nc = (D == 3) ? 6 : 3;
    const double cc = c->dx / c->dt, dt = c->dt;
    const int ci[6] = {0, 1, 2, 0, 0, 1}, cj[6] = {0, 1, 2, 1, 2, 2};
    const int ci2[3] = {0, 1, 0}, cj2[3] = {0, 1, 1};
    for (long n = 0; n < N; ++n) {
        orc_cfg ncfg;
        const orc_cfg* c = node_cfg(c0, n, &ncfg);     /* the node's field in induced runs */
        double sig[3][3] = {{0}}, rr = 0, vv[3] = {0, 0, 0}, nu;
        if (wid[n] == 0) {
            double fl[19];
            for (int a = 0; a < Q; ++a) fl[a] = f[a * N + n];
            macro_t_r m;
            macro_r(c, &L, fl, c->g, &m);
            double Th[3][3];
            theta_of(c, &m, Th);
            nu = dt * cc * cc * (m.tau - 0.5) / 3.0;
            if (variant == ORC_S1 || variant == ORC_S2) {
                /* Eq. (9): S_ij = -3/(2 tau dt c^2 rho) [sum e_i e_j (f - f^eq) + E_ij],
                 * E_ij = tau dt (u^eq_i rho a_j + u^eq_j rho a_i) - tau Theta_ij;
                 * Eq. (8): sigma = 2 rho nu S.  Variant 2 drops E_ij. */
                double fe[19];
                feq_r(c, &L, m.rho, m.ueq, fe);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double P = 0;
                        for (int a = 0; a < Q; ++a)
                            P += (cc * L.e[a][i]) * (cc * L.e[a][j]) * (fl[a] - fe[a]);
                        double E = m.tau * dt * (m.ueq[i] * m.rho * m.a[j] + m.ueq[j] * m.rho * m.a[i])
                                   - m.tau * Th[i][j];
                        double Sij = -3.0 / (2.0 * m.tau * dt * cc * cc * m.rho)
                                     * (P + (variant == ORC_S1 ? E : 0.0));
                        sig[i][j] = 2.0 * m.rho * nu * Sij;
                    }
                rr = m.rho;
                for (int k = 0; k < 3; ++k) vv[k] = m.v[k];
            } else {
                /* Eq. (27): f-bar = (f^rel(x,t) + f(x,t+dt))/2; sigma from its
                 * non-equilibrium part about f^eq(rho-bar, u-bar) (Eq. 28);
                 * variant 4 adds Theta_ij/2 (Eq. 30) */
                double fb[19], rb = 0, ub[3] = {0, 0, 0}, fe[19];
                for (int a = 0; a < Q; ++a) {
                    fb[a] = 0.5 * (frel[a * N + n] + fnext[a * N + n]);
                    rb += fb[a];
                    for (int k = 0; k < 3; ++k) ub[k] += (cc * L.e[a][k]) * fb[a];
                }
                for (int k = 0; k < 3; ++k) ub[k] /= rb;
                feq_r(c, &L, rb, ub, fe);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double P = 0;
                        for (int a = 0; a < Q; ++a)
                            P += (cc * L.e[a][i]) * (cc * L.e[a][j]) * (fb[a] - fe[a]);
                        sig[i][j] = -P + (variant == ORC_S4 ? 0.5 * Th[i][j] : 0.0);
                    }
                rr = rb;
                for (int k = 0; k < 3; ++k) vv[k] = ub[k];
            }
        } else {
            nu = 1.0;
        }
        for (int k = 0; k < nc; ++k) {
            int i = (D == 3) ? ci[k] : ci2[k], j = (D == 3) ? cj[k] : cj2[k];
            sigma[k * N + n] = sig[i][j];
            S[k * N + n] = (wid[n] == 0) ? sig[i][j] / (2.0 * rr * nu) : 0.0;
        }
        if (rho_out) rho_out[n] = rr;
        if (v_out)
            for (int k = 0; k < 3; ++k) v_out[k * N + n] = vv[k];
    }
}

void orc_balance(const orc_cfg* c, const unsigned char* wid, const double* f, double* out)
{
    lat_t L;
    get_lat(c->q, &L);
    const long N = nnodes(c);
    const double cc = c->dx / c->dt, vol = cell_volume(c, &L);
    for (int k = 0; k < 7; ++k) out[k] = 0.0;
    for (long n = 0; n < N; ++n) {
        if (wid[n] != 0) continue;
        double fl[19];
        for (int a = 0; a < L.q; ++a) {
            fl[a] = f[a * N + n];
            out[0] += vol * fl[a];
            for (int k = 0; k < 3; ++k) out[1 + k] += vol * (cc * L.e[a][k]) * fl[a];
        }
        macro_t_r m;
        macro_r(c, &L, fl, c->g, &m);
        for (int k = 0; k < 3; ++k) out[4 + k] += vol * m.rho * m.a[k];
    }
}

/* Steady-state residual (Sec. 6: the global balance of Eq. 32 between wall
 * force and body force holds once the flow no longer changes).  At every
 * fluid node the flow velocity v = u + dt a/2 of the canonical state f (text
 * after Eq. 1) is compared with a reference velocity field vref of an earlier
 * time:
 *   out[0] = sum_x |v(x) - vref(x)|,  out[1] = sum_x |v(x)|,
 *   out[2] = out[0] / out[1]  (0 when out[1] = 0),
 * with |.| the Euclidean norm and the sums over fluid nodes in node order.
 * vref: [3][N] (NULL: zero); v (may be NULL) receives v [3][N], 0 at solids. */
void orc_residual(const orc_cfg* c, const unsigned char* wid, const double* f, const double* vref,
                  double* v, double* out)
{
    lat_t L;
    get_lat(c->q, &L);
    const long N = nnodes(c);
    out[0] = out[1] = out[2] = 0.0;
    for (long n = 0; n < N; ++n) {
        if (wid[n] != 0) {
            if (v)
                for (int k = 0; k < 3; ++k) v[k * N + n] = 0.0;
            continue;
        }
        double fl[19];
        for (int a = 0; a < L.q; ++a) fl[a] = f[a * N + n];
        macro_t_r m;
        macro_r(c, &L, fl, c->g, &m);
        double dd = 0.0, vv = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double r = vref ? vref[k * N + n] : 0.0;
            dd += (m.v[k] - r) * (m.v[k] - r);
            vv += m.v[k] * m.v[k];
            if (v) v[k * N + n] = m.v[k];
        }
        out[0] += sqrt(dd);
        out[1] += sqrt(vv);
    }
    out[2] = out[1] > 0.0 ? out[0] / out[1] : 0.0;
}

/* forward run for the drag functional; stores f(t) for t < T if hist != NULL */
static double drag_forward(const orc_cfg* c, const lat_t* L, const unsigned char* wid,
                           const double* f0, int T, int wall, const double* d, double* hist)
{
    const long N = nnodes(c);
    const int Q = L->q;
    double* f = (double*)malloc(sizeof(double) * N * Q);
    double* frel = (double*)malloc(sizeof(double) * N * Q);
    double* fnew = (double*)malloc(sizeof(double) * N * Q);
    memcpy(f, f0, sizeof(double) * N * Q);
    double J = 0.0;
    for (int t = 0; t < T; ++t) {
        if (hist) memcpy(hist + (size_t)t * N * Q, f, sizeof(double) * N * Q);
        step_work(c, L, wid, f, frel, fnew, NULL);
        double F[3];
        orc_wall_force(c, wid, frel, f, wall, 0, F);
        J += (d[0] * F[0] + d[1] * F[1] + d[2] * F[2]) / T;
    }
    free(f);
    free(frel);
    free(fnew);
    return J;
}

double orc_drag_average(const orc_cfg* c, const unsigned char* wid, const double* f0, int T,
                        int wall, const double* d)
{
    lat_t L;
    get_lat(c->q, &L);
    return drag_forward(c, &L, wid, f0, T, wall, d, NULL);
}

int orc_adjoint_drag(const orc_cfg* c, const unsigned char* wid, const double* f0, int T,
                     int wall, const double* d, double* J, double* grad)
{
    lat_t L;
    if (get_lat(c->q, &L)) return -1;
    if (c->phi) return -2;        /* the transpose below is that of halfway bounce-back */
    const long N = nnodes(c);
    const int Q = L.q;
    const double cc = c->dx / c->dt, s = cell_volume(c, &L) / c->dt, h = 1e-30;
    double* hist = (double*)malloc(sizeof(double) * (size_t)T * N * Q);
    double* phi = (double*)calloc((size_t)N * Q, sizeof(double));   /* dJ/df(t+1) */
    double* psi = (double*)calloc((size_t)N * Q, sizeof(double));   /* dJ/dfrel(t) */
    if (!hist || !phi || !psi) { free(hist); free(phi); free(psi); return -2; }
    *J = drag_forward(c, &L, wid, f0, T, wall, d, hist);
    for (int k = 0; k < 6; ++k) grad[k] = 0.0;

    for (int t = T - 1; t >= 0; --t) {
        const double* ft = hist + (size_t)t * N * Q;
        /* transpose of propagation: frel_a(x) went to f_a(x + e_a), or to
         * f_opp(a)(x) through a wall; plus the drag's own dependence on
         * frel(t) and on u_w through the Ladd term */
        for (int z = 0; z < c->nz; ++z)
            for (int y = 0; y < c->ny; ++y)
                for (int x = 0; x < c->nx; ++x) {
                    long n = ((long)z * c->ny + y) * c->nx + x;
                    if (wid[n] != 0) continue;
                    for (int a = 0; a < Q; ++a) {
                        int lw = 0;
                        long dn = link_dest(c, &L, wid, x, y, z, a, &lw);
                        if (dn >= 0) {
                            psi[a * N + n] = phi[a * N + dn];
                            continue;
                        }
                        psi[a * N + n] = phi[L.opp[a] * N + n];
                        if (lw != wall) continue;
                        double de = 0;
                        for (int k = 0; k < 3; ++k) de += d[k] * cc * L.e[a][k];
                        /* F per link = s e_a (2 frel_a - ladd_a(u_w)) */
                        psi[a * N + n] += 2.0 * s * de / T;
                        for (int k = 0; k < 3; ++k) {
                            double dladd = 6.0 * L.w[a] * c->rho0 * (cc * L.e[a][k]) / (cc * cc);
                            grad[3 + k] += -dladd * phi[L.opp[a] * N + n];   /* via f(t+1) */
                            grad[3 + k] += -s * de * dladd / T;              /* via F(t) */
                        }
                    }
                }
        /* transpose of the collision at each node: phi_t = (dC/df)^T psi,
         * and the body-force gradient (dC/dg)^T psi */
        for (long n = 0; n < N; ++n) {
            if (wid[n] != 0) {
                for (int a = 0; a < Q; ++a) phi[a * N + n] = 0.0;
                continue;
            }
            double complex fc[19], gc[3], out[19];
            for (int a = 0; a < Q; ++a) fc[a] = ft[a * N + n];
            for (int k = 0; k < 3; ++k) gc[k] = c->g[k];
            double col[19];
            for (int b = 0; b < Q; ++b) {
                fc[b] += I * h;
                collide_c(c, &L, fc, gc, out);
                fc[b] = ft[b * N + n];
                double acc = 0;
                for (int a = 0; a < Q; ++a) acc += psi[a * N + n] * cimag(out[a]) / h;
                col[b] = acc;
            }
            for (int k = 0; k < L.d; ++k) {
                gc[k] += I * h;
                collide_c(c, &L, fc, gc, out);
                gc[k] = c->g[k];
                double acc = 0;
                for (int a = 0; a < Q; ++a) acc += psi[a * N + n] * cimag(out[a]) / h;
                grad[k] += acc;
            }
            for (int b = 0; b < Q; ++b) phi[b * N + n] = col[b];
        }
    }
    free(hist);
    free(phi);
    free(psi);
    return 0;
}
