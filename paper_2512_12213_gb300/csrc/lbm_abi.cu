// lbm_abi.cu -- host side of the C ABI declared in include/lbm.h: configuration
// checks, node classes and the boundary-link list, buffer binding, and the
// entry points that launch the kernels of lbm_kernels.cuh on the caller's
// stream.  No device memory is allocated here; every buffer is the caller's.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"
#include "lbm_staged.cuh"

using namespace lbm;

namespace {

thread_local std::string g_cfg_err;

int dims_of(const lbm_config* c) { return c->lattice == LBM_D2Q9 ? 2 : 3; }

long long nodes_of(const lbm_config* c) { return (long long)c->nx * c->ny * c->nz; }

int pitch_of(int nx) { return (nx + 63) / 64 * 64; }

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

size_t elem_of(int storage)
{
    switch (storage) {
    case LBM_STORE_F64: return 8;
    case LBM_STORE_F32: return 4;
    default: return 2;
    }
}

// the staged step serves 16-bit and FP32 storage with halfway walls and the
// node code of the imposed field (not walls off the half-grid, insulating
// walls or the induced field, whose state the staged kernel does not carry)
bool staged_applies(const lbm_config* c)
{
    return !c->curved && !c->insulating && !c->induced && c->storage != LBM_STORE_F64;
}

bool all_periodic(const lbm_config* c)
{
    return c->periodic[0] && c->periodic[1] && (c->lattice == LBM_D2Q9 || c->periodic[2]);
}


bool validate(const lbm_config* c, const uint8_t* wid, std::string& err)
{
    char buf[256];
    auto fail = [&](const char* m) { err = m; return false; };
    if (!c) return fail("config is NULL");
    if (c->lattice != LBM_D2Q9 && c->lattice != LBM_D3Q19) return fail("lattice must be 9 or 19");
    if (c->nx < 1 || c->ny < 1 || c->nz < 1) return fail("nx, ny, nz must be >= 1");
    if (c->lattice == LBM_D2Q9 && c->nz != 1) return fail("D2Q9 needs nz = 1");
    const long long np = (long long)pitch_of(c->nx) * c->ny * c->nz;
    if (np >= (1ll << 31)) return fail("domain too large (padded node count must be < 2^31)");
    if (!(c->dx > 0) || !(c->dt > 0)) return fail("dx and dt must be > 0");
    if (!(c->tau > 0.5)) return fail("tau must be > 1/2");
    if (!(c->rho0 > 0)) return fail("rho0 must be > 0");
    if (c->force_model < 0 || c->force_model > 4) return fail("force_model must be 0..4");
    if (c->storage < 0 || c->storage > 3) return fail("storage must be 0..3");
    if (c->n_walls < 0 || c->n_walls > LBM_MAX_WALLS) return fail("n_walls must be 0..16");
    for (int k = 0; k < 3; ++k)
        if (c->periodic[k] != 0 && c->periodic[k] != 1) return fail("periodic[] must be 0 or 1");
    for (int k = 0; k < dims_of(c); ++k)
        if (!c->periodic[k])
            for (int s = 0; s < 2; ++s) {
                const int w = c->face_wall[2 * k + s];
                if (w < 1 || w > c->n_walls) {
                    snprintf(buf, sizeof buf, "face_wall[%d] = %d is not a wall id in 1..n_walls", 2 * k + s, w);
                    err = buf;
                    return false;
                }
            }
    if (c->lorentz && !(c->sigma_e >= 0)) return fail("sigma_e must be >= 0");
    if (c->maxwell && !(c->mu > 0)) return fail("mu must be > 0");
    // Eq. (10) without -c^2 B^2/6 has zero mass and the Maxwell stress as its
    // second moment in 2-D only for a field in the simulated plane
    if (c->maxwell && c->lattice == LBM_D2Q9 && c->B[2] != 0.0)
        return fail("the 2-D Maxwell equilibrium needs an in-plane field (B[2] = 0)");
    if (c->les && !(c->cs >= 0)) return fail("cs must be >= 0");
    if (c->rounding != LBM_ROUND_NEAREST && c->rounding != LBM_ROUND_STOCHASTIC)
        return fail("rounding must be LBM_ROUND_NEAREST or LBM_ROUND_STOCHASTIC");
    if (c->rounding == LBM_ROUND_STOCHASTIC && c->storage != LBM_STORE_F16S && c->storage != LBM_STORE_BF16S)
        return fail("stochastic rounding applies to 16-bit storage only");
    if (c->insulating != 0 && c->insulating != 1) return fail("insulating must be 0 or 1");
    if (c->insulating && !c->lorentz) return fail("insulating walls need the Lorentz force (lorentz = 1)");
    if (c->curved != 0 && c->curved != 1) return fail("curved must be 0 or 1");
    if (c->stokes != 0 && c->stokes != 1) return fail("stokes must be 0 or 1");
    if (!(c->darcy >= 0.0) || !std::isfinite(c->darcy)) return fail("darcy must be finite and >= 0");
    if (c->induced != 0 && c->induced != 1) return fail("induced must be 0 or 1");
    if (c->induced) {
        if (!c->maxwell) return fail("the induced field acts through the Maxwell equilibrium (maxwell = 1)");
        if (c->lorentz || c->les || c->curved || c->insulating)
            return fail("the induced field needs lorentz = les = curved = insulating = 0");
        if (!(c->eta > 0.0) || !std::isfinite(c->eta)) return fail("eta must be finite and > 0");
        if (c->mag_conducting != 0 && c->mag_conducting != 1) return fail("mag_conducting must be 0 or 1");
    }
    if (c->step_kernel < LBM_STEP_AUTO || c->step_kernel > LBM_STEP_STAGED) return fail("step_kernel must be 0..2");
    if (c->step_kernel == LBM_STEP_STAGED && !staged_applies(c))
        return fail("the staged step kernel needs FP32 or 16-bit storage and none of curved, insulating, induced");
    if (!wid) return fail("wall_id is NULL");
    const long long N = nodes_of(c);
    for (long long n = 0; n < N; ++n)
        if (wid[n] > c->n_walls) {
            snprintf(buf, sizeof buf, "wall_id[%lld] = %d exceeds n_walls", n, (int)wid[n]);
            err = buf;
            return false;
        }
    return true;
}

// link leaving node (x,y,z) along E: fluid destination -> true; wall -> false + id.
// Periodic axes wrap; the first closed axis crossed (x, y, z) names the wall.
template <int Q>
bool host_push_dest(const lbm_config* c, const uint8_t* wid, int x, int y, int z, int a, long long& dn, int& wall)
{
    int p[3] = {x + EX<Q>(a), y + EY<Q>(a), z + EZ<Q>(a)};
    const int n[3] = {c->nx, c->ny, c->nz};
    const int per[3] = {c->periodic[0], c->periodic[1], Q == 9 ? 1 : c->periodic[2]};
    for (int k = 0; k < 3; ++k) {
        if (p[k] >= 0 && p[k] < n[k]) continue;
        if (per[k]) {
            p[k] = (p[k] + n[k]) % n[k];
        } else {
            wall = c->face_wall[2 * k + (p[k] < 0 ? 0 : 1)];
            return false;
        }
    }
    dn = ((long long)p[2] * c->ny + p[1]) * c->nx + p[0];
    if (wid[dn]) {
        wall = wid[dn];
        return false;
    }
    return true;
}

template <int Q>
void build_geometry(const lbm_config* c, const uint8_t* wid, int nxp, std::vector<uint8_t>& cls,
                    std::vector<Link>* links)
{
    cls.assign((size_t)nxp * c->ny * c->nz, NC_PAD);
    std::vector<Link> raw;
    const long long N = (long long)c->nx * c->ny * c->nz;
    bool any_solid = false;
    for (long long n = 0; n < N && !any_solid; ++n) any_solid = wid[n] != 0;
    const int per[3] = {c->periodic[0], c->periodic[1], Q == 9 ? 1 : c->periodic[2]};
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                const long long n = ((long long)z * c->ny + y) * c->nx + x;
                const long long np = ((long long)z * c->ny + y) * nxp + x;
                if (wid[n]) {
                    cls[np] = nc_make_solid(wid[n]);
                    continue;
                }
                // all-fluid geometry: only nodes on a closed face have wall links
                if (!any_solid && (per[0] || (x > 0 && x < c->nx - 1)) && (per[1] || (y > 0 && y < c->ny - 1)) &&
                    (per[2] || (z > 0 && z < c->nz - 1))) {
                    cls[np] = NC_BULK;
                    continue;
                }
                bool face = false, solid = false;
                for (int a = 1; a < Q; ++a) {
                    long long dn;
                    int wall;
                    if (!host_push_dest<Q>(c, wid, x, y, z, a, dn, wall)) {
                        // a wall link that stays inside the box hits a solid node
                        const int px = x + EX<Q>(a), py = y + EY<Q>(a), pz = z + EZ<Q>(a);
                        const bool in_box = (px >= 0 && px < c->nx) && (py >= 0 && py < c->ny) &&
                                            (pz >= 0 && pz < c->nz);
                        const bool wraps = (c->periodic[0] || (px >= 0 && px < c->nx)) &&
                                           (c->periodic[1] || (py >= 0 && py < c->ny)) &&
                                           ((Q == 9 || c->periodic[2]) || (pz >= 0 && pz < c->nz));
                        if (in_box || wraps) solid = true;
                        else face = true;
                        if (links) raw.push_back(Link{(uint32_t)np, (uint16_t)a, (uint16_t)wall});
                    }
                }
                cls[np] = solid ? NC_BOUND : (face ? NC_FACE : NC_BULK);
            }
    if (links) {
        links->clear();
        links->reserve(raw.size());
        for (int w = 0; w <= LBM_MAX_WALLS; ++w)
            for (const Link& L : raw)
                if (L.wall == w) links->push_back(L);
    }
}

// the 4-node chunks of the padded layout that hold a node other than a bulk
// fluid node or a node whose only wall links cross a closed box face (a
// solid neighbour, a solid node, padding): the first node of each, in order.
// The staged step leaves them to its boundary warps.
std::vector<uint32_t> special_chunks(const std::vector<uint8_t>& cls)
{
    std::vector<uint32_t> out;
    auto plain = [](uint8_t c) { return c == NC_BULK || c == NC_FACE; };
    for (size_t i = 0; i + 3 < cls.size(); i += 4)
        if (!plain(cls[i]) || !plain(cls[i + 1]) || !plain(cls[i + 2]) || !plain(cls[i + 3]))
            out.push_back((uint32_t)i);
    return out;
}

void count_links(const lbm_config* c, const uint8_t* wid, long long* per_wall /* MAX+1 */, long long* n_special)
{
    std::fill(per_wall, per_wall + LBM_MAX_WALLS + 1, 0);
    std::vector<uint8_t> cls;
    std::vector<Link> links;
    if (c->lattice == 9) build_geometry<9>(c, wid, pitch_of(c->nx), cls, &links);
    else build_geometry<19>(c, wid, pitch_of(c->nx), cls, &links);
    for (const Link& L : links) per_wall[L.wall]++;
    *n_special = (long long)special_chunks(cls).size();
}

// threads of the register-tiled step kernel: one per vector chunk
long long step_threads_of(const lbm_config* c)
{
    const int V = (c->storage == LBM_STORE_F64) ? 2 : 4;
    return (long long)(pitch_of(c->nx) / V) * c->ny * c->nz;
}

// insulating walls: one velocity-sum row per warp of the step grid (blocks of
// 128 threads; the warps past the last chunk write zero rows)
long long ins_rows_of(const lbm_config* c)
{
    return (step_threads_of(c) + 127) / 128 * 4;
}

// contexts that may run the staged step keep the list of special chunks in
// the node buffer, after the class bytes
bool keeps_special_list(const lbm_config* c)
{
    return c->step_kernel != LBM_STEP_REGISTER && staged_applies(c);
}

void sizes_of(const lbm_config* c, long long n_links, long long n_special, size_t s[LBM_NUM_BUFFERS])
{
    const long long sq = (long long)pitch_of(c->nx) * c->ny * c->nz;
    const long long N = nodes_of(c);
    s[LBM_BUF_POP_A] = s[LBM_BUF_POP_B] = round256((size_t)c->lattice * sq * elem_of(c->storage));
    s[LBM_BUF_NODE] = round256((size_t)sq) + (keeps_special_list(c) ? round256((size_t)n_special * 4) : 0);
    s[LBM_BUF_LINKS] = n_links ? round256((size_t)n_links * sizeof(Link)) : 0;
    s[LBM_BUF_SCRATCH] = round256(SCRATCH_DOUBLES * sizeof(double));
    if (c->insulating)
        s[LBM_BUF_SCRATCH] = round256((SCRATCH_INS_ROWS + 3 * (size_t)ins_rows_of(c)) * sizeof(double));
    s[LBM_BUF_STAGE] = round256((size_t)(c->lattice + 4) * N * sizeof(double));
    s[LBM_BUF_PHI] = c->curved ? round256((size_t)sq * sizeof(float)) : 0;
    // induced field: 3 components x (5 or 7) directions per padded node, compute precision
    const size_t mag = c->induced ? round256((size_t)3 * (c->lattice == 9 ? 5 : 7) * sq *
                                             (c->storage == LBM_STORE_F64 ? 8 : 4))
                                  : 0;
    s[LBM_BUF_MAG_A] = s[LBM_BUF_MAG_B] = mag;
}

// wax = 3 w_axis om and om1j = 1 - K wax of the uniform relaxation rate
// (K = 1/(3 w_axis): 6 in D3Q19, 3 in D2Q9), with om1j exact in the target
// format: the FP32 node-pair code relaxes the odd part with them, so the
// momentum of om1j d + W E.j is j exactly (momentum_coefs).  For om outside
// (0.75, 2) wax goes to a coarser grid until 1 - K wax is a float.
template <typename R> void momentum_coefs_host(const KP<double>& s, KP<R>& d)
{
    const double K = s.kmom;
    R wax = (R)(s.om0 / K);
    double o1 = 1.0 - K * (double)wax;
    for (int it = 0; it < 4 && (double)(R)o1 != o1; ++it) {
        // a grid step g of |o1|'s binade in R, and wax a multiple of g / 2^k
        // with K = 3 * 2^k, so that K wax is a multiple of g
        int e = 0;
        std::frexp(o1, &e);
        const double g = std::ldexp(1.0, e - (std::numeric_limits<R>::digits));
        const double step = g * 3.0 / K;
        wax = (R)(std::round((double)wax / step) * step);
        o1 = 1.0 - K * (double)wax;
    }
    d.wax = wax;
    d.om1j = (R)o1;
}

template <typename R> void cast_kp(const KP<double>& s, KP<R>& d)
{
    d.rho0 = (R)s.rho0; d.tau0 = (R)s.tau0; d.om0 = (R)s.om0;
    d.kmom = s.kmom;
    momentum_coefs_host(s, d);
    for (int k = 0; k < 3; ++k) {
        d.AG[k] = (R)s.AG[k]; d.AEB[k] = (R)s.AEB[k]; d.B[k] = (R)s.B[k];
    }
    d.model = s.model; d.lorentz = s.lorentz; d.kappa = (R)s.kappa; d.B2 = (R)s.B2; d.Bp2 = (R)s.Bp2;
    d.maxwell = s.maxwell;
    for (int a = 0; a < 19; ++a) d.mx[a] = (R)s.mx[a];
    for (int k = 0; k < 6; ++k) d.Lh[k] = (R)s.Lh[k];
    d.les = s.les; d.lesc = (R)s.lesc; d.face_ladd = s.face_ladd;
    d.stokes = s.stokes; d.darcy_h = (R)s.darcy_h;
    d.induced = s.induced; d.mag_cond = s.mag_cond; d.mxk = (R)s.mxk; d.om_m = (R)s.om_m;
    for (int k = 0; k < 3; ++k) d.Bext[k] = (R)s.Bext[k];
    d.mag = nullptr;
    for (int w = 0; w <= MAXW; ++w)
        for (int k = 0; k < 3; ++k) d.LW[w][k] = (R)s.LW[w][k];
    d.c = (R)s.c; d.dt = (R)s.dt; d.svol = (R)s.svol;
    for (int k = 0; k < 3; ++k) {
        d.ueq_c[k] = (R)s.ueq_c[k];
        d.uf_c[k] = (R)s.uf_c[k];
    }
    d.uf_u = (R)s.uf_u;
    d.Cf = (R)s.Cf;
    for (int a = 0; a < 19; ++a) {
        d.pe[a] = (R)s.pe[a];
        d.peq[a] = (R)s.peq[a];
        d.pf[a] = (R)s.pf[a];
    }
}

// constants of the node-pair path: the force model of Sec. 2 as u^eq = u +
// ueq_c, u^F = uf_u u + uf_c and C = Cf for a uniform A, and E_a . A
template <int Q> void pair_consts(KP<double>& p)
{
    const double h = 0.5;
    for (int k = 0; k < 3; ++k) {
        p.ueq_c[k] = (p.model == MODEL_E) ? h * p.AG[k] : 0.0;
        switch (p.model) {
        case MODEL_A: p.uf_c[k] = 0.0; break;
        case MODEL_B: p.uf_c[k] = 0.0; break;
        case MODEL_C: p.uf_c[k] = h * p.tau0 * p.AG[k]; break;
        default: p.uf_c[k] = h * p.AG[k]; break;
        }
    }
    p.uf_u = (p.model == MODEL_A) ? 0.0 : 1.0;
    p.Cf = (p.model == MODEL_E) ? 1.0 - h * p.om0 : 1.0;
    for (int a = 0; a < 19; ++a) {
        p.pe[a] = (a < Q) ? EX<Q>(a) * p.AG[0] + EY<Q>(a) * p.AG[1] + EZ<Q>(a) * p.AG[2] : 0.0;
        p.peq[a] = (a < Q) ? EX<Q>(a) * p.ueq_c[0] + EY<Q>(a) * p.ueq_c[1] + EZ<Q>(a) * p.ueq_c[2] : 0.0;
        p.pf[a] = (a < Q) ? EX<Q>(a) * p.uf_c[0] + EY<Q>(a) * p.uf_c[1] + EZ<Q>(a) * p.uf_c[2] : 0.0;
    }
}

template <int Q> void maxwell_table(const lbm_config* c, double* mx)
{
    const double cc = c->dx / c->dt;
    const double B2 = c->B[0] * c->B[0] + c->B[1] * c->B[1] + c->B[2] * c->B[2];
    for (int a = 0; a < 19; ++a) mx[a] = 0.0;
    for (int a = 0; a < Q; ++a) {
        const double E2 = SPEED2<Q>(a);
        const double EB = EX<Q>(a) * c->B[0] + EY<Q>(a) * c->B[1] + EZ<Q>(a) * c->B[2];
        double m = 0.5 * B2 * E2 - EB * EB;
        if (Q == 19) m -= B2 / 6.0;
        mx[a] = 9.0 * WD<Q>(a) / (2.0 * cc * cc * c->mu) * m;
    }
}

// insulating walls: the kernels read the force coefficient of the current
// field from the scratch block and the step writes its velocity rows there
void bind_insulating(Ctx& x)
{
    if (!x.insulating || !x.scratch) return;
    double* blk = x.scratch + SCRATCH_INS_OFF;
    x.kpd.aeb_dev = blk + INS_AEB_D;
    x.kpf.aeb_dev = reinterpret_cast<const float*>(blk + INS_AEB_F);
    x.kps.aeb_dev = reinterpret_cast<const float*>(blk + INS_AEB_S);
    x.kpd.ins_rows = x.kpf.ins_rows = x.kps.ins_rows = x.scratch + SCRATCH_INS_ROWS;
}

void fill_params(Ctx& x)
{
    const lbm_config* c = &x.cfg;
    KP<double>& p = x.kpd;
    memset(&p, 0, sizeof p);
    const double cc = c->dx / c->dt;
    const int D = dims_of(c);
    p.rho0 = c->rho0;
    p.tau0 = c->tau;
    p.om0 = 1.0 / c->tau;
    p.kmom = (c->lattice == LBM_D3Q19) ? 6 : 3;
    p.wax = p.om0 / p.kmom;
    p.om1j = 1.0 - p.om0;
    for (int k = 0; k < 3; ++k) p.AG[k] = (k < D) ? c->dt * c->g[k] / cc : 0.0;
    p.model = c->force_model;
    p.lorentz = c->lorentz;
    const double ExB[3] = {c->E[1] * c->B[2] - c->E[2] * c->B[1], c->E[2] * c->B[0] - c->E[0] * c->B[2],
                           c->E[0] * c->B[1] - c->E[1] * c->B[0]};
    for (int k = 0; k < 3; ++k) {
        p.AEB[k] = c->lorentz ? c->dt * c->sigma_e * ExB[k] / cc : 0.0;
        p.B[k] = c->B[k];
    }
    p.kappa = c->lorentz ? c->dt * c->sigma_e : 0.0;
    p.B2 = c->B[0] * c->B[0] + c->B[1] * c->B[1] + c->B[2] * c->B[2];
    p.Bp2 = c->B[0] * c->B[0] + c->B[1] * c->B[1] + (D == 3 ? c->B[2] * c->B[2] : 0.0);
    p.maxwell = c->maxwell;
    if (c->maxwell) {
        if (c->lattice == 9) maxwell_table<9>(c, p.mx);
        else maxwell_table<19>(c, p.mx);
        const int ci[6] = {0, 1, 2, 0, 0, 1}, cj[6] = {0, 1, 2, 1, 2, 2};
        for (int k = 0; k < 6; ++k)
            p.Lh[k] = ((ci[k] == cj[k] ? 0.5 * p.B2 : 0.0) - c->B[ci[k]] * c->B[cj[k]]) / (c->mu * cc * cc);
    }
    p.les = c->les;
    p.lesc = 18.0 * c->cs * c->cs;
    p.stokes = c->stokes;
    p.darcy_h = 0.5 * c->dt * c->darcy;
    p.induced = c->induced;
    if (c->induced) {
        // D2Q5 theta = 1/3, D3Q7 theta = 1/4: tau_m = 1/2 + eta / (theta c^2 dt)
        const double theta = (c->lattice == 9) ? 1.0 / 3.0 : 0.25;
        p.mag_cond = c->mag_conducting;
        p.mxk = 9.0 / (2.0 * cc * cc * c->mu);
        p.om_m = 1.0 / (0.5 + c->eta / (theta * cc * cc * c->dt));
        for (int k = 0; k < 3; ++k) p.Bext[k] = c->B[k];
    }
    p.face_ladd = 0;
    for (int k = 0; k < D; ++k)
        if (!c->periodic[k])
            for (int sd = 0; sd < 2; ++sd) {
                const int w = c->face_wall[2 * k + sd];
                if (w >= 1 && w <= c->n_walls)
                    for (int j = 0; j < D; ++j)
                        if (c->wall_u[w - 1][j] != 0.0) p.face_ladd = 1;
            }
    for (int w = 1; w <= c->n_walls; ++w)
        for (int k = 0; k < 3; ++k) p.LW[w][k] = (k < D) ? 6.0 * c->rho0 * c->wall_u[w - 1][k] / cc : 0.0;
    p.c = cc;
    p.dt = c->dt;
    p.svol = (D == 3 ? c->dx * c->dx * c->dx : c->dx * c->dx) / c->dt;
    if (c->lattice == 9) pair_consts<9>(p);
    else pair_consts<19>(p);
    cast_kp(p, x.kpf);
    // storage units: every term that adds to or is compared with a stored
    // deviation scales with it (rho0 enters rho = rho0 + sum d); velocities,
    // relaxation times and the body-force increment do not
    const double s = (c->storage == LBM_STORE_F16S) ? 4096.0 : 1.0;
    KP<double> q = p;
    q.rho0 *= s;
    q.kappa *= s;
    for (int k = 0; k < 3; ++k) q.AEB[k] *= s;
    for (int a = 0; a < 19; ++a) q.mx[a] *= s;
    q.mxk *= s;
    for (int k = 0; k < 6; ++k) q.Lh[k] *= s;
    for (int w = 0; w <= MAXW; ++w)
        for (int k = 0; k < 3; ++k) q.LW[w][k] *= s;
    cast_kp(q, x.kps);
    bind_insulating(x);
}

// shape of the staged step: tiles of R rows such that each direction's copy
// moves at least 2 KB (R nxp = 1024 nodes for 16-bit storage, 512 for FP32:
// a bulk copy costs the copy engine a fixed time, so small copies starve the
// pipeline), and as many stages (an even count, 4..8) as the shared memory
// holds; stage_R = 0
// where the kernel does not apply, was not asked for, or fewer than 4 stages
// fit (rows of more than ~1,100 16-bit or ~550 FP32 nodes): the
// register-tiled kernel serves those contexts
void choose_stage(Ctx& x)
{
    x.stage_R = 0;
    x.stage_n = 0;
    x.stage_tiles = 0;
    x.stage_smem = 0;
    x.stage_ready = false;
    if (!keeps_special_list(&x.cfg)) return;
    // automatic choice: the boundary warps keep pace while at most 2% of the
    // chunks are special (a sphere or a few bodies in a periodic box); boxes
    // full of small solids go to the register-tiled kernel
    if (x.cfg.step_kernel == LBM_STEP_AUTO && x.n_special * 50 > x.geo.sq / 4) return;
    // ... and 16-bit storage: with FP32 the register-tiled kernel already
    // keeps enough bytes in flight (measured on the sphere box: 0.84 of HBM
    // against 0.81 staged), with 16-bit it does not (0.52 against 0.80)
    if (x.cfg.step_kernel == LBM_STEP_AUTO && x.elem != 2) return;
    // (with 16-bit storage the staged kernel also wins with closed faces and
    // the EXT node code: LES cavity 256^3, binary16 with stochastic rounding,
    // 28.5k against 23.7k MLUPS; with FP32 it loses there too, 20.2k against
    // 26.7k)
    const size_t Q = x.cfg.lattice, nxp = x.geo.nxp;
    const size_t row_bytes = nxp * x.elem;
    const int R = (int)std::max<size_t>(1, std::min<size_t>((STG_COPY_BYTES + row_bytes - 1) / row_bytes,
                                                            (size_t)x.cfg.ny));
    const size_t stage = stg_stage_bytes((int)Q, R, (int)nxp, (int)x.elem);
    const size_t budget = (size_t)x.smem_optin - 1024;
    // an even count: each consumer group owns every other stage
    const int n = (int)std::min<size_t>(8, budget / (stage + 2 * sizeof(uint64_t))) & ~1;
    if (n < 4) return;
    const long long tiles = (long long)((x.cfg.ny + R - 1) / R) * x.cfg.nz;
    // automatic choice with closed faces or the EXT node code (longer tiles):
    // at least 16 tiles per block, else the tail of the persistent grid costs
    // more than the pipeline gains (LES cavity 128^3: 13 tiles per block,
    // 16.0k staged against 19.6k MLUPS register-tiled)
    const bool long_tiles = !all_periodic(&x.cfg) || x.ext;
    if (x.cfg.step_kernel == LBM_STEP_AUTO && long_tiles && tiles < 16ll * x.sm_count) return;
    x.stage_R = R;
    x.stage_n = n;
    x.stage_tiles = tiles;
    x.stage_smem = n * stage + 2 * n * sizeof(uint64_t);
}

// signed wall distance in the padded layout: the given canonical values, or
// +-1/2 (halfway bounce-back) when phi is null; padding gets 0
std::vector<float> padded_distance(const Ctx& x, const float* phi)
{
    std::vector<float> out((size_t)x.geo.sq, 0.0f);
    for (int z = 0; z < x.cfg.nz; ++z)
        for (int y = 0; y < x.cfg.ny; ++y)
            for (int xx = 0; xx < x.cfg.nx; ++xx) {
                const size_t n = ((size_t)z * x.cfg.ny + y) * x.cfg.nx + xx;
                const size_t pn = ((size_t)z * x.cfg.ny + y) * x.geo.nxp + xx;
                out[pn] = phi ? phi[n] : (x.host_wid[n] ? -0.5f : 0.5f);
            }
    return out;
}

struct DeviceGuard {
    int old = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&old) != cudaSuccess) { ok = false; return; }
        if (old != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int now = -1;
        if (old >= 0 && cudaGetDevice(&now) == cudaSuccess && now != old) cudaSetDevice(old);
    }
};

// seed of the stochastic rounding of step t (the same for lbm_step at time t
// and lbm_step_from(..., t, ...))
uint32_t step_seed(const Ctx& x, int64_t t)
{
    return hash32(x.cfg.seed ^ hash32((uint32_t)t ^ (uint32_t)((uint64_t)t >> 32) * 0x9e3779b9u));
}

lbm_status cuda_fail(Ctx& x, cudaError_t e, const char* what)
{
    x.err = std::string(what) + ": " + cudaGetErrorString(e);
    return LBM_ERR_CUDA;
}

lbm_status arg_fail(Ctx& x, const char* what)
{
    x.err = what;
    return LBM_ERR_ARG;
}

long long nodes(const Ctx& x) { return (long long)x.cfg.nx * x.cfg.ny * x.cfg.nz; }
size_t pop_bytes(const Ctx& x) { return (size_t)x.cfg.lattice * x.geo.sq * x.elem; }

#define CK(expr, what)                                        \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return cuda_fail(x, e_, what); \
    } while (0)

#define GUARD(x)                                                                 \
    DeviceGuard guard_((x).device);                                              \
    if (!guard_.ok) return cuda_fail((x), cudaErrorInvalidDevice, "set device");

// reduce nb partial rows of width W into out (device or host)
// the mode was checked by out_mode_ok before any launch
lbm_status finish_reduce(Ctx& x, const double* partials, int nb, int W, double* out, int mode, double weight,
                         bool accumulate, cudaStream_t st)
{
    if (mode == LBM_OUT_DEVICE) {
        CK(launch_reduce_rows(partials, nb, W, out, weight, accumulate ? 1 : 0, st), "reduce");
        return LBM_OK;
    }
    double* slot = x.scratch + SCRATCH_OUT_OFF;
    CK(launch_reduce_rows(partials, nb, W, slot, weight, 0, st), "reduce");
    if (mode == LBM_OUT_HOST_ASYNC) {
        CK(cudaMemcpyAsync(out, slot, sizeof(double) * W, cudaMemcpyDeviceToHost, st), "copy result");
        return LBM_OK;
    }
    double tmp[8];
    CK(cudaMemcpyAsync(tmp, slot, sizeof(double) * W, cudaMemcpyDeviceToHost, st), "copy result");
    CK(cudaStreamSynchronize(st), "synchronize");
    bool finite = true;
    for (int k = 0; k < W; ++k) {
        out[k] = accumulate ? out[k] + tmp[k] : tmp[k];
        finite = finite && std::isfinite(tmp[k]);
    }
    if (!finite) {
        x.err = "the reduction is not finite (the state holds NaN or Inf values)";
        return LBM_ERR_NAN;
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_config_error(void) { return g_cfg_err.c_str(); }

lbm_status lbm_buffer_sizes(const lbm_config* cfg, const uint8_t* host_wall_id, size_t sizes[LBM_NUM_BUFFERS])
{
    if (!sizes) {
        g_cfg_err = "sizes is NULL";
        return LBM_ERR_ARG;
    }
    if (!validate(cfg, host_wall_id, g_cfg_err)) return LBM_ERR_ARG;
    long long per_wall[LBM_MAX_WALLS + 1], n_special = 0;
    count_links(cfg, host_wall_id, per_wall, &n_special);
    long long nl = 0;
    for (int w = 0; w <= LBM_MAX_WALLS; ++w) nl += per_wall[w];
    sizes_of(cfg, nl, n_special, sizes);
    return LBM_OK;
}

lbm_status lbm_create(const lbm_config* cfg, const uint8_t* host_wall_id, void* const buffers[LBM_NUM_BUFFERS],
                      const size_t sizes[LBM_NUM_BUFFERS], void* stream, lbm_ctx** out)
{
    if (!out || !buffers || !sizes) {
        g_cfg_err = "NULL argument";
        return LBM_ERR_ARG;
    }
    *out = nullptr;
    if (!validate(cfg, host_wall_id, g_cfg_err)) return LBM_ERR_ARG;
    lbm_ctx* h = new (std::nothrow) lbm_ctx();
    if (!h) return LBM_ERR_OOM;
    Ctx& x = h->c;
    x.cfg = *cfg;
    if (x.cfg.lattice == LBM_D2Q9) x.cfg.periodic[2] = 1;
    x.ext = (cfg->lorentz || cfg->maxwell || cfg->les || cfg->stokes || cfg->darcy > 0.0 || cfg->induced) ? 1 : 0;
    // the FP32x2 LES pair code: 16-bit storage only (LES cavity 256^3 with
    // binary16 and stochastic rounding 26.4k -> 30.3k MLUPS, 512^3 27.8k ->
    // 36.8k); with FP32 storage it measured slower than the EXT pair code
    // (22.1k register-tiled, 19.7k staged against 25.2k at 256^3)
    x.les_pair = (cfg->les && !cfg->lorentz && !cfg->maxwell && !cfg->stokes && !(cfg->darcy > 0.0) &&
                  !cfg->induced && !cfg->insulating && !cfg->curved &&
                  (cfg->storage == LBM_STORE_F16S || cfg->storage == LBM_STORE_BF16S)) ? 1 : 0;
    x.sr = (cfg->rounding == LBM_ROUND_STOCHASTIC) ? 1 : 0;
    x.insulating = cfg->insulating != 0;
    x.ins_rows = ins_rows_of(cfg);
    x.n_fluid = 0;
    for (long long n = 0; n < (long long)cfg->nx * cfg->ny * cfg->nz; ++n) x.n_fluid += host_wall_id[n] == 0;
    x.geo.nx = cfg->nx;
    x.geo.ny = cfg->ny;
    x.geo.nz = cfg->nz;
    x.geo.nxp = pitch_of(cfg->nx);
    x.geo.sq = (long long)x.geo.nxp * cfg->ny * cfg->nz;
    for (int k = 0; k < 3; ++k) x.geo.periodic[k] = x.cfg.periodic[k];
    for (int k = 0; k < 6; ++k) x.geo.face_wall[k] = cfg->face_wall[k];
    x.elem = elem_of(cfg->storage);
    x.relem = cfg->storage == LBM_STORE_F64 ? 8 : 4;
    switch (cfg->storage) {
    case LBM_STORE_F64: x.ops = &dispatch_f64(); break;
    case LBM_STORE_F32: x.ops = &dispatch_f32(); break;
    case LBM_STORE_F16S: x.ops = &dispatch_f16(); break;
    default: x.ops = &dispatch_bf16(); break;
    }
    fill_params(x);

    std::vector<uint8_t> cls;
    std::vector<Link> links;
    if (cfg->lattice == 9) build_geometry<9>(&x.cfg, host_wall_id, x.geo.nxp, cls, &links);
    else build_geometry<19>(&x.cfg, host_wall_id, x.geo.nxp, cls, &links);
    x.n_links = (long long)links.size();
    for (int w = 0; w <= LBM_MAX_WALLS + 1; ++w) x.wall_begin[w] = 0;
    {
        long long pos = 0;
        for (int w = 0; w <= LBM_MAX_WALLS; ++w) {
            x.wall_begin[w] = pos;
            while (pos < x.n_links && links[pos].wall == w) ++pos;
        }
        x.wall_begin[LBM_MAX_WALLS + 1] = pos;
    }

    const std::vector<uint32_t> special = special_chunks(cls);
    x.n_special = (long long)special.size();
    size_t need[LBM_NUM_BUFFERS];
    sizes_of(&x.cfg, x.n_links, x.n_special, need);
    for (int b = 0; b < LBM_NUM_BUFFERS; ++b) {
        const bool optional = (b == LBM_BUF_STAGE) || ((b == LBM_BUF_LINKS || b == LBM_BUF_PHI || b == LBM_BUF_MAG_A ||
                                                         b == LBM_BUF_MAG_B) &&
                                                        need[b] == 0);
        if (!buffers[b]) {
            if (optional) continue;
            g_cfg_err = "required buffer " + std::to_string(b) + " is NULL";
            delete h;
            return LBM_ERR_ARG;
        }
        if (((uintptr_t)buffers[b]) % 256 != 0) {
            g_cfg_err = "buffer " + std::to_string(b) + " is not 256-byte aligned";
            delete h;
            return LBM_ERR_ARG;
        }
        if (sizes[b] < need[b]) {
            g_cfg_err = "buffer " + std::to_string(b) + " is smaller than required (" + std::to_string(sizes[b]) +
                        " < " + std::to_string(need[b]) + ")";
            delete h;
            return LBM_ERR_ARG;
        }
    }
    x.pop[0] = buffers[LBM_BUF_POP_A];
    x.pop[1] = buffers[LBM_BUF_POP_B];
    x.cur = 0;
    x.mag[0] = x.cfg.induced ? buffers[LBM_BUF_MAG_A] : nullptr;
    x.mag[1] = x.cfg.induced ? buffers[LBM_BUF_MAG_B] : nullptr;
    x.cls = (uint8_t*)buffers[LBM_BUF_NODE];
    x.special = keeps_special_list(&x.cfg)
                    ? reinterpret_cast<const uint32_t*>(x.cls + round256((size_t)x.geo.sq))
                    : nullptr;
    x.links = (Link*)buffers[LBM_BUF_LINKS];
    x.scratch = (double*)buffers[LBM_BUF_SCRATCH];
    bind_insulating(x);
    x.stage = buffers[LBM_BUF_STAGE];
    x.stage_bytes = x.stage ? sizes[LBM_BUF_STAGE] : 0;
    x.geo.phi = x.cfg.curved ? (const float*)buffers[LBM_BUF_PHI] : nullptr;
    if (x.cfg.curved) x.host_wid.assign(host_wall_id, host_wall_id + nodes_of(cfg));
    x.t = 0;
    x.prev_valid = false;
    if (cudaGetDevice(&x.device) != cudaSuccess) {
        g_cfg_err = "cudaGetDevice failed";
        delete h;
        return LBM_ERR_CUDA;
    }
    x.errflag = reinterpret_cast<unsigned*>(x.scratch + SCRATCH_FLAG_OFF);
    if (cudaDeviceGetAttribute(&x.sm_count, cudaDevAttrMultiProcessorCount, x.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&x.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, x.device) != cudaSuccess) {
        g_cfg_err = "cudaDeviceGetAttribute failed";
        delete h;
        return LBM_ERR_CUDA;
    }
    choose_stage(x);
    x.adj_blocks = 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(x.cls, cls.data(), cls.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && x.special && x.n_special)
        e = cudaMemcpyAsync((void*)x.special, special.data(), special.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                            st);
    if (e == cudaSuccess && x.n_links)
        e = cudaMemcpyAsync(x.links, links.data(), links.size() * sizeof(Link), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_zero(x.scratch, (long long)SCRATCH_DOUBLES, st);
    if (e == cudaSuccess && x.insulating) e = ins_reset(x, st);
    if (e == cudaSuccess && x.cfg.induced) e = x.ops->mag_init(x, st);
    std::vector<float> phi0;
    if (e == cudaSuccess && x.cfg.curved) {
        phi0 = padded_distance(x, nullptr);
        e = cudaMemcpyAsync((void*)x.geo.phi, phi0.data(), phi0.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    }
    // solid and padding entries of both population buffers start defined
    if (e == cudaSuccess) e = cudaMemsetAsync(x.pop[0], 0, need[LBM_BUF_POP_A], st);
    if (e == cudaSuccess) e = cudaMemsetAsync(x.pop[1], 0, need[LBM_BUF_POP_B], st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        g_cfg_err = std::string("upload: ") + cudaGetErrorString(e);
        delete h;
        return LBM_ERR_CUDA;
    }
    *out = h;
    return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx* ctx)
{
    delete ctx;
    return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->c.err.c_str() : "NULL context"; }

lbm_status lbm_link_count(const lbm_ctx* ctx, int wall, int64_t* count)
{
    if (!ctx || !count) return LBM_ERR_ARG;
    const Ctx& x = ctx->c;
    if (wall < 0) *count = x.n_links;
    else if (wall > LBM_MAX_WALLS) return LBM_ERR_ARG;
    else *count = x.wall_begin[wall + 1] - x.wall_begin[wall];
    return LBM_OK;
}

lbm_status lbm_set_body_force(lbm_ctx* ctx, const double g[3])
{
    if (!ctx || !g) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    for (int k = 0; k < 3; ++k) x.cfg.g[k] = g[k];
    fill_params(x);
    return LBM_OK;
}

lbm_status lbm_set_wall_velocity(lbm_ctx* ctx, int wall, const double u[3])
{
    if (!ctx || !u) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (wall < 1 || wall > x.cfg.n_walls) return arg_fail(x, "wall id out of range");
    for (int k = 0; k < 3; ++k) x.cfg.wall_u[wall - 1][k] = u[k];
    fill_params(x);
    return LBM_OK;
}

lbm_status lbm_init_equilibrium(lbm_ctx* ctx, const double* rho, const double* u, const double* xi, int on_host,
                                void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!rho || !u) return arg_fail(x, "rho and u are required");
    GUARD(x);
    cudaStream_t st = (cudaStream_t)stream;
    const long long N = nodes(x);
    const double *dr = rho, *du = u, *dxi = xi;
    if (on_host) {
        const size_t need = (size_t)(4 + (xi ? x.cfg.lattice : 0)) * N * sizeof(double);
        if (!x.stage || x.stage_bytes < need) return arg_fail(x, "host input needs the STAGE buffer");
        double* s = (double*)x.stage;
        CK(cudaMemcpyAsync(s, rho, N * sizeof(double), cudaMemcpyHostToDevice, st), "copy rho");
        CK(cudaMemcpyAsync(s + N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, st), "copy u");
        if (xi) CK(cudaMemcpyAsync(s + 4 * N, xi, (size_t)x.cfg.lattice * N * sizeof(double), cudaMemcpyHostToDevice, st),
                   "copy xi");
        dr = s;
        du = s + N;
        dxi = xi ? s + 4 * N : nullptr;
    }
    CK(x.ops->init_fields(x, dr, du, dxi, x.pop[x.cur], st), "init kernel");
    if (x.insulating) CK(ins_reset(x, st), "insulating-wall field");
    if (x.cfg.induced) CK(x.ops->mag_init(x, st), "induced-field reset");
    if (on_host) CK(cudaStreamSynchronize(st), "synchronize");
    x.t = 0;
    x.prev_valid = false;
    return LBM_OK;
}

lbm_status lbm_import_f(lbm_ctx* ctx, const void* src, int dtype, int on_host, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!src || (dtype != 0 && dtype != 1)) return arg_fail(x, "src must be non-NULL and dtype 0 or 1");
    GUARD(x);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)x.cfg.lattice * nodes(x) * (dtype == 0 ? 8 : 4);
    const void* dsrc = src;
    if (on_host) {
        if (!x.stage || x.stage_bytes < bytes) return arg_fail(x, "host input needs the STAGE buffer");
        CK(cudaMemcpyAsync(x.stage, src, bytes, cudaMemcpyHostToDevice, st), "copy f");
        dsrc = x.stage;
    }
    CK(x.ops->import_f(x, dsrc, dtype, x.pop[x.cur], st), "import kernel");
    if (x.insulating) CK(ins_reset(x, st), "insulating-wall field");
    if (x.cfg.induced) CK(x.ops->mag_init(x, st), "induced-field reset");
    if (on_host) CK(cudaStreamSynchronize(st), "synchronize");
    x.t = 0;
    x.prev_valid = false;
    return LBM_OK;
}

lbm_status lbm_export_f(lbm_ctx* ctx, void* dst, int dtype, int on_host, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!dst || (dtype != 0 && dtype != 1)) return arg_fail(x, "dst must be non-NULL and dtype 0 or 1");
    GUARD(x);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)x.cfg.lattice * nodes(x) * (dtype == 0 ? 8 : 4);
    void* ddst = dst;
    if (on_host) {
        if (!x.stage || x.stage_bytes < bytes) return arg_fail(x, "host output needs the STAGE buffer");
        ddst = x.stage;
    }
    CK(x.ops->export_f(x, x.pop[x.cur], ddst, dtype, st), "export kernel");
    if (on_host) {
        CK(cudaMemcpyAsync(dst, x.stage, bytes, cudaMemcpyDeviceToHost, st), "copy f");
        CK(cudaStreamSynchronize(st), "synchronize");
    }
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* ctx, int nsteps, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (nsteps < 0) return arg_fail(x, "nsteps must be >= 0");
    GUARD(x);
    cudaStream_t st = (cudaStream_t)stream;
    for (int s = 0; s < nsteps; ++s) {
        if (x.cfg.induced)
            CK(x.ops->mhd_step(x, x.pop[x.cur], x.pop[1 - x.cur], x.mag[x.cur], x.mag[1 - x.cur], step_seed(x, x.t), st),
               "coupled step kernel");
        else
            CK(x.ops->step(x, x.pop[x.cur], x.pop[1 - x.cur], step_seed(x, x.t), st), "step kernel");
        if (x.insulating) CK(ins_update(x, st), "insulating-wall field");
        x.cur = 1 - x.cur;
        x.t += 1;
        x.prev_valid = true;
    }
    return LBM_OK;
}

lbm_status lbm_step_from(lbm_ctx* ctx, const void* src, void* dst, int64_t t, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!src || !dst || src == dst) return arg_fail(x, "src and dst must be distinct non-NULL buffers");
    if (((uintptr_t)src) % 256 || ((uintptr_t)dst) % 256) return arg_fail(x, "buffers must be 256-byte aligned");
    if (t < 0) return arg_fail(x, "t must be >= 0");
    if (x.insulating || x.cfg.induced) {
        x.err = "lbm_step_from: with insulating walls or an induced field the field is state a population checkpoint "
                "does not hold";
        return LBM_ERR_UNSUPPORTED;
    }
    GUARD(x);
    CK(x.ops->step(x, src, dst, step_seed(x, t), (cudaStream_t)stream), "step kernel");
    return LBM_OK;
}

lbm_status lbm_save_state(lbm_ctx* ctx, void* dst, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!dst) return arg_fail(x, "dst is NULL");
    GUARD(x);
    CK(cudaMemcpyAsync(dst, x.pop[x.cur], pop_bytes(x), cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "save");
    return LBM_OK;
}

lbm_status lbm_load_state(lbm_ctx* ctx, const void* src, int64_t t, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!src || t < 0) return arg_fail(x, "src is NULL or t < 0");
    GUARD(x);
    CK(cudaMemcpyAsync(x.pop[x.cur], src, pop_bytes(x), cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "load");
    if (x.insulating) CK(ins_reset(x, (cudaStream_t)stream), "insulating-wall field");
    if (x.cfg.induced) CK(x.ops->mag_init(x, (cudaStream_t)stream), "induced-field reset");
    x.t = t;
    x.prev_valid = false;
    return LBM_OK;
}

lbm_status lbm_device_status(lbm_ctx* ctx, uint32_t* flags, int clear, void* stream)
{
    if (!ctx || !flags) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    GUARD(x);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(flags, x.errflag, sizeof(uint32_t), cudaMemcpyDeviceToHost, st), "copy flags");
    CK(cudaStreamSynchronize(st), "synchronize");
    if (clear) {
        CK(cudaMemsetAsync(x.errflag, 0, sizeof(uint32_t), st), "clear flags");
        // a step that stopped on a flag may have left the fused force's ticket set
        CK(cudaMemsetAsync(x.scratch + SCRATCH_TICKET_OFF, 0, sizeof(uint32_t), st), "clear ticket");
    }
    return LBM_OK;
}

lbm_status lbm_time(const lbm_ctx* ctx, int64_t* t)
{
    if (!ctx || !t) return LBM_ERR_ARG;
    *t = ctx->c.t;
    return LBM_OK;
}

lbm_status lbm_step_kernel(const lbm_ctx* ctx, int32_t* kind)
{
    if (!ctx || !kind) return LBM_ERR_ARG;
    *kind = ctx->c.stage_R > 0 ? LBM_STEP_STAGED : LBM_STEP_REGISTER;
    return LBM_OK;
}

lbm_status lbm_set_wall_distance(lbm_ctx* ctx, const float* phi_host, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!x.cfg.curved) return arg_fail(x, "lbm_set_wall_distance needs a context created with curved = 1");
    if (phi_host) {
        const long long N = nodes(x);
        for (long long n = 0; n < N; ++n) {
            const float v = phi_host[n];
            const bool ok = x.host_wid[n] ? (v < 0.0f) : (v > 0.0f);
            if (!ok || !std::isfinite(v)) {
                char buf[200];
                snprintf(buf, sizeof buf,
                         "wall distance %g at node %lld: it must be > 0 at fluid nodes and < 0 at solid nodes", (double)v,
                         n);
                return arg_fail(x, buf);
            }
        }
    }
    GUARD(x);
    const std::vector<float> ph = padded_distance(x, phi_host);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync((void*)x.geo.phi, ph.data(), ph.size() * sizeof(float), cudaMemcpyHostToDevice, st), "copy phi");
    CK(cudaStreamSynchronize(st), "synchronize");
    return LBM_OK;
}

lbm_status lbm_electric_field(lbm_ctx* ctx, double* E, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!E) return arg_fail(x, "E is NULL");
    if (!x.insulating) {
        for (int k = 0; k < 3; ++k) E[k] = x.cfg.E[k];
        return LBM_OK;
    }
    GUARD(x);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(E, x.scratch + SCRATCH_INS_OFF + INS_E, 3 * sizeof(double), cudaMemcpyDeviceToHost, st),
       "copy field");
    CK(cudaStreamSynchronize(st), "synchronize");
    return LBM_OK;
}

lbm_status lbm_export_field(lbm_ctx* ctx, double* B, int on_host, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!B) return arg_fail(x, "B is NULL");
    if (!x.cfg.induced) return arg_fail(x, "lbm_export_field needs a context created with induced = 1");
    GUARD(x);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = 3 * (size_t)nodes(x) * sizeof(double);
    double* dB = B;
    if (on_host) {
        if (!x.stage || x.stage_bytes < bytes) return arg_fail(x, "host output needs the STAGE buffer");
        dB = (double*)x.stage;
    }
    CK(x.ops->mag_field(x, dB, st), "field kernel");
    if (on_host) {
        CK(cudaMemcpyAsync(B, x.stage, bytes, cudaMemcpyDeviceToHost, st), "copy B");
        CK(cudaStreamSynchronize(st), "synchronize");
    }
    return LBM_OK;
}

lbm_status lbm_stress(lbm_ctx* ctx, int variant, void* sigma, void* S, void* rho, void* v, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (variant < LBM_S1 || variant > LBM_S4) return arg_fail(x, "variant must be 1..4");
    if (variant == LBM_S1 && x.cfg.stokes) {
        x.err = "stress variant S1 carries the artefact term of the full equilibrium; not with stokes = 1";
        return LBM_ERR_UNSUPPORTED;
    }
    if (variant >= LBM_S3 && x.cfg.induced) {
        x.err = "the half-step stress variants S3 / S4 are not defined with an induced field";
        return LBM_ERR_UNSUPPORTED;
    }
    if (variant >= LBM_S3 && (x.t < 1 || !x.prev_valid)) {
        x.err = "half-step stress needs at least one step since the last init/import/load";
        return LBM_ERR_STATE;
    }
    GUARD(x);
    CK(x.ops->stress(x, x.pop[x.cur], x.pop[1 - x.cur], variant, sigma, S, rho, v, (cudaStream_t)stream),
       "stress kernel");
    return LBM_OK;
}

lbm_status lbm_wall_force(lbm_ctx* ctx, int wall, unsigned flags, double weight, double* out, int out_on_host,
                          void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!out) return arg_fail(x, "out is NULL");
    if (wall > LBM_MAX_WALLS) return arg_fail(x, "wall id out of range");
    if (flags & ~7u) return arg_fail(x, "unknown flag");
    if (x.t < 1) {
        x.err = "the wall force needs at least one step";
        return LBM_ERR_STATE;
    }
    GUARD(x);
    if (!out_mode_ok(out_on_host, (flags & LBM_ACCUMULATE) != 0, out, x.err)) return LBM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const long long b = wall < 0 ? 0 : x.wall_begin[wall];
    const long long e = wall < 0 ? x.n_links : x.wall_begin[wall + 1];
    double* part = x.scratch + SCRATCH_RED_OFF;
    int nb = 0;
    if (e > b) CK(x.ops->links(x, x.pop[x.cur], b, e, flags & 3u, part, &nb, st), "link kernel");
    return finish_reduce(x, part, nb, 3, out, out_on_host, weight, (flags & LBM_ACCUMULATE) != 0, st);
}

lbm_status lbm_step_force(lbm_ctx* ctx, int wall, unsigned flags, double weight, double* out, int out_on_host,
                          void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!out) return arg_fail(x, "out is NULL");
    if (wall > LBM_MAX_WALLS) return arg_fail(x, "wall id out of range");
    if (flags & ~7u) return arg_fail(x, "unknown flag");
    if (x.t < 1) {
        x.err = "the wall force needs at least one step";
        return LBM_ERR_STATE;
    }
    GUARD(x);
    if (!out_mode_ok(out_on_host, (flags & LBM_ACCUMULATE) != 0, out, x.err)) return LBM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (x.stage_R <= 0 || !all_periodic(&x.cfg) || x.ext) {
        // the register-tiled step, or a staged step with closed faces (whose
        // face links the boundary warps do not see) or the EXT node code: the
        // two calls in sequence
        const lbm_status s = lbm_wall_force(ctx, wall, flags, weight, out, out_on_host, stream);
        if (s != LBM_OK) return s;
        return lbm_step(ctx, 1, stream);
    }
    StgForce fw;
    memset(&fw, 0, sizeof fw);
    fw.out = x.scratch + SCRATCH_RED_OFF;
    fw.wall = wall;
    fw.flags = flags & 1u;
    fw.c = x.kpd.c;
    fw.rho0 = x.kpd.rho0;
    fw.svol = x.kpd.svol;
    for (int w = 0; w <= MAXW; ++w)
        for (int k = 0; k < 3; ++k) fw.lw[w][k] = x.kpf.LW[w][k];
    // the kernel's last block writes the sum: to out (device output) or to
    // the result slot, copied to the host below
    fw.ticket = reinterpret_cast<unsigned*>(x.scratch + SCRATCH_TICKET_OFF);
    const bool dev = out_on_host == LBM_OUT_DEVICE;
    fw.result = dev ? out : x.scratch + SCRATCH_OUT_OFF;
    fw.weight = weight;
    fw.accumulate = dev && (flags & LBM_ACCUMULATE) ? 1 : 0;
    CK(x.ops->step_force(x, x.pop[x.cur], x.pop[1 - x.cur], step_seed(x, x.t), fw, st), "step kernel");
    x.cur = 1 - x.cur;
    x.t += 1;
    x.prev_valid = true;
    if (dev) return LBM_OK;
    if (out_on_host == LBM_OUT_HOST_ASYNC) {
        CK(cudaMemcpyAsync(out, fw.result, 3 * sizeof(double), cudaMemcpyDeviceToHost, st), "copy result");
        return LBM_OK;
    }
    double tmp[3];
    CK(cudaMemcpyAsync(tmp, fw.result, sizeof tmp, cudaMemcpyDeviceToHost, st), "copy result");
    CK(cudaStreamSynchronize(st), "synchronize");
    bool finite = true;
    for (int k = 0; k < 3; ++k) {
        out[k] = (flags & LBM_ACCUMULATE) ? out[k] + tmp[k] : tmp[k];
        finite = finite && std::isfinite(tmp[k]);
    }
    if (!finite) {
        x.err = "the wall force is not finite (the state holds NaN or Inf values)";
        return LBM_ERR_NAN;
    }
    return LBM_OK;
}

lbm_status lbm_balance(lbm_ctx* ctx, double* out, int out_on_host, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!out) return arg_fail(x, "out is NULL");
    GUARD(x);
    if (!out_mode_ok(out_on_host, false, out, x.err)) return LBM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double* part = x.scratch + SCRATCH_RED_OFF;
    int nb = 0;
    CK(x.ops->balance(x, x.pop[x.cur], part, &nb, st), "balance kernel");
    return finish_reduce(x, part, nb, 7, out, out_on_host, 1.0, false, st);
}

lbm_status lbm_residual(lbm_ctx* ctx, double* v_ref, int update, double* out, int out_on_host, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!out || !v_ref) return arg_fail(x, "out and v_ref are required");
    if (((uintptr_t)v_ref) % 8) return arg_fail(x, "v_ref must be 8-byte aligned");
    GUARD(x);
    if (!out_mode_ok(out_on_host, false, out, x.err)) return LBM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double* part = x.scratch + SCRATCH_RED_OFF;
    int nb = 0;
    CK(x.ops->residual(x, x.pop[x.cur], v_ref, update ? 1 : 0, part, &nb, st), "residual kernel");
    if (out_on_host == LBM_OUT_HOST) {
        double sums[2] = {0.0, 0.0};
        const lbm_status s = finish_reduce(x, part, nb, 2, sums, LBM_OUT_HOST, 1.0, false, st);
        out[0] = sums[0];
        out[1] = sums[1];
        out[2] = sums[1] > 0.0 ? sums[0] / sums[1] : 0.0;
        if (s == LBM_OK && !std::isfinite(out[2])) {
            x.err = "the residual is not finite";
            return LBM_ERR_NAN;
        }
        return s;
    }
    // device or page-locked host output: the two sums and their ratio in the
    // result slot, copied in stream order (HOST_ASYNC) or written to out
    double* slot = (out_on_host == LBM_OUT_DEVICE) ? out : x.scratch + SCRATCH_OUT_OFF;
    CK(launch_reduce_rows(part, nb, 2, slot, 1.0, 0, st), "reduce");
    CK(launch_ratio(slot, st), "ratio");
    if (out_on_host == LBM_OUT_HOST_ASYNC)
        CK(cudaMemcpyAsync(out, slot, 3 * sizeof(double), cudaMemcpyDeviceToHost, st), "copy result");
    return LBM_OK;
}

lbm_status lbm_run_steady(lbm_ctx* ctx, int every, double tol, int64_t max_steps, double* v_ref, double* r_out,
                          int64_t* steps_out, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (every < 1 || !(tol >= 0.0) || max_steps < 0 || !v_ref) return arg_fail(x, "every >= 1, tol >= 0, max_steps >= 0 and v_ref are required");
    double out[3];
    int64_t taken = 0;
    if (steps_out) *steps_out = 0;
    // the reference field of the starting state
    lbm_status s = lbm_residual(ctx, v_ref, 1, out, LBM_OUT_HOST, stream);
    if (s != LBM_OK) return s;
    double r = -1.0;
    while (taken < max_steps) {
        const int n = (int)std::min<int64_t>(every, max_steps - taken);
        s = lbm_step(ctx, n, stream);
        if (s != LBM_OK) return s;
        taken += n;
        s = lbm_residual(ctx, v_ref, 1, out, LBM_OUT_HOST, stream);
        if (steps_out) *steps_out = taken;
        if (s != LBM_OK) return s;
        r = out[2];
        if (r_out) *r_out = r;
        if (n == every && r <= tol) return LBM_OK;
    }
    char buf[160];
    snprintf(buf, sizeof buf, "not steady after %lld steps: residual %.3e over %d steps > %.3e", (long long)taken, r,
             every, tol);
    x.err = buf;
    return LBM_ERR_NOT_CONVERGED;
}

lbm_status lbm_adjoint_buffer_bytes(const lbm_ctx* ctx, size_t* bytes)
{
    if (!ctx || !bytes) return LBM_ERR_ARG;
    *bytes = round256((size_t)ctx->c.cfg.lattice * ctx->c.geo.sq * ctx->c.relem);
    return LBM_OK;
}

lbm_status lbm_adjoint_reset(lbm_ctx* ctx, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    GUARD(x);
    CK(launch_zero(x.scratch + SCRATCH_ADJ_OFF, (long long)ADJ_BLOCKS * 6, (cudaStream_t)stream), "zero");
    return LBM_OK;
}

lbm_status lbm_adjoint_step(lbm_ctx* ctx, const void* state_prev, const void* phi_next, void* phi_out, int wall,
                            const double* dir, double seed_weight, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (x.cfg.lorentz || x.cfg.les || x.cfg.curved || x.cfg.stokes || x.cfg.darcy > 0.0 || x.cfg.induced) {
        x.err = "the adjoint supports a uniform body force without LES, on halfway walls, with the equilibrium of Eq. (1)";
        return LBM_ERR_UNSUPPORTED;
    }
    if (!state_prev || !phi_out || !dir || phi_out == phi_next) return arg_fail(x, "bad adjoint buffers");
    if (wall < 1 || wall > x.cfg.n_walls) return arg_fail(x, "wall id out of range");
    GUARD(x);
    CK(x.ops->adjoint(x, state_prev, phi_next, phi_out, wall, dir, seed_weight, x.scratch + SCRATCH_ADJ_OFF,
                      (cudaStream_t)stream),
       "adjoint kernel");
    return LBM_OK;
}

lbm_status lbm_adjoint_gradient(lbm_ctx* ctx, double* out, int out_on_host, void* stream)
{
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!out) return arg_fail(x, "out is NULL");
    GUARD(x);
    if (!out_mode_ok(out_on_host, false, out, x.err)) return LBM_ERR_ARG;
    return finish_reduce(x, x.scratch + SCRATCH_ADJ_OFF, ADJ_BLOCKS, 6, out, out_on_host, 1.0, false,
                         (cudaStream_t)stream);
}

}  // extern "C"

// ------------------------------------------------------- small kernels
namespace lbm {

// warp k sums column k of the nb x W rows: lane l takes rows l, l+32, ...,
// then a fixed shuffle tree; the order never depends on timing
__global__ void k_reduce_rows(const double* __restrict__ partials, int nb, int W, double* __restrict__ out,
                              double weight, int accumulate)
{
    const int col = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (col >= W) return;
    double s = 0.0;
    for (int r = lane; r < nb; r += 32) s += partials[(long long)r * W + col];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[col] = (accumulate ? out[col] : 0.0) + weight * s;
}

cudaError_t launch_reduce_rows(const double* partials, int nb, int W, double* out, double weight, int accumulate,
                               cudaStream_t st)
{
    k_reduce_rows<<<1, 32 * W, 0, st>>>(partials, nb, W, out, weight, accumulate);
    return cudaGetLastError();
}

// insulating walls, after a step: block b sums the warp rows
// [b*chunk, (b+1)*chunk) of the step kernel's velocity sums in a fixed order;
// the last block to finish (ticket) sums the block sums in a fixed order and
// sets the field of Eq. (36), E = -<v> x B with <v> = c sum(v) / n_fluid, and
// its force coefficient dt sigma_e (E x B) / c in FP64, FP32 and FP32 storage
// units, then clears the ticket for the next step
__global__ void k_ins_update(const double* __restrict__ rows, long long n, long long chunk, double* part, double* blk,
                             double n_fluid, double c, double dt, double sigma, double B0, double B1, double B2,
                             double scale)
{
    __shared__ double sm[3 * 32];
    __shared__ int last;
    unsigned* ticket = reinterpret_cast<unsigned*>(blk + INS_TICKET);
    double v[3] = {0.0, 0.0, 0.0};
    const long long b0 = (long long)blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    for (long long r = b0 + threadIdx.x; r < b1; r += blockDim.x)
        for (int k = 0; k < 3; ++k) v[k] += rows[r * 3 + k];
    for (int k = 0; k < 3; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 3; ++k) sm[k * 32 + wid] = v[k];
    __syncthreads();
    if (wid == 0) {
        for (int k = 0; k < 3; ++k) {
            double s = (lane < nw) ? sm[k * 32 + lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) part[blockIdx.x * 3 + k] = s;
        }
        if (lane == 0) {
            __threadfence();
            last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1 : 0;
        }
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // warp k sums column k of the block sums: lane l takes rows l, l+32, ...,
    // then a fixed shuffle tree
    if (wid < 3) {
        double s = 0.0;
        for (int r = lane; r < (int)gridDim.x; r += 32) s += __ldcg(part + r * 3 + wid);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sm[wid] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double* vs = blk + INS_VSUM;
    for (int k = 0; k < 3; ++k) vs[k] = sm[k];
    const double vm[3] = {c * vs[0] / n_fluid, c * vs[1] / n_fluid, c * vs[2] / n_fluid};
    const double B[3] = {B0, B1, B2};
    double E[3];
    E[0] = -(vm[1] * B[2] - vm[2] * B[1]);
    E[1] = -(vm[2] * B[0] - vm[0] * B[2]);
    E[2] = -(vm[0] * B[1] - vm[1] * B[0]);
    const double ExB[3] = {E[1] * B[2] - E[2] * B[1], E[2] * B[0] - E[0] * B[2], E[0] * B[1] - E[1] * B[0]};
    float* af = reinterpret_cast<float*>(blk + INS_AEB_F);
    float* as = reinterpret_cast<float*>(blk + INS_AEB_S);
    for (int k = 0; k < 3; ++k) {
        const double aeb = dt * sigma * ExB[k] / c;
        blk[INS_E + k] = E[k];
        blk[INS_AEB_D + k] = aeb;
        af[k] = (float)aeb;
        as[k] = (float)(aeb * scale);
    }
    *ticket = 0u;
}

// the configured field (after create, init, import or load)
__global__ void k_ins_reset(double* blk, double E0, double E1, double E2, double a0, double a1, double a2,
                            float f0, float f1, float f2, float s0, float s1, float s2)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    blk[INS_E] = E0; blk[INS_E + 1] = E1; blk[INS_E + 2] = E2;
    blk[INS_AEB_D] = a0; blk[INS_AEB_D + 1] = a1; blk[INS_AEB_D + 2] = a2;
    float* af = reinterpret_cast<float*>(blk + INS_AEB_F);
    float* as = reinterpret_cast<float*>(blk + INS_AEB_S);
    af[0] = f0; af[1] = f1; af[2] = f2;
    as[0] = s0; as[1] = s1; as[2] = s2;
    *reinterpret_cast<unsigned*>(blk + INS_TICKET) = 0u;
}

__global__ void k_ratio(double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) out[2] = out[1] > 0.0 ? out[0] / out[1] : 0.0;
}

cudaError_t launch_ratio(double* out, cudaStream_t st)
{
    k_ratio<<<1, 32, 0, st>>>(out);
    return cudaGetLastError();
}

__global__ void k_zero(double* p, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = 0.0;
}

cudaError_t launch_zero(double* p, long long n, cudaStream_t st)
{
    k_zero<<<64, 256, 0, st>>>(p, n);
    return cudaGetLastError();
}

// after a step: sum the warps' velocity rows in a fixed order and set the field
cudaError_t ins_update(const Ctx& x, cudaStream_t st)
{
    const long long n = x.ins_rows;
    const long long chunk = std::max<long long>((n + INS_RED_ROWS - 1) / INS_RED_ROWS, 256);
    const int nb = (int)((n + chunk - 1) / chunk);
    const double scale = (x.cfg.storage == LBM_STORE_F16S) ? 4096.0 : 1.0;
    k_ins_update<<<nb, 256, 0, st>>>(x.scratch + SCRATCH_INS_ROWS, n, chunk, x.scratch + SCRATCH_INS_RED,
                                     x.scratch + SCRATCH_INS_OFF, (double)(x.n_fluid > 0 ? x.n_fluid : 1), x.kpd.c,
                                     x.kpd.dt, x.cfg.sigma_e, x.cfg.B[0], x.cfg.B[1], x.cfg.B[2], scale);
    return cudaGetLastError();
}

// the configured field and its force coefficients (fill_params computed them)
cudaError_t ins_reset(const Ctx& x, cudaStream_t st)
{
    k_ins_reset<<<1, 32, 0, st>>>(x.scratch + SCRATCH_INS_OFF, x.cfg.E[0], x.cfg.E[1], x.cfg.E[2], x.kpd.AEB[0],
                                  x.kpd.AEB[1], x.kpd.AEB[2], x.kpf.AEB[0], x.kpf.AEB[1], x.kpf.AEB[2], x.kps.AEB[0],
                                  x.kps.AEB[1], x.kps.AEB[2]);
    return cudaGetLastError();
}

}  // namespace lbm
