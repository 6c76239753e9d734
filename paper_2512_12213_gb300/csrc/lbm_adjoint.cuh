// lbm_adjoint.cuh -- the reverse step of the discrete adjoint of the
// collide-stream step and the momentum-exchange drag (arXiv 2512.12213,
// Eqs. 1-3 and 25), for gradients of time-averaged drag with respect to the
// body force and a wall velocity, and its launcher.  Included by
// lbm_kernels.cuh after the other launchers.
#pragma once

namespace lbm {

// per-launch constants of a reverse step, per direction a of a link into the
// target wall: the drag seed 2 w_J svol c (d . E_a) that the link adds to
// psi_a, and -6 w_a rho0 / c, the derivative of the Ladd term with respect
// to E_a . u_w
template <typename R> struct AdjConst {
    R seed[19];
    R gl[19];
};

// ---------------------------------------------------------------- adjoint
// One reverse step of the drag adjoint (uniform body force, any model).
// psi_a(x) = phi_next_a(x + E_a) through a fluid link, or phi_next_opp(a)(x)
// plus the drag seed through a link into the target wall; then
// phi_b = (1 - om) psi_b + A_rho + E_b . B_j, where A_rho and B_j collect the
// derivatives of G = f^eq/tau + F with respect to rho and j, formed from the
// weighted moments s0 = sum w psi, s1 = sum w psi E, s2 = sum w psi E E.
// One node per thread, psi in registers.  Bulk nodes (every link to a fluid
// node, periodic wrap allowed) address their neighbours through nine
// precomputed row offsets and three x positions, without branches; nodes
// next to a wall or a closed face take the general path.  Gradient terms are
// summed per thread in the compute precision and per block in FP64.
// blocks of RED_THREADS per SM: FP64 1; FP32 compute D3Q19 3 (80 registers,
// a few dozen bytes of spill; 18% faster than 2 blocks at 126 registers on
// the 128^3 sphere), D2Q9 2 (the 512 x 256 cylinder ran 23% slower at 3)
template <int Q, class S>
__global__ void __launch_bounds__(RED_THREADS, sizeof(typename S::R) == 8 ? 1 : (Q == 19 ? 3 : 2))
k_adjoint(const typename S::T* __restrict__ Pprev, const typename S::R* __restrict__ phin,
          typename S::R* __restrict__ phio, const uint8_t* __restrict__ cls, const Geo g,
          const KP<typename S::R> p, int target, const AdjConst<typename S::R> ac, double gscale,
          double* __restrict__ partials)
{
    using R = typename S::R;
    constexpr int D = LatDim<Q>::D;
    __shared__ double sm[6 * 32];
    R accg[3] = {0, 0, 0}, accw[3] = {0, 0, 0};
    const long long NP = (long long)g.nxp * g.ny * g.nz;
    // node indices fit in 32 bits (the padded node count is below 2^31)
    const unsigned nxp = (unsigned)g.nxp, ny = (unsigned)g.ny;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < NP; n += (long long)gridDim.x * blockDim.x) {
        const unsigned un = (unsigned)n, ur = un / nxp;
        const int x = (int)(un - ur * nxp);
        const int z = (int)(ur / ny), y = (int)(ur - (unsigned)z * ny);
        const uint8_t cl = cls[n];
        if (x >= g.nx || nc_solid(cl) || cl == NC_PAD) {
#pragma unroll
            for (int a = 0; a < Q; ++a) phio[(long long)a * g.sq + n] = R(0);
            continue;
        }
        Mom<R> mo;
        mom_zero(mo);
        R psi[Q];
        if (cl == NC_BULK) {
            // rows (y + dy, z + dz) and x +- 1, wrapped (bulk nodes wrap only on periodic axes)
            unsigned rows[3][3];
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dz = -1; dz <= 1; ++dz) {
                    const int yy = wrapi(y + dy, g.ny);
                    const int zz = (Q == 19) ? wrapi(z + dz, g.nz) : 0;
                    rows[dy + 1][dz + 1] = ((unsigned)zz * ny + (unsigned)yy) * nxp;
                }
            const unsigned xs[3] = {(unsigned)(x == 0 ? g.nx - 1 : x - 1), (unsigned)x,
                                    (unsigned)(x == g.nx - 1 ? 0 : x + 1)};
            auto at = [&](int ex, int ey, int ez) -> unsigned { return rows[ey + 1][ez + 1] + xs[ex + 1]; };
#pragma unroll
            for (int a = 0; a < Q; ++a)
                mom_add<R, Q, false>(mo, a, S::to_r(Pprev[(long long)a * g.sq + at(-EX<Q>(a), -EY<Q>(a), -EZ<Q>(a))]));
#pragma unroll
            for (int a = 0; a < Q; ++a) psi[a] = phin ? phin[(long long)a * g.sq + at(EX<Q>(a), EY<Q>(a), EZ<Q>(a))] : R(0);
        } else {
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                R v;
                long long sidx;
                int wall;
                if (a == 0) v = S::to_r(Pprev[n]);
                else if (pull_source(g, cls, x, y, z, EX<Q>(a), EY<Q>(a), EZ<Q>(a), sidx, wall))
                    v = S::to_r(Pprev[(long long)a * g.sq + sidx]);
                else
                    v = S::to_r(Pprev[(long long)OPP<Q>(a) * g.sq + n]) + ladd_of<Q, R>(p, a, wall);
                mom_add<R, Q, false>(mo, a, v);
            }
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                long long dn;
                int wall;
                if (a == 0) {
                    psi[0] = phin ? phin[n] : R(0);
                } else if (pull_source(g, cls, x, y, z, EX<Q>(OPP<Q>(a)), EY<Q>(OPP<Q>(a)), EZ<Q>(OPP<Q>(a)), dn,
                                       wall)) {
                    psi[a] = phin ? phin[(long long)a * g.sq + dn] : R(0);
                } else {
                    const R back = phin ? phin[(long long)OPP<Q>(a) * g.sq + n] : R(0);
                    psi[a] = back;
                    if (wall == target) {
                        psi[a] += ac.seed[a];
                        // u_w enters f(t+1) and F_t through the Ladd term
                        const R gl = ac.gl[a] * (back + R(0.5) * ac.seed[a]);
                        accw[0] += gl * R(EX<Q>(a));
                        accw[1] += gl * R(EY<Q>(a));
                        accw[2] += gl * R(EZ<Q>(a));
                    }
                }
            }
        }
        NodeM<R> m;
        macro_from_moments<R, Q, false>(mo, p, m);
        // omega-weighted moments of psi
        R s0 = 0, s1[3] = {0, 0, 0}, s2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const R wp = R(WD<Q>(a)) * psi[a];
            const int e[3] = {EX<Q>(a), EY<Q>(a), EZ<Q>(a)};
            s0 += wp;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                if (e[i]) s1[i] += R(e[i]) * wp;
#pragma unroll
                for (int j = 0; j < D; ++j)
                    if (e[i] * e[j]) s2[i][j] += R(e[i] * e[j]) * wp;
            }
        }
        // sum psi f^eq(rho, W) = rho Psi_e(W); grad_W = rho (3 s1 + 9 s2 W - 3 s0 W)
        // sum psi F = C rho Psi_f; grad_Wf = C rho (9 s2 A - 3 s0 A); grad_A = C rho (3 s1 - 3 s0 Wf + 9 s2 Wf)
        const R* W = m.weq;
        const R* Wf = m.wf;
        const R* A = m.A;
        R s2W[3] = {0, 0, 0}, s2A[3] = {0, 0, 0}, s2F[3] = {0, 0, 0};
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                s2W[i] += s2[i][j] * W[j];
                s2A[i] += s2[i][j] * A[j];
                s2F[i] += s2[i][j] * Wf[j];
            }
        R WW = 0, s1W = 0, WsW = 0, s1A = 0, FA = 0, FsA = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            WW += W[i] * W[i];
            s1W += s1[i] * W[i];
            WsW += W[i] * s2W[i];
            s1A += s1[i] * A[i];
            FA += Wf[i] * A[i];
            FsA += Wf[i] * s2A[i];
        }
        const bool ma = (p.model == MODEL_A);
        const R Psi_e = s0 + R(3) * s1W + R(4.5) * WsW - R(1.5) * WW * s0;
        const R Psi_f = ma ? R(3) * s1A : (R(3) * s1A - R(3) * FA * s0 + R(9) * FsA);
        R Ge[3], Gf[3], GA[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Ge[i] = (i < D) ? m.om * m.rho * (R(3) * s1[i] + R(9) * s2W[i] - R(3) * s0 * W[i]) : R(0);
            Gf[i] = (i < D && !ma) ? m.C * m.rho * (R(9) * s2A[i] - R(3) * s0 * A[i]) : R(0);
            GA[i] = (i < D) ? (ma ? m.C * m.rho * R(3) * s1[i]
                                  : m.C * m.rho * (R(3) * s1[i] - R(3) * s0 * Wf[i] + R(9) * s2F[i]))
                            : R(0);
        }
        // W and Wf move with u = j/rho: d/dj = I/rho, d/drho = -u/rho
        const R ir = R(1) / m.rho;
        R Arho = m.om * Psi_e + m.C * Psi_f;
        R Bj[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Arho -= (Ge[i] + Gf[i]) * m.u[i] * ir;
            Bj[i] = (Ge[i] + Gf[i]) * ir;
        }
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            const R phib = (R(1) - m.om) * psi[b] + Arho + R(EX<Q>(b)) * Bj[0] + R(EY<Q>(b)) * Bj[1] +
                           R(EZ<Q>(b)) * Bj[2];
            phio[(long long)b * g.sq + n] = phib;
        }
        // dJ/dg: A = dt g / c; W^eq moves with A/2 for [e]; W^F with tau/2 ([c]) or 1/2 ([d], [e])
        const R keq = (p.model == MODEL_E) ? R(0.5) : R(0);
        const R kf = (p.model == MODEL_C) ? R(0.5) * m.tau : ((p.model == MODEL_D || p.model == MODEL_E) ? R(0.5) : R(0));
#pragma unroll
        for (int i = 0; i < D; ++i) accg[i] += GA[i] + keq * Ge[i] + kf * Gf[i];
    }
    double acc[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        acc[k] = gscale * (double)accg[k];
        acc[3 + k] = (double)accw[k];
    }
    block_sum<6>(acc, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) partials[(long long)blockIdx.x * 6 + k] += acc[k];
}

// ---------------------------------------------------------------- launcher
template <int Q, class S>
cudaError_t launch_adjoint(const Ctx& c, const void* Pprev, const void* phin, void* phio, int wall,
                           const double* dir, double seedw, double* partials, cudaStream_t st)
{
    using T = typename S::T;
    using R = typename S::R;
    // a fixed grid per context, so every block owns the same partial row each
    // step: the blocks resident at once (SMs x occupancy), each walking the
    // nodes with the grid stride, so no partly filled last wave
    const long long NP = (long long)c.geo.nxp * c.geo.ny * c.geo.nz;
    if (c.adj_blocks == 0) {
        int occ = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adjoint<Q, S>, RED_THREADS, 0);
        if (e != cudaSuccess) return e;
        c.adj_blocks = (int)std::min<long long>(grid_for(NP, RED_THREADS, ADJ_BLOCKS),
                                                 (long long)std::max(occ, 1) * c.sm_count);
    }
    const int blocks = std::min(c.adj_blocks, ADJ_BLOCKS);
    const KP<R>& p = kp_of<S>(c);
    const KP<double>& pd = c.kpd;
    AdjConst<R> ac;
    for (int a = 0; a < 19; ++a) {
        ac.seed[a] = R(0);
        ac.gl[a] = R(0);
    }
    for (int a = 0; a < Q; ++a) {
        const double de = pd.c * (dir[0] * EX<Q>(a) + dir[1] * EY<Q>(a) + dir[2] * EZ<Q>(a));
        ac.seed[a] = R(seedw * 2.0 * pd.svol * de);
        ac.gl[a] = R(-6.0 * WD<Q>(a) * pd.rho0 / pd.c);
    }
    k_adjoint<Q, S><<<blocks, RED_THREADS, 0, st>>>((const T*)Pprev, (const R*)phin, (R*)phio, c.cls, c.geo, p, wall,
                                                    ac, pd.dt / pd.c, partials);
    return cudaGetLastError();
}

}  // namespace lbm
