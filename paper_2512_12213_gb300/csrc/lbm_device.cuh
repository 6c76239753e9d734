// lbm_device.cuh -- device-side lattice tables, population storage formats,
// kernel parameters and the per-node arithmetic of the BGK relaxation with a
// body-force term (arXiv 2512.12213, Sec. 2: Eqs. 1-5; Sec. 4: Eq. 10).
//
// Conventions inside the kernels
//   * populations are held as shifted deviations d_a = f_a - w_a rho0, so the
//     density is rho = rho0 + sum d and the momentum sum e f = c sum E d;
//   * E_a are the integer lattice directions (e_a = c E_a); velocities are
//     kept in units of c (W = u/c) and the body force as the velocity
//     increment per step A = dt a / c, so c drops out of Eqs. (1)-(3):
//       f^eq_a = rho w_a [1 + 3 E.W + 9/2 (E.W)^2 - 3/2 W.W]
//       F_a    = C rho w_a [3 E.A - 3 W^F.A + 9 (E.W^F)(E.A)]
//   * R is the compute type (double for FP64 storage, float otherwise).
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbm {

// ---------------------------------------------------------------- lattices
// D2Q9 : 0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
// D3Q19: 0 rest, 1/2 +-x, 3/4 +-y, 5/6 +-z, 7/8 +-(1,1,0), 9/10 +-(1,-1,0),
//        11/12 +-(1,0,1), 13/14 +-(1,0,-1), 15/16 +-(0,1,1), 17/18 +-(0,1,-1)
template <int Q> __host__ __device__ constexpr int EX(int a)
{
    constexpr int t9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int t19[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return Q == 9 ? t9[a] : t19[a];
}
template <int Q> __host__ __device__ constexpr int EY(int a)
{
    constexpr int t9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    constexpr int t19[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return Q == 9 ? t9[a] : t19[a];
}
template <int Q> __host__ __device__ constexpr int EZ(int a)
{
    constexpr int t19[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return Q == 9 ? 0 : t19[a];
}
template <int Q> __host__ __device__ constexpr int OPP(int a)
{
    constexpr int t9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    return Q == 9 ? t9[a] : (a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1));
}
// speed class: 0 rest, 1 axis, 2 diagonal
template <int Q> __host__ __device__ constexpr int SPEED2(int a)
{
    return EX<Q>(a) * EX<Q>(a) + EY<Q>(a) * EY<Q>(a) + EZ<Q>(a) * EZ<Q>(a);
}
template <int Q> __host__ __device__ constexpr double WD(int a)
{
    return Q == 9 ? (SPEED2<Q>(a) == 0 ? 4.0 / 9.0 : (SPEED2<Q>(a) == 1 ? 1.0 / 9.0 : 1.0 / 36.0))
                  : (SPEED2<Q>(a) == 0 ? 1.0 / 3.0 : (SPEED2<Q>(a) == 1 ? 1.0 / 18.0 : 1.0 / 36.0));
}
// the first direction of each opposite pair (the other is OPP of it)
template <int Q> __host__ __device__ constexpr int PAIR(int k)
{
    constexpr int t9[4] = {1, 2, 5, 6};
    return Q == 9 ? t9[k] : 2 * k + 1;
}
template <int Q> struct LatDim { static constexpr int D = (Q == 9) ? 2 : 3; static constexpr int NP = (Q - 1) / 2; };

// ------------------------------------------------------- storage formats
// Each format stores the shifted deviation d; V nodes fill one 16-byte vector.
// to_r/from_r convert to and from the physical deviation d; to_raw/from_raw
// keep the storage units (d times SCALE), in which the step kernels work
// with parameters scaled to match (see scale_params on the host).
struct StoreF64 {
    using T = double; using R = double; static constexpr int V = 2;
    static constexpr double SCALE = 1.0;
    __device__ static R to_r(T x) { return x; }
    __device__ static T from_r(R x) { return x; }
    __device__ static R to_raw(T x) { return x; }
    __device__ static T from_raw(R x) { return x; }
};
struct StoreF32 {
    using T = float; using R = float; static constexpr int V = 4;
    static constexpr double SCALE = 1.0;
    __device__ static R to_r(T x) { return x; }
    __device__ static T from_r(R x) { return x; }
    __device__ static R to_raw(T x) { return x; }
    __device__ static T from_raw(R x) { return x; }
};
// binary16 holds 2^12 d: typical deviations 1e-5..1e-1 then sit in the normal
// range of the format (min normal 6.1e-5, max 65504).
struct StoreF16 {
    using T = __half; using R = float; static constexpr int V = 4;
    static constexpr double SCALE = 4096.0;
    __device__ static R to_r(T x) { return __half2float(x) * (1.0f / 4096.0f); }
    __device__ static T from_r(R x) { return __float2half_rn(x * 4096.0f); }
    __device__ static R to_raw(T x) { return __half2float(x); }
    __device__ static T from_raw(R x) { return __float2half_rn(x); }
    // two packed values <-> two floats
    __device__ static float2 unpack2(uint32_t w)
    {
        __half2 h;
        memcpy(&h, &w, 4);
        return __half22float2(h);
    }
    // stochastic rounding by the sm_100-family convert: the magnitude is
    // rounded up with probability equal to the discarded fraction of one unit
    // in the last place (13 random bits per value: bits 0-12 of r for the low
    // half, 16-28 for the high half; exact in the subnormal range too),
    // saturating to the largest finite value
    __device__ static uint32_t cvt_rs(float hi, float lo, uint32_t r)
    {
        uint32_t w;
        asm volatile("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(w) : "f"(hi), "f"(lo), "r"(r));
        return w;
    }
    __device__ static T from_raw_sr(float v, uint32_t r)
    {
        return __ushort_as_half((unsigned short)(cvt_rs(0.0f, v, r) & 0xFFFFu));
    }
    __device__ static uint32_t pack2(float a, float b)
    {
        __half2 h = __floats2half2_rn(a, b);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
    // a (low half) and b (high half) rounded stochastically with the two
    // 13-bit fields of one random word
    __device__ static uint32_t pack2_sr(float a, float b, uint32_t r) { return cvt_rs(b, a, r); }
};
struct StoreBF16 {
    using T = __nv_bfloat16; using R = float; static constexpr int V = 4;
    static constexpr double SCALE = 1.0;
    __device__ static R to_r(T x) { return __bfloat162float(x); }
    __device__ static T from_r(R x) { return __float2bfloat16_rn(x); }
    __device__ static R to_raw(T x) { return __bfloat162float(x); }
    __device__ static T from_raw(R x) { return __float2bfloat16_rn(x); }
    __device__ static float2 unpack2(uint32_t w)
    {
        __nv_bfloat162 h;
        memcpy(&h, &w, 4);
        return __bfloat1622float2(h);
    }
    // stochastic rounding by the sm_100-family convert: 16 random bits per
    // value (bits 0-15 of r for the low half, 16-31 for the high half), the
    // magnitude rounded up with probability equal to the discarded fraction
    __device__ static uint32_t cvt_rs(float hi, float lo, uint32_t r)
    {
        uint32_t w;
        asm volatile("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(w) : "f"(hi), "f"(lo), "r"(r));
        return w;
    }
    __device__ static T from_raw_sr(float v, uint32_t r)
    {
        return __ushort_as_bfloat16((unsigned short)(cvt_rs(0.0f, v, r) & 0xFFFFu));
    }
    __device__ static uint32_t pack2(float a, float b)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
    // a (low half) and b (high half) rounded stochastically with the two
    // 16-bit fields of one random word
    __device__ static uint32_t pack2_sr(float a, float b, uint32_t r) { return cvt_rs(b, a, r); }
};

// one thread's vector of V consecutive stored values (16 or 8 bytes)
template <int B> struct RawVec;
template <> struct RawVec<16> { using type = uint4; };
template <> struct RawVec<8> { using type = uint2; };
template <class T, int V> union VecN {
    typename RawVec<sizeof(T) * V>::type raw;
    T e[V];
    uint32_t u[sizeof(T) * V / 4];
};

// ------------------------------------------------- counter-based random bits
// 32-bit integer hash of a counter: a multiply-xorshift finaliser with the
// published "lowbias32" shifts and multipliers found by C. Wellons' hash
// prospector; and the per-node stream: one hash of (node, step seed), then
// a linear congruential step per random word with the multiplier and
// increment of M. O'Neill's PCG32 (as in the pcg_hash of Jarzynski and
// Olano, JCGT 2020), output xor-shifted.  bits(a) gives a node's
// populations 16 bits each (two per word); word() gives one 32-bit word,
// whose two halves round the same direction of the two nodes of a packed
// pair.
__host__ __device__ inline uint32_t hash32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
struct NodeRng {
    uint32_t s;
    __device__ explicit NodeRng(uint32_t node, uint32_t seed) : s(hash32(node ^ hash32(seed))) {}
    // random bits for population a (two populations per generator step)
    __device__ uint32_t bits(int a)
    {
        if ((a & 1) == 0) s = s * 747796405u + 2891336453u;
        const uint32_t r = s ^ (s >> 13);
        return (a & 1) ? (r >> 16) : r;
    }
    // (the empty volatile statement keeps each word next to the conversion
    // that consumes it, instead of all of them held in registers at once)
    __device__ uint32_t word()
    {
        s = s * 747796405u + 2891336453u;
        asm volatile("" : "+r"(s));
        return s ^ (s >> 13);
    }
};

// ------------------------------------------------------------- geometry
// Populations (and node classes) use a padded pitch nxp (a multiple of 64
// nodes, so every row starts on a 128-byte boundary for every format); the
// planes of different directions are sq elements apart.
struct Geo {
    int nx, ny, nz, nxp;
    long long sq;           // elements between direction planes (= nxp*ny*nz)
    int periodic[3];
    int face_wall[6];
    const float* phi;       // signed wall distance per node (padded layout), or null: halfway walls
};

// node classes (one byte per node, padded layout)
// NC_BULK: every pull source is a fluid node (periodic wrap allowed);
// NC_FACE: some links cross a closed face of the box, none hits a solid;
// NC_BOUND: some link hits a solid node; 0x80 | id: solid of wall id; NC_PAD: padding
enum : uint8_t { NC_BULK = 0, NC_BOUND = 1, NC_FACE = 2, NC_PAD = 0xFF };
__host__ __device__ inline bool nc_has_wall(uint8_t c) { return c == NC_BOUND || c == NC_FACE; }
__host__ __device__ inline bool nc_solid(uint8_t c) { return (c & 0x80) && c != NC_PAD; }
__host__ __device__ inline int nc_wall(uint8_t c) { return c & 0x7F; }
__host__ __device__ inline uint8_t nc_make_solid(int wall) { return (uint8_t)(0x80 | wall); }

// ----------------------------------------------------------- parameters
enum { MODEL_A = 0, MODEL_B = 1, MODEL_C = 2, MODEL_D = 3, MODEL_E = 4 };
constexpr int MAXW = 16;

template <typename R> struct KP {
    R rho0, tau0, om0;
    // momentum-consistent relaxation of the odd part (FP32 node codes): the
    // axis directions' 3 w om as one constant wax, the diagonal ones' an
    // exact power-of-two fraction of it, and om1 = 1 - K wax (K = 1/(3 w) of
    // the axis directions: 6 for D3Q19, 3 for D2Q9) exact in this format
    R wax, om1j;
    int kmom;         // K
    R AG[3];          // dt g / c
    int model;
    int lorentz;
    R AEB[3];         // dt sigma_e (E x B) / c   (divided by rho per node)
    R kappa;          // dt sigma_e
    R B[3], B2, Bp2;  // field, |B|^2, |B restricted to the simulated plane|^2
    int maxwell;
    R mx[19];         // Maxwell term of Eq. (10) per direction
    R Lh[6];          // L / c^2: xx yy zz xy xz yz (zero without the Maxwell term)
    int les;
    R lesc;           // 18 Cs^2
    int stokes;       // linear equilibrium (no rho u u)
    R darcy_h;        // dt darcy / 2: porous resistance in the implicit v
    // induced field: the Maxwell term at the node's field, mxk w_a m_a(B) with
    // mxk = 9/(2 c^2 mu) (storage units where the step runs in them); the
    // field lattice's 1/tau_m, wall rule and external field; the current
    // field distributions (physical units, compute precision), set per launch
    int induced, mag_cond;
    R mxk, om_m;
    R Bext[3];
    const R* mag;     // set by the launcher of each kernel that reads the field
    int face_ladd;    // some closed face of the box is a moving wall
    R LW[MAXW + 1][3];  // 6 rho0 u_w / c per wall id (Ladd term = w_a E_a . LW)
    // per-launch constants of the node-pair path (uniform body force only):
    // u^eq = u + ueq_c, u^F = uf_u u + uf_c, C = Cf, E_a . A = pe[a],
    // E_a . ueq_c = peq[a], E_a . uf_c = pf[a]
    R ueq_c[3], uf_u, uf_c[3], Cf;
    R pe[19], peq[19], pf[19];
    // insulating walls: the force coefficient dt sigma_e (E x B) / c of the
    // current field, kept on the device (replaces AEB), and the per-thread
    // rows of the step kernel's flow-velocity sums; null otherwise
    const R* aeb_dev;
    double* ins_rows;
    // units for outputs
    R c, dt, svol;    // c, dt, dx^D / dt
};

// Maxwell term of Eq. (10) for direction a at the field B, in units with
// k = 9 / (2 c^2 mu): k w_a (B^2 |E_a|^2 / 2 - (E_a.B)^2 [- B^2/6 in 3-D])
template <int Q, typename R>
__device__ __forceinline__ R maxwell_at(R k, const R (&B)[3], int a)
{
    const R B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const R eb = R(EX<Q>(a)) * B[0] + R(EY<Q>(a)) * B[1] + R(EZ<Q>(a)) * B[2];
    R t = R(0.5) * B2 * R(SPEED2<Q>(a)) - eb * eb;
    if (Q == 19) t -= B2 / R(6);
    return k * R(WD<Q>(a)) * t;
}

// ---------------------------------------------------- per-node quantities
template <typename R> struct NodeM {
    R Bl[3];              // the node's field (induced field only)
    R rho, drho;
    R j[3];               // momentum sum E d (storage units)
    R u[3], A[3], v[3];   // in units of c (A: velocity increment per step)
    R weq[3], wf[3];      // u^eq / c and u^F / c (wf = 0 for model [a])
    R C, tau, om;
};

// raw moments of the shifted populations: sum d, sum E d, and (LES) sum E_i E_j d
template <typename R> struct Mom {
    R drho, j[3];
    R P[6];   // xx yy zz xy xz yz, only accumulated when LES is on
};

template <typename R, int Q, bool PI>
__device__ __forceinline__ void mom_add(Mom<R>& mo, int a, R v)
{
    mo.drho += v;
    const int ex = EX<Q>(a), ey = EY<Q>(a), ez = EZ<Q>(a);
    if (ex == 1) mo.j[0] += v; else if (ex == -1) mo.j[0] -= v;
    if (ey == 1) mo.j[1] += v; else if (ey == -1) mo.j[1] -= v;
    if (ez == 1) mo.j[2] += v; else if (ez == -1) mo.j[2] -= v;
    if (PI) {
        if (ex) mo.P[0] += v;
        if (ey) mo.P[1] += v;
        if (ez) mo.P[2] += v;
        if (ex * ey) mo.P[3] += R(ex * ey) * v;
        if (ex * ez) mo.P[4] += R(ex * ez) * v;
        if (ey * ez) mo.P[5] += R(ey * ez) * v;
    }
}

template <typename R> __device__ __forceinline__ void mom_zero(Mom<R>& mo)
{
    mo.drho = R(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) mo.j[k] = R(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) mo.P[k] = R(0);
}

// the per-node quantities of the text after Eq. (1) and the per-model
// choices of C, u^F and u^eq of Sec. 2, from the raw moments; EXT enables
// the Lorentz force and LES; INS reads the Lorentz coefficient of insulating
// walls from the device (kernels that never serve them compile without it)
template <typename R, int Q, bool EXT, bool INS = true>
__device__ __forceinline__ void macro_from_moments(const Mom<R>& mo, const KP<R>& p, NodeM<R>& m)
{
    constexpr int D = LatDim<Q>::D;
    const R drho = mo.drho;
    const R rho = p.rho0 + drho, ir = R(1) / rho;
    m.rho = rho;
    m.drho = drho;
    m.j[0] = mo.j[0]; m.j[1] = mo.j[1]; m.j[2] = (D == 3) ? mo.j[2] : R(0);
    m.u[0] = mo.j[0] * ir; m.u[1] = mo.j[1] * ir; m.u[2] = (D == 3) ? mo.j[2] * ir : R(0);
    m.A[0] = p.AG[0]; m.A[1] = p.AG[1]; m.A[2] = (D == 3) ? p.AG[2] : R(0);
    if (EXT && (p.lorentz || p.darcy_h != R(0))) {
        // v = u + A/2 with A = A_g + (kappa/rho)[(v.B)B - B^2 v] - dt darcy v in
        // the D simulated components: (1 + h + k B^2) v - k B_p (B_p . v) = w,
        // k = kappa/(2 rho), h = dt darcy/2, w = u + (A_g + A_EB/rho)/2,
        // solved with the Sherman-Morrison formula; A itself is formed as
        // 2 (v - u) = 2 (A_w/2 + s B - (h + k B^2) u) / (1 + h + k B^2), the
        // small terms directly (v - u taken as a difference would lose the
        // increment to the rounding of u and v in FP32).
        R wv[3], Ag[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const R aeb = (INS && p.aeb_dev) ? p.aeb_dev[k] : p.AEB[k];
            Ag[k] = (k < D) ? p.AG[k] + aeb * ir : R(0);
            wv[k] = m.u[k] + R(0.5) * Ag[k];
        }
        const R kk = R(0.5) * p.kappa * ir;
        const R Bw = p.B[0] * wv[0] + p.B[1] * wv[1] + ((D == 3) ? p.B[2] * wv[2] : R(0));
        const R al = R(1) + p.darcy_h;
        const R den = R(1) / (al + kk * p.B2);
        const R s = kk * Bw / (al + kk * (p.B2 - p.Bp2));
        const R hk = p.darcy_h + kk * p.B2;
#pragma unroll
        for (int k = 0; k < D; ++k) m.A[k] = R(2) * den * (R(0.5) * Ag[k] + s * p.B[k] - hk * m.u[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) m.v[k] = m.u[k] + R(0.5) * m.A[k];
    const bool ueq_v = (p.model == MODEL_E);
#pragma unroll
    for (int k = 0; k < 3; ++k) m.weq[k] = ueq_v ? m.v[k] : m.u[k];
    R tau = p.tau0, om = p.om0;
    if (EXT && p.les) {
        // Smagorinsky: tau_eff = (tau0 + sqrt(tau0^2 + 18 Cs^2 |Pi|/(rho c^2)))/2,
        // |Pi| = sqrt(2 Pi:Pi), Pi the non-equilibrium second moment
        // sum e e f - (p delta + rho u^eq u^eq + L) (E_ij neglected)
        const R third = R(1) / R(3);
        R PP = 0;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int i = (c < 3) ? c : (c == 5 ? 1 : 0);
            const int j = (c < 3) ? c : (c == 3 ? 1 : 2);
            if (D == 2 && (i == 2 || j == 2)) continue;
            R Pc = mo.P[c] - (p.stokes ? R(0) : rho * m.weq[i] * m.weq[j]) - (p.maxwell ? p.Lh[c] : R(0));
            if (i == j) Pc -= drho * third;
            PP += (i == j ? R(1) : R(2)) * Pc * Pc;
        }
        tau = R(0.5) * (p.tau0 + sqrt(p.tau0 * p.tau0 + p.lesc * sqrt(R(2) * PP) * ir));
        om = R(1) / tau;
    }
    m.tau = tau;
    m.om = om;
    m.C = (p.model == MODEL_E) ? R(1) - R(0.5) * om : R(1);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R wf;
        switch (p.model) {
        case MODEL_A: wf = R(0); break;
        case MODEL_B: wf = m.u[k]; break;
        case MODEL_C: wf = m.u[k] + R(0.5) * tau * m.A[k]; break;
        default: wf = m.v[k]; break;
        }
        m.wf[k] = wf;
    }
}

// moments and per-node quantities of the populations d[Q]
template <typename R, int Q, bool EXT, bool INS = true>
__device__ __forceinline__ void node_macro(const R (&d)[Q], const KP<R>& p, NodeM<R>& m)
{
    Mom<R> mo;
    mom_zero(mo);
    if (EXT && p.les) {
#pragma unroll
        for (int a = 0; a < Q; ++a) mom_add<R, Q, true>(mo, a, d[a]);
    } else {
#pragma unroll
        for (int a = 0; a < Q; ++a) mom_add<R, Q, false>(mo, a, d[a]);
    }
    macro_from_moments<R, Q, EXT, INS>(mo, p, m);
}

// The odd part's relaxation carries the momentum, and in FP32 a relative
// error e in its coefficient shifts the momentum that a node gains in a step
// by e om j against rho A: at |u| = 0.05 and a body force of 3e-7 one unit
// in the last place of the coefficient (6e-8) is a 1.5% error.  So the odd
// part relaxes with W_a = 3 w_a om per direction, W_axis rounded once and
// every other W_a an exact power-of-two fraction of it (w_diag / w_axis =
// 1/2 in D3Q19, 1/4 in D2Q9), and the population itself with
// om1 = 1 - K W_axis (one rounding, exact for om in (0.75, 2)): the
// momentum of (om1 d + W E.j) is then om1 j + K W_axis j = j exactly.
template <int Q, typename R>
__device__ __forceinline__ void momentum_coefs(R om, R& Wax, R& om1)
{
    constexpr R c = R(3 * WD<Q>(1)), K = R(Q == 19 ? 6 : 3);
    Wax = om * c;
    om1 = fma(-K, Wax, R(1));
}

// Eq. (2): d <- d + om (d^eq - d) + F for all populations of a node, in the
// form d_a' = (1 - om) d_a + Ps + Pa, d_opp' = (1 - om) d_opp + Ps - Pa per
// opposite pair, with t = E_a.W^eq, the even part
//   Ps = om w (drho - rho 3/2 W.W) - 3 w C rho W^F.A + om 9/2 w rho t^2
//        + 9 w C rho (E_a.W^F)(E_a.A)   (+ om Maxwell term)
// and the odd part Pa = om 3 w rho t + 3 w C rho (E_a.A), the coefficients
// taken once per speed class (Eqs. 1-3).
//
// The odd part is evaluated as Pa = 3 w (om E_a.j + rho E_a.A): with
// rho u = j, W^eq = u + A/2 and C = 1 - om/2 (model [e]) or W^eq = u and
// C = 1 (models [a]-[d]), om rho t + C rho E_a.A equals om E_a.j + rho E_a.A
// exactly.  The odd part alone carries momentum, and in this form the
// momentum that a node gains in a step is om j + rho A - om j = rho A up to
// the rounding of the small terms themselves: u = j / rho and u + A/2,
// rounded in FP32, never enter it.  (Rounded to nearest, u + A/2 misstates
// the increment by the same fraction of a unit in the last place at every
// node whose u shares a binade, which biases the momentum balance of a
// whole flow by ~0.5% in FP32 at a body force of 3e-7.)
template <typename R, int Q, bool EXT, bool MAGF = false>
__device__ __forceinline__ void node_relax(R (&d)[Q], const KP<R>& p, const NodeM<R>& m)
{
    constexpr int D = LatDim<Q>::D;
    const R om = m.om;
    const R rho = m.rho, Crho = m.C * m.rho;
    const bool sto = EXT && p.stokes;        // linear equilibrium: no u^eq u^eq terms
    const R usq = sto ? R(0) : R(1.5) * (m.weq[0] * m.weq[0] + m.weq[1] * m.weq[1] + ((D == 3) ? m.weq[2] * m.weq[2] : R(0)));
    const R fa = m.wf[0] * m.A[0] + m.wf[1] * m.A[1] + ((D == 3) ? m.wf[2] * m.A[2] : R(0));
    const R base = om * (m.drho - rho * usq) - R(3) * Crho * fa;   // times w
    const bool mxw = EXT && p.maxwell;
    // Maxwell term of Eq. (10): the configured table, or (MAGF) at the node's
    // induced field
    auto mx_of = [&](int a) -> R {
        if constexpr (MAGF) return maxwell_at<Q, R>(p.mxk, m.Bl, a);
        else return p.mx[a];
    };
    // odd part: d_a' = om1 d_a + w (ps + 3 rho E_a.A) + W_a E_a.j with
    // W_a = 3 w_a om and om1 = 1 - K W_axis (see momentum_coefs)
    R Wax, om1j;
    momentum_coefs<Q, R>(om, Wax, om1j);
    {
        constexpr R w0 = R(WD<Q>(0));
        d[0] = (sizeof(R) == 8 ? R(1) - om : om1j) * d[0] + w0 * base + (mxw ? om * mx_of(0) : R(0));
    }
    const R k1 = sto ? R(0) : R(4.5) * om * rho, k2 = R(9) * Crho, kf = R(3) * rho;
#pragma unroll
    for (int k = 0; k < LatDim<Q>::NP; ++k) {
        const int a = PAIR<Q>(k), b = OPP<Q>(a);
        const R w = R(WD<Q>(a));
        const int ex = EX<Q>(a), ey = EY<Q>(a), ez = EZ<Q>(a);
        const R t = R(ex) * m.weq[0] + R(ey) * m.weq[1] + ((D == 3) ? R(ez) * m.weq[2] : R(0));
        const R ea = R(ex) * m.A[0] + R(ey) * m.A[1] + ((D == 3) ? R(ez) * m.A[2] : R(0));
        const R ef = R(ex) * m.wf[0] + R(ey) * m.wf[1] + ((D == 3) ? R(ez) * m.wf[2] : R(0));
        const R ej = (sizeof(R) == 8) ? R(0) : R(ex) * m.j[0] + R(ey) * m.j[1] + ((D == 3) ? R(ez) * m.j[2] : R(0));
        R ps = w * (base + k1 * t * t + k2 * ef * ea);
        if (mxw) ps += om * mx_of(a);
        const R da = d[a], db = d[b];
        if constexpr (sizeof(R) == 8) {
            // FP64: the odd part in the paper's form om rho t + C rho E_a.A
            // (its rounding, 1e-16 relative, is far below any balance, and
            // the FP64 pipe bounds this path: no E_a.j and one FMA less)
            const R pa = w * (R(3) * om * rho * t + R(3) * Crho * ea);
            d[a] = fma(R(1) - om, da, ps + pa);
            d[b] = fma(R(1) - om, db, ps - pa);
        } else {
            const R pa = w * (kf * ea);
            const R Wa = Wax * R(WD<Q>(a) / WD<Q>(1));      // a power of two times Wax
            d[a] = fma(Wa, ej, fma(om1j, da, ps + pa));
            d[b] = fma(-Wa, ej, fma(om1j, db, ps - pa));
        }
    }
}

// ------------------------------------------------ node pairs in FP32x2
// Two nodes relaxed together with the packed FP32 instructions of the sm_100
// family: one instruction performs the same operation on both nodes
// (x = first node, y = second).  The arithmetic is that of node_macro and
// node_relax without the Lorentz force, Maxwell term and LES, with the force
// model folded into per-launch constants: u^eq = u + ueq_c,
// u^F = uf_u u + uf_c, C = Cf, and E_a . A = pe[a] (A is uniform).
struct F2 {
    float2 v;
};
__device__ __forceinline__ F2 f2s(float x) { return F2{make_float2(x, x)}; }
__device__ __forceinline__ F2 f2add(F2 a, F2 b) { return F2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 f2mul(F2 a, F2 b) { return F2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 f2fma(F2 a, F2 b, F2 c) { return F2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ F2 f2sub(F2 a, F2 b) { return f2fma(b, f2s(-1.0f), a); }

// E_a . x for a vector of pairs: positive components first, so no negation
template <int Q>
__device__ __forceinline__ F2 f2dot(int a, const F2 (&x)[3])
{
    const int e[3] = {EX<Q>(a), EY<Q>(a), EZ<Q>(a)};
    F2 s = f2s(0.0f);
    bool has = false;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        if (e[c] == 1) {
            s = has ? f2add(s, x[c]) : x[c];
            has = true;
        }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        if (e[c] == -1) {
            s = has ? f2sub(s, x[c]) : f2mul(x[c], f2s(-1.0f));
            has = true;
        }
    return s;
}

__device__ __forceinline__ F2 f2rcp(F2 a) { return F2{make_float2(__frcp_rn(a.v.x), __frcp_rn(a.v.y))}; }
__device__ __forceinline__ F2 f2sqrt(F2 a) { return F2{make_float2(__fsqrt_rn(a.v.x), __fsqrt_rn(a.v.y))}; }
// 1/rho and the Smagorinsky relaxation time of the pair codes with the
// approximate square root and reciprocal of the special-function unit (a
// unit or two in the last place): neither enters a balance -- the odd part
// relaxes from j with momentum_coefs of whatever om results -- and the
// IEEE-rounded forms cost ~10 instructions each (LES cavity 256^3 FP32
// 25.2k -> 27.4k MLUPS)
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ F2 f2sqrta(F2 a) { return F2{make_float2(sqrt_approx(a.v.x), sqrt_approx(a.v.y))}; }
__device__ __forceinline__ F2 f2rcpa(F2 a) { return F2{make_float2(rcp_approx(a.v.x), rcp_approx(a.v.y))}; }

// Eq. (2) with Eqs. (1) and (3) for two nodes: d <- (1 - om) d + om d^eq + F,
// per opposite pair d_a' = (1 - om) d_a + w (X + Y), d_opp' = (1 - om) d_opp
// + w (X - Y) with X = base + 9/2 om rho t^2 + 9 C rho (E_a.u^F)(E_a.A),
// t = E_a.u^eq, and the odd part Y = 3 om rho t + 3 C rho (E_a.A) evaluated
// as 3 om E_a.j + 3 rho E_a.A (equal for every model; node_relax says why).
// LES: the Smagorinsky relaxation time of each node (the arithmetic of
// macro_from_moments without the Maxwell term and the linear equilibrium),
// so om, C and (model [c]) u^F become per-node pairs; the uniform body force
// stays per launch.  GUO: a second relaxation loop for model [e] (u^F =
// u^eq), taken by the 16-bit storage paths (it measured faster there and
// cost the FP32 register-tiled kernel spills).
template <int Q, bool LES = false, bool GUO = false>
__device__ __forceinline__ void pair_collide(F2 (&d)[Q], const KP<float>& p)
{
    constexpr int D = LatDim<Q>::D, NP = LatDim<Q>::NP;
    // moments, from the even and odd parts of each opposite pair; LES adds
    // sum E_i E_j d (xx yy zz xy xz yz)
    F2 drho = d[0];
    F2 j[3] = {f2s(0.0f), f2s(0.0f), f2s(0.0f)};
    bool has[3] = {false, false, false};
    F2 P[6] = {f2s(0.0f), f2s(0.0f), f2s(0.0f), f2s(0.0f), f2s(0.0f), f2s(0.0f)};
    bool hp[6] = {false, false, false, false, false, false};
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int a = PAIR<Q>(k), b = OPP<Q>(a);
        const F2 sm = f2add(d[a], d[b]);
        drho = f2add(drho, sm);
        const F2 t = f2sub(d[a], d[b]);
        const int e[3] = {EX<Q>(a), EY<Q>(a), EZ<Q>(a)};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (e[c] == 0) continue;
            if (!has[c]) j[c] = (e[c] > 0) ? t : f2mul(t, f2s(-1.0f));
            else j[c] = (e[c] > 0) ? f2add(j[c], t) : f2sub(j[c], t);
            has[c] = true;
        }
        if constexpr (LES) {
            const int sg[6] = {e[0] * e[0], e[1] * e[1], e[2] * e[2], e[0] * e[1], e[0] * e[2], e[1] * e[2]};
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                if (sg[c] == 0) continue;
                if (!hp[c]) P[c] = (sg[c] > 0) ? sm : f2mul(sm, f2s(-1.0f));
                else P[c] = (sg[c] > 0) ? f2add(P[c], sm) : f2sub(P[c], sm);
                hp[c] = true;
            }
        }
    }
    // macroscopic quantities (text after Eq. 1, Sec. 2): the node scalars
    // u^eq.u^eq and u^F.A here; per direction below, E_a.u = (E_a.j) / rho,
    // E_a.u^eq = E_a.u + E_a.ueq_c and E_a.u^F = uf_u E_a.u + E_a.uf_c, so
    // that only j stays live through the relaxation
    const F2 rho = f2add(f2s(p.rho0), drho);
    const F2 ir = f2rcpa(rho);      // 1/rho enters the even part only (the odd part relaxes from j)
    F2 q, fa, weq[3];
    F2 om2, om12, C2, htau, wax2;      // per node with LES (htau = tau/2)
    {
        F2 u[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            u[c] = (c < D) ? f2mul(j[c], ir) : f2s(0.0f);
            weq[c] = (c < D) ? f2add(u[c], f2s(p.ueq_c[c])) : f2s(0.0f);
        }
        if constexpr (LES) {
            // tau_eff = (tau0 + sqrt(tau0^2 + 18 Cs^2 |Pi| / rho)) / 2 with
            // |Pi| = sqrt(2 Pi:Pi), Pi = sum E E d - (drho/3 I + rho u^eq u^eq)
            F2 PP = f2s(0.0f);
            const F2 dr3 = f2mul(drho, f2s(1.0f / 3.0f));
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const int i = (c < 3) ? c : (c == 5 ? 1 : 0);
                const int jj = (c < 3) ? c : (c == 3 ? 1 : 2);
                if (D == 2 && (i == 2 || jj == 2)) continue;
                F2 Pc = f2sub(P[c], f2mul(rho, f2mul(weq[i], weq[jj])));
                if (i == jj) Pc = f2sub(Pc, dr3);
                PP = f2fma(f2s(i == jj ? 1.0f : 2.0f), f2mul(Pc, Pc), PP);
            }
            const F2 inner = f2fma(f2mul(f2s(p.lesc), f2sqrta(f2mul(f2s(2.0f), PP))), ir, f2s(p.tau0 * p.tau0));
            const F2 tau = f2mul(f2s(0.5f), f2add(f2s(p.tau0), f2sqrta(inner)));
            om2 = f2rcpa(tau);
            // W_axis and om1 = 1 - K W_axis per node (momentum_coefs)
            wax2 = f2mul(om2, f2s((float)(3 * WD<Q>(1))));
            om12 = f2fma(f2s(Q == 19 ? -6.0f : -3.0f), wax2, f2s(1.0f));
            C2 = (p.model == MODEL_E) ? f2fma(f2s(-0.5f), om2, f2s(1.0f)) : f2s(1.0f);
            htau = f2mul(f2s(0.5f), tau);
        }
        q = f2mul(weq[0], weq[0]);
#pragma unroll
        for (int c = 1; c < D; ++c) q = f2fma(weq[c], weq[c], q);
        // u^F (model [c] with LES: u + tau A / 2 at the node's tau)
        auto wf = [&](int c) -> F2 {
            if (LES && p.model == MODEL_C) return f2fma(htau, f2s(p.AG[c]), u[c]);
            return f2fma(f2s(p.uf_u), u[c], f2s(p.uf_c[c]));
        };
        fa = f2mul(wf(0), f2s(p.AG[0]));
#pragma unroll
        for (int c = 1; c < D; ++c) fa = f2fma(wf(c), f2s(p.AG[c]), fa);
    }
    // relaxation constants: per node with LES, per launch otherwise
    F2 omv, om1v, Crho, Wax, nWax, Wdg, nWdg;
    constexpr float wr = (float)(WD<Q>(Q == 19 ? 7 : 5) / WD<Q>(1));   // w_diag / w_axis: 1/2 or 1/4
    if constexpr (LES) {
        omv = om2;
        om1v = om12;
        Crho = f2mul(C2, rho);
        Wax = wax2;
        nWax = f2mul(wax2, f2s(-1.0f));
        Wdg = f2mul(wax2, f2s(wr));
        nWdg = f2mul(wax2, f2s(-wr));
    } else {
        omv = f2s(p.om0);
        om1v = f2s(p.om1j);
        Crho = f2mul(f2s(p.Cf), rho);
        Wax = f2s(p.wax);
        nWax = f2s(-p.wax);
        Wdg = f2s(p.wax * wr);
        nWdg = f2s(-p.wax * wr);
    }
    // base = om (drho - 3/2 rho u^eq.u^eq) - 3 C rho u^F.A
    F2 base = f2fma(rho, f2mul(q, f2s(-1.5f)), drho);
    base = f2fma(omv, base, f2mul(Crho, f2mul(fa, f2s(-3.0f))));
    d[0] = f2fma(om1v, d[0], f2mul(f2s((float)WD<Q>(0)), base));
    const F2 k1 = LES ? f2mul(rho, f2mul(f2s(4.5f), omv)) : f2mul(rho, f2s(4.5f * p.om0));
    if (GUO && p.model == MODEL_E) {
        // u^F = u^eq: E_a.u^F = t, and the even part w X = w base +
        // t (9/2 w om rho t + 9 w C rho E_a.A) with its node scalars scaled
        // once per speed class
        constexpr float wax_w = (float)WD<Q>(1), wdg_w = (float)WD<Q>(Q == 19 ? 7 : 5);
        const F2 wb_ax = f2mul(f2s(wax_w), base), wb_dg = f2mul(f2s(wdg_w), base);
        const F2 wk_ax = f2mul(f2s(wax_w), k1), wk_dg = f2mul(f2s(wdg_w), k1);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int a = PAIR<Q>(k), b = OPP<Q>(a);
            const float w = (float)WD<Q>(a);
            const bool axis = SPEED2<Q>(a) == 1;
            const F2 t = f2dot<Q>(a, weq), ej = f2dot<Q>(a, j);
            const F2 wX = f2fma(t, f2fma(axis ? wk_ax : wk_dg, t, f2mul(Crho, f2s(9.0f * w * p.pe[a]))),
                                axis ? wb_ax : wb_dg);
            const F2 wY = f2mul(rho, f2s(3.0f * w * p.pe[a]));
            // the odd part's W_a E_a.j last (momentum_coefs)
            d[a] = f2fma(axis ? Wax : Wdg, ej, f2fma(om1v, d[a], f2add(wX, wY)));
            d[b] = f2fma(axis ? nWax : nWdg, ej, f2fma(om1v, d[b], f2sub(wX, wY)));
        }
        return;
    }
    // E_a.j, E_a.u^eq = (E_a.j)/rho + E_a.ueq_c, E_a.u^F = uf_u (E_a.j)/rho
    // + E_a.uf_c (model [c] with LES: (E_a.j)/rho + tau/2 E_a.A)
    auto dots = [&](int a, F2& t, F2& ef, F2& ej) {
        ej = f2dot<Q>(a, j);
        const F2 eu = f2mul(ej, ir);
        t = f2add(eu, f2s(p.peq[a]));
        if (LES && p.model == MODEL_C) ef = f2fma(htau, f2s(p.pe[a]), eu);
        else ef = f2fma(f2s(p.uf_u), eu, f2s(p.pf[a]));
    };
    if constexpr (LES) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int a = PAIR<Q>(k), b = OPP<Q>(a);
            const float w = (float)WD<Q>(a);
            const bool axis = SPEED2<Q>(a) == 1;
            F2 t, ef, ej;
            dots(a, t, ef, ej);
            F2 X = f2fma(k1, f2mul(t, t), base);
            X = f2fma(f2mul(Crho, f2s(9.0f * p.pe[a])), ef, X);
            const F2 wX = f2mul(f2s(w), X), wY = f2mul(rho, f2s(3.0f * w * p.pe[a]));
            // the odd part's W_a E_a.j last (momentum_coefs)
            d[a] = f2fma(axis ? Wax : Wdg, ej, f2fma(om1v, d[a], f2add(wX, wY)));
            d[b] = f2fma(axis ? nWax : nWdg, ej, f2fma(om1v, d[b], f2sub(wX, wY)));
        }
    } else {
        const float om1 = p.om1j;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int a = PAIR<Q>(k), b = OPP<Q>(a);
            const float w = (float)WD<Q>(a);
            F2 t, ef, ej;
            dots(a, t, ef, ej);
            // W_a = p.wax times an exact power of two (momentum_coefs)
            const float Wa = p.wax * (float)(WD<Q>(a) / WD<Q>(1));
            F2 X = f2fma(k1, f2mul(t, t), base);
            X = f2fma(f2mul(Crho, f2s(9.0f * p.pe[a])), ef, X);
            const F2 wX = f2mul(f2s(w), X), wY = f2mul(rho, f2s(3.0f * w * p.pe[a]));
            d[a] = f2fma(f2s(Wa), ej, f2fma(f2s(om1), d[a], f2add(wX, wY)));
            d[b] = f2fma(f2s(-Wa), ej, f2fma(f2s(om1), d[b], f2sub(wX, wY)));
        }
    }
}

// The EXT node code (Lorentz force and Darcy resistance in the implicit
// flow velocity, Smagorinsky LES, the Maxwell term of Eq. 10, the linear
// equilibrium) for two nodes at once: the arithmetic of macro_from_moments
// and node_relax lane by lane, with the per-node relaxation rate as a pair;
// square roots and reciprocals per lane in IEEE FP32.  Not for insulating
// walls (their coefficient lives on the device) or the induced field.
template <int Q>
__device__ __forceinline__ void pair_collide_ext(F2 (&d)[Q], const KP<float>& p)
{
    constexpr int D = LatDim<Q>::D, NP = LatDim<Q>::NP;
    // raw moments: sum d, sum E d and (LES) sum E_i E_j d
    F2 drho = d[0];
    F2 j[3] = {f2s(0.0f), f2s(0.0f), f2s(0.0f)};
    F2 P[6] = {f2s(0.0f), f2s(0.0f), f2s(0.0f), f2s(0.0f), f2s(0.0f), f2s(0.0f)};
    const bool les = p.les != 0;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int a = PAIR<Q>(k), b = OPP<Q>(a);
        const F2 sm = f2add(d[a], d[b]), df = f2sub(d[a], d[b]);
        drho = f2add(drho, sm);
        const int e[3] = {EX<Q>(a), EY<Q>(a), EZ<Q>(a)};
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (e[c]) j[c] = (e[c] > 0) ? f2add(j[c], df) : f2sub(j[c], df);
        if (les) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (e[c]) P[c] = f2add(P[c], sm);
            if (e[0] * e[1]) P[3] = (e[0] * e[1] > 0) ? f2add(P[3], sm) : f2sub(P[3], sm);
            if (e[0] * e[2]) P[4] = (e[0] * e[2] > 0) ? f2add(P[4], sm) : f2sub(P[4], sm);
            if (e[1] * e[2]) P[5] = (e[1] * e[2] > 0) ? f2add(P[5], sm) : f2sub(P[5], sm);
        }
    }
    const F2 rho = f2add(f2s(p.rho0), drho);
    const F2 ir = f2rcpa(rho);      // 1/rho enters the even part only (the odd part relaxes from j)
    F2 u[3], A[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        u[c] = (c < D) ? f2mul(j[c], ir) : f2s(0.0f);
        A[c] = f2s((c < D) ? p.AG[c] : 0.0f);
    }
    if (p.lorentz || p.darcy_h != 0.0f) {
        // (1 + h + k B^2) v - k B_p (B_p . v) = w, k = kappa/(2 rho)
        F2 wv[3], Ag[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Ag[c] = (c < D) ? f2fma(f2s(p.AEB[c]), ir, f2s(p.AG[c])) : f2s(0.0f);
            wv[c] = f2fma(f2s(0.5f), Ag[c], u[c]);
        }
        const F2 kk = f2mul(f2s(0.5f * p.kappa), ir);
        F2 Bw = f2mul(f2s(p.B[0]), wv[0]);
        Bw = f2fma(f2s(p.B[1]), wv[1], Bw);
        if (D == 3) Bw = f2fma(f2s(p.B[2]), wv[2], Bw);
        const float al = 1.0f + p.darcy_h;
        const F2 den = f2rcp(f2fma(kk, f2s(p.B2), f2s(al)));
        const F2 sB = f2mul(f2mul(kk, Bw), f2rcp(f2fma(kk, f2s(p.B2 - p.Bp2), f2s(al))));
        // A = 2 (A_w/2 + s B - (h + k B^2) u) / (1 + h + k B^2): the small
        // terms directly, as in macro_from_moments
        const F2 hk = f2fma(kk, f2s(p.B2), f2s(p.darcy_h));
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const F2 vu = f2fma(f2mul(hk, f2s(-1.0f)), u[c], f2fma(sB, f2s(p.B[c]), f2mul(f2s(0.5f), Ag[c])));
            A[c] = f2mul(f2mul(f2s(2.0f), den), vu);
        }
    }
    F2 v[3], weq[3];
    const bool model_e = (p.model == MODEL_E);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[c] = f2fma(f2s(0.5f), A[c], u[c]);
        weq[c] = model_e ? v[c] : u[c];
    }
    F2 tau = f2s(p.tau0), om = f2s(p.om0);
    if (les) {
        F2 PP = f2s(0.0f);
        const F2 dr3 = f2mul(drho, f2s(1.0f / 3.0f));
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int i = (c < 3) ? c : (c == 5 ? 1 : 0);
            const int jj = (c < 3) ? c : (c == 3 ? 1 : 2);
            if (D == 2 && (i == 2 || jj == 2)) continue;
            F2 Pc = P[c];
            if (!p.stokes) Pc = f2sub(Pc, f2mul(rho, f2mul(weq[i], weq[jj])));
            if (p.maxwell) Pc = f2sub(Pc, f2s(p.Lh[c]));
            if (i == jj) Pc = f2sub(Pc, dr3);
            PP = f2fma(f2s(i == jj ? 1.0f : 2.0f), f2mul(Pc, Pc), PP);
        }
        const F2 inner = f2fma(f2mul(f2s(p.lesc), f2sqrta(f2mul(f2s(2.0f), PP))), ir, f2s(p.tau0 * p.tau0));
        tau = f2mul(f2s(0.5f), f2add(f2s(p.tau0), f2sqrta(inner)));
        om = f2rcpa(tau);
    }
    const F2 C = model_e ? f2fma(f2s(-0.5f), om, f2s(1.0f)) : f2s(1.0f);
    F2 wf[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        switch (p.model) {
        case MODEL_A: wf[c] = f2s(0.0f); break;
        case MODEL_B: wf[c] = u[c]; break;
        case MODEL_C: wf[c] = f2fma(f2mul(f2s(0.5f), tau), A[c], u[c]); break;
        default: wf[c] = v[c]; break;
        }
    }
    // Eq. (2) with the equilibrium of Eq. (1) (+ Eq. 10) and the force of Eq. (3);
    // the odd part relaxes with W_axis and om1 = 1 - K W_axis (momentum_coefs)
    const F2 wax = f2mul(om, f2s((float)(3 * WD<Q>(1))));
    const F2 om1 = f2fma(f2s(Q == 19 ? -6.0f : -3.0f), wax, f2s(1.0f)), Crho = f2mul(C, rho);
    F2 usq = f2s(0.0f), fa = f2s(0.0f);
#pragma unroll
    for (int c = 0; c < D; ++c) {
        usq = f2fma(weq[c], weq[c], usq);
        fa = f2fma(wf[c], A[c], fa);
    }
    if (p.stokes) usq = f2s(0.0f);
    // base = om (drho - 3/2 rho u^eq.u^eq) - 3 C rho u^F.A
    const F2 base = f2fma(om, f2fma(rho, f2mul(usq, f2s(-1.5f)), drho), f2mul(Crho, f2mul(fa, f2s(-3.0f))));
    {
        F2 r0 = f2fma(f2s((float)WD<Q>(0)), base, f2mul(om1, d[0]));
        if (p.maxwell) r0 = f2fma(om, f2s(p.mx[0]), r0);
        d[0] = r0;
    }
    const F2 k1 = p.stokes ? f2s(0.0f) : f2mul(f2mul(f2s(4.5f), om), rho);
    // odd part W_a E_a.j + 3 w rho E_a.A (node_relax says why)
    const F2 k2 = f2mul(f2s(9.0f), Crho);
    constexpr float wr = (float)(WD<Q>(Q == 19 ? 7 : 5) / WD<Q>(1));   // w_diag / w_axis
    const F2 wdg = f2mul(wax, f2s(wr)), nax = f2mul(wax, f2s(-1.0f)), ndg = f2mul(wax, f2s(-wr));
    // 3 w rho per speed class (the odd force term 3 w rho E_a.A)
    const F2 kf_ax = f2mul(f2s((float)(3 * WD<Q>(1))), rho), kf_dg = f2mul(kf_ax, f2s(wr));
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int a = PAIR<Q>(k), b = OPP<Q>(a);
        const float w = (float)WD<Q>(a);
        const bool axis = SPEED2<Q>(a) == 1;
        const F2 t = f2dot<Q>(a, weq), ea = f2dot<Q>(a, A), ef = f2dot<Q>(a, wf), ej = f2dot<Q>(a, j);
        F2 ps = f2fma(k1, f2mul(t, t), base);
        ps = f2fma(k2, f2mul(ef, ea), ps);
        ps = f2mul(f2s(w), ps);
        if (p.maxwell) ps = f2fma(om, f2s(p.mx[a]), ps);
        const F2 pa = f2mul(axis ? kf_ax : kf_dg, ea);
        d[a] = f2fma(axis ? wax : wdg, ej, f2fma(om1, d[a], f2add(ps, pa)));
        d[b] = f2fma(axis ? nax : ndg, ej, f2fma(om1, d[b], f2sub(ps, pa)));
    }
}

// ---------------------------------------------------- closed box faces
// Ladd term w_a E_a . LW[wall] of an incoming population
template <int Q, typename R>
__device__ __forceinline__ R ladd_of(const KP<R>& p, int a, int wall)
{
    return R(WD<Q>(a)) * (R(EX<Q>(a)) * p.LW[wall][0] + R(EY<Q>(a)) * p.LW[wall][1] + R(EZ<Q>(a)) * p.LW[wall][2]);
}

// Box-face bounce-back inside the vectorised path (FACES = some axis is
// closed).  For direction a at a chunk of row (y, z): the pull-source row is
// outside a closed y or z face -> every node of the chunk bounces (own value
// of opp(a)); the first / last node of a row with a closed x face bounces the
// directions that pull across it.  The wall of a link follows the rule
// "first closed axis crossed, in x, y, z order".
struct FaceInfo {
    bool closed_x;
    bool yo_lo, yo_hi, zo_lo, zo_hi;     // pull rows y-(+1), y-(-1), z-(+1), z-(-1) outside
    int wy_lo, wy_hi, wz_lo, wz_hi, wx_lo, wx_hi;
};

template <int Q>
__device__ __forceinline__ bool row_out(const FaceInfo& fi, int a, int& wall)
{
    const int ey = EY<Q>(a), ez = EZ<Q>(a);
    if (ey == 1 && fi.yo_lo) { wall = fi.wy_lo; return true; }
    if (ey == -1 && fi.yo_hi) { wall = fi.wy_hi; return true; }
    if (ez == 1 && fi.zo_lo) { wall = fi.wz_lo; return true; }
    if (ez == -1 && fi.zo_hi) { wall = fi.wz_hi; return true; }
    return false;
}

// -------------------------------------------------------- addressing helpers
__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// one axis of a link: inside -> the coordinate; periodic -> wrapped; closed
// face -> false and the face's wall id (constant indices only, so the
// parameter struct never spills to local memory)
__device__ __forceinline__ bool axis_step(int v, int n, int per, int wlo, int whi, int& out, int& wall)
{
    if (v >= 0 && v < n) { out = v; return true; }
    if (per) { out = (v < 0) ? v + n : v - n; return true; }
    wall = (v < 0) ? wlo : whi;
    return false;
}

// Pull source of direction (ex,ey,ez) at node (x,y,z): returns true and the
// source index (padded layout) if it is a fluid node; false and the wall id
// if the link crosses a closed face (first axis x, y, z) or hits a solid.
__device__ __forceinline__ bool pull_source(const Geo& g, const uint8_t* __restrict__ cls, int x, int y,
                                            int z, int ex, int ey, int ez, long long& src, int& wall)
{
    int xs, ys, zs;
    if (!axis_step(x - ex, g.nx, g.periodic[0], g.face_wall[0], g.face_wall[1], xs, wall)) return false;
    if (!axis_step(y - ey, g.ny, g.periodic[1], g.face_wall[2], g.face_wall[3], ys, wall)) return false;
    if (!axis_step(z - ez, g.nz, g.periodic[2], g.face_wall[4], g.face_wall[5], zs, wall)) return false;
    src = ((long long)zs * g.ny + ys) * g.nxp + xs;
    const uint8_t c = cls[src];
    if (nc_solid(c)) {
        wall = nc_wall(c);
        return false;
    }
    return true;
}

// index of the node (x+ex, y+ey, z+ez), periodic axes wrapped; -1 through a
// closed face of the box
__device__ __forceinline__ long long link_target(const Geo& g, int x, int y, int z, int ex, int ey, int ez)
{
    int xs = 0, ys = 0, zs = 0, wall = 0;
    if (!axis_step(x + ex, g.nx, g.periodic[0], 0, 0, xs, wall)) return -1;
    if (!axis_step(y + ey, g.ny, g.periodic[1], 0, 0, ys, wall)) return -1;
    if (!axis_step(z + ez, g.nz, g.periodic[2], 0, 0, zs, wall)) return -1;
    return ((long long)zs * g.ny + ys) * g.nxp + xs;
}

// The population f_b(x, T) entering fluid node x (padded index own) through a
// link a = opp(b) that leaves x into a solid node or through a closed face
// (wall id `wall`), from the stored post-collision state P (deviations; RAW:
// storage units).  Halfway bounce-back P_a(x) + L with Ladd's term
// L = w_b E_b . LW; with a wall distance (g.phi) and a solid node x + E_a,
// the linear interpolation at the wall point x + q E_a,
// q = phi(x) / (phi(x) - phi(x + E_a)):
//   q <  1/2: 2q P_a(x) + (1 - 2q) P_a(x - E_a) + L   (halfway if x - E_a is no fluid node)
//   q >= 1/2: (P_a(x) + L)/(2q) + (1 - 1/(2q)) P_b(x)
// The weights sum to 1, so the rule holds for the shifted deviations too.
// CURVED = false: halfway only (callers that never see a wall distance).
template <int Q, class S, bool RAW, bool CURVED = true>
__device__ __forceinline__ typename S::R bounced(const typename S::T* __restrict__ P, const uint8_t* __restrict__ cls,
                                                 const Geo& g, const KP<typename S::R>& p, int x, int y, int z,
                                                 long long own, int b, int wall)
{
    using R = typename S::R;
    auto cv = [](typename S::T v) { return RAW ? S::to_raw(v) : S::to_r(v); };
    const int a = OPP<Q>(b);
    const R L = R(WD<Q>(b)) * (R(EX<Q>(b)) * p.LW[wall][0] + R(EY<Q>(b)) * p.LW[wall][1] + R(EZ<Q>(b)) * p.LW[wall][2]);
    const R Pa = cv(P[(long long)a * g.sq + own]);
    const R out = Pa + L;
    if (!CURVED || !g.phi) return out;
    const long long s = link_target(g, x, y, z, EX<Q>(a), EY<Q>(a), EZ<Q>(a));
    if (s < 0 || !nc_solid(cls[s])) return out;            // a closed box face
    const R pf = R(g.phi[own]), ps = R(g.phi[s]);
    const R q = pf / (pf - ps);
    if (q >= R(0.5)) return out / (R(2) * q) + (R(1) - R(1) / (R(2) * q)) * cv(P[(long long)b * g.sq + own]);
    long long ff;
    int w2;
    if (!pull_source(g, cls, x, y, z, EX<Q>(a), EY<Q>(a), EZ<Q>(a), ff, w2)) return out;
    return R(2) * q * Pa + (R(1) - R(2) * q) * cv(P[(long long)a * g.sq + ff]) + L;
}

// canonical post-propagation deviations at node (x,y,z) from a stored
// post-collision state: d_b(x) = P_b(x - E_b), or the bounced population
// through a wall (halfway or interpolated bounce-back, see bounced;
// CURVED = false: halfway only)
template <int Q, class S, bool RAW = false, bool CURVED = true>
__device__ __forceinline__ void gather_node(const typename S::T* __restrict__ P, const uint8_t* __restrict__ cls,
                                            const Geo& g, const KP<typename S::R>& p, int x, int y, int z,
                                            typename S::R (&d)[Q])
{
    using R = typename S::R;
    auto cv = [](typename S::T v) { return RAW ? S::to_raw(v) : S::to_r(v); };
    const long long own = ((long long)z * g.ny + y) * g.nxp + x;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
        long long src;
        int wall;
        if (b == 0) {
            d[0] = cv(P[own]);
        } else if (pull_source(g, cls, x, y, z, EX<Q>(b), EY<Q>(b), EZ<Q>(b), src, wall)) {
            d[b] = cv(P[(long long)b * g.sq + src]);
        } else {
            d[b] = bounced<Q, S, RAW, CURVED>(P, cls, g, p, x, y, z, own, b, wall);
        }
    }
}


// ----------------------------------------------------- induced field
// Field distributions on the axis velocities of the fluid lattice: the
// first QM fluid directions (rest, +-x, +-y [, +-z]) with weights W0, W1.
template <int Q> struct MagLat {
    static constexpr int QM = (Q == 9) ? 5 : 7;
    static constexpr double W0 = (Q == 9) ? 1.0 / 3.0 : 0.25;
    static constexpr double W1 = (Q == 9) ? 1.0 / 6.0 : 0.125;
    static constexpr double TH = (Q == 9) ? 1.0 / 3.0 : 0.25;       // sum W e e = TH I
};

// the canonical field distributions g(x, T) at node (x, y, z) (padded index
// own) from the stored post-collision ones G: G_i(x - e_i) through a fluid
// link, else -G_opp(i)(x) + 2 W_i B_ext (insulating) or G_opp(i)(x)
// (conducting)
template <int Q, typename R>
__device__ __forceinline__ void mag_gather(const R* __restrict__ G, const uint8_t* __restrict__ cls, const Geo& g,
                                           const KP<R>& p, int x, int y, int z, long long own,
                                           R (&gm)[3][MagLat<Q>::QM])
{
    constexpr int QM = MagLat<Q>::QM;
#pragma unroll
    for (int i = 0; i < QM; ++i) {
        const R W = R(i == 0 ? MagLat<Q>::W0 : MagLat<Q>::W1);
        long long src;
        int wall;
        const bool fluid = (i == 0) || pull_source(g, cls, x, y, z, EX<Q>(i), EY<Q>(i), EZ<Q>(i), src, wall);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (i == 0) gm[k][0] = G[(long long)(k * QM) * g.sq + own];
            else if (fluid) gm[k][i] = G[(long long)(k * QM + i) * g.sq + src];
            else {
                const R v = G[(long long)(k * QM + OPP<Q>(i)) * g.sq + own];
                gm[k][i] = p.mag_cond ? v : R(2) * W * p.Bext[k] - v;
            }
        }
    }
}

// the node's field B(x, T) = sum_i g_i(x, T)
template <int Q, typename R>
__device__ __forceinline__ void mag_field_at(const R* __restrict__ G, const uint8_t* __restrict__ cls, const Geo& g,
                                             const KP<R>& p, int x, int y, int z, long long own, R (&B)[3])
{
    R gm[3][MagLat<Q>::QM];
    mag_gather<Q, R>(G, cls, g, p, x, y, z, own, gm);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R s = R(0);
#pragma unroll
        for (int i = 0; i < MagLat<Q>::QM; ++i) s += gm[k][i];
        B[k] = s;
    }
}

}  // namespace lbm
