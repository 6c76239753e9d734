// lbm_staged.cuh -- the fused collide-stream step (Eq. 2 with Eqs. 1 and 3,
// and Eq. 10 with the Maxwell term) as a persistent kernel whose input rows
// are staged in shared memory by the bulk asynchronous copies of the tensor
// memory accelerator, for 16-bit or FP32 storage with halfway walls, closed
// or periodic box faces and every node code but curved walls, insulating
// walls and the induced field.
//
// Pull scheme: a tile is R consecutive rows (y0 .. y0+R-1) of one z plane;
// for direction a the tile reads the R source rows shifted by (E_y, E_z),
// which lie contiguously in that direction's plane, so one bulk copy per
// direction (two where the rows wrap around the periodic y axis) brings them
// in, and every stored population is read from HBM once per step.  The x
// shift of the pull is an offset inside the staged row (the periodic x wrap
// an index at the row ends): no shuffles, and no register holds a load in
// flight.  A bulk copy costs the copy engine of an SM a fixed time (measured
// ~33 ns on GB300 whether it moves 512 B or 1 KB), so R is chosen for copies
// of at least 2 KB per direction (R nxp = 1024 nodes for 16-bit storage, 512
// for FP32), and the relaxed populations leave with ordinary coalesced
// stores, which cost the copy engine nothing.
//
// One producer warp keeps up to 8 stages in flight (lane a copies direction
// a): it refills a stage as soon as the consumer warps that read it have
// released it (full / empty mbarriers, the full one with the copies'
// transaction bytes).  Consumer warps form two groups that take alternate
// tiles.  The stage count is even, so tile k uses stage k mod n and every
// stage belongs to one group, which consumes its uses in order: a warp can
// then only wait on the phase of a use whose predecessor its group has
// finished, and a parity wait cannot mistake a phase two uses old for the
// current one (with an odd count a stage alternates between the groups and
// a group running ahead could do exactly that).  A thread relaxes one pair
// of nodes of a 64-node warp task at a time (one 32-bit word per direction
// for 16-bit storage, one float2 for FP32) with k_step's node code for the
// configuration.  Closed faces follow k_step: a source row outside a closed
// y or z face is the node's own row of the opposite direction (the producer
// copies that row instead), the element outside a closed x face is the
// node's own opposite population (the producer stages these face values),
// and moving faces add Ladd's term.  The 4-node chunks that touch a solid
// node, a wall or the padding are not the pipeline's: a boundary warp per
// block takes its share of their list (built on the host) and computes them
// node by node from global memory with explicit bounce-back, exactly as
// k_step does, beside the pipeline -- inline, one such chunk held up its
// stage and with it the in-order producer (the sphere box ran at half the
// rate of the same box without the sphere).  The arithmetic and the
// stochastic rounding stream are those of k_step, so the two kernels store
// the same bits.
//
// Every mbarrier wait is bounded (about a second of the global timer); on
// expiry a warp records a flag for lbm_device_status and stops, and the
// producer waits (again bounded) for the copies it issued before it returns.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int STG_GROUPS = 2;                         // consumer groups (alternate tiles)
constexpr int STG_GROUP_WARPS = 8;                    // warps per group
constexpr int STG_CWARPS = STG_GROUPS * STG_GROUP_WARPS;
constexpr int STG_THREADS = 32 * (STG_CWARPS + 2);    // plus the producer and the boundary warp
constexpr int STG_COPY_BYTES = 2048;                  // least bytes per direction and tile
constexpr int STG_TASK_NODES = 64;                    // nodes per warp task (32 pairs)
constexpr int STG_MAX_STAGES = 8;
constexpr unsigned long long STG_WAIT_NS = 1000000000ull;   // bounded waits: 1 s
constexpr unsigned STG_ERR_TIMEOUT = 1u;
constexpr unsigned STG_ERR_CONFIG = 2u;                     // a launch with an odd stage count

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// true once the phase of this parity has completed; false after ~1 s
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > STG_WAIT_NS) return false;
    return true;
}
// bulk copy global -> shared, completing on the mbarrier's transaction count;
// both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__host__ __device__ inline size_t stg_round128(size_t b) { return (b + 127) / 128 * 128; }

// layout of one stage: Q directions x R rows x nxp values; R x nxp class
// bytes; at a 16-byte boundary the face values, [2][Q][R] values (the
// node's own opposite population at x = 0 and x = nx - 1, for boxes closed
// in x)
__host__ __device__ inline size_t stg_cls_off(int Q, int R, int nxp, int elem) { return (size_t)Q * R * nxp * elem; }
__host__ __device__ inline size_t stg_face_off(int Q, int R, int nxp, int elem)
{
    return (stg_cls_off(Q, R, nxp, elem) + (size_t)R * nxp + 15) / 16 * 16;
}
__host__ __device__ inline size_t stg_stage_bytes(int Q, int R, int nxp, int elem)
{
    return stg_round128(stg_face_off(Q, R, nxp, elem) + (size_t)2 * Q * R * elem);
}

// producer warp: stage the source rows of tile t (plane z, rows y0 .. y0+nr-1).
// Lane 0 arms the full barrier with the tile's copy bytes (its first
// arrival); lane a < Q copies direction a's rows and lane Q the class bytes,
// so the copies of a tile are issued in parallel.  A source row outside a
// closed y or z face is replaced by the node's own row of the opposite
// direction (the bounced population, k_step's rule).  With a closed x face
// the lanes then load the face values (plain loads) and lane 0 arrives a
// second time once they are in the stage.
template <int Q, class S, bool FACES>
__device__ __forceinline__ void stg_issue(const typename S::T* __restrict__ src, const uint8_t* __restrict__ cls,
                                          const Geo& g, int R, int nty, int t, unsigned char* stage, uint64_t* bar,
                                          int lane, int ey, int ez, int oa)
{
    using T = typename S::T;
    const int z = t / nty, y0 = (t - z * nty) * R;
    const int nr = min(R, g.ny - y0);
    const uint32_t rowb = (uint32_t)g.nxp * (uint32_t)sizeof(T);
    if (lane == 0) mbar_expect_tx(bar, (uint32_t)Q * nr * rowb + (uint32_t)nr * g.nxp);
    __syncwarp();
    if (lane < Q) {
        T* d = reinterpret_cast<T*>(stage) + (size_t)lane * R * g.nxp;
        // the node's own rows of the opposite direction (closed faces)
        const T* so = src + (long long)oa * g.sq + (long long)z * g.ny * g.nxp;
        const int zr = z - ez;
        if (FACES && !g.periodic[2] && (zr < 0 || zr >= g.nz)) {
            bulk_g2s(d, so + (long long)y0 * g.nxp, (uint32_t)nr * rowb, bar);
        } else {
            const T* s = src + (long long)lane * g.sq + (long long)wrapi(zr, g.nz) * g.ny * g.nxp;
            const int ys0 = y0 - ey;
            const bool cy = FACES && !g.periodic[1];
            if (ys0 < 0) {                       // row -1: row ny-1, or out of a closed face
                bulk_g2s(d, cy ? so + (long long)y0 * g.nxp : s + (long long)(g.ny - 1) * g.nxp, rowb, bar);
                if (nr > 1) bulk_g2s(d + g.nxp, s, (uint32_t)(nr - 1) * rowb, bar);
            } else if (ys0 + nr > g.ny) {        // row ny: row 0, or out of a closed face
                const int n1 = g.ny - ys0;
                if (n1 > 0) bulk_g2s(d, s + (long long)ys0 * g.nxp, (uint32_t)n1 * rowb, bar);
                bulk_g2s(d + (size_t)n1 * g.nxp, cy ? so + (long long)(y0 + n1) * g.nxp : s,
                         (uint32_t)(nr - n1) * rowb, bar);
            } else {
                bulk_g2s(d, s + (long long)ys0 * g.nxp, (uint32_t)nr * rowb, bar);
            }
        }
    } else if (lane == Q) {
        bulk_g2s(stage + stg_cls_off(Q, R, g.nxp, sizeof(T)), cls + ((long long)z * g.ny + y0) * g.nxp,
                 (uint32_t)nr * g.nxp, bar);
    }
    if (FACES && !g.periodic[0]) {
        // face values: own opposite population at x = 0 (side 0) and nx - 1
        T* fa = reinterpret_cast<T*>(stage + stg_face_off(Q, R, g.nxp, sizeof(T)));
        for (int i = lane; i < 2 * Q * nr; i += 32) {
            const int side = i / (Q * nr), rem = i - side * Q * nr, a = rem / nr, r = rem - a * nr;
            const long long row = ((long long)z * g.ny + y0 + r) * g.nxp;
            fa[(side * Q + a) * R + r] = src[(long long)OPP<Q>(a) * g.sq + row + (side ? g.nx - 1 : 0)];
        }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
}

// the pair (x0, x0+1) of direction a from a staged row: the pull sources
// x0 - ex and x0 + 1 - ex (ex = E_x, or 0 for a row that holds the node's own
// opposite populations), wrapped at the row ends of a periodic x axis; at a
// closed x face the element outside the box is the face value fl (x = 0) or
// fr (x = nx - 1)
template <class S>
__device__ __forceinline__ float2 stg_pair(const typename S::T* __restrict__ row, int ex, int x0, int nx,
                                           bool closed_x, typename S::T fl, typename S::T fr)
{
    using T = typename S::T;
    if constexpr (sizeof(T) == 2) {
        const uint32_t w = *reinterpret_cast<const uint32_t*>(row + x0);
        if (ex == 0) return S::unpack2(w);
        const unsigned short* h = reinterpret_cast<const unsigned short*>(row);
        union { T t; unsigned short u; } cv;
        if (ex == 1) {                                    // values x0-1, x0
            uint32_t e;
            if (x0 == 0) {
                cv.t = fl;
                e = closed_x ? (uint32_t)cv.u : (uint32_t)h[nx - 1];
            } else {
                e = h[x0 - 1];
            }
            return S::unpack2(__byte_perm(e, w, 0x5410));
        }
        uint32_t e;                                       // values x0+1, x0+2
        if (x0 + 2 >= nx) {
            cv.t = fr;
            e = closed_x ? (uint32_t)cv.u : (uint32_t)h[x0 + 2 - nx];
        } else {
            e = h[x0 + 2];
        }
        return S::unpack2(__byte_perm(w, e, 0x5432));
    } else {
        const float2 v = *reinterpret_cast<const float2*>(row + x0);
        if (ex == 0) return v;
        if (ex == 1) return make_float2(x0 == 0 ? (closed_x ? fl : row[nx - 1]) : row[x0 - 1], v.x);
        return make_float2(v.y, x0 + 2 >= nx ? (closed_x ? fr : row[x0 + 2 - nx]) : row[x0 + 2]);
    }
}

// the wall force fused into the staged step: the momentum exchange of Eq.
// (25) of the step that produced the stored state, summed over the links of
// one wall (wall < 0: every wall) in FP64; null `out`: not asked for
struct StgForce {
    double* out;          // one row of 3 doubles per block, or null
    int wall;
    unsigned flags;       // LBM_MOVING_CORR
    double c, rho0, svol; // physical units
    float lw[MAXW + 1][3];  // 6 rho0 u_w / c per wall id (physical units)
    // the last block to write its row sums the rows (ticket: zero between
    // launches) into result: result = (accumulate ? result : 0) + weight sum
    unsigned* ticket;
    double* result;
    double weight;
    int accumulate;
};

// the canonical post-propagation deviations d_b(x) (storage units) of a node
// of a box periodic on every axis with halfway walls, as gather_node: the
// pull source P_b(x - E_b), or through a link into a solid node the bounced
// P_opp(b)(x) plus Ladd's term of the solid's wall.  Every load is issued
// before any is used (one memory round trip for the boundary warps).  With
// a force asked for, each link (x, a' = opp(b)) into a solid adds
// (dx^D/dt) [e_a' (fbar_a' + fbar_b) (+ u_w (fbar_b - fbar_a'))] to acc, with
// fbar_a' = f^rel_a'(x, T-1) and fbar_b = f_b(x, T) its bounced population,
// as the link kernel of lbm_wall_force does.
template <int Q, class S>
__device__ __forceinline__ void gather_periodic(const typename S::T* __restrict__ P, const uint8_t* __restrict__ cls,
                                                const Geo& g, const KP<typename S::R>& p, int x, int y, int z,
                                                long long own, typename S::R (&d)[Q], const StgForce& fw,
                                                double (&acc)[3])
{
    using T = typename S::T;
    using R = typename S::R;
    uint8_t cs[Q];
    T pv[Q], bv[Q];
#pragma unroll
    for (int b = 1; b < Q; ++b) {
        const int xs = wrapi(x - EX<Q>(b), g.nx), ys = wrapi(y - EY<Q>(b), g.ny), zs = wrapi(z - EZ<Q>(b), g.nz);
        const long long src = ((long long)zs * g.ny + ys) * g.nxp + xs;
        cs[b] = cls[src];
        pv[b] = P[(long long)b * g.sq + src];
        bv[b] = P[(long long)OPP<Q>(b) * g.sq + own];
    }
    d[0] = S::to_raw(P[own]);
#pragma unroll
    for (int b = 1; b < Q; ++b) {
        if (nc_solid(cs[b])) {
            const int wall = nc_wall(cs[b]);
            const R L = R(WD<Q>(b)) * (R(EX<Q>(b)) * p.LW[wall][0] + R(EY<Q>(b)) * p.LW[wall][1] +
                                       R(EZ<Q>(b)) * p.LW[wall][2]);
            d[b] = S::to_raw(bv[b]) + L;
            if (fw.out && (fw.wall < 0 || fw.wall == wall)) {
                const float* lw = fw.lw[wall];
                const double w = WD<Q>(b);
                const float Lp = (float)w * ((float)EX<Q>(b) * lw[0] + (float)EY<Q>(b) * lw[1] + (float)EZ<Q>(b) * lw[2]);
                const double fo = (double)S::to_r(bv[b]) + w * fw.rho0;
                const double fi = (double)(S::to_r(bv[b]) + Lp) + w * fw.rho0;
                const int e[3] = {-EX<Q>(b), -EY<Q>(b), -EZ<Q>(b)};     // e_a', a' = opp(b)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    double t = fw.c * e[k] * (fo + fi);
                    if (fw.flags & 1u) t += (double)lw[k] * fw.c / (6.0 * fw.rho0) * (fi - fo);
                    acc[k] += fw.svol * t;
                }
            }
        } else {
            d[b] = S::to_raw(pv[b]);
        }
    }
}

// EXT: the node code with the Lorentz force, Maxwell term, LES, linear
// equilibrium or Darcy resistance; FACES: some box axis is closed.  The node
// code of each configuration is k_step's: the FP32x2 pair code without EXT,
// the FP32x2 EXT pair code for FP32 storage with closed faces, else the
// scalar EXT code node by node; LP: the FP32x2 pair code specialised for
// LES (LES-only contexts).
template <int Q, class S, bool SR, bool EXT = false, bool FACES = false, bool LP = false>
__global__ void __launch_bounds__(STG_THREADS, 1)
k_step_staged(const typename S::T* __restrict__ src, typename S::T* __restrict__ dst,
              const uint8_t* __restrict__ cls, const uint32_t* __restrict__ special, long long nspecial, const Geo g,
              const KP<float> p, uint32_t seed, int R, int ntiles, int nstages, unsigned* __restrict__ errflag,
              const StgForce fw)
{
    using T = typename S::T;
    using Rt = typename S::R;
    static_assert(sizeof(Rt) == 4, "the staged step computes in FP32");
    constexpr bool PAIRX = EXT && !LP && FACES && sizeof(T) == 4;
    extern __shared__ __align__(128) unsigned char smem[];
    const size_t stage_bytes = stg_stage_bytes(Q, R, g.nxp, sizeof(T));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)nstages * stage_bytes);
    uint64_t* empty = full + nstages;
    const int nty = (g.ny + R - 1) / R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the barrier protocol needs an even number of stages (see above)
    if (nstages < 2 || (nstages & 1) || nstages > STG_MAX_STAGES) {
        if (threadIdx.x == 0) atomicOr(errflag, STG_ERR_CONFIG);
        return;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < nstages; ++s) {
            mbar_init(&full[s], 2);          // the producer's two arrivals (copies armed, face values in)
            mbar_init(&empty[s], STG_GROUP_WARPS);
        }
        mbar_fence_init();
    }
    __syncthreads();
    const int my_tiles = ((int)blockIdx.x < ntiles) ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == STG_CWARPS) {
        // producer warp: refill a stage once the group that read it released it
        int ey = 0, ez = 0, oa = 0;          // the pull shift and opposite of this lane's direction
#pragma unroll
        for (int b = 0; b < Q; ++b)
            if (b == lane) {
                ey = EY<Q>(b);
                ez = EZ<Q>(b);
                oa = OPP<Q>(b);
            }
        int k = 0;
        for (; k < my_tiles; ++k) {
            const int s = k % nstages, use = k / nstages;
            if (use > 0) {
                int ok = 0;
                if (lane == 0) ok = mbar_wait_bounded(&empty[s], (uint32_t)(use - 1) & 1u) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) atomicOr(errflag, STG_ERR_TIMEOUT);
                    break;
                }
            }
            stg_issue<Q, S, FACES>(src, cls, g, R, nty, (int)blockIdx.x + k * (int)gridDim.x,
                                   smem + (size_t)s * stage_bytes, &full[s], lane, ey, ez, oa);
        }
        if (k < my_tiles && lane == 0) {
            // stopped early: let the copies already issued land before leaving
            for (int j = (k > nstages ? k - nstages : 0); j < k; ++j)
                mbar_wait_bounded(&full[j % nstages], (uint32_t)(j / nstages) & 1u);
        }
        return;
    }

    if (warp == STG_CWARPS + 1) {
        // boundary warp: the listed chunks, node by node (lane per node), and
        // the wall force of their links when asked for (each lane sums its
        // nodes in a fixed order, then a fixed shuffle tree, one row per block)
        double acc[3] = {0.0, 0.0, 0.0};
        const long long nn = 4 * nspecial;
        for (long long j = (long long)blockIdx.x * 32 + lane; j < nn; j += (long long)gridDim.x * 32) {
            const long long node = (long long)special[j >> 2] + (j & 3);
            const int x = (int)(node % g.nxp);
            const long long row = node / g.nxp;
            const int y = (int)(row % g.ny), z = (int)(row / g.ny);
            const uint8_t c = cls[node];
            if (x >= g.nx || nc_solid(c) || c == NC_PAD) {
#pragma unroll
                for (int a = 0; a < Q; ++a) dst[(long long)a * g.sq + node] = S::from_raw(Rt(0));
                continue;
            }
            Rt d[Q];
            if constexpr (FACES) gather_node<Q, S, true, false>(src, cls, g, p, x, y, z, d);
            else gather_periodic<Q, S>(src, cls, g, p, x, y, z, node, d, fw, acc);
            NodeM<Rt> m;
            node_macro<Rt, Q, EXT, false>(d, p, m);
            node_relax<Rt, Q, EXT>(d, p, m);
            if constexpr (SR) {
                NodeRng rng((uint32_t)node, seed);
#pragma unroll
                for (int a = 0; a < Q; ++a) dst[(long long)a * g.sq + node] = S::from_raw_sr(d[a], rng.bits(a));
            } else {
#pragma unroll
                for (int a = 0; a < Q; ++a) dst[(long long)a * g.sq + node] = S::from_raw(d[a]);
            }
        }
        if (!FACES && fw.out) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
                if (lane == 0) fw.out[(long long)blockIdx.x * 3 + k] = acc[k];
            }
            // the last block's boundary warp sums the rows: lane l takes rows
            // l, l+32, ..., then a fixed shuffle tree (the order of the
            // library's fixed-order pass), and clears the ticket
            __threadfence();
            unsigned last = 0;
            if (lane == 0) last = (atomicAdd(fw.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence();
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    double sum = 0.0;
                    for (int r = lane; r < (int)gridDim.x; r += 32) sum += __ldcg(fw.out + (long long)r * 3 + k);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
                    if (lane == 0) fw.result[k] = (fw.accumulate ? fw.result[k] : 0.0) + fw.weight * sum;
                }
                if (lane == 0) *fw.ticket = 0u;
            }
        }
        return;
    }

    const int group = warp / STG_GROUP_WARPS, gw = warp % STG_GROUP_WARPS;
    const int tasks_per_row = g.nxp / STG_TASK_NODES;
    const long long sq = g.sq;
    const bool closed_x = FACES && !g.periodic[0];
    for (int k = group; k < my_tiles; k += STG_GROUPS) {
        const int s = k % nstages, use = k / nstages;
        if (!mbar_wait_bounded(&full[s], (uint32_t)use & 1u)) {
            if (lane == 0) atomicOr(errflag, STG_ERR_TIMEOUT);
            return;
        }
        const int t = (int)blockIdx.x + k * (int)gridDim.x;
        const int z = t / nty, y0 = (t - z * nty) * R;
        const int nr = min(R, g.ny - y0);
        const T* sp = reinterpret_cast<const T*>(smem + (size_t)s * stage_bytes);
        const uint8_t* sc = smem + (size_t)s * stage_bytes + stg_cls_off(Q, R, g.nxp, sizeof(T));
        const T* fa = reinterpret_cast<const T*>(smem + (size_t)s * stage_bytes + stg_face_off(Q, R, g.nxp, sizeof(T)));
        for (int task = gw; task < nr * tasks_per_row; task += STG_GROUP_WARPS) {
            const int r = task / tasks_per_row;
            const int x0 = (task - r * tasks_per_row) * STG_TASK_NODES + 2 * lane;
            const int y = y0 + r;
            const long long base = ((long long)z * g.ny + y) * g.nxp + x0;
            // the pair path serves pairs whose aligned 4-node chunk holds only
            // bulk (and, with closed faces, face) nodes, as in k_step, whose
            // vector chunks are 4 nodes: both kernels run the same code on
            // every node
            const uint32_t cb = *reinterpret_cast<const uint32_t*>(sc + (size_t)r * g.nxp + (x0 & ~3));
            if ((cb & (FACES ? ~0x02020202u : ~0u)) != 0u) continue;   // the boundary warps' (listed on the host)
            FaceInfo fi;
            if constexpr (FACES) {
                fi.closed_x = closed_x;
                fi.yo_lo = !g.periodic[1] && y == 0;
                fi.yo_hi = !g.periodic[1] && y == g.ny - 1;
                fi.zo_lo = (Q == 19) && !g.periodic[2] && z == 0;
                fi.zo_hi = (Q == 19) && !g.periodic[2] && z == g.nz - 1;
                fi.wx_lo = g.face_wall[0]; fi.wx_hi = g.face_wall[1];
                fi.wy_lo = g.face_wall[2]; fi.wy_hi = g.face_wall[3];
                fi.wz_lo = g.face_wall[4]; fi.wz_hi = g.face_wall[5];
            }
            F2 dd[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                int wall = 0;
                const bool rout = FACES && row_out<Q>(fi, a, wall);
                const T fl = closed_x ? fa[a * R + r] : T(0);
                const T fr = closed_x ? fa[(Q + a) * R + r] : T(0);
                dd[a] = F2{stg_pair<S>(sp + ((size_t)a * R + r) * g.nxp, rout ? 0 : EX<Q>(a), x0, g.nx, closed_x, fl,
                                       fr)};
            }
            if (FACES && p.face_ladd && (cb & 0x02020202u)) {
                // Ladd terms of moving face walls (k_step's add_ladd2)
#pragma unroll
                for (int a = 1; a < Q; ++a) {
                    int wall = 0;
                    const bool hit = row_out<Q>(fi, a, wall);
                    int w0 = wall, w1 = wall;
                    bool h0 = hit, h1 = hit;
                    if (fi.closed_x) {
                        if (EX<Q>(a) == 1 && x0 == 0) { h0 = true; w0 = fi.wx_lo; }
                        if (EX<Q>(a) == -1 && x0 == g.nx - 1) { h0 = true; w0 = fi.wx_hi; }
                        if (EX<Q>(a) == -1 && x0 + 1 == g.nx - 1) { h1 = true; w1 = fi.wx_hi; }
                    }
                    if (h0) dd[a].v.x += ladd_of<Q, float>(p, a, w0);
                    if (h1) dd[a].v.y += ladd_of<Q, float>(p, a, w1);
                }
            }
            if constexpr (!EXT || LP || PAIRX) {
                if constexpr (PAIRX) pair_collide_ext<Q>(dd, p);
                else pair_collide<Q, LP, sizeof(T) == 2>(dd, p);
            } else {
                // the scalar EXT node code, node by node
                Rt d0[Q], d1[Q];
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    d0[a] = dd[a].v.x;
                    d1[a] = dd[a].v.y;
                }
                {
                    NodeM<Rt> m;
                    node_macro<Rt, Q, true, false>(d0, p, m);
                    node_relax<Rt, Q, true>(d0, p, m);
                }
                {
                    NodeM<Rt> m;
                    node_macro<Rt, Q, true, false>(d1, p, m);
                    node_relax<Rt, Q, true>(d1, p, m);
                }
#pragma unroll
                for (int a = 0; a < Q; ++a) dd[a].v = make_float2(d0[a], d1[a]);
            }
            if constexpr (sizeof(T) == 2) {
                if constexpr (SR) {
                    NodeRng rp((uint32_t)base, seed);
#pragma unroll
                    for (int a = 0; a < Q; ++a)
                        *reinterpret_cast<uint32_t*>(dst + (long long)a * sq + base) =
                            S::pack2_sr(dd[a].v.x, dd[a].v.y, rp.word());
                } else {
#pragma unroll
                    for (int a = 0; a < Q; ++a)
                        *reinterpret_cast<uint32_t*>(dst + (long long)a * sq + base) = S::pack2(dd[a].v.x, dd[a].v.y);
                }
            } else {
#pragma unroll
                for (int a = 0; a < Q; ++a) *reinterpret_cast<float2*>(dst + (long long)a * sq + base) = dd[a].v;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);     // this warp is done with stage s
    }
}

}  // namespace lbm
