// lbm_tile.cuh -- the fused collide-stream step as a persistent kernel that
// stages its input rows in shared memory with bulk asynchronous copies.
//
// A tile is R consecutive rows (y0 .. y0+R-1) of one z-plane.  In the pull
// scheme every direction a of the tile reads the R source rows shifted by
// (E_y(a), E_z(a)), which lie contiguously in that direction's plane array,
// so one cp.async.bulk per direction (two when the rows wrap around a
// periodic y face) brings them into shared memory, and every stored
// population is read from HBM exactly once per step.  The x shift is an
// index offset inside the staged row, so the periodic x wrap is free.
// A producer warp keeps 2..6 stages in flight: it refills a stage (full
// mbarrier with transaction count) as soon as the eight consumer warps have
// released it (empty mbarrier), so consumer warps never wait on each other.
// Each consumer thread relaxes one node (or a pair of nodes for 16-bit
// storage) at a time and stores the results with coalesced stores.  Nodes
// next to a wall take the bounced populations from their own stored values.
//
// Every mbarrier wait is bounded; on expiry the block records an error flag,
// waits (bounded) for its own copies in flight and returns.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int TILE_CWARPS = 8;                      // consumer warps
constexpr int TILE_THREADS = 32 * (TILE_CWARPS + 1);  // plus one producer warp
constexpr int TILE_MAX_STAGES = 6;
constexpr unsigned long long WAIT_LIMIT = 1ull << 26;   // try_wait polls before giving up
constexpr unsigned ERR_MBAR_TIMEOUT = 1u;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// bounded wait: true when the phase with this parity has completed
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    for (unsigned long long i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// 1-D bulk copy global -> shared; addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

struct TileShape {
    int R;            // rows per tile
    int ntiles;       // tiles per step
    size_t stage;     // bytes of one stage (populations + classes), 128-aligned
    size_t smem;      // dynamic shared memory of the kernel
};

__host__ __device__ inline size_t round128(size_t b) { return (b + 127) / 128 * 128; }

template <int Q, class S>
__host__ __device__ inline size_t tile_stage_bytes(int R, int nxp)
{
    return round128((size_t)Q * R * nxp * sizeof(typename S::T) + (size_t)R * nxp);
}

// producer: stage the source rows of tile t into buffer s (thread 0 only)
template <int Q, class S>
__device__ __forceinline__ void tile_issue(const typename S::T* __restrict__ src, const uint8_t* __restrict__ cls,
                                           const Geo& g, int R, int nty, int t, unsigned char* stage, uint64_t* bar)
{
    using T = typename S::T;
    const int z = t / nty, y0 = (t % nty) * R;
    const int nr = min(R, g.ny - y0);
    const uint32_t rowb = (uint32_t)g.nxp * sizeof(T);
    mbar_expect_tx(bar, (uint32_t)Q * nr * rowb + (uint32_t)nr * g.nxp);
    T* sp = reinterpret_cast<T*>(stage);
#pragma unroll 1
    for (int a = 0; a < Q; ++a) {
        int ey = 0, ez = 0;
#pragma unroll
        for (int b = 0; b < Q; ++b)
            if (b == a) { ey = EY<Q>(b); ez = EZ<Q>(b); }
        const int zs = wrapi(z - ez, g.nz);
        const int ys0 = y0 - ey;
        T* d = sp + (size_t)a * R * g.nxp;
        const T* s = src + (long long)a * g.sq + (long long)zs * g.ny * g.nxp;
        if (ys0 < 0) {
            bulk_g2s(d, s + (long long)(g.ny - 1) * g.nxp, rowb, bar);
            if (nr > 1) bulk_g2s(d + g.nxp, s, (uint32_t)(nr - 1) * rowb, bar);
        } else if (ys0 + nr > g.ny) {
            const int n1 = g.ny - ys0;
            if (n1 > 0) bulk_g2s(d, s + (long long)ys0 * g.nxp, (uint32_t)n1 * rowb, bar);
            bulk_g2s(d + (size_t)n1 * g.nxp, s, (uint32_t)(nr - n1) * rowb, bar);
        } else {
            bulk_g2s(d, s + (long long)ys0 * g.nxp, (uint32_t)nr * rowb, bar);
        }
    }
    bulk_g2s(stage + (size_t)Q * R * g.nxp * sizeof(T), cls + ((long long)z * g.ny + y0) * g.nxp,
             (uint32_t)nr * g.nxp, bar);
}

// nodes per lane slot (a pair for 16-bit storage, so that a lane stores
// 32 bits), slots per lane, and nodes per warp segment of a row
template <class S> struct TileLanes {
    static constexpr int P = (sizeof(typename S::T) == 2) ? 2 : 1;
    static constexpr int NV = (sizeof(typename S::T) == 4) ? 4 : 2;
    static constexpr int SEG = 32 * NV * P;
};

__device__ __forceinline__ int wrap_x(int x, int nx) { return x < 0 ? nx - 1 : (x >= nx ? 0 : x); }

// One warp relaxes the SEG nodes of a row segment starting at xb: lane l
// owns the slots x = xb + P (l + 32 j) (+ q), j < NV, q < P, so shared-memory
// reads and global stores of a warp are consecutive.  Pass 1 streams the
// staged populations once to accumulate moments; pass 2 streams each
// opposite pair again, relaxes it and stores it.  Slots that touch a wall,
// a solid or padding take the node-by-node path with explicit bounce-back.
// srow: staged populations of this row (direction a at srow + a R nxp);
// crow: staged node classes of this row.
template <int Q, class S, bool EXT>
__device__ __forceinline__ void tile_segment(const typename S::T* __restrict__ srow, const uint8_t* __restrict__ crow,
                                             const typename S::T* __restrict__ src, typename S::T* __restrict__ dst,
                                             const uint8_t* __restrict__ cls, const Geo& g,
                                             const KP<typename S::R>& p, int R, int xb, int y, int z, int lane)
{
    using T = typename S::T;
    using R_ = typename S::R;
    constexpr int P = TileLanes<S>::P, NV = TileLanes<S>::NV;
    const size_t dstride = (size_t)R * g.nxp;       // between directions in the stage
    const long long rowoff = ((long long)z * g.ny + y) * g.nxp;
    bool spec[NV];
    bool any = false;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        spec[j] = false;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int x = xb + P * (lane + 32 * j) + q;
            const uint8_t c = (x < g.nxp) ? crow[x] : (uint8_t)NC_PAD;
            spec[j] |= (c != NC_BULK);
        }
        any |= spec[j];
    }
    // pass 1: moments (every slot; the special ones are recomputed below)
    Mom<R_> mo[NV][P];
#pragma unroll
    for (int j = 0; j < NV; ++j)
#pragma unroll
        for (int q = 0; q < P; ++q) mom_zero(mo[j][q]);
    if (EXT && p.les) {
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const T* sa = srow + (size_t)a * dstride;
#pragma unroll
            for (int j = 0; j < NV; ++j)
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int x = xb + P * (lane + 32 * j) + q;
                    mom_add<R_, Q, true>(mo[j][q], a, S::to_raw(sa[wrap_x(x - EX<Q>(a), g.nx)]));
                }
        }
    } else {
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const T* sa = srow + (size_t)a * dstride;
#pragma unroll
            for (int j = 0; j < NV; ++j)
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int x = xb + P * (lane + 32 * j) + q;
                    mom_add<R_, Q, false>(mo[j][q], a, S::to_raw(sa[wrap_x(x - EX<Q>(a), g.nx)]));
                }
        }
    }
    Coef<R_> cf[NV][P];
#pragma unroll
    for (int j = 0; j < NV; ++j)
#pragma unroll
        for (int q = 0; q < P; ++q) {
            NodeM<R_> m;
            macro_from_moments<R_, Q, EXT>(mo[j][q], p, m);
            coef_of<R_, Q>(m, cf[j][q]);
        }
    // pass 2: relax by pairs and store
#pragma unroll
    for (int k = 0; k <= LatDim<Q>::NP; ++k) {
        const int a = (k == 0) ? 0 : PAIR<Q>(k - 1);
        const int b = (k == 0) ? 0 : OPP<Q>(a);
        const T* sa = srow + (size_t)a * dstride;
        const T* sb = srow + (size_t)b * dstride;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            R_ oa[P], ob[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int x = xb + P * (lane + 32 * j) + q;
                R_ da = S::to_raw(sa[wrap_x(x - EX<Q>(a), g.nx)]);
                if (k == 0) {
                    oa[q] = relax_rest<R_, Q, EXT>(da, cf[j][q], p);
                    ob[q] = R_(0);
                } else {
                    R_ db = S::to_raw(sb[wrap_x(x - EX<Q>(b), g.nx)]);
                    relax_pair<R_, Q, EXT>(a, da, db, cf[j][q], p);
                    oa[q] = da;
                    ob[q] = db;
                }
            }
            if (!spec[j]) {
                const int x = xb + P * (lane + 32 * j);
                if constexpr (P == 2) {
                    union { T t; unsigned short s; } lo, hi;
                    lo.t = S::from_raw(oa[0]);
                    hi.t = S::from_raw(oa[1]);
                    *reinterpret_cast<uint32_t*>(dst + (long long)a * g.sq + rowoff + x) =
                        (uint32_t)lo.s | ((uint32_t)hi.s << 16);
                    if (k > 0) {
                        lo.t = S::from_raw(ob[0]);
                        hi.t = S::from_raw(ob[1]);
                        *reinterpret_cast<uint32_t*>(dst + (long long)b * g.sq + rowoff + x) =
                            (uint32_t)lo.s | ((uint32_t)hi.s << 16);
                    }
                } else {
                    dst[(long long)a * g.sq + rowoff + x] = S::from_raw(oa[0]);
                    if (k > 0) dst[(long long)b * g.sq + rowoff + x] = S::from_raw(ob[0]);
                }
            }
        }
    }
    if (!any) return;
    // slots next to a wall, solid or padding: node by node
#pragma unroll 1
    for (int j = 0; j < NV; ++j) {
        if (!spec[j]) continue;
#pragma unroll 1
        for (int q = 0; q < P; ++q) {
            const int x = xb + P * (lane + 32 * j) + q;
            if (x >= g.nx) continue;
            const uint8_t c = crow[x];
            if (nc_solid(c)) {
#pragma unroll
                for (int a = 0; a < Q; ++a) dst[(long long)a * g.sq + rowoff + x] = S::from_raw(R_(0));
                continue;
            }
            R_ d[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) d[a] = S::to_raw(srow[(size_t)a * dstride + wrap_x(x - EX<Q>(a), g.nx)]);
            if (nc_has_wall(c)) {
#pragma unroll
                for (int a = 1; a < Q; ++a) {
                    long long sidx;
                    int wall;
                    if (!pull_source(g, cls, x, y, z, EX<Q>(a), EY<Q>(a), EZ<Q>(a), sidx, wall)) {
                        const R_ el = R_(EX<Q>(a)) * p.LW[wall][0] + R_(EY<Q>(a)) * p.LW[wall][1] +
                                      R_(EZ<Q>(a)) * p.LW[wall][2];
                        d[a] = S::to_raw(src[(long long)OPP<Q>(a) * g.sq + rowoff + x]) + R_(WD<Q>(a)) * el;
                    }
                }
            }
            NodeM<R_> m;
            node_macro<R_, Q, EXT>(d, p, m);
            node_relax<R_, Q, EXT>(d, p, m);
#pragma unroll
            for (int a = 0; a < Q; ++a) dst[(long long)a * g.sq + rowoff + x] = S::from_raw(d[a]);
        }
    }
}

template <int Q, class S, bool EXT>
__global__ void __launch_bounds__(TILE_THREADS, 1)
k_step_tile(const typename S::T* __restrict__ src, typename S::T* __restrict__ dst,
            const uint8_t* __restrict__ cls, const Geo g, const KP<typename S::R> p, int R, int ntiles,
            int nstages, unsigned* __restrict__ errflag)
{
    using T = typename S::T;
    constexpr int SEG = TileLanes<S>::SEG;
    extern __shared__ __align__(128) unsigned char smem[];
    const size_t stage_bytes = tile_stage_bytes<Q, S>(R, g.nxp);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + nstages * stage_bytes);
    uint64_t* empty = full + nstages;
    const int nty = (g.ny + R - 1) / R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < nstages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TILE_CWARPS);
        }
        mbar_fence_init();
    }
    __syncthreads();
    const int my_tiles = (blockIdx.x < ntiles) ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == TILE_CWARPS) {
        // producer warp: lane 0 refills a stage as soon as all consumer warps released it
        if (lane == 0) {
            int k = 0;
            for (; k < my_tiles; ++k) {
                const int s = k % nstages, use = k / nstages;
                if (use > 0 && !mbar_wait_bounded(&empty[s], (uint32_t)(use - 1) & 1u)) {
                    atomicOr(errflag, ERR_MBAR_TIMEOUT);
                    break;
                }
                tile_issue<Q, S>(src, cls, g, R, nty, blockIdx.x + k * gridDim.x, smem + (size_t)s * stage_bytes,
                                 &full[s]);
            }
            if (k < my_tiles) {
                // stopped early: let the copies already issued land before leaving
                for (int j = (k > nstages ? k - nstages : 0); j < k; ++j)
                    mbar_wait_bounded(&full[j % nstages], (uint32_t)(j / nstages) & 1u);
            }
        }
        return;
    }

    for (int k = 0; k < my_tiles; ++k) {
        const int s = k % nstages, use = k / nstages;
        if (!mbar_wait_bounded(&full[s], (uint32_t)use & 1u)) {
            if (lane == 0) atomicOr(errflag, ERR_MBAR_TIMEOUT);
            mbar_wait_bounded(&full[s], (uint32_t)use & 1u);
            return;
        }
        const int t = blockIdx.x + k * gridDim.x;
        const T* sp = reinterpret_cast<const T*>(smem + (size_t)s * stage_bytes);
        const uint8_t* sc = smem + (size_t)s * stage_bytes + (size_t)Q * R * g.nxp * sizeof(T);
        const int z = t / nty, y0 = (t % nty) * R;
        const int nr = min(R, g.ny - y0);
        const int nseg = (g.nxp + SEG - 1) / SEG;
        for (int sg = warp; sg < nr * nseg; sg += TILE_CWARPS) {
            const int r = sg / nseg;
            const int xb = (sg - r * nseg) * SEG;
            tile_segment<Q, S, EXT>(sp + (size_t)r * g.nxp, sc + (size_t)r * g.nxp, src, dst, cls, g, p, R, xb,
                                    y0 + r, z, lane);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);   // this warp is done with stage s
    }
}

}  // namespace lbm
