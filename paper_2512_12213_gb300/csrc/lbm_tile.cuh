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
// Two stages alternate: while the block computes tile i, the copies of its
// next tile are in flight (mbarrier with transaction count).  Each thread
// then relaxes one node (or a pair of nodes for 16-bit storage) at a time
// and stores the results with coalesced stores.  Nodes next to a wall take
// the bounced populations from their own stored values.
//
// Every mbarrier wait is bounded; on expiry the block records an error flag,
// waits (bounded) for its own copies in flight and returns.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int TILE_THREADS = 256;
constexpr int TILE_STAGES = 2;
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

template <int Q, class S, bool EXT>
__global__ void __launch_bounds__(TILE_THREADS)
k_step_tile(const typename S::T* __restrict__ src, typename S::T* __restrict__ dst,
            const uint8_t* __restrict__ cls, const Geo g, const KP<typename S::R> p, int R, int ntiles,
            unsigned* __restrict__ errflag)
{
    using T = typename S::T;
    using R_ = typename S::R;
    constexpr int P = (sizeof(T) == 2) ? 2 : 1;     // nodes per work item
    extern __shared__ __align__(128) unsigned char smem[];
    const size_t stage_bytes = tile_stage_bytes<Q, S>(R, g.nxp);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + TILE_STAGES * stage_bytes);
    const int nty = (g.ny + R - 1) / R;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TILE_STAGES; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && blockIdx.x < ntiles)
        tile_issue<Q, S>(src, cls, g, R, nty, blockIdx.x, smem, &bars[0]);

    const int per_row = g.nxp / P;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
        const int s = i % TILE_STAGES;
        const int tn = t + gridDim.x;
        if (threadIdx.x == 0 && tn < ntiles)
            tile_issue<Q, S>(src, cls, g, R, nty, tn, smem + (size_t)((i + 1) % TILE_STAGES) * stage_bytes,
                             &bars[(i + 1) % TILE_STAGES]);
        const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)(i / TILE_STAGES) & 1u);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(errflag, ERR_MBAR_TIMEOUT);
                // let this block's copies in flight land before returning
                mbar_wait_bounded(&bars[s], (uint32_t)(i / TILE_STAGES) & 1u);
                if (tn < ntiles) mbar_wait_bounded(&bars[(i + 1) % TILE_STAGES], (uint32_t)((i + 1) / TILE_STAGES) & 1u);
            }
            return;
        }
        const T* sp = reinterpret_cast<const T*>(smem + (size_t)s * stage_bytes);
        const uint8_t* sc = smem + (size_t)s * stage_bytes + (size_t)Q * R * g.nxp * sizeof(T);
        const int z = t / nty, y0 = (t % nty) * R;
        const int nr = min(R, g.ny - y0);
        for (int it = threadIdx.x; it < nr * per_row; it += blockDim.x) {
            const int r = it / per_row;
            const int x = (it - r * per_row) * P;
            const int y = y0 + r;
            const long long rowoff = ((long long)z * g.ny + y) * g.nxp;
            R_ out[P][Q];
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const int xj = x + j;
                const uint8_t c = sc[r * g.nxp + xj];
                if (xj >= g.nx || nc_solid(c) || c == NC_PAD) {
#pragma unroll
                    for (int a = 0; a < Q; ++a) out[j][a] = R_(0);
                    continue;
                }
                R_ d[Q];
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    int xs = xj - EX<Q>(a);
                    xs = (xs < 0) ? g.nx - 1 : (xs >= g.nx ? 0 : xs);
                    d[a] = S::to_r(sp[((size_t)a * R + r) * g.nxp + xs]);
                }
                if (c == NC_BOUND) {
                    // links into a wall: halfway bounce-back of the own stored value
#pragma unroll
                    for (int a = 1; a < Q; ++a) {
                        long long sidx;
                        int wall;
                        if (!pull_source(g, cls, xj, y, z, EX<Q>(a), EY<Q>(a), EZ<Q>(a), sidx, wall)) {
                            const R_ el = R_(EX<Q>(a)) * p.LW[wall][0] + R_(EY<Q>(a)) * p.LW[wall][1] +
                                          R_(EZ<Q>(a)) * p.LW[wall][2];
                            d[a] = S::to_r(src[(long long)OPP<Q>(a) * g.sq + rowoff + xj]) + R_(WD<Q>(a)) * el;
                        }
                    }
                }
                NodeM<R_> m;
                node_macro<R_, Q, EXT>(d, p, m);
                node_relax<R_, Q, EXT>(d, p, m);
#pragma unroll
                for (int a = 0; a < Q; ++a) out[j][a] = d[a];
            }
            if constexpr (P == 2) {
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    union { T t; unsigned short s; } lo, hi;
                    lo.t = S::from_r(out[0][a]);
                    hi.t = S::from_r(out[1][a]);
                    *reinterpret_cast<uint32_t*>(dst + (long long)a * g.sq + rowoff + x) =
                        (uint32_t)lo.s | ((uint32_t)hi.s << 16);
                }
            } else {
#pragma unroll
                for (int a = 0; a < Q; ++a) dst[(long long)a * g.sq + rowoff + x] = S::from_r(out[0][a]);
            }
        }
        __syncthreads();   // stage s is free for the copies of tile t + 2 * gridDim.x
    }
}

}  // namespace lbm
