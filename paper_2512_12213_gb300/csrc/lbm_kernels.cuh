// lbm_kernels.cuh -- CUDA kernels of the lattice Boltzmann hot path
// (arXiv 2512.12213) and their launchers, templated on the lattice (Q), the
// population storage format (S) and EXT (Lorentz force, Maxwell equilibrium
// or LES present).  Instantiated per storage format in inst_*.cu.
#pragma once

#include <algorithm>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_staged.cuh"

namespace lbm {

constexpr int STEP_THREADS = 128;
constexpr int NODE_THREADS = 256;
// blocks of NODE_THREADS per SM for the coupled field step: FP32 compute 3
// (85 registers, no spill), FP64 2
template <class S> struct MhdOcc {
    static constexpr int value = sizeof(typename S::R) == 8 ? 2 : 3;
};
constexpr int RED_THREADS = 256;

// ------------------------------------------------------------ warp helpers
template <class T> union Bits16 {
    T t;
    unsigned short s;
};
template <class T> __device__ __forceinline__ T shfl_up1(T v)
{
    if constexpr (sizeof(T) == 2) {
        Bits16<T> b;
        b.t = v;
        b.s = (unsigned short)__shfl_up_sync(0xffffffffu, (unsigned)b.s, 1);
        return b.t;
    } else {
        return __shfl_up_sync(0xffffffffu, v, 1);
    }
}
template <class T> __device__ __forceinline__ T shfl_down1(T v)
{
    if constexpr (sizeof(T) == 2) {
        Bits16<T> b;
        b.t = v;
        b.s = (unsigned short)__shfl_down_sync(0xffffffffu, (unsigned)b.s, 1);
        return b.t;
    } else {
        return __shfl_down_sync(0xffffffffu, v, 1);
    }
}

// sum W doubles over the block; thread 0 gets the totals in out[]
template <int W>
__device__ __forceinline__ void block_sum(double (&v)[W], double* smem /* >= W * 32 */)
{
#pragma unroll
    for (int k = 0; k < W; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < W; ++k) smem[k * 32 + wid] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < W; ++k) {
            double s = (lane < nw) ? smem[k * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            v[k] = s;
        }
    }
}

// ------------------------------------------------- fused collide-stream step
// One thread owns V consecutive nodes of a row (one 16-byte vector per
// direction).  For every direction it loads the aligned vector of the pull
// source row; the x-shifted directions take their edge element from the
// neighbouring lane (warp shuffle), or from one scalar load at a row edge or
// warp edge.  16-bit formats stay packed two to a register (the x shift is a
// byte permute) and are relaxed two nodes at a time.  A chunk that holds a
// boundary, solid or padding node is recomputed node by node with explicit
// bounce-back.  Populations are in storage units (kernel parameters scaled
// to match).
// blocks of 128 threads per SM the register allocation must allow: FP64 3
// (168 registers), else 4 (128; for 16-bit storage measured faster than 5
// blocks at 96 registers, which spill with the FP32x2 node pairs)
// (the EXT node code in FP32x2 node pairs, 32-bit storage with closed faces:
// 3, where it needs 158 registers without spill)
template <class S, bool EXT, bool FACES = false, bool FULL = false, bool LP = false> struct StepOcc {
    static constexpr bool PAIRX = EXT && !FULL && !LP && FACES && sizeof(typename S::T) == 4;
    static constexpr int value = (sizeof(typename S::T) == 8 || PAIRX) ? 3 : 4;
};

// FULL: the boundary path interpolates at walls off the half-grid and the
// EXT node code reads the Lorentz coefficient of insulating walls from the
// device and sums the flow velocity (contexts with a wall distance or
// insulating walls).  Kept out of the other instantiations: even as one
// out-of-line call the interpolation cost the fused step ~3% (inlined ~5%),
// and the insulating-wall code cost the LES cavity 8%.
// LP: the LES-only contexts with 16-bit storage (Smagorinsky with a uniform
// body force and no other EXT term) relax their all-fluid chunks with the
// FP32x2 pair code specialised for LES; chunks with a wall keep the scalar
// EXT node code.
template <int Q, class S, bool EXT, bool FACES, bool SR, bool FULL = false, bool LP = false>
__global__ void __launch_bounds__(STEP_THREADS, StepOcc<S, EXT, FACES, FULL, LP>::value)
k_step(const typename S::T* __restrict__ src, typename S::T* __restrict__ dst,
       const uint8_t* __restrict__ cls, const Geo g, const KP<typename S::R> p, uint32_t seed)
{
    using T = typename S::T;
    using R = typename S::R;
    constexpr int V = S::V;
    constexpr bool PACKED = sizeof(T) == 2;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int ncx = g.nxp / V;
    const long long nch = (long long)ncx * g.ny * g.nz;
    const bool active = tid < nch;
    const long long ch = active ? tid : nch - 1;
    const int cx = (int)(ch % ncx);
    const long long row = ch / ncx;
    const int y = (int)(row % g.ny);
    const int z = (int)(row / g.ny);
    const int x0 = cx * V;

    // class bytes of the chunk: fast path if all are bulk (or, with FACES, face)
    bool special, face_chunk = false;
    {
        const uint8_t* cp = cls + row * g.nxp + x0;
        unsigned long long cb;
        if constexpr (V == 8) {
            const uint2 cv = *reinterpret_cast<const uint2*>(cp);
            cb = ((unsigned long long)cv.y << 32) | cv.x;
        } else if constexpr (V == 4) {
            cb = *reinterpret_cast<const uint32_t*>(cp);
        } else {
            cb = *reinterpret_cast<const uint16_t*>(cp);
        }
        if (FACES) {
            special = (cb & ~0x0202020202020202ull) != 0ull;
            face_chunk = (cb & 0x0202020202020202ull) != 0ull;
        } else {
            special = cb != 0ull;
        }
    }
    FaceInfo fi;
    if (FACES) {
        fi.closed_x = !g.periodic[0];
        fi.yo_lo = !g.periodic[1] && y == 0;
        fi.yo_hi = !g.periodic[1] && y == g.ny - 1;
        fi.zo_lo = (Q == 19) && !g.periodic[2] && z == 0;
        fi.zo_hi = (Q == 19) && !g.periodic[2] && z == g.nz - 1;
        fi.wx_lo = g.face_wall[0]; fi.wx_hi = g.face_wall[1];
        fi.wy_lo = g.face_wall[2]; fi.wy_hi = g.face_wall[3];
        fi.wz_lo = g.face_wall[4]; fi.wz_hi = g.face_wall[5];
    }
    // row offsets of the pull sources, by (E_y, E_z)
    long long roff[3][3];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            const int ys = wrapi(y - dy, g.ny);
            const int zs = (Q == 19) ? wrapi(z - dz, g.nz) : 0;
            roff[dy + 1][dz + 1] = ((long long)zs * g.ny + ys) * g.nxp;
        }
    const long long own = row * g.nxp;

    using RawT = typename RawVec<sizeof(T) * V>::type;
    // shifted source values: packed words for 16-bit formats, else elements
    uint32_t w[Q][PACKED ? V / 2 : 1];
    T f[Q][PACKED ? 1 : V];
    if constexpr (!FACES) {
        // periodic box: per direction, vector load, shuffle, and a scalar load
        // at the warp or row edge (measured faster here than the split order
        // of the closed-face variant)
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const T* rp = src + (long long)a * g.sq + roff[EY<Q>(a) + 1][EZ<Q>(a) + 1];
            VecN<T, V> raw;
            raw.raw = __ldg(reinterpret_cast<const RawT*>(rp + x0));
            const int ex = EX<Q>(a);
            T edge = raw.e[0];
            // periodic x: the wrap of a row edge and the warp edge are plain loads
            if (EX<Q>(a) == 1) {
                edge = shfl_up1(raw.e[V - 1]);
                if (lane == 0 || cx == 0) edge = rp[cx == 0 ? g.nx - 1 : x0 - 1];
            } else if (EX<Q>(a) == -1) {
                edge = shfl_down1(raw.e[0]);
                if (lane == 31 || x0 + V >= g.nx) edge = rp[x0 + V >= g.nx ? 0 : x0 + V];
            }
            if constexpr (PACKED) {
                const uint32_t* rw = raw.u;
                Bits16<T> eb;
                eb.t = edge;
                const uint32_t ew = (uint32_t)eb.s;
                if (ex == 0) {
#pragma unroll
                    for (int i = 0; i < V / 2; ++i) w[a][i] = rw[i];
                } else if (ex == 1) {             // value k <- raw k-1
                    w[a][0] = __byte_perm(ew, rw[0], 0x5410);
#pragma unroll
                    for (int i = 1; i < V / 2; ++i) w[a][i] = __byte_perm(rw[i - 1], rw[i], 0x5432);
                } else {                           // value k <- raw k+1
#pragma unroll
                    for (int i = 0; i < V / 2 - 1; ++i) w[a][i] = __byte_perm(rw[i], rw[i + 1], 0x5432);
                    w[a][V / 2 - 1] = __byte_perm(rw[V / 2 - 1], ew, 0x5432);
                }
            } else {
                if (ex == 0) {
#pragma unroll
                    for (int k = 0; k < V; ++k) f[a][k] = raw.e[k];
                } else if (ex == 1) {
                    f[a][0] = edge;
#pragma unroll
                    for (int k = 1; k < V; ++k) f[a][k] = raw.e[k - 1];
                } else {
#pragma unroll
                    for (int k = 0; k < V - 1; ++k) f[a][k] = raw.e[k + 1];
                    f[a][V - 1] = edge;
                }
            }
        }
    } else {
        // closed faces: all vector loads first, then the edge-element loads,
        // and only then the shuffles that wait for them (one memory round trip)
        auto row_ptr = [&](int a, bool rout) -> const T* {
            // bounced rows read the node's own value of the opposite direction
            return rout ? src + (long long)OPP<Q>(a) * g.sq + own
                        : src + (long long)a * g.sq + roff[EY<Q>(a) + 1][EZ<Q>(a) + 1];
        };
        VecN<T, V> raw[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            int rwall = 0;
            const bool rout = row_out<Q>(fi, a, rwall);
            raw[a].raw = __ldg(reinterpret_cast<const RawT*>(row_ptr(a, rout) + x0));
        }
        // lanes at a warp edge or a row edge load the element the shuffle
        // cannot give them: the left neighbour of x0 (E_x = +1) or the right
        // neighbour of x0 + V - 1 (E_x = -1), wrapped on a periodic x axis, or
        // the node's own opposite population at a closed x face
        const bool needL = (lane == 0 || cx == 0), needR = (lane == 31 || x0 + V >= g.nx);
        T eload[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            eload[a] = raw[a].e[0];
            int rwall = 0;
            const bool rout = row_out<Q>(fi, a, rwall);
            const T* rp = row_ptr(a, rout);
            if (EX<Q>(a) == 1 && !rout && needL) {
                if (cx == 0 && fi.closed_x) eload[a] = src[(long long)OPP<Q>(a) * g.sq + own];
                else eload[a] = rp[cx == 0 ? g.nx - 1 : x0 - 1];
            } else if (EX<Q>(a) == -1 && !rout && needR) {
                if (x0 + V >= g.nx && fi.closed_x) eload[a] = src[(long long)OPP<Q>(a) * g.sq + own + g.nx - 1];
                else eload[a] = rp[x0 + V >= g.nx ? 0 : x0 + V];
            }
        }
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            int rwall = 0;
            const bool rout = row_out<Q>(fi, a, rwall);
            const int ex = rout ? 0 : EX<Q>(a);
            T edge = raw[a].e[0];
            if (EX<Q>(a) == 1) {
                edge = shfl_up1(raw[a].e[V - 1]);
                if (needL) edge = eload[a];
            } else if (EX<Q>(a) == -1) {
                edge = shfl_down1(raw[a].e[0]);
                if (needR) edge = eload[a];
            }
            if constexpr (PACKED) {
                const uint32_t* rw = raw[a].u;
                Bits16<T> eb;
                eb.t = edge;
                const uint32_t ew = (uint32_t)eb.s;
                if (ex == 0) {
#pragma unroll
                    for (int i = 0; i < V / 2; ++i) w[a][i] = rw[i];
                } else if (ex == 1) {             // value k <- raw k-1
                    w[a][0] = __byte_perm(ew, rw[0], 0x5410);
#pragma unroll
                    for (int i = 1; i < V / 2; ++i) w[a][i] = __byte_perm(rw[i - 1], rw[i], 0x5432);
                } else {                           // value k <- raw k+1
#pragma unroll
                    for (int i = 0; i < V / 2 - 1; ++i) w[a][i] = __byte_perm(rw[i], rw[i + 1], 0x5432);
                    w[a][V / 2 - 1] = __byte_perm(rw[V / 2 - 1], ew, 0x5432);
                }
            } else {
                if (ex == 0) {
#pragma unroll
                    for (int k = 0; k < V; ++k) f[a][k] = raw[a].e[k];
                } else if (ex == 1) {
                    f[a][0] = edge;
#pragma unroll
                    for (int k = 1; k < V; ++k) f[a][k] = raw[a].e[k - 1];
                } else {
#pragma unroll
                    for (int k = 0; k < V - 1; ++k) f[a][k] = raw[a].e[k + 1];
                    f[a][V - 1] = edge;
                }
            }
        }
    }
    // only the velocity rows of insulating walls need the lanes past the last chunk
    if (!(EXT && FULL) && !active) return;
    // insulating walls: this thread's sum of the flow velocity v over the
    // fluid nodes it relaxes, summed over the warp by a fixed shuffle tree in
    // FP64 (every thread of the block reaches it, inactive ones with zero),
    // one row per warp for the fixed-order reduction of the field
    R vs[3] = {R(0), R(0), R(0)};
    auto add_v = [&](const NodeM<R>& m) {
        if constexpr (EXT && FULL) {
            vs[0] += m.v[0];
            vs[1] += m.v[1];
            vs[2] += m.v[2];
        }
    };
    auto put_v = [&]() {
        if constexpr (EXT && FULL) {
            if (p.ins_rows) {
                double t[3] = {(double)vs[0], (double)vs[1], (double)vs[2]};
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int k = 0; k < 3; ++k) t[k] += __shfl_down_sync(0xffffffffu, t[k], o);
                if (lane == 0)
#pragma unroll
                    for (int k = 0; k < 3; ++k) p.ins_rows[(tid >> 5) * 3 + k] = t[k];
            }
        }
    };
    if (active) {

        // Ladd terms of moving face walls, added after unpacking (face chunks only)
        const bool ladd = FACES && face_chunk && p.face_ladd;
        auto add_ladd = [&](R (&d)[Q], int k) {
#pragma unroll
            for (int a = 1; a < Q; ++a) {
                int wall = 0;
                bool hit = row_out<Q>(fi, a, wall);
                if (fi.closed_x) {
                    if (EX<Q>(a) == 1 && x0 + k == 0) { hit = true; wall = fi.wx_lo; }
                    if (EX<Q>(a) == -1 && x0 + k == g.nx - 1) { hit = true; wall = fi.wx_hi; }
                }
                if (hit) d[a] += ladd_of<Q, R>(p, a, wall);
            }
        };

        // the same for two consecutive nodes k, k+1 held as pairs
        auto add_ladd2 = [&](F2 (&d)[Q], int k) {
#pragma unroll
            for (int a = 1; a < Q; ++a) {
                int wall = 0;
                const bool hit = row_out<Q>(fi, a, wall);
                int w0 = wall, w1 = wall;
                bool h0 = hit, h1 = hit;
                if (fi.closed_x) {
                    if (EX<Q>(a) == 1 && x0 + k == 0) { h0 = true; w0 = fi.wx_lo; }
                    if (EX<Q>(a) == -1 && x0 + k == g.nx - 1) { h0 = true; w0 = fi.wx_hi; }
                    if (EX<Q>(a) == -1 && x0 + k + 1 == g.nx - 1) { h1 = true; w1 = fi.wx_hi; }
                }
                if (h0) d[a].v.x += ladd_of<Q, R>(p, a, w0);
                if (h1) d[a].v.y += ladd_of<Q, R>(p, a, w1);
            }
        };
        // two nodes at a time in packed FP32x2 arithmetic (FP32 compute without
        // the Lorentz force, Maxwell term or LES)
        constexpr bool PAIR2 = (!EXT || LP) && sizeof(R) == 4;
    // the EXT node code in node pairs too: FP32 storage with closed faces (the
    // LES cavity 24.7k -> 26.6k MLUPS); measured slower for 16-bit storage
    // (-3.7%) and periodic FP32 boxes (-2.5%, spills), which keep the scalar code
    constexpr bool PAIRX = StepOcc<S, EXT, FACES, FULL, LP>::PAIRX;

        const long long base = row * g.nxp + x0;
        if (!special) {
            if constexpr (PACKED && (PAIR2 || PAIRX)) {
#pragma unroll
                for (int i = 0; i < V / 2; ++i) {
                    F2 dd[Q];
#pragma unroll
                    for (int a = 0; a < Q; ++a) dd[a] = F2{S::unpack2(w[a][i])};
                    if (ladd) add_ladd2(dd, 2 * i);
                    if constexpr (PAIR2) pair_collide<Q, LP, true>(dd, p);
                    else pair_collide_ext<Q>(dd, p);
                    if constexpr (SR) {
                        NodeRng rp((uint32_t)(base + 2 * i), seed);     // the pair's first node
#pragma unroll
                        for (int a = 0; a < Q; ++a) w[a][i] = S::pack2_sr(dd[a].v.x, dd[a].v.y, rp.word());
                    } else {
#pragma unroll
                        for (int a = 0; a < Q; ++a) w[a][i] = S::pack2(dd[a].v.x, dd[a].v.y);
                    }
                }
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    VecN<T, V> o;
#pragma unroll
                    for (int i = 0; i < V / 2; ++i) o.u[i] = w[a][i];
                    *reinterpret_cast<typename RawVec<sizeof(T) * V>::type*>(dst + (long long)a * g.sq + base) = o.raw;
                }
            } else if constexpr (PACKED) {
                // two nodes per packed word: unpack both, relax them, pack both
                // with one conversion
#pragma unroll
                for (int i = 0; i < V / 2; ++i) {
                    R d0[Q], d1[Q];
#pragma unroll
                    for (int a = 0; a < Q; ++a) {
                        const float2 v = S::unpack2(w[a][i]);
                        d0[a] = v.x;
                        d1[a] = v.y;
                    }
                    if (ladd) {
                        add_ladd(d0, 2 * i);
                        add_ladd(d1, 2 * i + 1);
                    }
                    {
                        NodeM<R> m;
                        node_macro<R, Q, EXT, FULL>(d0, p, m);
                        node_relax<R, Q, EXT>(d0, p, m);
                        add_v(m);
                    }
                    {
                        NodeM<R> m;
                        node_macro<R, Q, EXT, FULL>(d1, p, m);
                        node_relax<R, Q, EXT>(d1, p, m);
                        add_v(m);
                    }
                    if constexpr (SR) {
                        NodeRng rp((uint32_t)(base + 2 * i), seed);     // the pair's first node
#pragma unroll
                        for (int a = 0; a < Q; ++a) w[a][i] = S::pack2_sr(d0[a], d1[a], rp.word());
                    } else {
#pragma unroll
                        for (int a = 0; a < Q; ++a) w[a][i] = S::pack2(d0[a], d1[a]);
                    }
                }
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    VecN<T, V> o;
#pragma unroll
                    for (int i = 0; i < V / 2; ++i) o.u[i] = w[a][i];
                    *reinterpret_cast<typename RawVec<sizeof(T) * V>::type*>(dst + (long long)a * g.sq + base) = o.raw;
                }
            } else {
                if constexpr (PAIRX) {
                    // the EXT node code in node pairs, as a rolled queue of pairs
#pragma unroll 1
                    for (int k = 0; k < V / 2; ++k) {
                        F2 dd[Q];
#pragma unroll
                        for (int a = 0; a < Q; ++a) dd[a] = F2{make_float2(S::to_raw(f[a][0]), S::to_raw(f[a][1]))};
                        if (ladd) add_ladd2(dd, 2 * k);
                        pair_collide_ext<Q>(dd, p);
#pragma unroll
                        for (int a = 0; a < Q; ++a) {
#pragma unroll
                            for (int j = 0; j < V - 2; ++j) f[a][j] = f[a][j + 2];
                            f[a][V - 2] = S::from_raw(dd[a].v.x);
                            f[a][V - 1] = S::from_raw(dd[a].v.y);
                        }
                    }
                } else if constexpr (EXT && !LP) {
                    // larger node code (Lorentz / Maxwell / LES): the same rolled queue
#pragma unroll 1
                    for (int k = 0; k < V; ++k) {
                        R d[Q];
#pragma unroll
                        for (int a = 0; a < Q; ++a) d[a] = S::to_raw(f[a][0]);
                        if (ladd) add_ladd(d, k);
                        NodeM<R> m;
                        node_macro<R, Q, EXT, FULL>(d, p, m);
                        node_relax<R, Q, EXT>(d, p, m);
                        add_v(m);
#pragma unroll
                        for (int a = 0; a < Q; ++a) {
#pragma unroll
                            for (int j = 0; j < V - 1; ++j) f[a][j] = f[a][j + 1];
                            f[a][V - 1] = S::from_raw(d[a]);
                        }
                    }
                } else if constexpr (PAIR2) {
#pragma unroll
                    for (int i = 0; i < V / 2; ++i) {
                        F2 dd[Q];
#pragma unroll
                        for (int a = 0; a < Q; ++a) dd[a] = F2{make_float2(S::to_raw(f[a][2 * i]), S::to_raw(f[a][2 * i + 1]))};
                        if (ladd) add_ladd2(dd, 2 * i);
                        pair_collide<Q, LP>(dd, p);
#pragma unroll
                        for (int a = 0; a < Q; ++a) {
                            f[a][2 * i] = S::from_raw(dd[a].v.x);
                            f[a][2 * i + 1] = S::from_raw(dd[a].v.y);
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < V; ++k) {
                        R d[Q];
#pragma unroll
                        for (int a = 0; a < Q; ++a) d[a] = S::to_raw(f[a][k]);
                        if (ladd) add_ladd(d, k);
                        NodeM<R> m;
                        node_macro<R, Q, EXT, FULL>(d, p, m);
                        node_relax<R, Q, EXT>(d, p, m);
#pragma unroll
                        for (int a = 0; a < Q; ++a) f[a][k] = S::from_raw(d[a]);
                    }
                }
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    VecN<T, V> o;
#pragma unroll
                    for (int k = 0; k < V; ++k) o.e[k] = f[a][k];
                    *reinterpret_cast<typename RawVec<sizeof(T) * V>::type*>(dst + (long long)a * g.sq + base) = o.raw;
                }
            }
        } else {
            // chunk with a solid neighbour or padding: node by node
            for (int k = 0; k < V; ++k) {
                const int x = x0 + k;
                const uint8_t c = cls[base + k];
                if (x >= g.nx || nc_solid(c) || c == NC_PAD) {
#pragma unroll
                    for (int a = 0; a < Q; ++a) dst[(long long)a * g.sq + base + k] = S::from_raw(R(0));
                    continue;
                }
                R d[Q];
                gather_node<Q, S, true, FULL>(src, cls, g, p, x, y, z, d);
                NodeM<R> m;
                node_macro<R, Q, EXT, FULL>(d, p, m);
                node_relax<R, Q, EXT>(d, p, m);
                add_v(m);
                if constexpr (SR) {
                    NodeRng rng((uint32_t)(base + k), seed);
#pragma unroll
                    for (int a = 0; a < Q; ++a) dst[(long long)a * g.sq + base + k] = S::from_raw_sr(d[a], rng.bits(a));
                } else {
#pragma unroll
                    for (int a = 0; a < Q; ++a) dst[(long long)a * g.sq + base + k] = S::from_raw(d[a]);
                }
            }
        }
    }
    put_v();
}

// ------------------------------------------ inverse propagation (import/init)
// Stored state P with gather(P) = the given canonical f: P_a(y) = f_a(y + E_a)
// if y + E_a is fluid, else f_opp(a)(y) - (Ladd term of opp(a)).
struct SrcCanonD { const double* f; long long N; };
struct SrcCanonF { const float* f; long long N; };
struct SrcFields { const double* rho; const double* u; const double* xi; long long N; };

template <int Q, typename R>
__device__ __forceinline__ R src_value(const SrcCanonD& s, const KP<R>& p, int a, long long n)
{
    return R(s.f[(long long)a * s.N + n] - WD<Q>(a) * (double)p.rho0);
}
template <int Q, typename R>
__device__ __forceinline__ R src_value(const SrcCanonF& s, const KP<R>& p, int a, long long n)
{
    return R((double)s.f[(long long)a * s.N + n] - WD<Q>(a) * (double)p.rho0);
}
// Eq. (1) (+ Eq. 10) evaluated in double from the fields, times (1 + xi)
template <int Q, typename R>
__device__ __forceinline__ R src_value(const SrcFields& s, const KP<R>& p, int a, long long n)
{
    const double c = (double)p.c;
    const double rho = s.rho[n];
    const double W[3] = {s.u[n] / c, s.u[s.N + n] / c, (Q == 19) ? s.u[2 * s.N + n] / c : 0.0};
    const double eu = EX<Q>(a) * W[0] + EY<Q>(a) * W[1] + EZ<Q>(a) * W[2];
    const double ww = W[0] * W[0] + W[1] * W[1] + W[2] * W[2];
    double fe = p.stokes ? rho * WD<Q>(a) * (1.0 + 3.0 * eu) : rho * WD<Q>(a) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * ww);
    if (p.maxwell) fe += (double)p.mx[a];
    if (s.xi) fe *= 1.0 + s.xi[(long long)a * s.N + n];
    return R(fe - WD<Q>(a) * (double)p.rho0);
}

// canonical index of a fluid node given by its padded index
__device__ __forceinline__ long long canon_of(const Geo& g, long long padded)
{
    const int xs = (int)(padded % g.nxp);
    return (padded / g.nxp) * g.nx + xs;
}

// The stored value P_a(x) of a link a that leaves fluid node x (padded own,
// canonical nd) into a wall, such that the bounced population of opp(a) at x
// (see bounced) is the given f_opp(a)(x): the inverse of the halfway or
// interpolated rule.  Every case is explicit except both opposite links of
// x hitting solids with q >= 1/2, a 2 x 2 solve.
template <int Q, typename R, class Src>
__device__ R unbounced(const Src& s, const KP<R>& p, const Geo& g, const uint8_t* __restrict__ cls, int x, int y, int z,
                       long long own, long long nd, int a, int wall)
{
    const int b = OPP<Q>(a);
    const R Lb = R(WD<Q>(b)) * (R(EX<Q>(b)) * p.LW[wall][0] + R(EY<Q>(b)) * p.LW[wall][1] + R(EZ<Q>(b)) * p.LW[wall][2]);
    const R fb = src_value<Q, R>(s, p, b, nd);
    const R half = fb - Lb;
    if (!g.phi) return half;
    const long long sa = link_target(g, x, y, z, EX<Q>(a), EY<Q>(a), EZ<Q>(a));
    if (sa < 0 || !nc_solid(cls[sa])) return half;               // a closed box face
    const R qa = R(g.phi[own]) / (R(g.phi[own]) - R(g.phi[sa]));
    long long nb;
    int wb;
    const bool b_fluid = pull_source(g, cls, x, y, z, EX<Q>(a), EY<Q>(a), EZ<Q>(a), nb, wb);   // x + E_b = x - E_a
    if (qa < R(0.5)) {
        if (!b_fluid) return half;
        const R fa = src_value<Q, R>(s, p, a, nd);                // = P_a(x - E_a)
        return (fb - Lb - (R(1) - R(2) * qa) * fa) / (R(2) * qa);
    }
    R Pb;
    if (b_fluid) {
        Pb = src_value<Q, R>(s, p, b, canon_of(g, nb));           // node x + E_b pulls b from x
        return R(2) * qa * fb - (R(2) * qa - R(1)) * Pb - Lb;
    }
    // the link b of x hits a wall too (wall id wb)
    const R La = R(WD<Q>(a)) * (R(EX<Q>(a)) * p.LW[wb][0] + R(EY<Q>(a)) * p.LW[wb][1] + R(EZ<Q>(a)) * p.LW[wb][2]);
    const R fa = src_value<Q, R>(s, p, a, nd);
    const long long sb = link_target(g, x, y, z, EX<Q>(b), EY<Q>(b), EZ<Q>(b));
    const R qb = (sb >= 0 && nc_solid(cls[sb])) ? R(g.phi[own]) / (R(g.phi[own]) - R(g.phi[sb])) : R(0.5);
    if (qb < R(0.5) || !(sb >= 0 && nc_solid(cls[sb]))) {
        // b bounces halfway (its second node x + E_a is the solid, or a face)
        Pb = fa - La;
        return R(2) * qa * fb - (R(2) * qa - R(1)) * Pb - Lb;
    }
    const R A1 = R(2) * qa * fb - Lb, k1 = R(2) * qa - R(1);
    const R A2 = R(2) * qb * fa - La, k2 = R(2) * qb - R(1);
    return (A1 - k1 * A2) / (R(1) - k1 * k2);
}

template <int Q, class S, class Src>
__global__ void __launch_bounds__(NODE_THREADS)
k_inverse_stream(typename S::T* __restrict__ P, const uint8_t* __restrict__ cls, const Geo g,
                 const KP<typename S::R> p, const Src s)
{
    using R = typename S::R;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < (long long)g.nxp * g.ny * g.nz;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % g.nxp);
        const long long r = n / g.nxp;
        const int y = (int)(r % g.ny), z = (int)(r / g.ny);
        const uint8_t c = cls[n];
        if (x >= g.nx || nc_solid(c) || c == NC_PAD) {
#pragma unroll
            for (int a = 0; a < Q; ++a) P[(long long)a * g.sq + n] = S::from_r(R(0));
            continue;
        }
        const long long nd = ((long long)z * g.ny + y) * g.nx + x;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            // the link from y along a is the pull source of direction opp(a) at y
            long long srcp;
            int wall;
            R val;
            if (a == 0) {
                val = src_value<Q, R>(s, p, 0, nd);
            } else if (pull_source(g, cls, x, y, z, EX<Q>(OPP<Q>(a)), EY<Q>(OPP<Q>(a)), EZ<Q>(OPP<Q>(a)), srcp, wall)) {
                const int xs = (int)(srcp % g.nxp);
                const long long rs = srcp / g.nxp;
                const long long ns = rs * g.nx + xs;
                val = src_value<Q, R>(s, p, a, ns);
            } else {
                val = unbounced<Q, R>(s, p, g, cls, x, y, z, n, nd, a, wall);
            }
            P[(long long)a * g.sq + n] = S::from_r(val);
        }
    }
}

// ---------------------------------------------------------------- export
template <int Q, class S, typename OutT>
__global__ void __launch_bounds__(NODE_THREADS)
k_export(const typename S::T* __restrict__ P, const uint8_t* __restrict__ cls, const Geo g,
         const KP<typename S::R> p, OutT* __restrict__ out)
{
    using R = typename S::R;
    const long long N = (long long)g.nx * g.ny * g.nz;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % g.nx);
        const long long r = n / g.nx;
        const int y = (int)(r % g.ny), z = (int)(r / g.ny);
        const uint8_t c = cls[r * g.nxp + x];
        if (nc_solid(c)) {
#pragma unroll
            for (int a = 0; a < Q; ++a) out[(long long)a * N + n] = OutT(0);
            continue;
        }
        R d[Q];
        gather_node<Q, S>(P, cls, g, p, x, y, z, d);
#pragma unroll
        for (int a = 0; a < Q; ++a) out[(long long)a * N + n] = OutT((double)d[a] + WD<Q>(a) * (double)p.rho0);
    }
}

// ------------------------------------------------------------- wall force
// One thread per boundary link (x_f, a') of one wall: fbar_a' = P_a'(x_f)
// = f^rel(x_f, T-1), fbar_a = f_opp(a')(x_f, T), the bounced population
// (halfway: fbar_a' - w E_a'.LW; interpolated with a wall distance).
// Per link (dx^D/dt) [e_a' (fbar_a' + fbar_a) + corrections], in FP64.
template <int Q, class S>
__global__ void __launch_bounds__(RED_THREADS)
k_links(const typename S::T* __restrict__ P, const uint8_t* __restrict__ cls, const Link* __restrict__ links,
        long long begin, long long end, const Geo g, const KP<typename S::R> p, unsigned flags,
        double* __restrict__ partials)
{
    __shared__ double sm[3 * 32];
    double acc[3] = {0.0, 0.0, 0.0};
    const double c = (double)p.c, rho0 = (double)p.rho0, svol = (double)p.svol;
    for (long long i = begin + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < end;
         i += (long long)gridDim.x * blockDim.x) {
        const Link L = links[i];
        const int a = L.dir;
        double e[3], w = 0.0;
        double fo = 0.0;
        // direction tables by a small switch (a is data here)
#pragma unroll
        for (int b = 1; b < Q; ++b)
            if (b == a) {
                e[0] = EX<Q>(b); e[1] = EY<Q>(b); e[2] = EZ<Q>(b);
                w = WD<Q>(b);
            }
        fo = (double)S::to_r(P[(long long)a * g.sq + L.node]) + w * rho0;
        // bounced population f_opp(a')(x_f, T)
        const int xn = (int)(L.node % g.nxp);
        const long long rn = L.node / g.nxp;
        const int yn = (int)(rn % g.ny), zn = (int)(rn / g.ny);
        double fi = 0.0;
#pragma unroll
        for (int b = 1; b < Q; ++b)
            if (OPP<Q>(b) == a) fi = (double)bounced<Q, S, false>(P, cls, g, p, xn, yn, zn, L.node, b, L.wall) + w * rho0;
        double mxa = 0.0;
        if ((flags & 2u) && p.maxwell) {
            if (p.induced) {
                // the field of the collision that produced f^rel(x_f, T-1)
                typename S::R B[3];
                mag_field_at<Q>(p.mag, cls, g, p, xn, yn, zn, (long long)L.node, B);
#pragma unroll
                for (int b = 1; b < Q; ++b)
                    if (b == a) mxa = (double)maxwell_at<Q>(p.mxk, B, b);
            } else {
#pragma unroll
                for (int b = 1; b < Q; ++b)
                    if (b == a) mxa = (double)p.mx[b];
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double ek = c * e[k];
            double t = ek * (fo + fi);
            if (flags & 1u) t += (double)p.LW[L.wall][k] * c / (6.0 * rho0) * (fi - fo);
            if (flags & 2u) t -= 2.0 * ek * mxa;
            acc[k] += svol * t;
        }
    }
    block_sum<3>(acc, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) partials[(long long)blockIdx.x * 3 + k] = acc[k];
}

// ---------------------------------------------------------------- balance
template <int Q, class S, bool EXT>
__global__ void __launch_bounds__(RED_THREADS)
k_balance(const typename S::T* __restrict__ P, const uint8_t* __restrict__ cls, const Geo g,
          const KP<typename S::R> p, double vol, double* __restrict__ partials)
{
    using R = typename S::R;
    __shared__ double sm[7 * 32];
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const long long N = (long long)g.nx * g.ny * g.nz;
    const double c = (double)p.c;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % g.nx);
        const long long r = n / g.nx;
        const int y = (int)(r % g.ny), z = (int)(r / g.ny);
        if (nc_solid(cls[r * g.nxp + x])) continue;
        R d[Q];
        gather_node<Q, S>(P, cls, g, p, x, y, z, d);
        double dr = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const double da = (double)d[a];
            dr += da;
            jx += EX<Q>(a) * da;
            jy += EY<Q>(a) * da;
            jz += EZ<Q>(a) * da;
        }
        NodeM<R> m;
        node_macro<R, Q, EXT>(d, p, m);
        const double rho = (double)p.rho0 + dr;
        acc[0] += vol * rho;
        acc[1] += vol * c * jx;
        acc[2] += vol * c * jy;
        acc[3] += vol * c * jz;
        // rho a = rho (c/dt) A
        for (int k = 0; k < 3; ++k) acc[4 + k] += vol * rho * (c / (double)p.dt) * (double)m.A[k];
    }
    block_sum<7>(acc, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < 7; ++k) partials[(long long)blockIdx.x * 7 + k] = acc[k];
}

// ------------------------------------------------------- steady residual
// Sec. 6: the balance of Eq. (32) between wall force and body force holds
// once the flow stops changing.  Per fluid node of f(T): the flow velocity
// v = c (j/rho + A/2) (text after Eq. 1; the moments summed in FP64 from the
// stored values), |v - v_ref| and |v| (Euclidean norms), block sums in FP64
// for the fixed-order pass; with `update` the node's v replaces v_ref (each
// thread reads its own entries before it writes them; solid nodes get 0).
template <int Q, class S, bool EXT>
__global__ void __launch_bounds__(RED_THREADS)
k_residual(const typename S::T* __restrict__ P, const uint8_t* __restrict__ cls, const Geo g,
           const KP<typename S::R> p, double* __restrict__ vref, int update, double* __restrict__ partials)
{
    using R = typename S::R;
    __shared__ double sm[2 * 32];
    double acc[2] = {0.0, 0.0};
    const long long N = (long long)g.nx * g.ny * g.nz;
    const double c = (double)p.c;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % g.nx);
        const long long r = n / g.nx;
        const int y = (int)(r % g.ny), z = (int)(r / g.ny);
        if (nc_solid(cls[r * g.nxp + x])) {
            if (update)
#pragma unroll
                for (int k = 0; k < 3; ++k) vref[(long long)k * N + n] = 0.0;
            continue;
        }
        R d[Q];
        gather_node<Q, S>(P, cls, g, p, x, y, z, d);
        NodeM<R> m;
        node_macro<R, Q, EXT>(d, p, m);
        double dr = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const double da = (double)d[a];
            dr += da;
            j[0] += EX<Q>(a) * da;
            j[1] += EY<Q>(a) * da;
            j[2] += EZ<Q>(a) * da;
        }
        const double rho = (double)p.rho0 + dr;
        double dd = 0.0, vv = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double vk = c * (j[k] / rho + 0.5 * (double)m.A[k]);
            const double dk = vk - vref[(long long)k * N + n];
            dd += dk * dk;
            vv += vk * vk;
            if (update) vref[(long long)k * N + n] = vk;
        }
        acc[0] += sqrt(dd);
        acc[1] += sqrt(vv);
    }
    block_sum<2>(acc, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < 2; ++k) partials[(long long)blockIdx.x * 2 + k] = acc[k];
}

// ----------------------------------------------------------------- stress
// Variants 1, 2 at f(T) = gather(cur); 3, 4 at the half step between T-1 and
// T: fbar = (cur + gather(cur))/2 with the node's state at T-1 = gather(prev).
template <int Q, class S, bool EXT>
__global__ void __launch_bounds__(NODE_THREADS)
k_stress(const typename S::T* __restrict__ cur, const typename S::T* __restrict__ prev,
         const uint8_t* __restrict__ cls, const Geo g, const KP<typename S::R> p, int variant,
         typename S::R* __restrict__ sig, typename S::R* __restrict__ Sout, typename S::R* __restrict__ rho_out,
         typename S::R* __restrict__ v_out)
{
    using R = typename S::R;
    constexpr int D = LatDim<Q>::D;
    constexpr int NC = (D == 3) ? 6 : 3;
    const long long N = (long long)g.nx * g.ny * g.nz;
    const R c = p.c, c2 = p.c * p.c;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % g.nx);
        const long long r = n / g.nx;
        const int y = (int)(r % g.ny), z = (int)(r / g.ny);
        const long long own = r * g.nxp + x;
        R out[6] = {0, 0, 0, 0, 0, 0}, Sv[6] = {0, 0, 0, 0, 0, 0}, rr = 0, vv[3] = {0, 0, 0};
        if (!nc_solid(cls[own])) {
            R d[Q];
            NodeM<R> m;
            // component index -> (i, j)
            constexpr int ci3[6] = {0, 1, 2, 0, 0, 1}, cj3[6] = {0, 1, 2, 1, 2, 2};
            constexpr int ci2[3] = {0, 1, 0}, cj2[3] = {0, 1, 1};
            // L / c^2 of the Maxwell term: configured, or at the node's induced field B(x, T)
            R Lh[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) Lh[k] = p.Lh[k];
            if (EXT && p.induced) {
                R B[3];
                mag_field_at<Q>(p.mag, cls, g, p, x, y, z, own, B);
                const R kl = R(2) / R(9) * p.mxk, h = R(0.5) * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
                Lh[0] = kl * (h - B[0] * B[0]);
                Lh[1] = kl * (h - B[1] * B[1]);
                Lh[2] = kl * (h - B[2] * B[2]);
                Lh[3] = -kl * B[0] * B[1];
                Lh[4] = -kl * B[0] * B[2];
                Lh[5] = -kl * B[1] * B[2];
            }
            if (variant <= 2) {
                gather_node<Q, S>(cur, cls, g, p, x, y, z, d);
                node_macro<R, Q, EXT>(d, p, m);
                const R fac = -(R(1) - R(0.5) * m.om) * c2;
                const bool model_a = (p.model == MODEL_A);
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const int i = (D == 3) ? ci3[cc] : ci2[cc], j = (D == 3) ? cj3[cc] : cj2[cc];
                    const int lc = (D == 3) ? cc : (cc == 2 ? 3 : cc);   // index into Lh
                    R P2 = 0;
#pragma unroll
                    for (int a = 0; a < Q; ++a) {
                        const int ea[3] = {EX<Q>(a), EY<Q>(a), EZ<Q>(a)};
                        const int ee = ea[i] * ea[j];
                        if (ee) P2 += R(ee) * d[a];
                    }
                    // cheap form of Sec. 3: sum e e f - (p delta + rho u^eq u^eq + L)
                    R Pi = P2 - (p.stokes ? R(0) : m.rho * m.weq[i] * m.weq[j]) - (p.maxwell ? Lh[lc] : R(0));
                    if (i == j) Pi -= m.drho / R(3);
                    if (variant == 1) {
                        // E_ij = tau dt rho (u^eq a + a u^eq) - tau Theta_ij, in units of c^2
                        R E = m.tau * m.rho * (m.weq[i] * m.A[j] + m.weq[j] * m.A[i]);
                        if (!model_a) E -= m.tau * m.C * m.rho * (m.wf[i] * m.A[j] + m.wf[j] * m.A[i]);
                        Pi += E;
                    }
                    out[cc] = fac * Pi;
                }
                rr = m.rho;
#pragma unroll
                for (int k = 0; k < 3; ++k) vv[k] = c * m.v[k];
            } else {
                R dn[Q];
                gather_node<Q, S>(cur, cls, g, p, x, y, z, dn);
                R db[Q];
                R drb = 0, jb[3] = {0, 0, 0};
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    db[a] = R(0.5) * (S::to_r(cur[(long long)a * g.sq + own]) + dn[a]);
                    drb += db[a];
                    jb[0] += R(EX<Q>(a)) * db[a];
                    jb[1] += R(EY<Q>(a)) * db[a];
                    jb[2] += R(EZ<Q>(a)) * db[a];
                }
                const R rb = p.rho0 + drb;
                const R ub[3] = {jb[0] / rb, jb[1] / rb, jb[2] / rb};
                gather_node<Q, S>(prev, cls, g, p, x, y, z, d);
                node_macro<R, Q, EXT>(d, p, m);
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const int i = (D == 3) ? ci3[cc] : ci2[cc], j = (D == 3) ? cj3[cc] : cj2[cc];
                    const int lc = (D == 3) ? cc : (cc == 2 ? 3 : cc);
                    R P2 = 0;
#pragma unroll
                    for (int a = 0; a < Q; ++a) {
                        const int ea[3] = {EX<Q>(a), EY<Q>(a), EZ<Q>(a)};
                        const int ee = ea[i] * ea[j];
                        if (ee) P2 += R(ee) * db[a];
                    }
                    // sum e e (fbar - f^eq(rhobar, ubar)), in units of c^2
                    R Pi = P2 - (p.stokes ? R(0) : rb * ub[i] * ub[j]) - (p.maxwell ? Lh[lc] : R(0));
                    if (i == j) Pi -= drb / R(3);
                    R s = -c2 * Pi;
                    if (variant == 4 && p.model != MODEL_A)
                        s += R(0.5) * c2 * m.C * m.rho * (m.wf[i] * m.A[j] + m.wf[j] * m.A[i]);
                    out[cc] = s;
                }
                rr = rb;
#pragma unroll
                for (int k = 0; k < 3; ++k) vv[k] = c * ub[k];
            }
            const R nu = p.dt * c2 * (m.tau - R(0.5)) / R(3);
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) Sv[cc] = out[cc] / (R(2) * rr * nu);
        }
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
            if (sig) sig[(long long)cc * N + n] = out[cc];
            if (Sout) Sout[(long long)cc * N + n] = Sv[cc];
        }
        if (rho_out) rho_out[n] = rr;
        if (v_out)
#pragma unroll
            for (int k = 0; k < 3; ++k) v_out[(long long)k * N + n] = vv[k];
    }
}

// ---------------------------------------------------------- induced field
// One coupled step per node (one thread per padded node): the field
// distributions g(x, T) pulled from the stored post-collision ones, the
// node's field B = sum g, the fluid populations f(x, T) (gather_node) and
// their moments; the field relaxes toward W_i [B + e_i . (v B - B v)/theta]
// with the node's flow velocity v, the fluid with the Maxwell term of
// Eq. (10) at B.  Both write their post-collision values for the next pull.
template <int Q, class S, bool SR>
__global__ void __launch_bounds__(NODE_THREADS, MhdOcc<S>::value)
k_mhd_step(const typename S::T* __restrict__ src, typename S::T* __restrict__ dst,
           const typename S::R* __restrict__ G, typename S::R* __restrict__ Gn, const uint8_t* __restrict__ cls,
           const Geo g, const KP<typename S::R> p, uint32_t seed)
{
    using R = typename S::R;
    constexpr int QM = MagLat<Q>::QM;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.sq) return;
    const int x = (int)(n % g.nxp);
    const long long row = n / g.nxp;
    const int y = (int)(row % g.ny), z = (int)(row / g.ny);
    const uint8_t c = cls[n];
    if (x >= g.nx || nc_solid(c) || c == NC_PAD) {
#pragma unroll
        for (int a = 0; a < Q; ++a) dst[(long long)a * g.sq + n] = S::from_raw(R(0));
#pragma unroll
        for (int j = 0; j < 3 * QM; ++j) Gn[(long long)j * g.sq + n] = R(0);
        return;
    }
    R gm[3][QM];
    R d[Q];
    if (c == NC_BULK) {
        // every pull source is a fluid node (periodic wrap allowed): plain
        // indexed loads, no class bytes
        int ro[3][3];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dz = -1; dz <= 1; ++dz)
                ro[dy + 1][dz + 1] = (wrapi(z - dz, g.nz) * g.ny + wrapi(y - dy, g.ny)) * g.nxp;
        const int xm = wrapi(x - 1, g.nx), xp = wrapi(x + 1, g.nx);
        auto at = [&](int a) { return ro[EY<Q>(a) + 1][EZ<Q>(a) + 1] + (EX<Q>(a) == 0 ? x : (EX<Q>(a) == 1 ? xm : xp)); };
#pragma unroll
        for (int a = 0; a < Q; ++a) d[a] = S::to_raw(src[(long long)a * g.sq + at(a)]);
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int i = 0; i < QM; ++i) gm[k][i] = G[(long long)(k * QM + i) * g.sq + at(i)];
    } else {
        mag_gather<Q>(G, cls, g, p, x, y, z, n, gm);
        gather_node<Q, S, true, false>(src, cls, g, p, x, y, z, d);   // the induced field has no curved walls
    }
    NodeM<R> m;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R b = R(0);
#pragma unroll
        for (int i = 0; i < QM; ++i) b += gm[k][i];
        m.Bl[k] = b;
    }
    node_macro<R, Q, true>(d, p, m);
    // field: e_i is +-1 along one axis, so e_i . (v B_k - B v_k) = s (v_ax B_k - B_ax v_k)
    const R om = p.om_m, ith = R(1.0 / MagLat<Q>::TH);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < QM; ++i) {
            const int ax = (EX<Q>(i) != 0) ? 0 : ((EY<Q>(i) != 0) ? 1 : 2);
            const int sg = EX<Q>(i) + EY<Q>(i) + EZ<Q>(i);
            const R W = R(i == 0 ? MagLat<Q>::W0 : MagLat<Q>::W1);
            const R el = (i == 0) ? R(0) : R(sg) * (m.v[ax] * m.Bl[k] - m.Bl[ax] * m.v[k]);
            const R geq = W * (m.Bl[k] + ith * el);
            Gn[(long long)(k * QM + i) * g.sq + n] = gm[k][i] + om * (geq - gm[k][i]);
        }
    node_relax<R, Q, true, true>(d, p, m);
    if constexpr (SR) {
        NodeRng rng((uint32_t)n, seed);
#pragma unroll
        for (int a = 0; a < Q; ++a) dst[(long long)a * g.sq + n] = S::from_raw_sr(d[a], rng.bits(a));
    } else {
#pragma unroll
        for (int a = 0; a < Q; ++a) dst[(long long)a * g.sq + n] = S::from_raw(d[a]);
    }
}

// field distributions at rest in the external field, W_i B, in both buffers
template <int Q, typename R>
__global__ void __launch_bounds__(NODE_THREADS)
k_mag_init(R* __restrict__ G0, R* __restrict__ G1, const uint8_t* __restrict__ cls, const Geo g, const KP<R> p)
{
    constexpr int QM = MagLat<Q>::QM;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.sq) return;
    const uint8_t c = cls[n];
    const bool fluid = (int)(n % g.nxp) < g.nx && !nc_solid(c) && c != NC_PAD;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < QM; ++i) {
            const R v = fluid ? R(i == 0 ? MagLat<Q>::W0 : MagLat<Q>::W1) * p.Bext[k] : R(0);
            G0[(long long)(k * QM + i) * g.sq + n] = v;
            G1[(long long)(k * QM + i) * g.sq + n] = v;
        }
}

// B(x, T) in canonical order, zero at solid nodes
template <int Q, typename R>
__global__ void __launch_bounds__(NODE_THREADS)
k_mag_field(const R* __restrict__ G, const uint8_t* __restrict__ cls, const Geo g, const KP<R> p,
            double* __restrict__ Bout)
{
    const long long N = (long long)g.nx * g.ny * g.nz;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int x = (int)(n % g.nx);
    const long long r = n / g.nx;
    const int y = (int)(r % g.ny), z = (int)(r / g.ny);
    const long long own = r * g.nxp + x;
    R B[3] = {R(0), R(0), R(0)};
    if (!nc_solid(cls[own])) mag_field_at<Q>(G, cls, g, p, x, y, z, own, B);
#pragma unroll
    for (int k = 0; k < 3; ++k) Bout[(long long)k * N + n] = (double)B[k];
}

// ================================================================ launchers
inline int grid_for(long long n, int threads, long long cap)
{
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

template <class S> inline const KP<typename S::R>& kp_of(const Ctx& c)
{
    if constexpr (sizeof(typename S::R) == 8) return c.kpd;
    else return c.kpf;
}
// parameters in storage units, for the step kernels
template <class S> inline const KP<typename S::R>& kp_step_of(const Ctx& c)
{
    if constexpr (sizeof(typename S::R) == 8) return c.kpd;
    else return c.kps;
}

// a copy of the parameters that reads the field distributions G
template <typename R> inline KP<R> with_mag(const KP<R>& p, const void* G)
{
    KP<R> q = p;
    q.mag = static_cast<const R*>(G);
    return q;
}
// the wall force reads the field of the step that produced the stored state:
// B(T-1), pulled from the other field buffer
template <class S> inline KP<typename S::R> kp_links_of(const Ctx& c)
{
    return with_mag(kp_of<S>(c), c.cfg.induced ? c.mag[1 - c.cur] : nullptr);
}

template <int Q, class S, bool EXT, bool SR>
cudaError_t launch_step_q(const Ctx& c, const void* src, void* dst, uint32_t seed, cudaStream_t st)
{
    using T = typename S::T;
    const long long nch = (long long)(c.geo.nxp / S::V) * c.geo.ny * c.geo.nz;
    const int blocks = grid_for(nch, STEP_THREADS, 1ll << 31);
    const bool faces = !c.geo.periodic[0] || !c.geo.periodic[1] || (Q == 19 && !c.geo.periodic[2]);
    if constexpr (EXT && sizeof(typename S::T) == 2) {
        if (c.les_pair) {
            if (faces)
                k_step<Q, S, EXT, true, SR, false, true><<<blocks, STEP_THREADS, 0, st>>>(
                    (const T*)src, (T*)dst, c.cls, c.geo, kp_step_of<S>(c), seed);
            else
                k_step<Q, S, EXT, false, SR, false, true><<<blocks, STEP_THREADS, 0, st>>>(
                    (const T*)src, (T*)dst, c.cls, c.geo, kp_step_of<S>(c), seed);
            return cudaGetLastError();
        }
    }
    if ((c.cfg.curved || c.insulating) && faces)
        k_step<Q, S, EXT, true, SR, true><<<blocks, STEP_THREADS, 0, st>>>((const T*)src, (T*)dst, c.cls, c.geo,
                                                                           kp_step_of<S>(c), seed);
    else if (c.cfg.curved || c.insulating)
        k_step<Q, S, EXT, false, SR, true><<<blocks, STEP_THREADS, 0, st>>>((const T*)src, (T*)dst, c.cls, c.geo,
                                                                            kp_step_of<S>(c), seed);
    else if (faces)
        k_step<Q, S, EXT, true, SR><<<blocks, STEP_THREADS, 0, st>>>((const T*)src, (T*)dst, c.cls, c.geo,
                                                                     kp_step_of<S>(c), seed);
    else
        k_step<Q, S, EXT, false, SR><<<blocks, STEP_THREADS, 0, st>>>((const T*)src, (T*)dst, c.cls, c.geo,
                                                                      kp_step_of<S>(c), seed);
    return cudaGetLastError();
}

// the staged step (periodic boxes with the plain node code, 16-bit or FP32
// storage; the host chose the tile rows and stage count at create)
template <int Q, class S, bool SR, bool EXT, bool FACES, bool LP = false>
cudaError_t launch_step_staged_k(const Ctx& c, const void* src, void* dst, uint32_t seed, cudaStream_t st,
                                 const StgForce& fw)
{
    using T = typename S::T;
    auto kern = k_step_staged<Q, S, SR, EXT, FACES, LP>;
    // a context always launches the same instantiation: set its shared
    // memory limit on the first launch
    if (!c.stage_ready) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.stage_smem);
        if (e != cudaSuccess) return e;
        c.stage_ready = true;
    }
    kern<<<staged_blocks(c), STG_THREADS, c.stage_smem, st>>>((const T*)src, (T*)dst, c.cls, c.special, c.n_special,
                                                              c.geo, kp_step_of<S>(c), seed, c.stage_R,
                                                              c.stage_tiles, c.stage_n, c.errflag, fw);
    return cudaGetLastError();
}

// the staged step (the host chose the tile rows and stage count at create)
template <int Q, class S, bool SR>
cudaError_t launch_step_staged(const Ctx& c, const void* src, void* dst, uint32_t seed, cudaStream_t st,
                               const StgForce& fw)
{
    const bool faces = !c.geo.periodic[0] || !c.geo.periodic[1] || (Q == 19 && !c.geo.periodic[2]);
    if constexpr (sizeof(typename S::T) == 2) {
        if (c.les_pair)
            return faces ? launch_step_staged_k<Q, S, SR, true, true, true>(c, src, dst, seed, st, fw)
                         : launch_step_staged_k<Q, S, SR, true, false, true>(c, src, dst, seed, st, fw);
    }
    if (c.ext)
        return faces ? launch_step_staged_k<Q, S, SR, true, true>(c, src, dst, seed, st, fw)
                     : launch_step_staged_k<Q, S, SR, true, false>(c, src, dst, seed, st, fw);
    return faces ? launch_step_staged_k<Q, S, SR, false, true>(c, src, dst, seed, st, fw)
                 : launch_step_staged_k<Q, S, SR, false, false>(c, src, dst, seed, st, fw);
}

template <int Q, class S>
cudaError_t launch_step(const Ctx& c, const void* src, void* dst, uint32_t seed, cudaStream_t st,
                        const StgForce* fw = nullptr)
{
    StgForce none{};
    const StgForce& f = fw ? *fw : none;
    if constexpr (sizeof(typename S::T) == 2) {
        if (c.stage_R > 0)
            return c.sr ? launch_step_staged<Q, S, true>(c, src, dst, seed, st, f)
                        : launch_step_staged<Q, S, false>(c, src, dst, seed, st, f);
    } else if constexpr (sizeof(typename S::T) == 4) {
        if (c.stage_R > 0) return launch_step_staged<Q, S, false>(c, src, dst, seed, st, f);
    }
    if constexpr (sizeof(typename S::T) == 2) {
        if (c.sr)
            return c.ext ? launch_step_q<Q, S, true, true>(c, src, dst, seed, st)
                         : launch_step_q<Q, S, false, true>(c, src, dst, seed, st);
    }
    return c.ext ? launch_step_q<Q, S, true, false>(c, src, dst, seed, st)
                 : launch_step_q<Q, S, false, false>(c, src, dst, seed, st);
}

template <int Q, class S>
cudaError_t launch_import(const Ctx& c, const void* srcf, int dtype, void* dst, cudaStream_t st)
{
    using T = typename S::T;
    const long long NP = (long long)c.geo.nxp * c.geo.ny * c.geo.nz;
    const int blocks = grid_for(NP, NODE_THREADS, 65535ll * 16);
    const long long N = (long long)c.geo.nx * c.geo.ny * c.geo.nz;
    if (dtype == 0)
        k_inverse_stream<Q, S, SrcCanonD><<<blocks, NODE_THREADS, 0, st>>>((T*)dst, c.cls, c.geo, kp_of<S>(c),
                                                                          SrcCanonD{(const double*)srcf, N});
    else
        k_inverse_stream<Q, S, SrcCanonF><<<blocks, NODE_THREADS, 0, st>>>((T*)dst, c.cls, c.geo, kp_of<S>(c),
                                                                          SrcCanonF{(const float*)srcf, N});
    return cudaGetLastError();
}

template <int Q, class S>
cudaError_t launch_init(const Ctx& c, const double* rho, const double* u, const double* xi, void* dst,
                        cudaStream_t st)
{
    using T = typename S::T;
    const long long NP = (long long)c.geo.nxp * c.geo.ny * c.geo.nz;
    const int blocks = grid_for(NP, NODE_THREADS, 65535ll * 16);
    const long long N = (long long)c.geo.nx * c.geo.ny * c.geo.nz;
    k_inverse_stream<Q, S, SrcFields><<<blocks, NODE_THREADS, 0, st>>>((T*)dst, c.cls, c.geo, kp_of<S>(c),
                                                                      SrcFields{rho, u, xi, N});
    return cudaGetLastError();
}

template <int Q, class S>
cudaError_t launch_export(const Ctx& c, const void* P, void* out, int dtype, cudaStream_t st)
{
    using T = typename S::T;
    const long long N = (long long)c.geo.nx * c.geo.ny * c.geo.nz;
    const int blocks = grid_for(N, NODE_THREADS, 65535ll * 16);
    if (dtype == 0)
        k_export<Q, S, double><<<blocks, NODE_THREADS, 0, st>>>((const T*)P, c.cls, c.geo, kp_of<S>(c), (double*)out);
    else
        k_export<Q, S, float><<<blocks, NODE_THREADS, 0, st>>>((const T*)P, c.cls, c.geo, kp_of<S>(c), (float*)out);
    return cudaGetLastError();
}

template <int Q, class S>
cudaError_t launch_links(const Ctx& c, const void* P, long long begin, long long end, unsigned flags,
                         double* partials, int* nblocks, cudaStream_t st)
{
    using T = typename S::T;
    const int blocks = grid_for(end - begin, RED_THREADS, MAX_PARTIAL_ROWS);
    *nblocks = blocks;
    k_links<Q, S><<<blocks, RED_THREADS, 0, st>>>((const T*)P, c.cls, c.links, begin, end, c.geo, kp_links_of<S>(c),
                                                  flags, partials);
    return cudaGetLastError();
}

template <int Q, class S>
cudaError_t launch_balance(const Ctx& c, const void* P, double* partials, int* nblocks, cudaStream_t st)
{
    using T = typename S::T;
    const long long N = (long long)c.geo.nx * c.geo.ny * c.geo.nz;
    const int blocks = grid_for(N, RED_THREADS, MAX_PARTIAL_ROWS);
    *nblocks = blocks;
    const double vol = (Q == 9) ? c.cfg.dx * c.cfg.dx : c.cfg.dx * c.cfg.dx * c.cfg.dx;
    if (c.ext)
        k_balance<Q, S, true><<<blocks, RED_THREADS, 0, st>>>((const T*)P, c.cls, c.geo, kp_of<S>(c), vol, partials);
    else
        k_balance<Q, S, false><<<blocks, RED_THREADS, 0, st>>>((const T*)P, c.cls, c.geo, kp_of<S>(c), vol, partials);
    return cudaGetLastError();
}

template <int Q, class S>
cudaError_t launch_residual(const Ctx& c, const void* P, double* vref, int update, double* partials, int* nblocks,
                            cudaStream_t st)
{
    using T = typename S::T;
    const long long N = (long long)c.geo.nx * c.geo.ny * c.geo.nz;
    const int blocks = grid_for(N, RED_THREADS, MAX_PARTIAL_ROWS);
    *nblocks = blocks;
    if (c.ext)
        k_residual<Q, S, true><<<blocks, RED_THREADS, 0, st>>>((const T*)P, c.cls, c.geo, kp_of<S>(c), vref, update,
                                                               partials);
    else
        k_residual<Q, S, false><<<blocks, RED_THREADS, 0, st>>>((const T*)P, c.cls, c.geo, kp_of<S>(c), vref, update,
                                                                partials);
    return cudaGetLastError();
}

template <int Q, class S>
cudaError_t launch_stress(const Ctx& c, const void* cur, const void* prev, int variant, void* sig, void* Sv,
                          void* rho, void* v, cudaStream_t st)
{
    using T = typename S::T;
    using R = typename S::R;
    const long long N = (long long)c.geo.nx * c.geo.ny * c.geo.nz;
    const int blocks = grid_for(N, NODE_THREADS, 65535ll * 16);
    if (c.ext)
        k_stress<Q, S, true><<<blocks, NODE_THREADS, 0, st>>>((const T*)cur, (const T*)prev, c.cls, c.geo,
                                                              with_mag(kp_of<S>(c), c.mag[c.cur]), variant, (R*)sig,
                                                              (R*)Sv, (R*)rho, (R*)v);
    else
        k_stress<Q, S, false><<<blocks, NODE_THREADS, 0, st>>>((const T*)cur, (const T*)prev, c.cls, c.geo, kp_of<S>(c),
                                                               variant, (R*)sig, (R*)Sv, (R*)rho, (R*)v);
    return cudaGetLastError();
}

template <int Q, class S>
cudaError_t launch_mhd_step(const Ctx& c, const void* src, void* dst, const void* G, void* Gn, uint32_t seed,
                            cudaStream_t st)
{
    using T = typename S::T;
    using R = typename S::R;
    const int blocks = grid_for(c.geo.sq, NODE_THREADS, 1ll << 31);
    if constexpr (sizeof(T) == 2) {
        if (c.sr) {
            k_mhd_step<Q, S, true><<<blocks, NODE_THREADS, 0, st>>>((const T*)src, (T*)dst, (const R*)G, (R*)Gn, c.cls,
                                                                    c.geo, kp_step_of<S>(c), seed);
            return cudaGetLastError();
        }
    }
    k_mhd_step<Q, S, false><<<blocks, NODE_THREADS, 0, st>>>((const T*)src, (T*)dst, (const R*)G, (R*)Gn, c.cls,
                                                                 c.geo, kp_step_of<S>(c), seed);
    return cudaGetLastError();
}

template <int Q, class S>
cudaError_t launch_mag_init(const Ctx& c, cudaStream_t st)
{
    using R = typename S::R;
    const int blocks = grid_for(c.geo.sq, NODE_THREADS, 1ll << 31);
    k_mag_init<Q, R><<<blocks, NODE_THREADS, 0, st>>>((R*)c.mag[0], (R*)c.mag[1], c.cls, c.geo, kp_of<S>(c));
    return cudaGetLastError();
}

template <int Q, class S>
cudaError_t launch_mag_field(const Ctx& c, double* B, cudaStream_t st)
{
    using R = typename S::R;
    const long long N = (long long)c.geo.nx * c.geo.ny * c.geo.nz;
    const int blocks = grid_for(N, NODE_THREADS, 1ll << 31);
    k_mag_field<Q, R><<<blocks, NODE_THREADS, 0, st>>>((const R*)c.mag[c.cur], c.cls, c.geo, kp_of<S>(c), B);
    return cudaGetLastError();
}

}  // namespace lbm

#include "lbm_adjoint.cuh"  // the adjoint kernel and launch_adjoint; uses block_sum, grid_for, kp_of

namespace lbm {

template <class S> Dispatch make_dispatch()
{
    Dispatch d;
    d.step = [](const Ctx& c, const void* s, void* t, uint32_t seed, cudaStream_t st) {
        return c.cfg.lattice == 9 ? launch_step<9, S>(c, s, t, seed, st) : launch_step<19, S>(c, s, t, seed, st);
    };
    d.step_force = [](const Ctx& c, const void* s, void* t, uint32_t seed, const StgForce& fw, cudaStream_t st) {
        return c.cfg.lattice == 9 ? launch_step<9, S>(c, s, t, seed, st, &fw)
                                  : launch_step<19, S>(c, s, t, seed, st, &fw);
    };
    d.import_f = [](const Ctx& c, const void* s, int dt, void* t, cudaStream_t st) {
        return c.cfg.lattice == 9 ? launch_import<9, S>(c, s, dt, t, st) : launch_import<19, S>(c, s, dt, t, st);
    };
    d.init_fields = [](const Ctx& c, const double* r, const double* u, const double* xi, void* t, cudaStream_t st) {
        return c.cfg.lattice == 9 ? launch_init<9, S>(c, r, u, xi, t, st) : launch_init<19, S>(c, r, u, xi, t, st);
    };
    d.export_f = [](const Ctx& c, const void* P, void* o, int dt, cudaStream_t st) {
        return c.cfg.lattice == 9 ? launch_export<9, S>(c, P, o, dt, st) : launch_export<19, S>(c, P, o, dt, st);
    };
    d.links = [](const Ctx& c, const void* P, long long b, long long e, unsigned fl, double* pa, int* nb,
                 cudaStream_t st) {
        return c.cfg.lattice == 9 ? launch_links<9, S>(c, P, b, e, fl, pa, nb, st)
                                  : launch_links<19, S>(c, P, b, e, fl, pa, nb, st);
    };
    d.balance = [](const Ctx& c, const void* P, double* pa, int* nb, cudaStream_t st) {
        return c.cfg.lattice == 9 ? launch_balance<9, S>(c, P, pa, nb, st) : launch_balance<19, S>(c, P, pa, nb, st);
    };
    d.residual = [](const Ctx& c, const void* P, double* vr, int up, double* pa, int* nb, cudaStream_t st) {
        return c.cfg.lattice == 9 ? launch_residual<9, S>(c, P, vr, up, pa, nb, st)
                                  : launch_residual<19, S>(c, P, vr, up, pa, nb, st);
    };
    d.stress = [](const Ctx& c, const void* cu, const void* pr, int var, void* sg, void* Sv, void* rh, void* v,
                  cudaStream_t st) {
        return c.cfg.lattice == 9 ? launch_stress<9, S>(c, cu, pr, var, sg, Sv, rh, v, st)
                                  : launch_stress<19, S>(c, cu, pr, var, sg, Sv, rh, v, st);
    };
    d.mhd_step = [](const Ctx& c, const void* s, void* t, const void* G, void* Gn, uint32_t seed, cudaStream_t st) {
        return c.cfg.lattice == 9 ? launch_mhd_step<9, S>(c, s, t, G, Gn, seed, st)
                                  : launch_mhd_step<19, S>(c, s, t, G, Gn, seed, st);
    };
    d.mag_init = [](const Ctx& c, cudaStream_t st) {
        return c.cfg.lattice == 9 ? launch_mag_init<9, S>(c, st) : launch_mag_init<19, S>(c, st);
    };
    d.mag_field = [](const Ctx& c, double* B, cudaStream_t st) {
        return c.cfg.lattice == 9 ? launch_mag_field<9, S>(c, B, st) : launch_mag_field<19, S>(c, B, st);
    };
    d.adjoint = [](const Ctx& c, const void* Pp, const void* pn, void* po, int w, const double* dir, double sw,
                   double* pa, cudaStream_t st) {
        return c.cfg.lattice == 9 ? launch_adjoint<9, S>(c, Pp, pn, po, w, dir, sw, pa, st)
                                  : launch_adjoint<19, S>(c, Pp, pn, po, w, dir, sw, pa, st);
    };
    return d;
}

}  // namespace lbm
