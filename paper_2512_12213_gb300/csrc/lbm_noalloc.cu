// lbm_noalloc.cu -- lbm_wall_force_noalloc: the momentum-exchange wall force
// of lbm_wall_force, computed without any device memory from the caller
// beyond the context's inputs and the output.
//
// Who needs it: a caller that cannot allocate device memory when it asks for
// a force -- for example because its device memory is fully committed to
// population arrays (two copies of a 512^3 D3Q19 state in FP64 alone take
// 40 GB), or because that memory belongs to a host application or another
// runtime that hands this library nothing more -- and that cannot use the
// context's own scratch buffer at that moment because another reduction of
// the same context (lbm_balance, lbm_wall_force, the adjoint gradient) is
// queued on a different stream and owns it.
//
// How: the block partial sums and the result slot live in one file-scope
// static device array of fixed size, which every GPU that loads this library
// holds until the process exits.  The launch has exactly the shape of
// lbm_wall_force's (at most MAX_PARTIAL_ROWS blocks of RED_THREADS threads,
// each thread striding over the links), so the two add the same terms in the
// same order and agree bit for bit at every link count.  One call takes at
// most NOALLOC_MAX_LINKS links; larger requests are refused.
#include <cstdio>
#include <mutex>
#include <string>

#include "lbm_kernels.cuh"

namespace {

constexpr int NOALLOC_ROWS = lbm::MAX_PARTIAL_ROWS;                 // block partial rows (1024)
constexpr long long NOALLOC_MAX_LINKS = 1ll << 20;                  // 1,048,576 links per call
constexpr int NOALLOC_RESULT = NOALLOC_ROWS * 3;                     // offset of the 3-double result slot

// 1024 x 3 partial sums + one result slot: 24,640 bytes per device
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_ROWS * 3 + 8];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_addr[MAX_DEVICES];          // device address of g_noalloc_scratch, per device

// Looked up once per device, with that device current.  Host code must not
// use the symbol itself: on the host it names a stand-in, not device memory.
bool scratch_address(int dev, double** out, std::string& err)
{
    if (dev < 0 || dev >= MAX_DEVICES) {
        err = "device ordinal out of range for the static scratch table";
        return false;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e);
            return false;
        }
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return true;
}

template <int Q, class S>
cudaError_t launch_links_rows(const lbm::Ctx& c, const void* P, long long begin, long long end, unsigned flags,
                              double* partials, int rows, cudaStream_t st)
{
    using T = typename S::T;
    lbm::k_links<Q, S><<<rows, lbm::RED_THREADS, 0, st>>>((const T*)P, c.cls, c.links, begin, end, c.geo,
                                                         lbm::kp_links_of<S>(c), flags, partials);
    return cudaGetLastError();
}

template <class S>
cudaError_t links_rows(const lbm::Ctx& c, const void* P, long long b, long long e, unsigned flags, double* part,
                       int rows, cudaStream_t st)
{
    return c.cfg.lattice == 9 ? launch_links_rows<9, S>(c, P, b, e, flags, part, rows, st)
                              : launch_links_rows<19, S>(c, P, b, e, flags, part, rows, st);
}

}  // namespace

extern "C" lbm_status lbm_wall_force_noalloc(lbm_ctx* ctx, int wall, unsigned flags, double weight, double* out,
                                             int out_on_host, void* stream)
{
    using namespace lbm;
    if (!ctx) return LBM_ERR_ARG;
    Ctx& x = ctx->c;
    if (!out) {
        x.err = "out is NULL";
        return LBM_ERR_ARG;
    }
    if (wall > LBM_MAX_WALLS) {
        x.err = "wall id out of range";
        return LBM_ERR_ARG;
    }
    if (flags & ~7u) {
        x.err = "unknown flag";
        return LBM_ERR_ARG;
    }
    if (x.t < 1) {
        x.err = "the wall force needs at least one step";
        return LBM_ERR_STATE;
    }
    const long long b = wall < 0 ? 0 : x.wall_begin[wall];
    const long long e = wall < 0 ? x.n_links : x.wall_begin[wall + 1];
    if (e - b > NOALLOC_MAX_LINKS) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "lbm_wall_force_noalloc: %lld links requested, the static scratch holds partial sums for at most "
                 "%lld links per call; use lbm_wall_force",
                 e - b, NOALLOC_MAX_LINKS);
        x.err = buf;
        return LBM_ERR_ARG;
    }
    int old = -1;
    if (cudaGetDevice(&old) != cudaSuccess) {
        x.err = "cudaGetDevice failed";
        return LBM_ERR_CUDA;
    }
    if (old != x.device && cudaSetDevice(x.device) != cudaSuccess) {
        x.err = "cudaSetDevice failed";
        return LBM_ERR_CUDA;
    }
    if (!out_mode_ok(out_on_host, (flags & LBM_ACCUMULATE) != 0, out, x.err)) {
        if (old != x.device) cudaSetDevice(old);
        return LBM_ERR_ARG;
    }
    lbm_status status = LBM_OK;
    double* scratch = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t ce = cudaSuccess;
    if (!scratch_address(x.device, &scratch, x.err)) {
        status = LBM_ERR_CUDA;
    } else {
        // the grid of lbm_wall_force (launch_links): the same blocks, the same
        // per-thread strides, the same partial rows.  Every partial row and
        // the result slot are written before they are read, so nothing in the
        // array needs clearing between calls
        const int rows = (e > b) ? grid_for(e - b, RED_THREADS, NOALLOC_ROWS) : 0;
        if (rows > 0) {
            switch (x.cfg.storage) {
            case LBM_STORE_F64: ce = links_rows<StoreF64>(x, x.pop[x.cur], b, e, flags & 3u, scratch, rows, st); break;
            case LBM_STORE_F32: ce = links_rows<StoreF32>(x, x.pop[x.cur], b, e, flags & 3u, scratch, rows, st); break;
            case LBM_STORE_F16S: ce = links_rows<StoreF16>(x, x.pop[x.cur], b, e, flags & 3u, scratch, rows, st); break;
            default: ce = links_rows<StoreBF16>(x, x.pop[x.cur], b, e, flags & 3u, scratch, rows, st); break;
            }
        }
        const bool acc = (flags & LBM_ACCUMULATE) != 0;
        if (ce == cudaSuccess) {
            if (out_on_host == LBM_OUT_DEVICE) {
                ce = launch_reduce_rows(scratch, rows, 3, out, weight, acc ? 1 : 0, st);
            } else if (out_on_host == LBM_OUT_HOST_ASYNC) {
                double* slot = scratch + NOALLOC_RESULT;
                ce = launch_reduce_rows(scratch, rows, 3, slot, weight, 0, st);
                if (ce == cudaSuccess) ce = cudaMemcpyAsync(out, slot, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
            } else {
                double* slot = scratch + NOALLOC_RESULT;
                double tmp[3];
                ce = launch_reduce_rows(scratch, rows, 3, slot, weight, 0, st);
                if (ce == cudaSuccess) ce = cudaMemcpyAsync(tmp, slot, sizeof tmp, cudaMemcpyDeviceToHost, st);
                if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
                if (ce == cudaSuccess)
                    for (int k = 0; k < 3; ++k) out[k] = acc ? out[k] + tmp[k] : tmp[k];
            }
        }
        if (ce != cudaSuccess) {
            x.err = std::string("lbm_wall_force_noalloc: ") + cudaGetErrorString(ce);
            status = LBM_ERR_CUDA;
        }
    }
    if (old != x.device) cudaSetDevice(old);
    return status;
}
