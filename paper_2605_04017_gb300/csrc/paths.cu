// Many paths in one launch (lt_trace_paths): the flare workload of Sec. 4.2,
// where the same entrance rays follow the main path and every two-bounce
// ghost (i, j), each path with its own wavelength draw.
//
// Grid: blockIdx.y = path, blockIdx.x = tile of 256 rays.  Ghost rays die at
// very different depths, so the hardware block scheduler (which hands a free
// SM slot the next tile as soon as one retires) balances the load; a
// persistent loop would only re-implement it.  Valid rays are compacted per
// warp: a ballot, one atomic on the path's counter by the first valid lane,
// and rank-ordered writes into the path's segment.
#include "profile.h"
#include "rays.cuh"
#include "tracer.cuh"

namespace lt {

constexpr int kPathsBlock = 256;
constexpr int kMaxPaths = 1024;

struct PathTable {
    int8_t ij[2 * kMaxPaths];   // (i, j) of each path; (0, 0) is the main path
};

struct PathsOutDev {
    float *__restrict__ x, *__restrict__ y, *__restrict__ dx, *__restrict__ dy, *__restrict__ dz,
        *__restrict__ I;
    uint8_t* __restrict__ flags;
    uint32_t* __restrict__ ray_index;
    uint32_t* __restrict__ count;
    size_t capacity;
};

template <bool CAUCHY>
__global__ void __launch_bounds__(kPathsBlock)
trace_paths_kernel(const __grid_constant__ LensDev L, const __grid_constant__ PathTable P,
                   RaysInDev in, size_t lam_stride, PathsOutDev out, uint32_t n,
                   unsigned long long* work)
{
    const unsigned full = 0xffffffffu;
    const int p = blockIdx.y;
    const uint32_t r = blockIdx.x * kPathsBlock + threadIdx.x;
    const int pi = P.ij[2 * p], pj = P.ij[2 * p + 1];
    int nint = 0;
    TraceOut o;
    uint32_t f = 0;
    if (r < n)
        f = trace_ray<CAUCHY>(L, pi, pj, __ldg(in.x + r), __ldg(in.y + r), __ldg(in.dx + r),
                              __ldg(in.dy + r), __ldg(in.dz + r),
                              __ldg(in.lam + (size_t)p * lam_stride + r), o, nint);
    const bool v = (r < n) && (f & LT_FLAG_VALID);
    const unsigned m = __ballot_sync(full, v);
    if (m) {
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(m) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(out.count + p, (uint32_t)__popc(m));
        base = __shfl_sync(full, base, leader);
        if (v) {
            const uint32_t k = base + (uint32_t)__popc(m & ((1u << lane) - 1u));
            if (k < out.capacity) {
                const size_t e = (size_t)p * out.capacity + k;
                __stcs(out.x + e, o.x);
                __stcs(out.y + e, o.y);
                __stcs(out.dx + e, o.dx);
                __stcs(out.dy + e, o.dy);
                __stcs(out.dz + e, o.dz);
                __stcs(out.I + e, o.I);
                __stcs(out.ray_index + e, r);
                out.flags[e] = (uint8_t)f;
            }
        }
    }
    warp_add(work, (unsigned)nint);
}

}  // namespace lt

using namespace lt;

extern "C" lt_status lt_trace_paths(const lt_lens* L, const lt_rays_in* in, const float* lam,
                                    size_t lam_stride, const int32_t* path_ids, int32_t n_paths,
                                    const lt_paths_out* out, size_t n, lt_stream stream)
{
    clear_error();
    if (!L || !in || !out || !path_ids) return fail(LT_EINVAL, "lt_trace_paths: NULL argument");
    if (n_paths < 1 || n_paths > kMaxPaths)
        return fail(LT_EINVAL, "lt_trace_paths: n_paths must be in [1, %d]", kMaxPaths);
    if (n >= (1ull << 32)) return fail(LT_EINVAL, "lt_trace_paths: n must be < 2^32");
    if (out->capacity < 1) return fail(LT_EINVAL, "lt_trace_paths: capacity must be >= 1");
    if (!out->valid_count) return fail(LT_EINVAL, "lt_trace_paths: NULL valid_count");
    PathTable P{};
    for (int p = 0; p < n_paths; ++p) {
        int pi, pj;
        if (!path_ij(L->S, path_ids[p], &pi, &pj))
            return fail(LT_EINVAL, "lt_trace_paths: bad path id %d at %d", path_ids[p], p);
        P.ij[2 * p] = (int8_t)pi;
        P.ij[2 * p + 1] = (int8_t)pj;
    }
    cudaStream_t st = (cudaStream_t)stream;
    LT_CUDA_TRY(cudaMemsetAsync(out->valid_count, 0, (size_t)n_paths * 4, st));
    if (n == 0) return LT_OK;
    const void* ps[] = {in->x, in->y, in->dx, in->dy, in->dz, lam, out->x, out->y, out->dx,
                        out->dy, out->dz, out->I, out->ray_index};
    for (const void* q : ps)
        if (!q || !aligned16(q))
            return fail(LT_EINVAL, "lt_trace_paths: ray arrays must be non-NULL and 16-byte aligned");
    if (!out->flags) return fail(LT_EINVAL, "lt_trace_paths: NULL flags array");
    RaysInDev din{in->x, in->y, in->dx, in->dy, in->dz, lam};
    PathsOutDev dout{out->x, out->y, out->dx, out->dy, out->dz, out->I, out->flags,
                     out->ray_index, out->valid_count, out->capacity};
    const uint32_t nn = (uint32_t)n;
    const dim3 grid((unsigned)((n + kPathsBlock - 1) / kPathsBlock), (unsigned)n_paths);
    ProfScope prof("trace_paths_kernel", st);
    if (lens_all_cauchy(L->dev))
        trace_paths_kernel<true><<<grid, kPathsBlock, 0, st>>>(L->dev, P, din, lam_stride, dout, nn,
                                                               prof.work());
    else
        trace_paths_kernel<false><<<grid, kPathsBlock, 0, st>>>(L->dev, P, din, lam_stride, dout, nn,
                                                                prof.work());
    LT_CUDA_TRY(cudaGetLastError());
    return LT_OK;
}
