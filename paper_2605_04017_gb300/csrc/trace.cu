// Tracing kernels and the lt_trace / lt_trace_host entry points.
#include <algorithm>
#include <mutex>

#include "profile.h"
#include "rays.cuh"
#include "tracer.cuh"

namespace lt {

constexpr int kTraceBlock = 256;

// One thread per ray.  Inputs are read once through the non-coherent path,
// outputs written with an evict-first hint (nothing here re-reads them).
template <bool CAUCHY>
__global__ void __launch_bounds__(kTraceBlock)
trace_kernel(const __grid_constant__ LensDev L, int pi, int pj, RaysInDev in, RaysOutDev out,
             uint32_t n, unsigned long long* work)
{
    const uint32_t r = blockIdx.x * kTraceBlock + threadIdx.x;
    int nint = 0;
    if (r < n) {
        TraceOut o;
        const uint32_t f = trace_ray<CAUCHY>(L, pi, pj, __ldg(in.x + r), __ldg(in.y + r),
                                             __ldg(in.dx + r), __ldg(in.dy + r), __ldg(in.dz + r),
                                             __ldg(in.lam + r), o, nint);
        __stcs(out.x + r, o.x);
        __stcs(out.y + r, o.y);
        __stcs(out.dx + r, o.dx);
        __stcs(out.dy + r, o.dy);
        __stcs(out.dz + r, o.dz);
        __stcs(out.I + r, o.I);
        out.flags[r] = (uint8_t)f;
    }
    warp_add(work, (unsigned)nint);
}

// Grid of a persistent kernel: resident blocks per SM x SMs, but no more warps
// than there are chunks of work.
unsigned persistent_blocks(const void* kernel, int block, size_t items, size_t per_warp)
{
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
    if (per_sm < 1) per_sm = 1;
    const size_t warps_needed = (items + per_warp - 1) / per_warp;
    const size_t blocks_needed = (warps_needed * 32 + block - 1) / block;
    size_t g = (size_t)sms * per_sm;
    if (blocks_needed < g) g = blocks_needed;
    return (unsigned)(g ? g : 1);
}

lt_status launch_trace(const lt_lens* L, int pi, int pj, const RaysInDev& in,
                       const RaysOutDev& out, size_t n, cudaStream_t st)
{
    const bool cauchy = lens_all_cauchy(L->dev);
    for (size_t off = 0; off < n; off += ((size_t)1 << 30)) {
        const uint32_t m = (uint32_t)std::min<size_t>(n - off, (size_t)1 << 30);
        RaysInDev a{in.x + off, in.y + off, in.dx + off, in.dy + off, in.dz + off, in.lam + off};
        RaysOutDev b{out.x + off, out.y + off, out.dx + off, out.dy + off, out.dz + off,
                     out.I + off, out.flags + off};
        ProfScope prof("trace_kernel", st);
        const unsigned g = (m + kTraceBlock - 1) / kTraceBlock;
        if (cauchy)
            trace_kernel<true><<<g, kTraceBlock, 0, st>>>(L->dev, pi, pj, a, b, m, prof.work());
        else
            trace_kernel<false><<<g, kTraceBlock, 0, st>>>(L->dev, pi, pj, a, b, m, prof.work());
        LT_CUDA_TRY(cudaGetLastError());
    }
    return LT_OK;
}

// ---------------------------------------------------------------- host staging

Staging& host_staging()
{
    static Staging s;
    return s;
}

lt_status check_io(const lt_rays_in* in, const float* lam, const lt_rays_out* out, size_t n,
                   const char* who)
{
    if (!in || !out) return fail(LT_EINVAL, "%s: NULL ray struct", who);
    if (n == 0) return LT_OK;
    const void* ps[] = {in->x, in->y, in->dx, in->dy, in->dz, lam, out->x, out->y,
                        out->dx, out->dy, out->dz, out->I};
    for (const void* p : ps) {
        if (!p) return fail(LT_EINVAL, "%s: NULL ray array with n = %zu", who, n);
        if (!aligned16(p)) return fail(LT_EINVAL, "%s: ray arrays must be 16-byte aligned", who);
    }
    if (!out->flags) return fail(LT_EINVAL, "%s: NULL flags array", who);
    return LT_OK;
}

}  // namespace lt

using namespace lt;

extern "C" {

lt_status lt_trace(const lt_lens* L, const lt_rays_in* in, const float* lam, int32_t path_id,
                   const lt_rays_out* out, size_t n, lt_stream stream)
{
    clear_error();
    if (!L) return fail(LT_EINVAL, "lt_trace: NULL lens");
    int pi, pj;
    if (!path_ij(L->S, path_id, &pi, &pj)) return fail(LT_EINVAL, "lt_trace: bad path id %d", path_id);
    lt_status s = check_io(in, lam, out, n, "lt_trace");
    if (s != LT_OK || n == 0) return s;
    RaysInDev din{in->x, in->y, in->dx, in->dy, in->dz, lam};
    RaysOutDev dout{out->x, out->y, out->dx, out->dy, out->dz, out->I, out->flags};
    return launch_trace(L, pi, pj, din, dout, n, (cudaStream_t)stream);
}

lt_status lt_trace_host(const lt_lens* L, const lt_rays_in* in, const float* lam,
                        int32_t path_id, const lt_rays_out* out, size_t n)
{
    clear_error();
    if (!L) return fail(LT_EINVAL, "lt_trace_host: NULL lens");
    int pi, pj;
    if (!path_ij(L->S, path_id, &pi, &pj))
        return fail(LT_EINVAL, "lt_trace_host: bad path id %d", path_id);
    if (!in || !out) return fail(LT_EINVAL, "lt_trace_host: NULL ray struct");
    if (n == 0) return LT_OK;
    const void* ps[] = {in->x, in->y, in->dx, in->dy, in->dz, lam, out->x, out->y,
                        out->dx, out->dy, out->dz, out->I, out->flags};
    for (const void* p : ps)
        if (!p) return fail(LT_EINVAL, "lt_trace_host: NULL ray array");
    return run_host_pipelined(in, lam, out, n,
                              [&](const RaysInDev& a, const RaysOutDev& b, size_t m,
                                  cudaStream_t st) { return launch_trace(L, pi, pj, a, b, m, st); });
}

}  // extern "C"
