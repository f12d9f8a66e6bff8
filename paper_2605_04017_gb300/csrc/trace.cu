// Tracing kernels and the lt_trace / lt_trace_host entry points.
#include <algorithm>
#include <mutex>

#include "tracer.cuh"

namespace lt {

struct RaysInDev {
    const float *__restrict__ x, *__restrict__ y, *__restrict__ dx, *__restrict__ dy,
        *__restrict__ dz, *__restrict__ lam;
};
struct RaysOutDev {
    float *__restrict__ x, *__restrict__ y, *__restrict__ dx, *__restrict__ dy, *__restrict__ dz,
        *__restrict__ I;
    uint8_t* __restrict__ flags;
};

constexpr int kTraceBlock = 256;

// One thread per ray.  Inputs are read once through the non-coherent path,
// outputs are written with an evict-first hint (nothing re-reads them here).
__global__ void __launch_bounds__(kTraceBlock)
trace_kernel(const __grid_constant__ LensDev L, int pi, int pj, RaysInDev in, RaysOutDev out,
             size_t n)
{
    const size_t r = (size_t)blockIdx.x * kTraceBlock + threadIdx.x;
    if (r >= n) return;
    TraceOut o;
    const uint32_t f = trace_ray(L, pi, pj, __ldg(in.x + r), __ldg(in.y + r), __ldg(in.dx + r),
                                 __ldg(in.dy + r), __ldg(in.dz + r), __ldg(in.lam + r), o);
    __stcs(out.x + r, o.x);
    __stcs(out.y + r, o.y);
    __stcs(out.dx + r, o.dx);
    __stcs(out.dy + r, o.dy);
    __stcs(out.dz + r, o.dz);
    __stcs(out.I + r, o.I);
    out.flags[r] = (uint8_t)f;
}

static lt_status check_io(const lt_rays_in* in, const float* lam, const lt_rays_out* out,
                          size_t n, const char* who)
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

lt_status launch_trace(const lt_lens* L, int pi, int pj, const RaysInDev& in,
                       const RaysOutDev& out, size_t n, cudaStream_t st)
{
    if (n == 0) return LT_OK;
    const size_t blocks = (n + kTraceBlock - 1) / kTraceBlock;
    trace_kernel<<<(unsigned)blocks, kTraceBlock, 0, st>>>(L->dev, pi, pj, in, out, n);
    LT_CUDA_TRY(cudaGetLastError());
    return LT_OK;
}

// ---------------------------------------------------------------- host staging

// Pipelined host <-> device staging for the *_host entry points: two streams,
// each with its own device buffers; chunk c goes to stream c % 2 so copies of
// one chunk overlap the kernel of the other.
struct Staging {
    int device = -1;
    size_t cap = 0;
    cudaStream_t st[2] = {nullptr, nullptr};
    float* in[2][6] = {};
    float* out[2][6] = {};
    uint8_t* flags[2] = {};
    std::mutex mu;

    void release()
    {
        for (int b = 0; b < 2; ++b) {
            for (int q = 0; q < 6; ++q) {
                if (in[b][q]) cudaFree(in[b][q]);
                if (out[b][q]) cudaFree(out[b][q]);
                in[b][q] = out[b][q] = nullptr;
            }
            if (flags[b]) cudaFree(flags[b]);
            flags[b] = nullptr;
        }
        cap = 0;
    }

    lt_status reserve(size_t chunk)
    {
        int dev = 0;
        LT_CUDA_TRY(cudaGetDevice(&dev));
        if (dev != device) {
            // buffers of another device are left to process exit
            for (int b = 0; b < 2; ++b) st[b] = nullptr;
            for (int b = 0; b < 2; ++b) {
                for (int q = 0; q < 6; ++q) in[b][q] = out[b][q] = nullptr;
                flags[b] = nullptr;
            }
            cap = 0;
            device = dev;
        }
        for (int b = 0; b < 2; ++b)
            if (!st[b]) LT_CUDA_TRY(cudaStreamCreateWithFlags(&st[b], cudaStreamNonBlocking));
        if (chunk <= cap) return LT_OK;
        release();
        for (int b = 0; b < 2; ++b) {
            for (int q = 0; q < 6; ++q) {
                if (cudaMalloc(&in[b][q], chunk * sizeof(float)) != cudaSuccess ||
                    cudaMalloc(&out[b][q], chunk * sizeof(float)) != cudaSuccess) {
                    release();
                    return fail(LT_ENOMEM, "host staging: cudaMalloc failed");
                }
            }
            if (cudaMalloc(&flags[b], chunk) != cudaSuccess) {
                release();
                return fail(LT_ENOMEM, "host staging: cudaMalloc failed");
            }
        }
        cap = chunk;
        return LT_OK;
    }
};

static Staging g_staging;

size_t host_chunk(size_t n)
{
    // at least 4 chunks for overlap, at most 2^21 rays (~100 MB staged per buffer set)
    size_t c = (n + 3) / 4;
    c = std::max<size_t>(c, 65536);
    c = std::min<size_t>(c, (size_t)1 << 21);
    return (c + 63) & ~(size_t)63;
}

// Runs `kernel(in, out, m, stream)` over host arrays in pipelined chunks.
template <class Launch>
lt_status run_host_pipelined(const lt_rays_in* in, const float* lam, const lt_rays_out* out,
                             size_t n, Launch&& launch)
{
    std::lock_guard<std::mutex> lock(g_staging.mu);
    const size_t chunk = host_chunk(n);
    lt_status s = g_staging.reserve(chunk);
    if (s != LT_OK) return s;
    const float* hin[6] = {in->x, in->y, in->dx, in->dy, in->dz, lam};
    float* hout[6] = {out->x, out->y, out->dx, out->dy, out->dz, out->I};
    for (size_t off = 0, c = 0; off < n; off += chunk, ++c) {
        const int b = (int)(c & 1);
        cudaStream_t st = g_staging.st[b];
        const size_t m = std::min(chunk, n - off);
        for (int q = 0; q < 6; ++q)
            LT_CUDA_TRY(cudaMemcpyAsync(g_staging.in[b][q], hin[q] + off, m * sizeof(float),
                                        cudaMemcpyHostToDevice, st));
        RaysInDev din{g_staging.in[b][0], g_staging.in[b][1], g_staging.in[b][2],
                      g_staging.in[b][3], g_staging.in[b][4], g_staging.in[b][5]};
        RaysOutDev dout{g_staging.out[b][0], g_staging.out[b][1], g_staging.out[b][2],
                        g_staging.out[b][3], g_staging.out[b][4], g_staging.out[b][5],
                        g_staging.flags[b]};
        s = launch(din, dout, m, st);
        if (s != LT_OK) return s;
        for (int q = 0; q < 6; ++q)
            LT_CUDA_TRY(cudaMemcpyAsync(hout[q] + off, g_staging.out[b][q], m * sizeof(float),
                                        cudaMemcpyDeviceToHost, st));
        LT_CUDA_TRY(cudaMemcpyAsync(out->flags + off, g_staging.flags[b], m,
                                    cudaMemcpyDeviceToHost, st));
    }
    for (int b = 0; b < 2; ++b) LT_CUDA_TRY(cudaStreamSynchronize(g_staging.st[b]));
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
