// Tracing kernels and the lt_trace / lt_trace_host entry points.
#include <algorithm>
#include <mutex>

#include "profile.h"
#include "rays.cuh"
#include "tracer.cuh"

namespace lt {

constexpr int kTraceBlock = 256;

// The tracer runs as a two-kernel wavefront.  Most rays of a real lens die
// at its first surfaces (the entrance disk overfills the front aperture),
// the rest go on to the image; one thread per ray would keep each warp
// running to its longest ray with most lanes idle.
//  - trace_front_kernel: one thread per ray through the first kFront
//    interactions; finished rays are written at once (survivors' rows get a
//    placeholder), survivors' states go to a queue (block-aggregated appends,
//    structure of arrays).
//  - trace_rest_kernel: a persistent grid traces the queue to the end with
//    every lane busy and writes each result at its ray's index.
// Per-ray arithmetic is that of trace_ray, bit for bit.
// Paths of up to kShortPath interactions (the whole path is about as long
// as the front) run instead as one block-compacting kernel (trace_block),
// where queueing survivors would cost more than it saves.
constexpr int kShortPath = 4;
constexpr size_t kWaveRays = (size_t)1 << 24;   // rays per front/rest pair (queue <= 872 MB)

template <bool CAUCHY, bool MAIN>
__global__ void __launch_bounds__(kTraceBlock)
trace_short_kernel(const __grid_constant__ LensDev L, int pi, int pj, RaysInDev in, RaysOutDev out,
                   uint32_t n, unsigned long long* work)
{
    __shared__ TraceSmem<kTraceBlock> S;
    const uint32_t r0 = blockIdx.x * kTraceBlock;
    const int nint = trace_block<CAUCHY, kTraceBlock, MAIN>(L, pi, pj, in.x, in.y, in.dx, in.dy, in.dz, in.lam,
                                                            n, r0, S);
    __syncthreads();
    const int t = threadIdx.x;
    const uint32_t r = r0 + (uint32_t)t;
    if (r < n) {
        __stcs(out.x + r, S.ob[0][t]);
        __stcs(out.y + r, S.ob[1][t]);
        __stcs(out.dx + r, S.ob[2][t]);
        __stcs(out.dy + r, S.ob[3][t]);
        __stcs(out.dz + r, S.ob[4][t]);
        __stcs(out.I + r, S.ob[5][t]);
        out.flags[r] = S.of[t];
    }
    warp_add(work, (unsigned)nint);
}


__device__ __forceinline__ void store_result(const RaysOutDev& out, uint32_t r, const RayState& st, int res)
{
    const bool done = res == STEP_DONE;
    __stcs(out.x + r, done ? st.x : 0.0f);
    __stcs(out.y + r, done ? st.y : 0.0f);
    __stcs(out.dx + r, done ? st.dx : 0.0f);
    __stcs(out.dy + r, done ? st.dy : 0.0f);
    __stcs(out.dz + r, done ? st.dz : 0.0f);
    __stcs(out.I + r, done ? st.I : 0.0f);
    out.flags[r] = (uint8_t)(done ? st.flags : (st.flags & ~LT_FLAG_VALID));
}

template <bool CAUCHY, bool MAIN>
__global__ void __launch_bounds__(kTraceBlock)
trace_front_kernel(const __grid_constant__ LensDev L, int pi, int pj, RaysInDev in, RaysOutDev out,
                   uint32_t n, RayQueue Q, unsigned long long* work)
{
    const uint32_t r = blockIdx.x * kTraceBlock + threadIdx.x;
    const int K = path_length(L.S, pi, pj);
    RayState st;
    bool live = false;
    int nint = 0;
    if (r < n) {
        live = trace_init(__ldg(in.x + r), __ldg(in.y + r), __ldg(in.dx + r), __ldg(in.dy + r),
                          __ldg(in.dz + r), __ldg(in.lam + r), st);
        int res = live ? STEP_GO : STEP_DEAD;
        for (int i = 0; i < kFront && res == STEP_GO; ++i) res = trace_step<CAUCHY, MAIN>(L, pi, pj, K, st);
        if (res != STEP_GO) {
            if (live) nint = st.k + (res == STEP_DONE ? 1 : 0);
            live = false;
        }
        // Every output row is written here, a survivor's as a placeholder that
        // the rest kernel overwrites: the warp's stores then cover whole
        // sectors, which L2 takes without merging partial lines.
        store_result(out, r, st, live ? STEP_DEAD : res);
    }
    queue_push<kTraceBlock>(Q, live, st, r, 0);
    warp_add(work, (unsigned)nint);
}

template <bool CAUCHY, bool MAIN>
__global__ void __launch_bounds__(kTraceBlock)
trace_rest_kernel(const __grid_constant__ LensDev L, int pi, int pj, RayQueue Q, RaysOutDev out,
                  unsigned long long* work)
{
    const uint32_t cnt = *Q.count;
    const int K = path_length(L.S, pi, pj);
    int nint = 0;
    for (uint32_t i = blockIdx.x * kTraceBlock + threadIdx.x; i < cnt; i += gridDim.x * kTraceBlock) {
        RayState st;
        queue_load(Q, i, st);
        int res;
#pragma unroll 1
        do {
            res = trace_step<CAUCHY, MAIN>(L, pi, pj, K, st);
        } while (res == STEP_GO);
        nint += st.k + (res == STEP_DONE ? 1 : 0);
        store_result(out, Q.ray[i], st, res);
    }
    warp_add(work, (unsigned)nint);
}

// The tracer's reciprocal and square root, element by element (lt_tracer_math).
__global__ void __launch_bounds__(256)
tracer_math_kernel(const float* __restrict__ x, float* __restrict__ rcp, float* __restrict__ sq, size_t n)
{
    const size_t i = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const float v = x[i];
    rcp[i] = rcp_nr(v);
    sq[i] = fast_sqrt(v);
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
    const bool cauchy = lens_all_cauchy(L->dev), main = pj == 0;
    if (path_length(L->S, pi, pj) <= kShortPath) {
        for (size_t off = 0; off < n; off += ((size_t)1 << 30)) {
            const uint32_t m = (uint32_t)std::min<size_t>(n - off, (size_t)1 << 30);
            RaysInDev a{in.x + off, in.y + off, in.dx + off, in.dy + off, in.dz + off, in.lam + off};
            RaysOutDev b{out.x + off, out.y + off, out.dx + off, out.dy + off, out.dz + off,
                         out.I + off, out.flags + off};
            ProfScope prof("trace_kernel", st);
            const unsigned g = (m + kTraceBlock - 1) / kTraceBlock;
            if (cauchy && main) trace_short_kernel<true, true><<<g, kTraceBlock, 0, st>>>(L->dev, pi, pj, a, b, m, prof.work());
            else if (cauchy) trace_short_kernel<true, false><<<g, kTraceBlock, 0, st>>>(L->dev, pi, pj, a, b, m, prof.work());
            else if (main) trace_short_kernel<false, true><<<g, kTraceBlock, 0, st>>>(L->dev, pi, pj, a, b, m, prof.work());
            else trace_short_kernel<false, false><<<g, kTraceBlock, 0, st>>>(L->dev, pi, pj, a, b, m, prof.work());
            LT_CUDA_TRY(cudaGetLastError());
        }
        return LT_OK;
    }
    const size_t wave = std::min(n, kWaveRays);
    cudaMemPool_t pool;
    lt_status s = scratch_pool(&pool);
    if (s != LT_OK) return s;
    const size_t cap = (wave + 63) & ~(size_t)63;
    char* buf = nullptr;
    if (cudaMallocFromPoolAsync((void**)&buf, cap * kQueueBytesPerRay + 256, pool, st) != cudaSuccess)
        return fail(LT_ENOMEM, "lt_trace: ray queue allocation of %zu bytes failed", cap * kQueueBytesPerRay + 256);
    RayQueue Q;
    float** fq[10] = {&Q.x, &Q.y, &Q.z, &Q.dx, &Q.dy, &Q.dz, &Q.I, &Q.n, &Q.il2, &Q.l2};
    for (int q = 0; q < 10; ++q) *fq[q] = reinterpret_cast<float*>(buf + (size_t)q * cap * 4);
    Q.k = reinterpret_cast<int*>(buf + 10 * cap * 4);
    Q.flags = reinterpret_cast<uint32_t*>(buf + 11 * cap * 4);
    Q.ray = reinterpret_cast<uint32_t*>(buf + 12 * cap * 4);
    Q.path = nullptr;
    Q.count = reinterpret_cast<uint32_t*>(buf + 13 * cap * 4);
    const void* rest = cauchy ? (main ? (const void*)trace_rest_kernel<true, true> : (const void*)trace_rest_kernel<true, false>)
                              : (main ? (const void*)trace_rest_kernel<false, true> : (const void*)trace_rest_kernel<false, false>);
    for (size_t off = 0; off < n && s == LT_OK; off += wave) {
        const uint32_t m = (uint32_t)std::min(n - off, wave);
        RaysInDev a{in.x + off, in.y + off, in.dx + off, in.dy + off, in.dz + off, in.lam + off};
        RaysOutDev b{out.x + off, out.y + off, out.dx + off, out.dy + off, out.dz + off,
                     out.I + off, out.flags + off};
        ProfScope prof("trace_kernel", st);
        const cudaError_t em = cudaMemsetAsync(Q.count, 0, 4, st);
        if (em != cudaSuccess) { s = cuda_fail(em, "lt_trace: memset"); break; }
        const unsigned g = (m + kTraceBlock - 1) / kTraceBlock;
        // the rest kernel's grid: resident blocks, no more than the wave could need
        const unsigned gr = persistent_blocks(rest, kTraceBlock, m, 32);
        if (cauchy && main) {
            trace_front_kernel<true, true><<<g, kTraceBlock, 0, st>>>(L->dev, pi, pj, a, b, m, Q, prof.work());
            trace_rest_kernel<true, true><<<gr, kTraceBlock, 0, st>>>(L->dev, pi, pj, Q, b, prof.work());
        } else if (cauchy) {
            trace_front_kernel<true, false><<<g, kTraceBlock, 0, st>>>(L->dev, pi, pj, a, b, m, Q, prof.work());
            trace_rest_kernel<true, false><<<gr, kTraceBlock, 0, st>>>(L->dev, pi, pj, Q, b, prof.work());
        } else if (main) {
            trace_front_kernel<false, true><<<g, kTraceBlock, 0, st>>>(L->dev, pi, pj, a, b, m, Q, prof.work());
            trace_rest_kernel<false, true><<<gr, kTraceBlock, 0, st>>>(L->dev, pi, pj, Q, b, prof.work());
        } else {
            trace_front_kernel<false, false><<<g, kTraceBlock, 0, st>>>(L->dev, pi, pj, a, b, m, Q, prof.work());
            trace_rest_kernel<false, false><<<gr, kTraceBlock, 0, st>>>(L->dev, pi, pj, Q, b, prof.work());
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = cuda_fail(e, "lt_trace: launch");
    }
    cudaFreeAsync(buf, st);
    return s;
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

lt_status lt_tracer_math(const float* x, float* rcp, float* sqrt_out, size_t n, lt_stream stream)
{
    clear_error();
    if (n == 0) return LT_OK;
    if (!x || !rcp || !sqrt_out) return fail(LT_EINVAL, "lt_tracer_math: NULL array with n = %zu", n);
    if (n > ((size_t)1 << 38)) return fail(LT_EINVAL, "lt_tracer_math: n = %zu is too large", n);
    const size_t blocks = (n + 255) / 256;
    tracer_math_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(x, rcp, sqrt_out, n);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LT_OK : cuda_fail(e, "lt_tracer_math: launch");
}

}  // extern "C"
