// Many paths in one launch (lt_trace_paths): the flare workload of Sec. 4.2,
// where the same entrance rays follow the main path and every two-bounce
// ghost (i, j), each path with its own wavelength draw; and the same trace
// splatted onto the sensor as it goes (lt_splat_paths: forward light
// tracing, Sec. 3, Eq. 8).
//
// A wavefront per wave of paths: the front kernel (grid: tile of 256 rays x
// path) takes every ray through its first interactions, where most rays of a
// lens die; the survivors of all the wave's paths are queued and a
// persistent rest kernel traces them to the end in dense warps.  Valid rays
// are compacted into their path's segment: lanes grouped by path, one atomic
// on the path's counter per group, rank-ordered writes.
#include "profile.h"
#include "rays.cuh"
#include "tracer.cuh"

namespace lt {

constexpr int kPathsBlock = 256;
constexpr int kMaxPaths = 1024;
constexpr size_t kWavePairs = (size_t)1 << 24;   // (path, ray) pairs per front/rest pair

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

// Append a finished valid ray to its path's segment.  Lanes of a warp may
// hold different paths: lanes of one path are grouped, and each group's
// first lane takes one atomic on the path's counter.
__device__ __forceinline__ void paths_append(const PathsOutDev& out, bool v, int p, uint32_t r,
                                             const RayState& st)
{
    const unsigned full = 0xffffffffu;
    const unsigned act = __ballot_sync(full, v);
    if (!act) return;
    const int lane = threadIdx.x & 31;
    const unsigned grp = __match_any_sync(full, v ? p : -1);
    const int leader = __ffs(grp) - 1;
    uint32_t base = 0;
    if (v && lane == leader) base = atomicAdd(out.count + p, (uint32_t)__popc(grp));
    base = __shfl_sync(full, base, leader);
    if (v) {
        const uint32_t k = base + (uint32_t)__popc(grp & ((1u << lane) - 1u));
        if (k < out.capacity) {
            const size_t e = (size_t)p * out.capacity + k;
            __stcs(out.x + e, st.x);
            __stcs(out.y + e, st.y);
            __stcs(out.dx + e, st.dx);
            __stcs(out.dy + e, st.dy);
            __stcs(out.dz + e, st.dz);
            __stcs(out.I + e, st.I);
            __stcs(out.ray_index + e, r);
            out.flags[e] = (uint8_t)st.flags;
        }
    }
}

// What a finished ray becomes: appended to its path's segment, or splatted
// onto the sensor.  Both are called by every lane of the warp (v: the lane's
// ray reached the image plane).
struct AppendEmit {
    PathsOutDev out;
    __device__ __forceinline__ void operator()(bool v, int p, uint32_t r, const RayState& st) const
    {
        paths_append(out, v, p, r, st);
    }
};

// The sensor of lt_splat_paths as the kernels see it: pixel (i, j)'s centre
// is at continuous pixel coordinate (i, j), u = x / pixel + cx.
struct SplatEmit {
    float* image;
    size_t path_stride;     // floats between two paths' images (0: one image)
    int W, H;
    float inv_px, cx, cy, weight;
    // Eq. 8 for one ray: I * G * h at the (at most four) pixels the tent
    // filter of one pixel radius reaches, G = d_z of the exit direction.
    __device__ __forceinline__ void operator()(bool v, int p, uint32_t, const RayState& st) const
    {
        if (!v) return;
        const float u = fmaf(st.x, inv_px, cx), w = fmaf(st.y, inv_px, cy);
        const float fu = floorf(u), fw = floorf(w);
        const float ax = u - fu, ay = w - fw;
        const int i0 = (int)fu, j0 = (int)fw;
        if (i0 < -1 || i0 >= W || j0 < -1 || j0 >= H) return;
        const float e = st.I * st.dz * weight;
        float* img = image + (size_t)p * path_stride;
        const float wx[2] = {1.0f - ax, ax}, wy[2] = {1.0f - ay, ay};
#pragma unroll
        for (int dj = 0; dj < 2; ++dj) {
            const int j = j0 + dj;
            if (j < 0 || j >= H) continue;
#pragma unroll
            for (int di = 0; di < 2; ++di) {
                const int i = i0 + di;
                if (i < 0 || i >= W) continue;
                atomicAdd(img + (size_t)j * W + i, e * (wx[di] * wy[dj]));
            }
        }
    }
};

// Front of the wavefront: block (tile, path p0 + blockIdx.y), one thread per
// ray through the first kFront interactions; survivors are queued with
// their path.
template <bool CAUCHY, class Emit>
__global__ void __launch_bounds__(kPathsBlock)
paths_front_kernel(const __grid_constant__ LensDev L, const __grid_constant__ PathTable P, int p0,
                   RaysInDev in, size_t lam_stride, Emit emit, uint32_t n, RayQueue Q,
                   unsigned long long* work)
{
    const int p = p0 + (int)blockIdx.y;
    const int pi = P.ij[2 * p], pj = P.ij[2 * p + 1];
    const uint32_t r = blockIdx.x * kPathsBlock + threadIdx.x;
    const int K = path_length(L.S, pi, pj);
    RayState st;
    bool live = false, valid = false;
    int nint = 0;
    if (r < n) {
        live = trace_init(__ldg(in.x + r), __ldg(in.y + r), __ldg(in.dx + r), __ldg(in.dy + r),
                          __ldg(in.dz + r), __ldg(in.lam + (size_t)p * lam_stride + r), st);
        int res = live ? STEP_GO : STEP_DEAD;
        for (int i = 0; i < kFront && res == STEP_GO; ++i) res = trace_step<CAUCHY>(L, pi, pj, K, st);
        if (res != STEP_GO) {
            if (live) nint = st.k + (res == STEP_DONE ? 1 : 0);
            valid = res == STEP_DONE;
            live = false;
        }
    }
    emit(valid, p, r, st);
    queue_push<kPathsBlock>(Q, live, st, r, (uint16_t)p);
    warp_add(work, (unsigned)nint);
}

// Rest of the wavefront: a persistent grid traces the queue to the end.
template <bool CAUCHY, class Emit>
__global__ void __launch_bounds__(kPathsBlock)
paths_rest_kernel(const __grid_constant__ LensDev L, const __grid_constant__ PathTable P, RayQueue Q,
                  Emit emit, unsigned long long* work)
{
    const uint32_t cnt = *Q.count;
    int nint = 0;
    const uint32_t stride = gridDim.x * kPathsBlock;
    // every lane of a warp takes the same number of iterations (the append
    // is warp-collective), idle lanes past the end included
    const uint32_t rounds = (cnt + stride - 1) / stride;
    for (uint32_t q = 0; q < rounds; ++q) {
        const uint32_t i = q * stride + blockIdx.x * kPathsBlock + threadIdx.x;
        RayState st;
        bool valid = false;
        int p = 0;
        uint32_t r = 0;
        if (i < cnt) {
            queue_load(Q, i, st);
            p = Q.path[i];
            r = Q.ray[i];
            const int pi = P.ij[2 * p], pj = P.ij[2 * p + 1];
            const int K = path_length(L.S, pi, pj);
            int res;
#pragma unroll 1
            do {
                res = trace_step<CAUCHY>(L, pi, pj, K, st);
            } while (res == STEP_GO);
            nint += st.k + (res == STEP_DONE ? 1 : 0);
            valid = res == STEP_DONE;
        }
        emit(valid, p, r, st);
    }
    warp_add(work, (unsigned)nint);
}

}  // namespace lt

using namespace lt;

namespace {

// Validate the path ids into P; LT_OK or an LT_EINVAL naming the caller.
lt_status path_table(const lt_lens* L, const int32_t* path_ids, int32_t n_paths, PathTable& P, const char* who)
{
    if (n_paths < 1 || n_paths > kMaxPaths) return fail(LT_EINVAL, "%s: n_paths must be in [1, %d]", who, kMaxPaths);
    for (int p = 0; p < n_paths; ++p) {
        int pi, pj;
        if (!path_ij(L->S, path_ids[p], &pi, &pj))
            return fail(LT_EINVAL, "%s: bad path id %d at %d", who, path_ids[p], p);
        P.ij[2 * p] = (int8_t)pi;
        P.ij[2 * p + 1] = (int8_t)pj;
    }
    return LT_OK;
}

// The waves of front/rest pairs over n_paths paths of n rays, each finished
// ray handed to `emit`; the queue comes stream-ordered from the pool.
template <class Emit>
lt_status run_paths(const lt_lens* L, const PathTable& P, int32_t n_paths, const RaysInDev& din,
                    size_t lam_stride, const Emit& emit, size_t n, cudaStream_t st, const char* prof_name,
                    const char* who)
{
    const uint32_t nn = (uint32_t)n;
    const bool cauchy = lens_all_cauchy(L->dev);
    // waves of whole paths, at most 2^24 (path, ray) pairs (one path at least)
    const int per_wave = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_paths, kWavePairs / n));
    const size_t cap = (((size_t)per_wave * n) + 63) & ~(size_t)63;
    cudaMemPool_t pool;
    lt_status s = scratch_pool(&pool);
    if (s != LT_OK) return s;
    char* buf = nullptr;
    if (cudaMallocFromPoolAsync((void**)&buf, cap * kQueueBytesPerRay + 256, pool, st) != cudaSuccess)
        return fail(LT_ENOMEM, "%s: ray queue allocation of %zu bytes failed", who, cap * kQueueBytesPerRay + 256);
    RayQueue Q;
    float** fq[10] = {&Q.x, &Q.y, &Q.z, &Q.dx, &Q.dy, &Q.dz, &Q.I, &Q.n, &Q.il2, &Q.l2};
    for (int q = 0; q < 10; ++q) *fq[q] = reinterpret_cast<float*>(buf + (size_t)q * cap * 4);
    Q.k = reinterpret_cast<int*>(buf + 10 * cap * 4);
    Q.flags = reinterpret_cast<uint32_t*>(buf + 11 * cap * 4);
    Q.ray = reinterpret_cast<uint32_t*>(buf + 12 * cap * 4);
    Q.path = reinterpret_cast<uint16_t*>(buf + 13 * cap * 4);
    Q.count = reinterpret_cast<uint32_t*>(buf + 13 * cap * 4 + cap * 2 + 64);
    const void* rest = cauchy ? (const void*)paths_rest_kernel<true, Emit> : (const void*)paths_rest_kernel<false, Emit>;
    ProfScope prof(prof_name, st);
    for (int p0 = 0; p0 < n_paths && s == LT_OK; p0 += per_wave) {
        const int np = std::min(per_wave, n_paths - p0);
        const cudaError_t em = cudaMemsetAsync(Q.count, 0, 4, st);
        if (em != cudaSuccess) {
            s = cuda_fail(em, who);
            break;
        }
        const dim3 grid((unsigned)((n + kPathsBlock - 1) / kPathsBlock), (unsigned)np);
        const unsigned gr = persistent_blocks(rest, kPathsBlock, (size_t)np * n, 32);
        if (cauchy) {
            paths_front_kernel<true, Emit><<<grid, kPathsBlock, 0, st>>>(L->dev, P, p0, din, lam_stride, emit, nn, Q, prof.work());
            paths_rest_kernel<true, Emit><<<gr, kPathsBlock, 0, st>>>(L->dev, P, Q, emit, prof.work());
        } else {
            paths_front_kernel<false, Emit><<<grid, kPathsBlock, 0, st>>>(L->dev, P, p0, din, lam_stride, emit, nn, Q, prof.work());
            paths_rest_kernel<false, Emit><<<gr, kPathsBlock, 0, st>>>(L->dev, P, Q, emit, prof.work());
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = cuda_fail(e, who);
    }
    cudaFreeAsync(buf, st);
    return s;
}

}  // namespace

extern "C" lt_status lt_trace_paths(const lt_lens* L, const lt_rays_in* in, const float* lam,
                                    size_t lam_stride, const int32_t* path_ids, int32_t n_paths,
                                    const lt_paths_out* out, size_t n, lt_stream stream)
{
    clear_error();
    if (!L || !in || !out || !path_ids) return fail(LT_EINVAL, "lt_trace_paths: NULL argument");
    if (n >= (1ull << 32)) return fail(LT_EINVAL, "lt_trace_paths: n must be < 2^32");
    if (out->capacity < 1) return fail(LT_EINVAL, "lt_trace_paths: capacity must be >= 1");
    if (!out->valid_count) return fail(LT_EINVAL, "lt_trace_paths: NULL valid_count");
    PathTable P{};
    lt_status s = path_table(L, path_ids, n_paths, P, "lt_trace_paths");
    if (s != LT_OK) return s;
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
    AppendEmit emit{PathsOutDev{out->x, out->y, out->dx, out->dy, out->dz, out->I, out->flags,
                                out->ray_index, out->valid_count, out->capacity}};
    return run_paths(L, P, n_paths, din, lam_stride, emit, n, st, "trace_paths_kernel", "lt_trace_paths");
}

extern "C" lt_status lt_splat_paths(const lt_lens* L, const lt_rays_in* in, const float* lam,
                                    size_t lam_stride, const int32_t* path_ids, int32_t n_paths, size_t n,
                                    const lt_sensor* sensor, float* image, lt_stream stream)
{
    clear_error();
    if (!L || !in || !path_ids || !sensor || !image) return fail(LT_EINVAL, "lt_splat_paths: NULL argument");
    if (n >= (1ull << 32)) return fail(LT_EINVAL, "lt_splat_paths: n must be < 2^32");
    if (sensor->width < 1 || sensor->height < 1 || sensor->width > 65536 || sensor->height > 65536)
        return fail(LT_EINVAL, "lt_splat_paths: sensor of %d x %d pixels", sensor->width, sensor->height);
    if (!(sensor->pixel_mm > 0.0)) return fail(LT_EINVAL, "lt_splat_paths: pixel_mm must be > 0");
    PathTable P{};
    lt_status s = path_table(L, path_ids, n_paths, P, "lt_splat_paths");
    if (s != LT_OK) return s;
    if (n == 0) return LT_OK;
    const void* ps[] = {in->x, in->y, in->dx, in->dy, in->dz, lam, image};
    for (const void* q : ps)
        if (!q || !aligned16(q))
            return fail(LT_EINVAL, "lt_splat_paths: arrays must be non-NULL and 16-byte aligned");
    RaysInDev din{in->x, in->y, in->dx, in->dy, in->dz, lam};
    SplatEmit emit;
    emit.image = image;
    emit.path_stride = sensor->per_path ? (size_t)sensor->width * sensor->height : 0;
    emit.W = sensor->width;
    emit.H = sensor->height;
    emit.inv_px = (float)(1.0 / sensor->pixel_mm);
    emit.cx = (float)(sensor->width / 2.0 - 0.5);
    emit.cy = (float)(sensor->height / 2.0 - 0.5);
    emit.weight = sensor->weight;
    return run_paths(L, P, n_paths, din, lam_stride, emit, n, (cudaStream_t)stream, "splat_paths_kernel",
                     "lt_splat_paths");
}
