// Request server (lt_server_*, lt_submit, lt_poll): a native worker thread
// that launches submitted requests on a few streams, fuses small trace
// requests into one launch, holds requests back while their device memory
// would exceed a budget, expires requests past their deadline and reports
// completion through host functions enqueued behind each launch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "map_internal.h"
#include "profile.h"
#include "rays.cuh"
#include "tracer.cuh"

namespace lt {

using Clock = std::chrono::steady_clock;

constexpr int kServeBlock = 256;

struct FuseItem {
    const LensDev* L;     // device copy of the request's lens
    RaysInDev in;
    RaysOutDev out;
    uint32_t n;
    int32_t pi, pj;
};

// The request table of one fused launch, passed by value as the kernel
// parameter (about 15 KB): block b serves the last item whose first tile is
// <= b.
struct FuseTable {
    int n_items;
    uint32_t tile0[kMaxFuse + 1];
    FuseItem item[kMaxFuse];
};

static_assert(sizeof(LensDev) % 16 == 0, "LensDev is staged in 16-byte words");

__global__ void __launch_bounds__(kServeBlock)
serve_trace_kernel(const __grid_constant__ FuseTable T, unsigned long long* work)
{
    __shared__ LensDev sl;
    int lo = 0, hi = T.n_items - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.tile0[mid] <= blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const FuseItem& it = T.item[lo];
    {
        const int4* src = reinterpret_cast<const int4*>(it.L);
        int4* dst = reinterpret_cast<int4*>(&sl);
        for (int k = threadIdx.x; k < (int)(sizeof(LensDev) / 16); k += kServeBlock) dst[k] = __ldg(src + k);
    }
    __syncthreads();
    const uint32_t r = (blockIdx.x - T.tile0[lo]) * kServeBlock + threadIdx.x;
    int nint = 0;
    if (r < it.n) {
        TraceOut o;
        const uint32_t f = trace_ray<false>(sl, it.pi, it.pj, __ldg(it.in.x + r), __ldg(it.in.y + r),
                                            __ldg(it.in.dx + r), __ldg(it.in.dy + r), __ldg(it.in.dz + r),
                                            __ldg(it.in.lam + r), o, nint);
        __stcs(it.out.x + r, o.x);
        __stcs(it.out.y + r, o.y);
        __stcs(it.out.dx + r, o.dx);
        __stcs(it.out.dy + r, o.dy);
        __stcs(it.out.dz + r, o.dz);
        __stcs(it.out.I + r, o.I);
        it.out.flags[r] = (uint8_t)f;
    }
    warp_add(work, (unsigned)nint);
}

struct Ticket {
    lt_status status = LT_ENOTREADY;
    bool done = false;
    int fused = 1;
    Clock::time_point t_submit, t_launch, t_done;
};

struct Pending {
    uint64_t id;
    lt_request req;
    size_t bytes;
    Clock::time_point t_submit;
};

struct LensCopy {
    LensDev host;
    LensDev* dev = nullptr;
};

struct BlobCopy {
    std::vector<unsigned char> host;
    void* dev = nullptr;
};

struct Done;

}  // namespace lt

struct lt_server {
    int device = 0;
    lt_server_opts o{};
    std::vector<cudaStream_t> streams;
    size_t next_stream = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<lt::Pending> pending;
    std::unordered_map<uint64_t, lt::Ticket> tickets;
    uint64_t next_id = 1;
    size_t bytes_in_flight = 0;
    uint64_t launch_counter = 0;
    bool stop = false;
    lt_server_stats stats{};
    std::unordered_map<const lt_lens*, lt::LensCopy> lens_cache;   // worker thread only
    std::vector<lt::LensDev*> retired_lens;                         // freed at destroy
    // device copies of maps' and learned maps' constants for fused launches,
    // keyed by (object, precision) (worker thread only); stale copies are
    // kept until destroy, like the lenses'
    std::map<std::pair<const void*, int>, lt::BlobCopy> blob_cache;
    std::vector<void*> retired_blobs;
    std::thread worker;
};

namespace lt {

struct Done {
    lt_server* s;
    std::vector<uint64_t> ids;
    size_t bytes;
};

// Completes tickets with `st` (callers hold s->mu).
static void complete_locked(lt_server* s, const std::vector<uint64_t>& ids, lt_status st, Clock::time_point now)
{
    for (uint64_t id : ids) {
        auto t = s->tickets.find(id);
        if (t == s->tickets.end()) continue;
        t->second.done = true;
        t->second.status = st;
        t->second.t_done = now;
        if (st == LT_OK) s->stats.completed++;
        else if (st == LT_ETIMEOUT) s->stats.timed_out++;
        else s->stats.failed++;
    }
}

// Host function behind a launch: runs on a CUDA-owned thread once the
// stream has passed the launch; it makes no CUDA calls.
static void CUDART_CB on_done(void* p)
{
    Done* d = static_cast<Done*>(p);
    lt_server* s = d->s;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        complete_locked(s, d->ids, LT_OK, Clock::now());
        s->bytes_in_flight -= d->bytes;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    delete d;
}

static size_t round16(size_t b) { return (b + 15) & ~(size_t)15; }

// Device bytes a request holds while in flight: host staging, the ray
// queue of the tracer's second kernel (kQueueBytesPerRay per ray of a wave
// of at most 2^24 rays) for a trace launched on its own, and the trace
// queue of a map query (with a polynomial-patch map's sorted records).
static size_t request_bytes(const lt_request& r, size_t fuse_max_rays)
{
    size_t b = 0;
    if (r.flags & LT_REQ_HOST_BUFFERS) b += 12 * round16(r.n * 4) + round16(r.n);
    if (r.kind == LT_REQ_TRACE && (r.n > fuse_max_rays || (r.flags & LT_REQ_HOST_BUFFERS)))
        b += (std::min(r.n, (size_t)1 << 24) + 64) * kQueueBytesPerRay + 256;
    if (r.kind == LT_REQ_QUERY)
        b += r.map && r.map->kind == LT_MAP_KIND_POLY ? poly_scratch_bytes(r.n, r.map->pstats.patches)
                                                      : query_scratch_bytes(r.n);
    return b;
}

static lt_status lens_on_device(lt_server* s, const lt_lens* L, const LensDev** out)
{
    LensCopy& c = s->lens_cache[L];
    if (!c.dev || std::memcmp(&c.host, &L->dev, sizeof(LensDev)) != 0) {
        // a new lens, or another lens now at the same address: a fresh copy
        // (an older copy may still be read by a launch in flight, so it is
        // kept until the server is destroyed)
        LensDev* d = nullptr;
        LT_CUDA_TRY(cudaMalloc(&d, sizeof(LensDev)));
        LT_CUDA_TRY(cudaMemcpy(d, &L->dev, sizeof(LensDev), cudaMemcpyHostToDevice));
        if (c.dev) s->retired_lens.push_back(c.dev);
        c.dev = d;
        c.host = L->dev;
    }
    *out = c.dev;
    return LT_OK;
}

// One request on its own (device buffers already resolved).
static lt_status launch_single(const lt_request& r, const RaysInDev& in, const RaysOutDev& out,
                               cudaStream_t st)
{
    if (r.kind == LT_REQ_TRACE) {
        int pi, pj;
        path_ij(r.lens->S, r.path_id, &pi, &pj);
        return launch_trace(r.lens, pi, pj, in, out, r.n, st);
    }
    if (r.kind == LT_REQ_QUERY) return launch_query(r.map, in, out, (uint32_t)r.n, r.query_mode, st);
    lt_rays_in ri{in.x, in.y, in.dx, in.dy, in.dz};
    lt_rays_out ro{out.x, out.y, out.dx, out.dy, out.dz, out.I, out.flags};
    return lt_mlp_query(r.mlp, &ri, in.lam, &ro, r.n, r.precision, (lt_stream)st);
}

// A request with host buffers: stage in, run, stage out, on one stream.
static lt_status launch_staged(const lt_request& r, cudaStream_t st)
{
    cudaMemPool_t pool;
    lt_status s = scratch_pool(&pool);
    if (s != LT_OK) return s;
    const size_t a = round16(r.n * 4);
    char* buf = nullptr;
    if (cudaMallocFromPoolAsync((void**)&buf, 12 * a + round16(r.n), pool, st) != cudaSuccess)
        return fail(LT_ENOMEM, "server: staging allocation of %zu bytes failed", 12 * a + round16(r.n));
    float* f[12];
    for (int q = 0; q < 12; ++q) f[q] = reinterpret_cast<float*>(buf + q * a);
    uint8_t* flags = reinterpret_cast<uint8_t*>(buf + 12 * a);
    const float* hin[6] = {r.in.x, r.in.y, r.in.dx, r.in.dy, r.in.dz, r.lambda_nm};
    float* hout[6] = {r.out.x, r.out.y, r.out.dx, r.out.dy, r.out.dz, r.out.I};
    for (int q = 0; q < 6 && s == LT_OK; ++q)
        if (cudaMemcpyAsync(f[q], hin[q], r.n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
            s = cuda_fail(cudaGetLastError(), "server: input copy");
    if (s == LT_OK) {
        RaysInDev in{f[0], f[1], f[2], f[3], f[4], f[5]};
        RaysOutDev out{f[6], f[7], f[8], f[9], f[10], f[11], flags};
        s = launch_single(r, in, out, st);
    }
    for (int q = 0; q < 6 && s == LT_OK; ++q)
        if (cudaMemcpyAsync(hout[q], f[6 + q], r.n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            s = cuda_fail(cudaGetLastError(), "server: output copy");
    if (s == LT_OK && cudaMemcpyAsync(r.out.flags, flags, r.n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = cuda_fail(cudaGetLastError(), "server: flags copy");
    cudaFreeAsync(buf, st);
    return s;
}

// Requests that may share a launch: small requests on device buffers whose
// kernels are the same instantiation.  *key names that group: traces (any
// lens, any path), table-map queries by mode, node format and dispersion form,
// polynomial-patch map queries (LT_QUERY_TABLE only) by degree and
// dispersion form, learned-map queries by precision.
static bool fusable(const lt_server* s, const lt_request& r, int* key)
{
    if ((r.flags & LT_REQ_HOST_BUFFERS) || r.n > s->o.fuse_max_rays || s->o.fuse_max_requests < 2) return false;
    if (r.kind == LT_REQ_TRACE) {
        *key = 0;
        return true;
    }
    if (r.kind == LT_REQ_QUERY) {
        if (r.map->kind == LT_MAP_KIND_POLY) {
            if (r.query_mode != LT_QUERY_TABLE) return false;
            *key = 2000 + 2 * r.map->pdev.degree + (r.map->cauchy ? 1 : 0);
        } else {
            *key = 1000 + 4 * r.query_mode + 2 * (r.map->node_format == LT_NODE_S16 ? 1 : 0) + (r.map->cauchy ? 1 : 0);
        }
        return true;
    }
    *key = 3000 + r.precision;
    return true;
}

// The device copy of a request's map or learned-map constants (made once per
// object and precision, renewed if the object at that address changed).
static lt_status blob_on_device(lt_server* s, const lt_request& r, const void** out)
{
    std::vector<unsigned char> b;
    const void* obj = r.kind == LT_REQ_QUERY ? (const void*)r.map : (const void*)r.mlp;
    const int variant = r.kind == LT_REQ_QUERY ? -1 : r.precision;
    const lt_status st = r.kind == LT_REQ_QUERY ? serve_blob(r.map, b) : mlp_serve_blob(r.mlp, r.precision, b);
    if (st != LT_OK) return st;
    BlobCopy& c = s->blob_cache[std::make_pair(obj, variant)];
    if (!c.dev || c.host != b) {
        void* d = nullptr;
        LT_CUDA_TRY(cudaMalloc(&d, b.size()));
        LT_CUDA_TRY(cudaMemcpy(d, b.data(), b.size(), cudaMemcpyHostToDevice));
        if (c.dev) s->retired_blobs.push_back(c.dev);
        c.dev = d;
        c.host.swap(b);
    }
    *out = c.dev;
    return LT_OK;
}

// Finishes one launch: either enqueue the completion host function or, if
// the launch failed, complete its requests with the error now.
static void finish_launch(lt_server* s, cudaStream_t st, std::vector<uint64_t> ids, size_t bytes, size_t rays,
                          bool fused, lt_status ls)
{
    const Clock::time_point now = Clock::now();
    Done* d = nullptr;
    if (ls == LT_OK) {
        d = new Done{s, ids, bytes};
        if (cudaLaunchHostFunc(st, on_done, d) != cudaSuccess) {
            ls = cuda_fail(cudaGetLastError(), "server: completion callback");
            delete d;
            d = nullptr;
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    for (uint64_t id : ids) {
        auto t = s->tickets.find(id);
        if (t == s->tickets.end()) continue;
        t->second.t_launch = now;
        t->second.fused = (int)ids.size();
    }
    s->stats.launches++;
    s->stats.rays += rays;
    if (fused) {
        s->stats.fused_launches++;
        s->stats.fused_requests += ids.size();
    }
    if (ls != LT_OK) {
        complete_locked(s, ids, ls, now);
        s->bytes_in_flight -= bytes;
        s->cv_done.notify_all();
    }
}

// Host-side fault injection: the k-th launch is not made.
static bool injected_failure(lt_server* s)
{
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t k = ++s->launch_counter;
    return s->o.inject_fail_every > 0 && k % (uint64_t)s->o.inject_fail_every == 0;
}

static void launch_fused(lt_server* s, std::vector<Pending>& group)
{
    if (group.empty()) return;
    cudaStream_t st = s->streams[s->next_stream++ % s->streams.size()];
    std::vector<uint64_t> ids;
    size_t bytes = 0, rays = 0;
    FuseTable T;
    T.n_items = 0;
    uint32_t tiles = 0;
    lt_status ls = LT_OK;
    for (Pending& p : group) {
        ids.push_back(p.id);
        bytes += p.bytes;
        rays += p.req.n;
        const LensDev* Ld = nullptr;
        if (ls == LT_OK) ls = lens_on_device(s, p.req.lens, &Ld);
        if (ls != LT_OK) continue;
        FuseItem& it = T.item[T.n_items];
        it.L = Ld;
        it.in = RaysInDev{p.req.in.x, p.req.in.y, p.req.in.dx, p.req.in.dy, p.req.in.dz, p.req.lambda_nm};
        it.out = RaysOutDev{p.req.out.x, p.req.out.y, p.req.out.dx, p.req.out.dy, p.req.out.dz, p.req.out.I,
                            p.req.out.flags};
        it.n = (uint32_t)p.req.n;
        path_ij(p.req.lens->S, p.req.path_id, &it.pi, &it.pj);
        T.tile0[T.n_items] = tiles;
        tiles += (uint32_t)((p.req.n + kServeBlock - 1) / kServeBlock);
        T.n_items++;
    }
    T.tile0[T.n_items] = tiles;
    if (ls == LT_OK && injected_failure(s)) ls = fail(LT_ECUDA, "server: injected launch failure");
    if (ls == LT_OK) {
        ProfScope prof("serve_trace_kernel", st);
        serve_trace_kernel<<<tiles, kServeBlock, 0, st>>>(T, prof.work());
        if (cudaGetLastError() != cudaSuccess) ls = cuda_fail(cudaGetLastError(), "server: fused launch");
    }
    finish_launch(s, st, ids, bytes, rays, true, ls);
    group.clear();
}

// A fused launch of map or learned-map queries (every request of the group
// has the same fusion key).
static void launch_fused_queries(lt_server* s, std::vector<Pending>& group)
{
    if (group.empty()) return;
    cudaStream_t st = s->streams[s->next_stream++ % s->streams.size()];
    const lt_request& r0 = group[0].req;
    const uint32_t rpb = r0.kind == LT_REQ_QUERY ? kFusedQueryRays : fused_mlp_rays(r0.precision);
    std::vector<uint64_t> ids;
    size_t bytes = 0, rays = 0;
    ReqTable T;
    T.n_items = 0;
    uint32_t blocks = 0;
    lt_status ls = LT_OK;
    for (Pending& p : group) {
        ids.push_back(p.id);
        bytes += p.bytes;
        rays += p.req.n;
        const void* dev = nullptr;
        if (ls == LT_OK) ls = blob_on_device(s, p.req, &dev);
        if (ls != LT_OK) continue;
        ReqItem& it = T.item[T.n_items];
        it.dev = dev;
        it.in = RaysInDev{p.req.in.x, p.req.in.y, p.req.in.dx, p.req.in.dy, p.req.in.dz, p.req.lambda_nm};
        it.out = RaysOutDev{p.req.out.x, p.req.out.y, p.req.out.dx, p.req.out.dy, p.req.out.dz, p.req.out.I,
                            p.req.out.flags};
        it.n = (uint32_t)p.req.n;
        T.block0[T.n_items] = blocks;
        blocks += (uint32_t)((p.req.n + rpb - 1) / rpb);
        T.n_items++;
    }
    T.block0[T.n_items] = blocks;
    if (ls == LT_OK && injected_failure(s)) ls = fail(LT_ECUDA, "server: injected launch failure");
    if (ls == LT_OK) {
        if (r0.kind == LT_REQ_MLP) ls = launch_fused_mlp(T, r0.precision, st);
        else if (r0.map->kind == LT_MAP_KIND_POLY)
            ls = launch_fused_poly(T, r0.map->pdev.degree, r0.query_mode, r0.map->cauchy, st);
        else ls = launch_fused_table(T, r0.query_mode, r0.map->cauchy, r0.map->node_format == LT_NODE_S16, st);
    }
    finish_launch(s, st, ids, bytes, rays, true, ls);
    group.clear();
}

static void launch_one(lt_server* s, Pending& p)
{
    cudaStream_t st = s->streams[s->next_stream++ % s->streams.size()];
    lt_status ls = LT_OK;
    if (injected_failure(s)) ls = fail(LT_ECUDA, "server: injected launch failure");
    else if (p.req.flags & LT_REQ_HOST_BUFFERS) ls = launch_staged(p.req, st);
    else {
        const lt_request& r = p.req;
        RaysInDev in{r.in.x, r.in.y, r.in.dx, r.in.dy, r.in.dz, r.lambda_nm};
        RaysOutDev out{r.out.x, r.out.y, r.out.dx, r.out.dy, r.out.dz, r.out.I, r.out.flags};
        ls = launch_single(r, in, out, st);
    }
    finish_launch(s, st, {p.id}, p.bytes, p.req.n, false, ls);
}

static void worker_main(lt_server* s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    const size_t budget = s->o.mem_budget_bytes;
    while (true) {
        s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
        if (s->stop) break;
        if (s->o.batch_window_us > 0) {
            // hold the oldest request up to the window while more arrive
            const Clock::time_point until =
                s->pending.front().t_submit + std::chrono::microseconds(s->o.batch_window_us);
            while (!s->stop && (int)s->pending.size() < s->o.fuse_max_requests && Clock::now() < until)
                s->cv_work.wait_until(lk, until);
            if (s->stop) break;
        }
        // admit requests in arrival order while the budget allows; expire the
        // ones past their deadline
        std::vector<Pending> take;
        size_t admitted = 0;
        const Clock::time_point now = Clock::now();
        while (!s->pending.empty()) {
            Pending& p = s->pending.front();
            if (p.req.deadline_us &&
                now - p.t_submit > std::chrono::microseconds(p.req.deadline_us)) {
                complete_locked(s, {p.id}, LT_ETIMEOUT, now);
                s->pending.pop_front();
                s->cv_done.notify_all();
                continue;
            }
            const size_t held = s->bytes_in_flight + admitted;
            if (held > 0 && held + p.bytes > budget) break;
            admitted += p.bytes;
            take.push_back(p);
            s->pending.pop_front();
        }
        s->bytes_in_flight += admitted;
        s->stats.peak_bytes_in_flight = std::max(s->stats.peak_bytes_in_flight, s->bytes_in_flight);
        s->stats.bytes_in_flight = s->bytes_in_flight;
        if (take.empty()) {
            // waiting for memory: a completion wakes us; re-check deadlines
            s->cv_work.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        lk.unlock();
        // small requests of one fusion key share a launch (up to
        // fuse_max_requests each); the rest launch on their own
        std::map<int, std::vector<Pending>> groups;
        auto launch_group = [&](int key, std::vector<Pending>& g) {
            if (g.size() == 1) launch_one(s, g[0]);
            else if (key == 0) launch_fused(s, g);
            else launch_fused_queries(s, g);
            g.clear();
        };
        for (Pending& p : take) {
            int key = 0;
            if (fusable(s, p.req, &key)) {
                std::vector<Pending>& g = groups[key];
                g.push_back(p);
                if ((int)g.size() >= s->o.fuse_max_requests) launch_group(key, g);
            } else {
                launch_one(s, p);
            }
        }
        for (auto& kv : groups)
            if (!kv.second.empty()) launch_group(kv.first, kv.second);
        lk.lock();
    }
}

}  // namespace lt

using namespace lt;

extern "C" {

lt_status lt_server_create(const lt_server_opts* opts, lt_server** out)
{
    clear_error();
    if (!out) return fail(LT_EINVAL, "lt_server_create: NULL out");
    *out = nullptr;
    lt_server_opts o{};
    if (opts) o = *opts;
    if (o.mem_budget_bytes == 0) o.mem_budget_bytes = (size_t)1 << 30;
    if (o.n_streams == 0) o.n_streams = 4;
    if (o.fuse_max_requests == 0) o.fuse_max_requests = kMaxFuse;
    if (o.fuse_max_rays == 0) o.fuse_max_rays = 65536;
    if (o.n_streams < 1 || o.n_streams > 64) return fail(LT_EINVAL, "lt_server_create: n_streams in [1, 64]");
    if (o.fuse_max_requests < 1 || o.fuse_max_requests > kMaxFuse)
        return fail(LT_EINVAL, "lt_server_create: fuse_max_requests in [1, %d]", kMaxFuse);
    if (o.fuse_max_rays >= ((size_t)1 << 31)) return fail(LT_EINVAL, "lt_server_create: fuse_max_rays < 2^31");
    if (o.inject_fail_every < 0) return fail(LT_EINVAL, "lt_server_create: inject_fail_every >= 0");
    lt_server* s = new (std::nothrow) lt_server();
    if (!s) return fail(LT_ENOMEM, "lt_server_create: allocation");
    s->o = o;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return cuda_fail(cudaGetLastError(), "lt_server_create: no device");
    }
    for (int k = 0; k < o.n_streams; ++k) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
            delete s;
            return cuda_fail(cudaGetLastError(), "lt_server_create: stream");
        }
        s->streams.push_back(st);
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return LT_OK;
}

void lt_server_destroy(lt_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->worker.join();
    // every launched request (and its completion host function) finishes
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    for (auto& kv : s->lens_cache)
        if (kv.second.dev) cudaFree(kv.second.dev);
    for (LensDev* d : s->retired_lens) cudaFree(d);
    for (auto& kv : s->blob_cache)
        if (kv.second.dev) cudaFree(kv.second.dev);
    for (void* d : s->retired_blobs) cudaFree(d);
    delete s;
}

lt_status lt_submit(lt_server* s, const lt_request* r, uint64_t* ticket)
{
    clear_error();
    if (!s || !r || !ticket) return fail(LT_EINVAL, "lt_submit: NULL argument");
    if (r->n >= ((size_t)1 << 31)) return fail(LT_EINVAL, "lt_submit: n must be < 2^31");
    if (r->kind == LT_REQ_TRACE) {
        int pi, pj;
        if (!r->lens) return fail(LT_EINVAL, "lt_submit: TRACE without a lens");
        if (!path_ij(r->lens->S, r->path_id, &pi, &pj))
            return fail(LT_EINVAL, "lt_submit: bad path id %d", r->path_id);
    } else if (r->kind == LT_REQ_QUERY) {
        if (!r->map) return fail(LT_EINVAL, "lt_submit: QUERY without a map");
        if (r->query_mode != LT_QUERY_TABLE && r->query_mode != LT_QUERY_NO_MASK)
            return fail(LT_EINVAL, "lt_submit: bad query mode %d", r->query_mode);
    } else if (r->kind == LT_REQ_MLP) {
        if (!r->mlp) return fail(LT_EINVAL, "lt_submit: MLP without a learned map");
        if (r->precision < LT_MLP_F32 || r->precision > LT_MLP_F32_NOCLS)
            return fail(LT_EINVAL, "lt_submit: bad precision %d", r->precision);
    } else {
        return fail(LT_EINVAL, "lt_submit: unknown kind %d", r->kind);
    }
    if (r->flags & ~LT_REQ_HOST_BUFFERS) return fail(LT_EINVAL, "lt_submit: unknown flags 0x%x", r->flags);
    if (r->n > 0) {
        const void* ps[] = {r->in.x, r->in.y, r->in.dx, r->in.dy, r->in.dz, r->lambda_nm, r->out.x,
                            r->out.y, r->out.dx, r->out.dy, r->out.dz, r->out.I, r->out.flags};
        const bool host = (r->flags & LT_REQ_HOST_BUFFERS) != 0;
        for (int q = 0; q < 13; ++q) {
            if (!ps[q]) return fail(LT_EINVAL, "lt_submit: NULL ray array");
            if (!host && q < 12 && !aligned16(ps[q]))
                return fail(LT_EINVAL, "lt_submit: device ray arrays must be 16-byte aligned");
        }
    }
    const size_t bytes = request_bytes(*r, s->o.fuse_max_rays);
    if (bytes > s->o.mem_budget_bytes)
        return fail(LT_ENOMEM, "lt_submit: request needs %zu bytes, budget %zu", bytes, s->o.mem_budget_bytes);
    const Clock::time_point now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const uint64_t id = s->next_id++;
        Ticket& t = s->tickets[id];
        t.t_submit = now;
        s->stats.submitted++;
        if (r->n == 0) {
            t.t_launch = now;
            complete_locked(s, {id}, LT_OK, now);
        } else {
            s->pending.push_back(Pending{id, *r, bytes, now});
        }
        *ticket = id;
    }
    s->cv_work.notify_one();
    return LT_OK;
}

lt_status lt_poll_info(lt_server* s, uint64_t ticket, uint32_t timeout_us, lt_ticket_info* info)
{
    clear_error();
    if (!s) return fail(LT_EINVAL, "lt_poll: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(LT_EINVAL, "lt_poll: unknown ticket %llu", (unsigned long long)ticket);
    if (!it->second.done) {
        if (timeout_us == 0) return LT_ENOTREADY;
        const bool ok = s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] {
            auto t = s->tickets.find(ticket);
            return t == s->tickets.end() || t->second.done;
        });
        it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return fail(LT_EINVAL, "lt_poll: ticket released by another poll");
        if (!ok) return LT_ENOTREADY;
    }
    const Ticket t = it->second;
    s->tickets.erase(it);
    if (info) {
        const Clock::time_point launch = t.t_launch.time_since_epoch().count() ? t.t_launch : t.t_done;
        info->queue_us = std::chrono::duration<double, std::micro>(launch - t.t_submit).count();
        info->latency_us = std::chrono::duration<double, std::micro>(t.t_done - t.t_submit).count();
        info->fused = t.fused;
    }
    if (t.status != LT_OK) return fail(t.status, "lt_poll: request failed with status %d", t.status);
    return LT_OK;
}

lt_status lt_poll(lt_server* s, uint64_t ticket, uint32_t timeout_us)
{
    return lt_poll_info(s, ticket, timeout_us, nullptr);
}

lt_status lt_server_stats_get(lt_server* s, lt_server_stats* out)
{
    clear_error();
    if (!s || !out) return fail(LT_EINVAL, "lt_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->bytes_in_flight = s->bytes_in_flight;
    return LT_OK;
}

}  // extern "C"
