// Internal declarations of the tabulated map (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "lt_internal.h"
#include "rays.cuh"

enum { LT_CELL_INVALID = 0, LT_CELL_VALID = 1, LT_CELL_BOUNDARY = 2 };

namespace lt {

// The map as the kernels see it (a __grid_constant__ parameter, ~3 KB):
// the lens for the fallback tracer, the path, the FP32 lattice constants and
// the device tables.  Node strides: (x, y, s_x, s_y, lambda) row-major,
// lambda fastest; cell strides likewise over res - 1.
struct MapDev {
    LensDev L;
    int pi, pj;
    int res[5];
    float lo[5], step[5], inv[5], umax[5];
    uint32_t stride[5], cstride[5];
    const float* node;      // n_nodes x 8 floats (LT_NODE_F32)
    const uint32_t* cls;    // 2 bits per cell
    const uint4* node16;    // n_nodes x 16-byte records of 6 int16 (LT_NODE_S16)
    float qstep[6];         // LT_NODE_S16: the value of one integer step per output
};

// The map query's trace queue: per queued ray its entrance ray (structure of
// arrays) and its index (bit 31 set: outside the lattice box).  The queue is
// split into kQSegs segments of segcap entries, block b of the query kernel
// appending to segment b % kQSegs, so that the appends' atomics spread over
// kQSegs counters in separate 128-byte lines instead of one hot address:
// count[s * kQCountStride] counts segment s, count[kQSegs * kQCountStride]
// the chunks the tracer has taken.
constexpr int kQSegs = 64;
constexpr int kQCountStride = 32;
constexpr size_t kQHeaderBytes = (kQSegs + 1) * kQCountStride * 4 + 128;   // 8,448 bytes
struct TraceQueue {
    float *x, *y, *dx, *dy, *dz, *lam;
    uint32_t* tag;
    uint32_t* count;
    uint32_t segcap;
};
constexpr int kQTile = 256;   // rays per block of the query kernel
// entries per segment for n rays
constexpr size_t query_segcap(size_t n) { return ((n + kQTile - 1) / kQTile + kQSegs - 1) / kQSegs * kQTile; }
// scratch bytes of the queue for n rays: the counters, then 7 arrays of
// kQSegs * segcap words
constexpr size_t query_scratch_bytes(size_t n) { return kQHeaderBytes + 7 * 4 * kQSegs * query_segcap(n); }

// The polynomial-patch map's large-batch query also keeps, per tile of
// kSortTileRays rays, a record of each ray the polynomial answers (its
// patch-local coordinates, rotation, mirror, patch and index in the tile:
// 32 bytes) in the tile's region, sorted by patch with every patch's run
// padded to an even length (so that record pairs share a patch), and the
// tile's padded count.  A tile's region holds kSortTileRays + P records for
// a map of P patches.  Per tile, a bit per ray marks the rays handed to the
// trace queue (their rows are written by the tracer, not the evaluation).
constexpr size_t kSortTileRays = 1024;
constexpr size_t query_tiles(size_t n) { return (n + kSortTileRays - 1) / kSortTileRays; }
constexpr size_t poly_scratch_bytes(size_t n, size_t patches)
{
    return query_scratch_bytes(n) + query_tiles(n) * ((kSortTileRays + patches) * 32 + 4 + kSortTileRays / 8) + 256;
}
struct PolyScratch {
    float4* rec;          // query_tiles(n) x (kSortTileRays + patches) x 2 float4
    uint32_t* tile_nv;    // query_tiles(n)
    uint32_t* traced;     // query_tiles(n) x kSortTileRays / 32 words: the rays queued for the tracer
    uint32_t stride;      // records per tile region
};
// the records and counts after the queue of n rays in `scratch` (poly_scratch_bytes(n, patches))
PolyScratch poly_scratch_at(void* scratch, size_t n, size_t patches);

// the queue laid out in `scratch` (256-byte aligned, query_scratch_bytes(n))
TraceQueue trace_queue_at(void* scratch, size_t n);

// The map query of n < 2^31 rays on `st`: the classify-and-gather kernel,
// then the tracer over the rays it queued.  launch_query takes the queue from
// the library's stream-ordered pool (small batches run as one fused kernel
// that needs no queue); launch_query_with always runs the two kernels, on the
// caller's queue (its counters are cleared on `st`).
lt_status launch_query(const lt_map* map, const RaysInDev& in, const RaysOutDev& out, uint32_t n,
                       int mode, cudaStream_t st);
lt_status launch_query_with(const lt_map* map, const RaysInDev& in, const RaysOutDev& out, uint32_t n,
                            int mode, const TraceQueue& Q, cudaStream_t st);

// LT_EINVAL unless the current device is the one the map lives on.
lt_status check_map_device(const lt_map* m, const char* who);

// Pieces of the table map that the polynomial-patch map shares (map.cu).
constexpr uint32_t kOutsideBit = 0x80000000u;   // queue tag bit: ray outside the box
constexpr uint32_t kFusedMaxRays = 1u << 18;    // batches up to this size run as one fused kernel
// the exact tracer over a query's queue (map_trace_kernel), on `st`
lt_status launch_queue_trace(const lt_map* map, const RaysOutDev& out, uint32_t n, const TraceQueue& Q,
                             cudaStream_t st);
// the 2-bit classes from per-cell corner bits (bit0: class may be VALID, bit1:
// every corner invalid), fit-ray sightings (2 bits per cell: valid / invalid
// seen) and fit-ray residual maxima (FP32 bits; NULL: none); counts[0..2] +=
// INVALID, VALID, BOUNDARY cells
lt_status launch_map_classify(const uint8_t* corner_bits, const uint32_t* seen, const uint32_t* resmax,
                              float tol, uint32_t* cls, uint32_t NC, unsigned long long* counts,
                              cudaStream_t st);

// A fused serving launch: several small requests of one kind in one grid,
// each block serving one request.  The table is the kernel parameter (about
// 16 KB); `dev` points to a device copy of the request's constants (a
// MapDev, a map's MapDev + PolyDev, or a learned map's constants).
constexpr int kMaxFuse = 128;
struct ReqItem {
    const void* dev;
    RaysInDev in;
    RaysOutDev out;
    uint32_t n;
};
struct ReqTable {
    int n_items;
    uint32_t block0[kMaxFuse + 1];   // first block of each request; block0[n_items] = the grid
    ReqItem item[kMaxFuse];
};

// the request of block b: the last whose first block is <= b
__device__ __forceinline__ int req_of_block(const ReqTable& T, uint32_t b)
{
    int lo = 0, hi = T.n_items - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.block0[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// copy `bytes` (a multiple of 16) from global to shared memory with the
// whole block (the caller synchronises before use)
__device__ __forceinline__ void stage_words(void* dst, const void* src, size_t bytes)
{
    const int4* s = static_cast<const int4*>(src);
    int4* d = static_cast<int4*>(dst);
    for (int k = threadIdx.x; k < (int)(bytes / 16); k += blockDim.x) d[k] = __ldg(s + k);
}

// Fused launches of the server on `st` over the requests of T, whose block0
// counts blocks of the kind's rays per block (kFusedQueryRays for both map
// kinds, fused_mlp_rays(precision) for learned maps): table maps
// (launch_fused_table: every map of the same dispersion form, `cauchy`, and
// node format, `s16`),
// polynomial-patch maps (launch_fused_poly: the same degree and dispersion
// form) and learned maps (launch_fused_mlp: one precision).  Per-ray results
// equal those of the same request made alone.  LT_EINVAL for an empty or
// oversized table.
constexpr uint32_t kFusedQueryRays = kQTile;
uint32_t fused_mlp_rays(int precision);
// the device-copy bytes of a request's constants: a map (serve_blob) or a
// learned map at one precision (mlp_serve_blob; builds its tensor-core
// weight images first if they are out of date)
lt_status serve_blob(const lt_map* m, std::vector<unsigned char>& bytes);
lt_status mlp_serve_blob(const lt_mlp* m, int precision, std::vector<unsigned char>& bytes);
lt_status launch_fused_table(const ReqTable& T, int mode, bool cauchy, bool s16, cudaStream_t st);
lt_status launch_fused_poly(const ReqTable& T, int degree, int mode, bool cauchy, cudaStream_t st);
lt_status launch_fused_mlp(const ReqTable& T, int precision, cudaStream_t st);

// The polynomial-patch map as its query kernels see it (a __grid_constant__
// parameter): FP32 constants of the class grid over (r, p, q, w), the patch
// structure and the device tables.
struct PolyDev {
    float lo[4], inv[4], cmax[4], two_over_m[4];
    int C[4], m[4], P[4];
    uint32_t mdiv[4];                   // ceil(2^32 / m): cell / m = umulhi(cell, mdiv) for cell < 2^16
    uint32_t cstride[4], pstride[4];    // class-grid cell and patch strides (w fastest)
    int T, degree, n_patches;
    const float4* cg;                   // [patch][group of 4 terms][output]: coefficient groups
    const uint8_t* patch_ok;            // [patch]: 1 if the patch has a fit
    const uint32_t* cls;                // 2 bits per class-grid cell
};

// The polynomial-patch map's query on `st` (launch_query dispatches here for
// such maps): batches of at most kFusedMaxRays run as one kernel, larger
// ones take their queue and records from the pool.  launch_query_with, whose
// caller supplies only a queue, runs the one-kernel form in chunks.
lt_status launch_poly_query(const lt_map* map, const RaysInDev& in, const RaysOutDev& out, uint32_t n,
                            int mode, cudaStream_t st);
// the one-kernel form over n rays in chunks of at most kFusedMaxRays (no scratch)
lt_status launch_poly_fused(const lt_map* map, const RaysInDev& in, const RaysOutDev& out, uint32_t n, int mode,
                            cudaStream_t st);

}  // namespace lt

enum { LT_MAP_KIND_TABLE = 0, LT_MAP_KIND_POLY = 1 };

struct lt_map {
    lt_lens lens;             // copy of the lens the map was built on
    int kind = LT_MAP_KIND_TABLE;
    int path_id = 0;
    int res[5] = {};
    double lo[5] = {}, hi[5] = {};
    double tol = 0.0;
    uint64_t n_nodes = 0, n_cells = 0;
    float* node = nullptr;
    uint4* node16 = nullptr;  // LT_NODE_S16 table (node is then released after the build)
    int node_format = LT_NODE_F32;
    uint8_t* node_valid = nullptr;
    uint32_t* cls = nullptr;
    int device = 0;
    bool cauchy = true;       // every glass of the lens is Cauchy (single-FMA dispersion)
    lt_map_stats stats = {};
    lt::MapDev dev;           // the lens and path (for the fallback tracer); table constants
    // polynomial-patch maps
    lt_poly_opts popts = {};  // the build options (fit arrays cleared)
    lt_poly_stats pstats = {};
    lt::PolyDev pdev = {};
    float4* coefg = nullptr;  // the FP32 query table (coefficient groups)
    double* coef64 = nullptr; // patches x terms x 5, the FP64 fit
    uint8_t* patch_ok = nullptr;
    ~lt_map();
};
