// Tabulated lens transport map: build (node tracing, fit-ray reduction, cell
// classification) and query (mask lookup, 32-corner multilinear
// interpolation, exact-tracer fallback for BOUNDARY cells).
//
// The paper's factorisation (Sec. 4.2, Eq. 11): a valid/occluded mask g and a
// regressor f used only where g = 1.  Here the mask is 2 bits per lattice
// cell and the regressor a table of traced nodes; cells the mask cannot decide
// (BOUNDARY) are answered by the tracer itself.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <mutex>
#include <new>
#include <vector>

#include "map_internal.h"
#include "profile.h"
#include "tracer.cuh"

namespace lt {

constexpr int kQBlock = 128;   // rays per chunk (and threads per block) of the trace kernel

// ------------------------------------------------------------------ lattice (FP32 rule)

__device__ __forceinline__ float node_coord(const MapDev& M, int d, int i)
{
    return __fadd_rn(M.lo[d], __fmul_rn((float)i, M.step[d]));
}

// entrance ray of lattice node `idx`: direction normalize(s_x, s_y, 1), all
// operations correctly rounded (never contracted) so the oracle can rebuild it
__device__ __forceinline__ void node_ray(const MapDev& M, const int idx[5], float ray[6])
{
    float q[5];
#pragma unroll
    for (int d = 0; d < 5; ++d) q[d] = node_coord(M, d, idx[d]);
    const float a = __fmul_rn(q[2], q[2]);
    const float b = __fmul_rn(q[3], q[3]);
    const float s = __fadd_rn(a, b);
    const float n2 = __fadd_rn(s, 1.0f);
    const float len = __fsqrt_rn(n2);
    ray[0] = q[0];
    ray[1] = q[1];
    ray[2] = __fdiv_rn(q[2], len);
    ray[3] = __fdiv_rn(q[3], len);
    ray[4] = __fdiv_rn(1.0f, len);
    ray[5] = q[4];
}

// cell of a ray: returns false outside the box (or for dz <= 0 / NaN);
// f[d] = u - cell is the FP32 position inside the cell
__device__ __forceinline__ bool cell_of(const MapDev& M, float x, float y, float dx, float dy,
                                        float dz, float lam, uint32_t& cid, float f[5])
{
    if (!(dz > 0.0f)) return false;
    const float v[5] = {x, y, __fdiv_rn(dx, dz), __fdiv_rn(dy, dz), lam};
    bool inside = true;
    cid = 0;
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        const float u = __fmul_rn(__fsub_rn(v[d], M.lo[d]), M.inv[d]);
        inside &= (u >= 0.0f) & (u <= M.umax[d]);
        int c = (int)floorf(u);
        c = min(max(c, 0), M.res[d] - 2);
        f[d] = u - (float)c;
        cid += (uint32_t)c * M.cstride[d];
    }
    return inside;
}

__device__ __forceinline__ uint32_t cell_class(const MapDev& M, uint32_t cid)
{
    return (__ldg(M.cls + (cid >> 4)) >> ((cid & 15u) * 2u)) & 3u;
}

// node-table base index of the cell's (0,0,0,0,0) corner
__device__ __forceinline__ uint32_t cell_base(const MapDev& M, uint32_t cid)
{
    uint32_t base = 0;
#pragma unroll
    for (int d = 4; d >= 0; --d) {
        const uint32_t rd = (uint32_t)(M.res[d] - 1);
        const uint32_t c = cid % rd;
        cid /= rd;
        base += c * M.stride[d];
    }
    return base;
}

// Node records are 8 floats (32 bytes): x, y, dx, dy, dz, I, 0, 0.  The two
// lambda-adjacent nodes of a cell corner are then 64 contiguous, 64-byte
// aligned bytes: one sector pair, fetched by four 16-byte loads.
constexpr int kNodeFloats = 8;

// Scalar multilinear interpolation (one thread, 16 corner pairs) -- used by the
// map build; the query kernel uses the warp-cooperative form below.
__device__ __forceinline__ void interpolate(const MapDev& M, const float* __restrict__ node,
                                            uint32_t base, const float f[5], float o[6])
{
    const float w0[2] = {1.0f - f[0], f[0]}, w1[2] = {1.0f - f[1], f[1]};
    const float w2[2] = {1.0f - f[2], f[2]}, w3[2] = {1.0f - f[3], f[3]};
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float fl = f[4];
#pragma unroll 4
    for (int c = 0; c < 16; ++c) {
        const int b0 = (c >> 3) & 1, b1 = (c >> 2) & 1, b2 = (c >> 1) & 1, b3 = c & 1;
        const uint32_t off = base + b0 * M.stride[0] + b1 * M.stride[1] + b2 * M.stride[2] +
                             b3 * M.stride[3];
        const float4* p = reinterpret_cast<const float4*>(node + (size_t)off * kNodeFloats);
        const float4 a0 = __ldg(p + 0), a1 = __ldg(p + 1), c0 = __ldg(p + 2), c1 = __ldg(p + 3);
        const float w = (w0[b0] * w1[b1]) * (w2[b2] * w3[b3]);
        acc[0] = fmaf(w, fmaf(fl, c0.x - a0.x, a0.x), acc[0]);
        acc[1] = fmaf(w, fmaf(fl, c0.y - a0.y, a0.y), acc[1]);
        acc[2] = fmaf(w, fmaf(fl, c0.z - a0.z, a0.z), acc[2]);
        acc[3] = fmaf(w, fmaf(fl, c0.w - a0.w, a0.w), acc[3]);
        acc[4] = fmaf(w, fmaf(fl, c1.x - a1.x, a1.x), acc[4]);
        acc[5] = fmaf(w, fmaf(fl, c1.y - a1.y, a1.y), acc[5]);
    }
    const float n2 = fmaf(acc[2], acc[2], fmaf(acc[3], acc[3], acc[4] * acc[4]));
    float inv = n2 > 0.0f ? rsqrtf(n2) : 0.0f;
    inv = inv * fmaf(-0.5f * n2, inv * inv, 1.5f);
    o[0] = acc[0];
    o[1] = acc[1];
    o[2] = acc[2] * inv;
    o[3] = acc[3] * inv;
    o[4] = acc[4] * inv;
    o[5] = acc[5];
}

__device__ __forceinline__ void store_out(const RaysOutDev& out, uint32_t r, const float o[6],
                                          uint32_t flags)
{
    __stcs(out.x + r, o[0]);
    __stcs(out.y + r, o[1]);
    __stcs(out.dx + r, o[2]);
    __stcs(out.dy + r, o[3]);
    __stcs(out.dz + r, o[4]);
    __stcs(out.I + r, o[5]);
    out.flags[r] = (uint8_t)flags;
}

// ------------------------------------------------------------------ build kernels

// every lattice node traced exactly (one thread per node)
template <bool CAUCHY>
__global__ void __launch_bounds__(256)
map_node_kernel(const __grid_constant__ MapDev M, float* __restrict__ node,
                uint8_t* __restrict__ node_valid, uint32_t N)
{
    const uint32_t l = blockIdx.x * 256u + threadIdx.x;
    if (l >= N) return;
    int idx[5];
    uint32_t t = l;
#pragma unroll
    for (int d = 4; d >= 0; --d) {
        idx[d] = (int)(t % (uint32_t)M.res[d]);
        t /= (uint32_t)M.res[d];
    }
    float ray[6];
    node_ray(M, idx, ray);
    TraceOut o;
    int nint;
    const uint32_t f = trace_ray<CAUCHY>(M.L, M.pi, M.pj, ray[0], ray[1], ray[2], ray[3], ray[4],
                                         ray[5], o, nint);
    float4* p = reinterpret_cast<float4*>(node + (size_t)l * kNodeFloats);
    p[0] = make_float4(o.x, o.y, o.dx, o.dy);
    p[1] = make_float4(o.dz, o.I, 0.0f, 0.0f);
    node_valid[l] = (uint8_t)(f & LT_FLAG_VALID);
}

// per cell: bit0 = all 32 corners valid, bit1 = all invalid
__global__ void __launch_bounds__(256)
map_corner_kernel(const __grid_constant__ MapDev M, const uint8_t* __restrict__ node_valid,
                  uint8_t* __restrict__ corner_bits, uint32_t NC)
{
    const uint32_t cid = blockIdx.x * 256u + threadIdx.x;
    if (cid >= NC) return;
    const uint32_t base = cell_base(M, cid);
    int nv = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const uint32_t off = base + ((k >> 4) & 1) * M.stride[0] + ((k >> 3) & 1) * M.stride[1] +
                             ((k >> 2) & 1) * M.stride[2] + ((k >> 1) & 1) * M.stride[3] +
                             (k & 1) * M.stride[4];
        nv += __ldg(node_valid + off);
    }
    corner_bits[cid] = (uint8_t)((nv == 32 ? 1 : 0) | (nv == 0 ? 2 : 0));
}

struct FitAccum {
    unsigned long long inside, valid, n_res;
    double sumsq;
    unsigned int max_res_bits;
};

// one thread per fit ray: mark the cell as having seen a valid / invalid ray,
// and for valid rays in all-valid-corner cells reduce the interpolation residual
template <bool CAUCHY>
__global__ void __launch_bounds__(256)
map_fit_kernel(const __grid_constant__ MapDev M, RaysInDev fit, uint32_t nfit,
               const float* __restrict__ node, const uint8_t* __restrict__ corner_bits,
               uint32_t* __restrict__ seen, uint32_t* __restrict__ resmax, FitAccum* acc)
{
    const uint32_t r = blockIdx.x * 256u + threadIdx.x;
    bool inside = false, valid = false, has_res = false;
    float res = 0.0f;
    if (r < nfit) {
        const float x = __ldg(fit.x + r), y = __ldg(fit.y + r), dx = __ldg(fit.dx + r),
                    dy = __ldg(fit.dy + r), dz = __ldg(fit.dz + r), lam = __ldg(fit.lam + r);
        uint32_t cid;
        float f[5];
        inside = cell_of(M, x, y, dx, dy, dz, lam, cid, f);
        if (inside) {
            TraceOut o;
            int nint;
            valid = (trace_ray<CAUCHY>(M.L, M.pi, M.pj, x, y, dx, dy, dz, lam, o, nint) &
                     LT_FLAG_VALID) != 0;
            atomicOr(seen + (cid >> 4), (valid ? 1u : 2u) << ((cid & 15u) * 2u));
            if (valid && (__ldg(corner_bits + cid) & 1)) {
                float ip[6];
                interpolate(M, node, cell_base(M, cid), f, ip);
                res = hypotf(ip[0] - o.x, ip[1] - o.y);
                has_res = true;
                if (resmax) atomicMax(resmax + cid, __float_as_uint(res));
            }
        }
    }
    // warp reductions of the global statistics (FP64 sum of squares)
    const unsigned full = 0xffffffffu;
    unsigned long long cin = __popc(__ballot_sync(full, inside));
    unsigned long long cva = __popc(__ballot_sync(full, valid));
    unsigned long long cre = __popc(__ballot_sync(full, has_res));
    double sq = has_res ? (double)res * (double)res : 0.0;
    unsigned int mx = has_res ? __float_as_uint(res) : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sq += __shfl_xor_sync(full, sq, o);
        mx = max(mx, __shfl_xor_sync(full, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (cin) atomicAdd(&acc->inside, cin);
        if (cva) atomicAdd(&acc->valid, cva);
        if (cre) {
            atomicAdd(&acc->n_res, cre);
            atomicAdd(&acc->sumsq, sq);
            atomicMax(&acc->max_res_bits, mx);
        }
    }
}

// one thread per 16 cells (one word of 2-bit classes)
__global__ void __launch_bounds__(256)
map_classify_kernel(const uint8_t* __restrict__ corner_bits, const uint32_t* __restrict__ seen,
                    const uint32_t* __restrict__ resmax, uint32_t tol_bits, uint32_t* __restrict__ cls,
                    uint32_t NC, unsigned long long* counts)
{
    const uint32_t w = blockIdx.x * 256u + threadIdx.x;
    const uint32_t nw = (NC + 15) / 16;
    uint32_t word = 0, ninv = 0, nval = 0, nbnd = 0;
    if (w < nw) {
        const uint32_t sw = seen[w];
        for (int q = 0; q < 16; ++q) {
            const uint32_t cid = w * 16 + q;
            if (cid >= NC) break;
            const uint32_t cb = corner_bits[cid];
            const uint32_t s = (sw >> (2 * q)) & 3u;
            uint32_t c;
            if ((cb & 2u) && !(s & 1u)) c = LT_CELL_INVALID;
            else if ((cb & 1u) && !(s & 2u) && (!resmax || resmax[cid] <= tol_bits)) c = LT_CELL_VALID;
            else c = LT_CELL_BOUNDARY;
            word |= c << (2 * q);
            ninv += c == LT_CELL_INVALID;
            nval += c == LT_CELL_VALID;
            nbnd += c == LT_CELL_BOUNDARY;
        }
        cls[w] = word;
    }
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ninv += __shfl_xor_sync(full, ninv, o);
        nval += __shfl_xor_sync(full, nval, o);
        nbnd += __shfl_xor_sync(full, nbnd, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(counts + 0, (unsigned long long)ninv);
        atomicAdd(counts + 1, (unsigned long long)nval);
        atomicAdd(counts + 2, (unsigned long long)nbnd);
    }
}

// LT_NODE_S16 build: per output, the largest |value| over the valid nodes
// (as FP32 bits: non-negative floats order like their bit patterns)
__global__ void __launch_bounds__(256)
map_absmax_kernel(const float* __restrict__ node, const uint8_t* __restrict__ node_valid, uint32_t N,
                  unsigned* __restrict__ mx)
{
    float m[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (uint32_t l = blockIdx.x * 256u + threadIdx.x; l < N; l += gridDim.x * 256u) {
        if (!node_valid[l]) continue;
        const float4* p = reinterpret_cast<const float4*>(node + (size_t)l * kNodeFloats);
        const float4 a = __ldg(p), b = __ldg(p + 1);
        m[0] = fmaxf(m[0], fabsf(a.x));
        m[1] = fmaxf(m[1], fabsf(a.y));
        m[2] = fmaxf(m[2], fabsf(a.z));
        m[3] = fmaxf(m[3], fabsf(a.w));
        m[4] = fmaxf(m[4], fabsf(b.x));
        m[5] = fmaxf(m[5], fabsf(b.y));
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m[k] = fmaxf(m[k], __shfl_xor_sync(0xffffffffu, m[k], o));
        if ((threadIdx.x & 31) == 0) atomicMax(mx + k, __float_as_uint(m[k]));
    }
}

struct QuantInv {
    float inv[6];   // 2^(15 - e_k): exact powers of two
};

// LT_NODE_S16 build: each node's six outputs as int16 q = rint(v * inv_k)
// (ties to even), clamped to the int16 range; invalid nodes all zero.
__global__ void __launch_bounds__(256)
map_quantize_kernel(const float* __restrict__ node, const uint8_t* __restrict__ node_valid, uint32_t N,
                    QuantInv Q, uint4* __restrict__ node16)
{
    const uint32_t l = blockIdx.x * 256u + threadIdx.x;
    if (l >= N) return;
    const float4* p = reinterpret_cast<const float4*>(node + (size_t)l * kNodeFloats);
    const float4 a = __ldg(p), b = __ldg(p + 1);
    const float v[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
    uint32_t h[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int q = node_valid[l] ? max(-32768, min(32767, __float2int_rn(v[k] * Q.inv[k]))) : 0;
        h[k] = (uint32_t)q & 0xffffu;
    }
    node16[l] = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), 0u);
}

// ------------------------------------------------------------------ query kernels

// Cell of a ray for the query: as cell_of, plus the node index of the cell's
// (0,0,0,0,0) corner, taken from the per-dimension cell indices.
__device__ __forceinline__ bool cell_and_base(const MapDev& M, float x, float y, float dx, float dy,
                                              float dz, float lam, uint32_t& cid, uint32_t& base,
                                              float f[5])
{
    if (!(dz > 0.0f)) return false;
    const float v[5] = {x, y, __fdiv_rn(dx, dz), __fdiv_rn(dy, dz), lam};
    bool inside = true;
    cid = 0;
    base = 0;
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        const float u = __fmul_rn(__fsub_rn(v[d], M.lo[d]), M.inv[d]);
        inside &= (u >= 0.0f) & (u <= M.umax[d]);
        int c = (int)floorf(u);
        c = min(max(c, 0), M.res[d] - 2);
        f[d] = u - (float)c;
        cid += (uint32_t)c * M.cstride[d];
        base += (uint32_t)c * M.stride[d];
    }
    return inside;
}

// A VALID-cell ray of a warp waiting for its gather: its lane, the node
// index of its cell's first corner, its position in the cell.
struct __align__(16) GatherItem {
    uint32_t slot, base;
    float f[5];
    float pad;
};

// Row stride (words) of a warp's result rows in shared memory: 7 puts a
// ray's six outputs, and the rows of eight rays, in distinct banks.
constexpr int kObStride = 7;

// The map query runs as two kernels.
// map_query_kernel: each warp answers 32 consecutive rays on its own (no
// block-wide barrier, so warps of a block never wait for one another).
//  1. Each lane classifies its ray.  INVALID cells are answered at once;
//     VALID cells are queued in the warp's shared-memory list for a gather;
//     BOUNDARY cells and rays outside the lattice box go to the launch's
//     trace queue (entrance ray and index, bit 31 set for an outside ray;
//     one atomic per warp on its block's segment counter).
//  2. The warp gathers its queued rays eight at a time, a quad of lanes per
//     ray: each lane loads its 16-byte piece of the cell's 16 lambda pairs
//     (one 64-byte pair per quad and warp load, so each load instruction
//     reads eight whole pairs), weights it by the corner's multilinear
//     factor (the lambda factor included) and sums in registers; one
//     shuffle stage adds the quad's lower- and upper-lambda halves.
//  3. Each lane writes its own ray (coalesced; a queued ray's row gets a
//     placeholder the tracer overwrites); interpolated directions are
//     renormalised there.
// map_trace_kernel, a persistent grid, then traces the queue with the exact
// tracer, 128 rays per block at a time with survivors compacted (the rays
// of BOUNDARY cells die at every depth of the lens), and writes each result
// at its ray's index.
constexpr int kQWarps = kQTile / 32;

// A lane's ray after classification (step 1 of map_query_kernel).
struct Classified {
    bool ip, tr;                // VALID cell (to interpolate); BOUNDARY or outside (to trace)
    uint32_t tag, base;         // ray index (| kOutsideBit); node index of the cell's first corner
    float f[5];                 // position in the cell
    float x, y, dx, dy, dz, lam;
};

// Step 1: load ray r (if r < n) and classify it.
template <int MODE>
__device__ __forceinline__ Classified classify_ray(const MapDev& M, const RaysInDev& in, uint32_t n, uint32_t r)
{
    Classified c;
    c.ip = false;
    c.tr = false;
    c.tag = r;
    c.base = 0;
#pragma unroll
    for (int d = 0; d < 5; ++d) c.f[d] = 0.0f;
    c.x = c.y = c.dx = c.dy = c.dz = c.lam = 0.0f;
    if (r < n) {
        c.x = __ldg(in.x + r);
        c.y = __ldg(in.y + r);
        c.dx = __ldg(in.dx + r);
        c.dy = __ldg(in.dy + r);
        c.dz = __ldg(in.dz + r);
        c.lam = __ldg(in.lam + r);
        uint32_t cid = 0;
        if (!cell_and_base(M, c.x, c.y, c.dx, c.dy, c.dz, c.lam, cid, c.base, c.f)) {
            c.tr = true;
            c.tag |= kOutsideBit;
        } else {
            const uint32_t k = MODE == LT_QUERY_TABLE ? cell_class(M, cid) : (uint32_t)LT_CELL_VALID;
            c.ip = k == LT_CELL_VALID;
            c.tr = k != LT_CELL_VALID && k != LT_CELL_INVALID;
        }
    }
    return c;
}

// Steps 2 and 3 for a warp (all 32 lanes call it; gq and ob are the warp's
// shared-memory list and result rows): gather the warp's VALID rays eight at
// a time -- quad g of lanes (lane >> 2) interpolates listed ray g0 + g, lane
// part (lane & 3) its 16-byte piece of every lambda pair (0/1: the halves of
// the lower-lambda record, 2/3: of the upper one), summing the 16 pairs of
// (x, y, s_x, s_y) corners in registers; a shuffle adds the lower and upper
// halves -- then write every ray of the warp (a placeholder row for a ray to be
// traced).
__device__ __forceinline__ void gather_and_write(const MapDev& M, const RaysOutDev& out, uint32_t n, uint32_t r,
                                                 const Classified& c, GatherItem* gq, float* ob)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned mv = __ballot_sync(full, c.ip);
    const int nv = __popc(mv);
    if (c.ip) {
        GatherItem e;
        e.slot = (uint32_t)lane;
        e.base = c.base;
#pragma unroll
        for (int d = 0; d < 5; ++d) e.f[d] = c.f[d];
        e.pad = 0.0f;
        gq[__popc(mv & ((1u << lane) - 1u))] = e;
    }
    __syncwarp();
    const int part = lane & 3;
    const bool upper = (part & 2) != 0;
    const uint32_t s0 = M.stride[0], s1 = M.stride[1], s2 = M.stride[2], s3 = M.stride[3];
    const float4* __restrict__ node4 = reinterpret_cast<const float4*>(M.node);
#pragma unroll 1
    for (int g0 = 0; g0 < nv; g0 += 8) {
        const int gi = g0 + (lane >> 2);
        const bool act = gi < nv;
        const GatherItem e = gq[min(gi, nv - 1)];
        const float fl = upper ? e.f[4] : 1.0f - e.f[4];
        const float w1a = e.f[0], w0a = 1.0f - e.f[0];
        const float4* __restrict__ p = node4 + (size_t)e.base * 2 + part;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
#pragma unroll
            for (int qq = 0; qq < 8; ++qq) {
                const uint32_t off = ((qq & 4) ? s1 : 0u) + ((qq & 2) ? s2 : 0u) + ((qq & 1) ? s3 : 0u);
                const float4 a = __ldg(p + (size_t)off * 2);
                const float4 b = __ldg(p + (size_t)(off + s0) * 2);
                const float wq = (((qq & 4) ? e.f[1] : 1.0f - e.f[1]) * ((qq & 2) ? e.f[2] : 1.0f - e.f[2])) *
                                 (((qq & 1) ? e.f[3] : 1.0f - e.f[3]) * fl);
                const float w1 = wq * w1a, w0 = wq * w0a;
                acc.x = fmaf(w1, b.x, fmaf(w0, a.x, acc.x));
                acc.y = fmaf(w1, b.y, fmaf(w0, a.y, acc.y));
                acc.z = fmaf(w1, b.z, fmaf(w0, a.z, acc.z));
                acc.w = fmaf(w1, b.w, fmaf(w0, a.w, acc.w));
            }
        }
        acc.x += __shfl_xor_sync(full, acc.x, 2);
        acc.y += __shfl_xor_sync(full, acc.y, 2);
        acc.z += __shfl_xor_sync(full, acc.z, 2);
        acc.w += __shfl_xor_sync(full, acc.w, 2);
        if (act && part == 0) {
            float* o = ob + e.slot * kObStride;
            o[0] = acc.x;
            o[1] = acc.y;
            o[2] = acc.z;
            o[3] = acc.w;
        } else if (act && part == 1) {
            float* o = ob + e.slot * kObStride;
            o[4] = acc.x;
            o[5] = acc.y;
        }
    }
    __syncwarp();
    // Every row is written, a queued ray's as a placeholder that the tracer
    // overwrites later: the warp's stores then cover whole sectors, which L2
    // takes without merging partial lines.
    if (r < n) {
        float o[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (c.ip) {
#pragma unroll
            for (int k = 0; k < 6; ++k) o[k] = ob[lane * kObStride + k];
            const float n2 = fmaf(o[2], o[2], fmaf(o[3], o[3], o[4] * o[4]));
            float inv = n2 > 0.0f ? rsqrtf(n2) : 0.0f;
            inv = inv * fmaf(-0.5f * n2, inv * inv, 1.5f);
            o[2] *= inv;
            o[3] *= inv;
            o[4] *= inv;
        }
        store_out(out, r, o, c.ip ? LT_FLAG_VALID : 0u);
    }
}

// A 16-bit table entry as FP32: the sign-extended integer added to the bits
// of 1.5 * 2^23 gives the float 1.5 * 2^23 + q exactly (|q| < 2^22), from
// which subtracting 1.5 * 2^23 leaves q.
__device__ __forceinline__ float s16_lo(uint32_t w)
{
    return __int_as_float(0x4B400000 + (((int)(w << 16)) >> 16)) - 12582912.0f;
}
__device__ __forceinline__ float s16_hi(uint32_t w)
{
    return __int_as_float(0x4B400000 + (((int)w) >> 16)) - 12582912.0f;
}

// gather_and_write for an LT_NODE_S16 table: a pair of lanes per ray (part
// 0: the lower-lambda node of each of the 16 (x, y, s_x, s_y) corners, part
// 1: the upper), sixteen rays per round; each lane loads one 16-byte record
// per corner, weights its six integers by the corner's multilinear factor
// and sums in FP32; one shuffle adds the pair, and the sums are scaled by the
// steps.
__device__ __forceinline__ void gather_and_write_s16(const MapDev& M, const RaysOutDev& out, uint32_t n,
                                                     uint32_t r, const Classified& c, GatherItem* gq, float* ob)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned mv = __ballot_sync(full, c.ip);
    const int nv = __popc(mv);
    if (c.ip) {
        GatherItem e;
        e.slot = (uint32_t)lane;
        e.base = c.base;
#pragma unroll
        for (int d = 0; d < 5; ++d) e.f[d] = c.f[d];
        e.pad = 0.0f;
        gq[__popc(mv & ((1u << lane) - 1u))] = e;
    }
    __syncwarp();
    const int part = lane & 1;
    const uint32_t s0 = M.stride[0], s1 = M.stride[1], s2 = M.stride[2], s3 = M.stride[3];
#pragma unroll 1
    for (int g0 = 0; g0 < nv; g0 += 16) {
        const int gi = g0 + (lane >> 1);
        const bool act = gi < nv;
        const GatherItem e = gq[min(gi, nv - 1)];
        const float fl = part ? e.f[4] : 1.0f - e.f[4];
        const uint4* __restrict__ p = M.node16 + (size_t)e.base + part;
        float a[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (act) {
#pragma unroll
            for (int qq = 0; qq < 16; ++qq) {
                const uint32_t off = ((qq & 8) ? s0 : 0u) + ((qq & 4) ? s1 : 0u) + ((qq & 2) ? s2 : 0u) +
                                     ((qq & 1) ? s3 : 0u);
                const uint4 v = __ldg(p + off);
                const float w = (((qq & 8) ? e.f[0] : 1.0f - e.f[0]) * ((qq & 4) ? e.f[1] : 1.0f - e.f[1])) *
                                (((qq & 2) ? e.f[2] : 1.0f - e.f[2]) * (((qq & 1) ? e.f[3] : 1.0f - e.f[3]) * fl));
                a[0] = fmaf(w, s16_lo(v.x), a[0]);
                a[1] = fmaf(w, s16_hi(v.x), a[1]);
                a[2] = fmaf(w, s16_lo(v.y), a[2]);
                a[3] = fmaf(w, s16_hi(v.y), a[3]);
                a[4] = fmaf(w, s16_lo(v.z), a[4]);
                a[5] = fmaf(w, s16_hi(v.z), a[5]);
            }
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) a[k] += __shfl_xor_sync(full, a[k], 1);
        if (act && part == 0) {
            float* o = ob + e.slot * kObStride;
#pragma unroll
            for (int k = 0; k < 6; ++k) o[k] = a[k] * M.qstep[k];
        }
    }
    __syncwarp();
    if (r < n) {
        float o[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (c.ip) {
#pragma unroll
            for (int k = 0; k < 6; ++k) o[k] = ob[lane * kObStride + k];
            const float n2 = fmaf(o[2], o[2], fmaf(o[3], o[3], o[4] * o[4]));
            float inv = n2 > 0.0f ? rsqrtf(n2) : 0.0f;
            inv = inv * fmaf(-0.5f * n2, inv * inv, 1.5f);
            o[2] *= inv;
            o[3] *= inv;
            o[4] *= inv;
        }
        store_out(out, r, o, c.ip ? LT_FLAG_VALID : 0u);
    }
}

template <bool S16>
__device__ __forceinline__ void gather_any(const MapDev& M, const RaysOutDev& out, uint32_t n, uint32_t r,
                                           const Classified& c, GatherItem* gq, float* ob)
{
    if (S16) gather_and_write_s16(M, out, n, r, c, gq, ob);
    else gather_and_write(M, out, n, r, c, gq, ob);
}

template <int MODE, bool CAUCHY, bool S16>
__global__ void __launch_bounds__(kQTile)
map_query_kernel(const __grid_constant__ MapDev M, RaysInDev in, RaysOutDev out, uint32_t n, TraceQueue Q)
{
    __shared__ GatherItem gq_all[kQWarps][32];
    __shared__ float ob_all[kQWarps][32 * kObStride];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t r = blockIdx.x * kQTile + threadIdx.x;
    const Classified c = classify_ray<MODE>(M, in, n, r);
    const unsigned m = __ballot_sync(full, c.tr);
    if (m) {
        const int leader = __ffs(m) - 1;
        uint32_t b = 0;
        const uint32_t seg = blockIdx.x % kQSegs;
        if (lane == leader) b = atomicAdd(Q.count + seg * kQCountStride, (uint32_t)__popc(m));
        b = __shfl_sync(full, b, leader);
        if (c.tr) {
            const uint32_t k = seg * Q.segcap + b + __popc(m & ((1u << lane) - 1u));
            Q.x[k] = c.x;
            Q.y[k] = c.y;
            Q.dx[k] = c.dx;
            Q.dy[k] = c.dy;
            Q.dz[k] = c.dz;
            Q.lam[k] = c.lam;
            Q.tag[k] = c.tag;
        }
    }
    gather_any<S16>(M, out, n, r, c, gq_all[warp], ob_all[warp]);
}

// The one-kernel query's trace of its block's listed BOUNDARY and outside
// rays (tlist: the ray's slot in the block | the outside bit), with survivor
// compaction in S.
template <bool CAUCHY>
__device__ __forceinline__ void fused_trace_listed(const MapDev& M, const RaysInDev& in, const RaysOutDev& out,
                                                   uint32_t r0, uint32_t nt, const uint32_t* tlist,
                                                   TraceSmem<kQTile>& S, unsigned long long* work)
{
    const int t = threadIdx.x;
    // trace the listed rays, thread k taking entry k
    RayState st;
    bool live = false;
    uint32_t e = 0;
    S.of[t] = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) S.ob[q][t] = 0.0f;
    if ((uint32_t)t < nt) {
        e = tlist[t];
        const uint32_t rr = r0 + (e & ~kOutsideBit);
        live = trace_init(__ldg(in.x + rr), __ldg(in.y + rr), __ldg(in.dx + rr), __ldg(in.dy + rr),
                          __ldg(in.dz + rr), __ldg(in.lam + rr), st);
        if (!live) S.of[t] = (uint8_t)st.flags;
    }
    const int nint = trace_block_states<CAUCHY, kQTile>(M.L, M.pi, M.pj, live, st, S);
    __syncthreads();
    if ((uint32_t)t < nt) {
        const uint32_t rr = r0 + (e & ~kOutsideBit);
        const float o[6] = {S.ob[0][t], S.ob[1][t], S.ob[2][t], S.ob[3][t], S.ob[4][t], S.ob[5][t]};
        store_out(out, rr, o, S.of[t] | LT_FLAG_TRACED | ((e & kOutsideBit) ? LT_FLAG_OUTSIDE : 0u));
    }
    warp_add(work, (unsigned)nint);
}

// the same, as a call (its own register allocation)
template <bool CAUCHY>
__device__ __noinline__ void fused_trace_listed_call(const MapDev& M, const RaysInDev& in, const RaysOutDev& out,
                                                     uint32_t r0, uint32_t nt, const uint32_t* tlist,
                                                     TraceSmem<kQTile>& S, unsigned long long* work)
{
    fused_trace_listed<CAUCHY>(M, in, out, r0, nt, tlist, S, work);
}

// The whole query in one kernel, for small batches (fewer blocks than the
// GPU holds at once, where the second launch and its queue cost more than
// they save): each block classifies and gathers as map_query_kernel does,
// lists its BOUNDARY and outside rays in shared memory, and traces them
// itself with survivor compaction (trace_block_states).
//
// The body is a device function of the block index within the batch, so that
// the server's fused launch (serve_query_kernel) runs the same code for each
// request's blocks.
template <int MODE, bool CAUCHY, bool S16>
__device__ __forceinline__ void fused_query_block(const MapDev& M, const RaysInDev& in, const RaysOutDev& out,
                                                  uint32_t n, uint32_t blk, unsigned long long* work)
{
    __shared__ GatherItem gq_all[kQWarps][32];
    __shared__ float ob_all[kQWarps][32 * kObStride];
    __shared__ TraceSmem<kQTile> S;
    __shared__ uint32_t tlist[kQTile];
    __shared__ uint32_t tcount;
    const unsigned full = 0xffffffffu;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) tcount = 0;
    __syncthreads();
    const uint32_t r0 = blk * kQTile;
    const uint32_t r = r0 + t;
    const Classified c = classify_ray<MODE>(M, in, n, r);
    const unsigned m = __ballot_sync(full, c.tr);
    if (m) {
        const int leader = __ffs(m) - 1;
        uint32_t b = 0;
        if (lane == leader) b = atomicAdd(&tcount, (uint32_t)__popc(m));
        b = __shfl_sync(full, b, leader);
        if (c.tr) tlist[b + __popc(m & ((1u << lane) - 1u))] = (uint32_t)t | (c.tag & kOutsideBit);
    }
    gather_any<S16>(M, out, n, r, c, gq_all[warp], ob_all[warp]);
    __syncthreads();
    const uint32_t nt = tcount;
    if (nt == 0) return;
    // The FP32-node instantiation calls the tracer out of line: inlined, the
    // compiler gives the whole kernel 48 registers and the quad gather loses
    // loads in flight (65,536 singlet rays: 0.041 against 0.034 ms out of
    // line).  The 16-bit gather is faster with the tracer inlined (0.023
    // against 0.029 ms).
    if (S16) fused_trace_listed<CAUCHY>(M, in, out, r0, nt, tlist, S, work);
    else fused_trace_listed_call<CAUCHY>(M, in, out, r0, nt, tlist, S, work);
}

template <int MODE, bool CAUCHY, bool S16>
__global__ void __launch_bounds__(kQTile)
map_query_fused_kernel(const __grid_constant__ MapDev M, RaysInDev in, RaysOutDev out, uint32_t n,
                       unsigned long long* work)
{
    fused_query_block<MODE, CAUCHY, S16>(M, in, out, n, blockIdx.x, work);
}

// The server's fused launch of several small table-map queries (each block
// serves one request; every request's map has the same MODE and dispersion
// form): the block stages its request's map constants (a device copy of its
// MapDev) in shared memory and runs the one-kernel query on its rays.
static_assert(sizeof(MapDev) % 16 == 0, "MapDev is staged in 16-byte words");

template <int MODE, bool CAUCHY, bool S16>
__global__ void __launch_bounds__(kQTile)
serve_query_kernel(const __grid_constant__ ReqTable T, unsigned long long* work)
{
    __shared__ MapDev sm;
    const int k = req_of_block(T, blockIdx.x);
    const ReqItem& it = T.item[k];
    stage_words(&sm, it.dev, sizeof(MapDev));
    __syncthreads();
    fused_query_block<MODE, CAUCHY, S16>(sm, it.in, it.out, it.n, blockIdx.x - T.block0[k], work);
}

// The exact tracer over the query's trace queue (see map_query_kernel):
// blocks take kQBlock-ray chunks of the queue's segments from a counter until
// none is left (chunk c of the launch: segment s with cum[s] <= c <
// cum[s + 1], cum the prefix sum of the segments' chunk counts).
// Twelve resident 128-thread blocks per SM (40 registers, a few spilled):
// measured faster than 256-ray chunks, or fewer blocks at 48 or 60
// registers.  Launched as a programmatic dependent of map_query_kernel: its
// blocks may become resident while that kernel drains, and wait for it to
// complete (griddepcontrol.wait) before reading the queue.
template <bool CAUCHY>
__global__ void __launch_bounds__(kQBlock, 12)
map_trace_kernel(const __grid_constant__ MapDev M, RaysOutDev out, TraceQueue Q, unsigned long long* work)
{
    __shared__ TraceSmem<kQBlock> S;
    __shared__ uint32_t cnt[kQSegs], cum[kQSegs + 1];
    __shared__ uint32_t chunk, cseg;
    const int t = threadIdx.x;
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    if (t < kQSegs) cnt[t] = Q.count[t * kQCountStride];
    __syncthreads();
    if (t == 0) {
        uint32_t c = 0;
        for (int s = 0; s < kQSegs; ++s) {
            cum[s] = c;
            c += (cnt[s] + kQBlock - 1) / kQBlock;
        }
        cum[kQSegs] = c;
    }
    __syncthreads();
    const uint32_t nchunks = cum[kQSegs];
    int nint = 0;
#pragma unroll 1
    while (true) {
        if (t == 0) {
            const uint32_t c = atomicAdd(Q.count + kQSegs * kQCountStride, 1u);
            int s = 0;
            while (s < kQSegs - 1 && cum[s + 1] <= c) ++s;
            chunk = c;
            cseg = (uint32_t)s;
        }
        __syncthreads();
        if (chunk >= nchunks) break;
        const uint32_t sg = cseg;
        const uint32_t i = (chunk - cum[sg]) * (uint32_t)kQBlock + (uint32_t)t;   // entry within the segment
        const bool have = i < cnt[sg];
        const uint32_t k = sg * Q.segcap + i;
        uint32_t e = 0;
        RayState st;
        bool live = false;
        S.of[t] = 0;
#pragma unroll
        for (int q = 0; q < 6; ++q) S.ob[q][t] = 0.0f;
        if (have) {
            e = Q.tag[k];
            live = trace_init(Q.x[k], Q.y[k], Q.dx[k], Q.dy[k], Q.dz[k], Q.lam[k], st);
            if (!live) S.of[t] = (uint8_t)st.flags;
        }
        nint += trace_block_states<CAUCHY, kQBlock>(M.L, M.pi, M.pj, live, st, S);
        __syncthreads();
        if (have) {
            const uint32_t r = e & ~kOutsideBit;
            const float o[6] = {S.ob[0][t], S.ob[1][t], S.ob[2][t], S.ob[3][t], S.ob[4][t], S.ob[5][t]};
            store_out(out, r, o, S.of[t] | LT_FLAG_TRACED | ((e & kOutsideBit) ? LT_FLAG_OUTSIDE : 0u));
        }
        __syncthreads();
    }
    warp_add(work, (unsigned)nint);
}

// ------------------------------------------------------------------ scratch pool

static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

lt_status scratch_pool(cudaMemPool_t* pool)
{
    int dev = 0;
    LT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(LT_EINVAL, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        LT_CUDA_TRY(cudaMemPoolCreate(&g_pool[dev], &props));
        uint64_t keep = ~0ull;  // keep freed blocks for reuse by later calls
        LT_CUDA_TRY(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    }
    *pool = g_pool[dev];
    return LT_OK;
}

TraceQueue trace_queue_at(void* scratch, size_t n)
{
    char* p = static_cast<char*>(scratch);
    const size_t segcap = query_segcap(n), cap = (size_t)kQSegs * segcap;
    TraceQueue Q;
    Q.count = reinterpret_cast<uint32_t*>(p);
    Q.segcap = (uint32_t)segcap;
    float** fq[6] = {&Q.x, &Q.y, &Q.dx, &Q.dy, &Q.dz, &Q.lam};
    for (int q = 0; q < 6; ++q) *fq[q] = reinterpret_cast<float*>(p + kQHeaderBytes + (size_t)q * cap * 4);
    Q.tag = reinterpret_cast<uint32_t*>(p + kQHeaderBytes + 6 * cap * 4);
    return Q;
}

// a query kernel's instantiation by mode, dispersion form and node format
// (QM, QC, QS in the statement)
#define LT_QDISPATCH1(QMV, CA, S16, ...)                                                              \
    do {                                                                                              \
        constexpr int QM = QMV;                                                                       \
        if (CA) {                                                                                     \
            constexpr bool QC = true;                                                                 \
            if (S16) { constexpr bool QS = true; __VA_ARGS__; } else { constexpr bool QS = false; __VA_ARGS__; } \
        } else {                                                                                      \
            constexpr bool QC = false;                                                                \
            if (S16) { constexpr bool QS = true; __VA_ARGS__; } else { constexpr bool QS = false; __VA_ARGS__; } \
        }                                                                                             \
    } while (0)
#define LT_QDISPATCH(TABLE, CA, S16, ...)                                   \
    do {                                                                    \
        if (TABLE) LT_QDISPATCH1(LT_QUERY_TABLE, CA, S16, __VA_ARGS__);     \
        else LT_QDISPATCH1(LT_QUERY_NO_MASK, CA, S16, __VA_ARGS__);         \
    } while (0)

// the classify-and-gather kernel on `st` (the queue's counters already cleared)
static lt_status launch_classify(const lt_map* map, const RaysInDev& in, const RaysOutDev& out, uint32_t n,
                                 int mode, const TraceQueue& Q, cudaStream_t st)
{
    const unsigned blocks = (n + kQTile - 1) / kQTile;
    const bool table = mode == LT_QUERY_TABLE;
    ProfScope prof("map_query_kernel", st);
    LT_QDISPATCH(table, map->cauchy, map->node_format == LT_NODE_S16,
                 map_query_kernel<QM, QC, QS><<<blocks, kQTile, 0, st>>>(map->dev, in, out, n, Q));
    LT_CUDA_TRY(cudaGetLastError());
    return LT_OK;
}

// the tracer over the queue of a classify launch of n rays, on `st`
lt_status launch_queue_trace(const lt_map* map, const RaysOutDev& out, uint32_t n, const TraceQueue& Q,
                             cudaStream_t st)
{
    const void* trace = map->cauchy ? (const void*)map_trace_kernel<true> : (const void*)map_trace_kernel<false>;
    // resident blocks, but no more than a quarter of the rays could keep busy
    // (blocks take chunks from a counter, so any grid traces the whole queue)
    const unsigned gt = persistent_blocks(trace, kQBlock, ((size_t)n + 3) / 4, 32);
    ProfScope prof("map_trace_kernel", st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(gt);
    cfg.blockDim = dim3(kQBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    unsigned long long* w = prof.work();
    if (map->cauchy) LT_CUDA_TRY(cudaLaunchKernelEx(&cfg, map_trace_kernel<true>, map->dev, out, Q, w));
    else LT_CUDA_TRY(cudaLaunchKernelEx(&cfg, map_trace_kernel<false>, map->dev, out, Q, w));
    return LT_OK;
}

lt_status launch_query_with(const lt_map* map, const RaysInDev& in, const RaysOutDev& out, uint32_t n,
                            int mode, const TraceQueue& Q, cudaStream_t st)
{
    if (map->kind == LT_MAP_KIND_POLY) return launch_poly_fused(map, in, out, n, mode, st);
    LT_CUDA_TRY(cudaMemsetAsync(Q.count, 0, kQHeaderBytes, st));
    lt_status s = launch_classify(map, in, out, n, mode, Q, st);
    if (s != LT_OK) return s;
    return launch_queue_trace(map, out, n, Q, st);
}

lt_status launch_query(const lt_map* map, const RaysInDev& in, const RaysOutDev& out, uint32_t n,
                       int mode, cudaStream_t st)
{
    if (map->kind == LT_MAP_KIND_POLY) return launch_poly_query(map, in, out, n, mode, st);
    if (n <= kFusedMaxRays) {
        const unsigned blocks = (n + kQTile - 1) / kQTile;
        const bool table = mode == LT_QUERY_TABLE;
        ProfScope prof("map_query_fused_kernel", st);
        LT_QDISPATCH(table, map->cauchy, map->node_format == LT_NODE_S16,
                     map_query_fused_kernel<QM, QC, QS><<<blocks, kQTile, 0, st>>>(map->dev, in, out, n, prof.work()));
        LT_CUDA_TRY(cudaGetLastError());
        return LT_OK;
    }
    cudaMemPool_t pool;
    lt_status s = scratch_pool(&pool);
    if (s != LT_OK) return s;
    const size_t bytes = query_scratch_bytes(n);
    char* buf = nullptr;
    if (cudaMallocFromPoolAsync((void**)&buf, bytes, pool, st) != cudaSuccess)
        return fail(LT_ENOMEM, "lt_query: trace queue allocation of %zu bytes failed", bytes);
    s = launch_query_with(map, in, out, n, mode, trace_queue_at(buf, n), st);
    cudaFreeAsync(buf, st);
    return s;
}

lt_status launch_fused_table(const ReqTable& T, int mode, bool cauchy, bool s16, cudaStream_t st)
{
    if (T.n_items < 1 || T.n_items > kMaxFuse) return fail(LT_EINVAL, "fused query: %d requests", T.n_items);
    const unsigned blocks = T.block0[T.n_items];
    const bool table = mode == LT_QUERY_TABLE;
    ProfScope prof("serve_query_kernel", st);
    LT_QDISPATCH(table, cauchy, s16, serve_query_kernel<QM, QC, QS><<<blocks, kQTile, 0, st>>>(T, prof.work()));
    LT_CUDA_TRY(cudaGetLastError());
    return LT_OK;
}

lt_status launch_map_classify(const uint8_t* corner_bits, const uint32_t* seen, const uint32_t* resmax,
                              float tol, uint32_t* cls, uint32_t NC, unsigned long long* counts,
                              cudaStream_t st)
{
    uint32_t tol_bits;
    std::memcpy(&tol_bits, &tol, 4);
    const uint32_t NW = (NC + 15) / 16;
    map_classify_kernel<<<(NW + 255) / 256, 256, 0, st>>>(corner_bits, seen, resmax, tol_bits, cls, NC, counts);
    LT_CUDA_TRY(cudaGetLastError());
    return LT_OK;
}

// LT_NODE_S16: steps from the largest |value| of each output over the valid
// nodes (step_k = 2^(e_k - 15), 2^(e_k - 1) <= max < 2^e_k), the 16-bit
// records, then the FP32 table is released.
lt_status quantize_nodes(lt_map* m, cudaStream_t st)
{
    const uint32_t N = (uint32_t)m->n_nodes;
    unsigned* mx = nullptr;
    if (cudaMalloc(&mx, 6 * sizeof(unsigned)) != cudaSuccess) return fail(LT_ENOMEM, "lt_build_map: quantisation");
    unsigned hm[6] = {0, 0, 0, 0, 0, 0};
    cudaError_t e = cudaMemsetAsync(mx, 0, 6 * sizeof(unsigned), st);
    if (e == cudaSuccess) {
        const unsigned g = std::min<unsigned>((N + 255) / 256, 152u * 8u);
        map_absmax_kernel<<<g, 256, 0, st>>>(m->node, m->node_valid, N, mx);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hm, mx, sizeof hm, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(mx);
    if (e != cudaSuccess) return cuda_fail(e, "lt_build_map: quantisation");
    QuantInv Q;
    for (int k = 0; k < 6; ++k) {
        float mk;
        std::memcpy(&mk, &hm[k], 4);
        int ex = 0;
        if (mk > 0.0f) std::frexp((double)mk, &ex);
        m->dev.qstep[k] = (float)std::ldexp(1.0, ex - 15);
        Q.inv[k] = (float)std::ldexp(1.0, 15 - ex);
        m->stats.node_step[k] = m->dev.qstep[k];
    }
    if (cudaMalloc(&m->node16, (size_t)N * 16) != cudaSuccess) return fail(LT_ENOMEM, "lt_build_map: 16-bit table");
    map_quantize_kernel<<<(N + 255) / 256, 256, 0, st>>>(m->node, m->node_valid, N, Q, m->node16);
    LT_CUDA_TRY(cudaGetLastError());
    LT_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(m->node);
    m->node = nullptr;
    m->dev.node = nullptr;
    m->dev.node16 = m->node16;
    m->node_format = LT_NODE_S16;
    m->stats.node_format = LT_NODE_S16;
    return LT_OK;
}

// A map's tables live on the device it was built or loaded on; a call made
// with another device current would launch there and read them across
// devices.
lt_status check_map_device(const lt_map* m, const char* who)
{
    int dev = 0;
    LT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != m->device)
        return fail(LT_EINVAL, "%s: the map lives on device %d but device %d is current", who, m->device, dev);
    return LT_OK;
}

}  // namespace lt

using namespace lt;

lt_map::~lt_map()
{
    if (node) cudaFree(node);
    if (node16) cudaFree(node16);
    if (node_valid) cudaFree(node_valid);
    if (cls) cudaFree(cls);
    if (coefg) cudaFree(coefg);
    if (coef64) cudaFree(coef64);
    if (patch_ok) cudaFree(patch_ok);
}

extern "C" {

lt_status lt_build_map(const lt_lens* lens, const lt_map_opts* o, lt_map** out, lt_stream stream)
{
    clear_error();
    auto t0 = std::chrono::steady_clock::now();
    if (!lens || !o || !out) return fail(LT_EINVAL, "lt_build_map: NULL argument");
    *out = nullptr;
    int pi, pj;
    if (!path_ij(lens->S, o->path_id, &pi, &pj))
        return fail(LT_EINVAL, "lt_build_map: bad path id %d", o->path_id);
    uint64_t N = 1, NC = 1;
    for (int d = 0; d < 5; ++d) {
        if (o->res[d] < 2 || o->res[d] > 4096) return fail(LT_EINVAL, "lt_build_map: res[%d] = %d outside 2..4096", d, o->res[d]);
        if (!(o->hi[d] > o->lo[d])) return fail(LT_EINVAL, "lt_build_map: empty box on axis %d", d);
        N *= (uint64_t)o->res[d];
        NC *= (uint64_t)(o->res[d] - 1);
    }
    if (N * kNodeFloats >= (1ull << 32)) return fail(LT_EINVAL, "lt_build_map: %llu nodes is too many", (unsigned long long)N);
    if (o->node_format != LT_NODE_F32 && o->node_format != LT_NODE_S16)
        return fail(LT_EINVAL, "lt_build_map: unknown node format %d", o->node_format);
    if (o->n_fit > 0) {
        const void* ps[] = {o->fit_x, o->fit_y, o->fit_dx, o->fit_dy, o->fit_dz, o->fit_lambda};
        for (const void* p : ps)
            if (!p || !aligned16(p)) return fail(LT_EINVAL, "lt_build_map: fit arrays must be non-NULL and 16-byte aligned");
        if (o->n_fit >= (1ull << 31)) return fail(LT_EINVAL, "lt_build_map: too many fit rays");
    }
    cudaStream_t st = (cudaStream_t)stream;

    lt_map* m = new (std::nothrow) lt_map();
    if (!m) return fail(LT_ENOMEM, "lt_build_map: host allocation");
    m->lens = *lens;
    m->lens.presc.surfaces = m->lens.surf;
    m->lens.presc.glasses = m->lens.glass;
    m->path_id = o->path_id;
    m->n_nodes = N;
    m->n_cells = NC;
    m->tol = o->max_residual_mm;
    MapDev& D = m->dev;
    std::memset(&D, 0, sizeof D);
    D.L = lens->dev;
    m->cauchy = lens_all_cauchy(lens->dev);
    D.pi = pi;
    D.pj = pj;
    uint32_t stride = 1, cstride = 1;
    for (int d = 4; d >= 0; --d) {
        m->res[d] = o->res[d];
        m->lo[d] = o->lo[d];
        m->hi[d] = o->hi[d];
        D.res[d] = o->res[d];
        D.lo[d] = (float)o->lo[d];
        D.step[d] = (float)((o->hi[d] - o->lo[d]) / (double)(o->res[d] - 1));
        D.inv[d] = (float)((double)(o->res[d] - 1) / (o->hi[d] - o->lo[d]));
        D.umax[d] = (float)(o->res[d] - 1);
        D.stride[d] = stride;
        D.cstride[d] = cstride;
        stride *= (uint32_t)o->res[d];
        cstride *= (uint32_t)(o->res[d] - 1);
    }
    const uint32_t NW = (uint32_t)((NC + 15) / 16);
    auto bail = [&](lt_status s) { delete m; return s; };
    if (cudaMalloc(&m->node, N * kNodeFloats * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&m->node_valid, N) != cudaSuccess ||
        cudaMalloc(&m->cls, (size_t)NW * sizeof(uint32_t)) != cudaSuccess)
        return bail(fail(LT_ENOMEM, "lt_build_map: device allocation of the tables failed"));
    D.node = m->node;
    D.cls = m->cls;

    // temporaries
    uint8_t* corner_bits = nullptr;
    uint32_t* seen = nullptr;
    uint32_t* resmax = nullptr;
    FitAccum* acc = nullptr;
    unsigned long long* counts = nullptr;
    const bool use_tol = o->max_residual_mm > 0.0;
    lt_status s = LT_OK;
    do {
        if (cudaMalloc(&corner_bits, NC) != cudaSuccess ||
            cudaMalloc(&seen, (size_t)NW * 4) != cudaSuccess ||
            (use_tol && cudaMalloc(&resmax, NC * 4) != cudaSuccess) ||
            cudaMalloc(&acc, sizeof(FitAccum)) != cudaSuccess ||
            cudaMalloc(&counts, 3 * sizeof(unsigned long long)) != cudaSuccess) {
            s = fail(LT_ENOMEM, "lt_build_map: device allocation of temporaries failed");
            break;
        }
        if (cudaMemsetAsync(seen, 0, (size_t)NW * 4, st) != cudaSuccess ||
            (use_tol && cudaMemsetAsync(resmax, 0, NC * 4, st) != cudaSuccess) ||
            cudaMemsetAsync(acc, 0, sizeof(FitAccum), st) != cudaSuccess ||
            cudaMemsetAsync(counts, 0, 24, st) != cudaSuccess) {
            s = fail(LT_ECUDA, "lt_build_map: memset failed");
            break;
        }
        if (m->cauchy)
            map_node_kernel<true><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(D, m->node, m->node_valid, (uint32_t)N);
        else
            map_node_kernel<false><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(D, m->node, m->node_valid, (uint32_t)N);
        map_corner_kernel<<<(unsigned)((NC + 255) / 256), 256, 0, st>>>(D, m->node_valid, corner_bits, (uint32_t)NC);
        if (o->n_fit > 0) {
            RaysInDev fit{o->fit_x, o->fit_y, o->fit_dx, o->fit_dy, o->fit_dz, o->fit_lambda};
            const unsigned fb = (unsigned)((o->n_fit + 255) / 256);
            if (m->cauchy)
                map_fit_kernel<true><<<fb, 256, 0, st>>>(D, fit, (uint32_t)o->n_fit, m->node, corner_bits,
                                                          seen, resmax, acc);
            else
                map_fit_kernel<false><<<fb, 256, 0, st>>>(D, fit, (uint32_t)o->n_fit, m->node, corner_bits,
                                                           seen, resmax, acc);
        }
        float tol_f = use_tol ? (float)o->max_residual_mm : 0.0f;
        uint32_t tol_bits;
        std::memcpy(&tol_bits, &tol_f, 4);
        map_classify_kernel<<<(NW + 255) / 256, 256, 0, st>>>(corner_bits, seen, resmax, tol_bits, m->cls,
                                                               (uint32_t)NC, counts);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { s = cuda_fail(e, "lt_build_map launch"); break; }
        FitAccum ha;
        unsigned long long hc[3];
        if (cudaMemcpyAsync(&ha, acc, sizeof ha, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(hc, counts, sizeof hc, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            s = cuda_fail(e, "lt_build_map");
            break;
        }
        // valid nodes: count on the host from the byte array would need a copy; reuse counts
        m->stats.n_nodes = N;
        m->stats.n_cells = NC;
        m->stats.cells_invalid = hc[0];
        m->stats.cells_valid = hc[1];
        m->stats.cells_boundary = hc[2];
        m->stats.fit_inside = ha.inside;
        m->stats.fit_valid = ha.valid;
        m->stats.fit_residual_rms_mm = ha.n_res ? std::sqrt(ha.sumsq / (double)ha.n_res) : 0.0;
        float mx;
        std::memcpy(&mx, &ha.max_res_bits, 4);
        m->stats.fit_residual_max_mm = mx;
        m->stats.table_bytes = N * kNodeFloats * 4 + N + (uint64_t)NW * 4;
        m->stats.node_format = LT_NODE_F32;
        if (o->node_format == LT_NODE_S16) {
            // the half-size table from the FP32 one, which is then released
            s = quantize_nodes(m, st);
            if (s != LT_OK) break;
            m->stats.table_bytes = N * 16 + N + (uint64_t)NW * 4;
        }
    } while (0);
    if (corner_bits) cudaFree(corner_bits);
    if (seen) cudaFree(seen);
    if (resmax) cudaFree(resmax);
    if (acc) cudaFree(acc);
    if (counts) cudaFree(counts);
    if (s != LT_OK) return bail(s);
    cudaGetDevice(&m->device);
    m->stats.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = m;
    return LT_OK;
}

void lt_destroy_map(lt_map* m) { delete m; }

lt_status lt_map_stats_get(const lt_map* m, lt_map_stats* out)
{
    if (!m || !out) return fail(LT_EINVAL, "lt_map_stats_get: NULL argument");
    *out = m->stats;
    return LT_OK;
}

lt_status lt_query(const lt_map* m, const lt_rays_in* in, const float* lam, const lt_rays_out* out,
                   size_t n, int32_t mode, lt_stream stream)
{
    clear_error();
    if (!m) return fail(LT_EINVAL, "lt_query: NULL map");
    if (mode != LT_QUERY_TABLE && mode != LT_QUERY_NO_MASK) return fail(LT_EINVAL, "lt_query: unknown mode %d", mode);
    lt_status s = check_io(in, lam, out, n, "lt_query");
    if (s != LT_OK || n == 0) return s;
    s = check_map_device(m, "lt_query");
    if (s != LT_OK) return s;
    if (n >= (1ull << 31)) return fail(LT_EINVAL, "lt_query: n must be < 2^31");
    RaysInDev din{in->x, in->y, in->dx, in->dy, in->dz, lam};
    RaysOutDev dout{out->x, out->y, out->dx, out->dy, out->dz, out->I, out->flags};
    return launch_query(m, din, dout, (uint32_t)n, mode, (cudaStream_t)stream);
}

lt_status lt_query_host(const lt_map* m, const lt_rays_in* in, const float* lam,
                        const lt_rays_out* out, size_t n, int32_t mode)
{
    clear_error();
    if (!m) return fail(LT_EINVAL, "lt_query_host: NULL map");
    if (mode != LT_QUERY_TABLE && mode != LT_QUERY_NO_MASK) return fail(LT_EINVAL, "lt_query_host: unknown mode %d", mode);
    if (!in || !out) return fail(LT_EINVAL, "lt_query_host: NULL ray struct");
    if (n == 0) return LT_OK;
    const void* ps[] = {in->x, in->y, in->dx, in->dy, in->dz, lam, out->x, out->y,
                        out->dx, out->dy, out->dz, out->I, out->flags};
    for (const void* p : ps)
        if (!p) return fail(LT_EINVAL, "lt_query_host: NULL ray array");
    lt_status sd = check_map_device(m, "lt_query_host");
    if (sd != LT_OK) return sd;
    return run_host_pipelined(in, lam, out, n, [&](const RaysInDev& a, const RaysOutDev& b, size_t k, cudaStream_t st) {
        return launch_query(m, a, b, (uint32_t)k, mode, st);
    });
}

lt_status lt_map_export(const lt_map* m, float* node6, uint8_t* node_valid, uint8_t* cell_class)
{
    clear_error();
    if (!m) return fail(LT_EINVAL, "lt_map_export: NULL map");
    if (node6 && m->kind != LT_MAP_KIND_TABLE)
        return fail(LT_EINVAL, "lt_map_export: a polynomial-patch map has no node table (node6 must be NULL)");
    if (node6 && m->node_format == LT_NODE_S16) {
        // the decoded values q * step
        std::vector<int16_t> q(m->n_nodes * 8);
        LT_CUDA_TRY(cudaMemcpy(q.data(), m->node16, m->n_nodes * 16, cudaMemcpyDeviceToHost));
        for (uint64_t l = 0; l < m->n_nodes; ++l)
            for (int k = 0; k < 6; ++k) node6[l * 6 + k] = (float)q[l * 8 + k] * m->dev.qstep[k];
    } else if (node6) {
        LT_CUDA_TRY(cudaMemcpy2D(node6, 6 * sizeof(float), m->node, kNodeFloats * sizeof(float),
                                 6 * sizeof(float), m->n_nodes, cudaMemcpyDeviceToHost));
    }
    if (node_valid) LT_CUDA_TRY(cudaMemcpy(node_valid, m->node_valid, m->n_nodes, cudaMemcpyDeviceToHost));
    if (cell_class) {
        const size_t NW = (m->n_cells + 15) / 16;
        std::vector<uint32_t> w(NW);
        LT_CUDA_TRY(cudaMemcpy(w.data(), m->cls, NW * 4, cudaMemcpyDeviceToHost));
        for (uint64_t c = 0; c < m->n_cells; ++c) cell_class[c] = (uint8_t)((w[c >> 4] >> ((c & 15) * 2)) & 3);
    }
    return LT_OK;
}

// ---------------------------------------------------------------- save / load

struct MapFileHeader {
    char magic[8];
    uint32_t version;
    int32_t path_id;
    int32_t res[5];
    int32_t S, n_glass;
    double lo[5], hi[5];
    double tol;
    uint64_t n_nodes, n_cells;
};

lt_status lt_map_save(const lt_map* m, const char* path)
{
    clear_error();
    if (!m || !path) return fail(LT_EINVAL, "lt_map_save: NULL argument");
    if (m->kind != LT_MAP_KIND_TABLE || m->node_format != LT_NODE_F32)
        return fail(LT_EINVAL, "lt_map_save: only table maps with an FP32 node table are saved");
    std::vector<float> node(m->n_nodes * 6);
    std::vector<uint8_t> nv(m->n_nodes);
    const size_t NW = (m->n_cells + 15) / 16;
    std::vector<uint32_t> cls(NW);
    LT_CUDA_TRY(cudaMemcpy2D(node.data(), 6 * sizeof(float), m->node, kNodeFloats * sizeof(float),
                             6 * sizeof(float), m->n_nodes, cudaMemcpyDeviceToHost));
    LT_CUDA_TRY(cudaMemcpy(nv.data(), m->node_valid, nv.size(), cudaMemcpyDeviceToHost));
    LT_CUDA_TRY(cudaMemcpy(cls.data(), m->cls, NW * 4, cudaMemcpyDeviceToHost));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(LT_EIO, "lt_map_save: cannot open %s", path);
    MapFileHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "LTMAP01", 8);
    h.version = 2;   // 2: surface records carry the even-asphere terms
    h.path_id = m->path_id;
    for (int d = 0; d < 5; ++d) { h.res[d] = m->res[d]; h.lo[d] = m->lo[d]; h.hi[d] = m->hi[d]; }
    h.S = m->lens.S;
    h.n_glass = m->lens.n_glass;
    h.tol = m->tol;
    h.n_nodes = m->n_nodes;
    h.n_cells = m->n_cells;
    bool ok = std::fwrite(&h, sizeof h, 1, f) == 1;
    ok = ok && std::fwrite(m->lens.surf, sizeof(lt_surface), m->lens.S, f) == (size_t)m->lens.S;
    ok = ok && (m->lens.n_glass == 0 ||
                std::fwrite(m->lens.glass, sizeof(lt_glass), m->lens.n_glass, f) == (size_t)m->lens.n_glass);
    lt_prescription p = m->lens.presc;
    p.surfaces = nullptr;
    p.glasses = nullptr;
    ok = ok && std::fwrite(&p, sizeof p, 1, f) == 1;
    ok = ok && std::fwrite(&m->stats, sizeof m->stats, 1, f) == 1;
    ok = ok && std::fwrite(node.data(), 4, node.size(), f) == node.size();
    ok = ok && std::fwrite(nv.data(), 1, nv.size(), f) == nv.size();
    ok = ok && std::fwrite(cls.data(), 4, NW, f) == NW;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(LT_EIO, "lt_map_save: write to %s failed", path);
    return LT_OK;
}

lt_status lt_map_load(const char* path, lt_map** out)
{
    clear_error();
    if (!path || !out) return fail(LT_EINVAL, "lt_map_load: NULL argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(LT_EIO, "lt_map_load: cannot open %s", path);
    MapFileHeader h;
    lt_surface surf[LT_MAX_SURFACES];
    lt_glass glass[LT_MAX_GLASSES];
    lt_prescription p;
    lt_map_stats stats;
    bool ok = std::fread(&h, sizeof h, 1, f) == 1 && std::memcmp(h.magic, "LTMAP01", 8) == 0 &&
              h.version == 2 && h.S >= 1 && h.S <= LT_MAX_SURFACES && h.n_glass >= 0 && h.n_glass <= LT_MAX_GLASSES;
    ok = ok && std::fread(surf, sizeof(lt_surface), h.S, f) == (size_t)h.S;
    ok = ok && (h.n_glass == 0 || std::fread(glass, sizeof(lt_glass), h.n_glass, f) == (size_t)h.n_glass);
    ok = ok && std::fread(&p, sizeof p, 1, f) == 1 && std::fread(&stats, sizeof stats, 1, f) == 1 &&
         p.n_surfaces == h.S && p.n_glasses == h.n_glass;
    uint64_t N = 1, NC = 1;
    for (int d = 0; ok && d < 5; ++d) {
        ok = h.res[d] >= 2 && h.res[d] <= 4096 && std::isfinite(h.lo[d]) && std::isfinite(h.hi[d]) &&
             h.hi[d] > h.lo[d];
        N *= (uint64_t)h.res[d];
        NC *= (uint64_t)(h.res[d] - 1);
    }
    int pi = 0, pj = 0;
    ok = ok && path_ij(h.S, h.path_id, &pi, &pj);
    ok = ok && N == h.n_nodes && NC == h.n_cells && N * kNodeFloats < (1ull << 32);
    if (!ok) { std::fclose(f); return fail(LT_EIO, "lt_map_load: %s is not a map file", path); }
    std::vector<float> node(N * 6);
    std::vector<uint8_t> nv(N);
    const size_t NW = (NC + 15) / 16;
    std::vector<uint32_t> cls(NW);
    ok = std::fread(node.data(), 4, node.size(), f) == node.size() &&
         std::fread(nv.data(), 1, N, f) == N && std::fread(cls.data(), 4, NW, f) == NW;
    std::fclose(f);
    if (!ok) return fail(LT_EIO, "lt_map_load: %s is truncated", path);
    p.surfaces = surf;
    p.glasses = glass;
    lt_lens* lens = nullptr;
    lt_status s = lt_create_lens(&p, &lens);
    if (s != LT_OK) return s;
    // rebuild the map shell without tracing: corners-only options, then overwrite the tables
    lt_map* m = new (std::nothrow) lt_map();
    if (!m) { lt_destroy_lens(lens); return fail(LT_ENOMEM, "lt_map_load: host allocation"); }
    m->lens = *lens;
    m->lens.presc.surfaces = m->lens.surf;
    m->lens.presc.glasses = m->lens.glass;
    lt_destroy_lens(lens);
    m->path_id = h.path_id;
    m->n_nodes = N;
    m->n_cells = NC;
    m->tol = h.tol;
    m->stats = stats;
    MapDev& D = m->dev;
    std::memset(&D, 0, sizeof D);
    D.L = m->lens.dev;
    m->cauchy = lens_all_cauchy(m->lens.dev);
    D.pi = pi;
    D.pj = pj;
    uint32_t stride = 1, cstride = 1;
    for (int d = 4; d >= 0; --d) {
        m->res[d] = h.res[d];
        m->lo[d] = h.lo[d];
        m->hi[d] = h.hi[d];
        D.res[d] = h.res[d];
        D.lo[d] = (float)h.lo[d];
        D.step[d] = (float)((h.hi[d] - h.lo[d]) / (double)(h.res[d] - 1));
        D.inv[d] = (float)((double)(h.res[d] - 1) / (h.hi[d] - h.lo[d]));
        D.umax[d] = (float)(h.res[d] - 1);
        D.stride[d] = stride;
        D.cstride[d] = cstride;
        stride *= (uint32_t)h.res[d];
        cstride *= (uint32_t)(h.res[d] - 1);
    }
    if (cudaMalloc(&m->node, N * kNodeFloats * 4) != cudaSuccess || cudaMalloc(&m->node_valid, N) != cudaSuccess ||
        cudaMalloc(&m->cls, NW * 4) != cudaSuccess) {
        delete m;
        return fail(LT_ENOMEM, "lt_map_load: device allocation failed");
    }
    D.node = m->node;
    D.cls = m->cls;
    if (cudaMemset(m->node, 0, N * kNodeFloats * 4) != cudaSuccess ||
        cudaMemcpy2D(m->node, kNodeFloats * sizeof(float), node.data(), 6 * sizeof(float),
                     6 * sizeof(float), N, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->node_valid, nv.data(), N, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->cls, cls.data(), NW * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        delete m;
        return fail(LT_ECUDA, "lt_map_load: upload failed");
    }
    cudaGetDevice(&m->device);
    *out = m;
    return LT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free query

// The trace queue of lt_query_noalloc (layout of trace_queue_at for
// LT_NOALLOC_MAX_RAYS rays: 8,448 bytes of counters, then 28 bytes per
// ray).  A file-scope device array: every device that loads the library
// holds it until the process exits.
namespace {
constexpr size_t kNoallocQueueBytes = query_scratch_bytes(LT_NOALLOC_MAX_RAYS);
__device__ __align__(256) unsigned char g_noalloc_queue[kNoallocQueueBytes];

// Device address of the array on the current device.  In host code the
// symbol is only a host-side stand-in; kernels must be given this address.
// It is looked up on every call (a driver query that allocates nothing), so a
// device reset by the host application leaves no stale address behind.
lt_status noalloc_queue(void** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_queue);
    if (e != cudaSuccess || !p) return cuda_fail(e, "lt_query_noalloc: cudaGetSymbolAddress");
    *out = p;
    return LT_OK;
}
}  // namespace

extern "C" lt_status lt_query_noalloc(const lt_map* m, const lt_rays_in* in, const float* lam,
                                      const lt_rays_out* out, size_t n, int32_t mode,
                                      lt_stream stream)
{
    clear_error();
    if (!m) return fail(LT_EINVAL, "lt_query_noalloc: NULL map");
    if (mode != LT_QUERY_TABLE && mode != LT_QUERY_NO_MASK)
        return fail(LT_EINVAL, "lt_query_noalloc: unknown mode %d", mode);
    if (n > (size_t)LT_NOALLOC_MAX_RAYS)
        return fail(LT_EINVAL, "lt_query_noalloc: n = %zu exceeds LT_NOALLOC_MAX_RAYS (%d); split the batch",
                    n, LT_NOALLOC_MAX_RAYS);
    lt_status s = check_io(in, lam, out, n, "lt_query_noalloc");
    if (s != LT_OK || n == 0) return s;
    s = check_map_device(m, "lt_query_noalloc");
    if (s != LT_OK) return s;
    void* q = nullptr;
    s = noalloc_queue(&q);
    if (s != LT_OK) return s;
    RaysInDev din{in->x, in->y, in->dx, in->dy, in->dz, lam};
    RaysOutDev dout{out->x, out->y, out->dx, out->dy, out->dz, out->I, out->flags};
    // the queue's counters are cleared by launch_query_with on the call's stream
    return launch_query_with(m, din, dout, (uint32_t)n, mode, trace_queue_at(q, n), (cudaStream_t)stream);
}
