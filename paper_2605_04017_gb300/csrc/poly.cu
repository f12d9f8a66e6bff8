// Polynomial-patch lens transport map: build (unclipped-lens samples, FP64
// least-squares fit per patch, class-grid nodes through the real lens, cell
// classes) and query (symmetry reduction, mask lookup, FP32 Horner
// evaluation of the patch polynomial, exact-tracer fallback).
//
// The paper's factorisation (Sec. 4.2, Eq. 11) over its symmetry-reduced
// input (Sec. 4.1, Eq. 10): the mask g is 2 bits per class-grid cell, the
// regressor f a polynomial per patch fitted to traced rays.  The fit traces
// the unclipped lens (apertures and stop removed): apertures only decide
// whether a ray passes, so the function the valid rays follow is smooth
// across the vignetting edge and a low-degree polynomial on a coarse patch
// reproduces it to the FP32 tracer's own error, while the mask resolves the
// occlusion on a finer grid.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "map_internal.h"
#include "profile.h"
#include "tracer.cuh"

namespace lt {

constexpr int kPolyTile = 256;        // rays per block of the query kernels
constexpr int kMaxSamplesAxis = 8;

__host__ __device__ constexpr int poly_terms(int D) { return (D + 1) * (D + 2) * (D + 3) * (D + 4) / 24; }

// Exponents (a, b, c, e) of (xi_r, xi_p, xi_q, xi_w) in the order the Horner
// evaluation consumes coefficients: a, then b, then c, then e, each
// descending, over a + b + c + e <= D.
static void horner_exponents(int D, std::vector<int32_t>& e)
{
    e.clear();
    for (int a = D; a >= 0; --a)
        for (int b = D - a; b >= 0; --b)
            for (int c = D - a - b; c >= 0; --c)
                for (int d = D - a - b - c; d >= 0; --d) {
                    e.push_back(a);
                    e.push_back(b);
                    e.push_back(c);
                    e.push_back(d);
                }
}

// ------------------------------------------------------------------ evaluation

// The five outputs of a patch polynomial: (x', y'), (d_x', d_y') and I.
struct Acc5 {
    float2 p, d;
    float I;
};

__device__ __forceinline__ void acc_load(Acc5& a, const float4 v, float vi)
{
    a.p = make_float2(v.x, v.y);
    a.d = make_float2(v.z, v.w);
    a.I = vi;
}
__device__ __forceinline__ void acc_step(Acc5& a, float t, const float4 v, float vi)
{
    a.p.x = fmaf(a.p.x, t, v.x);
    a.p.y = fmaf(a.p.y, t, v.y);
    a.d.x = fmaf(a.d.x, t, v.z);
    a.d.y = fmaf(a.d.y, t, v.w);
    a.I = fmaf(a.I, t, vi);
}
__device__ __forceinline__ void acc_step(Acc5& a, float t, const Acc5& v)
{
    a.p.x = fmaf(a.p.x, t, v.p.x);
    a.p.y = fmaf(a.p.y, t, v.p.y);
    a.d.x = fmaf(a.d.x, t, v.d.x);
    a.d.y = fmaf(a.d.y, t, v.d.y);
    a.I = fmaf(a.I, t, v.I);
}

// Coefficient groups: per patch poly_groups(D) groups of four consecutive
// terms (horner_exponents order); group g is five float4s -- the x', y',
// d_x', d_y' and I coefficients of terms 4g .. 4g + 3 (zeros past the last
// term) -- so one 16-byte load brings an output's coefficients of four terms.
__host__ __device__ constexpr int poly_groups(int D) { return (poly_terms(D) + 3) / 4; }

__device__ __forceinline__ float f4c(const float4& v, int i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// The patch polynomial at NR points of one patch (NR = 1 or 2) by nested
// Horner steps (T - 1 FMAs per output and point):
// P = sum_a xi_r^a Q_a(xi_p, xi_q, xi_w), each Q_a likewise in the next
// variable.  The points share every coefficient load.
template <int D, int NR>
__device__ __forceinline__ void poly_eval(const float4* __restrict__ G, const float (*xi)[4], Acc5* res)
{
    float4 cur[5];
    int k = 0;
    Acc5 A0[NR];
#pragma unroll
    for (int a = D; a >= 0; --a) {
        Acc5 A1[NR];
#pragma unroll
        for (int b = D - a; b >= 0; --b) {
            Acc5 A2[NR];
#pragma unroll
            for (int c = D - a - b; c >= 0; --c) {
                Acc5 A3[NR];
#pragma unroll
                for (int e = D - a - b - c; e >= 0; --e) {
                    if (k % 4 == 0) {
#pragma unroll
                        for (int o = 0; o < 5; ++o) cur[o] = __ldg(G + (k / 4) * 5 + o);
                    }
                    const float4 v = make_float4(f4c(cur[0], k % 4), f4c(cur[1], k % 4), f4c(cur[2], k % 4),
                                                 f4c(cur[3], k % 4));
                    const float vi = f4c(cur[4], k % 4);
                    ++k;
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        if (e == D - a - b - c) acc_load(A3[r], v, vi);
                        else acc_step(A3[r], xi[r][3], v, vi);
                    }
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    if (c == D - a - b) A2[r] = A3[r];
                    else acc_step(A2[r], xi[r][2], A3[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (b == D - a) A1[r] = A2[r];
                else acc_step(A1[r], xi[r][1], A2[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (a == D) A0[r] = A1[r];
            else acc_step(A0[r], xi[r][0], A1[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) res[r] = A0[r];
}

// The same evaluation from a table in shared memory (plain loads).
template <int D, int NR>
__device__ __forceinline__ void poly_eval_tab(const float4* G, const float (*xi)[4], Acc5* res)
{
    float4 cur[5];
    int k = 0;
    Acc5 A0[NR];
#pragma unroll
    for (int a = D; a >= 0; --a) {
        Acc5 A1[NR];
#pragma unroll
        for (int b = D - a; b >= 0; --b) {
            Acc5 A2[NR];
#pragma unroll
            for (int c = D - a - b; c >= 0; --c) {
                Acc5 A3[NR];
#pragma unroll
                for (int e = D - a - b - c; e >= 0; --e) {
                    if (k % 4 == 0) {
#pragma unroll
                        for (int o = 0; o < 5; ++o) cur[o] = G[(k / 4) * 5 + o];
                    }
                    const float4 v = make_float4(f4c(cur[0], k % 4), f4c(cur[1], k % 4), f4c(cur[2], k % 4),
                                                 f4c(cur[3], k % 4));
                    const float vi = f4c(cur[4], k % 4);
                    ++k;
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        if (e == D - a - b - c) acc_load(A3[r], v, vi);
                        else acc_step(A3[r], xi[r][3], v, vi);
                    }
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    if (c == D - a - b) A2[r] = A3[r];
                    else acc_step(A2[r], xi[r][2], A3[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (b == D - a) A1[r] = A2[r];
                else acc_step(A1[r], xi[r][1], A2[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (a == D) A0[r] = A1[r];
            else acc_step(A0[r], xi[r][0], A1[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) res[r] = A0[r];
}

// The FP32 rule for the reduced coordinates (documented in lt.h): three
// correctly rounded divisions (1 / d_z, 1 / r, 1000 / lambda), every other
// operation a correctly rounded product, sum or square root; false for
// d_z <= 0, d_z infinite or lambda <= 0 (a NaN or infinity elsewhere makes
// the ray fall outside the box).
__device__ __forceinline__ bool poly_reduce(float x, float y, float dx, float dy, float dz, float lam,
                                            float u[4], float& c, float& s, float& m)
{
    // d_z must be positive and finite and lambda positive; any other NaN or
    // infinity reaches a reduced coordinate and fails the box test
    if (!((dz > 0.0f) & (dz < INFINITY) & (lam > 0.0f))) return false;
    const float idz = __frcp_rn(dz);
    const float sx = __fmul_rn(dx, idz), sy = __fmul_rn(dy, idz);
    const float r = __fsqrt_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)));
    c = 1.0f;
    s = 0.0f;
    if (r > 0.0f) {
        const float ir = __frcp_rn(r);
        c = __fmul_rn(x, ir);
        s = __fmul_rn(y, ir);
    }
    const float p = __fadd_rn(__fmul_rn(c, sx), __fmul_rn(s, sy));
    const float qq = __fsub_rn(__fmul_rn(c, sy), __fmul_rn(s, sx));
    m = qq < 0.0f ? -1.0f : 1.0f;
    const float t = __fdiv_rn(1000.0f, lam);
    u[0] = r;
    u[1] = p;
    u[2] = fabsf(qq);
    u[3] = __fmul_rn(t, t);
    return true;
}

// Read-once loads that leave L1 to the coefficient table: the rays' inputs
// stream through once, and the class lookups are random 4-byte reads of an
// L2-resident table that would otherwise each pull a 128-byte line into L1.
__device__ __forceinline__ float ld_stream(const float* p)
{
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p)
{
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t poly_patch_of(const PolyDev& P, int k, uint32_t cell)
{
    return P.m[k] == 1 ? cell : __umulhi(cell, P.mdiv[k]);
}

// Class-grid coordinates g, cell and patch of reduced coordinates u; false
// outside the box.
__device__ __forceinline__ bool poly_cell(const PolyDev& P, const float u[4], float g[4], uint32_t& cid,
                                          uint32_t& pid)
{
    bool inside = true;
    cid = 0;
    pid = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        g[k] = __fmul_rn(__fsub_rn(u[k], P.lo[k]), P.inv[k]);
        inside &= (g[k] >= 0.0f) & (g[k] <= P.cmax[k]);
        int cell = inside ? (int)floorf(g[k]) : 0;
        cell = min(max(cell, 0), P.C[k] - 1);
        cid += (uint32_t)cell * P.cstride[k];
        pid += poly_patch_of(P, k, (uint32_t)cell) * P.pstride[k];
    }
    return inside;
}

// Patch-local xi of class-grid coordinates g in patch pid.
__device__ __forceinline__ void poly_xi(const PolyDev& P, uint32_t pid, const float g[4], float xi[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t pk = (pid / P.pstride[k]) % (uint32_t)P.P[k];
        xi[k] = fmaf(g[k] - (float)(pk * (uint32_t)P.m[k]), P.two_over_m[k], -1.0f);
    }
}

// Cell, patch and patch-local xi; false outside the box.
__device__ __forceinline__ bool poly_locate(const PolyDev& P, const float u[4], uint32_t& cid, uint32_t& pid,
                                            float xi[4])
{
    float g[4];
    const bool inside = poly_cell(P, u, g, cid, pid);
    poly_xi(P, pid, g, xi);
    return inside;
}

__device__ __forceinline__ uint32_t poly_class(const PolyDev& P, uint32_t cid)
{
    return (ld_stream(P.cls + (cid >> 4)) >> ((cid & 15u) * 2u)) & 3u;
}

// Exit ray in the input frame from a patch polynomial's reduced-frame value
// (mirror m, rotation (c, s)).
__device__ __forceinline__ void poly_unreduce(const Acc5& a, float c, float s, float m, float o[6])
{
    const float yp = m * a.p.y, dyp = m * a.d.y;
    const float dz2 = fmaf(-a.d.x, a.d.x, fmaf(-dyp, dyp, 1.0f));
    o[0] = fmaf(c, a.p.x, -s * yp);
    o[1] = fmaf(s, a.p.x, c * yp);
    o[2] = fmaf(c, a.d.x, -s * dyp);
    o[3] = fmaf(s, a.d.x, c * dyp);
    o[4] = dz2 > 0.0f ? sqrtf(dz2) : 0.0f;
    o[5] = a.I;
}

__device__ __forceinline__ const float4* poly_patch_groups(const PolyDev& P, uint32_t pid, int D)
{
    return P.cg + (size_t)pid * poly_groups(D) * 5;
}

template <int D>
__device__ __forceinline__ void poly_output(const PolyDev& P, uint32_t pid, const float xi[4], float c, float s,
                                            float m, float o[6])
{
    const float x1[1][4] = {{xi[0], xi[1], xi[2], xi[3]}};
    Acc5 a;
    poly_eval<D, 1>(poly_patch_groups(P, pid, D), x1, &a);
    poly_unreduce(a, c, s, m, o);
}

// A ray of a query after classification.
struct PolyRay {
    bool ip, tr;                // answered by the polynomial; to be traced (BOUNDARY or outside)
    uint32_t tag;               // ray index (| kOutsideBit)
    float x, y, dx, dy, dz, lam;
    float o[6];
};

template <int D, int MODE>
__device__ __forceinline__ void poly_answer(const PolyDev& P, const RaysInDev& in, uint32_t n, uint32_t r,
                                            PolyRay& c)
{
    c.ip = false;
    c.tr = false;
    c.tag = r;
#pragma unroll
    for (int k = 0; k < 6; ++k) c.o[k] = 0.0f;
    c.x = c.y = c.dx = c.dy = c.dz = c.lam = 0.0f;
    if (r >= n) return;
    c.x = ld_stream(in.x + r);
    c.y = ld_stream(in.y + r);
    c.dx = ld_stream(in.dx + r);
    c.dy = ld_stream(in.dy + r);
    c.dz = ld_stream(in.dz + r);
    c.lam = ld_stream(in.lam + r);
    float u[4], xi[4], cs, sn, m;
    uint32_t cid, pid;
    if (!poly_reduce(c.x, c.y, c.dx, c.dy, c.dz, c.lam, u, cs, sn, m) || !poly_locate(P, u, cid, pid, xi)) {
        c.tr = true;
        c.tag |= kOutsideBit;
        return;
    }
    uint32_t k;
    if (MODE == LT_QUERY_TABLE) k = poly_class(P, cid);
    else k = __ldg(P.patch_ok + pid) ? (uint32_t)LT_CELL_VALID : (uint32_t)LT_CELL_BOUNDARY;
    if (k == LT_CELL_VALID) {
        poly_output<D>(P, pid, xi, cs, sn, m, c.o);
        c.ip = true;
    } else if (k != LT_CELL_INVALID) {
        c.tr = true;
    }
}

__device__ __forceinline__ void poly_store(const RaysOutDev& out, uint32_t r, const float o[6], uint32_t flags)
{
    __stcs(out.x + r, o[0]);
    __stcs(out.y + r, o[1]);
    __stcs(out.dx + r, o[2]);
    __stcs(out.dy + r, o[3]);
    __stcs(out.dz + r, o[4]);
    __stcs(out.I + r, o[5]);
    out.flags[r] = (uint8_t)flags;
}

// ------------------------------------------------------------------ query kernels

// Large batches: every lane answers its ray (polynomial, or "no output" for
// an INVALID cell) and writes its row -- a placeholder for a ray to be
// traced -- and BOUNDARY / outside rays go to the launch's trace queue (one
// atomic per warp on the block's segment counter); map_trace_kernel then
// traces the queue.
template <int D, int MODE>
__global__ void __launch_bounds__(kPolyTile)
poly_query_kernel(const __grid_constant__ PolyDev P, RaysInDev in, RaysOutDev out, uint32_t n, TraceQueue Q)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t r = blockIdx.x * kPolyTile + threadIdx.x;
    PolyRay c;
    poly_answer<D, MODE>(P, in, n, r, c);
    const unsigned mq = __ballot_sync(full, c.tr);
    if (mq) {
        const int leader = __ffs(mq) - 1;
        uint32_t b = 0;
        const uint32_t seg = blockIdx.x % kQSegs;
        if (lane == leader) b = atomicAdd(Q.count + seg * kQCountStride, (uint32_t)__popc(mq));
        b = __shfl_sync(full, b, leader);
        if (c.tr) {
            const uint32_t k = seg * Q.segcap + b + __popc(mq & ((1u << lane) - 1u));
            Q.x[k] = c.x;
            Q.y[k] = c.y;
            Q.dx[k] = c.dx;
            Q.dy[k] = c.dy;
            Q.dz[k] = c.dz;
            Q.lam[k] = c.lam;
            Q.tag[k] = c.tag;
        }
    }
    if (r < n) poly_store(out, r, c.o, c.ip ? LT_FLAG_VALID : 0u);
}

// Large batches, maps of at most kSortMaxPatches patches, run as two
// kernels: classify-and-sort, then evaluate-and-trace.
//
// poly_sort_kernel takes a tile of kSortTile rays per block:
//  A. classifies them (coalesced loads that bypass L1, four rounds of 256
//     consecutive rays, every input of the four in flight at once):
//     BOUNDARY / outside rays go to the trace queue, VALID rays count into
//     a shared-memory histogram over patches (the atomic's return value is
//     the ray's rank within its patch);
//  B. one warp turns the histogram into offsets (exclusive scan);
//  C. every VALID ray writes its record -- class-grid coordinates, rotation
//     (c, s), a word holding its mirror and patch, its index in the tile: 32
//     bytes, one sector -- to its sorted slot of the tile's region, every
//     patch's run padded to even length, and the count goes to the tile's
//     counter; a bit per queued ray goes to the tile's traced mask.
// Round j of tile b appends to queue segment (4 b + j) % kQSegs: the same
// segment a 256-ray block of the same rays would use, so the queue's
// capacity rule (query_segcap) holds.
//
// poly_eval_kernel, a persistent grid launched as a programmatic dependent
// of the sort kernel, copies the coefficient table to shared memory once
// per block (while the sort kernel drains) and then, tile after tile:
// evaluates the tile's records in sorted order (coalesced reads; adjacent
// records mostly share a patch, so a coefficient load is one or two
// shared-memory addresses for the whole warp); stages the tile's rows in
// shared memory (zeros for the INVALID rays); and stores every row but the
// queued rays'.  A block whose tiles are done takes chunks of the trace
// queue from a counter and traces them with the block tracer, writing those
// rows: the queue's tracing overlaps the other blocks' evaluation instead of
// following it as a third kernel.
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 4;
constexpr int kSortTile = kSortThreads * kSortRounds;
constexpr int kSortMaxPatches = 1024;
constexpr uint32_t kNoRay = 0xffffffffu;   // the index of a padding record
static_assert(kSortThreads == kQTile, "a sort round must be one queue block");
static_assert(kSortTile == (int)kSortTileRays, "the sorted-index region is laid out in sort tiles");
constexpr int kEvalThreads = 256;
// largest coefficient table the evaluation kernel keeps in shared memory
constexpr size_t kEvalMaxTableBytes = 96 * 1024;

template <int MODE>
__global__ void __launch_bounds__(kSortThreads)
poly_sort_kernel(const __grid_constant__ PolyDev P, RaysInDev in, uint32_t n, TraceQueue Q, PolyScratch R)
{
    __shared__ uint32_t hist[kSortMaxPatches];
    __shared__ float4 recA[kSortTile];      // class-grid coordinates g
    __shared__ float4 recB[kSortTile];      // c, s, (mirror << 31 | patch), index in the tile
    __shared__ uint32_t nvalid;
    const unsigned full = 0xffffffffu;
    const int t = threadIdx.x, lane = t & 31;
    const int NP = P.n_patches;
    for (int i = t; i < NP; i += kSortThreads) hist[i] = 0;
    __syncthreads();
    const uint32_t r0 = blockIdx.x * kSortTile;
    // A.1: every input of the thread's four rays in flight at once
    float x[kSortRounds], y[kSortRounds], dx[kSortRounds], dy[kSortRounds], dz[kSortRounds], lam[kSortRounds];
#pragma unroll
    for (int j = 0; j < kSortRounds; ++j) {
        const uint32_t r = r0 + (uint32_t)(j * kSortThreads + t);
        x[j] = y[j] = dx[j] = dy[j] = dz[j] = lam[j] = 0.0f;
        if (r < n) {
            x[j] = ld_stream(in.x + r);
            y[j] = ld_stream(in.y + r);
            dx[j] = ld_stream(in.dx + r);
            dy[j] = ld_stream(in.dy + r);
            dz[j] = ld_stream(in.dz + r);
            lam[j] = ld_stream(in.lam + r);
        }
    }
    // A.2: cells and patches; the class words of all four are requested
    // before any is used
    uint32_t cid[kSortRounds], pid[kSortRounds], word[kSortRounds], stat[kSortRounds];   // 0 none, 1 outside, 2 inside
#pragma unroll
    for (int j = 0; j < kSortRounds; ++j) {
        stat[j] = 0;
        cid[j] = pid[j] = 0;
        const uint32_t l = (uint32_t)(j * kSortThreads + t);
        if (r0 + l < n) {
            float u[4], g[4], cs, sn, m;
            stat[j] = 1;
            if (poly_reduce(x[j], y[j], dx[j], dy[j], dz[j], lam[j], u, cs, sn, m) && poly_cell(P, u, g, cid[j], pid[j])) {
                stat[j] = 2;
                recA[l] = make_float4(g[0], g[1], g[2], g[3]);
                recB[l] = make_float4(cs, sn, __uint_as_float((m < 0.0f ? 0x80000000u : 0u) | pid[j]),
                                      __uint_as_float(l));
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kSortRounds; ++j) {
        word[j] = 0;
        if (stat[j] == 2) {
            if (MODE == LT_QUERY_TABLE) word[j] = ld_stream(P.cls + (cid[j] >> 4));
            else word[j] = __ldg(P.patch_ok + pid[j]);
        }
    }
    // A.3: classes and histogram ranks; then the trace queue, whose four
    // appends (one per round, each one atomic per warp) are all issued before
    // any result is used
    uint32_t key[kSortRounds];
    unsigned mq[kSortRounds];
#pragma unroll
    for (int j = 0; j < kSortRounds; ++j) {
        key[j] = 0xffffffffu;
        bool tr = stat[j] == 1;
        if (stat[j] == 2) {
            uint32_t k;
            if (MODE == LT_QUERY_TABLE) k = (word[j] >> ((cid[j] & 15u) * 2u)) & 3u;
            else k = word[j] ? (uint32_t)LT_CELL_VALID : (uint32_t)LT_CELL_BOUNDARY;
            if (k == LT_CELL_VALID) key[j] = (pid[j] << 16) | atomicAdd(&hist[pid[j]], 1u);
            else tr = k != LT_CELL_INVALID;
        }
        mq[j] = __ballot_sync(full, tr);
        // the tile's traced-ray bits: word j * 8 + warp holds rays j * 256 + warp * 32 + lane
        if (lane == 0) R.traced[(size_t)blockIdx.x * (kSortTile / 32) + j * (kSortThreads / 32) + (t >> 5)] = mq[j];
    }
    uint32_t qb[kSortRounds];
#pragma unroll
    for (int j = 0; j < kSortRounds; ++j) {
        qb[j] = 0;
        if (mq[j] && lane == __ffs(mq[j]) - 1)
            qb[j] = atomicAdd(Q.count + ((blockIdx.x * kSortRounds + j) % kQSegs) * kQCountStride,
                              (uint32_t)__popc(mq[j]));
    }
#pragma unroll
    for (int j = 0; j < kSortRounds; ++j) {
        if (!mq[j]) continue;
        const uint32_t b = __shfl_sync(full, qb[j], __ffs(mq[j]) - 1);
        if ((mq[j] >> lane) & 1u) {
            const uint32_t seg = (blockIdx.x * kSortRounds + j) % kQSegs;
            const uint32_t k = seg * Q.segcap + b + __popc(mq[j] & ((1u << lane) - 1u));
            const uint32_t r = r0 + (uint32_t)(j * kSortThreads + t);
            Q.x[k] = x[j];
            Q.y[k] = y[j];
            Q.dx[k] = dx[j];
            Q.dy[k] = dy[j];
            Q.dz[k] = dz[j];
            Q.lam[k] = lam[j];
            Q.tag[k] = r | (stat[j] == 1 ? kOutsideBit : 0u);
        }
    }
    __syncthreads();
    // B
    if (t < 32) {
        const int per = (NP + 31) / 32;
        const int b0 = min(NP, lane * per), b1 = min(NP, b0 + per);
        uint32_t sum = 0;
        for (int b = b0; b < b1; ++b) sum += (hist[b] + 1u) & ~1u;
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(full, incl, o);
            if (lane >= o) incl += v;
        }
        uint32_t run = incl - sum;
        float4* rec = R.rec + (size_t)blockIdx.x * R.stride * 2;
        for (int b = b0; b < b1; ++b) {
            const uint32_t c = hist[b];
            hist[b] = run;
            // an odd run ends in a padding record (index kNoRay: evaluated, not stored)
            if (c & 1u) {
                rec[(run + c) * 2] = make_float4(0.f, 0.f, 0.f, 0.f);
                rec[(run + c) * 2 + 1] = make_float4(0.f, 0.f, __uint_as_float((uint32_t)b), __uint_as_float(kNoRay));
            }
            run += (c + 1u) & ~1u;
        }
        if (lane == 31) nvalid = run;
    }
    __syncthreads();
    // C
    float4* rec = R.rec + (size_t)blockIdx.x * R.stride * 2;
    if (t == 0) R.tile_nv[blockIdx.x] = nvalid;
#pragma unroll
    for (int j = 0; j < kSortRounds; ++j)
        if (key[j] != 0xffffffffu) {
            const uint32_t l = (uint32_t)(j * kSortThreads + t);
            const uint32_t slot = hist[key[j] >> 16] + (key[j] & 0xffffu);
            rec[slot * 2] = recA[l];
            rec[slot * 2 + 1] = recB[l];
        }
}

// The shared memory of poly_eval_kernel's two phases: a tile's staged rows
// while it evaluates, the block tracer's states once it traces.
union EvalSmem {
    struct {
        float ob[6][kSortTile];
        uint8_t of[kSortTile];
    } e;
    TraceSmem<kEvalThreads> t;
};

template <int D, bool CAUCHY>
__global__ void __launch_bounds__(kEvalThreads)
poly_eval_kernel(const __grid_constant__ PolyDev P, const __grid_constant__ MapDev M, RaysOutDev out, uint32_t n,
                 PolyScratch R, uint32_t ntiles, TraceQueue Q, unsigned long long* work)
{
    extern __shared__ float4 smc[];                 // the coefficient table
    __shared__ EvalSmem U;
    __shared__ uint32_t tmask[kSortTile / 32];      // the tile's traced rays
    __shared__ uint32_t cnt[kQSegs], cum[kQSegs + 1];
    __shared__ uint32_t chunk, cseg;
    const int t = threadIdx.x;
    const int ntab = P.n_patches * poly_groups(D) * 5;
    for (int i = t; i < ntab; i += kEvalThreads) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(smc + i);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(P.cg + i));
    }
    asm volatile("cp.async.commit_group;");
    // the sort kernel's records and queue are read only after it has completed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    // phase 1: the tiles of this block
#pragma unroll 1
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t r0 = tile * kSortTile;
        const uint32_t cnt_t = min((uint32_t)kSortTile, n - r0);
        for (uint32_t l = (uint32_t)t; l < (uint32_t)kSortTile; l += kEvalThreads) {
#pragma unroll
            for (int q = 0; q < 6; ++q) U.e.ob[q][l] = 0.0f;
            U.e.of[l] = 0;
        }
        if (t < kSortTile / 32) tmask[t] = R.traced[(size_t)tile * (kSortTile / 32) + t];
        __syncthreads();
        const uint32_t nv = R.tile_nv[tile];
        const float4* rec = R.rec + (size_t)tile * R.stride * 2;
#pragma unroll 1
        for (uint32_t s0 = 2u * (uint32_t)t; s0 < nv; s0 += 2u * kEvalThreads) {
            const float4 a0 = rec[s0 * 2], b0 = rec[s0 * 2 + 1], a1 = rec[s0 * 2 + 2], b1 = rec[s0 * 2 + 3];
            const uint32_t w0 = __float_as_uint(b0.z), w1 = __float_as_uint(b1.z);
            const uint32_t pid = w0 & 0x7fffffffu;
            const float g0[4] = {a0.x, a0.y, a0.z, a0.w}, g1[4] = {a1.x, a1.y, a1.z, a1.w};
            float xi[2][4];
            poly_xi(P, pid, g0, xi[0]);
            poly_xi(P, pid, g1, xi[1]);
            Acc5 acc[2];
            poly_eval_tab<D, 2>(smc + (size_t)pid * poly_groups(D) * 5, xi, acc);
            float o[6];
            uint32_t l = __float_as_uint(b0.w);
            poly_unreduce(acc[0], b0.x, b0.y, (w0 & 0x80000000u) ? -1.0f : 1.0f, o);
#pragma unroll
            for (int q = 0; q < 6; ++q) U.e.ob[q][l] = o[q];
            U.e.of[l] = LT_FLAG_VALID;
            l = __float_as_uint(b1.w);
            if (l != kNoRay) {
                poly_unreduce(acc[1], b1.x, b1.y, (w1 & 0x80000000u) ? -1.0f : 1.0f, o);
#pragma unroll
                for (int q = 0; q < 6; ++q) U.e.ob[q][l] = o[q];
                U.e.of[l] = LT_FLAG_VALID;
            }
        }
        __syncthreads();
        // every row but the queued rays', which the tracer writes
        for (uint32_t l = (uint32_t)t; l < cnt_t; l += kEvalThreads) {
            if ((tmask[l >> 5] >> (l & 31u)) & 1u) continue;
            const uint32_t r = r0 + l;
            __stcs(out.x + r, U.e.ob[0][l]);
            __stcs(out.y + r, U.e.ob[1][l]);
            __stcs(out.dx + r, U.e.ob[2][l]);
            __stcs(out.dy + r, U.e.ob[3][l]);
            __stcs(out.dz + r, U.e.ob[4][l]);
            __stcs(out.I + r, U.e.ob[5][l]);
            out.flags[r] = U.e.of[l];
        }
        __syncthreads();
    }
    // phase 2: the trace queue, kEvalThreads-ray chunks of its segments taken
    // from a counter until none is left (chunk c: segment s with cum[s] <= c <
    // cum[s + 1]), started by each block when its tiles are done
    if (t < kQSegs) cnt[t] = Q.count[t * kQCountStride];
    __syncthreads();
    if (t == 0) {
        uint32_t c = 0;
        for (int sg = 0; sg < kQSegs; ++sg) {
            cum[sg] = c;
            c += (cnt[sg] + kEvalThreads - 1) / kEvalThreads;
        }
        cum[kQSegs] = c;
    }
    __syncthreads();
    const uint32_t nchunks = cum[kQSegs];
    TraceSmem<kEvalThreads>& S = U.t;
    int nint = 0;
#pragma unroll 1
    while (true) {
        if (t == 0) {
            const uint32_t c = atomicAdd(Q.count + kQSegs * kQCountStride, 1u);
            int sg = 0;
            while (sg < kQSegs - 1 && cum[sg + 1] <= c) ++sg;
            chunk = c;
            cseg = (uint32_t)sg;
        }
        __syncthreads();
        if (chunk >= nchunks) break;
        const uint32_t sg = cseg;
        const uint32_t i = (chunk - cum[sg]) * (uint32_t)kEvalThreads + (uint32_t)t;   // entry within the segment
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
        nint += trace_block_states<CAUCHY, kEvalThreads>(M.L, M.pi, M.pj, live, st, S);
        __syncthreads();
        if (have) {
            const uint32_t r = e & ~kOutsideBit;
            const float o[6] = {S.ob[0][t], S.ob[1][t], S.ob[2][t], S.ob[3][t], S.ob[4][t], S.ob[5][t]};
            poly_store(out, r, o, S.of[t] | LT_FLAG_TRACED | ((e & kOutsideBit) ? LT_FLAG_OUTSIDE : 0u));
        }
        __syncthreads();
    }
    warp_add(work, (unsigned)nint);
}

// Small batches: the whole query in one kernel; each block traces its own
// BOUNDARY and outside rays with survivor compaction (trace_block_states).
// The body is a device function of the block index within the batch, shared
// with the server's fused launch (serve_poly_kernel).
template <int D, int MODE, bool CAUCHY>
__device__ __forceinline__ void poly_fused_block(const MapDev& M, const PolyDev& P, const RaysInDev& in,
                                                 const RaysOutDev& out, uint32_t n, uint32_t blk,
                                                 unsigned long long* work)
{
    __shared__ TraceSmem<kPolyTile> S;
    __shared__ uint32_t tlist[kPolyTile];
    __shared__ uint32_t tcount;
    const unsigned full = 0xffffffffu;
    const int t = threadIdx.x, lane = t & 31;
    if (t == 0) tcount = 0;
    __syncthreads();
    const uint32_t r0 = blk * kPolyTile;
    const uint32_t r = r0 + t;
    PolyRay c;
    poly_answer<D, MODE>(P, in, n, r, c);
    const unsigned mq = __ballot_sync(full, c.tr);
    if (mq) {
        const int leader = __ffs(mq) - 1;
        uint32_t b = 0;
        if (lane == leader) b = atomicAdd(&tcount, (uint32_t)__popc(mq));
        b = __shfl_sync(full, b, leader);
        if (c.tr) tlist[b + __popc(mq & ((1u << lane) - 1u))] = (uint32_t)t | (c.tag & kOutsideBit);
    }
    if (r < n && !c.tr) poly_store(out, r, c.o, c.ip ? LT_FLAG_VALID : 0u);
    __syncthreads();
    const uint32_t nt = tcount;
    if (nt == 0) return;
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
    const int nint = trace_block_states<CAUCHY, kPolyTile>(M.L, M.pi, M.pj, live, st, S);
    __syncthreads();
    if ((uint32_t)t < nt) {
        const uint32_t rr = r0 + (e & ~kOutsideBit);
        const float o[6] = {S.ob[0][t], S.ob[1][t], S.ob[2][t], S.ob[3][t], S.ob[4][t], S.ob[5][t]};
        poly_store(out, rr, o, S.of[t] | LT_FLAG_TRACED | ((e & kOutsideBit) ? LT_FLAG_OUTSIDE : 0u));
    }
    warp_add(work, (unsigned)nint);
}

template <int D, int MODE, bool CAUCHY>
__global__ void __launch_bounds__(kPolyTile)
poly_query_fused_kernel(const __grid_constant__ MapDev M, const __grid_constant__ PolyDev P, RaysInDev in,
                        RaysOutDev out, uint32_t n, unsigned long long* work)
{
    poly_fused_block<D, MODE, CAUCHY>(M, P, in, out, n, blockIdx.x, work);
}

// The server's fused launch of several small polynomial-patch map queries
// (each block serves one request; every request's map has the same degree,
// MODE and dispersion form): the block stages its request's constants (a
// device copy of the map's MapDev and PolyDev) in shared memory and runs the
// one-kernel query on its rays.
struct PolyServe {
    MapDev M;
    PolyDev P;
};
static_assert(sizeof(PolyServe) % 16 == 0, "PolyServe is staged in 16-byte words");
static_assert(kPolyTile == (int)kFusedQueryRays, "the server lays out fused blocks of kFusedQueryRays");

template <int D, int MODE, bool CAUCHY>
__global__ void __launch_bounds__(kPolyTile)
serve_poly_kernel(const __grid_constant__ ReqTable T, unsigned long long* work)
{
    __shared__ PolyServe sm;
    const int k = req_of_block(T, blockIdx.x);
    const ReqItem& it = T.item[k];
    stage_words(&sm, it.dev, sizeof(PolyServe));
    __syncthreads();
    poly_fused_block<D, MODE, CAUCHY>(sm.M, sm.P, it.in, it.out, it.n, blockIdx.x - T.block0[k], work);
}

// ------------------------------------------------------------------ build kernels

// Box and patch geometry for the build kernels (FP64 where the fit needs it).
struct PolyBuild {
    double lo[4], h[4];                  // box corner, patch sides
    double cheb[kMaxSamplesAxis];        // Chebyshev nodes cos(pi (k + 1/2) / ns)
    int P[4], ns, M, T;
    uint32_t pstride[4];
};

// One thread per (patch, sample): the sample's reduced ray (FP64, rounded
// once to FP32) traced through the unclipped lens; y = (x', y', d_x', d_y', I).
template <bool CAUCHY>
__global__ void __launch_bounds__(256)
poly_sample_kernel(const __grid_constant__ LensDev Lu, int pi, int pj, const __grid_constant__ PolyBuild B,
                   float* __restrict__ y, uint8_t* __restrict__ v, uint32_t total)
{
    const uint32_t l = blockIdx.x * 256u + threadIdx.x;
    if (l >= total) return;
    const uint32_t pid = l / (uint32_t)B.M, s = l % (uint32_t)B.M;
    double u[4];
    uint32_t sr = s;
#pragma unroll
    for (int k = 3; k >= 0; --k) {
        const int j = (int)(sr % (uint32_t)B.ns);
        sr /= (uint32_t)B.ns;
        const int pk = (int)((pid / B.pstride[k]) % (uint32_t)B.P[k]);
        u[k] = __dadd_rn(B.lo[k], __dmul_rn(__dadd_rn((double)pk, __dmul_rn(0.5, __dadd_rn(B.cheb[j], 1.0))), B.h[k]));
    }
    // uncontracted FP64 (each operation rounded once), then one rounding to FP32
    const double inv = 1.0 / sqrt(__dadd_rn(__dadd_rn(__dmul_rn(u[1], u[1]), __dmul_rn(u[2], u[2])), 1.0));
    TraceOut o;
    int nint;
    const uint32_t f = trace_ray<CAUCHY>(Lu, pi, pj, (float)u[0], 0.0f, (float)__dmul_rn(u[1], inv),
                                         (float)__dmul_rn(u[2], inv), (float)inv, (float)(1000.0 / sqrt(u[3])), o,
                                         nint);
    y[(size_t)l * 5 + 0] = o.x;
    y[(size_t)l * 5 + 1] = o.y;
    y[(size_t)l * 5 + 2] = o.dx;
    y[(size_t)l * 5 + 3] = o.dy;
    y[(size_t)l * 5 + 4] = o.I;
    v[l] = (uint8_t)(f & LT_FLAG_VALID);
}

// Normal equations of every patch (FP64 reductions over its valid samples):
// entry e < T(T+1)/2 is G[i][j] = sum a_i a_j (pairs from `ij`), the next 5T
// are R[i][o] = sum a_i y_o.  Grid (patches, entry blocks).
__global__ void __launch_bounds__(256)
poly_normal_kernel(const __grid_constant__ PolyBuild B, const double* __restrict__ A,
                   const uint16_t* __restrict__ ij, const float* __restrict__ y, const uint8_t* __restrict__ v,
                   double* __restrict__ G, double* __restrict__ R)
{
    const int T = B.T, M = B.M;
    const int NG = T * (T + 1) / 2;
    const int e = blockIdx.y * 256 + threadIdx.x;
    if (e >= NG + 5 * T) return;
    const uint32_t pid = blockIdx.x;
    const uint8_t* vp = v + (size_t)pid * M;
    const float* yp = y + (size_t)pid * M * 5;
    double acc = 0.0;
    if (e < NG) {
        const int i = ij[2 * e], j = ij[2 * e + 1];
        for (int s = 0; s < M; ++s)
            if (vp[s]) acc = fma(A[(size_t)s * T + i], A[(size_t)s * T + j], acc);
        G[(size_t)pid * T * T + (size_t)i * T + j] = acc;
        G[(size_t)pid * T * T + (size_t)j * T + i] = acc;
    } else {
        const int i = (e - NG) / 5, o = (e - NG) % 5;
        for (int s = 0; s < M; ++s)
            if (vp[s]) acc = fma(A[(size_t)s * T + i], (double)yp[(size_t)s * 5 + o], acc);
        R[(size_t)pid * T * 5 + (size_t)i * 5 + o] = acc;
    }
}

// One thread per patch: Cholesky factorisation of G (in place, lower
// triangle) and the two triangular solves for the 5 right-hand sides.  A
// patch with fewer valid samples than terms, or a pivot below 1e-13 of the
// largest diagonal entry, gets no fit.
__global__ void __launch_bounds__(64)
poly_solve_kernel(const __grid_constant__ PolyBuild B, const uint8_t* __restrict__ v, double* __restrict__ G,
                  const double* __restrict__ R, double* __restrict__ coef, uint8_t* __restrict__ ok, int npatch)
{
    const int pid = blockIdx.x * 64 + threadIdx.x;
    if (pid >= npatch) return;
    const int T = B.T, M = B.M;
    int nv = 0;
    for (int s = 0; s < M; ++s) nv += v[(size_t)pid * M + s];
    double* g = G + (size_t)pid * T * T;
    double* c = coef + (size_t)pid * T * 5;
    for (int q = 0; q < T * 5; ++q) c[q] = 0.0;
    ok[pid] = 0;
    if (nv < T) return;
    double dmax = 0.0;
    for (int j = 0; j < T; ++j) dmax = fmax(dmax, g[(size_t)j * T + j]);
    for (int j = 0; j < T; ++j) {
        double d = g[(size_t)j * T + j];
        for (int k = 0; k < j; ++k) d -= g[(size_t)j * T + k] * g[(size_t)j * T + k];
        if (!(d > 1e-13 * dmax)) return;
        const double ljj = sqrt(d);
        g[(size_t)j * T + j] = ljj;
        for (int i = j + 1; i < T; ++i) {
            double a = g[(size_t)i * T + j];
            for (int k = 0; k < j; ++k) a -= g[(size_t)i * T + k] * g[(size_t)j * T + k];
            g[(size_t)i * T + j] = a / ljj;
        }
    }
    const double* r = R + (size_t)pid * T * 5;
    for (int o = 0; o < 5; ++o) {
        // L z = r (z in c), then L^T x = z
        for (int i = 0; i < T; ++i) {
            double a = r[(size_t)i * 5 + o];
            for (int k = 0; k < i; ++k) a -= g[(size_t)i * T + k] * c[(size_t)k * 5 + o];
            c[(size_t)i * 5 + o] = a / g[(size_t)i * T + i];
        }
        for (int i = T - 1; i >= 0; --i) {
            double a = c[(size_t)i * 5 + o];
            for (int k = i + 1; k < T; ++k) a -= g[(size_t)k * T + i] * c[(size_t)k * 5 + o];
            c[(size_t)i * 5 + o] = a / g[(size_t)i * T + i];
        }
    }
    ok[pid] = 1;
}

// Largest |fit - traced| exit position over the valid samples of fitted
// patches (FP64; the maximum as ordered bits of a non-negative double), and
// the FP32 query table packed from the FP64 coefficients.
__global__ void __launch_bounds__(256)
poly_sample_residual_kernel(const __grid_constant__ PolyBuild B, const double* __restrict__ A,
                            const float* __restrict__ y, const uint8_t* __restrict__ v,
                            const double* __restrict__ coef, const uint8_t* __restrict__ ok,
                            unsigned long long* resmax, uint32_t total)
{
    const uint32_t l = blockIdx.x * 256u + threadIdx.x;
    double res = 0.0;
    if (l < total) {
        const uint32_t pid = l / (uint32_t)B.M, s = l % (uint32_t)B.M;
        if (v[l] && ok[pid]) {
            const double* c = coef + (size_t)pid * B.T * 5;
            double px = 0.0, py = 0.0;
            for (int k = 0; k < B.T; ++k) {
                const double a = A[(size_t)s * B.T + k];
                px = fma(a, c[(size_t)k * 5 + 0], px);
                py = fma(a, c[(size_t)k * 5 + 1], py);
            }
            res = hypot(px - (double)y[(size_t)l * 5 + 0], py - (double)y[(size_t)l * 5 + 1]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) res = fmax(res, __shfl_xor_sync(0xffffffffu, res, o));
    if ((threadIdx.x & 31) == 0 && res > 0.0) atomicMax(resmax, (unsigned long long)__double_as_longlong(res));
}

// The FP32 query table from the FP64 fit: one thread per (patch, group,
// output) float4.
__global__ void __launch_bounds__(256)
poly_pack_kernel(const double* __restrict__ coef, float4* __restrict__ cg, int T, int NG, uint32_t total)
{
    const uint32_t l = blockIdx.x * 256u + threadIdx.x;
    if (l >= total) return;
    const uint32_t o = l % 5, g = (l / 5) % (uint32_t)NG, pid = l / (5u * (uint32_t)NG);
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int k = (int)g * 4 + j;
        v[j] = k < T ? (float)coef[((size_t)pid * T + k) * 5 + o] : 0.0f;
    }
    cg[l] = make_float4(v[0], v[1], v[2], v[3]);
}

// One thread per class-grid node: its FP32 entrance ray (the rule in lt.h)
// traced through the real lens; the reduced-frame exit (x', y') kept for the
// corner residuals.
template <bool CAUCHY>
__global__ void __launch_bounds__(256)
poly_node_kernel(const __grid_constant__ LensDev L, int pi, int pj, const __grid_constant__ PolyDev P,
                 const float4 step, float2* __restrict__ nout, uint8_t* __restrict__ nvalid, uint32_t N)
{
    const uint32_t l = blockIdx.x * 256u + threadIdx.x;
    if (l >= N) return;
    const float stp[4] = {step.x, step.y, step.z, step.w};
    float v[4];
    uint32_t t = l;
#pragma unroll
    for (int k = 3; k >= 0; --k) {
        const uint32_t nk = (uint32_t)P.C[k] + 1u;
        const uint32_t i = t % nk;
        t /= nk;
        v[k] = __fadd_rn(P.lo[k], __fmul_rn((float)i, stp[k]));
    }
    const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(v[1], v[1]), __fmul_rn(v[2], v[2])), 1.0f);
    const float len = __fsqrt_rn(n2);
    TraceOut o;
    int nint;
    const uint32_t f = trace_ray<CAUCHY>(L, pi, pj, v[0], 0.0f, __fdiv_rn(v[1], len), __fdiv_rn(v[2], len),
                                         __fdiv_rn(1.0f, len), __fdiv_rn(1000.0f, __fsqrt_rn(v[3])), o, nint);
    nout[l] = make_float2(o.x, o.y);
    nvalid[l] = (uint8_t)(f & LT_FLAG_VALID);
}

// One thread per class-grid cell: corner bits for the classification (bit0:
// all 16 corners valid, the patch fitted and every corner's exit within tol
// of the FP32 polynomial; bit1: all 16 invalid), the largest corner residual.
template <int D>
__global__ void __launch_bounds__(256)
poly_cell_kernel(const __grid_constant__ PolyDev P, const float2* __restrict__ nout,
                 const uint8_t* __restrict__ nvalid, float tol, uint8_t* __restrict__ corner_bits,
                 unsigned int* __restrict__ resmax_all, uint32_t NC)
{
    const uint32_t cid = blockIdx.x * 256u + threadIdx.x;
    float worst = 0.0f;
    if (cid < NC) {
        int cell[4];
        uint32_t t = cid, nstride[4], s = 1;
#pragma unroll
        for (int k = 3; k >= 0; --k) {
            cell[k] = (int)(t % (uint32_t)P.C[k]);
            t /= (uint32_t)P.C[k];
            nstride[k] = s;
            s *= (uint32_t)P.C[k] + 1u;
        }
        uint32_t base = 0, pid = 0, pk[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            base += (uint32_t)cell[k] * nstride[k];
            pk[k] = poly_patch_of(P, k, (uint32_t)cell[k]);
            pid += pk[k] * P.pstride[k];
        }
        int nv = 0;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const uint32_t off = base + ((q >> 3) & 1) * nstride[0] + ((q >> 2) & 1) * nstride[1] +
                                 ((q >> 1) & 1) * nstride[2] + (q & 1) * nstride[3];
            nv += __ldg(nvalid + off);
        }
        uint32_t bits = nv == 0 ? 2u : 0u;
        if (nv == 16 && __ldg(P.patch_ok + pid)) {
#pragma unroll 1
            for (int q = 0; q < 16; ++q) {
                const int b[4] = {(q >> 3) & 1, (q >> 2) & 1, (q >> 1) & 1, q & 1};
                float xi[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    xi[k] = fmaf((float)((uint32_t)(cell[k] + b[k]) - pk[k] * (uint32_t)P.m[k]), P.two_over_m[k], -1.0f);
                const float x1[1][4] = {{xi[0], xi[1], xi[2], xi[3]}};
                Acc5 a;
                poly_eval<D, 1>(poly_patch_groups(P, pid, D), x1, &a);
                const uint32_t off = base + b[0] * nstride[0] + b[1] * nstride[1] + b[2] * nstride[2] + b[3] * nstride[3];
                const float2 tr = nout[off];
                worst = fmaxf(worst, hypotf(a.p.x - tr.x, a.p.y - tr.y));
            }
            if (!(tol > 0.0f) || worst <= tol) bits |= 1u;
        }
        corner_bits[cid] = (uint8_t)bits;
    }
    unsigned int wb = __float_as_uint(worst);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wb = max(wb, __shfl_xor_sync(0xffffffffu, wb, o));
    if ((threadIdx.x & 31) == 0 && wb) atomicMax(resmax_all, wb);
}

struct PolyFitAccum {
    unsigned long long inside, valid, n_res;
    double sumsq;
    unsigned int max_res_bits;
};

// One thread per fit ray: traced through the real lens; marks its cell as
// having seen a valid / invalid ray and, for a valid ray in a cell whose
// corners qualified, reduces |polynomial - traced| exit position (the
// polynomial as the query evaluates it).
template <int D, bool CAUCHY>
__global__ void __launch_bounds__(256)
poly_fit_kernel(const __grid_constant__ LensDev L, int pi, int pj, const __grid_constant__ PolyDev P,
                RaysInDev fit, uint32_t nfit, const uint8_t* __restrict__ corner_bits, uint32_t* __restrict__ seen,
                uint32_t* __restrict__ resmax, PolyFitAccum* acc)
{
    const uint32_t r = blockIdx.x * 256u + threadIdx.x;
    bool inside = false, valid = false, has_res = false;
    float res = 0.0f;
    if (r < nfit) {
        const float x = __ldg(fit.x + r), y = __ldg(fit.y + r), dx = __ldg(fit.dx + r), dy = __ldg(fit.dy + r),
                    dz = __ldg(fit.dz + r), lam = __ldg(fit.lam + r);
        float u[4], xi[4], cs, sn, m;
        uint32_t cid, pid;
        inside = poly_reduce(x, y, dx, dy, dz, lam, u, cs, sn, m) && poly_locate(P, u, cid, pid, xi);
        if (inside) {
            TraceOut o;
            int nint;
            valid = (trace_ray<CAUCHY>(L, pi, pj, x, y, dx, dy, dz, lam, o, nint) & LT_FLAG_VALID) != 0;
            atomicOr(seen + (cid >> 4), (valid ? 1u : 2u) << ((cid & 15u) * 2u));
            if (valid && (__ldg(corner_bits + cid) & 1u)) {
                float q[6];
                poly_output<D>(P, pid, xi, cs, sn, m, q);
                res = hypotf(q[0] - o.x, q[1] - o.y);
                has_res = true;
                if (resmax) atomicMax(resmax + cid, __float_as_uint(res));
            }
        }
    }
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

// ------------------------------------------------------------------ launches

#define LT_POLY_DISPATCH(D, ...)                                                     \
    switch (D) {                                                                     \
    case 1: { constexpr int DD = 1; __VA_ARGS__; } break;                            \
    case 2: { constexpr int DD = 2; __VA_ARGS__; } break;                            \
    case 3: { constexpr int DD = 3; __VA_ARGS__; } break;                            \
    case 4: { constexpr int DD = 4; __VA_ARGS__; } break;                            \
    default: { constexpr int DD = 5; __VA_ARGS__; } break;                           \
    }

PolyScratch poly_scratch_at(void* scratch, size_t n, size_t patches)
{
    char* p = static_cast<char*>(scratch) + query_scratch_bytes(n);
    PolyScratch R;
    R.stride = (uint32_t)(kSortTileRays + patches);
    R.rec = reinterpret_cast<float4*>(p);
    R.tile_nv = reinterpret_cast<uint32_t*>(p + query_tiles(n) * R.stride * 32);
    R.traced = R.tile_nv + query_tiles(n);
    return R;
}

lt_status launch_poly_fused(const lt_map* map, const RaysInDev& in, const RaysOutDev& out, uint32_t n, int mode,
                            cudaStream_t st)
{
    for (uint32_t a = 0; a < n; a += kFusedMaxRays) {
        const uint32_t k = std::min(kFusedMaxRays, n - a);
        const RaysInDev ia{in.x + a, in.y + a, in.dx + a, in.dy + a, in.dz + a, in.lam + a};
        const RaysOutDev oa{out.x + a, out.y + a, out.dx + a, out.dy + a, out.dz + a, out.I + a, out.flags + a};
        const lt_status s = launch_poly_query(map, ia, oa, k, mode, st);
        if (s != LT_OK) return s;
    }
    return LT_OK;
}

lt_status serve_blob(const lt_map* m, std::vector<unsigned char>& b)
{
    if (m->kind == LT_MAP_KIND_POLY) {
        PolyServe X{};
        X.M = m->dev;
        X.P = m->pdev;
        b.assign(reinterpret_cast<const unsigned char*>(&X), reinterpret_cast<const unsigned char*>(&X) + sizeof X);
    } else {
        b.assign(reinterpret_cast<const unsigned char*>(&m->dev),
                 reinterpret_cast<const unsigned char*>(&m->dev) + sizeof(MapDev));
    }
    return LT_OK;
}

// The server fuses LT_QUERY_TABLE requests only (LT_QUERY_NO_MASK ones run
// alone), which keeps the fused kernel to one instantiation per degree and
// dispersion form.
lt_status launch_fused_poly(const ReqTable& T, int degree, int mode, bool cauchy, cudaStream_t st)
{
    if (T.n_items < 1 || T.n_items > kMaxFuse) return fail(LT_EINVAL, "fused query: %d requests", T.n_items);
    if (mode != LT_QUERY_TABLE) return fail(LT_EINVAL, "fused polynomial query: mode %d not fused", mode);
    const unsigned blocks = T.block0[T.n_items];
    ProfScope prof("serve_poly_kernel", st);
    unsigned long long* w = prof.work();
    LT_POLY_DISPATCH(degree, {
        if (cauchy) serve_poly_kernel<DD, LT_QUERY_TABLE, true><<<blocks, kPolyTile, 0, st>>>(T, w);
        else serve_poly_kernel<DD, LT_QUERY_TABLE, false><<<blocks, kPolyTile, 0, st>>>(T, w);
    });
    LT_CUDA_TRY(cudaGetLastError());
    return LT_OK;
}

lt_status launch_poly_query(const lt_map* map, const RaysInDev& in, const RaysOutDev& out, uint32_t n,
                            int mode, cudaStream_t st)
{
    const bool table = mode == LT_QUERY_TABLE;
    const unsigned blocks = (n + kPolyTile - 1) / kPolyTile;
    const int D = map->pdev.degree;
    if (n <= kFusedMaxRays) {
        ProfScope prof("poly_query_fused_kernel", st);
        unsigned long long* w = prof.work();
        const bool ca = map->cauchy;
        LT_POLY_DISPATCH(D, {
            if (table) {
                if (ca) poly_query_fused_kernel<DD, LT_QUERY_TABLE, true><<<blocks, kPolyTile, 0, st>>>(map->dev, map->pdev, in, out, n, w);
                else poly_query_fused_kernel<DD, LT_QUERY_TABLE, false><<<blocks, kPolyTile, 0, st>>>(map->dev, map->pdev, in, out, n, w);
            } else {
                if (ca) poly_query_fused_kernel<DD, LT_QUERY_NO_MASK, true><<<blocks, kPolyTile, 0, st>>>(map->dev, map->pdev, in, out, n, w);
                else poly_query_fused_kernel<DD, LT_QUERY_NO_MASK, false><<<blocks, kPolyTile, 0, st>>>(map->dev, map->pdev, in, out, n, w);
            }
        });
        LT_CUDA_TRY(cudaGetLastError());
        return LT_OK;
    }
    cudaMemPool_t pool;
    lt_status s = scratch_pool(&pool);
    if (s != LT_OK) return s;
    const size_t bytes = poly_scratch_bytes(n, map->pdev.n_patches);
    char* buf = nullptr;
    if (cudaMallocFromPoolAsync((void**)&buf, bytes, pool, st) != cudaSuccess)
        return fail(LT_ENOMEM, "lt_query: scratch allocation of %zu bytes failed", bytes);
    const TraceQueue Q = trace_queue_at(buf, n);
    const PolyScratch R = poly_scratch_at(buf, n, map->pdev.n_patches);
    do {
        cudaError_t e = cudaMemsetAsync(Q.count, 0, kQHeaderBytes, st);
        if (e != cudaSuccess) { s = cuda_fail(e, "lt_query: clearing the queue"); break; }
        const size_t tab = (size_t)map->pdev.n_patches * poly_groups(D) * 5 * sizeof(float4);
        if (map->pdev.n_patches <= kSortMaxPatches && tab <= kEvalMaxTableBytes) {
            const unsigned sb = (n + kSortTile - 1) / kSortTile;
            {
                ProfScope prof("poly_sort_kernel", st);
                if (table) poly_sort_kernel<LT_QUERY_TABLE><<<sb, kSortThreads, 0, st>>>(map->pdev, in, n, Q, R);
                else poly_sort_kernel<LT_QUERY_NO_MASK><<<sb, kSortThreads, 0, st>>>(map->pdev, in, n, Q, R);
                e = cudaGetLastError();
                if (e != cudaSuccess) { s = cuda_fail(e, "lt_query: launch"); break; }
            }
            ProfScope prof("poly_eval_kernel", st);
            cudaLaunchConfig_t cfg = {};
            cfg.blockDim = dim3(kEvalThreads);
            cfg.dynamicSmemBytes = tab;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            unsigned long long* w = prof.work();
            const bool ca = map->cauchy;
            LT_POLY_DISPATCH(D, {
                const void* kf = ca ? (const void*)poly_eval_kernel<DD, true> : (const void*)poly_eval_kernel<DD, false>;
                e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab);
                if (e == cudaSuccess) {
                    int per_sm = 0, sms = 0, dev = 0;
                    cudaGetDevice(&dev);
                    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, kEvalThreads, tab);
                    cfg.gridDim = dim3(std::max(1u, std::min(sb, (unsigned)(std::max(per_sm, 1) * sms))));
                    if (ca) e = cudaLaunchKernelEx(&cfg, poly_eval_kernel<DD, true>, map->pdev, map->dev, out, n, R, sb, Q, w);
                    else e = cudaLaunchKernelEx(&cfg, poly_eval_kernel<DD, false>, map->pdev, map->dev, out, n, R, sb, Q, w);
                }
            });
            if (e != cudaSuccess) { s = cuda_fail(e, "lt_query: launch"); break; }
            // the evaluation kernel also traced the queue
            break;
        } else {
            ProfScope prof("poly_query_kernel", st);
            LT_POLY_DISPATCH(D, {
                if (table) poly_query_kernel<DD, LT_QUERY_TABLE><<<blocks, kPolyTile, 0, st>>>(map->pdev, in, out, n, Q);
                else poly_query_kernel<DD, LT_QUERY_NO_MASK><<<blocks, kPolyTile, 0, st>>>(map->pdev, in, out, n, Q);
            });
            e = cudaGetLastError();
            if (e != cudaSuccess) { s = cuda_fail(e, "lt_query: launch"); break; }
        }
        s = launch_queue_trace(map, out, n, Q, st);
    } while (0);
    if (buf) cudaFreeAsync(buf, st);
    return s;
}

}  // namespace lt

using namespace lt;

namespace {

lt_status poly_check_opts(const lt_lens* lens, const lt_poly_opts* o, int* pi, int* pj)
{
    if (!path_ij(lens->S, o->path_id, pi, pj)) return fail(LT_EINVAL, "lt_build_poly_map: bad path id %d", o->path_id);
    if (o->degree < 1 || o->degree > LT_POLY_MAX_DEGREE)
        return fail(LT_EINVAL, "lt_build_poly_map: degree %d outside 1..%d", o->degree, LT_POLY_MAX_DEGREE);
    if (o->samples < o->degree + 1 || o->samples > kMaxSamplesAxis)
        return fail(LT_EINVAL, "lt_build_poly_map: samples %d outside degree + 1 .. %d", o->samples, kMaxSamplesAxis);
    if (!(o->rho > 0.0) || !(o->smax > 0.0) || !(o->lam_lo > 0.0) || !(o->lam_hi > o->lam_lo) ||
        !std::isfinite(o->rho) || !std::isfinite(o->smax) || !std::isfinite(o->lam_hi))
        return fail(LT_EINVAL, "lt_build_poly_map: empty or non-finite box");
    uint64_t NC = 1, N = 1, NP = 1;
    for (int k = 0; k < 4; ++k) {
        if (o->patches[k] < 1 || o->cells[k] < 1)
            return fail(LT_EINVAL, "lt_build_poly_map: patches and cells must be >= 1");
        const uint64_t C = (uint64_t)o->patches[k] * (uint64_t)o->cells[k];
        if (C > 4096) return fail(LT_EINVAL, "lt_build_poly_map: %llu cells on axis %d (at most 4096)",
                                  (unsigned long long)C, k);
        NC *= C;
        N *= C + 1;
        NP *= (uint64_t)o->patches[k];
    }
    if (N >= (1ull << 31) || NC >= (1ull << 31))
        return fail(LT_EINVAL, "lt_build_poly_map: %llu class-grid nodes is too many", (unsigned long long)N);
    uint64_t M = 1;
    for (int k = 0; k < 4; ++k) M *= (uint64_t)o->samples;
    if (NP * M >= (1ull << 31)) return fail(LT_EINVAL, "lt_build_poly_map: too many samples");
    if (o->n_fit > 0) {
        const void* ps[] = {o->fit_x, o->fit_y, o->fit_dx, o->fit_dy, o->fit_dz, o->fit_lambda};
        for (const void* p : ps)
            if (!p || !aligned16(p)) return fail(LT_EINVAL, "lt_build_poly_map: fit arrays must be non-NULL and 16-byte aligned");
        if (o->n_fit >= (1ull << 31)) return fail(LT_EINVAL, "lt_build_poly_map: too many fit rays");
    }
    return LT_OK;
}

// RAII for the build's temporaries
struct DevBufs {
    std::vector<void*> p;
    ~DevBufs() { for (void* q : p) cudaFree(q); }
    template <class T>
    bool get(T** out, size_t bytes)
    {
        void* q = nullptr;
        if (cudaMalloc(&q, bytes ? bytes : 1) != cudaSuccess) return false;
        p.push_back(q);
        *out = static_cast<T*>(q);
        return true;
    }
};

}  // namespace

extern "C" {

lt_status lt_build_poly_map(const lt_lens* lens, const lt_poly_opts* o, lt_map** out, lt_stream stream)
{
    clear_error();
    auto t0 = std::chrono::steady_clock::now();
    if (!lens || !o || !out) return fail(LT_EINVAL, "lt_build_poly_map: NULL argument");
    *out = nullptr;
    int pi, pj;
    lt_status s = poly_check_opts(lens, o, &pi, &pj);
    if (s != LT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int D = o->degree, T = poly_terms(D), ns = o->samples;
    const int M = ns * ns * ns * ns;

    lt_map* m = new (std::nothrow) lt_map();
    if (!m) return fail(LT_ENOMEM, "lt_build_poly_map: host allocation");
    auto bail = [&](lt_status e) { delete m; return e; };
    m->kind = LT_MAP_KIND_POLY;
    m->lens = *lens;
    m->lens.presc.surfaces = m->lens.surf;
    m->lens.presc.glasses = m->lens.glass;
    m->path_id = o->path_id;
    m->tol = o->max_residual_mm;
    m->popts = *o;
    m->popts.fit_x = m->popts.fit_y = m->popts.fit_dx = m->popts.fit_dy = m->popts.fit_dz = m->popts.fit_lambda = nullptr;
    m->popts.n_fit = 0;
    std::memset(&m->dev, 0, sizeof m->dev);
    m->dev.L = lens->dev;
    m->dev.pi = pi;
    m->dev.pj = pj;
    m->cauchy = lens_all_cauchy(lens->dev);

    // box and grids
    const double lo[4] = {0.0, -o->smax, 0.0, (1000.0 / o->lam_hi) * (1000.0 / o->lam_hi)};
    const double hi[4] = {o->rho, o->smax, o->smax, (1000.0 / o->lam_lo) * (1000.0 / o->lam_lo)};
    PolyDev& P = m->pdev;
    PolyBuild B;
    std::memset(&B, 0, sizeof B);
    float step[4];
    uint64_t NC = 1, N = 1, NP = 1;
    uint32_t cs = 1, ps = 1;
    for (int k = 3; k >= 0; --k) {
        const int C = o->patches[k] * o->cells[k];
        P.lo[k] = (float)lo[k];
        P.inv[k] = (float)((double)C / (hi[k] - lo[k]));
        P.cmax[k] = (float)C;
        P.two_over_m[k] = (float)(2.0 / (double)o->cells[k]);
        P.C[k] = C;
        P.m[k] = o->cells[k];
        P.P[k] = o->patches[k];
        P.mdiv[k] = o->cells[k] == 1 ? 0u : (uint32_t)(((1ull << 32) + (uint64_t)o->cells[k] - 1) / (uint64_t)o->cells[k]);
        P.cstride[k] = cs;
        P.pstride[k] = ps;
        cs *= (uint32_t)C;
        ps *= (uint32_t)o->patches[k];
        step[k] = (float)((hi[k] - lo[k]) / (double)C);
        B.lo[k] = lo[k];
        B.h[k] = (hi[k] - lo[k]) / (double)o->patches[k];
        B.P[k] = o->patches[k];
        B.pstride[k] = P.pstride[k];
        NC *= (uint64_t)C;
        N *= (uint64_t)C + 1;
        NP *= (uint64_t)o->patches[k];
    }
    P.T = T;
    P.degree = D;
    P.n_patches = (int)NP;
    B.ns = ns;
    B.M = M;
    B.T = T;
    for (int j = 0; j < ns; ++j) B.cheb[j] = std::cos(M_PI * (j + 0.5) / ns);
    m->n_nodes = N;
    m->n_cells = NC;

    // design matrix (FP64, horner_exponents order) and the normal-equation pairs
    std::vector<int32_t> ex;
    horner_exponents(D, ex);
    std::vector<double> A((size_t)M * T);
    for (int sidx = 0; sidx < M; ++sidx) {
        double xi[4];
        int r = sidx;
        for (int k = 3; k >= 0; --k) { xi[k] = B.cheb[r % ns]; r /= ns; }
        for (int t = 0; t < T; ++t) {
            double v = 1.0;
            for (int k = 0; k < 4; ++k)
                for (int q = 0; q < ex[4 * t + k]; ++q) v *= xi[k];
            A[(size_t)sidx * T + t] = v;
        }
    }
    std::vector<uint16_t> pairs;
    for (int i = 0; i < T; ++i)
        for (int j = i; j < T; ++j) { pairs.push_back((uint16_t)i); pairs.push_back((uint16_t)j); }

    const uint32_t NW = (uint32_t)((NC + 15) / 16);
    const size_t nsamp = (size_t)NP * M;
    const int NG = (T + 3) / 4;
    if (cudaMalloc(&m->coefg, (size_t)NP * NG * 5 * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&m->coef64, (size_t)NP * T * 5 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->patch_ok, NP) != cudaSuccess || cudaMalloc(&m->node_valid, N) != cudaSuccess ||
        cudaMalloc(&m->cls, (size_t)NW * 4) != cudaSuccess)
        return bail(fail(LT_ENOMEM, "lt_build_poly_map: device allocation of the tables failed"));
    P.cg = m->coefg;
    P.patch_ok = m->patch_ok;
    P.cls = m->cls;

    // the unclipped lens: no clear apertures, no stop
    LensDev Lu = lens->dev;
    for (int k = 1; k <= Lu.S; ++k) {
        Lu.s[k].ap2 = INFINITY;
        Lu.s[k].eps2a = 0.0f;
    }
    Lu.stop_gap = -1;

    DevBufs tmp;
    double* dA = nullptr;
    uint16_t* dpairs = nullptr;
    float* ys = nullptr;
    uint8_t* vs = nullptr;
    double* G = nullptr;
    double* R = nullptr;
    float2* nout = nullptr;
    uint8_t* corner_bits = nullptr;
    uint32_t* seen = nullptr;
    uint32_t* resmax = nullptr;
    unsigned long long* sres = nullptr;
    unsigned int* cres = nullptr;
    PolyFitAccum* acc = nullptr;
    unsigned long long* counts = nullptr;
    const bool use_tol = o->max_residual_mm > 0.0;
    if (!tmp.get(&dA, A.size() * 8) || !tmp.get(&dpairs, pairs.size() * 2) || !tmp.get(&ys, nsamp * 5 * 4) ||
        !tmp.get(&vs, nsamp) || !tmp.get(&G, (size_t)NP * T * T * 8) || !tmp.get(&R, (size_t)NP * T * 5 * 8) ||
        !tmp.get(&nout, (size_t)N * sizeof(float2)) || !tmp.get(&corner_bits, NC) || !tmp.get(&seen, (size_t)NW * 4) ||
        (o->n_fit > 0 && use_tol && !tmp.get(&resmax, NC * 4)) || !tmp.get(&sres, 8) || !tmp.get(&cres, 4) ||
        !tmp.get(&acc, sizeof(PolyFitAccum)) || !tmp.get(&counts, 24))
        return bail(fail(LT_ENOMEM, "lt_build_poly_map: device allocation of temporaries failed"));

#define POLY_TRY(expr)                                               \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) return bail(cuda_fail(_e, #expr));    \
    } while (0)
    POLY_TRY(cudaMemcpyAsync(dA, A.data(), A.size() * 8, cudaMemcpyHostToDevice, st));
    POLY_TRY(cudaMemcpyAsync(dpairs, pairs.data(), pairs.size() * 2, cudaMemcpyHostToDevice, st));
    POLY_TRY(cudaMemsetAsync(seen, 0, (size_t)NW * 4, st));
    if (resmax) POLY_TRY(cudaMemsetAsync(resmax, 0, NC * 4, st));
    POLY_TRY(cudaMemsetAsync(sres, 0, 8, st));
    POLY_TRY(cudaMemsetAsync(cres, 0, 4, st));
    POLY_TRY(cudaMemsetAsync(acc, 0, sizeof(PolyFitAccum), st));
    POLY_TRY(cudaMemsetAsync(counts, 0, 24, st));

    // 1. regressor: samples through the unclipped lens, FP64 normal equations, solve, pack
    const unsigned sb = (unsigned)((nsamp + 255) / 256);
    if (m->cauchy) poly_sample_kernel<true><<<sb, 256, 0, st>>>(Lu, pi, pj, B, ys, vs, (uint32_t)nsamp);
    else poly_sample_kernel<false><<<sb, 256, 0, st>>>(Lu, pi, pj, B, ys, vs, (uint32_t)nsamp);
    const int NE = T * (T + 1) / 2 + 5 * T;
    poly_normal_kernel<<<dim3((unsigned)NP, (unsigned)((NE + 255) / 256)), 256, 0, st>>>(B, dA, dpairs, ys, vs, G, R);
    poly_solve_kernel<<<(unsigned)((NP + 63) / 64), 64, 0, st>>>(B, vs, G, R, m->coef64, m->patch_ok, (int)NP);
    poly_sample_residual_kernel<<<sb, 256, 0, st>>>(B, dA, ys, vs, m->coef64, m->patch_ok, sres, (uint32_t)nsamp);
    const uint32_t nc = (uint32_t)(NP * NG * 5);
    poly_pack_kernel<<<(nc + 255) / 256, 256, 0, st>>>(m->coef64, m->coefg, T, NG, nc);
    POLY_TRY(cudaGetLastError());

    // 2. mask: class-grid nodes through the real lens, corner classes
    const float4 stp = make_float4(step[0], step[1], step[2], step[3]);
    const unsigned nb = (unsigned)((N + 255) / 256);
    if (m->cauchy) poly_node_kernel<true><<<nb, 256, 0, st>>>(lens->dev, pi, pj, P, stp, nout, m->node_valid, (uint32_t)N);
    else poly_node_kernel<false><<<nb, 256, 0, st>>>(lens->dev, pi, pj, P, stp, nout, m->node_valid, (uint32_t)N);
    const float tol = use_tol ? (float)o->max_residual_mm : 0.0f;
    const unsigned cb = (unsigned)((NC + 255) / 256);
    LT_POLY_DISPATCH(D, { poly_cell_kernel<DD><<<cb, 256, 0, st>>>(P, nout, m->node_valid, tol, corner_bits, cres, (uint32_t)NC); });
    if (o->n_fit > 0) {
        RaysInDev fit{o->fit_x, o->fit_y, o->fit_dx, o->fit_dy, o->fit_dz, o->fit_lambda};
        const unsigned fb = (unsigned)((o->n_fit + 255) / 256);
        const bool ca = m->cauchy;
        LT_POLY_DISPATCH(D, {
            if (ca) poly_fit_kernel<DD, true><<<fb, 256, 0, st>>>(lens->dev, pi, pj, P, fit, (uint32_t)o->n_fit, corner_bits, seen, resmax, acc);
            else poly_fit_kernel<DD, false><<<fb, 256, 0, st>>>(lens->dev, pi, pj, P, fit, (uint32_t)o->n_fit, corner_bits, seen, resmax, acc);
        });
    }
    POLY_TRY(cudaGetLastError());
    s = launch_map_classify(corner_bits, seen, resmax, tol, m->cls, (uint32_t)NC, counts, st);
    if (s != LT_OK) return bail(s);

    // statistics
    PolyFitAccum ha;
    unsigned long long hc[3], hs;
    unsigned int hcr;
    std::vector<uint8_t> okh(NP), vh(nsamp);
    POLY_TRY(cudaMemcpyAsync(&ha, acc, sizeof ha, cudaMemcpyDeviceToHost, st));
    POLY_TRY(cudaMemcpyAsync(hc, counts, sizeof hc, cudaMemcpyDeviceToHost, st));
    POLY_TRY(cudaMemcpyAsync(&hs, sres, 8, cudaMemcpyDeviceToHost, st));
    POLY_TRY(cudaMemcpyAsync(&hcr, cres, 4, cudaMemcpyDeviceToHost, st));
    POLY_TRY(cudaMemcpyAsync(okh.data(), m->patch_ok, NP, cudaMemcpyDeviceToHost, st));
    POLY_TRY(cudaMemcpyAsync(vh.data(), vs, nsamp, cudaMemcpyDeviceToHost, st));
    POLY_TRY(cudaStreamSynchronize(st));
#undef POLY_TRY
    m->stats.n_nodes = N;
    m->stats.n_cells = NC;
    m->stats.cells_invalid = hc[0];
    m->stats.cells_valid = hc[1];
    m->stats.cells_boundary = hc[2];
    m->stats.fit_inside = ha.inside;
    m->stats.fit_valid = ha.valid;
    m->stats.fit_residual_rms_mm = ha.n_res ? std::sqrt(ha.sumsq / (double)ha.n_res) : 0.0;
    float fmx;
    std::memcpy(&fmx, &ha.max_res_bits, 4);
    m->stats.fit_residual_max_mm = fmx;
    m->stats.table_bytes = (uint64_t)NP * NG * 80 + NP + N + (uint64_t)NW * 4;
    lt_poly_stats& ps_ = m->pstats;
    ps_.patches = (uint32_t)NP;
    ps_.terms = (uint32_t)T;
    ps_.patches_fit = 0;
    for (uint8_t b : okh) ps_.patches_fit += b;
    ps_.samples_traced = nsamp;
    ps_.samples_valid = 0;
    for (uint8_t b : vh) ps_.samples_valid += b;
    double sr;
    std::memcpy(&sr, &hs, 8);
    ps_.sample_residual_max_mm = sr;
    float crf;
    std::memcpy(&crf, &hcr, 4);
    ps_.corner_residual_max_mm = crf;
    cudaGetDevice(&m->device);
    m->stats.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = m;
    return LT_OK;
}

lt_status lt_poly_stats_get(const lt_map* m, lt_poly_stats* out)
{
    clear_error();
    if (!m || !out) return fail(LT_EINVAL, "lt_poly_stats_get: NULL argument");
    if (m->kind != LT_MAP_KIND_POLY) return fail(LT_EINVAL, "lt_poly_stats_get: not a polynomial-patch map");
    *out = m->pstats;
    return LT_OK;
}

lt_status lt_poly_export(const lt_map* m, double* coef, int32_t* exps, uint8_t* patch_ok)
{
    clear_error();
    if (!m) return fail(LT_EINVAL, "lt_poly_export: NULL map");
    if (m->kind != LT_MAP_KIND_POLY) return fail(LT_EINVAL, "lt_poly_export: not a polynomial-patch map");
    const size_t NP = m->pstats.patches, T = m->pstats.terms;
    if (coef) LT_CUDA_TRY(cudaMemcpy(coef, m->coef64, NP * T * 5 * sizeof(double), cudaMemcpyDeviceToHost));
    if (patch_ok) LT_CUDA_TRY(cudaMemcpy(patch_ok, m->patch_ok, NP, cudaMemcpyDeviceToHost));
    if (exps) {
        std::vector<int32_t> ex;
        horner_exponents(m->pdev.degree, ex);
        std::memcpy(exps, ex.data(), ex.size() * sizeof(int32_t));
    }
    return LT_OK;
}

}  // extern "C"
