// Learned lens transport map: the paper's classifier / regressor MLPs
// (Sec. 4.2 "Neural Ray Masking", "C^1 Continuous Network"; Sec. 5.1 "MLP
// Training", "Inference") trained and queried by this library's kernels.
//
//   g: 4 -> 32 -> 32 -> 1 (tanh hidden, logit out), BCE loss
//   f: 4 -> 32 x 5 -> 6 (tanh hidden, linear out), MSE on position and
//      throughput + (1 - cosine) on direction
// Inputs: the symmetry-reduced entrance ray (Sec. 4.1, Eq. 10).  Training:
// Adam with lr * decay^(step / every) (Sec. 5.1); per-block gradient sums in
// FP32, the sum over blocks in FP64.  Queries: FP32 SIMT with a rational tanh
// (the paper approximates tanh by a rational function, Sec. 5.1; here the
// 9/10 truncation of Lambert's continued fraction), or BF16 / FP16 on the
// 5th-generation tensor cores (tcgen05.mma, FP32 accumulation in TMEM; see
// mlp_tc.cuh) with tanh.approx on packed pairs.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "map_internal.h"
#include "profile.h"
#include "rays.cuh"
#include "tracer.cuh"

#include "mlp_dev.cuh"

namespace lt {

// Trace each fit ray along the path; write network inputs X (n x 4), the
// reduced-frame targets T (n x 6, valid rays only) and labels; count each
// block's valid rays (bcount) and those among the first n_uniform
// (bcount_u).  The valid list is built from the labels in ray order by
// mlp_scan_kernel and mlp_compact_kernel, so that training is a pure
// function of its inputs.
template <bool CAUCHY>
__global__ void __launch_bounds__(256)
mlp_prep_kernel(const __grid_constant__ LensDev L, int pi, int pj, RaysInDev fit, uint32_t n,
                uint32_t n_uniform, MlpFrame F, float* __restrict__ X, float* __restrict__ T,
                float* __restrict__ label, uint32_t* __restrict__ bcount, uint32_t* __restrict__ bcount_u)
{
    const uint32_t r = blockIdx.x * 256u + threadIdx.x;
    bool valid = false;
    if (r < n) {
        const float x = __ldg(fit.x + r), y = __ldg(fit.y + r), dx = __ldg(fit.dx + r),
                    dy = __ldg(fit.dy + r), dz = __ldg(fit.dz + r), lam = __ldg(fit.lam + r);
        float xin[4];
        RedFrame rf;
        mlp_features(F, x, y, dx, dy, dz, lam, xin, rf);
        TraceOut o;
        int nint;
        const uint32_t f = trace_ray<CAUCHY>(L, pi, pj, x, y, dx, dy, dz, lam, o, nint);
        valid = (f & LT_FLAG_VALID) != 0 && (f & LT_FLAG_BAD_INPUT) == 0;
        const bool bad = (f & LT_FLAG_BAD_INPUT) != 0;
        reinterpret_cast<float4*>(X)[r] = bad ? make_float4(0.f, 0.f, 0.f, 0.f)
                                              : make_float4(xin[0], xin[1], xin[2], xin[3]);
        label[r] = valid ? 1.0f : 0.0f;
        float t[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (valid) {
            t[0] = fmaf(rf.c, o.x, rf.s * o.y);
            t[1] = rf.m * fmaf(-rf.s, o.x, rf.c * o.y);
            t[2] = fmaf(rf.c, o.dx, rf.s * o.dy);
            t[3] = rf.m * fmaf(-rf.s, o.dx, rf.c * o.dy);
            t[4] = o.dz;
            t[5] = o.I;
        }
        float2* tp = reinterpret_cast<float2*>(T + (size_t)r * 6);
        tp[0] = make_float2(t[0], t[1]);
        tp[1] = make_float2(t[2], t[3]);
        tp[2] = make_float2(t[4], t[5]);
    }
    const int c = __syncthreads_count(valid);
    const int cu = __syncthreads_count(valid && r < n_uniform);
    if (threadIdx.x == 0) {
        bcount[blockIdx.x] = (uint32_t)c;
        bcount_u[blockIdx.x] = (uint32_t)cu;
    }
}

// One block of 1024 threads: exclusive prefix sums of the per-block counts
// (boff) in chunks of 1024; vcount[0] = valid rays, vcount[1] = valid rays
// among the uniform prefix.
__global__ void __launch_bounds__(1024)
mlp_scan_kernel(const uint32_t* __restrict__ bcount, const uint32_t* __restrict__ bcount_u, uint32_t nb,
                uint32_t* __restrict__ boff, uint32_t* __restrict__ vcount)
{
    __shared__ uint32_t wsum[32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = 0, su = 0;
    for (uint32_t base = 0; base < nb; base += 1024u) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? bcount[i] : 0u;
        if (i < nb) su += bcount_u[i];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(full, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(full, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        if (i < nb) boff[i] = carry + (warp > 0 ? wsum[warp - 1] : 0u) + x - v;
        carry += wsum[31];
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) su += __shfl_xor_sync(full, su, o);
    if (lane == 0) wsum[warp] = su;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int k = 0; k < 32; ++k) t += wsum[k];
        vcount[0] = carry;
        vcount[1] = t;
    }
}

// The valid rays' indices in ray order (same blocks as mlp_prep_kernel).
__global__ void __launch_bounds__(256)
mlp_compact_kernel(const float* __restrict__ label, uint32_t n, const uint32_t* __restrict__ boff,
                   uint32_t* __restrict__ vlist)
{
    __shared__ uint32_t wc[8];
    const uint32_t r = blockIdx.x * 256u + threadIdx.x;
    const bool valid = r < n && label[r] != 0.0f;
    const unsigned full = 0xffffffffu;
    const unsigned m = __ballot_sync(full, valid);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wc[warp] = (uint32_t)__popc(m);
    __syncthreads();
    uint32_t off = boff[blockIdx.x];
    for (int k = 0; k < warp; ++k) off += wc[k];
    if (valid) vlist[off + __popc(m & ((1u << lane) - 1u))] = r;
}

// FP64 sums of the targets and their squares over the valid list: one
// partial per warp (part[warp][12]), summed in warp order by
// mlp_stats_sum_kernel.
constexpr int kStatsBlocks = 152 * 4;

__global__ void __launch_bounds__(256)
mlp_stats_kernel(const float* __restrict__ T, const uint32_t* __restrict__ vlist,
                 const uint32_t* __restrict__ vcount, double* __restrict__ part)
{
    const uint32_t cnt = *vcount;
    double s[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) s[q] = 0.0;
    for (uint32_t i = blockIdx.x * 256u + threadIdx.x; i < cnt; i += gridDim.x * 256u) {
        const float* t = T + (size_t)vlist[i] * 6;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const double v = t[q];
            s[q] += v;
            s[6 + q] += v * v;
        }
    }
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int q = 0; q < 12; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(full, s[q], o);
    }
    if ((threadIdx.x & 31) == 0) {
        double* p = part + ((size_t)blockIdx.x * 8u + (threadIdx.x >> 5)) * 12u;
#pragma unroll
        for (int q = 0; q < 12; ++q) p[q] = s[q];
    }
}

__global__ void mlp_stats_sum_kernel(const double* __restrict__ part, int nparts, double* __restrict__ sums)
{
    const int q = threadIdx.x;
    if (q >= 12) return;
    double t = 0.0;
    for (int k = 0; k < nparts; ++k) t += part[(size_t)k * 12 + q];
    sums[q] = t;
}

// ------------------------------------------------------------------ training step

// SplitMix64 (Steele, Lea and Flood, 2014): a counter-based 64-bit mixer.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

constexpr int kTB = 128;   // rays per training block
// Row stride (floats) of the block's activations and deltas in shared memory:
// odd, so that the weight-gradient products, whose lanes read one column of
// different rows, hit 32 different banks.
constexpr int kTS = kTB + 1;

struct TrainBatch {
    const float* X;          // inputs (n x 4)
    const float* T;          // REG: raw reduced-frame targets (n x 6) or standardised batch targets
    const float* label;      // CLS: labels
    const uint32_t* list;    // indices to draw from; NULL with n_list > 0: draw rows of [0, n_list);
    uint32_t n_list;         // NULL with n_list == 0: explicit batch, item b is row b
    uint64_t seed, step;
    int B;
    int standardised;        // targets already standardised (explicit batch)
};

// One forward + backward pass over rays [blockIdx.x * 128, +128) of the batch.
// Per-block gradient sums (FP32, over the block's rays) go to G[block][param],
// the block's loss sum (FP64) to loss[block].  Activations and deltas of the
// block live in shared memory for the weight-gradient products.
template <bool REG>
__global__ void __launch_bounds__(kTB)
mlp_train_kernel(const float* __restrict__ P, TrainBatch tb, MlpFrame F, float* __restrict__ G,
                 double* __restrict__ loss)
{
    using N = Net<REG>;
    extern __shared__ float sh[];
    float* W = sh;                                    // N::NP
    float* act = W + ((N::NP + 3) & ~3);              // L layers x 32 rows of kTS (layer 0 = inputs)
    float* dl = act + N::L * 32 * kTS;                // 32 rows of kTS deltas
    __shared__ double lsum[kTB / 32];
    for (int i = threadIdx.x; i < N::NP; i += kTB) W[i] = P[i];
    const int j = threadIdx.x;
    const int b = blockIdx.x * kTB + j;
    const bool live = b < tb.B;
    uint32_t row = 0;
    if (live) {
        if (tb.n_list) {
            const uint64_t h = splitmix64(tb.seed + tb.step * (uint64_t)tb.B + (uint64_t)b);
            row = tb.list ? tb.list[h % tb.n_list] : (uint32_t)(h % tb.n_list);
        } else {
            row = (uint32_t)b;
        }
    }
    float a[32];
    {
        const float4 x = live ? reinterpret_cast<const float4*>(tb.X)[row] : make_float4(0.f, 0.f, 0.f, 0.f);
        a[0] = x.x; a[1] = x.y; a[2] = x.z; a[3] = x.w;
        act[0 * kTS + j] = a[0];
        act[1 * kTS + j] = a[1];
        act[2 * kTS + j] = a[2];
        act[3 * kTS + j] = a[3];
    }
    __syncthreads();
    float z[N::NOUT];
    // forward
#pragma unroll
    for (int l = 0; l < N::L; ++l) {
        const int ni = N::in(l), no = N::out(l);
        const float* Wl = W + N::woff(l);
        const float* bl = W + N::boff(l);
        float t[32];
#pragma unroll
        for (int o = 0; o < 32; ++o) {
            if (o < no) {
                float s = bl[o];
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (k < ni) s = fmaf(Wl[o * ni + k], a[k], s);
                t[o] = s;
            }
        }
        if (l < N::L - 1) {
#pragma unroll
            for (int o = 0; o < 32; ++o) {
                a[o] = tanhf(t[o]);
                act[((l + 1) * 32 + o) * kTS + j] = a[o];
            }
        } else {
#pragma unroll
            for (int o = 0; o < N::NOUT; ++o) z[o] = t[o];
        }
    }
    // loss and its gradient w.r.t. the outputs (batch mean)
    float d[32];
    double lval = 0.0;
    const float invB = 1.0f / (float)tb.B;
    if (REG) {
        float t[6];
        if (live) {
            const float* tp = tb.T + (size_t)row * 6;
#pragma unroll
            for (int q = 0; q < 6; ++q)
                t[q] = tb.standardised ? tp[q] : (tp[q] - F.t_mean[q]) / F.t_std[q];
        } else {
#pragma unroll
            for (int q = 0; q < 6; ++q) t[q] = 0.0f;
        }
        const float e0 = z[0] - t[0], e1 = z[1] - t[1], e5 = z[5 % N::NOUT] - t[5];
        float dp[3], dt[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            dp[q] = fmaf(F.t_std[2 + q], z[(2 + q) % N::NOUT], F.t_mean[2 + q]);
            dt[q] = fmaf(F.t_std[2 + q], t[2 + q], F.t_mean[2 + q]);
        }
        const float npd = sqrtf(dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2]);
        const float ntd = sqrtf(dt[0] * dt[0] + dt[1] * dt[1] + dt[2] * dt[2]);
        const float cs = (dp[0] * dt[0] + dp[1] * dt[1] + dp[2] * dt[2]) / (npd * ntd);
        if (live) {
            lval = 0.5 * ((double)e0 * e0 + (double)e1 * e1) + (double)e5 * e5 + (1.0 - (double)cs);
            d[0] = e0 * invB;
            d[1] = e1 * invB;
            d[5 % N::NOUT] = 2.0f * e5 * invB;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float dc = dt[q] / (npd * ntd) - cs * dp[q] / (npd * npd);
                d[(2 + q) % N::NOUT] = -dc * F.t_std[2 + q] * invB;
            }
        } else {
#pragma unroll
            for (int q = 0; q < N::NOUT; ++q) d[q] = 0.0f;
        }
    } else {
        const float y = live ? tb.label[row] : 0.0f;
        const float zz = z[0];
        if (live) {
            lval = (double)fmaxf(zz, 0.0f) - (double)y * zz + log1p(exp(-(double)fabsf(zz)));
            const float sg = 1.0f / (1.0f + __expf(-zz));
            d[0] = (sg - y) * invB;
        } else {
            d[0] = 0.0f;
        }
    }
    {
        const unsigned full = 0xffffffffu;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lval += __shfl_xor_sync(full, lval, o);
        if ((j & 31) == 0) lsum[j >> 5] = lval;
    }
    // backward
    float* Gb = G + (size_t)blockIdx.x * N::NP;
#pragma unroll
    for (int l = N::L - 1; l >= 0; --l) {
        const int ni = N::in(l), no = N::out(l);
        const float* Wl = W + N::woff(l);
#pragma unroll
        for (int o = 0; o < 32; ++o)
            if (o < no) dl[o * kTS + j] = d[o];
        __syncthreads();
        // dW[o][k] = sum_j d[o][j] a_l[k][j], db[o] = sum_j d[o][j]: each
        // thread takes a tile of kGO x kGK weights, so that a delta and an
        // activation loaded from shared memory serve kGK and kGO products
        // (every entry still sums over the block's rays in ray order)
        const float* al = act + l * 32 * kTS;
        constexpr int kGO = 2, kGK = 4;
        const int nto = (no + kGO - 1) / kGO, ntk = (ni + kGK - 1) / kGK;
        for (int tile = j; tile < nto * ntk; tile += kTB) {
            const int o0 = (tile / ntk) * kGO, k0 = (tile % ntk) * kGK;
            const float* dr[kGO];
            const float* ar[kGK];
#pragma unroll
            for (int i = 0; i < kGO; ++i) dr[i] = dl + min(o0 + i, no - 1) * kTS;
#pragma unroll
            for (int c = 0; c < kGK; ++c) ar[c] = al + min(k0 + c, ni - 1) * kTS;
            float sacc[kGO][kGK];
#pragma unroll
            for (int i = 0; i < kGO; ++i)
#pragma unroll
                for (int c = 0; c < kGK; ++c) sacc[i][c] = 0.0f;
#pragma unroll 4
            for (int q = 0; q < kTB; ++q) {
                float dv[kGO], av[kGK];
#pragma unroll
                for (int i = 0; i < kGO; ++i) dv[i] = dr[i][q];
#pragma unroll
                for (int c = 0; c < kGK; ++c) av[c] = ar[c][q];
#pragma unroll
                for (int i = 0; i < kGO; ++i)
#pragma unroll
                    for (int c = 0; c < kGK; ++c) sacc[i][c] = fmaf(dv[i], av[c], sacc[i][c]);
            }
#pragma unroll
            for (int i = 0; i < kGO; ++i)
#pragma unroll
                for (int c = 0; c < kGK; ++c)
                    if (o0 + i < no && k0 + c < ni) Gb[N::woff(l) + (o0 + i) * ni + (k0 + c)] = sacc[i][c];
        }
        for (int o = j; o < no; o += kTB) {
            const float* dr = dl + o * kTS;
            float sb = 0.0f;
#pragma unroll 8
            for (int q = 0; q < kTB; ++q) sb += dr[q];
            Gb[N::boff(l) + o] = sb;
        }
        if (l > 0) {
            float nd[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                float s = 0.0f;
#pragma unroll
                for (int o = 0; o < 32; ++o)
                    if (o < no) s = fmaf(Wl[o * ni + k], d[o], s);
                const float ak = act[(l * 32 + k) * kTS + j];
                nd[k] = s * (1.0f - ak * ak);
            }
#pragma unroll
            for (int k = 0; k < 32; ++k) d[k] = nd[k];
        }
        __syncthreads();
    }
    if (j == 0) {
        double s = 0.0;
        for (int w = 0; w < kTB / 32; ++w) s += lsum[w];
        loss[blockIdx.x] = s;
    }
}

// Adam update (beta1 0.9, beta2 0.999, eps 1e-8): the batch gradient is the
// FP64 sum of the per-block partial sums.
__global__ void __launch_bounds__(256)
mlp_adam_kernel(float* __restrict__ P, const float* __restrict__ G, int nblocks, int np,
                double* __restrict__ m1, double* __restrict__ m2, double lr, double c1, double c2)
{
    const int p = blockIdx.x * 256 + threadIdx.x;
    if (p >= np) return;
    double g = 0.0;
    // unrolled so that sixteen partials' loads are in flight at once (the
    // sum keeps its order)
#pragma unroll 16
    for (int b = 0; b < nblocks; ++b) g += (double)G[(size_t)b * np + p];
    const double m = 0.9 * m1[p] + 0.1 * g;
    const double v = 0.999 * m2[p] + 0.001 * g * g;
    m1[p] = m;
    m2[p] = v;
    P[p] = (float)((double)P[p] - lr * (m / c1) / (sqrt(v / c2) + 1e-8));
}

}  // namespace lt


namespace lt {

// features only (for tests and callers that want the network inputs)
__global__ void __launch_bounds__(256)
mlp_features_kernel(MlpFrame F, RaysInDev in, float* __restrict__ X, uint32_t n)
{
    const uint32_t r = blockIdx.x * 256u + threadIdx.x;
    if (r >= n) return;
    float xin[4];
    RedFrame rf;
    mlp_features(F, __ldg(in.x + r), __ldg(in.y + r), __ldg(in.dx + r), __ldg(in.dy + r),
                 __ldg(in.dz + r), __ldg(in.lam + r), xin, rf);
    reinterpret_cast<float4*>(X)[r] = make_float4(xin[0], xin[1], xin[2], xin[3]);
}

}  // namespace lt

using namespace lt;

struct lt_mlp {
    lt_lens lens;
    int pi = 0, pj = 0;
    bool cauchy = true;
    lt_mlp_frame frame = {};
    double t_mean[6] = {}, t_std[6] = {};
    MlpFrame F = {};
    float* reg = nullptr;
    float* cls = nullptr;
    unsigned char* tc_bf16 = nullptr;   // tcgen05 weight images (BF16 / FP16 + FP32 biases)
    unsigned char* tc_f16 = nullptr;
    uint32_t* tc_err = nullptr;         // count of tensor-core waits that ran out
    TcBias tc_bias = {};                // FP32 biases of the tensor-core query
    bool frags_stale = true;            // tensor-core weight images out of date
    lt_mlp_stats stats = {};
    ~lt_mlp()
    {
        if (reg) cudaFree(reg);
        if (cls) cudaFree(cls);
        if (tc_bf16) cudaFree(tc_bf16);
        if (tc_f16) cudaFree(tc_f16);
        if (tc_err) cudaFree(tc_err);
    }
};

namespace lt {

static void set_frame(lt_mlp* m)
{
    MlpFrame& F = m->F;
    F.rho2_inv = (float)(2.0 / m->frame.rho);
    F.winv = (float)(1.0 / m->frame.wmax);
    F.winv2 = (float)(2.0 / m->frame.wmax);
    F.lam_lo = (float)m->frame.lam_lo;
    F.lam_scale = (float)(2.0 / (m->frame.lam_hi - m->frame.lam_lo));
    for (int q = 0; q < 6; ++q) {
        F.t_mean[q] = (float)m->t_mean[q];
        F.t_std[q] = (float)m->t_std[q];
    }
}

static lt_status check_frame(const lt_lens* lens, const lt_mlp_frame* fr, int* pi, int* pj)
{
    if (!path_ij(lens->S, fr->path_id, pi, pj)) return fail(LT_EINVAL, "learned map: bad path id %d", fr->path_id);
    if (!(fr->rho > 0.0) || !(fr->wmax > 0.0) || !(fr->lam_hi > fr->lam_lo))
        return fail(LT_EINVAL, "learned map: empty input box");
    return LT_OK;
}

static lt_mlp* new_mlp(const lt_lens* lens, const lt_mlp_frame* fr, int pi, int pj)
{
    lt_mlp* m = new (std::nothrow) lt_mlp();
    if (!m) return nullptr;
    m->lens = *lens;
    m->lens.presc.surfaces = m->lens.surf;
    m->lens.presc.glasses = m->lens.glass;
    m->pi = pi;
    m->pj = pj;
    m->cauchy = lens_all_cauchy(lens->dev);
    m->frame = *fr;
    if (cudaMalloc(&m->reg, LT_MLP_REG_PARAMS * 4) != cudaSuccess ||
        cudaMalloc(&m->cls, LT_MLP_CLS_PARAMS * 4) != cudaSuccess) {
        delete m;
        return nullptr;
    }
    return m;
}

// The tcgen05 weight images: every weight at its place in the canonical
// K-major layout (tc_elem_offset), zero padding elsewhere, then the FP32
// biases; one image in BF16 and one in FP16.
static lt_status build_tc_image(lt_mlp* m)
{
    std::vector<float> reg(LT_MLP_REG_PARAMS), cls(LT_MLP_CLS_PARAMS);
    LT_CUDA_TRY(cudaMemcpy(reg.data(), m->reg, reg.size() * 4, cudaMemcpyDeviceToHost));
    LT_CUDA_TRY(cudaMemcpy(cls.data(), m->cls, cls.size() * 4, cudaMemcpyDeviceToHost));
    std::vector<unsigned char> ib(kImgBytes, 0), ih(kImgBytes, 0);
    auto put = [&](int base, int N, int row, int k, float v) {
        const int off = base + tc_elem_offset(N, row, k);
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        const __half h = __float2half_rn(v);
        std::memcpy(&ib[off], &b, 2);
        std::memcpy(&ih[off], &h, 2);
    };
    using R = Net<true>;
    using C = Net<false>;
    for (int o = 0; o < 32; ++o)
        for (int k = 0; k < 4; ++k) {
            put(kImgB0, 64, o, k, reg[R::woff(0) + o * 4 + k]);
            put(kImgB0, 64, 32 + o, k, cls[C::woff(0) + o * 4 + k]);
        }
    for (int l = 1; l <= 4; ++l)
        for (int o = 0; o < 32; ++o)
            for (int k = 0; k < 32; ++k) put(kImgR1 + (l - 1) * kLayerBytes, 32, o, k, reg[R::woff(l) + o * 32 + k]);
    for (int o = 0; o < 6; ++o)
        for (int k = 0; k < 32; ++k) put(kImgR5, 32, o, k, reg[R::woff(5) + o * 32 + k]);
    for (int o = 0; o < 32; ++o)
        for (int k = 0; k < 32; ++k) put(kImgC1, 32, o, k, cls[C::woff(1) + o * 32 + k]);
    for (int k = 0; k < 32; ++k) put(kImgC2, 32, 0, k, cls[C::woff(2) + k]);
    for (int l = 0; l < 5; ++l)
        for (int o = 0; o < 32; ++o) m->tc_bias.b[kBiasReg + 32 * l + o] = reg[R::boff(l) + o];
    for (int q = 0; q < 6; ++q) m->tc_bias.b[kBiasRegOut + q] = reg[R::boff(5) + q];
    for (int l = 0; l < 2; ++l)
        for (int o = 0; o < 32; ++o) m->tc_bias.b[kBiasCls + 32 * l + o] = cls[C::boff(l) + o];
    m->tc_bias.b[kBiasClsOut] = cls[C::boff(2)];
    if (!m->tc_bf16 && cudaMalloc(&m->tc_bf16, kImgBytes) != cudaSuccess)
        return fail(LT_ENOMEM, "learned map: weight image allocation");
    if (!m->tc_f16 && cudaMalloc(&m->tc_f16, kImgBytes) != cudaSuccess)
        return fail(LT_ENOMEM, "learned map: weight image allocation");
    if (!m->tc_err) {
        if (cudaMalloc(&m->tc_err, 4) != cudaSuccess) return fail(LT_ENOMEM, "learned map: error counter");
        LT_CUDA_TRY(cudaMemset(m->tc_err, 0, 4));
    }
    LT_CUDA_TRY(cudaMemcpy(m->tc_bf16, ib.data(), kImgBytes, cudaMemcpyHostToDevice));
    LT_CUDA_TRY(cudaMemcpy(m->tc_f16, ih.data(), kImgBytes, cudaMemcpyHostToDevice));
    m->frags_stale = false;
    return LT_OK;
}

// ------------------------------------------------------------------ fused serving launches

lt_status mlp_serve_blob(const lt_mlp* mc, int precision, std::vector<unsigned char>& b)
{
    lt_mlp* m = const_cast<lt_mlp*>(mc);
    if (precision == LT_MLP_BF16 || precision == LT_MLP_F16) {
        if (m->frags_stale) {
            const lt_status s = build_tc_image(m);
            if (s != LT_OK) return s;
        }
        TcServe X{};
        X.F = m->F;
        X.B = m->tc_bias;
        X.img = precision == LT_MLP_BF16 ? m->tc_bf16 : m->tc_f16;
        X.err = m->tc_err;
        b.assign(reinterpret_cast<const unsigned char*>(&X), reinterpret_cast<const unsigned char*>(&X) + sizeof X);
        return LT_OK;
    }
    if (precision != LT_MLP_F32 && precision != LT_MLP_F32_NOCLS)
        return fail(LT_EINVAL, "learned map: unknown precision %d", precision);
    const MlpDev D{m->F, m->reg, m->cls};
    b.assign(reinterpret_cast<const unsigned char*>(&D), reinterpret_cast<const unsigned char*>(&D) + sizeof D);
    return LT_OK;
}

template <bool REG>
static size_t train_smem()
{
    return (size_t)(((Net<REG>::NP + 3) & ~3) + Net<REG>::L * 32 * kTS + 32 * kTS) * sizeof(float);
}

// one training step of net REG on the batch; returns the batch-mean loss when `want_loss`
template <bool REG>
static lt_status train_step(float* P, const TrainBatch& tb, const MlpFrame& F, float* G,
                            double* lossbuf, double* m1, double* m2, double lr, long t,
                            cudaStream_t st)
{
    const int blocks = (tb.B + kTB - 1) / kTB;
    {
        ProfScope prof(REG ? "mlp_train_reg_kernel" : "mlp_train_cls_kernel", st);
        mlp_train_kernel<REG><<<blocks, kTB, train_smem<REG>(), st>>>(P, tb, F, G, lossbuf);
    }
    LT_CUDA_TRY(cudaGetLastError());
    if (m1) {
        const double c1 = 1.0 - std::pow(0.9, (double)t), c2 = 1.0 - std::pow(0.999, (double)t);
        ProfScope prof("mlp_adam_kernel", st);
        mlp_adam_kernel<<<(Net<REG>::NP + 255) / 256, 256, 0, st>>>(P, G, blocks, Net<REG>::NP, m1, m2, lr, c1, c2);
        LT_CUDA_TRY(cudaGetLastError());
    }
    return LT_OK;
}

static lt_status set_train_attrs()
{
    static bool done = false;
    if (done) return LT_OK;
    LT_CUDA_TRY(cudaFuncSetAttribute(mlp_train_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)train_smem<true>()));
    LT_CUDA_TRY(cudaFuncSetAttribute(mlp_train_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)train_smem<false>()));
    done = true;
    return LT_OK;
}

// run `steps` Adam steps of one network; records the mean loss of the last 100
template <bool REG>
static lt_status train_net(lt_mlp* m, float* P, TrainBatch tb, int steps, double lr0, double decay,
                           int every, double* last_loss, cudaStream_t st)
{
    const int max_blocks = (tb.B + kTB - 1) / kTB;
    float* G = nullptr;
    double *lossbuf = nullptr, *m1 = nullptr, *m2 = nullptr;
    const int np = Net<REG>::NP;
    lt_status s = LT_OK;
    std::vector<double> hl;
    const int tail = std::min(steps, 100);
    double acc = 0.0;
    if (cudaMalloc(&G, (size_t)max_blocks * np * 4) != cudaSuccess ||
        cudaMalloc(&lossbuf, (size_t)max_blocks * 8 * (tail > 0 ? tail : 1)) != cudaSuccess ||
        cudaMalloc(&m1, np * 8) != cudaSuccess || cudaMalloc(&m2, np * 8) != cudaSuccess) {
        s = fail(LT_ENOMEM, "learned map: training buffers");
    } else {
        cudaMemsetAsync(m1, 0, np * 8, st);
        cudaMemsetAsync(m2, 0, np * 8, st);
        for (int k = 0; k < steps && s == LT_OK; ++k) {
            tb.step = (uint64_t)k;
            const double lr = lr0 * std::pow(decay, (double)(k / (every > 0 ? every : 1)));
            double* lb = lossbuf;
            if (k >= steps - tail) lb = lossbuf + (size_t)(k - (steps - tail)) * max_blocks;
            s = train_step<REG>(P, tb, m->F, G, lb, m1, m2, lr, k + 1, st);
        }
        if (s == LT_OK && tail > 0) {
            hl.resize((size_t)tail * max_blocks);
            if (cudaMemcpyAsync(hl.data(), lossbuf, hl.size() * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                s = fail(LT_ECUDA, "learned map: loss read-back");
            for (double v : hl) acc += v;
            *last_loss = acc / ((double)tail * tb.B);
        }
    }
    if (G) cudaFree(G);
    if (lossbuf) cudaFree(lossbuf);
    if (m1) cudaFree(m1);
    if (m2) cudaFree(m2);
    return s;
}

}  // namespace lt

extern "C" {

lt_status lt_mlp_create(const lt_lens* lens, const lt_mlp_frame* frame, const float* reg,
                        const float* cls, const double* t_mean, const double* t_std, lt_mlp** out)
{
    clear_error();
    if (!lens || !frame || !reg || !cls || !t_mean || !t_std || !out)
        return fail(LT_EINVAL, "lt_mlp_create: NULL argument");
    *out = nullptr;
    int pi, pj;
    lt_status s = check_frame(lens, frame, &pi, &pj);
    if (s != LT_OK) return s;
    lt_mlp* m = new_mlp(lens, frame, pi, pj);
    if (!m) return fail(LT_ENOMEM, "lt_mlp_create: allocation");
    for (int q = 0; q < 6; ++q) {
        if (!(t_std[q] > 0.0)) { delete m; return fail(LT_EINVAL, "lt_mlp_create: t_std must be > 0"); }
        m->t_mean[q] = t_mean[q];
        m->t_std[q] = t_std[q];
        m->stats.t_mean[q] = t_mean[q];
        m->stats.t_std[q] = t_std[q];
    }
    set_frame(m);
    if (cudaMemcpy(m->reg, reg, LT_MLP_REG_PARAMS * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->cls, cls, LT_MLP_CLS_PARAMS * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        delete m;
        return fail(LT_ECUDA, "lt_mlp_create: upload");
    }
    *out = m;
    return LT_OK;
}

void lt_destroy_mlp(lt_mlp* m) { delete m; }

lt_status lt_mlp_stats_get(const lt_mlp* m, lt_mlp_stats* out)
{
    if (!m || !out) return fail(LT_EINVAL, "lt_mlp_stats_get: NULL argument");
    *out = m->stats;
    out->tc_wait_timeouts = 0;
    if (m->tc_err) {
        uint32_t e = 0;
        LT_CUDA_TRY(cudaMemcpy(&e, m->tc_err, 4, cudaMemcpyDeviceToHost));
        out->tc_wait_timeouts = e;
    }
    return LT_OK;
}

lt_status lt_mlp_get_params(const lt_mlp* m, float* reg, float* cls)
{
    clear_error();
    if (!m) return fail(LT_EINVAL, "lt_mlp_get_params: NULL map");
    if (reg) LT_CUDA_TRY(cudaMemcpy(reg, m->reg, LT_MLP_REG_PARAMS * 4, cudaMemcpyDeviceToHost));
    if (cls) LT_CUDA_TRY(cudaMemcpy(cls, m->cls, LT_MLP_CLS_PARAMS * 4, cudaMemcpyDeviceToHost));
    return LT_OK;
}

lt_status lt_mlp_train(const lt_lens* lens, const lt_mlp_opts* o, lt_mlp** out, lt_stream stream)
{
    clear_error();
    auto t0 = std::chrono::steady_clock::now();
    if (!lens || !o || !out || !o->init_reg || !o->init_cls) return fail(LT_EINVAL, "lt_mlp_train: NULL argument");
    *out = nullptr;
    int pi, pj;
    lt_status s = check_frame(lens, &o->frame, &pi, &pj);
    if (s != LT_OK) return s;
    if (o->n_fit < 1 || o->n_fit >= (1ull << 31)) return fail(LT_EINVAL, "lt_mlp_train: n_fit out of range");
    if (o->n_fit_uniform > o->n_fit) return fail(LT_EINVAL, "lt_mlp_train: n_fit_uniform above n_fit");
    const void* ps[] = {o->fit_x, o->fit_y, o->fit_dx, o->fit_dy, o->fit_dz, o->fit_lambda};
    for (const void* p : ps)
        if (!p || !aligned16(p)) return fail(LT_EINVAL, "lt_mlp_train: fit arrays must be non-NULL and 16-byte aligned");
    if (o->reg_batch < 1 || o->cls_batch < 1 || o->reg_steps < 0 || o->cls_steps < 0 ||
        (o->ft_steps > 0 && o->ft_batch < 1))
        return fail(LT_EINVAL, "lt_mlp_train: bad step or batch count");
    if ((s = set_train_attrs()) != LT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    lt_mlp* m = new_mlp(lens, &o->frame, pi, pj);
    if (!m) return fail(LT_ENOMEM, "lt_mlp_train: allocation");
    const uint32_t n = (uint32_t)o->n_fit;
    float *X = nullptr, *T = nullptr, *lab = nullptr;
    uint32_t *vlist = nullptr, *vcount = nullptr, *bc = nullptr;
    double* sums = nullptr;
    const uint32_t nb = (n + 255) / 256;
    const int nparts = kStatsBlocks * 8;
    do {
        if (cudaMemcpy(m->reg, o->init_reg, LT_MLP_REG_PARAMS * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(m->cls, o->init_cls, LT_MLP_CLS_PARAMS * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            s = fail(LT_ECUDA, "lt_mlp_train: parameter upload");
            break;
        }
        if (cudaMalloc(&X, (size_t)n * 16) != cudaSuccess || cudaMalloc(&T, (size_t)n * 24) != cudaSuccess ||
            cudaMalloc(&lab, (size_t)n * 4) != cudaSuccess || cudaMalloc(&vlist, (size_t)n * 4) != cudaSuccess ||
            cudaMalloc(&vcount, 8) != cudaSuccess || cudaMalloc(&bc, (size_t)nb * 12) != cudaSuccess ||
            cudaMalloc(&sums, (size_t)(12 + nparts * 12) * 8) != cudaSuccess) {
            s = fail(LT_ENOMEM, "lt_mlp_train: training data allocation");
            break;
        }
        // provisional frame for the features (target statistics come next)
        for (int q = 0; q < 6; ++q) { m->t_mean[q] = 0.0; m->t_std[q] = 1.0; }
        set_frame(m);
        RaysInDev fit{o->fit_x, o->fit_y, o->fit_dx, o->fit_dy, o->fit_dz, o->fit_lambda};
        const uint32_t nu = o->n_fit_uniform == 0 ? n : (uint32_t)o->n_fit_uniform;
        uint32_t *bcount = bc, *bcount_u = bc + nb, *boff = bc + 2 * (size_t)nb;
        if (m->cauchy)
            mlp_prep_kernel<true><<<nb, 256, 0, st>>>(lens->dev, pi, pj, fit, n, nu, m->F, X, T, lab, bcount, bcount_u);
        else
            mlp_prep_kernel<false><<<nb, 256, 0, st>>>(lens->dev, pi, pj, fit, n, nu, m->F, X, T, lab, bcount, bcount_u);
        mlp_scan_kernel<<<1, 1024, 0, st>>>(bcount, bcount_u, nb, boff, vcount);
        mlp_compact_kernel<<<nb, 256, 0, st>>>(lab, n, boff, vlist);
        mlp_stats_kernel<<<kStatsBlocks, 256, 0, st>>>(T, vlist, vcount, sums + 12);
        mlp_stats_sum_kernel<<<1, 32, 0, st>>>(sums + 12, nparts, sums);
        uint32_t nvs[2] = {0, 0};
        double hs[12];
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(nvs, vcount, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(hs, sums, 96, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            s = fail(LT_ECUDA, "lt_mlp_train: data preparation");
            break;
        }
        const uint32_t nv = nvs[0];
        if (nv < 2) { s = fail(LT_EINVAL, "lt_mlp_train: fewer than 2 valid training rays"); break; }
        for (int q = 0; q < 6; ++q) {
            const double mean = hs[q] / nv;
            const double var = hs[6 + q] / nv - mean * mean;
            m->t_mean[q] = mean;
            m->t_std[q] = var > 1e-24 ? std::sqrt(var) : 1.0;
            m->stats.t_mean[q] = m->t_mean[q];
            m->stats.t_std[q] = m->t_std[q];
        }
        set_frame(m);
        m->stats.n_train = n;
        m->stats.n_valid = nv;
        m->stats.n_valid_uniform = nvs[1];
        TrainBatch tr{X, T, lab, vlist, nv, o->seed, 0, o->reg_batch, 0};
        if (o->reg_steps > 0 &&
            (s = train_net<true>(m, m->reg, tr, o->reg_steps, o->lr, o->lr_decay, o->decay_every,
                                 &m->stats.reg_loss, st)) != LT_OK)
            break;
        if (o->ft_steps > 0) {
            TrainBatch ft{X, T, lab, vlist, nv, o->seed ^ 0x5bd1e995ull, 0, o->ft_batch, 0};
            if ((s = train_net<true>(m, m->reg, ft, o->ft_steps, o->ft_lr, o->lr_decay, o->decay_every,
                                     &m->stats.reg_loss, st)) != LT_OK)
                break;
        }
        // classifier: batches drawn from all n rays
        TrainBatch tc{X, T, lab, nullptr, n, o->seed ^ 0x9e3779b97f4a7c15ull, 0, o->cls_batch, 0};
        if (o->cls_steps > 0 &&
            (s = train_net<false>(m, m->cls, tc, o->cls_steps, o->lr, o->lr_decay, o->decay_every,
                                  &m->stats.cls_loss, st)) != LT_OK)
            break;
        // valid-region samples after a uniform prefix: shift the classifier's
        // prior back to that of uniform draws (odds divided by k)
        if (nu < n && o->cls_steps > 0) {
            const double k = 1.0 + (double)(nv - nvs[1]) / (double)std::max<uint32_t>(nvs[1], 1u);
            const int bo = Net<false>::boff(Net<false>::L - 1);
            float b = 0.f;
            if (cudaMemcpyAsync(&b, m->cls + bo, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                s = fail(LT_ECUDA, "lt_mlp_train: classifier bias read-back");
                break;
            }
            m->stats.cls_prior_shift = std::log(k);
            b = (float)((double)b - m->stats.cls_prior_shift);
            if (cudaMemcpy(m->cls + bo, &b, 4, cudaMemcpyHostToDevice) != cudaSuccess) {
                s = fail(LT_ECUDA, "lt_mlp_train: classifier bias update");
                break;
            }
        }
    } while (0);
    if (X) cudaFree(X);
    if (T) cudaFree(T);
    if (lab) cudaFree(lab);
    if (vlist) cudaFree(vlist);
    if (vcount) cudaFree(vcount);
    if (bc) cudaFree(bc);
    if (sums) cudaFree(sums);
    if (s != LT_OK) { delete m; return s; }
    m->frags_stale = true;
    m->stats.train_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = m;
    return LT_OK;
}

lt_status lt_mlp_query(const lt_mlp* mc, const lt_rays_in* in, const float* lam, const lt_rays_out* out,
                       size_t n, int32_t precision, lt_stream stream)
{
    clear_error();
    lt_mlp* m = const_cast<lt_mlp*>(mc);
    if (!m) return fail(LT_EINVAL, "lt_mlp_query: NULL map");
    lt_status s = check_io(in, lam, out, n, "lt_mlp_query");
    if (s != LT_OK || n == 0) return s;
    if (n >= (1ull << 31)) return fail(LT_EINVAL, "lt_mlp_query: n must be < 2^31");
    cudaStream_t st = (cudaStream_t)stream;
    RaysInDev din{in->x, in->y, in->dx, in->dy, in->dz, lam};
    RaysOutDev dout{out->x, out->y, out->dx, out->dy, out->dz, out->I, out->flags};
    MlpDev D{m->F, m->reg, m->cls};
    const uint32_t nn = (uint32_t)n;
    if (precision == LT_MLP_F32 || precision == LT_MLP_F32_NOCLS) {
        ProfScope prof("mlp_query_f32_kernel", st);
        const unsigned g = (nn + kMB - 1) / kMB;
        if (precision == LT_MLP_F32) mlp_query_f32_kernel<true><<<g, kMB, 0, st>>>(D, din, dout, nn);
        else mlp_query_f32_kernel<false><<<g, kMB, 0, st>>>(D, din, dout, nn);
    } else if (precision == LT_MLP_BF16 || precision == LT_MLP_F16) {
        if (m->frags_stale && (s = build_tc_image(m)) != LT_OK) return s;
        const bool bf = precision == LT_MLP_BF16;
        // more than half of an SM's shared memory: one CTA (and one TMEM
        // allocation of all 512 columns) per SM
        const size_t smem = std::max(sizeof(TcShared) + 16, (size_t)116 * 1024);
        const void* k = bf ? (const void*)mlp_query_tc_kernel<true> : (const void*)mlp_query_tc_kernel<false>;
        LT_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const unsigned per_cta = 128 * kTcWG;
        const unsigned g = std::min<unsigned>((unsigned)sms, (nn + per_cta - 1) / per_cta);
        ProfScope prof(bf ? "mlp_query_bf16_kernel" : "mlp_query_f16_kernel", st);
        if (bf) mlp_query_tc_kernel<true><<<g, kTcThreads, smem, st>>>(m->F, m->tc_bias, m->tc_bf16, din, dout, nn, m->tc_err);
        else mlp_query_tc_kernel<false><<<g, kTcThreads, smem, st>>>(m->F, m->tc_bias, m->tc_f16, din, dout, nn, m->tc_err);
    } else {
        return fail(LT_EINVAL, "lt_mlp_query: unknown precision %d", precision);
    }
    LT_CUDA_TRY(cudaGetLastError());
    return LT_OK;
}

lt_status lt_mlp_grad(const lt_mlp* m, int32_t net, const float* X, const float* targets, int32_t B,
                      double* grad, double* loss)
{
    clear_error();
    if (!m || !X || !targets || !grad || B < 1) return fail(LT_EINVAL, "lt_mlp_grad: bad argument");
    if (net != 0 && net != 1) return fail(LT_EINVAL, "lt_mlp_grad: net must be 0 or 1");
    lt_status s = set_train_attrs();
    if (s != LT_OK) return s;
    const int blocks = (B + kTB - 1) / kTB;
    const int np = net == 0 ? LT_MLP_REG_PARAMS : LT_MLP_CLS_PARAMS;
    float* G = nullptr;
    double* lb = nullptr;
    if (cudaMalloc(&G, (size_t)blocks * np * 4) != cudaSuccess || cudaMalloc(&lb, (size_t)blocks * 8) != cudaSuccess) {
        if (G) cudaFree(G);
        return fail(LT_ENOMEM, "lt_mlp_grad: buffers");
    }
    TrainBatch tb{X, net == 0 ? targets : nullptr, net == 1 ? targets : nullptr, nullptr, 0, 0, 0, B, 1};
    if (net == 0) s = train_step<true>(m->reg, tb, m->F, G, lb, nullptr, nullptr, 0.0, 0, 0);
    else s = train_step<false>(m->cls, tb, m->F, G, lb, nullptr, nullptr, 0.0, 0, 0);
    std::vector<float> hg((size_t)blocks * np);
    std::vector<double> hl(blocks);
    if (s == LT_OK && (cudaMemcpy(hg.data(), G, hg.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
                       cudaMemcpy(hl.data(), lb, hl.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess))
        s = fail(LT_ECUDA, "lt_mlp_grad: read-back");
    cudaFree(G);
    cudaFree(lb);
    if (s != LT_OK) return s;
    for (int p = 0; p < np; ++p) {
        double g = 0.0;
        for (int b = 0; b < blocks; ++b) g += hg[(size_t)b * np + p];
        grad[p] = g;
    }
    if (loss) {
        double l = 0.0;
        for (double v : hl) l += v;
        *loss = l / B;
    }
    return LT_OK;
}

lt_status lt_mlp_features(const lt_mlp* m, const lt_rays_in* in, const float* lam, float* X, size_t n,
                          lt_stream stream)
{
    clear_error();
    if (!m || !in || !X) return fail(LT_EINVAL, "lt_mlp_features: NULL argument");
    if (n == 0) return LT_OK;
    RaysInDev din{in->x, in->y, in->dx, in->dy, in->dz, lam};
    mlp_features_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(m->F, din, X, (uint32_t)n);
    LT_CUDA_TRY(cudaGetLastError());
    return LT_OK;
}

}  // extern "C"
