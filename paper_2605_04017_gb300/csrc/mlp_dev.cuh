// Device code of the learned map shared by its translation units (mlp.cu:
// training, single queries; mlp_serve.cu: the server's fused queries): the
// network shapes, the symmetry-reduced input frame, the FP32 forward pass
// and the tensor-core query (mlp_tc.cuh).  Kernel templates defined here are
// compiled only in the unit that launches them.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "map_internal.h"
#include "rays.cuh"
#include "tracer.cuh"

namespace lt {

// ------------------------------------------------------------------ network shapes

template <bool REG>
struct Net {
    static constexpr int L = REG ? 6 : 3;
    static constexpr int NOUT = REG ? 6 : 1;
    __host__ __device__ static constexpr int in(int l) { return l == 0 ? 4 : 32; }
    __host__ __device__ static constexpr int out(int l) { return l == L - 1 ? NOUT : 32; }
    __host__ __device__ static constexpr int woff(int l)
    {
        int o = 0;
        for (int k = 0; k < l; ++k) o += out(k) * in(k) + out(k);
        return o;
    }
    __host__ __device__ static constexpr int boff(int l) { return woff(l) + out(l) * in(l); }
    static constexpr int NP = woff(L);
};
static_assert(Net<true>::NP == LT_MLP_REG_PARAMS, "regressor size");
static_assert(Net<false>::NP == LT_MLP_CLS_PARAMS, "classifier size");

// input normalisation and output de-standardisation, FP32
struct MlpFrame {
    float rho2_inv, winv, winv2, lam_lo, lam_scale;
    float t_mean[6], t_std[6];
};

struct RedFrame {
    float c, s, m;   // rotation cos/sin and mirror sign of the reduced frame
};

// Symmetry-reduced network input (Sec. 4.1): rotate the entrance point onto
// +x, mirror y when the rotated d_y < 0, normalise to [-1, 1].
__device__ __forceinline__ void mlp_features(const MlpFrame& F, float x, float y, float dx,
                                             float dy, float dz, float lam, float X[4],
                                             RedFrame& rf)
{
    const float r = sqrtf(fmaf(x, x, y * y));
    float c = 1.0f, s = 0.0f;
    if (r > 0.0f) {
        const float ir = 1.0f / r;
        c = x * ir;
        s = y * ir;
    }
    const float n2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float inv = rsqrtf(n2);
    inv = inv * fmaf(-0.5f * n2, inv * inv, 1.5f);
    dx *= inv;
    dy *= inv;
    const float dxr = fmaf(c, dx, s * dy);
    float dyr = fmaf(-s, dx, c * dy);
    const float m = dyr < 0.0f ? -1.0f : 1.0f;
    dyr *= m;
    X[0] = fmaf(r, F.rho2_inv, -1.0f);
    X[1] = dxr * F.winv;
    X[2] = fmaf(dyr, F.winv2, -1.0f);
    X[3] = fmaf(lam - F.lam_lo, F.lam_scale, -1.0f);
    rf = {c, s, m};
}

__device__ __forceinline__ void mlp_unreduce(const RedFrame& rf, const float red[6], float o[6])
{
    const float yr = red[1] * rf.m, dyr = red[3] * rf.m;
    o[0] = fmaf(rf.c, red[0], -rf.s * yr);
    o[1] = fmaf(rf.s, red[0], rf.c * yr);
    o[2] = fmaf(rf.c, red[2], -rf.s * dyr);
    o[3] = fmaf(rf.s, red[2], rf.c * dyr);
    o[4] = red[4];
    o[5] = red[5];
}

// Lambert's continued fraction tanh x = x / (1 + x^2 / (3 + x^2 / (5 + ...)))
// truncated at the 19 term: a 9/10 rational, clamped to +-1 for |x| >= 6.95
// (max |error| 1.8e-6 on the real line in FP64, 2.0e-6 evaluated in FP32).
// Coefficients normalised by the constant term.
__device__ __forceinline__ float tanh_rational(float x)
{
    const float ax = fabsf(x);
    if (ax >= 6.95f) return copysignf(1.0f, x);
    const float x2 = x * x;
    const float num = fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 8.400421197e-08f, 3.931397120e-05f),
                                             4.334365325e-03f), 1.403508772e-01f), 1.0f);
    const float den = fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 1.527349309e-09f, 2.268113723e-06f),
                                                       4.815961472e-04f), 2.889576883e-02f),
                                    4.736842105e-01f), 1.0f);
    return __fdividef(x * num, den);   // den >= 1: the fast division is within 2 ulp
}

// ------------------------------------------------------------------ training data

// ------------------------------------------------------------------ FP32 query

struct MlpDev {
    MlpFrame F;
    const float* reg;
    const float* cls;
};

template <bool REG>
__device__ __forceinline__ void forward_f32(const float* __restrict__ W, const float X[4],
                                            float z[Net<REG>::NOUT])
{
    using N = Net<REG>;
    float a[32];
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = X[k];
#pragma unroll
    for (int l = 0; l < N::L; ++l) {
        const int ni = N::in(l), no = N::out(l);
        const float4* Wl = reinterpret_cast<const float4*>(W + N::woff(l));   // rows of ni / 4 float4
        const float* bl = W + N::boff(l);
        float t[32];
#pragma unroll
        for (int o = 0; o < 32; ++o) {
            if (o < no) {
                float s = bl[o];
#pragma unroll
                for (int k4 = 0; k4 < 8; ++k4) {
                    if (4 * k4 < ni) {
                        const float4 w = Wl[o * (ni / 4) + k4];   // one shared-memory load, four FMAs
                        s = fmaf(w.x, a[4 * k4], s);
                        s = fmaf(w.y, a[4 * k4 + 1], s);
                        s = fmaf(w.z, a[4 * k4 + 2], s);
                        s = fmaf(w.w, a[4 * k4 + 3], s);
                    }
                }
                t[o] = s;
            }
        }
        if (l < N::L - 1) {
#pragma unroll
            for (int o = 0; o < 32; ++o) a[o] = tanh_rational(t[o]);
        } else {
#pragma unroll
            for (int o = 0; o < N::NOUT; ++o) z[o] = t[o];
        }
    }
}

__device__ __forceinline__ void finish_ray(const MlpFrame& F, const RedFrame& rf, const float zr[6],
                                           float o[6])
{
    float red[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) red[q] = fmaf(F.t_std[q], zr[q], F.t_mean[q]);
    const float n2 = fmaf(red[2], red[2], fmaf(red[3], red[3], red[4] * red[4]));
    float inv = n2 > 0.0f ? rsqrtf(n2) : 0.0f;
    inv = inv * fmaf(-0.5f * n2, inv * inv, 1.5f);
    red[2] *= inv;
    red[3] *= inv;
    red[4] *= inv;
    mlp_unreduce(rf, red, o);
}

__device__ __forceinline__ bool ray_ok(float x, float y, float dx, float dy, float dz, float lam)
{
    const bool finite = isfinite(x) & isfinite(y) & isfinite(dx) & isfinite(dy) & isfinite(dz) &
                        isfinite(lam);
    return finite && dz > 0.0f && lam > 0.0f;
}

constexpr int kMB = 128;

// The FP32 query of block `blk` of a batch (shared by mlp_query_f32_kernel
// and the server's fused launch, serve_mlp_f32_kernel).
template <bool USE_CLS>
__device__ __forceinline__ void f32_query_block(const MlpDev& D, const RaysInDev& in, const RaysOutDev& out,
                                                uint32_t n, uint32_t blk)
{
    // the classifier starts on a 16-byte boundary so both networks' weight
    // rows load as float4
    constexpr int kClsAt = (Net<true>::NP + 3) & ~3;
    __shared__ __align__(16) float W[kClsAt + Net<false>::NP];
    for (int i = threadIdx.x; i < Net<true>::NP; i += kMB) W[i] = D.reg[i];
    for (int i = threadIdx.x; i < Net<false>::NP; i += kMB) W[kClsAt + i] = D.cls[i];
    __syncthreads();
    const uint32_t r = blk * kMB + threadIdx.x;
    if (r >= n) return;
    const float x = __ldg(in.x + r), y = __ldg(in.y + r), dx = __ldg(in.dx + r),
                dy = __ldg(in.dy + r), dz = __ldg(in.dz + r), lam = __ldg(in.lam + r);
    float o[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    uint32_t f = 0;
    if (!ray_ok(x, y, dx, dy, dz, lam)) {
        f = LT_FLAG_BAD_INPUT;
    } else {
        float X[4];
        RedFrame rf;
        mlp_features(D.F, x, y, dx, dy, dz, lam, X, rf);
        bool valid = true;
        if (USE_CLS) {
            float logit[1];
            forward_f32<false>(W + kClsAt, X, logit);
            valid = logit[0] > 0.0f;
        }
        if (valid) {
            float zr[6];
            forward_f32<true>(W, X, zr);
            finish_ray(D.F, rf, zr, o);
            f = LT_FLAG_VALID;
        }
    }
    __stcs(out.x + r, o[0]);
    __stcs(out.y + r, o[1]);
    __stcs(out.dx + r, o[2]);
    __stcs(out.dy + r, o[3]);
    __stcs(out.dz + r, o[4]);
    __stcs(out.I + r, o[5]);
    out.flags[r] = (uint8_t)f;
}

template <bool USE_CLS>
__global__ void __launch_bounds__(kMB)
mlp_query_f32_kernel(const __grid_constant__ MlpDev D, RaysInDev in, RaysOutDev out, uint32_t n)
{
    f32_query_block<USE_CLS>(D, in, out, n, blockIdx.x);
}

// The server's fused launch of several small FP32 learned-map queries (each
// block serves one request): the block stages its request's MlpDev (a device
// copy) in shared memory, then its weights, and answers its rays.
template <bool USE_CLS>
__global__ void __launch_bounds__(kMB)
serve_mlp_f32_kernel(const __grid_constant__ ReqTable T)
{
    __shared__ MlpDev sd;
    const int k = req_of_block(T, blockIdx.x);
    const ReqItem& it = T.item[k];
    if (threadIdx.x == 0) sd = *static_cast<const MlpDev*>(it.dev);
    __syncthreads();
    f32_query_block<USE_CLS>(sd, it.in, it.out, it.n, blockIdx.x - T.block0[k]);
}

// ------------------------------------------------------------------ tensor-core query

template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    if (BF16) {
        __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&v);
    }
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// tanh of a packed pair, result packed (the next layer's A-operand word)
template <bool BF16>
__device__ __forceinline__ uint32_t tanh2(float lo, float hi)
{
    const uint32_t u = pack2<BF16>(lo, hi);
    uint32_t r;
    if (BF16)
        asm("tanh.approx.bf16x2 %0, %1;\n" : "=r"(r) : "r"(u));
    else
        asm("tanh.approx.f16x2 %0, %1;\n" : "=r"(r) : "r"(u));
    return r;
}
}  // namespace lt

#include "mlp_tc.cuh"
