// The valid-region sampler of Sec. 5.1 (data collection): Markov chains over
// the 5-D entrance-ray box (x, y, s_x, s_y, lambda) whose target is the
// binary visibility of a path -- for most ghost paths only a small fraction
// of the box gives valid rays, so uniform fitting data would be sparse.
//
// One thread runs one chain: it starts at the first valid independent
// uniform draw (at most init_tries), then each step proposes, with
// probability p_large, an independent uniform point of the box, else a
// uniform point of the box of half-width small * (hi - lo) around the state,
// and moves iff the proposal lies in the box and its ray is valid (the
// Metropolis rule for a binary target with symmetric proposals: the chain's
// stationary law is uniform over the valid region).  A proposal's validity
// is the exact FP32 tracer's (trace_ray).  Random numbers are counter-based:
// u(chain, i, k) = top 24 bits of SplitMix64(seed + (chain << 32 | i << 3 |
// k)) * 2^-24 (i: init try t, or init_tries + step; k: 0 the step kind,
// 1..5 the dimensions), and every proposal is computed with one rounding per
// operation, so the chains are a pure function of the options.
#include "profile.h"
#include "rays.cuh"
#include "tracer.cuh"

namespace lt {

constexpr int kMcmcBlock = 128;

struct McmcDev {
    float lo[5], hi[5], w[5], h[5];
    float p_large;
    uint64_t seed;
    uint32_t chains, steps, init_tries;
};

struct SamplesDev {
    float *x, *y, *dx, *dy, *dz, *lam;
    uint8_t* flags;
    uint32_t* accepted;
};

// SplitMix64 (Steele, Lea and Flood, 2014): the mix of z + 0x9E3779B97F4A7C15.
__device__ __forceinline__ uint64_t mcmc_mix(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float mcmc_uniform(uint64_t seed, uint32_t chain, uint32_t i, uint32_t k)
{
    const uint64_t h = mcmc_mix(seed + (((uint64_t)chain << 32) | ((uint64_t)i << 3) | k));
    return __fmul_rn(__uint2float_rn((uint32_t)(h >> 40)), 5.9604644775390625e-8f);   // * 2^-24, exact
}

// entrance ray of a state: direction normalize(s_x, s_y, 1), one rounding per operation
__device__ __forceinline__ void state_ray(const float u[5], float& x, float& y, float& dx, float& dy, float& dz,
                                          float& lam)
{
    const float a = __fmul_rn(u[2], u[2]);
    const float b = __fmul_rn(u[3], u[3]);
    const float ln = __fsqrt_rn(__fadd_rn(__fadd_rn(a, b), 1.0f));
    x = u[0];
    y = u[1];
    dx = __fdiv_rn(u[2], ln);
    dy = __fdiv_rn(u[3], ln);
    dz = __fdiv_rn(1.0f, ln);
    lam = u[4];
}

template <bool CAUCHY>
__device__ __forceinline__ bool state_valid(const LensDev& L, int pi, int pj, const float u[5], int& nint)
{
    float x, y, dx, dy, dz, lam;
    state_ray(u, x, y, dx, dy, dz, lam);
    TraceOut o;
    int k = 0;
    const uint32_t f = trace_ray<CAUCHY>(L, pi, pj, x, y, dx, dy, dz, lam, o, k);
    nint += k;
    return (f & LT_FLAG_VALID) != 0;
}

template <bool CAUCHY>
__global__ void __launch_bounds__(kMcmcBlock)
mcmc_kernel(const __grid_constant__ LensDev L, int pi, int pj, const __grid_constant__ McmcDev P, SamplesDev out,
            unsigned long long* work)
{
    const uint32_t c = blockIdx.x * kMcmcBlock + threadIdx.x;
    if (c >= P.chains) return;
    float u[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    bool started = false;
    int nint = 0;
#pragma unroll 1
    for (uint32_t t = 0; t < P.init_tries && !started; ++t) {
        float v[5];
#pragma unroll
        for (int d = 0; d < 5; ++d) v[d] = __fadd_rn(P.lo[d], __fmul_rn(mcmc_uniform(P.seed, c, t, 1 + d), P.w[d]));
        if (state_valid<CAUCHY>(L, pi, pj, v, nint)) {
#pragma unroll
            for (int d = 0; d < 5; ++d) u[d] = v[d];
            started = true;
        }
    }
    uint32_t acc = 0;
#pragma unroll 1
    for (uint32_t s = 0; s < P.steps; ++s) {
        if (started) {
            const uint32_t i = P.init_tries + s;
            const bool large = mcmc_uniform(P.seed, c, i, 0) < P.p_large;
            float v[5];
            bool inside = true;
#pragma unroll
            for (int d = 0; d < 5; ++d) {
                const float xi = mcmc_uniform(P.seed, c, i, 1 + d);
                v[d] = large ? __fadd_rn(P.lo[d], __fmul_rn(xi, P.w[d]))
                             : __fadd_rn(u[d], __fmul_rn(__fsub_rn(__fmul_rn(2.0f, xi), 1.0f), P.h[d]));
                inside &= (v[d] >= P.lo[d]) & (v[d] <= P.hi[d]);
            }
            if (inside && state_valid<CAUCHY>(L, pi, pj, v, nint)) {
#pragma unroll
                for (int d = 0; d < 5; ++d) u[d] = v[d];
                ++acc;
            }
        }
        float x, y, dx, dy, dz, lam;
        state_ray(u, x, y, dx, dy, dz, lam);
        const size_t e = (size_t)s * P.chains + c;
        __stcs(out.x + e, started ? x : 0.0f);
        __stcs(out.y + e, started ? y : 0.0f);
        __stcs(out.dx + e, started ? dx : 0.0f);
        __stcs(out.dy + e, started ? dy : 0.0f);
        __stcs(out.dz + e, started ? dz : 0.0f);
        __stcs(out.lam + e, started ? lam : 0.0f);
        out.flags[e] = started ? (uint8_t)LT_FLAG_VALID : (uint8_t)0;
    }
    if (out.accepted) out.accepted[c] = acc;
    warp_add(work, (unsigned)nint);
}

}  // namespace lt

using namespace lt;

extern "C" lt_status lt_mcmc_sample(const lt_lens* L, const lt_mcmc_opts* o, const lt_samples_out* out,
                                    lt_stream stream)
{
    clear_error();
    if (!L || !o || !out) return fail(LT_EINVAL, "lt_mcmc_sample: NULL argument");
    int pi, pj;
    if (!path_ij(L->S, o->path_id, &pi, &pj)) return fail(LT_EINVAL, "lt_mcmc_sample: bad path id %d", o->path_id);
    if (o->chains < 0 || o->steps < 0 || o->init_tries < 1)
        return fail(LT_EINVAL, "lt_mcmc_sample: chains and steps must be >= 0 and init_tries >= 1");
    if ((uint64_t)o->chains * (uint64_t)o->steps >= (1ull << 32))
        return fail(LT_EINVAL, "lt_mcmc_sample: chains x steps must be < 2^32");
    if ((uint64_t)o->init_tries + (uint64_t)o->steps >= (1ull << 29))
        return fail(LT_EINVAL, "lt_mcmc_sample: init_tries + steps must be < 2^29");
    if (!(o->small >= 0.0) || !(o->p_large >= 0.0 && o->p_large <= 1.0))
        return fail(LT_EINVAL, "lt_mcmc_sample: small must be >= 0 and p_large in [0, 1]");
    McmcDev P{};
    for (int d = 0; d < 5; ++d) {
        if (!(o->hi[d] > o->lo[d])) return fail(LT_EINVAL, "lt_mcmc_sample: empty box on axis %d", d);
        P.lo[d] = (float)o->lo[d];
        P.hi[d] = (float)o->hi[d];
        P.w[d] = (float)(o->hi[d] - o->lo[d]);
        P.h[d] = (float)o->small * P.w[d];   // one FP32 rounding, as the chain arithmetic
    }
    P.p_large = (float)o->p_large;
    P.seed = o->seed;
    P.chains = (uint32_t)o->chains;
    P.steps = (uint32_t)o->steps;
    P.init_tries = (uint32_t)o->init_tries;
    if (o->chains == 0 || o->steps == 0) return LT_OK;
    const void* ps[] = {out->x, out->y, out->dx, out->dy, out->dz, out->lambda_nm};
    for (const void* q : ps)
        if (!q || !aligned16(q)) return fail(LT_EINVAL, "lt_mcmc_sample: sample arrays must be non-NULL and 16-byte aligned");
    if (!out->flags) return fail(LT_EINVAL, "lt_mcmc_sample: NULL flags array");
    SamplesDev S{out->x, out->y, out->dx, out->dy, out->dz, out->lambda_nm, out->flags, out->accepted};
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned g = (unsigned)(((size_t)o->chains + kMcmcBlock - 1) / kMcmcBlock);
    ProfScope prof("mcmc_kernel", st);
    if (lens_all_cauchy(L->dev)) mcmc_kernel<true><<<g, kMcmcBlock, 0, st>>>(L->dev, pi, pj, P, S, prof.work());
    else mcmc_kernel<false><<<g, kMcmcBlock, 0, st>>>(L->dev, pi, pj, P, S, prof.work());
    LT_CUDA_TRY(cudaGetLastError());
    return LT_OK;
}
