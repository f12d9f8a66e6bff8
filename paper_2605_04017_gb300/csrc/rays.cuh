// Ray arrays as the kernels see them, argument checks and the pipelined
// host <-> device staging shared by the *_host entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "lt_internal.h"

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

lt_status check_io(const lt_rays_in* in, const float* lam, const lt_rays_out* out, size_t n,
                   const char* who);
lt_status launch_trace(const lt_lens* L, int pi, int pj, const RaysInDev& in,
                       const RaysOutDev& out, size_t n, cudaStream_t st);
// blocks for a persistent kernel: resident blocks per SM x SMs, capped by the work
unsigned persistent_blocks(const void* kernel, int block, size_t items, size_t per_warp);
// the library's stream-ordered memory pool of the current device (freed
// blocks are kept for reuse)
lt_status scratch_pool(cudaMemPool_t* pool);

// ---------------------------------------------------------------- host staging

// Pipelined host <-> device staging for the *_host entry points.  Chunk c
// uses buffer set c % kHostSets and passes through three library streams:
// copy-in, kernels, copy-out.  Events order each chunk's stages and keep a
// buffer set from being refilled before the chunk that last used it has been
// read or copied out.  With one stream per stage, every host-to-device copy
// waits only for a kernel of an older chunk, and every device-to-host copy
// only for its own chunk's kernel, so the two directions of the host link
// stay busy at the same time.
constexpr int kHostSets = 3;

struct Staging {
    int device = -1;
    size_t cap = 0;
    cudaStream_t s_in = nullptr, s_k = nullptr, s_out = nullptr;
    cudaEvent_t in_done[kHostSets] = {}, k_done[kHostSets] = {}, out_done[kHostSets] = {};
    // per buffer set: the six input arrays, then the six output arrays, then
    // the flags, one allocation, each array `cap` elements from the previous
    unsigned char* block[kHostSets] = {};
    float* in[kHostSets][6] = {};
    float* out[kHostSets][6] = {};
    uint8_t* flags[kHostSets] = {};
    std::mutex mu;

    void release()
    {
        for (int b = 0; b < kHostSets; ++b) {
            if (block[b]) cudaFree(block[b]);
            block[b] = nullptr;
            for (int q = 0; q < 6; ++q) in[b][q] = out[b][q] = nullptr;
            flags[b] = nullptr;
        }
        cap = 0;
    }

    lt_status reserve(size_t chunk)
    {
        int dev = 0;
        LT_CUDA_TRY(cudaGetDevice(&dev));
        if (dev != device) {
            // streams, events and buffers of another device are left to process exit
            s_in = s_k = s_out = nullptr;
            for (int b = 0; b < kHostSets; ++b) {
                in_done[b] = k_done[b] = out_done[b] = nullptr;
                block[b] = nullptr;
                for (int q = 0; q < 6; ++q) in[b][q] = out[b][q] = nullptr;
                flags[b] = nullptr;
            }
            cap = 0;
            device = dev;
        }
        cudaStream_t* ss[3] = {&s_in, &s_k, &s_out};
        for (cudaStream_t* p : ss)
            if (!*p) LT_CUDA_TRY(cudaStreamCreateWithFlags(p, cudaStreamNonBlocking));
        for (int b = 0; b < kHostSets; ++b) {
            cudaEvent_t* es[3] = {&in_done[b], &k_done[b], &out_done[b]};
            for (cudaEvent_t* e : es)
                if (!*e) LT_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        }
        if (chunk <= cap) return LT_OK;
        release();
        for (int b = 0; b < kHostSets; ++b) {
            if (cudaMalloc(&block[b], chunk * (12 * sizeof(float) + 1)) != cudaSuccess) {
                release();
                return fail(LT_ENOMEM, "host staging: cudaMalloc failed");
            }
            float* f = reinterpret_cast<float*>(block[b]);
            for (int q = 0; q < 6; ++q) {
                in[b][q] = f + q * chunk;
                out[b][q] = f + (6 + q) * chunk;
            }
            flags[b] = block[b] + 12 * sizeof(float) * chunk;
        }
        cap = chunk;
        return LT_OK;
    }
};


// Rays per chunk: about n / 8 (so the pipeline fills and drains in a small
// part of the call), between 2^16 and 2^20 rays, a multiple of 64 (which
// keeps every staged array 16-byte aligned).
inline size_t host_chunk(size_t n)
{
    size_t c = (n + 7) / 8;
    c = std::max<size_t>(c, 65536);
    c = std::min<size_t>(c, (size_t)1 << 20);
    return (c + 63) & ~(size_t)63;
}

// The byte distance between consecutive arrays of `a` when the six are
// equally spaced and at least `len` bytes apart (one strided copy then moves
// a chunk of all six); 0 otherwise.
inline size_t equal_pitch(const void* const a[6], size_t len)
{
    const char* p0 = static_cast<const char*>(a[0]);
    const ptrdiff_t d = static_cast<const char*>(a[1]) - p0;
    if (d < (ptrdiff_t)len || d >= ((ptrdiff_t)1 << 31)) return 0;   // a strided copy's pitch is below 2^31
    for (int q = 2; q < 6; ++q)
        if (static_cast<const char*>(a[q]) - p0 != d * q) return 0;
    return (size_t)d;
}

Staging& host_staging();

// Runs `launch(in, out, m, stream)` over host arrays in pipelined chunks:
// each chunk's inputs are copied to its device buffers, the kernels write its
// outputs to device buffers, and those are copied back.
template <class Launch>
lt_status host_chunks(Staging& S, const lt_rays_in* in, const float* lam, const lt_rays_out* out, size_t n,
                      size_t chunk, Launch&& launch)
{
    const float* hin[6] = {in->x, in->y, in->dx, in->dy, in->dz, lam};
    float* hout[6] = {out->x, out->y, out->dx, out->dy, out->dz, out->I};
    // host arrays laid out at equal distances (one allocation per direction):
    // one strided copy per direction and chunk instead of six
    const void* hi[6] = {hin[0], hin[1], hin[2], hin[3], hin[4], hin[5]};
    const void* ho[6] = {hout[0], hout[1], hout[2], hout[3], hout[4], hout[5]};
    const size_t pin = equal_pitch(hi, n * sizeof(float)), pout = equal_pitch(ho, n * sizeof(float));
    for (size_t off = 0, c = 0; off < n; off += chunk, ++c) {
        const int b = (int)(c % kHostSets);
        const size_t m = std::min(chunk, n - off);
        // buffer set b was last read by the kernel of chunk c - kHostSets
        if (c >= (size_t)kHostSets) LT_CUDA_TRY(cudaStreamWaitEvent(S.s_in, S.k_done[b], 0));
        if (pin)
            LT_CUDA_TRY(cudaMemcpy2DAsync(S.in[b][0], S.cap * sizeof(float), hin[0] + off, pin, m * sizeof(float), 6,
                                          cudaMemcpyHostToDevice, S.s_in));
        else
            for (int q = 0; q < 6; ++q)
                LT_CUDA_TRY(cudaMemcpyAsync(S.in[b][q], hin[q] + off, m * sizeof(float),
                                            cudaMemcpyHostToDevice, S.s_in));
        LT_CUDA_TRY(cudaEventRecord(S.in_done[b], S.s_in));
        LT_CUDA_TRY(cudaStreamWaitEvent(S.s_k, S.in_done[b], 0));
        // and its outputs were last copied out by chunk c - kHostSets
        if (c >= (size_t)kHostSets) LT_CUDA_TRY(cudaStreamWaitEvent(S.s_k, S.out_done[b], 0));
        RaysInDev din{S.in[b][0], S.in[b][1], S.in[b][2], S.in[b][3], S.in[b][4], S.in[b][5]};
        RaysOutDev dout{S.out[b][0], S.out[b][1], S.out[b][2], S.out[b][3], S.out[b][4], S.out[b][5],
                        S.flags[b]};
        const lt_status s = launch(din, dout, m, S.s_k);
        if (s != LT_OK) return s;
        LT_CUDA_TRY(cudaEventRecord(S.k_done[b], S.s_k));
        LT_CUDA_TRY(cudaStreamWaitEvent(S.s_out, S.k_done[b], 0));
        if (pout)
            LT_CUDA_TRY(cudaMemcpy2DAsync(hout[0] + off, pout, S.out[b][0], S.cap * sizeof(float), m * sizeof(float),
                                          6, cudaMemcpyDeviceToHost, S.s_out));
        else
            for (int q = 0; q < 6; ++q)
                LT_CUDA_TRY(cudaMemcpyAsync(hout[q] + off, S.out[b][q], m * sizeof(float),
                                            cudaMemcpyDeviceToHost, S.s_out));
        LT_CUDA_TRY(cudaMemcpyAsync(out->flags + off, S.flags[b], m, cudaMemcpyDeviceToHost, S.s_out));
        LT_CUDA_TRY(cudaEventRecord(S.out_done[b], S.s_out));
    }
    return LT_OK;
}

template <class Launch>
lt_status run_host_pipelined(const lt_rays_in* in, const float* lam, const lt_rays_out* out,
                             size_t n, Launch&& launch)
{
    std::lock_guard<std::mutex> lock(host_staging().mu);
    Staging& S = host_staging();
    const size_t chunk = host_chunk(n);
    lt_status s = S.reserve(chunk);
    if (s != LT_OK) return s;
    s = host_chunks(S, in, lam, out, n, chunk, launch);
    // on success and on failure alike, wait for every stage queued so far:
    // the caller's host arrays are in use until then
    const cudaStream_t streams[3] = {S.s_out, S.s_k, S.s_in};
    for (cudaStream_t q : streams) {
        const cudaError_t e = cudaStreamSynchronize(q);
        if (s == LT_OK && e != cudaSuccess) s = cuda_fail(e, "host pipeline: cudaStreamSynchronize");
    }
    return s;
}

}  // namespace lt
