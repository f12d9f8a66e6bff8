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

// Pipelined host <-> device staging for the *_host entry points: two streams,
// each with its own device buffers; chunk c goes to stream c % 2 so copies of
// one chunk overlap the kernel of the other.
struct Staging {
    int device = -1;
    size_t cap = 0;
    cudaStream_t st[2] = {nullptr, nullptr};
    float* in[2][6] = {};
    float* out[2][6] = {};
    uint8_t* flags[2] = {};
    std::mutex mu;

    void release()
    {
        for (int b = 0; b < 2; ++b) {
            for (int q = 0; q < 6; ++q) {
                if (in[b][q]) cudaFree(in[b][q]);
                if (out[b][q]) cudaFree(out[b][q]);
                in[b][q] = out[b][q] = nullptr;
            }
            if (flags[b]) cudaFree(flags[b]);
            flags[b] = nullptr;
        }
        cap = 0;
    }

    lt_status reserve(size_t chunk)
    {
        int dev = 0;
        LT_CUDA_TRY(cudaGetDevice(&dev));
        if (dev != device) {
            // buffers of another device are left to process exit
            for (int b = 0; b < 2; ++b) st[b] = nullptr;
            for (int b = 0; b < 2; ++b) {
                for (int q = 0; q < 6; ++q) in[b][q] = out[b][q] = nullptr;
                flags[b] = nullptr;
            }
            cap = 0;
            device = dev;
        }
        for (int b = 0; b < 2; ++b)
            if (!st[b]) LT_CUDA_TRY(cudaStreamCreateWithFlags(&st[b], cudaStreamNonBlocking));
        if (chunk <= cap) return LT_OK;
        release();
        for (int b = 0; b < 2; ++b) {
            for (int q = 0; q < 6; ++q) {
                if (cudaMalloc(&in[b][q], chunk * sizeof(float)) != cudaSuccess ||
                    cudaMalloc(&out[b][q], chunk * sizeof(float)) != cudaSuccess) {
                    release();
                    return fail(LT_ENOMEM, "host staging: cudaMalloc failed");
                }
            }
            if (cudaMalloc(&flags[b], chunk) != cudaSuccess) {
                release();
                return fail(LT_ENOMEM, "host staging: cudaMalloc failed");
            }
        }
        cap = chunk;
        return LT_OK;
    }
};


inline size_t host_chunk(size_t n)
{
    // at least 4 chunks for overlap, at most 2^21 rays (~100 MB staged per buffer set)
    size_t c = (n + 3) / 4;
    c = std::max<size_t>(c, 65536);
    c = std::min<size_t>(c, (size_t)1 << 21);
    return (c + 63) & ~(size_t)63;
}

Staging& host_staging();

// Runs `launch(in, out, m, stream)` over host arrays in pipelined chunks.
template <class Launch>
lt_status run_host_pipelined(const lt_rays_in* in, const float* lam, const lt_rays_out* out,
                             size_t n, Launch&& launch)
{
    std::lock_guard<std::mutex> lock(host_staging().mu);
    const size_t chunk = host_chunk(n);
    lt_status s = host_staging().reserve(chunk);
    if (s != LT_OK) return s;
    const float* hin[6] = {in->x, in->y, in->dx, in->dy, in->dz, lam};
    float* hout[6] = {out->x, out->y, out->dx, out->dy, out->dz, out->I};
    for (size_t off = 0, c = 0; off < n; off += chunk, ++c) {
        const int b = (int)(c & 1);
        cudaStream_t st = host_staging().st[b];
        const size_t m = std::min(chunk, n - off);
        for (int q = 0; q < 6; ++q)
            LT_CUDA_TRY(cudaMemcpyAsync(host_staging().in[b][q], hin[q] + off, m * sizeof(float),
                                        cudaMemcpyHostToDevice, st));
        RaysInDev din{host_staging().in[b][0], host_staging().in[b][1], host_staging().in[b][2],
                      host_staging().in[b][3], host_staging().in[b][4], host_staging().in[b][5]};
        RaysOutDev dout{host_staging().out[b][0], host_staging().out[b][1], host_staging().out[b][2],
                        host_staging().out[b][3], host_staging().out[b][4], host_staging().out[b][5],
                        host_staging().flags[b]};
        s = launch(din, dout, m, st);
        if (s != LT_OK) return s;
        for (int q = 0; q < 6; ++q)
            LT_CUDA_TRY(cudaMemcpyAsync(hout[q] + off, host_staging().out[b][q], m * sizeof(float),
                                        cudaMemcpyDeviceToHost, st));
        LT_CUDA_TRY(cudaMemcpyAsync(out->flags + off, host_staging().flags[b], m,
                                    cudaMemcpyDeviceToHost, st));
    }
    for (int b = 0; b < 2; ++b) LT_CUDA_TRY(cudaStreamSynchronize(host_staging().st[b]));
    return LT_OK;
}

}  // namespace lt
