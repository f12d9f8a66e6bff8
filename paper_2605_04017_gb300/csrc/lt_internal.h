// Internal declarations of liblt (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/lt.h"

namespace lt {

// Error reporting: a thread-local message per failing call.
lt_status fail(lt_status code, const char* fmt, ...);
lt_status cuda_fail(cudaError_t e, const char* what);
void clear_error();

#define LT_CUDA_TRY(expr)                                       \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return ::lt::cuda_fail(_e, #expr); \
    } while (0)

constexpr int kMaxS = LT_MAX_SURFACES;
constexpr int kMaxG = LT_MAX_GLASSES;

// One surface as the tracer reads it (64 bytes): both neighbouring media are
// resolved, so an interaction evaluates one dispersion formula.
struct __align__(16) SurfRec {
    float c, th_before, th_after, ap2;          // curvature, vertex gaps to s-1 and s+1, aperture^2
    float eps2a, A_before, B_before, A_after;   // near-edge band on r^2; Cauchy (A, B) of media s-1, s
    float B_after, g_before, g_after, kc;       // glass ids of media s-1, s (as float; -1 air); conic
    float a4, a6, a8, a10;                      // even-asphere polynomial (all zero with kc: a sphere)
};

// The lens as the kernels see it: FP32, passed by value as a __grid_constant__
// kernel parameter (about 2.7 KB, read through the constant cache; the lanes
// of a warp read the same surface at the same time).
//
// Axial positions are kept relative to the vertex the ray last met, so the
// FP32 z of a ray stays within a few mm of zero: vertex 0 is the entrance
// plane z = 0, vertex k (1..S) the vertex of surface k; s[k].th_before is the
// gap from vertex k-1 to k and s[k].th_after the gap from k to k+1.
struct LensDev {
    int S;                  // optical surfaces
    int stop_gap;           // stop in gap g (between vertex g and g+1; g = S: behind the last surface); -1 none
    float zs_lo, zs_hi;     // stop plane z relative to vertex g and to vertex g+1
    float a_stop2;          // stop radius squared
    float eps2a_stop;       // near-edge band on r^2: 2 * a * eps
    float z_img_rel;        // image plane z relative to vertex S
    float grazing_k;        // k below which a refraction is flagged ill-conditioned
    SurfRec s[kMaxS + 1];   // surfaces 1..S
    int8_t med[kMaxS + 2];  // glass of medium m (0..S); -1 = air
    int8_t gkind[kMaxG];
    float gA[kMaxG], gB[kMaxG];
    float gSB[kMaxG][3], gSC[kMaxG][3];
};

}  // namespace lt

struct lt_lens {
    int S;
    int n_glass;
    lt_surface surf[LT_MAX_SURFACES];
    lt_glass glass[LT_MAX_GLASSES];
    lt_prescription presc;          // arrays pointing at surf/glass above
    double zv[LT_MAX_SURFACES + 1]; // FP64 vertex z (index 0 = entrance plane)
    double z_stop;
    double z_image;
    lt::LensDev dev;
};

namespace lt {
// The profiler's work counters (profile.cpp): record r's count is the sum of
// kProfShards 64-bit counters at r + s * kProfMaxRecs, so that the kernels'
// per-warp additions spread over that many L2 lines instead of one address.
constexpr size_t kProfMaxRecs = 1 << 16;
constexpr int kProfShards = 8;
// Host FP64 paraxial ABCD data of a lens (defined in lens.cpp).
int paraxial(const lt_lens* L, double lambda_nm, double* efl, double* bfd);
bool path_ij(int S, int path_id, int* i, int* j);
bool aligned16(const void* p);
}  // namespace lt
