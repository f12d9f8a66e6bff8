// The server's fused learned-map launches (lt_submit requests of one
// precision served by one grid, each block or CTA serving one request): kept
// in a translation unit of their own so that the tensor-core kernels compile
// in parallel with mlp.cu's.
#include <algorithm>

#include "mlp_dev.cuh"
#include "profile.h"

namespace lt {

uint32_t fused_mlp_rays(int precision)
{
    return precision == LT_MLP_BF16 || precision == LT_MLP_F16 ? (uint32_t)(128 * kTcWG * kTcSlots)
                                                                : (uint32_t)kMB;
}

lt_status launch_fused_mlp(const ReqTable& T, int precision, cudaStream_t st)
{
    if (T.n_items < 1 || T.n_items > kMaxFuse) return fail(LT_EINVAL, "fused query: %d requests", T.n_items);
    const unsigned blocks = T.block0[T.n_items];
    if (precision == LT_MLP_F32 || precision == LT_MLP_F32_NOCLS) {
        ProfScope prof("serve_mlp_f32_kernel", st);
        if (precision == LT_MLP_F32) serve_mlp_f32_kernel<true><<<blocks, kMB, 0, st>>>(T);
        else serve_mlp_f32_kernel<false><<<blocks, kMB, 0, st>>>(T);
    } else if (precision == LT_MLP_BF16 || precision == LT_MLP_F16) {
        const bool bf = precision == LT_MLP_BF16;
        // as the single query: more than half of an SM's shared memory, so
        // one CTA (and one TMEM allocation of all 512 columns) per SM
        const size_t smem = std::max(kTcServeAt + sizeof(TcServe) + 16, (size_t)116 * 1024);
        const void* k = bf ? (const void*)serve_mlp_tc_kernel<true> : (const void*)serve_mlp_tc_kernel<false>;
        LT_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ProfScope prof(bf ? "serve_mlp_bf16_kernel" : "serve_mlp_f16_kernel", st);
        if (bf) serve_mlp_tc_kernel<true><<<blocks, kTcThreads, smem, st>>>(T);
        else serve_mlp_tc_kernel<false><<<blocks, kTcThreads, smem, st>>>(T);
    } else {
        return fail(LT_EINVAL, "fused learned-map query: unknown precision %d", precision);
    }
    LT_CUDA_TRY(cudaGetLastError());
    return LT_OK;
}

}  // namespace lt
