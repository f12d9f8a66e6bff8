// Learned-map query on the 5th-generation tensor cores (tcgen05, TMEM).
//
// One CTA of four warpgroups per SM; warpgroup g runs 128-ray tiles in a
// persistent loop inside its own 128 columns of the CTA's 512 TMEM columns:
//   cols  0..63  accumulators D (layer 0: regressor 0..31, classifier 32..63;
//                later layers: regressor 0..31, classifier 32..63)
//   cols 64..71  A operand of layer 0 (4 features + zero padding, K = 16)
//   cols 80..95  A operand of the regressor's next layer (K = 32)
//   cols 96..111 A operand of the classifier's next layer (K = 32)
// Thread i of the warpgroup owns ray i of the tile = TMEM lane i.  Each layer:
// one elected thread issues tcgen05.mma (M = 128, K = 16 per instruction,
// A from TMEM, B = weights in shared memory) and commits to the warpgroup's
// mbarrier; every thread waits (bounded), reads its row of D with
// tcgen05.ld, adds the FP32 bias, applies tanh.approx on packed pairs and
// writes the next A with tcgen05.st.  Six rounds per tile: regressor layers
// 0..5, with the classifier's layers riding in rounds 1..3.
//
// Weights sit in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, the two core matrices of a 16-wide
// K slice 128 bytes apart (leading byte offset), 8-row groups 256 bytes
// apart (stride byte offset).  Output layers are padded to N = 32.

namespace lt {

constexpr int kTcWG = 4;                    // warpgroups per CTA
constexpr int kTcThreads = 128 * kTcWG;
constexpr int kTcCols = 512;                // TMEM columns allocated per CTA
constexpr uint32_t kTcWaitPolls = 1u << 21; // bounded mbarrier wait

// byte offsets of the weight image (one 16-bit element per weight)
constexpr int kImgB0 = 0;                   // N = 64 (reg 0..31, cls 32..63), K = 16
constexpr int kImgR1 = 2048;                // regressor layers 1..4: N = 32, K = 32
constexpr int kImgR5 = kImgR1 + 4 * 2048;   // regressor output: N = 32 (6 used), K = 32
constexpr int kImgC1 = kImgR5 + 2048;       // classifier layer 1: N = 32, K = 32
constexpr int kImgC2 = kImgC1 + 2048;       // classifier output: N = 32 (1 used), K = 32
constexpr int kImgW = kImgC2 + 2048;        // 16,384 bytes of weights
// FP32 biases after the weights: reg layers 0..4 (32 each), reg out (32),
// cls layers 0..1 (32 each), cls out (32)
constexpr int kImgBias = kImgW;
constexpr int kImgBytes = kImgW + 9 * 32 * 4;
constexpr int kBiasReg = 0, kBiasRegOut = 5 * 32, kBiasCls = 6 * 32, kBiasClsOut = 8 * 32;

// byte offset of element (n, k) of a weight slice group with N rows and
// K = 16 * slices columns
__host__ __device__ constexpr int tc_elem_offset(int N, int n, int k)
{
    return (k / 16) * (N / 8) * 256 + (n / 8) * 256 + ((k % 16) / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading / stride byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulate, A and B of one type
// (BF16 or FP16), both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t tc_idesc(bool bf16, int n)
{
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
                 :: "r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 :: "r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void wg_sync(int g)
{
    asm volatile("bar.sync %0, 128;\n" :: "r"(g + 1) : "memory");
}

// bounded wait for phase `parity` of an mbarrier; false if it never came
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (uint32_t i = 0; i < kTcWaitPolls; ++i) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                   "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                   "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                   "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                   "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                   "=r"(v[7])
                 : "r"(taddr));
}

// tcgen05.ld writes its registers asynchronously: the wait takes them as
// read-write operands so no use can be scheduled before it
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
                   "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]),
                   "+r"(v[14]), "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]),
                   "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25]),
                   "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
                 :: "memory");
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[8])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
                   "+r"(v[7])
                 :: "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
                 "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};\n"
                 :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
                    "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]),
                    "r"(v[13]), "r"(v[14]), "r"(v[15])
                 : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n"
                 :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
                    "r"(v[6]), "r"(v[7])
                 : "memory");
}

// D row (32 FP32 columns) + bias -> tanh -> packed A row of the next layer
template <bool BF16>
__device__ __forceinline__ void tc_hidden(uint32_t dcol, uint32_t acol, const float* __restrict__ bias)
{
    uint32_t v[32];
    tmem_ld32(dcol, v);
    tmem_wait_ld(v);
    uint32_t a[16];
#pragma unroll
    for (int j = 0; j < 16; ++j)
        a[j] = tanh2<BF16>(__uint_as_float(v[2 * j]) + bias[2 * j], __uint_as_float(v[2 * j + 1]) + bias[2 * j + 1]);
    tmem_st16(acol, a);
}

// Per-CTA state in shared memory: the weight image, one mbarrier per
// warpgroup and the TMEM base address.
struct TcShared {
    alignas(16) unsigned char img[kImgBytes];
    alignas(8) unsigned long long mbar[kTcWG];
    uint32_t tmem;
    uint32_t abort[kTcWG];
};

template <bool BF16>
__global__ void __launch_bounds__(kTcThreads, 1)
mlp_query_tc_kernel(const __grid_constant__ MlpFrame F, const unsigned char* __restrict__ gimg,
                    RaysInDev in, RaysOutDev out, uint32_t n, uint32_t* __restrict__ err)
{
    extern __shared__ __align__(16) unsigned char tc_smem_raw[];
    TcShared& S = *reinterpret_cast<TcShared*>(tc_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, g = warp >> 2, row = tid & 127;
    // weights and biases into shared memory; made visible to the tensor cores
    for (int i = tid; i < kImgBytes / 16; i += kTcThreads)
        reinterpret_cast<uint4*>(S.img)[i] = __ldg(reinterpret_cast<const uint4*>(gimg) + i);
    if (tid < kTcWG) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_u32(&S.mbar[tid])) : "memory");
        S.abort[tid] = 0;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     :: "r"(smem_u32(&S.tmem)), "r"(kTcCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const uint32_t tbase = S.tmem + (uint32_t)(g * 128);           // this warpgroup's columns
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;      // this warp's TMEM lanes
    const uint32_t cD = tbase, cDc = tbase + 32, cAin = tbase + 64, cAr = tbase + 80, cAc = tbase + 96;
    const uint32_t mbar = smem_u32(&S.mbar[g]);
    const uint32_t img = smem_u32(S.img);
    const float* bias = reinterpret_cast<const float*>(S.img + kImgBias);
    const bool leader = row == 0;
    const uint32_t id64 = tc_idesc(BF16, 64), id32 = tc_idesc(BF16, 32);
    uint32_t parity = 0;
    bool ok_wait = true;

    const uint32_t tiles = (n + 127) / 128;
    for (uint32_t tile = blockIdx.x * kTcWG + g; tile < tiles; tile += gridDim.x * kTcWG) {
        const uint32_t r = tile * 128 + row;
        const bool live = r < n;
        float x = 0.f, y = 0.f, dx = 0.f, dy = 0.f, dz = 1.f, lam = 500.f;
        if (live) {
            x = __ldg(in.x + r); y = __ldg(in.y + r);
            dx = __ldg(in.dx + r); dy = __ldg(in.dy + r); dz = __ldg(in.dz + r);
            lam = __ldg(in.lam + r);
        }
        const bool ok = live && ray_ok(x, y, dx, dy, dz, lam);
        float X[4] = {0.f, 0.f, 0.f, 0.f};
        RedFrame rf = {1.f, 0.f, 1.f};
        if (ok) mlp_features(F, x, y, dx, dy, dz, lam, X, rf);
        {
            uint32_t a[8] = {pack2<BF16>(X[0], X[1]), pack2<BF16>(X[2], X[3]), 0u, 0u, 0u, 0u, 0u, 0u};
            tmem_st8(lanes | cAin, a);
        }
        float logit = 0.f, zr[6];
#pragma unroll 1
        for (int round = 0; round < 6; ++round) {
            tmem_wait_st();
            tc_fence_before();
            wg_sync(g);
            if (leader) {
                tc_fence_after();
                if (round == 0) {
                    tc_mma(cD, cAin, tc_desc(img + kImgB0, 128, 256), id64, 0u);
                } else {
                    const int wr = round < 5 ? kImgR1 + (round - 1) * 2048 : kImgR5;
                    tc_mma(cD, cAr, tc_desc(img + wr, 128, 256), id32, 0u);
                    tc_mma(cD, cAr + 8, tc_desc(img + wr + 1024, 128, 256), id32, 1u);
                    if (round <= 2) {
                        const int wc = round == 1 ? kImgC1 : kImgC2;
                        tc_mma(cDc, cAc, tc_desc(img + wc, 128, 256), id32, 0u);
                        tc_mma(cDc, cAc + 8, tc_desc(img + wc + 1024, 128, 256), id32, 1u);
                    }
                }
                tc_commit(mbar);
            }
            ok_wait &= mbar_wait(mbar, parity);
            parity ^= 1u;
            tc_fence_after();
            if (round < 4) {
                tc_hidden<BF16>(lanes | cD, lanes | cAr, bias + kBiasReg + 32 * round);
                if (round <= 1) tc_hidden<BF16>(lanes | cDc, lanes | cAc, bias + kBiasCls + 32 * round);
                if (round == 2) {
                    uint32_t v[8];
                    tmem_ld8(lanes | cDc, v);
                    tmem_wait_ld(v);
                    logit = __uint_as_float(v[0]) + bias[kBiasClsOut];
                }
            } else if (round == 4) {
                tc_hidden<BF16>(lanes | cD, lanes | cAr, bias + kBiasReg + 32 * 4);
            } else {
                uint32_t v[8];
                tmem_ld8(lanes | cD, v);
                tmem_wait_ld(v);
#pragma unroll
                for (int q = 0; q < 6; ++q) zr[q] = __uint_as_float(v[q]) + bias[kBiasRegOut + q];
            }
        }
        if (live) {
            const bool valid = ok && logit > 0.0f;
            float o[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (valid) finish_ray(F, rf, zr, o);
            __stcs(out.x + r, o[0]);
            __stcs(out.y + r, o[1]);
            __stcs(out.dx + r, o[2]);
            __stcs(out.dy + r, o[3]);
            __stcs(out.dz + r, o[4]);
            __stcs(out.I + r, o[5]);
            out.flags[r] = (uint8_t)(!ok ? LT_FLAG_BAD_INPUT : (valid ? LT_FLAG_VALID : 0u));
        }
        // a wait that ran out stops this warpgroup after the tile (every
        // thread of the warpgroup sees the flag after the same barrier)
        if (!ok_wait) S.abort[g] = 1;
        tmem_wait_st();
        tc_fence_before();
        wg_sync(g);
        if (S.abort[g]) break;
    }
    if (!ok_wait && row == 0) atomicAdd(err, 1u);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(S.tmem), "r"(kTcCols) : "memory");
}

}  // namespace lt
