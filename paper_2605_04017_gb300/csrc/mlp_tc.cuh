// Learned-map query on the 5th-generation tensor cores (tcgen05, TMEM).
//
// One CTA of eight warpgroups per SM (1,024 threads), each with one 128-ray
// tile in flight (a slot): while the tensor core runs one warpgroup's layer,
// the other warpgroups run their epilogues, so the MMA latency hides behind
// them.  The epilogues are the critical path, so the CTA takes as many warps
// as the register file and TMEM allow (64 registers a thread, 8 x 64 TMEM
// columns); the code also runs with several slots per warpgroup, which
// alternate within it (4 x 2 and 2 x 4 were measured slower).  Per slot:
//   TMEM cols 0..63 of the slot: accumulators D (layer 0: regressor 0..31,
//     classifier 32..63; later layers the same split)
//   shared memory: the A operand of the regressor's next layer (K = 32,
//     8 KB) and of the classifier's next layer (8 KB; before layer 0 it holds
//     the 4 features, K = 16), BF16 or FP16 in the canonical K-major layout.
// Thread i of the warpgroup owns ray i of each tile = TMEM lane i.  A layer:
// one elected thread issues tcgen05.mma (M = 128, K = 16 per instruction,
// A and B from shared memory) and commits to the slot's mbarrier; every
// thread waits (bounded, suspended in hardware), reads its row of D with
// tcgen05.ld, adds the FP32 bias (an immediate constant-bank operand),
// applies tanh.approx on packed pairs and stores its row of the next A.
// Six layers per tile: regressor layers 0..5, with the classifier's layers
// riding in layers 0..2.
//
// Operands sit in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, the two core matrices of a 16-wide
// K slice 128 bytes apart (leading byte offset), 8-row groups 256 bytes
// apart (stride byte offset).  Output layers are padded to N = 32.

namespace lt {

constexpr int kTcWG = 8;                    // warpgroups per CTA
constexpr int kTcThreads = 128 * kTcWG;
constexpr int kTcCols = 512;                // TMEM columns allocated per CTA (64 per slot)
constexpr int kTcSlots = 1;                 // tiles in flight per warpgroup
constexpr int kAbytes = 8192;               // one A operand: 128 rows x 32 x 16 bits
constexpr uint32_t kTcWaitPolls = 1u << 17; // bounded mbarrier wait (x up to 1 us each)

// byte offsets of the weight image (one 16-bit element per weight)
constexpr int kImgB0 = 0;                   // N = 64 (reg 0..31, cls 32..63), K = 16
constexpr int kLayerBytes = 2048;           // N = 32, K = 32 (2 slices of 1 KB)
constexpr int kImgR1 = 2048;                // regressor layers 1..4
constexpr int kImgR5 = kImgR1 + 4 * kLayerBytes;  // regressor output (6 of 32 rows used)
constexpr int kImgC1 = kImgR5 + kLayerBytes;      // classifier layer 1
constexpr int kImgC2 = kImgC1 + kLayerBytes;      // classifier output (1 of 32 rows used)
constexpr int kImgBytes = kImgC2 + kLayerBytes;   // 16,384 bytes
// FP32 biases, a kernel parameter (read through the constant bank): reg
// layers 0..4 (32 each), reg out (32), cls layers 0..1 (32 each), cls out (32)
constexpr int kBiasReg = 0, kBiasRegOut = 5 * 32, kBiasCls = 6 * 32, kBiasClsOut = 8 * 32;
struct TcBias {
    float b[9 * 32];
};

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

// D (TMEM) (+)= A (shared-memory descriptor) x B (shared-memory descriptor)
__device__ __forceinline__ void tc_mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
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

// bounded wait for phase `parity` of an mbarrier; false if it never came.
// try_wait suspends the thread in hardware (up to the hint, in ns) instead of
// spinning, so waiting warps take no issue slots.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (uint32_t i = 0; i < kTcWaitPolls; ++i) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done) : "r"(mbar), "r"(parity), "r"(1000u) : "memory");
        if (done) return true;
    }
    return false;
}

// tcgen05.ld and its wait in one statement: the registers are valid when it
// returns, and the compiler cannot schedule a use before the wait
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                   "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                   "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                   "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                   "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr) : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                   "=r"(v[7])
                 : "r"(taddr) : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// byte offset of row m, 8-element chunk c (k = 8c .. 8c + 7) of an A operand
// with M = 128 rows in the canonical K-major layout (16-wide K slices of 4 KB)
__device__ __forceinline__ uint32_t a_chunk_offset(int m, int c)
{
    return (uint32_t)((c >> 1) * 4096 + (m >> 3) * 256 + (c & 1) * 128 + (m & 7) * 16);
}

// D row (32 FP32 columns) + bias -> tanh -> this thread's row of the next A
template <bool BF16>
__device__ __forceinline__ void tc_hidden(uint32_t dcol, unsigned char* abuf, int m, const float* bias)
{
    uint32_t v[32];
    tmem_ld32(dcol, v);
    uint32_t a[16];
#pragma unroll
    for (int j = 0; j < 16; ++j)
        a[j] = tanh2<BF16>(__uint_as_float(v[2 * j]) + bias[2 * j], __uint_as_float(v[2 * j + 1]) + bias[2 * j + 1]);
#pragma unroll
    for (int c = 0; c < 4; ++c)
        *reinterpret_cast<uint4*>(abuf + a_chunk_offset(m, c)) = make_uint4(a[4 * c], a[4 * c + 1], a[4 * c + 2], a[4 * c + 3]);
}

// Per-CTA state in shared memory: the weight image, the A operands of every
// slot, one mbarrier per slot and the TMEM base address.
struct TcShared {
    alignas(16) unsigned char img[kImgBytes];
    alignas(16) unsigned char areg[kTcWG][kTcSlots][kAbytes];
    alignas(16) unsigned char acls[kTcWG][kTcSlots][kAbytes];
    alignas(8) unsigned long long mbar[kTcWG][kTcSlots];
    uint32_t tmem;
    uint32_t abort[kTcWG];
};

// One slot's tile: its rays' reduced frames and the classifier's decision.
struct TcTile {
    RedFrame rf;
    bool ok, live;
    float logit;
    uint32_t r;
};

// The query of one CTA: CTA `cta` of `ncta` takes tiles (cta * kTcWG + g) *
// kTcSlots + {0 .. kTcSlots - 1} and every ncta * kTcWG * kTcSlots tiles
// after them.
// `bias` holds the TcBias words (a kernel parameter, or a shared-memory copy
// in the server's fused launch).
template <bool BF16>
__device__ __forceinline__ void tc_query_cta(TcShared& S, const MlpFrame& F, const float* __restrict__ bias,
                                             const unsigned char* __restrict__ gimg, const RaysInDev& in,
                                             const RaysOutDev& out, uint32_t n, uint32_t* __restrict__ err,
                                             uint32_t cta, uint32_t ncta)
{
    const int tid = threadIdx.x, warp = tid >> 5, g = warp >> 2, row = tid & 127;
    // weights and biases into shared memory
    for (int i = tid; i < kImgBytes / 16; i += kTcThreads)
        reinterpret_cast<uint4*>(S.img)[i] = __ldg(reinterpret_cast<const uint4*>(gimg) + i);
    if (tid < kTcWG * kTcSlots) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_u32(&S.mbar[tid / kTcSlots][tid % kTcSlots])) : "memory");
        if (tid < kTcWG) S.abort[tid] = 0;
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

    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;      // this warp's TMEM lanes
    const uint32_t img = smem_u32(S.img);
    const bool leader = row == 0;
    const uint32_t id64 = tc_idesc(BF16, 64), id32 = tc_idesc(BF16, 32);
    uint32_t cD[kTcSlots], mbar[kTcSlots], parity[kTcSlots], ar[kTcSlots], ac[kTcSlots];
#pragma unroll
    for (int sl = 0; sl < kTcSlots; ++sl) {
        cD[sl] = S.tmem + (uint32_t)((g * kTcSlots + sl) * 64);
        mbar[sl] = smem_u32(&S.mbar[g][sl]);
        parity[sl] = 0;
        ar[sl] = smem_u32(S.areg[g][sl]);
        ac[sl] = smem_u32(S.acls[g][sl]);
    }
    bool ok_wait = true;

    // layer `layer` of a slot's tile (issued by one elected thread)
    auto issue_layer = [&](int sl, int layer) {
        tc_fence_after();
        if (layer == 0) {
            tc_mma_ss(cD[sl], tc_desc(ac[sl], 128, 256), tc_desc(img + kImgB0, 128, 256), id64, 0u);
        } else {
            const int wr = layer < 5 ? kImgR1 + (layer - 1) * kLayerBytes : kImgR5;
#pragma unroll
            for (int k = 0; k < 2; ++k)
                tc_mma_ss(cD[sl], tc_desc(ar[sl] + 4096 * k, 128, 256), tc_desc(img + wr + 1024 * k, 128, 256), id32,
                          k ? 1u : 0u);
            if (layer <= 2) {
                const int wc = layer == 1 ? kImgC1 : kImgC2;
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    tc_mma_ss(cD[sl] + 32, tc_desc(ac[sl] + 4096 * k, 128, 256), tc_desc(img + wc + 1024 * k, 128, 256),
                              id32, k ? 1u : 0u);
            }
        }
        tc_commit(mbar[sl]);
    };

    const uint32_t tiles = (n + 127) / 128;
    const uint32_t tstep = ncta * kTcWG * kTcSlots;
    for (uint32_t t0 = (cta * kTcWG + g) * kTcSlots; t0 < tiles; t0 += tstep) {
        TcTile T[kTcSlots];
        // layer-0 A operands (features) of both slots, then both layer-0 MMAs
#pragma unroll
        for (int sl = 0; sl < kTcSlots; ++sl) {
            const uint32_t tile = t0 + sl;
            const uint32_t r = tile * 128 + row;
            T[sl].r = r;
            T[sl].live = tile < tiles && r < n;
            T[sl].logit = 0.f;
            float x = 0.f, y = 0.f, dx = 0.f, dy = 0.f, dz = 1.f, lam = 500.f;
            if (T[sl].live) {
                x = __ldg(in.x + r); y = __ldg(in.y + r);
                dx = __ldg(in.dx + r); dy = __ldg(in.dy + r); dz = __ldg(in.dz + r);
                lam = __ldg(in.lam + r);
            }
            T[sl].ok = T[sl].live && ray_ok(x, y, dx, dy, dz, lam);
            float X[4] = {0.f, 0.f, 0.f, 0.f};
            T[sl].rf = {1.f, 0.f, 1.f};
            if (T[sl].ok) mlp_features(F, x, y, dx, dy, dz, lam, X, T[sl].rf);
            unsigned char* a0 = S.acls[g][sl];
            *reinterpret_cast<uint4*>(a0 + a_chunk_offset(row, 0)) =
                make_uint4(pack2<BF16>(X[0], X[1]), pack2<BF16>(X[2], X[3]), 0u, 0u);
            *reinterpret_cast<uint4*>(a0 + a_chunk_offset(row, 1)) = make_uint4(0u, 0u, 0u, 0u);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        tc_fence_before();
        wg_sync(g);
        if (leader) {
#pragma unroll
            for (int sl = 0; sl < kTcSlots; ++sl) issue_layer(sl, 0);
        }
        float zr[kTcSlots][6];
#pragma unroll
        for (int layer = 0; layer < 6; ++layer) {
#pragma unroll
            for (int sl = 0; sl < kTcSlots; ++sl) {
                ok_wait &= mbar_wait(mbar[sl], parity[sl]);
                parity[sl] ^= 1u;
                tc_fence_after();
                if (layer < 5) {
                    tc_hidden<BF16>(lanes | cD[sl], S.areg[g][sl], row, bias + kBiasReg + 32 * layer);
                    if (layer <= 1) tc_hidden<BF16>(lanes | (cD[sl] + 32), S.acls[g][sl], row, bias + kBiasCls + 32 * layer);
                    if (layer == 2) {
                        uint32_t v[8];
                        tmem_ld8(lanes | (cD[sl] + 32), v);
                        T[sl].logit = __uint_as_float(v[0]) + bias[kBiasClsOut];
                    }
                    // this slot's next layer goes to the tensor core while the
                    // warpgroup finishes the other slot
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    tc_fence_before();
                    wg_sync(g);
                    if (leader) issue_layer(sl, layer + 1);
                } else {
                    uint32_t v[8];
                    tmem_ld8(lanes | cD[sl], v);
#pragma unroll
                    for (int q = 0; q < 6; ++q) zr[sl][q] = __uint_as_float(v[q]) + bias[kBiasRegOut + q];
                }
            }
        }
#pragma unroll
        for (int sl = 0; sl < kTcSlots; ++sl) {
            if (!T[sl].live) continue;
            const uint32_t r = T[sl].r;
            const bool valid = T[sl].ok && T[sl].logit > 0.0f;
            float o[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (valid) finish_ray(F, T[sl].rf, zr[sl], o);
            __stcs(out.x + r, o[0]);
            __stcs(out.y + r, o[1]);
            __stcs(out.dx + r, o[2]);
            __stcs(out.dy + r, o[3]);
            __stcs(out.dz + r, o[4]);
            __stcs(out.I + r, o[5]);
            out.flags[r] = (uint8_t)(!T[sl].ok ? LT_FLAG_BAD_INPUT : (valid ? LT_FLAG_VALID : 0u));
        }
        // a wait that ran out stops this warpgroup after these tiles (every
        // thread of the warpgroup sees the flag after the same barrier)
        if (!ok_wait) S.abort[g] = 1;
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

template <bool BF16>
__global__ void __launch_bounds__(kTcThreads, 1)
mlp_query_tc_kernel(const __grid_constant__ MlpFrame F, const __grid_constant__ TcBias B,
                    const unsigned char* __restrict__ gimg, RaysInDev in, RaysOutDev out, uint32_t n,
                    uint32_t* __restrict__ err)
{
    extern __shared__ __align__(16) unsigned char tc_smem_raw[];
    TcShared& S = *reinterpret_cast<TcShared*>(tc_smem_raw);
    tc_query_cta<BF16>(S, F, B.b, gimg, in, out, n, err, blockIdx.x, gridDim.x);
}

// The constants of one learned map for the server's fused launch (a device
// copy per map and precision): frame, biases, weight image, wait-error counter.
struct alignas(16) TcServe {
    MlpFrame F;
    TcBias B;
    const unsigned char* img;
    uint32_t* err;
};
constexpr size_t kTcServeAt = (sizeof(TcShared) + 15) & ~(size_t)15;   // its place after TcShared

// The server's fused launch of several small tensor-core learned-map queries:
// each CTA serves one request (kTcWG * kTcSlots tiles of it, one pass), with
// that request's frame and biases staged in shared memory after TcShared.
template <bool BF16>
__global__ void __launch_bounds__(kTcThreads, 1)
serve_mlp_tc_kernel(const __grid_constant__ ReqTable T)
{
    extern __shared__ __align__(16) unsigned char tc_smem_raw[];
    TcShared& S = *reinterpret_cast<TcShared*>(tc_smem_raw);
    TcServe& X = *reinterpret_cast<TcServe*>(tc_smem_raw + kTcServeAt);
    const int k = req_of_block(T, blockIdx.x);
    const ReqItem& it = T.item[k];
    stage_words(&X, it.dev, sizeof(TcServe));
    __syncthreads();
    tc_query_cta<BF16>(S, X.F, X.B.b, X.img, it.in, it.out, it.n, X.err, blockIdx.x - T.block0[k],
                       T.block0[k + 1] - T.block0[k]);
}

}  // namespace lt
