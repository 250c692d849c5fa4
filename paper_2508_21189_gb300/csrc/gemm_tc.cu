// BF16 x BF16 -> FP32 GEMM on the fifth-generation tensor cores (tcgen05), both operands K-major:
//     D (M x N, column-major, ldd) = A (M x K) * B (N x K)^T
// the dense products of the randomized SVD (Alg. 1: Z = A^T Q, Y = A Z, B = Q^T A) with the
// rank r <= 512 as the N dimension.
//
// One CTA per 128-row tile of D (and per K split): 6 warps.
//   warp 0, one thread   TMA producer: per 64-wide K block, the 128 x 64 tile of A and the N x 64 tile of
//                        B (two boxes of N/2 rows) into one of 3 shared-memory stages (2 when N = 512; 128-byte swizzle),
//                        completion counted on the stage's `full` mbarrier
//   warp 1, one thread   MMA issuer: per K block, 4 K-steps of 16, each two tcgen05.mma (M = 128,
//                        N = N/2) into the TMEM accumulator (128 lanes x N FP32 columns); a tcgen05.commit
//                        on the stage's `empty` barrier frees it, a last one on `tmem_full` hands the
//                        accumulator to the epilogue.  Warp 1 also allocates and frees the TMEM.
//   warps 2-5            epilogue: tcgen05.ld of their 32 lanes (rows), 32 columns at a time, stored to
//                        D column by column (lanes = consecutive rows: coalesced).
// Every mbarrier wait is bounded; a wait that runs out records RSK_DEV_TIMEOUT, stops the roles, and
// before the CTA leaves the producer waits (bounded) for the copies still owed to a stage and the
// epilogue for the MMAs already issued, so no copy or MMA outlives the CTA's shared memory or TMEM.
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace {

constexpr int kBM = 128, kBK = 64, kThreads = 192;
// pipeline depth: 3 stages while they fit in 200 KB of shared memory, else 2
template <int NH>
constexpr int stages_for() {
    return 3 * (kBM * kBK * 2 + 2 * NH * kBK * 2) <= 200 * 1024 ? 3 : 2;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    // tcgen05 shared-memory matrix descriptor: K-major operand with the 128-byte swizzle: start address
    // (bits 0-13, >> 4), leading byte offset 1 (unused for swizzled K-major), stride byte offset 1024 B
    // between 8-row groups (bits 32-45, >> 4), descriptor version 1 (bits 46-47), swizzle mode 2 =
    // 128-byte (bits 61-63)
    uint64_t d = uint64_t((saddr & 0x3FFFFu) >> 4);
    d |= uint64_t(1) << 16;
    d |= uint64_t(1024 >> 4) << 32;
    d |= uint64_t(1) << 46;
    d |= uint64_t(2) << 61;
    return d;
}

// Instruction descriptor of tcgen05.mma.kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

__device__ __forceinline__ void tc_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(rskd::smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     rskd::smem_u32(bar))
                 : "memory");
}
// 32 lanes x 32 consecutive FP32 columns: thread t of the warp receives lane (base lane + t).
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct GemmArgs {
    int64_t M, K;
    int N;             // columns of D stored (<= 2 * NH)
    int kblocks;       // K blocks per split
    int64_t nk_total;  // K blocks overall
    float* D;
    int64_t ldd;
    int64_t split_stride;  // elements between the splits' partial outputs (0: one split)
    unsigned int* status;
};

template <int NH>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, const GemmArgs a) {
    constexpr int kStages = stages_for<NH>();
    constexpr int kABytes = kBM * kBK * 2;          // 16 KB
    constexpr int kBBytes = 2 * NH * kBK * 2;       // N x 64 BF16
    constexpr int kStage = kABytes + kBBytes;       // multiple of 1024
    constexpr uint32_t kTmemCols = (2 * NH <= 32) ? 32 : (2 * NH <= 64) ? 64 : (2 * NH <= 128) ? 128 : (2 * NH <= 256) ? 256 : 512;
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + kStages * kStage);
    uint64_t* empty = full + kStages;
    uint64_t* tfull = empty + kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tfull + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* consumed = abort_flag + 1;  // K blocks the MMA thread has waited for, per stage

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = int64_t(blockIdx.x) * kBM;
    const int split = blockIdx.y;
    const int64_t kb0 = int64_t(split) * a.kblocks;
    const int nk = int(std::min<int64_t>(a.kblocks, a.nk_total - kb0));

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            rskd::mbar_init(&full[s], 1);
            rskd::mbar_init(&empty[s], 1);
            consumed[s] = 0;
        }
        rskd::mbar_init(tfull, 1);
        *abort_flag = 0;
        rskd::fence_mbar_init();
    }
    if (warp == 1) tc_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued[kStages] = {};
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % kStages;
                if (kb >= kStages && !rskd::mbar_wait(&empty[s], uint32_t(((kb / kStages) & 1) ^ 1), a.status)) {
                    *abort_flag = 1;
                    break;
                }
                if (*abort_flag) break;
                uint8_t* st = sm + s * kStage;
                const int kx = int((kb0 + kb) * kBK);
                rskd::mbar_expect_tx(&full[s], uint32_t(kStage));
                rskd::tma_load_2d(st, &ta, kx, int(m0), &full[s]);
                rskd::tma_load_2d(st + kABytes, &tb, kx, 0, &full[s]);
                rskd::tma_load_2d(st + kABytes + NH * kBK * 2, &tb, kx, NH, &full[s]);
                ++issued[s];
            }
            // copies still owed to a stage (only after a timeout) land before the CTA leaves.  The MMA
            // thread advances consumed[s] concurrently: one read decides both whether a copy is owed
            // and which phase it completes (a second read could name a phase no copy will complete).
            for (int s = 0; s < kStages; ++s) {
                const int c = consumed[s];
                if (issued[s] > c) rskd::mbar_wait(&full[s], uint32_t(c & 1), a.status);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc(kBM, NH);
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % kStages;
                if (*abort_flag || !rskd::mbar_wait(&full[s], uint32_t((kb / kStages) & 1), a.status)) {
                    *abort_flag = 1;
                    break;
                }
                consumed[s] = consumed[s] + 1;
                tc_fence_after();
                const uint32_t sa = rskd::smem_u32(sm + s * kStage);
                const uint32_t sb = sa + kABytes;
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk) {
                    const uint64_t ad = smem_desc(sa + kk * 32);
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const uint64_t bd = smem_desc(sb + hh * NH * kBK * 2 + kk * 32);
                        tc_mma(tmem + uint32_t(hh * NH), ad, bd, idesc, (kb | kk) != 0 ? 1u : 0u);
                    }
                }
                tc_commit(&empty[s]);
            }
            // the accumulator is complete (or the issued MMAs are done, after a timeout)
            tc_commit(tfull);
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. rows m0 + 32 (w % 4) + lane
        const int q = warp & 3;
        // the TMEM loads below are warp-wide (.sync.aligned): the decision to run them is the warp's
        const bool ok = __all_sync(0xffffffffu, rskd::mbar_wait(tfull, 0u, a.status));
        tc_fence_after();
        if (ok && !*abort_flag && nk > 0) {
            const int64_t row = m0 + 32 * q + lane;
            float* out = a.D + int64_t(split) * a.split_stride;
            for (int c0 = 0; c0 < 2 * NH; c0 += 32) {
                uint32_t v[32];
                tc_ld32(tmem + (uint32_t(32 * q) << 16) + uint32_t(c0), v);
                if (row < a.M) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (c0 + j < a.N) out[int64_t(c0 + j) * a.ldd + row] = __uint_as_float(v[j]);
                }
            }
        } else if (nk == 0 && 0 < a.N) {
            const int64_t row = m0 + 32 * q + lane;
            float* out = a.D + int64_t(split) * a.split_stride;
            if (row < a.M)
                for (int c = 0; c < a.N; ++c) out[int64_t(c) * a.ldd + row] = 0.f;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tc_dealloc(tmem, kTmemCols);
    }
}

// D = sum over splits (in split order) of the partials.
__global__ void k_sum_splits(const float* __restrict__ part, int64_t stride, int nsplit, int64_t M, int N, int64_t ldd,
                             float* __restrict__ D) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    const int64_t c = idx / M, r = idx - c * M;
    float s = 0.f;
    for (int p = 0; p < nsplit; ++p) s += part[int64_t(p) * stride + c * M + r];
    D[c * ldd + r] = s;
}

template <int NH>
rsk_status launch_gemm(rsk_handle* h, const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& ga, int mtiles,
                       int nsplit, cudaStream_t stream) {
    constexpr int kStage = kBM * kBK * 2 + 2 * NH * kBK * 2;
    const int smem = stages_for<NH>() * kStage + 1024 + 256;
    auto kern = k_gemm_tc<NH>;
    RSK_CUDA_TRY(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_GEMM);
    kern<<<dim3(unsigned(mtiles), unsigned(nsplit)), kThreads, smem, stream>>>(ta, tb, ga);
    rsk::prof_end(h, stream, pr);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

}  // namespace

namespace rsk {
namespace tc {

size_t gemm_scratch_bytes(int64_t M, int N, int nsplit) {
    return nsplit > 1 ? size_t(nsplit) * size_t(M) * size_t(N) * 4 + 256 : 0;
}

// D (M x N column-major, ldd) = A (M x K, row-major = K-major, lda) * B (N x K, K-major, ldb)^T.
// nsplit > 1 splits K over that many CTAs per row tile (partials in scratch, summed in order).
rsk_status gemm_bf16(rsk_handle* h, const __nv_bfloat16* A, int64_t M, int64_t K, int64_t lda, const __nv_bfloat16* B,
                     int N, int64_t ldb, float* D, int64_t ldd, int nsplit, float* scratch, cudaStream_t stream) {
    if (M < 1 || K < 1 || N < 1 || N > 512 || ldd < M) return fail(h, RSK_ERR_INVALID_ARG, "gemm: bad shape");
    if ((lda * 2) % 16 || (ldb * 2) % 16 || reinterpret_cast<uintptr_t>(A) % 16 || reinterpret_cast<uintptr_t>(B) % 16)
        return fail(h, RSK_ERR_INVALID_ARG, "gemm: operands and row pitches must be 16-byte aligned");
    // N split into two halves of NH columns (a multiple of 16, the MMA's N step for M = 128)
    const int nh = std::max(16, ((N + 1) / 2 + 15) / 16 * 16);
    const int64_t nk = (K + kBK - 1) / kBK;
    nsplit = int(std::max<int64_t>(1, std::min<int64_t>(nsplit, nk)));
    const int kblocks = int((nk + nsplit - 1) / nsplit);
    nsplit = int((nk + kblocks - 1) / kblocks);
    CUtensorMap ta, tb;
    memset(&ta, 0, sizeof(ta));
    memset(&tb, 0, sizeof(tb));
    if (!encode_2d_swz128(h, &ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, A, uint64_t(K), uint64_t(M), uint64_t(lda) * 2, kBK,
                          kBM) ||
        !encode_2d_swz128(h, &tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B, uint64_t(K), uint64_t(N), uint64_t(ldb) * 2, kBK,
                          uint32_t(nh)))
        return fail(h, RSK_ERR_UNSUPPORTED, "gemm: tensor map encoding failed");
    GemmArgs ga;
    ga.M = M;
    ga.K = K;
    ga.N = N;
    ga.kblocks = kblocks;
    ga.nk_total = nk;
    ga.status = h->dev_status;
    if (nsplit > 1) {
        if (!scratch) return fail(h, RSK_ERR_INVALID_ARG, "gemm: split-K needs scratch");
        ga.D = scratch;
        ga.ldd = M;
        ga.split_stride = M * int64_t(N);
    } else {
        ga.D = D;
        ga.ldd = ldd;
        ga.split_stride = 0;
    }
    const int mtiles = int((M + kBM - 1) / kBM);
    rsk_status st;
    switch (nh) {
        case 16: st = launch_gemm<16>(h, ta, tb, ga, mtiles, nsplit, stream); break;
        case 32: st = launch_gemm<32>(h, ta, tb, ga, mtiles, nsplit, stream); break;
        case 48: st = launch_gemm<48>(h, ta, tb, ga, mtiles, nsplit, stream); break;
        case 64: st = launch_gemm<64>(h, ta, tb, ga, mtiles, nsplit, stream); break;
        case 96: st = launch_gemm<96>(h, ta, tb, ga, mtiles, nsplit, stream); break;
        case 128: st = launch_gemm<128>(h, ta, tb, ga, mtiles, nsplit, stream); break;
        case 160: st = launch_gemm<160>(h, ta, tb, ga, mtiles, nsplit, stream); break;
        case 192: st = launch_gemm<192>(h, ta, tb, ga, mtiles, nsplit, stream); break;
        case 256: st = launch_gemm<256>(h, ta, tb, ga, mtiles, nsplit, stream); break;
        default: return fail(h, RSK_ERR_UNSUPPORTED, "gemm: N = %d is not supported (half %d)", N, nh);
    }
    if (st != RSK_OK || nsplit == 1) return st;
    k_sum_splits<<<unsigned((M * N + 255) / 256), 256, 0, stream>>>(scratch, M * int64_t(N), nsplit, M, N, ldd, D);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

}  // namespace tc
}  // namespace rsk

extern "C" rsk_status rsk_gemm_bf16(rsk_handle* h, const void* A, int64_t M, int64_t K, int64_t lda, const void* B,
                                    int64_t N, int64_t ldb, float* D, int64_t ldd, int32_t nsplit, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!A || !B || !D) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (M < 1 || K < 1 || N < 1 || N > 512 || lda < K || ldb < K || ldd < M)
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "need M, K >= 1, 1 <= N <= 512, lda, ldb >= K, ldd >= M");
    nsplit = std::max(1, nsplit);
    float* scratch = nullptr;
    if (nsplit > 1) {
        rsk_status st = rsk::ensure_workspace(h, rsk::tc::gemm_scratch_bytes(M, int(N), nsplit), stream);
        if (st != RSK_OK) return st;
        scratch = static_cast<float*>(h->ws);
    }
    return rsk::tc::gemm_bf16(h, static_cast<const __nv_bfloat16*>(A), M, K, lda, static_cast<const __nv_bfloat16*>(B),
                              int(N), ldb, D, ldd, nsplit, scratch, stream);
}
