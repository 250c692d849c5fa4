// BF16 x BF16 -> FP32 products on the fifth-generation tensor cores (tcgen05): the dense products of
// the randomized SVD (Alg. 1: Y = A Z, Z = A^T Q, B = Q^T A) with the rank r <= 512 as the N dimension,
// and, through three-term BF16 splits, the FP32-accurate products of its orthonormalisation (Gram
// matrices X^T X, X R^{-1}) and of U = Q Uhat.
//
// One CTA per 128-row tile of D (and per K split): 6 warps.
//   warp 0, one thread   TMA producer: per 64-wide K block (of every pass), the 128 x 64 tile of A (one
//                        box for K-major A, two 64 x 64 boxes for MN-major A) and the N x 64 tile of B
//                        (two boxes of N/2 rows; with a cluster of 2 or 4 row tiles, this CTA's share of
//                        it, multicast to the cluster) into one of up to 4 shared-memory stages (128-byte
//                        swizzle), completion counted on the stage's `full` mbarrier
//   warp 1, one thread   MMA issuer: per K block, 4 K-steps of 16, each two tcgen05.mma (M = 128,
//                        N = N/2) into the TMEM accumulator (128 lanes x N FP32 columns); a tcgen05.commit
//                        on the stage's `empty` barrier frees it, a last one on `tmem_full` hands the
//                        accumulator to the epilogue.  Warp 1 also allocates and frees the TMEM.
//   warps 2-5            epilogue: tcgen05.ld of their 32 lanes (rows), 32 columns at a time, stored to
//                        D (column-major: lanes = consecutive rows, coalesced; row-major: each lane
//                        writes 128 contiguous bytes of its row).
// Every mbarrier wait is bounded; a wait that runs out records RSK_DEV_TIMEOUT, stops the roles, and
// before the CTA leaves the producer waits (bounded) for the copies still owed to a stage and the
// epilogue for the MMAs already issued, so no copy or MMA outlives the CTA's shared memory or TMEM.
#include "gemm_tc.cuh"

#include "dense.cuh"

#include <string.h>

#include <algorithm>
#include <utility>

namespace {

constexpr int kBM = 128, kBK = 64, kThreads = 192;
// pipeline depth: as many stages (at most 4) as fit in 227 KB of shared memory with the barriers
template <int NH, int NH2>
constexpr int stages_for() {
    return std::min(4, (227 * 1024 - 1024 - 256) / (kBM * kBK * 2 + (NH + NH2) * kBK * 2));
}

// tcgen05 shared-memory matrix descriptor, 128-byte swizzle: start address (bits 0-13, >> 4), leading
// byte offset (bits 16-29, >> 4), stride byte offset (bits 32-45, >> 4), descriptor version 1
// (bits 46-47), swizzle mode 2 = 128-byte (bits 61-63).
//   K-major operand: rows of 64 BF16 (128 bytes) along K, 8-row groups 1024 bytes apart (the stride
//   offset); the leading offset is unused (1).  A K-step of 16 advances the start by 32 bytes.
//   MN-major operand: rows of 64 BF16 along M, one row per K index, 8-row (K) groups 1024 bytes apart
//   (stride offset), the second 64-wide M group 8192 bytes further (leading offset).  A K-step of 16
//   advances the start by two groups (2048 bytes).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo) {
    uint64_t d = uint64_t((saddr & 0x3FFFFu) >> 4);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t(1024 >> 4) << 32;
    d |= uint64_t(1) << 46;
    d |= uint64_t(2) << 61;
    return d;
}

// Instruction descriptor of tcgen05.mma.kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), A MN-major when bit 15 is set (B always K-major: bit 16 = 0), N >> 3
// (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t instr_desc(int m, int n, bool a_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (a_mn ? (1u << 15) : 0u) | (uint32_t(n >> 3) << 17) |
           (uint32_t(m >> 4) << 24);
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
// The same arrive on the barrier at this offset in every CTA of `mask` (thread-block cluster).
__device__ __forceinline__ void tc_commit_mc(uint64_t* bar, uint16_t mask) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                     rskd::smem_u32(bar)),
                 "h"(mask)
                 : "memory");
}
// 2-D tiled TMA load delivered to the same shared-memory offset in every CTA of `mask`, completion
// counted on the barrier at the same offset in each of them.
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                               uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, {%2, "
        "%3}], [%4], %5;" ::"r"(rskd::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(rskd::smem_u32(bar)), "h"(mask)
        : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
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

// b: B with a box of the first half's rows (NH; NH / 2 for clusters of 4); b2: the same B with a box of
// the second half's rows (NH2).
struct GemmMaps {
    CUtensorMap a[rsk::tc::kMaxOperands];
    CUtensorMap b[rsk::tc::kMaxOperands];
    CUtensorMap b2[rsk::tc::kMaxOperands];
};

// Work items of the persistent kernel, counted in cluster units (CL consecutive row tiles that share
// the B tile): items [0, n_full) are the row-tile groups g = item over all of K, written to D; items
// [n_full, n_full + part_groups * nsplit) are (group, split) pairs, group = part_group0 + j % part_groups
// and split = j / part_groups for j = item - n_full, over K blocks [split * kb_part, ...), written to the
// column-major partials P + split * pstride (rows from prow0, leading dimension pld).
struct GemmArgs {
    int64_t M, K;
    int N;             // columns of D stored (<= NH + NH2)
    int64_t nk_total;  // K blocks of one pass overall
    int npass;
    uint8_t pa[rsk::tc::kMaxPasses], pb[rsk::tc::kMaxPasses];
    float* D;
    int64_t ldd;
    int row_major;     // D row-major
    int n_full, part_groups, part_group0, nsplit, kb_part, nitems;
    float* P;
    int64_t pstride, prow0, pld;
    unsigned int* status;
};

struct ItemRange {
    int group, kb0, nk;
    bool partial;
    int split;
};
__device__ __forceinline__ ItemRange decode_item(const GemmArgs& a, int item) {
    ItemRange r;
    if (item < a.n_full) {
        r.group = item;
        r.kb0 = 0;
        r.nk = int(a.nk_total);
        r.partial = false;
        r.split = 0;
    } else {
        const int j = item - a.n_full;
        r.split = j / a.part_groups;
        r.group = a.part_group0 + (j - r.split * a.part_groups);
        r.kb0 = r.split * a.kb_part;
        r.nk = int(min(int64_t(a.kb_part), a.nk_total - r.kb0));
        r.partial = true;
    }
    return r;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(rskd::smem_u32(bar)) : "memory");
}

// The N columns of the tile are two MMAs' worth: the first NH, then NH2 <= NH (each a multiple of 16,
// the MMA's N step for M = 128), accumulated side by side in tensor memory.
// Persistent: cluster c takes items c, c + C, c + 2C, ... (C clusters in the grid); CTA rank r of the
// cluster computes row tile CL * group + r of each.  The operand ring runs on across items: the
// producer fills stages for the next item while the MMAs of the current one finish and the epilogue
// drains its accumulator; the first MMA of an item waits until the epilogue has read the previous
// accumulator out of tensor memory (`tempty`), the epilogue waits for the item's last MMA (`tfull`).
// CL > 1: the CTAs of a cluster share the B tile: with CL = 2 CTA rank c loads half c of it, with
// CL = 4 (NH2 = NH only) rows [c NH/2, (c+1) NH/2), and multicasts its piece to the whole cluster, so
// each stage's `full` barrier counts the own A tile plus the CL pieces, and a stage is free again only
// when every CTA's MMAs are done with it (its `empty` barrier takes one multicast commit from each CTA).
template <int NH, int NH2, bool A_MN, int CL>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ GemmMaps maps, const GemmArgs a) {
    static_assert(NH2 <= NH && NH2 % 16 == 0 && NH2 >= 16, "second half: a multiple of 16, at most NH");
    static_assert(CL != 4 || NH2 == NH, "clusters of 4 split equal halves");
    constexpr int kStages = stages_for<NH, NH2>();
    constexpr int kABytes = kBM * kBK * 2;          // 16 KB
    constexpr int kBBytes = (NH + NH2) * kBK * 2;   // N x 64 BF16
    constexpr int kStage = kABytes + kBBytes;       // multiple of 1024
    constexpr int kNT = NH + NH2;
    constexpr uint32_t kTmemCols = (kNT <= 32) ? 32 : (kNT <= 64) ? 64 : (kNT <= 128) ? 128 : (kNT <= 256) ? 256 : 512;
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + kStages * kStage);
    uint64_t* empty = full + kStages;
    uint64_t* tfull = empty + kStages;
    uint64_t* tempty = tfull + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* consumed = abort_flag + 1;  // K blocks the MMA thread has waited for, per stage

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nclusters = int(gridDim.x) / CL;
    const int cluster_id = int(blockIdx.x) / CL;

    constexpr uint16_t kMask = uint16_t((1u << CL) - 1);
    constexpr int kPieceRows = CL == 4 ? NH / 2 : NH;      // B rows between consecutive CTAs' pieces
    const int rank = CL > 1 ? int(cluster_rank()) : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            rskd::mbar_init(&full[s], 1);
            rskd::mbar_init(&empty[s], CL);
            consumed[s] = 0;
        }
        rskd::mbar_init(tfull, 1);
        rskd::mbar_init(tempty, 4);   // one arrive per epilogue warp
        *abort_flag = 0;
        rskd::fence_mbar_init();
    }
    if (warp == 1) tc_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    if constexpr (CL > 1) cluster_sync();   // every CTA's barriers exist before any remote arrive
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued[kStages] = {};
            int it = 0;
            for (int item = cluster_id; item < a.nitems && !*abort_flag; item += nclusters) {
                const ItemRange ir = decode_item(a, item);
                const int64_t m0 = (int64_t(ir.group) * CL + rank) * kBM;
                const int total = ir.nk * a.npass;
                for (int t = 0; t < total; ++t, ++it) {
                    const int s = it % kStages;
                    if (it >= kStages && !rskd::mbar_wait(&empty[s], uint32_t(((it / kStages) & 1) ^ 1), a.status)) {
                        *abort_flag = 1;
                        break;
                    }
                    if (*abort_flag) break;
                    const int pass = t / ir.nk, kb = t - pass * ir.nk;
                    const CUtensorMap* ma = &maps.a[a.pa[pass]];
                    const CUtensorMap* mb = &maps.b[a.pb[pass]];
                    const CUtensorMap* mb2 = &maps.b2[a.pb[pass]];
                    uint8_t* st = sm + s * kStage;
                    const int kx = (ir.kb0 + kb) * kBK;
                    rskd::mbar_expect_tx(&full[s], uint32_t(kStage));
                    if constexpr (A_MN) {
                        rskd::tma_load_2d(st, ma, int(m0), kx, &full[s]);
                        rskd::tma_load_2d(st + kABytes / 2, ma, int(m0) + 64, kx, &full[s]);
                    } else {
                        rskd::tma_load_2d(st, ma, kx, int(m0), &full[s]);
                    }
                    if constexpr (CL == 1) {
                        rskd::tma_load_2d(st + kABytes, mb, kx, 0, &full[s]);
                        rskd::tma_load_2d(st + kABytes + NH * kBK * 2, mb2, kx, NH, &full[s]);
                    } else {
                        tma_load_2d_mc(st + kABytes + rank * kPieceRows * kBK * 2, (CL == 2 && rank == 1) ? mb2 : mb,
                                       kx, rank * kPieceRows, &full[s], kMask);
                    }
                    ++issued[s];
                }
            }
            if constexpr (CL > 1) {
                // every CTA's last release of every stage: after it no remote arrive or multicast
                // write targets this CTA's shared memory (skipped after a timeout: the bounded waits
                // of the other CTAs outlast their copies in flight)
                if (!*abort_flag)
                    for (int s = 0; s < kStages && s < it; ++s) {
                        const int last = (it - 1 - s) / kStages;   // use number of the stage's last fill
                        rskd::mbar_wait(&empty[s], uint32_t(last & 1), a.status);
                    }
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
            constexpr uint32_t idesc = instr_desc(kBM, NH, A_MN), idesc2 = instr_desc(kBM, NH2, A_MN);
            int it = 0, j = 0;
            for (int item = cluster_id; item < a.nitems && !*abort_flag; item += nclusters, ++j) {
                const ItemRange ir = decode_item(a, item);
                const int total = ir.nk * a.npass;
                // the epilogue has read the previous item's accumulator
                if (j > 0 && !rskd::mbar_wait(tempty, uint32_t((j - 1) & 1), a.status)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                bool stop = false;
                for (int t = 0; t < total; ++t, ++it) {
                    const int s = it % kStages;
                    if (*abort_flag || !rskd::mbar_wait(&full[s], uint32_t((it / kStages) & 1), a.status)) {
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    consumed[s] = consumed[s] + 1;
                    tc_fence_after();
                    const uint32_t sa = rskd::smem_u32(sm + s * kStage);
                    const uint32_t sb = sa + kABytes;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint64_t ad = A_MN ? smem_desc(sa + kk * 2048, kABytes / 2) : smem_desc(sa + kk * 32, 16);
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const uint64_t bd = smem_desc(sb + hh * NH * kBK * 2 + kk * 32, 16);
                            tc_mma(tmem + uint32_t(hh * NH), ad, bd, hh ? idesc2 : idesc, (t | kk) != 0 ? 1u : 0u);
                        }
                    }
                    if constexpr (CL == 1) tc_commit(&empty[s]);
                    else tc_commit_mc(&empty[s], kMask);
                }
                // the item's accumulator is complete (or, after a timeout, the issued MMAs are done)
                tc_commit(tfull);
                if (stop) break;
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. rows m0 + 32 (w % 4) + lane
        const int q = warp & 3;
        int j = 0;
        for (int item = cluster_id; item < a.nitems; item += nclusters, ++j) {
            // the TMEM loads below are warp-wide (.sync.aligned): the decision to run them is the warp's
            const bool ok = __all_sync(0xffffffffu, rskd::mbar_wait(tfull, uint32_t(j & 1), a.status));
            if (!ok || *abort_flag) {
                if (lane == 0) *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const ItemRange ir = decode_item(a, item);
            const int64_t row = (int64_t(ir.group) * CL + rank) * kBM + 32 * q + lane;
            float* out;
            int64_t ld, orow;
            bool rm;
            if (ir.partial) {
                out = a.P + int64_t(ir.split) * a.pstride;
                ld = a.pld;
                orow = row - a.prow0;
                rm = false;
            } else {
                out = a.D;
                ld = a.ldd;
                orow = row;
                rm = a.row_major != 0;
            }
            for (int c0 = 0; c0 < kNT; c0 += 32) {
                uint32_t v[32];
                tc_ld32(tmem + (uint32_t(32 * q) << 16) + uint32_t(c0), v);
                if (row < a.M && c0 < a.N) {
                    if (!rm) {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj)
                            if (c0 + jj < a.N) out[int64_t(c0 + jj) * ld + orow] = __uint_as_float(v[jj]);
                    } else if (c0 + 32 <= a.N && (ld & 3) == 0) {
                        float4* o4 = reinterpret_cast<float4*>(out + orow * ld + c0);
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj)
                            o4[jj] = make_float4(__uint_as_float(v[4 * jj]), __uint_as_float(v[4 * jj + 1]),
                                                 __uint_as_float(v[4 * jj + 2]), __uint_as_float(v[4 * jj + 3]));
                    } else {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj)
                            if (c0 + jj < a.N) out[orow * ld + c0 + jj] = __uint_as_float(v[jj]);
                    }
                }
            }
            // this warp's reads of the accumulator are complete: hand tensor memory back to the MMAs
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tc_dealloc(tmem, kTmemCols);
    }
    if constexpr (CL > 1) cluster_sync();   // no CTA leaves while another may still signal it
}

// Rows row0 + r (0 <= r < rows) of D = sum over splits (in split order) of the column-major partials
// (element (r, c) of split p at part[p * stride + c * rows + r]).
__global__ void k_sum_splits(const float* __restrict__ part, int64_t stride, int nsplit, int64_t row0, int64_t rows,
                             int N, int64_t ldd, int row_major, float* __restrict__ D) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= rows * N) return;
    const int64_t c = idx / rows, r = idx - c * rows;
    float s = 0.f;
    for (int p = 0; p < nsplit; ++p) s += part[int64_t(p) * stride + c * rows + r];
    const int64_t row = row0 + r;
    D[row_major ? row * ldd + c : c * ldd + row] = s;
}

// Three-term BF16 split, column c of X at X + c * ldx: x1 = bf16(x), x2 = bf16(x - x1), x3 =
// bf16(x - x1 - x2); both differences are exact in FP32 (each has at most 16 significant bits).
__global__ void k_split3(const float* __restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                         __nv_bfloat16* __restrict__ o1, __nv_bfloat16* __restrict__ o2,
                         __nv_bfloat16* __restrict__ o3, int64_t ldt) {
    for (int64_t c = blockIdx.y; c < cols; c += gridDim.y)
        for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x) {
            const float x = X[c * ldx + r];
            const __nv_bfloat16 b1 = __float2bfloat16_rn(x);
            const float r1 = x - __bfloat162float(b1);
            const __nv_bfloat16 b2 = __float2bfloat16_rn(r1);
            const float r2 = r1 - __bfloat162float(b2);
            o1[c * ldt + r] = b1;
            o2[c * ldt + r] = b2;
            o3[c * ldt + r] = __float2bfloat16_rn(r2);
        }
}

// The same split, four consecutive rows a thread (rows, ldx, ldt multiples of 4; X 16-byte and the
// outputs 8-byte aligned): one 16-byte load and three 8-byte stores.
__global__ void k_split3_v4(const float* __restrict__ X, int64_t rows4, int64_t cols, int64_t ldx,
                            __nv_bfloat16* __restrict__ o1, __nv_bfloat16* __restrict__ o2,
                            __nv_bfloat16* __restrict__ o3, int64_t ldt) {
    for (int64_t c = blockIdx.y; c < cols; c += gridDim.y)
        for (int64_t r4 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r4 < rows4;
             r4 += int64_t(gridDim.x) * blockDim.x) {
            const float4 x = *reinterpret_cast<const float4*>(X + c * ldx + 4 * r4);
            const float xs[4] = {x.x, x.y, x.z, x.w};
            __nv_bfloat16 b1[4], b2[4], b3[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                b1[i] = __float2bfloat16_rn(xs[i]);
                const float r1 = xs[i] - __bfloat162float(b1[i]);
                b2[i] = __float2bfloat16_rn(r1);
                b3[i] = __float2bfloat16_rn(r1 - __bfloat162float(b2[i]));
            }
            const int64_t o = c * ldt + 4 * r4;
            *reinterpret_cast<uint2*>(o1 + o) = *reinterpret_cast<const uint2*>(b1);
            *reinterpret_cast<uint2*>(o2 + o) = *reinterpret_cast<const uint2*>(b2);
            *reinterpret_cast<uint2*>(o3 + o) = *reinterpret_cast<const uint2*>(b3);
        }
}

__global__ void k_to_bf16(const float* __restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                          __nv_bfloat16* __restrict__ out, int64_t ldt) {
    for (int64_t c = blockIdx.y; c < cols; c += gridDim.y)
        for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x)
            out[c * ldt + r] = __float2bfloat16_rn(X[c * ldx + r]);
}

// Packed conversion (ldx == ldt == rows, count a multiple of 4, 16-byte aligned X): 4 elements a thread.
__global__ void k_to_bf16_flat(const float4* __restrict__ X, int64_t n4, uint2* __restrict__ out) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += int64_t(gridDim.x) * blockDim.x) {
        const float4 f = X[i];
        const __nv_bfloat162 lo = __floats2bfloat162_rn(f.x, f.y), hi = __floats2bfloat162_rn(f.z, f.w);
        uint2 o;
        o.x = *reinterpret_cast<const uint32_t*>(&lo);
        o.y = *reinterpret_cast<const uint32_t*>(&hi);
        out[i] = o;
    }
}

// Co-resident clusters of a kernel instance (at most one CTA per SM: the shared memory is the limit);
// 0 if the query fails.
int resident_clusters(const void* kern, cudaLaunchConfig_t cfg) {
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    return n;
}

// How the row-tile groups become work items: nsplit > 1 splits every group's K range; otherwise, with
// split_last and enough scratch, a last round of items that would leave more than half the clusters
// idle is split over K instead (2 to 4 ways, as many as fill the clusters).  sum_row0 / sum_splits
// (out) say which rows of D come from partials (sum_splits 0: none).
struct ItemPlan {
    int groups, cl, nsplit, kblocks;
    float* scratch;
    size_t scratch_bytes;
    bool split_last;
    int64_t sum_row0;
    int sum_splits;
};

void plan_items(GemmArgs& ga, ItemPlan& ip, int nc) {
    ga.P = ip.scratch;
    ip.sum_splits = 0;
    ip.sum_row0 = 0;
    if (ip.nsplit > 1) {
        ga.n_full = 0;
        ga.part_groups = ip.groups;
        ga.part_group0 = 0;
        ga.nsplit = ip.nsplit;
        ga.kb_part = ip.kblocks;
        ga.prow0 = 0;
        ga.pld = ga.M;
        ga.pstride = ga.M * int64_t(ga.N);
        ip.sum_splits = ip.nsplit;
    } else {
        ga.n_full = ip.groups;
        ga.part_groups = 0;
        ga.nsplit = 1;
        const int rem = nc > 0 ? ip.groups % nc : 0;
        if (ip.split_last && ip.scratch && ip.groups > nc && rem > 0 && 2 * rem <= nc && ga.nk_total >= 32) {
            int S = std::max(2, std::min(4, nc / rem));
            const int kb = int((ga.nk_total + S - 1) / S);
            S = int((ga.nk_total + kb - 1) / kb);
            const int64_t prow0 = int64_t(ip.groups - rem) * ip.cl * kBM;
            const int64_t pld = ga.M - prow0;
            if (pld > 0 && size_t(S) * size_t(pld) * size_t(ga.N) * 4 <= ip.scratch_bytes) {
                ga.n_full = ip.groups - rem;
                ga.part_groups = rem;
                ga.part_group0 = ga.n_full;
                ga.nsplit = S;
                ga.kb_part = kb;
                ga.prow0 = prow0;
                ga.pld = pld;
                ga.pstride = pld * int64_t(ga.N);
                ip.sum_row0 = prow0;
                ip.sum_splits = S;
            }
        }
    }
    ga.nitems = ga.n_full + ga.part_groups * ga.nsplit;
}

template <int NH, int NH2, bool A_MN, int CL>
rsk_status launch_gemm(rsk_handle* h, const GemmMaps& maps, GemmArgs ga, ItemPlan& ip, cudaStream_t stream) {
    constexpr int kStage = kBM * kBK * 2 + (NH + NH2) * kBK * 2;
    const int smem = stages_for<NH, NH2>() * kStage + 1024 + 256;
    auto kern = k_gemm_tc<NH, NH2, A_MN, CL>;
    RSK_CUDA_TRY(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = size_t(smem);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // persistent grid: as many clusters as can be resident together (no more than there are items);
    // the items are dealt round-robin, so a smaller grid is only slower, never wrong
    static int resident = -1;   // per kernel instance
    if (resident < 0) {
        cfg.gridDim = dim3(unsigned(CL));
        resident = resident_clusters(reinterpret_cast<const void*>(kern), cfg);
    }
    const int cap = resident > 0 ? resident : std::max(1, h->num_sms / CL);
    plan_items(ga, ip, cap);
    cfg.gridDim = dim3(unsigned(std::min(ga.nitems, cap) * CL));
    const int pr = rsk::prof_begin(h, stream, ga.npass > 1 ? RSK_KERNEL_GEMM_SPLIT : RSK_KERNEL_GEMM);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, maps, ga);
    rsk::prof_end(h, stream, pr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return rsk::fail(h, RSK_ERR_CUDA, "gemm launch: %s", cudaGetErrorString(e));
    }
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

// Clusters of 4 are built for the N halves of the RSVD's ranks (128, 160, 256) only.
constexpr bool cluster4_nh(int nh) { return nh == 128 || nh == 160 || nh == 256; }

// the N halves (nh, nh2): nh2 = nh, or nh - 16 (clusters of 1 or 2)
template <int NH, bool A_MN, int CL>
rsk_status launch_halves(rsk_handle* h, int nh2, const GemmMaps& maps, const GemmArgs& ga, ItemPlan& ip, cudaStream_t stream) {
    if constexpr (CL != 4 && NH >= 32) {
        if (nh2 == NH - 16) return launch_gemm<NH, NH - 16, A_MN, CL>(h, maps, ga, ip, stream);
    }
    if (nh2 != NH) return rsk::fail(h, RSK_ERR_INTERNAL, "gemm: N halves %d + %d are not built", NH, nh2);
    return launch_gemm<NH, NH, A_MN, CL>(h, maps, ga, ip, stream);
}

template <bool A_MN, int CL>
rsk_status dispatch_nh(rsk_handle* h, int nh, int nh2, const GemmMaps& maps, const GemmArgs& ga, ItemPlan& ip, cudaStream_t stream) {
    if constexpr (CL == 4) {
        switch (nh) {
            case 128: return launch_halves<128, A_MN, 4>(h, nh2, maps, ga, ip, stream);
            case 160: return launch_halves<160, A_MN, 4>(h, nh2, maps, ga, ip, stream);
            case 256: return launch_halves<256, A_MN, 4>(h, nh2, maps, ga, ip, stream);
            default: return rsk::fail(h, RSK_ERR_UNSUPPORTED, "gemm: clusters of 4 need N half 128, 160 or 256");
        }
    } else {
        switch (nh) {
            case 16: return launch_halves<16, A_MN, CL>(h, nh2, maps, ga, ip, stream);
            case 32: return launch_halves<32, A_MN, CL>(h, nh2, maps, ga, ip, stream);
            case 48: return launch_halves<48, A_MN, CL>(h, nh2, maps, ga, ip, stream);
            case 64: return launch_halves<64, A_MN, CL>(h, nh2, maps, ga, ip, stream);
            case 96: return launch_halves<96, A_MN, CL>(h, nh2, maps, ga, ip, stream);
            case 128: return launch_halves<128, A_MN, CL>(h, nh2, maps, ga, ip, stream);
            case 160: return launch_halves<160, A_MN, CL>(h, nh2, maps, ga, ip, stream);
            case 192: return launch_halves<192, A_MN, CL>(h, nh2, maps, ga, ip, stream);
            case 256: return launch_halves<256, A_MN, CL>(h, nh2, maps, ga, ip, stream);
            default: return rsk::fail(h, RSK_ERR_UNSUPPORTED, "gemm: N half %d is not supported", nh);
        }
    }
}

bool aligned16(const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

}  // namespace

namespace rsk {
namespace tc {

size_t gemm_scratch_bytes(int64_t M, int N, int nsplit) {
    return nsplit > 1 ? size_t(nsplit) * size_t(M) * size_t(N) * 4 + 256 : 0;
}

int wave_splits(int64_t M, int64_t K, int num_sms, int max_split) {
    const int64_t mtiles = (M + kBM - 1) / kBM;
    const int64_t tiles = mtiles >= 8 ? (mtiles + 1) / 2 * 2 : mtiles;   // the automatic cluster of 2
    const int64_t nk = (K + kBK - 1) / kBK;
    int best = 1;
    double best_eff = 0.0;
    for (int s = 1; s <= max_split && s <= nk; ++s) {
        const int64_t kb = (nk + s - 1) / s;
        const int64_t splits = (nk + kb - 1) / kb;
        const int64_t ctas = tiles * splits;
        const int64_t waves = (ctas + num_sms - 1) / num_sms;
        // busy fraction of the SMs over the waves, times the share of a CTA's time spent in its K loop
        // (about 12 K blocks' worth of setup, pipeline fill and epilogue per CTA)
        const double eff = double(ctas) / double(waves * num_sms) * double(kb) / double(kb + 12);
        if (eff > best_eff * 1.005) {
            best_eff = eff;
            best = int(splits);
        }
    }
    return best;
}

void set_split_passes(Product& p) {
    // The tensor cores' FP32 accumulation rounds toward zero: every MMA into an accumulator loses up to
    // one unit in the last place of the accumulator's current value.  The correction terms therefore
    // go first, smallest first, while the accumulator is small, and the main term x1 y1 last: the
    // bias is then that of the main term's own K steps alone.
    static const uint8_t pa[kMaxPasses] = {2, 0, 1, 1, 0, 0}, pb[kMaxPasses] = {0, 2, 1, 0, 1, 0};
    p.npass = kMaxPasses;
    for (int i = 0; i < kMaxPasses; ++i) {
        p.pa[i] = pa[i];
        p.pb[i] = pb[i];
    }
}

rsk_status gemm(rsk_handle* h, const Product& p, int nsplit, float* scratch, cudaStream_t stream, int cluster,
                size_t scratch_bytes, bool split_last) {
    if (p.M < 1 || p.K < 1 || p.N < 1 || p.N > 512 || p.ldd < (p.d_row_major ? p.N : p.M))
        return fail(h, RSK_ERR_INVALID_ARG, "gemm: bad shape");
    if (p.npass < 1 || p.npass > kMaxPasses || p.na < 1 || p.na > kMaxOperands || p.nb < 1 || p.nb > kMaxOperands)
        return fail(h, RSK_ERR_INVALID_ARG, "gemm: bad pass list");
    for (int i = 0; i < p.npass; ++i)
        if (p.pa[i] >= p.na || p.pb[i] >= p.nb) return fail(h, RSK_ERR_INVALID_ARG, "gemm: pass names a missing operand");
    if ((p.lda * 2) % 16 || (p.ldb * 2) % 16 || p.lda < (p.a_mn ? p.M : p.K) || p.ldb < p.K)
        return fail(h, RSK_ERR_INVALID_ARG, "gemm: leading dimensions must cover the operand and be multiples of 8");
    for (int i = 0; i < p.na; ++i)
        if (!p.a[i] || !aligned16(p.a[i])) return fail(h, RSK_ERR_INVALID_ARG, "gemm: A operands must be 16-byte aligned");
    for (int i = 0; i < p.nb; ++i)
        if (!p.b[i] || !aligned16(p.b[i])) return fail(h, RSK_ERR_INVALID_ARG, "gemm: B operands must be 16-byte aligned");
    // N split into two halves of NH columns (a multiple of 16, the MMA's N step for M = 128), rounded up
    // to a half width the kernel is built for (the extra rows of B are zero-filled by the copies and the
    // extra columns of D are not stored); the second half is 16 columns narrower when that still covers
    // N (N = 300: 160 + 144 = 304 columns computed instead of 320)
    static const int kHalves[] = {16, 32, 48, 64, 96, 128, 160, 192, 256};
    int nh = 256;
    for (int c : kHalves)
        if (2 * c >= p.N) {
            nh = c;
            break;
        }
    const int64_t nk = (p.K + kBK - 1) / kBK;
    nsplit = int(std::max<int64_t>(1, std::min<int64_t>(nsplit, nk)));
    const int kblocks = int((nk + nsplit - 1) / nsplit);
    nsplit = int((nk + kblocks - 1) / kblocks);
    const int mtiles = int((p.M + kBM - 1) / kBM);
    // row tiles per cluster sharing the B tile (multicast): automatic = 2 with at least 8 row tiles
    // (measured on the RSVD's 262144 x 8192 x 300 products: pairs 6% faster than single tiles, fours no
    // faster than pairs), else 1
    if (cluster != 0 && cluster != 1 && cluster != 2 && cluster != 4)
        return fail(h, RSK_ERR_INVALID_ARG, "gemm: cluster must be 0 (automatic), 1, 2 or 4");
    if (cluster == 4 && !cluster4_nh(nh))
        return fail(h, RSK_ERR_UNSUPPORTED, "gemm: clusters of 4 need N half 128, 160 or 256 (have %d)", nh);
    const int cl = cluster ? cluster : mtiles >= 8 ? 2 : 1;
    const int nh2 = (cl != 4 && nh >= 32 && 2 * nh - 16 >= p.N) ? nh - 16 : nh;
    GemmMaps maps;
    memset(&maps, 0, sizeof(maps));
    for (int i = 0; i < p.na; ++i) {
        const bool ok = p.a_mn ? encode_2d_swz128(h, &maps.a[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, p.a[i],
                                                  uint64_t(p.M), uint64_t(p.K), uint64_t(p.lda) * 2, 64, 64)
                               : encode_2d_swz128(h, &maps.a[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, p.a[i],
                                                  uint64_t(p.K), uint64_t(p.M), uint64_t(p.lda) * 2, kBK, kBM);
        if (!ok) return fail(h, RSK_ERR_UNSUPPORTED, "gemm: tensor map encoding failed (A)");
    }
    for (int i = 0; i < p.nb; ++i)
        if (!encode_2d_swz128(h, &maps.b[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, p.b[i], uint64_t(p.K), uint64_t(p.N),
                              uint64_t(p.ldb) * 2, kBK, uint32_t(cl == 4 ? nh / 2 : nh)) ||
            !encode_2d_swz128(h, &maps.b2[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, p.b[i], uint64_t(p.K), uint64_t(p.N),
                              uint64_t(p.ldb) * 2, kBK, uint32_t(cl == 4 ? nh / 2 : nh2)))
            return fail(h, RSK_ERR_UNSUPPORTED, "gemm: tensor map encoding failed (B)");
    GemmArgs ga;
    memset(&ga, 0, sizeof(ga));
    ga.M = p.M;
    ga.K = p.K;
    ga.N = p.N;
    ga.nk_total = nk;
    ga.npass = p.npass;
    for (int i = 0; i < p.npass; ++i) {
        ga.pa[i] = p.pa[i];
        ga.pb[i] = p.pb[i];
    }
    ga.status = h->dev_status;
    ga.D = p.D;
    ga.ldd = p.ldd;
    ga.row_major = p.d_row_major ? 1 : 0;
    if (nsplit > 1 && !scratch) return fail(h, RSK_ERR_INVALID_ARG, "gemm: split-K needs scratch");
    ItemPlan ip;
    ip.groups = (mtiles + cl - 1) / cl;
    ip.cl = cl;
    ip.nsplit = nsplit;
    ip.kblocks = kblocks;
    ip.scratch = scratch;
    ip.scratch_bytes = scratch_bytes;
    ip.split_last = split_last;
    ip.sum_row0 = 0;
    ip.sum_splits = 0;
    rsk_status st;
    if (cl == 4)
        st = p.a_mn ? dispatch_nh<true, 4>(h, nh, nh2, maps, ga, ip, stream)
                    : dispatch_nh<false, 4>(h, nh, nh2, maps, ga, ip, stream);
    else if (cl == 2)
        st = p.a_mn ? dispatch_nh<true, 2>(h, nh, nh2, maps, ga, ip, stream)
                    : dispatch_nh<false, 2>(h, nh, nh2, maps, ga, ip, stream);
    else
        st = p.a_mn ? dispatch_nh<true, 1>(h, nh, nh2, maps, ga, ip, stream)
                    : dispatch_nh<false, 1>(h, nh, nh2, maps, ga, ip, stream);
    if (st != RSK_OK || ip.sum_splits == 0) return st;
    const int64_t rows = p.M - ip.sum_row0;
    k_sum_splits<<<unsigned((rows * p.N + 255) / 256), 256, 0, stream>>>(scratch, rows * int64_t(p.N), ip.sum_splits,
                                                                         ip.sum_row0, rows, p.N, p.ldd,
                                                                         p.d_row_major ? 1 : 0, p.D);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

static dim3 elementwise_grid(int64_t rows, int64_t cols) {
    return dim3(unsigned(std::min<int64_t>((rows + 255) / 256, 64)), unsigned(std::min<int64_t>(cols, 16384)));
}

rsk_status split3(rsk_handle* h, const float* X, int64_t rows, int64_t cols, int64_t ldx, __nv_bfloat16* const* out,
                  int64_t ldt, cudaStream_t stream) {
    const int pr = prof_begin(h, stream, RSK_KERNEL_CONVERT);
    bool v4 = rows % 4 == 0 && ldx % 4 == 0 && ldt % 4 == 0 && aligned16(X);
    for (int i = 0; i < 3; ++i) v4 = v4 && reinterpret_cast<uintptr_t>(out[i]) % 8 == 0;
    if (v4)
        k_split3_v4<<<elementwise_grid(rows / 4, cols), 256, 0, stream>>>(X, rows / 4, cols, ldx, out[0], out[1], out[2],
                                                                          ldt);
    else
        k_split3<<<elementwise_grid(rows, cols), 256, 0, stream>>>(X, rows, cols, ldx, out[0], out[1], out[2], ldt);
    prof_end(h, stream, pr);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

rsk_status to_bf16(rsk_handle* h, const float* X, int64_t rows, int64_t cols, int64_t ldx, __nv_bfloat16* out,
                   int64_t ldt, cudaStream_t stream) {
    const int64_t count = rows * cols;
    const int pr = prof_begin(h, stream, RSK_KERNEL_CONVERT);
    if (ldx == rows && ldt == rows && count % 4 == 0 && aligned16(X) && reinterpret_cast<uintptr_t>(out) % 8 == 0) {
        const unsigned grid = unsigned(std::min<int64_t>((count / 4 + 255) / 256, int64_t(h->num_sms) * 16));
        k_to_bf16_flat<<<grid, 256, 0, stream>>>(reinterpret_cast<const float4*>(X), count / 4,
                                                 reinterpret_cast<uint2*>(out));
    } else {
        k_to_bf16<<<elementwise_grid(rows, cols), 256, 0, stream>>>(X, rows, cols, ldx, out, ldt);
    }
    prof_end(h, stream, pr);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

size_t f32_product_scratch_bytes(bool a_mn, int64_t M, int64_t K, int N, int nsplit) {
    const int64_t a_rows = a_mn ? M : K, a_cols = a_mn ? K : M;
    return 3 * Carver::round(size_t(pad8(a_rows)) * size_t(a_cols) * 2) + 3 * Carver::round(size_t(pad8(K)) * size_t(N) * 2) +
           Carver::round(gemm_scratch_bytes(M, N, nsplit) + 4) + 256;
}

rsk_status f32_product(rsk_handle* h, bool a_mn, const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M,
                       int64_t K, int N, float* D, int64_t ldd, bool d_row_major, int nsplit, void* scratch,
                       cudaStream_t stream) {
    Carver cv(scratch);
    // A's splits keep A's orientation: MN-major A is a column-major M x K matrix, K-major A a
    // column-major K x M one
    const int64_t a_rows = a_mn ? M : K, a_cols = a_mn ? K : M;
    const int64_t lta = pad8(a_rows), ltb = pad8(K);
    Product p;
    p.a_mn = a_mn;
    __nv_bfloat16* as[3];
    __nv_bfloat16* bs[3];
    for (int i = 0; i < 3; ++i) as[i] = cv.take<__nv_bfloat16>(size_t(lta) * size_t(a_cols));
    for (int i = 0; i < 3; ++i) bs[i] = cv.take<__nv_bfloat16>(size_t(ltb) * size_t(N));
    float* part = cv.take<float>(gemm_scratch_bytes(M, N, nsplit) / 4 + 1);
    rsk_status st = split3(h, A, a_rows, a_cols, lda, as, lta, stream);
    if (st == RSK_OK) st = split3(h, B, K, N, ldb, bs, ltb, stream);
    if (st != RSK_OK) return st;
    for (int i = 0; i < 3; ++i) {
        p.a[i] = as[i];
        p.b[i] = bs[i];
    }
    p.na = p.nb = 3;
    p.lda = lta;
    p.ldb = ltb;
    set_split_passes(p);
    p.M = M;
    p.K = K;
    p.N = N;
    p.D = D;
    p.ldd = ldd;
    p.d_row_major = d_row_major;
    return gemm(h, p, nsplit, part, stream);
}

// Accumulators of at most 16 K blocks (64 main-term steps) for a Gram over K rows: the truncated
// accumulation's relative bias stays below ~64 x 2^-24 ~ 4e-6.
static int gram_splits(int64_t K) {
    const int64_t nk = (K + 63) / 64;
    return int(std::max<int64_t>(1, (nk + 15) / 16));
}

size_t orth_scratch_bytes(int64_t rows, int r) {
    return 3 * Carver::round(size_t(pad8(rows)) * size_t(r) * 2) + 3 * Carver::round(size_t(pad8(r)) * size_t(r) * 2) +
           4 * Carver::round(size_t(r) * size_t(r) * 4) + Carver::round(gemm_scratch_bytes(r, r, gram_splits(rows)) + 4) +
           1024;
}

rsk_status orth(rsk_handle* h, float** X, float** Xalt, int64_t rows, int r, int64_t ldx, int rounds, int shifted,
                float* Racc, void* scratch, cudaStream_t s) {
    if (r < 1 || r > 330 || rows < r || ldx < rows || ldx % 8)
        return fail(h, RSK_ERR_UNSUPPORTED, "orth: need 1 <= r <= 330, rows >= r, ldx >= rows a multiple of 8");
    Carver cv(scratch);
    const int64_t lds = pad8(rows), ldr = pad8(r);
    __nv_bfloat16* S[3];
    __nv_bfloat16* Rs[3];
    for (int i = 0; i < 3; ++i) S[i] = cv.take<__nv_bfloat16>(size_t(lds) * r);
    for (int i = 0; i < 3; ++i) Rs[i] = cv.take<__nv_bfloat16>(size_t(ldr) * r);
    float* G = cv.take<float>(size_t(r) * r);
    float* R = cv.take<float>(size_t(r) * r);
    float* Ri = cv.take<float>(size_t(r) * r);
    float* Rtmp = cv.take<float>(size_t(r) * r);
    const int gs = gram_splits(rows);
    float* part = cv.take<float>(gemm_scratch_bytes(r, r, gs) / 4 + 1);
    const float coeff0 = 3e-5f;
    for (int round = 0; round < rounds; ++round) {
        rsk_status st = split3(h, *X, rows, r, ldx, S, lds, s);
        if (st != RSK_OK) return st;
        // G = X^T X: A = B = X^T, K-major (column c of X = row c of X^T), K = rows
        Product g;
        for (int i = 0; i < 3; ++i) {
            g.a[i] = S[i];
            g.b[i] = S[i];
        }
        g.na = g.nb = 3;
        g.lda = g.ldb = lds;
        set_split_passes(g);
        g.M = r;
        g.K = rows;
        g.N = r;
        g.D = G;
        g.ldd = r;
        st = gemm(h, g, gs, part, s);
        const int pr = prof_begin(h, s, RSK_KERNEL_FACTOR);
        if (st == RSK_OK) st = dense::cholesky(h, G, r, r, round < shifted ? coeff0 : 0.f, R, r, s);
        if (st == RSK_OK) st = dense::trinv(h, R, r, r, Ri, s);
        prof_end(h, s, pr);
        if (st == RSK_OK) st = split3(h, Ri, r, r, r, Rs, ldr, s);
        if (st != RSK_OK) return st;
        // X R^{-1}: A = X (MN-major: column k of X holds (m, k) for all m), B_op[n][k] = Rinv[k][n] =
        // column n of Rinv (column-major)
        Product p;
        p.a_mn = true;
        for (int i = 0; i < 3; ++i) {
            p.a[i] = S[i];
            p.b[i] = Rs[i];
        }
        p.na = p.nb = 3;
        p.lda = lds;
        p.ldb = ldr;
        set_split_passes(p);
        p.M = rows;
        p.K = r;
        p.N = r;
        p.D = *Xalt;
        p.ldd = ldx;
        st = gemm(h, p, 1, nullptr, s);
        if (st != RSK_OK) return st;
        std::swap(*X, *Xalt);
        if (Racc) {
            // R_total = R_round * R_total (upper triangular factors accumulate on the left)
            if (round == 0) {
                RSK_CUDA_TRY(h, cudaMemcpyAsync(Racc, R, size_t(r) * r * 4, cudaMemcpyDeviceToDevice, s));
            } else {
                st = dense::matmul_ts(h, R, r, r, r, Racc, r, r, Rtmp, r, s);
                if (st != RSK_OK) return st;
                RSK_CUDA_TRY(h, cudaMemcpyAsync(Racc, Rtmp, size_t(r) * r * 4, cudaMemcpyDeviceToDevice, s));
            }
        }
    }
    return RSK_OK;
}

}  // namespace tc
}  // namespace rsk

extern "C" rsk_status rsk_gemm_bf16_ex(rsk_handle* h, int32_t a_mn, const void* A, int64_t M, int64_t K, int64_t lda,
                                       const void* B, int64_t N, int64_t ldb, float* D, int64_t ldd,
                                       int32_t d_row_major, int32_t nsplit, int32_t cluster, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!A || !B || !D) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (M < 1 || K < 1 || N < 1 || N > 512 || lda < (a_mn ? M : K) || ldb < K || ldd < (d_row_major ? N : M))
        return rsk::fail(h, RSK_ERR_INVALID_ARG,
                         "need M, K >= 1, 1 <= N <= 512, lda >= (a_mn ? M : K), ldb >= K, ldd >= (row-major D ? N : M)");
    // nsplit 0: automatic (K splits that fill the SMs, and a last round of row tiles split over K)
    const bool automatic = nsplit == 0;
    nsplit = automatic ? rsk::tc::wave_splits(M, K, h->num_sms) : std::max(1, nsplit);
    float* scratch = nullptr;
    // the split last round needs at most 4 splits of fewer than M rows
    const size_t bytes = std::max(rsk::tc::gemm_scratch_bytes(M, int(N), nsplit),
                                  automatic ? rsk::tc::gemm_scratch_bytes(M, int(N), 4) : size_t(0));
    if (bytes > 0) {
        rsk_status st = rsk::ensure_workspace(h, bytes, stream);
        if (st != RSK_OK) return st;
        scratch = static_cast<float*>(h->ws);
    }
    rsk::tc::Product p;
    p.a_mn = a_mn != 0;
    p.a[0] = static_cast<const __nv_bfloat16*>(A);
    p.na = 1;
    p.lda = lda;
    p.b[0] = static_cast<const __nv_bfloat16*>(B);
    p.nb = 1;
    p.ldb = ldb;
    p.npass = 1;
    p.M = M;
    p.K = K;
    p.N = int(N);
    p.D = D;
    p.ldd = ldd;
    p.d_row_major = d_row_major != 0;
    return rsk::tc::gemm(h, p, nsplit, scratch, stream, cluster, bytes, automatic);
}

extern "C" rsk_status rsk_gemm_bf16(rsk_handle* h, const void* A, int64_t M, int64_t K, int64_t lda, const void* B,
                                    int64_t N, int64_t ldb, float* D, int64_t ldd, int32_t nsplit, cudaStream_t stream) {
    return rsk_gemm_bf16_ex(h, 0, A, M, K, lda, B, N, ldb, D, ldd, 0, nsplit, 0, stream);
}

extern "C" rsk_status rsk_gemm_f32(rsk_handle* h, int32_t a_mn, const float* A, int64_t M, int64_t K, int64_t lda,
                                   const float* B, int64_t N, int64_t ldb, float* D, int64_t ldd, int32_t d_row_major,
                                   int32_t nsplit, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!A || !B || !D) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (M < 1 || K < 1 || N < 1 || N > 512 || lda < (a_mn ? M : K) || ldb < K || ldd < (d_row_major ? N : M))
        return rsk::fail(h, RSK_ERR_INVALID_ARG,
                         "need M, K >= 1, 1 <= N <= 512, lda >= (a_mn ? M : K), ldb >= K, ldd >= (row-major D ? N : M)");
    nsplit = std::max(1, nsplit);
    rsk_status st = rsk::ensure_workspace(h, rsk::tc::f32_product_scratch_bytes(a_mn != 0, M, K, int(N), nsplit), stream);
    if (st != RSK_OK) return st;
    return rsk::tc::f32_product(h, a_mn != 0, A, lda, B, ldb, M, K, int(N), D, ldd, d_row_major != 0, nsplit, h->ws,
                                stream);
}
