// Subsampled randomized trigonometric transform with the Walsh-Hadamard transform (SRTT):
//     Y = sqrt(n/d) * P * (H_n / sqrt(n)) * D * A  =  d^{-1/2} * P * H_n * D * A
// Paper: the transform template Omega = D F S (Sec. 1.6, Eq. "intro-srtt") with F the unitary WHT and
// S a scaled restriction to d uniformly chosen coordinates; cost accounting steps 1-3 and the
// subsampled variant 2'-3' (Sec. 4.x "Arithmetic costs").
//
// Structure.  Write a row index i = b * 2048 + r (r < 2048).  Because H_n = H_{n/2048} (x) H_2048,
//     (H_n x)[p] = sum_b (-1)^{popcount(p_hi & b)} (H_2048 x_b)[p_lo],   p = p_hi * 2048 + p_lo,
// so each 2048-row block b is transformed in full on chip (11 butterfly stages: 6 in registers
// after one layout, 5 after a second) and every output row q then adds +-Z_b[p_lo(q)] into its
// register accumulators -- about 12 adds per element of A and one pass over A.  For n < 2048 the
// block is zero padded: the first n outputs of H_2048 on a zero-padded vector equal H_n.
//
// Kernels
//   k_srtt_draw   one CTA: P by Floyd's algorithm over [0, n) with d Philox draws (stream 2), the
//                 q-th inserted coordinate being output row q; membership in a shared hash set.
//   k_srtt_dbits  D as bits: word w of D is word(seed, 1, w >> 2, w & 3) (bit j set => D_{32w+j} = -1).
//   k_srtt        one CTA (256 threads) per (8-column slice, range of blocks): TMA double-buffered
//                 block staging, sign flip + convert + FWHT, gather-accumulate into per-range partials.
//   k_reduce_srtt sums the partials in range order and scales by d^{-1/2}.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "philox.cuh"

namespace {

constexpr int kBlk = 2048;           // rows per transform block
constexpr int kCols = 8;             // columns per CTA slice
constexpr int kThreads = 256;
constexpr int kBoxRows = 256;
constexpr uint32_t kStreamD = 1;
constexpr uint32_t kStreamP = 2;
// Z layout: row r of the transformed block starts at float offset r*8 + 8*(r >> 5) (a pad of 8
// floats after every 32 rows keeps both butterfly layouts free of bank conflicts).
constexpr int kZFloats = kBlk * kCols + (kBlk / 32) * kCols;
__device__ __forceinline__ int zoff(int r) { return r * kCols + kCols * (r >> 5); }

// ------------------------------------------------------------------------------------------
// P and D.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_srtt_draw(int64_t n, int d, uint64_t seed, int32_t* __restrict__ rows,
                                                     int64_t* __restrict__ rows64, int hash_bits,
                                                     unsigned int* status) {
    extern __shared__ __align__(16) uint8_t sm[];
    uint32_t* w = reinterpret_cast<uint32_t*>(sm);   // d draws
    uint32_t* table = w + d;                           // 2^hash_bits slots, 0xffffffff = empty
    const int cap = 1 << hash_bits;
    for (int q = threadIdx.x; q < d; q += blockDim.x) {
        const rskd::Block4 b = rskd::philox_block(seed, kStreamP, 0, uint32_t(q >> 2));
        w[q] = b.v[q & 3];
    }
    for (int i = threadIdx.x; i < cap; i += blockDim.x) table[i] = 0xffffffffu;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t mask = uint32_t(cap - 1);
        for (int q = 0; q < d; ++q) {
            const uint32_t m = uint32_t(n - d + q);
            const uint32_t t = uint32_t((uint64_t(w[q]) * (uint64_t(m) + 1)) >> 32);
            // is t already chosen?
            uint32_t h = (t * 2654435761u) >> (32 - hash_bits);
            bool taken = false;
            int probes = 0;
            while (table[h] != 0xffffffffu && probes < cap) {
                if (table[h] == t) {
                    taken = true;
                    break;
                }
                h = (h + 1) & mask;
                ++probes;
            }
            const uint32_t v = taken ? m : t;
            // insert v (m is never present yet: all chosen values so far are < m)
            h = (v * 2654435761u) >> (32 - hash_bits);
            probes = 0;
            while (table[h] != 0xffffffffu && probes < cap) {
                h = (h + 1) & mask;
                ++probes;
            }
            if (probes >= cap) {
                atomicOr(status, RSK_DEV_BOUNDS);
                return;
            }
            table[h] = v;
            if (rows) rows[q] = int32_t(v);
            if (rows64) rows64[q] = int64_t(v);
        }
    }
}

__global__ void k_srtt_dbits(int64_t nwords, uint64_t seed, uint32_t* __restrict__ out) {
    const int64_t wd = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (wd >= nwords) return;
    const rskd::Block4 b = rskd::philox_block(seed, kStreamD, uint64_t(wd >> 2), 0);
    out[wd] = b.v[wd & 3];
}

// ------------------------------------------------------------------------------------------
// The transform + gather kernel.
// ------------------------------------------------------------------------------------------
struct SrttArgs {
    const void* A;          // used by the plain-load path
    int64_t lda;
    int64_t n, k;
    int d, nblocks, nslices, nranges;
    const int32_t* prow;   // d selected rows
    void* partials;        // float or double [nranges][d][kpad]
    int64_t pstride, kpad;
    uint64_t seed;
    unsigned int* status;
};

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// 64 values held as v[x] for rows base + stride*x; butterflies over the 6 bits of x.
__device__ __forceinline__ void fwht64(float (&v)[64]) {
#pragma unroll
    for (int h = 1; h < 64; h <<= 1) {
#pragma unroll
        for (int x = 0; x < 64; ++x) {
            if ((x & h) == 0) {
                const float a = v[x], b = v[x + h];
                v[x] = a + b;
                v[x + h] = a - b;
            }
        }
    }
}
// 32 values per half: butterflies over the 5 bits of y inside each half of v.
__device__ __forceinline__ void fwht32x2(float (&v)[64]) {
#pragma unroll
    for (int h = 1; h < 32; h <<= 1) {
#pragma unroll
        for (int x = 0; x < 64; ++x) {
            if ((x & h) == 0 && ((x & 31) + h) < 32) {
                const float a = v[x], b = v[x + h];
                v[x] = a + b;
                v[x + h] = a - b;
            }
        }
    }
}

template <typename T, int QPT, bool TMA>
__global__ void __launch_bounds__(kThreads, 1) k_srtt(const __grid_constant__ CUtensorMap tmap, const SrttArgs a) {
    extern __shared__ __align__(128) uint8_t sm[];
    constexpr int kStageBytes = TMA ? kBlk * kCols * int(sizeof(T)) : 0;
    uint8_t* const stage0 = sm;
    uint8_t* const stage1 = sm + kStageBytes;
    float* Z = reinterpret_cast<float*>(sm + 2 * kStageBytes);
    uint32_t* dwords = reinterpret_cast<uint32_t*>(Z + kZFloats);  // 64 words of D for the block
    uint64_t* bars = reinterpret_cast<uint64_t*>(dwords + kBlk / 32);

    const int tid = threadIdx.x;
    int bidx = blockIdx.x;
    const int s = bidx % a.nslices;
    const int r = bidx / a.nslices;
    const int b0 = int(int64_t(r) * a.nblocks / a.nranges);
    const int b1 = int(int64_t(r + 1) * a.nblocks / a.nranges);

    // outputs of this thread: q = tid + 256*j
    int plo[QPT], phi[QPT];
    float acc[QPT][kCols];
#pragma unroll
    for (int j = 0; j < QPT; ++j) {
        const int q = tid + kThreads * j;
        const int p = q < a.d ? a.prow[q] : 0;
        plo[j] = p & (kBlk - 1);
        phi[j] = p >> 11;
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[j][c] = 0.f;
    }

    auto issue = [&](int blk, uint8_t* dst, uint64_t* bar) {
        const int64_t row0 = int64_t(blk) * kBlk;
        int nbox = 0;
        for (int bx = 0; bx < kBlk / kBoxRows; ++bx)
            if (row0 + bx * kBoxRows < a.n) ++nbox;
        rskd::mbar_expect_tx(bar, uint32_t(nbox * kBoxRows * kCols * sizeof(T)));
        for (int bx = 0; bx < nbox; ++bx)
            rskd::tma_load_2d(dst + bx * kBoxRows * kCols * sizeof(T), &tmap, s * kCols, int(row0 + bx * kBoxRows), bar);
    };
    if constexpr (TMA) {
        if (tid == 0) {
            rskd::mbar_init(&bars[0], 1);
            rskd::mbar_init(&bars[1], 1);
            rskd::fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0) {
            if (b0 < b1) issue(b0, stage0, &bars[0]);
            if (b0 + 1 < b1) issue(b0 + 1, stage1, &bars[1]);
        }
    }

    // pass-1 layout: column c1 = tid % 8, rows g1 + 32*x (x < 64), g1 = tid / 8
    const int c1 = tid & 7, g1 = tid >> 3;
    // pass-2 layout: column c2 = tid % 8, rows 32*(g2 + 32*h) + y (y < 32, h < 2), g2 = tid / 8
    const int c2 = tid & 7, g2 = tid >> 3;

    for (int blk = b0, it = 0; blk < b1; ++blk, ++it) {
        const int st = it & 1;
        // D words of this block (16 Philox blocks of 4 words)
        if (tid < 16) {
            const rskd::Block4 w = rskd::philox_block(a.seed, kStreamD, uint64_t(blk) * 16 + tid, 0);
            dwords[4 * tid + 0] = w.v[0];
            dwords[4 * tid + 1] = w.v[1];
            dwords[4 * tid + 2] = w.v[2];
            dwords[4 * tid + 3] = w.v[3];
        }
        bool ok = true;
        if constexpr (TMA) ok = rskd::mbar_wait(&bars[st], uint32_t((it >> 1) & 1), a.status);
        if (__syncthreads_or(!ok)) break;
        const T* raw = reinterpret_cast<const T*>(st ? stage1 : stage0);
        const T* gA = static_cast<const T*>(a.A);
        const int64_t row0 = int64_t(blk) * kBlk;
        const int64_t col = int64_t(s) * kCols + c1;
        float v[64];
        // pass 1: load, zero-pad beyond n (and beyond k), sign flip, stages on row bits 5..10
#pragma unroll
        for (int x = 0; x < 64; ++x) {
            const int row = g1 + 32 * x;
            float f;
            if constexpr (TMA)
                f = (row0 + row < a.n) ? to_f<T>(raw[row * kCols + c1]) : 0.f;
            else
                f = (row0 + row < a.n && col < a.k) ? to_f<T>(gA[(row0 + row) * a.lda + col]) : 0.f;
            const uint32_t neg = (dwords[row >> 5] >> (row & 31)) & 1u;
            v[x] = __uint_as_float(__float_as_uint(f) ^ (neg << 31));
        }
        fwht64(v);
#pragma unroll
        for (int x = 0; x < 64; ++x) Z[zoff(g1 + 32 * x) + c1] = v[x];
        __syncthreads();
        // stage buffer is free: refill it while the block is finished
        if (TMA && tid == 0 && blk + 2 < b1) {
            rskd::fence_proxy_async();
            issue(blk + 2, st ? stage1 : stage0, &bars[st]);
        }
        // pass 2: stages on row bits 0..4
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int y = 0; y < 32; ++y) v[32 * h + y] = Z[zoff(32 * (g2 + 32 * h) + y) + c2];
        fwht32x2(v);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int y = 0; y < 32; ++y) Z[zoff(32 * (g2 + 32 * h) + y) + c2] = v[32 * h + y];
        __syncthreads();
        // gather: Y[q] += (-1)^{popcount(p_hi & blk)} Z[p_lo]
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
            const float4* zr = reinterpret_cast<const float4*>(Z + zoff(plo[j]));
            const float4 z0 = zr[0], z1 = zr[1];
            const float sg = (__popc(uint32_t(phi[j]) & uint32_t(blk)) & 1) ? -1.f : 1.f;
            acc[j][0] += sg * z0.x;
            acc[j][1] += sg * z0.y;
            acc[j][2] += sg * z0.z;
            acc[j][3] += sg * z0.w;
            acc[j][4] += sg * z1.x;
            acc[j][5] += sg * z1.y;
            acc[j][6] += sg * z1.z;
            acc[j][7] += sg * z1.w;
        }
        __syncthreads();
    }

    float* part = static_cast<float*>(a.partials) + int64_t(r) * a.pstride;
#pragma unroll
    for (int j = 0; j < QPT; ++j) {
        const int q = tid + kThreads * j;
        if (q < a.d) {
            float4* dst = reinterpret_cast<float4*>(part + int64_t(q) * a.kpad + int64_t(s) * kCols);
            dst[0] = make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
            dst[1] = make_float4(acc[j][4], acc[j][5], acc[j][6], acc[j][7]);
        }
    }
}

template <typename Out>
__global__ void k_reduce_srtt(const float* __restrict__ partials, int64_t pstride, int64_t kpad, int nranges, int d,
                              int64_t k, double scale, Out* __restrict__ Y, int64_t ldy) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= int64_t(d) * k) return;
    const int64_t i = idx / k, col = idx - i * k;
    const float* p = partials + i * kpad + col;
    float sum = 0.f;
    for (int r = 0; r < nranges; ++r) sum += p[int64_t(r) * pstride];
    Y[i * ldy + col] = Out(double(sum) * scale);
}

int hash_bits_for(int d) {
    int b = 1;
    while ((1 << b) < 2 * d) ++b;
    return b;
}

rsk_status check_srtt(rsk_handle* h, int64_t n, int64_t d) {
    if (n < 1 || n >= (int64_t(1) << 31) || (n & (n - 1)))
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "SRTT needs n = 2^m < 2^31 (got %lld)", (long long)n);
    if (d < 1 || d > n || d > 8192)
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "SRTT needs 1 <= d <= min(n, 8192) (got %lld)", (long long)d);
    return RSK_OK;
}

rsk_status launch_draw(rsk_handle* h, int64_t n, int d, uint64_t seed, int32_t* rows, int64_t* rows64,
                       cudaStream_t stream) {
    const int hb = hash_bits_for(d);
    const size_t smem = (size_t(d) + (size_t(1) << hb)) * 4;
    RSK_CUDA_TRY(h, cudaFuncSetAttribute(k_srtt_draw, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_DENSE);
    k_srtt_draw<<<1, 1024, smem, stream>>>(n, d, seed, rows, rows64, hb, h->dev_status);
    rsk::prof_end(h, stream, pr);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

template <typename T, int QPT>
rsk_status launch_srtt_t(rsk_handle* h, const CUtensorMap& map, const SrttArgs& args, bool tma, cudaStream_t stream) {
    auto kern = tma ? k_srtt<T, QPT, true> : k_srtt<T, QPT, false>;
    const int smem = (tma ? 2 * kBlk * kCols * int(sizeof(T)) : 0) + kZFloats * 4 + (kBlk / 32) * 4 + 64;
    RSK_CUDA_TRY(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_SRTT_APPLY);
    kern<<<unsigned(args.nslices * args.nranges), kThreads, smem, stream>>>(map, args);
    rsk::prof_end(h, stream, pr);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

template <typename T>
rsk_status launch_srtt(rsk_handle* h, const CUtensorMap& map, const SrttArgs& args, bool tma, cudaStream_t stream) {
    const int qpt = (args.d + kThreads - 1) / kThreads;
    if (qpt <= 1) return launch_srtt_t<T, 1>(h, map, args, tma, stream);
    if (qpt <= 2) return launch_srtt_t<T, 2>(h, map, args, tma, stream);
    if (qpt <= 4) return launch_srtt_t<T, 4>(h, map, args, tma, stream);
    if (qpt <= 8) return launch_srtt_t<T, 8>(h, map, args, tma, stream);
    return rsk::fail(h, RSK_ERR_UNSUPPORTED, "SRTT apply supports d <= %d", 8 * kThreads);
}

}  // namespace

extern "C" {

rsk_status rsk_srtt_draw(rsk_handle* h, int64_t n, int64_t d, uint64_t seed, int64_t* rows, uint32_t* dbits,
                         cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    rsk_status st = check_srtt(h, n, d);
    if (st != RSK_OK) return st;
    if (rows) {
        st = launch_draw(h, n, int(d), seed, nullptr, rows, stream);
        if (st != RSK_OK) return st;
    }
    if (dbits) {
        const int64_t nw = (n + 31) / 32;
        k_srtt_dbits<<<unsigned((nw + 255) / 256), 256, 0, stream>>>(nw, seed, dbits);
        RSK_LAUNCH_CHECK(h);
    }
    return RSK_OK;
}

rsk_status rsk_srtt_apply(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k, int64_t lda,
                          int64_t d, uint64_t seed, void* Y, rsk_dtype y_dtype, int64_t ldy, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    rsk_status st = check_srtt(h, n, d);
    if (st != RSK_OK) return st;
    if (!A || !Y) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null matrix pointer");
    if (a_dtype != RSK_F32 && a_dtype != RSK_BF16)
        return rsk::fail(h, RSK_ERR_UNSUPPORTED, "SRTT apply takes F32 or BF16 input");
    if (y_dtype != RSK_F32 && y_dtype != RSK_F64) return rsk::fail(h, RSK_ERR_INVALID_ARG, "Y dtype must be F32 or F64");
    if (k < 1 || lda < k || ldy < k) return rsk::fail(h, RSK_ERR_INVALID_ARG, "need k >= 1, lda >= k, ldy >= k");
    const size_t es = rsk::dtype_size(a_dtype);
    bool tma = reinterpret_cast<uintptr_t>(A) % 16 == 0 && (lda * int64_t(es)) % 16 == 0;

    SrttArgs args;
    args.A = A;
    args.lda = lda;
    args.n = n;
    args.k = k;
    args.d = int(d);
    args.nblocks = int((n + kBlk - 1) / kBlk);
    args.nslices = int((k + kCols - 1) / kCols);
    args.nranges = std::max(1, std::min(args.nblocks, h->num_sms / args.nslices));
    args.kpad = int64_t(args.nslices) * kCols;
    args.pstride = int64_t(d) * args.kpad;
    args.seed = seed;
    args.status = h->dev_status;
    const size_t part_bytes = size_t(args.nranges) * args.pstride * 4;
    st = rsk::ensure_workspace(h, rsk::Carver::round(part_bytes) + rsk::Carver::round(size_t(d) * 4) + 512, stream);
    if (st != RSK_OK) return st;
    rsk::Carver cv(h->ws);
    int32_t* prow = cv.take<int32_t>(size_t(d));
    args.partials = cv.take<float>(size_t(args.nranges) * args.pstride);
    args.prow = prow;
    st = launch_draw(h, n, int(d), seed, prow, nullptr, stream);
    if (st != RSK_OK) return st;

    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    const CUtensorMapDataType tdt = a_dtype == RSK_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (tma) tma = rsk::encode_2d(h, &map, tdt, A, uint64_t(k), uint64_t(n), uint64_t(lda) * es, kCols, kBoxRows);
    st = a_dtype == RSK_F32 ? launch_srtt<float>(h, map, args, tma, stream)
                            : launch_srtt<__nv_bfloat16>(h, map, args, tma, stream);
    if (st != RSK_OK) return st;

    const int64_t total = d * k;
    const double scale = 1.0 / sqrt(double(d));
    const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_SRTT_REDUCE);
    if (y_dtype == RSK_F64)
        k_reduce_srtt<double><<<unsigned((total + 255) / 256), 256, 0, stream>>>(
            static_cast<const float*>(args.partials), args.pstride, args.kpad, args.nranges, int(d), k, scale,
            static_cast<double*>(Y), ldy);
    else
        k_reduce_srtt<float><<<unsigned((total + 255) / 256), 256, 0, stream>>>(
            static_cast<const float*>(args.partials), args.pstride, args.kpad, args.nranges, int(d), k, scale,
            static_cast<float*>(Y), ldy);
    rsk::prof_end(h, stream, pr);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

}  // extern "C"
