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
//   k_srtt_dbits_t the same bits transposed per 2048-row block, as the transform kernel reads them.
//   k_srtt_deal   one CTA: assigns the d output rows to the gather's slots so that the 8 lanes of each
//                 quarter-warp read 8 different shared-memory bank groups (no gather conflicts).
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
// floats after every 32 rows keeps both butterfly layouts free of bank conflicts), and its two
// 16-byte halves are swapped when bit 2 of r is set: a 16-byte load of a random row then falls on
// any of the 8 bank groups (not 4), while each butterfly access sees one permutation per warp.
constexpr int kZFloats = kBlk * kCols + (kBlk / 32) * kCols;
__device__ __forceinline__ int zoff(int r) { return r * kCols + kCols * (r >> 5); }
__device__ __forceinline__ int zswz(int r) { return ((r >> 2) & 1) << 2; }  // XOR on the column
__device__ __forceinline__ int zel(int r, int c) { return zoff(r) + (c ^ zswz(r)); }

// ------------------------------------------------------------------------------------------
// P and D.
// ------------------------------------------------------------------------------------------
// Floyd's sampling of d distinct rows of [0, n): step q (m = n - d + q) draws t = floor(w_q (m+1) / 2^32)
// and takes t unless an earlier step already holds it, in which case it takes m.  Every t is computed
// in parallel; a step can only find its t held if t >= n - d (an earlier m) or an earlier step drew
// the same t, so only those steps ("dirty", about d^2/n of them) are settled one after another in
// step order, each with one block-wide search of the earlier picks.  The picks equal those of the
// sequential loop.
__global__ void __launch_bounds__(1024) k_srtt_draw(int64_t n, int d, uint64_t seed, int32_t* __restrict__ rows,
                                                     int64_t* __restrict__ rows64, int hash_bits,
                                                     unsigned int* status) {
    extern __shared__ __align__(128) uint8_t sm[];
    uint32_t* pick = reinterpret_cast<uint32_t*>(sm);   // d values (t, then settled)
    uint32_t* keys = pick + d;                          // 2^hash_bits slots: t values
    int* first = reinterpret_cast<int*>(keys + (1 << hash_bits));  // first step drawing that t
    __shared__ int ndirty_s;
    __shared__ int dirty_s[1024];
    const int cap = 1 << hash_bits;
    const uint32_t mask = uint32_t(cap - 1);
    const uint32_t nd = uint32_t(n - d);
    for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        keys[i] = 0xffffffffu;
        first[i] = 0x7fffffff;
    }
    if (threadIdx.x == 0) ndirty_s = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < d; q += blockDim.x) {
        const rskd::Block4 b = rskd::philox_block(seed, kStreamP, 0, uint32_t(q >> 2));
        const uint32_t m = nd + uint32_t(q);
        const uint32_t t = uint32_t((uint64_t(b.v[q & 3]) * (uint64_t(m) + 1)) >> 32);
        pick[q] = t;
        // record the earliest step that drew t (t < 2^31, so 0xffffffff marks an empty slot)
        uint32_t h = (t * 2654435761u) >> (32 - hash_bits);
        for (int probe = 0; probe < cap; ++probe) {
            const uint32_t prev = atomicCAS(&keys[h], 0xffffffffu, t);
            if (prev == 0xffffffffu || prev == t) {
                atomicMin(&first[h], q);
                break;
            }
            h = (h + 1) & mask;
        }
    }
    __syncthreads();
    // dirty steps, collected in step order (a block-wide ordered compaction per 1024 steps)
    for (int base = 0; base < d; base += blockDim.x) {
        const int q = base + int(threadIdx.x);
        bool dirty = false;
        if (q < d) {
            const uint32_t t = pick[q];
            dirty = t >= nd;
            uint32_t h = (t * 2654435761u) >> (32 - hash_bits);
            for (int probe = 0; probe < cap && !dirty; ++probe) {
                if (keys[h] == t) {
                    dirty = first[h] < q;
                    break;
                }
                if (keys[h] == 0xffffffffu) break;
                h = (h + 1) & mask;
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, dirty);
        __shared__ int wcount[32];
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) wcount[w] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = ndirty_s;
            for (int i = 0; i < int(blockDim.x >> 5); ++i) {
                const int c = wcount[i];
                wcount[i] = acc;
                acc += c;
            }
            ndirty_s = acc;
        }
        __syncthreads();
        if (dirty) {
            const int slot = wcount[w] + __popc(bal & ((1u << l) - 1u));
            if (slot < 1024) dirty_s[slot] = q;
        }
        __syncthreads();
    }
    // settle the dirty steps in order (all steps when there are more than the list holds, as when
    // n is close to d); each is one block-wide search of the earlier picks
    const int ndirty = ndirty_s;
    const bool all = ndirty > 1024;
    const int count = all ? d : ndirty;
    for (int i = 0; i < count; ++i) {
        const int q = all ? i : dirty_s[i];
        const uint32_t t = pick[q];
        int hit = 0;
        for (int j = threadIdx.x; j < q; j += blockDim.x) hit |= pick[j] == t;
        if (__syncthreads_or(hit) && threadIdx.x == 0) pick[q] = nd + uint32_t(q);
        __syncthreads();
    }
    for (int q = threadIdx.x; q < d; q += blockDim.x) {
        if (rows) rows[q] = int32_t(pick[q]);
        if (rows64) rows64[q] = int64_t(pick[q]);
    }
    (void)status;
}

__global__ void k_srtt_dbits(int64_t nwords, uint64_t seed, uint32_t* __restrict__ out) {
    const int64_t wd = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (wd >= nwords) return;
    const rskd::Block4 b = rskd::philox_block(seed, kStreamD, uint64_t(wd >> 2), 0);
    out[wd] = b.v[wd & 3];
}

// D as the transform kernel reads it: per 2048-row block, word 2g + h holds the signs of rows
// g + 32 (32h + x), x = 0..31, in bit x (a 32 x 32 bit transpose of the block's natural words
// 32h .. 32h + 31, done with one ballot per bit).  One warp per (block, h).
// Block b of the output holds global block blk0 + b (row blocks of a row-sharded A).
__global__ void k_srtt_dbits_t(int64_t nblocks, uint64_t seed, int64_t blk0, uint32_t* __restrict__ out) {
    const int lane = threadIdx.x & 31, h = threadIdx.x >> 5;
    const int64_t b = blockIdx.x;
    if (b >= nblocks) return;
    const int64_t wd = (blk0 + b) * (kBlk / 32) + 32 * h + lane;  // natural word index: rows 32 wd .. 32 wd + 31
    const rskd::Block4 blk = rskd::philox_block(seed, kStreamD, uint64_t(wd >> 2), 0);
    const uint32_t word = blk.v[wd & 3];
    uint32_t mine = 0;
#pragma unroll
    for (int g = 0; g < 32; ++g) {
        const uint32_t t = __ballot_sync(0xffffffffu, (word >> g) & 1u);
        if (lane == g) mine = t;
    }
    out[b * (kBlk / 32) + 2 * lane + h] = mine;
}

// Bank group (16-byte unit modulo 8) of the first 16-byte load the gather makes for transformed
// row r; its second load falls on the group with the low bit flipped.
__host__ __device__ inline int gather_group(int r) { return 2 * ((r + (r >> 5)) & 3) + ((r >> 2) & 1); }

// Deal the d output rows to the gather's slots (slot tid + 256*j of k_srtt) so that the 8 lanes of
// every quarter-warp read 8 different bank groups: the i-th output row (in row order) whose sampled
// row falls in group g takes quarter i, lane g; rows beyond a group's share of quarters fill the
// quarters other groups left empty, in order.  Deterministic; every output row gets one slot.
__global__ void __launch_bounds__(1024) k_srtt_deal(const int32_t* __restrict__ prow, int d, int nslots,
                                                    int32_t* __restrict__ slot_q) {
    __shared__ int wc[32][8];
    __shared__ int base[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nq = nslots / 8;
    for (int s = tid; s < nslots; s += blockDim.x) slot_q[s] = -1;
    if (tid < 8) base[tid] = 0;
    __syncthreads();
    constexpr int kPer = 2;  // d <= 2048 = 2 * 1024
    int myg[kPer], myr[kPer];
#pragma unroll
    for (int c = 0; c < kPer; ++c) {
        const int q = c * 1024 + tid;
        const int g = q < d ? gather_group(prow[q] & (kBlk - 1)) : -1;
        int lrank = 0;
#pragma unroll
        for (int gg = 0; gg < 8; ++gg) {
            const unsigned bal = __ballot_sync(0xffffffffu, g == gg);
            if (lane == 0) wc[warp][gg] = __popc(bal);
            if (g == gg) lrank = __popc(bal & ((1u << lane) - 1u));
        }
        __syncthreads();
        if (tid < 8) {
            int acc = base[tid];
            for (int w = 0; w < 32; ++w) {
                const int t = wc[w][tid];
                wc[w][tid] = acc;
                acc += t;
            }
            base[tid] = acc;
        }
        __syncthreads();
        myg[c] = g;
        myr[c] = g >= 0 ? wc[warp][g] + lrank : 0;
        __syncthreads();
    }
    int hole_pre[9], ovf_pre[9];
    hole_pre[0] = ovf_pre[0] = 0;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        hole_pre[g + 1] = hole_pre[g] + max(0, nq - base[g]);
        ovf_pre[g + 1] = ovf_pre[g] + max(0, base[g] - nq);
    }
#pragma unroll
    for (int c = 0; c < kPer; ++c) {
        const int g = myg[c];
        if (g < 0) continue;
        int i = myr[c], l = g;
        if (i >= nq) {
            const int kk = ovf_pre[g] + (i - nq);
            int h = 0;
            while (h < 7 && hole_pre[h + 1] <= kk) ++h;
            i = base[h] + (kk - hole_pre[h]);
            l = h;
        }
        slot_q[8 * (i & 31) + l + 256 * (i >> 5)] = c * 1024 + tid;
    }
}

// ------------------------------------------------------------------------------------------
// The transform + gather kernel.
// ------------------------------------------------------------------------------------------
// Work items are (row band, column slice) pairs numbered band-major (item = band * nslices + slice);
// a band is nblocks / R consecutive 2048-row blocks.  Items are dealt round-robin to the CTAs, so the
// CTAs running together read the same rows (different 16- or 32-byte column slices of them, which
// then share DRAM sectors through L2).  Each item writes one partial [d][kCols]; the partials of a
// slice are summed in band order.
struct SrttArgs {
    const void* A;          // used by the plain-load path
    int64_t lda;
    int64_t n, k;            // rows of this A (a row block of the transform when blk0 > 0), columns
    int d, nblocks, nslices, R, nitems;
    int blk0;                // global index of this A's first 2048-row block
    const int32_t* prow;    // d selected rows
    const int32_t* slot_q;  // output row handled by slot tid + 256*j, or -1
    const uint32_t* dbits;  // nblocks * 64 words of D, transposed per block (k_srtt_dbits_t)
    float* partials;        // [item][d][kCols]
    int64_t pstride;        // d * kCols
    uint64_t seed;
    unsigned int* status;
    // SparseRTT: xi > 0 positions per output row (slot s = output row s), spos[i * nslots + s] =
    // position | (negative << 31); xi == 0 is the SRTT (one position per row, from prow/slot_q)
    int xi, nslots;
    const uint32_t* spos;
};

// Position in a CTA's sequence of (item, block): items blockIdx.x, + gridDim.x, ...
struct SrttCursor {
    int item, s, blk, b1;
};
__device__ __forceinline__ void cursor_item(const SrttArgs& a, SrttCursor& c, int item) {
    // bands are never empty (R <= nblocks), so one step always lands on a block
    c.item = item;
    if (item >= a.nitems) return;
    const int r = item / a.nslices;
    c.s = item - r * a.nslices;
    c.blk = int(int64_t(r) * a.nblocks / a.R);
    c.b1 = int(int64_t(r + 1) * a.nblocks / a.R);
}
__device__ __forceinline__ void cursor_next(const SrttArgs& a, SrttCursor& c) {
    if (++c.blk >= c.b1) cursor_item(a, c, c.item + int(gridDim.x));
}

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// 64 values held as v[x] for rows base + stride*x; butterflies over the 6 bits of x.  The values
// sit in register pairs (v[2i], v[2i+1]): the stage on bit 0 pairs the two halves of one register
// pair, every later stage pairs two whole register pairs, which one packed FP32x2 add and one packed
// subtract (fma by -1, exact) cover.
__device__ __forceinline__ float2 bf_sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ void fwht64(float2 (&w)[32]) {
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const float a = w[i].x, b = w[i].y;
        w[i] = make_float2(a + b, a - b);
    }
#pragma unroll
    for (int hh = 1; hh < 32; hh <<= 1) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            if ((i & hh) == 0) {
                const float2 a = w[i], b = w[i + hh];
                w[i] = __fadd2_rn(a, b);
                w[i + hh] = bf_sub2(a, b);
            }
        }
    }
}
// 32 values per half: butterflies over the 5 bits of y inside each half of v.
__device__ __forceinline__ void fwht32x2(float2 (&w)[32]) {
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const float a = w[i].x, b = w[i].y;
        w[i] = make_float2(a + b, a - b);
    }
#pragma unroll
    for (int hh = 1; hh < 16; hh <<= 1) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            if ((i & hh) == 0 && ((i & 15) + hh) < 16) {
                const float2 a = w[i], b = w[i + hh];
                w[i] = __fadd2_rn(a, b);
                w[i + hh] = bf_sub2(a, b);
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
    uint32_t* dwords = reinterpret_cast<uint32_t*>(Z + kZFloats);  // 64 words of D (plain-load path)
    uint32_t* dstage = dwords + kBlk / 32;                          // 2 x 64 words staged with the block (TMA)
    uint64_t* bars = reinterpret_cast<uint64_t*>(dstage + 2 * (kBlk / 32));

    const int tid = threadIdx.x;

    // outputs of this thread: q = tid + 256*j
    int plo[QPT], phi[QPT];
    float acc[QPT][kCols];
#pragma unroll
    for (int j = 0; j < QPT; ++j) {
        const int q = a.xi ? -1 : a.slot_q[tid + kThreads * j];
        const int p = q >= 0 ? a.prow[q] : 0;
        plo[j] = p & (kBlk - 1);
        phi[j] = p >> 11;
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[j][c] = 0.f;
    }

    auto issue = [&](const SrttCursor& c, uint8_t* dst, uint64_t* bar) {
        const int64_t row0 = int64_t(c.blk) * kBlk;
        int nbox = 0;
        for (int bx = 0; bx < kBlk / kBoxRows; ++bx)
            if (row0 + bx * kBoxRows < a.n) ++nbox;
        rskd::mbar_expect_tx(bar, uint32_t(nbox * kBoxRows * kCols * sizeof(T)) + uint32_t(kBlk / 32 * 4));
        for (int bx = 0; bx < nbox; ++bx)
            rskd::tma_load_2d(dst + bx * kBoxRows * kCols * sizeof(T), &tmap, c.s * kCols, int(row0 + bx * kBoxRows), bar);
        // the block's 64 words of D, drawn beforehand by k_srtt_dbits
        rskd::bulk_load(dstage + (dst == stage0 ? 0 : kBlk / 32), a.dbits + int64_t(c.blk) * (kBlk / 32),
                        uint32_t(kBlk / 32 * 4), bar);
    };
    SrttCursor cur, ahead;
    cursor_item(a, cur, int(blockIdx.x));
    ahead = cur;
    // copies issued into / completed waits on each stage (the same in every thread), so that a CTA
    // leaving early knows which stages may still receive bulk copies
    uint32_t issued0 = 0, issued1 = 0, waited0 = 0, waited1 = 0;
    if constexpr (TMA) {
        if (tid == 0) {
            rskd::mbar_init(&bars[0], 1);
            rskd::mbar_init(&bars[1], 1);
            rskd::fence_mbar_init();
        }
        __syncthreads();
        // two blocks in flight: `ahead` always points two positions past `cur`
        if (ahead.item < a.nitems) {
            if (tid == 0) issue(ahead, stage0, &bars[0]);
            ++issued0;
            cursor_next(a, ahead);
        }
        if (ahead.item < a.nitems) {
            if (tid == 0) issue(ahead, stage1, &bars[1]);
            ++issued1;
            cursor_next(a, ahead);
        }
    }
    auto flush = [&](int item) {
        float* part = a.partials + int64_t(item) * a.pstride;
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
            const int q = a.xi ? (tid + kThreads * j < a.d ? tid + kThreads * j : -1) : a.slot_q[tid + kThreads * j];
            if (q >= 0) {
                float4* dst = reinterpret_cast<float4*>(part + int64_t(q) * kCols);
                dst[0] = make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
                dst[1] = make_float4(acc[j][4], acc[j][5], acc[j][6], acc[j][7]);
            }
#pragma unroll
            for (int c = 0; c < kCols; ++c) acc[j][c] = 0.f;
        }
    };

    // pass-1 layout: column c1 = tid % 8, rows g1 + 32*x (x < 64), g1 = tid / 8
    const int c1 = tid & 7, g1 = tid >> 3;
    // pass-2 layout: column c2 = tid % 8, rows 32*(g2 + 32*h) + y (y < 32, h < 2), g2 = tid / 8
    const int c2 = tid & 7, g2 = tid >> 3;

    for (int it = 0; cur.item < a.nitems; ++it) {
        const int st = it & 1;
        const int s = cur.s;
        const int blk = cur.blk;
        // D words of this block (transposed layout): staged with the block on the TMA path
        if (!TMA && tid < kBlk / 32) dwords[tid] = a.dbits[int64_t(blk) * (kBlk / 32) + tid];
        bool ok = true;
        if constexpr (TMA) {
            ok = rskd::mbar_wait(&bars[st], uint32_t((it >> 1) & 1), a.status);
            if (ok) {
                if (st) ++waited1; else ++waited0;
            }
        }
        if (__syncthreads_or(!ok)) {
            if constexpr (TMA) {
                // a wait ran out: before the CTA (and its shared memory) goes away, wait once more,
                // bounded, for every copy still owed to a stage, so none lands after the exit
                if (tid == 0) {
                    if (issued0 > waited0) rskd::mbar_wait(&bars[0], waited0 & 1u, a.status);
                    if (issued1 > waited1) rskd::mbar_wait(&bars[1], waited1 & 1u, a.status);
                }
                __syncthreads();
            }
            break;
        }
        const uint32_t* dw = TMA ? dstage + st * (kBlk / 32) : dwords;
        const uint2 tw = *reinterpret_cast<const uint2*>(dw + 2 * g1);  // signs of rows g1 + 32x
        const T* raw = reinterpret_cast<const T*>(st ? stage1 : stage0);
        const T* gA = static_cast<const T*>(a.A);
        const int64_t row0 = int64_t(blk) * kBlk;
        const int64_t col = int64_t(s) * kCols + c1;
        float2 w[32];
        // pass 1: load, zero-pad beyond n (and beyond k), sign flip, stages on row bits 5..10
#pragma unroll
        for (int x = 0; x < 64; ++x) {
            const int row = g1 + 32 * x;
            float f;
            if constexpr (TMA)
                f = (row0 + row < a.n) ? to_f<T>(raw[row * kCols + c1]) : 0.f;
            else
                f = (row0 + row < a.n && col < a.k) ? to_f<T>(gA[(row0 + row) * a.lda + col]) : 0.f;
            const uint32_t sbit = ((x < 32 ? tw.x : tw.y) << (31 - (x & 31))) & 0x80000000u;
            const float fv = __uint_as_float(__float_as_uint(f) ^ sbit);
            if (x & 1) w[x >> 1].y = fv; else w[x >> 1].x = fv;
        }
        fwht64(w);
#pragma unroll
        for (int x = 0; x < 64; ++x) Z[zel(g1 + 32 * x, c1)] = (x & 1) ? w[x >> 1].y : w[x >> 1].x;
        __syncthreads();
        // stage buffer is free: refill it while the block is finished
        if (TMA && ahead.item < a.nitems) {
            if (tid == 0) {
                rskd::fence_proxy_async();
                issue(ahead, st ? stage1 : stage0, &bars[st]);
            }
            if (st) ++issued1; else ++issued0;
            cursor_next(a, ahead);
        }
        // pass 2: stages on row bits 0..4
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int y = 0; y < 32; y += 2)
                w[16 * h + (y >> 1)] = make_float2(Z[zel(32 * (g2 + 32 * h) + y, c2)], Z[zel(32 * (g2 + 32 * h) + y + 1, c2)]);
        fwht32x2(w);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int y = 0; y < 32; y += 2) {
                Z[zel(32 * (g2 + 32 * h) + y, c2)] = w[16 * h + (y >> 1)].x;
                Z[zel(32 * (g2 + 32 * h) + y + 1, c2)] = w[16 * h + (y >> 1)].y;
            }
        __syncthreads();
        if (a.xi) {
            // SparseRTT gather: Y[q] += sum_i rho_qi (-1)^{popcount(p_hi & blk)} Z[p_lo] over the xi
            // positions p = s_qi of output row q (slot q)
            const uint32_t gblk = uint32_t(a.blk0 + blk);
#pragma unroll
            for (int j = 0; j < QPT; ++j) {
                const int slot = tid + kThreads * j;
                if (slot >= a.d) continue;
                float2 s0 = make_float2(acc[j][0], acc[j][1]), s1 = make_float2(acc[j][2], acc[j][3]);
                float2 s2 = make_float2(acc[j][4], acc[j][5]), s3 = make_float2(acc[j][6], acc[j][7]);
                for (int i = 0; i < a.xi; ++i) {
                    const uint32_t w = __ldg(a.spos + int64_t(i) * a.nslots + slot);
                    const int lo = int(w & uint32_t(kBlk - 1));
                    const uint32_t hi = (w & 0x7fffffffu) >> 11;
                    const uint32_t neg = (w >> 31) ^ (__popc(hi & gblk) & 1u);
                    const float sg = neg ? -1.f : 1.f;
                    const float2 sg2 = make_float2(sg, sg);
                    const float4* zr = reinterpret_cast<const float4*>(Z + zoff(lo));
                    const int sw = (lo >> 2) & 1;
                    const float4 z0 = zr[sw], z1 = zr[sw ^ 1];
                    s0 = __ffma2_rn(make_float2(z0.x, z0.y), sg2, s0);
                    s1 = __ffma2_rn(make_float2(z0.z, z0.w), sg2, s1);
                    s2 = __ffma2_rn(make_float2(z1.x, z1.y), sg2, s2);
                    s3 = __ffma2_rn(make_float2(z1.z, z1.w), sg2, s3);
                }
                acc[j][0] = s0.x; acc[j][1] = s0.y; acc[j][2] = s1.x; acc[j][3] = s1.y;
                acc[j][4] = s2.x; acc[j][5] = s2.y; acc[j][6] = s3.x; acc[j][7] = s3.y;
            }
        } else {
        // gather: Y[q] += (-1)^{popcount(p_hi & blk)} Z[p_lo]
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
            const float4* zr = reinterpret_cast<const float4*>(Z + zoff(plo[j]));
            const int sw = (plo[j] >> 2) & 1;  // halves swapped for this row
            const float4 za = zr[sw], zb = zr[sw ^ 1];
            const float4 z0 = za, z1 = zb;
            const float sg = (__popc(uint32_t(phi[j]) & uint32_t(a.blk0 + blk)) & 1) ? -1.f : 1.f;
            const float2 sg2 = make_float2(sg, sg);
            float2 t0 = __ffma2_rn(make_float2(z0.x, z0.y), sg2, make_float2(acc[j][0], acc[j][1]));
            float2 t1 = __ffma2_rn(make_float2(z0.z, z0.w), sg2, make_float2(acc[j][2], acc[j][3]));
            float2 t2 = __ffma2_rn(make_float2(z1.x, z1.y), sg2, make_float2(acc[j][4], acc[j][5]));
            float2 t3 = __ffma2_rn(make_float2(z1.z, z1.w), sg2, make_float2(acc[j][6], acc[j][7]));
            acc[j][0] = t0.x; acc[j][1] = t0.y; acc[j][2] = t1.x; acc[j][3] = t1.y;
            acc[j][4] = t2.x; acc[j][5] = t2.y; acc[j][6] = t3.x; acc[j][7] = t3.y;
        }
        }
        __syncthreads();
        const int done_item = cur.item;
        cursor_next(a, cur);
        if (cur.item != done_item) flush(done_item);
    }
}

// Y[i, col] = scale * sum over bands of the partial of item (band, slice of col), in band order.
template <typename Out>
__global__ void k_reduce_srtt(const float* __restrict__ partials, int64_t pstride, int R, int nslices, int d,
                              int64_t k, double scale, Out* __restrict__ Y, int64_t ldy) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= int64_t(d) * k) return;
    const int64_t i = idx / k, col = idx - i * k;
    const int s = int(col / kCols);
    const float* p = partials + i * kCols + (col - int64_t(s) * kCols);
    float sum = 0.f;
    for (int r = 0; r < R; ++r) sum += p[(int64_t(r) * nslices + s) * pstride];
    Y[i * ldy + col] = Out(double(sum) * scale);
}

// SparseCol positions of SparseRTT (Def. SparseCol): output row q (a column of S) takes xi distinct
// positions of [0, n) by Floyd's algorithm with draws w_t = word(seed, 5, q, t), t < xi, and the
// sign of its t-th position is -1 iff bit t of w_xi is set.  One thread per output row.
constexpr uint32_t kStreamSparseCol = 5;
__global__ void k_sparsecol_draw(int64_t n, int d, int xi, uint64_t seed, int nslots, uint32_t* __restrict__ spos,
                                 int32_t* __restrict__ pos_out, uint32_t* __restrict__ signs_out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= d) return;
    uint32_t w[36];
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        if (4 * b <= xi) {
            const rskd::Block4 blk = rskd::philox_block(seed, kStreamSparseCol, uint64_t(q), uint32_t(b));
            w[4 * b + 0] = blk.v[0];
            w[4 * b + 1] = blk.v[1];
            w[4 * b + 2] = blk.v[2];
            w[4 * b + 3] = blk.v[3];
        }
    }
    uint32_t sb = 0;
#pragma unroll
    for (int t = 0; t <= 32; ++t)
        if (t == xi) sb = w[t];
    uint32_t p[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        if (t < xi) {
            const uint32_t m = uint32_t(n - xi + t);
            const uint32_t v = uint32_t((uint64_t(w[t]) * (uint64_t(m) + 1)) >> 32);
            bool taken = false;
#pragma unroll
            for (int r = 0; r < t; ++r) taken |= (p[r] == v);
            p[t] = taken ? m : v;
            const uint32_t neg = (sb >> t) & 1u;
            spos[int64_t(t) * nslots + q] = p[t] | (neg << 31);
            if (pos_out) pos_out[int64_t(q) * xi + t] = int32_t(p[t]);
        }
    }
    if (signs_out) signs_out[q] = xi >= 32 ? sb : (sb & ((1u << xi) - 1u));
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

// SparseRTT: n = 2^m (the WHT), 1 <= xi <= min(n, 32) positions per output row, and at most 2048
// output rows (the gather's register slots).
rsk_status check_sparse_rtt(rsk_handle* h, int64_t n, int64_t d, int xi) {
    if (n < 1 || n >= (int64_t(1) << 31) || (n & (n - 1)))
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "SparseRTT needs n = 2^m < 2^31 (got %lld)", (long long)n);
    if (d < 1 || d > 8 * kThreads)
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "SparseRTT needs 1 <= d <= %d (got %lld)", 8 * kThreads, (long long)d);
    if (xi < 1 || xi > 32 || xi > n)
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "SparseRTT needs 1 <= xi <= min(n, 32) (got %d)", xi);
    return RSK_OK;
}

rsk_status srtt_impl(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n_rows, int64_t k, int64_t lda,
                     int64_t row0, int64_t n, int64_t d, int xi, uint64_t seed, void* Y, rsk_dtype y_dtype,
                     int64_t ldy, cudaStream_t stream);

rsk_status launch_draw(rsk_handle* h, int64_t n, int d, uint64_t seed, int32_t* rows, int64_t* rows64,
                       cudaStream_t stream) {
    const int hb = hash_bits_for(d);
    const size_t smem = (size_t(d) + 2 * (size_t(1) << hb)) * 4;
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
    const int smem = (tma ? 2 * kBlk * kCols * int(sizeof(T)) : 0) + kZFloats * 4 + 3 * (kBlk / 32) * 4 + 64;
    RSK_CUDA_TRY(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_SRTT_APPLY);
    kern<<<unsigned(std::min(args.nitems, h->num_sms)), kThreads, smem, stream>>>(map, args);
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
    return rsk_srtt_apply_rows(h, A, a_dtype, n, k, lda, 0, n, d, seed, Y, y_dtype, ldy, stream);
}

rsk_status rsk_srtt_apply_rows(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n_rows, int64_t k,
                               int64_t lda, int64_t row0, int64_t n, int64_t d, uint64_t seed, void* Y,
                               rsk_dtype y_dtype, int64_t ldy, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    return srtt_impl(h, A, a_dtype, n_rows, k, lda, row0, n, d, 0, seed, Y, y_dtype, ldy, stream);
}

int32_t rsk_sparse_rtt_default_xi(int64_t d) {
    if (d < 1) return 0;
    const int xi = int(ceil(1.5 * log(double(d)) - 1e-12));
    return xi < 1 ? 1 : (xi > 32 ? 32 : xi);
}

rsk_status rsk_sparse_rtt_draw(rsk_handle* h, int64_t n, int64_t d, int32_t xi, uint64_t seed, int32_t* positions,
                               uint32_t* sign_bits, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (xi == 0) xi = rsk_sparse_rtt_default_xi(d);
    rsk_status st = check_sparse_rtt(h, n, d, xi);
    if (st != RSK_OK) return st;
    if (!positions && !sign_bits) return RSK_OK;
    st = rsk::ensure_workspace(h, size_t(d) * xi * 4 + 256, stream);
    if (st != RSK_OK) return st;
    k_sparsecol_draw<<<unsigned((d + 127) / 128), 128, 0, stream>>>(n, int(d), xi, seed, int(d),
                                                                    static_cast<uint32_t*>(h->ws), positions, sign_bits);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

rsk_status rsk_sparse_rtt_apply(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k, int64_t lda,
                                int64_t d, int32_t xi, uint64_t seed, void* Y, rsk_dtype y_dtype, int64_t ldy,
                                cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (xi == 0) xi = rsk_sparse_rtt_default_xi(d);
    rsk_status st = check_sparse_rtt(h, n, d, xi);
    if (st != RSK_OK) return st;
    return srtt_impl(h, A, a_dtype, n, k, lda, 0, n, d, xi, seed, Y, y_dtype, ldy, stream);
}

}  // extern "C"

namespace {
rsk_status srtt_impl(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n_rows, int64_t k, int64_t lda,
                     int64_t row0, int64_t n, int64_t d, int xi, uint64_t seed, void* Y, rsk_dtype y_dtype,
                     int64_t ldy, cudaStream_t stream) {
    rsk_status st = xi ? RSK_OK : check_srtt(h, n, d);
    if (st != RSK_OK) return st;
    if (n_rows < 1 || row0 < 0 || row0 % kBlk != 0 || row0 + n_rows > n)
        return rsk::fail(h, RSK_ERR_INVALID_ARG,
                         "row block [%lld, %lld) must start at a multiple of %d and lie in [0, n = %lld)",
                         (long long)row0, (long long)(row0 + n_rows), kBlk, (long long)n);
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
    args.n = n_rows;
    args.k = k;
    args.d = int(d);
    args.nblocks = int((n_rows + kBlk - 1) / kBlk);
    args.blk0 = int(row0 / kBlk);
    args.nslices = int((k + kCols - 1) / kCols);
    // bands: R = num_sms / gcd(nslices, num_sms) makes nslices * R a multiple of the SM count
    int gg = args.nslices, hh = h->num_sms;
    while (hh) {
        const int t_ = gg % hh;
        gg = hh;
        hh = t_;
    }
    args.R = std::max(1, std::min(args.nblocks, h->num_sms / gg));
    const int tuned = rsk::tuned_value(h, rsk::kTuneSrtt, int(a_dtype), n_rows, k, d);
    if (tuned > 0) args.R = std::max(1, std::min(args.nblocks, tuned));
    args.nitems = args.nslices * args.R;
    args.pstride = int64_t(d) * kCols;
    args.seed = seed;
    args.status = h->dev_status;
    const size_t part_bytes = size_t(args.nitems) * args.pstride * 4;
    const int64_t ndw = int64_t(args.nblocks) * (kBlk / 32);
    // gather slots: kThreads x QPT, QPT the power of two launch_srtt picks for d
    const int qpt_need = (int(d) + kThreads - 1) / kThreads;
    const int nslots = kThreads * (qpt_need <= 1 ? 1 : qpt_need <= 2 ? 2 : qpt_need <= 4 ? 4 : 8);
    args.xi = xi;
    args.nslots = nslots;
    st = rsk::ensure_workspace(h, rsk::Carver::round(part_bytes) + rsk::Carver::round(size_t(d) * 4) +
                                      rsk::Carver::round(size_t(ndw) * 4) + rsk::Carver::round(size_t(nslots) * 4) +
                                      rsk::Carver::round(size_t(nslots) * size_t(xi) * 4) + 768,
                               stream);
    if (st != RSK_OK) return st;
    rsk::Carver cv(h->ws);
    int32_t* prow = cv.take<int32_t>(size_t(d));
    args.partials = cv.take<float>(size_t(args.nitems) * args.pstride);
    uint32_t* dbits = cv.take<uint32_t>(size_t(ndw));
    int32_t* slot_q = cv.take<int32_t>(size_t(nslots));
    uint32_t* spos = cv.take<uint32_t>(size_t(nslots) * size_t(xi));
    k_srtt_dbits_t<<<unsigned(args.nblocks), 64, 0, stream>>>(args.nblocks, seed, int64_t(args.blk0), dbits);
    args.dbits = dbits;
    args.prow = prow;
    args.spos = spos;
    if (xi) {
        // SparseRTT: xi SparseCol positions per output row; slot s is output row s
        k_sparsecol_draw<<<unsigned((d + 127) / 128), 128, 0, stream>>>(n, int(d), xi, seed, nslots, spos, nullptr,
                                                                        nullptr);
        RSK_LAUNCH_CHECK(h);
    } else {
        st = launch_draw(h, n, int(d), seed, prow, nullptr, stream);
        if (st != RSK_OK) return st;
        if (d <= 8 * kThreads) {
            k_srtt_deal<<<1, 1024, 0, stream>>>(prow, int(d), nslots, slot_q);
            RSK_LAUNCH_CHECK(h);
        }
    }
    args.slot_q = slot_q;

    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    const CUtensorMapDataType tdt = a_dtype == RSK_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (tma) tma = rsk::encode_2d(h, &map, tdt, A, uint64_t(k), uint64_t(n_rows), uint64_t(lda) * es, kCols, kBoxRows);
    st = a_dtype == RSK_F32 ? launch_srtt<float>(h, map, args, tma, stream)
                            : launch_srtt<__nv_bfloat16>(h, map, args, tma, stream);
    if (st != RSK_OK) return st;

    const int64_t total = d * k;
    const double scale = 1.0 / sqrt(double(d) * double(xi ? xi : 1));
    const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_SRTT_REDUCE);
    if (y_dtype == RSK_F64)
        k_reduce_srtt<double><<<unsigned((total + 255) / 256), 256, 0, stream>>>(
            args.partials, args.pstride, args.R, args.nslices, int(d), k, scale, static_cast<double*>(Y), ldy);
    else
        k_reduce_srtt<float><<<unsigned((total + 255) / 256), 256, 0, stream>>>(
            args.partials, args.pstride, args.R, args.nslices, int(d), k, scale, static_cast<float*>(Y), ldy);
    rsk::prof_end(h, stream, pr);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

}  // namespace

