// Sparse sign embedding (left form of the paper's SparseUniform, Def. "SparseUniform", Sec. 3.2.1):
// drawing S, inverting its column->row map into a chunked CSR, and the deterministic gather
// S*A for tall A (cost O(zeta nnz(A)), Sec. 3.2).
//
// Kernels
//   k_generate  one thread per column j: Philox words -> Floyd sample of zeta distinct rows + signs.
//   k_index     one CTA per chunk of C columns (C = 768 for zeta <= 8): redraws the chunk's columns,
//               counts per sketch row, scans, scatters (j_local | neg<<15) through shared-memory
//               atomics, then sorts each sketch row's short list by j, so every sketch row lists its
//               columns in ascending j whatever order the atomics took.  Output is chunk-local.
//   k_apply     persistent CTAs (at most one per SM) over (range of chunks, 128-byte column slice, block
//               of sketch rows) items, numbered range-major and dealt round-robin.  Per chunk,
//               TMA streams the chunk's row slices of A and bulk copies bring the chunk's index into
//               shared memory (double buffered, one mbarrier per stage).  A group of 8 lanes owns
//               SLOTS consecutive sketch rows and gathers their entries' row slices (16 B per lane,
//               one 128-byte line per group: no bank conflicts), accumulating in registers.
//   k_reduce    sums the per-range partials in range order, scales by zeta^{-1/2}, casts, writes SA.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "common.cuh"
#include "philox.cuh"

namespace {

constexpr int kBoxRows = 128;       // rows per TMA box
constexpr int kRowBytes = 128;      // staged row slice of A
constexpr int kMaxChunkEntries = 6144;
constexpr int kApplyThreads = 512;
constexpr int kGroups = kApplyThreads / 8;
constexpr int kIndexThreads = 256;
constexpr uint32_t kStreamLeft = 0;

// Columns of S (= rows of A) per chunk: 768 for zeta <= 8, fewer for larger zeta so that a chunk
// holds at most kMaxChunkEntries entries (16-bit offsets, bounded shared memory).
__host__ __device__ inline int chunk_rows(int zeta) {
    int c = (kMaxChunkEntries / zeta) / kBoxRows * kBoxRows;
    return c > 768 ? 768 : (c < kBoxRows ? kBoxRows : c);
}
// Offsets of one chunk are stored with a row pitch that keeps every row 16-byte aligned.
__host__ __device__ inline int offsets_pitch(int d) { return (d + 1 + 7) & ~7; }
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline size_t align128(size_t x) { return (x + 127) & ~size_t(127); }

// ------------------------------------------------------------------------------------------
// Drawing one column of S.
// ------------------------------------------------------------------------------------------
// Column distributions: SparseUniform (Def. SparseUniform: zeta rows uniform without replacement,
// Floyd's algorithm) and SparseStack (Def. SparseStack: zeta stacked CountSketches, one row drawn
// uniformly in each block of b = d / zeta consecutive rows: row q*b + floor(w_q * b / 2^32)).
enum ColumnKind : int { kUniform = 0, kStack = 1 };
constexpr uint32_t kStreamStack = 4;

template <int ZMAX>
__device__ __forceinline__ void draw_column(uint64_t seed, uint32_t stream, uint64_t j, int d, int zeta,
                                            int (&rows)[ZMAX], uint32_t& negbits, int kind = kUniform) {
    uint32_t w[ZMAX + 4];
#pragma unroll
    for (int b = 0; b <= ZMAX / 4; ++b) {
        if (4 * b <= zeta) {
            const rskd::Block4 blk = rskd::philox_block(seed, stream, j, uint32_t(b));
            w[4 * b + 0] = blk.v[0];
            w[4 * b + 1] = blk.v[1];
            w[4 * b + 2] = blk.v[2];
            w[4 * b + 3] = blk.v[3];
        }
    }
    if (kind == kStack) {
        // one row per block of b rows: distinct by construction
        const uint32_t b = uint32_t(d / zeta);
#pragma unroll
        for (int q = 0; q < ZMAX; ++q)
            if (q < zeta) rows[q] = int(uint32_t(q) * b + __umulhi(w[q], b));
    } else {
        // Floyd: for m = d-zeta .. d-1 draw t uniform in [0, m]; keep t unless already taken, else m.
#pragma unroll
        for (int q = 0; q < ZMAX; ++q) {
            if (q < zeta) {
                const uint32_t m = uint32_t(d - zeta + q);
                const int t = int(__umulhi(w[q], m + 1u));
                bool taken = false;
#pragma unroll
                for (int p = 0; p < q; ++p) taken |= (rows[p] == t);
                rows[q] = taken ? int(m) : t;
            }
        }
    }
    uint32_t sb = 0;
#pragma unroll
    for (int t = 0; t <= ZMAX; ++t)
        if (t == zeta) sb = w[t];
    negbits = zeta >= 32 ? sb : (sb & ((1u << zeta) - 1u));
}

template <int ZMAX>
__global__ void k_generate(int64_t n, int d, int zeta, uint64_t seed, uint32_t stream, int32_t* __restrict__ rows,
                           uint32_t* __restrict__ signs, int kind) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int r[ZMAX];
    uint32_t nb;
    draw_column<ZMAX>(seed, stream, uint64_t(j), d, zeta, r, nb, kind);
    if (rows) {
#pragma unroll
        for (int q = 0; q < ZMAX; ++q)
            if (q < zeta) rows[j * zeta + q] = r[q];
    }
    if (signs) signs[j] = nb;
}

// ------------------------------------------------------------------------------------------
// Chunked inverted index.
// ------------------------------------------------------------------------------------------
struct IndexLayout {
    size_t tgt_off, neg_off, cnt_off, beg_off, out_off, scan_off, total;
};

__host__ __device__ inline IndexLayout index_layout(int d, int zeta) {
    const int C = chunk_rows(zeta);
    IndexLayout L;
    L.tgt_off = 0;
    L.neg_off = align16(L.tgt_off + size_t(C) * zeta * 2);
    L.cnt_off = align16(L.neg_off + size_t(C) * 4);
    L.beg_off = align16(L.cnt_off + size_t(d) * 4);
    L.out_off = align16(L.beg_off + size_t(d + 1) * 4);
    L.scan_off = align16(L.out_off + size_t(C) * zeta * 2);
    L.total = align16(L.scan_off + 2 * 32 * 4);
    return L;
}

template <int ZMAX>
__global__ void __launch_bounds__(kIndexThreads) k_index(int64_t n, int d, int zeta, uint64_t seed, uint32_t stream,
                                                         int64_t col0, int kind, uint16_t* __restrict__ offsets,
                                                         uint16_t* __restrict__ entries) {
    extern __shared__ __align__(16) uint8_t sm[];
    const IndexLayout L = index_layout(d, zeta);
    uint16_t* tgt = reinterpret_cast<uint16_t*>(sm + L.tgt_off);
    uint32_t* neg = reinterpret_cast<uint32_t*>(sm + L.neg_off);
    unsigned int* cnt = reinterpret_cast<unsigned int*>(sm + L.cnt_off);
    int* beg = reinterpret_cast<int*>(sm + L.beg_off);
    uint16_t* out = reinterpret_cast<uint16_t*>(sm + L.out_off);
    int* wsum = reinterpret_cast<int*>(sm + L.scan_off);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int C = chunk_rows(zeta);
    const int pitch = offsets_pitch(d);
    const int64_t ch = blockIdx.x;
    const int64_t j0 = ch * C;
    const int rows = int((n - j0) < C ? (n - j0) : C);
    const int nent = rows * zeta;

    // 1. draw the chunk's columns (global column col0 + j0 + r of S)
    for (int r = tid; r < rows; r += kIndexThreads) {
        int rr[ZMAX];
        uint32_t nb;
        draw_column<ZMAX>(seed, stream, uint64_t(col0 + j0 + r), d, zeta, rr, nb, kind);
        if (ZMAX == 8 && zeta == 8) {
            uint4 pk;
            pk.x = uint32_t(rr[0]) | (uint32_t(rr[1 % ZMAX]) << 16);
            pk.y = uint32_t(rr[2 % ZMAX]) | (uint32_t(rr[3 % ZMAX]) << 16);
            pk.z = uint32_t(rr[4 % ZMAX]) | (uint32_t(rr[5 % ZMAX]) << 16);
            pk.w = uint32_t(rr[6 % ZMAX]) | (uint32_t(rr[7 % ZMAX]) << 16);
            reinterpret_cast<uint4*>(tgt)[r] = pk;
        } else {
#pragma unroll
            for (int q = 0; q < ZMAX; ++q)
                if (q < zeta) tgt[r * zeta + q] = uint16_t(rr[q]);
        }
        neg[r] = nb;
    }
    for (int i = tid; i < d; i += kIndexThreads) cnt[i] = 0;
    __syncthreads();

    // 2. entries per sketch row
    for (int f = tid; f < nent; f += kIndexThreads) atomicAdd(&cnt[tgt[f]], 1u);
    __syncthreads();

    // 3. exclusive scan over sketch rows (warp w scans [w*R, (w+1)*R), lanes on consecutive rows)
    constexpr int kWarps = kIndexThreads / 32;
    const int R = (((d + kWarps - 1) / kWarps) + 31) & ~31;
    const int t0 = min(d, warp * R), t1 = min(d, t0 + R);
    int carry = 0;
    constexpr int kIt = (8192 / kWarps + 31) / 32;  // d <= 8192
    int tots[kIt];
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
        const int base = t0 + 32 * it;
        if (base >= t1) break;
        const int i = base + lane;
        const int tot = i < t1 ? int(cnt[i]) : 0;
        tots[it] = tot;
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) wsum[warp] = carry;
    __syncthreads();
    if (warp == 0) {
        const int v = lane < kWarps ? wsum[lane] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane < kWarps) wsum[32 + lane] = incl - v;
    }
    __syncthreads();
    carry = wsum[32 + warp];
    uint16_t* off_out = offsets + ch * pitch;
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
        const int base = t0 + 32 * it;
        if (base >= t1) break;
        const int i = base + lane;
        const int tot = tots[it];
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (i < t1) {
            const int run = carry + incl - tot;
            off_out[i] = uint16_t(run);
            beg[i] = run;
            cnt[i] = unsigned(run);
        }
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (tid == 0) beg[d] = nent;
    for (int i = d + tid; i < pitch; i += kIndexThreads) off_out[i] = uint16_t(nent);
    __syncthreads();

    // 4. scatter in any order (the slot a shared-memory atomic hands out)
    for (int f = tid; f < nent; f += kIndexThreads) {
        const int r = f / zeta, q = f - r * zeta;
        const unsigned pos = atomicAdd(&cnt[tgt[f]], 1u);
        out[pos] = uint16_t(r | (((neg[r] >> q) & 1u) << 15));
    }
    __syncthreads();

    // 5. order each sketch row's entries by column (columns within a row are distinct, so the
    //    order is unique): insertion sort of the short per-row lists
    for (int i = tid; i < d; i += kIndexThreads) {
        const int b = beg[i], e = beg[i + 1];
        for (int a = b + 1; a < e; ++a) {
            const uint16_t v = out[a];
            const int key = v & 0x7fff;
            int k = a;
            while (k > b && int(out[k - 1] & 0x7fff) > key) {
                out[k] = out[k - 1];
                --k;
            }
            out[k] = v;
        }
    }
    __syncthreads();

    // 6. write the chunk's entries (chunk blocks start at multiples of C*zeta*2 bytes, 16-aligned)
    uint16_t* dst = entries + ch * C * zeta;
    const int n16 = (nent * 2) / 16;
    for (int v = tid; v < n16; v += kIndexThreads)
        reinterpret_cast<uint4*>(dst)[v] = reinterpret_cast<const uint4*>(out)[v];
    for (int e = n16 * 8 + tid; e < nent; e += kIndexThreads) dst[e] = out[e];
}

// ------------------------------------------------------------------------------------------
// Gather apply.
// ------------------------------------------------------------------------------------------
// Per-lane accumulator of one sketch row over the lane's 16-byte column segment.  add() takes
// the 16 staged bytes of one entry and its sign bit.
struct AccF64 {
    static constexpr int kVec = 2;
    using store_t = double;
    double v[2];
    __device__ __forceinline__ void zero() { v[0] = v[1] = 0.0; }
    __device__ __forceinline__ void add(const uint4 x, uint32_t negative) {
        const uint32_t sm = negative << 31;
        v[0] += __hiloint2double(int(x.y ^ sm), int(x.x));
        v[1] += __hiloint2double(int(x.w ^ sm), int(x.z));
    }
    __device__ __forceinline__ void store(double* dst) const {
        dst[0] = v[0];
        dst[1] = v[1];
    }
};
struct AccF32 {
    static constexpr int kVec = 4;
    using store_t = float;
    float2 v[2];
    __device__ __forceinline__ void zero() { v[0] = v[1] = make_float2(0.f, 0.f); }
    __device__ __forceinline__ void add(const uint4 x, uint32_t negative) {
        const float s = __uint_as_float(0x3f800000u | (negative << 31));
        const float2 s2 = make_float2(s, s);
        v[0] = __ffma2_rn(make_float2(__uint_as_float(x.x), __uint_as_float(x.y)), s2, v[0]);
        v[1] = __ffma2_rn(make_float2(__uint_as_float(x.z), __uint_as_float(x.w)), s2, v[1]);
    }
    __device__ __forceinline__ void store(float* dst) const {
        reinterpret_cast<float4*>(dst)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    }
};
// bf16 entries are accumulated with the mixed-precision FMA acc = x * s + acc (x and s bf16, acc
// FP32), s = +-1 carrying the sign: the product is exact, so each step rounds once, exactly like an
// FP32 add of the widened entry, at one instruction per element and no unpacking.
struct AccBF16 {
    static constexpr int kVec = 8;
    using store_t = float;
    float2 v[4];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = make_float2(0.f, 0.f);
    }
    // acc += (low or high bf16 half of w) * s, s the bf16 pattern in the low 16 bits of `one`
    __device__ __forceinline__ static void fma_lo(float& acc, uint32_t w, uint32_t one) {
        asm("{\n\t.reg .b16 lo, hi, s;\n\tmov.b32 {lo, hi}, %1;\n\tcvt.u16.u32 s, %2;\n\t"
            "fma.rn.f32.bf16 %0, lo, s, %0;\n\t}"
            : "+f"(acc)
            : "r"(w), "r"(one));
    }
    __device__ __forceinline__ static void fma_hi(float& acc, uint32_t w, uint32_t one) {
        asm("{\n\t.reg .b16 lo, hi, s;\n\tmov.b32 {lo, hi}, %1;\n\tcvt.u16.u32 s, %2;\n\t"
            "fma.rn.f32.bf16 %0, hi, s, %0;\n\t}"
            : "+f"(acc)
            : "r"(w), "r"(one));
    }
    __device__ __forceinline__ void add(const uint4 x, uint32_t negative) {
        const uint32_t one = 0x3f80u | (negative << 15);  // bf16 +1 or -1
        fma_lo(v[0].x, x.x, one);
        fma_hi(v[0].y, x.x, one);
        fma_lo(v[1].x, x.y, one);
        fma_hi(v[1].y, x.y, one);
        fma_lo(v[2].x, x.z, one);
        fma_hi(v[2].y, x.z, one);
        fma_lo(v[3].x, x.w, one);
        fma_hi(v[3].y, x.w, one);
    }
    __device__ __forceinline__ void store(float* dst) const {
        reinterpret_cast<float4*>(dst)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        reinterpret_cast<float4*>(dst)[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
    }
};

// Interleaved double-float element: a = hi + lo (both FP32).
struct __align__(8) DF2 {
    float hi, lo;
    __host__ __device__ DF2() {}
    __host__ __device__ DF2(int) : hi(0.f), lo(0.f) {}
};
// Double-float accumulation of (hi, lo) pairs (Knuth's exact sum on the high parts), two pairs per
// 16 bytes; the partial is stored as the FP64 value hi + lo.
struct AccDF {
    static constexpr int kVec = 2;
    using store_t = double;
    float h[2], l[2];
    __device__ __forceinline__ void zero() { h[0] = h[1] = l[0] = l[1] = 0.f; }
    __device__ __forceinline__ static void acc1(float& hh, float& ll, float ah, float al) {
        const float s = hh + ah;
        const float bb = s - hh;
        float e = (hh - (s - bb)) + (ah - bb);
        e += ll + al;
        hh = s + e;
        ll = e - (hh - s);
    }
    __device__ __forceinline__ void add(const uint4 x, uint32_t negative) {
        const uint32_t sm = negative << 31;
        acc1(h[0], l[0], __uint_as_float(x.x ^ sm), __uint_as_float(x.y ^ sm));
        acc1(h[1], l[1], __uint_as_float(x.z ^ sm), __uint_as_float(x.w ^ sm));
    }
    __device__ __forceinline__ void store(double* dst) const {
        dst[0] = double(h[0]) + double(l[0]);
        dst[1] = double(h[1]) + double(l[1]);
    }
};

template <typename T>
struct Elem;
template <>
struct Elem<DF2> {
    using acc = AccDF;
};
template <>
struct Elem<double> {
    using acc = AccF64;
};
template <>
struct Elem<float> {
    using acc = AccF32;
};
template <>
struct Elem<__nv_bfloat16> {
    using acc = AccBF16;
};

struct ApplyArgs {
    const void* A;
    int64_t n, k, lda;
    int d, zeta, chunk, pitch, dsub, ntsub, nslices, nranges, nchunks, nitems;
    const uint16_t* offs;
    const uint16_t* ents;
    void* partials;
    int64_t pstride, kpad;
    unsigned int* status;
};

struct StageLayout {
    int a_bytes, e_bytes, o_bytes, bytes;
};
__host__ __device__ inline StageLayout stage_layout(int chunk, int zeta, int dsub) {
    StageLayout L;
    L.a_bytes = chunk * kRowBytes;
    L.e_bytes = int(align16(size_t(chunk) * zeta * 2));
    L.o_bytes = (dsub + 8) * 2;
    L.bytes = int(align128(size_t(L.a_bytes) + L.e_bytes + L.o_bytes));
    return L;
}

// Loads the SLOTS+1 offsets of one group from shared memory (SLOTS >= 8: 16-byte aligned).
template <int SLOTS>
__device__ __forceinline__ void load_offsets(const uint16_t* o, int (&out)[SLOTS + 1]) {
    if constexpr (SLOTS >= 8) {
#pragma unroll
        for (int b = 0; b < SLOTS / 8; ++b) {
            const uint4 v = reinterpret_cast<const uint4*>(o)[b];
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                out[8 * b + 2 * h] = int(w[h] & 0xffffu);
                out[8 * b + 2 * h + 1] = int(w[h] >> 16);
            }
        }
        out[SLOTS] = o[SLOTS];
    } else {
#pragma unroll
        for (int q = 0; q <= SLOTS; ++q) out[q] = o[q];
    }
}

template <typename T, int SLOTS, bool TMA>
__global__ void __launch_bounds__(kApplyThreads, 1)
    k_apply(const __grid_constant__ CUtensorMap tmap, const ApplyArgs a) {
    using Acc = typename Elem<T>::acc;
    constexpr int VEC = Acc::kVec;
    constexpr int C_COLS = 8 * VEC;  // columns of A per slice (128 bytes)
    extern __shared__ __align__(128) uint8_t sm[];
    const StageLayout SL = stage_layout(a.chunk, a.zeta, a.dsub);
    uint8_t* const stage0 = sm;
    uint8_t* const stage1 = sm + SL.bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + (TMA ? 2 : 1) * SL.bytes);

    const int tid = threadIdx.x, g = tid >> 3, l8 = tid & 7;
    // Work items are (row range, column slice, block of sketch rows), numbered range-major; CTA b
    // takes items b, b + gridDim.x, ...  The CTAs running together therefore work on the same rows.
    const int pairs = a.nslices * a.ntsub;
    struct Cursor {
        int item, r, s, t, ch, c1;
    };
    auto set_item = [&](Cursor& c, int item) {
        c.item = item;
        if (item >= a.nitems) return;
        c.r = item / pairs;
        const int pr = item - c.r * pairs;
        c.t = pr / a.nslices;
        c.s = pr - c.t * a.nslices;
        c.ch = int(int64_t(c.r) * a.nchunks / a.nranges);  // ranges are never empty (nranges <= nchunks)
        c.c1 = int(int64_t(c.r + 1) * a.nchunks / a.nranges);
    };
    auto advance = [&](Cursor& c) {
        if (++c.ch >= c.c1) set_item(c, c.item + int(gridDim.x));
    };

    Acc acc[SLOTS];
#pragma unroll
    for (int q = 0; q < SLOTS; ++q) acc[q].zero();

    auto issue = [&](const Cursor& c, uint8_t* dst, uint64_t* bar) {
        const int64_t row0 = int64_t(c.ch) * a.chunk;
        const int rows = int((a.n - row0) < a.chunk ? (a.n - row0) : a.chunk);
        const int nbox = (rows + kBoxRows - 1) / kBoxRows;
        const uint32_t eb = uint32_t(align16(size_t(rows) * a.zeta * 2));
        rskd::mbar_expect_tx(bar, uint32_t(nbox * kBoxRows * kRowBytes) + eb + uint32_t(SL.o_bytes));
        for (int bx = 0; bx < nbox; ++bx)
            rskd::tma_load_2d(dst + bx * kBoxRows * kRowBytes, &tmap, c.s * C_COLS, int(row0 + bx * kBoxRows), bar);
        rskd::bulk_load(dst + SL.a_bytes, a.ents + row0 * a.zeta, eb, bar);
        rskd::bulk_load(dst + SL.a_bytes + SL.e_bytes, a.offs + int64_t(c.ch) * a.pitch + int64_t(c.t) * a.dsub,
                        uint32_t(SL.o_bytes), bar);
    };

    Cursor cur, ahead;
    set_item(cur, int(blockIdx.x));
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
        // two chunks in flight: `ahead` always points two positions past `cur`
        if (ahead.item < a.nitems) {
            if (tid == 0) issue(ahead, stage0, &bars[0]);
            ++issued0;
            advance(ahead);
        }
        if (ahead.item < a.nitems) {
            if (tid == 0) issue(ahead, stage1, &bars[1]);
            ++issued1;
            advance(ahead);
        }
    }

    for (int it = 0; cur.item < a.nitems; ++it) {
        const int ch = cur.ch, s = cur.s, t = cur.t;
        const int first = t * a.dsub + g * SLOTS;  // this group's sketch rows: first .. first+SLOTS-1
        const uint8_t* buf;
        bool ok = true;
        if constexpr (TMA) {
            const int st = it & 1;
            // every thread waits on the stage's barrier itself (that is what makes the TMA writes
            // visible to it); a timeout skips the chunk and ends the loop at the barrier below
            ok = rskd::mbar_wait(&bars[st], uint32_t((it >> 1) & 1), a.status);
            if (ok) {
                if (st) ++waited1; else ++waited0;
            }
            buf = st ? stage1 : stage0;
        } else {
            // A not TMA-compatible: plain loads into the single stage.
            const T* A = static_cast<const T*>(a.A);
            const int64_t row0 = int64_t(ch) * a.chunk;
            for (int idx = tid; idx < a.chunk * 8; idx += kApplyThreads) {
                const int row = idx >> 3, piece = idx & 7;
                const int64_t gr = row0 + row;
                __align__(16) T vals[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    const int64_t col = int64_t(s) * C_COLS + piece * VEC + v;
                    vals[v] = (gr < a.n && col < a.k) ? A[gr * a.lda + col] : T(0);
                }
                *reinterpret_cast<uint4*>(stage0 + row * kRowBytes + piece * 16) = *reinterpret_cast<const uint4*>(vals);
            }
            const int rows = int((a.n - row0) < a.chunk ? (a.n - row0) : a.chunk);
            uint16_t* es = reinterpret_cast<uint16_t*>(stage0 + SL.a_bytes);
            for (int e = tid; e < rows * a.zeta; e += kApplyThreads) es[e] = a.ents[row0 * a.zeta + e];
            uint16_t* os = reinterpret_cast<uint16_t*>(stage0 + SL.a_bytes + SL.e_bytes);
            for (int e = tid; e < a.dsub + 8; e += kApplyThreads)
                os[e] = a.offs[int64_t(ch) * a.pitch + int64_t(t) * a.dsub + e];
            __syncthreads();
            buf = stage0;
        }
        if (ok) {
            const uint16_t* es = reinterpret_cast<const uint16_t*>(buf + SL.a_bytes);
            const uint16_t* os = reinterpret_cast<const uint16_t*>(buf + SL.a_bytes + SL.e_bytes);
            const uint8_t* lane_base = buf + l8 * 16;
            int o[SLOTS + 1];
            load_offsets<SLOTS>(os + g * SLOTS, o);
#pragma unroll
            for (int q = 0; q < SLOTS; ++q) {
                if (first + q < a.d) {
                    const int end = o[q + 1];
                    for (int e = o[q]; e < end; e += 4) {
                        uint32_t v[4];
                        uint4 x[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) v[u] = es[e + u];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (e + u < end) x[u] = *reinterpret_cast<const uint4*>(lane_base + (v[u] & 0x7fffu) * kRowBytes);
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (e + u < end) acc[q].add(x[u], v[u] >> 15);
                    }
                }
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
        if constexpr (TMA) {
            if (ahead.item < a.nitems) {
                const int st = it & 1;
                if (tid == 0) {
                    rskd::fence_proxy_async();
                    issue(ahead, st ? stage1 : stage0, &bars[st]);
                }
                if (st) ++issued1; else ++issued0;
                advance(ahead);
            }
        }
        const int done_item = cur.item, done_r = cur.r;
        advance(cur);
        if (cur.item != done_item) {
            // item finished: its partial sums go to the row range's slot, then start afresh
            using store_t = typename Acc::store_t;
            store_t* part = static_cast<store_t*>(a.partials) + int64_t(done_r) * a.pstride;
#pragma unroll
            for (int q = 0; q < SLOTS; ++q) {
                const int i = first + q;
                if (i < a.d) acc[q].store(part + int64_t(i) * a.kpad + int64_t(s) * C_COLS + l8 * VEC);
                acc[q].zero();
            }
        }
    }
}

template <typename Acc, typename Out>
__global__ void k_reduce(const Acc* __restrict__ partials, int64_t pstride, int64_t kpad, int nranges, int d,
                         int64_t k, double scale, Out* __restrict__ SA, int64_t ldsa) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= int64_t(d) * k) return;
    const int64_t i = idx / k, col = idx - i * k;
    const Acc* p = partials + i * kpad + col;
    Acc sum = Acc(0);
    for (int r = 0; r < nranges; ++r) sum += p[int64_t(r) * pstride];
    SA[i * ldsa + col] = Out(double(sum) * scale);
}

// SA = sum over blocks of the per-block sketches (d x k packed, block stride bstride), in order.
template <typename Out>
__global__ void k_sum_blocks(const Out* __restrict__ outs, int64_t bstride, int nblk, int d, int64_t k,
                             Out* __restrict__ SA, int64_t ldsa) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= int64_t(d) * k) return;
    const int64_t i = idx / k, col = idx - i * k;
    Out acc = Out(0);
    for (int b = 0; b < nblk; ++b) acc += outs[int64_t(b) * bstride + idx];
    SA[i * ldsa + col] = acc;
}

// ------------------------------------------------------------------------------------------
// Right sketch Y = A Omega = A S^T (A n x dc row-major, S k x dc): Y[i, c] = zeta^{-1/2} sum over the
// entries (j, sign) of row c of S of sign * A[i, j].  One CTA per tile of 32 rows of A at a time;
// per index chunk the tile's 32 x C block of A is staged transposed ([j][i], lane index XOR-swizzled
// by j so that the gathers are free of bank conflicts; rows read with 16-byte loads), and warp w
// accumulates output columns w, w + 8, ... for its 32 rows (lane = row): every lane of a warp walks
// the same entry list, so the gather does not diverge.  Chunks are summed in order (deterministic).
// ------------------------------------------------------------------------------------------
constexpr int kRightRows = 32;
constexpr int kRightThreads = 256;

template <int MAXC>
__global__ void __launch_bounds__(kRightThreads, 2)
    k_right(const float* __restrict__ A, int64_t n, int64_t dc, int64_t lda, int k, int zeta, int C, int pitch,
            const uint16_t* __restrict__ offs, const uint16_t* __restrict__ ents, int nchunks, float scale,
            float* __restrict__ Y, int64_t ldy, int vec4) {
    extern __shared__ __align__(16) uint8_t smr[];
    float* tile = reinterpret_cast<float*>(smr);                                   // C x 32
    uint16_t* es = reinterpret_cast<uint16_t*>(smr + size_t(C) * kRightRows * 4);  // C * zeta entries
    uint16_t* os = es + size_t(C) * zeta;                                          // k + 1 offsets
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ntiles = (n + kRightRows - 1) / kRightRows;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t i0 = t * kRightRows;
        float acc[MAXC];
#pragma unroll
        for (int cc = 0; cc < MAXC; ++cc) acc[cc] = 0.f;
        for (int ch = 0; ch < nchunks; ++ch) {
            const int64_t j0 = int64_t(ch) * C;
            const int cols = int(min(int64_t(C), dc - j0));
            if (vec4) {
                // warp w stages rows w, w + 8, ...; lanes take 16-byte column groups (coalesced rows)
                const int c4n = (cols + 3) >> 2;
                for (int r = warp; r < kRightRows; r += kRightThreads / 32) {
                    const bool live = i0 + r < n;
                    const float* arow = A + (i0 + r) * lda + j0;
#pragma unroll 4
                    for (int c4 = lane; c4 < c4n; c4 += 32) {
                        const int c = 4 * c4;
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (live) {
                            if (c + 4 <= cols) v = *reinterpret_cast<const float4*>(arow + c);
                            else {
                                v.x = arow[c];
                                if (c + 1 < cols) v.y = arow[c + 1];
                                if (c + 2 < cols) v.z = arow[c + 2];
                            }
                        }
                        tile[c * kRightRows + (r ^ (c & 31))] = v.x;
                        tile[(c + 1) * kRightRows + (r ^ ((c + 1) & 31))] = v.y;
                        tile[(c + 2) * kRightRows + (r ^ ((c + 2) & 31))] = v.z;
                        tile[(c + 3) * kRightRows + (r ^ ((c + 3) & 31))] = v.w;
                    }
                }
            } else {
                for (int idx = tid; idx < kRightRows * cols; idx += kRightThreads) {
                    const int r = idx / cols, c = idx - r * cols;
                    const float v = (i0 + r < n) ? A[(i0 + r) * lda + j0 + c] : 0.f;
                    tile[c * kRightRows + (r ^ (c & 31))] = v;
                }
            }
            const uint16_t* ce = ents + j0 * zeta;
            for (int e = tid; e < cols * zeta; e += kRightThreads) es[e] = ce[e];
            const uint16_t* co = offs + int64_t(ch) * pitch;
            for (int e = tid; e <= k; e += kRightThreads) os[e] = co[e];
            __syncthreads();
#pragma unroll
            for (int cc = 0; cc < MAXC; ++cc) {
                const int c = warp + 8 * cc;
                if (c < k) {
                    const int b = os[c], end = os[c + 1];
                    float a = acc[cc];
                    for (int e = b; e < end; ++e) {
                        const uint32_t v = es[e];
                        const int j = int(v & 0x7fffu);
                        const float x = tile[j * kRightRows + (lane ^ (j & 31))];
                        a += (v & 0x8000u) ? -x : x;
                    }
                    acc[cc] = a;
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int cc = 0; cc < MAXC; ++cc) {
            const int c = warp + 8 * cc;
            if (c < k && i0 + lane < n) Y[int64_t(c) * ldy + i0 + lane] = acc[cc] * scale;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Host side.
// ------------------------------------------------------------------------------------------
rsk_status check_dims(rsk_handle* h, int64_t n, int64_t d, int32_t zeta) {
    if (n < 1 || n >= (int64_t(1) << 31)) return rsk::fail(h, RSK_ERR_INVALID_ARG, "n=%lld out of range", (long long)n);
    if (d < 1 || d > 8192) return rsk::fail(h, RSK_ERR_INVALID_ARG, "d=%lld out of range [1, 8192]", (long long)d);
    if (zeta < 1 || zeta > 32 || zeta > d)
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "zeta=%d must satisfy 1 <= zeta <= min(d, 32)", zeta);
    return RSK_OK;
}

// SparseStack needs d to be a whole number of blocks: d = b * zeta.
rsk_status check_stack_dims(rsk_handle* h, int64_t n, int64_t d, int32_t zeta) {
    rsk_status st = check_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    if (d % zeta != 0)
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "SparseStack needs d = b * zeta (d=%lld, zeta=%d)", (long long)d, zeta);
    return RSK_OK;
}

int64_t n_chunks_of(int64_t n, int zeta) { return (n + chunk_rows(zeta) - 1) / chunk_rows(zeta); }

// Index storage: offsets (n_chunks rows of pitch entries, plus a tail so that any target-block
// window of the apply kernel stays in bounds) and entries (n*zeta, plus 16 bytes).
size_t offsets_count(int64_t n, int d, int zeta) { return size_t(n_chunks_of(n, zeta)) * offsets_pitch(d) + 8192 + 16; }
size_t entries_count(int64_t n, int zeta) { return size_t(n) * zeta + 16; }

rsk_status launch_index(rsk_handle* h, int64_t n, int d, int zeta, uint64_t seed, uint32_t stream_id,
                        uint16_t* offs, uint16_t* ents, cudaStream_t stream, int64_t col0 = 0, int kind = kUniform) {
    const IndexLayout L = index_layout(d, zeta);
    if (L.total > 227 * 1024) return rsk::fail(h, RSK_ERR_UNSUPPORTED, "index build needs %zu B of shared memory", L.total);
    const int64_t nch = n_chunks_of(n, zeta);
    auto go = [&](auto kern) -> rsk_status {
        RSK_CUDA_TRY(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L.total)));
        const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_SKETCH_INDEX);
        kern<<<unsigned(nch), kIndexThreads, L.total, stream>>>(n, d, zeta, seed, stream_id, col0, kind, offs, ents);
        rsk::prof_end(h, stream, pr);
        RSK_LAUNCH_CHECK(h);
        return RSK_OK;
    };
    if (zeta <= 8) return go(k_index<8>);
    if (zeta <= 16) return go(k_index<16>);
    return go(k_index<32>);
}

struct ApplyPlan {
    int slots, dsub, ntsub, nslices, nranges, nchunks, chunk, pitch, nitems;
    int64_t kpad, pstride;
    size_t partial_bytes;
};

ApplyPlan plan_apply(rsk_handle* h, int64_t n, int64_t k, int d, int zeta, rsk_dtype dt) {
    ApplyPlan p;
    const int vec = int(16 / rsk::dtype_size(dt));
    const int C = 8 * vec;
    const int max_slots = dt == RSK_BF16 ? 8 : 16;
    p.ntsub = (d + max_slots * kGroups - 1) / (max_slots * kGroups);
    const int need = (d + p.ntsub * kGroups - 1) / (p.ntsub * kGroups);
    p.slots = 1;
    while (p.slots < need) p.slots *= 2;
    p.dsub = p.slots * kGroups;
    p.nslices = int((k + C - 1) / C);
    p.chunk = chunk_rows(zeta);
    p.pitch = offsets_pitch(d);
    p.nchunks = int(n_chunks_of(n, zeta));
    const int pairs = p.nslices * p.ntsub;
    p.kpad = int64_t(p.nslices) * C;
    p.pstride = int64_t(p.ntsub) * p.dsub * p.kpad;
    const size_t acc = (dt == RSK_F64 || dt == RSK_F32X2) ? 8 : 4;
    // row ranges R with R * pairs a multiple of the SM count (R = num_sms / gcd(pairs, num_sms)), so
    // that the persistent CTAs get equal shares of (range, slice, sketch-row block) items; at most one
    // range per chunk and at most 512 MB of partial sums
    int gg = pairs, hh = h->num_sms;
    while (hh) {
        const int t_ = gg % hh;
        gg = hh;
        hh = t_;
    }
    int R = pairs >= h->num_sms ? 1 : h->num_sms / std::max(1, gg);
    const int tuned = rsk::tuned_value(h, rsk::kTuneApply, int(dt), n, k, d);
    if (tuned > 0) R = tuned;
    const int64_t cap = std::max<int64_t>(1, int64_t(512) * (1 << 20) / int64_t(p.pstride * acc));
    R = int(std::min<int64_t>(std::min<int64_t>(R, cap), p.nchunks));
    p.nranges = std::max(1, R);
    p.nitems = p.nranges * pairs;
    p.partial_bytes = size_t(p.nranges) * p.pstride * acc;
    return p;
}

template <typename T, int SLOTS>
rsk_status launch_apply_t(rsk_handle* h, const ApplyPlan& p, const ApplyArgs& args, bool use_tma,
                          const CUtensorMap& map, cudaStream_t stream) {
    const unsigned grid = unsigned(std::min(p.nitems, h->num_sms));
    const StageLayout SL = stage_layout(p.chunk, args.zeta, p.dsub);
    const int smem = (use_tma ? 2 : 1) * SL.bytes + 64;
    if (smem > 227 * 1024) return rsk::fail(h, RSK_ERR_UNSUPPORTED, "apply needs %d B of shared memory", smem);
    auto kern = use_tma ? k_apply<T, SLOTS, true> : k_apply<T, SLOTS, false>;
    RSK_CUDA_TRY(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_SKETCH_APPLY);
    kern<<<grid, kApplyThreads, smem, stream>>>(map, args);
    rsk::prof_end(h, stream, pr);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

template <typename T>
rsk_status launch_apply_slots(rsk_handle* h, const ApplyPlan& p, const ApplyArgs& args, bool use_tma,
                              const CUtensorMap& map, cudaStream_t stream) {
    switch (p.slots) {
        case 1: return launch_apply_t<T, 1>(h, p, args, use_tma, map, stream);
        case 2: return launch_apply_t<T, 2>(h, p, args, use_tma, map, stream);
        case 4: return launch_apply_t<T, 4>(h, p, args, use_tma, map, stream);
        case 8: return launch_apply_t<T, 8>(h, p, args, use_tma, map, stream);
        default:
            if constexpr (sizeof(T) >= 4) return launch_apply_t<T, 16>(h, p, args, use_tma, map, stream);
            return rsk::fail(h, RSK_ERR_INTERNAL, "bad slot count %d", p.slots);
    }
}

template <typename Acc>
rsk_status launch_reduce(rsk_handle* h, const ApplyPlan& p, const void* partials, int d, int64_t k, int zeta,
                         void* SA, rsk_dtype sa_dt, int64_t ldsa, cudaStream_t stream) {
    const int64_t total = int64_t(d) * k;
    const unsigned grid = unsigned((total + 255) / 256);
    const double scale = 1.0 / sqrt(double(zeta));
    const Acc* P = static_cast<const Acc*>(partials);
    const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_SKETCH_REDUCE);
    if (sa_dt == RSK_F64)
        k_reduce<Acc, double><<<grid, 256, 0, stream>>>(P, p.pstride, p.kpad, p.nranges, d, k, scale,
                                                        static_cast<double*>(SA), ldsa);
    else
        k_reduce<Acc, float><<<grid, 256, 0, stream>>>(P, p.pstride, p.kpad, p.nranges, d, k, scale,
                                                       static_cast<float*>(SA), ldsa);
    rsk::prof_end(h, stream, pr);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

rsk_status apply_with_index(rsk_handle* h, const uint16_t* offs, const uint16_t* ents, const void* A,
                            rsk_dtype a_dt, int64_t n, int64_t k, int64_t lda, int d, int zeta, void* SA,
                            rsk_dtype sa_dt, int64_t ldsa, void* partials, const ApplyPlan& p, cudaStream_t stream) {
    const size_t es = rsk::dtype_size(a_dt);
    const int C = int(128 / es);
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    bool use_tma = (reinterpret_cast<uintptr_t>(A) % 16 == 0) && ((lda * int64_t(es)) % 16 == 0);
    if (use_tma) {
        const CUtensorMapDataType tdt = (a_dt == RSK_F64 || a_dt == RSK_F32X2) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                        : a_dt == RSK_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                          : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
        use_tma = rsk::encode_2d(h, &map, tdt, A, uint64_t(k), uint64_t(n), uint64_t(lda) * es, uint32_t(C),
                                 uint32_t(kBoxRows));
    }
    ApplyArgs args;
    args.A = A;
    args.n = n;
    args.k = k;
    args.lda = lda;
    args.d = d;
    args.zeta = zeta;
    args.chunk = p.chunk;
    args.pitch = p.pitch;
    args.dsub = p.dsub;
    args.ntsub = p.ntsub;
    args.nslices = p.nslices;
    args.nranges = p.nranges;
    args.nchunks = p.nchunks;
    args.nitems = p.nitems;
    args.offs = offs;
    args.ents = ents;
    args.partials = partials;
    args.pstride = p.pstride;
    args.kpad = p.kpad;
    args.status = h->dev_status;
    rsk_status st;
    if (a_dt == RSK_F64) st = launch_apply_slots<double>(h, p, args, use_tma, map, stream);
    else if (a_dt == RSK_F32X2) st = launch_apply_slots<DF2>(h, p, args, use_tma, map, stream);
    else if (a_dt == RSK_F32) st = launch_apply_slots<float>(h, p, args, use_tma, map, stream);
    else st = launch_apply_slots<__nv_bfloat16>(h, p, args, use_tma, map, stream);
    if (st != RSK_OK) return st;
    if (a_dt == RSK_F64 || a_dt == RSK_F32X2)
        return launch_reduce<double>(h, p, partials, d, k, zeta, SA, sa_dt, ldsa, stream);
    return launch_reduce<float>(h, p, partials, d, k, zeta, SA, sa_dt, ldsa, stream);
}

rsk_status check_apply_args(rsk_handle* h, const void* A, int a_dt, int64_t k, int64_t lda, const void* SA,
                            int sa_dt, int64_t ldsa) {
    if (!A || !SA) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null matrix pointer");
    if (!rsk::sketch_dtype_ok(a_dt)) return rsk::fail(h, RSK_ERR_INVALID_ARG, "bad A dtype %d", a_dt);
    if (sa_dt != RSK_F64 && sa_dt != RSK_F32) return rsk::fail(h, RSK_ERR_INVALID_ARG, "SA dtype must be F64 or F32");
    if (k < 1 || lda < k || ldsa < k) return rsk::fail(h, RSK_ERR_INVALID_ARG, "need k >= 1, lda >= k, ldsa >= k");
    return RSK_OK;
}

rsk_status generate_kind(rsk_handle* h, int64_t n, int d, int zeta, uint64_t seed, uint32_t stream_id, int kind,
                         int32_t* rows, uint32_t* signs, cudaStream_t stream) {
    const unsigned grid = unsigned((n + 255) / 256);
    const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_SKETCH_GENERATE);
    if (zeta <= 8) k_generate<8><<<grid, 256, 0, stream>>>(n, d, zeta, seed, stream_id, rows, signs, kind);
    else if (zeta <= 16) k_generate<16><<<grid, 256, 0, stream>>>(n, d, zeta, seed, stream_id, rows, signs, kind);
    else k_generate<32><<<grid, 256, 0, stream>>>(n, d, zeta, seed, stream_id, rows, signs, kind);
    rsk::prof_end(h, stream, pr);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

// Index build + gather apply for the columns row0 .. row0 + n - 1 of a sketch of the given kind.
rsk_status apply_kind(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k, int64_t lda,
                      int64_t row0, int64_t d, int32_t zeta, uint64_t seed, void* SA, rsk_dtype sa_dtype,
                      int64_t ldsa, cudaStream_t stream, uint32_t stream_id, int kind);

}  // namespace

struct rsk_sketch_plan {
    int64_t n, d;
    int zeta;
    uint64_t seed;
    int64_t nchunks;
    uint16_t* offs;
    uint16_t* ents;
};

namespace rsk {
size_t sketch_partial_bytes(rsk_handle* h, int64_t n, int64_t k, int64_t d, int zeta, rsk_dtype a_dt) {
    return plan_apply(h, n, k, int(d), zeta, a_dt).partial_bytes;
}
rsk_status sketch_plan_apply_ws(rsk_handle* h, const rsk_sketch_plan* plan, const void* A, rsk_dtype a_dt, int64_t k,
                                int64_t lda, void* SA, rsk_dtype sa_dt, int64_t ldsa, void* partials,
                                cudaStream_t stream) {
    rsk_status st = check_apply_args(h, A, a_dt, k, lda, SA, sa_dt, ldsa);
    if (st != RSK_OK) return st;
    const ApplyPlan p = plan_apply(h, plan->n, k, int(plan->d), plan->zeta, a_dt);
    return apply_with_index(h, plan->offs, plan->ents, A, a_dt, plan->n, k, lda, int(plan->d), plan->zeta, SA, sa_dt,
                            ldsa, partials, p, stream);
}
// Every argument check of rsk_sparse_sign_apply, without a launch (h may be null: no message).
rsk_status sketch_check_args(rsk_handle* h, const void* A, rsk_dtype a_dt, int64_t n, int64_t k, int64_t lda,
                             int64_t d, int zeta, const void* SA, rsk_dtype sa_dt, int64_t ldsa) {
    rsk_status st = check_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    return check_apply_args(h, A, a_dt, k, lda, SA, sa_dt, ldsa);
}
// Scratch bytes of one sparse sign apply when the inverted index and the partials are carved from a
// single caller-provided buffer, and the apply that uses such a buffer.
size_t sketch_scratch_bytes(rsk_handle* h, int64_t n, int64_t k, int64_t d, int zeta, rsk_dtype a_dt) {
    const ApplyPlan p = plan_apply(h, n, k, int(d), zeta, a_dt);
    return Carver::round(offsets_count(n, int(d), zeta) * 2) + Carver::round(entries_count(n, zeta) * 2) +
           Carver::round(p.partial_bytes) + 256;
}
rsk_status sketch_apply_scratch(rsk_handle* h, const void* A, rsk_dtype a_dt, int64_t n, int64_t k, int64_t lda,
                                int64_t d, int zeta, uint64_t seed, void* SA, rsk_dtype sa_dt, int64_t ldsa,
                                void* scratch, cudaStream_t stream) {
    rsk_status st = check_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    st = check_apply_args(h, A, a_dt, k, lda, SA, sa_dt, ldsa);
    if (st != RSK_OK) return st;
    const ApplyPlan p = plan_apply(h, n, k, int(d), zeta, a_dt);
    Carver cv(scratch);
    uint16_t* offs = cv.take<uint16_t>(offsets_count(n, int(d), zeta));
    uint16_t* ents = cv.take<uint16_t>(entries_count(n, zeta));
    void* partials = cv.take<char>(p.partial_bytes);
    st = launch_index(h, n, int(d), zeta, seed, kStreamLeft, offs, ents, stream);
    if (st != RSK_OK) return st;
    return apply_with_index(h, offs, ents, A, a_dt, n, k, lda, int(d), zeta, SA, sa_dt, ldsa, partials, p, stream);
}
// Index built once into caller memory, then applied to several right-hand sides.
size_t sketch_index_bytes(int64_t n, int64_t d, int zeta) {
    return Carver::round(offsets_count(n, int(d), zeta) * 2) + Carver::round(entries_count(n, zeta) * 2) + 256;
}
rsk_status sketch_build_index(rsk_handle* h, int64_t n, int64_t d, int zeta, uint64_t seed, void* index_mem,
                              cudaStream_t stream) {
    rsk_status st = check_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    Carver cv(index_mem);
    uint16_t* offs = cv.take<uint16_t>(offsets_count(n, int(d), zeta));
    uint16_t* ents = cv.take<uint16_t>(entries_count(n, zeta));
    return launch_index(h, n, int(d), zeta, seed, kStreamLeft, offs, ents, stream);
}
rsk_status sketch_apply_built(rsk_handle* h, const void* index_mem, int64_t n, int64_t d, int zeta, const void* A,
                              rsk_dtype a_dt, int64_t k, int64_t lda, void* SA, rsk_dtype sa_dt, int64_t ldsa,
                              void* partials, cudaStream_t stream) {
    rsk_status st = check_apply_args(h, A, a_dt, k, lda, SA, sa_dt, ldsa);
    if (st != RSK_OK) return st;
    Carver cv(const_cast<void*>(index_mem));
    const uint16_t* offs = cv.take<uint16_t>(offsets_count(n, int(d), zeta));
    const uint16_t* ents = cv.take<uint16_t>(entries_count(n, zeta));
    const ApplyPlan p = plan_apply(h, n, k, int(d), zeta, a_dt);
    return apply_with_index(h, offs, ents, A, a_dt, n, k, lda, int(d), zeta, SA, sa_dt, ldsa, partials, p, stream);
}
// S b for one FP64 vector from a built index, in two launches: one thread per (chunk, sketch row)
// sums that row's entries of the chunk into partial[chunk][row]; one thread per row then adds the
// chunk partials in chunk order (so the result does not depend on scheduling) and scales.
__global__ void k_apply_vec_part(const uint16_t* __restrict__ offs, const uint16_t* __restrict__ ents,
                                 const double* __restrict__ b, int d, int zeta, int C, int pitch, int64_t nch,
                                 double* __restrict__ part) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= nch * d) return;
    const int64_t ch = idx / d;
    const int r = int(idx - ch * d);
    const uint16_t* o = offs + ch * pitch;
    const uint16_t* e = ents + ch * int64_t(C) * zeta;
    const double* bc = b + ch * C;
    double acc = 0.0;
    for (int t = o[r]; t < o[r + 1]; ++t) {
        const uint16_t v = e[t];
        const double x = bc[v & 0x7fff];
        acc += (v & 0x8000) ? -x : x;
    }
    part[idx] = acc;
}
__global__ void k_apply_vec_sum(const double* __restrict__ part, int d, int64_t nch, double scale,
                                double* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d) return;
    double acc = 0.0;
    for (int64_t ch = 0; ch < nch; ++ch) acc += part[ch * d + r];
    out[r] = acc * scale;
}
size_t sketch_vec_scratch_bytes(int64_t n, int64_t d, int zeta) { return size_t(n_chunks_of(n, zeta)) * size_t(d) * 8; }
rsk_status sketch_apply_vec_built(rsk_handle* h, const void* index_mem, int64_t n, int64_t d, int zeta,
                                  const double* b, double* Sb, double* scratch, cudaStream_t stream) {
    rsk_status st = check_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    if (!b || !Sb || !scratch) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null vector");
    Carver cv(const_cast<void*>(index_mem));
    const uint16_t* offs = cv.take<uint16_t>(offsets_count(n, int(d), zeta));
    const uint16_t* ents = cv.take<uint16_t>(entries_count(n, zeta));
    const int64_t nch = n_chunks_of(n, zeta);
    const int64_t total = nch * d;
    k_apply_vec_part<<<unsigned((total + 255) / 256), 256, 0, stream>>>(offs, ents, b, int(d), zeta, chunk_rows(zeta),
                                                                     offsets_pitch(int(d)), nch, scratch);
    k_apply_vec_sum<<<unsigned((d + 127) / 128), 128, 0, stream>>>(scratch, int(d), nch, 1.0 / sqrt(double(zeta)), Sb);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}
// Rows/signs of a SparseUniform (kind 0, stream 0) or SparseStack (kind 1, stream 4) sketch, and the
// apply of either kind (used by the Nystrom approximations, whose test matrix is a caller's choice).
rsk_status sketch_generate_kind(rsk_handle* h, int64_t n, int64_t d, int zeta, uint64_t seed, int kind, int32_t* rows,
                                uint32_t* signs, cudaStream_t stream) {
    rsk_status st = kind == kStack ? check_stack_dims(h, n, d, zeta) : check_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    return generate_kind(h, n, int(d), zeta, seed, kind == kStack ? kStreamStack : kStreamLeft, kind, rows, signs,
                         stream);
}
// The same draw for any d < 2^31 (no inverted index is built, so the index's d <= 8192 limit does not
// apply): rows int32[n * zeta], signs uint32[n].
rsk_status sketch_generate_large(rsk_handle* h, int64_t n, int64_t d, int zeta, uint64_t seed, int kind, int32_t* rows,
                                 uint32_t* signs, cudaStream_t stream) {
    if (n < 1 || n >= (int64_t(1) << 31) || d < 1 || d >= (int64_t(1) << 31) || zeta < 1 || zeta > 32 || zeta > d ||
        (kind == kStack && d % zeta != 0))
        return fail(h, RSK_ERR_INVALID_ARG, "draw needs n, d < 2^31, 1 <= zeta <= min(d, 32)");
    return generate_kind(h, n, int(d), zeta, seed, kind == kStack ? kStreamStack : kStreamLeft, kind, rows, signs,
                         stream);
}
rsk_status sketch_apply_kind(rsk_handle* h, int kind, const void* A, rsk_dtype a_dt, int64_t n, int64_t k,
                             int64_t lda, int64_t d, int zeta, uint64_t seed, void* SA, rsk_dtype sa_dt, int64_t ldsa,
                             cudaStream_t stream) {
    rsk_status st = kind == kStack ? check_stack_dims(h, n, d, zeta) : check_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    return apply_kind(h, A, a_dt, n, k, lda, 0, d, zeta, seed, SA, sa_dt, ldsa, stream,
                      kind == kStack ? kStreamStack : kStreamLeft, kind);
}
// Y = A Omega for Omega = S^T, S the k x dc sketch of the given kind: Y n x k column-major (ldy >= n).
rsk_status sketch_apply_right(rsk_handle* h, int kind, const float* A, int64_t n, int64_t dc, int64_t lda, int64_t k,
                              int zeta, uint64_t seed, float* Y, int64_t ldy, cudaStream_t stream, uint32_t stream_id) {
    rsk_status st = kind == kStack ? check_stack_dims(h, dc, k, zeta) : check_dims(h, dc, k, zeta);
    if (st != RSK_OK) return st;
    if (!A || !Y) return fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || lda < dc || ldy < n) return fail(h, RSK_ERR_INVALID_ARG, "need n >= 1, lda >= dc, ldy >= n");
    if (k > 512) return fail(h, RSK_ERR_UNSUPPORTED, "the right sketch supports k <= 512");
    const size_t ib = sketch_index_bytes(dc, k, zeta);
    st = ensure_workspace(h, ib + 256, stream);
    if (st != RSK_OK) return st;
    Carver cv(h->ws);
    uint16_t* offs = cv.take<uint16_t>(offsets_count(dc, int(k), zeta));
    uint16_t* ents = cv.take<uint16_t>(entries_count(dc, zeta));
    if (stream_id == ~0u) stream_id = kind == kStack ? kStreamStack : kStreamLeft;
    st = launch_index(h, dc, int(k), zeta, seed, stream_id, offs, ents, stream, 0, kind);
    if (st != RSK_OK) return st;
    const int C = chunk_rows(zeta);
    const int nch = int(n_chunks_of(dc, zeta));
    const size_t smem = size_t(C) * kRightRows * 4 + size_t(C) * zeta * 2 + size_t(k + 8) * 2;
    const int64_t ntiles = (n + kRightRows - 1) / kRightRows;
    const unsigned grid = unsigned(std::min<int64_t>(ntiles, int64_t(h->num_sms) * 2));
    const float scale = float(1.0 / sqrt(double(zeta)));
    auto go = [&](auto kern) -> rsk_status {
        RSK_CUDA_TRY(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        const int pr = prof_begin(h, stream, RSK_KERNEL_SKETCH_APPLY);
        // 16-byte staging loads when every row and every chunk start is 16-byte aligned
        const int vec4 = (reinterpret_cast<uintptr_t>(A) % 16 == 0 && lda % 4 == 0 && C % 4 == 0) ? 1 : 0;
        kern<<<grid, kRightThreads, smem, stream>>>(A, n, dc, lda, int(k), zeta, C, offsets_pitch(int(k)), offs, ents,
                                                    nch, scale, Y, ldy, vec4);
        prof_end(h, stream, pr);
        RSK_LAUNCH_CHECK(h);
        return RSK_OK;
    };
    if (k <= 64) return go(k_right<8>);
    if (k <= 128) return go(k_right<16>);
    if (k <= 256) return go(k_right<32>);
    return go(k_right<64>);
}
// Draw rows/signs of a sparse sign matrix from any Philox stream (the RSVD test matrix uses stream 3).
rsk_status sketch_generate(rsk_handle* h, int64_t n, int64_t d, int zeta, uint64_t seed, uint32_t stream_id,
                           int32_t* rows, uint32_t* signs, cudaStream_t stream) {
    rsk_status st = check_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    const unsigned grid = unsigned((n + 255) / 256);
    if (zeta <= 8) k_generate<8><<<grid, 256, 0, stream>>>(n, int(d), zeta, seed, stream_id, rows, signs, kUniform);
    else if (zeta <= 16) k_generate<16><<<grid, 256, 0, stream>>>(n, int(d), zeta, seed, stream_id, rows, signs, kUniform);
    else k_generate<32><<<grid, 256, 0, stream>>>(n, int(d), zeta, seed, stream_id, rows, signs, kUniform);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}
}  // namespace rsk

extern "C" {

rsk_status rsk_sparse_sign_generate(rsk_handle* h, int64_t n, int64_t d, int32_t zeta, uint64_t seed, int32_t* rows,
                                    uint32_t* sign_bits, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    rsk_status st = check_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    if (!rows && !sign_bits) return RSK_OK;
    const unsigned grid = unsigned((n + 255) / 256);
    return generate_kind(h, n, int(d), zeta, seed, kStreamLeft, kUniform, rows, sign_bits, stream);
}

rsk_status rsk_sparse_stack_generate(rsk_handle* h, int64_t n, int64_t d, int32_t zeta, uint64_t seed, int32_t* rows,
                                     uint32_t* sign_bits, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    rsk_status st = check_stack_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    if (!rows && !sign_bits) return RSK_OK;
    return generate_kind(h, n, int(d), zeta, seed, kStreamStack, kStack, rows, sign_bits, stream);
}

rsk_status rsk_sparse_stack_apply(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k, int64_t lda,
                                  int64_t d, int32_t zeta, uint64_t seed, void* SA, rsk_dtype sa_dtype, int64_t ldsa,
                                  cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    rsk_status st = check_stack_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    return apply_kind(h, A, a_dtype, n, k, lda, 0, d, zeta, seed, SA, sa_dtype, ldsa, stream, kStreamStack, kStack);
}

rsk_status rsk_sparse_sign_apply_right(rsk_handle* h, int32_t kind, const float* A, int64_t n, int64_t dc,
                                       int64_t lda, int64_t k, int32_t zeta, uint64_t seed, int32_t philox_stream,
                                       float* Y, int64_t ldy, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (kind != kUniform && kind != kStack) return rsk::fail(h, RSK_ERR_INVALID_ARG, "kind must be 0 or 1");
    if (philox_stream < -1) return rsk::fail(h, RSK_ERR_INVALID_ARG, "philox_stream must be -1 or a stream number");
    return rsk::sketch_apply_right(h, kind, A, n, dc, lda, k, zeta, seed, Y, ldy, stream,
                              philox_stream < 0 ? ~0u : uint32_t(philox_stream));
}

rsk_status rsk_sparse_sign_index_dims(int64_t n, int64_t d, int32_t zeta, int64_t* chunk_rows_out, int64_t* n_chunks,
                                      int64_t* offsets_pitch_out) {
    if (check_dims(nullptr, n, d, zeta) != RSK_OK || !chunk_rows_out || !n_chunks || !offsets_pitch_out)
        return RSK_ERR_INVALID_ARG;
    *chunk_rows_out = chunk_rows(zeta);
    *n_chunks = n_chunks_of(n, zeta);
    *offsets_pitch_out = offsets_pitch(int(d));
    return RSK_OK;
}

rsk_status rsk_sparse_sign_index(rsk_handle* h, int64_t n, int64_t d, int32_t zeta, uint64_t seed, uint16_t* offsets,
                                 uint16_t* entries, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    rsk_status st = check_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    if (!offsets || !entries) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null output pointer");
    if (reinterpret_cast<uintptr_t>(entries) % 16)
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "entries must be 16-byte aligned");
    return launch_index(h, n, int(d), zeta, seed, kStreamLeft, offsets, entries, stream);
}

rsk_status rsk_sparse_sign_apply(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k, int64_t lda,
                                 int64_t d, int32_t zeta, uint64_t seed, void* SA, rsk_dtype sa_dtype, int64_t ldsa,
                                 cudaStream_t stream) {
    return rsk_sparse_sign_apply_rows(h, A, a_dtype, n, k, lda, 0, d, zeta, seed, SA, sa_dtype, ldsa, stream);
}

rsk_status rsk_sparse_sign_apply_rows(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k,
                                      int64_t lda, int64_t row0, int64_t d, int32_t zeta, uint64_t seed, void* SA,
                                      rsk_dtype sa_dtype, int64_t ldsa, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    rsk_status st = check_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    return apply_kind(h, A, a_dtype, n, k, lda, row0, d, zeta, seed, SA, sa_dtype, ldsa, stream, kStreamLeft,
                      kUniform);
}

}  // extern "C"

namespace {
rsk_status apply_kind(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k, int64_t lda,
                      int64_t row0, int64_t d, int32_t zeta, uint64_t seed, void* SA, rsk_dtype sa_dtype,
                      int64_t ldsa, cudaStream_t stream, uint32_t stream_id, int kind) {
    if (row0 < 0 || row0 + n >= (int64_t(1) << 31))
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "row0=%lld: need 0 <= row0 and row0 + n < 2^31", (long long)row0);
    rsk_status st = check_apply_args(h, A, a_dtype, k, lda, SA, sa_dtype, ldsa);
    if (st != RSK_OK) return st;
    const ApplyPlan p = plan_apply(h, n, k, int(d), zeta, a_dtype);
    const size_t off_bytes = offsets_count(n, int(d), zeta) * 2;
    const size_t ent_bytes = entries_count(n, zeta) * 2;
    const size_t need = rsk::Carver::round(off_bytes) + rsk::Carver::round(ent_bytes) +
                        rsk::Carver::round(p.partial_bytes) + 256;
    st = rsk::ensure_workspace(h, need, stream);
    if (st != RSK_OK) return st;
    rsk::Carver cv(h->ws);
    uint16_t* offs = cv.take<uint16_t>(offsets_count(n, int(d), zeta));
    uint16_t* ents = cv.take<uint16_t>(entries_count(n, zeta));
    void* partials = cv.take<char>(p.partial_bytes);
    st = launch_index(h, n, int(d), zeta, seed, stream_id, offs, ents, stream, row0, kind);
    if (st != RSK_OK) return st;
    return apply_with_index(h, offs, ents, A, a_dtype, n, k, lda, int(d), zeta, SA, sa_dtype, ldsa, partials, p,
                            stream);
}
}  // namespace

extern "C" {

rsk_status rsk_sketch_sum_partials(rsk_handle* h, const void* parts, rsk_dtype dtype, int32_t count,
                                   int64_t part_stride, int64_t d, int64_t k, void* out, int64_t ldo,
                                   cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!parts || !out) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (dtype != RSK_F32 && dtype != RSK_F64) return rsk::fail(h, RSK_ERR_INVALID_ARG, "dtype must be F32 or F64");
    if (count < 1 || d < 1 || k < 1 || ldo < k || part_stride < d * k)
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "need count, d, k >= 1, ldo >= k, part_stride >= d*k");
    const int64_t total = d * k;
    const unsigned grid = unsigned((total + 255) / 256);
    if (dtype == RSK_F64)
        k_sum_blocks<double><<<grid, 256, 0, stream>>>(static_cast<const double*>(parts), part_stride, count, int(d), k,
                                                      static_cast<double*>(out), ldo);
    else
        k_sum_blocks<float><<<grid, 256, 0, stream>>>(static_cast<const float*>(parts), part_stride, count, int(d), k,
                                                     static_cast<float*>(out), ldo);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

rsk_status rsk_sparse_sign_apply_host(rsk_handle* h, const void* A_host, rsk_dtype a_dtype, int64_t n, int64_t k,
                                      int64_t lda, int64_t d, int32_t zeta, uint64_t seed, void* SA,
                                      rsk_dtype sa_dtype, int64_t ldsa, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    rsk_status st = check_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    st = check_apply_args(h, A_host, a_dtype, k, lda, SA, sa_dtype, ldsa);
    if (st != RSK_OK) return st;
    const size_t es = rsk::dtype_size(a_dtype);
    const int C = chunk_rows(zeta);
    // row blocks of whole chunks, about 256 MB of A each; two device staging buffers
    const int64_t row_bytes = k * int64_t(es);
    int64_t brows = std::max<int64_t>(C, ((int64_t(256) << 20) / row_bytes) / C * C);
    brows = std::min<int64_t>(brows, (n + C - 1) / C * C);
    const int64_t nblk = (n + brows - 1) / brows;
    const ApplyPlan p = plan_apply(h, std::min<int64_t>(n, brows), k, int(d), zeta, a_dtype);
    const size_t obytes = size_t(d) * k * (sa_dtype == RSK_F64 ? 8 : 4);
    const size_t need = rsk::Carver::round(offsets_count(n, int(d), zeta) * 2) +
                        rsk::Carver::round(entries_count(n, zeta) * 2) + rsk::Carver::round(p.partial_bytes) +
                        2 * rsk::Carver::round(size_t(brows) * row_bytes) + size_t(nblk) * rsk::Carver::round(obytes) +
                        1024;
    st = rsk::ensure_workspace(h, need, stream);
    if (st != RSK_OK) return st;
    st = rsk::ensure_streams(h, 2);
    if (st != RSK_OK) return st;
    rsk::Carver cv(h->ws);
    uint16_t* offs = cv.take<uint16_t>(offsets_count(n, int(d), zeta));
    uint16_t* ents = cv.take<uint16_t>(entries_count(n, zeta));
    void* partials = cv.take<char>(p.partial_bytes);
    char* stage[2] = {cv.take<char>(size_t(brows) * row_bytes), cv.take<char>(size_t(brows) * row_bytes)};
    char* outs = cv.take<char>(size_t(nblk) * rsk::Carver::round(obytes));
    const size_t ostride = rsk::Carver::round(obytes);
    cudaStream_t cs = h->streams[1];  // copy stream
    // every event created here is destroyed on every exit path below (a failed CUDA call only sets
    // st and skips the remaining work)
    cudaEvent_t ev_ready = nullptr, copied[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
    auto cuda_ok = [&](cudaError_t e, const char* what) {
        if (e == cudaSuccess) return true;
        st = rsk::fail(h, RSK_ERR_CUDA, "%s failed: %s", what, cudaGetErrorString(e));
        return false;
    };
    bool good = cuda_ok(cudaEventCreateWithFlags(&ev_ready, cudaEventDisableTiming), "cudaEventCreate");
    for (int i = 0; good && i < 2; ++i)
        good = cuda_ok(cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming), "cudaEventCreate") &&
               cuda_ok(cudaEventCreateWithFlags(&freed[i], cudaEventDisableTiming), "cudaEventCreate");
    // the copy stream starts after the caller's earlier work on `stream` (the workspace may be reused)
    good = good && cuda_ok(cudaEventRecord(ev_ready, stream), "cudaEventRecord") &&
           cuda_ok(cudaStreamWaitEvent(cs, ev_ready, 0), "cudaStreamWaitEvent");
    if (good) st = launch_index(h, n, int(d), zeta, seed, kStreamLeft, offs, ents, stream);
    for (int64_t b = 0; good && st == RSK_OK && b < nblk; ++b) {
        const int64_t r0 = b * brows, rows = std::min<int64_t>(brows, n - r0);
        char* buf = stage[b & 1];
        if (b >= 2 && !cuda_ok(cudaStreamWaitEvent(cs, freed[b & 1], 0), "cudaStreamWaitEvent")) break;
        const char* src = static_cast<const char*>(A_host) + size_t(r0) * size_t(lda) * es;
        const cudaError_t ce =
            lda == k ? cudaMemcpyAsync(buf, src, size_t(rows) * row_bytes, cudaMemcpyHostToDevice, cs)
                     : cudaMemcpy2DAsync(buf, size_t(row_bytes), src, size_t(lda) * es, size_t(row_bytes),
                                         size_t(rows), cudaMemcpyHostToDevice, cs);
        if (!cuda_ok(ce, "host-to-device copy of A") || !cuda_ok(cudaEventRecord(copied[b & 1], cs), "cudaEventRecord") ||
            !cuda_ok(cudaStreamWaitEvent(stream, copied[b & 1], 0), "cudaStreamWaitEvent"))
            break;
        // the block is whole chunks of the global index: its sub-index starts at chunk r0 / C
        const int64_t c0 = r0 / C;
        const ApplyPlan pb = plan_apply(h, rows, k, int(d), zeta, a_dtype);
        st = apply_with_index(h, offs + c0 * offsets_pitch(int(d)), ents + c0 * C * zeta, buf, a_dtype, rows, k, k,
                              int(d), zeta, outs + size_t(b) * ostride, sa_dtype, k, partials, pb, stream);
        if (st == RSK_OK && !cuda_ok(cudaEventRecord(freed[b & 1], stream), "cudaEventRecord")) break;
    }
    if (good && st == RSK_OK) {
        // SA = sum of the block sketches, in block order
        const int64_t total = d * k;
        if (sa_dtype == RSK_F64)
            k_sum_blocks<double><<<unsigned((total + 255) / 256), 256, 0, stream>>>(
                reinterpret_cast<const double*>(outs), int64_t(ostride / 8), int(nblk), int(d), k,
                static_cast<double*>(SA), ldsa);
        else
            k_sum_blocks<float><<<unsigned((total + 255) / 256), 256, 0, stream>>>(
                reinterpret_cast<const float*>(outs), int64_t(ostride / 4), int(nblk), int(d), k,
                static_cast<float*>(SA), ldsa);
        cuda_ok(cudaGetLastError(), "block sum launch");
    }
    // events may be destroyed while work is pending (the driver releases them on completion)
    if (ev_ready) cudaEventDestroy(ev_ready);
    for (int i = 0; i < 2; ++i) {
        if (copied[i]) cudaEventDestroy(copied[i]);
        if (freed[i]) cudaEventDestroy(freed[i]);
    }
    return st;
}

rsk_status rsk_sparse_sign_plan_create(rsk_handle* h, int64_t n, int64_t d, int32_t zeta, uint64_t seed,
                                       rsk_sketch_plan** plan, cudaStream_t stream) {
    if (!h || !plan) return RSK_ERR_INVALID_ARG;
    *plan = nullptr;
    rsk_status st = check_dims(h, n, d, zeta);
    if (st != RSK_OK) return st;
    rsk_sketch_plan* p = new (std::nothrow) rsk_sketch_plan();
    if (!p) return rsk::fail(h, RSK_ERR_NOMEM, "plan allocation failed");
    p->n = n;
    p->d = d;
    p->zeta = zeta;
    p->seed = seed;
    p->nchunks = n_chunks_of(n, zeta);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&p->offs), offsets_count(n, int(d), zeta) * 2, stream);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&p->ents), entries_count(n, zeta) * 2, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (p->offs) cudaFreeAsync(p->offs, stream);
        delete p;
        return rsk::fail(h, RSK_ERR_NOMEM, "plan device allocation failed: %s", cudaGetErrorString(e));
    }
    st = launch_index(h, n, int(d), zeta, seed, kStreamLeft, p->offs, p->ents, stream);
    if (st != RSK_OK) {
        cudaFreeAsync(p->offs, stream);
        cudaFreeAsync(p->ents, stream);
        delete p;
        return st;
    }
    *plan = p;
    return RSK_OK;
}

rsk_status rsk_sparse_sign_plan_apply(rsk_handle* h, const rsk_sketch_plan* plan, const void* A, rsk_dtype a_dtype,
                                      int64_t k, int64_t lda, void* SA, rsk_dtype sa_dtype, int64_t ldsa,
                                      cudaStream_t stream) {
    if (!h || !plan) return RSK_ERR_INVALID_ARG;
    rsk_status st = check_apply_args(h, A, a_dtype, k, lda, SA, sa_dtype, ldsa);
    if (st != RSK_OK) return st;
    const ApplyPlan p = plan_apply(h, plan->n, k, int(plan->d), plan->zeta, a_dtype);
    st = rsk::ensure_workspace(h, rsk::Carver::round(p.partial_bytes) + 256, stream);
    if (st != RSK_OK) return st;
    rsk::Carver cv(h->ws);
    void* partials = cv.take<char>(p.partial_bytes);
    return apply_with_index(h, plan->offs, plan->ents, A, a_dtype, plan->n, k, lda, int(plan->d), plan->zeta, SA,
                            sa_dtype, ldsa, partials, p, stream);
}

rsk_status rsk_sparse_sign_plan_destroy(rsk_handle* h, rsk_sketch_plan* plan, cudaStream_t stream) {
    if (!plan) return RSK_ERR_INVALID_ARG;
    cudaFreeAsync(plan->offs, stream);
    cudaFreeAsync(plan->ents, stream);
    delete plan;
    (void)h;
    return RSK_OK;
}

}  // extern "C"
