// Shared host/device plumbing of librsk: the handle, status reporting, the workspace and the
// bounded waits every kernel uses.  No arithmetic of the method lives here.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdarg.h>
#include <stdio.h>

#include <vector>

#include "rsk.h"

// Device status word bits (kernels OR them in; rsk_sync_status reads and clears the word).
#define RSK_DEV_TIMEOUT 1u
#define RSK_DEV_BOUNDS 2u

struct rsk_handle {
    int device = 0;
    int num_sms = 0;
    unsigned int* dev_status = nullptr;  // device word written by kernels
    void* ws = nullptr;                  // workspace (stream-ordered allocation)
    size_t ws_bytes = 0;
    void* encode_tiled = nullptr;        // cuTensorMapEncodeTiled from the driver
    char msg[1024] = {0};
    // optional per-kernel timing (rsk_profile_*)
    bool prof = false;
    struct Rec {
        int kernel;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> event_pool;
    std::vector<cudaStream_t> streams;  // internal non-blocking streams (batched solver)
    // pinned host words the solvers poll without stalling the stream (early exit of the inner CG)
    double* host_flags = nullptr;       // kHostFlags doubles
    cudaEvent_t flag_ev[2] = {nullptr, nullptr};
    // iteration limit of the bounded polls on global-memory flags (grid barrier, reflector-ready
    // flags); rsk_set_wait_limit changes it, 0 restores the default
    uint32_t wait_limit = 1u << 22;
    // launch-parameter override used while the autotuner times a candidate: 0 = the tuning table, then
    // the default rule; -1 = the default rule only; > 0 = this value
    int tune_override = 0;
};
constexpr int kHostFlags = 8;

namespace rsk {

rsk_status fail(rsk_handle* h, rsk_status st, const char* fmt, ...);

// Tuned launch parameters (tune.cu): the knob of `kernel` for a problem shape, or 0 when none is
// tuned.  Kernels: 0 = sparse gather apply (row ranges), 1 = SRTT (row bands), 2 = batched solver
// (rows per work tile).  The handle's tune_override takes precedence.
enum TuneKernel { kTuneApply = 0, kTuneSrtt = 1, kTuneBatchTile = 2 };
int tune_lookup(int kernel, int dtype, int64_t n, int64_t k, int64_t d, int sms);
inline int tuned_value(const rsk_handle* h, int kernel, int dtype, int64_t n, int64_t k, int64_t d) {
    if (h && h->tune_override > 0) return h->tune_override;
    if (h && h->tune_override < 0) return 0;
    return tune_lookup(kernel, dtype, n, k, d, h ? h->num_sms : 0);
}

// Make sure the handle owns at least `count` internal non-blocking streams.
rsk_status ensure_streams(rsk_handle* h, int count);

// Grow the handle's workspace to at least `bytes` (stream-ordered on `stream`).
rsk_status ensure_workspace(rsk_handle* h, size_t bytes, cudaStream_t stream);

// Carve aligned pieces out of the workspace in call order.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
    static size_t round(size_t bytes) { return (bytes + 255) & ~size_t(255); }
};

inline size_t dtype_size(rsk_dtype t) { return (t == RSK_F64 || t == RSK_F32X2) ? 8 : (t == RSK_F32 ? 4 : 2); }
inline bool dtype_ok(int t) { return t == RSK_F64 || t == RSK_F32 || t == RSK_BF16; }
// Sketch inputs may also be interleaved (hi, lo) FP32 pairs.
inline bool sketch_dtype_ok(int t) { return dtype_ok(t) || t == RSK_F32X2; }

// Profiling brackets around one kernel launch (no-ops unless rsk_profile_enable(h, 1)).
int prof_begin(rsk_handle* h, cudaStream_t stream, int kernel);
void prof_end(rsk_handle* h, cudaStream_t stream, int rec);

// Encode a 2-D tiled TMA descriptor (inner dim first).  Returns false if the driver refuses.
bool encode_2d(rsk_handle* h, CUtensorMap* map, CUtensorMapDataType dt, const void* base,
               uint64_t inner, uint64_t outer, uint64_t row_stride_bytes, uint32_t box_inner,
               uint32_t box_outer);

// The same with the 128-byte swizzle (the K-major operand layout of the tensor-core GEMM); box_inner
// times the element size must be at most 128 bytes.
bool encode_2d_swz128(rsk_handle* h, CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner,
                      uint64_t outer, uint64_t row_stride_bytes, uint32_t box_inner, uint32_t box_outer);

// Sparse sign apply with caller-provided scratch for the per-range partials (used by solvers that
// carve their own buffers out of the workspace).  sketch_partial_bytes gives the size needed.
size_t sketch_partial_bytes(rsk_handle* h, int64_t n, int64_t k, int64_t d, int zeta, rsk_dtype a_dt);
rsk_status sketch_plan_apply_ws(rsk_handle* h, const rsk_sketch_plan* plan, const void* A, rsk_dtype a_dt, int64_t k,
                                int64_t lda, void* SA, rsk_dtype sa_dt, int64_t ldsa, void* partials,
                                cudaStream_t stream);

rsk_status sketch_check_args(rsk_handle* h, const void* A, rsk_dtype a_dt, int64_t n, int64_t k, int64_t lda,
                             int64_t d, int zeta, const void* SA, rsk_dtype sa_dt, int64_t ldsa);
size_t sketch_scratch_bytes(rsk_handle* h, int64_t n, int64_t k, int64_t d, int zeta, rsk_dtype a_dt);
rsk_status sketch_apply_scratch(rsk_handle* h, const void* A, rsk_dtype a_dt, int64_t n, int64_t k, int64_t lda,
                                int64_t d, int zeta, uint64_t seed, void* SA, rsk_dtype sa_dt, int64_t ldsa,
                                void* scratch, cudaStream_t stream);

rsk_status sketch_generate(rsk_handle* h, int64_t n, int64_t d, int zeta, uint64_t seed, uint32_t stream_id,
                           int32_t* rows, uint32_t* signs, cudaStream_t stream);
// kind 0 = SparseUniform (Philox stream 0), 1 = SparseStack (stream 4): rows/signs of the n columns of
// the d x n sketch, and S * A (the workspace of rsk_sparse_sign_apply: uses the handle's workspace).
rsk_status sketch_generate_kind(rsk_handle* h, int64_t n, int64_t d, int zeta, uint64_t seed, int kind, int32_t* rows,
                                uint32_t* signs, cudaStream_t stream);
// Right sketch Y = A Omega = A S^T for A n x dc row-major FP32 and S the k x dc sketch of the kind: Y is
// n x k column-major (ldy >= n).  S comes from the kind's Philox stream, or from `stream_id` when it is
// not ~0u.  Uses the handle's workspace for the inverted index of S.
rsk_status sketch_apply_right(rsk_handle* h, int kind, const float* A, int64_t n, int64_t dc, int64_t lda, int64_t k,
                              int zeta, uint64_t seed, float* Y, int64_t ldy, cudaStream_t stream,
                              uint32_t stream_id = ~0u);
rsk_status sketch_generate_large(rsk_handle* h, int64_t n, int64_t d, int zeta, uint64_t seed, int kind, int32_t* rows,
                                 uint32_t* signs, cudaStream_t stream);
rsk_status sketch_apply_kind(rsk_handle* h, int kind, const void* A, rsk_dtype a_dt, int64_t n, int64_t k,
                             int64_t lda, int64_t d, int zeta, uint64_t seed, void* SA, rsk_dtype sa_dt, int64_t ldsa,
                             cudaStream_t stream);
size_t sketch_index_bytes(int64_t n, int64_t d, int zeta);
rsk_status sketch_build_index(rsk_handle* h, int64_t n, int64_t d, int zeta, uint64_t seed, void* index_mem,
                              cudaStream_t stream);
// S b for one FP64 vector from an index built by sketch_build_index; scratch holds
// sketch_vec_scratch_bytes(n, d, zeta) bytes (per-chunk partial sums, reduced in chunk order).
size_t sketch_vec_scratch_bytes(int64_t n, int64_t d, int zeta);
rsk_status sketch_apply_vec_built(rsk_handle* h, const void* index_mem, int64_t n, int64_t d, int zeta,
                                  const double* b, double* Sb, double* scratch, cudaStream_t stream);
rsk_status sketch_apply_built(rsk_handle* h, const void* index_mem, int64_t n, int64_t d, int zeta, const void* A,
                              rsk_dtype a_dt, int64_t k, int64_t lda, void* SA, rsk_dtype sa_dt, int64_t ldsa,
                              void* partials, cudaStream_t stream);

}  // namespace rsk

#define RSK_CUDA_TRY(h, call)                                                                  \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return rsk::fail((h), RSK_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define RSK_LAUNCH_CHECK(h)                                                                    \
    do {                                                                                       \
        cudaError_t e_ = cudaGetLastError();                                                   \
        if (e_ != cudaSuccess)                                                                 \
            return rsk::fail((h), RSK_ERR_CUDA, "kernel launch failed at %s:%d: %s", __FILE__, \
                             __LINE__, cudaGetErrorString(e_));                                \
    } while (0)

// ------------------------------------------------------------------------------------------
// Device-side helpers: mbarrier + TMA in inline PTX, with bounded waits.
// ------------------------------------------------------------------------------------------
#ifdef __CUDACC__
namespace rskd {

// Roughly a few seconds at most before a wait gives up and records RSK_DEV_TIMEOUT.  The mbarrier
// waits on TMA/bulk copies always use it; the polls on global-memory flags take the handle's
// wait_limit (this value unless rsk_set_wait_limit changed it).
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase.  On timeout records RSK_DEV_TIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned int* status) {
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 1024) __nanosleep(64);
    }
    atomicOr(status, RSK_DEV_TIMEOUT);
    return false;
}

// 2-D tiled TMA load of box (x = inner coordinate, y = outer) into shared memory; completion is
// signalled on `bar` as transaction bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completion
// signalled on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded software grid barrier for persistent kernels whose CTAs are all resident (cooperative
// launch).  count / gen are two zero-initialised words; returns false (and records
// RSK_DEV_TIMEOUT) if the other CTAs did not arrive within `limit` polls.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, volatile unsigned int* gen, unsigned int nblocks,
                                             unsigned int* status, uint32_t limit) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        const unsigned int g = *gen;
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            *count = 0;
            __threadfence();
            atomicAdd(const_cast<unsigned int*>(gen), 1u);
        } else {
            uint32_t it = 0;
            while (*gen == g) {
                if (++it > limit) {
                    atomicOr(status, RSK_DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
                if (it > 64) __nanosleep(64);
            }
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

}  // namespace rskd
#endif
