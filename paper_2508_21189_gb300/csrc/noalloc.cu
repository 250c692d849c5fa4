// rsk_sparse_sign_apply_noalloc: the sparse sign apply for callers that cannot allocate device
// memory -- code running where cudaMalloc is unavailable or forbidden, such as a host callback
// inside a library that owns the allocator, a plugin whose host application manages every device
// buffer, or a path that must not allocate at all after start-up.  It needs no rsk_handle (whose
// creation allocates) and takes its scratch from one fixed array in device memory.
//
// The scratch is the file-scope array g_scratch below, of kNoAllocScratchBytes.  Every GPU that
// loads librsk holds it until the process exits.  In host code the symbol g_scratch only stands
// in for the array: it is not a device address, and a kernel given it would fault or, where the
// GPU can reach host memory, silently use the wrong memory.  The real address comes from
// cudaGetSymbolAddress, taken once per device (with that device current) by the first call on
// that device, which is therefore the call to make before any stream capture.
//
// All calls share the array and it keeps the last call's contents.  Nothing in it has to start at
// zero: the index kernel writes every offset and entry the apply reads, and the apply writes every
// partial the reduction reads.  Calls whose work overlaps on the GPU (other streams, or without
// synchronisation in between) race on the array; the host-side set-up is not thread safe either.
//
// Device-side failures.  The kernels record a bounded wait that ran out, or a failed bounds check,
// in the device word g_status.  A call cannot return that status (it does not synchronise), so
// each call clears g_status in its first launch and, in its last, overwrites SA with NaN when the
// word is set: a result that may hold stale or missing partial sums is never returned as valid.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];
static __device__ unsigned int g_status;

__global__ void k_noalloc_clear_status() { g_status = 0u; }

// SA (d x k, leading dimension ldsa) := NaN if any kernel of this call recorded a failure.
template <typename T>
__global__ void k_noalloc_check_status(T* SA, int64_t d, int64_t k, int64_t ldsa) {
    if (*static_cast<volatile unsigned int*>(&g_status) == 0u) return;
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < d * k;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = idx / k, c = idx - i * k;
        SA[i * ldsa + c] = T(NAN);
    }
}

struct DeviceContext {
    bool ready = false;
    void* scratch = nullptr;  // device address of g_scratch on this device
    rsk_handle h;             // static context: no allocation, profiling off
};
static DeviceContext g_ctx[kMaxDevices];

rsk_status setup(DeviceContext& c, int dev) {
    void* scratch = nullptr;
    if (cudaGetSymbolAddress(&scratch, g_scratch) != cudaSuccess || !scratch) {
        cudaGetLastError();
        return RSK_ERR_CUDA;
    }
    void* status = nullptr;
    if (cudaGetSymbolAddress(&status, g_status) != cudaSuccess || !status) {
        cudaGetLastError();
        return RSK_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return RSK_ERR_CUDA;
    }
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        fn = nullptr;
    cudaGetLastError();
    c.scratch = scratch;
    c.h.device = dev;
    c.h.num_sms = sms;
    c.h.dev_status = static_cast<unsigned int*>(status);
    c.h.encode_tiled = fn;
    c.ready = true;
    return RSK_OK;
}

}  // namespace

extern "C" rsk_status rsk_sparse_sign_apply_noalloc(const void* A, rsk_dtype a_dtype, int64_t n, int64_t k,
                                                    int64_t lda, int64_t d, int32_t zeta, uint64_t seed, void* SA,
                                                    rsk_dtype sa_dtype, int64_t ldsa, cudaStream_t stream) {
    // every argument is checked before anything else (the scratch sizing below assumes valid sizes)
    rsk_status st = rsk::sketch_check_args(nullptr, A, a_dtype, n, k, lda, d, zeta, SA, sa_dtype, ldsa);
    if (st != RSK_OK) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return RSK_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return RSK_ERR_UNSUPPORTED;
    DeviceContext& c = g_ctx[dev];
    if (!c.ready) {
        st = setup(c, dev);
        if (st != RSK_OK) return st;
    }
    // sizes whose index and partials do not fit the fixed array are refused before any launch
    if (rsk::sketch_scratch_bytes(&c.h, n, k, d, zeta, a_dtype) > kNoAllocScratchBytes) return RSK_ERR_UNSUPPORTED;
    k_noalloc_clear_status<<<1, 1, 0, stream>>>();
    if (cudaGetLastError() != cudaSuccess) return RSK_ERR_CUDA;
    st = rsk::sketch_apply_scratch(&c.h, A, a_dtype, n, k, lda, d, zeta, seed, SA, sa_dtype, ldsa, c.scratch, stream);
    if (st != RSK_OK) return st;
    const unsigned grid = unsigned(std::min<int64_t>((d * k + 255) / 256, int64_t(c.h.num_sms) * 8));
    if (sa_dtype == RSK_F64)
        k_noalloc_check_status<double><<<grid, 256, 0, stream>>>(static_cast<double*>(SA), d, k, ldsa);
    else
        k_noalloc_check_status<float><<<grid, 256, 0, stream>>>(static_cast<float*>(SA), d, k, ldsa);
    if (cudaGetLastError() != cudaSuccess) return RSK_ERR_CUDA;
    return RSK_OK;
}
