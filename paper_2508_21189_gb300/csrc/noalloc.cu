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
#include <string.h>

#include "common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];
static __device__ unsigned int g_status;

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
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return RSK_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return RSK_ERR_UNSUPPORTED;
    DeviceContext& c = g_ctx[dev];
    if (!c.ready) {
        const rsk_status st = setup(c, dev);
        if (st != RSK_OK) return st;
    }
    if (n < 1 || k < 1 || d < 1 || zeta < 1) return RSK_ERR_INVALID_ARG;
    // sizes whose index and partials do not fit the fixed array are refused before any launch
    if (rsk::sketch_scratch_bytes(&c.h, n, k, d, zeta, a_dtype) > kNoAllocScratchBytes) return RSK_ERR_UNSUPPORTED;
    return rsk::sketch_apply_scratch(&c.h, A, a_dtype, n, k, lda, d, zeta, seed, SA, sa_dtype, ldsa, c.scratch,
                                     stream);
}
