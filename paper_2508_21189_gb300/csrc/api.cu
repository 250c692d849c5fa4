// Handle lifetime, error reporting, workspace and TMA descriptor encoding for librsk.
#include <stdlib.h>
#include <string.h>

#include <new>

#include <cudaTypedefs.h>

#include "common.cuh"

namespace rsk {

rsk_status fail(rsk_handle* h, rsk_status st, const char* fmt, ...) {
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->msg, sizeof(h->msg), fmt, ap);
        va_end(ap);
    }
    return st;
}

rsk_status ensure_workspace(rsk_handle* h, size_t bytes, cudaStream_t stream) {
    const char* inj = getenv("RSK_FAULT_NOMEM");
    if (inj && inj[0] == '1')
        return fail(h, RSK_ERR_NOMEM, "workspace allocation of %zu bytes refused (RSK_FAULT_NOMEM=1)", bytes);
    if (bytes <= h->ws_bytes) return RSK_OK;
    size_t want = bytes + bytes / 4;
    if (h->ws) {
        cudaError_t e = cudaFreeAsync(h->ws, stream);
        h->ws = nullptr;
        h->ws_bytes = 0;
        if (e != cudaSuccess) return fail(h, RSK_ERR_CUDA, "cudaFreeAsync: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaMallocAsync(&h->ws, want, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->ws = nullptr;
        return fail(h, RSK_ERR_NOMEM, "workspace allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
    }
    h->ws_bytes = want;
    return RSK_OK;
}

rsk_status ensure_streams(rsk_handle* h, int count) {
    while (int(h->streams.size()) < count) {
        cudaStream_t s = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(h, RSK_ERR_CUDA, "cudaStreamCreateWithFlags: %s", cudaGetErrorString(e));
        h->streams.push_back(s);
    }
    return RSK_OK;
}

bool encode_2d(rsk_handle* h, CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner,
               uint64_t outer, uint64_t row_stride_bytes, uint32_t box_inner, uint32_t box_outer) {
    if (!h->encode_tiled) return false;
    auto fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(h->encode_tiled);
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_stride_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_2d_swz128(rsk_handle* h, CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner,
                      uint64_t outer, uint64_t row_stride_bytes, uint32_t box_inner, uint32_t box_outer) {
    if (!h->encode_tiled) return false;
    auto fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(h->encode_tiled);
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_stride_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

static cudaEvent_t take_event(rsk_handle* h) {
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

int prof_begin(rsk_handle* h, cudaStream_t stream, int kernel) {
    if (!h || !h->prof) return -1;
    rsk_handle::Rec r;
    r.kernel = kernel;
    r.a = take_event(h);
    r.b = take_event(h);
    if (!r.a || !r.b) return -1;
    cudaEventRecord(r.a, stream);
    h->recs.push_back(r);
    return int(h->recs.size()) - 1;
}

void prof_end(rsk_handle* h, cudaStream_t stream, int rec) {
    if (!h || rec < 0 || rec >= int(h->recs.size())) return;
    cudaEventRecord(h->recs[rec].b, stream);
}

static void prof_clear(rsk_handle* h) {
    for (auto& r : h->recs) {
        h->event_pool.push_back(r.a);
        h->event_pool.push_back(r.b);
    }
    h->recs.clear();
}

}  // namespace rsk

extern "C" {

rsk_status rsk_profile_enable(rsk_handle* h, int32_t on) {
    if (!h) return RSK_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    rsk::prof_clear(h);
    h->prof = on != 0;
    return RSK_OK;
}

rsk_status rsk_profile_read(rsk_handle* h, int32_t kernel, double* total_ms, int64_t* launches) {
    if (!h || !total_ms || !launches) return RSK_ERR_INVALID_ARG;
    double ms = 0.0;
    int64_t cnt = 0;
    for (auto& r : h->recs) {
        if (r.kernel != kernel) continue;
        RSK_CUDA_TRY(h, cudaEventSynchronize(r.b));
        float t = 0.f;
        RSK_CUDA_TRY(h, cudaEventElapsedTime(&t, r.a, r.b));
        ms += t;
        ++cnt;
    }
    *total_ms = ms;
    *launches = cnt;
    return RSK_OK;
}

rsk_status rsk_create(rsk_handle** out) {
    if (!out) return RSK_ERR_INVALID_ARG;
    *out = nullptr;
    rsk_handle* h = new (std::nothrow) rsk_handle();
    if (!h) return RSK_ERR_NOMEM;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaMalloc(&h->dev_status, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(h->dev_status, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&h->host_flags), kHostFlags * sizeof(double),
                                            cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->flag_ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->flag_ev[1], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h->dev_status) cudaFree(h->dev_status);
        if (h->host_flags) cudaFreeHost(h->host_flags);
        if (h->flag_ev[0]) cudaEventDestroy(h->flag_ev[0]);
        if (h->flag_ev[1]) cudaEventDestroy(h->flag_ev[1]);
        delete h;
        return RSK_ERR_CUDA;
    }
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        h->encode_tiled = fn;
    cudaGetLastError();
    *out = h;
    return RSK_OK;
}

rsk_status rsk_destroy(rsk_handle* h) {
    if (!h) return RSK_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    rsk::prof_clear(h);
    for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
    for (cudaStream_t s : h->streams) cudaStreamDestroy(s);
    if (h->ws) cudaFree(h->ws);
    if (h->dev_status) cudaFree(h->dev_status);
    if (h->host_flags) cudaFreeHost(h->host_flags);
    for (cudaEvent_t e : h->flag_ev)
        if (e) cudaEventDestroy(e);
    delete h;
    return RSK_OK;
}

const char* rsk_last_error(const rsk_handle* h) { return h ? h->msg : "null handle"; }

rsk_status rsk_sync_status(rsk_handle* h, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    RSK_CUDA_TRY(h, cudaStreamSynchronize(stream));
    unsigned int word = 0;
    RSK_CUDA_TRY(h, cudaMemcpy(&word, h->dev_status, sizeof(word), cudaMemcpyDeviceToHost));
    RSK_CUDA_TRY(h, cudaMemset(h->dev_status, 0, sizeof(word)));
    if (word & RSK_DEV_TIMEOUT) return rsk::fail(h, RSK_ERR_TIMEOUT, "a bounded device wait ran out (status 0x%x)", word);
    if (word & RSK_DEV_BOUNDS) return rsk::fail(h, RSK_ERR_INTERNAL, "a device bounds check failed (status 0x%x)", word);
    return RSK_OK;
}

rsk_status rsk_set_wait_limit(rsk_handle* h, uint32_t spins) {
    if (!h) return RSK_ERR_INVALID_ARG;
    h->wait_limit = spins ? spins : rskd::kWaitLimit;
    return RSK_OK;
}

int32_t rsk_version(void) { return 200; }

}  // extern "C"
