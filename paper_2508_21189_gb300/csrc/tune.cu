// Autotuning of launch parameters: a process-wide table of tuned values keyed by
// (kernel, dtype, n, k, d, SM count), an on-disk text cache, and tuners that time candidate values
// of one knob on the device and keep the fastest.
//
// Knobs.  Sparse gather apply: the number of row ranges R (partial sums per range, reduced in range
// order; the default deals R * pairs items evenly over the SMs).  SRTT: the number of row bands R.
// Batched least squares: the rows per work tile of the persistent passes.
//
// A tuned value changes how partial sums are grouped, so results stay deterministic for a fixed table
// but can differ in the last bits from the untuned ones; tuning is explicit (these calls, or a cache
// file named by RSK_TUNE_CACHE, read at the first lookup).
//
// Cache format: text, one entry per line,
//     rsk-tune v1 kernel=<int> dtype=<int> n=<int> k=<int> d=<int> sms=<int> value=<int>
// lines starting with '#' are comments; later lines override earlier ones with the same key.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace {

using Key = std::tuple<int, int, int64_t, int64_t, int64_t, int>;

struct Table {
    std::mutex mu;
    std::map<Key, int> values;
    bool env_loaded = false;
};
Table& table() {
    static Table t;
    return t;
}

bool parse_line(const char* line, Key* key, int* value) {
    int kernel, dtype, sms, v;
    long long n, k, d;
    if (sscanf(line, " rsk-tune v1 kernel=%d dtype=%d n=%lld k=%lld d=%lld sms=%d value=%d", &kernel, &dtype, &n, &k, &d,
               &sms, &v) != 7)
        return false;
    if (v <= 0) return false;
    *key = Key(kernel, dtype, int64_t(n), int64_t(k), int64_t(d), sms);
    *value = v;
    return true;
}

rsk_status load_locked(Table& t, const char* path) {
    FILE* f = fopen(path, "r");
    if (!f) return RSK_ERR_INVALID_ARG;
    char line[512];
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        Key key;
        int v;
        if (parse_line(line, &key, &v)) t.values[key] = v;
    }
    fclose(f);
    return RSK_OK;
}

rsk_status save_locked(Table& t, const char* path) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return RSK_ERR_INVALID_ARG;
    fprintf(f, "# librsk tuned launch parameters (kernel 0: gather row ranges, 1: SRTT bands, 2: batched tile rows)\n");
    for (const auto& e : t.values) {
        const Key& k = e.first;
        fprintf(f, "rsk-tune v1 kernel=%d dtype=%d n=%lld k=%lld d=%lld sms=%d value=%d\n", std::get<0>(k), std::get<1>(k),
                (long long)std::get<2>(k), (long long)std::get<3>(k), (long long)std::get<4>(k), std::get<5>(k), e.second);
    }
    const bool ok = fclose(f) == 0;
    if (!ok || rename(tmp.c_str(), path) != 0) return RSK_ERR_INVALID_ARG;
    return RSK_OK;
}

void load_env_once(Table& t) {
    if (t.env_loaded) return;
    t.env_loaded = true;
    const char* p = getenv("RSK_TUNE_CACHE");
    if (p && p[0]) load_locked(t, p);
}

// value 0 removes the entry (the default rule applies)
void store(int kernel, int dtype, int64_t n, int64_t k, int64_t d, int sms, int value) {
    Table& t = table();
    std::lock_guard<std::mutex> g(t.mu);
    load_env_once(t);
    if (value > 0) t.values[Key(kernel, dtype, n, k, d, sms)] = value;
    else t.values.erase(Key(kernel, dtype, n, k, d, sms));
    const char* p = getenv("RSK_TUNE_CACHE");
    if (p && p[0]) save_locked(t, p);
}

__global__ void k_fill_pattern(uint32_t* __restrict__ w, int64_t words) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    // small finite values in every float / bf16 / double reading of the words
    if (i < words) w[i] = 0x3c003c00u ^ (uint32_t(i * 2654435761u) & 0x00ff00ffu);
}

// Median device time (ms) of `reps` calls of fn on `stream`, after one warm-up call.
template <typename F>
rsk_status time_calls(rsk_handle* h, F fn, int reps, cudaStream_t stream, double* ms) {
    rsk_status st = fn();
    if (st != RSK_OK) return st;
    std::vector<float> t;
    cudaEvent_t a, b;
    RSK_CUDA_TRY(h, cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return rsk::fail(h, RSK_ERR_CUDA, "cudaEventCreate failed");
    }
    for (int r = 0; r < reps && st == RSK_OK; ++r) {
        cudaEventRecord(a, stream);
        st = fn();
        cudaEventRecord(b, stream);
        if (cudaEventSynchronize(b) != cudaSuccess) st = rsk::fail(h, RSK_ERR_CUDA, "event synchronize failed");
        float x = 0.f;
        cudaEventElapsedTime(&x, a, b);
        t.push_back(x);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != RSK_OK) return st;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return RSK_OK;
}

std::vector<int> around(int v0, int lo, int hi) {
    std::vector<int> c;
    for (int v : {v0, v0 / 4, v0 / 2, v0 * 2, v0 * 4}) {
        v = std::max(lo, std::min(hi, v));
        if (std::find(c.begin(), c.end(), v) == c.end()) c.push_back(v);
    }
    return c;
}

}  // namespace

namespace rsk {
int tune_lookup(int kernel, int dtype, int64_t n, int64_t k, int64_t d, int sms) {
    Table& t = table();
    std::lock_guard<std::mutex> g(t.mu);
    load_env_once(t);
    auto it = t.values.find(Key(kernel, dtype, n, k, d, sms));
    return it == t.values.end() ? 0 : it->second;
}
}  // namespace rsk

extern "C" {

rsk_status rsk_tune_cache_load(const char* path) {
    if (!path) return RSK_ERR_INVALID_ARG;
    Table& t = table();
    std::lock_guard<std::mutex> g(t.mu);
    return load_locked(t, path);
}

rsk_status rsk_tune_cache_save(const char* path) {
    if (!path) return RSK_ERR_INVALID_ARG;
    Table& t = table();
    std::lock_guard<std::mutex> g(t.mu);
    return save_locked(t, path);
}

rsk_status rsk_tune_cache_clear(void) {
    Table& t = table();
    std::lock_guard<std::mutex> g(t.mu);
    t.values.clear();
    t.env_loaded = true;  // an explicit clear also drops what the environment's cache would add
    return RSK_OK;
}

rsk_status rsk_tune_cache_set(int32_t kernel, int32_t dtype, int64_t n, int64_t k, int64_t d, int32_t sms,
                              int32_t value) {
    if (kernel < 0 || kernel > 2 || value < 1) return RSK_ERR_INVALID_ARG;
    Table& t = table();
    std::lock_guard<std::mutex> g(t.mu);
    t.values[Key(kernel, dtype, n, k, d, sms)] = value;
    return RSK_OK;
}

rsk_status rsk_tune_cache_get(int32_t kernel, int32_t dtype, int64_t n, int64_t k, int64_t d, int32_t sms,
                              int32_t* value) {
    if (!value) return RSK_ERR_INVALID_ARG;
    *value = rsk::tune_lookup(kernel, dtype, n, k, d, sms);
    return RSK_OK;
}

rsk_status rsk_autotune_sketch(rsk_handle* h, int32_t kernel, rsk_dtype a_dtype, int64_t n, int64_t k, int64_t d,
                               int32_t zeta, int32_t* chosen, double* best_ms, cudaStream_t stream) {
    if (!h || !chosen) return RSK_ERR_INVALID_ARG;
    if (kernel != rsk::kTuneApply && kernel != rsk::kTuneSrtt)
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "kernel must be 0 (gather apply) or 1 (SRTT)");
    if (n < 1 || k < 1 || d < 1) return rsk::fail(h, RSK_ERR_INVALID_ARG, "empty shape");
    const size_t es = rsk::dtype_size(a_dtype);
    const size_t abytes = size_t(n) * size_t(k) * es;
    void* A = nullptr;
    void* SA = nullptr;
    cudaError_t e = cudaMallocAsync(&A, abytes + 16, stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&SA, size_t(d) * size_t(k) * 4, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (A) cudaFreeAsync(A, stream);
        return rsk::fail(h, RSK_ERR_NOMEM, "autotune buffers: %s", cudaGetErrorString(e));
    }
    const int64_t words = int64_t(abytes / 4);
    k_fill_pattern<<<unsigned((words + 255) / 256), 256, 0, stream>>>(static_cast<uint32_t*>(A), words);
    auto run = [&](uint64_t seed) -> rsk_status {
        return kernel == rsk::kTuneApply
                   ? rsk_sparse_sign_apply(h, A, a_dtype, n, k, k, d, zeta, seed, SA, RSK_F32, k, stream)
                   : rsk_srtt_apply(h, A, a_dtype, n, k, k, d, seed, SA, RSK_F32, k, stream);
    };
    // candidates around the default rule's value (sms / gcd(work pairs, sms)): the gather's pairs are
    // (128-byte column slices) x (sketch-row blocks), the SRTT's its 8-column slices
    auto gcd = [](int a, int b) {
        while (b) {
            const int t_ = a % b;
            a = b;
            b = t_;
        }
        return a;
    };
    int hi = 1, v0 = 1;
    if (kernel == rsk::kTuneApply) {
        const int64_t C = 768;  // rows per index chunk for zeta <= 8: no more ranges than chunks
        hi = int(std::max<int64_t>(1, (n + C - 1) / C));
        const int nslices = int((k + (128 / int(es)) - 1) / (128 / int(es)));
        const int max_slots = es == 2 ? 8 : 16;
        const int ntsub = int((d + max_slots * 64 - 1) / (max_slots * 64));
        const int pairs = nslices * ntsub;
        v0 = pairs >= h->num_sms ? 1 : h->num_sms / gcd(pairs, h->num_sms);
    } else {
        hi = int(std::max<int64_t>(1, (n + 2047) / 2048));
        const int nslices = int((k + 7) / 8);
        v0 = h->num_sms / gcd(nslices, h->num_sms);
    }
    v0 = std::max(1, std::min(hi, v0));
    std::vector<int> cand = around(std::max(1, v0), 1, hi);
    const int saved = h->tune_override;
    rsk_status st = RSK_OK;
    double best = 1e300;
    int pick = 0;
    // the default rule first (override -1), then each explicit candidate
    std::vector<int> tries = {-1};
    tries.insert(tries.end(), cand.begin(), cand.end());
    for (int v : tries) {
        h->tune_override = v;
        double ms = 0.0;
        st = time_calls(h, [&]() { return run(7); }, 3, stream, &ms);
        if (st != RSK_OK) break;
        if (ms < best) {
            best = ms;
            pick = v;
        }
    }
    h->tune_override = saved;
    cudaFreeAsync(A, stream);
    cudaFreeAsync(SA, stream);
    if (st != RSK_OK) return st;
    // the default rule winning leaves (or makes) the shape untuned
    if (pick < 0) pick = 0;
    store(kernel, int(a_dtype), n, k, d, h->num_sms, pick);
    *chosen = pick;
    if (best_ms) *best_ms = best;
    return RSK_OK;
}

rsk_status rsk_autotune_batched(rsk_handle* h, int32_t count, const rsk_lsq_problem* probs, const rsk_lsq_opts* opts,
                                int32_t* chosen, double* best_ms, cudaStream_t stream) {
    if (!h || !probs || !opts || !chosen || count < 1) return RSK_ERR_INVALID_ARG;
    std::vector<rsk_lsq_info> infos(static_cast<size_t>(count));
    int64_t total_rows = 0;
    for (int i = 0; i < count; ++i) total_rows += probs[i].n;
    const int saved = h->tune_override;
    rsk_status st = RSK_OK;
    double best = 1e300;
    int pick = 0;
    for (int v : {-1, 1024, 2048, 4096, 8192}) {
        h->tune_override = v;
        double ms = 0.0;
        st = time_calls(
            h,
            [&]() {
                const rsk_status s = rsk_lstsq_sketch_precond_batched(h, count, probs, opts, infos.data(), stream);
                return s == RSK_ERR_NOT_CONVERGED ? RSK_OK : s;
            },
            1, stream, &ms);
        if (st != RSK_OK) break;
        if (ms < best) {
            best = ms;
            pick = v;
        }
    }
    h->tune_override = saved;
    if (st != RSK_OK) return st;
    if (pick < 0) pick = 0;
    store(rsk::kTuneBatchTile, int(opts->inner_dtype), total_rows, count, 0, h->num_sms, pick);
    *chosen = pick;
    if (best_ms) *best_ms = best;
    return RSK_OK;
}

}  // extern "C"
