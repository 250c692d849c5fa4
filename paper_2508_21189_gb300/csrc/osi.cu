// Injectivity and dilation of a sparse test matrix on the adversarial subspace (Fig. 2, Sec. 1.5 and
// the experiment of Sec. 3): with Q = [e_1 ... e_r] and embedding dimension k, the estimates are
//     alpha = sigma_min^2(Omega^T Q),   beta = sigma_max^2(Omega^T Q),
// where Omega^T Q = S[:, 0:r] is the first r columns of the k x d sketch S (zeta nonzeros per column).
// They are the extreme eigenvalues of G = S_r^T S_r (r x r), estimated by `iters` Lanczos steps
// (no reorthogonalisation: the extreme Ritz values converge regardless, from inside the spectrum)
// and Sturm-count bisection on the Lanczos tridiagonal.
//
// Kernels
//   k_count / scan / k_fill / k_sort_rows   a deterministic CSR of S_r by rows: entries counted per row,
//                  an exclusive scan of the counts, each entry placed in its row's range by an atomic
//                  cursor, then every row's short list sorted by column (the order is unique)
//   k_rows_spmv    y = S_r v      (one thread per row of S_r, FP64)
//   k_cols_spmv    w = S_r^T y    (one thread per column: its zeta rows and signs as drawn)
//   k_dot_part / k_lanczos_*      FP64 reductions summed in block order, the three-term recurrence
//   k_sturm        bisection for the smallest and largest eigenvalue of the m x m tridiagonal
#include <math.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace {

constexpr int kScanBlock = 4096;  // elements per scan block (1024 threads x 4)

__global__ void k_count(const int32_t* __restrict__ rows, int64_t nnz, unsigned int* __restrict__ cnt) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < nnz) atomicAdd(cnt + rows[e], 1u);
}

// Exclusive scan of cnt[0 .. len) into ptr[0 .. len] (ptr[len] = total): block sums, a scan of the block
// sums in one CTA, then each block's local scan plus its offset.
__global__ void __launch_bounds__(1024) k_scan_blocks(const unsigned int* __restrict__ cnt, int64_t len,
                                                     unsigned long long* __restrict__ bsum) {
    __shared__ unsigned long long red[32];
    const int64_t base = int64_t(blockIdx.x) * kScanBlock;
    unsigned long long t = 0;
    for (int i = 0; i < 4; ++i) {
        const int64_t idx = base + threadIdx.x * 4 + i;
        if (idx < len) t += cnt[idx];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < 32; ++w) s += red[w];
        bsum[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(1024) k_scan_sums(unsigned long long* __restrict__ bsum, int nb) {
    __shared__ unsigned long long part[1024];
    const int per = (nb + 1023) / 1024;
    const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    unsigned long long t = 0;
    for (int b = b0; b < b1; ++b) t += bsum[b];
    part[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int i = 0; i < 1024; ++i) {
            const unsigned long long v = part[i];
            part[i] = run;
            run += v;
        }
    }
    __syncthreads();
    unsigned long long run = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        const unsigned long long v = bsum[b];
        bsum[b] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(1024) k_scan_local(const unsigned int* __restrict__ cnt, int64_t len,
                                                    const unsigned long long* __restrict__ boff,
                                                    int64_t* __restrict__ ptr) {
    __shared__ unsigned long long wsum[32];
    const int64_t base = int64_t(blockIdx.x) * kScanBlock;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long v[4], t = 0;
    for (int i = 0; i < 4; ++i) {
        const int64_t idx = base + threadIdx.x * 4 + i;
        v[i] = idx < len ? cnt[idx] : 0;
        t += v[i];
    }
    unsigned long long incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = wsum[lane];
        unsigned long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        wsum[lane] = wi - w;
    }
    __syncthreads();
    unsigned long long run = boff[blockIdx.x] + wsum[warp] + (incl - t);
    for (int i = 0; i < 4; ++i) {
        const int64_t idx = base + threadIdx.x * 4 + i;
        if (idx < len) ptr[idx] = int64_t(run);
        run += v[i];
        if (idx == len - 1) ptr[len] = int64_t(run);
    }
}

// Entry (j, q) goes to its row's next free slot; col = j | (negative << 31).
__global__ void k_fill(const int32_t* __restrict__ rows, const uint32_t* __restrict__ signs, int64_t r, int zeta,
                       const int64_t* __restrict__ ptr, unsigned int* __restrict__ cursor, uint32_t* __restrict__ col) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= r * zeta) return;
    const int64_t j = e / zeta;
    const int q = int(e - j * zeta);
    const int row = rows[e];
    const unsigned int slot = atomicAdd(cursor + row, 1u);
    col[ptr[row] + slot] = uint32_t(j) | (((signs[j] >> q) & 1u) << 31);
}

// Each row's list sorted by column (columns within a row are distinct, so the order is unique).
__global__ void k_sort_rows(const int64_t* __restrict__ ptr, int64_t k, uint32_t* __restrict__ col) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= k) return;
    const int64_t b = ptr[i], e = ptr[i + 1];
    for (int64_t a = b + 1; a < e; ++a) {
        const uint32_t v = col[a];
        const uint32_t key = v & 0x7fffffffu;
        int64_t t = a;
        while (t > b && (col[t - 1] & 0x7fffffffu) > key) {
            col[t] = col[t - 1];
            --t;
        }
        col[t] = v;
    }
}

__global__ void k_rows_spmv(const int64_t* __restrict__ ptr, const uint32_t* __restrict__ col, int64_t k,
                            const double* __restrict__ v, double scale, double* __restrict__ y) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= k) return;
    double t = 0.0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        const uint32_t c = col[e];
        const double x = v[c & 0x7fffffffu];
        t += (c >> 31) ? -x : x;
    }
    y[i] = t * scale;
}

__global__ void k_cols_spmv(const int32_t* __restrict__ rows, const uint32_t* __restrict__ signs, int64_t r, int zeta,
                            const double* __restrict__ y, double scale, double* __restrict__ w) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= r) return;
    const uint32_t sb = signs[j];
    double t = 0.0;
    for (int q = 0; q < zeta; ++q) {
        const double x = y[rows[j * zeta + q]];
        t += ((sb >> q) & 1u) ? -x : x;
    }
    w[j] = t * scale;
}

constexpr int kRedBlocks = 512;

// part[b] = sum over the block's grid-stride share of a[i] * b[i]
__global__ void k_dot_part(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                           double* __restrict__ part) {
    __shared__ double red[32];
    double t = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        t = fma(a[i], b[i], t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

// alpha[j] = sum of the parts (in block order)
__global__ void k_sum_parts(const double* __restrict__ part, int nparts, double* __restrict__ out, bool sqrt_it) {
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += part[i];
    *out = sqrt_it ? sqrt(s) : s;
}

// w = w - alpha v - beta_prev v_prev
__global__ void k_lanczos_update(double* __restrict__ w, const double* __restrict__ v, const double* __restrict__ vp,
                                 int64_t n, const double* __restrict__ alpha, const double* __restrict__ beta_prev) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double bp = beta_prev ? *beta_prev : 0.0;
    w[i] = w[i] - *alpha * v[i] - (vp ? bp * vp[i] : 0.0);
}

__global__ void k_fill_value(double* __restrict__ x, int64_t n, double val) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) x[i] = val;
}

// v_prev = v; v = w / beta (beta = 0 leaves v = 0: an invariant subspace was found)
__global__ void k_lanczos_next(double* __restrict__ vp, double* __restrict__ v, const double* __restrict__ w,
                               int64_t n, const double* __restrict__ beta) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double b = *beta;
    vp[i] = v[i];
    v[i] = b > 0.0 ? w[i] / b : 0.0;
}

// Number of eigenvalues of the tridiagonal (diag a[0..m), off-diagonal b[0..m-1)) below x.
__device__ int sturm_count(const double* a, const double* b, int m, double x) {
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
        const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
        d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++c;
    }
    return c;
}

// out[0] = smallest, out[1] = largest eigenvalue of the tridiagonal, by bisection from the Gershgorin
// interval (two threads).
__global__ void k_sturm(const double* __restrict__ a, const double* __restrict__ b, int m, double* __restrict__ out) {
    const int t = threadIdx.x;
    if (t > 1) return;
    // a vanishing b_j means the Krylov space closed after j + 1 steps (an invariant subspace): the
    // later steps ran on a zero vector, so only the leading (j + 1) x (j + 1) block is the tridiagonal
    double amax = 0.0;
    for (int i = 0; i < m; ++i) amax = fmax(amax, fabs(a[i]));
    for (int i = 0; i + 1 < m; ++i)
        if (!(fabs(b[i]) > 1e-13 * amax)) {
            m = i + 1;
            break;
        }
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; ++i) {
        const double rad = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0);
        lo = fmin(lo, a[i] - rad);
        hi = fmax(hi, a[i] + rad);
    }
    const int target = t == 0 ? 1 : m;  // smallest: count(x) >= 1; largest: count(x) >= m
    for (int it = 0; it < 200 && hi - lo > 1e-15 * fmax(fabs(lo), fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(a, b, m, mid) >= target) hi = mid;
        else lo = mid;
    }
    out[t] = 0.5 * (lo + hi);
}

}  // namespace

extern "C" rsk_status rsk_osi_estimate(rsk_handle* h, int64_t r, int64_t k, int32_t zeta, uint64_t seed, int32_t kind,
                                       int32_t iters, double* alpha, double* beta, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!alpha || !beta) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null output");
    if (r < 1 || k < 1 || r >= (int64_t(1) << 31) || k >= (int64_t(1) << 31) || r * int64_t(zeta) >= (int64_t(1) << 31))
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "need 1 <= r, k < 2^31 and r * zeta < 2^31");
    if (kind != 0 && kind != 1) return rsk::fail(h, RSK_ERR_INVALID_ARG, "kind must be 0 (SparseUniform) or 1 (SparseStack)");
    if (iters < 1 || iters > 100000) return rsk::fail(h, RSK_ERR_INVALID_ARG, "need 1 <= iters <= 100000");
    const int m = int(std::min<int64_t>(iters, r));
    const int64_t nnz = r * zeta;
    const int64_t nb = (k + 1 + kScanBlock - 1) / kScanBlock;
    using rsk::Carver;
    const size_t bytes = Carver::round(size_t(nnz) * 4) + Carver::round(size_t(r) * 4) + Carver::round(size_t(k) * 4) * 2 +
                         Carver::round(size_t(k + 1) * 8) + Carver::round(size_t(nb) * 8) + Carver::round(size_t(nnz) * 4) +
                         3 * Carver::round(size_t(r) * 8) + Carver::round(size_t(k) * 8) + 2 * Carver::round(size_t(m + 1) * 8) +
                         Carver::round(kRedBlocks * 8) + 1024;
    rsk_status st = rsk::ensure_workspace(h, bytes, stream);
    if (st != RSK_OK) return st;
    Carver cv(h->ws);
    int32_t* rows = cv.take<int32_t>(size_t(nnz));
    uint32_t* signs = cv.take<uint32_t>(size_t(r));
    unsigned int* cnt = cv.take<unsigned int>(size_t(k));
    unsigned int* cursor = cv.take<unsigned int>(size_t(k));
    int64_t* ptr = cv.take<int64_t>(size_t(k + 1));
    unsigned long long* bsum = cv.take<unsigned long long>(size_t(nb));
    uint32_t* col = cv.take<uint32_t>(size_t(nnz));
    double* vp = cv.take<double>(size_t(r));
    double* v = cv.take<double>(size_t(r));
    double* w = cv.take<double>(size_t(r));
    double* y = cv.take<double>(size_t(k));
    double* al = cv.take<double>(size_t(m + 1));
    double* be = cv.take<double>(size_t(m + 1));
    double* part = cv.take<double>(kRedBlocks);

    // S_r: the first r columns of the k x d sketch (they do not depend on d)
    st = rsk::sketch_generate_large(h, r, k, zeta, seed, kind, rows, signs, stream);
    if (st != RSK_OK) return st;
    RSK_CUDA_TRY(h, cudaMemsetAsync(cnt, 0, size_t(k) * 4, stream));
    RSK_CUDA_TRY(h, cudaMemsetAsync(cursor, 0, size_t(k) * 4, stream));
    const unsigned ge = unsigned((nnz + 255) / 256);
    k_count<<<ge, 256, 0, stream>>>(rows, nnz, cnt);
    k_scan_blocks<<<unsigned(nb), 1024, 0, stream>>>(cnt, k, bsum);
    k_scan_sums<<<1, 1024, 0, stream>>>(bsum, int(nb));
    k_scan_local<<<unsigned(nb), 1024, 0, stream>>>(cnt, k, bsum, ptr);
    k_fill<<<ge, 256, 0, stream>>>(rows, signs, r, zeta, ptr, cursor, col);
    k_sort_rows<<<unsigned((k + 255) / 256), 256, 0, stream>>>(ptr, k, col);
    RSK_LAUNCH_CHECK(h);

    // Lanczos on G = S_r^T S_r from v_1 = (1, ..., 1) / sqrt(r) (a fixed start; a random S_r makes it
    // orthogonal to no eigenvector with probability one)
    const double sc = 1.0 / sqrt(double(zeta));
    const unsigned gr = unsigned((r + 255) / 256), gk = unsigned((k + 255) / 256);
    k_fill_value<<<gr, 256, 0, stream>>>(v, r, 1.0 / sqrt(double(r)));
    RSK_CUDA_TRY(h, cudaMemsetAsync(vp, 0, size_t(r) * 8, stream));
    for (int j = 0; j < m; ++j) {
        k_rows_spmv<<<gk, 256, 0, stream>>>(ptr, col, k, v, sc, y);
        k_cols_spmv<<<gr, 256, 0, stream>>>(rows, signs, r, zeta, y, sc, w);
        k_dot_part<<<kRedBlocks, 256, 0, stream>>>(v, w, r, part);
        k_sum_parts<<<1, 1, 0, stream>>>(part, kRedBlocks, al + j, false);
        k_lanczos_update<<<gr, 256, 0, stream>>>(w, v, vp, r, al + j, j > 0 ? be + (j - 1) : nullptr);
        k_dot_part<<<kRedBlocks, 256, 0, stream>>>(w, w, r, part);
        k_sum_parts<<<1, 1, 0, stream>>>(part, kRedBlocks, be + j, true);
        k_lanczos_next<<<gr, 256, 0, stream>>>(vp, v, w, r, be + j);
    }
    RSK_LAUNCH_CHECK(h);
    k_sturm<<<1, 32, 0, stream>>>(al, be, m, part);
    RSK_LAUNCH_CHECK(h);
    double ext[2];
    RSK_CUDA_TRY(h, cudaMemcpyAsync(ext, part, 16, cudaMemcpyDeviceToHost, stream));
    RSK_CUDA_TRY(h, cudaStreamSynchronize(stream));
    *alpha = ext[0];
    *beta = ext[1];
    return RSK_OK;
}
