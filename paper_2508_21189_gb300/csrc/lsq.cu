// Sketch-and-precondition least squares (rows a5-a7): min_x ||A x - b||_2 for tall A (n x k).
// Paper: sketch-and-solve, Alg. 3 (Sec. 2.3) gives the warm start from the sketched problem; the
// paper names sketch-and-precondition as the standard high-accuracy route (remark closing Sec. 2.3)
// without stating it, so the steps are this library's reading:
//   L1  [Ahat | bhat] = S [A | b] with one sparse sign S (rsk_sparse_sign_plan_*).
//   L2  Householder QR of Ahat in FP64, one reflector per column: k_qr_col (one CTA per column,
//       column in registers, reflectors handed on through release/acquire flags) when k + 1 CTAs
//       fit on the GPU at once, else k_qr (persistent grid, bounded software grid barrier); Q^T bhat
//       comes out of the same sweep as an extra column.
//   L3  x0 = R^{-1} Q^T bhat; R^{-1} is formed explicitly (k_rinv, FP64) and applied as a matvec.
//   L4  refinement: g = A^T (b - A x) in FP64 (one fused pass over A), eta(x) = ||g|| / (||A||_F ||r||);
//       stop at eta <= tol; otherwise solve (M^T M) z = R^{-T} g with CG, M = A R^{-1}, whose
//       products M^T M p = R^{-T} A^T A R^{-1} p are one fused pass over A in the inner precision,
//       and set x += R^{-1} z.  Because the right-hand side is the FP64 normal-equation residual,
//       the fixed point is A^T r = 0 to FP64 accuracy whatever the inner precision; the inner
//       precision only sets the contraction per step.
#include <cuda_bf16.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kPassThreads = 256;      // fused normal-equation passes
constexpr int kMaxK = 1024;

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];  // same order in every thread
    return s;
}

// ------------------------------------------------------------------------------------------
// L2: Householder QR of W = [Ahat | bhat] (d x (k+1), column-major, leading dimension d).
// Column c is owned by CTA c % gridDim.x.  Step j: the owner of column j has it fully updated
// and forms reflector j (beta into W[j,j], v below the diagonal with v_j = 1 implicit, tau_j);
// after one grid barrier every CTA applies reflector j to the columns c > j it owns.
// ------------------------------------------------------------------------------------------
__device__ void make_reflector(double* col, int d, int j, double* tau, double* red) {
    double s = 0.0;
    for (int i = j + 1 + threadIdx.x; i < d; i += blockDim.x) {
        const double v = __ldcg(col + i);
        s += v * v;
    }
    const double sigma = block_sum(s, red);
    const double alpha = __ldcg(col + j);
    double t = 0.0, beta = alpha, scale = 0.0;
    if (sigma > 0.0) {
        const double nrm = sqrt(alpha * alpha + sigma);
        beta = alpha > 0.0 ? -nrm : nrm;
        t = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
    }
    if (sigma > 0.0)
        for (int i = j + 1 + threadIdx.x; i < d; i += blockDim.x) col[i] = __ldcg(col + i) * scale;
    __syncthreads();
    if (threadIdx.x == 0) {
        col[j] = beta;
        tau[j] = t;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_qr(double* W, int d, int k, double* tau, unsigned int* bar,
                                           unsigned int* status, uint32_t limit) {
    __shared__ double red[32];
    const unsigned int G = gridDim.x;
    const int cols = k + 1;
    if (blockIdx.x == 0) make_reflector(W, d, 0, tau, red);
    for (int j = 0; j < k; ++j) {
        if (!rskd::grid_barrier(bar, bar + 1, G, status, limit)) return;
        // Reflector j was written by another CTA: read it through L2 (ld.cg), never from a line this
        // SM's L1 may hold from an earlier step.
        const double* v = W + size_t(j) * d;
        const double tj = __ldcg(tau + j);
        for (int c = j + 1 + ((int(blockIdx.x) - (j + 1)) % int(G) + int(G)) % int(G); c < cols; c += G) {
            double* col = W + size_t(c) * d;
            double s = 0.0;
            for (int i = j + 1 + threadIdx.x; i < d; i += blockDim.x) s += __ldcg(v + i) * __ldcg(col + i);
            const double w = tj * (__ldcg(col + j) + block_sum(s, red));
            if (threadIdx.x == 0) col[j] = __ldcg(col + j) - w;
            for (int i = j + 1 + threadIdx.x; i < d; i += blockDim.x) col[i] = __ldcg(col + i) - w * __ldcg(v + i);
            __syncthreads();
            if (c == j + 1 && c < k) make_reflector(col, d, c, tau, red);
        }
    }
}

// The same QR with one CTA per column (grid = k + 1, all resident: cooperative launch) and no grid
// barrier.  CTA c keeps column c in registers (row i = threadIdx.x + 256 t, t < T).  For
// j = 0 .. min(c, k) - 1 it waits until reflector j is published (ready[j]), reads v_j and tau_j
// through L2 and applies H_j; CTA c < k then forms reflector c from rows c.., writes its column
// (R entries in rows < c, beta in row c, v_c below) and tau_c, and publishes ready[c].  Reflector
// j + 1 therefore follows reflector j after one flag hand-off, one L2 read of v_j and two block
// reductions, instead of a grid barrier and several L2 round trips of the column.
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int T>
__global__ void __launch_bounds__(256) k_qr_col(double* W, int d, int k, double* tau, unsigned int* ready,
                                               unsigned int* status, uint32_t limit) {
    __shared__ double red[32];
    __shared__ double xj_s;
    __shared__ int ok_s;
    const int c = blockIdx.x, tid = threadIdx.x;
    double* col = W + size_t(c) * d;
    double x[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int i = tid + 256 * t;
        x[t] = i < d ? col[i] : 0.0;
    }
    const int nref = c < k ? c : k;
    for (int j = 0; j < nref; ++j) {
        if (tid == 0) {
            uint32_t it = 0;
            int ok = 1;
            while (ld_acquire_u32(ready + j) == 0u) {
                if (++it > limit) {
                    atomicOr(status, RSK_DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
                if (it > 32) __nanosleep(32);
            }
            ok_s = ok;
        }
        __syncthreads();
        if (!ok_s) return;
        const double* v = W + size_t(j) * d;
        const double tj = __ldcg(tau + j);
        double vv[T];
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + 256 * t;
            vv[t] = (i > j && i < d) ? __ldcg(v + i) : 0.0;
            s += vv[t] * x[t];
            if (i == j) xj_s = x[t];
        }
        s = block_sum(s, red);  // its barriers also publish xj_s
        const double w = tj * (xj_s + s);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + 256 * t;
            x[t] -= (i == j) ? w : w * vv[t];
        }
    }
    if (c < k) {
        double sg = 0.0, ap = 0.0;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + 256 * t;
            if (i > c && i < d) sg += x[t] * x[t];
            if (i == c) ap = x[t];
        }
        const double sigma = block_sum(sg, red);
        const double alpha = block_sum(ap, red);  // one nonzero term: exact
        double tc = 0.0, beta = alpha, scale = 0.0;
        if (sigma > 0.0) {
            const double nrm = sqrt(alpha * alpha + sigma);
            beta = alpha > 0.0 ? -nrm : nrm;
            tc = (beta - alpha) / beta;
            scale = 1.0 / (alpha - beta);
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + 256 * t;
            if (i > c && sigma > 0.0) x[t] *= scale;
            if (i == c) x[t] = beta;
            if (i < d) col[i] = x[t];
        }
        if (tid == 0) tau[c] = tc;
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release_u32(ready + c, 1u);
    } else {
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + 256 * t;
            if (i < d) col[i] = x[t];
        }
    }
}

// R^{-1} of the upper triangle of W (column-major, ld d) into X (k x k column-major): one warp
// per column c solves R x = e_c by column-oriented back substitution.
__global__ void k_rinv(const double* __restrict__ W, int d, int k, double* __restrict__ X) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= k) return;
    const int c = warp;
    double* x = X + size_t(c) * k;
    for (int i = lane; i < k; i += 32) x[i] = (i == c) ? 1.0 : 0.0;
    __syncwarp();
    for (int l = c; l >= 0; --l) {
        const double* Rl = W + size_t(l) * d;  // column l of R
        const double xl = x[l] / Rl[l];
        __syncwarp();
        if (lane == 0) x[l] = xl;
        for (int i = lane; i < l; i += 32) x[i] -= Rl[i] * xl;
        __syncwarp();
    }
}

// y = op(X) v for X k x k column-major upper triangular (op = X or X^T); one warp per output.
__global__ void k_trmv(const double* __restrict__ X, int k, int trans, const double* __restrict__ v,
                       double* __restrict__ y) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= k) return;
    double s = 0.0;
    if (!trans) {
        for (int l = i + lane; l < k; l += 32) s += X[size_t(l) * k + i] * v[l];   // row i of X
    } else {
        for (int l = lane; l <= i; l += 32) s += X[size_t(i) * k + l] * v[l];      // column i of X
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[i] = s;
}

// ------------------------------------------------------------------------------------------
// Fused passes over A.  Each warp walks rows; lane l holds columns l, l+32, ... of the row.
//   CG pass   (Acc = float):  w_i = a_i . y,  q += w_i a_i          (q = A^T A y)
//   residual  (Acc = double): r_i = b_i - a_i . x, g += r_i a_i, rr += r_i^2, ff += |a_i|^2
// Per-CTA partials are reduced in CTA order by k_reduce_parts (deterministic).
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ float to_float(T v) {
    return float(v);
}

template <typename T, typename Acc, int M, bool RESID>
__global__ void __launch_bounds__(kPassThreads) k_pass(const T* __restrict__ A, int64_t n, int k, int64_t lda,
                                                        const Acc* __restrict__ y, const double* __restrict__ b,
                                                        Acc* __restrict__ part, double* __restrict__ part_s,
                                                        int want_frob) {
    // dynamic shared memory: gs[warps][k] (per-warp partial sums), ys[k]
    extern __shared__ __align__(16) uint8_t dsm[];
    Acc* gs = reinterpret_cast<Acc*>(dsm);
    Acc* ys = gs + size_t(kPassThreads / 32) * k;
    for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = y[j];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const int64_t r0 = int64_t(blockIdx.x) * n / gridDim.x, r1 = int64_t(blockIdx.x + 1) * n / gridDim.x;
    Acc g[M], yv[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        g[m] = Acc(0);
        const int j = lane + 32 * m;
        yv[m] = j < k ? ys[j] : Acc(0);
    }
    double rr = 0.0, ff = 0.0, bb = 0.0;
    for (int64_t i = r0 + warp; i < r1; i += nw) {
        const T* row = A + i * lda;
        Acc a[M];
        Acc dot = Acc(0);
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int j = lane + 32 * m;
            if constexpr (sizeof(Acc) == 8) a[m] = j < k ? Acc(row[j]) : Acc(0);
            else a[m] = j < k ? Acc(to_float<T>(row[j])) : Acc(0);
            dot += a[m] * yv[m];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        Acc w = dot;
        if constexpr (RESID) {
            w = Acc(b[i]) - dot;
            if (lane == 0) rr += double(w) * double(w);  // every lane holds the same r_i
            if (want_frob) {
#pragma unroll
                for (int m = 0; m < M; ++m) ff += double(a[m]) * double(a[m]);
                if (lane == 0) bb += b[i] * b[i];
            }
        }
#pragma unroll
        for (int m = 0; m < M; ++m) g[m] += w * a[m];
    }
    // reduce the warps' partial g in a fixed order through shared memory
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int j = lane + 32 * m;
        if (j < k) gs[size_t(warp) * k + j] = g[m];
    }
    __shared__ double ss[kPassThreads / 32][3];
    if constexpr (RESID) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rr += __shfl_xor_sync(0xffffffffu, rr, o);
            ff += __shfl_xor_sync(0xffffffffu, ff, o);
        }
        if (lane == 0) {
            ss[warp][0] = rr;
            ss[warp][1] = ff;
            ss[warp][2] = bb;
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        Acc s = Acc(0);
        for (int w = 0; w < nw; ++w) s += gs[size_t(w) * k + j];
        part[size_t(blockIdx.x) * k + j] = s;
    }
    if (RESID && threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < nw; ++w) {
            a0 += ss[w][0];
            a1 += ss[w][1];
            a2 += ss[w][2];
        }
        part_s[3 * blockIdx.x] = a0;
        part_s[3 * blockIdx.x + 1] = a1;
        part_s[3 * blockIdx.x + 2] = a2;
    }
}

// ---- double-float operator on interleaved (hi, lo) FP32 pairs ---------------------------------
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// (hi, lo) += (ah + al) * (yh + yl), dropping al*yl (below 2^-48 relative)
__device__ __forceinline__ void df_mac(float& hi, float& lo, float ah, float al, float yh, float yl) {
    const float p = ah * yh;
    const float pe = fmaf(ah, yh, -p);
    const float t = fmaf(ah, yl, fmaf(al, yh, pe));
    float s, e;
    two_sum_f(hi, p, s, e);
    e += lo + t;
    hi = s + e;
    lo = e - (hi - s);
}
__device__ __forceinline__ void df_add(float& hi, float& lo, float oh, float ol) {
    float s, e;
    two_sum_f(hi, oh, s, e);
    e += lo + ol;
    hi = s + e;
    lo = e - (hi - s);
}
__device__ __forceinline__ void df_xor_add(float& h, float& l, float sh, float sl, int o) {
    const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
    df_add(h, l, oh, ol);
}

// FP64 -> (hi, lo) with hi = RN32(a) and lo = RN32(a - hi), in integer arithmetic only (FP64
// conversions run on the FP64 pipe, which is the scarce unit on this part).  Values outside the
// FP32 normal range are flushed: |a| < 2^-126 gives (+-0, 0), |a| beyond FLT_MAX gives +-inf, a lo
// below 2^-126 becomes 0 -- a normwise perturbation of at most 2^-126 per entry.
__device__ __forceinline__ float2 split_pair(double a) {
    const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(a));
    const uint32_t sign = uint32_t(u >> 63) << 31;
    const int e = int((u >> 52) & 0x7ffu);
    const unsigned long long m = u & 0xfffffffffffffull;
    if (e == 0x7ff) return make_float2(__uint_as_float(sign | 0x7f800000u | (m ? 0x400000u : 0u)), 0.f);
    const int E = e - 1023;
    if (E < -126) return make_float2(__uint_as_float(sign), 0.f);
    if (E > 127) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
    const uint32_t mh = uint32_t(m >> 29);
    const uint32_t rem = uint32_t(m & 0x1fffffffu);
    const bool up = rem > 0x10000000u || (rem == 0x10000000u && (mh & 1u));
    // a carry out of the significand moves into the exponent field (and to inf past FLT_MAX)
    const uint32_t hb = (uint32_t(E + 127) << 23) + mh + (up ? 1u : 0u);
    const float hi = __uint_as_float(sign | hb);
    // a - hi = +rem * 2^(E-52) (rounded down) or -(2^29 - rem) * 2^(E-52) (rounded up), exactly
    const uint32_t r = up ? (0x20000000u - rem) : rem;
    if (r == 0u) return make_float2(hi, 0.f);
    const uint32_t lsign = up ? (sign ^ 0x80000000u) : sign;
    const int p = 31 - __clz(r);
    int el = p + E - 52;
    uint32_t ml;
    if (p > 23) {
        const int sh = p - 23;
        ml = r >> sh;
        const uint32_t rest = r & ((1u << sh) - 1u), half = 1u << (sh - 1);
        if (rest > half || (rest == half && (ml & 1u))) ++ml;
        if (ml == (1u << 24)) {
            ml >>= 1;
            ++el;
        }
    } else {
        ml = r << (23 - p);
    }
    if (el < -126) return make_float2(hi, 0.f);
    return make_float2(hi, __uint_as_float(lsign | (uint32_t(el + 127) << 23) | (ml & 0x7fffffu)));
}

// A (F64 or F32, lda) -> P (n x k interleaved pairs)
template <typename T>
__global__ void k_to_pairs(const T* __restrict__ A, int64_t n, int k, int64_t lda, float2* __restrict__ P) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    const int64_t i = idx / k, j = idx - i * k;
    if constexpr (sizeof(T) == 8) P[idx] = split_pair(A[i * lda + j]);
    else P[idx] = make_float2(float(A[i * lda + j]), 0.f);
}

// Fused pass over the pairs, two rows per warp at a time (partial dot products reduce-scattered
// so lane L ends with row bit4(L)).  RESID: r_i = b_i - a_i . x (b as pairs too), g += r_i a_i,
// ||r||^2, ||A||_F^2, ||b||^2.  CG: w_i = a_i . y, g += w_i a_i.
template <int M, bool RESID>
__global__ void __launch_bounds__(kPassThreads, 2) k_pass_pairs(const float2* __restrict__ P, int64_t n, int k,
                                                             const double* __restrict__ y,
                                                             const double* __restrict__ b,
                                                             double* __restrict__ part,
                                                             double* __restrict__ part_s, int want_frob) {
    extern __shared__ __align__(16) uint8_t dsm[];
    double* gs = reinterpret_cast<double*>(dsm);
    float* yh = reinterpret_cast<float*>(gs + size_t(kPassThreads / 32) * k);
    float* yl = yh + 32 * M;
    for (int j = threadIdx.x; j < 32 * M; j += blockDim.x) {
        const double v = j < k ? y[j] : 0.0;
        const float h = float(v);
        yh[j] = h;
        yl[j] = float(v - double(h));
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int mk = (k + 31) >> 5;
    const int64_t r0 = int64_t(blockIdx.x) * n / gridDim.x, r1 = int64_t(blockIdx.x + 1) * n / gridDim.x;
    float gh[M], gl[M];
#pragma unroll
    for (int m = 0; m < M; ++m) gh[m] = gl[m] = 0.f;
    float rrf = 0.f, fff = 0.f, bbf = 0.f;
    for (int64_t i0 = r0 + 2 * warp; i0 < r1; i0 += 2 * nw) {
        float2 a[2][M];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const bool valid = i0 + r < r1;
            const float2* row = P + (i0 + r) * int64_t(k);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int j = lane + 32 * m;
                a[r][m] = (m < mk && valid && j < k) ? row[j] : make_float2(0.f, 0.f);
            }
        }
        float ph[2] = {0.f, 0.f}, pl[2] = {0.f, 0.f};
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int m = 0; m < M; ++m)
                if (m < mk) {
                    const int j = lane + 32 * m;
                    df_mac(ph[r], pl[r], a[r][m].x, a[r][m].y, yh[j], yl[j]);
                    if (RESID && want_frob) fff = fmaf(a[r][m].x, a[r][m].x, fff);
                }
        // reduce-scatter: lanes with bit 4 clear keep row 0, set keep row 1
        const bool b4 = lane & 16;
        float dh = b4 ? ph[1] : ph[0], dl = b4 ? pl[1] : pl[0];
        df_xor_add(dh, dl, b4 ? ph[0] : ph[1], b4 ? pl[0] : pl[1], 16);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) df_xor_add(dh, dl, dh, dl, o);
        float wh = dh, wl = dl;
        if constexpr (RESID) {
            const int64_t irow = i0 + (b4 ? 1 : 0);
            wh = wl = 0.f;
            if (irow < r1) {
                const double bi = b[irow];
                const float bh = float(bi), bl = float(bi - double(bh));
                float s_, e_;
                two_sum_f(bh, -dh, s_, e_);
                e_ += bl - dl;
                wh = s_ + e_;
                wl = e_ - (wh - s_);
                if ((lane & 15) == 0) {
                    rrf = fmaf(wh, wh, rrf);
                    bbf = fmaf(bh, bh, bbf);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float w_h = __shfl_sync(0xffffffffu, wh, r << 4);
            const float w_l = __shfl_sync(0xffffffffu, wl, r << 4);
#pragma unroll
            for (int m = 0; m < M; ++m)
                if (m < mk) df_mac(gh[m], gl[m], a[r][m].x, a[r][m].y, w_h, w_l);
        }
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int j = lane + 32 * m;
        if (j < k) gs[size_t(warp) * k + j] = double(gh[m]) + double(gl[m]);
    }
    __shared__ double ss[kPassThreads / 32][3];
    if constexpr (RESID) {
        double rr = double(rrf), ff = double(fff), bb = double(bbf);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rr += __shfl_xor_sync(0xffffffffu, rr, o);
            ff += __shfl_xor_sync(0xffffffffu, ff, o);
            bb += __shfl_xor_sync(0xffffffffu, bb, o);
        }
        if (lane == 0) {
            ss[warp][0] = rr;
            ss[warp][1] = ff;
            ss[warp][2] = bb;
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double acc = 0.0;
        for (int w = 0; w < nw; ++w) acc += gs[size_t(w) * k + j];
        part[size_t(blockIdx.x) * k + j] = acc;
    }
    if (RESID && threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < nw; ++w) {
            a0 += ss[w][0];
            a1 += ss[w][1];
            a2 += ss[w][2];
        }
        part_s[3 * blockIdx.x] = a0;
        part_s[3 * blockIdx.x + 1] = a1;
        part_s[3 * blockIdx.x + 2] = a2;
    }
}

template <typename Acc>
__global__ void k_reduce_parts(const Acc* __restrict__ part, int nparts, int k, double* __restrict__ out,
                               const double* __restrict__ part_s, double* __restrict__ out_s) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) {
        double s = 0.0;
        for (int p = 0; p < nparts; ++p) s += double(part[size_t(p) * k + j]);
        out[j] = s;
    }
    if (part_s && j < 3) {
        double s = 0.0;
        for (int p = 0; p < nparts; ++p) s += part_s[3 * p + j];
        out_s[j] = s;
    }
}

// ------------------------------------------------------------------------------------------
// Small vector kernels (k entries, one CTA).
// ------------------------------------------------------------------------------------------
// State of the CG iteration: [0] rho, [1] rho0, [2] done flag, [3] iterations done.
__global__ void k_cg_init(const double* __restrict__ c, double* __restrict__ z, double* __restrict__ res,
                          double* __restrict__ p, int k, double* __restrict__ state) {
    __shared__ double red[32];
    double s = 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        z[j] = 0.0;
        res[j] = c[j];
        p[j] = c[j];
        s += c[j] * c[j];
    }
    const double rho = block_sum(s, red);
    if (threadIdx.x == 0) {
        state[0] = rho;
        state[1] = rho;
        state[2] = rho > 0.0 ? 0.0 : 1.0;
        state[3] = 0.0;
    }
}

// s = M^T M p (already computed); z += alpha p, res -= alpha s, p = res + beta p.
__global__ void k_cg_step(const double* __restrict__ s, double* __restrict__ z, double* __restrict__ res,
                          double* __restrict__ p, int k, double* __restrict__ state, double tol) {
    __shared__ double red[32];
    if (state[2] != 0.0) return;
    double ps = 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) ps += p[j] * s[j];
    const double pAp = block_sum(ps, red);
    const double rho = state[0];
    const double alpha = pAp > 0.0 ? rho / pAp : 0.0;
    double rn = 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        z[j] += alpha * p[j];
        res[j] -= alpha * s[j];
        rn += res[j] * res[j];
    }
    const double rho_new = block_sum(rn, red);
    const double beta = rho > 0.0 ? rho_new / rho : 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) p[j] = res[j] + beta * p[j];
    __syncthreads();
    if (threadIdx.x == 0) {
        state[0] = rho_new;
        state[3] += 1.0;
        if (!(pAp > 0.0) || rho_new <= tol * tol * state[1]) state[2] = 1.0;
    }
}

template <typename Acc>
__global__ void k_cast_vec(const double* __restrict__ src, Acc* __restrict__ dst, int k, const double* state) {
    if (state && state[2] != 0.0) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) dst[j] = Acc(src[j]);
}

__global__ void k_axpy(double* __restrict__ x, const double* __restrict__ dx, int k) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) x[j] += dx[j];
}

// [Ahat | bhat] row-major (d x k, ldsa; d x 1) -> W column-major FP64.
template <typename S>
__global__ void k_to_colmajor(const S* __restrict__ SA, int64_t ldsa, const double* __restrict__ Sb, int d, int k,
                              double* __restrict__ W) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= int64_t(d) * (k + 1)) return;
    const int c = int(idx / d), i = int(idx - int64_t(c) * d);
    W[idx] = c < k ? double(SA[int64_t(i) * ldsa + c]) : double(Sb[i]);
}

template <typename Src, typename Dst>
__global__ void k_convert(const Src* __restrict__ A, int64_t n, int k, int64_t lda, Dst* __restrict__ B) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    const int64_t i = idx / k, j = idx - i * k;
    B[idx] = Dst(float(A[i * lda + j]));
}
}  // namespace

// ------------------------------------------------------------------------------------------
// Host driver.
// ------------------------------------------------------------------------------------------
namespace rsk {

struct LsqWork {
    double *W, *tau, *Rinv, *x, *g, *c, *z, *res, *p, *s, *t, *stats, *parts_s;
    void* parts;
    void* yv;
    unsigned int* bar;
    float* SA32;
    double* SA64;
    void* Sb;
    void* Alow;  // converted copy of A (sketch / inner precision) when needed
};

template <typename T, typename Acc>
static rsk_status launch_pass(rsk_handle* h, const T* A, int64_t n, int k, int64_t lda, const Acc* y, const double* b,
                              Acc* parts, double* parts_s, int nparts, bool resid, bool frob, cudaStream_t stream) {
    const int M = (k + 31) / 32;
    const size_t smem = (size_t(kPassThreads / 32) + 1) * k * sizeof(Acc);
    rsk_status err = RSK_OK;
    auto go = [&](auto kern) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) {
            err = RSK_ERR_CUDA;
            return;
        }
        kern<<<unsigned(nparts), kPassThreads, smem, stream>>>(A, n, k, lda, y, b, parts, parts_s, frob ? 1 : 0);
    };
    const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_DENSE);
#define RSK_PASS_CASE(MM)                                          \
    case MM:                                                       \
        if (resid) go(k_pass<T, Acc, MM, true>);                   \
        else go(k_pass<T, Acc, MM, false>);                        \
        break;
    switch (M <= 4 ? 4 : (M <= 8 ? 8 : (M <= 16 ? 16 : 32))) {
        RSK_PASS_CASE(4)
        RSK_PASS_CASE(8)
        RSK_PASS_CASE(16)
        RSK_PASS_CASE(32)
        default: return rsk::fail(h, RSK_ERR_INTERNAL, "bad pass width");
    }
#undef RSK_PASS_CASE
    rsk::prof_end(h, stream, pr);
    if (err != RSK_OK) return rsk::fail(h, err, "cudaFuncSetAttribute failed for the fused pass");
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

static rsk_status launch_pass_pairs(rsk_handle* h, const float2* P, int64_t n, int k, const double* y,
                                    const double* b, double* parts, double* parts_s, int nparts, bool resid, bool frob,
                                    cudaStream_t stream) {
    const int M = (k + 31) / 32;
    const int Mt = M <= 4 ? 4 : M <= 8 ? 8 : M <= 16 ? 16 : 32;
    const size_t smem = size_t(kPassThreads / 32) * k * 8 + size_t(32) * Mt * 4 * 2;
    rsk_status err = RSK_OK;
    auto go = [&](auto kern) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) {
            err = RSK_ERR_CUDA;
            return;
        }
        kern<<<unsigned(nparts), kPassThreads, smem, stream>>>(P, n, k, y, b, parts, parts_s, frob ? 1 : 0);
    };
    const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_DENSE);
    if (Mt == 4) resid ? go(k_pass_pairs<4, true>) : go(k_pass_pairs<4, false>);
    else if (Mt == 8) resid ? go(k_pass_pairs<8, true>) : go(k_pass_pairs<8, false>);
    else if (Mt == 16) resid ? go(k_pass_pairs<16, true>) : go(k_pass_pairs<16, false>);
    else resid ? go(k_pass_pairs<32, true>) : go(k_pass_pairs<32, false>);
    rsk::prof_end(h, stream, pr);
    if (err != RSK_OK) return rsk::fail(h, err, "cudaFuncSetAttribute failed for the pair pass");
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

}  // namespace rsk

extern "C" rsk_status rsk_split_pairs(rsk_handle* h, const double* A, int64_t n, int64_t k, int64_t lda, float* P,
                                      cudaStream_t stream) {
    using namespace rsk;
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!A || !P) return fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (n < 0 || k < 0 || (k > 0 && lda < k) || n * k >= (int64_t(1) << 40))
        return fail(h, RSK_ERR_INVALID_ARG, "need n, k >= 0 and lda >= k");
    if (n == 0 || k == 0) return RSK_OK;
    k_to_pairs<double><<<unsigned((n * k + 255) / 256), 256, 0, stream>>>(A, n, int(k), lda,
                                                                         reinterpret_cast<float2*>(P));
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

extern "C" rsk_status rsk_lstsq_sketch_precond(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k,
                                               int64_t lda, const double* b, double* x, const rsk_lsq_opts* opts,
                                               rsk_lsq_info* info, cudaStream_t stream) {
    using namespace rsk;
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!A || !b || !x || !opts) return fail(h, RSK_ERR_INVALID_ARG, "null argument");
    if (a_dtype != RSK_F64 && a_dtype != RSK_F32) return fail(h, RSK_ERR_INVALID_ARG, "A must be F64 or F32");
    if (k < 1 || k > kMaxK || n < k || lda < k)
        return fail(h, RSK_ERR_INVALID_ARG, "need 1 <= k <= %d, n >= k, lda >= k", kMaxK);
    const int64_t d = opts->d;
    if (d < k || d > 8192) return fail(h, RSK_ERR_INVALID_ARG, "need k <= d <= 8192 (got d=%lld)", (long long)d);
    if (opts->sketch_dtype != RSK_F64 && opts->sketch_dtype != RSK_F32 && opts->sketch_dtype != RSK_BF16 &&
        opts->sketch_dtype != RSK_F32X2)
        return fail(h, RSK_ERR_INVALID_ARG, "bad sketch dtype");
    if (opts->inner_dtype != RSK_F64 && opts->inner_dtype != RSK_F32 && opts->inner_dtype != RSK_F32X2)
        return fail(h, RSK_ERR_INVALID_ARG, "inner dtype must be F64, F32 or F32X2");
    if (info) memset(info, 0, sizeof(*info));
    const bool dfl = opts->inner_dtype == RSK_F32X2;                        // CG over the pairs
    const bool pairs = dfl || opts->sketch_dtype == RSK_F32X2;              // A split once per solve
    const int K = int(k);
    const int nparts = std::max(1, std::min<int>(int((n + 255) / 256), 2 * h->num_sms));

    // ---- workspace
    // with F32X2 the hi array doubles as the FP32 copy the sketch may need
    const bool need_sk_copy = opts->sketch_dtype != a_dtype && opts->sketch_dtype != RSK_F32X2;
    const bool need_in_copy = opts->inner_dtype == RSK_F32 && a_dtype == RSK_F64;
    const size_t es_sk = dtype_size(opts->sketch_dtype);
    size_t bytes = 0;
    auto add = [&](size_t b_) { bytes += Carver::round(b_); };
    add(size_t(d) * (K + 1) * 8);   // W
    add(size_t(K) * 8 * 12);        // vectors
    add(size_t(K) * K * 8);         // Rinv
    add(size_t(nparts) * K * 8);    // parts
    add(size_t(nparts) * 3 * 8);    // parts_s
    add(64);                        // barrier
    add(size_t(K + 1) * 4 + 64);    // reflector-ready flags
    add(size_t(d) * K * 8);         // SA (f64 or f32)
    add(size_t(d) * 8);             // Sb
    if (need_sk_copy) add(size_t(n) * K * es_sk);
    if (need_in_copy) add(size_t(n) * K * 4);
    add(size_t(K) * 8);             // yv
    add(64);                        // CG state
    if (pairs) add(size_t(n) * K * 8);     // interleaved (hi, lo) pairs
    const size_t sk_part = std::max(sketch_partial_bytes(h, n, k, d, opts->zeta, opts->sketch_dtype),
                                    sketch_partial_bytes(h, n, 1, d, opts->zeta, RSK_F64));
    add(sk_part);
    rsk_status st = ensure_workspace(h, bytes + 4096, stream);
    if (st != RSK_OK) return st;
    Carver cv(h->ws);
    LsqWork w;
    w.W = cv.take<double>(size_t(d) * (K + 1));
    double* vecs = cv.take<double>(size_t(K) * 12);
    w.tau = vecs;
    w.x = vecs + K;
    w.g = vecs + 2 * K;
    w.c = vecs + 3 * K;
    w.z = vecs + 4 * K;
    w.res = vecs + 5 * K;
    w.p = vecs + 6 * K;
    w.s = vecs + 7 * K;
    w.t = vecs + 8 * K;
    w.stats = vecs + 9 * K;       // [0] rr, [1] ff (K >= 2 is not required: 12*K >= 12 slots)
    w.Rinv = cv.take<double>(size_t(K) * K);
    w.parts = cv.take<double>(size_t(nparts) * K);
    w.parts_s = cv.take<double>(size_t(nparts) * 3);
    w.bar = cv.take<unsigned int>(16);
    unsigned int* qr_ready = cv.take<unsigned int>(size_t(K + 1) + 16);
    w.SA64 = cv.take<double>(size_t(d) * K);
    w.SA32 = reinterpret_cast<float*>(w.SA64);
    w.Sb = cv.take<double>(size_t(d));
    void* Ask = need_sk_copy ? cv.take<char>(size_t(n) * K * es_sk) : nullptr;
    void* Ain = need_in_copy ? cv.take<char>(size_t(n) * K * 4) : nullptr;
    w.yv = cv.take<double>(size_t(K));
    double* cgstate = cv.take<double>(8);
    void* skpart = cv.take<char>(sk_part);
    float2* Ap = pairs ? cv.take<float2>(size_t(n) * K) : nullptr;
    RSK_CUDA_TRY(h, cudaMemsetAsync(w.bar, 0, 64, stream));

    // ---- L1: low-precision copies, sketch of [A | b]
    const unsigned cg = unsigned((n * k + 255) / 256);
    if (need_sk_copy) {
        if (opts->sketch_dtype == RSK_F32) {
            if (a_dtype == RSK_F64) k_convert<double, float><<<cg, 256, 0, stream>>>((const double*)A, n, K, lda, (float*)Ask);
        } else if (opts->sketch_dtype == RSK_BF16) {
            if (a_dtype == RSK_F64) k_convert<double, __nv_bfloat16><<<cg, 256, 0, stream>>>((const double*)A, n, K, lda, (__nv_bfloat16*)Ask);
            else k_convert<float, __nv_bfloat16><<<cg, 256, 0, stream>>>((const float*)A, n, K, lda, (__nv_bfloat16*)Ask);
        } else {
            k_convert<float, double><<<cg, 256, 0, stream>>>((const float*)A, n, K, lda, (double*)Ask);
        }
        RSK_LAUNCH_CHECK(h);
    }
    if (need_in_copy) {
        if (opts->sketch_dtype == RSK_F32 && need_sk_copy) Ain = Ask;
        else {
            k_convert<double, float><<<cg, 256, 0, stream>>>((const double*)A, n, K, lda, (float*)Ain);
            RSK_LAUNCH_CHECK(h);
        }
    }
    if (pairs) {
        if (a_dtype == RSK_F64) k_to_pairs<double><<<cg, 256, 0, stream>>>((const double*)A, n, K, lda, Ap);
        else k_to_pairs<float><<<cg, 256, 0, stream>>>((const float*)A, n, K, lda, Ap);
        RSK_LAUNCH_CHECK(h);
    }
    const bool sk_pairs = opts->sketch_dtype == RSK_F32X2;
    const void* A_sk = sk_pairs ? static_cast<const void*>(Ap) : (need_sk_copy ? Ask : A);
    const int64_t lda_sk = (sk_pairs || need_sk_copy) ? k : lda;
    rsk_sketch_plan* plan = nullptr;
    st = rsk_sparse_sign_plan_create(h, n, d, opts->zeta, opts->seed, &plan, stream);
    if (st != RSK_OK) return st;
    // double-float sketches keep their ~2^-44 accuracy only in an FP64 result
    const rsk_dtype sa_dt = (opts->sketch_dtype == RSK_F64 || opts->sketch_dtype == RSK_F32X2) ? RSK_F64 : RSK_F32;
    st = sketch_plan_apply_ws(h, plan, A_sk, opts->sketch_dtype, k, lda_sk, w.SA64, sa_dt, k, skpart, stream);
    if (st == RSK_OK) st = sketch_plan_apply_ws(h, plan, b, RSK_F64, 1, 1, w.Sb, RSK_F64, 1, skpart, stream);
    rsk_sparse_sign_plan_destroy(h, plan, stream);
    if (st != RSK_OK) return st;

    // ---- L2: QR of W = [SA | Sb]
    const unsigned gw = unsigned((int64_t(d) * (K + 1) + 255) / 256);
    if (sa_dt == RSK_F64) k_to_colmajor<double><<<gw, 256, 0, stream>>>(w.SA64, k, (const double*)w.Sb, int(d), K, w.W);
    else k_to_colmajor<float><<<gw, 256, 0, stream>>>(w.SA32, k, (const double*)w.Sb, int(d), K, w.W);
    RSK_LAUNCH_CHECK(h);
    // one CTA per column when k + 1 CTAs fit on the GPU at once, else the barrier sweep
    auto qr_col = [&](auto kern) -> int {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess) return -1;
        if (int64_t(per_sm) * h->num_sms < K + 1) return 0;
        RSK_CUDA_TRY(h, cudaMemsetAsync(qr_ready, 0, size_t(K + 1) * 4, stream));
        int dd = int(d);
        double* Wp = w.W;
        double* taup = w.tau;
        unsigned int* rp_ = qr_ready;
        unsigned int* stp = h->dev_status;
        uint32_t lim = h->wait_limit;
        void* args[] = {&Wp, &dd, const_cast<int*>(&K), &taup, &rp_, &stp, &lim};
        const int pr = prof_begin(h, stream, RSK_KERNEL_DENSE);
        const cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(kern), dim3(K + 1), dim3(256), args, 0, stream);
        prof_end(h, stream, pr);
        return e == cudaSuccess ? 1 : -1;
    };
    int qr_done = 0;
    if (d <= 2048) qr_done = qr_col(k_qr_col<8>);
    else if (d <= 4096) qr_done = qr_col(k_qr_col<16>);
    if (qr_done < 0) return fail(h, RSK_ERR_CUDA, "QR launch failed");
    if (!qr_done) {
        // cooperative launch: all CTAs of the persistent sweep are resident together
        // as many co-resident CTAs as the columns need: each step then waits on at most one column
        // update per CTA instead of ceil((k + 1) / num_sms)
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr, 256, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
        const int grid = std::min(h->num_sms * per_sm, K + 1);
        int dd = int(d);
        double* Wp = w.W;
        double* taup = w.tau;
        unsigned int* barp = w.bar;
        unsigned int* stp = h->dev_status;
        uint32_t lim = h->wait_limit;
        void* args[] = {&Wp, &dd, const_cast<int*>(&K), &taup, &barp, &stp, &lim};
        const int pr = prof_begin(h, stream, RSK_KERNEL_DENSE);
        RSK_CUDA_TRY(h, cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_qr), dim3(grid), dim3(256), args, 0, stream));
        prof_end(h, stream, pr);
    }
    k_rinv<<<unsigned((K * 32 + 255) / 256), 256, 0, stream>>>(w.W, int(d), K, w.Rinv);
    RSK_LAUNCH_CHECK(h);
    // ---- L3: x0 = R^{-1} (Q^T Sb)[0:k]
    const unsigned gv = unsigned((K * 32 + 255) / 256);
    k_trmv<<<gv, 256, 0, stream>>>(w.Rinv, K, 0, w.W + size_t(K) * d, w.x);
    RSK_LAUNCH_CHECK(h);

    // ---- L4: refinement
    const double tol = opts->tol_backward > 0 ? opts->tol_backward : 1e-10;
    const int max_refine = opts->max_refine >= 0 ? opts->max_refine : 20;
    const int max_inner = opts->max_inner_iters > 0 ? opts->max_inner_iters : 50;
    const double inner_tol = opts->inner_tol > 0 ? opts->inner_tol : 1e-6;
    double eta = 1.0, rnorm = 0.0, frob = 0.0, bnorm = 0.0;
    int inner_total = 0, steps = 0;
    for (steps = 0;; ++steps) {
        // g = A^T (b - A x) in FP64; rr = ||r||^2; ff = ||A||_F^2 on the first pass
        // an FP64 A is read as stored: the hi/lo split keeps only 48 bits, and the fixed point of the
        // refinement must be that of A itself.  An FP32 A is exact in hi (lo = 0): double-float sums.
        if (dfl && a_dtype == RSK_F32)
            st = launch_pass_pairs(h, Ap, n, K, w.x, b, (double*)w.parts, w.parts_s, nparts, true, steps == 0,
                                   stream);
        else if (a_dtype == RSK_F64)
            st = launch_pass<double, double>(h, (const double*)A, n, K, lda, w.x, b, (double*)w.parts, w.parts_s,
                                             nparts, true, steps == 0, stream);
        else
            st = launch_pass<float, double>(h, (const float*)A, n, K, lda, w.x, b, (double*)w.parts, w.parts_s,
                                            nparts, true, steps == 0, stream);
        if (st != RSK_OK) return st;
        k_reduce_parts<double><<<unsigned((K + 255) / 256), 256, 0, stream>>>((const double*)w.parts, nparts, K, w.g,
                                                                             w.parts_s, w.stats);
        RSK_LAUNCH_CHECK(h);
        double host[3];
        RSK_CUDA_TRY(h, cudaMemcpyAsync(host, w.stats, 24, cudaMemcpyDeviceToHost, stream));
        std::vector<double> gh(K), xh(K);
        RSK_CUDA_TRY(h, cudaMemcpyAsync(gh.data(), w.g, size_t(K) * 8, cudaMemcpyDeviceToHost, stream));
        RSK_CUDA_TRY(h, cudaMemcpyAsync(xh.data(), w.x, size_t(K) * 8, cudaMemcpyDeviceToHost, stream));
        RSK_CUDA_TRY(h, cudaStreamSynchronize(stream));
        if (steps == 0) {
            // a bounded wait of the QR that ran out leaves R undefined: stop before refining with it
            const rsk_status dev = rsk_sync_status(h, stream);
            if (dev != RSK_OK) return dev;
            frob = sqrt(host[1]);
            bnorm = sqrt(host[2]);
        }
        rnorm = sqrt(host[0]);
        double gn = 0.0, xn = 0.0;
        for (double v : gh) gn += v * v;
        for (double v : xh) xn += v * v;
        gn = sqrt(gn);
        xn = sqrt(xn);
        // min of the LSQR stopping quantities: ||A^T r|| / (||A||_F ||r||) and ||r|| / (||A||_F ||x|| + ||b||)
        eta = 0.0;
        if (rnorm > 0.0) {
            const double ls = frob > 0.0 ? gn / (frob * rnorm) : 0.0;
            const double den = frob * xn + bnorm;
            const double cons = den > 0.0 ? rnorm / den : ls;
            eta = std::min(ls, cons);
        }
        if (eta <= tol || steps >= max_refine) break;
        // c = R^{-T} g; CG on (M^T M) z = c with M = A R^{-1}
        k_trmv<<<gv, 256, 0, stream>>>(w.Rinv, K, 1, w.g, w.c);
        k_cg_init<<<1, 256, 0, stream>>>(w.c, w.z, w.res, w.p, K, cgstate);
        RSK_LAUNCH_CHECK(h);
        for (int it = 0; it < max_inner; ++it) {
            // early exit: the done flag of iteration it-2 was copied to pinned memory behind an event,
            // so the host checks it while iterations it-1 (and its pass over A) still run
            if (it >= 2) {
                RSK_CUDA_TRY(h, cudaEventSynchronize(h->flag_ev[it & 1]));
                if (h->host_flags[it & 1] != 0.0) break;
            }
            k_trmv<<<gv, 256, 0, stream>>>(w.Rinv, K, 0, w.p, w.t);   // t = R^{-1} p
            if (dfl) {
                st = launch_pass_pairs(h, Ap, n, K, w.t, nullptr, (double*)w.parts, nullptr, nparts, false, false,
                                       stream);
                if (st != RSK_OK) return st;
                k_reduce_parts<double><<<unsigned((K + 255) / 256), 256, 0, stream>>>((const double*)w.parts, nparts,
                                                                                     K, w.g, nullptr, nullptr);
            } else if (opts->inner_dtype == RSK_F32) {
                k_cast_vec<float><<<unsigned((K + 255) / 256), 256, 0, stream>>>(w.t, (float*)w.yv, K, cgstate);
                st = launch_pass<float, float>(h, (const float*)(a_dtype == RSK_F32 ? A : Ain), n, K,
                                               a_dtype == RSK_F32 ? lda : k, (const float*)w.yv, nullptr,
                                               (float*)w.parts, nullptr, nparts, false, false, stream);
                if (st != RSK_OK) return st;
                k_reduce_parts<float><<<unsigned((K + 255) / 256), 256, 0, stream>>>((const float*)w.parts, nparts, K,
                                                                                    w.g, nullptr, nullptr);
            } else {
                if (a_dtype == RSK_F64)
                    st = launch_pass<double, double>(h, (const double*)A, n, K, lda, w.t, nullptr, (double*)w.parts,
                                                     nullptr, nparts, false, false, stream);
                else
                    st = launch_pass<float, double>(h, (const float*)A, n, K, lda, w.t, nullptr, (double*)w.parts,
                                                    nullptr, nparts, false, false, stream);
                if (st != RSK_OK) return st;
                k_reduce_parts<double><<<unsigned((K + 255) / 256), 256, 0, stream>>>((const double*)w.parts, nparts,
                                                                                     K, w.g, nullptr, nullptr);
            }
            k_trmv<<<gv, 256, 0, stream>>>(w.Rinv, K, 1, w.g, w.s);  // s = R^{-T} A^T A R^{-1} p
            k_cg_step<<<1, 256, 0, stream>>>(w.s, w.z, w.res, w.p, K, cgstate, inner_tol);
            RSK_LAUNCH_CHECK(h);
            RSK_CUDA_TRY(h, cudaMemcpyAsync(&h->host_flags[it & 1], cgstate + 2, 8, cudaMemcpyDeviceToHost, stream));
            RSK_CUDA_TRY(h, cudaEventRecord(h->flag_ev[it & 1], stream));
        }
        double cgs[4];
        RSK_CUDA_TRY(h, cudaMemcpyAsync(cgs, cgstate, 32, cudaMemcpyDeviceToHost, stream));
        // x += R^{-1} z
        k_trmv<<<gv, 256, 0, stream>>>(w.Rinv, K, 0, w.z, w.t);
        k_axpy<<<unsigned((K + 255) / 256), 256, 0, stream>>>(w.x, w.t, K);
        RSK_LAUNCH_CHECK(h);
        RSK_CUDA_TRY(h, cudaStreamSynchronize(stream));
        inner_total += int(cgs[3]);
    }
    RSK_CUDA_TRY(h, cudaMemcpyAsync(x, w.x, size_t(K) * 8, cudaMemcpyDeviceToDevice, stream));
    RSK_CUDA_TRY(h, cudaStreamSynchronize(stream));
    if (info) {
        info->backward_err = eta;
        info->residual_norm = rnorm;
        info->frobenius_norm = frob;
        info->refine_steps = steps;
        info->inner_iters = inner_total;
        info->status = eta <= tol ? RSK_OK : RSK_ERR_NOT_CONVERGED;
    }
    rsk_status dev = rsk_sync_status(h, stream);
    if (dev != RSK_OK) return dev;
    if (eta > tol) return fail(h, RSK_ERR_NOT_CONVERGED, "backward error %.3e above tolerance %.1e after %d steps", eta,
                               tol, steps);
    return RSK_OK;
}
