// Quantiser training (Section 3.1 Stages 1-2; Alg. 1).
//
// Density: rho_i = 1 / (mean of the 10 smallest squared L2 distances to
// other points + 1e-6), from the GPU brute-force kNN, for every point when
// n <= 10,000, otherwise for the given sample (the others take the sample
// mean).  The kNN distances are FP32 sums; for integer-valued data below
// 2^24 they are exact, so the parameters equal an FP64 computation's.
// Per-column percentiles: exact order statistics by a radix select on the
// device (no copy of the base set to the host); the rest (delta, the
// type-7 interpolation, scale, weights, s_dist, eta, M_i, ef_c) is scalar
// host work on those few values.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "aqr_internal.h"

namespace aqr {
namespace {

__global__ void gather_rows(const float* __restrict__ x, int d, const int64_t* __restrict__ ids,
                            int64_t m, float* __restrict__ out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m * d;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = t / d;
        int c = (int)(t - r * d);
        out[t] = x[ids[r] * d + c];
    }
}

// ---- per-column order statistics by radix select --------------------------
// FP32 values map to uint32 keys that order like the values (positive:
// sign bit set; negative: all bits inverted), so the r-th smallest value of
// a column is the r-th smallest key.  Four passes pick the key's bytes from
// the top: each pass histograms the next byte of the keys whose higher
// bytes equal the prefix found so far, and the running rank selects the
// bucket.  kT order statistics per column are selected together.
constexpr int kT = 4;          // ranks per column: lo and lo + 1 of P_l and of P_h
constexpr int kSelCols = 16;   // columns per block of the histogram kernel

__device__ __forceinline__ uint32_t order_key(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Histogram of byte (key >> shift) & 255 over the keys of column c whose
// bits above shift + 8 equal prefix[c][t], for each target t.  Block:
// kSelCols columns x (blockDim.x / kSelCols) rows per step; rows split over
// gridDim.y.  Shared histograms [kSelCols][kT][256], added to hist.
__global__ void radix_hist_kernel(const float* __restrict__ x, int64_t n, int d,
                                  const uint32_t* __restrict__ prefix, int shift,
                                  unsigned int* __restrict__ hist) {
    extern __shared__ unsigned int sh[];
    const int nbins = kSelCols * kT * 256;
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int cl = threadIdx.x % kSelCols;
    const int c = blockIdx.x * kSelCols + cl;
    const int rstep = blockDim.x / kSelCols;
    const uint32_t hmask = shift >= 24 ? 0u : (0xFFFFFFFFu << (shift + 8));
    uint32_t pre[kT];
#pragma unroll
    for (int t = 0; t < kT; ++t) pre[t] = c < d ? prefix[c * kT + t] & hmask : 0u;
    const int64_t per = (n + gridDim.y - 1) / gridDim.y;
    const int64_t r0 = (int64_t)blockIdx.y * per, r1 = min(n, r0 + per);
    if (c < d)
        for (int64_t r = r0 + threadIdx.x / kSelCols; r < r1; r += rstep) {
            const uint32_t k = order_key(__ldg(x + r * d + c));
            const uint32_t b = (k >> shift) & 255u;
#pragma unroll
            for (int t = 0; t < kT; ++t)
                if ((k & hmask) == pre[t]) atomicAdd(&sh[(cl * kT + t) * 256 + b], 1u);
        }
    __syncthreads();
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
        const int cc = blockIdx.x * kSelCols + i / (kT * 256);
        if (cc < d && sh[i]) atomicAdd(&hist[(int64_t)blockIdx.x * nbins + i], sh[i]);
    }
}

// One thread per (column, target): the bucket that holds the remaining rank
// gives the next byte of the key; the rank becomes the rank inside it.
__global__ void radix_pick_kernel(int d, int shift, const unsigned int* __restrict__ hist,
                                  uint32_t* __restrict__ prefix, uint32_t* __restrict__ rank) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d * kT) return;
    const unsigned int* h = hist + (int64_t)i * 256;
    uint32_t r = rank[i];
    int b = 0;
    for (; b < 255; ++b) {
        if (r < h[b]) break;
        r -= h[b];
    }
    prefix[i] = (prefix[i] & (shift >= 24 ? 0u : (0xFFFFFFFFu << (shift + 8)))) |
                ((uint32_t)b << shift);
    rank[i] = r;
}

// Rank of the lower order statistic of the type-7 percentile p and its
// weight: h = (n - 1) p, lo = floor(h) (the largest when lo >= n - 1).
void pct7_rank(int64_t n, double p, int64_t* lo, double* frac) {
    const double h = (double)(n - 1) * p;
    int64_t l = (int64_t)std::floor(h);
    if (l < 0) l = 0;
    if (l >= n - 1) {
        *lo = n - 1;
        *frac = 0.0;
        return;
    }
    *lo = l;
    *frac = h - (double)l;
}

// The ranks rk[c * kT + t] of every column of x [n, d] (device, row-major)
// as FP32 values (host out[c * kT + t]); exact order statistics.
cudaError_t column_order_stats(const float* x, int64_t n, int d, const uint32_t* rk_host,
                               float* out_host, int num_sms, cudaStream_t s) {
    const int cblocks = (d + kSelCols - 1) / kSelCols;
    const int nbins = kSelCols * kT * 256;
    const size_t smem = (size_t)nbins * 4;  // 64 KB
    const int rows_blocks = std::max(1, (int)std::min<int64_t>((2 * num_sms + cblocks - 1) / cblocks,
                                                                (n + 1023) / 1024));
    uint32_t* d_prefix = nullptr;
    uint32_t* d_rank = nullptr;
    unsigned int* d_hist = nullptr;
    const size_t nt = (size_t)d * kT;
    cudaError_t e = cudaMalloc(&d_prefix, nt * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_rank, nt * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_hist, (size_t)cblocks * nbins * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_prefix, 0, nt * 4, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_rank, rk_host, nt * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(radix_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    for (int shift = 24; shift >= 0 && e == cudaSuccess; shift -= 8) {
        e = cudaMemsetAsync(d_hist, 0, (size_t)cblocks * nbins * 4, s);
        if (e != cudaSuccess) break;
        radix_hist_kernel<<<dim3(cblocks, rows_blocks), 512, smem, s>>>(x, n, d, d_prefix, shift,
                                                                         d_hist);
        radix_pick_kernel<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(d, shift, d_hist, d_prefix,
                                                                       d_rank);
        e = cudaGetLastError();
    }
    std::vector<uint32_t> keys(nt);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(keys.data(), d_prefix, nt * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_prefix);
    cudaFree(d_rank);
    cudaFree(d_hist);
    if (e != cudaSuccess) return e;
    for (size_t i = 0; i < nt; ++i) {
        const uint32_t k = keys[i];
        const uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
        std::memcpy(&out_host[i], &u, 4);
    }
    return cudaSuccess;
}

}  // namespace
}  // namespace aqr

using namespace aqr;

static aqr_status train_impl(aqr_ctx* ctx, const float* x_dev, int64_t n, int32_t d,
                             const int64_t* sample_host, int64_t n_s, double p_max, int32_t M0,
                             int32_t ef0, float* min_host, float* max_host, float* scale_host,
                             double* scalars_host) {
    NvtxRange range("aqr.train_quantizer");
    if (!ctx) return AQR_ERR_INVALID_ARG;
    if (!x_dev || n < 11 || d < 1 || d > 4096 || !min_host || !max_host || !scale_host ||
        !scalars_host || !(p_max >= 0.0 && p_max <= 0.5) || M0 < 2 || ef0 < 1)
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_train_quantizer: bad arguments");
    const bool sampled = n > 10000;
    if (sampled && (!sample_host || n_s < 1 || n_s > n))
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_train_quantizer: n > 10000 needs a sample");
    cudaSetDevice(ctx->device);
    const double eps = 1e-6;
    const int kd = 10;
    std::vector<int64_t> ids;
    if (sampled) {
        ids.assign(sample_host, sample_host + n_s);
        for (int64_t v : ids)
            if (v < 0 || v >= n) return fail(ctx, AQR_ERR_INVALID_ARG, "sample id out of range");
    } else {
        ids.resize(n);
        for (int64_t i = 0; i < n; ++i) ids[i] = i;
    }
    const int64_t m = (int64_t)ids.size();
    cudaStream_t s = ctx->own_stream;
    int64_t* d_ids = nullptr;
    float* d_q = nullptr;
    int64_t* d_nn = nullptr;
    float* d_dd = nullptr;
    std::vector<float> dd((size_t)m * kd);
    cudaError_t e = cudaMalloc(&d_ids, m * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_q, (size_t)m * d * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_nn, (size_t)m * kd * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_dd, (size_t)m * kd * 4);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ids, ids.data(), m * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        gather_rows<<<1024, 256, 0, s>>>(x_dev, d, d_ids, m, d_q);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = launch_knn(x_dev, n, d, d_q, m, kd, d_ids, d_nn, d_dd, ctx->num_sms, s,
                       ctx->d_knn_tensor);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dd.data(), d_dd, (size_t)m * kd * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_ids);
    cudaFree(d_q);
    cudaFree(d_nn);
    cudaFree(d_dd);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "density kNN");

    // Stage 1: densities and heterogeneity (Alg. 1).
    std::vector<double> rho(m);
    for (int64_t i = 0; i < m; ++i) {
        double sum = 0.0;
        for (int t = 0; t < kd; ++t) sum += (double)dd[i * kd + t];  // ascending
        rho[i] = 1.0 / (sum / (double)kd + eps);
    }
    double rmax = rho[0], rmin = rho[0], rsum = 0.0;
    for (double r : rho) {
        rmax = std::max(rmax, r);
        rmin = std::min(rmin, r);
        rsum += r;
    }
    const double rho_bar = rsum / (double)m;
    const double delta = (rmax - rmin) / (rmax + eps);
    // Stage 2: adaptive percentiles, per-dimension range and scale (Alg. 1):
    // type-7 percentiles a + (h - lo)(b - a) of the exact order statistics
    // a, b (ranks lo, lo + 1) selected on the device.
    const double P_l = delta * p_max, P_h = 1.0 - delta * p_max;
    int64_t lo_l, lo_h;
    double f_l, f_h;
    pct7_rank(n, P_l, &lo_l, &f_l);
    pct7_rank(n, P_h, &lo_h, &f_h);
    std::vector<uint32_t> rk((size_t)d * kT);
    for (int j = 0; j < d; ++j) {
        rk[j * kT + 0] = (uint32_t)lo_l;
        rk[j * kT + 1] = (uint32_t)std::min<int64_t>(lo_l + 1, n - 1);
        rk[j * kT + 2] = (uint32_t)lo_h;
        rk[j * kT + 3] = (uint32_t)std::min<int64_t>(lo_h + 1, n - 1);
    }
    std::vector<float> os((size_t)d * kT);
    e = column_order_stats(x_dev, n, d, rk.data(), os.data(), ctx->num_sms, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "percentile selection");
    for (int j = 0; j < d; ++j) {
        const double a_l = os[j * kT], b_l = os[j * kT + 1];
        const double a_h = os[j * kT + 2], b_h = os[j * kT + 3];
        const float lo = (float)(a_l + f_l * (b_l - a_l));
        const float hi = (float)(a_h + f_h * (b_h - a_h));
        min_host[j] = lo;
        max_host[j] = hi;
        scale_host[j] = (float)(255.0 / ((double)hi - (double)lo + eps));
    }
    // Density weights w_j = (1/n) sum_i rho_i (Alg. 1): the same for
    // every j; Eq. 1; eta from the shifted two-pass mean and deviation.
    const double w = (rsum + (double)(n - m) * rho_bar) / (double)n;
    std::vector<double> wj(d, w);
    double num = 0.0, den = 0.0;
    for (int j = 0; j < d; ++j) {
        double r = (double)max_host[j] - (double)min_host[j];
        num += r * r * wj[j];
        den += 255.0 * 255.0 * wj[j];
    }
    const double s_dist = std::sqrt(num / den);
    double shift = 0.0;
    for (int j = 0; j < d; ++j) shift += wj[j] - wj[0];
    const double wbar = wj[0] + shift / (double)d;
    double var = 0.0;
    for (int j = 0; j < d; ++j) var += (wj[j] - wbar) * (wj[j] - wbar);
    const double eta = std::sqrt(var / (double)d) / wbar;
    // Alg. 1.
    const int M_i = (int)std::floor((double)M0 * (1.0 + delta * (1.0 + eta)));
    const int ef_c = (int)std::floor((double)ef0 * (1.0 / (1.0 + delta * eta)));
    double* o = scalars_host;
    o[0] = delta;
    o[1] = rho_bar;
    o[2] = w;
    o[3] = s_dist;
    o[4] = eta;
    o[5] = M_i;
    o[6] = ef_c;
    o[7] = P_l;
    o[8] = P_h;
    o[9] = rmin;
    o[10] = rmax;
    return AQR_OK;
}

// Host allocations become AQR_ERR_NO_MEMORY, not an exception through the
// C boundary.
extern "C" aqr_status aqr_train_quantizer(aqr_ctx* ctx, const float* x_dev, int64_t n, int32_t d,
                                          const int64_t* sample_host, int64_t n_s, double p_max,
                                          int32_t M0, int32_t ef0, float* min_host,
                                          float* max_host, float* scale_host,
                                          double* scalars_host) {
    try {
        return train_impl(ctx, x_dev, n, d, sample_host, n_s, p_max, M0, ef0, min_host, max_host,
                          scale_host, scalars_host);
    } catch (const std::bad_alloc&) {
        return fail(ctx, AQR_ERR_NO_MEMORY, "aqr_train_quantizer: out of host memory");
    }
}
