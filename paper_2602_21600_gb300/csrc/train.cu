// Quantiser training (Section 3.1 Stages 1-2; Alg. 1).
//
// Density: rho_i = 1 / (mean of the 10 smallest squared L2 distances to
// other points + 1e-6), from the GPU brute-force kNN, for every point when
// n <= 10,000, otherwise for the given sample (the others take the sample
// mean).  The kNN distances are FP32 sums; for integer-valued data below
// 2^24 they are exact, so the parameters equal an FP64 computation's.
// The rest (delta, percentiles, scale, weights, s_dist, eta, M_i, ef_c) is
// scalar and per-column host work.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <new>
#include <system_error>
#include <thread>
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

// Type-7 percentile of column values (selection, not a full sort).
double pct7(std::vector<float>& v, double p) {
    const int64_t n = (int64_t)v.size();
    if (n == 1) return v[0];
    const double h = (double)(n - 1) * p;
    int64_t lo = (int64_t)std::floor(h);
    if (lo < 0) lo = 0;
    if (lo >= n - 1) {
        return (double)*std::max_element(v.begin(), v.end());
    }
    std::nth_element(v.begin(), v.begin() + lo, v.end());
    const double a = v[lo];
    const double b = *std::min_element(v.begin() + lo + 1, v.end());
    return a + (h - (double)lo) * (b - a);
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
        e = launch_knn(x_dev, n, d, d_q, m, kd, d_ids, d_nn, d_dd, ctx->num_sms, s);
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
    // Stage 2: adaptive percentiles, per-dimension range and scale (Alg. 1).
    const double P_l = delta * p_max, P_h = 1.0 - delta * p_max;
    std::vector<float> xh((size_t)n * d);
    e = cudaMemcpy(xh.data(), x_dev, (size_t)n * d * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy x to host");
    int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    std::atomic<bool> worker_failed{false};
    const auto columns = [&](int t) {
        try {  // no exception may leave a worker thread
            std::vector<float> col(n);
            for (int j = t; j < d; j += nth) {
                for (int64_t i = 0; i < n; ++i) col[i] = xh[(size_t)i * d + j];
                const float lo = (float)pct7(col, P_l);
                const float hi = (float)pct7(col, P_h);
                min_host[j] = lo;
                max_host[j] = hi;
                scale_host[j] = (float)(255.0 / ((double)hi - (double)lo + eps));
            }
        } catch (...) {
            worker_failed = true;
        }
    };
    try {
        for (int t = 0; t < nth; ++t) pool.emplace_back(columns, t);
    } catch (...) {
        for (auto& th : pool) th.join();
        throw;
    }
    for (auto& th : pool) th.join();
    if (worker_failed) return fail(ctx, AQR_ERR_NO_MEMORY, "aqr_train_quantizer: out of host memory");
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

// Host allocations (the base set copied to the host for the percentiles)
// become AQR_ERR_NO_MEMORY, not an exception through the C boundary.
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
    } catch (const std::system_error&) {
        return fail(ctx, AQR_ERR_INTERNAL, "aqr_train_quantizer: cannot start worker threads");
    }
}
