// Exact brute-force k nearest neighbours by FP32 squared L2, ties by id.
// Used for the density step of quantiser training (Section 3.1, Stage 1)
// and for ground truth.  Not on the query path.
//
// Pass 1: a block takes 64 queries and one contiguous split of the base
// set, computes 64 x 64 distance tiles (each thread a 4 x 4 micro-tile,
// dimensions accumulated in order j = 0..d-1 so that the sum is the same
// for every tile shape), and keeps a sorted top-k list per query in shared
// memory.  Pass 2 merges the per-split lists of each query.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "aqr_internal.h"

namespace aqr {

cudaError_t launch_knn_mma(const float* base, int64_t n, int d, const float* q, int64_t nq, int k,
                           const int64_t* self_ids, int64_t split_len, unsigned long long* part,
                           int S, unsigned int* flag_buf, cudaStream_t s);
int knn_mma_splits(int64_t nq, int d, int k, int num_sms);  // 0: no tensor pass for these sizes

namespace {

typedef unsigned long long u64;
constexpr int QB = 64, TB = 64, KC = 32;

__global__ void __launch_bounds__(256) knn_tile_kernel(const float* __restrict__ base, int64_t n,
                                                       int d, const float* __restrict__ q,
                                                       int64_t nq, int k,
                                                       const int64_t* __restrict__ self_ids,
                                                       int64_t split_len, u64* __restrict__ part,
                                                       int S, const unsigned int* skip) {
    // the tensor-core pass already produced the lists (see knn_mma.cu)
    if (skip && *(const volatile unsigned int*)skip) return;
    extern __shared__ __align__(16) unsigned char smem[];
    float* qs = (float*)smem;            // [QB][KC+1]
    float* xs = qs + QB * (KC + 1);      // [TB][KC+1]
    float* dt = xs + TB * (KC + 1);      // [QB][TB+1]
    u64* topk = (u64*)(dt + QB * (TB + 1));  // [QB][k]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ty = tid >> 4, tx = tid & 15;
    const int64_t q0 = (int64_t)blockIdx.x * QB;
    const int64_t b_begin = (int64_t)blockIdx.y * split_len;
    const int64_t b_end = (b_begin + split_len < n) ? b_begin + split_len : n;
    for (int i = tid; i < QB * k; i += 256) topk[i] = ~0ull;
    __syncthreads();

    for (int64_t t0 = b_begin; t0 < b_end; t0 += TB) {
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
        for (int k0 = 0; k0 < d; k0 += KC) {
            for (int i = tid; i < QB * KC; i += 256) {
                int r = i / KC, c = i % KC;
                int64_t qi = q0 + r;
                qs[r * (KC + 1) + c] = (qi < nq && k0 + c < d) ? q[qi * d + k0 + c] : 0.0f;
            }
            for (int i = tid; i < TB * KC; i += 256) {
                int r = i / KC, c = i % KC;
                int64_t bi = t0 + r;
                xs[r * (KC + 1) + c] = (bi < b_end && k0 + c < d) ? base[bi * d + k0 + c] : 0.0f;
            }
            __syncthreads();
            int kmax = min(KC, d - k0);
            for (int kk = 0; kk < kmax; ++kk) {
                float qv[4], xv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) qv[a] = qs[(ty * 4 + a) * (KC + 1) + kk];
#pragma unroll
                for (int b = 0; b < 4; ++b) xv[b] = xs[(tx * 4 + b) * (KC + 1) + kk];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        float t = qv[a] - xv[b];
                        acc[a][b] = fmaf(t, t, acc[a][b]);
                    }
            }
            __syncthreads();
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) dt[(ty * 4 + a) * (TB + 1) + tx * 4 + b] = acc[a][b];
        __syncthreads();
        // top-k update: warp w owns queries 8w .. 8w+7
        for (int r = warp * 8; r < warp * 8 + 8; ++r) {
            int64_t qi = q0 + r;
            if (qi >= nq) break;
            int64_t self = self_ids ? self_ids[qi] : -1;
            u64* L = topk + r * k;
            u64 cand[2];
            bool pass[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int c = lane + 32 * h;
                int64_t bi = t0 + c;
                bool ok = bi < b_end && bi != self;
                cand[h] = ok ? (((u64)__float_as_uint(dt[r * (TB + 1) + c]) << 32) | (u64)bi)
                             : ~0ull;
            }
            u64 thr = L[k - 1];
            pass[0] = cand[0] < thr;
            pass[1] = cand[1] < thr;
            for (int h = 0; h < 2; ++h) {
                uint32_t bal = __ballot_sync(0xFFFFFFFFu, pass[h]);
                while (bal) {
                    int src = __ffs(bal) - 1;
                    bal &= bal - 1;
                    u64 key = __shfl_sync(0xFFFFFFFFu, cand[h], src);
                    // insert key into the sorted list L[0..k)
                    u64 nv[4];
                    for (int t = 0; t < 4; ++t) {
                        int i = lane + 32 * t;
                        nv[t] = 0;
                        if (i < k) {
                            u64 cur = L[i];
                            u64 prev = i > 0 ? L[i - 1] : 0;
                            nv[t] = cur < key ? cur : ((i == 0 || prev < key) ? key : prev);
                        }
                    }
                    __syncwarp();
                    for (int t = 0; t < 4; ++t) {
                        int i = lane + 32 * t;
                        if (i < k) L[i] = nv[t];
                    }
                    __syncwarp();
                }
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < QB * k; i += 256) {
        int r = i / k, j = i % k;
        int64_t qi = q0 + r;
        if (qi < nq) part[(qi * S + blockIdx.y) * k + j] = topk[i];
    }
}

__global__ void knn_merge_kernel(const u64* __restrict__ part, int64_t nq, int S, int k,
                                 int64_t* __restrict__ ids, float* __restrict__ dists) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = S * k;
    int P = 1;
    while (P < per) P <<= 1;
    u64* buf = (u64*)smem + warp * P;
    int64_t qi = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (qi >= nq) return;
    for (int i = lane; i < P; i += 32) buf[i] = i < per ? part[qi * per + i] : ~0ull;
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncwarp();
            for (int t = lane; t < P / 2; t += 32) {
                int i = 2 * t - (t & (stride - 1));
                int j = i + stride;
                bool up = (i & size) == 0;
                u64 a = buf[i], b = buf[j];
                if ((a > b) == up) {
                    buf[i] = b;
                    buf[j] = a;
                }
            }
        }
    __syncwarp();
    for (int i = lane; i < k; i += 32) {
        u64 kk = buf[i];
        if (kk == ~0ull) {
            ids[qi * k + i] = -1;
            dists[qi * k + i] = __int_as_float(0x7f800000);
        } else {
            ids[qi * k + i] = (int64_t)(uint32_t)kk;
            dists[qi * k + i] = __uint_as_float((uint32_t)(kk >> 32));
        }
    }
}

}  // namespace

cudaError_t launch_knn(const float* base, int64_t n, int d, const float* q, int64_t nq, int k,
                       const int64_t* self_ids, int64_t* ids, float* dists, int num_sms,
                       cudaStream_t s, unsigned int* path_out) {
    if (nq == 0) return cudaSuccess;
    int64_t qblocks = (nq + QB - 1) / QB;
    int S = (int)std::max<int64_t>(1, (2 * (int64_t)num_sms + qblocks - 1) / qblocks);
    S = std::min(S, 8);
    // the tensor pass chooses its own split count (waves against the size
    // of a CTA's share); the lists of all splits are merged below
    const int S_mma = knn_mma_splits(nq, d, k, num_sms);
    if (S_mma > 0) S = S_mma;
    while (S > 1 && (n + S - 1) / S < TB) --S;
    int64_t split_len = (n + S - 1) / S;
    split_len = (split_len + TB - 1) / TB * TB;
    u64* part = nullptr;
    unsigned int* flags = nullptr;
    cudaError_t e = cudaMallocAsync(&part, (size_t)nq * S * k * sizeof(u64), s);
    if (e != cudaSuccess) return e;
    // tensor cores where they are exact for these sets (knn_mma.cu); the
    // CUDA-core tiles below then skip on the device
    const unsigned int* skip = nullptr;
    e = cudaMallocAsync(&flags, 8 * sizeof(unsigned int), s);
    if (e == cudaSuccess) {
        const cudaError_t em =
            launch_knn_mma(base, n, d, q, nq, k, self_ids, split_len, part, S, flags, s);
        if (em == cudaSuccess) skip = flags + 4;
        else if (em != cudaErrorNotSupported) e = em;
    }
    if (e == cudaSuccess && path_out)
        e = skip ? cudaMemcpyAsync(path_out, skip, sizeof(unsigned int), cudaMemcpyDeviceToDevice, s)
                 : cudaMemsetAsync(path_out, 0, sizeof(unsigned int), s);
    size_t smem = (size_t)(QB * (KC + 1) + TB * (KC + 1) + QB * (TB + 1)) * 4 + (size_t)QB * k * 8;
    std::unique_lock<std::mutex> g(kernel_attr_mutex());  // from each set to its launch
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(knn_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    if (e == cudaSuccess) {
        dim3 grid((unsigned)qblocks, (unsigned)S);
        knn_tile_kernel<<<grid, 256, smem, s>>>(base, n, d, q, nq, k, self_ids, split_len, part, S,
                                                skip);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        int P = 1;
        while (P < S * k) P <<= 1;
        size_t msmem = (size_t)4 * P * 8;
        e = cudaFuncSetAttribute(knn_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)msmem);
        if (e == cudaSuccess) {
            knn_merge_kernel<<<(unsigned)((nq + 3) / 4), 128, msmem, s>>>(part, nq, S, k, ids, dists);
            e = cudaGetLastError();
        }
    }
    cudaError_t e2 = cudaFreeAsync(part, s);
    if (flags) cudaFreeAsync(flags, s);
    return e != cudaSuccess ? e : e2;
}

}  // namespace aqr

// ---- brute-force kNN that allocates nothing --------------------------------
// The per-split partial top-k lists live in a file-scope device array
// instead of a cudaMallocAsync buffer.  Every GPU that loads the library
// holds this array until the process exits.

namespace aqr {
namespace {

constexpr int64_t kStaticKnnEntries = (16ll << 20) / 8;  // 16 MiB of 8-byte keys
__device__ __align__(256) unsigned long long g_knn_scratch[kStaticKnnEntries];

constexpr int kMaxDevices = 64;
std::mutex g_knn_scratch_mu;
void* g_knn_scratch_ptr[kMaxDevices] = {};
int g_knn_num_sms[kMaxDevices] = {};

// Device address of the array on the current device (set up once per device).
cudaError_t static_knn_setup(int dev, void** ptr, int* num_sms) {
    std::lock_guard<std::mutex> g(g_knn_scratch_mu);
    if (!g_knn_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_knn_scratch);
        if (e != cudaSuccess) return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_knn_scratch_ptr[dev] = p;
        g_knn_num_sms[dev] = sms;
    }
    *ptr = g_knn_scratch_ptr[dev];
    *num_sms = g_knn_num_sms[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace aqr

extern "C" aqr_status aqr_bruteforce_knn_static(const float* base_dev, int64_t n, int32_t d,
                                                const float* q_dev, int64_t nq, int32_t k,
                                                const int64_t* self_ids_dev, int64_t* ids_dev,
                                                float* dists_dev, void* stream) {
    using namespace aqr;
    if (n < 1 || d < 1 || nq < 0 || k < 1 || k > 128 || n > 0xFFFFFFFEll) return AQR_ERR_INVALID_ARG;
    if (nq * (int64_t)k > kStaticKnnEntries) return AQR_ERR_INVALID_ARG;  // beyond the scratch
    if (nq == 0) return AQR_OK;
    if (!base_dev || !q_dev || !ids_dev || !dists_dev) return AQR_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AQR_ERR_CUDA;
    void* scratch = nullptr;
    int num_sms = 0;
    if (static_knn_setup(dev, &scratch, &num_sms) != cudaSuccess) return AQR_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // as many base-set splits as the scratch holds, up to the usual count
    const int64_t qblocks = (nq + QB - 1) / QB;
    int S = (int)std::max<int64_t>(1, (2 * (int64_t)num_sms + qblocks - 1) / qblocks);
    S = std::min(S, 8);
    while (S > 1 && ((n + S - 1) / S < TB || nq * (int64_t)S * k > kStaticKnnEntries)) --S;
    int64_t split_len = (n + S - 1) / S;
    split_len = (split_len + TB - 1) / TB * TB;
    u64* part = (u64*)scratch;
    const size_t smem = (size_t)(QB * (KC + 1) + TB * (KC + 1) + QB * (TB + 1)) * 4 + (size_t)QB * k * 8;
    std::lock_guard<std::mutex> g(kernel_attr_mutex());  // from each set to its launch
    cudaError_t e = cudaFuncSetAttribute(knn_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        dim3 grid((unsigned)qblocks, (unsigned)S);
        knn_tile_kernel<<<grid, 256, smem, s>>>(base_dev, n, d, q_dev, nq, k, self_ids_dev, split_len, part, S,
                                                nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        int P = 1;
        while (P < S * k) P <<= 1;
        const size_t msmem = (size_t)4 * P * 8;
        e = cudaFuncSetAttribute(knn_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem);
        if (e == cudaSuccess) {
            knn_merge_kernel<<<(unsigned)((nq + 3) / 4), 128, msmem, s>>>(part, nq, S, k, ids_dev, dists_dev);
            e = cudaGetLastError();
        }
    }
    return e == cudaSuccess ? AQR_OK : AQR_ERR_CUDA;
}
