// Brute-force kNN on the tensor cores (tcgen05, sm_103a) for data whose
// squared distances the tensor path computes exactly: the density step of
// quantiser training (Section 3.1, Stage 1) and ground truth.  Not on the
// query path.
//
// d(q, x) = |q|^2 + |x|^2 - 2 q.x.  The dot products of a 128-query x
// 128-base-row tile come from tcgen05.mma (kind::f16, BF16 operands, FP32
// accumulators in tensor memory); the norms are FP32 sums.  Exactness: when
// every value is an integer with |v| <= 256 it is exact in BF16, products
// are exact, and when max |q|^2 + max |x|^2 < 2^24 every partial sum, norm
// and distance is an integer below 2^24, so the distance equals the FP32
// CUDA-core kernel's (also exact there) bit for bit, whatever the order of
// accumulation.  A conversion pass checks that on the device and writes a
// flag; the tensor kernel runs only when it is set and the CUDA-core
// kernel only when it is not, both launched on the stream (no host sync).
//
// Tile pipeline per CTA (128 threads, one query tile, one split of the base
// set): the query tile stays in shared memory; base tiles are copied with
// cp.async into two buffers in the canonical no-swizzle K-major layout
// (8-row x 16-byte core matrices, K-adjacent core matrices 128 bytes apart,
// 8-row groups Kp * 16 bytes apart); thread 0 issues Kp / 16 MMAs into the
// tile's accumulator and commits them to an mbarrier; after the wait every
// thread reads its own query row (its tensor-memory lane) with tcgen05.ld
// and updates that query's top-k list.  Waits are bounded: a timeout sets
// the error word, and tensor memory is freed on every path.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "aqr_internal.h"

namespace aqr {
namespace {

typedef unsigned long long u64;
constexpr int TM = 128;          // queries per tile (MMA M)
constexpr int TN = 128;          // base rows per tile (MMA N)
constexpr int kMmaMaxKp = 256;   // padded dimensions handled (shared-memory bound)
constexpr int kMmaMaxK = 32;     // neighbours per query handled
constexpr long long kSpinLimit = 1ll << 24;  // about a second of polling

// ---- conversion and the exactness test --------------------------------------
// rows [m, d] FP32 -> [m, Kp] BF16 (zero padded), norms |v|^2 in FP32, and
// flags[0] |= 1 for a value that is not an integer of magnitude <= 256;
// flags[1] = max norm bits (non-negative floats order like their bit
// patterns).  One warp per row.
__global__ void bf16_rows_kernel(const float* __restrict__ x, int64_t m, int d, int Kp,
                                 uint16_t* __restrict__ xb, float* __restrict__ norms,
                                 unsigned int* __restrict__ flags) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < m;
         r += warps) {
        const float* row = x + r * d;
        float part = 0.0f;
        bool bad = false;
        for (int j = lane; j < Kp; j += 32) {
            const float v = j < d ? row[j] : 0.0f;
            bad |= !(v == rintf(v) && fabsf(v) <= 256.0f);
            // integers of magnitude <= 256 are exact in BF16: truncation is exact
            xb[r * Kp + j] = (uint16_t)(__float_as_uint(v) >> 16);
            part = fmaf(v, v, part);
        }
        // exact whenever it matters (integer values, sums below 2^24)
#pragma unroll
        for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
        if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(flags, 1u);
        if (lane == 0) {
            norms[r] = part;
            atomicMax(flags + 1, __float_as_uint(part));
        }
    }
}

// flags[2] = 1 when the tensor path is exact for these query and base sets:
// no inexact value in either and max |q|^2 + max |x|^2 < 2^24.
__global__ void mma_exact_kernel(const unsigned int* fq, const unsigned int* fx,
                                 unsigned int* out) {
    const double s = (double)__uint_as_float(fq[1]) + (double)__uint_as_float(fx[1]);
    *out = (fq[0] == 0u && fx[0] == 0u && s < 16777216.0) ? 1u : 0u;
}

// ---- tcgen05 / mbarrier helpers (inline PTX) --------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// Shared-memory matrix descriptor, no swizzle: start address, leading byte
// offset (K-adjacent core matrices), stride byte offset (8-row groups), all
// in 16-byte units; bits 46-47 = 1 (descriptor version of sm_100 and later).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at
// bits 17-22, M / 16 at bits 24-28.
__host__ __device__ constexpr uint32_t mma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
        : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
}
// Bounded wait for the phase with parity `parity`; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < kSpinLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tmem_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
// 32 consecutive FP32 columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

// Copy rows [r0, r0 + 128) of a BF16 [rows, Kp] array (rows past `last`
// repeat row `last`; their results are masked) into the core-matrix layout:
// element (r, k) at ((r / 8) * (Kp / 8) + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
__device__ __forceinline__ void load_tile(uint32_t dst, const uint16_t* src, int64_t r0,
                                          int64_t last, int Kp) {
    const int kc = Kp >> 3;  // 16-byte chunks per row
    for (int i = threadIdx.x; i < TN * kc; i += blockDim.x) {
        const int r = i / kc, c = i - r * kc;
        const int64_t row = min(r0 + r, last);
        cp16(dst + (uint32_t)(((r >> 3) * kc + c) * 128 + (r & 7) * 16), src + row * Kp + c * 8);
    }
}

// One CTA of 16 warps: queries [q0, q0 + 128) against base rows of split
// blockIdx.y.  Warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its
// query rows) and accumulator columns 32 (w / 4) .. + 31 (a quarter of each
// base tile), so every thread scans 32 distances per tile and keeps its own
// top k; the four lists of a query are merged at the end into the per-query
// top k (sorted keys (distance bits << 32) | id), written to part as the
// CUDA-core kernel does.  Two base-tile buffers and two accumulators (256
// tensor-memory columns): while the epilogue of tile t reads accumulator
// t % 2, the MMAs of tile t + 1 fill the other one and the copy of tile
// t + 2 refills the buffer tile t used.  Shared memory: query tile, two
// base tiles, their base norms, the lists [4][k][128], two mbarriers and
// the tensor-memory address.
constexpr int kMmaThreads = 512;
__global__ void __launch_bounds__(kMmaThreads, 1)
    knn_mma_kernel(const uint16_t* __restrict__ xb, const float* __restrict__ xn, int64_t n,
                   const uint16_t* __restrict__ qb, const float* __restrict__ qn, int64_t nq,
                   int Kp, int k, const int64_t* __restrict__ self_ids, int64_t split_len,
                   u64* __restrict__ part, int S, unsigned int* exact, int* err) {
    if (*(volatile unsigned int*)exact == 0u) return;  // the CUDA-core kernel handles these sets
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (TM - 1);  // query row in the tile = tensor-memory lane
    const int cq = warp >> 2;        // column quarter of the tile
    const int tile_bytes = TN * Kp * 2;
    unsigned char* sA = smem;
    unsigned char* const sB0 = smem + tile_bytes;
    unsigned char* const sB1 = smem + 2 * tile_bytes;
    float* s_xn = (float*)(smem + 3 * tile_bytes);  // [2][TN]
    u64* L = (u64*)(s_xn + 2 * TN);                 // [4][k][TM]
    u64* mbar = L + (size_t)4 * k * TM;             // [2]
    uint32_t* s_tmem = (uint32_t*)(mbar + 2);
    const uint32_t mb0 = smem_u32(mbar), mb1 = smem_u32(mbar + 1);
    u64* myL = L + (size_t)cq * k * TM + row;       // element j at myL[j * TM]

    const int64_t q0 = (int64_t)blockIdx.x * TM;
    const int64_t b_begin = (int64_t)blockIdx.y * split_len;
    const int64_t b_end = min(n, b_begin + split_len);
    const int64_t nt = b_end > b_begin ? (b_end - b_begin + TN - 1) / TN : 0;  // tiles
    const int64_t qi = q0 + row;
    const bool qvalid = qi < nq;
    const float my_qn = qvalid ? qn[qi] : 0.0f;
    const int64_t self = (qvalid && self_ids) ? self_ids[qi] : -1;
    for (int j = 0; j < k; ++j) myL[j * TM] = ~0ull;
    const float kInf = __int_as_float(0x7f800000);
    float thr = kInf;  // distance of this list's k-th entry (+inf until k are held)

    if (tid == 0) {
        mbar_init(mb0, 1);
        mbar_init(mb1, 1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(
                         smem_u32(s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem = *s_tmem;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t idesc = mma_idesc_bf16(TM, TN);
    const uint32_t lbo = 128, sbo = (uint32_t)Kp * 16;  // core-matrix offsets (bytes)
    const auto issue = [&](int64_t t) {  // thread 0: the MMAs of tile t
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32((t & 1) ? sB1 : sB0);
        const uint32_t d = tmem + (uint32_t)((t & 1) * TN);
        for (int ks = 0; ks < Kp / 16; ++ks)  // K = 16 per MMA: two core matrices
            mma_bf16(d, smem_desc(a0 + ks * 256, lbo, sbo), smem_desc(b0 + ks * 256, lbo, sbo),
                     idesc, ks > 0 ? 1u : 0u);
        mma_commit((t & 1) ? mb1 : mb0);
    };
    const auto fetch = [&](int64_t t) {  // all threads: base tile t and its norms
        const int64_t r0 = b_begin + t * TN;
        load_tile(smem_u32((t & 1) ? sB1 : sB0), xb, r0, b_end - 1, Kp);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        if (tid < TN) s_xn[(t & 1) * TN + tid] = xn[min(r0 + tid, b_end - 1)];
    };

    load_tile(smem_u32(sA), qb, q0, nq - 1, Kp);
    if (nt > 0) fetch(0);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (nt > 1) fetch(1);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // visible to the MMA
    __syncthreads();
    if (tid == 0 && nt > 0) issue(0);
    uint32_t ph0 = 0u, ph1 = 0u;  // next phase parity of each mbarrier
    bool ok = true;
    for (int64_t t = 0; t < nt; ++t) {
        // tile t + 1 in shared memory, the epilogue of t - 1 done: start its MMAs
        if (t + 1 < nt) {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        }
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (tid == 0 && t + 1 < nt) issue(t + 1);
        // tile t's MMAs complete: its buffer is free for tile t + 2
        const bool waited = (t & 1) ? mbar_wait(mb1, ph1) : mbar_wait(mb0, ph0);
        if (__syncthreads_or(!waited)) {  // the same decision in every thread
            ok = false;
            break;
        }
        if (t & 1) ph1 ^= 1u;
        else ph0 ^= 1u;
        tmem_fence_after();
        const int64_t t0 = b_begin + t * TN;
        const int c0 = cq * 32;
        const int lim = (int)min((int64_t)TN, b_end - t0);
        const int self_c = (self >= t0 && self < t0 + TN) ? (int)(self - t0) : -1;
        const float* xn_t = s_xn + (t & 1) * TN + c0;
        float acc[32];
        tmem_ld32(tmem + lane_base + (uint32_t)((t & 1) * TN + c0), acc);
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const float dist = (my_qn + xn_t[c]) - 2.0f * acc[c];
            // ids rise within the split: an equal distance never displaces a
            // held entry, so < is the exact (distance, id) test
            if (dist < thr && c0 + c < lim && c0 + c != self_c) {
                const u64 key =
                    ((u64)__float_as_uint(fmaxf(dist, 0.0f)) << 32) | (u64)(t0 + c0 + c);
                int j = k - 1;
                while (j > 0 && myL[(j - 1) * TM] > key) {
                    myL[j * TM] = myL[(j - 1) * TM];
                    --j;
                }
                myL[j * TM] = key;
                const u64 kth = myL[(k - 1) * TM];
                thr = kth == ~0ull ? kInf : __uint_as_float((uint32_t)(kth >> 32));
            }
        }
        // this tile's buffer and norm slot take tile t + 2 (after every thread read them)
        if (t + 2 < nt) {
            __syncthreads();
            fetch(t + 2);
        }
    }
    if (!ok && tid == 0) {  // the CUDA-core kernel that follows recomputes every list
        atomicExch(exact, 0u);
        if (err) atomicAdd(err, 1);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem)
                     : "memory");
    // the k smallest of the query's four sorted lists
    if (cq == 0 && qvalid) {
        int h0 = 0, h1 = 0, h2 = 0, h3 = 0;
        const u64* l0 = L + row;
        const u64* l1 = l0 + (size_t)k * TM;
        const u64* l2 = l1 + (size_t)k * TM;
        const u64* l3 = l2 + (size_t)k * TM;
        for (int j = 0; j < k; ++j) {
            const u64 a = h0 < k ? l0[h0 * TM] : ~0ull, b = h1 < k ? l1[h1 * TM] : ~0ull;
            const u64 c = h2 < k ? l2[h2 * TM] : ~0ull, d = h3 < k ? l3[h3 * TM] : ~0ull;
            const u64 ab = a < b ? a : b, cd = c < d ? c : d;
            const u64 m = ab < cd ? ab : cd;
            if (m == a) ++h0;
            else if (m == b) ++h1;
            else if (m == c) ++h2;
            else ++h3;
            part[(qi * S + blockIdx.y) * k + j] = m;
        }
    }
}

}  // namespace
}  // namespace aqr

namespace aqr {

// Shared memory of knn_mma_kernel: at most two CTAs per SM (their 2 x 256
// tensor-memory columns fill the SM's 512, so no allocation ever waits).
size_t knn_mma_smem(int Kp, int k) {
    return std::max<size_t>((size_t)3 * TN * Kp * 2 + 2 * TN * 4 + (size_t)4 * k * TM * 8 + 32,
                            80 * 1024);
}

// Splits of the base set for nq queries: 128-query tiles, CTAs per SM from
// the shared memory; the count in 1..16 that minimises (waves / splits),
// i.e. the time of a CTA's share times the number of waves.
int knn_mma_splits(int64_t nq, int d, int k, int num_sms) {
    const int Kp = (d + 15) / 16 * 16;
    if (Kp > kMmaMaxKp || k > kMmaMaxK) return 0;
    const size_t smem = knn_mma_smem(Kp, k);
    if (smem > 227 * 1024) return 0;
    const int per_sm = std::max(1, std::min(2, (int)(233472 / (smem + 1024))));
    const int64_t slots = (int64_t)per_sm * num_sms, qt = (nq + TM - 1) / TM;
    int best = 1;
    double best_cost = 1e30;
    for (int S = 1; S <= 16; ++S) {
        const double cost = (double)((qt * S + slots - 1) / slots) / S;
        if (cost < best_cost - 1e-12) {
            best_cost = cost;
            best = S;
        }
    }
    return best;
}

// Tensor-core pass of launch_knn: converts both sets, tests exactness and,
// when exact, fills part [nq, S, k] for the split layout of the CUDA-core
// kernel.  *flag receives a device word that is 1 when the tensor pass
// produced the lists (the CUDA-core kernel then skips), 0 otherwise.  The
// temporaries are stream-ordered and freed on the stream; flag_buf [8] is
// the caller's device scratch.  Returns cudaErrorNotSupported (nothing
// launched) for shapes the kernel does not handle.
cudaError_t launch_knn_mma(const float* base, int64_t n, int d, const float* q, int64_t nq, int k,
                           const int64_t* self_ids, int64_t split_len, unsigned long long* part,
                           int S, unsigned int* flag_buf, cudaStream_t s) {
    const int Kp = (d + 15) / 16 * 16;
    if (Kp > kMmaMaxKp || k > kMmaMaxK || nq < 1 || n < 1) return cudaErrorNotSupported;
    const size_t smem = knn_mma_smem(Kp, k);
    if (smem > 227 * 1024) return cudaErrorNotSupported;
    uint16_t *qb = nullptr, *xb = nullptr;
    float *qn = nullptr, *xn = nullptr;
    cudaError_t e = cudaMallocAsync(&qb, (size_t)nq * Kp * 2, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&xb, (size_t)n * Kp * 2, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&qn, (size_t)nq * 4, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&xn, (size_t)n * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag_buf, 0, 8 * sizeof(unsigned int), s);
    if (e == cudaSuccess) {
        bf16_rows_kernel<<<1024, 256, 0, s>>>(q, nq, d, Kp, qb, qn, flag_buf);
        bf16_rows_kernel<<<2048, 256, 0, s>>>(base, n, d, Kp, xb, xn, flag_buf + 2);
        mma_exact_kernel<<<1, 1, 0, s>>>(flag_buf, flag_buf + 2, flag_buf + 4);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> g(kernel_attr_mutex());  // from the set to the launch
        e = cudaFuncSetAttribute(knn_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess) {
            dim3 grid((unsigned)((nq + TM - 1) / TM), (unsigned)S);
            knn_mma_kernel<<<grid, kMmaThreads, smem, s>>>(xb, xn, n, qb, qn, nq, Kp, k, self_ids,
                                                  split_len, part, S, flag_buf + 4,
                                                  (int*)(flag_buf + 5));
            e = cudaGetLastError();
        }
    }
    cudaFreeAsync(qb, s);
    cudaFreeAsync(xb, s);
    cudaFreeAsync(qn, s);
    cudaFreeAsync(xn, s);
    return e;
}

}  // namespace aqr
