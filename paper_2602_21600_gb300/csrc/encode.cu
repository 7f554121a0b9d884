// Vector encode (Alg. 1, Alg. 2, Section 3.3): shift by
// min_j, scale by scale_j, clip to [0, 255], round to nearest even.
// One thread per 16-byte output chunk; rows of the output are zero-padded
// to the code row stride so that distances over the padded row equal
// distances over the d real dimensions.
#include <cuda_runtime.h>
#include <stdint.h>

#include "aqr_internal.h"

namespace aqr {
namespace {

__global__ void encode_kernel(const float* __restrict__ x, int64_t n, int d, int64_t ldx,
                              const float* __restrict__ mn, const float* __restrict__ sc,
                              uint8_t* __restrict__ codes, int64_t ldc) {
    const int64_t chunks_per_row = (ldc + 15) / 16;
    const int64_t total = n * chunks_per_row;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = t / chunks_per_row;
        int c = (int)(t - r * chunks_per_row);
        const float* xr = x + r * ldx;
        uint8_t out[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            int j = c * 16 + u;
            uint32_t code = 0;
            if (j < d) {
                float v = __fmul_rn(__fsub_rn(xr[j], mn[j]), sc[j]);
                v = fminf(fmaxf(v, 0.0f), 255.0f);  // fmaxf(NaN, 0) = 0
                code = (uint32_t)__float2int_rn(v);
            }
            out[u] = (uint8_t)code;
        }
        uint8_t* dst = codes + r * ldc + (int64_t)c * 16;
        int64_t lim = ldc - (int64_t)c * 16;
        if (lim >= 16 && ((uintptr_t)dst & 15) == 0) {
            uint4 w;
            w.x = out[0] | (out[1] << 8) | (out[2] << 16) | ((uint32_t)out[3] << 24);
            w.y = out[4] | (out[5] << 8) | (out[6] << 16) | ((uint32_t)out[7] << 24);
            w.z = out[8] | (out[9] << 8) | (out[10] << 16) | ((uint32_t)out[11] << 24);
            w.w = out[12] | (out[13] << 8) | (out[14] << 16) | ((uint32_t)out[15] << 24);
            *(uint4*)dst = w;
        } else {
            for (int u = 0; u < 16 && u < lim; ++u) dst[u] = out[u];
        }
    }
}

}  // namespace

cudaError_t launch_encode(const float* x, int64_t n, int d, int64_t ldx, const float* mn,
                          const float* sc, uint8_t* codes, int64_t ldc, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int64_t total = n * ((ldc + 15) / 16);
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    encode_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, n, d, ldx, mn, sc, codes, ldc);
    return cudaGetLastError();
}

}  // namespace aqr
