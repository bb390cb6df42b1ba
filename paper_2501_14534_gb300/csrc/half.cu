// FP16 storage of trained Gaussians: the paper stores every Gaussian parameter as a 16-bit
// half after training (Sec. "Experiments", setup) and renders from it. The conversion rounds
// each float32 to the nearest IEEE half (ties to even; beyond the half range to +-inf); the
// render path widens the halves back to float32 as it loads them (preprocess.cu).
#include <cuda_fp16.h>

#include "tgs_internal.cuh"

namespace tgs {
namespace {

// Four values per thread where the pointers allow 16- and 8-byte accesses, else one.
__global__ void k_to_half(const float *__restrict__ src, __half *__restrict__ dst, int64_t n, bool vec) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vec) {
        const int64_t i = 4 * t;
        if (i + 3 < n) {
            const float4 v = *reinterpret_cast<const float4 *>(src + i);
            __half2 *d = reinterpret_cast<__half2 *>(dst + i);
            d[0] = __halves2half2(__float2half_rn(v.x), __float2half_rn(v.y));
            d[1] = __halves2half2(__float2half_rn(v.z), __float2half_rn(v.w));
        } else {
            for (int64_t k = i; k < n; k++) dst[k] = __float2half_rn(src[k]);
        }
    } else if (t < n) {
        dst[t] = __float2half_rn(src[t]);
    }
}

}  // namespace

void launch_to_half(const float *src, uint16_t *dst, int64_t n, cudaStream_t st) {
    if (n <= 0 || !src || !dst) return;
    const bool vec = ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 8 == 0);
    const int64_t threads = vec ? (n + 3) / 4 : n;
    count_launch();
    k_to_half<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(src, reinterpret_cast<__half *>(dst), n, vec);
}

}  // namespace tgs
