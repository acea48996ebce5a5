// k_store.cu -- reduced-precision device storage of per-Gaussian attributes:
// SH coefficients as FP16 and covariances as BF16 (round to nearest even),
// expanded back to FP32 in registers by the preprocess kernel.  Node centres,
// radii and opacities stay FP32, so cut membership and depth order do not
// change.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "vgr_internal.cuh"
#include "vgr_launch.h"

namespace vgr {

// src: n x k3 floats; dst: n x stride halves (stride a multiple of 8, zero padded)
__global__ void k_sh_half(const float* __restrict__ src, uint32_t n, uint32_t k3, __half* __restrict__ dst,
                          uint32_t stride) {
    const uint64_t total = (uint64_t)n * stride;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t node = i / stride;
        const uint32_t j = (uint32_t)(i - node * stride);
        dst[i] = j < k3 ? __float2half_rn(src[node * k3 + j]) : __float2half_rn(0.f);
    }
}

// src: n x 6 floats (xx xy xz yy yz zz); dst: n x 8 bf16 (2 spare, zero)
__global__ void k_cov_bf16(const float* __restrict__ src, uint32_t n, __nv_bfloat16* __restrict__ dst) {
    const uint64_t total = (uint64_t)n * 8;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t node = i >> 3;
        const uint32_t j = (uint32_t)(i & 7u);
        dst[i] = j < 6 ? __float2bfloat16_rn(src[node * 6 + j]) : __float2bfloat16_rn(0.f);
    }
}

void convert_sh_half(const float* src, uint32_t n, uint32_t k3, void* dst, uint32_t stride, cudaStream_t s) {
    k_sh_half<<<2048, 256, 0, s>>>(src, n, k3, reinterpret_cast<__half*>(dst), stride);
}

void convert_cov_bf16(const float* src6, uint32_t n, void* dst, cudaStream_t s) {
    k_cov_bf16<<<2048, 256, 0, s>>>(src6, n, reinterpret_cast<__nv_bfloat16*>(dst));
}

}  // namespace vgr
