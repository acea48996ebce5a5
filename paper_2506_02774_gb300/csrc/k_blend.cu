// k_blend.cu -- front-to-back alpha blending per 16x16 tile (paper
// Sec. 3.1 'Rasterization', Eq. 3) with the preemptive log-domain test of
// Sec. 4.2 (Eq. 4) in front of the exponential.
//
// One CTA of 256 threads per tile, one pixel per thread.  The tile's pair
// range is consumed in batches of 256: each thread gathers one Gaussian
// record (40 bytes, in depth-rank order) into shared memory, then every
// pixel walks the batch:
//   rho   = A dx^2 + B dx dy + C dy^2      (A = -a/2, B = -b, C = -c/2)
//   skip if rho < ln alpha* - ln theta     (Eq. 4: alpha < alpha*, no exp)
//   alpha = min(0.99, theta e^rho)         (Eq. 3)
//   T'    = T (1 - alpha); stop when T' < 1e-4 (this Gaussian excluded)
//   C    += alpha T rgb; T = T'
// The CTA leaves once every pixel has stopped.  Modes: canonical (alpha
// first, then the alpha* test, for the filtered-vs-unfiltered comparison)
// and the Eq. 5 lookup table for e^rho.
#include "vgr_internal.cuh"
#include "vgr_launch.h"

namespace vgr {

constexpr int BL_THREADS = 256;

template <int MODE>
__global__ void __launch_bounds__(BL_THREADS) k_blend(const uint2* __restrict__ ranges,
                                                      const uint32_t* __restrict__ pair_rank,
                                                      const float4* __restrict__ srecA,
                                                      const float4* __restrict__ srecB,
                                                      const float2* __restrict__ srecC,
                                                      const FrameParams* __restrict__ fp,
                                                      const float* __restrict__ lut, float* __restrict__ image,
                                                      Counters* __restrict__ ctr) {
    __shared__ float4 sA[BL_THREADS];
    __shared__ float4 sB[BL_THREADS];
    __shared__ float2 sC[BL_THREADS];
    __shared__ float s_lut[260];
    const uint32_t W = fp->width, H = fp->height, TW = fp->tiles_x;
    const uint32_t tile = blockIdx.x;
    const uint32_t px = (tile % TW) * TILE + (threadIdx.x & (TILE - 1));
    const uint32_t py = (tile / TW) * TILE + (threadIdx.x / TILE);
    const bool inside = px < W && py < H;
    const float fxp = (float)px + 0.5f, fyp = (float)py + 0.5f;
    uint32_t m = 0;
    float lut_scale = 0.f;
    if (MODE == 2) {
        m = fp->lut_size;
        lut_scale = -(float)m / 5.55f;
        for (uint32_t i = threadIdx.x; i <= m; i += BL_THREADS) s_lut[i] = lut[i];
    }
    const uint2 rg = ranges[tile];
    float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f;
    bool done = !inside;
    uint32_t evals = 0;
    for (uint32_t b = rg.x; b < rg.y; b += BL_THREADS) {
        if (__syncthreads_and(done)) break;
        const uint32_t j = b + threadIdx.x;
        if (j < rg.y) {
            const uint32_t rk = pair_rank[j];
            sA[threadIdx.x] = srecA[rk];
            sB[threadIdx.x] = srecB[rk];
            sC[threadIdx.x] = srecC[rk];
        }
        __syncthreads();
        if (!done) {
            const int cnt = (int)min((uint32_t)BL_THREADS, rg.y - b);
            for (int k = 0; k < cnt; ++k) {
                const float4 A = sA[k];
                const float dx = A.x - fxp, dy = A.y - fyp;
                const float4 B = sB[k];
                const float rho = fmaf(A.z * dx, dx, fmaf(B.x * dy, dy, A.w * dx * dy));
                ++evals;
                float alpha;
                if (MODE == 0) {  // preemptive: Eq. 4 before Eq. 3
                    if (rho < B.y) continue;
                    alpha = fminf(ALPHA_MAX, B.z * __expf(rho));
                } else if (MODE == 1) {  // canonical: Eq. 3, then the alpha* test
                    alpha = fminf(ALPHA_MAX, B.z * __expf(rho));
                    if (alpha < ALPHA_MIN) continue;
                } else {  // Eq. 4, then Eq. 5: nearest of m intervals over [-5.55, 0]
                    if (rho < B.y) continue;
                    const uint32_t idx = min(m, (uint32_t)__float2int_rn(rho * lut_scale));
                    alpha = fminf(ALPHA_MAX, B.z * s_lut[idx]);
                }
                const float Tn = T * (1.f - alpha);
                if (Tn < T_MIN) { done = true; break; }
                const float w = alpha * T;
                const float2 C2 = sC[k];
                cr = fmaf(w, B.w, cr);
                cg = fmaf(w, C2.x, cg);
                cb = fmaf(w, C2.y, cb);
                T = Tn;
            }
        }
    }
    if (inside) {
        float* o = image + ((size_t)py * W + px) * 3;
        o[0] = cr;
        o[1] = cg;
        o[2] = cb;
    }
    const uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, evals);
    if (lane_id() == 0 && wsum) atomicAdd(&ctr->pix_evals, (unsigned long long)wsum);
}

void launch_blend(uint32_t n_tiles, const uint2* ranges, const uint32_t* pair_rank, const float4* srecA,
                  const float4* srecB, const float2* srecC, const FrameParams* fp, const float* lut, float* image,
                  Counters* ctr, uint32_t filter, uint32_t exp_mode, cudaStream_t s) {
    if (filter == VGR_FILTER_CANONICAL)
        k_blend<1><<<n_tiles, BL_THREADS, 0, s>>>(ranges, pair_rank, srecA, srecB, srecC, fp, lut, image, ctr);
    else if (exp_mode == VGR_EXP_LUT)
        k_blend<2><<<n_tiles, BL_THREADS, 0, s>>>(ranges, pair_rank, srecA, srecB, srecC, fp, lut,
                                                                  image, ctr);
    else
        k_blend<0><<<n_tiles, BL_THREADS, 0, s>>>(ranges, pair_rank, srecA, srecB, srecC, fp, lut, image, ctr);
}

}  // namespace vgr
