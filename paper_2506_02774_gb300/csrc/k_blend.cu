// k_blend.cu -- front-to-back alpha blending per 16x16 tile (paper
// Sec. 3.1 'Rasterization', Eq. 3) with the preemptive log-domain test of
// Sec. 4.2 (Eq. 4) in front of the exponential.
//
// One CTA of 256 threads per tile, one pixel per thread; warp w shades pixel
// rows 2w and 2w+1.  The tile's pair range is consumed in batches of 256
// records (48 bytes each, depth-rank order) staged in shared memory.  Each
// record carries the half-height of its opacity-aware footprint box, outside
// which rho < ln alpha* - ln theta holds with a margin; from it every warp
// builds, in depth order, the list of batch records whose box reaches its two
// rows and walks only that list.  Pixels a warp skips this way would have
// failed the Eq. 4 test anyway, so the result is the same as walking the
// whole batch, but tiles crossing the horizon (tens of thousands of small,
// distant Gaussians over sky pixels that never saturate) cost each warp a
// fraction of the pairs.  Per pixel:
//   rho   = A dx^2 + B dx dy + C dy^2      (A = -a/2, B = -b, C = -c/2)
//   skip if rho < ln alpha* - ln theta     (Eq. 4: alpha < alpha*, no exp)
//   alpha = min(0.99, theta e^rho)         (Eq. 3)
//   T'    = T (1 - alpha); stop when T' < 1e-4 (this Gaussian excluded)
//   C    += alpha T rgb; T = T'
// CTAs take tiles heaviest first (k_tile_order).  The CTA leaves once all
// 256 pixels have stopped.  Modes: canonical (every
// pixel of the tile, alpha first, then the alpha* test; for the
// filtered-vs-unfiltered comparison) and the Eq. 5 lookup table for e^rho.
#include "vgr_internal.cuh"
#include "vgr_launch.h"

namespace vgr {

constexpr int BL_THREADS = TILE * TILE;  // 256, one pixel each
constexpr int BL_WARPS = BL_THREADS / 32;
constexpr int BL_BATCH = 256;

template <int MODE>
__global__ void __launch_bounds__(BL_THREADS) k_blend(const uint32_t* __restrict__ tile_order,
                                                      const uint2* __restrict__ ranges,
                                                      const uint32_t* __restrict__ pair_rank,
                                                      const float4* __restrict__ srecA,
                                                      const float4* __restrict__ srecB,
                                                      const float4* __restrict__ srecC,
                                                      const FrameParams* __restrict__ fp,
                                                      const float* __restrict__ lut, float* __restrict__ image,
                                                      Counters* __restrict__ ctr) {
    __shared__ float4 sA[BL_BATCH];
    __shared__ float4 sB[BL_BATCH];
    __shared__ float4 sC[BL_BATCH];
    __shared__ uint8_t s_mask[BL_BATCH];               // bit w: the record reaches warp w's rows
    __shared__ uint8_t s_list[BL_WARPS][BL_BATCH];     // per-warp record indices, depth order
    __shared__ float s_lut[260];
    const uint32_t W = fp->width, H = fp->height, TW = fp->tiles_x;
    const uint32_t tile = tile_order[blockIdx.x];  // heaviest tiles first
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t px = (tile % TW) * TILE + (threadIdx.x & (TILE - 1));
    const uint32_t ty0 = (tile / TW) * TILE;
    const uint32_t py = ty0 + (threadIdx.x / TILE);
    const bool inside = px < W && py < H;
    const float fxp = (float)px + 0.5f, fyp = (float)py + 0.5f;
    const float row0 = (float)ty0 + 0.5f;  // centre of the tile's first pixel row
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
    for (uint32_t b = rg.x; b < rg.y; b += BL_BATCH) {
        if (__syncthreads_and(done)) break;
        const uint32_t j = b + threadIdx.x;
        uint32_t mask = 0;
        if (j < rg.y) {
            const uint32_t rk = pair_rank[j];
            const float4 A = srecA[rk];
            const float4 B = srecB[rk];
            sA[threadIdx.x] = A;
            sB[threadIdx.x] = B;
            sC[threadIdx.x] = srecC[rk];
            if (MODE == 1) {
                mask = 0xFFu;
            } else {
                // rows r with |row0 + r - v| <= half-height, as row pairs (warps)
                const float lo = fmaxf(0.f, ceilf(A.y - B.w - row0));
                const float hi = fminf((float)(TILE - 1), floorf(A.y + B.w - row0));
                if (lo <= hi) {
                    const uint32_t w0 = (uint32_t)lo >> 1, w1 = (uint32_t)hi >> 1;
                    mask = ((2u << w1) - 1u) & ~((1u << w0) - 1u);
                }
            }
        }
        s_mask[threadIdx.x] = (uint8_t)mask;
        __syncthreads();
        // this warp's records, in depth order
        uint32_t n = 0;
#pragma unroll
        for (int c = 0; c < BL_BATCH / 32; ++c) {
            const bool bit = (s_mask[c * 32 + lane] >> warp) & 1u;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, bit);
            if (bit) s_list[warp][n + __popc(bal & lanemask_lt())] = (uint8_t)(c * 32 + lane);
            n += __popc(bal);
        }
        __syncwarp();
        if (!done) {
            for (uint32_t i = 0; i < n; ++i) {
                const uint32_t k = s_list[warp][i];
                const float4 A = sA[k];
                const float dx = A.x - fxp, dy = A.y - fyp;
                const float4 B = sB[k];
                const float rho = fmaf(A.z * dx, dx, fmaf(B.x * dy, dy, A.w * dx * dy));
                ++evals;
                float alpha;
                if (MODE == 1) {  // canonical: Eq. 3, then the alpha* test
                    alpha = fminf(ALPHA_MAX, B.z * __expf(rho));
                    if (alpha < ALPHA_MIN) continue;
                } else {
                    if (rho < B.y) continue;  // Eq. 4 before Eq. 3
                    if (MODE == 0) {
                        alpha = fminf(ALPHA_MAX, B.z * __expf(rho));
                    } else {  // Eq. 5: nearest of m intervals over [-5.55, 0]
                        const uint32_t idx = min(m, (uint32_t)__float2int_rn(rho * lut_scale));
                        alpha = fminf(ALPHA_MAX, B.z * s_lut[idx]);
                    }
                }
                const float Tn = T * (1.f - alpha);
                if (Tn < T_MIN) { done = true; break; }
                const float w = alpha * T;
                const float4 C4 = sC[k];
                cr = fmaf(w, C4.x, cr);
                cg = fmaf(w, C4.y, cg);
                cb = fmaf(w, C4.z, cb);
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
    if (lane == 0 && wsum) atomicAdd(&ctr->pix_evals, (unsigned long long)wsum);
}

void launch_blend(uint32_t n_tiles, const uint32_t* tile_order, const uint2* ranges, const uint32_t* pair_rank,
                  const float4* srecA,
                  const float4* srecB, const float4* srecC, const FrameParams* fp, const float* lut, float* image,
                  Counters* ctr, uint32_t filter, uint32_t exp_mode, cudaStream_t s) {
    if (filter == VGR_FILTER_CANONICAL)
        k_blend<1><<<n_tiles, BL_THREADS, 0, s>>>(tile_order, ranges, pair_rank, srecA, srecB, srecC, fp, lut, image, ctr);
    else if (exp_mode == VGR_EXP_LUT)
        k_blend<2><<<n_tiles, BL_THREADS, 0, s>>>(tile_order, ranges, pair_rank, srecA, srecB, srecC, fp, lut, image, ctr);
    else
        k_blend<0><<<n_tiles, BL_THREADS, 0, s>>>(tile_order, ranges, pair_rank, srecA, srecB, srecC, fp, lut, image, ctr);
}

}  // namespace vgr
