// k_blend.cu -- front-to-back alpha blending per 16x16 tile (paper
// Sec. 3.1 'Rasterization', Eq. 3) with the preemptive log-domain test of
// Sec. 4.2 (Eq. 4) in front of the exponential.
//
// One CTA of 256 threads per tile, one pixel per thread; warp w shades pixel
// rows 2w and 2w+1 and walks the tile's pair range on its own (no CTA-wide
// barrier): 32 records at a time (48 bytes each, depth-rank order), it keeps
// those whose opacity-aware footprint box reaches one of its two rows -- the
// box half-height is part of the record, and outside the box
// rho < ln alpha* - ln theta holds with a margin, so a skipped record would
// have failed the Eq. 4 test at every pixel of those rows -- stages them in
// its own slice of shared memory and walks them in order, two at a time for
// instruction-level parallelism.  The next 32 records are loaded while the
// current ones are walked; the eight warps of a tile read the same records,
// so all but the first read of each record hit L1.  A warp stops when its 32
// pixels have stopped; tiles crossing the horizon (tens of thousands of
// small distant Gaussians, each reaching one or two rows) cost each warp a
// fraction of the pairs.  Per pixel:
//   rho   = A dx^2 + B dx dy + C dy^2      (A = -a/2, B = -b, C = -c/2)
//   skip if rho < ln alpha* - ln theta     (Eq. 4: alpha < alpha*, no exp)
//   alpha = min(0.99, theta e^rho)         (Eq. 3)
//   T'    = T (1 - alpha); stop when T' < 1e-4 (this Gaussian excluded)
//   C    += alpha T rgb; T = T'
// CTAs take tiles heaviest first (k_tile_order).  Modes: canonical (every
// record at every pixel of the tile, alpha first, then the alpha* test; for
// the filtered-vs-unfiltered comparison) and the Eq. 5 lookup table for e^rho.
#include "vgr_internal.cuh"
#include "vgr_launch.h"

namespace vgr {

constexpr int BL_THREADS = TILE * TILE;  // 256, one pixel each
constexpr int BL_WARPS = BL_THREADS / 32;
constexpr uint32_t FULL = 0xFFFFFFFFu;

struct BlendPixel {
    float fxp, fyp;
    float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f;
    bool done;
    uint32_t evals = 0, contribs = 0;
};

// One record at one pixel; returns false once the pixel has stopped.
template <int MODE>
__device__ __forceinline__ bool blend_step(BlendPixel& p, const float4& A, const float4& B, const float4* __restrict__ sC,
                                           uint32_t k, float rho, const float* s_lut, uint32_t m, float lut_scale) {
    ++p.evals;
    float alpha;
    if (MODE == 1) {  // canonical: Eq. 3, then the alpha* test
        alpha = fminf(ALPHA_MAX, B.z * __expf(rho));
        if (alpha < ALPHA_MIN) return true;
    } else {
        if (rho < B.y) return true;  // Eq. 4 before Eq. 3
        if (MODE == 0) {
            alpha = fminf(ALPHA_MAX, B.z * __expf(rho));
        } else {  // Eq. 5: nearest of m intervals over [-5.55, 0]
            const uint32_t idx = min(m, (uint32_t)__float2int_rn(rho * lut_scale));
            alpha = fminf(ALPHA_MAX, B.z * s_lut[idx]);
        }
    }
    const float Tn = p.T * (1.f - alpha);
    if (Tn < T_MIN) { p.done = true; return false; }
    const float w = alpha * p.T;
    const float4 C4 = sC[k];
    p.cr = fmaf(w, C4.x, p.cr);
    p.cg = fmaf(w, C4.y, p.cg);
    p.cb = fmaf(w, C4.z, p.cb);
    p.T = Tn;
    ++p.contribs;
    return true;
}

__device__ __forceinline__ float blend_rho(const BlendPixel& p, const float4& A, const float4& B) {
    const float dx = A.x - p.fxp, dy = A.y - p.fyp;
    return fmaf(A.z * dx, dx, fmaf(B.x * dy, dy, A.w * dx * dy));
}

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
    __shared__ float4 sA[BL_WARPS][32];
    __shared__ float4 sB[BL_WARPS][32];
    __shared__ float4 sC[BL_WARPS][32];
    __shared__ float s_lut[260];
    const uint32_t W = fp->width, H = fp->height, TW = fp->tiles_x;
    const uint32_t tile = tile_order[blockIdx.x];  // heaviest tiles first
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t px = (tile % TW) * TILE + (lane & (TILE - 1));
    const uint32_t ty0 = (tile / TW) * TILE;
    const uint32_t py = ty0 + 2 * warp + (lane >> 4);
    const bool inside = px < W && py < H;
    const float rlo = (float)(ty0 + 2 * warp) + 0.5f;  // centre of the warp's first row
    uint32_t m = 0;
    float lut_scale = 0.f;
    if (MODE == 2) {
        m = fp->lut_size;
        lut_scale = -(float)m / 5.55f;
        for (uint32_t i = threadIdx.x; i <= m; i += BL_THREADS) s_lut[i] = lut[i];
        __syncthreads();
    }
    const uint2 rg = ranges[tile];
    BlendPixel p;
    p.fxp = (float)px + 0.5f;
    p.fyp = (float)py + 0.5f;
    p.done = !inside;
    float4* wA = sA[warp];
    float4* wB = sB[warp];
    float4* wC = sC[warp];
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 nA = z4, nB = z4, nC = z4;
    {
        const uint32_t j = rg.x + lane;
        if (j < rg.y) {
            const uint32_t rk = pair_rank[j];
            nA = srecA[rk]; nB = srecB[rk]; nC = srecC[rk];
        }
    }
    for (uint32_t b = rg.x; b < rg.y; b += 32) {
        if (__all_sync(FULL, p.done)) break;
        const float4 A = nA, B = nB, C = nC;
        bool hit = b + lane < rg.y;
        if (MODE != 1) hit = hit && (A.y - B.w <= rlo + 1.0f) && (A.y + B.w >= rlo);
        const uint32_t hits = __ballot_sync(FULL, hit);
        if (hit) {
            const uint32_t s = __popc(hits & lanemask_lt());
            wA[s] = A; wB[s] = B; wC[s] = C;
        }
        {   // next 32 records in flight while these are walked
            const uint32_t j = b + 32 + lane;
            if (j < rg.y) {
                const uint32_t rk = pair_rank[j];
                nA = srecA[rk]; nB = srecB[rk]; nC = srecC[rk];
            }
        }
        __syncwarp();
        const uint32_t nh = __popc(hits);
        if (!p.done) {
            uint32_t i = 0;
            for (; i + 2 <= nh; i += 2) {
                const float4 A0 = wA[i], B0 = wB[i], A1 = wA[i + 1], B1 = wB[i + 1];
                const float r0 = blend_rho(p, A0, B0), r1 = blend_rho(p, A1, B1);
                if (!blend_step<MODE>(p, A0, B0, wC, i, r0, s_lut, m, lut_scale)) break;
                if (!blend_step<MODE>(p, A1, B1, wC, i + 1, r1, s_lut, m, lut_scale)) break;
            }
            if (!p.done && i < nh) {
                const float4 A0 = wA[i], B0 = wB[i];
                blend_step<MODE>(p, A0, B0, wC, i, blend_rho(p, A0, B0), s_lut, m, lut_scale);
            }
        }
        __syncwarp();
    }
    if (inside) {
        float* o = image + ((size_t)py * W + px) * 3;
        o[0] = p.cr;
        o[1] = p.cg;
        o[2] = p.cb;
    }
    const uint32_t wsum = __reduce_add_sync(FULL, p.evals);
    const uint32_t csum = __reduce_add_sync(FULL, p.contribs);
    if (lane == 0 && wsum) {
        atomicAdd(&ctr->pix_evals, (unsigned long long)wsum);
        atomicAdd(&ctr->pix_contribs, (unsigned long long)csum);
    }
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
