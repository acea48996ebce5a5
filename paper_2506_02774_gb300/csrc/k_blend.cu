// k_blend.cu -- front-to-back alpha blending per 16x16 tile (paper
// Sec. 3.1 'Rasterization', Eq. 3) with the preemptive log-domain test of
// Sec. 4.2 (Eq. 4) in front of the exponential.
//
// One CTA of 256 threads per tile, one pixel per thread; warp w shades pixel
// rows 2w and 2w+1 and walks the tile's pair range on its own (no CTA-wide
// barrier).  Each pair value carries the Gaussian's index in the in-front
// arrays and its row mask in the tile (set by the emission from the
// footprint box: outside the box rho < ln alpha* - ln theta holds with a
// margin, so a pair whose box misses the warp's two rows would fail the
// Eq. 4 test at every one of its pixels); within a tile the pairs are in
// depth order.  The warp scans the pair values (coalesced, a batch ahead),
// queues those with its row bit in a ring, and copies the 48-byte records
// (mean, conic, threshold, opacity, colour) of 32 queued hits at a time with
// cp.async into its own double-buffered slice of shared memory; the copies
// of the next 32 hits are in flight while the current ones are walked, two
// at a time for instruction-level parallelism.  Before the walk each lane
// rewrites its staged record for the
// warp's two rows (the row offsets of the mean folded into the conic
// terms), so a pixel evaluates rho with one subtraction and two FMAs.
// Records are read only for the pairs a warp needs, and the eight warps of
// a tile share them through L1.  A warp stops when its 32 pixels have stopped; tiles crossing the
// horizon (tens of thousands of small distant Gaussians, each reaching one
// or two rows) cost each warp a scan of 4-byte values and a fraction of the
// records.  Per pixel:
//   rho   = A dx^2 + B dx dy + C dy^2      (A = -a/2, B = -b, C = -c/2)
//   skip if rho < ln alpha* - ln theta     (Eq. 4: alpha < alpha*, no exp)
//   alpha = min(0.99, theta e^rho)         (Eq. 3)
//   T'    = T (1 - alpha); stop when T' < 1e-4 (this Gaussian excluded)
//   C    += alpha T rgb; T = T'
// (the exact mode takes the same test and alpha in base 2 with ln theta
// folded into the exponent, see blend_prepare).
// CTAs take tiles heaviest first (k_tile_order).  Modes: canonical (every
// record at every pixel of the tile, alpha first, then the alpha* test; for
// the filtered-vs-unfiltered comparison; its row masks are all ones) and the
// Eq. 5 lookup table for e^rho.
#include "vgr_internal.cuh"
#include "vgr_launch.h"

namespace vgr {

constexpr int BL_THREADS = TILE * TILE;  // 256, one pixel each
constexpr int BL_WARPS = BL_THREADS / 32;
constexpr int BL_SCAN = 128;   // pair values scanned per batch (4 per lane, loaded one batch ahead)
constexpr int BL_RING = 256;   // queue capacity per warp: < 32 queued + BL_SCAN appended never exceeds it
constexpr uint32_t FULL = 0xFFFFFFFFu;

struct BlendPixel {
    float fxp, fyp;
    float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f;
    bool done;
    uint32_t evals = 0, contribs = 0;
};

constexpr float LOG2E = 1.4426950408889634f;
constexpr float LOG2_ALPHA_MIN = -7.9943534368588578f;  // log2(1/255)

// A staged record, rewritten for the warp's two pixel rows (dy0, dy1 the
// offsets of the mean from their centres):
//   X = (u, A, thr, theta),  R = (B dy0, C dy0^2, B dy1, C dy1^2)
// so that at a pixel of row r, dx = u - x:  rho = (A dx + B dy_r) dx + C dy_r^2,
// one subtraction and two FMAs (A = -a/2, B = -b, C = -c/2).  The exact mode
// works in base 2 with the opacity folded in: A, B, C scaled by log2 e and
// log2 theta added to the constant term, so that
//   rho' = (A' dx + B' dy_r) dx + (C' dy_r^2 + log2 theta) = log2(theta e^rho),
// Eq. 4 becomes rho' >= log2 alpha* (one constant) and Eq. 3 alpha =
// min(0.99, 2^rho'): X = (u, A', -, -).
template <int MODE>
__device__ __forceinline__ void blend_prepare(float4& a, float4& b, float row0) {
    const float dy0 = a.y - row0, dy1 = a.y - (row0 + 1.0f);
    if (MODE == 0) {
        const float Bc = a.w * LOG2E, Cc = b.x * LOG2E;
        const float l2th = (LN_ALPHA_MIN - b.y) * LOG2E;  // b.y = ln alpha* - ln theta
        const float4 X = make_float4(a.x, a.z * LOG2E, 0.f, 0.f);
        const float4 R = make_float4(Bc * dy0, fmaf(Cc * dy0, dy0, l2th), Bc * dy1, fmaf(Cc * dy1, dy1, l2th));
        a = X;
        b = R;
    } else {
        const float Bc = a.w, Cc = b.x;
        const float4 X = make_float4(a.x, a.z, b.y, b.z);
        const float4 R = make_float4(Bc * dy0, (Cc * dy0) * dy0, Bc * dy1, (Cc * dy1) * dy1);
        a = X;
        b = R;
    }
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One record at one pixel; returns false once the pixel has stopped.
template <int MODE>
__device__ __forceinline__ bool blend_step(BlendPixel& p, const float4& X, const float4* __restrict__ sC, uint32_t k,
                                           float rho, const float* s_lut, uint32_t m, float lut_scale) {
    float alpha;
    if (MODE == 0) {  // base 2, opacity folded in (see blend_prepare)
        if (rho < LOG2_ALPHA_MIN) return true;
        alpha = fminf(ALPHA_MAX, ex2_approx(rho));
    } else if (MODE == 1) {  // canonical: Eq. 3, then the alpha* test
        alpha = fminf(ALPHA_MAX, X.w * __expf(rho));
        if (alpha < ALPHA_MIN) return true;
    } else {
        if (rho < X.z) return true;  // Eq. 4 before Eq. 3
        // Eq. 5: nearest of m intervals over [-5.55, 0]
        const uint32_t idx = min(m, (uint32_t)__float2int_rn(rho * lut_scale));
        alpha = fminf(ALPHA_MAX, X.w * s_lut[idx]);
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

// The staged X of slot i: only (u, A') in the exact mode.
template <int MODE>
__device__ __forceinline__ float4 load_x(const float4* wA, uint32_t i) {
    if (MODE == 0) {
        const float2 x = reinterpret_cast<const float2*>(wA)[2 * i];
        return make_float4(x.x, x.y, 0.f, 0.f);
    }
    return wA[i];
}

__device__ __forceinline__ float blend_rho(const BlendPixel& p, const float4& X, const float2& R) {
    const float dx = X.x - p.fxp;
    return fmaf(fmaf(X.y, dx, R.x), dx, R.y);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int MODE>
__global__ void __launch_bounds__(BL_THREADS) k_blend(const uint32_t* __restrict__ tile_order,
                                                      const uint2* __restrict__ ranges,
                                                      const uint32_t* __restrict__ pair_val,
                                                      const float4* __restrict__ recA,
                                                      const float4* __restrict__ recB,
                                                      const float4* __restrict__ rgb,
                                                      const FrameParams* __restrict__ fp,
                                                      const float* __restrict__ lut, float* __restrict__ image,
                                                      Counters* __restrict__ ctr) {
    pdl_wait();
    // [buffer][record part A, B, C][warp][slot]
    __shared__ __align__(16) float4 sbuf[2][3][BL_WARPS][32];
    __shared__ uint32_t s_ring[BL_WARPS][BL_RING];  // per-warp queue of hit pair values
    __shared__ float s_lut[260];
    const uint32_t W = fp->width, H = fp->height, TW = fp->tiles_x;
    float* const host_image = fp->host_image;
    const uint32_t tile = tile_order[blockIdx.x];  // heaviest tiles first
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t px = (tile % TW) * TILE + (lane & (TILE - 1));
    const uint32_t ty0 = (tile / TW) * TILE;
    const uint32_t py = ty0 + 2 * warp + (lane >> 4);
    const bool inside = px < W && py < H;
    const uint32_t wbit = 1u << warp;
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
    // The warp's pairs (those whose row mask names it, in depth order) pass
    // through a ring of pair values: the range is scanned BL_SCAN values at a
    // time (loaded one batch ahead), hits are appended, and records are
    // staged 32 hits at a time, so staging and the walk run on full chunks
    // however sparse the warp's hits are among the tile's pairs.
    uint32_t* ring = s_ring[warp];
    uint32_t head = 0, tail = 0;
    uint32_t bp = rg.x;  // first pair value of the pending batch
    uint32_t pend[BL_SCAN / 32];
#pragma unroll
    for (int g = 0; g < BL_SCAN / 32; ++g) {
        const uint32_t j = bp + 32u * g + lane;
        pend[g] = j < rg.y ? pair_val[j] : 0u;
    }
    auto refill = [&]() {
        while (tail - head < 32u && bp < rg.y) {
#pragma unroll
            for (int g = 0; g < BL_SCAN / 32; ++g) {
                const uint32_t v = pend[g];
                const bool hit = (v & wbit) != 0u;  // entries past the range hold 0
                const uint32_t hits = __ballot_sync(FULL, hit);
                if (hit) ring[(tail + __popc(hits & lanemask_lt())) & (BL_RING - 1)] = v;
                tail += __popc(hits);
            }
            bp += BL_SCAN;
#pragma unroll
            for (int g = 0; g < BL_SCAN / 32; ++g) {
                const uint32_t j = bp + 32u * g + lane;
                pend[g] = j < rg.y ? pair_val[j] : 0u;
            }
        }
        __syncwarp();
    };
    // stage up to 32 queued hits into buffer buf; returns their number
    auto issue = [&](int buf) -> uint32_t {
        const uint32_t nh = min(32u, tail - head);
        if (lane < nh) {
            const uint32_t gi = ring[(head + lane) & (BL_RING - 1)] >> 8;
            cp_async16(&sbuf[buf][0][warp][lane], recA + gi);
            cp_async16(&sbuf[buf][1][warp][lane], recB + gi);
            cp_async16(&sbuf[buf][2][warp][lane], rgb + gi);
        }
        cp_async_commit();
        head += nh;
        return nh;
    };
    refill();
    uint32_t nh_cur = issue(0);
    int buf = 0;
    while (nh_cur > 0) {
        if (__all_sync(FULL, p.done)) break;
        refill();
        const uint32_t nh_next = issue(buf ^ 1);  // the next chunk in flight during this walk
        cp_async_wait<1>();  // this chunk's copies (all but the newest group)
        __syncwarp();
        float4* wA = sbuf[buf][0][warp];
        float4* wB = sbuf[buf][1][warp];
        const float4* wC = sbuf[buf][2][warp];
        const uint32_t nh = nh_cur;
        if (lane < nh) blend_prepare<MODE>(wA[lane], wB[lane], rlo);  // each lane its own slot
        __syncwarp();
        if (!p.done) {
            // rows 2w (lanes 0-15) and 2w + 1 (lanes 16-31): each reads its half of R
            const float2* wR = reinterpret_cast<const float2*>(wB) + (lane >> 4);
            uint32_t i = 0, ev = nh;
            for (; i + 2 <= nh; i += 2) {
                const float4 X0 = load_x<MODE>(wA, i), X1 = load_x<MODE>(wA, i + 1);
                const float2 R0 = wR[2 * i], R1 = wR[2 * i + 2];
                const float r0 = blend_rho(p, X0, R0), r1 = blend_rho(p, X1, R1);
                if (!blend_step<MODE>(p, X0, wC, i, r0, s_lut, m, lut_scale)) { ev = i + 1; break; }
                if (!blend_step<MODE>(p, X1, wC, i + 1, r1, s_lut, m, lut_scale)) { ev = i + 2; break; }
            }
            if (!p.done && i < nh) {
                const float4 X0 = load_x<MODE>(wA, i);
                if (!blend_step<MODE>(p, X0, wC, i, blend_rho(p, X0, wR[2 * i]), s_lut, m, lut_scale)) ev = i + 1;
            }
            p.evals += ev;
        }
        __syncwarp();  // the walk is done with this buffer before it is refilled
        buf ^= 1;
        nh_cur = nh_next;
    }
    cp_async_wait<0>();
    if (inside) {
        const size_t at = ((size_t)py * W + px) * 3;
        float* o = image + at;
        o[0] = p.cr;
        o[1] = p.cg;
        o[2] = p.cb;
        if (host_image) {  // the caller's pinned host buffer, over the host link
            float* q = host_image + at;
            q[0] = p.cr;
            q[1] = p.cg;
            q[2] = p.cb;
        }
    }
    const uint32_t wsum = __reduce_add_sync(FULL, p.evals);
    const uint32_t csum = __reduce_add_sync(FULL, p.contribs);
    if (lane == 0 && wsum) {
        atomicAdd(&ctr->pix_evals, (unsigned long long)wsum);
        atomicAdd(&ctr->pix_contribs, (unsigned long long)csum);
    }
}

void launch_blend(uint32_t n_tiles, const uint32_t* tile_order, const uint2* ranges, const uint32_t* pair_val,
                  const float4* recA, const float4* recB, const float4* rgb, const FrameParams* fp, const float* lut, float* image,
                  Counters* ctr, uint32_t filter, uint32_t exp_mode, cudaStream_t s) {
    if (filter == VGR_FILTER_CANONICAL)
        launch_k(k_blend<1>, n_tiles, BL_THREADS, s, tile_order, ranges, pair_val, recA, recB, rgb, fp, lut, image, ctr);
    else if (exp_mode == VGR_EXP_LUT)
        launch_k(k_blend<2>, n_tiles, BL_THREADS, s, tile_order, ranges, pair_val, recA, recB, rgb, fp, lut, image, ctr);
    else
        launch_k(k_blend<0>, n_tiles, BL_THREADS, s, tile_order, ranges, pair_val, recA, recB, rgb, fp, lut, image, ctr);
}

}  // namespace vgr
