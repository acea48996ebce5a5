// k_blend.cu -- front-to-back alpha blending per 16x16 tile (paper
// Sec. 3.1 'Rasterization', Eq. 3) with the preemptive log-domain test of
// Sec. 4.2 (Eq. 4) in front of the exponential.
//
// A tile of T x T pixels (T = 8, 16 or 32, a tuning knob) is T T / 32
// strips of 32 / T rows x T columns; one warp shades one strip, one pixel per
// lane.  The kernel is persistent: its CTAs (a few per SM) take tiles one at a
// time from a work list ordered heaviest first -- the tiles of one view, or
// of every view of a batch -- through a global counter, and the CTA's warps
// claim the strips of the CTA's tiles from a shared counter, so a warp that
// finishes a light strip moves on to the next strip at once instead of idling
// until its tile's heaviest strip is done, and the strips of a tile run on
// one SM, sharing its pair values and records through L1.
//
// Each pair value carries the Gaussian's index in the in-front arrays and its
// row mask in the tile (set by the emission from the footprint box: outside
// the box rho < ln alpha* - ln theta holds with a margin, so a pair whose box
// misses the strip's rows would fail the Eq. 4 test at every one of its
// pixels); within a tile the pairs are in depth order.  The warp scans its
// tile's pair values (coalesced, a batch ahead), queues those with its row
// bit in a ring, and copies the 48-byte records (mean, conic, threshold,
// opacity, colour) of DEPTH queued hits at a time with cp.async into its own
// double-buffered slice of shared memory; the copies of the next chunk are in
// flight while the current one is walked, two records at a time for
// instruction-level parallelism.  Before the walk each lane rewrites its
// staged records for the strip's rows (the row offsets of the mean folded
// into the conic terms), so a pixel evaluates rho with one subtraction and
// two FMAs.  Records are read only for the pairs a strip needs, and the warps
// of a CTA, working on the strips of the same tiles, share them through L1.
// A warp leaves a strip when its 32 pixels have stopped; tiles crossing the
// horizon (tens of thousands of small distant Gaussians, each reaching one or
// two rows) cost each strip a scan of 4-byte values and a fraction of the
// records.  Per pixel:
//   rho   = A dx^2 + B dx dy + C dy^2      (A = -a/2, B = -b, C = -c/2)
//   skip if rho < ln alpha* - ln theta     (Eq. 4: alpha < alpha*, no exp)
//   alpha = min(0.99, theta e^rho)         (Eq. 3)
//   T'    = T (1 - alpha); stop when T' < 1e-4 (this Gaussian excluded)
//   C    += alpha T rgb; T = T'
// (the exact mode takes the same test and alpha in base 2 with ln theta
// folded into the exponent, see blend_prepare).  Modes: canonical (every
// record at every pixel of the tile, alpha first, then the alpha* test; for
// the filtered-vs-unfiltered comparison; its row masks are all ones) and the
// Eq. 5 lookup table for e^rho.  DEPTH (hits staged per chunk: 16, 32 or 48)
// and T are tuning knobs; the image does not depend on them.
#include "vgr_internal.cuh"
#include "vgr_launch.h"

namespace vgr {

constexpr int BL_THREADS = 256;          // 8 warps: a warp shades one strip of 32 pixels at a time
constexpr int BL_WARPS = BL_THREADS / 32;
constexpr int BL_SCAN = 128;   // pair values scanned per batch (4 per lane, loaded one batch ahead)
constexpr int BL_MIN_CTAS = 4; // resident CTAs per SM the register budget is set for (up to 64 registers)
constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t WORK_TILE_BITS = 20;  // work item = view << 20 | tile
constexpr uint32_t WORK_TILE_MASK = (1u << WORK_TILE_BITS) - 1u;

struct BlendPixel {
    float fxp;
    float T, cr, cg, cb;
    bool done;
    uint32_t contribs;
};

constexpr float LOG2E = 1.4426950408889634f;
constexpr float LOG2_ALPHA_MIN = -7.9943534368588578f;  // log2(1/255)

// A staged record, rewritten for the strip's SR pixel rows (dy_r the offset of
// the mean from the centre of row r):
//   X = (u, A, thr, theta),  R_r = (B dy_r, C dy_r^2)
// so that at a pixel of row r, dx = u - x:  rho = (A dx + B dy_r) dx + C dy_r^2,
// one subtraction and two FMAs (A = -a/2, B = -b, C = -c/2).  The exact mode
// works in base 2 with the opacity folded in: A, B, C scaled by log2 e and
// log2 theta added to the constant term, so that
//   rho' = (A' dx + B' dy_r) dx + (C' dy_r^2 + log2 theta) = log2(theta e^rho),
// Eq. 4 becomes rho' >= log2 alpha* (one constant) and Eq. 3 alpha =
// min(0.99, 2^rho'): X = (u, A', -, -).  R_0, R_1 replace the raw second
// record half in b; rows 2 and 3 (strips of 4 rows) go to b2.
//
// Returns the record's pixel mask in the strip: bit q (pixel q = row q / T,
// column q % T) is set when q lies in the footprint box, the axis-aligned
// box of {rho >= ln alpha* - ln theta - 2e-3} (with a margin) that preprocess
// stored as FP16 half-extents rounded up.  Outside it the Eq. 4 test fails,
// so the pixel need not look at the record.  The canonical mode (no Eq. 4
// before Eq. 3) and 'full' mark every pixel.
template <int MODE, int SR, int T>
__device__ __forceinline__ uint32_t blend_prepare(float4& a, float4& b, float4& b2, float row0, float col0,
                                                  bool full) {
    uint32_t pmask = 0xFFFFFFFFu;
    if (MODE != 1 && !full) {
        const uint32_t hw = __float_as_uint(b.w);
        const float by = __half2float(__ushort_as_half((unsigned short)(hw & 0xFFFFu))) + 0.01f;
        const float bx = __half2float(__ushort_as_half((unsigned short)(hw >> 16))) + 0.01f;
        const float cl = ceilf(a.x - bx - col0), ch = floorf(a.x + bx - col0);  // columns c: |col0 + c - u| <= bx
        const float rl = ceilf(a.y - by - row0), rh = floorf(a.y + by - row0);  // rows of the strip likewise
        pmask = 0u;
        if (cl <= ch && rl <= rh && ch >= 0.f && cl <= (float)(T - 1) && rh >= 0.f && rl <= (float)(SR - 1)) {
            const uint32_t c0 = (uint32_t)fmaxf(cl, 0.f), c1 = (uint32_t)fminf(ch, (float)(T - 1));
            const uint32_t r0 = (uint32_t)fmaxf(rl, 0.f), r1 = (uint32_t)fminf(rh, (float)(SR - 1));
            const uint32_t cols = ((2u << c1) - 1u) & ~((1u << c0) - 1u);
#pragma unroll
            for (uint32_t r = 0; r < (uint32_t)SR; ++r)
                if (r >= r0 && r <= r1) pmask |= cols << (r * T);
        }
    }
    float Bc, Cc, add;
    if (MODE == 0) {
        Bc = a.w * LOG2E;
        Cc = b.x * LOG2E;
        add = (LN_ALPHA_MIN - b.y) * LOG2E;  // b.y = ln alpha* - ln theta: log2 theta
    } else {
        Bc = a.w;
        Cc = b.x;
        add = 0.f;
    }
    const float v = a.y;
    float R[2 * SR];
#pragma unroll
    for (int r = 0; r < SR; ++r) {
        const float dy = v - (row0 + (float)r);
        R[2 * r] = Bc * dy;
        R[2 * r + 1] = MODE == 0 ? fmaf(Cc * dy, dy, add) : (Cc * dy) * dy;
    }
    if (MODE == 0 && SR <= 2) {  // one float4 per row: (u, A', B' dy_r, C' dy_r^2 + log2 theta)
        const float u = a.x, Ap = a.z * LOG2E;
        a = make_float4(u, Ap, R[0], R[1]);
        if (SR == 2) b = make_float4(u, Ap, R[2 % (2 * SR)], R[3 % (2 * SR)]);
        return pmask;
    }
    const float4 X = MODE == 0 ? make_float4(a.x, a.z * LOG2E, 0.f, 0.f) : make_float4(a.x, a.z, b.y, b.z);
    a = X;
    b = make_float4(R[0], R[1], SR > 1 ? R[2 % (2 * SR)] : 0.f, SR > 1 ? R[3 % (2 * SR)] : 0.f);
    if (SR > 2) b2 = make_float4(R[4 % (2 * SR)], R[5 % (2 * SR)], R[6 % (2 * SR)], R[7 % (2 * SR)]);
    return pmask;
}

// Transpose of the 32 x 32 bit matrix held by a warp, lane l holding row l:
// afterwards lane q holds column q (bit l = bit q of lane l's row).  Five
// exchange steps, each swapping the off-diagonal blocks of half the size.
template <uint32_t J, uint32_t M>
__device__ __forceinline__ uint32_t transpose_step(uint32_t x, uint32_t lane) {
    const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, J);
    return (lane & J) ? ((x & ~M) | ((y & ~M) >> J)) : ((x & M) | ((y & M) << J));
}
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x) {
    const uint32_t lane = lane_id();
    x = transpose_step<16, 0x0000FFFFu>(x, lane);
    x = transpose_step<8, 0x00FF00FFu>(x, lane);
    x = transpose_step<4, 0x0F0F0F0Fu>(x, lane);
    x = transpose_step<2, 0x33333333u>(x, lane);
    return transpose_step<1, 0x55555555u>(x, lane);
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

// A warp's current item: where its strip reads and writes, copied from the
// view's frame parameters into shared memory when the warp takes the item and
// read from there at each use, so that neither the pointers nor the output
// location occupy registers during the walk; and the warp's blend statistics.
struct WarpItem {
    const uint32_t* pair_val;
    const float4* recA;
    const float4* recB;
    const float4* rgb;
    float* image;
    float* host_image;
    Counters* ctr;           // statistics of the view below
    unsigned long long evals, contribs;
    uint32_t at;             // index of the strip's first pixel
    uint32_t width;          // image width
    uint32_t nx, ny;         // columns and rows of the strip inside the image
    uint32_t view;
};

// The blend, for tiles of T x T pixels.  A strip is SR = 32 / T rows of T
// columns (one warp, one pixel per lane); a tile has NS = T T / 32 strips.  A
// pair's 8-bit row mask has one bit per MR = max(1, T / 8) rows, and strip s
// needs the bits of its rows.  Work: a CTA claims the next tile of the work
// list from the global counter 'next'; the strips of the CTA's tiles are
// claimed by its warps from a shared counter, in (slot, strip) order.  The
// warp that takes strip 0 of a slot claims that slot's tile and publishes it
// in a ring of 4 entries; the other strips' warps wait for it.  Before it
// reuses an entry the publishing warp waits until the entry's previous readers
// have read it.  Every wait is on a claim made earlier in the CTA's order, so
// none can close a cycle; each is still bounded and reports F_SPIN_TIMEOUT.
template <int MODE, int DEPTH, int T>
__global__ void __launch_bounds__(BL_THREADS, BL_MIN_CTAS) k_blend(const FrameParams* __restrict__ fp0,
                                                                   const FrameParams* const* __restrict__ fps,
                                                                   const uint32_t* __restrict__ work,
                                                                   uint32_t n_work, uint32_t* __restrict__ next) {
    constexpr int SR = 32 / T;                    // rows per strip
    constexpr int NS = T * T / 32;                // strips per tile
    constexpr int MR = T >= 8 ? T / 8 : 1;        // rows per mask bit
    constexpr int SB = SR >= MR ? SR / MR : 1;    // mask bits of one strip
    constexpr int RV = SR > 2 ? 2 : 1;            // float4 parts of the rewritten row terms
    constexpr int NP = 2 + RV;                    // staged parts: X, colour, row terms
    constexpr int RING = 256;                     // < DEPTH queued + BL_SCAN appended never exceeds it
    static_assert(T == 8 || T == 16 || T == 32, "tile size 8, 16 or 32");
    static_assert(DEPTH % 16 == 0 && DEPTH <= 48, "staging depth: 16, 32 or 48 hits");
    static_assert(DEPTH + BL_SCAN <= RING, "ring too small");
    pdl_wait();
    // [buffer][part: 0 = record A / X, 1 = colour, 2.. = record B / row terms][warp][slot]
    __shared__ __align__(16) float4 sbuf[2][NP][BL_WARPS][DEPTH];
    __shared__ uint32_t s_ring[BL_WARPS][RING];  // per-warp queue of hit pair values
    __shared__ float s_lut[MODE == 2 ? 260 : 1];
    __shared__ WarpItem s_item[BL_WARPS];
    __shared__ uint32_t s_pm[BL_WARPS][DEPTH];   // staged records' pixel masks
    __shared__ __align__(16) float s_px[BL_WARPS][96];  // a finished strip's pixels, RGB
    __shared__ uint32_t s_claim;                 // next (slot, strip) item of this CTA
    __shared__ uint32_t s_slot_tile[4], s_slot_tag[4], s_slot_read[4];
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t m = 0;
    float lut_scale = 0.f;
    if (threadIdx.x == 0) s_claim = 0u;
    if (threadIdx.x < 4) {
        s_slot_tag[threadIdx.x] = 0u;
        s_slot_read[threadIdx.x] = NS - 1;
    }
    if (lane == 0) {
        s_item[warp].ctr = nullptr;
        s_item[warp].evals = s_item[warp].contribs = 0ull;
        s_item[warp].view = 0xFFFFFFFFu;
    }
    if (MODE == 2) {  // the table mode runs on one view at a time
        m = fp0->lut_size;
        lut_scale = -(float)m / 5.55f;
        for (uint32_t i = threadIdx.x; i <= m; i += BL_THREADS) s_lut[i] = fp0->bl_lut[i];
    }
    __syncthreads();
    uint32_t* ring = s_ring[warp];
    volatile WarpItem& it = s_item[warp];
    const bool full_walk = (fp0->test_hooks & VGR_HOOK_FULL_STRIP_WALK) != 0u;
    volatile uint32_t* slot_tile = s_slot_tile;
    volatile uint32_t* slot_tag = s_slot_tag;
    volatile uint32_t* slot_read = s_slot_read;
    auto flush = [&]() {  // lane 0: the statistics of the warp's last view
        if (it.ctr && it.evals) {
            atomicAdd(&it.ctr->pix_evals, (unsigned long long)it.evals);
            atomicAdd(&it.ctr->pix_contribs, (unsigned long long)it.contribs);
        }
        it.evals = it.contribs = 0ull;
    };
    for (;;) {
        // ---- claim a (tile, strip) item
        uint32_t idx = 0, strip = 0;
        bool timed_out = false;
        if (lane == 0) {
            const uint32_t k = atomicAdd(&s_claim, 1u);
            const uint32_t slot = k / NS, e = slot & 3u;
            strip = k % NS;
            uint32_t spins = 0;
            if (strip == 0) {
                while (slot_read[e] < NS - 1) {  // the entry's last readers
                    if (++spins > SPIN_LIMIT) { timed_out = true; break; }
                    __nanosleep(32);
                }
                idx = atomicAdd(next, 1u);
                slot_read[e] = 0u;
                slot_tile[e] = idx;
                __threadfence_block();
                slot_tag[e] = slot + 1u;
            } else {
                while (slot_tag[e] != slot + 1u) {
                    if (++spins > SPIN_LIMIT) { timed_out = true; break; }
                    __nanosleep(32);
                }
                __threadfence_block();
                idx = slot_tile[e];
                atomicAdd(&s_slot_read[e], 1u);
            }
            if (timed_out) atomicOr(&fp0->bl_ctr->flags, F_SPIN_TIMEOUT);
        }
        idx = __shfl_sync(FULL, idx, 0);
        strip = __shfl_sync(FULL, strip, 0);
        if (__shfl_sync(FULL, (uint32_t)timed_out, 0) || idx >= n_work) break;
        uint2 rg;
        float rlo, clo;
        uint32_t wbits;
        bool inside;
        {
            const uint32_t item = work[idx];
            const uint32_t view = item >> WORK_TILE_BITS, tile = item & WORK_TILE_MASK;
            const FrameParams* fp = fps ? fps[view] : fp0;
            const uint32_t W = fp->width, H = fp->height, TW = fp->tiles_x;
            const uint32_t x0 = (tile % TW) * T, y0 = (tile / TW) * T + SR * strip;
            if (lane == 0) {
                if (view != it.view) {
                    flush();
                    it.view = view;
                    it.ctr = fp->bl_ctr;
                }
                it.pair_val = fp->bl_pair_val;
                it.recA = fp->bl_recA;
                it.recB = fp->bl_recB;
                it.rgb = fp->bl_rgb;
                it.image = fp->bl_image;
                it.host_image = fp->host_image;
                it.at = y0 * W + x0;
                it.width = W;
                it.nx = min((uint32_t)T, W - x0);
                it.ny = y0 < H ? min((uint32_t)SR, H - y0) : 0u;
            }
            rg = fp->bl_ranges[tile];
            inside = x0 + lane % T < W && y0 + lane / T < H;
            wbits = ((1u << SB) - 1u) << (SR * strip / MR);
            rlo = (float)y0 + 0.5f;  // centre of the strip's first row
            clo = (float)x0 + 0.5f;  // and column
            __syncwarp();
        }
        BlendPixel p;
        p.fxp = (float)(lane % T + it.at % it.width) + 0.5f;
        p.T = 1.f;
        p.cr = p.cg = p.cb = 0.f;
        p.contribs = 0;
        p.done = !inside;
        uint32_t evals = 0;
        // The strip's pairs (those whose row mask names its rows, in depth
        // order) pass through a ring of pair values: the range is scanned
        // BL_SCAN values at a time (loaded one batch ahead), hits are appended,
        // and records are staged DEPTH hits at a time, so staging and the walk
        // run on full chunks however sparse the strip's hits are among the
        // tile's pairs.
        uint32_t head = 0, tail = 0;
        uint32_t bp = rg.x;  // first pair value of the pending batch
        uint32_t pend[BL_SCAN / 32];
        {
            const uint32_t* pv = it.pair_val;
#pragma unroll
            for (int g = 0; g < BL_SCAN / 32; ++g) {
                const uint32_t j = bp + 32u * g + lane;
                pend[g] = j < rg.y ? pv[j] : 0u;
            }
        }
        auto refill = [&]() {
            while (tail - head < (uint32_t)DEPTH && bp < rg.y) {
#pragma unroll
                for (int g = 0; g < BL_SCAN / 32; ++g) {
                    const uint32_t v = pend[g];
                    const bool hit = (v & wbits) != 0u;  // entries past the range hold 0
                    const uint32_t hits = __ballot_sync(FULL, hit);
                    if (hit) ring[(tail + __popc(hits & lanemask_lt())) & (RING - 1)] = v;
                    tail += __popc(hits);
                }
                bp += BL_SCAN;
                const uint32_t* pv = it.pair_val;
#pragma unroll
                for (int g = 0; g < BL_SCAN / 32; ++g) {
                    const uint32_t j = bp + 32u * g + lane;
                    pend[g] = j < rg.y ? pv[j] : 0u;
                }
            }
            __syncwarp();
        };
        // stage up to DEPTH queued hits into buffer buf; returns their number
        auto issue = [&](int buf) -> uint32_t {
            const uint32_t nh = min((uint32_t)DEPTH, tail - head);
            const float4* rA = it.recA;
            const float4* rB = it.recB;
            const float4* rC = it.rgb;
#pragma unroll
            for (int q = 0; q < (DEPTH + 31) / 32; ++q) {
                const uint32_t sl = 32u * q + lane;
                if (sl < nh) {
                    const uint32_t gi = ring[(head + sl) & (RING - 1)] >> 8;
                    cp_async16(&sbuf[buf][0][warp][sl], rA + gi);
                    cp_async16(&sbuf[buf][2][warp][sl], rB + gi);
                    cp_async16(&sbuf[buf][1][warp][sl], rC + gi);
                }
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
            const float4* wC = sbuf[buf][1][warp];
            const uint32_t nh = nh_cur;
#pragma unroll
            for (int q = 0; q < (DEPTH + 31) / 32; ++q) {
                const uint32_t sl = 32u * q + lane;
                if (sl < (uint32_t)DEPTH)  // each lane its own slots; empty slots reach no pixel
                    s_pm[warp][sl] = sl < nh ? blend_prepare<MODE, SR, T>(wA[sl], sbuf[buf][2][warp][sl],
                                                                           sbuf[buf][NP - 1][warp][sl], rlo, clo,
                                                                           full_walk)
                                             : 0u;
            }
            __syncwarp();
            // the records that can reach this lane's pixel, as slot bits in
            // depth order: the transpose of the records' pixel masks
            uint32_t reach[(DEPTH + 31) / 32];
#pragma unroll
            for (int q = 0; q < (DEPTH + 31) / 32; ++q) {
                const uint32_t sl = 32u * q + lane;
                reach[q] = warp_transpose32(sl < (uint32_t)DEPTH ? s_pm[warp][sl] : 0u);
            }
            if (!p.done) {
                // this lane's row r = lane / T.  Exact mode with strips of one or two
                // rows: the row's whole record is the float4 of part 0 (row 0) or 2
                // (row 1), one load per evaluation.  Otherwise X of part 0 and the
                // row's terms: float2 (r & 1) of part 2 + r / 2.
                const uint32_t r = lane / T;
                const float4* wY = sbuf[buf][r == 0 ? 0 : 2][warp];
                const float2* wR = reinterpret_cast<const float2*>(sbuf[buf][2 + r / 2][warp]) + (r & 1u);
                auto eval = [&](uint32_t i, float4& X) -> float {
                    if constexpr (MODE == 0 && SR <= 2) {
                        X = wY[i];
                        const float dx = X.x - p.fxp;
                        return fmaf(fmaf(X.y, dx, X.z), dx, X.w);
                    } else {
                        X = load_x<MODE>(wA, i);
                        return blend_rho(p, X, wR[2 * i]);
                    }
                };
#pragma unroll
                for (int q = 0; q < (DEPTH + 31) / 32; ++q) {
                    uint32_t mm = reach[q];
                    while (mm != 0u) {  // two records at a time for instruction-level parallelism
                        const uint32_t i0 = 32u * q + __ffs(mm) - 1u;
                        mm &= mm - 1u;
                        const bool two = mm != 0u;
                        const uint32_t i1 = two ? 32u * q + __ffs(mm) - 1u : i0;
                        mm &= mm - 1u;
                        float4 X0, X1;
                        const float r0 = eval(i0, X0), r1 = eval(i1, X1);
                        ++evals;
                        if (!blend_step<MODE>(p, X0, wC, i0, r0, s_lut, m, lut_scale)) break;
                        if (two) {
                            ++evals;
                            if (!blend_step<MODE>(p, X1, wC, i1, r1, s_lut, m, lut_scale)) break;
                        }
                    }
                    if (p.done) break;
                }
            }
            __syncwarp();  // the walk is done with this buffer before it is refilled
            buf ^= 1;
            nh_cur = nh_next;
        }
        cp_async_wait<0>();  // the chunk staged ahead, if the strip stopped early
        const uint32_t cx = lane % T, cy = lane / T;
        float* const host_image = it.host_image;
        // a whole strip whose rows start 16-byte aligned (image width a multiple of
        // 4): its 32 pixels staged in shared memory and stored as float4, SR rows
        // of 3T/4 float4 each (long aligned bursts over the host link)
        const bool whole = it.nx == (uint32_t)T && it.ny == (uint32_t)SR && (it.width & 3u) == 0u &&
                           ((reinterpret_cast<uintptr_t>(host_image) & 15u) == 0u);
        if (whole) {
            float* s = s_px[warp];
            s[3 * lane + 0] = p.cr;
            s[3 * lane + 1] = p.cg;
            s[3 * lane + 2] = p.cb;
            __syncwarp();
            constexpr int F4_ROW = 3 * T / 4;
            if (lane < 24) {  // 96 floats = 24 float4
                const uint32_t r = lane / F4_ROW, c4 = lane % F4_ROW;
                const float4 val = reinterpret_cast<const float4*>(s)[lane];
                const size_t at4 = ((size_t)it.at + (size_t)r * it.width) * 3 + 4u * c4;
                *reinterpret_cast<float4*>(it.image + at4) = val;
                if (host_image) *reinterpret_cast<float4*>(host_image + at4) = val;  // pinned host buffer
            }
            __syncwarp();
        } else if (cx < it.nx && cy < it.ny) {
            const size_t at = ((size_t)it.at + (size_t)cy * it.width + cx) * 3;
            float* o = it.image + at;
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
        const uint32_t ev_w = __reduce_add_sync(FULL, evals), co_w = __reduce_add_sync(FULL, p.contribs);
        if (lane == 0) {
            it.evals = it.evals + ev_w;
            it.contribs = it.contribs + co_w;
        }
        __syncwarp();  // every lane is done with the item before lane 0 rewrites it
    }
    if (lane == 0) flush();
}

template <int MODE, int DEPTH, int T>
void launch_blend_t(const FrameParams* fp0, const FrameParams* const* fps, const uint32_t* work, uint32_t n_work,
                    uint32_t* next, int grid, cudaStream_t s) {
    launch_k(k_blend<MODE, DEPTH, T>, grid, BL_THREADS, s, fp0, fps, work, n_work, next);
}

// The default mode at every (depth, tile) of the tuner; the canonical and
// table modes at depth 32.
template <int T>
void launch_blend_tile(const FrameParams* fp0, const FrameParams* const* fps, const uint32_t* work, uint32_t n_work,
                       uint32_t* next, int grid, uint32_t filter, uint32_t exp_mode, uint32_t depth, cudaStream_t s) {
    if (filter == VGR_FILTER_CANONICAL) launch_blend_t<1, 32, T>(fp0, fps, work, n_work, next, grid, s);
    else if (exp_mode == VGR_EXP_LUT) launch_blend_t<2, 32, T>(fp0, fps, work, n_work, next, grid, s);
    else if (depth == 16) launch_blend_t<0, 16, T>(fp0, fps, work, n_work, next, grid, s);
    else if (depth == 48 && T != 8) launch_blend_t<0, (T != 8 ? 48 : 32), T>(fp0, fps, work, n_work, next, grid, s);
    else launch_blend_t<0, 32, T>(fp0, fps, work, n_work, next, grid, s);
}

template <int MODE, int DEPTH, int T>
int occupancy() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_blend<MODE, DEPTH, T>, BL_THREADS, 0);
    return n > 0 ? n : 1;
}

int blend_ctas_per_sm(uint32_t filter, uint32_t exp_mode, uint32_t depth, uint32_t tile) {
    // [mode][depth][tile], queried once each
    static int cache[3][3][3] = {};
    const int md = filter == VGR_FILTER_CANONICAL ? 1 : exp_mode == VGR_EXP_LUT ? 2 : 0;
    const int d = md != 0 ? 1 : depth == 16 ? 0 : (depth == 48 && tile != 8) ? 2 : 1;
    const int t = tile == 8 ? 0 : tile == 32 ? 2 : 1;
    int& c = cache[md][d][t];
    if (!c) {
        switch (md * 9 + d * 3 + t) {
            case 0: c = occupancy<0, 16, 8>(); break;
            case 1: c = occupancy<0, 16, 16>(); break;
            case 2: c = occupancy<0, 16, 32>(); break;
            case 3: c = occupancy<0, 32, 8>(); break;
            case 4: c = occupancy<0, 32, 16>(); break;
            case 5: c = occupancy<0, 32, 32>(); break;
            case 7: c = occupancy<0, 48, 16>(); break;
            case 8: c = occupancy<0, 48, 32>(); break;
            case 12: c = occupancy<1, 32, 8>(); break;
            case 13: c = occupancy<1, 32, 16>(); break;
            case 14: c = occupancy<1, 32, 32>(); break;
            case 21: c = occupancy<2, 32, 8>(); break;
            case 22: c = occupancy<2, 32, 16>(); break;
            case 23: c = occupancy<2, 32, 32>(); break;
            default: c = 1; break;
        }
    }
    return c;
}

void launch_blend(const FrameParams* fp0, const FrameParams* const* fps, const uint32_t* work, uint32_t n_work,
                  uint32_t* next, int grid, uint32_t filter, uint32_t exp_mode, uint32_t depth, uint32_t tile,
                  cudaStream_t s) {
    if (tile == 8) launch_blend_tile<8>(fp0, fps, work, n_work, next, grid, filter, exp_mode, depth, s);
    else if (tile == 32) launch_blend_tile<32>(fp0, fps, work, n_work, next, grid, filter, exp_mode, depth, s);
    else launch_blend_tile<16>(fp0, fps, work, n_work, next, grid, filter, exp_mode, depth, s);
}

}  // namespace vgr
