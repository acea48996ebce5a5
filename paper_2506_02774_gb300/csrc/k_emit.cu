// k_emit.cu -- emission of (tile, Gaussian) pairs in depth order with the
// tile-level preemptive alpha test, and the blend's tile order (which also
// finishes the per-tile ranges the last tile-sort pass records).
//
// Two kernels.  k_slot_scan gives every visible Gaussian, in depth order (the
// output of the depth sort), the first of its pair slots: an exclusive scan of
// the candidate-tile counts by decoupled look-back over tiles of 4096, whose
// per-tile work is light, so the chain of tiles moves fast.  k_emit then takes
// 512 Gaussians per CTA tile with no ticket and no look-back (their slot range
// is known): it gathers their records, and walks the tile's slots with all 256
// threads (slot -> Gaussian by a search over the CTA's offsets in shared
// memory), so a Gaussian with thousands of candidate tiles costs no more per
// thread than one with a single tile.  For each slot the tile-level form of
// Eq. 4 (paper Sec. 4.2) decides: a kept slot gets key = tile id, a dropped one
// the sentinel key, which the stable tile sort moves behind every real pair
// (which stay in depth order within a tile, the sort being stable).  The slot's
// value is the Gaussian's index in the in-front arrays << 8 | its row mask in
// that tile: bit w is set when the footprint box reaches one of the tile's
// pixel rows w MR .. w MR + MR - 1, MR = tile / 8 rows (1 for 8-pixel tiles);
// outside the box the Eq. 4 test fails at every pixel, so the blend reads only
// the records a strip needs, straight from the in-front arrays.  Indices
// therefore take 24 bits: a frame with more cut nodes in front of the camera
// reports an overflow.  The digit histograms of the tile sort are accumulated
// here as well.
#include <cuda_fp16.h>

#include "vgr_internal.cuh"
#include "vgr_launch.h"
#include "vgr_tiletest.cuh"

namespace vgr {

constexpr int EM_THREADS = 256;
constexpr int EM_ITEMS = 2;
constexpr int EM_TILE = EM_THREADS * EM_ITEMS;  // Gaussians per CTA tile
static_assert(EM_TILE == 512, "the owner search takes two ballots over 32 x 16 Gaussians");

uint32_t emit_tile() { return EM_TILE; }

constexpr int SS_THREADS = 256;
constexpr int SS_ITEMS = 16;
constexpr int SS_TILE = SS_THREADS * SS_ITEMS;  // Gaussians per look-back tile of the slot scan

uint32_t slot_scan_tile() { return SS_TILE; }

// off[r] = candidate slots of the Gaussians of depth rank < r (r <= n_vis);
// off[n_vis] is the frame's candidate-slot count.
__global__ void __launch_bounds__(SS_THREADS) k_slot_scan(const uint32_t* __restrict__ order, uint32_t cap_vis,
                                                          const uint32_t* __restrict__ ntile,
                                                          uint32_t* __restrict__ off, uint64_t cap_pairs,
                                                          unsigned long long* __restrict__ status,
                                                          Counters* __restrict__ ctr,
                                                          const FrameParams* __restrict__ fp) {
    pdl_wait();
    __shared__ uint32_t s_scan[9];
    __shared__ uint32_t s_tile, s_prefix;
    const uint32_t n_vis = min(ctr->n_vis, cap_vis);
    const uint32_t ntiles = (n_vis + SS_TILE - 1) / SS_TILE;
    const uint32_t epoch = fp->epoch;
    if (blockIdx.x == 0 && threadIdx.x == 0 && ctr->n_front > MAX_RANKS) atomicOr(&ctr->flags, F_OVF_VIS);
    if (n_vis == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            off[0] = 0u;
            ctr->n_cand = 0ull;
        }
        return;
    }
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&ctr->tickets[TK_EMIT], 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        // thread t owns ranks tile * SS_TILE + SS_ITEMS t .. + SS_ITEMS - 1 (gathers in flight together)
        const uint32_t r0 = tile * SS_TILE + SS_ITEMS * threadIdx.x;
        uint32_t c[SS_ITEMS], vi[SS_ITEMS];
#pragma unroll
        for (int k = 0; k < SS_ITEMS; ++k) vi[k] = r0 + k < n_vis ? order[r0 + k] : NONE;
#pragma unroll
        for (int k = 0; k < SS_ITEMS; ++k) c[k] = vi[k] != NONE ? ntile[vi[k]] : 0u;
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < SS_ITEMS; ++k) sum += c[k];
        uint32_t total;
        uint32_t run = block_excl_scan<SS_THREADS / 32>(sum, s_scan, &total);
        if (threadIdx.x < 32) {
            // (test hook: tile 0 stays silent, so the others' bounded waits run out)
            const bool silent = tile == 0 && (fp->test_hooks & VGR_HOOK_WITHHOLD_LOOKBACK);
            const uint32_t pre = silent ? 0u : lookback_warp(status, 1, tile, total, epoch, &ctr->flags);
            if (threadIdx.x == 0) s_prefix = pre;
        }
        __syncthreads();
        run += s_prefix;
#pragma unroll
        for (int k = 0; k < SS_ITEMS; ++k) {
            if (r0 + k < n_vis) off[r0 + k] = run;
            run += c[k];
        }
        if (tile == ntiles - 1 && threadIdx.x == 0) {
            const uint64_t ns = (uint64_t)s_prefix + total;
            off[n_vis] = (uint32_t)ns;
            ctr->n_cand = ns;
            if (ns > cap_pairs) atomicOr(&ctr->flags, F_OVF_PAIRS);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(EM_THREADS, 4) k_emit(const uint32_t* __restrict__ order, uint32_t cap_vis,
                                                     VisBuffers vis, const uint32_t* __restrict__ slot_off,
                                                     uint32_t* __restrict__ pair_key,
                                                     uint32_t* __restrict__ pair_val, uint64_t cap, int tile_passes,
                                                     uint32_t sentinel, Counters* __restrict__ ctr,
                                                     const FrameParams* __restrict__ fp) {
    pdl_wait();
    __shared__ uint32_t s_off[EM_TILE + 1];   // exclusive slot offsets within the CTA tile, then its total
    __shared__ float4 s_g[EM_TILE];           // u v a b
    __shared__ float4 s_h[EM_TILE];           // c rx ry thre
    __shared__ uint32_t s_rect[EM_TILE];      // x0 | y0 << 10 | width << 20 (tiles; 16384-px images: < 2^10)
    __shared__ __half s_hh[EM_TILE];          // footprint half-height, rounded up
    __shared__ uint32_t s_vi[EM_TILE];        // index in the in-front arrays
    __shared__ uint32_t s_hist[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&s_hist[0][0])[i] = 0u;
    const uint32_t n_vis = min(ctr->n_vis, cap_vis);
    const uint32_t ntiles = (n_vis + EM_TILE - 1) / EM_TILE;
    const uint32_t TW = fp->tiles_x;
    const int T = (int)fp->tile;
    const int MR = T >= 8 ? T / 8 : 1;  // tile rows per row-mask bit (8 bits)
    const float Wf = fp->width_f, Hf = fp->height_f;
    const bool canonical = fp->filter == VGR_FILTER_CANONICAL;
    uint32_t kept = 0;
    __shared__ uint32_t s_tile;
    __syncthreads();

    for (;;) {
        // tiles are claimed in order as CTAs free up: their slot counts vary widely
        if (threadIdx.x == 0) s_tile = atomicAdd(&ctr->tickets[TK_PRE], 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t g0 = tile * EM_TILE;
        const uint32_t base32 = slot_off[g0];
        // gather EM_ITEMS Gaussians per thread (independent loads in flight)
#pragma unroll
        for (int k = 0; k < EM_ITEMS; ++k) {
            const uint32_t q = k * EM_THREADS + threadIdx.x;  // position in depth order within the CTA tile
            const uint32_t r = g0 + q;
            if (r < n_vis) {
                const uint32_t vi = order[r];
                s_vi[q] = vi;
                const uint2 rect = vis.rect[vi];
                const float4 A = vis.recA[vi];
                const float4 B = vis.recB[vi];
                // the conic is stored pre-scaled (A = -a/2, B = -b, C = -c/2): exact to undo
                const float ca = -2.0f * A.z, cb = -A.w, cc = -2.0f * B.x;
                s_g[q] = make_float4(A.x, A.y, ca, cb);
                // edge optima dy* = (-b / c) dx, dx* = (-b / a) dy; an ulp or two of
                // error moves rho_max by far less than the test's 2e-3 slack
                s_h[q] = make_float4(cc, __fdividef(-cb, ca), __fdividef(-cb, cc), B.y - TILE_EPS);
                const uint32_t x0 = rect.x & 0xFFFFu, y0 = rect.x >> 16;
                s_rect[q] = x0 | (y0 << 10) | (((rect.y & 0xFFFFu) - x0 + 1u) << 20);
                s_hh[q] = __ushort_as_half((unsigned short)(__float_as_uint(B.w) & 0xFFFFu));  // half-height
            }
            // offsets within the tile; past the last Gaussian: the tile's total
            s_off[q] = slot_off[min(r, n_vis)] - base32;
        }
        if (threadIdx.x == 0) s_off[EM_TILE] = slot_off[min(g0 + EM_TILE, n_vis)] - base32;
        __syncthreads();
        const uint32_t total = s_off[EM_TILE];
        const uint64_t base = base32;
        // slots in warp-sized runs: the owner of the run's first slot by a
        // warp-wide search, the other lanes' owners by counting the
        // Gaussians that start inside the run (every visible Gaussian has at
        // least one slot, so starts are distinct)
        const uint32_t lane = lane_id();
        for (uint32_t j0 = (threadIdx.x & ~31u); j0 < total; j0 += EM_THREADS) {
            // the last Gaussian starting at or before j0 (offsets ascend, so the
            // test holds on a prefix): lane k tests Gaussian 16 k, then lanes 0..15
            // the 16 Gaussians of the last such stride -- two ballots
            const uint32_t cm = __ballot_sync(0xFFFFFFFFu, s_off[16u * lane] <= j0);  // bit 0: s_off[0] = 0
            const uint32_t kc = 31u - __clz(cm);
            const uint32_t fm = __ballot_sync(0xFFFFFFFFu, lane < 16u && s_off[16u * kc + (lane & 15u)] <= j0);
            const uint32_t lo = 16u * kc + 31u - __clz(fm);
            const uint32_t gi = lo + 1u + lane;
            const uint32_t d = (gi <= (uint32_t)EM_TILE ? s_off[gi] : 0xFFFFFFFFu) - j0;  // >= 1
            const uint32_t starts = __reduce_or_sync(0xFFFFFFFFu, d < 32u ? 1u << d : 0u);
            const uint32_t j = j0 + lane;
            const bool valid = j < total;
            const uint32_t g = lo + __popc(starts & ((2u << lane) - 1u));
            uint32_t key = 0xFFFFFFFFu;
            bool keep = false;
            uint32_t rows = 0xFFu;
            if (valid) {
                const uint32_t local = j - s_off[g];
                const uint32_t rc = s_rect[g];
                const uint32_t w = rc >> 20;
                // local / w and local % w: local < 2^20 and w <= 2^10, so (local + 1/2) / w is
                // at least 1 / 2^11 from an integer and its FP32 quotient floors exactly
                const uint32_t qy = (uint32_t)(((float)local + 0.5f) * __frcp_rn((float)w));
                const int tx = (int)(rc & 0x3FFu) + (int)(local - qy * w);
                const int ty = (int)((rc >> 10) & 0x3FFu) + (int)qy;
                keep = true;
                if (!canonical) {
                    const float4 G = s_g[g], Hh = s_h[g];
                    keep = tile_keep(G.x, G.y, G.z, G.w, Hh.x, Hh.y, Hh.z, Hh.w, tx, ty, Wf, Hf, T);
                    // tile rows r with |row0 + r - v| <= half-height, as groups of MR rows
                    const float row0 = (float)(ty * T) + 0.5f, hh = __half2float(s_hh[g]);
                    const float rlo = fmaxf(0.f, ceilf(G.y - hh - row0));
                    const float rhi = fminf((float)(T - 1), floorf(G.y + hh - row0));
                    rows = 0u;
                    if (rlo <= rhi) {
                        const uint32_t w0 = (uint32_t)rlo / MR, w1 = (uint32_t)rhi / MR;
                        rows = ((2u << w1) - 1u) & ~((1u << w0) - 1u);
                    }
                }
                key = keep ? (uint32_t)ty * TW + (uint32_t)tx : sentinel;
                kept += keep;
            }
            const uint64_t pos = base + j;
            const bool write = valid && pos < cap;
            if (write) {
                pair_key[pos] = key;
                pair_val[pos] = (s_vi[g] << 8) | rows;
                for (int p = 0; p < tile_passes; ++p) atomicAdd(&s_hist[p][(key >> (8 * p)) & 255u], 1u);
            }
        }
        __syncthreads();
    }
    const uint32_t wk = __reduce_add_sync(0xFFFFFFFFu, kept);
    if (lane_id() == 0 && wk) atomicAdd(&ctr->n_pairs, (unsigned long long)wk);
    __syncthreads();
    for (int i = threadIdx.x; i < tile_passes * 256; i += blockDim.x) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&ctr->tile_hist[0][0] + i, c);
    }
}

void launch_emit(const uint32_t* order, uint32_t cap_vis, VisBuffers vis, uint32_t* slot_off, uint32_t* pair_key,
                 uint32_t* pair_val, uint64_t cap_pairs, int tile_passes, uint32_t sentinel,
                 unsigned long long* status, Counters* ctr, const FrameParams* fp, int grid_scan, int grid,
                 cudaStream_t s) {
    launch_k(k_slot_scan, grid_scan, SS_THREADS, s, order, cap_vis, (const uint32_t*)vis.ntile, slot_off, cap_pairs,
             status, ctr, fp);
    launch_k(k_emit, grid, EM_THREADS, s, order, cap_vis, vis, (const uint32_t*)slot_off, pair_key, pair_val, cap_pairs,
             tile_passes, sentinel, ctr, fp);
}

// Blend order: tiles by descending pair count (classes of floor(log2(count+1)),
// heaviest class first), so the long tiles start in the first round and the
// short ones fill in behind them.  One CTA; the order inside a class does
// not matter (tiles are independent).  It also finishes the ranges the last
// tile-sort pass recorded as (start, ~end) by atomic minima from all ones:
// each becomes [start, end), or [0, 0) for a tile without pairs.  The class
// counts go to the frame's counters, for a batch's order over all its views.
// The few classes are counted and claimed once per run of equal classes in a
// warp (match instruction), not once per tile.
__global__ void __launch_bounds__(1024) k_tile_order(uint2* __restrict__ ranges, uint32_t n_tiles,
                                                     uint32_t* __restrict__ order, Counters* __restrict__ ctr) {
    pdl_wait();
    __shared__ uint32_t s_cnt[33], s_start[33];
    const uint32_t lane = lane_id();
    if (threadIdx.x < 33) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    for (uint32_t t0 = threadIdx.x & ~31u; t0 < n_tiles; t0 += blockDim.x) {  // warp-uniform trips
        const uint32_t t = t0 + lane;
        uint32_t cls = 64u;  // past the end: no class
        if (t < n_tiles) {
            uint2 r = ranges[t];
            r = r.x == 0xFFFFFFFFu ? make_uint2(0u, 0u) : make_uint2(r.x, ~r.y);
            ranges[t] = r;  // read back below by this same thread
            cls = 32 - __clz(r.y - r.x + 1u);
        }
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, cls);
        if (cls < 33u && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&s_cnt[cls], (uint32_t)__popc(peers));
    }
    __syncthreads();
    if (threadIdx.x < 33) ctr->tile_buckets[threadIdx.x] = s_cnt[threadIdx.x];
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 32; b >= 0; --b) { s_start[b] = run; run += s_cnt[b]; }
    }
    __syncthreads();
    for (uint32_t t0 = threadIdx.x & ~31u; t0 < n_tiles; t0 += blockDim.x) {
        const uint32_t t = t0 + lane;
        uint32_t cls = 64u;
        if (t < n_tiles) {
            const uint2 r = ranges[t];
            cls = 32 - __clz(r.y - r.x + 1u);
        }
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, cls);
        const int leader = __ffs(peers) - 1;
        uint32_t at = 0;
        if (cls < 33u && (int)lane == leader) at = atomicAdd(&s_start[cls], (uint32_t)__popc(peers));
        at = __shfl_sync(0xFFFFFFFFu, at, leader);
        if (cls < 33u) order[at + __popc(peers & lanemask_lt())] = t;
    }
}

void launch_tile_order(uint2* ranges, uint32_t n_tiles, uint32_t* order, Counters* ctr, cudaStream_t s) {
    launch_k(k_tile_order, 1, 1024, s, ranges, n_tiles, order, ctr);
}

// The blend order of a batch: the tiles of all its views by class, heaviest
// first, each view's tiles of a class in that view's own order.  Class b of
// view v starts at off(b, v) = (tiles of every view in the classes above b)
// + (class-b tiles of the views before v); within view v's own order the
// class starts at start(b, v) = (v's tiles in the classes above b), so a tile
// at position p of v's order goes to p + off(b, v) - start(b, v): one CTA
// computes that difference per (class, view), then a grid places the tiles.
constexpr uint32_t BATCH_MAX_VIEWS = 1024;

__global__ void __launch_bounds__(1024) k_batch_offsets(const FrameParams* const* __restrict__ fps, uint32_t n_views,
                                                        uint32_t* __restrict__ delta) {
    pdl_wait();
    __shared__ uint32_t s_scan[33];
    const uint32_t v = threadIdx.x;
    const Counters* c = v < n_views ? fps[v]->bl_ctr : nullptr;
    uint32_t run = 0, vstart = 0;
    for (int b = 32; b >= 0; --b) {
        const uint32_t cnt = c ? c->tile_buckets[b] : 0u;
        uint32_t total;
        const uint32_t pre = block_excl_scan<32>(cnt, s_scan, &total);
        if (c) delta[(size_t)b * n_views + v] = run + pre - vstart;
        vstart += cnt;
        run += total;
        __syncthreads();  // s_scan is reused by the next class
    }
}

__global__ void __launch_bounds__(256) k_batch_scatter(const FrameParams* const* __restrict__ fps, uint32_t n_views,
                                                       const uint32_t* const* __restrict__ orders,
                                                       const uint32_t* __restrict__ tile_base, uint32_t total,
                                                       const uint32_t* __restrict__ delta, uint32_t* __restrict__ work) {
    pdl_wait();
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = n_views;  // the view v with tile_base[v] <= g < tile_base[v + 1]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (tile_base[mid] <= g) lo = mid; else hi = mid;
        }
        const uint32_t v = lo, p = g - tile_base[v];
        const uint32_t t = orders[v][p];
        const uint2 r = fps[v]->bl_ranges[t];
        const uint32_t b = 32 - __clz(r.y - r.x + 1u);
        work[p + delta[(size_t)b * n_views + v]] = (v << 20) | t;
    }
}

void launch_batch_order(const FrameParams* const* fps, uint32_t n_views, const uint32_t* const* orders,
                        const uint32_t* tile_base, uint32_t total_tiles, uint32_t* delta, uint32_t* work, int grid,
                        cudaStream_t s) {
    launch_k(k_batch_offsets, 1, BATCH_MAX_VIEWS, s, fps, n_views, delta);
    launch_k(k_batch_scatter, grid, 256, s, fps, n_views, orders, tile_base, total_tiles, (const uint32_t*)delta, work);
}

}  // namespace vgr
