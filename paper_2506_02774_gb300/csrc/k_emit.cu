// k_emit.cu -- emission of the kept (tile, Gaussian) pairs in depth order,
// and the per-tile ranges of the sorted pair list.
//
// Visible Gaussians are visited in depth order (the output of the depth
// sort).  Each one's kept-tile count (from preprocess) is scanned across the
// whole list with a decoupled look-back, giving every Gaussian its run of
// pair slots; the tile-level preemptive test (Sec. 4.2, Eq. 4) is re-run with
// the same rounded intrinsics, so exactly the counted tiles are written.  The
// pair value is the Gaussian's depth rank; its record (mean, conic,
// threshold, opacity, colour) is copied to rank order so the blend reads
// records of a tile in increasing address order.  The digit histograms of
// the following tile sort are accumulated here as well.
#include "vgr_internal.cuh"
#include "vgr_launch.h"
#include "vgr_tiletest.cuh"

namespace vgr {

constexpr int EM_THREADS = 256;
constexpr uint32_t EM_COOP_MIN_AREA = 8;

uint32_t emit_tile() { return EM_THREADS; }

__global__ void __launch_bounds__(EM_THREADS) k_emit(const uint32_t* __restrict__ order, uint32_t cap_vis,
                                                     VisBuffers vis, float4* __restrict__ srecA,
                                                     float4* __restrict__ srecB, float2* __restrict__ srecC,
                                                     uint32_t* __restrict__ pair_key, uint32_t* __restrict__ pair_val,
                                                     uint64_t cap, int tile_passes,
                                                     unsigned long long* __restrict__ status,
                                                     Counters* __restrict__ ctr, const FrameParams* __restrict__ fp) {
    __shared__ uint32_t s_scan[9];
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ uint32_t s_hist[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&s_hist[0][0])[i] = 0u;
    const uint32_t n_vis = min(ctr->n_vis, cap_vis);
    const uint32_t ntiles = (n_vis + EM_THREADS - 1) / EM_THREADS;
    const uint32_t epoch = fp->epoch;
    const uint32_t TW = fp->tiles_x;
    const float Wf = fp->width_f, Hf = fp->height_f;
    const bool canonical = fp->filter == VGR_FILTER_CANONICAL;
    const uint32_t lane = lane_id();
    __syncthreads();

    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&ctr->tickets[TK_EMIT], 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t r = tile * EM_THREADS + threadIdx.x;
        const bool valid = r < n_vis;
        uint32_t nt = 0;
        uint2 rect = make_uint2(0u, 0u);
        float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A;
        if (valid) {
            const uint32_t vi = order[r];
            nt = vis.ntile[vi];
            rect = vis.rect[vi];
            A = vis.recA[vi];
            B = vis.recB[vi];
            const float2 C = vis.recC[vi];
            srecA[r] = A;
            srecB[r] = B;
            srecC[r] = C;
        }
        uint32_t total;
        const uint32_t excl = block_excl_scan<EM_THREADS / 32>(nt, s_scan, &total);
        if (threadIdx.x == 0) s_prefix = lookback(status, 1, tile, total, epoch, &ctr->flags);
        __syncthreads();
        const uint64_t off = (uint64_t)s_prefix + excl;

        const int tx0 = (int)(rect.x & 0xFFFFu), ty0 = (int)(rect.x >> 16);
        const int tx1 = (int)(rect.y & 0xFFFFu), ty1 = (int)(rect.y >> 16);
        const uint32_t wdt = nt ? (uint32_t)(tx1 - tx0 + 1) : 0u;
        const uint32_t area = nt ? wdt * (uint32_t)(ty1 - ty0 + 1) : 0u;
        // the conic is stored pre-scaled (A = -a/2, B = -b, C = -c/2): exact to undo
        const float ca = -2.0f * A.z, cb = -A.w, cc = -2.0f * B.x;
        const float rx = nt ? __fdiv_rn(-cb, ca) : 0.f, ry = nt ? __fdiv_rn(-cb, cc) : 0.f;
        const float thre = B.y - TILE_EPS;
        const bool coop = !canonical && area > EM_COOP_MIN_AREA;
        if (nt && !coop) {
            uint64_t o = off;
            const uint64_t oend = off + nt;
            for (int ty = ty0; ty <= ty1; ++ty)
                for (int tx = tx0; tx <= tx1; ++tx) {
                    if (!canonical && !tile_keep(A.x, A.y, ca, cb, cc, rx, ry, thre, tx, ty, Wf, Hf)) continue;
                    if (o < oend && o < cap) {
                        const uint32_t key = (uint32_t)ty * TW + (uint32_t)tx;
                        pair_key[o] = key;
                        pair_val[o] = r;
                        for (int p = 0; p < tile_passes; ++p) atomicAdd(&s_hist[p][(key >> (8 * p)) & 255u], 1u);
                    }
                    ++o;
                }
        }
        uint32_t mask = __ballot_sync(0xFFFFFFFFu, coop);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1u;
            const float su = __shfl_sync(0xFFFFFFFFu, A.x, src), sv = __shfl_sync(0xFFFFFFFFu, A.y, src);
            const float sa = __shfl_sync(0xFFFFFFFFu, ca, src), sb = __shfl_sync(0xFFFFFFFFu, cb, src);
            const float sc_ = __shfl_sync(0xFFFFFFFFu, cc, src), srx = __shfl_sync(0xFFFFFFFFu, rx, src);
            const float sry = __shfl_sync(0xFFFFFFFFu, ry, src), sth = __shfl_sync(0xFFFFFFFFu, thre, src);
            const int stx0 = __shfl_sync(0xFFFFFFFFu, tx0, src), sty0 = __shfl_sync(0xFFFFFFFFu, ty0, src);
            const uint32_t sw = __shfl_sync(0xFFFFFFFFu, wdt, src), sarea = __shfl_sync(0xFFFFFFFFu, area, src);
            const uint32_t snt = __shfl_sync(0xFFFFFFFFu, nt, src);
            const uint64_t soff = __shfl_sync(0xFFFFFFFFu, off, src);
            const uint32_t sr = __shfl_sync(0xFFFFFFFFu, r, src);
            uint64_t o = soff;
            for (uint32_t j0 = 0; j0 < sarea; j0 += 32u) {
                const uint32_t j = j0 + lane;
                const int tx = stx0 + (int)(j % sw), ty = sty0 + (int)(j / sw);
                const bool keep = j < sarea && tile_keep(su, sv, sa, sb, sc_, srx, sry, sth, tx, ty, Wf, Hf);
                const uint32_t kb = __ballot_sync(0xFFFFFFFFu, keep);
                if (keep) {
                    const uint64_t pos = o + __popc(kb & lanemask_lt());
                    if (pos < soff + snt && pos < cap) {
                        const uint32_t key = (uint32_t)ty * TW + (uint32_t)tx;
                        pair_key[pos] = key;
                        pair_val[pos] = sr;
                        for (int p = 0; p < tile_passes; ++p) atomicAdd(&s_hist[p][(key >> (8 * p)) & 255u], 1u);
                    }
                }
                o += __popc(kb);
            }
        }
        if (tile == ntiles - 1 && threadIdx.x == 0) {
            const uint64_t np = (uint64_t)s_prefix + total;
            ctr->n_pairs = np;
            if (np > cap) atomicOr(&ctr->flags, F_OVF_PAIRS);
        }
        __syncthreads();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < tile_passes * 256; i += blockDim.x) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&ctr->tile_hist[0][0] + i, c);
    }
}

void launch_emit(const uint32_t* order, uint32_t cap_vis, VisBuffers vis, float4* srecA, float4* srecB,
                 float2* srecC, uint32_t* pair_key, uint32_t* pair_val, uint64_t cap_pairs, int tile_passes,
                 unsigned long long* status, Counters* ctr, const FrameParams* fp, int grid, cudaStream_t s) {
    k_emit<<<grid, EM_THREADS, 0, s>>>(order, cap_vis, vis, srecA, srecB, srecC, pair_key, pair_val, cap_pairs,
                                       tile_passes, status, ctr, fp);
}

__global__ void k_ranges(const uint32_t* __restrict__ keys, const Counters* __restrict__ ctr, uint64_t cap,
                         uint2* __restrict__ ranges) {
    uint64_t n64 = ctr->n_pairs;
    if (n64 > cap) n64 = cap;
    const uint32_t n = (uint32_t)n64;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t t = keys[i];
        if (i == 0 || keys[i - 1] != t) ranges[t].x = i;
        if (i == n - 1 || keys[i + 1] != t) ranges[t].y = i + 1;
    }
}

void launch_ranges(const uint32_t* keys, const Counters* ctr, uint64_t cap_pairs, uint2* ranges, int grid,
                   cudaStream_t s) {
    k_ranges<<<grid, 256, 0, s>>>(keys, ctr, cap_pairs, ranges);
}

}  // namespace vgr
