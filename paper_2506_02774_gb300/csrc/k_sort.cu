// k_sort.cu -- stable LSD radix sort of (u32 key, u32 value) pairs, 8-bit
// digits, one kernel per digit pass ("onesweep": every tile ranks its keys
// locally, publishes its per-digit counts and finds its global offsets by a
// decoupled look-back over earlier tiles), plus an upfront histogram kernel
// giving each pass its digit totals.
//
// Used twice per frame (paper Sec. 3.1 'Sorting'): depth keys of the visible
// Gaussians (4 passes; equal depths keep their ascending node-id order), then
// tile ids of the kept pairs (2 passes at 1080p), which yields the
// (tile, depth, node id) order with nothing but stable passes.
#include "vgr_internal.cuh"
#include "vgr_launch.h"

namespace vgr {

constexpr int RS_THREADS = RADIX_THREADS;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = RADIX_ITEMS;
constexpr int RS_TILE = RADIX_TILE;  // 3840 keys per tile
constexpr int RS_BINS = 256;

uint32_t radix_tile() { return RS_TILE; }

// Digit histograms of up to 4 passes (shift 0, 8, 16, 24), aggregated per
// warp with match_any before the shared-memory atomics.
__global__ void __launch_bounds__(256) k_radix_hist(const uint32_t* __restrict__ keys,
                                                    const uint32_t* __restrict__ n32,
                                                    const unsigned long long* __restrict__ n64, uint64_t cap,
                                                    int passes, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[4][RS_BINS];
    for (int i = threadIdx.x; i < 4 * RS_BINS; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    uint64_t nv = n32 ? (uint64_t)*n32 : (uint64_t)*n64;
    if (nv > cap) nv = cap;
    const uint32_t n = (uint32_t)nv;
    const uint32_t lane = lane_id();
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n; base += stride) {
        const uint32_t i = base + lane;
        const bool valid = i < n;
        const uint32_t k = valid ? keys[i] : 0u;
        for (int p = 0; p < passes; ++p) {
            const uint32_t d = valid ? ((k >> (8 * p)) & 255u) : 256u;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            if (valid && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&h[p][d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RS_BINS; i += blockDim.x) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// One digit pass.  n comes from n32 (if non-null) or n64, clamped to cap.
__global__ void __launch_bounds__(RS_THREADS) k_radix_pass(const uint32_t* __restrict__ keys_in,
                                                           const uint32_t* __restrict__ vals_in,
                                                           uint32_t* __restrict__ keys_out,
                                                           uint32_t* __restrict__ vals_out,
                                                           const uint32_t* __restrict__ n32,
                                                           const unsigned long long* __restrict__ n64, uint64_t cap,
                                                           int shift, const uint32_t* __restrict__ hist,
                                                           unsigned long long* __restrict__ status,
                                                           uint32_t* __restrict__ ticket,
                                                           const FrameParams* __restrict__ fp,
                                                           Counters* __restrict__ ctr) {
    __shared__ uint32_t s_wh[RS_WARPS][RS_BINS];  // per-warp counts, then per-warp offsets
    __shared__ uint32_t s_gbase[RS_BINS];         // global start of each digit
    __shared__ uint32_t s_off[RS_BINS];           // start of this tile's run of each digit
    __shared__ uint32_t s_tile;
    uint64_t n64v = n32 ? (uint64_t)*n32 : (uint64_t)*n64;
    if (n64v > cap) n64v = cap;
    const uint32_t n = (uint32_t)n64v;
    const uint32_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    const uint32_t epoch = fp->epoch;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;

    // exclusive scan of the digit totals (thread t owns digit t)
    {
        const uint32_t c = hist[threadIdx.x];
        uint32_t total;
        __shared__ uint32_t s_scan[RS_WARPS + 1];
        s_gbase[threadIdx.x] = block_excl_scan<RS_WARPS>(c, s_scan, &total);
    }
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
        for (int w = 0; w < RS_WARPS; ++w) s_wh[w][threadIdx.x] = 0u;
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;

        uint32_t key[RS_ITEMS], val[RS_ITEMS], rank[RS_ITEMS];
        const uint32_t base = tile * RS_TILE + warp * (32 * RS_ITEMS) + lane;
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            const uint32_t idx = base + it * 32;
            const bool valid = idx < n;
            key[it] = valid ? keys_in[idx] : 0xFFFFFFFFu;
            val[it] = valid ? (vals_in ? vals_in[idx] : idx) : 0u;
        }
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            const uint32_t idx = base + it * 32;
            const bool valid = idx < n;
            const uint32_t d = valid ? ((key[it] >> shift) & 255u) : 256u;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            uint32_t r = 0;
            if (valid) r = s_wh[warp][d] + __popc(peers & lanemask_lt());
            __syncwarp();
            if (valid && lane == (uint32_t)(__ffs(peers) - 1)) s_wh[warp][d] += __popc(peers);
            __syncwarp();
            rank[it] = r;
        }
        __syncthreads();
        // digit t: offsets of each warp's run and the tile total
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t c = s_wh[w][threadIdx.x];
            s_wh[w][threadIdx.x] = run;
            run += c;
        }
        const uint32_t prefix = lookback(status + (size_t)threadIdx.x, RS_BINS, tile, run, epoch, &ctr->flags);
        s_off[threadIdx.x] = s_gbase[threadIdx.x] + prefix;
        __syncthreads();
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            const uint32_t idx = base + it * 32;
            if (idx < n) {
                const uint32_t d = (key[it] >> shift) & 255u;
                const uint32_t pos = s_off[d] + s_wh[warp][d] + rank[it];
                if (pos < n) {
                    keys_out[pos] = key[it];
                    vals_out[pos] = val[it];
                }
            }
        }
        __syncthreads();
    }
}

void launch_radix_hist(const uint32_t* keys, const uint32_t* n32, const unsigned long long* n64, uint64_t cap,
                       int passes, uint32_t* hist, int grid, cudaStream_t s) {
    k_radix_hist<<<grid, 256, 0, s>>>(keys, n32, n64, cap, passes, hist);
}

void launch_radix_pass(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                       const uint32_t* n32, const unsigned long long* n64, uint64_t cap, int shift,
                       const uint32_t* hist, unsigned long long* status, uint32_t* ticket, const FrameParams* fp,
                       Counters* ctr, int grid, cudaStream_t s) {
    k_radix_pass<<<grid, RS_THREADS, 0, s>>>(keys_in, vals_in, keys_out, vals_out, n32, n64, cap, shift, hist,
                                             status, ticket, fp, ctr);
}

}  // namespace vgr
