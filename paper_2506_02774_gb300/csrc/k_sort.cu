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

// Digit histograms of up to 4 passes (shift 0, 8, 16, 24): one shared-memory
// atomic per key and digit (equal digits within a warp are combined by the
// hardware), then one global atomic per nonzero bin and CTA.
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
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RS_BINS; i += blockDim.x) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// One digit pass.  n comes from n32 (if non-null) or n64, clamped to cap.
// Per tile of RS_TILE keys (warp w owns a contiguous run of 32 * RS_ITEMS):
//  1. each warp ranks its keys: peers with the same digit come from
//     the match instruction (last pass) or per-bit ballots; the run leader's shared atomicAdd on the warp's digit
//     counter returns the count of earlier keys, shuffled to the peers;
//  2. the tile's digit counts are published to the look-back words at once,
//     so later tiles rarely wait for this one;
//  3. keys and values are placed digit-sorted in shared memory (one 8-byte
//     store per element);
//  4. the look-back over earlier tiles gives each digit its global start;
//  5. every thread writes consecutive staged elements, so each digit's run
//     is stored contiguously (coalesced).
// The last pass of the tile sort also records each tile's range: a CTA's
// staged elements are in final key order and each key's run is one
// contiguous stretch of global positions, so the first and last element of
// every run it holds give atomicMin / atomicMax updates of [start, end) (the
// end kept as its complement, so both start from all ones and take a min).
// Keys >= n_ranges (dropped slots) have no range.
constexpr int LB_BATCH = 8;  // look-back words read per round trip

template <bool HW_MATCH>
__global__ void __launch_bounds__(RS_THREADS, 4) k_radix_pass(const uint32_t* __restrict__ keys_in,
                                                           const uint32_t* __restrict__ vals_in,
                                                           uint32_t* __restrict__ keys_out,
                                                           uint32_t* __restrict__ vals_out,
                                                           const uint32_t* __restrict__ n32,
                                                           const unsigned long long* __restrict__ n64, uint64_t cap,
                                                           int shift, const uint32_t* __restrict__ hist,
                                                           unsigned long long* __restrict__ status,
                                                           uint32_t* __restrict__ ticket,
                                                           const FrameParams* __restrict__ fp,
                                                           Counters* __restrict__ ctr, uint2* __restrict__ ranges,
                                                           uint32_t n_ranges) {
    pdl_wait();
    __shared__ uint32_t s_wc[RS_WARPS][RS_BINS];  // per-warp digit counts, then per-warp run offsets
    __shared__ uint32_t s_gbase[RS_BINS];         // global start of each digit (all tiles)
    __shared__ uint32_t s_lstart[RS_BINS];        // start of each digit's run in the staged tile
    __shared__ uint32_t s_gofs[RS_BINS];          // global index minus staged index, per digit
    __shared__ uint2 s_kv[RS_TILE];               // the tile staged digit-sorted: (key, value)
    __shared__ uint32_t s_scan[RS_WARPS + 1];
    __shared__ uint32_t s_tile;
    uint64_t n64v = n32 ? (uint64_t)*n32 : (uint64_t)*n64;
    if (n64v > cap) n64v = cap;
    const uint32_t n = (uint32_t)n64v;
    const uint32_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    const uint32_t epoch = fp->epoch;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    {
        uint32_t total;
        s_gbase[threadIdx.x] = block_excl_scan<RS_WARPS>(hist[threadIdx.x], s_scan, &total);
    }
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) s_wc[w][threadIdx.x] = 0u;
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t base = tile * RS_TILE + warp * (32 * RS_ITEMS) + lane;
        uint32_t key[RS_ITEMS], val[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            const uint32_t idx = base + it * 32;
            key[it] = idx < n ? keys_in[idx] : 0u;
            val[it] = idx < n ? (vals_in ? vals_in[idx] : idx) : 0u;
        }
        // 1. ranks within the warp, in (item, lane) = input order
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            const uint32_t idx = base + it * 32;
            const uint32_t d = idx < n ? ((key[it] >> shift) & 255u) : 256u;
            // the last pass (the top byte: few distinct digits per warp) by the match
            // instruction; the lower bytes (many distinct digits) by one ballot per
            // digit bit, faster there (depth keys and tile ids alike)
            const uint32_t peers = HW_MATCH ? __match_any_sync(0xFFFFFFFFu, d) : match_digit(d);
            const int leader = __ffs(peers) - 1;
            uint32_t before = 0;
            if (d < 256u && (int)lane == leader) before = atomicAdd(&s_wc[warp][d], (uint32_t)__popc(peers));
            before = __shfl_sync(0xFFFFFFFFu, before, leader);
            rank[it] = before + __popc(peers & lanemask_lt());
        }
        __syncthreads();
        // 2. digit d (thread d): per-warp run offsets, tile total, early publish
        const uint32_t d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t c = s_wc[w][d];
            s_wc[w][d] = run;
            run += c;
        }
        unsigned long long* my = status + (size_t)tile * RS_BINS + d;
        if (tile == 0) lb_store(my, lb_pack(epoch, 2u, run));
        else lb_store(my, lb_pack(epoch, 1u, run));
        {
            uint32_t total;
            s_lstart[d] = block_excl_scan<RS_WARPS>(run, s_scan, &total);
        }
        __syncthreads();
        // 3. stage digit-sorted
#pragma unroll
        for (int it = 0; it < RS_ITEMS; ++it) {
            const uint32_t idx = base + it * 32;
            if (idx < n) {
                const uint32_t dd = (key[it] >> shift) & 255u;
                const uint32_t pos = s_lstart[dd] + s_wc[warp][dd] + rank[it];
                s_kv[pos] = make_uint2(key[it], val[it]);
            }
        }
        // 4. look-back for digit d over earlier tiles (aggregate already
        // published), LB_BATCH status words per round trip: the words are
        // read together and consumed in order up to the first inclusive
        // prefix (done) or the first one not yet published (wait, retry there)
        uint32_t prefix = 0;
        if (tile > 0) {
            const uint32_t ep = epoch & 0x3FFFFFFFu;
            int64_t j = (int64_t)tile - 1;
            uint32_t spins = 0;
            for (;;) {
                unsigned long long wv[LB_BATCH];
#pragma unroll
                for (int q = 0; q < LB_BATCH; ++q)
                    wv[q] = j - q >= 0 ? lb_load(status + (size_t)(j - q) * RS_BINS + d) : 0ull;
                uint32_t consumed = 0;
                int state = 0;  // 0: all consumed, 1: inclusive prefix reached, 2: wait
#pragma unroll
                for (int q = 0; q < LB_BATCH; ++q) {
                    if (state == 0) {
                        const uint32_t wep = (uint32_t)(wv[q] >> 34), fl = (uint32_t)(wv[q] >> 32) & 3u;
                        if (wep != ep || fl == 0u) {
                            state = 2;
                        } else {
                            prefix += (uint32_t)wv[q];
                            ++consumed;
                            if (fl == 2u) state = 1;
                        }
                    }
                }
                if (state == 1) break;
                j -= consumed;  // tile 0 always holds an inclusive prefix, so j stays >= 0
                if (state == 2) {
                    if (++spins > SPIN_LIMIT) { atomicOr(&ctr->flags, F_SPIN_TIMEOUT); break; }
                    __nanosleep(20);
                }
            }
            lb_store(my, lb_pack(epoch, 2u, prefix + run));
        }
        s_gofs[d] = s_gbase[d] + prefix - s_lstart[d];
        __syncthreads();
        // 5. coalesced write of the staged tile
        const uint32_t tile_n = min((uint32_t)RS_TILE, n - tile * RS_TILE);
        for (uint32_t j0 = threadIdx.x & ~31u; j0 < tile_n; j0 += RS_THREADS) {  // warp-uniform trips
            const uint32_t j = j0 + lane;
            const bool valid = j < tile_n;
            const uint2 kv = valid ? s_kv[j] : make_uint2(0xFFFFFFFFu, 0u);
            const uint32_t pos = s_gofs[(kv.x >> shift) & 255u] + j;
            if (valid && pos < n) {
                if (keys_out) keys_out[pos] = kv.x;  // null: only the permutation is wanted
                vals_out[pos] = kv.y;
            }
            if (ranges) {  // neighbours' keys from the adjacent lanes, across warps from shared memory
                uint32_t kp = __shfl_up_sync(0xFFFFFFFFu, kv.x, 1), kn = __shfl_down_sync(0xFFFFFFFFu, kv.x, 1);
                if (lane == 0) kp = j > 0 ? s_kv[j - 1].x : ~kv.x;
                if (lane == 31) kn = j + 1 < tile_n ? s_kv[j + 1].x : ~kv.x;
                if (valid && pos < n && kv.x < n_ranges) {
                    if (kp != kv.x) atomicMin(&ranges[kv.x].x, pos);
                    if (kn != kv.x) atomicMin(&ranges[kv.x].y, ~(pos + 1u));
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
                       Counters* ctr, int grid, cudaStream_t s, int hw_match, uint2* ranges, uint32_t n_ranges) {
    if (hw_match)
        launch_k(k_radix_pass<true>, grid, RS_THREADS, s, keys_in, vals_in, keys_out, vals_out, n32,
                  n64, cap, shift, hist, status, ticket, fp, ctr, ranges, n_ranges);
    else
        launch_k(k_radix_pass<false>, grid, RS_THREADS, s, keys_in, vals_in, keys_out, vals_out, n32,
                  n64, cap, shift, hist, status, ticket, fp, ctr, ranges, n_ranges);
}

}  // namespace vgr
