// k_lod.cu -- LoD cut finding on the GPU (paper Sec. 3.1 'Cut Finding',
// Sec. 4.1 'Temporal-Aware LoD Search', Algorithm 1).
//
// The cut is written as a bitmap over node ids, then compacted into an
// ascending id list.  Two producers:
//  * k_lod_update: the temporal update.  Each node n of the previous cut
//    tests itself and its parent against the current camera:
//      parent does not expand  -> collapse: climb to the highest ancestor whose
//                                 parent expands (or the root); it joins the cut
//      n expands               -> expand: explore n's subtree depth-first;
//                                 non-expanding nodes reached join the cut
//      otherwise               -> n stays in the cut.
//    This is Algorithm 1 with single nodes in place of height-2 subtrees:
//    TOP (collapse) moves to the parent, BOTTOM (expand) to the children.
//    The result equals the top-down cut whenever the test is monotone
//    (a child expands only if its parent does), which the nested radii
//    guarantee; a violation raises F_NONMONOTONE.  A thread that would
//    explore more than the budget sets F_LOD_FALLBACK and the host redoes
//    the frame top-down.
//  * k_lod_level: one level of the from-scratch, top-down traversal (frame 0,
//    tau change, reset, fallback); frontiers are appended with one atomic per
//    warp after a warp scan of the child counts.
#include "vgr_internal.cuh"
#include "vgr_launch.h"

namespace vgr {

__global__ void __launch_bounds__(256) k_lod_update(const uint32_t* __restrict__ prev_cut,
                                                    const uint32_t* __restrict__ n_prev_p, uint32_t cap_prev,
                                                    SceneDev sc,
                                                    const FrameParams* __restrict__ fp, uint32_t* __restrict__ bitmap,
                                                    Counters* __restrict__ ctr) {
    const uint32_t n_prev = min(*n_prev_p, cap_prev);
    const float px = fp->pos[0], py = fp->pos[1], pz = fp->pos[2], k = fp->k;
    const uint32_t budget = fp->lod_budget, max_depth = fp->max_depth;
    uint32_t evals = 0, flags = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_prev; i += stride) {
        const uint32_t n = prev_cut[i];
        const bool en = lod_expand(sc.cr[n], px, py, pz, k);
        const uint32_t p = sc.parent[n];
        bool ep = true;
        ++evals;
        if (p != NONE) { ep = lod_expand(sc.cr[p], px, py, pz, k); ++evals; }
        if (!ep) {
            if (en) flags |= F_NONMONOTONE;
            // collapse: climb while the parent of a does not expand
            uint32_t a = p;
            for (uint32_t steps = 0;; ++steps) {
                const uint32_t pa = sc.parent[a];
                if (pa == NONE) break;
                ++evals;
                if (lod_expand(sc.cr[pa], px, py, pz, k)) break;
                a = pa;
                if (steps > max_depth) { flags |= F_LOD_FALLBACK; break; }
            }
            bitmap_set(bitmap, a);
        } else if (en) {
            // expand: depth-first over n's subtree, children ranges on a stack
            uint32_t nxt[MAX_TREE_DEPTH], end[MAX_TREE_DEPTH];
            const uint32_t c0 = sc.child[n];
            nxt[0] = c0 & CHILD_MASK;
            end[0] = nxt[0] + (c0 >> CHILD_SHIFT);
            int sp = 1;
            uint32_t local = 0;
            while (sp > 0) {
                if (nxt[sp - 1] == end[sp - 1]) { --sp; continue; }
                const uint32_t m = nxt[sp - 1]++;
                if (++local > budget) { flags |= F_LOD_FALLBACK; break; }
                if (lod_expand(sc.cr[m], px, py, pz, k)) {
                    if (sp == MAX_TREE_DEPTH) { flags |= F_LOD_FALLBACK; break; }
                    const uint32_t cm = sc.child[m];
                    nxt[sp] = cm & CHILD_MASK;
                    end[sp] = nxt[sp] + (cm >> CHILD_SHIFT);
                    ++sp;
                } else {
                    bitmap_set(bitmap, m);
                }
            }
            evals += local;
        } else {
            bitmap_set(bitmap, n);
        }
    }
    // one atomic per warp for the statistics
    uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, evals);
    uint32_t wflags = __reduce_or_sync(0xFFFFFFFFu, flags);
    if (lane_id() == 0) {
        if (wsum) atomicAdd(&ctr->nodes_eval, (unsigned long long)wsum);
        if (wflags) atomicOr(&ctr->flags, wflags);
    }
}

// One level of the top-down traversal.  Level 0 starts from the root.
__global__ void __launch_bounds__(256) k_lod_level(int level, const uint32_t* __restrict__ fin,
                                                   uint32_t* __restrict__ fout, uint32_t cap, SceneDev sc,
                                                   const FrameParams* __restrict__ fp,
                                                   uint32_t* __restrict__ bitmap, Counters* __restrict__ ctr) {
    const uint32_t n_in = level == 0 ? 1u : min(ctr->frontier_n[level], cap);
    uint32_t* n_out = &ctr->frontier_n[level + 1];
    const float px = fp->pos[0], py = fp->pos[1], pz = fp->pos[2], k = fp->k;
    const uint32_t lane = lane_id();
    const uint32_t warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    uint32_t evals = 0;
    for (uint32_t base = warp_global * 32u; base < n_in; base += nwarps * 32u) {
        const uint32_t i = base + lane;
        uint32_t cnt = 0, first = 0;
        if (i < n_in) {
            const uint32_t n = level == 0 ? 0u : fin[i];
            ++evals;
            if (lod_expand(sc.cr[n], px, py, pz, k)) {
                const uint32_t c = sc.child[n];
                first = c & CHILD_MASK;
                cnt = c >> CHILD_SHIFT;
            } else {
                bitmap_set(bitmap, n);
            }
        }
        uint32_t total;
        const uint32_t off = warp_excl_scan(cnt, &total);
        uint32_t basepos = 0;
        if (lane == 0 && total) basepos = atomicAdd(n_out, total);
        basepos = __shfl_sync(0xFFFFFFFFu, basepos, 0);
        for (uint32_t j = 0; j < cnt; ++j) {
            const uint32_t pos = basepos + off + j;
            if (pos < cap) fout[pos] = first + j;
            else atomicOr(&ctr->flags, F_OVF_FRONTIER);
        }
    }
    uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, evals);
    if (lane == 0 && wsum) atomicAdd(&ctr->nodes_eval, (unsigned long long)wsum);
}

// Bitmap -> ascending id list, clearing the bitmap for the next frame.
// Tiles of 256 threads x 4 words, ordered by a decoupled look-back scan.
constexpr int CC_WORDS = 4;
constexpr int CC_TILE_WORDS = 256 * CC_WORDS;

__global__ void __launch_bounds__(256) k_cut_compact(uint32_t* __restrict__ bitmap, uint32_t n_words,
                                                     uint32_t* __restrict__ cut, uint32_t cap,
                                                     uint32_t* __restrict__ n_cut_out,
                                                     unsigned long long* __restrict__ status,
                                                     Counters* __restrict__ ctr,
                                                     const FrameParams* __restrict__ fp) {
    __shared__ uint32_t s_scan[9];
    __shared__ uint32_t s_tile, s_prefix;
    const uint32_t ntiles = (n_words + CC_TILE_WORDS - 1) / CC_TILE_WORDS;
    const uint32_t epoch = fp->epoch;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&ctr->tickets[TK_COMPACT], 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t w0 = tile * CC_TILE_WORDS + threadIdx.x * CC_WORDS;
        // the bitmap is padded to a whole number of tiles
        uint4 w = *reinterpret_cast<const uint4*>(bitmap + w0);
        const uint32_t cnt = __popc(w.x) + __popc(w.y) + __popc(w.z) + __popc(w.w);
        uint32_t total;
        const uint32_t excl = block_excl_scan<8>(cnt, s_scan, &total);
        if (threadIdx.x == 0) s_prefix = lookback(status, 1, tile, total, epoch, &ctr->flags);
        __syncthreads();
        uint32_t off = s_prefix + excl;
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t x = ws[j];
            while (x) {
                const uint32_t b = __ffs(x) - 1u;
                if (off < cap) cut[off] = (w0 + j) * 32u + b;
                ++off;
                x &= x - 1u;
            }
        }
        if (cnt) *reinterpret_cast<uint4*>(bitmap + w0) = make_uint4(0u, 0u, 0u, 0u);
        if (tile == ntiles - 1 && threadIdx.x == 0) {
            const uint32_t n = s_prefix + total;
            *n_cut_out = n;
            if (n > cap) atomicOr(&ctr->flags, F_OVF_CUT);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ launchers
void launch_lod_update(const SceneDev& sc, const uint32_t* prev_cut, const uint32_t* n_prev, uint32_t cap_prev,
                       const FrameParams* fp, uint32_t* bitmap, Counters* ctr, int grid, cudaStream_t s) {
    k_lod_update<<<grid, 256, 0, s>>>(prev_cut, n_prev, cap_prev, sc, fp, bitmap, ctr);
}

void launch_lod_level(int level, const SceneDev& sc, const uint32_t* fin, uint32_t* fout, uint32_t cap,
                      const FrameParams* fp, uint32_t* bitmap, Counters* ctr, int grid, cudaStream_t s) {
    k_lod_level<<<grid, 256, 0, s>>>(level, fin, fout, cap, sc, fp, bitmap, ctr);
}

void launch_cut_compact(uint32_t* bitmap, uint32_t n_words, uint32_t* cut, uint32_t cap, uint32_t* n_cut_out,
                        unsigned long long* status, Counters* ctr, const FrameParams* fp, int grid,
                        cudaStream_t s) {
    k_cut_compact<<<grid, 256, 0, s>>>(bitmap, n_words, cut, cap, n_cut_out, status, ctr, fp);
}

uint32_t cut_compact_tiles(uint32_t n_words) { return (n_words + CC_TILE_WORDS - 1) / CC_TILE_WORDS; }
uint32_t cut_compact_tile_words() { return CC_TILE_WORDS; }

}  // namespace vgr
