// k_lod.cu -- LoD cut finding on the GPU (paper Sec. 3.1 'Cut Finding',
// Sec. 4.1 'Temporal-Aware LoD Search', Algorithm 1).
//
// The cut is written as a bitmap over node ids (plus a second bitmap of the
// cut nodes in front of the near plane), then compacted into ascending id
// lists.  Two producers:
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
//    the frame top-down.  The node's (mean, radius^2) and its parent's are
//    stored together in one 32-byte record per node (built at load), so a
//    cut node costs one sector and one round instead of waiting for the
//    parent's id first; the id itself is read only when the node collapses.
//  * k_lod_level: one level of the from-scratch, top-down traversal (frame 0,
//    tau change, reset, fallback); frontiers are appended with one atomic per
//    warp after a warp scan of the child counts.
#include "vgr_internal.cuh"
#include "vgr_launch.h"

namespace vgr {

// A cut node joins the cut bitmap, and the potentially-visible bitmap when
// its FP32 depth key is beyond the near plane (the same key and test as
// preprocess) and its footprint can reach the image.  The footprint test is
// a bound on the one preprocess applies: preprocess's box half-width is
//   bx = r sqrt(S'00) * 1.0001 + 1e-3,  r^2 = 2 (ln theta - ln alpha*) + 2 slack
//   <= 3.33 (slack included),  S'00 = m0^T S m0 + 0.3,  m0 = fx/z (R0 - tx R2),
// and |m0|^2 = (fx/z)^2 (1 + tx^2) <= (fx/z)^2 (1 + limx^2) while
// m0^T S m0 <= lambda_max(S) |m0|^2 <= L |m0|^2, L the largest absolute row
// sum of S (Gershgorin, stored per node at load); so with
//   Bx = 3.34 sqrt(L (fx/z)^2 (1 + limx^2) + 0.3) + 0.01
// a Gaussian with u + Bx < 0.5 or u - Bx > T tiles_x - 0.5 (or likewise in
// v) has no candidate tile in preprocess and can be left out here.  The
// canonical mode's 3-sigma box is bounded the same way.
// Set bit n of bm in the lanes where pred holds, one atomic per word: the
// lanes that hit the same word (the match instruction; a warp's nodes are
// few words) OR their bits together and the lowest of them stores them.
// All 32 lanes call it.
__device__ __forceinline__ void warp_bitmap_set(uint32_t* bm, uint32_t n, bool pred) {
    const uint32_t w = pred ? n >> 5 : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, w);
    const uint32_t bits = __reduce_or_sync(peers, pred ? 1u << (n & 31u) : 0u);
    if (pred && lane_id() == (uint32_t)(__ffs(peers) - 1)) atomicOr(&bm[w], bits);
}

// With weight interpolation the rendered Gaussian of a cut node n is not n's
// own: its mean lies on the segment from n's centre to its parent's and its
// covariance is a convex combination of theirs, so its largest eigenvalue is
// at most max(L_n, L_p).  When both centres are beyond the near plane the
// whole segment is, its projection is the segment between the two projected
// centres and its depth is at least the smaller of theirs: the union of the
// two boxes, widened for max(L_n, L_p) at that depth, bounds the footprint.
// A segment across the near plane is kept; one wholly behind it is dropped.
struct CutOut {
    uint32_t* cut_bm;
    uint32_t* front_bm;
    const float* lmax;
    const float4* cr;
    const uint32_t* parent;
    float R0, R1, R2, R3, R4, R5, R6, R7, R8, Cx, Cy, Cz, z_near;
    float fx, fy, cx, cy, kx, ky, umax, vmax;
    bool canonical;
    bool interp;  // weight interpolation: bound the interpolated Gaussian, not the node's own
    __device__ __forceinline__ void add(uint32_t n, float4 c) const {
        bitmap_set(cut_bm, n);
        if (visible(n, c, lmax[n])) bitmap_set(front_bm, n);
    }
    // may the Gaussian rendered for cut node n (centre c, lm = lmax[n]) reach the image?
    __device__ __forceinline__ bool visible(uint32_t n, float4 c, float lm) const {
        if (!interp) return in_front(c, lm);
        const uint32_t p = parent[n];
        if (p == NONE) return in_front(c, lm);
        return in_front_segment(c, lm, cr[p], lmax[p]);
    }
    __device__ __forceinline__ float depth(float4 c) const {
        const float dx = __fsub_rn(c.x, Cx), dy = __fsub_rn(c.y, Cy), dz = __fsub_rn(c.z, Cz);
        return __fadd_rn(__fadd_rn(__fmul_rn(R6, dx), __fmul_rn(R7, dy)), __fmul_rn(R8, dz));
    }
    __device__ __forceinline__ void project(float4 c, float z, float& u, float& v) const {
        const float dx = __fsub_rn(c.x, Cx), dy = __fsub_rn(c.y, Cy), dz = __fsub_rn(c.z, Cz);
        const float x = fmaf(R0, dx, fmaf(R1, dy, R2 * dz));
        const float y = fmaf(R3, dx, fmaf(R4, dy, R5 * dz));
        const float iz = 1.0f / z;
        u = fmaf(fx, x * iz, cx);
        v = fmaf(fy, y * iz, cy);
    }
    __device__ __forceinline__ void half_box(float lm, float z, float& bx, float& by) const {
        const float iz = 1.0f / z;
        const float t = lm * iz * iz;
        if (!canonical) {
            bx = 3.34f * sqrtf(fmaf(t, kx, 0.3f)) + 0.01f;
            by = 3.34f * sqrtf(fmaf(t, ky, 0.3f)) + 0.01f;
        } else {
            bx = by = 3.01f * sqrtf(fmaf(t, kx + ky, 1.0f)) + 1.01f;
        }
    }
    __device__ __forceinline__ bool in_front_segment(float4 cn, float lmn, float4 cp, float lmp) const {
        const float zn = depth(cn), zp = depth(cp);
        const float zeps = 1e-2f;  // far above the FP32 error of the interpolated mean's depth
        if (zn <= z_near - zeps && zp <= z_near - zeps) return false;
        if (!(zn > z_near + zeps) || !(zp > z_near + zeps)) return true;
        float un, vn, up, vp, bx, by;
        project(cn, zn, un, vn);
        project(cp, zp, up, vp);
        half_box(fmaxf(lmn, lmp), fminf(zn, zp), bx, by);
        const float ulo = fminf(un, up), uhi = fmaxf(un, up), vlo = fminf(vn, vp), vhi = fmaxf(vn, vp);
        const float su = 1e-5f * fmaxf(fabsf(ulo), fabsf(uhi)) + 1e-2f;
        const float sv = 1e-5f * fmaxf(fabsf(vlo), fabsf(vhi)) + 1e-2f;
        return !(uhi + bx < 0.5f - su || ulo - bx > umax + su || vhi + by < 0.5f - sv || vlo - by > vmax + sv);
    }
    // may node (centre c, lm = lmax[n]) reach the image in front of the near plane?
    __device__ __forceinline__ bool in_front(float4 c, float lm) const {
        const float dx = __fsub_rn(c.x, Cx), dy = __fsub_rn(c.y, Cy), dz = __fsub_rn(c.z, Cz);
        const float z = __fadd_rn(__fadd_rn(__fmul_rn(R6, dx), __fmul_rn(R7, dy)), __fmul_rn(R8, dz));
        if (!(z > z_near)) return false;
        const float x = fmaf(R0, dx, fmaf(R1, dy, R2 * dz));
        const float y = fmaf(R3, dx, fmaf(R4, dy, R5 * dz));
        const float iz = 1.0f / z;
        const float u = fmaf(fx, x * iz, cx), v = fmaf(fy, y * iz, cy);
        const float t = lm * iz * iz;
        float bx, by;
        if (!canonical) {
            bx = 3.34f * sqrtf(fmaf(t, kx, 0.3f)) + 0.01f;
            by = 3.34f * sqrtf(fmaf(t, ky, 0.3f)) + 0.01f;
        } else {
            // canonical: ceil(3 sqrt(lam)), lam <= S'00 + S'11 + 0.32 (its sqrt(max(0.1, .)) floor)
            bx = by = 3.01f * sqrtf(fmaf(t, kx + ky, 1.0f)) + 1.01f;
        }
        const float su = 1e-5f * fabsf(u) + 1e-2f, sv = 1e-5f * fabsf(v) + 1e-2f;  // FP32 slack
        return !(u + bx < 0.5f - su || u - bx > umax + su || v + by < 0.5f - sv || v - by > vmax + sv);
    }
};

template <bool IP>
__device__ __forceinline__ CutOut make_cut_out(const FrameParams* fp, const SceneDev& sc, uint32_t* cut_bm,
                                               uint32_t* front_bm) {
    CutOut o;
    o.cut_bm = cut_bm;
    o.front_bm = front_bm;
    o.lmax = sc.lmax;
    o.cr = sc.cr;
    o.parent = sc.parent;
    o.R0 = fp->R[0]; o.R1 = fp->R[1]; o.R2 = fp->R[2];
    o.R3 = fp->R[3]; o.R4 = fp->R[4]; o.R5 = fp->R[5];
    o.R6 = fp->R[6]; o.R7 = fp->R[7]; o.R8 = fp->R[8];
    o.Cx = fp->pos[0]; o.Cy = fp->pos[1]; o.Cz = fp->pos[2];
    o.z_near = fp->z_near;
    o.fx = fp->fx; o.fy = fp->fy; o.cx = fp->cx; o.cy = fp->cy;
    o.kx = fp->fx * fp->fx * (1.0f + fp->limx * fp->limx);
    o.ky = fp->fy * fp->fy * (1.0f + fp->limy * fp->limy);
    o.umax = (float)(fp->tile * fp->tiles_x) - 0.5f;
    o.vmax = (float)(fp->tile * fp->tiles_y) - 0.5f;
    o.canonical = fp->filter == VGR_FILTER_CANONICAL;
    o.interp = IP;  // a compile-time constant: the other form's code is not generated
    return o;
}

constexpr int LOD_UNROLL = 2;  // previous-cut nodes per thread and round

template <bool FR, bool IP>
__global__ void __launch_bounds__(256) k_lod_update(const uint32_t* __restrict__ prev_cut,
                                                    const uint32_t* __restrict__ n_prev_p, uint32_t cap_prev,
                                                    SceneDev sc, const FrameParams* __restrict__ fp,
                                                    uint32_t* __restrict__ bitmap, uint32_t* __restrict__ front,
                                                    Counters* __restrict__ ctr) {
    pdl_wait();
    const uint32_t n_prev = min(*n_prev_p, cap_prev);
    const float px = fp->pos[0], py = fp->pos[1], pz = fp->pos[2], k = fp->k;
    const uint32_t budget = fp->lod_budget, max_depth = fp->max_depth;
    const CutOut out = make_cut_out<IP>(fp, sc, bitmap, front);
    LodFrustum fr;
    if (FR) fr.load(fp, sc.box);
    // the granularity test, and in the frustum-aware variant the box test
    auto expand = [&](uint32_t node, float4 c) -> bool {
        if (!lod_expand(c, px, py, pz, k)) return false;
        if constexpr (FR) return fr.meets(node);
        return true;
    };
    uint32_t evals = 0, flags = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    // one previous-cut node: stay, collapse or expand
    // (a staying node is only reported: its bits are set warp-aggregated below).
    // cp is the parent's entry (w = +inf at the root); the parent's id p is
    // loaded with it by the frustum and interpolation variants (which test its
    // box or read its extent), else only when n collapses
    constexpr bool WITH_P = FR || IP;
    auto visit = [&](uint32_t n, float4 cn, uint32_t p, float4 cp) -> bool {
        const bool en = expand(n, cn);
        bool ep = true;
        ++evals;
        if (cp.w != INFINITY) { ep = expand(p, cp); ++evals; }
        if (!ep) {
            if (en) flags |= F_NONMONOTONE;
            // collapse: climb while the parent of a does not expand
            uint32_t a = WITH_P ? p : sc.parent[n];
            float4 ca = cp;
            for (uint32_t steps = 0;; ++steps) {
                const uint32_t pa = sc.parent[a];
                if (pa == NONE) break;
                ++evals;
                const float4 cpa = sc.cr[pa];
                if (expand(pa, cpa)) break;
                a = pa;
                ca = cpa;
                if (steps > max_depth) { flags |= F_LOD_FALLBACK; break; }
            }
            out.add(a, ca);
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
                const float4 cm = sc.cr[m];
                if (expand(m, cm)) {
                    if (sp == MAX_TREE_DEPTH) { flags |= F_LOD_FALLBACK; break; }
                    const uint32_t chm = sc.child[m];
                    nxt[sp] = chm & CHILD_MASK;
                    end[sp] = nxt[sp] + (chm >> CHILD_SHIFT);
                    ++sp;
                } else {
                    out.add(m, cm);
                }
            }
            evals += local;
        } else {
            return true;  // stay
        }
        return false;
    };
    // LOD_UNROLL nodes per thread and round, their loads in flight together;
    // warp-uniform rounds so the staying nodes' bits can be set per warp
    const uint32_t lane = lane_id();
    const uint32_t first = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u;
    uint32_t nx[LOD_UNROLL];  // the next round's node ids, loaded one round ahead
#pragma unroll
    for (int u = 0; u < LOD_UNROLL; ++u) {
        const uint32_t i = first + u * stride + lane;
        nx[u] = i < n_prev ? prev_cut[i] : 0u;
    }
    for (uint32_t b0 = first; b0 < n_prev; b0 += LOD_UNROLL * stride) {
        uint32_t nn[LOD_UNROLL], pp[LOD_UNROLL];
        float4 cc[LOD_UNROLL], qq[LOD_UNROLL];
        float ll[LOD_UNROLL];
        bool ok[LOD_UNROLL];
#pragma unroll
        for (int u = 0; u < LOD_UNROLL; ++u) {
            const uint32_t i = b0 + u * stride + lane;
            ok[u] = i < n_prev;
            nn[u] = nx[u];
            const uint32_t inext = i + LOD_UNROLL * stride;
            nx[u] = inext < n_prev ? prev_cut[inext] : 0u;
        }
#pragma unroll
        for (int u = 0; u < LOD_UNROLL; ++u) {
            cc[u] = sc.lodr[2 * (size_t)nn[u]];
            qq[u] = sc.lodr[2 * (size_t)nn[u] + 1];  // the parent's entry, same sector
            ll[u] = sc.lmax[nn[u]];
            pp[u] = WITH_P ? sc.parent[nn[u]] : NONE;
        }
#pragma unroll
        for (int u = 0; u < LOD_UNROLL; ++u) {
            const bool stay = ok[u] && visit(nn[u], cc[u], pp[u], qq[u]);
            warp_bitmap_set(bitmap, nn[u], stay);
            bool vis = false;
            if (stay) {
                if (!out.interp || pp[u] == NONE) vis = out.in_front(cc[u], ll[u]);
                else vis = out.in_front_segment(cc[u], ll[u], qq[u], sc.lmax[pp[u]]);
            }
            warp_bitmap_set(front, nn[u], vis);
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
template <bool FR, bool IP>
__global__ void __launch_bounds__(256) k_lod_level(int level, const uint32_t* __restrict__ fin,
                                                   uint32_t* __restrict__ fout, uint32_t cap, SceneDev sc,
                                                   const FrameParams* __restrict__ fp,
                                                   uint32_t* __restrict__ bitmap, uint32_t* __restrict__ front,
                                                   Counters* __restrict__ ctr) {
    pdl_wait();
    const uint32_t n_in = level == 0 ? 1u : min(ctr->frontier_n[level], cap);
    uint32_t* n_out = &ctr->frontier_n[level + 1];
    const float px = fp->pos[0], py = fp->pos[1], pz = fp->pos[2], k = fp->k;
    const CutOut out = make_cut_out<IP>(fp, sc, bitmap, front);
    LodFrustum fr;
    if (FR) fr.load(fp, sc.box);
    const uint32_t lane = lane_id();
    const uint32_t warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    uint32_t evals = 0;
    for (uint32_t base = warp_global * 32u; base < n_in; base += nwarps * 32u) {
        const uint32_t i = base + lane;
        uint32_t cnt = 0, first = 0, n = 0;
        bool is_cut = false, in_front = false;
        if (i < n_in) {
            n = level == 0 ? 0u : fin[i];
            const float4 cn = sc.cr[n];
            const float lm = sc.lmax[n];
            ++evals;
            if (lod_expand(cn, px, py, pz, k) && (!FR || fr.meets(n))) {
                const uint32_t c = sc.child[n];
                first = c & CHILD_MASK;
                cnt = c >> CHILD_SHIFT;
            } else {
                is_cut = true;
                in_front = out.visible(n, cn, lm);
            }
        }
        // one atomic per bitmap word and warp (a node's siblings are neighbours)
        warp_bitmap_set(bitmap, n, is_cut);
        warp_bitmap_set(front, n, in_front);
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

// Bitmaps -> ascending id lists (the cut, and its in-front part), clearing
// both bitmaps for the next frame.  Tiles of 256 threads x 4 words; two
// decoupled look-back chains (warp 0: cut, warp 1: in-front) give each tile
// its output offsets.  A warp owns 128 contiguous words of the tile and takes
// them in four rounds of 32 (lane l holds word 32 j + l of round j, so every
// load is coalesced): a shuffle scan of the words' bit counts places each
// lane's ids in the warp's staging buffer in shared memory, and the warp then
// stores the round's ids contiguously (coalesced) -- no serial per-word loop.
constexpr int CC_THREADS = 256;
constexpr int CC_WARPS = CC_THREADS / 32;
constexpr int CC_WORDS = 4;  // words per lane = rounds per warp
constexpr int CC_TILE_WORDS = CC_THREADS * CC_WORDS;

// One round of one bitmap: this lane's word `word` (index `wi`), the round's
// ids staged in `stage` (32 words x 32 bits at most) and stored from `off`.
__device__ __forceinline__ uint32_t cc_round(uint32_t word, uint32_t wi, uint32_t off, uint32_t* stage,
                                             uint32_t* out, uint32_t cap) {
    const uint32_t lane = lane_id();
    const uint32_t c = __popc(word);
    uint32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if ((int)lane >= d) incl += y;
    }
    const uint32_t n = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (n == 0u) return off;
    uint32_t p = incl - c;
    while (word) {
        stage[p++] = wi * 32u + (uint32_t)(__ffs(word) - 1);
        word &= word - 1u;
    }
    __syncwarp();
    for (uint32_t i = lane; i < n; i += 32u)
        if (off + i < cap) out[off + i] = stage[i];
    __syncwarp();  // the buffer is read before the next round writes it
    return off + n;
}

__global__ void __launch_bounds__(CC_THREADS) k_cut_compact(uint32_t* __restrict__ bitmap, uint32_t* __restrict__ front,
                                                            uint32_t n_words, uint32_t* __restrict__ cut,
                                                            uint32_t* __restrict__ front_list, uint32_t cap,
                                                            uint32_t* __restrict__ n_cut_out,
                                                            unsigned long long* __restrict__ status,
                                                            unsigned long long* __restrict__ status_front,
                                                            Counters* __restrict__ ctr,
                                                            const FrameParams* __restrict__ fp) {
    pdl_wait();
    __shared__ uint32_t s_stage[CC_WARPS][32 * 32];
    __shared__ uint32_t s_wtot[CC_WARPS];
    __shared__ uint32_t s_tile, s_prefix[2];
    const uint32_t ntiles = (n_words + CC_TILE_WORDS - 1) / CC_TILE_WORDS;
    const uint32_t epoch = fp->epoch;
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&ctr->tickets[TK_COMPACT], 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        // the bitmaps are padded to a whole number of tiles
        const uint32_t wbase = tile * CC_TILE_WORDS + warp * (32u * CC_WORDS);
        uint32_t a[CC_WORDS], b[CC_WORDS];
#pragma unroll
        for (int j = 0; j < CC_WORDS; ++j) {
            a[j] = bitmap[wbase + 32u * j + lane];
            b[j] = front[wbase + 32u * j + lane];
        }
        uint32_t cnt = 0;  // both counts packed: at most 32768 each per tile
#pragma unroll
        for (int j = 0; j < CC_WORDS; ++j) cnt += __popc(a[j]) | (__popc(b[j]) << 16);
        cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
        if (lane == 0) s_wtot[warp] = cnt;
        __syncthreads();
        uint32_t wexcl = 0, total = 0;
#pragma unroll
        for (int w = 0; w < CC_WARPS; ++w) {
            const uint32_t v = s_wtot[w];
            wexcl += (uint32_t)w < warp ? v : 0u;
            total += v;
        }
        if (warp < 2) {
            const uint32_t agg = warp == 0 ? (total & 0xFFFFu) : (total >> 16);
            const uint32_t pre = lookback_warp(warp == 0 ? status : status_front, 1, tile, agg, epoch, &ctr->flags);
            if (lane == 0) s_prefix[warp] = pre;
        }
        __syncthreads();
        uint32_t oa = s_prefix[0] + (wexcl & 0xFFFFu), ob = s_prefix[1] + (wexcl >> 16);
#pragma unroll
        for (int j = 0; j < CC_WORDS; ++j) {
            const uint32_t wi = wbase + 32u * j + lane;
            oa = cc_round(a[j], wi, oa, s_stage[warp], cut, cap);
            ob = cc_round(b[j], wi, ob, s_stage[warp], front_list, cap);
            if (a[j]) bitmap[wi] = 0u;
            if (b[j]) front[wi] = 0u;
        }
        if (tile == ntiles - 1 && threadIdx.x == 0) {
            const uint32_t n = s_prefix[0] + (total & 0xFFFFu);
            *n_cut_out = n;
            ctr->n_front = s_prefix[1] + (total >> 16);
            if (n > cap) atomicOr(&ctr->flags, F_OVF_CUT);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ launchers
void launch_lod_update(const SceneDev& sc, const uint32_t* prev_cut, const uint32_t* n_prev, uint32_t cap_prev,
                       const FrameParams* fp, uint32_t* bitmap, uint32_t* front, Counters* ctr, int grid,
                       bool frustum, bool interp, cudaStream_t s) {
#define VGR_LOD_UPDATE(FR, IP) \
    launch_k(k_lod_update<FR, IP>, grid, 256, s, prev_cut, n_prev, cap_prev, sc, fp, bitmap, front, ctr)
    if (frustum) {
        if (interp) VGR_LOD_UPDATE(true, true);
        else VGR_LOD_UPDATE(true, false);
    } else {
        if (interp) VGR_LOD_UPDATE(false, true);
        else VGR_LOD_UPDATE(false, false);
    }
#undef VGR_LOD_UPDATE
}

void launch_lod_level(int level, const SceneDev& sc, const uint32_t* fin, uint32_t* fout, uint32_t cap,
                      const FrameParams* fp, uint32_t* bitmap, uint32_t* front, Counters* ctr, int grid,
                      bool frustum, bool interp, cudaStream_t s) {
#define VGR_LOD_LEVEL(FR, IP) \
    launch_k(k_lod_level<FR, IP>, grid, 256, s, level, fin, fout, cap, sc, fp, bitmap, front, ctr)
    if (frustum) {
        if (interp) VGR_LOD_LEVEL(true, true);
        else VGR_LOD_LEVEL(true, false);
    } else {
        if (interp) VGR_LOD_LEVEL(false, true);
        else VGR_LOD_LEVEL(false, false);
    }
#undef VGR_LOD_LEVEL
}

void launch_cut_compact(uint32_t* bitmap, uint32_t* front, uint32_t n_words, uint32_t* cut, uint32_t* front_list,
                        uint32_t cap, uint32_t* n_cut_out, unsigned long long* status,
                        unsigned long long* status_front, Counters* ctr, const FrameParams* fp, int grid,
                        cudaStream_t s) {
    launch_k(k_cut_compact, grid, CC_THREADS, s, bitmap, front, n_words, cut, front_list, cap, n_cut_out, status,
                                       status_front, ctr, fp);
}

uint32_t cut_compact_tiles(uint32_t n_words) { return (n_words + CC_TILE_WORDS - 1) / CC_TILE_WORDS; }
uint32_t cut_compact_tile_words() { return CC_TILE_WORDS; }

}  // namespace vgr
