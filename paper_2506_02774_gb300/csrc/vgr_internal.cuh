// vgr_internal.cuh -- device-side structures and helpers shared by the
// kernels of the frame path (LoD cut, preprocess, sort, emit, blend).
#pragma once

#include <cuda/atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include "vgr.h"

namespace vgr {

constexpr int TILE_DEFAULT = 16;              // tiles of 16 x 16 pixels unless a view asks for 8 or 32
constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr float ALPHA_MIN = 1.0f / 255.0f;    // alpha* (Sec. 3.1 'Rasterization')
constexpr float LN_ALPHA_MIN = -5.5412635451584260f;  // ln(1/255)
constexpr float T_MIN = 1e-4f;                // early-termination transmittance
constexpr uint32_t MAX_RANKS = 1u << 24;        // visible Gaussians per frame (pair value = rank << 8 | row mask)
constexpr float ALPHA_MAX = 0.99f;            // Eq. 3 clamp
constexpr float DILATE = 0.3f;                // low-pass added to the 2D covariance
constexpr float TILE_EPS = 2e-3f;             // slack of the FP32 tile-level test (nats)
constexpr int MAX_TREE_DEPTH = 64;
constexpr uint32_t SPIN_LIMIT = 1u << 22;     // bounded waits in look-back scans
constexpr uint32_t CHILD_SHIFT = 28;          // child word: first_child | n_child << 28
constexpr uint32_t CHILD_MASK = (1u << CHILD_SHIFT) - 1u;
constexpr int RADIX_THREADS = 256;            // one radix-sort tile: 256 threads x 15 keys
constexpr int RADIX_ITEMS = 15;
constexpr int RADIX_TILE = RADIX_THREADS * RADIX_ITEMS;

// flags in Counters::flags
enum : uint32_t {
    F_LOD_FALLBACK = 1u,   // a thread exceeded its expansion budget: redo the cut top-down
    F_NONMONOTONE = 2u,    // child expands while the parent does not
    F_SPIN_TIMEOUT = 4u,   // a look-back wait ran out
    F_OVF_CUT = 8u,
    F_OVF_VIS = 16u,       // more visible Gaussians than a pair value's 24-bit rank holds
    F_OVF_PAIRS = 32u,
    F_OVF_FRONTIER = 64u,
};

// ticket slots (dynamic tile order for the chained scans)
enum : int { TK_COMPACT = 0, TK_PRE = 1, TK_EMIT = 2, TK_SORT0 = 3 /* .. TK_SORT0 + 7 */, TK_COUNT = 12 };

struct Counters;

// Per-frame parameters, uploaded once per frame (a graph replays them).
struct FrameParams {
    float R[9];
    float pos[3];
    float fx, fy, cx, cy;
    float z_near;
    float k;           // fl(fl(tau/f)^2)
    float limx, limy;  // 1.3 (W/2)/fx, 1.3 (H/2)/fy
    float width_f, height_f;
    uint32_t width, height, tiles_x, tiles_y;
    uint32_t tile;        // tile side in pixels: 8, 16 or 32
    uint32_t epoch;    // tags look-back words; new value per launch sequence
    uint32_t filter, exp_mode, lut_size;
    float lut_step;    // 5.55 / m
    uint32_t lod_budget;
    uint32_t max_depth;
    uint32_t test_hooks;  // vgr_view_opts.test_hooks (0 in normal use)
    float* host_image;    // device-accessible pinned host image the blend also writes, or null
    uint32_t lod_frustum; // frustum-aware expansion on (needs node boxes)
    uint32_t lod_interp;  // parent-child weight interpolation on
    float lod_t;          // fl(tau / f), the size ratio the interpolation weight is measured against
    // its planes: world normal w (xyz) and offset o (w), inside iff w.x - o >= 0 (read as float4)
    alignas(16) float frustum[5][4];
    // the buffers the blend reads and writes for this frame (a batch's blend
    // reaches every view's through these)
    const uint2* bl_ranges;      // [tiles] pair range of each tile
    const uint32_t* bl_pair_val; // sorted pair values (in-front index << 8 | row mask)
    const float4* bl_recA;
    const float4* bl_recB;
    const float4* bl_rgb;
    const float* bl_lut;         // Eq. 5 table (m + 1 entries)
    float* bl_image;             // H x W x 3
    Counters* bl_ctr;
};

// Zeroed at the start of every frame.  Scalars first: the host reads back
// only the head of the struct.
struct Counters {
    uint32_t n_vis;
    uint32_t flags;
    uint32_t n_front;  // cut nodes in front of the near plane
    uint32_t pad0;
    unsigned long long n_pairs;
    unsigned long long n_cand;
    unsigned long long nodes_eval;
    unsigned long long pix_evals;
    unsigned long long pix_contribs;
    uint32_t tickets[TK_COUNT];
    uint32_t frontier_n[MAX_TREE_DEPTH + 2];
    uint32_t depth_hist[4][256];
    uint32_t tile_hist[4][256];
    uint32_t tile_buckets[33];  // tiles per log2(pairs + 1) class (the blend order)
    uint32_t blend_next;        // the blend's next tile in its work list
};
constexpr size_t COUNTERS_HEAD = 56;  // bytes read back per frame (n_vis .. pix_contribs)

// Persistent per-view values (not cleared per frame).
struct ViewState {
    uint32_t n_cut[2];
};

// Device view of the hierarchy.
struct SceneDev {
    const float4* cr;          // mean xyz, w = radius2 (internal) or -radius2 (leaf: never expands)
    const float4* lodr;        // per node 2 float4: its cr entry, its parent's (the root's: w = +inf)
    const uint32_t* parent;
    const uint32_t* child;     // first_child | n_child << 28
    const float4* covA;        // xx xy xz yy
    const float4* covB;        // yz zz opacity ln(opacity)
    const float* lmax;         // upper bound of the covariance's largest eigenvalue (Gershgorin)
    const float2* box;         // nested node boxes, 3 per node: (lo, hi) in x, y, z; null if not loaded
    const void* sh;            // FP32 or FP16, sh_stride elements per node
    uint32_t n_nodes;
    uint32_t sh_degree;
    uint32_t sh_stride;        // elements per node (multiple of 4 for FP32, 8 for FP16)
    uint32_t storage;          // VGR_STORE_*
};

// ------------------------------------------------------------- helpers
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// First statement of every frame kernel: wait until the previous kernel in
// the stream has completed (a no-op when launched without programmatic
// stream serialization).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive warp scan of v over all 32 lanes; *total gets the warp sum.
__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, uint32_t* total) {
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane_id() >= (uint32_t)o) x += y;
    }
    *total = __shfl_sync(0xFFFFFFFFu, x, 31);
    return x - v;
}

// Block-wide exclusive scan (blockDim.x = 32 * NW).  smem: NW + 1 words.
template <int NW>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* smem, uint32_t* total) {
    uint32_t wt;
    uint32_t x = warp_excl_scan(v, &wt);
    const uint32_t w = threadIdx.x >> 5;
    if (lane_id() == 31) smem[w] = wt;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int i = 0; i < NW; ++i) { uint32_t c = smem[i]; smem[i] = run; run += c; }
        smem[NW] = run;
    }
    __syncthreads();
    uint32_t r = x + smem[w];
    *total = smem[NW];
    return r;
}

// ------------------------------------------- decoupled look-back words
// word = epoch(30) << 34 | flag(2) << 32 | value(32); flag 1 = tile
// aggregate, 2 = inclusive prefix.  Words of an older epoch read as empty.
__device__ __forceinline__ unsigned long long lb_pack(uint32_t epoch, uint32_t flag, uint32_t value) {
    return ((unsigned long long)(epoch & 0x3FFFFFFFu) << 34) | ((unsigned long long)flag << 32) | value;
}
__device__ __forceinline__ void lb_store(unsigned long long* p, unsigned long long w) {
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> a(*p);
    a.store(w, cuda::memory_order_relaxed);
}
__device__ __forceinline__ unsigned long long lb_load(unsigned long long* p) {
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> a(*p);
    return a.load(cuda::memory_order_relaxed);
}

// Publish this tile's aggregate, walk back to an inclusive prefix, publish
// the inclusive value; returns the exclusive prefix.  'status' points at
// this scan's word array with 'stride' words between consecutive tiles.
// Tiles are handed out in ticket order, so every predecessor is running or
// done; the wait is still bounded and reports F_SPIN_TIMEOUT.
__device__ __forceinline__ uint32_t lookback(unsigned long long* status, uint32_t stride, uint32_t tile,
                                             uint32_t agg, uint32_t epoch, uint32_t* flags) {
    const uint32_t ep = epoch & 0x3FFFFFFFu;
    if (tile == 0) {
        lb_store(status, lb_pack(epoch, 2u, agg));
        return 0;
    }
    lb_store(status + (size_t)tile * stride, lb_pack(epoch, 1u, agg));
    uint32_t prefix = 0;
    int64_t j = (int64_t)tile - 1;
    uint32_t spins = 0;
    while (j >= 0) {
        unsigned long long w = lb_load(status + (size_t)j * stride);
        uint32_t wep = (uint32_t)(w >> 34), fl = (uint32_t)(w >> 32) & 3u;
        if (wep != ep || fl == 0u) {
            if (++spins > SPIN_LIMIT) { atomicOr(flags, F_SPIN_TIMEOUT); break; }
            __nanosleep(20);
            continue;
        }
        prefix += (uint32_t)w;
        if (fl == 2u) break;
        --j;
    }
    lb_store(status + (size_t)tile * stride, lb_pack(epoch, 2u, prefix + agg));
    return prefix;
}

// Warp-wide variant (all 32 lanes of one warp call it): each step reads 32
// predecessor words at once, so the prefix is usually found after one L2
// round trip instead of one per predecessor.  Same words and result as
// lookback(); every lane returns the exclusive prefix.
__device__ __forceinline__ uint32_t lookback_warp(unsigned long long* status, uint32_t stride, uint32_t tile,
                                                  uint32_t agg, uint32_t epoch, uint32_t* flags) {
    const uint32_t lane = lane_id();
    const uint32_t ep = epoch & 0x3FFFFFFFu;
    if (tile == 0) {
        if (lane == 0) lb_store(status, lb_pack(epoch, 2u, agg));
        return 0;
    }
    if (lane == 0) lb_store(status + (size_t)tile * stride, lb_pack(epoch, 1u, agg));
    uint32_t prefix = 0;
    int64_t base = (int64_t)tile - 1;  // window [base - 31, base], lane i reads base - i
    uint32_t spins = 0;
    for (;;) {
        const int64_t j = base - (int64_t)lane;
        uint32_t val = 0, fl = 2u;
        bool ready = true;
        if (j >= 0) {
            const unsigned long long w = lb_load(status + (size_t)j * stride);
            fl = (uint32_t)(w >> 32) & 3u;
            ready = ((uint32_t)(w >> 34) == ep) && fl != 0u;
            val = (uint32_t)w;
        }
        const uint32_t incl = __ballot_sync(0xFFFFFFFFu, ready && fl == 2u);
        const uint32_t rdy = __ballot_sync(0xFFFFFFFFu, ready);
        if (incl) {
            const int k = __ffs(incl) - 1;  // nearest inclusive prefix in the window
            const uint32_t need = k == 31 ? 0xFFFFFFFFu : ((1u << (k + 1)) - 1u);
            if ((rdy & need) == need) {
                prefix += __reduce_add_sync(0xFFFFFFFFu, (int)lane <= k ? val : 0u);
                break;
            }
        } else if (rdy == 0xFFFFFFFFu) {  // 32 aggregates: take them and look further back
            prefix += __reduce_add_sync(0xFFFFFFFFu, val);
            base -= 32;
            continue;
        }
        if (++spins > SPIN_LIMIT) {
            if (lane == 0) atomicOr(flags, F_SPIN_TIMEOUT);
            break;
        }
        __nanosleep(20);
    }
    if (lane == 0) lb_store(status + (size_t)tile * stride, lb_pack(epoch, 2u, prefix + agg));
    return prefix;
}

// FP32 depth key of a node: z = ((R20 dx + R21 dy) + R22 dz), dx = fl(mu_x - C_x),
// every operation single-rounded.  The near-plane cull and the depth order use it.
__device__ __forceinline__ float depth_key(float4 m, float R6, float R7, float R8, float Cx, float Cy, float Cz) {
    const float dx = __fsub_rn(m.x, Cx), dy = __fsub_rn(m.y, Cy), dz = __fsub_rn(m.z, Cz);
    return __fadd_rn(__fadd_rn(__fmul_rn(R6, dx), __fmul_rn(R7, dy)), __fmul_rn(R8, dz));
}

// The granularity test, single-rounded FP32 (no contraction): expand iff
// fl(((dx dx + dy dy) + dz dz) k) < radius2; cr.w is -radius2 <= 0 for leaves.
__device__ __forceinline__ bool lod_expand(float4 c, float px, float py, float pz, float k) {
    float dx = __fsub_rn(px, c.x), dy = __fsub_rn(py, c.y), dz = __fsub_rn(pz, c.z);
    float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    return __fmul_rn(d2, k) < c.w;
}

// Frustum-aware variant of the granularity test: node n also needs its box
// to meet each of the five half-spaces {x : w.x - o >= 0} (near plane and the
// four planes through the camera centre and the guard-widened image edges).
// The box corner furthest along w is tested, single-rounded FP32 in a fixed
// order; rounding is monotone, so a box inside another never scores higher
// and nested boxes keep "child expands => parent expands".
// (The planes are read from the frame parameters at each test, through L1,
// rather than held in 20 registers.)
struct LodFrustum {
    const float4* planes;
    const float2* box;
    __device__ __forceinline__ void load(const FrameParams* fp, const float2* b) {
        planes = reinterpret_cast<const float4*>(fp->frustum);
        box = b;
    }
    __device__ __forceinline__ bool meets(uint32_t n) const {
        const float2 bx = box[3 * (size_t)n], by = box[3 * (size_t)n + 1], bz = box[3 * (size_t)n + 2];
        bool in = true;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float4 w = __ldg(planes + i);
            const float X = w.x >= 0.f ? bx.y : bx.x;
            const float Y = w.y >= 0.f ? by.y : by.x;
            const float Z = w.z >= 0.f ? bz.y : bz.x;
            const float s = __fsub_rn(__fadd_rn(__fadd_rn(__fmul_rn(w.x, X), __fmul_rn(w.y, Y)), __fmul_rn(w.z, Z)),
                                      w.w);
            in = in && s >= 0.f;
        }
        return in;
    }
};

// Weight of the parent in the interpolated Gaussian of cut node n (Sec. 3.1
// 'Weight Interpolation'): with a = sqrt(R^2 / d^2) the size ratio R / d of a
// node (its projected size over f) and t = tau / f,
//   w = clamp((t - a_n) / (a_p - a_n), 0, 1)  when a_p > a_n, else 0,
// single-rounded FP32 (IEEE division and square root), d^2 as in the
// granularity test.  w runs from 0 where n is about to expand (a_n = t) to 1
// where its parent is about to collapse (a_p = t).
__device__ __forceinline__ float lod_size_ratio(float4 c, float px, float py, float pz) {
    const float dx = __fsub_rn(px, c.x), dy = __fsub_rn(py, c.y), dz = __fsub_rn(pz, c.z);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    return __fsqrt_rn(__fdiv_rn(fabsf(c.w), d2));
}
__device__ __forceinline__ float lod_interp_weight(float an, float ap, float t) {
    if (!(ap > an)) return 0.f;
    const float w = __fdiv_rn(__fsub_rn(t, an), __fsub_rn(ap, an));
    return fminf(1.f, fmaxf(0.f, w));
}
// The interpolated mean, single-rounded per component: mn + w (mp - mn).
__device__ __forceinline__ float lod_lerp_rn(float a, float b, float w) {
    return __fadd_rn(a, __fmul_rn(w, __fsub_rn(b, a)));
}

__device__ __forceinline__ void bitmap_set(uint32_t* bm, uint32_t n) { atomicOr(&bm[n >> 5], 1u << (n & 31u)); }

// Lanes of the (full) warp holding the same 9-bit value (a radix digit
// 0..255, or 256 for "no digit"): one ballot per bit.
__device__ __forceinline__ uint32_t match_digit(uint32_t d) {
    uint32_t m = 0xFFFFFFFFu;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t vote = __ballot_sync(0xFFFFFFFFu, bit);
        m &= bit ? vote : ~vote;
    }
    return m;
}

}  // namespace vgr
