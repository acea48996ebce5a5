// vgr_capi.cu -- the C ABI (include/vgr.h): hierarchy upload and validation,
// per-view buffers, and the per-frame launch sequence
//   LoD (temporal update or top-down levels) -> cut compaction ->
//   preprocess (with colour) -> depth sort -> emission -> tile sort (its last
//   pass records the tile ranges) -> blend order -> blend
// all enqueued on the view's stream (or replayed as one captured graph).
// Counts stay on the device (every kernel reads its element count from
// device memory), so a frame needs no host round trip until its end, where
// a 56-byte status block and the cut sizes are read back: buffer overflows
// are handled by growing the buffer and replaying the frame, a temporal
// update that ran past its budget by replaying the frame with the top-down
// cut.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "vgr.h"
#include "vgr_internal.cuh"
#include "vgr_launch.h"

using namespace vgr;

namespace {

thread_local std::string g_err;

vgr_status fail(vgr_status s, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define VGR_CK(call)                                                                                        \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) {                                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? VGR_E_NOMEM : VGR_E_CUDA, "%s failed: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                                 \
        }                                                                                                   \
    } while (0)

template <typename T>
vgr_status dalloc(T** p, size_t count, uint64_t* acct) {
    *p = nullptr;
    if (count == 0) count = 1;
    const cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();  // not sticky: clear it so later launches are not blamed
        return fail(e == cudaErrorMemoryAllocation ? VGR_E_NOMEM : VGR_E_CUDA, "cudaMalloc of %zu bytes: %s",
                    count * sizeof(T), cudaGetErrorString(e));
    }
    // The zero fill runs on the legacy default stream, which does not order
    // with the views' non-blocking streams: wait for it here, or a frame
    // already running on such a stream could see the fill land on top of its
    // own writes (a range table reset to zero, look-back words cleared).
    VGR_CK(cudaMemset(*p, 0, count * sizeof(T)));
    VGR_CK(cudaStreamSynchronize(cudaStreamLegacy));
    if (acct) *acct += count * sizeof(T);
    return VGR_OK;
}

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

uint32_t ceil_div(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

}  // namespace

void vgr::set_last_error(const char* msg) { g_err = msg; }

bool vgr::pdl_enabled() {
    static const bool on = [] {
        const char* e = getenv("VGR_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

vgr::PdlState& vgr::pdl_state() {
    static thread_local PdlState st;
    return st;
}

struct vgr_hierarchy {
    SceneDev dev{};
    float4* cr = nullptr;
    float4* lodr = nullptr;  // per node its cr entry and its parent's (root: w = +inf), 32 bytes
    uint32_t* parent = nullptr;
    uint32_t* child = nullptr;
    float4* covA = nullptr;
    float4* covB = nullptr;
    float* lmax = nullptr;
    float2* box = nullptr;  // nested node boxes (optional)
    void* sh = nullptr;
    uint32_t n_nodes = 0, max_depth = 0;
    uint64_t bytes = 0;
    int device = 0;
    int num_sms = 0;
};

// A submitted frame, kept until vgr_finish_frame.
struct PendingFrame {
    vgr_camera cam{};
    float tau = 0.f, f = 0.f, t = 0.f, k = 0.f;
    bool scratch = false;
    int tile_passes = 1;
    uint32_t kernels = 0;
    float* host = nullptr;
    float* host_dev = nullptr;  // device address of host when the blend can write it directly
    bool pipe = false;          // host copy on the copy stream after the status check, not awaited
    int img = 0;                // device image written (0: image, 1: image_alt)
};

struct vgr_view {
    vgr_hierarchy* h = nullptr;
    vgr_view_opts opts{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int grid_wide = 0, grid_scan = 0;
    // capacities
    uint32_t cap_cut = 0, cap_vis = 0;  // visible arrays are indexed like the in-front list: cap_vis = cap_cut
    uint64_t cap_pairs = 0;
    uint32_t cap_pixels = 0, cap_tiles = 0;
    // device buffers
    uint32_t* cut[2] = {nullptr, nullptr};
    uint32_t* bitmap = nullptr;
    uint32_t* front_bm = nullptr;     // cut nodes in front of the near plane
    uint32_t* front_list = nullptr;   // their ids, ascending (cap_cut)
    uint32_t n_words = 0;
    uint32_t* frontier[2] = {nullptr, nullptr};
    VisBuffers vis{};
    uint32_t* sortK[2] = {nullptr, nullptr};
    uint32_t* sortV[2] = {nullptr, nullptr};
    uint32_t* slot_off = nullptr;  // first pair slot of each visible Gaussian by depth rank (cap_vis + 1)
    uint32_t* pairK[2] = {nullptr, nullptr};
    uint32_t* pairV[2] = {nullptr, nullptr};
    uint2* ranges = nullptr;
    uint32_t* tile_order = nullptr;  // blend order, heaviest tiles first
    float* image = nullptr;
    // pipelined host images: the second device image, the frame being
    // written, the copy stream and, per device image, the event its last copy
    // into host memory recorded
    float* image_alt = nullptr;
    float* cur_image = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ev[2] = {nullptr, nullptr};
    bool copy_pending[2] = {false, false};
    int img_sel = 0;  // device image the next pipelined frame writes
    float* lut = nullptr;
    unsigned long long* status = nullptr;
    size_t st_compact = 0, st_front = 0, st_emit = 0, st_depth = 0, st_tile = 0, st_depth_stride = 0,
           st_tile_stride = 0, st_words = 0;
    Counters* ctr = nullptr;
    ViewState* vstate = nullptr;
    FrameParams* fp_dev = nullptr;
    // pinned host mirrors
    FrameParams* fp_host = nullptr;
    unsigned char* ctr_host = nullptr;
    ViewState* vstate_host = nullptr;
    cudaEvent_t ev[VGR_N_STAGES + 1] = {};
    // temporal state
    bool has_prev = false;
    int parity = 0;  // buffer index holding the previous cut
    float prev_tau = -1.f, prev_f = -1.f;
    uint32_t epoch = 0;
    // last frame
    uint32_t last_w = 0, last_h = 0, last_tw = 0, last_th = 0;
    int last_tile_buf = 0;
    uint32_t last_n_cut = 0, last_n_vis = 0, last_n_front = 0;
    uint64_t last_n_pairs = 0;
    // captured frames, one per (top-down cut?, buffer parity); every kernel
    // argument they hold is a buffer address or a size fixed by the tile
    // grid, and the per-frame values travel through fp_host (read by the
    // captured host-to-device copy at replay), so a graph stays valid until a
    // buffer is reallocated or the tile grid changes
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    uint32_t graph_tiles = 0;
    // frame in flight between submit and finish
    bool pending = false;
    bool broken = false;  // a buffer could not be grown: its memory is gone, no further frames
    PendingFrame pend;
    cudaEvent_t done_ev = nullptr;
    cudaEvent_t join_ev = nullptr;  // end of this view's branch in a captured batch
    uint64_t uid = 0;               // unique per view ever created (batch graph keys)
    uint64_t gen = 0;               // bumped whenever the view's buffers change (graphs invalid)
    uint64_t vis_bytes = 0, pair_bytes = 0, img_bytes = 0, fixed_bytes = 0, status_bytes = 0, cut_bytes = 0;
};

extern "C" {

const char* vgr_last_error(void) { return g_err.c_str(); }

void vgr_default_view_opts(vgr_view_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->filter = VGR_FILTER_PREEMPTIVE;
    o->exp_mode = VGR_EXP_EXACT;
    o->lut_size = 32;
    o->temporal = 1;
    o->timing = 0;
    o->use_graph = 0;
    o->lod_budget = 4096;
    o->lod_frustum = 0;
    o->lod_frustum_guard = 2.0f;
    o->lod_interp = 0;
    o->blend_depth = 32;
    o->tile_size = TILE_DEFAULT;
}

// ------------------------------------------------------------- hierarchy
vgr_status vgr_load_hierarchy(const vgr_scene_desc* d, vgr_hierarchy** out) {
    if (!d || !out) return fail(VGR_E_INVALID, "null argument");
    *out = nullptr;
    const uint32_t N = d->n_nodes;
    if (N == 0 || N > CHILD_MASK) return fail(VGR_E_INVALID, "n_nodes must be in [1, 2^28)");
    if (d->sh_degree > 3) return fail(VGR_E_INVALID, "sh_degree must be <= 3");
    if (d->storage != VGR_STORE_FP32 && d->storage != VGR_STORE_HALF) return fail(VGR_E_INVALID, "bad storage");
    if (!d->parent || !d->first_child || !d->n_child || !d->mean || !d->cov6 || !d->opacity || !d->sh ||
        !d->radius2)
        return fail(VGR_E_INVALID, "null array in scene description");
    // shape: BFS order, contiguous child blocks, parent links
    if (d->parent[0] != NONE) return fail(VGR_E_INVALID, "node 0 must be the root (parent 0xFFFFFFFF)");
    std::vector<uint8_t> depth(N, 0);
    uint64_t expect = 1;
    uint32_t maxd = 0;
    for (uint32_t n = 0; n < N; ++n) {
        const uint32_t nc = d->n_child[n];
        if (nc > 8) return fail(VGR_E_INVALID, "node %u has %u > 8 children", n, nc);
        if (nc == 0) continue;
        if (d->first_child[n] != expect)
            return fail(VGR_E_INVALID, "children of node %u are not the next BFS block (first_child %u, expected %llu)",
                        n, d->first_child[n], (unsigned long long)expect);
        if (expect + nc > N) return fail(VGR_E_INVALID, "children of node %u run past n_nodes", n);
        for (uint32_t c = 0; c < nc; ++c) {
            const uint32_t ch = (uint32_t)expect + c;
            if (d->parent[ch] != n) return fail(VGR_E_INVALID, "parent[%u] != %u", ch, n);
            const uint32_t dd = depth[n] + 1u;
            if (dd >= MAX_TREE_DEPTH - 2) return fail(VGR_E_INVALID, "tree deeper than %d", MAX_TREE_DEPTH - 3);
            depth[ch] = (uint8_t)dd;
            maxd = std::max(maxd, dd);
        }
        expect += nc;
    }
    if (expect != N) return fail(VGR_E_INVALID, "not every node is reachable from the root (%llu of %u)",
                                 (unsigned long long)expect, N);
    for (uint32_t n = 0; n < N; ++n) {
        const float* m = d->mean + 3 * (size_t)n;
        if (!std::isfinite(m[0]) || !std::isfinite(m[1]) || !std::isfinite(m[2]))
            return fail(VGR_E_INVALID, "mean of node %u is not finite", n);
        const float op = d->opacity[n];
        if (!(op >= 0.f && op <= 1.f)) return fail(VGR_E_INVALID, "opacity of node %u outside [0, 1]", n);
        const float r2 = d->radius2[n];
        if (!(r2 >= 0.f) || !std::isfinite(r2)) return fail(VGR_E_INVALID, "radius2 of node %u invalid", n);
        for (int k = 0; k < 6; ++k)
            if (!std::isfinite(d->cov6[6 * (size_t)n + k])) return fail(VGR_E_INVALID, "cov of node %u not finite", n);
        if (n > 0) {
            const uint32_t p = d->parent[n];
            const float* mp = d->mean + 3 * (size_t)p;
            const double dx = (double)m[0] - mp[0], dy = (double)m[1] - mp[1], dz = (double)m[2] - mp[2];
            const double need = std::sqrt((double)r2) + std::sqrt(dx * dx + dy * dy + dz * dz);
            if (std::sqrt((double)d->radius2[p]) < need * (1.0 - 1e-6))
                return fail(VGR_E_INVALID, "radius of node %u does not contain child %u (nesting violated)", p, n);
        }
        if (d->bbox) {
            const float* b = d->bbox + 6 * (size_t)n;
            for (int a = 0; a < 3; ++a)
                if (!std::isfinite(b[a]) || !std::isfinite(b[3 + a]) || !(b[a] <= b[3 + a]))
                    return fail(VGR_E_INVALID, "box of node %u invalid", n);
            if (n > 0) {
                const float* bp = d->bbox + 6 * (size_t)d->parent[n];
                for (int a = 0; a < 3; ++a)
                    if (!(bp[a] <= b[a] && bp[3 + a] >= b[3 + a]))
                        return fail(VGR_E_INVALID, "box of node %u does not contain child %u (nesting violated)",
                                    d->parent[n], n);
            }
        }
    }

    int dev = 0;
    VGR_CK(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    VGR_CK(cudaGetDeviceProperties(&prop, dev));
    if (prop.major * 10 + prop.minor < 100)
        return fail(VGR_E_CUDA, "device %s (sm_%d%d) is not a Blackwell GPU", prop.name, prop.major, prop.minor);

    vgr_hierarchy* h = new vgr_hierarchy();
    h->n_nodes = N;
    h->max_depth = maxd;
    h->device = dev;
    h->num_sms = prop.multiProcessorCount;
    const uint32_t K3 = 3u * (d->sh_degree + 1) * (d->sh_degree + 1);
    const bool half = d->storage == VGR_STORE_HALF;
    const uint32_t stride = half ? (K3 + 7u) / 8u * 8u : (K3 + 3u) / 4u * 4u;
    vgr_status st = VGR_OK;
    auto cleanup = [&]() { dfree(h->cr); dfree(h->lodr); dfree(h->parent); dfree(h->child); dfree(h->covA); dfree(h->covB); dfree(h->lmax);
                           dfree(h->box); if (h->sh) cudaFree(h->sh); delete h; };
#define VGR_TRY(x)                 \
    do {                           \
        st = (x);                  \
        if (st != VGR_OK) {        \
            cleanup();             \
            return st;             \
        }                          \
    } while (0)
    VGR_TRY(dalloc(&h->cr, N, &h->bytes));
    VGR_TRY(dalloc(&h->lodr, 2 * (size_t)N, &h->bytes));
    VGR_TRY(dalloc(&h->parent, N, &h->bytes));
    VGR_TRY(dalloc(&h->child, N, &h->bytes));
    VGR_TRY(dalloc(&h->covA, N, &h->bytes));
    VGR_TRY(dalloc(&h->covB, N, &h->bytes));
    VGR_TRY(dalloc(&h->lmax, N, &h->bytes));
    if (d->bbox) VGR_TRY(dalloc(&h->box, 3 * (size_t)N, &h->bytes));
    {
        const size_t shb = (size_t)N * stride * (half ? 2 : 4);
        cudaError_t e = cudaMalloc(&h->sh, shb);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            return fail(VGR_E_NOMEM, "cudaMalloc sh (%zu bytes): %s", shb, cudaGetErrorString(e));
        }
        h->bytes += shb;
    }
    // staging in chunks through a pinned buffer
    const uint32_t CH = 1u << 20;
    void* pin = nullptr;
    const size_t pin_bytes = (size_t)CH * std::max<size_t>(64, (size_t)K3 * 4);
    if (cudaMallocHost(&pin, pin_bytes) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(VGR_E_NOMEM, "pinned staging");
    }
    float* tmp_dev = nullptr;
    if (half) {
        if (cudaMalloc(&tmp_dev, (size_t)CH * std::max<uint32_t>(K3, 6) * 4) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(pin); cleanup(); return fail(VGR_E_NOMEM, "conversion buffer");
        }
    }
    cudaError_t ce = cudaSuccess;
    for (uint32_t b = 0; b < N && ce == cudaSuccess; b += CH) {
        const uint32_t cnt = std::min(CH, N - b);
        float4* f4 = (float4*)pin;
        for (uint32_t i = 0; i < cnt; ++i) {
            const uint32_t n = b + i;
            const float* m = d->mean + 3 * (size_t)n;
            f4[i] = make_float4(m[0], m[1], m[2], d->n_child[n] ? d->radius2[n] : -d->radius2[n]);
        }
        ce = cudaMemcpy(h->cr + b, f4, cnt * sizeof(float4), cudaMemcpyHostToDevice);
        // the temporal update's record: the node's entry and its parent's in
        // one 32-byte sector, so a cut node costs one sector and one round;
        // the root's parent entry has w = +inf (radius2 is finite)
        for (uint32_t i = cnt; i-- > 0;) {  // in place, from the end: entry i moves to 2i
            const uint32_t n = b + i, p = d->parent[n];
            f4[2 * i] = f4[i];
            if (p == NONE) {
                f4[2 * i + 1] = make_float4(0.f, 0.f, 0.f, INFINITY);
            } else {
                const float* m = d->mean + 3 * (size_t)p;
                f4[2 * i + 1] = make_float4(m[0], m[1], m[2], d->radius2[p]);  // a parent is internal
            }
        }
        if (ce == cudaSuccess)
            ce = cudaMemcpy(h->lodr + 2 * (size_t)b, f4, 2 * (size_t)cnt * sizeof(float4), cudaMemcpyHostToDevice);
        uint32_t* u = (uint32_t*)pin;
        for (uint32_t i = 0; i < cnt; ++i) {
            const uint32_t n = b + i;
            u[i] = d->n_child[n] ? (d->first_child[n] | ((uint32_t)d->n_child[n] << CHILD_SHIFT)) : 0u;
        }
        if (ce == cudaSuccess) ce = cudaMemcpy(h->child + b, u, cnt * 4, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(h->parent + b, d->parent + b, cnt * 4, cudaMemcpyHostToDevice);
        if (d->bbox) {
            float2* f2 = (float2*)pin;  // (lo, hi) per axis
            for (uint32_t i = 0; i < cnt; ++i) {
                const float* bb = d->bbox + 6 * (size_t)(b + i);
                for (int a = 0; a < 3; ++a) f2[3 * i + a] = make_float2(bb[a], bb[3 + a]);
            }
            if (ce == cudaSuccess) ce = cudaMemcpy(h->box + 3 * (size_t)b, f2, (size_t)cnt * 24, cudaMemcpyHostToDevice);
        }
        {
            // largest absolute row sum of the covariance >= its largest eigenvalue;
            // widened for the rounding of the stored (FP32 or BF16) covariance
            float* lm = (float*)pin;
            const double widen = half ? 1.0 + 1.0 / 64.0 : 1.0 + 1e-5;
            for (uint32_t i = 0; i < cnt; ++i) {
                const float* c = d->cov6 + 6 * (size_t)(b + i);
                const double r0 = fabs(c[0]) + fabs(c[1]) + fabs(c[2]);
                const double r1 = fabs(c[1]) + fabs(c[3]) + fabs(c[4]);
                const double r2 = fabs(c[2]) + fabs(c[4]) + fabs(c[5]);
                lm[i] = (float)(std::max(r0, std::max(r1, r2)) * widen);
            }
            if (ce == cudaSuccess) ce = cudaMemcpy(h->lmax + b, lm, cnt * 4, cudaMemcpyHostToDevice);
        }
        if (!half) {
            for (uint32_t i = 0; i < cnt; ++i) {
                const float* c = d->cov6 + 6 * (size_t)(b + i);
                f4[i] = make_float4(c[0], c[1], c[2], c[3]);
            }
            if (ce == cudaSuccess) ce = cudaMemcpy(h->covA + b, f4, cnt * sizeof(float4), cudaMemcpyHostToDevice);
            for (uint32_t i = 0; i < cnt; ++i) {
                const float* c = d->cov6 + 6 * (size_t)(b + i);
                f4[i] = make_float4(c[4], c[5], d->opacity[b + i], 0.f);
            }
            if (ce == cudaSuccess) ce = cudaMemcpy(h->covB + b, f4, cnt * sizeof(float4), cudaMemcpyHostToDevice);
            float* fs = (float*)pin;
            for (uint32_t i = 0; i < cnt; ++i) {
                const float* s = d->sh + (size_t)(b + i) * K3;
                float* o = fs + (size_t)i * stride;
                memcpy(o, s, K3 * 4);
                for (uint32_t j = K3; j < stride; ++j) o[j] = 0.f;
            }
            if (ce == cudaSuccess)
                ce = cudaMemcpy((float*)h->sh + (size_t)b * stride, fs, (size_t)cnt * stride * 4, cudaMemcpyHostToDevice);
        } else {
            if (ce == cudaSuccess) ce = cudaMemcpy(tmp_dev, d->cov6 + 6 * (size_t)b, (size_t)cnt * 24, cudaMemcpyHostToDevice);
            if (ce == cudaSuccess) { convert_cov_bf16(tmp_dev, cnt, h->covA + b, 0); ce = cudaDeviceSynchronize(); }
            for (uint32_t i = 0; i < cnt; ++i) f4[i] = make_float4(d->opacity[b + i], 0.f, 0.f, 0.f);
            if (ce == cudaSuccess) ce = cudaMemcpy(h->covB + b, f4, cnt * sizeof(float4), cudaMemcpyHostToDevice);
            if (ce == cudaSuccess)
                ce = cudaMemcpy(tmp_dev, d->sh + (size_t)b * K3, (size_t)cnt * K3 * 4, cudaMemcpyHostToDevice);
            if (ce == cudaSuccess) {
                convert_sh_half(tmp_dev, cnt, K3, (char*)h->sh + (size_t)b * stride * 2, stride, 0);
                ce = cudaDeviceSynchronize();
            }
        }
    }
    cudaFreeHost(pin);
    if (tmp_dev) cudaFree(tmp_dev);
    if (ce != cudaSuccess) {
        cleanup();
        return fail(VGR_E_CUDA, "hierarchy upload: %s", cudaGetErrorString(ce));
    }
    if (half) prepare_scene_half(h->covB, N, 0);
    else prepare_scene(h->covB, N, 0);
    ce = cudaDeviceSynchronize();
    if (ce != cudaSuccess) { cleanup(); return fail(VGR_E_CUDA, "prepare: %s", cudaGetErrorString(ce)); }
#undef VGR_TRY
    h->dev.cr = h->cr;
    h->dev.lodr = h->lodr;
    h->dev.parent = h->parent;
    h->dev.child = h->child;
    h->dev.covA = h->covA;
    h->dev.covB = h->covB;
    h->dev.lmax = h->lmax;
    h->dev.box = h->box;
    h->dev.sh = h->sh;
    h->dev.n_nodes = N;
    h->dev.sh_degree = d->sh_degree;
    h->dev.sh_stride = stride;
    h->dev.storage = (uint32_t)d->storage;
    *out = h;
    return VGR_OK;
}

vgr_status vgr_free_hierarchy(vgr_hierarchy* h) {
    if (!h) return fail(VGR_E_INVALID, "null hierarchy");
    cudaSetDevice(h->device);
    dfree(h->cr); dfree(h->lodr); dfree(h->parent); dfree(h->child); dfree(h->covA); dfree(h->covB);
    dfree(h->lmax); dfree(h->box);
    if (h->sh) cudaFree(h->sh);
    delete h;
    return VGR_OK;
}

vgr_status vgr_hierarchy_info(const vgr_hierarchy* h, uint64_t* bytes, uint32_t* max_depth) {
    if (!h) return fail(VGR_E_INVALID, "null hierarchy");
    if (bytes) *bytes = h->bytes;
    if (max_depth) *max_depth = h->max_depth;
    return VGR_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ views
namespace {

// Captured batches (vgr_render_batch): one graph runs every view's frame as
// a parallel branch.  Keyed by each view's id, buffer generation, cut mode,
// buffer parity and tile grid; a few recent ones are kept per process.
struct BatchGraph {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    uint64_t last_use = 0;
    void* dev = nullptr;  // the batch blend's view table and work list
};

void destroy_batch(BatchGraph& b) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.dev) cudaFree(b.dev);
    b.exec = nullptr;
    b.dev = nullptr;
}
std::mutex g_batch_mu;
std::vector<BatchGraph> g_batches;
uint64_t g_batch_clock = 0;
constexpr size_t BATCH_GRAPHS_KEPT = 8;
std::atomic<uint32_t> g_batch_chains{0};  // parallel chains of a captured batch (0: one per view)

void forget_batches(uint64_t uid) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t i = 0; i < g_batches.size();) {
        bool hit = false;
        for (size_t k = 0; k < g_batches[i].key.size(); k += 6)
            if (g_batches[i].key[k] == uid) hit = true;
        if (hit) {
            destroy_batch(g_batches[i]);
            g_batches.erase(g_batches.begin() + (long)i);
        } else {
            ++i;
        }
    }
}

void drop_graphs(vgr_view* v) {
    for (auto& row : v->graph)
        for (auto& g : row)
            if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    ++v->gen;  // batch graphs holding this view's buffers no longer match
}

void free_vis(vgr_view* v) {
    drop_graphs(v);
    dfree(v->vis.depth); dfree(v->vis.ntile); dfree(v->vis.rect);
    dfree(v->vis.recA); dfree(v->vis.recB); dfree(v->vis.rgb); dfree(v->vis.lw);
    for (int i = 0; i < 2; ++i) { dfree(v->sortK[i]); dfree(v->sortV[i]); }
    dfree(v->slot_off);
    v->vis_bytes = 0;
}

vgr_status alloc_vis(vgr_view* v, uint32_t cap) {
    free_vis(v);
    uint64_t b = 0;
    vgr_status s;
    if ((s = dalloc(&v->vis.depth, cap, &b)) ||
        (s = dalloc(&v->vis.ntile, cap, &b)) || (s = dalloc(&v->vis.rect, cap, &b)) ||
        (s = dalloc(&v->vis.recA, cap, &b)) || (s = dalloc(&v->vis.recB, cap, &b)) ||
        (s = dalloc(&v->vis.rgb, cap, &b)) || (s = dalloc(&v->vis.lw, cap, &b)) ||
        (s = dalloc(&v->sortK[0], cap, &b)) ||
        (s = dalloc(&v->sortK[1], cap, &b)) || (s = dalloc(&v->sortV[0], cap, &b)) ||
        (s = dalloc(&v->sortV[1], cap, &b)) || (s = dalloc(&v->slot_off, (size_t)cap + 1, &b))) {
        free_vis(v);
        return s;
    }
    v->cap_vis = cap;
    v->vis_bytes = b;
    return VGR_OK;
}

void free_pairs(vgr_view* v) {
    drop_graphs(v);
    for (int i = 0; i < 2; ++i) { dfree(v->pairK[i]); dfree(v->pairV[i]); }
    v->pair_bytes = 0;
}

vgr_status alloc_pairs(vgr_view* v, uint64_t cap) {
    free_pairs(v);
    uint64_t b = 0;
    vgr_status s;
    if ((s = dalloc(&v->pairK[0], cap, &b)) || (s = dalloc(&v->pairK[1], cap, &b)) ||
        (s = dalloc(&v->pairV[0], cap, &b)) || (s = dalloc(&v->pairV[1], cap, &b))) {
        free_pairs(v);
        return s;
    }
    v->cap_pairs = cap;
    v->pair_bytes = b;
    return VGR_OK;
}

void free_cut(vgr_view* v) {
    drop_graphs(v);
    dfree(v->cut[0]); dfree(v->cut[1]); dfree(v->front_list);
    v->cut_bytes = 0;
}

vgr_status alloc_cut(vgr_view* v, uint32_t cap) {
    free_cut(v);
    uint64_t b = 0;
    vgr_status s;
    if ((s = dalloc(&v->cut[0], cap, &b)) || (s = dalloc(&v->cut[1], cap, &b)) ||
        (s = dalloc(&v->front_list, cap, &b))) {
        free_cut(v);
        return s;
    }
    v->cap_cut = cap;
    v->cut_bytes = b;
    return VGR_OK;
}

// look-back word regions; sized from the current capacities
vgr_status alloc_status(vgr_view* v) {
    drop_graphs(v);
    dfree(v->status);
    const uint32_t RT = radix_tile();
    v->st_compact = 0;
    v->st_front = v->st_compact + cut_compact_tiles(v->n_words) + 1;
    v->st_emit = v->st_front + cut_compact_tiles(v->n_words) + 1;
    v->st_depth = v->st_emit + ceil_div(v->cap_vis, emit_tile()) + 1;
    v->st_depth_stride = (size_t)(ceil_div(v->cap_vis, RT) + 1) * 256;
    v->st_tile = v->st_depth + 4 * v->st_depth_stride;
    v->st_tile_stride = (size_t)(ceil_div(v->cap_pairs, RT) + 1) * 256;
    v->st_words = v->st_tile + 4 * v->st_tile_stride;
    uint64_t b = 0;
    vgr_status s = dalloc(&v->status, v->st_words, &b);
    v->status_bytes = b;
    return s;
}

uint32_t tile_of(const vgr_view* v) { return v->opts.tile_size ? v->opts.tile_size : TILE_DEFAULT; }
uint32_t tiles_for(uint32_t W, uint32_t H, uint32_t T) { return ((W + T - 1) / T) * ((H + T - 1) / T); }

// Wait for every pipelined image copy of the view.
vgr_status wait_copies(vgr_view* v) {
    if (!v->copy_stream) return VGR_OK;
    v->copy_pending[0] = v->copy_pending[1] = false;
    VGR_CK(cudaStreamSynchronize(v->copy_stream));
    return VGR_OK;
}

// The second device image, the copy stream and its events, made on a view's
// first pipelined frame.
vgr_status ensure_pipeline(vgr_view* v) {
    if (!v->copy_stream) VGR_CK(cudaStreamCreateWithFlags(&v->copy_stream, cudaStreamNonBlocking));
    for (auto& e : v->copy_ev)
        if (!e) VGR_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (!v->image_alt) return dalloc(&v->image_alt, (size_t)v->cap_pixels * 3, &v->img_bytes);
    return VGR_OK;
}

vgr_status ensure_image(vgr_view* v, uint32_t W, uint32_t H) {
    const uint32_t T = tile_of(v);
    const uint32_t TW = (W + T - 1) / T, TH = (H + T - 1) / T;
    const uint64_t px = (uint64_t)W * H, tiles = (uint64_t)TW * TH;
    if (px <= v->cap_pixels && tiles <= v->cap_tiles) return VGR_OK;
    vgr_status s = wait_copies(v);  // copies into host memory still read the old images
    if (s != VGR_OK) return s;
    drop_graphs(v);
    dfree(v->image);
    dfree(v->image_alt);
    dfree(v->ranges);
    dfree(v->tile_order);
    v->img_bytes = 0;
    const uint32_t cp = (uint32_t)std::max<uint64_t>(px, v->cap_pixels);
    const uint32_t ct = (uint32_t)std::max<uint64_t>(tiles, v->cap_tiles);
    if ((s = dalloc(&v->image, (size_t)cp * 3, &v->img_bytes)) || (s = dalloc(&v->ranges, ct, &v->img_bytes)) ||
        (s = dalloc(&v->tile_order, ct, &v->img_bytes))) {
        v->cap_pixels = v->cap_tiles = 0;
        return s;
    }
    v->cap_pixels = cp;
    v->cap_tiles = ct;
    return VGR_OK;
}

void destroy_view(vgr_view* v) {
    drop_graphs(v);
    if (v->copy_stream) {
        cudaStreamSynchronize(v->copy_stream);
        cudaStreamDestroy(v->copy_stream);
    }
    for (auto& e : v->copy_ev)
        if (e) cudaEventDestroy(e);
    dfree(v->image_alt);
    free_vis(v);
    free_pairs(v);
    free_cut(v);
    dfree(v->bitmap); dfree(v->front_bm); dfree(v->frontier[0]); dfree(v->frontier[1]);
    dfree(v->ranges); dfree(v->tile_order); dfree(v->image); dfree(v->lut); dfree(v->status);
    dfree(v->ctr); dfree(v->vstate); dfree(v->fp_dev);
    if (v->fp_host) cudaFreeHost(v->fp_host);
    if (v->ctr_host) cudaFreeHost(v->ctr_host);
    if (v->vstate_host) cudaFreeHost(v->vstate_host);
    for (auto& e : v->ev)
        if (e) cudaEventDestroy(e);
    if (v->done_ev) cudaEventDestroy(v->done_ev);
    if (v->join_ev) cudaEventDestroy(v->join_ev);
    forget_batches(v->uid);
    if (v->own_stream && v->stream) cudaStreamDestroy(v->stream);
    delete v;
}

}  // namespace

extern "C" {

vgr_status vgr_create_view(vgr_hierarchy* h, const vgr_view_opts* opts, vgr_view** out) {
    if (!h || !out) return fail(VGR_E_INVALID, "null argument");
    *out = nullptr;
    VGR_CK(cudaSetDevice(h->device));
    vgr_view* v = new vgr_view();
    v->h = h;
    if (opts) v->opts = *opts;
    else vgr_default_view_opts(&v->opts);
    if (v->opts.filter > VGR_FILTER_CANONICAL || v->opts.exp_mode > VGR_EXP_LUT) {
        delete v;
        return fail(VGR_E_INVALID, "bad filter or exp_mode");
    }
    if (v->opts.lut_size == 0) v->opts.lut_size = 32;
    if (v->opts.lut_size > 256) { delete v; return fail(VGR_E_INVALID, "lut_size must be <= 256"); }
    if (v->opts.lod_budget == 0) v->opts.lod_budget = 4096;
    if (v->opts.blend_depth == 0) v->opts.blend_depth = 32;
    if (v->opts.tile_size == 0) v->opts.tile_size = TILE_DEFAULT;
    if (v->opts.blend_depth != 16 && v->opts.blend_depth != 32 && v->opts.blend_depth != 48) {
        delete v;
        return fail(VGR_E_INVALID, "blend_depth must be 16, 32 or 48");
    }
    if (v->opts.tile_size != 8 && v->opts.tile_size != 16 && v->opts.tile_size != 32) {
        delete v;
        return fail(VGR_E_INVALID, "tile_size must be 8, 16 or 32");
    }
    if (v->opts.tile_size == 8 && v->opts.blend_depth == 48) {
        delete v;
        return fail(VGR_E_INVALID, "blend_depth 48 needs tiles of 16 or 32 pixels");
    }
    if (v->opts.lod_frustum && !h->box) {
        delete v;
        return fail(VGR_E_INVALID, "lod_frustum needs node boxes (vgr_scene_desc.bbox)");
    }
    if (v->opts.lod_frustum && !(v->opts.lod_frustum_guard >= 0.f && v->opts.lod_frustum_guard <= 1e6f)) {
        delete v;
        return fail(VGR_E_INVALID, "lod_frustum_guard must be in [0, 1e6] pixels");
    }
    const uint32_t N = h->n_nodes;
    vgr_status s = VGR_OK;
#define VGR_VTRY(x)                 \
    do {                            \
        s = (x);                    \
        if (s != VGR_OK) {          \
            destroy_view(v);        \
            return s;               \
        }                           \
    } while (0)
    if (v->opts.stream) {
        v->stream = (cudaStream_t)v->opts.stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&v->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete v; return fail(VGR_E_CUDA, "stream: %s", cudaGetErrorString(e)); }
        v->own_stream = true;
    }
    v->grid_wide = v->opts.grid_wide ? (int)std::min<uint32_t>(v->opts.grid_wide, 1u << 16) : h->num_sms * 8;
    v->grid_scan = v->opts.grid_scan ? (int)std::min<uint32_t>(v->opts.grid_scan, 1u << 16) : h->num_sms * 4;
    const uint32_t cap_cut = (uint32_t)std::min<uint64_t>(N, v->opts.cut_capacity ? v->opts.cut_capacity
                                                                                  : std::max<uint64_t>(1u << 20, N / 4));
    const uint32_t cap_vis = cap_cut;
    const uint64_t cap_pairs = v->opts.pair_capacity ? v->opts.pair_capacity : (uint64_t)2 * cap_vis;
    VGR_VTRY(alloc_cut(v, cap_cut));
    VGR_VTRY(alloc_vis(v, cap_vis));
    VGR_VTRY(alloc_pairs(v, cap_pairs));
    const uint32_t TW = cut_compact_tile_words();
    v->n_words = (uint32_t)(((uint64_t)(N + 31) / 32 + TW - 1) / TW * TW);
    VGR_VTRY(dalloc(&v->bitmap, v->n_words, &v->fixed_bytes));
    VGR_VTRY(dalloc(&v->front_bm, v->n_words, &v->fixed_bytes));
    VGR_VTRY(dalloc(&v->frontier[0], N, &v->fixed_bytes));
    VGR_VTRY(dalloc(&v->frontier[1], N, &v->fixed_bytes));
    VGR_VTRY(dalloc(&v->ctr, 1, &v->fixed_bytes));
    VGR_VTRY(dalloc(&v->vstate, 1, &v->fixed_bytes));
    VGR_VTRY(dalloc(&v->fp_dev, 1, &v->fixed_bytes));
    VGR_VTRY(dalloc(&v->lut, 260, &v->fixed_bytes));
    VGR_VTRY(alloc_status(v));
    if (cudaMallocHost((void**)&v->fp_host, sizeof(FrameParams)) != cudaSuccess ||
        cudaMallocHost((void**)&v->ctr_host, sizeof(Counters)) != cudaSuccess ||
        cudaMallocHost((void**)&v->vstate_host, sizeof(ViewState)) != cudaSuccess) {
        cudaGetLastError();
        destroy_view(v);
        return fail(VGR_E_NOMEM, "pinned host buffers");
    }
    memset(v->fp_host, 0, sizeof(FrameParams));
    memset(v->ctr_host, 0, sizeof(Counters));
    for (auto& e : v->ev) {
        cudaError_t ce = cudaEventCreate(&e);
        if (ce != cudaSuccess) { destroy_view(v); return fail(VGR_E_CUDA, "event: %s", cudaGetErrorString(ce)); }
    }
    {
        cudaError_t ce = cudaEventCreateWithFlags(&v->done_ev, cudaEventDisableTiming);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&v->join_ev, cudaEventDisableTiming);
        if (ce != cudaSuccess) { destroy_view(v); return fail(VGR_E_CUDA, "event: %s", cudaGetErrorString(ce)); }
        static std::atomic<uint64_t> next_uid{1};
        v->uid = next_uid.fetch_add(1);
    }
    // Eq. 5 table: entry i = e^(-5.55 i / m), i = 0..m
    {
        float host_lut[260] = {0};
        const uint32_t m = v->opts.lut_size;
        for (uint32_t i = 0; i <= m; ++i) host_lut[i] = (float)std::exp(-5.55 * (double)i / (double)m);
        cudaError_t ce = cudaMemcpy(v->lut, host_lut, sizeof(host_lut), cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(cudaStreamLegacy);  // see dalloc
        if (ce != cudaSuccess) { destroy_view(v); return fail(VGR_E_CUDA, "lut: %s", cudaGetErrorString(ce)); }
    }
#undef VGR_VTRY
    *out = v;
    return VGR_OK;
}

vgr_status vgr_destroy_view(vgr_view* v) {
    if (!v) return fail(VGR_E_INVALID, "null view");
    cudaSetDevice(v->h->device);
    if (v->stream) cudaStreamSynchronize(v->stream);
    destroy_view(v);
    return VGR_OK;
}

vgr_status vgr_view_set_tuning(vgr_view* v, uint32_t grid_wide, uint32_t grid_scan, uint32_t blend_depth,
                               uint32_t tile_size) {
    if (!v) return fail(VGR_E_INVALID, "null view");
    if (v->pending) return fail(VGR_E_INVALID, "a frame of this view is in flight");
    if (blend_depth != 0 && blend_depth != 16 && blend_depth != 32 && blend_depth != 48)
        return fail(VGR_E_INVALID, "blend_depth must be 0, 16, 32 or 48");
    if (tile_size != 0 && tile_size != 8 && tile_size != 16 && tile_size != 32)
        return fail(VGR_E_INVALID, "tile_size must be 0, 8, 16 or 32");
    const uint32_t d = blend_depth ? blend_depth : v->opts.blend_depth;
    const uint32_t t = tile_size ? tile_size : v->opts.tile_size;
    if (t == 8 && d == 48) return fail(VGR_E_INVALID, "blend_depth 48 needs tiles of 16 or 32 pixels");
    if (grid_wide) v->grid_wide = (int)std::min<uint32_t>(grid_wide, 1u << 16);
    if (grid_scan) v->grid_scan = (int)std::min<uint32_t>(grid_scan, 1u << 16);
    v->opts.blend_depth = d;
    v->opts.tile_size = t;
    drop_graphs(v);  // captured frames hold the old launch shapes
    return VGR_OK;
}

vgr_status vgr_reset_view(vgr_view* v) {
    if (!v) return fail(VGR_E_INVALID, "null view");
    if (v->pending) return fail(VGR_E_INVALID, "a frame of this view is in flight");
    v->has_prev = false;
    return VGR_OK;
}

vgr_status vgr_view_bytes_estimate(const vgr_hierarchy* h, const vgr_view_opts* opts, uint32_t width,
                                   uint32_t height, uint64_t* bytes) {
    if (!h || !bytes) return fail(VGR_E_INVALID, "null argument");
    vgr_view_opts o;
    if (opts) o = *opts;
    else vgr_default_view_opts(&o);
    // the allocations of vgr_create_view and of the first frame at this size
    const uint64_t N = h->n_nodes;
    const uint64_t cap_cut = std::min<uint64_t>(N, o.cut_capacity ? o.cut_capacity : std::max<uint64_t>(1u << 20, N / 4));
    const uint64_t cap_vis = cap_cut;
    const uint64_t cap_pairs = o.pair_capacity ? o.pair_capacity : 2 * cap_vis;
    const uint64_t TW = cut_compact_tile_words();
    const uint64_t n_words = ((N + 31) / 32 + TW - 1) / TW * TW;
    const uint64_t per_vis = 3 * sizeof(uint32_t) + sizeof(uint2) + 3 * sizeof(float4) + sizeof(float) /* visible SoA */ +
                             sizeof(uint32_t) /* slot offsets */ +
                             4 * sizeof(uint32_t) /* depth-sort ping-pong */ + 3 * sizeof(float4) /* rank records */;
    const uint64_t RT = radix_tile();
    const uint64_t status_words = 2 * (cut_compact_tiles((uint32_t)n_words) + 1) + ceil_div(cap_vis, emit_tile()) + 1 +
                                  4 * (ceil_div(cap_vis, RT) + 1) * 256 + 4 * (ceil_div(cap_pairs, RT) + 1) * 256;
    const uint32_t T = o.tile_size ? o.tile_size : TILE_DEFAULT;
    const uint64_t tiles = (uint64_t)((width + T - 1) / T) * ((height + T - 1) / T);
    uint64_t b = 3 * 4 * cap_cut + per_vis * cap_vis + 4 * 4 * cap_pairs + 2 * 4 * n_words + 2 * 4 * N +
                 sizeof(Counters) + sizeof(ViewState) + sizeof(FrameParams) + 260 * 4 + 8 * status_words;
    b += (uint64_t)width * height * 3 * 4 + tiles * (sizeof(uint2) + 4);
    *bytes = b;
    return VGR_OK;
}

vgr_status vgr_view_device_bytes(const vgr_view* v, uint64_t* bytes) {
    if (!v || !bytes) return fail(VGR_E_INVALID, "null argument");
    *bytes = v->vis_bytes + v->pair_bytes + v->img_bytes + v->fixed_bytes + v->status_bytes + v->cut_bytes;
    return VGR_OK;
}

}  // extern "C"

namespace {

// Digit passes of the tile sort: tile ids 0 .. n_tiles-1 plus the sentinel
// (all ones in the sorted bits) that marks dropped candidate slots.
int tile_passes_for(uint32_t n_tiles) {
    int bits = 0;
    while (bits < 32 && ((uint64_t)1 << bits) <= n_tiles) ++bits;
    return std::max(1, (bits + 7) / 8);
}

// The emission's grid relative to the look-back kernels' (x/4): four CTAs
// per SM, like the radix passes (with room for 54 registers a thread it ran
// 0.199 ms on the city against 0.221 at six CTAs per SM and 40 registers).
constexpr int EMIT_GRID_NUM = 4;

uint32_t frame_kernels(const vgr_view* v, bool scratch, int tile_passes) {
    const uint32_t lod = scratch ? v->h->max_depth + 1u : 1u;
    return lod + 1u /*compact*/ + 1u /*preprocess, with colour*/ + 4u /*depth passes*/ +
           2u /*slot scan, emit*/ + (uint32_t)tile_passes + 1u /*tile order (finishes the ranges)*/ + 1u /*blend*/;
}

// The frame's status block and cut sizes, read back after its last kernel.
void frame_readback(vgr_view* v, cudaStream_t s) {
    cudaMemcpyAsync(v->ctr_host, v->ctr, COUNTERS_HEAD, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(v->vstate_host, v->vstate, sizeof(ViewState), cudaMemcpyDeviceToHost, s);
}

// Enqueue one frame.  'scratch' selects the top-down cut.  'own_blend' false:
// the frame stops before the blend, which a batch runs over all its views
// (frame_readback then follows that blend).  Returns the number of kernels
// launched.
uint32_t enqueue_frame(vgr_view* v, bool scratch, int tile_passes, bool own_blend = true) {
    const SceneDev& sc = v->h->dev;
    cudaStream_t s = v->stream;
    const bool timing = v->opts.timing != 0;
    auto mark = [&](int i) { if (timing) cudaEventRecord(v->ev[i], s); };
    const FrameParams& fh = *v->fp_host;
    const uint32_t n_tiles = fh.tiles_x * fh.tiles_y;
    cudaMemcpyAsync(v->fp_dev, v->fp_host, sizeof(FrameParams), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(v->ctr, 0, sizeof(Counters), s);
    cudaMemsetAsync(v->ranges, 0xFF, (size_t)n_tiles * sizeof(uint2), s);  // (start, ~end): both all ones
    // the first kernel waits for the copies above in plain stream order; with
    // stage events between the kernels none of them is launched early
    PdlScope pdl(!timing);
    const int prev = v->parity, cur = v->parity ^ 1;
    mark(VGR_STAGE_LOD);
    if (scratch) {
        for (uint32_t level = 0; level <= v->h->max_depth; ++level)
            launch_lod_level((int)level, sc, v->frontier[level & 1], v->frontier[(level + 1) & 1], v->h->n_nodes,
                             v->fp_dev, v->bitmap, v->front_bm, v->ctr, v->grid_wide, fh.lod_frustum != 0,
                             fh.lod_interp != 0, s);
    } else {
        launch_lod_update(sc, v->cut[prev], &v->vstate->n_cut[prev], v->cap_cut, v->fp_dev, v->bitmap, v->front_bm,
                          v->ctr, v->grid_wide, fh.lod_frustum != 0, fh.lod_interp != 0, s);
    }
    mark(VGR_STAGE_COMPACT);
    launch_cut_compact(v->bitmap, v->front_bm, v->n_words, v->cut[cur], v->front_list, v->cap_cut,
                       &v->vstate->n_cut[cur], v->status + v->st_compact, v->status + v->st_front, v->ctr, v->fp_dev,
                       v->grid_scan, s);
    mark(VGR_STAGE_PREPROCESS);
    launch_preprocess(sc, v->front_list, &v->ctr->n_front, v->cap_cut, v->fp_dev, v->vis, v->ctr, fh.lod_interp != 0,
                      v->grid_wide, s);
    mark(VGR_STAGE_DEPTH_SORT);
    // every potentially visible entry is sorted; culled ones carry the key
    // 0xFFFFFFFF and land last (the digit histograms come from preprocess)
    for (int p = 0; p < 4; ++p) {
        const uint32_t* kin = p == 0 ? v->vis.depth : v->sortK[(p + 1) & 1];
        const uint32_t* vin = p == 0 ? nullptr : v->sortV[(p + 1) & 1];
        // the last pass writes only the permutation (the sorted keys are not read)
        launch_radix_pass(kin, vin, p == 3 ? nullptr : v->sortK[p & 1], v->sortV[p & 1], &v->ctr->n_front, nullptr,
                          v->cap_vis, 8 * p,
                          v->ctr->depth_hist[p], v->status + v->st_depth + p * v->st_depth_stride,
                          &v->ctr->tickets[TK_SORT0 + p], v->fp_dev, v->ctr, v->grid_scan, s, p == 3 ? 1 : 0);
    }
    const uint32_t* order = v->sortV[1];  // after 4 passes
    mark(VGR_STAGE_COLOR);  // (evaluated in preprocess: the stage is empty)
    mark(VGR_STAGE_EMIT);
    const uint32_t sentinel = (uint32_t)((1ull << (8 * tile_passes)) - 1ull);
    launch_emit(order, v->cap_vis, v->vis, v->slot_off, v->pairK[0], v->pairV[0], v->cap_pairs, tile_passes, sentinel,
                v->status + v->st_emit, v->ctr, v->fp_dev, v->grid_scan, v->grid_scan * EMIT_GRID_NUM / 4, s);
    mark(VGR_STAGE_TILE_SORT);
    // (the last pass also records each tile's range)
    for (int p = 0; p < tile_passes; ++p) {
        const bool last = p + 1 == tile_passes;
        launch_radix_pass(v->pairK[p & 1], v->pairV[p & 1], v->pairK[(p + 1) & 1], v->pairV[(p + 1) & 1], nullptr,
                          &v->ctr->n_cand, v->cap_pairs, 8 * p, v->ctr->tile_hist[p],
                          v->status + v->st_tile + p * v->st_tile_stride, &v->ctr->tickets[TK_SORT0 + 4 + p],
                          v->fp_dev, v->ctr, v->grid_scan, s, last ? 1 : 0, last ? v->ranges : nullptr, n_tiles);
    }
    v->last_tile_buf = tile_passes & 1;
    mark(VGR_STAGE_RANGES);
    launch_tile_order(v->ranges, n_tiles, v->tile_order, v->ctr, s);
    if (!own_blend) return frame_kernels(v, scratch, tile_passes) - 1u;  // a batch blend follows
    mark(VGR_STAGE_BLEND);
    launch_blend(v->fp_dev, nullptr, v->tile_order, n_tiles, &v->ctr->blend_next,
                 v->h->num_sms * blend_ctas_per_sm(v->opts.filter, v->opts.exp_mode, v->opts.blend_depth, fh.tile),
                 v->opts.filter, v->opts.exp_mode, v->opts.blend_depth, fh.tile, s);
    mark(VGR_N_STAGES);
    frame_readback(v, s);
    return frame_kernels(v, scratch, tile_passes);
}

// One frame on the view's stream: the plain launch sequence, or (use_graph,
// no stage timing) the replay of the captured sequence for this
// (top-down?, parity) pair, captured on first use.
vgr_status run_frame(vgr_view* v, bool scratch, int tile_passes, uint32_t n_tiles, uint32_t* kernels) {
    if (!v->opts.use_graph || v->opts.timing) {
        *kernels += enqueue_frame(v, scratch, tile_passes);
        VGR_CK(cudaGetLastError());
        return VGR_OK;
    }
    if (v->graph_tiles != n_tiles) {
        drop_graphs(v);
        v->graph_tiles = n_tiles;
    }
    cudaGraphExec_t& ge = v->graph[scratch ? 1 : 0][v->parity];
    if (!ge) {
        VGR_CK(cudaStreamBeginCapture(v->stream, cudaStreamCaptureModeThreadLocal));
        enqueue_frame(v, scratch, tile_passes);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(v->stream, &g);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ge = nullptr;
            cudaGetLastError();
            return fail(VGR_E_CUDA, "frame capture: %s", cudaGetErrorString(e));
        }
    }
    v->last_tile_buf = tile_passes & 1;
    VGR_CK(cudaGraphLaunch(ge, v->stream));
    *kernels += frame_kernels(v, scratch, tile_passes);
    return VGR_OK;
}

vgr_status check_camera(const vgr_camera* c, float tau) {
    if (!c) return fail(VGR_E_INVALID, "null camera");
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(c->R[i])) return fail(VGR_E_INVALID, "camera R not finite");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(c->pos[i])) return fail(VGR_E_INVALID, "camera position not finite");
    if (!(c->fx > 0.f) || !(c->fy > 0.f) || !std::isfinite(c->fx) || !std::isfinite(c->fy))
        return fail(VGR_E_INVALID, "focal lengths must be positive");
    if (!std::isfinite(c->cx) || !std::isfinite(c->cy)) return fail(VGR_E_INVALID, "principal point not finite");
    if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384)
        return fail(VGR_E_INVALID, "image size must be in [1, 16384]");
    if (!(c->z_near > 0.f) || !std::isfinite(c->z_near)) return fail(VGR_E_INVALID, "z_near must be > 0");
    const float f = std::max(c->fx, c->fy);
    if (!(tau >= 0.f) || !(tau <= f)) return fail(VGR_E_INVALID, "tau must be in [0, max(fx, fy)]");
    return VGR_OK;
}

// Device address of a host image buffer the GPU can write directly (pinned
// memory of this device), or null: then the image is copied after the frame.
float* mapped_host(const vgr_view* v, float* host) {
    if (!host) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer || a.device != v->h->device) return nullptr;
    return static_cast<float*>(a.devicePointer);
}

// Planes of the frustum-aware granularity test.  Camera-space inward
// normals a with camera-space offset o_c (near: a = (0, 0, 1), o_c = z_near;
// the sides pass through the camera centre and the image edges moved out by
// g pixels: left (fx, 0, cx + g), right (-fx, 0, W - cx + g), top
// (0, fy, cy + g), bottom (0, -fy, H - cy + g), o_c = 0).  With p_cam =
// R (x - pos) the world normal is w = R^T a and the offset o = w . pos + o_c:
//   w_j = fl32(fma(R2j, a2, fma(R1j, a1, R0j a0)))   (FP64, correctly rounded fma)
//   o   = fl32(fma(w2, pos2, fma(w1, pos1, w0 pos0)) + o_c)
// Explicit fmas keep the values identical on every host compiler.
void frustum_planes(const vgr_camera* cam, float guard, float out[5][4]) {
    const double g = guard, fx = cam->fx, fy = cam->fy, cx = cam->cx, cy = cam->cy;
    const double W = cam->width, H = cam->height;
    const double a[5][4] = {{0.0, 0.0, 1.0, (double)cam->z_near},
                            {fx, 0.0, cx + g, 0.0},
                            {-fx, 0.0, (W - cx) + g, 0.0},
                            {0.0, fy, cy + g, 0.0},
                            {0.0, -fy, (H - cy) + g, 0.0}};
    const float* R = cam->R;
    for (int i = 0; i < 5; ++i) {
        float w[3];
        for (int j = 0; j < 3; ++j)
            w[j] = (float)std::fma((double)R[6 + j], a[i][2],
                                   std::fma((double)R[3 + j], a[i][1], (double)R[j] * a[i][0]));
        const double o = std::fma((double)w[2], (double)cam->pos[2],
                                  std::fma((double)w[1], (double)cam->pos[1], (double)w[0] * (double)cam->pos[0]));
        out[i][0] = w[0];
        out[i][1] = w[1];
        out[i][2] = w[2];
        out[i][3] = (float)(o + a[i][3]);
    }
}

void fill_params(vgr_view* v, const vgr_camera* cam, float t, float k, float* host_dev, int tile_passes) {
    const uint32_t W = cam->width, H = cam->height;
    FrameParams& p = *v->fp_host;
    memcpy(p.R, cam->R, sizeof(p.R));
    memcpy(p.pos, cam->pos, sizeof(p.pos));
    p.fx = cam->fx; p.fy = cam->fy; p.cx = cam->cx; p.cy = cam->cy;
    p.z_near = cam->z_near;
    p.k = k;
    p.limx = 1.3f * (0.5f * (float)W / cam->fx);
    p.limy = 1.3f * (0.5f * (float)H / cam->fy);
    p.width_f = (float)W; p.height_f = (float)H;
    p.width = W; p.height = H;
    p.tile = tile_of(v);
    p.tiles_x = (W + p.tile - 1) / p.tile; p.tiles_y = (H + p.tile - 1) / p.tile;
    p.epoch = ++v->epoch;  // fresh look-back tags for every launch sequence
    if ((p.epoch & 0x3FFFFFFFu) == 0) p.epoch = ++v->epoch;
    p.filter = v->opts.filter; p.exp_mode = v->opts.exp_mode; p.lut_size = v->opts.lut_size;
    p.lut_step = 5.55f / (float)v->opts.lut_size;
    p.lod_budget = v->opts.lod_budget;
    p.max_depth = v->h->max_depth;
    p.host_image = host_dev;
    p.test_hooks = v->opts.test_hooks;
    p.lod_frustum = v->opts.lod_frustum ? 1u : 0u;
    p.lod_interp = v->opts.lod_interp ? 1u : 0u;
    p.lod_t = t;
    if (p.lod_frustum) frustum_planes(cam, v->opts.lod_frustum_guard, p.frustum);
    // the blend's buffers: the tile sort's last pass leaves the pairs in
    // buffer (passes & 1)
    p.bl_ranges = v->ranges;
    p.bl_pair_val = v->pairV[tile_passes & 1];
    p.bl_recA = v->vis.recA;
    p.bl_recB = v->vis.recB;
    p.bl_rgb = v->vis.rgb;
    p.bl_lut = v->lut;
    p.bl_image = v->cur_image;
    p.bl_ctr = v->ctr;
}

// Enqueue the frame (and the image copy to host_rgb, if given) and record the
// view's completion event; nothing waits.
// Validate a frame and set up its parameters (pinned fp_host) without
// launching anything.
vgr_status prepare_frame(vgr_view* v, const vgr_camera* cam, float tau, float* host_rgb, bool pipe = false) {
    if (!v) return fail(VGR_E_INVALID, "null view");
    if (v->pending) return fail(VGR_E_INVALID, "a frame of this view is already in flight");
    if (v->broken) return fail(VGR_E_NOMEM, "a buffer of this view could not be grown; destroy the view");
    vgr_status s = check_camera(cam, tau);
    if (s != VGR_OK) return s;
    VGR_CK(cudaSetDevice(v->h->device));
    const uint32_t W = cam->width, H = cam->height;
    const uint32_t T = tile_of(v);
    if (T == 8 && (W > 8192 || H > 8192))
        return fail(VGR_E_INVALID, "8-pixel tiles need an image of at most 8192 x 8192");
    if ((s = ensure_image(v, W, H)) != VGR_OK) return s;
    if (pipe && (s = ensure_pipeline(v)) != VGR_OK) return s;
    const uint32_t TW = (W + T - 1) / T, TH = (H + T - 1) / T;
    PendingFrame& q = v->pend;
    q = PendingFrame{};
    q.pipe = pipe;
    q.img = pipe ? v->img_sel : 0;
    if (v->copy_pending[q.img]) {
        // the image this frame overwrites is still being copied out: a
        // pipelined frame waits for it on the device, any other frame (which
        // may run on a batch stream) on the host
        if (pipe) {
            VGR_CK(cudaStreamWaitEvent(v->stream, v->copy_ev[q.img], 0));
        } else {
            VGR_CK(cudaEventSynchronize(v->copy_ev[q.img]));
            v->copy_pending[q.img] = false;
        }
    }
    v->cur_image = q.img ? v->image_alt : v->image;
    q.cam = *cam;
    q.tau = tau;
    q.host = host_rgb;
    q.tile_passes = tile_passes_for(TW * TH);
    volatile float f = std::max(cam->fx, cam->fy);
    volatile float t = tau / f;
    volatile float k = t * t;
    q.f = f;
    q.t = t;
    q.k = k;
    q.scratch = !v->has_prev || !v->opts.temporal || tau != v->prev_tau || q.f != v->prev_f;
    q.host_dev = pipe ? nullptr : mapped_host(v, host_rgb);
    fill_params(v, cam, q.t, q.k, q.host_dev, q.tile_passes);
    return VGR_OK;
}

// After the frame's kernels (on stream s): the host copy when the blend does
// not write the host buffer itself, and the completion event.
vgr_status close_frame(vgr_view* v, cudaStream_t s) {
    PendingFrame& q = v->pend;
    if (q.host && !q.host_dev && !q.pipe)
        VGR_CK(cudaMemcpyAsync(q.host, v->cur_image, (size_t)q.cam.width * q.cam.height * 3 * sizeof(float),
                               cudaMemcpyDeviceToHost, s));
    VGR_CK(cudaEventRecord(v->done_ev, s));
    v->pending = true;
    return VGR_OK;
}

// NVTX range for tools that show the host timeline (ncu --nvtx, Nsight Systems)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

vgr_status submit_impl(vgr_view* v, const vgr_camera* cam, float tau, float* host_rgb, bool pipe = false) {
    NvtxRange r("vgr submit frame");
    vgr_status s = prepare_frame(v, cam, tau, host_rgb, pipe);
    if (s != VGR_OK) return s;
    PendingFrame& q = v->pend;
    if ((s = run_frame(v, q.scratch, q.tile_passes, tiles_for(q.cam.width, q.cam.height, tile_of(v)), &q.kernels)) !=
        VGR_OK)
        return s;
    return close_frame(v, v->stream);
}

// Per device: the stream batches are launched on and its fork event.
struct BatchStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr;
};
BatchStream g_bstream[64];

// Views whose blend joins the batch's single blend launch: the exact
// exponential and the preemptive filter (the kernel's default mode), at the
// first such view's staging depth and tile size, at most BATCH_VIEWS_MAX of
// them; the others blend in their own branch.
std::vector<uint32_t> batch_blend_views(vgr_view* const* views, uint32_t n) {
    std::vector<uint32_t> sh;
    uint32_t depth = 0, tile = 0;
    for (uint32_t i = 0; i < n && sh.size() < BATCH_VIEWS_MAX; ++i) {
        const vgr_view_opts& o = views[i]->opts;
        if (o.filter != VGR_FILTER_PREEMPTIVE || o.exp_mode != VGR_EXP_EXACT) continue;
        if (!depth) {
            depth = o.blend_depth;
            tile = o.tile_size;
        }
        if (o.blend_depth == depth && o.tile_size == tile) sh.push_back(i);
    }
    return sh;
}

// All views prepared: run their frames as one captured graph (captured on
// first use of this combination).  Each view's frame up to its tile order is
// a parallel branch on the view's stream; then one launch orders the tiles
// of all the views heaviest first and one persistent blend shades them all.
vgr_status launch_batch_graph(vgr_view* const* views, uint32_t n) {
    NvtxRange r("vgr batch graph");
    const int dev = views[0]->h->device;
    if (dev < 0 || dev >= 64) return fail(VGR_E_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchStream& bs = g_bstream[dev];
    if (!bs.s) {
        VGR_CK(cudaStreamCreateWithFlags(&bs.s, cudaStreamNonBlocking));
        VGR_CK(cudaEventCreateWithFlags(&bs.fork, cudaEventDisableTiming));
    }
    // the views' chains: largest image first, each to the chain with the
    // fewest pixels so far; a view follows the previous view of its chain
    const uint32_t k = g_batch_chains.load() == 0 ? n : std::min(n, g_batch_chains.load());
    std::vector<uint32_t> order(n);
    for (uint32_t i = 0; i < n; ++i) order[i] = i;
    auto pixels = [&](uint32_t i) { return (uint64_t)views[i]->pend.cam.width * views[i]->pend.cam.height; };
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return pixels(a) > pixels(b); });
    std::vector<uint64_t> load(k, 0);
    std::vector<int> chain_last(k, -1), prev(n, -1);
    std::vector<char> tail(n, 0);
    for (uint32_t i : order) {
        const uint32_t c = (uint32_t)(std::min_element(load.begin(), load.end()) - load.begin());
        prev[i] = chain_last[c];
        chain_last[c] = (int)i;
        load[c] += pixels(i);
    }
    for (int i : chain_last)
        if (i >= 0) tail[i] = 1;
    std::vector<uint64_t> key;
    key.reserve((size_t)n * 6 + 1);
    key.push_back(k);
    for (uint32_t i = 0; i < n; ++i) {
        const vgr_view* v = views[i];
        const PendingFrame& q = v->pend;
        const uint64_t tiles = tiles_for(q.cam.width, q.cam.height, tile_of(v));
        key.insert(key.end(), {v->uid, v->gen, (uint64_t)q.scratch, (uint64_t)v->parity, tiles,
                               (uint64_t)q.tile_passes});
    }
    const std::vector<uint32_t> sh = batch_blend_views(views, n);
    std::vector<char> shared(n, 0);
    for (uint32_t i : sh) shared[i] = 1;
    BatchGraph* bg = nullptr;
    for (auto& b : g_batches)
        if (b.key == key) bg = &b;
    if (!bg) {
        // the batch blend's table: per shared view its frame parameters and
        // tile order, the first tile of each view in the batch's tile count,
        // the per-(class, view) offsets, and the work list
        const uint32_t ns = (uint32_t)sh.size();
        std::vector<const FrameParams*> fps(ns);
        std::vector<const uint32_t*> orders(ns);
        std::vector<uint32_t> base(ns + 1, 0);
        for (uint32_t j = 0; j < ns; ++j) {
            const vgr_view* v = views[sh[j]];
            const uint32_t tiles = tiles_for(v->pend.cam.width, v->pend.cam.height, tile_of(v));
            fps[j] = v->fp_dev;
            orders[j] = v->tile_order;
            base[j + 1] = base[j] + tiles;
        }
        const uint32_t total = base[ns];
        const size_t off_orders = 8 * (size_t)ns, off_base = 16 * (size_t)ns,
                     off_delta = (off_base + 4 * (size_t)(ns + 1) + 15) / 16 * 16,
                     off_work = off_delta + 4 * 33 * (size_t)ns, off_next = off_work + 4 * (size_t)total,
                     bytes = off_next + 16;
        void* devbuf = nullptr;
        if (ns) {
            cudaError_t e = cudaMalloc(&devbuf, bytes);
            if (e == cudaSuccess) e = cudaMemcpy(devbuf, fps.data(), 8 * (size_t)ns, cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy((char*)devbuf + off_orders, orders.data(), 8 * (size_t)ns, cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy((char*)devbuf + off_base, base.data(), 4 * (size_t)(ns + 1), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                if (devbuf) cudaFree(devbuf);
                cudaGetLastError();
                return fail(e == cudaErrorMemoryAllocation ? VGR_E_NOMEM : VGR_E_CUDA, "batch blend table: %s",
                            cudaGetErrorString(e));
            }
        }
        VGR_CK(cudaStreamBeginCapture(bs.s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaEventRecord(bs.fork, bs.s);
        for (uint32_t i : order) {  // a view's predecessor in its chain is captured before it
            if (e != cudaSuccess) break;
            vgr_view* v = views[i];
            e = cudaStreamWaitEvent(v->stream, prev[i] < 0 ? bs.fork : views[prev[i]]->join_ev, 0);
            if (e != cudaSuccess) break;
            enqueue_frame(v, v->pend.scratch, v->pend.tile_passes, !shared[i]);
            e = cudaEventRecord(v->join_ev, v->stream);
            if (e == cudaSuccess && tail[i]) e = cudaStreamWaitEvent(bs.s, v->join_ev, 0);
        }
        if (e == cudaSuccess && ns) {
            PdlScope pdl(true);  // the first kernel follows the joins in plain stream order
            auto* fps_d = reinterpret_cast<const FrameParams* const*>(devbuf);
            auto* orders_d = reinterpret_cast<const uint32_t* const*>((char*)devbuf + off_orders);
            auto* base_d = reinterpret_cast<const uint32_t*>((char*)devbuf + off_base);
            auto* delta_d = reinterpret_cast<uint32_t*>((char*)devbuf + off_delta);
            auto* work_d = reinterpret_cast<uint32_t*>((char*)devbuf + off_work);
            auto* next_d = reinterpret_cast<uint32_t*>((char*)devbuf + off_next);
            const vgr_view* v0 = views[sh[0]];
            const uint32_t d = v0->opts.blend_depth, t = v0->opts.tile_size;
            e = cudaMemsetAsync(next_d, 0, sizeof(uint32_t), bs.s);  // the blend's tile counter
            launch_batch_order(fps_d, ns, orders_d, base_d, total, delta_d, work_d, v0->h->num_sms * 4, bs.s);
            launch_blend(v0->fp_dev, fps_d, work_d, total, next_d,
                         v0->h->num_sms * blend_ctas_per_sm(VGR_FILTER_PREEMPTIVE, VGR_EXP_EXACT, d, t),
                         VGR_FILTER_PREEMPTIVE, VGR_EXP_EXACT, d, t, bs.s);
            for (uint32_t j = 0; j < ns; ++j) frame_readback(views[sh[j]], bs.s);
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(bs.s, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGetLastError();
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (devbuf) cudaFree(devbuf);
            return fail(VGR_E_CUDA, "batch capture: %s", cudaGetErrorString(e));
        }
        if (g_batches.size() >= BATCH_GRAPHS_KEPT) {  // evict the least recently used
            size_t old = 0;
            for (size_t i = 1; i < g_batches.size(); ++i)
                if (g_batches[i].last_use < g_batches[old].last_use) old = i;
            destroy_batch(g_batches[old]);
            g_batches.erase(g_batches.begin() + (long)old);
        }
        g_batches.push_back(BatchGraph{key, exec, 0, devbuf});
        bg = &g_batches.back();
    }
    bg->last_use = ++g_batch_clock;
    VGR_CK(cudaGraphLaunch(bg->exec, bs.s));
    for (uint32_t i = 0; i < n; ++i) {
        vgr_view* v = views[i];
        v->last_tile_buf = v->pend.tile_passes & 1;
        v->pend.kernels += frame_kernels(v, v->pend.scratch, v->pend.tile_passes) - (shared[i] ? 1u : 0u);
        if (!sh.empty() && i == sh[0]) v->pend.kernels += 3u;  // class offsets, tile placement, the batch blend
        vgr_status s = close_frame(v, bs.s);
        if (s != VGR_OK) return s;
    }
    return VGR_OK;
}

// Wait for the submitted frame, read its status, replay it when the
// temporal update fell back or a buffer overflowed, and commit the view's
// temporal state.
vgr_status finish_impl(vgr_view* v, vgr_frame* out) {
    NvtxRange r("vgr finish frame");
    if (!v) return fail(VGR_E_INVALID, "null view");
    if (!v->pending) return fail(VGR_E_INVALID, "no frame of this view is in flight");
    v->pending = false;
    VGR_CK(cudaSetDevice(v->h->device));
    PendingFrame& q = v->pend;
    const uint32_t W = q.cam.width, H = q.cam.height;
    const uint32_t T = tile_of(v);
    const uint32_t TW = (W + T - 1) / T, TH = (H + T - 1) / T;
    const Counters* ch = reinterpret_cast<const Counters*>(v->ctr_host);
    VGR_CK(cudaEventSynchronize(v->done_ev));
    vgr_status s = VGR_OK;
    uint32_t replays = 0;
    for (int attempt = 0;; ++attempt) {
        const uint32_t flags = ch->flags;
        const int cur = v->parity ^ 1;
        const uint32_t n_cut = v->vstate_host->n_cut[cur];
        if (flags & F_SPIN_TIMEOUT) return fail(VGR_E_TIMEOUT, "a look-back wait timed out");
        if (flags & F_NONMONOTONE)
            return fail(VGR_E_NONMONOTONE, "granularity test not monotone: a child expands while its parent does not");
        if (flags & F_OVF_FRONTIER) return fail(VGR_E_OVERFLOW, "frontier overflow");
        if (flags & F_OVF_VIS) return fail(VGR_E_OVERFLOW, "more than 2^24 cut nodes in front of the camera in one frame");
        bool again = false;
        if ((flags & F_LOD_FALLBACK) && !q.scratch) {
            q.scratch = true;
            again = true;
        } else if (flags & F_LOD_FALLBACK) {
            return fail(VGR_E_TIMEOUT, "top-down cut exceeded the tree depth");
        } else if (flags & F_OVF_CUT) {
            const uint32_t nc = (uint32_t)std::min<uint64_t>(v->h->n_nodes, (uint64_t)n_cut + n_cut / 4 + 1024);
            if ((s = alloc_cut(v, nc)) != VGR_OK || (s = alloc_vis(v, nc)) != VGR_OK || (s = alloc_status(v)) != VGR_OK) {
                v->broken = true;
                return s;
            }
            q.scratch = true;  // the previous cut lived in the old buffers
            again = true;
        } else if (flags & F_OVF_PAIRS) {
            const uint64_t np = ch->n_cand + ch->n_cand / 4 + 4096;
            if (np >= 0xFFFFFFFFull) return fail(VGR_E_OVERFLOW, "more than 2^32 pairs");
            if ((s = alloc_pairs(v, np)) != VGR_OK || (s = alloc_status(v)) != VGR_OK) {
                v->broken = true;
                return s;
            }
            again = true;
        }
        if (!again) break;
        if (attempt >= 12) return fail(VGR_E_OVERFLOW, "frame did not settle after %d replays", attempt + 1);
        ++replays;
        fill_params(v, &q.cam, q.t, q.k, q.host_dev, q.tile_passes);
        if ((s = run_frame(v, q.scratch, q.tile_passes, TW * TH, &q.kernels)) != VGR_OK) return s;
        if (q.host && !q.host_dev && !q.pipe)
            VGR_CK(cudaMemcpyAsync(q.host, v->cur_image, (size_t)W * H * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                                   v->stream));
        VGR_CK(cudaStreamSynchronize(v->stream));
    }
    if (q.pipe) {
        // the frame has finished (done_ev, or the replay's synchronize): its
        // image goes out on the copy stream while the next frame runs
        VGR_CK(cudaStreamWaitEvent(v->copy_stream, v->done_ev, 0));
        VGR_CK(cudaMemcpyAsync(q.host, v->cur_image, (size_t)W * H * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                               v->copy_stream));
        VGR_CK(cudaEventRecord(v->copy_ev[q.img], v->copy_stream));
        v->copy_pending[q.img] = true;
        v->img_sel ^= 1;
    }
    const int cur = v->parity ^ 1;
    v->parity = cur;
    v->has_prev = true;
    v->prev_tau = q.tau;
    v->prev_f = q.f;
    v->last_w = W; v->last_h = H; v->last_tw = TW; v->last_th = TH;
    v->last_n_cut = v->vstate_host->n_cut[cur];
    v->last_n_vis = ch->n_vis;
    v->last_n_front = ch->n_front;
    v->last_n_pairs = ch->n_pairs;
    if (out) {
        memset(out, 0, sizeof(*out));
        out->image = v->cur_image;
        out->cut = v->cut[cur];
        out->cut_count = v->last_n_cut;
        out->width = W;
        out->height = H;
        vgr_frame_stats& st = out->stats;
        st.cut_count = v->last_n_cut;
        st.front_count = ch->n_front;
        st.visible_count = ch->n_vis;
        st.pair_count = ch->n_pairs;
        st.candidate_pairs = ch->n_cand;
        st.nodes_evaluated = ch->nodes_eval;
        st.lod_from_scratch = q.scratch ? 1u : 0u;
        st.replays = replays;
        st.kernels = q.kernels;
        st.pixel_pair_evals = ch->pix_evals;
        st.pixel_pair_contribs = ch->pix_contribs;
        if (v->opts.timing) {
            for (int i = 0; i < VGR_N_STAGES; ++i) cudaEventElapsedTime(&st.stage_ms[i], v->ev[i], v->ev[i + 1]);
            cudaEventElapsedTime(&st.frame_ms, v->ev[0], v->ev[VGR_N_STAGES]);
        }
    }
    return VGR_OK;
}

vgr_status render_impl(vgr_view* v, const vgr_camera* cam, float tau, float* host_rgb, vgr_frame* out,
                       bool pipe = false) {
    vgr_status s = submit_impl(v, cam, tau, host_rgb, pipe);
    if (s != VGR_OK) return s;
    return finish_impl(v, out);
}

}  // namespace

extern "C" {

vgr_status vgr_render_frame(vgr_view* v, const vgr_camera* cam, float tau, vgr_frame* out) {
    return render_impl(v, cam, tau, nullptr, out);
}

vgr_status vgr_render_frame_host(vgr_view* v, const vgr_camera* cam, float tau, float* host_rgb, vgr_frame* out) {
    if (!host_rgb) return fail(VGR_E_INVALID, "null host image");
    return render_impl(v, cam, tau, host_rgb, out);
}

vgr_status vgr_render_frame_pipelined(vgr_view* v, const vgr_camera* cam, float tau, float* host_rgb,
                                      vgr_frame* out) {
    if (!host_rgb) return fail(VGR_E_INVALID, "null host image");
    return render_impl(v, cam, tau, host_rgb, out, true);
}

vgr_status vgr_wait_host_images(vgr_view* v) {
    if (!v) return fail(VGR_E_INVALID, "null view");
    VGR_CK(cudaSetDevice(v->h->device));
    return wait_copies(v);
}

vgr_status vgr_submit_frame(vgr_view* v, const vgr_camera* cam, float tau, float* host_rgb) {
    return submit_impl(v, cam, tau, host_rgb);
}

vgr_status vgr_frame_done(vgr_view* v, int* done) {
    if (!v || !done) return fail(VGR_E_INVALID, "null argument");
    if (!v->pending) return fail(VGR_E_INVALID, "no frame of this view is in flight");
    const cudaError_t e = cudaEventQuery(v->done_ev);
    if (e == cudaErrorNotReady) { *done = 0; return VGR_OK; }
    if (e != cudaSuccess) return fail(VGR_E_CUDA, "cudaEventQuery: %s", cudaGetErrorString(e));
    *done = 1;
    return VGR_OK;
}

vgr_status vgr_finish_frame(vgr_view* v, vgr_frame* out) { return finish_impl(v, out); }

vgr_status vgr_render_batch(vgr_view* const* views, const vgr_camera* cams, const float* taus,
                            float* const* host_rgb, uint32_t n, vgr_frame* outs) {
    if (n == 0) return VGR_OK;
    if (!views || !cams || !taus) return fail(VGR_E_INVALID, "null argument");
    for (uint32_t i = 0; i < n; ++i) {
        if (!views[i]) return fail(VGR_E_INVALID, "views[%u] is null", i);
        for (uint32_t j = 0; j < i; ++j)
            if (views[j] == views[i]) return fail(VGR_E_INVALID, "views[%u] and views[%u] are the same view", j, i);
    }
    // every view replaying captured frames on its own stream, none in flight:
    // one graph for the whole batch
    bool whole = n >= 2;
    for (uint32_t i = 0; i < n && whole; ++i) {
        const vgr_view* v = views[i];
        whole = v->opts.use_graph && !v->opts.timing && !v->pending && v->own_stream &&
                v->h->device == views[0]->h->device;
    }
    if (whole) {
        uint32_t prepared = 0;
        vgr_status s = VGR_OK;
        for (; prepared < n; ++prepared) {
            s = prepare_frame(views[prepared], &cams[prepared], taus[prepared], host_rgb ? host_rgb[prepared] : nullptr);
            if (s != VGR_OK) return s;  // nothing has been launched
        }
        if ((s = launch_batch_graph(views, n)) != VGR_OK) {
            for (uint32_t i = 0; i < n; ++i)
                if (views[i]->pending) {  // launched: wait for it, keep the first error
                    const std::string msg = g_err;
                    finish_impl(views[i], nullptr);
                    g_err = msg;
                }
            return s;
        }
        vgr_status first = VGR_OK;
        std::string first_msg;
        for (uint32_t i = 0; i < n; ++i) {
            const vgr_status f = finish_impl(views[i], outs ? &outs[i] : nullptr);
            if (f != VGR_OK && first == VGR_OK) { first = f; first_msg = g_err; }
        }
        if (first != VGR_OK) g_err = first_msg;
        return first;
    }
    // otherwise submit every view, then finish them in order; on a failed
    // submission the views already submitted are still finished
    uint32_t submitted = 0;
    vgr_status first = VGR_OK;
    std::string first_msg;
    for (; submitted < n; ++submitted) {
        const vgr_status s = submit_impl(views[submitted], &cams[submitted], taus[submitted],
                                         host_rgb ? host_rgb[submitted] : nullptr);
        if (s != VGR_OK) { first = s; first_msg = g_err; break; }
    }
    for (uint32_t i = 0; i < submitted; ++i) {
        const vgr_status s = finish_impl(views[i], outs ? &outs[i] : nullptr);
        if (s != VGR_OK && first == VGR_OK) { first = s; first_msg = g_err; }
    }
    if (first != VGR_OK) g_err = first_msg;
    return first;
}

vgr_status vgr_set_batch_chains(uint32_t chains) {
    g_batch_chains.store(chains);
    return VGR_OK;
}

vgr_status vgr_view_debug(vgr_view* v, vgr_debug_buffers* o) {
    if (!v || !o) return fail(VGR_E_INVALID, "null argument");
    if (v->pending) return fail(VGR_E_INVALID, "a frame of this view is in flight");
    if (!v->has_prev) return fail(VGR_E_INVALID, "no frame rendered yet");
    memset(o, 0, sizeof(*o));
    o->n_cut = v->last_n_cut;
    o->n_visible = v->last_n_vis;
    o->n_front = v->last_n_front;
    o->n_pairs = v->last_n_pairs;
    o->tiles_x = v->last_tw;
    o->tiles_y = v->last_th;
    o->cut = v->cut[v->parity];
    o->vis_node = v->front_list;  // entry i's node id
    o->vis_depth = v->vis.depth;
    o->vis_ntile = v->vis.ntile;
    o->vis_rect = reinterpret_cast<const uint32_t*>(v->vis.rect);
    o->vis_recA = reinterpret_cast<const float*>(v->vis.recA);
    o->vis_recB = reinterpret_cast<const float*>(v->vis.recB);
    o->vis_rgb = reinterpret_cast<const float*>(v->vis.rgb);
    o->depth_order = v->sortV[1];
    o->pair_tile = v->pairK[v->last_tile_buf];
    o->pair_val = v->pairV[v->last_tile_buf];
    o->tile_range = reinterpret_cast<const uint32_t*>(v->ranges);
    o->tile_size = tile_of(v);
    return VGR_OK;
}

}  // extern "C"
