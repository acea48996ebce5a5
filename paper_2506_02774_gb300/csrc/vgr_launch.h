// vgr_launch.h -- host-side launchers of the frame-path kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vgr {

// vgr_capi.cu: the thread-local message returned by vgr_last_error()
void set_last_error(const char* msg);

// Kernels of a frame are launched with programmatic stream serialization:
// a kernel's CTAs may be scheduled while the previous kernel drains, and each
// kernel waits (griddepcontrol.wait, its first statement) until the previous
// one has completed and its writes are visible, so ordering is unchanged and
// only the launch latency overlaps.  That wait covers a preceding kernel only:
// a kernel that follows copies, memsets or event records in the stream is
// launched in plain stream order (PdlScope), so it cannot start before them.
// VGR_PDL=0 in the environment turns it off everywhere.
bool pdl_enabled();
struct PdlState {
    bool on = true;          // frame kernels may use it (off while stage events sit between kernels)
    bool plain_next = false; // the next launch follows a non-kernel operation
};
PdlState& pdl_state();  // per host thread
// For the kernels of one frame: the first launch in plain order, PDL for the
// rest unless 'on' is false; restores the defaults when it ends.
struct PdlScope {
    explicit PdlScope(bool on) {
        pdl_state().on = on;
        pdl_state().plain_next = true;
    }
    ~PdlScope() { pdl_state() = PdlState{}; }
};
template <typename... KArgs, typename... Args>
inline void launch_ks(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                      Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    PdlState& st = pdl_state();
    cfg.numAttrs = pdl_enabled() && st.on && !st.plain_next ? 1 : 0;
    st.plain_next = false;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, Args... args) {
    launch_ks(kernel, grid, block, 0, s, args...);
}

struct SceneDev;
struct FrameParams;
struct Counters;

// k_lod.cu
void launch_lod_update(const SceneDev& sc, const uint32_t* prev_cut, const uint32_t* n_prev, uint32_t cap_prev,
                       const FrameParams* fp, uint32_t* bitmap, uint32_t* front, Counters* ctr, int grid,
                       bool frustum, bool interp, cudaStream_t s);
void launch_lod_level(int level, const SceneDev& sc, const uint32_t* fin, uint32_t* fout, uint32_t cap,
                      const FrameParams* fp, uint32_t* bitmap, uint32_t* front, Counters* ctr, int grid,
                      bool frustum, bool interp, cudaStream_t s);
void launch_cut_compact(uint32_t* bitmap, uint32_t* front, uint32_t n_words, uint32_t* cut, uint32_t* front_list,
                        uint32_t cap, uint32_t* n_cut_out, unsigned long long* status,
                        unsigned long long* status_front, Counters* ctr, const FrameParams* fp, int grid,
                        cudaStream_t s);
uint32_t cut_compact_tiles(uint32_t n_words);
uint32_t cut_compact_tile_words();

// k_preprocess.cu
// Per in-front entry i (the entry's node id is the in-front list's entry i)
struct VisBuffers {
    uint32_t* depth;
    uint32_t* ntile;
    uint2* rect;
    float4* recA;   // u v A B   (rho = A dx^2 + B dx dy + C dy^2)
    float4* recB;   // C thr theta, and the footprint box's half-height | half-width << 16 (FP16 bits, rounded up)
    float4* rgb;    // r g b 0
    float* lw;      // parent weight of the interpolated Gaussian (weight interpolation only)
};
void launch_preprocess(const SceneDev& sc, const uint32_t* front, const uint32_t* n_front, uint32_t cap,
                       const FrameParams* fp, VisBuffers vis, Counters* ctr, bool interp, int grid, cudaStream_t s);
uint32_t preprocess_tile();
void prepare_scene(float4* covB, uint32_t n, cudaStream_t s);
void prepare_scene_half(float4* covB, uint32_t n, cudaStream_t s);

// k_sort.cu
uint32_t radix_tile();
void launch_radix_hist(const uint32_t* keys, const uint32_t* n32, const unsigned long long* n64, uint64_t cap,
                       int passes, uint32_t* hist /*[4][256]*/, int grid, cudaStream_t s);
void launch_radix_pass(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                       const uint32_t* n32, const unsigned long long* n64, uint64_t cap, int shift,
                       const uint32_t* hist, unsigned long long* status, uint32_t* ticket, const FrameParams* fp,
                       Counters* ctr, int grid, cudaStream_t s, int hw_match = 0, uint2* ranges = nullptr,
                       uint32_t n_ranges = 0);

// k_emit.cu
// k_slot_scan (slot offsets in depth order, into slot_off[cap_vis + 1]) then k_emit
void launch_emit(const uint32_t* order, uint32_t cap_vis, VisBuffers vis, uint32_t* slot_off, uint32_t* pair_key,
                 uint32_t* pair_val, uint64_t cap_pairs, int tile_passes, uint32_t sentinel,
                 unsigned long long* status, Counters* ctr, const FrameParams* fp, int grid_scan, int grid,
                 cudaStream_t s);
uint32_t emit_tile();
uint32_t slot_scan_tile();
void launch_tile_order(uint2* ranges, uint32_t n_tiles, uint32_t* order, Counters* ctr, cudaStream_t s);
constexpr uint32_t BATCH_VIEWS_MAX = 1024;  // views of one batch blend (k_batch_offsets: one thread each)

// k_blend.cu: the persistent blend over a work list of (view << 20 | tile)
// items in blend order; fps == null: every item is of the view of fp0.  'next'
// (zero before the launch) hands out the list's tiles.  grid = SMs x
// blend_ctas_per_sm(...); depth: hits staged per chunk (16, 32, 48; 48 needs
// tiles of 16 or 32); tile: 8, 16 or 32 pixels.
void launch_blend(const FrameParams* fp0, const FrameParams* const* fps, const uint32_t* work, uint32_t n_work,
                  uint32_t* next, int grid, uint32_t filter, uint32_t exp_mode, uint32_t depth, uint32_t tile,
                  cudaStream_t s);
int blend_ctas_per_sm(uint32_t filter, uint32_t exp_mode, uint32_t depth, uint32_t tile);
// k_emit.cu: the order of a batch's tiles over all its views (heaviest class
// first), from each view's tile order and class counts
void launch_batch_order(const FrameParams* const* fps, uint32_t n_views, const uint32_t* const* orders,
                        const uint32_t* tile_base, uint32_t total_tiles, uint32_t* delta, uint32_t* work,
                        int grid, cudaStream_t s);

// vgr_sort_api.cu: enqueue a standalone pair sort on caller-provided scratch
size_t sort_status_words(uint64_t n, int passes);
int sort_passes(uint32_t key_bits);
cudaError_t sort_pairs_enqueue(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                               uint32_t* vals_out, uint64_t n, uint32_t key_bits, FrameParams* fp, Counters* ctr,
                               unsigned long long* status, uint32_t* tmp_keys, uint32_t* tmp_vals, int grid,
                               cudaStream_t s);

// k_store.cu
void convert_sh_half(const float* src, uint32_t n, uint32_t k3, void* dst, uint32_t stride, cudaStream_t s);
void convert_cov_bf16(const float* src6, uint32_t n, void* dst, cudaStream_t s);

}  // namespace vgr
