/*
 * vgr.h -- C ABI of the GB300 frame path of a city-scale Gaussian-splatting
 * renderer: temporal-aware LoD cut update, projection, tile binning with
 * preemptive alpha filtering, sort and front-to-back alpha blending
 * (arXiv 2506.02774, "Voyager", Sec. 3.1 pipeline, Sec. 4.1, Sec. 4.2).
 *
 * Conventions for every function below:
 *  - Returns vgr_status; VGR_OK (0) on success.  Never aborts or exits.
 *    vgr_last_error() gives a thread-local message for the last failure.
 *  - Host arrays passed in are owned by the caller and only read during the
 *    call (they are copied to the device).  Device buffers are owned by the
 *    library; pointers handed out are borrowed and stay valid until the next
 *    call on the same object or its destruction.
 *  - A view is not thread-safe; distinct views may be used from distinct
 *    threads.  All device work of a view is ordered on its stream.
 *  - Requires a CUDA device of compute capability 10.3 (GB300); the library
 *    contains sm_103a code only.
 */
#ifndef VGR_H
#define VGR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VGR_OK = 0,
    VGR_E_INVALID = 1,     /* bad argument or malformed hierarchy */
    VGR_E_NOMEM = 2,       /* device or host allocation failed */
    VGR_E_CUDA = 3,        /* a CUDA call failed (message has the CUDA error) */
    VGR_E_TIMEOUT = 4,     /* a bounded device wait or loop ran out */
    VGR_E_NONMONOTONE = 5, /* a child expands while its parent does not */
    VGR_E_OVERFLOW = 6     /* a buffer could not be grown to the needed size */
} vgr_status;

/* Storage precision of per-Gaussian attributes on the device. */
enum {
    VGR_STORE_FP32 = 0, /* SH and covariance in FP32 */
    VGR_STORE_HALF = 1  /* SH in FP16, covariance in BF16; expanded to FP32 in registers */
};

/* Rasterization filter. */
enum {
    VGR_FILTER_PREEMPTIVE = 0, /* Sec. 4.2: log-domain alpha test, Gaussian- and tile-level filters */
    VGR_FILTER_CANONICAL = 1   /* 3-sigma square footprint, alpha = min(.99, theta e^rho) then test */
};

/* Exponential in the blend. */
enum {
    VGR_EXP_EXACT = 0, /* hardware exp2 */
    VGR_EXP_LUT = 1    /* Eq. 5: nearest entry of an m-interval table over rho in [-5.55, 0] */
};

typedef struct vgr_hierarchy vgr_hierarchy;
typedef struct vgr_view vgr_view;

/*
 * LoD tree (paper Sec. 3.1 "LoD Tree"): one Gaussian per node, nodes in
 * breadth-first order, node 0 the root (parent 0xFFFFFFFF), children of a
 * node contiguous at first_child .. first_child + n_child - 1 with ids larger
 * than the parent, n_child <= 8 (0 for a leaf).  Arrays have n_nodes entries
 * (times the stated width):
 *   mean     3 floats, world position (also the node centre of the LoD test)
 *   cov6     6 floats, covariance xx xy xz yy yz zz
 *   opacity  1 float in [0, 1]
 *   sh       3 (deg+1)^2 floats, coefficient-major, RGB innermost
 *   radius2  1 float, squared node radius R^2 of the granularity test; the
 *            radii must nest (R_parent >= R_child + |mean_parent - mean_child|)
 *            for the cut to be well defined under the test below.
 *   bbox     6 floats or NULL: axis-aligned node box lo x, y, z, hi x, y, z,
 *            nested exactly (a child's box inside its parent's); needed only
 *            by the frustum-aware granularity test (vgr_view_opts.lod_frustum).
 *            A box that covers the node's Gaussian and its subtree keeps that
 *            variant from coarsening anything that reaches the image.
 */
typedef struct {
    uint32_t n_nodes;
    uint32_t sh_degree; /* 0..3 */
    const uint32_t* parent;
    const uint32_t* first_child;
    const uint8_t* n_child;
    const float* mean;
    const float* cov6;
    const float* opacity;
    const float* sh;
    const float* radius2;
    int32_t storage; /* VGR_STORE_* */
    const float* bbox; /* optional, see above */
} vgr_scene_desc;

/*
 * Pinhole camera.  p_cam = R (p - pos) with R the world->camera rotation
 * (row-major) and pos the camera centre; camera axes x right, y down,
 * z forward.  A point projects to (fx x/z + cx, fy y/z + cy) in pixels;
 * pixel (i, j) covers [i, i+1) x [j, j+1).  Points with z <= z_near are culled.
 */
typedef struct {
    float R[9];
    float pos[3];
    float fx, fy, cx, cy;
    uint32_t width, height;
    float z_near;
} vgr_camera;

typedef struct {
    void* stream;            /* cudaStream_t to run on; NULL: the view creates its own */
    uint32_t filter;         /* VGR_FILTER_* */
    uint32_t exp_mode;       /* VGR_EXP_* */
    uint32_t lut_size;       /* m of Eq. 5 when exp_mode == VGR_EXP_LUT (1..256; default 32) */
    uint32_t temporal;       /* 1: temporal cut update between frames (default); 0: always from scratch */
    uint32_t timing;         /* 1: record per-stage device times into vgr_frame_stats */
    uint32_t use_graph;      /* 1: replay each frame as one captured CUDA graph (captured on first use per
                                cut mode and buffer parity; re-captured after a buffer grows or the image
                                size changes); ignored while timing is set.  Default 0. */
    uint64_t cut_capacity;   /* initial capacities; 0 = automatic.  Grown on demand. */
    uint64_t pair_capacity;
    uint32_t lod_budget;     /* max nodes one thread explores when expanding a cut node (0 = 4096) */
    uint32_t grid_wide;      /* CTAs of the grid-stride kernels (LoD, preprocess with colour, ranges);
                                0 = 8 per SM.  Launch geometry only: results do not depend on it. */
    uint32_t grid_scan;      /* CTAs of the ticketed look-back kernels (compaction, radix passes,
                                emission); 0 = 4 per SM.  Launch geometry only. */
    uint32_t test_hooks;     /* 0 in normal use.  VGR_HOOK_WITHHOLD_LOOKBACK: the emission's first
                                tile never publishes its look-back word, so the later tiles' bounded
                                waits run out and every frame reports VGR_E_TIMEOUT (the device
                                stays usable); for testing the timeout path. */
    uint32_t lod_frustum;    /* 1: frustum-aware granularity test (needs bbox; default 0), see
                                vgr_render_frame */
    float lod_frustum_guard; /* pixels the frustum test adds beyond each image edge (default 2) */
    uint32_t lod_interp;     /* 1: parent-child weight interpolation of the cut's Gaussians (default 0),
                                see vgr_render_frame */
    uint32_t blend_depth;    /* Gaussians the blend stages per warp and chunk: 16, 32 or 48 (0 = 32).
                                A tuning knob: results do not depend on it. */
    uint32_t tile_size;      /* side of a square tile in pixels: 8, 16 or 32 (0 = 16); 8 needs images of
                                at most 8192 x 8192 and a blend_depth of 16 or 32.  The pairs are per
                                tile; the cut and the image do not depend on it. */
} vgr_view_opts;

enum { VGR_HOOK_WITHHOLD_LOOKBACK = 1,
       VGR_HOOK_FULL_STRIP_WALK = 2  /* the blend walks every record of a strip at every pixel instead of only
                                        the records whose footprint box covers the pixel (same image) */ };

/* Stages of stage_ms.  The colour (SH -> RGB) is evaluated by the preprocess
 * kernel, so VGR_STAGE_PREPROCESS includes it and VGR_STAGE_COLOR stays
 * empty (kept so that the indices of the later stages do not move). */
enum { VGR_STAGE_LOD = 0, VGR_STAGE_COMPACT, VGR_STAGE_PREPROCESS, VGR_STAGE_DEPTH_SORT, VGR_STAGE_COLOR,
       VGR_STAGE_EMIT, VGR_STAGE_TILE_SORT, VGR_STAGE_RANGES, VGR_STAGE_BLEND, VGR_N_STAGES };

typedef struct {
    uint32_t cut_count;       /* |C| */
    uint32_t front_count;     /* cut nodes in front of the near plane */
    uint32_t visible_count;   /* |V|: cut Gaussians with at least one candidate tile */
    uint64_t pair_count;      /* P: (Gaussian, tile) pairs kept by the tile-level filter */
    uint64_t candidate_pairs; /* P0: candidate pairs examined by the tile-level filter */
    uint64_t nodes_evaluated; /* granularity tests made by the LoD step */
    uint32_t lod_from_scratch;/* 1 if the cut was found top-down this frame */
    uint32_t replays;         /* frame replays (buffer growth or LoD fallback) */
    uint32_t kernels;         /* kernel launches made for the frame, replays included */
    uint64_t pixel_pair_evals;/* X: (pixel, Gaussian) evaluations in the blend */
    uint64_t pixel_pair_contribs; /* of those, the ones blended (alpha >= alpha*, before termination) */
    float stage_ms[VGR_N_STAGES]; /* device time per stage (timing = 1), else 0 */
    float frame_ms;           /* device time of the frame (timing = 1), else 0 */
} vgr_frame_stats;

typedef struct {
    const float* image;       /* device, height x width x 3 FP32 RGB, background 0 */
    const uint32_t* cut;      /* device, cut_count node ids in ascending order */
    uint32_t cut_count;
    uint32_t width, height;
    vgr_frame_stats stats;
} vgr_frame;

/*
 * Device pointers of the intermediate buffers of the last frame (testing).
 * Per-Gaussian arrays are indexed like the in-front list (cut nodes in front
 * of the near plane, ascending node id); entries culled later have
 * vis_ntile = 0 and the depth key 0xFFFFFFFF.
 */
typedef struct {
    uint32_t n_cut, n_front, n_visible;
    uint64_t n_pairs;
    uint32_t tiles_x, tiles_y;
    const uint32_t* cut;          /* [n_cut] ascending node ids */
    const uint32_t* vis_node;     /* [n_front] node id */
    const uint32_t* vis_depth;    /* [n_front] FP32 depth key bits (0xFFFFFFFF if culled) */
    const uint32_t* vis_ntile;    /* [n_front] candidate tiles (area of vis_rect), 0 if culled */
    const uint32_t* vis_rect;     /* [2 n_front] candidate tiles: x0 | y0 << 16, x1 | y1 << 16 */
    const float* vis_recA;        /* [4 n_front] u v A B, rho = A dx^2 + B dx dy + C dy^2 */
    const float* vis_recB;        /* [4 n_front] C thr theta h, thr = ln alpha* - ln theta, h = the footprint box's
                                     half-height | half-width << 16 as FP16 bits (rounded up) */
    const float* vis_rgb;         /* [4 n_front] r g b 0 (visible entries only) */
    const uint32_t* depth_order;  /* [n_front] in-front index by depth rank; the first n_visible are visible */
    const uint32_t* pair_tile;    /* [n_pairs] tile id, sorted */
    const uint32_t* pair_val;     /* [n_pairs] in-front index << 8 | row mask (bit w: the footprint box reaches
                                     one of the tile's pixel rows w r .. w r + r - 1, r = max(1, tile_size / 8);
                                     all ones in the canonical mode) */
    const uint32_t* tile_range;   /* [2 tiles] start, end into the pair list */
    uint32_t tile_size;           /* side of a tile in pixels; a row-mask bit covers max(1, tile_size / 8) rows */
} vgr_debug_buffers;

void vgr_default_view_opts(vgr_view_opts* opts);

/*
 * Upload a LoD tree.  Validates the shape (BFS order, contiguous children,
 * n_child <= 8, radius nesting within a 1e-6 relative slack) and returns
 * VGR_E_INVALID otherwise.  Precomputes ln(opacity) on the device.
 */
vgr_status vgr_load_hierarchy(const vgr_scene_desc* desc, vgr_hierarchy** out);
vgr_status vgr_free_hierarchy(vgr_hierarchy* h);
/* Device bytes held by the hierarchy. */
vgr_status vgr_hierarchy_info(const vgr_hierarchy* h, uint64_t* device_bytes, uint32_t* max_depth);

/* A view keeps one client's state: previous cut, sort buffers, image. */
vgr_status vgr_create_view(vgr_hierarchy* h, const vgr_view_opts* opts, vgr_view** out);
vgr_status vgr_destroy_view(vgr_view* v);
/* Forget the previous cut: the next frame finds its cut top-down. */
vgr_status vgr_reset_view(vgr_view* v);
/*
 * Change a view's tuning knobs (vgr_view_opts.grid_wide, grid_scan,
 * blend_depth, tile_size; 0 keeps the current value) between frames, for an
 * autotuner.  The cut and the image do not depend on them (the pair lists
 * follow the tile size).  Captured frames are dropped and captured again on
 * next use; the previous cut is kept.  VGR_E_INVALID while a frame is in
 * flight, for a depth other than 16, 32, 48, a tile size other than 8, 16,
 * 32, or depth 48 with 8-pixel tiles.
 */
vgr_status vgr_view_set_tuning(vgr_view* v, uint32_t grid_wide, uint32_t grid_scan, uint32_t blend_depth,
                               uint32_t tile_size);
vgr_status vgr_view_device_bytes(const vgr_view* v, uint64_t* bytes);

/*
 * Render one frame with granularity threshold tau (pixels).  The cut is the
 * set of nodes whose every ancestor expands and which do not expand, where
 * with f = max(fx, fy), t = fl(tau / f), k = fl(t t) and single-rounded FP32
 * arithmetic:  d2 = (dx dx + dy dy) + dz dz,  (dx, dy, dz) = pos - mean[n],
 * expand(n) = n_child[n] > 0 and fl(d2 k) < radius2[n]   (Sec. 3.1).
 * With lod_frustum set, expand(n) also needs n's box to meet the view
 * frustum widened by g = lod_frustum_guard pixels (the tree "identifies the
 * Gaussians inside the view frustum", Sec. 3.1): for each of five planes
 * (camera-space inward normal a, offset o_c: near (0, 0, 1), z_near; left
 * (fx, 0, cx + g), right (-fx, 0, W - cx + g), top (0, fy, cy + g), bottom
 * (0, -fy, H - cy + g), 0) take w_j = fl32(fma(R2j, a2, fma(R1j, a1, R0j a0)))
 * and o = fl32(fma(w2, pos2, fma(w1, pos1, w0 pos0)) + o_c) in FP64, the box
 * corner X furthest along w (hi where w_j >= 0, else lo) and require
 * fl(fl(fl(w0 X0) + fl(w1 X1)) + fl(w2 X2)) - o >= 0 (single-rounded FP32).
 * Nested boxes keep this monotone, so the temporal update stays exact.
 * With lod_interp set, each cut node n with parent p is rendered as a
 * Gaussian interpolated towards p's (Sec. 3.1 "Weight Interpolation"; the
 * paper gives no formula, this is the one used): with t = fl(tau / f) and
 * a = fl(sqrt(fl(radius2 / d2))) a node's size ratio (single-rounded FP32,
 * d2 as above), w = clamp(fl(fl(t - a_n) / fl(a_p - a_n)), 0, 1) if a_p > a_n,
 * else 0 (and 0 at the root); mean_j = fl(mean_n + fl(w fl(mean_p - mean_n)));
 * covariance, SH coefficients and opacity move by w towards the parent's,
 * the parent's opacity taken as 1 - (1 - opacity_p)^(1 / n_child[p]) (its
 * share among the siblings).  The cut itself does not change.
 * Between frames with equal tau and f the cut is updated from the previous
 * one (Sec. 4.1, Algorithm 1); the result equals the top-down cut.
 * Requires 0 <= tau <= f, width, height in [1, 16384], z_near > 0.
 * Waits for the frame to finish before returning (status checks).
 */
vgr_status vgr_render_frame(vgr_view* v, const vgr_camera* cam, float tau, vgr_frame* out);

/*
 * As vgr_render_frame, and the image also lands in host memory host_rgb
 * (height x width x 3 floats, caller-owned).  Pinned memory of this view's
 * device is written by the blend itself, over the host link while the frame
 * runs; any other memory receives a copy after the frame.
 */
vgr_status vgr_render_frame_host(vgr_view* v, const vgr_camera* cam, float tau, float* host_rgb,
                                 vgr_frame* out);

/*
 * Pipelined host images, for a loop of frames whose images go to host
 * memory: as vgr_render_frame_host, except that the copy of the image into
 * host_rgb (caller-owned, height x width x 3 floats; pinned memory lets the
 * copy engine do it without the host) is enqueued on the view's copy stream
 * once the frame's status has been read, and overlaps the view's next frame,
 * which writes the view's other device image.  Returns when the frame's
 * kernels have finished (replays included) without waiting for the copy; out
 * is filled as by vgr_render_frame, out->image being the frame's device image
 * (valid until the next frame).  Copies land in the order of the frames.
 * vgr_wait_host_images waits until every copy enqueued this way has landed;
 * until then host_rgb must stay valid and does not yet hold the image.  A
 * frame that would overwrite a device image still being copied waits for
 * that copy (on the device).  The second device image is allocated by the
 * view's first pipelined frame.
 */
vgr_status vgr_render_frame_pipelined(vgr_view* v, const vgr_camera* cam, float tau, float* host_rgb,
                                      vgr_frame* out);
vgr_status vgr_wait_host_images(vgr_view* v);

/*
 * Asynchronous form of vgr_render_frame, for keeping several views' frames
 * on the GPU at once (a view created with stream 0 owns its own stream).
 * vgr_submit_frame validates the arguments as vgr_render_frame does and
 * enqueues the frame -- and, when host_rgb is not NULL, the copy of the image
 * into host_rgb (caller-owned, height x width x 3 floats, valid until
 * vgr_finish_frame returns) -- without waiting.  vgr_frame_done sets *done to
 * 1 when the submitted work has finished, 0 otherwise, without waiting.
 * vgr_finish_frame waits for it, reads the frame's status, replays the frame
 * when the temporal update fell back or a buffer had to grow (replays wait),
 * and fills out (may be NULL); the result equals vgr_render_frame's.  Each
 * successful submit is followed by exactly one finish; until then another
 * submit, vgr_reset_view and vgr_view_debug return VGR_E_INVALID.
 */
vgr_status vgr_submit_frame(vgr_view* v, const vgr_camera* cam, float tau, float* host_rgb);
vgr_status vgr_frame_done(vgr_view* v, int* done);
vgr_status vgr_finish_frame(vgr_view* v, vgr_frame* out);

/*
 * One frame on each of n distinct views (own camera, tau and image size
 * each; the views may share a hierarchy): every frame is submitted, then
 * every frame is finished in order, so frames of views on different streams
 * overlap on the GPU.  When every view uses graph replay on a stream of its
 * own (created with stream 0, no stage timing), the whole batch runs as one
 * captured CUDA graph, cached per combination of views, cut modes, buffer
 * parities and image sizes.  host_rgb is NULL or n pointers (NULL entries: no host
 * copy); outs is NULL or n frames.  Returns the first error (VGR_E_INVALID
 * for a repeated or NULL view, before anything is submitted); every frame
 * that was submitted is finished.  The paper renders one view at a time;
 * this call has no counterpart there.
 */
vgr_status vgr_render_batch(vgr_view* const* views, const vgr_camera* cams, const float* taus,
                            float* const* host_rgb, uint32_t n, vgr_frame* outs);

/*
 * How many views of a captured batch run at once (process-wide; a tuning
 * knob, results do not depend on it): with chains = c > 0 the views form c
 * parallel chains, assigned largest image first each to the chain with the
 * fewest pixels so far, a view starting when the previous view of its chain
 * has finished up to its tile order; 0 (the default) runs every view as its
 * own branch.  Large views' frames keep their sort and pair buffers in L2
 * only while few of them run at once; small views gain from running many at
 * once.  The batch's single blend launch follows every chain.
 */
vgr_status vgr_set_batch_chains(uint32_t chains);

vgr_status vgr_view_debug(vgr_view* v, vgr_debug_buffers* out);

/*
 * Device bytes a view created with opts (NULL: defaults) on h holds after
 * its first frame at width x height, before any buffer grows.
 */
vgr_status vgr_view_bytes_estimate(const vgr_hierarchy* h, const vgr_view_opts* opts, uint32_t width,
                                   uint32_t height, uint64_t* bytes);

/*
 * Frame server with continuous batching (no counterpart in the paper, which
 * renders one view).  Each client of a server owns a view (own stream),
 * created when the client's first request is admitted.  Admission requires
 * free device memory >= vgr_view_bytes_estimate at the request's image size
 * + hbm_reserve.  When that is short, the server (evict_idle set) releases
 * the views of idle clients -- no frame in flight and no request waiting --
 * least recently used first, until the view fits; if it still does not fit
 * while other frames are in flight, the request stays queued and admission
 * is tried again each time a frame completes.  Only a request that cannot
 * fit with nothing else in flight and no idle view left completes with
 * VGR_E_NOMEM.  A released client's next frame finds its cut top-down, which
 * gives the same cut as the temporal update.  A client's requests run in
 * arrival order, one frame in flight per client; frames of different clients
 * run concurrently on their own streams, at most max_inflight at a time, and
 * a request starts as soon as its client, a slot and the memory are free.
 */
typedef struct vgr_server vgr_server;

typedef struct {
    uint32_t n_clients;      /* clients 0 .. n_clients-1 (1..65536) */
    uint32_t max_inflight;   /* frames in flight at once (default 2); 1 = one frame at a time;
                                0 = n_clients.  A large frame's sort and pair buffers stay in
                                L2 only while few such frames run at once. */
    uint32_t host_images;    /* 1: every image is copied to the client's pinned host buffer */
    uint64_t hbm_reserve;    /* free device bytes admission keeps (default 1 GiB) */
    vgr_view_opts view;      /* options of every client's view; stream and timing are ignored
                                (default: vgr_default_view_opts with use_graph = 1) */
    uint32_t evict_idle;     /* 1 (default): release idle clients' views, least recently used
                                first, when admission lacks memory; 0: never release a view */
} vgr_serve_opts;

typedef struct {
    uint32_t client;
    float tau;
    double arrival_s;        /* seconds after the start of vgr_serve_trace; non-decreasing */
    vgr_camera cam;
    float* host_rgb;         /* NULL, or a caller-owned host buffer of cam.height x cam.width x 3
                                floats for this request's image (used instead of the client's
                                buffer); pinned memory of the server's device is written by the
                                blend itself, other memory receives a copy after the frame.  It
                                must stay valid until vgr_serve_trace returns. */
} vgr_request;

typedef struct {
    double start_s;          /* submission (after admission) */
    double finish_s;         /* completion seen by the server: image in device memory, and in the
                                request's or the client's host buffer when one is used */
    vgr_status status;       /* VGR_OK, VGR_E_NOMEM (could not be admitted) or the frame's error */
    uint32_t cut_count, visible_count;
    uint64_t pair_count;
    uint32_t replays, lod_from_scratch;
    uint32_t admission_waits;  /* times admission found too little memory and the request waited */
    uint32_t views_released;   /* idle clients' views released to admit this request */
} vgr_request_result;

void vgr_default_serve_opts(vgr_serve_opts* opts);
/* The server keeps h (which must outlive it) and copies opts. */
vgr_status vgr_create_server(vgr_hierarchy* h, const vgr_serve_opts* opts, vgr_server** out);
vgr_status vgr_destroy_server(vgr_server* s);
/*
 * Serve n requests (caller-owned, read only) in real time: request i is
 * released at arrival_s after the call starts; res (n entries) receives each
 * request's times and counts.  Returns when every request has completed.
 * Views persist across calls (a first trace can admit and warm up the
 * clients).  Returns VGR_E_INVALID for a bad client id or decreasing arrival
 * times (before anything runs), else the first frame error (refusals by
 * admission are reported per request only).  Not thread-safe per server.
 */
vgr_status vgr_serve_trace(vgr_server* s, const vgr_request* reqs, uint32_t n, vgr_request_result* res);
/* A client's view (NULL before admission) and its pinned host image (NULL without host_images). */
vgr_status vgr_server_client_view(vgr_server* s, uint32_t client, vgr_view** view, const float** host_rgb);

/*
 * The pair sort of the frame path as a standalone call (Sec. 3.1 "Sorting"):
 * stable LSD radix sort of n (key, value) pairs of u32 by the low
 * 8 * ceil(key_bits / 8) bits of the key, 8-bit digits, one pass per digit.
 * keys_in, vals_in, keys_out, vals_out are device pointers to n elements each;
 * the inputs are only read, the outputs receive the sorted pairs, and input
 * and output ranges must not overlap.  Equal keys keep their input order.
 * Runs on 'stream' (a cudaStream_t, NULL for the default stream) and waits
 * for it before returning.  Scratch (histograms, look-back words, the
 * ping-pong buffer of a multi-pass sort) is allocated by the library on
 * first use per device, grown when a larger n arrives and kept until exit;
 * calls on one device are serialised.  1 <= key_bits <= 32, n < 2^32 - 1
 * (n = 0 is a no-op).  Errors: VGR_E_INVALID, VGR_E_NOMEM, VGR_E_CUDA,
 * VGR_E_TIMEOUT (a bounded look-back wait ran out).
 */
vgr_status vgr_sort_pairs(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                          uint32_t* vals_out, uint64_t n, uint32_t key_bits, void* stream);

/* Largest n accepted by vgr_sort_pairs_noalloc. */
#define VGR_SORT_NOALLOC_MAX_N 262144u

/*
 * vgr_sort_pairs for callers that must not allocate device memory -- for
 * example code running as a plug-in inside a host application that owns all
 * device memory, or a frame loop with a fixed memory budget in which
 * cudaMalloc and cudaFree (which can synchronise the whole device) are not
 * allowed.  The paper has no counterpart; it is a service of this library.
 *
 * Same arguments, result and errors as vgr_sort_pairs, but it calls no
 * cudaMalloc, cudaFree or other allocating routine: all scratch (look-back
 * epoch, tickets, histograms, look-back words, the ping-pong buffer) lives in
 * one fixed array in device memory that the library declares and that every
 * GPU loading the library holds until the process exits (about 2.7 MB).
 *   - n is limited to VGR_SORT_NOALLOC_MAX_N (262,144) pairs; larger n
 *     returns VGR_E_INVALID without touching the GPU.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address, clears the array on 'stream' and waits for the
 *     clear; make that first call before any stream capture.
 *   - Every call waits for its stream before it returns, so a call made
 *     after another call has returned -- on any stream -- is ordered after
 *     it.  Every call on a device shares the one array, which keeps the last
 *     call's contents; each call clears what it needs at its start.  Calls
 *     that run at the same time (from different host threads, on different
 *     streams) race on the array and give wrong results: do not overlap
 *     them.
 */
vgr_status vgr_sort_pairs_noalloc(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                  uint32_t* vals_out, uint64_t n, uint32_t key_bits, void* stream);

const char* vgr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VGR_H */
