// vgr_serve.cu -- a frame server for many clients over one resident
// hierarchy, with continuous batching.
//
// Each client owns a view (its previous cut, buffers, image and stream),
// created when the client's first request is admitted.  A client's requests
// are rendered in arrival order (the temporal cut update of Sec. 4.1 needs
// the previous frame), different clients' frames run concurrently on their
// own streams, and a request starts as soon as a slot (a frame in flight) is
// free: it does not wait for a batch to fill or drain.  Admission compares
// the free device memory with the view's estimated footprint at the
// request's image size plus a reserve; when memory is short it releases idle
// clients' views (least recently used first), and a request that still does
// not fit waits in the queue until a frame completes.  The paper serves one
// view; nothing here has a counterpart in it.
//
// Host code only: the frames themselves go through vgr_submit_frame /
// vgr_frame_done / vgr_finish_frame.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <thread>
#include <vector>

#include "../../include/vgr.h"
#include "vgr_launch.h"

struct vgr_server {
    vgr_hierarchy* h = nullptr;
    vgr_serve_opts opts{};
    struct Client {
        vgr_view* view = nullptr;
        float* host = nullptr;  // pinned image buffer (host_images)
        size_t host_floats = 0;
    };
    std::vector<Client> clients;
};

namespace {

using clock_type = std::chrono::steady_clock;

// Per-trace scheduling state the admission step reads.
struct TraceState {
    std::vector<int64_t> inflight;   // request index in flight per client, -1 if none
    std::vector<uint32_t> queued;    // arrived, not started requests per client
    std::vector<uint64_t> last_use;  // completion tick of the client's last frame (LRU order)
};

// The least recently used client (other than c) whose view is idle: no frame
// in flight and no request waiting for it; -1 if there is none.
int64_t lru_idle(const vgr_server* sv, const TraceState& ts, uint32_t c) {
    int64_t best = -1;
    for (uint32_t j = 0; j < sv->clients.size(); ++j) {
        if (j == c || !sv->clients[j].view || ts.inflight[j] >= 0 || ts.queued[j] > 0) continue;
        if (best < 0 || ts.last_use[j] < ts.last_use[(size_t)best]) best = j;
    }
    return best;
}

vgr_status admit(vgr_server* sv, uint32_t c, const vgr_camera& cam, const TraceState& ts, uint32_t* released) {
    vgr_server::Client& cl = sv->clients[c];
    while (!cl.view) {
        uint64_t est = 0;
        vgr_status s = vgr_view_bytes_estimate(sv->h, &sv->opts.view, cam.width, cam.height, &est);
        if (s != VGR_OK) return s;
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            vgr::set_last_error("cudaMemGetInfo failed");
            return VGR_E_CUDA;
        }
        bool fits = (uint64_t)free_b >= est + sv->opts.hbm_reserve;
        if (fits) {
            vgr_view_opts vo = sv->opts.view;
            vo.stream = nullptr;  // every client gets its own stream
            vo.timing = 0;
            s = vgr_create_view(sv->h, &vo, &cl.view);
            if (s == VGR_OK) break;
            if (s != VGR_E_NOMEM) return s;
            cl.view = nullptr;  // the estimate was short: same as not fitting
        }
        const int64_t j = sv->opts.evict_idle ? lru_idle(sv, ts, c) : -1;
        if (j < 0) {
            vgr::set_last_error("admission: not enough free device memory for this client's view");
            return VGR_E_NOMEM;
        }
        vgr_destroy_view(sv->clients[(size_t)j].view);  // waits for its stream, frees its buffers
        sv->clients[(size_t)j].view = nullptr;
        ++*released;
    }
    return VGR_OK;
}

vgr_status host_buffer(vgr_server* sv, uint32_t c, const vgr_camera& cam) {
    vgr_server::Client& cl = sv->clients[c];
    const size_t need_floats = (size_t)cam.width * cam.height * 3;
    if (sv->opts.host_images && cl.host_floats < need_floats) {
        if (cl.host) cudaFreeHost(cl.host);
        cl.host = nullptr;
        cl.host_floats = 0;
        if (cudaMallocHost((void**)&cl.host, need_floats * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            vgr::set_last_error("pinned host image buffer");
            return VGR_E_NOMEM;
        }
        cl.host_floats = need_floats;
    }
    return VGR_OK;
}

}  // namespace

extern "C" {

void vgr_default_serve_opts(vgr_serve_opts* o) {
    if (!o) return;
    *o = vgr_serve_opts{};
    o->n_clients = 1;
    o->max_inflight = 2;  // more large frames at once push each other's sort buffers out of L2
    o->host_images = 0;
    o->hbm_reserve = 1ull << 30;
    vgr_default_view_opts(&o->view);
    o->view.use_graph = 1;
    o->evict_idle = 1;
}

vgr_status vgr_create_server(vgr_hierarchy* h, const vgr_serve_opts* opts, vgr_server** out) {
    if (!h || !opts || !out) {
        vgr::set_last_error("null argument");
        return VGR_E_INVALID;
    }
    *out = nullptr;
    if (opts->n_clients == 0 || opts->n_clients > 65536) {
        vgr::set_last_error("n_clients must be in [1, 65536]");
        return VGR_E_INVALID;
    }
    vgr_server* sv = new vgr_server();
    sv->h = h;
    sv->opts = *opts;
    if (sv->opts.max_inflight == 0 || sv->opts.max_inflight > sv->opts.n_clients)
        sv->opts.max_inflight = sv->opts.n_clients;
    sv->clients.resize(sv->opts.n_clients);
    *out = sv;
    return VGR_OK;
}

vgr_status vgr_destroy_server(vgr_server* sv) {
    if (!sv) {
        vgr::set_last_error("null server");
        return VGR_E_INVALID;
    }
    for (auto& cl : sv->clients) {
        if (cl.view) vgr_destroy_view(cl.view);
        if (cl.host) cudaFreeHost(cl.host);
    }
    delete sv;
    return VGR_OK;
}

vgr_status vgr_server_client_view(vgr_server* sv, uint32_t client, vgr_view** view, const float** host_rgb) {
    if (!sv || !view || client >= sv->clients.size()) {
        vgr::set_last_error("bad argument");
        return VGR_E_INVALID;
    }
    *view = sv->clients[client].view;
    if (host_rgb) *host_rgb = sv->clients[client].host;
    return VGR_OK;
}

vgr_status vgr_serve_trace(vgr_server* sv, const vgr_request* reqs, uint32_t n, vgr_request_result* res) {
    if (!sv || (n && (!reqs || !res))) {
        vgr::set_last_error("null argument");
        return VGR_E_INVALID;
    }
    for (uint32_t i = 0; i < n; ++i) {
        if (reqs[i].client >= sv->clients.size()) {
            vgr::set_last_error("request client id out of range");
            return VGR_E_INVALID;
        }
        if (!(reqs[i].arrival_s >= 0.0) || (i && reqs[i].arrival_s < reqs[i - 1].arrival_s)) {
            vgr::set_last_error("arrival times must be >= 0 and non-decreasing");
            return VGR_E_INVALID;
        }
    }
    for (uint32_t i = 0; i < n; ++i) res[i] = vgr_request_result{};
    nvtxRangePushA("vgr serve trace");
    const uint32_t C = (uint32_t)sv->clients.size();
    TraceState ts;
    ts.inflight.assign(C, -1);
    ts.queued.assign(C, 0);
    ts.last_use.assign(C, 0);
    std::deque<uint32_t> arrived;          // arrived and not started, arrival order
    // completion count when a request last failed admission for memory: it is
    // tried again only after another frame has completed
    std::vector<uint64_t> mem_wait(n, UINT64_MAX);
    uint64_t completions = 0;
    uint32_t next = 0, done = 0, n_inflight = 0;
    vgr_status first_err = VGR_OK;
    const auto t0 = clock_type::now();
    auto now_s = [&]() { return std::chrono::duration<double>(clock_type::now() - t0).count(); };

    while (done < n) {
        bool progress = false;
        double now = now_s();
        while (next < n && reqs[next].arrival_s <= now) {
            arrived.push_back(next);
            ++ts.queued[reqs[next].client];
            ++next;
            progress = true;
        }
        // completions
        for (uint32_t c = 0; c < C && n_inflight; ++c) {
            if (ts.inflight[c] < 0) continue;
            int fin = 0;
            vgr_status s = vgr_frame_done(sv->clients[c].view, &fin);
            if (s == VGR_OK && !fin) continue;
            vgr_frame fr;
            if (s == VGR_OK) s = vgr_finish_frame(sv->clients[c].view, &fr);
            vgr_request_result& r = res[ts.inflight[c]];
            r.finish_s = now_s();
            r.status = s;
            if (s == VGR_OK) {
                r.cut_count = fr.stats.cut_count;
                r.visible_count = fr.stats.visible_count;
                r.pair_count = fr.stats.pair_count;
                r.replays = fr.stats.replays;
                r.lod_from_scratch = fr.stats.lod_from_scratch;
            } else if (first_err == VGR_OK) {
                first_err = s;
            }
            ts.inflight[c] = -1;
            ts.last_use[c] = ++completions;
            --n_inflight;
            ++done;
            progress = true;
        }
        // starts: the earliest arrived request of a client with no frame in flight
        for (auto it = arrived.begin(); it != arrived.end() && n_inflight < sv->opts.max_inflight;) {
            const uint32_t i = *it;
            const uint32_t c = reqs[i].client;
            if (ts.inflight[c] >= 0 || mem_wait[i] == completions) { ++it; continue; }
            vgr_request_result& r = res[i];
            vgr_status s = admit(sv, c, reqs[i].cam, ts, &r.views_released);
            if (s == VGR_OK) s = host_buffer(sv, c, reqs[i].cam);
            float* dst = reqs[i].host_rgb ? reqs[i].host_rgb : (sv->opts.host_images ? sv->clients[c].host : nullptr);
            if (s == VGR_OK) {
                r.start_s = now_s();
                s = vgr_submit_frame(sv->clients[c].view, &reqs[i].cam, reqs[i].tau, dst);
            }
            if (s == VGR_E_NOMEM && n_inflight > 0) {
                // memory frees up as frames complete: keep the request queued
                if (mem_wait[i] == UINT64_MAX) ++r.admission_waits;
                mem_wait[i] = completions;
                ++it;
                continue;
            }
            it = arrived.erase(it);
            --ts.queued[c];
            progress = true;
            if (s != VGR_OK) {
                if (r.start_s == 0.0) r.start_s = now_s();
                r.finish_s = now_s();
                r.status = s;
                ++done;
                if (s != VGR_E_NOMEM && first_err == VGR_OK) first_err = s;  // refusals are results
                continue;
            }
            if (mem_wait[i] != UINT64_MAX) mem_wait[i] = UINT64_MAX;
            ts.inflight[c] = i;
            ++n_inflight;
        }
        if (!progress) {
            if (n_inflight == 0 && next < n) {
                // idle until the next arrival
                const double wait = reqs[next].arrival_s - now_s();
                if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 1e-4));
            } else {
                std::this_thread::yield();
            }
        }
    }
    nvtxRangePop();
    return first_err;
}

}  // extern "C"
