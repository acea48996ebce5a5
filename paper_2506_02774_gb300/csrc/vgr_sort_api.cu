// vgr_sort_api.cu -- the pair sort of the frame path (paper Sec. 3.1
// 'Sorting') as a standalone C-ABI call: stable LSD radix sort of u32
// (key, value) pairs on the device, 8-bit digits, one onesweep pass per digit
// (k_sort.cu).  Scratch (digit histograms, look-back words, the ping-pong
// buffer of multi-pass sorts) comes from a per-device cache owned by the
// library.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "vgr.h"
#include "vgr_internal.cuh"
#include "vgr_launch.h"

namespace vgr {

// Start of a sort: new look-back epoch, element count, zeroed tickets,
// histograms and flags.
__global__ void k_sort_setup(FrameParams* fp, Counters* ctr, unsigned long long n) {
    uint32_t* t = ctr->tickets;
    for (int i = threadIdx.x; i < TK_COUNT; i += blockDim.x) t[i] = 0u;
    uint32_t* h = &ctr->depth_hist[0][0];
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) h[i] = 0u;
    if (threadIdx.x == 0) {
        uint32_t e = fp->epoch + 1u;
        if ((e & 0x3FFFFFFFu) == 0u) ++e;
        fp->epoch = e;
        ctr->flags = 0u;
        ctr->n_pairs = n;
    }
}

size_t sort_status_words(uint64_t n, int passes) {
    return (size_t)passes * ((n + radix_tile() - 1) / radix_tile() + 1) * 256;
}

int sort_passes(uint32_t key_bits) { return (int)((key_bits + 7u) / 8u); }

// Enqueue a sort on 's' with the given scratch; returns a CUDA error code.
cudaError_t sort_pairs_enqueue(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                               uint32_t* vals_out, uint64_t n, uint32_t key_bits, FrameParams* fp, Counters* ctr,
                               unsigned long long* status, uint32_t* tmp_keys, uint32_t* tmp_vals, int grid,
                               cudaStream_t s) {
    const int passes = sort_passes(key_bits);
    k_sort_setup<<<1, 256, 0, s>>>(fp, ctr, (unsigned long long)n);
    launch_radix_hist(keys_in, nullptr, &ctr->n_pairs, n, passes, &ctr->depth_hist[0][0], grid, s);
    const size_t stride = sort_status_words(n, 1);
    // the last pass writes the output; earlier passes alternate backwards
    const uint32_t* kin = keys_in;
    const uint32_t* vin = vals_in;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) & 1) == 0;
        uint32_t* ko = to_out ? keys_out : tmp_keys;
        uint32_t* vo = to_out ? vals_out : tmp_vals;
        launch_radix_pass(kin, vin, ko, vo, nullptr, &ctr->n_pairs, n, 8 * p, ctr->depth_hist[p],
                          status + (size_t)p * stride, &ctr->tickets[TK_SORT0 + p], fp, ctr, grid, s,
                          p == passes - 1 ? 1 : 0);
        kin = ko;
        vin = vo;
    }
    return cudaGetLastError();
}

}  // namespace vgr

using namespace vgr;

namespace {

struct SortCache {
    std::mutex mu;
    FrameParams* fp = nullptr;
    Counters* ctr = nullptr;
    unsigned long long* status = nullptr;
    size_t status_words = 0;
    uint32_t* tmp = nullptr;
    uint64_t tmp_n = 0;
    int grid = 0;
};

SortCache g_cache[64];

vgr_status sort_fail(vgr_status s, const char* msg, cudaError_t e = cudaSuccess) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s%s%s", msg, e != cudaSuccess ? ": " : "", e != cudaSuccess ? cudaGetErrorString(e) : "");
    set_last_error(buf);
    return s;
}

}  // namespace

extern "C" vgr_status vgr_sort_pairs(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                     uint32_t* vals_out, uint64_t n, uint32_t key_bits, void* stream) {
    if (key_bits < 1 || key_bits > 32) return sort_fail(VGR_E_INVALID, "key_bits must be in [1, 32]");
    if (n == 0) return VGR_OK;
    if (n >= 0xFFFFFFFFull) return sort_fail(VGR_E_INVALID, "n must be below 2^32 - 1");
    if (!keys_in || !vals_in || !keys_out || !vals_out) return sort_fail(VGR_E_INVALID, "null pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return sort_fail(VGR_E_CUDA, "cudaGetDevice", e);
    SortCache& c = g_cache[dev];
    std::lock_guard<std::mutex> lock(c.mu);
    if (!c.fp) {
        if ((e = cudaMalloc(&c.fp, sizeof(FrameParams))) != cudaSuccess ||
            (e = cudaMemset(c.fp, 0, sizeof(FrameParams))) != cudaSuccess ||
            (e = cudaMalloc(&c.ctr, sizeof(Counters))) != cudaSuccess ||
            (e = cudaMemset(c.ctr, 0, sizeof(Counters))) != cudaSuccess ||
            (e = cudaStreamSynchronize(cudaStreamLegacy)) != cudaSuccess)  // the fills before any use on 's'
            return sort_fail(VGR_E_NOMEM, "sort scratch", e);
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        c.grid = std::max(1, sms * 4);
    }
    const int passes = sort_passes(key_bits);
    const size_t words = sort_status_words(n, passes);
    if (words > c.status_words) {
        if (c.status) cudaFree(c.status);
        c.status = nullptr;
        c.status_words = 0;
        if ((e = cudaMalloc(&c.status, words * sizeof(unsigned long long))) != cudaSuccess ||
            (e = cudaMemset(c.status, 0, words * sizeof(unsigned long long))) != cudaSuccess ||
            (e = cudaStreamSynchronize(cudaStreamLegacy)) != cudaSuccess)
            return sort_fail(VGR_E_NOMEM, "sort look-back words", e);
        c.status_words = words;
    }
    if (passes > 1 && n > c.tmp_n) {
        if (c.tmp) cudaFree(c.tmp);
        c.tmp = nullptr;
        c.tmp_n = 0;
        const uint64_t n_al = (n + 63u) & ~(uint64_t)63u;  // the value half starts 256-byte aligned
        if ((e = cudaMalloc(&c.tmp, 2 * n_al * sizeof(uint32_t))) != cudaSuccess)
            return sort_fail(VGR_E_NOMEM, "sort ping-pong buffer", e);
        c.tmp_n = n_al;
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = sort_pairs_enqueue(keys_in, vals_in, keys_out, vals_out, n, key_bits, c.fp, c.ctr, c.status, c.tmp,
                           c.tmp ? c.tmp + c.tmp_n : nullptr, c.grid, s);
    if (e != cudaSuccess) return sort_fail(VGR_E_CUDA, "sort launch", e);
    uint32_t flags = 0;
    if ((e = cudaMemcpyAsync(&flags, &c.ctr->flags, sizeof(flags), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return sort_fail(VGR_E_CUDA, "sort", e);
    if (flags & F_SPIN_TIMEOUT) return sort_fail(VGR_E_TIMEOUT, "a look-back wait of the sort timed out");
    return VGR_OK;
}
