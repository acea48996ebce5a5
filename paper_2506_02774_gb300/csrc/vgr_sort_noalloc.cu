// vgr_sort_noalloc.cu -- vgr_sort_pairs for callers that cannot allocate
// device memory: the same kernels, with every byte of scratch taken from one
// file-scope __device__ array of fixed size instead of cudaMalloc.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "vgr.h"
#include "vgr_internal.cuh"
#include "vgr_launch.h"

using namespace vgr;

namespace {

constexpr uint64_t NA_MAX_N = VGR_SORT_NOALLOC_MAX_N;
constexpr int NA_MAX_PASSES = 4;
constexpr size_t na_round(size_t x) { return (x + 255) / 256 * 256; }
// layout of the static scratch: frame params (look-back epoch) | counters
// (tickets, histograms, flags) | look-back words | ping-pong keys | ping-pong values
constexpr size_t NA_OFF_FP = 0;
constexpr size_t NA_OFF_CTR = na_round(sizeof(FrameParams));
constexpr size_t NA_OFF_STATUS = NA_OFF_CTR + na_round(sizeof(Counters));
constexpr size_t NA_STATUS_WORDS = (size_t)NA_MAX_PASSES * ((NA_MAX_N + RADIX_TILE - 1) / RADIX_TILE + 1) * 256;
constexpr size_t NA_OFF_TMP = NA_OFF_STATUS + na_round(NA_STATUS_WORDS * sizeof(unsigned long long));
constexpr size_t NA_BYTES = NA_OFF_TMP + 2 * NA_MAX_N * sizeof(uint32_t);

struct NaDevice {
    unsigned char* base = nullptr;  // device address of the scratch array on this device
    int grid = 0;
};
std::mutex g_na_mu;
NaDevice g_na_dev[64];

vgr_status na_fail(vgr_status s, const char* msg, cudaError_t e = cudaSuccess) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s%s%s", msg, e != cudaSuccess ? ": " : "", e != cudaSuccess ? cudaGetErrorString(e) : "");
    set_last_error(buf);
    return s;
}

}  // namespace

// Every GPU that loads the library holds this array until exit.  In host
// code the name is only a host-side handle: its device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_sort_scratch[NA_BYTES];

extern "C" vgr_status vgr_sort_pairs_noalloc(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                             uint32_t* vals_out, uint64_t n, uint32_t key_bits, void* stream) {
    if (key_bits < 1 || key_bits > 32) return na_fail(VGR_E_INVALID, "key_bits must be in [1, 32]");
    if (n == 0) return VGR_OK;
    if (n > NA_MAX_N) {
        char buf[160];
        snprintf(buf, sizeof(buf), "n = %llu exceeds the %llu-pair limit of the static scratch (use vgr_sort_pairs)",
                 (unsigned long long)n, (unsigned long long)NA_MAX_N);
        return na_fail(VGR_E_INVALID, buf);
    }
    if (!keys_in || !vals_in || !keys_out || !vals_out) return na_fail(VGR_E_INVALID, "null pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return na_fail(VGR_E_CUDA, "cudaGetDevice", e);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    int grid = 0;
    {
        std::lock_guard<std::mutex> lock(g_na_mu);
        NaDevice& d = g_na_dev[dev];
        if (!d.base) {
            // first call on this device, with it current: resolve the array's
            // device address and clear it (epoch and look-back words start at 0)
            void* p = nullptr;
            if ((e = cudaGetSymbolAddress(&p, g_sort_scratch)) != cudaSuccess)
                return na_fail(VGR_E_CUDA, "cudaGetSymbolAddress of the sort scratch", e);
            // the clear is waited for here, once, so that a later call on any
            // other stream is ordered after it
            if ((e = cudaMemsetAsync(p, 0, NA_BYTES, s)) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess)
                return na_fail(VGR_E_CUDA, "clearing the sort scratch", e);
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            d.grid = std::max(1, sms * 4);
            d.base = static_cast<unsigned char*>(p);
        }
        base = d.base;
        grid = d.grid;
    }
    FrameParams* fp = reinterpret_cast<FrameParams*>(base + NA_OFF_FP);
    Counters* ctr = reinterpret_cast<Counters*>(base + NA_OFF_CTR);
    unsigned long long* status = reinterpret_cast<unsigned long long*>(base + NA_OFF_STATUS);
    uint32_t* tmp = reinterpret_cast<uint32_t*>(base + NA_OFF_TMP);
    e = sort_pairs_enqueue(keys_in, vals_in, keys_out, vals_out, n, key_bits, fp, ctr, status, tmp, tmp + NA_MAX_N,
                           grid, s);
    if (e != cudaSuccess) return na_fail(VGR_E_CUDA, "sort launch", e);
    uint32_t flags = 0;
    if ((e = cudaMemcpyAsync(&flags, &ctr->flags, sizeof(flags), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return na_fail(VGR_E_CUDA, "sort", e);
    if (flags & F_SPIN_TIMEOUT) return na_fail(VGR_E_TIMEOUT, "a look-back wait of the sort timed out");
    return VGR_OK;
}
