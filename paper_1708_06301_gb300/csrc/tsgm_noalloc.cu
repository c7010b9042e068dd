// Disparity prediction without any device allocation: the z-buffer lives in a fixed array in
// this library's device memory instead of a context.
//
// Some callers cannot allocate device memory: for example a process whose GPU memory is owned by
// another framework's caching allocator (a cudaMalloc behind its back can fail once the pool holds
// the free memory, and it is not accounted for), or a real-time loop that must not call
// cudaMalloc because it can block on the device. They still need the prediction step. This entry
// point does the same work as tsgm_warp_predict with the scratch taken from a file-scope device
// array; it calls no cudaMalloc, cudaFree or other allocating routine.

#include <cfloat>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "tsgm_internal.cuh"

namespace {

// z-buffer keys for up to TSGM_NOALLOC_MAX_PIXELS pixels (16 MiB); every GPU that loads the
// library holds this array until the process exits.
__device__ __align__(256) unsigned long long g_noalloc_keys[TSGM_NOALLOC_MAX_PIXELS];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_keys_ptr[kMaxDevices] = {};

void put_error(char* buf, size_t len, const char* msg) {
    if (buf && len > 0) {
        std::strncpy(buf, msg, len - 1);
        buf[len - 1] = '\0';
    }
}

// Device address of the key array on the current device, resolved once per device. In host
// code the array's name is only a host-side stand-in, so the kernels get this address instead.
// The cached address belongs to the device's current context: after cudaDeviceReset (or any
// other teardown of the primary context) the module is loaded again and may sit elsewhere, so
// the entry point is not to be used across a device reset.
cudaError_t keys_on_current_device(unsigned long long** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_keys_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_keys);
        if (e != cudaSuccess) return e;
        g_keys_ptr[dev] = p;
    }
    *out = static_cast<unsigned long long*>(g_keys_ptr[dev]);
    return cudaSuccess;
}

}  // namespace

extern "C" tsgm_status tsgm_warp_predict_noalloc(const float* prev_D, const float* prev_P,
                                                 int32_t width, int32_t height, const float R[9],
                                                 const float t[3], const float K[9],
                                                 float baseline, float q, float* pred_D,
                                                 float* pred_P, void* cuda_stream, char* errbuf,
                                                 size_t errbuf_len) {
    if (!prev_D || !prev_P || !R || !t || !K || !pred_D || !pred_P) {
        put_error(errbuf, errbuf_len, "tsgm_warp_predict_noalloc: null pointer");
        return TSGM_ERR_INVALID_ARG;
    }
    // the gather writes pred_D[i], pred_P[i] while other threads still read the winners' source
    // values from prev_D, prev_P: outputs that alias inputs would race
    if (pred_D == prev_D || pred_P == prev_P || pred_D == prev_P || pred_P == prev_D) {
        put_error(errbuf, errbuf_len, "tsgm_warp_predict_noalloc: outputs alias inputs");
        return TSGM_ERR_INVALID_ARG;
    }
    if (width < 1 || height < 1 ||
        (int64_t)width * (int64_t)height > (int64_t)TSGM_NOALLOC_MAX_PIXELS) {
        char msg[200];
        std::snprintf(msg, sizeof(msg),
                      "tsgm_warp_predict_noalloc: %d x %d pixels exceeds the fixed scratch of %d "
                      "pixels (use tsgm_warp_predict with a context)",
                      (int)width, (int)height, (int)TSGM_NOALLOC_MAX_PIXELS);
        put_error(errbuf, errbuf_len, msg);
        return TSGM_ERR_INVALID_ARG;
    }
    if (!(q >= 0.0f && q <= FLT_MAX)) {
        put_error(errbuf, errbuf_len, "tsgm_warp_predict_noalloc: q must be finite and >= 0");
        return TSGM_ERR_INVALID_ARG;
    }
    float H32[16];
    if (tsgm_build_H(R, t, K, baseline, H32) != TSGM_OK) {
        put_error(errbuf, errbuf_len,
                  "tsgm_warp_predict_noalloc: invalid pose or calibration (f, baseline > 0)");
        return TSGM_ERR_INVALID_ARG;
    }
    unsigned long long* keys = nullptr;
    cudaError_t e = keys_on_current_device(&keys);
    if (e == cudaSuccess) {
        const int n = width * height;
        cudaStream_t st = (cudaStream_t)cuda_stream;
        // the array keeps the previous call's keys: every used key starts empty again
        e = cudaMemsetAsync(keys, 0xFF, sizeof(unsigned long long) * (size_t)n, st);
        if (e == cudaSuccess)
            e = tsgm::launch_warp_scatter(prev_D, prev_P, H32, K[2], K[5], width, height, keys, st);
        if (e == cudaSuccess)
            e = tsgm::launch_warp_gather(keys, prev_D, prev_P, q, n, pred_D, pred_P, st);
    }
    if (e != cudaSuccess) {
        char msg[200];
        std::snprintf(msg, sizeof(msg), "tsgm_warp_predict_noalloc: %s", cudaGetErrorString(e));
        put_error(errbuf, errbuf_len, msg);
        return TSGM_ERR_CUDA;
    }
    return TSGM_OK;
}
