// Operator apply for callers that cannot allocate device memory.
//
// This variant evaluates y = S x with the two-pass kernels, whose eliminated flux
// unknowns Z^1, Z^2 (2 x N x K values) travel through global scratch.  The scratch is
// one fixed array that is part of the library image, so the call itself never
// allocates or frees (festung_apply allocates its context workspace on first use).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"
#include "ops.h"

namespace {

// 32 MiB: room for Z^1 and Z^2 with N*K <= 2,097,152 in FP64 or 4,194,304 in FP32.
// Every device that loads the library holds this array until the process exits.
constexpr size_t kScratchBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_apply_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

}  // namespace

extern "C" int festung_apply_noalloc(festung_ctx *c, const void *x, void *y, int prec, double dt) {
    if (!c) return FESTUNG_EINVAL;
    if (c->p < 0) {
        c->err = "festung_setup has not been called";
        return FESTUNG_ESTATE;
    }
    if (!x || !y || x == y || !(dt >= 0.0) || (prec != FESTUNG_FP64 && prec != FESTUNG_FP32)) {
        c->err = "bad apply arguments";
        return FESTUNG_EINVAL;
    }
    const size_t elem = (prec == FESTUNG_FP64) ? sizeof(double) : sizeof(float);
    const size_t need = 2 * size_t(c->N) * size_t(c->K) * elem;
    if (need > kScratchBytes) {
        c->err = "festung_apply_noalloc: needs " + std::to_string(need) + " bytes of scratch for 2 x N x K = 2 x " +
                 std::to_string(c->N) + " x " + std::to_string(c->K) + " values, above the fixed " +
                 std::to_string(kScratchBytes) + " bytes; use festung_apply";
        return FESTUNG_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        c->err = std::string("festung_apply_noalloc: no usable current device: ") + cudaGetErrorString(e);
        return FESTUNG_ECUDA;
    }
    // The array's device address belongs to the device's current primary context, which a
    // cudaDeviceReset replaces.  So it is looked up again on every call made outside stream
    // capture (the lookup is cheap), and the last address found is used only while the
    // context's stream is being captured.  The first call on a device must therefore come
    // before any capture.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(c->stream, &cap);
    if (e != cudaSuccess) {
        c->err = std::string("festung_apply_noalloc: cudaStreamIsCapturing failed: ") + cudaGetErrorString(e);
        return FESTUNG_ECUDA;
    }
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_apply_scratch);
            if (e != cudaSuccess || !ptr) {
                c->err = std::string("festung_apply_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
                return FESTUNG_ECUDA;
            }
            g_scratch_addr[dev] = ptr;
        } else if (!g_scratch_addr[dev]) {
            c->err = "festung_apply_noalloc: the first call on a device must come before any stream capture";
            return FESTUNG_ESTATE;
        }
        base = g_scratch_addr[dev];
    }
    // Z^1 and Z^2 are written completely by the flux pass before the second pass reads
    // them, so nothing has to be cleared between calls.
    if (prec == FESTUNG_FP64) {
        double *Z1 = static_cast<double *>(base);
        festung::launch_apply_twopass<double>(c, static_cast<const double *>(x), static_cast<double *>(y), Z1,
                                      Z1 + c->N * c->K, dt, nullptr, c->stream);
    } else {
        float *Z1 = static_cast<float *>(base);
        festung::launch_apply_twopass<float>(c, static_cast<const float *>(x), static_cast<float *>(y), Z1, Z1 + c->N * c->K,
                                     (float)dt, nullptr, c->stream);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("festung_apply_noalloc: ") + cudaGetErrorString(e);
        return FESTUNG_ECUDA;
    }
    return FESTUNG_OK;
}
