// A small multilayer perceptron for the learned warm start of the Krylov solve:
// in -> 64 -> 64 -> out with ReLU after the two hidden layers.  Weights are BF16 (an
// FP32 master copy is kept for the optimiser), biases FP32, all accumulation FP32.
//
// One thread evaluates one row (one triangle's feature vector).  The weights of all
// layers are staged in shared memory as FP32 (converted from BF16 once per block).  The
// backward pass keeps each thread's hidden activations in shared memory and adds the
// weight gradients of its rows into a shared-memory copy of the gradient, which each
// block then adds to the global gradient.  Loss: (1 / 2R) sum over rows and outputs of
// (w (y - t))^2, with per-output row weights w (1 when none are given).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace {

constexpr int HID = 64;
constexpr int MLP_THREADS = 64;
constexpr int MAX_IN = 96, MAX_OUT = 32;

struct Dims {
    int in, out;
    // offsets into the parameter vector: W1 [HID][in], b1, W2 [HID][HID], b2, W3 [out][HID], b3
    int w1, b1, w2, b2, w3, b3, total;
};

Dims make_dims(int in, int out) {
    Dims d{in, out, 0, 0, 0, 0, 0, 0, 0};
    d.w1 = 0;
    d.b1 = d.w1 + HID * in;
    d.w2 = d.b1 + HID;
    d.b2 = d.w2 + HID * HID;
    d.w3 = d.b2 + HID;
    d.b3 = d.w3 + out * HID;
    d.total = d.b3 + out;
    return d;
}

// shared-memory copy of the parameters: weights from the BF16 copy, biases FP32
__device__ void stage_params(const Dims &d, const __nv_bfloat16 *wb, const float *master, float *sp) {
    for (int i = threadIdx.x; i < d.total; i += blockDim.x) {
        const bool bias = (i >= d.b1 && i < d.w2) || (i >= d.b2 && i < d.w3) || i >= d.b3;
        sp[i] = bias ? master[i] : __bfloat162float(wb[i]);
    }
}

// forward of one row; h1, h2 (HID each) receive the hidden activations
__device__ __forceinline__ void forward_row(const Dims &d, const float *sp, const float *x, float *h1, float *h2,
                                            float *y) {
    for (int i = 0; i < HID; ++i) {
        float a = sp[d.b1 + i];
        const float *w = sp + d.w1 + i * d.in;
        for (int j = 0; j < d.in; ++j) a = fmaf(w[j], x[j], a);
        h1[i] = fmaxf(a, 0.0f);
    }
    for (int i = 0; i < HID; ++i) {
        float a = sp[d.b2 + i];
        const float *w = sp + d.w2 + i * HID;
        for (int j = 0; j < HID; ++j) a = fmaf(w[j], h1[j], a);
        h2[i] = fmaxf(a, 0.0f);
    }
    for (int o = 0; o < d.out; ++o) {
        float a = sp[d.b3 + o];
        const float *w = sp + d.w3 + o * HID;
        for (int j = 0; j < HID; ++j) a = fmaf(w[j], h2[j], a);
        y[o] = a;
    }
}

__global__ void __launch_bounds__(MLP_THREADS) k_mlp_forward(Dims d, const __nv_bfloat16 *wb, const float *master,
                                                             const float *X, float *Y, int64_t rows) {
    extern __shared__ float smem[];
    float *sp = smem;
    float *h = sp + d.total + threadIdx.x * 2 * HID;  // per-thread hidden activations
    stage_params(d, wb, master, sp);
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        float x[MAX_IN], y[MAX_OUT];
        for (int j = 0; j < d.in; ++j) x[j] = X[r * d.in + j];
        forward_row(d, sp, x, h, h + HID, y);
        for (int o = 0; o < d.out; ++o) Y[r * d.out + o] = y[o];
    }
}

// gradient of the loss over rows; grad (d.total FP32) and loss (double) are accumulated
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_grad(Dims d, const __nv_bfloat16 *wb, const float *master,
                                                          const float *X, const float *T, const float *Wt,
                                                          int64_t rows, float *grad, double *loss) {
    extern __shared__ float smem[];
    float *sp = smem;
    float *sg = sp + d.total;                           // block's gradient
    float *h = sg + d.total + threadIdx.x * 3 * HID;    // h1, h2, delta of this thread
    stage_params(d, wb, master, sp);
    for (int i = threadIdx.x; i < d.total; i += blockDim.x) sg[i] = 0.0f;
    __syncthreads();
    const float inv_rows = 1.0f / (float)rows;
    double lsum = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        float x[MAX_IN], y[MAX_OUT];
        for (int j = 0; j < d.in; ++j) x[j] = X[r * d.in + j];
        float *h1 = h, *h2 = h + HID, *dl = h + 2 * HID;
        forward_row(d, sp, x, h1, h2, y);
        // output layer: e = w (y - t); dW3 = w e h2^T / R, db3 = w e / R
        for (int o = 0; o < d.out; ++o) {
            const float w = Wt ? Wt[r * d.out + o] : 1.0f;
            const float e = w * (y[o] - T[r * d.out + o]);
            lsum += 0.5 * (double)e * (double)e;
            y[o] = w * e * inv_rows;
            atomicAdd(sg + d.b3 + o, y[o]);
            for (int j = 0; j < HID; ++j) atomicAdd(sg + d.w3 + o * HID + j, y[o] * h2[j]);
        }
        // second hidden layer: delta2 = (W3^T e) * [a2 > 0]
        for (int j = 0; j < HID; ++j) {
            float a = 0.0f;
            for (int o = 0; o < d.out; ++o) a = fmaf(sp[d.w3 + o * HID + j], y[o], a);
            dl[j] = h2[j] > 0.0f ? a : 0.0f;
        }
        for (int i = 0; i < HID; ++i) {
            if (dl[i] == 0.0f) continue;
            atomicAdd(sg + d.b2 + i, dl[i]);
            for (int j = 0; j < HID; ++j) atomicAdd(sg + d.w2 + i * HID + j, dl[i] * h1[j]);
        }
        // first hidden layer: delta1 = (W2^T delta2) * [a1 > 0]  (into h2, no longer needed)
        for (int j = 0; j < HID; ++j) {
            float a = 0.0f;
            for (int i = 0; i < HID; ++i) a = fmaf(sp[d.w2 + i * HID + j], dl[i], a);
            h2[j] = h1[j] > 0.0f ? a : 0.0f;
        }
        for (int i = 0; i < HID; ++i) {
            if (h2[i] == 0.0f) continue;
            atomicAdd(sg + d.b1 + i, h2[i]);
            for (int j = 0; j < d.in; ++j) atomicAdd(sg + d.w1 + i * d.in + j, h2[i] * x[j]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d.total; i += blockDim.x)
        if (sg[i] != 0.0f) atomicAdd(grad + i, sg[i]);
    // loss: warp sums, one atomic per warp
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, lsum / (double)rows);
}

// Adam (Kingma & Ba, 2015) on the FP32 master weights, then their BF16 copy
__global__ void k_mlp_adam(int n, float *master, __nv_bfloat16 *wb, const float *grad, float *m, float *v, float lr,
                           float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float w = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        master[i] = w;
        wb[i] = __float2bfloat16_rn(w);
    }
}

__global__ void k_mlp_round(int n, float *master, __nv_bfloat16 *wb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16_rn(master[i]);
}

thread_local std::string g_mlp_err;

}  // namespace

struct festung_mlp {
    Dims d;
    float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wb = nullptr;
    double *loss = nullptr, *hloss = nullptr;
    int64_t steps = 0;
    cudaStream_t stream = nullptr;
    int sms = 1;
};

namespace {

int mlp_fail(festung_mlp *n, cudaError_t e) {
    g_mlp_err = std::string("CUDA: ") + cudaGetErrorString(e);
    (void)n;
    return e == cudaErrorMemoryAllocation ? FESTUNG_ENOMEM : FESTUNG_ECUDA;
}

size_t fwd_smem(const Dims &d) { return ((size_t)d.total + (size_t)MLP_THREADS * 2 * HID) * sizeof(float); }
size_t grad_smem(const Dims &d) { return ((size_t)2 * d.total + (size_t)MLP_THREADS * 3 * HID) * sizeof(float); }

}  // namespace

extern "C" {

int festung_mlp_create(int n_in, int n_out, uint64_t seed, festung_mlp **out) {
    g_mlp_err.clear();
    if (!out || n_in < 1 || n_in > MAX_IN || n_out < 1 || n_out > MAX_OUT) {
        g_mlp_err = "bad MLP dimensions (1..96 inputs, 1..32 outputs)";
        return FESTUNG_EINVAL;
    }
    festung_mlp *n = new (std::nothrow) festung_mlp();
    if (!n) return FESTUNG_ENOMEM;
    n->d = make_dims(n_in, n_out);
    const int T = n->d.total;
    // Glorot-uniform weights from a seeded 64-bit linear congruential generator
    // (Knuth's MMIX constants), zero biases
    std::vector<float> h(T, 0.0f);
    uint64_t s = seed * 2862933555777941757ull + 3037000493ull;
    auto uni = [&]() {
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        return (double)(s >> 11) / 9007199254740992.0;  // [0, 1)
    };
    auto fill = [&](int off, int rows, int cols) {
        const double a = std::sqrt(6.0 / (rows + cols));
        for (int i = 0; i < rows * cols; ++i) h[off + i] = (float)((2.0 * uni() - 1.0) * a);
    };
    fill(n->d.w1, HID, n_in);
    fill(n->d.w2, HID, HID);
    fill(n->d.w3, n_out, HID);
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaMalloc(&n->master, T * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&n->grad, T * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&n->m, T * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&n->v, T * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&n->wb, T * sizeof(__nv_bfloat16))) != cudaSuccess ||
        (e = cudaMalloc(&n->loss, sizeof(double))) != cudaSuccess ||
        (e = cudaMallocHost(&n->hloss, sizeof(double))) != cudaSuccess ||
        (e = cudaMemcpy(n->master, h.data(), T * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(n->m, 0, T * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(n->v, 0, T * sizeof(float))) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)grad_smem(n->d))) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fwd_smem(n->d))) != cudaSuccess) {
        int rc = mlp_fail(n, e);
        festung_mlp_destroy(n);
        return rc;
    }
    k_mlp_round<<<(T + 255) / 256, 256>>>(T, n->master, n->wb);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
        int rc = mlp_fail(n, e);
        festung_mlp_destroy(n);
        return rc;
    }
    *out = n;
    return FESTUNG_OK;
}

int festung_mlp_sizes(const festung_mlp *n, int *n_in, int *n_out, int *n_params) {
    if (!n) return FESTUNG_EINVAL;
    if (n_in) *n_in = n->d.in;
    if (n_out) *n_out = n->d.out;
    if (n_params) *n_params = n->d.total;
    return FESTUNG_OK;
}

int festung_mlp_set_stream(festung_mlp *n, void *stream) {
    if (!n) return FESTUNG_EINVAL;
    n->stream = (cudaStream_t)stream;
    return FESTUNG_OK;
}

int festung_mlp_forward(festung_mlp *n, const float *X, float *Y, int64_t rows) {
    if (!n || !X || !Y || rows < 0) return FESTUNG_EINVAL;
    if (rows == 0) return FESTUNG_OK;
    const int grid = (int)std::min<int64_t>((rows + MLP_THREADS - 1) / MLP_THREADS, (int64_t)n->sms * 8);
    k_mlp_forward<<<grid, MLP_THREADS, fwd_smem(n->d), n->stream>>>(n->d, n->wb, n->master, X, Y, rows);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FESTUNG_OK : mlp_fail(n, e);
}

int festung_mlp_grad(festung_mlp *n, const float *X, const float *T, const float *Wt, int64_t rows, double *loss) {
    if (!n || !X || !T || rows < 1) return FESTUNG_EINVAL;
    cudaError_t e;
    if ((e = cudaMemsetAsync(n->grad, 0, n->d.total * sizeof(float), n->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(n->loss, 0, sizeof(double), n->stream)) != cudaSuccess)
        return mlp_fail(n, e);
    const int grid = (int)std::min<int64_t>((rows + MLP_THREADS - 1) / MLP_THREADS, (int64_t)n->sms * 2);
    k_mlp_grad<<<grid, MLP_THREADS, grad_smem(n->d), n->stream>>>(n->d, n->wb, n->master, X, T, Wt, rows,
                                                                  n->grad, n->loss);
    if ((e = cudaGetLastError()) != cudaSuccess) return mlp_fail(n, e);
    if (loss) {
        if ((e = cudaMemcpyAsync(n->hloss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(n->stream)) != cudaSuccess)
            return mlp_fail(n, e);
        *loss = *n->hloss;
    }
    return FESTUNG_OK;
}

int festung_mlp_adam(festung_mlp *n, double lr) {
    if (!n || !(lr > 0.0)) return FESTUNG_EINVAL;
    n->steps += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)n->steps), c2 = 1.0f - std::pow(b2, (float)n->steps);
    const int T = n->d.total;
    k_mlp_adam<<<(T + 255) / 256, 256, 0, n->stream>>>(T, n->master, n->wb, n->grad, n->m, n->v, (float)lr, b1, b2,
                                                         1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FESTUNG_OK : mlp_fail(n, e);
}

int festung_mlp_get(const festung_mlp *n, float *params, float *grad) {
    if (!n) return FESTUNG_EINVAL;
    cudaError_t e = cudaStreamSynchronize(n->stream);
    if (e == cudaSuccess && params)
        e = cudaMemcpy(params, n->master, n->d.total * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && grad) e = cudaMemcpy(grad, n->grad, n->d.total * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? FESTUNG_OK : mlp_fail(const_cast<festung_mlp *>(n), e);
}

int festung_mlp_set(festung_mlp *n, const float *params) {
    if (!n || !params) return FESTUNG_EINVAL;
    cudaError_t e = cudaStreamSynchronize(n->stream);
    if (e == cudaSuccess) e = cudaMemcpy(n->master, params, n->d.total * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return mlp_fail(n, e);
    k_mlp_round<<<(n->d.total + 255) / 256, 256, 0, n->stream>>>(n->d.total, n->master, n->wb);
    e = cudaStreamSynchronize(n->stream);
    return e == cudaSuccess ? FESTUNG_OK : mlp_fail(n, e);
}

const char *festung_mlp_last_error(void) { return g_mlp_err.c_str(); }

void festung_mlp_destroy(festung_mlp *n) {
    if (!n) return;
    if (n->stream) cudaStreamSynchronize(n->stream);
    cudaFree(n->master);
    cudaFree(n->grad);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->wb);
    cudaFree(n->loss);
    if (n->hloss) cudaFreeHost(n->hloss);
    delete n;
}

}  // extern "C"
