// Krylov building blocks: fused vector updates with block-level partial dot products
// and single-block scalar updates.  All scalars live in device memory, so a sequence
// of iterations needs no host round trip and can be captured in one CUDA graph; once
// `done` is set every kernel of the sequence returns at entry.
#pragma once

#include <cstdint>

namespace festung {

struct KScal {
    double rho, alpha, omega, beta;
    double r2, b2, tol2;
    double den;
    double ss;    // BiCGStab: (s, s) of the current iteration
    double r2_0;  // (r, r) at the start of the solve
    int done, breakdown, iter, sconv;
    int first;    // BiCGStab: no update of x and r is owed from a previous iteration
    int pending;  // BiCGStab: x += alpha ph + omega sh, r = s - omega t still to apply
};

constexpr int RED_THREADS = 256;

// Per-problem view of the union of a batch of problems (krylov_solve_batch): every
// problem runs its own Krylov iteration with its own KScal; reductions are summed per
// problem.  eprob == nullptr: a single problem (block partials, one KScal).
struct BatchView {
    const int32_t *eprob = nullptr;  // K: problem of each element
    double *acc = nullptr;           // 4 x nprob sums, zero between reductions
    int *alldone = nullptr;          // 1 once every problem's iteration is done
    int nprob = 1;
};

// Reductions of a BiCGStab step fused into the end of an operator apply y = S x:
//   FUSED_EPI_NONE   none;
//   FUSED_EPI_ALPHA  y = v:  (r0, v) -> alpha;
//   FUSED_EPI_OMEGA  y = t:  (t, s), (t, t), (r0, s), (r0, t) -> omega, rho, beta.
constexpr int FUSED_EPI_NONE = 0;
constexpr int FUSED_EPI_ALPHA = 1;
constexpr int FUSED_EPI_OMEGA = 2;

// Block sum of up to 3 values; thread 0 writes part[p * nblk + blockIdx.x].
template <int NP>
__device__ __forceinline__ void block_partials(float (&v)[NP], double *part) {
    __shared__ double sh[NP][RED_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float a = v[p];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) sh[p][wid] = (double)a;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            double a = (lane < RED_THREADS / 32) ? sh[p][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) part[p * gridDim.x + blockIdx.x] = a;
        }
    }
}

template <int NP>
__device__ __forceinline__ void block_partials(double (&v)[NP], double *part) {
    __shared__ double sh[NP][RED_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        double a = v[p];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) sh[p][wid] = a;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            double a = (lane < RED_THREADS / 32) ? sh[p][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) part[p * gridDim.x + blockIdx.x] = a;
        }
    }
}

// Sum of the partials of slot p over nblk blocks (call from a single block of 1024 threads).
__device__ __forceinline__ double sum_partials(const double *part, int p, int nblk) {
    __shared__ double sh[32];
    double a = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) a += part[p * nblk + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = a;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    const double res = sh[0];
    __syncthreads();
    return res;
}

}  // namespace festung
