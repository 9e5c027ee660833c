// Kernels of one Krylov iteration with the scalar updates folded into the reductions.
//
// Each reducing kernel writes one partial per block; the last block to finish (found
// with a device-wide counter) sums the partials in block order, so results are
// bitwise reproducible, and updates the device-resident scalars.  A kernel that finds
// `done` set at entry returns at once, so a captured sequence of iterations costs
// nothing after convergence.  Vectors are N x K; flat kernels move 16 bytes per access.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

#include "krylov.cuh"

namespace festung {

template <typename T>
using Acc = typename std::conditional<std::is_same<T, float>::value, float, double>::type;

// y = P_k q for the BF16 block of triangle k (layout of k_blockinv: 16-byte chunks [q][K])
template <typename T, int N>
__device__ __forceinline__ void block_matvec(const __nv_bfloat16 *__restrict__ P, int K, int k, const T (&q)[N],
                                             T (&y)[N]) {
    constexpr int NQ = (N * N + 7) / 8;
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] = T(0);
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(P) + (int64_t)c * K + k);
        const __nv_bfloat16 *b = reinterpret_cast<const __nv_bfloat16 *>(&raw);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int e = 8 * c + t;
            if (e < N * N) y[e / N] += (T)__bfloat162float(b[t]) * q[e % N];
        }
    }
}

// Called by every thread of a block after its partials are written.  True in exactly
// one block, the last one, which then sees all partials.
__device__ __forceinline__ bool last_block(unsigned int *counter) {
    __shared__ bool amlast;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) amlast = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    return amlast;
}

// Sum of slot p of the partials of a grid of nblk blocks, read past L1 (the partials
// were written by other SMs); called by all threads of one block.
__device__ __forceinline__ double sum_partials_cg(const double *part, int p, int nblk) {
    __shared__ double sh[32];
    double a = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) a += __ldcg(part + p * nblk + i);
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

// 16-byte vector of T
template <typename T>
struct V16 {
    static constexpr int n = 16 / sizeof(T);
    T v[n];
};

template <typename T>
__device__ __forceinline__ V16<T> ld16(const T *p, int64_t i) {
    V16<T> r;
    *reinterpret_cast<float4 *>(r.v) = *reinterpret_cast<const float4 *>(p + i);
    return r;
}
template <typename T>
__device__ __forceinline__ void st16(T *p, int64_t i, const V16<T> &r) {
    *reinterpret_cast<float4 *>(p + i) = *reinterpret_cast<const float4 *>(r.v);
}

// Flat loop over n entries with 16-byte accesses; the body handles entries i0..i0+w-1.
#define FLAT_LOOP(n, ...)                                                                           \
    {                                                                                               \
        constexpr int W_ = 16 / sizeof(T);                                                          \
        const int64_t nv_ = (n) / W_;                                                               \
        for (int64_t q_ = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q_ < nv_;                 \
             q_ += (int64_t)gridDim.x * blockDim.x) {                                               \
            const int64_t i0 = q_ * W_;                                                             \
            constexpr int w = W_;                                                                   \
            __VA_ARGS__                                                                             \
        }                                                                                           \
        for (int64_t i0 = nv_ * W_ + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < (n);      \
             i0 += (int64_t)gridDim.x * blockDim.x) {                                               \
            constexpr int w = 1;                                                                    \
            __VA_ARGS__                                                                             \
        }                                                                                           \
    }

// ---------------------------------------------------------------------------
// BiCGStab (right preconditioner P^{-1} = block-Jacobi inverse, or 1/(2|T_k|))
// ---------------------------------------------------------------------------

// MODE 0: p = r + beta (p - omega v); out = P^{-1} p.
// MODE 1: s = r - alpha v; out = P^{-1} s; (s, s) -> last block: converged on s?
template <typename T, int N, int MODE>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_prec(int K, const T *__restrict__ r, T *__restrict__ pv,
                                                           const T *__restrict__ v, T *__restrict__ out,
                                                           const __nv_bfloat16 *__restrict__ P,
                                                           const T *__restrict__ inv, double *part, KScal *sc,
                                                           unsigned int *counter) {
    if (sc->done) return;
    const T beta = (T)sc->beta, omega = (T)sc->omega, alpha = (T)sc->alpha;
    Acc<T> acc[1] = {Acc<T>(0)};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        T q[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int i = j * K + k;
            const T qi = MODE == 0 ? r[i] + beta * (pv[i] - omega * v[i]) : r[i] - alpha * v[i];
            pv[i] = qi;
            q[j] = qi;
            if (MODE == 1) acc[0] += (Acc<T>)qi * (Acc<T>)qi;
        }
        if (P) {
            T y[N];
            block_matvec<T, N>(P, K, k, q, y);
#pragma unroll
            for (int i = 0; i < N; ++i) out[i * K + k] = y[i];
        } else {
            const T iv = inv[k];
#pragma unroll
            for (int i = 0; i < N; ++i) out[i * K + k] = q[i] * iv;
        }
    }
    if (MODE == 1) {
        block_partials<1>(acc, part);
        if (last_block(counter)) {
            const double s2 = sum_partials_cg(part, 0, gridDim.x);
            if (threadIdx.x == 0) {
                if (s2 <= sc->tol2 * sc->b2) {
                    sc->sconv = 1;
                    sc->r2 = s2;
                    sc->iter += 1;
                    sc->done = 1;
                }
                *counter = 0;
            }
        }
    }
}

// (r0, v) -> alpha = rho / (r0, v)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_alpha(int64_t n, const T *__restrict__ r0,
                                                            const T *__restrict__ v, double *part, KScal *sc,
                                                            unsigned int *counter) {
    if (sc->done) return;
    Acc<T> acc[1] = {Acc<T>(0)};
    FLAT_LOOP(n, {
        if (w > 1) {
            const V16<T> a = ld16(r0, i0), b = ld16(v, i0);
            for (int e = 0; e < w; ++e) acc[0] += (Acc<T>)a.v[e] * (Acc<T>)b.v[e];
        } else {
            acc[0] += (Acc<T>)r0[i0] * (Acc<T>)v[i0];
        }
    })
    block_partials<1>(acc, part);
    if (last_block(counter)) {
        const double den = sum_partials_cg(part, 0, gridDim.x);
        if (threadIdx.x == 0) {
            if (!(fabs(den) > 1e-300) || !isfinite(den)) {
                sc->breakdown = 1;
                sc->done = 1;
            } else {
                sc->alpha = sc->rho / den;
            }
            *counter = 0;
        }
    }
}

// (t, s), (t, t) -> omega = (t, s) / (t, t)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_omega(int64_t n, const T *__restrict__ t,
                                                            const T *__restrict__ s, double *part, KScal *sc,
                                                            unsigned int *counter) {
    if (sc->done) return;
    Acc<T> acc[2] = {Acc<T>(0), Acc<T>(0)};
    FLAT_LOOP(n, {
        if (w > 1) {
            const V16<T> a = ld16(t, i0), b = ld16(s, i0);
            for (int e = 0; e < w; ++e) {
                acc[0] += (Acc<T>)a.v[e] * (Acc<T>)b.v[e];
                acc[1] += (Acc<T>)a.v[e] * (Acc<T>)a.v[e];
            }
        } else {
            acc[0] += (Acc<T>)t[i0] * (Acc<T>)s[i0];
            acc[1] += (Acc<T>)t[i0] * (Acc<T>)t[i0];
        }
    })
    block_partials<2>(acc, part);
    if (last_block(counter)) {
        const double ts = sum_partials_cg(part, 0, gridDim.x);
        const double tt = sum_partials_cg(part, 1, gridDim.x);
        if (threadIdx.x == 0) {
            if (!(tt > 0.0) || !isfinite(ts) || ts == 0.0) {
                sc->breakdown = 1;
                sc->done = 1;
            } else {
                sc->omega = ts / tt;
            }
            *counter = 0;
        }
    }
}

// x += alpha ph + omega sh; r = s - omega t; (r0, r), (r, r) -> next rho, beta, convergence
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_xr(int64_t n, T *__restrict__ x, const T *__restrict__ ph,
                                                         const T *__restrict__ sh, const T *__restrict__ s,
                                                         const T *__restrict__ t, T *__restrict__ r,
                                                         const T *__restrict__ r0, double *part, KScal *sc,
                                                         unsigned int *counter) {
    if (sc->done) return;
    const T alpha = (T)sc->alpha, omega = (T)sc->omega;
    Acc<T> acc[2] = {Acc<T>(0), Acc<T>(0)};
    FLAT_LOOP(n, {
        if (w > 1) {
            V16<T> xv = ld16(x, i0);
            const V16<T> pa = ld16(ph, i0), sa = ld16(sh, i0), sv = ld16(s, i0), tv = ld16(t, i0),
                         rz = ld16(r0, i0);
            V16<T> rv;
            for (int e = 0; e < w; ++e) {
                xv.v[e] += alpha * pa.v[e] + omega * sa.v[e];
                rv.v[e] = sv.v[e] - omega * tv.v[e];
                acc[0] += (Acc<T>)rz.v[e] * (Acc<T>)rv.v[e];
                acc[1] += (Acc<T>)rv.v[e] * (Acc<T>)rv.v[e];
            }
            st16(x, i0, xv);
            st16(r, i0, rv);
        } else {
            x[i0] += alpha * ph[i0] + omega * sh[i0];
            const T ri = s[i0] - omega * t[i0];
            r[i0] = ri;
            acc[0] += (Acc<T>)r0[i0] * (Acc<T>)ri;
            acc[1] += (Acc<T>)ri * (Acc<T>)ri;
        }
    })
    block_partials<2>(acc, part);
    if (last_block(counter)) {
        const double rho_new = sum_partials_cg(part, 0, gridDim.x);
        const double r2 = sum_partials_cg(part, 1, gridDim.x);
        if (threadIdx.x == 0) {
            sc->iter += 1;
            sc->r2 = r2;
            if (r2 <= sc->tol2 * sc->b2) {
                sc->done = 1;
            } else if (!(fabs(rho_new) > 1e-300) || !isfinite(rho_new)) {
                sc->breakdown = 1;
                sc->done = 1;
            } else {
                sc->beta = (rho_new / sc->rho) * (sc->alpha / sc->omega);
                sc->rho = rho_new;
            }
            *counter = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// CG (symmetric S; preconditioner SPD)
// ---------------------------------------------------------------------------

// (p, q) -> alpha = (r, z) / (p, q)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_cg_alpha(int64_t n, const T *__restrict__ p,
                                                          const T *__restrict__ q, double *part, KScal *sc,
                                                          unsigned int *counter) {
    if (sc->done) return;
    Acc<T> acc[1] = {Acc<T>(0)};
    FLAT_LOOP(n, {
        if (w > 1) {
            const V16<T> a = ld16(p, i0), b = ld16(q, i0);
            for (int e = 0; e < w; ++e) acc[0] += (Acc<T>)a.v[e] * (Acc<T>)b.v[e];
        } else {
            acc[0] += (Acc<T>)p[i0] * (Acc<T>)q[i0];
        }
    })
    block_partials<1>(acc, part);
    if (last_block(counter)) {
        const double pq = sum_partials_cg(part, 0, gridDim.x);
        if (threadIdx.x == 0) {
            if (!(pq > 0.0) || !isfinite(pq)) {
                sc->breakdown = 1;
                sc->done = 1;
            } else {
                sc->alpha = sc->rho / pq;
            }
            *counter = 0;
        }
    }
}

// x += alpha p; r -= alpha q; partial (r, r) into part2 (consumed by k_cg_prec)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_cg_xr(int64_t n, T *__restrict__ x, const T *__restrict__ p,
                                                       const T *__restrict__ q, T *__restrict__ r, double *part2,
                                                       const KScal *sc) {
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    Acc<T> acc[1] = {Acc<T>(0)};
    FLAT_LOOP(n, {
        if (w > 1) {
            V16<T> xv = ld16(x, i0), rv = ld16(r, i0);
            const V16<T> pv = ld16(p, i0), qv = ld16(q, i0);
            for (int e = 0; e < w; ++e) {
                xv.v[e] += alpha * pv.v[e];
                rv.v[e] -= alpha * qv.v[e];
                acc[0] += (Acc<T>)rv.v[e] * (Acc<T>)rv.v[e];
            }
            st16(x, i0, xv);
            st16(r, i0, rv);
        } else {
            x[i0] += alpha * p[i0];
            const T ri = r[i0] - alpha * q[i0];
            r[i0] = ri;
            acc[0] += (Acc<T>)ri * (Acc<T>)ri;
        }
    })
    block_partials<1>(acc, part2);
}

// z = P^{-1} r; (r, z) -> with (r, r) from k_cg_xr: rho, beta, convergence.
// init: first call of a solve (only rho is set, no convergence test)
template <typename T, int N>
__global__ void __launch_bounds__(RED_THREADS) k_cg_prec(int K, const T *__restrict__ r, T *__restrict__ z,
                                                         const __nv_bfloat16 *__restrict__ P,
                                                         const T *__restrict__ inv, double *part,
                                                         const double *part2, int nblk2, KScal *sc,
                                                         unsigned int *counter, int init) {
    if (sc->done) return;
    Acc<T> acc[1] = {Acc<T>(0)};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        T q[N];
#pragma unroll
        for (int j = 0; j < N; ++j) q[j] = r[j * K + k];
        T y[N];
        if (P) {
            block_matvec<T, N>(P, K, k, q, y);
        } else {
#pragma unroll
            for (int i = 0; i < N; ++i) y[i] = q[i] * inv[k];
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            z[i * K + k] = y[i];
            acc[0] += (Acc<T>)y[i] * (Acc<T>)q[i];
        }
    }
    block_partials<1>(acc, part);
    if (last_block(counter)) {
        const double rz = sum_partials_cg(part, 0, gridDim.x);
        const double r2 = init ? 0.0 : sum_partials_cg(part2, 0, nblk2);
        if (threadIdx.x == 0) {
            if (init) {
                sc->rho = rz;
            } else {
                sc->iter += 1;
                sc->r2 = r2;
                if (r2 <= sc->tol2 * sc->b2) {
                    sc->done = 1;
                } else {
                    sc->beta = rz / sc->rho;
                    sc->rho = rz;
                }
            }
            *counter = 0;
        }
    }
}

// p = z + beta p   (init: p = z)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_cg_p(int64_t n, T *__restrict__ p, const T *__restrict__ z,
                                                      const KScal *sc, int init) {
    if (sc->done) return;
    const T beta = init ? T(0) : (T)sc->beta;
    FLAT_LOOP(n, {
        if (w > 1) {
            V16<T> pv = ld16(p, i0);
            const V16<T> zv = ld16(z, i0);
            for (int e = 0; e < w; ++e) pv.v[e] = init ? zv.v[e] : zv.v[e] + beta * pv.v[e];
            st16(p, i0, pv);
        } else {
            p[i0] = init ? z[i0] : z[i0] + beta * p[i0];
        }
    })
}

#undef FLAT_LOOP

}  // namespace festung
