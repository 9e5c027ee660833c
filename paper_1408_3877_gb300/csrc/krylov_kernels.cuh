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

// Block sum of NP values for any block size (a multiple of 32, at most 1024); thread 0
// of warp 0 writes part[p * gridDim.x + blockIdx.x].
template <int NP, typename A>
__device__ __forceinline__ void block_partials_any(A (&v)[NP], double *part) {
    __shared__ double sh[NP][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)((blockDim.x + 31) >> 5);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        A a = v[p];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) sh[p][wid] = (double)a;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            double a = lane < nw ? sh[p][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) part[p * gridDim.x + blockIdx.x] = a;
        }
    }
}

// Scalar updates of BiCGStab, run by one thread of the last block of a reduction.
// After v = S ph: alpha = rho / (r0, v).  The update owed from the previous iteration
// has been applied by now (k_bicg_next).
__device__ __forceinline__ void bicg_alpha_scalars(double r0v, KScal *sc) {
    if (!(fabs(r0v) > 1e-300) || !isfinite(r0v)) {
        sc->breakdown = 1;
        sc->done = 1;
    } else {
        sc->alpha = sc->rho / r0v;
    }
    sc->first = 0;
    sc->pending = 0;
}

// After t = S sh: omega = (t, s) / (t, t); the next residual r = s - omega t is not
// formed here, its dot products follow from those of s and t:
//   (r0, r) = (r0, s) - omega (r0, t),  (r, r) = (s, s) - omega (t, s);
// beta = ((r0, r) / rho) (alpha / omega).  The updates of x and r are left to the
// next iteration's k_bicg_next (or to k_bicg_finish once the solve stops).
__device__ __forceinline__ void bicg_omega_scalars(double ts, double tt, double r0s, double r0t, KScal *sc) {
    if (!(tt > 0.0) || !isfinite(ts) || ts == 0.0 || !isfinite(r0s) || !isfinite(r0t)) {
        sc->breakdown = 1;
        sc->done = 1;
        return;
    }
    const double omega = ts / tt;
    const double rho_new = r0s - omega * r0t;
    const double r2 = fmax(0.0, sc->ss - omega * ts);
    sc->omega = omega;
    sc->iter += 1;
    sc->r2 = r2;
    sc->pending = 1;
    if (r2 <= sc->tol2 * sc->b2) {
        sc->done = 1;
    } else if (!(fabs(rho_new) > 1e-300) || !isfinite(rho_new)) {
        sc->breakdown = 1;
        sc->done = 1;
    } else {
        sc->beta = (rho_new / sc->rho) * (sc->alpha / omega);
        sc->rho = rho_new;
    }
}

// Per-problem sums of a batch: all 32 lanes of the warp call this (q < 0: no
// contribution).  A warp whose lanes belong to one problem adds one atomic per value.
template <int ND>
__device__ __forceinline__ void batch_add(const BatchView &bv, int q, double (&v)[ND]) {
    const unsigned full = 0xffffffffu;
    const int q0 = __shfl_sync(full, q, 0);
    if (__all_sync(full, q == q0 || q < 0)) {
#pragma unroll
        for (int p = 0; p < ND; ++p) {
            double a = v[p];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(full, a, o);
            if ((threadIdx.x & 31) == 0 && q0 >= 0) atomicAdd(bv.acc + p * bv.nprob + q0, a);
        }
    } else if (q >= 0) {
#pragma unroll
        for (int p = 0; p < ND; ++p) atomicAdd(bv.acc + p * bv.nprob + q, v[p]);
    }
}

// In the last block of a batch reduction: for every problem whose iteration is still
// running, f(q, sums) updates its scalars; the sums are reset to zero, and alldone is
// set once no problem is running.  Called by all threads of the block.
template <int ND, typename Fn>
__device__ __forceinline__ void batch_finish(const BatchView &bv, KScal *sc, Fn f) {
    int open = 0;
    for (int q = threadIdx.x; q < bv.nprob; q += blockDim.x) {
        double sum[ND];
#pragma unroll
        for (int p = 0; p < ND; ++p) {
            sum[p] = __ldcg(bv.acc + p * bv.nprob + q);
            bv.acc[p * bv.nprob + q] = 0.0;
        }
        if (!sc[q].done) f(q, sum);
        open |= !sc[q].done;
    }
    const int any = __syncthreads_or(open);
    if (threadIdx.x == 0) *bv.alldone = any ? 0 : 1;
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

// s = r - alpha v; sh = P^{-1} s; (s, s) -> last block: converged on s?
template <typename T, int N>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_s(int K, const T *__restrict__ r, T *__restrict__ s,
                                                        const T *__restrict__ v, T *__restrict__ sh,
                                                        const __nv_bfloat16 *__restrict__ P,
                                                        const T *__restrict__ inv, double *part, KScal *sc,
                                                        unsigned int *counter) {
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    Acc<T> acc[1] = {Acc<T>(0)};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        T q[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int i = j * K + k;
            const T qi = r[i] - alpha * v[i];
            s[i] = qi;
            q[j] = qi;
            acc[0] += (Acc<T>)qi * (Acc<T>)qi;
        }
        if (P) {
            T y[N];
            block_matvec<T, N>(P, K, k, q, y);
#pragma unroll
            for (int i = 0; i < N; ++i) sh[i * K + k] = y[i];
        } else {
            const T iv = inv[k];
#pragma unroll
            for (int i = 0; i < N; ++i) sh[i * K + k] = q[i] * iv;
        }
    }
    block_partials<1>(acc, part);
    if (last_block(counter)) {
        const double s2 = sum_partials_cg(part, 0, gridDim.x);
        if (threadIdx.x == 0) {
            sc->ss = s2;
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

// Start of a BiCGStab iteration: the update owed from the previous iteration,
// x += alpha ph + omega sh and r = s - omega t (none in the first iteration of a
// solve), then p = r + beta (p - omega v) and ph = P^{-1} p.
template <typename T, int N>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_next(int K, T *__restrict__ x, T *ph,
                                                           const T *__restrict__ sh, const T *__restrict__ s,
                                                           const T *__restrict__ t, T *__restrict__ r,
                                                           T *__restrict__ pv, const T *__restrict__ v,
                                                           const __nv_bfloat16 *__restrict__ P,
                                                           const T *__restrict__ inv, const KScal *sc) {
    if (sc->done) return;
    const bool first = sc->first != 0;
    const T alpha = (T)sc->alpha, omega = (T)sc->omega, beta = (T)sc->beta;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        T q[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int i = j * K + k;
            T ri;
            if (first) {
                ri = r[i];
            } else {
                x[i] += alpha * ph[i] + omega * sh[i];
                ri = s[i] - omega * t[i];
                r[i] = ri;
            }
            q[j] = ri + beta * (pv[i] - omega * v[i]);
            pv[i] = q[j];
        }
        if (P) {
            T y[N];
            block_matvec<T, N>(P, K, k, q, y);
#pragma unroll
            for (int i = 0; i < N; ++i) ph[i * K + k] = y[i];
        } else {
            const T iv = inv[k];
#pragma unroll
            for (int i = 0; i < N; ++i) ph[i * K + k] = q[i] * iv;
        }
    }
}

// The reductions of FUSED_EPI_ALPHA / FUSED_EPI_OMEGA as a pass of their own over
// y = v or t (used where the apply has no fused epilogue).
template <typename T, int EPI>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_epi(int64_t n, const T *__restrict__ y,
                                                          const T *__restrict__ e1, const T *__restrict__ e2,
                                                          double *part, KScal *sc, unsigned int *counter) {
    if (sc->done) return;
    constexpr int ND = EPI == 2 ? 4 : 1;
    Acc<T> dots[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) dots[q] = Acc<T>(0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Acc<T> yi = (Acc<T>)y[i];
        if constexpr (EPI == 1) {
            dots[0] += (Acc<T>)e1[i] * yi;
        } else {
            const Acc<T> si = (Acc<T>)e1[i], ri = (Acc<T>)e2[i];
            dots[0] += yi * si;
            dots[1] += yi * yi;
            dots[2] += ri * si;
            dots[3] += ri * yi;
        }
    }
    block_partials_any<ND>(dots, part);
    if (last_block(counter)) {
        double sum[ND];
#pragma unroll
        for (int q = 0; q < ND; ++q) sum[q] = sum_partials_cg(part, q, gridDim.x);
        if (threadIdx.x == 0) {
            if constexpr (EPI == 1)
                bicg_alpha_scalars(sum[0], sc);
            else
                bicg_omega_scalars(sum[0], sum[1], sum[2], sum[3], sc);
            *counter = 0;
        }
    }
}

// After the last iteration of a solve: the owed x += alpha ph + omega sh.
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_finish(int64_t n, T *__restrict__ x, const T *__restrict__ ph,
                                                             const T *__restrict__ sh, const KScal *sc) {
    const T alpha = (T)sc->alpha, omega = (T)sc->omega;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += alpha * ph[i] + omega * sh[i];
}

// ---------------------------------------------------------------------------
// BiCGStab on the union of a batch: the kernels above with per-problem scalars.
// ---------------------------------------------------------------------------

// k_bicg_next for a batch; the elements of problems whose iteration is done are left alone
template <typename T, int N>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_next_b(int K, T *__restrict__ x, T *ph,
                                                             const T *__restrict__ sh, const T *__restrict__ s,
                                                             const T *__restrict__ t, T *__restrict__ r,
                                                             T *__restrict__ pv, const T *__restrict__ v,
                                                             const __nv_bfloat16 *__restrict__ P,
                                                             const T *__restrict__ inv, const KScal *sc,
                                                             BatchView bv) {
    if (*bv.alldone) return;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        const KScal &q = sc[bv.eprob[k]];
        if (q.done) continue;
        const bool first = q.first != 0;
        const T alpha = (T)q.alpha, omega = (T)q.omega, beta = (T)q.beta;
        T z[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int i = j * K + k;
            T ri;
            if (first) {
                ri = r[i];
            } else {
                x[i] += alpha * ph[i] + omega * sh[i];
                ri = s[i] - omega * t[i];
                r[i] = ri;
            }
            z[j] = ri + beta * (pv[i] - omega * v[i]);
            pv[i] = z[j];
        }
        if (P) {
            T y[N];
            block_matvec<T, N>(P, K, k, z, y);
#pragma unroll
            for (int i = 0; i < N; ++i) ph[i * K + k] = y[i];
        } else {
            const T iv = inv[k];
#pragma unroll
            for (int i = 0; i < N; ++i) ph[i * K + k] = z[i] * iv;
        }
    }
}

// k_bicg_s for a batch: s = r - alpha_q v; sh = P^{-1} s; (s, s) per problem
template <typename T, int N>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_s_b(int K, const T *__restrict__ r, T *__restrict__ s,
                                                          const T *__restrict__ v, T *__restrict__ sh,
                                                          const __nv_bfloat16 *__restrict__ P,
                                                          const T *__restrict__ inv, KScal *sc, BatchView bv,
                                                          unsigned int *counter) {
    if (*bv.alldone) return;
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < K; base += stride) {
        const int k = base + threadIdx.x;
        int q = -1;
        double acc[1] = {0.0};
        if (k < K && !sc[bv.eprob[k]].done) {
            q = bv.eprob[k];
            const T alpha = (T)sc[q].alpha;
            T z[N];
            Acc<T> a = Acc<T>(0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const int i = j * K + k;
                z[j] = r[i] - alpha * v[i];
                s[i] = z[j];
                a += (Acc<T>)z[j] * (Acc<T>)z[j];
            }
            acc[0] = (double)a;
            if (P) {
                T y[N];
                block_matvec<T, N>(P, K, k, z, y);
#pragma unroll
                for (int i = 0; i < N; ++i) sh[i * K + k] = y[i];
            } else {
                const T iv = inv[k];
#pragma unroll
                for (int i = 0; i < N; ++i) sh[i * K + k] = z[i] * iv;
            }
        }
        batch_add<1>(bv, q, acc);
    }
    if (last_block(counter)) {
        batch_finish<1>(bv, sc, [&](int q, const double *sum) {
            KScal &e = sc[q];
            e.ss = sum[0];
            if (sum[0] <= e.tol2 * e.b2) {
                e.sconv = 1;
                e.r2 = sum[0];
                e.iter += 1;
                e.done = 1;
            }
        });
        if (threadIdx.x == 0) *counter = 0;
    }
}

// After the iterations of a batch: each problem's owed update (x += alpha ph once it
// converged on s, else x += alpha ph + omega sh when pending)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_finish_b(int K, int N, T *__restrict__ x,
                                                               const T *__restrict__ ph, const T *__restrict__ sh,
                                                               const KScal *sc, BatchView bv) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        const KScal &q = sc[bv.eprob[k]];
        const T alpha = (T)q.alpha, omega = (T)q.omega;
        if (q.sconv) {
            for (int j = 0; j < N; ++j) x[j * K + k] += alpha * ph[j * K + k];
        } else if (q.pending) {
            for (int j = 0; j < N; ++j) x[j * K + k] += alpha * ph[j * K + k] + omega * sh[j * K + k];
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
