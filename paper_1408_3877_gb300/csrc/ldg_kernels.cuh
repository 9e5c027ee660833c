// Matrix-free LDG operator kernels (one thread per triangle, grid-stride).
//
// Vectors are stored N x K ("coefficient j of all triangles is contiguous"), so a
// warp reading coefficient j of 32 consecutive triangles issues one coalesced
// transaction.  Geometry is 4 x K (B11, B12, B21, B22) and the neighbour relation
// 3 x K codes: (k+ << 2) | n+ for an interior edge, -1 Dirichlet, -2 Neumann.
//
// Boundary samples (c_D, g_N) arrive in the caller's triangle order; perm maps the
// internal index to it.
//
// Reference tables (basis values and weighted gradients at the quadrature points)
// are staged once per block in shared memory; every table read is warp-uniform
// except the neighbour's edge trace, whose local edge n+ varies per thread.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

#include <type_traits>

#include "internal.h"
#include "krylov.cuh"

namespace festung {

constexpr int NBR_DIRICHLET = -1;
constexpr int NBR_NEUMANN = -2;

template <typename T, int N, int R2, int R1>
struct SmemTab {
    T phiQ[R2 * N];
    T gw1[R2 * N];
    T gw2[R2 * N];
    T H1[N * N];
    T H2[N * N];
    T phiE[3 * R1 * N];
    T wphiE[3 * R1 * N];
};

// Layout of the device table buffer (see table_offsets in festung.cu):
// phiQ | wphiQ | gw1 | gw2 | H1 | H2 | phiE | wphiE
template <typename T, int N, int R2, int R1>
__device__ __forceinline__ void load_tables(SmemTab<T, N, R2, R1> &s, const T *__restrict__ g) {
    const int o_phiQ = 0, o_gw1 = 2 * R2 * N, o_gw2 = 3 * R2 * N, o_H1 = 4 * R2 * N,
              o_H2 = o_H1 + N * N, o_phiE = o_H2 + N * N, o_wphiE = o_phiE + 3 * R1 * N;
    for (int i = threadIdx.x; i < R2 * N; i += blockDim.x) {
        s.phiQ[i] = g[o_phiQ + i];
        s.gw1[i] = g[o_gw1 + i];
        s.gw2[i] = g[o_gw2 + i];
    }
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
        s.H1[i] = g[o_H1 + i];
        s.H2[i] = g[o_H2 + i];
    }
    for (int i = threadIdx.x; i < 3 * R1 * N; i += blockDim.x) {
        s.phiE[i] = g[o_phiE + i];
        s.wphiE[i] = g[o_wphiE + i];
    }
}

// nu_kn |E_kn| (exterior normal times edge length) of local edge n from B_k:
// edge 0: a3 - a2 = B(:,2) - B(:,1); edge 1: a1 - a3 = -B(:,2); edge 2: a2 - a1 = B(:,1);
// the exterior normal of a counter-clockwise edge vector (ex, ey) is (ey, -ex).
template <typename T>
__device__ __forceinline__ void edge_normal(int n, T b11, T b12, T b21, T b22, T &nx, T &ny) {
    T ex, ey;
    if (n == 0) {
        ex = b12 - b11;
        ey = b22 - b21;
    } else if (n == 1) {
        ex = -b12;
        ey = -b22;
    } else {
        ex = b11;
        ey = b21;
    }
    nx = ey;
    ny = -ex;
}

// Trace of a coefficient vector on local edge n at the R1 Gauss points.
template <typename T, int N, int R1>
__device__ __forceinline__ void trace_own(const T *phiE, int n, const T (&c)[N], T (&out)[R1]) {
#pragma unroll
    for (int r = 0; r < R1; ++r) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) s += phiE[(n * R1 + r) * N + j] * c[j];
        out[r] = s;
    }
}

// Trace of the neighbour's field (global, N x K) on its edge n2, at the points that
// coincide with our Gauss points: every edge-to-edge map reverses the orientation
// (eq. mapEE), so our point r is the neighbour's point R1 - 1 - r.
// CG: load through L2 only (ld.global.cg), for vectors that other blocks of a persistent
// kernel write between phases; otherwise the ordinary (possibly read-only cached) load.
template <bool CG, typename T>
__device__ __forceinline__ T ldv(const T *p) {
    if constexpr (CG)
        return __ldcg(p);
    else
        return *p;
}

template <typename T, int N, int R1, bool CG = false>
__device__ __forceinline__ void trace_nbr(const T *phiE, const T *__restrict__ V, int64_t K, int64_t k2,
                                          int n2, T (&out)[R1]) {
#pragma unroll
    for (int r = 0; r < R1; ++r) out[r] = T(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const T v = ldv<CG>(V + j * K + k2);
#pragma unroll
        for (int r = 0; r < R1; ++r) out[r] += phiE[(n2 * R1 + (R1 - 1 - r)) * N + j] * v;
    }
}

// ---------------------------------------------------------------------------
// Pass 1: Z^m = -M^{-1} (B_m x),  B_m = -H^m + Q^m + Q_N^m  (block rows 1-2 of
// eq. timeDepSystem; H^m Sec. 3.6.2, Q^m eq. globQ, Q_N^m eq. globQm:N).
// ---------------------------------------------------------------------------
template <typename T, int N, int R2, int R1>
__global__ void __launch_bounds__(256) k_flux(const T *__restrict__ X, T *__restrict__ Z1,
                                              T *__restrict__ Z2, const T *__restrict__ Bg,
                                              const int32_t *__restrict__ nbr, int64_t K,
                                              const T *__restrict__ tabg, const int *__restrict__ skip) {
    __shared__ SmemTab<T, N, R2, R1> s;
    if (skip && *skip) return;
    load_tables(s, tabg);
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        T x[N];
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] = X[j * K + k];
        const T b11 = Bg[k], b12 = Bg[K + k], b21 = Bg[2 * K + k], b22 = Bg[3 * K + k];
        T a1[N], a2[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            T h1 = T(0), h2 = T(0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                h1 += s.H1[i * N + j] * x[j];
                h2 += s.H2[i * N + j] * x[j];
            }
            // H^1 = B22 H^_1 - B21 H^_2, H^2 = -B12 H^_1 + B11 H^_2 (Sec. 3.6.2)
            a1[i] = -(b22 * h1 - b21 * h2);
            a2[i] = -(b11 * h2 - b12 * h1);
        }
#pragma unroll 1
        for (int n = 0; n < 3; ++n) {
            const int code = nbr[n * K + k];
            if (code == NBR_DIRICHLET) continue;  // c_D enters the right-hand side only
            T nx, ny;
            edge_normal(n, b11, b12, b21, b22, nx, ny);
            T f[R1];
            trace_own<T, N, R1>(s.phiE, n, x, f);
            if (code >= 0) {
                T cp[R1];
                trace_nbr<T, N, R1>(s.phiE, X, K, code >> 2, code & 3, cp);
#pragma unroll
                for (int r = 0; r < R1; ++r) f[r] = T(0.5) * (f[r] + cp[r]);
            }
#pragma unroll
            for (int i = 0; i < N; ++i) {
                T t = T(0);
#pragma unroll
                for (int r = 0; r < R1; ++r) t += s.wphiE[(n * R1 + r) * N + i] * f[r];
                a1[i] += nx * t;
                a2[i] += ny * t;
            }
        }
        const T inv = T(1) / (b11 * b22 - b12 * b21);  // M^{-1} = 1 / (2|T_k|)
#pragma unroll
        for (int i = 0; i < N; ++i) {
            Z1[i * K + k] = -a1[i] * inv;
            Z2[i * K + k] = -a2[i] * inv;
        }
    }
}

// ---------------------------------------------------------------------------
// Pass 2.  MODE_APPLY:  y = mass M x + tau (eta (S + S_D) x + sum_m A_m Z^m)     (E1)
//          MODE_RHS:    y = mass M x + tau (M F + eta K_D - K_N + sum_m A_m Z^m) (E2)
// MODE_RHS leaves out the terms with Z and eta K_D: Z = M^{-1} J_D (the Dirichlet lift)
// vanishes except on the triangles next to a Dirichlet edge, so those terms only matter on
// the few triangles the lift reaches, and k_rhs_lift adds them there.
// (mass = 1 for a time step; mass = 0, tau = 1 for the stationary problem of Sec. 3.9)
// with A_m = -G^m + R^m + R_D^m (G^m Sec. 3.6.3, R^m eq. globR, R_D^m eq. globR:D,
// S eq. globS, S_D eq. globS:D, K_D eq. globK:D, K_N Sec. 3.6.12).  Volume terms use
// the triangle rule, edge terms the Gauss rule, as the reference integrals do.
// ---------------------------------------------------------------------------
constexpr int MODE_APPLY = 0;
constexpr int MODE_RHS = 1;

template <typename T, int N, int R2, int R1, int MODE>
__global__ void __launch_bounds__(256) k_apply(const T *__restrict__ X, const T *__restrict__ Z1,
                                               const T *__restrict__ Z2, const T *__restrict__ Dc,
                                               T *__restrict__ Y, const T *__restrict__ Bg,
                                               const int32_t *__restrict__ nbr, int64_t K, T tau, T eta, T mass,
                                               const T *__restrict__ tabg, const T *__restrict__ F,
                                               const T *__restrict__ cD, const T *__restrict__ gN,
                                               const int32_t *__restrict__ perm, const int *__restrict__ skip) {
    __shared__ SmemTab<T, N, R2, R1> s;
    if (skip && *skip) return;
    load_tables(s, tabg);
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        T x[N], z1[N], z2[N], d[N], acc[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            x[j] = X[j * K + k];
            z1[j] = Z1[j * K + k];
            z2[j] = Z2[j * K + k];
            d[j] = Dc[j * K + k];
            acc[j] = T(0);
        }
        const T b11 = Bg[k], b12 = Bg[K + k], b21 = Bg[2 * K + k], b22 = Bg[3 * K + k];
        // right-hand side: the terms with Z come from k_rhs_lift (see above)
        const bool aterms = MODE == MODE_APPLY;
        // volume term -sum_m G^m Z^m
#pragma unroll 1
        for (int r = 0; r < (aterms ? R2 : 0); ++r) {
            T dv = T(0), w1 = T(0), w2 = T(0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const T ph = s.phiQ[r * N + j];
                dv += ph * d[j];
                w1 += ph * z1[j];
                w2 += ph * z2[j];
            }
            const T u = dv * (b22 * w1 - b12 * w2);
            const T v = dv * (b11 * w2 - b21 * w1);
#pragma unroll
            for (int i = 0; i < N; ++i) acc[i] -= s.gw1[r * N + i] * u + s.gw2[r * N + i] * v;
        }
        // edge terms
#pragma unroll 1
        for (int n = 0; n < 3; ++n) {
            const int code = nbr[n * K + k];
            if (MODE == MODE_APPLY && code == NBR_NEUMANN) continue;
            if (!aterms && code != NBR_NEUMANN) continue;
            T nx, ny;
            edge_normal(n, b11, b12, b21, b22, nx, ny);
            T dm[R1], g[R1];
            trace_own<T, N, R1>(s.phiE, n, d, dm);
            if (code == NBR_NEUMANN) {
                // -K_N: -|E| sum_r w_r phi_i d^- g_N
                const T len = sqrt(nx * nx + ny * ny);
#pragma unroll
                for (int r = 0; r < R1; ++r) g[r] = -len * dm[r] * gN[((int64_t)perm[k] * 3 + n) * R1 + r];
            } else {
                T zm1[R1], zm2[R1];
                trace_own<T, N, R1>(s.phiE, n, z1, zm1);
                trace_own<T, N, R1>(s.phiE, n, z2, zm2);
                if (code >= 0) {
                    const int64_t k2 = code >> 2;
                    const int n2 = code & 3;
                    T dp[R1], zp1[R1], zp2[R1];
                    trace_nbr<T, N, R1>(s.phiE, Dc, K, k2, n2, dp);
                    trace_nbr<T, N, R1>(s.phiE, Z1, K, k2, n2, zp1);
                    trace_nbr<T, N, R1>(s.phiE, Z2, K, k2, n2, zp2);
#pragma unroll
                    for (int r = 0; r < R1; ++r)
                        g[r] = T(0.5) * (nx * (dm[r] * zm1[r] + dp[r] * zp1[r]) +
                                         ny * (dm[r] * zm2[r] + dp[r] * zp2[r]));
                    if (MODE == MODE_APPLY) {
                        T cm[R1], cp[R1];
                        trace_own<T, N, R1>(s.phiE, n, x, cm);
                        trace_nbr<T, N, R1>(s.phiE, X, K, k2, n2, cp);
#pragma unroll
                        for (int r = 0; r < R1; ++r) g[r] += eta * (cm[r] - cp[r]);
                    }
                } else {  // Dirichlet
#pragma unroll
                    for (int r = 0; r < R1; ++r) g[r] = dm[r] * (nx * zm1[r] + ny * zm2[r]);
                    if (MODE == MODE_APPLY) {
                        T cm[R1];
                        trace_own<T, N, R1>(s.phiE, n, x, cm);
#pragma unroll
                        for (int r = 0; r < R1; ++r) g[r] += eta * cm[r];
                    } else {
#pragma unroll
                        for (int r = 0; r < R1; ++r) g[r] += eta * cD[((int64_t)perm[k] * 3 + n) * R1 + r];
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < N; ++i) {
                T t = T(0);
#pragma unroll
                for (int r = 0; r < R1; ++r) t += s.wphiE[(n * R1 + r) * N + i] * g[r];
                acc[i] += t;
            }
        }
        const T det = b11 * b22 - b12 * b21;  // M = 2|T_k| I (Sec. 3.6.1)
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (MODE == MODE_RHS && F) acc[i] += det * F[i * K + k];
            Y[i * K + k] = mass * det * x[i] + tau * acc[i];
        }
    }
}

// The terms of the right-hand side that involve the Dirichlet lift Z = M^{-1} J_D^m:
// y += tau (sum_m A_m Z^m + eta K_D) on the triangles in `list` (the ones the lift
// reaches), after k_apply<MODE_RHS> wrote y without them.  One warp per triangle: its
// lanes take the R2 points of the volume term, then the R1 points of each edge, then the
// N test functions, so that the FP64 quadrature of a triangle runs 32 lanes wide (this
// device's FP64 pipe is narrow; a thread per triangle left the few listed triangles on a
// few SMs for 0.29 ms at p = 4).
constexpr int LIFT_WARPS = 4;  // triangles per block

template <int N, int R2, int R1>
__global__ void __launch_bounds__(32 * LIFT_WARPS)
    k_rhs_lift(const double *__restrict__ Z1, const double *__restrict__ Z2, const double *__restrict__ Dc,
               double *__restrict__ Y, const double *__restrict__ Bg, const int32_t *__restrict__ nbr, int64_t K,
               double tau, double eta, const double *__restrict__ tabg, const double *__restrict__ cD,
               const int32_t *__restrict__ perm, const int32_t *__restrict__ list, int64_t nlist) {
    static_assert(R2 <= 32 && N <= 32 && R1 <= 32, "one lane per point and per test function");
    __shared__ SmemTab<double, N, R2, R1> s;
    __shared__ double own[LIFT_WARPS][3][N], nb[LIFT_WARPS][3][N];  // d, z1, z2 of the triangle / a neighbour
    __shared__ double pt[LIFT_WARPS][2][32];                         // values at the points
    load_tables(s, tabg);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t it = (int64_t)blockIdx.x * LIFT_WARPS + w; it < nlist; it += (int64_t)gridDim.x * LIFT_WARPS) {
        const int64_t k = list[it];
        if (lane < N) {
            own[w][0][lane] = Dc[lane * K + k];
            own[w][1][lane] = Z1[lane * K + k];
            own[w][2][lane] = Z2[lane * K + k];
        }
        const double b11 = Bg[k], b12 = Bg[K + k], b21 = Bg[2 * K + k], b22 = Bg[3 * K + k];
        __syncwarp();
        // volume term -sum_m G^m Z^m: d_h, Z^1, Z^2 at point r = lane
        if (lane < R2) {
            double dv = 0.0, w1 = 0.0, w2 = 0.0;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const double ph = s.phiQ[lane * N + j];
                dv += ph * own[w][0][j];
                w1 += ph * own[w][1][j];
                w2 += ph * own[w][2][j];
            }
            pt[w][0][lane] = dv * (b22 * w1 - b12 * w2);
            pt[w][1][lane] = dv * (b11 * w2 - b21 * w1);
        }
        __syncwarp();
        double acc = 0.0;  // lane i < N: test function i
        if (lane < N) {
#pragma unroll 5
            for (int r = 0; r < R2; ++r) acc -= s.gw1[r * N + lane] * pt[w][0][r] + s.gw2[r * N + lane] * pt[w][1][r];
        }
        __syncwarp();
        // edge terms R^m, R_D^m with Z, and eta K_D: the flux at point r = lane
        for (int n = 0; n < 3; ++n) {
            const int code = nbr[n * K + k];
            if (code == NBR_NEUMANN) continue;
            double nx, ny;
            edge_normal(n, b11, b12, b21, b22, nx, ny);
            if (code >= 0 && lane < N) {
                const int64_t k2 = code >> 2;
                nb[w][0][lane] = Dc[lane * K + k2];
                nb[w][1][lane] = Z1[lane * K + k2];
                nb[w][2][lane] = Z2[lane * K + k2];
            }
            __syncwarp();
            if (lane < R1) {
                double dm = 0.0, zm1 = 0.0, zm2 = 0.0;
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const double ph = s.phiE[(n * R1 + lane) * N + j];
                    dm += ph * own[w][0][j];
                    zm1 += ph * own[w][1][j];
                    zm2 += ph * own[w][2][j];
                }
                double g;
                if (code >= 0) {
                    const int n2 = code & 3, rp = R1 - 1 - lane;  // the neighbour's point (eq. mapEE)
                    double dp = 0.0, zp1 = 0.0, zp2 = 0.0;
#pragma unroll
                    for (int j = 0; j < N; ++j) {
                        const double ph = s.phiE[(n2 * R1 + rp) * N + j];
                        dp += ph * nb[w][0][j];
                        zp1 += ph * nb[w][1][j];
                        zp2 += ph * nb[w][2][j];
                    }
                    g = 0.5 * (nx * (dm * zm1 + dp * zp1) + ny * (dm * zm2 + dp * zp2));
                } else {  // Dirichlet
                    g = dm * (nx * zm1 + ny * zm2) + eta * cD[((int64_t)perm[k] * 3 + n) * R1 + lane];
                }
                pt[w][0][lane] = g;
            }
            __syncwarp();
            if (lane < N) {
#pragma unroll
                for (int r = 0; r < R1; ++r) acc += s.wphiE[(n * R1 + r) * N + lane] * pt[w][0][r];
            }
            __syncwarp();
        }
        if (lane < N) Y[lane * K + k] += tau * acc;
        __syncwarp();
    }
}

// W^m = M^{-1} J_D^m (Sec. 3.6.10): Dirichlet data lifted into the flux equation.
template <typename T, int N, int R2, int R1>
__global__ void __launch_bounds__(256) k_dirichlet_lift(T *__restrict__ W1, T *__restrict__ W2,
                                                        const T *__restrict__ Bg,
                                                        const int32_t *__restrict__ nbr, int64_t K,
                                                        const T *__restrict__ tabg, const T *__restrict__ cD,
                                                        const int32_t *__restrict__ perm) {
    __shared__ SmemTab<T, N, R2, R1> s;
    load_tables(s, tabg);
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        const T b11 = Bg[k], b12 = Bg[K + k], b21 = Bg[2 * K + k], b22 = Bg[3 * K + k];
        T a1[N], a2[N];
#pragma unroll
        for (int i = 0; i < N; ++i) a1[i] = a2[i] = T(0);
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            if (nbr[n * K + k] != NBR_DIRICHLET) continue;
            T nx, ny;
            edge_normal(n, b11, b12, b21, b22, nx, ny);
#pragma unroll
            for (int i = 0; i < N; ++i) {
                T t = T(0);
#pragma unroll
                for (int r = 0; r < R1; ++r)
                    t += s.wphiE[(n * R1 + r) * N + i] * cD[((int64_t)perm[k] * 3 + n) * R1 + r];
                a1[i] += nx * t;
                a2[i] += ny * t;
            }
        }
        const T inv = T(1) / (b11 * b22 - b12 * b21);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            W1[i * K + k] = a1[i] * inv;
            W2[i * K + k] = a2[i] * inv;
        }
    }
}

}  // namespace festung

namespace festung {

// ---------------------------------------------------------------------------
// Diagonal blocks of the step operator, S_kk = M_k + tau (eta S_t,kk - sum_m sum_k'
// A_m,kk' M_k'^{-1} B_m,k'k), one column per unit coefficient vector e_j of triangle
// k.  A unit vector on k alone produces flux unknowns on k (through B_m,kk) and on
// each interior neighbour k' (through the central flux of eq. globQ:offdiag); S_kk e_j
// collects their contributions back on k.  Written to P[(i N + j) K + k] in FP32.
// ---------------------------------------------------------------------------
template <typename T, int N, int R2, int R1>
__global__ void __launch_bounds__(128) k_blockdiag(float *__restrict__ P, const T *__restrict__ Bg,
                                                   const int32_t *__restrict__ nbr, const T *__restrict__ Dc,
                                                   int64_t K, T tau, T eta, T mass, const T *__restrict__ tabg) {
    __shared__ SmemTab<T, N, R2, R1> s;
    load_tables(s, tabg);
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        const T b11 = Bg[k], b12 = Bg[K + k], b21 = Bg[2 * K + k], b22 = Bg[3 * K + k];
        const T det = b11 * b22 - b12 * b21;
        T d[N];
#pragma unroll
        for (int l = 0; l < N; ++l) d[l] = Dc[l * K + k];
        int code[3];
        T nx[3], ny[3], inv2[3];
        T dm[3][R1], dp[3][R1];
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            code[n] = nbr[n * K + k];
            edge_normal(n, b11, b12, b21, b22, nx[n], ny[n]);
            trace_own<T, N, R1>(s.phiE, n, d, dm[n]);
            inv2[n] = T(0);
#pragma unroll
            for (int r = 0; r < R1; ++r) dp[n][r] = T(0);
            if (code[n] >= 0) {
                const int64_t k2 = code[n] >> 2;
                trace_nbr<T, N, R1>(s.phiE, Dc, K, k2, code[n] & 3, dp[n]);
                inv2[n] = T(1) / (Bg[k2] * Bg[3 * K + k2] - Bg[K + k2] * Bg[2 * K + k2]);
            }
        }
        T dq[R2];
#pragma unroll 1
        for (int r = 0; r < R2; ++r) {
            T v = T(0);
#pragma unroll
            for (int l = 0; l < N; ++l) v += s.phiQ[r * N + l] * d[l];
            dq[r] = v;
        }
#pragma unroll 1
        for (int j = 0; j < N; ++j) {
            // Z_k = -M_k^{-1} B_m,kk e_j
            T z1[N], z2[N];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const T h1 = s.H1[i * N + j], h2 = s.H2[i * N + j];
                z1[i] = -(b22 * h1 - b21 * h2);
                z2[i] = -(b11 * h2 - b12 * h1);
            }
#pragma unroll
            for (int n = 0; n < 3; ++n) {
                if (code[n] == NBR_DIRICHLET) continue;
                const T fac = code[n] >= 0 ? T(0.5) : T(1);
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    T t = T(0);
#pragma unroll
                    for (int r = 0; r < R1; ++r) t += s.wphiE[(n * R1 + r) * N + i] * s.phiE[(n * R1 + r) * N + j];
                    z1[i] += fac * nx[n] * t;
                    z2[i] += fac * ny[n] * t;
                }
            }
            const T idet = T(1) / det;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                z1[i] *= -idet;
                z2[i] *= -idet;
            }
            T acc[N];
#pragma unroll
            for (int i = 0; i < N; ++i) acc[i] = T(0);
            // volume term -sum_m G^m Z^m
#pragma unroll 1
            for (int r = 0; r < R2; ++r) {
                T w1 = T(0), w2 = T(0);
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    w1 += s.phiQ[r * N + i] * z1[i];
                    w2 += s.phiQ[r * N + i] * z2[i];
                }
                const T u = dq[r] * (b22 * w1 - b12 * w2);
                const T v = dq[r] * (b11 * w2 - b21 * w1);
#pragma unroll
                for (int i = 0; i < N; ++i) acc[i] -= s.gw1[r * N + i] * u + s.gw2[r * N + i] * v;
            }
#pragma unroll 1
            for (int n = 0; n < 3; ++n) {
                if (code[n] == NBR_NEUMANN) continue;
                T zm1[R1], zm2[R1], g[R1];
                trace_own<T, N, R1>(s.phiE, n, z1, zm1);
                trace_own<T, N, R1>(s.phiE, n, z2, zm2);
                if (code[n] >= 0) {
                    const int n2 = code[n] & 3;
                    // neighbour's flux unknown from the trace of e_j: Z_k' = -M_k'^{-1} (1/2) nu_k'n' |E| S^(n', n) e_j,
                    // with nu_k'n' |E| = -nu_kn |E|
                    T q[N];
#pragma unroll
                    for (int i = 0; i < N; ++i) {
                        T t = T(0);
#pragma unroll
                        for (int r = 0; r < R1; ++r)
                            t += s.wphiE[(n2 * R1 + r) * N + i] * s.phiE[(n * R1 + (R1 - 1 - r)) * N + j];
                        q[i] = t;
                    }
                    T qt[R1];
#pragma unroll
                    for (int r = 0; r < R1; ++r) {
                        T t = T(0);
#pragma unroll
                        for (int i = 0; i < N; ++i) t += s.phiE[(n2 * R1 + (R1 - 1 - r)) * N + i] * q[i];
                        qt[r] = t;
                    }
                    const T c2 = T(0.5) * inv2[n];  // -M^{-1} * 1/2 * (-nu |E|) = +1/2 nu |E| / det'
#pragma unroll
                    for (int r = 0; r < R1; ++r) {
                        const T zp1 = c2 * nx[n] * qt[r], zp2 = c2 * ny[n] * qt[r];
                        const T cm = s.phiE[(n * R1 + r) * N + j];
                        g[r] = T(0.5) * (nx[n] * (dm[n][r] * zm1[r] + dp[n][r] * zp1) +
                                         ny[n] * (dm[n][r] * zm2[r] + dp[n][r] * zp2)) +
                               eta * cm;
                    }
                } else {  // Dirichlet
#pragma unroll
                    for (int r = 0; r < R1; ++r)
                        g[r] = dm[n][r] * (nx[n] * zm1[r] + ny[n] * zm2[r]) + eta * s.phiE[(n * R1 + r) * N + j];
                }
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    T t = T(0);
#pragma unroll
                    for (int r = 0; r < R1; ++r) t += s.wphiE[(n * R1 + r) * N + i] * g[r];
                    acc[i] += t;
                }
            }
#pragma unroll
            for (int i = 0; i < N; ++i)
                P[(int64_t)(i * N + j) * K + k] = (float)((i == j ? mass * det : T(0)) + tau * acc[i]);
        }
    }
}

// Inverse of every N x N block of P (layout [(i N + j) K + k]), one warp per block:
// lane l < 2N holds column l of the augmented matrix [A | I] in registers, and
// Gauss-Jordan elimination with partial pivoting runs in FP32 with the pivot column
// broadcast by warp shuffles (the preconditioner only steers convergence; its rounding
// does not enter the solution).  The inverse is stored in BF16 in Pinv as
// ceil(N^2 / 8) chunks of 16 bytes per triangle, chunk-major ([q][K]), so that a warp
// reads its 32 triangles' chunk q with one coalesced 512-byte access.  flags |= 1 if a
// block is singular.
template <int N>
__global__ void __launch_bounds__(128) k_blockinv(const float *__restrict__ P, __nv_bfloat16 *__restrict__ Pinv,
                                                  int64_t K, int *__restrict__ flags) {
    static_assert(2 * N <= 32, "one warp holds [A | I]");
    constexpr int NQ = (N * N + 7) / 8;
    __shared__ float stage[4][N * N + 1];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; k < K; k += nwarps) {
        float col[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (lane < N)
                col[i] = P[(int64_t)(i * N + lane) * K + k];
            else
                col[i] = (lane - N == i) ? 1.0f : 0.0f;
        }
        bool bad = false;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            // pivot row: largest |A[i][c]|, i >= c, found by lane c
            int prow = c;
            float best = fabsf(col[c]);
#pragma unroll
            for (int i = c + 1; i < N; ++i)
                if (fabsf(col[i]) > best) {
                    best = fabsf(col[i]);
                    prow = i;
                }
            prow = __shfl_sync(0xffffffffu, prow, c);
            best = __shfl_sync(0xffffffffu, best, c);
            if (!(best > 0.0f)) {
                bad = true;
                break;
            }
#pragma unroll
            for (int i = c + 1; i < N; ++i)
                if (i == prow) {
                    const float t = col[c];
                    col[c] = col[i];
                    col[i] = t;
                }
            const float ip = 1.0f / __shfl_sync(0xffffffffu, col[c], c);
            col[c] *= ip;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                if (i == c) continue;
                const float f = __shfl_sync(0xffffffffu, col[i], c);
                col[i] -= f * col[c];
            }
        }
        if (bad) {
            if (lane == 0) atomicOr(flags, 1);
            continue;
        }
        // lanes N..2N-1 hold the columns of the inverse; stage row-major, write chunks
        __syncwarp();
        if (lane >= N && lane < 2 * N) {
#pragma unroll
            for (int i = 0; i < N; ++i) stage[wib][i * N + (lane - N)] = col[i];
        }
        __syncwarp();
        if (lane < NQ) {
            __align__(16) __nv_bfloat16 v[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int e = 8 * lane + t;
                v[t] = __float2bfloat16(e < N * N ? stage[wib][e] : 0.0f);
            }
            reinterpret_cast<uint4 *>(Pinv)[(int64_t)lane * K + k] = *reinterpret_cast<const uint4 *>(v);
        }
        __syncwarp();
    }
}

}  // namespace festung
