// Single-pass operator apply y = S x (E1) over tiles of nearby triangles.
//
// Triangles are stored in Morton order of their centroids, so TE consecutive
// triangles form a compact patch ("tile").  One thread block handles one tile.  Phase A
// evaluates, for every triangle of the tile and of its halo (interior neighbours
// outside the tile), the flux unknowns Z^m = -M^{-1} B_m x (block rows 1-2 of eq.
// timeDepSystem) and the traces of x, d_h, z^1, z^2 on its three edges at the Gauss
// points; the traces go to shared memory.  Phase B adds, for every tile triangle, the
// volume term -sum_m G^m Z^m and the edge terms R^m, R_D^m, S, S_D, reading its
// neighbours' traces from shared memory.  The flux unknowns never leave the chip.
#pragma once

#include "ldg_kernels.cuh"

namespace festung {

// Reference tables of one (N, R2, R1) instantiation in the constant bank.  Every
// access below uses compile-time indices (all loops over table entries are unrolled),
// so each table entry is an immediate constant-bank operand of its multiply-add and
// occupies no register.  Only the neighbour's edge table, whose edge index varies from
// thread to thread, is read from shared memory.
template <typename T, int N, int R2, int R1>
struct CTab {
    T phiQ[R2 * N];
    T gw1[R2 * N];
    T gw2[R2 * N];
    T H1[N * N];
    T H2[N * N];
    T phiE[3 * R1 * N];
    T wphiE[3 * R1 * N];
};

template <typename T, int N, int R2, int R1>
__constant__ CTab<T, N, R2, R1> c_tab;

// own-edge trace with a compile-time edge index (constant-bank table)
template <typename T, int N, int R2, int R1, int n>
__device__ __forceinline__ void ctrace(const T (&c)[N], T (&out)[R1]) {
    const CTab<T, N, R2, R1> &t = c_tab<T, N, R2, R1>;
#pragma unroll
    for (int r = 0; r < R1; ++r) {
        T v = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) v += t.phiE[(n * R1 + r) * N + j] * c[j];
        out[r] = v;
    }
}

// Shared-memory trace of field f (0: x, 1: d_h, 2: z^1, 3: z^2) on edge n at point r.
template <int R1>
__device__ __forceinline__ int tr_index(int f, int n, int r, int slot, int NS) {
    return ((f * 3 + n) * R1 + r) * NS + slot;
}

// Phase A, edge n of triangle e: traces of x and d_h to shared memory, and the edge's
// contribution nu_en |E_en| int phi_i {c} to B_m x (central flux, eq. globQ; interior
// value on Neumann edges, eq. globQm:N; nothing on Dirichlet edges).
template <typename T, int N, int R2, int R1, int n>
__device__ __forceinline__ void slot_edge(const T *phiE_s, const T *__restrict__ X, int64_t K, int code,
                                          const T (&x)[N], const T (&d)[N], T b11, T b12, T b21, T b22,
                                          T *tr, int NS, int slot, T (&a1)[N], T (&a2)[N]) {
    const CTab<T, N, R2, R1> &t = c_tab<T, N, R2, R1>;
    T xt[R1], dt[R1];
    ctrace<T, N, R2, R1, n>(x, xt);
    ctrace<T, N, R2, R1, n>(d, dt);
#pragma unroll
    for (int r = 0; r < R1; ++r) {
        tr[tr_index<R1>(0, n, r, slot, NS)] = xt[r];
        tr[tr_index<R1>(1, n, r, slot, NS)] = dt[r];
    }
    if (code == NBR_DIRICHLET) return;  // c_D enters the right-hand side only
    T nx, ny;
    edge_normal(n, b11, b12, b21, b22, nx, ny);
    if (code >= 0) {
        T cp[R1];
        trace_nbr<T, N, R1>(phiE_s, X, K, code >> 2, code & 3, cp);
#pragma unroll
        for (int r = 0; r < R1; ++r) xt[r] = T(0.5) * (xt[r] + cp[r]);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T v = T(0);
#pragma unroll
        for (int r = 0; r < R1; ++r) v += t.wphiE[(n * R1 + r) * N + i] * xt[r];
        a1[i] += nx * v;
        a2[i] += ny * v;
    }
}

template <typename T, int N, int R2, int R1, int n>
__device__ __forceinline__ void slot_ztrace(const T (&z1)[N], const T (&z2)[N], T *tr, int NS, int slot) {
    T t1[R1], t2[R1];
    ctrace<T, N, R2, R1, n>(z1, t1);
    ctrace<T, N, R2, R1, n>(z2, t2);
#pragma unroll
    for (int r = 0; r < R1; ++r) {
        tr[tr_index<R1>(2, n, r, slot, NS)] = t1[r];
        tr[tr_index<R1>(3, n, r, slot, NS)] = t2[r];
    }
}

// Phase A for triangle e stored at shared-memory slot `slot`: Z^m = -M^{-1} B_m x and
// the traces of x, d_h, z^1, z^2.  Returns Z^1, Z^2 and d_h of e in z1, z2, d.
template <typename T, int N, int R2, int R1>
__device__ __forceinline__ void slot_traces(const T *phiE_s, const T *__restrict__ X, const T *__restrict__ Dc,
                                            const T *__restrict__ Bg, const int32_t *__restrict__ nbr, int64_t K,
                                            int64_t e, T *tr, int NS, int slot, T (&z1)[N], T (&z2)[N],
                                            T (&d)[N]) {
    const CTab<T, N, R2, R1> &t = c_tab<T, N, R2, R1>;
    T x[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        x[j] = X[j * K + e];
        d[j] = Dc[j * K + e];
    }
    const T b11 = Bg[e], b12 = Bg[K + e], b21 = Bg[2 * K + e], b22 = Bg[3 * K + e];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T h1 = T(0), h2 = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            h1 += t.H1[i * N + j] * x[j];
            h2 += t.H2[i * N + j] * x[j];
        }
        // -H^m x with H^1 = B22 H^_1 - B21 H^_2, H^2 = -B12 H^_1 + B11 H^_2 (Sec. 3.6.2)
        z1[i] = -(b22 * h1 - b21 * h2);
        z2[i] = -(b11 * h2 - b12 * h1);
    }
    const int c0 = nbr[e], c1 = nbr[K + e], c2 = nbr[2 * K + e];
    slot_edge<T, N, R2, R1, 0>(phiE_s, X, K, c0, x, d, b11, b12, b21, b22, tr, NS, slot, z1, z2);
    slot_edge<T, N, R2, R1, 1>(phiE_s, X, K, c1, x, d, b11, b12, b21, b22, tr, NS, slot, z1, z2);
    slot_edge<T, N, R2, R1, 2>(phiE_s, X, K, c2, x, d, b11, b12, b21, b22, tr, NS, slot, z1, z2);
    const T inv = T(-1) / (b11 * b22 - b12 * b21);  // Z = -M^{-1} (B_m x), M = 2|T_e| I
#pragma unroll
    for (int i = 0; i < N; ++i) {
        z1[i] *= inv;
        z2[i] *= inv;
    }
    slot_ztrace<T, N, R2, R1, 0>(z1, z2, tr, NS, slot);
    slot_ztrace<T, N, R2, R1, 1>(z1, z2, tr, NS, slot);
    slot_ztrace<T, N, R2, R1, 2>(z1, z2, tr, NS, slot);
}

// Phase B, edge n of tile triangle i: R^m, R_D^m (eq. globR, globR:D) and the penalty
// S, S_D (eq. globS, globS:D) from the traces in shared memory.
template <typename T, int N, int R2, int R1, int n>
__device__ __forceinline__ void tile_edge(int code, int sl, const T *tr, int NS, int i, T b11, T b12, T b21, T b22,
                                          T eta, T (&acc)[N]) {
    if (code == NBR_NEUMANN) return;
    const CTab<T, N, R2, R1> &t = c_tab<T, N, R2, R1>;
    T nx, ny;
    edge_normal(n, b11, b12, b21, b22, nx, ny);
    T g[R1];
    if (code >= 0) {
        const int n2 = code & 3;
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            const int rp = R1 - 1 - r;  // the neighbour's Gauss point at our point r (eq. mapEE)
            const T xm = tr[tr_index<R1>(0, n, r, i, NS)], xp = tr[tr_index<R1>(0, n2, rp, sl, NS)];
            const T dm = tr[tr_index<R1>(1, n, r, i, NS)], dp = tr[tr_index<R1>(1, n2, rp, sl, NS)];
            const T am = tr[tr_index<R1>(2, n, r, i, NS)], ap = tr[tr_index<R1>(2, n2, rp, sl, NS)];
            const T bm = tr[tr_index<R1>(3, n, r, i, NS)], bp = tr[tr_index<R1>(3, n2, rp, sl, NS)];
            g[r] = T(0.5) * (nx * (dm * am + dp * ap) + ny * (dm * bm + dp * bp)) + eta * (xm - xp);
        }
    } else {  // Dirichlet
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            const T xm = tr[tr_index<R1>(0, n, r, i, NS)];
            const T dm = tr[tr_index<R1>(1, n, r, i, NS)];
            const T am = tr[tr_index<R1>(2, n, r, i, NS)];
            const T bm = tr[tr_index<R1>(3, n, r, i, NS)];
            g[r] = dm * (nx * am + ny * bm) + eta * xm;
        }
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
        T v = T(0);
#pragma unroll
        for (int r = 0; r < R1; ++r) v += t.wphiE[(n * R1 + r) * N + j] * g[r];
        acc[j] += v;
    }
}

template <typename T, int N, int R2, int R1>
__global__ void __launch_bounds__(256) k_apply_fused(const T *__restrict__ X, T *__restrict__ Y,
                                                     const T *__restrict__ Dc, const T *__restrict__ Bg,
                                                     const int32_t *__restrict__ nbr, const int16_t *__restrict__ slotg,
                                                     const int32_t *__restrict__ halo_ptr,
                                                     const int32_t *__restrict__ halo, int64_t K, int TE, int NS,
                                                     T tau, T eta, const T *__restrict__ tabg,
                                                     const int *__restrict__ skip) {
    __shared__ T phiE_s[3 * R1 * N];
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    T *tr = reinterpret_cast<T *>(dyn_smem);
    if (skip && *skip) return;
    {
        const int o_phiE = 4 * R2 * N + 2 * N * N;  // table layout of table_offsets()
        for (int j = threadIdx.x; j < 3 * R1 * N; j += blockDim.x) phiE_s[j] = tabg[o_phiE + j];
    }
    const int64_t start = (int64_t)blockIdx.x * TE;
    const int cnt = (int)((K - start) < TE ? (K - start) : TE);
    const int h0 = halo_ptr[blockIdx.x], nh = halo_ptr[blockIdx.x + 1] - h0;
    __syncthreads();
    for (int j = threadIdx.x; j < nh; j += blockDim.x) {
        T z1[N], z2[N], d[N];
        slot_traces<T, N, R2, R1>(phiE_s, X, Dc, Bg, nbr, K, halo[h0 + j], tr, NS, TE + j, z1, z2, d);
    }
    const int i = threadIdx.x;
    const bool own = i < cnt;
    const int64_t k = start + i;
    T z1[N], z2[N], d[N];
    if (own) slot_traces<T, N, R2, R1>(phiE_s, X, Dc, Bg, nbr, K, k, tr, NS, i, z1, z2, d);
    __syncthreads();
    if (!own) return;
    const CTab<T, N, R2, R1> &t = c_tab<T, N, R2, R1>;
    const T b11 = Bg[k], b12 = Bg[K + k], b21 = Bg[2 * K + k], b22 = Bg[3 * K + k];
    T acc[N];
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j] = T(0);
    // volume term -sum_m G^m Z^m at the triangle points (Sec. 3.6.3)
#pragma unroll
    for (int r = 0; r < R2; ++r) {
        T dv = T(0), w1 = T(0), w2 = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const T ph = t.phiQ[r * N + j];
            dv += ph * d[j];
            w1 += ph * z1[j];
            w2 += ph * z2[j];
        }
        const T u = dv * (b22 * w1 - b12 * w2);
        const T v = dv * (b11 * w2 - b21 * w1);
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] -= t.gw1[r * N + j] * u + t.gw2[r * N + j] * v;
    }
    const int c0 = nbr[k], c1 = nbr[K + k], c2 = nbr[2 * K + k];
    tile_edge<T, N, R2, R1, 0>(c0, c0 >= 0 ? slotg[k] : 0, tr, NS, i, b11, b12, b21, b22, eta, acc);
    tile_edge<T, N, R2, R1, 1>(c1, c1 >= 0 ? slotg[K + k] : 0, tr, NS, i, b11, b12, b21, b22, eta, acc);
    tile_edge<T, N, R2, R1, 2>(c2, c2 >= 0 ? slotg[2 * K + k] : 0, tr, NS, i, b11, b12, b21, b22, eta, acc);
    const T det = b11 * b22 - b12 * b21;
#pragma unroll
    for (int j = 0; j < N; ++j) Y[j * K + k] = det * X[j * K + k] + tau * acc[j];
}

}  // namespace festung
