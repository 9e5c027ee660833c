// Single-pass operator apply y = S x (E1) over tiles of nearby triangles.
//
// Triangles are stored in Morton order of their centroids, so TE consecutive
// triangles form a compact patch ("tile").  One thread block handles one tile and its
// halo (the interior neighbours outside the tile), one triangle ("slot") per thread:
//   A1  traces of x on the three edges of every slot -> shared memory;
//   A2  flux unknowns Z^m = -M^{-1} B_m x (block rows 1-2 of eq. timeDepSystem) from
//       the slot's own and its neighbours' x traces, held in contravariant form
//       zeta = det(B) B^{-1} Z, and the normal fluxes sigma = d_h zeta . nu^ on the
//       three edges -> shared memory;
//   B   for every tile triangle, the volume term -sum_m G^m Z^m and the edge terms
//       R^m, R_D^m, S, S_D from its own and its neighbours' traces.
// In contravariant form the volume and edge quadratures are those of the reference
// triangle: the geometry enters once per slot, through the metric B^T B / det B.
// The flux unknowns never leave the chip, and every trace is evaluated once per slot.
#pragma once

#include <vector>

#include "dfloat.cuh"
#include "dispatch.h"
#include "krylov_kernels.cuh"
#include "ldg_kernels.cuh"
#include "ldg_tc.cuh"

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

// One copy of the tables per translation unit (internal linkage): every unit that
// launches fused kernels fills its own copy with upload_ctab, which has internal
// linkage too, so the linker cannot merge the units' instantiations.
namespace {
template <typename T, int N, int R2, int R1>
__constant__ CTab<T, N, R2, R1> c_tab;

// Copy the reference tables of the context's (N, R2, R1) into this translation unit's
// constant bank, once per device.  The tables depend only on p and the quadrature, so
// every context of the same shape writes identical values.
template <typename T>
cudaError_t upload_ctab(const festung_ctx *c) {
    cudaError_t err = cudaSuccess;
    int dev = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        static unsigned long long done = 0;  // bit d: device d holds the tables
        const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
        if (done & bit) return;
        CTab<T, N, R2, R1> h;
        const HostTables &t = c->tab;
        for (int i = 0; i < R2 * N; ++i) {
            h.phiQ[i] = (T)t.phiQ[i];
            h.gw1[i] = (T)t.gw1[i];
            h.gw2[i] = (T)t.gw2[i];
        }
        for (int i = 0; i < N * N; ++i) {
            h.H1[i] = (T)t.H1[i];
            h.H2[i] = (T)t.H2[i];
        }
        for (int i = 0; i < 3 * R1 * N; ++i) {
            h.phiE[i] = (T)t.phiE[i];
            h.wphiE[i] = (T)t.wphiE[i];
        }
        err = cudaMemcpyToSymbol(c_tab<T, N, R2, R1>, &h, sizeof(h));
        if (err == cudaSuccess) done |= bit;
    });
    return err;
}
}  // namespace

// The FP32 tables as compile-time constants: GenTab<N, R2, R1, kind> is specialised in
// festung_tables_gen.h, which the build writes from build_tables() (kind 0: FP32 values,
// kind 1: rounded to BF16).  An initialised constant object lets the compiler fold every
// access with a compile-time index into an immediate operand; FP64 and double-float
// kernels read the constant-bank copy c_tab filled by upload_ctab.
template <int N, int R2, int R1, int TK>
struct GenTab;
}  // namespace festung

#include "festung_tables_gen.h"

namespace festung {

template <typename T, int N, int R2, int R1, int TK>
__device__ __forceinline__ const CTab<T, N, R2, R1> &tab_ref() {
    if constexpr (std::is_same<T, float>::value)
        return GenTab<N, R2, R1, TK>::get();
    else
        return c_tab<T, N, R2, R1>;
}

// own-edge trace with a compile-time edge index
template <typename T, int N, int R2, int R1, int TK, int n>
__device__ __forceinline__ void ctrace(const T (&c)[N], T (&out)[R1]) {
    const CTab<T, N, R2, R1> &t = tab_ref<T, N, R2, R1, TK>();
#pragma unroll
    for (int r = 0; r < R1; ++r) {
        T v = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) v += t.phiE[(n * R1 + r) * N + j] * c[j];
        out[r] = v;
    }
}

// Shared-memory traces of field f (0: x, 1: sigma) on edge n of slot s.
// When padding the R1 Gauss points to 16 bytes costs little, a trace is one padded
// vector moved with 128-bit accesses; otherwise (R1 = 5 in FP32) the points are stored
// one array per point, which keeps the shared memory of a block small enough for two
// blocks per SM.
template <typename T, int R1>
struct TraceLayout {
    static constexpr int per16 = 16 / sizeof(T);
    static constexpr int RPAD = ((R1 + per16 - 1) / per16) * per16;
    // vector layout when padding wastes at most a quarter, else one value per access
    static constexpr bool vec = 4 * (RPAD - R1) <= RPAD;
    static constexpr int RP = vec ? RPAD : R1;
    static constexpr int nvec = RPAD / per16;
};

// vector layout: a trace is RP consecutive values at ((f * 3 + n) * NS + slot) * RP;
// scalar layout: point r of the trace at (((f * 3 + n) * R1 + r) * NS + slot)
template <typename T, int R1>
__device__ __forceinline__ void tr_store(T *tr, int f, int n, int slot, int NS, const T (&v)[R1]) {
    using L = TraceLayout<T, R1>;
    if constexpr (L::vec) {
        alignas(16) T buf[L::RP];
#pragma unroll
        for (int r = 0; r < L::RP; ++r) buf[r] = r < R1 ? v[r] : T(0);
        float4 *dst = reinterpret_cast<float4 *>(tr + ((size_t)(f * 3 + n) * NS + slot) * L::RP);
#pragma unroll
        for (int q = 0; q < L::nvec; ++q) dst[q] = reinterpret_cast<const float4 *>(buf)[q];
    } else {
#pragma unroll
        for (int r = 0; r < R1; ++r) tr[((size_t)(f * 3 + n) * R1 + r) * NS + slot] = v[r];
    }
}

template <typename T, int R1>
__device__ __forceinline__ void tr_load(const T *tr, int f, int n, int slot, int NS, T (&v)[R1]) {
    using L = TraceLayout<T, R1>;
    if constexpr (L::vec) {
        alignas(16) T buf[L::RP];
        const float4 *src = reinterpret_cast<const float4 *>(tr + ((size_t)(f * 3 + n) * NS + slot) * L::RP);
#pragma unroll
        for (int q = 0; q < L::nvec; ++q) reinterpret_cast<float4 *>(buf)[q] = src[q];
#pragma unroll
        for (int r = 0; r < R1; ++r) v[r] = buf[r];
    } else {
#pragma unroll
        for (int r = 0; r < R1; ++r) v[r] = tr[((size_t)(f * 3 + n) * R1 + r) * NS + slot];
    }
}

// Double-float arithmetic is 10-20 instructions per multiply-add: fully unrolled, its
// point loops would not fit the instruction cache.  For that type the loops over
// quadrature points stay rolled and traces are moved point by point.
template <typename T>
constexpr bool kCompactCode = std::is_same<T, dfloat>::value;

// The basis is hierarchical: functions 0 | 1-2 | 3-5 | 6-9 | 10-14 have degrees 0..4.
// d phi_i / dx^_m has degree deg(i) - 1, so it is orthogonal to every phi_j of degree
// >= deg(i): H^_m[i][j] = int d_m phi_i phi_j vanishes unless j < nbelow(i)
// (build_tables checks this and stores exact zeros there).
__host__ __device__ constexpr int basis_degree(int i) { return i < 1 ? 0 : i < 3 ? 1 : i < 6 ? 2 : i < 10 ? 3 : 4; }
__host__ __device__ constexpr int nbelow(int i) { return basis_degree(i) * (basis_degree(i) + 1) / 2; }

// point r of the trace of field f on edge n of slot s in shared memory (either layout)
template <typename T, int R1>
__device__ __forceinline__ T &tr_at(T *tr, int f, int n, int slot, int NS, int r) {
    using L = TraceLayout<T, R1>;
    if constexpr (L::vec)
        return tr[((size_t)(f * 3 + n) * NS + slot) * L::RP + r];
    else
        return tr[((size_t)(f * 3 + n) * R1 + r) * NS + slot];
}

// trace of c on own edge n into field f of the slot's shared-memory traces
template <typename T, int N, int R2, int R1, int TK, int n>
__device__ __forceinline__ void store_trace(const T (&c)[N], T *tr, int f, int NS, int slot) {
    if constexpr (kCompactCode<T>) {
        const CTab<T, N, R2, R1> &t = tab_ref<T, N, R2, R1, TK>();
#pragma unroll 1
        for (int r = 0; r < R1; ++r) {
            T v = T(0);
#pragma unroll
            for (int j = 0; j < N; ++j) v += t.phiE[(n * R1 + r) * N + j] * c[j];
            tr_at<T, R1>(tr, f, n, slot, NS, r) = v;
        }
    } else {
        T v[R1];
        ctrace<T, N, R2, R1, TK, n>(c, v);
        tr_store<T, R1>(tr, f, n, slot, NS, v);
    }
}

// Phase A1: traces of x on the three edges of a slot (field 0).
template <typename T, int N, int R2, int R1, int TK>
__device__ __forceinline__ void slot_xtraces(const T (&x)[N], T *tr, int NS, int slot) {
    store_trace<T, N, R2, R1, TK, 0>(x, tr, 0, NS, slot);
    store_trace<T, N, R2, R1, TK, 1>(x, tr, 0, NS, slot);
    store_trace<T, N, R2, R1, TK, 2>(x, tr, 0, NS, slot);
}

// Where the apply takes the x values of triangles: LoadX reads the N x K vector X (CG:
// through L2, see ldv).  A source has first(e, slot, x), called once per slot in phase
// A1 (slot: the triangle's slot in this block's tile and halo), get(e, slot, x) for a
// slot's later reads and for a neighbour outside tile and halo (slot -1), and comp(e, j)
// for one coefficient (the rolled loops of the double-float kernels).
template <typename T, int N, bool CG>
struct LoadX {
    const T *X;
    int Ki;
    __device__ __forceinline__ void first(int e, int, T (&x)[N]) const { get(e, -1, x); }
    __device__ __forceinline__ void get(int e, int, T (&x)[N]) const {
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] = ldv<CG>(X + j * Ki + e);
    }
    __device__ __forceinline__ T comp(int e, int j) const { return ldv<CG>(X + j * Ki + e); }
};

// trace_nbr with the neighbour's x from a source
template <typename T, int N, int R1, typename XS>
__device__ __forceinline__ void trace_nbr_src(const T *phiE, const XS &xs, int k2, int n2, T (&out)[R1]) {
#pragma unroll
    for (int r = 0; r < R1; ++r) out[r] = T(0);
    if constexpr (kCompactCode<T>) {
#pragma unroll 1
        for (int j = 0; j < N; ++j) {
            const T v = xs.comp(k2, j);
#pragma unroll
            for (int r = 0; r < R1; ++r) out[r] += phiE[(n2 * R1 + (R1 - 1 - r)) * N + j] * v;
        }
    } else {
        T v[N];
        xs.get(k2, -1, v);
#pragma unroll
        for (int j = 0; j < N; ++j) {
#pragma unroll
            for (int r = 0; r < R1; ++r) out[r] += phiE[(n2 * R1 + (R1 - 1 - r)) * N + j] * v[j];
        }
    }
}

// Central value {x} of the edge at our Gauss point r: the mean of our trace and the
// neighbour's, taken at its point R1 - 1 - r (the maps of eq. mapEE reverse the edge);
// our own trace on a Neumann edge (eq. globQm:N).  The neighbour's trace comes from its
// slot, or from global memory when the neighbour of a halo triangle has no slot (nsl = -2).
template <typename T, int N, int R2, int R1, int TK, int n, typename XS>
__device__ __forceinline__ void edge_mean(const T *phiE_s, const XS &xs, int code, int nsl,
                                          const T *tr, int NS, int slot, T (&f)[R1]) {
    tr_load<T, R1>(tr, 0, n, slot, NS, f);
    if (code >= 0) {
        T cp[R1];
        if (nsl >= 0) {
            T nb[R1];
            tr_load<T, R1>(tr, 0, code & 3, nsl, NS, nb);
#pragma unroll
            for (int r = 0; r < R1; ++r) cp[r] = nb[R1 - 1 - r];
        } else {
            trace_nbr_src<T, N, R1>(phiE_s, xs, code >> 2, code & 3, cp);
        }
#pragma unroll
        for (int r = 0; r < R1; ++r) f[r] = T(0.5) * (f[r] + cp[r]);
    }
}

// e += sgn * sum_r wphi_E[n][r][i] f_r: the edge's part of the reference flux (P or Q).
template <typename T, int N, int R2, int R1, int TK, int n>
__device__ __forceinline__ void edge_test_add(const T (&f)[R1], T (&a)[N], T (&b)[N], int which) {
    const CTab<T, N, R2, R1> &t = tab_ref<T, N, R2, R1, TK>();
    if constexpr (kCompactCode<T>) {
#pragma unroll 1
        for (int r = 0; r < R1; ++r) {
            const T fr = f[r];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const T v = t.wphiE[(n * R1 + r) * N + i] * fr;
                if (which == 0) {
                    a[i] -= v;
                    b[i] -= v;
                } else if (which == 1) {
                    a[i] += v;
                } else {
                    b[i] += v;
                }
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            T v = T(0);
#pragma unroll
            for (int r = 0; r < R1; ++r) v += t.wphiE[(n * R1 + r) * N + i] * f[r];
            if (which == 0) {
                a[i] -= v;
                b[i] -= v;
            } else if (which == 1) {
                a[i] += v;
            } else {
                b[i] += v;
            }
        }
    }
}

// sigma_n = d_h (nu^_n . zeta) at the Gauss points of edge n (field 1): the normal flux
// d_h z . nu |E| of the edge in reference coordinates (nu^_0 = (1, 1), nu^_1 = (-1, 0),
// nu^_2 = (0, -1)).
template <typename T, int N, int R2, int R1, int TK, int n>
__device__ __forceinline__ void store_sigma(const T (&d)[N], const T (&z1)[N], const T (&z2)[N], T *tr, int NS,
                                            int slot) {
    const CTab<T, N, R2, R1> &t = tab_ref<T, N, R2, R1, TK>();
    T w[N];
#pragma unroll
    for (int j = 0; j < N; ++j) w[j] = n == 0 ? z1[j] + z2[j] : (n == 1 ? -z1[j] : -z2[j]);
    if constexpr (kCompactCode<T>) {
#pragma unroll 1
        for (int r = 0; r < R1; ++r) {
            T dv = T(0), wv = T(0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                dv += t.phiE[(n * R1 + r) * N + j] * d[j];
                wv += t.phiE[(n * R1 + r) * N + j] * w[j];
            }
            tr_at<T, R1>(tr, 1, n, slot, NS, r) = dv * wv;
        }
    } else {
        T dv[R1], wv[R1];
        ctrace<T, N, R2, R1, TK, n>(d, dv);
        ctrace<T, N, R2, R1, TK, n>(w, wv);
#pragma unroll
        for (int r = 0; r < R1; ++r) dv[r] *= wv[r];
        tr_store<T, R1>(tr, 1, n, slot, NS, dv);
    }
}

// Phase A2 for triangle e at slot `slot`: the flux unknowns in contravariant form,
// zeta = det(B) B^{-1} Z (Z^m = -M^{-1} B_m x, block rows 1-2 of eq. timeDepSystem), and
// the normal-flux traces sigma of its three edges.
//
// With u^_m = H^_m x (Sec. 3.6.2) and e_n = sum_r wphi_E[n][r] {x}(r) the edge terms
// (eq. globQ, globQm:N; nothing on Dirichlet edges), the edge normals nu_n |E_n| of
// (Sec. 3.1) and the metric G = B^T B turn Z into
//   zeta^1 = (G22 P - G12 Q) / det B,  zeta^2 = (G11 Q - G12 P) / det B,
//   P = u^_1 - e_0 + e_1,  Q = u^_2 - e_0 + e_2,
// so that B enters through G and det B alone.  nsl[n]: slot of the neighbour across
// edge n (see edge_mean).
template <typename T, int N, int R2, int R1, int TK, typename XS>
__device__ __forceinline__ void slot_zeta(const T *phiE_s, const XS &xs, int e, const T (&x)[N],
                                          const T (&d)[N], const T (&bk)[4], const int (&code)[3],
                                          const int (&nsl)[3], T *tr, int NS, int slot, T (&z1)[N], T (&z2)[N]) {
    const CTab<T, N, R2, R1> &t = tab_ref<T, N, R2, R1, TK>();
    // P = H^_1 x, Q = H^_2 x (only the entries below the diagonal blocks of degree are nonzero)
    if constexpr (kCompactCode<T>) {
#pragma unroll
        for (int i = 0; i < N; ++i) z1[i] = z2[i] = T(0);
#pragma unroll 1
        for (int j = 0; j < N; ++j) {
            const T xj = xs.comp(e, j);
#pragma unroll
            for (int i = 0; i < N; ++i) {
                if (j < nbelow(i)) {
                    z1[i] += t.H1[i * N + j] * xj;
                    z2[i] += t.H2[i * N + j] * xj;
                }
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            T h1 = T(0), h2 = T(0);
#pragma unroll
            for (int j = 0; j < nbelow(i); ++j) {
                h1 += t.H1[i * N + j] * x[j];
                h2 += t.H2[i * N + j] * x[j];
            }
            z1[i] = h1;
            z2[i] = h2;
        }
    }
    const int c0 = code[0], c1 = code[1], c2 = code[2];
    {
        T f[R1];
        if (c0 != NBR_DIRICHLET) {
            edge_mean<T, N, R2, R1, TK, 0>(phiE_s, xs, c0, nsl[0], tr, NS, slot, f);
            edge_test_add<T, N, R2, R1, TK, 0>(f, z1, z2, 0);
        }
        if (c1 != NBR_DIRICHLET) {
            edge_mean<T, N, R2, R1, TK, 1>(phiE_s, xs, c1, nsl[1], tr, NS, slot, f);
            edge_test_add<T, N, R2, R1, TK, 1>(f, z1, z2, 1);
        }
        if (c2 != NBR_DIRICHLET) {
            edge_mean<T, N, R2, R1, TK, 2>(phiE_s, xs, c2, nsl[2], tr, NS, slot, f);
            edge_test_add<T, N, R2, R1, TK, 2>(f, z1, z2, 2);
        }
    }
    const T b11 = bk[0], b12 = bk[1], b21 = bk[2], b22 = bk[3];
    const T inv = T(1) / (b11 * b22 - b12 * b21);
    const T g11 = (b11 * b11 + b21 * b21) * inv, g12 = (b11 * b12 + b21 * b22) * inv,
            g22 = (b12 * b12 + b22 * b22) * inv;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const T P = z1[i], Q = z2[i];
        z1[i] = g22 * P - g12 * Q;
        z2[i] = g11 * Q - g12 * P;
    }
    store_sigma<T, N, R2, R1, TK, 0>(d, z1, z2, tr, NS, slot);
    store_sigma<T, N, R2, R1, TK, 1>(d, z1, z2, tr, NS, slot);
    store_sigma<T, N, R2, R1, TK, 2>(d, z1, z2, tr, NS, slot);
}

// Phase B, edge n of tile triangle i: R^m, R_D^m (eq. globR, globR:D) and the penalty
// S, S_D (eq. globS, globS:D) from the traces in shared memory.  On an interior edge
// the neighbour's outward normal is the opposite of ours, so the central flux
// 1/2 nu . (d^- z^- + d^+ z^+) |E| is (sigma^- - sigma^+) / 2.
template <typename T, int N, int R2, int R1, int TK, int n>
__device__ __forceinline__ void tile_edge(int code, int sl, const T *tr, int NS, int i, T eta, T (&acc)[N]) {
    if (code == NBR_NEUMANN) return;
    const CTab<T, N, R2, R1> &t = tab_ref<T, N, R2, R1, TK>();
    if constexpr (kCompactCode<T>) {
#pragma unroll 1
        for (int r = 0; r < R1; ++r) {
            const T xm = tr_at<T, R1>(const_cast<T *>(tr), 0, n, i, NS, r);
            const T sm = tr_at<T, R1>(const_cast<T *>(tr), 1, n, i, NS, r);
            T g;
            if (code >= 0) {
                const int n2 = code & 3, rp = R1 - 1 - r;
                const T xp = tr_at<T, R1>(const_cast<T *>(tr), 0, n2, sl, NS, rp);
                const T sp = tr_at<T, R1>(const_cast<T *>(tr), 1, n2, sl, NS, rp);
                g = T(0.5) * (sm - sp) + eta * (xm - xp);
            } else {
                g = sm + eta * xm;
            }
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] += t.wphiE[(n * R1 + r) * N + j] * g;
        }
    } else {
        T g[R1], xm[R1], sm[R1];
        tr_load<T, R1>(tr, 0, n, i, NS, xm);
        tr_load<T, R1>(tr, 1, n, i, NS, sm);
        if (code >= 0) {
            const int n2 = code & 3;
            T xp[R1], sp[R1];
            tr_load<T, R1>(tr, 0, n2, sl, NS, xp);
            tr_load<T, R1>(tr, 1, n2, sl, NS, sp);
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                const int rp = R1 - 1 - r;  // the neighbour's Gauss point at our point r (eq. mapEE)
                g[r] = T(0.5) * (sm[r] - sp[rp]) + eta * (xm[r] - xp[rp]);
            }
        } else {  // Dirichlet
#pragma unroll
            for (int r = 0; r < R1; ++r) g[r] = sm[r] + eta * xm[r];
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            T v = T(0);
#pragma unroll
            for (int r = 0; r < R1; ++r) v += t.wphiE[(n * R1 + r) * N + j] * g[r];
            acc[j] += v;
        }
    }
}

// The most threads of a fused-apply block: a tile of up to 256 triangles and whole warps
// of halo threads (a block is launched with its tile's size plus the warps its halo needs).
constexpr int FUSED_THREADS = 320;
constexpr int FUSED_MAX_TE = 256;

// Minimum resident blocks per SM asked of the register allocator: two for the FP32
// kernels of p >= 3, which would otherwise take 130-168 registers a thread and run
// one block per SM; four for p = 1, 2 (at most 51 registers: measured on 2,097,152
// triangles at p = 2, 141 us with the allocator's 64-register choice and three blocks
// per SM, 121 us with four); 0 leaves the allocator's default.
template <typename T, int N>
struct FusedOcc {
    static constexpr int min_blocks = (sizeof(T) == 4 && N >= 10) ? 2 : (sizeof(T) == 4 && N >= 3) ? 4 : 0;
};

// Volume term -sum_m G^m Z^m at the triangle points (Sec. 3.6.3).  In contravariant
// form the integrand grad phi_i . d_h z is (grad^ phi_i . d_h zeta) / det B and the
// quadrature weight carries det B, so no geometry enters: -sum_r d_h (w_r d_1 phi_i
// zeta^1 + w_r d_2 phi_i zeta^2) at q_r.  Tables in the constant bank.
template <typename T, int N, int R2, int R1, int TK>
__device__ __forceinline__ void volume_const(const T (&d)[N], const T (&z1)[N], const T (&z2)[N], T (&acc)[N]) {
    const CTab<T, N, R2, R1> &t = tab_ref<T, N, R2, R1, TK>();
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
        const T u = dv * w1;
        const T v = dv * w2;
        // d phi_0 / dx^ = 0: the constant function has no volume term
#pragma unroll
        for (int j = 1; j < N; ++j) acc[j] -= t.gw1[r * N + j] * u + t.gw2[r * N + j] * v;
    }
}

// the same with the point loop rolled and the tables read from shared memory in
// 16-byte vectors (row stride NP = N rounded up to 16 bytes); keeps the code of the
// high orders small
template <typename T, int N, int R2, int NP>
__device__ __forceinline__ void volume_smem(const T *phiQ_s, const T *gw1_s, const T *gw2_s, const T (&d)[N],
                                            const T (&z1)[N], const T (&z2)[N], T (&acc)[N]) {
#pragma unroll 1
    for (int r = 0; r < R2; ++r) {
        alignas(16) T ph[NP];
        alignas(16) T g1[NP];
        alignas(16) T g2[NP];
#pragma unroll
        for (int q = 0; q < NP * (int)sizeof(T) / 16; ++q) {
            reinterpret_cast<float4 *>(ph)[q] = reinterpret_cast<const float4 *>(phiQ_s + r * NP)[q];
            reinterpret_cast<float4 *>(g1)[q] = reinterpret_cast<const float4 *>(gw1_s + r * NP)[q];
            reinterpret_cast<float4 *>(g2)[q] = reinterpret_cast<const float4 *>(gw2_s + r * NP)[q];
        }
        T dv = T(0), w1 = T(0), w2 = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            dv += ph[j] * d[j];
            w1 += ph[j] * z1[j];
            w2 += ph[j] * z2[j];
        }
        const T u = dv * w1;
        const T v = dv * w2;
#pragma unroll
        for (int j = 1; j < N; ++j) acc[j] -= g1[j] * u + g2[j] * v;
    }
}

// The FP32 kernels of p >= 3 evaluate the volume term on the tensor cores (ldg_tc.cuh).
// The BF16-table operator (table kind 1) of p >= 3 evaluates its volume term on the tensor
// cores (ldg_tc.cuh).  The FP32 operator keeps it on the FP32 pipes: with immediate table
// operands that measured faster than the mma.sync form (131,072 triangles, p = 4: 29.6 us
// against 39.5 us; p = 3: 8.8 against 12.8 us).
template <typename T, int N, int TK>
constexpr bool kTensorVolume = std::is_same<T, float>::value && N >= 10 && TK == 1;

// Dynamic shared memory of one block: two traced fields (x and sigma) on three edges
// per slot, then (kTensorVolume) each tile warp's staged operands, from the next 16-byte
// boundary (they are read as 16-byte vectors; 2 x 3 x R1 x nslot values need not end on
// one).
template <typename T, int R1>
__host__ __device__ constexpr size_t trace_bytes_aligned(int nslot) {
    return (((size_t)2 * 3 * TraceLayout<T, R1>::RP * nslot * sizeof(T) + 15) / 16) * 16;
}
template <typename T, int N, int R1, int TK = 0>
constexpr size_t fused_smem(int nslot, int te) {
    return trace_bytes_aligned<T, R1>(nslot) +
           (kTensorVolume<T, N, TK> ? (size_t)(te / 32) * TC_STAGE_FLOATS * sizeof(float) : 0);
}

// Let a kernel take the device's opt-in maximum of dynamic shared memory (once per
// kernel; the launch then passes only what it needs).
template <typename Kern>
bool allow_max_smem(Kern kernel) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kernel) != cudaSuccess)
        return false;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes) == cudaSuccess;
}

// One tile of y = S x: phases A1, A2 and B by the block's threads (a tile of TE triangles,
// the threads past TE for its halo), x from the source xs (LoadX: a vector).
// EPI != FUSED_EPI_NONE adds the tile's part of the epilogue's dot products to dots: e1,
// e2 are r0 (ALPHA); s, r0 (OMEGA).  CG: e1 and e2 are read through L2 (ld.global.cg),
// for a persistent kernel whose other blocks write them between its phases; a block
// that runs several tiles in a row must call this between two block barriers.  Returns
// the number of the tile's triangles it applied (0 for a batch tile whose problems are
// all done).
template <typename T, int N, int R2, int R1, int EPI, int TK, bool CG, typename XS>
__device__ __forceinline__ int fused_tile(
    int tile, const XS &xs, T *__restrict__ Y, const T *__restrict__ Dc, const T *__restrict__ Bg,
    const int32_t *__restrict__ nbr, const int16_t *__restrict__ slotg, const int32_t *__restrict__ halo_ptr,
    const int32_t *__restrict__ halo, const int16_t *__restrict__ halo_slot, int Ki, int TE, int NS, T tau, T eta,
    T mass, const T *__restrict__ tabg, const T *__restrict__ e1, const T *__restrict__ e2, const KScal *sc,
    const BatchView &bv, Acc<T> (&dots)[EPI == FUSED_EPI_OMEGA ? 4 : 1]) {
    // FP32: the volume loop is unrolled with immediate table operands at every order (on
    // 131,072 triangles at p = 4: 29.6 us, against 34.9 us with the tables read from
    // shared memory in a rolled loop); FP64 and double-float keep the rolled loop at
    // high order, whose unrolled code would not fit the instruction cache
    constexpr bool kBigVolume = R2 * N > 150 && !std::is_same<T, float>::value;
    constexpr bool kTC = kTensorVolume<T, N, TK>;
    __shared__ __align__(16) float tc_s[kTC ? TC_TAB_FLOATS : 1];
    constexpr int NP = ((N * (int)sizeof(T) + 15) / 16) * 16 / (int)sizeof(T);
    constexpr int VOL = kBigVolume ? 3 * R2 * NP : 4;
    __shared__ __align__(16) T phiE_s[3 * R1 * N];
    __shared__ __align__(16) T vol_s[VOL];
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    T *tr = reinterpret_cast<T *>(dyn_smem);
    if constexpr (kTC) {
        const CTab<T, N, R2, R1> &ct = tab_ref<T, N, R2, R1, TK>();
        tc_fill_tables<N, R2>(tc_s, ct.phiQ, ct.gw1, ct.gw2);
    }
    {
        const int o_phiE = 4 * R2 * N + 2 * N * N;  // table layout of table_offsets()
        for (int j = threadIdx.x; j < 3 * R1 * N; j += blockDim.x) phiE_s[j] = tabg[o_phiE + j];
        if constexpr (kBigVolume) {
            const int o_phiQ = 0, o_gw1 = 2 * R2 * N, o_gw2 = 3 * R2 * N;
            for (int j = threadIdx.x; j < R2 * NP; j += blockDim.x) {
                const int r = j / NP, c = j - r * NP;
                vol_s[j] = c < N ? tabg[o_phiQ + r * N + c] : T(0);
                vol_s[R2 * NP + j] = c < N ? tabg[o_gw1 + r * N + c] : T(0);
                vol_s[2 * R2 * NP + j] = c < N ? tabg[o_gw2 + r * N + c] : T(0);
            }
        }
    }
    const int start = tile * TE;
    int cnt = (Ki - start) < TE ? (Ki - start) : TE;
    const int h0 = halo_ptr[tile];
    int nh = halo_ptr[tile + 1] - h0;
    if constexpr (EPI != FUSED_EPI_NONE) {
        if (bv.eprob && cnt > 0) {
            // a batch: a tile whose problems have all finished their iterations does no
            // work (it still takes part in the reduction)
            bool idle = true;
            for (int q = bv.eprob[start]; q <= bv.eprob[start + cnt - 1]; ++q) idle = idle && sc[q].done;
            if (idle) cnt = nh = 0;
        }
    }
    const int i = threadIdx.x;
    const int hstride = blockDim.x - TE;
    T z1[N], z2[N], d[N];
    if constexpr (EPI != FUSED_EPI_NONE && !CG) {
        // the epilogue's vectors: start their loads into L1 now, so that their latency
        // hides behind phases A and B
        if (i < cnt) {
#pragma unroll
            for (int j = 0; j < N; ++j) {
                asm volatile("prefetch.global.L1 [%0];" ::"l"(e1 + j * Ki + start + i));
                if constexpr (EPI == FUSED_EPI_OMEGA) asm volatile("prefetch.global.L1 [%0];" ::"l"(e2 + j * Ki + start + i));
            }
        }
    }
    T bk[4];
    int code[3], nsl[3];
    // A1: traces of x of every slot (tile triangles load d_h for the later phases)
    if (i < TE) {
        if (i < cnt) {
            const int k = start + i;
            T xa[N];
#pragma unroll
            for (int j = 0; j < N; ++j) d[j] = Dc[j * Ki + k];
            xs.first(k, i, xa);
            slot_xtraces<T, N, R2, R1, TK>(xa, tr, NS, i);
        }
    } else {
        for (int j = i - TE; j < nh; j += hstride) {
            const int eh = halo[h0 + j];
            T xh[N];
            xs.first(eh, TE + j, xh);
            slot_xtraces<T, N, R2, R1, TK>(xh, tr, NS, TE + j);
        }
    }
    __syncthreads();
    // A2: flux unknowns (contravariant form) and the normal-flux traces
    if (i < TE) {
        if (i < cnt) {
            const int k = start + i;
            T xa[N], ba[4];
            int ca[3];
            xs.get(k, i, xa);
#pragma unroll
            for (int q = 0; q < 4; ++q) ba[q] = Bg[q * Ki + k];
#pragma unroll
            for (int n = 0; n < 3; ++n) ca[n] = nbr[n * Ki + k];
            const int sa[3] = {slotg[k], slotg[Ki + k], slotg[2 * Ki + k]};
            slot_zeta<T, N, R2, R1, TK>(phiE_s, xs, k, xa, d, ba, ca, sa, tr, NS, i, z1, z2);
        }
        if constexpr (kTC) {
            // the volume operands go to the warp's stage now, so that their registers are
            // free in phase B (whole warps: TE is a multiple of 32; lanes past the end of
            // the last tile stage zeros)
            float *stage = reinterpret_cast<float *>(dyn_smem + trace_bytes_aligned<T, R1>(NS)) +
                           (size_t)(i >> 5) * TC_STAGE_FLOATS;
            tc_stage<N>(i < cnt, d, z1, z2, stage);
        }
    } else {
        for (int j = i - TE; j < nh; j += hstride) {
            const int eh = halo[h0 + j];
            const int q = 3 * (h0 + j);
            T xh[N], hd[N], hb[4], hz1[N], hz2[N];
            int hc[3];
            const int hs[3] = {halo_slot[q], halo_slot[q + 1], halo_slot[q + 2]};
            xs.get(eh, TE + j, xh);
#pragma unroll
            for (int l = 0; l < N; ++l) hd[l] = Dc[l * Ki + eh];
#pragma unroll
            for (int l = 0; l < 4; ++l) hb[l] = Bg[l * Ki + eh];
#pragma unroll
            for (int n = 0; n < 3; ++n) hc[n] = nbr[n * Ki + eh];
            slot_zeta<T, N, R2, R1, TK>(phiE_s, xs, eh, xh, hd, hb, hc, hs, tr, NS, TE + j, hz1, hz2);
        }
    }
    __syncthreads();
    using A = Acc<T>;
    T acc[N];
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j] = T(0);
    if constexpr (kTC) {
        // B, volume term on the tensor cores: whole warps of the tile
        if (i < TE) {
            float *stage = reinterpret_cast<float *>(dyn_smem + trace_bytes_aligned<T, R1>(NS)) +
                           (size_t)(i >> 5) * TC_STAGE_FLOATS;
            volume_tc<N, R2, TK == 1>(acc, stage, tc_s);
        }
    }
    if (i < cnt) {
        // B: volume and edge terms of the tile triangles
        const int k = start + i;
        if constexpr (kTC) {
        } else if constexpr (kBigVolume) {
            volume_smem<T, N, R2, NP>(vol_s, vol_s + R2 * NP, vol_s + 2 * R2 * NP, d, z1, z2, acc);
        } else {
            volume_const<T, N, R2, R1, TK>(d, z1, z2, acc);
        }
        // loaded after the volume term, whose registers are then free
#pragma unroll
        for (int n = 0; n < 3; ++n) code[n] = nbr[n * Ki + k];
#pragma unroll
        for (int n = 0; n < 3; ++n) nsl[n] = code[n] >= 0 ? slotg[n * Ki + k] : 0;
        tile_edge<T, N, R2, R1, TK, 0>(code[0], code[0] >= 0 ? nsl[0] : 0, tr, NS, i, eta, acc);
        tile_edge<T, N, R2, R1, TK, 1>(code[1], code[1] >= 0 ? nsl[1] : 0, tr, NS, i, eta, acc);
        tile_edge<T, N, R2, R1, TK, 2>(code[2], code[2] >= 0 ? nsl[2] : 0, tr, NS, i, eta, acc);
#pragma unroll
        for (int q = 0; q < 4; ++q) bk[q] = Bg[q * Ki + k];
        const T md = mass * (bk[0] * bk[3] - bk[1] * bk[2]);
        T xo[N];
        xs.get(k, i, xo);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const T yj = md * xo[j] + tau * acc[j];
            Y[j * Ki + k] = yj;
            if constexpr (EPI == FUSED_EPI_ALPHA) {
                dots[0] += (A)ldv<CG>(e1 + j * Ki + k) * (A)yj;
            } else if constexpr (EPI == FUSED_EPI_OMEGA) {
                const A sj = (A)ldv<CG>(e1 + j * Ki + k), rj = (A)ldv<CG>(e2 + j * Ki + k);
                dots[0] += (A)yj * sj;
                dots[1] += (A)yj * (A)yj;
                dots[2] += rj * sj;
                dots[3] += rj * (A)yj;
            }
        }
    }
    return cnt;
}

// y = S x, one tile per block.  EPI: reductions fused into the end of the apply
// (FUSED_EPI_* in krylov.cuh; one partial per block, the last block updates the
// scalars); e1, e2: r0 (ALPHA); s, r0 (OMEGA).
template <typename T, int N, int R2, int R1, int EPI = FUSED_EPI_NONE, int TK = 0>
__global__ void __launch_bounds__(FUSED_THREADS, FusedOcc<T, N>::min_blocks) k_apply_fused(
    const T *__restrict__ X, T *__restrict__ Y, const T *__restrict__ Dc, const T *__restrict__ Bg,
    const int32_t *__restrict__ nbr, const int16_t *__restrict__ slotg, const int32_t *__restrict__ halo_ptr,
    const int32_t *__restrict__ halo, const int16_t *__restrict__ halo_slot, int64_t K, int TE, int NS, T tau,
    T eta, T mass, const T *__restrict__ tabg, const int *__restrict__ skip, const T *__restrict__ e1 = nullptr,
    const T *__restrict__ e2 = nullptr, double *part = nullptr, KScal *sc = nullptr,
    unsigned int *counter = nullptr, BatchView bv = BatchView()) {
    if (skip && *skip) return;
    using A = Acc<T>;
    constexpr int ND = EPI == FUSED_EPI_OMEGA ? 4 : 1;
    A dots[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) dots[q] = A(0);
    // K * N < 2^31 (checked at setup): 32-bit offsets
    const LoadX<T, N, false> xs{X, (int)K};
    const int cnt = fused_tile<T, N, R2, R1, EPI, TK, false>(blockIdx.x, xs, Y, Dc, Bg, nbr, slotg, halo_ptr, halo, halo_slot,
                                             (int)K, TE, NS, tau, eta, mass, tabg, e1, e2, sc, bv, dots);
    if constexpr (EPI != FUSED_EPI_NONE) {
        if (bv.eprob) {
            // a batch: sums per problem, scalars of every running problem in the last block
            const int start = blockIdx.x * TE;
            const int i = threadIdx.x;
            double dd[ND];
#pragma unroll
            for (int q = 0; q < ND; ++q) dd[q] = (double)dots[q];
            batch_add<ND>(bv, i < cnt ? bv.eprob[start + i] : -1, dd);
            if (last_block(counter)) {
                batch_finish<ND>(bv, sc, [&](int q, const double *sum) {
                    if constexpr (EPI == FUSED_EPI_ALPHA)
                        bicg_alpha_scalars(sum[0], sc + q);
                    else
                        bicg_omega_scalars(sum[0], sum[1], sum[2], sum[3], sc + q);
                });
                if (threadIdx.x == 0) *counter = 0;
            }
            return;
        }
        block_partials_any<ND>(dots, part);
        if (last_block(counter)) {
            double sum[ND];
#pragma unroll
            for (int q = 0; q < ND; ++q) sum[q] = sum_partials_cg(part, q, gridDim.x);
            if (threadIdx.x == 0) {
                if constexpr (EPI == FUSED_EPI_ALPHA)
                    bicg_alpha_scalars(sum[0], sc);
                else
                    bicg_omega_scalars(sum[0], sum[1], sum[2], sum[3], sc);
                *counter = 0;
            }
        }
    }
}

}  // namespace festung
