// C ABI of the GB300 LDG solver: context, data upload, operator apply, the
// implicit-Euler step (BiCGStab / CG with device-resident scalars, optionally FP32
// inner iterations refined on residuals evaluated in double-float arithmetic), the
// stationary problem, flux recovery, batches of problems and the learned warm start.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "dfloat.cuh"
#include "internal.h"
#include "krylov.cuh"
#include "krylov_kernels.cuh"
#include "dispatch.h"
#include "ops.h"

using namespace festung;

namespace festung {

TableOffsets table_offsets(int N, int R2, int R1) {
    TableOffsets o;
    o.phiQ = 0;
    o.wphiQ = R2 * N;
    o.gw1 = 2 * R2 * N;
    o.gw2 = 3 * R2 * N;
    o.H1 = 4 * R2 * N;
    o.H2 = o.H1 + N * N;
    o.phiE = o.H2 + N * N;
    o.wphiE = o.phiE + 3 * R1 * N;
    o.total = o.wphiE + 3 * R1 * N;
    return o;
}

template <typename T>
struct Vecs {
    T *Z1 = nullptr, *Z2 = nullptr;                      // flux unknowns of the apply
    T *r = nullptr, *r0 = nullptr, *p = nullptr, *ph = nullptr, *v = nullptr;
    T *s = nullptr, *sh = nullptr, *t = nullptr, *x = nullptr, *b = nullptr;
    T *inv = nullptr;                                     // 1 / (2|T_k|), length K
    bool krylov = false;
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int solver = 0, chunk = 0, use_P = -1, tab_bf16 = 0;
    int64_t nodes = 0;
    double tau = 0.0, mass = 1.0;
    const void *x = nullptr, *b = nullptr;
};

struct Workspace {
    Vecs<double> d;
    Vecs<float> f;
    double *part = nullptr;  // reduction partials [4][nblk]
    KScal *scal = nullptr;   // device scalars
    KScal *h_scal = nullptr; // pinned host mirror
    int nblk = 0;
    double *scratch64 = nullptr;  // W^1, W^2 of the Dirichlet lift (2 x N x K)
    int *d_flags = nullptr, *h_flags = nullptr;
    float *P = nullptr;            // block-Jacobi diagonal blocks (FP32 scratch of the build)
    __nv_bfloat16 *Pb = nullptr;   // their inverses in BF16, [(i N + j) K + k]
    unsigned int *counter = nullptr;  // last-block counter of the reducing Krylov kernels
    double *part2 = nullptr;          // second partials buffer (CG: (r, r))
    double *res = nullptr, *h_res = nullptr;  // device / pinned host pair for residual norms
    dfloat *xdf = nullptr, *ydf = nullptr;    // N x K double-float operand and result of the residual apply
    int *loopctl = nullptr;    // device: chunks run by the Krylov graph's loop, and their bound
    int *h_loopctl = nullptr;  // pinned host mirror of loopctl[0]
    // persistent BiCGStab kernel (bicg_persist.cu): partials, grid-barrier counters, flag
    float *ppart = nullptr;
    void *pscal = nullptr;  // 256 bytes: the persistent kernel's scalars
    int pcap = 0;
    unsigned int *pbar = nullptr;
    int *perr = nullptr, *h_perr = nullptr;
    bool use_P = false;        // P is valid for the current step
    GraphCache g64, g32;
};

int elem_grid(const festung_ctx *c) {
    const int64_t need = (c->K + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)c->num_sms * 8));
}

}  // namespace festung

namespace {

thread_local std::string g_create_err;

#define FCK(call)                                                                  \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            c->err = std::string(#call) + ": " + cudaGetErrorString(e_);           \
            return e_ == cudaErrorMemoryAllocation ? FESTUNG_ENOMEM : FESTUNG_ECUDA; \
        }                                                                          \
    } while (0)

template <typename T> const T *geomB(const festung_ctx *c);
template <> const double *geomB<double>(const festung_ctx *c) { return c->dB; }
template <> const float *geomB<float>(const festung_ctx *c) { return c->fB; }
template <typename T> Vecs<T> &vecs(festung_ctx *c);
template <> Vecs<double> &vecs<double>(festung_ctx *c) { return c->ws->d; }
template <> Vecs<float> &vecs<float>(festung_ctx *c) { return c->ws->f; }

// ---------------------------------------------------------------------------
// projection of samples (K x R2, row-major) onto the basis (Sec. 3.4)
// ---------------------------------------------------------------------------
// The sums run in double-float arithmetic (dfloat.cuh, about 48 bits) on the FP32 pipe:
// this device's FP64 pipe would take about 100 us for the 375 multiply-adds per triangle
// of p = 4 on 131,072 triangles.  The checks of the samples look at their bits (bit0
// non-finite, bit1 not > 0, bit2 not all equal bit for bit).
template <int N, int R2>
__global__ void __launch_bounds__(256) k_project(const double *__restrict__ samp, double *__restrict__ out,
                                                 float *__restrict__ out32, const double *__restrict__ wphiQ,
                                                 int64_t K, int check_positive, const int32_t *__restrict__ perm,
                                                 int *__restrict__ flags) {
    __shared__ dfloat sw[R2 * N];
    for (int i = threadIdx.x; i < R2 * N; i += blockDim.x) sw[i] = dfloat(wphiQ[i]);
    __syncthreads();
    constexpr long long kExp = 0x7ff0000000000000ll, kMag = 0x7fffffffffffffffll;
    int fl = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
        dfloat acc[N];
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] = dfloat(0.0f, 0.0f);
        const double *sp = samp + (int64_t)perm[k] * R2;  // samples arrive in the caller's triangle order
        const long long first = __double_as_longlong(sp[0]);
#pragma unroll 5
        for (int r = 0; r < R2; ++r) {
            const double v = sp[r];
            const long long bits = __double_as_longlong(v), mag = bits & kMag;
            if (mag >= kExp) fl |= 1;                                  // Inf or NaN
            if (check_positive && (bits <= 0 || mag > kExp)) fl |= 2;  // <= +0, negative or NaN
            if (bits != first) fl |= 4;
            const dfloat dv(v);
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] += sw[r * N + j] * dv;
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            out[j * K + k] = (double)acc[j];
            if (out32) out32[j * K + k] = acc[j].hi;
        }
    }
    if (fl) atomicOr(flags, fl);
}

__global__ void k_check_finite(const double *__restrict__ a, int64_t n, int *__restrict__ flags) {
    int fl = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(a[i])) fl = 1;
    if (fl) atomicOr(flags, 1);
}

// public K x N (caller's triangle order, row-major) <-> internal N x K (internal order)
__global__ void k_to_internal(const double *__restrict__ a, double *__restrict__ b, int64_t K, int N,
                              const int32_t *__restrict__ perm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K * N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / K;
        const int64_t k = i - j * K;
        b[i] = a[(int64_t)perm[k] * N + j];
    }
}
__global__ void k_to_public(const double *__restrict__ b, double *__restrict__ a, int64_t K, int N,
                            const int32_t *__restrict__ perm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K * N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / K;
        const int64_t k = i - j * K;
        a[(int64_t)perm[k] * N + j] = b[i];
    }
}

template <typename T>
__global__ void k_inv_det(const T *__restrict__ B, T *__restrict__ inv, int64_t K) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x)
        inv[k] = T(1) / (B[k] * B[3 * K + k] - B[K + k] * B[2 * K + k]);
}

// ---------------------------------------------------------------------------
// Krylov vector kernels (N x K vectors, one thread per element, FP32 or FP64)
// ---------------------------------------------------------------------------
#define ELEM_LOOP(k) for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x)

// r = b - y (y = S x, or y = null for x = 0); shadow r0 = r (or, after a restart, r
// with a fixed pseudo-random reweighting so that the new Krylov process differs);
// p = v = 0; partials (r,r), (b,b)
template <typename T>
__global__ void k_kr_init(int64_t K, int N, const T *b, const T *y, T *r, T *r0, T *p, T *v, double *part,
                          int reweight) {
    using A = typename std::conditional<std::is_same<T, float>::value, float, double>::type;
    A acc[3] = {A(0), A(0), A(0)};
    ELEM_LOOP(k) {
        for (int j = 0; j < N; ++j) {
            const int64_t i = j * K + k;
            const T bi = b[i];
            const T ri = y ? bi - y[i] : bi;
            r[i] = ri;
            T wgt = T(1);
            if (reweight) {
                const uint32_t h = (uint32_t)(i * 2654435761ull) >> 8;
                wgt = T(0.5) + T(h & 0xffff) / T(65536);
            }
            r0[i] = ri * wgt;
            if (p) p[i] = T(0);
            if (v) v[i] = T(0);
            acc[0] += (A)ri * (A)ri;
            acc[1] += (A)bi * (A)bi;
            acc[2] += (A)(ri * wgt) * (A)ri;
        }
    }
    block_partials<3>(acc, part);
}

__global__ void k_fin_init(KScal *sc, const double *part, int nblk, double tol) {
    const double r2 = sum_partials(part, 0, nblk);
    const double b2 = sum_partials(part, 1, nblk);
    const double r0r = sum_partials(part, 2, nblk);
    if (threadIdx.x == 0) {
        sc->r2 = r2;
        sc->b2 = b2;
        sc->tol2 = tol * tol;
        sc->rho = r0r;  // (r0, r); CG sets rho = (r, z) itself
        sc->r2_0 = r2;
        sc->ss = r2;
        sc->first = 1;
        sc->pending = 0;
        sc->alpha = 1.0;
        sc->omega = 1.0;
        sc->beta = 0.0;
        sc->den = 0.0;
        sc->iter = 0;
        sc->breakdown = 0;
        sc->sconv = 0;
        sc->done = (r2 <= sc->tol2 * b2) ? 1 : 0;
    }
}

// x += alpha ph (used when BiCGStab converged on s)
template <typename T>
__global__ void k_axpy_alpha(int64_t K, int N, T *x, const T *ph, const KScal *sc) {
    const T alpha = (T)sc->alpha;
    ELEM_LOOP(k) {
        for (int j = 0; j < N; ++j) x[j * K + k] += alpha * ph[j * K + k];
    }
}

// partials of ||b - y||^2 and ||b||^2 in precision T
template <typename T>
__global__ void k_residual(int64_t K, int N, const T *b, const T *y, double *part) {
    using A = typename std::conditional<std::is_same<T, float>::value, float, double>::type;
    A acc[2] = {A(0), A(0)};
    ELEM_LOOP(k) {
        for (int j = 0; j < N; ++j) {
            const A bi = (A)b[j * K + k], ri = bi - (A)y[j * K + k];
            acc[0] += ri * ri;
            acc[1] += bi * bi;
        }
    }
    block_partials<2>(acc, part);
}

// refinement helpers
__global__ void k_residual64(int64_t n, const double *b, const double *y, double *r, double *part) {
    double acc[2] = {0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = b[i] - y[i];
        r[i] = ri;
        acc[0] += ri * ri;
        acc[1] += b[i] * b[i];
    }
    block_partials<2>(acc, part);
}

// r = b - y for a double-float y, with (r, r) and (b, b)
__global__ void k_residual_df(int64_t n, const double *b, const dfloat *y, double *r, double *part) {
    double acc[2] = {0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = b[i] - (double)y[i];
        r[i] = ri;
        acc[0] += ri * ri;
        acc[1] += b[i] * b[i];
    }
    block_partials<2>(acc, part);
}

__global__ void k_to_df(int64_t n, const double *a, dfloat *b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = dfloat(a[i]);
}

__global__ void k_from_df(int64_t n, const dfloat *a, double *b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

// Z^m = Zh^m - W^m in the caller's order: out[(m K + u) N + j], u = perm[i]
__global__ void k_flux_public(int64_t K, int N, const double *Z1, const double *Z2, const double *W1,
                              const double *W2, const int32_t *perm, double *out) {
    ELEM_LOOP(i) {
        const int64_t u = perm[i];
        for (int j = 0; j < N; ++j) {
            out[u * N + j] = Z1[j * K + i] - W1[j * K + i];
            out[(K + u) * N + j] = Z2[j * K + i] - W2[j * K + i];
        }
    }
}

struct QuadWeights {
    double w[32];
};

// Squared L2 error of c_h against samples of c at the triangle points (Sec. 3.5):
// sum_k 2|T_k| sum_r w_r (c_h(F_k(q_r)) - c(F_k(q_r)))^2; samples in the caller's order.
__global__ void k_l2_error(int64_t K, int N, int R2, const double *C, const double *samp, const double *phiQ,
                           QuadWeights qw, const double *Bg, const int32_t *perm, double *part) {
    double acc[1] = {0.0};
    ELEM_LOOP(i) {
        const int64_t u = perm[i];
        const double det = Bg[i] * Bg[3 * K + i] - Bg[K + i] * Bg[2 * K + i];
        double e = 0.0;
        for (int r = 0; r < R2; ++r) {
            double ch = 0.0;
            for (int j = 0; j < N; ++j) ch += C[j * K + i] * phiQ[r * N + j];
            const double dlt = ch - samp[u * R2 + r];
            e += qw.w[r] * dlt * dlt;
        }
        acc[0] += det * e;
    }
    block_partials<1>(acc, part);
}

__global__ void k_fin_sums(double *out, const double *part, int nblk, int np) {
    for (int p = 0; p < np; ++p) {
        const double v = sum_partials(part, p, nblk);
        if (threadIdx.x == 0) out[p] = v;
    }
}

__global__ void k_scale_to_f32(int64_t n, const double *a, float *b, double s) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)(a[i] * s);
}

__global__ void k_add_f32(int64_t n, double *x, const float *d, double s) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += s * (double)d[i];
}

__global__ void k_commit_coeff(int64_t n, const double *src, double *d, float *f) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = src[i];
        d[i] = v;
        f[i] = (float)v;
    }
}

// x = l0 C + l1 C_prev + l2 C_prev2
__global__ void k_extrapolate3(int64_t n, const double *C, const double *Cp, const double *Cpp, double *x, double l0,
                               double l1, double l2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = l0 * C[i] + l1 * Cp[i] + l2 * Cpp[i];
}

// features of the learned warm start, first pass: sum over triangles of |M^{-1} r_k|^2
// and of the mean of d_h (mode 0)
__global__ void k_ws_sums(int64_t K, int N, const double *r, const double *D, const double *Bg, double *part) {
    double acc[2] = {0.0, 0.0};
    ELEM_LOOP(k) {
        const double det = Bg[k] * Bg[3 * K + k] - Bg[K + k] * Bg[2 * K + k];
        for (int j = 0; j < N; ++j) {
            const double q = r[j * K + k] / det;
            acc[0] += q * q;
        }
        acc[1] += D[k];
    }
    block_partials<2>(acc, part);
}

// second pass: per triangle (row k of X, F = 3 + 4 N values): d_h modes 0..2 over the
// mean of mode 0; M^{-1} r of the triangle and of its neighbours across edges 0, 1, 2
// (zero on the boundary), over the RMS value rs
__global__ void k_ws_features(int64_t K, int N, const double *r, const double *D, const double *Bg,
                              const int32_t *nbr, double inv_rs, double inv_d, float *X) {
    const int F = 3 + 4 * N;
    ELEM_LOOP(k) {
        float *x = X + k * F;
        for (int j = 0; j < 3; ++j) x[j] = j < N ? (float)(D[j * K + k] * inv_d) : 0.0f;
        for (int e = 0; e < 4; ++e) {
            int64_t q = k;
            if (e > 0) {
                const int code = nbr[(e - 1) * K + k];
                q = code >= 0 ? (int64_t)(code >> 2) : -1;
            }
            float *y = x + 3 + e * N;
            if (q < 0) {
                for (int j = 0; j < N; ++j) y[j] = 0.0f;
                continue;
            }
            const double det = Bg[q] * Bg[3 * K + q] - Bg[K + q] * Bg[2 * K + q];
            for (int j = 0; j < N; ++j) y[j] = (float)(r[j * K + q] / det * inv_rs);
        }
    }
}

// loss weights of the learned warm start: sqrt(S_kk[j][j] / 2|T_k|) from the FP32 diagonal
// blocks P[(i N + j) K + k]
__global__ void k_ws_weights(int64_t K, int N, const float *P, const double *Bg, float *Wt) {
    ELEM_LOOP(k) {
        const double det = Bg[k] * Bg[3 * K + k] - Bg[K + k] * Bg[2 * K + k];
        for (int j = 0; j < N; ++j) {
            const double q = (double)P[((int64_t)j * N + j) * K + k] / det;
            Wt[k * N + j] = (float)std::sqrt(q > 0.0 ? q : 0.0);
        }
    }
}

// x = C + a (C - C_prev)
__global__ void k_extrapolate(int64_t n, const double *C, const double *Cp, double *x, double a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = C[i] + a * (C[i] - Cp[i]);
}

__global__ void k_zero_f32(int64_t n, float *a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = 0.0f;
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
template <typename T>
int alloc_vecs(festung_ctx *c, Vecs<T> &V, bool krylov) {
    const size_t n = (size_t)c->K * c->N * sizeof(T);
    if (!V.Z1) {
        FCK(cudaMalloc(&V.Z1, n));
        FCK(cudaMalloc(&V.Z2, n));
    }
    if (krylov && !V.krylov) {
        T **ptrs[] = {&V.r, &V.r0, &V.p, &V.ph, &V.v, &V.s, &V.sh, &V.t, &V.x, &V.b};
        for (T **q : ptrs) FCK(cudaMalloc(q, n));
        FCK(cudaMalloc(&V.inv, (size_t)c->K * sizeof(T)));
        k_inv_det<T><<<elem_grid(c), 256, 0, c->stream>>>(geomB<T>(c), V.inv, c->K); ++c->launches;
        FCK(cudaGetLastError());
        V.krylov = true;
    }
    return FESTUNG_OK;
}

template <typename T>
void free_vecs(Vecs<T> &V) {
    T *ptrs[] = {V.Z1, V.Z2, V.r, V.r0, V.p, V.ph, V.v, V.s, V.sh, V.t, V.x, V.b, V.inv};
    for (T *q : ptrs)
        if (q) cudaFree(q);
    V = Vecs<T>();
}

int ensure_ws(festung_ctx *c) {
    if (!c->ws) {
        c->ws = new (std::nothrow) Workspace();
        if (!c->ws) {
            c->err = "host allocation failed";
            return FESTUNG_ENOMEM;
        }
        Workspace &w = *c->ws;
        w.nblk = std::max(1, std::min(c->num_sms * 4, (int)((c->K + RED_THREADS - 1) / RED_THREADS)));
        // partials of the reducing kernels: 4 per block of a reduction or per tile of a
        // fused apply epilogue (tiles of at least 32 triangles, whatever the tiling)
        const int64_t tiles = (c->K + 31) / 32;
        FCK(cudaMalloc(&w.part, sizeof(double) * 4 * std::max<int64_t>(w.nblk, tiles)));
        FCK(cudaMalloc(&w.scal, sizeof(KScal)));
        FCK(cudaMallocHost(&w.h_scal, sizeof(KScal)));
        FCK(cudaMalloc(&w.d_flags, sizeof(int) * 4));
        FCK(cudaMalloc(&w.res, sizeof(double) * 2));
        FCK(cudaMalloc(&w.counter, sizeof(unsigned int)));
        FCK(cudaMemset(w.counter, 0, sizeof(unsigned int)));
        FCK(cudaMalloc(&w.part2, sizeof(double) * 4 * w.nblk));
        FCK(cudaMallocHost(&w.h_res, sizeof(double) * 2));
        FCK(cudaMallocHost(&w.h_flags, sizeof(int) * 4));
        FCK(cudaMalloc(&w.loopctl, sizeof(int) * 2));
        FCK(cudaMallocHost(&w.h_loopctl, sizeof(int)));
        if (bicg_persistent_supported(c)) {
            w.pcap = (int)std::min<int64_t>(tiles, 1 << 20);
            FCK(cudaMalloc(&w.ppart, sizeof(float) * 6 * (size_t)w.pcap));
            FCK(cudaMalloc(&w.pscal, 256));
            FCK(cudaMalloc(&w.pbar, sizeof(unsigned int) * 2));
            FCK(cudaMalloc(&w.perr, sizeof(int)));
            FCK(cudaMallocHost(&w.h_perr, sizeof(int)));
        }
    }
    return FESTUNG_OK;
}

void reset_graphs(festung_ctx *c) {
    if (!c->ws) return;
    for (GraphCache *g : {&c->ws->g64, &c->ws->g32}) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        *g = GraphCache();
    }
}

void free_ctx_device(festung_ctx *c) {
    if (c->coarse) {
        festung_destroy(c->coarse);
        c->coarse = nullptr;
    }
    reset_graphs(c);
    if (c->ws) {
        free_vecs(c->ws->d);
        free_vecs(c->ws->f);
        if (c->ws->part) cudaFree(c->ws->part);
        if (c->ws->scal) cudaFree(c->ws->scal);
        if (c->ws->h_scal) cudaFreeHost(c->ws->h_scal);
        if (c->ws->scratch64) cudaFree(c->ws->scratch64);
        if (c->ws->d_flags) cudaFree(c->ws->d_flags);
        if (c->ws->P) cudaFree(c->ws->P);
        if (c->ws->Pb) cudaFree(c->ws->Pb);
        if (c->ws->counter) cudaFree(c->ws->counter);
        if (c->ws->part2) cudaFree(c->ws->part2);
        if (c->ws->res) cudaFree(c->ws->res);
        if (c->ws->h_res) cudaFreeHost(c->ws->h_res);
        if (c->ws->h_flags) cudaFreeHost(c->ws->h_flags);
        if (c->ws->xdf) cudaFree(c->ws->xdf);
        if (c->ws->ydf) cudaFree(c->ws->ydf);
        if (c->ws->loopctl) cudaFree(c->ws->loopctl);
        if (c->ws->h_loopctl) cudaFreeHost(c->ws->h_loopctl);
        if (c->ws->ppart) cudaFree(c->ws->ppart);
        if (c->ws->pscal) cudaFree(c->ws->pscal);
        if (c->ws->pbar) cudaFree(c->ws->pbar);
        if (c->ws->perr) cudaFree(c->ws->perr);
        if (c->ws->h_perr) cudaFreeHost(c->ws->h_perr);
        delete c->ws;
        c->ws = nullptr;
    }
    void *ptrs[] = {c->dTab, c->fTab, c->bTab, c->dC, c->dD, c->dF, c->fD, c->dCD, c->dGN, c->dSamp, c->dCprev, c->dCprev2,
                    c->xD, c->xB, c->xTab, c->dGuess};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    c->dTab = nullptr;
    c->fTab = nullptr;
    c->bTab = nullptr;
    c->tab_bf16 = false;
    c->xD = c->xB = c->xTab = nullptr;
    c->xD_valid = false;
    c->dGuess = nullptr;
    c->has_guess = false;
    c->dC = c->dD = c->dF = c->dCD = c->dGN = c->dSamp = c->dCprev = c->dCprev2 = nullptr;
    c->hist = 0;
    ++c->state_gen;
    c->fD = nullptr;
}

int small_grid(int64_t n, const festung_ctx *c) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8));
}

// Copy an input array (host or device) into the device buffer dst and check finiteness.
int upload_checked(festung_ctx *c, const double *src, int loc, double *dst, int64_t n) {
    if (loc == FESTUNG_HOST)
        FCK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    else
        FCK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    int rc = ensure_ws(c);
    if (rc) return rc;
    FCK(cudaMemsetAsync(c->ws->d_flags, 0, sizeof(int), c->stream));
    k_check_finite<<<small_grid(n, c), 256, 0, c->stream>>>(dst, n, c->ws->d_flags); ++c->launches;
    FCK(cudaGetLastError());
    FCK(cudaMemcpyAsync(c->ws->h_flags, c->ws->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    FCK(cudaStreamSynchronize(c->stream));
    if (c->ws->h_flags[0]) {
        c->err = "non-finite value in input";
        return FESTUNG_EDATA;
    }
    return FESTUNG_OK;
}

// project K x R2 samples into out (N x K); flags: bit0 non-finite, bit1 non-positive, bit2 non-constant
int project_samples(festung_ctx *c, const double *samples, int loc, double *out, float *out32, int check_pos,
                    int *flags_out) {
    int rc = ensure_ws(c);
    if (rc) return rc;
    const int64_t n = c->K * c->R2;
    const double *src = samples;
    if (loc == FESTUNG_HOST) {
        FCK(cudaMemcpyAsync(c->dSamp, samples, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        src = c->dSamp;
    }
    FCK(cudaMemsetAsync(c->ws->d_flags, 0, sizeof(int), c->stream));
    const TableOffsets o = table_offsets(c->N, c->R2, c->R1);
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value;
        k_project<N, R2><<<elem_grid(c), 256, 0, c->stream>>>(src, out, out32, c->dTab + o.wphiQ, c->K, check_pos,
                                                             c->dPerm, c->ws->d_flags);
    });
    ++c->launches;
    FCK(cudaGetLastError());
    FCK(cudaMemcpyAsync(c->ws->h_flags, c->ws->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    FCK(cudaStreamSynchronize(c->stream));
    *flags_out = c->ws->h_flags[0];
    return FESTUNG_OK;
}

bool ready(festung_ctx *c) {
    if (!c) return false;
    if (c->p < 0) {
        c->err = "festung_setup has not been called";
        return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Krylov drivers
// ---------------------------------------------------------------------------
constexpr int CHUNK = 16;  // iterations per pass of the captured loop body

// The Krylov iterations of a solve run as one CUDA graph: a conditional while-node whose
// body is CHUNK iterations followed by k_loop_cond, which continues the loop while the
// iteration is not done and fewer than ctl[1] passes have run.  The bound ends the loop
// whatever the iteration does.
__global__ void k_loop_init(int *ctl, int max_chunks) {
    ctl[0] = 0;
    ctl[1] = max_chunks;
}

__global__ void k_loop_cond(cudaGraphConditionalHandle h, const KScal *sc, int *ctl) {
    const int n = ++ctl[0];
    cudaGraphSetConditional(h, (!sc->done && n < ctl[1]) ? 1u : 0u);
}

// preconditioned update kernels (templated on N)
// s = r - alpha v, sh = P^{-1} s, (s, s)
template <typename T>
void launch_bicg_s(festung_ctx *c, cudaStream_t st) {
    Workspace &w = *c->ws;
    Vecs<T> &V = vecs<T>(c);
    const __nv_bfloat16 *P = w.use_P ? w.Pb : nullptr;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto, auto) {
        constexpr int N = decltype(n_)::value;
        k_bicg_s<T, N><<<w.nblk, RED_THREADS, 0, st>>>((int)c->K, V.r, V.s, V.v, V.sh, P, V.inv, w.part, w.scal,
                                                       w.counter);
    });
    ++c->launches;
}

// the owed update of x and r, p = r + beta (p - omega v), ph = P^{-1} p
template <typename T>
void launch_bicg_next(festung_ctx *c, cudaStream_t st) {
    Workspace &w = *c->ws;
    Vecs<T> &V = vecs<T>(c);
    const __nv_bfloat16 *P = w.use_P ? w.Pb : nullptr;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto, auto) {
        constexpr int N = decltype(n_)::value;
        k_bicg_next<T, N><<<w.nblk, RED_THREADS, 0, st>>>((int)c->K, V.x, V.ph, V.sh, V.s, V.t, V.r, V.p, V.v, P,
                                                          V.inv, w.scal);
    });
    ++c->launches;
}

}  // namespace

namespace festung {

template <>
void launch_apply_bicg<double>(const festung_ctx *c, const double *x, double *y, double tau, int epi,
                               const double *e1, const double *e2, double *part, KScal *sc, unsigned int *counter,
                               const int *skip, cudaStream_t st, const BatchView &) {
    launch_apply<double>(c, x, y, nullptr, nullptr, tau, skip, st);
    const int g = c->ws->nblk;
    const int64_t n = c->K * c->N;
    if (epi == FUSED_EPI_ALPHA)
        k_bicg_epi<double, 1><<<g, RED_THREADS, 0, st>>>(n, y, e1, e2, part, sc, counter);
    else
        k_bicg_epi<double, 2><<<g, RED_THREADS, 0, st>>>(n, y, e1, e2, part, sc, counter);
    ++c->launches;
}

}  // namespace festung

namespace {

template <typename T>
void launch_cg_prec(festung_ctx *c, const T *r, T *z, int init, cudaStream_t st) {
    Workspace &w = *c->ws;
    const __nv_bfloat16 *P = w.use_P ? w.Pb : nullptr;
    const T *inv = vecs<T>(c).inv;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto, auto) {
        constexpr int N = decltype(n_)::value;
        k_cg_prec<T, N><<<w.nblk, RED_THREADS, 0, st>>>((int)c->K, r, z, P, inv, w.part, w.part2, w.nblk, w.scal,
                                                        w.counter, init);
    });
}

// record `CHUNK` iterations of the solver on stream st
template <typename T>
void record_iterations(festung_ctx *c, int solver, T tau, cudaStream_t st) {
    Workspace &w = *c->ws;
    Vecs<T> &V = vecs<T>(c);
    const int64_t n = c->K * c->N;
    const int g = w.nblk;
    const int *skip = &w.scal->done;
    for (int it = 0; it < CHUNK; ++it) {
        if (solver == FESTUNG_SOLVER_BICGSTAB) {
            // four launches per iteration: the reductions ride on the applies, and the
            // updates of x and r on the next iteration's first kernel
            launch_bicg_next<T>(c, st);                                          // (x, r), p, ph = P^{-1} p
            launch_apply_bicg<T>(c, V.ph, V.v, tau, FUSED_EPI_ALPHA, V.r0, nullptr, w.part, w.scal, w.counter,
                                 skip, st);                                      // v = S ph, alpha
            launch_bicg_s<T>(c, st);                                             // s, sh = P^{-1} s
            launch_apply_bicg<T>(c, V.sh, V.t, tau, FUSED_EPI_OMEGA, V.s, V.r0, w.part, w.scal, w.counter,
                                 skip, st);                                      // t = S sh, omega, beta
        } else {
            // CG: p (search), v = S p, s = z
            launch_apply<T>(c, V.p, V.v, V.Z1, V.Z2, tau, skip, st);
            k_cg_alpha<T><<<g, RED_THREADS, 0, st>>>(n, V.p, V.v, w.part, w.scal, w.counter);
            k_cg_xr<T><<<g, RED_THREADS, 0, st>>>(n, V.x, V.p, V.v, V.r, w.part2, w.scal);
            launch_cg_prec<T>(c, V.r, V.s, 0, st);
            k_cg_p<T><<<g, RED_THREADS, 0, st>>>(n, V.p, V.s, w.scal, 0);
        }
    }
}

template <typename T>
GraphCache &graph_of(festung_ctx *c);
template <>
GraphCache &graph_of<double>(festung_ctx *c) { return c->ws->g64; }
template <>
GraphCache &graph_of<float>(festung_ctx *c) { return c->ws->g32; }

// Solve S x = b (vectors V.x, V.b of precision T) to ||r|| <= tol ||b||.
// x_zero: x is 0 on entry.  Returns iterations in *iters and the final recursive ||r||^2, ||b||^2.
template <typename T>
int krylov_solve(festung_ctx *c, int solver, double tau, double tol, int max_iter, bool x_zero, int *iters,
                 double *r2, double *b2, bool *conv, bool reweight = false, double *relres0 = nullptr) {
    Workspace &w = *c->ws;
    Vecs<T> &V = vecs<T>(c);
    const int64_t K = c->K;
    const int N = c->N, g = w.nblk;
    cudaStream_t st = c->stream;
    int total = 0;
    *conv = false;
    for (int restart = 0; restart < 8; ++restart) {
        // r = b - S x
        if (x_zero && restart == 0) {
            k_kr_init<T><<<g, RED_THREADS, 0, st>>>(K, N, V.b, nullptr, V.r, V.r0, V.p, V.v, w.part, reweight ? 1 : 0);
            ++c->launches;
        } else {
            launch_apply<T>(c, V.x, V.t, V.Z1, V.Z2, (T)tau, nullptr, st);
            k_kr_init<T><<<g, RED_THREADS, 0, st>>>(K, N, V.b, V.t, V.r, V.r0, V.p, V.v, w.part,
                                                    (restart > 0 || reweight) ? 1 : 0);
            ++c->launches;
        }
        k_fin_init<<<1, 1024, 0, st>>>(w.scal, w.part, g, tol); ++c->launches;
        if (solver == FESTUNG_SOLVER_CG) {
            launch_cg_prec<T>(c, V.r, V.s, 1, st);                    // z = P^{-1} r, rho = (r, z)
            k_cg_p<T><<<g, RED_THREADS, 0, st>>>(K * N, V.p, V.s, w.scal, 1);  // p = z
            c->launches += 2;
        }
        FCK(cudaGetLastError());
        // FP32 BiCGStab at p <= 1: the iterations as one persistent kernel (bicg_persist.cu)
        bool persistent = std::is_same<T, float>::value && solver == FESTUNG_SOLVER_BICGSTAB && c->persistent &&
                          !c->persist_refused && w.ppart && bicg_persistent_supported(c);
        // else build (or reuse) the graph: while (not done and under the bound) { CHUNK iterations }
        GraphCache &gc = graph_of<T>(c);
        auto build_graph = [&]() -> int {
            if (gc.exec && gc.solver == solver && gc.tau == tau && gc.use_P == (int)w.use_P && gc.mass == c->mass &&
                gc.tab_bf16 == (int)c->tab_bf16)
                return FESTUNG_OK;
            if (gc.exec) cudaGraphExecDestroy(gc.exec);
            gc.exec = nullptr;
            cudaGraph_t graph;
            FCK(cudaGraphCreate(&graph, 0));
            cudaGraphConditionalHandle handle;
            cudaGraphNodeParams cp = {};
            cudaGraphNode_t node;
            cudaStream_t cs = nullptr;
            cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
            if (e == cudaSuccess) {
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = handle;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
            }
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            const int64_t saved = c->launches;
            if (e == cudaSuccess)
                e = cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                record_iterations<T>(c, solver, (T)tau, cs);
                k_loop_cond<<<1, 1, 0, cs>>>(handle, w.scal, w.loopctl);
                cudaGraph_t body = nullptr;
                e = cudaStreamEndCapture(cs, &body);
            }
            gc.nodes = c->launches - saved + 1;  // kernels per pass of the body
            c->launches = saved;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&gc.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (cs) cudaStreamDestroy(cs);
            FCK(e);
            gc.solver = solver;
            gc.tau = tau;
            gc.use_P = (int)w.use_P;
            gc.mass = c->mass;
            gc.tab_bf16 = (int)c->tab_bf16;
            return FESTUNG_OK;
        };
        int rc = persistent ? FESTUNG_OK : build_graph();
        if (rc) return rc;
        bool brk = false, drift = false;
        while (true) {
            FCK(cudaMemcpyAsync(w.h_scal, w.scal, sizeof(KScal), cudaMemcpyDeviceToHost, st));
            FCK(cudaStreamSynchronize(st));
            const KScal h = *w.h_scal;
            if (relres0 && restart == 0) *relres0 = h.b2 > 0 ? std::sqrt(h.r2_0 / h.b2) : std::sqrt(h.r2_0);
            if (h.done) {
                if (h.sconv) {
                    k_axpy_alpha<T><<<g, RED_THREADS, 0, st>>>(K, N, V.x, V.ph, w.scal); ++c->launches;
                    FCK(cudaGetLastError());
                } else if (h.pending) {
                    k_bicg_finish<T><<<g, RED_THREADS, 0, st>>>(K * N, V.x, V.ph, V.sh, w.scal); ++c->launches;
                    FCK(cudaGetLastError());
                }
                total += h.iter;
                *r2 = h.r2;
                *b2 = h.b2;
                if (h.breakdown) {
                    brk = true;
                } else {
                    // the recursively updated residual can drift from b - S x in low
                    // precision: check the true residual and restart if it is off by > 10x
                    launch_apply<T>(c, V.x, V.t, V.Z1, V.Z2, (T)tau, nullptr, st);
                    k_residual<T><<<g, RED_THREADS, 0, st>>>(K, N, V.b, V.t, w.part); ++c->launches;
                    k_fin_sums<<<1, 1024, 0, st>>>(w.res, w.part, g, 2); ++c->launches;
                    FCK(cudaMemcpyAsync(w.h_res, w.res, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
                    FCK(cudaStreamSynchronize(st));
                    const double tr2 = w.h_res[0], tb2 = w.h_res[1];
                    if (tr2 <= 100.0 * tol * tol * tb2 || restart >= 3) {
                        *conv = tr2 <= 100.0 * tol * tol * tb2;
                        *r2 = tr2;
                    } else {
                        drift = true;
                    }
                }
                break;
            }
            if (total + h.iter >= max_iter) {
                if (h.pending) {
                    k_bicg_finish<T><<<g, RED_THREADS, 0, st>>>(K * N, V.x, V.ph, V.sh, w.scal); ++c->launches;
                    FCK(cudaGetLastError());
                }
                total += h.iter;
                *r2 = h.r2;
                *b2 = h.b2;
                *iters = total;
                return FESTUNG_OK;
            }
            if (persistent) {
                if constexpr (std::is_same<T, float>::value) {
                    // Z1, Z2 (not used by the fused applies) serve as the second p and v buffers
                    const BicgVecs32 bv{V.x, V.r, V.p, V.v, V.ph, V.s, V.sh, V.t, V.Z1, V.Z2, V.r0, V.inv};
                    const cudaError_t e = launch_bicg_persistent(c, bv, w.use_P ? w.Pb : nullptr, (float)tau, w.scal,
                                                                 w.pscal, w.ppart, w.pcap, w.pbar, w.perr, max_iter - total, st);
                    if (e == cudaErrorNotSupported || e == cudaErrorCooperativeLaunchTooLarge) {
                        // the device cannot hold the grid: this context keeps to the graph
                        (void)cudaGetLastError();
                        persistent = false;
                        c->persist_refused = true;
                        if ((rc = build_graph())) return rc;
                        continue;
                    }
                    FCK(e);
                    ++c->launches;
                    FCK(cudaMemcpyAsync(w.h_perr, w.perr, sizeof(int), cudaMemcpyDeviceToHost, st));
                    FCK(cudaStreamSynchronize(st));
                    if (*w.h_perr) {
                        c->err = "persistent BiCGStab kernel: a grid barrier wait gave up";
                        return FESTUNG_ECUDA;
                    }
                }
                continue;
            }
            const int max_chunks = std::max(1, (max_iter - total - h.iter + CHUNK - 1) / CHUNK);
            k_loop_init<<<1, 1, 0, st>>>(w.loopctl, max_chunks); ++c->launches;
            FCK(cudaGraphLaunch(gc.exec, st));
            FCK(cudaMemcpyAsync(w.h_loopctl, w.loopctl, sizeof(int), cudaMemcpyDeviceToHost, st));
            FCK(cudaStreamSynchronize(st));
            c->launches += gc.nodes * (int64_t)*w.h_loopctl;
        }
        if (!brk && !drift) break;
        // breakdown or drift: restart from the current iterate
    }
    *iters = total;
    return FESTUNG_OK;
}

}  // namespace

namespace {

// y = S x in double-float arithmetic for an FP64 x (N x K): x is split into
// double-floats, the result is left in ws->ydf and, if y is given, written back as
// FP64.
int apply_df(festung_ctx *c, const double *x, double *y, double dt, cudaStream_t st) {
    Workspace &w = *c->ws;
    const int64_t KN = c->K * c->N;
    if (!w.xdf) FCK(cudaMalloc(&w.xdf, KN * sizeof(dfloat)));
    if (!w.ydf) FCK(cudaMalloc(&w.ydf, KN * sizeof(dfloat)));
    if (!c->xD_valid) {
        k_to_df<<<small_grid(KN, c), 256, 0, st>>>(KN, c->dD, c->xD); ++c->launches;
        c->xD_valid = true;
    }
    k_to_df<<<small_grid(KN, c), 256, 0, st>>>(KN, x, w.xdf); ++c->launches;
    launch_apply_df(c, w.xdf, w.ydf, dt, st);
    if (y) {
        k_from_df<<<small_grid(KN, c), 256, 0, st>>>(KN, w.ydf, y); ++c->launches;
    }
    FCK(cudaGetLastError());
    return FESTUNG_OK;
}

cudaError_t retile(festung_ctx *c, int te);

// Device copies of a mesh in internal order (geometry in FP64 and FP32, neighbour
// codes, permutation, lift flags) and a first tiling of 256 triangles.
cudaError_t upload_mesh(festung_ctx *c, const MeshOrder &mo) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t K = c->K;
    if ((e = cudaMalloc(&c->dB, 4 * K * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&c->fB, 4 * K * sizeof(float))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&c->dNbr, 3 * K * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&c->dPerm, K * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&c->dSlot, 3 * K * sizeof(int16_t))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&c->dLift, K * sizeof(uint8_t))) != cudaSuccess) return e;
    std::vector<float> fB(mo.B.begin(), mo.B.end());
    const struct {
        void *dst;
        const void *src;
        size_t bytes;
    } up[] = {{c->dB, mo.B.data(), 4 * K * sizeof(double)},
              {c->fB, fB.data(), 4 * K * sizeof(float)},
              {c->dNbr, mo.nbr.data(), 3 * K * sizeof(int32_t)},
              {c->dPerm, mo.perm.data(), K * sizeof(int32_t)},
              {c->dLift, mo.lift.data(), K * sizeof(uint8_t)}};
    for (const auto &u : up)
        if (u.bytes && (e = cudaMemcpy(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    return retile(c, 256);
}

// Tiles of te consecutive triangles of the internal order: halo lists and the
// shared-memory slots of every neighbour, uploaded to the device (the previous tiling
// is released on success).
cudaError_t retile(festung_ctx *c, int te) {
    MeshOrder mo;
    tile_mesh(c->hNbrInt, c->K, te, mo);
    const int64_t K = c->K, T = (K + te - 1) / te;
    std::vector<int16_t> slot16(mo.slot.begin(), mo.slot.end());
    std::vector<int16_t> hslot16(mo.halo_slot.begin(), mo.halo_slot.end());
    int32_t *hp = nullptr, *h = nullptr;
    int16_t *hs = nullptr;
    cudaError_t e;
    auto undo = [&](cudaError_t err) {
        cudaFree(hp);
        cudaFree(h);
        cudaFree(hs);
        return err;
    };
    if ((e = cudaMalloc(&hp, (T + 1) * sizeof(int32_t))) != cudaSuccess) return undo(e);
    if ((e = cudaMalloc(&h, std::max<size_t>(1, mo.halo.size()) * sizeof(int32_t))) != cudaSuccess) return undo(e);
    if ((e = cudaMalloc(&hs, std::max<size_t>(1, hslot16.size()) * sizeof(int16_t))) != cudaSuccess) return undo(e);
    if ((e = cudaMemcpy(hp, mo.halo_ptr.data(), (T + 1) * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess)
        return undo(e);
    if (!mo.halo.empty() &&
        (e = cudaMemcpy(h, mo.halo.data(), mo.halo.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess)
        return undo(e);
    if (!hslot16.empty() &&
        (e = cudaMemcpy(hs, hslot16.data(), hslot16.size() * sizeof(int16_t), cudaMemcpyHostToDevice)) != cudaSuccess)
        return undo(e);
    if ((e = cudaMemcpy(c->dSlot, slot16.data(), 3 * K * sizeof(int16_t), cudaMemcpyHostToDevice)) != cudaSuccess)
        return undo(e);
    cudaFree(c->dHaloPtr);
    cudaFree(c->dHalo);
    cudaFree(c->dHaloSlot);
    c->dHaloPtr = hp;
    c->dHalo = h;
    c->dHaloSlot = hs;
    c->TE = te;
    c->max_halo = mo.max_halo;
    c->nslot = te + mo.max_halo;
    // halo threads: whole warps for the largest halo, at least one warp, at most the
    // kernels' 320 threads in all (more halo slots are taken in turns)
    const int hw = std::min(std::max(32, ((mo.max_halo + 31) / 32) * 32), 320 - te);
    c->fthreads = te + std::max(32, hw);
    return cudaSuccess;
}

// Tile size for the kernels of the context's order: whole waves of the FP32 fused
// apply's resident blocks, and small enough that the FP64 kernel's traces fit in the
// shared memory of one block.
int choose_tiles(festung_ctx *c) {
    int dev = 0, optin = 0;
    FCK(cudaGetDevice(&dev));
    FCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int resident = fused_resident_blocks(c, c->nslot);
    int te = tile_size(c->K, resident, c->num_sms);
    for (;;) {
        if (te != c->TE) FCK(retile(c, te));
        // static shared memory of the kernels (tables) stays below 16 KB
        if (fused_smem_bytes(c, c->nslot, true) + 16384 <= (size_t)optin || te <= 32) break;
        te = std::max(32, ((te / 2 + 31) / 32) * 32);
    }
    if (fused_smem_bytes(c, c->nslot, true) + 16384 > (size_t)optin) {
        c->err = "mesh tiles need more shared memory than a block has (halo of " + std::to_string(c->max_halo) +
                 " triangles)";
        return FESTUNG_EMESH;
    }
    return FESTUNG_OK;
}

// Time the FP32 fused apply for tile sizes 96..256 (multiples of 32) around the
// heuristic choice and keep the fastest.  Tiles that would not fit the FP64 traces in a
// block's shared memory are skipped.  Only speed depends on the tiling.
int autotune_tiles(festung_ctx *c, int *chosen) {
    int rc = ensure_ws(c);
    if (rc) return rc;
    int dev = 0, optin = 0;
    FCK(cudaGetDevice(&dev));
    FCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int64_t KN = c->K * c->N;
    float *x = nullptr, *y = nullptr;
    FCK(cudaMalloc(&x, KN * sizeof(float)));
    cudaError_t e = cudaMalloc(&y, KN * sizeof(float));
    if (e != cudaSuccess) {
        cudaFree(x);
        FCK(e);
    }
    cudaStream_t st = c->stream;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaMemsetAsync(x, 0, KN * sizeof(float), st);
    const int64_t saved = c->launches;
    int best = c->TE;
    float best_ms = 1e30f;
    for (int te = 96; te <= 256; te += 32) {
        if ((e = retile(c, te)) != cudaSuccess) break;
        if (fused_smem_bytes(c, c->nslot, true) + 16384 > (size_t)optin) continue;
        launch_apply<float>(c, x, y, nullptr, nullptr, 1e-3f, nullptr, st);
        cudaEventRecord(a, st);
        for (int r = 0; r < 5; ++r) launch_apply<float>(c, x, y, nullptr, nullptr, 1e-3f, nullptr, st);
        cudaEventRecord(b, st);
        if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_ms) {
            best_ms = ms;
            best = te;
        }
    }
    c->launches = saved;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(x);
    cudaFree(y);
    FCK(e);
    FCK(retile(c, best));
    reset_graphs(c);  // captured iterations hold the old tiling
    if (chosen) *chosen = best;
    return FESTUNG_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int festung_autotune(festung_ctx *c, int *tile) {
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    return autotune_tiles(c, tile);
}

int festung_mesh_create(const double *coordV, int64_t numV, const int32_t *V0T, int64_t numT,
                        const int8_t *bdr_type, festung_ctx **out) {
    g_create_err.clear();
    if (!out) {
        g_create_err = "out is NULL";
        return FESTUNG_EINVAL;
    }
    *out = nullptr;
    if (!coordV || !V0T || !bdr_type || numV < 3 || numT < 1) {
        g_create_err = "NULL array or empty mesh";
        return FESTUNG_EINVAL;
    }
    festung_ctx *c = new (std::nothrow) festung_ctx();
    if (!c) return FESTUNG_ENOMEM;
    c->K = numT;
    c->numV = numV;
    std::vector<int32_t> nbr;
    int rc = build_mesh(coordV, numV, V0T, numT, bdr_type, c->hB, nbr, c->err);
    if (rc) {
        g_create_err = c->err;
        delete c;
        return rc;
    }
    c->coordV.assign(coordV, coordV + 2 * numV);
    c->V0T.assign(V0T, V0T + 3 * numT);
    c->bdr.assign(bdr_type, bdr_type + 3 * numT);
    for (int64_t i = 0; i < 3 * numT; ++i) {
        if (bdr_type[i] == FESTUNG_BDR_DIRICHLET) c->has_dirichlet = true;
        if (bdr_type[i] == FESTUNG_BDR_NEUMANN) c->has_neumann = true;
    }
    // internal order: Morton order of centroids; tiles of 256 triangles until
    // festung_setup sizes them for the kernels of the chosen order
    MeshOrder mo;
    order_mesh(coordV, V0T, numT, c->hB, nbr, mo);
    c->perm = mo.perm;
    c->hNbrInt = mo.nbr;
    auto fail = [&](cudaError_t e) {
        g_create_err = std::string("CUDA: ") + cudaGetErrorString(e);
        festung_destroy(c);
        return e == cudaErrorMemoryAllocation ? FESTUNG_ENOMEM : FESTUNG_ECUDA;
    };
    cudaError_t e = upload_mesh(c, mo);
    if (e != cudaSuccess) return fail(e);
    *out = c;
    return FESTUNG_OK;
}

int festung_setup(festung_ctx *c, int p, int quad_order, double eta) {
    if (!c) return FESTUNG_EINVAL;
    if (p < 0 || p > PMAX) {
        c->err = "p must be in 0..4";
        return FESTUNG_EINVAL;
    }
    if (!(eta > 0.0) || !std::isfinite(eta)) {
        c->err = "eta must be positive";
        return FESTUNG_EINVAL;
    }
    int qT = quad_order == 0 ? std::max(1, 2 * p) : quad_order;
    if (quad_order != 0 && !(quad_order == 2 * p || quad_order == 2 * p + 1 || (p == 0 && quad_order == 1))) {
        c->err = "quad_order must be 0, 2p or 2p+1";
        return FESTUNG_EINVAL;
    }
    if (c->K * (int64_t)num_dofs(p) >= (int64_t(1) << 31)) {
        c->err = "K * N must stay below 2^31";
        return FESTUNG_EINVAL;
    }
    HostTables T;
    try {
        build_tables(p, qT, T);
    } catch (const std::exception &ex) {
        c->err = std::string("reference tables: ") + ex.what();
        return FESTUNG_EINVAL;
    }
    if (!dispatch(T.N, T.R2, T.R1, [](auto, auto, auto) {})) {
        c->err = "unsupported quadrature combination";
        return FESTUNG_EINVAL;
    }
    // release previous order-dependent buffers
    free_ctx_device(c);
    c->p = p;
    c->N = T.N;
    c->R2 = T.R2;
    c->R1 = T.R1;
    c->qT = qT;
    c->eta = eta;
    c->tab = T;
    const TableOffsets o = table_offsets(T.N, T.R2, T.R1);
    std::vector<double> h(o.total, 0.0);
    std::copy(T.phiQ.begin(), T.phiQ.end(), h.begin() + o.phiQ);
    std::copy(T.wphiQ.begin(), T.wphiQ.end(), h.begin() + o.wphiQ);
    std::copy(T.gw1.begin(), T.gw1.end(), h.begin() + o.gw1);
    std::copy(T.gw2.begin(), T.gw2.end(), h.begin() + o.gw2);
    std::copy(T.H1.begin(), T.H1.end(), h.begin() + o.H1);
    std::copy(T.H2.begin(), T.H2.end(), h.begin() + o.H2);
    std::copy(T.phiE.begin(), T.phiE.end(), h.begin() + o.phiE);
    std::copy(T.wphiE.begin(), T.wphiE.end(), h.begin() + o.wphiE);
    std::vector<float> hf(h.begin(), h.end());
    std::vector<float> hb(h.size());
    for (size_t i = 0; i < h.size(); ++i) hb[i] = round_to_bf16(h[i]);
    const int64_t K = c->K, N = c->N;
    FCK(cudaMalloc(&c->dTab, o.total * sizeof(double)));
    FCK(cudaMalloc(&c->fTab, o.total * sizeof(float)));
    FCK(cudaMemcpy(c->dTab, h.data(), o.total * sizeof(double), cudaMemcpyHostToDevice));
    FCK(cudaMemcpy(c->fTab, hf.data(), o.total * sizeof(float), cudaMemcpyHostToDevice));
    FCK(cudaMalloc(&c->bTab, o.total * sizeof(float)));
    FCK(cudaMemcpy(c->bTab, hb.data(), o.total * sizeof(float), cudaMemcpyHostToDevice));
    FCK(upload_tables_f64(c));
    FCK(upload_tables_df(c));
    {
        // double-float copies of the tables and the geometry (residual applies)
        std::vector<dfloat> hx(o.total);
        for (int i = 0; i < o.total; ++i) hx[i] = dfloat(h[i]);
        FCK(cudaMalloc(&c->xTab, o.total * sizeof(dfloat)));
        FCK(cudaMemcpy(c->xTab, hx.data(), o.total * sizeof(dfloat), cudaMemcpyHostToDevice));
        FCK(cudaMalloc(&c->xB, 4 * c->K * sizeof(dfloat)));
        k_to_df<<<small_grid(4 * c->K, c), 256>>>(4 * c->K, c->dB, c->xB); ++c->launches;
        FCK(cudaGetLastError());
        FCK(cudaMalloc(&c->xD, c->K * c->N * sizeof(dfloat)));
        c->xD_valid = false;
    }
    if (int rc = choose_tiles(c)) return rc;
    FCK(cudaMalloc(&c->dC, K * N * sizeof(double)));
    FCK(cudaMalloc(&c->dD, K * N * sizeof(double)));
    FCK(cudaMalloc(&c->fD, K * N * sizeof(float)));
    FCK(cudaMalloc(&c->dF, K * N * sizeof(double)));
    FCK(cudaMalloc(&c->dCD, K * 3 * c->R1 * sizeof(double)));
    FCK(cudaMalloc(&c->dGN, K * 3 * c->R1 * sizeof(double)));
    FCK(cudaMalloc(&c->dSamp, K * c->R2 * sizeof(double)));
    FCK(cudaMemset(c->dC, 0, K * N * sizeof(double)));
    FCK(cudaMemset(c->dF, 0, K * N * sizeof(double)));
    FCK(cudaMemset(c->dCD, 0, K * 3 * c->R1 * sizeof(double)));
    FCK(cudaMemset(c->dGN, 0, K * 3 * c->R1 * sizeof(double)));
    // D = projection of d = 1: only the first mode, 1 / phi_1 = 1/sqrt(2)
    std::vector<double> ones((size_t)K * c->R2, 1.0);
    FCK(cudaMemcpy(c->dSamp, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice));
    int flags = 0;
    int rc = project_samples(c, c->dSamp, FESTUNG_DEVICE, c->dD, c->fD, 1, &flags);
    if (rc) return rc;
    c->symmetric = true;
    c->source_zero = true;
    c->bc_zero = true;
    return FESTUNG_OK;
}

int festung_sizes(const festung_ctx *c, int64_t *K, int *N, int *R2, int *R1) {
    if (!c) return FESTUNG_EINVAL;
    if (K) *K = c->K;
    if (N) *N = c->N;
    if (R2) *R2 = c->R2;
    if (R1) *R1 = c->R1;
    return FESTUNG_OK;
}

int festung_quad_points(const festung_ctx *cc, double *xy, double *exy) {
    festung_ctx *c = const_cast<festung_ctx *>(cc);
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    const int64_t K = c->K;
    const HostTables &T = c->tab;
    for (int64_t k = 0; k < K; ++k) {
        const double b11 = c->hB[k], b12 = c->hB[K + k], b21 = c->hB[2 * K + k], b22 = c->hB[3 * K + k];
        const double *a1 = &c->coordV[2 * (int64_t)c->V0T[3 * k]];
        if (xy)
            for (int r = 0; r < c->R2; ++r) {
                const double q1 = T.tri.x1[r], q2 = T.tri.x2[r];
                xy[(k * c->R2 + r) * 2 + 0] = b11 * q1 + b12 * q2 + a1[0];
                xy[(k * c->R2 + r) * 2 + 1] = b21 * q1 + b22 * q2 + a1[1];
            }
        if (exy)
            for (int n = 0; n < 3; ++n)
                for (int r = 0; r < c->R1; ++r) {
                    const double s = T.edge.s[r];
                    double q1 = 0, q2 = 0;
                    if (n == 0) { q1 = 1.0 - s; q2 = s; }
                    if (n == 1) { q1 = 0.0; q2 = 1.0 - s; }
                    if (n == 2) { q1 = s; q2 = 0.0; }
                    const int64_t o = ((k * 3 + n) * c->R1 + r) * 2;
                    exy[o + 0] = b11 * q1 + b12 * q2 + a1[0];
                    exy[o + 1] = b21 * q1 + b22 * q2 + a1[1];
                }
    }
    return FESTUNG_OK;
}

int festung_set_coeff(festung_ctx *c, const double *d_samples, int loc) {
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    if (!d_samples || (loc != FESTUNG_HOST && loc != FESTUNG_DEVICE)) {
        c->err = "d_samples is NULL or bad loc";
        return FESTUNG_EINVAL;
    }
    int rc = ensure_ws(c);
    if (rc) return rc;
    const int64_t KN = c->K * c->N;
    // project into scratch, validate, then commit (state unchanged on failure)
    Workspace &w = *c->ws;
    if (!w.scratch64) FCK(cudaMalloc(&w.scratch64, 2 * KN * sizeof(double)));
    int flags = 0;
    rc = project_samples(c, d_samples, loc, w.scratch64, nullptr, 1, &flags);
    if (rc) return rc;
    if (flags & 3) {
        c->err = (flags & 1) ? "non-finite diffusion sample" : "diffusion sample <= 0";
        return FESTUNG_EDATA;
    }
    k_commit_coeff<<<small_grid(KN, c), 256, 0, c->stream>>>(KN, w.scratch64, c->dD, c->fD); ++c->launches;
    FCK(cudaGetLastError());
    c->xD_valid = false;
    // S is symmetric iff d_h is elementwise constant (always so for p = 0)
    c->symmetric = (c->p == 0) || !(flags & 4);
    return FESTUNG_OK;
}

int festung_set_source(festung_ctx *c, const double *f_samples, int loc) {
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    if (!f_samples) {
        FCK(cudaMemsetAsync(c->dF, 0, c->K * c->N * sizeof(double), c->stream));
        c->source_zero = true;
        return FESTUNG_OK;
    }
    int rc = ensure_ws(c);
    if (rc) return rc;
    Workspace &w = *c->ws;
    if (!w.scratch64) FCK(cudaMalloc(&w.scratch64, 2 * c->K * c->N * sizeof(double)));
    int flags = 0;
    rc = project_samples(c, f_samples, loc, w.scratch64, nullptr, 0, &flags);
    if (rc) return rc;
    if (flags & 1) {
        c->err = "non-finite source sample";
        return FESTUNG_EDATA;
    }
    FCK(cudaMemcpyAsync(c->dF, w.scratch64, c->K * c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    c->source_zero = false;
    return FESTUNG_OK;
}

int festung_set_bc(festung_ctx *c, const double *cD, const double *gN, int loc) {
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    const int64_t n = c->K * 3 * c->R1;
    int rc;
    if (cD) {
        if ((rc = upload_checked(c, cD, loc, c->dCD, n))) return rc;
    } else {
        FCK(cudaMemsetAsync(c->dCD, 0, n * sizeof(double), c->stream));
    }
    if (gN) {
        if ((rc = upload_checked(c, gN, loc, c->dGN, n))) return rc;
    } else {
        FCK(cudaMemsetAsync(c->dGN, 0, n * sizeof(double), c->stream));
    }
    c->bc_zero = !cD && !gN;
    return FESTUNG_OK;
}

int festung_set_state(festung_ctx *c, const double *C, int is_samples, int loc) {
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    if (!C) {
        c->err = "C is NULL";
        return FESTUNG_EINVAL;
    }
    int rc = ensure_ws(c);
    if (rc) return rc;
    Workspace &w = *c->ws;
    const int64_t KN = c->K * c->N;
    if (!w.scratch64) FCK(cudaMalloc(&w.scratch64, 2 * KN * sizeof(double)));
    if (is_samples) {
        int flags = 0;
        rc = project_samples(c, C, loc, w.scratch64, nullptr, 0, &flags);
        if (rc) return rc;
        if (flags & 1) {
            c->err = "non-finite sample";
            return FESTUNG_EDATA;
        }
        FCK(cudaMemcpyAsync(c->dC, w.scratch64, KN * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    } else {
        double *tmp = w.scratch64 + KN;
        rc = upload_checked(c, C, loc, tmp, KN);
        if (rc) return rc;
        k_to_internal<<<small_grid(KN, c), 256, 0, c->stream>>>(tmp, c->dC, c->K, c->N, c->dPerm); ++c->launches;
        FCK(cudaGetLastError());
    }
    c->hist = 0;
    ++c->state_gen;
    c->has_guess = false;
    FCK(cudaStreamSynchronize(c->stream));
    return FESTUNG_OK;
}

int festung_get_state(const festung_ctx *cc, double *C, int loc) {
    festung_ctx *c = const_cast<festung_ctx *>(cc);
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    if (!C) {
        c->err = "C is NULL";
        return FESTUNG_EINVAL;
    }
    int rc = ensure_ws(c);
    if (rc) return rc;
    Workspace &w = *c->ws;
    const int64_t KN = c->K * c->N;
    if (!w.scratch64) FCK(cudaMalloc(&w.scratch64, 2 * KN * sizeof(double)));
    double *dst = (loc == FESTUNG_DEVICE) ? C : w.scratch64;
    k_to_public<<<small_grid(KN, c), 256, 0, c->stream>>>(c->dC, dst, c->K, c->N, c->dPerm); ++c->launches;
    FCK(cudaGetLastError());
    if (loc == FESTUNG_HOST)
        FCK(cudaMemcpyAsync(C, w.scratch64, KN * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    FCK(cudaStreamSynchronize(c->stream));
    return FESTUNG_OK;
}

int festung_apply(festung_ctx *c, const void *x, void *y, int prec, double dt) {
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    if (!x || !y || x == y || !(dt >= 0.0) ||
        (prec != FESTUNG_FP64 && prec != FESTUNG_FP32 && prec != FESTUNG_DFLOAT && prec != FESTUNG_BF16TAB)) {
        c->err = "bad apply arguments";
        return FESTUNG_EINVAL;
    }
    int rc = ensure_ws(c);
    if (rc) return rc;
    if (prec == FESTUNG_DFLOAT) {
        if ((rc = apply_df(c, (const double *)x, (double *)y, dt, c->stream))) return rc;
    } else if (prec == FESTUNG_FP64) {
        if ((rc = alloc_vecs<double>(c, c->ws->d, false))) return rc;
        launch_apply<double>(c, (const double *)x, (double *)y, c->ws->d.Z1, c->ws->d.Z2, dt, nullptr, c->stream);
    } else {
        if ((rc = alloc_vecs<float>(c, c->ws->f, false))) return rc;
        c->tab_bf16 = prec == FESTUNG_BF16TAB;
        launch_apply<float>(c, (const float *)x, (float *)y, c->ws->f.Z1, c->ws->f.Z2, (float)dt, nullptr,
                            c->stream);
        c->tab_bf16 = false;
    }
    FCK(cudaGetLastError());
    return FESTUNG_OK;
}

}  // extern "C"

namespace {

// Solve (mass M + dt (eta S_t - sum_m A_m M^{-1} B_m)) C = b: an implicit-Euler step
// (mass = 1, E1-E2) or the stationary problem of Sec. 3.9 (mass = 0, dt = 1).
// Step options with the defaults of festung_step; false if out of range.
bool step_options(const festung_step_opts *opts, festung_step_opts &o) {
    o.tol = 1e-10;
    o.max_iter = 20000;
    o.prec = FESTUNG_MIXED;
    o.inner_tol = 1e-2;
    o.max_outer = 50;
    o.solver = 0;
    if (opts) o = *opts;
    return o.tol > 0.0 && o.max_iter >= 1 &&
           (o.prec == FESTUNG_FP64 || o.prec == FESTUNG_MIXED || o.prec == FESTUNG_MIXED64 ||
            o.prec == FESTUNG_BF16TAB) &&
           o.max_outer >= 1 && o.inner_tol > 0.0 && o.inner_tol < 1.0 &&
           (o.solver == 0 || o.solver == FESTUNG_SOLVER_CG || o.solver == FESTUNG_SOLVER_BICGSTAB);
}

// Everything before the Krylov solve of a step: vectors, b (E2) into V.b (W^m of the
// Dirichlet lift left in scratch64), the block-Jacobi preconditioner, and the initial
// guess V.x extrapolated in time from the previous states.
int prepare_solve(festung_ctx *c, double dt, bool stationary, bool mixed) {
    int rc = ensure_ws(c);
    if (rc) return rc;
    Workspace &w = *c->ws;
    if ((rc = alloc_vecs<double>(c, w.d, true))) return rc;
    if (mixed && (rc = alloc_vecs<float>(c, w.f, true))) return rc;
    const int64_t KN = c->K * c->N;
    cudaStream_t st = c->stream;
    Vecs<double> &V = w.d;
    if (!w.scratch64) FCK(cudaMalloc(&w.scratch64, 2 * KN * sizeof(double)));
    // right-hand side b (E2): W^m = M^{-1} J_D^m, then b = M C^n + tau (M F + eta K_D - K_N + sum A_m W^m)
    double *W1 = w.scratch64, *W2 = w.scratch64 + KN;
    launch_rhs(c, W1, W2, V.b, dt, st);
    FCK(cudaGetLastError());
    // block-Jacobi preconditioner: inverse diagonal blocks of S for this D and dt, built on
    // a second stream while this one forms the guess and the first residual
    // (finish_precond joins it).  With festung_set_precond_reuse the blocks of an earlier
    // step serve while dt and the mass term are unchanged, the build is younger than the
    // reuse bound and the Krylov iterations have not grown much since the build (a lagged
    // preconditioner: S changes with D from step to step, the answer does not depend on P).
    c->P_built = !c->P_valid || c->P_dt != dt || c->P_mass != c->mass || c->P_age >= c->precond_reuse;
    if (c->P_built) {
        if (!w.P) FCK(cudaMalloc(&w.P, (size_t)c->N * c->N * c->K * sizeof(float)));
        if (!w.Pb) FCK(cudaMalloc(&w.Pb, (size_t)((c->N * c->N + 7) / 8) * c->K * 16));
        if (!c->side) {
            FCK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
            FCK(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
            FCK(cudaEventCreateWithFlags(&c->ev_P, cudaEventDisableTiming));
        }
        FCK(cudaEventRecord(c->ev_in, st));
        FCK(cudaStreamWaitEvent(c->side, c->ev_in, 0));
        FCK(cudaMemsetAsync(w.d_flags, 0, sizeof(int), c->side));
        launch_blockjacobi(c, w.P, w.Pb, dt, w.d_flags, c->side);
        FCK(cudaGetLastError());
        FCK(cudaEventRecord(c->ev_P, c->side));
        c->P_pending = true;
        c->P_valid = true;
        c->P_dt = dt;
        c->P_mass = c->mass;
        c->P_age = 0;
        c->P_iters0 = -1;
    }
    ++c->P_age;
    // initial guess: C^n plus a correction given with festung_set_guess, else
    // extrapolation in time from the previous states when they exist, else C^n (the
    // result does not depend on it beyond the tolerance)
    if (!stationary && c->has_guess) {
        k_extrapolate3<<<small_grid(KN, c), 256, 0, st>>>(KN, c->dC, c->dGuess, c->dGuess, V.x, 1.0, 1.0, 0.0);
        ++c->launches;
        c->has_guess = false;
    } else if (!stationary && c->hist >= 2 && c->dt_prev > 0.0 && c->dt_prev2 > 0.0) {
        // quadratic Lagrange extrapolation through t_{n-2}, t_{n-1}, t_n to t_{n+1}
        const double h0 = c->dt_prev2, h1 = c->dt_prev, h = dt;  // t_n - t_{n-1} = h1, t_{n-1} - t_{n-2} = h0
        const double tn = 0.0, tm1 = -h1, tm2 = -h1 - h0, tp = h;
        const double l0 = (tp - tm1) * (tp - tm2) / ((tn - tm1) * (tn - tm2));
        const double l1 = (tp - tn) * (tp - tm2) / ((tm1 - tn) * (tm1 - tm2));
        const double l2 = (tp - tn) * (tp - tm1) / ((tm2 - tn) * (tm2 - tm1));
        k_extrapolate3<<<small_grid(KN, c), 256, 0, st>>>(KN, c->dC, c->dCprev, c->dCprev2, V.x, l0, l1, l2);
        ++c->launches;
    } else if (!stationary && c->hist >= 1 && c->dt_prev > 0.0) {
        k_extrapolate<<<small_grid(KN, c), 256, 0, st>>>(KN, c->dC, c->dCprev, V.x, dt / c->dt_prev); ++c->launches;
    } else {
        FCK(cudaMemcpyAsync(V.x, c->dC, KN * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    return FESTUNG_OK;
}

// Join the preconditioner build of prepare_solve: the main stream waits for it, and the
// blocks are used unless one was singular.
int finish_precond(festung_ctx *c) {
    if (!c->P_pending) return FESTUNG_OK;
    Workspace &w = *c->ws;
    cudaStream_t st = c->stream;
    FCK(cudaStreamWaitEvent(st, c->ev_P, 0));
    FCK(cudaMemcpyAsync(w.h_flags, w.d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    FCK(cudaStreamSynchronize(st));
    w.use_P = (w.h_flags[0] == 0);
    c->P_pending = false;
    return FESTUNG_OK;
}

// C <- V.x after a converged solve; a time step also shifts the history of previous
// states for the next extrapolation.
int commit_solution(festung_ctx *c, double dt, bool stationary) {
    Workspace &w = *c->ws;
    const int64_t KN = c->K * c->N;
    cudaStream_t st = c->stream;
    if (stationary) {
        FCK(cudaMemcpyAsync(c->dC, w.d.x, KN * sizeof(double), cudaMemcpyDeviceToDevice, st));
        FCK(cudaStreamSynchronize(st));
        c->hist = 0;  // a stationary solve is no time step: the extrapolation restarts
        ++c->state_gen;
        return FESTUNG_OK;
    }
    if (!c->dCprev) FCK(cudaMalloc(&c->dCprev, KN * sizeof(double)));
    if (!c->dCprev2) FCK(cudaMalloc(&c->dCprev2, KN * sizeof(double)));
    std::swap(c->dCprev, c->dCprev2);  // C^{n-2} <- C^{n-1}
    FCK(cudaMemcpyAsync(c->dCprev, c->dC, KN * sizeof(double), cudaMemcpyDeviceToDevice, st));
    FCK(cudaMemcpyAsync(c->dC, w.d.x, KN * sizeof(double), cudaMemcpyDeviceToDevice, st));
    FCK(cudaStreamSynchronize(st));
    c->hist = std::min(c->hist + 1, 2);
    c->dt_prev2 = c->dt_prev;
    c->dt_prev = dt;
    ++c->state_gen;
    return FESTUNG_OK;
}

// The p = 1 problem of the coarse correction, for this step: built at first use from the
// context's mesh (the same internal order, checked), its d_h the P1 part of ours (the first
// three coefficients: the basis is hierarchical and orthonormal), the same mass term, its
// block-Jacobi preconditioner for dt.
int prepare_coarse(festung_ctx *c, double dt) {
    cudaStream_t st = c->stream;
    if (!c->coarse) {
        c->coarse_warm = false;
        festung_ctx *cc = nullptr;
        int rc = festung_mesh_create(c->coordV.data(), c->numV, c->V0T.data(), c->K, c->bdr.data(), &cc);
        if (rc == FESTUNG_OK) rc = festung_setup(cc, 1, 0, c->eta);
        if (rc == FESTUNG_OK && cc->perm != c->perm) rc = FESTUNG_EMESH;
        if (rc != FESTUNG_OK) {
            c->err = std::string("coarse problem: ") + (cc ? cc->err : festung_last_error(nullptr));
            festung_destroy(cc);
            return rc;
        }
        c->coarse = cc;
    }
    festung_ctx *cc = c->coarse;
    cc->stream = st;
    cc->persistent = c->persistent;
    cc->mass = c->mass;
    cc->symmetric = c->symmetric;
    int rc = ensure_ws(cc);
    if (rc) return rc;
    Workspace &w = *cc->ws;
    if ((rc = alloc_vecs<float>(cc, w.f, true))) return rc;
    const int64_t K3 = 3 * c->K;
    k_commit_coeff<<<small_grid(K3, c), 256, 0, st>>>(K3, c->dD, cc->dD, cc->fD); ++c->launches;
    cc->xD_valid = false;
    // the coarse blocks are rebuilt with the fine ones (festung_set_precond_reuse)
    if (w.P && !c->P_built && cc->P_dt == dt && cc->P_mass == c->mass) return FESTUNG_OK;
    cc->P_dt = dt;
    cc->P_mass = c->mass;
    if (!w.P) FCK(cudaMalloc(&w.P, (size_t)9 * cc->K * sizeof(float)));
    if (!w.Pb) FCK(cudaMalloc(&w.Pb, (size_t)((9 + 7) / 8) * cc->K * 16));
    FCK(cudaMemsetAsync(w.d_flags, 0, sizeof(int), st));
    launch_blockjacobi(cc, w.P, w.Pb, dt, w.d_flags, st);
    c->launches += 2;
    FCK(cudaGetLastError());
    FCK(cudaMemcpyAsync(w.h_flags, w.d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    FCK(cudaStreamSynchronize(st));
    w.use_P = (w.h_flags[0] == 0);
    return FESTUNG_OK;
}

int solve_system(festung_ctx *c, double dt, double mass, const festung_step_opts *opts, festung_step_info *info) {
    struct MassGuard {
        festung_ctx *c;
        ~MassGuard() {
            c->mass = 1.0;
            c->tab_bf16 = false;
        }
    } guard{c};
    c->mass = mass;
    const bool stationary = mass == 0.0;
    festung_step_opts o;
    if (!step_options(opts, o) || !(dt > 0.0)) {
        c->err = "bad step arguments";
        return FESTUNG_EINVAL;
    }
    int rc = prepare_solve(c, dt, stationary, o.prec != FESTUNG_FP64);
    if (rc) return rc;
    Workspace &w = *c->ws;
    const int solver = o.solver ? o.solver : (c->symmetric ? FESTUNG_SOLVER_CG : FESTUNG_SOLVER_BICGSTAB);
    const int64_t KN = c->K * c->N;
    cudaStream_t st = c->stream;
    Vecs<double> &V = w.d;
    double *W1 = w.scratch64;
    int iters = 0, outer = 0, iters64 = 0, coarse_iters = 0;
    const bool use_coarse = c->coarse_mode && c->p >= 2 && o.prec != FESTUNG_FP64;
    if (use_coarse && (rc = prepare_coarse(c, dt))) return rc;
    double r2 = 0, b2 = 0;
    bool conv = false;
    double relres = 0.0, relres0 = -1.0;
    // residual r = b - S x (FP64 vectors) and its norms (rn, bn)
    // (FESTUNG_MIXED: S x in double-float arithmetic, about 48 significant bits; the other
    // modes: S x in FP64)
    const bool df_residual = o.prec == FESTUNG_MIXED;
    auto residual64 = [&](double *rn, double *bn) -> int {
        if (df_residual) {
            if ((rc = apply_df(c, V.x, nullptr, dt, st))) return rc;
            k_residual_df<<<w.nblk, RED_THREADS, 0, st>>>(KN, V.b, w.ydf, V.r, w.part);
        } else {
            launch_apply<double>(c, V.x, V.t, V.Z1, V.Z2, dt, nullptr, st);
            k_residual64<<<w.nblk, RED_THREADS, 0, st>>>(KN, V.b, V.t, V.r, w.part);
        }
        k_fin_sums<<<1, 1024, 0, st>>>(W1, w.part, w.nblk, 2);
        c->launches += 2;
        double h[2];
        FCK(cudaMemcpyAsync(h, W1, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        FCK(cudaStreamSynchronize(st));
        *rn = std::sqrt(h[0]);
        *bn = std::sqrt(h[1]);
        return FESTUNG_OK;
    };
    bool fp64 = (o.prec == FESTUNG_FP64);
    if (!fp64) {
        // mixed precision: residual with S x in double-float arithmetic, FP32 inner solve of
        // S d = r / ||r||, C += ||r|| d.  An inner solve that does not lower the residual is
        // undone; after two such sweeps the step finishes in FP64.
        Vecs<float> &F = w.f;
        double prev_rn = -1.0, last_scale = 0.0;
        int failures = 0;
        bool applied = false;
        for (outer = 1; outer <= o.max_outer; ++outer) {
            double rn, bn;
            if ((rc = residual64(&rn, &bn))) return rc;
            if ((rc = finish_precond(c))) return rc;
            relres = bn > 0 ? rn / bn : rn;
            if (relres0 < 0.0) relres0 = relres;
            if (relres <= o.tol || rn == 0.0) {
                conv = true;
                break;
            }
            if (applied && !(rn < prev_rn)) {
                // the last sweep did not lower the residual: undo it
                k_add_f32<<<small_grid(KN, c), 256, 0, st>>>(KN, V.x, F.x, -last_scale); ++c->launches;
                applied = false;
                if (++failures >= 2) {
                    fp64 = true;
                    break;
                }
                if ((rc = residual64(&rn, &bn))) return rc;
                relres = bn > 0 ? rn / bn : rn;
            } else if (applied) {
                failures = 0;
            }
            if (iters >= o.max_iter) break;
            prev_rn = rn;
            k_scale_to_f32<<<small_grid(KN, c), 256, 0, st>>>(KN, V.r, F.b, 1.0 / rn); ++c->launches;
            k_zero_f32<<<small_grid(KN, c), 256, 0, st>>>(KN, F.x); ++c->launches;
            bool x_zero = true;
            if (use_coarse) {
                // coarse correction: the p = 1 problem for the P1 part of the right-hand side (the
                // first 3 K entries of the N x K layout), its solution as the sweep's start
                festung_ctx *cc = c->coarse;
                Vecs<float> &CF = cc->ws->f;
                const int64_t K3 = 3 * c->K;
                FCK(cudaMemcpyAsync(CF.b, F.b, K3 * sizeof(float), cudaMemcpyDeviceToDevice, st));
                int cit = 0;
                bool ccin = false;
                double cr2, cb2;
                const int csolver = cc->symmetric ? FESTUNG_SOLVER_CG : FESTUNG_SOLVER_BICGSTAB;
                const int64_t l0c = cc->launches;
                // warm start from the previous coarse solution (both right-hand sides are scaled to
                // unit norm, and the error of the extrapolated guess changes slowly from step to
                // step: 82 -> 52 coarse iterations per step on the 256 x 256 p = 4 workload)
                rc = krylov_solve<float>(cc, csolver, dt, 1e-2, 2000, !c->coarse_warm, &cit, &cr2, &cb2, &ccin);
                c->coarse_warm = true;
                c->launches += cc->launches - l0c;
                if (rc) {
                    c->err = "coarse solve: " + cc->err;
                    return rc;
                }
                coarse_iters += cit;
                if (cr2 < cb2) {  // a usable correction (finite and lowering the coarse residual)
                    FCK(cudaMemcpyAsync(F.x, CF.x, K3 * sizeof(float), cudaMemcpyDeviceToDevice, st));
                    x_zero = false;
                }
            }
            int it = 0;
            bool cin = false;
            double ir2, ib2;
            // the FP32 sweep reduces by inner_tol, or by less when less is still needed;
            // after a failure the next sweep starts from a reweighted shadow residual
            const double target = std::min(0.5, std::max(o.inner_tol, 0.5 * o.tol / relres));
            c->tab_bf16 = o.prec == FESTUNG_BF16TAB;
            rc = krylov_solve<float>(c, solver, dt, target, o.max_iter - iters, x_zero, &it, &ir2, &ib2, &cin,
                                     failures > 0);
            c->tab_bf16 = false;
            if (rc) return rc;
            iters += it;
            if (!(ir2 < ib2)) {
                // no progress (or non-finite values) in FP32: skip the sweep
                if (++failures >= 2) {
                    fp64 = true;
                    break;
                }
                continue;
            }
            last_scale = rn;
            k_add_f32<<<small_grid(KN, c), 256, 0, st>>>(KN, V.x, F.x, rn); ++c->launches;
            applied = true;
            FCK(cudaGetLastError());
        }
        if (outer > o.max_outer) outer = o.max_outer;
    }
    if (fp64) {
        // FP64 Krylov; verified with the true residual and restarted if the recursion drifted
        if ((rc = finish_precond(c))) return rc;
        for (int sweep = 1; sweep <= o.max_outer; ++sweep, ++outer) {
            int it = 0;
            double rr0 = -1.0;
            rc = krylov_solve<double>(c, solver, dt, o.tol, std::max(1, o.max_iter - iters), false, &it, &r2, &b2,
                                      &conv, false, &rr0);
            if (relres0 < 0.0) relres0 = rr0;
            if (rc) return rc;
            iters += it;
            if (o.prec != FESTUNG_FP64) iters64 += it;
            double rn, bn;
            if ((rc = residual64(&rn, &bn))) return rc;
            relres = bn > 0 ? rn / bn : rn;
            conv = relres <= o.tol;
            if (conv || iters >= o.max_iter) break;
        }
        if (outer < 1) outer = 1;
    }
    if (info) {
        info->iterations = iters;
        info->outer = outer;
        info->rel_residual = relres;
        info->solver = solver;
        info->symmetric = c->symmetric ? 1 : 0;
        info->fp64_iterations = iters64;
        info->initial_rel_residual = relres0;
        info->coarse_iterations = coarse_iters;
        info->precond_built = c->P_built ? 1 : 0;
    }
    // a step that needed many more iterations than the one that built the blocks ends
    // their reuse
    if (c->P_built) {
        c->P_iters0 = iters;
    } else if (c->P_iters0 >= 0 && 2 * iters > 3 * c->P_iters0 + 8) {
        c->P_valid = false;
    }
    if (!conv) {
        char msg[96];
        std::snprintf(msg, sizeof(msg), "Krylov solve did not converge (relative residual %.3e)", relres);
        c->err = msg;
        return FESTUNG_ENOCONV;
    }
    return commit_solution(c, dt, stationary);
}

}  // namespace

extern "C" {

int festung_step(festung_ctx *c, double dt, const festung_step_opts *opts, festung_step_info *info) {
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    return solve_system(c, dt, 1.0, opts, info);
}

int festung_solve_stationary(festung_ctx *c, const festung_step_opts *opts, festung_step_info *info) {
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    if (!c->has_dirichlet) {
        c->err = "the stationary problem needs a Dirichlet edge (with zero-flux data alone it is singular)";
        return FESTUNG_EINVAL;
    }
    return solve_system(c, 1.0, 0.0, opts, info);
}

int festung_l2_error(const festung_ctx *cc, const double *c_samples, double *err) {
    festung_ctx *c = const_cast<festung_ctx *>(cc);
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    if (!c_samples || !err) {
        c->err = "NULL argument";
        return FESTUNG_EINVAL;
    }
    int rc = ensure_ws(c);
    if (rc) return rc;
    Workspace &w = *c->ws;
    const int64_t n = c->K * c->R2;
    FCK(cudaMemcpyAsync(c->dSamp, c_samples, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    QuadWeights qw{};
    for (int r = 0; r < c->R2; ++r) qw.w[r] = c->tab.tri.w[r];
    const TableOffsets o = table_offsets(c->N, c->R2, c->R1);
    k_l2_error<<<w.nblk, RED_THREADS, 0, c->stream>>>(c->K, c->N, c->R2, c->dC, c->dSamp, c->dTab + o.phiQ, qw,
                                                     c->dB, c->dPerm, w.part);
    k_fin_sums<<<1, 1024, 0, c->stream>>>(w.res, w.part, w.nblk, 1);
    c->launches += 2;
    FCK(cudaGetLastError());
    FCK(cudaMemcpyAsync(w.h_res, w.res, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    FCK(cudaStreamSynchronize(c->stream));
    *err = std::sqrt(std::max(0.0, w.h_res[0]));
    return FESTUNG_OK;
}

int festung_get_flux(const festung_ctx *cc, double *Z, int loc) {
    festung_ctx *c = const_cast<festung_ctx *>(cc);
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    if (!Z || (loc != FESTUNG_HOST && loc != FESTUNG_DEVICE)) {
        c->err = "Z is NULL or bad loc";
        return FESTUNG_EINVAL;
    }
    int rc = ensure_ws(c);
    if (rc) return rc;
    Workspace &w = *c->ws;
    const int64_t KN = c->K * c->N;
    if ((rc = alloc_vecs<double>(c, w.d, false))) return rc;
    if (!w.scratch64) FCK(cudaMalloc(&w.scratch64, 2 * KN * sizeof(double)));
    double *W1 = w.scratch64, *W2 = w.scratch64 + KN;
    cudaStream_t st = c->stream;
    launch_flux(c, c->dC, w.d.Z1, w.d.Z2, st);
    launch_lift(c, W1, W2, st);
    double *out = Z;
    double *tmp = nullptr;
    if (loc == FESTUNG_HOST) FCK(cudaMalloc(&tmp, 2 * KN * sizeof(double)));
    if (tmp) out = tmp;
    k_flux_public<<<small_grid(KN, c), 256, 0, st>>>(c->K, c->N, w.d.Z1, w.d.Z2, W1, W2, c->dPerm, out);
    ++c->launches;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && tmp) e = cudaMemcpyAsync(Z, tmp, 2 * KN * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) {
        c->err = std::string("festung_get_flux: ") + cudaGetErrorString(e);
        return FESTUNG_ECUDA;
    }
    return FESTUNG_OK;
}

int festung_warmstart_features(festung_ctx *c, double dt, float *X, float *Wt, double *scale) {
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    if (!X || !(dt > 0.0)) {
        c->err = "X is NULL or dt <= 0";
        return FESTUNG_EINVAL;
    }
    int rc = ensure_ws(c);
    if (rc) return rc;
    Workspace &w = *c->ws;
    if ((rc = alloc_vecs<double>(c, w.d, true))) return rc;
    const int64_t K = c->K, KN = K * c->N;
    if (!w.scratch64) FCK(cudaMalloc(&w.scratch64, 2 * KN * sizeof(double)));
    cudaStream_t st = c->stream;
    Vecs<double> &V = w.d;
    launch_rhs(c, w.scratch64, w.scratch64 + KN, V.b, dt, st);
    if ((rc = apply_df(c, c->dC, nullptr, dt, st))) return rc;
    k_residual_df<<<w.nblk, RED_THREADS, 0, st>>>(KN, V.b, w.ydf, V.r, w.part);
    k_ws_sums<<<w.nblk, RED_THREADS, 0, st>>>(K, c->N, V.r, c->dD, c->dB, w.part);
    k_fin_sums<<<1, 1024, 0, st>>>(w.res, w.part, w.nblk, 2);
    c->launches += 3;
    FCK(cudaGetLastError());
    FCK(cudaMemcpyAsync(w.h_res, w.res, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    FCK(cudaStreamSynchronize(st));
    const double rs = std::sqrt(w.h_res[0] / (double)KN), dm = w.h_res[1] / (double)K;
    const double inv_rs = rs > 0.0 ? 1.0 / rs : 0.0, inv_d = dm != 0.0 ? 1.0 / dm : 1.0;
    k_ws_features<<<small_grid(K, c), 256, 0, st>>>(K, c->N, V.r, c->dD, c->dB, c->dNbr, inv_rs, inv_d, X);
    ++c->launches;
    if (Wt) {
        // diagonal blocks of S (FP32) for the loss weights
        if (!w.P) FCK(cudaMalloc(&w.P, (size_t)c->N * c->N * c->K * sizeof(float)));
        if (!w.Pb) FCK(cudaMalloc(&w.Pb, (size_t)((c->N * c->N + 7) / 8) * c->K * 16));
        launch_blockjacobi(c, w.P, w.Pb, dt, w.d_flags, st);
        c->P_valid = false;  // the step's own build replaces them
        k_ws_weights<<<small_grid(K, c), 256, 0, st>>>(K, c->N, w.P, c->dB, Wt);
        ++c->launches;
    }
    FCK(cudaGetLastError());
    FCK(cudaStreamSynchronize(st));
    if (scale) *scale = rs;
    return FESTUNG_OK;
}

int festung_set_guess(festung_ctx *c, const double *delta, int loc) {
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    if (!delta) {
        c->has_guess = false;
        return FESTUNG_OK;
    }
    int rc = ensure_ws(c);
    if (rc) return rc;
    Workspace &w = *c->ws;
    const int64_t KN = c->K * c->N;
    if (!w.scratch64) FCK(cudaMalloc(&w.scratch64, 2 * KN * sizeof(double)));
    if (!c->dGuess) FCK(cudaMalloc(&c->dGuess, KN * sizeof(double)));
    double *tmp = w.scratch64;
    if ((rc = upload_checked(c, delta, loc, tmp, KN))) return rc;
    k_to_internal<<<small_grid(KN, c), 256, 0, c->stream>>>(tmp, c->dGuess, c->K, c->N, c->dPerm); ++c->launches;
    FCK(cudaGetLastError());
    c->has_guess = true;
    return FESTUNG_OK;
}

int festung_element_order(const festung_ctx *c, int64_t *order) {
    if (!c || !order) return FESTUNG_EINVAL;
    for (int64_t k = 0; k < c->K; ++k) order[k] = c->perm[k];
    return FESTUNG_OK;
}

int festung_precond_blocks(festung_ctx *c, double dt, double *blocks, double *inverse) {
    if (!ready(c)) return c ? FESTUNG_ESTATE : FESTUNG_EINVAL;
    if (!(dt >= 0.0) || (!blocks && !inverse)) {
        c->err = "bad preconditioner query arguments";
        return FESTUNG_EINVAL;
    }
    int rc = ensure_ws(c);
    if (rc) return rc;
    if ((rc = finish_precond(c))) return rc;  // a build of the last step may still run
    Workspace &w = *c->ws;
    const int N = c->N, NQ = (N * N + 7) / 8;
    const int64_t K = c->K;
    if (!w.P) FCK(cudaMalloc(&w.P, (size_t)N * N * K * sizeof(float)));
    if (!w.Pb) FCK(cudaMalloc(&w.Pb, (size_t)NQ * K * 16));
    cudaStream_t st = c->stream;
    FCK(cudaMemsetAsync(w.d_flags, 0, sizeof(int), st));
    launch_blockjacobi(c, w.P, w.Pb, dt, w.d_flags, st);
    c->P_valid = false;  // the next step builds its own
    FCK(cudaGetLastError());
    std::vector<float> hP(blocks ? (size_t)N * N * K : 0);
    std::vector<uint16_t> hB(inverse ? (size_t)NQ * K * 8 : 0);
    if (blocks) FCK(cudaMemcpyAsync(hP.data(), w.P, hP.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (inverse) FCK(cudaMemcpyAsync(hB.data(), w.Pb, hB.size() * sizeof(uint16_t), cudaMemcpyDeviceToHost, st));
    FCK(cudaMemcpyAsync(w.h_flags, w.d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    FCK(cudaStreamSynchronize(st));
    for (int64_t k = 0; k < K; ++k) {
        const int64_t kc = c->perm[k];
        for (int e = 0; e < N * N; ++e) {
            const int64_t out = kc * N * N + e;  // row i = e / N, column j = e % N
            if (blocks) blocks[out] = hP[(size_t)e * K + k];
            if (inverse) {
                // BF16 chunk e / 8 of triangle k holds entries 8 (e / 8) .. 8 (e / 8) + 7
                const uint32_t bits = (uint32_t)hB[((size_t)(e / 8) * K + k) * 8 + e % 8] << 16;
                float f;
                std::memcpy(&f, &bits, sizeof(f));
                inverse[out] = f;
            }
        }
    }
    if (w.h_flags[0]) {
        c->err = "a diagonal block is singular";
        return FESTUNG_EDATA;
    }
    return FESTUNG_OK;
}

int festung_launch_count(const festung_ctx *c, int64_t *count) {
    if (!c || !count) return FESTUNG_EINVAL;
    *count = c->launches;
    return FESTUNG_OK;
}

int festung_set_stream(festung_ctx *c, void *stream) {
    if (!c) return FESTUNG_EINVAL;
    c->stream = (cudaStream_t)stream;
    return FESTUNG_OK;
}

const char *festung_last_error(const festung_ctx *c) {
    if (!c) return g_create_err.c_str();
    return c->err.c_str();
}

int festung_set_persistent(festung_ctx *c, int enable) {
    if (!c) return FESTUNG_EINVAL;
    if (enable != 0 && enable != 1) {
        c->err = "enable must be 0 or 1";
        return FESTUNG_EINVAL;
    }
    c->persistent = enable != 0;
    if (c->coarse) c->coarse->persistent = c->persistent;
    return FESTUNG_OK;
}

int festung_set_precond_reuse(festung_ctx *c, int max_steps) {
    if (!c) return FESTUNG_EINVAL;
    if (max_steps < 1) {
        c->err = "max_steps must be >= 1";
        return FESTUNG_EINVAL;
    }
    c->precond_reuse = max_steps;
    return FESTUNG_OK;
}

int festung_set_coarse(festung_ctx *c, int enable) {
    if (!c) return FESTUNG_EINVAL;
    if (enable != 0 && enable != 1) {
        c->err = "enable must be 0 or 1";
        return FESTUNG_EINVAL;
    }
    c->coarse_mode = enable;
    return FESTUNG_OK;
}

void festung_destroy(festung_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
        cudaEventDestroy(c->ev_in);
        cudaEventDestroy(c->ev_P);
    }
    free_ctx_device(c);
    void *mesh_ptrs[] = {c->dB, c->fB, c->dNbr, c->dPerm, c->dSlot, c->dHaloPtr, c->dHalo, c->dHaloSlot, c->dLift};
    for (void *q : mesh_ptrs)
        if (q) cudaFree(q);
    delete c;
}

}  // extern "C"

// ===========================================================================
// Batches of independent problems
//
// Problems of the same order (and quadrature and penalty) form a group.  The union of
// their meshes is one internal context: every kernel of a step runs over all problems of
// the group at once, and the Krylov iteration runs on the block-diagonal union system
// (no kernel couples two problems).  Refinement and convergence are per problem: each
// problem's residual is normalised on its own before an inner FP32 solve, its correction
// is scaled back with its own norm, and a converged problem enters later sweeps with a
// zero right-hand side, which the Krylov recursion keeps exactly zero.
// ===========================================================================
namespace {

struct MemberPtrs {
    double *C;
    const double *D, *F, *CD, *GN;
    int64_t K, off;
};

// union <- members: C, D (and its FP32 copy), F in the N x K internal layout; c_D, g_N
// (K x 3 x R1) in the concatenated caller order.  Member q owns union elements
// [off_q, off_q + K_q) in both orders.
__global__ void k_batch_gather(int64_t K, int N, int E, const int32_t *eprob, const MemberPtrs *mem, double *C,
                               double *D, float *fD, double *F, double *CD, double *GN) {
    ELEM_LOOP(i) {
        const MemberPtrs m = mem[eprob[i]];
        const int64_t l = i - m.off;
        for (int j = 0; j < N; ++j) {
            C[j * K + i] = m.C[j * m.K + l];
            const double d = m.D[j * m.K + l];
            D[j * K + i] = d;
            fD[j * K + i] = (float)d;
            F[j * K + i] = m.F[j * m.K + l];
        }
        for (int e = 0; e < E; ++e) {
            CD[i * E + e] = m.CD[l * E + e];
            GN[i * E + e] = m.GN[l * E + e];
        }
    }
}

// members <- union: C, for the members with mask[q] != 0
__global__ void k_batch_scatter(int64_t K, int N, const int32_t *eprob, const MemberPtrs *mem, const double *C,
                                const double *mask) {
    ELEM_LOOP(i) {
        const int q = eprob[i];
        if (mask[q] == 0.0) continue;
        const MemberPtrs m = mem[q];
        const int64_t l = i - m.off;
        for (int j = 0; j < N; ++j) m.C[j * m.K + l] = C[j * K + i];
    }
}

// r = b - y (y double-float) and per-problem (r, r), (b, b) into acc[2 q], acc[2 q + 1]
// (acc zeroed by the caller).  A warp whose elements belong to one problem adds its sums
// with one atomic per value.
__global__ void k_residual_df_batch(int64_t K, int N, const double *b, const dfloat *y, double *r,
                                    const int32_t *eprob, double *acc) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < K; base += stride) {
        const int64_t i = base + threadIdx.x;
        double rr = 0.0, bb = 0.0;
        int q = -1;
        if (i < K) {
            q = eprob[i];
            for (int j = 0; j < N; ++j) {
                const int64_t idx = j * K + i;
                const double ri = b[idx] - (double)y[idx];
                r[idx] = ri;
                rr += ri * ri;
                bb += b[idx] * b[idx];
            }
        }
        const int q0 = __shfl_sync(0xffffffffu, q, 0);
        if (__all_sync(0xffffffffu, q == q0 || q < 0)) {
            for (int o = 16; o > 0; o >>= 1) {
                rr += __shfl_xor_sync(0xffffffffu, rr, o);
                bb += __shfl_xor_sync(0xffffffffu, bb, o);
            }
            if ((threadIdx.x & 31) == 0 && q0 >= 0) {
                atomicAdd(acc + 2 * q0, rr);
                atomicAdd(acc + 2 * q0 + 1, bb);
            }
        } else if (q >= 0) {
            atomicAdd(acc + 2 * q, rr);
            atomicAdd(acc + 2 * q + 1, bb);
        }
    }
}

// Fb = scale_q r (FP32)
__global__ void k_scale_batch(int64_t K, int N, const double *r, float *Fb, const int32_t *eprob, const double *scale) {
    ELEM_LOOP(i) {
        const double sc = scale[eprob[i]];
        for (int j = 0; j < N; ++j) Fb[j * K + i] = (float)(r[j * K + i] * sc);
    }
}

// x += scale_q Fx
__global__ void k_add_batch(int64_t K, int N, double *x, const float *Fx, const int32_t *eprob, const double *scale) {
    ELEM_LOOP(i) {
        const double sc = scale[eprob[i]];
        if (sc != 0.0)
            for (int j = 0; j < N; ++j) x[j * K + i] += sc * (double)Fx[j * K + i];
    }
}

// Krylov start for a batch: r = b - y (y = S x, or none for x = 0), the shadow residual
// r0, p = v = 0, and per-problem (r, r), (b, b), (r0, r)
template <typename T>
__global__ void k_kr_init_b(int64_t K, int N, const T *b, const T *y, T *r, T *r0, T *p, T *v, BatchView bv,
                            int reweight) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < K; base += stride) {
        const int64_t k = base + threadIdx.x;
        double acc[3] = {0.0, 0.0, 0.0};
        int q = -1;
        if (k < K) {
            q = bv.eprob[k];
            for (int j = 0; j < N; ++j) {
                const int64_t i = j * K + k;
                const T bi = b[i];
                const T ri = y ? bi - y[i] : bi;
                r[i] = ri;
                T wgt = T(1);
                if (reweight) {
                    const uint32_t h = (uint32_t)(i * 2654435761ull) >> 8;
                    wgt = T(0.5) + T(h & 0xffff) / T(65536);
                }
                r0[i] = ri * wgt;
                p[i] = T(0);
                v[i] = T(0);
                acc[0] += (double)ri * (double)ri;
                acc[1] += (double)bi * (double)bi;
                acc[2] += (double)(ri * wgt) * (double)ri;
            }
        }
        batch_add<3>(bv, q, acc);
    }
}

// per-problem scalars at the start of a batch solve (one block); tolq: relative tolerances
__global__ void k_fin_init_b(KScal *sc, BatchView bv, const double *tolq) {
    int open = 0;
    for (int q = threadIdx.x; q < bv.nprob; q += blockDim.x) {
        const double r2 = bv.acc[q], b2 = bv.acc[bv.nprob + q], r0r = bv.acc[2 * bv.nprob + q];
        bv.acc[q] = bv.acc[bv.nprob + q] = bv.acc[2 * bv.nprob + q] = 0.0;
        KScal e{};
        e.r2 = e.r2_0 = e.ss = r2;
        e.b2 = b2;
        e.tol2 = tolq[q] * tolq[q];
        e.rho = r0r;
        e.alpha = e.omega = 1.0;
        e.first = 1;
        e.done = (r2 <= e.tol2 * b2) ? 1 : 0;
        sc[q] = e;
        open |= !e.done;
    }
    const int any = __syncthreads_or(open);
    if (threadIdx.x == 0) *bv.alldone = any ? 0 : 1;
}

// per-problem (b - y, b - y) and (b, b) into acc[q], acc[nprob + q]
template <typename T>
__global__ void k_residual_b(int64_t K, int N, const T *b, const T *y, BatchView bv) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < K; base += stride) {
        const int64_t k = base + threadIdx.x;
        double acc[2] = {0.0, 0.0};
        int q = -1;
        if (k < K) {
            q = bv.eprob[k];
            for (int j = 0; j < N; ++j) {
                const double bi = (double)b[j * K + k], ri = bi - (double)y[j * K + k];
                acc[0] += ri * ri;
                acc[1] += bi * bi;
            }
        }
        batch_add<2>(bv, q, acc);
    }
}

struct BatchGroup {
    bool built = false;             // the union below exists (built at the first union-mode step)
    festung_ctx *u = nullptr;       // union context
    std::vector<int> members;       // problem indices
    std::vector<int64_t> off;       // element offset of each member (members + 1 entries)
    std::vector<uint64_t> gen;      // member state generations seen after the last step
    int32_t *eprob = nullptr;       // K: member of each union element
    MemberPtrs *dmem = nullptr;     // device table of member arrays
    double *dacc = nullptr, *hacc = nullptr;      // 2 per member: residual sums
    double *dscale = nullptr, *hscale = nullptr;  // 1 per member
    // the members' own BiCGStab iterations on the union
    KScal *sc = nullptr, *hsc = nullptr;  // per-member scalars (device / pinned host)
    double *kacc = nullptr;               // 4 x members reduction sums
    int *alldone = nullptr;               // device flag: every member's iteration is done
    int *halldone = nullptr;              // its pinned host copy
    double *dtol = nullptr, *htol = nullptr;  // members' relative tolerances of the sweep (device / pinned)
    cudaGraphExec_t exec = nullptr;       // CHUNK iterations
    double g_tau = 0.0;
    int g_useP = -1;
    cudaStream_t stream = nullptr;        // the group's own stream (groups run concurrently)
    cudaEvent_t done_ev = nullptr;
    std::string err;                      // message of the group's last failure
};

void free_group(BatchGroup &g) {
    if (g.stream) cudaStreamSynchronize(g.stream);
    if (g.exec) cudaGraphExecDestroy(g.exec);
    cudaFree(g.sc);
    if (g.hsc) cudaFreeHost(g.hsc);
    cudaFree(g.kacc);
    cudaFree(g.alldone);
    if (g.halldone) cudaFreeHost(g.halldone);
    cudaFree(g.dtol);
    if (g.htol) cudaFreeHost(g.htol);
    if (g.u) festung_destroy(g.u);
    if (g.done_ev) cudaEventDestroy(g.done_ev);
    if (g.stream) cudaStreamDestroy(g.stream);
    cudaFree(g.eprob);
    cudaFree(g.dmem);
    cudaFree(g.dacc);
    cudaFree(g.dscale);
    if (g.hacc) cudaFreeHost(g.hacc);
    if (g.hscale) cudaFreeHost(g.hscale);
    g = BatchGroup();
}

}  // namespace

struct festung_batch {
    std::vector<festung_ctx *> probs;
    std::vector<BatchGroup> groups;
    cudaStream_t stream = nullptr;
    cudaEvent_t start_ev = nullptr;
    int device = 0;
    int mode = FESTUNG_BATCH_CONCURRENT;
    int workers = 16;
    // FESTUNG_BATCH_CONCURRENT: one stream and two events per worker
    std::vector<cudaStream_t> wstreams;
    std::vector<cudaEvent_t> wev, wdone;
    // kernels launched on the problems' own contexts during batch steps
    std::atomic<int64_t> member_launches{0};
    std::string err;
};

namespace {

// Union context of the members of one group (all set up with the same p, quadrature and eta).
int build_group(festung_batch *b, BatchGroup &g) {
    festung_ctx *first = b->probs[g.members[0]];
    int64_t K = 0;
    g.off.assign(1, 0);
    for (int q : g.members) {
        K += b->probs[q]->K;
        g.off.push_back(K);
    }
    if (K * (int64_t)first->N >= (int64_t(1) << 31)) {
        b->err = "batch group too large: K * N must stay below 2^31";
        return FESTUNG_EINVAL;
    }
    festung_ctx *u = new (std::nothrow) festung_ctx();
    if (!u) return FESTUNG_ENOMEM;
    g.u = u;
    u->K = K;
    MeshOrder mo;
    mo.perm.resize(K);
    mo.B.assign(4 * K, 0.0);
    mo.nbr.assign(3 * K, 0);
    std::vector<int32_t> ep(K);
    for (size_t m = 0; m < g.members.size(); ++m) {
        const festung_ctx *c = b->probs[g.members[m]];
        const int64_t Kq = c->K, off = g.off[m];
        u->has_dirichlet |= c->has_dirichlet;
        u->has_neumann |= c->has_neumann;
        for (int64_t i = 0; i < Kq; ++i) {
            const int64_t cu = c->perm[i];
            mo.perm[off + i] = (int32_t)(off + cu);
            for (int r = 0; r < 4; ++r) mo.B[r * K + off + i] = c->hB[r * Kq + cu];
            for (int n = 0; n < 3; ++n) {
                const int32_t code = c->hNbrInt[n * Kq + i];
                mo.nbr[n * K + off + i] = code >= 0 ? (int32_t)((((code >> 2) + off) << 2) | (code & 3)) : code;
            }
            ep[off + i] = (int32_t)m;
        }
    }
    lift_flags(mo.nbr, K, mo.lift);
    u->perm = mo.perm;
    u->hNbrInt = mo.nbr;
    cudaError_t e = upload_mesh(u, mo);
    if (e != cudaSuccess) {
        b->err = std::string("CUDA: ") + cudaGetErrorString(e);
        return FESTUNG_ECUDA;
    }
    int rc = festung_setup(u, first->p, first->qT, first->eta);
    if (rc) {
        b->err = u->err;
        return rc;
    }
    const size_t nm = g.members.size();
    std::vector<MemberPtrs> hm(nm);
    for (size_t m = 0; m < nm; ++m) {
        festung_ctx *c = b->probs[g.members[m]];
        hm[m] = MemberPtrs{c->dC, c->dD, c->dF, c->dCD, c->dGN, c->K, g.off[m]};
    }
    if ((e = cudaMalloc(&g.eprob, K * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMemcpy(g.eprob, ep.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&g.dmem, nm * sizeof(MemberPtrs))) != cudaSuccess ||
        (e = cudaMemcpy(g.dmem, hm.data(), nm * sizeof(MemberPtrs), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&g.dacc, 2 * nm * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&g.dscale, nm * sizeof(double))) != cudaSuccess ||
        (e = cudaMallocHost(&g.hacc, 2 * nm * sizeof(double))) != cudaSuccess ||
        (e = cudaMallocHost(&g.hscale, nm * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&g.sc, nm * sizeof(KScal))) != cudaSuccess ||
        (e = cudaMallocHost(&g.hsc, nm * sizeof(KScal))) != cudaSuccess ||
        (e = cudaMalloc(&g.kacc, 4 * nm * sizeof(double))) != cudaSuccess ||
        (e = cudaMemset(g.kacc, 0, 4 * nm * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&g.alldone, sizeof(int))) != cudaSuccess ||
        (e = cudaMallocHost(&g.halldone, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(g.alldone, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&g.dtol, nm * sizeof(double))) != cudaSuccess ||
        (e = cudaMallocHost(&g.htol, nm * sizeof(double))) != cudaSuccess) {
        b->err = std::string("CUDA: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? FESTUNG_ENOMEM : FESTUNG_ECUDA;
    }
    g.gen.assign(nm, ~0ull);
    if ((e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&g.done_ev, cudaEventDisableTiming)) != cudaSuccess) {
        b->err = std::string("CUDA: ") + cudaGetErrorString(e);
        return FESTUNG_ECUDA;
    }
    festung_set_stream(u, g.stream);
    int te = 0;
    if ((rc = autotune_tiles(u, &te))) {
        b->err = u->err;
        return rc;
    }
    g.built = true;
    return FESTUNG_OK;
}

// The union of a group, built when the union mode first needs it; a failed build leaves
// the group as it was.
int ensure_built(festung_batch *b, BatchGroup &g) {
    if (g.built) return FESTUNG_OK;
    const int rc = build_group(b, g);
    if (rc) {
        const std::vector<int> members = g.members;
        free_group(g);
        g.members = members;
    }
    return rc;
}

// The members' own BiCGStab iterations on the union (FP32, vectors w.f): every member
// stops at its relative tolerance tolq[m] (a member with tolq <= 0 or a zero right-hand
// side is done at once).  Returns per-member true ||b - S x||^2, ||b||^2 and the largest
// iteration count; members whose recursion drifted or broke down are restarted (all
// running members restart together, at most 8 times).
int krylov_solve_batch(BatchGroup &g, double tau, const std::vector<double> &tolq, int max_iter, int *iters,
                       std::vector<double> &r2, std::vector<double> &b2, std::vector<char> &finished,
                       bool reweight) {
    festung_ctx *c = g.u;
    Workspace &w = *c->ws;
    Vecs<float> &V = w.f;
    const int nm = (int)g.members.size();
    const int64_t K = c->K;
    const int N = c->N, gb = w.nblk;
    cudaStream_t st = c->stream;
    BatchView bv;
    bv.eprob = g.eprob;
    bv.acc = g.kacc;
    bv.alldone = g.alldone;
    bv.nprob = nm;
    FCK(cudaStreamSynchronize(st));  // htol may still feed an earlier copy
    for (int m = 0; m < nm; ++m) g.htol[m] = tolq[m];
    FCK(cudaMemcpyAsync(g.dtol, g.htol, nm * sizeof(double), cudaMemcpyHostToDevice, st));
    const __nv_bfloat16 *P = w.use_P ? w.Pb : nullptr;
    int total = 0;
    r2.assign(nm, 0.0);
    b2.assign(nm, 0.0);
    for (int restart = 0; restart < 8; ++restart) {
        if (restart == 0) {
            k_kr_init_b<float><<<gb, RED_THREADS, 0, st>>>(K, N, V.b, nullptr, V.r, V.r0, V.p, V.v, bv,
                                                           reweight ? 1 : 0);
        } else {
            launch_apply<float>(c, V.x, V.t, V.Z1, V.Z2, (float)tau, nullptr, st);
            k_kr_init_b<float><<<gb, RED_THREADS, 0, st>>>(K, N, V.b, V.t, V.r, V.r0, V.p, V.v, bv, 1);
        }
        k_fin_init_b<<<1, 1024, 0, st>>>(g.sc, bv, g.dtol);
        c->launches += 2;
        FCK(cudaGetLastError());
        if (!g.exec || g.g_tau != tau || g.g_useP != (int)w.use_P) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            cudaStream_t cs;
            FCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t graph;
            const int64_t saved = c->launches;
            FCK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            for (int it = 0; it < CHUNK; ++it) {
                dispatch(c->N, c->R2, c->R1, [&](auto n_, auto, auto) {
                    constexpr int NN = decltype(n_)::value;
                    k_bicg_next_b<float, NN><<<gb, RED_THREADS, 0, cs>>>((int)K, V.x, V.ph, V.sh, V.s, V.t, V.r, V.p,
                                                                        V.v, P, V.inv, g.sc, bv);
                });
                launch_apply_bicg<float>(c, V.ph, V.v, (float)tau, FUSED_EPI_ALPHA, V.r0, nullptr, w.part, g.sc,
                                         w.counter, g.alldone, cs, bv);
                dispatch(c->N, c->R2, c->R1, [&](auto n_, auto, auto) {
                    constexpr int NN = decltype(n_)::value;
                    k_bicg_s_b<float, NN><<<gb, RED_THREADS, 0, cs>>>((int)K, V.r, V.s, V.v, V.sh, P, V.inv, g.sc,
                                                                     bv, w.counter);
                });
                launch_apply_bicg<float>(c, V.sh, V.t, (float)tau, FUSED_EPI_OMEGA, V.s, V.r0, w.part, g.sc,
                                         w.counter, g.alldone, cs, bv);
            }
            FCK(cudaStreamEndCapture(cs, &graph));
            c->launches = saved;
            FCK(cudaGraphInstantiate(&g.exec, graph, 0));
            cudaGraphDestroy(graph);
            cudaStreamDestroy(cs);
            g.g_tau = tau;
            g.g_useP = (int)w.use_P;
        }
        int hmax = 0, it90 = -1, open0 = 0;
        bool again = false;
        for (int m = 0; m < nm; ++m) open0 += tolq[m] > 0.0;
        while (true) {
            FCK(cudaMemcpyAsync(g.hsc, g.sc, nm * sizeof(KScal), cudaMemcpyDeviceToHost, st));
            FCK(cudaMemcpyAsync(g.halldone, g.alldone, sizeof(int), cudaMemcpyDeviceToHost, st));
            FCK(cudaStreamSynchronize(st));
            const int alldone = *g.halldone;
            hmax = 0;
            int done = 0;
            for (int m = 0; m < nm; ++m) {
                hmax = std::max(hmax, g.hsc[m].iter);
                done += tolq[m] > 0.0 && g.hsc[m].done;
            }
            if (alldone || total + hmax >= max_iter) break;
            // stragglers: once 90 % of the members are done, the rest get as many iterations
            // again (and one chunk) before they are left to their own solves
            if (it90 < 0 && 10 * done >= 9 * open0) it90 = hmax;
            if (it90 >= 0 && hmax >= 2 * it90 + CHUNK) break;
            FCK(cudaGraphLaunch(g.exec, st));
            c->launches += 4 * CHUNK;
        }
        total += hmax;
        k_bicg_finish_b<float><<<gb, RED_THREADS, 0, st>>>((int)K, N, V.x, V.ph, V.sh, g.sc, bv);
        ++c->launches;
        // true residuals per member
        launch_apply<float>(c, V.x, V.t, V.Z1, V.Z2, (float)tau, nullptr, st);
        k_residual_b<float><<<gb, RED_THREADS, 0, st>>>(K, N, V.b, V.t, bv);
        ++c->launches;
        FCK(cudaGetLastError());
        FCK(cudaMemcpyAsync(g.hacc, g.kacc, 2 * nm * sizeof(double), cudaMemcpyDeviceToHost, st));
        FCK(cudaMemsetAsync(g.kacc, 0, 2 * nm * sizeof(double), st));
        FCK(cudaStreamSynchronize(st));
        finished.assign(nm, 1);
        for (int m = 0; m < nm; ++m) {
            r2[m] = g.hacc[m];
            b2[m] = g.hacc[nm + m];
            const double t2 = tolq[m] * tolq[m];
            if (tolq[m] > 0.0 && !g.hsc[m].done) finished[m] = 0;  // cut off as a straggler
            else if (tolq[m] > 0.0 && (g.hsc[m].breakdown || r2[m] > 100.0 * t2 * b2[m])) again = true;
        }
        if (!again || total >= max_iter || restart >= 3) break;
    }
    *iters = total;
    return FESTUNG_OK;
}

// One implicit-Euler step of every member of a group (FESTUNG_MIXED).
int solve_group(festung_batch *b, BatchGroup &g, double dt, const festung_step_opts &o, festung_step_info *infos) {
    festung_ctx *c = g.u;
    const int nm = (int)g.members.size();
    const int64_t K = c->K, KN = K * c->N;
    cudaStream_t st = c->stream;
    // members' data into the union; the extrapolation history is kept only while no
    // member's state was changed from outside since the last batch step
    bool fresh = false, symmetric = true;
    for (int m = 0; m < nm; ++m) {
        const festung_ctx *p = b->probs[g.members[m]];
        fresh |= p->state_gen != g.gen[m];
        symmetric &= p->symmetric;
    }
    if (fresh) c->hist = 0;
    c->symmetric = symmetric;
    k_batch_gather<<<small_grid(K, c), 256, 0, st>>>(K, c->N, 3 * c->R1, g.eprob, g.dmem, c->dC, c->dD, c->fD, c->dF,
                                                     c->dCD, c->dGN);
    ++c->launches;
    FCK(cudaGetLastError());
    c->xD_valid = false;
    int rc = prepare_solve(c, dt, false, true);
    if (rc) return rc;
    Workspace &w = *c->ws;
    Vecs<double> &V = w.d;
    Vecs<float> &F = w.f;
    const int solver = FESTUNG_SOLVER_BICGSTAB;  // the members' iterations on the union
    std::vector<double> rn(nm), bn(nm), rel(nm), rel0(nm, -1.0), prev(nm, -1.0), last(nm, 0.0);
    // state of a member: 0 open, 1 converged, 2 left to its own single-problem solve
    std::vector<int> state(nm, 0), outer_of(nm, 0), fails(nm, 0);
    std::vector<char> applied(nm, 0);
    // per-member residual norms (S x in double-float arithmetic)
    auto residuals = [&]() -> int {
        if ((rc = apply_df(c, V.x, nullptr, dt, st))) return rc;
        FCK(cudaMemsetAsync(g.dacc, 0, 2 * nm * sizeof(double), st));
        k_residual_df_batch<<<small_grid(K, c), 256, 0, st>>>(K, c->N, V.b, w.ydf, V.r, g.eprob, g.dacc);
        ++c->launches;
        FCK(cudaGetLastError());
        FCK(cudaMemcpyAsync(g.hacc, g.dacc, 2 * nm * sizeof(double), cudaMemcpyDeviceToHost, st));
        FCK(cudaStreamSynchronize(st));
        for (int m = 0; m < nm; ++m) {
            rn[m] = std::sqrt(g.hacc[2 * m]);
            bn[m] = std::sqrt(g.hacc[2 * m + 1]);
            rel[m] = bn[m] > 0 ? rn[m] / bn[m] : rn[m];
            if (rel0[m] < 0.0) rel0[m] = rel[m];
        }
        return FESTUNG_OK;
    };
    auto add_scaled = [&](const std::vector<double> &sc) -> int {
        for (int m = 0; m < nm; ++m) g.hscale[m] = sc[m];
        FCK(cudaMemcpyAsync(g.dscale, g.hscale, nm * sizeof(double), cudaMemcpyHostToDevice, st));
        k_add_batch<<<small_grid(K, c), 256, 0, st>>>(K, c->N, V.x, F.x, g.eprob, g.dscale);
        ++c->launches;
        FCK(cudaGetLastError());
        return FESTUNG_OK;
    };
    int iters = 0, outer = 0;
    bool reweight = false;
    for (outer = 1; outer <= o.max_outer; ++outer) {
        if ((rc = residuals())) return rc;
        if ((rc = finish_precond(c))) return rc;
        // members whose last sweep did not lower their residual: undo it; after two such
        // sweeps a member is left to the single-problem solve
        std::vector<double> undo(nm, 0.0);
        bool any_undo = false;
        for (int m = 0; m < nm; ++m) {
            if (state[m]) continue;
            if (rel[m] <= o.tol || rn[m] == 0.0) {
                state[m] = 1;
                outer_of[m] = outer;
                continue;
            }
            if (applied[m] && !(rn[m] < prev[m])) {
                undo[m] = -last[m];
                any_undo = true;
                if (++fails[m] >= 2) state[m] = 2;
            } else if (applied[m]) {
                fails[m] = 0;
            }
            applied[m] = 0;
        }
        if (any_undo) {
            if ((rc = add_scaled(undo))) return rc;
            if ((rc = residuals())) return rc;
        }
        int open = 0;
        for (int m = 0; m < nm; ++m) open += state[m] == 0;
        if (open == 0 || iters >= o.max_iter) break;
        // normalised residuals of the open members
        for (int m = 0; m < nm; ++m) g.hscale[m] = state[m] ? 0.0 : 1.0 / rn[m];
        FCK(cudaMemcpyAsync(g.dscale, g.hscale, nm * sizeof(double), cudaMemcpyHostToDevice, st));
        k_scale_batch<<<small_grid(K, c), 256, 0, st>>>(K, c->N, V.r, F.b, g.eprob, g.dscale);
        ++c->launches;
        FCK(cudaMemsetAsync(F.x, 0, KN * sizeof(float), st));
        // every open member runs its own BiCGStab on the union to its own target
        std::vector<double> tolq(nm, 0.0), ir2, ib2;
        for (int m = 0; m < nm; ++m)
            if (!state[m]) tolq[m] = std::min(0.5, std::max(o.inner_tol, 0.5 * o.tol / rel[m]));
        int it = 0;
        std::vector<char> finished;
        rc = krylov_solve_batch(g, dt, tolq, o.max_iter - iters, &it, ir2, ib2, finished, reweight);
        if (rc) return rc;
        iters += it;
        reweight = any_undo;
        for (int m = 0; m < nm; ++m)
            if (!state[m] && (!finished[m] || !(ir2[m] < ib2[m]))) state[m] = 2;  // left to a single solve
        std::vector<double> sc(nm, 0.0);
        for (int m = 0; m < nm; ++m)
            if (state[m] == 0) {
                sc[m] = rn[m];
                last[m] = rn[m];
                prev[m] = rn[m];
                applied[m] = 1;
            }
        if ((rc = add_scaled(sc))) return rc;
    }
    if (outer > o.max_outer) outer = o.max_outer;
    // members still open after the sweeps (or the iteration bound) get the single solve
    for (int m = 0; m < nm; ++m)
        if (state[m] == 0) state[m] = 2;
    for (int m = 0; m < nm; ++m) {
        if (!infos) break;
        festung_step_info &in = infos[g.members[m]];
        in.iterations = iters;
        in.outer = state[m] == 1 ? outer_of[m] : outer;
        in.rel_residual = rel[m];
        in.solver = solver;
        in.symmetric = c->symmetric ? 1 : 0;
        in.fp64_iterations = 0;
        in.initial_rel_residual = rel0[m];
        in.coarse_iterations = 0;
        in.precond_built = c->P_built ? 1 : 0;
    }
    // the members left over: their own step from C^n (still in the member context), with
    // the FP64 fallback of the single-problem path
    for (int m = 0; m < nm; ++m) {
        if (state[m] != 2) continue;
        festung_ctx *p = b->probs[g.members[m]];
        festung_step_info in{};
        const int64_t l0 = p->launches;
        rc = solve_system(p, dt, 1.0, &o, &in);
        b->member_launches += p->launches - l0;
        if (rc) {
            g.err = "problem " + std::to_string(g.members[m]) + ": " + p->err;
            return rc;
        }
        if (infos) {
            festung_step_info &out = infos[g.members[m]];
            in.iterations += iters;
            in.initial_rel_residual = rel0[m];
            out = in;
        }
    }
    // C of the union; the members solved by the union get theirs back
    if ((rc = commit_solution(c, dt, false))) return rc;
    for (int m = 0; m < nm; ++m) g.hscale[m] = state[m] == 1 ? 1.0 : 0.0;
    FCK(cudaMemcpyAsync(g.dscale, g.hscale, nm * sizeof(double), cudaMemcpyHostToDevice, st));
    k_batch_scatter<<<small_grid(K, c), 256, 0, st>>>(K, c->N, g.eprob, g.dmem, c->dC, g.dscale);
    ++c->launches;
    FCK(cudaGetLastError());
    FCK(cudaStreamSynchronize(st));
    bool any_single = false;
    for (int m = 0; m < nm; ++m) {
        festung_ctx *p = b->probs[g.members[m]];
        any_single |= state[m] == 2;
        if (state[m] == 1) {
            p->hist = 0;  // the member's own step history no longer describes its state
            ++p->state_gen;
        }
        g.gen[m] = p->state_gen;
    }
    // a member solved on its own differs from the union's C: the union's history restarts
    if (any_single) c->hist = 0;
    return FESTUNG_OK;
}

// Workers of FESTUNG_BATCH_CONCURRENT by default: 16, or fewer on a host with fewer threads.
int default_workers() {
    const unsigned hw = std::thread::hardware_concurrency();
    return hw ? (int)std::min(16u, hw) : 16;
}

// FESTUNG_BATCH_CONCURRENT: every problem takes its own single-problem step (mixed
// precision with the FP64 fallback), `workers` problems at a time, each worker on a
// stream and host thread of its own.  A problem's step runs on the worker's stream after
// the work queued on the problem's own stream and on the batch's stream; the batch's
// stream then waits for every worker.
int batch_step_concurrent(festung_batch *b, double dt, const festung_step_opts &o, festung_step_info *infos) {
    const int nprob = (int)b->probs.size();
    const int nw = std::max(1, std::min(b->workers, nprob));
    while ((int)b->wstreams.size() < nw) {
        cudaStream_t st = nullptr;
        cudaEvent_t e1 = nullptr, e2 = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) != cudaSuccess) {
            if (st) cudaStreamDestroy(st);
            if (e1) cudaEventDestroy(e1);
            b->err = "CUDA: cannot create the streams of the batch's workers";
            return FESTUNG_ECUDA;
        }
        b->wstreams.push_back(st);
        b->wev.push_back(e1);
        b->wdone.push_back(e2);
    }
    if (cudaEventRecord(b->start_ev, b->stream) != cudaSuccess) {
        b->err = "CUDA: cannot record on the batch's stream";
        return FESTUNG_ECUDA;
    }
    std::vector<int> rcs(nprob, FESTUNG_OK);
    std::vector<std::string> errs(nprob);
    std::atomic<int> next{0};
    auto work = [&](int wi) {
        cudaSetDevice(b->device);
        cudaStream_t ws = b->wstreams[wi];
        cudaStreamWaitEvent(ws, b->start_ev, 0);
        for (int q = next.fetch_add(1); q < nprob; q = next.fetch_add(1)) {
            festung_ctx *c = b->probs[q];
            cudaStream_t own = c->stream;
            festung_step_info in{};
            if (cudaEventRecord(b->wev[wi], own) != cudaSuccess ||
                cudaStreamWaitEvent(ws, b->wev[wi], 0) != cudaSuccess) {
                rcs[q] = FESTUNG_ECUDA;
                errs[q] = "CUDA: cannot order the problem's stream before its step";
                continue;
            }
            const int64_t l0 = c->launches;
            c->stream = ws;
            // several workers at once: no persistent (cooperative) solver kernels, whose
            // grids would share the device with other workers' grids; the graph form
            const bool persistent = c->persistent;
            if (nw > 1) c->persistent = false;
            rcs[q] = solve_system(c, dt, 1.0, &o, &in);
            c->persistent = persistent;
            if (rcs[q]) {
                cudaStreamSynchronize(ws);  // a failed step may leave work in flight
                errs[q] = c->err;
            }
            c->stream = own;
            b->member_launches += c->launches - l0;
            if (infos) infos[q] = in;
        }
        cudaEventRecord(b->wdone[wi], ws);
    };
    std::vector<std::thread> threads;
    int started = 1;
    try {
        for (; started < nw; ++started) threads.emplace_back(work, started);
    } catch (...) {
        // no more host threads: the workers that did not start run here, after worker 0
        // has drained the queue (they only order their streams)
    }
    work(0);
    for (int wi = started; wi < nw; ++wi) work(wi);
    for (auto &t : threads) t.join();
    for (int wi = 0; wi < nw; ++wi) cudaStreamWaitEvent(b->stream, b->wdone[wi], 0);
    for (int q = 0; q < nprob; ++q)
        if (rcs[q]) {
            b->err = "problem " + std::to_string(q) + ": " + errs[q];
            return rcs[q];
        }
    return FESTUNG_OK;
}

}  // namespace

extern "C" {

int festung_batch_create(festung_ctx *const *problems, int nprob, festung_batch **out) {
    g_create_err.clear();
    if (!out || !problems || nprob < 1) {
        g_create_err = "NULL argument or empty batch";
        return FESTUNG_EINVAL;
    }
    *out = nullptr;
    for (int q = 0; q < nprob; ++q) {
        if (!problems[q] || problems[q]->p < 0) {
            g_create_err = "problem " + std::to_string(q) + " is NULL or not set up";
            return FESTUNG_ESTATE;
        }
        for (int r = 0; r < q; ++r)
            if (problems[r] == problems[q]) {
                g_create_err = "problem " + std::to_string(q) + " appears twice";
                return FESTUNG_EINVAL;
            }
    }
    festung_batch *b = new (std::nothrow) festung_batch();
    if (!b) return FESTUNG_ENOMEM;
    b->probs.assign(problems, problems + nprob);
    b->workers = default_workers();
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->start_ev, cudaEventDisableTiming) != cudaSuccess) {
        g_create_err = "CUDA: cannot create the batch's event";
        delete b;
        return FESTUNG_ECUDA;
    }
    for (int q = 0; q < nprob; ++q) {
        const festung_ctx *c = problems[q];
        BatchGroup *hit = nullptr;
        for (auto &g : b->groups) {
            const festung_ctx *f = b->probs[g.members[0]];
            if (f->p == c->p && f->qT == c->qT && f->eta == c->eta) hit = &g;
        }
        if (!hit) {
            b->groups.emplace_back();
            hit = &b->groups.back();
        }
        hit->members.push_back(q);
    }
    *out = b;
    return FESTUNG_OK;
}

int festung_batch_set_stream(festung_batch *b, void *stream) {
    if (!b) return FESTUNG_EINVAL;
    b->stream = (cudaStream_t)stream;  // the groups run on their own streams, ordered after this one
    return FESTUNG_OK;
}

int festung_batch_step(festung_batch *b, double dt, const festung_step_opts *opts, festung_step_info *infos) {
    if (!b) return FESTUNG_EINVAL;
    festung_step_opts o;
    if (!step_options(opts, o) || !(dt > 0.0) || o.prec != FESTUNG_MIXED) {
        b->err = "bad batch step arguments (FESTUNG_MIXED only)";
        return FESTUNG_EINVAL;
    }
    if (b->mode == FESTUNG_BATCH_CONCURRENT) return batch_step_concurrent(b, dt, o, infos);
    for (auto &g : b->groups) {
        const int rc = ensure_built(b, g);
        if (rc) return rc;
    }
    // the groups run concurrently, each on its own stream and host thread, after the work
    // already queued on the batch's stream; the batch's stream then waits for all of them
    const size_t ng = b->groups.size();
    std::vector<int> rcs(ng, FESTUNG_OK);
    if (cudaEventRecord(b->start_ev, b->stream) != cudaSuccess) {
        b->err = "CUDA: cannot record on the batch's stream";
        return FESTUNG_ECUDA;
    }
    for (auto &g : b->groups) {
        g.err.clear();
        cudaStreamWaitEvent(g.stream, b->start_ev, 0);
    }
    auto run = [&](size_t i) {
        cudaSetDevice(b->device);
        rcs[i] = solve_group(b, b->groups[i], dt, o, infos);
    };
    std::vector<std::thread> threads;
    size_t started = 1;
    try {
        for (; started < ng; ++started) threads.emplace_back(run, started);
    } catch (...) {
        // no more host threads: the groups that did not start are stepped here in turn
    }
    run(0);
    for (size_t i = started; i < ng; ++i) run(i);
    for (auto &t : threads) t.join();
    for (auto &g : b->groups) {
        cudaEventRecord(g.done_ev, g.stream);
        cudaStreamWaitEvent(b->stream, g.done_ev, 0);
    }
    for (size_t i = 0; i < ng; ++i)
        if (rcs[i]) {
            BatchGroup &g = b->groups[i];
            b->err = !g.err.empty() && rcs[i] != FESTUNG_ECUDA ? g.err : g.u->err;
            return rcs[i];
        }
    return FESTUNG_OK;
}

int festung_batch_launch_count(const festung_batch *b, int64_t *n) {
    if (!b || !n) return FESTUNG_EINVAL;
    *n = b->member_launches.load();
    for (const auto &g : b->groups)
        if (g.u) *n += g.u->launches;
    return FESTUNG_OK;
}

int festung_batch_set_mode(festung_batch *b, int mode, int workers) {
    if (!b) return FESTUNG_EINVAL;
    if ((mode != FESTUNG_BATCH_UNION && mode != FESTUNG_BATCH_CONCURRENT) || workers < 0 || workers > 64) {
        b->err = "bad batch mode or worker count";
        return FESTUNG_EINVAL;
    }
    b->mode = mode;
    b->workers = workers ? workers : default_workers();
    return FESTUNG_OK;
}

const char *festung_batch_last_error(const festung_batch *b) { return b ? b->err.c_str() : g_create_err.c_str(); }

void festung_batch_destroy(festung_batch *b) {
    if (!b) return;
    for (auto &g : b->groups) free_group(g);
    for (size_t i = 0; i < b->wstreams.size(); ++i) {
        cudaStreamSynchronize(b->wstreams[i]);
        cudaStreamDestroy(b->wstreams[i]);
        cudaEventDestroy(b->wev[i]);
        cudaEventDestroy(b->wdone[i]);
    }
    if (b->start_ev) cudaEventDestroy(b->start_ev);
    delete b;
}

}  // extern "C"
