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
#include "solver.h"

using namespace festung;

namespace festung {

// message of the last failed festung_mesh_create / festung_batch_create of this thread
std::string &create_error() {
    thread_local std::string e;
    return e;
}

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

int elem_grid(const festung_ctx *c) {
    const int64_t need = (c->K + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)c->num_sms * 8));
}

}  // namespace festung

namespace {


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
}  // namespace

namespace festung {

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
template int alloc_vecs<double>(festung_ctx *, Vecs<double> &, bool);
template int alloc_vecs<float>(festung_ctx *, Vecs<float> &, bool);

}  // namespace festung

namespace {

template <typename T>
void free_vecs(Vecs<T> &V) {
    T *ptrs[] = {V.Z1, V.Z2, V.r, V.r0, V.p, V.ph, V.v, V.s, V.sh, V.t, V.x, V.b, V.inv};
    for (T *q : ptrs)
        if (q) cudaFree(q);
    V = Vecs<T>();
}

}  // namespace

namespace festung {

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

}  // namespace festung

namespace {

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

}  // namespace

namespace festung {

int small_grid(int64_t n, const festung_ctx *c) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8));
}

}  // namespace festung

namespace {

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

}  // namespace

namespace festung {

bool ready(festung_ctx *c) {
    if (!c) return false;
    if (c->p < 0) {
        c->err = "festung_setup has not been called";
        return false;
    }
    return true;
}

}  // namespace festung

namespace {

// ---------------------------------------------------------------------------
// Krylov drivers
// ---------------------------------------------------------------------------

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
// x_zero: x is 0 on entry.  Returns iterations in *iters and the final ||r||^2, ||b||^2:
// with verify, ||r||^2 of the true residual b - S x (the solve restarts when the recursion
// drifted from it by more than 10x); without, the recursive one.
template <typename T>
int krylov_solve(festung_ctx *c, int solver, double tau, double tol, int max_iter, bool x_zero, int *iters,
                 double *r2, double *b2, bool *conv, bool reweight = false, double *relres0 = nullptr,
                 bool verify = true) {
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
        // enqueue the iterations (the persistent kernel, or the graph's loop) and behind them
        // the copies of the scalars and of the kernel's flag or the loop's pass count, read
        // after one wait; a solve that is already done returns at once in either form
        int launched = 0;  // 1: persistent kernel, 2: graph
        auto enqueue = [&](int iter_now) -> int {
            launched = 0;
            if (persistent) {
                if constexpr (std::is_same<T, float>::value) {
                    // Z1, Z2 (not used by the fused applies) serve as the second p and v buffers
                    const BicgVecs32 bv{V.x, V.r, V.p, V.v, V.ph, V.s, V.sh, V.t, V.Z1, V.Z2, V.r0, V.inv};
                    const cudaError_t e = launch_bicg_persistent(c, bv, w.use_P ? w.Pb : nullptr, (float)tau, w.scal,
                                                                 w.pscal, w.ppart, w.pcap, w.pbar, w.perr,
                                                                 max_iter - total, c->test_barrier_extra, st);
                    if (e == cudaErrorNotSupported || e == cudaErrorCooperativeLaunchTooLarge) {
                        // the device cannot hold the grid: this context keeps to the graph
                        (void)cudaGetLastError();
                        persistent = false;
                        c->persist_refused = true;
                        if ((rc = build_graph())) return rc;
                    } else {
                        FCK(e);
                        ++c->launches;
                        FCK(cudaMemcpyAsync(w.h_perr, w.perr, sizeof(int), cudaMemcpyDeviceToHost, st));
                        launched = 1;
                    }
                }
            }
            if (!launched) {
                const int max_chunks = std::max(1, (max_iter - total - iter_now + CHUNK - 1) / CHUNK);
                k_loop_init<<<1, 1, 0, st>>>(w.loopctl, max_chunks); ++c->launches;
                FCK(cudaGraphLaunch(gc.exec, st));
                FCK(cudaMemcpyAsync(w.h_loopctl, w.loopctl, sizeof(int), cudaMemcpyDeviceToHost, st));
                launched = 2;
            }
            FCK(cudaMemcpyAsync(w.h_scal, w.scal, sizeof(KScal), cudaMemcpyDeviceToHost, st));
            return FESTUNG_OK;
        };
        if ((rc = enqueue(0))) return rc;
        while (true) {
            FCK(cudaStreamSynchronize(st));
            if (launched == 1 && *w.h_perr) {
                c->err = "persistent BiCGStab kernel: a grid barrier wait gave up";
                return FESTUNG_ECUDA;
            }
            if (launched == 2) c->launches += gc.nodes * (int64_t)*w.h_loopctl;
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
                } else if (!verify) {
                    *conv = h.r2 <= tol * tol * h.b2;
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
            if ((rc = enqueue(h.iter))) return rc;
        }
        if (!brk && !drift) break;
        // breakdown or drift: restart from the current iterate
    }
    *iters = total;
    return FESTUNG_OK;
}

}  // namespace

namespace festung {

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

// r = b - S x of the context's FP64 vectors (V.b, r into V.r) with S x in double-float
// arithmetic; the partials of ||r||^2, ||b||^2 go to ws->part
int residual_df(festung_ctx *c, const double *x, double dt, cudaStream_t st) {
    int rc = apply_df(c, x, nullptr, dt, st);
    if (rc) return rc;
    Workspace &w = *c->ws;
    k_residual_df<<<w.nblk, RED_THREADS, 0, st>>>(c->K * c->N, w.d.b, w.ydf, w.d.r, w.part);
    ++c->launches;
    FCK(cudaGetLastError());
    return FESTUNG_OK;
}

// out[0..np) = sums of np partial slots of nblk blocks (one block)
void launch_fin_sums(festung_ctx *c, double *out, const double *part, int nblk, int np, cudaStream_t st) {
    k_fin_sums<<<1, 1024, 0, st>>>(out, part, nblk, np);
    ++c->launches;
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
    std::vector<int32_t> lifted;
    for (int64_t k = 0; k < K; ++k)
        if (mo.lift[k] & 2) lifted.push_back((int32_t)k);
    c->nLift = (int64_t)lifted.size();
    if ((e = cudaMalloc(&c->dLiftList, std::max<size_t>(1, lifted.size()) * sizeof(int32_t))) != cudaSuccess) return e;
    if (!lifted.empty() &&
        (e = cudaMemcpy(c->dLiftList, lifted.data(), lifted.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
        return e;
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

}  // namespace festung

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
    create_error().clear();
    if (!out) {
        create_error() = "out is NULL";
        return FESTUNG_EINVAL;
    }
    *out = nullptr;
    if (!coordV || !V0T || !bdr_type || numV < 3 || numT < 1) {
        create_error() = "NULL array or empty mesh";
        return FESTUNG_EINVAL;
    }
    festung_ctx *c = new (std::nothrow) festung_ctx();
    if (!c) return FESTUNG_ENOMEM;
    c->K = numT;
    c->numV = numV;
    std::vector<int32_t> nbr;
    int rc = build_mesh(coordV, numV, V0T, numT, bdr_type, c->hB, nbr, c->err);
    if (rc) {
        create_error() = c->err;
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
        create_error() = std::string("CUDA: ") + cudaGetErrorString(e);
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

namespace festung {

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
                // (its result only starts the sweep, which the refinement verifies: no true
                // residual of its own)
                rc = krylov_solve<float>(cc, csolver, dt, 1e-2, 2000, !c->coarse_warm, &cit, &cr2, &cb2, &ccin,
                                         false, nullptr, false);
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

}  // namespace festung

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
    if (!c) return create_error().c_str();
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

int festung_test_barrier_timeout(festung_ctx *c, int enable) {
    if (!c) return FESTUNG_EINVAL;
    if (enable != 0 && enable != 1) {
        c->err = "enable must be 0 or 1";
        return FESTUNG_EINVAL;
    }
    c->test_barrier_extra = enable;
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
    void *mesh_ptrs[] = {c->dB, c->fB, c->dNbr, c->dPerm, c->dSlot, c->dHaloPtr, c->dHalo, c->dHaloSlot, c->dLift,
                         c->dLiftList};
    for (void *q : mesh_ptrs)
        if (q) cudaFree(q);
    delete c;
}

}  // extern "C"
