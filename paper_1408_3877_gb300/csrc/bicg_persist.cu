// The iterations of an FP32 BiCGStab solve in one persistent kernel (p <= 1).
//
// At p = 1 a tile of 256 triangles is little work: each of the four kernels of an
// iteration of the graph form (the update of x, r, p and ph = P^{-1} p; v = S ph with
// (r0, v); s = r - alpha v and sh = P^{-1} s with (s, s); t = S sh with its dot products)
// spends most of its time on launch, on a chain of dependent loads and on the serial
// tail of its reduction.  This kernel runs an iteration as two phases of one
// cooperative launch, each block keeping its tiles (one tile per block when the grid
// holds them all):
//   A  the owed x += alpha ph + omega sh and r = s - omega t, p = r + beta (p - omega v),
//      ph = P^{-1} p for the block's own triangles, then v = S ph and (r0, v);
//   B  s = r - alpha v, sh = P^{-1} s and (s, s) for its own triangles, then t = S sh,
//      (t, s), (t, t), (r0, s), (r0, t).
// The apply of a tile needs ph (sh) on its halo too, which other blocks own and write in
// the same phase: the block computes those values itself from the vectors of the
// previous phase, with the owners' arithmetic (the same function, explicit roundings),
// so the values are bit-identical.  p and v alternate between two buffers, so that the
// previous iteration's values stay readable while the owners write the new ones.  Two
// grid-wide barriers per iteration remain, after the two reductions: the last block to
// arrive sums the blocks' partials (compensated, in a fixed order) and updates the
// scalars in device memory before it releases the others.
#include <algorithm>

#include "dispatch.h"
#include "ldg_fused.cuh"
#include "ops.h"

namespace festung {

namespace {

// A waiting block gives up a barrier after a second (device global timer), or after
// 2^24 polls whatever the timer says.  Only a grid that is not resident as a whole could
// reach it, which the cooperative launch rules out (festung_test_barrier_timeout makes
// the waits run out on purpose, for the test of this path).
constexpr unsigned long long kWaitLimitNs = 1000000000ull;
constexpr unsigned int kSpinLimit = 1u << 24;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

struct PersistArgs {
    BicgVecs32 v;
    const __nv_bfloat16 *P;  // BF16 inverse blocks (k_blockinv layout), or null: v.inv
    const float *D, *B, *tab;
    const int32_t *nbr;
    const int16_t *slot;
    const int32_t *halo_ptr, *halo;
    const int16_t *halo_slot;
    int K, TE, NS, ntiles;
    float tau, eta, mass;
    KScal *sc;
    void *ps;           // the iteration's scalars while it runs (PScal)
    float *part;        // 6 x gridDim block partials: (r0, v) | (t, s), (t, t), (r0, s), (r0, t), (s, s)
    unsigned int *bar;  // [0] arrivals, [1] generation
    int *err;
    int max_iter;
    int bar_extra;  // testing only: blocks a barrier waits for beyond the grid
};

// The scalars of the iteration while the kernel runs, in FP32 and double-float (the
// FP64 pipe of this device would put a microsecond of divisions on the path of every
// reduction): the step sizes are FP32 values in the vector updates anyway, and the
// quantities formed by cancellation, rho = (r0, r) and the recursive ||r||^2 =
// (s, s) - omega (t, s), keep about 48 bits.  Converted from and to KScal once per launch.
struct PScal {
    dfloat rho, ss, r2, tol2b2;  // tol2b2 = tol^2 ||b||^2
    float alpha, omega, beta, pad;
    int iter, done, sconv, pending, breakdown, first, pad2, pad3;
};
static_assert(sizeof(PScal) <= 256 && sizeof(PScal) % 16 == 0, "PScal fits the workspace slot");

__device__ __forceinline__ dfloat df_of(double v) { return dfloat(v); }
__device__ __forceinline__ bool df_le(dfloat a, dfloat b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }

__device__ void pscal_from(const KScal &k, PScal &p) {
    p.rho = df_of(k.rho);
    p.ss = df_of(k.ss);
    p.r2 = df_of(k.r2);
    p.tol2b2 = df_of(k.tol2 * k.b2);
    p.alpha = (float)k.alpha;
    p.omega = (float)k.omega;
    p.beta = (float)k.beta;
    p.iter = k.iter;
    p.done = k.done;
    p.sconv = k.sconv;
    p.pending = k.pending;
    p.breakdown = k.breakdown;
    p.first = k.first;
}

__device__ void pscal_to(const PScal &p, KScal *k) {
    k->rho = (double)p.rho;
    k->ss = (double)p.ss;
    k->r2 = (double)p.r2;
    k->alpha = p.alpha;
    k->omega = p.omega;
    k->beta = p.beta;
    k->iter = p.iter;
    k->done = p.done;
    k->sconv = p.sconv;
    k->pending = p.pending;
    k->breakdown = p.breakdown;
    k->first = p.first;
}

// after v = S ph: alpha = rho / (r0, v) (bicg_alpha_scalars in FP32 / double-float)
__device__ void pscal_alpha(PScal &p, dfloat r0v) {
    if (!(fabsf(r0v.hi) > 1e-37f) || !isfinite(r0v.hi)) {
        p.breakdown = 1;
        p.done = 1;
    } else {
        p.alpha = p.rho.hi / r0v.hi;
    }
    p.first = 0;
    p.pending = 0;
}

// after t = S sh: converged on s, or omega, the recursive ||r||^2, rho and beta
// (bicg_omega_scalars in FP32 / double-float)
__device__ void pscal_omega(PScal &p, dfloat ts, dfloat tt, dfloat r0s, dfloat r0t, dfloat ss) {
    p.ss = ss;
    if (df_le(ss, p.tol2b2)) {
        p.sconv = 1;  // x += alpha ph is left to the caller
        p.r2 = ss;
        p.iter += 1;
        p.done = 1;
        return;
    }
    if (!(tt.hi > 0.0f) || !isfinite(ts.hi) || ts.hi == 0.0f || !isfinite(r0s.hi) || !isfinite(r0t.hi)) {
        p.breakdown = 1;
        p.done = 1;
        return;
    }
    const float omega = ts.hi / tt.hi;
    const dfloat w(omega, 0.0f);
    const dfloat rho_new = r0s - w * r0t;
    dfloat r2 = ss - w * ts;
    if (r2.hi < 0.0f) r2 = dfloat(0.0f, 0.0f);
    p.omega = omega;
    p.iter += 1;
    p.r2 = r2;
    p.pending = 1;
    if (df_le(r2, p.tol2b2)) {
        p.done = 1;
    } else if (!(fabsf(rho_new.hi) > 1e-37f) || !isfinite(rho_new.hi)) {
        p.breakdown = 1;
        p.done = 1;
    } else {
        p.beta = (rho_new.hi / p.rho.hi) * (p.alpha / omega);
        p.rho = rho_new;
    }
}

// y = P_k q (or q / (2|T_k|) without blocks), every rounding explicit: the owner of a
// triangle and the blocks whose halo holds it compute the same bits
template <int N>
__device__ __forceinline__ void prec_apply(const PersistArgs &a, int k, const float (&q)[N], float (&y)[N]) {
    if (a.P) {
        constexpr int NQ = (N * N + 7) / 8;
#pragma unroll
        for (int i = 0; i < N; ++i) y[i] = 0.0f;
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(a.P) + (int64_t)c * a.K + k);
            const __nv_bfloat16 *b = reinterpret_cast<const __nv_bfloat16 *>(&raw);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int e = 8 * c + t;
                if (e < N * N) y[e / N] = __fmaf_rn(__bfloat162float(b[t]), q[e % N], y[e / N]);
            }
        }
    } else {
        const float iv = a.v.inv[k];
#pragma unroll
        for (int i = 0; i < N; ++i) y[i] = __fmul_rn(q[i], iv);
    }
}

// Phase A values of triangle e: r = s - omega t (r itself in the first iteration) and
// p = r + beta (p_old - omega v_old)
template <int N>
__device__ __forceinline__ void phase_a_rp(const PersistArgs &a, int e, bool first, float omega, float beta,
                                           const float *pin, const float *vin, float (&r)[N], float (&p)[N]) {
    const BicgVecs32 &V = a.v;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int i = j * a.K + e;
        r[j] = first ? __ldcg(V.r + i) : __fsub_rn(__ldcg(V.s + i), __fmul_rn(omega, __ldcg(V.t + i)));
        p[j] = __fadd_rn(r[j], __fmul_rn(beta, __fsub_rn(__ldcg(pin + i), __fmul_rn(omega, __ldcg(vin + i)))));
    }
}

// Phase B value of triangle e: s = r - alpha v (v: this iteration's buffer)
template <int N>
__device__ __forceinline__ void phase_b_s(const PersistArgs &a, int e, float alpha, const float *v, float (&s)[N]) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int i = j * a.K + e;
        s[j] = __fsub_rn(__ldcg(a.v.r + i), __fmul_rn(alpha, __ldcg(v + i)));
    }
}

// x source of the applies (the interface of LoadX): the value of a slot is kept in
// shared memory (stash, N per slot; the tile's own slots are filled by the owner step
// before the apply), a triangle outside tile and halo is computed from the vectors.
// PH 0: ph of phase A (pin, vin: the previous p and v); PH 1: sh of phase B (vin: the
// v of this iteration).
template <int N, int PH>
struct PhaseSrc {
    const PersistArgs *a;
    float *stash;
    int TE;
    bool first_it;  // the first iteration (r itself, nothing owed)
    float alpha, omega, beta;
    const float *pin, *vin;
    __device__ __forceinline__ void compute(int e, float (&x)[N]) const {
        float q[N];
        if constexpr (PH == 0) {
            float r[N];
            phase_a_rp<N>(*a, e, first_it, omega, beta, pin, vin, r, q);
        } else {
            phase_b_s<N>(*a, e, alpha, vin, q);
        }
        prec_apply<N>(*a, e, q, x);
    }
    __device__ __forceinline__ void first(int e, int slot, float (&x)[N]) const {
        if (slot < TE) {
            get(e, slot, x);
        } else {
            compute(e, x);
#pragma unroll
            for (int j = 0; j < N; ++j) stash[slot * N + j] = x[j];
        }
    }
    __device__ __forceinline__ void get(int e, int slot, float (&x)[N]) const {
        if (slot >= 0) {
#pragma unroll
            for (int j = 0; j < N; ++j) x[j] = stash[slot * N + j];
        } else {
            compute(e, x);
        }
    }
    __device__ __forceinline__ float comp(int e, int j) const {
        float x[N];
        get(e, -1, x);
        return x[j];
    }
};

__device__ __forceinline__ dfloat shfl_down_df(dfloat a, int o) {
    return dfloat(__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o));
}

// This block's partials part[(slot + q) G + b]: the threads' float sums added in float
// (a block holds a few hundred triangles; the grid's sum is taken in double-float)
template <int ND>
__device__ __forceinline__ void write_partials(const float (&v)[ND], float *part, int slot) {
    __shared__ float ws[ND][FUSED_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int q = 0; q < ND; ++q) {
        float x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) ws[q][wid] = x;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < ND; ++q) {
            float x = lane < nw ? ws[q][lane] : 0.0f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) part[(slot + q) * gridDim.x + blockIdx.x] = x;
        }
    }
}

// Device-scope acquire / release operations of the barrier (PTX memory model): the
// arriving atomic releases the block's writes (cumulatively, after a block barrier) and,
// in the last block, acquires everyone's; the generation bump releases the scalars and
// the polling load acquires them.
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int *p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void red_release_gpu(unsigned int *p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier after a reduction (every block of the grid is resident).  A block
// arrives on bar[0]; in the last block to arrive, every thread adds the ND partial slots
// from `slot` of every blockDim-th block (compensated), the sums go through a
// double-float tree of warps (a fixed order), and thread 0 updates the block's scalars
// with fin(sums), stores them in a.ps, resets bar[0] and advances the generation
// bar[1], which the other blocks poll; they then load the scalars from a.ps.
// Everything written before the barrier is visible after it.  Returns true if some block
// gave up waiting (err set): the caller stops.
template <int ND, typename Fin>
__device__ bool barrier_reduce(const PersistArgs &a, int slot, PScal &ps, Fin fin) {
    __shared__ int last_s, abort_s;
    __shared__ dfloat wsum[ND][FUSED_THREADS / 32];
    __syncthreads();
    unsigned int g = 0;
    if (threadIdx.x == 0) {
        // the current generation: this block saw it advance at its last barrier, and it
        // cannot advance again before this block arrives (a relaxed read suffices)
        g = *(volatile unsigned int *)(a.bar + 1);
        last_s = atom_add_acq_rel_gpu(a.bar, 1u) == gridDim.x - 1 + (unsigned int)a.bar_extra;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    if (last_s) {
        float sm[ND], cp[ND];
#pragma unroll
        for (int q = 0; q < ND; ++q) sm[q] = cp[q] = 0.0f;
        const int G = gridDim.x;
        // Neumaier's compensated summation over blocks b = tid, tid + blockDim, ...; the
        // loads of two rounds are issued together
        for (int b0 = threadIdx.x; b0 < G; b0 += 2 * blockDim.x) {
            float v[2][ND];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int b = b0 + h * blockDim.x;
#pragma unroll
                for (int q = 0; q < ND; ++q) v[h][q] = b < G ? __ldcg(a.part + (slot + q) * G + b) : 0.0f;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int q = 0; q < ND; ++q) {
                    const float t = sm[q] + v[h][q];
                    cp[q] += fabsf(sm[q]) >= fabsf(v[h][q]) ? (sm[q] - t) + v[h][q] : (v[h][q] - t) + sm[q];
                    sm[q] = t;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < ND; ++q) {
            dfloat t = df_two_sum(sm[q], cp[q]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t = t + shfl_down_df(t, o);
            if (lane == 0) wsum[q][wid] = t;
        }
        __syncthreads();
        if (wid == 0) {
            dfloat tot[ND];
#pragma unroll
            for (int q = 0; q < ND; ++q) {
                tot[q] = lane < nw ? wsum[q][lane] : dfloat(0.0f, 0.0f);
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) tot[q] = tot[q] + shfl_down_df(tot[q], o);
            }
            if (lane == 0) {
                fin(tot);
                *reinterpret_cast<PScal *>(a.ps) = ps;
                atomicExch(a.bar, 0u);
                red_release_gpu(a.bar + 1, 1u);
            }
        }
    } else if (threadIdx.x == 0) {
        unsigned int n = 0;
        const unsigned long long t0 = globaltimer_ns();
        while (ld_acquire_gpu(a.bar + 1) == g) {
            if (*(volatile int *)a.err) break;  // another block gave up
            if (++n > 256) {
                __nanosleep(32);
                if ((n & 63) == 0 && (globaltimer_ns() - t0 > kWaitLimitNs || n > kSpinLimit)) {
                    atomicExch(a.err, 1);
                    break;
                }
            }
        }
    }
    if (threadIdx.x == 0) abort_s = *(volatile int *)a.err;
    __syncthreads();
    if (!last_s) {
        // the scalars from a.ps (read past L1)
        static_assert(sizeof(PScal) % 4 == 0, "PScal is read as 32-bit words");
        if (threadIdx.x < sizeof(PScal) / 4)
            reinterpret_cast<int *>(&ps)[threadIdx.x] = __ldcg(reinterpret_cast<const int *>(a.ps) + threadIdx.x);
        __syncthreads();
    }
    return abort_s != 0;
}

template <int N, int R2, int R1>
__global__ void __launch_bounds__(FUSED_THREADS, 4) k_bicg_persistent(const PersistArgs a) {
    __shared__ PScal s;  // the block's copy of the scalars (the same values in every block)
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    float *stash = reinterpret_cast<float *>(dyn_smem + trace_bytes_aligned<float, R1>(a.NS));
    if (threadIdx.x == 0) pscal_from(*a.sc, s);
    __syncthreads();
    if (s.done) return;
    const BicgVecs32 &V = a.v;
    const int G = gridDim.x, i = threadIdx.x, K = a.K;
    const BatchView bv;
    for (int it = 0; it <= a.max_iter; ++it) {
        const bool par = (it & 1) != 0;
        float *pin = par ? V.p2 : V.p, *pout = par ? V.p : V.p2;
        float *vin = par ? V.v2 : V.v, *vout = par ? V.v : V.v2;
        // A: v = S ph, (r0, v) -> alpha
        {
            const bool first = s.first != 0;
            const float alpha = s.alpha, omega = s.omega, beta = s.beta;
            const PhaseSrc<N, 0> src{&a, stash, a.TE, first, alpha, omega, beta, pin, vin};
            float d[1] = {0.0f};
            for (int tile = blockIdx.x; tile < a.ntiles; tile += G) {
                const int k = tile * a.TE + i;
                __syncthreads();
                if (i < a.TE && k < K) {
                    // owner: the owed update of x and r, then p and ph
                    float r[N], p[N], ph[N];
                    if (!first) {
#pragma unroll
                        for (int j = 0; j < N; ++j) {
                            const int e = j * K + k;
                            V.x[e] = __ldcg(V.x + e) + (alpha * __ldcg(V.ph + e) + omega * __ldcg(V.sh + e));
                        }
                    }
                    phase_a_rp<N>(a, k, first, omega, beta, pin, vin, r, p);
                    prec_apply<N>(a, k, p, ph);
#pragma unroll
                    for (int j = 0; j < N; ++j) {
                        const int e = j * K + k;
                        if (!first) V.r[e] = r[j];
                        pout[e] = p[j];
                        V.ph[e] = ph[j];
                        stash[i * N + j] = ph[j];
                    }
                }
                __syncthreads();
                fused_tile<float, N, R2, R1, FUSED_EPI_ALPHA, 0, true>(
                    tile, src, vout, a.D, a.B, a.nbr, a.slot, a.halo_ptr, a.halo, a.halo_slot, K, a.TE, a.NS, a.tau,
                    a.eta, a.mass, a.tab, V.r0, nullptr, nullptr, bv, d);
            }
            write_partials<1>(d, a.part, 0);
        }
        if (barrier_reduce<1>(a, 0, s, [&](const dfloat *sum) { pscal_alpha(s, sum[0]); })) break;
        if (s.done) break;  // breakdown
        // B: t = S sh; (t, s), (t, t), (r0, s), (r0, t), (s, s) -> omega, rho, beta
        {
            const float alpha = s.alpha;
            const PhaseSrc<N, 1> src{&a, stash, a.TE, false, alpha, 0.0f, 0.0f, nullptr, vout};
            float d[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            for (int tile = blockIdx.x; tile < a.ntiles; tile += G) {
                const int k = tile * a.TE + i;
                __syncthreads();
                if (i < a.TE && k < K) {
                    // owner: s and sh
                    float sv[N], sh[N];
                    phase_b_s<N>(a, k, alpha, vout, sv);
                    prec_apply<N>(a, k, sv, sh);
#pragma unroll
                    for (int j = 0; j < N; ++j) {
                        const int e = j * K + k;
                        V.s[e] = sv[j];
                        V.sh[e] = sh[j];
                        stash[i * N + j] = sh[j];
                        d[4] += sv[j] * sv[j];
                    }
                }
                __syncthreads();
                float d4[4] = {d[0], d[1], d[2], d[3]};
                fused_tile<float, N, R2, R1, FUSED_EPI_OMEGA, 0, true>(
                    tile, src, V.t, a.D, a.B, a.nbr, a.slot, a.halo_ptr, a.halo, a.halo_slot, K, a.TE, a.NS, a.tau,
                    a.eta, a.mass, a.tab, V.s, V.r0, nullptr, bv, d4);
#pragma unroll
                for (int q = 0; q < 4; ++q) d[q] = d4[q];
            }
            write_partials<5>(d, a.part, 1);
        }
        if (barrier_reduce<5>(a, 1, s, [&](const dfloat *sum) { pscal_omega(s, sum[0], sum[1], sum[2], sum[3], sum[4]); }))
            break;
        if (s.done || s.iter >= a.max_iter) break;  // the update of x and r stays owed (pending)
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) pscal_to(s, a.sc);
}

}  // namespace

bool bicg_persistent_supported(const festung_ctx *c) {
    return c->N <= 3 && !c->tab_bf16;
}

cudaError_t launch_bicg_persistent(const festung_ctx *c, const BicgVecs32 &v, const __nv_bfloat16 *P, float tau,
                                   KScal *sc, void *ps, float *part, int part_blocks, unsigned int *bar, int *err,
                                   int max_iter, int bar_extra, cudaStream_t st) {
    if (!bicg_persistent_supported(c)) return cudaErrorNotSupported;
    cudaError_t e = cudaErrorNotSupported;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        if constexpr (N <= 3) {
            auto kern = k_bicg_persistent<N, R2, R1>;
            static const bool smem_ok = allow_max_smem(kern);
            (void)smem_ok;
            // traces of the apply, then the stash of N values per slot
            const size_t smem = trace_bytes_aligned<float, R1>(c->nslot) + (size_t)c->nslot * N * sizeof(float);
            int per_sm = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, c->fthreads, smem)) != cudaSuccess)
                return;
            const int ntiles = (int)((c->K + c->TE - 1) / c->TE);
            const int grid = std::min(std::min(ntiles, per_sm * c->num_sms), part_blocks);
            if (grid < 1) {
                e = cudaErrorNotSupported;
                return;
            }
            PersistArgs a;
            a.v = v;
            a.P = P;
            a.D = c->fD;
            a.B = c->fB;
            a.tab = c->fTab;
            a.nbr = c->dNbr;
            a.slot = c->dSlot;
            a.halo_ptr = c->dHaloPtr;
            a.halo = c->dHalo;
            a.halo_slot = c->dHaloSlot;
            a.K = (int)c->K;
            a.TE = c->TE;
            a.NS = c->nslot;
            a.ntiles = ntiles;
            a.tau = tau;
            a.eta = (float)c->eta;
            a.mass = (float)c->mass;
            a.sc = sc;
            a.ps = ps;
            a.part = part;
            a.bar = bar;
            a.err = err;
            a.max_iter = max_iter;
            a.bar_extra = bar_extra;
            if ((e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), st)) != cudaSuccess) return;
            if ((e = cudaMemsetAsync(err, 0, sizeof(int), st)) != cudaSuccess) return;
            void *args[] = {&a};
            e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kern), dim3(grid), dim3(c->fthreads), args,
                                            smem, st);
        }
    });
    return e;
}

}  // namespace festung
