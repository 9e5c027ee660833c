// Batches of independent problems (festung_batch_*): the concurrent mode (every problem its
// own single-problem step, several at a time on streams of their own) and the union mode
// (one joined mesh per order, every problem its own BiCGStab and refinement).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "dfloat.cuh"
#include "dispatch.h"
#include "festung.h"
#include "internal.h"
#include "krylov.cuh"
#include "krylov_kernels.cuh"
#include "ops.h"
#include "solver.h"

using namespace festung;

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
    create_error().clear();
    if (!out || !problems || nprob < 1) {
        create_error() = "NULL argument or empty batch";
        return FESTUNG_EINVAL;
    }
    *out = nullptr;
    for (int q = 0; q < nprob; ++q) {
        if (!problems[q] || problems[q]->p < 0) {
            create_error() = "problem " + std::to_string(q) + " is NULL or not set up";
            return FESTUNG_ESTATE;
        }
        for (int r = 0; r < q; ++r)
            if (problems[r] == problems[q]) {
                create_error() = "problem " + std::to_string(q) + " appears twice";
                return FESTUNG_EINVAL;
            }
    }
    festung_batch *b = new (std::nothrow) festung_batch();
    if (!b) return FESTUNG_ENOMEM;
    b->probs.assign(problems, problems + nprob);
    b->workers = default_workers();
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->start_ev, cudaEventDisableTiming) != cudaSuccess) {
        create_error() = "CUDA: cannot create the batch's event";
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

const char *festung_batch_last_error(const festung_batch *b) { return b ? b->err.c_str() : create_error().c_str(); }

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
