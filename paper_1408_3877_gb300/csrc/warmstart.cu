// Features of the learned warm start (festung_warmstart_features): per triangle the
// coefficient field and the scaled residual of the current state on the triangle and its
// three neighbours, and the loss weights from the diagonal blocks of S.  The network
// itself is mlp.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "festung.h"
#include "internal.h"
#include "krylov.cuh"
#include "krylov_kernels.cuh"
#include "ops.h"
#include "solver.h"

using namespace festung;

namespace {

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

}  // namespace

extern "C" {

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
    if ((rc = residual_df(c, c->dC, dt, st))) return rc;
    k_ws_sums<<<w.nblk, RED_THREADS, 0, st>>>(K, c->N, V.r, c->dD, c->dB, w.part);
    ++c->launches;
    launch_fin_sums(c, w.res, w.part, w.nblk, 2, st);
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

}  // extern "C"
