// Internal interface of the solver translation units (festung.cu for single problems,
// batch.cu for batches): a context's workspace, the error macro of the host code and the
// steps of a solve that a batch reuses.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

#include "dfloat.cuh"
#include "festung.h"
#include "internal.h"
#include "krylov.cuh"

namespace festung {

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

template <typename T>
inline Vecs<T> &vecs(festung_ctx *c);
template <>
inline Vecs<double> &vecs<double>(festung_ctx *c) { return c->ws->d; }
template <>
inline Vecs<float> &vecs<float>(festung_ctx *c) { return c->ws->f; }
template <typename T>
inline const T *geomB(const festung_ctx *c);
template <>
inline const double *geomB<double>(const festung_ctx *c) { return c->dB; }
template <>
inline const float *geomB<float>(const festung_ctx *c) { return c->fB; }

// the grid-stride loop over the K triangles of an element-wise kernel
#define ELEM_LOOP(k) for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x)

// host code of a context: return the festung status of a failed CUDA call, with its
// message in the context
#define FCK(call)                                                                  \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            c->err = std::string(#call) + ": " + cudaGetErrorString(e_);           \
            return e_ == cudaErrorMemoryAllocation ? FESTUNG_ENOMEM : FESTUNG_ECUDA; \
        }                                                                          \
    } while (0)

constexpr int CHUNK = 8;  // Krylov iterations per pass of a solve's captured loop body

// message of the last failed festung_mesh_create / festung_batch_create of this thread
std::string &create_error();

// blocks of a grid-stride element-wise kernel over n values
int small_grid(int64_t n, const festung_ctx *c);
// the context's workspace (reduction buffers, scalars, host mirrors), made at first use
int ensure_ws(festung_ctx *c);
// the mesh order (tiles, halos, neighbour slots) of a context on the device
cudaError_t upload_mesh(festung_ctx *c, const MeshOrder &mo);
// time the FP32 apply for tile sizes 96..256 and keep the fastest (*chosen)
int autotune_tiles(festung_ctx *c, int *chosen);
// y = S x in double-float arithmetic for an FP64 x (result in ws->ydf, and in y if given)
int apply_df(festung_ctx *c, const double *x, double *y, double dt, cudaStream_t st);
// r = b - S x (V.b, V.r of the FP64 vectors) with S x in double-float arithmetic; the
// partials of ||r||^2, ||b||^2 in ws->part
int residual_df(festung_ctx *c, const double *x, double dt, cudaStream_t st);
// out[0..np) = the sums of np partial slots of nblk blocks
void launch_fin_sums(festung_ctx *c, double *out, const double *part, int nblk, int np, cudaStream_t st);
// false (with the message in the context) before festung_setup
bool ready(festung_ctx *c);
// the N x K vectors of a precision (the Krylov ones if krylov), made at first use
template <typename T>
int alloc_vecs(festung_ctx *c, Vecs<T> &V, bool krylov);
// step options with the defaults of festung_step; false if out of range
bool step_options(const festung_step_opts *opts, festung_step_opts &o);
// right-hand side, preconditioner build (or reuse) and initial guess of a solve
int prepare_solve(festung_ctx *c, double dt, bool stationary, bool mixed);
// join the preconditioner build of prepare_solve
int finish_precond(festung_ctx *c);
// C <- the solution; a time step also shifts the history of the extrapolation
int commit_solution(festung_ctx *c, double dt, bool stationary);
// one implicit-Euler step (mass = 1) or the stationary problem (mass = 0, dt = 1)
int solve_system(festung_ctx *c, double dt, double mass, const festung_step_opts *opts, festung_step_info *info);

}  // namespace festung
