// Launchers of the operator kernels (defined in apply_f64.cu / apply_f32.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "dfloat.cuh"
#include "krylov.cuh"

namespace festung {

// y = S x of the step operator (E1) with time step tau, one fused pass per tile (the
// flux unknowns stay in shared memory; Z1, Z2 are not used).  skip: optional device flag; when it is non-zero at
// launch the kernels return immediately (early exit inside captured graphs).
template <typename T>
void launch_apply(const festung_ctx *c, const T *x, T *y, T *Z1, T *Z2, T tau, const int *skip,
                  cudaStream_t st);

// y = S x followed by the reductions of one BiCGStab step, epi = 1 (FUSED_EPI_ALPHA):
// e1 = r0, (r0, y) -> alpha; epi = 2 (FUSED_EPI_OMEGA): e1 = s, e2 = r0, (y, s), (y, y),
// (r0, s), (r0, y) -> omega, rho, beta.  FP32: fused into the end of the apply (part
// holds 4 partials per tile); FP64: a reduction pass of its own after the apply (part
// holds 4 partials per block of that pass).
// bv: the union of a batch (per-problem scalars sc[q] and sums; FP32 only), or the
// default view of a single problem.
template <typename T>
void launch_apply_bicg(const festung_ctx *c, const T *x, T *y, T tau, int epi, const T *e1, const T *e2,
                       double *part, KScal *sc, unsigned int *counter, const int *skip, cudaStream_t st,
                       const BatchView &bv = BatchView());

// y = S x in double-float arithmetic (dfloat.cuh) from the double-float copies of D,
// the geometry and the tables (c->xD, c->xB, c->xTab); x, y: N x K double-floats.
void launch_apply_df(const festung_ctx *c, const dfloat *x, dfloat *y, double tau, cudaStream_t st);

// The same y = S x in two passes: k_flux writes Z^1, Z^2 to the N x K scratch arrays
// Z1, Z2 in global memory, k_apply reads them back.
template <typename T>
void launch_apply_twopass(const festung_ctx *c, const T *x, T *y, T *Z1, T *Z2, T tau, const int *skip,
                          cudaStream_t st);

// b of (E2) in FP64 from C^n, F, the boundary data and D; W1, W2: N x K scratch
// (the Dirichlet lift M^{-1} J_D^m).
void launch_rhs(const festung_ctx *c, double *W1, double *W2, double *b, double tau, cudaStream_t st);

// The flux unknowns of eq. timeDepSystem, block rows 1-2, in two parts (FP64, N x K):
// launch_flux: Z^m = -M^{-1} B_m x;  launch_lift: W^m = M^{-1} J_D^m from the context's c_D.
void launch_flux(const festung_ctx *c, const double *x, double *Z1, double *Z2, cudaStream_t st);
void launch_lift(const festung_ctx *c, double *W1, double *W2, cudaStream_t st);

int elem_grid(const festung_ctx *c);

// Blocks of the FP32 fused apply that run at once on the device (resident blocks per
// SM times SMs) for tiles with nslot shared-memory slots, and the dynamic shared
// memory of one block of the FP32 or FP64 kernel.
int fused_resident_blocks(const festung_ctx *c, int nslot);
size_t fused_smem_bytes(const festung_ctx *c, int nslot, bool fp64);

// The FP32 fused apply with the reference tables rounded to BF16 (FESTUNG_BF16TAB): plain
// and with the BiCGStab epilogue, as launch_apply / launch_apply_bicg.  The FP32
// launchers call these while the context's tab_bf16 is set.
void launch_apply_bf16tab(const festung_ctx *c, const float *x, float *y, float tau, const int *skip,
                          cudaStream_t st);
void launch_apply_bicg_bf16tab(const festung_ctx *c, const float *x, float *y, float tau, int epi, const float *e1,
                               const float *e2, double *part, KScal *sc, unsigned int *counter, const int *skip,
                               cudaStream_t st, const BatchView &bv);

// Reference tables of the context's (p, quadrature) into the constant bank of the FP64
// and double-float fused apply kernels (the FP32 kernels take them as compile-time
// constants, festung_tables_gen.h).
cudaError_t upload_tables_f64(const festung_ctx *c);
cudaError_t upload_tables_df(const festung_ctx *c);

// Block-Jacobi preconditioner: Pinv <- inverse of the N x N diagonal blocks of S (E1),
// built in FP32 (scratch P, layout [(i N + j) K + k]) from the FP32 copies of geometry,
// tables and D, inverted in FP32 (Gauss-Jordan, partial pivoting, one warp per block) and
// stored in BF16 (16-byte chunks [q][K]).  flags (device int) gets bit 0 set if a block
// is singular.
void launch_blockjacobi(const festung_ctx *c, float *P, __nv_bfloat16 *Pinv, double tau, int *flags,
                        cudaStream_t st);

// The vectors of an FP32 BiCGStab solve (N x K each; inv: 1 / (2|T_k|), length K); p2,
// v2: second buffers of p and v for the persistent kernel, which alternates them.
struct BicgVecs32 {
    float *x, *r, *p, *v, *ph, *s, *sh, *t, *p2, *v2;
    const float *r0, *inv;
};

// True if launch_bicg_persistent serves this context (p <= 1, FP32 tables).
bool bicg_persistent_supported(const festung_ctx *c);

// The BiCGStab iterations of an FP32 solve as one persistent cooperative kernel
// (bicg_persist.cu): from the state in *sc (k_fin_init and the vectors r, r0, p, v set
// up as for the graph of iterations) until the iteration is done or sc->iter reaches
// max_iter; *sc is then left as that graph leaves it (an update owed to x when pending
// or sconv is set); p and v are left in either buffer.  ps: 256 bytes of device memory
// for the scalars while the kernel runs.  part: partials, 6 floats per
// block of at most part_blocks blocks; bar: 2 counters and err: a flag (both zeroed
// here) of the grid barrier; err ends up non-zero if a barrier wait gave up.  bar_extra
// > 0 (testing only) makes every barrier wait for that many blocks more than the grid has,
// so that the waits run out.  cudaErrorNotSupported: the context's
// order or the device cannot run it (the caller uses the graph instead).
cudaError_t launch_bicg_persistent(const festung_ctx *c, const BicgVecs32 &v, const __nv_bfloat16 *P, float tau,
                                   KScal *sc, void *ps, float *part, int part_blocks, unsigned int *bar, int *err,
                                   int max_iter, int bar_extra, cudaStream_t st);

}  // namespace festung
