// Launchers of the operator kernels (defined in apply_f64.cu / apply_f32.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace festung {

// y = S x of the step operator (E1) with time step tau; Z1, Z2: N x K scratch for the
// eliminated flux unknowns.  skip: optional device flag; when it is non-zero at
// launch the kernels return immediately (early exit inside captured graphs).
template <typename T>
void launch_apply(const festung_ctx *c, const T *x, T *y, T *Z1, T *Z2, T tau, const int *skip,
                  cudaStream_t st);

// b of (E2) in FP64 from C^n, F, the boundary data and D; W1, W2: N x K scratch
// (the Dirichlet lift M^{-1} J_D^m).
void launch_rhs(const festung_ctx *c, double *W1, double *W2, double *b, double tau, cudaStream_t st);

int elem_grid(const festung_ctx *c);

}  // namespace festung
