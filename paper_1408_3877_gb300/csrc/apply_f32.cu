// FP32 instantiations of the operator kernels (inner iterations of the mixed solve).
#include "dispatch.h"
#include "ldg_kernels.cuh"
#include "ops.h"

namespace festung {

template <>
void launch_apply<float>(const festung_ctx *c, const float *x, float *y, float *Z1, float *Z2, float tau,
                         const int *skip, cudaStream_t st) {
    const int grid = elem_grid(c);
    c->launches += 2;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        k_flux<float, N, R2, R1><<<grid, 256, 0, st>>>(x, Z1, Z2, c->fB, c->dNbr, c->K, c->fTab, skip);
        k_apply<float, N, R2, R1, MODE_APPLY><<<grid, 256, 0, st>>>(x, Z1, Z2, c->fD, y, c->fB, c->dNbr, c->K, tau,
                                                                    (float)c->eta, c->fTab, nullptr, nullptr,
                                                                    nullptr, skip);
    });
}

}  // namespace festung
