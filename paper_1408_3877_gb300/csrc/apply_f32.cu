// FP32 instantiations of the operator kernels (inner iterations of the mixed solve).
#include <algorithm>

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

void launch_blockjacobi(const festung_ctx *c, float *P, double tau, int *flags, cudaStream_t st) {
    const int64_t need = (c->K + 127) / 128;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)c->num_sms * 8));
    c->launches += 2;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        k_blockdiag<float, N, R2, R1><<<grid, 128, 0, st>>>(P, c->fB, c->dNbr, c->fD, c->K, (float)tau,
                                                            (float)c->eta, c->fTab);
        k_blockinv<N><<<grid, 128, 0, st>>>(P, c->K, flags);
    });
}

template <>
void launch_precond<float>(const festung_ctx *c, const float *P, const float *x, float *y, double *part, int nblk,
                           const int *skip, cudaStream_t st) {
    c->launches += 1;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto, auto) {
        constexpr int N = decltype(n_)::value;
        k_precond<float, N><<<part ? nblk : elem_grid(c), 256, 0, st>>>(P, x, y, c->K, part, skip);
    });
}

}  // namespace festung
