// FP64 instantiations of the operator kernels and the right-hand side.
#include "dispatch.h"
#include "ldg_kernels.cuh"
#include "ops.h"

namespace festung {

template <>
void launch_apply<double>(const festung_ctx *c, const double *x, double *y, double *Z1, double *Z2, double tau,
                          const int *skip, cudaStream_t st) {
    const int grid = elem_grid(c);
    c->launches += 2;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        k_flux<double, N, R2, R1><<<grid, 256, 0, st>>>(x, Z1, Z2, c->dB, c->dNbr, c->K, c->dTab, skip);
        k_apply<double, N, R2, R1, MODE_APPLY><<<grid, 256, 0, st>>>(x, Z1, Z2, c->dD, y, c->dB, c->dNbr, c->K, tau,
                                                                     c->eta, c->dTab, nullptr, nullptr, nullptr,
                                                                     skip);
    });
}

void launch_rhs(const festung_ctx *c, double *W1, double *W2, double *b, double tau, cudaStream_t st) {
    const int grid = elem_grid(c);
    c->launches += 2;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        k_dirichlet_lift<double, N, R2, R1><<<grid, 256, 0, st>>>(W1, W2, c->dB, c->dNbr, c->K, c->dTab, c->dCD);
        k_apply<double, N, R2, R1, MODE_RHS><<<grid, 256, 0, st>>>(c->dC, W1, W2, c->dD, b, c->dB, c->dNbr, c->K,
                                                                   tau, c->eta, c->dTab, c->dF, c->dCD, c->dGN,
                                                                   nullptr);
    });
}

template <>
void launch_precond<double>(const festung_ctx *c, const float *P, const double *x, double *y, double *part, int nblk,
                            const int *skip, cudaStream_t st) {
    c->launches += 1;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto, auto) {
        constexpr int N = decltype(n_)::value;
        k_precond<double, N><<<part ? nblk : elem_grid(c), 256, 0, st>>>(P, x, y, c->K, part, skip);
    });
}

}  // namespace festung
