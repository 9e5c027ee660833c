// FP64 instantiations of the operator kernels and the right-hand side.
#include <algorithm>
#include "dispatch.h"
#include "ldg_fused.cuh"
#include "ops.h"

namespace festung {

template <>
void launch_apply<double>(const festung_ctx *c, const double *x, double *y, double *Z1, double *Z2, double tau,
                          const int *skip, cudaStream_t st) {
    (void)Z1;
    (void)Z2;
    const int tiles = (int)((c->K + c->TE - 1) / c->TE);
    c->launches += 1;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        const size_t smem = fused_smem<double, N, R1>(c->nslot, c->TE);
        static const bool smem_ok = allow_max_smem(k_apply_fused<double, N, R2, R1>);
        (void)smem_ok;
        k_apply_fused<double, N, R2, R1><<<tiles, c->fthreads, smem, st>>>(x, y, c->dD, c->dB, c->dNbr, c->dSlot, c->dHaloPtr,
                                                                c->dHalo, c->dHaloSlot, c->K, c->TE, c->nslot, tau, (double)c->eta, (double)c->mass,
                                                                c->dTab, skip);
    });
}

void launch_rhs(const festung_ctx *c, double *W1, double *W2, double *b, double tau, cudaStream_t st) {
    const int grid = elem_grid(c);
    const int grid_lift = (int)std::max<int64_t>(
        1, std::min<int64_t>((c->nLift + LIFT_WARPS - 1) / LIFT_WARPS, (int64_t)c->num_sms * 16));
    c->launches += c->nLift > 0 ? 3 : 2;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        k_dirichlet_lift<double, N, R2, R1><<<grid, 256, 0, st>>>(W1, W2, c->dB, c->dNbr, c->K, c->dTab, c->dCD,
                                                                  c->dPerm);
        // every triangle without the lift's terms, then those terms on the triangles it reaches
        k_apply<double, N, R2, R1, MODE_RHS><<<grid, 256, 0, st>>>(c->dC, W1, W2, c->dD, b, c->dB, c->dNbr, c->K,
                                                                   tau, c->eta, c->mass, c->dTab, c->dF, c->dCD, c->dGN,
                                                                   c->dPerm, nullptr);
        if (c->nLift > 0)
            k_rhs_lift<N, R2, R1><<<grid_lift, 32 * LIFT_WARPS, 0, st>>>(W1, W2, c->dD, b, c->dB, c->dNbr, c->K, tau,
                                                                        c->eta, c->dTab, c->dCD, c->dPerm,
                                                                        c->dLiftList, c->nLift);
    });
}

void launch_flux(const festung_ctx *c, const double *x, double *Z1, double *Z2, cudaStream_t st) {
    const int grid = elem_grid(c);
    c->launches += 1;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        k_flux<double, N, R2, R1><<<grid, 256, 0, st>>>(x, Z1, Z2, c->dB, c->dNbr, c->K, c->dTab, nullptr);
    });
}

void launch_lift(const festung_ctx *c, double *W1, double *W2, cudaStream_t st) {
    const int grid = elem_grid(c);
    c->launches += 1;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        k_dirichlet_lift<double, N, R2, R1><<<grid, 256, 0, st>>>(W1, W2, c->dB, c->dNbr, c->K, c->dTab, c->dCD,
                                                                  c->dPerm);
    });
}

template <>
void launch_apply_twopass<double>(const festung_ctx *c, const double *x, double *y, double *Z1, double *Z2, double tau,
                                  const int *skip, cudaStream_t st) {
    const int grid = elem_grid(c);
    c->launches += 2;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        k_flux<double, N, R2, R1><<<grid, 256, 0, st>>>(x, Z1, Z2, c->dB, c->dNbr, c->K, c->dTab, skip);
        k_apply<double, N, R2, R1, MODE_APPLY><<<grid, 256, 0, st>>>(x, Z1, Z2, c->dD, y, c->dB, c->dNbr, c->K, tau,
                                                                  (double)c->eta, (double)c->mass, c->dTab, nullptr, nullptr, nullptr,
                                                                  nullptr, skip);
    });
}

cudaError_t upload_tables_f64(const festung_ctx *c) { return upload_ctab<double>(c); }

}  // namespace festung
