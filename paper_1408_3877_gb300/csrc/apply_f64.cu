// FP64 instantiations of the operator kernels and the right-hand side.
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
        const size_t smem = fused_smem<double, R1>(c->nslot);
        static const bool smem_ok = allow_max_smem(k_apply_fused<double, N, R2, R1>);
        (void)smem_ok;
        k_apply_fused<double, N, R2, R1><<<tiles, FUSED_THREADS, smem, st>>>(x, y, c->dD, c->dB, c->dNbr, c->dSlot, c->dHaloPtr,
                                                                c->dHalo, c->dHaloSlot, c->K, c->TE, c->nslot, tau, (double)c->eta, (double)c->mass,
                                                                c->dTab, skip);
    });
}

void launch_rhs(const festung_ctx *c, double *W1, double *W2, double *b, double tau, cudaStream_t st) {
    const int grid = elem_grid(c);
    c->launches += 2;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        k_dirichlet_lift<double, N, R2, R1><<<grid, 256, 0, st>>>(W1, W2, c->dB, c->dNbr, c->K, c->dTab, c->dCD,
                                                                  c->dPerm);
        k_apply<double, N, R2, R1, MODE_RHS><<<grid, 256, 0, st>>>(c->dC, W1, W2, c->dD, b, c->dB, c->dNbr, c->K,
                                                                   tau, c->eta, c->mass, c->dTab, c->dF, c->dCD, c->dGN,
                                                                   c->dPerm, c->dLift, nullptr);
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
                                                                  nullptr, nullptr, skip);
    });
}

// Copy the reference tables of the context's (N, R2, R1) into the constant bank.  The
// tables depend only on p and the quadrature, so every context of the same shape
// writes identical values; the copy is done once per process and shape.
cudaError_t upload_tables_f64(const festung_ctx *c) {
    cudaError_t err = cudaSuccess;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        static bool done = false;
        if (done) return;
        CTab<double, N, R2, R1> h;
        const HostTables &t = c->tab;
        for (int i = 0; i < R2 * N; ++i) {
            h.phiQ[i] = (double)t.phiQ[i];
            h.gw1[i] = (double)t.gw1[i];
            h.gw2[i] = (double)t.gw2[i];
        }
        for (int i = 0; i < N * N; ++i) {
            h.H1[i] = (double)t.H1[i];
            h.H2[i] = (double)t.H2[i];
        }
        for (int i = 0; i < 3 * R1 * N; ++i) {
            h.phiE[i] = (double)t.phiE[i];
            h.wphiE[i] = (double)t.wphiE[i];
        }
        err = cudaMemcpyToSymbol(c_tab<double, N, R2, R1>, &h, sizeof(h));
        if (err == cudaSuccess) done = true;
    });
    return err;
}

}  // namespace festung
