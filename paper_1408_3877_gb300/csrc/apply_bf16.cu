// FP32 fused applies whose reference tables (basis values, weighted gradients, H^,
// edge traces) are rounded to BF16: the operator of the BF16-table arm of the precision
// sweep (FESTUNG_BF16TAB): the kernels of table kind 1, whose compile-time tables hold
// BF16 values (8-bit significand) widened exactly to FP32 operands; x, D, the geometry
// and every sum stay FP32.  At p >= 3 their volume term runs on the tensor cores
// (ldg_tc.cuh: BF16-valued tables times TF32-split operands, FP32 accumulation).
#include "dispatch.h"
#include "ldg_fused.cuh"
#include "ops.h"

namespace festung {

void launch_apply_bf16tab(const festung_ctx *c, const float *x, float *y, float tau, const int *skip,
                          cudaStream_t st) {
    const int tiles = (int)((c->K + c->TE - 1) / c->TE);
    c->launches += 1;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        const size_t smem = fused_smem<float, N, R1, 1>(c->nslot, c->TE);
        static const bool smem_ok = allow_max_smem(k_apply_fused<float, N, R2, R1, FUSED_EPI_NONE, 1>);
        (void)smem_ok;
        k_apply_fused<float, N, R2, R1, FUSED_EPI_NONE, 1><<<tiles, c->fthreads, smem, st>>>(
            x, y, c->fD, c->fB, c->dNbr, c->dSlot, c->dHaloPtr, c->dHalo, c->dHaloSlot, c->K, c->TE, c->nslot, tau,
            (float)c->eta, (float)c->mass, c->bTab, skip);
    });
}

void launch_apply_bicg_bf16tab(const festung_ctx *c, const float *x, float *y, float tau, int epi, const float *e1,
                               const float *e2, double *part, KScal *sc, unsigned int *counter, const int *skip,
                               cudaStream_t st, const BatchView &bv) {
    const int tiles = (int)((c->K + c->TE - 1) / c->TE);
    c->launches += 1;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        const size_t smem = fused_smem<float, N, R1, 1>(c->nslot, c->TE);
        static const bool smem_a = allow_max_smem(k_apply_fused<float, N, R2, R1, FUSED_EPI_ALPHA, 1>);
        static const bool smem_o = allow_max_smem(k_apply_fused<float, N, R2, R1, FUSED_EPI_OMEGA, 1>);
        (void)smem_a;
        (void)smem_o;
        auto kern = epi == FUSED_EPI_ALPHA ? k_apply_fused<float, N, R2, R1, FUSED_EPI_ALPHA, 1>
                                           : k_apply_fused<float, N, R2, R1, FUSED_EPI_OMEGA, 1>;
        kern<<<tiles, c->fthreads, smem, st>>>(x, y, c->fD, c->fB, c->dNbr, c->dSlot, c->dHaloPtr, c->dHalo,
                                                 c->dHaloSlot, c->K, c->TE, c->nslot, tau, (float)c->eta,
                                                 (float)c->mass, c->bTab, skip, e1, e2, part, sc, counter, bv);
    });
}

}  // namespace festung
