// FP32 fused applies with the BiCGStab reductions in their epilogue (a translation
// unit of their own, compiled in parallel with the plain applies).
#include "dispatch.h"
#include "ldg_fused.cuh"
#include "ops.h"

namespace festung {

template <>
void launch_apply_bicg<float>(const festung_ctx *c, const float *x, float *y, float tau, int epi, const float *e1,
                              const float *e2, double *part, KScal *sc, unsigned int *counter, const int *skip,
                              cudaStream_t st, const BatchView &bv) {
    if (c->tab_bf16) {
        launch_apply_bicg_bf16tab(c, x, y, tau, epi, e1, e2, part, sc, counter, skip, st, bv);
        return;
    }
    const int tiles = (int)((c->K + c->TE - 1) / c->TE);
    c->launches += 1;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        const size_t smem = fused_smem<float, N, R1>(c->nslot, c->TE);
        static const bool smem_a = allow_max_smem(k_apply_fused<float, N, R2, R1, FUSED_EPI_ALPHA>);
        static const bool smem_o = allow_max_smem(k_apply_fused<float, N, R2, R1, FUSED_EPI_OMEGA>);
        (void)smem_a;
        (void)smem_o;
        auto kern = epi == FUSED_EPI_ALPHA ? k_apply_fused<float, N, R2, R1, FUSED_EPI_ALPHA>
                                           : k_apply_fused<float, N, R2, R1, FUSED_EPI_OMEGA>;
        kern<<<tiles, c->fthreads, smem, st>>>(x, y, c->fD, c->fB, c->dNbr, c->dSlot, c->dHaloPtr, c->dHalo,
                                                 c->dHaloSlot, c->K, c->TE, c->nslot, tau, (float)c->eta,
                                                 (float)c->mass, c->fTab, skip, e1, e2, part, sc, counter, bv);
    });
}


}  // namespace festung
