// Double-float instantiation of the fused apply (pairs of FP32 values, about 48
// significant bits): the residual b - S x of the mixed-precision refinement.  The FP32
// pipes of a GB300 SM issue 64 times as many operations as its FP64 pipe, so the
// 10-20 FP32 operations of a double-float multiply-add still cost less than one FP64
// multiply-add.
#include "dfloat.cuh"
#include "dispatch.h"
#include "ldg_fused.cuh"
#include "ops.h"

namespace festung {

void launch_apply_df(const festung_ctx *c, const dfloat *x, dfloat *y, double tau, cudaStream_t st) {
    const int tiles = (int)((c->K + c->TE - 1) / c->TE);
    c->launches += 1;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        const size_t smem = fused_smem<dfloat, N, R1>(c->nslot, c->TE);
        static const bool smem_ok = allow_max_smem(k_apply_fused<dfloat, N, R2, R1>);
        (void)smem_ok;
        k_apply_fused<dfloat, N, R2, R1><<<tiles, c->fthreads, smem, st>>>(
            x, y, c->xD, c->xB, c->dNbr, c->dSlot, c->dHaloPtr, c->dHalo, c->dHaloSlot, c->K, c->TE, c->nslot,
            dfloat(tau), dfloat(c->eta), dfloat(c->mass), c->xTab, nullptr);
    });
}

cudaError_t upload_tables_df(const festung_ctx *c) { return upload_ctab<dfloat>(c); }

}  // namespace festung
