// FP32 instantiations of the operator kernels (inner iterations of the mixed solve).
#include <algorithm>

#include "dispatch.h"
#include "ldg_fused.cuh"
#include "ops.h"

namespace festung {

template <>
void launch_apply<float>(const festung_ctx *c, const float *x, float *y, float *Z1, float *Z2, float tau,
                          const int *skip, cudaStream_t st) {
    (void)Z1;
    (void)Z2;
    if (c->tab_bf16) {
        launch_apply_bf16tab(c, x, y, tau, skip, st);
        return;
    }
    const int tiles = (int)((c->K + c->TE - 1) / c->TE);
    c->launches += 1;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        const size_t smem = fused_smem<float, N, R1>(c->nslot, c->TE);
        static const bool smem_ok = allow_max_smem(k_apply_fused<float, N, R2, R1>);
        (void)smem_ok;
        k_apply_fused<float, N, R2, R1><<<tiles, c->fthreads, smem, st>>>(x, y, c->fD, c->fB, c->dNbr, c->dSlot, c->dHaloPtr,
                                                                c->dHalo, c->dHaloSlot, c->K, c->TE, c->nslot, tau, (float)c->eta, (float)c->mass,
                                                                c->fTab, skip);
    });
}

int fused_resident_blocks(const festung_ctx *c, int nslot) {
    int nb = 0;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        static const bool smem_ok = allow_max_smem(k_apply_fused<float, N, R2, R1>);
        (void)smem_ok;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_apply_fused<float, N, R2, R1>, c->fthreads,
                                                          fused_smem<float, N, R1>(nslot, c->TE)) != cudaSuccess)
            nb = 0;
    });
    return std::max(1, nb) * c->num_sms;
}

size_t fused_smem_bytes(const festung_ctx *c, int nslot, bool fp64) {
    size_t b = 0;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto, auto r1_) {
        constexpr int N = decltype(n_)::value, R1 = decltype(r1_)::value;
        b = fp64 ? fused_smem<double, N, R1>(nslot, c->TE) : fused_smem<float, N, R1>(nslot, c->TE);
    });
    return b;
}

void launch_blockjacobi(const festung_ctx *c, float *P, __nv_bfloat16 *Pinv, double tau, int *flags,
                        cudaStream_t st) {
    const int64_t need = (c->K + 127) / 128;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)c->num_sms * 8));
    c->launches += 2;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        k_blockdiag<float, N, R2, R1><<<grid, 128, 0, st>>>(P, c->fB, c->dNbr, c->fD, c->K, (float)tau,
                                                            (float)c->eta, (float)c->mass, c->fTab);
        k_blockinv<N><<<grid, 128, 0, st>>>(P, Pinv, c->K, flags);
    });
}

template <>
void launch_apply_twopass<float>(const festung_ctx *c, const float *x, float *y, float *Z1, float *Z2, float tau,
                                 const int *skip, cudaStream_t st) {
    const int grid = elem_grid(c);
    c->launches += 2;
    dispatch(c->N, c->R2, c->R1, [&](auto n_, auto r2_, auto r1_) {
        constexpr int N = decltype(n_)::value, R2 = decltype(r2_)::value, R1 = decltype(r1_)::value;
        k_flux<float, N, R2, R1><<<grid, 256, 0, st>>>(x, Z1, Z2, c->fB, c->dNbr, c->K, c->fTab, skip);
        k_apply<float, N, R2, R1, MODE_APPLY><<<grid, 256, 0, st>>>(x, Z1, Z2, c->fD, y, c->fB, c->dNbr, c->K, tau,
                                                                  (float)c->eta, (float)c->mass, c->fTab, nullptr, nullptr, nullptr,
                                                                  nullptr, skip);
    });
}


}  // namespace festung
