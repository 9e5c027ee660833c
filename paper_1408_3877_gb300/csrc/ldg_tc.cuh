// Volume term of the fused apply on the tensor cores (FP32 kernels, p >= 3).
//
// For the 32 triangles of a warp the volume term -sum_m G^m Z^m (Sec. 3.6.3, eq. hatG) in
// the contravariant form of ldg_fused.cuh is two passes of small dense products with the
// reference tables:
//   1. evaluation  [d_h | zeta^1 | zeta^2] (32 x 16, basis) . Phi^T (16 x R2p, points):
//      d_h, zeta^1, zeta^2 at the triangle points;
//   2. test        [u | v] (32 x R2p) . [w d1 phi; w d2 phi] (R2p x 16, basis) with
//      u = d_h zeta^1, v = d_h zeta^2 at every point,
// issued as mma.sync m16n8k8 TF32 products with FP32 accumulation.  FP32 accuracy comes
// from the three-term split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi of each operand into
// a TF32 value and a TF32 remainder (Henry, Tang and Heinecke 2019; Ootomo and Yokota
// 2022): the dropped a_lo b_lo and the truncation of the remainders are about 2^-20 of
// |a b|.  With tables held as BF16 values (FESTUNG_BF16TAB) b_lo is zero and two products
// suffice.
//
// Fragment layouts of mma.m16n8k8 with .tf32 (PTX ISA), g = lane / 4, t = lane % 4:
//   A (16 x 8):  a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4);
//   B (8 x 8):   b0 (t, g), b1 (t + 4, g);
//   C (16 x 8):  c0 (g, 2t), c1 (g, 2t + 1), c2 (g + 8, 2t), c3 (g + 8, 2t + 1).
// The products u, v of the first pass sit in C layout; the second pass uses them as A
// fragments directly by ordering its reduction index so that A column t is point 2t and
// column t + 4 is point 2t + 1 of each group of 8 points (the B rows follow the same
// order), with no data exchange between lanes.
#pragma once

#include <cstdint>

namespace festung {

constexpr int TC_SR = 20;  // row stride (floats) of the staged operands and of Phi: 16 + 4, no bank conflicts
constexpr int TC_GR = 40;  // row stride of the transposed test tables: 32 points + 8
// shared-memory tables: Phi_hi, Phi_lo [32 points][TC_SR]; G1_hi, G1_lo, G2_hi, G2_lo [16 basis][TC_GR]
constexpr int TC_TAB_FLOATS = 2 * 32 * TC_SR + 4 * 16 * TC_GR;
// staged operands of one warp: the A fragments of its 32 triangles (3 operands x 2 row blocks
// x 2 basis groups x 32 lanes x 4 registers); the result block [32][TC_SR] reuses them
constexpr int TC_STAGE_FLOATS = 3 * 2 * 2 * 32 * 4;
static_assert(32 * TC_SR <= TC_STAGE_FLOATS, "result block fits the staged operands");

__device__ __forceinline__ uint32_t tf32_of(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

// v = hi + lo with hi, lo TF32 values (lo the TF32 rounding of the exact remainder)
__device__ __forceinline__ void tf32_split(float v, uint32_t &hi, uint32_t &lo) {
    hi = tf32_of(v);
    lo = tf32_of(v - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Fill the shared-memory tables from the reference tables (phiQ, gw1, gw2 as [R2][N]):
// TF32 high parts and remainders, zero outside the R2 x N block.  All threads of the block.
template <int N, int R2>
__device__ __forceinline__ void tc_fill_tables(float *s, const float *phiQ, const float *gw1, const float *gw2) {
    float *phi_hi = s, *phi_lo = s + 32 * TC_SR;
    float *g = s + 2 * 32 * TC_SR;
    for (int q = threadIdx.x; q < 32 * TC_SR; q += blockDim.x) {
        const int r = q / TC_SR, j = q - r * TC_SR;
        const float v = (r < R2 && j < N) ? phiQ[r * N + j] : 0.0f;
        uint32_t hi, lo;
        tf32_split(v, hi, lo);
        phi_hi[q] = __uint_as_float(hi);
        phi_lo[q] = __uint_as_float(lo);
    }
    for (int q = threadIdx.x; q < 16 * TC_GR; q += blockDim.x) {
        const int j = q / TC_GR, r = q - j * TC_GR;
        const bool in = r < R2 && j < N;
        uint32_t hi, lo;
        tf32_split(in ? gw1[r * N + j] : 0.0f, hi, lo);
        g[q] = __uint_as_float(hi);
        g[16 * TC_GR + q] = __uint_as_float(lo);
        tf32_split(in ? gw2[r * N + j] : 0.0f, hi, lo);
        g[2 * 16 * TC_GR + q] = __uint_as_float(hi);
        g[3 * 16 * TC_GR + q] = __uint_as_float(lo);
    }
}

// TF32 split by truncation: hi keeps the sign, exponent and top 10 mantissa bits of v, and
// lo = v - hi is exact; the tensor cores read lo's top bits only (a TF32 operand ignores the
// low 13 bits), so hi + lo carries about 21 bits of v.
__device__ __forceinline__ void tf32_trunc_split(float v, uint32_t &hi, uint32_t &lo) {
    hi = __float_as_uint(v) & 0xffffe000u;
    lo = __float_as_uint(v - __uint_as_float(hi));
}

// Stage the lane's d_h, zeta^1, zeta^2 (zero-padded to 16 basis functions; zeros for a lane
// without a triangle) into `stage` in A-fragment order:
//   stage[((f * 4 + mt * 2 + ks) * 32 + L) * 4 + q]
// (operand f, row block mt = lane / 16, basis group ks) holds row r = lane % 16, column
// c = j % 8 at lane L = 4 (r % 8) + c % 4, register q = r / 8 + 2 (c / 4).  After this the
// operands need no registers.
template <int N>
__device__ __forceinline__ void tc_stage(bool valid, const float (&d)[N], const float (&z1)[N], const float (&z2)[N],
                                         float *stage) {
    const int lane = threadIdx.x & 31, mt = lane >> 4, r = lane & 15;
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float v = (valid && j < N) ? (f == 0 ? d[j] : f == 1 ? z1[j] : z2[j]) : 0.0f;
            const int ks = j >> 3, c = j & 7;
            const int L = 4 * (r & 7) + (c & 3), q = (r >> 3) + 2 * (c >> 2);
            stage[((f * 4 + mt * 2 + ks) * 32 + L) * 4 + q] = v;
        }
}

// acc[j] -= sum_r (w_r d1 phi_j d_h zeta^1 + w_r d2 phi_j d_h zeta^2)(q_r) for the triangle
// of this lane, from the operands that tc_stage left in `stage` (this warp's
// TC_STAGE_FLOATS floats); every lane of the warp takes part.  tab: the tables of
// tc_fill_tables.  BF: the tables hold BF16 values (their remainders are zero).
template <int N, int R2, bool BF>
__device__ __forceinline__ void volume_tc(float (&acc)[N], float *stage, const float *tab) {
    static_assert(N <= 16 && R2 <= 32, "tensor-core volume: N <= 16, R2 <= 32");
    constexpr int NT = (R2 + 7) / 8;  // groups of 8 points
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float *phi_hi = tab, *phi_lo = tab + 32 * TC_SR;
    const float *g1_hi = tab + 2 * 32 * TC_SR, *g1_lo = g1_hi + 16 * TC_GR, *g2_hi = g1_lo + 16 * TC_GR,
                *g2_lo = g2_hi + 16 * TC_GR;
    float *res = stage;  // the result block [32][TC_SR] reuses the fragments of row block 0
    float out[2][2][4];
    __syncwarp();
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int nb = 0; nb < 2; ++nb)
#pragma unroll
            for (int q = 0; q < 4; ++q) out[mt][nb][q] = 0.0f;
#pragma unroll 1
        for (int nt = 0; nt < NT; ++nt) {
            // first pass: d_h, zeta^1, zeta^2 at points 8 nt .. 8 nt + 7
            float c[3][4];
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int q = 0; q < 4; ++q) c[f][q] = 0.0f;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const int o = (8 * nt + g) * TC_SR + 8 * ks + t;
                const uint32_t bh0 = __float_as_uint(phi_hi[o]), bh1 = __float_as_uint(phi_hi[o + 4]);
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    const float4 a4 = *reinterpret_cast<const float4 *>(stage + ((f * 4 + mt * 2 + ks) * 32 + lane) * 4);
                    uint32_t ah[4], al[4];
                    tf32_trunc_split(a4.x, ah[0], al[0]);
                    tf32_trunc_split(a4.y, ah[1], al[1]);
                    tf32_trunc_split(a4.z, ah[2], al[2]);
                    tf32_trunc_split(a4.w, ah[3], al[3]);
                    mma_tf32(c[f], ah, bh0, bh1);
                    mma_tf32(c[f], al, bh0, bh1);
                    if constexpr (!BF)
                        mma_tf32(c[f], ah, __float_as_uint(phi_lo[o]), __float_as_uint(phi_lo[o + 4]));
                }
            }
            // u = d_h zeta^1, v = d_h zeta^2 at the points of this group, as A fragments of
            // second pass (column t <-> point 2t, column t + 4 <-> point 2t + 1)
            uint32_t uh[4], ul[4], vh[4], vl[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int p = q == 1 ? 2 : q == 2 ? 1 : q;
                tf32_trunc_split(c[0][p] * c[1][p], uh[q], ul[q]);
                tf32_trunc_split(c[0][p] * c[2][p], vh[q], vl[q]);
            }
            // second pass: test against the weighted gradients, both groups of 8 basis functions
#pragma unroll
            for (int nb = 0; nb < 2; ++nb) {
                const int o = (8 * nb + g) * TC_GR + 8 * nt + 2 * t;
                const float2 b1h = *reinterpret_cast<const float2 *>(g1_hi + o);
                const float2 b2h = *reinterpret_cast<const float2 *>(g2_hi + o);
                mma_tf32(out[mt][nb], uh, __float_as_uint(b1h.x), __float_as_uint(b1h.y));
                mma_tf32(out[mt][nb], ul, __float_as_uint(b1h.x), __float_as_uint(b1h.y));
                mma_tf32(out[mt][nb], vh, __float_as_uint(b2h.x), __float_as_uint(b2h.y));
                mma_tf32(out[mt][nb], vl, __float_as_uint(b2h.x), __float_as_uint(b2h.y));
                if constexpr (!BF) {
                    const float2 b1l = *reinterpret_cast<const float2 *>(g1_lo + o);
                    const float2 b2l = *reinterpret_cast<const float2 *>(g2_lo + o);
                    mma_tf32(out[mt][nb], uh, __float_as_uint(b1l.x), __float_as_uint(b1l.y));
                    mma_tf32(out[mt][nb], vh, __float_as_uint(b2l.x), __float_as_uint(b2l.y));
                }
            }
        }
    }
    // C layout -> the rows of the result block, then the lane's own row
    __syncwarp();
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nb = 0; nb < 2; ++nb) {
            float *r0 = res + (16 * mt + g) * TC_SR + 8 * nb + 2 * t;
            *reinterpret_cast<float2 *>(r0) = make_float2(out[mt][nb][0], out[mt][nb][1]);
            *reinterpret_cast<float2 *>(r0 + 8 * TC_SR) = make_float2(out[mt][nb][2], out[mt][nb][3]);
        }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j] -= res[lane * TC_SR + j];
}

}  // namespace festung
