// Double-float arithmetic: a value is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2 (about one ulp for a product, see operator*), about 48 significant
// bits from FP32 instructions.
//
// The error-free transformations are the classical ones: the sum of two floats and
// its exact rounding error (Knuth's two-sum, 6 operations; Dekker's fast two-sum, 3,
// when |a| >= |b|) and the product with its exact error from one fused multiply-add.
// Sums and products of double-floats follow Dekker (1971): combine the high parts
// exactly, add the low-order terms, renormalise (sums; a product is renormalised by the
// sum it feeds).  Each result carries an absolute
// error of a few units of 2^-48 times the magnitudes of the operands, which is the
// bound a residual b - S x needs (errors relative to |S| |x|, not to |S x|).
//
// Every operation goes through the __fadd_rn / __fmul_rn / __fmaf_rn intrinsics so the
// compiler cannot contract or reassociate the sequences.
#pragma once

#include <cuda_runtime.h>

namespace festung {

struct alignas(8) dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dfloat(int v) : hi((float)v), lo(0.0f) {}
    __host__ __device__ explicit dfloat(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dfloat(s, e);
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    const dfloat s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

// The product is left unnormalised: p + e is the value the renormalisation (an exact
// transformation) would give, with |e| at most about one ulp of p instead of half of one.
// Every sum renormalises (operator+), and a product of such a pair drops only the term
// a.lo b.lo either way, so results keep about 47 bits at three fewer instructions per
// multiply-add.
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the product of the high parts
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return dfloat(p, e);
}

// Division only where the kernels divide once per triangle: through FP64.
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) { return dfloat((double)a / (double)b); }

// Accumulation (acc += term): the high parts summed with their exact error, the low parts
// added, and no renormalisation: the pair still holds the sum, its low part growing by
// about an ulp of the terms per step, which the next operator+ or the conversion to FP64
// absorbs.  Errors stay a few units of 2^-48 of the terms' magnitudes (the bound the
// residual needs), at 8 instructions instead of 11.
__device__ __forceinline__ dfloat &operator+=(dfloat &a, dfloat b) {
    const dfloat s = df_two_sum(a.hi, b.hi);
    a.hi = s.hi;
    a.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return a;
}
__device__ __forceinline__ dfloat &operator-=(dfloat &a, dfloat b) { return a += -b; }
__device__ __forceinline__ dfloat &operator*=(dfloat &a, dfloat b) { return a = a * b; }

}  // namespace festung
