// ks_dfloat.cuh -- double-float numbers: a value held as an unevaluated sum of
// two FP32 numbers hi + lo (|lo| <= ulp(hi) / 2), about 44 significant bits,
// computed on the FP32 pipes.  The operations are the double-word algorithms
// built from error-free transformations: Knuth's TwoSum, Dekker's FastTwoSum
// and the FMA-based exact product (as analysed by Joldes, Muller and Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 2017: the accurate sum, and the product with an FMA).
// Relative error of a sum or product below about 2^-44; the compiler must not
// reassociate FP32 additions (no fast-math), which the build never enables.
#pragma once

namespace ks {

namespace dfx {

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly, given |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

}  // namespace dfx

struct dfloat {
    float hi, lo;
    __device__ __forceinline__ dfloat() : hi(0.f), lo(0.f) {}
    __device__ __forceinline__ dfloat(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ dfloat(int v) : hi((float)v), lo(0.f) {}
    __device__ __forceinline__ dfloat(float v) : hi(v), lo(0.f) {}
    // the double rounded to the nearest double-float (hi the nearest float)
    __device__ __forceinline__ dfloat(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __device__ __forceinline__ explicit operator float() const { return __fadd_rn(hi, lo); }
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dfloat operator-(dfloat a) { return {-a.hi, -a.lo}; }

// accurate double-word sum: two TwoSums, two renormalisations
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b)
{
    float sh, sl, th, tl;
    dfx::two_sum(a.hi, b.hi, sh, sl);
    dfx::two_sum(a.lo, b.lo, th, tl);
    sl = __fadd_rn(sl, th);
    dfx::fast_two_sum(sh, sl, sh, sl);
    sl = __fadd_rn(sl, tl);
    dfloat r;
    dfx::fast_two_sum(sh, sl, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

// double-word product with an FMA: the exact product of the high parts, the
// cross terms added to its error
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b)
{
    const float ch = __fmul_rn(a.hi, b.hi);
    const float cl1 = __fmaf_rn(a.hi, b.hi, -ch);
    const float tl = __fmul_rn(a.hi, b.lo);
    const float cl2 = __fmaf_rn(a.lo, b.hi, tl);
    const float cl3 = __fadd_rn(cl1, cl2);
    dfloat r;
    dfx::fast_two_sum(ch, cl3, r.hi, r.lo);
    return r;
}

// quotient by one correction step: q1 = a / b to FP32, then the remainder's
// quotient (used for the transforms' power-of-two scale factors)
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const dfloat r = a - b * dfloat(q1);
    const float q2 = __fdiv_rn(r.hi, b.hi);
    dfloat q;
    dfx::fast_two_sum(q1, q2, q.hi, q.lo);
    return q;
}

}  // namespace ks
