// Double-float ("float-float") arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers, |lo| <= ulp(hi)/2
// after normalization, which carries ~48 significant bits (relative rounding ~2^-48 = 3.6e-15) while every
// operation runs on the FP32 pipe.  On GB300 the FP32 pipe issues 64x as many FMAs per clock as the FP64 pipe, so an
// FP64-accurate operator evaluated this way is not bound by the FP64 rate.  The building blocks are the classical
// error-free transformations:
//   two_sum      Knuth's TwoSum (TAOCP Vol. 2, 4.2.2): s = fl(a + b) and the exact error e, a + b = s + e, 6 adds;
//   quick_sum    Dekker's Fast2Sum (1971): the same for |a| >= |b|, 3 adds;
//   two_prod     the FMA-based TwoProduct (Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26, 2005):
//                p = fl(a b), e = fma(a, b, -p), a b = p + e exactly.
// The double-float operations built from them follow Dekker's add2 / mul2 and the accumulating dot product of the
// same paper (Dot2: products by TwoProduct, partial sums by TwoSum, the errors summed separately).  Intrinsics with
// explicit rounding (__fadd_rn, __fmul_rn, __fmaf_rn) keep the compiler from contracting or reassociating them.
#pragma once

#include <cuda_runtime.h>

#include "evap_internal.cuh"

namespace evap {

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dfl quick_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// normalize an accumulator whose lo part has grown (|lo| may exceed ulp(hi))
__device__ __forceinline__ dfl df_norm(dfl a) { return quick_sum(a.hi, a.lo); }

// a + b (Dekker's add2): absolute error ~2^-48 (|a| + |b|)
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    dfl s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return quick_sum(s.hi, s.lo);
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

// a * b (Dekker's mul2 with an FMA): relative error ~2^-47
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    dfl p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return quick_sum(p.hi, p.lo);
}

// exact scaling by a power of two
__device__ __forceinline__ dfl df_scale2(dfl a, float pow2) { return {a.hi * pow2, a.lo * pow2}; }

// Dot2-style accumulation, acc += a b, without normalizing: the product by TwoProduct (its cross terms folded into
// the error), the partial sum of the high parts by TwoSum, all errors summed into acc.lo.  Normalize (df_norm) once
// the sum is complete.  Error of a completed dot product: ~2^-48 sum |a_k b_k| (plus the FP32 rounding of the lo sum,
// of the same order).
__device__ __forceinline__ void df_fma(dfl& acc, dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    const dfl s = two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}

// first term of an accumulation: acc = a b (no addition needed)
__device__ __forceinline__ dfl df_prod(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return {p, e};
}

// conversions (one FP64 add and three conversions: a few per nodal value, off the hot arithmetic)
__host__ __device__ __forceinline__ dfl df_from_double(double v) {
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}
__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

// Double-float copies of the 1D tables of the velocity element (built on the host from the FP64 basis).
struct DfBasis {
    dfl S[MAXQ][MAXQ];   // S[q][a] = l_a(t_q)
    dfl Dc[MAXQ][MAXQ];  // physical collocation derivative Dc[q][r] / h
    dfl N1[MAXQ][2];     // Q1 shape values at the Gauss points
    double t[MAXQ];      // the Gauss points on [0, 1] in FP64 (linear interpolation of nodal FP64 data)
};
DfBasis make_df_basis(const Basis<double>& b, double inv_h);

__device__ __forceinline__ dfl ld_df(const float2* p) {
    const float2 v = *p;
    return {v.x, v.y};
}

// dot product of Q double-float constants with Q values of a shared buffer (stride in dfl entries)
template <int Q>
__device__ __forceinline__ dfl df_dot(const dfl* c, const dfl* v, int stride) {
    dfl s = df_prod(c[0], v[0]);
#pragma unroll
    for (int k = 1; k < Q; ++k) df_fma(s, c[k], v[k * stride]);
    return df_norm(s);
}

}  // namespace evap
