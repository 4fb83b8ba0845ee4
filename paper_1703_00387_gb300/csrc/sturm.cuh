// Sturm counts of a symmetric tridiagonal matrix T (diagonal d, squared
// off-diagonal e2): the number of eigenvalues of T below x is the number of
// sign changes along the leading principal minors p_i = det(T_i - x I), with
// p_i = (d_i - x) p_(i-1) - e2_(i-1) p_(i-2) (Sturm sequence).
//
// Division-free: a zero minor is replaced by a tiny value of the sign opposite
// to its predecessor (the ratio form's negative tiny pivot), and every 8 rows
// both carried minors are scaled by a power of two read from their exponent
// bits (exact), which keeps them in range while ||T||^8 stays far below
// 2^800. NP points per thread run as independent chains that share the loads
// of d and e2; d and e2 may be in global or shared memory.
#pragma once
#include <cfloat>

namespace osmps {

template <int NP>
__device__ __forceinline__ void sturm_counts(const double* __restrict__ d,
                                             const double* __restrict__ e2, int n,
                                             const double (&x)[NP], int (&c)[NP]) {
  double pm[NP], p[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    pm[k] = 0.0;
    p[k] = 1.0;
    c[k] = 0;
  }
  for (int i = 0; i < n; ++i) {
    const double di = d[i];
    const double ei = i > 0 ? e2[i - 1] : 0.0;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      double pn = fma(di - x[k], p[k], -ei * pm[k]);
      const bool prev_neg = __double_as_longlong(p[k]) < 0;
      if ((__double_as_longlong(pn) << 1) == 0)  // zero minor: tiny, opposite sign
        pn = prev_neg ? DBL_MIN : -DBL_MIN;
      c[k] += (__double_as_longlong(pn) < 0) != prev_neg;
      pm[k] = p[k];
      p[k] = pn;
    }
    if ((i & 7) == 7) {  // keep |p|, |pm| near 1
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const long long bp = __double_as_longlong(p[k]) & 0x7FF0000000000000ll;
        const long long bq = __double_as_longlong(pm[k]) & 0x7FF0000000000000ll;
        const long long e = (bp > bq ? bp : bq) >> 52;  // biased exponent of the larger
        if (e < 1023 - 200 || e > 1023 + 200) {
          const double f = __longlong_as_double((long long)(2046 - e) << 52);  // 2^(1023 - e)
          p[k] *= f;
          pm[k] *= f;
        }
      }
    }
  }
}

// The same count in float32 (d, e2, x as floats), for narrowing a bracket
// before the float64 count resolves it: the count is exact for a tridiagonal
// within a few float32 ulps of T (entrywise), so it can misplace an
// eigenvalue by a few ulps of ||T||, no more. float32 has an 8-bit exponent:
// the minors are rescaled every 4 rows, and out of range at 2^+-60.
__device__ __forceinline__ int sturm_count_f32(const float* __restrict__ d,
                                               const float* __restrict__ e2, int n, float x) {
  float pm = 0.0f, p = 1.0f;
  int c = 0;
  for (int i = 0; i < n; ++i) {
    const float ei = i > 0 ? e2[i - 1] : 0.0f;
    float pn = fmaf(d[i] - x, p, -ei * pm);
    const bool prev_neg = __float_as_int(p) < 0;
    if ((__float_as_int(pn) << 1) == 0) pn = prev_neg ? FLT_MIN : -FLT_MIN;
    c += (__float_as_int(pn) < 0) != prev_neg;
    pm = p;
    p = pn;
    if ((i & 3) == 3) {
      const int bp = (__float_as_int(p) >> 23) & 0xFF, bq = (__float_as_int(pm) >> 23) & 0xFF;
      const int e = bp > bq ? bp : bq;  // biased exponent of the larger
      if (e < 127 - 60 || e > 127 + 60) {
        const float f = __int_as_float((254 - e) << 23);  // 2^(127 - e)
        p *= f;
        pm *= f;
      }
    }
  }
  return c;
}

}  // namespace osmps
