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

}  // namespace osmps
