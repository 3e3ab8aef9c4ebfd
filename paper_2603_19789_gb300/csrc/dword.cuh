// dword.cuh -- double-word arithmetic on FP32 pairs, for the FP64-accurate storage
// SSLBM_FP64_DW: a value is hi + lo with two floats (about 48 significant bits), and every
// operation of the SSLBM update is carried out on such pairs with error-free transformations
// in FP32, the arithmetic GB300 has 64 times more of than FP64.
//
// The algorithms are the published double-word building blocks of M. Joldes, J.-M. Muller
// and V. Popescu, "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM Trans. Math. Softw. 44(2), 2017 (relative error bounds in units of
// u = 2^-24: addition 3u^2, multiplication 4u^2, division 15u^2), built on Knuth's TwoSum,
// Dekker's Fast2Sum and the FMA-based exact product.  Every operation works on two
// independent lanes at once (the two columns a thread updates), with the packed FP32
// instructions, each component rounded like its scalar operation.
#pragma once
#include "sslbm_internal.cuh"

namespace sslbm {
namespace dw {

// Two double-word numbers (one per lane component): value_k = h_k + l_k, |l_k| <= ulp(h_k)/2.
struct W {
  float2 h, l;
};

// a - b in one instruction: b * (-1) is exact, so the fused multiply-add rounds a - b once,
// like the subtraction (the same bits as adding -b).
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return fma2(b, splat2(-1.f), a); }

// Knuth's TwoSum: s + e = a + b exactly, s = fl(a + b); no condition on a, b.
__device__ __forceinline__ W two_sum(float2 a, float2 b) {
  const float2 s = add2(a, b);
  const float2 ap = sub(s, b);
  const float2 bp = sub(s, ap);
  return W{s, add2(sub(a, ap), sub(b, bp))};
}

// Dekker's Fast2Sum: s + e = a + b exactly when the exponent of a is at least that of b.
__device__ __forceinline__ W fast_two_sum(float2 a, float2 b) {
  const float2 s = add2(a, b);
  return W{s, sub(b, sub(s, a))};
}

// Exact product with the FMA: p + e = a b.
__device__ __forceinline__ W two_prod(float2 a, float2 b) {
  const float2 p = mul2(a, b);
  return W{p, fma2(a, b, neg2(p))};
}

// x + y, the accurate double-word sum (relative error <= 3u^2, cancellation included).
__device__ __forceinline__ W add(const W& x, const W& y) {
  const W s = two_sum(x.h, y.h);
  const W t = two_sum(x.l, y.l);
  const W v = fast_two_sum(s.h, add2(s.l, t.h));
  return fast_two_sum(v.h, add2(t.l, v.l));
}

__device__ __forceinline__ W neg(const W& x) { return W{neg2(x.h), neg2(x.l)}; }
__device__ __forceinline__ W sub(const W& x, const W& y) { return add(x, neg(y)); }

// x + y with the low parts added in one rounding (the 'sloppy' double-word sum, 11 flops):
// for operands of one sign its relative error is below 3u^2; under cancellation its error
// is still below about 2u^2 (|x| + |y|) in absolute terms, the bound an update of O(1)
// fields measured against their peak needs.
__device__ __forceinline__ W add_abs(const W& x, const W& y) {
  const W s = two_sum(x.h, y.h);
  return fast_two_sum(s.h, add2(s.l, add2(x.l, y.l)));
}
__device__ __forceinline__ W sub_abs(const W& x, const W& y) { return add_abs(x, neg(y)); }

// ((l - c) + (r - c)) + ((u - c) + (d - c)) of double words, with one normalisation: the high
// parts' differences and their sums are exact (TwoSum), and their errors and the low parts'
// differences are added in FP32 once, so the result's absolute error stays of order
// u^2 (|c| + the neighbours), like a chain of add_abs (59 flops against 77).
__device__ __forceinline__ W lap5_diff(const W& c, const W& l, const W& r, const W& up, const W& dn) {
  const W d1 = two_sum(l.h, neg2(c.h)), d2 = two_sum(r.h, neg2(c.h));
  const W d3 = two_sum(up.h, neg2(c.h)), d4 = two_sum(dn.h, neg2(c.h));
  const W a = two_sum(d1.h, d2.h), b = two_sum(d3.h, d4.h), e = two_sum(a.h, b.h);
  const float2 lows = add2(add2(sub(l.l, c.l), sub(r.l, c.l)), add2(sub(up.l, c.l), sub(dn.l, c.l)));
  const float2 errs = add2(add2(add2(d1.l, d2.l), add2(d3.l, d4.l)), add2(add2(a.l, b.l), e.l));
  return fast_two_sum(e.h, add2(lows, errs));
}

// x y (relative error <= 4u^2).
__device__ __forceinline__ W mul(const W& x, const W& y) {
  const W c = two_prod(x.h, y.h);
  const float2 t = fma2(x.h, y.l, mul2(x.l, y.l));
  return fast_two_sum(c.h, add2(c.l, fma2(x.l, y.h, t)));
}

// x t for a float pair t (the division's remainder step).
__device__ __forceinline__ W mul_fp(const W& x, float2 t) {
  const W c = two_prod(x.h, t);
  return fast_two_sum(c.h, fma2(x.l, t, c.l));
}

// x / y (relative error <= 15u^2 + 56u^3): a float quotient of the high parts, corrected by
// the double-word remainder x - y q divided by y's high part.
__device__ __forceinline__ W div(const W& x, const W& y) {
  const float2 q = make_float2(__fdiv_rn(x.h.x, y.h.x), __fdiv_rn(x.h.y, y.h.y));
  const W r = mul_fp(y, q);
  const float2 d = add2(sub(x.h, r.h), sub(x.l, r.l));
  const float2 ql = make_float2(__fdiv_rn(d.x, y.h.x), __fdiv_rn(d.y, y.h.y));
  return fast_two_sum(q, ql);
}

// A double-word constant (hi, lo) for both lanes.
__device__ __forceinline__ W splat(float2 c) { return W{splat2(c.x), splat2(c.y)}; }

}  // namespace dw

// The update's coefficients (those of Coeffs<double>) as double-word pairs (hi, lo).
struct DwCoeffs {
  float2 dl[4];
  float2 bdt, adt, gdt, rdt, ddt;
};

}  // namespace sslbm
