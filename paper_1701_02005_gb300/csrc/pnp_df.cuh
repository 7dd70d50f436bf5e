// Double-float ("df") arithmetic on the FP32 pipe.
//
// A df value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// i.e. a 48-bit significand.  On this GPU the FP64 pipe issues about 1/64 of the
// FP32 rate, so the recurrences of the mixed path that need more than FP32
// (the ion state update and the spectral y-eliminations of the ill-conditioned
// low wavenumbers) run in df instead of FP64.  Building blocks: Knuth's
// error-free TwoSum, Dekker's FastTwoSum and the FMA form of Dekker's TwoProduct
// (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2).  Every operation uses the
// explicitly rounded intrinsics so that the compiler cannot contract a
// product and a sum into an FMA, which would break the error-free transforms.
#pragma once

#include <cuda_runtime.h>

namespace pnp {

struct dfl {
  float h, l;
};

// s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// Same, valid when |a| >= |b| (or a == 0).
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a * b for df operands; the lo * lo term is below the df resolution.
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return df_fast_two_sum(p, e);
}

// r - a * b with r a float and a, b df.
__device__ __forceinline__ dfl df_sub_mul(float r, dfl a, dfl b) {
  const dfl p = df_mul(a, b);
  const dfl s = df_two_sum(r, -p.h);
  return df_two_sum(s.h, __fsub_rn(s.l, p.l));   // s.h may have cancelled: full TwoSum
}

// x - a * b with x, a, b df.
__device__ __forceinline__ dfl df_sub_mul(dfl x, dfl a, dfl b) {
  const dfl p = df_mul(a, b);
  const dfl s = df_two_sum(x.h, -p.h);
  return df_two_sum(s.h, __fadd_rn(s.l, __fsub_rn(x.l, p.l)));
}

// x + d + f with x, d df and f a float; renormalised with TwoSum because the
// leading sum may cancel.
__device__ __forceinline__ dfl df_add2(dfl x, dfl d, float f) {
  const dfl s1 = df_two_sum(x.h, d.h);
  const dfl s2 = df_two_sum(s1.h, f);
  const float t = __fadd_rn(__fadd_rn(x.l, d.l), __fadd_rn(s1.l, s2.l));
  return df_two_sum(s2.h, t);
}

// x + y for df operands, with both the leading and the trailing parts summed
// by TwoSum (the accurate df sum: valid when x and y have opposite signs and
// cancel).
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  dfl s = df_two_sum(x.h, y.h);
  const dfl t = df_two_sum(x.l, y.l);
  s = df_fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return df_fast_two_sum(s.h, __fadd_rn(s.l, t.l));
}

// x + y for df operands with the trailing parts added in FP32 (Dekker's
// sum): error about 2^-47 (|x| + |y|), enough for running sums whose terms do
// not cancel to far below their own size.
__device__ __forceinline__ dfl df_add_fast(dfl x, dfl y) {
  const dfl s = df_two_sum(x.h, y.h);
  return df_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}

// a * b exactly, for float operands (TwoProduct).
__device__ __forceinline__ dfl df_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// Host-side split of a double into a df pair (hi = nearest float).
inline dfl df_split_host(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

}  // namespace pnp
