// Double-float (FP32 pair) arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2
// after normalisation.  Error-free transformations after Knuth (TwoSum) and the
// FMA-based exact product; the explicit round-to-nearest intrinsics keep the
// compiler from contracting a product and a sum into one FMA, which would
// break the exactness of the transformations.
#pragma once
#include <cuda_runtime.h>

namespace lpk {

// s + e = a + b exactly, s = fl(a + b)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (sh, sl) += a * (xh + xl), with a * xh formed exactly (p + e1)
__device__ __forceinline__ void df_fma(float a, float xh, float xl, float& sh, float& sl) {
  const float p = __fmul_rn(a, xh);
  const float e1 = fmaf(a, xh, -p);
  float s, t;
  two_sum(sh, p, s, t);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, fmaf(a, xl, e1)));
}

// renormalise so that |sl| <= ulp(sh)/2 (requires |sl| <= |sh| or sh == 0)
__device__ __forceinline__ void df_renorm(float& sh, float& sl) {
  const float s = __fadd_rn(sh, sl);
  sl = __fsub_rn(sl, __fsub_rn(s, sh));
  sh = s;
}

// (sh, sl) += (oh, ol)
__device__ __forceinline__ void df_add(float& sh, float& sl, float oh, float ol) {
  float s, t;
  two_sum(sh, oh, s, t);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, ol));
}

}  // namespace lpk

namespace lpk {

// ---- double-float values for scalar formulas (normalised results) ----
struct dfl {
  float h, l;
};

__device__ __forceinline__ dfl dfl_make(float h, float l) {
  const float s = __fadd_rn(h, l);
  return {s, __fsub_rn(l, __fsub_rn(s, h))};
}

__device__ __forceinline__ dfl dfl_neg(dfl a) { return {-a.h, -a.l}; }

__device__ __forceinline__ dfl dfl_add(dfl a, dfl b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return dfl_make(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ dfl dfl_sub(dfl a, dfl b) { return dfl_add(a, dfl_neg(b)); }

__device__ __forceinline__ dfl dfl_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return dfl_make(p, e);
}

// a / b: FP32 quotient, then one correction from the exact remainder
__device__ __forceinline__ dfl dfl_div(dfl a, dfl b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  const float p = __fmul_rn(q1, b.h);
  const float pe = fmaf(q1, b.h, -p);
  // r = a - q1 b, its leading part a.h - p is exact (Sterbenz)
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.h, p), pe), __fsub_rn(a.l, __fmul_rn(q1, b.l)));
  return dfl_make(q1, __fdiv_rn(r, b.h));
}

}  // namespace lpk
