// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  Built on
// the error-free transformations of Knuth (TwoSum), Dekker (Fast2Sum) and
// the FMA form of TwoProduct.  GB300 issues FP32 FMAs at 64x its FP64 rate,
// so the small dense solves of the inversion run faster in pairs of FP32
// numbers than in FP64 while keeping a precision close to it.
#pragma once

namespace vfisv {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_from(float a) { return dfl{a, 0.0f}; }

__device__ __forceinline__ dfl df_from_double(double a) {
  const float h = (float)a;
  return dfl{h, (float)(a - (double)h)};
}

__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly, no precondition.
__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = a + b;
  const float v = s - a;
  return dfl{s, (a - (s - v)) + (b - v)};
}

// s + e = a + b exactly when |a| >= |b| (or a == 0).
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = a + b;
  return dfl{s, b - (s - a)};
}

// p + e = a * b exactly (FMA).
__device__ __forceinline__ dfl two_prod(float a, float b) {
  const float p = a * b;
  return dfl{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  dfl s = two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dfl df_neg(dfl x) { return dfl{-x.hi, -x.lo}; }

__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  dfl p = two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}

// x * y + z
__device__ __forceinline__ dfl df_fma(dfl x, dfl y, dfl z) { return df_add(df_mul(x, y), z); }

// 1/sqrt(x) for x > 0: the FP32 estimate refined by one Newton step,
// r = r0 + r0 (1 - x r0^2) / 2, with the residual formed in double-float.
// Inputs below 2^-100 (subnormal ones included: the hardware estimate
// flushes those to zero) are scaled by 2^100 first and the result by 2^50,
// both exact.
__device__ __forceinline__ dfl df_rsqrt(dfl x) {
  float post = 1.0f;
  if (x.hi < 0x1p-100f) {
    x.hi *= 0x1p100f;
    x.lo *= 0x1p100f;
    post = 0x1p50f;
  }
  const float r0 = rsqrtf(x.hi);
  const dfl h = df_add(df_from(1.0f), df_neg(df_mul(x, two_prod(r0, r0))));
  const dfl r = fast_two_sum(r0, 0.5f * r0 * h.hi);
  return dfl{r.hi * post, r.lo * post};
}

}  // namespace vfisv
