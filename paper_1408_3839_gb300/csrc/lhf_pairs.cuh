// lhf_pairs.cuh -- error-free transforms on pairs of FP32 words (a value h + l with
// |l| <= ulp(h) / 2, 48 significant bits), shared by the mixed route's kernels.  Sums of products
// are compensated dot products (Ogita, Rump and Oishi 2005): each product's rounding error comes
// from an FMA, each sum's from Knuth's TwoSum, both gathered in a second FP32 word.  __fadd_rn and
// __fmul_rn keep the compiler from contracting the transforms into FMAs.
#pragma once

#include <cuda_runtime.h>

namespace lhf {

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float v = __fadd_rn(s, -a);
  e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -v)), __fadd_rn(b, -v));
}
// s + c += (xh + xl)(yh + yl)
__device__ __forceinline__ void acc_prod(float &s, float &c, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  float q = fmaf(xh, yh, -p);
  q = fmaf(xh, yl, q);
  q = fmaf(xl, yh, q);
  float t, e;
  two_sum(s, p, t, e);
  s = t;
  c = __fadd_rn(c, __fadd_rn(e, q));
}
// s + c += xh + xl
__device__ __forceinline__ void acc_add(float &s, float &c, float xh, float xl) {
  float t, e;
  two_sum(s, xh, t, e);
  s = t;
  c = __fadd_rn(c, __fadd_rn(e, xl));
}
__device__ __forceinline__ float2 df_norm(float s, float c) {
  const float h = __fadd_rn(s, c);
  return make_float2(h, __fadd_rn(c, -__fadd_rn(h, -s)));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  return df_norm(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float q = fmaf(a.x, b.x, -p);
  q = fmaf(a.x, b.y, q);
  q = fmaf(a.y, b.x, q);
  return df_norm(p, q);
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
// x as a pair of FP32 words h + l (h the rounded value, l the rounded remainder).
__device__ __forceinline__ float2 fp32_pair(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

}  // namespace lhf
