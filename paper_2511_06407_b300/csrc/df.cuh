// Double-float ("f32x2") arithmetic: a value is an unevaluated pair hi + lo of FP32 numbers
// (about 48 significant bits). On B300 the FP32 pipe runs at 64x the FP64 rate, so a multiply-add
// built from error-free FP32 transformations is several times faster than a DFMA. A dot product
// accumulates the hi*hi products with Knuth's two-sum and the fma-based two-product and folds the
// cross terms and rounding errors into a compensation word (the Dot2 scheme of Ogita, Rump and
// Oishi 2005): 12 FP32 instructions per multiply-add, a result as accurate as if computed with a
// 48-bit significand. The intrinsics __fmul_rn / __fadd_rn / __fsub_rn keep the compiler from
// contracting the transformations into FMAs, which would break their exactness.
#pragma once
#include <cuda_runtime.h>

namespace rmhmc {

__device__ __forceinline__ float2 df_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df_join(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ void dot2_step(float& s, float& c, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float ep = fmaf(a.x, b.x, -p);
  const float t = __fadd_rn(s, p);
  const float bb = __fsub_rn(t, s);
  const float es = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  s = t;
  c = __fadd_rn(c, __fadd_rn(ep, es));
  c = fmaf(a.x, b.y, c);
  c = fmaf(a.y, b.x, c);
}
__device__ __forceinline__ float2 df_renorm(float s, float c) {
  const float h = __fadd_rn(s, c);
  return make_float2(h, __fsub_rn(c, __fsub_rn(h, s)));
}

}  // namespace rmhmc
