// orrb_shading.cuh -- device helpers shared by the forward shading and its adjoint.
#pragma once

namespace orrb {

__device__ __forceinline__ float exp2f_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float log2f_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ndh^alpha = 2^(alpha * log2 ndh) for ndh in [0, 1], alpha >= 1 (the Blinn-Phong lobe),
// without a branch (both logarithms are formed and one is selected).
// Near 1, where the lobe is not negligible, d = 1 - ndh < 1/32 is exact (Sterbenz) and
// log2(1 - d) = -(d + d^2/2 + d^3/3 + ...) / ln 2 is summed to d^5/5 by Horner (the next
// term is below 5e-9 of the sum), so alpha*log2(ndh) = -t carries a relative error of
// ~1e-7 and ex2.approx adds 2^-22: the result's absolute error is at most
// ln2 * 1e-7 * t * 2^-t + 2.4e-7 * 2^-t < 3e-7.  Below ndh = 31/32, lg2.approx (absolute
// error 2^-22.6 on [0.5, 2], relative 2^-22 elsewhere) keeps the absolute error under
// 1.4e-6 because alpha * (31/32)^alpha <= 11.6; ndh = 0 gives log2 = -inf and exactly 0.
__device__ __forceinline__ float lobe_pow(float ndh, float alpha) {
  const float d = 1.0f - ndh;
  float s = 0.2f;
  s = fmaf(s, d, 0.25f);
  s = fmaf(s, d, 1.0f / 3.0f);
  s = fmaf(s, d, 0.5f);
  s = fmaf(s, d, 1.0f);
  const float near1 = -(d * s) * 1.4426950408889634f;  // log2(1 - d) = ln(1 - d) / ln 2
  const float lg = d < 0.03125f ? near1 : log2f_approx(ndh);
  return exp2f_approx(alpha * lg);
}

}  // namespace orrb
