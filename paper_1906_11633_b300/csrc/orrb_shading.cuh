// orrb_shading.cuh -- device helpers shared by the forward shading and its adjoint.
#pragma once

namespace orrb {

__device__ __forceinline__ float exp2f_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ndh^alpha for ndh in [0, 1], alpha >= 1 (the Blinn-Phong lobe).
// Near 1, where the lobe is not negligible, d = 1 - ndh < 1/8 is exact (Sterbenz) and
// log2(1 - d) = -(d + d^2/2 + d^3/3 + ...) / ln 2 is summed to d^8/8 by Horner (the
// next term is below 1.2e-8 of the sum), so alpha*log2(ndh) = -t carries a relative
// error of ~1e-7 and ex2.approx adds 2^-22: the result's absolute error is at most
// ln2 * 1e-7 * t * 2^-t + 2.4e-7 * 2^-t < 3e-7.  Below ndh = 7/8, __powf's absolute
// error (lg2.approx: 2^-22.6 absolute near 1, 2^-22 relative elsewhere) stays under
// 6.4e-7 because alpha * 0.875^alpha <= 2.8.
__device__ __forceinline__ float lobe_pow(float ndh, float alpha) {
  const float d = 1.0f - ndh;
  if (d < 0.125f) {
    float s = 0.125f;
    s = fmaf(s, d, 1.0f / 7.0f);
    s = fmaf(s, d, 1.0f / 6.0f);
    s = fmaf(s, d, 0.2f);
    s = fmaf(s, d, 0.25f);
    s = fmaf(s, d, 1.0f / 3.0f);
    s = fmaf(s, d, 0.5f);
    s = fmaf(s, d, 1.0f);
    const float log2x = -(d * s) * 1.4426950408889634f;  // log2(1 - d) = ln(1 - d) / ln 2
    return exp2f_approx(alpha * log2x);
  }
  return ndh > 0.0f ? __powf(ndh, alpha) : 0.0f;
}

}  // namespace orrb
