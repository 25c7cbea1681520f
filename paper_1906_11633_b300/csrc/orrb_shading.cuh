// orrb_shading.cuh -- device helpers shared by the forward shading and its adjoint.
#pragma once

namespace orrb {

__device__ __forceinline__ float exp2f_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/sqrt(x) by the hardware approximation (PTX rsqrt.approx, relative error below 2^-22.9) with
// subnormal inputs flushed to zero.  The inputs here are squared lengths; only a vector shorter
// than about 1e-19 would read as zero.
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
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

// The PCG hash (Jarzynski and Olano, "Hash Functions for GPU Rendering", JCGT 2020): one LCG
// step, a random xorshift and a multiply.
__host__ __device__ inline unsigned pcg_hash(unsigned v) {
  const unsigned state = v * 747796405u + 2891336453u;
  const unsigned word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
  return (word >> 22u) ^ word;
}

// The grain key of an image: the hash of the sample's grain seed and the camera's index within
// its sample.  A pixel's grain value is the hash of (key ^ pixel index within the image) scaled
// to [0, 1), minus 1/2.
__device__ __forceinline__ unsigned grain_key(const float* g, unsigned cam_local) {
  return pcg_hash(unsigned(g[7]) + 0x9E3779B9u * (cam_local + 1u));
}
__device__ __forceinline__ float grain_centred(unsigned key, unsigned pixel) {
  return float(pcg_hash(key ^ pixel)) * 2.3283064365386963e-10f - 0.5f;  // 2^-32
}

// Colour grading of a sample (g = hue, saturation, contrast, brightness, temperature, tint, grain,
// seed): white balance, the rotation about the grey axis, saturation, contrast and brightness are
// each affine in the colour, so they compose into one map c -> A c + t (rows of gm = A | t).
__device__ __forceinline__ void grading_map(const float* g, float gm[3][4]) {
  float hs, hc;
  sincosf(g[0], &hs, &hc);
  const float k = 0.57735026918962576f;  // 1/sqrt(3): the grey axis (k, k, k)
  // rotation R = cos I + sin [axis]x + (1 - cos) axis axis^T
  const float a = hc + (1.0f - hc) / 3.0f, b = (1.0f - hc) / 3.0f - k * hs, c = (1.0f - hc) / 3.0f + k * hs;
  const float R[3][3] = {{a, b, c}, {c, a, b}, {b, c, a}};
  const float wb[3] = {1.0f + g[4], 1.0f + g[5], 1.0f - g[4]};
  const float Yw[3] = {0.2126f, 0.7152f, 0.0722f};
  const float sat = g[1], con = g[2];
  // S = sat I + (1 - sat) 1 Yw^T; then contrast con and the offsets 0.5 (1 - con) + brightness
  for (int i = 0; i < 3; i++) {
    for (int j = 0; j < 3; j++) {
      float rw = 0.0f;  // (S R)_ij
      for (int m = 0; m < 3; m++) rw += ((i == m ? sat : 0.0f) + (1.0f - sat) * Yw[m]) * R[m][j];
      gm[i][j] = con * rw * wb[j];
    }
    gm[i][3] = 0.5f * (1.0f - con) + g[3];
  }
}

}  // namespace orrb
