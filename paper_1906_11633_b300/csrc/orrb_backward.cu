// orrb_backward.cu -- adjoint of the shading at fixed visibility (sm_103a).
//
// Given the G-buffer a render wrote (view-space position, unit normal,
// material slot per pixel) and dL/d rgb_linear, computes dL/d of the
// randomized parameters the paper's randomizers draw (Sec. 4.3.1): per
// material albedo (rgb), specular k_s and emission, per light position (or
// direction) and intensity, and the exposure.  Visibility does not depend on these
// parameters, so the gradient is exact, not an approximation.
//
// Pass 1 (grid = images x blocks_per_img): each CTA owns a fixed pixel range
// of one image, which its threads stream through shared memory (cp.async,
// three chunks of 256 pixels ahead, each thread its own pixels' words).  Light and exposure terms accumulate per thread; material
// terms accumulate per warp with a segmented reduction: for every material
// present in the warp's 32 pixels the lanes with that material are summed by
// a fixed shuffle tree.  The CTA then combines its warps in warp order,
// maps light gradients from view to world space (R^T) and writes one
// partial row.  Pass 2 sums the partial rows of a sample in (camera, block)
// order.  Every addition happens in an order fixed by the data layout, so
// the result is bit-identical from run to run.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "orrb.h"
#include "orrb_internal.h"
#include "orrb_shading.cuh"

namespace orrb {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBwdThreads = 256;
constexpr int kBwdWarps = kBwdThreads / 32;

// Pixel data are staged through shared memory kStages chunks ahead: each thread copies the ten
// words of the pixels it will shade (seven G-buffer planes, three dL/drgb) with cp.async, so the
// loads of later chunks are in flight while it shades the current one.
constexpr int kStages = 3;
constexpr int kWords = 10;

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int kN>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(kN) : "memory"); }

struct BwdShared {
  float V[12];
  float lv[kMaxLights][4];
  float la[kMaxLights][4];  // spot lights: view-space axis and -cos_o, over cos_i - cos_o
  float mat[kMaxMaterials][5];
  float emis[kMaxMaterials];
  float amb[3];
  float scale;
  int n_lights, light_type, ortho, s;
  float wmat[kBwdWarps][kMaxMaterials][5];      // per-warp material sums (albedo, specular, emission)
  float wred[kBwdWarps][kMaxLights * 4];        // per-warp light sums
  float wgrade[kBwdWarps][kGradeSums];          // per-warp grading sums (graded loss)
  float gm[3][4];                               // the image's grading map c' = A c + t
  float bg[3];
  unsigned gkey;                                // the image's grain key
  float stage[kStages][kWords][kBwdThreads];    // each thread's own staged pixel words
};

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Four sums over the warp at once (a fixed order, so the result is the same every run): the
// half-warps exchange two of the four values, the quarter-warps one of the remaining two, and the
// last three steps sum one value.  Lane l returns the sum of value (l >> 3) & 3, so lanes 0, 8, 16
// and 24 hold the four sums; six shuffles instead of twenty.
__device__ __forceinline__ float warp_sum4(float a0, float a1, float a2, float a3, int lane) {
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
  const float r0 = __shfl_xor_sync(kFull, h16 ? a0 : a2, 16);
  const float r1 = __shfl_xor_sync(kFull, h16 ? a1 : a3, 16);
  const float b0 = (h16 ? a2 : a0) + r0, b1 = (h16 ? a3 : a1) + r1;
  float c = (h8 ? b1 : b0) + __shfl_xor_sync(kFull, h8 ? b0 : b1, 8);
  for (int o = 4; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
  return c;
}

// 4 CTAs (32 warps) per SM: the per-pixel loads need the occupancy more than the adjoint needs registers.
// kGraded: the loss is on the graded colour c' = A c + t + grain: d_rgb holds dL/dc', the adjoint
// of the shading takes A^T dL/dc', and the image's sums sum dc' c^T, sum dc' and the grain term
// are written for the grading parameters' gradients (formed in the reduce kernel).
template <bool kGraded>
__global__ void __launch_bounds__(kBwdThreads, 4) backward_partial_kernel(BackwardParams bp) {
  const Params& p = bp.base;
  __shared__ BwdShared sh;
  const int cam = blockIdx.x, blk = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    int s = p.cam_sample[cam];
    if (s < 0 || s >= p.n_samples) s = 0;
    sh.s = s;
    for (int k = 0; k < 12; k++) sh.V[k] = p.cam_view[cam * 12 + k];
    sh.ortho = p.cam_intr[cam * 6 + 5] != 0.0f;
    int nl = p.light_meta[s * 2];
    const int lt = p.light_meta[s * 2 + 1];
    if (!(lt == 0 || lt == 1 || (lt == 2 && p.light_spot))) nl = 0;  // lights nothing (as in the render)
    sh.n_lights = nl < 0 ? 0 : (nl > kMaxLights ? kMaxLights : nl);
    sh.light_type = lt;
    for (int l = 0; l < sh.n_lights; l++) {
      const float* L4 = p.light + (s * kMaxLights + l) * 4;
      for (int i = 0; i < 3; i++) {
        float r = sh.V[i * 4 + 0] * L4[0] + sh.V[i * 4 + 1] * L4[1] + sh.V[i * 4 + 2] * L4[2];
        sh.lv[l][i] = lt == 1 ? -r : r + sh.V[i * 4 + 3];
      }
      sh.lv[l][3] = L4[3];
      if (lt == 2) {
        const float* sp = p.light_spot + (s * kMaxLights + l) * 5;
        const bool cone = sp[4] > sp[3];
        const float w = cone ? 1.0f / (sp[4] - sp[3]) : 0.0f;
        for (int i = 0; i < 3; i++)
          sh.la[l][i] = (sh.V[i * 4 + 0] * sp[0] + sh.V[i * 4 + 1] * sp[1] + sh.V[i * 4 + 2] * sp[2]) * w;
        sh.la[l][3] = cone ? -sp[3] * w : -1.0f;
      }
    }
    sh.scale = exp2f(p.exposure_ev[s]);
    for (int k = 0; k < 3; k++) sh.amb[k] = p.ambient[s * 3 + k];
    if (kGraded) {
      grading_map(p.grading + (size_t)s * 8, sh.gm);
      sh.gkey = grain_key(p.grading + (size_t)s * 8, unsigned(cam - p.cam_offset[s]));
      for (int k = 0; k < 3; k++) sh.bg[k] = p.background[s * 3 + k];
    }
  }
  for (int k = tid; k < kBwdWarps * kMaxMaterials * 5; k += kBwdThreads) (&sh.wmat[0][0][0])[k] = 0.0f;
  __syncthreads();
  for (int k = tid; k < kMaxMaterials * 5; k += kBwdThreads)
    sh.mat[k / 5][k % 5] = p.material[(size_t)sh.s * kMaxMaterials * 5 + k];
  for (int k = tid; k < kMaxMaterials; k += kBwdThreads)
    sh.emis[k] = p.emission ? p.emission[(size_t)sh.s * kMaxMaterials + k] : 0.0f;
  __syncthreads();

  const long long N = p.total_pixels;
  const long long npx = (long long)p.cam_wh[cam * 2] * p.cam_wh[cam * 2 + 1];
  const long long chunk = (npx + bp.blocks_per_img - 1) / bp.blocks_per_img;
  const long long i0 = blk * chunk, i1 = min(npx, i0 + chunk);
  const long long base = p.img_offset[cam];
  const float scale = sh.scale;

  float gsum[kGradeSums];  // graded loss: sum dc' c^T (row-major), sum dc', sum (sum dc') grain
  for (int k = 0; k < kGradeSums; k++) gsum[k] = 0.0f;
  float dlv[kMaxLights][3], dI[kMaxLights];
  for (int l = 0; l < kMaxLights; l++) {
    dlv[l][0] = dlv[l][1] = dlv[l][2] = 0.0f;
    dI[l] = 0.0f;
  }
  // the ten words of pixel r0 + tid into stage `st` (nothing past the range: its copies are skipped)
  auto stage_pixel = [&](long long r0, int st) {
    const long long i = r0 + tid;
    if (i < i1) {
      const long long o = base + i;
      for (int k = 0; k < 7; k++) cp_async4(&sh.stage[st][k][tid], bp.gbuffer + k * N + o);
      for (int k = 0; k < 3; k++) cp_async4(&sh.stage[st][7 + k][tid], bp.d_rgb + 3 * o + k);
    }
    cp_async_commit();  // (an empty group where the range has ended keeps the group count aligned)
  };
  for (int k = 0; k < kStages - 1; k++) stage_pixel(i0 + (long long)k * kBwdThreads, k);
  int st = 0;
  for (long long r0 = i0; r0 < i1; r0 += kBwdThreads, st = st == kStages - 1 ? 0 : st + 1) {
    stage_pixel(r0 + (long long)(kStages - 1) * kBwdThreads, st == 0 ? kStages - 1 : st - 1);
    cp_async_wait<kStages - 1>();  // this thread's copies of chunk r0 have landed
    const long long i = r0 + tid;
    int mat = -1, word = -1;
    float dm[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (i < i1) {
      const float* w = &sh.stage[st][0][tid];
      // the material word: slot in bits 0-7, light l's shadowed taps in bits 8 + 4l .. 11 + 4l
      word = __float_as_int(w[6 * kBwdThreads]);
      mat = word < 0 ? -1 : (word & 0xff);
      if (mat >= kMaxMaterials) mat = -1;
      // dL/d rgb_linear: the input itself, or for a graded loss A^T dL/dc'
      const float gp[3] = {w[7 * kBwdThreads], w[8 * kBwdThreads], w[9 * kBwdThreads]};
      float g[3] = {gp[0], gp[1], gp[2]};
      if (kGraded)
        for (int k = 0; k < 3; k++) g[k] = sh.gm[0][k] * gp[0] + sh.gm[1][k] * gp[1] + sh.gm[2][k] * gp[2];
      float c[3];  // the ungraded colour (graded loss only)
      if (kGraded && mat < 0)
        for (int k = 0; k < 3; k++) c[k] = sh.bg[k];
      if (mat >= 0) {
        const float P[3] = {w[0], w[kBwdThreads], w[2 * kBwdThreads]};
        const float n[3] = {w[3 * kBwdThreads], w[4 * kBwdThreads], w[5 * kBwdThreads]};
        const float* m = sh.mat[mat];
        float Vv[3];
        if (sh.ortho) {
          Vv[0] = 0.0f;
          Vv[1] = 0.0f;
          Vv[2] = 1.0f;
        } else {
          float rl = rsqrt_approx(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
          Vv[0] = -P[0] * rl;
          Vv[1] = -P[1] * rl;
          Vv[2] = -P[2] * rl;
        }
        const float G = g[0] + g[1] + g[2];
        const float gr = g[0] * m[0] + g[1] * m[1] + g[2] * m[2];
        float sum_endl = 0.0f, sum_epw = 0.0f;
#pragma unroll
        for (int l = 0; l < kMaxLights; l++) {
          if (l >= sh.n_lights) break;
          float L[3], Lv[3] = {0.0f, 0.0f, 0.0f}, E, d2 = 1.0f, rinv = 1.0f;
          // the shadow factor (9 - k) / 9 is held fixed: it scales the intensity
          const float vis = float(9 - ((word >> (8 + 4 * l)) & 15)) * (1.0f / 9.0f);
          const float I = sh.lv[l][3] * vis;
          float S = 1.0f, dS = 0.0f;  // spot cone factor, and its derivative in t
          if (sh.light_type != 1) {
            for (int k = 0; k < 3; k++) Lv[k] = sh.lv[l][k] - P[k];
            d2 = Lv[0] * Lv[0] + Lv[1] * Lv[1] + Lv[2] * Lv[2];
            rinv = rsqrt_approx(d2);
            for (int k = 0; k < 3; k++) L[k] = Lv[k] * rinv;
            if (sh.light_type == 2) {
              const float t = __saturatef(L[0] * -sh.la[l][0] + L[1] * -sh.la[l][1] + L[2] * -sh.la[l][2] +
                                          sh.la[l][3]);
              S = t * t * (3.0f - 2.0f * t);
              dS = 6.0f * t * (1.0f - t);  // zero where t is clamped
            }
            E = I * S * (rinv * rinv);
          } else {
            for (int k = 0; k < 3; k++) L[k] = sh.lv[l][k];
            E = I;
          }
          const float ndl_raw = n[0] * L[0] + n[1] * L[1] + n[2] * L[2];
          const bool lit = ndl_raw > 0.0f;
          const float ndl = lit ? ndl_raw : 0.0f;
          // the half vector Hv = L + V and its reciprocal length rh (H = Hv rh is not formed)
          float pw = 0.0f, ndh = 0.0f, Hv[3] = {0.0f, 0.0f, 0.0f}, rh = 0.0f;
          bool has_h = false;
          if (lit) {
            for (int k = 0; k < 3; k++) Hv[k] = L[k] + Vv[k];
            const float h2 = Hv[0] * Hv[0] + Hv[1] * Hv[1] + Hv[2] * Hv[2];
            if (h2 > 0.0f) {
              has_h = true;
              rh = rsqrt_approx(h2);
              ndh = fmaxf(0.0f, (n[0] * Hv[0] + n[1] * Hv[1] + n[2] * Hv[2]) * rh);
              pw = lobe_pow(ndh, m[4]);
            }
          }
          const float spec = m[3] * pw;
          sum_endl += E * ndl;
          sum_epw += E * pw;
          const float dE = scale * (gr * ndl + G * spec);
          const float dndl = lit ? scale * E * gr : 0.0f;
          // alpha * ndh^(alpha - 1) = alpha * pw / ndh for ndh > 0 (fast division: ~2 ulp)
          const float dndh = (has_h && ndh > 0.0f) ? scale * E * G * m[3] * m[4] * __fdividef(pw, ndh) : 0.0f;
          // through the half vector's normalisation, dL = dndl n + (dH - H (H . dH)) rh with dH = dndh n;
          // dndh is non-zero only where ndh = n . H > 0, so H . dH = dndh ndh and
          // dL = (dndl + dndh rh) n - (dndh ndh rh) H = (dndl + dndh rh) n - (dndh ndh rh^2) Hv
          const float cn = dndl + dndh * rh, ch = dndh * ndh * (rh * rh);
          float dL[3] = {cn * n[0] - ch * Hv[0], cn * n[1] - ch * Hv[1], cn * n[2] - ch * Hv[2]};
          if (sh.light_type != 1) {
            const float r2 = rinv * rinv;
            dI[l] += dE * S * r2 * vis;
            const float dd2 = -dE * E * r2;  // (E = I S r2)
            // spot: t = -(L . a) / (cos_i - cos_o) + ..., so dE/dL = -I |Lv|^-2 S'(t) la_xyz
            if (sh.light_type == 2) {
              const float ds = dE * I * (rinv * rinv) * dS;
              for (int k = 0; k < 3; k++) dL[k] -= ds * sh.la[l][k];
            }
            // through L = Lv / |Lv|: (dL - L (L . dL)) rinv = dL rinv - Lv (L . dL) rinv^2, plus the
            // inverse-square law's 2 dd2 Lv
            const float ld = L[0] * dL[0] + L[1] * dL[1] + L[2] * dL[2];
            const float cl = 2.0f * dd2 - ld * (rinv * rinv);
            for (int k = 0; k < 3; k++) dlv[l][k] += dL[k] * rinv + cl * Lv[k];
          } else {
            dI[l] += dE * vis;
            for (int k = 0; k < 3; k++) dlv[l][k] += dL[k];
          }
        }
        const float em = sh.emis[mat];
        for (int k = 0; k < 3; k++) dm[k] = g[k] * scale * (sh.amb[k] + em + sum_endl);
        dm[3] = scale * G * sum_epw;
        dm[4] = scale * gr;
        if (kGraded)
          for (int k = 0; k < 3; k++) c[k] = scale * (m[k] * (sh.amb[k] + em + sum_endl) + m[3] * sum_epw);
      }
      if (kGraded) {
        for (int a = 0; a < 3; a++) {
          for (int b = 0; b < 3; b++) gsum[a * 3 + b] += gp[a] * c[b];
          gsum[9 + a] += gp[a];
        }
        gsum[12] += (gp[0] + gp[1] + gp[2]) * grain_centred(sh.gkey, unsigned(i));
      }
    }
    // segmented warp reduction over the materials present in these 32 pixels; a warp on one
    // material (most steps: the table) reduces once without the segment search
    const int mat0 = __shfl_sync(kFull, mat, 0);
    if (__all_sync(kFull, mat == mat0) && mat0 >= 0) {
      const float v = warp_sum4(dm[0], dm[1], dm[2], dm[3], lane);
      const float v4 = bp.d_emission ? warp_sum(dm[4]) : 0.0f;
      if ((lane & 7) == 0) sh.wmat[warp][mat0][lane >> 3] += v;
      if (lane == 0) sh.wmat[warp][mat0][4] += v4;
      continue;
    }
    unsigned pending = __ballot_sync(kFull, mat >= 0);
    while (pending) {
      const int leader = __ffs(pending) - 1;
      const int mm = __shfl_sync(kFull, mat, leader);
      const bool mine = mat == mm;
      const float v = warp_sum4(mine ? dm[0] : 0.0f, mine ? dm[1] : 0.0f, mine ? dm[2] : 0.0f,
                                mine ? dm[3] : 0.0f, lane);
      // (the emission sums only when the caller asked for their gradients)
      const float v4 = bp.d_emission ? warp_sum(mine ? dm[4] : 0.0f) : 0.0f;
      if ((lane & 7) == 0) sh.wmat[warp][mm][lane >> 3] += v;
      if (lane == 0) sh.wmat[warp][mm][4] += v4;
      pending &= ~__ballot_sync(kFull, mine);
    }
  }
  // per-thread light and exposure sums -> per warp (fixed tree) -> per CTA (warp order)
  for (int l = 0; l < kMaxLights; l++) {
    const float v = warp_sum4(dlv[l][0], dlv[l][1], dlv[l][2], dI[l], lane);
    if ((lane & 7) == 0) sh.wred[warp][l * 4 + (lane >> 3)] = v;
  }
  if (kGraded)
    for (int k = 0; k < kGradeSums; k++) {
      const float v = warp_sum(gsum[k]);
      if (lane == 0) sh.wgrade[warp][k] = v;
    }
  __syncthreads();
  float* out = bp.partial + ((size_t)cam * bp.blocks_per_img + blk) * kGradFloats;
  for (int k = tid; k < kMaxMaterials * 5; k += kBwdThreads) {
    float v = 0.0f;
    for (int w = 0; w < kBwdWarps; w++) v += (&sh.wmat[w][0][0])[k];
    const int mm = k / 5, c = k % 5;
    out[c < 4 ? mm * 4 + c : kGradEmission + mm] = v;
  }
  if (tid < kMaxLights) {
    const int l = tid;
    float dv[3], di = 0.0f;
    for (int k = 0; k < 3; k++) {
      dv[k] = 0.0f;
      for (int w = 0; w < kBwdWarps; w++) dv[k] += sh.wred[w][l * 4 + k];
    }
    for (int w = 0; w < kBwdWarps; w++) di += sh.wred[w][l * 4 + 3];
    // view -> world: point p_v = R p + t, so dp = R^T dp_v; direction L_v = -R d, so dd = -R^T dL_v
    const float sgn = sh.light_type == 1 ? -1.0f : 1.0f;
    for (int j = 0; j < 3; j++)
      out[kMaxMaterials * 4 + l * 4 + j] =
          sgn * (sh.V[0 * 4 + j] * dv[0] + sh.V[1 * 4 + j] * dv[1] + sh.V[2 * 4 + j] * dv[2]);
    out[kMaxMaterials * 4 + l * 4 + 3] = di;
  }
  if (tid == 0) out[kMaxMaterials * 4 + kMaxLights * 4] = 0.0f;  // (the exposure: formed by the reduce kernel)
  if (tid >= 32 && tid < 32 + kGradeSums) {
    float v = 0.0f;
    if (kGraded)
      for (int w = 0; w < kBwdWarps; w++) v += sh.wgrade[w][tid - 32];
    out[kGradGrade + tid - 32] = v;
  }
}

// The gradients of the grading parameters from an image-summed graded loss: with c' = A c + t +
// a n per pixel, A = k S R W (contrast k, saturation S, rotation R by h about the grey axis, white
// balance W = diag(1 + t, 1 + u, 1 - t)) and t = (1 - k) / 2 + b, dL/dtheta = sum_ij dA_ij/dtheta
// M_ij + sum_i dt_i/dtheta s_i with M = sum dc' c^T and s = sum dc' (the partial rows' sums); the
// grain amplitude's is sum (sum_k dc'_k) n.  Out: d hue, saturation, contrast, brightness,
// temperature, tint, grain amplitude, 0 (the seed).
__device__ void grading_grads(const float* g, const float* sums, float* out) {
  float hs, hc;
  sincosf(g[0], &hs, &hc);
  const float kx = 0.57735026918962576f;
  const float a = hc + (1.0f - hc) / 3.0f, b = (1.0f - hc) / 3.0f - kx * hs, c = (1.0f - hc) / 3.0f + kx * hs;
  const float da = -2.0f * hs / 3.0f, db = hs / 3.0f - kx * hc, dc = hs / 3.0f + kx * hc;  // d/dh
  const float R[3][3] = {{a, b, c}, {c, a, b}, {b, c, a}};
  const float dR[3][3] = {{da, db, dc}, {dc, da, db}, {db, dc, da}};
  const float wb[3] = {1.0f + g[4], 1.0f + g[5], 1.0f - g[4]};
  const float Yw[3] = {0.2126f, 0.7152f, 0.0722f};
  const float sat = g[1], con = g[2];
  const float* M = sums;
  const float* sv = sums + 9;
  float d_h = 0.0f, d_sat = 0.0f, d_con = 0.0f, d_t = 0.0f, d_u = 0.0f;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      float sr = 0.0f, sdr = 0.0f, dsr = 0.0f;  // (S R)_ij, (S dR/dh)_ij, (dS/dsat R)_ij
      for (int m = 0; m < 3; m++) {
        const float S_im = (i == m ? sat : 0.0f) + (1.0f - sat) * Yw[m];
        const float dS_im = (i == m ? 1.0f : 0.0f) - Yw[m];
        sr += S_im * R[m][j];
        sdr += S_im * dR[m][j];
        dsr += dS_im * R[m][j];
      }
      const float Mij = M[i * 3 + j];
      d_h += con * sdr * wb[j] * Mij;
      d_sat += con * dsr * wb[j] * Mij;
      d_con += sr * wb[j] * Mij;
      d_t += con * sr * (j == 0 ? 1.0f : (j == 2 ? -1.0f : 0.0f)) * Mij;
      d_u += con * sr * (j == 1 ? 1.0f : 0.0f) * Mij;
    }
  const float ssum = sv[0] + sv[1] + sv[2];
  out[0] = d_h;
  out[1] = d_sat;
  out[2] = d_con - 0.5f * ssum;
  out[3] = ssum;
  out[4] = d_t;
  out[5] = d_u;
  out[6] = sums[12];
  out[7] = 0.0f;
}

// One thread per (sample, gradient float): sum the sample's partial rows in (camera, block) order;
// for a graded loss one thread then forms the grading gradients from the summed grading sums.
constexpr int kReduceThreads = 192;
static_assert(kGradFloats <= kReduceThreads, "one thread per gradient float");
__global__ void __launch_bounds__(kReduceThreads) backward_reduce_kernel(BackwardParams bp) {
  const Params& p = bp.base;
  const int s = blockIdx.x, k = threadIdx.x;
  __shared__ float gsums[kGradeSums];
  __shared__ float dmat[kMaxMaterials * 4];
  float v = 0.0f;
  if (k < kGradFloats)
    for (int c = p.cam_offset[s]; c < p.cam_offset[s + 1]; c++)
      for (int b = 0; b < bp.blocks_per_img; b++) v += bp.partial[((size_t)c * bp.blocks_per_img + b) * kGradFloats + k];
  if (k < kMaxMaterials * 4) {
    dmat[k] = v;
    if (bp.d_material) bp.d_material[(size_t)s * kMaxMaterials * 4 + k] = v;
  } else if (k < kMaxMaterials * 4 + kMaxLights * 4) {
    if (bp.d_light) bp.d_light[(size_t)s * kMaxLights * 4 + (k - kMaxMaterials * 4)] = v;
  } else if (k < kGradEmission) {
    // (the exposure slot of the partial rows is zero)
  } else if (k < kGradGrade) {
    if (bp.d_emission) bp.d_emission[(size_t)s * kMaxMaterials + (k - kGradEmission)] = v;
  } else if (k < kGradFloats) {
    gsums[k - kGradGrade] = v;
  }
  __syncthreads();
  // The linear colour is linear in each material's (albedo rgb, specular) with no constant term,
  // and the exposure scales all of it: d rgb / d ev = ln 2 rgb = ln 2 sum_m m . d rgb / d m.  So
  // dL/d ev = ln 2 sum over materials of m . dL/dm, formed here from the material gradients
  // instead of per pixel (materials in index order).
  if (k == 32 && bp.d_exposure) {
    const float* ms = p.material + (size_t)s * kMaxMaterials * 5;
    float e = 0.0f;
    for (int m = 0; m < kMaxMaterials; m++)
      e += ms[m * 5 + 0] * dmat[m * 4 + 0] + ms[m * 5 + 1] * dmat[m * 4 + 1] + ms[m * 5 + 2] * dmat[m * 4 + 2] +
           ms[m * 5 + 3] * dmat[m * 4 + 3];
    bp.d_exposure[s] = 0.69314718055994530942f * e;
  }
  if (k == 0 && bp.d_grading && p.grading)
    grading_grads(p.grading + (size_t)s * 8, gsums, bp.d_grading + (size_t)s * 8);
}

}  // namespace

int launch_backward(const BackwardParams& bp, int threads, void* stream, char* err, size_t errlen) {
  (void)threads;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (bp.d_grading && bp.base.grading)
    backward_partial_kernel<true><<<dim3(bp.base.n_cams, bp.blocks_per_img), kBwdThreads, 0, st>>>(bp);
  else
    backward_partial_kernel<false><<<dim3(bp.base.n_cams, bp.blocks_per_img), kBwdThreads, 0, st>>>(bp);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    backward_reduce_kernel<<<bp.base.n_samples, kReduceThreads, 0, st>>>(bp);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    snprintf(err, errlen, "backward launch failed: %s", cudaGetErrorString(e));
    return 1;
  }
  return 0;
}

}  // namespace orrb
