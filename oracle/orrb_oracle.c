/*
 * orrb_oracle.c -- plain CPU oracle of the batched renderer.
 *
 * TEST INFRASTRUCTURE ONLY (see orrb_oracle.h).  One image at a time, one
 * triangle at a time, every pixel of the triangle's bounding box tested: no
 * binning, no tiles, nothing shared with the CUDA path.
 *
 * What is computed (the paper fixes the channels -- RGB, segmentation, depth,
 * screen-space normal, Sec. 4.4 -- and the randomized inputs, Sec. 4.3.1; it
 * gives no rasterisation rule, so each numbered step below is the reading
 * this project adopts):
 *   1  world is z-up; the camera looks down -z with +y up; screen x right,
 *      y down; pixel (x, y) has its centre at (x + 1/2, y + 1/2).
 *   2  MV = V * M per (image, instance), fixed summation order; vertices and
 *      normals go to view space with the same fixed order.
 *   3  triangles are clipped against z <= -near (Sutherland-Hodgman); the
 *      cut point is always interpolated from the inside vertex towards the
 *      outside one, so two triangles sharing an edge cut it identically; the
 *      cut is computed in fp64 and rounded once to fp32, with z = -near
 *      exactly.  A clipped quad is split into (o0,o1,o2) sub 0 and
 *      (o0,o2,o3) sub 1.
 *   4  projection x_s = cx + fx*(x*iw), y_s = cy - fy*(y*iw), iw = 1/(-z)
 *      (orthographic: x_s = cx + fx*x, y_s = cy - fy*y, depth -z); snapped
 *      to 8 fractional bits with round-half-even; a triangle with a vertex
 *      beyond |x_s|, |y_s| >= 2^20 px is dropped and counted.
 *   5  integer edge functions E_ab(p) = (p.x-a.x)(b.y-a.y) - (p.y-a.y)(b.x-a.x)
 *      in 64 bits; area A = E_01(v2); triangles with A <= 0 are culled.
 *   6  pixel centre (256x+128, 256y+128) is covered iff every edge weight is
 *      > 0, or == 0 on a top edge (dy == 0, dx < 0) or left edge (dy > 0).
 *   7  depth = A / (w0*iw0 + w1*iw1 + w2*iw2) with the w_i, A converted to
 *      float and summed left to right (orthographic: (w0*d0+w1*d1+w2*d2)/A).
 *   8  the nearest fragment wins by (depth, key) ascending, key = 2*prim+sub,
 *      prim = triangle index in the sample's concatenated triangle list.
 *   9  G-buffer: P = (depth ux, depth uy, -depth) with ux = ((x + 1/2) - cx)
 *      * (1/fx), uy = -(((y + 1/2) - cy) * (1/fy)), each operation rounded
 *      separately, 1/fx the correctly rounded reciprocal (orthographic: (ux,
 *      uy, -depth)); normal = sum_i (w_i*iw_i) n_i normalised; material =
 *      base + tri_mat; seg id.
 *  10  Blinn-Phong over the sample's lights, inverse-square falloff for
 *      point and spot lights, white specular, plus (ambient + emission) *
 *      albedo, all times 2^EV.  Emission e is a scalar per material, the
 *      emitted colour e * albedo (a MuJoCo material's emission, Sec. 4.2).
 *      A spot light (type 2) is a point light times the cone factor
 *      S = t^2 (3 - 2t), t = clamp((x - cos_o) / (cos_i - cos_o), 0, 1), x
 *      the cosine between the spot axis and the direction from the light to
 *      the point: 1 inside the inner cone, 0 outside the outer one (Sec.
 *      4.3.1's spotlight angles).  A cone with cos_i <= cos_o, a type other
 *      than 0 point, 1 directional, 2 spot, or a spot without its cone table
 *      lights nothing.
 *  11  rgb8 = floor(clamp(rgb,0,1)*255 + 1/2); normal -> binary16 (RNE);
 *      background: rgb = background colour, depth 0, normal 0, seg 0.
 *  12  the adjoint of step 10 at fixed visibility, in fp64.
 *  13  optional colour grading of the rgb8 channel (the post-processing
 *      randomizer, Sec. 4.3.1), per sample g = (hue h, saturation s, contrast
 *      k, brightness b, temperature t, tint u, grain a, grain seed), applied to
 *      the linear colour (pixels and background) before step 11's
 *      quantisation, in this order and in fp32:
 *        white balance  r *= 1 + t, g *= 1 + u, b *= 1 - t;
 *        hue            rotation by h about the grey axis (1,1,1)/sqrt(3):
 *                       c' = c cos h + (k x c) sin h + k (k . c)(1 - cos h);
 *        saturation     c = Y + s (c - Y), Y = 0.2126 r + 0.7152 g + 0.0722 b;
 *        contrast       c = (c - 1/2) k + 1/2;   brightness  c = c + b;
 *        grain          c = c + a (n - 1/2) on all three channels, n in [0, 1)
 *                       from the PCG hash (Jarzynski and Olano, "Hash
 *                       Functions for GPU Rendering", 2020): n = pcg(pcg(seed
 *                       + 0x9E3779B9 (j + 1)) ^ i) / 2^32, j the camera's
 *                       index within its sample, i the pixel's within its
 *                       image.  rgb_linear stays ungraded.
 *  14  optional tracker rows (the Tracker component, Sec. 4.3.2; per camera
 *      and instance of its sample): the
 *      8.8 fixed-point screen box (x0, y0, x1, y1) of the instance's mesh
 *      vertices (those its triangles use) that lie in front of the near plane
 *      and inside the guard band, snapped as in step 4 (empty: x0 = y0 =
 *      INT32_MAX, x1 = y1 = INT32_MIN); the snapped projection (kx, ky) of the
 *      instance's origin (its pose translation); flags bit 0: box not empty,
 *      bit 1: origin projected; a zero.  An instance of a mesh without
 *      triangles keeps an empty row.
 *  15  optional shadow maps (soft shadows of the benchmark's lights, Sec. 5):
 *      each light has F shadow cameras ("faces": one for a spot light, six
 *      cube faces for a point light); face f of light l of sample s casts
 *      when l < the light count and its camera (view S, intrinsics fx, fy,
 *      cx, cy, near, bias, type: 0 perspective, 1 orthographic as for a
 *      directional light) has fx != 0.  Its R x R map holds, per pixel, the
 *      depth seen from that camera (steps 2-8 with it) of the nearest BACK
 *      face -- each triangle's second and third vertices swapped
 *      before step 5, so front faces are culled -- and 0 where there is none.
 *  16  shadow lookup in step 10: for a camera pixel with surface and each
 *      light with a casting face, in fp32, every operation rounded to nearest:
 *      P as in step 9; for the faces in order, M = S V^-1 (V^-1 = [R^T | -R^T t],
 *      products summed in index order, each operation rounded separately),
 *      q_i = fma(M_i2, P_z, fma(M_i1, P_y, fma(M_i0, P_x, M_i3))) (fused
 *      multiply-adds, one rounding each), z = -q_z, u = fma(fx, q_x (1/z), cx),
 *      v = fma(-fy, q_y (1/z), cy) (orthographic: u = fma(fx, q_x, cx),
 *      v = fma(-fy, q_y, cy)); the first face with
 *      z > near and (floor(u), floor(v)) inside its map decides (none: the
 *      light is unshadowed): over the 3 x 3 texels (floor(u) + a, floor(v) +
 *      b), a, b in {-1, 0, 1}, inside the map, count k those with map depth
 *      d > 0 and z - bias > d (percentage-closer filtering, Reeves, Salesin
 *      and Cook 1987); E_l is multiplied by (9 - k) / 9.  The G-buffer's material word
 *        carries k of light l in bits 8 + 4l .. 11 + 4l (the adjoint holds it
 *        fixed: visibility does not depend on the shading parameters).
 *  17  optional post-processing of a sample's images (the rest of the
 *      post-processing randomizer, Sec. 4.3.1: ambient-occlusion intensity a,
 *      bloom intensity beta and bloom radius sigma in pixels, per sample),
 *      applied to the linear colour c of every pixel (step 10, or the
 *      background) before step 13's grading and step 11's quantisation; it
 *      reads only the image's depth channel and its binary16 normals (n, as
 *      decoded), and is computed here in fp64, rounded to fp32 once at the end:
 *        ambient occlusion: for a pixel with surface, P its position as in
 *          step 9 from its depth, and each of eight offsets (dx, dy) =
 *          (2, 1), (-1, 3), (-4, -1), (1, -4), (5, 2), (-2, 5), (-5, -3), (3, -6)
 *          whose pixel lies in the image and has a surface, v = P' - P, L = |v|:
 *          o = max(0, (n . v) / L - 0.1) / (1 + L^2 / 0.05^2) (0 where L = 0);
 *          O = (sum of o) / 8 over all eight; c = c * max(0, 1 - a O).
 *          Pixels without surface keep c.
 *        bloom (where beta != 0 and sigma > 0): the bright part
 *          b = max(c - 1, 0) per channel is blurred by the Gaussian
 *          w_i = exp(-i^2 / (2 sigma^2)) / sum_j exp(-j^2 / (2 sigma^2)),
 *          |i|, |j| <= R = min(ceil(3 sigma), 16), first along rows, then along
 *          columns, pixel indices clamped to the image:
 *          B(x, y) = sum_j w_j sum_i w_i b(clamp(x + i), clamp(y + j));
 *          c = c + beta B.
 */
#include "orrb_oracle.h"

#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define GUARD_PX 1048576.0f /* 2^20 */

typedef struct {
  float p[3];
  float n[3];
} vtx;

typedef struct {
  int64_t key;
  float depth;
  float depth2;
  int32_t X[3], Y[3];
  float iw[3];
  float n[3][3];
  int32_t mat;
  int32_t seg;
  int32_t count;
} pixel_winner;

/* ------------------------------------------------------------------ */
/* step 2: MV = V * M with a fixed order of the sums                   */
/* ------------------------------------------------------------------ */
static void compose_mv(const float* V, const float* M, float* MV) {
  for (int i = 0; i < 3; i++) {
    for (int j = 0; j < 4; j++) {
      float s = V[i * 4 + 0] * M[0 * 4 + j];
      s = s + V[i * 4 + 1] * M[1 * 4 + j];
      s = s + V[i * 4 + 2] * M[2 * 4 + j];
      if (j == 3) s = s + V[i * 4 + 3];
      MV[i * 4 + j] = s;
    }
  }
}

static vtx to_view(const float* MV, const float* p, const float* n) {
  vtx v;
  for (int i = 0; i < 3; i++) {
    v.p[i] = ((MV[i * 4 + 0] * p[0] + MV[i * 4 + 1] * p[1]) + MV[i * 4 + 2] * p[2]) + MV[i * 4 + 3];
    v.n[i] = (MV[i * 4 + 0] * n[0] + MV[i * 4 + 1] * n[1]) + MV[i * 4 + 2] * n[2];
  }
  return v;
}

/* ------------------------------------------------------------------ */
/* step 3: near-plane clipping                                         */
/* ------------------------------------------------------------------ */
static vtx cut(const vtx* in, const vtx* out, float near) {
  /* fp64, rounded once to fp32: an fp32 lerp leaves an absolute error of
     the far vertex's magnitude, which seen from z = -near tilts the clipped
     triangle by (error / near) radians */
  double t = (-(double)near - (double)in->p[2]) / ((double)out->p[2] - (double)in->p[2]);
  vtx r;
  for (int k = 0; k < 3; k++) {
    r.p[k] = (float)((double)in->p[k] + t * ((double)out->p[k] - (double)in->p[k]));
    r.n[k] = (float)((double)in->n[k] + t * ((double)out->n[k] - (double)in->n[k]));
  }
  r.p[2] = -near; /* on the near plane by construction */
  return r;
}

static int clip_near(const vtx* v, float near, vtx* o) {
  int n = 0;
  for (int k = 0; k < 3; k++) {
    const vtx* a = &v[k];
    const vtx* b = &v[(k + 1) % 3];
    int ain = a->p[2] <= -near;
    int bin = b->p[2] <= -near;
    if (ain) o[n++] = *a;
    if (ain && !bin) o[n++] = cut(a, b, near);
    if (!ain && bin) o[n++] = cut(b, a, near);
  }
  return n;
}

/* ------------------------------------------------------------------ */
/* step 5 helpers                                                      */
/* ------------------------------------------------------------------ */
static int64_t edge(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t px, int64_t py) {
  return (px - ax) * (by - ay) - (py - ay) * (bx - ax);
}

static int top_left(int64_t ax, int64_t ay, int64_t bx, int64_t by) {
  int64_t dx = bx - ax, dy = by - ay;
  return (dy == 0 && dx < 0) || dy > 0;
}

static int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
  return q;
}

/* Coverage and visibility of one snapped triangle (steps 5-8).
 * Returns the number of covered pixels; updates the per-pixel winners. */
static int64_t raster_triangle(int32_t W, int32_t H, const int32_t X[3], const int32_t Y[3],
                               const float iw[3], int ortho, int64_t key, const float n[3][3],
                               int32_t mat, int32_t seg, pixel_winner* px, int64_t* culled) {
  int64_t A = edge(X[0], Y[0], X[1], Y[1], X[2], Y[2]);
  if (A <= 0) {
    if (culled) (*culled)++;
    return 0;
  }
  int tl0 = top_left(X[1], Y[1], X[2], Y[2]);
  int tl1 = top_left(X[2], Y[2], X[0], Y[0]);
  int tl2 = top_left(X[0], Y[0], X[1], Y[1]);
  int64_t xmin = X[0], xmax = X[0], ymin = Y[0], ymax = Y[0];
  for (int k = 1; k < 3; k++) {
    if (X[k] < xmin) xmin = X[k];
    if (X[k] > xmax) xmax = X[k];
    if (Y[k] < ymin) ymin = Y[k];
    if (Y[k] > ymax) ymax = Y[k];
  }
  /* pixel x has its centre at 256x+128: candidates are the centres inside the box */
  int64_t x0 = -floor_div(-(xmin - 128), 256), x1 = floor_div(xmax - 128, 256);
  int64_t y0 = -floor_div(-(ymin - 128), 256), y1 = floor_div(ymax - 128, 256);
  if (x0 < 0) x0 = 0;
  if (y0 < 0) y0 = 0;
  if (x1 > W - 1) x1 = W - 1;
  if (y1 > H - 1) y1 = H - 1;
  float fA = (float)A;
  int64_t covered = 0;
  for (int64_t y = y0; y <= y1; y++) {
    for (int64_t x = x0; x <= x1; x++) {
      int64_t cxp = 256 * x + 128, cyp = 256 * y + 128;
      int64_t w0 = edge(X[1], Y[1], X[2], Y[2], cxp, cyp);
      int64_t w1 = edge(X[2], Y[2], X[0], Y[0], cxp, cyp);
      int64_t w2 = edge(X[0], Y[0], X[1], Y[1], cxp, cyp);
      int in0 = w0 > 0 || (w0 == 0 && tl0);
      int in1 = w1 > 0 || (w1 == 0 && tl1);
      int in2 = w2 > 0 || (w2 == 0 && tl2);
      if (!(in0 && in1 && in2)) continue;
      float f0 = (float)w0, f1 = (float)w1, f2 = (float)w2;
      float depth;
      if (ortho) {
        float s = (f0 * iw[0] + f1 * iw[1]) + f2 * iw[2];
        depth = s / fA;
      } else {
        float s = (f0 * iw[0] + f1 * iw[1]) + f2 * iw[2];
        depth = fA / s;
      }
      covered++;
      pixel_winner* p = &px[y * W + x];
      p->count++;
      int wins = depth < p->depth || (depth == p->depth && key < p->key);
      if (wins) {
        if (p->key != key && p->depth < p->depth2) p->depth2 = p->depth;
        p->key = key;
        p->depth = depth;
        for (int k = 0; k < 3; k++) {
          p->X[k] = X[k];
          p->Y[k] = Y[k];
          p->iw[k] = iw[k];
          if (n) {
            p->n[k][0] = n[k][0];
            p->n[k][1] = n[k][1];
            p->n[k][2] = n[k][2];
          }
        }
        p->mat = mat;
        p->seg = seg;
      } else if (key != p->key && depth < p->depth2) {
        p->depth2 = depth;
      }
    }
  }
  return covered;
}

static void reset_winners(pixel_winner* px, int64_t n) {
  for (int64_t i = 0; i < n; i++) {
    px[i].key = -1;
    px[i].depth = INFINITY;
    px[i].depth2 = INFINITY;
    px[i].mat = -1;
    px[i].seg = 0;
    px[i].count = 0;
  }
}

/* ------------------------------------------------------------------ */
/* step 11: binary16 encoding, round to nearest even                   */
/* ------------------------------------------------------------------ */
uint16_t orc_f32_to_f16(float f) {
  uint32_t x;
  memcpy(&x, &f, 4);
  uint32_t sign = (x >> 16) & 0x8000u;
  int32_t exp = (int32_t)((x >> 23) & 0xffu);
  uint32_t man = x & 0x7fffffu;
  if (exp == 0xff) return (uint16_t)(sign | 0x7c00u | (man ? 0x200u : 0u));
  int32_t e = exp - 127 + 15;
  if (e >= 31) return (uint16_t)(sign | 0x7c00u);
  if (e <= 0) {
    if (exp == 0) return (uint16_t)sign; /* fp32 zero or subnormal: far below binary16 range */
    uint64_t M = (uint64_t)(man | 0x800000u);
    int shift = 14 - e;
    if (shift > 40) return (uint16_t)sign;
    uint64_t m = M >> shift;
    uint64_t rem = M & ((1ull << shift) - 1ull);
    uint64_t half = 1ull << (shift - 1);
    if (rem > half || (rem == half && (m & 1ull))) m++;
    return (uint16_t)(sign | (uint32_t)m);
  }
  uint32_t h = ((uint32_t)e << 10) | (man >> 13);
  uint32_t rem = man & 0x1fffu;
  if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) h++;
  return (uint16_t)(sign | h);
}

/* step 13: the PCG hash, as published (one LCG step, a random xorshift, a multiply) */
static uint32_t pcg_hash(uint32_t v) {
  uint32_t state = v * 747796405u + 2891336453u;
  uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
  return (word >> 22u) ^ word;
}

/* fp32 operations of one call that depend on the pixel: 3 white-balance products, the mean (3),
   the cross product (6), the rotation (15), the luma (5), the grain value (2) and 10 per channel
   (30); the per-sample factors 1 +- t, 1 + u, cos, sin and 1 - cos (6) are counted once per image */
#define ORC_GRADE_OPS 64
#define ORC_GRADE_IMAGE_OPS 6
static void grade(const float* g, int32_t cam_local, int64_t pixel, float c[3]) {
  float r = c[0] * (1.0f + g[4]), gr = c[1] * (1.0f + g[5]), bl = c[2] * (1.0f - g[4]);
  const float ch = cosf(g[0]), sh = sinf(g[0]);
  const float inv_sqrt3 = 0.57735026918962576f;
  const float mean = (r + gr + bl) / 3.0f;
  const float x0 = (bl - gr) * inv_sqrt3, x1 = (r - bl) * inv_sqrt3, x2 = (gr - r) * inv_sqrt3; /* k x c */
  float h[3] = {r * ch + x0 * sh + mean * (1.0f - ch), gr * ch + x1 * sh + mean * (1.0f - ch),
                bl * ch + x2 * sh + mean * (1.0f - ch)};
  const float Y = 0.2126f * h[0] + 0.7152f * h[1] + 0.0722f * h[2];
  const uint32_t seed = (uint32_t)g[7];
  const uint32_t h1 = pcg_hash(seed + 0x9E3779B9u * (uint32_t)(cam_local + 1));
  const float n = (float)pcg_hash(h1 ^ (uint32_t)pixel) * 2.3283064365386963e-10f; /* 2^-32 */
  for (int k = 0; k < 3; k++) {
    float v = Y + g[1] * (h[k] - Y);
    v = (v - 0.5f) * g[2] + 0.5f;
    v = v + g[3];
    c[k] = v + g[6] * (n - 0.5f);
  }
}

static uint8_t quantise(float v) {
  float c = v < 0.0f ? 0.0f : (v > 1.0f ? 1.0f : v);
  return (uint8_t)floorf(c * 255.0f + 0.5f);
}

/* ------------------------------------------------------------------ */
/* step 17: ambient occlusion and bloom, fp64                          */
/* ------------------------------------------------------------------ */
/* binary16 bits -> value (IEEE 754: sign, 5 exponent bits biased by 15, 10 fraction bits;
   exponent 0 holds the subnormals m * 2^-24) */
static double f16_value(uint16_t h) {
  const int sign = h >> 15, e = (h >> 10) & 31, m = h & 1023;
  double v;
  if (e == 0) v = ldexp((double)m, -24);
  else if (e == 31) v = m ? NAN : INFINITY;
  else v = ldexp(1024.0 + (double)m, e - 25);
  return sign ? -v : v;
}

static const int POST_DX[8] = {2, -1, -4, 1, 5, -2, -5, 3};
static const int POST_DY[8] = {1, 3, -1, -4, 2, 5, -3, -6};

int orc_post_image(int32_t W, int32_t H, const float* in, const float* q, float* col, const float* depth,
                   const uint16_t* normal) {
  const double a = q[0], beta = q[1], sigma = q[2];
  const int64_t N = (int64_t)W * H;
  double* c = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
  if (!c) return -1;
  for (int64_t i = 0; i < 3 * N; i++) c[i] = col[i];
  if (a != 0.0) {
    /* positions as in step 9, from the depth */
    const double fx = in[0], fy = in[1], cx = in[2], cy = in[3];
    const int ortho = in[5] != 0.0f;
    for (int32_t y = 0; y < H; y++)
      for (int32_t x = 0; x < W; x++) {
        const int64_t i = (int64_t)y * W + x;
        if (!(depth[i] > 0.0f)) continue;
        double P[3], n[3];
        const double ux = ((x + 0.5) - cx) / fx, uy = -(((y + 0.5) - cy) / fy), d = depth[i];
        P[0] = ortho ? ux : d * ux;
        P[1] = ortho ? uy : d * uy;
        P[2] = -d;
        for (int k = 0; k < 3; k++) n[k] = f16_value(normal[i * 3 + k]);
        double O = 0.0;
        for (int k = 0; k < 8; k++) {
          const int32_t qx = x + POST_DX[k], qy = y + POST_DY[k];
          if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
          const int64_t j = (int64_t)qy * W + qx;
          if (!(depth[j] > 0.0f)) continue;
          const double uxq = ((qx + 0.5) - cx) / fx, uyq = -(((qy + 0.5) - cy) / fy), dq = depth[j];
          const double v[3] = {(ortho ? uxq : dq * uxq) - P[0], (ortho ? uyq : dq * uyq) - P[1], -dq - P[2]};
          const double L2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
          if (!(L2 > 0.0)) continue;
          const double L = sqrt(L2);
          const double cosine = (n[0] * v[0] + n[1] * v[1] + n[2] * v[2]) / L - 0.1;
          if (cosine > 0.0) O += cosine / (1.0 + L2 / (0.05 * 0.05));
        }
        O /= 8.0;
        double f = 1.0 - a * O;
        if (f < 0.0) f = 0.0;
        for (int k = 0; k < 3; k++) c[i * 3 + k] *= f;
      }
  }
  if (beta != 0.0 && sigma > 0.0) {
    int R = (int)ceil(3.0 * sigma);
    if (R > 16) R = 16;
    double w[33], sw = 0.0;
    for (int i = -R; i <= R; i++) {
      w[i + 16] = exp(-(double)(i * i) / (2.0 * sigma * sigma));
      sw += w[i + 16];
    }
    for (int i = -R; i <= R; i++) w[i + 16] /= sw;
    double* h = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    if (!h) {
      free(c);
      return -1;
    }
    for (int32_t y = 0; y < H; y++) /* along rows */
      for (int32_t x = 0; x < W; x++)
        for (int k = 0; k < 3; k++) {
          double acc = 0.0;
          for (int i = -R; i <= R; i++) {
            int32_t xx = x + i;
            xx = xx < 0 ? 0 : (xx >= W ? W - 1 : xx);
            const double v = c[((int64_t)y * W + xx) * 3 + k] - 1.0;
            acc += w[i + 16] * (v > 0.0 ? v : 0.0);
          }
          h[((int64_t)y * W + x) * 3 + k] = acc;
        }
    for (int32_t y = 0; y < H; y++) /* then along columns, added to the colour */
      for (int32_t x = 0; x < W; x++)
        for (int k = 0; k < 3; k++) {
          double acc = 0.0;
          for (int j = -R; j <= R; j++) {
            int32_t yy = y + j;
            yy = yy < 0 ? 0 : (yy >= H ? H - 1 : yy);
            acc += w[j + 16] * h[((int64_t)yy * W + x) * 3 + k];
          }
          col[((int64_t)y * W + x) * 3 + k] = (float)(c[((int64_t)y * W + x) * 3 + k] + beta * acc);
        }
    free(h);
  } else {
    for (int64_t i = 0; i < 3 * N; i++) col[i] = (float)c[i];
  }
  free(c);
  return 0;
}

/* ------------------------------------------------------------------ */
/* step 10: shading in fp32                                            */
/* ------------------------------------------------------------------ */
/* the number of lights that shine: 0 for an unknown type or a spot light without its cone table */
static int32_t light_count(const orc_batch* b, int32_t s) {
  int32_t count = b->light_meta[s * 2 + 0], type = b->light_meta[s * 2 + 1];
  int ok = type == 0 || type == 1 || (type == 2 && b->light_spot != NULL);
  return ok ? count : 0;
}

/* the spot cone factor of step 10 at cosine x, in fp32 */
static float spot_f32(float x, float cos_o, float cos_i) {
  if (!(cos_i > cos_o)) return 0.0f;
  float t = (x - cos_o) / (cos_i - cos_o);
  t = t < 0.0f ? 0.0f : (t > 1.0f ? 1.0f : t);
  return t * t * (3.0f - 2.0f * t);
}

/* ops: the fp32 operations of the call that depend on the pixel are added (each +, -, *, /, sqrt,
   powf, negation, comparison and clamp counts once); the light's move to view space (18 per light),
   the spot axis's (15) and its cone width cos_i - cos_o (1), and 2^EV (1) depend on the image only
   and are counted once per image by the caller (orc_shade_image_ops). */
static void shade_f32(const orc_batch* b, int32_t s, const float* V, int ortho, const float P[3],
                      const float n[3], int32_t mat, const float vis[ORC_MAX_LIGHTS], float rgb[3], int64_t* ops) {
  int64_t k_ops = 0;
  const float* m = b->material + ((int64_t)s * ORC_MAX_MATERIALS + mat) * 5;
  const float* amb = b->ambient + (int64_t)s * 3;
  const float e = b->emission ? b->emission[(int64_t)s * ORC_MAX_MATERIALS + mat] : 0.0f;
  int32_t count = light_count(b, s);
  int32_t type = b->light_meta[s * 2 + 1];
  float c[3] = {0.0f, 0.0f, 0.0f};
  float Vv[3];
  if (ortho) {
    Vv[0] = 0.0f;
    Vv[1] = 0.0f;
    Vv[2] = 1.0f;
  } else {
    float lp = sqrtf((P[0] * P[0] + P[1] * P[1]) + P[2] * P[2]);
    for (int k = 0; k < 3; k++) Vv[k] = -P[k] / lp;
    k_ops += 6 + 6;
  }
  for (int l = 0; l < count; l++) {
    const float* L4 = b->light + ((int64_t)s * ORC_MAX_LIGHTS + l) * 4;
    float L[3], E;
    if (type != 1) {
      float Lv[3];
      for (int i = 0; i < 3; i++) {
        float lpv = ((V[i * 4 + 0] * L4[0] + V[i * 4 + 1] * L4[1]) + V[i * 4 + 2] * L4[2]) + V[i * 4 + 3];
        Lv[i] = lpv - P[i];
      }
      float d2 = (Lv[0] * Lv[0] + Lv[1] * Lv[1]) + Lv[2] * Lv[2];
      float dl = sqrtf(d2);
      for (int i = 0; i < 3; i++) L[i] = Lv[i] / dl;
      E = L4[3] / d2;
      k_ops += 3 + 5 + 1 + 3 + 1; /* L - P, d^2, d, the unit vector, the falloff */
      if (type == 2) { /* the cone about the spot axis, taken to view space like a direction */
        const float* sp = b->light_spot + ((int64_t)s * ORC_MAX_LIGHTS + l) * 5;
        float av[3];
        for (int i = 0; i < 3; i++) av[i] = (V[i * 4 + 0] * sp[0] + V[i * 4 + 1] * sp[1]) + V[i * 4 + 2] * sp[2];
        float x = -((L[0] * av[0] + L[1] * av[1]) + L[2] * av[2]);
        E = E * spot_f32(x, sp[3], sp[4]);
        /* x (6), the cone test (1), then (x - cos_o) / width with its clamp (4) and the smoothstep
           (4) when the cone is not null, and the product (1) */
        k_ops += 6 + 1 + (sp[4] > sp[3] ? 8 : 0) + 1;
      }
    } else {
      for (int i = 0; i < 3; i++) L[i] = -((V[i * 4 + 0] * L4[0] + V[i * 4 + 1] * L4[1]) + V[i * 4 + 2] * L4[2]);
      E = L4[3];
    }
    E = E * vis[l]; /* step 16 */
    float ndl = (n[0] * L[0] + n[1] * L[1]) + n[2] * L[2];
    if (ndl < 0.0f) ndl = 0.0f;
    float spec = 0.0f;
    k_ops += 1 + 6 + 1; /* the shadow factor, n . L with its clamp, the test below */
    if (ndl > 0.0f) {
      float Hv[3] = {L[0] + Vv[0], L[1] + Vv[1], L[2] + Vv[2]};
      float h2 = (Hv[0] * Hv[0] + Hv[1] * Hv[1]) + Hv[2] * Hv[2];
      k_ops += 3 + 5 + 1; /* L + V, its squared length, the test below */
      if (h2 > 0.0f) {
        float hl = sqrtf(h2);
        float H[3] = {Hv[0] / hl, Hv[1] / hl, Hv[2] / hl};
        float ndh = (n[0] * H[0] + n[1] * H[1]) + n[2] * H[2];
        if (ndh < 0.0f) ndh = 0.0f;
        spec = m[3] * powf(ndh, m[4]);
        k_ops += 1 + 3 + 5 + 1 + 2; /* |H|, H, n . H with its clamp, the lobe */
      }
    }
    for (int k = 0; k < 3; k++) c[k] = c[k] + E * (m[k] * ndl + spec);
    k_ops += 12;
  }
  float scale = exp2f(b->exposure_ev[s]);
  for (int k = 0; k < 3; k++) rgb[k] = scale * ((amb[k] * m[k] + e * m[k]) + c[k]);
  k_ops += 15;
  *ops += k_ops;
}

/* The fp32 operations of steps 10 and 13 that depend only on the image of sample s (counted once
   per image): each light moved to view space (18), each spot axis (15) and cone width (1), 2^EV (1),
   and the grading factors when the batch is graded. */
static int64_t orc_shade_image_ops(const orc_batch* b, int32_t s) {
  int32_t count = light_count(b, s), type = b->light_meta[s * 2 + 1];
  return (int64_t)count * (18 + (type == 2 ? 16 : 0)) + 1 + (b->grading ? ORC_GRADE_IMAGE_OPS : 0);
}

/* ------------------------------------------------------------------ */
/* steps 15-16: shadows                                                */
/* ------------------------------------------------------------------ */
/* faces per light (step 15) */
static int32_t shadow_faces(const orc_batch* b) { return b->shadow_faces > 0 ? b->shadow_faces : 1; }

/* index of face f of light l of sample s in the shadow arrays */
static int64_t shadow_index(const orc_batch* b, int32_t s, int l, int f) {
  return ((int64_t)s * ORC_MAX_LIGHTS + l) * shadow_faces(b) + f;
}

/* face f of light l of sample s casts a shadow (step 15) */
static int casts_shadow(const orc_batch* b, int32_t s, int l, int f) {
  return b->shadow_view && b->shadow_intr && b->shadow_res > 0 && l < light_count(b, s) &&
         b->shadow_intr[shadow_index(b, s, l, f) * 7 + 0] != 0.0f;
}

/* M = S V^-1 for the rigid camera view V = [R | t] (step 16) */
static void camera_to_shadow(const float* S, const float* V, float M[12]) {
  float Wi[12];
  for (int i = 0; i < 3; i++) {
    for (int j = 0; j < 3; j++) Wi[i * 4 + j] = V[j * 4 + i];
    Wi[i * 4 + 3] = -((V[0 * 4 + i] * V[3] + V[1 * 4 + i] * V[7]) + V[2 * 4 + i] * V[11]);
  }
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 4; j++) {
      float r = (S[i * 4 + 0] * Wi[0 * 4 + j] + S[i * 4 + 1] * Wi[1 * 4 + j]) + S[i * 4 + 2] * Wi[2 * 4 + j];
      M[i * 4 + j] = j == 3 ? r + S[i * 4 + 3] : r;
    }
}

/* the number of shadowed taps (0..9) at camera-space point P on one face, or -1 when the face's
   map does not contain P's projection (step 16) */
static int shadow_taps(const float M[12], const float* si, const float* map, int32_t R, const float P[3],
                       int64_t* ops) {
  float q[3];
  /* each row as three fused multiply-adds (one rounding each), the translation first */
  for (int i = 0; i < 3; i++) q[i] = fmaf(M[i * 4 + 2], P[2], fmaf(M[i * 4 + 1], P[1], fmaf(M[i * 4 + 0], P[0], M[i * 4 + 3])));
  float z = -q[2];
  *ops += 18 + 1 + 1; /* the projection (nine fused multiply-adds, two operations each), z, the near test */
  if (!(z > si[4])) return -1;
  float u, v;
  if (si[6] != 0.0f) { /* orthographic */
    u = fmaf(si[0], q[0], si[2]);
    v = fmaf(-si[1], q[1], si[3]);
    *ops += 4;
  } else {
    float iw = 1.0f / z;
    u = fmaf(si[0], q[0] * iw, si[2]);
    v = fmaf(-si[1], q[1] * iw, si[3]);
    *ops += 7;
  }
  *ops += 4; /* the guard-band tests */
  if (!(fabsf(u) < GUARD_PX) || !(fabsf(v) < GUARD_PX)) return -1;
  int32_t i0 = (int32_t)floorf(u), j0 = (int32_t)floorf(v);
  *ops += 4; /* floor and conversion of u and v */
  if (i0 < 0 || j0 < 0 || i0 >= R || j0 >= R) return -1;
  float zb = z - si[5];
  *ops += 1;
  int k = 0;
  for (int bb = -1; bb <= 1; bb++)
    for (int a = -1; a <= 1; a++) {
      int32_t i = i0 + a, j = j0 + bb;
      if (i < 0 || j < 0 || i >= R || j >= R) continue;
      float d = map[(int64_t)j * R + i];
      *ops += d > 0.0f ? 2 : 1; /* the occupancy test, then the depth test */
      if (d > 0.0f && zb > d) k++;
    }
  return k;
}

/* ------------------------------------------------------------------ */
/* steps 2-8 for one view of sample s                                 */
/* ------------------------------------------------------------------ */
/* in = fx, fy, cx, cy, near; back != 0 keeps back faces (step 15) */
static void visibility(const orc_meshes* me, const orc_batch* b, int32_t s, const float* V, const float* in, int ortho,
                       int32_t W, int32_t H, int back, pixel_winner* px, int64_t cnt[4]) {
  float fx = in[0], fy = in[1], cx = in[2], cy = in[3], near = in[4];
  int64_t frags = 0, culled = 0, clipped = 0, dropped = 0;
  reset_winners(px, (int64_t)W * H);
  int64_t prim_base = 0;
  for (int32_t inst = b->inst_offset[s]; inst < b->inst_offset[s + 1]; inst++) {
    int32_t mesh = (int32_t)b->inst_mesh[inst];
    float MV[12];
    compose_mv(V, b->inst_pose + (int64_t)inst * 12, MV);
    int32_t v0 = me->vert_offset[mesh];
    int32_t t0 = me->tri_offset[mesh], t1 = me->tri_offset[mesh + 1];
    for (int32_t t = t0; t < t1; t++) {
      vtx tri[3];
      for (int k = 0; k < 3; k++) {
        int64_t vi = (int64_t)v0 + me->idx[(int64_t)t * 3 + k];
        tri[k] = to_view(MV, me->pos + vi * 3, me->nrm + vi * 3);
      }
      vtx poly[4];
      int np = clip_near(tri, near, poly);
      if (!(tri[0].p[2] <= -near && tri[1].p[2] <= -near && tri[2].p[2] <= -near)) clipped++;
      int64_t prim = prim_base + (t - t0);
      int32_t mat = (int32_t)b->inst_mat_base[inst] + me->tri_mat[t];
      int32_t seg = b->inst_seg[inst];
      for (int sub = 0; sub + 2 < np; sub++) {
        const vtx* q[3] = {&poly[0], &poly[sub + 1], &poly[sub + 2]};
        if (back) { /* reversed: the back faces pass the cull of step 5 */
          const vtx* tmp = q[1];
          q[1] = q[2];
          q[2] = tmp;
        }
        int32_t X[3], Y[3];
        float iw[3], nn[3][3];
        int bad = 0;
        for (int k = 0; k < 3; k++) {
          float xs, ys;
          if (ortho) {
            iw[k] = -q[k]->p[2];
            xs = cx + fx * q[k]->p[0];
            ys = cy - fy * q[k]->p[1];
          } else {
            iw[k] = 1.0f / (-q[k]->p[2]);
            xs = cx + fx * (q[k]->p[0] * iw[k]);
            ys = cy - fy * (q[k]->p[1] * iw[k]);
          }
          if (!(fabsf(xs) < GUARD_PX) || !(fabsf(ys) < GUARD_PX)) bad = 1;
          X[k] = bad ? 0 : (int32_t)rintf(xs * 256.0f);
          Y[k] = bad ? 0 : (int32_t)rintf(ys * 256.0f);
          for (int d = 0; d < 3; d++) nn[k][d] = q[k]->n[d];
        }
        if (bad) {
          dropped++;
          continue;
        }
        frags += raster_triangle(W, H, X, Y, iw, ortho, 2 * prim + sub, (const float(*)[3])nn, mat, seg, px,
                                 &culled);
      }
    }
    prim_base += t1 - t0;
  }
  if (cnt) {
    cnt[0] += frags;
    cnt[1] += culled;
    cnt[2] += clipped;
    cnt[3] += dropped;
  }
}

/* ------------------------------------------------------------------ */
/* one image: steps 2-11, 13, 14, 16                                   */
/* ------------------------------------------------------------------ */
static int render_image(const orc_meshes* me, const orc_batch* b, int32_t c, const orc_outputs* out,
                        pixel_winner* px) {
  int32_t W = b->cam_wh[c * 2 + 0], H = b->cam_wh[c * 2 + 1];
  int32_t s = b->cam_sample[c];
  const float* V = b->cam_view + (int64_t)c * 12;
  const float* in = b->cam_intr + (int64_t)c * 6;
  float fx = in[0], fy = in[1], cx = in[2], cy = in[3], near = in[4];
  float inv_fx = 1.0f / fx, inv_fy = 1.0f / fy;
  int ortho = in[5] != 0.0f;
  int64_t base = b->img_offset[c];

  for (int32_t inst = b->inst_offset[s]; inst < b->inst_offset[s + 1]; inst++) {
    int32_t mesh = (int32_t)b->inst_mesh[inst];
    float MV[12];
    compose_mv(V, b->inst_pose + (int64_t)inst * 12, MV);
    if (out->tracker) { /* step 14 */
      int32_t* row = out->tracker + ((int64_t)c * out->tracker_stride + (inst - b->inst_offset[s])) * 8;
      int32_t x0 = INT32_MAX, y0 = INT32_MAX, x1 = INT32_MIN, y1 = INT32_MIN, flags = 0, kx = 0, ky = 0;
      const int32_t va = me->vert_offset[mesh], vb = me->vert_offset[mesh + 1];
      unsigned char* used = (unsigned char*)calloc((size_t)(vb - va) + 1, 1);
      if (!used) return -1;
      for (int32_t t = me->tri_offset[mesh]; t < me->tri_offset[mesh + 1]; t++)
        for (int k = 0; k < 3; k++) used[me->idx[(int64_t)t * 3 + k]] = 1;
      used[vb - va] = me->tri_offset[mesh + 1] > me->tri_offset[mesh]; /* (a mesh without triangles: no row) */
      for (int32_t v = va; v <= vb; v++) {
        const float origin[3] = {0.0f, 0.0f, 0.0f}, zero[3] = {0.0f, 0.0f, 0.0f};
        const int is_origin = v == vb; /* the last pass projects the origin */
        if (!used[v - va]) continue;
        vtx q = to_view(MV, is_origin ? origin : me->pos + (int64_t)v * 3, zero);
        if (!(q.p[2] <= -near)) continue;
        float xs, ys;
        if (ortho) {
          xs = cx + fx * q.p[0];
          ys = cy - fy * q.p[1];
        } else {
          float iwv = 1.0f / (-q.p[2]);
          xs = cx + fx * (q.p[0] * iwv);
          ys = cy - fy * (q.p[1] * iwv);
        }
        if (!(fabsf(xs) < GUARD_PX) || !(fabsf(ys) < GUARD_PX)) continue;
        int32_t X = (int32_t)rintf(xs * 256.0f), Y = (int32_t)rintf(ys * 256.0f);
        if (is_origin) {
          kx = X;
          ky = Y;
          flags |= 2;
        } else {
          if (X < x0) x0 = X;
          if (Y < y0) y0 = Y;
          if (X > x1) x1 = X;
          if (Y > y1) y1 = Y;
          flags |= 1;
        }
      }
      free(used);
      row[0] = x0; row[1] = y0; row[2] = x1; row[3] = y1;
      row[4] = kx; row[5] = ky; row[6] = flags; row[7] = 0;
    }
  }
  visibility(me, b, s, V, in, ortho, W, H, 0, px, out->counters);

  /* step 16: the camera-to-shadow maps of the casting faces */
  const int32_t F = shadow_faces(b);
  float (*Msh)[12] = (float (*)[12])malloc(sizeof(float) * 12 * ORC_MAX_LIGHTS * (size_t)F);
  int* cast = (int*)malloc(sizeof(int) * ORC_MAX_LIGHTS * (size_t)F);
  if (!Msh || !cast) {
    free(Msh);
    free(cast);
    return -1;
  }
  for (int l = 0; l < ORC_MAX_LIGHTS; l++)
    for (int f = 0; f < F; f++) {
      cast[l * F + f] = casts_shadow(b, s, l, f);
      if (cast[l * F + f]) camera_to_shadow(b->shadow_view + shadow_index(b, s, l, f) * 12, V, Msh[l * F + f]);
    }

  /* steps 9-11 per pixel.  ops counts the fp32 operations of steps 9-13 and 16 (out->flops): per
     visible pixel those that depend on the pixel, as the comments beside the code tally them; per
     background pixel only the grading and quantisation of a graded background colour (an ungraded
     one is the same for the whole image); once per image the set-up of the lights, the exposure,
     the grading factors and the reciprocal focal lengths (2). */
  int64_t ops = 2 + orc_shade_image_ops(b, s);
  const float* bg = b->background + (int64_t)s * 3;
  /* step 17: with post-processing the image's linear colour, depth and normals are kept until
     every pixel is shaded, then post-processed, graded and quantised */
  const float* post = b->post ? b->post + (int64_t)s * 4 : NULL;
  float* pcol = NULL;
  float* pdep = NULL;
  uint16_t* pnrm = NULL;
  if (post) {
    const size_t np = (size_t)W * (size_t)H + 1;
    pcol = (float*)malloc(sizeof(float) * 3 * np);
    pdep = (float*)malloc(sizeof(float) * np);
    pnrm = (uint16_t*)malloc(sizeof(uint16_t) * 3 * np);
    if (!pcol || !pdep || !pnrm) {
      free(pcol);
      free(pdep);
      free(pnrm);
      free(Msh);
      free(cast);
      return -1;
    }
  }
  for (int32_t y = 0; y < H; y++) {
    for (int32_t x = 0; x < W; x++) {
      int64_t i = (int64_t)y * W + x;
      int64_t o = base + i;
      pixel_winner* p = &px[i];
      if (out->prim) out->prim[o] = p->key;
      if (out->depth2) out->depth2[o] = p->depth2;
      if (p->key < 0) {
        if (post) {
          for (int k = 0; k < 3; k++) {
            pcol[i * 3 + k] = bg[k];
            pnrm[i * 3 + k] = 0;
          }
          pdep[i] = 0.0f;
        } else if (out->rgb || out->rgb_final) {
          float gc[3] = {bg[0], bg[1], bg[2]};
          if (b->grading) grade(b->grading + (int64_t)s * 8, c - b->cam_offset[s], i, gc);
          for (int k = 0; k < 3; k++) {
            if (out->rgb) out->rgb[o * 3 + k] = quantise(gc[k]);
            if (out->rgb_final) out->rgb_final[o * 3 + k] = gc[k];
          }
        }
        if (b->grading) ops += ORC_GRADE_OPS + 3 * 6; /* the grading and the three quantisations */
        if (out->rgb_linear)
          for (int k = 0; k < 3; k++) out->rgb_linear[o * 3 + k] = bg[k];
        if (out->depth) out->depth[o] = 0.0f;
        if (out->normal)
          for (int k = 0; k < 3; k++) out->normal[o * 3 + k] = 0;
        if (out->seg) out->seg[o] = 0;
        if (out->gb_pos)
          for (int k = 0; k < 3; k++) out->gb_pos[o * 3 + k] = 0.0f;
        if (out->gb_nrm)
          for (int k = 0; k < 3; k++) out->gb_nrm[o * 3 + k] = 0.0f;
        if (out->gb_mat) out->gb_mat[o] = -1;
        continue;
      }
      int64_t cxp = 256 * (int64_t)x + 128, cyp = 256 * (int64_t)y + 128;
      int64_t w0 = edge(p->X[1], p->Y[1], p->X[2], p->Y[2], cxp, cyp);
      int64_t w1 = edge(p->X[2], p->Y[2], p->X[0], p->Y[0], cxp, cyp);
      int64_t w2 = edge(p->X[0], p->Y[0], p->X[1], p->Y[1], cxp, cyp);
      float a0 = (float)w0, a1 = (float)w1, a2 = (float)w2;
      ops += 3;
      if (!ortho) {
        a0 = a0 * p->iw[0];
        a1 = a1 * p->iw[1];
        a2 = a2 * p->iw[2];
        ops += 3;
      }
      float n[3];
      for (int k = 0; k < 3; k++) n[k] = (a0 * p->n[0][k] + a1 * p->n[1][k]) + a2 * p->n[2][k];
      float len = sqrtf((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
      ops += 15 + 6 + 1; /* the interpolated normal, its length, the test below */
      if (len > 0.0f) {
        for (int k = 0; k < 3; k++) n[k] = n[k] / len;
        ops += 3;
      }
      float ux = ((float)x + 0.5f - cx) * inv_fx;
      float uy = -(((float)y + 0.5f - cy) * inv_fy);
      float P[3];
      ops += 4 + 5;
      if (ortho) {
        P[0] = ux;
        P[1] = uy;
        P[2] = -p->depth;
        ops += 1;
      } else {
        P[0] = p->depth * ux;
        P[1] = p->depth * uy;
        P[2] = -p->depth;
        ops += 3;
      }
      float vis[ORC_MAX_LIGHTS] = {1.0f, 1.0f, 1.0f, 1.0f};
      int32_t word = p->mat;
      for (int l = 0; l < ORC_MAX_LIGHTS; l++) {
        int k = -1;
        for (int f = 0; f < F && k < 0; f++) { /* the first face whose map contains the point */
          if (!cast[l * F + f]) continue;
          const int64_t si = shadow_index(b, s, l, f);
          k = shadow_taps(Msh[l * F + f], b->shadow_intr + si * 7,
                          b->shadow_map + si * b->shadow_res * b->shadow_res, b->shadow_res, P, &ops);
        }
        if (k <= 0) continue;
        vis[l] = (float)(9 - k) / 9.0f;
        ops += 2;
        word |= k << (8 + 4 * l);
      }
      float rgb[3];
      shade_f32(b, s, V, ortho, P, n, p->mat, vis, rgb, &ops);
      if (post) {
        for (int k = 0; k < 3; k++) {
          pcol[i * 3 + k] = rgb[k];
          pnrm[i * 3 + k] = orc_f32_to_f16(n[k]);
        }
        pdep[i] = p->depth;
      } else if (out->rgb || out->rgb_final) {
        float gc[3] = {rgb[0], rgb[1], rgb[2]};
        if (b->grading) grade(b->grading + (int64_t)s * 8, c - b->cam_offset[s], i, gc);
        for (int k = 0; k < 3; k++) {
          if (out->rgb) out->rgb[o * 3 + k] = quantise(gc[k]);
          if (out->rgb_final) out->rgb_final[o * 3 + k] = gc[k];
        }
      }
      /* the grading, three quantisations (clamp 2, scale, offset, floor, conversion) and three
         binary16 conversions of the normal */
      ops += (b->grading ? ORC_GRADE_OPS : 0) + 3 * 6 + 3;
      if (out->rgb_linear)
        for (int k = 0; k < 3; k++) out->rgb_linear[o * 3 + k] = rgb[k];
      if (out->depth) out->depth[o] = p->depth;
      if (out->normal)
        for (int k = 0; k < 3; k++) out->normal[o * 3 + k] = orc_f32_to_f16(n[k]);
      if (out->seg) out->seg[o] = (uint8_t)p->seg;
      if (out->gb_pos)
        for (int k = 0; k < 3; k++) out->gb_pos[o * 3 + k] = P[k];
      if (out->gb_nrm)
        for (int k = 0; k < 3; k++) out->gb_nrm[o * 3 + k] = n[k];
      if (out->gb_mat) out->gb_mat[o] = word;
    }
  }
  int rc = 0;
  if (post) {
    rc = orc_post_image(W, H, in, post, pcol, pdep, pnrm);
    for (int64_t i = 0; rc == 0 && i < (int64_t)W * H; i++) {
      float gc[3] = {pcol[i * 3 + 0], pcol[i * 3 + 1], pcol[i * 3 + 2]};
      if (b->grading) grade(b->grading + (int64_t)s * 8, c - b->cam_offset[s], i, gc);
      for (int k = 0; k < 3; k++) {
        if (out->rgb) out->rgb[(base + i) * 3 + k] = quantise(gc[k]);
        if (out->rgb_final) out->rgb_final[(base + i) * 3 + k] = gc[k];
      }
    }
    free(pcol);
    free(pdep);
    free(pnrm);
  }
  free(Msh);
  free(cast);
  if (out->flops) out->flops[0] += ops;
  return rc;
}

int orc_render_shadow_maps(const orc_meshes* m, const orc_batch* b, int32_t s_begin, int32_t s_end, float* maps) {
  const int32_t R = b->shadow_res;
  if (R <= 0 || !b->shadow_view || !b->shadow_intr) return 0;
  pixel_winner* px = (pixel_winner*)malloc(sizeof(pixel_winner) * (size_t)R * (size_t)R);
  if (!px) return -1;
  for (int32_t s = s_begin; s < s_end; s++)
    for (int l = 0; l < ORC_MAX_LIGHTS; l++)
      for (int f = 0; f < shadow_faces(b); f++) {
        if (!casts_shadow(b, s, l, f)) continue;
        const int64_t si = shadow_index(b, s, l, f);
        const float* in = b->shadow_intr + si * 7;
        visibility(m, b, s, b->shadow_view + si * 12, in, in[6] != 0.0f, R, R, 1, px, NULL);
        float* map = maps + si * R * R;
        for (int64_t i = 0; i < (int64_t)R * R; i++) map[i] = px[i].key < 0 ? 0.0f : px[i].depth;
      }
  free(px);
  return 0;
}

int orc_render(const orc_meshes* m, const orc_batch* b, int32_t cam_begin, int32_t cam_end,
               const orc_outputs* out) {
  int64_t maxpx = 0;
  for (int32_t c = cam_begin; c < cam_end; c++) {
    int64_t n = (int64_t)b->cam_wh[c * 2] * b->cam_wh[c * 2 + 1];
    if (n > maxpx) maxpx = n;
  }
  pixel_winner* px = (pixel_winner*)malloc((size_t)(maxpx > 0 ? maxpx : 1) * sizeof(pixel_winner));
  if (!px) return -1;
  int rc = 0;
  for (int32_t c = cam_begin; c < cam_end && rc == 0; c++) rc = render_image(m, b, c, out, px);
  free(px);
  return rc;
}

int orc_raster_fixed(int32_t W, int32_t H, int32_t n, const int32_t* X, const int32_t* Y, const float* iw,
                     int32_t ortho, int64_t* prim_out, float* depth_out, int32_t* count_out) {
  pixel_winner* px = (pixel_winner*)malloc((size_t)((int64_t)W * H > 0 ? (int64_t)W * H : 1) * sizeof(pixel_winner));
  if (!px) return -1;
  reset_winners(px, (int64_t)W * H);
  for (int32_t t = 0; t < n; t++)
    raster_triangle(W, H, X + 3 * t, Y + 3 * t, iw + 3 * t, ortho, 2 * (int64_t)t, NULL, 0, 0, px, NULL);
  for (int64_t i = 0; i < (int64_t)W * H; i++) {
    if (prim_out) prim_out[i] = px[i].key;
    if (depth_out) depth_out[i] = px[i].key < 0 ? 0.0f : px[i].depth;
    if (count_out) count_out[i] = px[i].count;
  }
  free(px);
  return 0;
}

/* ------------------------------------------------------------------ */
/* step 10 in fp64 (finite differences) and its adjoint (step 12)      */
/* ------------------------------------------------------------------ */
typedef struct {
  double L[3], E, ndl, spec, ndh, pw; /* pw = ndh^alpha */
  double H[3], hl, Lv[3], dl, d2;
  double S, dS; /* spot cone factor and its derivative in the cosine x (1 and 0 for other lights) */
  double vis;   /* shadow factor (9 - k) / 9 of step 16, held fixed */
  int lit, has_h;
} light_term;

/* view-space light positions (or directions to the light) and, for spot lights, view-space axes
   with the cone cosines: spot[l] = (axis xyz, cos_o, cos_i) */
static void view_lights_f64(const orc_batch* b, int32_t s, const float* V, const double* light,
                            double out[ORC_MAX_LIGHTS][3], double spot[ORC_MAX_LIGHTS][5]) {
  int32_t count = light_count(b, s), type = b->light_meta[s * 2 + 1];
  for (int l = 0; l < count; l++) {
    const double* L4 = light + ((int64_t)s * ORC_MAX_LIGHTS + l) * 4;
    for (int i = 0; i < 3; i++) {
      double r = (double)V[i * 4 + 0] * L4[0] + (double)V[i * 4 + 1] * L4[1] + (double)V[i * 4 + 2] * L4[2];
      out[l][i] = type == 1 ? -r : r + (double)V[i * 4 + 3];
    }
    if (type == 2) {
      const float* sp = b->light_spot + ((int64_t)s * ORC_MAX_LIGHTS + l) * 5;
      for (int i = 0; i < 3; i++)
        spot[l][i] = (double)V[i * 4 + 0] * sp[0] + (double)V[i * 4 + 1] * sp[1] + (double)V[i * 4 + 2] * sp[2];
      spot[l][3] = sp[3];
      spot[l][4] = sp[4];
    }
  }
}

/* spot: NULL, or (view-space axis, cos_o, cos_i) of a spot light; vis: the shadow factor */
static void light_eval(int type, const double Lp[3], double I, const double P[3], const double n[3],
                       const double Vv[3], double alpha, const double* spot, double vis, light_term* t) {
  memset(t, 0, sizeof(*t));
  t->S = 1.0;
  t->vis = vis;
  if (type != 1) {
    for (int i = 0; i < 3; i++) t->Lv[i] = Lp[i] - P[i];
    t->d2 = t->Lv[0] * t->Lv[0] + t->Lv[1] * t->Lv[1] + t->Lv[2] * t->Lv[2];
    t->dl = sqrt(t->d2);
    for (int i = 0; i < 3; i++) t->L[i] = t->Lv[i] / t->dl;
    if (spot) {
      const double x = -(t->L[0] * spot[0] + t->L[1] * spot[1] + t->L[2] * spot[2]);
      const double w = spot[4] - spot[3];
      t->S = 0.0;
      if (w > 0.0) {
        double u = (x - spot[3]) / w;
        if (u >= 1.0) {
          t->S = 1.0;
        } else if (u > 0.0) {
          t->S = u * u * (3.0 - 2.0 * u);
          t->dS = 6.0 * u * (1.0 - u) / w;
        }
      }
    }
    t->E = I * t->S * vis / t->d2;
  } else {
    for (int i = 0; i < 3; i++) t->L[i] = Lp[i];
    t->E = I * vis;
  }
  double ndl = n[0] * t->L[0] + n[1] * t->L[1] + n[2] * t->L[2];
  t->lit = ndl > 0.0;
  t->ndl = t->lit ? ndl : 0.0;
  if (t->lit) {
    double Hv[3] = {t->L[0] + Vv[0], t->L[1] + Vv[1], t->L[2] + Vv[2]};
    double h2 = Hv[0] * Hv[0] + Hv[1] * Hv[1] + Hv[2] * Hv[2];
    if (h2 > 0.0) {
      t->has_h = 1;
      t->hl = sqrt(h2);
      for (int i = 0; i < 3; i++) t->H[i] = Hv[i] / t->hl;
      double ndh = n[0] * t->H[0] + n[1] * t->H[1] + n[2] * t->H[2];
      t->ndh = ndh > 0.0 ? ndh : 0.0;
      t->pw = pow(t->ndh, alpha);
    }
  }
}

static void pixel_setup_f64(const float* gp, const float* gn, int ortho, double P[3], double n[3], double Vv[3]) {
  for (int k = 0; k < 3; k++) {
    P[k] = gp[k];
    n[k] = gn[k];
  }
  if (ortho) {
    Vv[0] = 0.0;
    Vv[1] = 0.0;
    Vv[2] = 1.0;
  } else {
    double lp = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
    for (int k = 0; k < 3; k++) Vv[k] = -P[k] / lp;
  }
}

void orc_shade_f64(const orc_batch* b, int32_t cam_begin, int32_t cam_end, const float* gb_pos,
                   const float* gb_nrm, const int32_t* gb_mat, const double* material, const double* light,
                   const double* exposure_ev, const double* ambient, const double* emission, double* rgb) {
  for (int32_t c = cam_begin; c < cam_end; c++) {
    int32_t s = b->cam_sample[c];
    const float* V = b->cam_view + (int64_t)c * 12;
    int ortho = b->cam_intr[c * 6 + 5] != 0.0f;
    int64_t npx = (int64_t)b->cam_wh[c * 2] * b->cam_wh[c * 2 + 1];
    int64_t base = b->img_offset[c];
    double Lp[ORC_MAX_LIGHTS][3], sp[ORC_MAX_LIGHTS][5];
    view_lights_f64(b, s, V, light, Lp, sp);
    int32_t count = light_count(b, s), type = b->light_meta[s * 2 + 1];
    double scale = exp2(exposure_ev[s]);
    for (int64_t i = 0; i < npx; i++) {
      int64_t o = base + i;
      int32_t word = gb_mat[o], mat = word & 0xff;
      if (word < 0) {
        for (int k = 0; k < 3; k++) rgb[o * 3 + k] = b->background[s * 3 + k];
        continue;
      }
      const double* m = material + ((int64_t)s * ORC_MAX_MATERIALS + mat) * 5;
      double P[3], n[3], Vv[3];
      pixel_setup_f64(gb_pos + o * 3, gb_nrm + o * 3, ortho, P, n, Vv);
      double acc[3] = {0, 0, 0};
      for (int l = 0; l < count; l++) {
        light_term t;
        light_eval(type, Lp[l], light[((int64_t)s * ORC_MAX_LIGHTS + l) * 4 + 3], P, n, Vv, m[4],
                   type == 2 ? sp[l] : NULL, (9 - ((word >> (8 + 4 * l)) & 15)) / 9.0, &t);
        double spec = m[3] * t.pw;
        for (int k = 0; k < 3; k++) acc[k] += t.E * (m[k] * t.ndl + spec);
      }
      const double e = emission ? emission[(int64_t)s * ORC_MAX_MATERIALS + mat] : 0.0;
      for (int k = 0; k < 3; k++) rgb[o * 3 + k] = scale * ((ambient[s * 3 + k] + e) * m[k] + acc[k]);
    }
  }
}

void orc_shade_backward_f64(const orc_batch* b, int32_t cam_begin, int32_t cam_end, const float* gb_pos,
                            const float* gb_nrm, const int32_t* gb_mat, const double* material,
                            const double* light, const double* exposure_ev, const double* ambient,
                            const double* emission, const double* d_rgb, double* d_material, double* d_light,
                            double* d_ev, double* d_emission) {
  const double ln2 = 0.69314718055994530942;
  for (int32_t c = cam_begin; c < cam_end; c++) {
    int32_t s = b->cam_sample[c];
    const float* V = b->cam_view + (int64_t)c * 12;
    int ortho = b->cam_intr[c * 6 + 5] != 0.0f;
    int64_t npx = (int64_t)b->cam_wh[c * 2] * b->cam_wh[c * 2 + 1];
    int64_t base = b->img_offset[c];
    double Lp[ORC_MAX_LIGHTS][3], sp[ORC_MAX_LIGHTS][5];
    view_lights_f64(b, s, V, light, Lp, sp);
    int32_t count = light_count(b, s), type = b->light_meta[s * 2 + 1];
    double scale = exp2(exposure_ev[s]);
    double dLp_view[ORC_MAX_LIGHTS][3];
    memset(dLp_view, 0, sizeof(dLp_view));
    for (int64_t i = 0; i < npx; i++) {
      int64_t o = base + i;
      int32_t word = gb_mat[o], mat = word & 0xff;
      if (word < 0) continue;
      const double* m = material + ((int64_t)s * ORC_MAX_MATERIALS + mat) * 5;
      const double* g = d_rgb + o * 3;
      double P[3], n[3], Vv[3];
      pixel_setup_f64(gb_pos + o * 3, gb_nrm + o * 3, ortho, P, n, Vv);
      double G = g[0] + g[1] + g[2];
      double gr = g[0] * m[0] + g[1] * m[1] + g[2] * m[2];
      double sum_endl = 0.0, sum_epw = 0.0, acc[3] = {0, 0, 0};
      for (int l = 0; l < count; l++) {
        light_term t;
        double I = light[((int64_t)s * ORC_MAX_LIGHTS + l) * 4 + 3];
        light_eval(type, Lp[l], I, P, n, Vv, m[4], type == 2 ? sp[l] : NULL, (9 - ((word >> (8 + 4 * l)) & 15)) / 9.0,
                   &t);
        double spec = m[3] * t.pw;
        for (int k = 0; k < 3; k++) acc[k] += t.E * (m[k] * t.ndl + spec);
        sum_endl += t.E * t.ndl;
        sum_epw += t.E * t.pw;
        /* rgb_k = scale*((amb_k + e)*rho_k + sum_l E_l*(rho_k*ndl_l + ks*ndh_l^alpha)),
           E_l = I_l S_l / d2_l (S_l = 1 but for spot lights) or I_l (directional) */
        double dE = scale * (gr * t.ndl + G * spec);
        double dndl = t.lit ? scale * t.E * gr : 0.0;
        double dndh = (t.has_h && t.ndh > 0.0) ? scale * t.E * G * m[3] * m[4] * pow(t.ndh, m[4] - 1.0) : 0.0;
        double dLvec[3];
        for (int k = 0; k < 3; k++) dLvec[k] = dndl * n[k];
        if (dndh != 0.0) {
          double dH[3] = {dndh * n[0], dndh * n[1], dndh * n[2]};
          double hd = t.H[0] * dH[0] + t.H[1] * dH[1] + t.H[2] * dH[2];
          for (int k = 0; k < 3; k++) dLvec[k] += (dH[k] - t.H[k] * hd) / t.hl;
        }
        double* dl = d_light + ((int64_t)s * ORC_MAX_LIGHTS + l) * 4;
        if (type != 1) {
          dl[3] += dE * t.S * t.vis / t.d2;
          double dd2 = -dE * I * t.S * t.vis / (t.d2 * t.d2);
          if (type == 2) /* x = -(L . axis): dE/dL = I vis/d2 * S'(x) * (-axis) */
            for (int k = 0; k < 3; k++) dLvec[k] -= dE * I * t.vis / t.d2 * t.dS * sp[l][k];
          double ld = t.L[0] * dLvec[0] + t.L[1] * dLvec[1] + t.L[2] * dLvec[2];
          for (int k = 0; k < 3; k++) dLp_view[l][k] += (dLvec[k] - t.L[k] * ld) / t.dl + 2.0 * dd2 * t.Lv[k];
        } else {
          dl[3] += dE * t.vis;
          for (int k = 0; k < 3; k++) dLp_view[l][k] += dLvec[k];
        }
      }
      const double e = emission ? emission[(int64_t)s * ORC_MAX_MATERIALS + mat] : 0.0;
      double* dm = d_material + ((int64_t)s * ORC_MAX_MATERIALS + mat) * 4;
      for (int k = 0; k < 3; k++) dm[k] += g[k] * scale * (ambient[s * 3 + k] + e + sum_endl);
      dm[3] += scale * G * sum_epw;
      if (d_emission) d_emission[(int64_t)s * ORC_MAX_MATERIALS + mat] += scale * gr;
      double dev = 0.0;
      for (int k = 0; k < 3; k++) dev += g[k] * scale * ((ambient[s * 3 + k] + e) * m[k] + acc[k]);
      d_ev[s] += ln2 * dev;
    }
    /* view-space light gradient back to world: point or spot p_v = R p + t, direction L = -R d */
    for (int l = 0; l < count; l++) {
      double* dl = d_light + ((int64_t)s * ORC_MAX_LIGHTS + l) * 4;
      for (int j = 0; j < 3; j++) {
        double r = 0.0;
        for (int i = 0; i < 3; i++) r += (double)V[i * 4 + j] * dLp_view[l][i];
        dl[j] += type == 1 ? -r : r;
      }
    }
  }
}

/* ------------------------------------------------------------------ */
/* step 13 in fp64 and its adjoint (a loss on the graded colour)       */
/* ------------------------------------------------------------------ */
/* The graded colour of every pixel of images [cam_begin, cam_end) from its linear colour rgb_in
   (the shading, or the background), the steps of grade() in fp64 and the same order, with the
   grading parameters taken from `grading` ([S][8], fp64 so that differences can perturb them). */
void orc_grade_f64(const orc_batch* b, int32_t cam_begin, int32_t cam_end, const double* grading,
                   const double* rgb_in, double* rgb_out) {
  const double k = 0.57735026918962576;
  const double Yw[3] = {0.2126, 0.7152, 0.0722};
  for (int32_t c = cam_begin; c < cam_end; c++) {
    const int32_t s = b->cam_sample[c];
    const double* g = grading + (int64_t)s * 8;
    const int64_t npx = (int64_t)b->cam_wh[c * 2] * b->cam_wh[c * 2 + 1], base = b->img_offset[c];
    const uint32_t h1 = pcg_hash((uint32_t)b->grading[(int64_t)s * 8 + 7] + 0x9E3779B9u * (uint32_t)(c - b->cam_offset[s] + 1));
    const double ch = cos(g[0]), sh = sin(g[0]);
    for (int64_t i = 0; i < npx; i++) {
      const double* in = rgb_in + (base + i) * 3;
      double* out = rgb_out + (base + i) * 3;
      const double r = in[0] * (1.0 + g[4]), gr = in[1] * (1.0 + g[5]), bl = in[2] * (1.0 - g[4]);
      const double mean = (r + gr + bl) / 3.0;
      const double x[3] = {(bl - gr) * k, (r - bl) * k, (gr - r) * k};
      const double c1[3] = {r, gr, bl};
      double h[3];
      for (int j = 0; j < 3; j++) h[j] = c1[j] * ch + x[j] * sh + mean * (1.0 - ch);
      const double Y = Yw[0] * h[0] + Yw[1] * h[1] + Yw[2] * h[2];
      const double n = (double)pcg_hash(h1 ^ (uint32_t)i) * 2.3283064365386963e-10;
      for (int j = 0; j < 3; j++) {
        double v = Y + g[1] * (h[j] - Y);
        v = (v - 0.5) * g[2] + 0.5;
        v = v + g[3];
        out[j] = v + g[6] * (n - 0.5);
      }
    }
  }
}

/* The adjoint of orc_grade_f64: given d_out = dL/d graded colour, the gradient dL/d rgb_in
   (written) and dL/d grading parameters (accumulated into d_grading [S][8]: hue, saturation,
   contrast, brightness, temperature, tint, grain amplitude; the seed gets none), each step of the
   grading taken back in reverse order. */
void orc_grade_backward_f64(const orc_batch* b, int32_t cam_begin, int32_t cam_end, const double* grading,
                            const double* rgb_in, const double* d_out, double* d_in, double* d_grading) {
  const double k = 0.57735026918962576;
  const double Yw[3] = {0.2126, 0.7152, 0.0722};
  for (int32_t c = cam_begin; c < cam_end; c++) {
    const int32_t s = b->cam_sample[c];
    const double* g = grading + (int64_t)s * 8;
    double* dg = d_grading + (int64_t)s * 8;
    const int64_t npx = (int64_t)b->cam_wh[c * 2] * b->cam_wh[c * 2 + 1], base = b->img_offset[c];
    const uint32_t h1 = pcg_hash((uint32_t)b->grading[(int64_t)s * 8 + 7] + 0x9E3779B9u * (uint32_t)(c - b->cam_offset[s] + 1));
    const double ch = cos(g[0]), sh = sin(g[0]);
    for (int64_t i = 0; i < npx; i++) {
      const double* in = rgb_in + (base + i) * 3;
      const double* dO = d_out + (base + i) * 3;
      /* the forward values the adjoint needs */
      const double r = in[0] * (1.0 + g[4]), gr = in[1] * (1.0 + g[5]), bl = in[2] * (1.0 - g[4]);
      const double mean = (r + gr + bl) / 3.0;
      const double x[3] = {(bl - gr) * k, (r - bl) * k, (gr - r) * k};
      const double c1[3] = {r, gr, bl};
      double h[3], v1[3];
      for (int j = 0; j < 3; j++) h[j] = c1[j] * ch + x[j] * sh + mean * (1.0 - ch);
      const double Y = Yw[0] * h[0] + Yw[1] * h[1] + Yw[2] * h[2];
      for (int j = 0; j < 3; j++) v1[j] = Y + g[1] * (h[j] - Y);
      const double n = (double)pcg_hash(h1 ^ (uint32_t)i) * 2.3283064365386963e-10;
      /* grain, brightness, contrast */
      double dv1[3], dh[3] = {0.0, 0.0, 0.0}, dY = 0.0;
      for (int j = 0; j < 3; j++) {
        dg[6] += dO[j] * (n - 0.5);
        dg[3] += dO[j];
        dg[2] += dO[j] * (v1[j] - 0.5);
        dv1[j] = dO[j] * g[2];
      }
      /* saturation v1 = Y + s (h - Y) */
      for (int j = 0; j < 3; j++) {
        dg[1] += dv1[j] * (h[j] - Y);
        dh[j] += dv1[j] * g[1];
        dY += dv1[j] * (1.0 - g[1]);
      }
      for (int j = 0; j < 3; j++) dh[j] += Yw[j] * dY;
      /* rotation h = c1 cos + x sin + mean (1 - cos) */
      double dc1[3], dx[3], dmean = 0.0, dch = 0.0, dsh = 0.0;
      for (int j = 0; j < 3; j++) {
        dch += dh[j] * (c1[j] - mean);
        dsh += dh[j] * x[j];
        dc1[j] = dh[j] * ch;
        dx[j] = dh[j] * sh;
        dmean += dh[j] * (1.0 - ch);
      }
      dg[0] += -sh * dch + ch * dsh;
      /* x = (bl - gr, r - bl, gr - r) k and mean = (r + gr + bl) / 3 */
      const double dr = dc1[0] + k * (dx[1] - dx[2]) + dmean / 3.0;
      const double dgr = dc1[1] + k * (dx[2] - dx[0]) + dmean / 3.0;
      const double dbl = dc1[2] + k * (dx[0] - dx[1]) + dmean / 3.0;
      /* white balance r = c0 (1 + t), gr = c1 (1 + u), bl = c2 (1 - t) */
      dg[4] += dr * in[0] - dbl * in[2];
      dg[5] += dgr * in[1];
      double* dI = d_in + (base + i) * 3;
      dI[0] = dr * (1.0 + g[4]);
      dI[1] = dgr * (1.0 + g[5]);
      dI[2] = dbl * (1.0 - g[4]);
    }
  }
}
