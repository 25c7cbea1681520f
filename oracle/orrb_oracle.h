/*
 * orrb_oracle.h -- plain, slow CPU oracle of the batched renderer.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only code that may load this.  It shares no code,
 * header, table or constant with the CUDA path; it is written from the
 * definition of the rendered channels (Sec. 4.4: RGB, segmentation, depth,
 * screen-space normal) and the randomized material / light / exposure
 * parameters (Sec. 4.3.1), with every numeric rule the paper leaves open
 * fixed by one stated reading (z-buffered rasterisation with one sample at
 * each pixel centre, 8 fractional bits, top-left fill rule, Blinn-Phong).
 *
 * Precision: the forward pass is fp32 with every + and x separately rounded
 * (build with -ffp-contract=off, no -ffast-math), IEEE division and sqrtf.
 * The shading used for finite differences and the shading adjoint are fp64.
 *
 * Layouts (all flat, row-major):
 *   pos/nrm        [V_total][3]   object space, per mesh at vert_offset[m]
 *   idx            [T_total][3]   mesh-local vertex indices, at tri_offset[m]
 *   inst_pose      [I][3][4]      world-from-object
 *   cam_view       [C][3][4]      camera-from-world, camera looks down -z, +y up
 *   cam_intr       [C][6]         fx, fy, cx, cy, near, type (0 persp, 1 ortho)
 *   light          [S][4][4]      xyz (point or spot position, or direction), intensity
 *   light_spot     [S][4][5]      spot axis xyz (unit, world), cos outer, cos inner
 *   material       [S][32][5]     albedo rgb, specular k_s, shininess alpha
 *   emission       [S][32]        emission e (emitted colour e * albedo)
 *   post           [S][4]         step 17: AO intensity, bloom intensity, bloom radius (px), 0
 *   outputs        flat over pixels; image c starts at pixel img_offset[c]
 */
#ifndef ORRB_ORACLE_H
#define ORRB_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_LIGHTS 4
#define ORC_MAX_MATERIALS 32

typedef struct {
  int32_t n_meshes;
  const int32_t* vert_offset;  /* [n_meshes + 1] */
  const int32_t* tri_offset;   /* [n_meshes + 1] */
  const float* pos;
  const float* nrm;
  const uint32_t* idx;
  const uint8_t* tri_mat;
} orc_meshes;

typedef struct {
  int32_t n_samples;
  const int32_t* inst_offset;   /* [S + 1] */
  const uint32_t* inst_mesh;    /* [I] */
  const float* inst_pose;       /* [I][3][4] */
  const uint8_t* inst_seg;      /* [I] */
  const int16_t* inst_mat_base; /* [I] */
  const int32_t* cam_offset;    /* [S + 1] */
  const int32_t* cam_sample;    /* [C] */
  const float* cam_view;        /* [C][3][4] */
  const float* cam_intr;        /* [C][6] */
  const int32_t* cam_wh;        /* [C][2] */
  const int64_t* img_offset;    /* [C] */
  const float* light;           /* [S][4][4] */
  const int32_t* light_meta;    /* [S][2] count, type (0 point, 1 directional, 2 spot) */
  const float* material;        /* [S][32][5] */
  const float* exposure_ev;     /* [S] */
  const float* ambient;         /* [S][3] */
  const float* background;      /* [S][3] */
  const float* grading;         /* [S][8] colour-grading epilogue (step 13), or NULL */
  const float* light_spot;      /* [S][4][5] spot cones (step 10), or NULL */
  const float* emission;        /* [S][32] material emission (step 10), or NULL for none */
  const float* shadow_view;     /* [S][4][F][3][4] shadow cameras of each light (step 15), or NULL */
  const float* shadow_intr;     /* [S][4][F][7] fx, fy, cx, cy, near, bias, type (0 persp, 1 ortho);
                                   fx == 0: no shadow */
  const float* shadow_map;      /* [S][4][F][R][R] maps of step 15, read by step 16 (or NULL) */
  int32_t shadow_res;           /* R, 0 for no shadows */
  int32_t shadow_faces;         /* F, shadow cameras per light (1 spot, 6 cube); 0 is read as 1 */
  const float* post;            /* [S][4] post-processing of step 17, or NULL for none */
} orc_batch;

typedef struct {                /* every pointer may be NULL */
  uint8_t* rgb;                 /* [N][3] */
  float* depth;                 /* [N] view-axis distance, 0 = background */
  uint16_t* normal;             /* [N][3] IEEE binary16 bits */
  uint8_t* seg;                 /* [N] */
  float* rgb_linear;            /* [N][3] before clamping and quantisation */
  float* gb_pos;                /* [N][3] view-space position */
  float* gb_nrm;                /* [N][3] unit view-space normal, fp32 */
  int32_t* gb_mat;              /* [N] material slot | shadowed taps of light l << (8 + 4l); -1 = background */
  int64_t* prim;                /* [N] winning key 2*prim_id + sub, -1 = background */
  float* depth2;                /* [N] depth of the nearest fragment of another key, +inf if none */
  int64_t* counters;            /* [4] fragments, triangles culled, clipped, dropped (accumulated) */
  int32_t* tracker;             /* [C][tracker_stride][8] per (camera, instance of its sample), step 14 */
  int32_t tracker_stride;
  int64_t* flops;               /* [1] fp32 operations of steps 9-13 and 16 (accumulated; see render_image) */
  float* rgb_final;             /* [N][3] the colour step 11 quantises: after steps 17 and 13 */
} orc_outputs;

/* Render images [cam_begin, cam_end).  Returns 0, or -1 on allocation failure. */
int orc_render(const orc_meshes* m, const orc_batch* b, int32_t cam_begin, int32_t cam_end,
               const orc_outputs* out);

/* Step 15: the shadow maps [S][4][F][R][R] of samples [s_begin, s_end) (maps of faces that cast
 * no shadow are left as they were).  Returns 0, or -1 on allocation failure. */
int orc_render_shadow_maps(const orc_meshes* m, const orc_batch* b, int32_t s_begin, int32_t s_end, float* maps);

/* Rasterise already-snapped screen triangles (8 fractional bits) into one
 * W x H image: coverage, depth and the (depth, key) visibility test only.
 * X, Y: [n][3] fixed-point; iw: [n][3] 1/w (perspective) or view depth
 * (ortho != 0).  prim_out [W*H] (-1 background), depth_out [W*H] (0 background),
 * count_out [W*H] number of fragments that covered each pixel; any may be NULL. */
int orc_raster_fixed(int32_t W, int32_t H, int32_t n, const int32_t* X, const int32_t* Y,
                     const float* iw, int32_t ortho, int64_t* prim_out, float* depth_out,
                     int32_t* count_out);

/* Step 17 on one W x H image (the post-processing randomizer's ambient occlusion and bloom,
 * Sec. 4.3.1): col [W*H][3] the linear colour, replaced by the post-processed colour; depth [W*H]
 * the depth channel (0: no surface); normal [W*H][3] the normal channel's binary16 bits; in the
 * camera's fx, fy, cx, cy, near, type; q the sample's AO intensity, bloom intensity, bloom radius
 * (px) and a 0.  Returns 0, or -1 on allocation failure. */
int orc_post_image(int32_t W, int32_t H, const float* in, const float* q, float* col, const float* depth,
                   const uint16_t* normal);
/* float -> binary16 bits, round to nearest even (the normal channel's encoding). */
uint16_t orc_f32_to_f16(float f);

/* fp64 shading of a G-buffer over images [cam_begin, cam_end), parameters in
 * fp64: material [S][32][5], light [S][4][4], exposure_ev [S], ambient [S][3],
 * emission [S][32] (or NULL); spot cones come from b.  gb_mat holds the
 * G-buffer's material words: the slot in bits 0-7 and light l's shadowed
 * taps (step 16) in bits 8 + 4l .. 11 + 4l, applied as the factor (9 - k) / 9.
 * Writes rgb [N][3] (background pixels get the background colour). */
void orc_shade_f64(const orc_batch* b, int32_t cam_begin, int32_t cam_end,
                   const float* gb_pos, const float* gb_nrm, const int32_t* gb_mat,
                   const double* material, const double* light, const double* exposure_ev,
                   const double* ambient, const double* emission, double* rgb);

/* fp64 adjoint of orc_shade_f64 at fixed visibility.  d_rgb [N][3] is dL/d rgb_linear.
 * Accumulates (+=) into d_material [S][32][4] (albedo rgb, specular),
 * d_light [S][4][4] (world position or direction xyz, intensity), d_ev [S] and,
 * unless NULL, d_emission [S][32].  The spot axis and cone are not differentiated. */
void orc_shade_backward_f64(const orc_batch* b, int32_t cam_begin, int32_t cam_end,
                            const float* gb_pos, const float* gb_nrm, const int32_t* gb_mat,
                            const double* material, const double* light, const double* exposure_ev,
                            const double* ambient, const double* emission, const double* d_rgb,
                            double* d_material, double* d_light, double* d_ev, double* d_emission);

/* Step 13 (colour grading) in fp64 on a linear colour rgb_in [N][3] (shading or background),
 * with the grading parameters `grading` [S][8]: writes the graded colour rgb_out [N][3] (the
 * grain's seed is taken from the batch). */
void orc_grade_f64(const orc_batch* b, int32_t cam_begin, int32_t cam_end, const double* grading,
                   const double* rgb_in, double* rgb_out);

/* Adjoint of orc_grade_f64: d_out = dL/d graded colour [N][3]; writes d_in = dL/d rgb_in [N][3]
 * and accumulates (+=) d_grading [S][8] (hue, saturation, contrast, brightness, temperature,
 * tint, grain amplitude; 0 for the seed). */
void orc_grade_backward_f64(const orc_batch* b, int32_t cam_begin, int32_t cam_end, const double* grading,
                            const double* rgb_in, const double* d_out, double* d_in, double* d_grading);

#ifdef __cplusplus
}
#endif
#endif
