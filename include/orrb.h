/*
 * orrb.h -- C-ABI of liborrb.so, a batched renderer for visually randomized
 * robotics scenes on one B300 GPU (sm_103a).
 *
 * What it computes.  For every camera of every sample in a batch it renders
 * the four channels the paper's capture pipeline produces (Sec. 4.4: RGB,
 * segmentation, depth and screen-space normal) from geometry that is shared
 * by all samples (Single Scene Multiple States, Sec. 3) and from per-sample
 * state and randomization parameters (Sec. 4.3.1: joint positions -> link
 * poses, camera pose, light positions and intensities, material tint /
 * specular / glossiness, exposure).  Randomization itself happens on the
 * host: the library renders the parameters it is given, so a sample renders
 * identically alone or in any batch (seeded determinism, Sec. 4.3).  Outputs
 * go to caller-preallocated batch buffers (Sec. 4.4: destination textures
 * for the whole batch are preallocated).
 *
 * The numeric rules the paper leaves open are fixed as follows (the CPU
 * oracle under oracle/ implements the same definition independently):
 *   - camera looks down -z, +y up; screen x right, y down; pixel centres at
 *     (x + 1/2, y + 1/2); triangles clipped at z = -near; vertices snapped to
 *     8 fractional bits (round-half-even); integer edge functions, top-left
 *     fill rule; triangles with non-positive screen area are culled;
 *   - depth = view-axis distance (metres), 0 for background; the nearest
 *     fragment wins by (depth, 2*prim + sub) where prim is the triangle's
 *     index in the sample's concatenated triangle list (instances in order,
 *     triangles in mesh order) and sub the half of a near-clipped quad;
 *   - normal = perspective-correct interpolated view-space unit normal,
 *     stored as IEEE binary16; seg = the instance's id, 0 for background;
 *   - rgb = 2^EV * ((ambient + e)*albedo + sum_l E_l (albedo*max(0,n.L) +
 *     k_s*max(0,n.H)^alpha [n.L > 0])), e the material's emission, E = I/d^2
 *     for point lights, I for directional ones and I S/d^2 for spot lights,
 *     S = t^2 (3 - 2t), t = clamp((x - cos_o)/(cos_i - cos_o), 0, 1), x the
 *     cosine between the spot axis and the direction from the light;
 *     quantised as floor(clamp(rgb,0,1)*255 + 1/2).
 *
 * Conventions of every entry point.
 *   Memory:    every device buffer is allocated and owned by the caller; the
 *              library owns only host metadata (the context).  Pointers
 *              marked "device" must be device memory of the context's GPU.
 *   Streams:   `stream` is a cudaStream_t passed as void*; all GPU work is
 *              enqueued asynchronously on it.  NULL means the legacy default
 *              stream.
 *   Errors:    functions return an orrb_status and never throw.  Host-side
 *              checks run before anything is enqueued.  Checks that need the
 *              contents of device arrays run inside the kernels: a violation
 *              sets a bit in the workspace status word and skips the
 *              offending image (or instance, triangle); read it with
 *              orrb_read_status().  orrb_last_error() gives a message for
 *              the last failure on the context.
 *   Threads:   a context may be used from several host threads; calls are
 *              serialised by a mutex inside the context.
 */
#ifndef ORRB_H
#define ORRB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORRB_MAX_LIGHTS 4
#define ORRB_MAX_MATERIALS 32
#define ORRB_MAX_RESOLUTION 4096
#define ORRB_MAX_INSTANCES 1024
#define ORRB_GBUFFER_PLANES 7

typedef int32_t orrb_status;
#define ORRB_OK 0
#define ORRB_ERR_INVALID_ARG 1   /* a host-side argument check failed */
#define ORRB_ERR_WORKSPACE 2     /* workspace or arena too small */
#define ORRB_ERR_CUDA 3          /* a CUDA runtime call failed */
#define ORRB_ERR_TIMEOUT 4       /* a bounded device wait gave up */
#define ORRB_ERR_NOT_FOUND 5     /* no mesh set uploaded on the context */
#define ORRB_ERR_UNSUPPORTED 6   /* device is not sm_103 or option unsupported */
#define ORRB_ERR_DEVICE 7        /* the device status word is non-zero */

/* Device status word bits (orrb_read_status). */
#define ORRB_DEV_BAD_CAMERA 0x1u     /* width/height outside [1, declared max] or bad intrinsics */
#define ORRB_DEV_BAD_INSTANCE 0x2u   /* mesh id out of range or too many instances */
#define ORRB_DEV_TOO_MANY_TRIS 0x4u  /* sample has more triangles than declared */
#define ORRB_DEV_BAD_MATERIAL 0x8u   /* material slot >= 32 (clamped to 31) */
#define ORRB_DEV_BAD_LIGHTS 0x10u    /* light count outside [0, 4] (clamped) */
#define ORRB_DEV_DROPPED 0x20u       /* a triangle left the +-2^20 px guard band and was dropped */
#define ORRB_DEV_TIMEOUT 0x40u       /* a bounded wait between CTAs gave up (outputs may be incomplete) */

typedef struct orrb_ctx orrb_ctx;

/* Create a context on CUDA device `device` (must be compute capability 10.3).
 * Returns ORRB_ERR_UNSUPPORTED on another architecture. */
orrb_status orrb_create(int device, orrb_ctx** out);
void orrb_destroy(orrb_ctx* ctx);
const char* orrb_status_string(orrb_status s);
/* Copies the message of the last failure on `ctx` into buf (NUL-terminated). */
orrb_status orrb_last_error(orrb_ctx* ctx, char* buf, size_t len);

/* ---------------------------------------------------------------------- */
/* Meshes (shared by all samples: Single Scene Multiple States, Sec. 3).   */
/* ---------------------------------------------------------------------- */
typedef struct {
  const float* pos;       /* host, [n_verts][3] object-space positions (metres) */
  const float* nrm;       /* host, [n_verts][3] unit vertex normals */
  int32_t n_verts;
  const uint32_t* idx;    /* host, [n_tris][3] vertex indices, counter-clockwise seen from outside */
  const uint8_t* tri_mat; /* host, [n_tris] material slot relative to the instance's base */
  int32_t n_tris;
} orrb_mesh_desc;

/* Bytes of device arena needed to hold meshes[0..n). */
orrb_status orrb_mesh_arena_size(const orrb_mesh_desc* meshes, int32_t n, size_t* bytes);

/* Split the meshes into clusters of at most 64 vertices / 128 triangles
 * (host), write them into the caller-owned device arena `dev_arena`
 * (256-byte aligned, `arena_bytes` long) on `stream`, and make them the
 * context's mesh set: mesh id k of later batches is meshes[k].  Returns
 * after the copy has completed; host arrays may be freed on return.  The
 * arena must stay alive and unmodified while batches that use it run.
 * Replaces any previous mesh set (whose arena the caller may then free once
 * its batches have finished). */
orrb_status orrb_upload_meshes(orrb_ctx* ctx, const orrb_mesh_desc* meshes, int32_t n, void* dev_arena,
                               size_t arena_bytes, void* stream);
/* Forget the mesh set (no device work). */
orrb_status orrb_release_meshes(orrb_ctx* ctx);

/* ---------------------------------------------------------------------- */
/* Batches                                                                  */
/* ---------------------------------------------------------------------- */
/* Host-side shape of a batch: sizes the workspace and the launch.  Every
 * bound is checked again on the device against the actual arrays. */
typedef struct {
  int32_t n_samples;
  int32_t n_cams;               /* total cameras = images */
  int32_t max_tris_per_sample;  /* >= triangles of any sample's instances */
  int32_t max_inst_per_sample;  /* <= ORRB_MAX_INSTANCES */
  int32_t max_cams_per_sample;
  int32_t max_width, max_height;/* <= ORRB_MAX_RESOLUTION */
  int64_t total_pixels;         /* sum of width*height over cameras */
  int32_t shadow_res;           /* side of the square shadow maps, <= ORRB_MAX_RESOLUTION; 0: no shadows */
  int32_t shadow_faces;         /* F, shadow cameras per light in [1, 6] (1: spot, 6: cube map); 0 means 1 */
  int32_t post_effects;         /* 1: the batch may carry post-processing parameters (batch.post), and
                                   the workspace holds the post pass's images (46 B per pixel); 0: none */
} orrb_batch_shape;

/* Per-sample state and randomization parameters; all device pointers. */
typedef struct {
  const int32_t* inst_offset;    /* [n_samples+1] CSR: instances of sample s are [off[s], off[s+1]) */
  const uint32_t* inst_mesh;     /* [n_inst] mesh id */
  const float* inst_pose;        /* [n_inst][3][4] world-from-object, rigid (rotation | translation) */
  const uint8_t* inst_seg;       /* [n_inst] segmentation id written for the instance's pixels */
  const int16_t* inst_mat_base;  /* [n_inst] first material slot; slot = base + tri_mat < 32 */
  const int32_t* cam_offset;     /* [n_samples+1] CSR of cameras per sample */
  const int32_t* cam_sample;     /* [n_cams] owning sample of each camera */
  const float* cam_view;         /* [n_cams][3][4] camera-from-world, OpenGL axes */
  const float* cam_intr;         /* [n_cams][6] fx, fy, cx, cy (pixels), near (m), type (0 persp, 1 ortho) */
  const int32_t* cam_wh;         /* [n_cams][2] width, height */
  const int64_t* img_offset;     /* [n_cams] first pixel of each image in the flat outputs */
  const float* light;            /* [n_samples][4][4] world position (point, spot) or travel direction
                                    (directional) xyz, intensity */
  const int32_t* light_meta;     /* [n_samples][2] light count (0..4), type (0 point, 1 directional,
                                    2 spot: needs light_spot).  Another type, or a spot type without
                                    light_spot, sets ORRB_DEV_BAD_LIGHTS and lights nothing. */
  const float* material;         /* [n_samples][32][5] albedo rgb, specular k_s, shininess alpha */
  const float* exposure_ev;      /* [n_samples] exposure in stops */
  const float* ambient;          /* [n_samples][3] */
  const float* background;       /* [n_samples][3] linear background colour */
  const float* grading;          /* [n_samples][8] or NULL: colour grading of the rgb output (the
                                    post-processing randomizer, Sec. 4.3.1), applied in fp32 to the
                                    linear colour of every pixel before quantisation, in this order:
                                    white balance r *= 1 + t, g *= 1 + u, b *= 1 - t; rotation by h
                                    about the grey axis (1,1,1)/sqrt(3); saturation c = Y + s (c - Y),
                                    Y the Rec. 709 luma; contrast c = (c - 1/2) k + 1/2; brightness
                                    c += b; grain c += a (n - 1/2), n in [0, 1) from the PCG hash of
                                    the seed, the camera's index within its sample and the pixel's
                                    index within its image.  Row: h, s, k, b, t, u, a, seed (an
                                    integer below 2^24).  rgb_linear is not graded. */
  const float* light_spot;       /* [n_samples][4][5] or NULL: the cones of spot lights (the
                                    LightRandomizer's spotlight angles, Sec. 4.3.1): world axis xyz
                                    (unit length, the direction the spot points), cos of the outer
                                    and of the inner half-angle.  A cone with cos_inner <= cos_outer
                                    lights nothing.  The kernels fold 1 / (cos_inner - cos_outer) into
                                    the axis, which scales the rounding of the cone's cosine by that
                                    factor: the rgb_linear contract (1e-4 against the oracle) is held
                                    for cos_inner - cos_outer >= 0.01 (tested at 0.01); a narrower
                                    ramp renders, but its pixels on the ramp may differ by more.
                                    Read only for samples of light type 2. */
  const float* emission;         /* [n_samples][32] or NULL (none): material emission e, the emitted
                                    colour being e * albedo (a MuJoCo material's emission, Sec. 4.2) */
  const float* shadow_view;      /* [n_samples][4][F][3][4] or NULL: per light F perspective shadow
                                    cameras ("faces": one for a spot light, six cube faces for a point
                                    light; camera-from-world, OpenGL axes, rigid) for the soft shadows
                                    of the benchmark's lights (Sec. 5); used when shape.shadow_res > 0 */
  const float* shadow_intr;      /* [n_samples][4][F][7] or NULL: each face's fx, fy, cx, cy (pixels
                                    of the shadow_res square map; pixels per metre when orthographic),
                                    near (m), depth bias (m) and type (0 perspective, 1 orthographic,
                                    as for a directional light); fx == 0: the face casts no shadow.  A face of a light l < the sample's
                                    light count with fx != 0 casts: its map holds the depth from its
                                    camera of the nearest back face of the sample's triangles (front
                                    faces are culled), rendered with the camera rules above, 0 where
                                    none.  A visible surface point is projected, for the light's
                                    casting faces in order, in fp32 with every operation rounded to
                                    nearest: P the G-buffer position (x_v = depth ((x + 1/2 - cx) *
                                    (1/fx)), y_v = -depth ((y + 1/2 - cy) * (1/fy)), z_v = -depth,
                                    1/fx rounded once), q = (S V^-1) P with V^-1 = [R^T | -R^T t] and
                                    products summed in index order, z = -q_z, u = cx + fx (q_x (1 /
                                    z)), v = cy - fy (q_y (1 / z)) (orthographic: u = cx + fx q_x, v
                                    = cy - fy q_y); the first face with z > near and
                                    (floor(u), floor(v)) inside its map decides (none: unshadowed):
                                    k of the 3 x 3 texels (floor(u) + a, floor(v) + b), a, b in {-1,
                                    0, 1}, shadow it when inside the map with depth d > 0 and (z -
                                    bias) > d (percentage-closer filtering), and the light's E is
                                    multiplied by (9 - k) / 9. */
  const float* post;             /* [n_samples][4] or NULL: ambient occlusion and bloom of the rgb output
                                    (the rest of the post-processing randomizer, Sec. 4.3.1): AO
                                    intensity a, bloom intensity beta, bloom radius sigma (pixels), 0.
                                    Needs shape.post_effects = 1.  Applied to the linear colour of every
                                    pixel after the shading and before the grading, in fp32, from the
                                    image's depth channel and binary16 normals only.  AO: for a pixel
                                    with surface, P its G-buffer position (as for the shadow lookup),
                                    n its decoded normal, over the eight offsets (2, 1), (-1, 3),
                                    (-4, -1), (1, -4), (5, 2), (-2, 5), (-5, -3), (3, -6) whose pixel is
                                    in the image and has a surface, v = P' - P, L = |v|:
                                    o = max(0, n.v / L - 0.1) / (1 + L^2 / 0.05^2); O = sum(o) / 8;
                                    c *= max(0, 1 - a O).  Bloom (beta != 0, sigma > 0): the bright part
                                    max(c - 1, 0) blurred by the normalised Gaussian of standard
                                    deviation sigma truncated at min(ceil(3 sigma), 16) pixels, rows
                                    then columns, indices clamped to the image, times beta, is added.
                                    rgb_linear stays the shading's colour.  Not differentiated. */
} orrb_batch_desc;

/* Caller-preallocated outputs, flat over all pixels of all images (image c
 * at img_offset[c], row-major, row 0 at the top); any pointer may be NULL. */
typedef struct {
  uint8_t* rgb;         /* device, [N][3] */
  float* depth;         /* device, [N] */
  uint16_t* normal;     /* device, [N][3] binary16 bits */
  uint8_t* seg;         /* device, [N] */
  float* rgb_linear;    /* device, [N][3] before clamp and quantisation */
  float* gbuffer;       /* device, [7][N] planes: position xyz, normal xyz (view space),
                           material word as int32 bits (-1 background): the slot in bits 0-7 and,
                           with shadows, light l's shadowing tap count k in bits 8 + 4l .. 11 + 4l;
                           input of the backward */
  int32_t* tracker;     /* device, [n_cams][max_inst_per_sample][8] per camera and instance of its
                           sample (the tracker output, Sec. 4.3.2): the 8.8 fixed-point screen box
                           x0, y0, x1, y1 of the instance's vertices that its triangles use, that
                           lie in front of the near plane and inside the guard band, snapped as the
                           triangle vertices are (empty: INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN;
                           a mesh without triangles keeps an empty row), the snapped
                           projection kx, ky of its origin, flags (bit 0 box, bit 1 origin), 0.
                           Rows past a sample's instance count are left as they were. */
  float* shadow_map;    /* device, [n_samples][4][F][shadow_res][shadow_res] depth (0: none); needed
                           when shape.shadow_res > 0 and the batch has shadow cameras.  Written for
                           the faces that cast, first (its own launch), then read by the shading.
                           Maps of faces that cast none are left as they were. */
  float* rgb_graded;    /* device, [N][3] or NULL: the colour after ambient occlusion and bloom
                           (batch.post) and the colour grading (batch.grading), before clamping and
                           quantisation, the input of a loss on the graded image (see
                           orrb_param_grads.d_grading, which needs a batch without post); for an
                           ungraded batch without post, rgb_linear */
} orrb_outputs;

#define ORRB_MODE_FUSED 0  /* one persistent launch over all images (work queue) */
#define ORRB_MODE_PLAIN 1  /* three launches (setup, bin, raster+shade) per sample */
#define ORRB_MODE_STAGED 2 /* the same three kernels, each launched once over a chunk of the batch's
                              images (every image's geometry, then binning, then raster+shade); a
                              chunk holds as many images as fit in 8 GiB of scratch, at least two
                              per SM.  Same outputs as the other modes; for comparison with the
                              fused launch */

typedef struct {
  int32_t mode;          /* ORRB_MODE_FUSED, ORRB_MODE_PLAIN or ORRB_MODE_STAGED */
  int32_t tile_w;        /* screen-tile width in pixels, multiple of 8 in [8, 512]; 0 = 256 (a narrower image uses its width) */
  int32_t tile_h;        /* screen-tile height in pixels, in [1, 64], tile_w * tile_h <= 8192; 0 = 2 */
  int32_t threads;       /* threads per CTA: 256 or 512; 0 = 512 */
  int32_t ctas_per_sm;   /* fused mode: resident CTAs per SM; 0 = as many as fit */
  int32_t reserved;      /* must be 0 */
  int64_t wait_cycles;   /* fused mode: a wait between CTAs (a CTA looking for raster tiles to help
                            with, an image's owner waiting for its helpers before it reuses its
                            scratch for the next image) gives up after this many
                            SM clock cycles, sets ORRB_DEV_TIMEOUT and leaves the launch (the
                            outputs may then be incomplete); 0 = 2e9, about a second.  A small value
                            makes the waits run out on purpose. */
} orrb_config;

/* Workspace bytes for `shape` under `cfg`.  The workspace is caller-owned
 * device memory (256-byte aligned); its first 256 bytes hold the status word. */
orrb_status orrb_workspace_size(orrb_ctx* ctx, const orrb_batch_shape* shape, const orrb_config* cfg,
                                size_t* bytes);

/* Render one batch into `out` (Sec. 4.4 channels), asynchronously on
 * `stream`.  Clears the workspace status word first. */
orrb_status orrb_render_batch(orrb_ctx* ctx, const orrb_batch_shape* shape, const orrb_batch_desc* batch,
                              const orrb_outputs* out, const orrb_config* cfg, void* workspace,
                              size_t ws_bytes, void* stream);

/* Render without any device allocation -- no counterpart in the paper.
 *
 * For callers that cannot hand the library a workspace: code running inside
 * another runtime that owns the GPU's memory pool (a framework's custom op, a
 * simulator's render callback) and may not call cudaMalloc, whether because
 * the pool has already claimed the memory or because cudaMalloc can
 * synchronise the device in the middle of that runtime's pipeline.  Same
 * inputs, outputs and results as orrb_render_batch in ORRB_MODE_FUSED; the
 * per-CTA scratch lives instead in one static device array of
 * ORRB_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  Fewer CTAs run when a sample's scratch slot is large;
 * a shape whose slot (about 740 bytes per triangle of the largest sample)
 * does not fit even once is rejected with ORRB_ERR_WORKSPACE.  The entry
 * point calls no cudaMalloc, cudaFree or allocating library routine.  A batch
 * with post-processing parameters (batch.post) is rejected with
 * ORRB_ERR_UNSUPPORTED: its images need the workspace.
 *   device_status: optional device pointer to one uint32 that receives the
 *     ORRB_DEV_* bits (cleared by this call); NULL discards them.
 * The first call on a device looks up the static array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The address is kept for the life of the process: after a device reset
 * (cudaDeviceReset, or a reset of the primary context) it is stale, and the
 * entry point must not be called again until the library is reloaded.
 * All calls share the one array: calls whose GPU work overlaps (different
 * streams, threads or contexts on the same device) race and corrupt each
 * other's results; serialise them on one stream. */
#define ORRB_NOALLOC_SCRATCH_BYTES (64u << 20)
orrb_status orrb_render_batch_noalloc(orrb_ctx* ctx, const orrb_batch_shape* shape, const orrb_batch_desc* batch,
                                      const orrb_outputs* out, const orrb_config* cfg, uint32_t* device_status,
                                      void* stream);

/* Synchronise `stream` and read the workspace status word (ORRB_DEV_* bits). */
orrb_status orrb_read_status(orrb_ctx* ctx, const void* workspace, void* stream, uint32_t* status);

/* ---------------------------------------------------------------------- */
/* Shading adjoint at fixed visibility                                      */
/* ---------------------------------------------------------------------- */
typedef struct {
  float* d_material;   /* device, [n_samples][32][4]: d albedo rgb, d specular (overwritten) */
  float* d_light;      /* device, [n_samples][4][4]: d world position/direction xyz, d intensity */
  float* d_exposure;   /* device, [n_samples] */
  float* d_emission;   /* device, [n_samples][32], or NULL: d emission (overwritten) */
  float* d_grading;    /* device, [n_samples][8], or NULL.  When given (the batch must be graded),
                          the loss is on the graded colour: the d_rgb_linear argument of
                          orrb_shade_backward holds dL/d rgb_graded instead, the adjoint goes back
                          through the grading (Sec. 4.3.1 post-processing randomizer) to every
                          parameter, and d_grading receives d hue, saturation, contrast,
                          brightness, temperature, tint, grain amplitude, and 0 for the seed.  The
                          background's colour is graded too: its pixels count for the grading
                          parameters (the background colour itself is not differentiated).  A
                          batch with post-processing (batch.post) is rejected with
                          ORRB_ERR_UNSUPPORTED: ambient occlusion and bloom are not differentiated. */
} orrb_param_grads;

/* Workspace bytes of orrb_shade_backward for `shape` (partial sums). */
orrb_status orrb_backward_workspace_size(orrb_ctx* ctx, const orrb_batch_shape* shape, size_t* bytes);

/* Gradients of a loss L w.r.t. the randomized material, light and exposure
 * parameters (Sec. 4.3.1), given d_rgb_linear = dL/d rgb_linear [N][3] and
 * the G-buffer a render wrote.  Visibility is held fixed (it does not depend
 * on these parameters).  Spot axes and cones, shininess and the ambient term
 * are not differentiated.  The reduction over pixels runs in a fixed order, so
 * results are bit-identical from run to run. */
orrb_status orrb_shade_backward(orrb_ctx* ctx, const orrb_batch_shape* shape, const orrb_batch_desc* batch,
                                const float* gbuffer, const float* d_rgb_linear, const orrb_param_grads* grads,
                                void* workspace, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif
