// orrb_internal.h -- layouts shared by the host API (orrb_api.cpp) and the
// CUDA kernels (orrb_render.cu, orrb_backward.cu).  Not part of the C-ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#ifdef __CUDACC__
#define ORRB_HD __host__ __device__
#else
#define ORRB_HD
#endif

namespace orrb {

constexpr int kMaxLights = 4;
constexpr int kMaxShadowFaces = 6;  // shadow cameras per light (a cube map)
constexpr int kMaxMaterials = 32;
constexpr int kMeshletVerts = 64;
constexpr int kMeshletTris = 128;
constexpr int kMaxSpanTiles = 64;      // a binned triangle overlaps at most this many tiles
constexpr float kGuardPx = 1048576.0f; // 2^20 px

// ---- mesh arena ----------------------------------------------------------
struct MeshEntry {        // 16 B
  int32_t meshlet_begin;
  int32_t meshlet_count;
  int32_t n_tris;
  int32_t n_verts;
};

struct MeshletEntry {     // 16 B
  int32_t vert_begin;     // into the arena's vertex arrays
  int32_t tri_begin;      // into the arena's packed triangle array
  int32_t counts;         // n_verts | n_tris << 16
  int32_t mesh_tri_base;  // mesh-local index of the meshlet's first triangle
};

struct ArenaLayout {      // byte offsets inside the arena, all 256-aligned
  size_t meshes, meshlets, bounds, vpos, vnrm, tris, total;
  int32_t n_meshes, n_meshlets, n_verts, n_tris;
};

// ---- one visible (sub)triangle, 96 B ---------------------------------------
// q0 = X0, Y0, X1, Y1 (8.8 fixed point)     q1 = X2, Y2, iw0, iw1 (float bits)
// q2 = iw2, float(area), pixel box x0 | x1 << 16, y0 | y1 << 16 | top-left << 28 | small << 31
// q3 = mat | seg << 16 | flat << 24, n0 xyz  q4 = n1 xyz, n2x   q5 = n2y, n2z, -, -
// iw = 1/w (perspective) or view depth (orthographic).
struct alignas(16) Record {
  int32_t q[24];
};

// ---- kernel parameters -----------------------------------------------------
struct Params {
  // batch (device)
  int32_t n_samples, n_cams;
  const int32_t* inst_offset;
  const uint32_t* inst_mesh;
  const float* inst_pose;
  const uint8_t* inst_seg;
  const int16_t* inst_mat_base;
  const int32_t* cam_offset;
  const int32_t* cam_sample;
  const float* cam_view;
  const float* cam_intr;
  const int32_t* cam_wh;
  const int64_t* img_offset;
  const float* light;
  const int32_t* light_meta;
  const float* material;
  const float* exposure_ev;
  const float* ambient;
  const float* background;
  const float* grading;  // [n_samples][8] or null
  const float* light_spot;  // [n_samples][4][5] or null
  const float* emission;    // [n_samples][32] or null
  const float* shadow_view;  // [n_samples][4][12] (with shadow_res > 0)
  const float* shadow_intr;  // [n_samples][4][6]
  float* shadow_map;         // [n_samples][4][R][R]: written by the shadow pass, read by the shading
  uint32_t* shadow_nb;       // [n_samples][4][R][R] or null: per texel over its 3 x 3 neighbourhood, the least
                             // depth > 0 (+inf if none, binary16 rounded down) | the largest (0 if none,
                             // binary16 rounded up) << 16
  uint8_t* shadow_cnt;       // [n_samples][4][R][R] (with shadow_nb): occupied texels (depth > 0) among the nine
  int32_t shadow_res;        // R, 0 without shadows
  int32_t shadow_faces;      // F, shadow cameras per light
  int32_t shadow_pass;       // this launch renders the shadow maps (images: (sample * 4 + light) * F + face)
  // outputs (device, any may be null)
  uint8_t* rgb;
  float* depth;
  uint16_t* normal;
  uint8_t* seg;
  float* rgb_linear;
  float* rgb_graded;  // [N][3] or null: the graded colour before clamping
  float* gbuffer;
  int32_t* tracker;  // [n_cams][inst_max][8] or null
  int64_t total_pixels;
  // mesh set
  const MeshEntry* meshes;
  const MeshletEntry* meshlets;
  const float4* cbounds;  // per cluster: object-space bounding sphere (centre xyz, radius)
  const float4* vpos;
  const float4* vnrm;
  const uint32_t* tris;  // 3 local vertex indices (u8) | tri_mat << 24
  int32_t n_meshes;
  // declared bounds
  int32_t t_max, inst_max, w_max, h_max;
  // tiling
  int32_t tile_w, tile_h, max_tiles;
  // workspace
  uint32_t* status;
  uint32_t* work_counter;
  uint32_t* images_done;
  char* scratch;
  size_t slot_bytes;
  int32_t n_slots;
  long long wait_cycles;  // bounded waits between CTAs give up after this many SM cycles
  // plain mode: the sample this launch renders (-1 in fused mode, kStagedLaunch in staged mode)
  int32_t plain_sample;
  int32_t stage_base;  // staged mode: the first image of this launch's chunk
};

// plain_sample of a staged launch: its CTAs take images stage_base + blockIdx.x.
constexpr int32_t kStagedLaunch = -2;

// Per-slot scratch (one image at a time): sizes in elements, from t_max.
struct SlotLayout {
  size_t rec, vis_key, vis_box, bins, big, tile_off, counts, header, pub, total;
};

// The image state an owner publishes in its slot for helpers (camera, lights, materials, the
// large triangles' row spans, shadow cameras): at most this many bytes.
constexpr size_t kPubBytes = 8192;

// Binning keeps its per-tile counters in shared memory up to this many tiles, else in the slot.
constexpr int kSmemCountTiles = 4094;

ORRB_HD inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

ORRB_HD inline SlotLayout slot_layout(int t_max, int max_tiles) {
  SlotLayout L;
  size_t cap = 2 * size_t(t_max) + 2;
  size_t o = 0;
  L.header = o;   o = align256(o + 64);
  L.pub = o;      o = align256(o + kPubBytes);
  L.rec = o;      o = align256(o + cap * sizeof(Record));
  L.vis_key = o;  o = align256(o + cap * 4);
  L.vis_box = o;  o = align256(o + cap * 8);
  L.bins = o;     o = align256(o + cap * kMaxSpanTiles * 4);
  L.big = o;      o = align256(o + cap * 4);
  L.tile_off = o; o = align256(o + 2 * size_t(max_tiles) * 4);  // per tile: first and end bin entry
  L.counts = o;   o = align256(o + (max_tiles > kSmemCountTiles ? 2 * (size_t(max_tiles) + 2) * 4 : 0));
  L.total = o;
  return L;
}

// Host entry points implemented in the .cu files.
int launch_render(const Params& p, int mode, int threads, int ctas_per_sm, int max_cams_per_sample,
                  void* stream, char* err, size_t errlen);
int launch_shadow_neighbourhoods(const Params& p, void* stream, char* err, size_t errlen);
size_t render_smem_bytes(int threads, int tile_w, int tile_h, int inst_max, int max_tiles, int w_max, bool shadows);

struct BackwardParams {
  Params base;           // batch + mesh-independent fields
  const float* gbuffer;
  const float* d_rgb;
  float* d_material;
  float* d_light;
  float* d_exposure;
  float* d_emission;     // or null
  float* d_grading;      // [n_samples][8] or null: the loss is on the graded colour (d_rgb = dL/d graded)
  float* partial;        // [n_cams][blocks_per_img][kGradFloats]
  int32_t blocks_per_img;
};
// per partial row: material [32][4], light [4][4], exposure, emission [32], and for a graded loss
// the sums sum dc' c^T [3][3], sum dc' [3] and sum (sum_k dc'_k) * grain over the image's pixels
constexpr int kGradEmission = kMaxMaterials * 4 + kMaxLights * 4 + 1;
constexpr int kGradGrade = kGradEmission + kMaxMaterials;
constexpr int kGradeSums = 13;
constexpr int kGradFloats = kGradGrade + kGradeSums;  // 190
int launch_backward(const BackwardParams& p, int threads, void* stream, char* err, size_t errlen);

// The post-processing pass (ambient occlusion and bloom) after the camera launch.
struct PostParams {
  const int32_t* cam_wh;
  const int64_t* img_offset;
  const float* cam_intr;
  const int32_t* cam_sample;
  const int32_t* cam_offset;
  const float* post;     // [n_samples][4] AO intensity, bloom intensity, bloom radius, 0
  const float* grading;  // [n_samples][8] or null
  int32_t n_cams, n_samples;
  const float* lin;         // [N][3] linear colour (the camera launch's rgb_linear)
  const float* depth;       // [N]
  const uint16_t* normal;   // [N][3] binary16
  float* cao;               // [N][3] scratch: the occluded colour
  float* hblur;             // [N][3] scratch: the bright parts blurred along rows
  uint8_t* rgb;             // [N][3] or null
  float* rgb_graded;        // [N][3] or null
};
int launch_post(const PostParams& q, int w_max, int h_max, void* stream, char* err, size_t errlen);

}  // namespace orrb
