// orrb_render.cu -- forward renderer kernels for sm_103a.
//
// One image is processed in three phases, written once as device functions
// and run either inside one persistent kernel (fused mode: each CTA pulls
// images from a queue and runs all three phases on its own scratch slot) or
// as three launches per sample (plain mode):
//
//   G  geometry: per (instance, 64-vertex/128-triangle mesh cluster) a warp
//      composes MV = V * M, transforms the cluster's vertices into view space,
//      projects and snaps them to 8 fractional bits, clips triangles at the
//      near plane (Sutherland-Hodgman, cut computed in fp64), sets up and
//      culls them, writes one 96-byte record per visible (sub)triangle at a
//      slot fixed by its primitive id, and appends (key, pixel box) to the
//      image's visible list with a warp prefix scan and one atomic per warp.
//   B  binning: triangles that touch at most 64 screen tiles are counted per
//      tile (the lanes of a warp that hit the same tile share one atomic), the
//      counts are prefix-summed and the keys scattered into per-tile bins; the
//      rest go to a "large" list that every tile tests itself (in practice the
//      table plane), whose exact covered interval per image row is tabulated in
//      shared memory when it fits.
//   R  raster + shade: each warp owns one tile at a time (default: two image
//      rows), claiming tiles from the image's counter, with its depth keys in
//      warp-private shared memory, so the phase needs no CTA-wide barrier.
//      Large triangles: the lanes walk the covered pixels of each row.  Binned
//      triangles: 32 at a time, their boxes prefix-summed and the (triangle,
//      pixel) candidates spread evenly over the lanes (each finds its triangle
//      from a ballot of the starts), each covered centre folding (depth bits
//      << 32 | key) into the tile's keys with a shared-memory 64-bit atomicMin.
//      Then every pixel resolves its winner, interpolates the normal, shades
//      (Blinn-Phong, point or directional lights, exposure) and writes the
//      four channels, consecutive lanes on consecutive pixels of a row.
//
// Everything that decides coverage, visibility or depth (transform, clip,
// projection, snapping, edge functions, depth) uses explicitly rounded fp32
// intrinsics (__fmul_rn, __fadd_rn, __fdiv_rn: never contracted to FMA) or
// integers, so those channels are bit-identical to any correct
// implementation of the same definition.  Shading uses ordinary fp32 math.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <climits>
#include <mutex>

#include "orrb.h"
#include "orrb_internal.h"
#include "orrb_shading.cuh"

namespace orrb {
namespace {

constexpr unsigned long long kEmpty = ~0ull;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kPlainRasterSplit = 8;  // plain mode: CTAs sharing one image's tiles
constexpr int kStagedRasterSplit = 2;  // staged mode (measured: 1, 2, 4, 8 -> 2 fastest)
// optional features of a batch, each compiled into kernel instances of its own
constexpr int kFeatGrade = 1;  // colour grading of the rgb output
constexpr int kFeatTrack = 2;  // tracker rows
constexpr int kFeatLight = 4;  // a cone table (spot lights may occur) or material emission
constexpr int kFeatShadow = 8;        // shadow-map lookups in the shading (implies kFeatLight)
constexpr int kFeatShadowPass = 16;   // the depth-only pass that renders the shadow maps
// (9 - k) / 9 for k shadowed taps of 9, each the correctly rounded fp32 quotient
__constant__ float kPcfFactor[10] = {1.0f,        0.8888889f, 0.7777778f, 0.6666667f, 0.5555556f,
                                     0.44444445f, 0.33333334f, 0.22222222f, 0.11111111f, 0.0f};


struct ImageInfo {
  int cam, s, W, H, inst0, n_inst, ortho, T, valid;
  int tw, th, ntx, n_tiles;
  unsigned m_tw, m_th;  // ceil(2^32 / d) (0 for d = 1): x / d = umulhi(x, m) exactly for x < 2^16, d <= 4096
  long long px_off;
  float fx, fy, cx, cy, near, inv_fx, inv_fy;
  float V[12];
  int n_lights, light_type;
  float scale;
  float amb[3], bg[3];
  alignas(16) float lv[kMaxLights][4];  // view-space light position (point, spot) or direction to the light, intensity
  // spot lights: the view-space axis a and -cos_o, both over cos_i - cos_o, so that the cone's
  // t = (x - cos_o) / (cos_i - cos_o) = -(Lv . a) |Lv|^-1 + la[3] (a null cone: 0, 0, 0, -1)
  alignas(16) float la[kMaxLights][4];
  // colour grading of the rgb output (when the batch has it): the affine map of its white
  // balance, hue, saturation, contrast and brightness (rows of A | t), the grain amplitude and
  // the grain hash of (seed, camera within the sample)
  float gm[3][4];
  float grain;
  unsigned grain_key;
};

// Shadows of the current image (the lookup instances; in dynamic shared memory right after the
// span table, present only in launches with shadow maps): per casting face of each light the
// camera-to-shadow-camera map S V^-1 and the shadow camera's fx, fy, cx, cy, near, bias.
struct ShadowInfo {
  int cast[kMaxLights][kMaxShadowFaces];
  alignas(16) float sm[kMaxLights][kMaxShadowFaces][12];  // (rows of 16-byte vector loads)
  alignas(16) float si[kMaxLights][kMaxShadowFaces][8];   // the seven intrinsics, padded
  unsigned long long map_off[kMaxLights][kMaxShadowFaces];  // first texel of the face's map
  float pcf[12];  // (9 - k) / 9 for k = 0..9 (a shared-memory copy: lanes index it divergently)
};

struct CtaShared {
  ImageInfo im;
  alignas(16) float mat[kMaxMaterials][8];  // albedo rgb, specular, shininess, emission (padded: vector loads)
  int n_vis, n_big, next_tile, next_job, img;
  int bin_overflow;  // phase B: some tile got more keys than its share of the bin array
  int help_slot, help_cam;
  int stop;  // a wait for helpers timed out: the CTA takes no further work
  float red_score[32];  // helper search: per-warp best score and slot
  int red_slot[32];
  int scan_tmp[33];
};

struct WarpG {  // per-warp cluster staging for phase G
  float mv[12];
  float pv[kMeshletVerts * 3];
  float nv[kMeshletVerts * 3];
  int X[kMeshletVerts];
  int Y[kMeshletVerts];
  float iw[kMeshletVerts];
  int flag[kMeshletVerts];  // bit 0: in front of the near plane; bit 1: inside the guard band
  uint32_t tri[kMeshletTris];  // the cluster's packed triangles
};

struct WarpTri {  // a binned triangle staged for the warp's fragment expansion (80 B)
  int X[3], Y[3];
  float iw[3];
  float fA;
  unsigned key;
  int flags;  // bits 0-2: top-left edges; bit 3: small (32-bit relative arithmetic)
  int px0, py0, bw, start;  // first row's (or the box's) first column and width; index of its first candidate
  int px1, bw1;             // tiles of at most two rows: the second row's first column and width
  int pad[2];
};

struct Scratch {
  char* pub;  // the image state the owner publishes for helpers (PubImage)
  Record* rec;
  uint32_t* vis_key;
  uint2* vis_box;
  uint32_t* bins;
  uint32_t* big;
  uint32_t* tile_off;
  // header: [0..1] claim word (camera + 1) << 32 | next tile, 0 while no raster phase is
  // open; [2] n_vis; [3] n_big; [4] tiles finished; [5] tiles of the open image; [6] helper CTAs
  // that joined the open image
  int* counts;  // per-tile counters and cursors when they do not fit in shared memory
  int* header;
  __device__ unsigned long long* claim() const { return reinterpret_cast<unsigned long long*>(header); }
};

// Row spans of the large triangles (one 32-bit entry per triangle and image row) are kept
// in shared memory when the image has at most this many (triangle, row) pairs.
constexpr int kSpanCap = 1024;

struct SmemLayout {
  size_t uni, g_size, b_size, spans;
  // phase R, per warp: depth keys of the tile and the staged triangles
  size_t w_keys, w_tri, w_bytes, r_size;
  size_t total;
};

struct SmemPtrs {
  int* mprefix;
  int* tprefix;
  int* mbegin;  // per instance: its mesh's first cluster
  char* uni;
  uint32_t* spans;
};

// What an owner publishes in its slot when it opens the raster phase, so that a helper takes
// the image's prepared state with one copy instead of setting the image up again.
struct PubImage {
  ImageInfo im;
  alignas(16) float mat[kMaxMaterials][8];
  int n_big, pad[3];
  uint32_t spans[kSpanCap];
  ShadowInfo sd;
};
static_assert(sizeof(PubImage) <= kPubBytes, "published image state exceeds its slot region");
static_assert(sizeof(PubImage) % 16 == 0 && alignof(PubImage) <= 16 && sizeof(ImageInfo) % 16 == 0 &&
                  sizeof(ShadowInfo) % 16 == 0, "published image state is copied in 16-byte words");

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

// shadows: the launch looks up shadow maps (a ShadowInfo follows the span table)
__host__ __device__ inline SmemLayout smem_layout(int threads, int tile_w, int tile_h, int inst_max, int max_tiles,
                                                  int w_max, bool shadows) {
  SmemLayout L;
  const size_t tw = size_t(tile_w < w_max ? tile_w : w_max), th = size_t(tile_h);
  L.uni = al16(size_t(3) * (inst_max + 2) * sizeof(int));
  L.g_size = size_t(threads / 32) * al16(sizeof(WarpG));
  L.b_size = max_tiles > kSmemCountTiles ? 0 : al16(size_t(2) * (max_tiles + 2) * sizeof(int));
  L.w_keys = 0;
  L.w_tri = al16(tw * th * 8);
  L.w_bytes = L.w_tri + al16(32 * sizeof(WarpTri));
  L.r_size = size_t(threads / 32) * L.w_bytes;
  size_t u = L.g_size > L.b_size ? L.g_size : L.b_size;
  u = u > L.r_size ? u : L.r_size;
  L.spans = L.uni + al16(u);
  L.total = L.spans + size_t(kSpanCap) * sizeof(uint32_t) + (shadows ? al16(sizeof(ShadowInfo)) : 0);
  return L;
}

__device__ inline Scratch slot_scratch(const Params& p, int slot) {
  SlotLayout L = slot_layout(p.t_max, p.max_tiles);
  char* b = p.scratch + size_t(slot) * p.slot_bytes;
  Scratch s;
  s.header = reinterpret_cast<int*>(b + L.header);
  s.pub = b + L.pub;
  s.rec = reinterpret_cast<Record*>(b + L.rec);
  s.vis_key = reinterpret_cast<uint32_t*>(b + L.vis_key);
  s.vis_box = reinterpret_cast<uint2*>(b + L.vis_box);
  s.bins = reinterpret_cast<uint32_t*>(b + L.bins);
  s.big = reinterpret_cast<uint32_t*>(b + L.big);
  s.tile_off = reinterpret_cast<uint32_t*>(b + L.tile_off);
  s.counts = reinterpret_cast<int*>(b + L.counts);
  return s;
}

__device__ inline void flag_status(const Params& p, unsigned bits) { atomicOr(p.status, bits); }

// Exclusive scan of a[0..n) in place over the whole block; writes the total to a[n].
__device__ void block_exclusive_scan(int* a, int n, int* tmp) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int per = (n + nt - 1) / nt;
  const int b = min(tid * per, n), e = min(b + per, n);
  int sum = 0;
  for (int i = b; i < e; i++) sum += a[i];
  const int lane = tid & 31, warp = tid >> 5;
  int incl = sum;
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int nw = nt >> 5;
    int v = lane < nw ? tmp[lane] : 0;
    int inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane < nw) tmp[lane] = inc - v;
    if (lane == nw - 1) tmp[32] = inc;
  }
  __syncthreads();
  int run = tmp[warp] + incl - sum;
  for (int i = b; i < e; i++) {
    int v = a[i];
    a[i] = run;
    run += v;
  }
  if (tid == 0) a[n] = tmp[32];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// per-image set-up (camera, lights, materials, instance tables)
// ---------------------------------------------------------------------------
// track: (with tables) also start this image's tracker rows empty.
// kPass: the shadow pass, whose image `cam` is the map of face cam % F of light (cam / F) % 4 of
// sample cam / (4 F).
template <bool kPass = false>
__device__ void setup_image(const Params& p, int cam, CtaShared& sh, int* mprefix, int* tprefix, int* mbegin,
                            bool tables, bool track = false) {
  ImageInfo& im = sh.im;
  const int tid = threadIdx.x;
  if (tid == 0) {
    im.cam = cam;
    int s = kPass ? cam / (kMaxLights * p.shadow_faces) : p.cam_sample[cam];
    im.s = s;
    im.W = kPass ? p.shadow_res : p.cam_wh[cam * 2 + 0];
    im.H = kPass ? p.shadow_res : p.cam_wh[cam * 2 + 1];
    im.valid = 1;
    const float* in = kPass ? p.shadow_intr + cam * 7 : p.cam_intr + cam * 6;
    im.fx = in[0];
    im.fy = in[1];
    im.cx = in[2];
    im.cy = in[3];
    im.near = in[4];
    im.ortho = (kPass ? in[6] : in[5]) != 0.0f;
    im.inv_fx = __frcp_rn(im.fx);  // correctly rounded: the G-buffer position uses it
    im.inv_fy = __frcp_rn(im.fy);
    if (kPass && in[0] == 0.0f) {  // the light casts no shadow: no map (not an error)
      im.valid = 0;
    } else if (s < 0 || s >= p.n_samples || im.W < 1 || im.H < 1 || im.W > p.w_max || im.H > p.h_max ||
               !(im.near > 0.0f) || !(im.fx != 0.0f) || !(im.fy != 0.0f)) {
      flag_status(p, ORRB_DEV_BAD_CAMERA);
      im.valid = 0;
      s = 0;
      im.s = 0;
    }
    for (int k = 0; k < 12; k++) im.V[k] = (kPass ? p.shadow_view : p.cam_view)[cam * 12 + k];
    im.px_off = kPass ? (long long)cam * p.shadow_res * p.shadow_res : p.img_offset[cam];
    if (im.valid && (im.px_off < 0 || im.px_off + (long long)im.W * im.H > p.total_pixels)) {
      flag_status(p, ORRB_DEV_BAD_CAMERA);  // the image would not fit in the output arrays
      im.valid = 0;
    }
    im.inst0 = p.inst_offset[s];
    im.n_inst = p.inst_offset[s + 1] - im.inst0;
    if (im.n_inst < 0 || im.n_inst > p.inst_max) {
      flag_status(p, ORRB_DEV_BAD_INSTANCE);
      im.valid = 0;
      im.n_inst = 0;
    }
    im.tw = min(im.W, p.tile_w);
    im.th = p.tile_h;
    im.ntx = (im.W + im.tw - 1) / im.tw;
    im.m_tw = im.tw > 1 ? unsigned((0x100000000ull + im.tw - 1) / im.tw) : 0u;
    im.m_th = im.th > 1 ? unsigned((0x100000000ull + im.th - 1) / im.th) : 0u;
    im.n_tiles = im.ntx * ((im.H + im.th - 1) / im.th);
    int nl = p.light_meta[s * 2 + 0];
    if (nl < 0 || nl > kMaxLights) {
      flag_status(p, ORRB_DEV_BAD_LIGHTS);
      nl = nl < 0 ? 0 : kMaxLights;
    }
    const int lt = p.light_meta[s * 2 + 1];
    if (!(lt == 0 || lt == 1 || (lt == 2 && p.light_spot))) {  // an unknown type lights nothing
      flag_status(p, ORRB_DEV_BAD_LIGHTS);
      nl = 0;
    }
    im.n_lights = nl;
    im.light_type = lt;
    if (kPass && (cam / p.shadow_faces) % kMaxLights >= nl) im.valid = 0;  // no such light: no map
    sh.n_vis = 0;
    sh.n_big = 0;
    sh.next_tile = 0;
    sh.next_job = 0;
  }
  __syncthreads();
  // lights into view space, exposure, ambient and background: one thread each
  if (tid < kMaxLights) {
    if (tid < im.n_lights) {
      const float* L4 = p.light + (im.s * kMaxLights + tid) * 4;
      for (int i = 0; i < 3; i++) {
        float r = im.V[i * 4 + 0] * L4[0] + im.V[i * 4 + 1] * L4[1] + im.V[i * 4 + 2] * L4[2];
        im.lv[tid][i] = im.light_type == 1 ? -r : r + im.V[i * 4 + 3];
      }
      im.lv[tid][3] = L4[3];
    }
  } else if (tid < kMaxLights + 3) {
    im.amb[tid - kMaxLights] = p.ambient[im.s * 3 + tid - kMaxLights];
  } else if (tid < kMaxLights + 6) {
    im.bg[tid - kMaxLights - 3] = p.background[im.s * 3 + tid - kMaxLights - 3];
  } else if (tid == kMaxLights + 6) {
    im.scale = exp2f(p.exposure_ev[im.s]);
  }
  for (int k = tid; k < kMaxMaterials * 5; k += blockDim.x)
    sh.mat[k / 5][k % 5] = p.material[(size_t)im.s * kMaxMaterials * 5 + k];
  if (tid >= 32 && tid < 32 + kMaxMaterials)  // column 5: emission (columns 6-7 unused); blocks have >= 256 threads
    sh.mat[tid - 32][5] = p.emission ? p.emission[(size_t)im.s * kMaxMaterials + tid - 32] : 0.0f;
  if (!tables) {
    __syncthreads();
    return;
  }
  const int n = im.n_inst;
  for (int i = tid; i < n; i += blockDim.x) {
    if (track) {  // this image's tracker rows start empty (phase G folds its vertices in)
      int4* row = reinterpret_cast<int4*>(p.tracker + ((size_t)im.cam * p.inst_max + i) * 8);
      row[0] = make_int4(INT_MAX, INT_MAX, INT_MIN, INT_MIN);
      row[1] = make_int4(0, 0, 0, 0);
    }
    uint32_t mesh = p.inst_mesh[im.inst0 + i];
    if (mesh >= (uint32_t)p.n_meshes) {
      flag_status(p, ORRB_DEV_BAD_INSTANCE);
      mprefix[i] = 0;
      tprefix[i] = 0;
      mbegin[i] = 0;
    } else {
      MeshEntry me = p.meshes[mesh];
      mprefix[i] = me.meshlet_count;
      tprefix[i] = me.n_tris;
      mbegin[i] = me.meshlet_begin;
    }
  }
  __syncthreads();
  block_exclusive_scan(mprefix, n, sh.scan_tmp);
  block_exclusive_scan(tprefix, n, sh.scan_tmp);
  if (tid == 0) {
    im.T = tprefix[n];
    if (im.T > p.t_max) {
      flag_status(p, ORRB_DEV_TOO_MANY_TRIS);
      im.valid = 0;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// phase G helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void project(const ImageInfo& im, float x, float y, float z, int& X, int& Y, float& iw,
                                        int& ok) {
  float xs, ys;
  if (im.ortho) {
    iw = -z;
    xs = __fadd_rn(im.cx, __fmul_rn(im.fx, x));
    ys = __fsub_rn(im.cy, __fmul_rn(im.fy, y));
  } else {
    iw = __fdiv_rn(1.0f, -z);
    xs = __fadd_rn(im.cx, __fmul_rn(im.fx, __fmul_rn(x, iw)));
    ys = __fsub_rn(im.cy, __fmul_rn(im.fy, __fmul_rn(y, iw)));
  }
  ok = fabsf(xs) < kGuardPx && fabsf(ys) < kGuardPx;
  X = ok ? __float2int_rn(__fmul_rn(xs, 256.0f)) : 0;
  Y = ok ? __float2int_rn(__fmul_rn(ys, 256.0f)) : 0;
}

__device__ __forceinline__ int top_left(int ax, int ay, int bx, int by) {
  int dx = bx - ax, dy = by - ay;
  return (dy == 0 && dx < 0) || dy > 0;
}

// Set up a snapped triangle: cull (area <= 0), clamp its pixel box to the image.
// Returns false if culled or entirely off-screen.  box.x = x0 | x1 << 16; box.y =
// y0 | y1 << 16 | top-left flags of edges 0..2 << 28 | small << 31, where "small"
// means a vertex box under 128 px, for which every edge function and every term of
// it fits in 32 bits relative to vertex 0.
__device__ __forceinline__ bool setup_box(const ImageInfo& im, const int X[3], const int Y[3], uint2& box,
                                          float& fA) {
  long long A = (long long)(X[2] - X[0]) * (Y[1] - Y[0]) - (long long)(Y[2] - Y[0]) * (X[1] - X[0]);
  if (A <= 0) return false;
  int xmin = min(X[0], min(X[1], X[2])), xmax = max(X[0], max(X[1], X[2]));
  int ymin = min(Y[0], min(Y[1], Y[2])), ymax = max(Y[0], max(Y[1], Y[2]));
  // pixel x has its centre at 256x + 128
  int x0 = max(0, -((128 - xmin) >> 8)), x1 = min(im.W - 1, (xmax - 128) >> 8);
  int y0 = max(0, -((128 - ymin) >> 8)), y1 = min(im.H - 1, (ymax - 128) >> 8);
  if (x0 > x1 || y0 > y1) return false;
  const unsigned tl = top_left(X[1], Y[1], X[2], Y[2]) | (top_left(X[2], Y[2], X[0], Y[0]) << 1) |
                      (top_left(X[0], Y[0], X[1], Y[1]) << 2);
  const unsigned small = (xmax - xmin) < 32768 && (ymax - ymin) < 32768;
  box.x = unsigned(x0) | (unsigned(x1) << 16);
  box.y = unsigned(y0) | (unsigned(y1) << 16) | (tl << 28) | (small << 31);
  fA = __ll2float_rn(A);
  return true;
}

__device__ __forceinline__ void write_record(Record* r, const int X[3], const int Y[3], const float iw[3],
                                             const float n[3][3], int mat, int seg, uint2 box, float fA) {
  int4* q = reinterpret_cast<int4*>(r);
  q[0] = make_int4(X[0], Y[0], X[1], Y[1]);
  q[1] = make_int4(X[2], Y[2], __float_as_int(iw[0]), __float_as_int(iw[1]));
  q[2] = make_int4(__float_as_int(iw[2]), __float_as_int(fA), int(box.x), int(box.y));
  // bit 24: the three vertex normals are bitwise equal (a flat face), so the interpolated
  // normal is n0 up to rounding and the resolve skips the interpolation
  const int flat = n[0][0] == n[1][0] && n[0][1] == n[1][1] && n[0][2] == n[1][2] && n[0][0] == n[2][0] &&
                   n[0][1] == n[2][1] && n[0][2] == n[2][2];
  q[3] = make_int4(mat | (seg << 16) | (flat << 24), __float_as_int(n[0][0]), __float_as_int(n[0][1]),
                   __float_as_int(n[0][2]));
  float4* f = reinterpret_cast<float4*>(r);
  f[4] = make_float4(n[1][0], n[1][1], n[1][2], n[2][0]);
  f[5] = make_float4(n[2][1], n[2][2], 0.0f, 0.0f);
}

struct CutVert {
  float p[3], n[3];
  int X, Y, ok;
  float iw;
};

// Cut point on edge (in -> out) with the near plane, fp64 rounded once to fp32, z = -near.
__device__ __noinline__ void cut_vertex(const ImageInfo& im, const float* pin, const float* nin, const float* pout,
                                        const float* nout, CutVert& c) {
  double t = __ddiv_rn(__dsub_rn(-(double)im.near, (double)pin[2]), __dsub_rn((double)pout[2], (double)pin[2]));
  for (int k = 0; k < 3; k++) {
    c.p[k] = __double2float_rn(__dadd_rn((double)pin[k], __dmul_rn(t, __dsub_rn((double)pout[k], (double)pin[k]))));
    c.n[k] = __double2float_rn(__dadd_rn((double)nin[k], __dmul_rn(t, __dsub_rn((double)nout[k], (double)nin[k]))));
  }
  c.p[2] = -im.near;
  project(im, c.p[0], c.p[1], c.p[2], c.X, c.Y, c.iw, c.ok);
}

// Near-plane clip of triangle (a, b, c) of the staged cluster; emits up to two
// sub-triangles.  Vertex order follows Sutherland-Hodgman: for each edge
// (v_k, v_k+1) emit v_k if inside, then the cut if the edge crosses.
// kBack: emit each sub-triangle reversed (the shadow pass keeps back faces).
template <int kBack>
__device__ __noinline__ int clip_triangle(int t_max, Record* rec, const ImageInfo& im, const WarpG* wg, int v0,
                                          int v1, int v2, int prim, int mat, int seg, unsigned* keys, uint2* boxes,
                                          unsigned* dropped) {
  const int vi[3] = {v0, v1, v2};
  CutVert poly[4];
  int np = 0;
  for (int k = 0; k < 3; k++) {
    int a = vi[k], b = vi[(k + 1) % 3];
    int ain = wg->flag[a] & 1, bin = wg->flag[b] & 1;
    if (ain) {
      CutVert& o = poly[np++];
      for (int d = 0; d < 3; d++) {
        o.p[d] = wg->pv[a * 3 + d];
        o.n[d] = wg->nv[a * 3 + d];
      }
      o.X = wg->X[a];
      o.Y = wg->Y[a];
      o.iw = wg->iw[a];
      o.ok = (wg->flag[a] >> 1) & 1;
    }
    if (ain && !bin) cut_vertex(im, &wg->pv[a * 3], &wg->nv[a * 3], &wg->pv[b * 3], &wg->nv[b * 3], poly[np++]);
    if (!ain && bin) cut_vertex(im, &wg->pv[b * 3], &wg->nv[b * 3], &wg->pv[a * 3], &wg->nv[a * 3], poly[np++]);
  }
  int emitted = 0;
  for (int sub = 0; sub + 2 < np; sub++) {
    const CutVert* q[3] = {&poly[0], &poly[sub + 1 + kBack], &poly[sub + 2 - kBack]};
    if (!(q[0]->ok && q[1]->ok && q[2]->ok)) {
      *dropped = 1;
      continue;
    }
    int X[3] = {q[0]->X, q[1]->X, q[2]->X}, Y[3] = {q[0]->Y, q[1]->Y, q[2]->Y};
    uint2 box;
    float fA;
    if (!setup_box(im, X, Y, box, fA)) continue;
    float iw[3] = {q[0]->iw, q[1]->iw, q[2]->iw};
    float n[3][3];
    for (int k = 0; k < 3; k++)
      for (int d = 0; d < 3; d++) n[k][d] = q[k]->n[d];
    write_record(rec + (size_t)sub * t_max + prim, X, Y, iw, n, mat, seg, box, fA);
    keys[emitted] = 2u * prim + sub;
    boxes[emitted] = box;
    emitted++;
  }
  return emitted;
}

// ---------------------------------------------------------------------------
// phase G: geometry of one image
// ---------------------------------------------------------------------------
// True when the bounding sphere b (object space) of a cluster, moved to view space by mv, lies
// wholly behind the near plane or wholly beyond one of the image's four edges (for a perspective
// view: in the half-space beyond the plane through the eye and that edge).  Every triangle of such
// a cluster is then clipped away or covers no pixel centre, so skipping it changes nothing.  The
// radius is widened by a millimetre and a thousandth, far beyond the fp32 error of the test.
__device__ __forceinline__ bool cluster_outside(const ImageInfo& im, const float* mv, float4 b) {
  const float x = mv[0] * b.x + mv[1] * b.y + mv[2] * b.z + mv[3];
  const float y = mv[4] * b.x + mv[5] * b.y + mv[6] * b.z + mv[7];
  const float z = mv[8] * b.x + mv[9] * b.y + mv[10] * b.z + mv[11];
  const float r = b.w * 1.001f + 1e-3f;
  if (z - r > -im.near) return true;
  const float W = float(im.W), H = float(im.H);
  if (im.ortho) {  // x_s = cx + fx x, y_s = cy - fy y
    return x + r < -im.cx / im.fx || x - r > (W - im.cx) / im.fx || y - r > im.cy / im.fy ||
           y + r < (im.cy - H) / im.fy;
  }
  // x_s < 0: fx x - cx z < 0;  x_s > W: fx x + (W - cx) z > 0;  y_s < 0: fy y + cy z > 0;
  // y_s > H: (H - cy) z - fy y > 0   (each side's normal length scales the radius)
  return im.fx * x - im.cx * z + r * sqrtf(im.fx * im.fx + im.cx * im.cx) < 0.0f ||
         im.fx * x + (W - im.cx) * z - r * sqrtf(im.fx * im.fx + (W - im.cx) * (W - im.cx)) > 0.0f ||
         im.fy * y + im.cy * z - r * sqrtf(im.fy * im.fy + im.cy * im.cy) > 0.0f ||
         (H - im.cy) * z - im.fy * y - r * sqrtf(im.fy * im.fy + (H - im.cy) * (H - im.cy)) > 0.0f;
}

// kTrack: the launch writes tracker rows (a separate instance, so that the common case carries none
// of that code).  kBack: keep back faces instead of front faces (the shadow pass): every triangle
// is taken with its second and third vertices swapped; clusters wholly outside the shadow camera's
// view are skipped (a cube face sees about a sixth of the scene).
template <bool kTrack, bool kBack = false>
__device__ void geometry_phase(const Params& p, CtaShared& sh, const int* mprefix, const int* tprefix,
                               const int* mbegin, WarpG* wgs, const Scratch& sc) {
  const ImageInfo& im = sh.im;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpG* wg = wgs + warp;
  const int jobs = mprefix[im.n_inst];
  unsigned dropped = 0, badmat = 0;
  while (true) {  // clusters are claimed one at a time: their cost varies with culling and clipping
    int j = 0;
    if (lane == 0) j = atomicAdd(&sh.next_job, 1);
    j = __shfl_sync(kFull, j, 0);
    if (j >= jobs) break;
    int lo = 0, hi = im.n_inst;  // mprefix[lo] <= j < mprefix[hi]
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (mprefix[mid] <= j) lo = mid;
      else hi = mid;
    }
    const int inst = im.inst0 + lo;
    const MeshletEntry ml = p.meshlets[mbegin[lo] + (j - mprefix[lo])];
    const int mat_base = p.inst_mat_base[inst];  // loads issued before the transform that follows
    const int seg = p.inst_seg[inst];
    if (lane < 12) {
      const int r = lane >> 2, c = lane & 3;
      const float* M = p.inst_pose + (size_t)inst * 12;
      float s = __fmul_rn(im.V[r * 4 + 0], M[0 * 4 + c]);
      s = __fadd_rn(s, __fmul_rn(im.V[r * 4 + 1], M[1 * 4 + c]));
      s = __fadd_rn(s, __fmul_rn(im.V[r * 4 + 2], M[2 * 4 + c]));
      if (c == 3) s = __fadd_rn(s, im.V[r * 4 + 3]);
      wg->mv[lane] = s;
    }
    __syncwarp();
    if (kBack && cluster_outside(im, wg->mv, __ldg(p.cbounds + mbegin[lo] + (j - mprefix[lo]))))
      continue;  // (warp-uniform: every lane tests the same sphere)
    const int nv = ml.counts & 0xffff, nt = ml.counts >> 16;
    // the cluster's triangle words and its vertices are all requested before any is used
    static_assert(kMeshletTris == 128 && kMeshletVerts == 64, "prefetch assumes 4 triangle and 2 vertex rounds");
    uint32_t tq[4];
#pragma unroll
    for (int i = 0; i < 4; i++) tq[i] = i * 32 + lane < nt ? p.tris[ml.tri_begin + i * 32 + lane] : 0u;
    int bx0 = INT_MAX, by0 = INT_MAX, bx1 = INT_MIN, by1 = INT_MIN;  // tracker box of the lane's vertices
    float4 Pq[2], Nq[2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
      const int v = i * 32 + lane;
      Pq[i] = v < nv ? p.vpos[ml.vert_begin + v] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      Nq[i] = v < nv ? p.vnrm[ml.vert_begin + v] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
#pragma unroll
    for (int i = 0; i < 4; i++) wg->tri[i * 32 + lane] = tq[i];
#pragma unroll
    for (int i = 0; i < 2; i++) {
      const int v = i * 32 + lane;
      if (v >= nv) break;
      const float4 P = Pq[i];
      const float4 N = Nq[i];
      float pc[3];
      for (int r = 0; r < 3; r++) {
        const float* m = &wg->mv[r * 4];
        pc[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(m[0], P.x), __fmul_rn(m[1], P.y)), __fmul_rn(m[2], P.z)), m[3]);
        wg->pv[v * 3 + r] = pc[r];
        wg->nv[v * 3 + r] = __fadd_rn(__fadd_rn(__fmul_rn(m[0], N.x), __fmul_rn(m[1], N.y)), __fmul_rn(m[2], N.z));
      }
      int inside = pc[2] <= -im.near;
      int X = 0, Y = 0, ok = 0;
      float iw = 0.0f;
      if (inside) project(im, pc[0], pc[1], pc[2], X, Y, iw, ok);
      wg->X[v] = X;
      wg->Y[v] = Y;
      wg->iw[v] = iw;
      wg->flag[v] = inside | (ok << 1);
      if (kTrack && inside && ok) {
        bx0 = min(bx0, X);
        by0 = min(by0, Y);
        bx1 = max(bx1, X);
        by1 = max(by1, Y);
      }
    }
    if (kTrack) {  // the cluster's box into the instance's row; its first cluster also projects the origin
      bx0 = __reduce_min_sync(kFull, bx0);
      by0 = __reduce_min_sync(kFull, by0);
      bx1 = __reduce_max_sync(kFull, bx1);
      by1 = __reduce_max_sync(kFull, by1);
      int* row = p.tracker + ((size_t)im.cam * p.inst_max + lo) * 8;
      if (lane == 0 && bx0 <= bx1) {
        atomicMin(row + 0, bx0);
        atomicMin(row + 1, by0);
        atomicMax(row + 2, bx1);
        atomicMax(row + 3, by1);
        atomicOr(row + 6, 1);
      }
      if (lane == 0 && j == mprefix[lo] && wg->mv[11] <= -im.near) {
        int kx, ky, kok;
        float kiw;
        project(im, wg->mv[3], wg->mv[7], wg->mv[11], kx, ky, kiw, kok);
        if (kok) {
          row[4] = kx;
          row[5] = ky;
          atomicOr(row + 6, 2);
        }
      }
    }
    __syncwarp();
    const int prim_base = tprefix[lo] + ml.mesh_tri_base;
    for (int base = 0; base < nt; base += 32) {
      const int t = base + lane;
      unsigned key0 = 0, key1 = 0;   // registers: the clip path writes its own arrays
      uint2 box0 = make_uint2(0, 0), box1 = make_uint2(0, 0);
      int cnt = 0;
      if (t < nt) {
        const uint32_t tri = wg->tri[t];
        const int ia = int((tri >> 8) & 0xff), ib = int((tri >> 16) & 0xff);
        const int vi[3] = {int(tri & 0xff), kBack ? ib : ia, kBack ? ia : ib};
        int mat = mat_base + int(tri >> 24);
        if (mat < 0 || mat >= kMaxMaterials) {
          badmat = 1;
          mat = mat < 0 ? 0 : kMaxMaterials - 1;
        }
        const int prim = prim_base + t;
        const int f0 = wg->flag[vi[0]], f1 = wg->flag[vi[1]], f2 = wg->flag[vi[2]];
        if (f0 & f1 & f2 & 1) {
          if (f0 & f1 & f2 & 2) {
            int X[3] = {wg->X[vi[0]], wg->X[vi[1]], wg->X[vi[2]]};
            int Y[3] = {wg->Y[vi[0]], wg->Y[vi[1]], wg->Y[vi[2]]};
            float fA;
            if (setup_box(im, X, Y, box0, fA)) {
              float iw[3] = {wg->iw[vi[0]], wg->iw[vi[1]], wg->iw[vi[2]]};
              float n[3][3];
              for (int k = 0; k < 3; k++)
                for (int d = 0; d < 3; d++) n[k][d] = wg->nv[vi[k] * 3 + d];
              write_record(sc.rec + prim, X, Y, iw, n, mat, seg, box0, fA);
              key0 = 2u * prim;
              cnt = 1;
            }
          } else {
            dropped = 1;
          }
        } else if ((f0 | f1 | f2) & 1) {
          unsigned kk[2];
          uint2 bb[2];
          unsigned drop = 0;
          // (the shadow pass clips the triangle in its own order and reverses what comes out)
          cnt = kBack ? clip_triangle<1>(p.t_max, sc.rec, im, wg, vi[0], vi[2], vi[1], prim, mat, seg, kk, bb, &drop)
                      : clip_triangle<0>(p.t_max, sc.rec, im, wg, vi[0], vi[1], vi[2], prim, mat, seg, kk, bb, &drop);
          dropped |= drop;
          key0 = kk[0];
          box0 = bb[0];
          key1 = kk[1];
          box1 = bb[1];
        }
      }
      // warp prefix scan of the per-lane counts, one atomic per warp
      int incl = cnt;
      for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
      }
      const int total = __shfl_sync(kFull, incl, 31);
      int wbase = 0;
      if (lane == 31 && total) wbase = atomicAdd(&sh.n_vis, total);
      wbase = __shfl_sync(kFull, wbase, 31);
      int pos = wbase + incl - cnt;
      if (cnt > 0) {
        sc.vis_key[pos] = key0;
        sc.vis_box[pos] = box0;
      }
      if (cnt > 1) {
        sc.vis_key[pos + 1] = key1;
        sc.vis_box[pos + 1] = box1;
      }
    }
    __syncwarp();
  }
  if (dropped) flag_status(p, ORRB_DEV_DROPPED);
  if (badmat) flag_status(p, ORRB_DEV_BAD_MATERIAL);
}

// ---------------------------------------------------------------------------
// phase B: screen-tile binning
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned udiv16(unsigned x, unsigned m) { return m ? __umulhi(x, m) : x; }

__device__ __forceinline__ bool binned_span(uint2 box, const ImageInfo& im, int& tx0, int& tx1, int& ty0, int& ty1) {
  const unsigned x0 = box.x & 0xffff, x1 = box.x >> 16, y0 = box.y & 0xffff, y1 = (box.y >> 16) & 0xfff;
  tx0 = udiv16(x0, im.m_tw);
  tx1 = udiv16(x1, im.m_tw);
  ty0 = udiv16(y0, im.m_th);
  ty1 = udiv16(y1, im.m_th);
  return (tx1 - tx0 + 1) * (ty1 - ty0 + 1) <= kMaxSpanTiles;
}

// Neighbouring visible triangles come from the same cluster and mostly share tiles, so the
// per-tile counter updates are aggregated per warp: the lanes that hit the same tile in a
// step (match.any) add their number with one atomic by the lowest of them.
// One pass: tile t's keys go to bins[t * cap, t * cap + count_t), cap being the tile's equal share
// of the bin array; only if some tile would exceed its share does a second pass redo the image
// with exact offsets (counts, prefix sum, scatter).  tile_off holds each tile's (first, end).
__device__ void bin_phase(const Params& p, CtaShared& sh, int* counts, int* cursor, const Scratch& sc) {
  const ImageInfo& im = sh.im;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < im.n_tiles; t += nt) counts[t] = 0;
  if (tid == 0) sh.bin_overflow = 0;
  __syncthreads();
  const int n = sh.n_vis;
  const int lane = tid & 31;
  const unsigned below = (1u << lane) - 1u;
  const int cap = int(size_t(2 * p.t_max + 2) * kMaxSpanTiles / size_t(im.n_tiles));
  for (int e0 = 0; e0 < n; e0 += nt) {
    const int e = e0 + tid;
    bool big = false;
    int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = 0;
    uint32_t key = 0;
    if (e < n) {
      key = sc.vis_key[e];
      if (!binned_span(sc.vis_box[e], im, tx0, tx1, ty0, ty1)) {
        big = true;
        tx1 = -1;
      }
    }
    const int w = tx1 - tx0 + 1, cnt = w > 0 ? w * (ty1 - ty0 + 1) : 0;
    const int steps = __reduce_max_sync(kFull, cnt);
    int tx = tx0, ty = ty0;
    for (int j = 0; j < steps; j++) {
      const int tile = j < cnt ? ty * im.ntx + tx : -1;
      const unsigned peers = __match_any_sync(kFull, tile);
      const int leader = __ffs(peers) - 1;
      int slot = 0;
      if (tile >= 0 && lane == leader) slot = atomicAdd(&counts[tile], __popc(peers));
      slot = __shfl_sync(kFull, slot, leader) + __popc(peers & below);
      if (tile >= 0) {
        if (slot < cap) sc.bins[size_t(tile) * cap + slot] = key;
        else sh.bin_overflow = 1;
      }
      if (++tx > tx1) tx = tx0, ty++;
    }
    // ballot compaction of the large list: one atomic per warp
    const unsigned m = __ballot_sync(kFull, big);
    int wbase = 0;
    if (lane == 0 && m) wbase = atomicAdd(&sh.n_big, __popc(m));
    wbase = __shfl_sync(kFull, wbase, 0);
    if (big) sc.big[wbase + __popc(m & below)] = key;
  }
  __syncthreads();
  if (!sh.bin_overflow) {
    for (int t = tid; t < im.n_tiles; t += nt) {
      sc.tile_off[2 * t] = t * cap;
      sc.tile_off[2 * t + 1] = t * cap + counts[t];
    }
    __syncthreads();
    return;
  }
  // second pass: exact offsets from the counts (the counts are complete even where bins overflowed)
  block_exclusive_scan(counts, im.n_tiles, sh.scan_tmp);
  for (int t = tid; t < im.n_tiles; t += nt) {
    sc.tile_off[2 * t] = counts[t];
    sc.tile_off[2 * t + 1] = counts[t + 1];
    cursor[t] = counts[t];
  }
  __syncthreads();
  for (int e0 = 0; e0 < n; e0 += nt) {
    const int e = e0 + tid;
    int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = 0;
    uint32_t key = 0;
    if (e < n) {
      if (binned_span(sc.vis_box[e], im, tx0, tx1, ty0, ty1)) key = sc.vis_key[e];
      else tx1 = -1;
    }
    const int w = tx1 - tx0 + 1, cnt = w > 0 ? w * (ty1 - ty0 + 1) : 0;
    const int steps = __reduce_max_sync(kFull, cnt);
    int tx = tx0, ty = ty0;
    for (int j = 0; j < steps; j++) {
      const int tile = j < cnt ? ty * im.ntx + tx : -1;
      const unsigned peers = __match_any_sync(kFull, tile);
      const int leader = __ffs(peers) - 1;
      int base = 0;
      if (tile >= 0 && lane == leader) base = atomicAdd(&cursor[tile], __popc(peers));
      base = __shfl_sync(kFull, base, leader);
      if (tile >= 0) sc.bins[base + __popc(peers & below)] = key;
      if (++tx > tx1) tx = tx0, ty++;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// phase R: raster + shade one tile
// ---------------------------------------------------------------------------

// Fragment test at pixel centre (cx, cy): returns the 64-bit key or kEmpty.
__device__ __forceinline__ unsigned long long fragment(const int X[3], const int Y[3], const float iw[3], float fA,
                                                       int tl, unsigned key, int ortho, int cx, int cy) {
  long long w0 = (long long)(cx - X[1]) * (Y[2] - Y[1]) - (long long)(cy - Y[1]) * (X[2] - X[1]);
  long long w1 = (long long)(cx - X[2]) * (Y[0] - Y[2]) - (long long)(cy - Y[2]) * (X[0] - X[2]);
  long long w2 = (long long)(cx - X[0]) * (Y[1] - Y[0]) - (long long)(cy - Y[0]) * (X[1] - X[0]);
  if (!(w0 + (tl & 1) > 0 && w1 + ((tl >> 1) & 1) > 0 && w2 + ((tl >> 2) & 1) > 0)) return kEmpty;
  float f0 = __ll2float_rn(w0), f1 = __ll2float_rn(w1), f2 = __ll2float_rn(w2);
  float s = __fadd_rn(__fadd_rn(__fmul_rn(f0, iw[0]), __fmul_rn(f1, iw[1])), __fmul_rn(f2, iw[2]));
  float depth = ortho ? __fdiv_rn(s, fA) : __fdiv_rn(fA, s);
  return ((unsigned long long)__float_as_uint(depth) << 32) | key;
}

__device__ __forceinline__ void load_tri(const Record* r, int X[3], int Y[3], float iw[3]) {
  const int4 q0 = reinterpret_cast<const int4*>(r)[0];
  const int4 q1 = reinterpret_cast<const int4*>(r)[1];
  const int q2x = reinterpret_cast<const int*>(r)[8];
  X[0] = q0.x;
  Y[0] = q0.y;
  X[1] = q0.z;
  Y[1] = q0.w;
  X[2] = q1.x;
  Y[2] = q1.y;
  iw[0] = __int_as_float(q1.z);
  iw[1] = __int_as_float(q1.w);
  iw[2] = __int_as_float(q2x);
}

// Set-up fields stored in the record by the geometry phase.
__device__ __forceinline__ void load_setup(const Record* r, float& fA, uint2& box) {
  const int4 q2 = reinterpret_cast<const int4*>(r)[2];
  fA = __int_as_float(q2.y);
  box = make_uint2(unsigned(q2.z), unsigned(q2.w));
}

// 32-bit fragment test for a "small" triangle: coordinates relative to vertex 0 keep every
// product below 2^30, so the integers equal the 64-bit ones bit for bit.
__device__ __forceinline__ unsigned long long fragment32(const int Xr[3], const int Yr[3], const float iw[3], float fA,
                                                         int tl, unsigned key, int ortho, int cxr, int cyr) {
  const int w0 = (cxr - Xr[1]) * (Yr[2] - Yr[1]) - (cyr - Yr[1]) * (Xr[2] - Xr[1]);
  const int w1 = (cxr - Xr[2]) * (Yr[0] - Yr[2]) - (cyr - Yr[2]) * (Xr[0] - Xr[2]);
  const int w2 = (cxr - Xr[0]) * (Yr[1] - Yr[0]) - (cyr - Yr[0]) * (Xr[1] - Xr[0]);
  if (!(w0 + (tl & 1) > 0 && w1 + ((tl >> 1) & 1) > 0 && w2 + ((tl >> 2) & 1) > 0)) return kEmpty;
  const float f0 = __int2float_rn(w0), f1 = __int2float_rn(w1), f2 = __int2float_rn(w2);
  const float s = __fadd_rn(__fadd_rn(__fmul_rn(f0, iw[0]), __fmul_rn(f1, iw[1])), __fmul_rn(f2, iw[2]));
  const float depth = ortho ? __fdiv_rn(s, fA) : __fdiv_rn(fA, s);
  return ((unsigned long long)__float_as_uint(depth) << 32) | key;
}

__device__ __forceinline__ const Record* rec_of(const Params& p, const Scratch& sc, unsigned key) {
  return sc.rec + (size_t)(key & 1u) * p.t_max + (key >> 1);
}

// Covered pixels of a large triangle on image row py, within its box columns [bx0, bx1]:
// edge e (vertex e+1 to vertex e+2) is w_e(px) = a * px + c with a = 256 dy, so its
// half-plane test w_e + tl_e > 0 holds on a half-line of px.  The float quotient lands
// within a pixel of the boundary (relative error ~2^-21 on values below 2^13 inside the
// box), and exact 64-bit tests of the neighbouring pixels settle it.  Returns
// lo | (hi + 1) << 16 (empty: lo > hi).
__device__ uint32_t row_span(const int X[3], const int Y[3], int tl, int py, int bx0, int bx1) {
  const int cy = 256 * py + 128;
  int lo = bx0, hi = bx1;
#pragma unroll
  for (int e = 0; e < 3; e++) {
    const int vs = e == 2 ? 0 : e + 1, ve = e == 0 ? 2 : e - 1;
    const long long dy = Y[ve] - Y[vs], dx = X[ve] - X[vs];
    const long long a = 256ll * dy;
    const long long ct = (128ll - X[vs]) * dy - (long long)(cy - Y[vs]) * dx + ((tl >> e) & 1);  // c + tl
    if (a > 0) {  // covered from the smallest px with a * px + ct > 0
      const float t = floorf(__fdividef(__ll2float_rn(-ct), __ll2float_rn(a))) + 1.0f;
      int q = int(fminf(fmaxf(t, float(bx0)), float(bx1 + 1)));
      for (int it = 0; it < 4 && q > bx0 && a * (q - 1) + ct > 0; it++) q--;
      for (int it = 0; it < 4 && q <= bx1 && !(a * q + ct > 0); it++) q++;
      lo = max(lo, q);
    } else if (a < 0) {  // covered up to the largest such px
      const float t = ceilf(__fdividef(__ll2float_rn(ct), __ll2float_rn(-a))) - 1.0f;
      int q = int(fminf(fmaxf(t, float(bx0 - 1)), float(bx1)));
      for (int it = 0; it < 4 && q < bx1 && a * (q + 1) + ct > 0; it++) q++;
      for (int it = 0; it < 4 && q >= bx0 && !(a * q + ct > 0); it++) q--;
      hi = min(hi, q);
    } else if (!(ct > 0)) {
      lo = bx1 + 1;
    }
  }
  if (lo > hi) lo = bx1 + 1, hi = bx1;
  return unsigned(lo) | (unsigned(hi + 1) << 16);
}

// Fills the span table of the image's large triangles (block-wide; the caller synchronises).
__device__ void big_spans(const Params& p, const CtaShared& sh, const Scratch& sc, uint32_t* spans) {
  const int H = sh.im.H, nb = sh.n_big;
  if ((long long)nb * H > kSpanCap) return;
  for (int idx = threadIdx.x; idx < nb * H; idx += blockDim.x) {
    const int b = idx / H, py = idx - b * H;
    const Record* r = rec_of(p, sc, sc.big[b]);
    float fA;
    uint2 box;
    load_setup(r, fA, box);
    const int by0 = int(box.y & 0xffff), by1 = int((box.y >> 16) & 0xfff);
    const int bx0 = int(box.x & 0xffff), bx1 = int(box.x >> 16);
    uint32_t v = unsigned(bx1 + 1) | (unsigned(bx1 + 1) << 16);  // empty
    if (py >= by0 && py <= by1) {
      int X[3], Y[3];
      float iw[3];
      load_tri(r, X, Y, iw);
      v = row_span(X, Y, (box.y >> 28) & 7, py, bx0, bx1);
    }
    spans[idx] = v;
  }
}

// kLight: the batch has a cone table (type-2, spot, lights can occur) or material emission.
// (The shadowed instances shade with shade_shadowed, below.)
template <bool kLight>
__device__ void shade(const CtaShared& sh, const float P[3], const float n[3], int mat, float rgb[3]) {
  const ImageInfo& im = sh.im;
  const float4 ma = *reinterpret_cast<const float4*>(sh.mat[mat]);
  float2 mb;  // shininess, emission
  if (kLight) mb = *reinterpret_cast<const float2*>(&sh.mat[mat][4]);
  else mb = make_float2(sh.mat[mat][4], 0.0f);
  const float m[5] = {ma.x, ma.y, ma.z, ma.w, mb.x};
  float Vv[3];
  if (im.ortho) {
    Vv[0] = 0.0f;
    Vv[1] = 0.0f;
    Vv[2] = 1.0f;
  } else {
    float rl = rsqrt_approx(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
    Vv[0] = -P[0] * rl;
    Vv[1] = -P[1] * rl;
    Vv[2] = -P[2] * rl;
  }
  // diffuse and specular irradiance summed over the lights, the albedo applied once:
  // rgb_k = scale * (m_k * (ambient_k + emission + sum E ndl) + sum E spec)
  float D = mb.y, S = 0.0f;
#pragma unroll
  for (int l = 0; l < kMaxLights; l++) {
    if (l >= im.n_lights) break;
    const float4 lq = *reinterpret_cast<const float4*>(im.lv[l]);
    float Lx, Ly, Lz, r, E;  // (Lx, Ly, Lz) * r is the unit vector to the light
    // point or spot (the other instances see only types 0 and 1: spot needs the cone table)
    if (kLight ? im.light_type != 1 : im.light_type == 0) {
      Lx = lq.x - P[0];
      Ly = lq.y - P[1];
      Lz = lq.z - P[2];
      r = rsqrt_approx(Lx * Lx + Ly * Ly + Lz * Lz);
      E = lq.w * (r * r);
      if (kLight && im.light_type == 2) {  // the spot cone: E *= t^2 (3 - 2t)
        const float4 sq = *reinterpret_cast<const float4*>(im.la[l]);
        const float t = __saturatef(fmaf(-(Lx * sq.x + Ly * sq.y + Lz * sq.z), r, sq.w));
        E *= t * t * (3.0f - 2.0f * t);
      }
    } else {
      Lx = lq.x;
      Ly = lq.y;
      Lz = lq.z;
      r = 1.0f;
      E = lq.w;
    }
    const float ndl = fmaxf(0.0f, (n[0] * Lx + n[1] * Ly + n[2] * Lz) * r);
    D = fmaf(E, ndl, D);
    if (ndl > 0.0f && m[3] != 0.0f) {
      const float H0 = fmaf(Lx, r, Vv[0]), H1 = fmaf(Ly, r, Vv[1]), H2 = fmaf(Lz, r, Vv[2]);
      const float h2 = H0 * H0 + H1 * H1 + H2 * H2;
      if (h2 > 0.0f) {
        const float ndh = fmaxf(0.0f, (n[0] * H0 + n[1] * H1 + n[2] * H2) * rsqrt_approx(h2));
        S = fmaf(E, m[3] * lobe_pow(ndh, m[4]), S);
      }
    }
  }
  rgb[0] = im.scale * fmaf(m[0], im.amb[0] + D, S);
  rgb[1] = im.scale * fmaf(m[1], im.amb[1] + D, S);
  rgb[2] = im.scale * fmaf(m[2], im.amb[2] + D, S);
}

// The image's grading (one thread, in the graded instances only, before a barrier that precedes
// the raster phase).  White balance, the rotation about the grey axis, saturation, contrast and
// brightness are each affine in the colour, so they compose into one map c -> A c + t, applied
// per pixel; the grain stays per pixel.
// Light l's shadow camera for this image (its thread, in the shadow instances only, after
// setup_image and before a barrier that precedes the raster phase): M = S V^-1 with
// V^-1 = [R^T | -R^T t], every product and sum rounded to nearest in index order, so the
// lookup below is the same fp32 computation wherever it runs.
__device__ void shadow_setup(const Params& p, const ImageInfo& im, ShadowInfo& sd, int l) {
  const float* V = im.V;
  float Wi[12];
  for (int i = 0; i < 3; i++) {
    for (int j = 0; j < 3; j++) Wi[i * 4 + j] = V[j * 4 + i];
    Wi[i * 4 + 3] = -__fadd_rn(__fadd_rn(__fmul_rn(V[0 * 4 + i], V[3]), __fmul_rn(V[1 * 4 + i], V[7])),
                               __fmul_rn(V[2 * 4 + i], V[11]));
  }
  for (int f = 0; f < kMaxShadowFaces; f++) {
    const size_t c = ((size_t)im.s * kMaxLights + l) * p.shadow_faces + f;
    const float* si = p.shadow_intr + c * 7;
    sd.cast[l][f] = f < p.shadow_faces && l < im.n_lights && si[0] != 0.0f;
    if (!sd.cast[l][f]) continue;
    const float* S = p.shadow_view + c * 12;
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 4; j++) {
        float r = __fadd_rn(__fadd_rn(__fmul_rn(S[i * 4 + 0], Wi[0 * 4 + j]), __fmul_rn(S[i * 4 + 1], Wi[1 * 4 + j])),
                            __fmul_rn(S[i * 4 + 2], Wi[2 * 4 + j]));
        sd.sm[l][f][j + 4 * i] = j == 3 ? __fadd_rn(r, S[i * 4 + 3]) : r;
      }
    for (int k = 0; k < 7; k++) sd.si[l][f][k] = si[k];
    sd.si[l][f][7] = 0.0f;
    sd.map_off[l][f] = (unsigned long long)c * p.shadow_res * p.shadow_res;
  }
  if (l == 0)
    for (int k = 0; k < 10; k++) sd.pcf[k] = kPcfFactor[k];
}

// The shadowed taps k (0..9) of light l at the G-buffer position P (whose three coordinates the
// resolve computes with separately rounded operations).  P is projected into the light's maps
// with round-to-nearest operations in a fixed order: each row of the projection and each image
// coordinate as fused multiply-adds, one rounding each (the reciprocal is correctly rounded, so it
// equals 1 / z); the first casting face whose map contains the projection decides, and the 3 x 3
// texels around it are compared with the point's depth less the bias.  The neighbourhood table
// settles lit points and points behind every occupied tap in one or two loads; the others count
// the taps.  A point that no face contains has k = 0.
__device__ __forceinline__ int shadow_lookup_one(const Params& p, const ImageInfo& im, const ShadowInfo& sd,
                                                 float P0, float P1, float P2, int l) {
  const int R = p.shadow_res, F = p.shadow_faces;
  for (int f = 0; f < F; f++) {  // the first casting face whose map contains the point decides
    if (!sd.cast[l][f]) continue;
    const float4* M4 = reinterpret_cast<const float4*>(sd.sm[l][f]);
    const float4 ma = M4[0], mb = M4[1], mc = M4[2];
    const float4 sa = reinterpret_cast<const float4*>(sd.si[l][f])[0];  // fx, fy, cx, cy
    const float4 sb = reinterpret_cast<const float4*>(sd.si[l][f])[1];  // near, bias, type
    // each row as three fused multiply-adds, the translation first (one rounding each)
    const float q2 = __fmaf_rn(mc.z, P2, __fmaf_rn(mc.y, P1, __fmaf_rn(mc.x, P0, mc.w)));
    const float z = -q2;
    if (!(z > sb.x)) continue;
    const float q0 = __fmaf_rn(ma.z, P2, __fmaf_rn(ma.y, P1, __fmaf_rn(ma.x, P0, ma.w)));
    const float q1 = __fmaf_rn(mb.z, P2, __fmaf_rn(mb.y, P1, __fmaf_rn(mb.x, P0, mb.w)));
    const bool ortho = sb.z != 0.0f;  // (orthographic: a directional light's camera)
    const float iw = ortho ? 1.0f : __frcp_rn(z);
    const float u = __fmaf_rn(sa.x, ortho ? q0 : __fmul_rn(q0, iw), sa.z);
    const float v = __fmaf_rn(-sa.y, ortho ? q1 : __fmul_rn(q1, iw), sa.w);
    if (!(fabsf(u) < kGuardPx) || !(fabsf(v) < kGuardPx)) continue;
    const int i0 = int(floorf(u)), j0 = int(floorf(v));
    if (i0 < 0 || j0 < 0 || i0 >= R || j0 >= R) continue;
    const float zb = __fsub_rn(z, sb.y);
    const size_t m0 = sd.map_off[l][f];
    int k = -1;
    if (p.shadow_nb) {  // one entry settles lit points and those behind every occupied tap
      const size_t t = m0 + (size_t)j0 * R + i0;
      const unsigned e = __ldg(p.shadow_nb + t);
      const float lo = __half2float(__ushort_as_half((unsigned short)(e & 0xffffu)));
      const float hi = __half2float(__ushort_as_half((unsigned short)(e >> 16)));
      if (!(zb > lo)) k = 0;  // no occupied tap is nearer than the point
      else if (zb > hi) k = __ldg(p.shadow_cnt + t);  // every occupied tap is nearer
    }
    if (k < 0) {
      k = 0;
      const float* map = p.shadow_map + m0;
      const bool col[3] = {i0 - 1 >= 0, true, i0 + 1 < R};
#pragma unroll
      for (int bb = -1; bb <= 1; bb++) {
        const int jj = j0 + bb;
        if (jj < 0 || jj >= R) continue;
        const float* row = map + jj * R + i0;  // (within a map, offsets fit 32 bits)
#pragma unroll
        for (int aa = -1; aa <= 1; aa++) {
          if (!col[aa + 1]) continue;
          const float d = __ldg(row + aa);
          k += d > 0.0f && zb > d;
        }
      }
    }
    return k;
  }
  return 0;
}

// The cone of spot light l in view space (its thread, in the spot instances only, after
// setup_image and before a barrier that precedes the raster phase).
__device__ void spot_setup(const Params& p, ImageInfo& im, int l) {
  if (im.light_type != 2 || l >= im.n_lights) return;
  const float* sp = p.light_spot + (im.s * kMaxLights + l) * 5;
  const float cos_o = sp[3], cos_i = sp[4];
  const bool cone = cos_i > cos_o;
  const float w = cone ? 1.0f / (cos_i - cos_o) : 0.0f;
  for (int i = 0; i < 3; i++)
    im.la[l][i] = (im.V[i * 4 + 0] * sp[0] + im.V[i * 4 + 1] * sp[1] + im.V[i * 4 + 2] * sp[2]) * w;
  im.la[l][3] = cone ? -cos_o * w : -1.0f;
}

__device__ void grading_setup(const Params& p, ImageInfo& im) {
  const float* g = p.grading + (size_t)im.s * 8;
  grading_map(g, im.gm);
  im.grain = g[6];
  im.grain_key = grain_key(g, unsigned(im.cam - p.cam_offset[im.s]));
}

// Colour grading of one pixel's linear colour (see orrb_batch_desc::grading); `pixel` is the
// pixel's index within its image.  The grain is the PCG hash of the image's key and the
// pixel index, scaled to [0, 1).
__device__ __forceinline__ void grade(const ImageInfo& im, unsigned pixel, float c[3]) {
  const float o = im.grain * grain_centred(im.grain_key, pixel);
  const float r = c[0], g = c[1], b = c[2];
#pragma unroll
  for (int i = 0; i < 3; i++) c[i] = fmaf(im.gm[i][0], r, fmaf(im.gm[i][1], g, fmaf(im.gm[i][2], b, im.gm[i][3] + o)));
}

// floor(clamp(v, 0, 1) * 255 + 0.5) with one rounding of the multiply-add (NaN -> 0)
__device__ __forceinline__ uint8_t quantise(float v) { return (uint8_t)__float2uint_rd(fmaf(__saturatef(v), 255.0f, 0.5f)); }


// Walks the pixels of a box (px0, py0, width bw) with index j = lane, lane+32, ...
// Shading in the shadowed instances, returning the G-buffer word (slot | k of light l << (8 + 4l)).
// Each light's lookup sits inside the light loop, and the loop is not unrolled: unrolled over four
// lights, the inlined lookups made the kernel's code large enough for instruction fetch to stall
// warps.  The arithmetic is that of shade<true>, with E scaled by the factor (9 - k) / 9 from a table.
__device__ int shade_shadowed(const Params& p, const CtaShared& sh, const ShadowInfo& sd, const float P[3],
                              const float n[3], int mat, float rgb[3]) {
  const ImageInfo& im = sh.im;
  const float4 ma = *reinterpret_cast<const float4*>(sh.mat[mat]);
  const float2 mb = *reinterpret_cast<const float2*>(&sh.mat[mat][4]);
  const float m[5] = {ma.x, ma.y, ma.z, ma.w, mb.x};
  float Vv[3];
  if (im.ortho) {
    Vv[0] = 0.0f;
    Vv[1] = 0.0f;
    Vv[2] = 1.0f;
  } else {
    float rl = rsqrt_approx(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
    Vv[0] = -P[0] * rl;
    Vv[1] = -P[1] * rl;
    Vv[2] = -P[2] * rl;
  }
  int word = mat;
  float D = mb.y, S = 0.0f;
#pragma unroll 1
  for (int l = 0; l < im.n_lights && l < kMaxLights; l++) {
    const int k = shadow_lookup_one(p, im, sd, P[0], P[1], P[2], l);
    word |= k << (8 + 4 * l);
    const float4 lq = *reinterpret_cast<const float4*>(im.lv[l]);
    float Lx, Ly, Lz, r, E;
    if (im.light_type != 1) {
      Lx = lq.x - P[0];
      Ly = lq.y - P[1];
      Lz = lq.z - P[2];
      r = rsqrt_approx(Lx * Lx + Ly * Ly + Lz * Lz);
      E = lq.w * (r * r);
      if (im.light_type == 2) {
        const float4 sq = *reinterpret_cast<const float4*>(im.la[l]);
        const float t = __saturatef(fmaf(-(Lx * sq.x + Ly * sq.y + Lz * sq.z), r, sq.w));
        E *= t * t * (3.0f - 2.0f * t);
      }
    } else {
      Lx = lq.x;
      Ly = lq.y;
      Lz = lq.z;
      r = 1.0f;
      E = lq.w;
    }
    E *= sd.pcf[k];
    const float ndl = fmaxf(0.0f, (n[0] * Lx + n[1] * Ly + n[2] * Lz) * r);
    D = fmaf(E, ndl, D);
    if (ndl > 0.0f && m[3] != 0.0f) {
      const float H0 = fmaf(Lx, r, Vv[0]), H1 = fmaf(Ly, r, Vv[1]), H2 = fmaf(Lz, r, Vv[2]);
      const float h2 = H0 * H0 + H1 * H1 + H2 * H2;
      if (h2 > 0.0f) {
        const float ndh = fmaxf(0.0f, (n[0] * H0 + n[1] * H1 + n[2] * H2) * rsqrt_approx(h2));
        S = fmaf(E, m[3] * lobe_pow(ndh, m[4]), S);
      }
    }
  }
  rgb[0] = im.scale * fmaf(m[0], im.amb[0] + D, S);
  rgb[1] = im.scale * fmaf(m[1], im.amb[1] + D, S);
  rgb[2] = im.scale * fmaf(m[2], im.amb[2] + D, S);
  return word;
}

struct BoxWalk {
  int px, py;
  __device__ __forceinline__ BoxWalk(int j, int px0, int py0, int bw) {
    const int dy = j < bw ? 0 : j / bw;
    px = px0 + (j - dy * bw);
    py = py0 + dy;
  }
};

// Phase R for one tile, by one warp, in warp-private shared memory.
// kF: the batch's optional features (kFeatGrade, kFeatTrack, kFeatLight); each combination is a
// kernel instance of its own, so that the common case carries none of their code.
template <int kF>
__device__ void raster_tile_warp(const Params& p, const CtaShared& sh, const Scratch& sc, int tile, char* wbase,
                                 const SmemLayout& L, const uint32_t* spans) {
  constexpr bool kGrade = (kF & kFeatGrade) != 0, kShadow = (kF & kFeatShadow) != 0;
  constexpr bool kPass = (kF & kFeatShadowPass) != 0;
  const ImageInfo& im = sh.im;
  const int lane = threadIdx.x & 31;
  const int tx = tile % im.ntx, ty = tile / im.ntx;
  const int x0 = tx * im.tw, y0 = ty * im.th;
  const int cw = min(im.tw, im.W - x0), ch = min(im.th, im.H - y0);
  const int npx = cw * ch;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(wbase + L.w_keys);
  for (int i = lane; i < npx; i += 32) keys[i] = kEmpty;
  __syncwarp();

  // large triangles: with the image's span table, the lanes walk only the covered pixels
  // of each row, one each; without it (too many triangle rows), they split the triangle's
  // box within the tile and test every pixel
  const int nbig = sh.n_big;
  const bool with_spans = (long long)nbig * im.H <= kSpanCap;
  for (int b = 0; b < nbig; b++) {
    const unsigned key = sc.big[b];
    int X[3], Y[3];
    float iw[3];
    const Record* rb = rec_of(p, sc, key);
    float fA;
    uint2 box;
    load_setup(rb, fA, box);
    const int bx0 = max(x0, int(box.x & 0xffff)), bx1 = min(x0 + cw - 1, int(box.x >> 16));
    const int by0 = max(y0, int(box.y & 0xffff)), by1 = min(y0 + ch - 1, int((box.y >> 16) & 0xfff));
    if (bx0 > bx1 || by0 > by1) continue;
    load_tri(rb, X, Y, iw);
    const int tl = (box.y >> 28) & 7;
    // the lane's pixels are px0 + lane + 32k, so each edge function advances by a constant
    // 32 * 256 * dy between them (exact 64-bit integer steps)
    const long long s0 = 8192ll * (Y[2] - Y[1]), s1 = 8192ll * (Y[0] - Y[2]), s2 = 8192ll * (Y[1] - Y[0]);
    for (int py = by0; py <= by1; py++) {
      int lo = bx0, hi = bx1;
      if (with_spans) {
        const uint32_t v = spans[b * im.H + py];
        lo = max(lo, int(v & 0xffff));
        hi = min(hi, int(v >> 16) - 1);
      }
      int px = lo + lane;
      if (px > hi) continue;
      const int cx = 256 * px + 128, cy = 256 * py + 128;
      long long w0 = (long long)(cx - X[1]) * (Y[2] - Y[1]) - (long long)(cy - Y[1]) * (X[2] - X[1]);
      long long w1 = (long long)(cx - X[2]) * (Y[0] - Y[2]) - (long long)(cy - Y[2]) * (X[0] - X[2]);
      long long w2 = (long long)(cx - X[0]) * (Y[1] - Y[0]) - (long long)(cy - Y[0]) * (X[1] - X[0]);
      unsigned long long* krow = keys + (py - y0) * cw - x0;
      for (; px <= hi; px += 32) {
        if (with_spans || (w0 + (tl & 1) > 0 && w1 + ((tl >> 1) & 1) > 0 && w2 + ((tl >> 2) & 1) > 0)) {
          const float f0 = __ll2float_rn(w0), f1 = __ll2float_rn(w1), f2 = __ll2float_rn(w2);
          const float sum = __fadd_rn(__fadd_rn(__fmul_rn(f0, iw[0]), __fmul_rn(f1, iw[1])), __fmul_rn(f2, iw[2]));
          const float depth = im.ortho ? __fdiv_rn(sum, fA) : __fdiv_rn(fA, sum);
          const unsigned long long f = ((unsigned long long)__float_as_uint(depth) << 32) | key;
          if (f < krow[px]) krow[px] = f;
        }
        w0 += s0;
        w1 += s1;
        w2 += s2;
      }
    }
    __syncwarp();
  }

  // binned triangles: 32 at a time, their clamped boxes prefix-summed and the
  // (triangle, pixel) candidates spread evenly over the lanes.  Triangles with candidates
  // are staged compacted, so candidate m belongs to staged triangle (number of starts <= m) - 1;
  // per chunk of 32 candidates that count is a ballot of the starts up to the chunk plus the
  // bits of the starts inside it (distinct, since every staged triangle has a candidate).
  WarpTri* wt = reinterpret_cast<WarpTri*>(wbase + L.w_tri);
  const int b0 = sc.tile_off[2 * tile], b1 = sc.tile_off[2 * tile + 1];
  for (int c = b0; c < b1; c += 32) {
    const int k = c + lane;
    int cnt = 0;
    WarpTri T;
    if (k < b1) {
      T.key = sc.bins[k];
      const Record* rb = rec_of(p, sc, T.key);
      uint2 box;
      load_setup(rb, T.fA, box);
      load_tri(rb, T.X, T.Y, T.iw);
      T.flags = (box.y >> 28) & 15;
      if (T.flags & 8) {  // small: relative to vertex 0 (exact 32-bit arithmetic)
        T.X[1] -= T.X[0];
        T.X[2] -= T.X[0];
        T.Y[1] -= T.Y[0];
        T.Y[2] -= T.Y[0];
      }
      T.px0 = max(x0, int(box.x & 0xffff));
      T.py0 = max(y0, int(box.y & 0xffff));
      int bw = min(x0 + cw - 1, int(box.x >> 16)) - T.px0 + 1;
      const int bh = min(y0 + ch - 1, int((box.y >> 16) & 0xfff)) - T.py0 + 1;
      if (ch <= 2 && bw > 0 && bh > 0) {
        // tiles of one or two rows: each row's candidates form one run of columns; for a small
        // triangle, only the columns whose centres lie within 2/256 px of its extent along the
        // row (float, relative to vertex 0, where every coordinate is exact and each crossing is
        // within 0.02/256 px); the exact edge test still decides every candidate
        int a0 = T.px0, n0 = bw, a1 = T.px0, n1 = bh == 2 ? bw : 0;
        if (T.flags & 8) {
          const float cy0 = float(256 * T.py0 + 128 - T.Y[0]), cy1 = cy0 + 256.0f;
          const float vx[3] = {0.0f, float(T.X[1]), float(T.X[2])}, vy[3] = {0.0f, float(T.Y[1]), float(T.Y[2])};
          float xl0 = 3.0e38f, xr0 = -3.0e38f, xl1 = 3.0e38f, xr1 = -3.0e38f;
#pragma unroll
          for (int e = 0; e < 3; e++) {
            const int e2 = e == 2 ? 0 : e + 1;
            const float ya = vy[e], yb = vy[e2], xa = vx[e], xb = vx[e2];
            const float ylo = fminf(ya, yb), yhi = fmaxf(ya, yb);
            const bool flat = ya == yb;
            const float slope = flat ? 0.0f : __fdividef(xb - xa, yb - ya);
            const float x0e = fmaf(cy0 - ya, slope, xa), x1e = fmaf(cy1 - ya, slope, xa);
            const float lo0 = flat ? fminf(xa, xb) : x0e, hi0 = flat ? fmaxf(xa, xb) : x0e;
            const float lo1 = flat ? fminf(xa, xb) : x1e, hi1 = flat ? fmaxf(xa, xb) : x1e;
            const bool c0 = ylo <= cy0 && cy0 <= yhi, c1 = ylo <= cy1 && cy1 <= yhi;
            xl0 = c0 ? fminf(xl0, lo0) : xl0;
            xr0 = c0 ? fmaxf(xr0, hi0) : xr0;
            xl1 = c1 ? fminf(xl1, lo1) : xl1;
            xr1 = c1 ? fmaxf(xr1, hi1) : xr1;
          }
          const float cx0 = float(256 * T.px0 + 128 - T.X[0]);  // the box's first column centre, relative
          const int jl0 = max(0, int(ceilf((xl0 - 2.0f - cx0) * (1.0f / 256.0f))));
          const int jr0 = min(bw - 1, int(floorf((xr0 + 2.0f - cx0) * (1.0f / 256.0f))));
          const int jl1 = max(0, int(ceilf((xl1 - 2.0f - cx0) * (1.0f / 256.0f))));
          const int jr1 = min(bw - 1, int(floorf((xr1 + 2.0f - cx0) * (1.0f / 256.0f))));
          a0 = T.px0 + jl0;
          n0 = xl0 <= xr0 ? max(0, jr0 - jl0 + 1) : 0;
          a1 = T.px0 + jl1;
          n1 = bh == 2 && xl1 <= xr1 ? max(0, jr1 - jl1 + 1) : 0;
        }
        T.px0 = a0;
        T.bw = n0;
        T.px1 = a1;
        T.bw1 = n1;
        cnt = n0 + n1;
      } else {
        T.bw = bw;
        cnt = (bw > 0 && bh > 0) ? bw * bh : 0;
      }
    }
    const int slot = __popc(__ballot_sync(kFull, cnt > 0) & ((1u << lane) - 1u));
    if (cnt > 0) wt[slot] = T;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += v;
    }
    const int start = incl - cnt;
    const int total = __shfl_sync(kFull, incl, 31);
    if (cnt > 0) wt[slot].start = start;
    __syncwarp();
    for (int base = 0; base < total; base += 32) {
      const unsigned upto = __ballot_sync(kFull, cnt > 0 && start <= base);
      const unsigned inside =
          __reduce_or_sync(kFull, (cnt > 0 && start > base && start < base + 32) ? 1u << (start - base) : 0u);
      const int m = base + lane;
      if (m < total) {
        const WarpTri& W = wt[__popc(upto) + __popc(inside & (0xffffffffu >> (31 - lane))) - 1];
        const int j = m - W.start;
        BoxWalk w(0, 0, 0, 1);
        if (ch <= 2) {  // the first row's run, then the second row's
          const bool r1 = j >= W.bw;
          w.px = r1 ? W.px1 + (j - W.bw) : W.px0 + j;
          w.py = W.py0 + (r1 ? 1 : 0);
        } else {
          w = BoxWalk(j, W.px0, W.py0, W.bw);
        }
        const int tl = W.flags & 7;
        unsigned long long f;
        if (W.flags & 8) {
          const int Xr[3] = {0, W.X[1], W.X[2]}, Yr[3] = {0, W.Y[1], W.Y[2]};
          f = fragment32(Xr, Yr, W.iw, W.fA, tl, W.key, im.ortho, 256 * w.px + 128 - W.X[0], 256 * w.py + 128 - W.Y[0]);
        } else {
          f = fragment(W.X, W.Y, W.iw, W.fA, tl, W.key, im.ortho, 256 * w.px + 128, 256 * w.py + 128);
        }
        if (f != kEmpty) atomicMin(&keys[(w.py - y0) * cw + (w.px - x0)], f);
      }
    }
    __syncwarp();
  }

  // resolve + shade; every channel goes straight out, lane-consecutive pixels per row
  const long long N = p.total_pixels;
  for (int ly = 0; ly < ch; ly++) {
    const long long orow = im.px_off + (long long)(y0 + ly) * im.W + x0;
    const int py = y0 + ly;
    const float uy = -__fmul_rn(__fsub_rn(__fadd_rn(float(py), 0.5f), im.cy), im.inv_fy);  // (no contraction)
    uint8_t* rgb_row = p.rgb ? p.rgb + 3 * orow : nullptr;
    uint16_t* nrm_row = p.normal ? p.normal + 3 * orow : nullptr;
    float* depth_row = p.depth ? p.depth + orow : nullptr;
    uint8_t* seg_row = p.seg ? p.seg + orow : nullptr;
    const unsigned long long* krow = keys + ly * cw;
    unsigned last = 0xffffffffu;  // the lane's previous winner and its material/segment/normal word
    int4 last_q3 = make_int4(0, 0, 0, 0);
    for (int lx = lane; lx < cw; lx += 32) {
      const int px = x0 + lx;
      const unsigned long long kk = krow[lx];
      if (kPass) {  // the shadow pass: the map's depth only
        if (depth_row) __stcs(depth_row + lx, kk == kEmpty ? 0.0f : __uint_as_float(unsigned(kk >> 32)));
        continue;
      }
      float rgb[3], depth = 0.0f, n[3] = {0.0f, 0.0f, 0.0f}, P[3] = {0.0f, 0.0f, 0.0f};
      int mat = -1, seg = 0;
      int word = -1;  // the G-buffer's material word
      if (kk == kEmpty) {
        rgb[0] = im.bg[0];
        rgb[1] = im.bg[1];
        rgb[2] = im.bg[2];
      } else {
        depth = __uint_as_float(unsigned(kk >> 32));
        const Record* r = rec_of(p, sc, unsigned(kk));
        if (unsigned(kk) != last) {  // 32 pixels apart, a lane often meets the same (large) triangle again
          last = unsigned(kk);
          last_q3 = reinterpret_cast<const int4*>(r)[3];
        }
        const int4 q3 = last_q3;
        mat = q3.x & 0xffff;
        seg = (q3.x >> 16) & 0xff;
        if (q3.x & (1 << 24)) {  // flat face: the normalised interpolated normal is the (unit) vertex normal
          n[0] = __int_as_float(q3.y);
          n[1] = __int_as_float(q3.z);
          n[2] = __int_as_float(q3.w);
        } else {
          const int4 q0 = reinterpret_cast<const int4*>(r)[0];
          const int4 q1 = reinterpret_cast<const int4*>(r)[1];
          const float iw2 = reinterpret_cast<const float*>(r)[8];
          const float4 q4 = reinterpret_cast<const float4*>(r)[4];
          const float2 q5 = reinterpret_cast<const float2*>(r)[10];
          const int cx = 256 * px + 128, cy = 256 * py + 128;
          float a0 = float(cx - q0.z) * float(q1.y - q0.w) - float(cy - q0.w) * float(q1.x - q0.z);
          float a1 = float(cx - q1.x) * float(q0.y - q1.y) - float(cy - q1.y) * float(q0.x - q1.x);
          float a2 = float(cx - q0.x) * float(q0.w - q0.y) - float(cy - q0.y) * float(q0.z - q0.x);
          if (!im.ortho) {
            a0 *= __int_as_float(q1.z);
            a1 *= __int_as_float(q1.w);
            a2 *= iw2;
          }
          n[0] = a0 * __int_as_float(q3.y) + a1 * q4.x + a2 * q4.w;
          n[1] = a0 * __int_as_float(q3.z) + a1 * q4.y + a2 * q5.x;
          n[2] = a0 * __int_as_float(q3.w) + a1 * q4.z + a2 * q5.y;
          const float l2 = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
          if (l2 > 0.0f) {
            const float rl = rsqrt_approx(l2);
            n[0] *= rl;
            n[1] *= rl;
            n[2] *= rl;
          }
        }
        // the G-buffer position, each operation rounded separately (the shadow lookup relies on it)
        const float ux = __fmul_rn(__fsub_rn(__fadd_rn(float(px), 0.5f), im.cx), im.inv_fx);
        if (im.ortho) {
          P[0] = ux;
          P[1] = uy;
          P[2] = -depth;
        } else {
          P[0] = __fmul_rn(depth, ux);
          P[1] = __fmul_rn(depth, uy);
          P[2] = -depth;
        }
        if (kShadow) {
          const ShadowInfo& sd = *reinterpret_cast<const ShadowInfo*>(spans + kSpanCap);
          word = shade_shadowed(p, sh, sd, P, n, mat, rgb);
        } else {
          shade<(kF & kFeatLight) != 0>(sh, P, n, mat, rgb);
        }
      }
      // consecutive lanes write consecutive pixels: the three byte (or half) stores of a
      // warp fill whole sectors of the row between them
      // (explicit global streaming stores: outputs are not re-read, and the compiler need not
      // assume they alias the shared-memory light and material tables)
      if (kGrade && (rgb_row || p.rgb_graded)) {
        float gc[3] = {rgb[0], rgb[1], rgb[2]};
        grade(im, unsigned(py * im.W + px), gc);
        if (rgb_row) {
          __stcs(rgb_row + 3 * lx + 0, quantise(gc[0]));
          __stcs(rgb_row + 3 * lx + 1, quantise(gc[1]));
          __stcs(rgb_row + 3 * lx + 2, quantise(gc[2]));
        }
        if (p.rgb_graded) {  // the graded colour before clamping (the input of a graded loss)
          float* o3 = p.rgb_graded + 3 * (orow + lx);
          __stcs(o3 + 0, gc[0]);
          __stcs(o3 + 1, gc[1]);
          __stcs(o3 + 2, gc[2]);
        }
      } else {
        if (rgb_row) {
          __stcs(rgb_row + 3 * lx + 0, quantise(rgb[0]));
          __stcs(rgb_row + 3 * lx + 1, quantise(rgb[1]));
          __stcs(rgb_row + 3 * lx + 2, quantise(rgb[2]));
        }
        if (p.rgb_graded) {  // (an ungraded batch: the graded colour is the linear colour)
          float* o3 = p.rgb_graded + 3 * (orow + lx);
          __stcs(o3 + 0, rgb[0]);
          __stcs(o3 + 1, rgb[1]);
          __stcs(o3 + 2, rgb[2]);
        }
      }
      if (nrm_row) {
        const __half2 h01 = __floats2half2_rn(n[0], n[1]);
        __stcs(nrm_row + 3 * lx + 0, __half_as_ushort(__low2half(h01)));
        __stcs(nrm_row + 3 * lx + 1, __half_as_ushort(__high2half(h01)));
        __stcs(nrm_row + 3 * lx + 2, __half_as_ushort(__float2half_rn(n[2])));
      }
      if (depth_row) __stcs(depth_row + lx, depth);
      if (seg_row) __stcs(seg_row + lx, (uint8_t)seg);
      if (p.rgb_linear) {
        float* o3 = p.rgb_linear + 3 * (orow + lx);
        __stcs(o3 + 0, rgb[0]);
        __stcs(o3 + 1, rgb[1]);
        __stcs(o3 + 2, rgb[2]);
      }
      if (p.gbuffer) {
        const long long o = orow + lx;
        __stcs(p.gbuffer + 0 * N + o, P[0]);
        __stcs(p.gbuffer + 1 * N + o, P[1]);
        __stcs(p.gbuffer + 2 * N + o, P[2]);
        __stcs(p.gbuffer + 3 * N + o, n[0]);
        __stcs(p.gbuffer + 4 * N + o, n[1]);
        __stcs(p.gbuffer + 5 * N + o, n[2]);
        __stcs(p.gbuffer + 6 * N + o, __int_as_float(kShadow ? word : mat));
      }
    }
  }
  __syncwarp();
}

// The owner's prepared image state (camera, lights, materials, grading, spot cones, the large
// triangles' row spans, shadow cameras) into its slot, every thread a share of the 16-byte words,
// each fencing its own writes before the barrier that precedes the opening of the raster phase.
template <bool kShadow>
__device__ void publish_image(const CtaShared& sh, const SmemPtrs& sp, char* pub) {
  PubImage* g = reinterpret_cast<PubImage*>(pub);
  const int tid = threadIdx.x, nt = blockDim.x;
  auto copy = [&](int4* dst, const int4* src, int n) {
    for (int i = tid; i < n; i += nt) dst[i] = src[i];
  };
  copy(reinterpret_cast<int4*>(&g->im), reinterpret_cast<const int4*>(&sh.im), int(sizeof(ImageInfo) / 16));
  copy(reinterpret_cast<int4*>(g->mat), reinterpret_cast<const int4*>(sh.mat), int(sizeof(g->mat) / 16));
  copy(reinterpret_cast<int4*>(g->spans), reinterpret_cast<const int4*>(sp.spans), kSpanCap / 4);
  if (kShadow)
    copy(reinterpret_cast<int4*>(&g->sd), reinterpret_cast<const int4*>(sp.spans + kSpanCap), int(sizeof(ShadowInfo) / 16));
  if (tid == 0) g->n_big = sh.n_big;
  __threadfence();
}

// A helper takes the published state of the image it joins (loads that bypass L1: the slot was
// written by another SM and may have held an earlier image).
template <bool kShadow>
__device__ void take_published(CtaShared& sh, const SmemPtrs& sp, const char* pub) {
  const PubImage* g = reinterpret_cast<const PubImage*>(pub);
  const int tid = threadIdx.x, nt = blockDim.x;
  auto copy = [&](int4* dst, const int4* src, int n) {
    for (int i = tid; i < n; i += nt) dst[i] = __ldcg(src + i);
  };
  copy(reinterpret_cast<int4*>(&sh.im), reinterpret_cast<const int4*>(&g->im), int(sizeof(ImageInfo) / 16));
  copy(reinterpret_cast<int4*>(sh.mat), reinterpret_cast<const int4*>(g->mat), int(sizeof(g->mat) / 16));
  copy(reinterpret_cast<int4*>(sp.spans), reinterpret_cast<const int4*>(g->spans), kSpanCap / 4);
  if (kShadow)
    copy(reinterpret_cast<int4*>(sp.spans + kSpanCap), reinterpret_cast<const int4*>(&g->sd), int(sizeof(ShadowInfo) / 16));
  if (tid == 0) sh.n_big = __ldcg(&g->n_big);
}

// Phase R for the current image: warps pull tiles first, first + stride, ... from the
// CTA's counter until none is left.
template <int kF>
__device__ void raster_phase(const Params& p, CtaShared& sh, const Scratch& sc, const SmemPtrs& sp, const SmemLayout& L,
                             int first = 0, int stride = 1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  char* wbase = sp.uni + (size_t)warp * L.w_bytes;
  while (true) {
    int k = 0;
    if (lane == 0) k = atomicAdd(&sh.next_tile, 1);
    const int t = first + stride * __shfl_sync(kFull, k, 0);
    if (t >= sh.im.n_tiles) break;
    raster_tile_warp<kF>(p, sh, sc, t, wbase, L, sp.spans);
  }
  __syncthreads();
}

__device__ inline SmemLayout layout_of(const Params& p) {
  return smem_layout(blockDim.x, p.tile_w, p.tile_h, p.inst_max, p.max_tiles, p.w_max,
                     p.shadow_res > 0 && !p.shadow_pass);
}

__device__ inline SmemPtrs carve(char* smem, const Params& p, const SmemLayout& L) {
  SmemPtrs s;
  s.mprefix = reinterpret_cast<int*>(smem);
  s.tprefix = s.mprefix + (p.inst_max + 2);
  s.mbegin = s.tprefix + (p.inst_max + 2);
  s.uni = smem + L.uni;
  s.spans = reinterpret_cast<uint32_t*>(smem + L.spans);
  return s;
}

// Bounded waits: a spin that exceeds p.wait_cycles SM cycles (by default about a second) sets
// ORRB_DEV_TIMEOUT and gives up instead of hanging.

// Raster tiles of the image whose claim word is `claim`, for camera `cam`.  The owner of
// the slot claims with atomicAdd and counts its own tiles in shared memory (its CTA wrote
// the records, so it needs no fence); a helper claims with compare-and-swap, so it never
// takes a tile of a later image that reused the slot, and publishes each finished tile
// in the slot's counter after a fence.
template <int kF>
__device__ void raster_claimed(const Params& p, CtaShared& sh, const Scratch& sc, const SmemPtrs& sp, const SmemLayout& L,
                               int cam, bool owner) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  char* wbase = sp.uni + (size_t)warp * L.w_bytes;
  unsigned long long* word = sc.claim();
  const unsigned long long tag = (unsigned long long)(cam + 1) << 32;
  const int n_tiles = sh.im.n_tiles;
  int mine = 0;
  unsigned long long next = 0;  // the owner claims its next tile before rastering the current one
  if (owner && lane == 0) next = atomicAdd(word, 1ull);
  while (true) {
    int t = 0;
    if (lane == 0) {
      if (owner) {
        t = int(unsigned(next));
        if (t < n_tiles) next = atomicAdd(word, 1ull);
      } else {
        t = n_tiles;
        unsigned long long w = atomicAdd(word, 0ull);
        while ((w & ~0xffffffffull) == tag && int(unsigned(w)) < n_tiles) {
          const unsigned long long seen = atomicCAS(word, w, w + 1);
          if (seen == w) {
            t = int(unsigned(w));
            break;
          }
          w = seen;
        }
      }
    }
    t = __shfl_sync(kFull, t, 0);
    if (t >= n_tiles) break;
    raster_tile_warp<kF>(p, sh, sc, t, wbase, L, sp.spans);
    mine++;
    if (!owner && lane == 0) {
      __threadfence();
      if (atomicAdd(reinterpret_cast<unsigned*>(sc.header + 4), 1u) + 1u == unsigned(n_tiles))
        atomicAdd(p.images_done, 1u);  // the image's last tile (the owner has added its own)
    }
  }
  if (owner && lane == 0) atomicAdd(&sh.next_tile, mine);  // the owner's own count (shared memory)
  __syncthreads();
}

// ---------------------------------------------------------------------------
// fused: one persistent launch.  CTAs pull whole images from a queue; once the
// queue is empty they help finish the raster phase of images other CTAs still own.
// ---------------------------------------------------------------------------
template <int kF>
__global__ void __launch_bounds__(512, 2) render_fused_kernel(Params p) {
  constexpr bool kGrade = (kF & kFeatGrade) != 0, kTrack = (kF & kFeatTrack) != 0, kLight = (kF & kFeatLight) != 0;
  constexpr bool kShadow = (kF & kFeatShadow) != 0, kPass = (kF & kFeatShadowPass) != 0;
  extern __shared__ __align__(16) char smem[];
  __shared__ CtaShared sh;
  const SmemLayout L = layout_of(p);
  SmemPtrs sp = carve(smem, p, L);
  const Scratch sc = slot_scratch(p, blockIdx.x);
  if (threadIdx.x == 0) {
    sh.stop = 0;
    sh.img = atomicAdd(p.work_counter, 1);
  }
  while (true) {
    __syncthreads();
    const int cam = sh.img;
    if (cam >= p.n_cams) break;
    setup_image<kPass>(p, cam, sh, sp.mprefix, sp.tprefix, sp.mbegin, true, kTrack);
    if (kGrade && threadIdx.x == 0 && sh.im.valid) grading_setup(p, sh.im);  // (read after phase G's barrier)
    if (kLight && threadIdx.x < kMaxLights && sh.im.valid) spot_setup(p, sh.im, threadIdx.x);
    if (kShadow && threadIdx.x < kMaxLights && sh.im.valid)
      shadow_setup(p, sh.im, *reinterpret_cast<ShadowInfo*>(sp.spans + kSpanCap), threadIdx.x);
    if (sh.im.valid) {
      geometry_phase<kTrack, kPass>(p, sh, sp.mprefix, sp.tprefix, sp.mbegin, reinterpret_cast<WarpG*>(sp.uni), sc);
      __syncthreads();
      int* counts = p.max_tiles > kSmemCountTiles ? sc.counts : reinterpret_cast<int*>(sp.uni);
      bin_phase(p, sh, counts, counts + (p.max_tiles + 2), sc);
      big_spans(p, sh, sc, sp.spans);
      __syncthreads();  // (the span table is complete)
      publish_image<kShadow>(sh, sp, sc.pub);
      if (threadIdx.x == 0) {
        sc.header[3] = sh.n_big;
        sc.header[4] = 0;
        sc.header[5] = sh.im.n_tiles;
        sc.header[6] = 0;
        sh.next_tile = 0;
      }
      __syncthreads();  // (every thread fenced its part of the published state)
      if (threadIdx.x == 0) {  // open the raster phase to helpers
        __threadfence();
        atomicExch(sc.claim(), (unsigned long long)(cam + 1) << 32);
      }
      __syncthreads();
      raster_claimed<kF>(p, sh, sc, sp, L, cam, true);
      if (threadIdx.x == 0) {
        // close the raster phase and add the own tiles to the slot's finished-tile count; whoever
        // brings that count to the image's tile count (owner or helper) counts the image done
        atomicExch(sc.claim(), 0ull);
        const unsigned n_tiles = unsigned(sh.im.n_tiles), mine = unsigned(sh.next_tile);
        __threadfence();
        // (with no own tile, helpers took every tile and the last of them counted the image)
        if (mine > 0 && atomicAdd(reinterpret_cast<unsigned*>(sc.header + 4), mine) + mine == n_tiles)
          atomicAdd(p.images_done, 1u);
        // the next image, popped before deciding whether to wait: only a CTA that reuses its slot
        // waits for the helpers still on its other tiles; once the queue is empty it goes on to
        // help other images at once (helpers exist only after the queue has emptied)
        sh.img = atomicAdd(p.work_counter, 1);
        const long long t0 = clock64();
        while (sh.img < p.n_cams && atomicAdd(reinterpret_cast<unsigned*>(sc.header + 4), 0u) < n_tiles) {
          if (clock64() - t0 > p.wait_cycles) {
            // a helper may still be reading this slot: the CTA leaves the launch, so that the
            // slot is never rewritten under it
            flag_status(p, ORRB_DEV_TIMEOUT);
            sh.stop = 1;
            break;
          }
          __nanosleep(200);
        }
      }
    } else if (threadIdx.x == 0) {  // an image that is not rendered (its status bits are set)
      __threadfence();
      atomicAdd(p.images_done, 1u);
      sh.img = atomicAdd(p.work_counter, 1);
    }
    __syncthreads();
    if (sh.stop) return;
  }
  // helper mode: join an open raster phase, until every image is done.  Every thread scores a
  // share of the slots by the tiles left per helper that already joined, so idle CTAs spread over
  // the open images instead of all choosing the same one.
  long long t0 = clock64();  // start of the current search (thread 0); reset whenever work is found
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  while (true) {
    float best_score = 0.0f;
    int best = -1;
    for (int s = threadIdx.x; s < p.n_slots; s += blockDim.x) {
      const int* h = reinterpret_cast<const int*>(p.scratch + size_t(s) * p.slot_bytes);  // (the header leads the slot)
      const unsigned long long w = *reinterpret_cast<const volatile unsigned long long*>(h);
      if (w == 0ull) continue;
      const int left = *reinterpret_cast<const volatile int*>(h + 5) - int(unsigned(w));
      if (left <= 0) continue;
      const float score = float(left) / float(1 + *reinterpret_cast<const volatile int*>(h + 6));
      if (score > best_score) {
        best_score = score;
        best = s;
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const float os = __shfl_down_sync(kFull, best_score, off);
      const int ob = __shfl_down_sync(kFull, best, off);
      if (os > best_score) {
        best_score = os;
        best = ob;
      }
    }
    if (lane == 0) {
      sh.red_score[warp] = best_score;
      sh.red_slot[warp] = best;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      best_score = 0.0f;
      best = -1;
      for (int k = 0; k < int(blockDim.x >> 5); k++)
        if (sh.red_score[k] > best_score) {
          best_score = sh.red_score[k];
          best = sh.red_slot[k];
        }
      int cam = -1;
      if (best >= 0) {
        int* h = reinterpret_cast<int*>(p.scratch + size_t(best) * p.slot_bytes);
        const unsigned long long w = *reinterpret_cast<volatile unsigned long long*>(h);
        cam = int(w >> 32) - 1;  // 0 -> -1: closed meanwhile, search again
        if (cam < 0) best = -1;
        else atomicAdd(h + 6, 1);
      }
      if (best >= 0) {
        t0 = clock64();
      } else {
        if (*reinterpret_cast<volatile unsigned*>(p.images_done) >= unsigned(p.n_cams)) cam = -2;
        else if (clock64() - t0 > p.wait_cycles) {
          flag_status(p, ORRB_DEV_TIMEOUT);
          cam = -2;
        } else {
          __nanosleep(500);
        }
      }
      sh.help_slot = best;
      sh.help_cam = cam;
    }
    __syncthreads();
    const int slot = sh.help_slot, cam = sh.help_cam;
    if (cam == -2) break;
    if (slot >= 0 && cam >= 0) {
      const Scratch o = slot_scratch(p, slot);
      __threadfence();
      take_published<kShadow>(sh, sp, o.pub);
      __syncthreads();
      raster_claimed<kF>(p, sh, o, sp, L, cam, false);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// plain: three launches per sample; scratch slot = camera index within the sample
// (in the shadow pass: the sample's map blockIdx.x, light-major then face).
// staged: the same three kernels, each launched once over a chunk of the batch's images
// (image stage_base + blockIdx.x; scratch slot = blockIdx.x).
// ---------------------------------------------------------------------------
__device__ inline int plain_cam(const Params& p) {
  const int s = p.plain_sample;
  if (s == kStagedLaunch) {
    const int c = p.stage_base + int(blockIdx.x);
    return c < p.n_cams ? c : -1;
  }
  if (p.shadow_pass) {
    const int per = kMaxLights * p.shadow_faces;
    return int(blockIdx.x) < per ? s * per + int(blockIdx.x) : -1;
  }
  const int c = p.cam_offset[s] + blockIdx.x;
  return c < p.cam_offset[s + 1] ? c : -1;
}

// kG: bit 0 tracker rows, bit 1 the shadow pass
template <int kG>
__global__ void __launch_bounds__(512, 2) plain_geometry_kernel(Params p) {
  constexpr bool kTrack = (kG & 1) != 0, kPass = (kG & 2) != 0;
  extern __shared__ __align__(16) char smem[];
  __shared__ CtaShared sh;
  const int cam = plain_cam(p);
  if (cam < 0) return;
  const SmemLayout L = layout_of(p);
  SmemPtrs sp = carve(smem, p, L);
  const Scratch sc = slot_scratch(p, blockIdx.x);
  setup_image<kPass>(p, cam, sh, sp.mprefix, sp.tprefix, sp.mbegin, true, kTrack);
  if (!sh.im.valid) {
    if (threadIdx.x == 0) sc.header[2] = -1;
    return;
  }
  geometry_phase<kTrack, kPass>(p, sh, sp.mprefix, sp.tprefix, sp.mbegin, reinterpret_cast<WarpG*>(sp.uni), sc);
  __syncthreads();
  if (threadIdx.x == 0) sc.header[2] = sh.n_vis;
}

__global__ void __launch_bounds__(512, 2) plain_bin_kernel(Params p) {
  extern __shared__ __align__(16) char smem[];
  __shared__ CtaShared sh;
  const int cam = plain_cam(p);
  if (cam < 0) return;
  const SmemLayout L = layout_of(p);
  SmemPtrs sp = carve(smem, p, L);
  const Scratch sc = slot_scratch(p, blockIdx.x);
  if (p.shadow_pass) setup_image<true>(p, cam, sh, sp.mprefix, sp.tprefix, sp.mbegin, false);
  else setup_image(p, cam, sh, sp.mprefix, sp.tprefix, sp.mbegin, false);
  const int nvis = sc.header[2];
  if (nvis < 0) return;
  if (threadIdx.x == 0) sh.n_vis = nvis;
  __syncthreads();
  int* counts = p.max_tiles > kSmemCountTiles ? sc.counts : reinterpret_cast<int*>(sp.uni);
  bin_phase(p, sh, counts, counts + (p.max_tiles + 2), sc);
  if (threadIdx.x == 0) sc.header[3] = sh.n_big;
}

template <int kF>
__global__ void __launch_bounds__(512, 2) plain_raster_kernel(Params p) {
  constexpr bool kGrade = (kF & kFeatGrade) != 0, kLight = (kF & kFeatLight) != 0;
  constexpr bool kShadow = (kF & kFeatShadow) != 0, kPass = (kF & kFeatShadowPass) != 0;
  extern __shared__ __align__(16) char smem[];
  __shared__ CtaShared sh;
  const int cam = plain_cam(p);
  if (cam < 0) return;
  const Scratch sc = slot_scratch(p, blockIdx.x);
  if (sc.header[2] < 0) return;
  const SmemLayout L = layout_of(p);
  SmemPtrs sp = carve(smem, p, L);
  setup_image<kPass>(p, cam, sh, sp.mprefix, sp.tprefix, sp.mbegin, false);
  if (threadIdx.x == 0) sh.n_big = sc.header[3];
  if (kGrade && threadIdx.x == 0) grading_setup(p, sh.im);
  if (kLight && threadIdx.x < kMaxLights) spot_setup(p, sh.im, threadIdx.x);
  if (kShadow && threadIdx.x < kMaxLights)
    shadow_setup(p, sh.im, *reinterpret_cast<ShadowInfo*>(sp.spans + kSpanCap), threadIdx.x);
  __syncthreads();
  big_spans(p, sh, sc, sp.spans);
  __syncthreads();
  raster_phase<kF>(p, sh, sc, sp, L, blockIdx.y, gridDim.y);
}

// Scratch of orrb_render_batch_noalloc: a file-scope device array, so that
// entry point never allocates.  Host code must not pass the symbol itself to
// a kernel (on the host it names a stand-in, not device memory); it passes
// the device address looked up below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ORRB_NOALLOC_SCRATCH_BYTES];

}  // namespace

// Device address of the static scratch on `device`, looked up once per device
// with that device current (the caller makes it current).  Returns a CUDA
// error code, 0 on success.
int noalloc_scratch(int device, void** ptr, size_t* bytes) {
  static std::mutex mu;
  static void* cache[256] = {};
  if (device < 0 || device >= 256) return (int)cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if (!cache[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return (int)e;
    cache[device] = p;
  }
  *ptr = cache[device];
  *bytes = ORRB_NOALLOC_SCRATCH_BYTES;
  return 0;
}

size_t render_smem_bytes(int threads, int tile_w, int tile_h, int inst_max, int max_tiles, int w_max, bool shadows) {
  return smem_layout(threads, tile_w, tile_h, inst_max, max_tiles, w_max, shadows).total;
}

namespace {
// The dynamic shared-memory limit is a per-device function attribute: raise it only when a
// larger size is needed, so steady-state launches (and launches inside a stream capture)
// make no attribute calls.
std::mutex g_attr_mu;
size_t g_attr_set[32][64] = {};  // per kernel instance: fused 0-12, plain geometry 13-15, bin 16, raster 20-26

cudaError_t ensure_smem(const void* fn, int which, size_t smem) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_attr_mu);
  if (g_attr_set[which][dev] >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) g_attr_set[which][dev] = smem;
  return e;
}
}  // namespace

// The feature bits of a launch's batch and outputs.
static int features(const Params& p) {
  if (p.shadow_pass) return kFeatShadowPass;
  int f = (p.grading ? kFeatGrade : 0) | (p.tracker ? kFeatTrack : 0) | (p.light_spot || p.emission ? kFeatLight : 0);
  if (p.shadow_res > 0) f |= kFeatShadow | kFeatLight;
  return f;
}

// The fused instances: feature sets 0-7, 12-15 (shadow lookups) and 16 (the shadow pass); slot k of
// the attribute cache is the k-th of kFusedSets.
constexpr int kFusedSets[13] = {0, 1, 2, 3, 4, 5, 6, 7, 12, 13, 14, 15, 16};
static int fused_slot(int f) {
  for (int k = 0; k < 13; k++)
    if (kFusedSets[k] == f) return k;
  return 0;
}
static const void* fused_fn(int f) {
  static const void* const fns[13] = {
      (const void*)render_fused_kernel<0>,  (const void*)render_fused_kernel<1>,  (const void*)render_fused_kernel<2>,
      (const void*)render_fused_kernel<3>,  (const void*)render_fused_kernel<4>,  (const void*)render_fused_kernel<5>,
      (const void*)render_fused_kernel<6>,  (const void*)render_fused_kernel<7>,  (const void*)render_fused_kernel<12>,
      (const void*)render_fused_kernel<13>, (const void*)render_fused_kernel<14>, (const void*)render_fused_kernel<15>,
      (const void*)render_fused_kernel<16>};
  return fns[fused_slot(f)];
}

// The plain raster instances (grading, light, shadow lookups, the shadow pass; slots 20 + k).
constexpr int kPlainRasterSets[7] = {0, 1, 4, 5, 12, 13, 16};
static int plain_raster_slot(int f) {
  const int g = f & (kFeatGrade | kFeatLight | kFeatShadow | kFeatShadowPass);
  for (int k = 0; k < 7; k++)
    if (kPlainRasterSets[k] == g) return k;
  return 0;
}
static const void* plain_raster_fn(int f) {
  static const void* const fns[7] = {
      (const void*)plain_raster_kernel<0>,  (const void*)plain_raster_kernel<1>,  (const void*)plain_raster_kernel<4>,
      (const void*)plain_raster_kernel<5>,  (const void*)plain_raster_kernel<12>, (const void*)plain_raster_kernel<13>,
      (const void*)plain_raster_kernel<16>};
  return fns[plain_raster_slot(f)];
}

int render_max_ctas_per_sm(int threads, size_t smem) {
  int n = 0;
  n = 1 << 30;  // every instance: the same launch bounds and shared memory; the least of their fits
  for (int k = 0; k < 13; k++) {
    int m = 0;
    if (ensure_smem(fused_fn(kFusedSets[k]), k, smem) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, fused_fn(kFusedSets[k]), threads, smem) != cudaSuccess)
      return -1;
    n = m < n ? m : n;
  }
  return n;
}

int launch_render(const Params& p, int mode, int threads, int n_ctas, int max_cams_per_sample, void* stream,
                  char* err, size_t errlen) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t smem = render_smem_bytes(threads, p.tile_w, p.tile_h, p.inst_max, p.max_tiles, p.w_max,
                                       p.shadow_res > 0 && !p.shadow_pass);
  cudaError_t e = cudaSuccess;
  const int f = features(p);
  if (mode == 0) {
    e = ensure_smem(fused_fn(f), fused_slot(f), smem);
    if (e == cudaSuccess) {  // slot headers (claim words, counters) start at zero
      const SlotLayout SL = slot_layout(p.t_max, p.max_tiles);
      e = cudaMemset2DAsync(p.scratch + SL.header, p.slot_bytes, 0, 64, (size_t)n_ctas, st);
    }
    if (e == cudaSuccess) {
      switch (f) {
        case 0: render_fused_kernel<0><<<n_ctas, threads, smem, st>>>(p); break;
        case 1: render_fused_kernel<1><<<n_ctas, threads, smem, st>>>(p); break;
        case 2: render_fused_kernel<2><<<n_ctas, threads, smem, st>>>(p); break;
        case 3: render_fused_kernel<3><<<n_ctas, threads, smem, st>>>(p); break;
        case 4: render_fused_kernel<4><<<n_ctas, threads, smem, st>>>(p); break;
        case 5: render_fused_kernel<5><<<n_ctas, threads, smem, st>>>(p); break;
        case 6: render_fused_kernel<6><<<n_ctas, threads, smem, st>>>(p); break;
        case 7: render_fused_kernel<7><<<n_ctas, threads, smem, st>>>(p); break;
        case 12: render_fused_kernel<12><<<n_ctas, threads, smem, st>>>(p); break;
        case 13: render_fused_kernel<13><<<n_ctas, threads, smem, st>>>(p); break;
        case 14: render_fused_kernel<14><<<n_ctas, threads, smem, st>>>(p); break;
        case 15: render_fused_kernel<15><<<n_ctas, threads, smem, st>>>(p); break;
        default: render_fused_kernel<16><<<n_ctas, threads, smem, st>>>(p); break;
      }
      e = cudaGetLastError();
    }
  } else {
    const int g = ((f & kFeatTrack) ? 1 : 0) | ((f & kFeatShadowPass) ? 2 : 0);
    const void* geo = g == 1 ? (const void*)plain_geometry_kernel<1>
                             : (g == 2 ? (const void*)plain_geometry_kernel<2> : (const void*)plain_geometry_kernel<0>);
    const void* ks[3] = {geo, (const void*)plain_bin_kernel, plain_raster_fn(f)};
    const int which[3] = {13 + g, 16, 20 + plain_raster_slot(f)};
    for (int k = 0; k < 3 && e == cudaSuccess; k++) e = ensure_smem(ks[k], which[k], smem);
    Params q = p;
    // plain: one sample's images per launch; staged: a chunk of n_ctas images per launch
    const bool staged = mode == ORRB_MODE_STAGED;
    const int per = staged ? n_ctas : max_cams_per_sample;
    const int n_launches = staged ? (p.n_cams + n_ctas - 1) / n_ctas : p.n_samples;
    const dim3 grid(per, staged ? kStagedRasterSplit : kPlainRasterSplit);
    for (int s = 0; s < n_launches && e == cudaSuccess; s++) {
      q.plain_sample = staged ? kStagedLaunch : s;
      q.stage_base = staged ? s * n_ctas : 0;
      switch (g) {
        case 1: plain_geometry_kernel<1><<<per, threads, smem, st>>>(q); break;
        case 2: plain_geometry_kernel<2><<<per, threads, smem, st>>>(q); break;
        default: plain_geometry_kernel<0><<<per, threads, smem, st>>>(q); break;
      }
      plain_bin_kernel<<<per, threads, smem, st>>>(q);
      switch (kPlainRasterSets[plain_raster_slot(f)]) {
        case 0: plain_raster_kernel<0><<<grid, threads, smem, st>>>(q); break;
        case 1: plain_raster_kernel<1><<<grid, threads, smem, st>>>(q); break;
        case 4: plain_raster_kernel<4><<<grid, threads, smem, st>>>(q); break;
        case 5: plain_raster_kernel<5><<<grid, threads, smem, st>>>(q); break;
        case 12: plain_raster_kernel<12><<<grid, threads, smem, st>>>(q); break;
        case 13: plain_raster_kernel<13><<<grid, threads, smem, st>>>(q); break;
        default: plain_raster_kernel<16><<<grid, threads, smem, st>>>(q); break;
      }
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) {
    snprintf(err, errlen, "render launch failed: %s", cudaGetErrorString(e));
    return 1;
  }
  return 0;
}

}  // namespace orrb
