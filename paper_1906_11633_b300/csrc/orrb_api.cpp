// orrb_api.cpp -- host side of the C-ABI declared in include/orrb.h.
//
// Owns only host metadata: the device index, the layout of the uploaded mesh
// arena and the last error message.  Every device buffer (mesh arena,
// workspace, outputs, batch arrays) belongs to the caller.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "orrb.h"
#include "orrb_internal.h"

namespace orrb {
int render_max_ctas_per_sm(int threads, size_t smem);
int noalloc_scratch(int device, void** ptr, size_t* bytes);
}

struct orrb_ctx {
  int device = 0;
  int sm_count = 0;
  std::vector<std::pair<std::pair<int, size_t>, int>> occupancy;  // (threads, smem) -> CTAs per SM
  std::mutex mu;
  std::string err;
  bool has_meshes = false;
  orrb::ArenaLayout arena{};
  const char* arena_ptr = nullptr;
};

namespace {

using namespace orrb;

// An NVTX range over one host-side step (a no-op unless a profiler is attached), so that a
// timeline shows which entry point and which launch of a render enqueued the kernels.
// A null name opens no range (the allocation-free entry point calls nothing it need not).
struct Range {
  explicit Range(const char* name) : on(name != nullptr) {
    if (on) nvtxRangePushA(name);
  }
  ~Range() {
    if (on) nvtxRangePop();
  }
  bool on;
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

orrb_status fail(orrb_ctx* ctx, orrb_status s, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return s;
}

// Restores the calling thread's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

struct Cluster {
  int vert_begin, tri_begin, n_verts, n_tris, mesh_tri_base;
};

// Greedy clustering in triangle order: a cluster closes when the next
// triangle would bring it over 64 distinct vertices or 128 triangles.
void build_clusters(const orrb_mesh_desc* meshes, int n, std::vector<MeshEntry>& me, std::vector<Cluster>& cl,
                    std::vector<float4>* vpos, std::vector<float4>* vnrm, std::vector<uint32_t>* tris) {
  int vtotal = 0, ttotal = 0;
  for (int m = 0; m < n; m++) {
    const orrb_mesh_desc& d = meshes[m];
    MeshEntry e;
    e.meshlet_begin = (int)cl.size();
    e.n_tris = d.n_tris;
    e.n_verts = d.n_verts;
    std::vector<int> local(d.n_verts, -1);
    std::vector<int> members;
    Cluster cur{vtotal, ttotal, 0, 0, 0};
    auto close = [&]() {
      if (cur.n_tris > 0) {
        cl.push_back(cur);
        vtotal += cur.n_verts;
        ttotal += cur.n_tris;
      }
      for (int v : members) local[v] = -1;
      members.clear();
    };
    for (int t = 0; t < d.n_tris; t++) {
      const uint32_t* tv = d.idx + 3 * (size_t)t;
      int fresh = 0;
      for (int k = 0; k < 3; k++) {
        bool dup = false;
        for (int j = 0; j < k; j++) dup |= tv[j] == tv[k];
        if (!dup && local[tv[k]] < 0) fresh++;
      }
      if (cur.n_verts + fresh > kMeshletVerts || cur.n_tris + 1 > kMeshletTris) {
        close();
        cur = Cluster{vtotal, ttotal, 0, 0, t};
      }
      uint32_t packed = 0;
      for (int k = 0; k < 3; k++) {
        int v = (int)tv[k];
        if (local[v] < 0) {
          local[v] = cur.n_verts++;
          members.push_back(v);
          if (vpos) {
            vpos->push_back(make_float4(d.pos[3 * v], d.pos[3 * v + 1], d.pos[3 * v + 2], 0.0f));
            vnrm->push_back(make_float4(d.nrm[3 * v], d.nrm[3 * v + 1], d.nrm[3 * v + 2], 0.0f));
          }
        }
        packed |= uint32_t(local[v]) << (8 * k);
      }
      if (tris) tris->push_back(packed | (uint32_t(d.tri_mat ? d.tri_mat[t] : 0) << 24));
      cur.n_tris++;
    }
    close();
    e.meshlet_count = (int)cl.size() - e.meshlet_begin;
    me.push_back(e);
  }
}

ArenaLayout arena_layout(int n_meshes, int n_meshlets, int n_verts, int n_tris) {
  ArenaLayout L{};
  size_t o = 0;
  L.meshes = o;
  o = align256(o + sizeof(MeshEntry) * (size_t)std::max(n_meshes, 1));
  L.meshlets = o;
  o = align256(o + sizeof(MeshletEntry) * (size_t)std::max(n_meshlets, 1));
  L.bounds = o;
  o = align256(o + 16 * (size_t)std::max(n_meshlets, 1));
  L.vpos = o;
  o = align256(o + 16 * (size_t)std::max(n_verts, 1));
  L.vnrm = o;
  o = align256(o + 16 * (size_t)std::max(n_verts, 1));
  L.tris = o;
  o = align256(o + 4 * (size_t)std::max(n_tris, 1));
  L.total = o;
  L.n_meshes = n_meshes;
  L.n_meshlets = n_meshlets;
  L.n_verts = n_verts;
  L.n_tris = n_tris;
  return L;
}

orrb_status check_meshes(orrb_ctx* ctx, const orrb_mesh_desc* meshes, int32_t n) {
  if (!meshes || n <= 0) return fail(ctx, ORRB_ERR_INVALID_ARG, "no meshes given");
  for (int m = 0; m < n; m++) {
    const orrb_mesh_desc& d = meshes[m];
    if (d.n_verts < 0 || d.n_tris < 0 || (d.n_verts > 0 && (!d.pos || !d.nrm)) || (d.n_tris > 0 && !d.idx))
      return fail(ctx, ORRB_ERR_INVALID_ARG, "mesh %d: bad counts or null arrays", m);
    if (d.n_tris > (1 << 24)) return fail(ctx, ORRB_ERR_INVALID_ARG, "mesh %d: more than 2^24 triangles", m);
    for (size_t i = 0; i < 3 * (size_t)d.n_tris; i++)
      if (d.idx[i] >= (uint32_t)d.n_verts)
        return fail(ctx, ORRB_ERR_INVALID_ARG, "mesh %d: vertex index %u out of range", m, d.idx[i]);
    for (size_t i = 0; i < 3 * (size_t)d.n_verts; i++)
      if (!std::isfinite(d.pos[i]) || !std::isfinite(d.nrm[i]))
        return fail(ctx, ORRB_ERR_INVALID_ARG, "mesh %d: non-finite vertex data", m);
  }
  return ORRB_OK;
}

void resolve_config(const orrb_config* in, orrb_config* out) {
  orrb_config c{};
  if (in) c = *in;
  if (c.tile_w == 0) c.tile_w = 256;
  if (c.tile_h == 0) c.tile_h = 2;
  if (c.threads == 0) c.threads = 512;
  if (c.wait_cycles == 0) c.wait_cycles = 2000000000ll;
  *out = c;
}

orrb_status check_config(orrb_ctx* ctx, const orrb_config& c) {
  if (c.mode != ORRB_MODE_FUSED && c.mode != ORRB_MODE_PLAIN && c.mode != ORRB_MODE_STAGED)
    return fail(ctx, ORRB_ERR_INVALID_ARG, "bad mode %d", c.mode);
  if (c.tile_w < 8 || c.tile_w > 512 || c.tile_w % 8) return fail(ctx, ORRB_ERR_INVALID_ARG, "tile_w %d", c.tile_w);
  if (c.tile_h < 1 || c.tile_h > 64) return fail(ctx, ORRB_ERR_INVALID_ARG, "tile_h %d", c.tile_h);
  if (c.tile_w * c.tile_h > 8192) return fail(ctx, ORRB_ERR_INVALID_ARG, "tile larger than 8192 px");
  if (c.threads != 256 && c.threads != 512) return fail(ctx, ORRB_ERR_INVALID_ARG, "threads %d", c.threads);
  if (c.ctas_per_sm < 0) return fail(ctx, ORRB_ERR_INVALID_ARG, "ctas_per_sm %d", c.ctas_per_sm);
  if (c.reserved != 0) return fail(ctx, ORRB_ERR_INVALID_ARG, "reserved config field must be 0");
  if (c.wait_cycles < 0) return fail(ctx, ORRB_ERR_INVALID_ARG, "wait_cycles %lld", (long long)c.wait_cycles);
  return ORRB_OK;
}

orrb_status check_shape(orrb_ctx* ctx, const orrb_batch_shape* s) {
  if (!s) return fail(ctx, ORRB_ERR_INVALID_ARG, "null shape");
  if (s->n_samples < 0 || s->n_cams < 0) return fail(ctx, ORRB_ERR_INVALID_ARG, "negative counts");
  if (s->max_width < 1 || s->max_height < 1 || s->max_width > ORRB_MAX_RESOLUTION ||
      s->max_height > ORRB_MAX_RESOLUTION)
    return fail(ctx, ORRB_ERR_INVALID_ARG, "resolution %dx%d outside [1, %d]", s->max_width, s->max_height,
                ORRB_MAX_RESOLUTION);
  if (s->max_inst_per_sample < 0 || s->max_inst_per_sample > ORRB_MAX_INSTANCES)
    return fail(ctx, ORRB_ERR_INVALID_ARG, "max_inst_per_sample %d outside [0, %d]", s->max_inst_per_sample,
                ORRB_MAX_INSTANCES);
  if (s->max_tris_per_sample < 0 || s->max_tris_per_sample > (1 << 26))
    return fail(ctx, ORRB_ERR_INVALID_ARG, "max_tris_per_sample %d", s->max_tris_per_sample);
  if (s->max_cams_per_sample < 0 || s->total_pixels < 0)
    return fail(ctx, ORRB_ERR_INVALID_ARG, "bad camera or pixel count");
  if (s->shadow_res < 0 || s->shadow_res > ORRB_MAX_RESOLUTION)
    return fail(ctx, ORRB_ERR_INVALID_ARG, "shadow_res %d outside [0, %d]", s->shadow_res, ORRB_MAX_RESOLUTION);
  if (s->shadow_faces < 0 || s->shadow_faces > kMaxShadowFaces)
    return fail(ctx, ORRB_ERR_INVALID_ARG, "shadow_faces %d outside [0, %d]", s->shadow_faces, kMaxShadowFaces);
  if (s->post_effects != 0 && s->post_effects != 1)
    return fail(ctx, ORRB_ERR_INVALID_ARG, "post_effects %d is neither 0 nor 1", s->post_effects);
  return ORRB_OK;
}

int faces_of(const orrb_batch_shape& s) { return s.shadow_faces > 0 ? s.shadow_faces : 1; }

int tiles_of(int w, int h, const orrb_config& c) {
  int tw = std::min(w, c.tile_w);
  return ((w + tw - 1) / tw) * ((h + c.tile_h - 1) / c.tile_h);
}

// the camera images' tiling, or the shadow maps' when they need more tiles
int max_tiles_of(const orrb_batch_shape& s, const orrb_config& c) {
  int t = tiles_of(s.max_width, s.max_height, c);
  if (s.shadow_res > 0) t = std::max(t, tiles_of(s.shadow_res, s.shadow_res, c));
  return t;
}

struct Plan {
  int n_slots, ctas_per_sm, max_tiles;
  size_t slot_bytes, smem, total;
  size_t nb_offset;   // the shadow maps' neighbourhood table (after the slots), 0 without shadows
  size_t cnt_offset;  // its occupied-texel counts (after the table)
  // the post pass's images (with shape.post_effects): linear colour, depth, normals, occluded
  // colour, row blur
  size_t post_lin, post_depth, post_normal, post_cao, post_hblur;
};

orrb_status plan(orrb_ctx* ctx, const orrb_batch_shape& s, const orrb_config& c, Plan* P) {
  P->max_tiles = max_tiles_of(s, c);
  SlotLayout L = slot_layout(s.max_tris_per_sample, P->max_tiles);
  P->slot_bytes = L.total;
  P->smem = render_smem_bytes(c.threads, c.tile_w, c.tile_h, s.max_inst_per_sample, P->max_tiles,
                              std::max(s.max_width, s.shadow_res), s.shadow_res > 0);
  if (P->smem > 227 * 1024) return fail(ctx, ORRB_ERR_INVALID_ARG, "tile / instance limits need %zu B of shared memory", P->smem);
  if (c.mode == ORRB_MODE_FUSED) {
    int fit = -1;
    for (const auto& o : ctx->occupancy)
      if (o.first.first == c.threads && o.first.second == P->smem) fit = o.second;
    if (fit < 0) {
      fit = render_max_ctas_per_sm(c.threads, P->smem);
      if (fit > 0) ctx->occupancy.push_back({{c.threads, P->smem}, fit});
    }
    if (fit <= 0) return fail(ctx, ORRB_ERR_CUDA, "occupancy query failed for %zu B shared memory", P->smem);
    P->ctas_per_sm = c.ctas_per_sm > 0 ? std::min(c.ctas_per_sm, fit) : fit;
    P->n_slots = ctx->sm_count * P->ctas_per_sm;
  } else if (c.mode == ORRB_MODE_STAGED) {
    // one slot per image of a chunk: every image of the launch (and every shadow map of the shadow
    // pass) while the slots fit in 8 GiB, else chunks of that many, at least two images per SM
    P->ctas_per_sm = 0;
    const long long images = std::max<long long>(
        std::max(s.n_cams, 1), s.shadow_res > 0 ? (long long)s.n_samples * kMaxLights * faces_of(s) : 1);
    const long long fit = (long long)((size_t(8) << 30) / std::max<size_t>(P->slot_bytes, 1));
    P->n_slots = (int)std::min(images, std::max(fit, 2LL * ctx->sm_count));
  } else {
    P->ctas_per_sm = 0;
    P->n_slots = std::max(std::max(s.max_cams_per_sample, 1), s.shadow_res > 0 ? kMaxLights * faces_of(s) : 1);
  }
  P->total = 256 + (size_t)P->n_slots * P->slot_bytes;
  P->nb_offset = 0;
  P->cnt_offset = 0;
  if (s.shadow_res > 0) {
    const size_t texels = (size_t)s.n_samples * kMaxLights * faces_of(s) * s.shadow_res * s.shadow_res;
    P->nb_offset = align256(P->total);
    P->cnt_offset = align256(P->nb_offset + texels * sizeof(uint32_t));
    P->total = P->cnt_offset + texels;
  }
  P->post_lin = P->post_depth = P->post_normal = P->post_cao = P->post_hblur = 0;
  if (s.post_effects) {
    const size_t n = (size_t)s.total_pixels;
    P->post_lin = align256(P->total);
    P->post_depth = align256(P->post_lin + 12 * n);
    P->post_normal = align256(P->post_depth + 4 * n);
    P->post_cao = align256(P->post_normal + 6 * n);
    P->post_hblur = align256(P->post_cao + 12 * n);
    P->total = P->post_hblur + 12 * n;
  }
  return ORRB_OK;
}

void fill_batch(Params& p, const orrb_batch_shape& s, const orrb_batch_desc& b) {
  p.n_samples = s.n_samples;
  p.n_cams = s.n_cams;
  p.inst_offset = b.inst_offset;
  p.inst_mesh = b.inst_mesh;
  p.inst_pose = b.inst_pose;
  p.inst_seg = b.inst_seg;
  p.inst_mat_base = b.inst_mat_base;
  p.cam_offset = b.cam_offset;
  p.cam_sample = b.cam_sample;
  p.cam_view = b.cam_view;
  p.cam_intr = b.cam_intr;
  p.cam_wh = b.cam_wh;
  p.img_offset = b.img_offset;
  p.light = b.light;
  p.light_meta = b.light_meta;
  p.material = b.material;
  p.exposure_ev = b.exposure_ev;
  p.ambient = b.ambient;
  p.background = b.background;
  p.grading = b.grading;
  p.light_spot = b.light_spot;
  p.emission = b.emission;
  p.shadow_view = b.shadow_view;
  p.shadow_intr = b.shadow_intr;
  p.shadow_res = s.shadow_res > 0 && b.shadow_view && b.shadow_intr ? s.shadow_res : 0;
  p.shadow_faces = faces_of(s);
  p.total_pixels = s.total_pixels;
  p.t_max = s.max_tris_per_sample;
  p.inst_max = s.max_inst_per_sample;
  p.w_max = s.max_width;
  p.h_max = s.max_height;
}

orrb_status check_desc(orrb_ctx* ctx, const orrb_batch_desc* b) {
  if (!b) return fail(ctx, ORRB_ERR_INVALID_ARG, "null batch");
  const void* req[] = {b->inst_offset, b->inst_mesh, b->inst_pose, b->inst_seg, b->inst_mat_base, b->cam_offset,
                       b->cam_sample,  b->cam_view,  b->cam_intr,  b->cam_wh,   b->img_offset,    b->light,
                       b->light_meta,  b->material,  b->exposure_ev, b->ambient, b->background};
  for (size_t i = 0; i < sizeof(req) / sizeof(req[0]); i++)
    if (!req[i]) return fail(ctx, ORRB_ERR_INVALID_ARG, "batch array %zu is null", i);
  return ORRB_OK;
}

// Enqueue one render: the shadow pass first when the batch has shadows (its own launch over
// the images sample * 4 + light, depth only, into the shadow maps), then the camera images.
// n_slots: the scratch slots the fused mode may use; ws: the status word and queue counters.
orrb_status enqueue_render(orrb_ctx* ctx, Params& p, const orrb_batch_shape& s, int mode, int threads, int n_slots,
                           char* ws, void* stream, bool trace = true) {
  char err[256] = {0};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (p.shadow_res > 0) {
    Range r(trace ? "orrb shadow pass + neighbourhood table" : nullptr);
    Params q = p;
    q.shadow_pass = 1;
    q.n_cams = s.n_samples * kMaxLights * p.shadow_faces;
    q.rgb = nullptr;
    q.normal = nullptr;
    q.seg = nullptr;
    q.rgb_linear = nullptr;
    q.rgb_graded = nullptr;
    q.gbuffer = nullptr;
    q.tracker = nullptr;
    q.grading = nullptr;
    q.depth = p.shadow_map;
    q.total_pixels = (int64_t)q.n_cams * s.shadow_res * s.shadow_res;
    q.w_max = q.h_max = s.shadow_res;
    const int n_ctas = mode != ORRB_MODE_PLAIN ? std::min(n_slots, std::max(q.n_cams, 1)) : 0;
    q.n_slots = n_ctas;
    if (launch_render(q, mode, threads, n_ctas, kMaxLights * p.shadow_faces, stream, err, sizeof(err)))
      return fail(ctx, ORRB_ERR_CUDA, "%s", err);
    if (p.shadow_nb && launch_shadow_neighbourhoods(q, stream, err, sizeof(err)))
      return fail(ctx, ORRB_ERR_CUDA, "%s", err);
    // the camera launch's image queue starts again at zero (the status word carries over)
    cudaError_t e = cudaMemsetAsync(ws + 4, 0, 8, st);
    if (e != cudaSuccess) return fail(ctx, ORRB_ERR_CUDA, "queue reset: %s", cudaGetErrorString(e));
  }
  Range r(!trace ? nullptr
                 : mode == ORRB_MODE_FUSED ? "orrb camera launch (fused)"
                 : mode == ORRB_MODE_STAGED ? "orrb camera launches (staged)" : "orrb camera launches (plain)");
  const int n_ctas = mode != ORRB_MODE_PLAIN ? std::min(n_slots, std::max(s.n_cams, 1)) : 0;
  p.n_slots = n_ctas;
  if (launch_render(p, mode, threads, n_ctas, std::max(s.max_cams_per_sample, 1), stream, err, sizeof(err)))
    return fail(ctx, ORRB_ERR_CUDA, "%s", err);
  return ORRB_OK;
}

}  // namespace

extern "C" {

const char* orrb_status_string(orrb_status s) {
  switch (s) {
    case ORRB_OK: return "ok";
    case ORRB_ERR_INVALID_ARG: return "invalid argument";
    case ORRB_ERR_WORKSPACE: return "workspace or arena too small";
    case ORRB_ERR_CUDA: return "CUDA error";
    case ORRB_ERR_TIMEOUT: return "device wait timed out";
    case ORRB_ERR_NOT_FOUND: return "no mesh set uploaded";
    case ORRB_ERR_UNSUPPORTED: return "unsupported device or option";
    case ORRB_ERR_DEVICE: return "device status word non-zero";
    default: return "unknown status";
  }
}

orrb_status orrb_create(int device, orrb_ctx** out) {
  if (!out) return ORRB_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return ORRB_ERR_INVALID_ARG;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return ORRB_ERR_CUDA;
  if (prop.major != 10 || prop.minor != 3) return ORRB_ERR_UNSUPPORTED;
  orrb_ctx* c = new orrb_ctx();
  c->device = device;
  c->sm_count = prop.multiProcessorCount;
  *out = c;
  return ORRB_OK;
}

void orrb_destroy(orrb_ctx* ctx) { delete ctx; }

orrb_status orrb_last_error(orrb_ctx* ctx, char* buf, size_t len) {
  if (!ctx || !buf || len == 0) return ORRB_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(ctx->mu);
  snprintf(buf, len, "%s", ctx->err.c_str());
  return ORRB_OK;
}

orrb_status orrb_mesh_arena_size(const orrb_mesh_desc* meshes, int32_t n, size_t* bytes) {
  if (!bytes) return ORRB_ERR_INVALID_ARG;
  orrb_status st = check_meshes(nullptr, meshes, n);
  if (st != ORRB_OK) return st;
  std::vector<MeshEntry> me;
  std::vector<Cluster> cl;
  build_clusters(meshes, n, me, cl, nullptr, nullptr, nullptr);
  int nv = 0, nt = 0;
  for (const Cluster& c : cl) {
    nv += c.n_verts;
    nt += c.n_tris;
  }
  *bytes = arena_layout(n, (int)cl.size(), nv, nt).total;
  return ORRB_OK;
}

orrb_status orrb_upload_meshes(orrb_ctx* ctx, const orrb_mesh_desc* meshes, int32_t n, void* dev_arena,
                               size_t arena_bytes, void* stream) {
  if (!ctx) return ORRB_ERR_INVALID_ARG;
  Range range("orrb_upload_meshes");
  std::lock_guard<std::mutex> g(ctx->mu);
  orrb_status st = check_meshes(ctx, meshes, n);
  if (st != ORRB_OK) return st;
  if (!dev_arena || (reinterpret_cast<uintptr_t>(dev_arena) & 255))
    return fail(ctx, ORRB_ERR_INVALID_ARG, "arena must be a 256-byte aligned device pointer");
  std::vector<MeshEntry> me;
  std::vector<Cluster> cl;
  std::vector<float4> vpos, vnrm;
  std::vector<uint32_t> tris;
  build_clusters(meshes, n, me, cl, &vpos, &vnrm, &tris);
  ArenaLayout L = arena_layout(n, (int)cl.size(), (int)vpos.size(), (int)tris.size());
  if (arena_bytes < L.total) return fail(ctx, ORRB_ERR_WORKSPACE, "arena needs %zu bytes, got %zu", L.total, arena_bytes);
  std::vector<char> host(L.total, 0);
  std::memcpy(host.data() + L.meshes, me.data(), sizeof(MeshEntry) * me.size());
  std::vector<MeshletEntry> ml(cl.size());
  for (size_t i = 0; i < cl.size(); i++)
    ml[i] = MeshletEntry{cl[i].vert_begin, cl[i].tri_begin, cl[i].n_verts | (cl[i].n_tris << 16), cl[i].mesh_tri_base};
  if (!ml.empty()) std::memcpy(host.data() + L.meshlets, ml.data(), sizeof(MeshletEntry) * ml.size());
  // per cluster a bounding sphere: the centre of its vertices' box and the largest distance to it,
  // in double, rounded outwards (the shadow pass skips clusters wholly outside a shadow camera's view)
  std::vector<float4> bounds(cl.size());
  for (size_t i = 0; i < cl.size(); i++) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int v = 0; v < cl[i].n_verts; v++) {
      const float4 q = vpos[cl[i].vert_begin + v];
      const double c[3] = {q.x, q.y, q.z};
      for (int k = 0; k < 3; k++) {
        lo[k] = std::min(lo[k], c[k]);
        hi[k] = std::max(hi[k], c[k]);
      }
    }
    double mid[3], r2 = 0.0;
    for (int k = 0; k < 3; k++) mid[k] = cl[i].n_verts ? 0.5 * (lo[k] + hi[k]) : 0.0;
    for (int v = 0; v < cl[i].n_verts; v++) {
      const float4 q = vpos[cl[i].vert_begin + v];
      const double d[3] = {q.x - mid[0], q.y - mid[1], q.z - mid[2]};
      r2 = std::max(r2, d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
    bounds[i] = make_float4((float)mid[0], (float)mid[1], (float)mid[2], (float)(std::sqrt(r2) * (1.0 + 1e-6) + 1e-6));
  }
  if (!bounds.empty()) std::memcpy(host.data() + L.bounds, bounds.data(), 16 * bounds.size());
  if (!vpos.empty()) {
    std::memcpy(host.data() + L.vpos, vpos.data(), 16 * vpos.size());
    std::memcpy(host.data() + L.vnrm, vnrm.data(), 16 * vnrm.size());
  }
  if (!tris.empty()) std::memcpy(host.data() + L.tris, tris.data(), 4 * tris.size());
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return fail(ctx, ORRB_ERR_CUDA, "cudaSetDevice(%d) failed", ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(dev_arena, host.data(), L.total, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, ORRB_ERR_CUDA, "arena upload: %s", cudaGetErrorString(e));
  ctx->arena = L;
  ctx->arena_ptr = static_cast<const char*>(dev_arena);
  ctx->has_meshes = true;
  return ORRB_OK;
}

orrb_status orrb_release_meshes(orrb_ctx* ctx) {
  if (!ctx) return ORRB_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->has_meshes = false;
  ctx->arena_ptr = nullptr;
  return ORRB_OK;
}

orrb_status orrb_workspace_size(orrb_ctx* ctx, const orrb_batch_shape* shape, const orrb_config* cfg, size_t* bytes) {
  if (!ctx || !bytes) return ORRB_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(ctx->mu);
  orrb_config c;
  resolve_config(cfg, &c);
  orrb_status st = check_config(ctx, c);
  if (st == ORRB_OK) st = check_shape(ctx, shape);
  if (st != ORRB_OK) return st;
  DeviceGuard dg(ctx->device);
  Plan P;
  st = plan(ctx, *shape, c, &P);
  if (st != ORRB_OK) return st;
  *bytes = P.total;
  return ORRB_OK;
}

orrb_status orrb_render_batch(orrb_ctx* ctx, const orrb_batch_shape* shape, const orrb_batch_desc* batch,
                              const orrb_outputs* out, const orrb_config* cfg, void* workspace, size_t ws_bytes,
                              void* stream) {
  if (!ctx) return ORRB_ERR_INVALID_ARG;
  Range range("orrb_render_batch");
  std::lock_guard<std::mutex> g(ctx->mu);
  if (!ctx->has_meshes) return fail(ctx, ORRB_ERR_NOT_FOUND, "upload meshes before rendering");
  orrb_config c;
  resolve_config(cfg, &c);
  orrb_status st = check_config(ctx, c);
  if (st == ORRB_OK) st = check_shape(ctx, shape);
  if (st == ORRB_OK) st = check_desc(ctx, batch);
  if (st != ORRB_OK) return st;
  if (!out) return fail(ctx, ORRB_ERR_INVALID_ARG, "null outputs");
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(ctx, ORRB_ERR_INVALID_ARG, "workspace must be a 256-byte aligned device pointer");
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return fail(ctx, ORRB_ERR_CUDA, "cudaSetDevice(%d) failed", ctx->device);
  Plan P;
  st = plan(ctx, *shape, c, &P);
  if (st != ORRB_OK) return st;
  if (ws_bytes < P.total) return fail(ctx, ORRB_ERR_WORKSPACE, "workspace needs %zu bytes, got %zu", P.total, ws_bytes);
  Params p{};
  fill_batch(p, *shape, *batch);
  p.rgb = out->rgb;
  p.depth = out->depth;
  p.normal = out->normal;
  p.seg = out->seg;
  p.rgb_linear = out->rgb_linear;
  p.rgb_graded = out->rgb_graded;
  p.gbuffer = out->gbuffer;
  p.tracker = out->tracker;
  p.shadow_map = out->shadow_map;
  if (p.shadow_res > 0 && !p.shadow_map) return fail(ctx, ORRB_ERR_INVALID_ARG, "a batch with shadows needs out->shadow_map");
  const ArenaLayout& A = ctx->arena;
  p.meshes = reinterpret_cast<const MeshEntry*>(ctx->arena_ptr + A.meshes);
  p.meshlets = reinterpret_cast<const MeshletEntry*>(ctx->arena_ptr + A.meshlets);
  p.cbounds = reinterpret_cast<const float4*>(ctx->arena_ptr + A.bounds);
  p.vpos = reinterpret_cast<const float4*>(ctx->arena_ptr + A.vpos);
  p.vnrm = reinterpret_cast<const float4*>(ctx->arena_ptr + A.vnrm);
  p.tris = reinterpret_cast<const uint32_t*>(ctx->arena_ptr + A.tris);
  p.n_meshes = A.n_meshes;
  p.tile_w = c.tile_w;
  p.tile_h = c.tile_h;
  p.max_tiles = P.max_tiles;
  char* ws = static_cast<char*>(workspace);
  p.status = reinterpret_cast<uint32_t*>(ws);
  p.work_counter = reinterpret_cast<uint32_t*>(ws + 4);
  p.images_done = reinterpret_cast<uint32_t*>(ws + 8);
  p.scratch = ws + 256;
  p.slot_bytes = P.slot_bytes;
  p.n_slots = P.n_slots;
  p.wait_cycles = c.wait_cycles;
  p.shadow_nb = p.shadow_res > 0 ? reinterpret_cast<uint32_t*>(ws + P.nb_offset) : nullptr;
  p.shadow_cnt = p.shadow_res > 0 ? reinterpret_cast<uint8_t*>(ws + P.cnt_offset) : nullptr;
  p.plain_sample = -1;
  p.stage_base = 0;
  // ambient occlusion and bloom: the camera launch writes the linear colour, depth and normals
  // (the caller's outputs where given, else the workspace's) and neither grades nor quantises; the
  // post pass then writes rgb and the graded colour
  PostParams pq{};
  const bool post = batch->post != nullptr;
  if (post) {
    if (!shape->post_effects)
      return fail(ctx, ORRB_ERR_INVALID_ARG, "batch.post needs shape.post_effects = 1 (it sizes the workspace)");
    pq.cam_wh = batch->cam_wh;
    pq.img_offset = batch->img_offset;
    pq.cam_intr = batch->cam_intr;
    pq.cam_sample = batch->cam_sample;
    pq.cam_offset = batch->cam_offset;
    pq.post = batch->post;
    pq.grading = batch->grading;
    pq.n_cams = shape->n_cams;
    pq.n_samples = shape->n_samples;
    pq.lin = out->rgb_linear ? out->rgb_linear : reinterpret_cast<float*>(ws + P.post_lin);
    pq.depth = out->depth ? out->depth : reinterpret_cast<float*>(ws + P.post_depth);
    pq.normal = out->normal ? out->normal : reinterpret_cast<uint16_t*>(ws + P.post_normal);
    pq.cao = reinterpret_cast<float*>(ws + P.post_cao);
    pq.hblur = reinterpret_cast<float*>(ws + P.post_hblur);
    pq.rgb = out->rgb;
    pq.rgb_graded = out->rgb_graded;
    p.rgb_linear = const_cast<float*>(pq.lin);
    p.depth = const_cast<float*>(pq.depth);
    p.normal = const_cast<uint16_t*>(pq.normal);
    p.rgb = nullptr;
    p.rgb_graded = nullptr;
    p.grading = nullptr;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(ws, 0, 16, s);
  if (e != cudaSuccess) return fail(ctx, ORRB_ERR_CUDA, "workspace clear: %s", cudaGetErrorString(e));
  if (shape->n_cams == 0 || shape->n_samples == 0) return ORRB_OK;
  st = enqueue_render(ctx, p, *shape, c.mode, c.threads, P.n_slots, ws, stream);
  if (st != ORRB_OK || !post) return st;
  char err[256] = {0};
  Range post_range("orrb post pass (ambient occlusion, bloom)");
  if (launch_post(pq, shape->max_width, shape->max_height, stream, err, sizeof(err)))
    return fail(ctx, ORRB_ERR_CUDA, "%s", err);
  return ORRB_OK;
}

orrb_status orrb_render_batch_noalloc(orrb_ctx* ctx, const orrb_batch_shape* shape, const orrb_batch_desc* batch,
                                      const orrb_outputs* out, const orrb_config* cfg, uint32_t* device_status,
                                      void* stream) {
  if (!ctx) return ORRB_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(ctx->mu);
  if (!ctx->has_meshes) return fail(ctx, ORRB_ERR_NOT_FOUND, "upload meshes before rendering");
  orrb_config c;
  resolve_config(cfg, &c);
  orrb_status st = check_config(ctx, c);
  if (st == ORRB_OK) st = check_shape(ctx, shape);
  if (st == ORRB_OK) st = check_desc(ctx, batch);
  if (st != ORRB_OK) return st;
  if (c.mode != ORRB_MODE_FUSED) return fail(ctx, ORRB_ERR_INVALID_ARG, "the allocation-free entry point runs the fused mode only");
  if (batch->post)
    return fail(ctx, ORRB_ERR_UNSUPPORTED, "the allocation-free entry point has no room for the post-processing images");
  if (!out) return fail(ctx, ORRB_ERR_INVALID_ARG, "null outputs");
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return fail(ctx, ORRB_ERR_CUDA, "cudaSetDevice(%d) failed", ctx->device);
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  int rc = noalloc_scratch(ctx->device, &scratch, &scratch_bytes);
  if (rc) return fail(ctx, ORRB_ERR_CUDA, "static scratch lookup: %s", cudaGetErrorString((cudaError_t)rc));
  Plan P;
  st = plan(ctx, *shape, c, &P);
  if (st != ORRB_OK) return st;
  const size_t fit = (scratch_bytes - 256) / P.slot_bytes;
  if (fit < 1)
    return fail(ctx, ORRB_ERR_WORKSPACE,
                "samples of up to %d triangles need %zu B of scratch per CTA; the static scratch holds %zu B",
                shape->max_tris_per_sample, P.slot_bytes, scratch_bytes - 256);
  const int n_slots = (int)std::min<size_t>((size_t)P.n_slots, fit);
  Params p{};
  fill_batch(p, *shape, *batch);
  p.rgb = out->rgb;
  p.depth = out->depth;
  p.normal = out->normal;
  p.seg = out->seg;
  p.rgb_linear = out->rgb_linear;
  p.rgb_graded = out->rgb_graded;
  p.gbuffer = out->gbuffer;
  p.tracker = out->tracker;
  p.shadow_map = out->shadow_map;
  if (p.shadow_res > 0 && !p.shadow_map) return fail(ctx, ORRB_ERR_INVALID_ARG, "a batch with shadows needs out->shadow_map");
  const ArenaLayout& A = ctx->arena;
  p.meshes = reinterpret_cast<const MeshEntry*>(ctx->arena_ptr + A.meshes);
  p.meshlets = reinterpret_cast<const MeshletEntry*>(ctx->arena_ptr + A.meshlets);
  p.cbounds = reinterpret_cast<const float4*>(ctx->arena_ptr + A.bounds);
  p.vpos = reinterpret_cast<const float4*>(ctx->arena_ptr + A.vpos);
  p.vnrm = reinterpret_cast<const float4*>(ctx->arena_ptr + A.vnrm);
  p.tris = reinterpret_cast<const uint32_t*>(ctx->arena_ptr + A.tris);
  p.n_meshes = A.n_meshes;
  p.tile_w = c.tile_w;
  p.tile_h = c.tile_h;
  p.max_tiles = P.max_tiles;
  char* ws = static_cast<char*>(scratch);
  p.status = device_status ? device_status : reinterpret_cast<uint32_t*>(ws);
  p.work_counter = reinterpret_cast<uint32_t*>(ws + 4);
  p.images_done = reinterpret_cast<uint32_t*>(ws + 8);
  p.scratch = ws + 256;
  p.slot_bytes = P.slot_bytes;
  p.wait_cycles = c.wait_cycles;
  p.plain_sample = -1;
  p.stage_base = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: the status word and the queue counters restart at zero
  cudaError_t e = cudaMemsetAsync(ws, 0, 16, s);
  if (e == cudaSuccess && device_status) e = cudaMemsetAsync(device_status, 0, 4, s);
  if (e != cudaSuccess) return fail(ctx, ORRB_ERR_CUDA, "scratch clear: %s", cudaGetErrorString(e));
  if (shape->n_cams == 0 || shape->n_samples == 0) return ORRB_OK;
  return enqueue_render(ctx, p, *shape, ORRB_MODE_FUSED, c.threads, n_slots, ws, stream, false);  // one slot per CTA
}

orrb_status orrb_read_status(orrb_ctx* ctx, const void* workspace, void* stream, uint32_t* status) {
  if (!ctx || !workspace || !status) return ORRB_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(ctx->mu);
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, workspace, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, ORRB_ERR_CUDA, "status read: %s", cudaGetErrorString(e));
  *status = v;
  return ORRB_OK;
}

static int backward_blocks_per_img(const orrb_batch_shape& s) {
  long long px = (long long)s.max_width * s.max_height;
  return (int)std::max<long long>(1, (px + 4095) / 4096);
}

orrb_status orrb_backward_workspace_size(orrb_ctx* ctx, const orrb_batch_shape* shape, size_t* bytes) {
  if (!ctx || !bytes) return ORRB_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(ctx->mu);
  orrb_status st = check_shape(ctx, shape);
  if (st != ORRB_OK) return st;
  *bytes = 256 + (size_t)std::max(shape->n_cams, 1) * backward_blocks_per_img(*shape) * kGradFloats * sizeof(float);
  return ORRB_OK;
}

orrb_status orrb_shade_backward(orrb_ctx* ctx, const orrb_batch_shape* shape, const orrb_batch_desc* batch,
                                const float* gbuffer, const float* d_rgb_linear, const orrb_param_grads* grads,
                                void* workspace, size_t ws_bytes, void* stream) {
  if (!ctx) return ORRB_ERR_INVALID_ARG;
  Range range("orrb_shade_backward");
  std::lock_guard<std::mutex> g(ctx->mu);
  orrb_status st = check_shape(ctx, shape);
  if (st == ORRB_OK) st = check_desc(ctx, batch);
  if (st != ORRB_OK) return st;
  if (!gbuffer || !d_rgb_linear || !grads) return fail(ctx, ORRB_ERR_INVALID_ARG, "null gbuffer, d_rgb or grads");
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(ctx, ORRB_ERR_INVALID_ARG, "workspace must be a 256-byte aligned device pointer");
  const int bpi = backward_blocks_per_img(*shape);
  size_t need = 256 + (size_t)std::max(shape->n_cams, 1) * bpi * kGradFloats * sizeof(float);
  if (ws_bytes < need) return fail(ctx, ORRB_ERR_WORKSPACE, "backward workspace needs %zu bytes, got %zu", need, ws_bytes);
  if (shape->n_cams == 0 || shape->n_samples == 0) return ORRB_OK;
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return fail(ctx, ORRB_ERR_CUDA, "cudaSetDevice(%d) failed", ctx->device);
  BackwardParams bp{};
  fill_batch(bp.base, *shape, *batch);
  bp.gbuffer = gbuffer;
  bp.d_rgb = d_rgb_linear;
  bp.d_material = grads->d_material;
  bp.d_light = grads->d_light;
  bp.d_exposure = grads->d_exposure;
  bp.d_emission = grads->d_emission;
  bp.d_grading = grads->d_grading;
  if (bp.d_grading && !batch->grading)
    return fail(ctx, ORRB_ERR_INVALID_ARG, "d_grading (a loss on the graded colour) needs a graded batch");
  if (bp.d_grading && batch->post)
    return fail(ctx, ORRB_ERR_UNSUPPORTED, "a loss on the graded colour is not differentiated through ambient occlusion and bloom");
  bp.partial = reinterpret_cast<float*>(static_cast<char*>(workspace) + 256);
  bp.blocks_per_img = bpi;
  char err[256] = {0};
  if (launch_backward(bp, 256, stream, err, sizeof(err))) return fail(ctx, ORRB_ERR_CUDA, "%s", err);
  return ORRB_OK;
}

}  // extern "C"
