// orrb_shadow_table.cu -- the neighbourhood table of the shadow maps for sm_103a.
//
// Runs between the depth-only shadow pass and the camera launch of a batch with shadow maps.
// Per texel it summarises the 3 x 3 neighbourhood that a percentage-closer lookup (3 x 3 taps,
// Reeves, Salesin and Cook 1987) reads, so that most lookups settle with one or two loads.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "orrb_internal.h"

namespace orrb {
namespace {

// The neighbourhood table of the shadow maps (after the shadow pass, before the camera launch):
// per texel over its 3 x 3 neighbourhood (texels outside the map count as empty), the least
// occupied depth (depth > 0; +inf if none), the largest (0 if none) and the number of occupied
// texels c.  A point with depth-less-bias zb is then unshadowed by every tap when zb <= the
// least, and shadowed by exactly the c occupied taps when zb > the largest (the empty ones
// light); only the others count taps.  The two depths are stored as binary16 rounded outward
// (the least down, the largest up), which keeps both shortcuts exact: what they cannot settle
// takes the nine taps.
// Each thread owns one column x of one map and walks down kNbRows rows of it, keeping the
// 3-texel summaries (least and largest occupied depth, occupied count) of the rows above, at
// and below in registers: three loads per texel.  A block covers 128 columns and kNbRows rows
// of one map (blocks stride over (map, column block, row block) triples).
constexpr int kNbRows = 32;

struct RowTriple {
  float lo, hi;
  int n;  // occupied texels among the three
};

__device__ __forceinline__ RowTriple row_triple(const float* map, int R, int x, int y) {
  RowTriple t{__int_as_float(0x7f800000), 0.0f, 0};
  if (y < 0 || y >= R) return t;
  const float* row = map + (size_t)y * R;
#pragma unroll
  for (int a = -1; a <= 1; a++) {
    const int xx = x + a;
    if (xx < 0 || xx >= R) continue;
    const float d = __ldg(row + xx);
    if (d > 0.0f) {
      t.lo = fminf(t.lo, d);
      t.hi = fmaxf(t.hi, d);
      t.n++;
    }
  }
  return t;
}

__global__ void __launch_bounds__(128) shadow_neighbourhood_kernel(Params p) {
  const int R = p.shadow_res, F = p.shadow_faces, n_maps = p.n_samples * kMaxLights * F;
  const int col_blocks = (R + 127) / 128, row_blocks = (R + kNbRows - 1) / kNbRows;
  const long long per_map = (long long)col_blocks * row_blocks;
  for (long long w = blockIdx.x; w < (long long)n_maps * per_map; w += gridDim.x) {
    const int m = int(w / per_map), wr = int(w % per_map);
    const int x = (wr % col_blocks) * 128 + int(threadIdx.x);
    const int y0 = (wr / col_blocks) * kNbRows, y1 = min(R, y0 + kNbRows);
    const int sl = m / F;  // sample * 4 + light
    if (sl % kMaxLights >= p.light_meta[(sl / kMaxLights) * 2] || p.shadow_intr[(size_t)m * 7] == 0.0f)
      continue;  // no such light, or a face that casts none: no map
    if (x >= R) continue;
    const float* map = p.shadow_map + (size_t)m * R * R;
    uint32_t* out = p.shadow_nb + (size_t)m * R * R + x;
    uint8_t* cnt = p.shadow_cnt + (size_t)m * R * R + x;
    RowTriple a = row_triple(map, R, x, y0 - 1), b = row_triple(map, R, x, y0);
#pragma unroll 4
    for (int y = y0; y < y1; y++) {
      const RowTriple c = row_triple(map, R, x, y + 1);
      const float lo = fminf(fminf(a.lo, b.lo), c.lo), hi = fmaxf(fmaxf(a.hi, b.hi), c.hi);
      out[(size_t)y * R] = unsigned(__half_as_ushort(__float2half_rd(lo))) |
                           (unsigned(__half_as_ushort(__float2half_ru(hi))) << 16);
      cnt[(size_t)y * R] = uint8_t(a.n + b.n + c.n);
      a = b;
      b = c;
    }
  }
}

// The same table, four columns per lane, for maps whose side is a multiple of 4 (and 16-byte
// aligned maps and table): a warp covers 128 columns and kNbRows rows of one map (warps stride
// over (map, column block, row block) triples).  Each lane loads a row's four texels with one
// 16-byte load and takes the texel left and right of them from its neighbours (lanes 0 and 31
// load theirs); a texel outside the map counts as empty, as in the scalar walk.  Minimum,
// maximum and count of the same nine texels do not depend on their order, so both kernels write
// the same table.
struct Row4 {
  float lo[4], hi[4];
  int n[4];
};

__device__ __forceinline__ void occ(float v, float& lo, float& hi, int& n) {
  const bool o = v > 0.0f;
  lo = o ? v : __int_as_float(0x7f800000);
  hi = o ? v : 0.0f;
  n = o;
}

__device__ __forceinline__ Row4 row4(const float* map, int R, int x, int y, bool in, int lane) {
  float4 c = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const bool row_in = y >= 0 && y < R;
  if (in && row_in) c = __ldg(reinterpret_cast<const float4*>(map + (size_t)y * R + x));
  float l = __shfl_up_sync(0xffffffffu, c.w, 1), r = __shfl_down_sync(0xffffffffu, c.x, 1);
  if (lane == 0) l = (in && row_in && x > 0) ? __ldg(map + (size_t)y * R + x - 1) : 0.0f;
  if (lane == 31) r = (in && row_in && x + 4 < R) ? __ldg(map + (size_t)y * R + x + 4) : 0.0f;
  if (x + 4 >= R) r = 0.0f;  // (the lane right of the last one holds no texel of this map)
  const float v[6] = {l, c.x, c.y, c.z, c.w, r};
  float lo[6], hi[6];
  int n[6];
#pragma unroll
  for (int i = 0; i < 6; i++) occ(v[i], lo[i], hi[i], n[i]);
  Row4 t;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    t.lo[i] = fminf(fminf(lo[i], lo[i + 1]), lo[i + 2]);
    t.hi[i] = fmaxf(fmaxf(hi[i], hi[i + 1]), hi[i + 2]);
    t.n[i] = n[i] + n[i + 1] + n[i + 2];
  }
  return t;
}

__global__ void __launch_bounds__(128) shadow_neighbourhood4_kernel(Params p) {
  const int R = p.shadow_res, F = p.shadow_faces, n_maps = p.n_samples * kMaxLights * F;
  const int col_blocks = (R + 127) / 128, row_blocks = (R + kNbRows - 1) / kNbRows;
  const long long per_map = (long long)col_blocks * row_blocks;
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < (long long)n_maps * per_map;
       w += warps) {
    const int m = int(w / per_map), wr = int(w % per_map);
    const int sl = m / F;  // sample * 4 + light
    if (sl % kMaxLights >= p.light_meta[(sl / kMaxLights) * 2] || p.shadow_intr[(size_t)m * 7] == 0.0f)
      continue;  // no such light, or a face that casts none: no map (the whole warp skips)
    const int x = (wr % col_blocks) * 128 + 4 * lane;
    const bool in = x < R;
    const int y0 = (wr / col_blocks) * kNbRows, y1 = min(R, y0 + kNbRows);
    const float* map = p.shadow_map + (size_t)m * R * R;
    uint32_t* out = p.shadow_nb + (size_t)m * R * R + x;
    uint8_t* cnt = p.shadow_cnt + (size_t)m * R * R + x;
    Row4 a = row4(map, R, x, y0 - 1, in, lane), b = row4(map, R, x, y0, in, lane);
#pragma unroll 2
    for (int y = y0; y < y1; y++) {
      const Row4 c = row4(map, R, x, y + 1, in, lane);
      uint32_t e[4];
      uint32_t nn = 0;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const float lo = fminf(fminf(a.lo[i], b.lo[i]), c.lo[i]), hi = fmaxf(fmaxf(a.hi[i], b.hi[i]), c.hi[i]);
        e[i] = unsigned(__half_as_ushort(__float2half_rd(lo))) | (unsigned(__half_as_ushort(__float2half_ru(hi))) << 16);
        nn |= uint32_t(a.n[i] + b.n[i] + c.n[i]) << (8 * i);
      }
      if (in) {
        *reinterpret_cast<uint4*>(out + (size_t)y * R) = make_uint4(e[0], e[1], e[2], e[3]);
        *reinterpret_cast<uint32_t*>(cnt + (size_t)y * R) = nn;
      }
      a = b;
      b = c;
    }
  }
}

}  // namespace

int launch_shadow_neighbourhoods(const Params& p, void* stream, char* err, size_t errlen) {
  const int n_maps = p.n_samples * kMaxLights * p.shadow_faces;
  const long long work = (long long)n_maps * ((p.shadow_res + 127) / 128) * ((p.shadow_res + kNbRows - 1) / kNbRows);
  const bool vec = p.shadow_res % 4 == 0 && (reinterpret_cast<uintptr_t>(p.shadow_map) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(p.shadow_nb) & 15) == 0 && (reinterpret_cast<uintptr_t>(p.shadow_cnt) & 3) == 0;
  if (vec) {  // one warp per work item, four per block
    const long long blocks = (work + 3) / 4;
    shadow_neighbourhood4_kernel<<<unsigned(blocks < (1 << 30) ? blocks : (1 << 30)), 128, 0,
                                   static_cast<cudaStream_t>(stream)>>>(p);
  } else {
    shadow_neighbourhood_kernel<<<unsigned(work < (1 << 30) ? work : (1 << 30)), 128, 0,
                                  static_cast<cudaStream_t>(stream)>>>(p);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(err, errlen, "shadow neighbourhood launch failed: %s", cudaGetErrorString(e));
    return 1;
  }
  return 0;
}

}  // namespace orrb
