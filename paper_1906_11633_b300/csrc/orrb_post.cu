// orrb_post.cu -- ambient occlusion and bloom of the rgb output (the post-processing randomizer's
// AO intensity and bloom intensity and radius, Sec. 4.3.1) for sm_103a.
//
// Runs after the camera launch, which then writes the linear colour, depth and binary16 normals of
// every pixel (to the caller's outputs or to the workspace) and neither grades nor quantises.
// Three launches over all images, each HBM-bound:
//   1  ambient occlusion: one thread per pixel samples eight fixed neighbours' depth and normal
//      and writes the occluded colour c_ao;
//   2  bloom along rows: a block stages one image row segment and its halo of bright parts
//      max(c_ao - 1, 0) in shared memory and writes their Gaussian blur along the row, H;
//   3  bloom along columns and the epilogue: a block stages a 32 x 32 tile of H and its halo rows,
//      blurs along the columns, adds beta times it to c_ao, grades, quantises and writes rgb (and
//      the graded colour).
// Images are flat over pixels (image c at img_offset[c]); blocks index (column block, row block,
// camera) and stride over the cameras beyond the grid's z extent.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "orrb.h"
#include "orrb_internal.h"
#include "orrb_shading.cuh"

namespace orrb {
namespace {

constexpr int kRowBlock = 128;   // pixels of a row per block in launches 1 and 2
constexpr int kMaxBloomR = 16;   // the blur's truncation radius is min(ceil(3 sigma), 16)
constexpr int kTile = 32;        // launch 3: 32 x 32 pixels per block, 32 x 8 threads
constexpr int kTileRows = 8;

struct PostImage {
  int W, H, s, R;
  long long base;
  float a, beta, sigma;
  bool bloom;
};

__device__ __forceinline__ PostImage post_image(const PostParams& q, int c) {
  PostImage m;
  m.W = q.cam_wh[2 * c];
  m.H = q.cam_wh[2 * c + 1];
  m.base = q.img_offset[c];
  int s = q.cam_sample[c];
  if (s < 0 || s >= q.n_samples) s = 0;  // (the camera launch flagged it already)
  m.s = s;
  m.a = q.post[4 * s];
  m.beta = q.post[4 * s + 1];
  m.sigma = q.post[4 * s + 2];
  m.bloom = m.beta != 0.0f && m.sigma > 0.0f;
  m.R = m.bloom ? min(int(ceilf(3.0f * m.sigma)), kMaxBloomR) : 0;
  return m;
}

// The normalised Gaussian weights w[-R..R] of the image's bloom (w[i + kMaxBloomR]), by the first
// warp; the caller synchronises the block before reading them.
__device__ void bloom_weights(const PostImage& m, float* w) {
  if (threadIdx.x >= 32 || threadIdx.y != 0) return;
  const int lane = threadIdx.x;
  const float k = -1.0f / (2.0f * m.sigma * m.sigma);
  float e0 = 0.0f, e1 = 0.0f;  // taps lane - R and lane + 32 - R
  if (lane <= 2 * m.R) e0 = expf(k * float((lane - m.R) * (lane - m.R)));
  if (lane + 32 <= 2 * m.R) e1 = expf(k * float((lane + 32 - m.R) * (lane + 32 - m.R)));
  float sum = e0 + e1;
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane <= 2 * m.R) w[lane - m.R + kMaxBloomR] = e0 / sum;
  if (lane + 32 <= 2 * m.R) w[lane + 32 - m.R + kMaxBloomR] = e1 / sum;
}

// 1: ambient occlusion.  P as the camera launch computes the G-buffer position (each operation
// rounded separately); the neighbours' positions the same way.
__global__ void __launch_bounds__(kRowBlock) post_ao_kernel(PostParams q) {
  const int x = blockIdx.x * kRowBlock + threadIdx.x, y = blockIdx.y;
  for (int c = blockIdx.z; c < q.n_cams; c += gridDim.z) {
    const PostImage m = post_image(q, c);
    if (x >= m.W || y >= m.H) continue;
    const long long i = m.base + (long long)y * m.W + x;
    float col[3] = {q.lin[3 * i], q.lin[3 * i + 1], q.lin[3 * i + 2]};
    const float d = q.depth[i];
    if (m.a != 0.0f && d > 0.0f) {
      const float* in = q.cam_intr + 6 * c;
      const float inv_fx = __frcp_rn(in[0]), inv_fy = __frcp_rn(in[1]), cx = in[2], cy = in[3];
      const bool ortho = in[5] != 0.0f;
      auto pos = [&](int px, int py, float dd, float P[3]) {
        const float ux = __fmul_rn(__fsub_rn(__fadd_rn(float(px), 0.5f), cx), inv_fx);
        const float uy = -__fmul_rn(__fsub_rn(__fadd_rn(float(py), 0.5f), cy), inv_fy);
        P[0] = ortho ? ux : __fmul_rn(dd, ux);
        P[1] = ortho ? uy : __fmul_rn(dd, uy);
        P[2] = -dd;
      };
      float P[3];
      pos(x, y, d, P);
      const float n[3] = {__half2float(__ushort_as_half(q.normal[3 * i])),
                          __half2float(__ushort_as_half(q.normal[3 * i + 1])),
                          __half2float(__ushort_as_half(q.normal[3 * i + 2]))};
      const int dx[8] = {2, -1, -4, 1, 5, -2, -5, 3}, dy[8] = {1, 3, -1, -4, 2, 5, -3, -6};
      float O = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int qx = x + dx[k], qy = y + dy[k];
        if (qx < 0 || qy < 0 || qx >= m.W || qy >= m.H) continue;
        const float dq = q.depth[m.base + (long long)qy * m.W + qx];
        if (!(dq > 0.0f)) continue;
        float Q[3];
        pos(qx, qy, dq, Q);
        const float v0 = Q[0] - P[0], v1 = Q[1] - P[1], v2 = Q[2] - P[2];
        const float L2 = v0 * v0 + v1 * v1 + v2 * v2;
        if (!(L2 > 0.0f)) continue;
        const float cosine = (n[0] * v0 + n[1] * v1 + n[2] * v2) * rsqrtf(L2) - 0.1f;
        if (cosine > 0.0f) O += cosine / (1.0f + L2 * 400.0f);  // (1 / 0.05^2)
      }
      const float f = fmaxf(0.0f, 1.0f - m.a * (O * 0.125f));
      for (int k = 0; k < 3; k++) col[k] *= f;
    }
    float* o = q.cao + 3 * i;
    o[0] = col[0];
    o[1] = col[1];
    o[2] = col[2];
  }
}

// 2: bloom along rows.  The block's row segment and R columns either side (indices clamped to the
// image) are staged as bright parts; each pixel sums its 2R + 1 taps.
__global__ void __launch_bounds__(kRowBlock) post_hblur_kernel(PostParams q) {
  __shared__ float4 bright[kRowBlock + 2 * kMaxBloomR];
  __shared__ float w[2 * kMaxBloomR + 1];
  const int x0 = blockIdx.x * kRowBlock, y = blockIdx.y, x = x0 + threadIdx.x;
  for (int c = blockIdx.z; c < q.n_cams; c += gridDim.z) {
    const PostImage m = post_image(q, c);
    if (!m.bloom || y >= m.H || x0 >= m.W) continue;  // (uniform over the block)
    bloom_weights(m, w);
    const long long row = m.base + (long long)y * m.W;
    for (int t = threadIdx.x; t < kRowBlock + 2 * m.R; t += kRowBlock) {
      const int xx = min(max(x0 - m.R + t, 0), m.W - 1);
      const float* v = q.cao + 3 * (row + xx);
      bright[t] = make_float4(fmaxf(v[0] - 1.0f, 0.0f), fmaxf(v[1] - 1.0f, 0.0f), fmaxf(v[2] - 1.0f, 0.0f), 0.0f);
    }
    __syncthreads();
    if (x < m.W) {
      float h0 = 0.0f, h1 = 0.0f, h2 = 0.0f;
      for (int i = -m.R; i <= m.R; i++) {
        const float4 b = bright[threadIdx.x + m.R + i];
        const float wi = w[i + kMaxBloomR];
        h0 = fmaf(wi, b.x, h0);
        h1 = fmaf(wi, b.y, h1);
        h2 = fmaf(wi, b.z, h2);
      }
      float* o = q.hblur + 3 * (row + x);
      o[0] = h0;
      o[1] = h1;
      o[2] = h2;
    }
    __syncthreads();  // (before the next camera's staging)
  }
}

// 3: bloom along columns, then the epilogue of the camera launch: grading (the same arithmetic as
// the camera launch's, so an image without AO and bloom gets the same bits) and quantisation.
__global__ void __launch_bounds__(kTile * kTileRows) post_final_kernel(PostParams q) {
  __shared__ float4 hs[(kTile + 2 * kMaxBloomR) * kTile];
  __shared__ float w[2 * kMaxBloomR + 1];
  __shared__ float gm[3][4];
  __shared__ float grain;
  __shared__ unsigned gkey;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile, x = x0 + tx;
  for (int c = blockIdx.z; c < q.n_cams; c += gridDim.z) {
    const PostImage m = post_image(q, c);
    if (x0 >= m.W || y0 >= m.H) continue;  // (uniform over the block)
    if (q.grading && tx == 0 && ty == 0) {
      const float* g = q.grading + (size_t)m.s * 8;
      grading_map(g, gm);
      grain = g[6];
      gkey = grain_key(g, unsigned(c - q.cam_offset[m.s]));
    }
    if (m.bloom) {
      bloom_weights(m, w);
      const int xx = min(x, m.W - 1);
      for (int r = ty; r < kTile + 2 * m.R; r += kTileRows) {
        const int yy = min(max(y0 - m.R + r, 0), m.H - 1);
        const float* v = q.hblur + 3 * (m.base + (long long)yy * m.W + xx);
        hs[r * kTile + tx] = make_float4(v[0], v[1], v[2], 0.0f);
      }
    }
    __syncthreads();
    for (int r = ty; r < kTile; r += kTileRows) {
      const int y = y0 + r;
      if (x >= m.W || y >= m.H) continue;
      const long long i = m.base + (long long)y * m.W + x;
      float col[3] = {q.cao[3 * i], q.cao[3 * i + 1], q.cao[3 * i + 2]};
      if (m.bloom) {
        float b0 = 0.0f, b1 = 0.0f, b2 = 0.0f;
        for (int j = -m.R; j <= m.R; j++) {
          const float4 h = hs[(r + m.R + j) * kTile + tx];
          const float wj = w[j + kMaxBloomR];
          b0 = fmaf(wj, h.x, b0);
          b1 = fmaf(wj, h.y, b1);
          b2 = fmaf(wj, h.z, b2);
        }
        col[0] = fmaf(m.beta, b0, col[0]);
        col[1] = fmaf(m.beta, b1, col[1]);
        col[2] = fmaf(m.beta, b2, col[2]);
      }
      if (q.grading) {
        const float o = grain * grain_centred(gkey, unsigned(y * m.W + x));
        const float r0 = col[0], g0 = col[1], b0 = col[2];
#pragma unroll
        for (int k = 0; k < 3; k++) col[k] = fmaf(gm[k][0], r0, fmaf(gm[k][1], g0, fmaf(gm[k][2], b0, gm[k][3] + o)));
      }
      if (q.rgb) {
        uint8_t* o = q.rgb + 3 * i;
#pragma unroll
        for (int k = 0; k < 3; k++) o[k] = (uint8_t)__float2uint_rd(fmaf(__saturatef(col[k]), 255.0f, 0.5f));
      }
      if (q.rgb_graded) {
        float* o = q.rgb_graded + 3 * i;
        o[0] = col[0];
        o[1] = col[1];
        o[2] = col[2];
      }
    }
    __syncthreads();  // (before the next camera's tables and staging)
  }
}

}  // namespace

int launch_post(const PostParams& q, int w_max, int h_max, void* stream, char* err, size_t errlen) {
  if (q.n_cams <= 0 || w_max <= 0 || h_max <= 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned gz = unsigned(q.n_cams < 65535 ? q.n_cams : 65535);
  const dim3 rows(unsigned((w_max + kRowBlock - 1) / kRowBlock), unsigned(h_max), gz);
  post_ao_kernel<<<rows, kRowBlock, 0, st>>>(q);
  post_hblur_kernel<<<rows, kRowBlock, 0, st>>>(q);
  const dim3 tiles(unsigned((w_max + kTile - 1) / kTile), unsigned((h_max + kTile - 1) / kTile), gz);
  post_final_kernel<<<tiles, dim3(kTile, kTileRows), 0, st>>>(q);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(err, errlen, "post-processing launch failed: %s", cudaGetErrorString(e));
    return 1;
  }
  return 0;
}

}  // namespace orrb
