// orrb_fp32_peak.cu -- a measured FP32 peak for the shading roofline.
//
// The shading roofline divides the algorithmic FP32 operations by the chip's FP32 rate.  This
// probe measures that rate on the device it runs on: every thread runs independent chains of
// fused multiply-adds (enough chains that the pipe, not the dependency latency, limits them), in
// two forms: scalar FFMA (one multiply-add per lane per instruction) and the packed
// two-element form of sm_100 and later (__ffma2_rn, two per lane per instruction).  A
// multiply-add counts as two operations.  The host times a launch with CUDA events after a warm-up
// launch and returns operations per second of the faster form, with both figures beside it.
//
// Built into its own library (libfp32peak.so); it is measurement infrastructure, not part of the
// renderer's C-ABI.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kChains = 16;  // independent accumulators per thread (ILP)

__global__ void __launch_bounds__(256) ffma_chain(float* out, int iters, float a, float b) {
  float acc[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) acc[k] = float(threadIdx.x + k);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < kChains; k++) acc[k] = fmaf(acc[k], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += acc[k];
  if (s == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(256) ffma2_chain(float* out, int iters, float a, float b) {
  float2 acc[kChains / 2];
#pragma unroll
  for (int k = 0; k < kChains / 2; k++) acc[k] = make_float2(float(threadIdx.x + 2 * k), float(threadIdx.x + 2 * k + 1));
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < kChains / 2; k++) acc[k] = __ffma2_rn(acc[k], a2, b2);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains / 2; k++) s += acc[k].x + acc[k].y;
  if (s == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

// Measures FP32 multiply-add throughput on the current device.  flops_scalar, flops_packed:
// operations per second of the scalar and the packed form (each the best of `reps` timed
// launches).  Returns 0, or a CUDA error code.  Allocates a small scratch buffer (cudaMalloc) and
// frees it.
int orrb_measure_fp32_peak(int reps, double* flops_scalar, double* flops_packed) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int threads = 256, blocks = sms * 8, iters = 16384;
  float* out = nullptr;
  e = cudaMalloc(&out, sizeof(float) * blocks * threads);
  if (e != cudaSuccess) return (int)e;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  const double ops = 2.0 * kChains * (double)iters * blocks * threads;
  double best[2] = {0.0, 0.0};
  for (int form = 0; form < 2 && e == cudaSuccess; form++) {
    for (int r = -1; r < reps && e == cudaSuccess; r++) {  // r = -1: warm-up
      cudaEventRecord(t0);
      if (form == 0) ffma_chain<<<blocks, threads>>>(out, iters, 0.999f, 0.001f);
      else ffma2_chain<<<blocks, threads>>>(out, iters, 0.999f, 0.001f);
      cudaEventRecord(t1);
      e = cudaEventSynchronize(t1);
      if (e == cudaSuccess) e = cudaGetLastError();
      float ms = 0.0f;
      if (e == cudaSuccess && r >= 0 && cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess && ms > 0.0f) {
        const double f = ops / (ms * 1e-3);
        if (f > best[form]) best[form] = f;
      }
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(out);
  if (e != cudaSuccess) return (int)e;
  *flops_scalar = best[0];
  *flops_packed = best[1];
  return 0;
}

}  // extern "C"
