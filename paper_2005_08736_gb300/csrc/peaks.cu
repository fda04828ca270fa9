// Measured arithmetic peaks of the current GPU: the throughput of fused
// multiply-adds in FP32, in packed FP32 pairs (one instruction performs two
// FP32 FMAs on a float2) and in FP64.  These are the denominators of the
// ALU rooflines of the step's kernels; the scheme itself has no part here.
//
// Each thread runs kChains independent FMA chains for `iters` iterations, so
// that the FMA latency is hidden by the chains and by the resident warps; the
// grid holds 8 CTAs of 256 threads per SM.  The chains' final values are
// written out so that the compiler cannot remove them.
#include <cuda_runtime.h>

#include "hgks.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_peak_f32(int iters, float a, float b, float* out) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = float(threadIdx.x + c) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_f32x2(int iters, float a, float b, float* out) {
  float2 x[kChains];
  const float2 av = make_float2(a, a), bv = make_float2(b, b);
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2(float(threadIdx.x + c) * 1e-3f, float(c) * 1e-3f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], av, bv);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  out[blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_f64(int iters, double a, double b, float* out) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = double(threadIdx.x + c) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * kThreads + threadIdx.x] = float(s);
}

}  // namespace

extern "C" hgks_status hgks_measure_fp_peaks(void* stream, double* tflops_out) {
  if (!tflops_out) return HGKS_E_INVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HGKS_E_CUDA;
  const int blocks = sms * 8;
  const double threads = double(blocks) * kThreads;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * blocks * kThreads) != cudaSuccess) return HGKS_E_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // Iterations per kind: about 10 ms per timed launch at the nominal rates.
  const int iters[3] = {40000, 20000, 1000};
  // flops per chain iteration: one FMA = 2 flops, a packed pair 4.
  const double per[3] = {2.0, 4.0, 2.0};
  hgks_status st = HGKS_OK;
  for (int k = 0; k < 3 && st == HGKS_OK; ++k) {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {  // the first launch warms up the clocks
      cudaEventRecord(e0, s);
      if (k == 0) k_peak_f32<<<blocks, kThreads, 0, s>>>(iters[k], 0.999999f, 1e-7f, out);
      else if (k == 1) k_peak_f32x2<<<blocks, kThreads, 0, s>>>(iters[k], 0.999999f, 1e-7f, out);
      else k_peak_f64<<<blocks, kThreads, 0, s>>>(iters[k], 0.999999999, 1e-12, out);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = HGKS_E_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best) best = ms;
    }
    if (st == HGKS_OK)
      tflops_out[k] = per[k] * kChains * double(iters[k]) * threads / (double(best) * 1e-3) / 1e12;
  }
  if (cudaGetLastError() != cudaSuccess) st = HGKS_E_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return st;
}
