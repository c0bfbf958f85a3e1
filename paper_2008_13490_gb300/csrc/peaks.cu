// Arithmetic peaks of the GPU this runs on, measured: the denominators of the
// rooflines of the kernels that are bound by plain FP32 or FP64 arithmetic
// rather than by HBM (the tile passes, the batched Pauli-vector kernel, the FP64
// paths).  Not part of the thesis's computation.
//
// Each thread runs kChains independent multiply-add chains (enough instruction-
// level parallelism to hide the pipeline latency) for `iters` iterations; the
// grid fills every SM with 2048 threads.  FP32 uses packed FP32x2 multiply-adds
// (two FMAs per instruction, the form the state-vector kernels issue), FP64
// plain DFMA.  flops = 2 per FMA.
#include <cuda_runtime.h>

#include "abi_guard.h"
#include "internal.h"

namespace qs {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) peak_fp32_kernel(float* out, float a, float b, int iters) {
  float2 acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = make_float2(threadIdx.x * 1e-3f + c, blockIdx.x * 1e-3f - c);
  const float2 va = make_float2(a, -a), vb = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = __ffma2_rn(acc[c], va, vb);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c].x + acc[c].y;
  if (s == 1234.5f) out[blockIdx.x] = s;   // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(kPeakThreads) peak_fp64_kernel(double* out, double a, double b, int iters) {
  double acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = threadIdx.x * 1e-3 + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  if (s == 1234.5) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status qs_alu_peak(int kind, double* flops_per_s, int* sm_count, double* ms_out, void* stream_) {
  return abi_guard(__func__, [&]() -> qs_status {
    if (!flops_per_s || (kind != 0 && kind != 1)) {
      set_error("qs_alu_peak: kind 0 (FP32) or 1 (FP64) and an output are required");
      return QS_EINVAL;
    }
    int dev = 0, sms = 0;
    QS_CUDA(cudaGetDevice(&dev));
    QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t stream = (cudaStream_t)stream_;
    const int blocks = sms * (2048 / kPeakThreads);
    // about 30 ms per launch at the nominal rates (FP32 ~80 TFLOP/s, FP64 ~1.3 TFLOP/s)
    const int iters = kind == 0 ? (1 << 18) : (1 << 13);
    cudaEvent_t e0, e1;
    QS_CUDA(cudaEventCreate(&e0));
    QS_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {   // the first launch warms up; the best of the rest counts
      cudaEventRecord(e0, stream);
      if (kind == 0) peak_fp32_kernel<<<blocks, kPeakThreads, 0, stream>>>(nullptr, 0.999f, 1e-3f, iters);
      else peak_fp64_kernel<<<blocks, kPeakThreads, 0, stream>>>(nullptr, 0.999, 1e-3, iters);
      cudaEventRecord(e1, stream);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_status(e, "qs_alu_peak");
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double fmas = (double)blocks * kPeakThreads * iters * kChains * (kind == 0 ? 2.0 : 1.0);
    *flops_per_s = 2.0 * fmas / (best * 1e-3);
    if (sm_count) *sm_count = sms;
    if (ms_out) *ms_out = best;
    return QS_OK;
  });
}
