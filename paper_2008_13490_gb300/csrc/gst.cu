// GST predictions for repeated gates (Eq. (GSTPrediction)):
//   p_J(r) = <<E_J| (G_s)^r G_(prep) |rho>>
// with Pauli transfer matrices on 1- or 2-qubit Pauli vectors (4^n <= 16).
//
//  gst_series_kernel  every r = 1..r_max, one warp per sequence: lane j < D
//                     holds entry j of the Pauli vector and row j of G_s (FP32
//                     registers); a step broadcasts the vector by shuffles, the
//                     lanes j < D form G v and lanes D..D+2^n-1, holding the
//                     effect rows, form the probabilities of the vector they saw.
//  gst_power_kernel   one r per sequence by repeated squaring (the binary digits
//                     of r: about 2 log2 r products of D x D matrices), FP64,
//                     one CTA per sequence, thread (i, k) forming entry (i, k).
#include <cuda_runtime.h>

#include <vector>

#include "abi_guard.h"
#include "internal.h"

namespace qs {
namespace {

constexpr int kGstMaxD = 16;
constexpr int kGstMaxPrep = 8;

struct GstArgs {
  int n, D, count, r_max, n_ptm;
  const double* ptms;
  const double* rho;
  const double* effects;
  const int32_t* gate;
  const int32_t* prep;   // count x kGstMaxPrep, -1 = end
};

// the sequence's gate and preparation indices address the PTM table (the arrays
// are caller-supplied device memory, so the kernels check them)
__device__ __forceinline__ bool seq_valid(const GstArgs& A, int seq) {
  if (A.gate[seq] < 0 || A.gate[seq] >= A.n_ptm) return false;
  for (int k = 0; k < kGstMaxPrep; ++k) {
    const int pk = A.prep[seq * kGstMaxPrep + k];
    if (pk < -1 || pk >= A.n_ptm) return false;
    if (pk < 0) break;
  }
  return true;
}

// v <- P v on the warp (lane j < D holds v_j)
__device__ __forceinline__ float warp_matvec(const double* P, float v, int D, int lane) {
  float acc = 0.f;
  for (int k = 0; k < D; ++k) {
    const float vk = __shfl_sync(0xffffffffu, v, k);
    if (lane < D) acc = fmaf((float)P[lane * D + k], vk, acc);
  }
  return lane < D ? acc : 0.f;
}

__global__ void __launch_bounds__(256) gst_series_kernel(GstArgs A, float* __restrict__ probs) {
  const int lane = threadIdx.x & 31;
  const int seq = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (seq >= A.count) return;   // whole warps leave together
  const int D = A.D, NJ = 1 << A.n;
  if (!seq_valid(A, seq)) {   // a bad index: NaN outputs
    for (int i = lane; i < A.r_max * NJ; i += 32)
      probs[(size_t)seq * A.r_max * NJ + i] = __int_as_float(0x7fc00000);
    return;
  }
  // G_(prep) |rho>>
  float v = lane < D ? (float)A.rho[lane] : 0.f;
  for (int k = 0; k < kGstMaxPrep; ++k) {
    const int pk = A.prep[seq * kGstMaxPrep + k];
    if (pk < 0) break;
    v = warp_matvec(A.ptms + (size_t)pk * D * D, v, D, lane);
  }
  // row of G_s (lanes < D) or effect row (lanes D .. D + 2^n - 1)
  float row[kGstMaxD];
  const double* G = A.ptms + (size_t)A.gate[seq] * D * D;
  const bool eff = lane >= D && lane < D + NJ;
#pragma unroll
  for (int k = 0; k < kGstMaxD; ++k) {
    float x = 0.f;
    if (k < D) {
      if (lane < D) x = (float)G[lane * D + k];
      else if (eff) x = (float)A.effects[(lane - D) * D + k];
    }
    row[k] = x;
  }
  float* out = probs + (size_t)seq * A.r_max * NJ;
  // step r: broadcast v_{r-1}; lanes < D form v_r, effect lanes p(r - 1) (r >= 2)
  for (int r = 1; r <= A.r_max + 1; ++r) {
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < kGstMaxD; ++k) {
      if (k >= D) break;
      acc = fmaf(row[k], __shfl_sync(0xffffffffu, v, k), acc);
    }
    if (eff && r >= 2) out[(size_t)(r - 2) * NJ + (lane - D)] = acc;
    if (lane < D) v = acc;
  }
}

__global__ void __launch_bounds__(256) gst_power_kernel(GstArgs A, const int64_t* __restrict__ reps,
                                                        double* __restrict__ probs) {
  __shared__ double R[kGstMaxD * kGstMaxD], B[kGstMaxD * kGstMaxD], T[kGstMaxD * kGstMaxD];
  __shared__ double v[kGstMaxD], w[kGstMaxD];
  const int seq = blockIdx.x, D = A.D, t = threadIdx.x;
  const int i = t / kGstMaxD, k = t % kGstMaxD;   // entry (i, k) of a product
  const bool ent = i < D && k < D;
  if (reps[seq] < 0 || !seq_valid(A, seq)) {   // the same for every thread of the CTA
    if (t < (1 << A.n)) probs[(size_t)seq * (1 << A.n) + t] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  if (t < D) v[t] = A.rho[t];
  __syncthreads();
  for (int q = 0; q < kGstMaxPrep; ++q) {
    const int pk = A.prep[seq * kGstMaxPrep + q];
    if (pk < 0) break;
    const double* P = A.ptms + (size_t)pk * D * D;
    if (t < D) {
      double acc = 0.0;
      for (int m = 0; m < D; ++m) acc = fma(P[t * D + m], v[m], acc);
      w[t] = acc;
    }
    __syncthreads();
    if (t < D) v[t] = w[t];
    __syncthreads();
  }
  const double* G = A.ptms + (size_t)A.gate[seq] * D * D;
  if (ent) {
    R[i * D + k] = i == k ? 1.0 : 0.0;
    B[i * D + k] = G[i * D + k];
  }
  __syncthreads();
  // R = G^r: for each binary digit of r (low first) R <- R B if set, then B <- B B
  for (uint64_t e = (uint64_t)reps[seq]; e; e >>= 1) {
    if (e & 1) {
      if (ent) {
        double acc = 0.0;
        for (int m = 0; m < D; ++m) acc = fma(R[i * D + m], B[m * D + k], acc);
        T[i * D + k] = acc;
      }
      __syncthreads();
      if (ent) R[i * D + k] = T[i * D + k];
      __syncthreads();
    }
    if (e > 1) {
      if (ent) {
        double acc = 0.0;
        for (int m = 0; m < D; ++m) acc = fma(B[i * D + m], B[m * D + k], acc);
        T[i * D + k] = acc;
      }
      __syncthreads();
      if (ent) B[i * D + k] = T[i * D + k];
      __syncthreads();
    }
  }
  // p_J = <<E_J| R v
  if (t < D) {
    double acc = 0.0;
    for (int m = 0; m < D; ++m) acc = fma(R[t * D + m], v[m], acc);
    w[t] = acc;
  }
  __syncthreads();
  const int NJ = 1 << A.n;
  if (t < NJ) {
    double acc = 0.0;
    for (int m = 0; m < D; ++m) acc = fma(A.effects[t * D + m], w[m], acc);
    probs[(size_t)seq * NJ + t] = acc;
  }
}

qs_status gst_args(const qs_gst_batch* b, GstArgs* A, cudaStream_t stream) {
  if (!b) {
    set_error("batch is NULL");
    return QS_EINVAL;
  }
  if (b->n < 1 || b->n > 2 || b->count < 0 || b->n_ptm < 1) {
    set_error("GST batch: n = %d (1 or 2), count = %d, n_ptm = %d", b->n, b->count, b->n_ptm);
    return QS_EINVAL;
  }
  if (!b->ptms || !b->rho || !b->effects || (b->count > 0 && (!b->gate || !b->prep))) {
    set_error("GST batch arrays missing");
    return QS_EINVAL;
  }
  if (b->flags & ~QS_DM_VALIDATE) {
    set_error("unknown GST batch flags 0x%x", b->flags);
    return QS_EINVAL;
  }
  if (b->flags & QS_DM_VALIDATE) {   // every PTM of the table must be a channel
    const size_t D = (size_t)1 << (2 * b->n);
    std::vector<double> h((size_t)b->n_ptm * D * D);
    QS_CUDA(cudaMemcpyAsync(h.data(), b->ptms, h.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
    QS_CUDA(cudaStreamSynchronize(stream));
    const qs_status s = ptm_validate(h.data(), b->n, b->n_ptm, "ptms", nullptr);
    if (s != QS_OK) return s;
  }
  A->n = b->n;
  A->D = 1 << (2 * b->n);
  A->count = b->count;
  A->r_max = b->r_max;
  A->n_ptm = b->n_ptm;
  A->ptms = b->ptms;
  A->rho = b->rho;
  A->effects = b->effects;
  A->gate = b->gate;
  A->prep = b->prep;
  return QS_OK;
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status dm_gst_series(const qs_gst_batch* b, float* probs, void* stream) {
  return abi_guard(__func__, [&]() -> qs_status {
    GstArgs A;
    qs_status s = gst_args(b, &A, (cudaStream_t)stream);
    if (s != QS_OK) return s;
    if (A.r_max < 1 || !probs) {
      set_error("GST series needs r_max >= 1 and an output");
      return QS_EINVAL;
    }
    if (A.count == 0) return QS_OK;
    const int warps = 8;
    gst_series_kernel<<<(A.count + warps - 1) / warps, 32 * warps, 0, (cudaStream_t)stream>>>(A, probs);
    QS_CUDA(cudaGetLastError());
    return QS_OK;
  });
}

extern "C" qs_status dm_gst_power(const qs_gst_batch* b, const int64_t* reps, double* probs, void* stream) {
  return abi_guard(__func__, [&]() -> qs_status {
    GstArgs A;
    qs_status s = gst_args(b, &A, (cudaStream_t)stream);
    if (s != QS_OK) return s;
    if (!reps || !probs) {
      set_error("GST power needs reps and an output");
      return QS_EINVAL;
    }
    if (A.count == 0) return QS_OK;
    gst_power_kernel<<<A.count, 256, 0, (cudaStream_t)stream>>>(A, reps, probs);
    QS_CUDA(cudaGetLastError());
    return QS_OK;
  });
}
