// qs_probs_noalloc: Born-rule probabilities, an optional marginal and the fp64
// norm of a caller-owned amplitude buffer, without allocating any memory.
//
// Who needs it: code that must not call cudaMalloc/cudaFree (or any allocator)
// at the point where it wants outcome probabilities -- for example a host that
// owns all device memory through its own pool and forbids library allocations,
// a latency-critical loop where an allocation could block on the device, or a
// caller holding the amplitudes in its own buffer without creating a
// qs_state_t (whose creation allocates).  The working memory of the reduction
// (per-block partial sums and marginal accumulators) lives in one fixed-size
// array in device global memory, defined at file scope below; every device
// that loads this library holds that array until the process exits.
//
// Limits: at most kNaMaxQubits = 36 qubits and marginals over at most
// kNaMaxMargBits = 12 qubits (4096 accumulators); larger requests are rejected
// with QS_EINVAL.  All calls share the one array and it keeps the previous
// call's contents, so the marginal accumulators are cleared on every call and
// calls whose work overlaps on the GPU (different streams, or host threads
// without ordering) race on it.
#include <cuda_runtime.h>

#include "abi_guard.h"
#include "internal.h"

namespace qs {
namespace {

constexpr int kNaBlocks = 1024;           // reduction blocks (partial sums)
constexpr int kNaMaxMargBits = 12;        // largest marginal
constexpr int kNaMaxQubits = 36;
constexpr int kNaPartials = 0;                             // kNaBlocks doubles
constexpr int kNaResult = kNaBlocks;                       // 1 double (+ padding)
constexpr int kNaMarg = kNaBlocks + 32;                    // 2^kNaMaxMargBits doubles
constexpr int kNaDoubles = kNaMarg + (1 << kNaMaxMargBits);

// The scratch array (about 41 KB).  Host code must not pass its name to a
// kernel: on the host it is only a stand-in, so the device address is taken
// with cudaGetSymbolAddress on every call, for the device that is current then
// (after a device reset the address of the reloaded module is found again).
// With lazy module loading (CUDA_MODULE_LOADING=LAZY, the default) the driver
// loads this file's module, and places the array in device memory, at the
// first such lookup on each device: that first call is the one that is not
// free of allocation, so callers make it once outside the regions where they
// may not allocate.
static __device__ __align__(256) double g_noalloc_scratch[kNaDoubles];

__device__ double na_block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}

// p_J = |a_J|^2 into out (float or double, may be NULL); block partial sums of
// p (and the marginal accumulators when k > 0) into the scratch array
template <typename R, typename O>
__global__ void __launch_bounds__(256)
    na_probs_kernel(const C2<R>* __restrict__ psi, O* __restrict__ out, uint64_t N,
                    double* __restrict__ scratch, uint64_t mask, int k) {
  __shared__ double hist[1 << kNaMaxMargBits];
  __shared__ uint8_t bits[64];
  const int H = 1 << k;
  if (k > 0) {
    for (int i = threadIdx.x; i < H; i += blockDim.x) hist[i] = 0.0;
    if (threadIdx.x == 0) {
      int j = 0;
      for (int b = 0; b < 64; ++b)
        if ((mask >> b) & 1ull) bits[j++] = (uint8_t)b;
    }
    __syncthreads();
  }
  double acc = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t J = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; J < N; J += stride) {
    const C2<R> a = psi[J];
    const R p = a.x * a.x + a.y * a.y;
    if (out) out[J] = (O)p;
    acc += (double)p;
    if (k > 0) {
      int K = 0;
      for (int i = 0; i < k; ++i) K |= (int)((J >> bits[i]) & 1ull) << i;
      atomicAdd(hist + K, (double)p);
    }
  }
  if (k > 0) {
    __syncthreads();
    for (int i = threadIdx.x; i < H; i += blockDim.x)
      if (hist[i] != 0.0) atomicAdd(scratch + kNaMarg + i, hist[i]);
  }
  acc = na_block_sum(acc);
  if (threadIdx.x == 0) scratch[kNaPartials + blockIdx.x] = acc;
}

__global__ void na_clear_kernel(double* __restrict__ scratch, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) scratch[kNaMarg + i] = 0.0;
}

template <typename O>
__global__ void na_finish_kernel(double* __restrict__ scratch, int blocks, O* __restrict__ marg_out,
                                 int H) {
  double s = 0.0;
  for (int i = threadIdx.x; i < blocks; i += blockDim.x) s += scratch[kNaPartials + i];
  s = na_block_sum(s);
  if (threadIdx.x == 0) scratch[kNaResult] = s;
  if (marg_out)
    for (int i = threadIdx.x; i < H; i += blockDim.x) marg_out[i] = (O)scratch[kNaMarg + i];
}

// Device address of the scratch array on the current device.
qs_status na_scratch(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
  *out = (double*)p;
  return QS_OK;
}

template <typename R>
qs_status na_run(const void* amps, int n, void* out, int out_fp64, uint64_t mask, int k,
                 double* scratch, cudaStream_t s) {
  const uint64_t N = 1ull << n;
  const C2<R>* psi = (const C2<R>*)amps;
  if (k > 0) {
    na_clear_kernel<<<1, 256, 0, s>>>(scratch, 1 << k);
    if (out_fp64) na_probs_kernel<R, double><<<kNaBlocks, 256, 0, s>>>(psi, nullptr, N, scratch, mask, k);
    else na_probs_kernel<R, float><<<kNaBlocks, 256, 0, s>>>(psi, nullptr, N, scratch, mask, k);
    if (out_fp64) na_finish_kernel<double><<<1, 256, 0, s>>>(scratch, kNaBlocks, (double*)out, 1 << k);
    else na_finish_kernel<float><<<1, 256, 0, s>>>(scratch, kNaBlocks, (float*)out, 1 << k);
  } else {
    if (out_fp64) na_probs_kernel<R, double><<<kNaBlocks, 256, 0, s>>>(psi, (double*)out, N, scratch, 0, 0);
    else na_probs_kernel<R, float><<<kNaBlocks, 256, 0, s>>>(psi, (float*)out, N, scratch, 0, 0);
    na_finish_kernel<double><<<1, 256, 0, s>>>(scratch, kNaBlocks, (double*)nullptr, 0);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "qs_probs_noalloc launch");
  return QS_OK;
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status qs_probs_noalloc(const void* amps, int n, int prec, void* out, int out_fp64,
                                      uint64_t marg_mask, double* norm_out, void* stream) {
  return abi_guard(__func__, [&]() -> qs_status {
    if (!amps) {
      set_error("amps is NULL");
      return QS_EINVAL;
    }
    if (n < 1 || n > kNaMaxQubits) {
      set_error("n = %d outside [1, %d]", n, kNaMaxQubits);
      return QS_EINVAL;
    }
    if (prec != QS_C64 && prec != QS_C128) {
      set_error("bad precision %d", prec);
      return QS_EINVAL;
    }
    if (marg_mask >> n) {
      set_error("marginal mask has bits beyond n = %d", n);
      return QS_EINVAL;
    }
    int k = __builtin_popcountll(marg_mask);
    if (k == n) k = 0;   // all bits: plain probabilities
    if (k > kNaMaxMargBits) {
      set_error("qs_probs_noalloc: marginal over %d qubits exceeds its fixed scratch limit of %d qubits",
                k, kNaMaxMargBits);
      return QS_EINVAL;
    }
    double* scratch = nullptr;
    qs_status s = na_scratch(&scratch);
    if (s != QS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t mask = k ? marg_mask : 0;
    s = prec == QS_C64 ? na_run<float>(amps, n, out, out_fp64, mask, k, scratch, st)
                       : na_run<double>(amps, n, out, out_fp64, mask, k, scratch, st);
    if (s != QS_OK) return s;
    if (norm_out) {
      QS_CUDA(cudaMemcpyAsync(norm_out, scratch + kNaResult, sizeof(double), cudaMemcpyDeviceToHost, st));
      QS_CUDA(cudaStreamSynchronize(st));
    }
    return QS_OK;
  });
}
