// [[4,2,2]] error-detection evaluation, simulation side (Eq.
// (errordetectionDbareenc)): from the outcome probabilities of the encoded
// (5 qubits: ancilla q0, data q1..q4) and bare (2 qubits) versions of a logical
// circuit, the postselected logical distribution -- outcomes with the ancilla
// flag q0 = 1 or an odd number of 1's on q1 q2 q3 q4 discarded, the rest mapped
// onto the logical basis of Eqs. (errordetection00L)-(errordetection11L) and
// renormalised -- the postselection ratio, and the statistical distances of the
// bare and encoded distributions to the ideal one.  A masked reduction, one
// thread per circuit, FP64 sums.
#include <cuda_runtime.h>

#include "abi_guard.h"
#include "internal.h"

namespace qs {
namespace {

// logical index (2 j0 + j1) of the data word w = q1 + 2 q2 + 4 q3 + 8 q4, -1 for
// odd parity: 0000, 1111 -> 00; 1100, 0011 -> 01; 1010, 0101 -> 10; 0110, 1001 -> 11
// (strings written q1 q2 q3 q4)
__constant__ int8_t c_logical[16] = {0, -1, -1, 1, -1, 2, 3, -1, -1, 3, 2, -1, 1, -1, -1, 0};

__global__ void __launch_bounds__(256)
    code422_eval_kernel(int count, const float* __restrict__ enc, const float* __restrict__ bare,
                        const float* __restrict__ ideal, float* __restrict__ p_enc,
                        float* __restrict__ ratio, float* __restrict__ d_bare, float* __restrict__ d_enc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= count) return;
  double q[4] = {0, 0, 0, 0};
  const float* e = enc + (size_t)c * 32;
#pragma unroll
  for (int J = 0; J < 32; J += 2) {   // even J: ancilla q0 = 0
    const int L = c_logical[J >> 1];
    if (L >= 0) q[L] += (double)e[J];
  }
  const double kept = q[0] + q[1] + q[2] + q[3];
  double db = 0, de = 0;
#pragma unroll
  for (int L = 0; L < 4; ++L) {
    const double pe = kept > 0 ? q[L] / kept : 0.0, pid = ideal[(size_t)c * 4 + L];
    p_enc[(size_t)c * 4 + L] = (float)pe;
    db += fabs((double)bare[(size_t)c * 4 + L] - pid);
    de += fabs(pe - pid);
  }
  ratio[c] = (float)kept;
  d_bare[c] = (float)(0.5 * db);
  d_enc[c] = (float)(0.5 * de);
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status dm_code422_eval(int count, const float* enc, const float* bare, const float* ideal,
                                     float* p_enc, float* ratio, float* d_bare, float* d_enc, void* stream) {
  return abi_guard(__func__, [&]() -> qs_status {
    if (count < 0 || (count > 0 && (!enc || !bare || !ideal || !p_enc || !ratio || !d_bare || !d_enc))) {
      set_error("dm_code422_eval: count < 0 or an array is NULL");
      return QS_EINVAL;
    }
    if (count == 0) return QS_OK;
    code422_eval_kernel<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(count, enc, bare, ideal, p_enc,
                                                                               ratio, d_bare, d_enc);
    QS_CUDA(cudaGetLastError());
    return QS_OK;
  });
}
