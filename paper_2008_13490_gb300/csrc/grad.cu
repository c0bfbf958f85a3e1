// Adjoint gradient of a probability functional of the final state.
//
// L(p) with p_J = |psi_J|^2 and psi = U_G ... U_1 psi_0.  With
// lambda = dL/dpsi^* = (dL/dp_J) psi_J at the end, the derivative with
// respect to an angle t of gate g is
//     dL/dt = 2 Re <lambda_g | dU_g/dt | psi_{g-1}>,
// where lambda_g = U_{g+1}^dagger ... U_G^dagger lambda and psi_{g-1} the
// state before gate g.  The sweep runs backwards over the gates.  For n >= 12
// it runs in fused tile passes (adjoint_pass_kernel: a tile of both states in
// registers, the U^dagger and derivative terms of all of a pass's gates in one
// read+write of psi and lambda; dL/dt = 2 Re <lambda_g | G psi_g> with
// G = (dU/dt) U^dagger).  Otherwise one kernel per gate computes
// psi_{g-1} = U_g^dagger psi_g, the derivative terms (fp64 block partials) and
// lambda_{g-1} = U_g^dagger lambda_g.
// Rotation derivatives follow from R(t) = exp(-i t sigma/2)
// (Eqs. (singlequbitrotationx)-(singlequbitrotationz)): dR/dt = -i/2 sigma R.
//
// States come either from uncomputing (psi <- U^dagger psi) or, for deep
// circuits, from checkpoints stored every K gates in the forward pass: each
// segment's final state is recomputed from its checkpoint and the segment is
// then swept backwards (fused), or its per-gate states are recomputed (per gate).
#include <cuda_runtime.h>

#include <cstring>

#include "abi_guard.h"
#include "internal.h"

namespace qs {

namespace {

template <typename R>
__device__ __forceinline__ C2<R> cmac(C2<R> acc, C2<R> m, C2<R> a) {
  acc.x = fma(m.x, a.x, acc.x);
  acc.x = fma(-m.y, a.y, acc.x);
  acc.y = fma(m.x, a.y, acc.y);
  acc.y = fma(m.y, a.x, acc.y);
  return acc;
}

// Gate matrices in the state's precision (converted on the host: a conversion
// from FP64 on the device runs on the slow FP64 pipe, and the compiler may
// repeat it at every use instead of keeping 32 values in registers).
template <typename R>
struct GradGate {
  int k;            // 1 or 2 qubits
  int q0, q1;       // q0 most significant of the local index
  int np;           // number of parameters
  C2<R> ud[16];     // U^dagger, complex row-major (k=1: 2x2 in the first 4)
  C2<R> du[3][16];  // dU/dt_p
};

__device__ double block_sum_g(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  __syncthreads();
  return s;
}

__device__ __forceinline__ uint64_t ins0(uint64_t i, int b) {
  const uint64_t m = (1ull << b) - 1ull;
  return ((i & ~m) << 1) | (i & m);
}

// Per-thread sum of the derivative terms.  For a complex64 state the terms are
// formed in FP32 and added with Kahan compensation, the block adds its threads'
// sums in FP32 (pairwise) and only the per-block sums are FP64 (GB300's FP64
// pipe is far slower than its FP32 pipe; one FP64 add per element made this
// HBM kernel FP64-bound).  For a complex128 state everything is FP64.  Each
// thread walks its groups in chunks of kChunkG.
constexpr int kChunkG = 32;
template <typename R>
struct TermSum {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct TermSum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// block sum of the threads' term sums, valid in thread 0: FP32 within the block
// for a complex64 state (a pairwise tree; the blocks' sums are added in FP64),
// FP64 throughout for a complex128 state
__device__ __forceinline__ double block_sum_terms(float v, float* redf, double*) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) redf[w] = v;
  __syncthreads();
  double sum = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) sum += (double)redf[i];
  return sum;
}
__device__ __forceinline__ double block_sum_terms(double v, float*, double* red) { return block_sum_g(v, red); }

// one backward step of a K-qubit gate: psi <- U^dagger psi, the derivative
// terms, lam <- U^dagger lam (K a template parameter so that the amplitude
// arrays stay in registers; the matrices are converted to R once per thread)
template <typename R, int K>
__global__ void __launch_bounds__(256)
    adjoint_step_kernel(C2<R>* __restrict__ psi, C2<R>* __restrict__ lam, int n, GradGate<R> g,
                        double* __restrict__ partials, unsigned* __restrict__ done, double* __restrict__ out3,
                        int psi_is_before) {
  constexpr int d = 1 << K;
  constexpr int NP = K == 1 ? 3 : 1;   // parameters of the gate set: <= 3 (one-qubit), <= 1 (two-qubit)
  __shared__ double red[8];
  __shared__ float redf[8];
  C2<R> ud[d * d], du[NP][d * d];
#pragma unroll
  for (int i = 0; i < d * d; ++i) {
    ud[i] = g.ud[i];
#pragma unroll
    for (int p = 0; p < NP; ++p) du[p][i] = g.du[p][i];
  }
  const int np = g.np < NP ? g.np : NP;
  TermSum<R> ts[NP];   // over all of the thread's groups (compensated for FP32)
  const uint64_t groups = 1ull << (n - K);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const int lo = K == 2 ? min(g.q0, g.q1) : g.q0, hi = K == 2 ? max(g.q0, g.q1) : g.q0;
  for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < groups; i0 += stride * kChunkG) {
    for (int j = 0; j < kChunkG; ++j) {
      const uint64_t i = i0 + (uint64_t)j * stride;
      if (i >= groups) break;
      uint64_t base = ins0(i, lo);
      if (K == 2) base = ins0(base, hi);
      uint64_t idx[d];
      C2<R> x[d], l[d], y[d], m[d];
#pragma unroll
      for (int a = 0; a < d; ++a) {
        idx[a] = base;
        if (K == 1) idx[a] |= (uint64_t)a << g.q0;
        else idx[a] |= ((uint64_t)(a >> 1) << g.q0) | ((uint64_t)(a & 1) << g.q1);
        x[a] = psi[idx[a]];
        l[a] = lam[idx[a]];
      }
      // y = state before the gate (given, or U^dagger x), m = U^dagger l
#pragma unroll
      for (int r = 0; r < d; ++r) {
        C2<R> sy{R(0), R(0)}, t{R(0), R(0)};
#pragma unroll
        for (int c = 0; c < d; ++c) {
          sy = cmac(sy, ud[r * d + c], x[c]);
          t = cmac(t, ud[r * d + c], l[c]);
        }
        y[r] = psi_is_before ? x[r] : sy;
        m[r] = t;
      }
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        if (p >= np) break;
        R a2 = R(0);
#pragma unroll
        for (int r = 0; r < d; ++r) {
          C2<R> sv{R(0), R(0)};
#pragma unroll
          for (int c = 0; c < d; ++c) sv = cmac(sv, du[p][r * d + c], y[c]);
          a2 = fma(l[r].x, sv.x, fma(l[r].y, sv.y, a2));   // Re(conj(l_r) sv)
        }
        ts[p].add(a2);
      }
#pragma unroll
      for (int a = 0; a < d; ++a) {
        if (!psi_is_before) psi[idx[a]] = y[a];
        lam[idx[a]] = m[a];
      }
    }
  }
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const R v = p < NP ? (R)ts[p < NP ? p : 0].value() : R(0);
    const double sum = block_sum_terms(v, redf, red);
    if (threadIdx.x == 0) partials[3 * blockIdx.x + p] = sum;
  }
  // the last block to finish adds the blocks' sums in block order (the result
  // does not depend on the order in which blocks finish) and resets the counter
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (int p = 0; p < 3; ++p) {
      double sum = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) sum += __ldcg(partials + 3 * b + p);
      sum = block_sum_g(sum, red);
      if (threadIdx.x == 0) out3[p] = 2.0 * sum;
    }
    if (threadIdx.x == 0) *done = 0u;
  }
}

// lambda = (dL/dp_J) psi_J and the loss partials
template <typename R>
__global__ void __launch_bounds__(256)
    seed_kernel(const C2<R>* __restrict__ psi, C2<R>* __restrict__ lam, const double* __restrict__ w,
                int mode, uint64_t N, double* __restrict__ partials) {
  __shared__ double red[8];
  double acc = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t J = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; J < N; J += stride) {
    const C2<R> a = psi[J];
    double p = (double)a.x * a.x + (double)a.y * a.y;
    double dl;
    if (mode == 0) {
      dl = w[J];
      acc += w[J] * p;
    } else {
      const double c = w[J];
      if (c > 0) {
        if (!(p > 0.0)) p = 1e-300;
        acc += c * log(p);
        dl = c / p;
      } else {
        dl = 0.0;
      }
    }
    C2<R> l;
    l.x = (R)(dl * (double)a.x);
    l.y = (R)(dl * (double)a.y);
    lam[J] = l;
  }
  const double s = block_sum_g(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void sum_partials1_kernel(const double* __restrict__ partials, int blocks,
                                     double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < blocks; i += blockDim.x) s += partials[i];
  s = block_sum_g(s, red);
  if (threadIdx.x == 0) *out = s;
}

constexpr int kGradBlocks = 1024;

template <typename R>
GradGate<R> make_grad_gate(const qs_gate& gate) {
  GradGate<R> g;
  std::memset(&g, 0, sizeof(g));
  cd m[16];
  int dim = 0;
  gate_matrix(gate, m, &dim);
  g.k = dim == 2 ? 1 : 2;
  g.q0 = gate.q[0];
  g.q1 = g.k == 2 ? gate.q[1] : gate.q[0];
  for (int r = 0; r < dim; ++r)
    for (int c = 0; c < dim; ++c) {
      const cd v = std::conj(m[c * dim + r]);
      g.ud[r * dim + c].x = (R)v.real();
      g.ud[r * dim + c].y = (R)v.imag();
    }
  g.np = gate_nparams(gate.kind);
  for (int p = 0; p < g.np; ++p) {
    cd dm[16];
    gate_dmatrix(gate, p, dm);
    for (int i = 0; i < dim * dim; ++i) {
      g.du[p][i].x = (R)dm[i].real();
      g.du[p][i].y = (R)dm[i].imag();
    }
  }
  return g;
}

// psi: the state after the gate (uncomputed in place) or, with before = true,
// the state before the gate (read only)
template <typename R>
qs_status backward_gate(State* st, C2<R>* psi, C2<R>* lam, const qs_gate& gate, double* partials,
                        unsigned* done, double* out3, bool before) {
  GradGate<R> g = make_grad_gate<R>(gate);
  const uint64_t groups = 1ull << (st->n - g.k);
  int blocks = (int)((groups + 255) / 256);
  if (blocks > kGradBlocks) blocks = kGradBlocks;
  if (g.k == 1)
    adjoint_step_kernel<R, 1><<<blocks, 256, 0, st->stream>>>(psi, lam, st->n, g, partials, done, out3,
                                                               before ? 1 : 0);
  else
    adjoint_step_kernel<R, 2><<<blocks, 256, 0, st->stream>>>(psi, lam, st->n, g, partials, done, out3,
                                                               before ? 1 : 0);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

template <typename R>
qs_status run_grad(State* st, const qs_gate* gates, size_t ng, const double* w, int mode, int K,
                   double* dtheta, double* loss) {
  const size_t sb = st->data_bytes;
  std::vector<void*> bufs;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st->stream);
    for (void* p : bufs) dev_free(st, p, sb);
  };
  auto alloc_state = [&]() -> void* {
    void* p = dev_alloc(st, sb);
    if (p) bufs.push_back(p);
    return p;
  };
  qs_status s = QS_OK;
  C2<R>* psi0 = (C2<R>*)alloc_state();
  C2<R>* lam = (C2<R>*)alloc_state();
  double* dth = (double*)dev_alloc(st, 3 * sizeof(double) * (ng + 1) + 8 * kGradBlocks * 3 + 16);
  if (!psi0 || !lam || !dth) {
    if (dth) dev_free(st, dth, 0);
    cleanup();
    set_error("device allocation for the gradient failed");
    return QS_ENOMEM;
  }
  double* partials = dth + 3 * (ng + 1);
  unsigned* done = (unsigned*)(partials + 3 * kGradBlocks);   // blocks finished (reset by the last)
  QS_CUDA(cudaMemsetAsync(done, 0, 16, st->stream));
  QS_CUDA(cudaMemcpyAsync(psi0, st->data, sb, cudaMemcpyDeviceToDevice, st->stream));
  // ---------------- forward (tiled), keeping checkpoints in checkpoint mode
  std::vector<C2<R>*> ckpt, segbuf;
  const bool use_ckpt = K > 0;
  if (use_ckpt) {
    for (size_t g0 = 0; g0 < ng && s == QS_OK; g0 += (size_t)K) {
      C2<R>* c = (C2<R>*)alloc_state();
      if (!c) {
        s = QS_ENOMEM;
        set_error("checkpoint allocation failed");
        break;
      }
      QS_CUDA(cudaMemcpyAsync(c, st->data, sb, cudaMemcpyDeviceToDevice, st->stream));
      ckpt.push_back(c);
      const size_t cnt = (g0 + K <= ng) ? (size_t)K : ng - g0;
      s = apply_gates(st, gates + g0, cnt, QS_METHOD_TILED, nullptr);
    }
  } else {
    s = apply_gates(st, gates, ng, QS_METHOD_TILED, nullptr);
  }
  // ---------------- seed
  if (s == QS_OK) {
    const uint64_t N = 1ull << st->n;
    int blocks = (int)((N + 255) / 256);
    if (blocks > kGradBlocks) blocks = kGradBlocks;
    seed_kernel<R><<<blocks, 256, 0, st->stream>>>((const C2<R>*)st->data, lam, w, mode, N, partials);
    sum_partials1_kernel<<<1, 256, 0, st->stream>>>(partials, blocks, dth + 3 * ng);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_status(e, "seed kernel");
  }
  // ---------------- backward: fused tile passes (n >= 12), else one launch per gate
  bool fused = st->n >= kTileBits;
  if (s == QS_OK && fused) {
    QS_CUDA(cudaMemsetAsync(dth, 0, sizeof(double) * 3 * ng, st->stream));
    if (!use_ckpt) {
      s = adjoint_tiled(st, lam, gates, 0, ng, dth);
    } else {
      // per segment (last first): the state after it, recomputed from its checkpoint
      for (size_t seg = ckpt.size(); seg-- > 0 && s == QS_OK;) {
        const size_t g0 = seg * (size_t)K;
        const size_t g1 = (g0 + K <= ng) ? g0 + (size_t)K : ng;
        QS_CUDA(cudaMemcpyAsync(st->data, ckpt[seg], sb, cudaMemcpyDeviceToDevice, st->stream));
        s = apply_gates(st, gates + g0, g1 - g0, QS_METHOD_TILED, nullptr);
        if (s == QS_OK) s = adjoint_tiled(st, lam, gates, g0, g1, dth);
      }
    }
  }
  if (s == QS_OK && !fused) {
    for (int k = 0; use_ckpt && k < K && s == QS_OK; ++k) {
      C2<R>* b = (C2<R>*)alloc_state();
      if (!b) {
        s = QS_ENOMEM;
        set_error("segment buffer allocation failed");
      }
      segbuf.push_back(b);
    }
  }
  if (s == QS_OK && !fused) {
    if (!use_ckpt) {
      for (size_t g = ng; g-- > 0 && s == QS_OK;)
        s = backward_gate<R>(st, (C2<R>*)st->data, lam, gates[g], partials, done, dth + 3 * g, false);
    } else {
      for (size_t seg = ckpt.size(); seg-- > 0 && s == QS_OK;) {
        const size_t g0 = seg * (size_t)K;
        const size_t g1 = (g0 + K <= ng) ? g0 + (size_t)K : ng;
        // states before each gate of the segment, recomputed forward from the checkpoint
        QS_CUDA(cudaMemcpyAsync(st->data, ckpt[seg], sb, cudaMemcpyDeviceToDevice, st->stream));
        for (size_t g = g0; g < g1 && s == QS_OK; ++g) {
          QS_CUDA(cudaMemcpyAsync(segbuf[g - g0], st->data, sb, cudaMemcpyDeviceToDevice, st->stream));
          if (g + 1 < g1) s = apply_gates(st, gates + g, 1, QS_METHOD_TILED, nullptr);
        }
        for (size_t g = g1; g-- > g0 && s == QS_OK;)
          s = backward_gate<R>(st, segbuf[g - g0], lam, gates[g], partials, done, dth + 3 * g, true);
      }
    }
  }
  if (s == QS_OK) {
    std::vector<double> host(3 * ng + 1);
    QS_CUDA(cudaMemcpyAsync(host.data(), dth, sizeof(double) * (3 * ng + 1), cudaMemcpyDeviceToHost,
                            st->stream));
    QS_CUDA(cudaMemcpyAsync(st->data, psi0, sb, cudaMemcpyDeviceToDevice, st->stream));
    QS_CUDA(cudaStreamSynchronize(st->stream));
    for (size_t g = 0; g < ng; ++g) {
      const int np = gate_nparams(gates[g].kind);
      for (int p = 0; p < 3; ++p) dtheta[3 * g + p] = p < np ? host[3 * g + p] : 0.0;
    }
    if (loss) *loss = host[3 * ng];
  }
  dev_free(st, dth, 0);
  cleanup();
  return s;
}

}  // namespace

}  // namespace qs

using namespace qs;

extern "C" qs_status sv_grad(qs_state_t h, const qs_gate* gates, size_t ngates, const double* weights,
                             int mode, int checkpoint_every, double* dtheta, double* loss) {
  return abi_guard(__func__, [&]() -> qs_status {
    State* st = h;
    if (!st) {
      set_error("state is NULL");
      return QS_EINVAL;
    }
    if (!weights || (ngates > 0 && !dtheta) || (mode != 0 && mode != 1) || checkpoint_every < 0) {
      set_error("bad sv_grad arguments");
      return QS_EINVAL;
    }
    qs_status s = validate_gates(gates, ngates, st->n);
    if (s != QS_OK) return s;
    if (st->prec == QS_C64)
      return run_grad<float>(st, gates, ngates, weights, mode, checkpoint_every, dtheta, loss);
    return run_grad<double>(st, gates, ngates, weights, mode, checkpoint_every, dtheta, loss);
  });
}
