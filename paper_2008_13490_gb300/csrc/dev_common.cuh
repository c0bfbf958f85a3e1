// Inline device helpers shared by the state-vector kernels (sv_kernels.cu) and
// the packed small-circuit kernel of the serving loop (serve.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace qs {

// m0*a + m1*b for complex numbers stored as (re, im)
template <typename R>
__device__ __forceinline__ C2<R> cfma2(C2<R> m0, C2<R> a, C2<R> m1, C2<R> b) {
  C2<R> r;
  r.x = m0.x * a.x;
  r.x = fma(-m0.y, a.y, r.x);
  r.x = fma(m1.x, b.x, r.x);
  r.x = fma(-m1.y, b.y, r.x);
  r.y = m0.x * a.y;
  r.y = fma(m0.y, a.x, r.y);
  r.y = fma(m1.x, b.y, r.y);
  r.y = fma(m1.y, b.x, r.y);
  return r;
}

// FP32: the same four products per component, in the same order, as packed
// FP32x2 multiply-adds (half the instructions; identical rounding)
template <>
__device__ __forceinline__ C2<float> cfma2<float>(C2<float> m0, C2<float> a, C2<float> m1, C2<float> b) {
  float2 r = __fmul2_rn(make_float2(m0.x, m0.x), make_float2(a.x, a.y));
  r = __ffma2_rn(make_float2(-m0.y, m0.y), make_float2(a.y, a.x), r);
  r = __ffma2_rn(make_float2(m1.x, m1.x), make_float2(b.x, b.y), r);
  r = __ffma2_rn(make_float2(-m1.y, m1.y), make_float2(b.y, b.x), r);
  return C2<float>{r.x, r.y};
}

template <typename R>
__device__ __forceinline__ C2<R> cmul(C2<R> a, C2<R> b) {
  C2<R> r;
  r.x = a.x * b.x;
  r.x = fma(-a.y, b.y, r.x);
  r.y = a.x * b.y;
  r.y = fma(a.y, b.x, r.y);
  return r;
}

template <typename R>
__device__ __forceinline__ C2<R> csel(bool s, C2<R> a, C2<R> b) {
  C2<R> r;
  r.x = s ? a.x : b.x;
  r.y = s ? a.y : b.y;
  return r;
}

template <typename R>
__device__ __forceinline__ C2<R> shfl_xor_c(C2<R> v, int m) {
  C2<R> r;
  r.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  r.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return r;
}

// bit-insert index of the thesis's reduced loop: ((i & ~m) << 1) | (i & m), m = 2^b - 1
__device__ __forceinline__ uint64_t insert_zero(uint64_t i, int b) {
  const uint64_t m = (1ull << b) - 1ull;
  return ((i & ~m) << 1) | (i & m);
}

// Sum over the block (result valid in thread 0); uses 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v) {
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

// Applies ops in order to a whole 2^n state held in shared memory by one CTA
// (pairs for one-qubit and choice ops, quads for dense two-qubit ops,
// elementwise phases for diagonal ops), with a barrier after each op.
template <typename R>
__device__ void small_apply_ops(C2<R>* sm, int n, const PlainOp<R>* __restrict__ ops, int nops) {
  const int N = 1 << n;
  for (int k = 0; k < nops; ++k) {
    const PlainOp<R>* op = ops + k;
    const int type = op->type;
    if (type == F_G1 || type == F_G1C) {
      const int t = op->t, c = op->c;
      for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
        const int i0 = (int)insert_zero(i, t), i1 = i0 | (1 << t);
        const C2<R>* m = op->m;
        if (type == F_G1C && ((i0 >> c) & 1)) m = op->m + 4;
        const C2<R> a = sm[i0], b = sm[i1];
        sm[i0] = cfma2(m[0], a, m[1], b);
        sm[i1] = cfma2(m[2], a, m[3], b);
      }
    } else if (type == F_D) {
      for (int J = threadIdx.x; J < N; J += blockDim.x) {
        const int ba = (J >> op->a) & 1;
        const int idx = op->b >= 0 ? ba * 2 + ((J >> op->b) & 1) : ba;
        sm[J] = cmul(sm[J], op->m[idx]);
      }
    } else {
      const int lo = op->a < op->b ? op->a : op->b, hi = op->a < op->b ? op->b : op->a;
      for (int i = threadIdx.x; i < N / 4; i += blockDim.x) {
        const int base = (int)insert_zero(insert_zero(i, lo), hi);
        int idx[4];
        C2<R> a[4];
        for (int l = 0; l < 4; ++l) {
          idx[l] = base | ((l >> 1) << op->a) | ((l & 1) << op->b);
          a[l] = sm[idx[l]];
        }
        for (int r = 0; r < 4; ++r) {
          C2<R> acc = cfma2(op->m[4 * r + 0], a[0], op->m[4 * r + 1], a[1]);
          const C2<R> acc2 = cfma2(op->m[4 * r + 2], a[2], op->m[4 * r + 3], a[3]);
          acc.x += acc2.x;
          acc.y += acc2.y;
          sm[idx[r]] = acc;
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace qs
