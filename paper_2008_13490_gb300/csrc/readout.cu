// Readout transforms for sm_103a.
//
//  meas_error_kernel  the measurement-error model of Eq.
//                     (errordetectionMeasurementError) in place on a probability
//                     vector: each bit of an outcome is misread independently,
//                     so the map is a Kronecker product of one 2x2
//                     column-stochastic matrix per qubit, applied 12 (first
//                     sweep) or 8 (later sweeps) qubits per HBM sweep.
//  bloch_kernel       the Bloch vectors of Eq. (multiqubitblochvector) of every
//                     qubit: sums over the amplitude pairs that differ in one
//                     bit, 12 or 8 qubits per read of the state.
//
// Tile.  A CTA of 256 threads owns 2^12 elements at bit positions pos[0..11]
// (ascending; the first sweep takes positions 0..11, every later one 0..3, its new
// positions and filler positions, so local bits 0..3 are always positions 0..3),
// the other bits fixed per tile.  A thread holds 16 elements in registers, and
// three layouts put a different 4 local bits into its registers:
//   A  thread t -> local bits 0..7,         registers -> local 8..11  (loads)
//   B  thread t -> local bits 0..3, 8..11,  registers -> local 4..7   (stores)
//   C  thread t -> local bits 4..11,        registers -> local 0..3
// A pair operation on a local bit runs in the layout that has it in registers.
// Global accesses in A and B are runs of 16 (or 32) consecutive elements.
// Between layouts the tile goes through shared memory at slot L ^ ((L >> 4) & 31),
// which keeps all three layouts free of bank conflicts for 4-, 8- and 16-byte
// elements.  Addresses are XOR-linear in the local index: two 64-entry tables.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "abi_guard.h"
#include "internal.h"

namespace qs {
namespace {

constexpr int kRoThreads = 256;
constexpr int kRoElems = 1 << kTileBits;   // 4096
constexpr int kBlochSlots = 3 * kTileBits;  // (x, y, z) per local bit

struct ReadoutPass {
  int32_t n_nt;                // bits outside the tile
  int32_t active;              // local bits this sweep transforms / sums
  uint8_t pos[kTileBits];      // physical position of local bit i (ascending)
  uint8_t nt_pos[52];          // physical position of non-tile bit j (tile index bit j)
  double e01[kTileBits];       // per local bit: P(read 1 | true 0)
  double e10[kTileBits];       //                P(read 0 | true 1)
};

__device__ __forceinline__ int lay_a(int t, int r) { return t | (r << 8); }
__device__ __forceinline__ int lay_b(int t, int r) { return (t & 15) | (r << 4) | ((t >> 4) << 8); }
__device__ __forceinline__ int lay_c(int t, int r) { return r | (t << 4); }
__device__ __forceinline__ int ro_slot(int L) { return L ^ ((L >> 4) & 31); }

// address tables (deposit of the local index bits into the tile positions)
__device__ __forceinline__ void build_tables(const ReadoutPass& P, uint64_t* alo, uint64_t* ahi) {
  const int tid = threadIdx.x;
  if (tid < 128) {
    const int v = tid & 63, h = tid >> 6;
    uint64_t a = 0;
    for (int i = 0; i < 6; ++i)
      if ((v >> i) & 1) a |= 1ull << P.pos[6 * h + i];
    (h ? ahi : alo)[v] = a;
  }
}

// offset of the tile's fixed bits: lane j < n_nt contributes bit j of the tile index
__device__ __forceinline__ uint64_t tile_base(const ReadoutPass& P, uint64_t tile) {
  const int lane = threadIdx.x & 31;
  uint64_t b = 0;
  if (lane < P.n_nt) b = ((tile >> lane) & 1ull) << P.nt_pos[lane];
  const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)b);
  const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(b >> 32));
  return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t local_off(const uint64_t* alo, const uint64_t* ahi, int L) {
  return alo[L & 63] | ahi[L >> 6];
}

// Offsets of a layout's 16 registers: the thread's part of the local index once
// per CTA, and register r adds the deposits g[k] of its bits (r is a
// compile-time constant in the unrolled loops, so each offset is one OR of the
// previous one).
struct LayoutAddr {
  uint64_t t;      // thread part
  uint64_t g[4];   // deposit of register bit k
  __device__ __forceinline__ uint64_t reg(int r) const {
    uint64_t o = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if ((r >> k) & 1) o |= g[k];
    return o;
  }
};
// layout A: thread -> local 0..7, registers -> local 8..11
__device__ __forceinline__ LayoutAddr addr_a(const ReadoutPass& P, const uint64_t* alo, const uint64_t* ahi) {
  LayoutAddr a;
  a.t = local_off(alo, ahi, lay_a(threadIdx.x, 0));
#pragma unroll
  for (int k = 0; k < 4; ++k) a.g[k] = 1ull << P.pos[8 + k];
  return a;
}
// layout B: thread -> local 0..3, 8..11, registers -> local 4..7
__device__ __forceinline__ LayoutAddr addr_b(const ReadoutPass& P, const uint64_t* alo, const uint64_t* ahi) {
  LayoutAddr a;
  a.t = local_off(alo, ahi, lay_b(threadIdx.x, 0));
#pragma unroll
  for (int k = 0; k < 4; ++k) a.g[k] = 1ull << P.pos[4 + k];
  return a;
}

// streaming (evict-first) load of one complex amplitude
__device__ __forceinline__ C2<float> ldcs_c(const C2<float>* p) {
  const float2 t = __ldcs(reinterpret_cast<const float2*>(p));
  return C2<float>{t.x, t.y};
}
__device__ __forceinline__ C2<double> ldcs_c(const C2<double>* p) {
  const double2 t = __ldcs(reinterpret_cast<const double2*>(p));
  return C2<double>{t.x, t.y};
}

// asynchronous global -> shared copies (cp.async; 4 and 8 bytes go through L1)
template <int B>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// the tile's 16 elements of this thread in layout A, copied into buf at their slots
template <typename E>
__device__ __forceinline__ void prefetch_tile(E* buf, const E* src, const LayoutAddr& la) {
#pragma unroll
  for (int r = 0; r < 16; ++r) cp_async<sizeof(E)>(buf + ro_slot(lay_a(threadIdx.x, r)), src + la.reg(r));
}

// ------------------------------------------------------------------ measurement error

// registers r and r | 2^k hold the pair (bit = 0, bit = 1) of local bit `loc`
template <typename T, int K>
__device__ __forceinline__ void flip_pairs(T* v, const T* m) {
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    if (r & (1 << K)) continue;
    const T x0 = v[r], x1 = v[r | (1 << K)];
    v[r] = fma(m[1], x1, m[0] * x0);            // read 0: true 0 kept, true 1 misread
    v[r | (1 << K)] = fma(m[3], x1, m[2] * x0);  // read 1
  }
}

// A thread's 16 values.  FP32 values are kept as 8 float2 (register bit 0 =
// the component) so that the pairs of register bits 1..3 are float2 registers
// and their maps use Blackwell's packed FP32x2 multiply-adds: half the
// instructions of this issue-bound sweep.
template <typename T>
struct Regs16 {
  T v[16];
  __device__ __forceinline__ T& at(int r) { return v[r]; }
};
template <>
struct Regs16<float> {
  float2 w[8];
  __device__ __forceinline__ float& at(int r) { return (r & 1) ? w[r >> 1].y : w[r >> 1].x; }
};

template <typename T>
__device__ __forceinline__ void flip_stage(Regs16<T>& x, int active, int first_local, const T (*m)[4]) {
  if ((active >> (first_local + 0)) & 1) flip_pairs<T, 0>(x.v, m[first_local + 0]);
  if ((active >> (first_local + 1)) & 1) flip_pairs<T, 1>(x.v, m[first_local + 1]);
  if ((active >> (first_local + 2)) & 1) flip_pairs<T, 2>(x.v, m[first_local + 2]);
  if ((active >> (first_local + 3)) & 1) flip_pairs<T, 3>(x.v, m[first_local + 3]);
}

// register bit K >= 1 of the float2 form: float2 registers i and i | 2^(K-1)
template <int K>
__device__ __forceinline__ void flip_pairs2(float2* w, const float* m) {
  const float2 m0 = make_float2(m[0], m[0]), m1 = make_float2(m[1], m[1]);
  const float2 m2 = make_float2(m[2], m[2]), m3 = make_float2(m[3], m[3]);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (i & (1 << (K - 1))) continue;
    const float2 x0 = w[i], x1 = w[i | (1 << (K - 1))];
    w[i] = __ffma2_rn(m1, x1, __fmul2_rn(m0, x0));
    w[i | (1 << (K - 1))] = __ffma2_rn(m3, x1, __fmul2_rn(m2, x0));
  }
}

template <>
__device__ __forceinline__ void flip_stage<float>(Regs16<float>& x, int active, int first_local,
                                                  const float (*m)[4]) {
  if ((active >> (first_local + 0)) & 1) {
    const float* q = m[first_local];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float x0 = x.w[i].x, x1 = x.w[i].y;
      x.w[i] = make_float2(fmaf(q[1], x1, q[0] * x0), fmaf(q[3], x1, q[2] * x0));
    }
  }
  if ((active >> (first_local + 1)) & 1) flip_pairs2<1>(x.w, m[first_local + 1]);
  if ((active >> (first_local + 2)) & 1) flip_pairs2<2>(x.w, m[first_local + 2]);
  if ((active >> (first_local + 3)) & 1) flip_pairs2<3>(x.w, m[first_local + 3]);
}

template <typename T>
__global__ void __launch_bounds__(kRoThreads, sizeof(T) == 4 ? 3 : 2)
    meas_error_kernel(T* __restrict__ p, const ReadoutPass P, uint64_t tiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  __shared__ uint64_t s_alo[64], s_ahi[64];
  __shared__ T s_m[kTileBits][4];
  const int tid = threadIdx.x;
  build_tables(P, s_alo, s_ahi);
  if (tid < kTileBits) {
    s_m[tid][0] = (T)(1.0 - P.e01[tid]);
    s_m[tid][1] = (T)P.e10[tid];
    s_m[tid][2] = (T)P.e01[tid];
    s_m[tid][3] = (T)(1.0 - P.e10[tid]);
  }
  __syncthreads();
  const int active = P.active;
  const LayoutAddr la = addr_a(P, s_alo, s_ahi), lb = addr_b(P, s_alo, s_ahi);
  // two shared tiles: the next tile's copies run while this one is transformed
  uint64_t tile = blockIdx.x;
  if (tile < tiles) prefetch_tile(sm, p + (tile_base(P, tile) | la.t), la);
  cp_async_commit();
  for (int cur = 0; tile < tiles; tile += gridDim.x, cur ^= 1) {
    T* b = sm + (cur ? kRoElems : 0);
    const uint64_t nxt = tile + gridDim.x;
    if (nxt < tiles) prefetch_tile(sm + (cur ? 0 : kRoElems), p + (tile_base(P, nxt) | la.t), la);
    cp_async_commit();
    cp_async_wait<1>();   // this tile's copies (every group but the newest) have landed
    __syncthreads();
    const uint64_t base = tile_base(P, tile);
    Regs16<T> v;
    if (active & 0xf00) {
#pragma unroll
      for (int r = 0; r < 16; ++r) v.at(r) = b[ro_slot(lay_a(tid, r))];
      flip_stage(v, active, 8, s_m);
#pragma unroll
      for (int r = 0; r < 16; ++r) b[ro_slot(lay_a(tid, r))] = v.at(r);
      __syncthreads();
    }
    if (active & 0xf) {
#pragma unroll
      for (int r = 0; r < 16; ++r) v.at(r) = b[ro_slot(lay_c(tid, r))];
      flip_stage(v, active, 0, s_m);
#pragma unroll
      for (int r = 0; r < 16; ++r) b[ro_slot(lay_c(tid, r))] = v.at(r);
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) v.at(r) = b[ro_slot(lay_b(tid, r))];
    flip_stage(v, active, 4, s_m);
    T* dst = p + (base | lb.t);
#pragma unroll
    for (int r = 0; r < 16; ++r) __stcs(dst + lb.reg(r), v.at(r));
    __syncthreads();   // b is the target of the next iteration's copies
  }
  cp_async_wait<0>();
}

// n < 12: the whole vector in one CTA's shared memory, one bit at a time
template <typename T>
__global__ void __launch_bounds__(kRoThreads)
    meas_error_small_kernel(T* __restrict__ p, int n, const ReadoutPass P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int N = 1 << n;
  for (int J = threadIdx.x; J < N; J += blockDim.x) sm[J] = p[J];
  __syncthreads();
  for (int q = 0; q < n; ++q) {
    const T m0 = (T)(1.0 - P.e01[q]), m1 = (T)P.e10[q], m2 = (T)P.e01[q], m3 = (T)(1.0 - P.e10[q]);
    for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
      const int j0 = ((i >> q) << (q + 1)) | (i & ((1 << q) - 1)), j1 = j0 | (1 << q);
      const T x0 = sm[j0], x1 = sm[j1];
      sm[j0] = fma(m1, x1, m0 * x0);
      sm[j1] = fma(m3, x1, m2 * x0);
    }
    __syncthreads();
  }
  for (int J = threadIdx.x; J < N; J += blockDim.x) p[J] = sm[J];
}

// ------------------------------------------------------------------ Bloch vectors

template <typename R>
__device__ __forceinline__ R warp_sum(R x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Across tiles a warp accumulates each slot in the state's precision: FP32 with
// Kahan compensation for complex64 states (GB300's FP64 pipe is far slower than
// its FP32 pipe, and an FP64 add per slot and tile bounded the sweep), FP64 for
// complex128 states.  FP64 from the per-CTA sums on.
template <typename R>
struct SlotAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(R x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct SlotAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// The warp totals of 16 values, scattered: afterwards lane L holds the total of
// value (L >> 1) & 15 (each step sends the half of its values that the partner
// lane keeps): 16 shuffles instead of 5 per value.
template <typename R>
__device__ __forceinline__ R reduce_scatter16(R (&x)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 8, m = 16; w >= 1; w >>= 1, m >>= 1) {
    const bool hi = (lane & m) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const R send = hi ? x[i] : x[i + w];
      const R keep = hi ? x[i + w] : x[i];
      x[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
  }
  return x[0] + __shfl_xor_sync(0xffffffffu, x[0], 1);
}

// Pair sums of the 4 local bits a layout holds in registers (register bit k =
// local bit first + k): value 3k + c, c = Re conj(a0) a1, Im conj(a0) a1,
// |a0|^2 - |a1|^2, over the thread's 8 pairs per bit, then over the warp into
// this lane's accumulator of the layout (value (lane >> 1) & 15).
template <typename R>
__device__ __forceinline__ void bloch_stage(const C2<R>* v, int active, int first, SlotAcc<R>& acc) {
  // z of a bit = (all 16 norms) - 2 (the norms with the bit set)
  R x[16], nrm[16], tot = 0;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    nrm[r] = fma(v[r].x, v[r].x, v[r].y * v[r].y);
    tot += nrm[r];
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!((active >> (first + k)) & 1)) continue;
    R re = 0, im = 0, z1 = 0;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      if (r & (1 << k)) continue;
      const C2<R> a0 = v[r], a1 = v[r | (1 << k)];
      re = fma(a0.x, a1.x, fma(a0.y, a1.y, re));
      im = fma(a0.x, a1.y, fma(-a0.y, a1.x, im));
      z1 += nrm[r | (1 << k)];
    }
    x[3 * k] = re;
    x[3 * k + 1] = im;
    x[3 * k + 2] = fma(R(-2), z1, tot);
  }
  acc.add(reduce_scatter16(x));
}

// partials: per CTA kBlochSlots FP64 sums (slot 3 loc + c; c = Re, Im, z)
template <typename R>
__global__ void __launch_bounds__(kRoThreads)
    bloch_kernel(const C2<R>* __restrict__ psi, const ReadoutPass P, uint64_t tiles,
                 double* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<R>* sm = reinterpret_cast<C2<R>*>(smem_raw);
  __shared__ uint64_t s_alo[64], s_ahi[64];
  __shared__ double s_red[kRoThreads / 32][kBlochSlots];
  const int tid = threadIdx.x;
  build_tables(P, s_alo, s_ahi);
  __syncthreads();
  const int active = P.active;
  SlotAcc<R> acc_a, acc_b, acc_c;   // layouts A (local 8..11), B (4..7), C (0..3)
  const LayoutAddr la = addr_a(P, s_alo, s_ahi);
  for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint64_t base = tile_base(P, tile);
    C2<R> v[16];
    const C2<R>* src = psi + (base | la.t);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = ldcs_c(src + la.reg(r));
    if (active & 0xf00) bloch_stage(v, active, 8, acc_a);
    if (active & 0xff) {
#pragma unroll
      for (int r = 0; r < 16; ++r) sm[ro_slot(lay_a(tid, r))] = v[r];
      __syncthreads();
      if (active & 0xf) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = sm[ro_slot(lay_c(tid, r))];
        bloch_stage(v, active, 0, acc_c);
      }
      if (active & 0xf0) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = sm[ro_slot(lay_b(tid, r))];
        bloch_stage(v, active, 4, acc_b);
      }
      __syncthreads();   // the next tile reuses the shared tile
    }
  }
  // lane L (even) holds value u = (L >> 1) & 15 = 3k + c of each layout: slot 3 (first + k) + c
  const int warp = tid >> 5, lane = tid & 31, u = (lane >> 1) & 15;
  if (!(lane & 1) && u < 12) {
    s_red[warp][3 * 8 + u] = acc_a.value();
    s_red[warp][3 * 4 + u] = acc_b.value();
    s_red[warp][u] = acc_c.value();
  }
  __syncthreads();
  if (tid < kBlochSlots) {
    double s = 0.0;
    for (int w = 0; w < kRoThreads / 32; ++w) s += s_red[w][tid];
    partials[(size_t)blockIdx.x * kBlochSlots + tid] = s;
  }
}

// out[3 pos + c] = sum over CTAs of slot 3 loc + c, for the sweep's active bits
// (r^x = 2 Re, r^y = 2 Im, r^z = z); fixed order: deterministic
__global__ void bloch_reduce_kernel(const double* __restrict__ partials, int nblocks, const ReadoutPass P,
                                    double* __restrict__ out) {
  const int s = threadIdx.x;
  if (s >= kBlochSlots) return;
  const int loc = s / 3, c = s % 3;
  if (!((P.active >> loc) & 1)) return;
  double acc = 0.0;
  for (int b = 0; b < nblocks; ++b) acc += partials[(size_t)b * kBlochSlots + s];
  out[3 * P.pos[loc] + c] = c < 2 ? 2.0 * acc : acc;
}

// n < 12: one CTA, bit by bit, FP64 block sums
template <typename R>
__global__ void __launch_bounds__(kRoThreads) bloch_small_kernel(const C2<R>* __restrict__ psi, int n,
                                                                 double* __restrict__ out) {
  __shared__ double s_red[3][kRoThreads / 32];
  const int N = 1 << n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = 0; q < n; ++q) {
    double re = 0, im = 0, z = 0;
    for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
      const int j0 = ((i >> q) << (q + 1)) | (i & ((1 << q) - 1)), j1 = j0 | (1 << q);
      const C2<R> a0 = psi[j0], a1 = psi[j1];
      re += (double)a0.x * a1.x + (double)a0.y * a1.y;
      im += (double)a0.x * a1.y - (double)a0.y * a1.x;
      z += (double)a0.x * a0.x + (double)a0.y * a0.y - (double)a1.x * a1.x - (double)a1.y * a1.y;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    z = warp_sum(z);
    if (lane == 0) {
      s_red[0][warp] = re;
      s_red[1][warp] = im;
      s_red[2][warp] = z;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double s = 0.0;
      for (int w = 0; w < kRoThreads / 32; ++w) s += s_red[threadIdx.x][w];
      out[3 * q + threadIdx.x] = threadIdx.x < 2 ? 2.0 * s : s;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ host

// Sweeps for n >= 12: positions 0..11 first, then 8 new positions per sweep on
// top of positions 0..3 (filled up with the lowest unused positions).
std::vector<ReadoutPass> plan_readout(int n, const double* e01, const double* e10) {
  std::vector<ReadoutPass> out;
  int next = 0;
  while (next < n) {
    ReadoutPass P;
    std::memset(&P, 0, sizeof(P));
    uint64_t tile = 0, act = 0;
    const int take = next == 0 ? kTileBits : 8;
    for (int q = next; q < n && q < next + take; ++q) act |= 1ull << q;
    tile = act | 0xfull;
    for (int q = 0; q < n && __builtin_popcountll(tile) < kTileBits; ++q) tile |= 1ull << q;
    int k = 0, j = 0;
    for (int q = 0; q < n; ++q) {
      if ((tile >> q) & 1) {
        P.pos[k] = (uint8_t)q;
        if ((act >> q) & 1) P.active |= 1 << k;
        if (e01) P.e01[k] = e01[q];
        if (e10) P.e10[k] = e10[q];
        ++k;
      } else {
        P.nt_pos[j++] = (uint8_t)q;
      }
    }
    P.n_nt = j;
    out.push_back(P);
    next += take;
  }
  return out;
}

int grid_for(const void* kern, size_t smem, uint64_t tiles) {
  int dev = 0, sms = 152, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRoThreads, smem);
  if (per_sm < 1) per_sm = 1;
  const uint64_t g = (uint64_t)sms * (uint64_t)per_sm;
  return (int)(tiles < g ? tiles : g);
}

template <typename F>
qs_status smem_attr(F* f, size_t bytes) {
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute");
  }
  return QS_OK;
}

template <typename T>
qs_status meas_error_launch(T* p, int n, const double* e01, const double* e10, cudaStream_t stream) {
  if (n < kTileBits) {
    ReadoutPass P;
    std::memset(&P, 0, sizeof(P));
    for (int q = 0; q < n; ++q) {
      P.e01[q] = e01[q];
      P.e10[q] = e10[q];
    }
    meas_error_small_kernel<T><<<1, kRoThreads, sizeof(T) << n, stream>>>(p, n, P);
    QS_CUDA(cudaGetLastError());
    return QS_OK;
  }
  const size_t smem = 2 * sizeof(T) * kRoElems;
  qs_status s = smem_attr(meas_error_kernel<T>, smem);
  if (s != QS_OK) return s;
  const uint64_t tiles = 1ull << (n - kTileBits);
  const int grid = grid_for((const void*)meas_error_kernel<T>, smem, tiles);
  for (const ReadoutPass& P : plan_readout(n, e01, e10)) {
    meas_error_kernel<T><<<grid, kRoThreads, smem, stream>>>(p, P, tiles);
    QS_CUDA(cudaGetLastError());
  }
  return QS_OK;
}

template <typename R>
qs_status bloch_launch(State* st, double* dev_out) {
  const C2<R>* psi = (const C2<R>*)st->data;
  const int n = st->n;
  if (n < kTileBits) {
    bloch_small_kernel<R><<<1, kRoThreads, 0, st->stream>>>(psi, n, dev_out);
    QS_CUDA(cudaGetLastError());
    return QS_OK;
  }
  const size_t smem = sizeof(C2<R>) * kRoElems;
  qs_status s = smem_attr(bloch_kernel<R>, smem);
  if (s != QS_OK) return s;
  const uint64_t tiles = 1ull << (n - kTileBits);
  const int grid = grid_for((const void*)bloch_kernel<R>, smem, tiles);
  // per-CTA partials in the state's marginal scratch (not in use between calls)
  double* partials = (double*)((unsigned char*)st->scratch + kScratchMarg);
  if ((size_t)grid * kBlochSlots > ((size_t)1 << kScratchMargLog2) - 256) {
    set_error("Bloch partials (%d CTAs) exceed the scratch", grid);
    return QS_EUNSUPPORTED;
  }
  for (const ReadoutPass& P : plan_readout(n, nullptr, nullptr)) {
    bloch_kernel<R><<<grid, kRoThreads, smem, st->stream>>>(psi, P, tiles, partials);
    QS_CUDA(cudaGetLastError());
    bloch_reduce_kernel<<<1, 64, 0, st->stream>>>(partials, grid, P, dev_out);
    QS_CUDA(cudaGetLastError());
  }
  return QS_OK;
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status sv_bloch(qs_state_t st_, double* r_out) {
  return abi_guard(__func__, [&]() -> qs_status {
    State* st = st_;
    if (!st || !r_out) {
      set_error("state and r_out are required");
      return QS_EINVAL;
    }
    const int n = st->n;
    // the result (3n doubles) at the end of the marginal scratch
    double* dev_out = (double*)((unsigned char*)st->scratch + kScratchMarg) + ((size_t)1 << kScratchMargLog2) - 256;
    qs_status s = st->prec == QS_C64 ? bloch_launch<float>(st, dev_out) : bloch_launch<double>(st, dev_out);
    if (s != QS_OK) return s;
    QS_CUDA(cudaMemcpyAsync(r_out, dev_out, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost, st->stream));
    QS_CUDA(cudaStreamSynchronize(st->stream));
    return QS_OK;
  });
}

extern "C" qs_status qs_meas_error(void* probs, int n, int fp64, const double* e01, const double* e10,
                                   void* stream) {
  return abi_guard(__func__, [&]() -> qs_status {
    if (!probs || !e01) {
      set_error("probs and e01 are required");
      return QS_EINVAL;
    }
    if (n < 1 || n > 40) {
      set_error("n = %d out of range [1, 40]", n);
      return QS_EINVAL;
    }
    if ((uintptr_t)probs & 15) {
      set_error("probs must be 16-byte aligned");
      return QS_EINVAL;
    }
    if (!e10) e10 = e01;
    for (int q = 0; q < n; ++q)
      if (!(e01[q] >= 0.0 && e01[q] <= 1.0 && e10[q] >= 0.0 && e10[q] <= 1.0)) {
        set_error("misread rates of qubit %d are not in [0, 1]", q);
        return QS_EINVAL;
      }
    cudaStream_t s = (cudaStream_t)stream;
    return fp64 ? meas_error_launch<double>((double*)probs, n, e01, e10, s)
                : meas_error_launch<float>((float*)probs, n, e01, e10, s);
  });
}
