// Batched density matrices in the Pauli basis (Pauli transfer matrices).
//
// A circuit's state is its Pauli vector r_i = Tr(P^_i rho), P^_i = P_i/sqrt(N)
// (Eq. (GSTVectorizedRho)), 4^n reals kept in one CTA's shared memory.  An op
// is a PTM acting on the base-4 digit(s) of its qubit(s); composition of maps
// is the product of their PTMs (section "Quantum operations").  Outcome
// probabilities p_J = <<E_J| r>> (Eq. (GSTBornRuleVectorized)): for
// E_J = |J><J| only the {I,Z}^n entries contribute, with sign
// (-1)^{|S & J|}, i.e. p = 2^{-n/2} WHT(r restricted to {I,Z}^n).
//
// PTMs of the gate set, each from G_ij = Tr(P_i E(P_j)) / 2 worked out by hand
// (rows/columns ordered I, x, y, z):
//   R^x(t): y -> cos t y + sin t z,  z -> cos t z - sin t y   (Eq. (singlequbitrotationx))
//   R^y(t): z -> cos t z + sin t x,  x -> cos t x - sin t z   (Eq. (singlequbitrotationy))
//   depolarizing, p_x = p_y = p_z = p/3 (Eq. (singletDepolarizingChannel)):
//                     diag(1, f, f, f), f = 1 - 4p/3
//   amplitude damping, decay parameter 1, rate g (Eqs. (singletAmplitudeDampingChannel1-2)):
//                     I -> I + g z, x -> s x, y -> s y, z -> (1-g) z, s = sqrt(1-g)
//   CZ: a signed permutation of the 16 two-qubit Paulis (computed on the host
//       from the trace formula).
// The noise channel after an op is C = AD(g) DEP(p) on each touched qubit.
//
// Gradient of l = sum_J n_J log p_J by an adjoint sweep: lambda_L = dl/dr =
// 2^{-n/2} WHT(n/p) on {I,Z}^n; backwards, each sub-op contributes
// <lambda, dG r_before> and lambda <- G^T lambda.  States before each op are
// recomputed from checkpoints stored every K ops (K ~ sqrt(L)).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include <cmath>
#include <mutex>

#include "internal.h"

namespace qs {

namespace {

constexpr int kDmThreads = 128;
constexpr int kDmMaxQ = 6;
constexpr int kOpChunk = 256;   // ops staged in shared memory at a time

struct DmArgs {
  int n_circuits, max_q, max_ops, K, nseg, n_ptm1, n_ptm2;
  const int32_t* nq;
  const int64_t* op_off;
  const int32_t* ops;
  const double* params;
  const int64_t* out_off;
  const int32_t* counts;
  const double* ptm1;
  const double* ptm2;
  float* probs;
  double* loglik;
  double* grad;
  float* scratch;              // per CTA: (nseg + K) * 4^max_q floats
  int* work;                   // work counter (zeroed before launch)
  const int* order;            // circuits in the order they are handed out, or NULL
  int8_t cz_dst[16];            // CZ: Pauli string j maps to +-(string cz_dst[j])
  int8_t cz_sgn[16];
  int8_t cz_inv[16];            // inverse: string l comes from cz_inv[l] with sign cz_isgn[l]
  int8_t cz_isgn[16];
};

// tables in shared memory (16 floats each)
enum {
  TB_GX = 0, TB_GY, TB_C,                     // forward PTMs
  TB_GX_T, TB_GX_P, TB_GX_G,                  // d GX / d(theta_x, p, gamma)
  TB_GY_T, TB_GY_P, TB_GY_G,                  // d GY / d(theta_y, p, gamma)
  TB_C_P, TB_C_G,                             // d C / d(p, gamma)
  TB_COUNT
};

struct SubOp {
  int kind;      // 0: 4x4 table on q; 1: CZ permutation on (a, b); 2: user 4x4; 3: user 16x16
  int q, b;      // qubits
  int table;     // TB_* (kind 0) or user index (kind 2, 3)
  int dtab[4];   // derivative tables per parameter (theta_x, theta_y, p, gamma) or -1
};

// number of sub-ops of an op, and sub-op j (formed on demand: an array of them
// indexed by a loop variable would live in local memory)
__device__ __forceinline__ int op_nsub(const int32_t* op, int n) {
  switch (op[0]) {
    case QS_DM_CZ: return 3;
    case QS_DM_IDLE: return n;
    default: return 1;
  }
}
__device__ __forceinline__ SubOp op_subop(const int32_t* op, int j) {
  const int code = op[0], a = op[1], b = op[2], aux = op[3];
  SubOp x;
  x.kind = 0;
  x.q = a;
  x.b = -1;
  x.table = TB_C;
  x.dtab[0] = x.dtab[1] = -1;
  x.dtab[2] = TB_C_P;
  x.dtab[3] = TB_C_G;
  switch (code) {
    case QS_DM_X90:
      x.table = TB_GX;
      x.dtab[0] = TB_GX_T;
      x.dtab[2] = TB_GX_P;
      x.dtab[3] = TB_GX_G;
      break;
    case QS_DM_Y90:
      x.table = TB_GY;
      x.dtab[1] = TB_GY_T;
      x.dtab[2] = TB_GY_P;
      x.dtab[3] = TB_GY_G;
      break;
    case QS_DM_CZ:   // the permutation, then the channel on a, then on b
      if (j == 0) {
        x.kind = 1;
        x.b = b;
        x.table = -1;
        x.dtab[2] = x.dtab[3] = -1;
      } else if (j == 2) {
        x.q = b;
      }
      break;
    case QS_DM_IDLE: x.q = j; break;   // the channel on every qubit
    case QS_DM_PTM1:
      x.kind = 2;
      x.table = aux;
      x.dtab[2] = x.dtab[3] = -1;
      break;
    default:   // QS_DM_PTM2
      x.kind = 3;
      x.b = b;
      x.table = aux;
      x.dtab[2] = x.dtab[3] = -1;
  }
  return x;
}

__device__ bool op_valid(const int32_t* op, int n, const DmArgs& A) {
  const int code = op[0], a = op[1], b = op[2], aux = op[3];
  switch (code) {
    case QS_DM_X90: case QS_DM_Y90: return a >= 0 && a < n;
    case QS_DM_CZ: return a >= 0 && a < n && b >= 0 && b < n && a != b;
    case QS_DM_IDLE: return true;
    case QS_DM_PTM1: return a >= 0 && a < n && aux >= 0 && aux < A.n_ptm1 && A.ptm1 != nullptr;
    case QS_DM_PTM2:
      return a >= 0 && a < n && b >= 0 && b < n && a != b && aux >= 0 && aux < A.n_ptm2 &&
             A.ptm2 != nullptr;
    default: return false;
  }
}

__device__ __forceinline__ int group_base(int g, int q) {
  // insert a zero base-4 digit at position q
  const int lo = g & ((1 << (2 * q)) - 1);
  return ((g >> (2 * q)) << (2 * q + 2)) | lo;
}

// Shared-memory layout of a Pauli vector: entry i sits at word swz(i) = i ^ m(i >> 5),
// with m a fixed GF(2)-linear map of the index bits 5..11 into the bank bits 0..4.
// The sweeps read the elements of a base-4 digit at strides 1, 4, 16, ... words, which
// put up to four lanes of a warp on one bank in the plain layout; m was chosen by a
// search over every access pattern of the sweeps below (one- and two-digit, 4..6
// qubits) so that a warp's accesses meet 1856 wavefronts over 1760 patterns against
// 7080 in the plain layout.  swz is linear over XOR, so the index of a group's base
// and of its elements' offsets (disjoint bits) combine by XOR.  m(h) bit r = parity
// of h & kSwzRow[r]; a CTA keeps m for h = 0..127 in s_swz.
__shared__ uint8_t s_swz[128];
__device__ __forceinline__ void swz_init() {
  constexpr unsigned kSwzRow[5] = {0x4f, 0x15, 0x6d, 0x33, 0x67};
  if (threadIdx.x < 128) {
    const unsigned h = threadIdx.x;
    unsigned m = 0;
#pragma unroll
    for (int r = 0; r < 5; ++r) m |= (unsigned)(__popc(h & kSwzRow[r]) & 1) << r;
    s_swz[h] = (uint8_t)m;
  }
}
__device__ __forceinline__ int swz(int i) { return i ^ (int)s_swz[i >> 5]; }
// the (swizzled) offsets of the four values of one digit at stride st; swz of
// 3 st is swz(st) ^ swz(2 st) (disjoint bits), so a run-time digit (the CZ
// permutation) costs two selects, no indexed load
struct Off4 {
  int o1, o2;
  __device__ __forceinline__ explicit Off4(int st) : o1(swz(st)), o2(swz(2 * st)) {}
  __device__ __forceinline__ int operator[](int d) const { return ((d & 1) ? o1 : 0) ^ ((d & 2) ? o2 : 0); }
};

// r <- G r (or G^T r) on digit q; G row-major 4x4 (output digit, input digit).
__device__ void apply4(float* r, int n, int q, const float* Gs, bool transpose) {
  const int groups = 1 << (2 * (n - 1));
  // the matrix in registers once per sweep
  float G[16];
#pragma unroll
  for (int d = 0; d < 4; ++d)
#pragma unroll
    for (int e = 0; e < 4; ++e) G[d * 4 + e] = transpose ? Gs[e * 4 + d] : Gs[d * 4 + e];
  const int st = 1 << (2 * q);
  const Off4 od(st);
  for (int g = threadIdx.x; g < groups; g += blockDim.x) {
    const int base = swz(group_base(g, q));
    float x[4], y[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) x[d] = r[base ^ od[d]];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      float acc = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e) acc = fmaf(G[d * 4 + e], x[e], acc);
      y[d] = acc;
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) r[base ^ od[d]] = y[d];
  }
}

// Adjoint of one 4x4 sub-op on digit q in one sweep.  Every derivative term
// lam . (dG x) (lam after the sub-op, x the state before it) equals
// sum_{d,e} dG[d][e] M[d][e] with M = sum over groups of lam x^T, so the sweep
// accumulates M (16 FP32 sums per thread), updates lam <- G^T lam in place, and
// contracts M with each parameter's derivative table once at the end (per-thread
// partials added to g in FP64).  x may be global (a stored state) or shared.
__device__ __forceinline__ void adj4(float* lam, const float* x_src, int n, int q, const float* Gs,
                                     const float* tabs, const int* dtab, double* g) {
  const int groups = 1 << (2 * (n - 1));
  float G[16], M[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    G[i] = Gs[i];
    M[i] = 0.f;
  }
  auto group = [&](const float (&x)[4], float (&l)[4]) {
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
      for (int e = 0; e < 4; ++e) M[d * 4 + e] = fmaf(l[d], x[e], M[d * 4 + e]);
    float y[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float acc = 0.f;
#pragma unroll
      for (int d = 0; d < 4; ++d) acc = fmaf(G[d * 4 + e], l[d], acc);
      y[e] = acc;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) l[e] = y[e];
  };
  {
    const int st = 1 << (2 * q);
    const Off4 od(st);
    for (int gi = threadIdx.x; gi < groups; gi += blockDim.x) {
      const int base = swz(group_base(gi, q));
      float x[4], l[4];
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        x[d] = x_src[base ^ od[d]];
        l[d] = lam[base ^ od[d]];
      }
      group(x, l);
#pragma unroll
      for (int d = 0; d < 4; ++d) lam[base ^ od[d]] = l[d];
    }
  }
#pragma unroll
  for (int pidx = 0; pidx < 4; ++pidx)
    if (dtab[pidx] >= 0) {
      const float* dG = tabs + 16 * dtab[pidx];
      float acc = 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) acc = fmaf(dG[i], M[i], acc);
      g[pidx] += (double)acc;
    }
}

__device__ __forceinline__ int group_base2(int g, int lo_q, int hi_q) {
  return group_base(group_base(g, lo_q), hi_q);
}

// two-digit ops: local index 4*d_a + d_b
__device__ void apply_cz(float* r, int n, int a, int b, const DmArgs& A, bool transpose) {
  const int groups = 1 << (2 * (n - 2));
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  const int sa = 1 << (2 * a), sb = 1 << (2 * b);
  const Off4 oa(sa), ob(sb);
  for (int g = threadIdx.x; g < groups; g += blockDim.x) {
    const int base = swz(group_base2(g, lo, hi));
    // forward: y[l] = isgn[l] x[inv[l]]; transpose: y[j] = sgn[j] x[dst[j]] (the
    // permutation is applied through the shared-memory addresses of the loads, so
    // every register index stays a compile-time constant)
    float y[16];
#pragma unroll
    for (int l = 0; l < 16; ++l) {
      const int src = transpose ? A.cz_dst[l] : A.cz_inv[l];
      const float sg = (float)(transpose ? A.cz_sgn[l] : A.cz_isgn[l]);
      y[l] = sg * r[base ^ oa[src >> 2] ^ ob[src & 3]];
    }
#pragma unroll
    for (int l = 0; l < 16; ++l) r[base ^ oa[l >> 2] ^ ob[l & 3]] = y[l];
  }
}

__device__ void apply16(float* r, int n, int a, int b, const double* G, bool transpose) {
  const int groups = 1 << (2 * (n - 2));
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  const int sa = 1 << (2 * a), sb = 1 << (2 * b);
  const Off4 oa(sa), ob(sb);
  for (int g = threadIdx.x; g < groups; g += blockDim.x) {
    const int base = swz(group_base2(g, lo, hi));
    float x[16];
    for (int l = 0; l < 16; ++l) x[l] = r[base ^ oa[l >> 2] ^ ob[l & 3]];
    for (int d = 0; d < 16; ++d) {
      float acc = 0.f;
      for (int e = 0; e < 16; ++e) acc = fmaf((float)(transpose ? G[e * 16 + d] : G[d * 16 + e]), x[e], acc);
      r[base ^ oa[d >> 2] ^ ob[d & 3]] = acc;
    }
  }
}

// Forward passes over two digits a != b at once (16-element groups, local index
// 4 d_a + d_b): an optional signed permutation applied through the load
// addresses (CZ), then Ga on digit a, then Gb on digit b -- the same operations,
// in the same order, as the separate one-digit passes, with one shared-memory
// sweep and one barrier instead of two or three.
template <bool CZ>
__device__ void pass2(float* r, int n, int a, const float* Ga, int b, const float* Gb, const DmArgs& A) {
  const int groups = 1 << (2 * (n - 2));
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  const int sa = 1 << (2 * a), sb = 1 << (2 * b);
  const Off4 oa(sa), ob(sb);
  const float* ga = Ga;   // shared memory (broadcast reads)
  const float* gb = Gb;
  for (int g = threadIdx.x; g < groups; g += blockDim.x) {
    const int base = swz(group_base2(g, lo, hi));
    float x[16], y[16];
#pragma unroll
    for (int l = 0; l < 16; ++l) {
      const int src = CZ ? A.cz_inv[l] : l;
      const float v = r[base ^ oa[src >> 2] ^ ob[src & 3]];
      x[l] = CZ ? (float)A.cz_isgn[l] * v : v;
    }
#pragma unroll
    for (int db = 0; db < 4; ++db)
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        float acc = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) acc = fmaf(ga[d * 4 + e], x[4 * e + db], acc);
        y[4 * d + db] = acc;
      }
#pragma unroll
    for (int da = 0; da < 4; ++da)
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        float acc = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) acc = fmaf(gb[d * 4 + e], y[4 * da + e], acc);
        x[4 * da + d] = acc;
      }
#pragma unroll
    for (int l = 0; l < 16; ++l) r[base ^ oa[l >> 2] ^ ob[l & 3]] = x[l];
  }
}

__device__ void apply_sub(float* r, int n, const SubOp& s, const float* tabs, float* user4,
                          const DmArgs& A, bool transpose) {
  switch (s.kind) {
    case 0: apply4(r, n, s.q, tabs + 16 * s.table, transpose); break;
    case 1: apply_cz(r, n, s.q, s.b, A, transpose); break;
    case 2: apply4(r, n, s.q, user4, transpose); break;
    default: apply16(r, n, s.q, s.b, A.ptm2 + 256 * (size_t)s.table, transpose); break;
  }
}

__device__ double block_sum_dm(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  __syncthreads();
  return s;   // valid in every thread
}

__device__ void build_tables(float* tabs, const double* prm) {
  // thread 0 only
  const double tx = prm[0], ty = prm[1], p = prm[2], g = prm[3];
  const double f = 1.0 - 4.0 * p / 3.0, s = sqrt(1.0 - g);
  double C[16] = {1, 0, 0, 0, 0, s * f, 0, 0, 0, 0, s * f, 0, g, 0, 0, (1 - g) * f};
  double Cp[16] = {0, 0, 0, 0, 0, -4.0 * s / 3.0, 0, 0, 0, 0, -4.0 * s / 3.0, 0, 0, 0, 0,
                   -(1 - g) * 4.0 / 3.0};
  double Cg[16] = {0, 0, 0, 0, 0, -f / (2 * s), 0, 0, 0, 0, -f / (2 * s), 0, 1, 0, 0, -f};
  const double cx = cos(tx), sx = sin(tx), cy = cos(ty), sy = sin(ty);
  double RX[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, cx, -sx, 0, 0, sx, cx};
  double dRX[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, -sx, -cx, 0, 0, cx, -sx};
  double RY[16] = {1, 0, 0, 0, 0, cy, 0, sy, 0, 0, 1, 0, 0, -sy, 0, cy};
  double dRY[16] = {0, 0, 0, 0, 0, -sy, 0, cy, 0, 0, 0, 0, 0, -cy, 0, -sy};
  auto mul = [](const double* A, const double* B, float* out) {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        double acc = 0;
        for (int k = 0; k < 4; ++k) acc += A[i * 4 + k] * B[k * 4 + j];
        out[i * 4 + j] = (float)acc;
      }
  };
  mul(C, RX, tabs + 16 * TB_GX);
  mul(C, RY, tabs + 16 * TB_GY);
  for (int i = 0; i < 16; ++i) tabs[16 * TB_C + i] = (float)C[i];
  mul(C, dRX, tabs + 16 * TB_GX_T);
  mul(Cp, RX, tabs + 16 * TB_GX_P);
  mul(Cg, RX, tabs + 16 * TB_GX_G);
  mul(C, dRY, tabs + 16 * TB_GY_T);
  mul(Cp, RY, tabs + 16 * TB_GY_P);
  mul(Cg, RY, tabs + 16 * TB_GY_G);
  for (int i = 0; i < 16; ++i) {
    tabs[16 * TB_C_P + i] = (float)Cp[i];
    tabs[16 * TB_C_G + i] = (float)Cg[i];
  }
}

// index of the Pauli string Z_S (digit 3 at the bits of S)
__device__ __forceinline__ int zs_index(int S, int n) {
  int idx = 0;
  for (int b = 0; b < n; ++b)
    if ((S >> b) & 1) idx |= 3 << (2 * b);
  return idx;
}

__device__ void wht(double* z, int N) {
  for (int h = 1; h < N; h <<= 1) {
    for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
      const int j = ((i & ~(h - 1)) << 1) | (i & (h - 1));
      const double a = z[j], b = z[j + h];
      z[j] = a + b;
      z[j + h] = a - b;
    }
    __syncthreads();
  }
}

// One op forward with the fused two-digit passes: CZ as its permutation and both
// channels in one pass, the idle op as channel pairs -- the operations of its
// sub-ops in the same order, with the same arithmetic.  user4 holds the op's PTM
// for QS_DM_PTM1.  Ends with a barrier.
__device__ void apply_op_fused(float* r, int n, const int32_t* op, const float* tabs,
                               const float* user4, const DmArgs& A) {
  const int code = op[0], a = op[1], b = op[2];
  const float* C = tabs + 16 * TB_C;
  if (code == QS_DM_X90 || code == QS_DM_Y90) {
    apply4(r, n, a, tabs + 16 * (code == QS_DM_X90 ? TB_GX : TB_GY), false);
  } else if (code == QS_DM_CZ) {
    pass2<true>(r, n, a, C, b, C, A);
  } else if (code == QS_DM_IDLE) {
    for (int q = 0; q + 1 < n; q += 2) {
      pass2<false>(r, n, q, C, q + 1, C, A);
      __syncthreads();
    }
    if (n & 1) apply4(r, n, n - 1, C, false);
  } else if (code == QS_DM_PTM1) {
    apply4(r, n, a, user4, false);
  } else {
    apply16(r, n, a, b, A.ptm2 + 256 * (size_t)op[3], false);
  }
  __syncthreads();
}

// Longest first: the persistent kernel hands out circuits in this order, so the
// longest ones start in the first wave instead of setting the batch time at its
// end.  Estimated cost (ops + 1) x (4^n + 64) (the Pauli-vector sweeps plus a
// per-op floor), sorted descending with a bitonic network in shared memory
// (keys: cost as float bits above the circuit index; one CTA, up to kOrderMax
// circuits; padding keys 0 sort last).  Used for the gradient pass, whose
// per-circuit time (forward, backward sweep, scratch traffic) makes its tail long;
// the forward pass keeps index order, where long and short circuits mixed on one
// SM overlap better (4096 mixed circuits: 1.40 ms in index order, 1.60 sorted;
// the gradient 8.63 -> 6.51 ms sorted).
constexpr int kOrderMax = 16384;

__global__ void __launch_bounds__(1024) dm_order_kernel(const int32_t* __restrict__ nq,
                                                        const int64_t* __restrict__ op_off, int n,
                                                        int* __restrict__ order) {
  extern __shared__ unsigned long long keys[];
  int P = 1;
  while (P < n) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    unsigned long long k = 0;
    if (i < n) {
      int q = nq[i];
      q = q < 1 ? 1 : (q > kDmMaxQ ? kDmMaxQ : q);
      long long L = op_off[i + 1] - op_off[i];
      L = L < 0 ? 0 : (L > (1 << 20) ? (1 << 20) : L);
      const float cost = (float)(L + 1) * (float)((1 << (2 * q)) + 64);
      k = ((unsigned long long)__float_as_uint(cost) << 32) | (unsigned)i;
    }
    keys[i] = k;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long a = keys[i], b = keys[l];
          const bool desc = (i & k) == 0;   // descending runs first
          if (desc ? (a < b) : (a > b)) {
            keys[i] = b;
            keys[l] = a;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < n; i += blockDim.x) order[i] = (int)(keys[i] & 0xffffffffu);
}

// dynamic shared memory: tables, user PTM, WHT buffer, then the Pauli vector r
// (and, with the gradient, lambda and a scratch vector)
constexpr int kDmHead = 16 * TB_COUNT + 16 + 128;   // floats before r (16-byte aligned)
// One circuit c (validated, tables built) on one CTA.
template <bool GRAD>
__device__ __forceinline__ void dm_circuit(const DmArgs& A, int c, int n, int L, const int32_t* ops, int64_t out0,
                                           int D, float* tabs, float* user4, double* z, float* r, float* lam,
                                           float* tmp, double* red, int4* s_ops, float* ckpt, float* segbuf,
                                           float* subst) {
  constexpr bool want_grad = GRAD;
  const int N = 1 << n;
  const int Dn = 1 << (2 * n);
  const float amp0 = 1.0f / sqrtf((float)N);
  // rho_0 = |0..0><0..0|: r_i = 2^{-n/2} on {I,Z}^n, 0 elsewhere
  for (int i = threadIdx.x; i < Dn; i += blockDim.x) {
    bool iz = true;
    for (int b = 0; b < n; ++b) {
      const int d = (i >> (2 * b)) & 3;
      iz = iz && (d == 0 || d == 3);
    }
    r[swz(i)] = iz ? amp0 : 0.f;
  }
  __syncthreads();
  // ---------------- forward
  const int4* ops4 = reinterpret_cast<const int4*>(ops);
  if constexpr (!GRAD) {
    for (int k = 0; k < L;) {
      if ((k % kOpChunk) == 0) {   // stage the next chunk of ops (one coalesced read)
        __syncthreads();
        for (int t = threadIdx.x; t < kOpChunk && k + t < L; t += blockDim.x) s_ops[t] = ops4[k + t];
        __syncthreads();
      }
      const int32_t* op = reinterpret_cast<const int32_t*>(&s_ops[k % kOpChunk]);
      const int code = op[0], a = op[1];
      const int32_t* nx = reinterpret_cast<const int32_t*>(&s_ops[(k + 1) % kOpChunk]);
      if ((code == QS_DM_X90 || code == QS_DM_Y90) && k + 1 < L && (k + 1) % kOpChunk != 0 &&
          (nx[0] == QS_DM_X90 || nx[0] == QS_DM_Y90) && nx[1] != a) {
        // this op and the next act on different qubits: one two-digit pass
        pass2<false>(r, n, a, tabs + 16 * (code == QS_DM_X90 ? TB_GX : TB_GY), nx[1],
                     tabs + 16 * (nx[0] == QS_DM_X90 ? TB_GX : TB_GY), A);
        __syncthreads();
        k += 2;
        continue;
      }
      if (code == QS_DM_PTM1) {
        if (threadIdx.x < 16) user4[threadIdx.x] = (float)A.ptm1[16 * (size_t)op[3] + threadIdx.x];
        __syncthreads();
      }
      apply_op_fused(r, n, op, tabs, user4, A);
      ++k;
    }
  }
  for (int k = 0; GRAD && k < L; ++k) {
    if ((k % kOpChunk) == 0) {   // stage the next chunk of ops (one coalesced read)
      __syncthreads();
      for (int t = threadIdx.x; t < kOpChunk && k + t < L; t += blockDim.x) s_ops[t] = ops4[k + t];
      __syncthreads();
    }
    if (want_grad && (k % A.K) == 0) {
      float* dst = ckpt + (size_t)(k / A.K) * D;
      for (int i = threadIdx.x; i < Dn; i += blockDim.x) dst[i] = r[i];
      __syncthreads();   // copies done before r is updated in place
    }
    const int32_t* op = reinterpret_cast<const int32_t*>(&s_ops[k % kOpChunk]);
    if (op[0] == QS_DM_PTM1) {
      if (threadIdx.x < 16) user4[threadIdx.x] = (float)A.ptm1[16 * (size_t)op[3] + threadIdx.x];
      __syncthreads();
    }
    apply_op_fused(r, n, op, tabs, user4, A);
  }
  // ---------------- probabilities: p = 2^{-n/2} WHT(r on {I,Z}^n)
  for (int S = threadIdx.x; S < N; S += blockDim.x) z[S] = (double)r[swz(zs_index(S, n))];
  __syncthreads();
  wht(z, N);
  const double scale = 1.0 / sqrt((double)N);
  double ll = 0.0;
  for (int J = threadIdx.x; J < N; J += blockDim.x) {
    double p = z[J] * scale;
    if (A.probs) A.probs[out0 + J] = (float)p;
    if (A.counts) {
      const int cnt = A.counts[out0 + J];
      if (!(p > 0.0)) p = 1e-300;
      if (cnt > 0) ll += (double)cnt * log(p);
      z[J] = cnt > 0 ? (double)cnt / p : 0.0;   // seed weights dl/dp_J
    }
  }
  if (A.counts) {
    const double tot = block_sum_dm(ll, red);
    if (threadIdx.x == 0 && A.loglik) A.loglik[c] = tot;
  }
  if constexpr (!GRAD) return;
  // ---------------- adjoint
  __syncthreads();
  wht(z, N);
  // lambda is linear in the seed: keep it in fp32 as lambda / lmax (no
  // overflow when some n_J / p_J is huge) and scale the fp64 sums back
  double lmax = 0.0;
  for (int S = 0; S < N; ++S) lmax = fmax(lmax, fabs(z[S]));
  const double lscale = lmax > 0.0 ? scale / lmax : 0.0;
  for (int i = threadIdx.x; i < Dn; i += blockDim.x) lam[i] = 0.f;
  __syncthreads();
  for (int S = threadIdx.x; S < N; S += blockDim.x) lam[swz(zs_index(S, n))] = (float)(z[S] * lscale);
  __syncthreads();
  double g[4] = {0, 0, 0, 0};
  const int nseg = (L + A.K - 1) / A.K;
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
    const int k0 = sgi * A.K, k1 = min(L, k0 + A.K);
    // recompute the states before each op of the segment
    const float* ck = ckpt + (size_t)sgi * D;
    for (int i = threadIdx.x; i < Dn; i += blockDim.x) r[i] = ck[i];
    __syncthreads();
    for (int k = k0; k < k1; ++k) {
      float* dst = segbuf + (size_t)(k - k0) * D;
      for (int i = threadIdx.x; i < Dn; i += blockDim.x) dst[i] = r[i];
      if (k + 1 == k1) break;
      const int32_t* op = ops + 4 * k;
      if (op[0] == QS_DM_PTM1) {
        __syncthreads();
        if (threadIdx.x < 16) user4[threadIdx.x] = (float)A.ptm1[16 * (size_t)op[3] + threadIdx.x];
        __syncthreads();
      }
      __syncthreads();
      apply_op_fused(r, n, op, tabs, user4, A);
    }
    __syncthreads();
    for (int k = k1 - 1; k >= k0; --k) {
      const int32_t* op = ops + 4 * k;
      if (op[0] == QS_DM_PTM1) {
        if (threadIdx.x < 16) user4[threadIdx.x] = (float)A.ptm1[16 * (size_t)op[3] + threadIdx.x];
      }
      const int ns = op_nsub(op, n);
      const float* before = segbuf + (size_t)(k - k0) * D;
      __syncthreads();
      // the states before the sub-ops, once: s_0 = before, s_{j+1} = sub_j s_j;
      // the last stays in tmp, the earlier ones with parameters go to subst
      if (ns > 1) {
        for (int i = threadIdx.x; i < Dn; i += blockDim.x) tmp[i] = before[i];
        __syncthreads();
        for (int j = 0; j + 1 < ns; ++j) {
          apply_sub(tmp, n, op_subop(op, j), tabs, user4, A, false);
          __syncthreads();
          if (j + 2 < ns && op_subop(op, j + 1).kind == 0) {
            for (int i = threadIdx.x; i < Dn; i += blockDim.x) subst[(size_t)(j + 1) * D + i] = tmp[i];
            __syncthreads();   // copied before sub-op j + 1 rewrites tmp
          }
        }
      }
      for (int j = ns - 1; j >= 0; --j) {
        const SubOp sj = op_subop(op, j);
        if (sj.kind == 0) {
          const float* sv = j + 1 == ns ? (ns > 1 ? tmp : before) : (j == 0 ? before : subst + (size_t)j * D);
          adj4(lam, sv, n, sj.q, tabs + 16 * sj.table, tabs, sj.dtab, g);
        } else {
          apply_sub(lam, n, sj, tabs, user4, A, true);
        }
        __syncthreads();
      }
    }
  }
  for (int pidx = 0; pidx < 4; ++pidx) {
    const double tot = block_sum_dm(g[pidx], red);
    if (threadIdx.x == 0) A.grad[4 * c + pidx] = tot * lmax;
  }
}

// GRAD: the gradient kernel (forward with checkpoints, then the adjoint sweep);
// otherwise probabilities / log-likelihood only, with one-qubit gate pairs fused
// too and a third of the shared memory (more CTAs per SM)
template <bool GRAD>
__global__ void __launch_bounds__(kDmThreads, GRAD ? 4 : 6) dm_batch_kernel(DmArgs A) {
  extern __shared__ __align__(16) float dsm[];
  const int D = 1 << (2 * A.max_q);
  float* tabs = dsm;                         // TB_COUNT * 16
  float* user4 = tabs + 16 * TB_COUNT;       // 16
  double* z = (double*)(user4 + 16);         // 64 doubles (8-byte aligned: offsets are multiples of 16 floats)
  float* r = dsm + kDmHead;
  float* lam = r + D;                        // GRAD only
  float* tmp = r + 2 * D;                    // GRAD only
  __shared__ double red[kDmThreads / 32];
  __shared__ int s_c;
  __shared__ int4 s_ops[kOpChunk];   // the current chunk of the circuit's ops
  float* my_scratch =
      A.scratch ? A.scratch + (size_t)blockIdx.x * (size_t)(A.nseg + A.K + kDmMaxQ) * D : nullptr;
  float* ckpt = my_scratch;
  float* segbuf = my_scratch ? my_scratch + (size_t)A.nseg * D : nullptr;
  float* subst = my_scratch ? my_scratch + (size_t)(A.nseg + A.K) * D : nullptr;
  swz_init();   // read after the first barrier of the loop below

  for (;;) {
    if (threadIdx.x == 0) {
      const int w = atomicAdd(A.work, 1);
      s_c = (A.order && w < A.n_circuits) ? A.order[w] : w;
    }
    __syncthreads();
    const int c = s_c;
    __syncthreads();
    if (c >= A.n_circuits) break;
    const int n = A.nq[c];
    const int64_t o0 = A.op_off[c];
    const int L = (int)(A.op_off[c + 1] - o0);
    const int32_t* ops = A.ops + 4 * o0;
    const int64_t out0 = A.out_off[c];
    const int N = 1 << n;
    // validation (device side: the arrays are caller-supplied device memory),
    // ops checked by all threads in parallel
    bool ok = n >= 1 && n <= A.max_q && L >= 0 && L <= A.max_ops && A.out_off[c + 1] - out0 == N;
    if (ok)
      for (int k = threadIdx.x; k < L; k += blockDim.x) ok = ok && op_valid(ops + 4 * k, n, A);
    const bool all_ok = __syncthreads_and(ok) != 0;
    if (all_ok && threadIdx.x == 0) build_tables(tabs, A.params + 4 * c);
    __syncthreads();
    if (!all_ok) {
      const float nanf_ = __int_as_float(0x7fc00000);
      if (threadIdx.x == 0) {
        if (A.loglik) A.loglik[c] = __longlong_as_double(0x7ff8000000000000ll);
        if (A.grad)
          for (int k = 0; k < 4; ++k) A.grad[4 * c + k] = __longlong_as_double(0x7ff8000000000000ll);
      }
      if (A.probs && n >= 1 && n <= kDmMaxQ && A.out_off[c + 1] - out0 == N)
        for (int J = threadIdx.x; J < N; J += blockDim.x) A.probs[out0 + J] = nanf_;
      continue;
    }
    dm_circuit<GRAD>(A, c, n, L, ops, out0, D, tabs, user4, z, r, lam, tmp, red, s_ops, ckpt, segbuf, subst);
    __syncthreads();
  }
}

// CZ as a signed permutation of two-qubit Pauli strings, from
// G_ij = Tr(P_i U P_j U^dagger) / 4 with U = diag(1, 1, 1, -1).
void cz_table(int8_t* dst, int8_t* sgn) {
  const cd I(0, 1);
  const cd P[4][4] = {{1, 0, 0, 1}, {0, 1, 1, 0}, {0, -I, I, 0}, {1, 0, 0, -1}};
  const double u[4] = {1, 1, 1, -1};
  auto pauli2 = [&](int idx, cd* M) {   // idx = 4*d_a + d_b, qubit a most significant
    const cd* A = P[idx >> 2];
    const cd* B = P[idx & 3];
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) M[r * 4 + c] = A[(r >> 1) * 2 + (c >> 1)] * B[(r & 1) * 2 + (c & 1)];
  };
  for (int j = 0; j < 16; ++j) {
    cd Pj[16], Pi[16], img[16];
    pauli2(j, Pj);
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) img[r * 4 + c] = u[r] * Pj[r * 4 + c] * u[c];
    for (int i = 0; i < 16; ++i) {
      pauli2(i, Pi);
      cd tr = 0;
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) tr += Pi[r * 4 + c] * img[c * 4 + r];
      const double v = tr.real() / 4.0;
      if (std::fabs(v) > 0.5) {
        dst[j] = (int8_t)i;
        sgn[j] = (int8_t)(v > 0 ? 1 : -1);
      }
    }
  }
}

}  // namespace

// QS_DM_VALIDATE: the user PTMs must be channels (trace preserving and completely
// positive), the built-in channels' parameters in range (p, gamma in [0, 1],
// finite angles); the device arrays are read on the host first.
qs_status dm_validate_batch(const qs_dm_batch* b, cudaStream_t stream) {
  if (b->n_ptm1 < 0 || b->n_ptm2 < 0 || (b->n_ptm1 > 0 && !b->ptm1) || (b->n_ptm2 > 0 && !b->ptm2)) {
    set_error("PTM tables: counts %d, %d with %s", b->n_ptm1, b->n_ptm2, "a missing array");
    return QS_EINVAL;
  }
  std::vector<double> h1((size_t)b->n_ptm1 * 16), h2((size_t)b->n_ptm2 * 256), par((size_t)b->n_circuits * 4);
  if (!h1.empty())
    QS_CUDA(cudaMemcpyAsync(h1.data(), b->ptm1, h1.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
  if (!h2.empty())
    QS_CUDA(cudaMemcpyAsync(h2.data(), b->ptm2, h2.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
  QS_CUDA(cudaMemcpyAsync(par.data(), b->params, par.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
  QS_CUDA(cudaStreamSynchronize(stream));
  qs_status s = ptm_validate(h1.data(), 1, b->n_ptm1, "ptm1", nullptr);
  if (s == QS_OK) s = ptm_validate(h2.data(), 2, b->n_ptm2, "ptm2", nullptr);
  if (s != QS_OK) return s;
  for (int c = 0; c < b->n_circuits; ++c) {
    const double* q = par.data() + 4 * (size_t)c;
    if (!std::isfinite(q[0]) || !std::isfinite(q[1]) || !(q[2] >= 0.0 && q[2] <= 1.0) ||
        !(q[3] >= 0.0 && q[3] <= 1.0)) {
      set_error("circuit %d: parameters (theta_x %g, theta_y %g, p %g, gamma %g) do not give channels "
                "(p and gamma must lie in [0, 1])", c, q[0], q[1], q[2], q[3]);
      return QS_EINVAL;
    }
  }
  return QS_OK;
}

}  // namespace qs

using namespace qs;

extern "C" qs_status dm_apply_channels(const qs_dm_batch* b, float* probs, double* loglik,
                                       double* grad, void* stream_) {
  if (!b) {
    set_error("batch is NULL");
    return QS_EINVAL;
  }
  if (b->n_circuits < 0 || b->max_qubits < 1 || b->max_qubits > kDmMaxQ || b->max_ops < 0) {
    set_error("bad batch sizes (n_circuits %d, max_qubits %d, max_ops %d)", b->n_circuits,
              b->max_qubits, b->max_ops);
    return QS_EINVAL;
  }
  if (!b->nq || !b->op_off || !b->params || !b->out_off || (b->max_ops > 0 && !b->ops)) {
    set_error("batch arrays missing");
    return QS_EINVAL;
  }
  if ((loglik || grad) && !b->counts) {
    set_error("loglik / grad need counts");
    return QS_EINVAL;
  }
  if (b->flags & ~QS_DM_VALIDATE) {
    set_error("unknown batch flags 0x%x", b->flags);
    return QS_EINVAL;
  }
  if (b->n_circuits == 0) return QS_OK;
  cudaStream_t stream = (cudaStream_t)stream_;
  if (b->flags & QS_DM_VALIDATE) {
    const qs_status vs = dm_validate_batch(b, stream);
    if (vs != QS_OK) return vs;
  }
  DmArgs A{};
  A.n_circuits = b->n_circuits;
  A.max_q = b->max_qubits;
  A.max_ops = b->max_ops;
  A.K = 1;
  while (A.K * A.K < b->max_ops) ++A.K;
  A.nseg = (b->max_ops + A.K - 1) / A.K + 1;
  A.n_ptm1 = b->n_ptm1;
  A.n_ptm2 = b->n_ptm2;
  A.nq = b->nq;
  A.op_off = b->op_off;
  A.ops = b->ops;
  A.params = b->params;
  A.out_off = b->out_off;
  A.counts = b->counts;
  A.ptm1 = b->ptm1;
  A.ptm2 = b->ptm2;
  A.probs = probs;
  A.loglik = loglik;
  A.grad = grad;
  cz_table(A.cz_dst, A.cz_sgn);
  for (int j = 0; j < 16; ++j) {
    A.cz_inv[A.cz_dst[j]] = (int8_t)j;
    A.cz_isgn[A.cz_dst[j]] = A.cz_sgn[j];
  }

  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int D = 1 << (2 * A.max_q);
  const bool with_grad = grad != nullptr;
  const size_t smem = (size_t)(kDmHead + (with_grad ? 3 : 1) * D) * sizeof(float);
  auto kern = with_grad ? dm_batch_kernel<true> : dm_batch_kernel<false>;
  if (smem > 48 * 1024) {
    cudaError_t ea = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ea != cudaSuccess) return cuda_status(ea, "cudaFuncSetAttribute");
  }
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDmThreads, smem);
  if (per_sm < 1) per_sm = 1;
  int grid = sms * per_sm;
  if (grid > b->n_circuits) grid = b->n_circuits;

  const size_t scratch_floats = grad ? (size_t)grid * (A.nseg + A.K + kDmMaxQ) * D : 0;
  const bool sort = grad && A.n_circuits > 1 && A.n_circuits <= kOrderMax;
  const size_t order_bytes = sort ? ((sizeof(int) * (size_t)A.n_circuits + 255) & ~size_t(255)) : 0;
  const size_t bytes = 256 + order_bytes + scratch_floats * sizeof(float);
  void* mem = nullptr;
  cudaError_t e = cudaMallocAsync(&mem, bytes, stream);
  if (e != cudaSuccess) return cuda_status(e, "cudaMallocAsync (dm scratch)");
  A.work = (int*)mem;
  A.order = sort ? (const int*)((char*)mem + 256) : nullptr;
  A.scratch = grad ? (float*)((char*)mem + 256 + order_bytes) : nullptr;
  e = cudaMemsetAsync(mem, 0, 256, stream);
  if (e != cudaSuccess) return cuda_status(e, "cudaMemsetAsync");
  if (sort) {
    int P = 1;
    while (P < A.n_circuits) P <<= 1;
    const size_t osmem = sizeof(unsigned long long) * (size_t)P;
    if (osmem > 48 * 1024) {
      e = cudaFuncSetAttribute(dm_order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)osmem);
      if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute");
    }
    dm_order_kernel<<<1, 1024, osmem, stream>>>(A.nq, A.op_off, A.n_circuits, (int*)A.order);
  }
  kern<<<grid, kDmThreads, smem, stream>>>(A);
  e = cudaGetLastError();
  cudaFreeAsync(mem, stream);
  if (e != cudaSuccess) return cuda_status(e, "dm_batch_kernel launch");
  return QS_OK;
}
