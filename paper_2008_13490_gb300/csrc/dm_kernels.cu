// Batched density matrices in the Pauli basis (Pauli transfer matrices).
//
// A circuit's state is its Pauli vector r_i = Tr(P^_i rho), P^_i = P_i/sqrt(N)
// (Eq. (GSTVectorizedRho)), 4^n reals kept in shared memory (one CTA or one warp per
// circuit) or, for 1 and 2 qubits in the forward pass, in registers.  An op
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
//   CZ: a signed permutation of the 16 two-qubit Paulis (evaluated from the
//       trace formula at compile time).
// The noise channel after an op is C = AD(g) DEP(p) on each touched qubit.
//
// Gradient of l = sum_J n_J log p_J by an adjoint sweep: lambda_L = dl/dr =
// 2^{-n/2} WHT(n/p) on {I,Z}^n; backwards, each sub-op contributes
// <lambda, dG r_before> and lambda <- G^T lambda.  States before each op are
// recomputed from checkpoints stored every K ops (K ~ sqrt(L)).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "abi_guard.h"
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

// CZ conjugation as a signed permutation of the 16 two-qubit Pauli strings (index
// 4 d_a + d_b, digits I, x, y, z): G_ij = Tr(P_i U P_j U^dagger) / 4 with
// U = diag(1, 1, 1, -1), evaluated at compile time in Gaussian integers (the Pauli
// matrices' entries are 0, +-1, +-i) and packed 4 bits (string) / 1 bit (sign)
// per entry, so that the sweeps' loads and signs fold into constants.
namespace czc {
struct Gi {
  int re, im;
};
constexpr Gi mul(Gi a, Gi b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
constexpr Gi pauli(int d, int r, int c) {   // I, X, Y = [[0, -i], [i, 0]], Z
  return d == 0   ? Gi{r == c ? 1 : 0, 0}
         : d == 1 ? Gi{r != c ? 1 : 0, 0}
         : d == 2 ? Gi{0, r == c ? 0 : (r == 0 ? -1 : 1)}
                  : Gi{r == c ? (r == 0 ? 1 : -1) : 0, 0};
}
constexpr Gi pauli2(int idx, int r, int c) {   // qubit a (digit idx >> 2) most significant
  return mul(pauli(idx >> 2, r >> 1, c >> 1), pauli(idx & 3, r & 1, c & 1));
}
constexpr int trace4(int i, int j) {   // 4 G_ij = sum_{r,c} P_i[r][c] u_c P_j[c][r] u_r
  int t = 0;
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) t += (r == 3 ? -1 : 1) * (c == 3 ? -1 : 1) * mul(pauli2(i, r, c), pauli2(j, c, r)).re;
  return t;
}
constexpr int image(int j) {   // the string P_j goes to
  for (int i = 0; i < 16; ++i)
    if (trace4(i, j) != 0) return i;
  return -1;
}
constexpr bool is_signed_permutation() {
  bool hit[16] = {};
  for (int j = 0; j < 16; ++j) {
    int nz = 0;
    for (int i = 0; i < 16; ++i) {
      const int t = trace4(i, j);
      if (t != 0) {
        if (t != 4 && t != -4) return false;
        ++nz;
      }
    }
    if (nz != 1 || hit[image(j)]) return false;
    hit[image(j)] = true;
  }
  return true;
}
constexpr uint64_t pack_dst() {
  uint64_t p = 0;
  for (int j = 0; j < 16; ++j) p |= (uint64_t)image(j) << (4 * j);
  return p;
}
constexpr uint32_t pack_sgn() {
  uint32_t p = 0;
  for (int j = 0; j < 16; ++j) p |= (trace4(image(j), j) < 0 ? 1u : 0u) << j;
  return p;
}
constexpr uint64_t pack_inv() {
  uint64_t p = 0;
  for (int j = 0; j < 16; ++j) p |= (uint64_t)j << (4 * image(j));
  return p;
}
constexpr uint32_t pack_isgn() {
  uint32_t p = 0;
  for (int j = 0; j < 16; ++j) p |= (trace4(image(j), j) < 0 ? 1u : 0u) << image(j);
  return p;
}
}  // namespace czc
static_assert(czc::is_signed_permutation(), "CZ must permute the Pauli strings up to sign");
constexpr uint64_t kCzDst = czc::pack_dst();    // string j -> +-(string dst(j))
constexpr uint32_t kCzSgn = czc::pack_sgn();
constexpr uint64_t kCzInv = czc::pack_inv();    // string l <- +-(string inv(l))
constexpr uint32_t kCzISgn = czc::pack_isgn();
__device__ __forceinline__ int cz_dst(int j) { return (int)((kCzDst >> (4 * j)) & 15); }
__device__ __forceinline__ int cz_inv(int l) { return (int)((kCzInv >> (4 * l)) & 15); }
__device__ __forceinline__ bool cz_neg(int j) { return (kCzSgn >> j) & 1; }
__device__ __forceinline__ bool cz_ineg(int l) { return (kCzISgn >> l) & 1; }

// The threads that share one circuit's Pauli vector: a whole CTA (3 to 6 qubits in
// the forward pass, 5 and 6 with the gradient) or one warp (the gradient pass, up
// to kWarpMaxQ qubits, four circuits per CTA, no block barriers).  rank / kSize stride the sweeps, sync() orders the
// shared-memory updates between sweeps, kChunk ops are staged at a time.
constexpr int kWarpMaxQ = 4;
constexpr int kWarpD = 1 << (2 * kWarpMaxQ);   // 256 floats per Pauli vector
constexpr int kWarpChunk = 64;
struct CtaTeam {
  static constexpr int kSize = kDmThreads;
  static constexpr int kChunk = kOpChunk;
  double* red;   // kDmThreads / 32 doubles
  __device__ __forceinline__ int rank() const { return threadIdx.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ bool all(bool v) const { return __syncthreads_and(v) != 0; }
  __device__ double sum(double v) const {   // valid in every thread
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < kDmThreads / 32; ++i) s += red[i];
    __syncthreads();
    return s;
  }
};
struct WarpTeam {
  static constexpr int kSize = 32;
  static constexpr int kChunk = kWarpChunk;
  int lane;
  __device__ __forceinline__ int rank() const { return lane; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
  __device__ __forceinline__ bool all(bool v) const { return __all_sync(0xffffffffu, v) != 0; }
  __device__ __forceinline__ double sum(double v) const {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  }
};

// Nonzero pattern of a 4x4 table, known at compile time.  Every table that
// build_tables writes (the gates with their channel, the channel alone, and all
// their derivatives) has row 0 = (m00, 0, 0, 0) and m10 = m20 = 0 (trace
// preservation; amplitude damping feeds I into z only), and m12 = m21 = 0 (R^x
// mixes y with z, R^y mixes x with z, the channel keeps x and y apart): kTP, 9
// entries.  The
// channel alone is diag(1, sf, sf, hf) plus m30: kChan, 5 entries.  User PTMs are
// kDense.  The sweeps skip the structural zeros, adding the other terms in the
// same order as the dense sums, so the results are the same bits.
enum { kDense = 0, kTP = 1, kChan = 2 };
// Row 0 of every table applied through kTP or kChan is exactly (1, 0, 0, 0): they are
// the gates with their channel and the channel alone (the derivative tables, whose
// row 0 is zero, are only contracted with M, never applied), so the sweeps copy
// the I entry instead of forming 1 * x.
template <int F>
__host__ __device__ constexpr bool unit_row0() { return F != kDense; }
template <int F>
__host__ __device__ constexpr bool nz(int d, int e) {
  return F == kDense ? true
         : F == kTP  ? (d == 0 ? e == 0 : d == 1 ? (e == 1 || e == 3) : d == 2 ? (e == 2 || e == 3) : true)
                     : (d == e || (d == 3 && e == 0));
}

// A 4x4 table (shared memory, 16-byte aligned) into registers with four 16-byte
// loads (the same address in every lane: one broadcast wavefront each).
__device__ __forceinline__ void load16(const float* src, float (&G)[16]) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 v = s4[i];
    G[4 * i] = v.x;
    G[4 * i + 1] = v.y;
    G[4 * i + 2] = v.z;
    G[4 * i + 3] = v.w;
  }
}

// r <- G r (or G^T r, F = kDense only) on digit q; G row-major 4x4 (output digit,
// input digit) of pattern F.
template <class T, int F = kDense>
__device__ void apply4(const T& t, float* r, int n, int q, const float* Gs, bool transpose) {
  const int groups = 1 << (2 * (n - 1));
  // the matrix in registers once per sweep
  float G0[16], G[16];
  load16(Gs, G0);
#pragma unroll
  for (int d = 0; d < 4; ++d)
#pragma unroll
    for (int e = 0; e < 4; ++e) G[d * 4 + e] = transpose ? G0[e * 4 + d] : G0[d * 4 + e];
  const int st = 1 << (2 * q);
  const Off4 od(st);
  for (int g = t.rank(); g < groups; g += T::kSize) {
    const int base = swz(group_base(g, q));
    float x[4], y[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) x[d] = r[base ^ od[d]];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      if (d == 0 && unit_row0<F>()) {
        y[0] = x[0];
        continue;
      }
      float acc = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (nz<F>(d, e)) acc = fmaf(G[d * 4 + e], x[e], acc);
      y[d] = acc;
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) r[base ^ od[d]] = y[d];
  }
}

// Adjoint of one 4x4 sub-op on digit q in one sweep (a built-in table: pattern
// kTP, the derivative tables too, so the other entries of M are never needed).  Every derivative term
// lam . (dG x) (lam after the sub-op, x the state before it) equals
// sum_{d,e} dG[d][e] M[d][e] with M = sum over groups of lam x^T, so the sweep
// accumulates M (16 FP32 sums per thread), updates lam <- G^T lam in place, and
// contracts M with each parameter's derivative table once at the end (per-thread
// partials added to g in FP64).  x may be global (a stored state) or shared.
template <class T>
__device__ __forceinline__ void adj4(const T& t, float* lam, const float* x_src, int n, int q, const float* Gs,
                                     const float* tabs, const int* dtab, double* g) {
  const int groups = 1 << (2 * (n - 1));
  float G[16], M[16];
  load16(Gs, G);
#pragma unroll
  for (int i = 0; i < 16; ++i) M[i] = 0.f;
  const int st = 1 << (2 * q);
  const Off4 od(st);
  for (int gi = t.rank(); gi < groups; gi += T::kSize) {
    const int base = swz(group_base(gi, q));
    float x[4], l[4], y[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      x[d] = x_src[base ^ od[d]];
      l[d] = lam[base ^ od[d]];
    }
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (nz<kTP>(d, e)) M[d * 4 + e] = fmaf(l[d], x[e], M[d * 4 + e]);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float acc = 0.f;
#pragma unroll
      for (int d = 0; d < 4; ++d)
        if (nz<kTP>(d, e)) acc = fmaf(G[d * 4 + e], l[d], acc);
      y[e] = acc;
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) lam[base ^ od[d]] = y[d];
  }
#pragma unroll
  for (int pidx = 0; pidx < 4; ++pidx)
    if (dtab[pidx] >= 0) {
      const float* dG = tabs + 16 * dtab[pidx];
      float acc = 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (nz<kTP>(i >> 2, i & 3)) acc = fmaf(dG[i], M[i], acc);
      g[pidx] += (double)acc;
    }
}

__device__ __forceinline__ int group_base2(int g, int lo_q, int hi_q) {
  return group_base(group_base(g, lo_q), hi_q);
}

// two-digit ops: local index 4*d_a + d_b.  The CZ permutation goes through the
// load addresses (forward: y[l] = +-x[inv(l)]; transpose: y[j] = +-x[dst(j)]),
// so every register index stays a compile-time constant.
template <class T, bool TR>
__device__ void apply_cz_t(const T& t, float* r, int n, int a, int b) {
  const int groups = 1 << (2 * (n - 2));
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  const Off4 oa(1 << (2 * a)), ob(1 << (2 * b));
  for (int g = t.rank(); g < groups; g += T::kSize) {
    const int base = swz(group_base2(g, lo, hi));
    float y[16];
#pragma unroll
    for (int l = 0; l < 16; ++l) {
      const int src = TR ? cz_dst(l) : cz_inv(l);
      const float v = r[base ^ oa[src >> 2] ^ ob[src & 3]];
      y[l] = (TR ? cz_neg(l) : cz_ineg(l)) ? -v : v;
    }
#pragma unroll
    for (int l = 0; l < 16; ++l) r[base ^ oa[l >> 2] ^ ob[l & 3]] = y[l];
  }
}
template <class T>
__device__ void apply_cz(const T& t, float* r, int n, int a, int b, bool transpose) {
  if (transpose)
    apply_cz_t<T, true>(t, r, n, a, b);
  else
    apply_cz_t<T, false>(t, r, n, a, b);
}

template <class T>
__device__ void apply16(const T& t, float* r, int n, int a, int b, const double* G, bool transpose) {
  const int groups = 1 << (2 * (n - 2));
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  const Off4 oa(1 << (2 * a)), ob(1 << (2 * b));
  for (int g = t.rank(); g < groups; g += T::kSize) {
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

// One 4x4 table of pattern F on digit a (stage_a: out[4d + j] = sum_e G[d][e] in[4e + j])
// or digit b (stage_b: out[4j + d] = sum_e G[d][e] in[4j + e]) of a 16-element group
// in registers; the table's rows are 16-byte broadcast reads from shared memory.
template <int F>
__device__ __forceinline__ void stage_a(const float* G, const float (&in)[16], float (&out)[16]) {
  const float4* g4 = reinterpret_cast<const float4*>(G);
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    if (d == 0 && unit_row0<F>()) {
#pragma unroll
      for (int j = 0; j < 4; ++j) out[j] = in[j];
      continue;
    }
    const float4 row = g4[d];
    const float gr[4] = {row.x, row.y, row.z, row.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (nz<F>(d, e)) acc = fmaf(gr[e], in[4 * e + j], acc);
      out[4 * d + j] = acc;
    }
  }
}
template <int F>
__device__ __forceinline__ void stage_b(const float* G, const float (&in)[16], float (&out)[16]) {
  const float4* g4 = reinterpret_cast<const float4*>(G);
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    if (d == 0 && unit_row0<F>()) {
#pragma unroll
      for (int j = 0; j < 4; ++j) out[4 * j] = in[4 * j];
      continue;
    }
    const float4 row = g4[d];
    const float gr[4] = {row.x, row.y, row.z, row.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (nz<F>(d, e)) acc = fmaf(gr[e], in[4 * j + e], acc);
      out[4 * j + d] = acc;
    }
  }
}

// Forward passes over two digits a != b at once (16-element groups, local index
// 4 d_a + d_b): an optional signed permutation applied through the load addresses
// (CZ), then Ga on digit a, then Gb on digit b -- the operations of the separate
// one-digit passes, in the same order, with one shared-memory sweep and one
// barrier instead of two or three.  (Folding a following idle op's channels into
// the same pass saved a sweep on 5- and 6-qubit circuits but made the mixed
// 4096-circuit batch slower, 0.49-0.51 against 0.53 ms: three more pass variants
// in the instruction stream of every SM.)
template <class T, bool CZ, int FA, int FB>
__device__ void pass2(const T& t, float* r, int n, int a, const float* Ga, int b, const float* Gb) {
  const int groups = 1 << (2 * (n - 2));
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  const Off4 oa(1 << (2 * a)), ob(1 << (2 * b));
  for (int g = t.rank(); g < groups; g += T::kSize) {
    const int base = swz(group_base2(g, lo, hi));
    float x[16], y[16];
#pragma unroll
    for (int l = 0; l < 16; ++l) {
      const int src = CZ ? cz_inv(l) : l;
      const float v = r[base ^ oa[src >> 2] ^ ob[src & 3]];
      x[l] = (CZ && cz_ineg(l)) ? -v : v;
    }
    stage_a<FA>(Ga, x, y);
    stage_b<FB>(Gb, y, x);
#pragma unroll
    for (int l = 0; l < 16; ++l) r[base ^ oa[l >> 2] ^ ob[l & 3]] = x[l];
  }
}

template <class T>
__device__ void apply_sub(const T& t, float* r, int n, const SubOp& s, const float* tabs, float* user4,
                          const DmArgs& A, bool transpose) {
  switch (s.kind) {
    case 0: apply4<T, kTP>(t, r, n, s.q, tabs + 16 * s.table, false); break;   // never transposed
    case 1: apply_cz(t, r, n, s.q, s.b, transpose); break;
    case 2: apply4(t, r, n, s.q, user4, transpose); break;
    default: apply16(t, r, n, s.q, s.b, A.ptm2 + 256 * (size_t)s.table, transpose); break;
  }
}

// The circuit's PTM tables (forward and derivatives), by rank 0 (sc: sin and cos of
// theta_x, then of theta_y).  The products
// C R^x and C R^y are written out entry by entry (C, R^x, R^y are sparse), in
// FP64 and rounded once to FP32; the FP64 pipe is narrow, so the dense 4x4
// products would hold the team for several microseconds per circuit.
__device__ void build_tables(float* tabs, const double* prm, const double* sc) {
  const double tx = prm[0], ty = prm[1], p = prm[2], g = prm[3];
  const double f = 1.0 - 4.0 * p / 3.0, s = sqrt(1.0 - g);
  const double sf = s * f, hf = (1.0 - g) * f;   // C = [[1,0,0,0],[0,sf,0,0],[0,0,sf,0],[g,0,0,hf]]
  const double dsf_p = -4.0 * s / 3.0, dhf_p = -(1.0 - g) * 4.0 / 3.0;   // d/dp
  const double dsf_g = -f / (2.0 * s), dhf_g = -f;                       // d/dgamma (and d g/dgamma = 1)
  (void)tx;
  (void)ty;
  const double sx = sc[0], cx = sc[1], sy = sc[2], cy = sc[3];   // sincos(tx), sincos(ty)
  // row-major; row 0 is (m00, 0, 0, 0), column 0 below it (0, 0, m30)
  auto put = [&](int tb, double m00, double m11, double m12, double m13, double m21, double m22,
                 double m23, double m30, double m31, double m32, double m33) {
    float* o = tabs + 16 * tb;
    o[0] = (float)m00;
    o[1] = 0.f;
    o[2] = 0.f;
    o[3] = 0.f;
    o[4] = 0.f;
    o[5] = (float)m11;
    o[6] = (float)m12;
    o[7] = (float)m13;
    o[8] = 0.f;
    o[9] = (float)m21;
    o[10] = (float)m22;
    o[11] = (float)m23;
    o[12] = (float)m30;
    o[13] = (float)m31;
    o[14] = (float)m32;
    o[15] = (float)m33;
  };
  // R^x = [[1,0,0,0],[0,1,0,0],[0,0,cx,-sx],[0,0,sx,cx]], dR^x/dtx = [[0..],[0..],[0,0,-sx,-cx],[0,0,cx,-sx]]
  // C R^x: row 1 sf e1; row 2 sf (0,0,cx,-sx); row 3 (g, 0, hf sx, hf cx)
  put(TB_GX, 1, sf, 0, 0, 0, sf * cx, -sf * sx, g, 0, hf * sx, hf * cx);
  put(TB_GX_T, 0, 0, 0, 0, 0, -sf * sx, -sf * cx, 0, 0, hf * cx, -hf * sx);
  put(TB_GX_P, 0, dsf_p, 0, 0, 0, dsf_p * cx, -dsf_p * sx, 0, 0, dhf_p * sx, dhf_p * cx);
  put(TB_GX_G, 0, dsf_g, 0, 0, 0, dsf_g * cx, -dsf_g * sx, 1, 0, dhf_g * sx, dhf_g * cx);
  // R^y = [[1,0,0,0],[0,cy,0,sy],[0,0,1,0],[0,-sy,0,cy]]
  // C R^y: row 1 sf (0,cy,0,sy); row 2 sf e2; row 3 (g, -hf sy, 0, hf cy)
  put(TB_GY, 1, sf * cy, 0, sf * sy, 0, sf, 0, g, -hf * sy, 0, hf * cy);
  put(TB_GY_T, 0, -sf * sy, 0, sf * cy, 0, 0, 0, 0, -hf * cy, 0, -hf * sy);
  put(TB_GY_P, 0, dsf_p * cy, 0, dsf_p * sy, 0, dsf_p, 0, 0, -dhf_p * sy, 0, dhf_p * cy);
  put(TB_GY_G, 0, dsf_g * cy, 0, dsf_g * sy, 0, dsf_g, 0, 1, -dhf_g * sy, 0, dhf_g * cy);
  put(TB_C, 1, sf, 0, 0, 0, sf, 0, g, 0, 0, hf);
  put(TB_C_P, 0, dsf_p, 0, 0, 0, dsf_p, 0, 0, 0, 0, dhf_p);
  put(TB_C_G, 0, dsf_g, 0, 0, 0, dsf_g, 0, 1, 0, 0, dhf_g);
}

// index of the Pauli string Z_S (digit 3 at the bits of S)
__device__ __forceinline__ int zs_index(int S, int n) {
  int idx = 0;
  for (int b = 0; b < n; ++b)
    if ((S >> b) & 1) idx |= 3 << (2 * b);
  return idx;
}

template <class T>
__device__ void wht(const T& t, double* z, int N) {
  for (int h = 1; h < N; h <<= 1) {
    for (int i = t.rank(); i < N / 2; i += T::kSize) {
      const int j = ((i & ~(h - 1)) << 1) | (i & (h - 1));
      const double a = z[j], b = z[j + h];
      z[j] = a + b;
      z[j + h] = a - b;
    }
    t.sync();
  }
}

// One op forward with the fused two-digit passes: CZ as its permutation and both
// channels in one pass, the idle op as channel pairs -- the operations of its
// sub-ops in the same order, with the same arithmetic.  user4 holds the op's PTM
// for QS_DM_PTM1.  Ends with a team sync.
template <class T>
__device__ void apply_op_fused(const T& t, float* r, int n, const int32_t* op, const float* tabs,
                               const float* user4, const DmArgs& A) {
  const int code = op[0], a = op[1], b = op[2];
  const float* C = tabs + 16 * TB_C;
  if (code == QS_DM_X90 || code == QS_DM_Y90) {
    apply4<T, kTP>(t, r, n, a, tabs + 16 * (code == QS_DM_X90 ? TB_GX : TB_GY), false);
  } else if (code == QS_DM_CZ) {
    pass2<T, true, kChan, kChan>(t, r, n, a, C, b, C);
  } else if (code == QS_DM_IDLE) {
    for (int q = 0; q + 1 < n; q += 2) {
      pass2<T, false, kChan, kChan>(t, r, n, q, C, q + 1, C);
      t.sync();
    }
    if (n & 1) apply4<T, kChan>(t, r, n, n - 1, C, false);
  } else if (code == QS_DM_PTM1) {
    apply4(t, r, n, a, user4, false);
  } else {
    apply16(t, r, n, a, b, A.ptm2 + 256 * (size_t)op[3], false);
  }
  t.sync();
}

// Hand-out order.  Small circuits come last: a CTA that draws one switches for the
// rest of the launch to one circuit per warp (lane mode in the forward pass for 1
// and 2 qubits, warp mode in the gradient pass for up to kWarpMaxQ qubits).
// Forward: 5 and 6 qubits, then 3 and 4, then 1 and 2, each class in index order
// (a one-CTA stable partition; longest first within the classes ran slower, 0.55
// against 0.52 ms for 4096 mixed circuits: all long 6-qubit circuits then share
// the SMs at once).  Gradient: small (up to kWarpMaxQ qubits) after large, longest
// first within each (estimated cost (ops + 1) x (4^n + 64), the sweeps plus a
// per-op floor), sorted descending with a bitonic network in shared memory (keys:
// class bit 63, bit 62 set, cost as float bits in 32..61, circuit index; padding
// keys 0 sort last): the per-circuit time of the gradient (forward, backward sweep,
// scratch traffic) makes its tail long (8.63 -> 6.51 ms for 4096 circuits).  The
// sort takes up to kOrderMax circuits; larger gradient batches use the partition.
constexpr int kOrderMax = 16384;

__device__ __forceinline__ bool warp_sized(int q) { return q >= 1 && q <= kWarpMaxQ; }

// ---------------------------------------------------------------------------
// Lane mode (forward, registers of one or two qubits): a warp runs one circuit
// with the whole Pauli vector (4 or 16 floats) in registers, the same values in
// every lane (no shared state, no divergence, no barrier per op); the lanes only
// share the staging of the op stream (kWarpChunk ops per coalesced load into the
// warp's slice of shared memory).  Each warp draws its next circuit from the
// hand-out counter.  The arithmetic is that of the team sweeps: the same table
// entries (built in FP64, rounded once), the same FP32 fused multiply-adds in the
// same order per element, the probabilities and log-likelihood in FP64.
constexpr int kThreadMaxQ = 2;
__device__ __forceinline__ bool thread_sized(int q) { return q >= 1 && q <= kThreadMaxQ; }

// The nonzero entries of the three built-in tables (rows/columns I, x, y, z), from
// the same FP64 expressions as build_tables: C (channel), GX = C R^x, GY = C R^y.
struct ThreadTabs {
  float sf, hf, g;                       // C: m11 = m22 = sf, m30 = g, m33 = hf
  float x22, x23, x32, x33;              // GX: m11 = sf, m30 = g, and these
  float y11, y13, y31, y33;              // GY: m22 = sf, m30 = g, and these
};
__device__ ThreadTabs thread_tabs(const double* prm) {
  const double tx = prm[0], ty = prm[1], p = prm[2], g = prm[3];
  const double f = 1.0 - 4.0 * p / 3.0, s = sqrt(1.0 - g);
  const double sf = s * f, hf = (1.0 - g) * f;
  double cx, sx, cy, sy;
  sincos(tx, &sx, &cx);
  sincos(ty, &sy, &cy);
  ThreadTabs T;
  T.sf = (float)sf;
  T.hf = (float)hf;
  T.g = (float)g;
  T.x22 = (float)(sf * cx);
  T.x23 = (float)(-sf * sx);
  T.x32 = (float)(hf * sx);
  T.x33 = (float)(hf * cx);
  T.y11 = (float)(sf * cy);
  T.y13 = (float)(sf * sy);
  T.y31 = (float)(-hf * sy);
  T.y33 = (float)(hf * cy);
  return T;
}

// Built-in table K (0 GX, 1 GY, 2 C) on the four values v of one digit, in place:
// each output the FMA chain over its nonzero inputs in index order (the skipped
// terms are exact zeros of the dense sum).
template <int K>
__device__ __forceinline__ void tab4(const ThreadTabs& T, float& v0, float& v1, float& v2, float& v3) {
  const float x0 = v0, x1 = v1, x2 = v2, x3 = v3;
  v0 = fmaf(1.0f, x0, 0.f);
  if (K == 0) {        // GX rows: (1,0,0,0) (0,sf,0,0) (0,0,x22,x23) (g,0,x32,x33)
    v1 = fmaf(T.sf, x1, 0.f);
    v2 = fmaf(T.x23, x3, fmaf(T.x22, x2, 0.f));
    v3 = fmaf(T.x33, x3, fmaf(T.x32, x2, fmaf(T.g, x0, 0.f)));
  } else if (K == 1) { // GY rows: (1,0,0,0) (0,y11,0,y13) (0,0,sf,0) (g,y31,0,y33)
    v1 = fmaf(T.y13, x3, fmaf(T.y11, x1, 0.f));
    v2 = fmaf(T.sf, x2, 0.f);
    v3 = fmaf(T.y33, x3, fmaf(T.y31, x1, fmaf(T.g, x0, 0.f)));
  } else {             // C rows: (1,0,0,0) (0,sf,0,0) (0,0,sf,0) (g,0,0,hf)
    v1 = fmaf(T.sf, x1, 0.f);
    v2 = fmaf(T.sf, x2, 0.f);
    v3 = fmaf(T.hf, x3, fmaf(T.g, x0, 0.f));
  }
}
// A dense user table (FP64 in global memory, rounded to FP32 per entry) on v.
__device__ __forceinline__ void user4(const double* G, float& v0, float& v1, float& v2, float& v3) {
  const float x[4] = {v0, v1, v2, v3};
  float y[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    float acc = 0.f;
#pragma unroll
    for (int e = 0; e < 4; ++e) acc = fmaf((float)G[4 * d + e], x[e], acc);
    y[d] = acc;
  }
  v0 = y[0];
  v1 = y[1];
  v2 = y[2];
  v3 = y[3];
}

// One-digit op on qubit q of an NQ-qubit register x (index sum_q d_q 4^q): K as in
// tab4, K = 3 a user table.
template <int NQ, int K>
__device__ __forceinline__ void thread_digit(float* x, int q, const ThreadTabs& T, const double* U) {
  auto one = [&](float& a, float& b, float& c, float& d) {
    if (K == 3)
      user4(U, a, b, c, d);
    else
      tab4<K>(T, a, b, c, d);
  };
  if (NQ == 1) {
    one(x[0], x[1], x[2], x[3]);
  } else if (q == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) one(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) one(x[j], x[4 + j], x[8 + j], x[12 + j]);
  }
}

// Two-qubit ops of a two-qubit register (local index 4 d_a + d_b; A1 = (a == 1):
// local index l sits at register l, else at its digit transpose).
template <bool A1>
__device__ __forceinline__ int loc(int l) { return A1 ? l : ((l & 3) << 2) | (l >> 2); }
template <bool A1>
__device__ __forceinline__ void thread_cz(float* x) {
  float y[16];
#pragma unroll
  for (int l = 0; l < 16; ++l) {
    const float v = x[loc<A1>(cz_inv(l))];
    y[loc<A1>(l)] = cz_ineg(l) ? -v : v;
  }
#pragma unroll
  for (int l = 0; l < 16; ++l) x[l] = y[l];
}
template <bool A1>
__device__ __forceinline__ void thread_ptm2(float* x, const double* G) {
  float in[16], y[16];
#pragma unroll
  for (int l = 0; l < 16; ++l) in[l] = x[loc<A1>(l)];
  for (int d = 0; d < 16; ++d) {
    float acc = 0.f;
#pragma unroll
    for (int e = 0; e < 16; ++e) acc = fmaf((float)G[d * 16 + e], in[e], acc);
    y[d] = acc;
  }
#pragma unroll
  for (int l = 0; l < 16; ++l) x[loc<A1>(l)] = y[l];
}

// Circuit c (n = NQ) on this warp (s_ops: the warp's kWarpChunk staged ops);
// invalid circuits get NaN outputs.
template <int NQ>
__device__ void lane_circuit(const DmArgs& A, int c, int lane, int4* s_ops) {
  constexpr int N = 1 << NQ, Dn = 1 << (2 * NQ);
  const int64_t o0 = A.op_off[c];
  const int L = (int)(A.op_off[c + 1] - o0);
  const int64_t out0 = A.out_off[c];
  bool ok = NQ <= A.max_q && L >= 0 && L <= A.max_ops && A.out_off[c + 1] - out0 == N;
  float x[Dn];
  const float amp0 = 1.0f / sqrtf((float)N);
#pragma unroll
  for (int i = 0; i < Dn; ++i) {
    bool iz = true;
#pragma unroll
    for (int b = 0; b < NQ; ++b) {
      const int d = (i >> (2 * b)) & 3;
      iz = iz && (d == 0 || d == 3);
    }
    x[i] = iz ? amp0 : 0.f;
  }
  const ThreadTabs T = thread_tabs(A.params + 4 * c);
  const int4* ops = reinterpret_cast<const int4*>(A.ops + 4 * o0);
  for (int k = 0; ok && k < L; ++k) {
    if ((k % kWarpChunk) == 0) {
      __syncwarp();
      for (int u = lane; u < kWarpChunk && k + u < L; u += 32) s_ops[u] = ops[k + u];
      __syncwarp();
    }
    const int4 op = s_ops[k % kWarpChunk];
    ok = op_valid(reinterpret_cast<const int32_t*>(&op), NQ, A);
    if (!ok) break;
    switch (op.x) {
      case QS_DM_X90: thread_digit<NQ, 0>(x, op.y, T, nullptr); break;
      case QS_DM_Y90: thread_digit<NQ, 1>(x, op.y, T, nullptr); break;
      case QS_DM_PTM1: thread_digit<NQ, 3>(x, op.y, T, A.ptm1 + 16 * (size_t)op.w); break;
      case QS_DM_IDLE:
        thread_digit<NQ, 2>(x, 0, T, nullptr);
        if (NQ == 2) thread_digit<NQ, 2>(x, 1, T, nullptr);
        break;
      default:   // CZ or a user two-qubit PTM (NQ == 2: validated)
        if (NQ == 2) {
          if (op.x == QS_DM_CZ) {
            if (op.y == 1) thread_cz<true>(x); else thread_cz<false>(x);
            thread_digit<NQ, 2>(x, op.y, T, nullptr);
            thread_digit<NQ, 2>(x, op.z, T, nullptr);
          } else {
            const double* G = A.ptm2 + 256 * (size_t)op.w;
            if (op.y == 1) thread_ptm2<true>(x, G); else thread_ptm2<false>(x, G);
          }
        }
    }
  }
  __syncwarp();   // the staged ops are read before the next circuit restages them
  if (!ok) {
    if (A.loglik && lane == 0) A.loglik[c] = __longlong_as_double(0x7ff8000000000000ll);
    if (A.probs && lane < N && A.out_off[c + 1] - out0 == N) A.probs[out0 + lane] = __int_as_float(0x7fc00000);
    return;
  }
  // probabilities: p = 2^{-n/2} WHT(r on {I,Z}^n), the butterflies of wht()
  double z[N];
#pragma unroll
  for (int S = 0; S < N; ++S) {
    int idx = 0;
#pragma unroll
    for (int b = 0; b < NQ; ++b)
      if ((S >> b) & 1) idx |= 3 << (2 * b);
    z[S] = (double)x[idx];
  }
#pragma unroll
  for (int h = 1; h < N; h <<= 1)
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const int j = ((i & ~(h - 1)) << 1) | (i & (h - 1));
      const double a = z[j], b = z[j + h];
      z[j] = a + b;
      z[j + h] = a - b;
    }
  const double scale = 1.0 / sqrt((double)N);
  double ll = 0.0;
#pragma unroll
  for (int J = 0; J < N; ++J) {
    double p = z[J] * scale;
    if (A.probs && lane == J) A.probs[out0 + J] = (float)p;
    if (A.counts) {
      const int cnt = A.counts[out0 + J];
      if (!(p > 0.0)) p = 1e-300;
      if (cnt > 0) ll += (double)cnt * log(p);
    }
  }
  if (A.counts && A.loglik && lane == 0) A.loglik[c] = ll;
}

// Every warp of the CTA runs small circuits on its own; warp 0 starts with c.
// s_ops: 4 x kWarpChunk staged ops.
__device__ void dm_lanes(const DmArgs& A, int c, int4* s_ops) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto draw = [&]() {
    int v = 0;
    if (lane == 0) v = atomicAdd(A.work, 1);
    v = __shfl_sync(0xffffffffu, v, 0);
    return v < A.n_circuits ? A.order[v] : A.n_circuits;
  };
  if (w != 0) c = draw();
  while (c < A.n_circuits) {
    if (A.nq[c] == 1)
      lane_circuit<1>(A, c, lane, s_ops + w * kWarpChunk);
    else
      lane_circuit<2>(A, c, lane, s_ops + w * kWarpChunk);
    c = draw();
  }
}


// class of a circuit in the forward hand-out order: 0 team (5, 6 qubits or
// invalid), 1 team (3, 4 qubits), 2 lane mode (1, 2 qubits)
__device__ __forceinline__ int fwd_class(int q) { return thread_sized(q) ? 2 : (warp_sized(q) ? 1 : 0); }

__global__ void __launch_bounds__(1024) dm_partition_kernel(const int32_t* __restrict__ nq, int n,
                                                            int* __restrict__ order) {
  __shared__ int cnt0[1024], cnt1[1024];
  const int per = (n + 1023) / 1024;
  const int lo = min(n, threadIdx.x * per), hi = min(n, lo + per);
  int c0 = 0, c1 = 0;
  for (int i = lo; i < hi; ++i) {
    const int k = fwd_class(nq[i]);
    c0 += k == 0;
    c1 += k == 1;
  }
  cnt0[threadIdx.x] = c0;
  cnt1[threadIdx.x] = c1;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {   // inclusive scans (Hillis-Steele)
    const int v0 = threadIdx.x >= o ? cnt0[threadIdx.x - o] : 0;
    const int v1 = threadIdx.x >= o ? cnt1[threadIdx.x - o] : 0;
    __syncthreads();
    cnt0[threadIdx.x] += v0;
    cnt1[threadIdx.x] += v1;
    __syncthreads();
  }
  const int n0 = cnt0[1023], n1 = cnt1[1023];
  int p0 = cnt0[threadIdx.x] - c0, p1 = cnt1[threadIdx.x] - c1;   // before this chunk
  int p2 = n0 + n1 + (lo - p0 - p1);
  p1 += n0;
  for (int i = lo; i < hi; ++i) {
    const int k = fwd_class(nq[i]);
    order[k == 0 ? p0++ : (k == 1 ? p1++ : p2++)] = i;
  }
}

__global__ void __launch_bounds__(1024) dm_order_kernel(const int32_t* __restrict__ nq,
                                                        const int64_t* __restrict__ op_off, int n,
                                                        int* __restrict__ order) {
  extern __shared__ unsigned long long keys[];
  int P = 1;
  while (P < n) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    unsigned long long k = 0;
    if (i < n) {
      const int q0 = nq[i];
      const int q = q0 < 1 ? 1 : (q0 > kDmMaxQ ? kDmMaxQ : q0);
      long long L = op_off[i + 1] - op_off[i];
      L = L < 0 ? 0 : (L > (1 << 20) ? (1 << 20) : L);
      const float cost = (float)(L + 1) * (float)((1 << (2 * q)) + 64);   // < 2^30 as float bits
      k = ((unsigned long long)(warp_sized(q0) ? 0 : 1) << 63) | (1ull << 62) |
          ((unsigned long long)__float_as_uint(cost) << 32) | (unsigned)i;
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
// (and, with the gradient, lambda and a scratch vector); in warp mode the space
// from r on holds four per-warp regions (tables, user PTM, WHT buffer, r[, lam,
// tmp], staged ops)
constexpr int kDmHead = 16 * TB_COUNT + 16 + 128;   // floats before r (16-byte aligned)
constexpr int kWarpHead = 16 * TB_COUNT + 16 + 32;  // tables, user PTM, 16 doubles
constexpr int kWarpRegionFwd = kWarpHead + kWarpD + 4 * kWarpChunk;
constexpr int kWarpRegionGrad = kWarpHead + 3 * kWarpD + 4 * kWarpChunk;
static_assert(kDmHead % 4 == 0 && kWarpHead % 4 == 0 && kWarpRegionFwd % 4 == 0 && kWarpRegionGrad % 4 == 0,
              "16-byte aligned regions");

// One validated circuit c on team t (tables built).  stride: floats between the
// stored states in scratch.
template <bool GRAD, class T>
__device__ __forceinline__ void dm_circuit(const T& t, const DmArgs& A, int c, int n, int L, const int32_t* ops,
                                           int64_t out0, int stride, float* tabs, float* user4, double* z,
                                           float* r, float* lam, float* tmp, int4* s_ops, float* ckpt,
                                           float* segbuf, float* subst) {
  constexpr int kC = T::kChunk;
  const int N = 1 << n;
  const int Dn = 1 << (2 * n);
  const int tid = t.rank();
  const float amp0 = 1.0f / sqrtf((float)N);
  // rho_0 = |0..0><0..0|: r_i = 2^{-n/2} on {I,Z}^n, 0 elsewhere
  for (int i = tid; i < Dn; i += T::kSize) {
    bool iz = true;
    for (int b = 0; b < n; ++b) {
      const int d = (i >> (2 * b)) & 3;
      iz = iz && (d == 0 || d == 3);
    }
    r[swz(i)] = iz ? amp0 : 0.f;
  }
  t.sync();
  // ---------------- forward
  const int4* ops4 = reinterpret_cast<const int4*>(ops);
  if constexpr (!GRAD) {
    for (int k = 0; k < L;) {
      if ((k % kC) == 0) {   // stage the next chunk of ops (one coalesced read)
        t.sync();
        for (int u = tid; u < kC && k + u < L; u += T::kSize) s_ops[u] = ops4[k + u];
        t.sync();
      }
      const int32_t* op = reinterpret_cast<const int32_t*>(&s_ops[k % kC]);
      const int code = op[0], a = op[1];
      const int32_t* nx = reinterpret_cast<const int32_t*>(&s_ops[(k + 1) % kC]);
      if ((code == QS_DM_X90 || code == QS_DM_Y90) && k + 1 < L && (k + 1) % kC != 0 &&
          (nx[0] == QS_DM_X90 || nx[0] == QS_DM_Y90) && nx[1] != a) {
        // this op and the next act on different qubits: one two-digit pass
        pass2<T, false, kTP, kTP>(t, r, n, a, tabs + 16 * (code == QS_DM_X90 ? TB_GX : TB_GY), nx[1],
                                  tabs + 16 * (nx[0] == QS_DM_X90 ? TB_GX : TB_GY));
        t.sync();
        k += 2;
        continue;
      }
      if (code == QS_DM_PTM1) {
        if (tid < 16) user4[tid] = (float)A.ptm1[16 * (size_t)op[3] + tid];
        t.sync();
      }
      apply_op_fused(t, r, n, op, tabs, user4, A);
      ++k;
    }
  }
  for (int k = 0; GRAD && k < L; ++k) {
    if ((k % kC) == 0) {   // stage the next chunk of ops (one coalesced read)
      t.sync();
      for (int u = tid; u < kC && k + u < L; u += T::kSize) s_ops[u] = ops4[k + u];
      t.sync();
    }
    if ((k % A.K) == 0) {
      float* dst = ckpt + (size_t)(k / A.K) * stride;
      for (int i = tid; i < Dn; i += T::kSize) dst[i] = r[i];
      t.sync();   // copies done before r is updated in place
    }
    const int32_t* op = reinterpret_cast<const int32_t*>(&s_ops[k % kC]);
    if (op[0] == QS_DM_PTM1) {
      if (tid < 16) user4[tid] = (float)A.ptm1[16 * (size_t)op[3] + tid];
      t.sync();
    }
    apply_op_fused(t, r, n, op, tabs, user4, A);
  }
  // ---------------- probabilities: p = 2^{-n/2} WHT(r on {I,Z}^n)
  for (int S = tid; S < N; S += T::kSize) z[S] = (double)r[swz(zs_index(S, n))];
  t.sync();
  wht(t, z, N);
  const double scale = 1.0 / sqrt((double)N);
  double ll = 0.0;
  for (int J = tid; J < N; J += T::kSize) {
    double p = z[J] * scale;
    if (A.probs) A.probs[out0 + J] = (float)p;
    if (A.counts) {
      const int cnt = A.counts[out0 + J];
      if (!(p > 0.0)) p = 1e-300;
      if (cnt > 0) ll += (double)cnt * log(p);
      if constexpr (GRAD) z[J] = cnt > 0 ? (double)cnt / p : 0.0;   // seed weights dl/dp_J
    }
  }
  if (A.counts) {
    const double tot = t.sum(ll);
    if (tid == 0 && A.loglik) A.loglik[c] = tot;
  }
  if constexpr (!GRAD) return;
  // ---------------- adjoint
  t.sync();
  wht(t, z, N);
  // lambda is linear in the seed: keep it in fp32 as lambda / lmax (no
  // overflow when some n_J / p_J is huge) and scale the fp64 sums back
  double lmax = 0.0;
  for (int S = 0; S < N; ++S) lmax = fmax(lmax, fabs(z[S]));
  const double lscale = lmax > 0.0 ? scale / lmax : 0.0;
  for (int i = tid; i < Dn; i += T::kSize) lam[i] = 0.f;
  t.sync();
  for (int S = tid; S < N; S += T::kSize) lam[swz(zs_index(S, n))] = (float)(z[S] * lscale);
  t.sync();
  double g[4] = {0, 0, 0, 0};
  const int nseg = (L + A.K - 1) / A.K;
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
    const int k0 = sgi * A.K, k1 = min(L, k0 + A.K);
    // recompute the states before each op of the segment
    const float* ck = ckpt + (size_t)sgi * stride;
    for (int i = tid; i < Dn; i += T::kSize) r[i] = ck[i];
    t.sync();
    for (int k = k0; k < k1; ++k) {
      float* dst = segbuf + (size_t)(k - k0) * stride;
      for (int i = tid; i < Dn; i += T::kSize) dst[i] = r[i];
      if (k + 1 == k1) break;
      const int32_t* op = ops + 4 * k;
      if (op[0] == QS_DM_PTM1) {
        t.sync();
        if (tid < 16) user4[tid] = (float)A.ptm1[16 * (size_t)op[3] + tid];
        t.sync();
      }
      t.sync();
      apply_op_fused(t, r, n, op, tabs, user4, A);
    }
    t.sync();
    for (int k = k1 - 1; k >= k0; --k) {
      const int32_t* op = ops + 4 * k;
      if (op[0] == QS_DM_PTM1) {
        if (tid < 16) user4[tid] = (float)A.ptm1[16 * (size_t)op[3] + tid];
      }
      const int ns = op_nsub(op, n);
      const float* before = segbuf + (size_t)(k - k0) * stride;
      t.sync();
      // the states before the sub-ops, once: s_0 = before, s_{j+1} = sub_j s_j;
      // the last stays in tmp, the earlier ones with parameters go to subst
      if (ns > 1) {
        for (int i = tid; i < Dn; i += T::kSize) tmp[i] = before[i];
        t.sync();
        for (int j = 0; j + 1 < ns; ++j) {
          apply_sub(t, tmp, n, op_subop(op, j), tabs, user4, A, false);
          t.sync();
          if (j + 2 < ns && op_subop(op, j + 1).kind == 0) {
            for (int i = tid; i < Dn; i += T::kSize) subst[(size_t)(j + 1) * stride + i] = tmp[i];
            t.sync();   // copied before sub-op j + 1 rewrites tmp
          }
        }
      }
      for (int j = ns - 1; j >= 0; --j) {
        const SubOp sj = op_subop(op, j);
        if (sj.kind == 0) {
          const float* sv =
              j + 1 == ns ? (ns > 1 ? tmp : before) : (j == 0 ? before : subst + (size_t)j * stride);
          adj4(t, lam, sv, n, sj.q, tabs + 16 * sj.table, tabs, sj.dtab, g);
        } else {
          apply_sub(t, lam, n, sj, tabs, user4, A, true);
        }
        t.sync();
      }
    }
  }
  for (int pidx = 0; pidx < 4; ++pidx) {
    const double tot = t.sum(g[pidx]);
    if (tid == 0) A.grad[4 * c + pidx] = tot * lmax;
  }
}

// Circuit c on team t: device-side validation (the arrays are caller-supplied
// device memory; ops checked by the team in parallel), tables, then the circuit;
// an invalid circuit gets NaN outputs.  Ends with a team sync.
template <bool GRAD, class T>
__device__ void run_circuit(const T& t, const DmArgs& A, int c, int stride, float* tabs, float* user4, double* z,
                            float* r, float* lam, float* tmp, int4* s_ops, float* ckpt, float* segbuf,
                            float* subst) {
  const int tid = t.rank();
  const int n = A.nq[c];
  const int64_t o0 = A.op_off[c];
  const int L = (int)(A.op_off[c + 1] - o0);
  const int32_t* ops = A.ops + 4 * o0;
  const int64_t out0 = A.out_off[c];
  const int N = 1 << n;
  bool ok = n >= 1 && n <= A.max_q && L >= 0 && L <= A.max_ops && A.out_off[c + 1] - out0 == N;
  if (ok)
    for (int k = tid; k < L; k += T::kSize) ok = ok && op_valid(ops + 4 * k, n, A);
  const bool all_ok = t.all(ok);
  if (all_ok && tid < 2) {   // the two angles' sincos side by side (lanes 0 and 1), into z
    double sn, cs;
    sincos(A.params[4 * c + tid], &sn, &cs);
    z[2 * tid] = sn;
    z[2 * tid + 1] = cs;
  }
  t.sync();
  if (all_ok && tid == 0) build_tables(tabs, A.params + 4 * c, z);
  t.sync();
  if (!all_ok) {
    const float nanf_ = __int_as_float(0x7fc00000);
    if (tid == 0) {
      if (A.loglik) A.loglik[c] = __longlong_as_double(0x7ff8000000000000ll);
      if (A.grad)
        for (int k = 0; k < 4; ++k) A.grad[4 * c + k] = __longlong_as_double(0x7ff8000000000000ll);
    }
    if (A.probs && n >= 1 && n <= kDmMaxQ && A.out_off[c + 1] - out0 == N)
      for (int J = tid; J < N; J += T::kSize) A.probs[out0 + J] = nanf_;
  } else {
    dm_circuit<GRAD>(t, A, c, n, L, ops, out0, stride, tabs, user4, z, r, lam, tmp, s_ops, ckpt, segbuf, subst);
  }
  t.sync();
}

// Warp mode: every warp of the CTA runs small circuits on its own, drawing the
// next one from the hand-out counter; warp 0 starts with c (drawn by the CTA).
template <bool GRAD>
__device__ void dm_warps(const DmArgs& A, int c, float* base, float* scratch) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpTeam t{lane};
  float* reg = base + (size_t)w * (GRAD ? kWarpRegionGrad : kWarpRegionFwd);
  float* tabs = reg;
  float* user4 = reg + 16 * TB_COUNT;
  double* z = reinterpret_cast<double*>(user4 + 16);
  float* r = reg + kWarpHead;
  float* lam = r + kWarpD;
  float* tmp = r + 2 * kWarpD;
  int4* s_ops = reinterpret_cast<int4*>(r + (GRAD ? 3 : 1) * kWarpD);
  const size_t per = (size_t)(A.nseg + A.K + kDmMaxQ) * kWarpD;
  float* ckpt = scratch ? scratch + (size_t)w * per : nullptr;
  float* segbuf = ckpt ? ckpt + (size_t)A.nseg * kWarpD : nullptr;
  float* subst = ckpt ? ckpt + (size_t)(A.nseg + A.K) * kWarpD : nullptr;
  auto draw = [&]() {
    int v = 0;
    if (lane == 0) v = atomicAdd(A.work, 1);
    v = __shfl_sync(0xffffffffu, v, 0);
    return v < A.n_circuits ? A.order[v] : A.n_circuits;
  };
  if (w != 0) c = draw();
  while (c < A.n_circuits) {
    run_circuit<GRAD>(t, A, c, kWarpD, tabs, user4, z, r, lam, tmp, s_ops, ckpt, segbuf, subst);
    c = draw();
  }
}

// GRAD: the gradient kernel (forward with checkpoints, then the adjoint sweep);
// otherwise probabilities / log-likelihood only, with one-qubit gate pairs fused
// too and a third of the shared memory (more CTAs per SM).  A CTA draws circuits
// from the hand-out order; with an order, the first small one (all later ones are
// small too) switches it to warp mode (gradient, up to kWarpMaxQ qubits) or lane
// mode (forward, up to kThreadMaxQ qubits).
template <bool GRAD>
__global__ void __launch_bounds__(kDmThreads, GRAD ? 4 : 6) dm_batch_kernel(DmArgs A) {
  extern __shared__ __align__(16) float dsm[];
  const int D = 1 << (2 * A.max_q);
  const int Dscr = D > 4 * kWarpD ? D : 4 * kWarpD;   // scratch floats per stored state and CTA
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
      A.scratch ? A.scratch + (size_t)blockIdx.x * (size_t)(A.nseg + A.K + kDmMaxQ) * Dscr : nullptr;
  float* ckpt = my_scratch;
  float* segbuf = my_scratch ? my_scratch + (size_t)A.nseg * D : nullptr;
  float* subst = my_scratch ? my_scratch + (size_t)(A.nseg + A.K) * D : nullptr;
  const CtaTeam t{red};
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
    if (GRAD && A.order && warp_sized(A.nq[c])) {
      dm_warps<GRAD>(A, c, r, my_scratch);
      return;
    }
    if (!GRAD && A.order && thread_sized(A.nq[c])) {
      dm_lanes(A, c, reinterpret_cast<int4*>(r));
      return;
    }
    run_circuit<GRAD>(t, A, c, D, tabs, user4, z, r, lam, tmp, s_ops, ckpt, segbuf, subst);
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
  return abi_guard(__func__, [&]() -> qs_status {
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

    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int D = 1 << (2 * A.max_q);
    const bool with_grad = grad != nullptr;
    const int warp_need = 4 * (with_grad ? kWarpRegionGrad : kWarpRegionFwd);
    const int cta_need = (with_grad ? 3 : 1) * D;
    const size_t smem = (size_t)(kDmHead + (cta_need > warp_need ? cta_need : warp_need)) * sizeof(float);
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

    const size_t Dscr = (size_t)(D > 4 * kWarpD ? D : 4 * kWarpD);
    const size_t scratch_floats = grad ? (size_t)grid * (A.nseg + A.K + kDmMaxQ) * Dscr : 0;
    // hand-out order: the gradient sorted (up to kOrderMax circuits), otherwise the
    // stable partition large | small
    const bool sort = grad && A.n_circuits > 1 && A.n_circuits <= kOrderMax;
    const bool part = !sort && A.n_circuits > 1;
    const size_t order_bytes =
        (sort || part) ? ((sizeof(int) * (size_t)A.n_circuits + 255) & ~size_t(255)) : 0;
    const size_t bytes = 256 + order_bytes + scratch_floats * sizeof(float);
    void* mem = nullptr;
    cudaError_t e = cudaMallocAsync(&mem, bytes, stream);
    if (e != cudaSuccess) return cuda_status(e, "cudaMallocAsync (dm scratch)");
    A.work = (int*)mem;
    A.order = (sort || part) ? (const int*)((char*)mem + 256) : nullptr;
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
    } else if (part) {
      dm_partition_kernel<<<1, 1024, 0, stream>>>(A.nq, A.n_circuits, (int*)A.order);
    }
    kern<<<grid, kDmThreads, smem, stream>>>(A);
    e = cudaGetLastError();
    cudaFreeAsync(mem, stream);
    if (e != cudaSuccess) return cuda_status(e, "dm_batch_kernel launch");
    return QS_OK;
  });
}
