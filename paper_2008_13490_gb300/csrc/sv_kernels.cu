// State-vector kernels for sm_103a.
//
//  tile_pass_kernel   one HBM read+write of the state applies every op of a
//                     pass: a CTA owns a tile of 2^12 amplitudes (12 qubits,
//                     any bit positions that include bits 0,1), lanes hold the 5
//                     lowest tile bits (gates there use warp shuffles), each
//                     thread holds 16 amplitudes in registers (4 tile bits),
//                     and shared memory transposes swap register and warp bits
//                     between stages.
//  plain_*_kernel     one launch per gate, the pair/quad update of the thesis's
//                     four-component loops (Eq. (psioft4componentupdates)) with
//                     the bit-insert index of its reduced loop, 64-bit indices.
//  small_state_kernel whole state in one CTA's shared memory (n < 12).
//  remap_kernel       permutes bit positions inside a 12-bit tile (in place).
//  probs / marginal / loglik / reduce: Born rule p_J = |a_J|^2 with fp64
//                     accumulation of the sums.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "internal.h"
#include "tile_cp.h"

namespace qs {

// ------------------------------------------------------------------ tile pass

template <int J, typename R>
__device__ __forceinline__ void reg_gate(C2<R>* v, const C2<R>* m) {
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    if (r & (1 << J)) continue;
    const C2<R> a = v[r], b = v[r | (1 << J)];
    v[r] = cfma2(m[0], a, m[1], b);
    v[r | (1 << J)] = cfma2(m[2], a, m[3], b);
  }
}

template <int J, int K, typename R>
__device__ __forceinline__ void reg_gate_choice(C2<R>* v, const C2<R>* m0, const C2<R>* m1) {
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    if (r & (1 << J)) continue;
    const C2<R>* m = ((r >> K) & 1) ? m1 : m0;
    const C2<R> a = v[r], b = v[r | (1 << J)];
    v[r] = cfma2(m[0], a, m[1], b);
    v[r | (1 << J)] = cfma2(m[2], a, m[3], b);
  }
}

template <int K, typename R>
__device__ __forceinline__ void lane_gate_choice(C2<R>* v, int mask, C2<R> o0, C2<R> p0, C2<R> o1,
                                                 C2<R> p1) {
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const C2<R> q = shfl_xor_c(v[r], mask);
    if ((r >> K) & 1) v[r] = cfma2(o1, v[r], p1, q);
    else v[r] = cfma2(o0, v[r], p0, q);
  }
}

// ---- dense 4x4 ops on two qubits a (local index msb) and b: y = G x on each quad

template <typename R>
__device__ __forceinline__ C2<R> sel4(int o, C2<R> g0, C2<R> g1, C2<R> g2, C2<R> g3) {
  return csel(o >= 2, csel(o == 3, g3, g2), csel(o == 1, g1, g0));
}

// both qubits in register slots KA, KB: the quad of each r is in registers
template <int KA, int KB, typename R>
__device__ __forceinline__ void reg_g2(C2<R>* v, const C2<R>* g) {
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    if ((r >> KA) & 1 || (r >> KB) & 1) continue;
    C2<R> x[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) x[l] = v[r | ((l >> 1) << KA) | ((l & 1) << KB)];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const C2<R> y0 = cfma2(g[4 * o], x[0], g[4 * o + 1], x[1]);
      const C2<R> y1 = cfma2(g[4 * o + 2], x[2], g[4 * o + 3], x[3]);
      v[r | ((o >> 1) << KA) | ((o & 1) << KB)] = C2<R>{y0.x + y1.x, y0.y + y1.y};
    }
  }
}

// one qubit on lane bit (mask), the other in register slot K; A_LANE: qubit a is
// the lane one.  Each lane holds two of a quad's amplitudes (register bit 0, 1),
// its partner lane the other two.
template <int K, bool A_LANE, typename R>
__device__ __forceinline__ void lane_reg_g2(C2<R>* v, const C2<R>* g, int mask, int u) {
  // quad index of (lane value w, register value c)
  auto q = [](int w, int c) { return A_LANE ? 2 * w + c : 2 * c + w; };
  C2<R> co[2][4];   // output c: coefficients of own c'=0, own 1, partner 0, partner 1
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cc = j & 1, partner = j >> 1;
      // lane value of the input: own u or partner 1 - u; output at q(u, c)
      const C2<R> at0 = g[4 * q(0, c) + q(partner ? 1 : 0, cc)];   // u = 0
      const C2<R> at1 = g[4 * q(1, c) + q(partner ? 0 : 1, cc)];   // u = 1
      co[c][j] = csel(u != 0, at1, at0);
    }
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    if ((r >> K) & 1) continue;
    const C2<R> e0 = v[r], e1 = v[r | (1 << K)];
    const C2<R> p0 = shfl_xor_c(e0, mask), p1 = shfl_xor_c(e1, mask);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const C2<R> y0 = cfma2(co[c][0], e0, co[c][1], e1);
      const C2<R> y1 = cfma2(co[c][2], p0, co[c][3], p1);
      v[r | (c << K)] = C2<R>{y0.x + y1.x, y0.y + y1.y};
    }
  }
}

// both qubits on lane bits: each lane holds one amplitude of every quad
template <typename R>
__device__ __forceinline__ void lane_lane_g2(C2<R>* v, const C2<R>* g, int ma, int mb, int o) {
  // o = own quad index 2 ua + ub; the amplitude at quad index o ^ f comes from lane ^ mask(f)
  const C2<R> c0 = sel4(o, g[0], g[5], g[10], g[15]);                    // f = 0: G[o][o]
  const C2<R> c1 = sel4(o, g[1], g[4], g[11], g[14]);                    // f = 1: G[o][o ^ 1]
  const C2<R> c2 = sel4(o, g[2], g[7], g[8], g[13]);                     // f = 2: G[o][o ^ 2]
  const C2<R> c3 = sel4(o, g[3], g[6], g[9], g[12]);                     // f = 3: G[o][o ^ 3]
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const C2<R> x = v[r];
    const C2<R> xb = shfl_xor_c(x, mb), xa = shfl_xor_c(x, ma), xab = shfl_xor_c(x, ma | mb);
    const C2<R> y0 = cfma2(c0, x, c1, xb);
    const C2<R> y1 = cfma2(c2, xa, c3, xab);
    v[r] = C2<R>{y0.x + y1.x, y0.y + y1.y};
  }
}

template <typename R>
__device__ __forceinline__ void apply_g2(C2<R>* v, const TileOp<R>* __restrict__ opp, int lane) {
  C2<R> g[16];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    g[i] = opp[0].m0[i];
    g[4 + i] = opp[0].m1[i];
    g[8 + i] = opp[1].m0[i];
    g[12 + i] = opp[1].m1[i];
  }
  const uint8_t sa = opp->csrc, ba = opp->cbit, sb = opp->dsrc, bb = opp->dbit;
  // the host orders the qubits: register slots ascending, a lane qubit first
  if (sa == CS_REG && sb == CS_REG) {
    switch (ba * 4 + bb) {
      case 1: reg_g2<0, 1>(v, g); break;
      case 2: reg_g2<0, 2>(v, g); break;
      case 3: reg_g2<0, 3>(v, g); break;
      case 6: reg_g2<1, 2>(v, g); break;
      case 7: reg_g2<1, 3>(v, g); break;
      default: reg_g2<2, 3>(v, g); break;
    }
    return;
  }
  if (sb == CS_LANE) {
    lane_lane_g2(v, g, 1 << ba, 1 << bb, 2 * ((lane >> ba) & 1) + ((lane >> bb) & 1));
    return;
  }
  const int mask = 1 << ba, u = (lane >> ba) & 1;   // a on the lane, b in register slot bb
  switch (bb) {
    case 0: lane_reg_g2<0, true>(v, g, mask, u); break;
    case 1: lane_reg_g2<1, true>(v, g, mask, u); break;
    case 2: lane_reg_g2<2, true>(v, g, mask, u); break;
    default: lane_reg_g2<3, true>(v, g, mask, u); break;
  }
}

template <typename R>
__device__ __forceinline__ int src_bit(uint8_t src, uint8_t bit, uint64_t tile, int lane, int warp) {
  switch (src) {
    case CS_TILE: return (int)((tile >> bit) & 1ull);
    case CS_LANE: return (lane >> bit) & 1;
    case CS_WARP: return (warp >> bit) & 1;
    default: return 0;
  }
}

// G2: the pass holds dense two-qubit ops (a kernel variant of its own, so that
// passes without them keep the leaner code)
template <typename R, bool G2>
__device__ __forceinline__ void apply_tile_op(C2<R>* v, const TileOp<R>* __restrict__ opp,
                                              uint64_t tile, int lane, int warp) {
  const uint8_t kind = opp->kind, slot = opp->slot, csrc = opp->csrc, cbit = opp->cbit;
  if constexpr (G2) {
    if (kind == TK_G2) {   // reads its continuation opp[1]
      apply_g2(v, opp, lane);
      return;
    }
  }
  C2<R> m0[4], m1[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) m0[i] = opp->m0[i];
  if (csrc == CS_NONE && kind != TK_DIAG) {   // no choice bit: one matrix, no matrix selects
    if (kind == TK_REG) {
      switch (slot) {
        case 0: reg_gate<0>(v, m0); break;
        case 1: reg_gate<1>(v, m0); break;
        case 2: reg_gate<2>(v, m0); break;
        default: reg_gate<3>(v, m0); break;
      }
      return;
    }
    const int mask = 1 << slot;
    const bool b = (lane >> slot) & 1;
    const C2<R> o = csel(b, m0[3], m0[0]), p = csel(b, m0[2], m0[1]);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const C2<R> q = shfl_xor_c(v[r], mask);
      v[r] = cfma2(o, v[r], p, q);
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) m1[i] = opp->m1[i];
  if (kind == TK_REG) {
    if (csrc == CS_REG) {
      switch (slot * 4 + cbit) {
        case 1: reg_gate_choice<0, 1>(v, m0, m1); break;
        case 2: reg_gate_choice<0, 2>(v, m0, m1); break;
        case 3: reg_gate_choice<0, 3>(v, m0, m1); break;
        case 4: reg_gate_choice<1, 0>(v, m0, m1); break;
        case 6: reg_gate_choice<1, 2>(v, m0, m1); break;
        case 7: reg_gate_choice<1, 3>(v, m0, m1); break;
        case 8: reg_gate_choice<2, 0>(v, m0, m1); break;
        case 9: reg_gate_choice<2, 1>(v, m0, m1); break;
        case 11: reg_gate_choice<2, 3>(v, m0, m1); break;
        case 12: reg_gate_choice<3, 0>(v, m0, m1); break;
        case 13: reg_gate_choice<3, 1>(v, m0, m1); break;
        case 14: reg_gate_choice<3, 2>(v, m0, m1); break;
        default: break;
      }
      return;
    }
    const bool s = (csrc != CS_NONE) && src_bit<R>(csrc, cbit, tile, lane, warp);
    C2<R> m[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) m[i] = csel(s, m1[i], m0[i]);
    switch (slot) {
      case 0: reg_gate<0>(v, m); break;
      case 1: reg_gate<1>(v, m); break;
      case 2: reg_gate<2>(v, m); break;
      default: reg_gate<3>(v, m); break;
    }
    return;
  }
  if (kind == TK_LANE) {
    const int mask = 1 << slot;
    const bool b = (lane >> slot) & 1;
    // out = own-coefficient * own + partner-coefficient * partner
    const C2<R> o0 = csel(b, m0[3], m0[0]), p0 = csel(b, m0[2], m0[1]);
    const C2<R> o1 = csel(b, m1[3], m1[0]), p1 = csel(b, m1[2], m1[1]);
    if (csrc == CS_REG) {
      switch (cbit) {
        case 0: lane_gate_choice<0>(v, mask, o0, p0, o1, p1); break;
        case 1: lane_gate_choice<1>(v, mask, o0, p0, o1, p1); break;
        case 2: lane_gate_choice<2>(v, mask, o0, p0, o1, p1); break;
        default: lane_gate_choice<3>(v, mask, o0, p0, o1, p1); break;
      }
      return;
    }
    const bool s = (csrc != CS_NONE) && src_bit<R>(csrc, cbit, tile, lane, warp);
    const C2<R> o = csel(s, o1, o0), p = csel(s, p1, p0);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const C2<R> q = shfl_xor_c(v[r], mask);
      v[r] = cfma2(o, v[r], p, q);
    }
    return;
  }
  // TK_DIAG ops go through DiagRun below.
}

// A run of consecutive diagonal ops (they commute) collapses, per thread, into a
// diagonal over the 4 register bits: a scalar s (ops whose bits are all lane,
// warp or tile-constant bits) times one 2-entry factor f[k] per register slot k
// (ops with one bit in a register).  An op with both bits in registers
// multiplies v directly.  flush() multiplies the collected diagonal into v once
// the run ends.  Per op this is 1-2 complex products per thread instead of 16.
template <typename R>
struct DiagRun {
  C2<R> s, f0[2], f1[2], f2[2], f3[2];   // compile-time indices only (registers)

  __device__ __forceinline__ void reset() {
    const C2<R> one{R(1), R(0)};
    s = one;
    f0[0] = f0[1] = f1[0] = f1[1] = f2[0] = f2[1] = f3[0] = f3[1] = one;
  }
  __device__ __forceinline__ void fold(int k, C2<R> e0, C2<R> e1) {
    switch (k) {
      case 0: f0[0] = cmul(f0[0], e0); f0[1] = cmul(f0[1], e1); break;
      case 1: f1[0] = cmul(f1[0], e0); f1[1] = cmul(f1[1], e1); break;
      case 2: f2[0] = cmul(f2[0], e0); f2[1] = cmul(f2[1], e1); break;
      default: f3[0] = cmul(f3[0], e0); f3[1] = cmul(f3[1], e1); break;
    }
  }
  // d[2*bit_a + bit_b] (d[bit_a] for one-qubit diagonals); with TWO the
  // direct products go to v2 as well (the adjoint pass carries two states)
  template <bool TWO = false>
  __device__ __forceinline__ void add(C2<R>* v, const TileOp<R>* __restrict__ opp, uint64_t tile,
                                      int lane, int warp, C2<R>* v2 = nullptr) {
    const uint8_t csrc = opp->csrc, cbit = opp->cbit, dsrc = opp->dsrc, dbit = opp->dbit;
    C2<R> d[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = opp->m0[i];
    const bool two = dsrc != CS_NONE;
    const bool ra = csrc == CS_REG, rb = dsrc == CS_REG;
    if (ra && rb) {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int idx = ((r >> cbit) & 1) * 2 + ((r >> dbit) & 1);
        const C2<R> f = csel(idx >= 2, csel(idx == 3, d[3], d[2]), csel(idx == 1, d[1], d[0]));
        v[r] = cmul(v[r], f);
        if (TWO) v2[r] = cmul(v2[r], f);
      }
      return;
    }
    const int ua = ra ? 0 : src_bit<R>(csrc, cbit, tile, lane, warp);
    const int ub = (two && !rb) ? src_bit<R>(dsrc, dbit, tile, lane, warp) : 0;
    if (ra) {   // entries for bit_a = 0 and 1 at this thread's bit_b
      if (two) fold(cbit, csel(ub, d[1], d[0]), csel(ub, d[3], d[2]));
      else fold(cbit, d[0], d[1]);
    } else if (rb) {   // entries for bit_b = 0 and 1 at this thread's bit_a
      fold(dbit, csel(ua, d[2], d[0]), csel(ua, d[3], d[1]));
    } else {
      const int idx = two ? (ua * 2 + ub) : ua;
      s = cmul(s, csel(idx >= 2, csel(idx == 3, d[3], d[2]), csel(idx == 1, d[1], d[0])));
    }
  }
  // TK_CP: one complex multiply into the factor of the register bit (or into
  // s), selected by the other bit; 16 selected multiplies when both bits are
  // register bits
  // (hdr = the op's first 16 bytes, read with one load: kind, slot, csrc,
  // cbit | dsrc, dbit, term | pad[0..3] | pad[4..7])
  __device__ __forceinline__ void add_cp(C2<R>* v, const TileOp<R>* __restrict__ opp, uint4 hdr,
                                         uint64_t ctx) {
    const uint32_t csrc = (hdr.x >> 16) & 0xffu, cbit = hdr.x >> 24, dsrc = hdr.y & 0xffu,
                   dbit = (hdr.y >> 8) & 0xffu, pa = hdr.z & 0xffu, pb = (hdr.z >> 8) & 0xffu;
    const C2<R> p = opp->m0[0], one{R(1), R(0)};
    const bool ra = csrc == CS_REG, rb = dsrc == CS_REG;
    if (ra && rb) {
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], csel(((r >> cbit) & (r >> dbit) & 1) != 0, p, one));
      return;
    }
    const int ua = ra ? 1 : (int)((ctx >> pa) & 1ull);
    const int ub = rb ? 1 : (int)((ctx >> pb) & 1ull);
    const C2<R> e = csel((ua & ub) != 0, p, one);
    if (ra || rb) {
      switch (ra ? cbit : dbit) {
        case 0: f0[1] = cmul(f0[1], e); break;
        case 1: f1[1] = cmul(f1[1], e); break;
        case 2: f2[1] = cmul(f2[1], e); break;
        default: f3[1] = cmul(f3[1], e); break;
      }
    } else {
      s = cmul(s, e);
    }
  }
  // TK_RUN (tile_cp.h): the residual entries, the CTA's prologue factors U of the
  // run's jobs, and the (lane, warp) / register tables of the pass (lw = warp * 32 +
  // lane)
  __device__ __forceinline__ void add_run(C2<R>* v, const TileOp<R>* __restrict__ opp, uint64_t ctx, int lw,
                                          const C2<R>* U, const C2<R>* __restrict__ tabs) {
    RunHeader h;
    memcpy(&h, &opp->m0[0], sizeof(h));
    const RunEntry<R>* __restrict__ e = reinterpret_cast<const RunEntry<R>*>(opp + 1);
    const C2<R> one{R(1), R(0)};
    int i = 0;
    for (const int n = h.n_s; i < n; ++i) {
      const RunEntry<R> x = e[i];
      s = cmul(s, csel(((ctx >> x.pa) & (ctx >> x.pb) & 1ull) != 0, x.p, one));
    }
    for (const int n = i + h.n_f[0]; i < n; ++i) {
      const RunEntry<R> x = e[i];
      f0[1] = cmul(f0[1], csel(((ctx >> x.pa) & 1ull) != 0, x.p, one));
    }
    for (const int n = i + h.n_f[1]; i < n; ++i) {
      const RunEntry<R> x = e[i];
      f1[1] = cmul(f1[1], csel(((ctx >> x.pa) & 1ull) != 0, x.p, one));
    }
    for (const int n = i + h.n_f[2]; i < n; ++i) {
      const RunEntry<R> x = e[i];
      f2[1] = cmul(f2[1], csel(((ctx >> x.pa) & 1ull) != 0, x.p, one));
    }
    for (const int n = i + h.n_f[3]; i < n; ++i) {
      const RunEntry<R> x = e[i];
      f3[1] = cmul(f3[1], csel(((ctx >> x.pa) & 1ull) != 0, x.p, one));
    }
    if (h.umask) {
      int u = h.ubase;
      if (h.umask & 1) s = cmul(s, U[u++]);
      if (h.umask & 2) f0[1] = cmul(f0[1], U[u++]);
      if (h.umask & 4) f1[1] = cmul(f1[1], U[u++]);
      if (h.umask & 8) f2[1] = cmul(f2[1], U[u++]);
      if (h.umask & 16) f3[1] = cmul(f3[1], U[u++]);
    }
    if (h.tmask) {
      const C2<R>* __restrict__ T = tabs + h.toff;
      if (h.tmask & 1) {
        s = cmul(s, T[lw]);
        T += kRunTable;
      }
      if (h.tmask & 2) {
        f0[1] = cmul(f0[1], T[lw]);
        T += kRunTable;
      }
      if (h.tmask & 4) {
        f1[1] = cmul(f1[1], T[lw]);
        T += kRunTable;
      }
      if (h.tmask & 8) {
        f2[1] = cmul(f2[1], T[lw]);
        T += kRunTable;
      }
      if (h.tmask & 16) {
        f3[1] = cmul(f3[1], T[lw]);
        T += kRunTable;
      }
      if (h.tmask & 32) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], T[r]);
      }
    }
  }
  template <bool TWO = false>
  __device__ __forceinline__ void flush(C2<R>* v, C2<R>* v2 = nullptr) {
    // D(r) = s f0[r0] f1[r1] f2[r2] f3[r3] as (s f0 f1)[r & 3] * (f2 f3)[r >> 2]
    const C2<R> a0 = cmul(s, f0[0]), a1 = cmul(s, f0[1]);
    const C2<R> lo[4] = {cmul(a0, f1[0]), cmul(a1, f1[0]), cmul(a0, f1[1]), cmul(a1, f1[1])};
    const C2<R> hi[4] = {cmul(f2[0], f3[0]), cmul(f2[1], f3[0]), cmul(f2[0], f3[1]),
                         cmul(f2[1], f3[1])};
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const C2<R> D = cmul(lo[r & 3], hi[r >> 2]);
      v[r] = cmul(v[r], D);
      if (TWO) v2[r] = cmul(v2[r], D);
    }
    reset();
  }
};

// G2: the pass holds dense two-qubit ops; RUNS: it holds packed diagonal runs
// (TK_RUN).  Each combination is its own instantiation, so that a pass without
// them keeps the leaner code and register allocation.
template <typename R, bool G2, bool RUNS>
__global__ void __launch_bounds__(kTileThreads)
    tile_pass_kernel(C2<R>* __restrict__ psi, const __grid_constant__ TileParams<R> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<R>* sm = reinterpret_cast<C2<R>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t tile = blockIdx.x;

  __shared__ uint8_t s_pos[kTileBits];
  __shared__ uint64_t s_base;
  __shared__ C2<R> s_U[RUNS ? kMaxRunJobs : 1];   // the CTA's run-job factors
  if (tid == 0) {
    const int n_nt = P.pass.n_nt;
    uint64_t base = 0;
    for (int j = 0; j < n_nt; ++j) base |= ((tile >> j) & 1ull) << P.pass.nt_pos[j];
    s_base = base;
  }
  if (tid < kTileBits) s_pos[tid] = P.pass.pos[tid];
  if constexpr (RUNS) {
    // one job per thread: the product of its entries' phases at this tile (bits
    // below kCtxOne are tile bits, kCtxOne the constant 1)
    if (tid < P.n_jobs) {
      RunJob jb;
      memcpy(&jb, P.jobs + sizeof(RunJob) * tid, sizeof(jb));
      const uint64_t tctx = tile | (1ull << kCtxOne);
      const RunEntry<R>* __restrict__ e = reinterpret_cast<const RunEntry<R>*>(P.ops + jb.op + 1) + jb.first;
      const C2<R> one{R(1), R(0)};
      C2<R> u = one;
      for (int i = 0; i < jb.count; ++i) {
        const RunEntry<R> x = e[i];
        const uint64_t b = jb.scalar ? ((tctx >> x.pa) & (tctx >> x.pb)) : (tctx >> x.pa);
        u = cmul(u, csel((b & 1ull) != 0, x.p, one));
      }
      s_U[tid] = u;
    }
  }
  __syncthreads();
  const uint64_t base = s_base;
  uint64_t loff = 0;
#pragma unroll
  for (int k = 0; k < kLaneBits; ++k)
    if ((lane >> k) & 1) loff |= 1ull << s_pos[k];

  const int nst = P.pass.n_stages;
  const TileStage* __restrict__ S = P.stages;
  const TileOp<R>* __restrict__ ops = P.ops;
  // context word of TK_CP bits: tile index, a constant 1 at bit 47, lane, warp
  const uint64_t ctx = tile | (1ull << kCtxOne) | ((uint64_t)lane << kCtxLane) | ((uint64_t)warp << kCtxWarp);
  C2<R> v[16];
  {
    const TileStage s0 = S[0];
    uint64_t g[kRegBits];
#pragma unroll
    for (int k = 0; k < kRegBits; ++k) g[k] = 1ull << s_pos[s0.reg[k]];
    uint64_t woff = 0;
#pragma unroll
    for (int k = 0; k < kWarpBits; ++k)
      if ((warp >> k) & 1) woff |= 1ull << s_pos[s0.warp[k]];
    const C2<R>* __restrict__ src = psi + (base | loff | woff);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      uint64_t o = 0;
#pragma unroll
      for (int k = 0; k < kRegBits; ++k)
        if ((r >> k) & 1) o |= g[k];
      v[r] = src[o];
    }
  }
  for (int s = 0; s < nst; ++s) {
    const TileStage cur = S[s];
    if (s > 0) {
      const TileStage prev = S[s - 1];
      int rb[kRegBits];
      int wo = lane;
#pragma unroll
      for (int k = 0; k < kRegBits; ++k) rb[k] = 1 << prev.reg[k];
#pragma unroll
      for (int k = 0; k < kWarpBits; ++k)
        if ((warp >> k) & 1) wo |= 1 << prev.warp[k];
      if (s > 1) __syncthreads();
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        int o = wo;
#pragma unroll
        for (int k = 0; k < kRegBits; ++k)
          if ((r >> k) & 1) o |= rb[k];
        sm[o] = v[r];
      }
      __syncthreads();
      int ro = lane;
#pragma unroll
      for (int k = 0; k < kRegBits; ++k) rb[k] = 1 << cur.reg[k];
#pragma unroll
      for (int k = 0; k < kWarpBits; ++k)
        if ((warp >> k) & 1) ro |= 1 << cur.warp[k];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        int o = ro;
#pragma unroll
        for (int k = 0; k < kRegBits; ++k)
          if ((r >> k) & 1) o |= rb[k];
        v[r] = sm[o];
      }
    }
    for (int o = cur.op_begin; o < cur.op_end;) {
      const uint8_t k0 = ops[o].kind;
      if (k0 != TK_DIAG && k0 != TK_CP && !(RUNS && k0 == TK_RUN)) {
        apply_tile_op<R, G2>(v, ops + o, tile, lane, warp);
        o += (G2 && k0 == TK_G2) ? 2 : 1;   // a dense two-qubit op spans two entries
        continue;
      }
      DiagRun<R> dr;   // live only over the run
      dr.reset();
      uint4 hdr = *reinterpret_cast<const uint4*>(ops + o);
      do {
        const uint32_t kind = hdr.x & 0xffu;
        if (RUNS && kind == TK_RUN) {
          dr.add_run(v, ops + o, ctx, tid, s_U, P.tabs);
          o += 1 + (int)((hdr.x >> 8) & 0xffu);   // the header and its entry slots
        } else {
          if (kind == TK_CP) dr.add_cp(v, ops + o, hdr, ctx);
          else dr.add(v, ops + o, tile, lane, warp);
          ++o;
        }
        if (o >= cur.op_end) break;
        hdr = *reinterpret_cast<const uint4*>(ops + o);
      } while ((hdr.x & 0xffu) == TK_DIAG || (hdr.x & 0xffu) == TK_CP || (RUNS && (hdr.x & 0xffu) == TK_RUN));
      dr.flush(v);
    }
  }
  {
    const TileStage sl = S[nst - 1];
    uint64_t g[kRegBits];
#pragma unroll
    for (int k = 0; k < kRegBits; ++k) g[k] = 1ull << s_pos[sl.reg[k]];
    uint64_t woff = 0;
#pragma unroll
    for (int k = 0; k < kWarpBits; ++k)
      if ((warp >> k) & 1) woff |= 1ull << s_pos[sl.warp[k]];
    C2<R>* __restrict__ dst = psi + (base | loff | woff);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      uint64_t o = 0;
#pragma unroll
      for (int k = 0; k < kRegBits; ++k)
        if ((r >> k) & 1) o |= g[k];
      dst[o] = v[r];
    }
  }
}

// ------------------------------------------------------------------ adjoint pass
//
// The backward sweep of the adjoint gradient over one tile pass.  With
// lambda = dL/dpsi^* propagated backwards, dL/dt of a gate's parameter is
// 2 Re <lambda_g | dU/dt | psi_{g-1}> = 2 Re <lambda_g | G psi_g> with
// G = (dU/dt) U^dagger, psi_g and lambda_g the states after the gate.  The host
// lists, for each gate from the last, one op per parameter carrying G (term >= 0)
// and then U^dagger; the tile planner keeps the order of ops that share a qubit,
// and a term op commutes with the U^dagger of a gate on other qubits (that unitary
// cancels from the inner product).  Here a tile of psi and one of lambda stay in
// registers through the pass: U^dagger ops act on both, a term op adds
// Re sum_J conj(lambda_J) (G psi)_J over the tile into s_term[term] (warp sums,
// shared-memory atomics), written per tile to partial[tile][term].

// Re sum over this thread's 16 amplitudes of conj(l) (G p), G the op's matrix
template <typename R>
__device__ __forceinline__ R term_of_op(const C2<R>* vp, const C2<R>* vl, const TileOp<R>* __restrict__ opp,
                                        uint64_t tile, int lane, int warp) {
  C2<R> g[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) g[i] = opp->m0[i];
  R t = 0;
  auto dotre = [](C2<R> a, C2<R> b) { return fma(a.x, b.x, a.y * b.y); };   // Re conj(a) b
  if (opp->kind == TK_REG) {
    // pairs (r, r | 2^k) of register slot k; a switch keeps register indices constant
    switch (opp->slot) {
      case 0:
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          if (r & 1) continue;
          t += dotre(vl[r], cfma2(g[0], vp[r], g[1], vp[r | 1])) + dotre(vl[r | 1], cfma2(g[2], vp[r], g[3], vp[r | 1]));
        }
        break;
      case 1:
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          if (r & 2) continue;
          t += dotre(vl[r], cfma2(g[0], vp[r], g[1], vp[r | 2])) + dotre(vl[r | 2], cfma2(g[2], vp[r], g[3], vp[r | 2]));
        }
        break;
      case 2:
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          if (r & 4) continue;
          t += dotre(vl[r], cfma2(g[0], vp[r], g[1], vp[r | 4])) + dotre(vl[r | 4], cfma2(g[2], vp[r], g[3], vp[r | 4]));
        }
        break;
      default:
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          if (r & 8) continue;
          t += dotre(vl[r], cfma2(g[0], vp[r], g[1], vp[r | 8])) + dotre(vl[r | 8], cfma2(g[2], vp[r], g[3], vp[r | 8]));
        }
    }
    return t;
  }
  if (opp->kind == TK_LANE) {
    const int mask = 1 << opp->slot;
    const bool b = (lane & mask) != 0;
    const C2<R> o = csel(b, g[3], g[0]), q = csel(b, g[2], g[1]);   // own and partner coefficients
#pragma unroll
    for (int r = 0; r < 16; ++r) t += dotre(vl[r], cfma2(o, vp[r], q, shfl_xor_c(vp[r], mask)));
    return t;
  }
  // TK_DIAG: (G p)_J = d[2 bit_a + bit_b] p_J
  const uint8_t csrc = opp->csrc, cbit = opp->cbit, dsrc = opp->dsrc, dbit = opp->dbit;
  const bool two = dsrc != CS_NONE;
  const int ua = csrc == CS_REG ? 0 : src_bit<R>(csrc, cbit, tile, lane, warp);
  const int ub = (two && dsrc != CS_REG) ? src_bit<R>(dsrc, dbit, tile, lane, warp) : 0;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int ba = csrc == CS_REG ? ((r >> cbit) & 1) : ua;
    const int bb = two ? (dsrc == CS_REG ? ((r >> dbit) & 1) : ub) : 0;
    const int idx = two ? ba * 2 + bb : ba;
    const C2<R> f = csel(idx >= 2, csel(idx == 3, g[3], g[2]), csel(idx == 1, g[1], g[0]));
    t += dotre(vl[r], cmul(f, vp[r]));
  }
  return t;
}

template <typename R, bool G2>
__global__ void __launch_bounds__(kTileThreads, sizeof(R) == 4 ? 2 : 1)
    adjoint_pass_kernel(C2<R>* __restrict__ psi, C2<R>* __restrict__ lam,
                        const __grid_constant__ TileParams<R> P, R* __restrict__ partial, int nterm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<R>* smp = reinterpret_cast<C2<R>*>(smem_raw);
  C2<R>* sml = smp + (1 << kTileBits);
  __shared__ R s_term[TileLimits<R>::kMaxOps];   // the state's precision
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t tile = blockIdx.x;

  __shared__ uint8_t s_pos[kTileBits];
  __shared__ uint64_t s_base;
  if (tid == 0) {
    const int n_nt = P.pass.n_nt;
    uint64_t base = 0;
    for (int j = 0; j < n_nt; ++j) base |= ((tile >> j) & 1ull) << P.pass.nt_pos[j];
    s_base = base;
  }
  if (tid < kTileBits) s_pos[tid] = P.pass.pos[tid];
  for (int i = tid; i < nterm; i += kTileThreads) s_term[i] = R(0);
  __syncthreads();
  const uint64_t base = s_base;
  uint64_t loff = 0;
#pragma unroll
  for (int k = 0; k < kLaneBits; ++k)
    if ((lane >> k) & 1) loff |= 1ull << s_pos[k];

  const int nst = P.pass.n_stages;
  const TileStage* __restrict__ S = P.stages;
  const TileOp<R>* __restrict__ ops = P.ops;
  C2<R> vp[16], vl[16];
  {
    const TileStage s0 = S[0];
    uint64_t g[kRegBits];
#pragma unroll
    for (int k = 0; k < kRegBits; ++k) g[k] = 1ull << s_pos[s0.reg[k]];
    uint64_t woff = 0;
#pragma unroll
    for (int k = 0; k < kWarpBits; ++k)
      if ((warp >> k) & 1) woff |= 1ull << s_pos[s0.warp[k]];
    const uint64_t off0 = base | loff | woff;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      uint64_t o = 0;
#pragma unroll
      for (int k = 0; k < kRegBits; ++k)
        if ((r >> k) & 1) o |= g[k];
      vp[r] = psi[off0 + o];
      vl[r] = lam[off0 + o];
    }
  }
  for (int s = 0; s < nst; ++s) {
    const TileStage cur = S[s];
    if (s > 0) {
      const TileStage prev = S[s - 1];
      int rb[kRegBits];
      int wo = lane;
#pragma unroll
      for (int k = 0; k < kRegBits; ++k) rb[k] = 1 << prev.reg[k];
#pragma unroll
      for (int k = 0; k < kWarpBits; ++k)
        if ((warp >> k) & 1) wo |= 1 << prev.warp[k];
      if (s > 1) __syncthreads();
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        int o = wo;
#pragma unroll
        for (int k = 0; k < kRegBits; ++k)
          if ((r >> k) & 1) o |= rb[k];
        smp[o] = vp[r];
        sml[o] = vl[r];
      }
      __syncthreads();
      int ro = lane;
#pragma unroll
      for (int k = 0; k < kRegBits; ++k) rb[k] = 1 << cur.reg[k];
#pragma unroll
      for (int k = 0; k < kWarpBits; ++k)
        if ((warp >> k) & 1) ro |= 1 << cur.warp[k];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        int o = ro;
#pragma unroll
        for (int k = 0; k < kRegBits; ++k)
          if ((r >> k) & 1) o |= rb[k];
        vp[r] = smp[o];
        vl[r] = sml[o];
      }
    }
    for (int o = cur.op_begin; o < cur.op_end;) {
      const TileOp<R>* op = ops + o;
      if (op->term >= 0) {
        R t = term_of_op<R>(vp, vl, op, tile, lane, warp);
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
        if (lane == 0) atomicAdd(&s_term[op->term], t);
        ++o;
        continue;
      }
      if (op->kind != TK_DIAG) {
        apply_tile_op<R, G2>(vp, op, tile, lane, warp);
        apply_tile_op<R, G2>(vl, op, tile, lane, warp);
        o += (G2 && op->kind == TK_G2) ? 2 : 1;   // a dense two-qubit op spans two entries
        continue;
      }
      DiagRun<R> dr;   // a run of diagonal U^dagger ops, on both states
      dr.reset();
      do {
        dr.template add<true>(vp, ops + o, tile, lane, warp, vl);
        ++o;
      } while (o < cur.op_end && ops[o].kind == TK_DIAG && ops[o].term < 0);
      dr.template flush<true>(vp, vl);
    }
  }
  {
    const TileStage sl = S[nst - 1];
    uint64_t g[kRegBits];
#pragma unroll
    for (int k = 0; k < kRegBits; ++k) g[k] = 1ull << s_pos[sl.reg[k]];
    uint64_t woff = 0;
#pragma unroll
    for (int k = 0; k < kWarpBits; ++k)
      if ((warp >> k) & 1) woff |= 1ull << s_pos[sl.warp[k]];
    const uint64_t off0 = base | loff | woff;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      uint64_t o = 0;
#pragma unroll
      for (int k = 0; k < kRegBits; ++k)
        if ((r >> k) & 1) o |= g[k];
      psi[off0 + o] = vp[r];
      lam[off0 + o] = vl[r];
    }
  }
  __syncthreads();
  for (int i = tid; i < nterm; i += kTileThreads) partial[(size_t)tile * nterm + i] = s_term[i];
}

// dth[slots[i]] += 2 sum over tiles of partial[tile][i] (FP64, one block per term)
template <typename R>
__global__ void __launch_bounds__(256)
    term_reduce_kernel(const R* __restrict__ partial, uint64_t tiles, int nterm,
                       const int* __restrict__ slots, double* __restrict__ dth) {
  const int i = blockIdx.x;
  double acc = 0.0;
  for (uint64_t t = threadIdx.x; t < tiles; t += blockDim.x) acc += (double)partial[t * nterm + i];
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) dth[slots[i]] += 2.0 * tot;
}

// ------------------------------------------------------------------ plain per-gate

template <typename R>
__global__ void plain_g1_kernel(C2<R>* __restrict__ psi, int n, PlainOp<R> op) {
  const uint64_t half = 1ull << (n - 1);
  const int t = op.t;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < half;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = insert_zero(i, t), i1 = i0 | (1ull << t);
    const C2<R>* m = op.m;
    if (op.type == F_G1C && ((i0 >> op.c) & 1ull)) m = op.m + 4;
    const C2<R> a = psi[i0], b = psi[i1];
    psi[i0] = cfma2(m[0], a, m[1], b);
    psi[i1] = cfma2(m[2], a, m[3], b);
  }
}

template <typename R>
__global__ void plain_diag_kernel(C2<R>* __restrict__ psi, int n, PlainOp<R> op) {
  const uint64_t N = 1ull << n;
  for (uint64_t J = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; J < N;
       J += (uint64_t)gridDim.x * blockDim.x) {
    const int ba = (int)((J >> op.a) & 1ull);
    const int idx = op.b >= 0 ? ba * 2 + (int)((J >> op.b) & 1ull) : ba;
    psi[J] = cmul(psi[J], op.m[idx]);
  }
}

template <typename R>
__global__ void plain_g2_kernel(C2<R>* __restrict__ psi, int n, PlainOp<R> op) {
  const uint64_t quarter = 1ull << (n - 2);
  const int lo = op.a < op.b ? op.a : op.b, hi = op.a < op.b ? op.b : op.a;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < quarter;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t base = insert_zero(insert_zero(i, lo), hi);
    uint64_t idx[4];
    C2<R> a[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {   // local index 2*bit_a + bit_b
      idx[l] = base | ((uint64_t)(l >> 1) << op.a) | ((uint64_t)(l & 1) << op.b);
      a[l] = psi[idx[l]];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      C2<R> acc = cfma2(op.m[4 * r + 0], a[0], op.m[4 * r + 1], a[1]);
      const C2<R> acc2 = cfma2(op.m[4 * r + 2], a[2], op.m[4 * r + 3], a[3]);
      acc.x += acc2.x;
      acc.y += acc2.y;
      psi[idx[r]] = acc;
    }
  }
}

// ------------------------------------------------------------------ small states

template <typename R>
__global__ void __launch_bounds__(256)
    small_state_kernel(C2<R>* __restrict__ psi, int n, const PlainOp<R>* __restrict__ ops, int nops) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<R>* sm = reinterpret_cast<C2<R>*>(smem_raw);
  const int N = 1 << n;
  for (int J = threadIdx.x; J < N; J += blockDim.x) sm[J] = psi[J];
  __syncthreads();
  small_apply_ops(sm, n, ops, nops);
  for (int J = threadIdx.x; J < N; J += blockDim.x) psi[J] = sm[J];
}

// ------------------------------------------------------------------ remap

__device__ __forceinline__ uint64_t tiles_of(const RemapDesc& d) { return 1ull << d.n_nt; }

template <typename R>
__global__ void __launch_bounds__(kTileThreads, sizeof(R) == 4 ? 3 : 2)
    remap_kernel(C2<R>* __restrict__ psi, const __grid_constant__ RemapDesc D) {
  const RemapDesc* d = &D;   // kernel parameter (constant bank)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<R>* sm = reinterpret_cast<C2<R>*>(smem_raw);
  // Every map below is linear over GF(2) in the bits of a 12-bit local index, so
  // each is the XOR of a table entry for the low 6 and one for the high 6 bits:
  //   address  local index -> offset in psi (deposit into the tile positions),
  //   slot     input index -> shared-memory slot (bank swizzle, below),
  //   gather   output index -> slot of the input amplitude it takes.
  // complex64 moves amplitude pairs (local bit 0 = position 0, which every remap
  // holds): one 16-byte global access per pair and one 16-byte shared store, the
  // two gathered amplitudes read separately.  The swizzle adds to every input
  // bit i >= kB a low slot bit, chosen so that the lanes of a wavefront hit
  // distinct banks both when the tile is written in input order and when it is
  // read in output order: kB = 4 bank-pair bits, output bits 1-4 over the lanes
  // of a half-warp (8-byte reads of complex64 pairs); kB = 3, output bits 0-2
  // over a quarter-warp (16-byte complex128 amplitudes).
  constexpr bool kPairs = sizeof(C2<R>) == 8;
  constexpr int kB = kPairs ? 4 : 3, kK0 = kPairs ? 1 : 0;
  __shared__ uint64_t s_alo[64], s_ahi[64];
  __shared__ uint16_t s_slo[64], s_shi[64], s_glo[64], s_ghi[64];
  __shared__ uint16_t s_m[kTileBits];
  const int tid = threadIdx.x;
  // the tile's bits outside the tile positions, deposited at nt_pos
  auto base_of = [&](uint64_t tile) {
    uint64_t base = 0;
    for (int j = 0; j < d->n_nt; ++j) base |= ((tile >> j) & 1ull) << d->nt_pos[j];
    return base;
  };
  if (tid == 0) {
    int used = 0;
    for (int k = kK0; k < kK0 + kB; ++k)
      if (d->src[k] < kB) used |= 1 << d->src[k];
    for (int i = 0; i < kTileBits; ++i) s_m[i] = (uint16_t)(1 << i);
    for (int k = kK0; k < kK0 + kB; ++k) {
      const int sk = d->src[k];
      if (sk < kB) continue;
      const int free_bits = ~used & ((1 << kB) - 1);
      const int j = free_bits & -free_bits;   // lowest unused bank bit
      used |= j;
      s_m[sk] = (uint16_t)(s_m[sk] ^ j);
    }
  }
  __syncthreads();
  if (tid < 128) {
    const int v = tid & 63, h = tid >> 6;   // entry v of the low (h = 0) or high table
    uint64_t a = 0;
    int slot = 0, gather = 0;
    for (int i = 0; i < 6; ++i)
      if ((v >> i) & 1) {
        a |= 1ull << d->pos[6 * h + i];
        slot ^= s_m[6 * h + i];
        gather ^= s_m[d->src[6 * h + i]];
      }
    (h ? s_ahi : s_alo)[v] = a;
    (h ? s_shi : s_slo)[v] = (uint16_t)slot;
    (h ? s_ghi : s_glo)[v] = (uint16_t)gather;
  }
  __syncthreads();
  // Persistent over tiles (grid = a few CTAs per SM): the next tile's loads are
  // issued into registers before the current tile is gathered and stored, so a
  // CTA keeps reads in flight through its exchange and store phases.
  const uint64_t tiles = tiles_of(D);
  uint64_t tile = blockIdx.x;
  if (tile >= tiles) return;
  if (kPairs && d->pos[0] == 0) {
    // slot(L ^ 1) = slot(L) ^ 1: a pair fills one aligned 16-byte slot pair.  A
    // thread's offsets, slots and gathers are the same for every tile: read from
    // the tables once, kept in registers.
    constexpr int kPer = (1 << kTileBits) / (2 * kTileThreads);
    float4* sm4 = reinterpret_cast<float4*>(smem_raw);
    const float* smf = reinterpret_cast<const float*>(smem_raw);
    float4* psi4 = reinterpret_cast<float4*>(psi);
    const int g1 = s_glo[1];   // gather(L ^ 1) = gather(L) ^ g1
    uint64_t ad[kPer];
    int sl[kPer], ga[kPer];
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int L = 2 * (tid + r * kTileThreads);
      ad[r] = (s_alo[L & 63] | s_ahi[L >> 6]) >> 1;
      sl[r] = s_slo[L & 63] ^ s_shi[L >> 6];
      ga[r] = s_glo[L & 63] ^ s_ghi[L >> 6];
    }
    uint64_t base = base_of(tile) >> 1;
    float4 q[kPer];
#pragma unroll
    for (int r = 0; r < kPer; ++r) q[r] = __ldcs(psi4 + (base | ad[r]));
    for (;;) {
#pragma unroll
      for (int r = 0; r < kPer; ++r)
        sm4[sl[r] >> 1] = (sl[r] & 1) ? make_float4(q[r].z, q[r].w, q[r].x, q[r].y) : q[r];
      __syncthreads();
      const uint64_t next = tile + gridDim.x;
      const uint64_t nbase = next < tiles ? base_of(next) >> 1 : 0;
      if (next < tiles) {
#pragma unroll
        for (int r = 0; r < kPer; ++r) q[r] = __ldcs(psi4 + (nbase | ad[r]));
      }
#pragma unroll
      for (int r = 0; r < kPer; ++r) {
        const float2 a0 = *reinterpret_cast<const float2*>(smf + 2 * ga[r]);
        const float2 a1 = *reinterpret_cast<const float2*>(smf + 2 * (ga[r] ^ g1));
        __stcs(psi4 + (base | ad[r]), make_float4(a0.x, a0.y, a1.x, a1.y));
      }
      if (next >= tiles) return;
      __syncthreads();   // the tile is gathered before the next one is written to shared memory
      tile = next;
      base = nbase;
    }
  }
  constexpr int kPer = (1 << kTileBits) / kTileThreads;
  uint64_t base = base_of(tile);
  C2<R> q[kPer];
#pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const int L = tid + r * kTileThreads;
    q[r] = psi[base | s_alo[L & 63] | s_ahi[L >> 6]];
  }
  for (;;) {
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int L = tid + r * kTileThreads;
      sm[s_slo[L & 63] ^ s_shi[L >> 6]] = q[r];
    }
    __syncthreads();
    const uint64_t next = tile + gridDim.x;
    const uint64_t nbase = next < tiles ? base_of(next) : 0;
    if (next < tiles) {
#pragma unroll
      for (int r = 0; r < kPer; ++r) {
        const int L = tid + r * kTileThreads;
        q[r] = psi[nbase | s_alo[L & 63] | s_ahi[L >> 6]];
      }
    }
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int L = tid + r * kTileThreads;
      psi[base | s_alo[L & 63] | s_ahi[L >> 6]] = sm[s_glo[L & 63] ^ s_ghi[L >> 6]];
    }
    if (next >= tiles) return;
    __syncthreads();
    tile = next;
    base = nbase;
  }
}

// ------------------------------------------------------------------ reductions

// Per-thread sums of probabilities.  For an FP32 state each thread adds the
// probabilities of a chunk of kChunk of its elements in FP32 with Kahan
// compensation (the chunk sum is good to about one FP32 rounding), and only the
// chunk sums go into its FP64 accumulator: GB300's FP64 pipe is far slower
// than its FP32 pipe, and one FP64 add per element made this HBM-bound kernel
// FP64-bound.  The inner loop holds no FP64 instruction (a fold inside it is
// predicated into every iteration).  The reductions across threads and blocks
// are FP64.
constexpr int kChunk = 32;

struct Kahan32 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float p) {
    const float y = p - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <typename R, typename O>
__global__ void __launch_bounds__(256)
    probs_kernel(const C2<R>* __restrict__ psi, O* __restrict__ out, uint64_t N,
                 double* __restrict__ partials) {
  double acc = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if constexpr (sizeof(R) == 8) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
      const C2<R> a = psi[i];
      const R p = a.x * a.x + a.y * a.y;
      if (out) out[i] = (O)p;
      acc += p;
    }
  } else {
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < N; i0 += stride * kChunk) {
      Kahan32 k;
      for (int j = 0; j < kChunk; ++j) {
        const uint64_t i = i0 + (uint64_t)j * stride;
        if (i < N) {
          const C2<R> a = psi[i];
          const float p = a.x * a.x + a.y * a.y;
          if (out) out[i] = (O)p;
          k.add(p);
        }
      }
      acc += k.value();
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// float specialisation: two amplitudes (16 bytes) per load, two floats per store
__global__ void __launch_bounds__(256)
    probs_kernel_f32x2(const float4* __restrict__ psi2, float2* __restrict__ out2, uint64_t N2,
                       double* __restrict__ partials) {
  double acc = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  constexpr int kBatch = 8;   // loads in flight per thread
  for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < N2; i0 += stride * kChunk) {
    Kahan32 k;
#pragma unroll
    for (int jb = 0; jb < kChunk; jb += kBatch) {
      float4 a[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const uint64_t i = i0 + (uint64_t)(jb + u) * stride;
        a[u] = i < N2 ? __ldcs(psi2 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const uint64_t i = i0 + (uint64_t)(jb + u) * stride;
        float2 p;
        p.x = a[u].x * a[u].x + a[u].y * a[u].y;
        p.y = a[u].z * a[u].z + a[u].w * a[u].w;
        if (out2 && i < N2) __stcs(out2 + i, p);
        k.add(p.x);
        k.add(p.y);
      }
    }
    acc += k.value();
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

template <typename R>
__global__ void __launch_bounds__(256)
    marginal_kernel(const C2<R>* __restrict__ psi, uint64_t N, const uint8_t* __restrict__ bits,
                    int k, double* __restrict__ acc_out, double* __restrict__ partials) {
  extern __shared__ double hist[];
  const int H = 1 << k;
  const bool use_smem = k <= 12;
  if (use_smem)
    for (int i = threadIdx.x; i < H; i += blockDim.x) hist[i] = 0.0;
  __shared__ uint8_t s_bits[64];
  if (threadIdx.x < k) s_bits[threadIdx.x] = bits[threadIdx.x];
  __syncthreads();
  double tot = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t J = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; J < N; J += stride) {
    const C2<R> a = psi[J];
    const double p = (double)(a.x * a.x + a.y * a.y);
    int K = 0;
    for (int i = 0; i < k; ++i) K |= (int)((J >> s_bits[i]) & 1ull) << i;
    if (use_smem) atomicAdd(hist + K, p);
    else atomicAdd(acc_out + K, p);
    tot += p;
  }
  __syncthreads();
  if (use_smem)
    for (int i = threadIdx.x; i < H; i += blockDim.x)
      if (hist[i] != 0.0) atomicAdd(acc_out + i, hist[i]);
  tot = block_sum(tot);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

template <typename O>
__global__ void convert_kernel(const double* __restrict__ in, O* __restrict__ out, uint64_t count) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = (O)in[i];
}

template <typename R>
__global__ void __launch_bounds__(256)
    loglik_kernel(const C2<R>* __restrict__ psi, const uint32_t* __restrict__ counts, uint64_t N,
                  double* __restrict__ partials, unsigned long long* __restrict__ clamps) {
  double acc = 0.0;
  unsigned long long nclamp = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t J = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; J < N; J += stride) {
    const uint32_t c = counts[J];
    if (c == 0) continue;
    const C2<R> a = psi[J];
    double p = (double)(a.x * a.x + a.y * a.y);
    if (!(p > 0.0)) {
      p = 1e-300;
      ++nclamp;
    }
    acc += (double)c * log(p);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  if (nclamp) atomicAdd(clamps, nclamp);
}

__global__ void reduce_partials_kernel(const double* __restrict__ partials, int count,
                                       double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) s += partials[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

template <typename R>
__global__ void set_one_kernel(C2<R>* psi, uint64_t J) {
  C2<R> one;
  one.x = R(1);
  one.y = R(0);
  psi[J] = one;
}

// ------------------------------------------------------------------ launchers

namespace {
int grid_for(uint64_t work, int threads) {
  uint64_t g = (work + threads - 1) / threads;
  const uint64_t cap = 152ull * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename F>
qs_status set_smem(F* f, size_t bytes) {
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute");
  }
  return QS_OK;
}
}  // namespace

qs_status launch_set_basis(State* st, uint64_t J) {
  QS_CUDA(cudaMemsetAsync(st->data, 0, st->data_bytes, st->stream));
  if (st->prec == QS_C64) set_one_kernel<float><<<1, 1, 0, st->stream>>>((C2<float>*)st->data, J);
  else set_one_kernel<double><<<1, 1, 0, st->stream>>>((C2<double>*)st->data, J);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

// does the pass (a host TileParams image) hold a dense two-qubit op?
template <typename R>
static bool pass_has_g2(const TileParams<R>& P) {
  const int nops = P.pass.n_stages > 0 ? P.stages[P.pass.n_stages - 1].op_end : 0;
  for (int o = 0; o < nops; ++o)
    if (P.ops[o].kind == TK_G2) return true;
  return false;
}

// which op kinds a forward pass holds, walking op headers only (a dense
// two-qubit op spans two slots; a TK_RUN header is followed by its entry slots,
// whose bytes are not op headers)
template <typename R>
static void pass_kinds(const TileParams<R>& P, bool* g2, bool* runs) {
  *g2 = *runs = false;
  const int nops = P.pass.n_stages > 0 ? P.stages[P.pass.n_stages - 1].op_end : 0;
  for (int o = 0; o < nops;) {
    const uint8_t k = P.ops[o].kind;
    if (k == TK_RUN) {
      *runs = true;
      o += 1 + P.ops[o].slot;
    } else if (k == TK_G2) {
      *g2 = true;
      o += 2;
    } else {
      ++o;
    }
  }
}

template <typename R, bool G2, bool RUNS>
static qs_status tile_launch_t(State* st, const TileParams<R>& P) {
  const uint64_t tiles = 1ull << (st->n - kTileBits);
  const size_t smem = sizeof(C2<R>) << kTileBits;
  qs_status s = set_smem(tile_pass_kernel<R, G2, RUNS>, smem);
  if (s != QS_OK) return s;
  tile_pass_kernel<R, G2, RUNS><<<(unsigned)tiles, kTileThreads, smem, st->stream>>>((C2<R>*)st->data, P);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

template <typename R>
static qs_status tile_launch_any(State* st, const TileParams<R>& P) {
  bool g2 = false, runs = false;
  pass_kinds(P, &g2, &runs);
  if (g2) return runs ? tile_launch_t<R, true, true>(st, P) : tile_launch_t<R, true, false>(st, P);
  return runs ? tile_launch_t<R, false, true>(st, P) : tile_launch_t<R, false, false>(st, P);
}

qs_status launch_tile_pass(State* st, const void* params) {
  if (st->prec == QS_C64) return tile_launch_any(st, *(const TileParams<float>*)params);
  return tile_launch_any(st, *(const TileParams<double>*)params);
}

template <typename R, bool G2>
static qs_status adjoint_launch_t(State* st, void* lam, const TileParams<R>& P, void* partial, int nterm) {
  const uint64_t tiles = 1ull << (st->n - kTileBits);
  const size_t smem = 2 * (sizeof(C2<R>) << kTileBits);
  qs_status s = set_smem(adjoint_pass_kernel<R, G2>, smem);
  if (s != QS_OK) return s;
  adjoint_pass_kernel<R, G2><<<(unsigned)tiles, kTileThreads, smem, st->stream>>>(
      (C2<R>*)st->data, (C2<R>*)lam, P, (R*)partial, nterm);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_adjoint_pass(State* st, void* lam, const void* params, void* partial, int nterm) {
  if (st->prec == QS_C64) {
    const TileParams<float>& P = *(const TileParams<float>*)params;
    return pass_has_g2(P) ? adjoint_launch_t<float, true>(st, lam, P, partial, nterm)
                          : adjoint_launch_t<float, false>(st, lam, P, partial, nterm);
  }
  const TileParams<double>& P = *(const TileParams<double>*)params;
  return pass_has_g2(P) ? adjoint_launch_t<double, true>(st, lam, P, partial, nterm)
                        : adjoint_launch_t<double, false>(st, lam, P, partial, nterm);
}

qs_status launch_term_reduce(State* st, const void* partial, int nterm, const int* slots, double* dth) {
  if (nterm <= 0) return QS_OK;
  const uint64_t tiles = 1ull << (st->n - kTileBits);
  if (st->prec == QS_C64)
    term_reduce_kernel<float><<<nterm, 256, 0, st->stream>>>((const float*)partial, tiles, nterm, slots, dth);
  else
    term_reduce_kernel<double><<<nterm, 256, 0, st->stream>>>((const double*)partial, tiles, nterm, slots, dth);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

template <typename R>
static qs_status plain_launch_t(State* st, const PlainOp<R>& op) {
  const int n = st->n;
  C2<R>* psi = (C2<R>*)st->data;
  if (op.type == F_G1 || op.type == F_G1C)
    plain_g1_kernel<R><<<grid_for(1ull << (n - 1), 256), 256, 0, st->stream>>>(psi, n, op);
  else if (op.type == F_D)
    plain_diag_kernel<R><<<grid_for(1ull << n, 256), 256, 0, st->stream>>>(psi, n, op);
  else
    plain_g2_kernel<R><<<grid_for(1ull << (n - 2), 256), 256, 0, st->stream>>>(psi, n, op);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_plain_op(State* st, const void* op_host, int /*type*/) {
  if (st->prec == QS_C64) return plain_launch_t<float>(st, *(const PlainOp<float>*)op_host);
  return plain_launch_t<double>(st, *(const PlainOp<double>*)op_host);
}

qs_status launch_small(State* st, const void* ops_dev, int nops) {
  const size_t smem = st->amp_bytes << st->n;
  if (st->prec == QS_C64) {
    qs_status s = set_smem(small_state_kernel<float>, smem);
    if (s != QS_OK) return s;
    small_state_kernel<float><<<1, 256, smem, st->stream>>>((C2<float>*)st->data, st->n,
                                                            (const PlainOp<float>*)ops_dev, nops);
  } else {
    qs_status s = set_smem(small_state_kernel<double>, smem);
    if (s != QS_OK) return s;
    small_state_kernel<double><<<1, 256, smem, st->stream>>>((C2<double>*)st->data, st->n,
                                                             (const PlainOp<double>*)ops_dev, nops);
  }
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_remap(State* st, const RemapDesc& d) {
  const uint64_t tiles = 1ull << (st->n - kTileBits);
  // persistent: as many CTAs as fit on the SMs (shared memory: one tile each)
  auto grid_for = [&](const void* kern, size_t smem) {
    int dev = 0, sms = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kTileThreads, smem);
    const uint64_t g = (uint64_t)sms * (uint64_t)(per < 1 ? 1 : per);
    return (unsigned)(g < tiles ? g : tiles);
  };
  if (st->prec == QS_C64) {
    const size_t smem = sizeof(C2<float>) << kTileBits;
    remap_kernel<float><<<grid_for((const void*)remap_kernel<float>, smem), kTileThreads, smem, st->stream>>>(
        (C2<float>*)st->data, d);
  } else {
    const size_t smem = sizeof(C2<double>) << kTileBits;
    qs_status s = set_smem(remap_kernel<double>, smem);
    if (s != QS_OK) return s;
    remap_kernel<double><<<grid_for((const void*)remap_kernel<double>, smem), kTileThreads, smem, st->stream>>>(
        (C2<double>*)st->data, d);
  }
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_probs_range(State* st, uint64_t off, uint64_t count, void* out, int out_fp64,
                             double* partials) {
  if (st->prec == QS_C64 && !out_fp64 && (off % 2) == 0 && (count % 2) == 0) {
    probs_kernel_f32x2<<<kReduceBlocks, 256, 0, st->stream>>>((const float4*)((const C2<float>*)st->data + off),
                                                              (float2*)out, count / 2, partials);
  } else if (st->prec == QS_C64) {
    if (out_fp64)
      probs_kernel<float, double><<<kReduceBlocks, 256, 0, st->stream>>>(
          (const C2<float>*)st->data + off, (double*)out, count, partials);
    else
      probs_kernel<float, float><<<kReduceBlocks, 256, 0, st->stream>>>(
          (const C2<float>*)st->data + off, (float*)out, count, partials);
  } else if (out_fp64) {
    probs_kernel<double, double><<<kReduceBlocks, 256, 0, st->stream>>>(
        (const C2<double>*)st->data + off, (double*)out, count, partials);
  } else {
    probs_kernel<double, float><<<kReduceBlocks, 256, 0, st->stream>>>(
        (const C2<double>*)st->data + off, (float*)out, count, partials);
  }
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_probs(State* st, void* out, int out_fp64, uint64_t mask, double* partials,
                       uint8_t* dbits, double* marg_acc) {
  const uint64_t N = 1ull << st->n;
  const uint64_t full = (st->n >= 64) ? ~0ull : ((1ull << st->n) - 1);
  const bool marginal = mask != 0 && (mask & full) != full;
  if (!marginal) {
    if (st->prec == QS_C64 && !out_fp64 && st->n >= 1) {
      probs_kernel_f32x2<<<kReduceBlocks, 256, 0, st->stream>>>((const float4*)st->data,
                                                                (float2*)out, N / 2, partials);
    } else if (st->prec == QS_C64) {
      probs_kernel<float, double><<<kReduceBlocks, 256, 0, st->stream>>>(
          (const C2<float>*)st->data, (double*)out, N, partials);
    } else if (out_fp64) {
      probs_kernel<double, double><<<kReduceBlocks, 256, 0, st->stream>>>(
          (const C2<double>*)st->data, (double*)out, N, partials);
    } else {
      probs_kernel<double, float><<<kReduceBlocks, 256, 0, st->stream>>>(
          (const C2<double>*)st->data, (float*)out, N, partials);
    }
    QS_CUDA(cudaGetLastError());
    return QS_OK;
  }
  // marginal over the bits of mask
  uint8_t hbits[64];
  int k = 0;
  for (int b = 0; b < st->n; ++b)
    if ((mask >> b) & 1) hbits[k++] = (uint8_t)b;
  QS_CUDA(cudaMemcpyAsync(dbits, hbits, 64, cudaMemcpyHostToDevice, st->stream));
  const uint64_t H = 1ull << k;
  QS_CUDA(cudaMemsetAsync(marg_acc, 0, H * sizeof(double), st->stream));
  const size_t smem = k <= 12 ? (sizeof(double) << k) : 0;
  if (st->prec == QS_C64)
    marginal_kernel<float><<<kReduceBlocks, 256, smem, st->stream>>>((const C2<float>*)st->data, N,
                                                                     dbits, k, marg_acc, partials);
  else
    marginal_kernel<double><<<kReduceBlocks, 256, smem, st->stream>>>((const C2<double>*)st->data,
                                                                      N, dbits, k, marg_acc, partials);
  QS_CUDA(cudaGetLastError());
  if (out) {
    if (out_fp64)
      QS_CUDA(cudaMemcpyAsync(out, marg_acc, H * sizeof(double), cudaMemcpyDeviceToDevice, st->stream));
    else {
      convert_kernel<float><<<grid_for(H, 256), 256, 0, st->stream>>>(marg_acc, (float*)out, H);
      QS_CUDA(cudaGetLastError());
    }
  }
  return QS_OK;
}

qs_status launch_reduce_partials(State* st, const double* partials, int count, double* out) {
  reduce_partials_kernel<<<1, 1024, 0, st->stream>>>(partials, count, out);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_loglik(State* st, const uint32_t* counts, double* partials,
                        unsigned long long* clamps) {
  const uint64_t N = 1ull << st->n;
  QS_CUDA(cudaMemsetAsync(clamps, 0, sizeof(unsigned long long), st->stream));
  if (st->prec == QS_C64)
    loglik_kernel<float><<<kReduceBlocks, 256, 0, st->stream>>>((const C2<float>*)st->data, counts, N,
                                                                partials, clamps);
  else
    loglik_kernel<double><<<kReduceBlocks, 256, 0, st->stream>>>((const C2<double>*)st->data, counts,
                                                                 N, partials, clamps);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

}  // namespace qs
