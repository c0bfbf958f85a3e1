// Controlled-phase form of a tile-pass diagonal (forward passes only).
#pragma once

#include <cstdint>

#include "internal.h"

namespace qs {

// TK_CP: diagonal diag(1, .., 1, p) (a controlled phase, or a one-qubit phase
// diag(1, p)): the phase p = m0[0] multiplies the amplitudes whose op bits are
// all 1; pad[0] / pad[1] give the position of bit a / b in the thread's context
// word (tile index | 1 << 47 | lane << 48 | warp << 56; bit 47 is the constant 1
// that stands for the missing bit b of a one-qubit phase).
constexpr uint8_t TK_CP = 5;
constexpr int kCtxOne = 47, kCtxLane = 48, kCtxWarp = 56;

// TK_RUN: a run of TK_CP ops of one stage packed by the host into entry lists
// (forward passes only).  Diagonal ops commute, so the run's ops are regrouped by
// where their factor goes: n_s entries whose two bits are both context bits
// (factor into the thread's scalar), then, for register slot k = 0..3, n_f[k]
// entries with one bit in slot k and the other a context bit (factor into the
// slot's factor for bit value 1), then n_rr entries with both bits in register
// slots k and l.  The header op's m0 bytes hold the counts (uint16 n_s, n_f[4],
// n_rr); slot = the number of op slots the entries fill after the header.
constexpr uint8_t TK_RUN = 6;
template <typename R>
struct alignas(8) RunEntry {
  C2<R> p;          // the phase of the ops' all-ones entry
  uint8_t pa, pb;   // context-word positions of the op's bits (pb = kCtxOne for a one-bit op)
  uint8_t k, l;     // register slots (n_rr entries)
  uint8_t pad[4];
};

}  // namespace qs
