// Controlled-phase form of a tile-pass diagonal (forward passes only).
#pragma once

#include <cstdint>

namespace qs {

// TK_CP: diagonal diag(1, .., 1, p) (a controlled phase, or a one-qubit phase
// diag(1, p)): the phase p = m0[0] multiplies the amplitudes whose op bits are
// all 1; pad[0] / pad[1] give the position of bit a / b in the thread's context
// word (tile index | 1 << 47 | lane << 48 | warp << 56; bit 47 is the constant 1
// that stands for the missing bit b of a one-qubit phase).
constexpr uint8_t TK_CP = 5;
constexpr int kCtxOne = 47, kCtxLane = 48, kCtxWarp = 56;

}  // namespace qs
