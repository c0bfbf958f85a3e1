// Controlled-phase form of a tile-pass diagonal (forward passes only).
#pragma once

#include <cstdint>
#include <vector>

#include "internal.h"

namespace qs {

// TK_CP: diagonal diag(1, .., 1, p) (a controlled phase, or a one-qubit phase
// diag(1, p)): the phase p = m0[0] multiplies the amplitudes whose op bits are
// all 1; pad[0] / pad[1] give the position of bit a / b in the thread's context
// word (tile index | 1 << 47 | lane << 48 | warp << 56; bit 47 is the constant 1
// that stands for the missing bit b of a one-qubit phase).
constexpr uint8_t TK_CP = 5;
constexpr int kCtxOne = 47, kCtxLane = 48, kCtxWarp = 56;

// TK_RUN: a run of TK_CP ops of one stage packed by the host (forward passes
// only).  Diagonal ops commute, so the run's ops are regrouped by what their
// factor depends on; with positions in the context word, a bit is a tile bit
// (< kCtxOne: the same for the whole CTA) or a thread bit (the constant 1, lane or
// warp bits):
//   thread x thread          -> table S over (lane, warp): a factor of the scalar
//   register slot k x thread -> table N_k over (lane, warp): a factor of f_k[1]
//   register x register      -> table RR over the 16 register indices: into v
//   tile x tile              -> one factor of the scalar per CTA (a job)
//   register slot k x tile   -> one factor of f_k[1] per CTA (a job)
//   tile x thread            -> entries each thread applies (n_s, the residual)
// The tables do not depend on the tile: the host builds them (FP64 products,
// rounded once) into the pass's table buffer.  A job's product is formed once per
// CTA in the kernel's prologue from its entries.  Entries follow the header in
// the run's op slots: the residual ones, then the jobs' (slot = the number of op
// slots they fill).  Header fields (in m0):
struct RunHeader {
  uint16_t n_s;        // residual entries (per thread)
  uint16_t n_f[4];     // residual register-slot entries (per thread; jobs that did not fit)
  uint16_t ubase;      // first prologue factor of the run's jobs
  uint8_t umask;       // jobs present: bit 0 scalar, bit 1 + k slot k
  uint8_t tmask;       // tables present: bit 0 S, bit 1 + k N_k, bit 5 RR
  uint32_t toff;       // first table entry (complex index into the pass's table buffer)
};
constexpr uint8_t TK_RUN = 6;
template <typename R>
struct alignas(8) RunEntry {
  C2<R> p;          // the phase of the ops' all-ones entry
  uint8_t pa, pb;   // context-word positions of the op's bits (pb = kCtxOne for a one-bit op)
  uint8_t k, l;     // register slots
  uint8_t pad[4];
};
// A prologue job: the product over count entries of the run whose header is op
// `op`, starting at entry `first`: scalar (both bits tile bits) or slot (pa the
// tile bit); the CTA's factor goes to U[index of the job in the pass].
struct RunJob {
  uint16_t op, first, count;
  uint8_t scalar, pad;
};
constexpr int kMaxRunJobs = 64;
constexpr int kRunTable = 1 << (kLaneBits + kWarpBits);   // (lane, warp) entries of S and N_k

// The kernel-parameter image of one forward tile pass (ops in their TK_CP / TK_RUN
// forms, stage op ranges relative to the pass) and its run tables, as the library
// launches it; offsets in the run headers are relative to the start of tabs.
template <typename R>
void tile_pass_image(const Plan& pl, const TilePass& pass, TileParams<R>* tp, std::vector<C2<R>>& tabs);

}  // namespace qs
