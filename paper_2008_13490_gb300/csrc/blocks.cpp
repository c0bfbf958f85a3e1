// Host fusion of a circuit into dense 5-qubit blocks.
//
// The circuit is an ordered product of gate matrices (section "Quantum
// circuits"); any run of gates whose qubits lie in one set of 5 qubits
// multiplies into one 32x32 unitary.  The planner picks, like the tile planner,
// the gates that are ready (no earlier unapplied gate on a shared qubit) and fit
// in the set, then multiplies them in order into the block.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace qs {

namespace {

// U <- G U, G acting on the block-local bits ia (and ib, the less significant
// bit of G's 4x4 local index) of the 32-dimensional block space.
void apply_to_block(std::vector<cd>& U, const cd* g, int dim, int ia, int ib) {
  // a diagonal gate scales rows (entries exactly 1 leave them alone)
  bool diag = true;
  for (int o = 0; o < dim; ++o)
    for (int l = 0; l < dim; ++l)
      if (o != l && g[o * dim + l] != cd(0)) diag = false;
  if (diag) {
    for (int r = 0; r < 32; ++r) {
      const int l = dim == 2 ? ((r >> ia) & 1) : (((r >> ia) & 1) << 1) | ((r >> ib) & 1);
      const cd d = g[l * dim + l];
      if (d == cd(1)) continue;
      for (int c = 0; c < 32; ++c) U[r * 32 + c] *= d;
    }
    return;
  }
  if (dim == 2) {
    for (int r = 0; r < 32; ++r) {
      if ((r >> ia) & 1) continue;
      const int r1 = r | (1 << ia);
      for (int c = 0; c < 32; ++c) {
        const cd a = U[r * 32 + c], b = U[r1 * 32 + c];
        U[r * 32 + c] = g[0] * a + g[1] * b;
        U[r1 * 32 + c] = g[2] * a + g[3] * b;
      }
    }
    return;
  }
  for (int r = 0; r < 32; ++r) {
    if (((r >> ia) & 1) || ((r >> ib) & 1)) continue;
    int idx[4];
    for (int l = 0; l < 4; ++l) idx[l] = r | ((l >> 1) << ia) | ((l & 1) << ib);
    for (int c = 0; c < 32; ++c) {
      cd x[4];
      for (int l = 0; l < 4; ++l) x[l] = U[idx[l] * 32 + c];
      for (int o = 0; o < 4; ++o) {
        cd acc = 0;
        for (int l = 0; l < 4; ++l) acc += g[o * 4 + l] * x[l];
        U[idx[o] * 32 + c] = acc;
      }
    }
  }
}

uint64_t gate_mask(const qs_gate& g) {
  uint64_t m = 1ull << g.q[0];
  if (gate_is_two_qubit(g.kind)) m |= 1ull << g.q[1];
  return m;
}

// The gates a block on qubit set S absorbs: in circuit order, every remaining gate
// whose qubits lie in S and that no skipped earlier gate on a shared qubit
// precedes.  Stops once every qubit of S is blocked.
int absorb(const qs_gate* gates, const std::vector<size_t>& rem, uint64_t S, std::vector<size_t>* sel) {
  uint64_t blocked = 0;
  int cnt = 0;
  for (size_t gi : rem) {
    const uint64_t qm = gate_mask(gates[gi]);
    if ((qm & blocked) || (qm & ~S)) {
      blocked |= qm;
      if ((blocked & S) == S) break;
      continue;
    }
    ++cnt;
    if (sel) sel->push_back(gi);
  }
  return cnt;
}

// qubit set grown in circuit order from remaining gate `start` (the gates that
// are ready and fit), filled up to 5 with the lowest free qubits
uint64_t grown_set(const qs_gate* gates, const std::vector<size_t>& rem, size_t start, int n) {
  uint64_t S = 0, blocked = 0;
  for (size_t i = start; i < rem.size() && __builtin_popcountll(S) < 5; ++i) {
    const uint64_t qm = gate_mask(gates[rem[i]]);
    if (qm & blocked) {
      blocked |= qm;
      continue;
    }
    if (__builtin_popcountll(S | qm) <= 5) S |= qm;
    else blocked |= qm;
  }
  for (int q = 0; q < n && __builtin_popcountll(S) < 5; ++q) S |= 1ull << q;
  return S;
}

}  // namespace

// Each block takes, among candidate qubit sets, the one that absorbs the most
// remaining gates (ties: the first candidate): the sets grown from each of the
// first kSeeds remaining gates, and every window of 5 consecutive qubits (the
// light cones of nearest-neighbour circuits).  On 40 layers of Haar + brickwork
// CZ at 30 qubits this gives 100 blocks where growing from the first remaining
// gate alone gives 148.
void plan_blocks(const qs_gate* gates, size_t ngates, int n, std::vector<Block>& out) {
  constexpr int kSeeds = 64;
  out.clear();
  std::vector<size_t> remaining(ngates);
  for (size_t i = 0; i < ngates; ++i) remaining[i] = i;
  std::vector<uint64_t> cands;
  while (!remaining.empty()) {
    cands.clear();
    for (int k = 0; k < kSeeds && k < (int)remaining.size(); ++k) {
      const uint64_t S = grown_set(gates, remaining, (size_t)k, n);
      if (std::find(cands.begin(), cands.end(), S) == cands.end()) cands.push_back(S);
    }
    for (int a = 0; a + 5 <= n; ++a) {
      const uint64_t S = 31ull << a;
      if (std::find(cands.begin(), cands.end(), S) == cands.end()) cands.push_back(S);
    }
    uint64_t best = cands[0];
    int best_cnt = -1;
    for (uint64_t S : cands) {
      const int c = absorb(gates, remaining, S, nullptr);
      if (c > best_cnt) {
        best_cnt = c;
        best = S;
      }
    }
    std::vector<size_t> sel;
    absorb(gates, remaining, best, &sel);
    // ascending positions: local bit i of the block = its i-th lowest qubit (the
    // kernel relies on the block qubits among the 4 lowest positions being its
    // lowest local bits)
    Block b;
    for (int q = 0, i = 0; q < n && i < 5; ++q)
      if ((best >> q) & 1) b.q[i++] = q;
    b.U.assign(32 * 32, cd(0));
    for (int i = 0; i < 32; ++i) b.U[i * 32 + i] = 1.0;
    for (size_t gi : sel) {
      const qs_gate& g = gates[gi];
      cd m[16];
      int dim = 0;
      gate_matrix(g, m, &dim);
      auto local = [&](int q) {
        for (int i = 0; i < 5; ++i)
          if (b.q[i] == q) return i;
        return -1;
      };
      apply_to_block(b.U, m, dim, local(g.q[0]), dim == 4 ? local(g.q[1]) : -1);
    }
    b.ngates = (int)sel.size();
    b.gate_idx = sel;
    out.push_back(std::move(b));
    // the rest, in order (sel is a subsequence of remaining)
    std::vector<size_t> rest;
    rest.reserve(remaining.size() - sel.size());
    size_t j = 0;
    for (size_t gi : remaining) {
      if (j < sel.size() && sel[j] == gi) {
        ++j;
        continue;
      }
      rest.push_back(gi);
    }
    remaining.swap(rest);
  }
}

int block_nonzeros(const Block& b) {
  int nz = 0;
  for (const cd& u : b.U) nz += std::abs(u) > 0.0 ? 1 : 0;
  return nz;
}

}  // namespace qs
