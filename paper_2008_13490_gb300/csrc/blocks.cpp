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

}  // namespace

void plan_blocks(const qs_gate* gates, size_t ngates, int n, std::vector<Block>& out) {
  out.clear();
  std::vector<size_t> remaining(ngates);
  for (size_t i = 0; i < ngates; ++i) remaining[i] = i;
  while (!remaining.empty()) {
    std::vector<int> S;
    uint64_t Smask = 0, blocked = 0;
    std::vector<size_t> sel, rest;
    for (size_t gi : remaining) {
      const qs_gate& g = gates[gi];
      const int nq = gate_is_two_qubit(g.kind) ? 2 : 1;
      uint64_t qm = 0;
      for (int k = 0; k < nq; ++k) qm |= 1ull << g.q[k];
      if (qm & blocked) {
        blocked |= qm;
        rest.push_back(gi);
        continue;
      }
      const uint64_t need = qm & ~Smask;
      if (__builtin_popcountll(Smask | need) <= 5) {
        for (int k = 0; k < nq; ++k)
          if (need & (1ull << g.q[k])) S.push_back(g.q[k]);
        Smask |= need;
        sel.push_back(gi);
      } else {
        blocked |= qm;
        rest.push_back(gi);
      }
    }
    for (int q = 0; q < n && (int)S.size() < 5; ++q)
      if (!((Smask >> q) & 1)) {
        S.push_back(q);
        Smask |= 1ull << q;
      }
    // ascending positions: local bit i of the block = its i-th lowest qubit (the
    // kernel relies on the block qubits among the 4 lowest positions being its
    // lowest local bits)
    std::sort(S.begin(), S.end());
    Block b;
    for (int i = 0; i < 5; ++i) b.q[i] = S[i];
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
    out.push_back(std::move(b));
    remaining.swap(rest);
  }
}

}  // namespace qs
