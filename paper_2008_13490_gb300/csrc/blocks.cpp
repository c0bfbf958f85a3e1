// Host fusion of a circuit into dense 5-qubit blocks.
//
// The circuit is an ordered product of gate matrices (section "Quantum
// circuits"); any run of gates whose qubits lie in one set of 5 qubits
// multiplies into one 32x32 unitary.  The planner picks, like the tile planner,
// the gates that are ready (no earlier unapplied gate on a shared qubit) and fit
// in the set, then multiplies them in order into the block.
#include <algorithm>
#include <cstring>

#include "auto_plan.h"
#include "host_par.h"
#include "internal.h"

namespace qs {

namespace {

// U <- G U, G acting on the block-local bits ia (and ib, the less significant
// bit of G's 4x4 local index) of the 32-dimensional block space.  Written out in
// real arithmetic along a row's 32 columns; every complex product is
// (x_re y_re - x_im y_im, x_re y_im + x_im y_re) and the sums run in gate-entry
// order, as the complex-typed expressions would compute them.
void apply_to_block(std::vector<cd>& Uv, const cd* g, int dim, int ia, int ib) {
  double* U = reinterpret_cast<double*>(Uv.data());   // row r: 32 (re, im) pairs from U + 64 r
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
      const double dr = d.real(), di = d.imag();
      double* u = U + 64 * r;
      for (int c = 0; c < 32; ++c) {
        const double ur = u[2 * c], ui = u[2 * c + 1];
        u[2 * c] = ur * dr - ui * di;
        u[2 * c + 1] = ur * di + ui * dr;
      }
    }
    return;
  }
  if (dim == 2) {
    const double g0r = g[0].real(), g0i = g[0].imag(), g1r = g[1].real(), g1i = g[1].imag();
    const double g2r = g[2].real(), g2i = g[2].imag(), g3r = g[3].real(), g3i = g[3].imag();
    for (int r = 0; r < 32; ++r) {
      if ((r >> ia) & 1) continue;
      double* A = U + 64 * r;
      double* B = U + 64 * (r | (1 << ia));
      for (int c = 0; c < 32; ++c) {
        const double ar = A[2 * c], ai = A[2 * c + 1], br = B[2 * c], bi = B[2 * c + 1];
        A[2 * c] = (g0r * ar - g0i * ai) + (g1r * br - g1i * bi);
        A[2 * c + 1] = (g0r * ai + g0i * ar) + (g1r * bi + g1i * br);
        B[2 * c] = (g2r * ar - g2i * ai) + (g3r * br - g3i * bi);
        B[2 * c + 1] = (g2r * ai + g2i * ar) + (g3r * bi + g3i * br);
      }
    }
    return;
  }
  double gr[16], gi[16];
  for (int k = 0; k < 16; ++k) gr[k] = g[k].real(), gi[k] = g[k].imag();
  for (int r = 0; r < 32; ++r) {
    if (((r >> ia) & 1) || ((r >> ib) & 1)) continue;
    double* row[4];
    for (int l = 0; l < 4; ++l) row[l] = U + 64 * (r | ((l >> 1) << ia) | ((l & 1) << ib));
    for (int c = 0; c < 32; ++c) {
      double xr[4], xi[4];
      for (int l = 0; l < 4; ++l) xr[l] = row[l][2 * c], xi[l] = row[l][2 * c + 1];
      for (int o = 0; o < 4; ++o) {
        double sr = 0.0, si = 0.0;
        for (int l = 0; l < 4; ++l) {
          sr += gr[o * 4 + l] * xr[l] - gi[o * 4 + l] * xi[l];
          si += gr[o * 4 + l] * xi[l] + gi[o * 4 + l] * xr[l];
        }
        row[o][2 * c] = sr;
        row[o][2 * c + 1] = si;
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
// precedes.  Stops once every qubit of S is blocked.  rem_m[i] is the qubit mask
// of remaining gate rem[i].
int absorb(const std::vector<uint64_t>& rem_m, const std::vector<size_t>& rem, uint64_t S,
           std::vector<size_t>* sel) {
  uint64_t blocked = 0;
  int cnt = 0;
  for (size_t i = 0; i < rem_m.size(); ++i) {
    const uint64_t qm = rem_m[i];
    if ((qm & blocked) || (qm & ~S)) {
      blocked |= qm;
      if ((blocked & S) == S) break;
      continue;
    }
    ++cnt;
    if (sel) sel->push_back(rem[i]);
  }
  return cnt;
}

// qubit set grown in circuit order from remaining gate `start` (the gates that
// are ready and fit), filled up to 5 with the lowest free qubits
uint64_t grown_set(const std::vector<uint64_t>& rem_m, size_t start, int n) {
  uint64_t S = 0, blocked = 0;
  for (size_t i = start; i < rem_m.size() && __builtin_popcountll(S) < 5; ++i) {
    const uint64_t qm = rem_m[i];
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

// The distinct candidate sets of one block, in first-seen order: a set of nonzero
// qubit masks (at most kSeeds + 60 of them) by open addressing in 256 slots
// (multiplicative hashing), cleared per block.
struct MaskSet {
  uint64_t slot[256];
  MaskSet() { clear(); }
  void clear() { std::memset(slot, 0, sizeof(slot)); }
  bool insert(uint64_t m) {   // true if m was not in the set yet
    unsigned h = (unsigned)((m * 0x9E3779B97F4A7C15ull) >> 56);
    while (slot[h]) {
      if (slot[h] == m) return false;
      h = (h + 1) & 255;
    }
    slot[h] = m;
    return true;
  }
};

// U of block b: the product of its gates, in circuit order
void block_product(const qs_gate* gates, Block& b) {
  b.U.assign(32 * 32, cd(0));
  for (int i = 0; i < 32; ++i) b.U[i * 32 + i] = 1.0;
  auto local = [&](int q) {
    for (int i = 0; i < 5; ++i)
      if (b.q[i] == q) return i;
    return -1;
  };
  for (size_t gi : b.gate_idx) {
    const qs_gate& g = gates[gi];
    cd m[16];
    int dim = 0;
    gate_matrix(g, m, &dim);
    apply_to_block(b.U, m, dim, local(g.q[0]), dim == 4 ? local(g.q[1]) : -1);
  }
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
  std::vector<uint64_t> rem_m(ngates);   // qubit masks of the remaining gates, in the same order
  for (size_t i = 0; i < ngates; ++i) {
    remaining[i] = i;
    rem_m[i] = gate_mask(gates[i]);
  }
  std::vector<uint64_t> cands;
  MaskSet seen;
  while (!remaining.empty()) {
    cands.clear();
    seen.clear();
    for (int k = 0; k < kSeeds && k < (int)remaining.size(); ++k) {
      const uint64_t S = grown_set(rem_m, (size_t)k, n);
      if (seen.insert(S)) cands.push_back(S);
    }
    for (int a = 0; a + 5 <= n; ++a) {
      const uint64_t S = 31ull << a;
      if (seen.insert(S)) cands.push_back(S);
    }
    uint64_t best = cands[0];
    int best_cnt = -1;
    for (uint64_t S : cands) {
      const int c = absorb(rem_m, remaining, S, nullptr);
      if (c > best_cnt) {
        best_cnt = c;
        best = S;
      }
    }
    std::vector<size_t> sel;
    absorb(rem_m, remaining, best, &sel);
    // ascending positions: local bit i of the block = its i-th lowest qubit (the
    // kernel relies on the block qubits among the 4 lowest positions being its
    // lowest local bits)
    Block b;
    for (int q = 0, i = 0; q < n && i < 5; ++q)
      if ((best >> q) & 1) b.q[i++] = q;
    b.ngates = (int)sel.size();
    b.gate_idx = sel;
    out.push_back(std::move(b));
    // the rest, in order (sel is a subsequence of remaining)
    size_t w = 0, j = 0;
    for (size_t i = 0; i < remaining.size(); ++i) {
      if (j < sel.size() && sel[j] == remaining[i]) {
        ++j;
        continue;
      }
      remaining[w] = remaining[i];
      rem_m[w++] = rem_m[i];
    }
    remaining.resize(w);
    rem_m.resize(w);
  }
  // each block's product of its gates (blocks are independent)
  parallel_for(out.size(), 8, [&](size_t bi) { block_product(gates, out[bi]); });
}

bool auto_all_tiles(const qs_gate* gates, size_t ngates, int n, const std::vector<Block>& blocks,
                    std::vector<FOp>* fops, std::vector<int>* vmap) {
  int dense = 0;
  for (const Block& b : blocks) dense += block_nonzeros(b) > 512 ? 1 : 0;
  if (dense < 1 || dense > 2 || dense == (int)blocks.size()) return false;
  // tile passes and remaps of a gate list, fused as the default method fuses it
  auto count = [&](const std::vector<qs_gate>& seg, int* passes, int* remaps) {
    build_fused_ops(seg.data(), seg.size(), n, *fops, *vmap, /*fuse=*/true, /*relabel=*/true);
    Plan pl;
    plan_circuit(*fops, n, *vmap, pl, TileLimits<float>::kMaxOps, kMaxTileStages);
    *passes += (int)pl.passes.size();
    *remaps += (int)pl.remaps.size();
  };
  int seg_passes = 0, seg_remaps = 0;
  for (size_t i = 0; i < blocks.size();) {   // the runs of sparse blocks
    std::vector<qs_gate> seg;
    size_t j = i;
    while (j < blocks.size() && block_nonzeros(blocks[j]) <= 512) {
      for (size_t gi : blocks[j].gate_idx) seg.push_back(gates[gi]);
      ++j;
    }
    if (!seg.empty()) count(seg, &seg_passes, &seg_remaps);
    i = j == i ? i + 1 : j;
  }
  int all_passes = 0, all_remaps = 0;   // the whole circuit (its ops stay in *fops)
  count(std::vector<qs_gate>(gates, gates + ngates), &all_passes, &all_remaps);
  return all_passes <= seg_passes && all_remaps <= seg_remaps;
}

int block_nonzeros(const Block& b) {
  int nz = 0;
  for (const cd& u : b.U) nz += std::abs(u) > 0.0 ? 1 : 0;
  return nz;
}

}  // namespace qs
