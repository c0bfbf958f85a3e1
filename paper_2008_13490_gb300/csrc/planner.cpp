// Host fusion planner: gates -> fused ops -> tile passes (+ plain ops, remaps).
//
// The circuit is the ordered product of gates (section "Quantum circuits").
// The planner only regroups that product where it is exact:
//   * consecutive one-qubit gates on a qubit are multiplied;
//   * diagonal gates (CZ, CP, Z, S, T, R^z, U1, R(k)) are diagonal in the
//     computational basis, so they are evaluated from index bits -- the same
//     idea as the diagonal factors of the thesis's product formula (Eq.
//     (HtotalDecompositionH0DiagonalImplementation)) -- and are folded into a
//     neighbouring one-qubit gate as a choice between two matrices selected by
//     a bit ("controlled" form), moved only across gates they commute with;
//   * CNOT and other block-diagonal two-qubit gates become "choice" gates
//     (target matrix selected by the control bit);
//   * SWAP is a relabeling of qubits; the final layout is restored by remaps.
// A tile pass then applies every op whose non-diagonal qubit lies in a set of
// 12 qubits (the tile) in one read+write of the state.
#include <algorithm>
#include <utility>
#include <cstring>

#include "fuse_merge.h"
#include "internal.h"

namespace qs {

namespace {

constexpr double kTiny = 0.0;   // exact zero tests: gate tables give exact zeros

bool is_zero(cd z) { return z.real() == kTiny && z.imag() == kTiny; }

void mat2_mul(const cd* A, const cd* B, cd* C) {   // C = A B (2x2)
  cd r[4];
  r[0] = A[0] * B[0] + A[1] * B[2];
  r[1] = A[0] * B[1] + A[1] * B[3];
  r[2] = A[2] * B[0] + A[3] * B[2];
  r[3] = A[2] * B[1] + A[3] * B[3];
  for (int i = 0; i < 4; ++i) C[i] = r[i];
}

void diag_mul_right(const cd* U, cd d0, cd d1, cd* out) {   // U diag(d0, d1)
  out[0] = U[0] * d0;
  out[1] = U[1] * d1;
  out[2] = U[2] * d0;
  out[3] = U[3] * d1;
}

void diag_mul_left(cd d0, cd d1, const cd* U, cd* out) {    // diag(d0, d1) U
  out[0] = d0 * U[0];
  out[1] = d0 * U[1];
  out[2] = d1 * U[2];
  out[3] = d1 * U[3];
}

uint64_t nd_mask(const FOp& o) {
  switch (o.type) {
    case F_G1: case F_G1C: return 1ull << o.t;
    case F_G2: return (1ull << o.a) | (1ull << o.b);
    default: return 0;
  }
}

uint64_t d_mask(const FOp& o) {
  switch (o.type) {
    case F_G1C: return 1ull << o.c;
    case F_D: return (1ull << o.a) | (o.b >= 0 ? (1ull << o.b) : 0);
    default: return 0;
  }
}

// diagonal entries of a one-qubit D op or of the part of a two-qubit D op
// acting on `t` when the other qubit's bit is v.
void d_restrict(const FOp& D, int t, int v, cd* d0, cd* d1) {
  if (D.b < 0) {
    *d0 = D.d[0];
    *d1 = D.d[1];
  } else if (t == D.a) {
    *d0 = D.d[0 * 2 + v];
    *d1 = D.d[1 * 2 + v];
  } else {
    *d0 = D.d[v * 2 + 0];
    *d1 = D.d[v * 2 + 1];
  }
}

// Try to fold diagonal op D into G (a G1 or G1C acting non-diagonally on a
// qubit of D).  after = true: D acts after G (D G); else D acts before G (G D).
bool fold_into(const FOp& D, FOp& G, bool after) {
  int t = G.t;
  bool t_in = (t == D.a) || (t == D.b);
  if (!t_in) return false;
  int other = (D.b < 0) ? -1 : (t == D.a ? D.b : D.a);
  if (G.type == F_G1) {
    if (other < 0) {
      cd d0, d1;
      d_restrict(D, t, 0, &d0, &d1);
      if (after) diag_mul_left(d0, d1, G.m0, G.m0);
      else diag_mul_right(G.m0, d0, d1, G.m0);
      return true;
    }
    cd U[4];
    for (int i = 0; i < 4; ++i) U[i] = G.m0[i];
    for (int v = 0; v < 2; ++v) {
      cd d0, d1;
      d_restrict(D, t, v, &d0, &d1);
      cd* M = v ? G.m1 : G.m0;
      if (after) diag_mul_left(d0, d1, U, M);
      else diag_mul_right(U, d0, d1, M);
    }
    G.type = F_G1C;
    G.c = other;
    return true;
  }
  if (G.type == F_G1C) {
    if (other >= 0 && other != G.c) return false;
    for (int v = 0; v < 2; ++v) {
      cd d0, d1;
      d_restrict(D, t, other < 0 ? 0 : v, &d0, &d1);
      cd* M = v ? G.m1 : G.m0;
      if (after) diag_mul_left(d0, d1, M, M);
      else diag_mul_right(M, d0, d1, M);
    }
    return true;
  }
  return false;
}

}  // namespace

void build_fused_ops(const qs_gate* gates, size_t ngates, int n, std::vector<FOp>& out,
                     std::vector<int>& vmap_out, bool fuse, bool relabel) {
  out.clear();
  out.reserve(ngates);
  std::vector<int> cur(n);
  for (int q = 0; q < n; ++q) cur[q] = q;
  for (size_t i = 0; i < ngates; ++i) {
    const qs_gate& g = gates[i];
    cd m[16];
    int dim = 0;
    gate_matrix(g, m, &dim);
    if (dim != 2 && g.kind == QS_SWAP && relabel) {
      std::swap(cur[g.q[0]], cur[g.q[1]]);
      continue;
    }
    FOp& o = out.emplace_back();   // built in place
    if (dim == 2) {
      int v = cur[g.q[0]];
      if (is_zero(m[1]) && is_zero(m[2])) {
        o.type = F_D;
        o.a = v;
        o.b = -1;
        o.d[0] = m[0];
        o.d[1] = m[3];
      } else {
        o.type = F_G1;
        o.t = v;
        for (int k = 0; k < 4; ++k) o.m0[k] = m[k];
      }
      continue;
    }
    int v0 = cur[g.q[0]], v1 = cur[g.q[1]];
    bool diag = true, blk0 = true, blk1 = true;
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        if (is_zero(m[4 * r + c])) continue;
        if (r != c) diag = false;
        if ((r >> 1) != (c >> 1)) blk0 = false;   // block-diagonal in qubit 0 (msb)
        if ((r & 1) != (c & 1)) blk1 = false;     // block-diagonal in qubit 1 (lsb)
      }
    if (diag) {
      o.type = F_D;
      o.a = v0;
      o.b = v1;
      for (int k = 0; k < 4; ++k) o.d[k] = m[5 * k];
    } else if (blk0) {   // target q1, choice q0
      o.type = F_G1C;
      o.t = v1;
      o.c = v0;
      o.m0[0] = m[0]; o.m0[1] = m[1]; o.m0[2] = m[4]; o.m0[3] = m[5];
      o.m1[0] = m[10]; o.m1[1] = m[11]; o.m1[2] = m[14]; o.m1[3] = m[15];
    } else if (blk1) {   // target q0, choice q1
      o.type = F_G1C;
      o.t = v0;
      o.c = v1;
      o.m0[0] = m[0]; o.m0[1] = m[2]; o.m0[2] = m[8]; o.m0[3] = m[10];
      o.m1[0] = m[5]; o.m1[1] = m[7]; o.m1[2] = m[13]; o.m1[3] = m[15];
    } else {
      o.type = F_G2;
      o.a = v0;
      o.b = v1;
      for (int k = 0; k < 16; ++k) o.g[k] = m[k];
    }
    if (o.type == F_G1C) {
      bool same = true;
      for (int k = 0; k < 4; ++k) same = same && (o.m0[k] == o.m1[k]);
      if (same) {
        o.type = F_G1;
        o.c = -1;
      }
    }
  }
  vmap_out = cur;
  if (!fuse) return;

  // (1) multiply runs of one-qubit ops (G1 / one-qubit D) on the same qubit;
  // the merged list is compacted in place (it never runs ahead of the input)
  {
    size_t w = 0;
    std::vector<int> last1(n, -1);   // index in the merged prefix of the open one-qubit op on q
    for (size_t i = 0; i < out.size(); ++i) {
      const FOp& o = out[i];
      bool one_q = (o.type == F_G1) || (o.type == F_D && o.b < 0);
      if (one_q) {
        int q = (o.type == F_G1) ? o.t : o.a;
        int j = last1[q];
        if (j >= 0) {
          FOp& p = out[j];
          cd A[4], B[4];
          if (p.type == F_G1) for (int k = 0; k < 4; ++k) A[k] = p.m0[k];
          else { A[0] = p.d[0]; A[1] = 0; A[2] = 0; A[3] = p.d[1]; }
          if (o.type == F_G1) for (int k = 0; k < 4; ++k) B[k] = o.m0[k];
          else { B[0] = o.d[0]; B[1] = 0; B[2] = 0; B[3] = o.d[1]; }
          cd C[4];
          mat2_mul(B, A, C);   // later op on the left
          if (is_zero(C[1]) && is_zero(C[2])) {
            p.type = F_D; p.a = q; p.b = -1; p.t = -1; p.d[0] = C[0]; p.d[1] = C[3];
          } else {
            p.type = F_G1; p.t = q; p.a = -1; for (int k = 0; k < 4; ++k) p.m0[k] = C[k];
          }
          continue;
        }
        if (w != i) out[w] = o;
        last1[q] = (int)w++;
        continue;
      }
      uint64_t touched = nd_mask(o) | d_mask(o);
      for (int q = 0; q < n; ++q)
        if ((touched >> q) & 1) last1[q] = -1;
      if (w != i) out[w] = o;
      ++w;
    }
    out.resize(w);
  }

  // (2) fold diagonal ops into a neighbouring non-diagonal one-qubit op: the
  // nearest op in each direction that does not commute with D (one acting
  // non-diagonally on a qubit of D) is the only candidate.  The scans read the
  // ops' non-diagonal qubit masks, which folding leaves unchanged.
  bool any_diag = false;
  for (const FOp& o : out) any_diag = any_diag || o.type == F_D;
  if (any_diag) {
    std::vector<char> dead(out.size(), 0);
    // per qubit, in increasing order, the ops acting non-diagonally on it (diagonal
    // ops, folded or not, are in none of the lists)
    std::vector<std::vector<int>> on(n);
    for (size_t i = 0; i < out.size(); ++i) {
      const uint64_t m = nd_mask(out[i]);
      for (int q = 0; q < n; ++q)
        if ((m >> q) & 1) on[q].push_back((int)i);
    }
    for (size_t i = 0; i < out.size(); ++i) {
      if (out[i].type != F_D) continue;
      const FOp D = out[i];
      const int qa = D.a, qb = D.b;
      // the nearest ops after and before D on D's qubits
      int after = -1, before = -1;
      for (int q : {qa, qb}) {
        if (q < 0) continue;
        const std::vector<int>& L = on[q];
        auto it = std::upper_bound(L.begin(), L.end(), (int)i);
        if (it != L.end() && (after < 0 || *it < after)) after = *it;
        auto jt = std::lower_bound(L.begin(), L.end(), (int)i);
        if (jt != L.begin() && *(jt - 1) > before) before = *(jt - 1);
      }
      bool done = after >= 0 && fold_into(D, out[(size_t)after], /*after=*/false);
      if (!done && before >= 0) done = fold_into(D, out[(size_t)before], /*after=*/true);
      if (done) dead[i] = 1;
    }
    size_t w = 0;
    for (size_t i = 0; i < out.size(); ++i)
      if (!dead[i]) {
        if (w != i) out[w] = out[i];
        ++w;
      }
    out.resize(w);
  }
}

void mark_one_qubit_merges(std::vector<FOp>& ops, int n, std::vector<int>* into_out) {
  const size_t m = ops.size();
  std::vector<int>& into = *into_out;   // input op -> the later op it was merged into
  into.assign(m, -1);
  std::vector<int> open(n, -1);   // per target qubit: the movable one-qubit op, or -1
  std::vector<int> open_c(n, -1); // its choice bit (-1: none)
  uint64_t open_mask = 0;         // targets with a movable op
  for (size_t i = 0; i < m; ++i) {
    FOp& Y = ops[i];
    const bool one = (Y.type == F_G1 || Y.type == F_G1C) && Y.term < 0;
    const int t = one ? Y.t : -1;
    // Y fixes the ops on every qubit it touches (but for a merge partner on its own
    // target) and those whose choice bit it changes
    const uint64_t nd = nd_mask(Y), touched = nd | d_mask(Y);
    for (uint64_t cand = open_mask & ~(t >= 0 ? 1ull << t : 0ull); cand; cand &= cand - 1) {
      const int q = __builtin_ctzll(cand);
      if (((touched >> q) & 1) || (open_c[q] >= 0 && ((nd >> open_c[q]) & 1))) {
        open[q] = -1;
        open_mask &= ~(1ull << q);
      }
    }
    if (!one) continue;   // (a term op is in its own touched set: its target is closed)
    const int x = open[t];
    if (x >= 0) {
      FOp& X = ops[(size_t)x];
      const int cx = X.type == F_G1C ? X.c : -1, cy = Y.type == F_G1C ? Y.c : -1;
      if (cx < 0 || cy < 0 || cx == cy) {
        const int c = cy >= 0 ? cy : cx;
        cd C0[4], C1[4];
        mat2_mul(Y.m0, X.m0, C0);   // the later op on the left
        if (c >= 0) mat2_mul(cy >= 0 ? Y.m1 : Y.m0, cx >= 0 ? X.m1 : X.m0, C1);
        for (int k = 0; k < 4; ++k) {
          Y.m0[k] = C0[k];
          Y.m1[k] = c >= 0 ? C1[k] : cd(0);
        }
        if (c >= 0) {
          Y.type = F_G1C;
          Y.c = c;
        }
        into[(size_t)x] = (int)i;
      }
    }
    open[t] = (int)i;
    open_c[t] = Y.type == F_G1C ? Y.c : -1;
    open_mask |= 1ull << t;
  }
}

void merge_one_qubit_ops(std::vector<FOp>& ops, int n, std::vector<int>* group) {
  const size_t m = ops.size();
  std::vector<int> into;
  mark_one_qubit_merges(ops, n, &into);
  // compact; inputs follow their merge chains to the op that survives
  std::vector<int> pos(m, -1);
  size_t w = 0;
  for (size_t i = 0; i < m; ++i)
    if (into[i] < 0) {
      pos[i] = (int)w;
      if (w != i) ops[w] = ops[i];
      ++w;
    }
  if (group) {
    group->assign(m, -1);
    for (size_t i = m; i-- > 0;) (*group)[i] = into[i] < 0 ? pos[i] : (*group)[(size_t)into[i]];
  }
  ops.resize(w);
}

// ---------------------------------------------------------------------------
// tile-pass planning
// ---------------------------------------------------------------------------

namespace {

struct Encoder {
  // physical layout for the pass
  int n;
  uint8_t pos[kTileBits];
  int local_of_phys[64];   // -1 if not in tile
  int nt_rank[64];         // rank among non-tile positions
  const int* l2p;          // virtual -> physical
  int reg[kRegBits];
  int warp[kWarpBits];

  void src_of(int v, uint8_t* src, uint8_t* bit) const {
    int p = l2p[v];
    int loc = local_of_phys[p];
    if (loc < 0) {
      *src = CS_TILE;
      *bit = (uint8_t)nt_rank[p];
      return;
    }
    if (loc < kLaneBits) {
      *src = CS_LANE;
      *bit = (uint8_t)loc;
      return;
    }
    for (int k = 0; k < kRegBits; ++k)
      if (reg[k] == loc) {
        *src = CS_REG;
        *bit = (uint8_t)k;
        return;
      }
    for (int k = 0; k < kWarpBits; ++k)
      if (warp[k] == loc) {
        *src = CS_WARP;
        *bit = (uint8_t)k;
        return;
      }
    *src = CS_NONE;
    *bit = 0;
  }
};

int popc(uint64_t x) { return __builtin_popcountll(x); }

}  // namespace

void plan_circuit(const std::vector<FOp>& ops, int n, const std::vector<int>& vmap_final,
                  Plan& plan, int max_ops_per_pass, int max_stages_per_pass) {
  plan = Plan{};
  std::vector<int> l2p(n), p2l(n);
  for (int q = 0; q < n; ++q) l2p[q] = p2l[q] = q;

  std::vector<int> remaining;
  remaining.reserve(ops.size());
  for (size_t i = 0; i < ops.size(); ++i) remaining.push_back((int)i);

  const int kLow = 2;   // physical bits always in a tile (contiguous 32-byte sectors)
  // plans of adjoint sweeps (ops with derivative terms) keep every op as it is
  bool merge = true;
  for (const FOp& o : ops) merge = merge && o.term < 0;

  while (!remaining.empty()) {
    // ---- choose the tile's qubits and the ops of this pass (a dense two-qubit
    // op takes two op slots: its 16 entries span two tile ops).  The ops of a pass
    // are, in order, those whose non-diagonal qubits lie in the tile set and that
    // no skipped earlier op conflicts with.  Candidate tile sets: the set grown
    // from the ops in the order they become ready, and every window of
    // consecutive qubits (with the qubits at the low physical positions, which
    // every tile holds); a window keeps the deep light cone of a nearest-neighbour
    // circuit (the 30-qubit layered circuit: 20 passes instead of 47).  The
    // candidate that takes the most ops wins (ties: the grown set).
    uint64_t low = 0;
    for (int p = 0; p < kLow; ++p) low |= 1ull << p2l[p];
    // fixed == 0: grow the set from `low`; otherwise the set is `fixed`
    auto select = [&](uint64_t fixed, std::vector<int>* sel_out, std::vector<int>* rest_out) {
      uint64_t T = fixed ? fixed : low;
      uint64_t nd_blk = 0, d_blk = 0;
      int slots_used = 0;
      for (int idx : remaining) {
        const FOp& o = ops[idx];
        uint64_t ndq = nd_mask(o), dq = d_mask(o);
        bool conflict = (ndq & (nd_blk | d_blk)) || (dq & nd_blk);
        const int cost = o.type == F_G2 ? 2 : 1;
        if (!conflict && slots_used + cost <= max_ops_per_pass) {
          uint64_t need = ndq & ~T;
          if (fixed ? need == 0 : popc(T | need) <= kTileBits) {
            T |= need;
            if (sel_out) sel_out->push_back(idx);
            slots_used += cost;
            continue;
          }
        }
        nd_blk |= ndq;
        d_blk |= dq;
        if (rest_out) rest_out->push_back(idx);
      }
      return std::make_pair(slots_used, T);
    };
    uint64_t best_set = 0;
    int best = select(0, nullptr, nullptr).first;
    for (int a = 0; a < n; ++a) {
      uint64_t W = low;
      for (int q = a; q < n && popc(W) < kTileBits; ++q) W |= 1ull << q;
      for (int q = a - 1; q >= 0 && popc(W) < kTileBits; --q) W |= 1ull << q;
      const int c = select(W, nullptr, nullptr).first;
      if (c > best) {
        best = c;
        best_set = W;
      }
    }
    std::vector<int> sel;
    std::vector<int> rest;
    uint64_t T = select(best_set, &sel, &rest).second;
    // fill the tile up to kTileBits with the lowest remaining physical positions
    for (int p = 0; p < n && popc(T) < kTileBits; ++p) T |= 1ull << p2l[p];

    // ---- layout
    Encoder enc{};
    enc.n = n;
    enc.l2p = l2p.data();
    for (int p = 0; p < 64; ++p) enc.local_of_phys[p] = -1, enc.nt_rank[p] = -1;
    TilePass tp{};
    {
      int k = 0, r = 0;
      for (int p = 0; p < n; ++p) {
        if ((T >> p2l[p]) & 1) {
          enc.pos[k] = (uint8_t)p;
          tp.pos[k] = (uint8_t)p;
          enc.local_of_phys[p] = k++;
        } else {
          tp.nt_pos[r] = (uint8_t)p;
          enc.nt_rank[p] = r++;
        }
      }
      tp.n_nt = r;
    }
    tp.stage_begin = (int)plan.stages.size();

    // ---- the pass's ops, one-qubit ops on a target merged inside the pass (its
    // ops commute with every op deferred to a later pass, so they form a program
    // of their own); grp[j] = the merged op that op sel[j] went into
    std::vector<FOp> pv;
    pv.reserve(sel.size());
    for (int idx : sel) pv.push_back(ops[idx]);
    std::vector<int> grp(sel.size());
    if (merge) merge_one_qubit_ops(pv, n, &grp);
    else
      for (size_t j = 0; j < sel.size(); ++j) grp[j] = (int)j;

    // ---- stages
    std::vector<int> pending(pv.size());
    for (size_t k = 0; k < pv.size(); ++k) pending[k] = (int)k;
    while (!pending.empty()) {
      if ((int)plan.stages.size() - tp.stage_begin >= max_stages_per_pass) {
        // stage budget of the pass used up: the rest waits for the next pass as
        // the original ops it was made of (merging by op index keeps program order)
        for (int k : pending)
          for (size_t j = 0; j < sel.size(); ++j)
            if (grp[j] == k) rest.push_back(sel[j]);
        std::sort(rest.begin(), rest.end());
        break;
      }
      int R[kRegBits];
      int nR = 0;
      uint64_t snd = 0, sd = 0;
      std::vector<int> stage_ops, later;
      for (int idx : pending) {
        const FOp& o = pv[idx];
        uint64_t ndq = nd_mask(o), dq = d_mask(o);
        bool conflict = (ndq & (snd | sd)) || (dq & snd);
        bool ok = false;
        if (!conflict && o.type == F_G2) {
          // both qubits on lanes or in this stage's registers
          const int la = enc.local_of_phys[l2p[o.a]], lb = enc.local_of_phys[l2p[o.b]];
          int add[2], na = 0;
          for (int loc : {la, lb}) {
            if (loc < kLaneBits) continue;
            bool in = false;
            for (int k = 0; k < nR; ++k) in = in || (R[k] == loc);
            if (!in) add[na++] = loc;
          }
          if (nR + na <= kRegBits) {
            for (int k = 0; k < na; ++k) R[nR++] = add[k];
            ok = true;
          }
        } else if (!conflict) {
          if (o.type == F_D) {
            ok = true;
          } else {
            int loc = enc.local_of_phys[l2p[o.t]];
            if (loc < kLaneBits) {
              ok = true;
            } else {
              bool in = false;
              for (int k = 0; k < nR; ++k) in = in || (R[k] == loc);
              if (in) ok = true;
              else if (nR < kRegBits) {
                R[nR++] = loc;
                ok = true;
              }
            }
          }
        }
        if (ok) stage_ops.push_back(idx);
        else {
          snd |= ndq;
          sd |= dq;
          later.push_back(idx);
        }
      }
      // complete the register set (prefer targets needed next)
      for (int idx : later) {
        if (nR >= kRegBits) break;
        const FOp& o = pv[idx];
        if (o.type == F_D) continue;
        for (int v : {o.type == F_G2 ? o.a : o.t, o.type == F_G2 ? o.b : -1}) {
          if (v < 0 || nR >= kRegBits) continue;
          int loc = enc.local_of_phys[l2p[v]];
          if (loc < kLaneBits) continue;
          bool in = false;
          for (int k = 0; k < nR; ++k) in = in || (R[k] == loc);
          if (!in) R[nR++] = loc;
        }
      }
      for (int loc = kLaneBits; loc < kTileBits && nR < kRegBits; ++loc) {
        bool in = false;
        for (int k = 0; k < nR; ++k) in = in || (R[k] == loc);
        if (!in) R[nR++] = loc;
      }
      TileStage ts{};
      for (int k = 0; k < kRegBits; ++k) ts.reg[k] = (uint8_t)R[k], enc.reg[k] = R[k];
      {
        int w = 0;
        for (int loc = kLaneBits; loc < kTileBits; ++loc) {
          bool in = false;
          for (int k = 0; k < kRegBits; ++k) in = in || (R[k] == loc);
          if (!in) {
            ts.warp[w] = (uint8_t)loc;
            enc.warp[w++] = loc;
          }
        }
      }
      ts.op_begin = (int)plan.tile_fops.size();
      for (int idx : stage_ops) {
        const FOp& o = pv[idx];
        uint8_t kind = TK_DIAG, slot = 0, csrc = CS_NONE, cbit = 0, dsrc = CS_NONE, dbit = 0;
        if (o.type == F_G2) {
          // sources (lane or register) of qubit a (local index msb) and b; the op's
          // 16 entries continue in a second tile op (TK_G2C)
          enc.src_of(o.a, &csrc, &cbit);
          enc.src_of(o.b, &dsrc, &dbit);
          for (int part = 0; part < 2; ++part) {
            plan.tile_fops.push_back(o);
            plan.tile_kind.push_back(part ? TK_G2C : TK_G2);
            plan.tile_slot.push_back(0);
            plan.tile_csrc.push_back(csrc);
            plan.tile_cbit.push_back(cbit);
            plan.tile_dsrc.push_back(dsrc);
            plan.tile_dbit.push_back(dbit);
          }
          continue;
        }
        if (o.type == F_D) {
          enc.src_of(o.a, &csrc, &cbit);
          if (o.b >= 0) enc.src_of(o.b, &dsrc, &dbit);
        } else {
          int loc = enc.local_of_phys[l2p[o.t]];
          if (loc < kLaneBits) {
            kind = TK_LANE;
            slot = (uint8_t)loc;
          } else {
            kind = TK_REG;
            for (int k = 0; k < kRegBits; ++k)
              if (R[k] == loc) slot = (uint8_t)k;
          }
          if (o.type == F_G1C) enc.src_of(o.c, &csrc, &cbit);
        }
        plan.tile_fops.push_back(o);
        plan.tile_kind.push_back(kind);
        plan.tile_slot.push_back(slot);
        plan.tile_csrc.push_back(csrc);
        plan.tile_cbit.push_back(cbit);
        plan.tile_dsrc.push_back(dsrc);
        plan.tile_dbit.push_back(dbit);
      }
      ts.op_end = (int)plan.tile_fops.size();
      plan.stages.push_back(ts);
      pending.swap(later);
    }
    tp.n_stages = (int)plan.stages.size() - tp.stage_begin;
    plan.passes.push_back(tp);
    plan.steps.push_back({PlanStep::TILE, (int)plan.passes.size() - 1});
    remaining.swap(rest);
  }

  // ---- restore the canonical layout: logical q must sit at physical q.
  // Virtual vmap_final[q] holds logical q and sits at physical l2p[...].
  std::vector<int> where(n);   // where[q] = current physical position of logical q
  for (int q = 0; q < n; ++q) where[q] = l2p[vmap_final[q]];
  for (int guard = 0; guard < 4 * n + 8; ++guard) {
    bool ok = true;
    for (int q = 0; q < n; ++q) ok = ok && (where[q] == q);
    if (ok) break;
    // content at physical p is logical who[p]; it must move to physical who[p]
    std::vector<int> who(n);
    for (int q = 0; q < n; ++q) who[where[q]] = q;
    // positions taking part; the two lowest stay in for contiguous sectors
    uint64_t S = 3;
    std::vector<char> seen(n, 0);
    for (int p = 0; p < n; ++p) {
      if (seen[p] || who[p] == p) continue;
      std::vector<int> cyc;
      int x = p;
      while (!seen[x]) {
        seen[x] = 1;
        cyc.push_back(x);
        x = who[x];   // content of x goes to who[x]
      }
      uint64_t cm = 0;
      for (int y : cyc) cm |= 1ull << y;
      int room = kTileBits - popc(S);
      if (popc(cm & ~S) <= room) {
        S |= cm;
      } else {
        // a prefix of the cycle: all but its last element land correctly
        for (int y : cyc) {
          if (popc(S) >= kTileBits) break;
          S |= 1ull << y;
        }
      }
    }
    // low positions keep loads/stores contiguous: fill with the lowest ones
    for (int p = 0; p < n && popc(S) < kTileBits; ++p) S |= 1ull << p;
    RemapDesc rd{};
    int k = 0, r = 0;
    int loc[64];
    for (int p = 0; p < n; ++p) {
      if ((S >> p) & 1) {
        rd.pos[k] = (uint8_t)p;
        loc[p] = k++;
      } else {
        rd.nt_pos[r++] = (uint8_t)p;
        loc[p] = -1;
      }
    }
    rd.n_t = k;
    rd.n_nt = r;
    // destination inside S for every source position in S
    std::vector<int> dest(n, -1);
    std::vector<char> taken(n, 0);
    for (int p = 0; p < n; ++p)
      if (((S >> p) & 1) && ((S >> who[p]) & 1)) {
        dest[p] = who[p];
        taken[who[p]] = 1;
      }
    for (int p = 0; p < n; ++p)
      if (((S >> p) & 1) && dest[p] < 0) {
        for (int t = 0; t < n; ++t)
          if (((S >> t) & 1) && !taken[t]) {
            dest[p] = t;
            taken[t] = 1;
            break;
          }
      }
    // src_of_out: the remap kernel reads local in-bit src[j] for out-local bit j
    for (int p = 0; p < n; ++p)
      if ((S >> p) & 1) rd.src[loc[dest[p]]] = (uint8_t)loc[p];
    plan.remaps.push_back(rd);
    plan.steps.push_back({PlanStep::REMAP, (int)plan.remaps.size() - 1});
    std::vector<int> nw(n);
    for (int q = 0; q < n; ++q) {
      int p = where[q];
      nw[q] = ((S >> p) & 1) ? dest[p] : p;
    }
    where.swap(nw);
  }
  plan.n_ops = (int64_t)ops.size();
}

}  // namespace qs
