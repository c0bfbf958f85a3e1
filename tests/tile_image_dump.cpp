// Writes, as text, the kernel-parameter images the library launches for the tile
// passes of a gate list (complex128 images, host side only):
// usage: tile_image_dump gates.bin n fuse relabel out.txt.
// Sections (one record per line, numbers separated by blanks):
//   steps K     / kind index                        (0 tile, 1 plain, 2 remap)
//   pass i S J T / n_nt pos[12] nt_pos[n_nt]        (S stages, J prologue jobs, T table entries)
//     stage      / reg[4] warp[3] op_begin op_end
//     op         / index kind slot csrc cbit dsrc dbit pad[0] pad[1] then m0, m1 (4 complex each)
//     run        / index n_s n_f[4] ubase umask tmask toff count, then count entries
//     entry      / re im pa pb k l
//     job        / op first count scalar
//     tab        / re im
//   plainops Q  / type t c a b then m0, m1, d, g     (as tile_plan_dump)
//   remaps R    / pos[12] src[12] n_nt nt_pos[n_nt]
// Built against the library by test_tile_planner.py.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <vector>

#include "internal.h"
#include "tile_cp.h"

using namespace qs;

static void put_c(FILE* o, const cd* v, int k) {
  for (int i = 0; i < k; ++i) std::fprintf(o, " %.17g %.17g", v[i].real(), v[i].imag());
}
static void put_c2(FILE* o, const C2<double>* v, int k) {
  for (int i = 0; i < k; ++i) std::fprintf(o, " %.17g %.17g", v[i].x, v[i].y);
}

int main(int argc, char** argv) {
  if (argc != 6) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  std::vector<qs_gate> g;
  qs_gate one;
  while (std::fread(&one, sizeof(qs_gate), 1, f) == 1) g.push_back(one);
  std::fclose(f);
  const int n = std::atoi(argv[2]);
  std::vector<FOp> fops;
  std::vector<int> vmap;
  build_fused_ops(g.data(), g.size(), n, fops, vmap, std::atoi(argv[3]) != 0, std::atoi(argv[4]) != 0);
  Plan pl;
  plan_circuit(fops, n, vmap, pl, TileLimits<double>::kMaxOps, kMaxTileStages);
  FILE* o = std::fopen(argv[5], "w");
  if (!o) return 2;
  std::fprintf(o, "steps %zu\n", pl.steps.size());
  for (const PlanStep& s : pl.steps) std::fprintf(o, "%d %d\n", (int)s.kind, s.index);
  std::unique_ptr<TileParams<double>> tp(new TileParams<double>());
  std::vector<C2<double>> tabs;
  for (size_t pi = 0; pi < pl.passes.size(); ++pi) {
    tile_pass_image<double>(pl, pl.passes[pi], tp.get(), tabs);
    const TilePass& P = tp->pass;
    std::fprintf(o, "pass %zu %d %d %zu\n", pi, P.n_stages, tp->n_jobs, tabs.size());
    std::fprintf(o, "%d", P.n_nt);
    for (int i = 0; i < kTileBits; ++i) std::fprintf(o, " %d", P.pos[i]);
    for (int i = 0; i < P.n_nt; ++i) std::fprintf(o, " %d", P.nt_pos[i]);
    std::fprintf(o, "\n");
    for (int s = 0; s < P.n_stages; ++s) {
      const TileStage& ts = tp->stages[s];
      std::fprintf(o, "stage");
      for (int k = 0; k < kRegBits; ++k) std::fprintf(o, " %d", ts.reg[k]);
      for (int k = 0; k < kWarpBits; ++k) std::fprintf(o, " %d", ts.warp[k]);
      std::fprintf(o, " %d %d\n", ts.op_begin, ts.op_end);
      for (int i = ts.op_begin; i < ts.op_end;) {
        const TileOp<double>& t = tp->ops[i];
        if (t.kind == TK_RUN) {
          RunHeader h;
          std::memcpy(&h, &t.m0[0], sizeof(h));
          const RunEntry<double>* e = reinterpret_cast<const RunEntry<double>*>(&tp->ops[i + 1]);
          const int count = (int)(t.slot * (sizeof(TileOp<double>) / sizeof(RunEntry<double>)));
          std::fprintf(o, "run %d %d %d %d %d %d %d %d %d %u %d\n", i, h.n_s, h.n_f[0], h.n_f[1], h.n_f[2],
                       h.n_f[3], h.ubase, h.umask, h.tmask, h.toff, count);
          for (int k = 0; k < count; ++k)
            std::fprintf(o, "entry %.17g %.17g %d %d %d %d\n", e[k].p.x, e[k].p.y, e[k].pa, e[k].pb, e[k].k, e[k].l);
          i += 1 + t.slot;
          continue;
        }
        std::fprintf(o, "op %d %d %d %d %d %d %d %d %d", i, t.kind, t.slot, t.csrc, t.cbit, t.dsrc, t.dbit, t.pad[0],
                     t.pad[1]);
        put_c2(o, t.m0, 4);
        put_c2(o, t.m1, 4);
        std::fprintf(o, "\n");
        ++i;
      }
    }
    for (int j = 0; j < tp->n_jobs; ++j) {
      RunJob jb;
      std::memcpy(&jb, tp->jobs + sizeof(RunJob) * j, sizeof(jb));
      std::fprintf(o, "job %d %d %d %d\n", jb.op, jb.first, jb.count, jb.scalar);
    }
    for (const C2<double>& x : tabs) std::fprintf(o, "tab %.17g %.17g\n", x.x, x.y);
  }
  std::fprintf(o, "plainops %zu\n", pl.plain_fops.size());
  for (const FOp& op : pl.plain_fops) {
    std::fprintf(o, "%d %d %d %d %d", (int)op.type, op.t, op.c, op.a, op.b);
    put_c(o, op.m0, 4);
    put_c(o, op.m1, 4);
    put_c(o, op.d, 4);
    put_c(o, op.g, 16);
    std::fprintf(o, "\n");
  }
  std::fprintf(o, "remaps %zu\n", pl.remaps.size());
  for (const RemapDesc& r : pl.remaps) {
    for (int i = 0; i < kTileBits; ++i) std::fprintf(o, "%d ", r.pos[i]);
    for (int i = 0; i < kTileBits; ++i) std::fprintf(o, "%d ", r.src[i]);
    std::fprintf(o, "%d", r.n_nt);
    for (int i = 0; i < r.n_nt; ++i) std::fprintf(o, " %d", r.nt_pos[i]);
    std::fprintf(o, "\n");
  }
  std::fclose(o);
  return 0;
}
