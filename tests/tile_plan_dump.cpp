// Writes, as text, the tile-pass plan the library makes of a gate list (host
// side only): usage: tile_plan_dump gates.bin n fuse relabel out.txt [max_stages [max_ops]]
// (the pass limits; the library's own by default).
// Sections (one record per line, numbers separated by blanks):
//   steps K      / kind index                       (0 tile, 1 plain, 2 remap, 3 small)
//   passes P     / n_stages stage_begin n_nt pos[12] nt_pos[n_nt]
//   stages S     / reg[4] warp[3] op_begin op_end
//   tileops T    / kind slot csrc cbit dsrc dbit type  then m0, m1, d (4 complex each), g (16)
//   plainops Q   / type t c a b  then m0, m1, d, g
//   remaps R     / pos[12] src[12] n_nt nt_pos[n_nt]
// Built against the library by test_tile_planner.py.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "internal.h"

using namespace qs;

static void put_c(FILE* o, const cd* v, int k) {
  for (int i = 0; i < k; ++i) std::fprintf(o, " %.17g %.17g", v[i].real(), v[i].imag());
}

int main(int argc, char** argv) {
  if (argc < 6 || argc > 8) return 2;
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
  const int max_stages = argc > 6 ? std::atoi(argv[6]) : kMaxTileStages;
  const int max_ops = argc > 7 ? std::atoi(argv[7]) : TileLimits<float>::kMaxOps;
  plan_circuit(fops, n, vmap, pl, max_ops, max_stages);
  FILE* o = std::fopen(argv[5], "w");
  if (!o) return 2;
  std::fprintf(o, "steps %zu\n", pl.steps.size());
  for (const PlanStep& s : pl.steps) std::fprintf(o, "%d %d\n", (int)s.kind, s.index);
  std::fprintf(o, "passes %zu\n", pl.passes.size());
  for (const TilePass& p : pl.passes) {
    std::fprintf(o, "%d %d %d", p.n_stages, p.stage_begin, p.n_nt);
    for (int i = 0; i < kTileBits; ++i) std::fprintf(o, " %d", p.pos[i]);
    for (int i = 0; i < p.n_nt; ++i) std::fprintf(o, " %d", p.nt_pos[i]);
    std::fprintf(o, "\n");
  }
  std::fprintf(o, "stages %zu\n", pl.stages.size());
  for (const TileStage& s : pl.stages) {
    for (int k = 0; k < kRegBits; ++k) std::fprintf(o, "%d ", s.reg[k]);
    for (int k = 0; k < kWarpBits; ++k) std::fprintf(o, "%d ", s.warp[k]);
    std::fprintf(o, "%d %d\n", s.op_begin, s.op_end);
  }
  std::fprintf(o, "tileops %zu\n", pl.tile_fops.size());
  for (size_t i = 0; i < pl.tile_fops.size(); ++i) {
    const FOp& op = pl.tile_fops[i];
    std::fprintf(o, "%d %d %d %d %d %d %d", pl.tile_kind[i], pl.tile_slot[i], pl.tile_csrc[i], pl.tile_cbit[i],
                 pl.tile_dsrc[i], pl.tile_dbit[i], (int)op.type);
    put_c(o, op.m0, 4);
    put_c(o, op.m1, 4);
    put_c(o, op.d, 4);
    put_c(o, op.g, 16);
    std::fprintf(o, "\n");
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
