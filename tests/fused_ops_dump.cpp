// Writes, as text, the fused op list the library runs on a state held by one CTA
// (n < 12, and the server's packed circuits): build_fused_ops with fusion, then
// optionally merge_one_qubit_ops (host side only).
// usage: fused_ops_dump gates.bin n merge out.txt
// One record per line: type t c a b, then m0, m1, d (4 complex each), g (16).
// Built against the library by test_tile_planner.py.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "fuse_merge.h"
#include "internal.h"

using namespace qs;

int main(int argc, char** argv) {
  if (argc != 5) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  std::vector<qs_gate> g;
  qs_gate one;
  while (std::fread(&one, sizeof(qs_gate), 1, f) == 1) g.push_back(one);
  std::fclose(f);
  const int n = std::atoi(argv[2]);
  std::vector<FOp> fops;
  std::vector<int> vmap;
  build_fused_ops(g.data(), g.size(), n, fops, vmap, true, false);
  if (std::atoi(argv[3]) != 0) merge_one_qubit_ops(fops, n, nullptr);
  FILE* o = std::fopen(argv[4], "w");
  if (!o) return 2;
  std::fprintf(o, "ops %zu\n", fops.size());
  for (const FOp& x : fops) {
    std::fprintf(o, "%d %d %d %d %d", (int)x.type, x.t, x.c, x.a, x.b);
    const cd* parts[4] = {x.m0, x.m1, x.d, x.g};
    const int len[4] = {4, 4, 4, 16};
    for (int p = 0; p < 4; ++p)
      for (int i = 0; i < len[p]; ++i) std::fprintf(o, " %.17g %.17g", parts[p][i].real(), parts[p][i].imag());
    std::fprintf(o, "\n");
  }
  std::fclose(o);
  return 0;
}
