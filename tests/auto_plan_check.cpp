// Prints 1 when the default method would run a gate list on tile passes alone
// (auto_all_tiles), else 0, and the number of dense blocks (host side only).
// usage: auto_plan_check gates.bin n.  Built against the library by
// test_block_planner.py.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "auto_plan.h"
#include "internal.h"

using namespace qs;

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  std::vector<qs_gate> g;
  qs_gate one;
  while (std::fread(&one, sizeof(qs_gate), 1, f) == 1) g.push_back(one);
  std::fclose(f);
  const int n = std::atoi(argv[2]);
  std::vector<Block> blocks;
  plan_blocks(g.data(), g.size(), n, blocks);
  int dense = 0;
  for (const Block& b : blocks) dense += block_nonzeros(b) > 512 ? 1 : 0;
  std::vector<FOp> fops;
  std::vector<int> vmap;
  const bool tiles = auto_all_tiles(g.data(), g.size(), n, blocks, &fops, &vmap);
  std::printf("%d %d\n", tiles ? 1 : 0, dense);
  return 0;
}
