// Writes the 5-qubit blocks the planner makes of a gate list (host side only):
// usage: block_plan_dump gates.bin n out.bin.  Per block: 5 int32 qubits (q[i] is
// bit i of the block's local index), int32 unitary flag, 32x32 complex128
// row-major U[out][in].  Built against the library by test_block_planner.py.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "internal.h"

using namespace qs;

int main(int argc, char** argv) {
  if (argc != 4) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  std::vector<qs_gate> g;
  qs_gate one;
  while (std::fread(&one, sizeof(qs_gate), 1, f) == 1) g.push_back(one);
  std::fclose(f);
  std::vector<Block> blocks;
  plan_blocks(g.data(), g.size(), std::atoi(argv[2]), blocks);
  FILE* o = std::fopen(argv[3], "wb");
  if (!o) return 2;
  for (const Block& b : blocks) {
    const int u = block_is_unitary(b.U.data()) ? 1 : 0;
    std::fwrite(b.q, sizeof(int), 5, o);
    std::fwrite(&u, sizeof(int), 1, o);
    std::fwrite(b.U.data(), sizeof(cd), 1024, o);
  }
  std::fclose(o);
  return 0;
}
