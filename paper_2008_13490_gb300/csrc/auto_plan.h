// The default method's choice between its segment plan and tile passes only.
#pragma once

#include <vector>

#include "internal.h"

namespace qs {

// blocks: the 5-qubit blocks of gates[0..ngates) (plan_blocks).  With one or two
// dense blocks (more than 512 of 1024 entries nonzero) among sparse ones, the
// whole circuit on tile passes saves the blocks' sweeps when it takes no more tile
// passes and no more remaps than the runs of sparse blocks alone.  Returns true
// in that case, with the whole circuit's fused ops and final qubit map in *fops
// and *vmap (for the tiled run); false otherwise (the segment plan stands).
bool auto_all_tiles(const qs_gate* gates, size_t ngates, int n, const std::vector<Block>& blocks,
                    std::vector<FOp>* fops, std::vector<int>* vmap);

}  // namespace qs
