// Merging of one-qubit ops on a target across the ops between them.
#pragma once

#include <vector>

#include "internal.h"

namespace qs {

// ops: fused ops in application order.  A one-qubit op X (G1, or G1C with choice
// bit c) stays movable while no later op touches its target and, for a G1C, none
// acts non-diagonally on c: it then commutes with every op in between (an op
// block-diagonal in c commutes with ops that are diagonal on c and miss its
// target), so it moves up to the next one-qubit op Y on its target, and Y X is one
// op when the two have at most one distinct choice bit between them (Y_b X_b for
// each value b of it, an FP64 2x2 product).  Ops that carry a derivative term are
// never merged.  On return ops holds the surviving ops in order; if group is not
// NULL, (*group)[i] is the index in the result of the op that input op i went into.
void merge_one_qubit_ops(std::vector<FOp>& ops, int n, std::vector<int>* group);
// The same merge without moving the ops: on return (*into)[i] is the index of the
// later op that op i was merged into, or -1 for the ops that remain (in order).
void mark_one_qubit_merges(std::vector<FOp>& ops, int n, std::vector<int>* into);

}  // namespace qs
