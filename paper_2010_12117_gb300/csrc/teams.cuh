// Per-order launch table of the condensation kernels.
#pragma once

#include "../../include/polydet.h"

// Lanes per matrix (T), the resident CTAs of 128 threads the condensation
// kernel of each order n is compiled for (its __launch_bounds__ minimum) and
// the steps its fast pass takes at a time (2: Schur complement of a 2 x 2
// block, Fast2Step; 3: of a 3 x 3 block, Fast3Step), chosen per order from a
// sweep of all three on GB300 with random 31-bit matrices and 2^19 nodes:
// one lane while the whole matrix fits in registers (n <= 12), then 2, 4
// and 8 lanes; three steps where they beat two by 3 % or more (8-25 % at the
// orders that take them; at 9, 14, 16, 24 and 32 they tied or lost).  Orders
// 25-31 were not swept: they take the choice of n = 32.
constexpr int kTeam[POLYDET_MAX_N + 1] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2,
                                          2, 2, 2, 4, 4, 4, 4, 4, 8, 8, 8, 8, 8, 8, 8, 8};
constexpr int kMinBlocks[POLYDET_MAX_N + 1] = {1, 1, 1, 1, 3, 2, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4,
                                               4, 3, 3, 4, 4, 4, 4, 3, 3, 3, 3, 3, 3, 3, 3, 3};
constexpr int kStep[POLYDET_MAX_N + 1] = {2, 2, 2, 2, 2, 2, 2, 2, 3, 2, 3, 3, 3, 3, 2, 3, 2,
                                          3, 3, 3, 3, 3, 3, 3, 2, 2, 2, 2, 2, 2, 2, 2, 2};
