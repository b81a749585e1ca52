// Per-order launch table of the condensation kernels.
#pragma once

#include "../../include/polydet.h"

// Lanes per matrix (T) and the resident CTAs of 128 threads the condensation
// kernel of each order n is compiled for (its __launch_bounds__ minimum),
// chosen per order from a sweep of both on GB300 with the two-step
// elimination, random 31-bit matrices and 2^19 nodes: one lane while the
// whole matrix fits in registers (n <= 13), then 2, 4 and 8 lanes; three
// CTAs per SM (168 registers) wherever the matrix needs them, four where it
// fits in 128.  Orders 25-31 were not swept: they take the choice of n = 32.
constexpr int kTeam[POLYDET_MAX_N + 1] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 2, 2, 2,
                                          4, 2, 4, 4, 4, 4, 4, 4, 8, 8, 8, 8, 8, 8, 8, 8};
constexpr int kMinBlocks[POLYDET_MAX_N + 1] = {1, 1, 1, 1, 3, 2, 4, 4, 2, 4, 3, 3, 3, 1, 4, 4, 4,
                                               4, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3};
