// Per-order launch table of the condensation kernels.
#pragma once

#include "../../include/polydet.h"

// Lanes per matrix (T) and the resident CTAs of 128 threads the condensation
// kernel of each order n is compiled for (its __launch_bounds__ minimum),
// chosen per order from a sweep of both on GB300 with random 31-bit matrices
// (2^18 nodes): one lane while the whole matrix fits in registers (except
// n = 13, where two lanes with 3 CTAs per SM hide more latency), then the
// pair that kept the elimination the least latency-bound.
constexpr int kTeam[POLYDET_MAX_N + 1] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 2, 1, 1, 2,
                                          2, 4, 4, 4, 4, 4, 4, 8, 8, 8, 8, 8, 8, 8, 8, 16};
constexpr int kMinBlocks[POLYDET_MAX_N + 1] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 3, 1, 1, 2,
                                               3, 4, 4, 4, 3, 3, 3, 4, 4, 4, 4, 3, 3, 3, 3, 4};
