// Per-order launch table of the condensation kernels.
#pragma once

#include "../../include/polydet.h"

// Lanes per matrix (T), the resident CTAs per SM the condensation kernel of
// each order n is compiled for (its __launch_bounds__ minimum), the steps its
// fast pass takes at a time (2: Schur complement of a 2 x 2 block,
// Fast2Step; 3: of a 3 x 3 block, Fast3Step) and its threads per CTA.
// First chosen per order from sweeps on GB300 with random 31-bit matrices on
// 2^19 nodes: one lane while the whole matrix fits in registers (n <= 12),
// then 2, 4 and 8 lanes; three steps where they beat two by 3 % or more
// (8-25 % at the orders that take them).  Then, for orders 14-24, every
// alternative was timed on the launches the batched workload itself makes
// (the sweep's single large launch did not always predict them: taking rows
// two at a time or four steps per pass won there and lost here), and the
// table keeps what won on the workload: at n = 24 two steps on two CTAs of
// 192 threads (4 % over three CTAs of 128; three steps on the same CTAs won
// 2.6 % on launches of the workload's jobs in their input variable order but
// not on the benchmark's own, so two stay), at n = 22 and 20 two steps on
// 256-thread CTAs, at 21 three steps on 256-thread CTAs.
// Threads per CTA: the fully unrolled elimination of the large orders is
// longer than the instruction cache, so fewer, larger CTAs per SM, whose
// warps walk the same code together, stall less on instruction fetch (ncu at
// n = 24: 0.24 instead of 1.30 no-instruction stalls per issue with two CTAs
// of 192 threads instead of three of 128, the same 12 warps and registers).
// Orders 25-31 were not swept: they take the choice of n = 32.
constexpr int kTeam[POLYDET_MAX_N + 1] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2,
                                          2, 2, 2, 4, 4, 4, 4, 4, 8, 8, 8, 8, 8, 8, 8, 8};
constexpr int kMinBlocks[POLYDET_MAX_N + 1] = {1, 1, 1, 1, 3, 2, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4,
                                               4, 3, 3, 2, 2, 2, 4, 2, 3, 3, 3, 3, 3, 3, 3, 3};
constexpr int kStep[POLYDET_MAX_N + 1] = {2, 2, 2, 2, 2, 2, 2, 2, 3, 2, 3, 3, 3, 3, 2, 3, 2,
                                          3, 3, 3, 2, 3, 2, 3, 2, 2, 2, 2, 2, 2, 2, 2, 2};
constexpr int kThreads[POLYDET_MAX_N + 1] = {128, 128, 128, 128, 128, 128, 128, 128, 128, 128, 128,
                                             128, 128, 128, 128, 128, 128, 128, 128, 128, 256, 256,
                                             256, 128, 192, 128, 128, 128, 128, 128, 128, 128, 128};
