// Condensation kernels for n = 13..16 (one translation unit per range so
// that the fully unrolled instantiations compile in parallel).
#include "condense.cuh"

int pd_condense_b(const polydet_plan_s *pl, const uint32_t *evals, int prime_lo, int nprimes,
                     uint32_t *detvals, cudaStream_t st) {
  switch (pl->n) {
    PD_CONDENSE_CASE(13)
    PD_CONDENSE_CASE(14)
    PD_CONDENSE_CASE(15)
    PD_CONDENSE_CASE(16)
    default:
      return POLYDET_EINVAL;
  }
}
