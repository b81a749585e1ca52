// Condensation kernels for n = 25..32 (one translation unit per range so
// that the fully unrolled instantiations compile in parallel).
#include "condense.cuh"

int pd_condense_d(const polydet_plan_s *pl, const uint32_t *evals, int prime_lo, int nprimes,
                     uint32_t *detvals, cudaStream_t st) {
  switch (pl->n) {
    PD_CONDENSE_CASE(25)
    PD_CONDENSE_CASE(26)
    PD_CONDENSE_CASE(27)
    PD_CONDENSE_CASE(28)
    PD_CONDENSE_CASE(29)
    PD_CONDENSE_CASE(30)
    PD_CONDENSE_CASE(31)
    PD_CONDENSE_CASE(32)
    default:
      return POLYDET_EINVAL;
  }
}
