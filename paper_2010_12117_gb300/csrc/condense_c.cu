// Condensation kernels for n = 17..24 (one translation unit per range so
// that the fully unrolled instantiations compile in parallel).
#include "condense.cuh"

int pd_condense_c(const polydet_plan_s *pl, const uint32_t *evals, int prime_lo, int nprimes,
                     uint32_t *detvals, cudaStream_t st) {
  switch (pl->n) {
    PD_CONDENSE_CASE(17)
    PD_CONDENSE_CASE(18)
    PD_CONDENSE_CASE(19)
    PD_CONDENSE_CASE(20)
    PD_CONDENSE_CASE(21)
    PD_CONDENSE_CASE(22)
    PD_CONDENSE_CASE(23)
    PD_CONDENSE_CASE(24)
    default:
      return POLYDET_EINVAL;
  }
}
