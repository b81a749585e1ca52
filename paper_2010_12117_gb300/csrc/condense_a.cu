// Condensation kernels for n = 1..12 (one translation unit per range so
// that the fully unrolled instantiations compile in parallel).
#include "condense.cuh"

int pd_condense_a(const polydet_plan_s *pl, const uint32_t *evals, int prime_lo, int nprimes,
                     uint32_t *detvals, cudaStream_t st) {
  switch (pl->n) {
    PD_CONDENSE_CASE(1)
    PD_CONDENSE_CASE(2)
    PD_CONDENSE_CASE(3)
    PD_CONDENSE_CASE(4)
    PD_CONDENSE_CASE(5)
    PD_CONDENSE_CASE(6)
    PD_CONDENSE_CASE(7)
    PD_CONDENSE_CASE(8)
    PD_CONDENSE_CASE(9)
    PD_CONDENSE_CASE(10)
    PD_CONDENSE_CASE(11)
    PD_CONDENSE_CASE(12)
    default:
      return POLYDET_EINVAL;
  }
}

int pd_condense_b(const polydet_plan_s *, const uint32_t *, int, int, uint32_t *, cudaStream_t);
int pd_condense_c(const polydet_plan_s *, const uint32_t *, int, int, uint32_t *, cudaStream_t);
int pd_condense_d(const polydet_plan_s *, const uint32_t *, int, int, uint32_t *, cudaStream_t);

int pd_launch_condense(const polydet_plan_s *pl, const uint32_t *evals, int prime_lo, int nprimes,
                       uint32_t *detvals, cudaStream_t st) {
  if (pl->n <= 12) return pd_condense_a(pl, evals, prime_lo, nprimes, detvals, st);
  if (pl->n <= 16) return pd_condense_b(pl, evals, prime_lo, nprimes, detvals, st);
  if (pl->n <= 24) return pd_condense_c(pl, evals, prime_lo, nprimes, detvals, st);
  return pd_condense_d(pl, evals, prime_lo, nprimes, detvals, st);
}
