// One object of condensation kernels per range of matrix orders: the build
// compiles this file once per range with -DPD_N_LO=.. -DPD_N_HI=.. so the
// fully unrolled instantiations compile in parallel.
#include "condense.cuh"

#define PD_CAT2(a, b) a##b
#define PD_CAT(a, b) PD_CAT2(a, b)

int PD_CAT(pd_condense_from_, PD_N_LO)(const polydet_plan_s *pl, const uint32_t *evals,
                                       EvLayout lay, int64_t G, int64_t det_stride, int prime_lo,
                                       int nprimes, uint32_t *detvals, int ctas_per_sm,
                                       cudaStream_t st) {
  return condense_dispatch<PD_N_LO, PD_N_HI>(pl, evals, lay, G, det_stride, prime_lo, nprimes, detvals,
                                             ctas_per_sm, st);
}
