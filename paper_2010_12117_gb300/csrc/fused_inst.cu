// One object of fused kernels per range of matrix orders (see
// condense_inst.cu): compiled with -DPD_N_LO=.. -DPD_N_HI=..
#include "fused.cuh"

#define PD_CAT2(a, b) a##b
#define PD_CAT(a, b) PD_CAT2(a, b)

int PD_CAT(pd_fused_from_, PD_N_LO)(int n, const FusedSeg *segs, int nsegs, int64_t nitems,
                                    const uint32_t *partial, uint32_t *detvals,
                                    unsigned long long *counter, int threads, int blocks,
                                    size_t qwords, int nbuf, cudaStream_t st) {
  return fused_dispatch<PD_N_LO, PD_N_HI>(n, segs, nsegs, nitems, partial, detvals, counter, threads,
                                          blocks, qwords, nbuf, st);
}

int PD_CAT(pd_fused_occ_from_, PD_N_LO)(int n, int threads, size_t qwords, int nbuf, int *bps) {
  return fused_occ_dispatch<PD_N_LO, PD_N_HI>(n, threads, qwords, nbuf, bps);
}
