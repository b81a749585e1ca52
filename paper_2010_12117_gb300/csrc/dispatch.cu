// Matrix order -> kernel object.  The ranges must match KERNEL_RANGES in
// build.py, which compiles condense_inst.cu and fused_inst.cu once per range.
#include "common.cuh"

int pd_condense_from_1(const polydet_plan_s *, const uint32_t *, EvLayout, int64_t, int64_t, int, int,
                         uint32_t *, int, cudaStream_t);
int pd_condense_from_7(const polydet_plan_s *, const uint32_t *, EvLayout, int64_t, int64_t, int, int,
                         uint32_t *, int, cudaStream_t);
int pd_condense_from_11(const polydet_plan_s *, const uint32_t *, EvLayout, int64_t, int64_t, int, int,
                         uint32_t *, int, cudaStream_t);
int pd_condense_from_13(const polydet_plan_s *, const uint32_t *, EvLayout, int64_t, int64_t, int, int,
                         uint32_t *, int, cudaStream_t);
int pd_condense_from_17(const polydet_plan_s *, const uint32_t *, EvLayout, int64_t, int64_t, int, int,
                         uint32_t *, int, cudaStream_t);
int pd_condense_from_21(const polydet_plan_s *, const uint32_t *, EvLayout, int64_t, int64_t, int, int,
                         uint32_t *, int, cudaStream_t);
int pd_condense_from_25(const polydet_plan_s *, const uint32_t *, EvLayout, int64_t, int64_t, int, int,
                         uint32_t *, int, cudaStream_t);
int pd_condense_from_29(const polydet_plan_s *, const uint32_t *, EvLayout, int64_t, int64_t, int, int,
                         uint32_t *, int, cudaStream_t);
int pd_fused_from_1(int, const FusedSeg *, int, int64_t, const uint32_t *, uint32_t *,
                   unsigned long long *, int, int, size_t, int, cudaStream_t);
int pd_fused_occ_from_1(int, int, size_t, int, int *);
int pd_fused_from_7(int, const FusedSeg *, int, int64_t, const uint32_t *, uint32_t *,
                   unsigned long long *, int, int, size_t, int, cudaStream_t);
int pd_fused_occ_from_7(int, int, size_t, int, int *);
int pd_fused_from_11(int, const FusedSeg *, int, int64_t, const uint32_t *, uint32_t *,
                   unsigned long long *, int, int, size_t, int, cudaStream_t);
int pd_fused_occ_from_11(int, int, size_t, int, int *);
int pd_fused_from_13(int, const FusedSeg *, int, int64_t, const uint32_t *, uint32_t *,
                   unsigned long long *, int, int, size_t, int, cudaStream_t);
int pd_fused_occ_from_13(int, int, size_t, int, int *);
int pd_fused_from_17(int, const FusedSeg *, int, int64_t, const uint32_t *, uint32_t *,
                   unsigned long long *, int, int, size_t, int, cudaStream_t);
int pd_fused_occ_from_17(int, int, size_t, int, int *);
int pd_fused_from_21(int, const FusedSeg *, int, int64_t, const uint32_t *, uint32_t *,
                   unsigned long long *, int, int, size_t, int, cudaStream_t);
int pd_fused_occ_from_21(int, int, size_t, int, int *);
int pd_fused_from_25(int, const FusedSeg *, int, int64_t, const uint32_t *, uint32_t *,
                   unsigned long long *, int, int, size_t, int, cudaStream_t);
int pd_fused_occ_from_25(int, int, size_t, int, int *);
int pd_fused_from_29(int, const FusedSeg *, int, int64_t, const uint32_t *, uint32_t *,
                   unsigned long long *, int, int, size_t, int, cudaStream_t);
int pd_fused_occ_from_29(int, int, size_t, int, int *);

int pd_launch_condense(const polydet_plan_s *pl, const uint32_t *evals, EvLayout lay, int prime_lo,
                       int nprimes, uint32_t *detvals, cudaStream_t st, int ctas_per_sm) {
  return pd_launch_condense_nodes(pl, evals, lay, pl->G, pl->G, prime_lo, nprimes, detvals, st, ctas_per_sm);
}

int pd_launch_condense_nodes(const polydet_plan_s *pl, const uint32_t *evals, EvLayout lay, int64_t G,
                             int64_t det_stride, int prime_lo, int nprimes, uint32_t *detvals,
                             cudaStream_t st, int ctas_per_sm) {
  const int n = pl->n;
  if (n < 1 || G < 1) return POLYDET_EINVAL;
  if (n <= 6) return pd_condense_from_1(pl, evals, lay, G, det_stride, prime_lo, nprimes, detvals, ctas_per_sm, st);
  if (n <= 10) return pd_condense_from_7(pl, evals, lay, G, det_stride, prime_lo, nprimes, detvals, ctas_per_sm, st);
  if (n <= 12) return pd_condense_from_11(pl, evals, lay, G, det_stride, prime_lo, nprimes, detvals, ctas_per_sm, st);
  if (n <= 16) return pd_condense_from_13(pl, evals, lay, G, det_stride, prime_lo, nprimes, detvals, ctas_per_sm, st);
  if (n <= 20) return pd_condense_from_17(pl, evals, lay, G, det_stride, prime_lo, nprimes, detvals, ctas_per_sm, st);
  if (n <= 24) return pd_condense_from_21(pl, evals, lay, G, det_stride, prime_lo, nprimes, detvals, ctas_per_sm, st);
  if (n <= 28) return pd_condense_from_25(pl, evals, lay, G, det_stride, prime_lo, nprimes, detvals, ctas_per_sm, st);
  if (n <= 32) return pd_condense_from_29(pl, evals, lay, G, det_stride, prime_lo, nprimes, detvals, ctas_per_sm, st);
  return POLYDET_EINVAL;
}

int pd_fused_launch(int n, const FusedSeg *segs, int nsegs, int64_t nitems, const uint32_t *partial,
                    uint32_t *detvals, unsigned long long *counter, int threads, int blocks,
                    size_t qwords, int nbuf, cudaStream_t st) {
  if (n < 1) return POLYDET_EINVAL;
  if (n <= 6) return pd_fused_from_1(n, segs, nsegs, nitems, partial, detvals, counter, threads, blocks, qwords, nbuf, st);
  if (n <= 10) return pd_fused_from_7(n, segs, nsegs, nitems, partial, detvals, counter, threads, blocks, qwords, nbuf, st);
  if (n <= 12) return pd_fused_from_11(n, segs, nsegs, nitems, partial, detvals, counter, threads, blocks, qwords, nbuf, st);
  if (n <= 16) return pd_fused_from_13(n, segs, nsegs, nitems, partial, detvals, counter, threads, blocks, qwords, nbuf, st);
  if (n <= 20) return pd_fused_from_17(n, segs, nsegs, nitems, partial, detvals, counter, threads, blocks, qwords, nbuf, st);
  if (n <= 24) return pd_fused_from_21(n, segs, nsegs, nitems, partial, detvals, counter, threads, blocks, qwords, nbuf, st);
  if (n <= 28) return pd_fused_from_25(n, segs, nsegs, nitems, partial, detvals, counter, threads, blocks, qwords, nbuf, st);
  if (n <= 32) return pd_fused_from_29(n, segs, nsegs, nitems, partial, detvals, counter, threads, blocks, qwords, nbuf, st);
  return POLYDET_EINVAL;
}

int pd_fused_occupancy(int n, int threads, size_t qwords, int nbuf, int *bps) {
  if (n < 1) return POLYDET_EINVAL;
  if (n <= 6) return pd_fused_occ_from_1(n, threads, qwords, nbuf, bps);
  if (n <= 10) return pd_fused_occ_from_7(n, threads, qwords, nbuf, bps);
  if (n <= 12) return pd_fused_occ_from_11(n, threads, qwords, nbuf, bps);
  if (n <= 16) return pd_fused_occ_from_13(n, threads, qwords, nbuf, bps);
  if (n <= 20) return pd_fused_occ_from_17(n, threads, qwords, nbuf, bps);
  if (n <= 24) return pd_fused_occ_from_21(n, threads, qwords, nbuf, bps);
  if (n <= 28) return pd_fused_occ_from_25(n, threads, qwords, nbuf, bps);
  if (n <= 32) return pd_fused_occ_from_29(n, threads, qwords, nbuf, bps);
  return POLYDET_EINVAL;
}

int pd_fused_team(int n) { return (n >= 1 && n <= POLYDET_MAX_N) ? kTeam[n] : 1; }

extern "C" int polydet_team_size(int n) {
  return (n >= 1 && n <= POLYDET_MAX_N) ? kTeam[n] : POLYDET_EINVAL;
}

extern "C" int polydet_condense_steps(int n) {
  return (n >= 1 && n <= POLYDET_MAX_N) ? kStep[n] : POLYDET_EINVAL;
}
