// Fused evaluation + condensation for batches of matrices of any shape: the
// last variable's evaluation (the last pass of Algorithm 2) is folded into
// the determinant kernel (Algorithm 3), so the evaluated matrices are never
// written to memory.
//
// Input per (job, prime): the partially evaluated tensor Q[row][entry][Lp],
// every variable but x_k already evaluated (row = node of x_1..x_{k-1}), the
// L = d_k + 1 coefficients of x_k left as they are.  One-variable jobs have
// no pass before this one: their tensor is the coefficient array reduced mod
// p (one row).
//
// The kernel is persistent: CTAs take items - S consecutive nodes of one
// (job, prime) segment, S = threads / lanes per determinant - from a counter
// in global memory until the list is exhausted, so one launch covers every
// (job, prime) pair of a matrix order, whatever the mix of grid sizes.  Per
// item:
//  0. the Q rows its nodes need (about S / M_k + 1, contiguous) reach shared
//     memory by one bulk copy that thread 0 started while the CTA computed
//     the previous item (two buffers, one mbarrier each; a wait that runs
//     out after a second sets POLYDET_STATUS_TIMEOUT and ends the CTA, after
//     one more bounded wait for every copy it issued; a copy still
//     outstanding then also sets POLYDET_STATUS_INFLIGHT, after which the
//     host must treat the CUDA context as unusable and tear it down).
//     Rows whose start or size is not a multiple of 16 bytes are copied by
//     the CTA itself;
//  1. a team of T lanes owns node g = (row, i): it forms x, the node's power
//     of w_k (Montgomery form, from the twiddle table) and its powers, and evaluates
//     each entry of its columns, sum_l Q[row][entry][l] x^l, with one REDC per
//     two products (2 p^2 < p 2^32), into its own slice of shared memory
//     (rolled loops: small code, no register pressure);
//  2. the slice is loaded into the register-resident matrix and goes through
//     the two-step elimination of condense_kernel (Algorithm 3).
#pragma once

#include "bulk.cuh"
#include "condense.cuh"

// Words of shared memory for the entry slices of a CTA of `threads` lanes.
template <int NN>
__host__ __device__ constexpr size_t fused_slice_words(int threads) {
  return (size_t)((NN + TeamFor<NN>::value - 1) / TeamFor<NN>::value) * NN * threads;
}

template <int NN, int T>
__device__ __forceinline__ void fused_eval_entries(const uint32_t *qrow, int t, const uint32_t (&X)[8],
                                                   int L, int Lp, uint32_t p, uint32_t pinv,
                                                   uint32_t *mine, int bd) {
  constexpr int M = (NN + T - 1) / T;
#pragma unroll 1
  for (int m = 0; m < M; ++m) {
    const int j = col_of<NN, T>(t, m);
    if (j < 0) continue;  // padding slot (condense.cuh): its registers are zeroed on load
#pragma unroll 2
    for (int i = 0; i < NN; ++i) {
      const uint32_t *q = qrow + (i * NN + j) * Lp;
      uint32_t v[8];
      if (Lp >= 4) {
        const uint4 lo4 = *reinterpret_cast<const uint4 *>(q);
        v[0] = lo4.x; v[1] = lo4.y; v[2] = lo4.z; v[3] = lo4.w;
        if (Lp == 8) {
          const uint4 hi4 = *(reinterpret_cast<const uint4 *>(q) + 1);
          v[4] = hi4.x; v[5] = hi4.y; v[6] = hi4.z; v[7] = hi4.w;
        } else {
          v[4] = v[5] = v[6] = v[7] = 0u;
        }
      } else if (Lp == 2) {
        const uint2 w2 = *reinterpret_cast<const uint2 *>(q);
        v[0] = w2.x; v[1] = w2.y;
        v[2] = v[3] = v[4] = v[5] = v[6] = v[7] = 0u;
      } else {
        v[0] = q[0];
        v[1] = v[2] = v[3] = v[4] = v[5] = v[6] = v[7] = 0u;
      }
      uint32_t acc = v[0];
      if (L > 1) {
        uint64_t s = (uint64_t)v[1] * X[1];
        if (L > 2) s += (uint64_t)v[2] * X[2];
        acc = addm(acc, redc(s, p, pinv), p);
      }
      if (L > 3) {
        uint64_t s = (uint64_t)v[3] * X[3];
        if (L > 4) s += (uint64_t)v[4] * X[4];
        acc = addm(acc, redc(s, p, pinv), p);
      }
      if (L > 5) {
        uint64_t s = (uint64_t)v[5] * X[5];
        if (L > 6) s += (uint64_t)v[6] * X[6];
        acc = addm(acc, redc(s, p, pinv), p);
      }
      if (L > 7) acc = addm(acc, mmul(v[7], X[7], p, pinv), p);
      mine[(m * NN + i) * bd] = acc;
    }
  }
}

// The pivoting elimination of the team's slice, for the rare warp in which
// the fast pass met a zero pivot; out of line so that it costs the fast pass
// no registers.
template <int NN, int T>
__device__ __noinline__ uint2 fused_det_search(const uint32_t *mine, int bd, int t, ModP md) {
  constexpr int M = (NN + T - 1) / T;
  uint32_t a[M][NN];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = col_of<NN, T>(t, m);
#pragma unroll
    for (int i = 0; i < NN; ++i) a[m][i] = (j >= 0) ? mine[(m * NN + i) * bd] : 0u;
  }
  uint32_t Q = md.r1, den = md.r1;
  ElimStep<NN, T, 0>::run(a, t, md.p, md.pinv, Q, den);
  return make_uint2(Q, den);
}

// Node g's determinant (one team), from the entries in its slice.  Kept out
// of line so that the register allocation of this straight-line body is not
// constrained by the persistent loop around it.
template <int NN, int T>
__device__ __noinline__ uint2 fused_det(const uint32_t *mine, int bd, int t, ModP md) {
  constexpr int M = (NN + T - 1) / T;
  const uint32_t p = md.p, pinv = md.pinv;
  uint32_t a[M][NN];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = col_of<NN, T>(t, m);
#pragma unroll
    for (int i = 0; i < NN; ++i) a[m][i] = (j >= 0) ? mine[(m * NN + i) * bd] : 0u;
  }
  uint32_t Q = md.r1, den = md.r1;
  bool zero = false;
  if constexpr (kStep[NN] == 3) {
    Fast3Step<NN, T, 0>::run(a, p, pinv, Q, den, zero);
  } else {
    Fast2Step<NN, T, 0>::run(a, p, pinv, Q, den, zero);
    zero |= p > PD_FOLD3_MAX;  // as in condense_kernel: larger primes redo every matrix
  }
  if (__any_sync(PD_FULL, zero))  // a zero pivot in this warp: redo with the search
    return fused_det_search<NN, T>(mine, bd, t, md);
  return make_uint2(Q, den);
}

// Geometry of one item: its first node g0, the first of the partial-tensor
// rows it spans and how many, and where those rows start (words into
// `partial`; they are contiguous).
struct FusedItem {
  int64_t g0, row0, src;
  int nrows, words;
};

template <int NN>
__device__ __forceinline__ FusedItem fused_item(const FusedSeg &sg, long long item, int S) {
  FusedItem f;
  f.g0 = (item - sg.item0) * S;
  f.row0 = f.g0 / sg.Mk;
  const int64_t glast = min(f.g0 + S, sg.G) - 1;
  f.nrows = (int)(glast / sg.Mk - f.row0 + 1);
  f.words = f.nrows * NN * NN * sg.Lp;
  f.src = sg.q_off + f.row0 * NN * NN * (int64_t)sg.Lp;
  return f;
}

template <int NN, int T>
__global__ void __launch_bounds__(128) fused_kernel(const FusedSeg *__restrict__ segs, int nsegs,
                                                    long long nitems,
                                                    const uint32_t *__restrict__ partial,
                                                    uint32_t *__restrict__ detvals,
                                                    unsigned long long *counter, int qwords,
                                                    int nbuf) {
  constexpr int NN2 = NN * NN;
  extern __shared__ uint4 fused_smem_u4[];
  __shared__ long long s_item[2];
  __shared__ int s_seg[2], s_bulk[2];
  __shared__ __align__(8) uint64_t s_bar[2];
  const int bd = blockDim.x;
  uint32_t *ent = reinterpret_cast<uint32_t *>(fused_smem_u4);  // [M * NN][bd]
  uint32_t *qbuf = ent + fused_slice_words<NN>(bd);             // nbuf x [rows][NN2][Lp]
  const int t = (int)(threadIdx.x & (T - 1));
  const int team = threadIdx.x / T;
  __shared__ uint32_t fin_q[128], fin_d[128];
  const int S = bd / T;

  // thread 0: take the next item from the counter into slot b and start the
  // bulk copy of its rows into the slot's buffer (when source, destination
  // and size are 16-byte multiples; otherwise the CTA copies them itself
  // later).  With two buffers slot b uses buffer b and the copy overlaps the
  // previous item; with one (when two do not fit in shared memory) both
  // slots use buffer 0 and the next item is fetched after the current one.
  // s_bulk: 0 the CTA copies, 1 a bulk copy is in flight, 2 the test hook
  // withheld the copy (the wait for it runs out)
  auto fetch = [&](int b) {
    const long long it = (long long)atomicAdd(counter, 1ull);
    int lo = 0, bulk = 0;
    if (it < nitems) {
      int hi = nsegs - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].item0 <= it) lo = mid; else hi = mid - 1;
      }
      const FusedItem f = fused_item<NN>(segs[lo], it, S);
      const uint32_t *src = partial + f.src;
      uint32_t *dst = qbuf + (size_t)(nbuf == 2 ? b : 0) * qwords;
      bulk = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0 &&
             (f.words & 3) == 0 && f.words <= qwords;
      if (bulk && segs[lo].drop_copies) {
        bulk = 2;
      } else if (bulk) {
        pd_fence_proxy_async();
        pd_mbar_expect_tx(&s_bar[b], (uint32_t)f.words * 4u);
        pd_bulk_g2s(dst, src, (uint32_t)f.words * 4u, &s_bar[b]);
      }
    }
    s_item[b] = it;
    s_seg[b] = lo;
    s_bulk[b] = bulk;
  };

  if (threadIdx.x == 0) {
    pd_mbar_init(&s_bar[0], 1);
    pd_mbar_init(&s_bar[1], 1);
    pd_mbar_init_fence();
    fetch(0);
  }
  __syncthreads();

  uint32_t phase = 0u;  // bit b: parity of buffer b's barrier phase to wait for
  for (int cur = 0;; cur ^= 1) {
    const long long item = s_item[cur];  // written before the last barrier
    if (item >= nitems) return;          // the same for every thread; nothing in flight
    const int si = s_seg[cur];
    const int bulk = s_bulk[cur];
    // the next item's rows stream in while this one is computed (its slot and
    // buffer were last read before the barriers of the previous iteration)
    if (nbuf == 2 && threadIdx.x == 0) fetch(cur ^ 1);

    const FusedSeg &sg = segs[si];
    const FusedItem f = fused_item<NN>(sg, item, S);
    uint32_t *qsm = qbuf + (size_t)(nbuf == 2 ? cur : 0) * qwords;
    int late = 0;
    if (bulk) {
      late = !pd_mbar_wait_bounded(&s_bar[cur], (phase >> cur) & 1u);
      phase ^= 1u << cur;
    } else {  // 0. this item's rows into shared memory by the CTA
      const uint32_t *src = partial + f.src;
      for (int w = threadIdx.x; w < f.words; w += bd) qsm[w] = __ldg(src + w);
    }
    if (__syncthreads_or(late)) {
      // a copy did not land in time: report it, give both copies that may
      // still be in flight - this item's (when one was issued) and the next
      // item's started above - one more bounded wait each, and stop this
      // CTA.  If either is still outstanding after that, it could land in
      // shared memory that a later CTA owns: POLYDET_STATUS_INFLIGHT tells
      // the host that the context must not be trusted any more.
      if (threadIdx.x == 0) {
        bool gone = true;
        if (bulk == 1) gone &= pd_mbar_wait_bounded(&s_bar[cur], ((phase >> cur) & 1u) ^ 1u);
        if (nbuf == 2 && s_bulk[cur ^ 1] == 1)
          gone &= pd_mbar_wait_bounded(&s_bar[cur ^ 1], (phase >> (cur ^ 1)) & 1u);
        atomicOr(sg.status, POLYDET_STATUS_TIMEOUT | (gone ? 0u : POLYDET_STATUS_INFLIGHT));
      }
      return;
    }

    const uint32_t p = sg.md.p, pinv = sg.md.pinv;
    const int logNk = sg.logNk;
    const int64_t Mk = sg.Mk;
    const int Lp = sg.Lp;
    const int64_t g0 = f.g0, row0 = f.row0;
    const int64_t glast = min(g0 + S, sg.G) - 1;
    const int64_t g = g0 + team;
    const bool active = g < sg.G;
    const int64_t gg = active ? g : glast;
    const int64_t grow = gg / Mk;
    const int ik = (int)(gg - grow * Mk);
    const int L = sg.L;
    uint32_t X[8];
    X[0] = sg.md.r1;
    if (logNk == 0) {
      X[1] = sg.md.r1;
    } else {
      const int ex = node_exp(ik, 1 << logNk, sg.LPk);  // node ik of x_k is w^ex
      X[1] = __ldg(sg.tw + ex);
    }
#pragma unroll
    for (int l = 2; l < 8; ++l) X[l] = (l < L) ? mmul(X[l - 1], X[1], p, pinv) : 0u;

    // 1. entries of this lane's columns at its node, into its slice
    uint32_t *mine = ent + threadIdx.x;
    fused_eval_entries<NN, T>(qsm + (grow - row0) * NN2 * Lp, t, X, L, Lp, p, pinv, mine,
                              bd);
    // 2. elimination in registers; 3. one lane per node finishes its
    // determinant (one inversion each) and the item's results are stored
    // contiguously
    const uint2 qd = fused_det<NN, T>(mine, bd, t, sg.md);
    if (t == 0) {
      fin_q[team] = qd.x;
      fin_d[team] = qd.y;
    }
    __syncthreads();
    if ((int)threadIdx.x < S && g0 + threadIdx.x < sg.G)
      detvals[sg.det_off + g0 + threadIdx.x] =
          finish_det(fin_q[threadIdx.x], fin_d[threadIdx.x], sg.md, sg.rn);
    if (nbuf == 1) {  // the one buffer was last read before the barrier above
      if (threadIdx.x == 0) fetch(cur ^ 1);
      __syncthreads();
    }
    (void)active;
  }
}

// Dynamic shared memory of a fused CTA: entry slices + `nbuf` buffers of
// `qwords` words of Q rows (qwords a multiple of 4: each starts on 16 bytes).
template <int NN>
constexpr size_t fused_smem(int threads, size_t qwords, int nbuf) {
  return (fused_slice_words<NN>(threads) + (size_t)nbuf * qwords) * sizeof(uint32_t);
}

template <int NN, int HI>
static int fused_dispatch(int n, const FusedSeg *segs, int nsegs, int64_t nitems,
                          const uint32_t *partial, uint32_t *detvals, unsigned long long *counter,
                          int threads, int blocks, size_t qwords, int nbuf, cudaStream_t st) {
  if (n == NN) {
    fused_kernel<NN, TeamFor<NN>::value><<<blocks, threads, fused_smem<NN>(threads, qwords, nbuf), st>>>(
        segs, nsegs, (long long)nitems, partial, detvals, counter, (int)qwords, nbuf);
    PD_CUDA(cudaGetLastError());
    return POLYDET_OK;
  }
  if constexpr (NN < HI) {
    return fused_dispatch<NN + 1, HI>(n, segs, nsegs, nitems, partial, detvals, counter, threads,
                                      blocks, qwords, nbuf, st);
  }
  return POLYDET_EINVAL;
}

// Occupancy of order n at `threads` lanes and `nbuf` buffers of `qwords`
// words of Q rows; also
// raises the kernel's dynamic shared-memory limit (call before any graph
// capture: the batch plan and polydet_batch_set_launch do).  Reports 0 when
// the CTA does not fit.
template <int NN, int HI>
static int fused_occ_dispatch(int n, int threads, size_t qwords, int nbuf, int *bps) {
  if (n == NN) {
    const size_t smem = fused_smem<NN>(threads, qwords, nbuf);
    if (smem > 220 * 1024) {
      *bps = 0;
      return POLYDET_OK;
    }
    PD_CUDA(cudaFuncSetAttribute(fused_kernel<NN, TeamFor<NN>::value>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, fused_kernel<NN, TeamFor<NN>::value>,
                                                          threads, smem));
    return POLYDET_OK;
  }
  if constexpr (NN < HI) return fused_occ_dispatch<NN + 1, HI>(n, threads, qwords, nbuf, bps);
  return POLYDET_EINVAL;
}
