// Determinant mod p of one n x n matrix per grid node (Sec. 3.2, Algorithm 3).
//
// A team of T consecutive lanes owns one matrix: lane t holds the columns
// j = t - s, t - s + T, t - s + 2T, ... entirely in registers (one lane for
// most n <= 15, up to 16 lanes at n = 32; the per-order T and the CTAs per SM the
// kernel is compiled for are the table of teams.cuh).  The s = T ceil(n/T) - n
// padding slots (j < 0) sit in the first block of T columns, which drops out
// of the elimination after its first steps; in the last block they would be
// computed and discarded at almost every step.  Every index into the register
// array is a compile-time constant after unrolling, and there are no
// barriers: the team talks through warp shuffles.
//
// Elimination is fraction free (the update of Algorithm 3):
// at step c every column j > c of every row i > c becomes
// a_cc * a_ij - a_ic * a_cj, evaluated with one Montgomery REDC of the two
// 62-bit products.  Reading every stored value s as the Montgomery form of
// v = s / R, that update is exactly v_cc v_ij - v_ic v_cj, so with the pivots
// v_cc of the steps, det(V) = prod_c v_cc / prod_c v_cc^(n-1-c), and the
// input A = R * V gives det(A) = R^n det(V).  The denominator is accumulated
// as prod_{c<n-1} Q_c with Q_c = prod_{j<=c} v_jj, and inverted once by
// Fermat's little theorem at the end, instead of one inverse per step.
//
// The fast pass takes the steps two or three at a time, per order (Fast2Step:
// the Schur complement of the leading 2 x 2 block, one three-product sum and
// one REDC per element and pair of steps; Fast3Step: of the leading 3 x 3
// block, four products and one REDC per element and triple of steps) and runs
// without any search and without a warp vote per step; a zero pivot (a zero
// block determinant) is only recorded.
// Pivot search (Algorithm 3's first nonzero entry), for the rare warp that
// met one: the matrices are redone one step at a time (ElimStep, out of
// line); when the pivot a_cc is zero, the first row r > c with a_rc != 0 is
// added to row c, which leaves the determinant unchanged.  If the column is
// zero below c the pivot stays 0 and the result is 0, as the paper states.
#pragma once

#include "common.cuh"

#define PD_FULL 0xffffffffu

// Column slots of a team of T lanes: M per lane, the first S of block 0
// padding (no column).
template <int NN, int T>
struct ColLayout {
  static constexpr int M = (NN + T - 1) / T;
  static constexpr int S = T * M - NN;
};

// The column held in slot m of lane t (negative: padding).
template <int NN, int T>
PD_D int col_of(int t, int m) {
  return T * m + t - ColLayout<NN, T>::S;
}

// Whether lane t's m-th column j = col_of(t, m) lies strictly between lo and
// NN.  After unrolling m and lo are constants, so every part that does not
// depend on t folds away: columns wholly inside or outside the range cost
// nothing, only a column block that straddles `lo` keeps a run-time test.
template <int NN, int T>
PD_D bool col_in(int t, int m, int lo) {
  constexpr int S = ColLayout<NN, T>::S;
  const int jmin = T * m - S, jmax = T * m + T - 1 - S;
  if (jmin > lo && jmax < NN) return true;
  if (jmax <= lo || jmin >= NN) return false;
  const int j = jmin + t;
  return j > lo && j < NN;
}

// One lane per determinant: the (numerator, denominator) pair of the
// elimination gives det(A) = R^n num / den (see ElimStep), finished by one
// Fermat inversion.
PD_D uint32_t finish_det(uint32_t Q, uint32_t den, const ModP &md, uint32_t rn) {
  const uint32_t inv = mpow(den, md.p - 2u, md.r1, md.p, md.pinv);
  return mmul(mmul(Q, inv, md.p, md.pinv), rn, md.p, md.pinv);
}

// One elimination step c, with c a template parameter so that every index
// into the register array is a compile-time constant.
template <int NN, int T, int c>
struct ElimStep {
  static constexpr int M = (NN + T - 1) / T;
  static PD_D void run(uint32_t (&a)[M][NN], int t, uint32_t p, uint32_t pinv, uint32_t &Q,
                       uint32_t &den) {
    constexpr int owner = (c + ColLayout<NN, T>::S) % T;
    constexpr int mc = (c + ColLayout<NN, T>::S) / T;
    uint32_t piv = (T == 1) ? a[mc][c] : __shfl_sync(PD_FULL, a[mc][c], owner, T);
    if (c < NN - 1) {
      if (__any_sync(PD_FULL, piv == 0u)) {
        int r = NN;
#pragma unroll
        for (int i = NN - 1; i > c; --i)
          if (a[mc][i] != 0u) r = i;
        if (T > 1) r = __shfl_sync(PD_FULL, r, owner, T);
        const bool fix = (piv == 0u) && (r < NN);
#pragma unroll
        for (int m = 0; m < M; ++m) {
          if (col_in<NN, T>(t, m, c - 1)) {
            uint32_t add = 0u;
#pragma unroll
            for (int i = c + 1; i < NN; ++i) add = (i == r) ? a[m][i] : add;
            a[m][c] = fix ? addm(a[m][c], add, p) : a[m][c];
          }
        }
        piv = (T == 1) ? a[mc][c] : __shfl_sync(PD_FULL, a[mc][c], owner, T);
      }
      uint32_t f[NN];
#pragma unroll
      for (int i = c + 1; i < NN; ++i)
        f[i] = (T == 1) ? a[mc][i] : __shfl_sync(PD_FULL, a[mc][i], owner, T);
#pragma unroll
      for (int m = 0; m < M; ++m) {
        if (col_in<NN, T>(t, m, c)) {
          const uint32_t acj = a[m][c];
#pragma unroll
          for (int i = c + 1; i < NN; ++i) a[m][i] = mfms(piv, a[m][i], f[i], acj, p, pinv);
        }
      }
      Q = mmul(Q, piv, p, pinv);
      den = mmul(den, Q, p, pinv);
      ElimStep<NN, T, c + 1>::run(a, t, p, pinv, Q, den);
    } else {
      Q = mmul(Q, piv, p, pinv);
    }
  }
};

template <int NN, int T>
struct ElimStep<NN, T, NN> {
  static constexpr int M = (NN + T - 1) / T;
  static PD_D void run(uint32_t (&)[M][NN], int, uint32_t, uint32_t, uint32_t &, uint32_t &) {}
};

// Two elimination steps at once (columns c and c + 1), the form the fast
// pass uses: with the trailing matrix's leading 2 x 2 block
// [[a_cc, a_c,c+1], [a_c+1,c, a_c+1,c+1]] of determinant D2 and its Schur
// complement S, for i, j >= c + 2
//   D2 S_ij = D2 a_ij + C1_j a_ic + C2_j a_i,c+1,
//   C1_j = a_c,c+1 a_c+1,j - a_c+1,c+1 a_cj,  C2_j = a_c+1,c a_cj - a_cc a_c+1,j,
// and det(trailing) = D2 det(S) = det(D2 S) / D2^(m - 1) with m = n - c - 2
// rows left.  Each element costs one three-product sum and one REDC
// (mfms3) instead of the two products and two REDCs of two single steps;
// C1_j and C2_j cost two REDCs per column and pair of steps.  The pivot
// bookkeeping is ElimStep's with D2 as the pivot of a step that removes two
// rows: den gains Q^2 (Q^1 for a single step) before Q gains the pivot, so
// that every pivot ends up in den to the power of the rows left after its
// step.  A zero D2 is only recorded (the caller redoes the matrix with
// ElimStep); an odd order ends with one single step (the last 1 x 1 pivot).
// Needs p <= PD_FOLD3_MAX.
template <int NN, int T, int c>
struct Fast2Step {
  static constexpr int M = (NN + T - 1) / T;
  static constexpr int S = ColLayout<NN, T>::S;
  static PD_D uint32_t bcast(uint32_t v, int owner) {
    return (T == 1) ? v : __shfl_sync(PD_FULL, v, owner, T);
  }
  static PD_D void run(uint32_t (&a)[M][NN], uint32_t p, uint32_t pinv, uint32_t &Q,
                       uint32_t &den, bool &zero) {
    constexpr int o0 = (c + S) % T, m0 = (c + S) / T;  // owner and slot of column c
    if constexpr (c == NN - 1) {
      const uint32_t piv = bcast(a[m0][c], o0);
      zero |= (piv == 0u);
      den = mmul(den, Q, p, pinv);
      Q = mmul(Q, piv, p, pinv);
    } else {
      constexpr int o1 = (c + 1 + S) % T, m1 = (c + 1 + S) / T;  // column c + 1
      const uint32_t a00 = bcast(a[m0][c], o0), a10 = bcast(a[m0][c + 1], o0);
      const uint32_t a01 = bcast(a[m1][c], o1), a11 = bcast(a[m1][c + 1], o1);
      const uint32_t d2 = mfms(a00, a11, a10, a01, p, pinv);
      zero |= (d2 == 0u);
      den = mmul(den, mmul(Q, Q, p, pinv), p, pinv);
      Q = mmul(Q, d2, p, pinv);
      if constexpr (c + 2 < NN) {
        // every block that still holds a column j > c + 1 updates all its
        // lanes, with no select: the other slots of a block that straddles
        // c + 1 (columns <= c + 1, padding) are never read again, and blocks
        // wholly left of c + 2 drop out at compile time
        uint32_t c1[M], c2[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          if (T * m + T - 1 - S > c + 1) {
            c1[m] = mfms(a01, a[m][c + 1], a11, a[m][c], p, pinv);
            c2[m] = mfms(a10, a[m][c], a00, a[m][c + 1], p, pinv);
          }
        }
        // row by row: the two broadcast column entries of row i are read
        // before any lane rewrites row i
#pragma unroll
        for (int i = c + 2; i < NN; ++i) {
          const uint32_t bi = bcast(a[m0][i], o0), ei = bcast(a[m1][i], o1);
#pragma unroll
          for (int m = 0; m < M; ++m) {
            if (T * m + T - 1 - S > c + 1) a[m][i] = mfms3(d2, a[m][i], c1[m], bi, c2[m], ei, p, pinv);
          }
        }
        Fast2Step<NN, T, c + 2>::run(a, p, pinv, Q, den, zero);
      }
    }
  }
};

// Words from a node's value of its first evals entry to its value of entry
// (i, j), for every (i, j): e * (words per entry) normally; with an entry map
// (repeated and zero entries) the slot of (i, j) times the same.  Passed by
// value as a kernel parameter (compile-time indices after unrolling: the
// loads take their offsets from the constant bank).
template <int NN>
struct EntryOff {
  int64_t o[NN * NN];
};

// Three elimination steps at once (columns c, c + 1, c + 2): with the
// trailing matrix's leading 3 x 3 block A11 of determinant D3, its cofactors
// cof_lk and Schur complement S, for i, j >= c + 3
//   D3 S_ij = D3 a_ij + sum_k C_kj a_i,c+k,  C_kj = -sum_l cof_lk a_c+l,j
// (adj(A11) = cof^T), and det(trailing) = D3 det(D3 S) / D3^m, m = n - c - 3.
// Each element costs four products and one REDC (redc4, any p < 2^31) for
// three steps; each column three REDCs of three products per triple of
// steps.  Fewer than three steps left: Fast2Step finishes.  A zero D3 is
// only recorded, as in Fast2Step.
template <int NN, int T, int c>
struct Fast3Step {
  static constexpr int M = (NN + T - 1) / T;
  static constexpr int S = ColLayout<NN, T>::S;
  static PD_D uint32_t bcast(uint32_t v, int owner) {
    return (T == 1) ? v : __shfl_sync(PD_FULL, v, owner, T);
  }
  static PD_D uint32_t neg(uint32_t v, uint32_t p) { return v ? p - v : 0u; }
  static PD_D void run(uint32_t (&a)[M][NN], uint32_t p, uint32_t pinv, uint32_t &Q,
                       uint32_t &den, bool &zero) {
    if constexpr (NN - c < 3) {
      Fast2Step<NN, T, c>::run(a, p, pinv, Q, den, zero);
    } else {
      constexpr int o0 = (c + S) % T, m0 = (c + S) / T;
      constexpr int o1 = (c + 1 + S) % T, m1 = (c + 1 + S) / T;
      constexpr int o2 = (c + 2 + S) % T, m2 = (c + 2 + S) / T;
      // A11[k][l] = a_{c+k, c+l}: column c+l is held by owner o_l in slot m_l
      const uint32_t a00 = bcast(a[m0][c], o0), a10 = bcast(a[m0][c + 1], o0), a20 = bcast(a[m0][c + 2], o0);
      const uint32_t a01 = bcast(a[m1][c], o1), a11 = bcast(a[m1][c + 1], o1), a21 = bcast(a[m1][c + 2], o1);
      const uint32_t a02 = bcast(a[m2][c], o2), a12 = bcast(a[m2][c + 1], o2), a22 = bcast(a[m2][c + 2], o2);
      const uint32_t c00 = mfms(a11, a22, a12, a21, p, pinv), c01 = mfms(a12, a20, a10, a22, p, pinv),
                     c02 = mfms(a10, a21, a11, a20, p, pinv);
      const uint32_t c10 = mfms(a02, a21, a01, a22, p, pinv), c11 = mfms(a00, a22, a02, a20, p, pinv),
                     c12 = mfms(a01, a20, a00, a21, p, pinv);
      const uint32_t c20 = mfms(a01, a12, a02, a11, p, pinv), c21 = mfms(a02, a10, a00, a12, p, pinv),
                     c22 = mfms(a00, a11, a01, a10, p, pinv);
      const uint32_t d3 = redc4((uint64_t)a00 * c00 + (uint64_t)a01 * c01 + (uint64_t)a02 * c02, p, pinv);
      zero |= (d3 == 0u);
      const uint32_t q2 = mmul(Q, Q, p, pinv);
      den = mmul(den, mmul(q2, Q, p, pinv), p, pinv);
      Q = mmul(Q, d3, p, pinv);
      if constexpr (c + 3 < NN) {
        // C_kj = -(cof_0k v_0 + cof_1k v_1 + cof_2k v_2), v_l = a_{c+l, j}
        const uint32_t n00 = neg(c00, p), n10 = neg(c10, p), n20 = neg(c20, p);
        const uint32_t n01 = neg(c01, p), n11 = neg(c11, p), n21 = neg(c21, p);
        const uint32_t n02 = neg(c02, p), n12 = neg(c12, p), n22 = neg(c22, p);
        uint32_t k0[M], k1[M], k2[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          if (T * m + T - 1 - S > c + 2) {
            const uint32_t v0 = a[m][c], v1 = a[m][c + 1], v2 = a[m][c + 2];
            k0[m] = redc4((uint64_t)n00 * v0 + (uint64_t)n10 * v1 + (uint64_t)n20 * v2, p, pinv);
            k1[m] = redc4((uint64_t)n01 * v0 + (uint64_t)n11 * v1 + (uint64_t)n21 * v2, p, pinv);
            k2[m] = redc4((uint64_t)n02 * v0 + (uint64_t)n12 * v1 + (uint64_t)n22 * v2, p, pinv);
          }
        }
#pragma unroll
        for (int i = c + 3; i < NN; ++i) {
          const uint32_t b0 = bcast(a[m0][i], o0), b1 = bcast(a[m1][i], o1), b2 = bcast(a[m2][i], o2);
#pragma unroll
          for (int m = 0; m < M; ++m) {
            if (T * m + T - 1 - S > c + 2)
              a[m][i] = redc4((uint64_t)d3 * a[m][i] + (uint64_t)k0[m] * b0 + (uint64_t)k1[m] * b1 +
                                  (uint64_t)k2[m] * b2, p, pinv);
          }
        }
        Fast3Step<NN, T, c + 3>::run(a, p, pinv, Q, den, zero);
      }
    }
  }
};

// The pivoting elimination of one matrix read again from `base` (entry
// (i, j) at base[off[i NN + j]]).  Kept out of line so that the rare redo
// does not add to the register pressure of the fast pass.
template <int NN, int T>
__device__ __noinline__ uint2 elim_search(const uint32_t *base, const int64_t *off, int t, ModP md) {
  constexpr int M = (NN + T - 1) / T;
  uint32_t a[M][NN];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = col_of<NN, T>(t, m);
#pragma unroll
    for (int i = 0; i < NN; ++i) a[m][i] = (j >= 0) ? base[off[i * NN + j]] : 0u;
  }
  uint32_t Q = md.r1, den = md.r1;
  ElimStep<NN, T, 0>::run(a, t, md.p, md.pinv, Q, den);
  return make_uint2(Q, den);
}

// G nodes per prime (node g of prime slot q: entry (i, j) at
// evals[q prime_words + (g / rowlen) rowstride + g % rowlen + off[i n + j]]);
// determinant of node g of prime slot q to detvals[q det_stride + g].
template <int NN, int T, int MINB, int TH>
__global__ void __launch_bounds__(TH, MINB) condense_kernel(const uint32_t *__restrict__ evals,
                                                       uint32_t *__restrict__ detvals, int64_t G,
                                                       int64_t det_stride, EvLayout lay,
                                                       int64_t prime_words,
                                                       const ModP *__restrict__ mod,
                                                       const uint32_t *__restrict__ rn,
                                                       int prime_lo,
                                                       const __grid_constant__ EntryOff<NN> off) {
  constexpr int M = (NN + T - 1) / T;
  const int qrel = blockIdx.y;
  const int q = prime_lo + qrel;
  const ModP md = mod[q];
  const uint32_t p = md.p, pinv = md.pinv;
  const int t = (int)(threadIdx.x & (T - 1));
  const int64_t g = ((int64_t)blockIdx.x * TH + threadIdx.x) / T;
  const bool active = g < G;
  const int64_t gg = active ? g : (G - 1);
  const int64_t row = gg / lay.rowlen;
  const uint32_t *base = evals + (int64_t)qrel * prime_words + row * lay.rowstride + (gg - row * lay.rowlen);

  uint32_t a[M][NN];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = col_of<NN, T>(t, m);
#pragma unroll
    for (int i = 0; i < NN; ++i) a[m][i] = (j >= 0) ? __ldg(base + off.o[i * NN + j]) : 0u;
  }

  uint32_t Q = md.r1, den = md.r1;
  bool zero = false;
  constexpr int STEP = kStep[NN];
  if constexpr (STEP == 3) {
    Fast3Step<NN, T, 0>::run(a, p, pinv, Q, den, zero);
  } else {
    Fast2Step<NN, T, 0>::run(a, p, pinv, Q, den, zero);
    // the two-step pass needs p <= PD_FOLD3_MAX: larger primes (only plans of
    // more than 67 primes reach them) redo every matrix with the pivoting
    // elimination (the fast pass is not skipped: a branch around it costs
    // the common case its register allocation)
    zero |= p > PD_FOLD3_MAX;
  }
  if (__any_sync(PD_FULL, zero)) {  // some matrix of this warp met a zero pivot
    const uint2 qd = elim_search<NN, T>(base, off.o, t, md);
    Q = qd.x;
    den = qd.y;
  }
  // Every lane of a team holds the same (Q, den): hand them to one lane per
  // determinant so that the CTA's inversions run once each, in as few warps
  // as possible, and the results are stored contiguously.
  __shared__ uint32_t fin_q[TH], fin_d[TH];
  constexpr int S = TH / T;
  const int team = threadIdx.x / T;
  if (t == 0) {
    fin_q[team] = Q;
    fin_d[team] = den;
  }
  __syncthreads();
  if ((int)threadIdx.x < S) {
    const int64_t gd = (int64_t)blockIdx.x * S + threadIdx.x;
    if (gd < G)
      detvals[(int64_t)qrel * det_stride + gd] = finish_det(fin_q[threadIdx.x], fin_d[threadIdx.x], md, rn[q]);
  }
  (void)active;
}

template <int NN>
struct TeamFor {
  static constexpr int value = kTeam[NN];      // lanes per matrix
  static constexpr int minb = kMinBlocks[NN];  // CTAs per SM the kernel is built for
  static constexpr int step = kStep[NN];       // steps per pass of the fast elimination
  static constexpr int threads = kThreads[NN]; // threads per CTA
};

// Dynamic shared memory that leaves room for at most `ctas` CTAs of the
// condensation kernel per SM (0: none reserved, residency set by registers).
// The kernel does not use it: it only keeps registers free for CTAs of other
// kernels running beside it (the batched form's first-variable passes).
static inline size_t condense_reserve_bytes(int ctas) {
  if (ctas <= 0) return 0;
  int dev = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
    return 0;
  return (size_t)per_sm / (size_t)(ctas + 1) + 1024;
}

template <int NN, int HI>
static int condense_dispatch(const polydet_plan_s *pl, const uint32_t *evals, EvLayout lay,
                             int64_t G, int64_t det_stride, int prime_lo, int nprimes,
                             uint32_t *detvals, int ctas_per_sm, cudaStream_t st) {
  if (pl->n == NN) {
    constexpr int T = TeamFor<NN>::value;
    constexpr int threads = TeamFor<NN>::threads;
    auto kern = condense_kernel<NN, T, TeamFor<NN>::minb, threads>;
    const size_t reserve = condense_reserve_bytes(ctas_per_sm);
    if (reserve) {
      static PdPerDevice attr;
      const int rc = pd_once_per_device(attr, [&] {
        PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        return POLYDET_OK;
      });
      if (rc) return rc;
    }
    const int64_t teams_per_cta = threads / T;
    EntryOff<NN> off;
    for (int e = 0; e < NN * NN; ++e) off.o[e] = (int64_t)pl->ent[e] * lay.entry;
    dim3 grid((unsigned)((G + teams_per_cta - 1) / teams_per_cta), (unsigned)nprimes);
    kern<<<grid, threads, reserve, st>>>(evals, detvals, G, det_stride, lay, (int64_t)pl->nent * lay.entry,
                                         pl->d_mod, pl->d_rn, prime_lo, off);
    PD_CUDA(cudaGetLastError());
    return POLYDET_OK;
  }
  if constexpr (NN < HI)
    return condense_dispatch<NN + 1, HI>(pl, evals, lay, G, det_stride, prime_lo, nprimes, detvals,
                                         ctas_per_sm, st);
  return POLYDET_EINVAL;
}
