// Evaluation (Sec. 3.1, Algorithm 2) and interpolation (Sec. 3.3) as passes of
// one batched 1-D NTT kernel, one pass per variable.
//
// A pass views every batch item (one matrix entry, or one prime's determinant
// values) as a tensor [A][L][B] and transforms the middle axis: column (a, b)
// of Lin input values becomes Lout output values of the N-point NTT (zero
// padded when Lin < N, truncated when Lout < N).  Evaluating x_k first and
// x_1 last grows the tensor from [L_1..L_k] to [N_1..N_k] = G while every
// pass reads and writes whole 128-byte rows; this replaces the paper's
// transposition kernel and rotation of d (Algorithm 2).
//
// A CTA owns Ct columns: it stages their Lin x Ct tile in shared memory in
// bit-reversed row order, runs the log2(N) radix-2 stages there (decimation
// in time; the output is in natural order) and writes Lout x Ct back.  Data
// are plain residues; twiddles are stored in Montgomery form so one REDC per
// butterfly gives a plain product.
#include <stdio.h>

#include "common.cuh"
#include "ntt_direct.cuh"

__global__ void __launch_bounds__(256) coltx_kernel(TxArgs a) {
  extern __shared__ uint32_t sm[];
  const int q = a.prime_lo + blockIdx.z;
  const ModP md = a.mod[q];
  const int Ct = a.Ct, S = a.Ct + 1;  // padded row stride
  const int N = a.N;
  const int64_t ncols = a.A * a.B;
  const int64_t col0 = (int64_t)blockIdx.x * Ct;
  const int64_t in_base = (int64_t)blockIdx.z * a.in_prime_stride + (int64_t)blockIdx.y * a.in_item_stride;
  const int64_t out_base = (int64_t)blockIdx.z * a.out_prime_stride + (int64_t)blockIdx.y * a.out_item_stride;
  const bool rowmajor = (a.B == 1);  // columns are contiguous rows of the item
  const int tot = Ct * N;

  for (int f = threadIdx.x; f < tot; f += blockDim.x) {
    int r, c;
    if (rowmajor) {
      c = f >> a.logN;
      r = f & (N - 1);
    } else {
      r = f >> a.logCt;
      c = f & (Ct - 1);
    }
    const int64_t col = col0 + c;
    uint32_t v = 0;
    const bool zero_item = a.zero_item_plus1 && (int)blockIdx.y >= a.zero_item_plus1 - 1;
    if (r < a.Lin && col < ncols && !zero_item) {
      const int64_t aa = col / a.B, bb = col - aa * a.B;
      const int64_t idx = in_base + (aa * a.Lin + r) * a.B + bb;
      v = a.in_is_i32 ? reduce_i32(((const int32_t *)a.in)[idx], md.p) : ((const uint32_t *)a.in)[idx];
    }
    const int rr = a.logN ? (int)(__brev((unsigned)r) >> (32 - a.logN)) : 0;
    sm[rr * S + c] = v;
  }
  __syncthreads();

  const uint32_t *tw = a.tw + (size_t)q * a.tw_len + a.tw_off;
  for (int s = 0; s < a.logN; ++s) {
    const int h = 1 << s;
    const int step = N >> (s + 1);
    for (int j = threadIdx.x; j < (N >> 1) * Ct; j += blockDim.x) {
      const int c = j & (Ct - 1);
      const int bj = j >> a.logCt;
      const int pos = bj & (h - 1);
      const int i0 = ((bj >> s) << (s + 1)) + pos;
      const int i1 = i0 + h;
      const uint32_t w = __ldg(tw + pos * step);
      const uint32_t u = sm[i0 * S + c];
      const uint32_t t = mmul(w, sm[i1 * S + c], md.p, md.pinv);
      sm[i0 * S + c] = addm(u, t, md.p);
      sm[i1 * S + c] = subm(u, t, md.p);
    }
    __syncthreads();
  }

  const uint32_t scale = a.inverse ? a.ninv[q * a.nvars + a.var] : 0u;
  bool bad = false;
  for (int f = threadIdx.x; f < tot; f += blockDim.x) {
    int r, c;
    if (rowmajor) {
      c = f >> a.logN;
      r = f & (N - 1);
    } else {
      r = f >> a.logCt;
      c = f & (Ct - 1);
    }
    const int64_t col = col0 + c;
    if (col >= ncols) continue;
    uint32_t v = sm[r * S + c];
    // natural output index r -> its row in the node order (r = j + (N/L) t
    // is node j L + t)
    const int L = a.olp > 1 ? a.olp : 1;
    const int J = N / L;
    const int rk = (r % J) * L + r / J;
    const int rlo = a.row_lo, rhi = a.row_hi ? a.row_hi : a.Lout;
    if (rk >= rlo && rk < rhi) {
      if (a.inverse) v = mmul(scale, v, md.p, md.pinv);
      const int64_t aa = col / a.B, bb = col - aa * a.B;
      if (a.il_L) {
        const int64_t row = (int64_t)rk * (a.B / a.il_L) + bb / a.il_L;
        a.out[(int64_t)blockIdx.z * a.out_prime_stride + (row * a.il_n2 + blockIdx.y) * a.il_Lp +
              bb % a.il_L] = v;
      } else {
        const int64_t orow = a.out_row ? a.out_row : a.B;
        a.out[out_base + (aa * (rhi - rlo) + rk - rlo) * orow + bb] = v;
      }
    } else if (a.inverse && rk >= a.Lout && v != 0u) {
      bad = true;
    }
  }
  if (bad) atomicOr(a.status, POLYDET_STATUS_BOUND);
}

static int ilog2(int64_t x) {
  int l = 0;
  while (((int64_t)1 << l) < x) ++l;
  return l;
}

template <int CPT>
static int launch_direct(const TxArgs &a, int64_t ncols, int items, int nprimes, cudaStream_t st) {
  constexpr int TH = kDirectThreads;
  dim3 grid((unsigned)((ncols + TH * CPT - 1) / (TH * CPT)), (unsigned)items, (unsigned)nprimes);
  if (a.flat_items)
    grid = dim3((unsigned)((ncols * items * a.flat_groups + TH - 1) / TH), 1u, (unsigned)nprimes);
  switch (a.Lin) {
    case 1: coltx_direct_kernel<1, CPT><<<grid, TH, 0, st>>>(a); break;
    case 2: coltx_direct_kernel<2, CPT><<<grid, TH, 0, st>>>(a); break;
    case 3: coltx_direct_kernel<3, CPT><<<grid, TH, 0, st>>>(a); break;
    case 4: coltx_direct_kernel<4, CPT><<<grid, TH, 0, st>>>(a); break;
    case 5: coltx_direct_kernel<5, CPT><<<grid, TH, 0, st>>>(a); break;
    case 6: coltx_direct_kernel<6, CPT><<<grid, TH, 0, st>>>(a); break;
    case 7: coltx_direct_kernel<7, CPT><<<grid, TH, 0, st>>>(a); break;
    default: coltx_direct_kernel<8, CPT><<<grid, TH, 0, st>>>(a); break;
  }
  PD_CUDA(cudaGetLastError());
  return POLYDET_OK;
}

static int launch_pass(TxArgs a, int items, int nprimes, cudaStream_t st) {
  int64_t ncols = a.A * a.B;
  // short forward transforms over many columns: the register-direct kernel
  const int lp_in = a.Lin <= 1 ? 1 : a.Lin <= 2 ? 2 : a.Lin <= 4 ? 4 : 8;
  // rows of fewer than 8 columns (a job's first pass: B = 1) only with the
  // flattened grid below, and not into the interleaved partial layout
  const bool rows_ok = a.B >= 8 || (!a.il_L && ncols * items < ((int64_t)1 << 31) - 256);
  const bool window_ok = a.row_hi == 0 || (a.olp > 1 && a.olp == lp_in && a.row_lo % lp_in == 0);
  if (!a.inverse && a.Lin <= 8 && a.N <= kDirectTwSmem && rows_ok && window_ok &&
      (a.olp <= 1 || a.olp == lp_in)) {
    // columns per thread: more share each coset's twiddles, fewer leave
    // fewer idle lanes in the last CTA of a row of B columns (measured: two
    // per thread from rows of about 1000 columns on; four only for inputs of
    // at most five words, whose registers still allow two CTAs per SM)
    int cpt = a.B < 8 ? 1 : (ncols >= 8192 ? 4 : (ncols >= 1024 ? 2 : 1));
    if (cpt == 4 && a.Lin > 5) cpt = 2;
    // short rows (one column per thread): one grid axis over (item, column)
    // pairs, so that rows shorter than a CTA, or a row's last CTA, leave no
    // threads idle
    a.flat_items = (cpt == 1 && ncols * items < ((int64_t)1 << 31) - 256) ? items : 0;
    // few columns in all (a job's first pass): cut each column's cosets into
    // groups until the grid holds about 152 x 1024 threads
    a.flat_groups = 1;
    if (a.flat_items) {
      const int J = a.N / lp_in;
      const int rhi = a.row_hi ? a.row_hi : a.Lout;
      const int Jc = (a.olp > 1) ? (rhi + lp_in - 1) / lp_in - a.row_lo / lp_in : J;
      const int64_t base = ncols * items * nprimes;
      int64_t g = (152 * 1024 + base - 1) / base;
      g = std::min<int64_t>(g, Jc);
      while (g > 1 && ncols * items * g >= ((int64_t)1 << 31) - 256) --g;
      a.flat_groups = (int)std::max<int64_t>(1, g);
    }
    switch (cpt) {
      case 4: return launch_direct<4>(a, ncols, items, nprimes, st);
      case 2: return launch_direct<2>(a, ncols, items, nprimes, st);
      default: return launch_direct<1>(a, ncols, items, nprimes, st);
    }
  }
  // Ct: columns per CTA, a power of two with N * (Ct + 1) words <= 64 KB.
  int ct = 32;
  while (ct > 1 && (int64_t)a.N * (ct + 1) > 16384) ct >>= 1;
  while (ct > 1 && ct / 2 >= ncols) ct >>= 1;
  a.Ct = ct;
  a.logCt = ilog2(ct);
  size_t smem = (size_t)a.N * (ct + 1) * sizeof(uint32_t);
  static PdPerDevice attr;
  int rc = pd_once_per_device(attr, [] {
    PD_CUDA(cudaFuncSetAttribute(coltx_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    return POLYDET_OK;
  });
  if (rc) return rc;
  dim3 grid((unsigned)((ncols + ct - 1) / ct), (unsigned)items, (unsigned)nprimes);
  coltx_kernel<<<grid, 256, smem, st>>>(a);
  PD_CUDA(cudaGetLastError());
  return POLYDET_OK;
}

static int check_range(const polydet_plan_s *pl, int lo, int hi) {
  return (pl && lo >= 0 && hi <= pl->P && lo < hi) ? POLYDET_OK : POLYDET_EINVAL;
}

extern "C" int polydet_eval(polydet_plan_t pl, const int32_t *coeffs, int lo, int hi,
                            uint32_t *evals, uint32_t *ws, void *stream) {
  if (check_range(pl, lo, hi) || !coeffs || !evals) return POLYDET_EINVAL;
  if (pl->eval_ws_words && !ws) return POLYDET_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int k = pl->nvars, np = hi - lo;
  const int64_t n2 = (int64_t)pl->n * pl->n;
  const uint64_t slot = n2 ? pl->eval_ws_words / (uint64_t)n2 : 0;
  // with an entry map only the distinct entries are evaluated, and the zero
  // entry's slot is cleared
  const int64_t items = pl->nitems, nent = pl->nent;
  const void *cur_in = coeffs;
  int64_t cur_item = pl->E, cur_prime = 0;
  int cur_i32 = 1;
  for (int v = k - 1; v >= 0; --v) {
    TxArgs a = {};
    a.A = 1;
    for (int u = 0; u < v; ++u) a.A *= pl->d[u] + 1;
    a.B = 1;
    for (int u = v + 1; u < k; ++u) a.B *= pl->M[u];
    a.Lin = pl->d[v] + 1;
    a.N = pl->N[v];
    a.logN = pl->logN[v];
    a.Lout = pl->M[v];  // the first M_v nodes (in the plan's order) of the N_v-point transform
    a.olp = pl->LPo[v];
    a.in = cur_in;
    a.in_item_stride = cur_item;
    a.in_prime_stride = cur_prime;
    a.in_is_i32 = cur_i32;
    if (v % 2 == 0) {  // even passes land in the output array (slot G per entry)
      a.out = evals;
      a.out_item_stride = pl->G;
      a.out_prime_stride = nent * pl->G;
    } else {
      a.out = ws;
      a.out_item_stride = (int64_t)slot;
      a.out_prime_stride = items * a.out_item_stride;
    }
    a.inverse = 0;
    a.prime_lo = lo;
    a.mod = pl->d_mod;
    a.tw = pl->d_tw_fwd;
    a.tw_len = pl->tw_len;
    a.tw_off = pl->tw_off[v];
    a.ninv = pl->d_ninv;
    a.nvars = k;
    a.var = v;
    a.status = pl->d_status;
    // the last pass also writes the zero entry's slot (entry map): one more
    // item that reads nothing; earlier passes skip a map without entries
    int launch_items = (int)items;
    if (v == 0 && nent > items) {
      a.zero_item_plus1 = (int)items + 1;
      launch_items = (int)nent;
    }
    if (launch_items > 0) {
      int rc = launch_pass(a, launch_items, np, st);
      if (rc) return rc;
    }
    cur_in = a.out;
    cur_item = a.out_item_stride;
    cur_prime = a.out_prime_stride;
    cur_i32 = 0;
  }
  return POLYDET_OK;
}

// Node-grid interpolation of one variable (Sec. 3.3 on the node grid): every
// column (a, b) of the tensor [A][m][B] holds the values at the m nodes (in
// coset order: node k = j L + t is w^j psi^t, psi = w^(N/L)) of a polynomial
// P of degree < m in that variable; its coefficients replace them.  With
// P(x) = sum_{r<L} x^r Q_r(x^L) and x^L = z_j = w^(L j) on coset j:
//  1. per whole coset j < Jf: an inverse DFT of size L of its L values, times
//     L^-1 w^(-j r), gives Q_r(z_j) for every r;
//  2. per r: the Jf coefficients through z_0..z_{Jf-1} (inverse Vandermonde
//     of size Jf: Jf^2 L products instead of m^2);
//  3. the s = m - Jf L nodes of the last coset fix the top coefficient
//     lambda_r of Q_r for r < s (Q_r = interpolant + lambda_r Pi, Pi =
//     prod_j (z - z_j)): an s x s solve after subtracting the known part.
// A CTA stages Ct columns; every phase runs over (row, column) items.
struct CiArgs {
  const uint32_t *in;
  uint32_t *out;
  int64_t in_prime_stride, out_prime_stride;
  int64_t A, B;
  int m, Jf, s, Ct;
  int prime_lo;
  const ModP *mod;
  const uint32_t *tab;  // this variable's tables for prime 0
  int tab_len;          // words per prime
};

// Sum of two products of residues reduced once (2 p^2 < p 2^32).
PD_D uint32_t mac2(uint32_t a0, uint32_t b0, uint32_t a1, uint32_t b1, uint32_t p, uint32_t pinv) {
  return redc((uint64_t)a0 * b0 + (uint64_t)a1 * b1, p, pinv);
}

// sum_{j<len} x[j] y[j s] / R mod p (x from global memory, y from shared
// memory with stride s): four products per REDC (redc4: 4 p^2 < p 2^32 for
// any p < 2^31), then pairs and a single one for the tail.
PD_D uint32_t dot_strided(const uint32_t *x, const uint32_t *y, int s, int len, uint32_t p, uint32_t pinv) {
  uint32_t acc = 0u;
  int j = 0;
  for (; j + 3 < len; j += 4)
    acc = addm(acc,
               redc4((uint64_t)__ldg(x + j) * y[j * s] + (uint64_t)__ldg(x + j + 1) * y[(j + 1) * s] +
                         (uint64_t)__ldg(x + j + 2) * y[(j + 2) * s] + (uint64_t)__ldg(x + j + 3) * y[(j + 3) * s],
                     p, pinv),
               p);
  for (; j + 1 < len; j += 2) acc = addm(acc, mac2(__ldg(x + j), y[j * s], __ldg(x + j + 1), y[(j + 1) * s], p, pinv), p);
  if (j < len) acc = addm(acc, mmul(__ldg(x + j), y[j * s], p, pinv), p);
  return acc;
}

// X_r = sum_t x_t rho^(t r) for L in {1, 2, 4, 8}; rk[k] = rho^k (Montgomery).
template <int L>
PD_D void small_dft(uint32_t (&x)[L], const uint32_t *rk, uint32_t p, uint32_t pinv) {
  if constexpr (L == 2) {
    const uint32_t a = x[0], b = x[1];
    x[0] = addm(a, b, p);
    x[1] = subm(a, b, p);
  } else if constexpr (L == 4) {
    uint32_t y[4], xx[4] = {x[0], x[1], x[2], x[3]};
    dft4<false, false, false, false>(xx, y, __ldg(rk + 1), p, pinv);
#pragma unroll
    for (int r = 0; r < 4; ++r) x[r] = y[r];
  } else if constexpr (L == 8) {
    uint32_t xe[4] = {x[0], x[2], x[4], x[6]}, xo[4] = {x[1], x[3], x[5], x[7]}, E[4], O[4];
    const uint32_t r2 = __ldg(rk + 2);
    dft4<false, false, false, false>(xe, E, r2, p, pinv);
    dft4<false, false, false, false>(xo, O, r2, p, pinv);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint32_t o = r ? mmul(__ldg(rk + r), O[r], p, pinv) : O[r];
      x[r] = addm(E[r], o, p);
      x[r + 4] = subm(E[r], o, p);
    }
  }
}

template <int L>
__global__ void __launch_bounds__(256) cinterp_kernel(CiArgs a) {
  extern __shared__ uint32_t sm[];
  const int q = a.prime_lo + blockIdx.z;
  const ModP md = a.mod[q];
  const uint32_t p = md.p, pinv = md.pinv;
  const int m = a.m, Jf = a.Jf, s = a.s, Ct = a.Ct, S = Ct + 1;
  const int64_t ncols = a.A * a.B;
  const int64_t col0 = (int64_t)blockIdx.x * Ct;
  const uint32_t *in = a.in + (int64_t)blockIdx.z * a.in_prime_stride;
  uint32_t *out = a.out + (int64_t)blockIdx.z * a.out_prime_stride;
  const uint32_t *tab = a.tab + (size_t)q * a.tab_len;
  const uint32_t *VfInv = tab;
  const uint32_t *tw1 = VfInv + Jf * Jf;
  const uint32_t *rk = tw1 + Jf * L;
  const uint32_t *H = rk + L;
  const uint32_t *Bm = H + s * L * Jf;
  const uint32_t *pic = Bm + s * s;
  uint32_t *Y = sm;                      // [m][S]   node values
  uint32_t *Qv = Y + (size_t)m * S;      // [L][Jf][S] Q_r(z_j)
  uint32_t *Qt = Qv + (size_t)L * Jf * S;  // [L][Jf + 1][S] coefficients of Q_r
  uint32_t *Dv = Qt + (size_t)L * (Jf + 1) * S;  // [s][L][S] partial sums, then [s][S] residuals
  const int tid = threadIdx.x, bd = blockDim.x;

  for (int f = tid; f < m * Ct; f += bd) {
    const int r = f / Ct, c = f - r * Ct;
    const int64_t col = col0 + c;
    uint32_t v = 0u;
    if (col < ncols) {
      const int64_t aa = col / a.B, bb = col - aa * a.B;
      v = in[(aa * m + r) * a.B + bb];
    }
    Y[r * S + c] = v;
  }
  __syncthreads();
  // 1. inverse DFT of each whole coset, twisted: Qv[r][j] = Q_r(z_j)
  for (int f = tid; f < Jf * Ct; f += bd) {
    const int j = f / Ct, c = f - j * Ct;
    uint32_t x[L];
#pragma unroll
    for (int t = 0; t < L; ++t) x[t] = Y[(j * L + t) * S + c];
    small_dft<L>(x, rk, p, pinv);
#pragma unroll
    for (int r = 0; r < L; ++r) Qv[(r * Jf + j) * S + c] = mmul(x[r], __ldg(tw1 + j * L + r), p, pinv);
  }
  __syncthreads();
  // 2. Qt[r][u] = sum_j VfInv[u][j] Qv[r][j]; Qt[r][Jf] = 0
  for (int f = tid; f < L * (Jf + 1) * Ct; f += bd) {
    const int ru = f / Ct, c = f - ru * Ct;
    const int r = ru / (Jf + 1), u = ru - r * (Jf + 1);
    Qt[ru * S + c] = (u < Jf) ? dot_strided(VfInv + u * Jf, Qv + (size_t)r * Jf * S + c, S, Jf, p, pinv) : 0u;
  }
  __syncthreads();
  if (s > 0) {
    // 3a. partial sums of the known part at the last coset's nodes
    for (int f = tid; f < s * L * Ct; f += bd) {
      const int tr = f / Ct, c = f - tr * Ct;
      const int r = tr % L;
      Dv[tr * S + c] = dot_strided(H + tr * Jf, Qt + (size_t)r * (Jf + 1) * S + c, S, Jf, p, pinv);
    }
    __syncthreads();
    // 3b. residuals d_t = y_{Jf L + t} - sum_r partial[t][r] (into row t L)
    for (int f = tid; f < s * Ct; f += bd) {
      const int t = f / Ct, c = f - t * Ct;
      uint32_t k = 0u;
      for (int r = 0; r < L; ++r) k = addm(k, Dv[(t * L + r) * S + c], p);
      Dv[(t * L) * S + c] = subm(Y[(Jf * L + t) * S + c], k, p);
    }
    __syncthreads();
    // 3c. lambda_r = sum_t B[r][t] d_t, then Qt[r][u] += lambda_r pi_u (r < s)
    for (int f = tid; f < s * Ct; f += bd) {
      const int r = f / Ct, c = f - r * Ct;
      uint32_t lam = 0u;
      for (int t = 0; t < s; ++t) lam = addm(lam, mmul(__ldg(Bm + r * s + t), Dv[(t * L) * S + c], p, pinv), p);
      Y[r * S + c] = lam;  // the node values are no longer needed (rows < s <= m)
    }
    __syncthreads();
    for (int f = tid; f < s * (Jf + 1) * Ct; f += bd) {
      const int ru = f / Ct, c = f - ru * Ct;
      const int r = ru / (Jf + 1), u = ru - r * (Jf + 1);
      Qt[ru * S + c] = addm(Qt[ru * S + c], mmul(Y[r * S + c], __ldg(pic + u), p, pinv), p);
    }
    __syncthreads();
  }
  // 4. coefficient e = L u + r of each column is Qt[r][u]
  for (int f = tid; f < m * Ct; f += bd) {
    const int e = f / Ct, c = f - e * Ct;
    const int64_t col = col0 + c;
    if (col >= ncols) continue;
    const int r = e % L, u = e / L;
    const int64_t aa = col / a.B, bb = col - aa * a.B;
    out[(aa * m + e) * a.B + bb] = Qt[(r * (Jf + 1) + u) * S + c];
  }
}

static size_t cinterp_rows(int m, int L) {
  const int Jf = m / L, s = m % L;
  return (size_t)m + (size_t)L * Jf + (size_t)L * (Jf + 1) + (size_t)s * L;
}

static int interp_nodes(polydet_plan_t pl, const uint32_t *detvals, int lo, int hi,
                        uint32_t *residues, uint32_t *ws, cudaStream_t st) {
  const int k = pl->nvars, np = hi - lo;
  const uint64_t slot = pl->interp_ws_words / 2;
  constexpr size_t kMaxSmem = 200 * 1024;
  int dev = 0, sms = 0;
  PD_CUDA(cudaGetDevice(&dev));
  PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  static PdPerDevice attr;
  const int arc = pd_once_per_device(attr, [] {
    PD_CUDA(cudaFuncSetAttribute(cinterp_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PD_CUDA(cudaFuncSetAttribute(cinterp_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PD_CUDA(cudaFuncSetAttribute(cinterp_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    PD_CUDA(cudaFuncSetAttribute(cinterp_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    return POLYDET_OK;
  });
  if (arc) return arc;
  const uint32_t *cur = detvals;
  int64_t cur_prime = pl->G;
  int t = 0;
  for (int v = k - 1; v >= 0; --v, ++t) {
    CiArgs a = {};
    a.A = 1;
    for (int u = 0; u < v; ++u) a.A *= pl->M[u];
    a.B = 1;
    for (int u = v + 1; u < k; ++u) a.B *= pl->M[u];
    const int L = pl->LPo[v];
    a.m = pl->M[v];
    a.Jf = a.m / L;
    a.s = a.m % L;
    const size_t rows = cinterp_rows(a.m, L);
    int ct = 32;
    while (ct > 1 && rows * (ct + 1) * sizeof(uint32_t) > 48 * 1024) ct >>= 1;
    while (ct > 1 && ct / 2 >= a.A * a.B) ct >>= 1;
    // small passes (a job's few columns): fewer columns per CTA, so that the
    // grid still spreads over the SMs (two CTAs each) and every CTA's
    // phases, which run one after another, are short
    while (ct > 4 && (a.A * a.B + ct - 1) / ct * np < 2 * sms) ct >>= 1;
    if (rows * (ct + 1) * sizeof(uint32_t) > kMaxSmem) return POLYDET_EINVAL;
    a.Ct = ct;
    a.in = cur;
    a.in_prime_stride = cur_prime;
    if (v == 0) {
      a.out = residues;
      a.out_prime_stride = pl->C;
    } else {
      a.out = ws + (uint64_t)(t % 2) * slot * (uint64_t)np;
      a.out_prime_stride = (int64_t)slot;
    }
    a.prime_lo = lo;
    a.mod = pl->d_mod;
    a.tab = pl->d_itab + pl->itab_off[v];
    a.tab_len = pl->itab_len;
    const size_t smem = rows * (ct + 1) * sizeof(uint32_t);
    dim3 grid((unsigned)((a.A * a.B + ct - 1) / ct), 1, (unsigned)np);
    switch (L) {
      case 1: cinterp_kernel<1><<<grid, 256, smem, st>>>(a); break;
      case 2: cinterp_kernel<2><<<grid, 256, smem, st>>>(a); break;
      case 4: cinterp_kernel<4><<<grid, 256, smem, st>>>(a); break;
      default: cinterp_kernel<8><<<grid, 256, smem, st>>>(a); break;
    }
    PD_CUDA(cudaGetLastError());
    cur = a.out;
    cur_prime = a.out_prime_stride;
  }
  return POLYDET_OK;
}

extern "C" int polydet_interp(polydet_plan_t pl, const uint32_t *detvals, int lo, int hi,
                              uint32_t *residues, uint32_t *ws, void *stream) {
  if (check_range(pl, lo, hi) || !detvals || !residues) return POLYDET_EINVAL;
  if (pl->interp_ws_words && !ws) return POLYDET_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!pl->full) return interp_nodes(pl, detvals, lo, hi, residues, ws, st);
  const int k = pl->nvars, np = hi - lo;
  const uint64_t slot = pl->interp_ws_words / 2;
  const void *cur_in = detvals;
  int64_t cur_prime = pl->G;
  int t = 0;
  for (int v = k - 1; v >= 0; --v, ++t) {
    TxArgs a = {};
    a.A = 1;
    for (int u = 0; u < v; ++u) a.A *= pl->N[u];
    a.B = 1;
    for (int u = v + 1; u < k; ++u) a.B *= pl->D[u] + 1;
    a.Lin = pl->N[v];
    a.N = pl->N[v];
    a.logN = pl->logN[v];
    a.Lout = pl->D[v] + 1;
    a.in = cur_in;
    a.in_item_stride = 0;
    a.in_prime_stride = cur_prime;
    a.in_is_i32 = 0;
    if (v == 0) {
      a.out = residues;
      a.out_prime_stride = pl->C;
    } else {
      a.out = ws + (uint64_t)(t % 2) * slot * (uint64_t)np;
      a.out_prime_stride = (int64_t)slot;
    }
    a.out_item_stride = 0;
    a.inverse = 1;
    a.prime_lo = lo;
    a.mod = pl->d_mod;
    a.tw = pl->d_tw_inv;
    a.tw_len = pl->tw_len;
    a.tw_off = pl->tw_off[v];
    a.ninv = pl->d_ninv;
    a.nvars = k;
    a.var = v;
    a.status = pl->d_status;
    int rc = launch_pass(a, 1, np, st);
    if (rc) return rc;
    cur_in = a.out;
    cur_prime = a.out_prime_stride;
  }
  return POLYDET_OK;
}

// Words per entry of the tensor after the passes of x_k, ..., x_{v+1}:
// prod_{u<=v} L_u * prod_{u>v} M_u (0-based v; L_u = d_u + 1).
static uint64_t words_after(const polydet_plan_s *pl, int v) {
  uint64_t s = 1;
  for (int u = 0; u < pl->nvars; ++u) s *= (u <= v) ? (uint64_t)(pl->d[u] + 1) : (uint64_t)pl->M[u];
  return s;
}

uint64_t pd_head_words(const polydet_plan_s *pl) { return words_after(pl, 0); }

uint64_t pd_head_ws_words(const polydet_plan_s *pl) {
  // passes v >= 2 with v even land in the scratch (so that v = 1 lands in head)
  uint64_t best = 0;
  for (int v = 2; v < pl->nvars; v += 2) best = std::max(best, words_after(pl, v - 1));
  return best * (uint64_t)pl->nitems;
}

__global__ void reduce_kernel(const int32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t len,
                              const ModP *__restrict__ mod, int lo) {
  const uint32_t p = mod[lo + blockIdx.y].p;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < len;
       f += (int64_t)gridDim.x * blockDim.x)
    out[(int64_t)blockIdx.y * len + f] = reduce_i32(in[f], p);
}

static TxArgs forward_pass(const polydet_plan_s *pl, int v, int lo) {
  TxArgs a = {};
  a.A = 1;
  for (int u = 0; u < v; ++u) a.A *= pl->d[u] + 1;
  a.B = 1;
  for (int u = v + 1; u < pl->nvars; ++u) a.B *= pl->M[u];
  a.Lin = pl->d[v] + 1;
  a.N = pl->N[v];
  a.logN = pl->logN[v];
  a.Lout = pl->M[v];
  a.olp = pl->LPo[v];
  a.inverse = 0;
  a.prime_lo = lo;
  a.mod = pl->d_mod;
  a.tw = pl->d_tw_fwd;
  a.tw_len = pl->tw_len;
  a.tw_off = pl->tw_off[v];
  a.ninv = pl->d_ninv;
  a.nvars = pl->nvars;
  a.var = v;
  a.status = pl->d_status;
  return a;
}

int pd_eval_head(const polydet_plan_s *pl, const int32_t *coeffs, int lo, int hi, uint32_t *head,
                 uint32_t *ws, cudaStream_t st) {
  if (check_range(pl, lo, hi)) return POLYDET_EINVAL;
  const int k = pl->nvars;
  const int64_t items = pl->nitems;
  if (items == 0) return POLYDET_OK;
  if (k == 1) {
    const int64_t len = items * pl->E;
    const unsigned blocks = (unsigned)std::min<int64_t>((len + 255) / 256, 4096);
    reduce_kernel<<<dim3(blocks, hi - lo), 256, 0, st>>>(coeffs, head, len, pl->d_mod, lo);
    PD_CUDA(cudaGetLastError());
    return POLYDET_OK;
  }
  const int64_t S1 = (int64_t)pd_head_words(pl);
  int64_t S2 = 0;
  for (int v = 2; v < k; v += 2) S2 = std::max<int64_t>(S2, (int64_t)words_after(pl, v - 1));
  const void *cur_in = coeffs;
  int64_t cur_item = pl->E, cur_prime = 0;
  int cur_i32 = 1;
  for (int v = k - 1; v >= 1; --v) {
    TxArgs a = forward_pass(pl, v, lo);
    a.in = cur_in;
    a.in_item_stride = cur_item;
    a.in_prime_stride = cur_prime;
    a.in_is_i32 = cur_i32;
    a.out = (v % 2) ? head : ws;
    a.out_item_stride = (v % 2) ? S1 : S2;
    a.out_prime_stride = items * a.out_item_stride;
    int rc = launch_pass(a, (int)items, hi - lo, st);
    if (rc) return rc;
    cur_in = a.out;
    cur_item = a.out_item_stride;
    cur_prime = a.out_prime_stride;
    cur_i32 = 0;
  }
  return POLYDET_OK;
}

EvLayout pd_tail_layout(const polydet_plan_s *pl, int rows) {
  const int64_t B = pl->G / pl->M[0];  // nodes of the other variables: one row
  const int64_t Bs = B >= 1024 ? (B + 31) / 32 * 32 : B;  // padding <= 3 % of a row
  return EvLayout{B, Bs, (int64_t)(rows > 0 ? rows : pl->M[0]) * Bs};
}

int pd_eval_tail(const polydet_plan_s *pl, const uint32_t *head, int head_q0, int lo, int hi,
                 int row_lo, int row_hi, uint32_t *evals, EvLayout lay, cudaStream_t st) {
  if (check_range(pl, lo, hi) || !head || !evals || lo < head_q0) return POLYDET_EINVAL;
  const int64_t items = pl->nitems, nent = pl->nent;
  const int64_t S1 = (int64_t)pd_head_words(pl);
  TxArgs a = forward_pass(pl, 0, lo);
  if (row_lo < 0 || row_hi > pl->M[0] || row_lo >= row_hi) return POLYDET_EINVAL;
  if (lay.rowlen != a.B || lay.entry != (int64_t)(row_hi - row_lo) * lay.rowstride) return POLYDET_EINVAL;
  if (row_lo > 0 || row_hi < pl->M[0]) {
    a.row_lo = row_lo;
    a.row_hi = row_hi;
  }
  if (nent > items) a.zero_item_plus1 = (int)items + 1;  // the zero entry's slot (entry map)
  a.in = head + (int64_t)(lo - head_q0) * items * S1;
  a.in_item_stride = S1;
  a.in_prime_stride = items * S1;
  a.in_is_i32 = 0;
  a.out = evals;
  a.out_row = lay.rowstride;
  a.out_item_stride = lay.entry;
  a.out_prime_stride = nent * lay.entry;
  return launch_pass(a, (int)nent, hi - lo, st);
}

uint64_t pd_partial_ws_words(const polydet_plan_s *pl) {
  // pass v >= 1 output per entry: prod_{u<v} L_u * prod_{v<=u<k-1} N_u * L_{k-1}
  const int k = pl->nvars;
  uint64_t best = 0;
  for (int v = 1; v <= k - 2; ++v) {
    uint64_t s = (uint64_t)(pl->d[k - 1] + 1);
    for (int u = 0; u < k - 1; ++u) s *= (u < v) ? (uint64_t)(pl->d[u] + 1) : (uint64_t)pl->M[u];
    if (s > best) best = s;
  }
  return 2 * best * (uint64_t)pl->n * pl->n;
}

int pd_eval_partial(const polydet_plan_s *pl, const int32_t *coeffs, int lo, int hi, uint32_t *out,
                    int Lp, uint32_t *ws, cudaStream_t st) {
  const int k = pl->nvars, np = hi - lo;
  if (k < 2) return POLYDET_EINVAL;
  const int64_t n2 = (int64_t)pl->n * pl->n;
  const int Lk = pl->d[k - 1] + 1;
  int64_t rows = 1;
  for (int u = 0; u < k - 1; ++u) rows *= pl->M[u];
  const uint64_t slot = pd_partial_ws_words(pl) / (2 * (uint64_t)n2);
  const void *cur_in = coeffs;
  int64_t cur_item = pl->E, cur_prime = 0;
  int cur_i32 = 1;
  int t = 0;
  for (int v = k - 2; v >= 0; --v, ++t) {
    TxArgs a = {};
    a.A = 1;
    for (int u = 0; u < v; ++u) a.A *= pl->d[u] + 1;
    a.B = Lk;
    for (int u = v + 1; u < k - 1; ++u) a.B *= pl->M[u];
    a.Lin = pl->d[v] + 1;
    a.N = pl->N[v];
    a.logN = pl->logN[v];
    a.Lout = pl->M[v];
    a.olp = pl->LPo[v];
    a.in = cur_in;
    a.in_item_stride = cur_item;
    a.in_prime_stride = cur_prime;
    a.in_is_i32 = cur_i32;
    if (v == 0) {
      a.out = out;
      a.out_prime_stride = rows * n2 * Lp;
      a.il_L = Lk;
      a.il_Lp = Lp;
      a.il_n2 = n2;
    } else {
      a.out = ws + (uint64_t)(t % 2) * slot * (uint64_t)n2 * (uint64_t)np;
      a.out_item_stride = (int64_t)slot;
      a.out_prime_stride = n2 * (int64_t)slot;
    }
    a.prime_lo = lo;
    a.mod = pl->d_mod;
    a.tw = pl->d_tw_fwd;
    a.tw_len = pl->tw_len;
    a.tw_off = pl->tw_off[v];
    a.ninv = pl->d_ninv;
    a.nvars = k;
    a.var = v;
    a.status = pl->d_status;
    int rc = launch_pass(a, (int)n2, np, st);
    if (rc) return rc;
    cur_in = a.out;
    cur_item = a.out_item_stride;
    cur_prime = a.out_prime_stride;
    cur_i32 = 0;
  }
  return POLYDET_OK;
}

extern "C" int polydet_condense_batch(polydet_plan_t pl, const uint32_t *evals, int lo, int hi,
                                      uint32_t *detvals, void *stream) {
  if (check_range(pl, lo, hi) || !evals || !detvals) return POLYDET_EINVAL;
  const EvLayout lay = {pl->G, pl->G, pl->G};
  return pd_launch_condense(pl, evals, lay, lo, hi - lo, detvals, (cudaStream_t)stream);
}

// Streamed evaluation + condensation (multi-round evaluation of Sec. 3.1):
// the workspace holds one prime's head tensor (every variable but x_1
// evaluated) and, after it, the head passes' scratch, which the slabs of
// evaluated matrices reuse once the head is complete.
static int stream_quantum(const polydet_plan_s *pl) {
  return pl->full ? 1 : pl->LPo[0];  // slab starts on a coset of x_1 (node grid)
}

static uint64_t stream_head_words(const polydet_plan_s *pl) {
  return ((uint64_t)pl->nitems * pd_head_words(pl) + 63) / 64 * 64;
}

extern "C" uint64_t polydet_stream_ws_words(polydet_plan_t pl, int rows) {
  if (!pl || rows < 1) return 0;
  const int qn = stream_quantum(pl);
  rows = std::min(pl->M[0], (rows + qn - 1) / qn * qn);
  const uint64_t slab = (uint64_t)pl->nent * (uint64_t)pd_tail_layout(pl, rows).entry;
  return stream_head_words(pl) + std::max<uint64_t>(pd_head_ws_words(pl), slab);
}

extern "C" int polydet_eval_condense(polydet_plan_t pl, const int32_t *coeffs, int lo, int hi,
                                     uint32_t *detvals, uint32_t *ws, uint64_t ws_words, void *stream) {
  if (check_range(pl, lo, hi) || !coeffs || !detvals || !ws) return POLYDET_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int qn = stream_quantum(pl), M0 = pl->M[0];
  const uint64_t hw = stream_head_words(pl);
  if (ws_words < polydet_stream_ws_words(pl, 1)) return POLYDET_EINVAL;
  // slab rows: as many as the workspace holds, a multiple of the coset size
  const uint64_t row_words = (uint64_t)pl->nent * (uint64_t)pd_tail_layout(pl, 1).entry;
  int R = (int)std::min<uint64_t>((uint64_t)M0, (ws_words - hw) / std::max<uint64_t>(row_words, 1));
  if (R < M0) R = std::max(qn, R / qn * qn);
  uint32_t *head = ws, *rest = ws + hw;
  const int64_t B = pl->G / M0;
  for (int q = lo; q < hi; ++q) {
    int rc = pd_eval_head(pl, coeffs, q, q + 1, head, rest, st);
    if (rc) return rc;
    for (int r0 = 0; r0 < M0; r0 += R) {
      const int r1 = std::min(M0, r0 + R);
      const EvLayout lay = pd_tail_layout(pl, r1 - r0);
      rc = pd_eval_tail(pl, head, q, q, q + 1, r0, r1, rest, lay, st);
      if (rc) return rc;
      rc = pd_launch_condense_nodes(pl, rest, lay, (int64_t)(r1 - r0) * B, pl->G, q, 1,
                                    detvals + (int64_t)(q - lo) * pl->G + (int64_t)r0 * B, st);
      if (rc) return rc;
    }
  }
  return POLYDET_OK;
}
