// Evaluation (Sec. 3.1, Algorithm 2) and interpolation (Sec. 3.3) as passes of
// one batched 1-D NTT kernel, one pass per variable.
//
// A pass views every batch item (one matrix entry, or one prime's determinant
// values) as a tensor [A][L][B] and transforms the middle axis: column (a, b)
// of Lin input values becomes Lout output values of the N-point NTT (zero
// padded when Lin < N, truncated when Lout < N).  Evaluating x_k first and
// x_1 last grows the tensor from [L_1..L_k] to [N_1..N_k] = G while every
// pass reads and writes whole 128-byte rows; this replaces the paper's
// transposition kernel and rotation of d (Algorithm 2, lines 8-13).
//
// A CTA owns Ct columns: it stages their Lin x Ct tile in shared memory in
// bit-reversed row order, runs the log2(N) radix-2 stages there (decimation
// in time; the output is in natural order) and writes Lout x Ct back.  Data
// are plain residues; twiddles are stored in Montgomery form so one REDC per
// butterfly gives a plain product.
#include <stdio.h>

#include "common.cuh"

struct TxArgs {
  const void *in;
  uint32_t *out;
  int64_t in_prime_stride, in_item_stride;
  int64_t out_prime_stride, out_item_stride;
  int64_t A, B;
  int Lin, Lout, N, logN;
  int Ct, logCt;
  int in_is_i32;
  int inverse;
  int prime_lo;
  const ModP *mod;
  const uint32_t *tw;
  int tw_len, tw_off;
  const uint32_t *ninv;
  int nvars, var;
  uint32_t *status;
  // interleaved output (partial evaluation, A == 1): element (r, b) of entry
  // e goes to ((r * (B / il_L) + b / il_L) * il_n2 + e) * il_Lp + b % il_L
  int il_L, il_Lp;
  int64_t il_n2;
};

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
    if (r < a.Lin && col < ncols) {
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
    if (r < a.Lout) {
      if (a.inverse) v = mmul(scale, v, md.p, md.pinv);
      const int64_t aa = col / a.B, bb = col - aa * a.B;
      if (a.il_L) {
        const int64_t row = (int64_t)r * (a.B / a.il_L) + bb / a.il_L;
        a.out[(int64_t)blockIdx.z * a.out_prime_stride + (row * a.il_n2 + blockIdx.y) * a.il_Lp +
              bb % a.il_L] = v;
      } else {
        a.out[out_base + (aa * a.Lout + r) * a.B + bb] = v;
      }
    } else if (a.inverse && v != 0u) {
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

static int launch_pass(TxArgs a, int items, int nprimes, cudaStream_t st) {
  // Ct: columns per CTA, a power of two with N * (Ct + 1) words <= 64 KB.
  int64_t ncols = a.A * a.B;
  int ct = 32;
  while (ct > 1 && (int64_t)a.N * (ct + 1) > 16384) ct >>= 1;
  while (ct > 1 && ct / 2 >= ncols) ct >>= 1;
  a.Ct = ct;
  a.logCt = ilog2(ct);
  size_t smem = (size_t)a.N * (ct + 1) * sizeof(uint32_t);
  static bool attr_set = false;
  if (!attr_set) {
    PD_CUDA(cudaFuncSetAttribute(coltx_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
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
  const void *cur_in = coeffs;
  int64_t cur_item = pl->E, cur_prime = 0;
  int cur_i32 = 1;
  for (int v = k - 1; v >= 0; --v) {
    TxArgs a = {};
    a.A = 1;
    for (int u = 0; u < v; ++u) a.A *= pl->d[u] + 1;
    a.B = 1;
    for (int u = v + 1; u < k; ++u) a.B *= pl->N[u];
    a.Lin = pl->d[v] + 1;
    a.N = pl->N[v];
    a.logN = pl->logN[v];
    a.Lout = a.N;
    a.in = cur_in;
    a.in_item_stride = cur_item;
    a.in_prime_stride = cur_prime;
    a.in_is_i32 = cur_i32;
    if (v % 2 == 0) {  // even passes land in the output array (slot G per entry)
      a.out = evals;
      a.out_item_stride = pl->G;
    } else {
      a.out = ws;
      a.out_item_stride = (int64_t)slot;
    }
    a.out_prime_stride = n2 * a.out_item_stride;
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
    int rc = launch_pass(a, (int)n2, np, st);
    if (rc) return rc;
    cur_in = a.out;
    cur_item = a.out_item_stride;
    cur_prime = a.out_prime_stride;
    cur_i32 = 0;
  }
  return POLYDET_OK;
}

extern "C" int polydet_interp(polydet_plan_t pl, const uint32_t *detvals, int lo, int hi,
                              uint32_t *residues, uint32_t *ws, void *stream) {
  if (check_range(pl, lo, hi) || !detvals || !residues) return POLYDET_EINVAL;
  if (pl->interp_ws_words && !ws) return POLYDET_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
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

uint64_t pd_partial_ws_words(const polydet_plan_s *pl) {
  // pass v >= 1 output per entry: prod_{u<v} L_u * prod_{v<=u<k-1} N_u * L_{k-1}
  const int k = pl->nvars;
  uint64_t best = 0;
  for (int v = 1; v <= k - 2; ++v) {
    uint64_t s = (uint64_t)(pl->d[k - 1] + 1);
    for (int u = 0; u < k - 1; ++u) s *= (u < v) ? (uint64_t)(pl->d[u] + 1) : (uint64_t)pl->N[u];
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
  for (int u = 0; u < k - 1; ++u) rows *= pl->N[u];
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
    for (int u = v + 1; u < k - 1; ++u) a.B *= pl->N[u];
    a.Lin = pl->d[v] + 1;
    a.N = pl->N[v];
    a.logN = pl->logN[v];
    a.Lout = a.N;
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
  return pd_launch_condense(pl, evals, lo, hi - lo, detvals, (cudaStream_t)stream);
}
