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
  // output row stride (words between rows r and r + 1 of a column); 0: B
  int64_t out_row;
  // node order of the output rows (forward passes): row k holds the value at
  // w^node_exp(k, N, olp); 0 or 1: natural order
  int olp;
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
    // natural output index r -> its row in the node order (r = j + (N/L) t
    // is node j L + t)
    const int L = a.olp > 1 ? a.olp : 1;
    const int J = N / L;
    const int rk = (r % J) * L + r / J;
    if (rk < a.Lout) {
      if (a.inverse) v = mmul(scale, v, md.p, md.pinv);
      const int64_t aa = col / a.B, bb = col - aa * a.B;
      if (a.il_L) {
        const int64_t row = (int64_t)rk * (a.B / a.il_L) + bb / a.il_L;
        a.out[(int64_t)blockIdx.z * a.out_prime_stride + (row * a.il_n2 + blockIdx.y) * a.il_Lp +
              bb % a.il_L] = v;
      } else {
        const int64_t orow = a.out_row ? a.out_row : a.B;
        a.out[out_base + (aa * a.Lout + rk) * orow + bb] = v;
      }
    } else if (a.inverse && v != 0u) {
      bad = true;
    }
  }
  if (bad) atomicOr(a.status, POLYDET_STATUS_BOUND);
}

// Forward pass for short inputs (Lin <= 8): no shared memory.  The N outputs
// y_i = sum_{e<Lin} c_e w^(i e) are produced coset by coset: for
// i = j + (N/LP) t (LP = Lin rounded up to a power of two),
// y = DFT_LP(c_e w^(j e))[t] with the LP-th root psi = w^(N/LP): Lin - 1
// twiddle products and a register DFT of size LP per LP outputs, in which
// the LP - Lin inputs that are zero are folded away at compile time.  A
// thread owns CPT columns (blockDim apart, so every store of a row stays
// coalesced) and loads each coset's twiddles once for all of them.
__device__ __forceinline__ uint32_t tw_pow(const uint32_t *tw, int k) {
  return __ldg(tw + k);  // w^k * R for 0 <= k < N: the table holds the whole circle
}

// x + y and x - y mod p where ZX / ZY say that x / y is known to be zero.
template <bool ZX, bool ZY>
PD_D uint32_t add_z(uint32_t x, uint32_t y, uint32_t p) {
  if (ZY) return x;
  if (ZX) return y;
  return addm(x, y, p);
}
template <bool ZX, bool ZY>
PD_D uint32_t sub_z(uint32_t x, uint32_t y, uint32_t p) {
  if (ZY) return x;
  if (ZX) return y ? p - y : 0u;
  return subm(x, y, p);
}

// DFT_4 of (x0, x1, x2, x3), xe known zero where Ze; r4 = primitive 4th root
// (Montgomery form).  y_t = sum_e x_e r4^(t e).
template <bool Z0, bool Z1, bool Z2, bool Z3>
PD_D void dft4(const uint32_t (&x)[4], uint32_t (&y)[4], uint32_t r4, uint32_t p, uint32_t pinv) {
  const uint32_t a0 = add_z<Z0, Z2>(x[0], x[2], p), a1 = sub_z<Z0, Z2>(x[0], x[2], p);
  constexpr bool ZA = Z0 && Z2, ZB = Z1 && Z3;
  const uint32_t b0 = add_z<Z1, Z3>(x[1], x[3], p);
  const uint32_t b1 = ZB ? 0u : mmul(r4, sub_z<Z1, Z3>(x[1], x[3], p), p, pinv);
  y[0] = add_z<ZA, ZB>(a0, b0, p);
  y[2] = sub_z<ZA, ZB>(a0, b0, p);
  y[1] = add_z<ZA, ZB>(a1, b1, p);
  y[3] = sub_z<ZA, ZB>(a1, b1, p);
}

template <int LIN>
struct DirectLP {
  static constexpr int value = LIN <= 1 ? 1 : LIN <= 2 ? 2 : LIN <= 4 ? 4 : 8;
};

template <int LIN, int CPT>
__global__ void __launch_bounds__(256) coltx_direct_kernel(TxArgs a) {
  constexpr int LP = DirectLP<LIN>::value;
  const int q = a.prime_lo + blockIdx.z;
  const ModP md = a.mod[q];
  const uint32_t p = md.p, pinv = md.pinv;
  const int64_t ncols = a.A * a.B;
  const int64_t col0 = (int64_t)blockIdx.x * blockDim.x * CPT + threadIdx.x;
  if (col0 >= ncols) return;
  const int64_t in_base = (int64_t)blockIdx.z * a.in_prime_stride + (int64_t)blockIdx.y * a.in_item_stride;
  const int N = a.N;
  const int J = N / LP;
  int64_t ostride;
  if (a.il_L)
    ostride = (a.B / a.il_L) * a.il_n2 * a.il_Lp;  // row r -> row index r * (B / L)
  else
    ostride = a.out_row ? a.out_row : a.B;
  uint32_t c[CPT][LIN];
  uint32_t *op[CPT];  // output row 0 of each column (null past the last column)
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t col = col0 + (int64_t)k * blockDim.x;
    const bool ok = col < ncols;
    const int64_t cc = ok ? col : col0;
    const int64_t aa = (a.A == 1) ? 0 : cc / a.B, bb = cc - aa * a.B;
#pragma unroll
    for (int e = 0; e < LIN; ++e) {
      const int64_t idx = in_base + (aa * LIN + e) * a.B + bb;
      c[k][e] = a.in_is_i32 ? reduce_i32(((const int32_t *)a.in)[idx], p) : ((const uint32_t *)a.in)[idx];
    }
    int64_t obase;
    if (a.il_L)
      obase = (int64_t)blockIdx.z * a.out_prime_stride + ((bb / a.il_L) * a.il_n2 + blockIdx.y) * a.il_Lp +
              bb % a.il_L;
    else
      obase = (int64_t)blockIdx.z * a.out_prime_stride + (int64_t)blockIdx.y * a.out_item_stride +
              aa * a.Lout * ostride + bb;
    op[k] = ok ? a.out + obase : nullptr;
  }
  const uint32_t *tw = a.tw + (size_t)q * a.tw_len + a.tw_off;
  uint32_t r4 = 0u, psi1 = 0u, psi2 = 0u, psi3 = 0u;
  if (LP >= 4) r4 = __ldg(tw + (N >> 2));  // w^(N/4), a primitive 4th root
  if (LP == 8) {
    psi1 = __ldg(tw + (N >> 3));
    psi2 = r4;
    psi3 = __ldg(tw + 3 * (N >> 3));
  }
  // Natural order (olp <= 1): coset j holds rows j + J t, stored while
  // j < lim[t].  Coset order (olp == LP): coset j holds rows j LP + t, so
  // only the first ceil(Lout / LP) cosets are computed.
  const bool coset_rows = a.olp > 1;
  const int Jc = coset_rows ? (a.Lout + LP - 1) / LP : J;
  int lim[LP];
  int64_t toff[LP];  // words from a coset's first row to its row t
#pragma unroll
  for (int t = 0; t < LP; ++t) {
    lim[t] = coset_rows ? a.Lout - t : a.Lout - J * t;
    toff[t] = (int64_t)(coset_rows ? t : J * t) * ostride;
  }
  const int64_t jstep = (int64_t)(coset_rows ? LP : 1) * ostride;  // next coset's first row
  for (int j = 0; j < Jc; ++j) {
    uint32_t w[LIN];
    w[0] = md.r1;
#pragma unroll
    for (int e = 1; e < LIN; ++e) w[e] = tw_pow(tw, j * e);

#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      uint32_t z[LP];
      z[0] = c[k][0];
#pragma unroll
      for (int e = 1; e < LP; ++e) z[e] = (e < LIN) ? mmul(w[e], c[k][e], p, pinv) : 0u;
      uint32_t y[LP];
      if (LP == 1) {
        y[0] = z[0];
      } else if (LP == 2) {
        y[0] = add_z<false, LIN < 2>(z[0], z[1], p);
        y[1] = sub_z<false, LIN < 2>(z[0], z[1], p);
      } else if (LP == 4) {
        uint32_t x[4] = {z[0], z[1], z[2], z[3 % LP]}, yy[4];
        dft4<false, false, (LIN <= 2), (LIN <= 3)>(x, yy, r4, p, pinv);
#pragma unroll
        for (int t = 0; t < 4; ++t) y[t] = yy[t];
      } else {
        // even and odd halves, then y_t = E_t + psi^t O_t, y_{t+4} = E_t - psi^t O_t
        uint32_t xe[4] = {z[0], z[2 % LP], z[4 % LP], z[6 % LP]};
        uint32_t xo[4] = {z[1 % LP], z[3 % LP], z[5 % LP], z[7 % LP]};
        uint32_t E[4], O[4];
        dft4<false, false, (LIN <= 4), (LIN <= 6)>(xe, E, r4, p, pinv);
        dft4<false, (LIN <= 3), (LIN <= 5), (LIN <= 7)>(xo, O, r4, p, pinv);
        const uint32_t t1 = mmul(psi1, O[1], p, pinv);
        const uint32_t t2 = mmul(psi2, O[2], p, pinv);
        const uint32_t t3 = mmul(psi3, O[3], p, pinv);
        y[0] = addm(E[0], O[0], p);
        y[4] = subm(E[0], O[0], p);
        y[1] = addm(E[1], t1, p);
        y[5] = subm(E[1], t1, p);
        y[2] = addm(E[2], t2, p);
        y[6] = subm(E[2], t2, p);
        y[3] = addm(E[3], t3, p);
        y[7] = subm(E[3], t3, p);
      }
      if (op[k]) {
        const int jr = coset_rows ? j * LP : j;  // compared with lim[t]
#pragma unroll
        for (int t = 0; t < LP; ++t)
          if (jr < lim[t]) op[k][toff[t]] = y[t];
        op[k] += jstep;
      }
    }
  }
}

static int ilog2(int64_t x) {
  int l = 0;
  while (((int64_t)1 << l) < x) ++l;
  return l;
}

template <int CPT>
static int launch_direct(const TxArgs &a, int64_t ncols, int items, int nprimes, cudaStream_t st) {
  dim3 grid((unsigned)((ncols + 256 * CPT - 1) / (256 * CPT)), (unsigned)items, (unsigned)nprimes);
  switch (a.Lin) {
    case 1: coltx_direct_kernel<1, CPT><<<grid, 256, 0, st>>>(a); break;
    case 2: coltx_direct_kernel<2, CPT><<<grid, 256, 0, st>>>(a); break;
    case 3: coltx_direct_kernel<3, CPT><<<grid, 256, 0, st>>>(a); break;
    case 4: coltx_direct_kernel<4, CPT><<<grid, 256, 0, st>>>(a); break;
    case 5: coltx_direct_kernel<5, CPT><<<grid, 256, 0, st>>>(a); break;
    case 6: coltx_direct_kernel<6, CPT><<<grid, 256, 0, st>>>(a); break;
    case 7: coltx_direct_kernel<7, CPT><<<grid, 256, 0, st>>>(a); break;
    default: coltx_direct_kernel<8, CPT><<<grid, 256, 0, st>>>(a); break;
  }
  PD_CUDA(cudaGetLastError());
  return POLYDET_OK;
}

static int launch_pass(TxArgs a, int items, int nprimes, cudaStream_t st) {
  int64_t ncols = a.A * a.B;
  // short forward transforms over many columns: the register-direct kernel
  const int lp_in = a.Lin <= 1 ? 1 : a.Lin <= 2 ? 2 : a.Lin <= 4 ? 4 : 8;
  if (!a.inverse && a.Lin <= 8 && a.B >= 8 && (a.olp <= 1 || a.olp == lp_in)) {
    // columns per thread: more share each coset's twiddles, fewer leave
    // fewer idle lanes in the last CTA of a row of B columns
    const int cpt = ncols >= 8192 ? 4 : (ncols >= 2048 ? 2 : 1);
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

// Node-grid interpolation of one variable: every column (a, b) of the tensor
// [A][m][B] holds the values at the nodes w^0..w^(m-1) of a polynomial of
// degree < m in that variable; its coefficients are V^-1 y (V the Vandermonde
// matrix of the nodes, its inverse in Montgomery form in `vinv`).  A CTA
// stages Ct columns x m values in shared memory; each thread then forms
// output coefficients as dot products with rows of V^-1, read by every lane
// of a warp at the same address (broadcast).
struct VmArgs {
  const uint32_t *in;
  uint32_t *out;
  int64_t in_prime_stride, out_prime_stride;
  int64_t A, B;
  int m, Ct;
  int prime_lo;
  const ModP *mod;
  const uint32_t *vinv;  // this variable's table for prime 0
  int vinv_len;          // words per prime
};

__global__ void __launch_bounds__(256) vmat_kernel(VmArgs a) {
  extern __shared__ uint32_t sm[];
  const int q = a.prime_lo + blockIdx.z;
  const ModP md = a.mod[q];
  const int m = a.m, Ct = a.Ct, S = Ct + 1;
  const int64_t ncols = a.A * a.B;
  const int64_t col0 = (int64_t)blockIdx.x * Ct;
  const uint32_t *in = a.in + (int64_t)blockIdx.z * a.in_prime_stride;
  uint32_t *out = a.out + (int64_t)blockIdx.z * a.out_prime_stride;
  for (int f = threadIdx.x; f < m * Ct; f += blockDim.x) {
    const int r = f / Ct, c = f - r * Ct;
    const int64_t col = col0 + c;
    uint32_t v = 0u;
    if (col < ncols) {
      const int64_t aa = col / a.B, bb = col - aa * a.B;
      v = in[(aa * m + r) * a.B + bb];
    }
    sm[r * S + c] = v;
  }
  __syncthreads();
  const uint32_t *V = a.vinv + (size_t)q * a.vinv_len;
  for (int f = threadIdx.x; f < m * Ct; f += blockDim.x) {
    const int e = f / Ct, c = f - e * Ct;
    const int64_t col = col0 + c;
    if (col >= ncols) continue;
    const uint32_t *row = V + (size_t)e * m;
    uint32_t acc = 0u;
    int i = 0;
    for (; i + 1 < m; i += 2) {  // two products per REDC: 2 p^2 < p 2^32
      const uint64_t s2 = (uint64_t)__ldg(row + i) * sm[i * S + c] +
                          (uint64_t)__ldg(row + i + 1) * sm[(i + 1) * S + c];
      acc = addm(acc, redc(s2, md.p, md.pinv), md.p);
    }
    if (i < m) acc = addm(acc, mmul(__ldg(row + i), sm[i * S + c], md.p, md.pinv), md.p);
    const int64_t aa = col / a.B, bb = col - aa * a.B;
    out[(aa * m + e) * a.B + bb] = acc;
  }
}

static int interp_nodes(polydet_plan_t pl, const uint32_t *detvals, int lo, int hi,
                        uint32_t *residues, uint32_t *ws, cudaStream_t st) {
  const int k = pl->nvars, np = hi - lo;
  const uint64_t slot = pl->interp_ws_words / 2;
  static bool attr_set = false;
  if (!attr_set) {
    PD_CUDA(cudaFuncSetAttribute(vmat_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  const uint32_t *cur = detvals;
  int64_t cur_prime = pl->G;
  int t = 0;
  for (int v = k - 1; v >= 0; --v, ++t) {
    VmArgs a = {};
    a.A = 1;
    for (int u = 0; u < v; ++u) a.A *= pl->M[u];
    a.B = 1;
    for (int u = v + 1; u < k; ++u) a.B *= pl->M[u];
    a.m = pl->M[v];
    int ct = 32;
    while (ct > 1 && (int64_t)a.m * (ct + 1) > 16384) ct >>= 1;
    while (ct > 1 && ct / 2 >= a.A * a.B) ct >>= 1;
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
    a.vinv = pl->d_vinv + pl->vinv_off[v];
    a.vinv_len = pl->vinv_len;
    const size_t smem = (size_t)a.m * (ct + 1) * sizeof(uint32_t);
    dim3 grid((unsigned)((a.A * a.B + ct - 1) / ct), 1, (unsigned)np);
    vmat_kernel<<<grid, 256, smem, st>>>(a);
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
  return best * (uint64_t)pl->n * pl->n * (uint64_t)pl->P;
}

__global__ void reduce_kernel(const int32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t len,
                              const ModP *__restrict__ mod) {
  const uint32_t p = mod[blockIdx.y].p;
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

int pd_eval_head(const polydet_plan_s *pl, const int32_t *coeffs, uint32_t *head, uint32_t *ws,
                 cudaStream_t st) {
  const int k = pl->nvars;
  const int64_t n2 = (int64_t)pl->n * pl->n;
  if (k == 1) {
    const int64_t len = n2 * pl->E;
    const unsigned blocks = (unsigned)std::min<int64_t>((len + 255) / 256, 4096);
    reduce_kernel<<<dim3(blocks, pl->P), 256, 0, st>>>(coeffs, head, len, pl->d_mod);
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
    TxArgs a = forward_pass(pl, v, 0);
    a.in = cur_in;
    a.in_item_stride = cur_item;
    a.in_prime_stride = cur_prime;
    a.in_is_i32 = cur_i32;
    a.out = (v % 2) ? head : ws;
    a.out_item_stride = (v % 2) ? S1 : S2;
    a.out_prime_stride = n2 * a.out_item_stride;
    int rc = launch_pass(a, (int)n2, pl->P, st);
    if (rc) return rc;
    cur_in = a.out;
    cur_item = a.out_item_stride;
    cur_prime = a.out_prime_stride;
    cur_i32 = 0;
  }
  return POLYDET_OK;
}

EvLayout pd_tail_layout(const polydet_plan_s *pl) {
  const int64_t B = pl->G / pl->M[0];  // nodes of the other variables: one row
  const int64_t Bs = B >= 1024 ? (B + 31) / 32 * 32 : B;  // padding <= 3 % of a row
  return EvLayout{B, Bs, (int64_t)pl->M[0] * Bs};
}

int pd_eval_tail(const polydet_plan_s *pl, const uint32_t *head, int lo, int hi, uint32_t *evals,
                 EvLayout lay, cudaStream_t st) {
  if (check_range(pl, lo, hi) || !head || !evals) return POLYDET_EINVAL;
  const int64_t n2 = (int64_t)pl->n * pl->n;
  const int64_t S1 = (int64_t)pd_head_words(pl);
  TxArgs a = forward_pass(pl, 0, lo);
  if (lay.rowlen != a.B || lay.entry != (int64_t)pl->M[0] * lay.rowstride) return POLYDET_EINVAL;
  a.in = head + (int64_t)lo * n2 * S1;
  a.in_item_stride = S1;
  a.in_prime_stride = n2 * S1;
  a.in_is_i32 = 0;
  a.out = evals;
  a.out_row = lay.rowstride;
  a.out_item_stride = lay.entry;
  a.out_prime_stride = n2 * lay.entry;
  return launch_pass(a, (int)n2, hi - lo, st);
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
