// The arguments of one batched 1-D pass (ntt.cu) and the register-direct
// forward kernel for short inputs (Lin <= 8), kept in a header of their own
// so that launch shapes can be timed apart from the library.
#pragma once

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
  // register-direct kernel only: 0 = one grid row per item (blockIdx.y);
  // otherwise the number of items, and the grid's x axis runs over
  // (item, column, coset group) triples, so that short rows still fill whole
  // CTAs; each column's cosets are cut into flat_groups consecutive groups
  int flat_items, flat_groups;
  // forward passes: only output rows [row_lo, row_hi) are stored, as rows
  // 0 .. row_hi - row_lo of the output (row_hi = 0: all Lout rows).  The
  // register-direct kernel takes a window only in coset order, with row_lo
  // a multiple of the coset size
  int row_lo, row_hi;
  // items from zero_item_plus1 - 1 on read nothing and write zeros (the zero
  // entry of an entry map, one item past the evaluated ones); 0: none
  int zero_item_plus1;
};

// Output rows one column of a pass stores.
PD_HD int out_rows(const TxArgs &a) { return a.row_hi ? a.row_hi - a.row_lo : a.Lout; }

// Forward pass for short inputs (Lin <= 8).  The N outputs
// y_i = sum_{e<Lin} c_e w^(i e) are produced coset by coset: for
// i = j + (N/LP) t (LP = Lin rounded up to a power of two),
// y = DFT_LP(c_e w^(j e))[t] with the LP-th root psi = w^(N/LP): Lin - 1
// twiddle products and a register DFT of size LP per LP outputs, in which
// the LP - Lin inputs that are zero are folded away at compile time.  A
// thread owns CPT columns (kDirectThreads apart, so every store of a row
// stays coalesced) and loads each coset's twiddles once for all of them.
// With one column per thread the grid may instead run over (item, column,
// coset group) triples (TxArgs::flat_items): short rows then fill whole CTAs,
// and a pass with few columns in all spreads each column's cosets over
// several threads.
//
// The integer multiply pipe, which also executes much of the address and
// move arithmetic, bounds the pass together with the write bandwidth, so the
// loop is kept lean: the twiddle circle is staged in shared memory once per
// CTA and read with 32-bit indices, and the cosets whose rows are all stored
// go through one pointer per output row with the columns at fixed offsets
// from it, without per-store predicates; only the ragged last coset takes
// the predicated path.  Plans keep D_v <= n d_v, so with at most 8 inputs
// (d_v <= 7) and n <= 32 a circle has N <= 256 points; launch_pass sends
// anything longer to the shared-memory pass kernel.
constexpr int kDirectThreads = 256;
constexpr int kDirectTwSmem = 256;

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

// The outputs y[k][t] of coset j for the thread's CPT columns (TW(k): the
// twiddle w^k in Montgomery form).
template <int LIN, int CPT, class Tw>
PD_D void direct_coset(int j, const uint32_t (&c)[CPT][LIN], uint32_t (&y)[CPT][DirectLP<LIN>::value],
                       const Tw &TW, uint32_t r1, uint32_t r4, uint32_t psi1, uint32_t psi2, uint32_t psi3,
                       uint32_t p, uint32_t pinv) {
  constexpr int LP = DirectLP<LIN>::value;
  uint32_t w[LIN];
  w[0] = r1;
#pragma unroll
  for (int e = 1; e < LIN; ++e) w[e] = TW(j * e);
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    uint32_t z[LP];
    z[0] = c[k][0];
#pragma unroll
    for (int e = 1; e < LP; ++e) z[e] = (e < LIN) ? mmul(w[e], c[k][e], p, pinv) : 0u;
    if (LP == 1) {
      y[k][0] = z[0];
    } else if (LP == 2) {
      y[k][0] = add_z<false, LIN < 2>(z[0], z[1 % LP], p);
      y[k][1 % LP] = sub_z<false, LIN < 2>(z[0], z[1 % LP], p);
    } else if (LP == 4) {
      uint32_t x[4] = {z[0], z[1 % LP], z[2 % LP], z[3 % LP]}, yy[4];
      dft4<false, false, (LIN <= 2), (LIN <= 3)>(x, yy, r4, p, pinv);
#pragma unroll
      for (int t = 0; t < 4; ++t) y[k][t % LP] = yy[t];
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
      y[k][0] = addm(E[0], O[0], p);
      y[k][4 % LP] = subm(E[0], O[0], p);
      y[k][1 % LP] = addm(E[1], t1, p);
      y[k][5 % LP] = subm(E[1], t1, p);
      y[k][2 % LP] = addm(E[2], t2, p);
      y[k][6 % LP] = subm(E[2], t2, p);
      y[k][3 % LP] = addm(E[3], t3, p);
      y[k][7 % LP] = subm(E[3], t3, p);
    }
  }
}

// Cosets [jlo, jhi) of the thread's columns: the full ones (j < jfull)
// through the row pointers rp[t] = op[0] + toff[t] (fast_store: all CPT
// columns exist and lie kDirectThreads words apart in the output), the rest
// predicated per store.
template <int LIN, int CPT, class Tw>
PD_D void direct_cosets(const TxArgs &a, const Tw &TW, const uint32_t (&c)[CPT][LIN], uint32_t *(&op)[CPT],
                        bool fast_store, int jlo, int jhi, int64_t ostride, uint32_t r1, uint32_t p,
                        uint32_t pinv) {
  constexpr int LP = DirectLP<LIN>::value;
  const int N = a.N;
  const int J = N / LP;
  uint32_t r4 = 0u, psi1 = 0u, psi2 = 0u, psi3 = 0u;
  if (LP >= 4) r4 = TW(N >> 2);  // w^(N/4), a primitive 4th root
  if (LP == 8) {
    psi1 = TW(N >> 3);
    psi2 = r4;
    psi3 = TW(3 * (N >> 3));
  }
  // Natural order (olp <= 1): coset j holds rows j + J t, stored while
  // j < lim[t].  Coset order (olp == LP): coset j holds rows j LP + t, so
  // only the cosets of the stored rows are computed: those of
  // [row_lo, row_hi) (row_lo a multiple of LP), whose first one lands in
  // output row 0.
  const bool coset_rows = a.olp > 1;
  const int rhi = a.row_hi ? a.row_hi : a.Lout;
  int lim[LP];
  int64_t toff[LP];  // words from a coset's first row to its row t
#pragma unroll
  for (int t = 0; t < LP; ++t) {
    lim[t] = coset_rows ? rhi - t : a.Lout - J * t;
    toff[t] = (int64_t)(coset_rows ? t : J * t) * ostride;
  }
  const int64_t jstep = (int64_t)(coset_rows ? LP : 1) * ostride;  // next coset's first row
  int jfull = fast_store ? (coset_rows ? rhi / LP : a.Lout - J * (LP - 1)) : jlo;
  jfull = max(jlo, min(jhi, jfull));
  if (jfull > jlo) {
    uint32_t *rp[LP];
#pragma unroll
    for (int t = 0; t < LP; ++t) rp[t] = op[0] + toff[t];
    for (int j = jlo; j < jfull; ++j) {
      uint32_t y[CPT][LP];
      direct_coset<LIN, CPT>(j, c, y, TW, r1, r4, psi1, psi2, psi3, p, pinv);
#pragma unroll
      for (int t = 0; t < LP; ++t) {
#pragma unroll
        for (int k = 0; k < CPT; ++k) rp[t][k * kDirectThreads] = y[k][t];
        rp[t] += jstep;
      }
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) op[k] += (int64_t)(jfull - jlo) * jstep;
  }
  for (int j = jfull; j < jhi; ++j) {
    uint32_t y[CPT][LP];
    direct_coset<LIN, CPT>(j, c, y, TW, r1, r4, psi1, psi2, psi3, p, pinv);
    const int jr = coset_rows ? j * LP : j;  // compared with lim[t]
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      if (op[k]) {
#pragma unroll
        for (int t = 0; t < LP; ++t)
          if (jr < lim[t]) op[k][toff[t]] = y[k][t];
        op[k] += jstep;
      }
    }
  }
}

template <int LIN, int CPT>
__global__ void __launch_bounds__(kDirectThreads) coltx_direct_kernel(TxArgs a) {
  constexpr int LP = DirectLP<LIN>::value;
  __shared__ uint32_t s_tw[kDirectTwSmem];
  const int q = a.prime_lo + blockIdx.z;
  const uint32_t *tw = a.tw + (size_t)q * a.tw_len + a.tw_off;
  // every twiddle index used is below N (j < N / LP and e < LP), and
  // N <= kDirectTwSmem (launch_pass); staged before any thread leaves
  for (int i = threadIdx.x; i < a.N; i += kDirectThreads) s_tw[i] = __ldg(tw + i);
  __syncthreads();
  const ModP md = a.mod[q];
  const uint32_t p = md.p, pinv = md.pinv;
  const int64_t ncols = a.A * a.B;
  int64_t item, col0;
  int grp = 0;
  if (a.flat_items) {  // CPT == 1; items * ncols * groups < 2^31 (launch_pass)
    const int gc = (int)(blockIdx.x * kDirectThreads + threadIdx.x);
    if (gc >= a.flat_items * (int)ncols * a.flat_groups) return;
    const int pair = gc / a.flat_groups;
    grp = gc - pair * a.flat_groups;
    item = pair / (int)ncols;
    col0 = pair - item * ncols;
  } else {
    item = blockIdx.y;
    col0 = (int64_t)blockIdx.x * kDirectThreads * CPT + threadIdx.x;
    if (col0 >= ncols) return;
  }
  const int64_t in_base = (int64_t)blockIdx.z * a.in_prime_stride + item * a.in_item_stride;
  int64_t ostride;
  if (a.il_L)
    ostride = (a.B / a.il_L) * a.il_n2 * a.il_Lp;  // row r -> row index r * (B / L)
  else
    ostride = a.out_row ? a.out_row : a.B;
  uint32_t c[CPT][LIN];
  uint32_t *op[CPT];  // output row 0 of each column (null past the last column)
  bool all_cols = true;
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int64_t col = col0 + (int64_t)k * kDirectThreads;
    const bool ok = col < ncols;
    all_cols = all_cols && ok;
    const int64_t cc = ok ? col : col0;
    const int64_t aa = (a.A == 1) ? 0 : cc / a.B, bb = cc - aa * a.B;
    const bool zero_item = a.zero_item_plus1 && item >= a.zero_item_plus1 - 1;
#pragma unroll
    for (int e = 0; e < LIN; ++e) {
      const int64_t idx = in_base + (aa * LIN + e) * a.B + bb;
      c[k][e] = zero_item ? 0u
                          : (a.in_is_i32 ? reduce_i32(((const int32_t *)a.in)[idx], p)
                                         : ((const uint32_t *)a.in)[idx]);
    }
    int64_t obase;
    if (a.il_L)
      obase = (int64_t)blockIdx.z * a.out_prime_stride + ((bb / a.il_L) * a.il_n2 + item) * a.il_Lp +
              bb % a.il_L;
    else
      obase = (int64_t)blockIdx.z * a.out_prime_stride + item * a.out_item_stride +
              aa * out_rows(a) * ostride + bb;
    op[k] = ok ? a.out + obase : nullptr;
  }
  // with one block of columns (A == 1) and the plain layout, column k sits
  // k * kDirectThreads words after column 0 in every row
  const bool fast_store = all_cols && a.A == 1 && !a.il_L;
  const bool coset_rows = a.olp > 1;
  const int rhi = a.row_hi ? a.row_hi : a.Lout;
  const int jbeg = coset_rows ? a.row_lo / LP : 0;
  const int jend = coset_rows ? (rhi + LP - 1) / LP : a.N / LP;
  int jlo = jbeg, jhi = jend;  // this thread's cosets
  if (a.flat_items && a.flat_groups > 1) {
    const int nj = jend - jbeg;
    const int per = (nj + a.flat_groups - 1) / a.flat_groups;
    jlo = jbeg + min(nj, grp * per);
    jhi = jbeg + min(nj, (jlo - jbeg) + per);
    const int64_t jstep = (int64_t)(coset_rows ? LP : 1) * ostride;
#pragma unroll
    for (int k = 0; k < CPT; ++k)
      if (op[k]) op[k] += (jlo - jbeg) * jstep;
  }
  auto TW = [&](int k) -> uint32_t { return s_tw[k]; };  // w^k R: the whole circle
  direct_cosets<LIN, CPT>(a, TW, c, op, fast_store, jlo, jhi, ostride, md.r1, p, pinv);
}
