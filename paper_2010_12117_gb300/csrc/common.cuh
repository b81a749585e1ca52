// Internal definitions shared by the libpolydet translation units: the plan
// structure, host-side arithmetic, and the launchers of the separate
// translation units.  Device arithmetic is in modarith.cuh, the per-order
// launch table of the condensation kernels in teams.cuh.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/polydet.h"
#include "modarith.cuh"
#include "teams.cuh"

// ---------------------------------------------------------------------------
// Host-side arithmetic used while building plans.
// ---------------------------------------------------------------------------
static inline uint32_t h_mulmod(uint32_t a, uint32_t b, uint32_t p) {
  return (uint32_t)((uint64_t)a * b % p);
}
static inline uint32_t h_powmod(uint32_t a, uint64_t e, uint32_t p) {
  uint64_t r = 1 % p, x = a % p;
  while (e) {
    if (e & 1) r = r * x % p;
    x = x * x % p;
    e >>= 1;
  }
  return (uint32_t)r;
}
static inline uint32_t h_mont(uint32_t a, uint32_t p) {  // a * R mod p
  return (uint32_t)(((uint64_t)a << 32) % p);
}

// ---------------------------------------------------------------------------
// The plan.
// ---------------------------------------------------------------------------
struct polydet_plan_s {
  int n, nvars, P, W;
  int64_t E, G, C;
  int d[POLYDET_MAX_VARS], D[POLYDET_MAX_VARS], N[POLYDET_MAX_VARS], logN[POLYDET_MAX_VARS];
  // nodes per variable: D_v + 1 (node grid: the first D_v + 1 powers of w_v)
  // or N_v (full grid, POLYDET_FLAG_FULL_GRID); G = prod_v M_v
  int M[POLYDET_MAX_VARS];
  int LPo[POLYDET_MAX_VARS];  // node order: node k is w^(k / LPo + (N / LPo)(k mod LPo))
  int full;                        // 1: full power-of-two grid + inverse NTT
  int itab_off[POLYDET_MAX_VARS];  // node grid: offset of variable v's interpolation tables
  int itab_len;                    // node grid: their words per prime
  uint32_t *d_itab;                // [P][itab_len] (layout in plan.cu, Montgomery forms)
  int tw_len;                      // sum_v N_v: twiddles per prime
  uint32_t primes[POLYDET_MAX_PRIMES];
  uint32_t roots[POLYDET_MAX_PRIMES][POLYDET_MAX_VARS];
  ModP mod_h[POLYDET_MAX_PRIMES];   // host copies of the per-prime constants
  uint32_t rn_h[POLYDET_MAX_PRIMES];

  // device tables
  ModP *d_mod;            // [P]
  uint32_t *d_tw_fwd;     // [P][tw_len]  w^j * R, per variable at offset tw_off[v]
  uint32_t *d_tw_inv;     // [P][tw_len]  w^-j * R
  uint32_t *d_ninv;       // [P][nvars]   N_v^-1 * R
  uint32_t *d_rn;         // [P]          R^n mod p (condensation output scale)
  uint32_t *d_garner;     // [P][P]       (prod_{l<j} p_l mod p_i) * R, j < i; diagonal: c_i * R
  // host copies for the CRT kernels of P <= 32 (passed as kernel parameters):
  // crt_gs[i][j] = -(prod_{l<j} p_l) c_i * R mod p_i (j < i), crt_gs[i][i] = c_i * R,
  // so that alpha_i = x_i c_i - sum_{j<i} alpha_j (prod_{l<j} p_l) c_i is one dot product
  uint32_t crt_gs[32 * 32];
  uint32_t crt_mh[32], crt_mf[32];  // (M - 1) / 2 and M, limbs
  uint32_t *d_mhalf;      // [W] (M-1)/2
  uint32_t *d_mfull;      // [W] M
  uint32_t *d_status;     // 1 word
  int status_shared;      // 1: d_status belongs to a batch (one word for all its jobs)
  void *tables;           // the shape's shared device tables (plan.cu's cache entry)
  // entries: evaluated matrix entry e = i n + j of a node is entry ent[e] of
  // the evals tensor, which holds nent entries per prime; nitems of them are
  // evaluated from coefficients (all n^2 by default; with an entry map the U
  // distinct ones, and entry U is the zero entry)
  int ent[POLYDET_MAX_N * POLYDET_MAX_N];
  int nent, nitems;
  uint64_t eval_ws_words;   // caller scratch per prime for polydet_eval
  uint64_t interp_ws_words; // caller scratch per prime for polydet_interp
  int tw_off[POLYDET_MAX_VARS];
};

// Error plumbing shared by the translation units.
void pd_set_error(const char *what, cudaError_t e);
#define PD_CUDA(call)                        \
  do {                                       \
    cudaError_t _e = (call);                 \
    if (_e != cudaSuccess) {                 \
      pd_set_error(#call, _e);               \
      return POLYDET_ECUDA;                  \
    }                                        \
  } while (0)

// Plan construction (plan.cu); `shared_status`, when not null, is the status
// word the plan reports into (a batch's), else the plan allocates its own.
int pd_plan_impl(polydet_plan_t *out, int n, int nvars, const int32_t *entry_deg,
                 const int32_t *det_deg, int nprimes, uint32_t flags, uint32_t *shared_status);

// Per-device one-time set-up of a call site (kernel attributes such as the
// dynamic shared-memory limit are per device): runs `set` the first time the
// call site runs with a given device current, under a lock.
struct PdPerDevice {
  std::mutex mu;
  bool done[64] = {};
};
template <class F>
int pd_once_per_device(PdPerDevice &pd, F &&set) {
  int dev = 0;
  PD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return POLYDET_EINVAL;
  std::lock_guard<std::mutex> lock(pd.mu);
  if (pd.done[dev]) return POLYDET_OK;
  const int rc = set();
  if (rc == POLYDET_OK) pd.done[dev] = true;
  return rc;
}

// Launchers implemented in separate translation units.
// Where node g's evaluated matrix sits: entry e of node g of prime slot q at
// q * n^2 * entry + e * entry + (g / rowlen) * rowstride + g % rowlen.  The
// public layout [P][n^2][G] is {G, G, G}; the batched form's materialized
// chunks pad each row of the first variable to 128 bytes.
struct EvLayout {
  int64_t rowlen, rowstride, entry;
};
// ctas_per_sm > 0 caps the condensation kernel's residency at that many CTAs
// per SM (reserved shared memory), leaving registers to kernels beside it.
int pd_launch_condense(const polydet_plan_s *pl, const uint32_t *evals, EvLayout lay, int prime_lo,
                       int nprimes, uint32_t *detvals, cudaStream_t st, int ctas_per_sm = 0);
// The same over G nodes per prime (a slab of the grid), determinants of prime
// slot q at detvals + q * det_stride.
int pd_launch_condense_nodes(const polydet_plan_s *pl, const uint32_t *evals, EvLayout lay, int64_t G,
                             int64_t det_stride, int prime_lo, int nprimes, uint32_t *detvals,
                             cudaStream_t st, int ctas_per_sm = 0);

// Evaluation of every variable but the last (x_k), for the fused kernels:
// out[q][row][entry][Lp] with row over prod_{v<k} M_v (lex) holding the
// coefficients of x_k^l, l < L = d_k + 1 (Lp >= L, padding unwritten).
// Needs pd_partial_ws_words(pl) * (hi - lo) words of scratch.
int pd_eval_partial(const polydet_plan_s *pl, const int32_t *coeffs, int lo, int hi,
                    uint32_t *out, int Lp, uint32_t *ws, cudaStream_t st);
uint64_t pd_partial_ws_words(const polydet_plan_s *pl);

// Evaluation in two parts, for the batched form's materialized classes and
// the streamed single-plan form.
// Head: passes of x_k, ..., x_2 for primes [lo, hi) into
// head[q - lo][item][S1] with S1 = pd_head_words(pl) (x_1 still in
// coefficients: (d_1 + 1) rows of prod_{v>1} M_v nodes); needs
// pd_head_ws_words(pl) words of scratch per prime.  One variable: the
// coefficients reduced mod p_q.  Items are the plan's evaluated entries
// (n^2, or the distinct ones of an entry map).
// Tail: the x_1 pass of primes [lo, hi) from the head (whose slot 0 is prime
// head_q0) into evals[q - lo][entry][rows][B'] for the x_1 nodes
// [row_lo, row_hi), the layout the condensation kernel reads.
uint64_t pd_head_words(const polydet_plan_s *pl);
uint64_t pd_head_ws_words(const polydet_plan_s *pl);
int pd_eval_head(const polydet_plan_s *pl, const int32_t *coeffs, int lo, int hi, uint32_t *head,
                 uint32_t *ws, cudaStream_t st);
int pd_eval_tail(const polydet_plan_s *pl, const uint32_t *head, int head_q0, int lo, int hi,
                 int row_lo, int row_hi, uint32_t *evals, EvLayout lay, cudaStream_t st);
// The tail's layout for `rows` nodes of x_1 (0: all M_1): rows of the other
// variables' B nodes, padded to 32 words when a row holds at least 1024 nodes
// (aligned rows store at full bandwidth; on shorter rows the padding would
// cost more read traffic than it saves).
EvLayout pd_tail_layout(const polydet_plan_s *pl, int rows = 0);

// One (job, prime) pair of a fused launch: the nodes [0, G) of that job and
// prime, cut into items of S consecutive nodes (S = threads / lanes per det).
struct FusedSeg {
  int64_t item0;       // index of the segment's first item
  int64_t G;           // grid nodes
  int64_t q_off;       // words into the partial tensor (or the int32 coefficients)
  int64_t det_off;     // words into the determinant values
  const uint32_t *tw;  // w_k^j * R for j < N_k (last variable, this prime)
  ModP md;
  uint32_t rn;         // R^n mod p
  int32_t logNk;       // log2 N_k (twiddle table of the last variable)
  int32_t Mk;          // nodes of the last variable (M_k): node g = row * Mk + i
  int32_t L, Lp;       // coefficients of x_k per entry, stride of the partial tensor
  int32_t LPk;         // node order radix of the last variable (node_exp)
  uint32_t *status;    // the job plan's device status word
  int32_t drop_copies; // test hook: issue no bulk copy for this segment's items
};

int pd_fused_launch(int n, const FusedSeg *segs, int nsegs, int64_t nitems, const uint32_t *partial,
                    uint32_t *detvals, unsigned long long *counter, int threads, int blocks,
                    size_t qwords, int nbuf, cudaStream_t st);
// qwords: words of partial-tensor rows one item can span (rows per item x n^2 x
// Lp, rounded up to a multiple of 4); a CTA holds nbuf (2, or 1 where two do
// not fit) such buffers
int pd_fused_occupancy(int n, int threads, size_t qwords, int nbuf, int *blocks_per_sm);
int pd_fused_team(int n);

// Node exponent of node k of a variable with N points and order radix L
// (L = 1: natural order): cosets of the L-th roots, one after another.
PD_HD int node_exp(int k, int N, int L) { return k / L + (N / L) * (k % L); }
// Order radix of a variable of entry degree d on the node grid.
PD_HD int node_radix(int d) {
  const int lin = d + 1 < 8 ? d + 1 : 8;
  return lin <= 1 ? 1 : lin <= 2 ? 2 : lin <= 4 ? 4 : 8;
}


