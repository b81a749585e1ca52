/*
 * polydet.h - C ABI of libpolydet: exact determinants of n x n matrices over
 * Z[x1..xk] by the modular method of arXiv 2010.12117 (Wei & Chen,
 * "Optimized Multivariate Polynomial Determinant on GPU"), on one GB300.
 *
 * Algorithm 1 of the paper runs, for every prime p_i, an evaluation on a grid
 * of roots of unity (Sec. 3.1, Algorithm 2), a determinant of every evaluated
 * matrix mod p_i (Sec. 3.2, Algorithm 3) and an interpolation (Sec. 3.3), then
 * reconstructs the integer coefficients by mixed-radix CRT (Sec. 3.4,
 * Algorithm 4).  Each stage is one call below; each call only enqueues work.
 *
 * Conventions for every call:
 *  - Pointers marked "device" are CUDA device pointers owned by the caller
 *    (the plan never frees them); pointers marked "host" are host memory.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Calls return after enqueueing kernels on it.
 *  - Residues are plain (not Montgomery) integers in [0, p).
 *  - Multi-index arrays are row-major with the last index fastest.
 *  - Per-prime arrays passed with a range [prime_lo, prime_hi) start at prime
 *    prime_lo: slot 0 of the array belongs to prime prime_lo.
 *  - A negative return value is an error code; nothing was enqueued.  Device
 *    side failures (a degree bound that did not hold, a bounded wait that ran
 *    out) are recorded in the plan's status word, read by polydet_sync_status.
 *
 * Grid and coefficient layouts (Sec. 2, dense encoding, x1 slowest):
 *  - entry coefficients: int32 [n][n][E], E = prod_v (d_v + 1), exponent
 *    vectors (e1..ek) with 0 <= e_v <= d_v in lex order;
 *  - evaluation nodes: G = prod_v M_v nodes, node (k1..kk) with
 *    0 <= k_v < M_v is x_v = w_v^(s_v(k_v)), with w_v = g^((p-1)/N_v) for
 *    the least generator g of (Z/pZ)^*, N_v = nextpow2(D_v + 1),
 *    D_v = n * d_v, M_v = D_v + 1 (node grid, default) or N_v
 *    (POLYDET_FLAG_FULL_GRID); flat index lex (k1 slowest).  Full grid:
 *    s_v(k) = k.  Node grid: coset order s_v(k) = k / L + (N_v / L) (k mod L)
 *    with L = the smallest power of two >= min(d_v + 1, 8), so that the
 *    first M_v nodes are whole cosets of the subgroup of L-th roots (one
 *    register DFT of size L evaluates a coset; at most L - 1 nodes are
 *    computed beyond M_v).  polydet_plan_nodes returns s_v;
 *  - determinant coefficients: C = prod_v (D_v + 1), lex over e_v <= D_v.
 */
#ifndef POLYDET_H
#define POLYDET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define POLYDET_OK 0
#define POLYDET_EINVAL (-1)   /* bad argument (null, size, range, layout)   */
#define POLYDET_EDEGREE (-2)  /* some N_v above POLYDET_MAX_GRID_DIM         */
#define POLYDET_EPRIMES (-3)  /* more primes than the table holds            */
#define POLYDET_ENOMEM (-4)   /* device allocation failed (plan only)        */
#define POLYDET_ECUDA (-5)    /* a CUDA runtime call failed                  */
#define POLYDET_ETIMEOUT (-6) /* a bounded device wait gave up               */
#define POLYDET_EBOUND (-7)   /* interpolation found a coefficient beyond D_v */

/* Bits of the device status word (polydet_sync_status). */
#define POLYDET_STATUS_BOUND 0x1u   /* interpolation tail was nonzero */
#define POLYDET_STATUS_TIMEOUT 0x2u /* a bounded wait gave up         */
/* A bulk copy was still outstanding after a timed-out CTA's last bounded
 * wait: it may yet land in shared memory another CTA owns, so the CUDA
 * context is no longer trustworthy and should be torn down. */
#define POLYDET_STATUS_INFLIGHT 0x4u

/* Limits. */
#define POLYDET_MAX_N 32          /* matrix order                          */
#define POLYDET_MAX_VARS 6        /* number of variables k                 */
#define POLYDET_MAX_GRID_DIM 8192 /* N_v cap (the paper's MAX_FFT_DIM, Sec. 3.1:
                                     one column's transform runs in one CTA's
                                     shared memory)                         */
#define POLYDET_MAX_PRIMES 91     /* primes c*2^20+1 in (2^30, 2^31)       */

typedef struct polydet_plan_s *polydet_plan_t;

typedef struct polydet_plan_info {
  int32_t n;                       /* matrix order                         */
  int32_t nvars;                   /* k                                    */
  int32_t P;                       /* primes in the plan                   */
  int32_t W;                       /* 32-bit words per output coefficient  */
  int64_t E;                       /* coefficients per entry               */
  int64_t G;                       /* grid nodes per prime                 */
  int64_t C;                       /* determinant coefficients             */
  int32_t d[POLYDET_MAX_VARS];     /* entry degree bound per variable      */
  int32_t D[POLYDET_MAX_VARS];     /* determinant degree bound, n * d_v    */
  int32_t N[POLYDET_MAX_VARS];     /* grid size per variable               */
  uint64_t eval_ws_words;          /* polydet_eval scratch per prime       */
  uint64_t interp_ws_words;        /* polydet_interp scratch per prime     */
  int32_t M[POLYDET_MAX_VARS];     /* evaluation nodes per variable        */
  uint32_t flags;                  /* the plan's flags                     */
  int32_t entries;                 /* entries per prime of the evals tensor
                                      (n^2, or U + 1 with an entry map)    */
  int32_t unique;                  /* U with an entry map, else -1         */
} polydet_plan_info;

/* Plan flag: evaluate on the full power-of-two grid (N_v nodes per variable)
 * and interpolate by inverse NTT, as the paper does (Sec. 3.1, 3.3).  Without
 * it the plan evaluates on the node grid: D_v + 1 distinct powers of w_v
 * (the first D_v + 1 in coset order), i.e. exactly as many nodes as the
 * degree bound needs (Sec. 2), and interpolates through them exactly (the
 * unique polynomial of degree <= D_v, see polydet_interp).  Both give the
 * same determinant; the node grid condenses prod (D_v+1) / prod N_v as many
 * matrices. */
#define POLYDET_FLAG_FULL_GRID 0x1u

/* Primes of Eq. 1 with q = 20: every p = c * 2^20 + 1 in (2^30, 2^31); the 67
 * up to 1865126253 first, then the 24 above it, each group largest first
 * (plans take the first P: condensation runs its two-step elimination on
 * primes up to that value, and the pivoting single-step one above it).
 * Returns the table size (91) when `out` is NULL, else writes that many
 * values to host `out`. */
int polydet_prime_table(uint32_t *out);

/* Coefficient bound and prime count (Sec. 2: the product of the primes must
 * exceed the bound; signed output needs more than twice the bound).
 * bound = min over rows / columns of prod_i (sum_j l1[i][j]^2)^(1/2), where
 * host `entry_l1` [n][n] holds the l1 norm of each entry's coefficients.
 * Writes the smallest P >= 2 (Sec. 4.1 uses at least two primes) with
 * sum_i log2 p_i > 1 + log2(bound) + 1e-6, and log2(bound).  Returns
 * POLYDET_EPRIMES when the table is too short. */
int polydet_hadamard_primes(int n, const int64_t *entry_l1, int *nprimes_out,
                            double *log2_bound_out);

/* Build a plan for n x n matrices in `nvars` variables whose entries have
 * degree <= entry_deg[v] (host array) in x_v, using the first `nprimes`
 * primes of the table (must be >= 1).  The plan's small device tables
 * (Montgomery constants, twiddles, Garner and interpolation tables) are
 * shared by every plan of the same shape (n, degrees, prime count, grid, on
 * one device): the first plan of a shape allocates and uploads them as one
 * block, later plans of that shape copy nothing and allocate only their
 * status word, and the block is kept after the last such plan is destroyed
 * (up to 256 unused shapes, least recently used dropped first;
 * polydet_plan_cache_clear frees them).  Blocks and status words come from
 * the library's own stream-ordered memory pool on its own non-blocking
 * stream: planning and destroying never synchronise the device.  No later
 * call allocates device memory: scratch is passed in by the caller.  `flags`
 * is 0 or
 * POLYDET_FLAG_FULL_GRID.  The plan must be destroyed with
 * polydet_plan_destroy, after the work enqueued with it has completed. */
int polydet_plan(polydet_plan_t *out, int n, int nvars, const int32_t *entry_deg,
                 int nprimes, uint32_t flags);

/* Degree bound of det(A) per variable from the degrees of the entries
 * (Sec. 2 needs D_v + 1 interpolation nodes in x_v).  Host `entry_degs`
 * [n][n][nvars] holds deg_{x_v} a_ij, or -1 in every variable for an
 * identically zero entry.  Writes D_out[v] = the largest
 * sum_i deg_v a_{i s(i)} over the permutations s that avoid zero entries
 * (every term of the Leibniz expansion is such a product; 0 when no
 * permutation avoids them, i.e. det = 0): never above the row-sum and
 * column-sum bounds, nor above n * d_v, and exact for the resultant degree
 * of a Sylvester matrix (Sec. 6).  Maximum-weight perfect matching by the
 * Hungarian method, O(n^3) per variable; host only. */
int polydet_det_degree_bound(int n, int nvars, const int32_t *entry_degs, int32_t *D_out);

/* polydet_plan with explicit determinant degree bounds: host det_deg[nvars]
 * with 0 <= det_deg[v] <= n * entry_deg[v] (e.g. from
 * polydet_det_degree_bound) replaces n * entry_deg[v].  The grid then has
 * D_v + 1 nodes per variable on the node grid, and N_v = the power of two
 * >= max(D_v, d_v) + 1; the output has C = prod (D_v + 1) coefficients.  A
 * bound below the true degree is an error the interpolation cannot always
 * see: the caller must pass a valid bound. */
int polydet_plan_degrees(polydet_plan_t *out, int n, int nvars, const int32_t *entry_deg,
                         const int32_t *det_deg, int nprimes, uint32_t flags);

/* Repeated entries (the factor mu of Sec. 5's prediction, and the reuse of
 * a Sylvester matrix's repeated coefficients in Sec. 6).  Host `coeffs`
 * [n*n][E]: writes map_out[n*n] (the index of entry (i, j) among the
 * distinct nonzero entries in order of first occurrence, -1 for a zero
 * entry), *U_out = their number, and, if `unique_out` is not NULL, their
 * coefficients to host unique_out[U][E].  Host only. */
int polydet_unique_entries(int n, int64_t E, const int32_t *coeffs, int32_t *map_out,
                           int32_t *U_out, int32_t *unique_out);

/* Attach an entry map to a plan (host map[n*n] as written by
 * polydet_unique_entries; every index in [0, U) must occur).  From then on
 * polydet_eval takes the U distinct entries, coeffs [U][E], evaluates only
 * those, and writes evals [prime][U + 1][G] with slot U all zero;
 * polydet_condense_batch and polydet_eval_condense read entry (i, j) of a
 * node from slot map[i n + j] (slot U for -1).  Evaluation work and the
 * evals tensor shrink by n^2 / (U + 1). */
int polydet_plan_set_entry_map(polydet_plan_t plan, const int32_t *map, int U);
int polydet_plan_destroy(polydet_plan_t plan);
/* Free the shared tables of every shape that no live plan uses. */
int polydet_plan_cache_clear(void);
int polydet_plan_query(polydet_plan_t plan, polydet_plan_info *info);
/* Host copies: primes [P]; roots w_{q,v} as [P][nvars]. */
int polydet_plan_primes(polydet_plan_t plan, uint32_t *primes_out);
int polydet_plan_roots(polydet_plan_t plan, uint32_t *roots_out);
/* Host copy of the node exponents of variable v: exps_out[k] = s_v(k) for
 * k < M_v (node k of x_v is w_v^(s_v(k))). */
int polydet_plan_nodes(polydet_plan_t plan, int var, int32_t *exps_out);

/* Stage 1, evaluation (Sec. 3.1, Algorithm 2): for every prime q in
 * [prime_lo, prime_hi) and entry e, the multivariate NTT of the zero-padded
 * coefficients, i.e. the entry at every grid node mod p_q.
 * coeffs_dev: device int32 [n*n][E] (|c| < 2^31; [U][E] with an entry map).
 * evals_dev: device uint32 [prime_hi - prime_lo][info.entries][G].  ws_dev: device scratch of
 * (prime_hi - prime_lo) * info.eval_ws_words words (NULL allowed when that
 * is 0, e.g. for one variable). */
int polydet_eval(polydet_plan_t plan, const int32_t *coeffs_dev, int prime_lo,
                 int prime_hi, uint32_t *evals_dev, uint32_t *ws_dev, void *stream);

/* Stage 2, condensation (Sec. 3.2, Algorithm 3): det of the n x n matrix at
 * every grid node mod p_q, by fraction-free elimination with a search for the
 * first nonzero pivot.  evals_dev as written by polydet_eval; detvals_dev:
 * device uint32 [prime_hi - prime_lo][G]. */
int polydet_condense_batch(polydet_plan_t plan, const uint32_t *evals_dev,
                           int prime_lo, int prime_hi, uint32_t *detvals_dev,
                           void *stream);

/* Stages 1 and 2 streamed through a fixed workspace (Sec. 3.1's multi-round
 * evaluation when the evaluated tensor does not fit: one prime's
 * [entries][G] never has to be resident).  For every prime q in
 * [prime_lo, prime_hi): the passes of x_k, ..., x_2 into a head tensor
 * [items][(d_1 + 1)][B] (B = prod_{v>1} M_v), then slab by slab - R
 * consecutive nodes of x_1 at a time, R as large as `ws_words` allows - the
 * x_1 pass of the slab's rows into [entries][R][B] and the condensation of
 * those R * B nodes into detvals_dev[q - prime_lo][r0 B .. (r0 + R) B).
 * coeffs_dev as for polydet_eval; detvals_dev: device uint32
 * [prime_hi - prime_lo][G]; ws_dev: device scratch of ws_words words, at
 * least polydet_stream_ws_words(plan, 1) (POLYDET_EINVAL otherwise).  On
 * the node grid R is a multiple of the coset size of x_1 (up to 8).
 * Everything is enqueued on `stream`; nothing is allocated. */
uint64_t polydet_stream_ws_words(polydet_plan_t plan, int rows);
int polydet_eval_condense(polydet_plan_t plan, const int32_t *coeffs_dev, int prime_lo,
                          int prime_hi, uint32_t *detvals_dev, uint32_t *ws_dev, uint64_t ws_words,
                          void *stream);

/* Stage 3, interpolation (Sec. 3.3): on the full grid the inverse NTT with the
 * 1/N factor, keeping the C coefficients with e_v <= D_v (any nonzero
 * coefficient with e_v > D_v sets POLYDET_STATUS_BOUND); on the node grid the
 * unique interpolant through the nodes, one variable at a time, solved coset
 * by coset (an inverse DFT of size L per whole coset, then L inverse
 * Vandermonde solves of size M_v / L and a correction from the last partial
 * coset).  detvals_dev: device uint32
 * [prime_hi - prime_lo][G] (read only); residues_dev: device uint32
 * [prime_hi - prime_lo][C]; ws_dev: device scratch of
 * (prime_hi - prime_lo) * info.interp_ws_words words (NULL allowed when 0).
 * These per-prime residues are the restart point of a run (Sec. 4.3): a
 * resumed run recomputes only the missing primes. */
int polydet_interp(polydet_plan_t plan, const uint32_t *detvals_dev, int prime_lo,
                   int prime_hi, uint32_t *residues_dev, uint32_t *ws_dev, void *stream);

/* Interpolation without any device allocation (the paper has no counterpart;
 * this exists for callers of the library).
 * Some callers cannot call cudaMalloc when they need the result: code that
 * runs while a stream is being captured into a CUDA graph in the global
 * capture mode (where cudaMalloc is not permitted), processes whose device
 * memory is reserved up front by another allocator or memory pool, and
 * latency-bound loops that must not stall on cudaMalloc/cudaFree (both
 * synchronise the device).  polydet_interp_static does exactly what
 * polydet_interp does, with its scratch taken from a file-scope device array
 * of POLYDET_STATIC_SCRATCH_WORDS words (16 MiB) instead of a caller
 * workspace.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *  - Every GPU that loads the library holds that array until the process
 *    exits.
 *  - The first call on a device (with that device current) looks up the
 *    array's device address once; make that first call before any stream
 *    capture.
 *  - Requests needing more than the array, i.e. (prime_hi - prime_lo) *
 *    info.interp_ws_words > POLYDET_STATIC_SCRATCH_WORDS, return
 *    POLYDET_ETOOBIG and enqueue nothing: split the prime range.
 *  - All calls share the one array and it keeps the last call's contents
 *    (nothing in it needs clearing: each pass overwrites what the next reads).
 *    Calls that overlap on the GPU - on different streams, or from different
 *    threads - race on it: issue them on one stream, or use polydet_interp
 *    with separate workspaces.
 * Arguments, layouts and the status word are as for polydet_interp. */
#define POLYDET_ETOOBIG (-8) /* request larger than a fixed internal buffer */
#define POLYDET_STATIC_SCRATCH_WORDS (4u * 1024u * 1024u)
int polydet_interp_static(polydet_plan_t plan, const uint32_t *detvals_dev, int prime_lo,
                          int prime_hi, uint32_t *residues_dev, void *stream);

/* Stage 4, CRT (Sec. 3.4, Algorithm 4): mixed-radix (Garner) digits of each
 * coefficient over all P primes, converted to the signed integer in
 * (-M/2, M/2), M = prod p.  residues_dev: device uint32 [P][C]; limbs_dev:
 * device uint32 [C][W], little-endian two's complement. */
int polydet_crt(polydet_plan_t plan, const uint32_t *residues_dev, uint32_t *limbs_dev,
                void *stream);

/* Early termination (no counterpart in the paper: it stops adding primes
 * once the reconstruction stops changing, instead of always using the prime
 * count of the coefficient bound).  After primes 0 .. i of a plan (i >= 1,
 * i < P) have their residues, computes the mixed-radix (Garner) digit i of
 * every coefficient and ORs 1 into device word *unstable_dev if for some
 * coefficient the symmetric lift of its residues over the first i primes
 * differs from the lift over the first i + 1 (i.e. digit i is not 0 for a
 * value in the lower half of [0, M_i), nor p_i - 1 for one in the upper
 * half).  residues_dev: device uint32 [P][C] (primes 0 .. i valid);
 * digits_dev: device uint32 [P][C], digits 0 .. i - 1 as left by the calls
 * for 1 .. i - 1 (the call for i = 1 also writes digit 0); the caller clears
 * *unstable_dev.  When a call leaves it 0, every coefficient is already
 * determined by i primes unless, for each coefficient still wrong, p_i
 * divides (true value - lift) / M_i: with the check prime regarded as
 * random among the table primes not yet used, a chance of at most
 * log2(2 B / M_i) / 30 over their number for a bound B on the coefficients.
 * The caller then takes the CRT over the first i + 1 primes. */
int polydet_crt_check(polydet_plan_t plan, const uint32_t *residues_dev, uint32_t *digits_dev,
                      int i, uint32_t *unstable_dev, void *stream);

/* Synchronise `stream`, return the plan's status word in *status_out and clear
 * it.  Returns POLYDET_EBOUND / POLYDET_ETIMEOUT if the matching bit was set. */
int polydet_sync_status(polydet_plan_t plan, void *stream, uint32_t *status_out);

/* ------------------------------------------------------------------------
 * Batches: many jobs of uneven order, variable count, degree and prime
 * count in one run (the data-parallel loop of Algorithm 1 over matrices,
 * primes and nodes at once).  Each matrix order runs in one of two modes:
 *   POLYDET_BATCH_FUSED: evaluation of the last variable is fused into the
 *     determinant kernel, so evaluated matrices never reach memory: one
 *     persistent kernel per order takes (job, prime, node-block) items from
 *     a counter kept in the caller's workspace, and the bulk-copy engine
 *     (cp.async.bulk on an mbarrier) stages the next item's rows of the
 *     partial tensor in shared memory while the current item is computed;
 *   POLYDET_BATCH_MATERIALIZED: the first variable's NTT pass writes the
 *     evaluated matrices of a chunk of primes into one of two workspace
 *     buffers and the condensation kernel of polydet_condense_batch reads
 *     them back (cheaper per node than fused evaluation when n^2 entries
 *     dominate); the passes run on a stream of the batch's own, joined to the
 *     caller's stream by events, so a pass overlaps the previous chunk's
 *     condensation and the whole run still captures into one CUDA graph.
 * The default is fused for n < POLYDET_BATCH_MATERIALIZE_N, materialized
 * from there on; polydet_batch_set_mode changes it per order (the
 * autotuner's second knob).
 *
 * Buffers are caller-owned device arrays laid out by the batch; job j
 * occupies words [off[j], off[j+1]) of each (polydet_batch_offsets):
 *   coeffs   int32  : job j's [n][n][E] coefficients, as for polydet_eval
 *   partial  uint32 : eval -> condense: every variable but the last evaluated
 *                      (fused), or every variable but the first (materialized)
 *   detvals  uint32 : [P][G] determinants at the nodes (as condense_batch)
 *   residues uint32 : [P][C] determinant residues (as polydet_interp)
 *   limbs    uint32 : [C][W] signed coefficients (as polydet_crt)
 *   workspace uint32: info.workspace_words words (counters + scratch).
 * Constraint: the last variable's entry degree d_k is at most 7.
 * A run is eval, condense, interp, crt on one stream; no call in a run
 * allocates or synchronises, so a run can be captured in a CUDA graph.
 * ------------------------------------------------------------------------ */
typedef struct polydet_job {
  int32_t n;                   /* matrix order, 1..32                     */
  int32_t nvars;               /* variables, 1..POLYDET_MAX_VARS          */
  int32_t nprimes;             /* primes (polydet_hadamard_primes)        */
  int32_t d[POLYDET_MAX_VARS]; /* entry degree bound per variable         */
  uint32_t flags;              /* 0 or POLYDET_FLAG_FULL_GRID             */
} polydet_job;

typedef struct polydet_batch_s *polydet_batch_t;

typedef struct polydet_batch_info {
  int32_t njobs;
  int64_t coeff_words, partial_words, detval_words, residue_words, limb_words;
  uint64_t workspace_words;           /* for the current modes              */
  int64_t items[POLYDET_MAX_N + 1];   /* fused work items per matrix order  */
  int32_t threads[POLYDET_MAX_N + 1]; /* CTA size per matrix order          */
  int32_t blocks[POLYDET_MAX_N + 1];  /* persistent CTAs per matrix order   */
  int32_t mode[POLYDET_MAX_N + 1];    /* POLYDET_BATCH_* per matrix order   */
  uint64_t chunk_words;               /* materialized chunk budget          */
} polydet_batch_info;

#define POLYDET_BATCH_FUSED 0
#define POLYDET_BATCH_MATERIALIZED 1
#define POLYDET_BATCH_MATERIALIZE_N 14
/* Materialized mode: default words of evaluated matrices one chunk may
 * hold; a chunk is as many primes of one job as fit, and never less than
 * one (polydet_batch_set_chunk_words changes the budget). */
#define POLYDET_BATCH_CHUNK_WORDS (512ull * 1024ull * 1024ull)

#define POLYDET_OFF_COEFFS 0
#define POLYDET_OFF_PARTIAL 1
#define POLYDET_OFF_DETVALS 2
#define POLYDET_OFF_RESIDUES 3
#define POLYDET_OFF_LIMBS 4

/* Plan a batch from host `jobs[njobs]` (one polydet_plan per job, with the
 * shared tables of polydet_plan).  The batch's streams, events, status word
 * and segment tables come from a per-process pool and return to it when the
 * batch is destroyed, so planning batch after batch creates no stream and
 * allocates nothing once the pool and the shape cache are warm.  Destroy a
 * batch only after the work enqueued with it has completed.  flags must be
 * 0. */
int polydet_batch_plan(polydet_batch_t *out, const polydet_job *jobs, int njobs, uint32_t flags);
int polydet_batch_destroy(polydet_batch_t batch);
int polydet_batch_query(polydet_batch_t batch, polydet_batch_info *info);
/* Host `out[njobs + 1]` word offsets of buffer `which` (POLYDET_OFF_*). */
int polydet_batch_offsets(polydet_batch_t batch, int which, int64_t *out);
/* The plan of job `job` (owned by the batch; do not destroy).  Every job plan
 * of a batch reports into one status word, the batch's: polydet_sync_status
 * on a job plan reads and clears the whole batch's status. */
int polydet_batch_job_plan(polydet_batch_t batch, int job, polydet_plan_t *plan_out);
/* CTA size (multiple of 32 and of the lanes per determinant, <= 128) of the
 * fused kernel for matrix order n; the autotuner's knob.  Not during a
 * graph capture (uploads the segment table). */
int polydet_batch_set_launch(polydet_batch_t batch, int n, int threads);

/* Mode (POLYDET_BATCH_*) of matrix order n.  Changes the partial tensor's
 * content and the workspace size (query again); rerun polydet_batch_eval
 * before the next condense.  Not during a graph capture. */
int polydet_batch_set_mode(polydet_batch_t batch, int n, int mode);
/* Materialized mode: at most `ctas_per_sm` CTAs of the condensation kernel
 * per SM (0, the default: as many as its registers allow; 1..16 reserve
 * shared memory the kernel does not use so that no more fit), which leaves
 * registers for the first-variable passes to run beside the condensation
 * instead of waiting for it. */
int polydet_batch_set_condense_ctas(polydet_batch_t batch, int ctas_per_sm);
/* Chunk budget of the materialized mode in words (>= 1; the workspace size
 * changes: query again).  Not during a graph capture. */
int polydet_batch_set_chunk_words(polydet_batch_t batch, uint64_t words);
/* Test hook for failure detection (no counterpart in the paper), off by
 * default.  With on = 1 the fused kernels withhold the bulk copies of their
 * staged rows (those that would be issued), so each CTA's bounded wait for
 * them runs out after about one second; the CTA then sets
 * POLYDET_STATUS_TIMEOUT in its job plan's status word
 * (polydet_batch_sync_status returns POLYDET_ETIMEOUT) and ends, and the
 * determinant values of those items are not written.  on = 0 restores normal
 * operation.  Not during a graph capture (uploads the segment tables). */
int polydet_batch_test_drop_copies(polydet_batch_t batch, int on);
/* Lanes that share one determinant in the condensation kernels of order n
 * (a CTA size must be a multiple of it); POLYDET_EINVAL outside 1..32.  Host
 * only: no device call. */
int polydet_team_size(int n);
/* Elimination steps the condensation kernels of order n take per pass (2 or
 * 3; the instruction mix, and so the integer-pipe ceiling, depends on it);
 * POLYDET_EINVAL outside 1..32.  Host only. */
int polydet_condense_steps(int n);

/* Stage 1 of a batch (Sec. 3.1): every variable but the last (fused orders)
 * or but the first (materialized orders); all orders (n = 0 in
 * polydet_batch_eval_n) or only the jobs of order n. */
int polydet_batch_eval(polydet_batch_t batch, const int32_t *coeffs_dev, uint32_t *partial_dev,
                       uint32_t *ws_dev, void *stream);
int polydet_batch_eval_n(polydet_batch_t batch, int n, const int32_t *coeffs_dev,
                         uint32_t *partial_dev, uint32_t *ws_dev, void *stream);
/* Stage 2 (Sec. 3.1-3.2): the remaining variable's evaluation and the
 * condensation, all orders (n = 0 in polydet_batch_condense_n) or only
 * order n. */
int polydet_batch_condense(polydet_batch_t batch, const uint32_t *partial_dev,
                           uint32_t *detvals_dev, uint32_t *ws_dev, void *stream);
int polydet_batch_condense_n(polydet_batch_t batch, int n, const uint32_t *partial_dev,
                             uint32_t *detvals_dev, uint32_t *ws_dev, void *stream);
/* Stage 3: interpolation per job (Sec. 3.3). */
int polydet_batch_interp(polydet_batch_t batch, const uint32_t *detvals_dev,
                         uint32_t *residues_dev, uint32_t *ws_dev, void *stream);
/* Stage 4: Garner CRT per job (Sec. 3.4). */
int polydet_batch_crt(polydet_batch_t batch, const uint32_t *residues_dev, uint32_t *limbs_dev,
                      void *stream);
/* The batch's status word, the OR of what any job reported (synchronises
 * `stream` and clears it). */
int polydet_batch_sync_status(polydet_batch_t batch, void *stream, uint32_t *status_out);

/* ------------------------------------------------------------------------
 * Run-time / memory predictor for scheduling (generalises the prediction of
 * Sec. 5, T = C_p r^2 Round(mean T_e, 2) mu): an fp32 MLP 8 -> 64 -> 64 -> 2
 * with ReLU.  Parameters are one device float array of POLYDET_MLP_PARAMS:
 * W1[64][8] b1[64] W2[64][64] b2[64] W3[2][64] b3[2] (row = output unit).
 * Loss: L = 1/(2B) sum_b sum_o (y_bo - t_bo)^2.  All pointers are device
 * memory owned by the caller; nothing is allocated.
 * ------------------------------------------------------------------------ */
#define POLYDET_MLP_IN 8
#define POLYDET_MLP_HIDDEN 64
#define POLYDET_MLP_OUT 2
#define POLYDET_MLP_PARAMS 4866
/* y[B][2] = MLP(x[B][8]).  act_ws: [B][128] floats receiving the hidden
 * activations (needed by polydet_mlp_backward), or NULL for inference. */
int polydet_mlp_forward(const float *params, const float *x, int batch, float *y, float *act_ws,
                        void *stream);
/* Gradient of L at (x, target) after polydet_mlp_forward wrote y and act_ws:
 * grads[POLYDET_MLP_PARAMS] (overwritten), *loss (device float, may be
 * NULL); delta_ws: [B][130] floats of scratch.  Deterministic: every sum runs
 * over the batch in sample order. */
int polydet_mlp_backward(const float *params, const float *x, const float *target, int batch,
                         const float *y, const float *act_ws, float *delta_ws, float *grads,
                         float *loss, void *stream);
/* One Adam step (bias-corrected, step >= 1) with decoupled weight decay:
 * p -= lr * (m_hat / (sqrt(v_hat) + eps) + weight_decay * p). */
int polydet_mlp_adam(float *params, const float *grads, float *m, float *v, int step, float lr,
                     float beta1, float beta2, float eps, float weight_decay, void *stream);

/* Measurement utility (not a stage of the method): runs four in-register
 * integer streams on every SM and reports their rates, the ceilings of the
 * condensation kernels - plain 32-bit multiply-adds per second, single-step
 * modular updates (a*b - c*d)/2^32 mod p per second, two-step element
 * updates (a*b + c*d + e*f)/2^32 mod p per second (each stands for two
 * single-step updates) and three-step element updates
 * (a*b + c*d + e*f + g*h)/2^32 mod p per second (each stands for three).
 * Every product takes an operand computed in the previous iteration, so none is
 * loop-invariant.  Allocates and frees a small buffer; synchronises
 * `stream`. */
int polydet_probe_int_peaks(void *stream, double *imad_per_s, double *update_per_s,
                            double *pair_update_per_s, double *triple_update_per_s);

/* Last CUDA error string seen by the library (host, static storage). */
const char *polydet_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* POLYDET_H */
