// Batches of determinant jobs of uneven shape (order, variables, degrees,
// prime count): one plan per job, a shared layout of every buffer, and the
// per-order segment tables of the fused kernels.
//
// A run is four calls on one stream (the whole run can be captured in a CUDA
// graph; nothing in it allocates or synchronises):
//   polydet_batch_eval      per job, NTT passes of every variable but the last
//                           (fused orders) or but the first (materialized)
//   polydet_batch_condense  fused orders: one persistent fused kernel each;
//                           materialized orders: per job and chunk of primes,
//                           the first variable's pass into the workspace and
//                           the condensation kernel over it
//   polydet_batch_interp    inverse NTT per job
//   polydet_batch_crt       Garner CRT per job
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace {
constexpr int kCounterWords = 2 * (POLYDET_MAX_N + 1);  // one 64-bit counter per order
constexpr uint64_t kWsHead = 256;                       // words reserved for the counters
constexpr int kFan = 4;                                 // streams for the per-job stages

int pow2_at_least(int x) {
  int v = 1;
  while (v < x) v <<= 1;
  return v;
}
}  // namespace

// The streams, events, status word and segment-table buffer a batch needs,
// recycled through a per-process pool: a batch takes a set when it is planned
// and returns it when destroyed, so batches planned one after another (a
// server's waves) create no stream or event and allocate nothing but a
// larger segment buffer when one is needed.
struct BatchRes {
  int dev = 0;
  cudaStream_t side = nullptr;
  cudaEvent_t ev[6] = {};
  cudaStream_t fan[kFan] = {};
  cudaEvent_t fev[kFan + 1] = {};
  uint32_t *d_status = nullptr;
  FusedSeg *segs = nullptr;
  size_t segs_cap = 0;
};

static std::mutex g_res_mu;
static std::vector<BatchRes *> g_res_free;

static void free_res(BatchRes *r) {
  if (!r) return;
  for (auto e : r->ev)
    if (e) cudaEventDestroy(e);
  for (auto e : r->fev)
    if (e) cudaEventDestroy(e);
  if (r->side) cudaStreamDestroy(r->side);
  for (auto f : r->fan)
    if (f) cudaStreamDestroy(f);
  cudaFree(r->d_status);
  cudaFree(r->segs);
  delete r;
}

static int take_res(BatchRes **out) {
  int dev = 0;
  PD_CUDA(cudaGetDevice(&dev));
  BatchRes *r = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_res_mu);
    for (size_t i = 0; i < g_res_free.size(); ++i) {
      if (g_res_free[i]->dev == dev) {
        r = g_res_free[i];
        g_res_free.erase(g_res_free.begin() + i);
        break;
      }
    }
  }
  if (!r) {
    r = new BatchRes();
    r->dev = dev;
    // the materialized orders' first-variable passes run on the side stream
    // at the highest priority: their CTAs take SM slots as soon as
    // condensation CTAs retire, so the HBM-bound passes run beside the
    // integer-bound condensation instead of after it
    int least = 0, greatest = 0;
    bool ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
              cudaStreamCreateWithPriority(&r->side, cudaStreamNonBlocking, greatest) == cudaSuccess &&
              cudaMalloc((void **)&r->d_status, sizeof(uint32_t)) == cudaSuccess;
    for (auto &e : r->ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    for (auto &e : r->fev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    for (auto &f : r->fan) ok = ok && cudaStreamCreateWithFlags(&f, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
      free_res(r);
      return POLYDET_ECUDA;
    }
  }
  // a fresh status word (the set's previous batch has been destroyed)
  if (cudaMemset(r->d_status, 0, sizeof(uint32_t)) != cudaSuccess) {
    free_res(r);
    return POLYDET_ECUDA;
  }
  *out = r;
  return POLYDET_OK;
}

static void give_res(BatchRes *r) {
  if (!r) return;
  std::lock_guard<std::mutex> lock(g_res_mu);
  g_res_free.push_back(r);
}

struct polydet_batch_s {
  int njobs = 0;
  std::vector<polydet_plan_t> plans;
  std::vector<int> Lp;
  std::vector<int64_t> coeff_off, part_off, det_off, res_off, limb_off;  // [njobs + 1]
  uint64_t ws_words = 0;
  int sms = 0;
  int threads[POLYDET_MAX_N + 1] = {};
  int blocks[POLYDET_MAX_N + 1] = {};
  int64_t nitems[POLYDET_MAX_N + 1] = {};
  size_t qwords[POLYDET_MAX_N + 1] = {};
  int nbuf[POLYDET_MAX_N + 1] = {};  // buffers of staged rows per fused CTA (2, or 1 where 2 do not fit)
  std::vector<FusedSeg> segs[POLYDET_MAX_N + 1];
  FusedSeg *d_segs[POLYDET_MAX_N + 1] = {};
  int mode[POLYDET_MAX_N + 1] = {};
  std::vector<int> jobs_of[POLYDET_MAX_N + 1];
  uint64_t chunk_words = POLYDET_BATCH_CHUNK_WORDS;
  uint64_t chunk_max = 0;  // words of the largest materialized chunk (one of two buffers)
  // materialized chunks: first-variable passes on `side`, condensation on the
  // caller's stream; ev[0..1] = pass of buffer b done, ev[2..3] = condensation
  // of buffer b done, ev[4] / ev[5] = fork / join
  cudaStream_t side = nullptr;
  cudaEvent_t *ev = nullptr;
  // per-job launches of stages 1, 3, 4 fan out over kFan streams (job j on
  // fan[j % kFan], with its own scratch slice), joined back by events
  cudaStream_t *fan = nullptr;
  cudaEvent_t *fev = nullptr;
  uint64_t scratch_stride = 0;
  // one status word for every job of the batch (each job plan points at
  // it), so that reading the batch's status is one copy, not one per job
  uint32_t *d_status = nullptr;
  BatchRes *res = nullptr;  // the pooled set the pointers above come from
  // materialized orders: condensation CTAs per SM (0: as many as registers
  // allow), so that the first-variable passes find room beside them
  int condense_ctas = 0;
};

static int fan_begin(polydet_batch_s *b, cudaStream_t st) {
  PD_CUDA(cudaEventRecord(b->fev[kFan], st));
  for (int i = 0; i < kFan; ++i) PD_CUDA(cudaStreamWaitEvent(b->fan[i], b->fev[kFan], 0));
  return POLYDET_OK;
}

static int fan_end(polydet_batch_s *b, cudaStream_t st) {
  for (int i = 0; i < kFan; ++i) {
    PD_CUDA(cudaEventRecord(b->fev[i], b->fan[i]));
    PD_CUDA(cudaStreamWaitEvent(st, b->fev[i], 0));
  }
  return POLYDET_OK;
}

// Primes of job `pl` per materialized chunk: as many as fit in the chunk
// budget, at least one.
static int chunk_primes(const polydet_batch_s *b, const polydet_plan_s *pl) {
  const uint64_t per = (uint64_t)pl->n * pl->n * (uint64_t)pd_tail_layout(pl).entry;
  const uint64_t c = b->chunk_words / std::max<uint64_t>(per, 1);
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(c, (uint64_t)pl->P));
}

// Workspace words for the current modes: the counters, then the largest
// scratch any job needs in any stage (stages run one after another).
static void update_ws(polydet_batch_s *b) {
  uint64_t scratch = 0, cmax = 0;
  for (int j = 0; j < b->njobs; ++j) {
    const polydet_plan_s *pl = b->plans[j];
    uint64_t need = pl->interp_ws_words * (uint64_t)pl->P;
    if (b->mode[pl->n] == POLYDET_BATCH_FUSED) {
      if (pl->nvars > 1) need = std::max<uint64_t>(need, pd_partial_ws_words(pl) * (uint64_t)pl->P);
    } else {
      need = std::max<uint64_t>(need, pd_head_ws_words(pl) * (uint64_t)pl->P);
      cmax = std::max<uint64_t>(cmax, (uint64_t)chunk_primes(b, pl) * pl->n * pl->n *
                                          (uint64_t)pd_tail_layout(pl).entry);
    }
    scratch = std::max(scratch, need);
  }
  b->scratch_stride = (scratch + 63) / 64 * 64;
  b->chunk_max = (cmax + 63) / 64 * 64;
  // stages run one after another: the fan-out scratch slices (stages 1, 3)
  // and the two chunk buffers (stage 2) share the same words
  b->ws_words = kWsHead + std::max<uint64_t>(kFan * b->scratch_stride, 2 * b->chunk_max);
}

static void destroy_batch(polydet_batch_s *b) {
  if (!b) return;
  for (auto p : b->plans) polydet_plan_destroy(p);
  give_res(b->res);
  delete b;
}

// (Re)number the items of order n for the current CTA size and upload.
static int build_class(polydet_batch_s *b, int n) {
  auto &v = b->segs[n];
  if (v.empty()) return POLYDET_OK;
  const int S = b->threads[n] / pd_fused_team(n);
  int64_t it = 0;
  for (auto &s : v) {
    s.item0 = it;
    it += (s.G + S - 1) / S;
  }
  b->nitems[n] = it;
  // shared memory for the partial-tensor rows one item can span
  size_t qw = 0;
  for (const auto &s : v) {  // an item of S nodes spans at most ceil(S / M_k) + 1 rows
    const int64_t rows = std::min<int64_t>((S + s.Mk - 1) / s.Mk + 1, (s.G + s.Mk - 1) / s.Mk);
    qw = std::max<size_t>(qw, (size_t)rows * n * n * s.Lp);
  }
  qw = (qw + 3) / 4 * 4;  // both buffers start on 16 bytes
  b->qwords[n] = qw;
  int bps = 0, nbuf = 2;
  int rc = pd_fused_occupancy(n, b->threads[n], qw, nbuf, &bps);
  if (rc) return rc;
  if (bps < 1) {  // no room to prefetch: one buffer, the next item's copy after the current item
    nbuf = 1;
    rc = pd_fused_occupancy(n, b->threads[n], qw, nbuf, &bps);
    if (rc) return rc;
  }
  if (bps < 1) return POLYDET_EINVAL;  // the CTA's shared memory does not fit
  b->nbuf[n] = nbuf;
  b->blocks[n] = (int)std::min<int64_t>(it, (int64_t)bps * b->sms);
  PD_CUDA(cudaMemcpy(b->d_segs[n], v.data(), v.size() * sizeof(FusedSeg), cudaMemcpyHostToDevice));
  return POLYDET_OK;
}

extern "C" int polydet_batch_plan(polydet_batch_t *out, const polydet_job *jobs, int njobs,
                                  uint32_t flags) {
  if (!out || !jobs || njobs < 1 || flags != 0) return POLYDET_EINVAL;
  polydet_batch_s *b = new polydet_batch_s();
  b->njobs = njobs;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete b;
    return POLYDET_ECUDA;
  }
  {
    const int rc = take_res(&b->res);
    if (rc) {
      delete b;
      return rc;
    }
  }
  b->side = b->res->side;
  b->ev = b->res->ev;
  b->fan = b->res->fan;
  b->fev = b->res->fev;
  b->d_status = b->res->d_status;
  b->coeff_off.assign(1, 0);
  b->part_off.assign(1, 0);
  b->det_off.assign(1, 0);
  b->res_off.assign(1, 0);
  b->limb_off.assign(1, 0);
  for (int j = 0; j < njobs; ++j) {
    const polydet_job &jb = jobs[j];
    if (jb.nvars < 1 || jb.nvars > POLYDET_MAX_VARS || jb.d[jb.nvars - 1] + 1 > 8) {
      destroy_batch(b);
      return POLYDET_EINVAL;
    }
    polydet_plan_t pl = nullptr;  // reports into the batch's status word
    int rc = pd_plan_impl(&pl, jb.n, jb.nvars, jb.d, nullptr, jb.nprimes, jb.flags, b->d_status);
    if (rc) {
      destroy_batch(b);
      return rc;
    }
    b->plans.push_back(pl);
    const int k = pl->nvars;
    const int L = pl->d[k - 1] + 1;
    const int Lp = pow2_at_least(L);
    b->Lp.push_back(Lp);
    const int64_t n2 = (int64_t)pl->n * pl->n;
    const int64_t rows = pl->G / pl->M[k - 1];
    // room for either mode's partial tensor, so offsets do not move with it
    const int64_t fused_part = (int64_t)pl->P * rows * n2 * Lp;
    const int64_t mat_part = (int64_t)pl->P * n2 * (int64_t)pd_head_words(pl);
    const int64_t part = (std::max(fused_part, mat_part) + 7) / 8 * 8;
    b->coeff_off.push_back(b->coeff_off.back() + n2 * pl->E);
    b->part_off.push_back(b->part_off.back() + part);
    b->det_off.push_back(b->det_off.back() + (int64_t)pl->P * pl->G);
    b->res_off.push_back(b->res_off.back() + (int64_t)pl->P * pl->C);
    b->limb_off.push_back(b->limb_off.back() + pl->C * pl->W);
    b->jobs_of[pl->n].push_back(j);
  }
  for (int n = 1; n <= POLYDET_MAX_N; ++n)
    b->mode[n] = n >= POLYDET_BATCH_MATERIALIZE_N ? POLYDET_BATCH_MATERIALIZED : POLYDET_BATCH_FUSED;
  update_ws(b);
  for (int j = 0; j < njobs; ++j) {
    polydet_plan_s *pl = b->plans[j];
    const int k = pl->nvars;
    const int64_t n2 = (int64_t)pl->n * pl->n;
    const int64_t rows = pl->G / pl->M[k - 1];
    for (int q = 0; q < pl->P; ++q) {
      FusedSeg s = {};
      s.G = pl->G;
      s.q_off = b->part_off[j] + (int64_t)q * rows * n2 * b->Lp[j];
      s.det_off = b->det_off[j] + (int64_t)q * pl->G;
      s.tw = pl->d_tw_fwd + (size_t)q * pl->tw_len + pl->tw_off[k - 1];
      s.md = pl->mod_h[q];
      s.rn = pl->rn_h[q];
      s.logNk = pl->logN[k - 1];
      s.Mk = pl->M[k - 1];
      s.L = pl->d[k - 1] + 1;
      s.Lp = b->Lp[j];
      s.LPk = pl->LPo[k - 1];
      s.status = pl->d_status;
      b->segs[pl->n].push_back(s);
    }
  }
  // the segment tables of every order in the pooled buffer (grown if needed)
  size_t nseg = 0;
  for (int n = 1; n <= POLYDET_MAX_N; ++n) nseg += b->segs[n].size();
  if (nseg > b->res->segs_cap) {
    cudaFree(b->res->segs);
    b->res->segs = nullptr;
    b->res->segs_cap = 0;
    if (cudaMalloc((void **)&b->res->segs, nseg * sizeof(FusedSeg)) != cudaSuccess) {
      destroy_batch(b);
      return POLYDET_ENOMEM;
    }
    b->res->segs_cap = nseg;
  }
  for (int n = 1, at = 0; n <= POLYDET_MAX_N; ++n) {
    b->d_segs[n] = b->res->segs + at;
    at += (int)b->segs[n].size();
  }
  for (int n = 1; n <= POLYDET_MAX_N; ++n) {
    b->threads[n] = 128;
    int rc = build_class(b, n);
    if (rc) {
      destroy_batch(b);
      return rc;
    }
  }
  *out = b;
  return POLYDET_OK;
}

extern "C" int polydet_batch_test_drop_copies(polydet_batch_t b, int on) {
  if (!b || (on != 0 && on != 1)) return POLYDET_EINVAL;
  for (int n = 1; n <= POLYDET_MAX_N; ++n) {
    if (b->segs[n].empty()) continue;
    for (auto &s : b->segs[n]) s.drop_copies = on;
    int rc = build_class(b, n);
    if (rc) return rc;
  }
  return POLYDET_OK;
}

extern "C" int polydet_batch_destroy(polydet_batch_t b) {
  if (!b) return POLYDET_EINVAL;
  destroy_batch(b);
  return POLYDET_OK;
}

extern "C" int polydet_batch_query(polydet_batch_t b, polydet_batch_info *info) {
  if (!b || !info) return POLYDET_EINVAL;
  memset(info, 0, sizeof *info);
  info->njobs = b->njobs;
  info->coeff_words = b->coeff_off.back();
  info->partial_words = b->part_off.back();
  info->detval_words = b->det_off.back();
  info->residue_words = b->res_off.back();
  info->limb_words = b->limb_off.back();
  info->workspace_words = b->ws_words;
  for (int n = 1; n <= POLYDET_MAX_N; ++n) {
    info->items[n] = b->nitems[n];
    info->threads[n] = b->threads[n];
    info->blocks[n] = b->blocks[n];
    info->mode[n] = b->mode[n];
  }
  info->chunk_words = b->chunk_words;
  return POLYDET_OK;
}

extern "C" int polydet_batch_offsets(polydet_batch_t b, int which, int64_t *out) {
  if (!b || !out) return POLYDET_EINVAL;
  const std::vector<int64_t> *v = nullptr;
  switch (which) {
    case POLYDET_OFF_COEFFS: v = &b->coeff_off; break;
    case POLYDET_OFF_PARTIAL: v = &b->part_off; break;
    case POLYDET_OFF_DETVALS: v = &b->det_off; break;
    case POLYDET_OFF_RESIDUES: v = &b->res_off; break;
    case POLYDET_OFF_LIMBS: v = &b->limb_off; break;
    default: return POLYDET_EINVAL;
  }
  memcpy(out, v->data(), v->size() * sizeof(int64_t));
  return POLYDET_OK;
}

extern "C" int polydet_batch_job_plan(polydet_batch_t b, int job, polydet_plan_t *plan_out) {
  if (!b || !plan_out || job < 0 || job >= b->njobs) return POLYDET_EINVAL;
  *plan_out = b->plans[job];
  return POLYDET_OK;
}

extern "C" int polydet_batch_set_launch(polydet_batch_t b, int n, int threads) {
  if (!b || n < 1 || n > POLYDET_MAX_N) return POLYDET_EINVAL;
  const int T = pd_fused_team(n);
  if (threads < 32 || threads > 128 || threads % 32 || threads % T) return POLYDET_EINVAL;
  b->threads[n] = threads;
  return build_class(b, n);
}

extern "C" int polydet_batch_set_mode(polydet_batch_t b, int n, int mode) {
  if (!b || n < 1 || n > POLYDET_MAX_N ||
      (mode != POLYDET_BATCH_FUSED && mode != POLYDET_BATCH_MATERIALIZED))
    return POLYDET_EINVAL;
  b->mode[n] = mode;
  update_ws(b);
  return POLYDET_OK;
}

extern "C" int polydet_batch_set_condense_ctas(polydet_batch_t b, int ctas_per_sm) {
  if (!b || ctas_per_sm < 0 || ctas_per_sm > 16) return POLYDET_EINVAL;
  b->condense_ctas = ctas_per_sm;
  return POLYDET_OK;
}

extern "C" int polydet_batch_set_chunk_words(polydet_batch_t b, uint64_t words) {
  if (!b || words < 1) return POLYDET_EINVAL;
  b->chunk_words = words;
  update_ws(b);
  return POLYDET_OK;
}

// One-variable jobs: the partial tensor is the coefficients mod p_q,
// out[q][entry][Lp] (l < L written).
__global__ void repack_kernel(const int32_t *__restrict__ coeffs, uint32_t *__restrict__ out,
                              int64_t n2, int L, int Lp, const ModP *__restrict__ mod) {
  const int q = blockIdx.y;
  const uint32_t p = mod[q].p;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < n2 * L;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = f / L;
    const int l = (int)(f - e * L);
    out[(int64_t)q * n2 * Lp + e * Lp + l] = reduce_i32(coeffs[f], p);
  }
}

extern "C" int polydet_batch_eval_n(polydet_batch_t b, int n, const int32_t *coeffs,
                                    uint32_t *partial, uint32_t *ws, void *stream) {
  if (!b || !coeffs || !partial || !ws || n < 0 || n > POLYDET_MAX_N) return POLYDET_EINVAL;
  cudaStream_t st0 = (cudaStream_t)stream;
  int rc = fan_begin(b, st0);
  if (rc) return rc;
  for (int j = 0; j < b->njobs; ++j) {
    polydet_plan_s *pl = b->plans[j];
    if (n && pl->n != n) continue;
    cudaStream_t st = b->fan[j % kFan];
    uint32_t *scratch = ws + kWsHead + (uint64_t)(j % kFan) * b->scratch_stride;
    if (b->mode[pl->n] == POLYDET_BATCH_MATERIALIZED) {
      rc = pd_eval_head(pl, coeffs + b->coeff_off[j], 0, pl->P, partial + b->part_off[j], scratch, st);
      if (rc) return rc;
      continue;
    }
    if (pl->nvars == 1) {
      const int64_t n2 = (int64_t)pl->n * pl->n;
      const int L = pl->d[0] + 1;
      const unsigned blocks = (unsigned)std::min<int64_t>((n2 * L + 255) / 256, 1024);
      repack_kernel<<<dim3(blocks, pl->P), 256, 0, st>>>(coeffs + b->coeff_off[j],
                                                         partial + b->part_off[j], n2, L, b->Lp[j],
                                                         pl->d_mod);
      PD_CUDA(cudaGetLastError());
      continue;
    }
    rc = pd_eval_partial(pl, coeffs + b->coeff_off[j], 0, pl->P, partial + b->part_off[j], b->Lp[j],
                         scratch, st);
    if (rc) return rc;
  }
  return fan_end(b, st0);
}

extern "C" int polydet_batch_eval(polydet_batch_t b, const int32_t *coeffs, uint32_t *partial,
                                  uint32_t *ws, void *stream) {
  return polydet_batch_eval_n(b, 0, coeffs, partial, ws, stream);
}

// Materialized order: per job and chunk of primes, the first variable's pass
// into one of two chunk buffers, then the condensation kernel over it.  The
// passes run on a side stream, so the pass of chunk c + 1 overlaps the
// condensation of chunk c (filling the SMs its last wave leaves idle); a
// buffer is refilled only after the condensation that read it.  Event
// dependencies only: the whole sequence can be captured in a CUDA graph.
static int condense_materialized(polydet_batch_s *b, int n, const uint32_t *partial,
                                 uint32_t *detvals, uint32_t *ws, cudaStream_t st) {
  cudaStream_t sd = b->side;
  PD_CUDA(cudaEventRecord(b->ev[4], st));  // fork
  PD_CUDA(cudaStreamWaitEvent(sd, b->ev[4], 0));
  int c = 0;
  for (int j : b->jobs_of[n]) {
    polydet_plan_s *pl = b->plans[j];
    const int cp = chunk_primes(b, pl);
    const EvLayout lay = pd_tail_layout(pl);
    for (int lo = 0; lo < pl->P; lo += cp, ++c) {
      const int hi = std::min(pl->P, lo + cp);
      const int buf = c & 1;
      uint32_t *chunk = ws + kWsHead + (uint64_t)buf * b->chunk_max;
      if (c >= 2) PD_CUDA(cudaStreamWaitEvent(sd, b->ev[2 + buf], 0));  // its last reader is done
      int rc = pd_eval_tail(pl, partial + b->part_off[j], 0, lo, hi, 0, pl->M[0], chunk, lay, sd);
      if (rc) return rc;
      PD_CUDA(cudaEventRecord(b->ev[buf], sd));
      PD_CUDA(cudaStreamWaitEvent(st, b->ev[buf], 0));
      rc = pd_launch_condense(pl, chunk, lay, lo, hi - lo, detvals + b->det_off[j] + (int64_t)lo * pl->G,
                              st, b->condense_ctas);
      if (rc) return rc;
      PD_CUDA(cudaEventRecord(b->ev[2 + buf], st));
    }
  }
  PD_CUDA(cudaEventRecord(b->ev[5], sd));  // join
  PD_CUDA(cudaStreamWaitEvent(st, b->ev[5], 0));
  return POLYDET_OK;
}

extern "C" int polydet_batch_condense_n(polydet_batch_t b, int n, const uint32_t *partial,
                                        uint32_t *detvals, uint32_t *ws, void *stream) {
  if (!b || !partial || !detvals || !ws || n < 0 || n > POLYDET_MAX_N) return POLYDET_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long *counters = reinterpret_cast<unsigned long long *>(ws);
  if (n == 0) {
    PD_CUDA(cudaMemsetAsync(counters, 0, kCounterWords * sizeof(uint32_t), st));
  } else {
    PD_CUDA(cudaMemsetAsync(counters + n, 0, sizeof(unsigned long long), st));
  }
  for (int m = 1; m <= POLYDET_MAX_N; ++m) {
    if ((n && m != n) || b->segs[m].empty()) continue;
    if (b->mode[m] == POLYDET_BATCH_MATERIALIZED) {
      int rc = condense_materialized(b, m, partial, detvals, ws, st);
      if (rc) return rc;
      continue;
    }
    int rc = pd_fused_launch(m, b->d_segs[m], (int)b->segs[m].size(), b->nitems[m], partial,
                             detvals, counters + m, b->threads[m], b->blocks[m], b->qwords[m], b->nbuf[m], st);
    if (rc) return rc;
  }
  return POLYDET_OK;
}

extern "C" int polydet_batch_condense(polydet_batch_t b, const uint32_t *partial, uint32_t *detvals,
                                      uint32_t *ws, void *stream) {
  return polydet_batch_condense_n(b, 0, partial, detvals, ws, stream);
}

extern "C" int polydet_batch_interp(polydet_batch_t b, const uint32_t *detvals, uint32_t *residues,
                                    uint32_t *ws, void *stream) {
  if (!b || !detvals || !residues || !ws) return POLYDET_EINVAL;
  cudaStream_t st0 = (cudaStream_t)stream;
  int rc = fan_begin(b, st0);
  if (rc) return rc;
  for (int j = 0; j < b->njobs; ++j) {
    polydet_plan_s *pl = b->plans[j];
    rc = polydet_interp(pl, detvals + b->det_off[j], 0, pl->P, residues + b->res_off[j],
                        ws + kWsHead + (uint64_t)(j % kFan) * b->scratch_stride, b->fan[j % kFan]);
    if (rc) return rc;
  }
  return fan_end(b, st0);
}

extern "C" int polydet_batch_crt(polydet_batch_t b, const uint32_t *residues, uint32_t *limbs,
                                 void *stream) {
  if (!b || !residues || !limbs) return POLYDET_EINVAL;
  cudaStream_t st0 = (cudaStream_t)stream;
  int rc = fan_begin(b, st0);
  if (rc) return rc;
  for (int j = 0; j < b->njobs; ++j) {
    rc = polydet_crt(b->plans[j], residues + b->res_off[j], limbs + b->limb_off[j], b->fan[j % kFan]);
    if (rc) return rc;
  }
  return fan_end(b, st0);
}

extern "C" int polydet_batch_sync_status(polydet_batch_t b, void *stream, uint32_t *status_out) {
  if (!b) return POLYDET_EINVAL;
  // every job plan shares the batch's word: reading one plan reads them all
  return polydet_sync_status(b->plans[0], stream, status_out);
}
