// Host side of libpolydet: the prime table (Eq. 1), the coefficient bound and
// prime count (Sec. 2), plan construction (grid sizes, roots of unity,
// twiddles, Montgomery and Garner constants) and status plumbing.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"

static char g_err[256] = "";

void pd_set_error(const char *what, cudaError_t e) {
  snprintf(g_err, sizeof g_err, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char *polydet_last_error(void) { return g_err; }

// ---------------------------------------------------------------------------
// Prime table: p = c * 2^20 + 1 in (2^30, 2^31): the 67 primes up to
// PD_FOLD3_MAX first, largest first, then the 24 above it, largest first (the
// condensation's two-step elimination needs p <= PD_FOLD3_MAX, so every
// plan of up to 67 primes runs it on all of them).  Primality by
// Miller-Rabin with bases 2, 7, 61 (deterministic below 4,759,123,141).
// ---------------------------------------------------------------------------
static bool is_prime_u32(uint32_t n) {
  if (n < 2) return false;
  for (uint32_t q : {2u, 3u, 5u, 7u, 11u, 13u, 61u})
    if (n % q == 0) return n == q;
  uint32_t d = n - 1;
  int s = 0;
  while (!(d & 1)) {
    d >>= 1;
    ++s;
  }
  for (uint32_t a : {2u, 7u, 61u}) {
    uint32_t x = h_powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; ++r) {
      x = h_mulmod(x, x, n);
      if (x == n - 1) {
        comp = false;
        break;
      }
    }
    if (comp) return false;
  }
  return true;
}

static const std::vector<uint32_t> &prime_table() {
  static std::vector<uint32_t> t;
  if (t.empty()) {
    for (int above = 0; above < 2; ++above) {
      for (uint32_t c = (0x7fffffffu >> 20); c > (0x40000000u >> 20); --c) {
        uint32_t p = (c << 20) + 1u;
        if ((p > PD_FOLD3_MAX) == (above == 1) && p > 0x40000000u && p < 0x80000000u && is_prime_u32(p))
          t.push_back(p);
      }
    }
  }
  return t;
}

// Least generator of (Z/pZ)^*: p - 1 = c * 2^20.
static uint32_t least_generator(uint32_t p) {
  std::vector<uint32_t> fs;
  uint32_t m = p - 1;
  for (uint32_t q = 2; (uint64_t)q * q <= m; ++q) {
    if (m % q == 0) {
      fs.push_back(q);
      while (m % q == 0) m /= q;
    }
  }
  if (m > 1) fs.push_back(m);
  for (uint32_t g = 2;; ++g) {
    bool ok = true;
    for (uint32_t q : fs)
      if (h_powmod(g, (p - 1) / q, p) == 1) {
        ok = false;
        break;
      }
    if (ok) return g;
  }
}

extern "C" int polydet_prime_table(uint32_t *out) {
  const auto &t = prime_table();
  if (out) memcpy(out, t.data(), t.size() * sizeof(uint32_t));
  return (int)t.size();
}

extern "C" int polydet_hadamard_primes(int n, const int64_t *entry_l1, int *nprimes_out,
                                       double *log2_bound_out) {
  if (n < 1 || n > POLYDET_MAX_N || !entry_l1 || !nprimes_out) return POLYDET_EINVAL;
  // log2 of prod_i sqrt(sum_j l1^2), rows and columns; the smaller is used.
  long double lr = 0, lc = 0;
  bool zero_r = false, zero_c = false;
  for (int i = 0; i < n; ++i) {
    long double sr = 0, sc = 0;
    for (int j = 0; j < n; ++j) {
      if (entry_l1[i * n + j] < 0 || entry_l1[j * n + i] < 0) return POLYDET_EINVAL;
      long double a = (long double)entry_l1[i * n + j];
      long double b = (long double)entry_l1[j * n + i];
      sr += a * a;
      sc += b * b;
    }
    if (sr == 0) zero_r = true; else lr += 0.5L * log2l(sr);
    if (sc == 0) zero_c = true; else lc += 0.5L * log2l(sc);
  }
  bool zero = zero_r || zero_c;  // a zero row or column: det = 0
  long double lb = zero ? -1.0L : (lr < lc ? lr : lc);
  const auto &t = prime_table();
  long double acc = 0;
  int P = 0;
  for (size_t i = 0; i < t.size(); ++i) {
    acc += log2l((long double)t[i]);
    if ((int)i + 1 >= 2 && acc > 1.0L + lb + 1e-6L) {
      P = (int)i + 1;
      break;
    }
  }
  if (!P) return POLYDET_EPRIMES;
  *nprimes_out = P;
  if (log2_bound_out) *log2_bound_out = (double)lb;
  return POLYDET_OK;
}

// Largest weight of a perfect matching of the n x n weights w (row-major;
// forbidden pairs marked by ok[i * n + j] == 0), by the Hungarian method with
// potentials on costs -w (O(n^3)); -1 when every perfect matching uses a
// forbidden pair.
static int64_t max_matching(int n, const std::vector<int64_t> &w, const std::vector<char> &ok) {
  const int64_t INF = (int64_t)1 << 50, FORBID = (int64_t)1 << 40;
  std::vector<int64_t> u(n + 1, 0), v(n + 1, 0), way(n + 1, 0), minv(n + 1);
  std::vector<int> pcol(n + 1, 0);  // pcol[j] = row matched to column j (1-based)
  std::vector<char> used(n + 1);
  auto cost = [&](int i, int j) { return ok[(size_t)i * n + j] ? -w[(size_t)i * n + j] : FORBID; };
  for (int i = 1; i <= n; ++i) {
    pcol[0] = i;
    int j0 = 0;
    std::fill(minv.begin(), minv.end(), INF);
    std::fill(used.begin(), used.end(), 0);
    do {
      used[j0] = 1;
      const int i0 = pcol[j0];
      int64_t delta = INF;
      int j1 = 0;
      for (int j = 1; j <= n; ++j) {
        if (used[j]) continue;
        const int64_t cur = cost(i0 - 1, j - 1) - u[i0] - v[j];
        if (cur < minv[j]) {
          minv[j] = cur;
          way[j] = j0;
        }
        if (minv[j] < delta) {
          delta = minv[j];
          j1 = j;
        }
      }
      for (int j = 0; j <= n; ++j) {
        if (used[j]) {
          u[pcol[j]] += delta;
          v[j] -= delta;
        } else {
          minv[j] -= delta;
        }
      }
      j0 = j1;
    } while (pcol[j0] != 0);
    do {
      const int j1 = (int)way[j0];
      pcol[j0] = pcol[j1];
      j0 = j1;
    } while (j0);
  }
  int64_t tot = 0;
  for (int j = 1; j <= n; ++j) {
    const int i = pcol[j] - 1;
    if (!ok[(size_t)i * n + (j - 1)]) return -1;
    tot += w[(size_t)i * n + (j - 1)];
  }
  return tot;
}

extern "C" int polydet_det_degree_bound(int n, int nvars, const int32_t *entry_degs, int32_t *D_out) {
  if (n < 1 || n > POLYDET_MAX_N || nvars < 1 || nvars > POLYDET_MAX_VARS || !entry_degs || !D_out)
    return POLYDET_EINVAL;
  const size_t nn = (size_t)n * n;
  std::vector<char> ok(nn);
  for (size_t e = 0; e < nn; ++e) {
    bool zero = true, bad = false;
    for (int v = 0; v < nvars; ++v) {
      const int32_t d = entry_degs[e * nvars + v];
      if (d >= 0) zero = false;
      if (d < -1) bad = true;
    }
    // an entry is either zero (-1 in every variable) or has a degree in each
    for (int v = 0; v < nvars && !zero; ++v)
      if (entry_degs[e * nvars + v] < 0) bad = true;
    if (bad) return POLYDET_EINVAL;
    ok[e] = zero ? 0 : 1;
  }
  std::vector<int64_t> w(nn);
  for (int v = 0; v < nvars; ++v) {
    for (size_t e = 0; e < nn; ++e) w[e] = ok[e] ? entry_degs[e * nvars + v] : 0;
    const int64_t best = max_matching(n, w, ok);
    D_out[v] = best < 0 ? 0 : (int32_t)best;
  }
  return POLYDET_OK;
}

static int pow2_at_least(int64_t x) {
  int64_t n = 1;
  while (n < x) n <<= 1;
  return (int)n;
}

// Words of the interpolation tables of one variable (see polydet_plan).
static int itab_words(int M, int L) {
  const int Jf = M / L, s = M % L;
  return Jf * Jf + Jf * L + L + s * L * Jf + s * s + Jf + 1;
}

// Inverse of an n x n matrix mod p by Gauss-Jordan (n < 8 here; always
// invertible: a scaled Vandermonde matrix of distinct nodes).
static std::vector<uint64_t> mat_inv_mod(std::vector<uint64_t> A, int n, uint64_t p) {
  std::vector<uint64_t> I((size_t)n * n, 0);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1;
  for (int c = 0; c < n; ++c) {
    int r = c;
    while (r < n && A[(size_t)r * n + c] == 0) ++r;
    for (int k = 0; k < n; ++k) {
      std::swap(A[(size_t)c * n + k], A[(size_t)r * n + k]);
      std::swap(I[(size_t)c * n + k], I[(size_t)r * n + k]);
    }
    const uint64_t iv = h_powmod((uint32_t)A[(size_t)c * n + c], p - 2, (uint32_t)p);
    for (int k = 0; k < n; ++k) {
      A[(size_t)c * n + k] = A[(size_t)c * n + k] * iv % p;
      I[(size_t)c * n + k] = I[(size_t)c * n + k] * iv % p;
    }
    for (int i = 0; i < n; ++i) {
      if (i == c || A[(size_t)i * n + c] == 0) continue;
      const uint64_t f = A[(size_t)i * n + c];
      for (int k = 0; k < n; ++k) {
        A[(size_t)i * n + k] = (A[(size_t)i * n + k] + (p - f) * A[(size_t)c * n + k]) % p;
        I[(size_t)i * n + k] = (I[(size_t)i * n + k] + (p - f) * I[(size_t)c * n + k]) % p;
      }
    }
  }
  return I;
}

// The interpolation tables of one (prime, variable), in the layout of
// polydet_plan's comment.  They depend on (p, w, N, L, M) only and are
// memoised for the process.
static void interp_tables(uint32_t p32, uint32_t w32, int N, int L, int M, uint32_t *dst) {
  static std::mutex mu;
  static std::map<std::tuple<uint32_t, uint32_t, int, int>, std::vector<uint32_t>> cache;
  const auto key = std::make_tuple(p32, w32, L, M);
  const int words = itab_words(M, L);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      memcpy(dst, it->second.data(), (size_t)words * sizeof(uint32_t));
      return;
    }
  }
  const uint64_t p = p32, w = w32;
  auto pw = [&](uint64_t b, uint64_t e) { return (uint64_t)h_powmod((uint32_t)b, e, p32); };
  auto inv = [&](uint64_t a) { return (uint64_t)h_powmod((uint32_t)(a % p), p - 2, p32); };
  auto mont = [&](uint64_t a) { return h_mont((uint32_t)(a % p), p32); };
  const int Jf = M / L, s = M % L;
  const uint64_t psi = pw(w, (uint64_t)(N / L)), ipsi = inv(psi);
  std::vector<uint64_t> z(Jf + 1);
  for (int j = 0; j <= Jf; ++j) z[j] = pw(w, (uint64_t)L * j);
  uint32_t *o = dst;
  // VfInv by Lagrange: Vf^-1[u][j] = [z^u] q_j(z) / q_j(z_j), q_j = Pi / (z - z_j)
  std::vector<uint64_t> pic(Jf + 1, 0);  // Pi(z), built factor by factor
  pic[0] = 1;
  for (int j = 0; j < Jf; ++j) {
    for (int k = j + 1; k >= 1; --k) pic[k] = (pic[k - 1] + (p - z[j]) * pic[k]) % p;
    pic[0] = (p - z[j]) * pic[0] % p;
  }
  std::vector<uint64_t> qc(Jf > 0 ? Jf : 1);
  for (int j = 0; j < Jf; ++j) {
    qc[Jf - 1] = 1;  // q_j = Pi / (z - z_j): q_{k-1} = pi_k + z_j q_k
    for (int k = Jf - 1; k >= 1; --k) qc[k - 1] = (pic[k] + z[j] * qc[k]) % p;
    uint64_t den = 0;
    for (int k = Jf - 1; k >= 0; --k) den = (den * z[j] + qc[k]) % p;
    const uint64_t id = inv(den);
    for (int u = 0; u < Jf; ++u) o[(size_t)u * Jf + j] = mont(qc[u] * id % p);
  }
  o += (size_t)Jf * Jf;
  const uint64_t Linv = inv((uint64_t)L);
  for (int j = 0; j < Jf; ++j)
    for (int r = 0; r < L; ++r) o[(size_t)j * L + r] = mont(Linv * inv(pw(w, (uint64_t)j * r)) % p);
  o += (size_t)Jf * L;
  for (int k = 0; k < L; ++k) o[k] = mont(pw(ipsi, (uint64_t)k));
  o += L;
  for (int t = 0; t < s; ++t)
    for (int r = 0; r < L; ++r)
      for (int u = 0; u < Jf; ++u)
        o[((size_t)t * L + r) * Jf + u] =
            mont(pw(psi, (uint64_t)t * r) * pw(w, (uint64_t)Jf * r) % p * pw(z[Jf], (uint64_t)u) % p);
  o += (size_t)s * L * Jf;
  if (s > 0) {
    uint64_t piz = 0;  // Pi(z_Jf)
    for (int k = Jf; k >= 0; --k) piz = (piz * z[Jf] + pic[k]) % p;
    std::vector<uint64_t> A((size_t)s * s);
    for (int t = 0; t < s; ++t)
      for (int r = 0; r < s; ++r) A[(size_t)t * s + r] = pw(psi, (uint64_t)t * r) * pw(w, (uint64_t)Jf * r) % p * piz % p;
    const std::vector<uint64_t> B = mat_inv_mod(A, s, p);
    for (int i = 0; i < s * s; ++i) o[i] = mont(B[i]);
  }
  o += (size_t)s * s;
  for (int k = 0; k <= Jf; ++k) o[k] = mont(pic[k]);
  std::lock_guard<std::mutex> lock(mu);
  cache.emplace(key, std::vector<uint32_t>(dst, dst + words));
}

// ---------------------------------------------------------------------------
// Plan tables are shared by every plan of the same shape (order, variables,
// entry and determinant degrees, primes, grid): one packed device block per
// shape, built on the first plan of that shape and kept, once its last plan
// is gone, until more than kCacheShapes unused shapes are held (least
// recently used first) or polydet_plan_cache_clear() is called.  A plan of
// a cached shape is a host copy of the shape's template plan: no host table
// is recomputed and no device memory is allocated for it (its status word
// aside, which a batch provides for its jobs).
// ---------------------------------------------------------------------------
namespace {
// Table blocks come from a private stream-ordered memory pool of the device
// and move on a private non-blocking stream, so that building a new shape or
// freeing an evicted one (a server's waves plan and drop many shapes) never
// synchronises the device the way cudaMalloc / cudaFree can: an upload waits
// for that stream alone, and a free is queued on it.  Tables are freed only
// once no plan of their shape is left, i.e. after every launch that read them
// has completed (plans are destroyed after their work, polydet_plan_destroy).
struct TableArena {
  cudaStream_t st = nullptr;
  cudaMemPool_t pool = nullptr;
};
std::mutex g_arena_mu;
TableArena g_arena[64];

int table_arena(TableArena **out) {
  int dev = 0;
  PD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return POLYDET_EINVAL;
  std::lock_guard<std::mutex> lock(g_arena_mu);
  TableArena &a = g_arena[dev];
  if (!a.st) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    PD_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = UINT64_MAX;  // hold freed blocks for the next shapes
    PD_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    cudaStream_t st = nullptr;
    PD_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    a.pool = pool;
    a.st = st;
  }
  *out = &a;
  return POLYDET_OK;
}

struct PlanTables {
  void *dev = nullptr;  // every device table of the shape, packed
  cudaStream_t st = nullptr;  // its arena's stream (frees are queued there)
  int refs = 0;
  uint64_t last_use = 0;
  bool cached = false;             // held by g_cache (else freed with its last plan)
  polydet_plan_s *tmpl = nullptr;  // host template: the plan's fields with device pointers set
};
constexpr size_t kCacheShapes = 256;
std::mutex g_cache_mu;
std::map<std::vector<int64_t>, PlanTables *> g_cache;
uint64_t g_cache_clock = 0;

std::vector<int64_t> shape_key(int dev, int n, int nvars, const int *d, const int *D, int P, int full) {
  std::vector<int64_t> k = {dev, n, nvars, P, full};
  for (int v = 0; v < nvars; ++v) {
    k.push_back(d[v]);
    k.push_back(D[v]);
  }
  return k;
}

void drop_unused(size_t keep) {  // with g_cache_mu held
  while (true) {
    size_t unused = 0;
    auto victim = g_cache.end();
    for (auto it = g_cache.begin(); it != g_cache.end(); ++it) {
      if (it->second->refs) continue;
      ++unused;
      if (victim == g_cache.end() || it->second->last_use < victim->second->last_use) victim = it;
    }
    if (unused <= keep || victim == g_cache.end()) return;
    cudaFreeAsync(victim->second->dev, victim->second->st);
    delete victim->second->tmpl;
    delete victim->second;
    g_cache.erase(victim);
  }
}
}  // namespace

static void free_plan(polydet_plan_s *pl) {
  if (!pl) return;
  if (!pl->status_shared && pl->tables)  // allocated with its tables, on their device's arena
    cudaFreeAsync(pl->d_status, static_cast<PlanTables *>(pl->tables)->st);
  if (pl->tables) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    PlanTables *t = static_cast<PlanTables *>(pl->tables);
    if (--t->refs == 0 && !t->cached) {
      cudaFreeAsync(t->dev, t->st);
      delete t->tmpl;
      delete t;
    }
    drop_unused(kCacheShapes);
  }
  delete pl;
}

extern "C" int polydet_plan_cache_clear(void) {
  {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    drop_unused(0);
  }
  // hand the freed blocks back to the device, not only to the pool
  std::lock_guard<std::mutex> lock(g_arena_mu);
  for (TableArena &a : g_arena) {
    if (!a.st) continue;
    PD_CUDA(cudaStreamSynchronize(a.st));
    PD_CUDA(cudaMemPoolTrimTo(a.pool, 0));
  }
  return POLYDET_OK;
}

// Bytes of a packed table block and the offset of each table (256-byte aligned).
struct Packer {
  std::vector<uint8_t> host;
  template <class T>
  size_t add(const std::vector<T> &v) {
    const size_t off = (host.size() + 255) / 256 * 256;
    host.resize(off + std::max<size_t>(v.size() * sizeof(T), sizeof(T)), 0);
    if (!v.empty()) memcpy(host.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
};

// The plan's own status word (or the batch's), then hand it out.
static int finish_plan(polydet_plan_s *pl, uint32_t *shared_status, polydet_plan_t *out) {
  if (shared_status) {
    pl->d_status = shared_status;
    pl->status_shared = 1;
  } else {
    pl->status_shared = 0;
    pl->d_status = nullptr;
    TableArena *arena = nullptr;
    const int arc = table_arena(&arena);
    cudaError_t e = arc ? cudaErrorUnknown
                        : cudaMallocFromPoolAsync((void **)&pl->d_status, sizeof(uint32_t), arena->pool,
                                                  arena->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_status, 0, sizeof(uint32_t), arena->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(arena->st);
    if (e != cudaSuccess) {
      pd_set_error("cudaMallocFromPoolAsync (status word)", e);
      if (pl->d_status && arena) cudaFreeAsync(pl->d_status, arena->st);
      pl->status_shared = 1;  // nothing of its own to free
      free_plan(pl);
      return POLYDET_ENOMEM;
    }
  }
  *out = pl;
  return POLYDET_OK;
}

int pd_plan_impl(polydet_plan_t *out, int n, int nvars, const int32_t *entry_deg,
                 const int32_t *det_deg, int nprimes, uint32_t flags, uint32_t *shared_status) {
  if (!out || n < 1 || n > POLYDET_MAX_N || nvars < 1 || nvars > POLYDET_MAX_VARS ||
      !entry_deg || (flags & ~POLYDET_FLAG_FULL_GRID))
    return POLYDET_EINVAL;
  const auto &table = prime_table();
  if (nprimes < 1) return POLYDET_EINVAL;
  if (nprimes > (int)table.size()) return POLYDET_EPRIMES;
  int dev_id = 0;
  PD_CUDA(cudaGetDevice(&dev_id));
  std::vector<int64_t> key;
  {
    int dd[POLYDET_MAX_VARS], DD[POLYDET_MAX_VARS];
    for (int v = 0; v < nvars; ++v) {
      if (entry_deg[v] < 0) return POLYDET_EINVAL;
      dd[v] = entry_deg[v];
      DD[v] = det_deg ? det_deg[v] : n * entry_deg[v];
    }
    key = shape_key(dev_id, n, nvars, dd, DD, nprimes, (flags & POLYDET_FLAG_FULL_GRID) ? 1 : 0);
  }
  polydet_plan_s *hit = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {  // a known shape: copy its template, share its tables
      PlanTables *t = it->second;
      ++t->refs;
      t->last_use = ++g_cache_clock;
      hit = new polydet_plan_s(*t->tmpl);
      hit->tables = t;
      hit->d_status = nullptr;
      hit->status_shared = 1;
    }
  }
  if (hit) return finish_plan(hit, shared_status, out);  // outside the lock: it may free the plan

  polydet_plan_s *pl = new polydet_plan_s();
  memset(pl, 0, sizeof *pl);
  pl->n = n;
  pl->nvars = nvars;
  pl->P = nprimes;
  pl->E = 1;
  pl->G = 1;
  pl->C = 1;
  int off = 0;
  for (int v = 0; v < nvars; ++v) {
    if (entry_deg[v] < 0) {
      delete pl;
      return POLYDET_EINVAL;
    }
    pl->d[v] = entry_deg[v];
    pl->D[v] = det_deg ? det_deg[v] : n * entry_deg[v];
    if (pl->D[v] < 0 || (int64_t)pl->D[v] > (int64_t)n * entry_deg[v]) {
      delete pl;
      return POLYDET_EINVAL;
    }
    // D_v + 1 nodes for the interpolation, and at least d_v + 1 points in
    // the transform so that an entry's d_v + 1 coefficients are not aliased
    int64_t need = std::max<int64_t>((int64_t)pl->D[v] + 1, (int64_t)pl->d[v] + 1);
    if (need > POLYDET_MAX_GRID_DIM) {
      delete pl;
      return POLYDET_EDEGREE;
    }
    pl->N[v] = pow2_at_least(need);
    int lg = 0;
    while ((1 << lg) < pl->N[v]) ++lg;
    pl->logN[v] = lg;
    pl->E *= (int64_t)(pl->d[v] + 1);
    pl->M[v] = (flags & POLYDET_FLAG_FULL_GRID) ? pl->N[v] : pl->D[v] + 1;
    pl->LPo[v] = (flags & POLYDET_FLAG_FULL_GRID) ? 1 : node_radix(pl->d[v]);
    pl->G *= pl->M[v];
    pl->C *= (int64_t)(pl->D[v] + 1);
    pl->tw_off[v] = off;
    off += pl->N[v];  // the whole circle: a twiddle is one load, no sign flip
  }
  pl->tw_len = off > 0 ? off : 1;

  // Primes, roots, Montgomery constants, twiddles.
  std::vector<ModP> mod(nprimes);
  std::vector<uint32_t> twf((size_t)nprimes * pl->tw_len, 0), twi((size_t)nprimes * pl->tw_len, 0);
  std::vector<uint32_t> ninv((size_t)nprimes * nvars), rn(nprimes);
  for (int q = 0; q < nprimes; ++q) {
    uint32_t p = table[q];
    pl->primes[q] = p;
    uint32_t inv = 1;  // Newton iteration for p^-1 mod 2^32
    for (int it = 0; it < 5; ++it) inv *= 2u - p * inv;
    mod[q].p = p;
    mod[q].pinv = inv;
    mod[q].r1 = h_mont(1, p);
    mod[q].r2 = h_mont(mod[q].r1, p);
    uint32_t g = least_generator(p);
    for (int v = 0; v < nvars; ++v) {
      int N = pl->N[v];
      uint32_t w = h_powmod(g, (uint64_t)(p - 1) / N, p);
      uint32_t wi = h_powmod(w, p - 2, p);
      pl->roots[q][v] = w;
      uint32_t x = 1, y = 1;
      for (int j = 0; j < N; ++j) {
        twf[(size_t)q * pl->tw_len + pl->tw_off[v] + j] = h_mont(x, p);
        twi[(size_t)q * pl->tw_len + pl->tw_off[v] + j] = h_mont(y, p);
        x = h_mulmod(x, w, p);
        y = h_mulmod(y, wi, p);
      }
      ninv[(size_t)q * nvars + v] = h_mont(h_powmod(N % p, p - 2, p), p);
    }
    rn[q] = h_powmod(mod[q].r1, (uint64_t)n, p);  // (R mod p)^n = R^n mod p
    pl->mod_h[q] = mod[q];
    pl->rn_h[q] = rn[q];
  }

  // Garner tables (Sec. 3.4 with the standard reading of its constants):
  // g[i][j] = (prod_{l<j} p_l mod p_i) * R for j < i, g[i][i] = c_i * R with
  // c_i = (prod_{l<i} p_l)^-1 mod p_i.
  std::vector<uint32_t> garner((size_t)nprimes * nprimes, 0);
  for (int i = 0; i < nprimes; ++i) {
    uint32_t p = table[i];
    uint32_t m = 1;
    for (int j = 0; j < i; ++j) {
      garner[(size_t)i * nprimes + j] = h_mont(m, p);
      m = h_mulmod(m, table[j] % p, p);
    }
    garner[(size_t)i * nprimes + i] = h_mont(h_powmod(m, p - 2, p), p);
  }
  if (nprimes <= 32) {
    for (int i = 0; i < nprimes; ++i) {
      const uint32_t p = table[i];
      uint32_t m = 1;
      for (int j = 0; j < i; ++j) m = h_mulmod(m, table[j] % p, p);
      const uint32_t ci = h_powmod(m, p - 2, p);  // (prod_{l<i} p_l)^-1 mod p_i
      uint32_t mj = 1;
      for (int j = 0; j < i; ++j) {
        const uint32_t t = h_mulmod(mj, ci, p);
        pl->crt_gs[i * nprimes + j] = h_mont(t ? p - t : 0u, p);
        mj = h_mulmod(mj, table[j] % p, p);
      }
      pl->crt_gs[i * nprimes + i] = h_mont(ci, p);
    }
  }
  // M = prod p as 32-bit limbs; W = ceil(bitlen(M) / 32).
  std::vector<uint32_t> M(nprimes + 1, 0);
  M[0] = 1;
  int used = 1;
  for (int i = 0; i < nprimes; ++i) {
    uint64_t carry = 0;
    for (int w = 0; w < used; ++w) {
      uint64_t t = (uint64_t)M[w] * table[i] + carry;
      M[w] = (uint32_t)t;
      carry = t >> 32;
    }
    if (carry) M[used++] = (uint32_t)carry;
  }
  pl->W = used;
  M.resize(used);
  std::vector<uint32_t> H(used);
  for (int w = 0; w < used; ++w) {  // (M - 1) / 2; M is odd
    uint32_t lo = (w == 0) ? (M[0] - 1u) : M[w];
    uint32_t hi_bit = (w + 1 < used) ? (M[w + 1] & 1u) : 0u;
    H[w] = (lo >> 1) | (hi_bit << 31);
  }
  for (int w = 0; w < used && w < 32; ++w) {
    pl->crt_mh[w] = H[w];
    pl->crt_mf[w] = M[w];
  }

  // Caller scratch per prime (words): evaluation keeps its odd passes there,
  // interpolation all passes but the last, ping-ponging between two halves.
  int64_t n2 = (int64_t)n * n;
  uint64_t eval_slot = 0, interp_slot = 0;
  for (int v = 1; v < nvars; v += 2) {  // eval pass v output: prod_{u<v} L_u * prod_{u>=v} M_u
    uint64_t s = 1;
    for (int u = 0; u < nvars; ++u) s *= (u < v) ? (uint64_t)(pl->d[u] + 1) : (uint64_t)pl->M[u];
    if (s > eval_slot) eval_slot = s;
  }
  for (int v = 1; v < nvars; ++v) {  // interp pass v output: prod_{u<v} M_u * prod_{u>=v} (D_u+1)
    uint64_t s = 1;
    for (int u = 0; u < nvars; ++u) s *= (u < v) ? (uint64_t)pl->M[u] : (uint64_t)(pl->D[u] + 1);
    if (s > interp_slot) interp_slot = s;
  }

  // Node grid interpolation tables (Sec. 3.3: the interpolating polynomial of
  // degree < M through M distinct nodes is unique), for the coset-structured
  // solve of ntt.cu: with the nodes in coset order (L = LPo[v], Jf = M / L
  // whole cosets, s = M mod L nodes of one more), P(x) = sum_r x^r Q_r(x^L)
  // and x^L = z_j = w^(L j) on coset j, so an inverse DFT of size L per coset
  // gives Q_r(z_j) and each Q_r is interpolated through z_0..z_{Jf-1}; the
  // last s nodes fix the top coefficient of Q_r for r < s.  Per (prime,
  // variable), Montgomery forms:
  //   VfInv [Jf][Jf]   inverse Vandermonde of z_0..z_{Jf-1} (V[j][u] = z_j^u)
  //   tw1   [Jf][L]    L^-1 w^(-j r)
  //   ipsi  [L]        psi^-k, psi = w^(N / L)
  //   H     [s][L][Jf] psi^(t r) w^(Jf r) z_Jf^u
  //   B     [s][s]     inverse of A[t][r] = psi^(t r) w^(Jf r) Pi(z_Jf), r, t < s
  //   pi    [Jf + 1]   coefficients of Pi(z) = prod_{j<Jf} (z - z_j)
  std::vector<uint32_t> itab;
  pl->full = (flags & POLYDET_FLAG_FULL_GRID) ? 1 : 0;
  if (!pl->full) {
    int off2 = 0;
    for (int v = 0; v < nvars; ++v) {
      pl->itab_off[v] = off2;
      off2 += itab_words(pl->M[v], pl->LPo[v]);
    }
    pl->itab_len = off2;
    itab.assign((size_t)nprimes * off2, 0u);
    for (int q = 0; q < nprimes; ++q) {
      for (int v = 0; v < nvars; ++v) {
        uint32_t *dst = itab.data() + (size_t)q * off2 + pl->itab_off[v];
        interp_tables(table[q], pl->roots[q][v], pl->N[v], pl->LPo[v], pl->M[v], dst);
      }
    }
  }
  pl->eval_ws_words = eval_slot * (uint64_t)n2;
  pl->interp_ws_words = 2 * interp_slot;

  // one packed block for every table; the plan becomes the shape's template
  Packer pk;
  const size_t o_mod = pk.add(mod), o_twf = pk.add(twf), o_twi = pk.add(twi), o_ninv = pk.add(ninv),
               o_rn = pk.add(rn), o_gar = pk.add(garner), o_mh = pk.add(H), o_mf = pk.add(M),
               o_itab = pk.add(itab);
  TableArena *arena = nullptr;
  int arc = table_arena(&arena);
  if (arc) {
    delete pl;
    return arc;
  }
  void *dev = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&dev, pk.host.size(), arena->pool, arena->st);
  if (e != cudaSuccess) {
    pd_set_error("cudaMallocFromPoolAsync", e);
    delete pl;
    return POLYDET_ENOMEM;
  }
  // pageable source: the copy is staged before the call returns; the stream
  // synchronisation makes the tables visible to every stream that follows
  e = cudaMemcpyAsync(dev, pk.host.data(), pk.host.size(), cudaMemcpyHostToDevice, arena->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(arena->st);
  if (e != cudaSuccess) {
    pd_set_error("cudaMemcpyAsync (plan tables)", e);
    cudaFreeAsync(dev, arena->st);
    delete pl;
    return POLYDET_ECUDA;
  }
  uint8_t *b = static_cast<uint8_t *>(dev);
  pl->d_mod = reinterpret_cast<ModP *>(b + o_mod);
  pl->d_tw_fwd = reinterpret_cast<uint32_t *>(b + o_twf);
  pl->d_tw_inv = reinterpret_cast<uint32_t *>(b + o_twi);
  pl->d_ninv = reinterpret_cast<uint32_t *>(b + o_ninv);
  pl->d_rn = reinterpret_cast<uint32_t *>(b + o_rn);
  pl->d_garner = reinterpret_cast<uint32_t *>(b + o_gar);
  pl->d_mhalf = reinterpret_cast<uint32_t *>(b + o_mh);
  pl->d_mfull = reinterpret_cast<uint32_t *>(b + o_mf);
  pl->d_itab = pl->full ? nullptr : reinterpret_cast<uint32_t *>(b + o_itab);
  for (int q = 0; q < n * n; ++q) pl->ent[q] = q;
  pl->nent = n * n;
  pl->nitems = n * n;
  PlanTables *t = new PlanTables();
  t->dev = dev;
  t->st = arena->st;
  t->tmpl = new polydet_plan_s(*pl);
  {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    t->refs = 1;
    t->last_use = ++g_cache_clock;
    // a shape built concurrently by two threads: the first one stays cached,
    // the other's tables go with its plan
    t->cached = g_cache.emplace(key, t).second;
  }
  pl->tables = t;
  return finish_plan(pl, shared_status, out);
}

extern "C" int polydet_plan(polydet_plan_t *out, int n, int nvars, const int32_t *entry_deg,
                            int nprimes, uint32_t flags) {
  return pd_plan_impl(out, n, nvars, entry_deg, nullptr, nprimes, flags, nullptr);
}

extern "C" int polydet_plan_degrees(polydet_plan_t *out, int n, int nvars, const int32_t *entry_deg,
                                    const int32_t *det_deg, int nprimes, uint32_t flags) {
  if (!det_deg) return POLYDET_EINVAL;
  return pd_plan_impl(out, n, nvars, entry_deg, det_deg, nprimes, flags, nullptr);
}

extern "C" int polydet_plan_set_entry_map(polydet_plan_t pl, const int32_t *map, int U) {
  if (!pl || !map || U < 0 || U > pl->n * pl->n) return POLYDET_EINVAL;
  const int n2 = pl->n * pl->n;
  std::vector<char> seen(U > 0 ? U : 1, 0);
  for (int e = 0; e < n2; ++e) {
    if (map[e] < -1 || map[e] >= U) return POLYDET_EINVAL;
    if (map[e] >= 0) seen[map[e]] = 1;
  }
  for (int u = 0; u < U; ++u)
    if (!seen[u]) return POLYDET_EINVAL;  // every distinct entry is used somewhere
  for (int e = 0; e < n2; ++e) pl->ent[e] = map[e] < 0 ? U : map[e];
  pl->nitems = U;
  pl->nent = U + 1;  // slot U holds the zero entry
  return POLYDET_OK;
}

// FNV-1a over an entry's coefficient words (the hash only groups candidates;
// equality is decided by comparing the words).
static uint64_t hash_words(const int32_t *x, int64_t len) {
  uint64_t h = 1469598103934665603ull;
  for (int64_t i = 0; i < len; ++i) {
    uint32_t w = (uint32_t)x[i];
    for (int b = 0; b < 4; ++b) {
      h ^= (w >> (8 * b)) & 0xffu;
      h *= 1099511628211ull;
    }
  }
  return h;
}

extern "C" int polydet_unique_entries(int n, int64_t E, const int32_t *coeffs, int32_t *map_out,
                                      int32_t *U_out, int32_t *unique_out) {
  if (n < 1 || n > POLYDET_MAX_N || E < 1 || !coeffs || !map_out || !U_out) return POLYDET_EINVAL;
  std::map<uint64_t, std::vector<int>> buckets;  // hash -> distinct entries (indices into firsts)
  std::vector<int> firsts;                        // matrix entry where each distinct entry first occurs
  for (int e = 0; e < n * n; ++e) {
    const int32_t *c = coeffs + (int64_t)e * E;
    bool zero = true;
    for (int64_t i = 0; i < E && zero; ++i) zero = c[i] == 0;
    if (zero) {
      map_out[e] = -1;
      continue;
    }
    auto &b = buckets[hash_words(c, E)];
    int found = -1;
    for (int u : b)
      if (memcmp(coeffs + (int64_t)firsts[u] * E, c, (size_t)E * sizeof(int32_t)) == 0) {
        found = u;
        break;
      }
    if (found < 0) {
      found = (int)firsts.size();
      firsts.push_back(e);
      b.push_back(found);
    }
    map_out[e] = found;
  }
  *U_out = (int32_t)firsts.size();
  if (unique_out)
    for (size_t u = 0; u < firsts.size(); ++u)
      memcpy(unique_out + (int64_t)u * E, coeffs + (int64_t)firsts[u] * E, (size_t)E * sizeof(int32_t));
  return POLYDET_OK;
}

extern "C" int polydet_plan_destroy(polydet_plan_t plan) {
  if (!plan) return POLYDET_EINVAL;
  free_plan(plan);
  return POLYDET_OK;
}

extern "C" int polydet_plan_query(polydet_plan_t pl, polydet_plan_info *info) {
  if (!pl || !info) return POLYDET_EINVAL;
  memset(info, 0, sizeof *info);
  info->n = pl->n;
  info->nvars = pl->nvars;
  info->P = pl->P;
  info->W = pl->W;
  info->E = pl->E;
  info->G = pl->G;
  info->C = pl->C;
  for (int v = 0; v < pl->nvars; ++v) {
    info->d[v] = pl->d[v];
    info->D[v] = pl->D[v];
    info->N[v] = pl->N[v];
    info->M[v] = pl->M[v];
  }
  info->flags = pl->full ? POLYDET_FLAG_FULL_GRID : 0u;
  info->eval_ws_words = pl->eval_ws_words;
  info->interp_ws_words = pl->interp_ws_words;
  info->entries = pl->nent;
  info->unique = (pl->nitems == pl->n * pl->n && pl->nent == pl->nitems) ? -1 : pl->nitems;
  return POLYDET_OK;
}

extern "C" int polydet_plan_primes(polydet_plan_t pl, uint32_t *primes_out) {
  if (!pl || !primes_out) return POLYDET_EINVAL;
  memcpy(primes_out, pl->primes, pl->P * sizeof(uint32_t));
  return POLYDET_OK;
}

extern "C" int polydet_plan_roots(polydet_plan_t pl, uint32_t *roots_out) {
  if (!pl || !roots_out) return POLYDET_EINVAL;
  for (int q = 0; q < pl->P; ++q)
    for (int v = 0; v < pl->nvars; ++v) roots_out[q * pl->nvars + v] = pl->roots[q][v];
  return POLYDET_OK;
}

extern "C" int polydet_plan_nodes(polydet_plan_t pl, int var, int32_t *exps_out) {
  if (!pl || !exps_out || var < 0 || var >= pl->nvars) return POLYDET_EINVAL;
  for (int k = 0; k < pl->M[var]; ++k) exps_out[k] = node_exp(k, pl->N[var], pl->LPo[var]);
  return POLYDET_OK;
}

extern "C" int polydet_sync_status(polydet_plan_t pl, void *stream, uint32_t *status_out) {
  if (!pl) return POLYDET_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t s = 0;
  PD_CUDA(cudaMemcpyAsync(&s, pl->d_status, sizeof s, cudaMemcpyDeviceToHost, st));
  PD_CUDA(cudaStreamSynchronize(st));
  PD_CUDA(cudaMemsetAsync(pl->d_status, 0, sizeof(uint32_t), st));
  PD_CUDA(cudaStreamSynchronize(st));
  if (status_out) *status_out = s;
  if (s & POLYDET_STATUS_TIMEOUT) return POLYDET_ETIMEOUT;
  if (s & POLYDET_STATUS_BOUND) return POLYDET_EBOUND;
  return POLYDET_OK;
}
