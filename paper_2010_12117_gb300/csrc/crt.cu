// Mixed-radix CRT (Sec. 3.4, Algorithm 4): one thread per determinant
// coefficient, as in the paper.
//
// Digits (standard Garner, the reading of the paper's garbled constants):
//   alpha_0 = x_0,
//   alpha_i = (x_i - sum_{j<i} alpha_j * (prod_{l<j} p_l mod p_i)) * c_i mod p_i,
//   c_i = (prod_{l<i} p_l)^-1 mod p_i,
// so X = sum_i alpha_i prod_{l<i} p_l, evaluated by Horner's rule
// X = alpha_0 + p_0 (alpha_1 + p_1 (...)) on 32-bit limbs, then lifted to
// (-M/2, M/2) and stored as W little-endian two's-complement words.
// The digits and the limbs of a CTA sit in shared memory as [word][thread]
// so that the output tile [coefficient][W] is written with coalesced stores.
#include "common.cuh"

__global__ void __launch_bounds__(128) crt_kernel(const uint32_t *__restrict__ res,
                                                  uint32_t *__restrict__ limbs, int64_t C, int P,
                                                  int W, const ModP *__restrict__ mod,
                                                  const uint32_t *__restrict__ garner,
                                                  const uint32_t *__restrict__ mhalf,
                                                  const uint32_t *__restrict__ mfull) {
  extern __shared__ uint32_t sh[];
  const int bd = blockDim.x, tid = threadIdx.x;
  uint32_t *alpha = sh;          // [P][bd]
  uint32_t *X = sh + P * bd;     // [W][bd]
  const int64_t c0 = (int64_t)blockIdx.x * bd;
  const int64_t c = c0 + tid;
  const bool act = c < C;

  for (int i = 0; i < P; ++i) {
    const ModP m = mod[i];
    const uint32_t x = act ? res[(int64_t)i * C + c] : 0u;
    uint32_t acc = 0u;
    for (int j = 0; j < i; ++j)
      acc = addm(acc, mmul(alpha[j * bd + tid], __ldg(garner + i * P + j), m.p, m.pinv), m.p);
    alpha[i * bd + tid] = mmul(subm(x, acc, m.p), __ldg(garner + i * P + i), m.p, m.pinv);
  }

  for (int w = 0; w < W; ++w) X[w * bd + tid] = 0u;
  X[tid] = alpha[(P - 1) * bd + tid];
  for (int i = P - 2; i >= 0; --i) {
    const uint32_t pi = mod[i].p;
    uint64_t carry = alpha[i * bd + tid];
    const int lim = min(W, P - i);
    for (int w = 0; w < lim; ++w) {
      const uint64_t t = (uint64_t)X[w * bd + tid] * pi + carry;
      X[w * bd + tid] = (uint32_t)t;
      carry = t >> 32;
    }
  }

  int cmp = 0;  // compare X with (M - 1) / 2 from the top word down
  for (int w = W - 1; w >= 0; --w) {
    const uint32_t xv = X[w * bd + tid], hv = __ldg(mhalf + w);
    if (cmp == 0) cmp = (xv > hv) ? 1 : ((xv < hv) ? -1 : 0);
  }
  if (cmp > 0) {  // X - M
    uint32_t borrow = 0u;
    for (int w = 0; w < W; ++w) {
      const uint64_t t = (uint64_t)X[w * bd + tid] - __ldg(mfull + w) - borrow;
      X[w * bd + tid] = (uint32_t)t;
      borrow = (uint32_t)(t >> 63);
    }
  }
  __syncthreads();

  const int64_t ncoef = min((int64_t)bd, C - c0);
  for (int64_t f = tid; f < ncoef * W; f += bd) {
    const int64_t cc = f / W;
    const int w = (int)(f - cc * W);
    limbs[c0 * W + f] = X[w * bd + cc];
  }
}

// The same computation with the prime count a compile-time constant (P <= 32,
// so W <= P): digits, limbs and the Horner carries stay in registers, and a
// grid-stride loop covers the coefficients.  The constants of the P-prime CRT
// are passed by value: kernel parameters live in the constant bank, so every
// table entry (indexed at compile time) is an instruction operand, not a load.
template <int PT>
struct CrtTab {
  uint32_t gs[PT * PT];  // see polydet_plan_s::crt_gs
  uint32_t p[PT], pinv[PT];
};

template <int PT>
__global__ void __launch_bounds__(256) crt_kernel_p(const uint32_t *__restrict__ res,
                                                    uint32_t *__restrict__ limbs, int64_t C, int W,
                                                    const CrtTab<PT> tab) {
  // per warp: its 32 coefficients' limbs, written out as one contiguous run
  // (coefficients c .. c + 31 own words [c W, (c + 32) W) of the output)
  __shared__ uint32_t stage[256 / 32][32 * PT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *sw = stage[warp];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // residues of the next coefficient are loaded while this one is computed
  uint32_t xn[PT];
  int64_t c0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  if (c0 < C) {
    const uint32_t *rp = res + (c0 + lane < C ? c0 + lane : C - 1);
#pragma unroll
    for (int i = 0; i < PT; ++i, rp += C) xn[i] = __ldg(rp);
  }
  for (; c0 < C; c0 += stride) {
    uint32_t x[PT], al[PT];
#pragma unroll
    for (int i = 0; i < PT; ++i) x[i] = xn[i];
    if (c0 + stride < C) {
      // the warp stays whole: lanes past the end read the last coefficient
      const uint32_t *rp = res + (c0 + stride + lane < C ? c0 + stride + lane : C - 1);
#pragma unroll
      for (int i = 0; i < PT; ++i, rp += C) xn[i] = __ldg(rp);
    }
    // Garner digits (Sec. 3.4): alpha_i = x_i c_i - sum_{j<i} alpha_j m_j c_i
    // mod p_i as one dot product; three 62-bit products share one REDC (every
    // prime of a plan of at most 32 is at most PD_FOLD3_MAX, see redc3)
    al[0] = x[0];
#pragma unroll
    for (int i = 1; i < PT; ++i) {
      const uint32_t p = tab.p[i], pinv = tab.pinv[i];
      uint32_t acc = 0u;
#pragma unroll
      for (int j = 0; j <= i; j += 3) {
        uint64_t sum = (uint64_t)(j < i ? al[j] : x[i]) * tab.gs[i * PT + j];
        if (j + 1 <= i) sum += (uint64_t)(j + 1 < i ? al[j + 1] : x[i]) * tab.gs[i * PT + j + 1];
        if (j + 2 <= i) sum += (uint64_t)(j + 2 < i ? al[j + 2] : x[i]) * tab.gs[i * PT + j + 2];
        const uint32_t r = (j + 2 <= i) ? redc3(sum, p, pinv) : redc(sum, p, pinv);
        acc = (j == 0) ? r : addm(acc, r, p);
      }
      al[i] = acc;
    }
    // symmetric lift from the digits: X > (M - 1) / 2 exactly when the digit
    // vector, read from the top, first differs from that of (M - 1) / 2, whose
    // digits are (p_j - 1) / 2, by exceeding it.  Then X - M = -(Y + 1) with
    // Y = M - 1 - X, whose digits are p_j - 1 - alpha_j: Horner on those
    // digits and the bitwise complement of the words give X - M in two's
    // complement.
    int cmp = 0;
#pragma unroll
    for (int i = PT - 1; i >= 0; --i) {
      const uint32_t h = (tab.p[i] - 1u) >> 1;
      if (cmp == 0) cmp = (al[i] > h) ? 1 : ((al[i] < h) ? -1 : 0);
    }
    const bool neg = cmp > 0;
#pragma unroll
    for (int i = 0; i < PT; ++i) al[i] = neg ? tab.p[i] - 1u - al[i] : al[i];
    // mixed radix to binary by Horner: X = (..(alpha_{P-1} p_{P-2} + alpha_{P-2}) ..) p_0 + alpha_0
    uint32_t X[PT];
#pragma unroll
    for (int w = 0; w < PT; ++w) X[w] = 0u;
    X[0] = al[PT - 1];
#pragma unroll
    for (int i = PT - 2; i >= 0; --i) {
      uint64_t carry = al[i];
      const uint32_t pi = tab.p[i];
#pragma unroll
      for (int w = 0; w < PT - i; ++w) {
        const uint64_t t = (uint64_t)X[w] * pi + carry;
        X[w] = (uint32_t)t;
        carry = t >> 32;
      }
    }
#pragma unroll
    for (int w = 0; w < PT; ++w)
      if (w < W) sw[lane * W + w] = neg ? ~X[w] : X[w];
    __syncwarp();
    const int nw = (C - c0 < 32 ? (int)(C - c0) : 32) * W;  // words of this warp's coefficients
    uint32_t *o = limbs + c0 * W;
#pragma unroll
    for (int k = 0; k < PT; ++k) {  // W <= PT rounds of 32 consecutive words
      const int f = lane + 32 * k;
      if (k < W && f < nw) o[f] = sw[f];
    }
    __syncwarp();
  }
}

template <int PT>
static int launch_crt_p(const polydet_plan_s *pl, const uint32_t *residues, uint32_t *limbs,
                        cudaStream_t st) {
  if (pl->P == PT) {
    int dev = 0, sms = 0;
    PD_CUDA(cudaGetDevice(&dev));
    PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CrtTab<PT> tab;
    for (int i = 0; i < PT * PT; ++i) tab.gs[i] = pl->crt_gs[i];
    for (int i = 0; i < PT; ++i) {
      tab.p[i] = pl->mod_h[i].p;
      tab.pinv[i] = pl->mod_h[i].pinv;
    }
    const int threads = 256;
    const int64_t want = (pl->C + threads - 1) / threads;
    const unsigned blocks = (unsigned)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    crt_kernel_p<PT><<<blocks, threads, 0, st>>>(residues, limbs, pl->C, pl->W, tab);
    PD_CUDA(cudaGetLastError());
    return POLYDET_OK;
  }
  if constexpr (PT < 32) return launch_crt_p<PT + 1>(pl, residues, limbs, st);
  return POLYDET_EINVAL;
}

extern "C" int polydet_crt(polydet_plan_t pl, const uint32_t *residues, uint32_t *limbs,
                           void *stream) {
  if (!pl || !residues || !limbs) return POLYDET_EINVAL;
  if (pl->P <= 32 && pl->W <= pl->P) return launch_crt_p<1>(pl, residues, limbs, (cudaStream_t)stream);
  const int threads = 128;
  const size_t smem = (size_t)(pl->P + pl->W) * threads * sizeof(uint32_t);
  static PdPerDevice attr;
  int rc = pd_once_per_device(attr, [] {
    PD_CUDA(cudaFuncSetAttribute(crt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    return POLYDET_OK;
  });
  if (rc) return rc;
  const unsigned blocks = (unsigned)((pl->C + threads - 1) / threads);
  crt_kernel<<<blocks, threads, smem, (cudaStream_t)stream>>>(residues, limbs, pl->C, pl->P, pl->W,
                                                               pl->d_mod, pl->d_garner, pl->d_mhalf,
                                                               pl->d_mfull);
  PD_CUDA(cudaGetLastError());
  return POLYDET_OK;
}

// Early termination (no counterpart in the paper): digit i of every
// coefficient, from the stored digits 0 .. i-1, and whether the symmetric
// reconstruction from the first i primes survives prime i.  With
// X_i = sum_{j<i} alpha_j prod_{l<j} p_l in [0, M_i), the symmetric lift is
// X_i itself when X_i <= (M_i - 1) / 2 and X_i - M_i otherwise; it is also
// the lift over M_{i+1} exactly when alpha_i = 0 (first case) or
// alpha_i = p_i - 1 (second case).  The mixed-radix digits of (M_i - 1) / 2
// are (p_j - 1) / 2 for every j (the sum telescopes), so the comparison of
// X_i with it runs over the digits from the top.
__global__ void __launch_bounds__(256) crt_check_kernel(const uint32_t *__restrict__ res,
                                                        uint32_t *__restrict__ digits, int64_t C,
                                                        int P, int i, const ModP *__restrict__ mod,
                                                        const uint32_t *__restrict__ garner,
                                                        uint32_t *__restrict__ unstable) {
  const ModP m = mod[i];
  bool bad = false;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
       c += (int64_t)gridDim.x * blockDim.x) {
    if (i == 1) digits[c] = res[c];  // alpha_0 = x_0
    uint32_t acc = 0u;
    int cmp = 0;  // X_i against (M_i - 1) / 2, decided by the highest differing digit
    for (int j = i - 1; j >= 0; --j) {
      const uint32_t a = digits[(int64_t)j * C + c];
      acc = addm(acc, mmul(a, __ldg(garner + i * P + j), m.p, m.pinv), m.p);
      const uint32_t h = (mod[j].p - 1u) >> 1;
      if (cmp == 0) cmp = (a > h) ? 1 : ((a < h) ? -1 : 0);
    }
    const uint32_t x = res[(int64_t)i * C + c];
    const uint32_t ai = mmul(subm(x, acc, m.p), __ldg(garner + i * P + i), m.p, m.pinv);
    digits[(int64_t)i * C + c] = ai;
    bad |= (cmp > 0) ? (ai != m.p - 1u) : (ai != 0u);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(unstable, 1u);
}

extern "C" int polydet_crt_check(polydet_plan_t pl, const uint32_t *residues, uint32_t *digits,
                                 int i, uint32_t *unstable, void *stream) {
  if (!pl || !residues || !digits || !unstable || i < 1 || i >= pl->P) return POLYDET_EINVAL;
  int dev = 0, sms = 0;
  PD_CUDA(cudaGetDevice(&dev));
  PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256;
  const int64_t want = (pl->C + threads - 1) / threads;
  const unsigned blocks = (unsigned)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
  crt_check_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(residues, digits, pl->C, pl->P, i,
                                                                 pl->d_mod, pl->d_garner, unstable);
  PD_CUDA(cudaGetLastError());
  return POLYDET_OK;
}
