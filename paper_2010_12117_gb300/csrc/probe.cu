// Measurement utility: the integer-pipe ceilings that bound condensation.
//
// Four in-register streams with eight independent values per thread, enough
// warps per SM to hide latency, and no memory traffic.  Every product of an
// iteration takes at least one operand computed in the previous iteration
// (value j is updated from values j, j + 1, ... of the last iteration), so that
// no product is loop-invariant and none can be hoisted out of the loop, as
// in the elimination, where every operand is a run-time value:
//  - plain 32-bit multiply-adds (x = x * x + c), the IMAD rate;
//  - the single-step update r = (a*b - c*d) / R mod p (two 32x32->64
//    multiply-adds, one REDC), the fused-update rate;
//  - the two-step element update r = (a*b + c*d + e*f) / R mod p (three
//    multiply-adds, one REDC; each stands for two single-step updates) and
//    the three-step one (four multiply-adds, one REDC; three updates), the
//    rates that bound the condensation kernels' fast pass.
// The rates bound the determinant kernels the way a copy bounds a memory
// kernel.
#include "common.cuh"

__global__ void __launch_bounds__(256) imad_probe(uint32_t *out, int iters, uint32_t seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = seed + tid * 8u + j;
  // x <- x * x + j: a quadratic map, so no two iterations fold into one
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = x[j] * x[j] + (uint32_t)j;
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s ^= x[j];
  if (s == 0x12345678u) out[tid] = s;  // practically never taken; keeps the chains live
}

__global__ void __launch_bounds__(256) update_probe(uint32_t *out, int iters, uint32_t p,
                                                    uint32_t pinv, uint32_t seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = (seed + tid * 8u + j * 7919u) % p;
  const uint32_t piv = (seed ^ 0x5bd1e995u) % p, c = (seed + 12345u) % p;
  for (int it = 0; it < iters; ++it) {
    uint32_t b[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) b[j] = mfms(piv, a[j], a[(j + 1) & 7], c, p, pinv);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = b[j];
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s ^= a[j];
  if (s == 0x12345678u) out[tid] = s;
}

__global__ void __launch_bounds__(256) pair_probe(uint32_t *out, int iters, uint32_t p,
                                                  uint32_t pinv, uint32_t seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = (seed + tid * 8u + j * 7919u) % p;
  const uint32_t d2 = (seed ^ 0x5bd1e995u) % p, c1 = (seed + 12345u) % p, c2 = (seed + 54321u) % p;
  for (int it = 0; it < iters; ++it) {
    uint32_t b[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) b[j] = mfms3(d2, a[j], c1, a[(j + 1) & 7], c2, a[(j + 2) & 7], p, pinv);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = b[j];
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s ^= a[j];
  if (s == 0x12345678u) out[tid] = s;
}

__global__ void __launch_bounds__(256) triple_probe(uint32_t *out, int iters, uint32_t p,
                                                    uint32_t pinv, uint32_t seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = (seed + tid * 8u + j * 7919u) % p;
  const uint32_t d3 = (seed ^ 0x5bd1e995u) % p, c0 = (seed + 12345u) % p, c1 = (seed + 54321u) % p,
                 c2 = (seed + 99991u) % p;
  for (int it = 0; it < iters; ++it) {
    uint32_t b[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      b[j] = redc4((uint64_t)d3 * a[j] + (uint64_t)c0 * a[(j + 1) & 7] + (uint64_t)c1 * a[(j + 2) & 7] +
                       (uint64_t)c2 * a[(j + 3) & 7],
                   p, pinv);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = b[j];
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s ^= a[j];
  if (s == 0x12345678u) out[tid] = s;
}

extern "C" int polydet_probe_int_peaks(void *stream, double *imad_per_s, double *update_per_s,
                                       double *pair_update_per_s, double *triple_update_per_s) {
  if (!imad_per_s || !update_per_s || !pair_update_per_s || !triple_update_per_s) return POLYDET_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  PD_CUDA(cudaGetDevice(&dev));
  PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 8;
  uint32_t *out = nullptr;  // never written in practice; a valid target all the same
  PD_CUDA(cudaMallocAsync((void **)&out, (size_t)blocks * threads * sizeof(uint32_t), st));
  cudaEvent_t e0, e1;
  PD_CUDA(cudaEventCreate(&e0));
  PD_CUDA(cudaEventCreate(&e1));
  const uint32_t p = 2130706433u;
  uint32_t pinv = 1;
  for (int i = 0; i < 5; ++i) pinv *= 2u - p * pinv;
  const int iters = 4096;
  float ms = 0;
  // warm-up, then timed
  imad_probe<<<blocks, threads, 0, st>>>(out, iters, 1u);
  PD_CUDA(cudaEventRecord(e0, st));
  imad_probe<<<blocks, threads, 0, st>>>(out, iters, 2u);
  PD_CUDA(cudaEventRecord(e1, st));
  PD_CUDA(cudaEventSynchronize(e1));
  PD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  *imad_per_s = (double)blocks * threads * iters * 8.0 / (ms * 1e-3);
  update_probe<<<blocks, threads, 0, st>>>(out, iters / 4, p, pinv, 1u);
  PD_CUDA(cudaEventRecord(e0, st));
  update_probe<<<blocks, threads, 0, st>>>(out, iters / 4, p, pinv, 2u);
  PD_CUDA(cudaEventRecord(e1, st));
  PD_CUDA(cudaEventSynchronize(e1));
  PD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  *update_per_s = (double)blocks * threads * (iters / 4) * 8.0 / (ms * 1e-3);
  const uint32_t p3 = 1863319553u;  // a table prime <= PD_FOLD3_MAX, as mfms3 needs
  uint32_t pinv3 = 1;
  for (int i = 0; i < 5; ++i) pinv3 *= 2u - p3 * pinv3;
  pair_probe<<<blocks, threads, 0, st>>>(out, iters / 4, p3, pinv3, 1u);
  PD_CUDA(cudaEventRecord(e0, st));
  pair_probe<<<blocks, threads, 0, st>>>(out, iters / 4, p3, pinv3, 2u);
  PD_CUDA(cudaEventRecord(e1, st));
  PD_CUDA(cudaEventSynchronize(e1));
  PD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  *pair_update_per_s = (double)blocks * threads * (iters / 4) * 8.0 / (ms * 1e-3);
  triple_probe<<<blocks, threads, 0, st>>>(out, iters / 4, p, pinv, 1u);
  PD_CUDA(cudaEventRecord(e0, st));
  triple_probe<<<blocks, threads, 0, st>>>(out, iters / 4, p, pinv, 2u);
  PD_CUDA(cudaEventRecord(e1, st));
  PD_CUDA(cudaEventSynchronize(e1));
  PD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  *triple_update_per_s = (double)blocks * threads * (iters / 4) * 8.0 / (ms * 1e-3);
  PD_CUDA(cudaFreeAsync(out, st));
  PD_CUDA(cudaStreamSynchronize(st));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return POLYDET_OK;
}
