// fp32 multilayer perceptron 8 -> 64 -> 64 -> 2 (ReLU) that predicts a
// determinant job's run time and device memory from its shape; it drives
// admission in the serving loop.  It generalises the run-time prediction of
// Sec. 5 (T = C_p r^2 mean(T_e) mu) to the batched GPU form.
//
// Parameters, one flat float array (POLYDET_MLP_PARAMS = 4866):
//   W1[64][8] b1[64] W2[64][64] b2[64] W3[2][64] b3[2]   (row = output unit)
// Loss: mean squared error over the batch and both outputs,
//   L = 1/(2B) sum_b sum_o (y_bo - t_bo)^2.
// Kernels: forward (one thread per sample, weights in shared memory);
// backward in two deterministic passes - per-sample deltas, then one thread
// per parameter summing over the batch in a fixed order; Adam.
#include "common.cuh"

namespace {
constexpr int kIn = POLYDET_MLP_IN, kHid = POLYDET_MLP_HIDDEN, kOut = POLYDET_MLP_OUT;
constexpr int oW1 = 0, ob1 = oW1 + kHid * kIn, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid,
              oW3 = ob2 + kHid, ob3 = oW3 + kOut * kHid, kParams = ob3 + kOut;
static_assert(kParams == POLYDET_MLP_PARAMS, "parameter count");
}  // namespace

__global__ void __launch_bounds__(128) mlp_fwd_kernel(const float *__restrict__ prm,
                                                      const float *__restrict__ X, int B,
                                                      float *__restrict__ Y, float *__restrict__ H) {
  __shared__ float w[kParams];
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) w[i] = prm[i];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float x[kIn], h1[kHid];
#pragma unroll
  for (int i = 0; i < kIn; ++i) x[i] = X[(int64_t)b * kIn + i];
#pragma unroll
  for (int o = 0; o < kHid; ++o) {
    float s = w[ob1 + o];
#pragma unroll
    for (int i = 0; i < kIn; ++i) s = fmaf(w[oW1 + o * kIn + i], x[i], s);
    h1[o] = fmaxf(s, 0.f);
  }
  float y0 = w[ob3], y1 = w[ob3 + 1];
  for (int o = 0; o < kHid; ++o) {
    float s = w[ob2 + o];
#pragma unroll
    for (int i = 0; i < kHid; ++i) s = fmaf(w[oW2 + o * kHid + i], h1[i], s);
    const float h2 = fmaxf(s, 0.f);
    y0 = fmaf(w[oW3 + o], h2, y0);
    y1 = fmaf(w[oW3 + kHid + o], h2, y1);
    if (H) H[(int64_t)b * 2 * kHid + kHid + o] = h2;
  }
  if (H) {
#pragma unroll
    for (int o = 0; o < kHid; ++o) H[(int64_t)b * 2 * kHid + o] = h1[o];
  }
  Y[(int64_t)b * kOut] = y0;
  Y[(int64_t)b * kOut + 1] = y1;
}

// Per-sample deltas: dY = (y - t) / B; dH2 = W3^T dY * [h2 > 0];
// dH1 = W2^T dH2 * [h1 > 0].  D[b] = {dY[2], dH2[64], dH1[64]}.
__global__ void __launch_bounds__(128) mlp_delta_kernel(const float *__restrict__ prm,
                                                        const float *__restrict__ T, int B,
                                                        const float *__restrict__ Y,
                                                        const float *__restrict__ H,
                                                        float *__restrict__ D) {
  __shared__ float w[kParams];
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) w[i] = prm[i];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float *h = H + (int64_t)b * 2 * kHid;
  float *d = D + (int64_t)b * (kOut + 2 * kHid);
  const float dy0 = (Y[(int64_t)b * kOut] - T[(int64_t)b * kOut]) / (float)B;
  const float dy1 = (Y[(int64_t)b * kOut + 1] - T[(int64_t)b * kOut + 1]) / (float)B;
  d[0] = dy0;
  d[1] = dy1;
  float dh2[kHid];
#pragma unroll
  for (int o = 0; o < kHid; ++o) {
    const float g = w[oW3 + o] * dy0 + w[oW3 + kHid + o] * dy1;
    dh2[o] = h[kHid + o] > 0.f ? g : 0.f;
    d[kOut + o] = dh2[o];
  }
  for (int i = 0; i < kHid; ++i) {
    float s = 0.f;
#pragma unroll
    for (int o = 0; o < kHid; ++o) s = fmaf(w[oW2 + o * kHid + i], dh2[o], s);
    d[kOut + kHid + i] = h[i] > 0.f ? s : 0.f;
  }
}

// One thread per parameter (and one more for the loss): sums over the batch
// in sample order.
__global__ void mlp_grad_kernel(const float *__restrict__ X, const float *__restrict__ T, int B,
                                const float *__restrict__ Y, const float *__restrict__ H,
                                const float *__restrict__ D, float *__restrict__ grads,
                                float *__restrict__ loss) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int dstride = kOut + 2 * kHid;
  float s = 0.f;
  if (k < ob1) {  // W1[o][i]: sum_b dH1[b][o] * x[b][i]
    const int o = k / kIn, i = k % kIn;
    for (int b = 0; b < B; ++b) s = fmaf(D[(int64_t)b * dstride + kOut + kHid + o], X[(int64_t)b * kIn + i], s);
  } else if (k < oW2) {  // b1[o]
    const int o = k - ob1;
    for (int b = 0; b < B; ++b) s += D[(int64_t)b * dstride + kOut + kHid + o];
  } else if (k < ob2) {  // W2[o][i]: sum_b dH2[b][o] * h1[b][i]
    const int o = (k - oW2) / kHid, i = (k - oW2) % kHid;
    for (int b = 0; b < B; ++b) s = fmaf(D[(int64_t)b * dstride + kOut + o], H[(int64_t)b * 2 * kHid + i], s);
  } else if (k < oW3) {  // b2[o]
    const int o = k - ob2;
    for (int b = 0; b < B; ++b) s += D[(int64_t)b * dstride + kOut + o];
  } else if (k < ob3) {  // W3[o][i]: sum_b dY[b][o] * h2[b][i]
    const int o = (k - oW3) / kHid, i = (k - oW3) % kHid;
    for (int b = 0; b < B; ++b) s = fmaf(D[(int64_t)b * dstride + o], H[(int64_t)b * 2 * kHid + kHid + i], s);
  } else if (k < kParams) {  // b3[o]
    const int o = k - ob3;
    for (int b = 0; b < B; ++b) s += D[(int64_t)b * dstride + o];
  } else if (k == kParams) {  // the loss
    for (int b = 0; b < B; ++b)
      for (int o = 0; o < kOut; ++o) {
        const float e = Y[(int64_t)b * kOut + o] - T[(int64_t)b * kOut + o];
        s = fmaf(e, e, s);
      }
    if (loss) *loss = s / (2.f * (float)B);
    return;
  } else {
    return;
  }
  grads[k] = s;
}

__global__ void mlp_adam_kernel(float *__restrict__ prm, const float *__restrict__ g,
                                float *__restrict__ m, float *__restrict__ v, float lr, float b1,
                                float b2, float eps, float wd, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kParams) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float mh = mk / c1, vh = vk / c2;
  prm[k] -= lr * (mh / (sqrtf(vh) + eps) + wd * prm[k]);
}

extern "C" int polydet_mlp_forward(const float *params, const float *x, int batch, float *y,
                                   float *act_ws, void *stream) {
  if (!params || !x || !y || batch < 1) return POLYDET_EINVAL;
  const int th = 128;
  mlp_fwd_kernel<<<(batch + th - 1) / th, th, 0, (cudaStream_t)stream>>>(params, x, batch, y, act_ws);
  PD_CUDA(cudaGetLastError());
  return POLYDET_OK;
}

extern "C" int polydet_mlp_backward(const float *params, const float *x, const float *target,
                                    int batch, const float *y, const float *act_ws, float *delta_ws,
                                    float *grads, float *loss, void *stream) {
  if (!params || !x || !target || !y || !act_ws || !delta_ws || !grads || batch < 1)
    return POLYDET_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int th = 128;
  mlp_delta_kernel<<<(batch + th - 1) / th, th, 0, st>>>(params, target, batch, y, act_ws, delta_ws);
  PD_CUDA(cudaGetLastError());
  mlp_grad_kernel<<<(kParams + 1 + th - 1) / th, th, 0, st>>>(x, target, batch, y, act_ws, delta_ws,
                                                              grads, loss);
  PD_CUDA(cudaGetLastError());
  return POLYDET_OK;
}

extern "C" int polydet_mlp_adam(float *params, const float *grads, float *m, float *v, int step,
                                float lr, float beta1, float beta2, float eps, float weight_decay,
                                void *stream) {
  if (!params || !grads || !m || !v || step < 1) return POLYDET_EINVAL;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  const int th = 256;
  mlp_adam_kernel<<<(kParams + th - 1) / th, th, 0, (cudaStream_t)stream>>>(
      params, grads, m, v, lr, beta1, beta2, eps, weight_decay, c1, c2);
  PD_CUDA(cudaGetLastError());
  return POLYDET_OK;
}
