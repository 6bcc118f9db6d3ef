// The launch-shape cost model's network on the GPU: forward, loss and
// gradient by back-propagation, and Adam (not in the paper; it serves the
// launch-shape selection the library adds).
//
// A 2-layer MLP with parameters packed in one FP32 array: W1 (d x h,
// row-major, W1[i * h + j] maps input i to hidden unit j), b1 (h), W2
// (h x h), b2 (h), w3 (h), b3 (1).  Forward: h1 = relu(x W1 + b1),
// h2 = relu(h1 W2 + b2), y = h2 . w3 + b3; loss = mean (y - t)^2.  Every
// sum runs in a fixed order (no atomics), so a training run is
// reproducible bit for bit; the long sums over the batch use TwoSum
// compensation.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "coot_internal.h"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void two_sum(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

// out[b, j] = relu(sum_i in[b, i] W[i, j] + bias[j]),  b < B, j < H, i < K
__global__ void layer_kernel(const float* __restrict__ in, const float* __restrict__ W, const float* __restrict__ bias,
                             float* __restrict__ out, int B, int K, int H) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * H) return;
  const int b = (int)(t / H), j = (int)(t - (int64_t)b * H);
  float s = bias[j];
  const float* row = in + (int64_t)b * K;
  for (int i = 0; i < K; ++i) s = fmaf(row[i], W[(int64_t)i * H + j], s);
  out[t] = s > 0.f ? s : 0.f;
}

// y[b] = sum_j h2[b, j] w3[j] + b3
__global__ void out_kernel(const float* __restrict__ h2, const float* __restrict__ w3, const float* __restrict__ b3,
                           float* __restrict__ y, int B, int H) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float s = b3[0];
  const float* row = h2 + (int64_t)b * H;
  for (int j = 0; j < H; ++j) s = fmaf(row[j], w3[j], s);
  y[b] = s;
}

// dy[b] = 2 (y[b] - t[b]) / B, and the loss mean (y - t)^2 by one block in a
// fixed order
__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
                            float* __restrict__ loss, int B) {
  __shared__ double red[kThreads];
  double acc = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float e = y[b] - t[b];
    dy[b] = 2.f * e / (float)B;
    acc += (double)e * (double)e;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = (float)(red[0] / (double)B);
}

// dh2[b, j] = dy[b] w3[j] [h2[b, j] > 0]
__global__ void dh2_kernel(const float* __restrict__ dy, const float* __restrict__ w3, const float* __restrict__ h2,
                           float* __restrict__ dh2, int B, int H) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * H) return;
  const int b = (int)(t / H), j = (int)(t - (int64_t)b * H);
  dh2[t] = h2[t] > 0.f ? dy[b] * w3[j] : 0.f;
}

// dh1[b, i] = (sum_j dh2[b, j] W2[i, j]) [h1[b, i] > 0]
__global__ void dh1_kernel(const float* __restrict__ dh2, const float* __restrict__ W2, const float* __restrict__ h1,
                           float* __restrict__ dh1, int B, int H) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * H) return;
  const int b = (int)(t / H), i = (int)(t - (int64_t)b * H);
  if (!(h1[t] > 0.f)) {
    dh1[t] = 0.f;
    return;
  }
  float s = 0.f;
  const float* row = dh2 + (int64_t)b * H;
  for (int j = 0; j < H; ++j) s = fmaf(row[j], W2[(int64_t)i * H + j], s);
  dh1[t] = s;
}

// g[i * N + j] = sum_b A[b, i] D[b, j]  (A == nullptr: A = 1, a bias
// gradient), b in increasing order with TwoSum
__global__ void wgrad_kernel(const float* __restrict__ A, const float* __restrict__ D, float* __restrict__ g, int B,
                             int K, int N) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)K * N) return;
  const int i = (int)(t / N), j = (int)(t - (int64_t)i * N);
  float s = 0.f, c = 0.f;
  for (int b = 0; b < B; ++b) {
    const float a = A ? A[(int64_t)b * K + i] : 1.f;
    two_sum(s, c, __fmul_rn(a, D[(int64_t)b * N + j]));
  }
  g[t] = s + c;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

unsigned blocks(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

coot_status check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return coot::fail(COOT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return COOT_OK;
}

coot_status check_dims(int d, int h, int batch) {
  if (d < 1 || d > 4096 || h < 1 || h > 4096 || batch < 1 || batch > (1 << 24))
    return coot::fail(COOT_ERR_INVALID_ARG, "MLP sizes out of range");
  return COOT_OK;
}

}  // namespace

extern "C" {

coot_status coot_mlp_forward(const float* params, int d, int h, const float* x, int batch, float* y, float* act,
                             void* stream) {
  coot::clear_error();
  coot_status s = check_dims(d, h, batch);
  if (s != COOT_OK) return s;
  if (!params || !x || !y || !act) return coot::fail(COOT_ERR_INVALID_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const float* W1 = params;
  const float* b1 = W1 + (int64_t)d * h;
  const float* W2 = b1 + h;
  const float* b2 = W2 + (int64_t)h * h;
  const float* w3 = b2 + h;
  const float* b3 = w3 + h;
  float* h1 = act;
  float* h2 = act + (int64_t)batch * h;
  layer_kernel<<<blocks((int64_t)batch * h), kThreads, 0, st>>>(x, W1, b1, h1, batch, d, h);
  layer_kernel<<<blocks((int64_t)batch * h), kThreads, 0, st>>>(h1, W2, b2, h2, batch, h, h);
  out_kernel<<<blocks(batch), kThreads, 0, st>>>(h2, w3, b3, y, batch, h);
  return check_launch("MLP forward");
}

coot_status coot_mlp_loss_grad(const float* params, int d, int h, const float* x, const float* t, int batch,
                               const float* y, const float* act, float* grad, float* loss, float* work,
                               void* stream) {
  coot::clear_error();
  coot_status s = check_dims(d, h, batch);
  if (s != COOT_OK) return s;
  if (!params || !x || !t || !y || !act || !grad || !loss || !work)
    return coot::fail(COOT_ERR_INVALID_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const float* W2 = params + (int64_t)d * h + h;
  const float* w3 = W2 + (int64_t)h * h + h;
  const float* h1 = act;
  const float* h2 = act + (int64_t)batch * h;
  float* dy = work;
  float* dh2 = work + batch;
  float* dh1 = dh2 + (int64_t)batch * h;
  float* gW1 = grad;
  float* gb1 = gW1 + (int64_t)d * h;
  float* gW2 = gb1 + h;
  float* gb2 = gW2 + (int64_t)h * h;
  float* gw3 = gb2 + h;
  float* gb3 = gw3 + h;
  loss_kernel<<<1, kThreads, 0, st>>>(y, t, dy, loss, batch);
  dh2_kernel<<<blocks((int64_t)batch * h), kThreads, 0, st>>>(dy, w3, h2, dh2, batch, h);
  dh1_kernel<<<blocks((int64_t)batch * h), kThreads, 0, st>>>(dh2, W2, h1, dh1, batch, h);
  wgrad_kernel<<<blocks(h), kThreads, 0, st>>>(h2, dy, gw3, batch, h, 1);
  wgrad_kernel<<<1, kThreads, 0, st>>>(nullptr, dy, gb3, batch, 1, 1);
  wgrad_kernel<<<blocks((int64_t)h * h), kThreads, 0, st>>>(h1, dh2, gW2, batch, h, h);
  wgrad_kernel<<<blocks(h), kThreads, 0, st>>>(nullptr, dh2, gb2, batch, 1, h);
  wgrad_kernel<<<blocks((int64_t)d * h), kThreads, 0, st>>>(x, dh1, gW1, batch, d, h);
  wgrad_kernel<<<blocks(h), kThreads, 0, st>>>(nullptr, dh1, gb1, batch, 1, h);
  return check_launch("MLP gradient");
}

coot_status coot_mlp_adam(float* params, const float* grad, float* m, float* v, int n, int step, float lr,
                          float beta1, float beta2, float eps, void* stream) {
  coot::clear_error();
  if (!params || !grad || !m || !v || n < 1 || step < 1) return coot::fail(COOT_ERR_INVALID_ARG, "bad Adam arguments");
  const float c1 = 1.f - (float)std::pow((double)beta1, (double)step);
  const float c2 = 1.f - (float)std::pow((double)beta2, (double)step);
  adam_kernel<<<blocks(n), kThreads, 0, (cudaStream_t)stream>>>(params, grad, m, v, n, lr, beta1, beta2, eps, c1, c2);
  return check_launch("Adam");
}

}  // extern "C"
