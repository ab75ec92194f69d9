// Training of the tile-proposal network on the GPU (psdf_trainer_*).
//
// Model: s = w2 . relu(W1 x) + b2, x in R^16 (input 15 is the constant 1, so
// W1's column 15 is the hidden bias), 64 hidden units.  Loss: mean squared
// error against the exact per-tile signed distances.  Per step:
//   1. train_forward   one thread per row: hidden activations, residual,
//                      ds = 2 (s - y) / N
//   2. train_partial   one thread per (parameter, chunk of rows): the chunk's
//                      gradient contribution, rows in a fixed order
//   3. train_reduce    one thread per parameter: sum of the chunks in order
//   4. train_adam      Adam update with bias correction
// No floating-point atomics are used, so a step is bit-for-bit reproducible
// (checkpoint/resume gives identical weights).
#include <cmath>
#include <cstring>
#include <vector>

#include "profile.h"
#include "psdf_internal.h"

namespace psdf {

constexpr int kIn = PSDF_MLP_IN;
constexpr int kHid = PSDF_MLP_HIDDEN;
constexpr int kParams = kHid * kIn + kHid + 1;  // W1 | w2 | b2
constexpr int kChunkRows = 1024;

}  // namespace psdf

struct psdf_trainer {
  float *d_param = nullptr;  // [kParams]
  float *d_m = nullptr, *d_v = nullptr;
  float *d_grad = nullptr;
  float *d_partial = nullptr;  // [chunks][kParams + 1] (+1: loss)
  float *d_hid = nullptr;      // [cap][kHid] relu activations
  float *d_ds = nullptr;       // [cap]
  float *d_res2 = nullptr;     // [cap] squared residuals
  float *d_loss = nullptr;     // [1]
  int64_t cap = 0;
  int64_t step = 0;
  float lr = 1e-3f;
};

namespace psdf {

__global__ void train_forward(const float *__restrict__ param, const float *__restrict__ X,
                              const float *__restrict__ y, const int *__restrict__ idx,
                              long long N, float *__restrict__ hid, float *__restrict__ ds,
                              float *__restrict__ res2)
{
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const long long row = idx ? idx[n] : n;
  float x[kIn];
#pragma unroll
  for (int k = 0; k < kIn; ++k) x[k] = X[row * kIn + k];
  const float *W1 = param, *w2 = param + kHid * kIn;
  float s = param[kHid * kIn + kHid];
  for (int h = 0; h < kHid; ++h) {
    float a = 0.f;
#pragma unroll
    for (int k = 0; k < kIn; ++k) a = fmaf(W1[h * kIn + k], x[k], a);
    a = fmaxf(a, 0.f);
    hid[n * kHid + h] = a;
    s = fmaf(w2[h], a, s);
  }
  const float r = s - y[row];
  ds[n] = 2.f * r / (float)N;
  res2[n] = r * r;
}

// blockIdx.y = chunk of kChunkRows rows; thread = parameter (plus one slot for
// the loss)
__global__ void train_partial(const float *__restrict__ param, const float *__restrict__ X,
                              const int *__restrict__ idx, long long N,
                              const float *__restrict__ hid, const float *__restrict__ ds,
                              const float *__restrict__ res2, float *__restrict__ partial)
{
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > kParams) return;
  const long long r0 = (long long)blockIdx.y * kChunkRows;
  const long long r1 = min(N, r0 + kChunkRows);
  const float *w2 = param + kHid * kIn;
  float acc = 0.f;
  if (j < kHid * kIn) {  // dW1[h][k] = sum ds * w2[h] * [a > 0] * x[k]
    const int h = j / kIn, k = j % kIn;
    const float wh = w2[h];
    for (long long n = r0; n < r1; ++n) {
      const long long row = idx ? idx[n] : n;
      const float a = hid[n * kHid + h];
      acc = fmaf(a > 0.f ? ds[n] * wh : 0.f, X[row * kIn + k], acc);
    }
  } else if (j < kHid * kIn + kHid) {  // dw2[h] = sum ds * relu(a)
    const int h = j - kHid * kIn;
    for (long long n = r0; n < r1; ++n) acc = fmaf(ds[n], hid[n * kHid + h], acc);
  } else if (j == kParams - 1) {  // db2
    for (long long n = r0; n < r1; ++n) acc += ds[n];
  } else {  // loss numerator
    for (long long n = r0; n < r1; ++n) acc += res2[n];
  }
  partial[(long long)blockIdx.y * (kParams + 1) + j] = acc;
}

__global__ void train_reduce(const float *__restrict__ partial, int chunks, long long N,
                             float *__restrict__ grad, float *__restrict__ loss)
{
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > kParams) return;
  float acc = 0.f;
  for (int c = 0; c < chunks; ++c) acc += partial[(long long)c * (kParams + 1) + j];
  if (j < kParams) grad[j] = acc;
  else if (loss) *loss = acc / (float)N;
}

__global__ void train_adam(float *__restrict__ param, float *__restrict__ m, float *__restrict__ v,
                           const float *__restrict__ grad, float lr, float c1, float c2)
{
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kParams) return;
  const float g = grad[j];
  const float mj = 0.9f * m[j] + 0.1f * g;
  const float vj = 0.999f * v[j] + 0.001f * g * g;
  m[j] = mj;
  v[j] = vj;
  param[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + 1e-8f);
}

static int ensure_capacity(psdf_trainer *t, long long N)
{
  if (N <= t->cap) return PSDF_OK;
  cudaFree(t->d_hid);
  cudaFree(t->d_ds);
  cudaFree(t->d_res2);
  cudaFree(t->d_partial);
  t->d_hid = t->d_ds = t->d_res2 = t->d_partial = nullptr;
  t->cap = 0;
  const long long chunks = (N + kChunkRows - 1) / kChunkRows;
  cudaError_t e = cudaMalloc(&t->d_hid, sizeof(float) * kHid * N);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_ds, sizeof(float) * N);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_res2, sizeof(float) * N);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_partial, sizeof(float) * (kParams + 1) * chunks);
  if (e != cudaSuccess) return cuda_fail(e, "trainer workspace");
  t->cap = N;
  return PSDF_OK;
}

static int grad_common(psdf_trainer *t, const float *X, const float *y, const int *idx,
                       long long N, float *grad, float *loss, cudaStream_t st)
{
  if (N < 1) return fail(PSDF_ERR_ARG, "N < 1");
  if (!X || !y || !grad) return fail(PSDF_ERR_ARG, "NULL argument");
  int rc = ensure_capacity(t, N);
  if (rc) return rc;
  const int chunks = (int)((N + kChunkRows - 1) / kChunkRows);
  train_forward<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(t->d_param, X, y, idx, N, t->d_hid,
                                                            t->d_ds, t->d_res2);
  dim3 g((kParams + 1 + 127) / 128, chunks);
  train_partial<<<g, 128, 0, st>>>(t->d_param, X, idx, N, t->d_hid, t->d_ds, t->d_res2,
                                   t->d_partial);
  train_reduce<<<(kParams + 1 + 127) / 128, 128, 0, st>>>(t->d_partial, chunks, N, grad, loss);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch");
}

}  // namespace psdf

using namespace psdf;

extern "C" int psdf_trainer_create(const float *W1, const float *w2, float b2, float lr,
                                   psdf_trainer **out)
{
  if (!W1 || !w2 || !out) return fail(PSDF_ERR_ARG, "NULL argument");
  if (!(lr > 0.f)) return fail(PSDF_ERR_ARG, "lr must be > 0");
  *out = nullptr;
  std::vector<float> p(kParams, 0.f);
  std::memcpy(p.data(), W1, sizeof(float) * kHid * kIn);
  std::memcpy(p.data() + kHid * kIn, w2, sizeof(float) * kHid);
  p[kParams - 1] = b2;
  psdf_trainer *t = new psdf_trainer();
  t->lr = lr;
  cudaError_t e = cudaMalloc(&t->d_param, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_m, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_v, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_grad, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(t->d_param, p.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(t->d_m, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(t->d_v, 0, sizeof(float) * kParams);
  if (e != cudaSuccess) {
    cudaFree(t->d_param); cudaFree(t->d_m); cudaFree(t->d_v); cudaFree(t->d_grad); cudaFree(t->d_loss);
    delete t;
    return cuda_fail(e, "psdf_trainer_create");
  }
  *out = t;
  return PSDF_OK;
}

extern "C" int psdf_trainer_destroy(psdf_trainer *t)
{
  if (!t) return PSDF_OK;
  cudaFree(t->d_param); cudaFree(t->d_m); cudaFree(t->d_v); cudaFree(t->d_grad);
  cudaFree(t->d_loss); cudaFree(t->d_hid); cudaFree(t->d_ds); cudaFree(t->d_res2);
  cudaFree(t->d_partial);
  delete t;
  return PSDF_OK;
}

extern "C" int psdf_trainer_grad(psdf_trainer *t, const float *X, const float *y, int64_t N,
                                 float *grad, float *loss, void *stream)
{
  if (!t) return fail(PSDF_ERR_ARG, "trainer is NULL");
  return grad_common(t, X, y, nullptr, N, grad, loss, (cudaStream_t)stream);
}

extern "C" int psdf_trainer_step(psdf_trainer *t, const float *X, const float *y,
                                 const int32_t *idx, int64_t N, float *loss, void *stream)
{
  if (!t) return fail(PSDF_ERR_ARG, "trainer is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  ProfileScope prof("train_step", st);
  int rc = grad_common(t, X, y, idx, N, t->d_grad, loss ? loss : t->d_loss, st);
  if (rc) return rc;
  t->step += 1;
  const float c1 = 1.f - (float)std::pow(0.9, (double)t->step);
  const float c2 = 1.f - (float)std::pow(0.999, (double)t->step);
  train_adam<<<(kParams + 127) / 128, 128, 0, st>>>(t->d_param, t->d_m, t->d_v, t->d_grad,
                                                   t->lr, c1, c2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "kernel launch");
}

extern "C" int psdf_trainer_set_lr(psdf_trainer *t, float lr)
{
  if (!t || !(lr > 0.f)) return fail(PSDF_ERR_ARG, "bad trainer or lr");
  t->lr = lr;
  return PSDF_OK;
}

extern "C" int psdf_trainer_get(const psdf_trainer *t, float *params, float *m, float *v,
                                int64_t *step)
{
  if (!t) return fail(PSDF_ERR_ARG, "trainer is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && params) e = cudaMemcpy(params, t->d_param, sizeof(float) * kParams, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && m) e = cudaMemcpy(m, t->d_m, sizeof(float) * kParams, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v) e = cudaMemcpy(v, t->d_v, sizeof(float) * kParams, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "psdf_trainer_get");
  if (step) *step = t->step;
  return PSDF_OK;
}

extern "C" int psdf_trainer_set(psdf_trainer *t, const float *params, const float *m,
                                const float *v, int64_t step)
{
  if (!t || !params || !m || !v || step < 0) return fail(PSDF_ERR_ARG, "bad argument");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(t->d_param, params, sizeof(float) * kParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t->d_m, m, sizeof(float) * kParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t->d_v, v, sizeof(float) * kParams, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "psdf_trainer_set");
  t->step = step;
  return PSDF_OK;
}
