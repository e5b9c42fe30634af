// K8: the learned cost model -- a 3-layer perceptron F -> H -> H -> 1 (FP32,
// ReLU) trained on the engine's own per-launch timings to predict log time,
// with hand-written forward, backward and Adam kernels.
//
// Parameters are one packed FP32 vector: W1 [H][F], b1 [H], W2 [H][H], b2 [H],
// W3 [H], b3.  The loss is the mean squared error over the N rows.
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "tdq_internal.h"

namespace tdq {

namespace {

constexpr int kRows = 32;  // rows per CTA tile
constexpr int kMaxF = 32, kMaxH = 64;

struct MlpDims {
  int F, H;
  int oW1, ob1, oW2, ob2, oW3, ob3, total;
};

MlpDims dims_of(int F, int H) {
  MlpDims d;
  d.F = F;
  d.H = H;
  d.oW1 = 0;
  d.ob1 = d.oW1 + H * F;
  d.oW2 = d.ob1 + H;
  d.ob2 = d.oW2 + H * H;
  d.oW3 = d.ob2 + H;
  d.ob3 = d.oW3 + H;
  d.total = d.ob3 + 1;
  return d;
}

// Forward (and with GRAD the loss gradient) of one tile of kRows rows; one
// thread per hidden unit (blockDim.x == H).
template <bool GRAD>
__global__ void k_mlp(const float* __restrict__ X, const float* __restrict__ t, int N, MlpDims d,
                      const float* __restrict__ p, float* y, float* g, float* loss) {
  extern __shared__ float sm[];
  const int F = d.F, H = d.H;
  float* W = sm;                              // all parameters
  float* xs = W + d.total;                    // [kRows][F]
  float* h1 = xs + kRows * F;                 // [kRows][H]
  float* h2 = h1 + kRows * H;                 // [kRows][H]
  float* dz = h2 + kRows * H;                 // [kRows][H] (backward)
  float* dy = dz + kRows * H;                 // [kRows]
  const int j = threadIdx.x;
  const int r0 = blockIdx.x * kRows;
  const int nr = min(kRows, N - r0);
  for (int i = j; i < d.total; i += blockDim.x) W[i] = p[i];
  for (int i = j; i < kRows * F; i += blockDim.x) xs[i] = (i / F) < nr ? X[(size_t)r0 * F + i] : 0.f;
  __syncthreads();
  for (int r = 0; r < nr; r++) {
    float z = W[d.ob1 + j];
    for (int f = 0; f < F; f++) z = fmaf(W[d.oW1 + j * F + f], xs[r * F + f], z);
    h1[r * H + j] = fmaxf(z, 0.f);
  }
  __syncthreads();
  for (int r = 0; r < nr; r++) {
    float z = W[d.ob2 + j];
    for (int i = 0; i < H; i++) z = fmaf(W[d.oW2 + j * H + i], h1[r * H + i], z);
    h2[r * H + j] = fmaxf(z, 0.f);
  }
  __syncthreads();
  if (j < nr) {
    float o = W[d.ob3];
    for (int i = 0; i < H; i++) o = fmaf(W[d.oW3 + i], h2[j * H + i], o);
    if (!GRAD) y[r0 + j] = o;
    else {
      const float e = o - t[r0 + j];
      dy[j] = 2.f * e / (float)N;
      atomicAdd(loss, e * e / (float)N);
    }
  }
  if (!GRAD) return;
  __syncthreads();
  // layer 3: dW3[j] = sum_r dy h2[r][j]; dz2 = dy W3 relu'(z2)
  float gw3 = 0.f, gb2 = 0.f;
  for (int r = 0; r < nr; r++) {
    gw3 = fmaf(dy[r], h2[r * H + j], gw3);
    const float v = h2[r * H + j] > 0.f ? dy[r] * W[d.oW3 + j] : 0.f;
    dz[r * H + j] = v;
    gb2 += v;
  }
  atomicAdd(&g[d.oW3 + j], gw3);
  atomicAdd(&g[d.ob2 + j], gb2);
  if (j == 0) {
    float s = 0.f;
    for (int r = 0; r < nr; r++) s += dy[r];
    atomicAdd(&g[d.ob3], s);
  }
  __syncthreads();
  // layer 2: dW2[j][i] = sum_r dz2[r][j] h1[r][i]
  for (int i = 0; i < H; i++) {
    float s = 0.f;
    for (int r = 0; r < nr; r++) s = fmaf(dz[r * H + j], h1[r * H + i], s);
    atomicAdd(&g[d.oW2 + j * H + i], s);
  }
  // dz1[r][j] = (sum_i W2[i][j] dz2[r][i]) relu'(z1[r][j]) -> kept in registers per r
  float d1[kRows];
  for (int r = 0; r < kRows; r++) {
    float s = 0.f;
    if (r < nr)
      for (int i = 0; i < H; i++) s = fmaf(W[d.oW2 + i * H + j], dz[r * H + i], s);
    d1[r] = (r < nr && h1[r * H + j] > 0.f) ? s : 0.f;
  }
  // layer 1: dW1[j][f] = sum_r dz1[r][j] x[r][f], db1[j] = sum_r dz1[r][j]
  float gb1 = 0.f;
  for (int r = 0; r < nr; r++) gb1 += d1[r];
  atomicAdd(&g[d.ob1 + j], gb1);
  for (int f = 0; f < F; f++) {
    float s = 0.f;
    for (int r = 0; r < nr; r++) s = fmaf(d1[r], xs[r * F + f], s);
    atomicAdd(&g[d.oW1 + j * F + f], s);
  }
}

// Adam (Kingma and Ba): moments m, v; step count tstep >= 1.
__global__ void k_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                       int tstep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(b1, (float)tstep));
  const float vh = vi / (1.f - powf(b2, (float)tstep));
  p[i] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace

}  // namespace tdq

using namespace tdq;

struct tdq_costmodel {
  int dev = 0;
  MlpDims d{};
  float* p = nullptr;  // parameters
  float* g = nullptr;  // gradient of the last loss_grad
  float* m = nullptr;  // Adam moments
  float* v = nullptr;
  float* loss = nullptr;
  int steps = 0;
  ~tdq_costmodel() {
    cudaFree(p);
    cudaFree(g);
    cudaFree(m);
    cudaFree(v);
    cudaFree(loss);
  }
  size_t smem() const {
    return sizeof(float) * ((size_t)d.total + (size_t)kRows * d.F + 3 * (size_t)kRows * d.H + kRows);
  }
};

extern "C" {

tdq_status tdq_costmodel_create(int n_features, int hidden, uint64_t seed, int device, tdq_costmodel** out) {
  if (!out || n_features < 1 || n_features > kMaxF || hidden < 32 || hidden > kMaxH || hidden % 32)
    return fail(TDQ_ERR_ARG, "tdq_costmodel_create: need 1 <= features <= 32, hidden in {32, 64}");
  *out = nullptr;
  tdq_costmodel* c = new (std::nothrow) tdq_costmodel();
  if (!c) return fail(TDQ_ERR_OOM, "tdq_costmodel_create: host allocation");
  c->dev = device;
  c->d = dims_of(n_features, hidden);
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return fail(TDQ_ERR_CUDA, "tdq_costmodel_create: cudaSetDevice");
  }
  const size_t bytes = sizeof(float) * c->d.total;
  if (cudaMalloc(&c->p, bytes) != cudaSuccess || cudaMalloc(&c->g, bytes) != cudaSuccess ||
      cudaMalloc(&c->m, bytes) != cudaSuccess || cudaMalloc(&c->v, bytes) != cudaSuccess ||
      cudaMalloc(&c->loss, sizeof(float)) != cudaSuccess) {
    delete c;
    return fail(TDQ_ERR_OOM, "tdq_costmodel_create: device memory");
  }
  // He-uniform weights from a splitmix64 stream, zero biases
  std::vector<float> h(c->d.total, 0.f);
  uint64_t s = seed;
  auto uni = [&]() {
    s += 0x9e3779b97f4a7c15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  };
  const MlpDims& d = c->d;
  for (int i = 0; i < d.H * d.F; i++) h[d.oW1 + i] = (float)(uni() * std::sqrt(6.0 / d.F));
  for (int i = 0; i < d.H * d.H; i++) h[d.oW2 + i] = (float)(uni() * std::sqrt(6.0 / d.H));
  for (int i = 0; i < d.H; i++) h[d.oW3 + i] = (float)(uni() * std::sqrt(6.0 / d.H));
  cudaMemcpy(c->p, h.data(), bytes, cudaMemcpyHostToDevice);
  cudaMemset(c->m, 0, bytes);
  cudaMemset(c->v, 0, bytes);
  cudaMemset(c->g, 0, bytes);
  if (cudaFuncSetAttribute(k_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem()) != cudaSuccess ||
      cudaFuncSetAttribute(k_mlp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem()) != cudaSuccess) {
    delete c;
    return fail(TDQ_ERR_CUDA, "tdq_costmodel_create: shared memory attribute");
  }
  *out = c;
  return ok();
}

tdq_status tdq_costmodel_params(tdq_costmodel* c, float* host, int* n_params, int set) {
  if (!c) return fail(TDQ_ERR_ARG, "tdq_costmodel_params: NULL model");
  if (n_params) *n_params = c->d.total;
  if (!host) return ok();
  TDQ_CUDA_TRY(cudaSetDevice(c->dev));
  const size_t bytes = sizeof(float) * c->d.total;
  if (set) {
    TDQ_CUDA_TRY(cudaMemcpy(c->p, host, bytes, cudaMemcpyHostToDevice));
    TDQ_CUDA_TRY(cudaMemset(c->m, 0, bytes));
    TDQ_CUDA_TRY(cudaMemset(c->v, 0, bytes));
    c->steps = 0;
  } else {
    TDQ_CUDA_TRY(cudaMemcpy(host, c->p, bytes, cudaMemcpyDeviceToHost));
  }
  return ok();
}

tdq_status tdq_costmodel_loss_grad(tdq_costmodel* c, const float* d_X, const float* d_t, int N, float* d_loss,
                                   float* d_grads, void* stream) {
  if (!c || !d_X || !d_t || N < 1) return fail(TDQ_ERR_ARG, "tdq_costmodel_loss_grad: bad argument");
  TDQ_CUDA_TRY(cudaSetDevice(c->dev));
  cudaStream_t st = (cudaStream_t)stream;
  TDQ_CUDA_TRY(cudaMemsetAsync(c->g, 0, sizeof(float) * c->d.total, st));
  TDQ_CUDA_TRY(cudaMemsetAsync(c->loss, 0, sizeof(float), st));
  k_mlp<true><<<(N + kRows - 1) / kRows, c->d.H, c->smem(), st>>>(d_X, d_t, N, c->d, c->p, nullptr, c->g, c->loss);
  TDQ_CUDA_TRY(cudaGetLastError());
  if (d_loss) TDQ_CUDA_TRY(cudaMemcpyAsync(d_loss, c->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (d_grads)
    TDQ_CUDA_TRY(cudaMemcpyAsync(d_grads, c->g, sizeof(float) * c->d.total, cudaMemcpyDeviceToDevice, st));
  return ok();
}

tdq_status tdq_costmodel_adam_step(tdq_costmodel* c, float lr, void* stream) {
  if (!c || !(lr > 0.f)) return fail(TDQ_ERR_ARG, "tdq_costmodel_adam_step: bad argument");
  TDQ_CUDA_TRY(cudaSetDevice(c->dev));
  c->steps++;
  k_adam<<<(c->d.total + 255) / 256, 256, 0, (cudaStream_t)stream>>>(c->p, c->g, c->m, c->v, c->d.total, lr, 0.9f,
                                                                     0.999f, 1e-8f, c->steps);
  TDQ_CUDA_TRY(cudaGetLastError());
  return ok();
}

tdq_status tdq_costmodel_train(tdq_costmodel* c, const float* d_X, const float* d_t, int N, int epochs, float lr,
                               float* d_losses, void* stream) {
  if (!c || epochs < 1) return fail(TDQ_ERR_ARG, "tdq_costmodel_train: bad argument");
  for (int e = 0; e < epochs; e++) {
    tdq_status s = tdq_costmodel_loss_grad(c, d_X, d_t, N, d_losses ? d_losses + e : nullptr, nullptr, stream);
    if (s != TDQ_OK) return s;
    s = tdq_costmodel_adam_step(c, lr, stream);
    if (s != TDQ_OK) return s;
  }
  return ok();
}

tdq_status tdq_costmodel_predict(tdq_costmodel* c, const float* d_X, int N, float* d_y, void* stream) {
  if (!c || !d_X || !d_y || N < 1) return fail(TDQ_ERR_ARG, "tdq_costmodel_predict: bad argument");
  TDQ_CUDA_TRY(cudaSetDevice(c->dev));
  k_mlp<false><<<(N + kRows - 1) / kRows, c->d.H, c->smem(), (cudaStream_t)stream>>>(d_X, nullptr, N, c->d, c->p,
                                                                                     d_y, nullptr, nullptr);
  TDQ_CUDA_TRY(cudaGetLastError());
  return ok();
}

tdq_status tdq_costmodel_destroy(tdq_costmodel* c) {
  delete c;
  return ok();
}

}  // extern "C"
