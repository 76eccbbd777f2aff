// Learned Krylov control: a 16 -> 64 -> 64 -> 2 multilayer perceptron (GELU
// hidden activations) with BF16 weights and FP32 accumulation, trained on the
// GPU by the hand-written forward/backward kernels below (mean squared error,
// Adam on FP32 master weights, BF16 copies refreshed after every update).
//
// Parameter layout (floats): W1[64][16], b1[64], W2[64][64], b2[64], W3[2][64],
// b3[2].  Normalisation (floats): input mean[16], input std[16], output
// mean[2], output std[2]; the network works on standardised values.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "swepi_internal.h"

namespace swepi {

namespace {

constexpr int NI = 16, NH = 64, NO = 2;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH, NPARAM = OFF_B3 + NO;
constexpr int NNORM = 2 * NI + 2 * NO;
constexpr int TRAIN_CTAS = 64;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  // d/dx [x Phi(x)] = Phi(x) + x phi(x)
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

struct Acts {
  float x[NI], z1[NH], h1[NH], z2[NH], h2[NH], y[NO];
};

// forward pass of one standardised sample by a block of NH threads
__device__ void forward_one(const __nv_bfloat16* __restrict__ w, Acts& a) {
  const int t = threadIdx.x;
  if (t < NH) {
    float s = __bfloat162float(w[OFF_B1 + t]);
    for (int i = 0; i < NI; ++i) s = fmaf(__bfloat162float(w[OFF_W1 + t * NI + i]), a.x[i], s);
    a.z1[t] = s;
    a.h1[t] = gelu(s);
  }
  __syncthreads();
  if (t < NH) {
    float s = __bfloat162float(w[OFF_B2 + t]);
    for (int k = 0; k < NH; ++k) s = fmaf(__bfloat162float(w[OFF_W2 + t * NH + k]), a.h1[k], s);
    a.z2[t] = s;
    a.h2[t] = gelu(s);
  }
  __syncthreads();
  if (t < NO) {
    float s = __bfloat162float(w[OFF_B3 + t]);
    for (int j = 0; j < NH; ++j) s = fmaf(__bfloat162float(w[OFF_W3 + t * NH + j]), a.h2[j], s);
    a.y[t] = s;
  }
  __syncthreads();
}

// inference: one block per sample, raw features in, raw outputs out
__global__ void __launch_bounds__(NH) mlp_forward_kernel(const __nv_bfloat16* __restrict__ w,
                                                         const float* __restrict__ norm, const float* __restrict__ X,
                                                         int n, float* __restrict__ Y) {
  __shared__ Acts a;
  const int s = blockIdx.x;
  if (s >= n) return;
  if (threadIdx.x < NI) a.x[threadIdx.x] = (X[s * NI + threadIdx.x] - norm[threadIdx.x]) / norm[NI + threadIdx.x];
  __syncthreads();
  forward_one(w, a);
  if (threadIdx.x < NO) Y[s * NO + threadIdx.x] = a.y[threadIdx.x] * norm[2 * NI + NO + threadIdx.x] + norm[2 * NI + threadIdx.x];
}

// gradient of the mean squared error over all samples, on standardised
// targets; block g accumulates samples g, g + G, ... into its own partial sums
// (each gradient entry owned by one thread: deterministic)
__global__ void __launch_bounds__(NH) mlp_grad_kernel(const __nv_bfloat16* __restrict__ w,
                                                      const float* __restrict__ norm, const float* __restrict__ X,
                                                      const float* __restrict__ T, int n, float* __restrict__ part,
                                                      float* __restrict__ loss_part) {
  __shared__ Acts a;
  __shared__ float g[NPARAM];
  __shared__ float dz2[NH], dy[NO];
  const int t = threadIdx.x;
  for (int p = t; p < NPARAM; p += blockDim.x) g[p] = 0.0f;
  float loss = 0.0f;
  const float inv = 1.0f / (float)(n * NO);
  __syncthreads();
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    if (t < NI) a.x[t] = (X[s * NI + t] - norm[t]) / norm[NI + t];
    __syncthreads();
    forward_one(w, a);
    if (t < NO) {
      const float target = (T[s * NO + t] - norm[2 * NI + t]) / norm[2 * NI + NO + t];
      const float r = a.y[t] - target;
      dy[t] = 2.0f * r * inv;
      loss += r * r * inv;
    }
    __syncthreads();
    if (t < NH) {
      float dh2 = 0.0f;
      for (int o = 0; o < NO; ++o) {
        g[OFF_W3 + o * NH + t] += dy[o] * a.h2[t];
        dh2 = fmaf(__bfloat162float(w[OFF_W3 + o * NH + t]), dy[o], dh2);
      }
      if (t < NO) g[OFF_B3 + t] += dy[t];
      const float d2 = dh2 * gelu_grad(a.z2[t]);
      dz2[t] = d2;
      g[OFF_B2 + t] += d2;
      for (int k = 0; k < NH; ++k) g[OFF_W2 + t * NH + k] += d2 * a.h1[k];
    }
    __syncthreads();
    if (t < NH) {
      float dh1 = 0.0f;
      for (int j = 0; j < NH; ++j) dh1 = fmaf(__bfloat162float(w[OFF_W2 + j * NH + t]), dz2[j], dh1);
      const float d1 = dh1 * gelu_grad(a.z1[t]);
      g[OFF_B1 + t] += d1;
      for (int i = 0; i < NI; ++i) g[OFF_W1 + t * NI + i] += d1 * a.x[i];
    }
    __syncthreads();
  }
  for (int p = t; p < NPARAM; p += blockDim.x) part[(long long)blockIdx.x * NPARAM + p] = g[p];
  __shared__ float ls[NO];
  if (t < NO) ls[t] = loss;
  __syncthreads();
  if (t == 0) loss_part[blockIdx.x] = ls[0] + ls[1];
}

// deterministic reduction of the partial gradients, then an Adam step on the
// FP32 master weights and the BF16 refresh (adam == 0: reduce only)
__global__ void mlp_update_kernel(const float* __restrict__ part, int nparts, float* __restrict__ grad,
                                  float* __restrict__ master, float* __restrict__ m1, float* __restrict__ m2,
                                  __nv_bfloat16* __restrict__ w, int adam, float lr, float b1c, float b2c,
                                  const float* __restrict__ loss_part, float* __restrict__ loss_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss_out) {
    float l = 0.0f;
    for (int c = 0; c < nparts; ++c) l += loss_part[c];
    *loss_out = l;
  }
  if (p >= NPARAM) return;
  float gsum = 0.0f;
  for (int c = 0; c < nparts; ++c) gsum += part[(long long)c * NPARAM + p];
  grad[p] = gsum;
  if (!adam) return;
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  const float a = beta1 * m1[p] + (1.0f - beta1) * gsum;
  const float b = beta2 * m2[p] + (1.0f - beta2) * gsum * gsum;
  m1[p] = a;
  m2[p] = b;
  const float mh = a / b1c, vh = b / b2c;
  const float nw = master[p] - lr * mh / (sqrtf(vh) + eps);
  master[p] = nw;
  w[p] = __float2bfloat16(nw);
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16(src[i]);
}

}  // namespace

struct Mlp {
  float* master = nullptr;
  __nv_bfloat16* w = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  float* norm = nullptr;
  float* part = nullptr;
  float* grad = nullptr;
  float* loss_part = nullptr;
  float* loss = nullptr;
  float* io = nullptr;      // inference scratch: 16 inputs + 2 outputs
  float* h_io = nullptr;    // pinned
  int adam_t = 0;
};

int mlp_nparam() { return NPARAM; }
int mlp_nnorm() { return NNORM; }

int mlp_create(Mlp** out) {
  Mlp* m = new (std::nothrow) Mlp();
  if (!m) return SW_ENOMEM;
  bool ok = cudaMalloc(&m->master, sizeof(float) * NPARAM) == cudaSuccess &&
            cudaMalloc(&m->w, sizeof(__nv_bfloat16) * NPARAM) == cudaSuccess &&
            cudaMalloc(&m->m1, sizeof(float) * NPARAM) == cudaSuccess &&
            cudaMalloc(&m->m2, sizeof(float) * NPARAM) == cudaSuccess &&
            cudaMalloc(&m->norm, sizeof(float) * NNORM) == cudaSuccess &&
            cudaMalloc(&m->part, sizeof(float) * NPARAM * TRAIN_CTAS) == cudaSuccess &&
            cudaMalloc(&m->grad, sizeof(float) * NPARAM) == cudaSuccess &&
            cudaMalloc(&m->loss_part, sizeof(float) * TRAIN_CTAS) == cudaSuccess &&
            cudaMalloc(&m->loss, sizeof(float)) == cudaSuccess &&
            cudaMalloc(&m->io, sizeof(float) * 32) == cudaSuccess &&
            cudaMallocHost(&m->h_io, sizeof(float) * 32) == cudaSuccess;
  if (!ok) {
    mlp_destroy(m);
    return SW_ENOMEM;
  }
  *out = m;
  return SW_OK;
}

void mlp_destroy(Mlp* m) {
  if (!m) return;
  float* fs[] = {m->master, m->m1, m->m2, m->norm, m->part, m->grad, m->loss_part, m->loss, m->io};
  for (float* p : fs)
    if (p) cudaFree(p);
  if (m->w) cudaFree(m->w);
  if (m->h_io) cudaFreeHost(m->h_io);
  delete m;
}

int mlp_set(Mlp* m, const float* params, const float* norm) {
  if (params) {
    if (cudaMemcpy(m->master, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess)
      return SW_ECUDA;
    to_bf16_kernel<<<(NPARAM + 255) / 256, 256>>>(m->master, m->w, NPARAM);
    if (cudaMemset(m->m1, 0, sizeof(float) * NPARAM) != cudaSuccess ||
        cudaMemset(m->m2, 0, sizeof(float) * NPARAM) != cudaSuccess)
      return SW_ECUDA;
    m->adam_t = 0;
  }
  if (norm && cudaMemcpy(m->norm, norm, sizeof(float) * NNORM, cudaMemcpyHostToDevice) != cudaSuccess)
    return SW_ECUDA;
  return cuda_status(cudaDeviceSynchronize());
}

int mlp_get(Mlp* m, float* params, float* bf16_as_float) {
  if (params && cudaMemcpy(params, m->master, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess)
    return SW_ECUDA;
  if (bf16_as_float) {
    std::vector<__nv_bfloat16> tmp(NPARAM);
    if (cudaMemcpy(tmp.data(), m->w, sizeof(__nv_bfloat16) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess)
      return SW_ECUDA;
    for (int i = 0; i < NPARAM; ++i) bf16_as_float[i] = __bfloat162float(tmp[i]);
  }
  return SW_OK;
}

int mlp_forward(Mlp* m, const float* X, int n, float* Y, cudaStream_t s) {
  mlp_forward_kernel<<<n, NH, 0, s>>>(m->w, m->norm, X, n, Y);
  return cuda_status(cudaGetLastError());
}

int mlp_step(Mlp* m, const float* X, const float* T, int n, bool adam, float lr, float* loss_host, cudaStream_t s) {
  mlp_grad_kernel<<<TRAIN_CTAS, NH, 0, s>>>(m->w, m->norm, X, T, n, m->part, m->loss_part);
  float b1c = 1.0f, b2c = 1.0f;
  if (adam) {
    m->adam_t++;
    b1c = 1.0f - powf(0.9f, (float)m->adam_t);
    b2c = 1.0f - powf(0.999f, (float)m->adam_t);
  }
  mlp_update_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(m->part, TRAIN_CTAS, m->grad, m->master, m->m1, m->m2, m->w,
                                                         adam ? 1 : 0, lr, b1c, b2c, m->loss_part, m->loss);
  if (loss_host && cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return SW_ECUDA;
  return cuda_status(cudaGetLastError());
}

int mlp_grad_host(Mlp* m, float* grad_host) {
  return cuda_status(cudaMemcpy(grad_host, m->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
}

// one prediction from host features (synchronises the stream)
int mlp_predict_host(Mlp* m, const float* feat, float* out2, cudaStream_t s) {
  std::memcpy(m->h_io, feat, sizeof(float) * NI);
  if (cudaMemcpyAsync(m->io, m->h_io, sizeof(float) * NI, cudaMemcpyHostToDevice, s) != cudaSuccess) return SW_ECUDA;
  mlp_forward_kernel<<<1, NH, 0, s>>>(m->w, m->norm, m->io, 1, m->io + NI);
  if (cudaMemcpyAsync(m->h_io + NI, m->io + NI, sizeof(float) * NO, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return SW_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SW_ECUDA;
  out2[0] = m->h_io[NI];
  out2[1] = m->h_io[NI + 1];
  return SW_OK;
}

}  // namespace swepi
