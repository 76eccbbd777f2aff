// Krylov-side kernels of the phi-function solver (Eq. 29): deterministic grid
// reductions (dot, 2-norm, 1-norm), the incomplete Gram-Schmidt updates, the
// exponential of the small augmented Hessenberg matrix and the combination of
// the basis.  All FP64.
#include <cuda_runtime.h>

#include <cmath>

#include "krylov_device.cuh"
#include "swepi_internal.h"

namespace swepi {

namespace {

constexpr int RED_THREADS = kPassThreads;

enum { OP_DOT = 0, OP_NORM2 = 1, OP_NORM1 = 2 };

struct RedOut {
  double* dst;
  double tol;       // OP_NORM2: set the happy flag when sqrt(sum) < tol
  int* happy;       // [0] flag, [1] Krylov size at breakdown
  int happy_value;
};

// Two-level deterministic reduction: every block writes its partial sum, the
// last block to finish (atomic ticket) adds the partials in index order.
template <int OP>
__global__ void __launch_bounds__(RED_THREADS) reduce_kernel(const double* __restrict__ x,
                                                             const double* __restrict__ y, long long n,
                                                             double* partials, unsigned int* ticket, RedOut out,
                                                             const int* skip) {
  if (skip && *skip) return;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double a = x[i];
    if (OP == OP_DOT) acc = fma(a, y[i], acc);
    else if (OP == OP_NORM2) acc = fma(a, a, acc);
    else acc += fabs(a);
  }
  double b = block_sum(acc);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = b;
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(partials + i);
  s = block_sum(s);
  if (threadIdx.x == 0) {
    if (OP == OP_NORM2) {
      double r = sqrt(s);
      *out.dst = r;
      if (out.happy && r < out.tol && out.happy[0] == 0) {
        out.happy[0] = 1;
        out.happy[1] = out.happy_value;
      }
    } else {
      *out.dst = s;
    }
    *ticket = 0u;
  }
}

__global__ void axpy_dev_kernel(double* __restrict__ y, const double* __restrict__ x, const double* alpha, long long n,
                                const int* skip) {
  if (skip && *skip) return;
  const double a = *alpha;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(-a, x[i], y[i]);
}

__global__ void scale_inv_kernel(double* __restrict__ y, const double* __restrict__ x, const double* s, long long n,
                                 const int* skip) {
  if (skip && *skip) return;
  const double r = 1.0 / *s;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * r;
}

struct Tail {
  double v[MAX_NB];
};
__global__ void set_tail_kernel(double* x, int p, Tail t) {
  if (threadIdx.x < p) x[threadIdx.x] = t.v[threadIdx.x];
}

struct Lin {
  const double* x[MAX_NB + 2];
  double c[MAX_NB + 2];
};
__global__ void lincomb_kernel(double* __restrict__ out, long long n, int k, Lin L) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < k; ++j)
      if (L.x[j]) s = fma(L.c[j], L.x[j][i], s);
    out[i] = s;
  }
}

__global__ void to_float_scaled_kernel(const double* __restrict__ src, float* __restrict__ dst, long long n,
                                       double scale) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)(scale * src[i]);
}

// w = beta sum_{k<j} F[k][0] V_k (first n entries), beta = scal[0]
__global__ void combine_kernel(double* __restrict__ X, const double* __restrict__ V, long long ldv, long long n, int j,
                               const double* __restrict__ F, int ldh, const double* scal) {
  __shared__ double coef[160];
  for (int k = threadIdx.x; k < j; k += blockDim.x) coef[k] = F[(long long)k * ldh];
  __syncthreads();
  const double beta = scal[0];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < j; ++k) s = fma(coef[k], V[k * ldv + i], s);
    X[i] = beta * s;
  }
}

// ------------------------------------------------------------ expm
// (scheme and workspace slots: krylov_device.cuh)
__global__ void expm_prep_kernel(const double* __restrict__ H, int ldh, int j, double tau, double tau_happy,
                                 const int* happy, double* A, double* stat) {
  expm_prep_body(H, ldh, j, tau, tau_happy, happy, A, stat);
}

// one product over the whole grid (8 x 8 outputs per block)
__global__ void __launch_bounds__(64) small_gemm_kernel(double* __restrict__ ws, int N, int sc, int sa, int sb,
                                                        MatEpi e) {
  const int r = blockIdx.y * 8 + threadIdx.y, c = blockIdx.x * 8 + threadIdx.x;
  if (r >= N || c >= N) return;
  expm_gemm_entry(ws, N, sc, sa, sb, e, r, c);
}

__global__ void expm_finish_kernel(const double* __restrict__ P, int N, double* F, int ldh, double* stat) {
  for (long long i = threadIdx.x + (long long)blockIdx.x * blockDim.x; i < (long long)N * N;
       i += (long long)blockDim.x * gridDim.x)
    expm_finish_entry(P, N, F, ldh, stat, i);
}

__global__ void __launch_bounds__(RED_THREADS) update_norm_kernel(double* __restrict__ z, const double* __restrict__ VA,
                                                                  const double* __restrict__ VB, const double* h1p,
                                                                  const double* h2p, long long n, double* partials,
                                                                  unsigned int* ticket, double* hsub, double tol,
                                                                  int* happy, int happy_value,
                                                                  const double* __restrict__ VC, const double* h0p) {
  pdl_wait();
  pdl_trigger();
  update_norm_dev(z, VA, VB, h1p, h2p, n, partials, ticket, hsub, tol, happy, happy_value, VC, h0p);
}

__global__ void __launch_bounds__(RED_THREADS) scale_dot_kernel(double* __restrict__ z, const double* __restrict__ VB,
                                                                const double* hsub, long long n, double* partials,
                                                                unsigned int* ticket, double* c_out, const int* happy,
                                                                const double* __restrict__ VA, double* c2_out,
                                                                float* __restrict__ z32) {
  pdl_wait();
  pdl_trigger();
  scale_dot_dev(z, VB, hsub, n, partials, ticket, c_out, happy, VA, c2_out, z32);
}

// both passes in one cooperative launch (orth_fused_dev)
__global__ void __launch_bounds__(RED_THREADS, 4) orth_fused_kernel(
    double* __restrict__ z, const double* __restrict__ VA, const double* __restrict__ VB, const double* h1p,
    const double* h2p, long long n, double* partials, unsigned int* ticket, double* hsub, double tol, int* happy,
    int happy_value, const double* __restrict__ VC, const double* h0p, double* c_out, const double* __restrict__ VA2,
    double* c2_out, float* __restrict__ z32, unsigned int* gen, int* err) {
  pdl_trigger();
  orth_fused_dev(z, VA, VB, h1p, h2p, n, partials, ticket, hsub, tol, happy, happy_value, VC, h0p, c_out, VA2, c2_out,
                 z32, gen, err);
}

// the dot pass of the complex64-bulk form (orth_dots_dev)
__global__ void __launch_bounds__(RED_THREADS) orth_dots_kernel(
    const double* __restrict__ z, const double* __restrict__ VB, const double* __restrict__ VA,
    const double* __restrict__ VC, long long n, double* partials, unsigned int* ticket, const int* happy,
    double* h0_out, double* h1_out, double* h2_out, double* cdot_out, double* cdot2_out, const double* cprevAC) {
  pdl_wait();
  pdl_trigger();
  orth_dots_dev(z, VB, VA, VC, n, partials, ticket, happy, h0_out, h1_out, h2_out, cdot_out, cdot2_out, cprevAC);
}

// the dot, update and scale passes in one cooperative launch (orth3_fused_dev)
__global__ void __launch_bounds__(RED_THREADS, 4) orth3_fused_kernel(
    double* __restrict__ z, const double* __restrict__ VA, const double* __restrict__ VB,
    const double* __restrict__ VC, long long n, double* partials, unsigned int* ticket, double tol, int* happy,
    int happy_value, double* h0p, double* h1p, double* h2p, double* hsub, double* cdot_out, double* cdot2_out,
    const double* cprevAC, float* __restrict__ z32, unsigned int* gen, int* err) {
  pdl_trigger();
  orth3_fused_dev(z, VA, VB, VC, n, partials, ticket, tol, happy, happy_value, h0p, h1p, h2p, hsub, cdot_out,
                  cdot2_out, cprevAC, z32, gen, err);
}

int blocks_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 4 * 152 * 4) b = 4 * 152 * 4;
  if (b < 1) b = 1;
  return (int)b;
}

// FP64 FMA throughput probe: 8 independent FMA chains per thread, registers only
__global__ void fma_probe_kernel(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = threadIdx.x + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  if (s == 12345.678) out[0] = s;   // keeps the chains live; never true in practice
}

}  // namespace

double fp64_fma_peak_tflops() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return -1.0;
  const int blocks = sms * 4, threads = 256, iters = 4096;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 3; ++w) fma_probe_kernel<<<blocks, threads>>>(out, iters, 0.999, 0.001);
  cudaEventRecord(e0);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) fma_probe_kernel<<<blocks, threads>>>(out, iters, 0.999, 0.001);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess || ms <= 0.f) return -1.0;
  double fmas = (double)blocks * threads * iters * 8.0 * reps;
  return 2.0 * fmas / (ms * 1e-3) / 1e12;
}

int launch_dot(Ctx& c, const double* x, const double* y, long long n, double* dst, const int* skip, cudaStream_t s) {
  RedOut o{dst, 0.0, nullptr, 0};
  reduce_kernel<OP_DOT><<<RED_BLOCKS, RED_THREADS, 0, s>>>(x, y, n, c.d_partials, (unsigned int*)(c.d_flags + 8), o,
                                                          skip);
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_norm2(Ctx& c, const double* x, long long n, double* dst, double tol, int* happy, int happy_value,
                 const int* skip, cudaStream_t s) {
  RedOut o{dst, tol, happy, happy_value};
  reduce_kernel<OP_NORM2><<<RED_BLOCKS, RED_THREADS, 0, s>>>(x, nullptr, n, c.d_partials,
                                                            (unsigned int*)(c.d_flags + 8), o, skip);
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_norm1(Ctx& c, const double* x, long long n, double* dst, cudaStream_t s) {
  RedOut o{dst, 0.0, nullptr, 0};
  reduce_kernel<OP_NORM1><<<RED_BLOCKS, RED_THREADS, 0, s>>>(x, nullptr, n, c.d_partials,
                                                            (unsigned int*)(c.d_flags + 8), o, nullptr);
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_axpy_dev(Ctx& c, double* y, const double* x, const double* alpha, long long n, const int* skip,
                    cudaStream_t s) {
  axpy_dev_kernel<<<blocks_for(n, 256), 256, 0, s>>>(y, x, alpha, n, skip);
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_scale_inv(Ctx& c, double* y, const double* x, const double* s_dev, long long n, const int* skip,
                     cudaStream_t s) {
  scale_inv_kernel<<<blocks_for(n, 256), 256, 0, s>>>(y, x, s_dev, n, skip);
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_update_norm(Ctx& c, double* z, const double* VA, const double* VB, const double* h1, const double* h2,
                       long long N, double* hsub, double tol, int happy_value, cudaStream_t s, const double* VC,
                       const double* h0) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (prof_on(c, PK_ORTH)) {
    e0 = prof_event(c);
    e1 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  if (launch_pdl(update_norm_kernel, dim3(RED_BLOCKS), dim3(RED_THREADS), s, z, VA, VB, h1, h2, N, c.d_partials,
                 (unsigned int*)(c.d_flags + 8), hsub, tol, c.d_flags, happy_value, VC, h0) != cudaSuccess)
    return SW_ECUDA;
  if (prof_on(c, PK_ORTH)) {
    cudaEventRecord(e1, s);
    prof_record(c, PK_ORTH, e0, e1);
  }
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_scale_dot(Ctx& c, double* z, const double* VB, const double* hsub, long long N, double* c_out,
                     cudaStream_t s, const double* VA, double* c2_out, float* z32) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (prof_on(c, PK_ORTH)) {
    e0 = prof_event(c);
    e1 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  if (launch_pdl(scale_dot_kernel, dim3(RED_BLOCKS), dim3(RED_THREADS), s, z, VB, hsub, N, c.d_partials,
                 (unsigned int*)(c.d_flags + 8), c_out, c.d_flags, VA, c2_out, z32) != cudaSuccess)
    return SW_ECUDA;
  if (prof_on(c, PK_ORTH)) {
    cudaEventRecord(e1, s);
    prof_record(c, PK_ORTH, e0, e1);
  }
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int orth_fused_available(Ctx& c) {
  if (c.orth_fused == 0) {
    // both cooperative kernels (two and three phases) hold the whole grid at once
    int coop = 0, sms = 0, nb = 0, nb3 = 0;
    c.orth_fused = -1;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c.device) == cudaSuccess && coop &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, orth_fused_kernel, RED_THREADS, 0) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb3, orth3_fused_kernel, RED_THREADS, 0) == cudaSuccess &&
        (long long)nb * sms >= RED_BLOCKS && (long long)nb3 * sms >= RED_BLOCKS)
      c.orth_fused = 1;
  }
  return c.orth_fused > 0;
}

int launch_orth_dots(Ctx& c, const double* z, const double* VB, const double* VA, const double* VC, long long N,
                     double* h0_out, double* h1_out, double* h2_out, double* cdot_out, double* cdot2_out,
                     const double* cprevAC, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (prof_on(c, PK_ORTH)) {
    e0 = prof_event(c);
    e1 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  if (launch_pdl(orth_dots_kernel, dim3(RED_BLOCKS), dim3(RED_THREADS), s, z, VB, VA, VC, N, c.d_partials,
                 reinterpret_cast<unsigned int*>(c.d_flags + 8), static_cast<const int*>(c.d_flags), h0_out, h1_out,
                 h2_out, cdot_out, cdot2_out, cprevAC) != cudaSuccess)
    return SW_ECUDA;
  if (prof_on(c, PK_ORTH)) {
    cudaEventRecord(e1, s);
    prof_record(c, PK_ORTH, e0, e1);
  }
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_orth3_fused(Ctx& c, double* z, const double* VA, const double* VB, const double* VC, long long N,
                       double tol, int happy_value, double* h0p, double* h1p, double* h2p, double* hsub,
                       double* cdot_out, double* cdot2_out, const double* cprevAC, float* z32, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (prof_on(c, PK_ORTH)) {
    e0 = prof_event(c);
    e1 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(RED_BLOCKS);
  cfg.blockDim = dim3(RED_THREADS);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, orth3_fused_kernel, z, VA, VB, VC, N, c.d_partials,
                         reinterpret_cast<unsigned int*>(c.d_flags + 8), tol, c.d_flags, happy_value, h0p, h1p, h2p,
                         hsub, cdot_out, cdot2_out, cprevAC, z32, reinterpret_cast<unsigned int*>(c.d_flags + 10),
                         c.d_flags + 3) != cudaSuccess)
    return SW_ECUDA;
  if (prof_on(c, PK_ORTH)) {
    cudaEventRecord(e1, s);
    prof_record(c, PK_ORTH, e0, e1);
    prof_record(c, PK_ORTH, e1, e1);   // counted as the two passes of the other forms
  }
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_orth_fused(Ctx& c, double* z, const double* VA, const double* VB, const double* h1, const double* h2,
                      long long N, double* hsub, double tol, int happy_value, const double* VC, const double* h0,
                      double* c_out, const double* VA2, double* c2_out, float* z32, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (prof_on(c, PK_ORTH)) {
    e0 = prof_event(c);
    e1 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(RED_BLOCKS);
  cfg.blockDim = dim3(RED_THREADS);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, orth_fused_kernel, z, VA, VB, h1, h2, N, c.d_partials,
                         reinterpret_cast<unsigned int*>(c.d_flags + 8), hsub, tol, c.d_flags, happy_value, VC, h0,
                         c_out, VA2, c2_out, z32, reinterpret_cast<unsigned int*>(c.d_flags + 10),
                         c.d_flags + 3) != cudaSuccess)
    return SW_ECUDA;
  if (prof_on(c, PK_ORTH)) {
    cudaEventRecord(e1, s);
    prof_record(c, PK_ORTH, e0, e1);
    prof_record(c, PK_ORTH, e1, e1);   // counted as the two passes it replaces
  }
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_set_tail(Ctx& c, double* x, long long n, int p, const double* vals, cudaStream_t s) {
  Tail t{};
  for (int l = 0; l < p && l < MAX_NB; ++l) t.v[l] = vals[l];
  set_tail_kernel<<<1, 32, 0, s>>>(x + n, p, t);
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_lincomb(Ctx& c, double* out, long long n, int k, const double* const* xs, const double* coef,
                   cudaStream_t s) {
  if (k > MAX_NB + 2) return SW_EINVAL;
  Lin L{};
  for (int j = 0; j < k; ++j) { L.x[j] = xs[j]; L.c[j] = coef[j]; }
  lincomb_kernel<<<blocks_for(n, 256), 256, 0, s>>>(out, n, k, L);
  c.launches++;
  return cuda_status(cudaGetLastError());
}

__global__ void to_float_rn_kernel(const double* __restrict__ src, float* __restrict__ dst, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = f64_to_f32_bits(src[i]);
}

int launch_to_float(Ctx& c, const double* src, float* dst, long long n, cudaStream_t s) {
  to_float_rn_kernel<<<blocks_for(n, 256), 256, 0, s>>>(src, dst, n);
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_to_float_scaled(Ctx& c, const double* src, float* dst, long long n, double scale, cudaStream_t s) {
  to_float_scaled_kernel<<<blocks_for(n, 256), 256, 0, s>>>(src, dst, n, scale);
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_combine(Ctx& c, int j, long long n, cudaStream_t s) {
  if (j > 160) return SW_EINVAL;
  combine_kernel<<<blocks_for(n, 256), 256, 0, s>>>(c.d_X, c.d_V, c.ldv, n, j, c.d_F, c.ldh, c.d_scal);
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_expm_prep(Ctx& c, int j, double tau, double tau_happy, cudaStream_t s) {
  if (j + 1 > MAX_EXPM) return SW_EINVAL;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (prof_on(c, PK_EXPM)) {
    e0 = prof_event(c);
    e1 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  expm_prep_kernel<<<1, 256, 0, s>>>(c.d_H, c.ldh, j, tau, tau_happy, c.d_flags, c.d_expm_ws, c.d_scal + 8);
  if (prof_on(c, PK_EXPM)) {
    cudaEventRecord(e1, s);
    prof_record(c, PK_EXPM, e0, e1);
  }
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_expm_eval(Ctx& c, int N, double norm1, int* squarings, cudaStream_t s) {
  if (N < 2 || N > MAX_EXPM || !std::isfinite(norm1)) return SW_EINVAL;
  const int sq = expm_squarings(norm1);
  if (sq < 0) return SW_ENONFINITE;
  if (squarings) *squarings = sq;
  const long long NN = (long long)N * N;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (prof_on(c, PK_EXPM)) {
    e0 = prof_event(c);
    e1 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  ExpmProduct pr[8];
  expm_products(sq, pr);
  const dim3 blk(8, 8), grd((N + 7) / 8, (N + 7) / 8);
  for (int k = 0; k < 8; ++k) small_gemm_kernel<<<grd, blk, 0, s>>>(c.d_expm_ws, N, pr[k].c, pr[k].a, pr[k].b, pr[k].e);
  const MatEpi none{0, 0, 0, 0, -1, -1, -1, 1.0};
  for (int q = 0; q < sq; ++q) {
    const int src = expm_square_src(q);
    small_gemm_kernel<<<grd, blk, 0, s>>>(c.d_expm_ws, N, expm_square_dst(q), src, src, none);
  }
  expm_finish_kernel<<<(unsigned)((NN + 255) / 256), 256, 0, s>>>(c.d_expm_ws + expm_result_slot(sq) * NN, N, c.d_F,
                                                                 c.ldh, c.d_scal + 8);
  if (prof_on(c, PK_EXPM)) {
    cudaEventRecord(e1, s);
    prof_record(c, PK_EXPM, e0, e1);
  }
  c.launches += 9 + sq;
  return cuda_status(cudaGetLastError());
}

}  // namespace swepi
