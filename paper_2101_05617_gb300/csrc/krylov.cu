// Krylov-side kernels of the phi-function solver (Eq. 29): deterministic grid
// reductions (dot, 2-norm, 1-norm), the incomplete Gram-Schmidt updates, the
// exponential of the small augmented Hessenberg matrix and the combination of
// the basis.  All FP64.
#include <cuda_runtime.h>

#include <cmath>

#include "swepi_internal.h"

namespace swepi {

namespace {

constexpr int RED_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block sum in a fixed order; result valid in thread 0
__device__ double block_sum(double v) {
  __shared__ double ws[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) ws[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? ws[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

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
// exp(A) by scaling and squaring with the [13/13] Pade approximant (Higham,
// "The scaling and squaring method for the matrix exponential revisited",
// SIAM J. Matrix Anal. Appl. 26 (2005)), one thread block, FP64, matrices of
// order N <= MAX_EXPM in global workspace (L2 resident).
constexpr int MAX_EXPM = 160;
constexpr int EXPM_THREADS = 512;

struct Pade {
  double b[14];
  double theta13;
};

__device__ void mm(double* C, const double* A, const double* B, int N) {
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    int r = t / N, c = t % N;
    double s = 0.0;
    for (int k = 0; k < N; ++k) s = fma(A[r * N + k], B[k * N + c], s);
    C[t] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(EXPM_THREADS) expm_kernel(const double* __restrict__ H, int ldh, int j, double tau,
                                                            double tau_happy, const int* happy, double* F,
                                                            double* ws, double* stat, Pade pd) {
  const int jj = happy[0] ? happy[1] : j;
  const double t = happy[0] ? tau_happy : tau;
  const int N = jj + 1;
  const int NN = N * N;
  double* A = ws;
  double* A2 = A + NN;
  double* A4 = A2 + NN;
  double* A6 = A4 + NN;
  double* U = A6 + NN;
  double* V = U + NN;
  double* T1 = V + NN;
  double* T2 = T1 + NN;
  __shared__ double colsum[MAX_EXPM];
  __shared__ int s_sq;
  __shared__ int piv;
  // A = t [[H_jj, e_1], [0, 0]]
  for (int i = threadIdx.x; i < NN; i += blockDim.x) {
    int r = i / N, c = i % N;
    double v = 0.0;
    if (r < jj && c < jj) v = H[(long long)r * ldh + c];
    else if (r == 0 && c == jj) v = 1.0;
    A[i] = t * v;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < N; ++r) s += fabs(A[r * N + c]);
    colsum[c] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double nrm = 0.0;
    for (int c = 0; c < N; ++c) nrm = fmax(nrm, colsum[c]);
    int s = 0;
    if (nrm > pd.theta13) s = (int)ceil(log2(nrm / pd.theta13));
    s_sq = s;
  }
  __syncthreads();
  const double sc = ldexp(1.0, -s_sq);
  for (int i = threadIdx.x; i < NN; i += blockDim.x) A[i] *= sc;
  __syncthreads();
  mm(A2, A, A, N);
  mm(A4, A2, A2, N);
  mm(A6, A4, A2, N);
  const double* b = pd.b;
  for (int i = threadIdx.x; i < NN; i += blockDim.x) {
    T1[i] = b[13] * A6[i] + b[11] * A4[i] + b[9] * A2[i];
    T2[i] = b[12] * A6[i] + b[10] * A4[i] + b[8] * A2[i];
  }
  __syncthreads();
  mm(U, A6, T1, N);   // U holds A6 (b13 A6 + b11 A4 + b9 A2)
  mm(V, A6, T2, N);   // V holds A6 (b12 A6 + b10 A4 + b8 A2)
  for (int i = threadIdx.x; i < NN; i += blockDim.x) {
    int r = i / N, c = i % N;
    double id = (r == c) ? 1.0 : 0.0;
    T1[i] = U[i] + b[7] * A6[i] + b[5] * A4[i] + b[3] * A2[i] + b[1] * id;
    V[i] = V[i] + b[6] * A6[i] + b[4] * A4[i] + b[2] * A2[i] + b[0] * id;
  }
  __syncthreads();
  mm(U, A, T1, N);
  // Q = V - U (in T1), P = V + U (in T2); solve Q X = P
  for (int i = threadIdx.x; i < NN; i += blockDim.x) {
    T1[i] = V[i] - U[i];
    T2[i] = V[i] + U[i];
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int br = k;
      for (int r = k + threadIdx.x; r < N; r += 32) {
        double v = fabs(T1[r * N + k]);
        if (v > best) { best = v; br = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_down_sync(0xffffffffu, best, o);
        int orow = __shfl_down_sync(0xffffffffu, br, o);
        if (ob > best || (ob == best && orow < br)) { best = ob; br = orow; }
      }
      if (threadIdx.x == 0) piv = br;
    }
    __syncthreads();
    const int pr = piv;
    if (pr != k) {
      for (int c = threadIdx.x; c < N; c += blockDim.x) {
        double a1 = T1[k * N + c]; T1[k * N + c] = T1[pr * N + c]; T1[pr * N + c] = a1;
        double a2 = T2[k * N + c]; T2[k * N + c] = T2[pr * N + c]; T2[pr * N + c] = a2;
      }
      __syncthreads();
    }
    const double inv = 1.0 / T1[k * N + k];
    const int rows = N - k - 1;
    const int w = (N - k - 1) + N;   // columns k+1..N-1 of Q, all of P
    for (int t2 = threadIdx.x; t2 < rows * w; t2 += blockDim.x) {
      int r = k + 1 + t2 / w, c = t2 % w;
      double l = T1[r * N + k] * inv;
      if (c < N - k - 1) {
        int cc = k + 1 + c;
        T1[r * N + cc] = fma(-l, T1[k * N + cc], T1[r * N + cc]);
      } else {
        int cc = c - (N - k - 1);
        T2[r * N + cc] = fma(-l, T2[k * N + cc], T2[r * N + cc]);
      }
    }
    __syncthreads();
    // column k below the pivot is not read again
  }
  for (int k = N - 1; k >= 0; --k) {
    const double inv = 1.0 / T1[k * N + k];
    for (int c = threadIdx.x; c < N; c += blockDim.x) T2[k * N + c] *= inv;
    __syncthreads();
    for (int t2 = threadIdx.x; t2 < k * N; t2 += blockDim.x) {
      int r = t2 / N, c = t2 % N;
      T2[r * N + c] = fma(-T1[r * N + k], T2[k * N + c], T2[r * N + c]);
    }
    __syncthreads();
  }
  double* X = T2;
  double* Y = T1;
  for (int q = 0; q < s_sq; ++q) {
    mm(Y, X, X, N);
    double* tmp = X; X = Y; Y = tmp;
  }
  for (int i = threadIdx.x; i < NN; i += blockDim.x) {
    int r = i / N, c = i % N;
    F[(long long)r * ldh + c] = X[i];
  }
  if (threadIdx.x == 0) {
    stat[0] = X[(jj - 1) * N + jj];   // F[jj-1][jj] for the error estimate
    stat[1] = (double)jj;
    stat[2] = t;
    stat[3] = (double)s_sq;
    stat[4] = happy[0] ? 0.0 : H[(long long)jj * ldh + jj - 1];   // h_{j+1,j}
  }
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

int launch_combine(Ctx& c, int j, long long n, cudaStream_t s) {
  if (j > 160) return SW_EINVAL;
  combine_kernel<<<blocks_for(n, 256), 256, 0, s>>>(c.d_X, c.d_V, c.ldv, n, j, c.d_F, c.ldh, c.d_scal);
  c.launches++;
  return cuda_status(cudaGetLastError());
}

int launch_expm_hess(Ctx& c, int j, double tau, double tau_happy, cudaStream_t s) {
  if (j + 1 > MAX_EXPM) return SW_EINVAL;
  Pade pd{};
  // Pade [13/13] coefficients b_k = (26-k)! 13! / (26! k! (13-k)!)
  const int m = 13;
  pd.b[0] = 1.0;
  for (int k = 1; k <= m; ++k) pd.b[k] = pd.b[k - 1] * (double)(m - k + 1) / ((double)k * (double)(2 * m - k + 1));
  // the b_k above are normalised to b_0 = 1 (Higham's table scales them by 26!/13!)
  pd.theta13 = 5.371920351148152;  // Higham (2005), Table 2.3
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c.prof) {
    e0 = prof_event(c);
    e1 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  expm_kernel<<<1, EXPM_THREADS, 0, s>>>(c.d_H, c.ldh, j, tau, tau_happy, c.d_flags, c.d_F, c.d_expm_ws,
                                         c.d_scal + 8, pd);
  if (c.prof) {
    cudaEventRecord(e1, s);
    prof_record(c, PK_EXPM, e0, e1);
  }
  c.launches++;
  return cuda_status(cudaGetLastError());
}

}  // namespace swepi
