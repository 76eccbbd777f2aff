// Device pieces of the Krylov side shared by the single-grid launchers
// (krylov.cu) and the batched ensemble (ensemble.cu): fixed-order block
// reductions and the exponential of the small augmented Hessenberg matrix.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "convert.cuh"

namespace swepi {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// threads of the vector-pass and reduction launches (krylov.cu, the
// device-driven solver)
constexpr int kPassThreads = 256;

// block sum in a fixed order over a block of THREADS threads (all of which
// call it); result valid in thread 0.  Every thread stores its value in shared
// memory and warp 0 alone sums them (a stride of 32, then a shuffle tree): on
// this GPU a shuffle tree in every warp would cost each warp five FP64 adds on
// the slow FP64 pipe.
template <int THREADS = kPassThreads>
__device__ __forceinline__ double block_sum(double v) {
  static_assert(THREADS >= 32 && THREADS <= 1024 && THREADS % 32 == 0, "block of whole warps");
  __shared__ double sb[THREADS];
  __syncthreads();   // an earlier call's readers are done with sb
  if (threadIdx.x < THREADS) sb[threadIdx.x] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = sb[threadIdx.x];
#pragma unroll
    for (int i = threadIdx.x + 32; i < THREADS; i += 32) r += sb[i];
    r = warp_sum(r);
  }
  return r;
}

// K block sums at once (K <= the block's warps): every thread stores its K
// values, warp k sums value k exactly as block_sum does (a stride of 32, then a
// shuffle tree; the same result bit for bit), so the sums run side by side on
// the SM's warp schedulers instead of one after another in warp 0.  Results
// valid in thread 0.
template <int K, int THREADS = kPassThreads>
__device__ __forceinline__ void block_sums_k(double v[K]) {
  static_assert(K >= 1 && K <= THREADS / 32, "one warp per value");
  __shared__ double sb[K * THREADS];
  __shared__ double res[K];
  __syncthreads();   // an earlier call's readers are done with sb
#pragma unroll
  for (int k = 0; k < K; ++k) sb[k * THREADS + threadIdx.x] = v[k];
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < K) {
    double r = sb[w * THREADS + lane];
#pragma unroll
    for (int i = lane + 32; i < THREADS; i += 32) r += sb[w * THREADS + i];
    r = warp_sum(r);
    if (lane == 0) res[w] = r;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = res[k];
  }
}

// ------------------------------------------------------------ orthogonalisation passes
// The two vector passes of the window-2 modified Gram-Schmidt step over the
// indices i0, i0 + stride, ... < i1 of one thread, eight elements in flight
// with two window vectors, four with three (the 64-register budget of the
// cooperative grid); the order of the operations is the same either way
// (z was written by another kernel or CTA: read through L2).
//   z -= h0 VC + h1 VA + h2 VB (VC, VA may be null; oldest first); returns the
//   thread's sum of z_i^2
// HA, HC: VA, VC present (compiled in, so that no guarded-off FP64
// instruction takes the FP64 pipe's issue slots)
template <bool HA, bool HC>
__device__ __forceinline__ double mgs_update_range_t(double* __restrict__ z, const double* __restrict__ VA,
                                                     const double* __restrict__ VB, double h1, double h2, long long i,
                                                     long long i1, long long stride, const double* __restrict__ VC,
                                                     double h0) {
  constexpr int D = HC ? 4 : 8;   // entries in flight per thread
  double acc = 0.0;
  for (; i + (D - 1) * stride < i1; i += D * stride) {
    double v[D], b[D], a[D], c[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      v[k] = __ldcg(z + i + k * stride);
      b[k] = VB[i + k * stride];
      if (HA) a[k] = VA[i + k * stride];
      if (HC) c[k] = VC[i + k * stride];
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (HC) v[k] = fma(-h0, c[k], v[k]);
      if (HA) v[k] = fma(-h1, a[k], v[k]);
      v[k] = fma(-h2, b[k], v[k]);
      z[i + k * stride] = v[k];
      acc = fma(v[k], v[k], acc);
    }
  }
  for (; i < i1; i += stride) {
    double v = __ldcg(z + i);
    if (HC) v = fma(-h0, VC[i], v);
    if (HA) v = fma(-h1, VA[i], v);
    v = fma(-h2, VB[i], v);
    z[i] = v;
    acc = fma(v, v, acc);
  }
  return acc;
}

__device__ __forceinline__ double mgs_update_range(double* __restrict__ z, const double* __restrict__ VA,
                                                   const double* __restrict__ VB, double h1, double h2, long long i,
                                                   long long i1, long long stride,
                                                   const double* __restrict__ VC = nullptr, double h0 = 0.0) {
  if (VC) {
    return VA ? mgs_update_range_t<true, true>(z, VA, VB, h1, h2, i, i1, stride, VC, h0)
              : mgs_update_range_t<false, true>(z, VA, VB, h1, h2, i, i1, stride, VC, h0);
  }
  return VA ? mgs_update_range_t<true, false>(z, VA, VB, h1, h2, i, i1, stride, VC, h0)
            : mgs_update_range_t<false, false>(z, VA, VB, h1, h2, i, i1, stride, VC, h0);
}

//   z *= r; returns the thread's sum of z_i VB_i, and with VA also the sum of
//   z_i VA_i in *za; with z32, also the FP32 copy of the scaled z (rounded to
//   nearest) for the complex64-bulk form's kernels
__device__ __forceinline__ double scale_dot_range(double* __restrict__ z, const double* __restrict__ VB, double r,
                                                  long long i, long long i1, long long stride,
                                                  const double* __restrict__ VA = nullptr, double* za = nullptr,
                                                  float* __restrict__ z32 = nullptr) {
  if (VA) {
    double acc = 0.0, acc2 = 0.0;
    for (; i + 3 * stride < i1; i += 4 * stride) {
      double v[4], b[4], a[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        v[k] = __ldcg(z + i + k * stride);
        b[k] = VB[i + k * stride];
        a[k] = VA[i + k * stride];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        v[k] *= r;
        z[i + k * stride] = v[k];
        if (z32) z32[i + k * stride] = f64_to_f32_bits(v[k]);
        acc = fma(v[k], b[k], acc);
        acc2 = fma(v[k], a[k], acc2);
      }
    }
    for (; i < i1; i += stride) {
      const double v = __ldcg(z + i) * r;
      z[i] = v;
      if (z32) z32[i] = f64_to_f32_bits(v);
      acc = fma(v, VB[i], acc);
      acc2 = fma(v, VA[i], acc2);
    }
    *za = acc2;
    return acc;
  }
  double acc = 0.0;
  for (; i + 3 * stride < i1; i += 4 * stride) {
    double v[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = __ldcg(z + i + k * stride);
      b[k] = VB[i + k * stride];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] *= r;
      z[i + k * stride] = v[k];
      if (z32) z32[i + k * stride] = f64_to_f32_bits(v[k]);
      acc = fma(v[k], b[k], acc);
    }
  }
  for (; i < i1; i += stride) {
    const double v = __ldcg(z + i) * r;
    z[i] = v;
    if (z32) z32[i] = f64_to_f32_bits(v);
    acc = fma(v, VB[i], acc);
  }
  return acc;
}

// The two vector passes of the fused incomplete orthogonalisation, as device
// functions of a whole grid (the stream kernels of krylov.cu and the
// device-driven solver call them).
// z -= h0 V_C + h1 V_A + h2 V_B (the modified Gram-Schmidt updates, oldest
// first; V_C, V_A may be absent), then ||z||_2 -> *hsub with the
// happy-breakdown flag below tol.  Returns 0 when the basis had already broken
// down (nothing done), 2 in the CTA that finished last (it wrote *hsub), else 1
// (uniform over each CTA).
__device__ __forceinline__ int update_norm_dev(double* __restrict__ z, const double* __restrict__ VA,
                                               const double* __restrict__ VB, const double* h1p, const double* h2p,
                                               long long n, double* partials, unsigned int* ticket, double* hsub,
                                               double tol, int* happy, int happy_value, const double* __restrict__ VC,
                                               const double* h0p) {
  if (__ldcg(happy)) return 0;
  // through L2: in a fused launch another CTA has just written them
  const double h1 = VA ? __ldcg(h1p) : 0.0, h2 = __ldcg(h2p), h0 = VC ? __ldcg(h0p) : 0.0;
  const double acc = mgs_update_range(z, VA, VB, h1, h2, (long long)blockIdx.x * blockDim.x + threadIdx.x, n,
                                      (long long)gridDim.x * blockDim.x, VC, h0);
  double b = block_sum(acc);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = b;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return 1;
  __threadfence();
  double sum = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) sum += __ldcg(partials + i);
  sum = block_sum(sum);
  if (threadIdx.x == 0) {
    const double r = sqrt(sum);
    *hsub = r;
    if (r < tol) {
      happy[0] = 1;
      happy[1] = happy_value;
    }
    *ticket = 0u;
  }
  return 2;
}

// V_next = z / *hsub in place, V_next . V_B -> *c_out and, with V_A, V_next .
// V_A -> *c2_out (used by the next iterations' orthogonalisation); with z32
// also the FP32 copy of V_next
__device__ __forceinline__ void scale_dot_dev(double* __restrict__ z, const double* __restrict__ VB,
                                              const double* hsub, long long n, double* partials, unsigned int* ticket,
                                              double* c_out, const int* happy, const double* __restrict__ VA,
                                              double* c2_out, float* __restrict__ z32) {
  // through L2: in the fused launch another CTA has just written them
  if (__ldcg(happy)) return;
  const double r = 1.0 / __ldcg(hsub);
  if (!c_out) {   // scale only (the next volume kernel forms the dots)
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const double v = __ldcg(z + i) * r;
      z[i] = v;
      if (z32) z32[i] = f64_to_f32_bits(v);
    }
    return;
  }
  double acc2 = 0.0;
  const double acc = scale_dot_range(z, VB, r, (long long)blockIdx.x * blockDim.x + threadIdx.x, n,
                                     (long long)gridDim.x * blockDim.x, VA, &acc2, z32);
  const double b = block_sum(acc);
  const double b2 = VA ? block_sum(acc2) : 0.0;   // uniform condition
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = b;
    partials[2 * blockIdx.x + 1] = b2;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double sum = 0.0, sum2 = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    sum += __ldcg(partials + 2 * i);
    if (VA) sum2 += __ldcg(partials + 2 * i + 1);
  }
  sum = block_sum(sum);
  if (VA) sum2 = block_sum(sum2);
  if (threadIdx.x == 0) {
    *c_out = sum;
    if (VA) *c2_out = sum2;
    *ticket = 0u;
  }
}

// polls of the fused pass's grid-wide wait (each after a short sleep: about a
// second in all) before it gives up
constexpr unsigned int kOrthWaitPolls = 1u << 23;

// Both passes in one launch of a grid whose CTAs are all resident at once (a
// cooperative launch): the update pass, then -- once the CTA that finished it
// last has published ||z|| by advancing the counter *gen -- the scale pass.
// The same arithmetic in the same order as update_norm_dev followed by
// scale_dot_dev on the same grid (bitwise the same results); it saves the
// second launch and its ramp.  A CTA that waits past the bound sets *err and
// leaves its share of the scale pass undone (the caller reports a timeout).
__device__ __forceinline__ void orth_fused_dev(double* __restrict__ z, const double* __restrict__ VA,
                                               const double* __restrict__ VB, const double* h1p, const double* h2p,
                                               long long n, double* partials, unsigned int* ticket, double* hsub,
                                               double tol, int* happy, int happy_value, const double* __restrict__ VC,
                                               const double* h0p, double* c_out, const double* __restrict__ VA2,
                                               double* c2_out, float* __restrict__ z32, unsigned int* gen, int* err) {
  __shared__ unsigned int g0;
  __shared__ int gave_up;
  // read before this CTA's ticket (ordered by the fence ahead of it): the
  // counter can only advance after every CTA has taken its ticket
  if (threadIdx.x == 0) {
    g0 = *reinterpret_cast<volatile unsigned int*>(gen);
    gave_up = 0;
  }
  const int st = update_norm_dev(z, VA, VB, h1p, h2p, n, partials, ticket, hsub, tol, happy, happy_value, VC, h0p);
  if (st == 0) return;   // uniform over the grid
  if (threadIdx.x == 0) {
    if (st == 2) {
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      unsigned int polls = 0;
      while (*reinterpret_cast<volatile unsigned int*>(gen) == g0) {
        if (++polls > kOrthWaitPolls) {
          gave_up = 1;
          atomicExch(err, 1);
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
  }
  __syncthreads();
  if (gave_up) return;
  scale_dot_dev(z, VB, hsub, n, partials, ticket, c_out, happy, VA2, c2_out, z32);
}

// The window dots of the incomplete orthogonalisation as a pass of their own
// (the complex64-bulk form, whose FP32 volume kernel forms none), over the N
// entries of the augmented vectors (the tails included): z . V_{j-1}, z . V_j,
// z . V_{j-2}, V_j . V_{j-1}, V_j . V_{j-2} into s[0..4] for one thread's
// indices.  HA, HC: V_{j-1}, V_{j-2} present.
template <bool HA, bool HC>
__device__ __forceinline__ void orth_dots_range_t(const double* __restrict__ z, const double* __restrict__ VB,
                                                  const double* __restrict__ VA, const double* __restrict__ VC,
                                                  long long i, long long i1, long long stride, double s[5]) {
  double da = 0.0, db = 0.0, dc = 0.0, dab = 0.0, dbc = 0.0;
  for (; i + 3 * stride < i1; i += 4 * stride) {
    double zz[4], b[4], a[4], c[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      zz[k] = __ldcg(z + i + k * stride);
      b[k] = VB[i + k * stride];
      if (HA) a[k] = VA[i + k * stride];
      if (HC) c[k] = VC[i + k * stride];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      db = fma(zz[k], b[k], db);
      if (HA) {
        da = fma(zz[k], a[k], da);
        dab = fma(b[k], a[k], dab);
      }
      if (HC) {
        dc = fma(zz[k], c[k], dc);
        dbc = fma(b[k], c[k], dbc);
      }
    }
  }
  for (; i < i1; i += stride) {
    const double zz = __ldcg(z + i), b = VB[i];
    db = fma(zz, b, db);
    if (HA) {
      const double a = VA[i];
      da = fma(zz, a, da);
      dab = fma(b, a, dab);
    }
    if (HC) {
      const double c = VC[i];
      dc = fma(zz, c, dc);
      dbc = fma(b, c, dbc);
    }
  }
  s[0] = da;
  s[1] = db;
  s[2] = dc;
  s[3] = dab;
  s[4] = dbc;
}

// The dot pass over a whole grid: the five sums above; the CTA that finishes
// last forms the modified Gram-Schmidt coefficients from them exactly as the
// volume epilogue does (h0 = z . V_{j-2}; h1 = z . V_{j-1} - h0 V_{j-1} . V_{j-2};
// h2 = z . V_j - h0 V_j . V_{j-2} - h1 V_j . V_{j-1}, with the window's vectors
// present) and stores V_j . V_{j-1}, V_j . V_{j-2} for the next iterations.
// partials: 5 per CTA.  Returns 0 when the basis had already broken down
// (nothing done), 2 in the CTA that finished last, else 1.
__device__ __forceinline__ int orth_dots_dev(const double* __restrict__ z, const double* __restrict__ VB,
                                             const double* __restrict__ VA, const double* __restrict__ VC,
                                             long long n, double* partials, unsigned int* ticket, const int* happy,
                                             double* h0_out, double* h1_out, double* h2_out, double* cdot_out,
                                             double* cdot2_out, const double* cprevAC) {
  if (__ldcg(happy)) return 0;
  double s[5];
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  if (VC) {
    if (VA)
      orth_dots_range_t<true, true>(z, VB, VA, VC, i0, n, stride, s);
    else
      orth_dots_range_t<false, true>(z, VB, VA, VC, i0, n, stride, s);
  } else if (VA) {
    orth_dots_range_t<true, false>(z, VB, VA, VC, i0, n, stride, s);
  } else {
    orth_dots_range_t<false, false>(z, VB, VA, VC, i0, n, stride, s);
  }
  block_sums_k<5>(s);
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) partials[5 * blockIdx.x + k] = s[k];
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return 1;
  __threadfence();
  double u[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 5; ++k) u[k] += __ldcg(partials + 5 * i + k);
  }
  block_sums_k<5>(u);
  if (threadIdx.x == 0) {
    const double a = u[0], bb = u[1], c3 = u[2];
    if (VA) *cdot_out = u[3];    // V_j . V_{j-1}
    if (VC) *cdot2_out = u[4];   // V_j . V_{j-2}
    if (VC) {
      const double h0 = c3;
      const double h1 = a - h0 * __ldcg(cprevAC);
      *h0_out = h0;
      *h1_out = h1;
      *h2_out = bb - h0 * u[4] - h1 * u[3];
    } else if (VA) {
      *h1_out = a;
      *h2_out = bb - a * u[3];
    } else {
      *h2_out = bb;
    }
    *ticket = 0u;
  }
  return 2;
}

// One grid-wide step of a cooperative launch (all CTAs call it, every thread):
// the CTA that finished a phase last (`last`) advances *gen; the others wait,
// bounded, until *gen has reached `target`.  False when the wait gave up (the
// CTA then leaves its remaining phases undone and *err is set).
__device__ __forceinline__ bool grid_step(unsigned int* gen, unsigned int target, bool last, int* err) {
  __shared__ int gave_up;
  if (threadIdx.x == 0) {
    gave_up = 0;
    if (last) {
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      unsigned int polls = 0;
      while ((int)(*reinterpret_cast<volatile unsigned int*>(gen) - target) < 0) {
        if (++polls > kOrthWaitPolls) {
          gave_up = 1;
          atomicExch(err, 1);
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
  }
  __syncthreads();
  return !gave_up;
}

// The dot pass, the update pass and the scale pass of the complex64-bulk form
// in one cooperative launch (two grid-wide steps); the same arithmetic in the
// same order as orth_dots_dev, update_norm_dev and scale_dot_dev on the same
// grid.  The H entries and the norm pass between the phases through L2.
__device__ __forceinline__ void orth3_fused_dev(double* __restrict__ z, const double* __restrict__ VA,
                                                const double* __restrict__ VB, const double* __restrict__ VC,
                                                long long n, double* partials, unsigned int* ticket, double tol,
                                                int* happy, int happy_value, double* h0p, double* h1p, double* h2p,
                                                double* hsub, double* cdot_out, double* cdot2_out,
                                                const double* cprevAC, float* __restrict__ z32, unsigned int* gen,
                                                int* err) {
  __shared__ unsigned int g0;
  // read before this CTA's first ticket (ordered by the fence ahead of it)
  if (threadIdx.x == 0) g0 = *reinterpret_cast<volatile unsigned int*>(gen);
  int st = orth_dots_dev(z, VB, VA, VC, n, partials, ticket, happy, h0p, h1p, h2p, cdot_out, cdot2_out, cprevAC);
  if (st == 0) return;   // uniform over the grid
  if (!grid_step(gen, g0 + 1u, st == 2, err)) return;
  st = update_norm_dev(z, VA, VB, h1p, h2p, n, partials, ticket, hsub, tol, happy, happy_value, VC, h0p);
  if (st == 0) return;
  if (!grid_step(gen, g0 + 2u, st == 2, err)) return;
  scale_dot_dev(z, VB, hsub, n, partials, ticket, nullptr, happy, nullptr, nullptr, z32);
}

// ------------------------------------------------------------ expm
// F = exp(A), A = t [[H_j, e_1], [0, 0]] (order N = j + 1 <= MAX_EXPM): scaling
// and squaring (Moler and Van Loan, "Nineteen dubious ways to compute the
// exponential of a matrix, twenty-five years later", SIAM Rev. 45, 2003) with
// the degree-16 Taylor polynomial, evaluated by the Paterson-Stockmeyer scheme
// (SIAM J. Comput. 2, 1973) in blocks of four powers: 8 matrix products (the
// first is the scaling), then s squarings, s = max(0, ceil(log2(||A||_1 / 0.8))).
// At ||X||_1 <= 0.8 the truncated tail is below 0.8^17/17! = 6e-17.  The
// matrices live in a workspace of XS_COUNT dense N x N slots.
constexpr int MAX_EXPM = 160;
constexpr double kTaylorTheta = 0.8;
enum ExpmSlot { XS_A = 0, XS_X, XS_X2, XS_X3, XS_X4, XS_P0, XS_P1, XS_COUNT };

struct MatEpi {
  // C = alpha * A B + cI * I + c1 * M1 + c2 * M2 + c3 * M3 (slot -1: absent;
  // A or B absent means the identity)
  double cI, c1, c2, c3;
  int s1, s2, s3;
  double alpha;
};

struct ExpmProduct {
  int c, a, b;
  MatEpi e;
};

// the 8 products before the squarings, for s squarings
inline __host__ __device__ void expm_products(int sq, ExpmProduct out[8]) {
  double cf[17];
  cf[0] = 1.0;
  for (int k = 1; k <= 16; ++k) cf[k] = cf[k - 1] / k;   // 1/k!
  const MatEpi none{0, 0, 0, 0, -1, -1, -1, 1.0};
  MatEpi sc = none;
  sc.alpha = ::ldexp(1.0, -sq);
  out[0] = {XS_X, XS_A, -1, sc};                          // X = A / 2^s
  out[1] = {XS_X2, XS_X, XS_X, none};
  out[2] = {XS_X3, XS_X2, XS_X, none};
  out[3] = {XS_X4, XS_X2, XS_X2, none};
  // Paterson-Stockmeyer: T = B0 + X4 (B1 + X4 (B2 + X4 (B3 + c16 X4))), B_i = sum_k c_{4i+k} X^k
  out[4] = {XS_P0, XS_X4, -1, {cf[12], cf[13], cf[14], cf[15], XS_X, XS_X2, XS_X3, cf[16]}};
  out[5] = {XS_P1, XS_X4, XS_P0, {cf[8], cf[9], cf[10], cf[11], XS_X, XS_X2, XS_X3, 1.0}};
  out[6] = {XS_P0, XS_X4, XS_P1, {cf[4], cf[5], cf[6], cf[7], XS_X, XS_X2, XS_X3, 1.0}};
  out[7] = {XS_P1, XS_X4, XS_P0, {cf[0], cf[1], cf[2], cf[3], XS_X, XS_X2, XS_X3, 1.0}};
}

// number of squarings for ||A||_1 (-1: too large to be finite)
inline __host__ __device__ int expm_squarings(double norm1) {
  int sq = 0;
  if (norm1 > kTaylorTheta) sq = (int)::ceil(::log2(norm1 / kTaylorTheta));
  return (sq > 200) ? -1 : sq;
}
// squaring q reads slot expm_square_src(q) and writes the other one
inline __host__ __device__ int expm_square_src(int q) { return (q % 2 == 0) ? XS_P1 : XS_P0; }
inline __host__ __device__ int expm_square_dst(int q) { return (q % 2 == 0) ? XS_P0 : XS_P1; }
// slot holding exp(A) after s squarings
inline __host__ __device__ int expm_result_slot(int sq) { return expm_square_src(sq); }

// one block: build A (dense, leading dimension N) in slot XS_A and its
// 1-norm; stat[1] = j used, stat[2] = t, stat[4] = h_{j+1,j}, stat[5] = ||A||_1
__device__ __forceinline__ void expm_prep_body(const double* __restrict__ H, int ldh, int j, double tau,
                                               double tau_happy, const int* happy, double* A, double* stat) {
  const int jj = happy[0] ? happy[1] : j;
  const double t = happy[0] ? tau_happy : tau;
  const int N = jj + 1;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    int r = i / N, c = i % N;
    double v = 0.0;
    if (r < jj && c < jj) v = H[(long long)r * ldh + c];
    else if (r == 0 && c == jj) v = 1.0;
    A[i] = t * v;
  }
  __syncthreads();
  __shared__ double colsum[MAX_EXPM];
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    double sum = 0.0;
    for (int r = 0; r < N; ++r) sum += fabs(A[r * N + c]);
    colsum[c] = sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double nrm = 0.0;
    for (int c = 0; c < N; ++c) nrm = fmax(nrm, colsum[c]);
    stat[1] = (double)jj;
    stat[2] = t;
    stat[4] = happy[0] ? 0.0 : H[(long long)jj * ldh + jj - 1];   // h_{j+1,j}
    stat[5] = nrm;
  }
}

// entry (r, c) of one product in the workspace ws (slots of N x N)
__device__ __forceinline__ void expm_gemm_entry(double* __restrict__ ws, int N, int sc, int sa, int sb,
                                                const MatEpi& e, int r, int c) {
  const long long NN = (long long)N * N;
  const double* A = (sa >= 0) ? ws + sa * NN : nullptr;
  const double* B = (sb >= 0) ? ws + sb * NN : nullptr;
  double s = 0.0;
  if (A && B) {
    for (int k = 0; k < N; ++k) s = fma(A[r * N + k], B[k * N + c], s);
  } else if (A) {
    s = A[r * N + c];
  } else if (B) {
    s = B[r * N + c];
  } else {
    s = (r == c) ? 1.0 : 0.0;
  }
  const int i = r * N + c;
  double v = (r == c) ? e.cI : 0.0;
  if (e.s1 >= 0) v = fma(e.c1, ws[e.s1 * NN + i], v);
  if (e.s2 >= 0) v = fma(e.c2, ws[e.s2 * NN + i], v);
  if (e.s3 >= 0) v = fma(e.c3, ws[e.s3 * NN + i], v);
  ws[sc * NN + i] = e.alpha * s + v;
}

// F (leading dimension ldh) = the result slot; stat[0] = F[j-1][j]
__device__ __forceinline__ void expm_finish_entry(const double* __restrict__ P, int N, double* F, int ldh,
                                                  double* stat, long long i) {
  if (i < (long long)N * N) F[(i / N) * ldh + (i % N)] = P[i];
  if (i == 0) stat[0] = P[(N - 2) * N + (N - 1)];
}

}  // namespace swepi
