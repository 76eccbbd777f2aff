// Device-side building blocks shared by the DFR kernels: the complex-step
// number type, state loads, the AUSM interface flux (App. D/E) and the trace
// extrapolation (Eq. 7 at the element ends).  See dfr.cu for the arithmetic
// conventions of the complex step.
#pragma once

#include <cuda_runtime.h>

#include "swepi_internal.h"

namespace swepi {

struct cs {
  double re, im;
};
__device__ __forceinline__ cs operator+(cs a, cs b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cs operator-(cs a, cs b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cs operator*(cs a, cs b) { return {a.re * b.re, fma(a.re, b.im, a.im * b.re)}; }
__device__ __forceinline__ cs operator*(double k, cs a) { return {k * a.re, k * a.im}; }
__device__ __forceinline__ cs operator+(cs a, double k) { return {a.re + k, a.im}; }
__device__ __forceinline__ cs cs_rcp(cs a) {
  double r = 1.0 / a.re;
  return {r, -a.im * r * r};
}
__device__ __forceinline__ cs cs_div(cs a, cs b) {
  double r = 1.0 / b.re;
  double qr = a.re * r;
  return {qr, (a.im - qr * b.im) * r};
}
__device__ __forceinline__ cs cs_sqrt(cs a) {
  double s = sqrt(a.re);
  return {s, a.im * (0.5 / s)};
}
__device__ __forceinline__ double re(cs a) { return a.re; }
__device__ __forceinline__ double im(cs a) { return a.im; }
__device__ __forceinline__ cs mk(double r, double i, cs*) { return {r, i}; }

// real instantiation (the RHS): same code path on plain doubles
__device__ __forceinline__ double cs_rcp(double a) { return 1.0 / a; }
__device__ __forceinline__ double cs_div(double a, double b) { return a / b; }
__device__ __forceinline__ double cs_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ double re(double a) { return a; }
__device__ __forceinline__ double im(double) { return 0.0; }
__device__ __forceinline__ double mk(double r, double, double*) { return r; }

// the part of a result the caller wants: the imaginary part for the JVP, the
// value for the RHS
__device__ __forceinline__ double part(cs a) { return a.im; }
__device__ __forceinline__ double part(double a) { return a; }

template <typename T>
__device__ __forceinline__ T load_state(const double* __restrict__ q, const double* __restrict__ v, double eps,
                                        long long i) {
  return mk(__ldg(q + i), v ? eps * __ldg(v + i) : 0.0, (T*)nullptr);
}

// ---------------------------------------------------------------- AUSM
// basic AUSM splittings (reading of App. D Eq. 138-139; [41] Eq. 6 and 8)
template <typename T>
__device__ __forceinline__ void ausm_side(const T q[3], int d, double ad, double p1, double p2, T& M, T A[3], T P[3]) {
  T a = cs_sqrt(ad * q[0]);                       // a^d = sqrt(h^dd g_r H), App. E
  T u = cs_div(q[d], q[0]);                       // u^d
  M = cs_div(u, a);                               // Froude number
  A[0] = a * q[0];                                // A^{mu d} = a q^mu
  A[1] = a * q[1];
  A[2] = a * q[2];
  T q0sq = q[0] * q[0];
  P[0] = 0.0 * q[0];
  P[1] = p1 * q0sq;                               // P^{mu d} = g_r h^{mu d} (q^0)^2 / (2 sqrt g)
  P[2] = p2 * q0sq;
}

template <typename T>
__device__ __forceinline__ void ausm_flux(const T qL[3], const T qR[3], int d, double ad, double p1, double p2,
                                          T flux[3]) {
  T ML, MR, AL[3], AR[3], PL[3], PR[3];
  ausm_side(qL, d, ad, p1, p2, ML, AL, PL);
  ausm_side(qR, d, ad, p1, p2, MR, AR, PR);
  // M+(M_L), beta+(M_L)
  T mp, bp, mm, bm;
  if (fabs(re(ML)) <= 1.0) {
    T t = ML + 1.0;
    mp = 0.25 * (t * t);
    bp = (0.25 * (t * t)) * (2.0 * mk(1.0, 0.0, (T*)nullptr) - ML);
  } else if (re(ML) > 0.0) {
    mp = ML;
    bp = mk(1.0, 0.0, (T*)nullptr);
  } else {
    mp = 0.0 * ML;
    bp = 0.0 * ML;
  }
  // M-(M_R), beta-(M_R)
  if (fabs(re(MR)) <= 1.0) {
    T t = MR + (-1.0);
    mm = -0.25 * (t * t);
    bm = (0.25 * (t * t)) * (MR + 2.0);
  } else if (re(MR) > 0.0) {
    mm = 0.0 * MR;
    bm = 0.0 * MR;
  } else {
    mm = MR;
    bm = mk(1.0, 0.0, (T*)nullptr);
  }
  T Mh = mp + mm;
  bool pos = re(Mh) > 0.0;
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    T adv = pos ? Mh * AL[mu] : Mh * AR[mu];
    flux[mu] = (adv + bp * PL[mu]) + bm * PR[mu];
  }
}

template <typename T, int NS>
__device__ __forceinline__ void trace(const double* __restrict__ q, const double* __restrict__ v, double eps,
                                      long long nodes, int elem, int edge, int i, const DfrConst& dc, T out[3]) {
  const long long base = (long long)elem * NS * NS;
  const double* w = (edge == 0 || edge == 2) ? dc.lm : dc.lp;
#pragma unroll
  for (int var = 0; var < 3; ++var) {
    T acc = mk(0.0, 0.0, (T*)nullptr);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      long long idx = base + ((edge <= 1) ? (i * NS + k) : (k * NS + i)) + var * nodes;
      acc = acc + w[k] * load_state<T>(q, v, eps, idx);
    }
    out[var] = acc;
  }
}

template <int NS>
struct VolShape {
  static constexpr int EPB = (256 / (NS * NS)) > 0 ? (256 / (NS * NS)) : 1;
  static constexpr int THREADS = EPB * NS * NS;
};


template <int THREADS, bool W3, bool CD>
__device__ __forceinline__ void epilogue_finish(const AugEpilogue& ep, double da, double db, double dcc,
                                                unsigned int blk, unsigned int nblk, double dab, double dbc,
                                                double* sbuf);

// Epilogue of the volume kernels (all threads of the block call it; blk/nblk:
// this block's index and the number of blocks working on the same vector):
// out = scale * res + nu * sum_l y_l b_{p-l} (the augmented operator of the
// phi-function solver), the shift of the augmented tail, and -- when dotB is
// set -- the window dot products of the incomplete orthogonalisation (two or
// three vectors; see AugEpilogue).
// SCALED: the caller has already multiplied res by scale.  W3: compiled for
// the window of three (dotC may be set); W3 = false drops that code.  B64:
// the b-column terms are added here in FP64; false: the caller has added them
// already (the FP32 kernels of the complex64-bulk form, from ep.b32).  CD:
// compiled to form the V . V products when ep.cdot_out asks for them (the
// complex64-bulk kernels); without it the block sums carry three values.
// the tail coefficients nu * y_l of the augmented operator into coef[MAX_NB]
// (shared memory; the caller synchronises before reading them)
__device__ __forceinline__ void epilogue_coefs(const AugEpilogue& ep, double* coef) {
  if (threadIdx.x < MAX_NB) {
    const int l = threadIdx.x;
    coef[l] = (l < ep.p && ep.b[l]) ? ep.nu * ep.tail_in[l] : 0.0;
  }
}

// Per-node half of the volume epilogue: o = res + sum_l coef_l b_l (B64),
// stored at out, and this node's terms of the window dots added to the
// thread's partial sums (da = z . V_{j-1}, db = z . V_j, dcc = z . V_{j-2},
// and with CD the V . V products dab, dbc).
template <bool W3, bool B64, bool CD>
__device__ __forceinline__ void epilogue_node(const AugEpilogue& ep, const double* coef, long long idx, long long N,
                                              const double res[3], double* __restrict__ out, double& da, double& db,
                                              double& dcc, double& dab, double& dbc) {
  double ob[3] = {res[0], res[1], res[2]};
  // a loop over the p columns, not an unrolled one over MAX_NB with a guard:
  // guarded-off FP64 instructions still take the FP64 pipe's issue slots
  if (B64) {
    const int p = ep.p < MAX_NB ? ep.p : MAX_NB;
#pragma unroll 1
    for (int l = 0; l < p; ++l) {
      const double* bl = ep.b[l];
      if (!bl) continue;
      const double cl = coef[l];
#pragma unroll
      for (int mu = 0; mu < 3; ++mu) ob[mu] = fma(cl, bl[idx + mu * N], ob[mu]);
    }
  }
  const bool cd = CD && ep.cdot_out != nullptr;
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    const double o = ob[mu];
    out[idx + mu * N] = o;
    if (ep.dotB) {
      const double vb = ep.dotB[idx + mu * N];
      db = fma(o, vb, db);
      if (ep.dotA) {
        const double va = ep.dotA[idx + mu * N];
        da = fma(o, va, da);
        if (cd) dab = fma(vb, va, dab);
      }
      if (W3 && ep.dotC) {
        const double vc = ep.dotC[idx + mu * N];
        dcc = fma(o, vc, dcc);
        if (cd) dbc = fma(vb, vc, dbc);
      }
    }
  }
}

template <int THREADS, bool SCALED = false, bool W3 = false, bool B64 = true, bool CD = false>
__device__ __forceinline__ void volume_epilogue(const AugEpilogue& ep, bool active, long long idx, long long N,
                                                const double res[3], double* __restrict__ out, unsigned int blk,
                                                unsigned int nblk) {
  __shared__ double coef[MAX_NB];
  if (B64) epilogue_coefs(ep, coef);
  __syncthreads();
  double da = 0.0, db = 0.0, dcc = 0.0, dab = 0.0, dbc = 0.0;
  if (active) {
    double r[3];
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) r[mu] = SCALED ? res[mu] : ep.scale * res[mu];
    epilogue_node<W3, B64, CD>(ep, coef, idx, N, r, out, da, db, dcc, dab, dbc);
  }
  __shared__ double sred[(CD ? 5 : 3) * THREADS];
  epilogue_finish<THREADS, W3, CD>(ep, da, db, dcc, blk, nblk, dab, dbc, sred);
}

// Sums of K values over the block in a fixed order, through shared scratch of
// K * THREADS doubles: every thread stores its values, warp k sums value k with
// a stride of 32 and a shuffle tree; the results are valid in thread 0.  (On
// this GPU a shuffle tree in every warp would cost each thread 5 K FP64 adds,
// more than the dots themselves.)
template <int THREADS, int K>
__device__ __forceinline__ void block_sums(double v[K], double* sbuf) {
  static_assert(THREADS >= 32 * K, "one warp per value");
  __shared__ double res[K];
#pragma unroll
  for (int k = 0; k < K; ++k) sbuf[k * THREADS + threadIdx.x] = v[k];
  __syncthreads();
  // warp k sums value k (a stride of 32, then a shuffle tree): the K sums run
  // side by side on the SM's schedulers, each in the order one warp gave it
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < K) {
    double a = 0.0;
    for (int i = lane; i < THREADS; i += 32) a += sbuf[w * THREADS + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) res[w] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = res[k];
  }
}

// Second half of the volume epilogue (all threads of the block call it, with
// their partial window dots da = z . V_{j-1}, db = z . V_j, dcc = z . V_{j-2}
// over their nodes, and -- when ep.cdot_out is set -- dab = V_j . V_{j-1} and
// dbc = V_j . V_{j-2}): the shift of the augmented tail, the tail's share of
// the dots, the block sums and -- in the last block to finish -- the modified
// Gram-Schmidt coefficients (with the V . V products of this launch when they
// are formed here, else those stored by the scale pass).  sbuf: K * THREADS
// doubles of shared scratch, K = 5 with CD, else 3.
template <int THREADS, bool W3, bool CD>
__device__ __forceinline__ void epilogue_finish(const AugEpilogue& ep, double da, double db, double dcc,
                                                unsigned int blk, unsigned int nblk, double dab, double dbc,
                                                double* sbuf) {
  if (ep.tail_out && blk == 0 && threadIdx.x < ep.p)
    ep.tail_out[threadIdx.x] = (threadIdx.x + 1 < ep.p) ? ep.tail_in[threadIdx.x + 1] : 0.0;
  if (!ep.dotB) return;   // uniform over the grid
  const bool cd = CD && ep.cdot_out != nullptr;   // uniform over the grid
  if (blk == 0 && threadIdx.x == 0) {
    for (int l = 0; l < ep.p; ++l) {
      const double zt = (l + 1 < ep.p) ? ep.tail_in[l + 1] : 0.0;
      db = fma(zt, ep.dotB[ep.n + l], db);
      if (ep.dotA) da = fma(zt, ep.dotA[ep.n + l], da);
      if (W3 && ep.dotC) dcc = fma(zt, ep.dotC[ep.n + l], dcc);
      if (cd && ep.dotA) dab = fma(ep.tail_in[l], ep.dotA[ep.n + l], dab);
      if (cd && W3 && ep.dotC) dbc = fma(ep.tail_in[l], ep.dotC[ep.n + l], dbc);
    }
  }
  constexpr int K = CD ? 5 : 3;
  __shared__ bool last;
  double v[5] = {da, db, dcc, dab, dbc};
  block_sums<THREADS, K>(v, sbuf);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) ep.dpart[K * blk + k] = v[k];
    __threadfence();
    const unsigned int t = atomicAdd(ep.dticket, 1u);
    last = (t == nblk - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double u[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int k = threadIdx.x; k < (int)nblk; k += THREADS) {
#pragma unroll
    for (int i = 0; i < K; ++i) u[i] += __ldcg(ep.dpart + K * k + i);
  }
  __syncthreads();   // the scratch is reused
  block_sums<THREADS, K>(u, sbuf);
  if (threadIdx.x == 0) {
    const double a = u[0], b = u[1], c3 = u[2];
    const bool three = W3 && ep.dotC != nullptr;
    double cprev = 0.0, cprevC = 0.0;
    if (ep.dotA) {
      cprev = cd ? u[3] : *ep.cprev;
      if (cd) *ep.cdot_out = u[3];   // V_j . V_{j-1}
    }
    if (three) {
      cprevC = cd ? u[4] : *ep.cprevC;
      if (cd) *ep.cdot2_out = u[4];   // V_j . V_{j-2}
    }
    // modified Gram-Schmidt coefficients, oldest vector first
    if (three) {
      const double h0 = c3;                               // V_{j-2} . z
      const double h1 = a - h0 * (*ep.cprevAC);            // V_{j-1} . (z - h0 V_{j-2})
      *ep.h0_out = h0;
      *ep.h1_out = h1;
      *ep.h2_out = b - h0 * cprevC - h1 * cprev;
    } else if (ep.dotA) {
      *ep.h1_out = a;
      *ep.h2_out = b - a * cprev;   // V_j . (z - h1 V_{j-1})
    } else {
      *ep.h2_out = b;
    }
    *ep.dticket = 0u;
  }
}

}  // namespace swepi
