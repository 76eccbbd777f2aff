// Imaginary half of the split complex-step JVP (see dfr_split.cu): device
// bodies shared by the single-grid kernels (dfr_split.cu) and the batched
// ensemble kernels (ensemble.cu).
#pragma once

#include <cuda_runtime.h>

#include "check.cuh"
#include "convert.cuh"
#include "dfr_device.cuh"
#include "swepi_internal.h"

namespace swepi {

// ---------------------------------------------------------------- tangent
// The imaginary half in arithmetic type T: double (the FP64 path) or float
// (the complex64-bulk form: tables rounded from the FP64 linearisation, FP32
// accumulation).  Krylov vectors in and out stay FP64; the orthogonalisation
// dots of the epilogue are FP64 in both.
//
template <typename T, int NS>
__device__ __forceinline__ void trace_tan(const double* __restrict__ v, const float* __restrict__ v32, long long nodes,
                                          int elem, int edge, int i, const DfrConst& dc, T out[3]) {
  const long long base = (long long)elem * NS * NS;
  const double* w = (edge == 0 || edge == 2) ? dc.lm : dc.lp;
  const float* w32 = (edge == 0 || edge == 2) ? dc.lm32 : dc.lp32;
#pragma unroll
  for (int var = 0; var < 3; ++var) {
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const long long idx = base + ((edge <= 1) ? (i * NS + k) : (k * NS + i)) + var * nodes;
      if constexpr (sizeof(T) == 4) {
        const float x = v32 ? __ldg(v32 + idx) : f64_to_f32_bits(__ldg(v + idx));
        acc = fmaf(w32[k], x, acc);
      } else {
        acc = fma(w[k], __ldg(v + idx), acc);
      }
    }
    out[var] = acc;
  }
}

template <typename T>
struct TanFaceArgs {
  const double* v;
  const float* v32;   // FP32 copy of v (complex64-bulk form), or null
  long long nodes;
  const FaceLine* lines;
  const double* fc;
  const T* lf;
  long long nfacepts;
  T* fb;
  const int* skip;
};

// imaginary half at interface point t of one grid
template <typename T, int NS>
__device__ __forceinline__ void face_tangent_body(const TanFaceArgs<T>& a, const DfrConst& dc, long long t) {
  if (t >= a.nfacepts) return;
  const int line = (int)(t / NS), i = (int)(t % NS);
  const FaceLine L = a.lines[line];
  if (!face_line_ok<NS>(L, a.nodes)) return;
  const int in = L.reversed ? NS - 1 - i : i;
  T vo[3], vn[3];
  trace_tan<T, NS>(a.v, a.v32, a.nodes, L.owner, L.owner_edge, i, dc, vo);
  trace_tan<T, NS>(a.v, a.v32, a.nodes, L.nbr, L.nbr_edge, in, dc, vn);
  const long long P = a.nfacepts;
  const T* lf = a.lf + t;
  T f[3];
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    T s = lf[(mu * 3) * P] * vo[0];
    s = fma(lf[(mu * 3 + 1) * P], vo[1], s);
    s = fma(lf[(mu * 3 + 2) * P], vo[2], s);
    s = fma(lf[(9 + mu * 3) * P], vn[0], s);
    s = fma(lf[(9 + mu * 3 + 1) * P], vn[1], s);
    s = fma(lf[(9 + mu * 3 + 2) * P], vn[2], s);
    f[mu] = s;
  }
  T sig, M00, M01, M10, M11;
  if constexpr (sizeof(T) == 4) {   // FP32 copies of the hand-back coefficients after the 18 map rows
    M00 = lf[18 * P];
    M01 = lf[19 * P];
    M10 = lf[20 * P];
    M11 = lf[21 * P];
    sig = lf[22 * P];
  } else {
    const double* fc = a.fc + t;
    sig = fc[FC_SIG * P];
    M00 = fc[FC_M00 * P];
    M01 = fc[FC_M01 * P];
    M10 = fc[FC_M10 * P];
    M11 = fc[FC_M11 * P];
  }
  T* fo = a.fb + ((long long)L.owner * 4 + L.owner_edge) * 3 * NS + i;
  fo[0] = f[0];
  fo[NS] = f[1];
  fo[2 * NS] = f[2];
  T* fn = a.fb + ((long long)L.nbr * 4 + L.nbr_edge) * 3 * NS + in;
  fn[0] = sig * f[0];
  fn[NS] = M00 * f[1] + M01 * f[2];
  fn[2 * NS] = M10 * f[1] + M11 * f[2];
}

template <typename T>
struct TanVolArgs {
  const double* v;
  long long nodes;
  long long nelem;
  const T* ln;
  const T* fb;
  double* out;
  AugEpilogue ep;
};

// shared memory of one element tile
template <typename T, int NS, int EPB>
struct VolSmem {
  T sF[EPB][2][3][NS * NS];   // fluxes along xi^1 and xi^2
  T sB[EPB][4][3][NS];        // interface fluxes of the four edges
  T sD[NS][NS + 3];           // derivative matrix, padded rows: distinct banks per k
};

// derivative matrix pre-multiplied by -(2/dx) * scale (Eq. 14 and the
// augmented operator's dt) into shared memory: each output is then one chain
// of fused multiply-adds started from scale * source
template <typename T, int NS, int EPB, int BLOCK>
__device__ __forceinline__ void tile_dmat(const TanVolArgs<T>& a, const DfrConst& dc, VolSmem<T, NS, EPB>& sm) {
  const double dscale = -dc.two_over_dx * a.ep.scale;
  for (int t = threadIdx.x; t < NS * (NS + 2); t += BLOCK)
    sm.sD[t / (NS + 2)][t % (NS + 2)] = from_f64<T>(dscale * dc.D[t / (NS + 2)][t % (NS + 2)]);
}

// interface fluxes of the four edges of the elements eb .. eb + EPB - 1 (those
// below e_end) into shared memory
template <typename T, int NS, int EPB, int BLOCK>
__device__ __forceinline__ void tile_edges(const TanVolArgs<T>& a, VolSmem<T, NS, EPB>& sm, long long eb,
                                           long long e_end) {
  for (int t = threadIdx.x; t < EPB * 12 * NS; t += BLOCK) {
    const int e = t / (12 * NS), r = t % (12 * NS);
    const long long ge = eb + e;
    (&sm.sB[e][0][0][0])[r] = (ge < e_end) ? a.fb[ge * 12 * NS + r] : T(0);
  }
}

// pointwise imaginary fluxes of node idx (element le of the tile, node
// `node`) into shared memory; the sources S^1, S^2 returned
template <typename T, int NS, int EPB>
__device__ __forceinline__ void tile_fluxes(const TanVolArgs<T>& a, VolSmem<T, NS, EPB>& sm, int le, int node,
                                            long long idx, T& S1, T& S2) {
  const long long N = a.nodes;
  const T v0 = from_f64<T>(__ldg(a.v + idx)), v1 = from_f64<T>(__ldg(a.v + idx + N));
  const T v2 = from_f64<T>(__ldg(a.v + idx + 2 * N));
  const T* ln = a.ln + idx;
  const T u1 = ln[LN_U1 * N], u2 = ln[LN_U2 * N];
  const T F11 = fma(T(2) * u1, v1, ln[LN_A11 * N] * v0);
  const T F12 = fma(u2, v1, fma(u1, v2, ln[LN_A12 * N] * v0));
  const T F22 = fma(T(2) * u2, v2, ln[LN_A22 * N] * v0);
  S1 = fma(ln[LN_S11 * N], v1, fma(ln[LN_S12 * N], v2, ln[LN_S10 * N] * v0));
  S2 = fma(ln[LN_S21 * N], v1, fma(ln[LN_S22 * N], v2, ln[LN_S20 * N] * v0));
  sm.sF[le][0][0][node] = v1;
  sm.sF[le][0][1][node] = F11;
  sm.sF[le][0][2][node] = F12;
  sm.sF[le][1][0][node] = v2;
  sm.sF[le][1][1][node] = F12;
  sm.sF[le][1][2][node] = F22;
}

// the two DFR sweeps of one node (rows Da, Db of the scaled derivative
// matrix) started from sc * source; in the complex64-bulk form also the
// b-column terms nu y_l b_l in FP32 (coef32: the rounded nu y_l)
template <typename T, int NS, int EPB>
__device__ __forceinline__ void tile_sweep(const TanVolArgs<T>& a, const VolSmem<T, NS, EPB>& sm, int le, int k1,
                                           int k2, long long idx, const T (&Da)[NS + 2], const T (&Db)[NS + 2],
                                           T sc, T S1, T S2, const float* coef32, double res[3]) {
  const T src[3] = {T(0), S1, S2};
  T acc[3];
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    T c = (mu == 0) ? T(0) : sc * src[mu];
    c = fma(Da[0], sm.sB[le][0][mu][k2], c);
    c = fma(Da[NS + 1], sm.sB[le][1][mu][k2], c);
#pragma unroll
    for (int l = 0; l < NS; ++l) c = fma(Da[l + 1], sm.sF[le][0][mu][k2 * NS + l], c);
    c = fma(Db[0], sm.sB[le][2][mu][k1], c);
    c = fma(Db[NS + 1], sm.sB[le][3][mu][k1], c);
#pragma unroll
    for (int l = 0; l < NS; ++l) c = fma(Db[l + 1], sm.sF[le][1][mu][l * NS + k1], c);
    acc[mu] = c;
  }
  if constexpr (sizeof(T) == 4) {
    const long long N = a.nodes;
    const int p = a.ep.p < MAX_NB ? a.ep.p : MAX_NB;
#pragma unroll 1
    for (int l = 0; l < p; ++l) {
      const float* bl = a.ep.b32[l];
      if (!bl) continue;
#pragma unroll
      for (int mu = 0; mu < 3; ++mu) acc[mu] = fma(T(coef32[l]), T(__ldg(bl + idx + mu * N)), acc[mu]);
    }
  }
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) res[mu] = to_f64<T>(acc[mu]);
}

// the complex64-bulk form's FP32 tail coefficients nu * y_l (once per block)
template <typename T>
__device__ __forceinline__ void tile_coef32(const AugEpilogue& ep, float* coef32) {
  if (sizeof(T) == 4 && threadIdx.x < MAX_NB) {
    const int l = threadIdx.x;
    coef32[l] = (l < ep.p && ep.b32[l]) ? f64_to_f32_bits(ep.tail_in[l]) : 0.f;
  }
}

// imaginary half of EPB elements per block: block blk of nblk working on one
// grid; the block has BLOCK >= EPB * NS^2 threads (one per solution point, the
// rest idle), all of which call this function
template <typename T, int NS, int EPB, int BLOCK = EPB * NS * NS, bool W3 = false>
__device__ __forceinline__ void volume_tangent_body(const TanVolArgs<T>& a, const DfrConst& dc, unsigned int blk,
                                                    unsigned int nblk, VolSmem<T, NS, EPB>& sm) {
  constexpr int NN = NS * NS;
  static_assert(EPB * NN <= BLOCK, "block too small for the element tile");
  tile_dmat<T, NS, EPB, BLOCK>(a, dc, sm);
  const int le = threadIdx.x / NN, node = threadIdx.x % NN;
  const long long eb = (long long)blk * EPB;
  const long long elem = eb + le;
  const bool active = threadIdx.x < EPB * NN && elem < a.nelem;
  const int k2 = node / NS, k1 = node % NS;
  const long long idx = elem * NN + node;
  tile_edges<T, NS, EPB, BLOCK>(a, sm, eb, a.nelem);
  T S1 = T(0), S2 = T(0);
  if (active) tile_fluxes<T, NS, EPB>(a, sm, le, node, idx, S1, S2);
  constexpr bool F32 = sizeof(T) == 4;
  __shared__ float coef32[MAX_NB];
  tile_coef32<T>(a.ep, coef32);
  __syncthreads();
  double res[3] = {0.0, 0.0, 0.0};
  if (active) {
    // this thread's rows of the derivative matrix, from shared memory into registers
    // (a per-thread row index into the constant bank would serialise the warp)
    T Da[NS + 2], Db[NS + 2];
#pragma unroll
    for (int n = 0; n < NS + 2; ++n) {
      Da[n] = sm.sD[k1][n];
      Db[n] = sm.sD[k2][n];
    }
    tile_sweep<T, NS, EPB>(a, sm, le, k1, k2, idx, Da, Db, from_f64<T>(a.ep.scale), S1, S2, coef32, res);
  }
  volume_epilogue<BLOCK, true, W3, !F32, F32>(a.ep, active, idx, a.nodes, res, a.out, blk, nblk);
}

// The same imaginary half as a persistent grid: CTA b of the grid takes the
// elements [E b / G, E (b + 1) / G) (E elements, G CTAs) in tiles of EPB, adds
// its window-dot terms up across its tiles and reduces them once.  The even
// split keeps the last tiles from running on a few SMs alone; the single
// reduction per CTA saves the per-tile block sums (FP64 adds on the slow pipe).
template <typename T, int NS, int EPB, int BLOCK, bool W3>
__device__ __forceinline__ void volume_tangent_persistent(const TanVolArgs<T>& a, const DfrConst& dc,
                                                          VolSmem<T, NS, EPB>& sm) {
  constexpr int NN = NS * NS;
  constexpr bool F32 = sizeof(T) == 4;
  static_assert(EPB * NN <= BLOCK, "block too small for the element tile");
  const long long e0 = a.nelem * blockIdx.x / gridDim.x, e1 = a.nelem * (blockIdx.x + 1) / gridDim.x;
  tile_dmat<T, NS, EPB, BLOCK>(a, dc, sm);
  __shared__ double coef[MAX_NB];
  __shared__ float coef32[MAX_NB];
  if (!F32) epilogue_coefs(a.ep, coef);
  tile_coef32<T>(a.ep, coef32);
  __syncthreads();
  const int le = threadIdx.x / NN, node = threadIdx.x % NN;
  const int k2 = node / NS, k1 = node % NS;
  const bool lane_on = threadIdx.x < EPB * NN;
  T Da[NS + 2], Db[NS + 2];
#pragma unroll
  for (int n = 0; n < NS + 2; ++n) {
    Da[n] = lane_on ? sm.sD[k1][n] : T(0);
    Db[n] = lane_on ? sm.sD[k2][n] : T(0);
  }
  const T sc = from_f64<T>(a.ep.scale);
  double da = 0.0, db = 0.0, dcc = 0.0, dab = 0.0, dbc = 0.0;
  for (long long eb = e0; eb < e1; eb += EPB) {
    const long long elem = eb + le;
    const bool active = lane_on && elem < e1;
    const long long idx = elem * NN + node;
    __syncthreads();   // the previous tile's readers are done with sF and sB
    tile_edges<T, NS, EPB, BLOCK>(a, sm, eb, e1);
    T S1 = T(0), S2 = T(0);
    if (active) tile_fluxes<T, NS, EPB>(a, sm, le, node, idx, S1, S2);
    __syncthreads();
    if (active) {
      double res[3];
      tile_sweep<T, NS, EPB>(a, sm, le, k1, k2, idx, Da, Db, sc, S1, S2, coef32, res);
      epilogue_node<W3, !F32, F32>(a.ep, coef, idx, a.nodes, res, a.out, da, db, dcc, dab, dbc);
    }
  }
  __shared__ double sred[(F32 ? 5 : 3) * BLOCK];
  epilogue_finish<BLOCK, W3, F32>(a.ep, da, db, dcc, blockIdx.x, gridDim.x, dab, dbc, sred);
}

}  // namespace swepi
