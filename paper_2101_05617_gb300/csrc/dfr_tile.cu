// Imaginary half of the split complex-step JVP (Eq. 28) in the complex64-bulk
// form, with each element tile staged in shared memory by bulk asynchronous
// copies (the Hopper/Blackwell copy engine: cp.async.bulk completing on an
// mbarrier).
//
// Per element tile, one thread issues the one-dimensional copies of everything the
// tile's nodes read -- the Krylov vector v (its FP32 copy when the solver keeps
// one, else FP64), the FP32 linearisation
// coefficients, the FP32 interface fluxes of the tile's elements (written by
// the face kernel), the FP32 b-column copies of the augmented operator and the
// FP64 orthogonalisation window vectors -- so that all of a tile's HBM traffic
// is in flight at once; the threads then compute from shared memory exactly
// what volume_tangent_body computes (pointwise imaginary fluxes and sources,
// the DFR sweeps of Eq. 12-14, the augmented operator, the window dots of the
// incomplete orthogonalisation) and share its epilogue.
//
// The copies need 16-byte aligned addresses and sizes: a tile holds EPB
// elements with EPB (p+1)^2 a multiple of four, and the launcher falls back to
// the register-and-cache kernel (dfr_split.cu) when the grid or a pointer does
// not satisfy this.  Two persistent CTAs per SM loop over the tiles with two
// stages, so the copies of a CTA's next tile are in flight while it computes the
// current one.  The waits on the mbarriers are bounded: after ~2 s the CTA sets
// the context's flag (reported as SW_ETIMEOUT by the phi-function solver),
// waits once more with the same bound for its own copies, leaves its tile loop,
// takes part in the epilogue's reduction with zero contributions and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "dfr_tangent.cuh"
#include "kiops_dev.h"
#include "swepi_internal.h"

namespace swepi {

namespace {

constexpr int KMAXB = kTileMaxB;   // b-column vectors staged per tile (EPI orders up to 6 use p <= 4)

constexpr int tile_epb(int nn) {
  int e = (256 / nn) > 0 ? (256 / nn) : 1;
  while (e > 1 && (e * nn) % 4 != 0) --e;
  return e;
}

template <int NS>
struct TileShape {
  static constexpr int NN = NS * NS;
  static constexpr int EPB = tile_epb(NN);
  static constexpr int TN = EPB * NN;   // nodes (threads) per tile
};

constexpr size_t up16(size_t b) { return (b + 15) / 16 * 16; }

// byte offsets of the regions of the dynamic shared memory: two stages of the
// staged operands of one tile, then the scratch of the tile being computed.
// DOTS: the stages hold the three FP64 window vectors of the orthogonalisation
// dots; without them (the dots in a pass of their own) a stage is about two
// thirds of the size and three CTAs fit on an SM.
template <int NS, bool DOTS = true>
struct TileLayout {
  static constexpr int TN = TileShape<NS>::TN, EPB = TileShape<NS>::EPB, NN = NS * NS;
  // one stage
  static constexpr size_t v = 0;                                            // double [3][TN]
  static constexpr size_t dots = v + up16(sizeof(double) * 3 * TN);         // double [3 (C, A, B)][3][TN]
  static constexpr size_t ln = dots + (DOTS ? up16(sizeof(double) * 9 * TN) : 0);   // float [LN_COUNT][TN]
  static constexpr size_t b32 = ln + up16(sizeof(float) * LN_COUNT * TN);   // float [KMAXB][3][TN]
  static constexpr size_t fb = b32 + up16(sizeof(float) * KMAXB * 3 * TN);  // float [EPB][4][3][NS]
  static constexpr size_t stage = fb + up16(sizeof(float) * EPB * 12 * NS);
  // scratch and barriers after the two stages: the flux scratch twice (tile k
  // uses buffer k mod 2, so the next tile's fluxes can be written while slow
  // warps still read this tile's)
  static constexpr size_t flux = 2 * stage;                                 // float [2][EPB][2][3][NN]
  static constexpr size_t flux_bytes = up16(sizeof(float) * EPB * 6 * NN);
  static constexpr size_t dmat = flux + 2 * flux_bytes;                     // float [NS][NS + 3]
  static constexpr size_t mbar = dmat + up16(sizeof(float) * NS * (NS + 3)); // two mbarriers
  static constexpr size_t bytes = mbar + 16;
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(mbar))
               : "memory");
}

// wait for the phase of the mbarrier with the given parity to complete; false
// after ~2 s (or 2^26 polls)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, unsigned parity) {
  const unsigned m = smem_addr(mbar);
  const unsigned long long t0 = now_ns();
  for (unsigned it = 0; it < (1u << 26); ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(m), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255u) == 255u && now_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}

// checked build: every copy of a tile (tile0 .. tile0 + tn of the N solution
// points, whole elements) lies inside its arrays, starts on a 16-byte boundary
// and moves a multiple of 16 bytes
template <int NS, bool W3, bool DOTS>
__device__ __forceinline__ bool tile_copies_ok(const TanVolArgs<float>& a, long long tile0, int tn,
                                               const double* const dsrc[3]) {
  constexpr int NN = NS * NS;
  const long long N = a.nodes;
  if (tile0 < 0 || tn <= 0 || tn % NN != 0 || tile0 + tn > N || N != a.nelem * NN) return false;
  const AugEpilogue& ep = a.ep;
  auto al = [](const void* p) { return (reinterpret_cast<unsigned long long>(p) & 15ull) == 0ull; };
  const bool b16 = (sizeof(double) * tn) % 16 == 0 && (sizeof(float) * tn) % 16 == 0;
  bool ok = b16 && al(a.ln + tile0) && al(a.ln + N) && al(a.fb + tile0 / NN * 12 * NS) &&
            (sizeof(float) * (tn / NN) * 12 * NS) % 16 == 0;
  if (ep.v32) ok = ok && al(ep.v32 + tile0) && al(ep.v32 + N);
  else ok = ok && al(a.v + tile0) && al(a.v + N);
  for (int k = 0; k < 3; ++k)
    if (dsrc[k]) ok = ok && al(dsrc[k] + tile0) && al(dsrc[k] + N);
  for (int l = 0; l < ep.p && l < KMAXB; ++l)
    if (ep.b32[l]) ok = ok && al(ep.b32[l] + tile0) && al(ep.b32[l] + N);
  return ok;
}

// issue the bulk copies of tile `tile` into stage buffer `st` (one thread)
template <int NS, bool W3, bool DOTS>
__device__ __forceinline__ void issue_tile(const TanVolArgs<float>& a, long long tile, unsigned char* st,
                                           uint64_t* mbar) {
  using L = TileLayout<NS, DOTS>;
  constexpr int NN = NS * NS, EPB = TileShape<NS>::EPB, TN = TileShape<NS>::TN;
  const AugEpilogue& ep = a.ep;
  const long long N = a.nodes, tile0 = tile * TN;
  const int tn = (N - tile0) < TN ? (int)(N - tile0) : TN;
  const int ne = tn / NN;
  const unsigned bd = (unsigned)(sizeof(double) * tn), bf = (unsigned)(sizeof(float) * tn);
  const double* dsrc[3] = {(DOTS && W3) ? ep.dotC : nullptr, DOTS ? ep.dotA : nullptr, DOTS ? ep.dotB : nullptr};
  unsigned tx = 3 * (ep.v32 ? bf : bd) + LN_COUNT * bf + (unsigned)(sizeof(float) * ne * 12 * NS);
  for (int k = 0; k < 3; ++k)
    if (dsrc[k]) tx += 3 * bd;
  for (int l = 0; l < ep.p && l < KMAXB; ++l)
    if (ep.b32[l]) tx += 3 * bf;
  if (kChecked && !tile_copies_ok<NS, W3, DOTS>(a, tile0, tn, dsrc)) {
    // checked build: no copy from a range outside the arrays; the phase
    // completes without data and the tile's results are not valid
    check_fail(CHK_TILE_RANGE);
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mbar)) : "memory");
    return;
  }
  // the stage was last read through the generic proxy: order that before the copies
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(tx) : "memory");
  double* sv = reinterpret_cast<double*>(st + L::v);
  double* sdot = reinterpret_cast<double*>(st + L::dots);
  float* sln = reinterpret_cast<float*>(st + L::ln);
  float* sb32 = reinterpret_cast<float*>(st + L::b32);
  float* sfb = reinterpret_cast<float*>(st + L::fb);
  if (ep.v32) {   // v from its FP32 copy: [3][TN] floats in the same region
    float* svf = reinterpret_cast<float*>(st + L::v);
    for (int var = 0; var < 3; ++var) bulk_g2s(svf + var * TN, ep.v32 + tile0 + var * N, bf, mbar);
  } else {
    for (int var = 0; var < 3; ++var) bulk_g2s(sv + var * TN, a.v + tile0 + var * N, bd, mbar);
  }
  for (int k = 0; k < 3; ++k) {
    if (!dsrc[k]) continue;
    for (int var = 0; var < 3; ++var) bulk_g2s(sdot + (k * 3 + var) * TN, dsrc[k] + tile0 + var * N, bd, mbar);
  }
  for (int c = 0; c < LN_COUNT; ++c) bulk_g2s(sln + c * TN, a.ln + tile0 + c * N, bf, mbar);
  for (int l = 0; l < ep.p && l < KMAXB; ++l) {
    if (!ep.b32[l]) continue;
    for (int var = 0; var < 3; ++var) bulk_g2s(sb32 + (l * 3 + var) * TN, ep.b32[l] + tile0 + var * N, bf, mbar);
  }
  bulk_g2s(sfb, a.fb + tile * EPB * 12 * NS, (unsigned)(sizeof(float) * ne * 12 * NS), mbar);
}

// Persistent: CTA b takes tiles b, b + G, b + 2G, ... (G CTAs); stage s = k mod
// 2 holds its k-th tile, and once every thread is past tile k - 1 (the first
// barrier of tile k) that tile's stage takes tile k + 1's copies, so the copies
// of the next tile are in flight while the current one computes.  Two barriers
// per tile: after the stage has landed, after the fluxes are written.
// Each thread accumulates its window dots over all its tiles; one block
// reduction per CTA then feeds the shared epilogue.
template <int NS, bool W3, bool DOTS>
__device__ __forceinline__ void tile_body(const TanVolArgs<float>& a, const DfrConst& dc, int* err,
                                          unsigned char* sm) {
  using L = TileLayout<NS, DOTS>;
  constexpr int NN = NS * NS, TN = TileShape<NS>::TN;
  float (*sD)[NS + 3] = reinterpret_cast<float (*)[NS + 3]>(sm + L::dmat);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + L::mbar);

  const AugEpilogue& ep = a.ep;
  if (ep.skip && *ep.skip) return;
  const long long N = a.nodes;
  const long long ntiles = (N + TN - 1) / TN;
  const long long G = gridDim.x;
  const bool dA = DOTS && ep.dotA != nullptr, dB = DOTS && ep.dotB != nullptr, dC = DOTS && W3 && ep.dotC != nullptr;
  const bool f32v = ep.v32 != nullptr;

  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      const long long tile = blockIdx.x + s * G;
      if (tile < ntiles) issue_tile<NS, W3, DOTS>(a, tile, sm + s * L::stage, mbar + s);
    }
  }
  const double dscale = -dc.two_over_dx * ep.scale;
  for (int t = threadIdx.x; t < NS * (NS + 2); t += TN)
    sD[t / (NS + 2)][t % (NS + 2)] = f64_to_f32_bits(dscale * dc.D[t / (NS + 2)][t % (NS + 2)]);
  __shared__ float coef32[KMAXB];
  if (threadIdx.x < KMAXB) {
    const int l = threadIdx.x;
    coef32[l] = (l < ep.p && ep.b32[l]) ? f64_to_f32_bits(ep.tail_in[l]) : 0.f;
  }
  const float sc = f64_to_f32_bits(ep.scale);
  const int t = threadIdx.x;
  const int le = t / NN, node = t % NN, k2 = node / NS, k1 = node % NS;
  double da = 0.0, db = 0.0, dcc = 0.0, dab = 0.0, dbc = 0.0;
  const bool cd = DOTS && ep.cdot_out != nullptr;
  bool ok = true;
  int k = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += G, ++k) {
    const int s = k & 1;
    unsigned char* st = sm + s * L::stage;
    const double* sv = reinterpret_cast<const double*>(st + L::v);
    const float* svf = reinterpret_cast<const float*>(st + L::v);
    const double* sdot = reinterpret_cast<const double*>(st + L::dots);
    const float* sln = reinterpret_cast<const float*>(st + L::ln);
    const float* sb32 = reinterpret_cast<const float*>(st + L::b32);
    const float* sfb = reinterpret_cast<const float*>(st + L::fb);
    const long long tile0 = tile * TN;
    const int tn = (N - tile0) < TN ? (int)(N - tile0) : TN;
    bool got = ok && mbar_wait_bounded(mbar + s, (unsigned)((k >> 1) & 1));
    if (ok && !got) {
      atomicExch(err, 1);
      mbar_wait_bounded(mbar + s, (unsigned)((k >> 1) & 1));   // do not leave with copies still landing
    }
    // also orders the coefficient tables written above, and every thread is
    // done with tile k - 1: its stage takes tile k + 1's copies now
    ok = __syncthreads_and(got) != 0;
    if (!ok) break;
    if (threadIdx.x == 0 && k >= 1 && tile + G < ntiles)
      issue_tile<NS, W3, DOTS>(a, tile + G, sm + (s ^ 1) * L::stage, mbar + (s ^ 1));
    float (*sF)[2][3][NN] = reinterpret_cast<float (*)[2][3][NN]>(sm + L::flux + s * L::flux_bytes);
    const bool active = t < tn;
    float S1 = 0.f, S2 = 0.f;
    if (active) {
      float v0, v1, v2;
      if (f32v) {
        v0 = svf[t];
        v1 = svf[TN + t];
        v2 = svf[2 * TN + t];
      } else {
        v0 = f64_to_f32_bits(sv[t]);
        v1 = f64_to_f32_bits(sv[TN + t]);
        v2 = f64_to_f32_bits(sv[2 * TN + t]);
      }
      const float u1 = sln[LN_U1 * TN + t], u2 = sln[LN_U2 * TN + t];
      const float F11 = fmaf(2.f * u1, v1, sln[LN_A11 * TN + t] * v0);
      const float F12 = fmaf(u2, v1, fmaf(u1, v2, sln[LN_A12 * TN + t] * v0));
      const float F22 = fmaf(2.f * u2, v2, sln[LN_A22 * TN + t] * v0);
      S1 = fmaf(sln[LN_S11 * TN + t], v1, fmaf(sln[LN_S12 * TN + t], v2, sln[LN_S10 * TN + t] * v0));
      S2 = fmaf(sln[LN_S21 * TN + t], v1, fmaf(sln[LN_S22 * TN + t], v2, sln[LN_S20 * TN + t] * v0));
      sF[le][0][0][node] = v1;
      sF[le][0][1][node] = F11;
      sF[le][0][2][node] = F12;
      sF[le][1][0][node] = v2;
      sF[le][1][1][node] = F12;
      sF[le][1][2][node] = F22;
    }
    __syncthreads();
    if (active) {
      float Da[NS + 2], Db[NS + 2];
#pragma unroll
      for (int n = 0; n < NS + 2; ++n) {
        Da[n] = sD[k1][n];
        Db[n] = sD[k2][n];
      }
      const float src[3] = {0.f, S1, S2};
      const float* fbe = sfb + le * 12 * NS;   // [edge][mu][k] of this element
      const long long idx = tile0 + t;
#pragma unroll
      for (int mu = 0; mu < 3; ++mu) {
        float acc = (mu == 0) ? 0.f : sc * src[mu];
        acc = fmaf(Da[0], fbe[(0 * 3 + mu) * NS + k2], acc);
        acc = fmaf(Da[NS + 1], fbe[(1 * 3 + mu) * NS + k2], acc);
#pragma unroll
        for (int l = 0; l < NS; ++l) acc = fmaf(Da[l + 1], sF[le][0][mu][k2 * NS + l], acc);
        acc = fmaf(Db[0], fbe[(2 * 3 + mu) * NS + k1], acc);
        acc = fmaf(Db[NS + 1], fbe[(3 * 3 + mu) * NS + k1], acc);
#pragma unroll
        for (int l = 0; l < NS; ++l) acc = fmaf(Db[l + 1], sF[le][1][mu][l * NS + k1], acc);
#pragma unroll
        for (int l = 0; l < KMAXB; ++l)
          if (l < ep.p && ep.b32[l]) acc = fmaf(coef32[l], sb32[(l * 3 + mu) * TN + t], acc);
        const double o = f32_to_f64_bits(acc);
        a.out[idx + mu * N] = o;
        if (DOTS && dB) {
          const double vb = sdot[(2 * 3 + mu) * TN + t];
          db = fma(o, vb, db);
          if (dA) {
            const double va = sdot[(1 * 3 + mu) * TN + t];
            da = fma(o, va, da);
            if (cd) dab = fma(vb, va, dab);
          }
          if (dC) {
            const double vc = sdot[(0 * 3 + mu) * TN + t];
            dcc = fma(o, vc, dcc);
            if (cd) dbc = fma(vb, vc, dbc);
          }
        }
      }
    }
  }
  __syncthreads();   // every thread is done with the last tile's stage
  // a CTA that gave up contributes zeros; the reduction protocol still completes
  if (!ok) da = db = dcc = dab = dbc = 0.0;
  // the stage buffers are free after the last tile (every copy issued was
  // waited for; after a wait that gave up the call reports SW_ETIMEOUT and its
  // result is not used): the first one holds the reduction scratch (5 TN doubles)
  static_assert(5 * TN * sizeof(double) <= L::stage, "reduction scratch larger than a stage");
  epilogue_finish<TN, W3, true>(ep, da, db, dcc, blockIdx.x, gridDim.x, dab, dbc, reinterpret_cast<double*>(sm));
}

// CTAs of the persistent grid per SM: two with the window vectors staged, three without
template <bool DOTS>
constexpr int tile_ctas_per_sm() { return DOTS ? 2 : 3; }

template <int NS, bool W3, bool DOTS>
__global__ void __launch_bounds__(TileShape<NS>::TN, tile_ctas_per_sm<DOTS>()) volume_tangent_tile_f32_kernel(
    TanVolArgs<float> a, DfrConst dc, int* err) {
  extern __shared__ __align__(16) unsigned char sm[];
  pdl_wait();
  pdl_trigger();
  tile_body<NS, W3, DOTS>(a, dc, err, sm);
}

// the same for the device-driven solver: the iteration index and the augmented
// operator come from its device state
template <int NS, bool W3, bool DOTS>
__global__ void __launch_bounds__(TileShape<NS>::TN, tile_ctas_per_sm<DOTS>()) volume_tangent_tile_dev_kernel(
    const KDev* __restrict__ kd, KFix f, TanVolArgs<float> a0, DfrConst dc, int* err) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ TanVolArgs<float> a;
  if (threadIdx.x == 0) {
    a = a0;
    const int it = kd->it;
    a.v = f.V + (long long)it * f.ldv;
    a.out = f.V + (long long)(it + 1) * f.ldv;
    iter_epilogue_dev(a.ep, *kd, f, it, W3, true);
  }
  __syncthreads();
  tile_body<NS, W3, DOTS>(a, dc, err, sm);
}

template <int NS, bool W3, bool DEV, bool DOTS>
int set_tile_smem() {
  static bool configured = false;
  if (configured) return SW_OK;
  const int bytes = (int)TileLayout<NS, DOTS>::bytes;
  const cudaError_t e =
      DEV ? cudaFuncSetAttribute(volume_tangent_tile_dev_kernel<NS, W3, DOTS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
          : cudaFuncSetAttribute(volume_tangent_tile_f32_kernel<NS, W3, DOTS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return SW_ECUDA;
  configured = true;
  return SW_OK;
}

int persistent_ctas(const Ctx& c, long long tiles, int per_sm) {
  int sms = 0;   // per call: a process may hold contexts on GPUs of different sizes
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess || sms < 1) return -1;
  return (int)std::min<long long>(tiles, (long long)per_sm * sms);
}

template <int NS>
bool tile_eligible(const Ctx& c, const double* v, const double* out, const AugEpilogue& ep) {
  auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (c.nodes % 4 != 0 || ep.p > KMAXB || !al(v) || !al(c.d_lin_node32) || !al(c.d_fb)) return false;
  if (ep.v32 && !al(ep.v32)) return false;
  if ((ep.dotA && !al(ep.dotA)) || (ep.dotB && !al(ep.dotB)) || (ep.dotC && !al(ep.dotC))) return false;
  for (int l = 0; l < ep.p && l < MAX_NB; ++l) {
    if (ep.b[l] && !ep.b32[l]) return false;
    if (ep.b32[l] && !al(ep.b32[l])) return false;
  }
  (void)out;
  return true;
}

template <int NS, bool W3, bool DOTS>
int launch_tile(Ctx& c, const double* v, double* out, const AugEpilogue& ep, cudaStream_t s) {
  using L = TileLayout<NS, DOTS>;
  auto kernel = volume_tangent_tile_f32_kernel<NS, W3, DOTS>;
  if (int rc = set_tile_smem<NS, W3, false, DOTS>()) return rc;
  TanVolArgs<float> va{v, c.nodes, c.nelem, c.d_lin_node32, reinterpret_cast<const float*>(c.d_fb), out, ep};
  const long long tiles = (c.nodes + TileShape<NS>::TN - 1) / TileShape<NS>::TN;
  const int ctas = persistent_ctas(c, tiles, tile_ctas_per_sm<DOTS>());
  if (ctas < 0) return SW_ECUDA;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3(TileShape<NS>::TN);
  cfg.dynamicSmemBytes = L::bytes;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int* err = c.d_flags + 3;
  if (cudaLaunchKernelEx(&cfg, kernel, va, c.dc, err) != cudaSuccess) return SW_ECUDA;
  c.launches++;
  return SW_OK;
}

}  // namespace

// returns SW_OK after launching, 1 when the grid or a pointer is not eligible
// (the caller then launches the register-and-cache kernel)
template <int NS>
int launch_volume_tile_f32(Ctx& c, const double* v, double* out, const AugEpilogue& ep, cudaStream_t s) {
  if (!tile_eligible<NS>(c, v, out, ep)) return 1;
  if (!ep.dotB) return launch_tile<NS, false, false>(c, v, out, ep, s);   // the dots in a pass of their own
  return ep.dotC ? launch_tile<NS, true, true>(c, v, out, ep, s) : launch_tile<NS, false, true>(c, v, out, ep, s);
}

// the device-driven solver's form: the dots in a pass of their own, so the
// staged kernel without window vectors
template <int NS>
int capture_volume_tile_dev(Ctx& c, KDev* kd, const KFix& f, bool w3, cudaStream_t s) {
  (void)w3;
  // eligibility with the buffers every iteration uses (basis rows, their FP32
  // copies, the b-column copies)
  AugEpilogue ep;
  ep.p = 1;
  ep.v32 = f.V32;
  if (!f.V32 || !tile_eligible<NS>(c, f.V, f.V, ep)) return 1;
  if (f.b32 && (reinterpret_cast<uintptr_t>(f.b32) & 15u)) return 1;
  if ((f.n * sizeof(float)) % 16 != 0) return 1;
  using L = TileLayout<NS, false>;
  if (int rc = set_tile_smem<NS, false, true, false>()) return rc;
  TanVolArgs<float> va{nullptr, c.nodes, c.nelem, c.d_lin_node32, reinterpret_cast<const float*>(c.d_fb), nullptr,
                       AugEpilogue{}};
  const long long tiles = (c.nodes + TileShape<NS>::TN - 1) / TileShape<NS>::TN;
  const int ctas = persistent_ctas(c, tiles, tile_ctas_per_sm<false>());
  if (ctas < 0) return SW_ECUDA;
  int* err = c.d_flags + 3;
  volume_tangent_tile_dev_kernel<NS, false, false><<<ctas, TileShape<NS>::TN, L::bytes, s>>>(kd, f, va, c.dc, err);
  c.launches++;
  return cuda_status(cudaGetLastError());
}

template <int NS>
int prepare_dev() {
  return set_tile_smem<NS, false, true, false>();
}

int prepare_volume_tile_dev(const Ctx& c) {
  switch (c.ns) {
    case 1: return prepare_dev<1>();
    case 2: return prepare_dev<2>();
    case 3: return prepare_dev<3>();
    case 4: return prepare_dev<4>();
    case 5: return prepare_dev<5>();
    case 6: return prepare_dev<6>();
    case 7: return prepare_dev<7>();
    case 8: return prepare_dev<8>();
    default: return SW_EINVAL;
  }
}

template int capture_volume_tile_dev<1>(Ctx&, KDev*, const KFix&, bool, cudaStream_t);
template int capture_volume_tile_dev<2>(Ctx&, KDev*, const KFix&, bool, cudaStream_t);
template int capture_volume_tile_dev<3>(Ctx&, KDev*, const KFix&, bool, cudaStream_t);
template int capture_volume_tile_dev<4>(Ctx&, KDev*, const KFix&, bool, cudaStream_t);
template int capture_volume_tile_dev<5>(Ctx&, KDev*, const KFix&, bool, cudaStream_t);
template int capture_volume_tile_dev<6>(Ctx&, KDev*, const KFix&, bool, cudaStream_t);
template int capture_volume_tile_dev<7>(Ctx&, KDev*, const KFix&, bool, cudaStream_t);
template int capture_volume_tile_dev<8>(Ctx&, KDev*, const KFix&, bool, cudaStream_t);

template int launch_volume_tile_f32<1>(Ctx&, const double*, double*, const AugEpilogue&, cudaStream_t);
template int launch_volume_tile_f32<2>(Ctx&, const double*, double*, const AugEpilogue&, cudaStream_t);
template int launch_volume_tile_f32<3>(Ctx&, const double*, double*, const AugEpilogue&, cudaStream_t);
template int launch_volume_tile_f32<4>(Ctx&, const double*, double*, const AugEpilogue&, cudaStream_t);
template int launch_volume_tile_f32<5>(Ctx&, const double*, double*, const AugEpilogue&, cudaStream_t);
template int launch_volume_tile_f32<6>(Ctx&, const double*, double*, const AugEpilogue&, cudaStream_t);
template int launch_volume_tile_f32<7>(Ctx&, const double*, double*, const AugEpilogue&, cudaStream_t);
template int launch_volume_tile_f32<8>(Ctx&, const double*, double*, const AugEpilogue&, cudaStream_t);

// this translation unit's check word (bounds-checked builds; sw_check_status)
SW_CHECK_READER(check_word_tile)

}  // namespace swepi
