// State of the device-driven phi-function solver (kiops_graph.cu): the
// controller and loop variables live in device memory, so that one CUDA graph
// with conditional WHILE nodes (substep attempts, Krylov iterations,
// squarings of the exponential) runs a whole call of Eq. (29) without a host
// round trip.  KDev is written by the host before each launch and read back
// after it; KFix holds the context's fixed buffers (kernel parameters).
#pragma once

#include "kiops_ctl.h"
#include "swepi_internal.h"

namespace swepi {

constexpr int kDevMaxAttempts = 2000;    // substep attempts per call (then SW_EKRYLOV)
constexpr int kDevMaxSquarings = 200;    // squarings of one exponential, the host driver's bound (then SW_ENONFINITE)
constexpr int kTileMaxB = 4;             // b-column vectors the staged complex64-bulk volume kernel takes

struct KDev {
  KiopsController K;
  // the call (uploaded by the host)
  double dt = 0.0, tau_end = 1.0, tol = 1e-10, tau0 = 1.0;
  int p = 1, m0 = 10, m_min = 10, m_max = 128;
  const double* b[MAX_NB] = {};   // b-column vectors in the augmented operator's order (b_p .. b_1)
  const float* b32[MAX_NB] = {};  // their FP32 copies (complex64-bulk form)
  // computed on the device
  double nu = 1.0, mu = 1.0, normb = 0.0, beta0 = 0.0;
  int it = 0, m_cur = 0, skip0 = 0, accept = 0, err = 0, attempts = 0;
  int N = 0, sq = 0, sq_i = 0, pad = 0;
};

struct KFix {
  double* V;          // Krylov basis [vcap][ldv]
  float* V32;         // its FP32 copy (complex64-bulk form) or null
  float* b32;         // FP32 b-column buffer [p][n] (complex64-bulk form) or null
  long long ldv, n, N;   // leading dimension, unknowns, augmented length n + p
  double* H;
  int ldh;
  double* F;
  double* X;
  int* flags;
  double* scal;
  double* cdot;
  double* cdot2;
  double* vpart;
  double* partials;
  double* ws;         // exponential workspace
};

#ifdef __CUDACC__
// the augmented-operator epilogue of Krylov iteration `it`, exactly as the
// host driver (kiops.cu) sets it
__device__ __forceinline__ void iter_epilogue_dev(AugEpilogue& ep, const KDev& kd, const KFix& f, int it, bool w3,
                                                  bool fp32) {
  ep.scale = kd.dt;
  ep.nu = kd.nu;
  ep.p = kd.p;
  for (int l = 0; l < MAX_NB; ++l) {
    ep.b[l] = kd.b[l];
    ep.b32[l] = fp32 ? kd.b32[l] : nullptr;
  }
  const double* Vi = f.V + (long long)it * f.ldv;
  double* Vn = f.V + (long long)(it + 1) * f.ldv;
  ep.tail_in = Vi + f.n;
  ep.tail_out = Vn + f.n;
  ep.skip = f.flags;
  // complex64-bulk form (FP32 basis copy): the dots in a pass of their own
  const bool sep = fp32 && f.V32;
  ep.dotA = (!sep && it >= 1) ? Vi - f.ldv : nullptr;
  ep.dotB = sep ? nullptr : Vi;
  ep.dotC = (!sep && w3 && it >= 2) ? Vi - 2 * f.ldv : nullptr;
  ep.cprev = f.cdot + it;
  ep.cprevC = f.cdot2 + it;
  ep.cprevAC = (it >= 1) ? f.cdot + it - 1 : nullptr;
  ep.h0_out = (w3 && it >= 2) ? f.H + (long long)(it - 2) * f.ldh + it : nullptr;
  ep.h1_out = (it >= 1) ? f.H + (long long)(it - 1) * f.ldh + it : nullptr;
  ep.h2_out = f.H + (long long)it * f.ldh + it;
  ep.dpart = f.vpart;
  ep.dticket = reinterpret_cast<unsigned int*>(f.flags + 9);
  ep.n = f.n;
  ep.v32 = sep ? f.V32 + (long long)it * f.ldv : nullptr;
  ep.cdot_out = ep.cdot2_out = nullptr;
}
#endif

// captures the face and volume kernels of one Krylov iteration (the iteration
// index read from kd on the device) on stream s (dfr_split.cu)
int capture_iter_jvp(Ctx& c, KDev* kd, const KFix& f, bool fp32, bool w3, int p, cudaStream_t s);
// the staged complex64-bulk volume kernel in that form (dfr_tile.cu); 1 when
// the context's buffers are not eligible
template <int NS>
int capture_volume_tile_dev(Ctx& c, KDev* kd, const KFix& f, bool w3, cudaStream_t s);
// function attributes of that kernel, set before any stream capture (dfr_tile.cu)
int prepare_volume_tile_dev(const Ctx& c);
// the grid-size queries of the persistent volume kernels in that form, run
// before any stream capture (dfr_split.cu)
int prepare_volume_dev(const Ctx& c, bool fp32);

}  // namespace swepi
