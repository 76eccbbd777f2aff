// DFR right-hand side and complex-step Jacobian-vector product on sm_103a.
//
// F(q) (Eq. 1-2 discretised by Sec. 3) is evaluated in two kernels:
//   face_flux_kernel   one thread per interface point: traces of both sides
//                      (Eq. 7 at xi = +-1), the App. C transform of the
//                      neighbour state into the owner's coordinates, the AUSM
//                      flux (App. D/E) and its hand-back to the neighbour;
//                      results go to the per-element face-flux buffer.
//   volume_kernel      one thread per solution point, a block holds whole
//                      elements: pointwise fluxes and sources (Eq. 2, 136),
//                      tangent parts staged in shared memory, the extended-node
//                      derivative sweeps (Eq. 12-14) in both directions, and an
//                      epilogue that can fold the augmented-operator terms of the
//                      Krylov solver into the output.
//
// Complex-step arithmetic (Eq. 28).  The JVP evaluates F at q + i eps v.  With
// eps = 1e-30 every imaginary part is ~1e-25 of its real part or smaller, so the
// O(eps^2) cross terms of complex products, quotients and square roots lie far
// below FP64 rounding of the real parts; the `cs` type below carries a complex
// number as (real, imaginary) and evaluates each operation without those terms:
//   (a + ib)(c + id) -> ac + i(ad + bc)
//   (a + ib)/(c + id) -> a/c + i(b - (a/c) d)/c
//   sqrt(a + ib)      -> sqrt(a) + i b / (2 sqrt(a))   (principal root, a > 0)
// Real parts are therefore the FP64 evaluation of F(q) and imaginary parts the
// first-order term, equal to the full complex result up to rounding.  Branches
// (AUSM's |M| <= 1, max/min) test the real part, ties going to the <= 0 side.
#include <cuda_runtime.h>

#include "check.cuh"
#include "dfr_device.cuh"
#include "swepi_internal.h"

namespace swepi {

// ---------------------------------------------------------------- face flux
struct FaceArgs {
  const double* q;
  const double* v;
  double eps;
  long long nodes;
  const FaceLine* lines;
  const double* fc;
  long long nfacepts;
  double* fb;
  const int* skip;
};

template <typename T, int NS>
__global__ void __launch_bounds__(128) face_flux_kernel(FaceArgs a, DfrConst dc) {
  if (a.skip && *a.skip) return;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nfacepts) return;
  const int line = (int)(t / NS), i = (int)(t % NS);
  const FaceLine L = a.lines[line];
  if (!face_line_ok<NS>(L, a.nodes)) return;
  const int in = L.reversed ? NS - 1 - i : i;
  T qo[3], qn[3];
  trace<T, NS>(a.q, a.v, a.eps, a.nodes, L.owner, L.owner_edge, i, dc, qo);
  trace<T, NS>(a.q, a.v, a.eps, a.nodes, L.nbr, L.nbr_edge, in, dc, qn);
  const long long P = a.nfacepts;
  const double* fc = a.fc + t;
  const double T00 = fc[FC_T00 * P], T01 = fc[FC_T01 * P], T10 = fc[FC_T10 * P], T11 = fc[FC_T11 * P];
  T qt[3];
  qt[0] = qn[0];
  qt[1] = T00 * qn[1] + T01 * qn[2];
  qt[2] = T10 * qn[1] + T11 * qn[2];
  T fl[3];
  const double ad = fc[FC_AD * P], p1 = fc[FC_P1 * P], p2 = fc[FC_P2 * P];
  if (L.owner_is_left)
    ausm_flux<T>(qo, qt, L.dir, ad, p1, p2, fl);
  else
    ausm_flux<T>(qt, qo, L.dir, ad, p1, p2, fl);
  const double sig = fc[FC_SIG * P];
  const double M00 = fc[FC_M00 * P], M01 = fc[FC_M01 * P], M10 = fc[FC_M10 * P], M11 = fc[FC_M11 * P];
  double f0 = part(fl[0]), f1 = part(fl[1]), f2 = part(fl[2]);
  double* fo = a.fb + ((long long)L.owner * 4 + L.owner_edge) * 3 * NS + i;
  fo[0] = f0;
  fo[NS] = f1;
  fo[2 * NS] = f2;
  double* fn = a.fb + ((long long)L.nbr * 4 + L.nbr_edge) * 3 * NS + in;
  fn[0] = sig * f0;
  fn[NS] = M00 * f1 + M01 * f2;
  fn[2 * NS] = M10 * f1 + M11 * f2;
}

// ---------------------------------------------------------------- volume
struct VolArgs {
  const double* q;
  const double* v;
  double eps;
  long long nodes;
  long long nelem;
  const double* nc;
  const double* fb;
  double* out;
  AugEpilogue ep;
};

template <typename T, int NS, bool W3 = false>
__global__ void __launch_bounds__(VolShape<NS>::THREADS) volume_kernel(VolArgs a, DfrConst dc) {
  constexpr int EPB = VolShape<NS>::EPB;
  constexpr int NN = NS * NS;
  if (a.ep.skip && *a.ep.skip) return;
  __shared__ double sF[EPB][2][3][NN];       // [dir][mu][k2*NS+k1]
  __shared__ double sB[EPB][4][3][NS];       // face fluxes [edge][mu][pt]
  __shared__ double sD[NS][NS + 3];          // padded rows: distinct banks per k
  for (int t = threadIdx.x; t < NS * (NS + 2); t += blockDim.x) sD[t / (NS + 2)][t % (NS + 2)] = dc.D[t / (NS + 2)][t % (NS + 2)];
  const int le = threadIdx.x / NN, node = threadIdx.x % NN;
  const long long elem = (long long)blockIdx.x * EPB + le;
  const bool active = elem < a.nelem;
  const int k2 = node / NS, k1 = node % NS;
  const long long idx = elem * NN + node;

  // face fluxes of this block's elements
  for (int t = threadIdx.x; t < EPB * 12 * NS; t += blockDim.x) {
    int e = t / (12 * NS), r = t % (12 * NS);
    long long ge = (long long)blockIdx.x * EPB + e;
    (&sB[e][0][0][0])[r] = (ge < a.nelem) ? a.fb[ge * 12 * NS + r] : 0.0;
  }

  T S[3];
  if (active) {
    const long long N = a.nodes;
    T q0 = load_state<T>(a.q, a.v, a.eps, idx);
    T q1 = load_state<T>(a.q, a.v, a.eps, idx + N);
    T q2 = load_state<T>(a.q, a.v, a.eps, idx + 2 * N);
    const double* nc = a.nc + idx;
    T r = cs_rcp(q0);
    T u1 = q1 * r, u2 = q2 * r;
    T q0sq = q0 * q0;
    T F11 = q1 * u1 + nc[NC_C11 * N] * q0sq;     // sqrt(g) T^{mu nu}, Eq. (136)
    T F12 = q1 * u2 + nc[NC_C12 * N] * q0sq;
    T F22 = q2 * u2 + nc[NC_C22 * N] * q0sq;
    T q1u1 = q1 * u1, q1u2 = q1 * u2, q2u2 = q2 * u2;
    // sources of Eq. (2): Coriolis, metric (Gamma^i_jk), topography
    S[0] = mk(0.0, 0.0, (T*)nullptr);
    S[1] = (nc[NC_K11 * N] * q1 + nc[NC_K12 * N] * q2) - (nc[NC_G1A * N] * q1u1 + nc[NC_G1B * N] * q1u2) +
           nc[NC_B1 * N] * q0;
    S[2] = (nc[NC_K21 * N] * q1 + nc[NC_K22 * N] * q2) - (nc[NC_G2A * N] * q1u2 + nc[NC_G2B * N] * q2u2) +
           nc[NC_B2 * N] * q0;
    sF[le][0][0][node] = part(q1);
    sF[le][0][1][node] = part(F11);
    sF[le][0][2][node] = part(F12);
    sF[le][1][0][node] = part(q2);
    sF[le][1][1][node] = part(F12);
    sF[le][1][2][node] = part(F22);
  }
  __syncthreads();

  // DFR sweeps: extended flux [F(-1), f_1..f_NS, F(+1)] per line (Eq. 11-14)
  // this thread's rows of the derivative matrix, from shared memory into registers
  // (a per-thread row index into the constant bank would serialise the warp)
  double res[3] = {0.0, 0.0, 0.0};
  double Da[NS + 2], Db[NS + 2];
#pragma unroll
  for (int n = 0; n < NS + 2; ++n) {
    Da[n] = sD[k1][n];
    Db[n] = sD[k2][n];
  }
  if (active) {
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
      double d1 = Da[0] * sB[le][0][mu][k2] + Da[NS + 1] * sB[le][1][mu][k2];
      double d2 = Db[0] * sB[le][2][mu][k1] + Db[NS + 1] * sB[le][3][mu][k1];
#pragma unroll
      for (int l = 0; l < NS; ++l) {
        d1 = fma(Da[l + 1], sF[le][0][mu][k2 * NS + l], d1);
        d2 = fma(Db[l + 1], sF[le][1][mu][l * NS + k1], d2);
      }
      res[mu] = -dc.two_over_dx * (d1 + d2) + part(S[mu]);
    }
  }
  if (active) {
    const double sc = a.v ? 1.0 / a.eps : 1.0;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) res[mu] *= sc;
  }
  volume_epilogue<VolShape<NS>::THREADS, false, W3>(a.ep, active, idx, a.nodes, res, a.out, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------- launchers
template <typename T, int NS>
static int launch_ns(Ctx& c, const double* q, const double* v, double eps, double* out, const AugEpilogue& ep,
                     cudaStream_t s) {
  FaceArgs fa{q, v, eps, c.nodes, c.d_lines, c.d_face_coef, c.nfacepts, c.d_fb, ep.skip};
  int fthreads = 128;
  long long fblocks = (c.nfacepts + fthreads - 1) / fthreads;
  const bool jvp = v != nullptr;
  const int kf = jvp ? PK_FACE_JVP : PK_FACE_RHS, kv = jvp ? PK_VOL_JVP : PK_VOL_RHS;
  const bool pf = prof_take(c, kf), pv = prof_take(c, kv);
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  if (pf) {
    e0 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  face_flux_kernel<T, NS><<<(unsigned)fblocks, fthreads, 0, s>>>(fa, c.dc);
  if (pf || pv) {
    e1 = prof_event(c);
    cudaEventRecord(e1, s);
  }
  VolArgs va{q, v, eps, c.nodes, c.nelem, c.d_node_coef, c.d_fb, out, ep};
  long long vblocks = (c.nelem + VolShape<NS>::EPB - 1) / VolShape<NS>::EPB;
  if (ep.dotC)
    volume_kernel<T, NS, true><<<(unsigned)vblocks, VolShape<NS>::THREADS, 0, s>>>(va, c.dc);
  else
    volume_kernel<T, NS, false><<<(unsigned)vblocks, VolShape<NS>::THREADS, 0, s>>>(va, c.dc);
  if (pv) {
    e2 = prof_event(c);
    cudaEventRecord(e2, s);
    prof_record(c, kv, e1, e2);
  }
  if (pf) prof_record(c, kf, e0, e1);
  c.launches += 2;
  return cuda_status(cudaGetLastError());
}

template <typename T>
static int launch_any(Ctx& c, const double* q, const double* v, double eps, double* out, const AugEpilogue& ep,
                      cudaStream_t s) {
  switch (c.ns) {
    case 1: return launch_ns<T, 1>(c, q, v, eps, out, ep, s);
    case 2: return launch_ns<T, 2>(c, q, v, eps, out, ep, s);
    case 3: return launch_ns<T, 3>(c, q, v, eps, out, ep, s);
    case 4: return launch_ns<T, 4>(c, q, v, eps, out, ep, s);
    case 5: return launch_ns<T, 5>(c, q, v, eps, out, ep, s);
    case 6: return launch_ns<T, 6>(c, q, v, eps, out, ep, s);
    case 7: return launch_ns<T, 7>(c, q, v, eps, out, ep, s);
    case 8: return launch_ns<T, 8>(c, q, v, eps, out, ep, s);
    default: return SW_EINVAL;
  }
}

template <int NS>
static int launch_fb_ns(Ctx& c, const double* q, const double* v, double eps, double* out, double* fb,
                        cudaStream_t s) {
  FaceArgs fa{q, v, eps, c.nodes, c.d_lines, c.d_face_coef, c.nfacepts, fb, nullptr};
  const int fthreads = 128;
  const long long fblocks = (c.nfacepts + fthreads - 1) / fthreads;
  face_flux_kernel<cs, NS><<<(unsigned)fblocks, fthreads, 0, s>>>(fa, c.dc);
  AugEpilogue ep;
  VolArgs va{q, v, eps, c.nodes, c.nelem, c.d_node_coef, fb, out, ep};
  const long long vblocks = (c.nelem + VolShape<NS>::EPB - 1) / VolShape<NS>::EPB;
  volume_kernel<cs, NS><<<(unsigned)vblocks, VolShape<NS>::THREADS, 0, s>>>(va, c.dc);
  c.launches += 2;
  return cuda_status(cudaGetLastError());
}

int launch_jvp_fb(Ctx& c, const double* q, const double* v, double eps, double* out, double* fb,
                  cudaStream_t s) {
  switch (c.ns) {
    case 1: return launch_fb_ns<1>(c, q, v, eps, out, fb, s);
    case 2: return launch_fb_ns<2>(c, q, v, eps, out, fb, s);
    case 3: return launch_fb_ns<3>(c, q, v, eps, out, fb, s);
    case 4: return launch_fb_ns<4>(c, q, v, eps, out, fb, s);
    case 5: return launch_fb_ns<5>(c, q, v, eps, out, fb, s);
    case 6: return launch_fb_ns<6>(c, q, v, eps, out, fb, s);
    case 7: return launch_fb_ns<7>(c, q, v, eps, out, fb, s);
    case 8: return launch_fb_ns<8>(c, q, v, eps, out, fb, s);
    default: return SW_EINVAL;
  }
}

int launch_rhs(Ctx& c, const double* q, double* F, cudaStream_t s) {
  AugEpilogue ep;
  return launch_any<double>(c, q, nullptr, 1.0, F, ep, s);
}

int launch_jvp(Ctx& c, const double* q, const double* v, double eps, double* out, const AugEpilogue& ep,
               cudaStream_t s) {
  return launch_any<cs>(c, q, v, eps, out, ep, s);
}

// this translation unit's check word (bounds-checked builds; sw_check_status)
SW_CHECK_READER(check_word_dfr)

}  // namespace swepi
