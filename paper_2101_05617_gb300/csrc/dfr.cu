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

template <typename T, int NS>
__global__ void __launch_bounds__(128) face_flux_kernel(FaceArgs a, DfrConst dc) {
  if (a.skip && *a.skip) return;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nfacepts) return;
  const int line = (int)(t / NS), i = (int)(t % NS);
  const FaceLine L = a.lines[line];
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

template <int NS>
struct VolShape {
  static constexpr int EPB = (256 / (NS * NS)) > 0 ? (256 / (NS * NS)) : 1;
  static constexpr int THREADS = EPB * NS * NS;
};

template <typename T, int NS>
__global__ void __launch_bounds__(VolShape<NS>::THREADS) volume_kernel(VolArgs a, DfrConst dc) {
  constexpr int EPB = VolShape<NS>::EPB;
  constexpr int NN = NS * NS;
  if (a.ep.skip && *a.ep.skip) return;
  __shared__ double sF[EPB][2][3][NN];       // [dir][mu][k2*NS+k1]
  __shared__ double sB[EPB][4][3][NS];       // face fluxes [edge][mu][pt]
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
  if (!active) return;

  // DFR sweeps: extended flux [F(-1), f_1..f_NS, F(+1)] per line (Eq. 11-14)
  double res[3];
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    double d1 = dc.D[k1][0] * sB[le][0][mu][k2] + dc.D[k1][NS + 1] * sB[le][1][mu][k2];
    double d2 = dc.D[k2][0] * sB[le][2][mu][k1] + dc.D[k2][NS + 1] * sB[le][3][mu][k1];
#pragma unroll
    for (int l = 0; l < NS; ++l) {
      d1 = fma(dc.D[k1][l + 1], sF[le][0][mu][k2 * NS + l], d1);
      d2 = fma(dc.D[k2][l + 1], sF[le][1][mu][l * NS + k1], d2);
    }
    res[mu] = -dc.two_over_dx * (d1 + d2) + part(S[mu]);
  }
  const double scale = a.v ? a.ep.scale / a.eps : a.ep.scale;
  const long long N = a.nodes;
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    double o = scale * res[mu];
    if (a.ep.p > 0) {
#pragma unroll
      for (int l = 0; l < MAX_NB; ++l)
        if (l < a.ep.p && a.ep.b[l]) o = fma(a.ep.nu * a.ep.tail_in[l], a.ep.b[l][idx + mu * N], o);
    }
    a.out[idx + mu * N] = o;
  }
  if (a.ep.tail_out && blockIdx.x == 0 && threadIdx.x < a.ep.p)
    a.ep.tail_out[threadIdx.x] = (threadIdx.x + 1 < a.ep.p) ? a.ep.tail_in[threadIdx.x + 1] : 0.0;
}

// ---------------------------------------------------------------- launchers
template <typename T, int NS>
static int launch_ns(Ctx& c, const double* q, const double* v, double eps, double* out, const AugEpilogue& ep,
                     cudaStream_t s) {
  FaceArgs fa{q, v, eps, c.nodes, c.d_lines, c.d_face_coef, c.nfacepts, c.d_fb, ep.skip};
  int fthreads = 128;
  long long fblocks = (c.nfacepts + fthreads - 1) / fthreads;
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  if (c.prof) {
    e0 = prof_event(c);
    e1 = prof_event(c);
    e2 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  face_flux_kernel<T, NS><<<(unsigned)fblocks, fthreads, 0, s>>>(fa, c.dc);
  if (c.prof) cudaEventRecord(e1, s);
  VolArgs va{q, v, eps, c.nodes, c.nelem, c.d_node_coef, c.d_fb, out, ep};
  long long vblocks = (c.nelem + VolShape<NS>::EPB - 1) / VolShape<NS>::EPB;
  volume_kernel<T, NS><<<(unsigned)vblocks, VolShape<NS>::THREADS, 0, s>>>(va, c.dc);
  if (c.prof) {
    cudaEventRecord(e2, s);
    const bool jvp = v != nullptr;
    prof_record(c, jvp ? PK_FACE_JVP : PK_FACE_RHS, e0, e1);
    prof_record(c, jvp ? PK_VOL_JVP : PK_VOL_RHS, e1, e2);
  }
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

}  // namespace swepi
