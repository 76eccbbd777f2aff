// Complex-step JVP split into its real and imaginary halves.
//
// Every JVP of one Krylov solve, and the remainder products of one EPI step,
// is taken at the same linearisation point q_n (Eq. 33-35).  In the
// complex-step evaluation F(q_n + i eps v) the real part of every intermediate
// (1/q^0, u^i, a^d, the Froude numbers, the AUSM splittings, ...) depends on q_n
// only, while the imaginary part is a linear function of v whose coefficients
// are those real parts.  The split path therefore evaluates the real half once
// per linearisation point and stores, per solution point and per interface
// point, the coefficients of the imaginary half:
//   lin_node_kernel   per node: u^1, u^2 and the coefficients of the imaginary
//                     parts of sqrt(g) T^{ij} (Eq. 136) and of the sources of
//                     Eq. (2) as functions of Im q;
//   lin_face_kernel   per interface point: the 3 x 6 matrix taking the
//                     imaginary parts of the two traces to the imaginary part of
//                     the AUSM flux, obtained by propagating unit imaginary
//                     parts through the same complex-step AUSM code as the
//                     plain kernels (the neighbour's App. C transform folded in).
// Each JVP then runs only the imaginary half, in real arithmetic:
//   face_tangent_kernel   traces of v, the 3 x 6 map, the hand-back;
//   volume_tangent_kernel pointwise imaginary fluxes and sources, the DFR
//                         sweeps (Eq. 12-14) and the augmented-operator epilogue.
// The imaginary parts are proportional to eps, so the tangent is propagated for
// v itself and the final division by eps is omitted.  Results equal the plain
// path up to rounding; no FP64 division or square root remains per JVP.
#include <cuda_runtime.h>

#include <algorithm>

#include "dfr_device.cuh"
#include "dfr_tangent.cuh"
#include "kiops_dev.h"
#include "swepi_internal.h"

namespace swepi {

namespace {

// ---------------------------------------------------------------- linearise
__global__ void lin_node_kernel(const double* __restrict__ q, const double* __restrict__ nc, long long nodes,
                                double* __restrict__ ln) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nodes) return;
  const long long N = nodes;
  const double q0 = q[i], q1 = q[i + N], q2 = q[i + 2 * N];
  const double r = 1.0 / q0;
  const double u1 = q1 * r, u2 = q2 * r;
  const double c11 = nc[NC_C11 * N + i], c12 = nc[NC_C12 * N + i], c22 = nc[NC_C22 * N + i];
  const double g1a = nc[NC_G1A * N + i], g1b = nc[NC_G1B * N + i];
  const double g2a = nc[NC_G2A * N + i], g2b = nc[NC_G2B * N + i];
  // Im sqrt(g)T^{ij} = u^j Im q^i + u^i Im q^j + (g_r h^ij q^0 / sqrt g - u^i u^j) Im q^0
  ln[LN_U1 * N + i] = u1;
  ln[LN_U2 * N + i] = u2;
  ln[LN_A11 * N + i] = 2.0 * c11 * q0 - u1 * u1;
  ln[LN_A12 * N + i] = 2.0 * c12 * q0 - u1 * u2;
  ln[LN_A22 * N + i] = 2.0 * c22 * q0 - u2 * u2;
  // Im S^i = s_i1 Im q^1 + s_i2 Im q^2 + s_i0 Im q^0 (Coriolis, Gamma^i_jk, topography terms of Eq. 2)
  ln[LN_S11 * N + i] = nc[NC_K11 * N + i] - 2.0 * g1a * u1 - g1b * u2;
  ln[LN_S12 * N + i] = nc[NC_K12 * N + i] - g1b * u1;
  ln[LN_S10 * N + i] = g1a * u1 * u1 + g1b * u1 * u2 + nc[NC_B1 * N + i];
  ln[LN_S21 * N + i] = nc[NC_K21 * N + i] - g2a * u2;
  ln[LN_S22 * N + i] = nc[NC_K22 * N + i] - g2a * u1 - 2.0 * g2b * u2;
  ln[LN_S20 * N + i] = g2a * u1 * u2 + g2b * u2 * u2 + nc[NC_B2 * N + i];
}

struct LinFaceArgs {
  const double* q;
  long long nodes;
  const FaceLine* lines;
  const double* fc;
  long long nfacepts;
  double* lf;   // [18][nfacepts]: owner-trace block then neighbour-trace block
};

template <int NS>
__global__ void __launch_bounds__(128) lin_face_kernel(LinFaceArgs a, DfrConst dc) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nfacepts) return;
  const int line = (int)(t / NS), i = (int)(t % NS);
  const FaceLine L = a.lines[line];
  if (!face_line_ok<NS>(L, a.nodes)) return;
  const int in = L.reversed ? NS - 1 - i : i;
  double qo[3], qn[3];
  trace<double, NS>(a.q, nullptr, 0.0, a.nodes, L.owner, L.owner_edge, i, dc, qo);
  trace<double, NS>(a.q, nullptr, 0.0, a.nodes, L.nbr, L.nbr_edge, in, dc, qn);
  const long long P = a.nfacepts;
  const double* fc = a.fc + t;
  const double T00 = fc[FC_T00 * P], T01 = fc[FC_T01 * P], T10 = fc[FC_T10 * P], T11 = fc[FC_T11 * P];
  const double qt[3] = {qn[0], T00 * qn[1] + T01 * qn[2], T10 * qn[1] + T11 * qn[2]};
  const double ad = fc[FC_AD * P], p1 = fc[FC_P1 * P], p2 = fc[FC_P2 * P];
  const double* qL = L.owner_is_left ? qo : qt;
  const double* qR = L.owner_is_left ? qt : qo;
  double J[3][6];
#pragma unroll 1
  for (int col = 0; col < 6; ++col) {
    cs zL[3], zR[3], fl[3];
    for (int k = 0; k < 3; ++k) {
      zL[k] = {qL[k], (col == k) ? 1.0 : 0.0};
      zR[k] = {qR[k], (col == k + 3) ? 1.0 : 0.0};
    }
    ausm_flux<cs>(zL, zR, L.dir, ad, p1, p2, fl);
    for (int mu = 0; mu < 3; ++mu) J[mu][col] = fl[mu].im;
  }
  // columns of the owner trace and of the neighbour trace (own coordinates)
  const int co = L.owner_is_left ? 0 : 3, cn = L.owner_is_left ? 3 : 0;
  double* out = a.lf + t;
  for (int mu = 0; mu < 3; ++mu) {
    for (int k = 0; k < 3; ++k) out[(mu * 3 + k) * P] = J[mu][co + k];
    // neighbour: Im q_t = blockdiag(1, T) Im q_n
    out[(9 + mu * 3 + 0) * P] = J[mu][cn + 0];
    out[(9 + mu * 3 + 1) * P] = J[mu][cn + 1] * T00 + J[mu][cn + 2] * T10;
    out[(9 + mu * 3 + 2) * P] = J[mu][cn + 1] * T01 + J[mu][cn + 2] * T11;
  }
}

// single-grid kernels around the shared bodies (dfr_tangent.cuh)
template <typename T, int NS>
__global__ void __launch_bounds__(128) face_tangent_kernel(TanFaceArgs<T> a, DfrConst dc) {
  pdl_wait();
  pdl_trigger();
  if (a.skip && *a.skip) return;
  face_tangent_body<T, NS>(a, dc, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// W3: with the orthogonalisation window of three in the epilogue; a
// persistent grid (volume_ctas)
template <typename T, int NS, bool W3>
__global__ void __launch_bounds__(VolShape<NS>::THREADS, 4) volume_tangent_kernel(TanVolArgs<T> a, DfrConst dc) {
  pdl_wait();
  pdl_trigger();
  if (a.ep.skip && *a.ep.skip) return;
  __shared__ VolSmem<T, NS, VolShape<NS>::EPB> sm;
  volume_tangent_persistent<T, NS, VolShape<NS>::EPB, VolShape<NS>::THREADS, W3>(a, dc, sm);
}

// the same kernels for the device-driven solver: the Krylov iteration index and
// the augmented operator come from its device state
template <typename T, int NS>
__global__ void __launch_bounds__(128) face_tangent_dev_kernel(const KDev* __restrict__ kd, KFix f,
                                                               TanFaceArgs<T> a, DfrConst dc) {
  if (*a.skip) return;
  const long long it = kd->it;
  a.v = f.V + it * f.ldv;
  a.v32 = (sizeof(T) == 4 && f.V32) ? f.V32 + it * f.ldv : nullptr;
  face_tangent_body<T, NS>(a, dc, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T, int NS, bool W3>
__global__ void __launch_bounds__(VolShape<NS>::THREADS, 4) volume_tangent_dev_kernel(const KDev* __restrict__ kd, KFix f,
                                                                                   TanVolArgs<T> a0, DfrConst dc) {
  __shared__ TanVolArgs<T> a;
  if (threadIdx.x == 0) {
    a = a0;
    const int it = kd->it;
    a.v = f.V + (long long)it * f.ldv;
    a.out = f.V + (long long)(it + 1) * f.ldv;
    iter_epilogue_dev(a.ep, *kd, f, it, W3, sizeof(T) == 4);
  }
  __syncthreads();
  if (*a.ep.skip) return;
  __shared__ VolSmem<T, NS, VolShape<NS>::EPB> sm;
  volume_tangent_persistent<T, NS, VolShape<NS>::EPB, VolShape<NS>::THREADS, W3>(a, dc, sm);
}

// CTAs of a persistent volume grid: as many as fit on the GPU at once (the
// kernel's occupancy x SMs), at most one per element tile.  Queried once per
// kernel and device; prepare_volume_dev runs the queries of the device-driven
// solver's kernels before its stream capture.
constexpr int kMaxDevices = 64;
// Element tiles per CTA of a volume grid large enough to fill the GPU three
// times over: three tiles a CTA, the CTAs in waves.  Measured at 6 x 60 x 60,
// p = 5 (FP64, live): 149 / 142 / 137 / 151 us per launch with 1 / 2 / 3 / 4
// tiles a CTA and 142 us with one wave of resident CTAs taking an even share
// (the four CTAs of an SM then run their load and compute phases in step).
// Smaller grids take one wave of resident CTAs with an even share each.
constexpr int kVolTilesPerCta = 3;

template <typename T, int NS, bool W3, bool DEV>
int volume_ctas(int device, long long tiles) {
  static int fit[kMaxDevices] = {};
  if (device < 0 || device >= kMaxDevices) return -1;
  if (!fit[device]) {
    int sms = 0, nb = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -1;
    const cudaError_t e =
        DEV ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, volume_tangent_dev_kernel<T, NS, W3>,
                                                            VolShape<NS>::THREADS, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, volume_tangent_kernel<T, NS, W3>,
                                                            VolShape<NS>::THREADS, 0);
    if (e != cudaSuccess || nb < 1) return -1;
    fit[device] = nb * sms;
  }
  if (tiles >= (long long)kVolTilesPerCta * fit[device]) return (int)((tiles + kVolTilesPerCta - 1) / kVolTilesPerCta);
  return (int)std::min<long long>(std::max<long long>(tiles, 1), fit[device]);
}

__global__ void to_float_kernel(const double* __restrict__ src, float* __restrict__ dst, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

template <int NS>
int linearize_ns(Ctx& c, const double* q, cudaStream_t s) {
  const int th = 256;
  lin_node_kernel<<<(unsigned)((c.nodes + th - 1) / th), th, 0, s>>>(q, c.d_node_coef, c.nodes, c.d_lin_node);
  LinFaceArgs fa{q, c.nodes, c.d_lines, c.d_face_coef, c.nfacepts, c.d_lin_face};
  lin_face_kernel<NS><<<(unsigned)((c.nfacepts + 127) / 128), 128, 0, s>>>(fa, c.dc);
  c.launches += 2;
  return cuda_status(cudaGetLastError());
}

template <typename T, int NS>
int tangent_ns(Ctx& c, const double* v, double* out, const AugEpilogue& ep, const T* ln, const T* lf, T* fb,
               cudaStream_t s) {
  const bool pf = prof_take(c, PK_FACE_JVP), pv = prof_take(c, PK_VOL_JVP);
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  if (pf) {
    e0 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  TanFaceArgs<T> fa{v, sizeof(T) == 4 ? ep.v32 : nullptr, c.nodes, c.d_lines, c.d_face_coef, lf, c.nfacepts, fb,
                    ep.skip};
  if (launch_pdl(face_tangent_kernel<T, NS>, dim3((unsigned)((c.nfacepts + 127) / 128)), dim3(128), s, fa, c.dc) !=
      cudaSuccess)
    return SW_ECUDA;
  if (pf || pv) {
    e1 = prof_event(c);
    cudaEventRecord(e1, s);
  }
  TanVolArgs<T> va{v, c.nodes, c.nelem, ln, fb, out, ep};
  const long long vblocks = (c.nelem + VolShape<NS>::EPB - 1) / VolShape<NS>::EPB;
  int rt = 1;
  if (sizeof(T) == 4) {   // complex64-bulk form: element tiles staged by bulk copies where aligned
    rt = launch_volume_tile_f32<NS>(c, v, out, ep, s);
    if (rt < 0) return rt;
    if (rt == SW_OK) c.launches--;   // counted below
  }
  if (rt != SW_OK) {
    const int ctas = ep.dotC ? volume_ctas<T, NS, true, false>(c.device, vblocks)
                             : volume_ctas<T, NS, false, false>(c.device, vblocks);
    if (ctas < 1) return SW_ECUDA;
    const cudaError_t ev = ep.dotC ? launch_pdl(volume_tangent_kernel<T, NS, true>, dim3((unsigned)ctas),
                                                 dim3(VolShape<NS>::THREADS), s, va, c.dc)
                                   : launch_pdl(volume_tangent_kernel<T, NS, false>, dim3((unsigned)ctas),
                                                dim3(VolShape<NS>::THREADS), s, va, c.dc);
    if (ev != cudaSuccess) return SW_ECUDA;
  }
  if (pv) {
    e2 = prof_event(c);
    cudaEventRecord(e2, s);
    prof_record(c, PK_VOL_JVP, e1, e2);
  }
  if (pf) prof_record(c, PK_FACE_JVP, e0, e1);
  c.launches += 2;
  return cuda_status(cudaGetLastError());
}

template <int NS>
int tangent_any(Ctx& c, const double* v, double* out, const AugEpilogue& ep, bool fp32, cudaStream_t s) {
  if (fp32)
    return tangent_ns<float, NS>(c, v, out, ep, c.d_lin_node32, c.d_lin_face32, reinterpret_cast<float*>(c.d_fb), s);
  return tangent_ns<double, NS>(c, v, out, ep, c.d_lin_node, c.d_lin_face, c.d_fb, s);
}

template <typename T, int NS>
int capture_iter_ns(Ctx& c, KDev* kd, const KFix& f, bool w3, int p, cudaStream_t s) {
  const bool fp32 = sizeof(T) == 4;
  const T* lf = fp32 ? reinterpret_cast<const T*>(c.d_lin_face32) : reinterpret_cast<const T*>(c.d_lin_face);
  const T* ln = fp32 ? reinterpret_cast<const T*>(c.d_lin_node32) : reinterpret_cast<const T*>(c.d_lin_node);
  T* fb = reinterpret_cast<T*>(c.d_fb);
  TanFaceArgs<T> fa{nullptr, nullptr, c.nodes, c.d_lines, c.d_face_coef, lf, c.nfacepts, fb, c.d_flags};
  face_tangent_dev_kernel<T, NS><<<(unsigned)((c.nfacepts + 127) / 128), 128, 0, s>>>(kd, f, fa, c.dc);
  c.launches++;
  if (cudaGetLastError() != cudaSuccess) return SW_ECUDA;
  if (fp32 && p <= kTileMaxB) {   // the staged kernel where the buffers allow it
    const int rt = capture_volume_tile_dev<NS>(c, kd, f, w3, s);
    if (rt <= 0) return rt;
  }
  TanVolArgs<T> va{nullptr, c.nodes, c.nelem, ln, fb, nullptr, AugEpilogue{}};
  const long long vblocks = (c.nelem + VolShape<NS>::EPB - 1) / VolShape<NS>::EPB;
  const int ctas = w3 ? volume_ctas<T, NS, true, true>(c.device, vblocks)
                      : volume_ctas<T, NS, false, true>(c.device, vblocks);
  if (ctas < 1) return SW_ECUDA;
  if (w3)
    volume_tangent_dev_kernel<T, NS, true><<<(unsigned)ctas, VolShape<NS>::THREADS, 0, s>>>(kd, f, va, c.dc);
  else
    volume_tangent_dev_kernel<T, NS, false><<<(unsigned)ctas, VolShape<NS>::THREADS, 0, s>>>(kd, f, va, c.dc);
  c.launches++;
  return cuda_status(cudaGetLastError());
}

template <int NS>
int capture_iter_any(Ctx& c, KDev* kd, const KFix& f, bool fp32, bool w3, int p, cudaStream_t s) {
  return fp32 ? capture_iter_ns<float, NS>(c, kd, f, w3, p, s) : capture_iter_ns<double, NS>(c, kd, f, w3, p, s);
}

template <int NS>
int prepare_dev_ns(const Ctx& c, bool fp32) {
  const int a = fp32 ? volume_ctas<float, NS, false, true>(c.device, 1) : volume_ctas<double, NS, false, true>(c.device, 1);
  const int b = fp32 ? volume_ctas<float, NS, true, true>(c.device, 1) : volume_ctas<double, NS, true, true>(c.device, 1);
  return (a < 1 || b < 1) ? SW_ECUDA : SW_OK;
}

}  // namespace

int prepare_volume_dev(const Ctx& c, bool fp32) {
  switch (c.ns) {
    case 1: return prepare_dev_ns<1>(c, fp32);
    case 2: return prepare_dev_ns<2>(c, fp32);
    case 3: return prepare_dev_ns<3>(c, fp32);
    case 4: return prepare_dev_ns<4>(c, fp32);
    case 5: return prepare_dev_ns<5>(c, fp32);
    case 6: return prepare_dev_ns<6>(c, fp32);
    case 7: return prepare_dev_ns<7>(c, fp32);
    case 8: return prepare_dev_ns<8>(c, fp32);
    default: return SW_EINVAL;
  }
}

int capture_iter_jvp(Ctx& c, KDev* kd, const KFix& f, bool fp32, bool w3, int p, cudaStream_t s) {
  switch (c.ns) {
    case 1: return capture_iter_any<1>(c, kd, f, fp32, w3, p, s);
    case 2: return capture_iter_any<2>(c, kd, f, fp32, w3, p, s);
    case 3: return capture_iter_any<3>(c, kd, f, fp32, w3, p, s);
    case 4: return capture_iter_any<4>(c, kd, f, fp32, w3, p, s);
    case 5: return capture_iter_any<5>(c, kd, f, fp32, w3, p, s);
    case 6: return capture_iter_any<6>(c, kd, f, fp32, w3, p, s);
    case 7: return capture_iter_any<7>(c, kd, f, fp32, w3, p, s);
    case 8: return capture_iter_any<8>(c, kd, f, fp32, w3, p, s);
    default: return SW_EINVAL;
  }
}

int launch_linearize(Ctx& c, const double* q, cudaStream_t s) {
  if (!c.d_lin_node && cudaMalloc(&c.d_lin_node, sizeof(double) * LN_COUNT * c.nodes) != cudaSuccess)
    return SW_ENOMEM;
  if (!c.d_lin_face && cudaMalloc(&c.d_lin_face, sizeof(double) * 18 * c.nfacepts) != cudaSuccess)
    return SW_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool pl = prof_on(c, PK_LIN);
  if (pl) {
    e0 = prof_event(c);
    e1 = prof_event(c);
    cudaEventRecord(e0, s);
  }
  int rc;
  switch (c.ns) {
    case 1: rc = linearize_ns<1>(c, q, s); break;
    case 2: rc = linearize_ns<2>(c, q, s); break;
    case 3: rc = linearize_ns<3>(c, q, s); break;
    case 4: rc = linearize_ns<4>(c, q, s); break;
    case 5: rc = linearize_ns<5>(c, q, s); break;
    case 6: rc = linearize_ns<6>(c, q, s); break;
    case 7: rc = linearize_ns<7>(c, q, s); break;
    case 8: rc = linearize_ns<8>(c, q, s); break;
    default: return SW_EINVAL;
  }
  if (rc == SW_OK && c.jvp_mode == 2) {
    // complex64-bulk form: FP32 copies of the coefficient tables
    if (!c.d_lin_node32 && cudaMalloc(&c.d_lin_node32, sizeof(float) * LN_COUNT * c.nodes) != cudaSuccess)
      return SW_ENOMEM;
    if (!c.d_lin_face32 && cudaMalloc(&c.d_lin_face32, sizeof(float) * 23 * c.nfacepts) != cudaSuccess)
      return SW_ENOMEM;
    to_float_kernel<<<1024, 256, 0, s>>>(c.d_lin_node, c.d_lin_node32, (long long)LN_COUNT * c.nodes);
    to_float_kernel<<<1024, 256, 0, s>>>(c.d_lin_face, c.d_lin_face32, 18LL * c.nfacepts);
    // M00, M01, M10, M11, sigma (consecutive rows of the face table) after the map rows
    to_float_kernel<<<1024, 256, 0, s>>>(c.d_face_coef + (long long)FC_M00 * c.nfacepts,
                                         c.d_lin_face32 + 18LL * c.nfacepts, 5LL * c.nfacepts);
    c.launches += 3;
    rc = cuda_status(cudaGetLastError());
  }
  if (pl) {
    cudaEventRecord(e1, s);
    prof_record(c, PK_LIN, e0, e1);
  }
  if (rc == SW_OK) c.linearized = true;
  return rc;
}

int launch_jvp_lin(Ctx& c, const double* v, double* out, const AugEpilogue& ep, cudaStream_t s, bool fp32) {
  if (!c.linearized) return SW_EINVAL;
  if (fp32 && !c.d_lin_node32) return SW_EINVAL;
  // the FP32 kernels take the b-column terms from their FP32 copies only
  for (int l = 0; fp32 && l < ep.p && l < MAX_NB; ++l)
    if (ep.b[l] && !ep.b32[l]) return SW_EINVAL;
  switch (c.ns) {
    case 1: return tangent_any<1>(c, v, out, ep, fp32, s);
    case 2: return tangent_any<2>(c, v, out, ep, fp32, s);
    case 3: return tangent_any<3>(c, v, out, ep, fp32, s);
    case 4: return tangent_any<4>(c, v, out, ep, fp32, s);
    case 5: return tangent_any<5>(c, v, out, ep, fp32, s);
    case 6: return tangent_any<6>(c, v, out, ep, fp32, s);
    case 7: return tangent_any<7>(c, v, out, ep, fp32, s);
    case 8: return tangent_any<8>(c, v, out, ep, fp32, s);
    default: return SW_EINVAL;
  }
}

// this translation unit's check word (bounds-checked builds; sw_check_status)
SW_CHECK_READER(check_word_split)

}  // namespace swepi
