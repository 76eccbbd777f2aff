// Diagnostics of Sec. 5: the Gauss-Legendre global integral (Eq. 42) of mass,
// total energy and potential enstrophy (the invariants whose normalised drift
// Eq. 44 monitors), relative vorticity (Eq. 43) with the Coriolis parameter of
// Eq. (46), and the error norms of Eq. (39)-(41).  The derivative in Eq. (43)
// is the element-local collocation derivative of the covariant velocity
// u_j = g_jk u^k.  Integrals omit the element Jacobian (dx/2)^2 as Eq. (42)
// does.  Reductions are deterministic: fixed block partials, the last block
// adds them in order.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "swepi_internal.h"

namespace swepi {

namespace {

enum DiagTab { DT_SG = 0, DT_W, DT_G11, DT_G12, DT_G22, DT_F, DT_HB, DT_COUNT };
constexpr int NRED = 6;

template <int THREADS>
__device__ void block_reduce_and_finish(double v[NRED], const bool is_max[NRED], double* part, unsigned int* ticket,
                                        double* out) {
  __shared__ double sh[NRED][THREADS];
  __shared__ bool last;
  for (int k = 0; k < NRED; ++k) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < NRED; ++k) {
      double a = is_max[k] ? 0.0 : 0.0;
      for (int t = 0; t < THREADS; ++t) a = is_max[k] ? fmax(a, sh[k][t]) : a + sh[k][t];
      part[(long long)blockIdx.x * NRED + k] = a;
    }
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  for (int k = 0; k < NRED; ++k) {
    double a = 0.0;
    for (unsigned int b = 0; b < gridDim.x; ++b) {
      const double x = __ldcg(part + (long long)b * NRED + k);
      a = is_max[k] ? fmax(a, x) : a + x;
    }
    out[k] = a;
  }
  *ticket = 0u;
}

template <int NS>
struct DiagShape {
  static constexpr int EPB = (256 / (NS * NS)) > 0 ? (256 / (NS * NS)) : 1;
  static constexpr int THREADS = EPB * NS * NS;
};

// invariants: out = {mass, energy, potential enstrophy, max |zeta|, 0, 0}
template <int NS>
__global__ void __launch_bounds__(DiagShape<NS>::THREADS) invariants_kernel(
    const double* __restrict__ q, const double* __restrict__ tab, long long nodes, long long nelem, DfrConst dc,
    double gr, double* __restrict__ zeta_out, double* part, unsigned int* ticket, double* out) {
  constexpr int EPB = DiagShape<NS>::EPB, NN = NS * NS;
  __shared__ double c1[EPB][NN], c2[EPB][NN];
  const int le = threadIdx.x / NN, node = threadIdx.x % NN;
  const long long elem = (long long)blockIdx.x * EPB + le;
  const bool active = elem < nelem;
  const int k2 = node / NS, k1 = node % NS;
  const long long i = elem * NN + node;
  const long long N = nodes;
  double H = 0, u1 = 0, u2 = 0, sg = 1, w = 0, uu = 0;
  if (active) {
    sg = tab[DT_SG * N + i];
    w = tab[DT_W * N + i];
    const double q0 = q[i];
    H = q0 / sg;
    u1 = q[i + N] / q0;
    u2 = q[i + 2 * N] / q0;
    const double g11 = tab[DT_G11 * N + i], g12 = tab[DT_G12 * N + i], g22 = tab[DT_G22 * N + i];
    c1[le][node] = g11 * u1 + g12 * u2;
    c2[le][node] = g12 * u1 + g22 * u2;
    uu = u1 * c1[le][node] + u2 * c2[le][node];
  }
  __syncthreads();
  double v[NRED] = {0, 0, 0, 0, 0, 0};
  if (active) {
    double d1 = 0.0, d2 = 0.0;
    for (int l = 0; l < NS; ++l) {
      d1 = fma(dc.Dg[k1][l], c2[le][k2 * NS + l], d1);
      d2 = fma(dc.Dg[k2][l], c1[le][l * NS + k1], d2);
    }
    const double zeta = dc.two_over_dx * (d1 - d2) / sg;
    if (zeta_out) zeta_out[i] = zeta;
    const double hB = tab[DT_HB * N + i], f = tab[DT_F * N + i];
    const double wt = sg * w;
    v[0] = H * wt;
    v[1] = 0.5 * (H * uu + gr * ((H + hB) * (H + hB) - hB * hB)) * wt;
    v[2] = (zeta + f) * (zeta + f) / (2.0 * H) * wt;
    v[3] = fabs(zeta);
  }
  const bool is_max[NRED] = {false, false, false, true, false, false};
  block_reduce_and_finish<DiagShape<NS>::THREADS>(v, is_max, part, ticket, out);
}

// error norms of H against a reference: out = {I|dH|, I dH^2, I H_T, I H_T^2, max|dH|, max|H_T|}
template <int NS>
__global__ void __launch_bounds__(DiagShape<NS>::THREADS) norms_kernel(const double* __restrict__ q,
                                                                       const double* __restrict__ qr,
                                                                       const double* __restrict__ tab, long long nodes,
                                                                       double* part, unsigned int* ticket,
                                                                       double* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v[NRED] = {0, 0, 0, 0, 0, 0};
  if (i < nodes) {
    const double sg = tab[DT_SG * nodes + i], wt = sg * tab[DT_W * nodes + i];
    const double H = q[i] / sg, HT = qr[i] / sg, d = H - HT;
    v[0] = fabs(d) * wt;
    v[1] = d * d * wt;
    v[2] = HT * wt;
    v[3] = HT * HT * wt;
    v[4] = fabs(d);
    v[5] = fabs(HT);
  }
  const bool is_max[NRED] = {false, false, false, false, true, true};
  block_reduce_and_finish<DiagShape<NS>::THREADS>(v, is_max, part, ticket, out);
}

template <int NS>
int launch_diag_ns(Ctx& c, const double* q, const double* qref, double* zeta, cudaStream_t s) {
  unsigned int* ticket = reinterpret_cast<unsigned int*>(c.d_diag_flags);
  double* out = c.d_diag_out;
  if (!qref) {
    const long long blocks = (c.nelem + DiagShape<NS>::EPB - 1) / DiagShape<NS>::EPB;
    invariants_kernel<NS><<<(unsigned)blocks, DiagShape<NS>::THREADS, 0, s>>>(
        q, c.d_diag_tab, c.nodes, c.nelem, c.dc, c.prm.gravity, zeta, c.d_diag_part, ticket, out);
  } else {
    const long long blocks = (c.nodes + DiagShape<NS>::THREADS - 1) / DiagShape<NS>::THREADS;
    norms_kernel<NS><<<(unsigned)blocks, DiagShape<NS>::THREADS, 0, s>>>(q, qref, c.d_diag_tab, c.nodes,
                                                                         c.d_diag_part, ticket, out);
  }
  c.launches++;
  return cuda_status(cudaGetLastError());
}

}  // namespace

int ensure_diag(Ctx& c) {
  if (c.d_diag_tab) return SW_OK;
  std::vector<double> tab((size_t)DT_COUNT * c.nodes);
  diag_tables_host(c, tab.data());
  if (cudaMalloc(&c.d_diag_tab, sizeof(double) * tab.size()) != cudaSuccess) return SW_ENOMEM;
  // block partials: at most one block per element (invariants) or per 128 nodes (norms)
  if (cudaMalloc(&c.d_diag_part, sizeof(double) * NRED * (c.nelem + c.nodes / 128 + 2)) != cudaSuccess)
    return SW_ENOMEM;
  if (cudaMalloc(&c.d_diag_out, sizeof(double) * NRED) != cudaSuccess) return SW_ENOMEM;
  if (cudaMalloc(&c.d_diag_flags, sizeof(unsigned int) * 4) != cudaSuccess) return SW_ENOMEM;
  if (cudaMemset(c.d_diag_flags, 0, sizeof(unsigned int) * 4) != cudaSuccess) return SW_ECUDA;
  return cuda_status(cudaMemcpy(c.d_diag_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
}

int refresh_diag_bottom(Ctx& c, const double* hB) {
  if (!c.d_diag_tab) return SW_OK;
  return cuda_status(cudaMemcpy(c.d_diag_tab + (size_t)DT_HB * c.nodes, hB, sizeof(double) * c.nodes,
                                cudaMemcpyHostToDevice));
}

int launch_diagnostics(Ctx& c, const double* q, const double* qref, double* zeta, double* out_host, cudaStream_t s) {
  int rc = ensure_diag(c);
  if (rc) return rc;
  switch (c.ns) {
    case 1: rc = launch_diag_ns<1>(c, q, qref, zeta, s); break;
    case 2: rc = launch_diag_ns<2>(c, q, qref, zeta, s); break;
    case 3: rc = launch_diag_ns<3>(c, q, qref, zeta, s); break;
    case 4: rc = launch_diag_ns<4>(c, q, qref, zeta, s); break;
    case 5: rc = launch_diag_ns<5>(c, q, qref, zeta, s); break;
    case 6: rc = launch_diag_ns<6>(c, q, qref, zeta, s); break;
    case 7: rc = launch_diag_ns<7>(c, q, qref, zeta, s); break;
    case 8: rc = launch_diag_ns<8>(c, q, qref, zeta, s); break;
    default: return SW_EINVAL;
  }
  if (rc) return rc;
  if (cudaMemcpyAsync(out_host, c.d_diag_out, sizeof(double) * NRED, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return SW_ECUDA;
  return cuda_status(cudaStreamSynchronize(s));
}

}  // namespace swepi
