// Host-side construction of the rotated cubed-sphere grid and the DFR tables
// (paper Sec. 3, App. B, App. C).  Everything here runs once in sw_init.
#include <cmath>
#include <cstring>
#include <new>

#include "swepi_internal.h"

namespace swepi {
namespace {

const double kQuarterPi = 0.78539816339744830962;

// Legendre P_N and its derivative at x by the three-term recurrence.
void legendre(int N, double x, double& P, double& dP) {
  double p0 = 1.0, p1 = x;
  if (N == 0) { P = 1.0; dP = 0.0; return; }
  for (int k = 2; k <= N; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  dP = N * (x * p1 - p0) / (x * x - 1.0);
}

// Gauss-Legendre points (ascending) and weights: Newton iteration on P_N
// (Sec. 3.1: the solution points are the roots of the Legendre polynomial).
void gauss_legendre(int N, std::vector<double>& x, std::vector<double>& w) {
  x.assign(N, 0.0);
  w.assign(N, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < N; ++i) {
    double z = -std::cos(pi * (i + 0.75) / (N + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(N, z, P, dP);
      double dz = P / dP;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double P, dP;
    legendre(N, z, P, dP);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dP * dP);
  }
}

// Barycentric weights of a node set.
std::vector<double> bary_weights(const std::vector<double>& z) {
  int n = (int)z.size();
  std::vector<double> b(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) b[j] /= (z[j] - z[k]);
  return b;
}

// Differentiation matrix of the Lagrange basis of z evaluated at the nodes
// themselves: Dz[i][j] = l_j'(z_i) (barycentric form; rows sum to zero).
std::vector<double> bary_diff(const std::vector<double>& z) {
  int n = (int)z.size();
  std::vector<double> b = bary_weights(z), D(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      D[i * n + j] = (b[j] / b[i]) / (z[i] - z[j]);
      diag -= D[i * n + j];
    }
    D[i * n + i] = diag;
  }
  return D;
}

// Lagrange basis of z evaluated at a point x that is not a node.
std::vector<double> bary_eval(const std::vector<double>& z, double x) {
  int n = (int)z.size();
  std::vector<double> b = bary_weights(z), l(n);
  double den = 0.0;
  for (int j = 0; j < n; ++j) den += b[j] / (x - z[j]);
  for (int j = 0; j < n; ++j) l[j] = b[j] / (x - z[j]) / den;
  return l;
}

struct V3 { double x, y, z; };
V3 v3(double a, double b, double c) { return {a, b, c}; }
V3 neg(V3 a) { return {-a.x, -a.y, -a.z}; }

// Panel frames: panel 0 from the rotation (lambda0, phi0, alpha0), the other
// five by the symmetries of the cube (panel p's centre and axes are panel 0's
// axes permuted and negated; equivalent to Eq. 81-95 with the branch choice).
void make_frames(Ctx& c) {
  const double l0 = c.prm.lambda0, f0 = c.prm.phi0, a0 = c.prm.alpha0;
  V3 ctr = v3(std::cos(f0) * std::cos(l0), std::cos(f0) * std::sin(l0), std::sin(f0));
  V3 el = v3(-std::sin(l0), std::cos(l0), 0.0);
  V3 ef = v3(-std::sin(f0) * std::cos(l0), -std::sin(f0) * std::sin(l0), std::cos(f0));
  V3 e1 = v3(std::cos(a0) * el.x - std::sin(a0) * ef.x, std::cos(a0) * el.y - std::sin(a0) * ef.y,
             std::cos(a0) * el.z - std::sin(a0) * ef.z);
  V3 e2 = v3(std::sin(a0) * el.x + std::cos(a0) * ef.x, std::sin(a0) * el.y + std::cos(a0) * ef.y,
             std::sin(a0) * el.z + std::cos(a0) * ef.z);
  V3 fr[6][3] = {{ctr, e1, e2},      {e1, neg(ctr), e2}, {neg(ctr), neg(e1), e2},
                 {neg(e1), ctr, e2}, {e2, e1, neg(ctr)}, {neg(e2), e1, ctr}};
  for (int p = 0; p < 6; ++p)
    for (int k = 0; k < 3; ++k) {
      c.frame[p][k][0] = fr[p][k].x;
      c.frame[p][k][1] = fr[p][k].y;
      c.frame[p][k][2] = fr[p][k].z;
    }
}

struct Metric { double sqrtg, h11, h12, h22; };
Metric metric_at(double X, double Y, double a) {
  double d2 = 1.0 + X * X + Y * Y, d = std::sqrt(d2);
  Metric m;
  m.sqrtg = a * a * (1 + X * X) * (1 + Y * Y) / (d2 * d);            // Eq. (70)
  m.h11 = d2 / (a * a * (1 + X * X));                                 // Eq. (67)
  m.h12 = X * Y * d2 / (a * a * (1 + X * X) * (1 + Y * Y));           // Eq. (68)
  m.h22 = d2 / (a * a * (1 + Y * Y));                                 // Eq. (69)
  return m;
}

// Element-local coordinate of (element e, point k) along an axis.
double line_coord(const Ctx& c, int e, int k) {
  return -kQuarterPi + (e + 0.5) * c.dx + c.xi[k] * c.dx * 0.5;
}

long long elem_index(const Ctx& c, int p, int e2, int e1) { return ((long long)p * c.ne + e2) * c.ne + e1; }

// Edge codes: 0 = W (x1 = -pi/4), 1 = E, 2 = S (x2 = -pi/4), 3 = N.
// Element of panel p at along-edge position e of edge `edge`.
void edge_element(const Ctx& c, int edge, int e, int& e2, int& e1) {
  int last = c.ne - 1;
  switch (edge) {
    case 0: e1 = 0; e2 = e; break;
    case 1: e1 = last; e2 = e; break;
    case 2: e2 = 0; e1 = e; break;
    default: e2 = last; e1 = e; break;
  }
}

// The twelve panel interfaces: (panel a, edge a, panel b, edge b, reversed).
// Along-edge coordinates run with x^2 on W/E edges and x^1 on S/N edges.
struct Iface { int pa, ea, pb, eb, rev; };
const Iface kIfaces[12] = {
    {0, 1, 1, 0, 0}, {1, 1, 2, 0, 0}, {2, 1, 3, 0, 0}, {0, 0, 3, 1, 0},
    {0, 3, 4, 2, 0}, {1, 3, 4, 1, 0}, {2, 3, 4, 3, 1}, {3, 3, 4, 0, 1},
    {0, 2, 5, 3, 0}, {1, 2, 5, 1, 1}, {2, 2, 5, 2, 1}, {3, 2, 5, 0, 0},
};

// App. C, Eq. (100)-(135): contravariant components on panel a from those on
// panel b at their common edge, Z = tan of the along-edge coordinate on panel
// a.  The paper prints each relation in one direction (panel q -> p, with the
// coordinate named on q); the other direction is the 2x2 inverse.
void appc_transform(int pa, int pb, double Z, double T[2][2]) {
  double s = 2.0 * Z / (1.0 + Z * Z);
  double P[2][2];
  bool direct;  // printed relation maps b -> a directly
  if (pb == 4 || pb == 5) {
    // printed as A_(cap) = P A_(pa) with X on panel pa
    static const double tab4[4][2][2][2] = {
        // [q][row][col][{const, coefficient of s}]
        {{{1, 0}, {0, -1}}, {{0, 0}, {1, 0}}},    // (4,0) Eq. 104-105
        {{{0, 0}, {-1, 0}}, {{1, 0}, {0, -1}}},   // (4,1) Eq. 108-109
        {{{-1, 0}, {0, 1}}, {{0, 0}, {-1, 0}}},   // (4,2) Eq. 112-113
        {{{0, 0}, {1, 0}}, {{-1, 0}, {0, 1}}},    // (4,3) Eq. 116-117
    };
    static const double tab5[4][2][2][2] = {
        {{{1, 0}, {0, 1}}, {{0, 0}, {1, 0}}},     // (5,0) Eq. 120-121
        {{{0, 0}, {1, 0}}, {{-1, 0}, {0, -1}}},   // (5,1) Eq. 124-125
        {{{-1, 0}, {0, -1}}, {{0, 0}, {-1, 0}}},  // (5,2) Eq. 128-129
        {{{0, 0}, {-1, 0}}, {{1, 0}, {0, 1}}},    // (5,3) Eq. 132-133
    };
    const double(*t)[2][2] = (pb == 4) ? tab4[pa] : tab5[pa];
    for (int r = 0; r < 2; ++r)
      for (int k = 0; k < 2; ++k) P[r][k] = t[r][k][0] + t[r][k][1] * s;
    direct = false;  // P maps a -> cap (= b)
  } else {
    // ring: (p, q) = (0,1), (1,2), (2,3), (3,0): A_(p) = [[1, 0], [s, 1]] A_(q), Eq. 100-101
    P[0][0] = 1; P[0][1] = 0; P[1][0] = s; P[1][1] = 1;
    direct = (pb == (pa + 1) % 4);  // (p, q) = (a, b)
  }
  if (direct) {
    std::memcpy(T, P, sizeof(P));
  } else {
    double det = P[0][0] * P[1][1] - P[0][1] * P[1][0];
    T[0][0] = P[1][1] / det; T[0][1] = -P[0][1] / det;
    T[1][0] = -P[1][0] / det; T[1][1] = P[0][0] / det;
  }
}

// Gauss-Legendre points and weights of ns points, the DFR derivative matrix
// (Eq. 13: derivatives at the solution points of the Lagrange basis on the
// extended nodes {-1, xi, +1}, ns x (ns + 2) row-major) and the trace rows
// l_k(-1), l_k(+1) (Eq. 8).
void dfr_operators(int ns, std::vector<double>& xi, std::vector<double>& w, std::vector<double>& D,
                   std::vector<double>& lm, std::vector<double>& lp) {
  gauss_legendre(ns, xi, w);
  std::vector<double> ext(ns + 2);
  ext[0] = -1.0;
  for (int k = 0; k < ns; ++k) ext[k + 1] = xi[k];
  ext[ns + 1] = 1.0;
  std::vector<double> De = bary_diff(ext);
  D.assign((size_t)ns * (ns + 2), 0.0);
  for (int k = 0; k < ns; ++k)
    for (int m = 0; m < ns + 2; ++m) D[(size_t)k * (ns + 2) + m] = De[(k + 1) * (ns + 2) + m];
  if (ns == 1) {
    lm.assign(1, 1.0);
    lp.assign(1, 1.0);
  } else {
    lm = bary_eval(xi, -1.0);
    lp = bary_eval(xi, 1.0);
  }
}

// Node coefficients of one point (X, Y) = (tan x^1, tan x^2) of panel p: the
// pressure factors g_r h^ij / (2 sqrt g), -2 Gamma^i_{0j} (Eq. 71-74, with the
// bracket sin(latitude) * delta = z-component of c + X e1 + Y e2) and the
// spatial Christoffel symbols (Eq. 75-80); entry k goes to out[k * stride].
// The topography entries NC_B1, NC_B2 are left alone.
void node_coefficients(const Ctx& c, int p, double X, double Y, double* out, long long stride) {
  const double a = c.prm.radius, gr = c.prm.gravity, om = c.prm.omega;
  const double cz = c.frame[p][0][2], e1z = c.frame[p][1][2], e2z = c.frame[p][2][2];
  double d2 = 1 + X * X + Y * Y;
  Metric m = metric_at(X, Y, a);
  out[NC_C11 * stride] = 0.5 * gr * m.h11 / m.sqrtg;
  out[NC_C12 * stride] = 0.5 * gr * m.h12 / m.sqrtg;
  out[NC_C22 * stride] = 0.5 * gr * m.h22 / m.sqrtg;
  double s = cz + X * e1z + Y * e2z;
  out[NC_K11 * stride] = -2.0 * om * X * Y * s / d2;
  out[NC_K12 * stride] = 2.0 * om * (1 + Y * Y) * s / d2;
  out[NC_K21 * stride] = -2.0 * om * (1 + X * X) * s / d2;
  out[NC_K22 * stride] = 2.0 * om * X * Y * s / d2;
  out[NC_G1A * stride] = 2.0 * X * Y * Y / d2;
  out[NC_G1B * stride] = -2.0 * Y * (1 + Y * Y) / d2;
  out[NC_G2A * stride] = -2.0 * X * (1 + X * X) / d2;
  out[NC_G2B * stride] = 2.0 * X * X * Y / d2;
}

}  // namespace

int build_tables(Ctx& c) {
  const int ne = c.ne, ns = c.ns;
  c.dx = (2.0 * kQuarterPi) / ne;
  c.nelem = 6LL * ne * ne;
  c.nodes = c.nelem * ns * ns;
  c.n = 3 * c.nodes;
  // DFR matrices: extended nodes {-1, xi, +1} (Sec. 3.1)
  std::vector<double> D, lm, lp;
  dfr_operators(ns, c.xi, c.wq, D, lm, lp);
  make_frames(c);
  std::memset(&c.dc, 0, sizeof(c.dc));
  for (int k = 0; k < ns; ++k)
    for (int m = 0; m < ns + 2; ++m) c.dc.D[k][m] = D[(size_t)k * (ns + 2) + m];
  for (int k = 0; k < ns; ++k) {
    c.dc.lm[k] = lm[k];
    c.dc.lp[k] = lp[k];
    c.dc.lm32[k] = (float)lm[k];
    c.dc.lp32[k] = (float)lp[k];
  }
  c.Dg = (ns == 1) ? std::vector<double>(1, 0.0) : bary_diff(c.xi);
  for (int k = 0; k < ns; ++k)
    for (int l = 0; l < ns; ++l) c.dc.Dg[k][l] = c.Dg[k * ns + l];
  c.dc.two_over_dx = 2.0 / c.dx;
  c.dc.gravity = c.prm.gravity;

  const double a = c.prm.radius, gr = c.prm.gravity;

  // node coefficients
  c.node_coef_h.assign((size_t)NC_COUNT * c.nodes, 0.0);
  for (int p = 0; p < 6; ++p)
    for (int e2 = 0; e2 < ne; ++e2)
      for (int e1 = 0; e1 < ne; ++e1)
        for (int k2 = 0; k2 < ns; ++k2)
          for (int k1 = 0; k1 < ns; ++k1) {
            long long i = elem_index(c, p, e2, e1) * ns * ns + k2 * ns + k1;
            double X = std::tan(line_coord(c, e1, k1)), Y = std::tan(line_coord(c, e2, k2));
            node_coefficients(c, p, X, Y, &c.node_coef_h[(size_t)i], c.nodes);
          }

  // face lines: interior x1 faces, interior x2 faces, then panel interfaces
  std::vector<FaceLine> lines;
  std::vector<double> fc;  // [nfacepts][FC_COUNT] (transposed below)
  auto push_line = [&](FaceLine L, const double* x1, const double* x2, const double T[2][2], const double M[2][2],
                       double sig) {
    lines.push_back(L);
    for (int i = 0; i < ns; ++i) {
      double X = std::tan(x1[i]), Y = std::tan(x2[i]);
      Metric m = metric_at(X, Y, a);
      double hdd = (L.dir == 1) ? m.h11 : m.h22;
      double h1d = (L.dir == 1) ? m.h11 : m.h12;
      double h2d = (L.dir == 1) ? m.h12 : m.h22;
      double v[FC_COUNT] = {gr * hdd / m.sqrtg, 0.5 * gr * h1d / m.sqrtg, 0.5 * gr * h2d / m.sqrtg,
                            T[0][0], T[0][1], T[1][0], T[1][1], M[0][0], M[0][1], M[1][0], M[1][1], sig};
      (void)i;
      fc.insert(fc.end(), v, v + FC_COUNT);
    }
  };
  const double I2[2][2] = {{1, 0}, {0, 1}};
  std::vector<double> x1(ns), x2(ns);
  for (int p = 0; p < 6; ++p)
    for (int e2 = 0; e2 < ne; ++e2)
      for (int e1 = 0; e1 + 1 < ne; ++e1) {
        FaceLine L{(int)elem_index(c, p, e2, e1), 1, (int)elem_index(c, p, e2, e1 + 1), 0, 0, 1, 1, 0};
        for (int i = 0; i < ns; ++i) { x1[i] = -kQuarterPi + (e1 + 1) * c.dx; x2[i] = line_coord(c, e2, i); }
        push_line(L, x1.data(), x2.data(), I2, I2, 1.0);
      }
  for (int p = 0; p < 6; ++p)
    for (int e2 = 0; e2 + 1 < ne; ++e2)
      for (int e1 = 0; e1 < ne; ++e1) {
        FaceLine L{(int)elem_index(c, p, e2, e1), 3, (int)elem_index(c, p, e2 + 1, e1), 2, 0, 2, 1, 0};
        for (int i = 0; i < ns; ++i) { x1[i] = line_coord(c, e1, i); x2[i] = -kQuarterPi + (e2 + 1) * c.dx; }
        push_line(L, x1.data(), x2.data(), I2, I2, 1.0);
      }
  for (const Iface& f : kIfaces) {
    int da = (f.ea <= 1) ? 1 : 2, db = (f.eb <= 1) ? 1 : 2;
    for (int e = 0; e < ne; ++e) {
      int oe2, oe1, ne2, ne1;
      edge_element(c, f.ea, e, oe2, oe1);
      edge_element(c, f.eb, f.rev ? ne - 1 - e : e, ne2, ne1);
      FaceLine L{(int)elem_index(c, f.pa, oe2, oe1), f.ea, (int)elem_index(c, f.pb, ne2, ne1), f.eb,
                 f.rev, da, (f.ea == 1 || f.ea == 3) ? 1 : 0, 0};
      double edge_c = (f.ea == 1 || f.ea == 3) ? kQuarterPi : -kQuarterPi;
      for (int i = 0; i < ns; ++i) {
        double t = line_coord(c, e, i);
        if (da == 1) { x1[i] = edge_c; x2[i] = t; } else { x1[i] = t; x2[i] = edge_c; }
      }
      // per point transforms (they vary along the edge)
      lines.push_back(L);
      for (int i = 0; i < ns; ++i) {
        double t = line_coord(c, e, i);
        double T[2][2], Tinv[2][2];
        appc_transform(f.pa, f.pb, std::tan(t), T);  // owner (a) <- neighbour (b)
        double det = T[0][0] * T[1][1] - T[0][1] * T[1][0];
        Tinv[0][0] = T[1][1] / det; Tinv[0][1] = -T[0][1] / det;
        Tinv[1][0] = -T[1][0] / det; Tinv[1][1] = T[0][0] / det;
        double sig = Tinv[db - 1][da - 1] > 0 ? 1.0 : -1.0;
        double X = std::tan(x1[i]), Y = std::tan(x2[i]);
        Metric m = metric_at(X, Y, a);
        double hdd = (da == 1) ? m.h11 : m.h22;
        double h1d = (da == 1) ? m.h11 : m.h12;
        double h2d = (da == 1) ? m.h12 : m.h22;
        double v[FC_COUNT] = {gr * hdd / m.sqrtg, 0.5 * gr * h1d / m.sqrtg, 0.5 * gr * h2d / m.sqrtg,
                              T[0][0], T[0][1], T[1][0], T[1][1],
                              sig * Tinv[0][0], sig * Tinv[0][1], sig * Tinv[1][0], sig * Tinv[1][1], sig};
        fc.insert(fc.end(), v, v + FC_COUNT);
      }
    }
  }
  c.nlines = (int)lines.size();
  c.nfacepts = (long long)c.nlines * ns;
  if (c.nlines != 12 * ne * ne) return SW_EINVAL;

  std::vector<double> fcT((size_t)FC_COUNT * c.nfacepts);
  for (long long i = 0; i < c.nfacepts; ++i)
    for (int k = 0; k < FC_COUNT; ++k) fcT[(size_t)k * c.nfacepts + i] = fc[(size_t)i * FC_COUNT + k];

  cudaError_t e;
  e = cudaMalloc(&c.d_node_coef, sizeof(double) * NC_COUNT * c.nodes);
  if (e != cudaSuccess) return SW_ENOMEM;
  e = cudaMalloc(&c.d_face_coef, sizeof(double) * fcT.size());
  if (e != cudaSuccess) return SW_ENOMEM;
  e = cudaMalloc(&c.d_lines, sizeof(FaceLine) * lines.size());
  if (e != cudaSuccess) return SW_ENOMEM;
  e = cudaMalloc(&c.d_fb, sizeof(double) * c.nelem * 4 * 3 * ns);
  if (e != cudaSuccess) return SW_ENOMEM;
  if (cudaMemcpy(c.d_node_coef, c.node_coef_h.data(), sizeof(double) * c.node_coef_h.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c.d_face_coef, fcT.data(), sizeof(double) * fcT.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c.d_lines, lines.data(), sizeof(FaceLine) * lines.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return SW_ECUDA;
  return SW_OK;
}

void node_unit_xyz(const Ctx& c, double* xyz) {
  const int ne = c.ne, ns = c.ns;
  for (int p = 0; p < 6; ++p)
    for (int e2 = 0; e2 < ne; ++e2)
      for (int e1 = 0; e1 < ne; ++e1)
        for (int k2 = 0; k2 < ns; ++k2)
          for (int k1 = 0; k1 < ns; ++k1) {
            long long i = elem_index(c, p, e2, e1) * ns * ns + k2 * ns + k1;
            double X = std::tan(line_coord(c, e1, k1)), Y = std::tan(line_coord(c, e2, k2));
            double d = std::sqrt(1 + X * X + Y * Y);
            for (int k = 0; k < 3; ++k)
              xyz[k * c.nodes + i] = (c.frame[p][0][k] + X * c.frame[p][1][k] + Y * c.frame[p][2][k]) / d;
          }
}

int bottom_coefficients(Ctx& c, const double* hB) {
  const int ne = c.ne, ns = c.ns;
  c.hB_h.assign(hB, hB + c.nodes);
  const double a = c.prm.radius, gr = c.prm.gravity;
  for (long long el = 0; el < c.nelem; ++el) {
    int e1 = (int)(el % ne), e2 = (int)((el / ne) % ne);
    const double* h = hB + el * ns * ns;
    for (int k2 = 0; k2 < ns; ++k2)
      for (int k1 = 0; k1 < ns; ++k1) {
        double d1 = 0, d2 = 0;
        for (int l = 0; l < ns; ++l) {
          d1 += c.Dg[k1 * ns + l] * h[k2 * ns + l];
          d2 += c.Dg[k2 * ns + l] * h[l * ns + k1];
        }
        d1 *= c.dc.two_over_dx;
        d2 *= c.dc.two_over_dx;
        double X = std::tan(line_coord(c, e1, k1)), Y = std::tan(line_coord(c, e2, k2));
        Metric m = metric_at(X, Y, a);
        long long i = el * ns * ns + k2 * ns + k1;
        c.node_coef_h[(size_t)NC_B1 * c.nodes + i] = -gr * (m.h11 * d1 + m.h12 * d2);
        c.node_coef_h[(size_t)NC_B2 * c.nodes + i] = -gr * (m.h12 * d1 + m.h22 * d2);
      }
  }
  cudaError_t e = cudaMemcpy(c.d_node_coef + (size_t)NC_B1 * c.nodes, c.node_coef_h.data() + (size_t)NC_B1 * c.nodes,
                             sizeof(double) * 2 * c.nodes, cudaMemcpyHostToDevice);
  return cuda_status(e);
}

// per-node tables of the diagnostics: sqrt g, w_m w_n, g_11, g_12, g_22, the
// Coriolis parameter f = 2 Omega s / delta (Eq. 46) and h_B
void diag_tables_host(const Ctx& c, double* tab) {
  const int ne = c.ne, ns = c.ns;
  const double a = c.prm.radius, om = c.prm.omega;
  const long long N = c.nodes;
  for (int p = 0; p < 6; ++p) {
    const double cz = c.frame[p][0][2], e1z = c.frame[p][1][2], e2z = c.frame[p][2][2];
    for (int e2 = 0; e2 < ne; ++e2)
      for (int e1 = 0; e1 < ne; ++e1)
        for (int k2 = 0; k2 < ns; ++k2)
          for (int k1 = 0; k1 < ns; ++k1) {
            long long i = elem_index(c, p, e2, e1) * ns * ns + k2 * ns + k1;
            double X = std::tan(line_coord(c, e1, k1)), Y = std::tan(line_coord(c, e2, k2));
            double d2 = 1 + X * X + Y * Y;
            Metric m = metric_at(X, Y, a);
            tab[0 * N + i] = m.sqrtg;
            tab[1 * N + i] = c.wq[k1] * c.wq[k2];
            tab[2 * N + i] = a * a / (d2 * d2) * (1 + X * X) * (1 + X * X) * (1 + Y * Y);   // Eq. (64)
            tab[3 * N + i] = -a * a / (d2 * d2) * X * Y * (1 + X * X) * (1 + Y * Y);        // Eq. (65)
            tab[4 * N + i] = a * a / (d2 * d2) * (1 + X * X) * (1 + Y * Y) * (1 + Y * Y);   // Eq. (66)
            tab[5 * N + i] = 2.0 * om * (cz + X * e1z + Y * e2z) / std::sqrt(d2);
            tab[6 * N + i] = c.hB_h.empty() ? 0.0 : c.hB_h[i];
          }
  }
}

int fields_to_state(const Ctx& c, const double* h, const double* hB, const double* V, double* q) {
  const int ne = c.ne, ns = c.ns;
  const double a = c.prm.radius;
  for (int p = 0; p < 6; ++p) {
    const double* C = c.frame[p][0];
    const double* E1 = c.frame[p][1];
    const double* E2 = c.frame[p][2];
    for (int e2 = 0; e2 < ne; ++e2)
      for (int e1 = 0; e1 < ne; ++e1)
        for (int k2 = 0; k2 < ns; ++k2)
          for (int k1 = 0; k1 < ns; ++k1) {
            long long i = elem_index(c, p, e2, e1) * ns * ns + k2 * ns + k1;
            double X = std::tan(line_coord(c, e1, k1)), Y = std::tan(line_coord(c, e2, k2));
            double d2 = 1 + X * X + Y * Y, d = std::sqrt(d2);
            // covariant basis t_j = d(a r)/dx^j, r = (C + X E1 + Y E2)/delta
            double t1[3], t2[3], vc1 = 0, vc2 = 0;
            for (int k = 0; k < 3; ++k) {
              double P = C[k] + X * E1[k] + Y * E2[k];
              t1[k] = a * (1 + X * X) * (E1[k] / d - P * X / (d2 * d));
              t2[k] = a * (1 + Y * Y) * (E2[k] / d - P * Y / (d2 * d));
              vc1 += V[k * c.nodes + i] * t1[k];
              vc2 += V[k * c.nodes + i] * t2[k];
            }
            Metric m = metric_at(X, Y, a);
            double u1 = m.h11 * vc1 + m.h12 * vc2, u2 = m.h12 * vc1 + m.h22 * vc2;
            double q0 = m.sqrtg * (h[i] - hB[i]);
            q[i] = q0;
            q[c.nodes + i] = q0 * u1;
            q[2 * c.nodes + i] = q0 * u2;
          }
  }
  return SW_OK;
}

}  // namespace swepi

extern "C" int sw_dfr_operators(int p, double* xi, double* w, double* D_ext, double* l_minus, double* l_plus) {
  if (p < 0 || p > swepi::MAX_NS - 1) return SW_EINVAL;
  const int ns = p + 1;
  std::vector<double> x, wq, D, lm, lp;
  try {
    swepi::dfr_operators(ns, x, wq, D, lm, lp);
  } catch (...) {
    return SW_ENOMEM;
  }
  for (int k = 0; k < ns; ++k) {
    if (xi) xi[k] = x[k];
    if (w) w[k] = wq[k];
    if (l_minus) l_minus[k] = lm[k];
    if (l_plus) l_plus[k] = lp[k];
  }
  if (D_ext)
    for (size_t i = 0; i < D.size(); ++i) D_ext[i] = D[i];
  return SW_OK;
}

extern "C" int sw_node_coefficients(const sw_params* prm, int panel, int npts, const double* X, const double* Y,
                                    double* out) {
  if (!prm || panel < 0 || panel > 5 || npts < 0 || (npts > 0 && (!X || !Y || !out))) return SW_EINVAL;
  swepi::Ctx* c = new (std::nothrow) swepi::Ctx();
  if (!c) return SW_ENOMEM;
  c->prm = *prm;
  swepi::make_frames(*c);
  for (int k = 0; k < swepi::NC_COUNT; ++k)
    for (int i = 0; i < npts; ++i) out[(long long)k * npts + i] = 0.0;
  for (int i = 0; i < npts; ++i) swepi::node_coefficients(*c, panel, X[i], Y[i], out + i, npts);
  delete c;
  return SW_OK;
}

extern "C" int sw_interface_transform(int k, double t, int* pa, int* ea, int* pb, int* eb, int* rev, double* T) {
  if (k < 0 || k > 11) return SW_EINVAL;
  const swepi::Iface& f = swepi::kIfaces[k];
  if (pa) *pa = f.pa;
  if (ea) *ea = f.ea;
  if (pb) *pb = f.pb;
  if (eb) *eb = f.eb;
  if (rev) *rev = f.rev;
  if (T) {
    double M[2][2];
    swepi::appc_transform(f.pa, f.pb, std::tan(t), M);
    T[0] = M[0][0];
    T[1] = M[0][1];
    T[2] = M[1][0];
    T[3] = M[1][1];
  }
  return SW_OK;
}
