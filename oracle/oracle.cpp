// Plain FP64 CPU oracle for the compact simple HWENO scheme with ADER time
// discretization on triangular meshes (Luo, Zhao, Qiu, Chen).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
// that the CUDA library is checked against.  Only the test suite, the smoke
// check and the CPU-baseline leg of the benchmark may load it.  It shares no
// code, header, table or constant generator with the CUDA library; the two are
// independent readings of the paper.
//
// Structure (deliberately unlike the GPU path):
//   * connectivity by sorting edge keys (Section 2, mesh of triangles);
//   * per cell, Step 1 and Step 2 of Section 2.2 solved as constrained least
//     squares problems by Gaussian elimination on the KKT / normal equations;
//   * Steps 3-6 (linear weights Eq. pxy, smoothness indicators Eq. smoo1,
//     nonlinear weights Eq. nonlinearweight, reconstruction Eq. recon) evaluated
//     polynomial by polynomial at each edge Gauss point, in the paper's order;
//   * the Lax-Wendroff procedure of Section 2.1 written with the flux Jacobian
//     and Hessian contractions f', f'', g', g'' (obtained by exact forward-mode
//     differentiation of the flux functions f, g);
//   * a loop over edges that forms the local Lax-Friedrichs flux at Gauss-Lobatto
//     time nodes (Eqs. flux, tay, tayext, taylor2dtime) once per edge and
//     scatters it to both cells (Eqs. flx, fx), together with the central value
//     of Eq. timeflux for the Green-Gauss update (Eqs. derave2d1, derave2d2).
//
// The whole step is templated on the scalar type, so a forward-mode dual number
// gives the exact directional derivative of the discrete map (reference
// gradient for the adjoint).
//
// Readings of points the paper leaves open (each is named here and used by the
// CUDA path too):
//   R1  two Gauss-Legendre points per edge, weights 1/2 (Eq. fx);
//   R2  three-node Gauss-Lobatto (Simpson) time rule, nodes 0, dt/2, dt with
//       weights 1/6, 2/3, 1/6 (Eq. flux with the Lobatto remark of Sec. 2.3);
//   R3  least-squares rows in the frame scaled by h0 = sqrt(|K0|)
//       (derivative rows multiplied by h0), unweighted;
//   R4  the garbled subscripts of Step 1 read as V_{K_l2}, Y_{K_l3};
//   R6  beta sums each multi-index s with 1<=|s|<=k once, at the barycenter;
//   R7  W_ave taken per component;
//   R10 alpha = max spectral radius of d(F.n)/dW at the two cell averages;
//   R11 the exterior value is the neighbour's own reconstruction;
//   R12 dt = CFL * min_K r_K / lambda_K(Wbar_K), r_K the inradius, lambda_K the
//       spectral radius over all directions; last step clipped to T;
//   R13 non-periodic boundaries are transmissive: the ghost cell is the mirror
//       image of the cell with the cell's own data, and W^ext = W^int on the
//       boundary edge;
//   R25 reflective and inflow boundaries (the walls and the inflow/outflow
//       ends of Section 3's shock tubes): the ghost is the same mirror image
//       of the cell; at a wall it carries the mirrored solution (momentum
//       reflected, derivative averages by the chain rule) and W^ext is the
//       mirrored interior value; at an inflow edge it carries the imposed
//       state with zero derivative averages and W^ext is that state;
//       outflow is transmissive;
//   R23 (with the scale limiter) each edge flux blended with the first-order
//       LLF flux of the two averages so that the new averages stay admissible;
//   R22 (option) the time rule of Eq. flux as two-node Gauss-Legendre, nodes
//       dt (1/2 -+ sqrt(3)/6), weights 1/2, with the central values of Eq.
//       timeflux from a separate Taylor evaluation at t_{n+1};
//   R18 the scale limiter (optional, Euler): Zhang-Shu positivity scaling of
//       the final reconstruction toward the cell average over the six edge
//       Gauss points (density first, then pressure through the smallest
//       non-negative root of a quadratic, clamped to 1), eps = min(1e-13,
//       rho_bar, p_bar); then the same scaling of the space-time Taylor data
//       over the points and the three time nodes.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

namespace {

// ------------------------------------------------------------------ scalars
// Forward-mode dual number: value and one directional derivative.
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline Dual fabs(Dual a) { return a.v < 0 ? -a : a; }
inline double val(double x) { return x; }
inline double val(Dual x) { return x.v; }
using std::fabs;
using std::sqrt;

template <class S> S smax(S a, S b) { return (val(a) >= val(b)) ? a : b; }

// Hyper-dual number over scalar S: two infinitesimal directions a, b and their
// product ab.  Evaluating a flux with it gives F, F'[a], F'[b] and F''[a][b]
// exactly.
template <class S> struct HD {
  S v, a, b, ab;
};
template <class S> HD<S> hd_const(S x) { return HD<S>{x, S(0.0), S(0.0), S(0.0)}; }
template <class S> HD<S> operator+(HD<S> x, HD<S> y) { return {x.v + y.v, x.a + y.a, x.b + y.b, x.ab + y.ab}; }
template <class S> HD<S> operator-(HD<S> x, HD<S> y) { return {x.v - y.v, x.a - y.a, x.b - y.b, x.ab - y.ab}; }
template <class S> HD<S> operator*(HD<S> x, HD<S> y) {
  return {x.v * y.v, x.a * y.v + x.v * y.a, x.b * y.v + x.v * y.b,
          x.ab * y.v + x.a * y.b + x.b * y.a + x.v * y.ab};
}
template <class S> HD<S> operator*(double c, HD<S> x) { return {x.v * c, x.a * c, x.b * c, x.ab * c}; }
template <class S> HD<S> recip(HD<S> y) {
  S r = S(1.0) / y.v;
  S r2 = r * r;
  return {r, S(0.0) - y.a * r2, S(0.0) - y.b * r2, S(2.0) * y.a * y.b * r2 * r - y.ab * r2};
}
template <class S> HD<S> operator/(HD<S> x, HD<S> y) { return x * recip(y); }

// ------------------------------------------------------------------ problem
enum { EQ_ADVECTION = 0, EQ_BURGERS = 1, EQ_EULER = 2 };
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2, BC_INFLOW = 3 };

struct Params {
  int eq;
  int m;            // number of conserved components
  double ax, ay;    // advection velocity
  double gam;       // ratio of specific heats (Euler)
  double cfl;       // CFL number (Sec. 3: 0.5)
  double glin[4];   // linear weights gamma_1..gamma_4 (Step 3)
  double eps;       // epsilon of Eq. nonlinearweight (1e-8)
  int linear_only;  // debug: replace nonlinear weights by the linear ones
  int positivity;   // scale limiter of Zhang and Shu on the reconstruction (R18)
  int time_rule;    // 0: Gauss-Lobatto time nodes (R2); 1: two Gauss-Legendre nodes (R22)
};

struct EdgeRec {
  int32_t L, R;     // cells on the two sides; R = -1 on a boundary
  int jL, jR;       // local edge index in L and in R
  double Ax, Ay, Bx, By;   // endpoints in L's unwrapped frame, A->B CCW for L
  double nx, ny, len;      // outward unit normal of L, length
  double sx, sy;           // R's frame + (sx, sy) = L's frame
};

struct Problem {
  Params P;
  int64_t nv = 0, nt = 0;
  double Lx = 0, Ly = 0;
  int bc = BC_PERIODIC;
  std::vector<double> vx, vy;          // unwrapped vertices [nt][3]
  std::vector<double> area, cx, cy, inr, perim;
  std::vector<std::array<int32_t, 3>> nbr;   // neighbour across local edge j (-1: boundary)
  std::vector<std::array<int32_t, 3>> nbe;   // neighbour's local edge index
  std::vector<std::array<double, 6>> nbshift;  // (sx, sy) per local edge: nb frame + shift = own frame
  std::vector<EdgeRec> edges;
  std::vector<std::array<int64_t, 3>> cell_edge;   // index in edges of local edge j of each cell
  std::vector<std::array<int, 3>> ebc;       // type of each boundary edge (R13, R25)
  double win[4] = {1.0, 0.0, 0.0, 2.5};      // state imposed at inflow edges (conservative)
  std::string err;
};

thread_local std::string g_err;

// ------------------------------------------------------------------ geometry
double wrap(double d, double L) {
  if (L <= 0) return d;
  return d - L * std::floor(d / L + 0.5);
}

// Build connectivity by sorting the 3*nt edge keys (min vertex, max vertex).
bool build_connectivity(Problem& pb, const int32_t* tri) {
  const int64_t nt = pb.nt;
  struct Key { int32_t a, b; int32_t cell; int j; };
  std::vector<Key> keys;
  keys.reserve(3 * nt);
  for (int64_t t = 0; t < nt; ++t)
    for (int j = 0; j < 3; ++j) {
      int32_t a = tri[3 * t + j], b = tri[3 * t + (j + 1) % 3];
      keys.push_back({std::min(a, b), std::max(a, b), (int32_t)t, j});
    }
  std::sort(keys.begin(), keys.end(), [](const Key& x, const Key& y) {
    if (x.a != y.a) return x.a < y.a;
    if (x.b != y.b) return x.b < y.b;
    if (x.cell != y.cell) return x.cell < y.cell;
    return x.j < y.j;
  });
  pb.nbr.assign(nt, {-1, -1, -1});
  pb.nbe.assign(nt, {-1, -1, -1});
  size_t i = 0;
  while (i < keys.size()) {
    size_t k = i + 1;
    while (k < keys.size() && keys[k].a == keys[i].a && keys[k].b == keys[i].b) ++k;
    size_t cnt = k - i;
    if (cnt == 2) {
      const Key &p = keys[i], &q = keys[i + 1];
      if (p.cell == q.cell) { g_err = "degenerate triangle edge"; return false; }
      pb.nbr[p.cell][p.j] = q.cell; pb.nbe[p.cell][p.j] = q.j;
      pb.nbr[q.cell][q.j] = p.cell; pb.nbe[q.cell][q.j] = p.j;
    } else if (cnt == 1) {
      if (pb.bc == BC_PERIODIC) { g_err = "open edge on a periodic mesh"; return false; }
    } else {
      g_err = "non-manifold edge";
      return false;
    }
    i = k;
  }
  return true;
}

bool build_geometry(Problem& pb, const double* xy, const int32_t* tri) {
  const int64_t nt = pb.nt;
  pb.vx.resize(3 * nt); pb.vy.resize(3 * nt);
  pb.area.resize(nt); pb.cx.resize(nt); pb.cy.resize(nt); pb.inr.resize(nt); pb.perim.resize(nt);
  for (int64_t t = 0; t < nt; ++t) {
    double x0 = xy[2 * tri[3 * t]], y0 = xy[2 * tri[3 * t] + 1];
    for (int v = 0; v < 3; ++v) {
      double x = xy[2 * tri[3 * t + v]], y = xy[2 * tri[3 * t + v] + 1];
      pb.vx[3 * t + v] = x0 + wrap(x - x0, pb.Lx);
      pb.vy[3 * t + v] = y0 + wrap(y - y0, pb.Ly);
    }
    double *X = &pb.vx[3 * t], *Y = &pb.vy[3 * t];
    double a = 0.5 * ((X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]));
    if (!(a > 0)) { g_err = "triangle not counter-clockwise or degenerate"; return false; }
    pb.area[t] = a;
    pb.cx[t] = (X[0] + X[1] + X[2]) / 3.0;
    pb.cy[t] = (Y[0] + Y[1] + Y[2]) / 3.0;
    double per = 0;
    for (int j = 0; j < 3; ++j) per += std::hypot(X[(j + 1) % 3] - X[j], Y[(j + 1) % 3] - Y[j]);
    pb.inr[t] = 2.0 * a / per;
    pb.perim[t] = per;
  }
  // periodic shift of each neighbour and the edge list (one record per edge)
  pb.ebc.assign(nt, {BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE});
  pb.cell_edge.assign(nt, {-1, -1, -1});
  pb.nbshift.assign(nt, {0, 0, 0, 0, 0, 0});
  pb.edges.clear();
  for (int64_t t = 0; t < nt; ++t) {
    for (int j = 0; j < 3; ++j) {
      double Ax = pb.vx[3 * t + j], Ay = pb.vy[3 * t + j];
      double Bx = pb.vx[3 * t + (j + 1) % 3], By = pb.vy[3 * t + (j + 1) % 3];
      int32_t u = pb.nbr[t][j];
      double sx = 0, sy = 0;
      if (u >= 0) {
        int ju = pb.nbe[t][j];
        // in u's frame the shared edge runs from B' to A'; A' is u's vertex ju+1
        double Apx = pb.vx[3 * u + (ju + 1) % 3], Apy = pb.vy[3 * u + (ju + 1) % 3];
        sx = Ax - Apx; sy = Ay - Apy;
        if (pb.Lx > 0) sx = pb.Lx * std::round(sx / pb.Lx); else sx = 0;
        if (pb.Ly > 0) sy = pb.Ly * std::round(sy / pb.Ly); else sy = 0;
      }
      pb.nbshift[t][2 * j] = sx; pb.nbshift[t][2 * j + 1] = sy;
      if (u < 0 || t < u) {
        EdgeRec e;
        e.L = (int32_t)t; e.R = u; e.jL = j; e.jR = (u >= 0) ? pb.nbe[t][j] : -1;
        e.Ax = Ax; e.Ay = Ay; e.Bx = Bx; e.By = By;
        e.len = std::hypot(Bx - Ax, By - Ay);
        e.nx = (By - Ay) / e.len; e.ny = -(Bx - Ax) / e.len;
        e.sx = sx; e.sy = sy;
        pb.cell_edge[t][j] = (int64_t)pb.edges.size();
        if (u >= 0) pb.cell_edge[u][pb.nbe[t][j]] = (int64_t)pb.edges.size();
        pb.edges.push_back(e);
      }
    }
  }
  return true;
}

// ------------------------------------------------------------------ linear algebra
// Solve A x = b (n x n, row-major A in double, right-hand side of scalar S) by
// Gaussian elimination with partial pivoting.  Returns false if singular.
template <class S>
bool gauss_solve(int n, std::vector<double> A, std::vector<S> b, std::vector<S>& x) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[piv * n + k])) piv = i;
    if (std::fabs(A[piv * n + k]) < 1e-300) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[piv * n + j]);
      std::swap(b[k], b[piv]);
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      if (f == 0.0) continue;
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] = b[i] - S(f) * b[k];
    }
  }
  x.assign(n, S(0.0));
  for (int i = n - 1; i >= 0; --i) {
    S s = b[i];
    for (int j = i + 1; j < n; ++j) s = s - S(A[i * n + j]) * x[j];
    x[i] = s / S(A[i * n + i]);
  }
  return true;
}

// ------------------------------------------------------------------ polynomials
// A polynomial of degree <= 2 around (x0, y0) in the scaled variables
// xi = (x - x0)/h, eta = (y - y0)/h:
//   p = c0 + c1 xi + c2 eta + c3 (xi^2 - M3) + c4 (xi eta - M4) + c5 (eta^2 - M5)
// where M3, M4, M5 are the K0 means of xi^2, xi*eta, eta^2.
template <class S> struct Poly {
  double x0, y0, h, M3, M4, M5;
  S c[6];
};

// value and physical derivatives (p, p_x, p_y, p_xx, p_xy, p_yy) at (x, y)
template <class S> void poly_eval(const Poly<S>& p, double x, double y, S out[6]) {
  double xi = (x - p.x0) / p.h, et = (y - p.y0) / p.h;
  double ih = 1.0 / p.h;
  out[0] = p.c[0] + p.c[1] * S(xi) + p.c[2] * S(et) + p.c[3] * S(xi * xi - p.M3) +
           p.c[4] * S(xi * et - p.M4) + p.c[5] * S(et * et - p.M5);
  out[1] = (p.c[1] + S(2.0 * xi) * p.c[3] + S(et) * p.c[4]) * S(ih);
  out[2] = (p.c[2] + S(xi) * p.c[4] + S(2.0 * et) * p.c[5]) * S(ih);
  out[3] = S(2.0 * ih * ih) * p.c[3];
  out[4] = S(ih * ih) * p.c[4];
  out[5] = S(2.0 * ih * ih) * p.c[5];
}

// basis functions phi_1..phi_5 at a point of the scaled frame
void basis_vals(double xi, double et, double M3, double M4, double M5, double phi[6]) {
  phi[0] = 1.0; phi[1] = xi; phi[2] = et;
  phi[3] = xi * xi - M3; phi[4] = xi * et - M4; phi[5] = et * et - M5;
}

// cell mean of the basis over a triangle with scaled vertices (X[3], Y[3]);
// the three-edge-midpoint rule is exact for quadratics.
void basis_means(const double* X, const double* Y, double M3, double M4, double M5, double mean[6]) {
  for (int j = 0; j < 6; ++j) mean[j] = 0;
  for (int e = 0; e < 3; ++e) {
    double mx = 0.5 * (X[e] + X[(e + 1) % 3]), my = 0.5 * (Y[e] + Y[(e + 1) % 3]);
    double phi[6];
    basis_vals(mx, my, M3, M4, M5, phi);
    for (int j = 0; j < 6; ++j) mean[j] += phi[j] / 3.0;
  }
}

// ------------------------------------------------------------------ reconstruction
template <class S> struct CellRecon {
  Poly<S> p[4];      // p1 (quadratic), p2, p3, p4 (linear)
  S beta[4], omega[4];
  S wbar;            // cell average of the component
  S theta;           // spatial scale factor of the limiter (1: unchanged)
  S theta_t;         // scale factor of the limiter on the time Taylor data (1: unchanged)
  bool ok;
};

// State access: U[(k*m + c)*nt + i], k = 0 (Wbar), 1 (Vbar), 2 (Ybar).
template <class S> inline S Uat(const S* U, const Problem& pb, int k, int c, int64_t i) {
  return U[(k * pb.P.m + c) * pb.nt + i];
}

// Stencil member l (1..3) of cell t: its vertices in t's frame (physical
// coordinates), area, and the cell whose data it carries.
void stencil_member(const Problem& pb, int64_t t, int l, double X[3], double Y[3], double& a, int64_t& src) {
  int j = l - 1;
  int32_t u = pb.nbr[t][j];
  if (u >= 0) {
    double sx = pb.nbshift[t][2 * j], sy = pb.nbshift[t][2 * j + 1];
    for (int v = 0; v < 3; ++v) { X[v] = pb.vx[3 * u + v] + sx; Y[v] = pb.vy[3 * u + v] + sy; }
    a = pb.area[u];
    src = u;
  } else {
    // transmissive ghost (R13): mirror image of t across its edge j, t's data
    double Ax = pb.vx[3 * t + j], Ay = pb.vy[3 * t + j];
    double Bx = pb.vx[3 * t + (j + 1) % 3], By = pb.vy[3 * t + (j + 1) % 3];
    double dx = Bx - Ax, dy = By - Ay, dd = dx * dx + dy * dy;
    for (int v = 0; v < 3; ++v) {
      double px = pb.vx[3 * t + v] - Ax, py = pb.vy[3 * t + v] - Ay;
      double s = (px * dx + py * dy) / dd;
      double fx = s * dx, fy = s * dy;  // foot of the perpendicular
      X[v] = Ax + 2 * fx - px; Y[v] = Ay + 2 * fy - py;
    }
    std::swap(X[1], X[2]); std::swap(Y[1], Y[2]);  // keep counter-clockwise
    a = pb.area[t];
    src = t;
  }
}

// Unit normal of local edge j of cell t, outward of t.
void edge_normal(const Problem& pb, int64_t t, int j, double& nx, double& ny) {
  const double Ax = pb.vx[3 * t + j], Ay = pb.vy[3 * t + j];
  const double Bx = pb.vx[3 * t + (j + 1) % 3], By = pb.vy[3 * t + (j + 1) % 3];
  const double len = std::hypot(Bx - Ax, By - Ay);
  nx = (By - Ay) / len; ny = -(Bx - Ax) / len;
}

// Mirror of an Euler state across a wall with unit normal n: density and
// energy kept, momentum reflected, m -> m - 2 (m . n) n.
template <class S> void mirror_state(double nx, double ny, const S* W, S* Wm) {
  const S mn = W[1] * S(nx) + W[2] * S(ny);
  Wm[0] = W[0];
  Wm[1] = W[1] - S(2.0 * nx) * mn;
  Wm[2] = W[2] - S(2.0 * ny) * mn;
  Wm[3] = W[3];
}

// Data carried by the ghost across boundary edge j of cell t, all components
// (R13, R25).  The ghost is the mirror image of t across the edge.
//   transmissive: t's own averages;
//   reflective (Euler; the scalar equations treat it as transmissive): the
//     mirrored solution W_g(x) = M W(Rx), R the reflection across the edge
//     line and M the state mirror above, so that Wbar_g = M Wbar and the
//     averages of the gradient follow the chain rule, grad W_g = M (grad W) R;
//   inflow: the imposed state, with zero derivative averages.
template <class S> void ghost_data(const Problem& pb, const S* U, int64_t t, int j, S W[4], S V[4], S Y[4]) {
  const int m = pb.P.m;
  const int type = pb.ebc[t][j];
  if (type == BC_INFLOW) {
    for (int c = 0; c < m; ++c) { W[c] = S(pb.win[c]); V[c] = S(0.0); Y[c] = S(0.0); }
    return;
  }
  for (int c = 0; c < m; ++c) { W[c] = Uat(U, pb, 0, c, t); V[c] = Uat(U, pb, 1, c, t); Y[c] = Uat(U, pb, 2, c, t); }
  if (type != BC_REFLECTIVE || pb.P.eq != EQ_EULER) return;
  double nx, ny;
  edge_normal(pb, t, j, nx, ny);
  S Wm[4], Vm[4], Ym[4];
  mirror_state(nx, ny, W, Wm);
  mirror_state(nx, ny, V, Vm);   // the state mirror applied to the x- and y-derivative averages
  mirror_state(nx, ny, Y, Ym);
  // then the reflection R = I - 2 n n^T acting on (d/dx, d/dy) of every component
  for (int c = 0; c < 4; ++c) {
    const S dn = Vm[c] * S(nx) + Ym[c] * S(ny);
    V[c] = Vm[c] - S(2.0 * nx) * dn;
    Y[c] = Ym[c] - S(2.0 * ny) * dn;
    W[c] = Wm[c];
  }
}

// Steps 1-5 of Section 2.2 for component c of cell t.
template <class S> CellRecon<S> reconstruct(const Problem& pb, const S* U, int64_t t, int c) {
  CellRecon<S> R;
  R.ok = true;
  R.theta = S(1.0);
  R.theta_t = S(1.0);
  R.wbar = Uat(U, pb, 0, c, t);
  const double x0 = pb.cx[t], y0 = pb.cy[t], A0 = pb.area[t], h0 = std::sqrt(A0);
  // scaled vertices of K0 and its second moments
  double X0[3], Y0[3];
  for (int v = 0; v < 3; ++v) { X0[v] = (pb.vx[3 * t + v] - x0) / h0; Y0[v] = (pb.vy[3 * t + v] - y0) / h0; }
  double raw[6];
  basis_means(X0, Y0, 0, 0, 0, raw);
  const double M3 = raw[3], M4 = raw[4], M5 = raw[5];
  // stencil data
  double Xs[4][3], Ys[4][3], As[4];
  S Wb[4], Vb[4], Yb[4];
  for (int v = 0; v < 3; ++v) { Xs[0][v] = X0[v]; Ys[0][v] = Y0[v]; }
  As[0] = A0;
  Wb[0] = Uat(U, pb, 0, c, t); Vb[0] = Uat(U, pb, 1, c, t); Yb[0] = Uat(U, pb, 2, c, t);
  for (int l = 1; l <= 3; ++l) {
    double X[3], Y[3], a; int64_t src;
    stencil_member(pb, t, l, X, Y, a, src);
    for (int v = 0; v < 3; ++v) { Xs[l][v] = (X[v] - x0) / h0; Ys[l][v] = (Y[v] - y0) / h0; }
    As[l] = a;
    if (pb.nbr[t][l - 1] >= 0) {
      Wb[l] = Uat(U, pb, 0, c, src); Vb[l] = Uat(U, pb, 1, c, src); Yb[l] = Uat(U, pb, 2, c, src);
    } else {
      S gw[4], gv[4], gy[4];
      ghost_data(pb, U, t, l - 1, gw, gv, gy);
      Wb[l] = gw[c]; Vb[l] = gv[c]; Yb[l] = gy[c];
    }
  }
  double mean[4][6];
  for (int l = 0; l < 4; ++l) basis_means(Xs[l], Ys[l], M3, M4, M5, mean[l]);

  // ---- Step 1: p1.  c0 = Wbar_0 (K0 average, exact because the basis has
  // zero K0 mean).  Unknowns c1..c5.
  //   equality rows (l = 1..3):  sum_j c_j mean_l(phi_j) = Wbar_l - Wbar_0
  //   least-squares rows (l = 1..3), scaled by h0 (R3):
  //     h0 * mean_{K_l + K_0}(dp1/dx) = h0 (|K_l| Vbar_l + |K_0| Vbar_0) / (|K_l| + |K_0|)
  //     h0 * mean_{K_l + K_0}(dp1/dy) = h0 (|K_l| Ybar_l + |K_0| Ybar_0) / (|K_l| + |K_0|)
  // d(phi_j)/d(xi) = (0, 1, 0, 2 xi, eta, 0); d(phi_j)/d(eta) = (0, 0, 1, 0, xi, 2 eta):
  // their means over a triangle are those values at its barycenter.
  double Bm[6][5];
  S dvec[6];
  for (int l = 1; l <= 3; ++l) {
    double bxi[2], bet[2], w[2] = {As[l], As[0]};
    const int idx[2] = {l, 0};
    for (int q = 0; q < 2; ++q) {
      bxi[q] = (Xs[idx[q]][0] + Xs[idx[q]][1] + Xs[idx[q]][2]) / 3.0;
      bet[q] = (Ys[idx[q]][0] + Ys[idx[q]][1] + Ys[idx[q]][2]) / 3.0;
    }
    double rx[5] = {0, 0, 0, 0, 0}, ry[5] = {0, 0, 0, 0, 0};
    for (int q = 0; q < 2; ++q) {
      double f = w[q] / (w[0] + w[1]);
      rx[0] += f * 1.0; rx[2] += f * 2.0 * bxi[q]; rx[3] += f * bet[q];
      ry[1] += f * 1.0; ry[3] += f * bxi[q]; ry[4] += f * 2.0 * bet[q];
    }
    for (int j = 0; j < 5; ++j) { Bm[2 * (l - 1)][j] = rx[j]; Bm[2 * (l - 1) + 1][j] = ry[j]; }
    dvec[2 * (l - 1)] = S(h0) * (S(As[l]) * Vb[l] + S(As[0]) * Vb[0]) / S(As[l] + As[0]);
    dvec[2 * (l - 1) + 1] = S(h0) * (S(As[l]) * Yb[l] + S(As[0]) * Yb[0]) / S(As[l] + As[0]);
  }
  // KKT system [B^T B  C^T; C 0] [c; mu] = [B^T d; e]
  std::vector<double> K(64, 0.0);
  std::vector<S> rhs(8, S(0.0)), sol;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      double s = 0;
      for (int r = 0; r < 6; ++r) s += Bm[r][i] * Bm[r][j];
      K[i * 8 + j] = s;
    }
  for (int i = 0; i < 5; ++i) {
    S s(0.0);
    for (int r = 0; r < 6; ++r) s = s + S(Bm[r][i]) * dvec[r];
    rhs[i] = s;
  }
  for (int l = 1; l <= 3; ++l) {
    for (int j = 0; j < 5; ++j) {
      K[(4 + l) * 8 + j] = mean[l][j + 1];
      K[j * 8 + (4 + l)] = mean[l][j + 1];
    }
    rhs[4 + l] = Wb[l] - Wb[0] * S(mean[l][0]);
  }
  if (!gauss_solve(8, K, rhs, sol)) R.ok = false;
  Poly<S>& p1 = R.p[0];
  p1.x0 = x0; p1.y0 = y0; p1.h = h0; p1.M3 = M3; p1.M4 = M4; p1.M5 = M5;
  p1.c[0] = Wb[0];
  for (int j = 0; j < 5; ++j) p1.c[j + 1] = R.ok ? sol[j] : S(0.0);

  // ---- Step 2: p2, p3, p4, linear on {K0, K_l}; the K0 average holds by
  // construction (c0 = Wbar_0), the three remaining rows (scaled by h0, R3)
  //   c1 xibar_l + c2 etabar_l = Wbar_l - Wbar_0,  c1 = h0 Vbar_l,  c2 = h0 Ybar_l
  // are solved in the least-squares sense through the normal equations.
  for (int l = 1; l <= 3; ++l) {
    double xb = mean[l][1], eb = mean[l][2];
    double G[3][2] = {{xb, eb}, {1, 0}, {0, 1}};
    S r[3] = {Wb[l] - Wb[0], S(h0) * Vb[l], S(h0) * Yb[l]};
    std::vector<double> N(4, 0.0);
    std::vector<S> nb(2, S(0.0)), bsol;
    for (int i = 0; i < 2; ++i) {
      for (int j = 0; j < 2; ++j) for (int q = 0; q < 3; ++q) N[i * 2 + j] += G[q][i] * G[q][j];
      for (int q = 0; q < 3; ++q) nb[i] = nb[i] + S(G[q][i]) * r[q];
    }
    if (!gauss_solve(2, N, nb, bsol)) R.ok = false;
    Poly<S>& pl = R.p[l];
    pl.x0 = x0; pl.y0 = y0; pl.h = h0; pl.M3 = M3; pl.M4 = M4; pl.M5 = M5;
    pl.c[0] = Wb[0]; pl.c[1] = R.ok ? bsol[0] : S(0.0); pl.c[2] = R.ok ? bsol[1] : S(0.0);
    pl.c[3] = pl.c[4] = pl.c[5] = S(0.0);
  }

  // ---- Step 4: smoothness indicators (Eq. smoo1) in physical derivatives at
  // the barycenter (R6): beta = sum_{1<=|s|<=k} |K0|^{|s|} (d^s p)^2.
  for (int l = 0; l < 4; ++l) {
    S d[6];
    poly_eval(R.p[l], x0, y0, d);
    S b = S(A0) * (d[1] * d[1] + d[2] * d[2]);
    if (l == 0) b = b + S(A0 * A0) * (d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
    R.beta[l] = b;
  }
  // ---- Step 5: nonlinear weights (Eq. nonlinearweight), per component (R7).
  const double* g = pb.P.glin;
  if (pb.P.linear_only) {
    for (int l = 0; l < 4; ++l) R.omega[l] = S(g[l]);
  } else {
    S Wave = (Wb[0] + Wb[1] + Wb[2] + Wb[3]) / S(4.0) + S(1e-30);
    S tau = fabs(R.beta[0] - R.beta[1]) + fabs(R.beta[0] - R.beta[2]) + fabs(R.beta[0] - R.beta[3]);
    S kappa = tau * tau / S(9.0);
    S W2 = Wave * Wave, W4 = W2 * W2;
    S wb[4], sum(0.0);
    for (int l = 0; l < 4; ++l) {
      wb[l] = S(g[l]) * (S(1.0) + kappa / (W4 * S(pb.P.eps) + W2 * R.beta[l]));
      sum = sum + wb[l];
    }
    for (int l = 0; l < 4; ++l) R.omega[l] = wb[l] / sum;
  }
  return R;
}

const double kGLpt = 0.28867513459481288225;  // sqrt(3)/6: Gauss-Legendre points at 1/2 -+ kGLpt

// ---- Step 6 (Eq. recon): value and derivatives of the final reconstruction at
// the point (x, y) of t's frame, evaluated polynomial by polynomial.
template <class S> void recon_at(const CellRecon<S>& R, const double* g, double x, double y, S out[6]) {
  S v[4][6];
  for (int l = 0; l < 4; ++l) poly_eval(R.p[l], x, y, v[l]);
  for (int d = 0; d < 6; ++d) {
    S inner = v[0][d] / S(g[0]);
    for (int l = 1; l < 4; ++l) inner = inner - S(g[l] / g[0]) * v[l][d];
    S o = R.omega[0] * inner;
    for (int l = 1; l < 4; ++l) o = o + R.omega[l] * v[l][d];
    out[d] = o;
  }
  // scale limiter: W~ = Wbar + theta (W - Wbar), derivatives scaled by theta
  if (val(R.theta) != 1.0) {
    out[0] = R.wbar + R.theta * (out[0] - R.wbar);
    for (int d = 1; d < 6; ++d) out[d] = R.theta * out[d];
  }
}

// Pressure of a conservative state (Eq. 2d equation of state).
template <class S> S pressure(double gam, const S* W) {
  return S(gam - 1.0) * (W[3] - S(0.5) * (W[1] * W[1] + W[2] * W[2]) / W[0]);
}

// Largest f in [0, 1] with p(Wb + f d) >= eps along the segment from the cell
// average Wb (R18), by bisection on the pressure itself.  Where the density is
// positive the pressure is a concave function of the conservative variables,
// so the admissible part of the segment is an interval [0, f*] (p(Wb) > eps
// at its start); f* is where p first falls to eps.  The limiter is not
// differentiated (the adjoint excludes it), so the search runs on the values.
template <class S> S pressure_root(double gam, const S Wb[4], const S d[4], double eps) {
  auto p_at = [&](double f) {
    double w[4];
    for (int c = 0; c < 4; ++c) w[c] = val(Wb[c]) + f * val(d[c]);
    return (gam - 1.0) * (w[3] - 0.5 * (w[1] * w[1] + w[2] * w[2]) / w[0]);
  };
  if (p_at(1.0) >= eps) return S(1.0);
  double lo = 0.0, hi = 1.0;   // p_at(lo) >= eps > p_at(hi)
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;   // lo and hi are adjacent doubles
    if (p_at(mid) >= eps) lo = mid; else hi = mid;
  }
  return S(lo);
}

// Positivity-preserving scaling of Zhang and Shu (the "scale limiter" of
// Section 3), applied to the final reconstruction of one Euler cell (R18):
// over the six edge Gauss points, first scale the density part around its
// cell average so that it stays >= eps, then scale all components so that the
// pressure stays >= eps, eps = min(1e-13, rho_bar, p_bar).
template <class S> void positivity_scaling(const Problem& pb, CellRecon<S>* rec, int64_t t) {
  const double gam = pb.P.gam;
  S Wb[4];
  for (int c = 0; c < 4; ++c) Wb[c] = rec[c].wbar;
  const S pb0 = pressure(gam, Wb);
  if (!(val(Wb[0]) > 0) || !(val(pb0) > 0)) return;  // the average itself is not admissible
  const double eps = std::min(1e-13, std::min(val(Wb[0]), val(pb0)));
  S q[6][4];
  for (int j = 0; j < 3; ++j)
    for (int gi = 0; gi < 2; ++gi) {
      const double s = (gi == 0) ? 0.5 - kGLpt : 0.5 + kGLpt;
      const double Ax = pb.vx[3 * t + j], Ay = pb.vy[3 * t + j];
      const double Bx = pb.vx[3 * t + (j + 1) % 3], By = pb.vy[3 * t + (j + 1) % 3];
      for (int c = 0; c < 4; ++c) {
        S o[6];
        recon_at(rec[c], pb.P.glin, Ax + s * (Bx - Ax), Ay + s * (By - Ay), o);
        q[2 * j + gi][c] = o[0];
      }
    }
  // density
  S rmin = q[0][0];
  for (int k = 1; k < 6; ++k) if (val(q[k][0]) < val(rmin)) rmin = q[k][0];
  S th1 = S(1.0);
  if (val(rmin) < eps) th1 = (Wb[0] - S(eps)) / (Wb[0] - rmin);
  // pressure along the segment from the average to each limited point value
  S th2 = S(1.0);
  for (int k = 0; k < 6; ++k) {
    S w[4] = {Wb[0] + th1 * (q[k][0] - Wb[0]), q[k][1], q[k][2], q[k][3]};
    if (val(pressure(gam, w)) >= eps) continue;
    S d[4];
    for (int c = 0; c < 4; ++c) d[c] = w[c] - Wb[c];
    const S tk = pressure_root(gam, Wb, d, eps);
    if (val(tk) < val(th2)) th2 = tk;
  }
  rec[0].theta = th1 * th2;
  for (int c = 1; c < 4; ++c) rec[c].theta = th2;
}

// ------------------------------------------------------------------ fluxes
// f(W), g(W) of the equation (Eq. 2 with Eq. 2d for Euler), for any scalar T.
template <class T> void flux_fg(const Params& P, const T* W, T* f, T* g) {
  if (P.eq == EQ_ADVECTION) {
    f[0] = P.ax * W[0];
    g[0] = P.ay * W[0];
  } else if (P.eq == EQ_BURGERS) {
    f[0] = 0.5 * (W[0] * W[0]);
    g[0] = f[0];
  } else {
    const T &rho = W[0], &mx = W[1], &my = W[2], &E = W[3];
    T u = mx / rho, v = my / rho;
    T p = (P.gam - 1.0) * (E - 0.5 * (mx * u + my * v));
    f[0] = mx; f[1] = mx * u + p; f[2] = my * u; f[3] = (E + p) * u;
    g[0] = my; g[1] = mx * v; g[2] = my * v + p; g[3] = (E + p) * v;
  }
}

// Directional derivatives of f and g at W:  f'a, f'b, f''[a]b (and g).
template <class S>
void flux_derivs(const Params& P, const S* W, const S* a, const S* b, S* fa, S* fb, S* fab, S* ga, S* gb, S* gab) {
  const int m = P.m;
  HD<S> Wh[4], fh[4], gh[4];
  for (int c = 0; c < m; ++c) Wh[c] = HD<S>{W[c], a[c], b[c], S(0.0)};
  flux_fg(P, Wh, fh, gh);
  for (int c = 0; c < m; ++c) {
    fa[c] = fh[c].a; fb[c] = fh[c].b; fab[c] = fh[c].ab;
    ga[c] = gh[c].a; gb[c] = gh[c].b; gab[c] = gh[c].ab;
  }
}

// Lax-Wendroff procedure of Section 2.1: from the spatial jet
// J[d][c], d = (W, Wx, Wy, Wxx, Wxy, Wyy), compute Wt, Wtx, Wty, Wtt.
template <class S> void lax_wendroff(const Params& P, const S J[6][4], S Wt[4], S Wtx[4], S Wty[4], S Wtt[4]) {
  const int m = P.m;
  const S *W = J[0], *Wx = J[1], *Wy = J[2], *Wxx = J[3], *Wxy = J[4], *Wyy = J[5];
  S fa[4], fb[4], fab[4], ga[4], gb[4], gab[4];
  // Wt = -(f' Wx + g' Wy)
  S fWx[4], gWy[4];
  flux_derivs(P, W, Wx, Wy, fWx, fb, fab, ga, gWy, gab);
  for (int c = 0; c < m; ++c) Wt[c] = S(0.0) - (fWx[c] + gWy[c]);
  // Wtx = -(f''[Wx]Wx + f' Wxx + g''[Wx]Wy + g' Wxy)
  S fxx[4], gxy[4], fWxx[4], gWxy[4];
  flux_derivs(P, W, Wx, Wx, fa, fb, fxx, ga, gb, gab);  // f''[Wx]Wx
  flux_derivs(P, W, Wx, Wy, fa, fb, fab, ga, gb, gxy);   // gab = g''[Wx]Wy
  flux_derivs(P, W, Wxx, Wxy, fWxx, fb, fab, ga, gWxy, gab);
  for (int c = 0; c < m; ++c) Wtx[c] = S(0.0) - (fxx[c] + fWxx[c] + gxy[c] + gWxy[c]);
  // Wty = -(f''[Wy]Wx + f' Wxy + g''[Wy]Wy + g' Wyy)
  S fyx[4], gyy[4], fWxy[4], gWyy[4];
  flux_derivs(P, W, Wy, Wx, fa, fb, fyx, ga, gb, gab);   // f''[Wy]Wx
  flux_derivs(P, W, Wy, Wy, fa, fb, fab, ga, gb, gyy);   // g''[Wy]Wy
  flux_derivs(P, W, Wxy, Wyy, fWxy, fb, fab, ga, gWyy, gab);
  for (int c = 0; c < m; ++c) Wty[c] = S(0.0) - (fyx[c] + fWxy[c] + gyy[c] + gWyy[c]);
  // Wtt = -(f''[Wt]Wx + f' Wtx + g''[Wt]Wy + g' Wty)
  S ftx[4], gty[4], fWtx[4], gWty[4];
  flux_derivs(P, W, Wt, Wx, fa, fb, ftx, ga, gb, gab);   // f''[Wt]Wx
  flux_derivs(P, W, Wt, Wy, fa, fb, fab, ga, gb, gty);   // g''[Wt]Wy
  flux_derivs(P, W, Wtx, Wty, fWtx, fb, fab, ga, gWty, gab);
  for (int c = 0; c < m; ++c) Wtt[c] = S(0.0) - (ftx[c] + fWtx[c] + gty[c] + gWty[c]);
}

// F(W) . n for the local Lax-Friedrichs flux
template <class S> void flux_normal(const Params& P, const S* W, double nx, double ny, S* H) {
  S f[4], g[4];
  flux_fg(P, W, f, g);
  for (int c = 0; c < P.m; ++c) H[c] = f[c] * S(nx) + g[c] * S(ny);
}

// largest eigenvalue in magnitude of d(F.n)/dW at W (R10)
template <class S> S spectral_radius_n(const Params& P, const S* W, double nx, double ny) {
  if (P.eq == EQ_ADVECTION) return S(std::fabs(P.ax * nx + P.ay * ny));
  if (P.eq == EQ_BURGERS) return fabs(W[0] * S(nx + ny));
  S u = W[1] / W[0], v = W[2] / W[0];
  S p = S(P.gam - 1.0) * (W[3] - S(0.5) * (W[1] * u + W[2] * v));
  S cs = sqrt(S(P.gam) * p / W[0]);
  return fabs(u * S(nx) + v * S(ny)) + cs;
}

// spectral radius over all directions (R12)
double spectral_radius_all(const Params& P, const double* W) {
  if (P.eq == EQ_ADVECTION) return std::sqrt(P.ax * P.ax + P.ay * P.ay);
  if (P.eq == EQ_BURGERS) return std::sqrt(2.0) * std::fabs(W[0]);
  double u = W[1] / W[0], v = W[2] / W[0];
  double p = (P.gam - 1.0) * (W[3] - 0.5 * (W[1] * u + W[2] * v));
  return std::sqrt(u * u + v * v) + std::sqrt(P.gam * p / W[0]);
}

// ------------------------------------------------------------------ one step
const double kGL = 0.28867513459481288225;  // sqrt(3)/6
const double kTau[3] = {0.0, 0.5, 1.0};                  // R2: Lobatto nodes
const double kWt[3] = {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0};  // R2: Lobatto weights
const double kTauGL[2] = {0.5 - kGL, 0.5 + kGL};          // R22: Gauss-Legendre nodes
const double kWtGL[2] = {0.5, 0.5};                       // R22: Gauss-Legendre weights

// Taylor data (W, Wt, Wtt) at the point (x, y) of a cell's own frame from the
// cell's reconstructions rec[0..m-1] (Eq. recon, then Section 2.1).
template <class S>
void side_taylor(const Problem& pb, const CellRecon<S>* rec, double x, double y, S W[4], S Wt[4], S Wtt[4]) {
  const int m = pb.P.m;
  S J[6][4];
  for (int c = 0; c < m; ++c) {
    S o[6];
    recon_at(rec[c], pb.P.glin, x, y, o);
    for (int d = 0; d < 6; ++d) J[d][c] = o[d];
  }
  S Wtx[4], Wty[4];
  lax_wendroff(pb.P, J, Wt, Wtx, Wty, Wtt);
  for (int c = 0; c < m; ++c) W[c] = J[0][c];
  // limiter on the space-time Taylor data (R18): scale toward the average
  if (val(rec[0].theta_t) != 1.0)
    for (int c = 0; c < m; ++c) {
      W[c] = rec[c].wbar + rec[c].theta_t * (W[c] - rec[c].wbar);
      Wt[c] = rec[c].theta_t * Wt[c];
      Wtt[c] = rec[c].theta_t * Wtt[c];
    }
}

// Largest f in [0, 1] with rho, p >= eps on Wb + f (w - Wb): density first,
// then pressure through the quadratic in f (R18).
template <class S> S admissible_fraction(double gam, const S Wb[4], const S w[4], double eps) {
  S f1 = S(1.0);
  if (val(w[0]) < eps) f1 = (Wb[0] - S(eps)) / (Wb[0] - w[0]);
  S d[4];
  for (int c = 0; c < 4; ++c) d[c] = f1 * (w[c] - Wb[c]);
  S v[4];
  for (int c = 0; c < 4; ++c) v[c] = Wb[c] + d[c];
  if (val(pressure(gam, v)) >= eps) return f1;
  const S tk = pressure_root(gam, Wb, d, eps);
  return f1 * tk;
}

// Limiter on the space-time data of one Euler cell: the Taylor values at its
// six edge Gauss points and the three Lobatto time nodes are pulled toward the
// cell average by one common factor so that rho, p >= eps at all of them.
template <class S> void positivity_time_scaling(const Problem& pb, CellRecon<S>* rec, int64_t t, double dt) {
  const double gam = pb.P.gam;
  S Wb[4];
  for (int c = 0; c < 4; ++c) Wb[c] = rec[c].wbar;
  const S pb0 = pressure(gam, Wb);
  if (!(val(Wb[0]) > 0) || !(val(pb0) > 0)) return;
  const double eps = std::min(1e-13, std::min(val(Wb[0]), val(pb0)));
  S th = S(1.0);
  for (int j = 0; j < 3; ++j)
    for (int gi = 0; gi < 2; ++gi) {
      const double s = (gi == 0) ? 0.5 - kGLpt : 0.5 + kGLpt;
      const double Ax = pb.vx[3 * t + j], Ay = pb.vy[3 * t + j];
      const double Bx = pb.vx[3 * t + (j + 1) % 3], By = pb.vy[3 * t + (j + 1) % 3];
      S W[4], Wt[4], Wtt[4];
      side_taylor(pb, rec, Ax + s * (Bx - Ax), Ay + s * (By - Ay), W, Wt, Wtt);
      for (int si = 0; si < 3; ++si) {
        const double tau = kTau[si] * dt;
        S w[4];
        for (int c = 0; c < 4; ++c) w[c] = W[c] + Wt[c] * S(tau) + Wtt[c] * S(0.5 * tau * tau);
        const S f = admissible_fraction(gam, Wb, w, eps);
        if (val(f) < val(th)) th = f;
      }
    }
  for (int c = 0; c < 4; ++c) rec[c].theta_t = th;
}

// Positivity-preserving flux blending (R23, with the scale limiter, Euler).
// The scale limiter keeps the point values admissible, but a one-step (ADER)
// update built from time-Taylor values is not a convex combination of them, so
// the new cell averages can still lose positivity.  Following Hu, Adams and
// Shu (2013), each cell average is written as
//   Wbar^{n+1} = sum_e (|e| / P) Phi_e,
//   Phi_e = Wbar - (dt P / |K|) (Fhat_e - F(Wbar) . n_e)
// (P the perimeter; sum_e |e| n_e = 0), and the edge flux is replaced by
// Fhat = FL + theta (FH - FL), FL the first-order local Lax-Friedrichs flux of
// the two cell averages (WL, WR; on a boundary WR is the ghost's) with the same alpha, theta in [0, 1] the largest value
// that keeps Phi_e admissible on both sides of the edge (the scale limiter's
// fraction along the segment from Phi_e(0) to Phi_e(1)).  Both sides use the
// same theta, so the update stays conservative.  Fe is the high-order edge
// flux times |e| on entry and the blended one on exit.
template <class S>
void flux_blend(const Problem& pb, const S* WL, const S* WR, const EdgeRec& e, S alpha, double dt, S Fe[4]) {
  const double gam = pb.P.gam;
  S HL[4], HR[4], FL[4], FH[4];
  flux_normal(pb.P, WL, e.nx, e.ny, HL);
  flux_normal(pb.P, WR, e.nx, e.ny, HR);
  for (int c = 0; c < 4; ++c) {
    FL[c] = S(0.5) * (HL[c] + HR[c] - alpha * (WR[c] - WL[c]));
    FH[c] = Fe[c] / S(e.len);
  }
  S theta = S(1.0);
  for (int side = 0; side < (e.R >= 0 ? 2 : 1); ++side) {
    const int64_t k = side == 0 ? e.L : e.R;
    const S* Wk = side == 0 ? WL : WR;
    const S* Hk = side == 0 ? HL : HR;
    const double sg = side == 0 ? 1.0 : -1.0;   // the edge normal is outward for L, inward for R
    const S pk = pressure(gam, Wk);
    if (!(val(Wk[0]) > 0) || !(val(pk) > 0)) continue;   // the average itself is not admissible
    const double eps = std::min(1e-13, std::min(val(Wk[0]), val(pk)));
    const S lam = S(sg * dt * pb.perim[k] / pb.area[k]);
    S phi0[4], phi1[4];
    for (int c = 0; c < 4; ++c) {
      phi0[c] = Wk[c] - lam * (FL[c] - Hk[c]);
      phi1[c] = Wk[c] - lam * (FH[c] - Hk[c]);
    }
    S th = S(0.0);
    if (val(phi0[0]) >= eps && val(pressure(gam, phi0)) >= eps) th = admissible_fraction(gam, phi0, phi1, eps);
    if (val(th) < val(theta)) theta = th;
  }
  if (val(theta) < 1.0)
    for (int c = 0; c < 4; ++c) Fe[c] = S(e.len) * (FL[c] + theta * (FH[c] - FL[c]));
}

// One time step for the cells `targets` (ascending, all cells for a full
// step): out[(k m + c) nout + r] = new value of (k, c) of targets[r].  Each
// target's three edges are processed once per edge, in the order of the edge
// list (an edge is formed when its first cell comes up), so a full step forms
// every edge flux once, in the edge-list order.  The cost is proportional to
// the number of targets.
template <class S>
int step_cells(const Problem& pb, const S* U, double dt, const std::vector<int64_t>& targets, S* out) {
  const int m = pb.P.m;
  const int64_t nout = (int64_t)targets.size();
  const bool all = nout == pb.nt;
  // positions of the targets and of the cells to reconstruct (targets and neighbours)
  std::unordered_map<int64_t, int64_t> tpos, slot;
  std::vector<int64_t> need;
  auto tslot = [&](int64_t i) -> int64_t {
    if (all) return i;
    auto it = tpos.find(i);
    return it == tpos.end() ? -1 : it->second;
  };
  if (!all) for (int64_t r = 0; r < nout; ++r) tpos[targets[r]] = r;
  auto add_need = [&](int64_t i) {
    if (all) return;
    if (slot.emplace(i, (int64_t)need.size()).second) need.push_back(i);
  };
  for (int64_t i : targets) {
    add_need(i);
    for (int j = 0; j < 3; ++j) if (pb.nbr[i][j] >= 0) add_need(pb.nbr[i][j]);
  }
  auto rslot = [&](int64_t i) -> int64_t { return all ? i : slot.at(i); };
  const int64_t nneed = all ? pb.nt : (int64_t)need.size();
  std::vector<CellRecon<S>> rec(nneed * m);
  for (int64_t k = 0; k < nneed; ++k) {
    const int64_t i = all ? k : need[k];
    for (int c = 0; c < m; ++c) {
      rec[k * m + c] = reconstruct(pb, U, i, c);
      if (!rec[k * m + c].ok) { g_err = "singular reconstruction system"; return 4; }
    }
    if (pb.P.positivity && pb.P.eq == EQ_EULER) {
      positivity_scaling(pb, &rec[k * m], i);
      positivity_time_scaling(pb, &rec[k * m], i, dt);
    }
  }
  std::vector<S> Rf(nout * m, S(0.0)), GV(nout * m, S(0.0)), GY(nout * m, S(0.0));
  for (int64_t i : targets)
    for (int j = 0; j < 3; ++j) {
      const EdgeRec& e = pb.edges[pb.cell_edge[i][j]];
      // form the edge once: when its L cell comes up, or its R cell if L is not a target
      if (!(e.L == i || tslot(e.L) < 0)) continue;
      const int64_t sL = tslot(e.L), sR = e.R >= 0 ? tslot(e.R) : -1;
      S Fe[4], Se[4];
      for (int c = 0; c < m; ++c) { Fe[c] = S(0.0); Se[c] = S(0.0); }
      // alpha from the cell averages of both sides (R10)
      S WL[4], WR[4];
      for (int c = 0; c < m; ++c) {
        WL[c] = Uat(U, pb, 0, c, e.L);
        WR[c] = Uat(U, pb, 0, c, e.R >= 0 ? e.R : e.L);
      }
      if (e.R < 0) {   // the ghost's average (R13, R25)
        S gv[4], gy[4];
        ghost_data(pb, U, e.L, e.jL, WR, gv, gy);
      }
      S alpha = smax(spectral_radius_n(pb.P, WL, e.nx, e.ny), spectral_radius_n(pb.P, WR, e.nx, e.ny));
      for (int gi = 0; gi < 2; ++gi) {
        double s = (gi == 0) ? 0.5 - kGL : 0.5 + kGL;
        double x = e.Ax + s * (e.Bx - e.Ax), y = e.Ay + s * (e.By - e.Ay);
        S Wi[4], Wti[4], Wtti[4], We[4], Wte[4], Wtte[4];
        side_taylor(pb, rec.data() + rslot(e.L) * m, x, y, Wi, Wti, Wtti);
        if (e.R >= 0) {
          side_taylor(pb, rec.data() + rslot(e.R) * m, x - e.sx, y - e.sy, We, Wte, Wtte);
        } else {
          // boundary: the ghost's Taylor data at the edge point (R13, R25)
          const int type = pb.ebc[e.L][e.jL];
          if (type == BC_INFLOW) {
            for (int c = 0; c < m; ++c) { We[c] = S(pb.win[c]); Wte[c] = S(0.0); Wtte[c] = S(0.0); }
          } else if (type == BC_REFLECTIVE && pb.P.eq == EQ_EULER) {
            mirror_state(e.nx, e.ny, Wi, We);      // the mirrored solution at a point of the wall
            mirror_state(e.nx, e.ny, Wti, Wte);
            mirror_state(e.nx, e.ny, Wtti, Wtte);
          } else {
            for (int c = 0; c < m; ++c) { We[c] = Wi[c]; Wte[c] = Wti[c]; Wtte[c] = Wtti[c]; }
          }
        }
        // Eqs. tay / tayext at the time nodes, LLF flux, time quadrature (Eq. flux)
        const bool gauss = pb.P.time_rule == 1;
        for (int si = 0; si < (gauss ? 2 : 3); ++si) {
          double tau = (gauss ? kTauGL[si] : kTau[si]) * dt;
          S a[4], b[4], Ha[4], Hb[4];
          for (int c = 0; c < m; ++c) {
            a[c] = Wi[c] + Wti[c] * S(tau) + Wtti[c] * S(0.5 * tau * tau);
            b[c] = We[c] + Wte[c] * S(tau) + Wtte[c] * S(0.5 * tau * tau);
          }
          flux_normal(pb.P, a, e.nx, e.ny, Ha);
          flux_normal(pb.P, b, e.nx, e.ny, Hb);
          for (int c = 0; c < m; ++c) {
            S H = S(0.5) * (Hb[c] + Ha[c] - alpha * (b[c] - a[c]));
            Fe[c] = Fe[c] + S((gauss ? kWtGL[si] : kWt[si]) * 0.5 * e.len) * H;  // w_s * w_G * |e|
          }
          if (!gauss && si == 2) {
            // Eq. timeflux: central value at t_{n+1} (Lobatto node tau = dt)
            for (int c = 0; c < m; ++c) Se[c] = Se[c] + S(0.5 * e.len) * (S(0.5) * (a[c] + b[c]));
          }
        }
        if (gauss) {
          // Eq. timeflux: the central value at t_{n+1} from its own Taylor evaluation
          S a[4], b[4];
          for (int c = 0; c < m; ++c) {
            a[c] = Wi[c] + Wti[c] * S(dt) + Wtti[c] * S(0.5 * dt * dt);
            b[c] = We[c] + Wte[c] * S(dt) + Wtte[c] * S(0.5 * dt * dt);
            Se[c] = Se[c] + S(0.5 * e.len) * (S(0.5) * (a[c] + b[c]));
          }
        }
      }
      if (pb.P.positivity == 1 && pb.P.eq == EQ_EULER) flux_blend(pb, WL, WR, e, alpha, dt, Fe);
      for (int c = 0; c < m; ++c) {
        if (sL >= 0) {
          Rf[sL * m + c] = Rf[sL * m + c] + Fe[c];
          GV[sL * m + c] = GV[sL * m + c] + Se[c] * S(e.nx);
          GY[sL * m + c] = GY[sL * m + c] + Se[c] * S(e.ny);
        }
        if (sR >= 0) {
          Rf[sR * m + c] = Rf[sR * m + c] - Fe[c];
          GV[sR * m + c] = GV[sR * m + c] - Se[c] * S(e.nx);
          GY[sR * m + c] = GY[sR * m + c] - Se[c] * S(e.ny);
        }
      }
      }
  // Eq. flx and Eq. derave2d2
  for (int64_t r = 0; r < nout; ++r) {
    const int64_t i = targets[r];
    for (int c = 0; c < m; ++c) {
      out[(0 * m + c) * nout + r] = Uat(U, pb, 0, c, i) - S(dt / pb.area[i]) * Rf[r * m + c];
      out[(1 * m + c) * nout + r] = GV[r * m + c] / S(pb.area[i]);
      out[(2 * m + c) * nout + r] = GY[r * m + c] / S(pb.area[i]);
    }
  }
  return 0;
}

// One time step of all cells, or (mask non-null) of the cells with
// mask[i] != 0, whose new values are written while the others are copied.
template <class S> int step_impl(const Problem& pb, const S* U, double dt, S* Unew, const uint8_t* mask) {
  const int m = pb.P.m;
  const int64_t nt = pb.nt;
  std::vector<int64_t> targets;
  for (int64_t i = 0; i < nt; ++i) if (!mask || mask[i]) targets.push_back(i);
  std::vector<S> out(3 * m * targets.size());
  const int rc = step_cells(pb, U, dt, targets, out.data());
  if (rc) return rc;
  if (mask) std::copy(U, U + 3 * m * nt, Unew);
  const int64_t nout = (int64_t)targets.size();
  for (int k = 0; k < 3 * m; ++k)
    for (int64_t r = 0; r < nout; ++r) Unew[k * nt + targets[r]] = out[k * nout + r];
  return 0;
}

double cfl_dt(const Problem& pb, const double* U) {
  double best = 1e300;
  for (int64_t i = 0; i < pb.nt; ++i) {
    double W[4];
    for (int c = 0; c < pb.P.m; ++c) W[c] = U[c * pb.nt + i];
    double lam = spectral_radius_all(pb.P, W);
    if (lam > 0) best = std::min(best, pb.inr[i] / lam);
  }
  return pb.P.cfl * best;
}

}  // namespace

// ====================================================================== C API
extern "C" {

typedef struct orc_problem orc_problem;

const char* orc_last_error(void) { return g_err.c_str(); }

int orc_create(const double* xy, int64_t nv, const int32_t* tri, int64_t nt, double Lx, double Ly, int bc,
               int eq, double ax, double ay, double gam, double cfl, const double* glin, double eps,
               int linear_only, orc_problem** out) {
  if (!xy || !tri || nt <= 0 || nv <= 0 || !out) { g_err = "bad arguments"; return 1; }
  if (eq < 0 || eq > 2) { g_err = "bad equation"; return 1; }
  Problem* pb = new Problem();
  pb->nv = nv; pb->nt = nt; pb->Lx = Lx; pb->Ly = Ly; pb->bc = bc;
  pb->P.eq = eq; pb->P.m = (eq == EQ_EULER) ? 4 : 1;
  pb->P.ax = ax; pb->P.ay = ay; pb->P.gam = gam; pb->P.cfl = cfl;
  for (int l = 0; l < 4; ++l) pb->P.glin[l] = glin ? glin[l] : (l == 0 ? 0.94 : 0.02);
  pb->P.eps = eps; pb->P.linear_only = linear_only; pb->P.positivity = 0; pb->P.time_rule = 0;
  for (int64_t i = 0; i < 3 * nt; ++i)
    if (tri[i] < 0 || tri[i] >= nv) { g_err = "vertex index out of range"; delete pb; return 4; }
  if (!build_connectivity(*pb, tri) || !build_geometry(*pb, xy, tri)) { delete pb; return 4; }
  *out = reinterpret_cast<orc_problem*>(pb);
  return 0;
}

void orc_destroy(orc_problem* p) { delete reinterpret_cast<Problem*>(p); }

// Positivity: 0 off; 1 the scale limiter (R18) with the flux blending (R23);
// 2 the scale limiter alone (the literal reading of Section 3, for tests).
int orc_set_positivity(orc_problem* p, int on) {
  if (on < 0 || on > 2) { g_err = "positivity must be 0, 1 or 2"; return 1; }
  reinterpret_cast<Problem*>(p)->P.positivity = on;
  return 0;
}

// Boundary types (R13, R25): edge_bc[3 t + j] for local edge j of cell t, read
// where the edge is on the boundary: 1 transmissive, 2 reflective, 3 inflow.
int orc_set_boundary(orc_problem* p, const int32_t* edge_bc) {
  Problem* pb = reinterpret_cast<Problem*>(p);
  for (int64_t t = 0; t < pb->nt; ++t)
    for (int j = 0; j < 3; ++j) {
      if (pb->nbr[t][j] >= 0) continue;
      const int b = edge_bc[3 * t + j];
      if (b < BC_TRANSMISSIVE || b > BC_INFLOW) { g_err = "boundary type must be 1, 2 or 3"; return 1; }
      pb->ebc[t][j] = b;
    }
  return 0;
}

// The state imposed at inflow edges (conservative variables, m values).
int orc_set_inflow(orc_problem* p, const double* W) {
  Problem* pb = reinterpret_cast<Problem*>(p);
  for (int c = 0; c < pb->P.m; ++c) pb->win[c] = W[c];
  return 0;
}

// Time rule of the edge flux: 0 three-node Gauss-Lobatto (R2), 1 two-node
// Gauss-Legendre (R22).
int orc_set_time_rule(orc_problem* p, int rule) {
  if (rule != 0 && rule != 1) { g_err = "time rule must be 0 or 1"; return 1; }
  reinterpret_cast<Problem*>(p)->P.time_rule = rule;
  return 0;
}

int orc_neighbors(const orc_problem* p, int32_t* nbr, int32_t* nbe) {
  const Problem* pb = reinterpret_cast<const Problem*>(p);
  for (int64_t t = 0; t < pb->nt; ++t)
    for (int j = 0; j < 3; ++j) {
      nbr[3 * t + j] = pb->nbr[t][j];
      if (nbe) nbe[3 * t + j] = pb->nbe[t][j];
    }
  return 0;
}

// per-cell geometry: area, barycenter x, y, inradius  -> out[4][nt]
int orc_cell_geometry(const orc_problem* p, double* out) {
  const Problem* pb = reinterpret_cast<const Problem*>(p);
  for (int64_t t = 0; t < pb->nt; ++t) {
    out[t] = pb->area[t]; out[pb->nt + t] = pb->cx[t]; out[2 * pb->nt + t] = pb->cy[t]; out[3 * pb->nt + t] = pb->inr[t];
  }
  return 0;
}

double orc_cfl_dt(const orc_problem* p, const double* U) { return cfl_dt(*reinterpret_cast<const Problem*>(p), U); }

int orc_step(const orc_problem* p, const double* U, double dt, double* Unew, const uint8_t* mask) {
  return step_impl<double>(*reinterpret_cast<const Problem*>(p), U, dt, Unew, mask);
}

// One step of the cells `cells` only (ascending caller indices): out[3][m][n]
// receives their new values.  The cost grows with n, not with the mesh.
int orc_step_cells(const orc_problem* p, const double* U, double dt, const int64_t* cells, int64_t n, double* out) {
  std::vector<int64_t> t(cells, cells + n);
  return step_cells<double>(*reinterpret_cast<const Problem*>(p), U, dt, t, out);
}

// Run from t0 to T with the CFL time step (R12).  U is updated in place.
// dts (optional, capacity max_steps) receives the time steps taken.
int orc_run_to(const orc_problem* p, double* U, double t0, double T, int64_t max_steps, int64_t* nsteps, double* dts) {
  const Problem* pb = reinterpret_cast<const Problem*>(p);
  const int64_t n = 3 * pb->P.m * pb->nt;
  std::vector<double> tmp(n);
  double t = t0;
  int64_t k = 0;
  while (t < T * (1.0 - 1e-14) && k < max_steps) {
    double dt = cfl_dt(*pb, U);
    if (t + dt > T) dt = T - t;
    int rc = step_impl<double>(*pb, U, dt, tmp.data(), nullptr);
    if (rc) return rc;
    std::memcpy(U, tmp.data(), n * sizeof(double));
    if (dts) dts[k] = dt;
    t += dt;
    ++k;
  }
  *nsteps = k;
  return 0;
}

// Advance with a prescribed sequence of time steps (no CFL), carrying a
// forward-mode tangent dU alongside U: on exit U holds the state and dU the
// exact directional derivative of the discrete map along the initial dU.
int orc_run_dual(const orc_problem* p, double* U, double* dU, const double* dts, int64_t nsteps) {
  const Problem* pb = reinterpret_cast<const Problem*>(p);
  const int64_t n = 3 * pb->P.m * pb->nt;
  std::vector<Dual> a(n), b(n);
  for (int64_t i = 0; i < n; ++i) a[i] = Dual(U[i], dU[i]);
  for (int64_t k = 0; k < nsteps; ++k) {
    int rc = step_impl<Dual>(*pb, a.data(), dts[k], b.data(), nullptr);
    if (rc) return rc;
    a.swap(b);
  }
  for (int64_t i = 0; i < n; ++i) { U[i] = a[i].v; dU[i] = a[i].d; }
  return 0;
}

// Diagnostics of the reconstruction of component c of cell t.
//   polys[4][6][6]: p1..p4 value and derivatives (W, Wx, Wy, Wxx, Wxy, Wyy) at
//                   the 6 edge Gauss points (edge j, point g -> index 2j+g)
//   recon[6][6]   : final reconstruction (Eq. recon) at the same points
//   beta[4], omega[4]
//   gp[6][2]      : the Gauss point coordinates (t's frame)
int orc_reconstruct_cell(const orc_problem* p, const double* U, int64_t t, int c, double* polys, double* recon,
                         double* beta, double* omega, double* gp) {
  const Problem* pb = reinterpret_cast<const Problem*>(p);
  CellRecon<double> R = reconstruct<double>(*pb, U, t, c);
  if (!R.ok) { g_err = "singular reconstruction system"; return 4; }
  for (int j = 0; j < 3; ++j)
    for (int gi = 0; gi < 2; ++gi) {
      double s = (gi == 0) ? 0.5 - kGL : 0.5 + kGL;
      double Ax = pb->vx[3 * t + j], Ay = pb->vy[3 * t + j];
      double Bx = pb->vx[3 * t + (j + 1) % 3], By = pb->vy[3 * t + (j + 1) % 3];
      double x = Ax + s * (Bx - Ax), y = Ay + s * (By - Ay);
      int q = 2 * j + gi;
      if (gp) { gp[2 * q] = x; gp[2 * q + 1] = y; }
      for (int l = 0; l < 4; ++l) {
        double o[6];
        poly_eval(R.p[l], x, y, o);
        for (int d = 0; d < 6; ++d) polys[(l * 6 + q) * 6 + d] = o[d];
      }
      double o[6];
      recon_at(R, pb->P.glin, x, y, o);
      for (int d = 0; d < 6; ++d) recon[q * 6 + d] = o[d];
    }
  for (int l = 0; l < 4; ++l) { beta[l] = R.beta[l]; omega[l] = R.omega[l]; }
  return 0;
}

// Taylor data (W, Wt, Wtt) at the six edge Gauss points of cell t for a step
// of size dt, after the limiter when it is on: out[6][3][m].
int orc_cell_taylor(const orc_problem* p, const double* U, double dt, int64_t t, double* out) {
  const Problem* pb = reinterpret_cast<const Problem*>(p);
  const int m = pb->P.m;
  std::vector<CellRecon<double>> rec(m);
  for (int c = 0; c < m; ++c) {
    rec[c] = reconstruct<double>(*pb, U, t, c);
    if (!rec[c].ok) { g_err = "singular reconstruction system"; return 4; }
  }
  if (pb->P.positivity && pb->P.eq == EQ_EULER) {
    positivity_scaling(*pb, rec.data(), t);
    positivity_time_scaling(*pb, rec.data(), t, dt);
  }
  for (int j = 0; j < 3; ++j)
    for (int gi = 0; gi < 2; ++gi) {
      const double s = (gi == 0) ? 0.5 - kGL : 0.5 + kGL;
      const double Ax = pb->vx[3 * t + j], Ay = pb->vy[3 * t + j];
      const double Bx = pb->vx[3 * t + (j + 1) % 3], By = pb->vy[3 * t + (j + 1) % 3];
      double W[4], Wt[4], Wtt[4];
      side_taylor(*pb, rec.data(), Ax + s * (Bx - Ax), Ay + s * (By - Ay), W, Wt, Wtt);
      const int q = 2 * j + gi;
      for (int c = 0; c < m; ++c) {
        out[(q * 3 + 0) * m + c] = W[c];
        out[(q * 3 + 1) * m + c] = Wt[c];
        out[(q * 3 + 2) * m + c] = Wtt[c];
      }
    }
  return 0;
}

// Lax-Wendroff procedure at one point: jet[6][m] -> out[4][m] = Wt, Wtx, Wty, Wtt
int orc_lax_wendroff(int eq, double ax, double ay, double gam, const double* jet, double* out) {
  Params P{};
  P.eq = eq; P.m = (eq == EQ_EULER) ? 4 : 1; P.ax = ax; P.ay = ay; P.gam = gam;
  double J[6][4], Wt[4], Wtx[4], Wty[4], Wtt[4];
  for (int d = 0; d < 6; ++d) for (int c = 0; c < P.m; ++c) J[d][c] = jet[d * P.m + c];
  lax_wendroff<double>(P, J, Wt, Wtx, Wty, Wtt);
  for (int c = 0; c < P.m; ++c) {
    out[c] = Wt[c]; out[P.m + c] = Wtx[c]; out[2 * P.m + c] = Wty[c]; out[3 * P.m + c] = Wtt[c];
  }
  return 0;
}

// Spectral radii at W (R10, R12): out[0] = largest |eigenvalue| of
// d(F.n)/dW for the unit normal (nx, ny), out[1] = the largest over all
// directions.
int orc_spectral_radius(int eq, double ax, double ay, double gam, const double* W, double nx, double ny, double* out) {
  Params P{};
  P.eq = eq; P.m = (eq == EQ_EULER) ? 4 : 1; P.ax = ax; P.ay = ay; P.gam = gam;
  out[0] = spectral_radius_n<double>(P, W, nx, ny);
  out[1] = spectral_radius_all(P, W);
  return 0;
}

// Scale-limiter fraction (R18): the largest f in [0, 1] such that
// Wb + f (w - Wb) has density and pressure >= eps (Euler, gamma gam).
double orc_admissible_fraction(double gam, const double* Wb, const double* w, double eps) {
  return admissible_fraction<double>(gam, Wb, w, eps);
}

// Flux directional derivatives at W: out[6][m] = f'a, f'b, f''[a]b, g'a, g'b, g''[a]b
int orc_flux_derivs(int eq, double ax, double ay, double gam, const double* W, const double* a, const double* b, double* out) {
  Params P{};
  P.eq = eq; P.m = (eq == EQ_EULER) ? 4 : 1; P.ax = ax; P.ay = ay; P.gam = gam;
  int m = P.m;
  flux_derivs<double>(P, W, a, b, out, out + m, out + 2 * m, out + 3 * m, out + 4 * m, out + 5 * m);
  return 0;
}

}  // extern "C"
