// Device-side building blocks of the HWENO step: state/geometry views,
// the per-cell reconstruction (Section 2.2), the Lax-Wendroff procedure
// (Section 2.1) and the flux functions.  Included by the kernel files only.
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace hw {

// Device-resident scalars of one solve (time, step, target, flags).
struct DevScalars {
  double t;                          // current time
  double dt;                         // step to take next (CFL, clipped)
  double T;                          // target time when has_T
  double cfl;
  unsigned long long lam_min_bits;   // min_K inradius/lambda as the bits of a positive double
  unsigned int counter;              // blocks done (last-block finalisation)
  unsigned int flags;                // bit 0: non-finite / non-physical, bit 1: spin limit, bit 2: a state row index out of range
  long long nsteps;                  // steps taken
  int done;                          // target reached
  int has_T;
  int pad[2];
};

struct EqParams {
  double ax, ay, gam, eps;
  double g[4];
  int positivity;   // scale limiter on (Euler)
  int time_rule;    // 0: Gauss-Lobatto time nodes (0, dt/2, dt); 1: two Gauss-Legendre nodes
  // derived on the host by eq_params_finish: gamma - 1, |a|, and every
  // constant rounded once to float for the single-precision kernels (a
  // conversion or a double operation inside a kernel runs on the slow
  // double-precision pipe)
  double win[4];    // state imposed at inflow boundary edges (conservative)
  double gm1, amag;
  float axf, ayf, gamf, gm1f, epsf, amagf, gf[4], winf[4];
};

inline void eq_params_finish(EqParams& P) {
  P.gm1 = P.gam - 1.0;
  P.amag = std::sqrt(P.ax * P.ax + P.ay * P.ay);
  P.axf = (float)P.ax; P.ayf = (float)P.ay; P.gamf = (float)P.gam; P.gm1f = (float)P.gm1;
  P.epsf = (float)P.eps; P.amagf = (float)P.amag;
  for (int l = 0; l < 4; ++l) { P.gf[l] = (float)P.g[l]; P.winf[l] = (float)P.win[l]; }
}

// 1 / x correctly rounded (the same value as the IEEE division 1 / x)
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }

// the constants in the working precision R
template <typename R> struct EqC {
  static __device__ __forceinline__ R ax(const EqParams& P) { if constexpr (sizeof(R) == 8) return P.ax; else return P.axf; }
  static __device__ __forceinline__ R ay(const EqParams& P) { if constexpr (sizeof(R) == 8) return P.ay; else return P.ayf; }
  static __device__ __forceinline__ R gam(const EqParams& P) { if constexpr (sizeof(R) == 8) return P.gam; else return P.gamf; }
  static __device__ __forceinline__ R gm1(const EqParams& P) { if constexpr (sizeof(R) == 8) return P.gm1; else return P.gm1f; }
  static __device__ __forceinline__ R eps(const EqParams& P) { if constexpr (sizeof(R) == 8) return P.eps; else return P.epsf; }
  static __device__ __forceinline__ R amag(const EqParams& P) { if constexpr (sizeof(R) == 8) return P.amag; else return P.amagf; }
  static __device__ __forceinline__ R g(const EqParams& P, int l) { if constexpr (sizeof(R) == 8) return P.g[l]; else return P.gf[l]; }
  static __device__ __forceinline__ R win(const EqParams& P, int c) { if constexpr (sizeof(R) == 8) return P.win[c]; else return P.winf[c]; }
};


template <typename R> struct GeoView {
  const R* __restrict__ rg;        // [NRGEO][ld]
  const int32_t* __restrict__ ig;  // [NIGEO][ld]
  int N;                           // cells
  int ld;                          // plane stride (multiple of 32 cells)
  __device__ __forceinline__ R r(int p, int i) const { return __ldg(rg + (size_t)p * ld + i); }
  __device__ __forceinline__ int32_t n(int p, int i) const { return __ldg(ig + (size_t)p * ld + i); }
};

constexpr int kEqAdvection = 0, kEqBurgers = 1, kEqEuler = 2;
template <int EQ> struct EqTraits { static constexpr int m = (EQ == kEqEuler) ? 4 : 1; };

// ---------------------------------------------------------------- boundary ghosts
// Type of the ghost across local edge j (bits 9 + 2j of the packed edge plane):
// transmissive (the cell's own data), a reflective wall (the mirrored
// solution; Euler, the scalar equations treat it as transmissive) or an inflow
// edge (the imposed state, flat).
constexpr int kGhostTransmissive = 0, kGhostWall = 1, kGhostInflow = 2;
__device__ __forceinline__ int ghost_type(int packed, int j) { return (packed >> (9 + 2 * j)) & 3; }

// Component c of the mirror of a 4-vector of Euler quantities across a wall
// with unit normal n: momentum reflected, m -> m - 2 (m . n) n.
template <typename R> __device__ __forceinline__ R mirror_c(R nx, R ny, const R* X, int c) {
  if (c == 1 || c == 2) {
    const R xn = X[1] * nx + X[2] * ny;
    return X[c] - R(2) * (c == 1 ? nx : ny) * xn;
  }
  return X[c];
}

// Component c of the averages (W, W_x, W_y) carried by the ghost across a
// boundary edge with outward unit normal n; own: the cell's state record.
// Wall: W_g(x) = M W(Rx) with M the state mirror and R the reflection across
// the edge line, so Wbar_g = M Wbar and the derivative averages are M applied
// to the components, then R to (d/dx, d/dy).
template <typename R, int EQ>
__device__ __forceinline__ void ghost_component(int type, const R* own, R nx, R ny, int c, const EqParams& P, R& W,
                                                R& V, R& Y) {
  constexpr int m = EqTraits<EQ>::m;
  if (type == kGhostInflow) {
    W = EqC<R>::win(P, c); V = R(0); Y = R(0);
    return;
  }
  if (EQ != kEqEuler || type != kGhostWall) {
    W = own[c]; V = own[m + c]; Y = own[2 * m + c];
    return;
  }
  W = mirror_c(nx, ny, own, c);
  const R vm = mirror_c(nx, ny, own + m, c), ym = mirror_c(nx, ny, own + 2 * m, c);
  const R dn = vm * nx + ym * ny;
  V = vm - R(2) * nx * dn;
  Y = ym - R(2) * ny * dn;
}

__device__ __forceinline__ double dmax(double a, double b) { return a > b ? a : b; }

// ---------------------------------------------------------------- nonlinear weights
// Step 5 (Eq. nonlinearweight) for one component; also returns nothing else.
// In double the paper's expression is evaluated as written.
__device__ __forceinline__ void nonlinear_weights(double Wave, const double beta[4], const EqParams& P, double om[4]) {
  const double* g = P.g;
  const double eps = P.eps;
  const double tau = fabs(beta[0] - beta[1]) + fabs(beta[0] - beta[2]) + fabs(beta[0] - beta[3]);
  const double kappa = tau * tau / 9.0;
  const double W2 = Wave * Wave, W4 = W2 * W2;
  double wb[4], s = 0.0;
#pragma unroll
  for (int l = 0; l < 4; ++l) { wb[l] = g[l] * (1.0 + kappa / (W4 * eps + W2 * beta[l])); s += wb[l]; }
#pragma unroll
  for (int l = 0; l < 4; ++l) om[l] = wb[l] / s;
}

// Single precision: the same expression in float while W_ave^4 * eps stays a
// normal float; below that (|W_ave| < 2^-20) the terms cannot be represented in
// float and the expression is evaluated in double.  A non-finite sum falls back
// to the linear weights.
__device__ __forceinline__ void nonlinear_weights(float Wave, const float beta[4], const EqParams& P, float om[4]) {
  if (fabsf(Wave) < 9.5367431640625e-07f) {
    double bd[4] = {beta[0], beta[1], beta[2], beta[3]}, od[4];
    nonlinear_weights((double)Wave, bd, P, od);
#pragma unroll
    for (int l = 0; l < 4; ++l) om[l] = (float)od[l];
    return;
  }
  const float tau = fabsf(beta[0] - beta[1]) + fabsf(beta[0] - beta[2]) + fabsf(beta[0] - beta[3]);
  const float kappa = tau * tau * (1.0f / 9.0f);
  const float W2 = Wave * Wave, W4e = W2 * W2 * P.epsf;
  float wb[4], s = 0.f;
#pragma unroll
  for (int l = 0; l < 4; ++l) { wb[l] = P.gf[l] * (1.0f + kappa / (W4e + W2 * beta[l])); s += wb[l]; }
  if (!isfinite(s) || s <= 0.f) {
#pragma unroll
    for (int l = 0; l < 4; ++l) om[l] = P.gf[l];
    return;
  }
  const float is = recip(s);
#pragma unroll
  for (int l = 0; l < 4; ++l) om[l] = wb[l] * is;
}

// ---------------------------------------------------------------- reconstruction
// Steps 1-6 of Section 2.2 for NC components of cell i: returns each
// component's combined quadratic (Eq. recon) as monomials in the scaled frame
// of the cell,
//   q(xi, eta) = q0 + q1 xi + q2 eta + q3 xi^2 + q4 xi eta + q5 eta^2.
// GA: accessor of this cell's geometry planes, ga(p) = plane p (see RGeo);
// each plane is read once for the NC components, whose arithmetic is that of
// one component, term by term.  W0, V0, Y0: the cell's averages; Wl, Vl, Yl:
// those of the stencil members K1..K3 (a boundary ghost carries the cell's
// own values).
template <typename R, int NC, typename GA>
__device__ __forceinline__ void reconstruct_components(const GA& ga, const R* W0, const R* V0, const R* Y0,
                                                       const R (*Wl)[3], const R (*Vl)[3], const R (*Yl)[3],
                                                       const EqParams& P, R (*q)[6]) {
  // Step 1: constrained least squares solved once on the host; here the operator
  R rhs[NC][9];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const R w = ga(G_W + l);
#pragma unroll
    for (int n = 0; n < NC; ++n) {
      rhs[n][l] = Wl[n][l] - W0[n];
      rhs[n][3 + 2 * l] = V0[n] + w * (Vl[n][l] - V0[n]);
      rhs[n][4 + 2 * l] = Y0[n] + w * (Yl[n][l] - Y0[n]);
    }
  }
  R cc[NC][5];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    R s[NC];
#pragma unroll
    for (int n = 0; n < NC; ++n) s[n] = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const R g = ga(G_M1 + r * 9 + k);
#pragma unroll
      for (int n = 0; n < NC; ++n) s[n] += g * rhs[n][k];
    }
#pragma unroll
    for (int n = 0; n < NC; ++n) cc[n][r] = s[n];
  }
  // Step 2: linear polynomials on {K0, K_l}
  R b[NC][3][2];
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const R g0 = ga(G_P + l * 6 + r * 3 + 0), g1 = ga(G_P + l * 6 + r * 3 + 1), g2 = ga(G_P + l * 6 + r * 3 + 2);
#pragma unroll
      for (int n = 0; n < NC; ++n) b[n][l][r] = g0 * (Wl[n][l] - W0[n]) + g1 * Vl[n][l] + g2 * Yl[n][l];
    }
  const R m3 = ga(G_MOM), m4 = ga(G_MOM + 1), m5 = ga(G_MOM + 2);
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    // Step 4 (Eq. smoo1): in the frame scaled by h0 = sqrt|K0| the factors
    // |K0|^|s| cancel the chain-rule factors, leaving the scaled derivatives.
    R beta[4];
    beta[0] = cc[n][0] * cc[n][0] + cc[n][1] * cc[n][1] + R(4) * cc[n][2] * cc[n][2] + cc[n][3] * cc[n][3] +
              R(4) * cc[n][4] * cc[n][4];
#pragma unroll
    for (int l = 0; l < 3; ++l) beta[l + 1] = b[n][l][0] * b[n][l][0] + b[n][l][1] * b[n][l][1];
    // Step 5
    const R Wave = (W0[n] + Wl[n][0] + Wl[n][1] + Wl[n][2]) * R(0.25) + R(1e-30);
    R om[4];
    nonlinear_weights(Wave, beta, P, om);
    // Step 6: q = (om1/g1) p1 + sum_l (om_l - om1 g_l / g1) p_l
    const R a1 = om[0] / EqC<R>::g(P, 0);
    R al[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) al[l] = om[l + 1] - a1 * EqC<R>::g(P, l + 1);
    R q1 = a1 * cc[n][0], q2 = a1 * cc[n][1];
#pragma unroll
    for (int l = 0; l < 3; ++l) { q1 += al[l] * b[n][l][0]; q2 += al[l] * b[n][l][1]; }
    const R q3 = a1 * cc[n][2], q4 = a1 * cc[n][3], q5 = a1 * cc[n][4];
    // the constant parts of p1..p4 all equal Wbar_0 and the coefficients sum to one
    q[n][0] = W0[n] - q3 * m3 - q4 * m4 - q5 * m5;
    q[n][1] = q1; q[n][2] = q2; q[n][3] = q3; q[n][4] = q4; q[n][5] = q5;
  }
}

// One component (the same arithmetic).
template <typename R, typename GA>
__device__ __forceinline__ void reconstruct_component(const GA& ga, const R W0, const R V0, const R Y0,
                                                      const R Wl[3], const R Vl[3], const R Yl[3],
                                                      const EqParams& P, R q[6]) {
  R wl[1][3], vl[1][3], yl[1][3], qq[1][6];
#pragma unroll
  for (int l = 0; l < 3; ++l) { wl[0][l] = Wl[l]; vl[0][l] = Vl[l]; yl[0][l] = Yl[l]; }
  reconstruct_components<R, 1>(ga, &W0, &V0, &Y0, wl, vl, yl, P, qq);
#pragma unroll
  for (int k = 0; k < 6; ++k) q[k] = qq[0][k];
}

// ---------------------------------------------------------------- Lax-Wendroff
// Second-order jets in (x, y) extended by the time directions t, xt, yt.
template <typename R> struct Jet {
  R v, x, y, xx, xy, yy, t, xt, yt;
};
template <typename R> __device__ __forceinline__ Jet<R> jadd(const Jet<R>& a, const Jet<R>& b) {
  return {a.v + b.v, a.x + b.x, a.y + b.y, a.xx + b.xx, a.xy + b.xy, a.yy + b.yy, a.t + b.t, a.xt + b.xt, a.yt + b.yt};
}
template <typename R> __device__ __forceinline__ Jet<R> jscale(R s, const Jet<R>& a) {
  return {s * a.v, s * a.x, s * a.y, s * a.xx, s * a.xy, s * a.yy, s * a.t, s * a.xt, s * a.yt};
}
template <typename R> __device__ __forceinline__ Jet<R> jmul(const Jet<R>& a, const Jet<R>& b) {
  Jet<R> c;
  c.v = a.v * b.v;
  c.x = a.x * b.v + a.v * b.x;
  c.y = a.y * b.v + a.v * b.y;
  c.xx = a.xx * b.v + R(2) * a.x * b.x + a.v * b.xx;
  c.xy = a.xy * b.v + a.x * b.y + a.y * b.x + a.v * b.xy;
  c.yy = a.yy * b.v + R(2) * a.y * b.y + a.v * b.yy;
  c.t = a.t * b.v + a.v * b.t;
  c.xt = a.xt * b.v + a.x * b.t + a.t * b.x + a.v * b.xt;
  c.yt = a.yt * b.v + a.y * b.t + a.t * b.y + a.v * b.yt;
  return c;
}
template <typename R> __device__ __forceinline__ Jet<R> jrecip(const Jet<R>& a) {
  Jet<R> r;
  r.v = recip(a.v);
  const R r2 = r.v * r.v;
  r.x = -a.x * r2;
  r.y = -a.y * r2;
  r.t = -a.t * r2;
  r.xx = -a.xx * r2 - R(2) * a.x * r.v * r.x;
  r.xy = -a.xy * r2 - R(2) * a.x * r.v * r.y;
  r.yy = -a.yy * r2 - R(2) * a.y * r.v * r.y;
  r.xt = -a.xt * r2 - R(2) * a.t * r.v * r.x;
  r.yt = -a.yt * r2 - R(2) * a.t * r.v * r.y;
  return r;
}

// Euler fluxes f, g (Eq. 2d) propagated through jets.
template <typename R>
__device__ __forceinline__ void euler_flux_jets(const Jet<R> W[4], R gm1, Jet<R> f[4], Jet<R> g[4]) {
  const Jet<R> ir = jrecip(W[0]);
  const Jet<R> u = jmul(W[1], ir), v = jmul(W[2], ir);
  const Jet<R> mu = jmul(W[1], u), nv = jmul(W[2], v), nu = jmul(W[2], u);
  const Jet<R> p = jscale(gm1, jadd(W[3], jscale(R(-0.5), jadd(mu, nv))));
  const Jet<R> H = jadd(W[3], p);
  f[0] = W[1]; f[1] = jadd(mu, p); f[2] = nu; f[3] = jmul(H, u);
  g[0] = W[2]; g[1] = nu; g[2] = jadd(nv, p); g[3] = jmul(H, v);
}

// Lax-Wendroff procedure at one point (Section 2.1): from (W, Wx, Wy) and the
// cell-constant second derivatives, the first and second time derivatives.
template <typename R, int EQ>
__device__ __forceinline__ void lax_wendroff(const R* W, const R* Wx, const R* Wy, const R* Wxx, const R* Wxy,
                                             const R* Wyy, const EqParams& P, R* Wt, R* Wtt) {
  if constexpr (EQ == kEqAdvection) {
    const R ax = EqC<R>::ax(P), ay = EqC<R>::ay(P);
    Wt[0] = -(ax * Wx[0] + ay * Wy[0]);
    Wtt[0] = ax * ax * Wxx[0] + R(2) * ax * ay * Wxy[0] + ay * ay * Wyy[0];
  } else if constexpr (EQ == kEqBurgers) {
    // f = g = W^2 / 2:  Wt = -W s, s = Wx + Wy;  Wtt = -(Wt s + W (Wtx + Wty))
    const R s = Wx[0] + Wy[0];
    const R wt = -W[0] * s;
    const R wtx = -(Wx[0] * s + W[0] * (Wxx[0] + Wxy[0]));
    const R wty = -(Wy[0] * s + W[0] * (Wxy[0] + Wyy[0]));
    Wt[0] = wt;
    Wtt[0] = -(wt * s + W[0] * (wtx + wty));
  } else {
    const R gm1 = EqC<R>::gm1(P);
    Jet<R> J[4], f[4], g[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) J[c] = {W[c], Wx[c], Wy[c], Wxx[c], Wxy[c], Wyy[c], R(0), R(0), R(0)};
    euler_flux_jets(J, gm1, f, g);
    // Wt = -(f_x + g_y), Wtx = -(f_xx + g_xy), Wty = -(f_xy + g_yy)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      J[c].t = -(f[c].x + g[c].y);
      J[c].xt = -(f[c].xx + g[c].xy);
      J[c].yt = -(f[c].xy + g[c].yy);
    }
    euler_flux_jets(J, gm1, f, g);
    // Wtt = -(f_xt + g_yt)
#pragma unroll
    for (int c = 0; c < 4; ++c) { Wt[c] = J[c].t; Wtt[c] = -(f[c].xt + g[c].yt); }
  }
}

// ---------------------------------------------------------------- fluxes
// F(W) . n
template <typename R, int EQ>
__device__ __forceinline__ void flux_n(const R* W, R nx, R ny, const EqParams& P, R* H) {
  if constexpr (EQ == kEqAdvection) {
    H[0] = (EqC<R>::ax(P) * nx + EqC<R>::ay(P) * ny) * W[0];
  } else if constexpr (EQ == kEqBurgers) {
    H[0] = R(0.5) * W[0] * W[0] * (nx + ny);
  } else {
    const R ir = recip(W[0]);
    const R u = W[1] * ir, v = W[2] * ir;
    const R p = EqC<R>::gm1(P) * (W[3] - R(0.5) * (W[1] * u + W[2] * v));
    const R un = u * nx + v * ny;
    H[0] = W[0] * un;
    H[1] = W[1] * un + p * nx;
    H[2] = W[2] * un + p * ny;
    H[3] = (W[3] + p) * un;
  }
}

// Largest eigenvalue in magnitude of d(F.n)/dW at a cell average.
template <typename R, int EQ>
__device__ __forceinline__ R spectral_radius_n(const R* W, R nx, R ny, const EqParams& P) {
  if constexpr (EQ == kEqAdvection) {
    return fabs(EqC<R>::ax(P) * nx + EqC<R>::ay(P) * ny);
  } else if constexpr (EQ == kEqBurgers) {
    return fabs(W[0] * (nx + ny));
  } else {
    const R ir = recip(W[0]);
    const R u = W[1] * ir, v = W[2] * ir;
    const R p = EqC<R>::gm1(P) * (W[3] - R(0.5) * (W[1] * u + W[2] * v));
    return fabs(u * nx + v * ny) + sqrt(EqC<R>::gam(P) * p * ir);
  }
}

// Spectral radius over all directions (CFL time step), in the working
// precision R.
template <typename R, int EQ>
__device__ __forceinline__ R spectral_radius_all(const R* W, const EqParams& P) {
  if constexpr (EQ == kEqAdvection) {
    return EqC<R>::amag(P);
  } else if constexpr (EQ == kEqBurgers) {
    return R(1.4142135623730951) * fabs(W[0]);
  } else {
    const R ir = recip(W[0]);
    const R u = W[1] * ir, v = W[2] * ir;
    const R p = EqC<R>::gm1(P) * (W[3] - R(0.5) * (W[1] * u + W[2] * v));
    return sqrt(u * u + v * v) + sqrt(EqC<R>::gam(P) * p * ir);
  }
}

// Floor of the scale limiter: min(1e-13, rho_bar, p_bar) in double (Zhang and
// Shu's choice).  In float the floor is min(2^-20, rho_bar, p_bar): a point
// density pulled down to 1e-13 next to an O(1) momentum overflows the float
// Lax-Wendroff jets (their second derivatives carry 1 / rho^3).
__device__ __forceinline__ double positivity_floor(double rho, double p) { return fmin(1e-13, fmin(rho, p)); }
__device__ __forceinline__ float positivity_floor(float rho, float p) {
  return fminf(9.5367431640625e-07f, fminf(rho, p));
}

// Scale limiter (Zhang and Shu), Euler.  Pressure of a conservative state.
template <typename R> __device__ __forceinline__ R pressure_of(R gam, const R* W) {
  return (gam - R(1)) * (W[3] - R(0.5) * (W[1] * W[1] + W[2] * W[2]) / W[0]);
}

// Smallest root in [0, 1] of p(Wb + f d) = eps (times the density, a
// quadratic in f); 0 if none.
template <typename R> __device__ __forceinline__ R pressure_root(R gam, const R Wb[4], const R d[4], R eps) {
  const R g1 = gam - R(1);
  const R a = g1 * (d[3] * d[0] - R(0.5) * (d[1] * d[1] + d[2] * d[2]));
  const R b = g1 * (Wb[3] * d[0] + Wb[0] * d[3] - (Wb[1] * d[1] + Wb[2] * d[2])) - eps * d[0];
  const R c0 = g1 * (Wb[3] * Wb[0] - R(0.5) * (Wb[1] * Wb[1] + Wb[2] * Wb[2])) - eps * Wb[0];
  R tk = R(0);
  if (fabs(a) < R(sizeof(R) == 8 ? 1e-300 : 1e-37)) {
    if (b < R(0)) tk = -c0 / b;
    if (tk > R(1)) tk = R(1);
  } else {
    const R disc = b * b - R(4) * a * c0;
    const R sq = disc > R(0) ? sqrt(disc) : R(0);
    const R r1 = (-b - sq) / (R(2) * a), r2 = (-b + sq) / (R(2) * a);
    // smallest non-negative root, clamped to 1 (continuous at the boundary)
    R best = R(-1);
    if (r1 >= R(0)) best = r1;
    if (r2 >= R(0) && (best < R(0) || r2 < best)) best = r2;
    tk = best < R(0) ? R(0) : (best > R(1) ? R(1) : best);
  }
  return tk;
}

// Single precision: the quadratic's coefficients cancel badly in float near
// the admissible boundary, so the root is taken in double (a rare path: only
// where the pressure bound is active).
__device__ __forceinline__ float pressure_root(float gam, const float Wb[4], const float d[4], float eps) {
  const double Wd[4] = {Wb[0], Wb[1], Wb[2], Wb[3]}, dd[4] = {d[0], d[1], d[2], d[3]};
  return (float)pressure_root<double>((double)gam, Wd, dd, (double)eps);
}

// Largest f in [0, 1] such that Wb + f (w - Wb) has density and pressure >= eps:
// density first, then the pressure root.
template <typename R>
__device__ __forceinline__ R admissible_fraction(R gam, const R Wb[4], const R w[4], R eps) {
  R f1 = R(1);
  if (w[0] < eps) f1 = (Wb[0] - eps) / (Wb[0] - w[0]);
  R d[4], v[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) { d[c] = f1 * (w[c] - Wb[c]); v[c] = Wb[c] + d[c]; }
  if (pressure_of(gam, v) >= eps) return f1;
  return f1 * pressure_root(gam, Wb, d, eps);
}

template <typename R, int EQ> __device__ __forceinline__ bool physical(const R* W, const EqParams& P) {
  constexpr int m = EqTraits<EQ>::m;
  bool ok = true;
#pragma unroll
  for (int c = 0; c < m; ++c) ok = ok && isfinite(W[c]);
  if constexpr (EQ == kEqEuler) {
    if (ok) {
      const R p = EqC<R>::gm1(P) * (W[3] - R(0.5) * (W[1] * W[1] + W[2] * W[2]) / W[0]);
      ok = (W[0] > R(0)) && (p > R(0));
    }
  }
  return ok;
}

}  // namespace hw
