// Reverse-mode (vector-Jacobian) counterparts of the device building blocks of
// one ADER-HWENO step for the Euler system: the local Lax-Friedrichs flux at
// the Gauss-Lobatto nodes, the flux functions, the spectral radius behind the
// numerical viscosity, the Lax-Wendroff procedure (second-order jets) and the
// reconstruction Steps 1-6 (Section 2.2).  Each *_vjp takes the forward inputs
// (the forward values are recomputed), the cotangents of the outputs, and
// accumulates the cotangents of the inputs.  Non-smooth points (|.|, max) take
// the branch the forward evaluation takes.  Included by adjoint.cu only.
#pragma once
#include "device.cuh"

namespace hw {

// ---------------------------------------------------------------- jets
template <typename R> __device__ __forceinline__ Jet<R> jzero() {
  return {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
}
template <typename R> __device__ __forceinline__ void jacc(Jet<R>& a, const Jet<R>& b) { a = jadd(a, b); }

// c = a * b
template <typename R>
__device__ __forceinline__ void jmul_vjp(const Jet<R>& a, const Jet<R>& b, const Jet<R>& cb, Jet<R>& ab, Jet<R>& bb) {
  ab.v += cb.v * b.v + cb.x * b.x + cb.y * b.y + cb.xx * b.xx + cb.xy * b.xy + cb.yy * b.yy + cb.t * b.t +
          cb.xt * b.xt + cb.yt * b.yt;
  ab.x += cb.x * b.v + R(2) * cb.xx * b.x + cb.xy * b.y + cb.xt * b.t;
  ab.y += cb.y * b.v + cb.xy * b.x + R(2) * cb.yy * b.y + cb.yt * b.t;
  ab.xx += cb.xx * b.v;
  ab.xy += cb.xy * b.v;
  ab.yy += cb.yy * b.v;
  ab.t += cb.t * b.v + cb.xt * b.x + cb.yt * b.y;
  ab.xt += cb.xt * b.v;
  ab.yt += cb.yt * b.v;
  bb.v += cb.v * a.v + cb.x * a.x + cb.y * a.y + cb.xx * a.xx + cb.xy * a.xy + cb.yy * a.yy + cb.t * a.t +
          cb.xt * a.xt + cb.yt * a.yt;
  bb.x += cb.x * a.v + R(2) * cb.xx * a.x + cb.xy * a.y + cb.xt * a.t;
  bb.y += cb.y * a.v + cb.xy * a.x + R(2) * cb.yy * a.y + cb.yt * a.t;
  bb.xx += cb.xx * a.v;
  bb.xy += cb.xy * a.v;
  bb.yy += cb.yy * a.v;
  bb.t += cb.t * a.v + cb.xt * a.x + cb.yt * a.y;
  bb.xt += cb.xt * a.v;
  bb.yt += cb.yt * a.v;
}

// r = 1 / a (r: the forward result)
template <typename R>
__device__ __forceinline__ void jrecip_vjp(const Jet<R>& a, const Jet<R>& r, const Jet<R>& rb, Jet<R>& ab) {
  const R rv = r.v, r2 = rv * rv;
  R Rx = rb.x, Ry = rb.y, r2b = R(0), rvb = R(0);
  ab.yt += -r2 * rb.yt; r2b += -a.yt * rb.yt; ab.t += R(-2) * rv * r.y * rb.yt; rvb += R(-2) * a.t * r.y * rb.yt;
  Ry += R(-2) * a.t * rv * rb.yt;
  ab.xt += -r2 * rb.xt; r2b += -a.xt * rb.xt; ab.t += R(-2) * rv * r.x * rb.xt; rvb += R(-2) * a.t * r.x * rb.xt;
  Rx += R(-2) * a.t * rv * rb.xt;
  ab.yy += -r2 * rb.yy; r2b += -a.yy * rb.yy; ab.y += R(-2) * rv * r.y * rb.yy; rvb += R(-2) * a.y * r.y * rb.yy;
  Ry += R(-2) * a.y * rv * rb.yy;
  ab.xy += -r2 * rb.xy; r2b += -a.xy * rb.xy; ab.x += R(-2) * rv * r.y * rb.xy; rvb += R(-2) * a.x * r.y * rb.xy;
  Ry += R(-2) * a.x * rv * rb.xy;
  ab.xx += -r2 * rb.xx; r2b += -a.xx * rb.xx; ab.x += R(-2) * rv * r.x * rb.xx; rvb += R(-2) * a.x * r.x * rb.xx;
  Rx += R(-2) * a.x * rv * rb.xx;
  ab.t += -r2 * rb.t; r2b += -a.t * rb.t;
  ab.y += -r2 * Ry; r2b += -a.y * Ry;
  ab.x += -r2 * Rx; r2b += -a.x * Rx;
  rvb += R(2) * rv * r2b;
  ab.v += -r2 * (rb.v + rvb);
}

// Euler fluxes through jets (forward in device.cuh: euler_flux_jets)
template <typename R>
__device__ __forceinline__ void euler_flux_jets_vjp(const Jet<R> W[4], R gm1, const Jet<R> fb[4], const Jet<R> gb[4],
                                                    Jet<R> Wb[4]) {
  const Jet<R> ir = jrecip(W[0]);
  const Jet<R> u = jmul(W[1], ir), v = jmul(W[2], ir);
  const Jet<R> mu = jmul(W[1], u), nv = jmul(W[2], v);
  const Jet<R> p = jscale(gm1, jadd(W[3], jscale(R(-0.5), jadd(mu, nv))));
  const Jet<R> H = jadd(W[3], p);
  Jet<R> irb = jzero<R>(), ub = jzero<R>(), vb = jzero<R>(), mub = jzero<R>(), nvb = jzero<R>(), nub = jzero<R>();
  Jet<R> pb = jzero<R>(), Hb = jzero<R>();
  jacc(Wb[1], fb[0]);
  jacc(mub, fb[1]); jacc(pb, fb[1]);
  jacc(nub, fb[2]);
  jmul_vjp(H, u, fb[3], Hb, ub);
  jacc(Wb[2], gb[0]);
  jacc(nub, gb[1]);
  jacc(nvb, gb[2]); jacc(pb, gb[2]);
  jmul_vjp(H, v, gb[3], Hb, vb);
  jacc(Wb[3], Hb); jacc(pb, Hb);
  jacc(Wb[3], jscale(gm1, pb));
  jacc(mub, jscale(R(-0.5) * gm1, pb));
  jacc(nvb, jscale(R(-0.5) * gm1, pb));
  jmul_vjp(W[2], u, nub, Wb[2], ub);
  jmul_vjp(W[2], v, nvb, Wb[2], vb);
  jmul_vjp(W[1], u, mub, Wb[1], ub);
  jmul_vjp(W[2], ir, vb, Wb[2], irb);
  jmul_vjp(W[1], ir, ub, Wb[1], irb);
  jrecip_vjp(W[0], ir, irb, Wb[0]);
}

// Lax-Wendroff procedure (Euler), reverse: cotangents of (W_t, W_tt) -> of the
// spatial jet (W, W_x, W_y, W_xx, W_xy, W_yy), accumulated into Jb.
template <typename R>
__device__ __forceinline__ void lax_wendroff_euler_vjp(const R* W, const R* Wx, const R* Wy, const R* Wxx,
                                                       const R* Wxy, const R* Wyy, R gm1, const R* Wtb,
                                                       const R* Wttb, Jet<R> Jb[4]) {
  Jet<R> J[4], f[4], g[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) J[c] = {W[c], Wx[c], Wy[c], Wxx[c], Wxy[c], Wyy[c], R(0), R(0), R(0)};
  euler_flux_jets(J, gm1, f, g);
  Jet<R> J2[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    J2[c] = J[c];
    J2[c].t = -(f[c].x + g[c].y);
    J2[c].xt = -(f[c].xx + g[c].xy);
    J2[c].yt = -(f[c].xy + g[c].yy);
  }
  // pass 2: W_tt = -(f.xt + g.yt)
  Jet<R> f2b[4], g2b[4], J2b[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    f2b[c] = jzero<R>(); g2b[c] = jzero<R>(); J2b[c] = jzero<R>();
    f2b[c].xt = -Wttb[c];
    g2b[c].yt = -Wttb[c];
  }
  euler_flux_jets_vjp(J2, gm1, f2b, g2b, J2b);
  // W_t = J2.t
  Jet<R> f1b[4], g1b[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const R tb = J2b[c].t + Wtb[c];
    f1b[c] = jzero<R>(); g1b[c] = jzero<R>();
    f1b[c].x = -tb; g1b[c].y = -tb;
    f1b[c].xx = -J2b[c].xt; g1b[c].xy = -J2b[c].xt;
    f1b[c].xy = -J2b[c].yt; g1b[c].yy = -J2b[c].yt;
  }
  Jet<R> J1b[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) J1b[c] = jzero<R>();
  euler_flux_jets_vjp(J, gm1, f1b, g1b, J1b);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    Jb[c].v += J2b[c].v + J1b[c].v;
    Jb[c].x += J2b[c].x + J1b[c].x;
    Jb[c].y += J2b[c].y + J1b[c].y;
    Jb[c].xx += J2b[c].xx + J1b[c].xx;
    Jb[c].xy += J2b[c].xy + J1b[c].xy;
    Jb[c].yy += J2b[c].yy + J1b[c].yy;
  }
}

// ---------------------------------------------------------------- fluxes
// H = F(W) . n, reverse (Euler)
template <typename R>
__device__ __forceinline__ void flux_n_euler_vjp(const R* W, R nx, R ny, R gm1, const R* Hb, R* Wb) {
  const R ir = R(1) / W[0];
  const R u = W[1] * ir, v = W[2] * ir;
  const R p = gm1 * (W[3] - R(0.5) * (W[1] * u + W[2] * v));
  const R un = u * nx + v * ny;
  Wb[0] += Hb[0] * un;
  const R unb = Hb[0] * W[0] + Hb[1] * W[1] + Hb[2] * W[2] + Hb[3] * (W[3] + p);
  Wb[1] += Hb[1] * un;
  Wb[2] += Hb[2] * un;
  Wb[3] += Hb[3] * un;
  const R pb = Hb[1] * nx + Hb[2] * ny + Hb[3] * un;
  R ub = nx * unb, vb = ny * unb;
  Wb[3] += gm1 * pb;
  Wb[1] += R(-0.5) * gm1 * u * pb;
  ub += R(-0.5) * gm1 * W[1] * pb;
  Wb[2] += R(-0.5) * gm1 * v * pb;
  vb += R(-0.5) * gm1 * W[2] * pb;
  R irb = W[2] * vb + W[1] * ub;
  Wb[2] += ir * vb;
  Wb[1] += ir * ub;
  Wb[0] += -ir * ir * irb;
}

// lambda = |u.n| + c at a cell average, reverse (Euler)
template <typename R>
__device__ __forceinline__ void spectral_radius_n_euler_vjp(const R* W, R nx, R ny, R gam, R lb, R* Wb) {
  const R gm1 = gam - R(1);
  const R ir = R(1) / W[0];
  const R u = W[1] * ir, v = W[2] * ir;
  const R p = gm1 * (W[3] - R(0.5) * (W[1] * u + W[2] * v));
  const R un = u * nx + v * ny;
  const R c = sqrt(gam * p * ir);
  const R unb = un < R(0) ? -lb : lb;
  const R cb = lb;
  const R pb = gam * ir * cb / (R(2) * c);
  R irb = gam * p * cb / (R(2) * c);
  R ub = nx * unb, vb = ny * unb;
  Wb[3] += gm1 * pb;
  Wb[1] += R(-0.5) * gm1 * u * pb;
  ub += R(-0.5) * gm1 * W[1] * pb;
  Wb[2] += R(-0.5) * gm1 * v * pb;
  vb += R(-0.5) * gm1 * W[2] * pb;
  irb += W[2] * vb + W[1] * ub;
  Wb[2] += ir * vb;
  Wb[1] += ir * ub;
  Wb[0] += -ir * ir * irb;
}

// ---------------------------------------------------------------- nonlinear weights
template <typename T>
__device__ __forceinline__ void nonlinear_weights_vjp_t(T Wave, const T beta[4], const double g[4], double eps,
                                                        const T omb[4], T& Waveb, T betab[4]) {
  const T tau = fabs(beta[0] - beta[1]) + fabs(beta[0] - beta[2]) + fabs(beta[0] - beta[3]);
  const T kappa = tau * tau / T(9);
  const T W2 = Wave * Wave, W4 = W2 * W2;
  T D[4], wb[4], s = T(0);
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    D[l] = W4 * T(eps) + W2 * beta[l];
    wb[l] = T(g[l]) * (T(1) + kappa / D[l]);
    s += wb[l];
  }
  T dot = T(0);
#pragma unroll
  for (int l = 0; l < 4; ++l) dot += omb[l] * (wb[l] / s);
  T kappab = T(0), W4b = T(0), W2b = T(0);
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const T wbb = (omb[l] - dot) / s;
    kappab += T(g[l]) * wbb / D[l];
    const T Db = -T(g[l]) * kappa * wbb / (D[l] * D[l]);
    W4b += T(eps) * Db;
    W2b += beta[l] * Db;
    betab[l] += W2 * Db;
  }
  W2b += T(2) * W2 * W4b;
  Waveb += T(2) * Wave * W2b;
  const T taub = T(2) * tau * kappab / T(9);
#pragma unroll
  for (int l = 1; l < 4; ++l) {
    const T sl = (beta[0] - beta[l] < T(0)) ? T(-1) : T(1);
    betab[0] += sl * taub;
    betab[l] += -sl * taub;
  }
}

__device__ __forceinline__ void nonlinear_weights_vjp(double Wave, const double beta[4], const double g[4], double eps,
                                                      const double omb[4], double& Waveb, double betab[4]) {
  nonlinear_weights_vjp_t<double>(Wave, beta, g, eps, omb, Waveb, betab);
}

// float: the same branch as the forward (double where W_ave^4 eps is not a
// normal float)
__device__ __forceinline__ void nonlinear_weights_vjp(float Wave, const float beta[4], const double g[4], double eps,
                                                      const float omb[4], float& Waveb, float betab[4]) {
  if (fabsf(Wave) < 9.5367431640625e-07f) {
    double bd[4] = {beta[0], beta[1], beta[2], beta[3]}, od[4] = {omb[0], omb[1], omb[2], omb[3]};
    double wab = 0.0, bbd[4] = {0, 0, 0, 0};
    nonlinear_weights_vjp_t<double>((double)Wave, bd, g, eps, od, wab, bbd);
    Waveb += (float)wab;
#pragma unroll
    for (int l = 0; l < 4; ++l) betab[l] += (float)bbd[l];
    return;
  }
  nonlinear_weights_vjp_t<float>(Wave, beta, g, eps, omb, Waveb, betab);
}

// ---------------------------------------------------------------- reconstruction
// Reverse of reconstruct_component (Steps 1-6): q-cotangent qb[6] -> cotangents
// of W0, V0, Y0 (o0[3]) and of the stencil members (ol[3][3]: W, V, Y of K_l).
template <typename R, typename GA>
__device__ __forceinline__ void reconstruct_component_vjp(const GA& ga, const R W0, const R V0, const R Y0,
                                                          const R Wl[3], const R Vl[3], const R Yl[3],
                                                          const EqParams& P, const R qb[6], R o0[3], R ol[3][3]) {
  R rhs[9];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    rhs[l] = Wl[l] - W0;
    const R w = ga(G_W + l);
    rhs[3 + 2 * l] = V0 + w * (Vl[l] - V0);
    rhs[4 + 2 * l] = Y0 + w * (Yl[l] - Y0);
  }
  R cc[5];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    R s = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) s += ga(G_M1 + r * 9 + k) * rhs[k];
    cc[r] = s;
  }
  R b[3][2];
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int r = 0; r < 2; ++r)
      b[l][r] = ga(G_P + l * 6 + r * 3 + 0) * (Wl[l] - W0) + ga(G_P + l * 6 + r * 3 + 1) * Vl[l] +
                ga(G_P + l * 6 + r * 3 + 2) * Yl[l];
  R beta[4];
  beta[0] = cc[0] * cc[0] + cc[1] * cc[1] + R(4) * cc[2] * cc[2] + cc[3] * cc[3] + R(4) * cc[4] * cc[4];
#pragma unroll
  for (int l = 0; l < 3; ++l) beta[l + 1] = b[l][0] * b[l][0] + b[l][1] * b[l][1];
  const R Wave = (W0 + Wl[0] + Wl[1] + Wl[2]) * R(0.25) + R(1e-30);
  R om[4];
  nonlinear_weights(Wave, beta, P.g, P.eps, om);
  const R a1 = om[0] / R(P.g[0]);
  R al[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) al[l] = om[l + 1] - a1 * R(P.g[l + 1]);
  // ---- reverse
  R q3b = qb[3], q4b = qb[4], q5b = qb[5];
  R W0b = qb[0];
  q3b += -ga(G_MOM) * qb[0];
  q4b += -ga(G_MOM + 1) * qb[0];
  q5b += -ga(G_MOM + 2) * qb[0];
  R a1b = qb[1] * cc[0] + qb[2] * cc[1] + q3b * cc[2] + q4b * cc[3] + q5b * cc[4];
  R ccb[5] = {a1 * qb[1], a1 * qb[2], a1 * q3b, a1 * q4b, a1 * q5b};
  R bb[3][2];
  R omb[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const R alb = qb[1] * b[l][0] + qb[2] * b[l][1];
    bb[l][0] = al[l] * qb[1];
    bb[l][1] = al[l] * qb[2];
    omb[l + 1] += alb;
    a1b += -R(P.g[l + 1]) * alb;
  }
  omb[0] += a1b / R(P.g[0]);
  R Waveb = R(0), betab[4] = {R(0), R(0), R(0), R(0)};
  nonlinear_weights_vjp(Wave, beta, P.g, P.eps, omb, Waveb, betab);
  R Wlb[3], Vlb[3], Ylb[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) { Wlb[l] = Waveb * R(0.25); Vlb[l] = R(0); Ylb[l] = R(0); }
  W0b += Waveb * R(0.25);
  ccb[0] += R(2) * cc[0] * betab[0];
  ccb[1] += R(2) * cc[1] * betab[0];
  ccb[2] += R(8) * cc[2] * betab[0];
  ccb[3] += R(2) * cc[3] * betab[0];
  ccb[4] += R(8) * cc[4] * betab[0];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    bb[l][0] += R(2) * b[l][0] * betab[l + 1];
    bb[l][1] += R(2) * b[l][1] * betab[l + 1];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const R p0 = ga(G_P + l * 6 + r * 3 + 0);
      Wlb[l] += p0 * bb[l][r];
      W0b += -p0 * bb[l][r];
      Vlb[l] += ga(G_P + l * 6 + r * 3 + 1) * bb[l][r];
      Ylb[l] += ga(G_P + l * 6 + r * 3 + 2) * bb[l][r];
    }
  }
  R rhsb[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    R s = 0;
#pragma unroll
    for (int r = 0; r < 5; ++r) s += ga(G_M1 + r * 9 + k) * ccb[r];
    rhsb[k] = s;
  }
  R V0b = R(0), Y0b = R(0);
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    Wlb[l] += rhsb[l];
    W0b += -rhsb[l];
    const R w = ga(G_W + l);
    V0b += (R(1) - w) * rhsb[3 + 2 * l];
    Vlb[l] += w * rhsb[3 + 2 * l];
    Y0b += (R(1) - w) * rhsb[4 + 2 * l];
    Ylb[l] += w * rhsb[4 + 2 * l];
  }
  o0[0] = W0b; o0[1] = V0b; o0[2] = Y0b;
#pragma unroll
  for (int l = 0; l < 3; ++l) { ol[l][0] = Wlb[l]; ol[l][1] = Vlb[l]; ol[l][2] = Ylb[l]; }
}

}  // namespace hw
