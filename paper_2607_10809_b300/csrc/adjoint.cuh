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
// The reverse pass works on the smallest jets that carry the outputs it needs
// (the forward evaluation in device.cuh uses full jets; the compiler drops the
// unused parts there, but cannot drop products with cotangents that are zero
// only by structure):
//   SJet (v, x, y, xx, xy, yy): second-order spatial jet, first pass
//        (W_t, W_tx, W_ty come from f_x, f_xx, f_xy, g_y, g_xy, g_yy);
//   HJet (v, a, t, at): hyper-dual in one space direction a and time, second
//        pass (W_tt needs f_xt with a = x and g_yt with a = y only).
// Every kept component is formed by the same expression as in the full jet.
template <typename R> struct SJet {
  R v, x, y, xx, xy, yy;
};
template <typename R> struct HJet {
  R v, a, t, at;
};

template <typename R> __device__ __forceinline__ SJet<R> jadd(const SJet<R>& a, const SJet<R>& b) {
  return {a.v + b.v, a.x + b.x, a.y + b.y, a.xx + b.xx, a.xy + b.xy, a.yy + b.yy};
}
template <typename R> __device__ __forceinline__ SJet<R> jscale(R s, const SJet<R>& a) {
  return {s * a.v, s * a.x, s * a.y, s * a.xx, s * a.xy, s * a.yy};
}
template <typename R> __device__ __forceinline__ SJet<R> jmul(const SJet<R>& a, const SJet<R>& b) {
  SJet<R> c;
  c.v = a.v * b.v;
  c.x = a.x * b.v + a.v * b.x;
  c.y = a.y * b.v + a.v * b.y;
  c.xx = a.xx * b.v + R(2) * a.x * b.x + a.v * b.xx;
  c.xy = a.xy * b.v + a.x * b.y + a.y * b.x + a.v * b.xy;
  c.yy = a.yy * b.v + R(2) * a.y * b.y + a.v * b.yy;
  return c;
}
template <typename R> __device__ __forceinline__ SJet<R> jrecip(const SJet<R>& a) {
  SJet<R> r;
  r.v = R(1) / a.v;
  const R r2 = r.v * r.v;
  r.x = -a.x * r2;
  r.y = -a.y * r2;
  r.xx = -a.xx * r2 - R(2) * a.x * r.v * r.x;
  r.xy = -a.xy * r2 - R(2) * a.x * r.v * r.y;
  r.yy = -a.yy * r2 - R(2) * a.y * r.v * r.y;
  return r;
}
// c = a * b, reverse
template <typename R>
__device__ __forceinline__ void jmul_vjp(const SJet<R>& a, const SJet<R>& b, const SJet<R>& cb, SJet<R>& ab,
                                         SJet<R>& bb) {
  ab.v += cb.v * b.v + cb.x * b.x + cb.y * b.y + cb.xx * b.xx + cb.xy * b.xy + cb.yy * b.yy;
  ab.x += cb.x * b.v + R(2) * cb.xx * b.x + cb.xy * b.y;
  ab.y += cb.y * b.v + cb.xy * b.x + R(2) * cb.yy * b.y;
  ab.xx += cb.xx * b.v;
  ab.xy += cb.xy * b.v;
  ab.yy += cb.yy * b.v;
  bb.v += cb.v * a.v + cb.x * a.x + cb.y * a.y + cb.xx * a.xx + cb.xy * a.xy + cb.yy * a.yy;
  bb.x += cb.x * a.v + R(2) * cb.xx * a.x + cb.xy * a.y;
  bb.y += cb.y * a.v + cb.xy * a.x + R(2) * cb.yy * a.y;
  bb.xx += cb.xx * a.v;
  bb.xy += cb.xy * a.v;
  bb.yy += cb.yy * a.v;
}
// r = 1 / a (r: the forward result), reverse
template <typename R>
__device__ __forceinline__ void jrecip_vjp(const SJet<R>& a, const SJet<R>& r, const SJet<R>& rb, SJet<R>& ab) {
  const R rv = r.v, r2 = rv * rv;
  R Rx = rb.x, Ry = rb.y, r2b = R(0), rvb = R(0);
  ab.yy += -r2 * rb.yy; r2b += -a.yy * rb.yy; ab.y += R(-2) * rv * r.y * rb.yy; rvb += R(-2) * a.y * r.y * rb.yy;
  Ry += R(-2) * a.y * rv * rb.yy;
  ab.xy += -r2 * rb.xy; r2b += -a.xy * rb.xy; ab.x += R(-2) * rv * r.y * rb.xy; rvb += R(-2) * a.x * r.y * rb.xy;
  Ry += R(-2) * a.x * rv * rb.xy;
  ab.xx += -r2 * rb.xx; r2b += -a.xx * rb.xx; ab.x += R(-2) * rv * r.x * rb.xx; rvb += R(-2) * a.x * r.x * rb.xx;
  Rx += R(-2) * a.x * rv * rb.xx;
  ab.y += -r2 * Ry; r2b += -a.y * Ry;
  ab.x += -r2 * Rx; r2b += -a.x * Rx;
  rvb += R(2) * rv * r2b;
  ab.v += -r2 * (rb.v + rvb);
}

template <typename R> __device__ __forceinline__ HJet<R> jadd(const HJet<R>& a, const HJet<R>& b) {
  return {a.v + b.v, a.a + b.a, a.t + b.t, a.at + b.at};
}
template <typename R> __device__ __forceinline__ HJet<R> jscale(R s, const HJet<R>& a) {
  return {s * a.v, s * a.a, s * a.t, s * a.at};
}
template <typename R> __device__ __forceinline__ HJet<R> jmul(const HJet<R>& a, const HJet<R>& b) {
  HJet<R> c;
  c.v = a.v * b.v;
  c.a = a.a * b.v + a.v * b.a;
  c.t = a.t * b.v + a.v * b.t;
  c.at = a.at * b.v + a.a * b.t + a.t * b.a + a.v * b.at;
  return c;
}
template <typename R> __device__ __forceinline__ HJet<R> jrecip(const HJet<R>& a) {
  HJet<R> r;
  r.v = R(1) / a.v;
  const R r2 = r.v * r.v;
  r.a = -a.a * r2;
  r.t = -a.t * r2;
  r.at = -a.at * r2 - R(2) * a.t * r.v * r.a;
  return r;
}
template <typename R>
__device__ __forceinline__ void jmul_vjp(const HJet<R>& a, const HJet<R>& b, const HJet<R>& cb, HJet<R>& ab,
                                         HJet<R>& bb) {
  ab.v += cb.v * b.v + cb.a * b.a + cb.t * b.t + cb.at * b.at;
  ab.a += cb.a * b.v + cb.at * b.t;
  ab.t += cb.t * b.v + cb.at * b.a;
  ab.at += cb.at * b.v;
  bb.v += cb.v * a.v + cb.a * a.a + cb.t * a.t + cb.at * a.at;
  bb.a += cb.a * a.v + cb.at * a.t;
  bb.t += cb.t * a.v + cb.at * a.a;
  bb.at += cb.at * a.v;
}
template <typename R>
__device__ __forceinline__ void jrecip_vjp(const HJet<R>& a, const HJet<R>& r, const HJet<R>& rb, HJet<R>& ab) {
  const R rv = r.v, r2 = rv * rv;
  R Ra = rb.a, r2b = R(0), rvb = R(0);
  ab.at += -r2 * rb.at; r2b += -a.at * rb.at; ab.t += R(-2) * rv * r.a * rb.at; rvb += R(-2) * a.t * r.a * rb.at;
  Ra += R(-2) * a.t * rv * rb.at;
  ab.t += -r2 * rb.t; r2b += -a.t * rb.t;
  ab.a += -r2 * Ra; r2b += -a.a * Ra;
  rvb += R(2) * rv * r2b;
  ab.v += -r2 * (rb.v + rvb);
}

template <typename J> __device__ __forceinline__ J jzero() { return J{}; }
template <typename J> __device__ __forceinline__ void jacc(J& a, const J& b) { a = jadd(a, b); }

// Euler fluxes through jets, reverse: cotangents of f (if F) and g (if G) ->
// cotangents of W, accumulated into Wb.  The forward intermediates are those
// of euler_flux_jets (device.cuh).
template <typename R, typename JT, bool F, bool G>
__device__ __forceinline__ void euler_flux_jets_vjp(const JT W[4], R gm1, const JT fb[4], const JT gb[4], JT Wb[4]) {
  const JT ir = jrecip(W[0]);
  const JT u = jmul(W[1], ir), v = jmul(W[2], ir);
  const JT mu = jmul(W[1], u), nv = jmul(W[2], v);
  const JT p = jscale(gm1, jadd(W[3], jscale(R(-0.5), jadd(mu, nv))));
  const JT H = jadd(W[3], p);
  JT irb = jzero<JT>(), ub = jzero<JT>(), vb = jzero<JT>(), mub = jzero<JT>(), nvb = jzero<JT>(),
     nub = jzero<JT>(), pb = jzero<JT>(), Hb = jzero<JT>();
  if constexpr (F) {
    jacc(Wb[1], fb[0]);
    jacc(mub, fb[1]); jacc(pb, fb[1]);
    jacc(nub, fb[2]);
    jmul_vjp(H, u, fb[3], Hb, ub);
  }
  if constexpr (G) {
    jacc(Wb[2], gb[0]);
    jacc(nub, gb[1]);
    jacc(nvb, gb[2]); jacc(pb, gb[2]);
    jmul_vjp(H, v, gb[3], Hb, vb);
  }
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
                                                       const R* Wttb, SJet<R> Jb[4]) {
  // forward first pass: W_t, W_tx, W_ty
  SJet<R> J[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) J[c] = {W[c], Wx[c], Wy[c], Wxx[c], Wxy[c], Wyy[c]};
  R wt[4], wtx[4], wty[4];
  {
    const SJet<R> ir = jrecip(J[0]);
    const SJet<R> u = jmul(J[1], ir), v = jmul(J[2], ir);
    const SJet<R> mu = jmul(J[1], u), nv = jmul(J[2], v), nu = jmul(J[2], u);
    const SJet<R> p = jscale(gm1, jadd(J[3], jscale(R(-0.5), jadd(mu, nv))));
    const SJet<R> H = jadd(J[3], p);
    const SJet<R> f[4] = {J[1], jadd(mu, p), nu, jmul(H, u)};
    const SJet<R> g[4] = {J[2], nu, jadd(nv, p), jmul(H, v)};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      wt[c] = -(f[c].x + g[c].y);
      wtx[c] = -(f[c].xx + g[c].xy);
      wty[c] = -(f[c].xy + g[c].yy);
    }
  }
  // second pass, reverse: W_tt = -(f_xt + g_yt) on the (x, t) and (y, t) hyper-duals
  R tb[4], txb[4], tyb[4];
  {
    HJet<R> A[4], Ab[4], fb[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      A[c] = {W[c], Wx[c], wt[c], wtx[c]};
      Ab[c] = jzero<HJet<R>>();
      fb[c] = jzero<HJet<R>>();
      fb[c].at = -Wttb[c];
    }
    euler_flux_jets_vjp<R, HJet<R>, true, false>(A, gm1, fb, fb, Ab);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      Jb[c].v += Ab[c].v;
      Jb[c].x += Ab[c].a;
      tb[c] = Ab[c].t + Wtb[c];
      txb[c] = Ab[c].at;
    }
  }
  {
    HJet<R> B[4], Bb[4], gb[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      B[c] = {W[c], Wy[c], wt[c], wty[c]};
      Bb[c] = jzero<HJet<R>>();
      gb[c] = jzero<HJet<R>>();
      gb[c].at = -Wttb[c];
    }
    euler_flux_jets_vjp<R, HJet<R>, false, true>(B, gm1, gb, gb, Bb);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      Jb[c].v += Bb[c].v;
      Jb[c].y += Bb[c].a;
      tb[c] += Bb[c].t;
      tyb[c] = Bb[c].at;
    }
  }
  // first pass, reverse: seeds on f_x, f_xx, f_xy and g_y, g_xy, g_yy
  SJet<R> f1b[4], g1b[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    f1b[c] = {R(0), -tb[c], R(0), -txb[c], -tyb[c], R(0)};
    g1b[c] = {R(0), R(0), -tb[c], R(0), -txb[c], -tyb[c]};
  }
  euler_flux_jets_vjp<R, SJet<R>, true, true>(J, gm1, f1b, g1b, Jb);
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
// g, eps: the linear weights and epsilon in the precision T
template <typename T>
__device__ __forceinline__ void nonlinear_weights_vjp_t(T Wave, const T beta[4], const T g[4], T eps, const T omb[4],
                                                        T& Waveb, T betab[4]) {
  const T tau = fabs(beta[0] - beta[1]) + fabs(beta[0] - beta[2]) + fabs(beta[0] - beta[3]);
  const T kappa = tau * tau / T(9);
  const T W2 = Wave * Wave, W4 = W2 * W2;
  T D[4], wb[4], s = T(0);
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    D[l] = W4 * eps + W2 * beta[l];
    wb[l] = g[l] * (T(1) + kappa / D[l]);
    s += wb[l];
  }
  T dot = T(0);
#pragma unroll
  for (int l = 0; l < 4; ++l) dot += omb[l] * (wb[l] / s);
  T kappab = T(0), W4b = T(0), W2b = T(0);
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const T wbb = (omb[l] - dot) / s;
    kappab += g[l] * wbb / D[l];
    const T Db = -g[l] * kappa * wbb / (D[l] * D[l]);
    W4b += eps * Db;
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

__device__ __forceinline__ void nonlinear_weights_vjp(double Wave, const double beta[4], const EqParams& P,
                                                      const double omb[4], double& Waveb, double betab[4]) {
  nonlinear_weights_vjp_t<double>(Wave, beta, P.g, P.eps, omb, Waveb, betab);
}

// float: the same branch as the forward (double where W_ave^4 eps is not a
// normal float)
__device__ __forceinline__ void nonlinear_weights_vjp(float Wave, const float beta[4], const EqParams& P,
                                                      const float omb[4], float& Waveb, float betab[4]) {
  if (fabsf(Wave) < 9.5367431640625e-07f) {
    double bd[4] = {beta[0], beta[1], beta[2], beta[3]}, od[4] = {omb[0], omb[1], omb[2], omb[3]};
    double wab = 0.0, bbd[4] = {0, 0, 0, 0};
    nonlinear_weights_vjp_t<double>((double)Wave, bd, P.g, P.eps, od, wab, bbd);
    Waveb += (float)wab;
#pragma unroll
    for (int l = 0; l < 4; ++l) betab[l] += (float)bbd[l];
    return;
  }
  nonlinear_weights_vjp_t<float>(Wave, beta, P.gf, P.epsf, omb, Waveb, betab);
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
  nonlinear_weights(Wave, beta, P, om);
  const R a1 = om[0] / EqC<R>::g(P, 0);
  R al[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) al[l] = om[l + 1] - a1 * EqC<R>::g(P, l + 1);
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
    a1b += -EqC<R>::g(P, l + 1) * alb;
  }
  omb[0] += a1b / EqC<R>::g(P, 0);
  R Waveb = R(0), betab[4] = {R(0), R(0), R(0), R(0)};
  nonlinear_weights_vjp(Wave, beta, P, omb, Waveb, betab);
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
