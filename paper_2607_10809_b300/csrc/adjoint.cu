// Adjoint of one ADER-HWENO time step (Euler; scale limiter off), with the
// time step held fixed: given the cotangent of U^{n+1}, the cotangent of U^n.
// Gather-only (no atomics, deterministic):
//   k_adj_edge  : per cell and Gauss point, the reverse of the point flux and
//                 of the central value (Eqs. flux, timeflux) under the
//                 cotangents of both cells of the edge; keeps this cell's share:
//                 the cotangent of its edge-point Taylor data and of its own
//                 cell average (identity term of Eq. flx and the viscosity).
//   k_adj_recon : per cell, the reverse of the Lax-Wendroff procedure at its six
//                 points, of the point evaluation and of Steps 1-6 (Section
//                 2.2); writes one contribution per stencil member.
//   k_adj_gather: per cell, sums its own contributions and those its
//                 neighbours wrote for it.
// The forward Taylor data of U^n are recomputed first by k_recon.
#include <cuda.h>

#include <cstdint>

#include "adjoint.cuh"
#include "kernels.h"

namespace hw {

namespace {
constexpr int kM = 4;   // Euler
constexpr int kAdjCells = 32;
constexpr int kAdjThreads = 6 * kAdjCells;

template <typename R> struct GlobalGeo {
  const GeoView<R>* G;
  int i;
  __device__ __forceinline__ R operator()(int p) const { return G->r(p, i); }
};
}  // namespace

// ---------------------------------------------------------------- edge
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_adj_edge(GeoView<R> G, const R* __restrict__ U,
                                                          const R* __restrict__ Pb, const R* __restrict__ Ub1,
                                                          R* __restrict__ Pbb, R* __restrict__ Ubw, EqParams P,
                                                          double dt) {
  constexpr int m = kM;
  __shared__ R wpart[m][6][kAdjCells];
  const int N = G.N;
  const int cell0 = blockIdx.x * kAdjCells;
  const int t = threadIdx.x, lc = t % kAdjCells, qp = t / kAdjCells, i = cell0 + lc;
  const R gam = R(P.gam), gm1 = R(P.gam - 1.0), dtr = R(dt);
  if (i < N) {
    const int j = qp >> 1, gm = qp & 1;
    const int nb = G.n(I_NBR + j, i);
    const int je = (G.n(I_NBE, i) >> (2 * j)) & 3;
    const bool left = (nb < 0) || (i < nb);
    const R nx = G.r(G_NRM + 2 * j, i), ny = G.r(G_NRM + 2 * j + 1, i);
    const R el = G.r(G_EL + j, i);
    R Wi[m], Wn[m];
#pragma unroll
    for (int c = 0; c < m; ++c) {
      Wi[c] = U[(size_t)i * 3 * m + c];
      Wn[c] = nb >= 0 ? U[(size_t)nb * 3 * m + c] : Wi[c];
    }
    const R aL = left ? spectral_radius_n<R, kEqEuler>(Wi, nx, ny, P) : spectral_radius_n<R, kEqEuler>(Wn, nx, ny, P);
    const R aR = left ? spectral_radius_n<R, kEqEuler>(Wn, nx, ny, P) : spectral_radius_n<R, kEqEuler>(Wi, nx, ny, P);
    const R alpha = aL > aR ? aL : aR;
    const int qm = 2 * j + gm, qn = 2 * je + (1 - gm);
    R mine[3 * m], theirs[3 * m];
#pragma unroll
    for (int k = 0; k < 3 * m; ++k) {
      mine[k] = Pb[(size_t)i * 18 * m + qm * 3 * m + k];
      theirs[k] = nb >= 0 ? Pb[(size_t)nb * 18 * m + qn * 3 * m + k] : mine[k];
    }
    R a[3][m], b[3][m];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int c = 0; c < m; ++c) {
        a[k][c] = left ? mine[k * m + c] : theirs[k * m + c];
        b[k][c] = left ? theirs[k * m + c] : mine[k * m + c];
      }
    // cotangents of this point's time-integrated flux and central value:
    // both cells of the edge use them (signs +- of the canonical normal)
    const R sgn = left ? R(1) : R(-1);
    R Feb[m], Shb[m];
#pragma unroll
    for (int c = 0; c < m; ++c) {
      const R wi = Ub1[(size_t)i * 3 * m + c], vi = Ub1[(size_t)i * 3 * m + m + c], yi = Ub1[(size_t)i * 3 * m + 2 * m + c];
      Feb[c] = R(-0.5) * dtr * sgn * el * wi;
      Shb[c] = R(0.5) * sgn * el * (nx * vi + ny * yi);
    }
    if (nb >= 0) {
      const R eln = G.r(G_EL + je, nb);
#pragma unroll
      for (int c = 0; c < m; ++c) {
        const R wn = Ub1[(size_t)nb * 3 * m + c], vn = Ub1[(size_t)nb * 3 * m + m + c],
                yn = Ub1[(size_t)nb * 3 * m + 2 * m + c];
        Feb[c] += R(-0.5) * dtr * (-sgn) * eln * wn;
        Shb[c] += R(0.5) * (-sgn) * eln * (nx * vn + ny * yn);
      }
    }
    // reverse of the Lobatto sum of the LLF flux (and of Eq. timeflux at tau = dt)
    const R tau[3] = {R(0), R(0.5) * dtr, dtr};
    const R wts[3] = {R(1.0 / 6.0), R(4.0 / 6.0), R(1.0 / 6.0)};
    R ab[3][m], bb[3][m], alphab = R(0);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int c = 0; c < m; ++c) { ab[k][c] = R(0); bb[k][c] = R(0); }
#pragma unroll
    for (int si = 0; si < 3; ++si) {
      const R hs = R(0.5) * tau[si] * tau[si];
      R WL[m], WR[m], HLb[m], HRb[m], WLb[m], WRb[m];
#pragma unroll
      for (int c = 0; c < m; ++c) {
        WL[c] = a[0][c] + tau[si] * a[1][c] + hs * a[2][c];
        WR[c] = b[0][c] + tau[si] * b[1][c] + hs * b[2][c];
        const R fb = wts[si] * R(0.5) * Feb[c];
        HLb[c] = fb; HRb[c] = fb;
        WLb[c] = alpha * fb; WRb[c] = -alpha * fb;
        alphab += -fb * (WR[c] - WL[c]);
        if (si == 2) { WLb[c] += R(0.5) * Shb[c]; WRb[c] += R(0.5) * Shb[c]; }
      }
      flux_n_euler_vjp(WL, nx, ny, gm1, HLb, WLb);
      flux_n_euler_vjp(WR, nx, ny, gm1, HRb, WRb);
#pragma unroll
      for (int c = 0; c < m; ++c) {
        ab[0][c] += WLb[c]; ab[1][c] += tau[si] * WLb[c]; ab[2][c] += hs * WLb[c];
        bb[0][c] += WRb[c]; bb[1][c] += tau[si] * WRb[c]; bb[2][c] += hs * WRb[c];
      }
    }
    // this cell's share: its Taylor data, and its average through the viscosity
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int c = 0; c < m; ++c) {
        R v = left ? ab[k][c] : bb[k][c];
        if (nb < 0) v = ab[k][c] + bb[k][c];   // boundary: W^ext = W^int
        Pbb[(size_t)i * 18 * m + qm * 3 * m + k * m + c] = v;
      }
    R Wib[m] = {R(0), R(0), R(0), R(0)};
    const bool right_wins = !(aL > aR);
    const bool mine_wins = left ? !right_wins : right_wins;
    if (nb >= 0 && mine_wins) spectral_radius_n_euler_vjp(Wi, nx, ny, gam, alphab, Wib);
#pragma unroll
    for (int c = 0; c < m; ++c) wpart[c][qp][lc] = Wib[c];
  }
  __syncthreads();
  for (int k = t; k < 3 * m * kAdjCells; k += kAdjThreads) {
    const int l = k % kAdjCells, o = k / kAdjCells, ii = cell0 + l;
    if (ii >= N) continue;
    R v = R(0);
    if (o < m) {   // identity term of Eq. flx plus the viscosity shares
      v = Ub1[(size_t)ii * 3 * m + o];
#pragma unroll
      for (int q = 0; q < 6; ++q) v += wpart[o][q][l];
    }
    Ubw[(size_t)ii * 3 * m + o] = v;
  }
}

// ---------------------------------------------------------------- reconstruction
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_adj_recon(GeoView<R> G, const R* __restrict__ U,
                                                           const R* __restrict__ Pbb, R* __restrict__ Cb, EqParams P) {
  constexpr int m = kM;
  __shared__ R qs[m][6][kAdjCells];
  __shared__ R qbs[m][6][6][kAdjCells];   // [component][coefficient][point][cell]
  const int N = G.N;
  const int cell0 = blockIdx.x * kAdjCells;
  const int t = threadIdx.x;
  const GeoView<R>* Gp = &G;
  // phase 1: forward reconstruction per (cell, component)
  if (t < m * kAdjCells) {
    const int lc = t % kAdjCells, c = t / kAdjCells, i = cell0 + lc;
    if (i < N) {
      R Wl[3], Vl[3], Yl[3];
      const R* own = U + (size_t)i * 3 * m;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int nb = G.n(I_NBR + j, i);
        const R* rec = nb >= 0 ? U + (size_t)nb * 3 * m : own;
        Wl[j] = rec[c]; Vl[j] = rec[m + c]; Yl[j] = rec[2 * m + c];
      }
      R q[6];
      reconstruct_component<R>(GlobalGeo<R>{Gp, i}, own[c], own[m + c], own[2 * m + c], Wl, Vl, Yl, P, q);
#pragma unroll
      for (int k = 0; k < 6; ++k) qs[c][k][lc] = q[k];
    }
  }
  __syncthreads();
  // phase 2: per (cell, point): reverse of the Lax-Wendroff procedure and of the
  // point evaluation -> cotangents of the combined quadratic
  {
    const int lc = t % kAdjCells, qp = t / kAdjCells, i = cell0 + lc;
    if (i < N) {
      const int j = qp >> 1, g = qp & 1, jn = (j + 1) % 3;
      const R sg = g == 0 ? R(0.5) - R(0.28867513459481288225) : R(0.5) + R(0.28867513459481288225);
      const R xa = G.r(G_VX + 2 * j, i), ya = G.r(G_VX + 2 * j + 1, i);
      const R xi = xa + sg * (G.r(G_VX + 2 * jn, i) - xa);
      const R et = ya + sg * (G.r(G_VX + 2 * jn + 1, i) - ya);
      const R ih = G.r(G_IH, i), ih2 = ih * ih;
      R W[m], Wx[m], Wy[m], Wxx[m], Wxy[m], Wyy[m];
#pragma unroll
      for (int c = 0; c < m; ++c) {
        const R q0 = qs[c][0][lc], q1 = qs[c][1][lc], q2 = qs[c][2][lc];
        const R q3 = qs[c][3][lc], q4 = qs[c][4][lc], q5 = qs[c][5][lc];
        W[c] = q0 + xi * (q1 + q3 * xi + q4 * et) + et * (q2 + q5 * et);
        Wx[c] = (q1 + R(2) * q3 * xi + q4 * et) * ih;
        Wy[c] = (q2 + q4 * xi + R(2) * q5 * et) * ih;
        Wxx[c] = R(2) * q3 * ih2; Wxy[c] = q4 * ih2; Wyy[c] = R(2) * q5 * ih2;
      }
      R Wb0[m], Wtb[m], Wttb[m];
#pragma unroll
      for (int c = 0; c < m; ++c) {
        Wb0[c] = Pbb[(size_t)i * 18 * m + qp * 3 * m + c];
        Wtb[c] = Pbb[(size_t)i * 18 * m + qp * 3 * m + m + c];
        Wttb[c] = Pbb[(size_t)i * 18 * m + qp * 3 * m + 2 * m + c];
      }
      Jet<R> Jb[4];
#pragma unroll
      for (int c = 0; c < m; ++c) { Jb[c] = jzero<R>(); Jb[c].v = Wb0[c]; }
      lax_wendroff_euler_vjp(W, Wx, Wy, Wxx, Wxy, Wyy, R(P.gam - 1.0), Wtb, Wttb, Jb);
#pragma unroll
      for (int c = 0; c < m; ++c) {
        const R wv = Jb[c].v, wx = Jb[c].x * ih, wy = Jb[c].y * ih;
        qbs[c][0][qp][lc] = wv;
        qbs[c][1][qp][lc] = xi * wv + wx;
        qbs[c][2][qp][lc] = et * wv + wy;
        qbs[c][3][qp][lc] = xi * xi * wv + R(2) * xi * wx + R(2) * ih2 * Jb[c].xx;
        qbs[c][4][qp][lc] = xi * et * wv + et * wx + xi * wy + ih2 * Jb[c].xy;
        qbs[c][5][qp][lc] = et * et * wv + R(2) * et * wy + R(2) * ih2 * Jb[c].yy;
      }
    }
  }
  __syncthreads();
  // phase 3: per (cell, component): reverse of Steps 1-6
  if (t < m * kAdjCells) {
    const int lc = t % kAdjCells, c = t / kAdjCells, i = cell0 + lc;
    if (i < N) {
      R qb[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        R s = R(0);
#pragma unroll
        for (int q = 0; q < 6; ++q) s += qbs[c][k][q][lc];
        qb[k] = s;
      }
      R Wl[3], Vl[3], Yl[3];
      int nbs[3];
      const R* own = U + (size_t)i * 3 * m;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        nbs[j] = G.n(I_NBR + j, i);
        const R* rec = nbs[j] >= 0 ? U + (size_t)nbs[j] * 3 * m : own;
        Wl[j] = rec[c]; Vl[j] = rec[m + c]; Yl[j] = rec[2 * m + c];
      }
      R o0[3], ol[3][3];
      reconstruct_component_vjp<R>(GlobalGeo<R>{Gp, i}, own[c], own[m + c], own[2 * m + c], Wl, Vl, Yl, P, qb, o0,
                                   ol);
      // contributions: slot 0 = the cell itself, slot 1 + j = its neighbour j
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (nbs[j] < 0)
#pragma unroll
          for (int k = 0; k < 3; ++k) { o0[k] += ol[j][k]; ol[j][k] = R(0); }
      R* out = Cb + (size_t)i * 4 * 3 * m;
#pragma unroll
      for (int k = 0; k < 3; ++k) out[0 * 3 * m + k * m + c] = o0[k];
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) out[(1 + j) * 3 * m + k * m + c] = ol[j][k];
    }
  }
}

// ---------------------------------------------------------------- gather
template <typename R>
__global__ void __launch_bounds__(256) k_adj_gather(GeoView<R> G, const R* __restrict__ Ubw, const R* __restrict__ Cb,
                                                    R* __restrict__ Ub0) {
  constexpr int m = kM;
  const int N = G.N;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = idx / (3 * m), o = idx % (3 * m);
  if (i >= N) return;
  R v = Ubw[(size_t)i * 3 * m + o] + Cb[(size_t)i * 4 * 3 * m + o];
  const int packed = G.n(I_NBE, i);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int nb = G.n(I_NBR + j, i);
    if (nb >= 0) {
      const int slot = 1 + ((packed >> (2 * j)) & 3);   // this cell is nb's neighbour across nb's local edge
      v += Cb[(size_t)nb * 4 * 3 * m + slot * 3 * m + o];
    }
  }
  Ub0[(size_t)i * 3 * m + o] = v;
}

// ---------------------------------------------------------------- launchers
namespace {
template <typename R> void launch_adjoint_t(const AdjointArgs& a, cudaStream_t st) {
  GeoView<R> G{reinterpret_cast<const R*>(a.rgeo), a.igeo, a.N, a.ld};
  const int nb = (a.N + kAdjCells - 1) / kAdjCells;
  k_adj_edge<R><<<nb, kAdjThreads, 0, st>>>(G, reinterpret_cast<const R*>(a.U), reinterpret_cast<const R*>(a.Pb),
                                            reinterpret_cast<const R*>(a.Ubar_next), reinterpret_cast<R*>(a.Pbb),
                                            reinterpret_cast<R*>(a.Ubw), a.P, a.dt);
  k_adj_recon<R><<<nb, kAdjThreads, 0, st>>>(G, reinterpret_cast<const R*>(a.U), reinterpret_cast<const R*>(a.Pbb),
                                             reinterpret_cast<R*>(a.Cb), a.P);
  const long long total = (long long)a.N * 3 * kM;
  k_adj_gather<R><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(G, reinterpret_cast<const R*>(a.Ubw),
                                                                  reinterpret_cast<const R*>(a.Cb),
                                                                  reinterpret_cast<R*>(a.Ubar));
}
}  // namespace

void launch_adjoint(int prec, const AdjointArgs& a, cudaStream_t st) {
  if (prec == 0) launch_adjoint_t<double>(a, st);
  else launch_adjoint_t<float>(a, st);
}

}  // namespace hw
