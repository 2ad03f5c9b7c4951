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

}  // namespace

// 16-byte copies of `bytes` (a multiple of 16) from 16-byte aligned global
// memory (read through the non-coherent path) to shared memory
__device__ __forceinline__ void copy16(void* dst, const void* src, int bytes, int t, int nt) {
  const int n = bytes / 16;
  for (int k = t; k < n; k += nt) reinterpret_cast<uint4*>(dst)[k] = __ldg(reinterpret_cast<const uint4*>(src) + k);
}

// `n` words of R (n * sizeof(R) a multiple of 16) from 16-byte aligned global memory
template <typename R, int n> __device__ __forceinline__ void load_vec(R (&dst)[n], const R* src) {
  static_assert((n * sizeof(R)) % 16 == 0, "whole 16-byte chunks");
#pragma unroll
  for (int k = 0; k < (int)(n * sizeof(R) / 16); ++k) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(src) + k);
    memcpy(reinterpret_cast<char*>(dst) + 16 * k, &v, 16);
  }
}

// ---------------------------------------------------------------- edge
// Shared-memory tile of k_adj_edge (32 cells).  The point-record tile is
// overwritten in place by the point cotangents (each thread owns one point).
template <typename R> struct AdjEdgeTile {
  R pb[kAdjCells][18 * kM];
  R u[kAdjCells][3 * kM];
  R ub[kAdjCells][3 * kM];
  R geo[kEdgePlanes][kAdjCells];
  R wpart[kM][6][kAdjCells];
  int nb[4][kAdjCells];
};

template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_adj_edge(GeoView<R> G, const R* __restrict__ U,
                                                          const R* __restrict__ Pb, const R* __restrict__ Ub1,
                                                          R* __restrict__ Pbb, R* __restrict__ Ubw, EqParams P,
                                                          double dt) {
  constexpr int m = kM, rec = 3 * m, prec = 18 * m;
  __shared__ __align__(16) AdjEdgeTile<R> S;
  const int N = G.N;
  const int cell0 = blockIdx.x * kAdjCells;
  const int t = threadIdx.x, lc = t % kAdjCells, qp = t / kAdjCells, i = cell0 + lc;
  const R gam = EqC<R>::gam(P), gm1 = EqC<R>::gm1(P), dtr = R(dt);
  // stage the tile's own records (contiguous; the buffers hold whole tiles),
  // flux geometry and neighbour tables
  copy16(&S.pb[0][0], Pb + (size_t)cell0 * prec, kAdjCells * prec * (int)sizeof(R), t, kAdjThreads);
  copy16(&S.u[0][0], U + (size_t)cell0 * rec, kAdjCells * rec * (int)sizeof(R), t, kAdjThreads);
  copy16(&S.ub[0][0], Ub1 + (size_t)cell0 * rec, kAdjCells * rec * (int)sizeof(R), t, kAdjThreads);
  for (int k = t; k < kEdgePlanes * kAdjCells; k += kAdjThreads) {
    const int p = k / kAdjCells, l = k % kAdjCells;
    S.geo[p][l] = G.r(G_NRM + p, cell0 + l);
  }
  for (int k = t; k < 4 * kAdjCells; k += kAdjThreads) {
    const int j = k / kAdjCells, l = k % kAdjCells;
    S.nb[j][l] = cell0 + l < N ? G.n(I_NBR + j, cell0 + l) : -1;
  }
  __syncthreads();
  if (i < N) {
    const int j = qp >> 1, gm = qp & 1;   // this thread's point: local edge j, Gauss point gm (record qp)
    const int nb = S.nb[j][lc];
    const int je = (S.nb[3][lc] >> (2 * j)) & 3;
    const bool left = (nb < 0) || (i < nb);
    const R nx = S.geo[G_NRM - G_NRM + 2 * j][lc], ny = S.geo[G_NRM - G_NRM + 2 * j + 1][lc];
    const R el = S.geo[G_EL - G_NRM + j][lc];
    R Wi[m], Wn[m];
#pragma unroll
    for (int c = 0; c < m; ++c) Wi[c] = S.u[lc][c];
    R mine[rec], theirs[rec], ubn[rec];
#pragma unroll
    for (int k = 0; k < rec; ++k) mine[k] = S.pb[lc][qp * rec + k];
    if (nb >= 0) {
      load_vec<R, m>(Wn, U + (size_t)nb * rec);
      load_vec<R, rec>(theirs, Pb + (size_t)nb * prec + (2 * je + (1 - gm)) * rec);   // reversed point order
      load_vec<R, rec>(ubn, Ub1 + (size_t)nb * rec);
    } else {
#pragma unroll
      for (int c = 0; c < m; ++c) Wn[c] = Wi[c];
#pragma unroll
      for (int k = 0; k < rec; ++k) { theirs[k] = mine[k]; ubn[k] = R(0); }
    }
    const R aL = left ? spectral_radius_n<R, kEqEuler>(Wi, nx, ny, P) : spectral_radius_n<R, kEqEuler>(Wn, nx, ny, P);
    const R aR = left ? spectral_radius_n<R, kEqEuler>(Wn, nx, ny, P) : spectral_radius_n<R, kEqEuler>(Wi, nx, ny, P);
    const R alpha = aL > aR ? aL : aR;
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
      const R wi = S.ub[lc][c], vi = S.ub[lc][m + c], yi = S.ub[lc][2 * m + c];
      Feb[c] = R(-0.5) * dtr * sgn * el * wi;
      Shb[c] = R(0.5) * sgn * el * (nx * vi + ny * yi);
    }
    if (nb >= 0) {
      const R eln = G.r(G_EL + je, nb);
#pragma unroll
      for (int c = 0; c < m; ++c) {
        Feb[c] += R(-0.5) * dtr * (-sgn) * eln * ubn[c];
        Shb[c] += R(0.5) * (-sgn) * eln * (nx * ubn[m + c] + ny * ubn[2 * m + c]);
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
    // this cell's share: its Taylor data (in place of its point record), and
    // its average through the viscosity
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int c = 0; c < m; ++c) {
        R v = left ? ab[k][c] : bb[k][c];
        if (nb < 0) v = ab[k][c] + bb[k][c];   // boundary: W^ext = W^int
        S.pb[lc][qp * rec + k * m + c] = v;
      }
    R Wib[m] = {R(0), R(0), R(0), R(0)};
    const bool right_wins = !(aL > aR);
    const bool mine_wins = left ? !right_wins : right_wins;
    if (nb >= 0 && mine_wins) spectral_radius_n_euler_vjp(Wi, nx, ny, gam, alphab, Wib);
#pragma unroll
    for (int c = 0; c < m; ++c) S.wpart[c][qp][lc] = Wib[c];
  }
  __syncthreads();
  const int valid = N - cell0 < kAdjCells ? N - cell0 : kAdjCells;
  for (int k = t; k < valid * prec * (int)sizeof(R) / 16; k += kAdjThreads)
    reinterpret_cast<uint4*>(Pbb + (size_t)cell0 * prec)[k] = reinterpret_cast<const uint4*>(&S.pb[0][0])[k];
  for (int k = t; k < rec * valid; k += kAdjThreads) {
    const int l = k / rec, o = k % rec;
    R v = R(0);
    if (o < m) {   // identity term of Eq. flx plus the viscosity shares
      v = S.ub[l][o];
#pragma unroll
      for (int q = 0; q < 6; ++q) v += S.wpart[o][q][l];
    }
    Ubw[(size_t)(cell0 + l) * rec + o] = v;
  }
}

// ---------------------------------------------------------------- reconstruction
// Shared-memory tile of k_adj_recon (32 cells).  The point-cotangent tile is
// reused for the contribution tile once the points are done.
template <typename R> struct AdjReconTile {
  R geo[kReconPlanes][kAdjCells];        // reconstruction geometry, planes 0 .. G_IH
  R us[4][kAdjCells][3 * kM];             // stencil records: 0 = the cell, 1 + j = neighbour j (the cell itself at a boundary)
  R pbb[kAdjCells][18 * kM];              // point cotangents; then the contributions [cell][4 slots][3m]
  R qs[kM][6][kAdjCells];                 // combined quadratic
  R qbs[kM][6][6][kAdjCells];             // its cotangent per point: [component][coefficient][point][cell]
  int nb[3][kAdjCells];
};

template <typename R> struct TileGeo {
  const R (*geo)[kAdjCells];
  int l;
  __device__ __forceinline__ R operator()(int p) const { return geo[p][l]; }
};

template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_adj_recon(GeoView<R> G, const R* __restrict__ U,
                                                           const R* __restrict__ Pbb, R* __restrict__ Cb, EqParams P) {
  constexpr int m = kM, rec = 3 * m;
  extern __shared__ __align__(16) unsigned char adj_smem[];
  AdjReconTile<R>& S = *reinterpret_cast<AdjReconTile<R>*>(adj_smem);
  const int N = G.N;
  const int cell0 = blockIdx.x * kAdjCells;
  const int t = threadIdx.x;
  // stage: geometry planes (coalesced per plane), neighbours, point cotangents
  // (one contiguous block of records; the buffers hold whole tiles)
  for (int k = t; k < kReconPlanes * kAdjCells; k += kAdjThreads) {
    const int p = k / kAdjCells, l = k % kAdjCells;
    S.geo[p][l] = G.r(p, cell0 + l);
  }
  for (int k = t; k < 3 * kAdjCells; k += kAdjThreads) {
    const int j = k / kAdjCells, l = k % kAdjCells, i = cell0 + l;
    S.nb[j][l] = i < N ? G.n(I_NBR + j, i) : -1;
  }
  copy16(&S.pbb[0][0], Pbb + (size_t)cell0 * 18 * m, kAdjCells * 18 * m * (int)sizeof(R), t, kAdjThreads);
  __syncthreads();
  {
    constexpr int c16 = rec * (int)sizeof(R) / 16;   // 16-byte chunks per record
    for (int k = t; k < 4 * kAdjCells * c16; k += kAdjThreads) {
      const int q = k % c16, l = (k / c16) % kAdjCells, slot = k / (c16 * kAdjCells), i = cell0 + l;
      int src = i < N ? i : 0;
      if (slot > 0 && i < N && S.nb[slot - 1][l] >= 0) src = S.nb[slot - 1][l];
      reinterpret_cast<uint4*>(&S.us[slot][l][0])[q] = __ldg(reinterpret_cast<const uint4*>(U + (size_t)src * rec) + q);
    }
  }
  __syncthreads();
  // phase 1: forward reconstruction per (cell, component)
  if (t < m * kAdjCells) {
    const int lc = t % kAdjCells, c = t / kAdjCells;
    if (cell0 + lc < N) {
      R Wl[3], Vl[3], Yl[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) { Wl[j] = S.us[1 + j][lc][c]; Vl[j] = S.us[1 + j][lc][m + c]; Yl[j] = S.us[1 + j][lc][2 * m + c]; }
      R q[6];
      reconstruct_component<R>(TileGeo<R>{S.geo, lc}, S.us[0][lc][c], S.us[0][lc][m + c], S.us[0][lc][2 * m + c], Wl,
                               Vl, Yl, P, q);
#pragma unroll
      for (int k = 0; k < 6; ++k) S.qs[c][k][lc] = q[k];
    }
  }
  __syncthreads();
  // phase 2: per (cell, point): reverse of the Lax-Wendroff procedure and of the
  // point evaluation -> cotangents of the combined quadratic
  {
    const int lc = t % kAdjCells, qp = t / kAdjCells;
    if (cell0 + lc < N) {
      const int j = qp >> 1, g = qp & 1, jn = (j + 1) % 3;
      const R sg = g == 0 ? R(0.5) - R(0.28867513459481288225) : R(0.5) + R(0.28867513459481288225);
      const R xa = S.geo[G_VX + 2 * j][lc], ya = S.geo[G_VX + 2 * j + 1][lc];
      const R xi = xa + sg * (S.geo[G_VX + 2 * jn][lc] - xa);
      const R et = ya + sg * (S.geo[G_VX + 2 * jn + 1][lc] - ya);
      const R ih = S.geo[G_IH][lc], ih2 = ih * ih;
      R W[m], Wx[m], Wy[m], Wxx[m], Wxy[m], Wyy[m];
#pragma unroll
      for (int c = 0; c < m; ++c) {
        const R q0 = S.qs[c][0][lc], q1 = S.qs[c][1][lc], q2 = S.qs[c][2][lc];
        const R q3 = S.qs[c][3][lc], q4 = S.qs[c][4][lc], q5 = S.qs[c][5][lc];
        W[c] = q0 + xi * (q1 + q3 * xi + q4 * et) + et * (q2 + q5 * et);
        Wx[c] = (q1 + R(2) * q3 * xi + q4 * et) * ih;
        Wy[c] = (q2 + q4 * xi + R(2) * q5 * et) * ih;
        Wxx[c] = R(2) * q3 * ih2; Wxy[c] = q4 * ih2; Wyy[c] = R(2) * q5 * ih2;
      }
      R Wtb[m], Wttb[m];
      SJet<R> Jb[4];
#pragma unroll
      for (int c = 0; c < m; ++c) {
        Jb[c] = jzero<SJet<R>>();
        Jb[c].v = S.pbb[lc][qp * rec + c];
        Wtb[c] = S.pbb[lc][qp * rec + m + c];
        Wttb[c] = S.pbb[lc][qp * rec + 2 * m + c];
      }
      lax_wendroff_euler_vjp(W, Wx, Wy, Wxx, Wxy, Wyy, EqC<R>::gm1(P), Wtb, Wttb, Jb);
#pragma unroll
      for (int c = 0; c < m; ++c) {
        const R wv = Jb[c].v, wx = Jb[c].x * ih, wy = Jb[c].y * ih;
        S.qbs[c][0][qp][lc] = wv;
        S.qbs[c][1][qp][lc] = xi * wv + wx;
        S.qbs[c][2][qp][lc] = et * wv + wy;
        S.qbs[c][3][qp][lc] = xi * xi * wv + R(2) * xi * wx + R(2) * ih2 * Jb[c].xx;
        S.qbs[c][4][qp][lc] = xi * et * wv + et * wx + xi * wy + ih2 * Jb[c].xy;
        S.qbs[c][5][qp][lc] = et * et * wv + R(2) * et * wy + R(2) * ih2 * Jb[c].yy;
      }
    }
  }
  __syncthreads();
  // phase 3: per (cell, component): reverse of Steps 1-6; contributions into
  // the tile: slot 0 = the cell itself, slot 1 + j = its neighbour j
  R* cbt = &S.pbb[0][0];
  if (t < m * kAdjCells) {
    const int lc = t % kAdjCells, c = t / kAdjCells;
    if (cell0 + lc < N) {
      R qb[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        R s = R(0);
#pragma unroll
        for (int q = 0; q < 6; ++q) s += S.qbs[c][k][q][lc];
        qb[k] = s;
      }
      R Wl[3], Vl[3], Yl[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) { Wl[j] = S.us[1 + j][lc][c]; Vl[j] = S.us[1 + j][lc][m + c]; Yl[j] = S.us[1 + j][lc][2 * m + c]; }
      R o0[3], ol[3][3];
      reconstruct_component_vjp<R>(TileGeo<R>{S.geo, lc}, S.us[0][lc][c], S.us[0][lc][m + c], S.us[0][lc][2 * m + c],
                                   Wl, Vl, Yl, P, qb, o0, ol);
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (S.nb[j][lc] < 0)
#pragma unroll
          for (int k = 0; k < 3; ++k) { o0[k] += ol[j][k]; ol[j][k] = R(0); }
      R* out = cbt + lc * 4 * rec;
#pragma unroll
      for (int k = 0; k < 3; ++k) out[k * m + c] = o0[k];
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) out[(1 + j) * rec + k * m + c] = ol[j][k];
    }
  }
  __syncthreads();
  const int valid = N - cell0 < kAdjCells ? N - cell0 : kAdjCells;
  for (int k = t; k < valid * 4 * rec * (int)sizeof(R) / 16; k += kAdjThreads)
    reinterpret_cast<uint4*>(Cb + (size_t)cell0 * 4 * rec)[k] = reinterpret_cast<const uint4*>(cbt)[k];
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
  cudaFuncSetAttribute(k_adj_recon<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(AdjReconTile<R>));
  k_adj_recon<R><<<nb, kAdjThreads, sizeof(AdjReconTile<R>), st>>>(G, reinterpret_cast<const R*>(a.U),
                                                                     reinterpret_cast<const R*>(a.Pbb),
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
