// Adjoint of one ADER-HWENO time step (Euler; scale limiter off), with the
// time step held fixed: given the cotangent of U^{n+1}, the cotangent of U^n.
// Gather-only (no atomics, deterministic):
//   k_adj_step  : persistent over tiles of 32 cells; the next tile's inputs
//                 are prefetched into shared memory (cp.async, double
//                 buffered) while the current one is processed:
//                 per (cell, point): the reverse of the point flux and of the
//                 central value (Eqs. flux, timeflux) under the cotangents of
//                 both cells of the edge, keeping this cell's share, then the
//                 reverse of the Lax-Wendroff procedure and of the point
//                 evaluation; per (cell, component): the reverse of Steps 1-6
//                 (Section 2.2).  Writes one contribution per stencil member
//                 (slot 0 also carries the identity term of Eq. flx and the
//                 cell's share of the numerical viscosity).
//   k_adj_gather: per cell, sums its own contributions and those its
//                 neighbours wrote for it.
// The forward Taylor data of U^n are recomputed first by k_recon.
#include <cuda.h>

#include <algorithm>
#include <cstdint>

#include "adjoint.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace hw {

namespace {
constexpr int kM = 4;   // Euler
constexpr int kAdjCells = 32;
constexpr int kAdjThreads = 6 * kAdjCells;

// cp.async: 16-byte and one-word asynchronous copies global -> shared, grouped
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
template <int bytes> __device__ __forceinline__ void cp_async_word(void* dst, const void* src) {
  static_assert(bytes == 4 || bytes == 8, "one word");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int n> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory");
}
}  // namespace

// One tile's inputs, staged ahead of use.
template <typename R> struct AdjIn {
  R geo[kStepPlanes][kAdjCells];    // the geometry planes of the step
  R pb[kAdjCells][18 * kM];         // own edge-point Taylor records; later the contribution tile [cell][4][3m]
  R us[4][kAdjCells][3 * kM];       // state records: 0 = the cell, 1 + j = neighbour j
  R ub[4][kAdjCells][3 * kM];       // cotangent-of-U^{n+1} records, same slots
  R pbn[6][kAdjCells][3 * kM];      // the neighbour's record of each edge point (its own point order)
  R eln[3][kAdjCells];              // |e_j| / |K_nb| seen from the neighbour across edge j
  int nb[4][kAdjCells];             // neighbours, packed local edges
};
template <typename R> struct AdjTile {
  AdjIn<R> in[2];
  R qs[kM][6][kAdjCells];           // combined quadratic
  R qbs[kM][6][6][kAdjCells];       // its cotangent per point: [component][coefficient][point][cell]
  R wpart[kM][6][kAdjCells];        // viscosity shares to the cell's own average, per point
};

template <typename R> struct TileGeo {
  const R (*geo)[kAdjCells];
  int l;
  __device__ __forceinline__ R operator()(int p) const { return geo[p][l]; }
};

struct AdjPtrs {
  const void* rg;
  const int32_t* ig;
  const void* U;
  const void* Pb;
  const void* Ub1;
  int N, ld;
};

// Stage 1 of a tile: the contiguous inputs (geometry planes, own records,
// neighbour tables).  Whole tiles are in bounds: every buffer holds ld cells.
template <typename R> __device__ __forceinline__ void issue_base(AdjIn<R>& B, const AdjPtrs& a, int cell0, int t) {
  constexpr int m = kM, rec = 3 * m, prec = 18 * m, cpr = (int)sizeof(R) * kAdjCells / 16;   // chunks per plane row
  const R* rg = static_cast<const R*>(a.rg);
  for (int k = t; k < kStepPlanes * cpr; k += kAdjThreads) {
    const int p = k / cpr, q = k % cpr;
    cp_async16(reinterpret_cast<char*>(&B.geo[p][0]) + 16 * q,
               reinterpret_cast<const char*>(rg + (size_t)p * a.ld + cell0) + 16 * q);
  }
  for (int k = t; k < 4 * 8; k += kAdjThreads) {   // 4 int planes x 32 cells = 8 chunks each
    const int p = k / 8, q = k % 8;
    cp_async16(reinterpret_cast<char*>(&B.nb[p][0]) + 16 * q,
               reinterpret_cast<const char*>(a.ig + (size_t)(I_NBR + p) * a.ld + cell0) + 16 * q);
  }
  const int cp = kAdjCells * prec * (int)sizeof(R) / 16, cr = kAdjCells * rec * (int)sizeof(R) / 16;
  const char* pb = reinterpret_cast<const char*>(static_cast<const R*>(a.Pb) + (size_t)cell0 * prec);
  for (int k = t; k < cp; k += kAdjThreads) cp_async16(reinterpret_cast<char*>(&B.pb[0][0]) + 16 * k, pb + 16 * k);
  const char* u = reinterpret_cast<const char*>(static_cast<const R*>(a.U) + (size_t)cell0 * rec);
  const char* ub = reinterpret_cast<const char*>(static_cast<const R*>(a.Ub1) + (size_t)cell0 * rec);
  for (int k = t; k < cr; k += kAdjThreads) {
    cp_async16(reinterpret_cast<char*>(&B.us[0][0][0]) + 16 * k, u + 16 * k);
    cp_async16(reinterpret_cast<char*>(&B.ub[0][0][0]) + 16 * k, ub + 16 * k);
  }
}

// Stage 2: the neighbours' records (needs the tile's neighbour table).
// Boundary ghosts take the cell's own state record; their other slots are
// not read.
template <typename R> __device__ __forceinline__ void issue_gather(AdjIn<R>& B, const AdjPtrs& a, int cell0, int t) {
  constexpr int m = kM, rec = 3 * m, prec = 18 * m, c16 = rec * (int)sizeof(R) / 16;
  const R* U = static_cast<const R*>(a.U);
  const R* Ub1 = static_cast<const R*>(a.Ub1);
  const R* Pb = static_cast<const R*>(a.Pb);
  const R* rg = static_cast<const R*>(a.rg);
  for (int k = t; k < 3 * kAdjCells * c16; k += kAdjThreads) {
    const int q = k % c16, l = (k / c16) % kAdjCells, j = k / (c16 * kAdjCells), i = cell0 + l;
    if (i >= a.N) continue;
    const int nb = B.nb[j][l];
    const int src = nb >= 0 ? nb : i;
    cp_async16(reinterpret_cast<char*>(&B.us[1 + j][l][0]) + 16 * q,
               reinterpret_cast<const char*>(U + (size_t)src * rec) + 16 * q);
    if (nb >= 0)
      cp_async16(reinterpret_cast<char*>(&B.ub[1 + j][l][0]) + 16 * q,
                 reinterpret_cast<const char*>(Ub1 + (size_t)nb * rec) + 16 * q);
  }
  for (int k = t; k < 6 * kAdjCells * c16; k += kAdjThreads) {
    const int q = k % c16, l = (k / c16) % kAdjCells, qp = k / (c16 * kAdjCells), i = cell0 + l;
    if (i >= a.N) continue;
    const int j = qp >> 1, gm = qp & 1;
    const int nb = B.nb[j][l];
    if (nb < 0) continue;
    const int je = (B.nb[3][l] >> (2 * j)) & 3;
    cp_async16(reinterpret_cast<char*>(&B.pbn[qp][l][0]) + 16 * q,
               reinterpret_cast<const char*>(Pb + (size_t)nb * prec + (2 * je + (1 - gm)) * rec) + 16 * q);
  }
  for (int k = t; k < 3 * kAdjCells; k += kAdjThreads) {
    const int l = k % kAdjCells, j = k / kAdjCells, i = cell0 + l;
    if (i >= a.N) continue;
    const int nb = B.nb[j][l];
    if (nb < 0) continue;
    const int je = (B.nb[3][l] >> (2 * j)) & 3;
    cp_async_word<(int)sizeof(R)>(&B.eln[j][l], rg + (size_t)(G_EL + je) * a.ld + nb);
  }
}

// ---------------------------------------------------------------- fused step adjoint
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_adj_step(AdjPtrs a, R* __restrict__ Cb, EqParams P, double dt,
                                                          int ntiles) {
  constexpr int m = kM, rec = 3 * m;
  extern __shared__ __align__(16) unsigned char adj_smem[];
  AdjTile<R>& S = *reinterpret_cast<AdjTile<R>*>(adj_smem);
  const int N = a.N;
  const int t = threadIdx.x;
  const R gam = EqC<R>::gam(P), gm1 = EqC<R>::gm1(P), dtr = R(dt);
  int tile = blockIdx.x;
  if (tile >= ntiles) return;
  // prologue: tile's inputs complete, the next tile's contiguous inputs in flight
  issue_base(S.in[0], a, tile * kAdjCells, t);
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  issue_gather(S.in[0], a, tile * kAdjCells, t);
  cp_async_commit();
  if (tile + (int)gridDim.x < ntiles) issue_base(S.in[1], a, (tile + gridDim.x) * kAdjCells, t);
  cp_async_commit();
  cp_async_wait<1>();
  __syncthreads();
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    AdjIn<R>& B = S.in[it & 1];
    AdjIn<R>& Bn = S.in[(it + 1) & 1];
    const int cell0 = tile * kAdjCells, next = tile + gridDim.x;
    // phase 1: forward reconstruction per (cell, component)
    if (t < m * kAdjCells) {
      const int lc = t % kAdjCells, c = t / kAdjCells;
      if (cell0 + lc < N) {
        R Wl[3], Vl[3], Yl[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) { Wl[j] = B.us[1 + j][lc][c]; Vl[j] = B.us[1 + j][lc][m + c]; Yl[j] = B.us[1 + j][lc][2 * m + c]; }
        R q[6];
        reconstruct_component<R>(TileGeo<R>{B.geo, lc}, B.us[0][lc][c], B.us[0][lc][m + c], B.us[0][lc][2 * m + c],
                                 Wl, Vl, Yl, P, q);
#pragma unroll
        for (int k = 0; k < 6; ++k) S.qs[c][k][lc] = q[k];
      }
    }
    // the next tile's neighbour records, now that its neighbour table is in
    cp_async_wait<0>();
    __syncthreads();
    if (next < ntiles) issue_gather(Bn, a, next * kAdjCells, t);
    cp_async_commit();
    // phase 2: per (cell, point)
    {
      const int lc = t % kAdjCells, qp = t / kAdjCells, i = cell0 + lc;
      if (i < N) {
        const int j = qp >> 1, g = qp & 1, jn = (j + 1) % 3;
        const int nb = B.nb[j][lc];
        const bool left = (B.nb[3][lc] >> (6 + j)) & 1;   // this cell owns the edge: canonical left side
        const R nx = B.geo[G_NRM + 2 * j][lc], ny = B.geo[G_NRM + 2 * j + 1][lc];
        const R el = B.geo[G_EL + j][lc];
        // (a) edge: reverse of the Lobatto sum of the LLF flux and of Eq. timeflux
        R Wb0[m], Wtb[m], Wttb[m];
        {
          R Wi[m], Wn[m];
#pragma unroll
          for (int c = 0; c < m; ++c) { Wi[c] = B.us[0][lc][c]; Wn[c] = B.us[1 + j][lc][c]; }
          const R* mine = &B.pb[lc][qp * rec];
          const R* theirs = nb >= 0 ? &B.pbn[qp][lc][0] : mine;
          const R aL = left ? spectral_radius_n<R, kEqEuler>(Wi, nx, ny, P) : spectral_radius_n<R, kEqEuler>(Wn, nx, ny, P);
          const R aR = left ? spectral_radius_n<R, kEqEuler>(Wn, nx, ny, P) : spectral_radius_n<R, kEqEuler>(Wi, nx, ny, P);
          const R alpha = aL > aR ? aL : aR;
          const R* pa = left ? mine : theirs;
          const R* pbp = left ? theirs : mine;
          // cotangents of this point's time-integrated flux and central value:
          // both cells of the edge use them (signs +- of the canonical normal)
          const R sgn = left ? R(1) : R(-1);
          R Feb[m], Shb[m];
#pragma unroll
          for (int c = 0; c < m; ++c) {
            const R wi = B.ub[0][lc][c], vi = B.ub[0][lc][m + c], yi = B.ub[0][lc][2 * m + c];
            Feb[c] = R(-0.5) * dtr * sgn * el * wi;
            Shb[c] = R(0.5) * sgn * el * (nx * vi + ny * yi);
          }
          if (nb >= 0) {
            const R eln = B.eln[j][lc];
#pragma unroll
            for (int c = 0; c < m; ++c) {
              const R wn = B.ub[1 + j][lc][c], vn = B.ub[1 + j][lc][m + c], yn = B.ub[1 + j][lc][2 * m + c];
              Feb[c] += R(-0.5) * dtr * (-sgn) * eln * wn;
              Shb[c] += R(0.5) * (-sgn) * eln * (nx * vn + ny * yn);
            }
          }
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
              WL[c] = pa[c] + tau[si] * pa[m + c] + hs * pa[2 * m + c];
              WR[c] = pbp[c] + tau[si] * pbp[m + c] + hs * pbp[2 * m + c];
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
          // this cell's share: its point's Taylor data, and its average through the viscosity
#pragma unroll
          for (int c = 0; c < m; ++c) {
            Wb0[c] = nb < 0 ? ab[0][c] + bb[0][c] : (left ? ab[0][c] : bb[0][c]);   // boundary: W^ext = W^int
            Wtb[c] = nb < 0 ? ab[1][c] + bb[1][c] : (left ? ab[1][c] : bb[1][c]);
            Wttb[c] = nb < 0 ? ab[2][c] + bb[2][c] : (left ? ab[2][c] : bb[2][c]);
          }
          R Wib[m] = {R(0), R(0), R(0), R(0)};
          const bool right_wins = !(aL > aR);
          const bool mine_wins = left ? !right_wins : right_wins;
          if (nb >= 0 && mine_wins) spectral_radius_n_euler_vjp(Wi, nx, ny, gam, alphab, Wib);
#pragma unroll
          for (int c = 0; c < m; ++c) S.wpart[c][qp][lc] = Wib[c];
        }
        // (b) reverse of the Lax-Wendroff procedure and of the point evaluation
        const R sg = g == 0 ? R(0.5) - R(0.28867513459481288225) : R(0.5) + R(0.28867513459481288225);
        const R xa = B.geo[G_VX + 2 * j][lc], ya = B.geo[G_VX + 2 * j + 1][lc];
        const R xi = xa + sg * (B.geo[G_VX + 2 * jn][lc] - xa);
        const R et = ya + sg * (B.geo[G_VX + 2 * jn + 1][lc] - ya);
        const R ih = B.geo[G_IH][lc], ih2 = ih * ih;
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
        SJet<R> Jb[4];
#pragma unroll
        for (int c = 0; c < m; ++c) { Jb[c] = jzero<SJet<R>>(); Jb[c].v = Wb0[c]; }
        lax_wendroff_euler_vjp(W, Wx, Wy, Wxx, Wxy, Wyy, gm1, Wtb, Wttb, Jb);
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
    // the tile (in place of the point records): slot 0 = the cell itself
    // (plus the identity term of Eq. flx and its viscosity shares), slot 1 + j
    // = its neighbour j
    R* cbt = &B.pb[0][0];
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
        for (int j = 0; j < 3; ++j) { Wl[j] = B.us[1 + j][lc][c]; Vl[j] = B.us[1 + j][lc][m + c]; Yl[j] = B.us[1 + j][lc][2 * m + c]; }
        R o0[3], ol[3][3];
        reconstruct_component_vjp<R>(TileGeo<R>{B.geo, lc}, B.us[0][lc][c], B.us[0][lc][m + c],
                                     B.us[0][lc][2 * m + c], Wl, Vl, Yl, P, qb, o0, ol);
#pragma unroll
        for (int j = 0; j < 3; ++j)
          if (B.nb[j][lc] < 0)
#pragma unroll
            for (int k = 0; k < 3; ++k) { o0[k] += ol[j][k]; ol[j][k] = R(0); }
        R w = B.ub[0][lc][c];
#pragma unroll
        for (int q = 0; q < 6; ++q) w += S.wpart[c][q][lc];
        o0[0] += w;
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
    __syncthreads();   // this buffer is free: stage the tile after next into it
    if (next + (int)gridDim.x < ntiles) issue_base(B, a, (next + gridDim.x) * kAdjCells, t);
    cp_async_commit();
    cp_async_wait<1>();   // the next tile's neighbour records (all but the newest group)
    __syncthreads();
  }
}

// ---------------------------------------------------------------- gather
template <typename R>
__global__ void __launch_bounds__(256) k_adj_gather(GeoView<R> G, const R* __restrict__ Cb, R* __restrict__ Ub0) {
  constexpr int m = kM;
  const int N = G.N;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = idx / (3 * m), o = idx % (3 * m);
  if (i >= N) return;
  R v = Cb[(size_t)i * 4 * 3 * m + o];
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
  const size_t smem = sizeof(AdjTile<R>);
  static_assert(sizeof(AdjTile<R>) <= 227 * 1024, "tile fits the shared memory of one block");
  static const int cap = [smem] {   // resident blocks (occupancy x SMs), once per process
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_adj_step<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_step<R>, kAdjThreads, smem);
    return sms * std::max(1, per_sm);
  }();
  const int ntiles = (a.N + kAdjCells - 1) / kAdjCells;
  const int grid = std::max(1, std::min(ntiles, cap));
  AdjPtrs p{a.rgeo, a.igeo, a.U, a.Pb, a.Ubar_next, a.N, a.ld};
  k_adj_step<R><<<grid, kAdjThreads, smem, st>>>(p, reinterpret_cast<R*>(a.Cb), a.P, a.dt, ntiles);
  GeoView<R> G{reinterpret_cast<const R*>(a.rgeo), a.igeo, a.N, a.ld};
  const long long total = (long long)a.N * 3 * kM;
  k_adj_gather<R><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(G, reinterpret_cast<const R*>(a.Cb),
                                                                  reinterpret_cast<R*>(a.Ubar));
}
}  // namespace

void launch_adjoint(int prec, const AdjointArgs& a, cudaStream_t st) {
  if (prec == 0) launch_adjoint_t<double>(a, st);
  else launch_adjoint_t<float>(a, st);
}

}  // namespace hw
