// Kernels of one ADER-HWENO time step on a triangular mesh.
//
//   k_recon : Steps 1-6 of Section 2.2 (Eqs. pxy, smoo1, nonlinearweight,
//             recon) per cell, then at its six edge Gauss points the
//             Lax-Wendroff procedure of Section 2.1; writes the Taylor data
//             (W, W_t, W_tt) of Eqs. tay / tayext to the edge-point buffer.
//   k_edge  : per cell (owner computes, no atomics), at the six Gauss points
//             of its edges the local Lax-Friedrichs flux at the time nodes
//             (Eqs. fx, flux; Gauss-Lobatto, or as an option two Gauss-Legendre
//             nodes) in a canonical orientation, so both
//             cells of an edge obtain bitwise-identical values; the update of
//             the cell average (Eq. flx) and of the derivative averages by
//             Green-Gauss from the central values at t_{n+1} (Eqs. derave2d2,
//             timeflux, taylor2dtime); the CFL step of the next step.  In
//             FP32 the update of the average is a compensated sum (one FP32
//             compensation word per cell and component).
//   k_edge_flux, k_edge_update: the same flux phase with every edge
//             evaluated once, by its left cell, into a per-point buffer, then
//             the update of every cell from its own or its neighbour's slots
//             (bit for bit k_edge's result; the FP64 default).
//   k_batch : many solves in one persistent cooperative launch (grid
//             barriers between the phases); k_batch_recon, k_batch_edge,
//             k_batch_finish: the same step as three launches.
//   k_fused : reconstruction and flux of a tile and its halo in one kernel
//             (option).
//   k_cfl, k_consv, k_scatter_state, k_gather_state: CFL step of a state,
//             FP64 conservation sums, host-order <-> internal-order copies.
//
// Layout: geometry and neighbour indices are planes of ld cells; the state
// (3m values per cell) and the edge-point data (6 points x 3 x m values per
// cell) are records, one contiguous record per cell, so that a neighbour's
// data are a few 16-byte vector loads.
//
// Both main kernels walk tiles of kCells consecutive (Hilbert-ordered) cells:
// k_recon with 2 threads per cell (the per-component and per-point tasks of a
// tile in whole passes; 6 per cell with the scale limiter), k_edge and the
// batched kernel with 6.  A block stages each tile's dense operands
// (geometry planes and neighbour indices by TMA tensor loads, the tile's own
// state or edge-point records by bulk copies) in shared memory,
// double-buffered: the copies of the block's next tile are in flight while the
// current tile is computed.  Neighbour records are gathered with ordinary
// vector loads (mostly L2 hits thanks to the Hilbert order).
#include <cuda.h>

#include <type_traits>

#include <cstddef>
#include <cstdint>

#include "device.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace hw {

namespace {

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double dinf() { return __longlong_as_double(0x7ff0000000000000ll); }

// Block-wide min of a positive double, then the last block to finish turns the
// grid-wide minimum into the next time step (threadfence reduction; no spin).
__device__ void finish_step(DevScalars* sc, double local_min, double dt_taken, bool advance) {
  __shared__ double smin[32];
  __shared__ bool am_last;
  double v = local_min;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) smin[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = smin[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = fmin(b, smin[w]);
    atomicMin(&sc->lam_min_bits, dbits(b));
    __threadfence();
    const unsigned ticket = atomicAdd(&sc->counter, 1u);
    am_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last && threadIdx.x == 0) {
    __threadfence();
    volatile DevScalars* vs = sc;
    const double mn = __longlong_as_double((long long)atomicAdd(&sc->lam_min_bits, 0ull));
    double t = vs->t;
    if (advance) {
      t += dt_taken;
      vs->t = t;
      vs->nsteps = vs->nsteps + 1;
    }
    double dtn = vs->cfl * mn;
    int done = 0;
    if (vs->has_T) {
      const double T = vs->T;
      if (t >= T * (1.0 - 1e-14)) done = 1;
      else if (t + dtn > T) dtn = T - t;
    }
    vs->dt = dtn;
    vs->done = done;
    atomicExch(&sc->lam_min_bits, dbits(dinf()));
    atomicExch(&sc->counter, 0u);
  }
}

// n contiguous values src -> dst with 16-byte vector accesses when possible
// (dst, src 16-byte aligned whenever n * sizeof(R) is a multiple of 16).
template <typename R, int n> __device__ __forceinline__ void copy_rec(R* dst, const R* src) {
  if constexpr ((n * sizeof(R)) % 16 == 0) {
    constexpr int v = n * sizeof(R) / 16;
#pragma unroll
    for (int k = 0; k < v; ++k) reinterpret_cast<float4*>(dst)[k] = reinterpret_cast<const float4*>(src)[k];
  } else {
#pragma unroll
    for (int k = 0; k < n; ++k) dst[k] = src[k];
  }
}

template <typename R> struct SmemGeo {
  const R* base;  // [plane][kCells]
  int lc;
  __device__ __forceinline__ R operator()(int p) const { return base[p * kCells + lc]; }
};

// Cells of tile `tile`: [cell0, cell0 + count), cell0 a multiple of kCells.
__device__ __forceinline__ void tile_range(const TileSet& ts, int N, int tile, int& cell0, int& count) {
  if (ts.table) {
    const int2 e = ts.table[tile];
    cell0 = e.x;
    count = e.y;
  } else {
    cell0 = tile * kCells;
    count = min(kCells, N - cell0);
  }
}

}  // namespace

// ---------------------------------------------------------------- tile contexts
// A phase walks the tiles a context exposes.  SingleCtx: one mesh, one time
// step for all cells.  BatchCtx (several meshes side by side): each tile
// belongs to one solve, with that solve's time step, buffer parity and status.
template <typename R> struct SingleCtx {
  TileSet ts;
  int N;
  const R* U;
  R* Un;
  double dt;
  DevScalars* sc;
  double local_min;   // CFL minimum of this thread over its tiles
  R* C;               // compensation of the cell averages (FP32 form) or nullptr
  __device__ __forceinline__ R* comp(int) const { return C; }
  __device__ __forceinline__ int ntiles() const { return ts.ntiles; }
  __device__ __forceinline__ bool active(int) const { return true; }
  __device__ __forceinline__ void range(int tile, int& c0, int& cnt) const { tile_range(ts, N, tile, c0, cnt); }
  __device__ __forceinline__ const R* uin(int) const { return U; }
  __device__ __forceinline__ R* uout(int) const { return Un; }
  __device__ __forceinline__ double dt_of(int) const { return dt; }
  __device__ __forceinline__ void flag(unsigned f) { atomicOr(&sc->flags, f); }
  __device__ __forceinline__ void bad_cell(int) { atomicOr(&sc->flags, 1u); }
  // called by the 32 threads of warp 0 after a tile; v = this thread's value
  __device__ __forceinline__ void tile_min(int, double v) { local_min = v < local_min ? v : local_min; }
};

template <typename R> struct BatchCtx {
  const int4* tiles;   // (first cell, count, solve, 0)
  int nt;
  R* C;                // FP32: compensation words of the cell averages (compensated updates), or nullptr
  __device__ __forceinline__ R* comp(int) const { return C; }
  BatchSolve* bs;
  BatchCtl* ctl;
  R* U0;
  R* U1;
  __device__ __forceinline__ int solve(int tile) const { return tiles[tile].z; }
  __device__ __forceinline__ int ntiles() const { return nt; }
  __device__ __forceinline__ bool active(int tile) const {
    return *(volatile const int*)&bs[solve(tile)].done == 0;
  }
  __device__ __forceinline__ void range(int tile, int& c0, int& cnt) const {
    const int4 e = tiles[tile];
    c0 = e.x;
    cnt = e.y;
  }
  __device__ __forceinline__ bool odd(int tile) const {
    return (*(volatile const long long*)&bs[solve(tile)].nsteps) & 1;
  }
  __device__ __forceinline__ const R* uin(int tile) const { return odd(tile) ? U1 : U0; }
  __device__ __forceinline__ R* uout(int tile) const { return odd(tile) ? U0 : U1; }
  __device__ __forceinline__ double dt_of(int tile) const { return *(volatile const double*)&bs[solve(tile)].dt; }
  __device__ __forceinline__ void flag(unsigned f) { atomicOr(&ctl->flags, f); }
  __device__ __forceinline__ void bad_cell(int tile) {
    atomicOr(&ctl->flags, 1u);
    atomicExch(&bs[solve(tile)].failed, 1);
  }
  __device__ __forceinline__ void tile_min(int tile, double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v < dinf()) atomicMin(&bs[solve(tile)].lam_min_bits, dbits(v));
  }
};

// First tile at or after `tile` (stride gridDim.x) that the context keeps.
template <typename Ctx> __device__ __forceinline__ int next_active(const Ctx& ctx, int tile) {
  while (tile < ctx.ntiles() && !ctx.active(tile)) tile += gridDim.x;
  return tile;
}

// ---------------------------------------------------------------- reconstruction
template <typename R, int EQ> struct ReconStage {
  static constexpr int m = EqTraits<EQ>::m;
  R geo[kReconPlanes][kCells];   // TMA tensor box: planes x cells
  int32_t idx[4][kCells];        // TMA tensor box
  R u[kCells][3 * m];            // bulk copy of the tile's state records
};

template <typename R, int EQ> constexpr size_t recon_smem_bytes() {
  return 2 * sizeof(ReconStage<R, EQ>) + sizeof(R) * (EqTraits<EQ>::m + 1) * 6 * kCells + 2 * sizeof(uint64_t) + 128;
}

// Shared-memory carve-up common to both phases: stages at the start (128-byte
// aligned), then phase scratch; the two mbarriers live at a fixed offset set by
// the caller.
__device__ __forceinline__ unsigned char* smem_base(unsigned char* raw) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 127) & ~uintptr_t(127));
}

// Cells of a reconstruction block staged in shared memory (TMA boxes of a
// contiguous 32-cell tile): geometry planes, neighbour indices, state records.
template <typename R, int EQ> struct StagedCells {
  static constexpr int m = EqTraits<EQ>::m;
  const ReconStage<R, EQ>* S;
  __device__ __forceinline__ R geo(int p, int lc) const { return S->geo[p][lc]; }
  __device__ __forceinline__ const R* own(int lc) const { return S->u[lc]; }
  __device__ __forceinline__ int nbr(int j, int lc) const { return S->idx[j][lc]; }
  __device__ __forceinline__ int nbe(int lc) const { return S->idx[3][lc]; }
  __device__ __forceinline__ SmemGeo<R> geo_of(int lc) const { return SmemGeo<R>{&S->geo[0][0], lc}; }
};

// Cells of a reconstruction block read straight from global memory: cells[lc]
// is the internal index of the block's cell lc (entries beyond the block's
// count hold a valid cell).  Used for the halo of a fused tile.
template <typename R> struct GlobalGeo {
  const R* __restrict__ rg;
  int ld, i;
  __device__ __forceinline__ R operator()(int p) const { return __ldg(rg + (size_t)p * ld + i); }
};
template <typename R, int EQ> struct GlobalCells {
  static constexpr int m = EqTraits<EQ>::m;
  const R* __restrict__ rg;
  const int32_t* __restrict__ ig;
  const R* __restrict__ U;
  const int* cells;
  int ld;
  __device__ __forceinline__ R geo(int p, int lc) const { return __ldg(rg + (size_t)p * ld + cells[lc]); }
  __device__ __forceinline__ const R* own(int lc) const { return U + (size_t)cells[lc] * 3 * m; }
  __device__ __forceinline__ int nbr(int j, int lc) const { return __ldg(ig + (size_t)(I_NBR + j) * ld + cells[lc]); }
  __device__ __forceinline__ int nbe(int lc) const { return __ldg(ig + (size_t)I_NBE * ld + cells[lc]); }
  __device__ __forceinline__ GlobalGeo<R> geo_of(int lc) const { return GlobalGeo<R>{rg, ld, cells[lc]}; }
};

// Components c0 .. c0 + NC - 1 of the three fields (Wbar, Vbar, Ybar) of a
// state record with m components; a pair (c0 even, the record 16-byte aligned)
// in one 8- or 16-byte load per field.
template <typename R, int NC>
__device__ __forceinline__ void load_fields(const R* rec, int m, int c0, R* w, R* v, R* y) {
  if constexpr (NC == 2) {
    using V2 = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const V2 a = *reinterpret_cast<const V2*>(rec + c0);
    const V2 b = *reinterpret_cast<const V2*>(rec + m + c0);
    const V2 c = *reinterpret_cast<const V2*>(rec + 2 * m + c0);
    w[0] = a.x; w[1] = a.y; v[0] = b.x; v[1] = b.y; y[0] = c.x; y[1] = c.y;
  } else {
#pragma unroll
    for (int n = 0; n < NC; ++n) { w[n] = rec[c0 + n]; v[n] = rec[m + c0 + n]; y[n] = rec[2 * m + c0 + n]; }
  }
}

// Reconstruction (Steps 1-6) and the Lax-Wendroff procedure at the six edge
// Gauss points of up to kCells cells.  NT: threads of the block; phase A runs
// the (cell, component) tasks and phase B the (cell, point) tasks in passes of
// NT; the limiter's phase B synchronises per point and needs one thread per
// (cell, point).  out(lc, qp, rec) stores the Taylor record (W, W_t, W_tt) of
// point qp of cell lc.  U: the state (neighbour records); dtr: the time step.
template <typename R, int EQ, bool LIM, int NT, typename Src, typename Out>
__device__ __forceinline__ void recon_lw_block(const Src& src, int count, const R* __restrict__ U, R dtr,
                                               const EqParams& P, R (*qs)[6][kCells], R (*lim)[kCells], Out out) {
  constexpr int m = EqTraits<EQ>::m;
  static_assert(!LIM || NT == 6 * kCells, "the limiter path takes one thread per (cell, point)");
  const int t = threadIdx.x;
  // phase A: NC components of a cell per task (two with 2 threads per cell, so
  // that the cell's geometry planes are read once for both)
  constexpr int NC = (NT == 2 * kCells && m % 2 == 0) ? 2 : 1;
  for (int task = t; task < (m / NC) * kCells; task += NT) {
    const int lc = task % kCells, c0 = (task / kCells) * NC;
    if (lc < count) {
      R W0[NC], V0[NC], Y0[NC], Wl[NC][3], Vl[NC][3], Yl[NC][3];
      const R* own = src.own(lc);
      load_fields<R, NC>(own, m, c0, W0, V0, Y0);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int nb = src.nbr(j, lc);
        if (nb >= 0) {
          R w[NC], v[NC], y[NC];
          load_fields<R, NC>(U + (size_t)nb * 3 * m, m, c0, w, v, y);
#pragma unroll
          for (int n = 0; n < NC; ++n) { Wl[n][j] = w[n]; Vl[n][j] = v[n]; Yl[n][j] = y[n]; }
        } else {
          // boundary ghost: outward unit normal of edge j from the scaled vertices
          const int jn = (j + 1) % 3;
          const R dx = src.geo(G_VX + 2 * jn, lc) - src.geo(G_VX + 2 * j, lc);
          const R dy = src.geo(G_VX + 2 * jn + 1, lc) - src.geo(G_VX + 2 * j + 1, lc);
          const R il = R(1) / sqrt(dx * dx + dy * dy);
#pragma unroll
          for (int n = 0; n < NC; ++n)
            ghost_component<R, EQ>(ghost_type(src.nbe(lc), j), own, dy * il, -dx * il, c0 + n, P, Wl[n][j],
                                   Vl[n][j], Yl[n][j]);
        }
      }
      R q[NC][6];
      reconstruct_components<R, NC>(src.geo_of(lc), W0, V0, Y0, Wl, Vl, Yl, P, q);
#pragma unroll
      for (int n = 0; n < NC; ++n)
#pragma unroll
        for (int k = 0; k < 6; ++k) qs[c0 + n][k][lc] = q[n][k];
    }
  }
  __syncthreads();
  for (int task = t; task < 6 * kCells; task += NT) {
    const int lc = task % kCells, qp = task / kCells;
    const bool act = lc < count;
    R W[m], Wx[m], Wy[m], Wxx[m], Wxy[m], Wyy[m], Wt[m], Wtt[m];
    if (act) {
      const int j = qp >> 1, g = qp & 1, jn = (j + 1) % 3;
      const R sg = g == 0 ? R(0.5) - R(0.28867513459481288225) : R(0.5) + R(0.28867513459481288225);
      const R xj = src.geo(G_VX + 2 * j, lc), yj = src.geo(G_VX + 2 * j + 1, lc);
      const R xi = xj + sg * (src.geo(G_VX + 2 * jn, lc) - xj);
      const R et = yj + sg * (src.geo(G_VX + 2 * jn + 1, lc) - yj);
      const R ih = src.geo(G_IH, lc), ih2 = ih * ih;
#pragma unroll
      for (int c = 0; c < m; ++c) {
        const R q0 = qs[c][0][lc], q1 = qs[c][1][lc], q2 = qs[c][2][lc];
        const R q3 = qs[c][3][lc], q4 = qs[c][4][lc], q5 = qs[c][5][lc];
        W[c] = q0 + xi * (q1 + q3 * xi + q4 * et) + et * (q2 + q5 * et);
        Wx[c] = (q1 + R(2) * q3 * xi + q4 * et) * ih;
        Wy[c] = (q2 + q4 * xi + R(2) * q5 * et) * ih;
        Wxx[c] = R(2) * q3 * ih2; Wxy[c] = q4 * ih2; Wyy[c] = R(2) * q5 * ih2;
      }
    }
    if constexpr (EQ == kEqEuler && LIM) {
      // scale limiter: spatial scaling over the six Gauss points, then the
      // Lax-Wendroff data, then scaling of the space-time Taylor data over
      // the points and the three time nodes
      const R gam = EqC<R>::gam(P);
      R Wb[4] = {R(0), R(0), R(0), R(0)};
      if (act) {
        const R* own = src.own(lc);
#pragma unroll
        for (int c = 0; c < 4; ++c) Wb[c] = own[c];
      }
      const R pb0 = act ? pressure_of(gam, Wb) : R(0);
      const bool ok = act && Wb[0] > R(0) && pb0 > R(0);
      const R eps = ok ? positivity_floor(Wb[0], pb0) : R(0);
      if (act) lim[qp][lc] = W[0];
      __syncthreads();
      R th1 = R(1), th2 = R(1);
      if (ok) {
        R rmin = lim[0][lc];
#pragma unroll
        for (int k = 1; k < 6; ++k) rmin = lim[k][lc] < rmin ? lim[k][lc] : rmin;
        if (rmin < eps) th1 = (Wb[0] - eps) / (Wb[0] - rmin);
      }
      __syncthreads();
      R f = R(1);
      if (ok) {
        R w[4] = {Wb[0] + th1 * (W[0] - Wb[0]), W[1], W[2], W[3]};
        if (pressure_of(gam, w) < eps) {
          R d[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) d[c] = w[c] - Wb[c];
          f = pressure_root(gam, Wb, d, eps);
        }
      }
      if (act) lim[qp][lc] = f;
      __syncthreads();
      if (ok) {
#pragma unroll
        for (int k = 0; k < 6; ++k) th2 = lim[k][lc] < th2 ? lim[k][lc] : th2;
      }
      __syncthreads();
      if (ok && (th1 != R(1) || th2 != R(1))) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const R th = c == 0 ? th1 * th2 : th2;
          W[c] = Wb[c] + th * (W[c] - Wb[c]);
          Wx[c] *= th; Wy[c] *= th; Wxx[c] *= th; Wxy[c] *= th; Wyy[c] *= th;
        }
      }
      if (act) lax_wendroff<R, EQ>(W, Wx, Wy, Wxx, Wxy, Wyy, P, Wt, Wtt);
      R ft = R(1);
      if (ok) {
        const R tau[3] = {R(0), R(0.5) * dtr, dtr};
#pragma unroll
        for (int si = 0; si < 3; ++si) {
          R w[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) w[c] = W[c] + Wt[c] * tau[si] + Wtt[c] * (R(0.5) * tau[si] * tau[si]);
          const R fs = admissible_fraction(gam, Wb, w, eps);
          ft = fs < ft ? fs : ft;
        }
      }
      if (act) lim[qp][lc] = ft;
      __syncthreads();
      R tht = R(1);
      if (ok) {
#pragma unroll
        for (int k = 0; k < 6; ++k) tht = lim[k][lc] < tht ? lim[k][lc] : tht;
      }
      if (ok && tht != R(1)) {
#pragma unroll
        for (int c = 0; c < 4; ++c) { W[c] = Wb[c] + tht * (W[c] - Wb[c]); Wt[c] *= tht; Wtt[c] *= tht; }
      }
    } else if (act) {
      lax_wendroff<R, EQ>(W, Wx, Wy, Wxx, Wxy, Wyy, P, Wt, Wtt);
    }
    if (act) {
      R rec[3 * m];
#pragma unroll
      for (int c = 0; c < m; ++c) { rec[c] = W[c]; rec[m + c] = Wt[c]; rec[2 * m + c] = Wtt[c]; }
      out(lc, qp, rec);
    }
  }
  __syncthreads();
}

// Reconstruction + Lax-Wendroff over the context's tiles (double-buffered TMA
// staging), writing the edge-point records to Pb.  bar: two initialised
// mbarriers, ph: their phase bits (kept across calls).  Returns false if a
// bounded wait gave up (flag 2 raised).
template <typename R, int EQ, bool LIM, int NT, typename Ctx>
__device__ bool recon_phase(Ctx& ctx, const CUtensorMap* mGeo, const CUtensorMap* mIdx, const EqParams& P,
                            R* __restrict__ Pb, unsigned char* base, uint64_t* bar, unsigned* ph) {
  constexpr int m = EqTraits<EQ>::m;
  using Stage = ReconStage<R, EQ>;
  Stage* st = reinterpret_cast<Stage*>(base);
  R (*qs)[6][kCells] = reinterpret_cast<R (*)[6][kCells]>(base + 2 * sizeof(Stage));
  R (*lim)[kCells] = reinterpret_cast<R (*)[kCells]>(base + 2 * sizeof(Stage) + sizeof(R) * m * 6 * kCells);
  const int ntiles = ctx.ntiles();
  const int t = threadIdx.x;
  constexpr unsigned kBytes = sizeof(Stage);
  auto issue = [&](int s, int tile) {
    int c0, cnt;
    ctx.range(tile, c0, cnt);
    mbar_arrive_expect_tx(&bar[s], kBytes);
    tma_load_2d(&st[s].geo[0][0], mGeo, c0, 0, &bar[s]);
    tma_load_2d(&st[s].idx[0][0], mIdx, c0, 0, &bar[s]);
    bulk_load(&st[s].u[0][0], ctx.uin(tile) + (size_t)c0 * 3 * m, kCells * 3 * m * sizeof(R), &bar[s]);
  };
  int tile = next_active(ctx, blockIdx.x);
  if (t == 0 && tile < ntiles) {
    fence_proxy_async();
    issue(0, tile);
  }
  int s = 0;
  for (; tile < ntiles; s ^= 1) {
    const int next = next_active(ctx, tile + gridDim.x);
    if (t == 0 && next < ntiles) {
      fence_proxy_async();
      issue(s ^ 1, next);
    }
    const bool ok = mbar_wait(&bar[s], ph[s]);
    ph[s] ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        ctx.flag(2u);
        if (next < ntiles && mbar_wait(&bar[s ^ 1], ph[s ^ 1])) ph[s ^ 1] ^= 1u;   // drain the copy in flight
      }
      return false;
    }
    int cell0, count;
    ctx.range(tile, cell0, count);
    const R dtr = R(ctx.dt_of(tile));   // time nodes of the limiter
    recon_lw_block<R, EQ, LIM, NT>(StagedCells<R, EQ>{&st[s]}, count, ctx.uin(tile), dtr, P, qs, lim,
                                   [&](int lc, int qp, const R* rec) {
                                     copy_rec<R, 3 * m>(Pb + (size_t)(cell0 + lc) * 18 * m + qp * 3 * m, rec);
                                   });
    tile = next;
  }
  return true;
}

// ---------------------------------------------------------------- flux + update
template <typename R, int EQ> struct EdgeStage {
  static constexpr int m = EqTraits<EQ>::m;
  R geo[kEdgePlanes][kCells];    // TMA tensor box: planes x cells
  int32_t idx[4][kCells];        // TMA tensor box
  R lg[kLimPlanes][kCells];      // TMA tensor box: flux-blending geometry (scale limiter only)
  R pb[kCells][18 * m];          // bulk copy of the tile's edge-point records
  R u[kCells][3 * m];            // bulk copy of the tile's state records
  R cc[kCells][m];               // bulk copy of the compensation words (FP32 form; else unused)
};

static_assert(sizeof(EdgeStage<float, 2>) % 128 == 0 && sizeof(EdgeStage<double, 2>) % 128 == 0 &&
                  sizeof(EdgeStage<float, 0>) % 128 == 0 && sizeof(EdgeStage<double, 0>) % 128 == 0,
              "every stage starts 128-byte aligned (TMA destination)");

template <typename R, int EQ> constexpr size_t edge_smem_bytes() {
  return 2 * sizeof(EdgeStage<R, EQ>) + sizeof(R) * 3 * EqTraits<EQ>::m * 6 * kCells +
         sizeof(R) * EqTraits<EQ>::m * kCells + 2 * sizeof(uint64_t) + 128;
}

// Flux at the time nodes, cell-average and Green-Gauss update, CFL candidates
// over the context's tiles.  GL = false: the three Gauss-Lobatto nodes, the
// last of which (t_{n+1}) also gives the central values of Eq. timeflux; GL =
// true: two Gauss-Legendre nodes and a separate Taylor evaluation at t_{n+1}.
// LIM (Euler with the scale limiter): each edge flux is blended with the
// first-order LLF flux of the two cell averages so that the new averages stay
// admissible (see blend_theta).  Returns false if a bounded wait gave up.
constexpr double kGaussNode = 0.28867513459481288225;   // sqrt(3) / 6

// Positivity-preserving flux blending (Hu, Adams and Shu 2013), Euler, with
// the scale limiter.  The limiter keeps the point values admissible, but a
// one-step update built from time-Taylor values is not a convex combination of
// them, so a new cell average can still lose positivity.  Each average is
//   Wbar^{n+1} = sum_e (|e| / P) Phi_e,  Phi_e = Wbar - (dt P / |K|) (Fhat_e - F(Wbar) . n_e)
// (P the perimeter; the |e| n_e of a cell sum to zero); with Fhat = FL + theta
// (FH - FL), FL the first-order LLF flux of the two averages (same alpha),
// theta is the largest value in [0, 1] that keeps Phi_e admissible on both
// sides.  Inputs in the edge's canonical orientation (n outward of the left
// cell): averages WL, WR, their F.n HL, HR, the blended fluxes' end points FL,
// FH, and lamL = dt P_L / |K_L|, lamR likewise (lamR < 0 ignored: boundary).
template <typename R>
__device__ __forceinline__ R blend_theta(R gam, const R WL[4], const R WR[4], const R HL[4], const R HR[4],
                                         const R FL[4], const R FH[4], R lamL, R lamR) {
  R theta = R(1);
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    const R* Wk = side == 0 ? WL : WR;
    const R* Hk = side == 0 ? HL : HR;
    const R lam = side == 0 ? lamL : -lamR;   // the normal points into the right cell
    if (side == 1 && lamR < R(0)) break;
    const R pk = pressure_of(gam, Wk);
    if (!(Wk[0] > R(0)) || !(pk > R(0))) continue;   // the average itself is not admissible
    const R eps = positivity_floor(Wk[0], pk);
    R phi0[4], phi1[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      phi0[c] = Wk[c] - lam * (FL[c] - Hk[c]);
      phi1[c] = Wk[c] - lam * (FH[c] - Hk[c]);
    }
    R th = R(0);
    if (phi0[0] >= eps && pressure_of(gam, phi0) >= eps) th = admissible_fraction(gam, phi0, phi1, eps);
    theta = th < theta ? th : theta;
  }
  return theta;
}

// LLF viscosity of an edge: the larger spectral radius of the flux Jacobian
// along n at the two cells' averages (canonical left / right).
template <typename R, int EQ>
__device__ __forceinline__ R edge_alpha(const R* Wi, const R* Wn, bool left, R nx, R ny, const EqParams& P) {
  R aL, aR;
  if (left) { aL = spectral_radius_n<R, EQ>(Wi, nx, ny, P); aR = spectral_radius_n<R, EQ>(Wn, nx, ny, P); }
  else      { aL = spectral_radius_n<R, EQ>(Wn, nx, ny, P); aR = spectral_radius_n<R, EQ>(Wi, nx, ny, P); }
  return aL > aR ? aL : aR;
}

// One Gauss point of an edge: the LLF flux integrated over the time nodes
// (Eq. flux; n outward of the edge's left cell) and the central value at
// t_{n+1} (Eq. timeflux), from the Taylor records (W, W_t, W_tt) of the two
// sides at that point.  mine: the calling cell's record; theirs: the other
// cell's, or nullptr on a boundary edge, whose ghost record follows from
// gtype (inflow: the imposed state; wall: the mirrored interior record;
// transmissive: the interior record).  left: the calling cell is the edge's
// left cell.
template <typename R, int EQ, bool GL>
__device__ __forceinline__ void edge_point_flux(const R* mine_src, const R* theirs_src, int gtype, bool left, R nx,
                                                R ny, R alpha, R dtr, const EqParams& P, R* Fe, R* Sh) {
  constexpr int m = EqTraits<EQ>::m;
  R mine[3 * m], theirs[3 * m];
  copy_rec<R, 3 * m>(mine, mine_src);
  if (theirs_src) {
    copy_rec<R, 3 * m>(theirs, theirs_src);
  } else if (gtype == kGhostInflow) {   // the imposed state, constant in time
#pragma unroll
    for (int c = 0; c < m; ++c) { theirs[c] = EqC<R>::win(P, c); theirs[m + c] = R(0); theirs[2 * m + c] = R(0); }
  } else if (EQ == kEqEuler && gtype == kGhostWall) {   // the mirrored interior Taylor data
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int c = 0; c < m; ++c) theirs[k * m + c] = mirror_c(nx, ny, mine + k * m, c);
  } else {
    copy_rec<R, 3 * m>(theirs, mine);   // transmissive: W^ext = W^int
  }
  R a0[m], a1[m], a2[m], b0[m], b1[m], b2[m];
#pragma unroll
  for (int c = 0; c < m; ++c) {
    a0[c] = left ? mine[c] : theirs[c];
    a1[c] = left ? mine[m + c] : theirs[m + c];
    a2[c] = left ? mine[2 * m + c] : theirs[2 * m + c];
    b0[c] = left ? theirs[c] : mine[c];
    b1[c] = left ? theirs[m + c] : mine[m + c];
    b2[c] = left ? theirs[2 * m + c] : mine[2 * m + c];
  }
  constexpr int ns = GL ? 2 : 3;   // time nodes
  R tau[3], wts[3];
  if constexpr (GL) {
    tau[0] = dtr * R(0.5 - kGaussNode); tau[1] = dtr * R(0.5 + kGaussNode);
    wts[0] = R(0.5); wts[1] = R(0.5);
  } else {
    tau[0] = R(0); tau[1] = R(0.5) * dtr; tau[2] = dtr;
    wts[0] = R(1.0 / 6.0); wts[1] = R(4.0 / 6.0); wts[2] = R(1.0 / 6.0);
  }
#pragma unroll
  for (int c = 0; c < m; ++c) Fe[c] = R(0);
#pragma unroll
  for (int si = 0; si < ns; ++si) {
    R WL[m], WR[m], HL[m], HR[m];
    const R hs = R(0.5) * tau[si] * tau[si];
#pragma unroll
    for (int c = 0; c < m; ++c) {
      WL[c] = a0[c] + tau[si] * a1[c] + hs * a2[c];
      WR[c] = b0[c] + tau[si] * b1[c] + hs * b2[c];
    }
    flux_n<R, EQ>(WL, nx, ny, P, HL);
    flux_n<R, EQ>(WR, nx, ny, P, HR);
#pragma unroll
    for (int c = 0; c < m; ++c) Fe[c] += wts[si] * (R(0.5) * (HR[c] + HL[c] - alpha * (WR[c] - WL[c])));
    if (!GL && si == 2) {
#pragma unroll
      for (int c = 0; c < m; ++c) Sh[c] = R(0.5) * (WL[c] + WR[c]);   // Eq. timeflux
    }
  }
  if constexpr (GL) {   // Eq. timeflux from its own Taylor evaluation at t_{n+1}
    const R hs = R(0.5) * dtr * dtr;
#pragma unroll
    for (int c = 0; c < m; ++c)
      Sh[c] = R(0.5) * ((a0[c] + dtr * a1[c] + hs * a2[c]) + (b0[c] + dtr * b1[c] + hs * b2[c]));
  }
}

// Flux blending of one Gauss point (Euler, scale limiter): FH is the mean of
// the edge's two Gauss-point fluxes, pown / pnb the perimeter over area of
// the calling cell and of the other one (has_nb false: a boundary edge).
template <typename R, int EQ>
__device__ __forceinline__ void blend_point(const R* Wi, const R* Wn, bool left, bool has_nb, R nx, R ny, R alpha,
                                            const R* FH, R pown, R pnb, R dtr, const EqParams& P, R* Fe) {
  R FL[4], WL[4], WR[4], HL[4], HR[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    WL[c] = left ? Wi[c] : Wn[c];
    WR[c] = left ? Wn[c] : Wi[c];
  }
  flux_n<R, EQ>(WL, nx, ny, P, HL);
  flux_n<R, EQ>(WR, nx, ny, P, HR);
#pragma unroll
  for (int c = 0; c < 4; ++c) FL[c] = R(0.5) * (HL[c] + HR[c] - alpha * (WR[c] - WL[c]));
  const R lamL = dtr * (left ? pown : pnb);
  const R lamR = has_nb ? dtr * (left ? pnb : pown) : R(-1);
  const R theta = blend_theta(EqC<R>::gam(P), WL, WR, HL, HR, FL, FH, lamL, lamR);
  if (theta < R(1)) {
#pragma unroll
    for (int c = 0; c < 4; ++c) Fe[c] = FL[c] + theta * (Fe[c] - FL[c]);
  }
}

// Green-Gauss and flux shares of one (cell, point) into part: Gauss weight
// 1/2 and the cell's outward normal (+-n).  In FP32 the Green-Gauss terms are
// taken relative to the cell's own average: the cell's |e| n sum to zero, so
// the result is the same, while the terms shrink from |W| / h to |grad W| and
// their rounding with them.
template <typename R, int m>
__device__ __forceinline__ void point_shares(bool left, R el, R nx, R ny, const R* Fe, const R* Sh, const R* Wi,
                                             int qp, int lc, R (*part)[m][6][kCells]) {
  const R sgn = left ? R(0.5) * el : R(-0.5) * el;
#pragma unroll
  for (int c = 0; c < m; ++c) {
    const R sh = sizeof(R) == 4 ? Sh[c] - Wi[c] : Sh[c];
    part[0][c][qp][lc] = sgn * Fe[c];
    part[1][c][qp][lc] = sgn * nx * sh;
    part[2][c][qp][lc] = sgn * ny * sh;
  }
}

// After the shares of a tile are in part (and a barrier): the six-way sums,
// the cell-average update (compensated in FP32) and the new derivative
// averages into Un, the CFL candidates of the new averages; ends with a
// barrier.  S: the tile's staged state (u), compensation words (cc) and flux
// geometry (geo, planes G_NRM ..).
template <typename R, int EQ, typename Ctx, typename FS>
__device__ __forceinline__ void sum_update_cfl(Ctx& ctx, int tile, int cell0, int count, const FS& S,
                                               R* __restrict__ Un, R dtr, const EqParams& P,
                                               R (*part)[EqTraits<EQ>::m][6][kCells], R (*wn)[kCells]) {
  constexpr int m = EqTraits<EQ>::m;
  const int t = threadIdx.x;
  // sums of the six shares: thread (cell, output) for the 3m outputs
  for (int k = t; k < 3 * m * kCells; k += kThreads) {
    const int lc = k % kCells, o = k / kCells;   // o = kind * m + c
    if (lc < count) {
      const int kind = o / m, c = o % m;
      R r = R(0);
#pragma unroll
      for (int qp = 0; qp < 6; ++qp) r += part[kind][c][qp][lc];
      R v = r;
      if (kind == 0) {
        R* Cp = ctx.comp(tile);
        if (Cp) {
          // compensated summation of the updates: the rounding error of each
          // new average is carried into the next update, so that the FP32
          // averages do not accumulate one rounding per step
          const R y = -dtr * r - S.cc[lc][c];
          const R w = S.u[lc][c];
          v = w + y;
          Cp[(size_t)(cell0 + lc) * m + c] = (v - w) - y;
        } else {
          v = S.u[lc][c] - dtr * r;
        }
        wn[c][lc] = v;
      }
      Un[(size_t)(cell0 + lc) * 3 * m + o] = v;
    }
  }
  __syncthreads();
  if (t < kCells) {
    double v = dinf();
    if (t < count) {
      R Wnew[m];
#pragma unroll
      for (int c = 0; c < m; ++c) Wnew[c] = wn[c][t];
      if (!physical<R, EQ>(Wnew, P)) ctx.bad_cell(tile);
      const R lam = spectral_radius_all<R, EQ>(Wnew, P);
      if (lam > R(0)) {
        const double r = (double)(S.geo[G_INR - G_NRM][t] / lam);
        if (r >= 0) v = r;
      }
    }
    ctx.tile_min(tile, v);
  }
  __syncthreads();
}

// Flux at the time nodes, cell-average and Green-Gauss update and CFL
// candidates of up to kCells cells whose flux geometry, indices, state and
// compensation words are staged in S (members geo, idx, lg, u, cc).  recs
// gives the Taylor records: recs.mine(lc, q) of the cell's own point q,
// recs.theirs(lc, j, nb, qn) the record of point qn of the neighbour nb
// across edge j.  part, wn: shared scratch.
template <typename R, int EQ, bool GL, bool LIM, typename Ctx, typename FS, typename Recs>
__device__ __forceinline__ void flux_update_block(Ctx& ctx, int tile, int cell0, int count, const FS& S,
                                                  const Recs& recs, const R* __restrict__ U, R* __restrict__ Un,
                                                  R dtr, const EqParams& P, R (*part)[EqTraits<EQ>::m][6][kCells],
                                                  R (*wn)[kCells]) {
  constexpr int m = EqTraits<EQ>::m;
  const int t = threadIdx.x;
  {
    const int lc = t % kCells, qp = t / kCells;
    const bool act = lc < count;
    const int j = qp >> 1, gm = qp & 1;
    R Wi[m], Wn[m], Fe[m], Sh[m];
    R nx = R(0), ny = R(0), el = R(0), alpha = R(0);
    bool left = true;
    int nb = -1;
    if (act) {
      nb = S.idx[j][lc];
      const int je = (S.idx[3][lc] >> (2 * j)) & 3;
      left = (S.idx[3][lc] >> (6 + j)) & 1;   // this cell owns the edge: canonical left side
      nx = S.geo[2 * j][lc]; ny = S.geo[2 * j + 1][lc];
      el = S.geo[6 + j][lc];
      copy_rec<R, m>(Wi, S.u[lc]);
      const int gtype = nb >= 0 ? kGhostTransmissive : ghost_type(S.idx[3][lc], j);
      if (nb >= 0) {
        copy_rec<R, m>(Wn, U + (size_t)nb * 3 * m);
      } else {
        // the ghost's average; a boundary edge belongs to its cell, so n is outward
#pragma unroll
        for (int c = 0; c < m; ++c) {
          R v, yv;
          ghost_component<R, EQ>(gtype, S.u[lc], nx, ny, c, P, Wn[c], v, yv);
        }
      }
      alpha = edge_alpha<R, EQ>(Wi, Wn, left, nx, ny, P);
      // this cell's Taylor data at its point (j, gm); the neighbour's at the
      // same physical point, its point (je, 1 - gm); canonical left / right
      const int qm = 2 * j + gm, qn = 2 * je + (1 - gm);
      edge_point_flux<R, EQ, GL>(recs.mine(lc, qm), nb >= 0 ? recs.theirs(lc, j, nb, qn) : nullptr, gtype, left, nx,
                                 ny, alpha, dtr, P, Fe, Sh);
    }
    if constexpr (LIM) {
      // flux blending: the edge's high-order flux is the mean of its two
      // Gauss points' (the same sum on both sides of the edge)
      if (act) {
#pragma unroll
        for (int c = 0; c < m; ++c) part[0][c][qp][lc] = Fe[c];
      }
      __syncthreads();
      if (act) {
        R FH[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) FH[c] = R(0.5) * (part[0][c][2 * j][lc] + part[0][c][2 * j + 1][lc]);
        blend_point<R, EQ>(Wi, Wn, left, nb >= 0, nx, ny, alpha, FH, S.lg[0][lc], S.lg[1 + j][lc], dtr, P, Fe);
      }
      __syncthreads();
    }
    if (act) point_shares<R, m>(left, el, nx, ny, Fe, Sh, Wi, qp, lc, part);
  }
  __syncthreads();
  sum_update_cfl<R, EQ>(ctx, tile, cell0, count, S, Un, dtr, P, part, wn);
}

// Edge-point records of a tile staged in an EdgeStage (own) and in global
// memory (neighbours).
template <typename R, int EQ> struct StagedRecs {
  static constexpr int m = EqTraits<EQ>::m;
  const EdgeStage<R, EQ>* S;
  const R* __restrict__ Pb;
  __device__ __forceinline__ const R* mine(int lc, int q) const { return &S->pb[lc][q * 3 * m]; }
  __device__ __forceinline__ const R* theirs(int, int, int nb, int qn) const {
    return Pb + (size_t)nb * 18 * m + qn * 3 * m;
  }
};

template <typename R, int EQ, bool GL, bool LIM, typename Ctx>
__device__ bool edge_phase(Ctx& ctx, const CUtensorMap* mEgeo, const CUtensorMap* mIdx, const CUtensorMap* mLgeo,
                           const EqParams& P, const R* __restrict__ Pb, unsigned char* base, uint64_t* bar,
                           unsigned* ph) {
  constexpr int m = EqTraits<EQ>::m;
  static_assert(!LIM || EQ == kEqEuler, "flux blending is for the Euler equations");
  using Stage = EdgeStage<R, EQ>;
  static_assert(offsetof(Stage, lg) % 128 == 0, "TMA destination alignment");
  Stage* st = reinterpret_cast<Stage*>(base);
  R (*part)[m][6][kCells] = reinterpret_cast<R (*)[m][6][kCells]>(base + 2 * sizeof(Stage));
  R (*wn)[kCells] = reinterpret_cast<R (*)[kCells]>(base + 2 * sizeof(Stage) + sizeof(R) * 3 * m * 6 * kCells);
  const int ntiles = ctx.ntiles();
  const int t = threadIdx.x;
  constexpr unsigned kBytes = sizeof(Stage);
  auto issue = [&](int s, int tile) {
    int c0, cnt;
    ctx.range(tile, c0, cnt);
    const R* C = ctx.comp(tile);
    mbar_arrive_expect_tx(&bar[s], kBytes - (C ? 0u : (unsigned)sizeof(Stage::cc)) -
                                       (LIM ? 0u : (unsigned)sizeof(Stage::lg)));
    tma_load_2d(&st[s].geo[0][0], mEgeo, c0, 0, &bar[s]);
    tma_load_2d(&st[s].idx[0][0], mIdx, c0, 0, &bar[s]);
    if (LIM) tma_load_2d(&st[s].lg[0][0], mLgeo, c0, 0, &bar[s]);
    bulk_load(&st[s].pb[0][0], Pb + (size_t)c0 * 18 * m, kCells * 18 * m * sizeof(R), &bar[s]);
    bulk_load(&st[s].u[0][0], ctx.uin(tile) + (size_t)c0 * 3 * m, kCells * 3 * m * sizeof(R), &bar[s]);
    if (C) bulk_load(&st[s].cc[0][0], C + (size_t)c0 * m, kCells * m * sizeof(R), &bar[s]);
  };
  int tile = next_active(ctx, blockIdx.x);
  if (t == 0 && tile < ntiles) {
    fence_proxy_async();
    issue(0, tile);
  }
  int s = 0;
  for (; tile < ntiles; s ^= 1) {
    const int next = next_active(ctx, tile + gridDim.x);
    if (t == 0 && next < ntiles) {
      fence_proxy_async();
      issue(s ^ 1, next);
    }
    const bool ok = mbar_wait(&bar[s], ph[s]);
    ph[s] ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        ctx.flag(2u);
        if (next < ntiles && mbar_wait(&bar[s ^ 1], ph[s ^ 1])) ph[s ^ 1] ^= 1u;
      }
      return false;
    }
    int cell0, count;
    ctx.range(tile, cell0, count);
    const R* U = ctx.uin(tile);
    R* Un = ctx.uout(tile);
    const R dtr = R(ctx.dt_of(tile));
    const Stage& S = st[s];
    flux_update_block<R, EQ, GL, LIM>(ctx, tile, cell0, count, S, StagedRecs<R, EQ>{&S, Pb}, U, Un, dtr, P, part, wn);
    tile = next;
  }
  return true;
}

// ---------------------------------------------------------------- single-solve kernels
template <typename R, int EQ, bool LIM>
__global__ void __launch_bounds__(LIM ? kThreads : kLeanThreads) k_recon(const __grid_constant__ CUtensorMap mGeo,
                                                     const __grid_constant__ CUtensorMap mIdx, GeoView<R> G,
                                                     const R* __restrict__ U, R* __restrict__ Pb, EqParams P,
                                                     DevScalars* sc, double dt_fixed, TileSet ts) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = smem_base(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + recon_smem_bytes<R, EQ>() - 128 - 2 * sizeof(uint64_t));
  const volatile DevScalars* vsc = sc;
  if (vsc->done) return;
  SingleCtx<R> ctx{ts, G.N, U, nullptr, dt_fixed > 0 ? dt_fixed : vsc->dt, sc, dinf(), nullptr};
  if (threadIdx.x == 0) {
    prefetch_tensormap(&mGeo); prefetch_tensormap(&mIdx);
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  unsigned ph[2] = {0u, 0u};
  recon_phase<R, EQ, LIM, LIM ? kThreads : kLeanThreads>(ctx, &mGeo, &mIdx, P, Pb, base, bar, ph);
}

// Resident blocks per SM the flux kernel is compiled for (register budget):
// FP32 Euler takes HW_EDGE_MIN_BLOCKS (4: 72 registers, no spills; the
// boundary-ghost branches would otherwise raise it to 95 and cost a block per
// SM), the rest the compiler's choice.
#ifndef HW_EDGE_MIN_BLOCKS
#define HW_EDGE_MIN_BLOCKS 4
#endif
template <typename R, int EQ> constexpr int edge_min_blocks() {
  return (sizeof(R) == 4 && EQ == kEqEuler) ? HW_EDGE_MIN_BLOCKS : 1;
}

template <typename R, int EQ, bool GL, bool LIM>
__global__ void __launch_bounds__(kThreads, edge_min_blocks<R, EQ>()) k_edge(const __grid_constant__ CUtensorMap mEgeo,
                                                    const __grid_constant__ CUtensorMap mIdx,
                                                    const __grid_constant__ CUtensorMap mLgeo, GeoView<R> G,
                                                    const R* __restrict__ U, R* __restrict__ Un,
                                                    const R* __restrict__ Pb, R* C, EqParams P, DevScalars* sc,
                                                    double dt_fixed, TileSet ts) {
  constexpr int m = EqTraits<EQ>::m;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = smem_base(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + edge_smem_bytes<R, EQ>() - 128 - 2 * sizeof(uint64_t));
  const int N = G.N;
  const int t = threadIdx.x;
  const volatile DevScalars* vs = sc;
  if (vs->done) {  // target reached: keep the state, preserving the buffer alternation
    for (int tile = blockIdx.x; tile < ts.ntiles; tile += gridDim.x) {
      int cell0, count;
      tile_range(ts, N, tile, cell0, count);
      for (int k = t; k < 3 * m * count; k += kThreads) Un[(size_t)cell0 * 3 * m + k] = U[(size_t)cell0 * 3 * m + k];
    }
    return;
  }
  const double dt = dt_fixed > 0 ? dt_fixed : vs->dt;
  SingleCtx<R> ctx{ts, N, U, Un, dt, sc, dinf(), C};
  if (t == 0) {
    prefetch_tensormap(&mEgeo); prefetch_tensormap(&mIdx);
    if (LIM) prefetch_tensormap(&mLgeo);
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  unsigned ph[2] = {0u, 0u};
  if (!edge_phase<R, EQ, GL, LIM>(ctx, &mEgeo, &mIdx, &mLgeo, P, Pb, base, bar, ph)) ctx.local_min = dinf();
  finish_step(sc, ctx.local_min, dt, true);
}

// ---------------------------------------------------------------- edge-once flux phase
// The two-kernel flux phase evaluates each edge once instead of once per
// cell: k_edge_flux, one thread per edge (listed by its left, owning cell),
// computes both Gauss points' time-integrated flux and central value (with
// the flux blending of the scale limiter) into EP; k_edge_update then runs the
// update of every cell (shares of its six points, read from its own slots or
// from the neighbour's slot of the same point, sums, update, CFL).  The values
// are those the owning cell computes in k_edge, so both paths give the same
// bits; this one does half the flux arithmetic, which pays where the FP64
// pipe bounds the step.
constexpr int kFluxThreads = 128;

template <typename R, int EQ, bool GL, bool LIM>
__global__ void __launch_bounds__(kFluxThreads) k_edge_flux(GeoView<R> G, const R* __restrict__ U,
                                                            const R* __restrict__ Pb, R* __restrict__ EP,
                                                            const int32_t* __restrict__ oedges, int ne, EqParams P,
                                                            DevScalars* sc, double dt_fixed) {
  constexpr int m = EqTraits<EQ>::m;
  static_assert(!LIM || EQ == kEqEuler, "flux blending is for the Euler equations");
  const volatile DevScalars* vs = sc;
  if (vs->done) return;
  const R dtr = R(dt_fixed > 0 ? dt_fixed : vs->dt);
  for (int e = blockIdx.x * kFluxThreads + threadIdx.x; e < ne; e += gridDim.x * kFluxThreads) {
    const int code = oedges[e], i = code >> 2, j = code & 3;
    const int nb = G.n(I_NBR + j, i), packed = G.n(I_NBE, i);
    const int je = (packed >> (2 * j)) & 3;
    const R nx = G.r(G_NRM + 2 * j, i), ny = G.r(G_NRM + 2 * j + 1, i);
    const R* ui = U + (size_t)i * 3 * m;
    R Wi[m], Wn[m];
    copy_rec<R, m>(Wi, ui);
    const int gtype = nb >= 0 ? kGhostTransmissive : ghost_type(packed, j);
    if (nb >= 0) {
      copy_rec<R, m>(Wn, U + (size_t)nb * 3 * m);
    } else {
#pragma unroll
      for (int c = 0; c < m; ++c) {
        R v, yv;
        ghost_component<R, EQ>(gtype, ui, nx, ny, c, P, Wn[c], v, yv);
      }
    }
    const R alpha = edge_alpha<R, EQ>(Wi, Wn, true, nx, ny, P);
    R Fe[2][m], Sh[2][m];
#pragma unroll
    for (int gm = 0; gm < 2; ++gm)
      edge_point_flux<R, EQ, GL>(Pb + (size_t)i * 18 * m + (2 * j + gm) * 3 * m,
                                 nb >= 0 ? Pb + (size_t)nb * 18 * m + (2 * je + 1 - gm) * 3 * m : nullptr, gtype,
                                 true, nx, ny, alpha, dtr, P, Fe[gm], Sh[gm]);
    if constexpr (LIM) {
      R FH[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) FH[c] = R(0.5) * (Fe[0][c] + Fe[1][c]);
      const R pown = G.r(G_PK, i), pnb = G.r(G_PN + j, i);
#pragma unroll
      for (int gm = 0; gm < 2; ++gm)
        blend_point<R, EQ>(Wi, Wn, true, nb >= 0, nx, ny, alpha, FH, pown, pnb, dtr, P, Fe[gm]);
    }
#pragma unroll
    for (int gm = 0; gm < 2; ++gm) {
      R* out = EP + ((size_t)i * 6 + 2 * j + gm) * 2 * m;
#pragma unroll
      for (int c = 0; c < m; ++c) { out[c] = Fe[gm][c]; out[m + c] = Sh[gm][c]; }
    }
  }
}

template <typename R, int EQ> struct UpdStage {
  static constexpr int m = EqTraits<EQ>::m;
  R geo[kEdgePlanes][kCells];    // TMA tensor box: planes x cells
  int32_t idx[4][kCells];        // TMA tensor box
  R u[kCells][3 * m];            // bulk copy of the tile's state records
  R cc[kCells][m];               // bulk copy of the compensation words (FP32 form; else unused)
};
static_assert(sizeof(UpdStage<float, 2>) % 128 == 0 && sizeof(UpdStage<double, 2>) % 128 == 0 &&
                  sizeof(UpdStage<float, 0>) % 128 == 0 && sizeof(UpdStage<double, 0>) % 128 == 0,
              "every stage starts 128-byte aligned (TMA destination)");

template <typename R, int EQ> constexpr size_t update_smem_bytes() {
  return 2 * sizeof(UpdStage<R, EQ>) + sizeof(R) * 3 * EqTraits<EQ>::m * 6 * kCells +
         sizeof(R) * EqTraits<EQ>::m * kCells + 2 * sizeof(uint64_t) + 128;
}

template <typename R, int EQ>
__global__ void __launch_bounds__(kThreads) k_edge_update(const __grid_constant__ CUtensorMap mEgeo,
                                                          const __grid_constant__ CUtensorMap mIdx, GeoView<R> G,
                                                          const R* __restrict__ U, R* __restrict__ Un,
                                                          const R* __restrict__ EP, R* C, EqParams P, DevScalars* sc,
                                                          double dt_fixed, TileSet ts) {
  constexpr int m = EqTraits<EQ>::m;
  using Stage = UpdStage<R, EQ>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = smem_base(smem_raw);
  Stage* st = reinterpret_cast<Stage*>(base);
  R (*part)[m][6][kCells] = reinterpret_cast<R (*)[m][6][kCells]>(base + 2 * sizeof(Stage));
  R (*wn)[kCells] = reinterpret_cast<R (*)[kCells]>(base + 2 * sizeof(Stage) + sizeof(R) * 3 * m * 6 * kCells);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + update_smem_bytes<R, EQ>() - 128 - 2 * sizeof(uint64_t));
  const int N = G.N;
  const int t = threadIdx.x;
  const volatile DevScalars* vs = sc;
  if (vs->done) {  // target reached: keep the state, preserving the buffer alternation
    for (int tile = blockIdx.x; tile < ts.ntiles; tile += gridDim.x) {
      int cell0, count;
      tile_range(ts, N, tile, cell0, count);
      for (int k = t; k < 3 * m * count; k += kThreads) Un[(size_t)cell0 * 3 * m + k] = U[(size_t)cell0 * 3 * m + k];
    }
    return;
  }
  const double dt = dt_fixed > 0 ? dt_fixed : vs->dt;
  const R dtr = R(dt);
  SingleCtx<R> ctx{ts, N, U, Un, dt, sc, dinf(), C};
  if (t == 0) {
    prefetch_tensormap(&mEgeo); prefetch_tensormap(&mIdx);
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  constexpr unsigned kBytes = sizeof(Stage);
  auto issue = [&](int sidx, int tile) {
    int c0, cnt;
    tile_range(ts, N, tile, c0, cnt);
    mbar_arrive_expect_tx(&bar[sidx], kBytes - (C ? 0u : (unsigned)sizeof(Stage::cc)));
    tma_load_2d(&st[sidx].geo[0][0], &mEgeo, c0, 0, &bar[sidx]);
    tma_load_2d(&st[sidx].idx[0][0], &mIdx, c0, 0, &bar[sidx]);
    bulk_load(&st[sidx].u[0][0], U + (size_t)c0 * 3 * m, kCells * 3 * m * sizeof(R), &bar[sidx]);
    if (C) bulk_load(&st[sidx].cc[0][0], C + (size_t)c0 * m, kCells * m * sizeof(R), &bar[sidx]);
  };
  unsigned ph[2] = {0u, 0u};
  int tile = blockIdx.x;
  if (t == 0 && tile < ts.ntiles) {
    fence_proxy_async();
    issue(0, tile);
  }
  bool ok = true;
  for (int s = 0; tile < ts.ntiles; s ^= 1) {
    const int next = tile + gridDim.x;
    if (t == 0 && next < ts.ntiles) {
      fence_proxy_async();
      issue(s ^ 1, next);
    }
    const bool w = mbar_wait(&bar[s], ph[s]);
    ph[s] ^= 1u;
    if (__syncthreads_or(!w)) {
      if (t == 0) {
        ctx.flag(2u);
        if (next < ts.ntiles && mbar_wait(&bar[s ^ 1], ph[s ^ 1])) ph[s ^ 1] ^= 1u;   // drain the copy in flight
      }
      ok = false;
      break;
    }
    int cell0, count;
    tile_range(ts, N, tile, cell0, count);
    const Stage& S = st[s];
    {
      const int lc = t % kCells, qp = t / kCells;
      if (lc < count) {
        const int j = qp >> 1, gm = qp & 1;
        const int nb = S.idx[j][lc];
        const int je = (S.idx[3][lc] >> (2 * j)) & 3;
        const bool left = (S.idx[3][lc] >> (6 + j)) & 1;
        // this point's values: the cell's own slot if it owns the edge, else
        // the neighbour's slot of the same physical point (its point (je, 1 - gm))
        const size_t slot = left ? (size_t)(cell0 + lc) * 6 + qp : (size_t)nb * 6 + 2 * je + (1 - gm);
        R FS[2 * m];
        copy_rec<R, 2 * m>(FS, EP + slot * 2 * m);
        point_shares<R, m>(left, S.geo[6 + j][lc], S.geo[2 * j][lc], S.geo[2 * j + 1][lc], FS, FS + m, S.u[lc], qp,
                           lc, part);
      }
    }
    __syncthreads();
    sum_update_cfl<R, EQ>(ctx, tile, cell0, count, S, Un, dtr, P, part, wn);
    tile = next;
  }
  if (!ok) ctx.local_min = dinf();
  finish_step(sc, ctx.local_min, dt, true);
}

// ---------------------------------------------------------------- fused step
// One kernel for the whole step: a block takes a tile of TT consecutive
// (Hilbert-ordered) cells, reconstructs them and runs the Lax-Wendroff
// procedure at their edge Gauss points (32-cell sub-tiles, TMA-staged
// geometry), does the same for the tile's halo (the cells outside the tile
// that share an edge with it; their geometry and stencils are gathered from
// global memory), keeps all those Taylor records in shared memory, and then
// forms the fluxes and updates the tile's cells (32-cell sub-tiles again).  The
// edge-point records never reach global memory; the price is the halo's
// reconstruction, done by both tiles it borders.

// Flux stage of the fused kernel: an EdgeStage without the edge-point records
// but with the packed neighbour slots of the 32 cells.
template <typename R, int EQ> struct FluxStage {
  static constexpr int m = EqTraits<EQ>::m;
  R geo[kEdgePlanes][kCells];    // TMA tensor box
  int32_t idx[4][kCells];        // TMA tensor box
  R lg[kLimPlanes][kCells];      // TMA tensor box (scale limiter only)
  R u[kCells][3 * m];            // bulk copy of the state records
  R cc[kCells][m];               // bulk copy of the compensation words (FP32 form)
  int32_t slot[kCells];          // bulk copy of the neighbour slots
};

template <typename R, int EQ> constexpr size_t round128(size_t x) { return (x + 127) / 128 * 128; }

// Shared-memory layout of the fused kernel (byte offsets from the 128-byte
// aligned base).
template <typename R, int EQ, int TT, int HC> struct FusedSmem {
  static constexpr int m = EqTraits<EQ>::m;
  static constexpr size_t stage = round128<R, EQ>(sizeof(ReconStage<R, EQ>) > sizeof(FluxStage<R, EQ>)
                                                       ? sizeof(ReconStage<R, EQ>) : sizeof(FluxStage<R, EQ>));
  static constexpr size_t pt = 2 * stage;                                   // [TT][18m] tile records
  static constexpr size_t ph = pt + sizeof(R) * TT * 18 * m;                // [HC][18m] halo records
  static constexpr size_t qs = ph + sizeof(R) * HC * 18 * m;                // [m][6][32]
  static constexpr size_t lim = qs + sizeof(R) * m * 6 * kCells;            // [6][32]
  static constexpr size_t part = lim + sizeof(R) * 6 * kCells;              // [3][m][6][32]
  static constexpr size_t wn = part + sizeof(R) * 3 * m * 6 * kCells;       // [m][32]
  static constexpr size_t hc = wn + sizeof(R) * m * kCells;                 // [HC + 32] halo cells
  static constexpr size_t bar = round128<R, EQ>(hc + sizeof(int) * (HC + kCells));
  static constexpr size_t bytes = bar + 2 * sizeof(uint64_t) + 128;         // + alignment slack
};

// Edge-point records of a fused tile: the tile's own in Pt (tile-local index),
// the halo's in Ph; slot: the packed neighbour slots of the 32 cells of the
// current sub-tile (3 x 10 bits: < TT tile-local, TT + h halo h).
template <typename R, int EQ> struct FusedRecs {
  static constexpr int m = EqTraits<EQ>::m;
  const R* Pt;
  const R* Ph;
  const int32_t* slot;
  int sub0;    // tile-local index of the sub-tile's first cell
  int tt;      // cells per tile
  int lim;     // tt + halo capacity: slots at or above it are invalid
  __device__ __forceinline__ const R* mine(int lc, int q) const { return Pt + (size_t)(sub0 + lc) * 18 * m + q * 3 * m; }
  __device__ __forceinline__ const R* theirs(int lc, int j, int, int qn) const {
    int v = (slot[lc] >> (kSlotBits * j)) & kSlotNone;
    if (v >= lim) v = sub0 + lc;   // never for tables built by the host; keeps the read in bounds
    return (v < tt ? Pt + (size_t)v * 18 * m : Ph + (size_t)(v - tt) * 18 * m) + qn * 3 * m;
  }
};

template <typename R, int EQ, bool GL, bool LIM, int TT, int HC>
__global__ void __launch_bounds__(kThreads) k_fused(const __grid_constant__ CUtensorMap mGeo,
                                                     const __grid_constant__ CUtensorMap mEgeo,
                                                     const __grid_constant__ CUtensorMap mIdx,
                                                     const __grid_constant__ CUtensorMap mLgeo, GeoView<R> G,
                                                     const R* __restrict__ U, R* __restrict__ Un, R* C, EqParams P,
                                                     DevScalars* sc, double dt_fixed, FusedTiles ft) {
  constexpr int m = EqTraits<EQ>::m;
  static_assert(TT % kCells == 0 && TT + HC <= kSlotNone, "tile and halo fit the slot encoding");
  using L = FusedSmem<R, EQ, TT, HC>;
  using RS = ReconStage<R, EQ>;
  using FS = FluxStage<R, EQ>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = smem_base(smem_raw);
  R* Pt = reinterpret_cast<R*>(base + L::pt);
  R* Ph = reinterpret_cast<R*>(base + L::ph);
  R (*qs)[6][kCells] = reinterpret_cast<R (*)[6][kCells]>(base + L::qs);
  R (*lim)[kCells] = reinterpret_cast<R (*)[kCells]>(base + L::lim);
  R (*part)[m][6][kCells] = reinterpret_cast<R (*)[m][6][kCells]>(base + L::part);
  R (*wn)[kCells] = reinterpret_cast<R (*)[kCells]>(base + L::wn);
  int* hcells = reinterpret_cast<int*>(base + L::hc);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + L::bar);
  const int N = G.N, t = threadIdx.x;
  const volatile DevScalars* vs = sc;
  if (vs->done) {  // target reached: keep the state, preserving the buffer alternation
    for (int tile = blockIdx.x; tile < ft.ntiles; tile += gridDim.x) {
      const int cell0 = tile * TT, count = min(TT, N - cell0);
      for (int k = t; k < 3 * m * count; k += kThreads) Un[(size_t)cell0 * 3 * m + k] = U[(size_t)cell0 * 3 * m + k];
    }
    return;
  }
  const double dt = dt_fixed > 0 ? dt_fixed : vs->dt;
  const R dtr = R(dt);
  SingleCtx<R> ctx{TileSet{nullptr, 0}, N, U, Un, dt, sc, dinf(), C};
  if (t == 0) {
    prefetch_tensormap(&mGeo); prefetch_tensormap(&mEgeo); prefetch_tensormap(&mIdx);
    if (LIM) prefetch_tensormap(&mLgeo);
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto stage_ptr = [&](int s) { return base + (size_t)s * L::stage; };
  auto nsub = [&](int tile) { return (min(TT, N - tile * TT) + kCells - 1) / kCells; };
  // work items of this block, in order: per tile the reconstruction sub-tiles
  // (kind 0), then the flux sub-tiles (kind 1)
  struct Item { int tile, kind, sub; };
  auto advance = [&](Item it) {
    if (++it.sub == nsub(it.tile)) {
      it.sub = 0;
      if (it.kind == 0) it.kind = 1;
      else { it.kind = 0; it.tile += gridDim.x; }
    }
    return it;
  };
  auto issue = [&](int s, const Item& it) {
    const int c0 = it.tile * TT + it.sub * kCells;
    if (it.kind == 0) {
      RS* S = reinterpret_cast<RS*>(stage_ptr(s));
      mbar_arrive_expect_tx(&bar[s], (unsigned)sizeof(RS));
      tma_load_2d(&S->geo[0][0], &mGeo, c0, 0, &bar[s]);
      tma_load_2d(&S->idx[0][0], &mIdx, c0, 0, &bar[s]);
      bulk_load(&S->u[0][0], U + (size_t)c0 * 3 * m, kCells * 3 * m * sizeof(R), &bar[s]);
    } else {
      FS* S = reinterpret_cast<FS*>(stage_ptr(s));
      const unsigned bytes = (unsigned)(sizeof(S->geo) + sizeof(S->idx) + (LIM ? sizeof(S->lg) : 0) + sizeof(S->u) +
                                        (C ? sizeof(S->cc) : 0) + sizeof(S->slot));
      mbar_arrive_expect_tx(&bar[s], bytes);
      tma_load_2d(&S->geo[0][0], &mEgeo, c0, 0, &bar[s]);
      tma_load_2d(&S->idx[0][0], &mIdx, c0, 0, &bar[s]);
      if (LIM) tma_load_2d(&S->lg[0][0], &mLgeo, c0, 0, &bar[s]);
      bulk_load(&S->u[0][0], U + (size_t)c0 * 3 * m, kCells * 3 * m * sizeof(R), &bar[s]);
      if (C) bulk_load(&S->cc[0][0], C + (size_t)c0 * m, kCells * m * sizeof(R), &bar[s]);
      bulk_load(&S->slot[0], ft.slot + c0, kCells * sizeof(int32_t), &bar[s]);
    }
  };
  unsigned ph[2] = {0u, 0u};
  Item cur{(int)blockIdx.x, 0, 0};
  if (t == 0 && cur.tile < ft.ntiles) {
    fence_proxy_async();
    issue(0, cur);
  }
  int s = 0;
  while (cur.tile < ft.ntiles) {
    const Item nxt = advance(cur);
    if (t == 0 && nxt.tile < ft.ntiles) {
      fence_proxy_async();
      issue(s ^ 1, nxt);
    }
    const bool ok = mbar_wait(&bar[s], ph[s]);
    ph[s] ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        ctx.flag(2u);
        if (nxt.tile < ft.ntiles && mbar_wait(&bar[s ^ 1], ph[s ^ 1])) ph[s ^ 1] ^= 1u;   // drain the copy in flight
      }
      ctx.local_min = dinf();
      break;
    }
    const int c0 = cur.tile * TT + cur.sub * kCells, count = min(kCells, N - c0);
    if (cur.kind == 0) {
      const RS* S = reinterpret_cast<const RS*>(stage_ptr(s));
      R* dst = Pt + (size_t)cur.sub * kCells * 18 * m;
      recon_lw_block<R, EQ, LIM, kThreads>(StagedCells<R, EQ>{S}, count, U, dtr, P, qs, lim,
                                           [&](int lc, int qp, const R* rec) {
                                             copy_rec<R, 3 * m>(dst + (size_t)lc * 18 * m + qp * 3 * m, rec);
                                           });
      if (cur.sub == nsub(cur.tile) - 1) {
        // the tile's halo, 32 cells at a time (the first flux stage is in flight)
        const int h0 = ft.halo_off[cur.tile];
        const int H = min(ft.halo_off[cur.tile + 1] - h0, HC);
        for (int k = t; k < HC + kCells; k += kThreads) hcells[k] = H > 0 ? ft.halo[h0 + min(k, H - 1)] : 0;
        __syncthreads();
        for (int hb = 0; hb < H; hb += kCells) {
          R* hdst = Ph + (size_t)hb * 18 * m;
          recon_lw_block<R, EQ, LIM, kThreads>(GlobalCells<R, EQ>{G.rg, G.ig, U, hcells + hb, G.ld}, min(kCells, H - hb),
                                               U, dtr, P, qs, lim, [&](int lc, int qp, const R* rec) {
                                                 copy_rec<R, 3 * m>(hdst + (size_t)lc * 18 * m + qp * 3 * m, rec);
                                               });
        }
      }
    } else {
      const FS* S = reinterpret_cast<const FS*>(stage_ptr(s));
      flux_update_block<R, EQ, GL, LIM>(ctx, 0, c0, count, *S,
                                        FusedRecs<R, EQ>{Pt, Ph, S->slot, cur.sub * kCells, TT, TT + HC}, U, Un,
                                        dtr, P, part, wn);
    }
    s ^= 1;
    cur = nxt;
  }
  finish_step(sc, ctx.local_min, dt, true);
}

// ---------------------------------------------------------------- batched persistent kernel
// Grid-wide barrier of a cooperative launch; the spin is bounded: on time-out
// the barrier reports false (flag 2 raised by the caller).  `skip` (tests
// only) makes this block leave without arriving, so that the others time out.
__device__ bool grid_barrier(BatchCtl* ctl, unsigned long long spin_limit, bool skip) {
  __shared__ int ok_s;
  // the phase's plain stores (edge-point data, new states) are read by bulk
  // copies after the barrier: order them for the async proxy first
  fence_proxy_async_global();
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (skip) {
      ok = 0;
    } else {
      volatile unsigned* gen = &ctl->bar_gen;
      const unsigned g = *gen;
      __threadfence();
      const unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
      if (arrived == gridDim.x - 1) {
        atomicExch(&ctl->bar_count, 0u);
        __threadfence();
        atomicAdd(&ctl->bar_gen, 1u);
      } else {
        unsigned long long it = 0;
        while (*gen == g) {
          if (++it > spin_limit) { ok = 0; break; }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// All steps of all solves of a batch in one launch: per step a
// reconstruction phase over the tiles of the running solves, a grid barrier,
// the flux/update phase (per-solve CFL minima), a barrier, the per-solve time
// step / status update, a barrier.  Leaves when no solve is running or after
// max_steps steps.
// Resident blocks per SM of the batched kernel (register budget), FP32.
#ifndef HW_BATCH_MIN_BLOCKS
#define HW_BATCH_MIN_BLOCKS 3
#endif
template <typename R> constexpr int batch_min_blocks() { return sizeof(R) == 4 ? HW_BATCH_MIN_BLOCKS : 1; }

// End of a batched step, thread gid for solve gid: time, step count, status
// and next time step of every running solve (its CFL minimum taken over the
// step's tiles); counts the solves still running in active[slot].
__device__ __forceinline__ void batch_finish_step(BatchSolve* bs, BatchCtl* ctl, int gid, int nsolves, double cfl,
                                                  int slot) {
  if (gid < nsolves) {
    volatile BatchSolve* b = &bs[gid];
    if (!b->done) {
      const double tn = b->t + b->dt;
      b->t = tn;
      b->nsteps = b->nsteps + 1;
      const double mn = __longlong_as_double((long long)atomicAdd(&bs[gid].lam_min_bits, 0ull));
      double dtn = cfl * mn;
      int done = 0;
      if (b->failed) done = 1;
      else if (tn >= b->T * (1.0 - 1e-14)) done = 1;
      else if (tn + dtn > b->T) dtn = b->T - tn;
      b->dt = dtn;
      b->done = done;
      atomicExch(&bs[gid].lam_min_bits, dbits(dinf()));
      if (!done) atomicAdd(&ctl->active[slot], 1u);
    }
  }
  if (gid == 0) {
    atomicExch(&ctl->active[slot ^ 1], 0u);
    atomicAdd(&ctl->steps_run, 1);
  }
}

template <typename R, int EQ, bool LIM>
__global__ void __launch_bounds__(kThreads, batch_min_blocks<R>()) k_batch(const __grid_constant__ CUtensorMap mGeo,
                                                     const __grid_constant__ CUtensorMap mEgeo,
                                                     const __grid_constant__ CUtensorMap mIdx,
                                                     const __grid_constant__ CUtensorMap mLgeo, R* U0, R* U1,
                                                     R* __restrict__ Pb, EqParams P, BatchCtx<R> ctx, int nsolves,
                                                     double cfl, int max_steps, unsigned long long spin_limit,
                                                     int withhold_block) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = smem_base(smem_raw);
  constexpr size_t kStageBytes = recon_smem_bytes<R, EQ>() > edge_smem_bytes<R, EQ>() ? recon_smem_bytes<R, EQ>()
                                                                                     : edge_smem_bytes<R, EQ>();
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + kStageBytes - 128 - 2 * sizeof(uint64_t));
  BatchCtl* ctl = ctx.ctl;
  if (threadIdx.x == 0) {
    prefetch_tensormap(&mGeo); prefetch_tensormap(&mEgeo); prefetch_tensormap(&mIdx);
    if (LIM) prefetch_tensormap(&mLgeo);
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  unsigned ph[2] = {0u, 0u};
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const bool skip = (int)blockIdx.x == withhold_block;
  bool ok = true;
  for (int step = 0; step < max_steps && ok; ++step) {
    const int slot = step & 1;
    ok = recon_phase<R, EQ, LIM, kThreads>(ctx, &mGeo, &mIdx, P, Pb, base, bar, ph);
    if (!grid_barrier(ctl, spin_limit, skip || !ok)) ok = false;
    if (!ok) break;
    ok = edge_phase<R, EQ, false, LIM>(ctx, &mEgeo, &mIdx, &mLgeo, P, Pb, base, bar, ph);
    if (!grid_barrier(ctl, spin_limit, !ok)) ok = false;
    if (!ok) break;
    batch_finish_step(ctx.bs, ctl, gid, nsolves, cfl, slot);
    if (!grid_barrier(ctl, spin_limit, false)) { ok = false; break; }
    if (*(volatile unsigned*)&ctl->active[slot] == 0) break;
  }
  if (!ok && threadIdx.x == 0) atomicOr(&ctl->flags, 2u);
}

// The batched step as three launches (schedule launch_mode 1): the same
// phases as k_batch without grid barriers, each kernel at its own register
// budget and occupancy; the launches of many steps are captured in one graph.
template <typename R, int EQ, bool LIM>
__global__ void __launch_bounds__(LIM ? kThreads : kLeanThreads) k_batch_recon(
    const __grid_constant__ CUtensorMap mGeo, const __grid_constant__ CUtensorMap mIdx, R* __restrict__ Pb, EqParams P,
    BatchCtx<R> ctx) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = smem_base(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + recon_smem_bytes<R, EQ>() - 128 - 2 * sizeof(uint64_t));
  if (threadIdx.x == 0) {
    prefetch_tensormap(&mGeo); prefetch_tensormap(&mIdx);
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  unsigned ph[2] = {0u, 0u};
  recon_phase<R, EQ, LIM, LIM ? kThreads : kLeanThreads>(ctx, &mGeo, &mIdx, P, Pb, base, bar, ph);
}

template <typename R, int EQ, bool LIM>
__global__ void __launch_bounds__(kThreads, edge_min_blocks<R, EQ>()) k_batch_edge(
    const __grid_constant__ CUtensorMap mEgeo, const __grid_constant__ CUtensorMap mIdx,
    const __grid_constant__ CUtensorMap mLgeo, R* __restrict__ Pb, EqParams P, BatchCtx<R> ctx) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = smem_base(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + edge_smem_bytes<R, EQ>() - 128 - 2 * sizeof(uint64_t));
  if (threadIdx.x == 0) {
    prefetch_tensormap(&mEgeo); prefetch_tensormap(&mIdx);
    if (LIM) prefetch_tensormap(&mLgeo);
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  unsigned ph[2] = {0u, 0u};
  edge_phase<R, EQ, false, LIM>(ctx, &mEgeo, &mIdx, &mLgeo, P, Pb, base, bar, ph);
}

__global__ void k_batch_finish(BatchSolve* bs, BatchCtl* ctl, int nsolves, double cfl, int slot) {
  batch_finish_step(bs, ctl, blockIdx.x * blockDim.x + threadIdx.x, nsolves, cfl, slot);
}

// CFL step of the current state (after an upload or a change of target).
template <typename R, int EQ>
__global__ void __launch_bounds__(256) k_cfl(GeoView<R> G, const R* __restrict__ U, EqParams P, DevScalars* sc) {
  constexpr int m = EqTraits<EQ>::m;
  const int N = G.N, ld = G.ld;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double local_min = dinf();
  if (i < N) {
    R W[m];
#pragma unroll
    for (int c = 0; c < m; ++c) W[c] = U[(size_t)i * 3 * m + c];
    if (!physical<R, EQ>(W, P)) atomicOr(&sc->flags, 1u);
    const R lam = spectral_radius_all<R, EQ>(W, P);
    if (lam > R(0)) local_min = (double)(G.r(G_INR, i) / lam);
    if (!(local_min >= 0)) local_min = dinf();
  }
  finish_step(sc, local_min, 0.0, false);
}

// Deterministic FP64 sums of |K| Wbar_K: fixed grid, fixed tree, then one block.
template <typename R>
__global__ void __launch_bounds__(256) k_consv_partial(const R* __restrict__ U, const R* __restrict__ C,
                                                        const double* __restrict__ area, int N, int ld, int m,
                                                        double* __restrict__ partial) {
  __shared__ double sh[256];
  for (int c = 0; c < m; ++c) {
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
      s += area[i] * ((double)U[(size_t)i * 3 * m + c] + (C ? (double)C[(size_t)i * m + c] : 0.0));
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[c * gridDim.x + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

__global__ void k_consv_final(const double* __restrict__ partial, int nparts, int m, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    for (int c = 0; c < m; ++c) {
      double s = 0.0;
      for (int k = 0; k < nparts; ++k) s += partial[c * nparts + k];
      out[c] = s;
    }
}

// host order (double, [planes][N]) -> internal order (R, [planes][ld]), and back
template <typename R>
__global__ void k_scatter_state(const double* __restrict__ host_order, const int32_t* __restrict__ perm, int N, int ld,
                                int planes, R* __restrict__ U) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int src = perm[i];
  for (int k = 0; k < planes; ++k) U[(size_t)i * planes + k] = (R)host_order[(size_t)k * N + src];
}
template <typename R>
__global__ void k_gather_state(const R* __restrict__ U, const R* __restrict__ C, int m,
                               const int32_t* __restrict__ perm, int N, int ld, int planes,
                               double* __restrict__ host_order) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int dst = perm[i];
  for (int k = 0; k < planes; ++k) {
    double v = (double)U[(size_t)i * planes + k];
    if (C && k < m) v += (double)C[(size_t)i * m + k];   // the cell averages with their compensation
    host_order[(size_t)k * N + dst] = v;
  }
}

__global__ void k_reset(DevScalars* sc, double t, double cfl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc->t = t; sc->dt = 0.0; sc->T = 0.0; sc->cfl = cfl;
    sc->lam_min_bits = 0x7ff0000000000000ull;
    sc->counter = 0u; sc->flags = 0u; sc->nsteps = 0; sc->done = 0; sc->has_T = 0;
  }
}

__global__ void k_set_target(DevScalars* sc, double T, int has_T) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc->has_T = has_T;
    sc->T = T;
    int done = 0;
    if (has_T) {
      if (sc->t >= T * (1.0 - 1e-14)) done = 1;
      else if (sc->t + sc->dt > T) sc->dt = T - sc->t;
    }
    sc->done = done;
  }
}

// ---------------------------------------------------------------- batch helpers
// CFL candidates of every tile of a batch (state buffer 0 at set-up): warp
// minimum, one atomic per tile on the tile's solve.
template <typename R, int EQ>
__global__ void __launch_bounds__(256) k_batch_cfl(GeoView<R> G, const R* __restrict__ U, const int4* __restrict__ tiles,
                                                   int ntiles, EqParams P, BatchSolve* bs, BatchCtl* ctl) {
  constexpr int m = EqTraits<EQ>::m;
  const int tile = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x & 31;
  if (tile >= ntiles) return;   // whole warps leave together
  const int4 e = tiles[tile];
  double v = dinf();
  if (lane < e.y) {
    const int i = e.x + lane;
    R W[m];
#pragma unroll
    for (int c = 0; c < m; ++c) W[c] = U[(size_t)i * 3 * m + c];
    if (!physical<R, EQ>(W, P)) {
      atomicOr(&ctl->flags, 1u);
      atomicExch(&bs[e.z].failed, 1);
    }
    const R lam = spectral_radius_all<R, EQ>(W, P);
    if (lam > R(0)) {
      const double r = (double)(G.r(G_INR, i) / lam);
      if (r >= 0) v = r;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0 && v < dinf()) atomicMin(&bs[e.z].lam_min_bits, dbits(v));
}

// Per solve: time step from the CFL minimum (clipped to the target when one is
// set), done flag; resets the minimum.
__global__ void k_batch_dt(BatchSolve* bs, int n, double cfl, double T, int has_T) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  BatchSolve& b = bs[s];
  const double mn = __longlong_as_double((long long)b.lam_min_bits);
  if (has_T) b.T = T;
  if (mn < dinf()) b.dt = cfl * mn;
  b.lam_min_bits = dbits(dinf());
  int done = b.failed ? 1 : 0;
  if (has_T) {
    if (b.t >= b.T * (1.0 - 1e-14)) done = 1;
    else if (b.t + b.dt > b.T) b.dt = b.T - b.t;
  }
  b.done = done;
}

__global__ void k_batch_reset_ctl(BatchCtl* ctl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->bar_count = 0u; ctl->bar_gen = 0u; ctl->active[0] = 0u; ctl->active[1] = 0u; ctl->flags = 0u;
    ctl->steps_run = 0;
  }
}

// ---------------------------------------------------------------- launchers
namespace {
// Resident blocks of a kernel on the current device (occupancy x SMs); the
// launches use min(tiles, this) blocks.
template <typename K> int resident_blocks(K kernel, int threads, size_t smem) {
  int dev = 0, sms = 148, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  return sms * (per_sm > 0 ? per_sm : 1);
}

template <typename R, int EQ, bool LIM> int recon_cap() {
  static const int cap = resident_blocks(k_recon<R, EQ, LIM>, LIM ? kThreads : kLeanThreads, recon_smem_bytes<R, EQ>());
  return cap;
}
template <typename R, int EQ, bool GL, bool LIM> int edge_cap() {
  static const int cap = resident_blocks(k_edge<R, EQ, GL, LIM>, kThreads, edge_smem_bytes<R, EQ>());
  return cap;
}
template <typename R, int EQ> void prepare_t() {
  (void)recon_cap<R, EQ, false>();
  if constexpr (EQ == kEqEuler) (void)recon_cap<R, EQ, true>();
  (void)edge_cap<R, EQ, false, false>();
  (void)edge_cap<R, EQ, true, false>();
  if constexpr (EQ == kEqEuler) (void)edge_cap<R, EQ, false, true>();
}

template <typename R, int EQ, bool LIM> void launch_recon_lim(const StepArgs& a, cudaStream_t st) {
  GeoView<R> G{reinterpret_cast<const R*>(a.rgeo), a.igeo, a.N, a.ld};
  constexpr size_t smem = recon_smem_bytes<R, EQ>();
  const int cap = recon_cap<R, EQ, LIM>();
  const int nt = a.tiles.ntiles;
  k_recon<R, EQ, LIM><<<nt < cap ? (nt > 0 ? nt : 1) : cap, LIM ? kThreads : kLeanThreads, smem, st>>>(
      a.maps->geo, a.maps->idx, G, reinterpret_cast<const R*>(a.U), reinterpret_cast<R*>(a.Pb), a.P, a.sc,
      a.dt_fixed, a.tiles);
}
template <typename R, int EQ> void launch_recon_t(const StepArgs& a, cudaStream_t st) {
  if constexpr (EQ == kEqEuler) {
    if (a.P.positivity) {
      launch_recon_lim<R, EQ, true>(a, st);
      return;
    }
  }
  launch_recon_lim<R, EQ, false>(a, st);
}
template <typename R, int EQ, bool GL, bool LIM> void launch_edge_rule(const StepArgs& a, cudaStream_t st) {
  GeoView<R> G{reinterpret_cast<const R*>(a.rgeo), a.igeo, a.N, a.ld};
  constexpr size_t smem = edge_smem_bytes<R, EQ>();
  const int cap = edge_cap<R, EQ, GL, LIM>();
  const int nt = a.tiles.ntiles;
  k_edge<R, EQ, GL, LIM><<<nt < cap ? (nt > 0 ? nt : 1) : cap, kThreads, smem, st>>>(
      a.maps->egeo, a.maps->idx, a.maps->lgeo, G, reinterpret_cast<const R*>(a.U), reinterpret_cast<R*>(a.Un),
      reinterpret_cast<const R*>(a.Pb), reinterpret_cast<R*>(a.C), a.P, a.sc, a.dt_fixed, a.tiles);
}
template <typename R, int EQ, bool GL, bool LIM> int flux_cap() {
  static const int cap = resident_blocks(k_edge_flux<R, EQ, GL, LIM>, kFluxThreads, 0);
  return cap;
}
template <typename R, int EQ> int update_cap() {
  static const int cap = resident_blocks(k_edge_update<R, EQ>, kThreads, update_smem_bytes<R, EQ>());
  return cap;
}
template <typename R, int EQ, bool GL, bool LIM> void launch_edge_once(const StepArgs& a, cudaStream_t st) {
  GeoView<R> G{reinterpret_cast<const R*>(a.rgeo), a.igeo, a.N, a.ld};
  const int nb = (a.n_oedges + kFluxThreads - 1) / kFluxThreads, fc = flux_cap<R, EQ, GL, LIM>();
  k_edge_flux<R, EQ, GL, LIM><<<nb < fc ? (nb > 0 ? nb : 1) : fc, kFluxThreads, 0, st>>>(
      G, reinterpret_cast<const R*>(a.U), reinterpret_cast<const R*>(a.Pb), reinterpret_cast<R*>(a.EP), a.oedges,
      a.n_oedges, a.P, a.sc, a.dt_fixed);
  const int nt = a.tiles.ntiles, uc = update_cap<R, EQ>();
  k_edge_update<R, EQ><<<nt < uc ? (nt > 0 ? nt : 1) : uc, kThreads, update_smem_bytes<R, EQ>(), st>>>(
      a.maps->egeo, a.maps->idx, G, reinterpret_cast<const R*>(a.U), reinterpret_cast<R*>(a.Un),
      reinterpret_cast<const R*>(a.EP), reinterpret_cast<R*>(a.C), a.P, a.sc, a.dt_fixed, a.tiles);
}
template <typename R, int EQ> void launch_edge_t(const StepArgs& a, cudaStream_t st) {
  if constexpr (EQ == kEqEuler) {
    if (a.P.positivity) {   // the Gauss-Legendre rule is refused with the limiter
      if (a.EP) launch_edge_once<R, EQ, false, true>(a, st);
      else launch_edge_rule<R, EQ, false, true>(a, st);
      return;
    }
  }
  if (a.P.time_rule == 1) {
    if (a.EP) launch_edge_once<R, EQ, true, false>(a, st);
    else launch_edge_rule<R, EQ, true, false>(a, st);
  } else {
    if (a.EP) launch_edge_once<R, EQ, false, false>(a, st);
    else launch_edge_rule<R, EQ, false, false>(a, st);
  }
}
template <typename R, int EQ> void prepare_edge_once_t() {
  (void)flux_cap<R, EQ, false, false>();
  (void)flux_cap<R, EQ, true, false>();
  if constexpr (EQ == kEqEuler) (void)flux_cap<R, EQ, false, true>();
  (void)update_cap<R, EQ>();
}
template <typename R> struct FusedShape {
  static constexpr int TT = sizeof(R) == 4 ? kFusedTile32 : kFusedTile64;
  static constexpr int HC = sizeof(R) == 4 ? kFusedHalo32 : kFusedHalo64;
};
template <typename R, int EQ, bool GL, bool LIM> int fused_cap() {
  constexpr int TT = FusedShape<R>::TT, HC = FusedShape<R>::HC;
  static const int cap = resident_blocks(k_fused<R, EQ, GL, LIM, TT, HC>, kThreads, FusedSmem<R, EQ, TT, HC>::bytes);
  return cap;
}
template <typename R, int EQ> void prepare_fused_t() {
  (void)fused_cap<R, EQ, false, false>();
  (void)fused_cap<R, EQ, true, false>();
  if constexpr (EQ == kEqEuler) (void)fused_cap<R, EQ, false, true>();
}
template <typename R, int EQ, bool GL, bool LIM> void launch_fused_v(const StepArgs& a, cudaStream_t st) {
  constexpr int TT = FusedShape<R>::TT, HC = FusedShape<R>::HC;
  GeoView<R> G{reinterpret_cast<const R*>(a.rgeo), a.igeo, a.N, a.ld};
  const int cap = fused_cap<R, EQ, GL, LIM>();
  const int nt = a.fused.ntiles;
  k_fused<R, EQ, GL, LIM, TT, HC><<<nt < cap ? (nt > 0 ? nt : 1) : cap, kThreads, FusedSmem<R, EQ, TT, HC>::bytes, st>>>(
      a.maps->geo, a.maps->egeo, a.maps->idx, a.maps->lgeo, G, reinterpret_cast<const R*>(a.U),
      reinterpret_cast<R*>(a.Un), reinterpret_cast<R*>(a.C), a.P, a.sc, a.dt_fixed, a.fused);
}
template <typename R, int EQ> void launch_fused_t(const StepArgs& a, cudaStream_t st) {
  if constexpr (EQ == kEqEuler) {
    if (a.P.positivity) {   // the Gauss-Legendre rule is refused with the limiter
      launch_fused_v<R, EQ, false, true>(a, st);
      return;
    }
  }
  if (a.P.time_rule == 1) launch_fused_v<R, EQ, true, false>(a, st);
  else launch_fused_v<R, EQ, false, false>(a, st);
}
template <typename R, int EQ> void launch_cfl_t(const StepArgs& a, cudaStream_t st) {
  GeoView<R> G{reinterpret_cast<const R*>(a.rgeo), a.igeo, a.N, a.ld};
  k_cfl<R, EQ><<<(a.N + 255) / 256, 256, 0, st>>>(G, reinterpret_cast<const R*>(a.U), a.P, a.sc);
}
}  // namespace

#define HW_DISPATCH(fn, prec, eq, ...)                 \
  do {                                                 \
    if ((prec) == 0) {                                 \
      if ((eq) == 0) fn<double, 0>(__VA_ARGS__);       \
      else if ((eq) == 1) fn<double, 1>(__VA_ARGS__);  \
      else fn<double, 2>(__VA_ARGS__);                 \
    } else {                                           \
      if ((eq) == 0) fn<float, 0>(__VA_ARGS__);        \
      else if ((eq) == 1) fn<float, 1>(__VA_ARGS__);   \
      else fn<float, 2>(__VA_ARGS__);                  \
    }                                                  \
  } while (0)

void prepare_step_kernels(int prec, int eq) { HW_DISPATCH(prepare_t, prec, eq); }
void launch_recon(int prec, int eq, const StepArgs& a, cudaStream_t st) { HW_DISPATCH(launch_recon_t, prec, eq, a, st); }
void launch_edge(int prec, int eq, const StepArgs& a, cudaStream_t st) { HW_DISPATCH(launch_edge_t, prec, eq, a, st); }
void launch_step(int prec, int eq, const StepArgs& a, cudaStream_t st) {
  launch_recon(prec, eq, a, st);
  launch_edge(prec, eq, a, st);
}
void launch_cfl(int prec, int eq, const StepArgs& a, cudaStream_t st) { HW_DISPATCH(launch_cfl_t, prec, eq, a, st); }
void launch_fused(int prec, int eq, const StepArgs& a, cudaStream_t st) { HW_DISPATCH(launch_fused_t, prec, eq, a, st); }
void prepare_fused_kernel(int prec, int eq) { HW_DISPATCH(prepare_fused_t, prec, eq); }
void prepare_edge_once_kernels(int prec, int eq) { HW_DISPATCH(prepare_edge_once_t, prec, eq); }

void launch_reset(DevScalars* sc, double t, double cfl, cudaStream_t st) { k_reset<<<1, 32, 0, st>>>(sc, t, cfl); }

void launch_set_target(DevScalars* sc, double T, int has_T, cudaStream_t st) {
  k_set_target<<<1, 32, 0, st>>>(sc, T, has_T);
}

void launch_consv(int prec, const void* U, const void* C, const double* area, int N, int ld, int m, double* partial,
                  double* out, cudaStream_t st) {
  if (prec == 0)
    k_consv_partial<double><<<kConsvBlocks, 256, 0, st>>>(reinterpret_cast<const double*>(U),
                                                          reinterpret_cast<const double*>(C), area, N, ld, m, partial);
  else
    k_consv_partial<float><<<kConsvBlocks, 256, 0, st>>>(reinterpret_cast<const float*>(U),
                                                         reinterpret_cast<const float*>(C), area, N, ld, m, partial);
  k_consv_final<<<1, 32, 0, st>>>(partial, kConsvBlocks, m, out);
}

void launch_scatter(int prec, const double* host_order, const int32_t* perm, int N, int ld, int planes, void* U,
                    cudaStream_t st) {
  const int nb = (N + 255) / 256;
  if (prec == 0)
    k_scatter_state<double><<<nb, 256, 0, st>>>(host_order, perm, N, ld, planes, reinterpret_cast<double*>(U));
  else
    k_scatter_state<float><<<nb, 256, 0, st>>>(host_order, perm, N, ld, planes, reinterpret_cast<float*>(U));
}

namespace {
template <typename R, int EQ, bool LIM> constexpr size_t batch_smem() {
  return recon_smem_bytes<R, EQ>() > edge_smem_bytes<R, EQ>() ? recon_smem_bytes<R, EQ>() : edge_smem_bytes<R, EQ>();
}
template <typename R, int EQ, bool LIM> int batch_cap_t() {
  static const int cap = [] {
    int per_sm = 0;
    cudaFuncSetAttribute(k_batch<R, EQ, LIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem<R, EQ, LIM>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<R, EQ, LIM>, kThreads, batch_smem<R, EQ, LIM>());
    return per_sm;
  }();
  return cap;
}
template <typename R, int EQ, bool LIM> cudaError_t launch_batch_t(const BatchArgs& a, cudaStream_t st) {
  BatchCtx<R> ctx{a.tiles, a.ntiles, reinterpret_cast<R*>(a.C), a.bs, a.ctl, reinterpret_cast<R*>(a.U0),
                  reinterpret_cast<R*>(a.U1)};
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(a.grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = batch_smem<R, EQ, LIM>();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch<R, EQ, LIM>, a.maps->geo, a.maps->egeo, a.maps->idx, a.maps->lgeo,
                            reinterpret_cast<R*>(a.U0), reinterpret_cast<R*>(a.U1), reinterpret_cast<R*>(a.Pb), a.P,
                            ctx, a.nsolves, a.cfl, a.max_steps, a.spin_limit, a.withhold_block);
}
template <typename R, int EQ> void launch_batch_cfl_t(const BatchArgs& a, cudaStream_t st) {
  GeoView<R> G{reinterpret_cast<const R*>(a.rgeo), a.igeo, a.N, a.ld};
  k_batch_cfl<R, EQ><<<(a.ntiles * 32 + 255) / 256, 256, 0, st>>>(G, reinterpret_cast<const R*>(a.U0), a.tiles,
                                                                  a.ntiles, a.P, a.bs, a.ctl);
}
}  // namespace

int batch_blocks_per_sm(int prec, int eq, bool lim) {
  if (prec == 0) {
    if (eq == 0) return batch_cap_t<double, 0, false>();
    if (eq == 1) return batch_cap_t<double, 1, false>();
    return lim ? batch_cap_t<double, 2, true>() : batch_cap_t<double, 2, false>();
  }
  if (eq == 0) return batch_cap_t<float, 0, false>();
  if (eq == 1) return batch_cap_t<float, 1, false>();
  return lim ? batch_cap_t<float, 2, true>() : batch_cap_t<float, 2, false>();
}

cudaError_t launch_batch(int prec, int eq, const BatchArgs& a, cudaStream_t st) {
  const bool lim = eq == 2 && a.P.positivity;
  if (prec == 0) {
    if (eq == 0) return launch_batch_t<double, 0, false>(a, st);
    if (eq == 1) return launch_batch_t<double, 1, false>(a, st);
    return lim ? launch_batch_t<double, 2, true>(a, st) : launch_batch_t<double, 2, false>(a, st);
  }
  if (eq == 0) return launch_batch_t<float, 0, false>(a, st);
  if (eq == 1) return launch_batch_t<float, 1, false>(a, st);
  return lim ? launch_batch_t<float, 2, true>(a, st) : launch_batch_t<float, 2, false>(a, st);
}

namespace {
template <typename R, int EQ, bool LIM> int batch_recon_cap() {
  static const int cap = resident_blocks(k_batch_recon<R, EQ, LIM>, LIM ? kThreads : kLeanThreads,
                                         recon_smem_bytes<R, EQ>());
  return cap;
}
template <typename R, int EQ, bool LIM> int batch_edge_cap() {
  static const int cap = resident_blocks(k_batch_edge<R, EQ, LIM>, kThreads, edge_smem_bytes<R, EQ>());
  return cap;
}
template <typename R, int EQ, bool LIM> cudaError_t launch_batch_step_t(const BatchArgs& a, int slot, cudaStream_t st) {
  BatchCtx<R> ctx{a.tiles, a.ntiles, reinterpret_cast<R*>(a.C), a.bs, a.ctl, reinterpret_cast<R*>(a.U0),
                  reinterpret_cast<R*>(a.U1)};
  const int nt = a.ntiles > 0 ? a.ntiles : 1;
  const int rc = batch_recon_cap<R, EQ, LIM>(), ec = batch_edge_cap<R, EQ, LIM>();
  k_batch_recon<R, EQ, LIM><<<nt < rc ? nt : rc, LIM ? kThreads : kLeanThreads, recon_smem_bytes<R, EQ>(), st>>>(
      a.maps->geo, a.maps->idx, reinterpret_cast<R*>(a.Pb), a.P, ctx);
  k_batch_edge<R, EQ, LIM><<<nt < ec ? nt : ec, kThreads, edge_smem_bytes<R, EQ>(), st>>>(
      a.maps->egeo, a.maps->idx, a.maps->lgeo, reinterpret_cast<R*>(a.Pb), a.P, ctx);
  k_batch_finish<<<(a.nsolves + 127) / 128, 128, 0, st>>>(a.bs, a.ctl, a.nsolves, a.cfl, slot);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_batch_step(int prec, int eq, const BatchArgs& a, int slot, cudaStream_t st) {
  const bool lim = eq == 2 && a.P.positivity;
  if (prec == 0) {
    if (eq == 0) return launch_batch_step_t<double, 0, false>(a, slot, st);
    if (eq == 1) return launch_batch_step_t<double, 1, false>(a, slot, st);
    return lim ? launch_batch_step_t<double, 2, true>(a, slot, st) : launch_batch_step_t<double, 2, false>(a, slot, st);
  }
  if (eq == 0) return launch_batch_step_t<float, 0, false>(a, slot, st);
  if (eq == 1) return launch_batch_step_t<float, 1, false>(a, slot, st);
  return lim ? launch_batch_step_t<float, 2, true>(a, slot, st) : launch_batch_step_t<float, 2, false>(a, slot, st);
}

void launch_batch_cfl(int prec, int eq, const BatchArgs& a, cudaStream_t st) {
  HW_DISPATCH(launch_batch_cfl_t, prec, eq, a, st);
}

void launch_batch_dt(BatchSolve* bs, int n, double cfl, double T, int has_T, cudaStream_t st) {
  k_batch_dt<<<(n + 127) / 128, 128, 0, st>>>(bs, n, cfl, T, has_T);
}

void launch_batch_reset_ctl(BatchCtl* ctl, cudaStream_t st) { k_batch_reset_ctl<<<1, 32, 0, st>>>(ctl); }

void launch_gather(int prec, const void* U, const void* C, int m, const int32_t* perm, int N, int ld, int planes,
                   double* host_order, cudaStream_t st) {
  const int nb = (N + 255) / 256;
  if (prec == 0)
    k_gather_state<double><<<nb, 256, 0, st>>>(reinterpret_cast<const double*>(U), reinterpret_cast<const double*>(C),
                                               m, perm, N, ld, planes, host_order);
  else
    k_gather_state<float><<<nb, 256, 0, st>>>(reinterpret_cast<const float*>(U), reinterpret_cast<const float*>(C), m,
                                              perm, N, ld, planes, host_order);
}

}  // namespace hw
