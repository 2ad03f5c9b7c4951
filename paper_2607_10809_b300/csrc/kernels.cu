// Kernels of one ADER-HWENO time step on a triangular mesh.
//
//   k_recon : per cell, Steps 1-6 of Section 2.2 (Eqs. pxy, smoo1,
//             nonlinearweight, recon), then at its six edge Gauss points the
//             Lax-Wendroff procedure of Section 2.1; writes the Taylor data
//             (W, W_t, W_tt) of Eqs. tay / tayext to the edge-point buffer.
//   k_edge  : per cell (owner computes, no atomics), for its three edges the
//             local Lax-Friedrichs flux at the Gauss-Lobatto time nodes (Eqs.
//             fx, flux), evaluated in a canonical orientation so that both
//             cells of an edge obtain bitwise-identical fluxes; the update of
//             the cell average (Eq. flx) and of the derivative averages by
//             Green-Gauss from the central values at t_{n+1} (Eqs. derave2d2,
//             timeflux, taylor2dtime); the CFL step for the next step.
//   k_cfl, k_consv, k_scatter_state, k_gather_state: CFL step of a state,
//             FP64 conservation sums, host-order <-> Hilbert-order copies.
#include <cstdint>

#include "device.cuh"
#include "kernels.h"

namespace hw {

namespace {

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

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
    atomicExch(&sc->lam_min_bits, dbits(__longlong_as_double(0x7ff0000000000000ll)));
    atomicExch(&sc->counter, 0u);
  }
}

}  // namespace

// ---------------------------------------------------------------- reconstruction
template <typename R, int EQ>
__global__ void __launch_bounds__(128) k_recon(GeoView<R> G, const R* __restrict__ U, R* __restrict__ Pb,
                                                EqParams P, const DevScalars* __restrict__ sc) {
  constexpr int m = EqTraits<EQ>::m;
  if (*(volatile const int*)&sc->done) return;
  const int N = G.N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int src[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int nb = G.n(I_NBR + j, i);
    src[j] = nb >= 0 ? nb : i;   // transmissive ghost carries the cell's own data
  }
  R q[m][6];
#pragma unroll
  for (int c = 0; c < m; ++c) reconstruct_component<R, m>(G, U, N, i, src, c, P, q[c]);
  const R ih = G.r(G_IH, i);
  const R ih2 = ih * ih;
  R Wxx[m], Wxy[m], Wyy[m];
#pragma unroll
  for (int c = 0; c < m; ++c) { Wxx[c] = R(2) * q[c][3] * ih2; Wxy[c] = q[c][4] * ih2; Wyy[c] = R(2) * q[c][5] * ih2; }
  R vx[3], vy[3];
#pragma unroll
  for (int v = 0; v < 3; ++v) { vx[v] = G.r(G_VX + 2 * v, i); vy[v] = G.r(G_VX + 2 * v + 1, i); }
  const R gs[2] = {R(0.5) - R(0.28867513459481288225), R(0.5) + R(0.28867513459481288225)};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int jn = (j + 1) % 3;
      const R xi = vx[j] + gs[g] * (vx[jn] - vx[j]);
      const R et = vy[j] + gs[g] * (vy[jn] - vy[j]);
      R W[m], Wx[m], Wy[m], Wt[m], Wtt[m];
#pragma unroll
      for (int c = 0; c < m; ++c) {
        W[c] = q[c][0] + xi * (q[c][1] + q[c][3] * xi + q[c][4] * et) + et * (q[c][2] + q[c][5] * et);
        Wx[c] = (q[c][1] + R(2) * q[c][3] * xi + q[c][4] * et) * ih;
        Wy[c] = (q[c][2] + q[c][4] * xi + R(2) * q[c][5] * et) * ih;
      }
      lax_wendroff<R, EQ>(W, Wx, Wy, Wxx, Wxy, Wyy, P, Wt, Wtt);
      const int qp = 2 * j + g;
#pragma unroll
      for (int c = 0; c < m; ++c) {
        Pb[(size_t)((qp * 3 + 0) * m + c) * N + i] = W[c];
        Pb[(size_t)((qp * 3 + 1) * m + c) * N + i] = Wt[c];
        Pb[(size_t)((qp * 3 + 2) * m + c) * N + i] = Wtt[c];
      }
    }
  }
}

// ---------------------------------------------------------------- flux + update
template <typename R, int EQ>
__global__ void __launch_bounds__(128) k_edge(GeoView<R> G, const R* __restrict__ U, R* __restrict__ Un,
                                               const R* __restrict__ Pb, EqParams P, DevScalars* sc,
                                               double dt_fixed) {
  constexpr int m = EqTraits<EQ>::m;
  const int N = G.N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const volatile DevScalars* vs = sc;
  if (vs->done) {
    if (i < N)
      for (int k = 0; k < 3 * m; ++k) Un[(size_t)k * N + i] = U[(size_t)k * N + i];
    return;
  }
  const double dt = dt_fixed > 0 ? dt_fixed : vs->dt;
  double local_min = __longlong_as_double(0x7ff0000000000000ll);
  if (i < N) {
    const R dtr = R(dt);
    const R tau[3] = {R(0), R(0.5) * dtr, dtr};
    const R wts[3] = {R(1.0 / 6.0), R(4.0 / 6.0), R(1.0 / 6.0)};
    R Wi[m];
#pragma unroll
    for (int c = 0; c < m; ++c) Wi[c] = U[(size_t)c * N + i];
    const int packed = G.n(I_NBE, i);
    R Racc[m], GV[m], GY[m];
#pragma unroll
    for (int c = 0; c < m; ++c) { Racc[c] = R(0); GV[c] = R(0); GY[c] = R(0); }
#pragma unroll 1
    for (int j = 0; j < 3; ++j) {
      const int nb = G.n(I_NBR + j, i);
      const int je = (packed >> (2 * j)) & 3;
      const bool left = (nb < 0) || (i < nb);
      const R nx = G.r(G_NRM + 2 * j, i), ny = G.r(G_NRM + 2 * j + 1, i);
      const R el = G.r(G_EL + j, i);
      R Wn[m];
#pragma unroll
      for (int c = 0; c < m; ++c) Wn[c] = nb >= 0 ? U[(size_t)c * N + nb] : Wi[c];
      R WbL[m], WbR[m];
#pragma unroll
      for (int c = 0; c < m; ++c) { WbL[c] = left ? Wi[c] : Wn[c]; WbR[c] = left ? Wn[c] : Wi[c]; }
      const R aL = spectral_radius_n<R, EQ>(WbL, nx, ny, P), aR = spectral_radius_n<R, EQ>(WbR, nx, ny, P);
      const R alpha = aL > aR ? aL : aR;
      // cells and point indices of the two sides, left side's Gauss-point order
      const int cl = left ? i : nb, cr = left ? (nb >= 0 ? nb : i) : i;
      const int el_ = left ? j : je;                              // left cell's local edge
      const int er_ = left ? (nb >= 0 ? je : j) : j;              // right cell's local edge
      R Fe[m], Se[m];
#pragma unroll
      for (int c = 0; c < m; ++c) { Fe[c] = R(0); Se[c] = R(0); }
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int ql = 2 * el_ + g;
        const int qr = (nb >= 0) ? 2 * er_ + (1 - g) : ql;        // boundary: W^ext = W^int
        R a0[m], a1[m], a2[m], b0[m], b1[m], b2[m];
#pragma unroll
        for (int c = 0; c < m; ++c) {
          a0[c] = Pb[(size_t)((ql * 3 + 0) * m + c) * N + cl];
          a1[c] = Pb[(size_t)((ql * 3 + 1) * m + c) * N + cl];
          a2[c] = Pb[(size_t)((ql * 3 + 2) * m + c) * N + cl];
          b0[c] = Pb[(size_t)((qr * 3 + 0) * m + c) * N + cr];
          b1[c] = Pb[(size_t)((qr * 3 + 1) * m + c) * N + cr];
          b2[c] = Pb[(size_t)((qr * 3 + 2) * m + c) * N + cr];
        }
#pragma unroll
        for (int s = 0; s < 3; ++s) {
          R WL[m], WR[m], HL[m], HR[m];
          const R hs = R(0.5) * tau[s] * tau[s];
#pragma unroll
          for (int c = 0; c < m; ++c) {
            WL[c] = a0[c] + tau[s] * a1[c] + hs * a2[c];
            WR[c] = b0[c] + tau[s] * b1[c] + hs * b2[c];
          }
          flux_n<R, EQ>(WL, nx, ny, P, HL);
          flux_n<R, EQ>(WR, nx, ny, P, HR);
#pragma unroll
          for (int c = 0; c < m; ++c) Fe[c] += wts[s] * (R(0.5) * (HR[c] + HL[c] - alpha * (WR[c] - WL[c])));
          if (s == 2) {
#pragma unroll
            for (int c = 0; c < m; ++c) Se[c] += R(0.5) * (WL[c] + WR[c]);
          }
        }
      }
      // two Gauss points of weight 1/2; the cell's outward normal is +-n
      const R sg = left ? R(0.5) * el : R(-0.5) * el;
#pragma unroll
      for (int c = 0; c < m; ++c) {
        Racc[c] += sg * Fe[c];
        GV[c] += sg * nx * Se[c];
        GY[c] += sg * ny * Se[c];
      }
    }
    R Wnew[m];
#pragma unroll
    for (int c = 0; c < m; ++c) {
      Wnew[c] = Wi[c] - dtr * Racc[c];
      Un[(size_t)(0 * m + c) * N + i] = Wnew[c];
      Un[(size_t)(1 * m + c) * N + i] = GV[c];
      Un[(size_t)(2 * m + c) * N + i] = GY[c];
    }
    if (!physical<R, EQ>(Wnew, P)) atomicOr(&sc->flags, 1u);
    const double lam = spectral_radius_all<R, EQ>(Wnew, P);
    if (lam > 0) local_min = (double)G.r(G_INR, i) / lam;
    if (!(local_min >= 0)) local_min = __longlong_as_double(0x7ff0000000000000ll);
  }
  finish_step(sc, local_min, dt, true);
}

// CFL step of the current state (after an upload or a change of target).
template <typename R, int EQ>
__global__ void __launch_bounds__(256) k_cfl(GeoView<R> G, const R* __restrict__ U, EqParams P, DevScalars* sc) {
  constexpr int m = EqTraits<EQ>::m;
  const int N = G.N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double local_min = __longlong_as_double(0x7ff0000000000000ll);
  if (i < N) {
    R W[m];
#pragma unroll
    for (int c = 0; c < m; ++c) W[c] = U[(size_t)c * N + i];
    if (!physical<R, EQ>(W, P)) atomicOr(&sc->flags, 1u);
    const double lam = spectral_radius_all<R, EQ>(W, P);
    if (lam > 0) local_min = (double)G.r(G_INR, i) / lam;
    if (!(local_min >= 0)) local_min = __longlong_as_double(0x7ff0000000000000ll);
  }
  finish_step(sc, local_min, 0.0, false);
}

// Deterministic FP64 sums of |K| Wbar_K: fixed grid, fixed tree, then one block.
template <typename R>
__global__ void __launch_bounds__(256) k_consv_partial(const R* __restrict__ U, const double* __restrict__ area, int N,
                                                        int m, double* __restrict__ partial) {
  __shared__ double sh[256];
  for (int c = 0; c < m; ++c) {
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
      s += area[i] * (double)U[(size_t)c * N + i];
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

// host order (double) -> internal order (R), and back
template <typename R>
__global__ void k_scatter_state(const double* __restrict__ host_order, const int32_t* __restrict__ perm, int N,
                                int planes, R* __restrict__ U) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int src = perm[i];
  for (int k = 0; k < planes; ++k) U[(size_t)k * N + i] = (R)host_order[(size_t)k * N + src];
}
template <typename R>
__global__ void k_gather_state(const R* __restrict__ U, const int32_t* __restrict__ perm, int N, int planes,
                               double* __restrict__ host_order) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int dst = perm[i];
  for (int k = 0; k < planes; ++k) host_order[(size_t)k * N + dst] = (double)U[(size_t)k * N + i];
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

// ---------------------------------------------------------------- launchers
namespace {
template <typename R, int EQ> void launch_recon_t(const StepArgs& a, cudaStream_t st) {
  GeoView<R> G{reinterpret_cast<const R*>(a.rgeo), a.igeo, a.N};
  k_recon<R, EQ><<<(a.N + 127) / 128, 128, 0, st>>>(G, reinterpret_cast<const R*>(a.U), reinterpret_cast<R*>(a.Pb),
                                                     a.P, a.sc);
}
template <typename R, int EQ> void launch_edge_t(const StepArgs& a, cudaStream_t st) {
  GeoView<R> G{reinterpret_cast<const R*>(a.rgeo), a.igeo, a.N};
  k_edge<R, EQ><<<(a.N + 127) / 128, 128, 0, st>>>(G, reinterpret_cast<const R*>(a.U), reinterpret_cast<R*>(a.Un),
                                                    reinterpret_cast<const R*>(a.Pb), a.P, a.sc, a.dt_fixed);
}
template <typename R, int EQ> void launch_cfl_t(const StepArgs& a, cudaStream_t st) {
  GeoView<R> G{reinterpret_cast<const R*>(a.rgeo), a.igeo, a.N};
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

void launch_recon(int prec, int eq, const StepArgs& a, cudaStream_t st) { HW_DISPATCH(launch_recon_t, prec, eq, a, st); }
void launch_edge(int prec, int eq, const StepArgs& a, cudaStream_t st) { HW_DISPATCH(launch_edge_t, prec, eq, a, st); }
void launch_step(int prec, int eq, const StepArgs& a, cudaStream_t st) {
  launch_recon(prec, eq, a, st);
  launch_edge(prec, eq, a, st);
}

void launch_cfl(int prec, int eq, const StepArgs& a, cudaStream_t st) { HW_DISPATCH(launch_cfl_t, prec, eq, a, st); }

void launch_reset(DevScalars* sc, double t, double cfl, cudaStream_t st) { k_reset<<<1, 32, 0, st>>>(sc, t, cfl); }

void launch_set_target(DevScalars* sc, double T, int has_T, cudaStream_t st) {
  k_set_target<<<1, 32, 0, st>>>(sc, T, has_T);
}

void launch_consv(int prec, const void* U, const double* area, int N, int m, double* partial, double* out,
                  cudaStream_t st) {
  if (prec == 0) k_consv_partial<double><<<kConsvBlocks, 256, 0, st>>>(reinterpret_cast<const double*>(U), area, N, m, partial);
  else k_consv_partial<float><<<kConsvBlocks, 256, 0, st>>>(reinterpret_cast<const float*>(U), area, N, m, partial);
  k_consv_final<<<1, 32, 0, st>>>(partial, kConsvBlocks, m, out);
}

void launch_scatter(int prec, const double* host_order, const int32_t* perm, int N, int planes, void* U,
                    cudaStream_t st) {
  const int nb = (N + 255) / 256;
  if (prec == 0) k_scatter_state<double><<<nb, 256, 0, st>>>(host_order, perm, N, planes, reinterpret_cast<double*>(U));
  else k_scatter_state<float><<<nb, 256, 0, st>>>(host_order, perm, N, planes, reinterpret_cast<float*>(U));
}

void launch_gather(int prec, const void* U, const int32_t* perm, int N, int planes, double* host_order,
                   cudaStream_t st) {
  const int nb = (N + 255) / 256;
  if (prec == 0) k_gather_state<double><<<nb, 256, 0, st>>>(reinterpret_cast<const double*>(U), perm, N, planes, host_order);
  else k_gather_state<float><<<nb, 256, 0, st>>>(reinterpret_cast<const float*>(U), perm, N, planes, host_order);
}

// geometry rounding (FP64 host precompute -> device precision)
__global__ void k_round_geo(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    dst[k] = (float)src[k];
}
void launch_round_geo(const double* src, float* dst, size_t n, cudaStream_t st) {
  k_round_geo<<<1184, 256, 0, st>>>(src, dst, n);
}

}  // namespace hw
