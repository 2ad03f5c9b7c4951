// Host FP64 precompute for the HWENO library: connectivity (half-edges
// grouped by their smaller vertex), Hilbert renumbering, and per-cell
// reconstruction operators of Section 2.2 (Steps 1 and 2) with the edge
// geometry of Eqs. fx and derave2d2.  The per-cell passes run on the host's
// cores; every value is computed by the same arithmetic whatever the thread
// count, so the result is bit for bit that of one thread.
#include <sched.h>
#include <sys/mman.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <system_error>
#include <thread>

#include "internal.h"

namespace hw {
namespace {

// Host threads for the precompute: the CPUs this process may run on (at most 64).
int host_threads() {
  cpu_set_t set;
  if (sched_getaffinity(0, sizeof(set), &set) == 0) {
    const int n = CPU_COUNT(&set);
    if (n > 0) return std::min(n, 64);
  }
  const unsigned n = std::thread::hardware_concurrency();
  return n ? (int)std::min(n, 64u) : 1;
}

// fn(begin, end) over consecutive ranges that cover [0, n), each on its own
// thread (the caller runs the first, and any range whose thread could not be
// started).  fn must write only outputs owned by its indices.
template <class F>
void parallel_ranges(int64_t n, const F& fn) {
  constexpr int64_t kGrain = 8192;
  const int nw = (int)std::min<int64_t>(host_threads(), (n + kGrain - 1) / kGrain);
  if (nw <= 1) {
    if (n > 0) fn(int64_t(0), n);
    return;
  }
  auto lo = [n, nw](int w) { return n * w / nw; };
  std::vector<std::thread> pool;
  int w = 1;
  try {
    pool.reserve((size_t)nw - 1);
    for (; w < nw; ++w) pool.emplace_back([&fn, &lo, w] { fn(lo(w), lo(w + 1)); });
  } catch (const std::exception&) {
    // fewer threads than ranges: the caller takes the rest below
  }
  fn(lo(0), lo(1));
  for (int r = w; r < nw; ++r) fn(lo(r), lo(r + 1));
  for (auto& t : pool) t.join();
}

// The error a one-thread pass would meet first: every range reports its own
// first failing index, and the lowest index over all ranges wins.
struct FirstError {
  std::mutex mu;
  int64_t at = LLONG_MAX;
  const char* msg = nullptr;
  void report(int64_t i, const char* m) {
    std::lock_guard<std::mutex> g(mu);
    if (i < at) { at = i; msg = m; }
  }
};

// Hilbert index of (x, y) on an n x n grid, n = 2^order: walk the quadrants
// from the coarsest level, accumulating the quadrant rank and rotating /
// reflecting the coordinates into the child's orientation.
uint64_t hilbert_key(uint32_t x, uint32_t y, int order) {
  const uint32_t n = 1u << order;
  uint64_t d = 0;
  for (uint32_t s = n >> 1; s > 0; s >>= 1) {
    const uint32_t rx = (x & s) ? 1u : 0u;
    const uint32_t ry = (y & s) ? 1u : 0u;
    d += (uint64_t)s * s * ((3u * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) { x = n - 1 - x; y = n - 1 - y; }
      const uint32_t tmp = x; x = y; y = tmp;
    }
  }
  return d;
}

// Means over a triangle (vertices X[3], Y[3]) of x, y, x^2, xy, y^2.
void tri_moments(const double* X, const double* Y, double m[5]) {
  m[0] = (X[0] + X[1] + X[2]) / 3.0;
  m[1] = (Y[0] + Y[1] + Y[2]) / 3.0;
  m[2] = (X[0] * X[0] + X[1] * X[1] + X[2] * X[2] + X[0] * X[1] + X[0] * X[2] + X[1] * X[2]) / 6.0;
  m[3] = (2.0 * (X[0] * Y[0] + X[1] * Y[1] + X[2] * Y[2]) + X[0] * Y[1] + X[1] * Y[0] + X[0] * Y[2] +
          X[2] * Y[0] + X[1] * Y[2] + X[2] * Y[1]) / 12.0;
  m[4] = (Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2] + Y[0] * Y[1] + Y[0] * Y[2] + Y[1] * Y[2]) / 6.0;
}

// Householder QR of the 5x3 matrix A (column major a[col][row]); returns Q
// (5x5, q[row][col]) and R (3x3 upper, r[row][col]).
void householder_qr_5x3(double a[3][5], double q[5][5], double r[3][3]) {
  double Q[5][5];
  for (int i = 0; i < 5; ++i) for (int j = 0; j < 5; ++j) Q[i][j] = (i == j) ? 1.0 : 0.0;
  for (int k = 0; k < 3; ++k) {
    double nrm = 0;
    for (int i = k; i < 5; ++i) nrm += a[k][i] * a[k][i];
    nrm = std::sqrt(nrm);
    double alpha = (a[k][k] > 0) ? -nrm : nrm;
    double v[5] = {0, 0, 0, 0, 0};
    for (int i = k; i < 5; ++i) v[i] = a[k][i];
    v[k] -= alpha;
    double vn = 0;
    for (int i = k; i < 5; ++i) vn += v[i] * v[i];
    if (vn > 0) {
      for (int c = k; c < 3; ++c) {  // A <- (I - 2 v v^T / v^T v) A
        double s = 0;
        for (int i = k; i < 5; ++i) s += v[i] * a[c][i];
        s *= 2.0 / vn;
        for (int i = k; i < 5; ++i) a[c][i] -= s * v[i];
      }
      for (int row = 0; row < 5; ++row) {  // Q <- Q (I - 2 v v^T / v^T v)
        double s = 0;
        for (int i = k; i < 5; ++i) s += Q[row][i] * v[i];
        s *= 2.0 / vn;
        for (int i = k; i < 5; ++i) Q[row][i] -= s * v[i];
      }
    }
  }
  for (int i = 0; i < 5; ++i) for (int j = 0; j < 5; ++j) q[i][j] = Q[i][j];
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) r[i][j] = (j >= i) ? a[j][i] : 0.0;
}

}  // namespace

std::string build_mesh(const double* xy, int64_t nv, const int32_t* tri, int64_t nt, double Lx, double Ly, int bc,
                       HostMesh& M) {
  if (nt <= 0 || nt > (int64_t)0x3fffffff) return "ntri out of range";
  M.nv = nv; M.nt = nt; M.Lx = Lx; M.Ly = Ly; M.bc = bc;
  for (int64_t i = 0; i < 3 * nt; ++i)
    if (tri[i] < 0 || tri[i] >= nv) return "vertex index out of range";
  if (bc == 0 && (Lx <= 0 || Ly <= 0)) return "periodic boundary needs Lx > 0 and Ly > 0";

  // ---- connectivity: the half-edges (3t + j, from vertex j to vertex j+1 of
  // triangle t) grouped by their smaller vertex with a counting sort, then by
  // their larger vertex inside each group; two half-edges with the same vertex
  // pair are one interior edge.  A fault is reported at the half-edge where a
  // scan in triangle order would first see it: a repeated vertex at that
  // half-edge, a triangle meeting itself at the second half-edge of a pair, a
  // non-manifold edge at the third.
  M.nbr_orig.assign(3 * nt, -1);
  M.nbe_orig.assign(3 * nt, -1);
  {
    const int64_t nh = 3 * nt;
    int64_t fault_at = LLONG_MAX;
    const char* fault = nullptr;
    auto note = [&](int64_t h, const char* msg) {
      if (h < fault_at) { fault_at = h; fault = msg; }
    };
    std::vector<int64_t> first((size_t)nv + 1, 0);
    for (int64_t h = 0; h < nh; ++h) {
      const int32_t a = tri[h], b = tri[h - h % 3 + (h % 3 + 1) % 3];
      if (a == b) note(h, "degenerate triangle");
      else ++first[(size_t)std::min(a, b) + 1];
    }
    for (int64_t v = 0; v < nv; ++v) first[(size_t)v + 1] += first[(size_t)v];
    // entries of a group in ascending half-edge order: (larger vertex, half-edge)
    std::vector<std::pair<int32_t, int64_t>> ent((size_t)first[(size_t)nv]);
    {
      std::vector<int64_t> fill(first.begin(), first.end() - 1);
      for (int64_t h = 0; h < nh; ++h) {
        const int32_t a = tri[h], b = tri[h - h % 3 + (h % 3 + 1) % 3];
        if (a != b) ent[(size_t)fill[(size_t)std::min(a, b)]++] = {std::max(a, b), h};
      }
    }
    FirstError fe;   // the groups hold half-edges in any order: each range keeps its lowest fault
    parallel_ranges(nv, [&](int64_t v0, int64_t v1) {
      int64_t at = LLONG_MAX;
      const char* msg = nullptr;
      auto note_here = [&](int64_t h, const char* m) {
        if (h < at) { at = h; msg = m; }
      };
      for (int64_t v = v0; v < v1; ++v) {
        auto* g0 = ent.data() + first[(size_t)v];
        auto* g1 = ent.data() + first[(size_t)v + 1];
        std::sort(g0, g1);   // by larger vertex, then by half-edge
        for (auto* r = g0; r < g1;) {
          auto* e = r + 1;
          while (e < g1 && e->first == r->first) ++e;
          if (e - r >= 3) note_here(r[2].second, "non-manifold edge (shared by more than two triangles)");
          if (e - r >= 2) {
            const int64_t h1 = r[0].second, h2 = r[1].second;
            const int64_t t1 = h1 / 3, t2 = h2 / 3;
            if (t1 == t2) {
              note_here(h2, "triangle is its own neighbour (mesh too coarse for its period)");
            } else {
              M.nbr_orig[h2] = (int32_t)t1; M.nbe_orig[h2] = (int32_t)(h1 % 3);
              M.nbr_orig[h1] = (int32_t)t2; M.nbe_orig[h1] = (int32_t)(h2 % 3);
            }
          }
          r = e;
        }
      }
      if (msg) fe.report(at, msg);
    });
    if (fe.msg) note(fe.at, fe.msg);
    if (fault) return fault;
    if (bc == 0)
      for (int64_t i = 0; i < nh; ++i)
        if (M.nbr_orig[i] < 0) return "open edge on a periodic mesh";
  }

  // ---- unwrapped vertex coordinates, areas, barycenters
  std::vector<double> VX(3 * nt), VY(3 * nt), A(nt), CX(nt), CY(nt);
  {
    auto near = [](double d, double L) { return L > 0 ? d - L * std::nearbyint(d / L) : d; };
    FirstError fe;
    parallel_ranges(nt, [&](int64_t t0, int64_t t1) {
      for (int64_t t = t0; t < t1; ++t) {
        const double x0 = xy[2 * tri[3 * t]], y0 = xy[2 * tri[3 * t] + 1];
        for (int v = 0; v < 3; ++v) {
          VX[3 * t + v] = x0 + near(xy[2 * tri[3 * t + v]] - x0, Lx);
          VY[3 * t + v] = y0 + near(xy[2 * tri[3 * t + v] + 1] - y0, Ly);
        }
        const double* X = &VX[3 * t]; const double* Y = &VY[3 * t];
        A[t] = 0.5 * ((X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]));
        if (!(A[t] > 0)) { fe.report(t, "triangle not counter-clockwise or degenerate"); return; }
        CX[t] = (X[0] + X[1] + X[2]) / 3.0;
        CY[t] = (Y[0] + Y[1] + Y[2]) / 3.0;
      }
    });
    if (fe.msg) return fe.msg;
  }

  // ---- Hilbert renumbering of the barycenters (sorted by key, ties by the
  // caller's index)
  {
    std::vector<double> bx(nt), by(nt);
    std::mutex mu;
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    parallel_ranges(nt, [&](int64_t t0, int64_t t1) {
      double lx0 = 1e300, lx1 = -1e300, ly0 = 1e300, ly1 = -1e300;
      for (int64_t t = t0; t < t1; ++t) {
        bx[t] = Lx > 0 ? CX[t] - Lx * std::floor(CX[t] / Lx) : CX[t];
        by[t] = Ly > 0 ? CY[t] - Ly * std::floor(CY[t] / Ly) : CY[t];
        lx0 = std::min(lx0, bx[t]); lx1 = std::max(lx1, bx[t]);
        ly0 = std::min(ly0, by[t]); ly1 = std::max(ly1, by[t]);
      }
      std::lock_guard<std::mutex> g(mu);
      x0 = std::min(x0, lx0); x1 = std::max(x1, lx1);
      y0 = std::min(y0, ly0); y1 = std::max(y1, ly1);
    });
    const int order = 16;   // keys below 4^16 = 2^32
    const double span = std::max(x1 - x0, y1 - y0) * (1 + 1e-12) + 1e-300;
    std::vector<uint64_t> key(nt);   // Hilbert key in the high word, caller's index in the low word
    parallel_ranges(nt, [&](int64_t t0, int64_t t1) {
      for (int64_t t = t0; t < t1; ++t) {
        uint32_t ix = (uint32_t)std::min(65535.0, std::floor((bx[t] - x0) / span * 65536.0));
        uint32_t iy = (uint32_t)std::min(65535.0, std::floor((by[t] - y0) / span * 65536.0));
        key[t] = (hilbert_key(ix, iy, order) << 32) | (uint64_t)t;
      }
    });
    std::sort(key.begin(), key.end());
    M.perm.resize(nt);
    M.inv.resize(nt);
    parallel_ranges(nt, [&](int64_t k0, int64_t k1) {
      for (int64_t k = k0; k < k1; ++k) M.perm[k] = (int32_t)(key[k] & 0xffffffffu);
    });
    parallel_ranges(nt, [&](int64_t k0, int64_t k1) {
      for (int64_t k = k0; k < k1; ++k) M.inv[M.perm[k]] = (int32_t)k;
    });
  }

  // ---- per-cell operators, internal order
  {
    // the largest host array (90 doubles per cell): ask for huge pages before
    // its first touch, which halves the time of the fill below (advice only)
    const size_t n = (size_t)NRGEO * nt;
    M.rgeo.reserve(n);
    const uintptr_t huge = uintptr_t(1) << 21;
    const uintptr_t a = (reinterpret_cast<uintptr_t>(M.rgeo.data()) + huge - 1) & ~(huge - 1);
    const uintptr_t e = (reinterpret_cast<uintptr_t>(M.rgeo.data()) + n * sizeof(double)) & ~(huge - 1);
    if (e > a) madvise(reinterpret_cast<void*>(a), e - a, MADV_HUGEPAGE);
  }
  M.rgeo.assign((size_t)NRGEO * nt, 0.0);
  M.igeo.assign((size_t)NIGEO * nt, -1);
  M.area.resize(nt);
  auto R = [&](int p, int64_t k) -> double& { return M.rgeo[(size_t)p * nt + k]; };
  auto I = [&](int p, int64_t k) -> int32_t& { return M.igeo[(size_t)p * nt + k]; };
  FirstError fe;
  parallel_ranges(nt, [&](int64_t k0, int64_t k1) {
  for (int64_t k = k0; k < k1; ++k) {
    const int64_t t = M.perm[k];
    const double A0 = A[t], h0 = std::sqrt(A0), ih = 1.0 / h0;
    M.area[k] = A0;
    double X0[3], Y0[3];
    for (int v = 0; v < 3; ++v) { X0[v] = (VX[3 * t + v] - CX[t]) * ih; Y0[v] = (VY[3 * t + v] - CY[t]) * ih; }
    double m0[5];
    tri_moments(X0, Y0, m0);
    const double M3 = m0[2], M4 = m0[3], M5 = m0[4];
    for (int v = 0; v < 3; ++v) { R(G_VX + 2 * v, k) = X0[v]; R(G_VX + 2 * v + 1, k) = Y0[v]; }
    R(G_MOM, k) = M3; R(G_MOM + 1, k) = M4; R(G_MOM + 2, k) = M5;
    R(G_IH, k) = ih;
    double per = 0;
    for (int j = 0; j < 3; ++j) per += std::hypot(VX[3 * t + (j + 1) % 3] - VX[3 * t + j], VY[3 * t + (j + 1) % 3] - VY[3 * t + j]);
    R(G_INR, k) = 2.0 * A0 / per;

    // stencil members in the scaled frame of K0
    double Cm[3][5], Bm[6][5], wl[3], bar[3][2];
    int packed = 0;
    for (int j = 0; j < 3; ++j) {
      const int32_t u = M.nbr_orig[3 * t + j];
      double X[3], Y[3], Au;
      if (u >= 0) {
        const double sx = Lx > 0 ? Lx * std::nearbyint((CX[t] - CX[u]) / Lx) : 0.0;
        const double sy = Ly > 0 ? Ly * std::nearbyint((CY[t] - CY[u]) / Ly) : 0.0;
        for (int v = 0; v < 3; ++v) { X[v] = (VX[3 * u + v] + sx - CX[t]) * ih; Y[v] = (VY[3 * u + v] + sy - CY[t]) * ih; }
        Au = A[u];
        I(I_NBR + j, k) = M.inv[u];
        packed |= (M.nbe_orig[3 * t + j] & 3) << (2 * j);
        if (t < u) packed |= 1 << (6 + j);   // this cell owns the edge (lower index in the caller's numbering)
      } else {
        // transmissive ghost: K0 reflected across edge j (it carries K0's data)
        const double ax = X0[j], ay = Y0[j], bx = X0[(j + 1) % 3], by = Y0[(j + 1) % 3];
        const double dx = bx - ax, dy = by - ay, dd = dx * dx + dy * dy;
        for (int v = 0; v < 3; ++v) {
          const double px = X0[v] - ax, py = Y0[v] - ay, s = (px * dx + py * dy) / dd;
          X[v] = ax + 2.0 * s * dx - px; Y[v] = ay + 2.0 * s * dy - py;
        }
        Au = A0;
        I(I_NBR + j, k) = -1;
        packed |= 1 << (6 + j);   // a boundary edge belongs to its cell
      }
      double mu[5];
      tri_moments(X, Y, mu);
      Cm[j][0] = mu[0]; Cm[j][1] = mu[1];
      Cm[j][2] = mu[2] - M3; Cm[j][3] = mu[3] - M4; Cm[j][4] = mu[4] - M5;
      bar[j][0] = mu[0]; bar[j][1] = mu[1];
      wl[j] = Au / (Au + A0);
      // least-squares rows: mean over K_l + K_0 of d/dxi and d/deta of the basis
      const double ux = wl[j] * mu[0], uy = wl[j] * mu[1];
      const double rx[5] = {1.0, 0.0, 2.0 * ux, uy, 0.0};
      const double ry[5] = {0.0, 1.0, 0.0, ux, 2.0 * uy};
      for (int c = 0; c < 5; ++c) { Bm[2 * j][c] = rx[c]; Bm[2 * j + 1][c] = ry[c]; }
      R(G_W + j, k) = wl[j];
    }
    I(I_NBE, k) = packed;

    // Step 1 (constrained least squares) by the null-space method:
    // C^T = Q R, c = Q1 R1^{-T} e + N z, z = (H^T H)^{-1} H^T (d - B c_p), H = B N.
    double a[3][5], Q[5][5], Rr[3][3];
    for (int j = 0; j < 3; ++j) for (int c = 0; c < 5; ++c) a[j][c] = Cm[j][c];
    householder_qr_5x3(a, Q, Rr);
    double rmax = 0, rmin = 1e300;
    for (int i = 0; i < 3; ++i) { rmax = std::max(rmax, std::fabs(Rr[i][i])); rmin = std::min(rmin, std::fabs(Rr[i][i])); }
    if (!(rmin > 1e-10 * rmax)) { fe.report(k, "ill-conditioned stencil (cell-average constraints)"); return; }
    // P0 = Q1 R1^{-T}  (5x3): solve R1^T y = e_i for unit e_i
    double Rinvt[3][3];
    for (int i = 0; i < 3; ++i) {
      double y[3];
      for (int r = 0; r < 3; ++r) {
        double s = (r == i) ? 1.0 : 0.0;
        for (int c = 0; c < r; ++c) s -= Rr[c][r] * y[c];
        y[r] = s / Rr[r][r];
      }
      for (int r = 0; r < 3; ++r) Rinvt[r][i] = y[r];
    }
    double P0[5][3];
    for (int r = 0; r < 5; ++r)
      for (int i = 0; i < 3; ++i) {
        double s = 0;
        for (int c = 0; c < 3; ++c) s += Q[r][c] * Rinvt[c][i];
        P0[r][i] = s;
      }
    double Nn[5][2];
    for (int r = 0; r < 5; ++r) { Nn[r][0] = Q[r][3]; Nn[r][1] = Q[r][4]; }
    double H[6][2];
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 2; ++c) {
        double s = 0;
        for (int q = 0; q < 5; ++q) s += Bm[r][q] * Nn[q][c];
        H[r][c] = s;
      }
    double HtH[2][2] = {{0, 0}, {0, 0}};
    for (int r = 0; r < 6; ++r)
      for (int i = 0; i < 2; ++i) for (int j2 = 0; j2 < 2; ++j2) HtH[i][j2] += H[r][i] * H[r][j2];
    const double det = HtH[0][0] * HtH[1][1] - HtH[0][1] * HtH[1][0];
    if (!(det > 1e-12 * (HtH[0][0] * HtH[1][1] + 1e-300))) {
      fe.report(k, "ill-conditioned stencil (least-squares rows)");
      return;
    }
    const double G[2][2] = {{HtH[1][1] / det, -HtH[0][1] / det}, {-HtH[1][0] / det, HtH[0][0] / det}};
    // K = N G H^T  (5x6)
    double Kd[5][6];
    for (int r = 0; r < 5; ++r)
      for (int c = 0; c < 6; ++c) {
        double s = 0;
        for (int i = 0; i < 2; ++i) for (int j2 = 0; j2 < 2; ++j2) s += Nn[r][i] * G[i][j2] * H[c][j2];
        Kd[r][c] = s;
      }
    // Me = (I - K B) P0  (5x3)
    double Me[5][3];
    for (int r = 0; r < 5; ++r)
      for (int i = 0; i < 3; ++i) {
        double s = P0[r][i];
        for (int c = 0; c < 6; ++c) {
          double bp = 0;
          for (int q = 0; q < 5; ++q) bp += Bm[c][q] * P0[q][i];
          s -= Kd[r][c] * bp;
        }
        Me[r][i] = s;
      }
    for (int r = 0; r < 5; ++r) {
      for (int i = 0; i < 3; ++i) R(G_M1 + r * 9 + i, k) = Me[r][i];
      for (int c = 0; c < 6; ++c) R(G_M1 + r * 9 + 3 + c, k) = Kd[r][c] * h0;
    }

    // Step 2: p_l = Wbar_0 + b1 xi + b2 eta, least squares on
    // [xibar_l, etabar_l] b = dW, b1 = h0 Vbar_l, b2 = h0 Ybar_l.
    for (int j = 0; j < 3; ++j) {
      const double xb = bar[j][0], eb = bar[j][1];
      const double dn = 1.0 + xb * xb + eb * eb;
      const double inv[2][2] = {{(1.0 + eb * eb) / dn, -xb * eb / dn}, {-xb * eb / dn, (1.0 + xb * xb) / dn}};
      const double Gt[2][3] = {{xb, 1.0, 0.0}, {eb, 0.0, 1.0}};
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
          double s = inv[r][0] * Gt[0][c] + inv[r][1] * Gt[1][c];
          if (c > 0) s *= h0;
          R(G_P + j * 6 + r * 3 + c, k) = s;
        }
    }
  }
  });
  if (fe.msg) return fe.msg;

  // ---- perimeter / area of each cell and of its neighbours (one FP64 value per
  // cell, so that both cells of an edge see the same numbers)
  {
    std::vector<double> pk(nt);
    parallel_ranges(nt, [&](int64_t t0, int64_t t1) {
      for (int64_t t = t0; t < t1; ++t) {
        double per = 0;
        for (int j = 0; j < 3; ++j)
          per += std::hypot(VX[3 * t + (j + 1) % 3] - VX[3 * t + j], VY[3 * t + (j + 1) % 3] - VY[3 * t + j]);
        pk[t] = per / A[t];
      }
    });
    parallel_ranges(nt, [&](int64_t k0, int64_t k1) {
      for (int64_t k = k0; k < k1; ++k) {
        const int64_t t = M.perm[k];
        R(G_PK, k) = pk[t];
        for (int j = 0; j < 3; ++j) {
          const int32_t u = M.nbr_orig[3 * t + j];
          R(G_PN + j, k) = u >= 0 ? pk[u] : pk[t];
        }
      }
    });
  }

  // ---- edge geometry: canonical normal, outward of the edge's owner, the
  // cell with the lower index in the caller's numbering, and computed in the
  // owner's frame: every edge gets one normal and one length whatever the
  // renumbering (on a periodic seam the two cells' frames differ by a shift
  // that is not exact in floating point)
  parallel_ranges(nt, [&](int64_t k0, int64_t k1) {
  for (int64_t k = k0; k < k1; ++k) {
    const int64_t t = M.perm[k];
    for (int j = 0; j < 3; ++j) {
      const int32_t un = I(I_NBR + j, k);
      const bool left = (un < 0) || (t < M.perm[un]);
      int64_t owner = left ? t : M.perm[un];
      int jo = left ? j : M.nbe_orig[3 * t + j];
      const double ax = VX[3 * owner + jo], ay = VY[3 * owner + jo];
      const double bx = VX[3 * owner + (jo + 1) % 3], by = VY[3 * owner + (jo + 1) % 3];
      const double len = std::hypot(bx - ax, by - ay);
      R(G_NRM + 2 * j, k) = (by - ay) / len;
      R(G_NRM + 2 * j + 1, k) = -(bx - ax) / len;
      R(G_EL + j, k) = len / A[t];
    }
  }
  });
  return "";
}

}  // namespace hw
