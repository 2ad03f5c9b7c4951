// Internal declarations shared by the host precompute, the kernels and the
// C-ABI layer of the HWENO library (not part of the public interface).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace hw {

// ---------------------------------------------------------------- geometry planes
// Per-cell real-valued geometry, structure of arrays: plane p of cell i lives
// at rgeo[p * ntri + i] (cells in Hilbert order).  Built in FP64 on the host,
// stored on the device in the solver's precision.
enum RGeo : int {
  G_M1 = 0,    // 45: Step-1 operator, c_r = sum_k M1[r][k] * rhs_k, r = 0..4 (coefficients of
               //     xi, eta, xi^2-M3, xi*eta-M4, eta^2-M5), k = 0..8:
               //     (Wbar_l - Wbar_0, l = 1..3), then per l: x-row, y-row right-hand
               //     sides (Vbar_0 + w_l (Vbar_l - Vbar_0)), h0 folded into the operator
  G_W = 45,    // 3: w_l = |K_l| / (|K_l| + |K_0|)
  G_P = 48,    // 18: Step-2 operators, b_r = sum_k P[l][r][k] * (Wbar_l - Wbar_0, Vbar_l, Ybar_l), h0 folded
  G_VX = 66,   // 6: vertices in the scaled frame (xi_v, eta_v), v = 0..2
  G_MOM = 72,  // 3: M3, M4, M5 = K0 means of xi^2, xi*eta, eta^2
  G_IH = 75,   // 1: 1 / h0
  G_NRM = 76,  // 6: canonical unit normal of local edge j (outward of the lower-numbered cell)
  G_EL = 82,   // 3: |e_j| / |K|
  G_INR = 85,  // 1: inradius 2|K| / perimeter
  G_PK = 86,   // 1: perimeter / |K| of the cell        } positivity-preserving flux blending
  G_PN = 87,   // 3: perimeter / |K| of the neighbour    } (scale limiter on); the ghost of a
               //    across local edge j                 } boundary edge is the cell itself
  NRGEO = 90
};
// Planes of the step without the scale limiter (and of the adjoint step).
constexpr int kStepPlanes = G_INR + 1;
// Per-cell integer planes.
enum IGeo : int {
  I_NBR = 0,   // 3: neighbour across local edge j (internal numbering), -1 on a boundary
  I_NBE = 3,   // 1: packed: bits 2j, 2j+1: the neighbour's local index of edge j; bit 6 + j: this cell
               //    owns edge j (lower index in the caller's numbering, or a boundary edge); bits
               //    9 + 2j, 10 + 2j: the ghost of a boundary edge j (0 transmissive, 1 wall, 2 inflow)
  NIGEO = 4
};

struct HostMesh {
  int64_t nv = 0, nt = 0;
  double Lx = 0, Ly = 0;
  int bc = 0;
  std::vector<int32_t> perm;      // perm[k] = caller's index of internal cell k
  std::vector<int32_t> inv;       // inv[caller index] = internal index
  std::vector<int32_t> nbr_orig;  // [nt*3] caller numbering
  std::vector<int32_t> nbe_orig;  // [nt*3]
  std::vector<double> rgeo;       // [NRGEO * nt], internal order
  std::vector<int32_t> igeo;      // [NIGEO * nt]
  std::vector<double> area;       // [nt] internal order
  bool special_bc = false;        // some boundary edge is a wall or an inflow edge
};

// Builds everything above; returns an error message or "" on success.
std::string build_mesh(const double* xy, int64_t nv, const int32_t* tri, int64_t nt, double Lx, double Ly, int bc,
                       HostMesh& M);

}  // namespace hw

// Opaque mesh handle of the C ABI.
struct hw_mesh {
  hw::HostMesh M;
};

// Records the message returned by hw_last_error() on this thread.
void hw_set_last_error_internal(const char* msg);
