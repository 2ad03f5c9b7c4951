// C ABI of the HWENO library (declared in include/hweno.h): mesh handles,
// caller-owned device workspace, state I/O in the caller's numbering, single
// steps, and run_to through a captured CUDA graph of several steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hweno.h"
#include "internal.h"
#include "nvtx.h"
#include "state_rows.h"
#include "kernels.h"

using namespace hw;

namespace {
thread_local std::string g_last_error;

hw_status fail(hw_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define HW_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(HW_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr int kGraphSteps = 16;  // steps per captured graph (even: the state parity is preserved)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t rgeo, igeo, U0, U1, Pb, comp, comp_bytes, area, perm, stage, sc, partial, consv, fslot, fhoff, fhalo;
  size_t oedges, EP, EP_bytes, total;
};

// Tile shape of the fused step in a precision.
int fused_tile(int prec) { return prec == HW_FP32 ? kFusedTile32 : kFusedTile64; }
int fused_halo_cap(int prec) { return prec == HW_FP32 ? kFusedHalo32 : kFusedHalo64; }

// The flux phase evaluates each edge once (step_kernels 3, and the default
// in FP64, where the FP64 pipe bounds the step and the halved flux arithmetic
// pays; in FP32 the two-sided k_edge is faster): edge list and per-point flux
// buffer in the workspace.
bool edge_once_mode(const hw_options* o, int prec) {
  return o->step_kernels == 3 || (o->step_kernels == 0 && prec == HW_FP64);
}

Layout make_layout(int64_t N, int m, int prec, bool edge_once) {
  const size_t s = prec == HW_FP64 ? 8 : 4;
  const size_t ld = (size_t)padded_cells(N);   // plane stride
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
  L.rgeo = take((size_t)NRGEO * ld * s);
  L.igeo = take((size_t)NIGEO * ld * 4);
  L.U0 = take((size_t)3 * m * ld * s);
  L.U1 = take((size_t)3 * m * ld * s);
  L.Pb = take((size_t)18 * m * ld * s);
  // FP32 form: compensation of the cell averages (compensated summation of the updates)
  L.comp_bytes = prec == HW_FP32 ? (size_t)m * ld * 4 : 0;
  L.comp = take(L.comp_bytes);
  L.area = take((size_t)N * 8);
  L.perm = take((size_t)N * 4);
  L.stage = take((size_t)3 * m * N * 8);
  L.sc = take(sizeof(DevScalars));
  L.partial = take((size_t)kConsvBlocks * 4 * 8);
  L.consv = take(4 * 8);
  // tables of the fused step: neighbour slots per cell, halo offsets and cells per tile
  const size_t ntiles = (size_t)((N + fused_tile(prec) - 1) / fused_tile(prec));
  L.fslot = take(ld * 4);
  L.fhoff = take((ntiles + 1) * 4);
  L.fhalo = take(ntiles * (size_t)fused_halo_cap(prec) * 4);
  // edge-once flux phase: owned edges (at most 3 per cell) and [ld][6][2m] values
  L.oedges = take(edge_once ? (size_t)3 * N * 4 : 0);
  L.EP_bytes = edge_once ? (size_t)12 * m * ld * s : 0;
  L.EP = take(L.EP_bytes);
  L.total = o;
  return L;
}

// Tables of the fused step for tiles of TT consecutive internal cells: the
// halo of each tile (cells outside it that share an edge with one of its
// cells, ascending) and per cell the packed slots of its three neighbours.
// Returns false (tables unusable) if a tile's halo exceeds HC cells.
bool build_fused_tables(const HostMesh& M, int TT, int HC, std::vector<int32_t>& slot, std::vector<int32_t>& off,
                        std::vector<int32_t>& halo) {
  const int64_t nt = M.nt, ntiles = (nt + TT - 1) / TT;
  slot.assign((size_t)nt, 0);
  off.assign((size_t)ntiles + 1, 0);
  halo.clear();
  std::vector<int32_t> loc;
  for (int64_t b = 0; b < ntiles; ++b) {
    const int64_t c0 = b * TT, c1 = std::min<int64_t>(nt, c0 + TT);
    loc.clear();
    for (int64_t k = c0; k < c1; ++k)
      for (int j = 0; j < 3; ++j) {
        const int32_t u = M.igeo[(size_t)(I_NBR + j) * nt + k];
        if (u >= 0 && (u < c0 || u >= c1)) loc.push_back(u);
      }
    std::sort(loc.begin(), loc.end());
    loc.erase(std::unique(loc.begin(), loc.end()), loc.end());
    if ((int)loc.size() > HC) return false;
    off[(size_t)b] = (int32_t)halo.size();
    halo.insert(halo.end(), loc.begin(), loc.end());
    for (int64_t k = c0; k < c1; ++k) {
      int32_t packed = 0;
      for (int j = 0; j < 3; ++j) {
        const int32_t u = M.igeo[(size_t)(I_NBR + j) * nt + k];
        int v = kSlotNone;
        if (u >= c0 && u < c1) v = (int)(u - c0);
        else if (u >= 0) v = TT + (int)(std::lower_bound(loc.begin(), loc.end(), u) - loc.begin());
        packed |= v << (kSlotBits * j);
      }
      slot[(size_t)k] = packed;
    }
  }
  off[(size_t)ntiles] = (int32_t)halo.size();
  return true;
}

int ncomp(int eq) { return eq == HW_EULER ? 4 : 1; }

hw_status check_options(const hw_options* o) {
  if (!o) return fail(HW_EINVAL, "options is NULL");
  if (o->eq < 0 || o->eq > 2) return fail(HW_EINVAL, "unknown equation");
  if (!(o->cfl > 0)) return fail(HW_EINVAL, "cfl must be positive");
  if (o->eq == HW_EULER && !(o->gamma_gas > 1)) return fail(HW_EINVAL, "gamma_gas must exceed 1");
  // Section 2.2, Step 3: the linear weights are positive and sum to one
  double gsum = 0.0;
  for (int l = 0; l < 4; ++l) {
    if (!(o->gamma_lin[l] > 0)) return fail(HW_EINVAL, "every linear weight gamma_l must be positive");
    gsum += o->gamma_lin[l];
  }
  if (!(std::fabs(gsum - 1.0) <= 1e-12)) return fail(HW_EINVAL, "the linear weights must sum to 1");
  if (!(o->eps > 0)) return fail(HW_EINVAL, "eps must be positive");
  if (o->positivity != 0 && o->positivity != 1) return fail(HW_EINVAL, "positivity must be 0 or 1");
  if (o->time_rule != 0 && o->time_rule != 1) return fail(HW_EINVAL, "time_rule must be 0 or 1");
  if (o->time_rule == 1 && o->positivity)
    return fail(HW_EINVAL, "the Gauss-Legendre time rule is not combined with the scale limiter");
  if (o->step_kernels < 0 || o->step_kernels > 3) return fail(HW_EINVAL, "step_kernels must be 0, 1, 2 or 3");
  return HW_OK;
}
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// 2-D TMA descriptor over `rows` planes of N cells with plane stride ld
// elements; box = kCells cells x all rows; out-of-range cells read as zero.
hw_status encode_planes(CUtensorMap* map, CUtensorMapDataType dt, size_t esize, void* base, int64_t N, int rows,
                        int64_t ld) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return fail(HW_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
  const cuuint32_t box[2] = {(cuuint32_t)kCells, (cuuint32_t)rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HW_ECUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return HW_OK;
}
}  // namespace

namespace {
// Device address of the static scratch array of hw_step_static_scratch on the
// current device (defined with the array below).
hw_status static_scratch_address(void** out);
}  // namespace

void hw_set_last_error_internal(const char* msg) { g_last_error = msg ? msg : ""; }

// TMA descriptors of the geometry and index planes (shared with batches).
hw_status hw_encode_plane_maps(TensorMaps* maps, int precision, char* rgeo, char* igeo, int64_t N, int64_t ld) {
  const size_t es = precision == HW_FP64 ? 8 : 4;
  const CUtensorMapDataType dt = precision == HW_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  hw_status st = encode_planes(&maps->geo, dt, es, rgeo, N, kReconPlanes, ld);
  if (st == HW_OK) st = encode_planes(&maps->egeo, dt, es, rgeo + (size_t)G_NRM * (size_t)ld * es, N, kEdgePlanes, ld);
  if (st == HW_OK) st = encode_planes(&maps->idx, CU_TENSOR_MAP_DATA_TYPE_INT32, 4, igeo, N, NIGEO, ld);
  if (st == HW_OK) st = encode_planes(&maps->lgeo, dt, es, rgeo + (size_t)G_PK * (size_t)ld * es, N, kLimPlanes, ld);
  return st;
}

struct hw_solver {
  hw_options opt;
  int prec = 0, eq = 0, m = 1;
  int64_t N = 0;
  int64_t ld = 0;  // plane stride (cells, multiple of kCells)
  TensorMaps maps{};
  char* ws = nullptr;
  Layout L{};
  int cur = 0;  // index of the current state buffer
  bool special_bc = false;   // the mesh has walls or inflow edges
  bool fused = false;        // steps run the fused reconstruct-and-flux kernel
  int fused_ntiles = 0;      // tiles of the fused step (0: tables not available)
  int n_oedges = 0;          // edges of the edge-once flux phase (0: that phase is off)
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  DevScalars* h_sc = nullptr;  // pinned mirror for readback
  double* h_consv = nullptr;
  // per-kernel event timing (hw_profile)
  bool profiling = false;
  std::vector<cudaEvent_t> ev;  // 3 per profiled step: before recon, between, after edge
  int64_t nprof = 0;

  void* U(int k) { return ws + (k == 0 ? L.U0 : L.U1); }
  DevScalars* sc() { return reinterpret_cast<DevScalars*>(ws + L.sc); }
  void* comp() { return L.comp_bytes ? ws + L.comp : nullptr; }
  hw_status clear_comp() {
    if (L.comp_bytes) HW_CUDA(cudaMemsetAsync(ws + L.comp, 0, L.comp_bytes, stream));
    return HW_OK;
  }
  StepArgs args(int from, double dt_fixed) {
    StepArgs a{};
    a.rgeo = ws + L.rgeo;
    a.igeo = reinterpret_cast<const int32_t*>(ws + L.igeo);
    a.N = (int)N;
    a.ld = (int)ld;
    a.from = from;
    a.maps = &maps;
    a.tiles = TileSet{nullptr, (int)((N + kCells - 1) / kCells)};
    a.U = U(from);
    a.Un = U(1 - from);
    a.Pb = ws + L.Pb;
    a.C = comp();
    a.sc = sc();
    a.dt_fixed = dt_fixed;
    a.P.ax = opt.ax; a.P.ay = opt.ay; a.P.gam = opt.gamma_gas; a.P.eps = opt.eps;
    a.P.positivity = (opt.eq == HW_EULER && opt.positivity) ? 1 : 0;
    a.P.time_rule = opt.time_rule;
    for (int l = 0; l < 4; ++l) { a.P.g[l] = opt.gamma_lin[l]; a.P.win[l] = opt.inflow[l]; }
    eq_params_finish(a.P);
    a.fused = FusedTiles{reinterpret_cast<const int32_t*>(ws + L.fslot), reinterpret_cast<const int32_t*>(ws + L.fhoff),
                         reinterpret_cast<const int32_t*>(ws + L.fhalo), fused_ntiles};
    a.oedges = reinterpret_cast<const int32_t*>(ws + L.oedges);
    a.n_oedges = n_oedges;
    a.EP = n_oedges > 0 ? ws + L.EP : nullptr;
    return a;
  }
  // one step on stream st: the fused kernel, or reconstruction then flux
  void launch(const StepArgs& a, cudaStream_t st) {
    if (fused) launch_fused(prec, eq, a, st);
    else launch_step(prec, eq, a, st);
  }
};

extern "C" {

const char* hw_last_error(void) { return g_last_error.c_str(); }

void hw_options_default(hw_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->eq = HW_ADVECTION;
  o->ax = 1.0; o->ay = 1.0;
  o->gamma_gas = 1.4;
  o->cfl = 0.5;
  o->gamma_lin[0] = 0.94; o->gamma_lin[1] = 0.02; o->gamma_lin[2] = 0.02; o->gamma_lin[3] = 0.02;
  o->eps = 1e-8;
  o->inflow[0] = 1.0; o->inflow[3] = 2.5;   // rest state, rho = 1, p = 1 (gamma 1.4)
}

hw_status hw_mesh_create(const double* xy, int64_t nvert, const int32_t* tri, int64_t ntri, double Lx, double Ly,
                         int32_t bc, hw_mesh** out) {
  hw::NvtxRange nvtx_("hw_mesh_create");
  if (!xy || !tri || !out || nvert <= 0 || ntri <= 0) return fail(HW_EINVAL, "null pointer or empty mesh");
  if (bc != HW_BC_PERIODIC && bc != HW_BC_TRANSMISSIVE) return fail(HW_EINVAL, "unknown boundary condition");
  hw_mesh* h = new (std::nothrow) hw_mesh();
  if (!h) return fail(HW_ENOMEM, "host allocation failed");
  std::string err;
  try {
    err = build_mesh(xy, nvert, tri, ntri, Lx, Ly, bc, h->M);
  } catch (const std::bad_alloc&) {
    delete h;
    return fail(HW_ENOMEM, "host allocation failed while building the mesh");
  }
  if (!err.empty()) {
    delete h;
    const bool inval = err.find("out of range") != std::string::npos || err.find("needs") != std::string::npos;
    return fail(inval ? HW_EINVAL : HW_EMESH, err);
  }
  *out = h;
  return HW_OK;
}

hw_status hw_mesh_set_boundary(hw_mesh* mesh, const int32_t* edge_bc) {
  if (!mesh || !edge_bc) return fail(HW_EINVAL, "null pointer");
  HostMesh& M = mesh->M;
  const int64_t nt = M.nt;
  for (int64_t t = 0; t < nt; ++t)
    for (int j = 0; j < 3; ++j)
      if (M.nbr_orig[3 * t + j] < 0) {
        const int b = edge_bc[3 * t + j];
        if (b != HW_BC_TRANSMISSIVE && b != HW_BC_REFLECTIVE && b != HW_BC_INFLOW)
          return fail(HW_EINVAL, "boundary edges take HW_BC_TRANSMISSIVE, HW_BC_REFLECTIVE or HW_BC_INFLOW");
      }
  bool special = false;
  for (int64_t t = 0; t < nt; ++t) {
    int32_t& packed = M.igeo[(size_t)I_NBE * nt + M.inv[t]];
    for (int j = 0; j < 3; ++j) {
      packed &= ~(3 << (9 + 2 * j));
      if (M.nbr_orig[3 * t + j] >= 0) continue;
      const int code = edge_bc[3 * t + j] - HW_BC_TRANSMISSIVE;   // 0 transmissive, 1 wall, 2 inflow
      packed |= code << (9 + 2 * j);
      special = special || code != 0;
    }
  }
  M.special_bc = special;
  return HW_OK;
}

hw_status hw_mesh_destroy(hw_mesh* mesh) {
  delete mesh;
  return HW_OK;
}

int64_t hw_mesh_ntri(const hw_mesh* mesh) { return mesh ? mesh->M.nt : -1; }

hw_status hw_mesh_neighbors(const hw_mesh* mesh, int32_t* nbr, int32_t* nbe) {
  if (!mesh || !nbr) return fail(HW_EINVAL, "null pointer");
  std::memcpy(nbr, mesh->M.nbr_orig.data(), mesh->M.nbr_orig.size() * sizeof(int32_t));
  if (nbe) std::memcpy(nbe, mesh->M.nbe_orig.data(), mesh->M.nbe_orig.size() * sizeof(int32_t));
  return HW_OK;
}

hw_status hw_mesh_permutation(const hw_mesh* mesh, int32_t* perm) {
  if (!mesh || !perm) return fail(HW_EINVAL, "null pointer");
  std::memcpy(perm, mesh->M.perm.data(), mesh->M.perm.size() * sizeof(int32_t));
  return HW_OK;
}

hw_status hw_workspace_bytes(const hw_mesh* mesh, const hw_options* opt, int32_t precision, size_t* bytes) {
  if (!mesh || !bytes) return fail(HW_EINVAL, "null pointer");
  if (hw_status s = check_options(opt)) return s;
  if (precision != HW_FP64 && precision != HW_FP32) return fail(HW_EINVAL, "unknown precision");
  *bytes = make_layout(mesh->M.nt, ncomp(opt->eq), precision, edge_once_mode(opt, precision)).total;
  return HW_OK;
}

static hw_status upload_state(hw_solver* s, const double* W, const double* V, const double* Y, double t) {
  const size_t plane = (size_t)s->m * s->N * sizeof(double);
  double* stage = reinterpret_cast<double*>(s->ws + s->L.stage);
  HW_CUDA(cudaMemcpyAsync(stage, W, plane, cudaMemcpyHostToDevice, s->stream));
  HW_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(stage) + plane, V, plane, cudaMemcpyHostToDevice, s->stream));
  HW_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(stage) + 2 * plane, Y, plane, cudaMemcpyHostToDevice, s->stream));
  launch_scatter(s->prec, stage, reinterpret_cast<const int32_t*>(s->ws + s->L.perm), (int)s->N, (int)s->ld,
                 3 * s->m, s->U(s->cur), s->stream);
  if (hw_status st = s->clear_comp()) return st;
  launch_reset(s->sc(), t, s->opt.cfl, s->stream);
  launch_cfl(s->prec, s->eq, s->args(s->cur, 0.0), s->stream);
  HW_CUDA(cudaGetLastError());
  return HW_OK;
}

hw_status hw_state_init(const hw_mesh* mesh, const hw_options* opt, int32_t precision, const double* Wbar,
                        const double* Vbar, const double* Ybar, void* workspace, size_t workspace_bytes,
                        void* cuda_stream, hw_solver** out) {
  hw::NvtxRange nvtx_("hw_state_init");
  if (!mesh || !Wbar || !Vbar || !Ybar || !workspace || !out) return fail(HW_EINVAL, "null pointer");
  if (hw_status st = check_options(opt)) return st;
  if (precision != HW_FP64 && precision != HW_FP32) return fail(HW_EINVAL, "unknown precision");
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(HW_EINVAL, "workspace must be 256-byte aligned");
  const HostMesh& M = mesh->M;
  hw_solver* s = new (std::nothrow) hw_solver();
  if (!s) return fail(HW_ENOMEM, "host allocation failed");
  s->opt = *opt;
  s->prec = precision;
  s->eq = opt->eq;
  s->m = ncomp(opt->eq);
  s->N = M.nt;
  s->ld = padded_cells(M.nt);
  s->special_bc = M.special_bc;
  s->L = make_layout(M.nt, s->m, precision, edge_once_mode(opt, precision));
  if (workspace_bytes < s->L.total) { delete s; return fail(HW_ENOMEM, "workspace smaller than hw_workspace_bytes"); }
  s->ws = static_cast<char*>(workspace);
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  auto bail = [&](hw_status st) { hw_solver_destroy(s); return st; };
  if (cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost(&s->h_sc, sizeof(DevScalars)) != cudaSuccess ||
      cudaMallocHost(&s->h_consv, 4 * sizeof(double)) != cudaSuccess)
    return bail(fail(HW_ECUDA, "stream / pinned host buffer creation failed"));
  // geometry in the solver precision, planes of stride ld
  const size_t nt = (size_t)M.nt, ld = (size_t)s->ld;
  cudaError_t e;
  if (precision == HW_FP64) {
    e = cudaMemcpy2DAsync(s->ws + s->L.rgeo, ld * 8, M.rgeo.data(), nt * 8, nt * 8, NRGEO, cudaMemcpyHostToDevice,
                          s->stream);
  } else {
    std::vector<float> tmp((size_t)NRGEO * nt);
    for (size_t k = 0; k < tmp.size(); ++k) tmp[k] = (float)M.rgeo[k];
    e = cudaMemcpy2DAsync(s->ws + s->L.rgeo, ld * 4, tmp.data(), nt * 4, nt * 4, NRGEO, cudaMemcpyHostToDevice,
                          s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(s->ws + s->L.igeo, ld * 4, M.igeo.data(), nt * 4, nt * 4, NIGEO, cudaMemcpyHostToDevice,
                          s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->ws + s->L.area, M.area.data(), nt * 8, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->ws + s->L.perm, M.perm.data(), nt * 4, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return bail(fail(HW_ECUDA, std::string("geometry upload: ") + cudaGetErrorString(e)));
  // TMA descriptors of the workspace
  if (hw_status st = hw_encode_plane_maps(&s->maps, precision, s->ws + s->L.rgeo, s->ws + s->L.igeo, M.nt, s->ld))
    return bail(st);
  prepare_step_kernels(precision, s->eq);
  // fused step (step_kernels 2): tables for tiles of fused_tile(precision) cells
  {
    std::vector<int32_t> slot, off, halo;
    const bool ok = build_fused_tables(M, fused_tile(precision), fused_halo_cap(precision), slot, off, halo);
    if (s->opt.step_kernels == 2 && !ok)
      return bail(fail(HW_EINVAL, "the fused step needs every tile's halo to fit its capacity; use step_kernels 1"));
    if (ok) {
      e = cudaMemcpyAsync(s->ws + s->L.fslot, slot.data(), slot.size() * 4, cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->ws + s->L.fhoff, off.data(), off.size() * 4, cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess && !halo.empty())
        e = cudaMemcpyAsync(s->ws + s->L.fhalo, halo.data(), halo.size() * 4, cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);   // the host tables go out of scope
      if (e != cudaSuccess) return bail(fail(HW_ECUDA, std::string("fused tables: ") + cudaGetErrorString(e)));
      s->fused_ntiles = (int)(off.size() - 1);
      s->fused = s->opt.step_kernels == 2;
      if (s->fused) prepare_fused_kernel(precision, s->eq);
    }
  }
  // edge-once flux phase (step_kernels 3): every edge once, by its left cell
  if (edge_once_mode(&s->opt, precision)) {
    if (M.nt >= (int64_t(1) << 29)) return bail(fail(HW_EINVAL, "the edge-once flux phase takes fewer than 2^29 cells"));
    std::vector<int32_t> oedges;
    oedges.reserve((size_t)3 * M.nt);
    const int32_t* nbe = M.igeo.data() + (size_t)I_NBE * M.nt;
    for (int64_t i = 0; i < M.nt; ++i)
      for (int j = 0; j < 3; ++j)
        if ((nbe[i] >> (6 + j)) & 1) oedges.push_back((int32_t)(i * 4 + j));
    if (!oedges.empty()) {
      e = cudaMemcpyAsync(s->ws + s->L.oedges, oedges.data(), oedges.size() * 4, cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);   // the host list goes out of scope
      if (e != cudaSuccess) return bail(fail(HW_ECUDA, std::string("edge list: ") + cudaGetErrorString(e)));
    }
    s->n_oedges = (int)oedges.size();
    prepare_edge_once_kernels(precision, s->eq);
  }
  // Look up the static scratch array of hw_step_static_scratch on this device
  // now: the lookup loads the module that holds the array, which commits its
  // memory, so that a later step without caller scratch allocates nothing.
  void* scratch = nullptr;
  if (hw_status st = static_scratch_address(&scratch)) return bail(st);
  s->cur = 0;
  if (hw_status st = upload_state(s, Wbar, Vbar, Ybar, 0.0)) return bail(st);
  if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
    return bail(fail(HW_ECUDA, std::string("state_init: ") + cudaGetErrorString(e)));
  *out = s;
  return HW_OK;
}

hw_status hw_set_state(hw_solver* s, const double* Wbar, const double* Vbar, const double* Ybar, double t) {
  hw::NvtxRange nvtx_("hw_set_state");
  if (!s || !Wbar || !Vbar || !Ybar) return fail(HW_EINVAL, "null pointer");
  return upload_state(s, Wbar, Vbar, Ybar, t);
}

constexpr int64_t kMaxProfiledSteps = 4096;

hw_status hw_step(hw_solver* s, double dt) {
  hw::NvtxRange nvtx_("hw_step");
  if (!s) return fail(HW_EINVAL, "null solver");
  const StepArgs a = s->args(s->cur, dt > 0 ? dt : 0.0);
  if (s->profiling && s->nprof < kMaxProfiledSteps) {
    cudaEvent_t* e = &s->ev[3 * s->nprof];
    HW_CUDA(cudaEventRecord(e[0], s->stream));
    if (s->fused) {
      launch_fused(s->prec, s->eq, a, s->stream);
      HW_CUDA(cudaEventRecord(e[1], s->stream));
    } else {
      launch_recon(s->prec, s->eq, a, s->stream);
      HW_CUDA(cudaEventRecord(e[1], s->stream));
      launch_edge(s->prec, s->eq, a, s->stream);
    }
    HW_CUDA(cudaEventRecord(e[2], s->stream));
    ++s->nprof;
  } else {
    s->launch(a, s->stream);
  }
  HW_CUDA(cudaGetLastError());
  s->cur = 1 - s->cur;
  return HW_OK;
}

static hw_status ensure_graph(hw_solver* s, int parity) {
  if (s->graph[parity]) return HW_OK;
  cudaGraph_t g = nullptr;
  HW_CUDA(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
  int cur = parity;
  for (int k = 0; k < kGraphSteps; ++k) {
    s->launch(s->args(cur, 0.0), s->cap_stream);
    cur = 1 - cur;
  }
  cudaError_t e = cudaStreamEndCapture(s->cap_stream, &g);
  if (e != cudaSuccess) return fail(HW_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&s->graph[parity], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(HW_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return HW_OK;
}

hw_status hw_run_to(hw_solver* s, double T, int64_t* nsteps) {
  hw::NvtxRange nvtx_("hw_run_to");
  if (!s) return fail(HW_EINVAL, "null solver");
  if (!(T == T)) return fail(HW_EINVAL, "T is NaN");
  HW_CUDA(cudaMemcpyAsync(s->h_sc, s->sc(), sizeof(DevScalars), cudaMemcpyDeviceToHost, s->stream));
  HW_CUDA(cudaStreamSynchronize(s->stream));
  const long long n0 = s->h_sc->nsteps;
  // The target holds only inside this call: the captured graph runs several
  // steps per launch and the steps past T must leave the state as it is.
  // Afterwards hw_step steps again (with the unclipped CFL step).
  struct ClearTarget {
    hw_solver* s;
    ~ClearTarget() { launch_set_target(s->sc(), 0.0, 0, s->stream); }
  };
  launch_set_target(s->sc(), T, 1, s->stream);
  ClearTarget clear_{s};
  if (hw_status st = ensure_graph(s, s->cur)) return st;
  for (long long iter = 0;; ++iter) {
    HW_CUDA(cudaMemcpyAsync(s->h_sc, s->sc(), sizeof(DevScalars), cudaMemcpyDeviceToHost, s->stream));
    HW_CUDA(cudaStreamSynchronize(s->stream));
    if (s->h_sc->flags & 1u) {
      if (nsteps) *nsteps = s->h_sc->nsteps - n0;
      return fail(HW_ENONFINITE, "state became non-finite or non-physical");
    }
    if (s->h_sc->done) break;
    if (!(s->h_sc->dt > 0) || iter > (1ll << 26))
      return fail(HW_ESTATE, "time step vanished before reaching T");
    HW_CUDA(cudaGraphLaunch(s->graph[s->cur], s->stream));
  }
  if (nsteps) *nsteps = s->h_sc->nsteps - n0;
  return HW_OK;
}

hw_status hw_get_state(hw_solver* s, double* Wbar, double* Vbar, double* Ybar, double* t) {
  hw::NvtxRange nvtx_("hw_get_state");
  if (!s) return fail(HW_EINVAL, "null solver");
  const size_t plane = (size_t)s->m * s->N * sizeof(double);
  double* stage = reinterpret_cast<double*>(s->ws + s->L.stage);
  launch_gather(s->prec, s->U(s->cur), s->comp(), s->m, reinterpret_cast<const int32_t*>(s->ws + s->L.perm),
                (int)s->N, (int)s->ld, 3 * s->m, stage, s->stream);
  HW_CUDA(cudaGetLastError());
  if (Wbar) HW_CUDA(cudaMemcpyAsync(Wbar, stage, plane, cudaMemcpyDeviceToHost, s->stream));
  if (Vbar) HW_CUDA(cudaMemcpyAsync(Vbar, reinterpret_cast<char*>(stage) + plane, plane, cudaMemcpyDeviceToHost, s->stream));
  if (Ybar) HW_CUDA(cudaMemcpyAsync(Ybar, reinterpret_cast<char*>(stage) + 2 * plane, plane, cudaMemcpyDeviceToHost, s->stream));
  HW_CUDA(cudaMemcpyAsync(s->h_sc, s->sc(), sizeof(DevScalars), cudaMemcpyDeviceToHost, s->stream));
  HW_CUDA(cudaStreamSynchronize(s->stream));
  if (t) *t = s->h_sc->t;
  return HW_OK;
}

hw_status hw_conservation(hw_solver* s, double* sums) {
  if (!s || !sums) return fail(HW_EINVAL, "null pointer");
  double* partial = reinterpret_cast<double*>(s->ws + s->L.partial);
  double* out = reinterpret_cast<double*>(s->ws + s->L.consv);
  launch_consv(s->prec, s->U(s->cur), s->comp(), reinterpret_cast<const double*>(s->ws + s->L.area), (int)s->N,
               (int)s->ld, s->m, partial, out, s->stream);
  HW_CUDA(cudaGetLastError());
  HW_CUDA(cudaMemcpyAsync(s->h_consv, out, s->m * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  HW_CUDA(cudaStreamSynchronize(s->stream));
  for (int c = 0; c < s->m; ++c) sums[c] = s->h_consv[c];
  return HW_OK;
}

hw_status hw_status_flags(hw_solver* s, uint32_t* flags) {
  if (!s || !flags) return fail(HW_EINVAL, "null pointer");
  HW_CUDA(cudaMemcpyAsync(s->h_sc, s->sc(), sizeof(DevScalars), cudaMemcpyDeviceToHost, s->stream));
  HW_CUDA(cudaStreamSynchronize(s->stream));
  *flags = s->h_sc->flags;
  HW_CUDA(cudaMemsetAsync(&s->sc()->flags, 0, sizeof(unsigned int), s->stream));
  HW_CUDA(cudaStreamSynchronize(s->stream));
  return HW_OK;
}

hw_status hw_time(hw_solver* s, double* t, double* dt, int64_t* nsteps) {
  if (!s) return fail(HW_EINVAL, "null solver");
  HW_CUDA(cudaMemcpyAsync(s->h_sc, s->sc(), sizeof(DevScalars), cudaMemcpyDeviceToHost, s->stream));
  HW_CUDA(cudaStreamSynchronize(s->stream));
  if (t) *t = s->h_sc->t;
  if (dt) *dt = s->h_sc->dt;
  if (nsteps) *nsteps = s->h_sc->nsteps;
  return HW_OK;
}

hw_status hw_profile(hw_solver* s, int32_t enable) {
  if (!s) return fail(HW_EINVAL, "null solver");
  if (enable && s->ev.empty()) {
    s->ev.resize(3 * kMaxProfiledSteps);
    for (auto& e : s->ev) HW_CUDA(cudaEventCreate(&e));
  }
  s->profiling = enable != 0;
  s->nprof = 0;
  return HW_OK;
}

hw_status hw_profile_read(hw_solver* s, double* ms, int64_t* nsteps) {
  if (!s || !ms) return fail(HW_EINVAL, "null pointer");
  ms[0] = ms[1] = 0.0;
  for (int64_t k = 0; k < s->nprof; ++k) {
    float a = 0.f, b = 0.f;
    HW_CUDA(cudaEventSynchronize(s->ev[3 * k + 2]));
    HW_CUDA(cudaEventElapsedTime(&a, s->ev[3 * k], s->ev[3 * k + 1]));
    HW_CUDA(cudaEventElapsedTime(&b, s->ev[3 * k + 1], s->ev[3 * k + 2]));
    ms[0] += a;
    ms[1] += b;
  }
  if (nsteps) *nsteps = s->nprof;
  return HW_OK;
}

hw_status hw_step_kernels(const hw_solver* s, int32_t* path) {
  if (!s || !path) return fail(HW_EINVAL, "null pointer");
  *path = s->fused ? 2 : s->n_oedges > 0 ? 3 : 1;
  return HW_OK;
}

hw_status hw_solver_destroy(hw_solver* s) {
  if (!s) return HW_OK;
  for (auto& e : s->ev) cudaEventDestroy(e);
  for (int p = 0; p < 2; ++p)
    if (s->graph[p]) cudaGraphExecDestroy(s->graph[p]);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  if (s->h_sc) cudaFreeHost(s->h_sc);
  if (s->h_consv) cudaFreeHost(s->h_consv);
  delete s;
  return HW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Step without any device allocation by the caller for scratch.
//
// Some callers cannot call cudaMalloc at all: code running inside a host that
// owns the device memory pool and forbids other allocators, plug-ins that are
// handed fixed buffers, or runtimes that must not allocate once they are
// running.  For them the edge-point buffer (the Taylor data written by the
// reconstruction kernel and read back by the flux kernels, the largest scratch
// of a step) lives in the file-scope device array below instead of in the
// workspace; the per-point flux buffer of the edge-once flux phase stays in
// the workspace the caller passed at hw_state_init.  Every GPU that loads this
// library holds the array until the process exits.
namespace {
constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxScratchDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxScratchDevices] = {};

// Device address of g_static_scratch on the current device, looked up once per
// device.  In host code the array's name is only a host-side handle, so the
// kernels must be given this address.
hw_status static_scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(HW_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxScratchDevices) return fail(HW_EINVAL, "device ordinal out of range for the static scratch");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(HW_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HW_OK;
}
}  // namespace

extern "C" hw_status hw_step_static_scratch(hw_solver* s, double dt) {
  if (!s) return fail(HW_EINVAL, "null solver");
  // the edge-point buffer spans the padded plane stride ld (ntri rounded up to a multiple of 32)
  const size_t need = (size_t)18 * s->m * s->ld * (s->prec == HW_FP64 ? 8 : 4);
  if (need > kStaticScratchBytes)
    return fail(HW_EINVAL, "hw_step_static_scratch: the mesh needs " + std::to_string(need) +
                               " bytes of scratch, more than the static maximum of " +
                               std::to_string(kStaticScratchBytes) + " bytes; use hw_step");
  void* scratch = nullptr;
  if (hw_status st = static_scratch_address(&scratch)) return st;
  StepArgs a = s->args(s->cur, dt > 0 ? dt : 0.0);
  a.Pb = scratch;  // every cell's slots are written by k_recon before k_edge reads them: no clearing needed
  launch_recon(s->prec, s->eq, a, s->stream);
  launch_edge(s->prec, s->eq, a, s->stream);
  HW_CUDA(cudaGetLastError());
  s->cur = 1 - s->cur;
  return HW_OK;
}

// ---------------------------------------------------------------------------
// State buffers on the device, and the adjoint of a step.
namespace {
// Internal state buffer: the records [ld][3m] in the solver's precision, then
// (FP32) the compensation words [ld][m] of the averages.
size_t state_record_bytes(const hw_solver* s) { return (size_t)3 * s->m * s->ld * (s->prec == HW_FP64 ? 8 : 4); }
size_t state_bytes(const hw_solver* s) { return state_record_bytes(s) + s->L.comp_bytes; }

struct AdjointScratch {
  size_t Cb, sc, total;
};
AdjointScratch adjoint_layout(const hw_solver* s) {
  const size_t es = s->prec == HW_FP64 ? 8 : 4, ld = (size_t)s->ld, m = (size_t)s->m;
  AdjointScratch a{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
  a.Cb = take(12 * m * ld * es);
  a.sc = take(sizeof(DevScalars));
  a.total = o;
  return a;
}
}  // namespace

extern "C" {

hw_status hw_state_bytes(const hw_solver* s, size_t* bytes) {
  if (!s || !bytes) return fail(HW_EINVAL, "null pointer");
  *bytes = state_bytes(s);
  return HW_OK;
}

hw_status hw_state_export(hw_solver* s, void* dst) {
  if (!s || !dst) return fail(HW_EINVAL, "null pointer");
  const size_t rb = state_record_bytes(s);
  HW_CUDA(cudaMemcpyAsync(dst, s->U(s->cur), rb, cudaMemcpyDeviceToDevice, s->stream));
  if (s->L.comp_bytes)
    HW_CUDA(cudaMemcpyAsync(static_cast<char*>(dst) + rb, s->comp(), s->L.comp_bytes, cudaMemcpyDeviceToDevice,
                            s->stream));
  return HW_OK;
}

hw_status hw_state_import(hw_solver* s, const void* src, double t) {
  if (!s || !src) return fail(HW_EINVAL, "null pointer");
  const size_t rb = state_record_bytes(s);
  HW_CUDA(cudaMemcpyAsync(s->U(s->cur), src, rb, cudaMemcpyDeviceToDevice, s->stream));
  if (s->L.comp_bytes)
    HW_CUDA(cudaMemcpyAsync(s->comp(), static_cast<const char*>(src) + rb, s->L.comp_bytes,
                            cudaMemcpyDeviceToDevice, s->stream));
  launch_reset(s->sc(), t, s->opt.cfl, s->stream);
  launch_cfl(s->prec, s->eq, s->args(s->cur, 0.0), s->stream);
  HW_CUDA(cudaGetLastError());
  return HW_OK;
}

hw_status hw_state_row_words(const hw_solver* s, int32_t* words) {
  if (!s || !words) return fail(HW_EINVAL, "null pointer");
  *words = (s->L.comp_bytes ? 4 : 3) * s->m;
  return HW_OK;
}

hw_status hw_state_rows_export(hw_solver* s, const int32_t* rows, int64_t n, void* buf) {
  hw::NvtxRange nvtx_("hw_state_rows_export");
  if (!s || n < 0 || (n > 0 && (!rows || !buf))) return fail(HW_EINVAL, "null pointer or negative count");
  launch_rows_gather(s->prec, s->U(s->cur), s->comp(), s->m, (int)s->N, rows, n, buf, &s->sc()->flags, s->stream);
  HW_CUDA(cudaGetLastError());
  return HW_OK;
}

hw_status hw_state_rows_import(hw_solver* s, const int32_t* rows, int64_t n, const void* buf, int32_t refresh) {
  hw::NvtxRange nvtx_("hw_state_rows_import");
  if (!s || n < 0 || (n > 0 && (!rows || !buf))) return fail(HW_EINVAL, "null pointer or negative count");
  launch_rows_scatter(s->prec, s->U(s->cur), s->comp(), s->m, (int)s->N, rows, n, buf, &s->sc()->flags, s->stream);
  if (refresh) launch_cfl(s->prec, s->eq, s->args(s->cur, 0.0), s->stream);
  HW_CUDA(cudaGetLastError());
  return HW_OK;
}

hw_status hw_host_to_internal(hw_solver* s, const double* Wbar, const double* Vbar, const double* Ybar, void* dst) {
  if (!s || !Wbar || !Vbar || !Ybar || !dst) return fail(HW_EINVAL, "null pointer");
  const size_t plane = (size_t)s->m * s->N * sizeof(double);
  double* stage = reinterpret_cast<double*>(s->ws + s->L.stage);
  HW_CUDA(cudaMemcpyAsync(stage, Wbar, plane, cudaMemcpyHostToDevice, s->stream));
  HW_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(stage) + plane, Vbar, plane, cudaMemcpyHostToDevice, s->stream));
  HW_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(stage) + 2 * plane, Ybar, plane, cudaMemcpyHostToDevice, s->stream));
  launch_scatter(s->prec, stage, reinterpret_cast<const int32_t*>(s->ws + s->L.perm), (int)s->N, (int)s->ld,
                 3 * s->m, dst, s->stream);
  if (s->L.comp_bytes)   // a state given as plain values: no compensation
    HW_CUDA(cudaMemsetAsync(static_cast<char*>(dst) + state_record_bytes(s), 0, s->L.comp_bytes, s->stream));
  HW_CUDA(cudaGetLastError());
  HW_CUDA(cudaStreamSynchronize(s->stream));
  return HW_OK;
}

hw_status hw_internal_to_host(hw_solver* s, const void* src, double* Wbar, double* Vbar, double* Ybar) {
  if (!s || !src) return fail(HW_EINVAL, "null pointer");
  const size_t plane = (size_t)s->m * s->N * sizeof(double);
  double* stage = reinterpret_cast<double*>(s->ws + s->L.stage);
  launch_gather(s->prec, src, nullptr, s->m, reinterpret_cast<const int32_t*>(s->ws + s->L.perm), (int)s->N,
                (int)s->ld, 3 * s->m, stage, s->stream);
  HW_CUDA(cudaGetLastError());
  if (Wbar) HW_CUDA(cudaMemcpyAsync(Wbar, stage, plane, cudaMemcpyDeviceToHost, s->stream));
  if (Vbar) HW_CUDA(cudaMemcpyAsync(Vbar, reinterpret_cast<char*>(stage) + plane, plane, cudaMemcpyDeviceToHost, s->stream));
  if (Ybar) HW_CUDA(cudaMemcpyAsync(Ybar, reinterpret_cast<char*>(stage) + 2 * plane, plane, cudaMemcpyDeviceToHost, s->stream));
  HW_CUDA(cudaStreamSynchronize(s->stream));
  return HW_OK;
}

hw_status hw_pb_bytes(const hw_solver* s, size_t* bytes) {
  if (!s || !bytes) return fail(HW_EINVAL, "null pointer");
  *bytes = (size_t)18 * s->m * s->ld * (s->prec == HW_FP64 ? 8 : 4);
  return HW_OK;
}

hw_status hw_step_keep(hw_solver* s, double dt, void* pb_out) {
  hw::NvtxRange nvtx_("hw_step_keep");
  if (!s || !pb_out) return fail(HW_EINVAL, "null pointer");
  if (reinterpret_cast<uintptr_t>(pb_out) % 16) return fail(HW_EINVAL, "edge-point buffer must be 16-byte aligned");
  StepArgs a = s->args(s->cur, dt > 0 ? dt : 0.0);
  a.Pb = pb_out;
  launch_step(s->prec, s->eq, a, s->stream);
  HW_CUDA(cudaGetLastError());
  s->cur = 1 - s->cur;
  return HW_OK;
}

hw_status hw_adjoint_scratch_bytes(const hw_solver* s, size_t* bytes) {
  if (!s || !bytes) return fail(HW_EINVAL, "null pointer");
  *bytes = adjoint_layout(s).total;
  return HW_OK;
}

hw_status hw_step_adjoint(hw_solver* s, double dt, const void* U_n, const void* Pb_n, const void* Ubar_next,
                          void* Ubar_n, void* scratch, size_t scratch_bytes) {
  hw::NvtxRange nvtx_("hw_step_adjoint");
  if (!s || !U_n || !Ubar_next || !Ubar_n || !scratch) return fail(HW_EINVAL, "null pointer");
  if (s->eq != HW_EULER) return fail(HW_EINVAL, "the adjoint step is implemented for the Euler equations");
  if (s->opt.positivity) return fail(HW_EINVAL, "the adjoint step does not cover the scale limiter");
  if (s->opt.time_rule != 0) return fail(HW_EINVAL, "the adjoint step follows the Gauss-Lobatto time rule only");
  if (s->special_bc) return fail(HW_EINVAL, "the adjoint step covers periodic and transmissive boundaries only");
  if (!(dt > 0)) return fail(HW_EINVAL, "the adjoint step needs the (fixed) time step dt > 0");
  if ((reinterpret_cast<uintptr_t>(U_n) | reinterpret_cast<uintptr_t>(Pb_n) | reinterpret_cast<uintptr_t>(Ubar_next) |
       reinterpret_cast<uintptr_t>(Ubar_n)) % 16)
    return fail(HW_EINVAL, "state and edge-point buffers must be 16-byte aligned");
  const AdjointScratch L = adjoint_layout(s);
  if (scratch_bytes < L.total) return fail(HW_ENOMEM, "scratch smaller than hw_adjoint_scratch_bytes");
  if (reinterpret_cast<uintptr_t>(scratch) % 256 != 0) return fail(HW_EINVAL, "scratch must be 256-byte aligned");
  char* sb = static_cast<char*>(scratch);
  StepArgs a = s->args(s->cur, dt);
  a.U = U_n;
  if (Pb_n) {
    a.Pb = const_cast<void*>(Pb_n);   // read only below
  } else {
    DevScalars* asc = reinterpret_cast<DevScalars*>(sb + L.sc);
    launch_reset(asc, 0.0, s->opt.cfl, s->stream);   // a private, never-done scalar block for the recomputation
    a.sc = asc;
    launch_recon(s->prec, s->eq, a, s->stream);
  }
  AdjointArgs b{};
  b.rgeo = a.rgeo;
  b.igeo = a.igeo;
  b.N = a.N;
  b.ld = a.ld;
  b.U = U_n;
  b.Pb = a.Pb;
  b.Ubar_next = Ubar_next;
  b.Cb = sb + L.Cb;
  b.Ubar = Ubar_n;
  b.P = a.P;
  b.dt = dt;
  launch_adjoint(s->prec, b, s->stream);
  HW_CUDA(cudaGetLastError());
  return HW_OK;
}

}  // extern "C"

