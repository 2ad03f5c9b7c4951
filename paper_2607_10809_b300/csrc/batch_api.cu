// C ABI of batched runs (declared in include/hweno.h): many independent solves
// on meshes of different sizes, all time steps of all solves in one persistent
// cooperative launch captured in a CUDA graph, with the launch schedule (blocks
// per SM, tile order) picked by a measured autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/hweno.h"
#include "internal.h"
#include "nvtx.h"
#include "kernels.h"

using namespace hw;

namespace {
constexpr int kCompactChunk = 128;   // steps per launch of a run, at most (tail compaction between launches)
hw_status bfail(hw_status s, const std::string& msg) {
  hw_set_last_error_internal(msg.c_str());
  return s;
}

#define HB_CUDA(call)                                                                                \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return bfail(HW_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct BatchLayout {
  size_t rgeo, igeo, U0, U1, Uinit, Pb, comp, comp_bytes, perm, stage, tiles, bs, bs_init, ctl, total;
};

struct Plan {
  std::vector<int64_t> off, nt;
  int64_t Ntot = 0, ld = 0, maxnt = 0;
  int ntiles = 0;
};

Plan make_plan(const hw_mesh* const* meshes, int n) {
  Plan p;
  int64_t o = 0;
  for (int k = 0; k < n; ++k) {
    const int64_t nt = meshes[k]->M.nt;
    p.off.push_back(o);
    p.nt.push_back(nt);
    p.maxnt = std::max(p.maxnt, nt);
    p.ntiles += (int)((nt + kCells - 1) / kCells);
    o += padded_cells(nt);
  }
  p.Ntot = n > 0 ? p.off.back() + p.nt.back() : 0;
  p.ld = padded_cells(p.Ntot);
  return p;
}

BatchLayout make_batch_layout(const Plan& p, int n, int m, int prec) {
  const size_t s = prec == HW_FP64 ? 8 : 4, ld = (size_t)p.ld;
  BatchLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = a256(o + bytes); return at; };
  L.rgeo = take((size_t)NRGEO * ld * s);
  L.igeo = take((size_t)NIGEO * ld * 4);
  L.U0 = take((size_t)3 * m * ld * s);
  L.U1 = take((size_t)3 * m * ld * s);
  L.Uinit = take((size_t)3 * m * ld * s);
  L.Pb = take((size_t)18 * m * ld * s);
  // FP32: compensation words of the cell averages (compensated summation of the updates)
  L.comp_bytes = prec == HW_FP32 ? (size_t)m * ld * 4 : 0;
  L.comp = take(L.comp_bytes);
  L.perm = take(ld * 4);
  L.stage = take((size_t)3 * m * p.maxnt * 8);
  L.tiles = take((size_t)p.ntiles * sizeof(int4));
  L.bs = take((size_t)n * sizeof(BatchSolve));
  L.bs_init = take((size_t)n * sizeof(BatchSolve));
  L.ctl = take(sizeof(BatchCtl));
  L.total = o;
  return L;
}

hw_status check_batch_args(const hw_mesh* const* meshes, int32_t n, const hw_options* opt, int32_t precision) {
  if (!meshes || n <= 0 || !opt) return bfail(HW_EINVAL, "null pointer or empty batch");
  for (int k = 0; k < n; ++k)
    if (!meshes[k]) return bfail(HW_EINVAL, "null mesh in batch");
  if (opt->eq < 0 || opt->eq > 2 || !(opt->cfl > 0)) return bfail(HW_EINVAL, "bad options");
  if (opt->time_rule != 0) return bfail(HW_EINVAL, "the batched form uses the Gauss-Lobatto time rule only");
  if (precision != HW_FP64 && precision != HW_FP32) return bfail(HW_EINVAL, "unknown precision");
  return HW_OK;
}
}  // namespace

struct hw_batch {
  hw_options opt;
  int prec = 0, eq = 0, m = 1, n = 0;
  Plan plan;
  BatchLayout L{};
  char* ws = nullptr;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  TensorMaps maps{};
  std::vector<int32_t> sizes_order;   // solves by size, descending
  hw_batch_schedule sched{};
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  int graph_ntiles = 0;                 // tile count the graph was captured for
  int cur_ntiles = 0;                   // tiles in the device table (all, or the running solves')
  int sms = 148;
  BatchSolve* h_bs = nullptr;          // pinned mirrors
  BatchCtl* h_ctl = nullptr;

  BatchSolve* bs() { return reinterpret_cast<BatchSolve*>(ws + L.bs); }
  BatchCtl* ctl() { return reinterpret_cast<BatchCtl*>(ws + L.ctl); }
  BatchArgs args(int steps) {
    BatchArgs a{};
    a.rgeo = ws + L.rgeo;
    a.igeo = reinterpret_cast<const int32_t*>(ws + L.igeo);
    a.N = (int)plan.Ntot;
    a.ld = (int)plan.ld;
    a.U0 = ws + L.U0;
    a.U1 = ws + L.U1;
    a.Pb = ws + L.Pb;
    a.C = L.comp_bytes ? ws + L.comp : nullptr;
    a.maps = &maps;
    a.tiles = reinterpret_cast<const int4*>(ws + L.tiles);
    a.ntiles = cur_ntiles > 0 ? cur_ntiles : plan.ntiles;
    a.bs = bs();
    a.ctl = ctl();
    a.nsolves = n;
    a.cfl = opt.cfl;
    a.max_steps = steps;
    a.spin_limit = sched.spin_limit > 0 ? (unsigned long long)sched.spin_limit : (1ull << 25);
    a.withhold_block = sched.withhold_block;
    const int per_sm = batch_blocks_per_sm(prec, eq, eq == HW_EULER && opt.positivity);
    const int bps = std::max(1, std::min(sched.blocks_per_sm > 0 ? sched.blocks_per_sm : per_sm, per_sm));
    a.grid = std::max(1, std::min(bps * sms, a.ntiles));
    a.P.ax = opt.ax; a.P.ay = opt.ay; a.P.gam = opt.gamma_gas; a.P.eps = opt.eps;
    for (int l = 0; l < 4; ++l) { a.P.g[l] = opt.gamma_lin[l]; a.P.win[l] = opt.inflow[l]; }
    eq_params_finish(a.P);
    a.P.positivity = (opt.eq == HW_EULER && opt.positivity) ? 1 : 0;
    a.P.time_rule = 0;
    return a;
  }
};

namespace {
// Tile table in the order of the schedule: 0 = solve by solve, 1 = largest
// solves first, 2 = round robin over the solves (tile k of every solve, then
// tile k + 1, ...).
std::vector<int4> tile_table(const hw_batch* b, int order) {
  std::vector<int> solves(b->n);
  std::iota(solves.begin(), solves.end(), 0);
  if (order == 1) solves = std::vector<int>(b->sizes_order.begin(), b->sizes_order.end());
  std::vector<int4> t;
  t.reserve(b->plan.ntiles);
  auto tiles_of = [&](int s) { return (int)((b->plan.nt[s] + kCells - 1) / kCells); };
  auto add = [&](int s, int k) {
    const int64_t c0 = b->plan.off[s] + (int64_t)k * kCells;
    const int cnt = (int)std::min<int64_t>(kCells, b->plan.nt[s] - (int64_t)k * kCells);
    t.push_back(make_int4((int)c0, cnt, s, 0));
  };
  if (order == 2) {
    int kmax = 0;
    for (int s = 0; s < b->n; ++s) kmax = std::max(kmax, tiles_of(s));
    for (int k = 0; k < kmax; ++k)
      for (int s : solves)
        if (k < tiles_of(s)) add(s, k);
  } else {
    for (int s : solves)
      for (int k = 0; k < tiles_of(s); ++k) add(s, k);
  }
  return t;
}

hw_status upload_table(hw_batch* b, const std::vector<int4>& t) {
  HB_CUDA(cudaMemcpyAsync(b->ws + b->L.tiles, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
  HB_CUDA(cudaStreamSynchronize(b->stream));
  b->cur_ntiles = (int)t.size();
  return HW_OK;
}

hw_status upload_tiles(hw_batch* b) { return upload_table(b, tile_table(b, b->sched.tile_order)); }

// Tail compaction of a run: keep only the tiles of the solves still running
// (same order), so that the persistent grid and its barriers shrink with them.
hw_status compact_tiles(hw_batch* b) {
  std::vector<int4> t;
  for (const int4& e : tile_table(b, b->sched.tile_order))
    if (!b->h_bs[e.z].done) t.push_back(e);
  if (t.empty()) return HW_OK;
  return upload_table(b, t);
}

hw_status capture_graph(hw_batch* b, int steps) {
  if (b->graph && b->graph_steps == steps && b->graph_ntiles == b->cur_ntiles) return HW_OK;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  cudaGraph_t g = nullptr;
  HB_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  launch_batch_reset_ctl(b->ctl(), b->cap_stream);
  cudaError_t e = cudaSuccess;
  if (b->sched.launch_mode == 1) {   // three launches per step; a finished solve's tiles are skipped
    const BatchArgs a = b->args(steps);
    for (int k = 0; k < steps && e == cudaSuccess; ++k) e = launch_batch_step(b->prec, b->eq, a, k & 1, b->cap_stream);
  } else {                           // one persistent cooperative launch with grid barriers
    e = launch_batch(b->prec, b->eq, b->args(steps), b->cap_stream);
  }
  cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(HW_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(HW_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
  b->graph_steps = steps;
  b->graph_ntiles = b->cur_ntiles;
  return HW_OK;
}

hw_status read_status(hw_batch* b) {
  HB_CUDA(cudaMemcpyAsync(b->h_bs, b->bs(), b->n * sizeof(BatchSolve), cudaMemcpyDeviceToHost, b->stream));
  HB_CUDA(cudaMemcpyAsync(b->h_ctl, b->ctl(), sizeof(BatchCtl), cudaMemcpyDeviceToHost, b->stream));
  HB_CUDA(cudaStreamSynchronize(b->stream));
  return HW_OK;
}

hw_status restore_initial(hw_batch* b) {
  const size_t sz = (size_t)3 * b->m * b->plan.ld * (b->prec == HW_FP64 ? 8 : 4);
  HB_CUDA(cudaMemcpyAsync(b->ws + b->L.U0, b->ws + b->L.Uinit, sz, cudaMemcpyDeviceToDevice, b->stream));
  HB_CUDA(cudaMemcpyAsync(b->ws + b->L.bs, b->ws + b->L.bs_init, b->n * sizeof(BatchSolve), cudaMemcpyDeviceToDevice,
                          b->stream));
  if (b->L.comp_bytes) HB_CUDA(cudaMemsetAsync(b->ws + b->L.comp, 0, b->L.comp_bytes, b->stream));
  return HW_OK;
}
}  // namespace

extern "C" {

void hw_batch_schedule_default(hw_batch_schedule* s) {
  if (!s) return;
  std::memset(s, 0, sizeof(*s));
  s->blocks_per_sm = 0;      // 0: as many as fit
  s->tile_order = 0;
  s->steps_per_launch = 1 << 20;
  s->spin_limit = 0;         // 0: default
  s->withhold_block = -1;
  s->launch_mode = 0;
}

hw_status hw_batch_workspace_bytes(const hw_mesh* const* meshes, int32_t n, const hw_options* opt, int32_t precision,
                                   size_t* bytes) {
  if (hw_status st = check_batch_args(meshes, n, opt, precision)) return st;
  if (!bytes) return bfail(HW_EINVAL, "null pointer");
  const Plan p = make_plan(meshes, n);
  *bytes = make_batch_layout(p, n, opt->eq == HW_EULER ? 4 : 1, precision).total;
  return HW_OK;
}

hw_status hw_batch_create(const hw_mesh* const* meshes, int32_t n, const hw_options* opt, int32_t precision,
                          const double* const* Wbar, const double* const* Vbar, const double* const* Ybar,
                          void* workspace, size_t workspace_bytes, void* cuda_stream, hw_batch** out) {
  hw::NvtxRange nvtx_("hw_batch_create");
  if (hw_status st = check_batch_args(meshes, n, opt, precision)) return st;
  if (!Wbar || !Vbar || !Ybar || !workspace || !out) return bfail(HW_EINVAL, "null pointer");
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return bfail(HW_EINVAL, "workspace must be 256-byte aligned");
  hw_batch* b = new (std::nothrow) hw_batch();
  if (!b) return bfail(HW_ENOMEM, "host allocation failed");
  auto bail = [&](hw_status st) { hw_batch_destroy(b); return st; };
  b->opt = *opt;
  b->prec = precision;
  b->eq = opt->eq;
  b->m = opt->eq == HW_EULER ? 4 : 1;
  b->n = n;
  b->plan = make_plan(meshes, n);
  b->L = make_batch_layout(b->plan, n, b->m, precision);
  if (workspace_bytes < b->L.total) { delete b; return bfail(HW_ENOMEM, "workspace smaller than hw_batch_workspace_bytes"); }
  if (b->plan.ld > 0x3fffffff) { delete b; return bfail(HW_EINVAL, "batch too large"); }
  b->ws = static_cast<char*>(workspace);
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  hw_batch_schedule_default(&b->sched);
  b->sizes_order.resize(n);
  std::iota(b->sizes_order.begin(), b->sizes_order.end(), 0);
  std::stable_sort(b->sizes_order.begin(), b->sizes_order.end(),
                   [&](int x, int y) { return b->plan.nt[x] > b->plan.nt[y]; });
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost(&b->h_bs, n * sizeof(BatchSolve)) != cudaSuccess ||
      cudaMallocHost(&b->h_ctl, sizeof(BatchCtl)) != cudaSuccess)
    return bail(bfail(HW_ECUDA, "stream / pinned host buffer creation failed"));
  const size_t es = precision == HW_FP64 ? 8 : 4, ld = (size_t)b->plan.ld, m = (size_t)b->m;
  // geometry and indices of every solve at its offset
  std::vector<int32_t> perm_all(ld, 0);
  for (int k = 0; k < n; ++k) {
    const HostMesh& M = meshes[k]->M;
    const size_t nt = (size_t)M.nt, off = (size_t)b->plan.off[k];
    cudaError_t e;
    if (precision == HW_FP64) {
      e = cudaMemcpy2DAsync(b->ws + b->L.rgeo + off * 8, ld * 8, M.rgeo.data(), nt * 8, nt * 8, NRGEO,
                            cudaMemcpyHostToDevice, b->stream);
    } else {
      std::vector<float> tmp((size_t)NRGEO * nt);
      for (size_t q = 0; q < tmp.size(); ++q) tmp[q] = (float)M.rgeo[q];
      e = cudaMemcpy2DAsync(b->ws + b->L.rgeo + off * 4, ld * 4, tmp.data(), nt * 4, nt * 4, NRGEO,
                            cudaMemcpyHostToDevice, b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    std::vector<int32_t> ig(M.igeo);
    for (int j = 0; j < 3; ++j)
      for (size_t i = 0; i < nt; ++i) {
        int32_t& v = ig[(size_t)(I_NBR + j) * nt + i];
        if (v >= 0) v += (int32_t)off;
      }
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(b->ws + b->L.igeo + off * 4, ld * 4, ig.data(), nt * 4, nt * 4, NIGEO,
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bail(bfail(HW_ECUDA, std::string("batch geometry upload: ") + cudaGetErrorString(e)));
    std::copy(M.perm.begin(), M.perm.end(), perm_all.begin() + off);
  }
  HB_CUDA(cudaMemcpyAsync(b->ws + b->L.perm, perm_all.data(), ld * 4, cudaMemcpyHostToDevice, b->stream));
  // TMA descriptors over all cells
  {
    const hw_status st = hw_encode_plane_maps(&b->maps, precision, b->ws + b->L.rgeo, b->ws + b->L.igeo,
                                              b->plan.Ntot, b->plan.ld);
    if (st != HW_OK) return bail(st);
  }
  // initial states (host order per solve) -> buffer 0 and the saved copy
  double* stage = reinterpret_cast<double*>(b->ws + b->L.stage);
  for (int k = 0; k < n; ++k) {
    const size_t nt = (size_t)b->plan.nt[k], off = (size_t)b->plan.off[k];
    if (!Wbar[k] || !Vbar[k] || !Ybar[k]) return bail(bfail(HW_EINVAL, "null state array in batch"));
    const size_t plane = m * nt * 8;
    HB_CUDA(cudaMemcpyAsync(stage, Wbar[k], plane, cudaMemcpyHostToDevice, b->stream));
    HB_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(stage) + plane, Vbar[k], plane, cudaMemcpyHostToDevice, b->stream));
    HB_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(stage) + 2 * plane, Ybar[k], plane, cudaMemcpyHostToDevice,
                            b->stream));
    launch_scatter(precision, stage, reinterpret_cast<const int32_t*>(b->ws + b->L.perm) + off, (int)nt, 0,
                   (int)(3 * m), b->ws + b->L.U0 + off * 3 * m * es, b->stream);
    HB_CUDA(cudaGetLastError());
  }
  HB_CUDA(cudaMemcpyAsync(b->ws + b->L.Uinit, b->ws + b->L.U0, 3 * m * ld * es, cudaMemcpyDeviceToDevice, b->stream));
  if (b->L.comp_bytes) HB_CUDA(cudaMemsetAsync(b->ws + b->L.comp, 0, b->L.comp_bytes, b->stream));
  // per-solve state: t = 0, CFL step
  std::vector<BatchSolve> bs0(n);
  for (auto& x : bs0) {
    std::memset(&x, 0, sizeof(x));
    x.lam_min_bits = 0x7ff0000000000000ull;
  }
  HB_CUDA(cudaMemcpyAsync(b->bs(), bs0.data(), n * sizeof(BatchSolve), cudaMemcpyHostToDevice, b->stream));
  launch_batch_reset_ctl(b->ctl(), b->stream);
  if (hw_status st = upload_tiles(b)) return bail(st);
  prepare_step_kernels(precision, b->eq);
  (void)batch_blocks_per_sm(precision, b->eq, b->eq == HW_EULER && opt->positivity);
  launch_batch_cfl(precision, b->eq, b->args(1), b->stream);
  launch_batch_dt(b->bs(), n, opt->cfl, 0.0, 0, b->stream);
  HB_CUDA(cudaGetLastError());
  HB_CUDA(cudaMemcpyAsync(b->ws + b->L.bs_init, b->bs(), n * sizeof(BatchSolve), cudaMemcpyDeviceToDevice,
                          b->stream));
  HB_CUDA(cudaStreamSynchronize(b->stream));
  *out = b;
  return HW_OK;
}

hw_status hw_batch_set_schedule(hw_batch* b, const hw_batch_schedule* s) {
  if (!b || !s) return bfail(HW_EINVAL, "null pointer");
  if (s->tile_order < 0 || s->tile_order > 2 || s->blocks_per_sm < 0 || s->steps_per_launch <= 0 ||
      s->launch_mode < 0 || s->launch_mode > 1)
    return bfail(HW_EINVAL, "bad schedule");
  if (s->launch_mode == 1 && s->withhold_block >= 0)
    return bfail(HW_EINVAL, "withhold_block tests the grid barrier of launch_mode 0");
  const bool order_changed = s->tile_order != b->sched.tile_order;
  b->sched = *s;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  if (order_changed) return upload_tiles(b);
  return HW_OK;
}

hw_status hw_batch_get_schedule(const hw_batch* b, hw_batch_schedule* s, int32_t* grid_blocks) {
  if (!b || !s) return bfail(HW_EINVAL, "null pointer");
  *s = b->sched;
  if (grid_blocks) *grid_blocks = const_cast<hw_batch*>(b)->args(1).grid;
  return HW_OK;
}

hw_status hw_batch_run_to(hw_batch* b, double T, int64_t* cell_steps) {
  hw::NvtxRange nvtx_("hw_batch_run_to");
  if (!b) return bfail(HW_EINVAL, "null batch");
  if (!(T == T)) return bfail(HW_EINVAL, "T is NaN");
  launch_batch_dt(b->bs(), b->n, b->opt.cfl, T, 1, b->stream);
  HB_CUDA(cudaGetLastError());
  // chunks of at most kCompactChunk steps; between chunks, once the running
  // solves hold at most half of the current tiles, the table shrinks to them
  const int chunk = std::max(1, std::min(b->sched.steps_per_launch, kCompactChunk));
  if (hw_status st = read_status(b)) return st;
  std::vector<long long> n0(b->n);
  for (int k = 0; k < b->n; ++k) n0[k] = b->h_bs[k].nsteps;
  hw_status result = HW_OK;
  for (long long iter = 0;; ++iter) {
    bool all_done = true;
    int64_t active_tiles = 0;
    for (int k = 0; k < b->n; ++k) {
      all_done = all_done && b->h_bs[k].done;
      if (!b->h_bs[k].done) active_tiles += (b->plan.nt[k] + kCells - 1) / kCells;
    }
    if (all_done) break;
    if (iter > (1ll << 24)) { result = bfail(HW_ESTATE, "batch did not reach T"); break; }
    if (2 * active_tiles <= b->cur_ntiles)
      if ((result = compact_tiles(b)) != HW_OK) break;
    if ((result = capture_graph(b, chunk)) != HW_OK) break;
    HB_CUDA(cudaGraphLaunch(b->graph, b->stream));
    if ((result = read_status(b)) != HW_OK) break;
    if (b->h_ctl->flags & 2u) { result = bfail(HW_ETIMEOUT, "batched kernel: a bounded wait gave up"); break; }
  }
  if (b->cur_ntiles != b->plan.ntiles) {   // the full table again for the next call
    if (hw_status st = upload_tiles(b)) return st;
  }
  if (result != HW_OK) return result;
  if (cell_steps) {
    int64_t cs = 0;
    for (int k = 0; k < b->n; ++k) cs += (b->h_bs[k].nsteps - n0[k]) * b->plan.nt[k];
    *cell_steps = cs;
  }
  for (int k = 0; k < b->n; ++k)
    if (b->h_bs[k].failed) return bfail(HW_ENONFINITE, "solve " + std::to_string(k) + " became non-physical");
  return HW_OK;
}

hw_status hw_batch_steps(hw_batch* b, int32_t steps, double* ms) {
  hw::NvtxRange nvtx_("hw_batch_steps");
  if (!b || steps <= 0) return bfail(HW_EINVAL, "bad arguments");
  launch_batch_dt(b->bs(), b->n, b->opt.cfl, 1e300, 1, b->stream);
  // the three-launch form captures at most kCompactChunk steps per graph (three
  // nodes per step); longer runs replay it, reading the flags in between (each
  // replay starts by clearing them)
  const int chunk = b->sched.launch_mode == 1 ? std::min<int>(steps, kCompactChunk) : steps;
  if (hw_status st = capture_graph(b, chunk)) return st;
  struct Events {   // destroyed on every return path
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Events() {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    }
  } ev;
  HB_CUDA(cudaEventCreate(&ev.e0));
  HB_CUDA(cudaEventCreate(&ev.e1));
  cudaEvent_t e0 = ev.e0, e1 = ev.e1;
  unsigned flags = 0u;
  HB_CUDA(cudaEventRecord(e0, b->stream));
  for (int done = 0; done < steps;) {
    const int n = std::min(chunk, steps - done);
    if (hw_status st = capture_graph(b, n)) return st;   // the chunk, or the last, shorter one
    HB_CUDA(cudaGraphLaunch(b->graph, b->stream));
    done += n;
    if (done < steps) {
      if (hw_status st = read_status(b)) return st;
      flags |= b->h_ctl->flags;
    }
  }
  HB_CUDA(cudaEventRecord(e1, b->stream));
  HB_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  if (ms) *ms = t;
  if (hw_status st = read_status(b)) return st;
  flags |= b->h_ctl->flags;
  if (flags & 2u) return bfail(HW_ETIMEOUT, "batched kernel: a bounded wait gave up");
  return HW_OK;
}

hw_status hw_batch_reset(hw_batch* b) {
  if (!b) return bfail(HW_EINVAL, "null batch");
  if (hw_status st = restore_initial(b)) return st;
  HB_CUDA(cudaStreamSynchronize(b->stream));
  return HW_OK;
}

hw_status hw_batch_autotune(hw_batch* b, int32_t trial_steps, hw_batch_schedule* best, double* best_ms) {
  hw::NvtxRange nvtx_("hw_batch_autotune");
  if (!b || trial_steps <= 0) return bfail(HW_EINVAL, "bad arguments");
  const int per_sm = batch_blocks_per_sm(b->prec, b->eq, b->eq == HW_EULER && b->opt.positivity);
  hw_batch_schedule base = b->sched, pick = b->sched;
  double pick_ms = 1e300;
  for (int mode = 0; mode <= 1; ++mode)
  for (int order = 0; order <= 2; ++order)
    for (int bps = 1; bps <= (mode == 0 ? per_sm : 1); ++bps) {   // the three-launch form sizes its own grids
      hw_batch_schedule s = base;
      s.launch_mode = mode;
      s.withhold_block = -1;
      s.tile_order = order;
      s.blocks_per_sm = mode == 0 ? bps : 0;
      s.steps_per_launch = trial_steps;
      if (hw_status st = hw_batch_set_schedule(b, &s)) return st;
      if (hw_status st = hw_batch_reset(b)) return st;
      double ms = 0;
      if (hw_status st = hw_batch_steps(b, trial_steps, &ms)) return st;   // first run: warm-up
      if (hw_status st = hw_batch_reset(b)) return st;
      if (hw_status st = hw_batch_steps(b, trial_steps, &ms)) return st;
      if (ms < pick_ms) { pick_ms = ms; pick = s; }
    }
  pick.steps_per_launch = base.steps_per_launch;
  if (hw_status st = hw_batch_set_schedule(b, &pick)) return st;
  if (hw_status st = hw_batch_reset(b)) return st;
  if (best) *best = pick;
  if (best_ms) *best_ms = pick_ms;
  return HW_OK;
}

hw_status hw_batch_get_state(hw_batch* b, int32_t solve, double* Wbar, double* Vbar, double* Ybar, double* t,
                             int64_t* nsteps, int32_t* failed) {
  if (!b || solve < 0 || solve >= b->n) return bfail(HW_EINVAL, "bad solve index");
  if (hw_status st = read_status(b)) return st;
  const BatchSolve& x = b->h_bs[solve];
  const size_t es = b->prec == HW_FP64 ? 8 : 4, m = (size_t)b->m;
  const size_t nt = (size_t)b->plan.nt[solve], off = (size_t)b->plan.off[solve];
  const char* U = b->ws + ((x.nsteps & 1) ? b->L.U1 : b->L.U0) + off * 3 * m * es;
  double* stage = reinterpret_cast<double*>(b->ws + b->L.stage);
  const char* Cw = b->L.comp_bytes ? b->ws + b->L.comp + off * m * 4 : nullptr;   // FP32 compensation words
  launch_gather(b->prec, U, Cw, (int)m, reinterpret_cast<const int32_t*>(b->ws + b->L.perm) + off, (int)nt, 0,
                (int)(3 * m),
                stage, b->stream);
  HB_CUDA(cudaGetLastError());
  const size_t plane = m * nt * 8;
  if (Wbar) HB_CUDA(cudaMemcpyAsync(Wbar, stage, plane, cudaMemcpyDeviceToHost, b->stream));
  if (Vbar) HB_CUDA(cudaMemcpyAsync(Vbar, reinterpret_cast<char*>(stage) + plane, plane, cudaMemcpyDeviceToHost, b->stream));
  if (Ybar)
    HB_CUDA(cudaMemcpyAsync(Ybar, reinterpret_cast<char*>(stage) + 2 * plane, plane, cudaMemcpyDeviceToHost, b->stream));
  HB_CUDA(cudaStreamSynchronize(b->stream));
  if (t) *t = x.t;
  if (nsteps) *nsteps = x.nsteps;
  if (failed) *failed = x.failed;
  return HW_OK;
}

hw_status hw_batch_destroy(hw_batch* b) {
  if (!b) return HW_OK;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->h_bs) cudaFreeHost(b->h_bs);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  delete b;
  return HW_OK;
}

}  // extern "C"
