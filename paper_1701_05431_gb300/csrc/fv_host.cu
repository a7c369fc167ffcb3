// fv_host.cu -- C ABI of the finite-volume library (include/fv.h): context,
// validation, device buffers, kernel choice, the CUDA-graph time loop and
// error reporting.  Every numerical step runs in the kernels of fv_step*.cu,
// fv_spray.cu and fv_aux.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/fv.h"
#include "fv_internal.h"
#include "fv_tune.h"
#include "fv_step.cuh"
#include "fv_tb.cuh"

namespace fv {

const std::vector<Variant> &all_variants() {
  static std::vector<Variant> v;
  static std::once_flag once;
  std::call_once(once, [] {
    register_step_advection(v);
    register_step_euler(v);
    register_step_spray(v);
  });
  return v;
}

static int nvar_of(int system) {
  switch (system) {
    case kAdvection: return 1;
    case kEuler: return 4;
    case kSpray: return 6;
    default: return 0;
  }
}

}  // namespace fv

using namespace fv;

struct fv_ctx {
  fv_config cfg;
  int nvar = 0;
  size_t esize = 0;
  long long pitch = 0, plane = 0;
  size_t buf_bytes = 0;
  // FP64 Euler: each state buffer also holds the primitives u, v, p, c of
  // its cells (planes 4..7) for the kernels that carry them (Variant::carry)
  int nplanes = 0;
  bool pc_dirty = false;         // planes 4..7 of the current state are stale
  double bc_pc[4][4] = {};       // primitives of the four boundary states
  // two time steps per launch (fixed dt, periodic): its kernel and grid
  int tb_variant = -1;
  int tb_grid = 0;
  bool tb_np = false;            // some side is not periodic: the two-step kernel's ghost-handling build
  // in-place mode: buf[1] == buf[0], overlap strips of the two parities
  bool inplace = false;
  void *ovl = nullptr;
  size_t ovl_parity_bytes = 0;
  int ovl_task = 0;
  void *buf[2] = {nullptr, nullptr};
  Ctrl *ctrl = nullptr;
  Ctrl *h_ctrl = nullptr;        // pinned mirror, mapped for the device
  Ctrl *h_ctrl_dev = nullptr;    // its device address
  double *h_scalar = nullptr;    // pinned scratch for small uploads
  void *staging = nullptr;
  size_t staging_bytes = 0;
  double *partials = nullptr;
  double *d_totals = nullptr;
  double *lamw = nullptr;        // spray: multipliers of the last three solves (12 planes)
  double *ecache = nullptr;      // spray: exponentials of the last solve (Q planes)
  double *nodes = nullptr;       // spray: quadrature table
  int spray_Q = 0;
  int src_grid = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // graph capture needs a non-legacy stream
  // asynchronous snapshots: staging buffer, side stream, events
  void *snap_buf = nullptr;
  size_t snap_bytes = 0;
  cudaStream_t snap_stream = nullptr;
  cudaEvent_t snap_ready = nullptr, snap_done = nullptr;
  bool snap_pending = false;
  // asynchronous input prefetch: device buffer, side stream, events
  void *pre_buf = nullptr;
  size_t pre_bytes = 0;
  cudaStream_t pre_stream = nullptr;
  cudaEvent_t pre_copied = nullptr, pre_consumed = nullptr;
  bool pre_pending = false;    // a prefetched state waits to be loaded
  bool pre_used = false;       // pre_consumed has been recorded at least once
  int pre_dtype = 0, pre_layout = 0;
  bool has_state = false;
  int variant = -1;
  int grid = 0;
  int ty = 0;                    // rows per warp task of the selected kernel
  std::string choice;            // how that kernel was chosen (fv_kernel_choice)
  std::string tb_choice;         // how the two-step kernel was chosen
  int single_variant = -1;       // the two-buffer kernel (restored when in-place mode ends)
  std::string single_choice;
  std::string desc;              // its description with the task rows
  double dx = 0, dy = 0;
  std::map<int, cudaGraphExec_t> graphs;
  std::string err;
  int device = 0;
  int sms = 0;
  bool tuned = false;
};

static std::string g_init_error;

namespace fv {
void set_global_error(const std::string &msg) { g_init_error = msg; }
}  // namespace fv

static fv_status fail(fv_ctx *c, fv_status s, const std::string &msg) {
  if (c) c->err = msg;
  else g_init_error = msg;
  return s;
}

static fv_status cuda_fail(fv_ctx *c, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(c, e == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA, m);
}

#define FV_CUDA(c, call)                                 \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)

extern "C" const char *fv_status_string(fv_status s) {
  switch (s) {
    case FV_OK: return "ok";
    case FV_ERR_INVALID_ARG: return "invalid argument";
    case FV_ERR_CUDA: return "CUDA error";
    case FV_ERR_OOM: return "out of device memory";
    case FV_ERR_CFL: return "fixed time step violates the CFL condition";
    case FV_ERR_NONPHYSICAL: return "non-physical state";
    case FV_ERR_TIMEOUT: return "device wait timed out";
    case FV_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

extern "C" const char *fv_last_error(const fv_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

static fv_status validate(const fv_config *c) {
  if (!c) return fail(nullptr, FV_ERR_INVALID_ARG, "config is NULL");
  if (nvar_of(c->system) == 0) return fail(nullptr, FV_ERR_INVALID_ARG, "unknown system");
  if (c->precision != FV_F64 && c->precision != FV_F32 && c->precision != FV_BF16)
    return fail(nullptr, FV_ERR_INVALID_ARG, "unknown precision");
  if (c->precision == FV_BF16 && c->system == FV_SPRAY)
    return fail(nullptr, FV_ERR_INVALID_ARG, "bf16 storage is not available for the spray system");
  if (c->nx < 1 || c->ny < 1) return fail(nullptr, FV_ERR_INVALID_ARG, "nx and ny must be >= 1");
  if ((long long)c->nx * c->ny > (1LL << 34))
    return fail(nullptr, FV_ERR_INVALID_ARG, "grid too large");
  if (c->npart_x < 1 || c->npart_y < 1 || c->npart_x > c->nx || c->npart_y > c->ny)
    return fail(nullptr, FV_ERR_INVALID_ARG, "need 1 <= npart_x <= nx and 1 <= npart_y <= ny");
  if (!(c->xmax > c->xmin) || !(c->ymax > c->ymin))
    return fail(nullptr, FV_ERR_INVALID_ARG, "empty domain");
  for (int s = 0; s < 4; ++s)
    if (c->bc[s] < 0 || c->bc[s] > 2) return fail(nullptr, FV_ERR_INVALID_ARG, "unknown boundary condition");
  if ((c->bc[FV_SIDE_E] == FV_BC_PERIODIC) != (c->bc[FV_SIDE_W] == FV_BC_PERIODIC))
    return fail(nullptr, FV_ERR_INVALID_ARG, "periodic E must pair with periodic W");
  if ((c->bc[FV_SIDE_N] == FV_BC_PERIODIC) != (c->bc[FV_SIDE_S] == FV_BC_PERIODIC))
    return fail(nullptr, FV_ERR_INVALID_ARG, "periodic N must pair with periodic S");
  if (!(c->fixed_dt > 0.0) && !(c->cfl > 0.0))
    return fail(nullptr, FV_ERR_INVALID_ARG, "need cfl > 0 or fixed_dt > 0");
  if (!std::isfinite(c->cfl) || !std::isfinite(c->fixed_dt))
    return fail(nullptr, FV_ERR_INVALID_ARG, "cfl and fixed_dt must be finite");
  if (c->system == FV_EULER && !(c->params[0] > 1.0))
    return fail(nullptr, FV_ERR_INVALID_ARG, "Euler needs gamma > 1");
  if (c->system == FV_SPRAY) {
    int Q = (int)c->params[3];
    if (Q < 0 || Q > 64) return fail(nullptr, FV_ERR_INVALID_ARG, "spray quadrature: 0 <= Q <= 64");
    if (c->params[0] < 0.0) return fail(nullptr, FV_ERR_INVALID_ARG, "spray K must be >= 0");
  }
  return FV_OK;
}

// Blocks of a kernel candidate resident per SM (its register target MINB if
// the occupancy query fails).
static int resident_blocks(const Variant &V) {
  if (V.smem > 0 &&
      cudaFuncSetAttribute(V.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, V.smem) != cudaSuccess)
    return V.MINB;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, V.kernel, V.NW * 32, V.smem) != cudaSuccess || nb < 1)
    return V.MINB;
  return nb;
}

// Rows per warp task within [max(1, TY/16), 5 TY/4] that minimise waves x
// (rows + 3) for an nx x ny grid over W resident warps (see balanced_rows);
// *cost receives that product.  (On a grid too small to fill the GPU even
// with one-row tasks the fewest rows win: C1, 128^2, runs 1-row tasks at
// 1.68 G cell-updates/s against 1.62 with 4-row tasks.)
static int balance_rows_for(const Variant &V, int nx, int ny, long long W, long long *cost) {
  const long long nstrips = (nx + 30 * V.V - 1) / (30 * V.V);
  int best = V.TY;
  long long best_cost = -1;
  for (int ty = std::max(1, V.TY / 16); ty <= (5 * V.TY) / 4; ++ty) {
    const long long tasks = nstrips * ((ny + ty - 1) / ty);
    const long long cst = ((tasks + W - 1) / W) * (ty + 3);
    if (best_cost < 0 || cst < best_cost ||
        (cst == best_cost && std::abs(ty - V.TY) < std::abs(best - V.TY))) {
      best_cost = cst;
      best = ty;
    }
  }
  if (cost) *cost = best_cost;
  return best;
}

// Default kernel for an nx x ny grid: the first candidate of (system,
// precision), in the table's order of preference, whose warp tasks fill the
// GPU (at least two per resident warp); if none does, the one with the most
// tasks per resident warp.
static int default_variant_for(int system, int prec, int nx, int ny, int sms, int inplace = 0, int tb = 0) {
  const auto &vs = all_variants();
  int best = -1;
  double best_ratio = -1.0;
  if (prec == 0 && !inplace && !tb) {
    // FP64 single-step kernels get their rows per task balanced: among the
    // candidates of the first one's kind (same warps, register target and
    // staging; TY and cells per lane differ), take the one whose balanced
    // launch the time model finds shortest, a warp's row costing its cells
    // per lane (the first of equals)
    long long best_cost = -1;
    const Variant *first = nullptr;
    for (size_t k = 0; k < vs.size(); ++k) {
      const Variant &V = vs[k];
      if (V.system != system || V.precision != prec || V.inplace || V.tb) continue;
      if (!first) first = &V;
      if (V.NW != first->NW || V.MINB != first->MINB || V.D != first->D) continue;
      long long cost = 0;
      balance_rows_for(V, nx, ny, (long long)resident_blocks(V) * V.NW * sms, &cost);
      cost *= V.V;
      if (best_cost < 0 || cost < best_cost) {
        best_cost = cost;
        best = (int)k;
      }
    }
    return best;
  }
  for (size_t k = 0; k < vs.size(); ++k) {
    const Variant &V = vs[k];
    if (V.system != system || V.precision != prec || V.inplace != inplace || V.tb != tb) continue;
    const double tasks = (double)((nx + 30 * V.V - 1) / (30 * V.V)) * (double)((ny + V.TY - 1) / V.TY);
    const double ratio = tasks / ((double)resident_blocks(V) * V.NW * sms);
    if (ratio >= 2.0) return (int)k;
    if (ratio > best_ratio) {
      best_ratio = ratio;
      best = (int)k;
    }
  }
  return best;
}

static std::vector<int> candidates(int system, int prec) {
  std::vector<int> out;
  const auto &vs = all_variants();
  for (size_t k = 0; k < vs.size(); ++k)
    if (vs[k].system == system && vs[k].precision == prec && !vs[k].inplace && !vs[k].tb) out.push_back((int)k);
  return out;
}

// The variant the recorded table names for this key (mode: TuneMode), or -1;
// *how receives the table entry's description.
static int table_variant(int system, int prec, int nx, int ny, int mode, std::string *how) {
  const TuneEntry *e = tune_lookup(system, prec, (long long)nx * ny, mode);
  if (!e) return -1;
  const auto &vs = all_variants();
  for (size_t k = 0; k < vs.size(); ++k) {
    const Variant &V = vs[k];
    if (V.system != system || V.precision != prec || V.inplace != (mode == kTuneInplace ? 1 : 0) ||
        V.tb != (mode == kTuneTwoStep ? 2 : 0))
      continue;
    if (std::string(V.desc) == e->kernel) {
      if (how) *how = tune_describe(*e);
      return (int)k;
    }
  }
  return -1;
}

static const char *kHeuristic = "heuristic (no table entry): the first candidate whose warp tasks fill the GPU";

static void free_graphs(fv_ctx *c) {
  for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
}

// Rows per warp task of an FP64 single-step kernel: from TY/4 (at least 4)
// to 5 TY/4, the count that minimises waves x (rows + 3), the time of a persistent
// launch whose resident warps take the tasks round robin (a task costs its
// rows plus about three: the halo row and the first row's fluxes); ties go
// to the count nearest TY.  The model holds where the FP64 pipe bounds the
// kernel, so that a task's time follows its rows (measured: 4.35 against
// 4.07 G cell-updates/s on the 2048^2 four-quadrant case, 1.66 against 0.91
// on 128^2 advection, where one wave of 4-row tasks replaces 16-row ones).
// The FP32 and BF16 kernels are bound by HBM bandwidth on large grids, which
// a last partial wave of warps still draws; balanced rows made them slower
// there (170 against 175 G on 8192^2), so from 2^24 cells on they keep TY.
// Below that the state sits in or near L2 and a launch's last partial wave
// is what costs: balanced rows give the fastest candidate on the 2048^2
// four-quadrant case 108 against 104 G cell-updates/s.
static int balanced_rows(const fv_ctx *c, const Variant &V, int nb) {
  return balance_rows_for(V, c->cfg.nx, c->cfg.ny, (long long)nb * V.NW * c->sms, nullptr);
}

static fv_status select_variant(fv_ctx *c, int vi) {
  const Variant &V = all_variants()[vi];
  int nb = 0;
  if (V.smem > 0)
    FV_CUDA(c, cudaFuncSetAttribute(V.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, V.smem));
  FV_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, V.kernel, V.NW * 32, V.smem));
  if (nb < 1) return fail(c, FV_ERR_CUDA, std::string("kernel cannot launch: ") + V.desc);
  const bool small = (long long)c->cfg.nx * c->cfg.ny < (1LL << 24);
  c->ty = (V.inplace || V.tb || (V.precision != 0 && !small)) ? V.TY : balanced_rows(c, V, nb);
  const int nstrips = (c->cfg.nx + 30 * V.V - 1) / (30 * V.V);
  const int nchunks = (c->cfg.ny + c->ty - 1) / c->ty;
  const long long ntasks = (long long)nstrips * nchunks;
  long long need = (ntasks + V.NW - 1) / V.NW;
  long long grid = (long long)nb * c->sms;
  if (need < grid) grid = need;
  if (grid < 1) grid = 1;
  c->variant = vi;
  c->grid = (int)grid;
  free_graphs(c);
  return FV_OK;
}

template <class R>
static StepArgs<R> make_args(const fv_ctx *c, const Variant &V) {
  StepArgs<R> a;
  std::memset(&a, 0, sizeof(a));
  a.buf0 = (R *)c->buf[0];
  a.buf1 = (R *)c->buf[1];
  if (c->inplace) {
    a.ovl[0] = (R *)c->ovl;
    a.ovl[1] = (R *)((char *)c->ovl + c->ovl_parity_bytes);
    a.ovl_task = c->ovl_task;
    a.ovl_bc = (const R *)((char *)c->ovl + 2 * c->ovl_parity_bytes);
  }
  a.ctrl = c->ctrl;
  a.nx = c->cfg.nx;
  a.ny = c->cfg.ny;
  a.pitch = c->pitch;
  a.plane = c->plane;
  a.nstrips = (c->cfg.nx + 30 * V.V - 1) / (30 * V.V);
  a.ty = (V.inplace || V.tb || c->ty < 1) ? V.TY : c->ty;
  a.nchunks = (c->cfg.ny + a.ty - 1) / a.ty;
  a.ntasks = a.nstrips * a.nchunks;
  a.dx = c->dx;
  a.dy = c->dy;
  a.pol.h = c->dx < c->dy ? c->dx : c->dy;
  a.pol.cfl = c->cfg.cfl;
  a.pol.fixed_dt = c->cfg.fixed_dt;
  a.pol.dt_cap = 1.0e308;
  if (c->cfg.system == FV_SPRAY && c->cfg.params[1] > 0.0) a.pol.dt_cap = 0.5 * c->cfg.params[1];
  using PT = typename ParamOf<R>::T;
  if (c->cfg.system == FV_ADVECTION) {
    a.sp.p0 = (PT)c->cfg.params[0];
    a.sp.p1 = (PT)c->cfg.params[1];
  } else if (c->cfg.system == FV_EULER) {
    a.sp.p0 = (PT)c->cfg.params[0];
    a.sp.p1 = (PT)(c->cfg.params[0] - 1.0);
  }
  for (int s = 0; s < 4; ++s) {
    a.bc[s] = c->cfg.bc[s];
    for (int v = 0; v < 8; ++v) a.bc_state[s][v] = (PT)c->cfg.bc_state[s][v];
    // carried primitives of a Dirichlet ghost (slots 4..7)
    if (V.carry)
      for (int v = 0; v < 4; ++v) a.bc_state[s][4 + v] = (PT)c->bc_pc[s][v];
  }
  return a;
}

static fv_status launch_step(fv_ctx *c, cudaStream_t s) {
  const Variant &V = all_variants()[c->variant];
  dim3 grid(c->grid), block(V.NW * 32);
  cudaError_t e;
  DtPolicy pol;
  if (V.precision == 0) {
    StepArgs<double> a = make_args<double>(c, V);
    pol = a.pol;
    void *args[] = {&a};
    e = cudaLaunchKernel(V.kernel, grid, block, args, V.smem, s);
  } else if (V.precision == 1) {
    StepArgs<float> a = make_args<float>(c, V);
    pol = a.pol;
    void *args[] = {&a};
    e = cudaLaunchKernel(V.kernel, grid, block, args, V.smem, s);
  } else {
    StepArgs<__nv_bfloat16> a = make_args<__nv_bfloat16>(c, V);
    pol = a.pol;
    void *args[] = {&a};
    e = cudaLaunchKernel(V.kernel, grid, block, args, V.smem, s);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
  if (c->cfg.system == FV_SPRAY) {
    // split source step, Eq. (SourceTerm); it closes the step
    SourceLaunch L;
    L.prec = V.precision;
    L.buf0 = c->buf[0];
    L.buf1 = c->buf[1];
    L.ctrl = c->ctrl;
    L.lamw = c->lamw;
    L.ecache = c->ecache;
    L.nodes = c->nodes;
    L.nx = c->cfg.nx;
    L.ny = c->cfg.ny;
    L.pitch = c->pitch;
    L.plane = c->plane;
    L.dx = c->dx;
    L.dy = c->dy;
    L.xmin = c->cfg.xmin;
    L.ymin = c->cfg.ymin;
    L.pol = pol;
    L.K = c->cfg.params[0];
    L.theta = c->cfg.params[1];
    L.ug_mode = (int)c->cfg.params[2];
    L.Q = c->spray_Q;
    L.tol = c->cfg.params[4] > 0.0 ? c->cfg.params[4] : 1e-13;
    e = launch_spray_source(L, c->src_grid, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "spray source launch");
  }
  return FV_OK;
}

// One two-step pass (fv_tb.cuh) on stream s.
static fv_status launch_tb(fv_ctx *c, cudaStream_t s) {
  const Variant &V = all_variants()[c->tb_variant];
  dim3 grid(c->tb_grid), block(V.NW * 32);
  const void *k = c->tb_np ? V.kernel_np : V.kernel;
  cudaError_t e;
  if (V.precision == 0) {
    StepArgs<double> a = make_args<double>(c, V);
    void *args[] = {&a};
    e = cudaLaunchKernel(k, grid, block, args, V.smem, s);
  } else if (V.precision == 1) {
    StepArgs<float> a = make_args<float>(c, V);
    void *args[] = {&a};
    e = cudaLaunchKernel(k, grid, block, args, V.smem, s);
  } else {
    StepArgs<__nv_bfloat16> a = make_args<__nv_bfloat16>(c, V);
    void *args[] = {&a};
    e = cudaLaunchKernel(k, grid, block, args, V.smem, s);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "two-step kernel launch");
  return FV_OK;
}

// Graphs of n single steps (key n) or of n two-step passes (key -n).
static fv_status get_graph(fv_ctx *c, int nsteps, cudaGraphExec_t *out, bool passes = false) {
  const int key = passes ? -nsteps : nsteps;
  auto it = c->graphs.find(key);
  if (it != c->graphs.end()) {
    *out = it->second;
    return FV_OK;
  }
  if (c->graphs.size() > 16) free_graphs(c);
  FV_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  fv_status st = FV_OK;
  for (int k = 0; k < nsteps && st == FV_OK; ++k) st = passes ? launch_tb(c, c->cap_stream) : launch_step(c, c->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (st != FV_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  c->graphs[key] = ge;
  *out = ge;
  return FV_OK;
}

// Read the control block back after the work queued on the stream.  A
// kernel writes it into the mapped host mirror: a device-to-host memcpy of
// its 72 bytes would wait on the copy engine behind large copies other
// streams have running (an asynchronous snapshot of the state took 3.5 ms of
// the next job's load that way).
static fv_status read_ctrl(fv_ctx *c) {
  FV_CUDA(c, launch_ctrl_readback(c->ctrl, c->h_ctrl_dev, c->stream));
  FV_CUDA(c, cudaStreamSynchronize(c->stream));
  return FV_OK;
}

static fv_status status_of_flags(fv_ctx *c, unsigned e) {
  if (e & kErrTimeout) return fail(c, FV_ERR_TIMEOUT, "device wait timed out");
  if (e & kErrCfl) return fail(c, FV_ERR_CFL, "fixed dt * lmax > min(dx, dy)");
  if (e & kErrNonphysical) return fail(c, FV_ERR_NONPHYSICAL, "non-physical state reached");
  if (e & kErrZeroSpeed)
    return fail(c, FV_ERR_INVALID_ARG, "lmax = 0 leaves the adaptive time step unbounded");
  return FV_OK;
}

extern "C" fv_status fv_init(const fv_config *cfg, fv_ctx **out) {
  if (!out) return fail(nullptr, FV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  fv_status st = validate(cfg);
  if (st != FV_OK) return st;
  fv_ctx *c = new fv_ctx();
  c->cfg = *cfg;
  c->nvar = nvar_of(cfg->system);
  c->esize = cfg->precision == FV_F64 ? 8 : cfg->precision == FV_F32 ? 4 : 2;
  // pitch: a multiple of 32 elements (128 B in FP32, 256 B in FP64) so every
  // row and every V-wide vector access is aligned
  c->pitch = ((long long)cfg->nx + 31) / 32 * 32;
  c->plane = c->pitch * cfg->ny;
  c->nplanes = (cfg->system == FV_EULER && cfg->precision == FV_F64) ? 8 : c->nvar;
  c->buf_bytes = (size_t)c->plane * c->nplanes * c->esize;
  c->dx = (cfg->xmax - cfg->xmin) / cfg->nx;
  c->dy = (cfg->ymax - cfg->ymin) / cfg->ny;
  c->stream = (cudaStream_t)cfg->stream;
  cudaError_t e;
  if ((e = cudaGetDevice(&c->device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess) {
    cuda_fail(nullptr, e, "device query");
    delete c;
    return FV_ERR_CUDA;
  }
  auto bail = [&](cudaError_t e2, const char *what) {
    cuda_fail(nullptr, e2, what);
    fv_destroy(c);
    return e2 == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA;
  };
  if ((e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(e, "cudaStreamCreate");
  for (int b = 0; b < 2; ++b)
    if ((e = cudaMalloc(&c->buf[b], c->buf_bytes)) != cudaSuccess) return bail(e, "cudaMalloc(state)");
  if ((e = cudaMalloc(&c->ctrl, sizeof(Ctrl))) != cudaSuccess) return bail(e, "cudaMalloc(ctrl)");
  if ((e = cudaHostAlloc(&c->h_ctrl, sizeof(Ctrl), cudaHostAllocMapped)) != cudaSuccess)
    return bail(e, "cudaHostAlloc(ctrl mirror)");
  if ((e = cudaHostGetDevicePointer(&c->h_ctrl_dev, c->h_ctrl, 0)) != cudaSuccess)
    return bail(e, "cudaHostGetDevicePointer(ctrl mirror)");
  if ((e = cudaMallocHost(&c->h_scalar, 64)) != cudaSuccess) return bail(e, "cudaMallocHost");
  const int nb = totals_blocks(cfg->ny);
  if ((e = cudaMalloc(&c->partials, sizeof(double) * 2 * 8 * nb)) != cudaSuccess)
    return bail(e, "cudaMalloc(partials)");
  if ((e = cudaMalloc(&c->d_totals, sizeof(double) * 8)) != cudaSuccess) return bail(e, "cudaMalloc(totals)");
  if ((e = cudaMemset(c->ctrl, 0, sizeof(Ctrl))) != cudaSuccess) return bail(e, "cudaMemset");
  if (cfg->system == FV_SPRAY) {
    const int Q = cfg->params[3] > 0.0 ? (int)cfg->params[3] : 32;
    std::vector<double> x(Q), w(Q), tab((size_t)Q * kSprayNodeStride);
    fv_gauss_legendre(Q, x.data(), w.data());
    for (int q = 0; q < Q; ++q) {
      double *r = &tab[(size_t)q * kSprayNodeStride];
      r[0] = x[q];
      double xk = 1.0;
      for (int k = 0; k < 7; ++k) {
        r[1 + k] = w[q] * 2.0 * x[q] * xk;  // weight of S^(k/2) n(S) dS in x = sqrt(S)
        xk *= x[q];
      }
      r[8] = 2.0 * w[q];                    // weight of S^(-1/2) n(S) dS
    }
    c->spray_Q = Q;
    if ((e = cudaMalloc(&c->nodes, sizeof(double) * tab.size())) != cudaSuccess) return bail(e, "cudaMalloc(nodes)");
    if ((e = cudaMemcpy(c->nodes, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(e, "cudaMemcpy(nodes)");
    if ((e = cudaMalloc(&c->lamw, sizeof(double) * 12 * c->plane)) != cudaSuccess) return bail(e, "cudaMalloc(lamw)");
    if ((e = cudaMalloc(&c->ecache, sizeof(double) * Q * c->plane)) != cudaSuccess)
      return bail(e, "cudaMalloc(exponential cache)");
    c->src_grid = spray_source_grid(cfg->precision == FV_F64 ? 0 : 1, Q, c->sms);
  }
  if (c->nplanes > c->nvar) {
    // primitives of the boundary states, computed by the kernels' own prims
    double *d_bc = nullptr;
    double h_bc[32];
    for (int s2 = 0; s2 < 4; ++s2)
      for (int v = 0; v < 8; ++v) h_bc[8 * s2 + v] = cfg->bc_state[s2][v];
    if ((e = cudaMalloc(&d_bc, sizeof(double) * 48)) != cudaSuccess) return bail(e, "cudaMalloc(bc)");
    if ((e = cudaMemcpy(d_bc, h_bc, sizeof(h_bc), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = launch_bc_prims(d_bc, cfg->params[0], d_bc + 32, c->cap_stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->cap_stream)) != cudaSuccess ||
        (e = cudaMemcpy(&c->bc_pc[0][0], d_bc + 32, sizeof(double) * 16, cudaMemcpyDeviceToHost)) != cudaSuccess) {
      cudaFree(d_bc);
      return bail(e, "boundary primitives");
    }
    cudaFree(d_bc);
  }
  int prec = cfg->precision;  // 0 f64, 1 f32, 2 bf16 storage
  int vi = cfg->tune == 0 ? table_variant(cfg->system, prec, cfg->nx, cfg->ny, kTuneSingle, &c->choice) : -1;
  if (vi < 0) {
    vi = default_variant_for(cfg->system, prec, cfg->nx, cfg->ny, c->sms);
    c->choice = cfg->tune == 1 ? "autotuned: the fastest candidate on one timed step before the first run"
                               : kHeuristic;
  }
  if (cfg->tune >= 2) {
    auto cand = candidates(cfg->system, prec);
    if (cfg->tune - 2 >= (int)cand.size()) {
      fv_destroy(c);
      return fail(nullptr, FV_ERR_INVALID_ARG, "tune index out of range");
    }
    vi = cand[cfg->tune - 2];
    c->choice = "forced: candidate " + std::to_string(cfg->tune - 2);
  }
  if (vi < 0) {
    fv_destroy(c);
    return fail(nullptr, FV_ERR_INVALID_ARG, "no kernel built for this system and precision");
  }
  st = select_variant(c, vi);
  if (st != FV_OK) {
    g_init_error = c->err;
    fv_destroy(c);
    return st;
  }
  c->single_variant = vi;
  c->single_choice = c->choice;
  *out = c;
  return FV_OK;
}

extern "C" void fv_destroy(fv_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->snap_stream) {
    cudaStreamSynchronize(c->snap_stream);
    cudaStreamDestroy(c->snap_stream);
  }
  if (c->snap_ready) cudaEventDestroy(c->snap_ready);
  if (c->snap_done) cudaEventDestroy(c->snap_done);
  if (c->snap_buf) cudaFree(c->snap_buf);
  if (c->pre_stream) {
    cudaStreamSynchronize(c->pre_stream);
    cudaStreamDestroy(c->pre_stream);
  }
  if (c->pre_copied) cudaEventDestroy(c->pre_copied);
  if (c->pre_consumed) cudaEventDestroy(c->pre_consumed);
  if (c->pre_buf) cudaFree(c->pre_buf);
  free_graphs(c);
  for (int b = 0; b < 2; ++b)
    if (c->buf[b] && (b == 0 || c->buf[1] != c->buf[0])) cudaFree(c->buf[b]);
  if (c->ovl) cudaFree(c->ovl);
  if (c->ctrl) cudaFree(c->ctrl);
  if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
  if (c->h_scalar) cudaFreeHost(c->h_scalar);
  if (c->staging) cudaFree(c->staging);
  if (c->partials) cudaFree(c->partials);
  if (c->d_totals) cudaFree(c->d_totals);
  if (c->lamw) cudaFree(c->lamw);
  if (c->ecache) cudaFree(c->ecache);
  if (c->nodes) cudaFree(c->nodes);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

static fv_status ensure_staging(fv_ctx *c, size_t bytes) {
  if (c->staging_bytes >= bytes) return FV_OK;
  if (c->staging) {
    FV_CUDA(c, cudaStreamSynchronize(c->stream));
    cudaFree(c->staging);
    c->staging = nullptr;
    c->staging_bytes = 0;
  }
  FV_CUDA(c, cudaMalloc(&c->staging, bytes));
  c->staging_bytes = bytes;
  return FV_OK;
}

// Recompute lmax of the current state into slot `step % 3`, clear the other
// slots and report an inadmissible state.
// In-place mode: overlap strips of parity step % 2 from the state.
// The overlap strips of both parities from the state (the step reads those
// of parity step % 2; filling the other parity too leaves no strip cell
// unset, also the ones a ragged last strip never rewrites), and the four
// sides' prescribed states as stored cells after them.
static fv_status fill_ovl(fv_ctx *c, long long step) {
  (void)step;
  const Variant &V = all_variants()[c->variant];
  const int sw = 30 * V.V;
  const int nstrips = (c->cfg.nx + sw - 1) / sw, nchunks = (c->cfg.ny + V.TY - 1) / V.TY;
  // kernels that carry the primitives keep them in the strips too
  const int nv = V.carry ? c->nplanes : c->nvar;
  const long long total = (long long)nstrips * nchunks * nv * (2 * V.TY * V.V + 2 * sw);
  const int th = 256;
  const int g = (int)std::min<long long>((total + th - 1) / th, 4LL * c->sms * 8);
  const int p = c->cfg.precision;
  for (int parity = 0; parity < 2; ++parity) {
    void *dst = (char *)c->ovl + (parity ? c->ovl_parity_bytes : 0);
    if (p == 0)
      fill_ovl_kernel<double><<<g, th, 0, c->stream>>>((const double *)c->buf[0], c->cfg.nx, c->cfg.ny, c->pitch,
                                                       c->plane, nv, nstrips, nchunks, V.TY, V.V, sw, c->ovl_task,
                                                       (double *)dst);
    else if (p == 1)
      fill_ovl_kernel<float><<<g, th, 0, c->stream>>>((const float *)c->buf[0], c->cfg.nx, c->cfg.ny, c->pitch,
                                                      c->plane, nv, nstrips, nchunks, V.TY, V.V, sw, c->ovl_task,
                                                      (float *)dst);
    else
      fill_ovl_kernel<__nv_bfloat16><<<g, th, 0, c->stream>>>((const __nv_bfloat16 *)c->buf[0], c->cfg.nx,
                                                              c->cfg.ny, c->pitch, c->plane, nv, nstrips, nchunks,
                                                              V.TY, V.V, sw, c->ovl_task, (__nv_bfloat16 *)dst);
    FV_CUDA(c, cudaGetLastError());
  }
  // slots 4..7 of a Dirichlet state: its carried primitives, as make_args passes them
  void *bc = (char *)c->ovl + 2 * c->ovl_parity_bytes;
  auto bc_cells = [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    BcCells<S> b;
    for (int s2 = 0; s2 < 4; ++s2) {
      for (int v = 0; v < 8; ++v) b.v[s2][v] = (typename ParamOf<S>::T)c->cfg.bc_state[s2][v];
      if (V.carry)
        for (int v = 0; v < 4; ++v) b.v[s2][4 + v] = (typename ParamOf<S>::T)c->bc_pc[s2][v];
    }
    fill_bc_cells_kernel<S><<<1, 128, 0, c->stream>>>(b, nv, V.V, (S *)bc);
  };
  if (p == 0) bc_cells((double *)nullptr);
  else if (p == 1) bc_cells((float *)nullptr);
  else bc_cells((__nv_bfloat16 *)nullptr);
  FV_CUDA(c, cudaGetLastError());
  FV_CUDA(c, cudaStreamSynchronize(c->stream));
  return FV_OK;
}

// Planes 4..7 (carried primitives) of state buffer b from its planes 0..3.
static fv_status fill_prims(fv_ctx *c, unsigned b) {
  FV_CUDA(c, launch_fill_prims((double *)c->buf[b], c->cfg.nx, c->cfg.ny, c->pitch, c->plane, c->cfg.params[0],
                               c->stream));
  c->pc_dirty = false;
  return FV_OK;
}

// Before a kernel that reads carried primitives: refresh them when a kernel
// that does not carry them (in place, two steps per launch) wrote the state.
static fv_status ensure_prims(fv_ctx *c) {
  if (!c->pc_dirty || c->variant < 0 || !all_variants()[c->variant].carry) return FV_OK;
  fv_status st = read_ctrl(c);
  if (st != FV_OK) return st;
  return fill_prims(c, c->h_ctrl->cur);
}

static fv_status seed(fv_ctx *c, long long step, double t, unsigned cur) {
  Ctrl h;
  std::memset(&h, 0, sizeof(h));
  h.step = step;
  h.t = t;
  h.cur = cur;
  *c->h_ctrl = h;
  FV_CUDA(c, cudaMemcpyAsync(c->ctrl, c->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, c->stream));
  if (c->lamw)  // all-ones bytes are NaNs: every cell starts its Newton solve cold
    FV_CUDA(c, cudaMemsetAsync(c->lamw, 0xff, sizeof(double) * 12 * c->plane, c->stream));
  if (c->nplanes > c->nvar) {
    fv_status st0 = fill_prims(c, cur);
    if (st0 != FV_OK) return st0;
  }
  double p0 = c->cfg.params[0], p1 = c->cfg.params[1];
  if (c->cfg.system == FV_EULER) p1 = c->cfg.params[0] - 1.0;
  FV_CUDA(c, launch_seed_lambda(c->cfg.system, c->cfg.precision, c->buf[cur],
                                c->cfg.nx, c->cfg.ny, c->pitch, c->plane, p0, p1, c->ctrl,
                                (int)(step % 3), c->stream));
  fv_status st = read_ctrl(c);
  if (st != FV_OK) return st;
  unsigned bad = c->h_ctrl->err_pending;
  if (bad) {
    // keep nothing: clear the flag so a corrected state can be loaded later
    c->h_ctrl->err_pending = 0;
    FV_CUDA(c, cudaMemcpyAsync(c->ctrl, c->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, c->stream));
    FV_CUDA(c, cudaStreamSynchronize(c->stream));
    c->has_state = false;
    return fail(c, FV_ERR_NONPHYSICAL, "state has rho <= 0, p <= 0, non-finite or non-realizable values");
  }
  c->has_state = true;
  if (c->inplace) return fill_ovl(c, step);
  return FV_OK;
}

extern "C" fv_status fv_set_state(fv_ctx *c, const void *src, int src_is_device, int src_dtype,
                                  int layout) {
  if (!c) return FV_ERR_INVALID_ARG;
  if (!src) return fail(c, FV_ERR_INVALID_ARG, "src is NULL");
  if (src_dtype != FV_F64 && src_dtype != FV_F32) return fail(c, FV_ERR_INVALID_ARG, "bad src_dtype");
  if (layout != FV_CONSERVED && layout != FV_PRIMITIVE) return fail(c, FV_ERR_INVALID_ARG, "bad layout");
  const long long ncell = (long long)c->cfg.nx * c->cfg.ny;
  const size_t sbytes = (size_t)ncell * c->nvar * (src_dtype == FV_F64 ? 8 : 4);
  const void *dsrc = src;
  if (!src_is_device) {
    fv_status st = ensure_staging(c, sbytes);
    if (st != FV_OK) return st;
    FV_CUDA(c, cudaMemcpyAsync(c->staging, src, sbytes, cudaMemcpyHostToDevice, c->stream));
    dsrc = c->staging;
  }
  const int prec = c->cfg.precision;
  FV_CUDA(c, launch_load_state(c->cfg.system, prec, dsrc, src_dtype == FV_F32, layout == FV_PRIMITIVE,
                               c->buf[0], c->cfg.nx, c->cfg.ny, c->pitch, c->plane, c->cfg.params[0],
                               c->stream));
  return seed(c, 0, 0.0, 0u);
}

extern "C" fv_status fv_prefetch_state(fv_ctx *c, const void *src, int src_dtype, int layout) {
  if (!c) return FV_ERR_INVALID_ARG;
  if (!src) return fail(c, FV_ERR_INVALID_ARG, "src is NULL");
  if (src_dtype != FV_F64 && src_dtype != FV_F32) return fail(c, FV_ERR_INVALID_ARG, "bad src_dtype");
  if (layout != FV_CONSERVED && layout != FV_PRIMITIVE) return fail(c, FV_ERR_INVALID_ARG, "bad layout");
  if (!c->pre_stream) {
    FV_CUDA(c, cudaStreamCreateWithFlags(&c->pre_stream, cudaStreamNonBlocking));
    FV_CUDA(c, cudaEventCreateWithFlags(&c->pre_copied, cudaEventDisableTiming));
    FV_CUDA(c, cudaEventCreateWithFlags(&c->pre_consumed, cudaEventDisableTiming));
  }
  const size_t need = (size_t)c->cfg.nx * c->cfg.ny * c->nvar * (src_dtype == FV_F64 ? 8 : 4);
  if (c->pre_bytes < need) {
    // the old buffer may still be read by a queued load or written by a copy
    FV_CUDA(c, cudaStreamSynchronize(c->pre_stream));
    FV_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->pre_buf) cudaFree(c->pre_buf);
    c->pre_buf = nullptr;
    c->pre_bytes = 0;
    c->pre_used = false;
    FV_CUDA(c, cudaMalloc(&c->pre_buf, need));
    c->pre_bytes = need;
  }
  // the load of the previous prefetch must have read the buffer first
  if (c->pre_used) FV_CUDA(c, cudaStreamWaitEvent(c->pre_stream, c->pre_consumed, 0));
  FV_CUDA(c, cudaMemcpyAsync(c->pre_buf, src, need, cudaMemcpyHostToDevice, c->pre_stream));
  FV_CUDA(c, cudaEventRecord(c->pre_copied, c->pre_stream));
  c->pre_dtype = src_dtype;
  c->pre_layout = layout;
  c->pre_pending = true;
  return FV_OK;
}

extern "C" fv_status fv_set_state_prefetched(fv_ctx *c) {
  if (!c) return FV_ERR_INVALID_ARG;
  if (!c->pre_pending) return fail(c, FV_ERR_STATE, "no prefetched state");
  c->pre_pending = false;
  FV_CUDA(c, cudaStreamWaitEvent(c->stream, c->pre_copied, 0));
  FV_CUDA(c, launch_load_state(c->cfg.system, c->cfg.precision, c->pre_buf, c->pre_dtype == FV_F32,
                               c->pre_layout == FV_PRIMITIVE, c->buf[0], c->cfg.nx, c->cfg.ny, c->pitch,
                               c->plane, c->cfg.params[0], c->stream));
  FV_CUDA(c, cudaEventRecord(c->pre_consumed, c->stream));
  c->pre_used = true;
  return seed(c, 0, 0.0, 0u);
}

extern "C" fv_status fv_get_state(fv_ctx *c, void *dst, int dst_is_device, int dst_dtype) {
  if (!c) return FV_ERR_INVALID_ARG;
  if (!dst) return fail(c, FV_ERR_INVALID_ARG, "dst is NULL");
  if (dst_dtype != FV_F64 && dst_dtype != FV_F32) return fail(c, FV_ERR_INVALID_ARG, "bad dst_dtype");
  if (!c->has_state) return fail(c, FV_ERR_STATE, "no state set");
  fv_status st = read_ctrl(c);
  if (st != FV_OK) return st;
  const void *cur = c->buf[c->h_ctrl->cur];
  const int prec = c->cfg.precision;
  const size_t dsz = dst_dtype == FV_F64 ? 8 : 4;
  const bool same = (dst_dtype == FV_F64 && prec == 0) || (dst_dtype == FV_F32 && prec == 1);
  const long long ncell = (long long)c->cfg.nx * c->cfg.ny;
  if (same) {
    // planes are contiguous at stride ny * pitch: one 2D copy of nvar * ny rows
    FV_CUDA(c, cudaMemcpy2DAsync(dst, c->cfg.nx * dsz, cur, c->pitch * c->esize, c->cfg.nx * dsz,
                                 (size_t)c->nvar * c->cfg.ny,
                                 dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 c->stream));
  } else {
    void *target = dst;
    if (!dst_is_device) {
      st = ensure_staging(c, (size_t)ncell * c->nvar * dsz);
      if (st != FV_OK) return st;
      target = c->staging;
    }
    FV_CUDA(c, launch_store_state(prec, c->nvar, cur, target, dst_dtype == FV_F32, c->cfg.nx, c->cfg.ny,
                                  c->pitch, c->plane, c->stream));
    if (!dst_is_device)
      FV_CUDA(c, cudaMemcpyAsync(dst, c->staging, (size_t)ncell * c->nvar * dsz, cudaMemcpyDeviceToHost,
                                 c->stream));
  }
  FV_CUDA(c, cudaStreamSynchronize(c->stream));
  return FV_OK;
}

extern "C" fv_status fv_snapshot(fv_ctx *c, void *dst, int dst_dtype) {
  if (!c) return FV_ERR_INVALID_ARG;
  if (!dst) return fail(c, FV_ERR_INVALID_ARG, "dst is NULL");
  if (dst_dtype != FV_F64 && dst_dtype != FV_F32) return fail(c, FV_ERR_INVALID_ARG, "bad dst_dtype");
  if (!c->has_state) return fail(c, FV_ERR_STATE, "no state set");
  fv_status st = read_ctrl(c);
  if (st != FV_OK) return st;
  if (!c->snap_stream) {
    FV_CUDA(c, cudaStreamCreateWithFlags(&c->snap_stream, cudaStreamNonBlocking));
    FV_CUDA(c, cudaEventCreateWithFlags(&c->snap_ready, cudaEventDisableTiming));
    FV_CUDA(c, cudaEventCreateWithFlags(&c->snap_done, cudaEventDisableTiming));
  }
  const size_t need = (size_t)c->cfg.nx * c->cfg.ny * c->nvar * (dst_dtype == FV_F64 ? 8 : 4);
  if (c->snap_bytes < need) {
    if (c->snap_pending) FV_CUDA(c, cudaEventSynchronize(c->snap_done));
    c->snap_pending = false;
    if (c->snap_buf) cudaFree(c->snap_buf);
    c->snap_buf = nullptr;
    c->snap_bytes = 0;
    FV_CUDA(c, cudaMalloc(&c->snap_buf, need));
    c->snap_bytes = need;
  }
  // the previous host copy must be done before the staging buffer is refilled
  if (c->snap_pending) FV_CUDA(c, cudaStreamWaitEvent(c->stream, c->snap_done, 0));
  const void *cur = c->buf[c->h_ctrl->cur];
  FV_CUDA(c, launch_store_state(c->cfg.precision, c->nvar, cur, c->snap_buf, dst_dtype == FV_F32, c->cfg.nx,
                                c->cfg.ny, c->pitch, c->plane, c->stream));
  FV_CUDA(c, cudaEventRecord(c->snap_ready, c->stream));
  FV_CUDA(c, cudaStreamWaitEvent(c->snap_stream, c->snap_ready, 0));
  FV_CUDA(c, cudaMemcpyAsync(dst, c->snap_buf, need, cudaMemcpyDeviceToHost, c->snap_stream));
  FV_CUDA(c, cudaEventRecord(c->snap_done, c->snap_stream));
  c->snap_pending = true;
  return FV_OK;
}

extern "C" fv_status fv_snapshot_wait(fv_ctx *c) {
  if (!c) return FV_ERR_INVALID_ARG;
  if (!c->snap_pending) return FV_OK;
  FV_CUDA(c, cudaEventSynchronize(c->snap_done));
  c->snap_pending = false;
  return FV_OK;
}

// Autotuner: time every compiled candidate of this (system, precision) on
// one step from the current state and keep the fastest.  The control block
// is restored before every trial launch and at the end, so the state, t and
// n are untouched (a trial only writes the other ping-pong buffer).
static fv_status autotune(fv_ctx *c) {
  fv_status st = read_ctrl(c);
  if (st != FV_OK) return st;
  Ctrl saved = *c->h_ctrl;
  const Variant &cur = all_variants()[c->variant];
  auto cand = candidates(cur.system, cur.precision);
  cudaEvent_t e0, e1;
  FV_CUDA(c, cudaEventCreate(&e0));
  FV_CUDA(c, cudaEventCreate(&e1));
  int best = c->variant;
  float best_ms = 1e30f;
  for (int vi : cand) {
    st = select_variant(c, vi);
    if (st != FV_OK) break;
    std::vector<float> ms;
    for (int rep = 0; rep < 4 && st == FV_OK; ++rep) {
      *c->h_ctrl = saved;
      FV_CUDA(c, cudaMemcpyAsync(c->ctrl, c->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, c->stream));
      FV_CUDA(c, cudaEventRecord(e0, c->stream));
      st = launch_step(c, c->stream);
      FV_CUDA(c, cudaEventRecord(e1, c->stream));
      FV_CUDA(c, cudaEventSynchronize(e1));
      float t = 0;
      FV_CUDA(c, cudaEventElapsedTime(&t, e0, e1));
      if (rep > 0) ms.push_back(t);
    }
    if (st != FV_OK) break;
    std::sort(ms.begin(), ms.end());
    const float med = ms[ms.size() / 2];
    if (med < best_ms) {
      best_ms = med;
      best = vi;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *c->h_ctrl = saved;
  FV_CUDA(c, cudaMemcpyAsync(c->ctrl, c->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, c->stream));
  FV_CUDA(c, cudaStreamSynchronize(c->stream));
  if (st != FV_OK) return st;
  c->tuned = true;
  c->single_variant = best;
  return select_variant(c, best);
}

extern "C" fv_status fv_run(fv_ctx *c, int nsteps, double t_end, double *t_out) {
  if (!c) return FV_ERR_INVALID_ARG;
  if (nsteps < 0) return fail(c, FV_ERR_INVALID_ARG, "nsteps < 0");
  if (!c->has_state) return fail(c, FV_ERR_STATE, "no state set");
  if (!std::isfinite(t_end)) return fail(c, FV_ERR_INVALID_ARG, "t_end must be finite");
  {
    fv_status st0 = ensure_prims(c);
    if (st0 != FV_OK) return st0;
  }
  // (a trial step would overwrite the state in place: no tuning there)
  if (c->cfg.tune == 1 && !c->tuned && nsteps > 0 && !c->inplace) {
    fv_status st = autotune(c);
    if (st != FV_OK) return st;
  }
  *c->h_scalar = t_end;
  FV_CUDA(c, cudaMemcpyAsync(&c->ctrl->t_end, c->h_scalar, sizeof(double), cudaMemcpyHostToDevice,
                             c->stream));
  const int chunk = 64;
  int left = nsteps;
  if (c->tb_variant >= 0 && t_end <= 0.0 && nsteps >= 2) {
    // two steps per launch; a pass that finds W^{n+1} failing the paper's
    // check leaves everything as it was and flags kErrReplay, and the steps
    // from there are run one at a time (stopping where they would have)
    fv_status st = read_ctrl(c);
    if (st != FV_OK) return st;
    const long long start = c->h_ctrl->step;
    int passes = nsteps / 2;
    while (passes > 0) {
      const int n = passes >= chunk / 2 ? chunk / 2 : passes;
      cudaGraphExec_t g;
      st = get_graph(c, n, &g, true);
      if (st != FV_OK) return st;
      FV_CUDA(c, cudaGraphLaunch(g, c->stream));
      passes -= n;
    }
    // the two-step kernels update planes 0..3 only
    if (c->nplanes > c->nvar) c->pc_dirty = true;
    st = read_ctrl(c);
    if (st != FV_OK) return st;
    if (c->h_ctrl->err_committed & kErrReplay) {
      c->h_ctrl->err_committed &= ~kErrReplay;
      FV_CUDA(c, cudaMemcpyAsync(&c->ctrl->err_committed, &c->h_ctrl->err_committed, sizeof(unsigned),
                                 cudaMemcpyHostToDevice, c->stream));
    }
    left = nsteps - (int)(c->h_ctrl->step - start);
    if (left > 0) {
      st = ensure_prims(c);
      if (st != FV_OK) return st;
    }
  }
  if (left > 0 && c->nplanes > c->nvar && !all_variants()[c->variant].carry) c->pc_dirty = true;
  while (left > 0) {
    const int n = left >= chunk ? chunk : left;
    cudaGraphExec_t g;
    fv_status st = get_graph(c, n, &g);
    if (st != FV_OK) return st;
    FV_CUDA(c, cudaGraphLaunch(g, c->stream));
    left -= n;
  }
  fv_status st = read_ctrl(c);
  if (st != FV_OK) return st;
  if (t_out) *t_out = c->h_ctrl->t;
  return status_of_flags(c, c->h_ctrl->err_committed);
}

extern "C" fv_status fv_set_time_blocking(fv_ctx *c, int steps_per_pass) {
  if (!c) return FV_ERR_INVALID_ARG;
  if (steps_per_pass == 1) {
    c->tb_variant = -1;
    free_graphs(c);
    return FV_OK;
  }
  if (steps_per_pass != 2) return fail(c, FV_ERR_INVALID_ARG, "steps per pass must be 1 or 2");
  if (!(c->cfg.fixed_dt > 0.0)) return fail(c, FV_ERR_INVALID_ARG, "two steps per pass need the fixed-dt mode");
  if (c->inplace) return fail(c, FV_ERR_INVALID_ARG, "two steps per pass do not run in place");
  std::string how = kHeuristic;
  int vi = c->cfg.tune == 0
               ? table_variant(c->cfg.system, c->cfg.precision, c->cfg.nx, c->cfg.ny, kTuneTwoStep, &how)
               : -1;
  if (vi < 0) vi = default_variant_for(c->cfg.system, c->cfg.precision, c->cfg.nx, c->cfg.ny, c->sms, 0, 2);
  if (vi < 0) return fail(c, FV_ERR_INVALID_ARG, "no two-step kernel for this system and precision");
  if (c->cfg.tune >= 2) {
    // a forced candidate: the (tune - 2)-th two-step kernel of (system, precision)
    const auto &vs = all_variants();
    int k = 0;
    vi = -1;
    for (size_t q = 0; q < vs.size(); ++q)
      if (vs[q].system == c->cfg.system && vs[q].precision == c->cfg.precision && vs[q].tb == 2 &&
          k++ == c->cfg.tune - 2) {
        vi = (int)q;
        break;
      }
    if (vi < 0) return fail(c, FV_ERR_INVALID_ARG, "tune index out of range for two-step kernels");
    how = "forced: two-step candidate " + std::to_string(c->cfg.tune - 2);
  }
  const Variant &V = all_variants()[vi];
  bool np = false;
  for (int s2 = 0; s2 < 4; ++s2) np |= c->cfg.bc[s2] != FV_BC_PERIODIC;
  const void *kern = np ? V.kernel_np : V.kernel;
  if (!kern) return fail(c, FV_ERR_INVALID_ARG, "no two-step kernel for this system and precision");
  if (V.smem > 0)
    FV_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, V.smem));
  int nb = 0;
  FV_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, V.NW * 32, V.smem));
  if (nb < 1) return fail(c, FV_ERR_CUDA, std::string("kernel cannot launch: ") + V.desc);
  const long long ntasks = (long long)((c->cfg.nx + 30 * V.V - 1) / (30 * V.V)) * ((c->cfg.ny + V.TY - 1) / V.TY);
  long long grid = (long long)nb * c->sms, need = (ntasks + V.NW - 1) / V.NW;
  if (need < grid) grid = need;
  c->tb_variant = vi;
  c->tb_grid = (int)(grid < 1 ? 1 : grid);
  c->tb_np = np;
  c->tb_choice = how;
  free_graphs(c);
  return FV_OK;
}

extern "C" fv_status fv_step(fv_ctx *c, double *dt_used) {
  if (!c) return FV_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, FV_ERR_STATE, "no state set");
  fv_status st = read_ctrl(c);
  if (st != FV_OK) return st;
  const long long before = c->h_ctrl->step;
  st = fv_run(c, 1, 0.0, nullptr);
  if (dt_used) *dt_used = c->h_ctrl->step > before ? c->h_ctrl->dt_last : 0.0;
  return st;
}

extern "C" fv_status fv_totals(fv_ctx *c, double *totals) {
  if (!c) return FV_ERR_INVALID_ARG;
  if (!totals) return fail(c, FV_ERR_INVALID_ARG, "totals is NULL");
  if (!c->has_state) return fail(c, FV_ERR_STATE, "no state set");
  fv_status st = read_ctrl(c);
  if (st != FV_OK) return st;
  const int nb = totals_blocks(c->cfg.ny);
  FV_CUDA(c, launch_totals(c->cfg.precision, c->nvar, c->buf[c->h_ctrl->cur],
                           c->cfg.nx, c->cfg.ny, c->pitch, c->plane, c->partials, nb, c->d_totals,
                           c->dx * c->dy, c->stream));
  FV_CUDA(c, cudaMemcpyAsync(c->h_scalar, c->d_totals, sizeof(double) * c->nvar, cudaMemcpyDeviceToHost,
                             c->stream));
  FV_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int v = 0; v < c->nvar; ++v) totals[v] = c->h_scalar[v];
  return FV_OK;
}

extern "C" fv_status fv_time(fv_ctx *c, double *t, long long *step) {
  if (!c) return FV_ERR_INVALID_ARG;
  fv_status st = read_ctrl(c);
  if (st != FV_OK) return st;
  if (t) *t = c->h_ctrl->t;
  if (step) *step = c->h_ctrl->step;
  return FV_OK;
}

extern "C" fv_status fv_set_time(fv_ctx *c, double t, long long step) {
  if (!c) return FV_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, FV_ERR_STATE, "no state set");
  if (step < 0 || !std::isfinite(t)) return fail(c, FV_ERR_INVALID_ARG, "bad time or step");
  fv_status st = read_ctrl(c);
  if (st != FV_OK) return st;
  // the state stays in its buffer
  return seed(c, step, t, c->h_ctrl->cur);
}

extern "C" fv_status fv_lambda_max(fv_ctx *c, double *lmax) {
  if (!c || !lmax) return FV_ERR_INVALID_ARG;
  if (!c->has_state) return fail(c, FV_ERR_STATE, "no state set");
  fv_status st = read_ctrl(c);
  if (st != FV_OK) return st;
  *lmax = __builtin_bit_cast(double, c->h_ctrl->lam[c->h_ctrl->step % 3]);
  return FV_OK;
}

extern "C" fv_status fv_kernel_info(fv_ctx *c, int *variant, const char **desc) {
  if (!c) return FV_ERR_INVALID_ARG;
  const Variant &V = all_variants()[c->variant];
  if (variant) {
    auto cand = candidates(V.system, V.precision);
    int idx = 0;
    for (size_t k = 0; k < cand.size(); ++k)
      if (cand[k] == c->variant) idx = (int)k;
    *variant = idx;
  }
  if (desc) {
    c->desc = V.desc;
    if (!V.inplace && !V.tb && c->ty != V.TY) c->desc += ", " + std::to_string(c->ty) + "-row tasks";
    *desc = c->desc.c_str();
  }
  return FV_OK;
}

extern "C" const char *fv_kernel_info_two_step(const fv_ctx *c) {
  if (!c || c->tb_variant < 0) return nullptr;
  return all_variants()[c->tb_variant].desc;
}

// Gauss-Legendre rule on [0,1]: roots of P_Q by Newton's method on the
// three-term recurrence, weights 2/((1 - t^2) P_Q'(t)^2) halved for [0,1].
extern "C" fv_status fv_gauss_legendre(int Q, double *x, double *w) {
  if (Q < 1 || Q > 128 || !x || !w) return FV_ERR_INVALID_ARG;
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < Q; ++i) {
    double t = std::cos(pi * (4.0 * i + 3.0) / (4.0 * Q + 2.0));
    double pq = 0, pq1 = 0;
    for (int it = 0; it < 100; ++it) {
      double a = 1.0, b = t;  // P_0, P_1
      for (int k = 2; k <= Q; ++k) {
        double nxt = ((2.0 * k - 1.0) * t * b - (k - 1.0) * a) / k;
        a = b;
        b = nxt;
      }
      pq = Q == 0 ? 1.0 : b;
      pq1 = Q == 1 ? 1.0 : a;
      const double d = Q * (pq1 - t * pq) / (1.0 - t * t);  // P_Q'
      const double step = pq / d;
      t -= step;
      if (std::fabs(step) <= 1e-16 * std::fabs(t) + 1e-300) break;
    }
    double a = 1.0, b = t;
    for (int k = 2; k <= Q; ++k) {
      double nxt = ((2.0 * k - 1.0) * t * b - (k - 1.0) * a) / k;
      a = b;
      b = nxt;
    }
    pq1 = Q == 1 ? 1.0 : a;
    pq = b;
    const double d = Q * (pq1 - t * pq) / (1.0 - t * t);
    x[Q - 1 - i] = 0.5 * (1.0 + t);
    w[Q - 1 - i] = 1.0 / ((1.0 - t * t) * d * d);
  }
  return FV_OK;
}

extern "C" fv_status fv_set_inplace(fv_ctx *c, int on) {
  if (!c) return FV_ERR_INVALID_ARG;
  on = on ? 1 : 0;
  if (on == (int)c->inplace) return FV_OK;
  if (c->cfg.system == FV_SPRAY) return fail(c, FV_ERR_INVALID_ARG, "in-place mode: advection and Euler only");
  if (on && c->tb_variant >= 0) return fail(c, FV_ERR_INVALID_ARG, "in-place mode does not run two steps per pass");
  long long step = 0;
  if (c->has_state) {
    fv_status st = read_ctrl(c);
    if (st != FV_OK) return st;
    step = c->h_ctrl->step;
  }
  FV_CUDA(c, cudaStreamSynchronize(c->stream));
  if (on) {
    std::string how = kHeuristic;
    int vi = c->cfg.tune == 0
                 ? table_variant(c->cfg.system, c->cfg.precision, c->cfg.nx, c->cfg.ny, kTuneInplace, &how)
                 : -1;
    if (vi < 0) vi = default_variant_for(c->cfg.system, c->cfg.precision, c->cfg.nx, c->cfg.ny, c->sms, 1);
    if (vi < 0) return fail(c, FV_ERR_INVALID_ARG, "no in-place kernel for this system and precision");
    if (c->cfg.tune >= 2) {
      // a forced candidate: the (tune - 2)-th in-place kernel of (system, precision)
      const auto &vs = all_variants();
      int k = 0;
      vi = -1;
      for (size_t q = 0; q < vs.size(); ++q)
        if (vs[q].system == c->cfg.system && vs[q].precision == c->cfg.precision && vs[q].inplace &&
            k++ == c->cfg.tune - 2) {
          vi = (int)q;
          break;
        }
      if (vi < 0) return fail(c, FV_ERR_INVALID_ARG, "tune index out of range for in-place kernels");
      how = "forced: in-place candidate " + std::to_string(c->cfg.tune - 2);
    }
    const Variant &V = all_variants()[vi];
    const int sw = 30 * V.V;
    const long long ntasks = (long long)((c->cfg.nx + sw - 1) / sw) * ((c->cfg.ny + V.TY - 1) / V.TY);
    const int q = (int)(16 / c->esize);  // keep every task's strips 16-byte aligned
    const int nv = V.carry ? c->nplanes : c->nvar;  // strips hold the carried planes too
    const int ts = (nv * (2 * V.TY * V.V + 2 * sw) + q - 1) / q * q;
    const size_t pb = ((size_t)ntasks * ts * c->esize + 255) / 256 * 256;
    void *ovl = nullptr;
    // two parities of strips, then the sides' prescribed states as cells
    // (4 sides x up to 8 variables x 4 cells of up to 8 bytes)
    cudaError_t e = cudaMalloc(&ovl, 2 * pb + 1024);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc(overlap strips)");
    if (c->has_state && c->h_ctrl->cur == 1u) {
      // the state goes to buffer 0, which becomes the only one
      FV_CUDA(c, cudaMemcpyAsync(c->buf[0], c->buf[1], c->buf_bytes, cudaMemcpyDeviceToDevice, c->stream));
      c->h_ctrl->cur = 0u;
      FV_CUDA(c, cudaMemcpyAsync(c->ctrl, c->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, c->stream));
    }
    FV_CUDA(c, cudaStreamSynchronize(c->stream));
    cudaFree(c->buf[1]);
    c->buf[1] = c->buf[0];
    c->ovl = ovl;
    c->ovl_parity_bytes = pb;
    c->ovl_task = ts;
    c->inplace = true;
    c->choice = how;
    fv_status st = select_variant(c, vi);
    if (st != FV_OK) return st;
    if (c->has_state) {
      st = ensure_prims(c);  // the strips copy the carried planes of the state
      if (st != FV_OK) return st;
      return fill_ovl(c, step);
    }
    return FV_OK;
  }
  void *b1 = nullptr;
  cudaError_t e = cudaMalloc(&b1, c->buf_bytes);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc(state)");
  if (c->has_state && c->h_ctrl->cur != 0u) {
    // in place both indices name buffer 0, where the state is
    c->h_ctrl->cur = 0u;
    FV_CUDA(c, cudaMemcpyAsync(c->ctrl, c->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, c->stream));
  }
  FV_CUDA(c, cudaStreamSynchronize(c->stream));
  c->buf[1] = b1;
  cudaFree(c->ovl);
  c->ovl = nullptr;
  c->ovl_parity_bytes = 0;
  c->ovl_task = 0;
  c->inplace = false;
  c->choice = c->single_choice;
  return select_variant(c, c->single_variant);
}

extern "C" fv_status fv_kernel_choice(const fv_ctx *c, int two_step, const char **how) {
  if (!c || !how) return FV_ERR_INVALID_ARG;
  if (two_step) {
    if (c->tb_variant < 0) return fail(const_cast<fv_ctx *>(c), FV_ERR_STATE, "two steps per pass are off");
    *how = c->tb_choice.c_str();
  } else {
    *how = c->choice.c_str();
  }
  return FV_OK;
}

extern "C" fv_status fv_kernel_candidate(int system, int precision, int index, const char **desc) {
  if (!desc || (precision != FV_F64 && precision != FV_F32 && precision != FV_BF16)) return FV_ERR_INVALID_ARG;
  auto cand = candidates(system, precision);
  if (index < 0 || index >= (int)cand.size()) return FV_ERR_INVALID_ARG;
  *desc = all_variants()[cand[index]].desc;
  return FV_OK;
}
