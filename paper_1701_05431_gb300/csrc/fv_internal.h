// fv_internal.h -- host-side declarations shared by the library's translation
// units (kernel variant registry and auxiliary kernel launchers).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "fv_device.cuh"

namespace fv {

// One compiled step-kernel candidate.
struct Variant {
  int system;      // kAdvection / kEuler / kSpray
  int precision;   // 0: f64, 1: f32
  int V;           // cells per lane along x (values per lane x cells per value)
  int TY;          // rows per warp task
  int NW;          // warps per block
  int MINB;        // blocks per SM the register budget is cut for
  int D;           // row staging: 0 register prefetch, > 0 TMA ring depth, < 0 cp.async ring depth
  int smem;        // dynamic shared memory per block (bytes)
  const void *kernel;
  const char *desc;
  int inplace;     // 1: in-place kernel (one state buffer plus overlap strips)
  int tb;          // 2: two time steps per launch (fixed dt, periodic); 0: one
  int carry = 0;   // 1: FP64 Euler with carried primitives (planes 4..7 of the state)
  const void *kernel_np = nullptr;  // two-step kernels: the build for grids with a non-periodic side
};

// Registration hooks, one per translation unit of step kernels.
void register_step_advection(std::vector<Variant> &out);
void register_step_euler(std::vector<Variant> &out);
void register_step_euler_tb(std::vector<Variant> &out);
void register_step_spray(std::vector<Variant> &out);

const std::vector<Variant> &all_variants();

// Auxiliary kernels (fv_aux.cu).  `R` storage precision: 0 f64, 1 f32.
cudaError_t launch_load_state(int system, int prec, const void *src, int src_f32, int primitive,
                              void *state, int nx, int ny, long long pitch, long long plane,
                              double gamma, cudaStream_t s);
cudaError_t launch_store_state(int prec, int nvar, const void *state, void *dst, int dst_f32, int nx,
                               int ny, long long pitch, long long plane, cudaStream_t s);
cudaError_t launch_seed_lambda(int system, int prec, const void *state, int nx, int ny,
                               long long pitch, long long plane, double p0, double p1, Ctrl *ctrl,
                               int slot, cudaStream_t s);
cudaError_t launch_totals(int prec, int nvar, const void *state, int nx, int ny, long long pitch,
                          long long plane, double *partials, int nblocks, double *out,
                          double cell_area, cudaStream_t s);
int totals_blocks(int ny);
// Copy the control block into host memory mapped for the device, by a kernel
// on stream s (no copy engine: a small device-to-host copy would queue behind
// large copies already running on the engine, such as a snapshot's).
cudaError_t launch_ctrl_readback(const Ctrl *src, Ctrl *dst_mapped, cudaStream_t s);
// FP64 Euler with carried primitives: planes 4..7 (u, v, p, c) of a state
// from its planes 0..3, and the same of the four boundary states (bc_dev:
// 4 x 8 doubles, out_dev: 4 x 4 doubles).
cudaError_t launch_fill_prims(double *state, int nx, int ny, long long pitch, long long plane, double gamma,
                              cudaStream_t s);
cudaError_t launch_bc_prims(const double *bc_dev, double gamma, double *out_dev, cudaStream_t s);

// Record the message fv_last_error(NULL) returns (fv_host.cu).
void set_global_error(const std::string &msg);

// Spray source step (fv_spray.cu).
struct SourceLaunch {
  int prec;
  void *buf0, *buf1;
  Ctrl *ctrl;
  double *lamw;
  double *ecache;        // Q planes: the exponentials of the last solve (nullable)
  const double *nodes;
  int nx, ny;
  long long pitch, plane;
  double dx, dy, xmin, ymin;
  DtPolicy pol;
  double K, theta, tol;
  int ug_mode, Q;
};
int spray_source_grid(int prec, int Q, int sms);
cudaError_t launch_spray_source(const SourceLaunch &L, int grid, cudaStream_t s);
constexpr int kSprayNodeStride = 9;

}  // namespace fv
