// fv_noalloc.cu -- conservation totals of a caller-owned state with no device
// allocation by the library.
//
// Some callers cannot let a library allocate device memory: real-time or
// latency-bound loops that forbid allocator calls and the synchronisation
// cudaMalloc/cudaFree can cause, and frameworks that hand all device memory
// out of their own pool and account for every byte.  fv_totals_noalloc
// serves them: it computes the same per-variable totals as fv_totals, but its
// per-block partial sums live in a fixed array compiled into the library's
// device image (a file-scope static __device__ array), so no cudaMalloc,
// cudaFree or allocating library routine is ever called.
//
// The array holds 2 x 8 x 1024 doubles (128 KiB).  Every GPU that loads the
// library holds its own copy until the process exits.  All calls on a device
// share it and it keeps the last call's contents; each call writes every
// partial sum before reading it back, so nothing needs clearing between
// calls.  Two calls whose work overlaps on the GPU (for example on two
// streams with no ordering between them) race on the array: the caller must
// order them.  The array's device address is looked up once per device and
// kept; a cudaDeviceReset destroys the context that address belongs to, so
// calling this entry point after one in the same process is not supported.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fv.h"
#include "fv_internal.h"

namespace fv {

constexpr int kNoAllocMaxVar = 8;
constexpr int kNoAllocMaxBlocks = 1024;  // totals_blocks() never exceeds this
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_totals_scratch[2 * kNoAllocMaxVar * kNoAllocMaxBlocks];

// Device address of the scratch array on the current device.  In host code
// the array's name only stands for it; the address must be asked for once per
// device, with that device current, which the first call on each device does.
static fv_status scratch_address(double **out) {
  static std::mutex mu;
  static double *addr[kNoAllocMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_global_error(std::string("fv_totals_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_global_error("fv_totals_noalloc: device index beyond 63");
    return FV_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_totals_scratch);
    if (e != cudaSuccess || !p) {
      set_global_error(std::string("fv_totals_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return FV_ERR_CUDA;
    }
    addr[dev] = static_cast<double *>(p);
  }
  *out = addr[dev];
  return FV_OK;
}

}  // namespace fv

using namespace fv;

extern "C" fv_status fv_totals_noalloc(const void *state, int dtype, int nvar, int nx, int ny, double cell_area,
                                       double *totals, void *stream) {
  if (!state || !totals) {
    set_global_error("fv_totals_noalloc: state and totals must be device pointers");
    return FV_ERR_INVALID_ARG;
  }
  if (dtype != FV_F64 && dtype != FV_F32) {
    set_global_error("fv_totals_noalloc: dtype must be FV_F64 or FV_F32");
    return FV_ERR_INVALID_ARG;
  }
  if (nvar < 1 || nvar > kNoAllocMaxVar) {
    set_global_error("fv_totals_noalloc: nvar must be between 1 and 8 (the fixed scratch holds 8 variables)");
    return FV_ERR_INVALID_ARG;
  }
  if (nx < 1 || ny < 1 || !(cell_area > 0.0)) {
    set_global_error("fv_totals_noalloc: need nx, ny >= 1 and cell_area > 0");
    return FV_ERR_INVALID_ARG;
  }
  const int nblocks = totals_blocks(ny);
  if (nblocks > kNoAllocMaxBlocks) {
    set_global_error("fv_totals_noalloc: more partial sums than the fixed scratch holds");
    return FV_ERR_INVALID_ARG;
  }
  double *scratch = nullptr;
  fv_status st = scratch_address(&scratch);
  if (st != FV_OK) return st;
  const long long pitch = nx, plane = (long long)nx * ny;  // the ABI's contiguous layout
  cudaError_t e = launch_totals(dtype == FV_F64 ? 0 : 1, nvar, state, nx, ny, pitch, plane, scratch, nblocks,
                                totals, cell_area, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_global_error(std::string("fv_totals_noalloc: launch: ") + cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  return FV_OK;
}
