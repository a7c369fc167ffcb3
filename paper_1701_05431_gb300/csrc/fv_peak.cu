// fv_peak.cu -- measured throughput of the FP64 and FP32 fused multiply-add
// pipes of the current GPU.
//
// The FP64 Euler step and the spray source's maximum-entropy Newton solve are
// bound by GB300's FP64 pipe, not by HBM, so their roofline needs the rate at
// which that pipe retires fused multiply-adds.  fv_fma_peak measures it the
// way a copy test measures HBM: every thread runs four or eight independent
// chains of a = a * b + c (no loads, no stores, enough warps on every SM to
// hide the pipe's latency), and the rate is FMAs retired / CUDA-event time of
// the launch, the better of the two chain counts.  The chains converge to
// c / (1 - b), about 1, so no value overflows or turns subnormal; the final
// sum is compared with a value it can never take, which keeps the chains
// live without storing anything.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/fv.h"
#include "fv_internal.h"

namespace fv {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSM = 8;  // 2048 threads: a full SM
constexpr int kPeakUnroll = 8;       // FMAs per chain per loop trip

static __device__ double g_peak_sink;

// b and c differ per thread (by far less than they matter), so that every
// operand is a register: with b and c read from the constant bank (shared by
// the grid) the FP64 pipe was busy 84% of the time, with register operands
// 99.5% (ncu, 152 SMs).
template <typename T, int CHAINS>
__global__ void __launch_bounds__(kPeakThreads) fma_chain_kernel(int iters, T b0, T c0) {
  const T b = b0 + (T)threadIdx.x * (T)1e-12;
  const T c = c0 * ((T)1 + (T)threadIdx.x * (T)1e-9);
  T a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < kPeakUnroll; ++r)
#pragma unroll
      for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  T s = (T)0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += a[k];
  if (s == (T)-1) g_peak_sink = (double)s;  // every a[k] stays positive
}

template <typename T, int CHAINS>
static cudaError_t time_launch(int grid, int iters, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                               float *ms) {
  cudaError_t e;
  if ((e = cudaEventRecord(e0, st)) != cudaSuccess) return e;
  fma_chain_kernel<T, CHAINS><<<grid, kPeakThreads, 0, st>>>(iters, (T)0.9999, (T)1e-4);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaEventRecord(e1, st)) != cudaSuccess) return e;
  if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
  return cudaEventElapsedTime(ms, e0, e1);
}

template <typename T, int CHAINS>
static cudaError_t measure(double seconds, cudaStream_t st, double *rate) {
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int grid = sms * kPeakBlocksPerSM;
  const double per_trip = (double)grid * kPeakThreads * CHAINS * kPeakUnroll;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  float ms = 0.f;
  // calibration (also the warm-up): 64 trips, then as many trips as take
  // about `seconds`; the best of three timed launches
  int iters = 64;
  e = time_launch<T, CHAINS>(grid, iters, st, e0, e1, &ms);
  if (e == cudaSuccess) {
    const double scale = seconds * 1e3 / std::max(ms, 1e-3f);
    iters = (int)std::min(2.0e9, std::max(64.0, iters * scale));
    float best = 0.f;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
      e = time_launch<T, CHAINS>(grid, iters, st, e0, e1, &ms);
      if (e == cudaSuccess && (k == 0 || ms < best)) best = ms;
    }
    if (e == cudaSuccess) *rate = per_trip * iters / (best * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace fv

using namespace fv;

extern "C" fv_status fv_fma_peak(int precision, double seconds, double *fma_per_s, void *stream) {
  if (!fma_per_s || (precision != FV_F64 && precision != FV_F32)) {
    set_global_error("fv_fma_peak: precision must be FV_F64 or FV_F32 and fma_per_s non-NULL");
    return FV_ERR_INVALID_ARG;
  }
  if (!(seconds >= 1e-3 && seconds <= 2.0)) {
    set_global_error("fv_fma_peak: seconds must lie in [0.001, 2]");
    return FV_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // the best of two chain counts per thread (4 and 8 independent chains)
  double r4 = 0.0, r8 = 0.0;
  cudaError_t e = precision == FV_F64 ? measure<double, 4>(seconds, st, &r4) : measure<float, 4>(seconds, st, &r4);
  if (e == cudaSuccess)
    e = precision == FV_F64 ? measure<double, 8>(seconds, st, &r8) : measure<float, 8>(seconds, st, &r8);
  *fma_per_s = r4 > r8 ? r4 : r8;
  if (e != cudaSuccess) {
    set_global_error(std::string("fv_fma_peak: ") + cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  return FV_OK;
}
