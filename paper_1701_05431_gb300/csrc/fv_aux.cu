// fv_aux.cu -- auxiliary kernels around the fused step: loading a state
// (with the primitive -> conserved map of the initial condition,
// Eq. (initial_condition)), storing it back in a caller's dtype, the seed
// reduction of lmax(W^0) for the first dt (Eq. (CFL_cond)) and the
// compensated conservation totals.
#include <cuda_runtime.h>

#include <type_traits>

#include "fv_device.cuh"
#include "fv_internal.h"

namespace fv {

// ------------------------------------------------------------------ load
template <class S>
static __device__ __forceinline__ double rd(const S *p, long long k) { return (double)p[k]; }

// a / c correctly rounded for a divisor c fixed for the whole launch, from
// y = RN(1/c): q = RN(a y) is within an ulp of a / c, the remainder
// a - c q is then exact (one FMA), and RN(q + (a - c q) y) is RN(a / c)
// (Markstein, IBM J. Res. Dev. 34(1), 1990; round to nearest, no overflow or
// underflow).  Three FP64 operations instead of a division per cell.
static __device__ __forceinline__ double div_by(double a, double c, double y) {
  const double q = __dmul_rn(a, y);
  const double r = __fma_rn(-c, q, a);
  return __fma_rn(r, y, q);
}

// Narrowing of a double to a storage type (round to nearest even).
template <class R> static __device__ __forceinline__ R from_double(double x) { return (R)x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double x) {
  return __double2bfloat16(x);
}

// Threads stride along a row, blocks along y over rows (no integer division
// per cell).  src is contiguous nvar x ny x nx; state is pitched.
// Primitive -> conserved, in FP64 and in the same operation order as the
// definition: rho E = p/(gamma - 1) + rho (u u + v v)/2; momenta = rho u, rho v
// (Euler) or m1 u, m1 v (spray).
template <class S, class R>
__global__ void load_state_kernel(int system, const S *__restrict__ src, int primitive,
                                  R *__restrict__ state, int nx, int ny, long long pitch,
                                  long long plane, double gamma) {
  const long long ncell = (long long)nx * ny;
  const double gm1 = __dsub_rn(gamma, 1.0), inv_gm1 = __drcp_rn(gm1);
  for (int j = blockIdx.y; j < ny; j += gridDim.y)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x) {
    const long long k = (long long)j * nx + i;
    const long long o = (long long)j * pitch + i;
    if (system == kAdvection) {
      state[o] = from_double<R>(rd(src, k));
    } else if (std::is_same<S, float>::value && std::is_same<R, float>::value && system == kEuler) {
      // FP32 in, FP32 state: a product of two FP32 values is exact in FP64,
      // so rounding it to FP32 is the FP32 product; only rho E needs FP64
      const float rho = (float)src[k], a1 = (float)src[ncell + k], a2 = (float)src[2 * ncell + k],
                  a3 = (float)src[3 * ncell + k];
      float w1 = a1, w2 = a2, w3 = a3;
      if (primitive) {
        const double u = a1, v = a2;
        w1 = __fmul_rn(rho, a1);
        w2 = __fmul_rn(rho, a2);
        const double q = __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v));
        w3 = (float)__dadd_rn(div_by((double)a3, gm1, inv_gm1),
                              __dmul_rn(__dmul_rn((double)rho, q), 0.5));
      }
      state[o] = (R)rho;
      state[plane + o] = (R)w1;
      state[2 * plane + o] = (R)w2;
      state[3 * plane + o] = (R)w3;
    } else if (system == kEuler) {
      double w0 = rd(src, k), w1 = rd(src, ncell + k), w2 = rd(src, 2 * ncell + k),
             w3 = rd(src, 3 * ncell + k);
      if (primitive) {
        const double rho = w0, u = w1, v = w2, p = w3;
        w1 = __dmul_rn(rho, u);
        w2 = __dmul_rn(rho, v);
        const double q = __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v));
        // (halving is exact: the product by 0.5 is the quotient by 2)
        w3 = __dadd_rn(div_by(p, gm1, inv_gm1), __dmul_rn(__dmul_rn(rho, q), 0.5));
      }
      state[o] = from_double<R>(w0);
      state[plane + o] = from_double<R>(w1);
      state[2 * plane + o] = from_double<R>(w2);
      state[3 * plane + o] = from_double<R>(w3);
    } else {
      double w[6];
#pragma unroll
      for (int v = 0; v < 6; ++v) w[v] = rd(src, v * ncell + k);
      if (primitive) {
        w[4] = __dmul_rn(w[2], w[4]);
        w[5] = __dmul_rn(w[2], w[5]);
      }
#pragma unroll
      for (int v = 0; v < 6; ++v) state[v * plane + o] = from_double<R>(w[v]);
    }
  }
}

// Blocks of `threads` along x (a row) and over rows along y, about 32 per SM
// of a 152-SM GPU in all.
static dim3 grid_for(int nx, int ny, int threads) {
  int gx = (nx + threads - 1) / threads;
  if (gx > 64) gx = 64;
  if (gx < 1) gx = 1;
  int gy = 152 * 32 / gx;
  if (gy > ny) gy = ny;
  if (gy < 1) gy = 1;
  return dim3((unsigned)gx, (unsigned)gy);
}

cudaError_t launch_load_state(int system, int prec, const void *src, int src_f32, int primitive,
                              void *state, int nx, int ny, long long pitch, long long plane,
                              double gamma, cudaStream_t s) {
  const int th = 256;
  const dim3 g = grid_for(nx, ny, th);
  if (prec == 0) {
    if (src_f32)
      load_state_kernel<float, double><<<g, th, 0, s>>>(system, (const float *)src, primitive,
                                                        (double *)state, nx, ny, pitch, plane, gamma);
    else
      load_state_kernel<double, double><<<g, th, 0, s>>>(system, (const double *)src, primitive,
                                                         (double *)state, nx, ny, pitch, plane, gamma);
  } else if (prec == 1) {
    if (src_f32)
      load_state_kernel<float, float><<<g, th, 0, s>>>(system, (const float *)src, primitive,
                                                       (float *)state, nx, ny, pitch, plane, gamma);
    else
      load_state_kernel<double, float><<<g, th, 0, s>>>(system, (const double *)src, primitive,
                                                        (float *)state, nx, ny, pitch, plane, gamma);
  } else {
    if (src_f32)
      load_state_kernel<float, __nv_bfloat16><<<g, th, 0, s>>>(system, (const float *)src, primitive,
                                                               (__nv_bfloat16 *)state, nx, ny, pitch, plane, gamma);
    else
      load_state_kernel<double, __nv_bfloat16><<<g, th, 0, s>>>(system, (const double *)src, primitive,
                                                                (__nv_bfloat16 *)state, nx, ny, pitch, plane, gamma);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ store
template <class R, class D>
__global__ void store_state_kernel(int nvar, const R *__restrict__ state, D *__restrict__ dst, int nx,
                                   int ny, long long pitch, long long plane) {
  const long long ncell = (long long)nx * ny;
  for (int j = blockIdx.y; j < ny; j += gridDim.y)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x) {
    const long long k = (long long)j * nx + i;
    const long long o = (long long)j * pitch + i;
    for (int v = 0; v < nvar; ++v) dst[v * ncell + k] = (D)to_double(state[v * plane + o]);
  }
}

cudaError_t launch_store_state(int prec, int nvar, const void *state, void *dst, int dst_f32, int nx,
                               int ny, long long pitch, long long plane, cudaStream_t s) {
  const int th = 256;
  const dim3 g = grid_for(nx, ny, th);
  if (prec == 0) {
    if (dst_f32)
      store_state_kernel<double, float><<<g, th, 0, s>>>(nvar, (const double *)state, (float *)dst, nx,
                                                         ny, pitch, plane);
    else
      store_state_kernel<double, double><<<g, th, 0, s>>>(nvar, (const double *)state, (double *)dst,
                                                          nx, ny, pitch, plane);
  } else if (prec == 1) {
    if (dst_f32)
      store_state_kernel<float, float><<<g, th, 0, s>>>(nvar, (const float *)state, (float *)dst, nx,
                                                        ny, pitch, plane);
    else
      store_state_kernel<float, double><<<g, th, 0, s>>>(nvar, (const float *)state, (double *)dst, nx,
                                                         ny, pitch, plane);
  } else {
    if (dst_f32)
      store_state_kernel<__nv_bfloat16, float><<<g, th, 0, s>>>(nvar, (const __nv_bfloat16 *)state, (float *)dst,
                                                                nx, ny, pitch, plane);
    else
      store_state_kernel<__nv_bfloat16, double><<<g, th, 0, s>>>(nvar, (const __nv_bfloat16 *)state,
                                                                 (double *)dst, nx, ny, pitch, plane);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ seed lmax
// lmax(W^0) and admissibility of a freshly loaded state, with the same
// per-cell function the step kernel applies to every new state.
template <class Sys, class A>
__global__ void seed_lambda_kernel(const typename Ops<A>::S *__restrict__ state, int nx, int ny, long long pitch,
                                   long long plane, SysParams<typename Ops<A>::P> Pp, Ctrl *ctrl, int slot) {
  constexpr int NV = Sys::NV;
  const SysParams<A> P = splat_params<A>(Pp);
  typename Ops<A>::P l = 0;
  bool bad = false;
  for (int j = blockIdx.y; j < ny; j += gridDim.y)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x) {
    const long long o = (long long)j * pitch + i;
    A W[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) W[v] = Ops<A>::pack(state + v * plane + o);
    unsigned b;
    const A lc = Sys::lambda(W, P, b);
    bad |= b != 0u;
    l = fmax(l, Ops<A>::hmax(lc, 1u));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l = fmax(l, __shfl_xor_sync(0xffffffffu, l, o));
  const int anybad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (l > 0) atomicMax(&ctrl->lam[slot], lam_bits((double)l));
    if (anybad) atomicOr(&ctrl->err_pending, kErrNonphysical);
  }
}

// The control block copied by one warp into host memory mapped for the
// device (its 8-byte words, one per lane).
__global__ void ctrl_readback_kernel(const Ctrl *__restrict__ src, Ctrl *dst) {
  constexpr int words = (int)(sizeof(Ctrl) / sizeof(unsigned long long));
  static_assert(sizeof(Ctrl) % sizeof(unsigned long long) == 0 && words <= 32, "control block of 8-byte words");
  const int l = threadIdx.x;
  if (l < words)
    reinterpret_cast<volatile unsigned long long *>(dst)[l] = __ldcg(reinterpret_cast<const unsigned long long *>(src) + l);
}

cudaError_t launch_ctrl_readback(const Ctrl *src, Ctrl *dst_mapped, cudaStream_t s) {
  ctrl_readback_kernel<<<1, 32, 0, s>>>(src, dst_mapped);
  return cudaGetLastError();
}

cudaError_t launch_seed_lambda(int system, int prec, const void *state, int nx, int ny,
                               long long pitch, long long plane, double p0, double p1, Ctrl *ctrl,
                               int slot, cudaStream_t s) {
  const int th = 256;
  const dim3 g = grid_for(nx, ny, th);
  if (prec == 0) {
    SysParams<double> P{p0, p1};
    const double *st = (const double *)state;
    if (system == kAdvection) seed_lambda_kernel<Advection, double><<<g, th, 0, s>>>(st, nx, ny, pitch, plane, P, ctrl, slot);
    else if (system == kEuler) seed_lambda_kernel<Euler, double><<<g, th, 0, s>>>(st, nx, ny, pitch, plane, P, ctrl, slot);
    else seed_lambda_kernel<Spray, double><<<g, th, 0, s>>>(st, nx, ny, pitch, plane, P, ctrl, slot);
  } else if (prec == 1) {
    SysParams<float> P{(float)p0, (float)p1};
    const float *st = (const float *)state;
    if (system == kAdvection) seed_lambda_kernel<Advection, float><<<g, th, 0, s>>>(st, nx, ny, pitch, plane, P, ctrl, slot);
    else if (system == kEuler) seed_lambda_kernel<Euler, float><<<g, th, 0, s>>>(st, nx, ny, pitch, plane, P, ctrl, slot);
    else seed_lambda_kernel<Spray, float><<<g, th, 0, s>>>(st, nx, ny, pitch, plane, P, ctrl, slot);
  } else {
    SysParams<float> P{(float)p0, (float)p1};
    const __nv_bfloat16 *st = (const __nv_bfloat16 *)state;
    if (system == kAdvection) seed_lambda_kernel<Advection, BF><<<g, th, 0, s>>>(st, nx, ny, pitch, plane, P, ctrl, slot);
    else if (system == kEuler) seed_lambda_kernel<Euler, BF><<<g, th, 0, s>>>(st, nx, ny, pitch, plane, P, ctrl, slot);
    else return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ carried primitives
// Planes 4..7 of an FP64 Euler state (u, v, p, c of every cell, Euler::prims
// of planes 0..3), for the kernels that carry them from step to step.
__global__ void fill_prims_kernel(double *__restrict__ state, int nx, int ny, long long pitch, long long plane,
                                  SysParams<double> P) {
  for (int j = blockIdx.y; j < ny; j += gridDim.y)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x) {
    const long long o = (long long)j * pitch + i;
    const double W[4] = {state[o], state[plane + o], state[2 * plane + o], state[3 * plane + o]};
    double u, v, p, c;
    Euler::prims(W, P, u, v, p, c);
    state[4 * plane + o] = u;
    state[5 * plane + o] = v;
    state[6 * plane + o] = p;
    state[7 * plane + o] = c;
  }
}

// The same four values of the four boundary states (Dirichlet ghosts).
__global__ void bc_prims_kernel(const double *__restrict__ bc, SysParams<double> P, double *__restrict__ out) {
  const int s = threadIdx.x;
  if (s >= 4) return;
  const double W[4] = {bc[8 * s], bc[8 * s + 1], bc[8 * s + 2], bc[8 * s + 3]};
  Euler::prims(W, P, out[4 * s], out[4 * s + 1], out[4 * s + 2], out[4 * s + 3]);
}

cudaError_t launch_fill_prims(double *state, int nx, int ny, long long pitch, long long plane, double gamma,
                              cudaStream_t s) {
  const int th = 256;
  const dim3 g = grid_for(nx, ny, th);
  SysParams<double> P{gamma, gamma - 1.0};
  fill_prims_kernel<<<g, th, 0, s>>>(state, nx, ny, pitch, plane, P);
  return cudaGetLastError();
}

cudaError_t launch_bc_prims(const double *bc_dev, double gamma, double *out_dev, cudaStream_t s) {
  SysParams<double> P{gamma, gamma - 1.0};
  bc_prims_kernel<<<1, 32, 0, s>>>(bc_dev, P, out_dev);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ totals
// Neumaier compensated summation: s + c tracks the exact running sum far
// better than s alone.
struct Neu {
  double s, c;
};
static __device__ __forceinline__ void neu_add(Neu &a, double x) {
  const double t = __dadd_rn(a.s, x);
  if (fabs(a.s) >= fabs(x)) a.c = __dadd_rn(a.c, __dadd_rn(__dsub_rn(a.s, t), x));
  else a.c = __dadd_rn(a.c, __dadd_rn(__dsub_rn(x, t), a.s));
  a.s = t;
}
static __device__ __forceinline__ void neu_merge(Neu &a, const Neu &b) {
  neu_add(a, b.s);
  a.c = __dadd_rn(a.c, b.c);
}

constexpr int kTotThreads = 256;

int totals_blocks(int ny) { return ny < 1024 ? ny : 1024; }

// Block b sums rows b, b + gridDim.x, ...; within a block, threads stride
// along x; the block combines its threads in a fixed tree order.
template <class R>
__global__ void totals_partial_kernel(int nvar, const R *__restrict__ state, int nx, int ny,
                                      long long pitch, long long plane, double *partials) {
  __shared__ Neu sh[kTotThreads];
  for (int v = 0; v < nvar; ++v) {
    Neu acc{0.0, 0.0};
    for (int j = blockIdx.x; j < ny; j += gridDim.x) {
      const R *row = state + v * plane + (long long)j * pitch;
      for (int i = threadIdx.x; i < nx; i += blockDim.x) neu_add(acc, to_double(row[i]));
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kTotThreads / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) neu_merge(sh[threadIdx.x], sh[threadIdx.x + o]);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      partials[2 * (v * gridDim.x + blockIdx.x)] = sh[0].s;
      partials[2 * (v * gridDim.x + blockIdx.x) + 1] = sh[0].c;
    }
    __syncthreads();
  }
}

__global__ void totals_final_kernel(int nvar, const double *partials, int nblocks, double *out,
                                    double cell_area) {
  const int v = threadIdx.x;
  if (v >= nvar) return;
  Neu acc{0.0, 0.0};
  for (int b = 0; b < nblocks; ++b) {
    Neu p{partials[2 * (v * nblocks + b)], partials[2 * (v * nblocks + b) + 1]};
    neu_merge(acc, p);
  }
  out[v] = __dmul_rn(__dadd_rn(acc.s, acc.c), cell_area);
}

cudaError_t launch_totals(int prec, int nvar, const void *state, int nx, int ny, long long pitch,
                          long long plane, double *partials, int nblocks, double *out,
                          double cell_area, cudaStream_t s) {
  if (prec == 0)
    totals_partial_kernel<double><<<nblocks, kTotThreads, 0, s>>>(nvar, (const double *)state, nx, ny,
                                                                  pitch, plane, partials);
  else if (prec == 1)
    totals_partial_kernel<float><<<nblocks, kTotThreads, 0, s>>>(nvar, (const float *)state, nx, ny,
                                                                 pitch, plane, partials);
  else
    totals_partial_kernel<__nv_bfloat16><<<nblocks, kTotThreads, 0, s>>>(nvar, (const __nv_bfloat16 *)state, nx,
                                                                         ny, pitch, plane, partials);
  totals_final_kernel<<<1, 32, 0, s>>>(nvar, partials, nblocks, out, cell_area);
  return cudaGetLastError();
}

}  // namespace fv
