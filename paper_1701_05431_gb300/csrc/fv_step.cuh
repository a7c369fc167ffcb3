// fv_step.cuh -- the fused finite-volume step kernel (arXiv:1701.05431,
// Sec. 2.2.1 and Sec. 4.2): overlap fill, Lax-Friedrichs flux on every face
// (each face evaluated once), residual, forward-Euler update and the reduction
// of the largest wave speed for the next step's dt, in one launch.
//
// Work decomposition.  The grid is cut into warp tasks: a strip of 30*V
// output columns by TY rows.  Lane l of a warp holds V consecutive cells of a
// row (one coalesced V-wide vector load per variable); lanes 0 and 31 hold the
// strip's west and east neighbours (the "overlap" cells of Sec. 4.1.2) and
// write nothing.  The warp marches up its rows keeping the current row, its
// y-fluxes and the south face flux in registers, so every y-face is evaluated
// once and shared by the two cells around it; x-faces are evaluated once by
// the lane owning the cell east of the face, and passed to the lane on the
// west with a shuffle.  No shared memory and no barrier is used in the march.
// Ghost rows and columns at the physical boundary are produced by the row
// loader from the boundary condition, which replaces copyOverlaps and the
// ovlpE/N/W/S buffers.
//
// Ping-pong: step n reads buffer n % 2 and writes buffer (n + 1) % 2; n, dt
// and lmax come from the device control block, so one graph of identical
// launches advances any number of steps from any starting step.
#pragma once

#include "fv_device.cuh"

namespace fv {

template <class R> struct StepArgs {
  R *buf0;
  R *buf1;
  Ctrl *ctrl;
  int nx, ny;
  long long pitch;   // elements between rows
  long long plane;   // elements between variables
  int nstrips, nchunks, ntasks;
  double dx, dy;
  DtPolicy pol;
  SysParams<R> sp;
  int bc[4];
  R bc_state[4][8];
  int finalize;      // 1: this launch reduces lmax and closes the step
};

template <class R, int V> struct VecIO;
template <> struct VecIO<float, 1> {
  static __device__ __forceinline__ void ld(const float *p, float (&o)[1]) { o[0] = __ldg(p); }
  static __device__ __forceinline__ void st(float *p, const float (&o)[1]) { __stcs(p, o[0]); }
};
template <> struct VecIO<float, 2> {
  static __device__ __forceinline__ void ld(const float *p, float (&o)[2]) {
    float2 t = __ldg(reinterpret_cast<const float2 *>(p));
    o[0] = t.x; o[1] = t.y;
  }
  static __device__ __forceinline__ void st(float *p, const float (&o)[2]) {
    __stcs(reinterpret_cast<float2 *>(p), make_float2(o[0], o[1]));
  }
};
template <> struct VecIO<float, 4> {
  static __device__ __forceinline__ void ld(const float *p, float (&o)[4]) {
    float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  }
  static __device__ __forceinline__ void st(float *p, const float (&o)[4]) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(o[0], o[1], o[2], o[3]));
  }
};
template <> struct VecIO<double, 1> {
  static __device__ __forceinline__ void ld(const double *p, double (&o)[1]) { o[0] = __ldg(p); }
  static __device__ __forceinline__ void st(double *p, const double (&o)[1]) { __stcs(p, o[0]); }
};
template <> struct VecIO<double, 2> {
  static __device__ __forceinline__ void ld(const double *p, double (&o)[2]) {
    double2 t = __ldg(reinterpret_cast<const double2 *>(p));
    o[0] = t.x; o[1] = t.y;
  }
  static __device__ __forceinline__ void st(double *p, const double (&o)[2]) {
    __stcs(reinterpret_cast<double2 *>(p), make_double2(o[0], o[1]));
  }
};

// Load V cells of row j starting at column X into W[c][v], applying the
// boundary conditions for the ghost row/column just outside the domain.
// Columns further out (only reached by the idle halo lane of a ragged strip)
// are clamped to a real cell; their values are never used.
template <int NV, int V, class R>
static __device__ __forceinline__ void load_row(const StepArgs<R> &a, const R *__restrict__ src,
                                                int j, int X, R (&W)[V][NV]) {
  int side = -1, sj = j;
  if (j < 0) {
    side = kS;
    sj = a.bc[kS] == kPeriodic ? a.ny - 1 : 0;
  } else if (j >= a.ny) {
    side = kN;
    sj = a.bc[kN] == kPeriodic ? 0 : a.ny - 1;
  }
  if (side >= 0 && a.bc[side] == kDirichlet) {
#pragma unroll
    for (int c = 0; c < V; ++c)
#pragma unroll
      for (int v = 0; v < NV; ++v) W[c][v] = a.bc_state[side][v];
    return;
  }
  const R *row = src + (long long)sj * a.pitch;
  if (X >= 0 && X + V <= a.nx) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      R t[V];
      VecIO<R, V>::ld(row + v * a.plane + X, t);
#pragma unroll
      for (int c = 0; c < V; ++c) W[c][v] = t[c];
    }
  } else {
#pragma unroll
    for (int c = 0; c < V; ++c) {
      int col = X + c, sc = col, cs = -1;
      if (col < 0) {
        if (col == -1) { cs = kW; sc = a.bc[kW] == kPeriodic ? a.nx - 1 : 0; }
        else sc = 0;
      } else if (col >= a.nx) {
        if (col == a.nx) { cs = kE; sc = a.bc[kE] == kPeriodic ? 0 : a.nx - 1; }
        else sc = a.nx - 1;
      }
      if (cs >= 0 && a.bc[cs] == kDirichlet) {
#pragma unroll
        for (int v = 0; v < NV; ++v) W[c][v] = a.bc_state[cs][v];
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) W[c][v] = __ldg(row + v * a.plane + sc);
      }
    }
  }
}

// x-direction work on a freshly loaded row: physical fluxes of every cell,
// the west-face flux of each cell (the first cell's west neighbour is the
// previous lane's last cell), the east face from the next lane, and
// dX = F~_{i+1/2} - F~_{i-1/2}.  Also returns the y-fluxes and y-speeds.
template <class Sys, int V, class R>
static __device__ __forceinline__ void row_x(const SysParams<R> &P, const R (&W)[V][Sys::NV],
                                             R (&Fy)[V][Sys::NV], R (&sy)[V],
                                             R (&dX)[V][Sys::NV]) {
  constexpr int NV = Sys::NV;
  using O = Ops<R>;
  R Fx[V][NV], sx[V];
#pragma unroll
  for (int c = 0; c < V; ++c) Sys::fluxes(W[c], P, Fx[c], sx[c], Fy[c], sy[c]);
  R Fw[V][NV];
  {
    const R sL = __shfl_up_sync(0xffffffffu, sx[V - 1], 1);
    const R hs = O::mul((R)0.5, O::max(sL, sx[0]));
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R WL = __shfl_up_sync(0xffffffffu, W[V - 1][v], 1);
      const R FL = __shfl_up_sync(0xffffffffu, Fx[V - 1][v], 1);
      Fw[0][v] = lf_face(WL, FL, W[0][v], Fx[0][v], hs);
    }
  }
#pragma unroll
  for (int c = 1; c < V; ++c) {
    const R hs = O::mul((R)0.5, O::max(sx[c - 1], sx[c]));
#pragma unroll
    for (int v = 0; v < NV; ++v) Fw[c][v] = lf_face(W[c - 1][v], Fx[c - 1][v], W[c][v], Fx[c][v], hs);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
#pragma unroll
    for (int c = 0; c + 1 < V; ++c) dX[c][v] = O::sub(Fw[c + 1][v], Fw[c][v]);
    const R Fe = __shfl_down_sync(0xffffffffu, Fw[0][v], 1);
    dX[V - 1][v] = O::sub(Fe, Fw[V - 1][v]);
  }
}

template <class Sys, class R, int V, int TY, int NW>
__global__ void __launch_bounds__(NW * 32)
fv_step_kernel(const StepArgs<R> a) {
  constexpr int NV = Sys::NV;
  using O = Ops<R>;
  __shared__ double s_lam[NW];
  __shared__ int s_bad[NW];
  __shared__ double s_dt;
  __shared__ int s_run;
  __shared__ unsigned s_err;
  __shared__ long long s_step;

  if (threadIdx.x == 0) {
    Ctrl c;
    c.step = __ldcg(&a.ctrl->step);
    c.t = __ldcg(&a.ctrl->t);
    c.t_end = __ldcg(&a.ctrl->t_end);
    c.err_committed = __ldcg(&a.ctrl->err_committed);
    const double lam = lam_value(__ldcg(&a.ctrl->lam[c.step % 3]));
    double dt = 0.0;
    unsigned err = 0u;
    s_run = choose_dt(a.pol, c, lam, &dt, &err) ? 1 : 0;
    s_dt = dt;
    s_err = err;
    s_step = c.step;
  }
  __syncthreads();
  const int run = s_run;
  const long long n = s_step;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  R lam_loc = (R)0;
  bool bad = false;

  if (run) {
    const R *__restrict__ src = (n & 1) ? a.buf1 : a.buf0;
    R *__restrict__ dst = (n & 1) ? a.buf0 : a.buf1;
    const R lx = (R)(s_dt / a.dx);
    const R ly = (R)(s_dt / a.dy);
    const bool writer = lane >= 1 && lane <= 30;
    const int gw = blockIdx.x * NW + warp;
    const int GW = gridDim.x * NW;
    for (int task = gw; task < a.ntasks; task += GW) {
      const int sx_ = task % a.nstrips;
      const int cy = task / a.nstrips;
      const int X = sx_ * (30 * V) + (lane - 1) * V;
      const int y0 = cy * TY;
      const int y1 = min(y0 + TY, a.ny);

      R Wa[V][NV], Fya[V][NV], sya[V], dXa[V][NV], Fs[V][NV];
      R Wb[V][NV], Fyb[V][NV], syb[V], dXb[V][NV];
      R Wp[V][NV];
      // row below the strip: only its y-fluxes are needed
      load_row<NV, V>(a, src, y0 - 1, X, Wa);
      load_row<NV, V>(a, src, y0, X, Wb);
      if (y0 + 1 <= y1) load_row<NV, V>(a, src, y0 + 1, X, Wp);
#pragma unroll
      for (int c = 0; c < V; ++c) {
        R Fx_[NV], sx_unused;
        Sys::fluxes(Wa[c], a.sp, Fx_, sx_unused, Fya[c], sya[c]);
      }
      row_x<Sys, V>(a.sp, Wb, Fyb, syb, dXb);
#pragma unroll
      for (int c = 0; c < V; ++c) {
        const R hs = O::mul((R)0.5, O::max(sya[c], syb[c]));
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          Fs[c][v] = lf_face(Wa[c][v], Fya[c][v], Wb[c][v], Fyb[c][v], hs);
          Wa[c][v] = Wb[c][v];
          Fya[c][v] = Fyb[c][v];
          dXa[c][v] = dXb[c][v];
        }
        sya[c] = syb[c];
      }

      for (int j = y0; j < y1; ++j) {
#pragma unroll
        for (int c = 0; c < V; ++c)
#pragma unroll
          for (int v = 0; v < NV; ++v) Wb[c][v] = Wp[c][v];
        if (j + 2 <= y1) load_row<NV, V>(a, src, j + 2, X, Wp);
        row_x<Sys, V>(a.sp, Wb, Fyb, syb, dXb);
        R Wn[V][NV];
#pragma unroll
        for (int c = 0; c < V; ++c) {
          const R hs = O::mul((R)0.5, O::max(sya[c], syb[c]));
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const R Fn = lf_face(Wa[c][v], Fya[c][v], Wb[c][v], Fyb[c][v], hs);
            Wn[c][v] = fv_update(Wa[c][v], dXa[c][v], O::sub(Fn, Fs[c][v]), lx, ly);
            Fs[c][v] = Fn;
            Wa[c][v] = Wb[c][v];
            Fya[c][v] = Fyb[c][v];
            dXa[c][v] = dXb[c][v];
          }
          sya[c] = syb[c];
        }
        if (writer) {
          R *row = dst + (long long)j * a.pitch;
          if (X + V <= a.nx) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              R t[V];
#pragma unroll
              for (int c = 0; c < V; ++c) t[c] = Wn[c][v];
              VecIO<R, V>::st(row + v * a.plane + X, t);
            }
          } else {
#pragma unroll
            for (int c = 0; c < V; ++c)
              if (X + c < a.nx) {
#pragma unroll
                for (int v = 0; v < NV; ++v) __stcs(row + v * a.plane + X + c, Wn[c][v]);
              }
          }
          if (a.finalize) {
#pragma unroll
            for (int c = 0; c < V; ++c) {
              if (X + c < a.nx) {
                bool b;
                const R l = Sys::lambda(Wn[c], a.sp, b);
                lam_loc = O::max(lam_loc, l);
                bad |= b;
              }
            }
          }
        }
      }
    }
  }

  if (!a.finalize) return;
  // block reduction of lmax(W^{n+1}) and of the admissibility flag
  double l = (double)lam_loc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l = fmax(l, __shfl_xor_sync(0xffffffffu, l, o));
  const int anybad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    s_lam[warp] = l;
    s_bad[warp] = anybad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bl = 0.0;
    int bb = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      bl = fmax(bl, s_lam[w]);
      bb |= s_bad[w];
    }
    Ctrl *ctrl = a.ctrl;
    if (run) {
      if (bl > 0.0 || bb) atomicMax(&ctrl->lam[(n + 1) % 3], lam_bits(bb ? __longlong_as_double(0x7ff8000000000000LL) : bl));
      if (bb) atomicOr(&ctrl->err_pending, kErrNonphysical);
    }
    __threadfence();
    const unsigned prev = atomicAdd(&ctrl->blocks_done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      ctrl->blocks_done = 0u;
      unsigned e = atomicExch(&ctrl->err_pending, 0u) | s_err;
      if (run) {
        ctrl->t = ctrl->t + s_dt;
        ctrl->dt_last = s_dt;
        ctrl->step = n + 1;
        ctrl->lam[(n + 2) % 3] = 0ull;
      }
      if (e) ctrl->err_committed |= e;
      __threadfence();
    }
  }
}

}  // namespace fv
