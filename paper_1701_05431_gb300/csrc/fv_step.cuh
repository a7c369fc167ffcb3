// fv_step.cuh -- the fused finite-volume step kernel (arXiv:1701.05431,
// Sec. 2.2.1 and Sec. 4.2): overlap fill, Lax-Friedrichs flux on every face
// (each face evaluated once), residual, forward-Euler update and the reduction
// of the largest wave speed for the next step's dt, in one launch.
//
// Work decomposition.  The grid is cut into warp tasks: a strip of 30*V*K
// output columns by TY rows.  Lane l of a warp holds V*K consecutive cells of
// a row (V values of the arithmetic type A, each packing K cells; one
// coalesced vector load per variable); lanes 0 and 31 hold the strip's west
// and east neighbours (the "overlap" cells of Sec. 4.1.2) and write nothing.
// The warp marches up its rows keeping the current row, its y-fluxes and the
// south face flux in registers, so every y-face is evaluated once and shared
// by the two cells around it; x-faces are evaluated once by the lane owning
// the cell east of the face, and passed to the lane on the west with a
// shuffle.  No barrier is used in the march.  Ghost rows and columns at the
// physical boundary are produced by the row loader from the boundary
// condition, which replaces copyOverlaps and the ovlpE/N/W/S buffers.
//
// Rows reach the registers in one of three ways (template parameter D):
//   D = 0   register prefetch of the next row;
//   D > 0   a D-deep ring of row segments in shared memory filled by TMA bulk
//           copies (cp.async.bulk + mbarrier), one lane per warp issuing;
//   D < 0   a -D-deep ring filled by each lane with cp.async for its own
//           cells (no cross-lane synchronisation).
// Strips touching the east or west boundary always use register prefetch.
//
// Ping-pong: step n reads buffer n % 2 and writes buffer (n + 1) % 2; n, dt
// and lmax come from the device control block, so one graph of identical
// launches advances any number of steps from any starting step.
#pragma once

#include <type_traits>

#include "fv_device.cuh"

namespace fv {

// Launch arguments, in the storage type S of the state.
template <class S> struct StepArgs {
  S *buf0;
  S *buf1;
  Ctrl *ctrl;
  int nx, ny;
  long long pitch;   // elements between rows
  long long plane;   // elements between variables
  int nstrips, nchunks, ntasks;
  int ty;            // rows per warp task (the kernel's TY in place and two-step)
  double dx, dy;
  DtPolicy pol;
  SysParams<typename ParamOf<S>::T> sp;
  int bc[4];
  typename ParamOf<S>::T bc_state[4][8];
  // in-place mode: the overlap strips of the two step parities (null in the
  // default ping-pong mode, where buf0 != buf1)
  S *ovl[2];
  int ovl_task;      // elements of one task's strips in one parity
  const S *ovl_bc;   // the four sides' prescribed states as stored cells, [side][variable][cells per lane]
};

// What the march reads of the launch arguments.  The single-instance kernel
// passes its StepArgs (constants of the launch); the batched kernel builds
// this in registers from the instance's arguments in shared memory, keeping
// the boundary states there (read through the pointer on ghost cells only),
// because the march's stores into shared memory would otherwise force every
// field to be reloaded.
template <class S> struct MarchGeo {
  Ctrl *ctrl;
  int nx, ny;
  long long pitch, plane;
  int bc[4];
  const typename ParamOf<S>::T (*bc_state)[8];
};

// ld: read-only path (state never written during the launch); ldcg: L2-coherent
// loads for the persistent batched kernel, whose launch also writes the state.
template <class S, int N> struct VecIO;
template <> struct VecIO<float, 1> {
  static __device__ __forceinline__ void ld(const float *p, float (&o)[1]) { o[0] = __ldg(p); }
  static __device__ __forceinline__ void ldcg(const float *p, float (&o)[1]) { o[0] = __ldcg(p); }
  static __device__ __forceinline__ void st(float *p, const float (&o)[1]) { __stcs(p, o[0]); }
};
template <> struct VecIO<float, 2> {
  static __device__ __forceinline__ void ld(const float *p, float (&o)[2]) {
    float2 t = __ldg(reinterpret_cast<const float2 *>(p));
    o[0] = t.x; o[1] = t.y;
  }
  static __device__ __forceinline__ void ldcg(const float *p, float (&o)[2]) {
    float2 t = __ldcg(reinterpret_cast<const float2 *>(p));
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
  static __device__ __forceinline__ void ldcg(const float *p, float (&o)[4]) {
    float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  }
  static __device__ __forceinline__ void st(float *p, const float (&o)[4]) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(o[0], o[1], o[2], o[3]));
  }
};
template <> struct VecIO<double, 1> {
  static __device__ __forceinline__ void ld(const double *p, double (&o)[1]) { o[0] = __ldg(p); }
  static __device__ __forceinline__ void ldcg(const double *p, double (&o)[1]) { o[0] = __ldcg(p); }
  static __device__ __forceinline__ void st(double *p, const double (&o)[1]) { __stcs(p, o[0]); }
};
template <> struct VecIO<double, 2> {
  static __device__ __forceinline__ void ld(const double *p, double (&o)[2]) {
    double2 t = __ldg(reinterpret_cast<const double2 *>(p));
    o[0] = t.x; o[1] = t.y;
  }
  static __device__ __forceinline__ void ldcg(const double *p, double (&o)[2]) {
    double2 t = __ldcg(reinterpret_cast<const double2 *>(p));
    o[0] = t.x; o[1] = t.y;
  }
  static __device__ __forceinline__ void st(double *p, const double (&o)[2]) {
    __stcs(reinterpret_cast<double2 *>(p), make_double2(o[0], o[1]));
  }
};

template <> struct VecIO<__nv_bfloat16, 2> {
  static __device__ __forceinline__ void ld(const __nv_bfloat16 *p, __nv_bfloat16 (&o)[2]) {
    const __nv_bfloat162 t = __ldg(reinterpret_cast<const __nv_bfloat162 *>(p));
    o[0] = t.x; o[1] = t.y;
  }
  static __device__ __forceinline__ void ldcg(const __nv_bfloat16 *p, __nv_bfloat16 (&o)[2]) {
    const __nv_bfloat162 t = __ldcg(reinterpret_cast<const __nv_bfloat162 *>(p));
    o[0] = t.x; o[1] = t.y;
  }
  static __device__ __forceinline__ void st(__nv_bfloat16 *p, const __nv_bfloat16 (&o)[2]) {
    __nv_bfloat162 t;
    t.x = o[0]; t.y = o[1];
    __stcs(reinterpret_cast<__nv_bfloat162 *>(p), t);
  }
};
template <> struct VecIO<__nv_bfloat16, 4> {
  static __device__ __forceinline__ void ld(const __nv_bfloat16 *p, __nv_bfloat16 (&o)[4]) {
    const uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&t.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&t.y);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
  static __device__ __forceinline__ void ldcg(const __nv_bfloat16 *p, __nv_bfloat16 (&o)[4]) {
    const uint2 t = __ldcg(reinterpret_cast<const uint2 *>(p));
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&t.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&t.y);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
  static __device__ __forceinline__ void st(__nv_bfloat16 *p, const __nv_bfloat16 (&o)[4]) {
    __nv_bfloat162 a, b;
    a.x = o[0]; a.y = o[1]; b.x = o[2]; b.y = o[3];
    uint2 t;
    t.x = *reinterpret_cast<const unsigned *>(&a);
    t.y = *reinterpret_cast<const unsigned *>(&b);
    __stcs(reinterpret_cast<uint2 *>(p), t);
  }
};

// Where a lane's N storage cells come from.  Interior strips (every lane's
// cells inside [0, nx)) read N-wide vectors at column X; strips touching the
// east or west boundary map each cell once per task: a real column, the ghost
// column of the boundary condition, or (only for the idle halo lane of a
// ragged strip) a clamped column whose values are never used.
template <int N> struct LaneCols {
  int col[N];
  int dir[N];  // Dirichlet side of a ghost cell, -1 otherwise
};

template <int N, class G>
static __device__ __forceinline__ LaneCols<N> lane_cols(const G &a, int X) {
  LaneCols<N> L;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    const int col = X + c;
    int sc = col, dir = -1;
    if (col < 0) {
      if (col == -1 && a.bc[kW] == kDirichlet) dir = kW;
      sc = (col == -1 && a.bc[kW] == kPeriodic) ? a.nx - 1 : 0;
    } else if (col >= a.nx) {
      if (col == a.nx && a.bc[kE] == kDirichlet) dir = kE;
      sc = (col == a.nx && a.bc[kE] == kPeriodic) ? 0 : a.nx - 1;
    }
    L.col[c] = sc;
    L.dir[c] = dir;
  }
  return L;
}

// Source row of row j (ghost rows -1 and ny from the boundary condition);
// returns the Dirichlet side when the ghost row is a prescribed state.
template <class G>
static __device__ __forceinline__ int row_src(const G &a, int j, int &dir) {
  dir = -1;
  if (j < 0) {
    if (a.bc[kS] == kDirichlet) dir = kS;
    return a.bc[kS] == kPeriodic ? a.ny - 1 : 0;
  }
  if (j >= a.ny) {
    if (a.bc[kN] == kDirichlet) dir = kN;
    return a.bc[kN] == kPeriodic ? 0 : a.ny - 1;
  }
  return j;
}

// Load the lane's V values (V*K cells) of row j of every variable into W.
template <int NV, int V, bool XIN, bool CG, class A, class G>
static __device__ __forceinline__ void load_row(const G &a,
                                                const typename Ops<A>::S *__restrict__ base,
                                                const LaneCols<V * Ops<A>::K> &L, int j, A (&W)[V][NV]) {
  using S = typename Ops<A>::S;
  constexpr int K = Ops<A>::K, N = V * K;
  int dir;
  const int sj = row_src(a, j, dir);
  if (dir >= 0) {
    // the prescribed state in the storage type, as every other loader and
    // the ghost columns below give it (bfloat16 storage rounds it)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      S t[K];
#pragma unroll
      for (int k = 0; k < K; ++k) t[k] = (S)a.bc_state[dir][v];
#pragma unroll
      for (int c = 0; c < V; ++c) W[c][v] = Ops<A>::pack(t);
    }
    return;
  }
  const S *row = base + (long long)sj * a.pitch;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    S t[N];
    if (XIN) {
      if (CG) VecIO<S, N>::ldcg(row + v * a.plane, t);
      else VecIO<S, N>::ld(row + v * a.plane, t);
    } else {
#pragma unroll
      for (int c = 0; c < N; ++c) {
        if (L.dir[c] >= 0) t[c] = (S)a.bc_state[L.dir[c]][v];
        else t[c] = CG ? __ldcg(row + v * a.plane + L.col[c]) : __ldg(row + v * a.plane + L.col[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < V; ++c) W[c][v] = Ops<A>::pack(t + c * K);
  }
}

// x-direction work on a freshly loaded row: physical fluxes of every cell,
// the west-face flux of each cell (the first cell's west neighbour is the
// previous lane's last cell), the east face from the next lane, and
// dX = F~_{i+1/2} - F~_{i-1/2}.  Also returns the y-fluxes and y-speeds.
// USEQ: the cells' primitives are given in Q (Euler), not recovered here.
template <class Sys, int V, bool USEQ = false, class A>
static __device__ __forceinline__ void row_x(const SysParams<A> &P, const A (&W)[V][Sys::NV],
                                             A (&Fy)[V][Sys::NV], A (&sy)[V], A (&dX)[V][Sys::NV],
                                             const A (*Q)[4] = nullptr) {
  constexpr int NV = Sys::NV;
  using O = Ops<A>;
  A Fx[V][NV], sx[V];
#pragma unroll
  for (int c = 0; c < V; ++c) {
    if constexpr (USEQ) Sys::fluxes_from(W[c], Q[c], Fx[c], sx[c], Fy[c], sy[c]);
    else Sys::fluxes(W[c], P, Fx[c], sx[c], Fy[c], sy[c]);
  }
  A Fw[V][NV];
#pragma unroll
  for (int c = 0; c < V; ++c) {
    // values of the cells just west of this value's cells
    const A sprev = c == 0 ? O::shfl_up(sx[V - 1], 1) : sx[c - 1];
    const A sL = O::shift_in(sprev, sx[c]);
    const A sg = O::max(sL, sx[c]);
#pragma unroll
    for (int v = 0; v < Sys::NU; ++v) {
      const A wprev = c == 0 ? O::shfl_up(W[V - 1][v], 1) : W[c - 1][v];
      const A fprev = c == 0 ? O::shfl_up(Fx[V - 1][v], 1) : Fx[c - 1][v];
      Fw[c][v] = lf_face2(O::shift_in(wprev, W[c][v]), O::shift_in(fprev, Fx[c][v]), W[c][v], Fx[c][v], sg);
    }
  }
#pragma unroll
  for (int v = 0; v < Sys::NU; ++v) {
    const A first_next = O::shfl_down(Fw[0][v], 1);
#pragma unroll
    for (int c = 0; c < V; ++c) {
      const A next = c + 1 < V ? Fw[c + 1][v] : first_next;
      dX[c][v] = O::sub(O::shift_out(Fw[c][v], next), Fw[c][v]);
    }
  }
}

// ---------------------------------------------------------------- in place
// In-place mode keeps ONE state buffer.  A task updates its own cells in
// place; the cells of its halo that belong to other tasks are read from the
// overlap strips those tasks wrote one step earlier (the paper's ovlpE/N/W/S
// buffers, Sec. 4.1.2, filled by the producing task instead of a copy task):
// per task and step parity, for every variable, its first and last N
// columns (the west and east column strips, TY rows of N cells: exactly the
// cells the halo lane of the neighbouring task holds, so that lane reads one
// vector per row like every other lane) and its first and last rows (the
// south and north row strips, 30 N cells).  Step n reads the strips of
// parity n % 2 and writes those of parity (n + 1) % 2, so no task reads a
// value another task is overwriting.  A task's own rows are read (through
// the ring, several rows ahead) before it overwrites them.
template <class S> struct Ovl {
  const S *op;     // own rows: source of row y0 (the state, a neighbour's column strip, or prescribed cells)
  int task;        // the warp task: strip task % nstrips, chunk task / nstrips
  int y0, y1;      // first and end row of the task
  unsigned flags;  // kPercell | fixW (bits 1-2) | fixE (bits 3-4) | kLastFull | own-row source kind | kOdd
  // kept only with fewer than four cells per lane (see ovl_opaque)
  int sx, cy;      // the task's strip and chunk
  int ors;         // row stride of op
  long long ovs;   // variable stride of op
  const S *rd;     // strips of parity n % 2
  S *wb;           // this task's strips of parity (n + 1) % 2
};
// kOwnStrip: own rows from a column strip (row stride N, variable stride ty N);
// kOwnDir: from the prescribed cells (row stride 0, variable stride N);
// neither: from the state (pitch, plane).  kOdd: the step is odd, so the
// strips of W^n are those of parity 1.
enum : unsigned { kPercell = 1u, kFixWShift = 1, kFixEShift = 3, kLastFull = 32u, kOwnStrip = 64u, kOwnDir = 128u,
                  kOdd = 256u };

// Element offsets inside one task's strips (NV variables each).
template <int NV, int N, int SW> struct OvlLayout {
  static __device__ __forceinline__ int colW(int ty) { return 0; }
  static __device__ __forceinline__ int colE(int ty) { return NV * ty * N; }
  static __device__ __forceinline__ int rowS(int ty) { return 2 * NV * ty * N; }
  static __device__ __forceinline__ int rowN(int ty) { return 2 * NV * ty * N + NV * SW; }
};

// The strips of W^n (read) and of W^{n+1} (written) this step.  With four
// or more cells per lane the march has no registers to spare, so the task
// index passes through an opaque copy where a value is derived per row: the
// compiler then recomputes the few integer operations instead of keeping
// loop-invariant pointers in registers.  With fewer cells it keeps them.
template <int N> static __device__ __forceinline__ int ovl_opaque(int x) {
  if constexpr (N < 4) return x;
  int y;
  asm volatile("mov.b32 %0, %1;" : "=r"(y) : "r"(x));
  return y;
}
template <int N, class G, class S> static __device__ __forceinline__ const S *ovl_rd(const G &a, const Ovl<S> &o) {
  if constexpr (N < 4) return o.rd;
  return (o.flags & kOdd) ? a.ovl[1] : a.ovl[0];
}
template <int N, class G, class S> static __device__ __forceinline__ S *ovl_wb(const G &a, const Ovl<S> &o) {
  if constexpr (N < 4) return o.wb;
  return ((o.flags & kOdd) ? a.ovl[0] : a.ovl[1]) + (long long)ovl_opaque<N>(o.task) * a.ovl_task;
}

// Per-lane in-place bookkeeping of one task: where the lane's N cells of the
// task's own rows come from, whether a ghost column has to be set after a
// read, and whether the strip reaches past the grid.  Lanes 1..30 read
// their own cells from the state; the halo lanes read the neighbouring
// task's column strip (periodic sides: the task across the boundary), on a
// Dirichlet side the prescribed state's cells, and on a transmissive side
// some of their own task's cells, the ghost being set in registers
// (ovl_fix_cols).  Lanes of a ragged last strip that reach past the grid go
// cell by cell.
template <int NV, int N, int TY, class G, class S>
static __device__ __forceinline__ void ovl_lane_setup(const G &a, const S *W, Ovl<S> &o, int X, int lane, int sx,
                                                      int cy, long long n) {
  constexpr int SW = 30 * N;
  using L = OvlLayout<NV, N, SW>;
  const int X0 = sx * SW;
  const bool full = X0 + SW <= a.nx;  // every column of the strip lies in the grid
  unsigned f = (lane >= 1 && X + N > a.nx) ? kPercell : 0u;
  if (n & 1) f |= kOdd;
  const S *rd = (n & 1) ? a.ovl[1] : a.ovl[0];
  o.op = W + (long long)o.y0 * a.pitch + X;
  if (lane == 0) {
    if (sx > 0 || a.bc[kW] == kPeriodic) {
      o.op = rd + (long long)(cy * a.nstrips + (sx > 0 ? sx - 1 : a.nstrips - 1)) * a.ovl_task + L::colE(TY);
      f |= kOwnStrip;
    } else if (a.bc[kW] == kDirichlet) {
      o.op = a.ovl_bc + kW * NV * N;  // the same N cells every row
      f |= kOwnDir;
    } else {
      o.op = W + (long long)o.y0 * a.pitch + X0;
    }
  } else if (lane == 31 && !(f & kPercell)) {
    if (sx < a.nstrips - 1 || a.bc[kE] == kPeriodic) {
      o.op = rd + (long long)(cy * a.nstrips + (sx < a.nstrips - 1 ? sx + 1 : 0)) * a.ovl_task + L::colW(TY);
      f |= kOwnStrip;
    } else if (a.bc[kE] == kDirichlet) {
      o.op = a.ovl_bc + kE * NV * N;
      f |= kOwnDir;
    } else {
      o.op = W + (long long)o.y0 * a.pitch + (X - N);
    }
  }
  // transmissive west or east side: the halo lane's ghost cell is a copy of the border column
  if (sx == 0 && a.bc[kW] == kTransmissive) f |= 1u << kFixWShift;
  if (full && sx == a.nstrips - 1 && a.bc[kE] == kTransmissive) f |= 1u << kFixEShift;
  if (full) f |= kLastFull;
  o.flags = f;
  if constexpr (N < 4) {
    o.sx = sx;
    o.cy = cy;
    o.ors = (f & kOwnStrip) ? N : (f & kOwnDir) ? 0 : (int)a.pitch;
    o.ovs = (f & kOwnStrip) ? (long long)TY * N : (f & kOwnDir) ? (long long)N : a.plane;
    o.rd = rd;
    o.wb = ((n & 1) ? a.ovl[0] : a.ovl[1]) + (long long)o.task * a.ovl_task;
  }
}

// Source of a lane's N cells of halo row j (j = y0 - 1 or y1), always a
// vector inside the strips: the row strip of the task below or above
// (across a periodic side: the task at the other end), for a transmissive
// ghost row the task's own border row strip (its border row of W^n), or the
// prescribed state's cells.  The halo lanes' cells there are tile corners no
// face uses: they read the strip at lane 1's or lane 30's position, and so
// do the lanes of a ragged last strip past the grid.
template <int NV, int N, int TY, class G, class S>
static __device__ __forceinline__ const S *ovl_halo_src(const G &a, const Ovl<S> &o, int X, int j, long long &vs) {
  constexpr int SW = 30 * N;
  using L = OvlLayout<NV, N, SW>;
  const int task = ovl_opaque<N>(o.task);
  const int sx = N < 4 ? o.sx : task % a.nstrips, cy = N < 4 ? o.cy : task / a.nstrips;
  const int xo = min(max(X - sx * SW, 0), SW - N);
  const S *rd = ovl_rd<N>(a, o);
  vs = SW;
  if (j < o.y0) {
    if (cy > 0 || a.bc[kS] == kPeriodic)
      return rd + (long long)((cy > 0 ? cy - 1 : a.nchunks - 1) * a.nstrips + sx) * a.ovl_task + L::rowN(TY) + xo;
    if (a.bc[kS] == kDirichlet) {
      vs = N;
      return a.ovl_bc + kS * NV * N;
    }
    // transmissive: the task's own first row, as its south row strip holds it
    return rd + (long long)task * a.ovl_task + L::rowS(TY) + xo;
  }
  if (cy < a.nchunks - 1 || a.bc[kN] == kPeriodic)
    return rd + (long long)((cy < a.nchunks - 1 ? cy + 1 : 0) * a.nstrips + sx) * a.ovl_task + L::rowS(TY) + xo;
  if (a.bc[kN] == kDirichlet) {
    vs = N;
    return a.ovl_bc + kN * NV * N;
  }
  // transmissive: the task's own last row, as its north row strip holds it
  return rd + (long long)task * a.ovl_task + L::rowN(TY) + xo;
}

// Ghost columns of a row just read, on a transmissive west or east side
// (warp-uniform): lane 0's last cell becomes lane 1's first, lane 31's first
// cell lane 30's last -- copies of the border columns, what the two-buffer
// loader reads there.  (The ghost of a ragged last strip comes cell by cell.)
template <class A, int V, int NV, class G, class S>
static __device__ __forceinline__ void ovl_fix_cols(const G &a, const Ovl<S> &o, A (&W)[V][NV], int lane) {
  using O = Ops<A>;
  static_assert(O::K == 1, "in-place kernels hold one cell per value");
  if (o.flags & ((3u << kFixWShift) | (3u << kFixEShift))) {
    const bool fw = lane == 0 && (o.flags & (3u << kFixWShift));
    const bool fe = lane == 31 && (o.flags & (3u << kFixEShift));
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const A w0 = O::shfl_down(W[0][v], 1);
      const A wl = O::shfl_up(W[V - 1][v], 1);
      if (fw) W[V - 1][v] = w0;
      if (fe) W[0][v] = wl;
    }
  }
}

// In-place mode: the writer lanes' share of the task's new border strips
// (row y0 -> south row strip, row y1 - 1 -> north row strip; lanes 1 and 30
// -> the west and east column strips, N cells a row; on a ragged last strip
// the lane holding the task's last column puts it in cell N - 1 of the east
// column strip), values of W^{n+1} in storage type, t[v][c] for the lane's
// N cells.
template <int NV, int N, int TY, class G, class S>
static __device__ __forceinline__ void write_strips(const G &a, const Ovl<S> &o, int X, int j, const S (&t)[NV][N]) {
  constexpr int SW = 30 * N;
  using L = OvlLayout<NV, N, SW>;
  const int lane = threadIdx.x & 31;
  const int xo = (lane - 1) * N;  // X minus the strip's first column
  if (j == o.y0 || j == o.y1 - 1) {
    S *wb = ovl_wb<N>(a, o);
    // a one-row task writes its row to both row strips
    const int first = j == o.y0 ? L::rowS(TY) : L::rowN(TY);
#pragma unroll
    for (int v = 0; v < NV; ++v) VecIO<S, N>::st(wb + first + v * SW + xo, t[v]);
    if (o.y1 - o.y0 == 1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) VecIO<S, N>::st(wb + L::rowN(TY) + v * SW + xo, t[v]);
    }
  }
  const int jr = j - o.y0;
  const bool full = (o.flags & kLastFull) != 0u;
  if (lane == 1 || (full && lane == 30)) {
    S *cs = ovl_wb<N>(a, o) + (lane == 1 ? L::colW(TY) : L::colE(TY)) + jr * N;
#pragma unroll
    for (int v = 0; v < NV; ++v) VecIO<S, N>::st(cs + (long long)v * TY * N, t[v]);
  }
  if (!full) {
    const int ecell = min(X - xo + SW, a.nx) - 1 - X;  // the task's last column, if this lane holds it
    S *wb = ovl_wb<N>(a, o);
#pragma unroll
    for (int c = 0; c < N; ++c)
      if (c == ecell) {
#pragma unroll
        for (int v = 0; v < NV; ++v) wb[L::colE(TY) + v * TY * N + jr * N + (N - 1)] = t[v][c];
      }
  }
}

// Registers of one row of the march.
template <class A, int V, int NV> struct RowState {
  A W[V][NV];
  A Fy[V][NV];
  A sy[V];
  A dX[V][NV];
};

// The y-faces between rows j (cur) and j+1 (nxt), evaluated once, and the
// updated values of row j: Fs holds the south faces of row j on entry and
// those of row j+1 on return.  FP64 Euler and spray on square cells take
// fv_update_sq (lx == ly: every kernel computes lx and ly the same way, so
// every kernel takes the same form on the same grid); the scalar advection
// kernels, bound by latency rather than by the FP64 pipe, keep the general
// form.
template <class Sys, class A, int V>
static __device__ __forceinline__ void faces_update_row(const RowState<A, V, Sys::NV> &cur,
                                                        const RowState<A, V, Sys::NV> &nxt, A (&Fs)[V][Sys::NV],
                                                        A lx, A ly, A (&Wn)[V][Sys::NV]) {
  using O = Ops<A>;
  auto run = [&](auto sq) {
#pragma unroll
    for (int c = 0; c < V; ++c) {
      const A sg = O::max(cur.sy[c], nxt.sy[c]);
#pragma unroll
      for (int v = 0; v < Sys::NU; ++v) {
        const A Fn = lf_face2(cur.W[c][v], cur.Fy[c][v], nxt.W[c][v], nxt.Fy[c][v], sg);
        const A dY = O::sub(Fn, Fs[c][v]);
        if constexpr (decltype(sq)::value) Wn[c][v] = fv_update_sq(cur.W[c][v], cur.dX[c][v], dY, lx);
        else Wn[c][v] = fv_update(cur.W[c][v], cur.dX[c][v], dY, lx, ly);
        Fs[c][v] = Fn;
      }
    }
  };
  if constexpr (std::is_same<A, double>::value && Sys::NV > 1) {
    if (lx == ly) run(std::true_type{});
    else run(std::false_type{});
  } else {
    run(std::false_type{});
  }
}

// Compute part of one row of the march (rows j and j+1 in registers): x-work
// of row j+1, the y-face between rows j and j+1 evaluated once, update and
// store of row j (by the writer lanes), and the new state's wave speed.
template <class Sys, class A, int V, bool XIN, bool FIN, bool INPL = false, int TYC = 0, class G>
static __device__ __forceinline__ void advance_row(const G &a, const SysParams<A> &P,
                                                   typename Ops<A>::S *dst_lane, int X, int j,
                                                   bool writer, A lx, A ly, RowState<A, V, Sys::NV> &cur,
                                                   RowState<A, V, Sys::NV> &nxt, A (&Fs)[V][Sys::NV],
                                                   typename Ops<A>::P &lam_loc, unsigned &bad,
                                                   bool xin = false,
                                                   const Ovl<typename Ops<A>::S> *ovl = nullptr) {
  using S = typename Ops<A>::S;
  constexpr int NV = Sys::NV, K = Ops<A>::K, N = V * K;
  using O = Ops<A>;
  row_x<Sys, V>(P, nxt.W, nxt.Fy, nxt.sy, nxt.dX);
  A Wn[V][NV];
  faces_update_row<Sys, A, V>(cur, nxt, Fs, lx, ly, Wn);
  // carried planes (primitives of the new state) follow from the updated ones
  if constexpr (Sys::NU != Sys::NV) {
#pragma unroll
    for (int c = 0; c < V; ++c) Sys::complete(Wn[c], P);
  }
  // interior strip: XIN at compile time, or xin at run time
  const bool in = XIN || xin;
  if (writer) {
    S *row = dst_lane + (long long)j * a.pitch;
    S t[NV][N];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int c = 0; c < V; ++c) O::unpack(Wn[c][v], t[v] + c * K);
    if (in || X + N <= a.nx) {
#pragma unroll
      for (int v = 0; v < NV; ++v) VecIO<S, N>::st(row + v * a.plane, t[v]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int c = 0; c < N; ++c)
          if (X + c < a.nx) __stcs(row + v * a.plane + c, t[v][c]);
    }
    if constexpr (INPL) write_strips<NV, N, TYC>(a, *ovl, X, j, t);
    if (FIN) {
#pragma unroll
      for (int c = 0; c < V; ++c) {
        // packed cells inside the grid (all of them on interior strips)
        unsigned valid = (1u << K) - 1u;
        if (!in) {
          valid = 0u;
#pragma unroll
          for (int k = 0; k < K; ++k)
            if (X + c * K + k < a.nx) valid |= 1u << k;
        }
        unsigned b;
        const A l = Sys::lambda(Wn[c], P, b);
        lam_loc = fmax(lam_loc, O::hmax(l, valid));
        bad |= b & valid;
      }
    }
  }
}

// One row of the march with register prefetch: `nxt` receives row j+1
// (already prefetched in Pf) and Pf is refilled with row j+2.
template <class Sys, class A, int V, bool XIN, bool FIN, bool CG, class G>
static __device__ __forceinline__ void march_row(const G &a, const SysParams<A> &P,
                                                 const typename Ops<A>::S *__restrict__ src,
                                                 typename Ops<A>::S *__restrict__ dst_lane,
                                                 const LaneCols<V * Ops<A>::K> &L, int X, int j, int y1,
                                                 bool writer, A lx, A ly, RowState<A, V, Sys::NV> &cur,
                                                 RowState<A, V, Sys::NV> &nxt, A (&Pf)[V][Sys::NV],
                                                 A (&Fs)[V][Sys::NV], typename Ops<A>::P &lam_loc,
                                                 unsigned &bad) {
  constexpr int NV = Sys::NV;
#pragma unroll
  for (int c = 0; c < V; ++c)
#pragma unroll
    for (int v = 0; v < NV; ++v) nxt.W[c][v] = Pf[c][v];
  if (j + 2 <= y1) load_row<NV, V, XIN, CG>(a, src, L, j + 2, Pf);
  advance_row<Sys, A, V, XIN, FIN>(a, P, dst_lane, X, j, writer, lx, ly, cur, nxt, Fs, lam_loc, bad);
}

// March one warp task with register prefetch: rows [y0, y1) of the strip
// whose lane l holds the V*K cells starting at column X.
template <class Sys, class A, int V, bool XIN, bool FIN, bool CG = false, class G>
static __device__ __forceinline__ void march(const G &a, const SysParams<A> &P,
                                             const typename Ops<A>::S *__restrict__ src,
                                             typename Ops<A>::S *__restrict__ dst, int X, int y0, int y1,
                                             bool writer, A lx, A ly, typename Ops<A>::P &lam_loc,
                                             unsigned &bad) {
  using S = typename Ops<A>::S;
  constexpr int NV = Sys::NV, N = V * Ops<A>::K;
  using O = Ops<A>;
  LaneCols<N> L;
  if (!XIN) L = lane_cols<N>(a, X);
  const S *base = XIN ? src + X : src;
  S *dst_lane = dst + X;
  RowState<A, V, NV> RA, RB;
  A Pf[V][NV], Fs[V][NV];
  // row below the strip: only its y-fluxes are needed
  load_row<NV, V, XIN, CG>(a, base, L, y0 - 1, RA.W);
  load_row<NV, V, XIN, CG>(a, base, L, y0, RB.W);
  if (y0 + 1 <= y1) load_row<NV, V, XIN, CG>(a, base, L, y0 + 1, Pf);
#pragma unroll
  for (int c = 0; c < V; ++c) {
    A Fx_[NV], sx_;
    Sys::fluxes(RA.W[c], P, Fx_, sx_, RA.Fy[c], RA.sy[c]);
  }
  row_x<Sys, V>(P, RB.W, RB.Fy, RB.sy, RB.dX);
#pragma unroll
  for (int c = 0; c < V; ++c) {
    const A sg = O::max(RA.sy[c], RB.sy[c]);
#pragma unroll
    for (int v = 0; v < Sys::NU; ++v) Fs[c][v] = lf_face2(RA.W[c][v], RA.Fy[c][v], RB.W[c][v], RB.Fy[c][v], sg);
  }
  // the two row states swap roles every row (unrolled by two: no copies)
  int j = y0;
  while (true) {
    if (j >= y1) break;
    march_row<Sys, A, V, XIN, FIN, CG>(a, P, base, dst_lane, L, X, j, y1, writer, lx, ly, RB, RA, Pf, Fs, lam_loc, bad);
    ++j;
    if (j >= y1) break;
    march_row<Sys, A, V, XIN, FIN, CG>(a, P, base, dst_lane, L, X, j, y1, writer, lx, ly, RA, RB, Pf, Fs, lam_loc, bad);
    ++j;
  }
}

// ---------------------------------------------------------------- TMA rows
// Interior strips can stage their rows through shared memory with bulk
// asynchronous copies (TMA, cp.async.bulk) instead of register prefetch: each
// warp owns a ring of D row slots, one mbarrier per slot; lane 0 issues, for
// every variable, one bulk copy of the strip's row segment (widened to 16-byte
// boundaries), so D rows per warp are in flight without spending registers.
// A lane reads its cells of a slot after the slot's barrier completes.
// Every wait is bounded (%globaltimer); a wait that runs out marks the step
// with a timeout error and the warp stops waiting (the step is then reported
// as failed, never silently used).

static __device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
static __device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
static __device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
static __device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
static __device__ __forceinline__ void bulk_load(void *sdst, const void *gsrc, unsigned bytes,
                                                 unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(sdst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
static __device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
static __device__ __forceinline__ unsigned long long timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <class S> struct TmaGeom {
  static constexpr int kAlign = 16 / (int)sizeof(S);  // elements per 16 bytes
  static constexpr __host__ __device__ int seg(int N) { return 32 * N + 2 * kAlign; }  // slot elements per variable
};

template <class A, int V, int NV, int D> struct RowRing {
  using S = typename Ops<A>::S;
  static constexpr int N = V * Ops<A>::K;
  static constexpr int SEG = TmaGeom<S>::seg(N);
  S *buf;                     // D slots x NV variables x SEG elements
  unsigned long long *bar;    // D barriers
  unsigned phase;             // bit k: parity the next wait on slot k expects
  int seg0;                   // first column of the staged segment (16-byte aligned)
  int lane_off;               // X - seg0
  unsigned bytes;             // bytes per variable per row
  bool broken;
};

// Lane 0 stages row j (relative row r of the task) into slot r % D.
template <class A, int V, int NV, int D, class G>
static __device__ __forceinline__ void ring_issue(const G &a,
                                                  const typename Ops<A>::S *__restrict__ src,
                                                  RowRing<A, V, NV, D> &rg, int r, int j) {
  using S = typename Ops<A>::S;
  using RG = RowRing<A, V, NV, D>;
  int dir;
  const int sj = row_src(a, j, dir);
  if (dir >= 0 || rg.broken) return;  // a prescribed ghost row is not staged
  if ((threadIdx.x & 31) == 0) {
    const int slot = r % D;
    unsigned long long *bar = rg.bar + slot;
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, rg.bytes * NV);
    const S *g = src + (long long)sj * a.pitch + rg.seg0;
    S *sm = rg.buf + slot * NV * RG::SEG;
#pragma unroll
    for (int v = 0; v < NV; ++v) bulk_load(sm + v * RG::SEG, g + v * a.plane, rg.bytes, bar);
  }
}

// Every lane takes its cells of row j (relative row r) out of its slot,
// then the slot is refilled with relative row r + D (row j + D) if any.
template <class A, int V, int NV, int D, class G>
static __device__ __forceinline__ void ring_fetch(const G &a,
                                                  const typename Ops<A>::S *__restrict__ src,
                                                  RowRing<A, V, NV, D> &rg, int r, int j, int nrows,
                                                  A (&W)[V][NV]) {
  using S = typename Ops<A>::S;
  using RG = RowRing<A, V, NV, D>;
  constexpr int K = Ops<A>::K;
  int dir;
  row_src(a, j, dir);
  const int slot = r % D;
  if (dir >= 0) {
#pragma unroll
    for (int c = 0; c < V; ++c)
#pragma unroll
      for (int v = 0; v < NV; ++v) W[c][v] = Ops<A>::splat(a.bc_state[dir][v]);
  } else {
    if (!rg.broken) {
      const unsigned par = (rg.phase >> slot) & 1u;
      bool done = mbar_try_wait(rg.bar + slot, par);
      if (!done) {
        const unsigned long long t0 = timer_ns();
        while (!(done = mbar_try_wait(rg.bar + slot, par))) {
          if (timer_ns() - t0 > 20000000ull) break;  // 20 ms: a staged row never takes that long
        }
      }
      done = __all_sync(0xffffffffu, done);
      if (!done) {
        rg.broken = true;
        if ((threadIdx.x & 31) == 0) atomicOr(&a.ctrl->err_pending, kErrTimeout);
      }
      rg.phase ^= 1u << slot;
    }
    const S *sm = rg.buf + slot * NV * RG::SEG + rg.lane_off;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int c = 0; c < V; ++c) W[c][v] = Ops<A>::pack(sm + v * RG::SEG + c * K);
  }
  __syncwarp();
  if (r + D < nrows) ring_issue<A, V, NV, D>(a, src, rg, r + D, j + D);
}

// March one interior warp task through the TMA ring.
template <class Sys, class A, int V, int D, bool FIN, class G>
static __device__ __forceinline__ void march_tma(const G &a, const SysParams<A> &P,
                                                 const typename Ops<A>::S *__restrict__ src,
                                                 typename Ops<A>::S *__restrict__ dst,
                                                 RowRing<A, V, Sys::NV, D> &rg, int X, int y0, int y1,
                                                 bool writer, A lx, A ly, typename Ops<A>::P &lam_loc,
                                                 unsigned &bad) {
  using S = typename Ops<A>::S;
  constexpr int NV = Sys::NV, N = V * Ops<A>::K;
  using O = Ops<A>;
  // the lanes' cells span [X_0, X_31 + N); stage that span widened to 16 bytes
  const int x_first = __shfl_sync(0xffffffffu, X, 0);
  const int x_end = x_first + 32 * N;
  constexpr int AL = TmaGeom<S>::kAlign;
  rg.seg0 = x_first / AL * AL;
  const int seg1 = (x_end + AL - 1) / AL * AL;
  rg.bytes = (unsigned)((seg1 - rg.seg0) * (int)sizeof(S));
  rg.lane_off = X - rg.seg0;
  S *dst_lane = dst + X;
  const int nrows = y1 - y0 + 2;  // rows y0 - 1 .. y1
  const int pre = nrows < D ? nrows : D;
  for (int r = 0; r < pre; ++r) ring_issue<A, V, NV, D>(a, src, rg, r, y0 - 1 + r);
  RowState<A, V, NV> RA, RB;
  A Fs[V][NV];
  ring_fetch<A, V, NV, D>(a, src, rg, 0, y0 - 1, nrows, RA.W);
#pragma unroll
  for (int c = 0; c < V; ++c) {
    A Fx_[NV], sx_;
    Sys::fluxes(RA.W[c], P, Fx_, sx_, RA.Fy[c], RA.sy[c]);
  }
  ring_fetch<A, V, NV, D>(a, src, rg, 1, y0, nrows, RB.W);
  row_x<Sys, V>(P, RB.W, RB.Fy, RB.sy, RB.dX);
#pragma unroll
  for (int c = 0; c < V; ++c) {
    const A sg = O::max(RA.sy[c], RB.sy[c]);
#pragma unroll
    for (int v = 0; v < Sys::NU; ++v) Fs[c][v] = lf_face2(RA.W[c][v], RA.Fy[c][v], RB.W[c][v], RB.Fy[c][v], sg);
  }
  int j = y0;
  while (true) {
    if (j >= y1) break;
    ring_fetch<A, V, NV, D>(a, src, rg, j - y0 + 2, j + 1, nrows, RA.W);
    advance_row<Sys, A, V, true, FIN>(a, P, dst_lane, X, j, writer, lx, ly, RB, RA, Fs, lam_loc, bad);
    ++j;
    if (j >= y1) break;
    ring_fetch<A, V, NV, D>(a, src, rg, j - y0 + 2, j + 1, nrows, RB.W);
    advance_row<Sys, A, V, true, FIN>(a, P, dst_lane, X, j, writer, lx, ly, RA, RB, Fs, lam_loc, bad);
    ++j;
  }
}

// ---------------------------------------------------------------- cp.async rows
// Second staging scheme for interior strips: every lane copies its own cells
// of a row into its own slot of a per-warp ring in shared memory with
// cp.async (each lane later reads only what it copied, so no cross-lane
// synchronisation is needed); D - 1 rows stay in flight per lane.

static __device__ __forceinline__ void cp_async_bytes4(void *sdst, const void *gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
static __device__ __forceinline__ void cp_async_bytes8(void *sdst, const void *gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
static __device__ __forceinline__ void cp_async_bytes16(void *sdst, const void *gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int W>
static __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(W) : "memory");
}

template <class S, int N>
static __device__ __forceinline__ void cp_async_cells(S *sdst, const S *gsrc) {
  constexpr int B = N * (int)sizeof(S);
  if (B == 4) cp_async_bytes4(sdst, gsrc);
  else if (B == 8) cp_async_bytes8(sdst, gsrc);
  else if (B == 16) cp_async_bytes16(sdst, gsrc);
  else {
#pragma unroll
    for (int c = 0; c < N; ++c) {
      if (sizeof(S) == 8) cp_async_bytes8(sdst + c, gsrc + c);
      else cp_async_bytes4(sdst + c, gsrc + c);
    }
  }
}

// A lane's private ring: D slots x NV variables x N cells, lanes interleaved
// so a warp's copies of one variable land in one contiguous 32 * N span.
template <class S, int N, int NV, int D> struct LaneRing {
  S *buf;
  __device__ __forceinline__ S *slot(int s, int v) const { return buf + ((s * NV + v) * 32) * N; }
};

// Issue the copies of row j into ring slot r % D.  Interior strips (xin)
// copy each lane's N contiguous cells per variable; strips at the east or
// west boundary map every cell through lane_cols: a real or ghost column is
// copied on its own (4 or 8 bytes; 2-byte cells are loaded and stored
// directly), a Dirichlet ghost value is stored directly.  Direct stores land
// in the lane's own slots, so program order makes them visible to its reads.
template <class A, int V, int NV, int D, class G>
static __device__ __forceinline__ void lring_issue(const G &a,
                                                   const typename Ops<A>::S *__restrict__ src, int X, bool xin,
                                                   const LaneRing<typename Ops<A>::S, V * Ops<A>::K, NV, D> &rg,
                                                   int r, int j) {
  using S = typename Ops<A>::S;
  constexpr int N = V * Ops<A>::K;
  int dir;
  const int sj = row_src(a, j, dir);
  const int slot = r % D;
  if (dir >= 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int c = 0; c < N; ++c) rg.slot(slot, v)[c] = (S)a.bc_state[dir][v];
  } else if (xin) {
    const S *g = src + X + (long long)sj * a.pitch;
#pragma unroll
    for (int v = 0; v < NV; ++v) cp_async_cells<S, N>(rg.slot(slot, v), g + v * a.plane);
  } else {
    const LaneCols<N> L = lane_cols<N>(a, X);
    const S *g = src + (long long)sj * a.pitch;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int c = 0; c < N; ++c) {
        S *d = rg.slot(slot, v) + c;
        if (L.dir[c] >= 0) *d = (S)a.bc_state[L.dir[c]][v];
        else if (sizeof(S) >= 4) cp_async_cells<S, 1>(d, g + v * a.plane + L.col[c]);
        else *d = __ldcg(g + v * a.plane + L.col[c]);
      }
  }
  cp_async_commit();
}

// Own row j of a lane of a ragged last strip whose cells reach past the
// grid, cell by cell: columns inside the grid from the state, the ghost
// column nx from the boundary condition (the first column's cell of the
// west column strip of the task at the start of the row, across the
// periodic side; the task's own last column; or the prescribed state), the
// cells past it (which no face uses) from the same source.
template <class A, int V, int NV, int D, int TY, class G>
static __device__ __forceinline__ void lring_issue_cells(const G &a, const typename Ops<A>::S *W, int X,
                                                         const Ovl<typename Ops<A>::S> &o,
                                                         const LaneRing<typename Ops<A>::S, V * Ops<A>::K, NV, D> &rg,
                                                         int slot, int j) {
  using S = typename Ops<A>::S;
  constexpr int N = V * Ops<A>::K, SW = 30 * N;
  using L = OvlLayout<NV, N, SW>;
  const S *g;
  long long gvs;
  if (a.bc[kE] == kPeriodic) {
    // the first task of this chunk (strip 0): task - task % nstrips
    const int task = ovl_opaque<N>(o.task);
    g = ovl_rd<N>(a, o) + (long long)(task - task % a.nstrips) * a.ovl_task + L::colW(TY) + (j - o.y0) * N;
    gvs = (long long)TY * N;
  } else if (a.bc[kE] == kDirichlet) {
    g = a.ovl_bc + kE * NV * N;
    gvs = N;
  } else {
    g = W + (long long)j * a.pitch + (a.nx - 1);
    gvs = a.plane;
  }
  const S *row = W + (long long)j * a.pitch;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    const bool in = X + c < a.nx;
    const S *q = in ? row + X + c : g;
    const long long vs = in ? a.plane : gvs;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      S *d = rg.slot(slot, v) + c;
      if (sizeof(S) >= 4) cp_async_cells<S, 1>(d, q + v * vs);
      else *d = __ldcg(q + v * vs);
    }
  }
}

// In-place counterpart of lring_issue.  A lane copies one vector of N cells
// per variable from the source ovl_halo_src (halo rows) or ovl_lane_setup
// (own rows) gives: its own cells of the state, a neighbour's column or row
// strip, or the prescribed state's cells; only the own rows of the lanes of
// a ragged last strip that reach past the grid go cell by cell.
template <class A, int V, int NV, int D, int TY, class G>
static __device__ __forceinline__ void lring_issue_inplace(const G &a, const typename Ops<A>::S *W, int X,
                                                           const Ovl<typename Ops<A>::S> &o,
                                                           const LaneRing<typename Ops<A>::S, V * Ops<A>::K, NV, D> &rg,
                                                           int r, int j) {
  using S = typename Ops<A>::S;
  constexpr int N = V * Ops<A>::K;
  const int slot = r % D;
  const bool own = j >= o.y0 && j < o.y1;
  if (!own) {
    long long vs;
    const S *p = ovl_halo_src<NV, N, TY>(a, o, X, j, vs);
#pragma unroll
    for (int v = 0; v < NV; ++v) cp_async_cells<S, N>(rg.slot(slot, v), p + v * vs);
  } else if (__builtin_expect((o.flags & kPercell) != 0u, 0)) {
    lring_issue_cells<A, V, NV, D, TY>(a, W, X, o, rg, slot, j);
  } else {
    int ors;
    long long ovs;
    if constexpr (N < 4) {
      ors = o.ors;
      ovs = o.ovs;
    } else {
      ors = (o.flags & kOwnStrip) ? N : (o.flags & kOwnDir) ? 0 : (int)a.pitch;
      ovs = (o.flags & kOwnStrip) ? (long long)TY * N : (o.flags & kOwnDir) ? (long long)N : a.plane;
    }
    const S *p = o.op + (long long)(j - o.y0) * ors;
#pragma unroll
    for (int v = 0; v < NV; ++v) cp_async_cells<S, N>(rg.slot(slot, v), p + v * ovs);
  }
  cp_async_commit();
}

template <class A, int V, int NV, int D>
static __device__ __forceinline__ void lring_read(const LaneRing<typename Ops<A>::S, V * Ops<A>::K, NV, D> &rg,
                                                  int r, A (&W)[V][NV]) {
  constexpr int K = Ops<A>::K;
  const int slot = r % D;
  if constexpr (std::is_same<A, BF>::value && V % 2 == 0) {
    // bfloat16 cells two at a time from the slot's 32-bit words: a bfloat16
    // is the upper half of an FP32, so the cell in the low half (the lower
    // address) widens to the word shifted up by 16, the one in the high half
    // to the word with its low 16 bits cleared -- one bit operation per cell
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const unsigned *q = reinterpret_cast<const unsigned *>(rg.slot(slot, v));
#pragma unroll
      for (int c = 0; c < V; c += 2) {
        const unsigned w = q[c / 2];
        W[c][v].v = __uint_as_float(w << 16);
        W[c + 1][v].v = __uint_as_float(w & 0xffff0000u);
      }
    }
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const typename Ops<A>::S *p = rg.slot(slot, v);
#pragma unroll
      for (int c = 0; c < V; ++c) W[c][v] = Ops<A>::pack(p + c * K);
    }
  }
}

// March one warp task through the per-lane cp.async ring (xin: interior
// strip, every lane's cells inside the grid; one code body serves both kinds
// of strips, which keeps the instruction footprint small when a launch mixes
// them).  Rows
// are numbered r = 0 .. nrows - 1 (row y0 - 1 + r); before reading row r the
// lane has issued rows up to r + D - 2 and waits until at most D - 2 copy
// groups are pending, i.e. row r has landed.  A slot is refilled only after
// the row read from it has been consumed by the flux computation.
template <class Sys, class A, int V, int D, bool FIN, bool INPL = false, int TYC = 0, class G>
static __device__ __forceinline__ void march_async(const G &a, const SysParams<A> &P,
                                                   const typename Ops<A>::S *src,
                                                   typename Ops<A>::S *dst,
                                                   const LaneRing<typename Ops<A>::S, V * Ops<A>::K, Sys::NV, D> &rg,
                                                   int X, bool xin, int y0, int y1, bool writer, A lx, A ly,
                                                   typename Ops<A>::P &lam_loc, unsigned &bad,
                                                   const Ovl<typename Ops<A>::S> *ovl = nullptr) {
  using S = typename Ops<A>::S;
  constexpr int NV = Sys::NV;
  using O = Ops<A>;
  S *dst_lane = dst + X;
  const int nrows = y1 - y0 + 2;
  auto issue = [&](int r, int j) {
    if constexpr (INPL) lring_issue_inplace<A, V, NV, D, TYC>(a, src, X, *ovl, rg, r, j);
    else lring_issue<A, V, NV, D>(a, src, X, xin, rg, r, j);
  };
  // prologue: rows 0 .. D-2 in flight (empty groups past the end keep the count)
#pragma unroll
  for (int r = 0; r < D - 1; ++r) {
    if (r < nrows) issue(r, y0 - 1 + r);
    else cp_async_commit();
  }
  RowState<A, V, NV> RA, RB;
  A Fs[V][NV];
  const int lane = threadIdx.x & 31;
  auto read = [&](int r, A(&W)[V][NV]) {
    lring_read<A, V, NV, D>(rg, r, W);
    if constexpr (INPL) ovl_fix_cols<A, V, NV>(a, *ovl, W, lane);
  };
  cp_async_wait<D - 2>();
  read(0, RA.W);
#pragma unroll
  for (int c = 0; c < V; ++c) {
    A Fx_[NV], sx_;
    Sys::fluxes(RA.W[c], P, Fx_, sx_, RA.Fy[c], RA.sy[c]);
  }
  if (D - 1 < nrows) issue(D - 1, y0 - 1 + D - 1);
  else cp_async_commit();
  cp_async_wait<D - 2>();
  read(1, RB.W);
  row_x<Sys, V>(P, RB.W, RB.Fy, RB.sy, RB.dX);
  if (D < nrows) issue(D, y0 - 1 + D);
  else cp_async_commit();
#pragma unroll
  for (int c = 0; c < V; ++c) {
    const A sg = O::max(RA.sy[c], RB.sy[c]);
#pragma unroll
    for (int v = 0; v < Sys::NU; ++v) Fs[c][v] = lf_face2(RA.W[c][v], RA.Fy[c][v], RB.W[c][v], RB.Fy[c][v], sg);
  }
  int j = y0;
  while (true) {
    if (j >= y1) break;
    {
      const int r = j - y0 + 2;
      cp_async_wait<D - 2>();
      read(r, RA.W);
      advance_row<Sys, A, V, false, FIN, INPL, TYC>(a, P, dst_lane, X, j, writer, lx, ly, RB, RA, Fs, lam_loc, bad, xin, ovl);
      if (r + D - 1 < nrows) issue(r + D - 1, y0 - 1 + r + D - 1);
      else cp_async_commit();
    }
    ++j;
    if (j >= y1) break;
    {
      const int r = j - y0 + 2;
      cp_async_wait<D - 2>();
      read(r, RB.W);
      advance_row<Sys, A, V, false, FIN, INPL, TYC>(a, P, dst_lane, X, j, writer, lx, ly, RA, RB, Fs, lam_loc, bad, xin, ovl);
      if (r + D - 1 < nrows) issue(r + D - 1, y0 - 1 + r + D - 1);
      else cp_async_commit();
    }
    ++j;
  }
  cp_async_wait<0>();
}

// Dynamic shared memory per block of the staging rings.
template <class A, int V, int NV, int D>
constexpr __host__ __device__ int tma_smem_bytes(int NW) {
  using S = typename Ops<A>::S;
  return NW * (D * NV * TmaGeom<S>::seg(V * Ops<A>::K) * (int)sizeof(S) + D * 8);
}
template <class A, int V, int NV, int D>
constexpr __host__ __device__ int async_smem_bytes(int NW) {
  return NW * D * NV * 32 * V * Ops<A>::K * (int)sizeof(typename Ops<A>::S);
}

// The fused step.  A: arithmetic type (float, double or F2 = two packed FP32
// cells); V: values of A per lane; TY: rows per warp task; NW: warps per block;
// FIN: this launch also reduces lmax(W^{n+1}) and closes the step (every
// system but spray, whose source kernel closes the step instead); MINB: blocks
// per SM the register budget targets; D: row staging (see the file header).
template <class Sys, class A, int V, int TY, int NW, bool FIN = true, int MINB = 1, int D = 0, bool INPL = false>
__global__ void __launch_bounds__(NW * 32, MINB)
fv_step_kernel(const StepArgs<typename Ops<A>::S> a) {
  using S = typename Ops<A>::S;
  constexpr int NV = Sys::NV, N = V * Ops<A>::K;
  __shared__ double s_lam[NW];
  __shared__ int s_bad[NW];
  __shared__ StepStart s_st;
  extern __shared__ __align__(128) unsigned char s_dyn[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  constexpr int DT = D > 0 ? D : 1;
  constexpr int DA = D < 0 ? -D : 2;
  RowRing<A, V, NV, DT> rg;
  LaneRing<S, N, NV, DA> lrg;
  if (D > 0) {
    constexpr int slot_bytes = DT * NV * RowRing<A, V, NV, DT>::SEG * (int)sizeof(S);
    unsigned char *mine = s_dyn + warp * (slot_bytes + DT * 8);
    rg.buf = reinterpret_cast<S *>(mine);
    rg.bar = reinterpret_cast<unsigned long long *>(mine + slot_bytes);
    rg.phase = 0u;
    rg.broken = false;
    if (lane == 0)
      for (int k = 0; k < DT; ++k) mbar_init(rg.bar + k, 1);
    fence_proxy_async();
    __syncwarp();
  }
  if (D < 0) lrg.buf = reinterpret_cast<S *>(s_dyn) + warp * (DA * NV * 32 * N) + lane * N;
  if (threadIdx.x == 0) s_st = read_step_start(a.pol, a.ctrl);
  __syncthreads();
  const StepStart st = s_st;
  typename Ops<A>::P lam_loc = 0;
  unsigned bad = 0u;

  if (st.run) {
    const long long n = st.step;
    // in place: buf0 == buf1, so src == dst
    const S *src = st.cur ? a.buf1 : a.buf0;
    S *dst = st.cur ? a.buf0 : a.buf1;
    const SysParams<A> P = splat_params<A>(a.sp);
    // half steps: the face fluxes are carried doubled (see lf_face2)
    const A lx = Ops<A>::splat((typename Ops<A>::P)(0.5 * (st.dt / a.dx)));
    const A ly = Ops<A>::splat((typename Ops<A>::P)(0.5 * (st.dt / a.dy)));
    const bool writer = lane >= 1 && lane <= 30;
    const int gw = blockIdx.x * NW + warp;
    const int GW = gridDim.x * NW;
    for (int task = gw; task < a.ntasks; task += GW) {
      const int sx_ = task % a.nstrips;
      const int cy = task / a.nstrips;
      const int X = sx_ * (30 * N) + (lane - 1) * N;
      const int ty = INPL ? TY : a.ty;
      const int y0 = cy * ty;
      const int y1 = min(y0 + ty, a.ny);
      // warp-uniform: does every lane of the strip read real columns only?
      const bool xin = __all_sync(0xffffffffu, X >= 0 && X + N <= a.nx);
      if constexpr (INPL && D < 0) {
        Ovl<S> o;
        o.task = task;
        o.y0 = y0;
        o.y1 = y1;
        ovl_lane_setup<NV, N, TY>(a, src, o, X, lane, sx_, cy, n);
        march_async<Sys, A, V, DA, FIN, true, TY>(a, P, src, dst, lrg, X, xin, y0, y1, writer, lx, ly, lam_loc, bad, &o);
      } else {
        if (D > 0 && xin) march_tma<Sys, A, V, DT, FIN>(a, P, src, dst, rg, X, y0, y1, writer, lx, ly, lam_loc, bad);
        else if (D < 0) march_async<Sys, A, V, DA, FIN>(a, P, src, dst, lrg, X, xin, y0, y1, writer, lx, ly, lam_loc, bad);
        else if (xin) march<Sys, A, V, true, FIN>(a, P, src, dst, X, y0, y1, writer, lx, ly, lam_loc, bad);
        else march<Sys, A, V, false, FIN>(a, P, src, dst, X, y0, y1, writer, lx, ly, lam_loc, bad);
      }
    }
  }

  if (!FIN) return;
  finish_step<NW>(a.ctrl, st, (double)lam_loc, bad != 0u, s_lam, s_bad);
}

// In-place mode: the overlap strips of one parity from the state itself,
// after the host loaded or moved the state (layout of OvlLayout; cells of a
// strip past the task's last column get that column's values, so every
// strip cell is a finite state value).
// In-place mode: the prescribed state of each side as stored cells,
// [side][variable][n cells] (converted to the storage type exactly as the
// ring's Dirichlet ghosts are).
template <class S> struct BcCells {
  typename ParamOf<S>::T v[4][8];
};
template <class S>
__global__ void fill_bc_cells_kernel(BcCells<S> bc, int nv, int n, S *dst) {
  const int k = threadIdx.x;
  if (k < 4 * nv * n) dst[k] = (S)bc.v[k / (nv * n)][(k / n) % nv];
}

template <class S>
__global__ void fill_ovl_kernel(const S *W, int nx, int ny, long long pitch, long long plane, int nv,
                                int nstrips, int nchunks, int ty, int n, int sw, int ts, S *ovl) {
  const long long per = (long long)nv * (2 * ty * n + 2 * sw);
  const long long total = (long long)nstrips * nchunks * per;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(k / per);
    const int e = (int)(k - (long long)t * per);
    const int sx = t % nstrips, cy = t / nstrips;
    const int X0 = sx * sw, y0 = cy * ty, y1 = min(y0 + ty, ny);
    const int last = min(X0 + sw, nx) - 1;
    int j, col, v;
    if (e < 2 * nv * ty * n) {
      // column strips: west = the task's first n columns, east = its last n
      const int which = e / (nv * ty * n), rem = e % (nv * ty * n);
      v = rem / (ty * n);
      const int rc = rem % (ty * n);
      j = y0 + rc / n;
      const int c = rc % n;
      col = which == 0 ? min(X0 + c, last) : max(last - (n - 1 - c), X0);
      if (j >= y1) j = y1 - 1;
    } else {
      const int e2 = e - 2 * nv * ty * n;
      const int which = e2 / (nv * sw), rem = e2 % (nv * sw);
      v = rem / sw;
      col = min(X0 + rem % sw, last);
      j = which == 0 ? y0 : y1 - 1;
    }
    ovl[(long long)t * ts + e] = W[(long long)v * plane + (long long)j * pitch + col];
  }
}

}  // namespace fv
