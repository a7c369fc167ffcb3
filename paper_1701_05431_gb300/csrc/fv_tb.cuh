// fv_tb.cuh -- two time steps per pass over the state (temporal blocking),
// for the paper's constant dt (Sec. 2.2.1), with any boundary conditions.
//
// One warp task marches up its strip as in fv_step.cuh, but each row of W^n
// it loads feeds two levels of the march: level 1 turns W^n rows into W^{n+1}
// rows in registers, level 2 turns those into W^{n+2} rows, which alone are
// stored.  The state is read once and written once per two steps, halving
// the bytes per cell-update.  A task of TY output rows reads W^n rows
// y0 - 2 .. y1 + 1, and each lane holds V >= 2 cells, so the halo lanes 0
// and 31 carry the two halo columns a double step needs; level 1 computes
// W^{n+1} on the one-cell ring around the task (its other halo values are
// never used).  Ghost cells of a periodic side are cells of the grid, so
// there rows and columns simply wrap.  On a transmissive or Dirichlet side
// the ring cells beyond the boundary are ghosts of W^{n+1}, not cells of
// the scheme: level 1 loads the ghosts of W^n from the boundary condition
// (a second ghost layer, which only feeds ring cells that are replaced, is
// a copy of the first), and before level 2 reads a level-1 row, its ghost
// cells are replaced by the boundary condition applied to W^{n+1} (a copy
// of the border cell as stored, or the prescribed state), exactly what the
// single step's loader would give them.
//
// Level 1 and level 2 use exactly the arithmetic of a single step, so a pass
// gives the bits of two single steps.  The paper's check dt lmax(W^{n+1}) <=
// min(dx, dy) is made on the W^{n+1} cells each task owns; if it fails (or
// W^{n+1} is inadmissible) the pass changes nothing but a flag, and the host
// redoes the two steps one at a time, so errors come at the same step as
// without blocking.
#pragma once

#include "fv_step.cuh"

namespace fv {

enum : unsigned { kErrReplay = 16u };  // a two-step pass found W^{n+1} failing the check

static __device__ __forceinline__ int tb_wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Source of index i (a row or a column, any integer) of W^n along an axis of
// n cells whose low and high sides have boundary conditions blo and bhi: the
// wrapped index on a periodic axis; else the index itself inside the grid
// and, beyond it, the border cell (transmissive) or, through *dir, the
// Dirichlet side (sides slo and shi).  Only the first ghost layer feeds
// cells the pass keeps; the second one just has to be finite.
static __device__ __forceinline__ int tb_src(int i, int n, int blo, int bhi, int slo, int shi, int &dir) {
  dir = -1;
  if (i < 0) {
    if (blo == kPeriodic) return tb_wrap(i, n);
    if (blo == kDirichlet) dir = slo;
    return 0;
  }
  if (i >= n) {
    if (bhi == kPeriodic) return tb_wrap(i, n);
    if (bhi == kDirichlet) dir = shi;
    return n - 1;
  }
  return i;
}

// Copies of W^n row j (any integer) into ring slot r % D: each lane's N
// cells, wrapped when every side is periodic (NP false), else through
// tb_src in both directions, Dirichlet ghost cells being stored directly in
// the storage type, as the single step's ring does.
template <class A, int V, int NV, int D, bool NP, class G>
static __device__ __forceinline__ void tb_issue(const G &a, const typename Ops<A>::S *src, int X, bool xin,
                                                const LaneRing<typename Ops<A>::S, V * Ops<A>::K, NV, D> &rg,
                                                int r, int j) {
  using S = typename Ops<A>::S;
  constexpr int N = V * Ops<A>::K;
  const int slot = r % D;
  if constexpr (!NP) {
    // every side periodic: rows and columns wrap
    const S *g = src + (long long)tb_wrap(j, a.ny) * a.pitch;
    if (xin) {
#pragma unroll
      for (int v = 0; v < NV; ++v) cp_async_cells<S, N>(rg.slot(slot, v), g + X + v * a.plane);
    } else {
#pragma unroll
      for (int c = 0; c < N; ++c) {
        const int col = tb_wrap(X + c, a.nx);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          S *d = rg.slot(slot, v) + c;
          if (sizeof(S) >= 4) cp_async_cells<S, 1>(d, g + col + v * a.plane);
          else *d = __ldcg(g + col + v * a.plane);
        }
      }
    }
    cp_async_commit();
    return;
  }
  int rdir;
  const int sj = tb_src(j, a.ny, a.bc[kS], a.bc[kN], kS, kN, rdir);
  const S *g = src + (long long)sj * a.pitch;
  if (rdir >= 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int c = 0; c < N; ++c) rg.slot(slot, v)[c] = (S)a.bc_state[rdir][v];
  } else if (xin) {
#pragma unroll
    for (int v = 0; v < NV; ++v) cp_async_cells<S, N>(rg.slot(slot, v), g + X + v * a.plane);
  } else {
#pragma unroll
    for (int c = 0; c < N; ++c) {
      int cdir;
      const int col = tb_src(X + c, a.nx, a.bc[kW], a.bc[kE], kW, kE, cdir);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        S *d = rg.slot(slot, v) + c;
        if (cdir >= 0) *d = (S)a.bc_state[cdir][v];
        else if (sizeof(S) >= 4) cp_async_cells<S, 1>(d, g + col + v * a.plane);
        else *d = __ldcg(g + col + v * a.plane);
      }
    }
  }
  cp_async_commit();
}

// The prescribed state of side `side` as a stored cell (rounded to the
// storage type), in every cell of a row of the lane.
template <class A, int V, int NV, class G>
static __device__ __forceinline__ void tb_dirichlet_row(const G &a, int side, A (&W)[V][NV]) {
  using S = typename Ops<A>::S;
  constexpr int K = Ops<A>::K;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    S t[K];
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = (S)a.bc_state[side][v];
#pragma unroll
    for (int c = 0; c < V; ++c) W[c][v] = Ops<A>::pack(t);
  }
}

// Ghost columns of a level-1 row (W^{n+1}, rounded to storage) on the
// non-periodic sides: column -1 (lane 0's last cell on the first strip) and
// column nx (in the lane whose cells reach past the grid on the last strip)
// take the boundary condition applied to W^{n+1}.  Every lane takes part in
// the shuffles.  X0: the strip's first column.
template <class A, int V, int NV, class G>
static __device__ __forceinline__ void tb_fix_cols(const G &a, A (&W)[V][NV], int X, int X0, int lane) {
  static_assert(Ops<A>::K == 1, "two-step passes use one cell per value");
  using O = Ops<A>;
  using S = typename O::S;
  constexpr int N = V;
  if (a.bc[kW] != kPeriodic && X0 == 0) {
    A g[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const A w0 = O::shfl_down(W[0][v], 1);  // lane 1's first cell: column 0
      S t[1] = {(S)a.bc_state[kW][v]};
      g[v] = a.bc[kW] == kDirichlet ? O::pack(t) : w0;
    }
    if (lane == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) W[V - 1][v] = g[v];
    }
  }
  if (a.bc[kE] != kPeriodic && X0 + 30 * N >= a.nx) {
    A up[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) up[v] = O::shfl_up(W[V - 1][v], 1);  // the west lane's last cell
    const int rel = a.nx - X;  // this lane's cell holding column nx, if 0 <= rel < N
#pragma unroll
    for (int c = 0; c < V; ++c)
      if (c == rel) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          S t[1] = {(S)a.bc_state[kE][v]};
          W[c][v] = a.bc[kE] == kDirichlet ? O::pack(t) : (c == 0 ? up[v] : W[c > 0 ? c - 1 : 0][v]);
        }
      }
  }
}

// One row of one level: x-work of `nxt`, the y-face between `cur` and `nxt`,
// and the updated values of `cur`'s row for every lane (the arithmetic of
// advance_row, without the store).
template <class Sys, class A, int V, bool USEQ = false>
static __device__ __forceinline__ void tb_level_row(const SysParams<A> &P, RowState<A, V, Sys::NV> &cur,
                                                    RowState<A, V, Sys::NV> &nxt, A (&Fs)[V][Sys::NV], A lx, A ly,
                                                    A (&Wn)[V][Sys::NV], const A (*Q)[4] = nullptr) {
  row_x<Sys, V, USEQ>(P, nxt.W, nxt.Fy, nxt.sy, nxt.dX, Q);
  static_assert(Sys::NU == Sys::NV, "two-step passes carry no planes");
  faces_update_row<Sys, A, V>(cur, nxt, Fs, lx, ly, Wn);
}

// A level-1 row as the state stores it: rounded to the storage type, as a
// single step's store and the next step's load would round it (a no-op for
// FP32 and FP64 storage).
template <class A, int V, int NV>
static __device__ __forceinline__ void tb_round_to_storage(A (&W)[V][NV]) {
  using O = Ops<A>;
  using S = typename O::S;
  constexpr int K = O::K;
#pragma unroll
  for (int c = 0; c < V; ++c)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      S t[K];
      O::unpack(W[c][v], t);
      W[c][v] = O::pack(t);
    }
}

// Wave speed and admissibility of the cells of a produced row this lane owns.
template <class Sys, class A, int V>
static __device__ __forceinline__ void tb_lambda(const SysParams<A> &P, const A (&Wn)[V][Sys::NV], int X, int nx,
                                                 bool writer, typename Ops<A>::P &lam, unsigned &bad) {
  using O = Ops<A>;
  constexpr int K = Ops<A>::K;
  if (!writer) return;
#pragma unroll
  for (int c = 0; c < V; ++c) {
    unsigned valid = 0u;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (X + c * K + k < nx) valid |= 1u << k;
    unsigned b;
    const A l = Sys::lambda(Wn[c], P, b);
    lam = fmax(lam, O::hmax(l, valid));
    bad |= b & valid;
  }
}

// The same from the cells' primitives Q (Euler): the bits of tb_lambda.
template <class Sys, class A, int V>
static __device__ __forceinline__ void tb_lambda_q(const A (&Wn)[V][Sys::NV], const A (&Q)[V][4], int X, int nx,
                                                   bool writer, typename Ops<A>::P &lam, unsigned &bad) {
  using O = Ops<A>;
  if (!writer) return;
#pragma unroll
  for (int c = 0; c < V; ++c) {
    const unsigned valid = X + c < nx ? 1u : 0u;
    unsigned b;
    const A l = Sys::lambda_from(Wn[c], Q[c], b);
    lam = fmax(lam, O::hmax(l, valid));
    bad |= b & valid;
  }
}

// Level 1's rows feed level 2 as they are produced: with FP32 or FP64
// storage (no rounding between the levels) the primitives of a level-1 row
// serve both its wave-speed check and level 2's fluxes of that row, one
// recovery instead of two.  The ghost columns and rows are set first, so
// the primitives are those of the row level 2 reads; the check only looks at
// cells inside the grid, which the ghosts leave alone.
template <class Sys, class A>
struct TbReuse {
  static constexpr bool value = std::is_same<Sys, Euler>::value &&
                                (std::is_same<A, float>::value || std::is_same<A, double>::value);
};

template <class Sys, class A, int V, class G>
static __device__ __forceinline__ void tb_store(const G &a, const A (&Wn)[V][Sys::NV], typename Ops<A>::S *dst_lane,
                                                int X, int j, bool writer) {
  using S = typename Ops<A>::S;
  using O = Ops<A>;
  constexpr int NV = Sys::NV, K = Ops<A>::K, N = V * K;
  if (!writer) return;
  S *row = dst_lane + (long long)j * a.pitch;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    S t[N];
#pragma unroll
    for (int c = 0; c < V; ++c) O::unpack(Wn[c][v], t + c * K);
    if (X + N <= a.nx) {
      VecIO<S, N>::st(row + v * a.plane, t);
    } else {
#pragma unroll
      for (int c = 0; c < N; ++c)
        if (X + c < a.nx) __stcs(row + v * a.plane + c, t[c]);
    }
  }
}

// The two-level march of one warp task (rows [y0, y1) of W^{n+2}).
template <class Sys, class A, int V, int D, bool NP, class G>
static __device__ __forceinline__ void march_tb(const G &a, const SysParams<A> &P, const typename Ops<A>::S *src,
                                                typename Ops<A>::S *dst,
                                                const LaneRing<typename Ops<A>::S, V * Ops<A>::K, Sys::NV, D> &rg,
                                                int X, int X0, int lane, bool xin, int y0, int y1, bool writer,
                                                A lx, A ly, typename Ops<A>::P &lam1, unsigned &bad1,
                                                typename Ops<A>::P &lam2, unsigned &bad2) {
  using S = typename Ops<A>::S;
  constexpr int NV = Sys::NV;
  constexpr bool REUSE = TbReuse<Sys, A>::value;
  using O = Ops<A>;
  S *dst_lane = dst + X;
  // ghost rows of W^{n+1} below row 0 and above row ny - 1 on non-periodic
  // sides (NP: the kernel built for grids with such sides)
  const bool gS = NP && a.bc[kS] != kPeriodic && y0 == 0;
  const bool gN = NP && a.bc[kN] != kPeriodic && y1 == a.ny;
  const int nrows = y1 - y0 + 4;  // W^n rows y0 - 2 .. y1 + 1
  auto issue = [&](int r) {
    if (r < nrows) tb_issue<A, V, NV, D, NP>(a, src, X, xin, rg, r, y0 - 2 + r);
    else cp_async_commit();
  };
  auto fetch = [&](int r, A(&W)[V][NV]) {
    cp_async_wait<D - 2>();
    lring_read<A, V, NV, D>(rg, r, W);
    issue(r + D - 1);
  };
#pragma unroll
  for (int r = 0; r < D - 1; ++r) issue(r);
  RowState<A, V, NV> R1a, R1b, R2a, R2b;
  A Fs1[V][NV], Fs2[V][NV], Wn[V][NV], Wm[V][NV];
  // level 1 prologue: rows y0 - 2 (its y-fluxes) and y0 - 1
  fetch(0, R1a.W);
#pragma unroll
  for (int c = 0; c < V; ++c) {
    A Fx_[NV], sx_;
    Sys::fluxes(R1a.W[c], P, Fx_, sx_, R1a.Fy[c], R1a.sy[c]);
  }
  fetch(1, R1b.W);
  row_x<Sys, V>(P, R1b.W, R1b.Fy, R1b.sy, R1b.dX);
#pragma unroll
  for (int c = 0; c < V; ++c) {
    const A sg = O::max(R1a.sy[c], R1b.sy[c]);
#pragma unroll
    for (int v = 0; v < NV; ++v) Fs1[c][v] = lf_face2(R1a.W[c][v], R1a.Fy[c][v], R1b.W[c][v], R1b.Fy[c][v], sg);
  }
  // W^{n+1} row y0 - 1: level 2's south halo row (its y-fluxes only)
  fetch(2, R1a.W);
  tb_level_row<Sys, A, V>(P, R1b, R1a, Fs1, lx, ly, Wn);
  tb_round_to_storage<A, V, NV>(Wn);
  if constexpr (NP) tb_fix_cols<A, V, NV>(a, Wn, X, X0, lane);
#pragma unroll
  for (int c = 0; c < V; ++c)
#pragma unroll
    for (int v = 0; v < NV; ++v) R2a.W[c][v] = Wn[c][v];
  // W^{n+1} row y0: level 2's first own row
  fetch(3, R1b.W);
  tb_level_row<Sys, A, V>(P, R1a, R1b, Fs1, lx, ly, Wn);
  tb_lambda<Sys, A, V>(P, Wn, X, a.nx, writer, lam1, bad1);
  tb_round_to_storage<A, V, NV>(Wn);
  if constexpr (NP) tb_fix_cols<A, V, NV>(a, Wn, X, X0, lane);
#pragma unroll
  for (int c = 0; c < V; ++c)
#pragma unroll
    for (int v = 0; v < NV; ++v) R2b.W[c][v] = Wn[c][v];
  // below row 0 of a non-periodic grid the halo row is the ghost of W^{n+1}
  if (gS) {
    if (a.bc[kS] == kDirichlet) {
      tb_dirichlet_row<A, V, NV>(a, kS, R2a.W);
    } else {
#pragma unroll
      for (int c = 0; c < V; ++c)
#pragma unroll
        for (int v = 0; v < NV; ++v) R2a.W[c][v] = R2b.W[c][v];
    }
  }
#pragma unroll
  for (int c = 0; c < V; ++c) {
    A Fx_[NV], sx_;
    Sys::fluxes(R2a.W[c], P, Fx_, sx_, R2a.Fy[c], R2a.sy[c]);
  }
  row_x<Sys, V>(P, R2b.W, R2b.Fy, R2b.sy, R2b.dX);
#pragma unroll
  for (int c = 0; c < V; ++c) {
    const A sg = O::max(R2a.sy[c], R2b.sy[c]);
#pragma unroll
    for (int v = 0; v < NV; ++v) Fs2[c][v] = lf_face2(R2a.W[c][v], R2a.Fy[c][v], R2b.W[c][v], R2b.Fy[c][v], sg);
  }
  // rows k = y0 + 1 .. y1 of W^{n+1}; each gives row k - 1 of W^{n+2}
  // (both levels swap their row states every row: unrolled by two)
  int k = y0 + 1;
  while (true) {
    if (k > y1) break;
    fetch(k - y0 + 3, R1a.W);
    tb_level_row<Sys, A, V>(P, R1b, R1a, Fs1, lx, ly, Wn);
    if constexpr (!REUSE) {
      if (k < y1) tb_lambda<Sys, A, V>(P, Wn, X, a.nx, writer, lam1, bad1);
    }
    tb_round_to_storage<A, V, NV>(Wn);
    if constexpr (NP) tb_fix_cols<A, V, NV>(a, Wn, X, X0, lane);
#pragma unroll
    for (int c = 0; c < V; ++c)
#pragma unroll
      for (int v = 0; v < NV; ++v) R2a.W[c][v] = Wn[c][v];
    if (gN && k == y1) {
      // row ny: the ghost of W^{n+1} above the grid (R2b holds row ny - 1)
      if (a.bc[kN] == kDirichlet) {
        tb_dirichlet_row<A, V, NV>(a, kN, R2a.W);
      } else {
#pragma unroll
        for (int c = 0; c < V; ++c)
#pragma unroll
          for (int v = 0; v < NV; ++v) R2a.W[c][v] = R2b.W[c][v];
      }
    }
    if constexpr (REUSE) {
      A Q[V][4];
#pragma unroll
      for (int c = 0; c < V; ++c) Sys::prims4(R2a.W[c], P, Q[c]);
      if (k < y1) tb_lambda_q<Sys, A, V>(R2a.W, Q, X, a.nx, writer, lam1, bad1);
      tb_level_row<Sys, A, V, true>(P, R2b, R2a, Fs2, lx, ly, Wm, Q);
    } else {
      tb_level_row<Sys, A, V>(P, R2b, R2a, Fs2, lx, ly, Wm);
    }
    tb_store<Sys, A, V>(a, Wm, dst_lane, X, k - 1, writer);
    tb_lambda<Sys, A, V>(P, Wm, X, a.nx, writer, lam2, bad2);
    ++k;
    if (k > y1) break;
    fetch(k - y0 + 3, R1b.W);
    tb_level_row<Sys, A, V>(P, R1a, R1b, Fs1, lx, ly, Wn);
    if constexpr (!REUSE) {
      if (k < y1) tb_lambda<Sys, A, V>(P, Wn, X, a.nx, writer, lam1, bad1);
    }
    tb_round_to_storage<A, V, NV>(Wn);
    if constexpr (NP) tb_fix_cols<A, V, NV>(a, Wn, X, X0, lane);
#pragma unroll
    for (int c = 0; c < V; ++c)
#pragma unroll
      for (int v = 0; v < NV; ++v) R2b.W[c][v] = Wn[c][v];
    if (gN && k == y1) {
      if (a.bc[kN] == kDirichlet) {
        tb_dirichlet_row<A, V, NV>(a, kN, R2b.W);
      } else {
#pragma unroll
        for (int c = 0; c < V; ++c)
#pragma unroll
          for (int v = 0; v < NV; ++v) R2b.W[c][v] = R2a.W[c][v];
      }
    }
    if constexpr (REUSE) {
      A Q[V][4];
#pragma unroll
      for (int c = 0; c < V; ++c) Sys::prims4(R2b.W[c], P, Q[c]);
      if (k < y1) tb_lambda_q<Sys, A, V>(R2b.W, Q, X, a.nx, writer, lam1, bad1);
      tb_level_row<Sys, A, V, true>(P, R2a, R2b, Fs2, lx, ly, Wm, Q);
    } else {
      tb_level_row<Sys, A, V>(P, R2a, R2b, Fs2, lx, ly, Wm);
    }
    tb_store<Sys, A, V>(a, Wm, dst_lane, X, k - 1, writer);
    tb_lambda<Sys, A, V>(P, Wm, X, a.nx, writer, lam2, bad2);
    ++k;
  }
  cp_async_wait<0>();
}

// Close a two-step pass.  lmax(W^{n+2}) is gathered in the slot of step
// n + 1 (zero when step n starts) and moved to the slot of step n + 2; the
// slot of step n + 3 (that of step n) is cleared.  If some block found
// W^{n+1} failing the paper's check, nothing advances and kErrReplay is
// committed: every later launch then does nothing until the host clears it.
template <int NW>
static __device__ __forceinline__ void finish_tb(Ctrl *ctrl, const StepStart &st, const DtPolicy &pol,
                                                 double lam1, bool bad1, double lam2, bool bad2,
                                                 double (*s_lam)[2], int (*s_bad)[2]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lam1 = fmax(lam1, __shfl_xor_sync(0xffffffffu, lam1, o));
    lam2 = fmax(lam2, __shfl_xor_sync(0xffffffffu, lam2, o));
  }
  const int any1 = __any_sync(0xffffffffu, bad1), any2 = __any_sync(0xffffffffu, bad2);
  if (lane == 0) {
    s_lam[warp][0] = lam1;
    s_lam[warp][1] = lam2;
    s_bad[warp][0] = any1;
    s_bad[warp][1] = any2;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double l1 = 0.0, l2 = 0.0;
  int b1 = 0, b2 = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    l1 = fmax(l1, s_lam[w][0]);
    l2 = fmax(l2, s_lam[w][1]);
    b1 |= s_bad[w][0];
    b2 |= s_bad[w][1];
  }
  const long long n = st.step;
  if (st.run) {
    if (b1 || !(pol.fixed_dt * l1 <= pol.h)) {
      atomicOr(&ctrl->err_pending, kErrReplay);
    } else {
      if (b2) atomicMax(&ctrl->lam[(n + 1) % 3], 0x7ff8000000000000ull);
      else if (l2 > 0.0) atomicMax(&ctrl->lam[(n + 1) % 3], lam_bits(l2));
      if (b2) atomicOr(&ctrl->err_pending, kErrNonphysical);
    }
  }
  __threadfence();
  const unsigned prev = atomicAdd(&ctrl->blocks_done, 1u);
  if (prev == gridDim.x - 1) {
    __threadfence();
    ctrl->blocks_done = 0u;
    const unsigned e = atomicExch(&ctrl->err_pending, 0u) | st.err;
    if (st.run && (e & kErrReplay)) {
      // a void pass: back to how step n started (blocks without a failing
      // W^{n+1} cell may have gathered lmax(W^{n+2}) and flags of W^{n+2})
      ctrl->lam[(n + 1) % 3] = 0ull;
      ctrl->err_committed |= kErrReplay;
    } else {
      if (st.run) {
        // two single steps' additions, in order
        ctrl->t = (__ldcg(&ctrl->t) + st.dt) + st.dt;
        ctrl->dt_last = st.dt;
        ctrl->step = n + 2;
        ctrl->cur = st.cur ^ 1u;
        ctrl->lam[(n + 2) % 3] = __ldcg(&ctrl->lam[(n + 1) % 3]);
        ctrl->lam[n % 3] = 0ull;
      }
      if (e) ctrl->err_committed |= e;
    }
    __threadfence();
  }
}

// The two-step kernel (cp.async ring staging only, D < 0).  NP: built for
// grids with a transmissive or Dirichlet side (the ghost handling costs
// registers, so grids periodic on every side run the kernel without it).
template <class Sys, class A, int V, int TY, int NW, int MINB, int D, bool NP = false>
__global__ void __launch_bounds__(NW * 32, MINB)
fv_step_kernel_tb(const StepArgs<typename Ops<A>::S> a) {
  static_assert(D < 0 && V * Ops<A>::K >= 2, "two-step passes need the cp.async ring and two halo cells per lane");
  using S = typename Ops<A>::S;
  constexpr int NV = Sys::NV, N = V * Ops<A>::K, DA = -D;
  __shared__ double s_lam[NW][2];
  __shared__ int s_bad[NW][2];
  __shared__ StepStart s_st;
  extern __shared__ __align__(128) unsigned char s_dyn[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  LaneRing<S, N, NV, DA> lrg;
  lrg.buf = reinterpret_cast<S *>(s_dyn) + warp * (DA * NV * 32 * N) + lane * N;
  if (threadIdx.x == 0) s_st = read_step_start(a.pol, a.ctrl);
  __syncthreads();
  const StepStart st = s_st;
  typename Ops<A>::P lam1 = 0, lam2 = 0;
  unsigned bad1 = 0u, bad2 = 0u;
  if (st.run) {
    const S *src = st.cur ? a.buf1 : a.buf0;
    S *dst = st.cur ? a.buf0 : a.buf1;
    const SysParams<A> P = splat_params<A>(a.sp);
    const A lx = Ops<A>::splat((typename Ops<A>::P)(0.5 * (st.dt / a.dx)));
    const A ly = Ops<A>::splat((typename Ops<A>::P)(0.5 * (st.dt / a.dy)));
    const bool writer = lane >= 1 && lane <= 30;
    const int gw = blockIdx.x * NW + warp;
    const int GW = gridDim.x * NW;
    for (int task = gw; task < a.ntasks; task += GW) {
      const int sx_ = task % a.nstrips;
      const int cy = task / a.nstrips;
      const int X0 = sx_ * (30 * N);
      const int X = X0 + (lane - 1) * N;
      const int y0 = cy * TY;
      const int y1 = min(y0 + TY, a.ny);
      const bool xin = __all_sync(0xffffffffu, X >= 0 && X + N <= a.nx);
      march_tb<Sys, A, V, DA, NP>(a, P, src, dst, lrg, X, X0, lane, xin, y0, y1, writer, lx, ly, lam1, bad1,
                                  lam2, bad2);
    }
  }
  finish_tb<NW>(a.ctrl, st, a.pol, (double)lam1, bad1 != 0u, (double)lam2, bad2 != 0u, s_lam, s_bad);
}

}  // namespace fv
