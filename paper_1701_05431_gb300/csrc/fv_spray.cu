// fv_spray.cu -- split source step of the evaporating-spray moment system
// (arXiv:1701.05431, Sec. 2.2.2 Eq. (SourceTerm), Sec. 6.1 Eq. (Essadki),
// Sec. 6.2): W^{n+1} = W* + dt S(W*) per cell, where the evaporation terms
// need n(S = 0) and m_{-1/2} of the maximum-entropy size distribution
// n(S) = exp(-(lam0 + lam1 S^1/2 + lam2 S + lam3 S^3/2)) that matches the
// moments m0, m1/2, m1, m3/2.
//
// One thread per cell.  The multipliers are found by damped Newton on the
// convex dual, in FP64 in every storage precision (an FP32 Hessian of these
// Hankel-type moment matrices loses too many digits); the moments of a trial
// density are Gauss-Legendre sums in x = sqrt(S) whose nodes and
// pre-multiplied weights sit in shared memory.  The multipliers of each cell
// are kept between steps (warm start), those of the three last steps, and
// the solve starts from their quadratic extrapolation: the moments move
// smoothly, by O(dt) per step, so Newton usually needs two moment
// evaluations instead of eight.
// Only the first evaluation of a solve computes the Q exponentials
// e_q = exp(-p(x_q)) (p the multipliers' polynomial); they stay in shared
// memory, and after a Newton step d with sum |d_k| small (2^-10 with FP64
// storage, 2^-6 with FP32) the next evaluation multiplies them by
// exp(-p_d(x_q)), |p_d| within the same bound, from its Taylor polynomial of
// degree 5 or 7 (truncation < 1e-19 relative), which costs five or seven
// FMAs instead of an exponential per node.  The exponentials of each
// cell's last solve are kept between steps too (Q planes), so that even the
// first evaluation of a solve is such an update when the start is close to
// the last solution; every 32 steps they are computed afresh.
// After the update the kernel reduces lmax(W^{n+1}) and closes the step.
#include <cuda_runtime.h>

#include "fv_device.cuh"
#include "fv_internal.h"
#include "fv_step.cuh"

namespace fv {

constexpr int kSrcThreads = 128;
constexpr int kSrcWarps = kSrcThreads / 32;
constexpr int kMaxQ = 64;
constexpr int kNodeStride = 9;  // x, w 2x x^k (k = 0..6), 2w

template <class R> struct SourceArgs {
  R *buf0;
  R *buf1;
  Ctrl *ctrl;
  double *lamw;          // 12 planes of ny x pitch: multipliers of the last three solves
  double *ecache;        // Q planes of ny x pitch: exp(-p(x_q)) at the last solve's multipliers
  const double *nodes;   // Q x kNodeStride
  int nx, ny;
  long long pitch, plane;
  double dx, dy, xmin, ymin;
  DtPolicy pol;
  double K, theta, tol;
  int ug_mode, Q;
};

// Moments M_k = sum_q w_q 2 x_q x_q^k n(x_q^2) of the trial density, in
// three passes over the nodes so that no solve computes a moment it does not
// use: M_0..M_3 with the values e_q = n(x_q^2), which every evaluation needs
// (the residual); M_4..M_6 from the cached e_q, only before a Newton step
// (the Hessian); M_{-1} = sum_q 2 w_q n(x_q^2) (= m_{-1/2}) once, at the
// solution.  Each moment is the same FMA sequence in node order whichever
// pass computes it.  e: the thread's exponential cache (stride es).
static __device__ __forceinline__ void me_moments(const double *nd, int Q, const double (&lam)[4],
                                                  double (&M)[8], double *e, int es) {
#pragma unroll
  for (int k = 0; k < 4; ++k) M[k] = 0.0;
  for (int q = 0; q < Q; ++q) {
    const double *r = nd + q * kNodeStride;
    const double x = r[0];
    const double poly = fma(fma(fma(lam[3], x, lam[2]), x, lam[1]), x, lam[0]);
    const double eq = exp(-poly);
    e[q * es] = eq;
#pragma unroll
    for (int k = 0; k < 4; ++k) M[k] = fma(r[1 + k], eq, M[k]);
  }
}

// M_4..M_6 (the rest of the Hessian) from the cached e_q.
static __device__ __forceinline__ void me_moments_hessian(const double *nd, int Q, double (&M)[8], const double *e,
                                                          int es) {
#pragma unroll
  for (int k = 4; k < 7; ++k) M[k] = 0.0;
  for (int q = 0; q < Q; ++q) {
    const double *r = nd + q * kNodeStride;
    const double eq = e[q * es];
#pragma unroll
    for (int k = 4; k < 7; ++k) M[k] = fma(r[1 + k], eq, M[k]);
  }
}

// M_{-1} = m_{-1/2} from the cached e_q.
static __device__ __forceinline__ double me_moment_minus_half(const double *nd, int Q, const double *e, int es) {
  double s = 0.0;
  for (int q = 0; q < Q; ++q) s = fma(nd[q * kNodeStride + 8], e[q * es], s);
  return s;
}

// Incremental updates of the cached exponentials: exp(-t) from its Taylor
// polynomial of degree DEG (Horner form) for |t| <= Upd<R>::bound.  The pairs
// keep the truncation e^|t| |t|^(DEG+1) / (DEG+1)! below 1e-19, a thousandth
// of an ulp: degree 5 for |t| <= 2^-10, degree 7 for |t| <= 2^-6.  With FP64
// storage the multipliers move smoothly between steps and the short update
// serves nearly every evaluation (C5 FP64: 0.217 G cell-updates/s, against
// 0.205 with degree 7 and 0.191 with degree 10 for 2^-6); with FP32 storage
// the rounded moments move them by more, and the wider bound keeps more
// evaluations incremental (0.194, against 0.163 with degree 5).
template <class R> struct Upd {
  static constexpr int deg = 7;
  static constexpr double bound = 0x1p-6;
};
template <> struct Upd<double> {
  static constexpr int deg = 5;
  static constexpr double bound = 0x1p-10;
};

template <int DEG>
static __device__ __forceinline__ double exp_neg_small(double t) {
  constexpr double inv_fact[8] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0, 1.0 / 5040.0};
  static_assert(DEG >= 1 && DEG <= 7, "degree 1..7");
  const double u = -t;
  double p = inv_fact[DEG];
#pragma unroll
  for (int k = DEG - 1; k >= 0; --k) p = fma(p, u, inv_fact[k]);
  return p;
}

// M_0..M_3 after the multipliers moved by d, from the cached e_q of the
// previous multipliers: e_q <- e_q exp(-(d0 + d1 x + d2 x^2 + d3 x^3)).
// Requires |d0| + |d1| + |d2| + |d3| <= the bound of degree DEG.
template <int DEG>
static __device__ __forceinline__ void me_moments_step(const double *nd, int Q, const double (&d)[4],
                                                       double (&M)[8], double *e, int es) {
#pragma unroll
  for (int k = 0; k < 4; ++k) M[k] = 0.0;
  for (int q = 0; q < Q; ++q) {
    const double *r = nd + q * kNodeStride;
    const double x = r[0];
    const double pd = fma(fma(fma(d[3], x, d[2]), x, d[1]), x, d[0]);
    const double eq = e[q * es] * exp_neg_small<DEG>(pd);
    e[q * es] = eq;
#pragma unroll
    for (int k = 0; k < 4; ++k) M[k] = fma(r[1 + k], eq, M[k]);
  }
}

// Cholesky solve of the 4 x 4 SPD system H d = r; false if H is not SPD.
static __device__ __forceinline__ bool spd_solve4(const double (&M)[8], const double (&r)[4],
                                                  double (&d)[4]) {
  double L[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      double s = M[i + j];
#pragma unroll
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[i][i] = sqrt(s);
      } else {
        L[i][j] = s / L[j][j];
      }
    }
  }
  double y[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double s = r[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
    y[i] = s / L[i][i];
  }
#pragma unroll
  for (int i = 3; i >= 0; --i) {
    double s = y[i];
#pragma unroll
    for (int k = i + 1; k < 4; ++k) s -= L[k][i] * d[k];
    d[i] = s / L[i][i];
  }
  return true;
}

// Interior of the moment space of measures on [0,1] (positive Hankel
// determinants of the measure and of its products with x and 1 - x).
static __device__ __forceinline__ bool realizable(const double (&c)[4]) {
  return c[0] > 0.0 && c[1] > 0.0 && c[0] - c[1] > 0.0 && c[0] * c[2] - c[1] * c[1] > 0.0 &&
         c[1] - c[2] > 0.0 && c[1] * c[3] - c[2] * c[2] > 0.0 &&
         (c[0] - c[1]) * (c[2] - c[3]) - (c[1] - c[2]) * (c[1] - c[2]) > 0.0;
}

// Maximum-entropy reconstruction: returns false when Newton fails.  e is
// the thread's exponential cache (Q values, stride es).
template <class U>
static __device__ bool maxent(const double *nd, int Q, double tol, const double (&m)[4], double (&lam)[4],
                              double &n0, double &mmh, double *e, int es, int have0, const double (&d0)[4]) {
  double M[8];
  bool ok = false;
  // how the moments of the current multipliers are obtained: 0 from scratch,
  // 1 from the cache and the last full Newton step `d` (on entry: the cache
  // holds the exponentials at lam - d0 if have0 == 1), 2 already in M
  int have = have0;
  double d[4] = {d0[0], d0[1], d0[2], d0[3]};
  for (int it = 0; it < 100; ++it) {
    if (have == 0) me_moments(nd, Q, lam, M, e, es);
    else if (have == 1) me_moments_step<U::deg>(nd, Q, d, M, e, es);
    double r[4], worst = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      r[k] = M[k] - m[k];
      worst = fmax(worst, fabs(r[k]) / m[k]);
    }
    if (worst <= tol) {
      ok = true;
      break;
    }
    if (!(worst == worst)) return false;
    me_moments_hessian(nd, Q, M, e, es);
    if (!spd_solve4(M, r, d)) return false;
    if (worst >= 1e-3) {
      // far from the solution: halve the step until the dual
      // Phi = int n dS + sum lam_k m_k decreases (Armijo)
      const double phi0 = M[0] + lam[0] * m[0] + lam[1] * m[1] + lam[2] * m[2] + lam[3] * m[3];
      const double slope = -(r[0] * d[0] + r[1] * d[1] + r[2] * d[2] + r[3] * d[3]);
      double alpha = 1.0, trial[4];
      for (int ls = 0; ls < 60; ++ls) {
#pragma unroll
        for (int k = 0; k < 4; ++k) trial[k] = lam[k] + alpha * d[k];
        // the last trial evaluated is the one accepted: its moments and
        // exponentials are those of the new multipliers
        me_moments(nd, Q, trial, M, e, es);
        const double phi = M[0] + trial[0] * m[0] + trial[1] * m[1] + trial[2] * m[2] + trial[3] * m[3];
        if (phi <= phi0 + 1e-4 * alpha * slope + 4e-16 * fabs(phi0)) break;
        alpha *= 0.5;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) lam[k] = trial[k];
      have = 2;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) lam[k] += d[k];
      have = fabs(d[0]) + fabs(d[1]) + fabs(d[2]) + fabs(d[3]) <= U::bound ? 1 : 0;
    }
  }
  if (!ok) {
    // accept a result that stalled at round-off level
    me_moments(nd, Q, lam, M, e, es);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (!(fabs(M[k] - m[k]) <= 1e-10 * m[k])) return false;
  }
  n0 = exp(-lam[0]);
  mmh = me_moment_minus_half(nd, Q, e, es);
  return true;
}

template <class R>
__global__ void __launch_bounds__(kSrcThreads, 3)
fv_spray_source_kernel(const SourceArgs<R> a) {
  __shared__ double s_lam[kSrcWarps];
  __shared__ int s_bad[kSrcWarps];
  __shared__ StepStart s_st;
  __shared__ double s_nodes[kMaxQ * kNodeStride];
  extern __shared__ double s_exp[];  // Q x kSrcThreads exponentials, one column per thread
  for (int k = threadIdx.x; k < a.Q * kNodeStride; k += blockDim.x) s_nodes[k] = a.nodes[k];
  if (threadIdx.x == 0) s_st = read_step_start(a.pol, a.ctrl);
  __syncthreads();
  const StepStart st = s_st;
  double lmax = 0.0;
  bool bad = false;
  if (st.run) {
    R *__restrict__ W = st.cur ? a.buf0 : a.buf1;  // the transport output
    const double dt = st.dt;
    const long long ncell = (long long)a.nx * a.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ncell;
         k += (long long)gridDim.x * blockDim.x) {
      const int j = (int)(k / a.nx), i = (int)(k % a.nx);
      const long long o = (long long)j * a.pitch + i;
      double w[6];
#pragma unroll
      for (int v = 0; v < 6; ++v) w[v] = (double)W[v * a.plane + o];
      const double m[4] = {w[0], w[1], w[2], w[3]};
      bool cell_bad = !realizable(m);
      // start from the multipliers of the last solve, extrapolated in time
      // from the last two or three solves that exist (the moments move
      // smoothly from step to step: a quadratic extrapolation lands within
      // O(dt^3) of the solution, close enough for one Newton step)
      double lam[4], lam_prev[4], lam_prev2[4];
      const double warm0 = a.lamw[o], prev0 = a.lamw[4 * a.plane + o], prev20 = a.lamw[8 * a.plane + o];
      if (warm0 == warm0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          lam_prev[q] = a.lamw[q * a.plane + o];
          lam_prev2[q] = a.lamw[(4 + q) * a.plane + o];
          lam[q] = lam_prev[q];
        }
        if (prev0 == prev0 && prev20 == prev20) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            lam[q] = 3.0 * (lam_prev[q] - lam_prev2[q]) + a.lamw[(8 + q) * a.plane + o];
        } else if (prev0 == prev0) {
#pragma unroll
          for (int q = 0; q < 4; ++q) lam[q] = 2.0 * lam_prev[q] - lam_prev2[q];
        }
      } else {
        lam[0] = -log(m[0]);
        lam[1] = lam[2] = lam[3] = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) lam_prev[q] = lam_prev2[q] = __longlong_as_double(0x7ff8000000000000LL);
      }
      // the first evaluation updates the last solve's exponentials when the
      // start moved little from its multipliers (a full evaluation every 32
      // steps bounds the roundings the updates accumulate)
      int have0 = 0;
      double d0[4] = {0.0, 0.0, 0.0, 0.0};
      if (a.ecache && warm0 == warm0 && (st.step & 31) != 0) {
        double moved = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          d0[q] = lam[q] - lam_prev[q];
          moved += fabs(d0[q]);
        }
        if (moved <= Upd<R>::bound) {
          for (int q = 0; q < a.Q; ++q) s_exp[q * kSrcThreads + threadIdx.x] = a.ecache[q * a.plane + o];
          have0 = 1;
        }
      }
      double n0 = 0.0, mmh = 0.0;
      if (!cell_bad)
        cell_bad = !maxent<Upd<R>>(s_nodes, a.Q, a.tol, m, lam, n0, mmh, s_exp + threadIdx.x, kSrcThreads, have0, d0);
      if (!cell_bad && a.ecache)
        for (int q = 0; q < a.Q; ++q) a.ecache[q * a.plane + o] = s_exp[q * kSrcThreads + threadIdx.x];
      if (!cell_bad) {
        const double K = a.K;
        const double u = w[4] / w[2], v = w[5] / w[2];
        double S[6];
        S[0] = -K * n0;
        S[1] = -K / 2.0 * mmh;
        S[2] = -K * m[0];
        S[3] = -3.0 * K / 2.0 * m[1];
        S[4] = -K * m[0] * u;
        S[5] = -K * m[0] * v;
        if (a.theta > 0.0) {
          double ug = 0.0, vg = 0.0;
          if (a.ug_mode == 1) {
            const double x = a.xmin + (i + 0.5) * a.dx, y = a.ymin + (j + 0.5) * a.dy;
            ug = sinpi(2.0 * x) * cospi(2.0 * y);
            vg = -cospi(2.0 * x) * sinpi(2.0 * y);
          }
          S[4] += m[0] * (ug - u) / a.theta;
          S[5] += m[0] * (vg - v) / a.theta;
        }
        R wn[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) wn[q] = (R)(w[q] + dt * S[q]);
#pragma unroll
        for (int q = 0; q < 6; ++q) W[q * a.plane + o] = wn[q];
        const double c[4] = {(double)wn[0], (double)wn[1], (double)wn[2], (double)wn[3]};
        cell_bad = !realizable(c);
        SysParams<R> P{(R)0, (R)0};
        unsigned b;
        const R l = Spray::lambda<R>(wn, P, b);
        cell_bad |= b != 0u;
        lmax = fmax(lmax, (double)l);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a.lamw[(8 + q) * a.plane + o] = lam_prev2[q];
          a.lamw[(4 + q) * a.plane + o] = lam_prev[q];
          a.lamw[q * a.plane + o] = lam[q];
        }
      } else {
        a.lamw[o] = __longlong_as_double(0x7ff8000000000000LL);
        a.lamw[4 * a.plane + o] = __longlong_as_double(0x7ff8000000000000LL);
        a.lamw[8 * a.plane + o] = __longlong_as_double(0x7ff8000000000000LL);
      }
      bad |= cell_bad;
    }
  }
  finish_step<kSrcWarps>(a.ctrl, st, lmax, bad, s_lam, s_bad);
}

template <class R>
static SourceArgs<R> make_source_args(const SourceLaunch &L) {
  SourceArgs<R> a;
  a.buf0 = (R *)L.buf0;
  a.buf1 = (R *)L.buf1;
  a.ctrl = L.ctrl;
  a.lamw = L.lamw;
  a.ecache = L.ecache;
  a.nodes = L.nodes;
  a.nx = L.nx;
  a.ny = L.ny;
  a.pitch = L.pitch;
  a.plane = L.plane;
  a.dx = L.dx;
  a.dy = L.dy;
  a.xmin = L.xmin;
  a.ymin = L.ymin;
  a.pol = L.pol;
  a.K = L.K;
  a.theta = L.theta;
  a.tol = L.tol;
  a.ug_mode = L.ug_mode;
  a.Q = L.Q;
  return a;
}

static size_t source_smem(int Q) { return (size_t)Q * kSrcThreads * sizeof(double); }

int spray_source_grid(int prec, int Q, int sms) {
  int nb = 0;
  const void *k = prec == 0 ? (const void *)&fv_spray_source_kernel<double>
                            : (const void *)&fv_spray_source_kernel<float>;
  const size_t sm = source_smem(Q);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kSrcThreads, sm) != cudaSuccess || nb < 1)
    nb = 1;
  return nb * sms;
}

cudaError_t launch_spray_source(const SourceLaunch &L, int grid, cudaStream_t s) {
  long long need = ((long long)L.nx * L.ny + kSrcThreads - 1) / kSrcThreads;
  if (need < grid) grid = (int)need;
  if (grid < 1) grid = 1;
  const size_t sm = source_smem(L.Q);
  if (L.prec == 0) {
    SourceArgs<double> a = make_source_args<double>(L);
    fv_spray_source_kernel<double><<<grid, kSrcThreads, sm, s>>>(a);
  } else {
    SourceArgs<float> a = make_source_args<float>(L);
    fv_spray_source_kernel<float><<<grid, kSrcThreads, sm, s>>>(a);
  }
  return cudaGetLastError();
}

// Transport step kernels of the spray system (the source kernel closes the
// step, so they run with finalize = 0).
#define FV_VARIANT(R, PREC, V, TY, NW, MB, DESC)                                                  \
  out.push_back(Variant{kSpray, PREC, V, TY, NW, MB, 0, 0,                                         \
                        reinterpret_cast<const void *>(&fv_step_kernel<Spray, R, V, TY, NW, false, MB>), \
                        DESC})

void register_step_spray(std::vector<Variant> &out) {
  FV_VARIANT(double, 0, 1, 32, 4, 1, "spray f64 v1 ty32 w4");
  FV_VARIANT(float, 1, 1, 32, 4, 1, "spray f32 v1 ty32 w4");
  FV_VARIANT(float, 1, 2, 32, 4, 1, "spray f32 v2 ty32 w4");
}

}  // namespace fv
