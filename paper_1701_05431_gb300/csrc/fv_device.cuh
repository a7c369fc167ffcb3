// fv_device.cuh -- device-side building blocks of the fused finite-volume
// step (arXiv:1701.05431, Sec. 2.2): explicitly rounded arithmetic, the
// physical fluxes of the three systems, the Lax-Friedrichs face flux and the
// control block that carries lmax, dt and t between steps.
//
// Every floating-point operation of the flux, face and update arithmetic goes
// through Ops<R> (explicitly rounded intrinsics), so the compiler never
// contracts or reorders it: the x and y code paths then round identically,
// which makes the x<->y transposition of a state commute with the step bit for
// bit, and any tile shape gives the same bits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fv {

enum : int { kAdvection = 0, kEuler = 1, kSpray = 2 };
enum : int { kPeriodic = 0, kTransmissive = 1, kDirichlet = 2 };
enum : int { kE = 0, kN = 1, kW = 2, kS = 3 };
enum : unsigned { kErrCfl = 1u, kErrNonphysical = 2u, kErrZeroSpeed = 4u, kErrTimeout = 8u };

// Control block in device memory.  Step n reads lmax(W^n) from lam[n % 3]
// and accumulates lmax(W^{n+1}) into lam[(n+1) % 3]; the last block of step n
// clears lam[(n+2) % 3] for the step after.  Only that last block writes t,
// step and err_committed, after every block has read them, so all blocks of
// one kernel see the same values.
struct Ctrl {
  unsigned long long lam[3];  // bit patterns of non-negative doubles
  double t;
  double dt_last;
  double t_end;               // <= 0: no end time
  long long step;
  unsigned int blocks_done;
  unsigned int err_pending;   // raised by any block during a step
  unsigned int err_committed; // folded in by the step's last block
  unsigned int cur;           // buffer (0/1) that holds W^step (single-instance contexts)
};

template <class R> struct Ops;

// Every arithmetic type A used by the kernels provides:
//   S        storage type of one cell value (float, double or bfloat16)
//   P        type of parameters, boundary states and wave-speed maxima
//   K        cells packed in one A (1, or 2 for F2)
//   add/sub/mul/fma/rcp/sqrt/abs/max/neg   per component, explicitly rounded
//                         (max is only taken of non-negative values: speeds)
//   splat(s), pack(p), unpack(x, p)        conversions to and from storage
//   shfl_up/shfl_down                      warp shuffles of whole values
//   shift_in(prev, cur)   the values one cell to the west of `cur`, given the
//                         value `prev` that precedes `cur` (K = 1: prev;
//                         K = 2: (prev.y, cur.x))
//   shift_out(cur, next)  the values one cell to the east of `cur`
//   not_pos(x), not_fin(x)  bit k set when component k is not > 0 / not a
//                         finite value below 3e38
//   hmax(x, mask)         largest component among those selected by mask

template <> struct Ops<double> {
  using S = double;
  using P = double;
  static constexpr int K = 1;
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
  static __device__ __forceinline__ double rcp(double a) { return __drcp_rn(a); }
  static __device__ __forceinline__ double sqrt(double a) { return __dsqrt_rn(a); }
  static __device__ __forceinline__ double abs(double a) { return fabs(a); }
  // The FP64 pipe bounds the FP64 kernels, so comparisons run on the integer
  // pipe: non-negative doubles order like their bit patterns read as signed
  // 64-bit integers (a NaN operand with a clear sign bit is returned, where
  // fmax would drop it; a NaN speed flags the step either way).
  static __device__ __forceinline__ double max(double a, double b) {
    const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
    return __longlong_as_double(x > y ? x : y);
  }
  static __device__ __forceinline__ double neg(double a) { return -a; }
  static __device__ __forceinline__ double splat(double s) { return s; }
  static __device__ __forceinline__ double pack(const double *p) { return p[0]; }
  static __device__ __forceinline__ void unpack(double x, double *p) { p[0] = x; }
  static __device__ __forceinline__ double shfl_up(double x, int d) { return __shfl_up_sync(0xffffffffu, x, d); }
  static __device__ __forceinline__ double shfl_down(double x, int d) { return __shfl_down_sync(0xffffffffu, x, d); }
  static __device__ __forceinline__ double shift_in(double prev, double) { return prev; }
  static __device__ __forceinline__ double shift_out(double, double next) { return next; }
  // x > 0 exactly as the FP64 comparison decides it (false for NaN, -0 and
  // +0): the bit pattern minus one lies below that of +Inf
  static __device__ __forceinline__ unsigned not_pos(double x) {
    return ((unsigned long long)__double_as_longlong(x) - 1ull < 0x7ff0000000000000ull) ? 0u : 1u;
  }
  // |x| <= 3e38 on the magnitude bits (NaN and Inf lie above)
  static __device__ __forceinline__ unsigned not_fin(double x) {
    return ((unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull) <=
                   (unsigned long long)__double_as_longlong(3.0e38) ? 0u : 1u;
  }
  static __device__ __forceinline__ double hmax(double x, unsigned mask) { return (mask & 1u) ? x : 0.0; }
};

template <> struct Ops<float> {
  using S = float;
  using P = float;
  static constexpr int K = 1;
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  // FP32 reciprocal and square root use the single-instruction approximations
  // of the special-function unit (relative error of a few ulp); FP32 results
  // are held to a 1e-5 relative L1 bound against the FP64 oracle, far above it.
  static __device__ __forceinline__ float rcp(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
  }
  static __device__ __forceinline__ float sqrt(float a) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
  }
  static __device__ __forceinline__ float abs(float a) { return fabsf(a); }
  static __device__ __forceinline__ float max(float a, float b) { return fmaxf(a, b); }
  static __device__ __forceinline__ float neg(float a) { return -a; }
  static __device__ __forceinline__ float splat(float s) { return s; }
  static __device__ __forceinline__ float pack(const float *p) { return p[0]; }
  static __device__ __forceinline__ void unpack(float x, float *p) { p[0] = x; }
  static __device__ __forceinline__ float shfl_up(float x, int d) { return __shfl_up_sync(0xffffffffu, x, d); }
  static __device__ __forceinline__ float shfl_down(float x, int d) { return __shfl_down_sync(0xffffffffu, x, d); }
  static __device__ __forceinline__ float shift_in(float prev, float) { return prev; }
  static __device__ __forceinline__ float shift_out(float, float next) { return next; }
  static __device__ __forceinline__ unsigned not_pos(float x) { return (x > 0.0f) ? 0u : 1u; }
  static __device__ __forceinline__ unsigned not_fin(float x) { return (fabsf(x) <= 3.0e38f) ? 0u : 1u; }
  static __device__ __forceinline__ float hmax(float x, unsigned mask) { return (mask & 1u) ? x : 0.0f; }
};

// Two adjacent cells of one variable in one 64-bit register pair.  add, sub
// and fma use Blackwell's packed FP32x2 instructions (one instruction for
// both cells, each component rounded exactly like the scalar instruction), so
// a kernel on F2 gives the same bits as the scalar FP32 kernel.
struct __align__(8) F2 {
  float x, y;
};

template <> struct Ops<F2> {
  using S = float;
  using P = float;
  static constexpr int K = 2;
  static __device__ __forceinline__ unsigned long long b(F2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
  }
  static __device__ __forceinline__ F2 f(unsigned long long r) {
    F2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
  }
  static __device__ __forceinline__ F2 add(F2 a, F2 c) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(b(a)), "l"(b(c)));
    return f(d);
  }
  static __device__ __forceinline__ F2 sub(F2 a, F2 c) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(b(a)), "l"(b(c)));
    return f(d);
  }
  // Multiplies stay per component: with packed multiplies the fused step
  // rounded a few percent of its cells differently from the scalar kernel
  // (one ulp), although packed and scalar multiplies agree in isolation; with
  // per-component multiplies every F2 kernel gives the scalar kernel's bits.
  static __device__ __forceinline__ F2 mul(F2 a, F2 c) { return F2{__fmul_rn(a.x, c.x), __fmul_rn(a.y, c.y)}; }
  static __device__ __forceinline__ F2 fma(F2 a, F2 c, F2 e) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(b(a)), "l"(b(c)), "l"(b(e)));
    return f(d);
  }
  static __device__ __forceinline__ F2 rcp(F2 a) { return F2{Ops<float>::rcp(a.x), Ops<float>::rcp(a.y)}; }
  static __device__ __forceinline__ F2 sqrt(F2 a) { return F2{Ops<float>::sqrt(a.x), Ops<float>::sqrt(a.y)}; }
  static __device__ __forceinline__ F2 abs(F2 a) { return F2{fabsf(a.x), fabsf(a.y)}; }
  static __device__ __forceinline__ F2 max(F2 a, F2 c) { return F2{fmaxf(a.x, c.x), fmaxf(a.y, c.y)}; }
  static __device__ __forceinline__ F2 neg(F2 a) { return F2{-a.x, -a.y}; }
  static __device__ __forceinline__ F2 splat(float s) { return F2{s, s}; }
  static __device__ __forceinline__ F2 pack(const float *p) { return F2{p[0], p[1]}; }
  static __device__ __forceinline__ void unpack(F2 a, float *p) {
    p[0] = a.x;
    p[1] = a.y;
  }
  static __device__ __forceinline__ F2 shfl_up(F2 a, int d) {
    return F2{__shfl_up_sync(0xffffffffu, a.x, d), __shfl_up_sync(0xffffffffu, a.y, d)};
  }
  static __device__ __forceinline__ F2 shfl_down(F2 a, int d) {
    return F2{__shfl_down_sync(0xffffffffu, a.x, d), __shfl_down_sync(0xffffffffu, a.y, d)};
  }
  static __device__ __forceinline__ F2 shift_in(F2 prev, F2 cur) { return F2{prev.y, cur.x}; }
  static __device__ __forceinline__ F2 shift_out(F2 cur, F2 next) { return F2{cur.y, next.x}; }
  static __device__ __forceinline__ unsigned not_pos(F2 a) {
    return ((a.x > 0.0f) ? 0u : 1u) | ((a.y > 0.0f) ? 0u : 2u);
  }
  static __device__ __forceinline__ unsigned not_fin(F2 a) {
    return ((fabsf(a.x) <= 3.0e38f) ? 0u : 1u) | ((fabsf(a.y) <= 3.0e38f) ? 0u : 2u);
  }
  static __device__ __forceinline__ float hmax(F2 a, unsigned mask) {
    return fmaxf((mask & 1u) ? a.x : 0.0f, (mask & 2u) ? a.y : 0.0f);
  }
};

// One cell held in FP32 for arithmetic and stored as bfloat16 (16 bytes per
// Euler cell-update instead of 32): loads widen bfloat16 to FP32 exactly,
// stores round to nearest even.  All arithmetic is the FP32 arithmetic of
// Ops<float>.
struct BF {
  float v;
};

template <> struct Ops<BF> {
  using S = __nv_bfloat16;
  using P = float;
  static constexpr int K = 1;
  using F = Ops<float>;
  static __device__ __forceinline__ BF add(BF a, BF b) { return BF{F::add(a.v, b.v)}; }
  static __device__ __forceinline__ BF sub(BF a, BF b) { return BF{F::sub(a.v, b.v)}; }
  static __device__ __forceinline__ BF mul(BF a, BF b) { return BF{F::mul(a.v, b.v)}; }
  static __device__ __forceinline__ BF fma(BF a, BF b, BF c) { return BF{F::fma(a.v, b.v, c.v)}; }
  static __device__ __forceinline__ BF rcp(BF a) { return BF{F::rcp(a.v)}; }
  static __device__ __forceinline__ BF sqrt(BF a) { return BF{F::sqrt(a.v)}; }
  static __device__ __forceinline__ BF abs(BF a) { return BF{fabsf(a.v)}; }
  static __device__ __forceinline__ BF max(BF a, BF b) { return BF{fmaxf(a.v, b.v)}; }
  static __device__ __forceinline__ BF neg(BF a) { return BF{-a.v}; }
  static __device__ __forceinline__ BF splat(float s) { return BF{s}; }
  static __device__ __forceinline__ BF pack(const __nv_bfloat16 *p) { return BF{__bfloat162float(p[0])}; }
  static __device__ __forceinline__ void unpack(BF a, __nv_bfloat16 *p) { p[0] = __float2bfloat16_rn(a.v); }
  static __device__ __forceinline__ BF shfl_up(BF a, int d) { return BF{__shfl_up_sync(0xffffffffu, a.v, d)}; }
  static __device__ __forceinline__ BF shfl_down(BF a, int d) { return BF{__shfl_down_sync(0xffffffffu, a.v, d)}; }
  static __device__ __forceinline__ BF shift_in(BF prev, BF) { return prev; }
  static __device__ __forceinline__ BF shift_out(BF, BF next) { return next; }
  static __device__ __forceinline__ unsigned not_pos(BF a) { return (a.v > 0.0f) ? 0u : 1u; }
  static __device__ __forceinline__ unsigned not_fin(BF a) { return (fabsf(a.v) <= 3.0e38f) ? 0u : 1u; }
  static __device__ __forceinline__ float hmax(BF a, unsigned mask) { return (mask & 1u) ? a.v : 0.0f; }
};

// Widening of a stored value to double (totals, conversions).
static __device__ __forceinline__ double to_double(double x) { return x; }
static __device__ __forceinline__ double to_double(float x) { return (double)x; }
static __device__ __forceinline__ double to_double(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

// Parameter type of a storage type.
template <class S> struct ParamOf { using T = S; };
template <> struct ParamOf<__nv_bfloat16> { using T = float; };

// Parameters of the system, in the arithmetic precision.
template <class R> struct SysParams {
  R p0, p1;   // advection: a_x, a_y | Euler: gamma, gamma - 1 | spray: unused
};

template <class A>
static __device__ __forceinline__ SysParams<A> splat_params(const SysParams<typename Ops<A>::P> &p) {
  return SysParams<A>{Ops<A>::splat(p.p0), Ops<A>::splat(p.p1)};
}

// ---------------------------------------------------------------- systems
// Each system provides, for one cell W:
//   fluxes(): F(W).(1,0), the largest |eigenvalue| along x, F(W).(0,1) and
//             the largest |eigenvalue| along y;
//   lambda(): max of the two (the cell's term of Eq. (CFL_cond)) and, per
//             packed cell, a bit set when the state is not admissible.

// Scalar advection, F = a u: eigenvalue a.n.
struct Advection {
  static constexpr int NV = 1;
  static constexpr int NU = NV;  // variables the scheme updates (the rest are carried)
  template <class R>
  static __device__ __forceinline__ void fluxes(const R (&W)[NV], const SysParams<R> &P,
                                                R (&Fx)[NV], R &sx, R (&Fy)[NV], R &sy) {
    using O = Ops<R>;
    Fx[0] = O::mul(P.p0, W[0]);
    Fy[0] = O::mul(P.p1, W[0]);
    sx = O::abs(P.p0);
    sy = O::abs(P.p1);
  }
  template <class R>
  static __device__ __forceinline__ R lambda(const R (&W)[NV], const SysParams<R> &P, unsigned &bad) {
    using O = Ops<R>;
    R l = O::max(O::abs(P.p0), O::abs(P.p1));
    bad = O::not_fin(W[0]);
    return l;
  }
};

// Euler, Eq. (Euler): W = (rho, rho u, rho v, rho E),
// p = (gamma - 1)(rho E - (rho u u + rho v v)/2), c^2 = gamma p / rho,
// F.x = (rho u, rho u u + p, rho u v, u (rho E + p)), eigenvalues u -+ c, u.
struct Euler {
  static constexpr int NV = 4;
  static constexpr int NU = NV;
  template <class R>
  static __device__ __forceinline__ void prims(const R (&W)[NV], const SysParams<R> &P, R &u,
                                               R &v, R &p, R &c) {
    using O = Ops<R>;
    R inv = O::rcp(W[0]);
    u = O::mul(W[1], inv);
    v = O::mul(W[2], inv);
    // twice the kinetic energy: a plain sum of two rounded products keeps
    // x <-> y symmetry; p = (gamma - 1) rho E - ((gamma - 1)/2) (that sum),
    // the second product fused
    const R s = O::add(O::mul(W[1], u), O::mul(W[2], v));
    p = O::fma(O::neg(O::mul(O::splat(0.5), P.p1)), s, O::mul(P.p1, W[3]));
    c = O::sqrt(O::mul(O::mul(P.p0, p), inv));
  }
  // The fluxes and speeds of a cell from its primitives q = (u, v, p, c).
  template <class R>
  static __device__ __forceinline__ void fluxes_from(const R (&W)[NV], const R (&q)[4], R (&Fx)[NV], R &sx,
                                                     R (&Fy)[NV], R &sy) {
    using O = Ops<R>;
    const R u = q[0], v = q[1], p = q[2], c = q[3];
    R Ep = O::add(W[3], p);
    Fx[0] = W[1];
    Fx[1] = O::fma(W[1], u, p);
    Fx[2] = O::mul(W[1], v);
    Fx[3] = O::mul(u, Ep);
    Fy[0] = W[2];
    Fy[1] = O::mul(W[2], u);
    Fy[2] = O::fma(W[2], v, p);
    Fy[3] = O::mul(v, Ep);
    sx = O::add(O::abs(u), c);
    sy = O::add(O::abs(v), c);
  }
  // The wave speed and admissibility of a cell from its primitives.
  template <class R>
  static __device__ __forceinline__ R lambda_from(const R (&W)[NV], const R (&q)[4], unsigned &bad) {
    using O = Ops<R>;
    R l = O::add(O::max(O::abs(q[0]), O::abs(q[1])), q[3]);
    bad = O::not_pos(W[0]) | O::not_pos(q[2]) | O::not_fin(l);
    return l;
  }
  template <class R>
  static __device__ __forceinline__ void prims4(const R (&W)[NV], const SysParams<R> &P, R (&q)[4]) {
    prims(W, P, q[0], q[1], q[2], q[3]);
  }
  template <class R>
  static __device__ __forceinline__ void fluxes(const R (&W)[NV], const SysParams<R> &P,
                                                R (&Fx)[NV], R &sx, R (&Fy)[NV], R &sy) {
    R q[4];
    prims4(W, P, q);
    fluxes_from(W, q, Fx, sx, Fy, sy);
  }
  template <class R>
  static __device__ __forceinline__ R lambda(const R (&W)[NV], const SysParams<R> &P, unsigned &bad) {
    R q[4];
    prims4(W, P, q);
    return lambda_from(W, q, bad);
  }
};

// Euler with carried primitives (FP64 kernels): each cell stores, after its
// four conserved variables, the u, v, p, c that Euler::prims gives for them
// (planes 4..7).  The step that produces W^{n+1} computes those anyway for
// the wave speed of Eq. (CFL_cond) and stores them; the next step's fluxes
// read them instead of recomputing them, which saves one reciprocal, one
// square root and ten operations per cell on the FP64 pipe.  The fluxes,
// speeds and admissibility are those of Euler bit for bit.
struct EulerPC {
  static constexpr int NV = 8;  // planes loaded and stored
  static constexpr int NU = 4;  // variables the scheme updates
  template <class R>
  static __device__ __forceinline__ void complete(R (&W)[NV], const SysParams<R> &P) {
    R Wc[4] = {W[0], W[1], W[2], W[3]};
    Euler::prims(Wc, P, W[4], W[5], W[6], W[7]);
  }
  template <class R>
  static __device__ __forceinline__ void fluxes(const R (&W)[NV], const SysParams<R> &P,
                                                R (&Fx)[NV], R &sx, R (&Fy)[NV], R &sy) {
    using O = Ops<R>;
    const R u = W[4], v = W[5], p = W[6], c = W[7];
    R Ep = O::add(W[3], p);
    Fx[0] = W[1];
    Fx[1] = O::fma(W[1], u, p);
    Fx[2] = O::mul(W[1], v);
    Fx[3] = O::mul(u, Ep);
    Fy[0] = W[2];
    Fy[1] = O::mul(W[2], u);
    Fy[2] = O::fma(W[2], v, p);
    Fy[3] = O::mul(v, Ep);
    sx = O::add(O::abs(u), c);
    sy = O::add(O::abs(v), c);
  }
  template <class R>
  static __device__ __forceinline__ R lambda(const R (&W)[NV], const SysParams<R> &P, unsigned &bad) {
    using O = Ops<R>;
    const R u = W[4], v = W[5], p = W[6], c = W[7];
    R l = O::add(O::max(O::abs(u), O::abs(v)), c);
    bad = O::not_pos(W[0]) | O::not_pos(p) | O::not_fin(l);
    return l;
  }
};

// Spray moments, Eq. (Essadki): W = (m0, m1/2, m1, m3/2, m1 u, m1 v), all
// transported by u = (m1 u)/m1; every eigenvalue is u.n.
struct Spray {
  static constexpr int NV = 6;
  static constexpr int NU = NV;
  template <class R>
  static __device__ __forceinline__ void fluxes(const R (&W)[NV], const SysParams<R> &P,
                                                R (&Fx)[NV], R &sx, R (&Fy)[NV], R &sy) {
    using O = Ops<R>;
    R inv = O::rcp(W[2]);
    R u = O::mul(W[4], inv);
    R v = O::mul(W[5], inv);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      Fx[k] = O::mul(W[k], u);
      Fy[k] = O::mul(W[k], v);
    }
    sx = O::abs(u);
    sy = O::abs(v);
  }
  template <class R>
  static __device__ __forceinline__ R lambda(const R (&W)[NV], const SysParams<R> &P, unsigned &bad) {
    static_assert(Ops<R>::K == 1, "spray cells are not packed");
    using O = Ops<R>;
    R inv = O::rcp(W[2]);
    R u = O::mul(W[4], inv);
    R v = O::mul(W[5], inv);
    R l = O::max(O::abs(u), O::abs(v));
    // moments (m0, m1/2, m1, m3/2) strictly inside the moment space of
    // measures on [0,1]: positive Hankel determinants (checked in FP64)
    const double c0 = W[0], c1 = W[1], c2 = W[2], c3 = W[3];
    const bool inside = c0 > 0.0 && c1 > 0.0 && c0 - c1 > 0.0 && c0 * c2 - c1 * c1 > 0.0 &&
                        c1 - c2 > 0.0 && c1 * c3 - c2 * c2 > 0.0 &&
                        (c0 - c1) * (c2 - c3) - (c1 - c2) * (c1 - c2) > 0.0;
    bad = (!inside || !(l <= (R)3.0e38)) ? 1u : 0u;
    return l;
  }
};

// Lax-Friedrichs face flux of Sec. 2.2.1 for one variable, carried doubled:
// 2 F~ = (F_L + F_R) - sigma (W_R - W_L).  Scaling by 2 is exact in binary
// floating point, so this is bit for bit twice the flux written with the
// halves (F~ = (F_L + F_R)/2 - (sigma/2)(W_R - W_L)); the kernels fold the
// remaining 1/2 into dt/dx and dt/dy, which saves two multiplies per face.
template <class R>
static __device__ __forceinline__ R lf_face2(R WL, R FL, R WR, R FR, R sigma) {
  using O = Ops<R>;
  return O::fma(O::neg(sigma), O::sub(WR, WL), O::add(FL, FR));
}

// Residual and forward-Euler update of Eq. (VF_scheme) for one variable:
// W + ( -(lx (Fe - Fw)) - (ly (Fn - Fs)) ), called with doubled face fluxes
// and lx = dt/(2 dx), ly = dt/(2 dy) (same bits as the undoubled form).
template <class R>
static __device__ __forceinline__ R fv_update(R W, R dX, R dY, R lx, R ly) {
  using O = Ops<R>;
  return O::add(W, O::sub(O::neg(O::mul(lx, dX)), O::mul(ly, dY)));
}

// The same update on square cells (dx = dy, so lx = ly):
// W - lx ((Fe - Fw) + (Fn - Fs)) with one FMA, symmetric in x and y like
// the general form.  The FP64 Euler and spray kernels use it (their FP64
// pipe is the bound and it saves two of its operations per variable);
// rounding aside it is the same expression.
template <class R>
static __device__ __forceinline__ R fv_update_sq(R W, R dX, R dY, R l) {
  using O = Ops<R>;
  return O::fma(O::neg(l), O::add(dX, dY), W);
}

static __device__ __forceinline__ unsigned long long lam_bits(double l) {
  return (unsigned long long)__double_as_longlong(l);
}
static __device__ __forceinline__ double lam_value(unsigned long long b) {
  return __longlong_as_double((long long)b);
}

// Time step of step n from lmax(W^n), Eq. (CFL_cond):
//   adaptive: dt = cfl * min(dx, dy) / lmax (capped for the spray drag);
//   fixed:    dt = fixed_dt after checking fixed_dt * lmax <= min(dx, dy);
//   both clipped to land on t_end.
// Returns false when the step must not run; *err then holds the reason
// (0 when the run simply reached t_end or an earlier error is pending).
struct DtPolicy {
  double h;         // min(dx, dy)
  double cfl;
  double fixed_dt;
  double dt_cap;    // +inf unless the system caps dt
};

static __device__ __forceinline__ bool choose_dt(const DtPolicy &pol, const Ctrl &c, double lam,
                                                 double *dt, unsigned *err) {
  *err = 0u;
  if (c.err_committed != 0u) return false;
  if (c.t_end > 0.0 && c.t >= c.t_end) return false;
  if (!(lam <= 1.0e300)) { *err = kErrNonphysical; return false; }
  double d;
  if (pol.fixed_dt > 0.0) {
    if (pol.fixed_dt * lam > pol.h) { *err = kErrCfl; return false; }
    d = pol.fixed_dt;
  } else {
    d = lam > 0.0 ? pol.cfl * pol.h / lam : 1.0e308;
    if (pol.dt_cap < d) d = pol.dt_cap;
    if (!(d < 1.0e300)) { *err = kErrZeroSpeed; return false; }
  }
  if (c.t_end > 0.0 && c.t + d > c.t_end) d = c.t_end - c.t;
  *dt = d;
  return true;
}

// Every step kernel starts by reading the control block once (thread 0) and
// deciding whether the step runs and with which dt.
struct StepStart {
  double dt;
  long long step;
  unsigned err;
  int run;
  unsigned cur;  // buffer holding W^step
};

static __device__ __forceinline__ StepStart read_step_start(const DtPolicy &pol, Ctrl *ctrl) {
  Ctrl c;
  c.step = __ldcg(&ctrl->step);
  c.t = __ldcg(&ctrl->t);
  c.t_end = __ldcg(&ctrl->t_end);
  c.err_committed = __ldcg(&ctrl->err_committed);
  const double lam = lam_value(__ldcg(&ctrl->lam[c.step % 3]));
  StepStart s;
  s.dt = 0.0;
  s.step = c.step;
  s.cur = __ldcg(&ctrl->cur);
  s.run = choose_dt(pol, c, lam, &s.dt, &s.err) ? 1 : 0;
  return s;
}

// Close a step: reduce lmax(W^{n+1}) and the admissibility flag over the
// block (warp shuffles, then one shared slot per warp), fold them into the
// control block with one atomic each, and let the last block to finish
// advance t and n, clear the lmax slot of step n + 2 and commit the error
// flags.  Must be reached by every thread of every block.
template <int NW>
static __device__ __forceinline__ void finish_step(Ctrl *ctrl, const StepStart &st, double lam,
                                                   bool bad, double *s_lam, int *s_bad) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  const int anybad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    s_lam[warp] = lam;
    s_bad[warp] = anybad;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double bl = 0.0;
  int bb = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    bl = fmax(bl, s_lam[w]);
    bb |= s_bad[w];
  }
  const long long n = st.step;
  if (st.run) {
    // an inadmissible state poisons the slot with a NaN so the next dt fails too
    if (bb) atomicMax(&ctrl->lam[(n + 1) % 3], 0x7ff8000000000000ull);
    else if (bl > 0.0) atomicMax(&ctrl->lam[(n + 1) % 3], lam_bits(bl));
    if (bb) atomicOr(&ctrl->err_pending, kErrNonphysical);
  }
  __threadfence();
  const unsigned prev = atomicAdd(&ctrl->blocks_done, 1u);
  if (prev == gridDim.x - 1) {
    __threadfence();
    ctrl->blocks_done = 0u;
    const unsigned e = atomicExch(&ctrl->err_pending, 0u) | st.err;
    if (st.run) {
      ctrl->t = __ldcg(&ctrl->t) + st.dt;
      ctrl->dt_last = st.dt;
      ctrl->step = n + 1;
      ctrl->cur = st.cur ^ 1u;
      ctrl->lam[(n + 2) % 3] = 0ull;
    }
    if (e) ctrl->err_committed |= e;
    __threadfence();
  }
}

}  // namespace fv
