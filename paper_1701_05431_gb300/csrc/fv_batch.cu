// fv_batch.cu -- many independent finite-volume problems (instances of any
// sizes, each with its own dt) advanced by ONE persistent kernel per run of
// n steps, captured in a CUDA graph.  Each step of each instance is the fused
// step of fv_step.cuh (same arithmetic, so a batched instance gives the same
// bits as the instance run alone).
//
// Work list.  A run of n steps has n * T tasks (T = warp tasks of all
// instances for one step), numbered step-major then instance-major.  Warps
// take tickets from one global counter in increasing order.  Before working
// on step s of instance i a warp waits until instance i has released step s,
// i.e. all its tasks of step s - 1 are done: their writes are visible, every
// read of the buffer step s is about to overwrite is over, and lmax(W^s),
// hence dt_s, is complete.  The warp that completes the last task of a step
// advances the instance's t and step, clears the lmax slot two steps ahead
// and releases the next step.  Tickets are monotone, so a waiting warp only
// waits on tickets already held by running warps: no deadlock, whatever the
// number of resident blocks.  Every wait is bounded (%globaltimer); on
// timeout the kernel raises an abort flag, every warp leaves at its next
// ticket, and the host reports FV_ERR_TIMEOUT.
//
// Dataflow mode (the paper's fixed dt, Sec. 2.2.1, with its task graph of
// Sec. 3.2 on the device).  With a constant dt no step waits for a global
// lmax: a task of step s only needs its own and its (up to eight) neighbour
// tasks' step s - 1 to be done, the neighbours being the tasks whose cells
// its halo reads (across a periodic boundary too).  Every task publishes
// the number of steps it has completed in this run (release store) and lanes
// 0..8 of a warp wait on one dependency each (acquire, bounded).  Each task
// checks the paper's condition dt lmax <= min(dx, dy) on the cells it
// produced; a violation (or an inadmissible state) flags its instance, whose
// later tasks then do no work.  Tasks far from the violation may already have
// advanced past it, so the run keeps a copy of every instance's state at its
// start: the host puts flagged instances back and replays them with the
// step-gated kernel, which stops exactly at the failing step, as without
// dataflow.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/fv.h"
#include "fv_internal.h"
#include "fv_tune.h"
#include "fv_step.cuh"

namespace fv {

struct RunCounters {
  unsigned done;      // tasks of this instance completed during this run
  unsigned released;  // steps of this instance open during this run (step s needs released >= s)
};

// The dt decision of one step of one instance, made once by the warp that
// closes the previous step (lmax(W^n) is complete then), so that the warps
// of step n read it instead of each repeating the FP64 divisions.
struct StepPlan {
  long long step;  // the step this plan is for (-1: none)
  double dt;
  double hx, hy;   // dt / (2 dx), dt / (2 dy): the update's factors (doubled face fluxes)
  int run;
  unsigned err;
};

// What one run needs to know per instance (written by the host before it).
struct RunInfo {
  long long base;            // step count at the start of the run
  int active;                // 0: the instance does not advance in this run
  int pad_;
  double dt, hx, hy;         // dataflow: the fixed dt and dt / (2 dx), dt / (2 dy)
};

template <class R> struct BatchArgs {
  const StepArgs<R> *inst;   // per-instance geometry, buffers, dt policy, BCs
  Ctrl *ictrl;               // per-instance lmax slots, t, step, error flags
  StepPlan *plan;            // per-instance dt decision of its next step
  RunCounters *rc;           // per-instance counters of this run
  const int *task_inst;      // T entries: instance of each task of a step
  const int *task_base;      // first task of each instance within a step
  unsigned *ticket;          // global ticket counter of this run
  unsigned *abort;           // set on timeout; every warp leaves
  int nsteps, T;
  long long timeout_ns;
  int skip_release;          // instance whose steps are never released (-1: none)
  int dataflow;              // 1: neighbour dependencies, fixed dt (see the file header)
  const RunInfo *info;       // per instance
  unsigned *tdone;           // T entries: steps of this run each task has completed (dataflow)
  unsigned *flagged;         // per instance: violation seen in this run (dataflow)
};

static __device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

static __device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

static __device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait (one lane) until *flag >= target; false on timeout or abort.
static __device__ bool wait_at_least(const unsigned *flag, unsigned target, long long timeout_ns,
                                     unsigned *abort) {
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    if (ld_acquire(flag) >= target) return true;
    if (ld_acquire(abort) != 0u) return false;
    if (it > 4) __nanosleep(128);
    // time limit, plus an iteration cap in case the timer stalls
    if ((long long)(global_ns() - t0) > timeout_ns || it > (1u << 26)) {
      atomicOr(abort, kErrTimeout);
      return false;
    }
  }
}

// D = 0: register prefetch with L2 loads (ld.cg).  D < 0: rows staged through
// a per-lane cp.async ring of -D slots (dynamic shared memory), as in the
// single-instance kernel.  Both may read data written earlier in the same
// launch: a warp starts a task only after lane 0's acquire load has seen the
// step released (the release follows every write of the previous step) and
// __syncwarp has ordered that acquire before the other lanes' loads, so the
// memory model guarantees that no load, cached or asynchronous, sees stale
// values.
template <class Sys, class R, int V, int TY, int NW, int MINB, int D = 0>
__global__ void __launch_bounds__(NW * 32, MINB)
fv_batch_kernel(const BatchArgs<R> b) {
  __shared__ StepArgs<R> s_args[NW];
  extern __shared__ __align__(128) unsigned char s_dyn[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  StepArgs<R> &a = s_args[warp];
  constexpr int DA = D < 0 ? -D : 2;
  LaneRing<R, V, Sys::NV, DA> lrg;
  if (D < 0) lrg.buf = reinterpret_cast<R *>(s_dyn) + warp * (DA * Sys::NV * 32 * V) + lane * V;
  const unsigned total = (unsigned)b.nsteps * (unsigned)b.T;
  const bool writer = lane >= 1 && lane <= 30;
  int cur_inst = -1;
  for (;;) {
    unsigned t = 0;
    if (lane == 0) t = ld_acquire(b.abort) ? total : atomicAdd(b.ticket, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= total) break;
    const unsigned s = t / (unsigned)b.T;
    const int r = (int)(t - s * (unsigned)b.T);
    const int i = b.task_inst[r];
    const int lt = r - b.task_base[i];
    if (!__ldg(&b.info[i].active)) continue;  // warp-uniform
    if (i != cur_inst) {
      const unsigned *src = reinterpret_cast<const unsigned *>(&b.inst[i]);
      unsigned *dstw = reinterpret_cast<unsigned *>(&a);
      for (int k = lane; k < (int)(sizeof(StepArgs<R>) / 4); k += 32) dstw[k] = __ldg(src + k);
      __syncwarp();
      cur_inst = i;
    }
    int ok = 1;
    if (b.dataflow) {
      // lanes 0..8 wait on the task itself and its neighbours (dx, dy in -1..1)
      if (lane < 9 && s > 0u) {
        int nsx = lt % a.nstrips + lane % 3 - 1, ncy = lt / a.nstrips + lane / 3 - 1;
        bool dep = true;
        if (nsx < 0) { if (a.bc[kW] == kPeriodic) nsx += a.nstrips; else dep = false; }
        if (nsx >= a.nstrips) { if (a.bc[kE] == kPeriodic) nsx -= a.nstrips; else dep = false; }
        if (ncy < 0) { if (a.bc[kS] == kPeriodic) ncy += a.nchunks; else dep = false; }
        if (ncy >= a.nchunks) { if (a.bc[kN] == kPeriodic) ncy -= a.nchunks; else dep = false; }
        if (dep)
          ok = wait_at_least(&b.tdone[b.task_base[i] + ncy * a.nstrips + nsx], s, b.timeout_ns, b.abort) ? 1 : 0;
      }
      ok = __all_sync(0xffffffffu, ok != 0) ? 1 : 0;
    } else {
      if (lane == 0) ok = wait_at_least(&b.rc[i].released, s, b.timeout_ns, b.abort) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
    }
    __syncwarp();
    if (!ok) break;
    Ctrl *ic = &b.ictrl[i];
    // dt of this step of instance i (same rule as the single-instance kernel):
    // from the plan the previous step's closing warp left, else computed here
    // (the first step of a run)
    const long long n = b.dataflow ? __ldg(&b.info[i].base) + (long long)s : __ldcg(&ic->step);
    double dt = 0.0, hx = 0.0, hy = 0.0;
    unsigned err = 0u;
    bool run;
    if (b.dataflow) {
      run = __ldcg(&b.flagged[i]) == 0u;
      dt = __ldg(&b.info[i].dt);
      hx = __ldg(&b.info[i].hx);
      hy = __ldg(&b.info[i].hy);
    } else if (__ldcg(&b.plan[i].step) == n) {
      run = __ldcg(&b.plan[i].run) != 0;
      err = __ldcg(&b.plan[i].err);
      dt = __ldcg(&b.plan[i].dt);
      hx = __ldcg(&b.plan[i].hx);
      hy = __ldcg(&b.plan[i].hy);
    } else {
      Ctrl c;
      c.step = n;
      c.t = __ldcg(&ic->t);
      c.t_end = 0.0;
      c.err_committed = __ldcg(&ic->err_committed);
      run = choose_dt(a.pol, c, lam_value(__ldcg(&ic->lam[n % 3])), &dt, &err);
      hx = 0.5 * (dt / a.dx);
      hy = 0.5 * (dt / a.dy);
    }
    R lam_loc = (R)0;
    unsigned bad = 0u;
    if (run) {
      // the instance's geometry in registers (see MarchGeo)
      MarchGeo<R> g;
      g.ctrl = a.ctrl;
      g.nx = a.nx;
      g.ny = a.ny;
      g.pitch = a.pitch;
      g.plane = a.plane;
#pragma unroll
      for (int q = 0; q < 4; ++q) g.bc[q] = a.bc[q];
      g.bc_state = a.bc_state;
      const R *src = (n & 1) ? a.buf1 : a.buf0;
      R *dst = (n & 1) ? a.buf0 : a.buf1;
      const SysParams<R> P = a.sp;
      // half steps: the face fluxes are carried doubled (see lf_face2)
      const R lx = (R)hx, ly = (R)hy;
      const int strip = lt % a.nstrips, chunk = lt / a.nstrips;
      const int X = strip * (30 * V) + (lane - 1) * V;
      const int y0 = chunk * TY, y1 = min(y0 + TY, g.ny);
      const bool xin = __all_sync(0xffffffffu, X >= 0 && X + V <= g.nx);
      if (D < 0) march_async<Sys, R, V, DA, true>(g, P, src, dst, lrg, X, xin, y0, y1, writer, lx, ly, lam_loc, bad);
      else if (xin) march<Sys, R, V, true, true, true>(g, P, src, dst, X, y0, y1, writer, lx, ly, lam_loc, bad);
      else march<Sys, R, V, false, true, true>(g, P, src, dst, X, y0, y1, writer, lx, ly, lam_loc, bad);
    }
    // the maximum is exact in any precision: reduce in R, widen once
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lam_loc = fmax(lam_loc, __shfl_xor_sync(0xffffffffu, lam_loc, o));
    const double l = (double)lam_loc;
    const int anybad = __any_sync(0xffffffffu, bad != 0u);
    __syncwarp();  // every lane's stores of this task precede lane 0's fence below
    if (b.dataflow) {
      if (lane == 0) {
        if (run) {
          // the paper's check on the produced cells: dt lmax <= min(dx, dy)
          if (anybad || !(dt * l <= a.pol.h)) atomicExch(&b.flagged[i], 1u);
          if (anybad) atomicOr(&ic->err_pending, kErrNonphysical);
          // lmax of the final state, for the steps after this run
          if (s + 1u == (unsigned)b.nsteps && !anybad && l > 0.0) atomicMax(&ic->lam[(n + 1) % 3], lam_bits(l));
        }
        __threadfence();
        if (i != b.skip_release) st_release(&b.tdone[r], s + 1u);
      }
      __syncwarp();
      continue;
    }
    if (lane == 0) {
      if (run) {
        if (anybad) atomicMax(&ic->lam[(n + 1) % 3], 0x7ff8000000000000ull);
        else if (l > 0.0) atomicMax(&ic->lam[(n + 1) % 3], lam_bits(l));
        if (anybad) atomicOr(&ic->err_pending, kErrNonphysical);
      }
      if (err) atomicOr(&ic->err_pending, err);
      __threadfence();
      const unsigned nt = (unsigned)(a.nstrips * a.nchunks);
      const unsigned prev = atomicAdd(&b.rc[i].done, 1u);
      if (prev == (s + 1) * nt - 1) {
        // last task of step s of instance i: close the step
        __threadfence();
        const unsigned e = atomicExch(&ic->err_pending, 0u);
        Ctrl c;
        c.step = n;
        // L2 reads: another SM wrote these fields during this launch
        c.t = __ldcg(&ic->t);
        c.t_end = 0.0;
        c.err_committed = __ldcg(&ic->err_committed);
        if (run) {
          c.t += dt;
          c.step = n + 1;
          ic->t = c.t;
          ic->dt_last = dt;
          ic->step = n + 1;
          ic->lam[(n + 2) % 3] = 0ull;
        }
        if (e) c.err_committed = atomicOr(&ic->err_committed, e) | e;
        // plan the next step: lmax(W^{n+1}) is complete now
        StepPlan pl;
        pl.step = c.step;
        pl.dt = 0.0;
        pl.run = choose_dt(a.pol, c, lam_value(__ldcg(&ic->lam[c.step % 3])), &pl.dt, &pl.err) ? 1 : 0;
        pl.hx = 0.5 * (pl.dt / a.dx);
        pl.hy = 0.5 * (pl.dt / a.dy);
        b.plan[i] = pl;
        __threadfence();
        if (i != b.skip_release) st_release(&b.rc[i].released, s + 1);
      }
    }
    __syncwarp();
  }
}

struct BatchVariant {
  int system, precision, V, TY, NW;
  int smem;  // dynamic shared memory per block (cp.async ring)
  const void *kernel;
  const char *desc;
};

#define FV_BVARIANT(SYS, SYSID, R, PREC, V, TY, NW, MB, D, DESC)                                   \
  out.push_back(BatchVariant{SYSID, PREC, V, TY, NW,                                              \
                             (D) < 0 ? async_smem_bytes<R, V, SYS::NV, ((D) < 0 ? -(D) : 2)>(NW) : 0,     \
                             reinterpret_cast<const void *>(&fv_batch_kernel<SYS, R, V, TY, NW, MB, D>), DESC})

static const std::vector<BatchVariant> &batch_variants() {
  static std::vector<BatchVariant> out;
  if (out.empty()) {
    FV_BVARIANT(Euler, kEuler, float, 1, 2, 64, 4, 4, -6, "batch euler f32 v2 ty64 w4 b4 async6");
    FV_BVARIANT(Euler, kEuler, float, 1, 2, 64, 4, 4, -4, "batch euler f32 v2 ty64 w4 b4 async4");
    FV_BVARIANT(Euler, kEuler, float, 1, 2, 64, 4, 4, -8, "batch euler f32 v2 ty64 w4 b4 async8");
    FV_BVARIANT(Euler, kEuler, float, 1, 2, 32, 4, 4, -6, "batch euler f32 v2 ty32 w4 b4 async6");
    FV_BVARIANT(Euler, kEuler, float, 1, 2, 128, 4, 4, -6, "batch euler f32 v2 ty128 w4 b4 async6");
    FV_BVARIANT(Euler, kEuler, float, 1, 2, 128, 4, 4, -4, "batch euler f32 v2 ty128 w4 b4 async4");
    FV_BVARIANT(Euler, kEuler, float, 1, 2, 256, 4, 4, -6, "batch euler f32 v2 ty256 w4 b4 async6");
    FV_BVARIANT(Euler, kEuler, float, 1, 1, 64, 4, 5, -6, "batch euler f32 v1 ty64 w4 b5 async6");
    FV_BVARIANT(Euler, kEuler, float, 1, 1, 64, 4, 6, -4, "batch euler f32 v1 ty64 w4 b6 async4");
    FV_BVARIANT(Euler, kEuler, float, 1, 1, 64, 4, 5, 0, "batch euler f32 v1 ty64 w4 b5");
    FV_BVARIANT(EulerPC, kEuler, double, 0, 1, 64, 4, 3, -4, "batch euler f64 v1 ty64 w4 b3 async4 pc");
    FV_BVARIANT(EulerPC, kEuler, double, 0, 1, 32, 4, 2, 0, "batch euler f64 v1 ty32 w4 b2 pc");
    FV_BVARIANT(Advection, kAdvection, double, 0, 1, 32, 4, 4, 0, "batch advection f64 v1 ty32 w4 b4");
    FV_BVARIANT(Advection, kAdvection, float, 1, 1, 64, 4, 6, 0, "batch advection f32 v1 ty64 w4 b6");
    FV_BVARIANT(Advection, kAdvection, float, 1, 1, 64, 4, 6, -6, "batch advection f32 v1 ty64 w4 b6 async6");
  }
  return out;
}

}  // namespace fv

using namespace fv;

struct fv_batch {
  int n = 0;
  int system = 0, prec = 0, nvar = 0;
  // FP64 Euler: each buffer also holds the primitives u, v, p, c of its cells
  // (planes 4..7, the EulerPC system), and each instance's boundary states
  // their primitives (4 sides x 4 values)
  int nplanes = 0;
  std::vector<double> bc_pc;
  size_t esize = 0;
  std::vector<fv_config> cfg;
  std::vector<long long> pitch, plane;
  std::vector<size_t> off;     // byte offset of each instance's first buffer
  std::vector<size_t> bytes;   // bytes of one buffer of each instance
  std::vector<double> dx, dy;
  std::vector<int> has_state;
  char *arena = nullptr;
  void *d_args = nullptr;      // StepArgs<R>[n]
  Ctrl *ictrl = nullptr;
  Ctrl *h_ictrl = nullptr;
  StepPlan *plan = nullptr;    // per-instance dt decision of the next step
  unsigned char *runblock = nullptr;  // RunCounters[n] + ticket + abort
  size_t runblock_bytes = 0;
  unsigned *h_abort = nullptr;
  int *task_inst = nullptr, *task_base = nullptr;
  int T = 0;
  int variant = -1;
  int grid = 0;
  int sms = 0;
  long long timeout_ns = 2000000000LL;
  int skip_release = -1;
  bool tuned = false;
  std::string choice;          // how the kernel was chosen (fv_batch_kernel_choice)
  int dataflow = 0;
  RunInfo *info = nullptr, *h_info = nullptr;  // per instance, device and pinned host
  char *ckpt = nullptr;                        // dataflow: every instance's state at run start
  std::vector<size_t> ck_off;
  size_t tdone_off = 0, flagged_off = 0;       // inside runblock
  void *staging = nullptr;
  size_t staging_bytes = 0;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  std::map<int, cudaGraphExec_t> graphs;
  std::string err;
};

static fv_status bfail(fv_batch *b, fv_status s, const std::string &m) {
  if (b) b->err = m;
  return s;
}

#define FV_BCUDA(b, call)                                                                         \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA,                 \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                           \
  } while (0)

static void bfree_graphs(fv_batch *b) {
  for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

extern "C" const char *fv_batch_last_error(const fv_batch *b) { return b ? b->err.c_str() : ""; }

extern "C" void fv_batch_destroy(fv_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  bfree_graphs(b);
  if (b->arena) cudaFree(b->arena);
  if (b->d_args) cudaFree(b->d_args);
  if (b->ictrl) cudaFree(b->ictrl);
  if (b->plan) cudaFree(b->plan);
  if (b->info) cudaFree(b->info);
  if (b->h_info) cudaFreeHost(b->h_info);
  if (b->ckpt) cudaFree(b->ckpt);
  if (b->h_ictrl) cudaFreeHost(b->h_ictrl);
  if (b->runblock) cudaFree(b->runblock);
  if (b->h_abort) cudaFreeHost(b->h_abort);
  if (b->task_inst) cudaFree(b->task_inst);
  if (b->task_base) cudaFree(b->task_base);
  if (b->staging) cudaFree(b->staging);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

template <class R>
static void fill_args(const fv_batch *b, int k, const BatchVariant &V, StepArgs<R> &a) {
  std::memset(&a, 0, sizeof(a));
  const fv_config &c = b->cfg[k];
  a.buf0 = (R *)(b->arena + b->off[k]);
  a.buf1 = (R *)(b->arena + b->off[k] + b->bytes[k]);
  a.ctrl = b->ictrl + k;
  a.nx = c.nx;
  a.ny = c.ny;
  a.pitch = b->pitch[k];
  a.plane = b->plane[k];
  a.nstrips = (c.nx + 30 * V.V - 1) / (30 * V.V);
  a.nchunks = (c.ny + V.TY - 1) / V.TY;
  a.ntasks = a.nstrips * a.nchunks;
  a.dx = b->dx[k];
  a.dy = b->dy[k];
  a.pol.h = a.dx < a.dy ? a.dx : a.dy;
  a.pol.cfl = c.cfl;
  a.pol.fixed_dt = c.fixed_dt;
  a.pol.dt_cap = 1.0e308;
  if (c.system == FV_ADVECTION) {
    a.sp.p0 = (R)c.params[0];
    a.sp.p1 = (R)c.params[1];
  } else {
    a.sp.p0 = (R)c.params[0];
    a.sp.p1 = (R)(c.params[0] - 1.0);
  }
  for (int s = 0; s < 4; ++s) {
    a.bc[s] = c.bc[s];
    for (int v = 0; v < 8; ++v) a.bc_state[s][v] = (R)c.bc_state[s][v];
    if (b->nplanes > b->nvar)  // carried primitives of a Dirichlet ghost
      for (int v = 0; v < 4; ++v) a.bc_state[s][4 + v] = (R)b->bc_pc[16 * k + 4 * s + v];
  }
}

static fv_status batch_select(fv_batch *b, int vi) {
  const BatchVariant &V = batch_variants()[vi];
  // per-instance args and the task tables of one step
  std::vector<int> tinst, tbase(b->n);
  int T = 0;
  std::vector<unsigned char> args;
  const size_t asz = b->prec == 0 ? sizeof(StepArgs<double>) : sizeof(StepArgs<float>);
  args.resize(asz * b->n);
  for (int k = 0; k < b->n; ++k) {
    int nt;
    if (b->prec == 0) {
      StepArgs<double> a;
      fill_args<double>(b, k, V, a);
      std::memcpy(&args[asz * k], &a, asz);
      nt = a.ntasks;
    } else {
      StepArgs<float> a;
      fill_args<float>(b, k, V, a);
      std::memcpy(&args[asz * k], &a, asz);
      nt = a.ntasks;
    }
    tbase[k] = T;
    for (int q = 0; q < nt; ++q) tinst.push_back(k);
    T += nt;
  }
  if (b->task_inst) cudaFree(b->task_inst);
  if (b->task_base) cudaFree(b->task_base);
  b->task_inst = b->task_base = nullptr;
  FV_BCUDA(b, cudaMalloc(&b->task_inst, sizeof(int) * T));
  FV_BCUDA(b, cudaMalloc(&b->task_base, sizeof(int) * b->n));
  FV_BCUDA(b, cudaMemcpy(b->task_inst, tinst.data(), sizeof(int) * T, cudaMemcpyHostToDevice));
  FV_BCUDA(b, cudaMemcpy(b->task_base, tbase.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice));
  FV_BCUDA(b, cudaMemcpy(b->d_args, args.data(), asz * b->n, cudaMemcpyHostToDevice));
  if (V.smem > 0)
    FV_BCUDA(b, cudaFuncSetAttribute(V.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, V.smem));
  int nb = 0;
  FV_BCUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, V.kernel, V.NW * 32, V.smem));
  if (nb < 1) return bfail(b, FV_ERR_CUDA, "batched kernel cannot launch");
  b->grid = nb * b->sms;
  b->T = T;
  b->variant = vi;
  bfree_graphs(b);
  // run counters: RunCounters[n], ticket, abort, flagged[n], tdone[T]
  b->flagged_off = sizeof(RunCounters) * b->n + 2 * sizeof(unsigned);
  b->tdone_off = b->flagged_off + sizeof(unsigned) * b->n;
  const size_t rb = b->tdone_off + sizeof(unsigned) * (size_t)T;
  if (rb != b->runblock_bytes) {
    if (b->runblock) cudaFree(b->runblock);
    b->runblock = nullptr;
    b->runblock_bytes = 0;
    FV_BCUDA(b, cudaMalloc(&b->runblock, rb));
    FV_BCUDA(b, cudaMemset(b->runblock, 0, rb));
    b->runblock_bytes = rb;
  }
  return FV_OK;
}

extern "C" fv_status fv_batch_init(const fv_config *cfgs, int n, fv_batch **out) {
  if (!out || !cfgs || n < 1) return FV_ERR_INVALID_ARG;
  *out = nullptr;
  fv_batch *b = new fv_batch();
  b->n = n;
  b->system = cfgs[0].system;
  b->prec = cfgs[0].precision == FV_F64 ? 0 : 1;
  b->esize = b->prec == 0 ? 8 : 4;
  for (int k = 0; k < n; ++k) {
    const fv_config &c = cfgs[k];
    if (c.system != cfgs[0].system || c.precision != cfgs[0].precision || c.stream != cfgs[0].stream ||
        c.tune != cfgs[0].tune) {
      fv_batch_destroy(b);
      return FV_ERR_INVALID_ARG;
    }
    if (c.system == FV_SPRAY || (c.precision != FV_F64 && c.precision != FV_F32) || c.nx < 1 ||
        c.ny < 1 || !(c.xmax > c.xmin) || !(c.ymax > c.ymin) || c.npart_x < 1 || c.npart_y < 1 ||
        c.npart_x > c.nx || c.npart_y > c.ny || (!(c.cfl > 0.0) && !(c.fixed_dt > 0.0)) ||
        ((c.bc[0] == 0) != (c.bc[2] == 0)) || ((c.bc[1] == 0) != (c.bc[3] == 0)) ||
        (c.system == FV_EULER && !(c.params[0] > 1.0))) {
      fv_batch_destroy(b);
      return FV_ERR_INVALID_ARG;
    }
    for (int s = 0; s < 4; ++s)
      if (c.bc[s] < 0 || c.bc[s] > 2) {
        fv_batch_destroy(b);
        return FV_ERR_INVALID_ARG;
      }
  }
  b->nvar = b->system == FV_ADVECTION ? 1 : 4;
  b->nplanes = (b->system == FV_EULER && b->prec == 0) ? 8 : b->nvar;
  b->cfg.assign(cfgs, cfgs + n);
  b->stream = (cudaStream_t)cfgs[0].stream;
  b->has_state.assign(n, 0);
  size_t total = 0;
  for (int k = 0; k < n; ++k) {
    const long long pitch = ((long long)cfgs[k].nx + 31) / 32 * 32;
    const long long plane = pitch * cfgs[k].ny;
    const size_t bytes = ((size_t)plane * b->nplanes * b->esize + 255) / 256 * 256;
    b->pitch.push_back(pitch);
    b->plane.push_back(plane);
    b->bytes.push_back(bytes);
    b->off.push_back(total);
    total += 2 * bytes;
    b->dx.push_back((cfgs[k].xmax - cfgs[k].xmin) / cfgs[k].nx);
    b->dy.push_back((cfgs[k].ymax - cfgs[k].ymin) / cfgs[k].ny);
  }
  int dev = 0;
  cudaError_t e;
  auto bail = [&](cudaError_t e2, const char *what) {
    fv_batch_destroy(b);
    (void)what;
    return e2 == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA;
  };
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return bail(e, "device");
  if ((e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return bail(e, "device");
  if ((e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(e, "stream");
  if ((e = cudaMalloc(&b->arena, total)) != cudaSuccess) return bail(e, "arena");
  const size_t asz = b->prec == 0 ? sizeof(StepArgs<double>) : sizeof(StepArgs<float>);
  if ((e = cudaMalloc(&b->d_args, asz * n)) != cudaSuccess) return bail(e, "args");
  if ((e = cudaMalloc(&b->ictrl, sizeof(Ctrl) * n)) != cudaSuccess) return bail(e, "ctrl");
  if ((e = cudaMemset(b->ictrl, 0, sizeof(Ctrl) * n)) != cudaSuccess) return bail(e, "ctrl");
  // all-ones: step -1, no plan yet
  if ((e = cudaMalloc(&b->plan, sizeof(StepPlan) * n)) != cudaSuccess) return bail(e, "plan");
  if ((e = cudaMemset(b->plan, 0xff, sizeof(StepPlan) * n)) != cudaSuccess) return bail(e, "plan");
  if ((e = cudaMallocHost(&b->h_ictrl, sizeof(Ctrl) * n)) != cudaSuccess) return bail(e, "ctrl");
  if ((e = cudaMalloc(&b->info, sizeof(RunInfo) * n)) != cudaSuccess) return bail(e, "run info");
  if ((e = cudaMallocHost(&b->h_info, sizeof(RunInfo) * n)) != cudaSuccess) return bail(e, "run info");
  for (int k = 0; k < n; ++k) {
    std::memset(&b->h_info[k], 0, sizeof(RunInfo));
    b->h_info[k].active = 1;
  }
  if ((e = cudaMemcpy(b->info, b->h_info, sizeof(RunInfo) * n, cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e, "run info");
  if ((e = cudaMallocHost(&b->h_abort, sizeof(unsigned))) != cudaSuccess) return bail(e, "abort");
  if (b->nplanes > b->nvar) {
    // primitives of every instance's boundary states, by the kernels' own prims
    b->bc_pc.assign((size_t)16 * n, 0.0);
    double *d_bc = nullptr;
    if ((e = cudaMalloc(&d_bc, sizeof(double) * 48)) != cudaSuccess) return bail(e, "bc");
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
      double h_bc[32];
      for (int s2 = 0; s2 < 4; ++s2)
        for (int v = 0; v < 8; ++v) h_bc[8 * s2 + v] = cfgs[k].bc_state[s2][v];
      if ((e = cudaMemcpy(d_bc, h_bc, sizeof(h_bc), cudaMemcpyHostToDevice)) == cudaSuccess &&
          (e = launch_bc_prims(d_bc, cfgs[k].params[0], d_bc + 32, b->cap_stream)) == cudaSuccess &&
          (e = cudaStreamSynchronize(b->cap_stream)) == cudaSuccess)
        e = cudaMemcpy(&b->bc_pc[16 * (size_t)k], d_bc + 32, sizeof(double) * 16, cudaMemcpyDeviceToHost);
    }
    cudaFree(d_bc);
    if (e != cudaSuccess) return bail(e, "boundary primitives");
  }
  int vi = -1;
  const auto &vs = batch_variants();
  std::vector<int> cand;
  for (size_t k = 0; k < vs.size(); ++k)
    if (vs[k].system == b->system && vs[k].precision == b->prec) cand.push_back((int)k);
  if (cand.empty()) {
    fv_batch_destroy(b);
    return FV_ERR_INVALID_ARG;
  }
  vi = cand[0];
  b->choice = cfgs[0].tune == 1 ? "autotuned: the fastest candidate on one timed step before the first run"
                                : "heuristic (no table entry): the first candidate";
  if (cfgs[0].tune == 0) {
    long long cells = 0;
    for (int k = 0; k < n; ++k) cells += (long long)cfgs[k].nx * cfgs[k].ny;
    if (const TuneEntry *te = tune_lookup(b->system, b->prec, cells, kTuneBatch))
      for (int k : cand)
        if (std::string(vs[k].desc) == te->kernel) {
          vi = k;
          b->choice = tune_describe(*te);
        }
  }
  if (cfgs[0].tune >= 2) {
    if (cfgs[0].tune - 2 >= (int)cand.size()) {
      fv_batch_destroy(b);
      return FV_ERR_INVALID_ARG;
    }
    vi = cand[cfgs[0].tune - 2];
    b->choice = "forced: candidate " + std::to_string(cfgs[0].tune - 2);
  }
  fv_status st = batch_select(b, vi);
  if (st != FV_OK) {
    fv_batch_destroy(b);
    return st;
  }
  *out = b;
  return FV_OK;
}

static fv_status read_ictrl(fv_batch *b) {
  FV_BCUDA(b, cudaMemcpyAsync(b->h_ictrl, b->ictrl, sizeof(Ctrl) * b->n, cudaMemcpyDeviceToHost, b->stream));
  FV_BCUDA(b, cudaStreamSynchronize(b->stream));
  return FV_OK;
}

extern "C" fv_status fv_batch_set_state(fv_batch *b, int k, const void *src, int src_is_device, int src_dtype,
                                        int layout) {
  if (!b) return FV_ERR_INVALID_ARG;
  if (k < 0 || k >= b->n || !src || (src_dtype != FV_F64 && src_dtype != FV_F32) ||
      (layout != FV_CONSERVED && layout != FV_PRIMITIVE))
    return bfail(b, FV_ERR_INVALID_ARG, "bad argument");
  const fv_config &c = b->cfg[k];
  const long long ncell = (long long)c.nx * c.ny;
  const size_t sbytes = (size_t)ncell * b->nvar * (src_dtype == FV_F64 ? 8 : 4);
  const void *dsrc = src;
  if (!src_is_device) {
    if (b->staging_bytes < sbytes) {
      if (b->staging) {
        FV_BCUDA(b, cudaStreamSynchronize(b->stream));
        cudaFree(b->staging);
        b->staging = nullptr;
        b->staging_bytes = 0;
      }
      FV_BCUDA(b, cudaMalloc(&b->staging, sbytes));
      b->staging_bytes = sbytes;
    }
    FV_BCUDA(b, cudaMemcpyAsync(b->staging, src, sbytes, cudaMemcpyHostToDevice, b->stream));
    dsrc = b->staging;
  }
  // the instance restarts at t = 0, step 0, with no plan
  Ctrl h;
  std::memset(&h, 0, sizeof(h));
  FV_BCUDA(b, cudaMemcpy(b->ictrl + k, &h, sizeof(Ctrl), cudaMemcpyHostToDevice));
  FV_BCUDA(b, cudaMemset(b->plan + k, 0xff, sizeof(StepPlan)));
  void *buf0 = b->arena + b->off[k];
  FV_BCUDA(b, launch_load_state(b->system, b->prec, dsrc, src_dtype == FV_F32, layout == FV_PRIMITIVE, buf0,
                                c.nx, c.ny, b->pitch[k], b->plane[k], c.params[0], b->stream));
  if (b->nplanes > b->nvar)
    FV_BCUDA(b, launch_fill_prims((double *)buf0, c.nx, c.ny, b->pitch[k], b->plane[k], c.params[0], b->stream));
  double p0 = c.params[0], p1 = c.params[1];
  if (b->system == FV_EULER) p1 = c.params[0] - 1.0;
  FV_BCUDA(b, launch_seed_lambda(b->system, b->prec, buf0, c.nx, c.ny, b->pitch[k], b->plane[k], p0, p1,
                                 b->ictrl + k, 0, b->stream));
  FV_BCUDA(b, cudaMemcpyAsync(b->h_ictrl + k, b->ictrl + k, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream));
  FV_BCUDA(b, cudaStreamSynchronize(b->stream));
  if (b->h_ictrl[k].err_pending) {
    std::memset(&h, 0, sizeof(h));
    FV_BCUDA(b, cudaMemcpy(b->ictrl + k, &h, sizeof(Ctrl), cudaMemcpyHostToDevice));
    b->has_state[k] = 0;
    return bfail(b, FV_ERR_NONPHYSICAL, "instance state is not admissible");
  }
  b->has_state[k] = 1;
  return FV_OK;
}

template <class R>
static BatchArgs<R> make_batch_args(const fv_batch *b, int nsteps) {
  BatchArgs<R> a;
  a.inst = (const StepArgs<R> *)b->d_args;
  a.ictrl = b->ictrl;
  a.plan = b->plan;
  a.rc = (RunCounters *)b->runblock;
  a.task_inst = b->task_inst;
  a.task_base = b->task_base;
  a.ticket = (unsigned *)(b->runblock + sizeof(RunCounters) * b->n);
  a.abort = a.ticket + 1;
  a.nsteps = nsteps;
  a.T = b->T;
  a.timeout_ns = b->timeout_ns;
  a.skip_release = b->skip_release;
  a.dataflow = b->dataflow;
  a.info = b->info;
  a.flagged = (unsigned *)(b->runblock + b->flagged_off);
  a.tdone = (unsigned *)(b->runblock + b->tdone_off);
  return a;
}

static fv_status batch_graph(fv_batch *b, int nsteps, int dataflow, cudaGraphExec_t *out) {
  const int key = 2 * nsteps + (dataflow ? 1 : 0);
  auto it = b->graphs.find(key);
  if (it != b->graphs.end()) {
    *out = it->second;
    return FV_OK;
  }
  if (b->graphs.size() > 8) bfree_graphs(b);
  const BatchVariant &V = batch_variants()[b->variant];
  FV_BCUDA(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaMemsetAsync(b->runblock, 0, b->runblock_bytes, b->cap_stream);
  if (e == cudaSuccess) {
    if (b->prec == 0) {
      BatchArgs<double> a = make_batch_args<double>(b, nsteps);
      a.dataflow = dataflow;
      void *args[] = {&a};
      e = cudaLaunchKernel(V.kernel, dim3(b->grid), dim3(V.NW * 32), args, V.smem, b->cap_stream);
    } else {
      BatchArgs<float> a = make_batch_args<float>(b, nsteps);
      a.dataflow = dataflow;
      void *args[] = {&a};
      e = cudaLaunchKernel(V.kernel, dim3(b->grid), dim3(V.NW * 32), args, V.smem, b->cap_stream);
    }
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, FV_ERR_CUDA, std::string("batched graph capture: ") +
                                     cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  cudaGraphExec_t ge;
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, FV_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  b->graphs[key] = ge;
  *out = ge;
  return FV_OK;
}

// Autotuner (tune = 1): before the first run, time one step of every
// candidate kernel of this system and precision on the batch's own state and
// keep the fastest (median of three timings after one warm-up).  A timed step
// writes only the buffers that the next step overwrites, and the control
// blocks are put back after every timing, so states, times and step counts
// are unchanged.
static fv_status batch_autotune(fv_batch *b) {
  fv_status st = read_ictrl(b);
  if (st != FV_OK) return st;
  const std::vector<Ctrl> saved(b->h_ictrl, b->h_ictrl + b->n);
  auto restore = [&]() -> fv_status {
    std::memcpy(b->h_ictrl, saved.data(), sizeof(Ctrl) * b->n);
    FV_BCUDA(b, cudaMemcpyAsync(b->ictrl, b->h_ictrl, sizeof(Ctrl) * b->n, cudaMemcpyHostToDevice, b->stream));
    return FV_OK;
  };
  const auto &vs = batch_variants();
  std::vector<int> cand;
  for (size_t k = 0; k < vs.size(); ++k)
    if (vs[k].system == b->system && vs[k].precision == b->prec) cand.push_back((int)k);
  cudaEvent_t e0, e1;
  FV_BCUDA(b, cudaEventCreate(&e0));
  FV_BCUDA(b, cudaEventCreate(&e1));
  int best = b->variant;
  float best_ms = 1e30f;
  for (int vi : cand) {
    if ((st = batch_select(b, vi)) != FV_OK) break;
    cudaGraphExec_t g;
    if ((st = batch_graph(b, 1, 0, &g)) != FV_OK) break;
    std::vector<float> ms;
    for (int rep = 0; rep < 4 && st == FV_OK; ++rep) {
      if ((st = restore()) != FV_OK) break;
      cudaError_t e = cudaEventRecord(e0, b->stream);
      if (e == cudaSuccess) e = cudaGraphLaunch(g, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_abort, b->runblock + sizeof(RunCounters) * b->n + sizeof(unsigned),
                                                sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e != cudaSuccess) st = bfail(b, FV_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
      else if (*b->h_abort & kErrTimeout) st = bfail(b, FV_ERR_TIMEOUT, "a batched-step wait timed out");
      else if (rep > 0) ms.push_back(t);
    }
    if (st != FV_OK) break;
    std::sort(ms.begin(), ms.end());
    if (ms[ms.size() / 2] < best_ms) {
      best_ms = ms[ms.size() / 2];
      best = vi;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const fv_status rs = restore();
  if (st == FV_OK) st = rs;
  if (st == FV_OK) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) st = bfail(b, FV_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
  }
  if (st != FV_OK) return st;
  b->tuned = true;
  return batch_select(b, best);
}

// One launch of the persistent kernel for nsteps steps (step-gated or
// dataflow) and the timeout check; synchronises and refreshes h_ictrl.
static fv_status batch_launch(fv_batch *b, int nsteps, int dataflow) {
  cudaGraphExec_t g;
  fv_status st = batch_graph(b, nsteps, dataflow, &g);
  if (st != FV_OK) return st;
  FV_BCUDA(b, cudaGraphLaunch(g, b->stream));
  FV_BCUDA(b, cudaMemcpyAsync(b->h_abort, b->runblock + sizeof(RunCounters) * b->n + sizeof(unsigned),
                              sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
  st = read_ictrl(b);
  if (st != FV_OK) return st;
  if (*b->h_abort & kErrTimeout) return bfail(b, FV_ERR_TIMEOUT, "a batched-step wait timed out");
  return FV_OK;
}

static fv_status upload_info(fv_batch *b) {
  FV_BCUDA(b, cudaMemcpyAsync(b->info, b->h_info, sizeof(RunInfo) * b->n, cudaMemcpyHostToDevice, b->stream));
  return FV_OK;
}

static char *instance_buffer(fv_batch *b, int k, long long step) {
  return b->arena + b->off[k] + ((step & 1) ? b->bytes[k] : 0);
}

// Dataflow run (see the file header): instances whose state at the start
// already fails the paper's check, or that carry a committed error, and the
// instances flagged during the run, are replayed from their state at the
// start by the step-gated kernel.
static fv_status batch_run_dataflow(fv_batch *b, int nsteps) {
  fv_status st = read_ictrl(b);
  if (st != FV_OK) return st;
  const std::vector<Ctrl> saved(b->h_ictrl, b->h_ictrl + b->n);
  std::vector<int> replay;
  for (int k = 0; k < b->n; ++k) {
    const Ctrl &c = saved[k];
    const double dt = b->cfg[k].fixed_dt, h = b->dx[k] < b->dy[k] ? b->dx[k] : b->dy[k];
    double lam;
    std::memcpy(&lam, &c.lam[c.step % 3], sizeof(lam));
    const bool ok = c.err_committed == 0u && lam <= 1.0e300 && !(dt * lam > h);
    RunInfo &r = b->h_info[k];
    r.base = c.step;
    r.active = ok ? 1 : 0;
    r.dt = dt;
    r.hx = 0.5 * (dt / b->dx[k]);
    r.hy = 0.5 * (dt / b->dy[k]);
    if (!ok) {
      replay.push_back(k);
      continue;
    }
    b->h_ictrl[k].lam[(c.step + nsteps) % 3] = 0ull;  // filled by the run's last step
    FV_BCUDA(b, cudaMemcpyAsync(b->ckpt + b->ck_off[k], instance_buffer(b, k, c.step), b->bytes[k],
                                cudaMemcpyDeviceToDevice, b->stream));
  }
  if ((st = upload_info(b)) != FV_OK) return st;
  FV_BCUDA(b, cudaMemcpyAsync(b->ictrl, b->h_ictrl, sizeof(Ctrl) * b->n, cudaMemcpyHostToDevice, b->stream));
  if ((st = batch_launch(b, nsteps, 1)) != FV_OK) return st;
  std::vector<unsigned> flagged(b->n);
  FV_BCUDA(b, cudaMemcpy(flagged.data(), b->runblock + b->flagged_off, sizeof(unsigned) * b->n,
                         cudaMemcpyDeviceToHost));
  for (int k = 0; k < b->n; ++k) {
    if (!b->h_info[k].active) continue;
    Ctrl &c = b->h_ictrl[k];
    if (flagged[k]) {
      // back to the state at the start of the run, then replayed below
      FV_BCUDA(b, cudaMemcpyAsync(instance_buffer(b, k, saved[k].step), b->ckpt + b->ck_off[k], b->bytes[k],
                                  cudaMemcpyDeviceToDevice, b->stream));
      c = saved[k];
      replay.push_back(k);
      continue;
    }
    // what the step-gated kernel's closing warps would have left: t advanced
    // by the same FP64 additions, the step count, and the lmax slots
    double t = saved[k].t;
    for (int j = 0; j < nsteps; ++j) t += b->h_info[k].dt;
    c.t = t;
    c.dt_last = b->h_info[k].dt;
    c.step = saved[k].step + nsteps;
    c.lam[(c.step + 1) % 3] = 0ull;
    c.err_pending = 0u;
    c.blocks_done = 0u;
  }
  FV_BCUDA(b, cudaMemcpyAsync(b->ictrl, b->h_ictrl, sizeof(Ctrl) * b->n, cudaMemcpyHostToDevice, b->stream));
  FV_BCUDA(b, cudaMemsetAsync(b->plan, 0xff, sizeof(StepPlan) * b->n, b->stream));
  if (!replay.empty()) {
    for (int k = 0; k < b->n; ++k) b->h_info[k].active = 0;
    for (int k : replay) b->h_info[k].active = 1;
    if ((st = upload_info(b)) != FV_OK) return st;
    if ((st = batch_launch(b, nsteps, 0)) != FV_OK) return st;
  }
  FV_BCUDA(b, cudaStreamSynchronize(b->stream));
  return read_ictrl(b);
}

extern "C" fv_status fv_batch_run(fv_batch *b, int nsteps) {
  if (!b) return FV_ERR_INVALID_ARG;
  if (nsteps < 0) return bfail(b, FV_ERR_INVALID_ARG, "nsteps < 0");
  for (int k = 0; k < b->n; ++k)
    if (!b->has_state[k]) return bfail(b, FV_ERR_STATE, "an instance has no state");
  if (nsteps == 0) return FV_OK;
  // tickets of one run must fit the 32-bit counter
  if ((unsigned long long)nsteps * (unsigned long long)b->T >= (1ull << 31))
    return bfail(b, FV_ERR_INVALID_ARG, "too many steps in one run");
  if (b->cfg[0].tune == 1 && !b->tuned) {
    fv_status st = batch_autotune(b);
    if (st != FV_OK) return st;
  }
  fv_status st;
  if (b->dataflow) {
    st = batch_run_dataflow(b, nsteps);
    // every instance active again for the runs that follow, whatever happened
    for (int k = 0; k < b->n; ++k) b->h_info[k].active = 1;
    fv_status st2 = upload_info(b);
    if (st2 == FV_OK && cudaStreamSynchronize(b->stream) != cudaSuccess)
      st2 = bfail(b, FV_ERR_CUDA, "synchronise after a dataflow run");
    if (st == FV_OK) st = st2;
  } else {
    st = batch_launch(b, nsteps, 0);
  }
  if (st != FV_OK) return st;
  unsigned all = 0;
  for (int k = 0; k < b->n; ++k) all |= b->h_ictrl[k].err_committed;
  if (all & kErrCfl) return bfail(b, FV_ERR_CFL, "an instance's fixed dt violates the CFL condition");
  if (all & kErrNonphysical) return bfail(b, FV_ERR_NONPHYSICAL, "an instance reached a non-physical state");
  if (all & kErrZeroSpeed) return bfail(b, FV_ERR_INVALID_ARG, "an instance has lmax = 0");
  return FV_OK;
}

extern "C" fv_status fv_batch_set_dataflow(fv_batch *b, int on) {
  if (!b) return FV_ERR_INVALID_ARG;
  if (on) {
    for (int k = 0; k < b->n; ++k)
      if (!(b->cfg[k].fixed_dt > 0.0))
        return bfail(b, FV_ERR_INVALID_ARG, "dataflow needs every instance in fixed-dt mode (fixed_dt > 0)");
    if (!b->ckpt) {
      size_t total = 0;
      b->ck_off.assign(b->n, 0);
      for (int k = 0; k < b->n; ++k) {
        b->ck_off[k] = total;
        total += b->bytes[k];
      }
      FV_BCUDA(b, cudaMalloc(&b->ckpt, total));
    }
  }
  b->dataflow = on ? 1 : 0;
  return FV_OK;
}

extern "C" fv_status fv_batch_get_state(fv_batch *b, int k, void *dst, int dst_is_device, int dst_dtype) {
  if (!b) return FV_ERR_INVALID_ARG;
  if (k < 0 || k >= b->n || !dst || (dst_dtype != FV_F64 && dst_dtype != FV_F32))
    return bfail(b, FV_ERR_INVALID_ARG, "bad argument");
  if (!b->has_state[k]) return bfail(b, FV_ERR_STATE, "instance has no state");
  fv_status st = read_ictrl(b);
  if (st != FV_OK) return st;
  const fv_config &c = b->cfg[k];
  const char *cur = b->arena + b->off[k] + ((b->h_ictrl[k].step & 1) ? b->bytes[k] : 0);
  const size_t dsz = dst_dtype == FV_F64 ? 8 : 4;
  const long long ncell = (long long)c.nx * c.ny;
  if ((dst_dtype == FV_F64) == (b->prec == 0)) {
    FV_BCUDA(b, cudaMemcpy2DAsync(dst, c.nx * dsz, cur, b->pitch[k] * b->esize, c.nx * dsz,
                                  (size_t)b->nvar * c.ny,
                                  dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
  } else {
    void *target = dst;
    const size_t need = (size_t)ncell * b->nvar * dsz;
    if (!dst_is_device) {
      if (b->staging_bytes < need) {
        FV_BCUDA(b, cudaStreamSynchronize(b->stream));
        if (b->staging) cudaFree(b->staging);
        b->staging = nullptr;
        b->staging_bytes = 0;
        FV_BCUDA(b, cudaMalloc(&b->staging, need));
        b->staging_bytes = need;
      }
      target = b->staging;
    }
    FV_BCUDA(b, launch_store_state(b->prec, b->nvar, cur, target, dst_dtype == FV_F32, c.nx, c.ny, b->pitch[k],
                                   b->plane[k], b->stream));
    if (!dst_is_device)
      FV_BCUDA(b, cudaMemcpyAsync(dst, b->staging, need, cudaMemcpyDeviceToHost, b->stream));
  }
  FV_BCUDA(b, cudaStreamSynchronize(b->stream));
  return FV_OK;
}

extern "C" fv_status fv_batch_time(fv_batch *b, int k, double *t, long long *step) {
  if (!b || k < 0 || k >= b->n) return FV_ERR_INVALID_ARG;
  fv_status st = read_ictrl(b);
  if (st != FV_OK) return st;
  if (t) *t = b->h_ictrl[k].t;
  if (step) *step = b->h_ictrl[k].step;
  return FV_OK;
}

extern "C" fv_status fv_batch_kernel_info(fv_batch *b, int *variant, const char **desc) {
  if (!b) return FV_ERR_INVALID_ARG;
  const BatchVariant &V = batch_variants()[b->variant];
  if (variant) {
    int idx = 0;
    for (int k = 0; k < b->variant; ++k)
      if (batch_variants()[k].system == V.system && batch_variants()[k].precision == V.precision) ++idx;
    *variant = idx;
  }
  if (desc) *desc = V.desc;
  return FV_OK;
}

extern "C" fv_status fv_batch_kernel_choice(const fv_batch *b, const char **how) {
  if (!b || !how) return FV_ERR_INVALID_ARG;
  *how = b->choice.c_str();
  return FV_OK;
}

extern "C" fv_status fv_batch_set_wait_limit(fv_batch *b, double seconds, int never_release_instance) {
  if (!b || !(seconds > 0.0) || seconds > 60.0 || never_release_instance < -1 || never_release_instance >= b->n)
    return FV_ERR_INVALID_ARG;
  b->timeout_ns = (long long)(seconds * 1e9);
  b->skip_release = never_release_instance;
  bfree_graphs(b);
  return FV_OK;
}
