// fv_step_euler_tb.cu -- two-time-steps-per-launch kernels of the Euler
// system (the paper's fixed dt, Sec. 2.2.1; see fv_tb.cuh), each candidate
// built twice: for grids periodic on every side and, with the ghost
// handling of the intermediate state, for grids with a transmissive or
// Dirichlet side.  A translation unit of their own so the build compiles
// them beside the single-step kernels.
#include "fv_internal.h"
#include "fv_step.cuh"
#include "fv_tb.cuh"

namespace fv {

// Two-step kernels (fixed dt): the periodic build, then the build for grids with a non-periodic side.
#define FV_VARIANT_TB(A, PREC, V, TY, NW, MB, D, DESC)                                                \
  out.push_back(Variant{kEuler, PREC, (V) * Ops<A>::K, TY, NW, MB, D,                                   \
                        async_smem_bytes<A, V, 4, (D < 0 ? -D : 1)>(NW),                                \
                        reinterpret_cast<const void *>(&fv_step_kernel_tb<Euler, A, V, TY, NW, MB, D>), \
                        DESC, 0, 2, 0,                                                                  \
                        reinterpret_cast<const void *>(&fv_step_kernel_tb<Euler, A, V, TY, NW, MB, D, true>)})

void register_step_euler_tb(std::vector<Variant> &out) {
  FV_VARIANT_TB(float, 1, 2, 64, 4, 3, -4, "euler f32 v2 ty64 w4 b3 async4 tb2");
  FV_VARIANT_TB(float, 1, 2, 128, 4, 3, -4, "euler f32 v2 ty128 w4 b3 async4 tb2");
  FV_VARIANT_TB(float, 1, 2, 32, 4, 3, -4, "euler f32 v2 ty32 w4 b3 async4 tb2");
  FV_VARIANT_TB(float, 1, 2, 64, 4, 3, -3, "euler f32 v2 ty64 w4 b3 async3 tb2");
  FV_VARIANT_TB(float, 1, 2, 64, 4, 2, -4, "euler f32 v2 ty64 w4 b2 async4 tb2");
  FV_VARIANT_TB(float, 1, 2, 16, 4, 3, -4, "euler f32 v2 ty16 w4 b3 async4 tb2");
  FV_VARIANT_TB(double, 0, 2, 16, 4, 1, -4, "euler f64 v2 ty16 w4 b1 async4 tb2");
  FV_VARIANT_TB(BF, 2, 2, 64, 4, 3, -4, "euler bf16 v2 ty64 w4 b3 async4 tb2");
  FV_VARIANT_TB(BF, 2, 2, 32, 4, 2, -4, "euler bf16 v2 ty32 w4 b2 async4 tb2");
  FV_VARIANT_TB(BF, 2, 2, 16, 4, 3, -4, "euler bf16 v2 ty16 w4 b3 async4 tb2");
}

}  // namespace fv
