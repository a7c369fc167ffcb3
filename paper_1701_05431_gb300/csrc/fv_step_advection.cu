// fv_step_advection.cu -- fused step kernels of scalar linear advection
// (F = a u), one per tile candidate.
#include "fv_internal.h"
#include "fv_step.cuh"
#include "fv_tb.cuh"

namespace fv {

#define FV_VARIANT(R, PREC, V, TY, NW, MB, DESC)                                                     \
  out.push_back(Variant{kAdvection, PREC, V, TY, NW, MB, 0, 0,                                        \
                        reinterpret_cast<const void *>(&fv_step_kernel<Advection, R, V, TY, NW, true, MB>), \
                        DESC})

#define FV_VARIANT_INPL(R, PREC, V, TY, NW, MB, D, DESC)                                            \
  out.push_back(Variant{kAdvection, PREC, V, TY, NW, MB, D, async_smem_bytes<R, V, 1, -(D)>(NW),        \
                        reinterpret_cast<const void *>(&fv_step_kernel<Advection, R, V, TY, NW, true, MB, D, true>), \
                        DESC, 1})

#define FV_VARIANT_TB(R, PREC, V, TY, NW, MB, D, DESC)                                              \
  out.push_back(Variant{kAdvection, PREC, V, TY, NW, MB, D, async_smem_bytes<R, V, 1, -(D)>(NW),        \
                        reinterpret_cast<const void *>(&fv_step_kernel_tb<Advection, R, V, TY, NW, MB, D>), \
                        DESC, 0, 2, 0,                                                                  \
                        reinterpret_cast<const void *>(&fv_step_kernel_tb<Advection, R, V, TY, NW, MB, D, true>)})

void register_step_advection(std::vector<Variant> &out) {
  FV_VARIANT_TB(double, 0, 2, 32, 4, 2, -4, "advection f64 v2 ty32 w4 b2 async4 tb2");
  FV_VARIANT_TB(double, 0, 2, 16, 4, 2, -4, "advection f64 v2 ty16 w4 b2 async4 tb2");
  FV_VARIANT_TB(float, 1, 4, 32, 4, 2, -4, "advection f32 v4 ty32 w4 b2 async4 tb2");
  FV_VARIANT_TB(float, 1, 2, 16, 4, 2, -4, "advection f32 v2 ty16 w4 b2 async4 tb2");
  FV_VARIANT_INPL(double, 0, 2, 32, 4, 2, -4, "advection f64 v2 ty32 w4 b2 async4 inplace");
  FV_VARIANT_INPL(double, 0, 1, 16, 4, 2, -4, "advection f64 v1 ty16 w4 b2 async4 inplace");
  FV_VARIANT_INPL(float, 1, 4, 32, 4, 2, -4, "advection f32 v4 ty32 w4 b2 async4 inplace");
  FV_VARIANT_INPL(float, 1, 2, 16, 4, 2, -4, "advection f32 v2 ty16 w4 b2 async4 inplace");
  FV_VARIANT(double, 0, 2, 32, 4, 1, "advection f64 v2 ty32 w4");
  FV_VARIANT(double, 0, 1, 16, 4, 1, "advection f64 v1 ty16 w4");
  FV_VARIANT(float, 1, 4, 32, 4, 1, "advection f32 v4 ty32 w4");
  FV_VARIANT(float, 1, 2, 16, 4, 1, "advection f32 v2 ty16 w4");
}

}  // namespace fv
