// fv_step_advection.cu -- fused step kernels of scalar linear advection
// (F = a u), one per tile candidate.
#include "fv_internal.h"
#include "fv_step.cuh"

namespace fv {

#define FV_VARIANT(R, PREC, V, TY, NW, MB, DESC)                                                     \
  out.push_back(Variant{kAdvection, PREC, V, TY, NW, MB, 0, 0,                                        \
                        reinterpret_cast<const void *>(&fv_step_kernel<Advection, R, V, TY, NW, true, MB>), \
                        DESC})

void register_step_advection(std::vector<Variant> &out) {
  FV_VARIANT(double, 0, 2, 32, 4, 1, "advection f64 v2 ty32 w4");
  FV_VARIANT(double, 0, 1, 16, 4, 1, "advection f64 v1 ty16 w4");
  FV_VARIANT(float, 1, 4, 32, 4, 1, "advection f32 v4 ty32 w4");
  FV_VARIANT(float, 1, 2, 16, 4, 1, "advection f32 v2 ty16 w4");
}

}  // namespace fv
