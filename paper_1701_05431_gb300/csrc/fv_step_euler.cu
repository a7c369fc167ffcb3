// fv_step_euler.cu -- fused step kernels of the Euler system (Sec. 5,
// Eq. (Euler)), one per tile candidate.
#include "fv_internal.h"
#include "fv_step.cuh"

namespace fv {

#define FV_VARIANT(R, PREC, V, TY, NW, DESC)                                              \
  out.push_back(Variant{kEuler, PREC, V, TY, NW,                                           \
                        reinterpret_cast<const void *>(&fv_step_kernel<Euler, R, V, TY, NW>), \
                        DESC})

void register_step_euler(std::vector<Variant> &out) {
  FV_VARIANT(double, 0, 1, 32, 4, "euler f64 v1 ty32 w4");
  FV_VARIANT(double, 0, 2, 32, 4, "euler f64 v2 ty32 w4");
  FV_VARIANT(double, 0, 1, 64, 8, "euler f64 v1 ty64 w8");
  FV_VARIANT(float, 1, 2, 32, 4, "euler f32 v2 ty32 w4");
  FV_VARIANT(float, 1, 4, 32, 4, "euler f32 v4 ty32 w4");
  FV_VARIANT(float, 1, 2, 64, 8, "euler f32 v2 ty64 w8");
  FV_VARIANT(float, 1, 2, 16, 4, "euler f32 v2 ty16 w4");
}

}  // namespace fv
