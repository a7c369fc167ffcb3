// fv_step_euler.cu -- fused step kernels of the Euler system (Sec. 5,
// Eq. (Euler)), one per tile candidate: cells per lane V, rows per warp task
// TY, warps per block NW, and the blocks per SM the register budget targets.
#include "fv_internal.h"
#include "fv_step.cuh"

namespace fv {

#define FV_VARIANT(R, PREC, V, TY, NW, MB, DESC)                                                 \
  out.push_back(Variant{kEuler, PREC, V, TY, NW, MB,                                              \
                        reinterpret_cast<const void *>(&fv_step_kernel<Euler, R, V, TY, NW, true, MB>), \
                        DESC})

void register_step_euler(std::vector<Variant> &out) {
  FV_VARIANT(double, 0, 1, 32, 4, 1, "euler f64 v1 ty32 w4");
  FV_VARIANT(double, 0, 1, 64, 4, 1, "euler f64 v1 ty64 w4");
  FV_VARIANT(double, 0, 1, 64, 4, 5, "euler f64 v1 ty64 w4 b5");
  FV_VARIANT(double, 0, 2, 32, 4, 1, "euler f64 v2 ty32 w4");
  FV_VARIANT(float, 1, 1, 64, 4, 6, "euler f32 v1 ty64 w4 b6");
  FV_VARIANT(float, 1, 1, 32, 4, 6, "euler f32 v1 ty32 w4 b6");
  FV_VARIANT(float, 1, 1, 64, 4, 8, "euler f32 v1 ty64 w4 b8");
  FV_VARIANT(float, 1, 1, 128, 4, 6, "euler f32 v1 ty128 w4 b6");
  FV_VARIANT(float, 1, 2, 64, 4, 1, "euler f32 v2 ty64 w4");
  FV_VARIANT(float, 1, 2, 32, 4, 1, "euler f32 v2 ty32 w4");
  FV_VARIANT(float, 1, 2, 64, 4, 5, "euler f32 v2 ty64 w4 b5");
  FV_VARIANT(float, 1, 4, 64, 4, 1, "euler f32 v4 ty64 w4");
}

}  // namespace fv
