// fv_step_euler.cu -- fused step kernels of the Euler system (Sec. 5,
// Eq. (Euler)), one per tile candidate: arithmetic type (FP64, FP32, or F2 =
// two FP32 cells per packed FP32x2 instruction), values per lane V, rows per
// warp task TY, warps per block NW, the blocks per SM the register budget
// targets, and the row staging D (0 register prefetch, > 0 TMA ring,
// < 0 cp.async ring).  The FP64 single-step and in-place kernels run the
// EulerPC system: the same arithmetic, with each cell's primitives carried
// in four more state planes from the step that computes them to the next.
#include "fv_internal.h"
#include "fv_step.cuh"

namespace fv {

#define FV_VARIANT(A, PREC, V, TY, NW, MB, D, DESC)                                                   \
  out.push_back(Variant{kEuler, PREC, (V) * Ops<A>::K, TY, NW, MB, D,                                   \
                        (D) > 0 ? tma_smem_bytes<A, V, 4, (D > 0 ? D : 1)>(NW)                          \
                                : (D) < 0 ? async_smem_bytes<A, V, 4, (D < 0 ? -D : 1)>(NW) : 0,         \
                        reinterpret_cast<const void *>(&fv_step_kernel<Euler, A, V, TY, NW, true, MB, D>), DESC})

// FP64 two-buffer kernels: Euler with carried primitives (EulerPC, eight
// planes per state: the conserved variables, then u, v, p, c).
#define FV_VARIANT_PC(PREC, V, TY, NW, MB, D, DESC)                                                 \
  out.push_back(Variant{kEuler, PREC, V, TY, NW, MB, D,                                               \
                        (D) < 0 ? async_smem_bytes<double, V, 8, (D < 0 ? -D : 1)>(NW) : 0,            \
                        reinterpret_cast<const void *>(&fv_step_kernel<EulerPC, double, V, TY, NW, true, MB, D>), \
                        DESC, 0, 0, 1})

// FP64 in-place kernels carry the primitives too (strips of eight variables).
#define FV_VARIANT_INPL_PC(PREC, V, TY, NW, MB, D, DESC)                                            \
  out.push_back(Variant{kEuler, PREC, V, TY, NW, MB, D,                                               \
                        async_smem_bytes<double, V, 8, (D < 0 ? -D : 1)>(NW),                          \
                        reinterpret_cast<const void *>(&fv_step_kernel<EulerPC, double, V, TY, NW, true, MB, D, true>), \
                        DESC, 1, 0, 1})

// In-place kernels (cp.async ring only): one state buffer plus overlap strips.
#define FV_VARIANT_INPL(A, PREC, V, TY, NW, MB, D, DESC)                                              \
  out.push_back(Variant{kEuler, PREC, (V) * Ops<A>::K, TY, NW, MB, D,                                   \
                        async_smem_bytes<A, V, 4, (D < 0 ? -D : 1)>(NW),                                \
                        reinterpret_cast<const void *>(&fv_step_kernel<Euler, A, V, TY, NW, true, MB, D, true>), \
                        DESC, 1})

void register_step_euler(std::vector<Variant> &out) {
  register_step_euler_tb(out);  // two-step kernels first (fv_step_euler_tb.cu)
  FV_VARIANT_INPL_PC(0, 1, 64, 4, 3, -4, "euler f64 v1 ty64 w4 b3 async4 inplace pc");
  FV_VARIANT_INPL_PC(0, 1, 16, 4, 3, -4, "euler f64 v1 ty16 w4 b3 async4 inplace pc");
  FV_VARIANT_INPL(float, 1, 4, 32, 4, 3, -4, "euler f32 v4 ty32 w4 b3 async4 inplace");
  FV_VARIANT_INPL(float, 1, 2, 16, 4, 4, -6, "euler f32 v2 ty16 w4 b4 async6 inplace");
  FV_VARIANT_INPL(float, 1, 2, 32, 4, 4, -6, "euler f32 v2 ty32 w4 b4 async6 inplace");
  FV_VARIANT_INPL(float, 1, 4, 64, 4, 3, -4, "euler f32 v4 ty64 w4 b3 async4 inplace");
  FV_VARIANT_INPL(BF, 2, 4, 32, 4, 3, -4, "euler bf16 v4 ty32 w4 b3 async4 inplace");
  FV_VARIANT_INPL(BF, 2, 2, 16, 4, 4, -6, "euler bf16 v2 ty16 w4 b4 async6 inplace");
  FV_VARIANT_PC(0, 1, 64, 4, 1, 0, "euler f64 v1 ty64 w4 pc");
  FV_VARIANT_PC(0, 1, 32, 4, 1, 0, "euler f64 v1 ty32 w4 pc");
  FV_VARIANT_PC(0, 1, 16, 4, 1, 0, "euler f64 v1 ty16 w4 pc");
  FV_VARIANT_PC(0, 1, 64, 4, 4, -4, "euler f64 v1 ty64 w4 b4 async4 pc");
  FV_VARIANT(float, 1, 4, 32, 4, 3, -4, "euler f32 v4 ty32 w4 b3 async4");
  FV_VARIANT(float, 1, 4, 64, 4, 3, -4, "euler f32 v4 ty64 w4 b3 async4");
  FV_VARIANT(float, 1, 4, 16, 4, 3, -4, "euler f32 v4 ty16 w4 b3 async4");
  FV_VARIANT(float, 1, 4, 64, 4, 3, -3, "euler f32 v4 ty64 w4 b3 async3");
  FV_VARIANT(float, 1, 4, 64, 4, 3, -6, "euler f32 v4 ty64 w4 b3 async6");
  FV_VARIANT(float, 1, 2, 64, 4, 5, -6, "euler f32 v2 ty64 w4 b5 async6");
  FV_VARIANT(float, 1, 2, 64, 4, 4, -6, "euler f32 v2 ty64 w4 b4 async6");
  FV_VARIANT(float, 1, 2, 64, 4, 5, -4, "euler f32 v2 ty64 w4 b5 async4");
  FV_VARIANT(float, 1, 2, 64, 4, 4, -8, "euler f32 v2 ty64 w4 b4 async8");
  FV_VARIANT(float, 1, 2, 32, 4, 5, -6, "euler f32 v2 ty32 w4 b5 async6");
  FV_VARIANT(float, 1, 2, 16, 4, 5, -6, "euler f32 v2 ty16 w4 b5 async6");
  FV_VARIANT(float, 1, 2, 64, 4, 4, 0, "euler f32 v2 ty64 w4 b4");
  FV_VARIANT(float, 1, 2, 64, 4, 4, 4, "euler f32 v2 ty64 w4 b4 tma4");
  FV_VARIANT(float, 1, 1, 64, 4, 6, 0, "euler f32 v1 ty64 w4 b6");
  FV_VARIANT(F2, 1, 1, 64, 4, 4, -6, "euler f32 x2 v1 ty64 w4 b4 async6");
  FV_VARIANT(BF, 2, 4, 32, 4, 3, -4, "euler bf16 v4 ty32 w4 b3 async4");
  FV_VARIANT(BF, 2, 4, 64, 4, 3, -4, "euler bf16 v4 ty64 w4 b3 async4");
  FV_VARIANT(BF, 2, 2, 64, 4, 5, -6, "euler bf16 v2 ty64 w4 b5 async6");
  FV_VARIANT(BF, 2, 2, 16, 4, 5, -6, "euler bf16 v2 ty16 w4 b5 async6");
  FV_VARIANT(BF, 2, 2, 64, 4, 4, -6, "euler bf16 v2 ty64 w4 b4 async6");
  FV_VARIANT(BF, 2, 2, 64, 4, 4, 0, "euler bf16 v2 ty64 w4 b4");
}

}  // namespace fv
