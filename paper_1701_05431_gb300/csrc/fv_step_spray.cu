// fv_step_spray.cu -- transport kernels of the spray moment system
// (Sec. 6.1, Eq. (Essadki)); the source step follows in fv_spray.cu.
#include "fv_internal.h"
#include "fv_step.cuh"

namespace fv {

void register_step_spray(std::vector<Variant> &out) { (void)out; }

}  // namespace fv
