// Validation kernel instances for robots of at most 15 links.
#include "vp_validate.cuh"

namespace vp {

const KernelSet &kernel_set_l15() {
    static const KernelSet s = make_kernel_set<15>();
    return s;
}

}  // namespace vp
