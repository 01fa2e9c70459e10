// Validation kernel instances for robots of at most 17 links.
#include "vp_validate.cuh"

namespace vp {

const KernelSet &kernel_set_l17() {
    static const KernelSet s = make_kernel_set<17>();
    return s;
}

}  // namespace vp
