// Validation kernel instances for robots of at most 8 links.
#include "vp_validate.cuh"

namespace vp {

const KernelSet &kernel_set_l8() {
    static const KernelSet s = make_kernel_set<8>();
    return s;
}

}  // namespace vp
