// Validation kernel instances for robots of at most 9 links.
#include "vp_validate.cuh"

namespace vp {

const KernelSet &kernel_set_l9() {
    static const KernelSet s = make_kernel_set<9>();
    return s;
}

}  // namespace vp
