// Validation kernel instances for one link bound VP_INST_LMAX and one family
// of check orders VP_INST_FAM.  The build compiles this file once per pair
// (link bounds 8, 9, 15 and 17; families 0 pose-all, 1 interleaved,
// 2 frequent-first), so that the twelve sets compile in parallel; compiled
// without the two definitions it is empty.
#include "vp_validate.cuh"

#if defined(VP_INST_LMAX) && defined(VP_INST_FAM)
#define VP_FILL_NAME2(L, F) kernel_set_fill_l##L##_f##F
#define VP_FILL_NAME(L, F) VP_FILL_NAME2(L, F)

namespace vp {

void VP_FILL_NAME(VP_INST_LMAX, VP_INST_FAM)(KernelSet &s) { fill_kernel_set<VP_INST_LMAX, VP_INST_FAM>(s); }

}  // namespace vp
#endif
