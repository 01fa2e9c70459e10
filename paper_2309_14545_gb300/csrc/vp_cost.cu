#include "vp_cost.h"

namespace vp {
int cost_launch(const RobotParams &, const EnvView &, const float *, int64_t, float, float *, float *, unsigned *,
                int, size_t, cudaStream_t, std::string *msg) { *msg = "not built"; return 2; }
}  // namespace vp
