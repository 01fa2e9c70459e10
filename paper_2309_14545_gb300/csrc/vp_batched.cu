#include "vp_batched.h"

namespace vp {
int batched_validate(BatchedState &, const BatchedArgs &, std::string *msg) { *msg = "not built"; return 2; }
int batched_autotune(BatchedState &, const BatchedArgs &, std::string *msg) { *msg = "not built"; return 2; }
void batched_invalidate(BatchedState &) {}
void batched_release(BatchedState &) {}
}  // namespace vp
