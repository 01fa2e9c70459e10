// Penetration cost and its reverse-mode FK adjoint.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "vp_types.h"

namespace vp {

// 0 = ok, 1 = capacity, 2 = CUDA error (message in *msg)
int cost_launch(const RobotParams &P, const EnvView &env, const float *q, int64_t n, float margin, float *cost,
                float *grad, unsigned *status, int num_sms, size_t smem_optin, cudaStream_t st, std::string *msg);

}  // namespace vp
