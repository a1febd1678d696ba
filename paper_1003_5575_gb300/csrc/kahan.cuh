// Compensated (Kahan) FP32 summation, shared by the prediction and the adjoint.
#pragma once
#include <cuda_runtime.h>

namespace rts {

// compensated summation step: the running total is sum - comp
__device__ inline void kahan_add(float& sum, float& comp, float x) {
  const float y = x - comp;
  const float t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

}  // namespace rts
