// qlga_step2d.cuh -- fused 2D FP32 QLGA step (placeholder until the y-marching kernel lands).
#pragma once

#include <cuda_runtime.h>

#include "qlga_device.cuh"

namespace qlga {

inline bool step2d_f32_supported(int64_t, int64_t) { return false; }

inline int step2d_f32_launch(const float*, float*, int64_t, int64_t, int, PotParams, unsigned*,
                             cudaStream_t) {
    return 1;
}

}  // namespace qlga
