// Zero fill of the output's unwritten sector blocks (fill.cu), used by the
// planner (plan.cpp).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace symctr {

// Most sector combinations of W whose fill a bitmask passed by value can
// describe (1 KB of kernel parameters).
constexpr int64_t kFillMaskCombos = 8192;

// Zero the doubles of W's sector combinations c < n_combo whose bit in
// `written` (host memory, (n_combo + 31) / 32 words) is clear; combination c
// spans doubles [c bv, (c + 1) bv).  cudaErrorInvalidValue for more than
// kFillMaskCombos combinations.
cudaError_t launch_fill_dead(double* w, int64_t bv, int64_t n_combo, const uint32_t* written,
                             cudaStream_t st);

}  // namespace symctr
