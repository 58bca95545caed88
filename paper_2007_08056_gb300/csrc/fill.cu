// Zero fill of the output's sector blocks that no irrep writes (Alg. 2's
// output step: an entry of W whose aligned irrep carries no work is zero).
//
// In a uniform plan each sector combination of W's reduced form (its stored
// sector labels; the block axes are innermost) is either written whole by one
// irrep's rows and columns or not written at all.  The planner marks the
// written combinations in a bitmask, passed here by value, and this kernel
// zeroes the others only, instead of zeroing all of W before the contraction
// overwrites the written part.
#include <cstdint>

#include "fill.h"
#include "symctr_internal.h"

namespace symctr {

namespace {

constexpr int kFillThreads = 256;
constexpr int64_t kFillChunk = 16384;   // doubles per work item (128 KB)

struct FillMask {
  uint32_t bits[kFillMaskCombos / 32];   // bit c: combination c is written
};

// Work item (combination c, chunk j): doubles [c bv + j kFillChunk, ...) of
// combination c, skipped whole when c is written.
__global__ void __launch_bounds__(kFillThreads) fill_dead_kernel(double* __restrict__ w, int64_t bv,
                                                                 int64_t chunks, int64_t items,
                                                                 const __grid_constant__ FillMask m) {
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t c = it / chunks;
    if ((m.bits[c >> 5] >> (c & 31)) & 1u) continue;
    const int64_t beg = c * bv + (it - c * chunks) * kFillChunk;
    const int64_t lim = (c + 1) * bv, end = beg + kFillChunk < lim ? beg + kFillChunk : lim;
    for (int64_t i = beg + threadIdx.x; i < end; i += kFillThreads) w[i] = 0.0;
  }
}

}  // namespace

cudaError_t launch_fill_dead(double* w, int64_t bv, int64_t n_combo, const uint32_t* written,
                             cudaStream_t st) {
  if (n_combo <= 0 || bv <= 0) return cudaSuccess;
  if (n_combo > kFillMaskCombos) return cudaErrorInvalidValue;
  FillMask m{};
  for (int64_t k = 0; k < (n_combo + 31) / 32; ++k) m.bits[k] = written[k];
  const int64_t chunks = (bv + kFillChunk - 1) / kFillChunk, items = n_combo * chunks;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = (int64_t)sms * 8;
  fill_dead_kernel<<<(int)(items < cap ? items : cap), kFillThreads, 0, st>>>(w, bv, chunks, items, m);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace symctr
