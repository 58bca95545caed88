// symctr_contract_static_scratch: the contraction for callers that cannot
// allocate device memory themselves.
//
// Some callers of this library have no way to obtain a device workspace: code
// that runs inside another framework's allocator-free region, plugins that are
// handed only input and output buffers, or hosts whose memory budget is fixed
// before they call us.  For them, the scratch this contraction needs (offset
// tables, BF16 slices, row exponents, split-K partial sums, the error word)
// lives in one file-scope device array below, which the CUDA runtime places on
// a GPU together with this library's code.  Nothing here calls cudaMalloc,
// cudaFree or any allocating routine.
//
// Costs and rules of that choice:
//   * every GPU on which this code is loaded holds kStaticScratchBytes (64 MiB)
//     until the process exits;
//   * a plan whose workspace_bytes exceeds 64 MiB is rejected with
//     SYMCTR_ERR_WORKSPACE before anything is launched;
//   * all calls share the one array on a device: calls that overlap on the GPU
//     (different streams, no ordering between them) race and corrupt each
//     other's results; calls on one stream are fine;
//   * the array keeps the last call's contents; the contraction clears what
//     must start at zero (the error word, exponent maxima, split-K sums);
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it; make that
//     first call before any stream capture begins.  The cache is keyed by the
//     device index and does not survive cudaDeviceReset or a switch to another
//     context on that device (the module is loaded again there, at another
//     address): after either, this entry point must not be called again in
//     the process;
//   * a plan whose workspace_bytes exceeds the array but whose
//     workspace_bytes_min fits runs in several passes over the irreps Q, as
//     symctr_contract does with a small workspace;
//   * device-side failures are recorded in the array's first word;
//     symctr_check_device_error with a NULL workspace reads and clears it.
#include <mutex>
#include <string>

#include "symctr_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" SYMCTR_API symctr_status symctr_contract_static_scratch(const symctr_plan* plan,
                                                                   const double* u_red,
                                                                   const double* v_red,
                                                                   double* w_red, void* stream) {
  if (!plan) return symctr::record_error(SYMCTR_ERR_NULLPTR, "NULL plan");
  // the smallest workspace the plan accepts (one pass per group of irreps)
  const uint64_t need = symctr::plan_workspace_bytes_min(plan);
  if (need > kStaticScratchBytes) {
    std::string msg = "plan needs at least " + std::to_string(need) +
                      " bytes of scratch; the static scratch holds " +
                      std::to_string(kStaticScratchBytes) + " bytes (use symctr_contract)";
    return symctr::record_error(SYMCTR_ERR_WORKSPACE, msg.c_str());
  }
  symctr_status st = SYMCTR_OK;
  void* scratch = symctr::static_scratch_address(&st);
  if (!scratch) return st;
  return symctr::contract_into_workspace(plan, u_red, v_red, w_red, scratch, kStaticScratchBytes,
                                         (cudaStream_t)stream);
}

namespace symctr {

void* static_scratch_address(symctr_status* st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    *st = record_error(SYMCTR_ERR_CUDA, cudaGetErrorString(e));
    return nullptr;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    *st = record_error(SYMCTR_ERR_UNSUPPORTED, "device index >= 64");
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* addr = nullptr;
    e = cudaGetSymbolAddress(&addr, g_static_scratch);
    if (e != cudaSuccess || !addr) {
      *st = record_error(SYMCTR_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e) : "no symbol address");
      return nullptr;
    }
    g_scratch_addr[dev] = addr;
  }
  return g_scratch_addr[dev];
}

}  // namespace symctr
