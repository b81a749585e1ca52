// Interpolation that allocates nothing: the scratch of the inverse-NTT
// passes lives in a file-scope device array instead of a caller workspace.
//
// The array is part of the library's device image, so every GPU that loads
// the library holds it (POLYDET_STATIC_SCRATCH_WORDS words) until the
// process exits.  Host code cannot use the symbol itself as a device pointer:
// the entry point looks up the array's device address with
// cudaGetSymbolAddress once per device (on its first call with that device
// current) and passes that address to the kernels.
#include <mutex>

#include "common.cuh"

static __device__ __align__(256) uint32_t g_interp_scratch[POLYDET_STATIC_SCRATCH_WORDS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};
}  // namespace

extern "C" int polydet_interp_static(polydet_plan_t pl, const uint32_t *detvals, int lo, int hi,
                                     uint32_t *residues, void *stream) {
  if (!pl || !detvals || !residues || lo < 0 || hi > pl->P || lo >= hi) return POLYDET_EINVAL;
  const uint64_t need = pl->interp_ws_words * (uint64_t)(hi - lo);
  if (need > (uint64_t)POLYDET_STATIC_SCRATCH_WORDS) {
    pd_set_error("polydet_interp_static: the prime range needs more scratch than the static array "
                 "holds; pass fewer primes per call",
                 cudaSuccess);
    return POLYDET_ETOOBIG;
  }
  int dev = 0;
  PD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return POLYDET_EINVAL;
  void *addr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      cudaError_t e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_interp_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        pd_set_error("cudaGetSymbolAddress(g_interp_scratch)", e);
        return POLYDET_ECUDA;
      }
    }
    addr = g_scratch_addr[dev];
  }
  // Every pass writes its whole output region before the next pass reads it,
  // so the array needs no clearing between calls.
  return polydet_interp(pl, detvals, lo, hi, residues, static_cast<uint32_t *>(addr), stream);
}
