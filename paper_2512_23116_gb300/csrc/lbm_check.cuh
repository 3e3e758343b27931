// Bounds checks of the checked build (-DLBM_BOUNDS_CHECK), a stand-in for a
// device memory checker: every checked access evaluates its condition first;
// a failed check sets this translation unit's bounds word and the access is
// skipped (a load reads zero, a copy or store is not issued).  Nothing traps or
// asserts; the host reads the words at the next synchronising call and reports
// LBM_ERR_CUDA.  In the normal build every check is the constant true and
// compiles to nothing.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace lbm {

#ifdef LBM_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
// One word per translation unit (static): the host reads each through the
// reader that unit defines.
static __device__ uint32_t g_bounds_word;
__device__ __forceinline__ bool in_bounds(bool ok) {
  if (!ok) atomicOr(&g_bounds_word, 1u);
  return ok;
}
// This translation unit's word, cleared after reading (host).
static inline uint32_t take_bounds_word() {
  uint32_t v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_bounds_word, sizeof v) != cudaSuccess) return 0xFFFFFFFFu;
  if (v) (void)cudaMemcpyToSymbol(g_bounds_word, &z, sizeof z);
  return v;
}
#else
constexpr bool kBoundsCheck = false;
__device__ __forceinline__ constexpr bool in_bounds(bool) { return true; }
static inline uint32_t take_bounds_word() { return 0u; }
#endif

// [p, p + n) inside [lo, lo + size) (bytes).
__device__ __forceinline__ bool range_in(const void* p, int64_t n, const void* lo, int64_t size) {
  const char* a = static_cast<const char*>(p);
  const char* b = static_cast<const char*>(lo);
  return n >= 0 && a >= b && a + n <= b + size;
}

}  // namespace lbm
