// The status bits the kernels raise, and the range checks of the checked
// build.  Compiled with -DWQ_CHECKED=1 (see
// build.build's extra_nvcc), every guarded global access first checks that
// [off, off + n) lies inside its buffer of `total` elements; a failed check
// sets kBitChecked in the call's status word (wq_status_check then returns
// WQ_ERR_CHECK) and the access is skipped.  Nothing traps.  The default build
// compiles the checks away.
#pragma once

#include <cuda_runtime.h>

namespace wq {

constexpr unsigned kBitGeometry = 1u;
constexpr unsigned kBitNonFinite = 2u;
constexpr unsigned kBitInternal = 4u;  // a kernel met a size it was not built for
constexpr unsigned kBitChecked = 8u;   // a failed range check of the checked build

__device__ __forceinline__ bool check_range(unsigned *status, long long off, long long n, long long total) {
#if defined(WQ_CHECKED) && WQ_CHECKED
  if (off < 0 || n < 0 || off + n > total) {
    atomicOr(status, kBitChecked);
    return false;
  }
#else
  (void)status;
  (void)off;
  (void)n;
  (void)total;
#endif
  return true;
}

}  // namespace wq
