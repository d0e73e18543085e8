// Bounds checks of the indices the iteration kernels read from memory (scan
// ids of the slots, voxel ids of the scan-major copy, the scan order),
// compiled in only with -DMMBA_CHECKED: the checked library variant, which
// stands in for a memory sanitizer.  An index outside [0, n) sets the state's
// sticky error word to kErrIndex and is replaced by 0, so the access stays in
// bounds and the host reports the error.  Without the flag MMBA_IDX is the
// index itself.
#pragma once
#include "mmba_internal.cuh"

namespace mmba {

constexpr int32_t kErrTimeout = 1;  // error word: a bounded wait gave up
constexpr int32_t kErrIndex = 2;    // error word: an index was out of range (checked builds)

#ifdef MMBA_CHECKED
// (kernels that only read the state still record the error in it)
template <typename I>
__device__ __forceinline__ I checked_index(I i, int64_t n, const DevState* st) {
  if (i >= 0 && (int64_t)i < n) return i;
  atomicExch(&const_cast<DevState*>(st)->wait_timeout, kErrIndex);
  return I(0);
}
#define MMBA_IDX(i, n, st) ::mmba::checked_index((i), (int64_t)(n), (st))
#else
#define MMBA_IDX(i, n, st) (i)
#endif

}  // namespace mmba
