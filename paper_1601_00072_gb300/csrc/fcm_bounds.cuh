// Bounds guards of the FCM_DEBUG_BOUNDS build (compute-sanitizer is not
// available, so the kernels that issue TMA copies or index lookup tables can
// check their own indices instead).
//
// In a build with -DFCM_DEBUG_BOUNDS a guarded access whose condition fails is
// skipped, and FCM_FLAG_BOUNDS is recorded where the entry point reports it;
// a skipped TMA copy still arrives on its mbarrier, so no wait is left
// waiting. In the normal build every guard is the constant true.
#pragma once

#include "fcm.h"

namespace fcm {

#ifdef FCM_DEBUG_BOUNDS
constexpr bool kBoundsChecks = true;
#else
constexpr bool kBoundsChecks = false;
#endif

// True when the access may go ahead. A false condition in a guarded build
// sets `bit` (FCM_FLAG_BOUNDS unless given) in *word.
__device__ __forceinline__ bool in_bounds(bool ok, unsigned* word, unsigned bit = FCM_FLAG_BOUNDS) {
    if (kBoundsChecks && !ok) {
        atomicOr(word, bit);
        return false;
    }
    return true;
}

}  // namespace fcm
