// Device bounds checks of the debug build.
#pragma once

#include <cstdint>

#include "model.h"

// Compiled with -DQED_CHECKS=1 (build(checks=True) -> libqed_checks.so), every index that
// the split step's kernels read from a table (jump sources, incoming-list entries, work
// items) is checked before the access it guards: a failed check records kErrBounds in the
// error word (qed_sync_status then reports it) and the access is skipped.  Nothing traps.
// The regular build compiles the checks away.
#ifndef QED_CHECKS
#define QED_CHECKS 0
#endif

namespace qed {

__device__ __forceinline__ bool qed_check(uint32_t *err, bool ok) {
    if (!QED_CHECKS || ok) return true;
    atomicOr(err, kErrBounds);
    return false;
}

}  // namespace qed
