// Bulk prefetch into L2 through the TMA engine (cp.async.bulk.prefetch): one
// instruction requests a whole range, with no completion to wait for.  The
// global address must be 16-byte aligned and the size a multiple of 16.
#pragma once

#include <stdint.h>

namespace gofd {

__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

}  // namespace gofd
