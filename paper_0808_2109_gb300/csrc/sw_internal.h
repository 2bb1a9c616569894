// sw_internal.h -- host helpers shared by the library's translation units
// (not part of the C ABI, not exported).
#pragma once

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

// Bond threshold floor(p * 2^32) for a bond probability p in [0, 1].
__attribute__((visibility("hidden"))) int sw_threshold_p_internal(double p, uint64_t *out);

#ifdef __cplusplus
}

#include <mutex>

// Serialises CUDA graph capture against the library's own device-wide
// synchronising calls (cudaMalloc, cudaFree): such a call made by another
// host thread in the middle of a capture invalidates it.
__attribute__((visibility("hidden"))) std::mutex &sw_capture_mutex();

// Fault injection for tests (sw_debug_fail_allocations): true while injected
// allocation failures remain, consuming one.  Every device allocation of the
// library asks first and reports cudaErrorMemoryAllocation instead.
__attribute__((visibility("hidden"))) bool sw_inject_alloc_failure();
#endif
