// Per-thread asynchronous copies global -> shared memory (cp.async; completion tracked per thread by commit and
// wait groups): a thread that copies an entry and later reads only its own entries needs no block barrier.
#pragma once

namespace evap {

// 8-byte asynchronous copy global -> shared; both addresses 8-byte aligned
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

}  // namespace evap
