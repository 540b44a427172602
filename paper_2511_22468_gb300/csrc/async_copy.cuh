// async_copy.cuh -- asynchronous global -> shared copies (cp.async, sm_80+):
// each thread copies 16 bytes without passing them through its registers;
// copies issued by a thread are grouped by commit and waited for by
// wait_group (a hardware wait, no polling loop).
#pragma once

#include <cuda_runtime.h>

namespace nb {

static __device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const size_t g = __cvta_generic_to_global(gmem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g) : "memory");
}

static __device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// wait until every group this thread committed has landed
static __device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

}  // namespace nb
