// Definitions shared by every translation unit of libxdg's kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>

namespace xdg {

constexpr int kThreads = 256;

// Programmatic dependent launch (sm_90+): a kernel may be launched before its predecessor in
// the stream has finished; it then waits at griddepcontrol.wait, which returns once every
// prerequisite grid has completed and its memory operations are visible. Every kernel of the
// library waits first, before any global memory access, so reads after writes and writes after
// reads across consecutive kernels keep their order. It then lets its own dependents launch,
// so their CTAs are scheduled as soon as SM slots free up instead of after a launch gap. For a
// kernel launched without the attribute both instructions have no effect.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_entry() {
  pdl_wait();
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace xdg
