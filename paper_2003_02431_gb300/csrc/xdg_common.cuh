// Definitions shared by every translation unit of libxdg's kernels (sm_103a).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

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

// ---- warp-level tensor-core products (mma.sync, BF16 operands, FP32 accumulators) ----

// v = hi + mid + lo + O(2^-24 |v|), each part a BF16 number (the split of an FP32 operand into
// low-precision terms, Markidis et al. 2018: products of BF16 parts are exact in FP32, so a few
// of them reproduce an FP32 product to the FP32 rounding level)
__device__ __forceinline__ void split_bf16x3(float v, __nv_bfloat16& hi, __nv_bfloat16& mid, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(hi);
  mid = __float2bfloat16_rn(r1);
  lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
}

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo_half, __nv_bfloat16 hi_half) {
  return (uint32_t)__bfloat16_as_ushort(lo_half) | ((uint32_t)__bfloat16_as_ushort(hi_half) << 16);
}

// d += a b for one 16 x 8 x 16 tile: BF16 operands, FP32 accumulators. Fragments (PTX ISA,
// mma.m16n8k16 with .bf16): with g = lane / 4 and t = lane % 4, a holds rows g and g + 8 at
// columns 2t, 2t+1 (a[0], a[1]) and 2t+8, 2t+9 (a[2], a[3]); b holds rows 2t, 2t+1 and 2t+8,
// 2t+9 of column g; d holds rows g, g + 8 at columns 2t, 2t+1.
__device__ __forceinline__ void mma_16816_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

}  // namespace xdg
