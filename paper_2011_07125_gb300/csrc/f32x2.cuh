// Packed FP32 arithmetic on sm_100-class GPUs: two FP32 lanes of one 64-bit
// register per instruction (PTX fma.rn.f32x2).  Each lane is an IEEE fused
// multiply-add rounded to nearest, so a packed FMA gives bitwise the results of
// two fmaf calls in half the issued instructions.
#pragma once

#include <cstdint>

namespace fn {

typedef unsigned long long f2_t;  // lanes: low 32 bits, high 32 bits

__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ f2_t f2_splat(float v) { return f2_pack(v, v); }
__device__ __forceinline__ float f2_lo(f2_t v) { return __uint_as_float((unsigned)(v & 0xffffffffull)); }
__device__ __forceinline__ float f2_hi(f2_t v) { return __uint_as_float((unsigned)(v >> 32)); }

// acc = a * b + acc, lane by lane
__device__ __forceinline__ void f2_fma(f2_t& acc, f2_t a, f2_t b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

}  // namespace fn
