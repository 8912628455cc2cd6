// Packed single-precision arithmetic of sm_100-class GPUs: add, sub, mul and
// fma.rn.f32x2 apply one operation to the two FP32 lanes of a 64-bit register
// pair with one issued instruction.  The collapse-time passes are bound by
// instruction issue (the z pass) or close to it (the x and y passes), so their
// complex butterflies (the two lanes of a complex value) and the per-particle
// arithmetic of two particles (one per lane) use these.  Rounding is that of
// the scalar .rn instructions; only where a scalar expression would have been
// contracted into an fma does the result differ, by FP32 rounding.
#pragma once
#include <cuda_runtime.h>

namespace pin {
namespace x2 {

__device__ __forceinline__ unsigned long long bits(float2 a) { return *reinterpret_cast<unsigned long long*>(&a); }
__device__ __forceinline__ float2 unbits(unsigned long long a) { return *reinterpret_cast<float2*>(&a); }
__device__ __forceinline__ float2 add(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(bits(a)), "l"(bits(b)));
  return unbits(r);
}
__device__ __forceinline__ float2 sub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(bits(a)), "l"(bits(b)));
  return unbits(r);
}
__device__ __forceinline__ float2 mul(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(bits(a)), "l"(bits(b)));
  return unbits(r);
}
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(bits(a)), "l"(bits(b)), "l"(bits(c)));
  return unbits(r);
}
__device__ __forceinline__ float2 splat(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 swap(float2 a) { return make_float2(a.y, a.x); }

}  // namespace x2
}  // namespace pin
