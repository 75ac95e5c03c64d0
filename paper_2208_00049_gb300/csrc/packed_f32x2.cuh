// Packed pairs of FP32 in one 64-bit register and the sm_100+ packed
// arithmetic on them (fma.rn.f32x2, mul.rn.f32x2): a complex64 value
// (re, im) times a real weight pair (w, w) in one instruction.
#pragma once

namespace nfftgb {

typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float x, float y) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 unpack2(f32x2 v) {
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(v));
  return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// acc += x with the rounding error of that addition added to comp: Knuth's
// TwoSum (t = a + b, b' = t - a, a' = t - b', err = (a - a') + (b - b'), exact
// for any magnitudes in round-to-nearest), on both halves of the pairs.  The
// packed operations are opaque to the compiler, so it cannot reassociate them
// away.  The caller adds comp to acc once, at the end.
__device__ __forceinline__ void two_sum_acc2(f32x2& acc, f32x2& comp, f32x2 x) {
  const f32x2 t = add2(acc, x);
  const f32x2 bp = sub2(t, acc);
  const f32x2 ap = sub2(t, bp);
  const f32x2 err = add2(sub2(acc, ap), sub2(x, bp));
  comp = add2(comp, err);
  acc = t;
}

// A shared-memory load of a pair that the compiler keeps where it is written:
// it is neither hoisted out of a loop nor merged, for tables whose values
// would otherwise be held in registers for the whole loop at the cost of
// occupancy.
__device__ __forceinline__ f32x2 lds_f32x2(const f32x2* p) {
  f32x2 r;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(r) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
  return r;
}

}  // namespace nfftgb
