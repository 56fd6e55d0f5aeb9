// Two float32 lanes in one 64-bit register (the .f32x2 instructions of sm_100 and later):
// each lane rounds exactly as the scalar instruction does, at one instruction for both.
#pragma once

#include "common.cuh"

namespace bvls {

typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 x2_sub(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 x2_pack(float lo, float hi) {
  f32x2 d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void x2_unpack(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// (s, c) += a (h + l) lane by lane, as df_fma: FMA TwoProd of a h, rounded a l, TwoSum of
// the product into s, both errors into c.  The rounded product is formed as fma(a, h, +0):
// a packed mul.rn whose result feeds a packed add.rn was found fused into one multiply-add
// by the code generator (with or without volatile, with -fmad=false too), which leaves
// TwoSum's error term wrong; the fma form is bit-identical to the scalar sequence.
__device__ __forceinline__ void df_fma_x2(f32x2& s, f32x2& c, f32x2 a, f32x2 h, f32x2 l) {
  const f32x2 p = x2_fma(a, h, 0ull);
  f32x2 e = x2_fma(a, h, x2_sub(0ull, p));
  e = x2_fma(a, l, e);
  const f32x2 t = x2_add(s, p);
  const f32x2 bb = x2_sub(t, s);
  const f32x2 err = x2_add(x2_sub(s, x2_sub(t, bb)), x2_sub(p, bb));
  c = x2_add(c, x2_add(err, e));
  s = t;
}

// (s, c) += (s2, c2) lane by lane, as df_add.
__device__ __forceinline__ void df_add_x2(f32x2& s, f32x2& c, f32x2 s2, f32x2 c2) {
  const f32x2 t = x2_add(s, s2);
  const f32x2 bb = x2_sub(t, s);
  const f32x2 err = x2_add(x2_sub(s, x2_sub(t, bb)), x2_sub(s2, bb));
  c = x2_add(c, x2_add(err, c2));
  s = t;
}

}  // namespace bvls
