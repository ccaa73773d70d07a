// FP32 -> TF32 rounding (8-bit exponent, 10 stored mantissa bits), to
// nearest with ties to even, the result kept in FP32 storage with the 13
// dropped bits zero.  The hardware conversion (cvt.rn.tf32.f32) rounds:
// ties go to even, subnormals round on the same grid, values past the
// largest TF32 become infinities, and every NaN comes back as the canonical
// NaN 0x7fffe000 (checked on the device), so the mask cannot turn a NaN into
// an infinity.  For finite values the result equals adding 0x0fff + bit 13
// to the bit pattern and clearing the low 13 bits, which the one-step
// kernels use.
#pragma once

namespace qtt {

__device__ __forceinline__ float tf32_rn(float x) {
  unsigned r;
  asm("cvt.rn.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r & 0xffffe000u);
}

}  // namespace qtt
