// Two-limb f32 split of a double without the FP64 pipe: f1 = RN32(v) and
// f2 = RN32(v - f1), formed from the bit pattern with integer operations
// (round to nearest even on the 52-bit significand; the remainder is an
// exact signed 30-bit integer times 2^(e-1075), converted once with RN).
// Values whose limbs would leave the normal f32 range (|v| < 2^-74 or
// |v| >= 2^127, zeros, infinities, NaN) take the FP64 conversions.
#pragma once
#include <cstdint>

namespace nsgb {

__device__ __forceinline__ void split_f64_f32(double v, float& f1, float& f2) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const int e = static_cast<int>((b >> 52) & 0x7FFull);
  if (e < 949 || e > 1149) {
    f1 = static_cast<float>(v);
    f2 = static_cast<float>(v - static_cast<double>(f1));
    return;
  }
  const unsigned long long sig = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // 53 bits
  const unsigned hi24 = static_cast<unsigned>(sig >> 29);                 // 24 bits
  const int rem = static_cast<int>(sig & 0x1FFFFFFFull);                  // 29 bits
  const int up = (rem > 0x10000000) || (rem == 0x10000000 && (hi24 & 1u));
  const unsigned sbit = static_cast<unsigned>(b >> 63) << 31;
  // exponent and significand fields added as one integer: a carry out of the
  // significand moves to the next binade, as RNE requires
  const unsigned bits1 = (static_cast<unsigned>(e - 1023 + 127) << 23) + (hi24 - (1u << 23)) + static_cast<unsigned>(up);
  f1 = __uint_as_float(sbit | bits1);
  const int ri = rem - (up ? 0x20000000 : 0);  // v - f1 = sign * ri * 2^(e - 1075)
  const float scale = __uint_as_float(static_cast<unsigned>(e - 1075 + 127) << 23);
  const float r = __int2float_rn(ri) * scale;  // exact scaling: the result is a normal float
  f2 = ri == 0 ? 0.f : (sbit ? -r : r);        // an exact split leaves +0, as v - f1 does
}

}  // namespace nsgb
