// split32.cuh -- FP64 -> FP32 hi/lo split of the FP32 path (Sec. 4.7: the
// coordinates the single-precision kernel works on): hi = RN_f32(v),
// lo = RN_f32(v - hi), where v - hi is exact in FP64.
//
// The FP64 <-> FP32 conversions of the direct form run at the FP64 rate
// (1/64 of FP32 on this GPU), which made the per-evaluation split of every
// particle compute-bound.  The same bits come from integer operations on the
// IEEE pattern: with v = +-S 2^(E-52), S the 53-bit significand,
//   hi: the top 24 bits of S rounded to nearest, ties to even (a carry out
//       of 24 bits raises the exponent by one);
//   lo: t = (low 29 bits of S) - 2^29 if hi rounded up, |t| <= 2^28, so
//       v - hi = +-t 2^(E-52) exactly, and RN_f32 of that is RN_f32(+-t)
//       (an int -> float conversion) scaled by 2^(E-52), exact while the
//       result stays a normal float.
// Both stay normal for -74 <= E <= 126; zero, subnormal, very small or
// large values, infinities and NaN take the direct FP64 form.  v - hi = 0
// gives lo = +0, as the FP64 subtraction does.
#pragma once

#include <cstdint>

namespace bh {

__device__ __forceinline__ void split_f32_direct(double v, float& hi, float& lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(__dsub_rn(v, (double)hi));
}

__device__ __forceinline__ void split_f32(double v, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int E = (int)((b >> 52) & 0x7ffu) - 1023;
    if (E < -74 || E > 126) {  // also zero, subnormals (E = -1023), infinities and NaN (E = 1024)
        split_f32_direct(v, hi, lo);
        return;
    }
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const unsigned long long S = (b & ((1ull << 52) - 1)) | (1ull << 52);
    unsigned q = (unsigned)(S >> 29);           // 24 bits, top bit set
    const unsigned r = (unsigned)(S & ((1u << 29) - 1));
    const bool up = r > (1u << 28) || (r == (1u << 28) && (q & 1u));
    q += up ? 1u : 0u;
    int Eh = E;
    if (q == (1u << 24)) {  // carried out of 24 bits
        q = 1u << 23;
        ++Eh;
    }
    hi = __uint_as_float(sign | ((unsigned)(Eh + 127) << 23) | (q & ((1u << 23) - 1)));
    const int t = (int)r - (up ? (1 << 29) : 0);
    if (t == 0) {
        lo = 0.0f;
        return;
    }
    const float f = __int2float_rn(sign ? -t : t);  // RN_f32 of the exact remainder, unscaled
    lo = __uint_as_float(__float_as_uint(f) + ((unsigned)(E - 52) << 23));  // exponent field stays in [1, 254]
}

}  // namespace bh
