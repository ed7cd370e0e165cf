// Double-word ("double-float") arithmetic: a value is the unevaluated sum
// hi + lo of two IEEE single-precision numbers, |lo| <= ulp(hi)/2, which
// carries 48 significand bits.  Used to compute products and sums of FP64
// operands in the FP32 pipeline.  Building blocks: Knuth's TwoSum and
// Dekker's FastTwoSum (exact error-free transformations), the FMA-based
// exact product error, and integer-only conversions between double and
// (hi, lo) so that no step issues an FP64 instruction.
#pragma once
#include <stdint.h>

namespace sg {

// Bounds for the emulated path: every non-zero input magnitude must lie in
// [2^-32, 2^32) so that products, their low parts, the captured rounding
// errors and sums of up to 2^20 terms stay normal floats.
constexpr unsigned DW_EMIN = 1023 - 32, DW_EMAX = 1023 + 31;

// Split a double into hi (its leading 24 significand bits, exact) and lo (the
// remaining 29 bits rounded to a float), so x = hi + lo + e, |e| <= 2^-48 |x|.
// ok becomes false when x is non-zero and outside the supported range.
__device__ __forceinline__ float2 dw_split(double x, bool &ok) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned E = (hw >> 20) & 0x7ffu;
    const unsigned sign = hw & 0x80000000u;
    if ((b << 1) == 0) return make_float2(0.f, 0.f);
    if (E < DW_EMIN || E > DW_EMAX) {
        ok = false;
        return make_float2(0.f, 0.f);
    }
    const unsigned top = ((hw & 0xfffffu) << 3) | (lw >> 29);
    const float hi = __uint_as_float(sign | ((E - 896u) << 23) | top);
    const unsigned rem = lw & 0x1fffffffu;
    const float scale = __uint_as_float((E - 1075u + 127u) << 23);   // 2^(E-1075)
    const float lo = __uint_as_float(__float_as_uint(__uint2float_rn(rem) * scale) | sign);
    return make_float2(hi, lo);
}

// Exact double value of a float from its bits (no FP64 instruction).
__device__ __forceinline__ unsigned long long f2d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0) return (unsigned long long)(u & 0x80000000u) << 32;   // zero (subnormals flushed)
    return ((unsigned long long)(u & 0x80000000u) << 32) |
           ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
}

// Nearest-below double of hi + lo (|lo| <= ulp(hi)/2) with integer operations:
// both significands are aligned on a common fixed point, added as signed
// integers and renormalised; the result is within one double ulp.
__device__ __forceinline__ double dw_to_double(float hi, float lo) {
    const unsigned uh = __float_as_uint(hi), ul = __float_as_uint(lo);
    const int eh = (int)((uh >> 23) & 0xffu);
    if (eh == 0) return __longlong_as_double((long long)f2d_bits(lo));
    const int el = (int)((ul >> 23) & 0xffu);
    // hi significand at bit 29 (54-bit field), lo shifted by the exponent gap
    long long X = (long long)((uh & 0x7fffffu) | 0x800000u) << 29;
    if (uh & 0x80000000u) X = -X;
    if (el != 0) {
        const int sh = el - eh + 29;   // lo significand position relative to hi's field
        long long L = (long long)((ul & 0x7fffffu) | 0x800000u);
        L = sh >= 0 ? (L << sh) : (sh > -40 ? (L >> -sh) : 0);
        X += (ul & 0x80000000u) ? -L : L;
    }
    if (X == 0) return 0.0;
    const unsigned long long s = X < 0 ? 0x8000000000000000ull : 0ull;
    unsigned long long M = (unsigned long long)(X < 0 ? -X : X);
    const int lz = __clzll((long long)M);
    const int p = 63 - lz;                  // leading bit position; value = M * 2^(eh-127-52)
    M = p >= 52 ? (M >> (p - 52)) : (M << (52 - p));
    const long long E = (long long)eh - 127 - 52 + p + 1023;   // unbiased exponent of the result
    return __longlong_as_double((long long)(s | ((unsigned long long)E << 52) | (M & 0xfffffffffffffull)));
}

// Product of two double-words, returned unnormalised (ph + pl).
__device__ __forceinline__ float2 dw_mul(float2 a, float2 b) {
    const float ph = __fmul_rn(a.x, b.x);
    float pl = fmaf(a.x, b.x, -ph);
    pl = fmaf(a.x, b.y, pl);
    pl = fmaf(a.y, b.x, pl);
    return make_float2(ph, pl);
}

// s <- s + p (double-word accumulate): TwoSum of the high parts, low parts
// added to the error, FastTwoSum to renormalise.
__device__ __forceinline__ float2 dw_add(float2 s, float2 p) {
    const float t = __fadd_rn(s.x, p.x);
    const float bb = __fsub_rn(t, s.x);
    const float e1 = __fadd_rn(__fsub_rn(s.x, __fsub_rn(t, bb)), __fsub_rn(p.x, bb));
    const float e = __fadd_rn(e1, __fadd_rn(s.y, p.y));
    const float h = __fadd_rn(t, e);
    const float l = __fsub_rn(e, __fsub_rn(h, t));
    return make_float2(h, l);
}

}  // namespace sg
