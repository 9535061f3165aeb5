// IEEE-754 binary64 multiplication and addition, rounded to nearest (ties to
// even), computed with 32-bit integer instructions.
//
// This GPU issues double-precision instructions at 2 per clock per SM and
// integer instructions at 64 per clock per SM per pipe. The plain FP64 kernels
// are bound by the double pipe while the integer pipes idle, so they run a part
// of their double multiplications and additions here instead. These are the
// same IEEE operations, not approximations: for normal operands and a normal
// result the value returned is the correctly rounded product or sum, bit for
// bit what the double-precision instruction returns; so is the signed zero of a
// product with a zero operand. Subnormal, infinite and NaN operands, and results
// that would leave the normal range, go to the double-precision instruction
// itself (i64_dmul, i64_dadd), or are reported to the caller, which redoes its
// work on the double pipe (i64_dmul_nz), so every input gives the hardware's
// result. The fused multiply-adds stay on the double pipe.
//
// The algorithms are the textbook ones of IEEE arithmetic on integer
// significands (e.g. Muller et al., Handbook of Floating-Point Arithmetic,
// 2nd ed., 2018, Ch. 7): the exact 106-bit product of the 53-bit significands,
// or the sum of the significands aligned with guard bits and a sticky bit, then
// normalisation and rounding to nearest even; the significand's carry on
// rounding up propagates into the exponent field when the result is packed.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace fe {

// Significand product of normal operands whose product stays normal (biased
// exponent before normalisation e0 in [1, 2044]): the exact 106-bit product,
// normalised and rounded to nearest even, packed with the exponent and without
// the sign.
__device__ __forceinline__ unsigned long long i64_dmul_packed(uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl,
                                                              int e0) {
    const uint32_t mah = (ah & 0xFFFFFu) | 0x100000u, mbh = (bh & 0xFFFFFu) | 0x100000u;
    // P = (mah 2^32 + al)(mbh 2^32 + bl) = H 2^64 + M 2^32 + L, 2^104 <= P < 2^106
    const unsigned long long t0 = static_cast<unsigned long long>(al) * bl;
    const unsigned long long t1 = static_cast<unsigned long long>(mah) * bl + (t0 >> 32);
    const unsigned long long t2 = static_cast<unsigned long long>(al) * mbh + static_cast<uint32_t>(t1);
    const unsigned long long H = static_cast<unsigned long long>(mah) * mbh + (t1 >> 32) + (t2 >> 32);
    const uint32_t M = static_cast<uint32_t>(t2), L = static_cast<uint32_t>(t0);
    const uint32_t s = static_cast<uint32_t>(H >> 41);                 // 1 if P >= 2^105
    const unsigned long long Q = (H << 12) | (M >> 20);               // P >> 52
    unsigned long long m = Q >> s;                                     // 53 significant bits
    const uint32_t rbit = s ? static_cast<uint32_t>(Q & 1u) : ((M >> 19) & 1u);
    const uint32_t sticky = (M & (s ? 0xFFFFFu : 0x7FFFFu)) | L;
    m += rbit & ((sticky != 0u) | static_cast<uint32_t>(m & 1u));
    return (static_cast<unsigned long long>(e0 + int(s) - 1) << 52) + m;
}

// The product for every input: integer instructions for normal operands with a
// normal product, the DMUL instruction otherwise.
__device__ __forceinline__ double i64_dmul(double a, double b) {
    const unsigned long long ua = static_cast<unsigned long long>(__double_as_longlong(a));
    const unsigned long long ub = static_cast<unsigned long long>(__double_as_longlong(b));
    const uint32_t ah = static_cast<uint32_t>(ua >> 32), bh = static_cast<uint32_t>(ub >> 32);
    const uint32_t ea = (ah >> 20) & 0x7FFu, eb = (bh >> 20) & 0x7FFu;
    // biased exponent of the result before normalisation (one more if the
    // significands' product reaches 2)
    const int e0 = int(ea) + int(eb) - 1023;
    if (!((ea - 1u) < 2046u && (eb - 1u) < 2046u && e0 >= 1 && e0 <= 2044)) return __dmul_rn(a, b);
    const unsigned long long r = i64_dmul_packed(ah, static_cast<uint32_t>(ua), bh, static_cast<uint32_t>(ub), e0);
    const unsigned long long sg = static_cast<unsigned long long>((ah ^ bh) & 0x80000000u) << 32;
    return __longlong_as_double(static_cast<long long>(r | sg));
}

// The product for normal or zero operands whose result is normal or zero, bit
// for bit the DMUL result; any other case (a subnormal, infinite or NaN operand,
// a result outside the normal range) sets `special` and returns an unspecified
// value, so that the caller can redo its work on the double pipe. Kernels that
// call this form take that decision once per element: the DMUL beside every
// product in i64_dmul is issued (predicated off) on every call and holds the
// double pipe as long as an executed one.
__device__ __forceinline__ double i64_dmul_nz(double a, double b, bool &special) {
    const unsigned long long ua = static_cast<unsigned long long>(__double_as_longlong(a));
    const unsigned long long ub = static_cast<unsigned long long>(__double_as_longlong(b));
    const uint32_t ah = static_cast<uint32_t>(ua >> 32), bh = static_cast<uint32_t>(ub >> 32);
    const uint32_t al = static_cast<uint32_t>(ua), bl = static_cast<uint32_t>(ub);
    const uint32_t ea = (ah >> 20) & 0x7FFu, eb = (bh >> 20) & 0x7FFu;
    const int e0 = int(ea) + int(eb) - 1023;
    const bool na = (ea - 1u) < 2046u, nb = (eb - 1u) < 2046u;
    const bool za = ((ah & 0x7FFFFFFFu) | al) == 0u, zb = ((bh & 0x7FFFFFFFu) | bl) == 0u;
    const bool normal = na && nb && e0 >= 1 && e0 <= 2044;
    const bool zero = (za && (nb || zb)) || (zb && na);
    special |= !(normal || zero);
    const unsigned long long sg = static_cast<unsigned long long>((ah ^ bh) & 0x80000000u) << 32;
    const unsigned long long r = i64_dmul_packed(ah, al, bh, bl, e0);
    return __longlong_as_double(static_cast<long long>(zero ? sg : (r | sg)));
}

__device__ __forceinline__ double i64_dadd(double a, double b) {
    const unsigned long long ua = static_cast<unsigned long long>(__double_as_longlong(a));
    const unsigned long long ub = static_cast<unsigned long long>(__double_as_longlong(b));
    const uint32_t ea = static_cast<uint32_t>(ua >> 52) & 0x7FFu, eb = static_cast<uint32_t>(ub >> 52) & 0x7FFu;
    if (!((ea - 1u) < 2046u && (eb - 1u) < 2046u)) return __dadd_rn(a, b);
    // x the operand of larger magnitude
    const bool swap = (ub & 0x7FFFFFFFFFFFFFFFull) > (ua & 0x7FFFFFFFFFFFFFFFull);
    const unsigned long long x = swap ? ub : ua, y = swap ? ua : ub;
    const uint32_t ex = swap ? eb : ea, ey = swap ? ea : eb;
    // significands with the leading one at bit 62 (ten guard bits below the last)
    const unsigned long long mx = ((x & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 10;
    unsigned long long my = ((y & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 10;
    const uint32_t d = min(ex - ey, 63u);
    const unsigned long long lost = my & ((1ull << d) - 1ull);         // shifted out: the sticky bit
    my = (my >> d) | static_cast<unsigned long long>(lost != 0ull);
    unsigned long long S = ((x ^ y) >> 63) ? mx - my : mx + my;
    if (S == 0ull) return 0.0;                                          // exact cancellation: +0
    const int lz = __clzll(static_cast<long long>(S));                  // 0 on a carry out of bit 62
    const int e = int(ex) + 1 - lz;
    if (!(e >= 1 && e <= 2045)) return __dadd_rn(a, b);
    S = lz == 0 ? ((S >> 1) | (S & 1ull)) : (S << (lz - 1));            // leading one to bit 62
    unsigned long long m = S >> 10;
    const uint32_t rbit = static_cast<uint32_t>(S >> 9) & 1u;
    m += rbit & (((S & 0x1FFull) != 0ull) | static_cast<uint32_t>(m & 1u));
    const unsigned long long r = (static_cast<unsigned long long>(e - 1) << 52) + m;
    return __longlong_as_double(static_cast<long long>(r | (x & 0x8000000000000000ull)));
}

// The sum for normal or zero operands whose result is normal or zero, bit for bit
// the DADD result (an exact cancellation gives +0, as rounding to nearest does;
// a zero operand returns the other one, and two zeros the sign rule's zero); any
// other case (a subnormal, infinite or NaN operand, a result outside the normal
// range) sets `special` and returns an unspecified value, so that the caller can
// redo its work on the double pipe, as with i64_dmul_nz.
__device__ __forceinline__ double i64_dadd_nz(double a, double b, bool &special) {
    const unsigned long long ua = static_cast<unsigned long long>(__double_as_longlong(a));
    const unsigned long long ub = static_cast<unsigned long long>(__double_as_longlong(b));
    const uint32_t ea = static_cast<uint32_t>(ua >> 52) & 0x7FFu, eb = static_cast<uint32_t>(ub >> 52) & 0x7FFu;
    const bool na = (ea - 1u) < 2046u, nb = (eb - 1u) < 2046u;
    const bool za = (ua << 1) == 0ull, zb = (ub << 1) == 0ull;
    const bool swap = (ub & 0x7FFFFFFFFFFFFFFFull) > (ua & 0x7FFFFFFFFFFFFFFFull);
    const unsigned long long x = swap ? ub : ua, y = swap ? ua : ub;
    const uint32_t ex = swap ? eb : ea, ey = swap ? ea : eb;
    const unsigned long long mx = ((x & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 10;
    unsigned long long my = ((y & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 10;
    const uint32_t d = min(ex - ey, 63u);
    const unsigned long long lost = my & ((1ull << d) - 1ull);
    my = (my >> d) | static_cast<unsigned long long>(lost != 0ull);
    unsigned long long S = ((x ^ y) >> 63) ? mx - my : mx + my;
    const bool zs = S == 0ull;
    const int lz = __clzll(static_cast<long long>(S));
    const int e = int(ex) + 1 - lz;
    S = lz == 0 ? ((S >> 1) | (S & 1ull)) : (S << ((lz - 1) & 63));
    unsigned long long m = S >> 10;
    const uint32_t rbit = static_cast<uint32_t>(S >> 9) & 1u;
    m += rbit & (((S & 0x1FFull) != 0ull) | static_cast<uint32_t>(m & 1u));
    const unsigned long long r = ((static_cast<unsigned long long>(e - 1) << 52) + m) | (x & 0x8000000000000000ull);
    special |= !((na || za) && (nb || zb) && (za || zb || zs || (e >= 1 && e <= 2045)));
    const unsigned long long z = za ? (zb ? (ua & ub) : ub) : (zb ? ua : (zs ? 0ull : r));
    return __longlong_as_double(static_cast<long long>(z));
}

// The double operations of a kernel: multiplications and additions either on the
// double pipe (INT = false) or in integer instructions (INT = true), fused
// multiply-adds always on the double pipe. Written with the round-to-nearest
// intrinsics so that nothing is contracted or reordered: the two choices give
// the same bits.
template <bool INT> struct F64 {
    __device__ __forceinline__ static double mul(double a, double b) { return INT ? i64_dmul(a, b) : __dmul_rn(a, b); }
    // the same product with the special cases left to the caller (i64_dmul_nz)
    __device__ __forceinline__ static double mul(double a, double b, bool &special) {
        return INT ? i64_dmul_nz(a, b, special) : __dmul_rn(a, b);
    }
    __device__ __forceinline__ static double add(double a, double b) { return INT ? i64_dadd(a, b) : __dadd_rn(a, b); }
    // the same sum with the special cases left to the caller (i64_dadd_nz)
    __device__ __forceinline__ static double add(double a, double b, bool &special) {
        return INT ? i64_dadd_nz(a, b, special) : __dadd_rn(a, b);
    }
    __device__ __forceinline__ static double sub(double a, double b) { return add(a, -b); }
    __device__ __forceinline__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

}  // namespace fe
