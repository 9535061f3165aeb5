// Double-word arithmetic on the float pipes: a value is the unevaluated sum
// h + l of two floats with |l| < ulp(h) (Dekker, Numer. Math. 18, 1971). Sums
// use Knuth's TwoSum and Dekker's Fast2Sum; the product takes the exact error of
// h*h' from the fused multiply-add and the cross terms h*l' + l*h' (the
// double-word times double-word scheme analysed by Joldes, Muller and Popescu,
// ACM TOMS 44(2), 2017, without the negligible l*l' term). Each operation has a
// relative error of a few 2^-48 in the absence of cancellation; under
// cancellation its absolute error stays a few 2^-48 (|x| + |y|), the same order
// as the error its inputs already carry.
//
// This is what lets the double-precision form run on a GPU whose double pipe
// issues at 1/64 of the float rate: the element arithmetic is done in double-word,
// the edge vectors x_k - x_0 in double (a handful of DADDs), and the conversions
// to and from double with integer operations only.
//
// Every step uses the round-to-nearest intrinsics so that the compiler neither
// contracts a product and a sum into one rounding nor reorders them.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace fe {

struct DW {
    float h, l;
    DW() = default;
    __host__ __device__ constexpr DW(float hh, float ll) : h(hh), l(ll) {}
    // Constants: the nearest float and the nearest float to the remainder.
    // Only for values known at compile time (a run-time double would cost
    // double-pipe conversions).
    __host__ __device__ explicit constexpr DW(double c)
        : h(static_cast<float>(c)), l(static_cast<float>(c - static_cast<double>(static_cast<float>(c)))) {}
    __host__ __device__ explicit constexpr DW(int c) : DW(static_cast<double>(c)) {}
    __device__ explicit operator float() const { return h; }
};

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ DW dw_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float ap = __fadd_rn(s, -b);
    const float bp = __fadd_rn(s, -ap);
    return {s, __fadd_rn(__fadd_rn(a, -ap), __fadd_rn(b, -bp))};
}
// s + e = a + b exactly when exponent(a) >= exponent(b) (Dekker).
__device__ __forceinline__ DW dw_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fadd_rn(b, -__fadd_rn(s, -a))};
}

__device__ __forceinline__ DW operator+(DW x, DW y) {
    const DW s = dw_two_sum(x.h, y.h);
    return dw_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ DW operator-(DW x) { return {-x.h, -x.l}; }
__device__ __forceinline__ DW operator-(DW x, DW y) { return x + (-y); }
__device__ __forceinline__ DW operator*(DW x, DW y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    return dw_fast_two_sum(p, e);
}
__device__ __forceinline__ DW &operator+=(DW &x, DW y) { return x = x + y; }
__device__ __forceinline__ DW &operator*=(DW &x, DW y) { return x = x * y; }
__device__ __forceinline__ bool operator<(DW x, DW y) { return x.h < y.h || (x.h == y.h && x.l < y.l); }

__device__ __forceinline__ DW dw_abs(DW x) { return x.h < 0.0f ? -x : x; }

// 1/x: float reciprocal r, then one Newton step r (1 + e) with e = 1 - x r
// evaluated by fused multiply-adds (1 - x_h r is exact to float precision of
// e, as x_h r is within an ulp of 1). Relative error a few 2^-48.
__device__ __forceinline__ DW dw_recip(DW x) {
    const float r = __frcp_rn(x.h);
    float e = __fmaf_rn(-x.h, r, 1.0f);
    e = __fmaf_rn(-x.l, r, e);
    return dw_fast_two_sum(r, __fmul_rn(r, e));
}

// ---------------------------------------------------------------------------
// double -> double-word with integer operations: h = x truncated to 24
// significant bits, l = the next 23 bits (relative error below 2^-47). The
// accepted magnitudes are 2^(ELO-1023) <= |x| < 2^(EHI-1022) (ELO, EHI biased
// double exponents). Zero stays zero; below the window the value becomes zero
// (FLUSH) or NaN; above it NaN, so that a value outside the window poisons the
// element's results and sends it to the double path.
// ---------------------------------------------------------------------------
template <unsigned ELO, unsigned EHI, bool FLUSH> __device__ __forceinline__ DW split_dw(double x) {
    static_assert(ELO >= 920 && EHI <= 1150 && ELO <= EHI, "window outside the float range of h and l");
    const uint32_t hw = static_cast<uint32_t>(__double2hiint(x));
    const uint32_t lw = static_cast<uint32_t>(__double2loint(x));
    const uint32_t sign = hw & 0x80000000u;
    const uint32_t e = (hw >> 20) & 0x7FFu;
    const uint32_t frac23 = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    const uint32_t elo = (e - 919u) << 23;  // float 2^(E-23)
    // 2^(E-23) (1 + next23 / 2^23) - 2^(E-23): exact (Sterbenz)
    const float lo_mag = __fadd_rn(__uint_as_float(elo | ((lw >> 6) & 0x7FFFFFu)), -__uint_as_float(elo));
    const bool in = (e - ELO) <= (EHI - ELO);
    const bool zero = FLUSH ? e < ELO : ((hw & 0x7FFFFFFFu) | lw) == 0u;
    DW r;
    r.h = in ? __uint_as_float(sign | ((e - 896u) << 23) | frac23) : (zero ? 0.0f : __uint_as_float(0x7FC00000u));
    r.l = in ? __uint_as_float(__float_as_uint(lo_mag) | sign) : 0.0f;
    return r;
}

// Windows of the double-word form. Edge components: |e| < 2^64, tiny ones
// (< 2^-100) flushed to zero. Coefficients: 2^-50 <= |c| < 2^51 or exactly 0.
constexpr unsigned kDwEdgeLo = 923, kDwEdgeHi = 1086;
constexpr unsigned kDwCoefLo = 973, kDwCoefHi = 1073;
__device__ __forceinline__ DW dw_edge(double d) { return split_dw<kDwEdgeLo, kDwEdgeHi, true>(d); }
__device__ __forceinline__ DW dw_coef(double c) { return split_dw<kDwCoefLo, kDwCoefHi, false>(c); }

// |det J| of a double-word element must lie in [2^-60, 2^60]: with the shape test
// passed this keeps every intermediate (edge products up to h^4, 1/det, the
// coefficient products) well inside the normal float range of both words.
__device__ __forceinline__ bool dw_det_ok(float det_h) {
    const float a = fabsf(det_h);
    return a >= 0x1p-60f && a <= 0x1p60f;
}

// A group of results (A^e or b^e) is accepted when all are finite and the sum of
// their magnitudes is zero or in [2^-80, 2^100], so that the low words of the
// entries that carry the group's norm are normal floats and what falls below the
// float range is negligible against the group.
template <int N> __device__ __forceinline__ float dw_abs_sum(const DW *v) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) s = __fadd_rn(s, fabsf(v[k].h));
    return s;
}
__device__ __forceinline__ bool dw_sum_ok(float s) { return s == 0.0f || (s >= 0x1p-80f && s <= 0x1p100f); }
template <int N> __device__ __forceinline__ bool dw_group_ok(const DW *v) { return dw_sum_ok(dw_abs_sum<N>(v)); }

// ---------------------------------------------------------------------------
// double-word -> double: each float becomes its exact double by re-biasing its
// bits (integer operations), and one double addition rounds h + l correctly; no
// normalisation of (h, l) is needed. Zero and subnormal floats become zero (an
// absolute error below 2^-126, negligible against a result group of at least
// 2^-80); non-finite floats are not preserved, which only matters for flagged
// elements, whose results the fix-up overwrites.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double f2d_bits(float f) {
    const uint32_t b = __float_as_uint(f);
    const bool normal = (b & 0x7F800000u) != 0u;
    const uint32_t hi = normal ? ((((b >> 3) & 0x0FFFFFFFu) + 0x38000000u) | (b & 0x80000000u)) : (b & 0x80000000u);
    const uint32_t lo = normal ? (b << 29) : 0u;
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}
__device__ __forceinline__ double dw_to_double(DW v) { return f2d_bits(v.h) + f2d_bits(v.l); }

// The same conversion with integer operations only, for kernels whose double pipe
// is the busier one: after renormalisation (|l| <= ulp(h)/2) the double of h is
// exact, and l is added as an integer count k of ulps of that double,
// k = trunc(l / ulp), |k| < 2^30 (error below one ulp of the result). When h is a
// power of two and l has the opposite sign the result lies in the binade below,
// whose ulp is half as large. Zero and subnormal h give a signed zero.
__device__ __forceinline__ double dw_to_double_int(DW v) {
    const DW n = dw_two_sum(v.h, v.l);
    const uint32_t bh = __float_as_uint(n.h), bl = __float_as_uint(n.l);
    const uint32_t eh = (bh >> 23) & 0xFFu, el = (bl >> 23) & 0xFFu;
    const uint32_t sh = bh & 0x80000000u;
    const bool nh = eh != 0u;
    const uint32_t whi = nh ? ((((bh >> 3) & 0x0FFFFFFFu) + 0x38000000u) | sh) : sh;
    const uint32_t wlo = nh ? (bh << 29) : 0u;
    const bool down = (bh & 0x7FFFFFu) == 0u && ((bl ^ bh) & 0x80000000u) != 0u;
    // biased exponent of t = l * 2^(52 - E_h), one more in the binade below
    const int te = int(el) - int(eh) + (down ? 180 : 179);
    int k = 0;
    if (el != 0u && te >= 1 && nh) k = __float2int_rz(__uint_as_float((bl & 0x807FFFFFu) | (uint32_t(te) << 23)));
    // k has l's sign; the bit pattern holds |h|, so negate for negative h
    const long long d = sh ? -static_cast<long long>(k) : static_cast<long long>(k);
    return __longlong_as_double(
        static_cast<long long>(((static_cast<unsigned long long>(whi) << 32) | wlo) + static_cast<unsigned long long>(d)));
}

// Sum of N products of double-words, accumulated as in the Dot2 algorithm of
// Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26(6), 2005): the float products
// h_i h'_i are summed with TwoSum, and their rounding errors, the TwoSum errors
// and the cross terms h_i l'_i + l_i h'_i are gathered in one float. Error a few
// N^2 2^-48 sum |x_i y_i|. SIGN[i] = -1 subtracts the i-th product.
template <int N>
__device__ __forceinline__ DW dw_dot(const DW *x, const DW *y, const int *sign = nullptr) {
    float p = __fmul_rn(x[0].h, y[0].h);
    float c = __fmaf_rn(x[0].h, y[0].h, -p);
    c = __fmaf_rn(x[0].h, y[0].l, c);
    c = __fmaf_rn(x[0].l, y[0].h, c);
    if (sign && sign[0] < 0) {
        p = -p;
        c = -c;
    }
#pragma unroll
    for (int i = 1; i < N; ++i) {
        const float xh = (sign && sign[i] < 0) ? -x[i].h : x[i].h;
        const float xl = (sign && sign[i] < 0) ? -x[i].l : x[i].l;
        const float q = __fmul_rn(xh, y[i].h);
        const float e = __fmaf_rn(xh, y[i].h, -q);
        const DW s = dw_two_sum(p, q);
        p = s.h;
        c = __fadd_rn(c, __fadd_rn(s.l, e));
        c = __fmaf_rn(xh, y[i].l, c);
        c = __fmaf_rn(xl, y[i].h, c);
    }
    return dw_fast_two_sum(p, c);
}
// z + sum of N products of double-words, the same accumulation started from z.
template <int N> __device__ __forceinline__ DW dw_dot_add(const DW *x, const DW *y, DW z) {
    float p = z.h;
    float c = z.l;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const float q = __fmul_rn(x[i].h, y[i].h);
        const float e = __fmaf_rn(x[i].h, y[i].h, -q);
        const DW s = dw_two_sum(p, q);
        p = s.h;
        c = __fadd_rn(c, __fadd_rn(s.l, e));
        c = __fmaf_rn(x[i].h, y[i].l, c);
        c = __fmaf_rn(x[i].l, y[i].h, c);
    }
    return dw_fast_two_sum(p, c);
}
// 4 q - (p1 + p2 + p3), the high words summed with TwoSum and every error and
// low word gathered in one float (4 q is exact).
__device__ __forceinline__ DW dw_lin4(DW p1, DW p2, DW p3, DW q) {
    float p = __fmul_rn(4.0f, q.h);
    float c = __fmul_rn(4.0f, q.l);
    const DW v[3] = {p1, p2, p3};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const DW s = dw_two_sum(p, -v[i].h);
        p = s.h;
        c = __fadd_rn(c, __fadd_rn(s.l, -v[i].l));
    }
    return dw_fast_two_sum(p, c);
}

// acc += x y, acc held as an unnormalised pair (p, c): p the float sum of the
// high products, c gathering the TwoSum errors, the products' rounding errors and
// the cross terms, as the Dot2 accumulation above keeps them across its terms;
// dw_acc_norm makes the pair a double-word again (after the last term).
__device__ __forceinline__ void dw_acc(DW &acc, DW x, DW y) {
    const float q = __fmul_rn(x.h, y.h);
    const float e = __fmaf_rn(x.h, y.h, -q);
    const DW s = dw_two_sum(acc.h, q);
    float c = __fadd_rn(acc.l, __fadd_rn(s.l, e));
    c = __fmaf_rn(x.h, y.l, c);
    c = __fmaf_rn(x.l, y.h, c);
    acc = DW(s.h, c);
}
// acc += x for the same unnormalised pair (the TwoSum error and x's low word
// gathered in the low word).
__device__ __forceinline__ void dw_acc_add(DW &acc, DW x) {
    const DW s = dw_two_sum(acc.h, x.h);
    acc = DW(s.h, __fadd_rn(acc.l, __fadd_rn(s.l, x.l)));
}
__device__ __forceinline__ DW dw_acc_norm(DW acc) { return dw_two_sum(acc.h, acc.l); }

// a b - c d
__device__ __forceinline__ DW dw_diff_prod(DW a, DW b, DW c, DW d) {
    const DW x[2] = {a, c}, y[2] = {b, d};
    const int sg[2] = {1, -1};
    return dw_dot<2>(x, y, sg);
}

}  // namespace fe
