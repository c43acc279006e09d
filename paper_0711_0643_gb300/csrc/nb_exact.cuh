// Exact FP64 helpers for the step kernels. On this GPU an FP64 warp instruction
// occupies the SM sub-partition's FP64 unit for ~70 clocks whatever the number
// of active lanes, an IEEE FP64 division or square root costs ~10 of them, and
// so does nothing else in the step kernels. Every helper here returns exactly
// the bits of the plain IEEE expression it replaces (stated with each one),
// using fewer FP64 instructions or none.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

namespace nb {

__host__ __device__ __forceinline__ long long dbits(double x)
{
#ifdef __CUDA_ARCH__
    return __double_as_longlong(x);
#else
    long long b;
    std::memcpy(&b, &x, 8);
    return b;
#endif
}
__host__ __device__ __forceinline__ double dfrom(long long b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double x;
    std::memcpy(&x, &b, 8);
    return x;
#endif
}
__host__ __device__ __forceinline__ float ffrom(unsigned u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float x;
    std::memcpy(&x, &u, 4);
    return x;
#endif
}
__host__ __device__ __forceinline__ int fbits(float x)
{
#ifdef __CUDA_ARCH__
    return __float_as_int(x);
#else
    int b;
    std::memcpy(&b, &x, 4);
    return b;
#endif
}
__host__ __device__ __forceinline__ int clz32(unsigned u)
{
#ifdef __CUDA_ARCH__
    return __clz((int)u);
#else
    return u ? __builtin_clz(u) : 32;
#endif
}
__host__ __device__ __forceinline__ int dexpo(double x) { return (int)((dbits(x) >> 52) & 0x7ff); }

// Finite (not inf or NaN), from the exponent field alone.
__device__ __forceinline__ bool dfinite(double x) { return dexpo(x) != 0x7ff; }

// The IEEE product x * p for p = 2^e, on the integer pipe: exact exponent shift
// when x is normal and the product stays normal, zeros keep their sign; any
// other case (subnormal, inf, NaN, under/overflow) takes the FP64 multiply out
// of line (a call, so the compiler cannot predicate it into the common path).
static __device__ __noinline__ double dmul_slow(double x, double p) { return __dmul_rn(x, p); }
__host__ __device__ __forceinline__ bool scale2_fast(long long xb, int e)
{
    const int ex = (int)((xb >> 52) & 0x7ff);
    return ex != 0 && ex != 0x7ff && ex + e > 0 && ex + e < 0x7ff;
}
__device__ __forceinline__ double scale2(double x, int e, double p)
{
    const long long xb = dbits(x);
    if (scale2_fast(xb, e)) return dfrom(xb + ((long long)e << 52));
    if ((xb & 0x7FFFFFFFFFFFFFFFll) == 0) return x;
    return dmul_slow(x, p);
}

// Double-single split (hi, lo) = (RN32(x), RN32(x - RN32(x))) on the integer
// pipe, for |x| in [2^-60, 2^100] (both parts then normal floats); returns
// false otherwise and the caller converts with the FP64 unit. hi rounds the
// 52-bit significand to 23 bits, ties to even; x - hi is the exact remainder
// (at most 29 bits, sign flipped when hi rounded up in magnitude), rounded to
// 24 bits the same way.
__host__ __device__ __forceinline__ bool ds_split_int(double x, unsigned &hi, unsigned &lo)
{
    const long long xb = dbits(x);
    const int E = (int)((xb >> 52) & 0x7ff);
    if (E < 1023 - 60 || E > 1023 + 100) return false;
    const unsigned sign = (unsigned)((unsigned long long)xb >> 63) << 31;
    const unsigned long long M = (unsigned long long)xb & ((1ull << 52) - 1);
    unsigned mh = (unsigned)(M >> 29);
    const unsigned rem = (unsigned)(M & ((1u << 29) - 1));
    const bool up = rem > (1u << 28) || (rem == (1u << 28) && (mh & 1u));
    int Eh = E;
    if (up && ++mh == (1u << 23)) {
        mh = 0;
        ++Eh;
    }
    hi = sign | ((unsigned)(Eh - 896) << 23) | mh;
    // remainder x - hi = +-L * 2^(E - 1075), L < 2^29
    const unsigned L = up ? (1u << 29) - rem : rem;
    if (L == 0) {
        lo = 0u;
        return true;
    }
    const unsigned lsign = up ? (sign ^ 0x80000000u) : sign;
    const int p = 31 - clz32(L);           // top bit of L
    int el = E - 1075 + p + 127;           // biased float exponent of the leading bit
    unsigned ml;
    if (p <= 23) {
        ml = L << (23 - p);
    } else {
        const int sh = p - 23;
        ml = L >> sh;
        const unsigned r = L & ((1u << sh) - 1u), half = 1u << (sh - 1);
        if (r > half || (r == half && (ml & 1u))) {
            if (++ml == (1u << 24)) {
                ml = 1u << 23;
                ++el;
            }
        }
    }
    lo = lsign | ((unsigned)el << 23) | (ml & 0x7fffffu);
    return true;
}

// y / full, correctly rounded, where full = d * scale^-1 with scale a power of two
// and c = RN(1/d). Markstein's theorem (IBM J. Res. Dev. 34, 1990): if c is within
// half an ulp of 1/d and q within one ulp of y/d, the residual r = y - q d is exact
// (one fused multiply-add) and RN(q + r c) = RN(y/d). q = RN(y c) is within one ulp
// for d = 3 (RN(1/3) is off by at most 2^-54 relative, under half an ulp). Scaling
// by a power of two is exact while the result stays normal, which the exponent
// window [63, 2023] of y guarantees; outside it the IEEE division is used. (The
// FP64 predictor's k d^3 / 6; the corrector uses the integer div3_int below.)
__device__ __forceinline__ double div_const(double y, double d, double c, double scale, double full)
{
    const int e = dexpo(y);
    if (e >= 63 && e <= 2023) {
        const double q = y * c;
        const double r = fma(-q, d, y);
        return fma(r, c, q) * scale;
    }
    return y / full;
}
__device__ __forceinline__ double div6(double y) { return div_const(y, 3.0, 1.0 / 3.0, 0.5, 6.0); }

// High 64 bits of the 128-bit product a b.
__host__ __device__ __forceinline__ unsigned long long umulhi64(unsigned long long a, unsigned long long b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (unsigned long long)(((unsigned __int128)a * b) >> 64);
#endif
}

// Correctly rounded y / 3 * 2^-s (s = 1: y / 6, s = 3: y / 24) and y / 15 * 2^-s
// (s = 3: y / 120) on the integer pipe; false when the biased exponent E of y is
// outside [64, 2046] (zero, subnormal, inf, NaN and huge values: the caller
// divides in FP64). With y = +-M 2^(E - 1075), M in [2^52, 2^53), N = M 2^k puts
// N / d in [2^52, 2^53); Q = floor(N / d) is a multiply-high by m = ceil(2^(64+l)
// / d) and a shift by l (Granlund and Montgomery, "Division by invariant integers
// using multiplication", PLDI 1994: m d - 2^(64+l) <= 2^l holds, 1 for d = 3,
// l = 1 and 7 for d = 15, l = 3). The exact quotient is Q + R / d with R = N - d Q;
// rounding to nearest takes Q + 1 when R / d > 1/2 (R / d = 1/2 is impossible for
// odd d), and Q + 1 < 2^53 always.
__host__ __device__ __forceinline__ bool div3_int(double y, int s, double &out)
{
    const long long yb = dbits(y);
    const int E = (int)((yb >> 52) & 0x7ff);
    if (E < 64 || E > 2046) return false;
    const unsigned long long M = ((unsigned long long)yb & ((1ull << 52) - 1)) | (1ull << 52);
    const int k = M >= (3ull << 51) ? 1 : 2;
    const unsigned long long N = M << k;
    const unsigned long long Q = umulhi64(N, 0xAAAAAAAAAAAAAAABull) >> 1;
    const unsigned long long Qr = Q + ((N - 3 * Q) == 2 ? 1 : 0);
    out = dfrom((long long)((unsigned long long)yb & 0x8000000000000000ull) | ((long long)(E - k - s) << 52) |
                (long long)(Qr - (1ull << 52)));
    return true;
}
__host__ __device__ __forceinline__ bool div15_int(double y, int s, double &out)
{
    const long long yb = dbits(y);
    const int E = (int)((yb >> 52) & 0x7ff);
    if (E < 64 || E > 2046) return false;
    const unsigned long long M = ((unsigned long long)yb & ((1ull << 52) - 1)) | (1ull << 52);
    const int k = M >= (15ull << 49) ? 3 : 4;
    const unsigned long long N = M << k;
    const unsigned long long Q = umulhi64(N, 0x8888888888888889ull) >> 3;
    const unsigned long long Qr = Q + ((N - 15 * Q) >= 8 ? 1 : 0);
    out = dfrom((long long)((unsigned long long)yb & 0x8000000000000000ull) | ((long long)(E - k - s) << 52) |
                (long long)(Qr - (1ull << 52)));
    return true;
}

// Correctly rounded 3 y 2^s (0 <= s <= 3) on the integer pipe, ties to even;
// false outside biased exponents [1, 2040] of y. P = 3 M has 54 or 55 bits; the
// low sh = 1 or 2 bits are rounded off and a carry to 2^53 renormalises.
__host__ __device__ __forceinline__ bool mul3_int(double y, int s, double &out)
{
    const long long yb = dbits(y);
    const int E = (int)((yb >> 52) & 0x7ff);
    if (E < 1 || E > 2040) return false;
    const unsigned long long M = ((unsigned long long)yb & ((1ull << 52) - 1)) | (1ull << 52);
    const unsigned long long P = 3 * M;
    const int sh = P >= (1ull << 54) ? 2 : 1;
    unsigned long long q = P >> sh;
    const unsigned long long r = P & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    q += (r > half || (r == half && (q & 1))) ? 1 : 0;
    int Eo = E + sh + s;
    if (q == (1ull << 53)) {
        q >>= 1;
        ++Eo;
    }
    out = dfrom((long long)((unsigned long long)yb & 0x8000000000000000ull) | ((long long)Eo << 52) |
                (long long)(q - (1ull << 52)));
    return true;
}

// 1/p for a power of two p whose reciprocal is normal (biased exponent of p in
// [1, 2045]): the exponent field reflected about the bias, no FP64 instruction.
__host__ __device__ __forceinline__ double recip_pow2(double p) { return dfrom((0x7FEll << 52) - dbits(p)); }

// Bits of the largest power of two <= cand for cand > 0 finite and normal,
// +inf for +inf, 0 for subnormal cand (frexp/ldexp's answer is then below any
// normal step bound, which is all the quantisation rule looks at).
// RN32(x), ties to even, on the integer pipe, for |x| < 2^60; values whose
// float would be subnormal give 0 (as a flush-to-zero FP32 unit would). False
// for |x| >= 2^60, infinities and NaN.
__host__ __device__ __forceinline__ bool rn32_int(double x, float &f)
{
    const long long xb = dbits(x);
    const int E = (int)((xb >> 52) & 0x7ff);
    if (E >= 1023 + 60) return false;
    if (E < 1023 - 126) {
        f = 0.f;
        return true;
    }
    const unsigned sign = (unsigned)((unsigned long long)xb >> 63) << 31;
    const unsigned long long M = (unsigned long long)xb & ((1ull << 52) - 1);
    unsigned mh = (unsigned)(M >> 29);
    const unsigned rem = (unsigned)(M & ((1u << 29) - 1));
    const bool up = rem > (1u << 28) || (rem == (1u << 28) && (mh & 1u));
    int Eh = E;
    if (up && ++mh == (1u << 23)) {
        mh = 0;
        ++Eh;
    }
    f = ffrom(sign | ((unsigned)(Eh - 896) << 23) | mh);
    return true;
}

// f^2 in FP32, flushed to 0 below 2^-126 (a flush-to-zero unit's result). The
// corrector's step estimate sums three of these in the oracle's order (x^2 +
// y^2) + z^2 from RN32 copies of FP64 components; the sum counts as in range in
// [2^-100, 2^120], where a flushed square changes it by under 2^-26 relative.
__host__ __device__ __forceinline__ float sq_ftz(float f)
{
    const float q = f * f;
    return q < 1.17549435e-38f ? 0.f : q;
}
__host__ __device__ __forceinline__ bool norm2_f32_in_range(float S)
{
    return S >= 7.88860905e-31f && S <= 1.32922800e+36f;   // 2^-100, 2^120
}

__host__ __device__ __forceinline__ long long pow2_floor_bits(double cand)
{
    return dbits(cand) & (long long)0xFFF0000000000000ull;
}

// cand > 0 (false for NaN, zeros and negatives), on the integer pipe.
__host__ __device__ __forceinline__ bool dpositive(double cand)
{
    const long long b = dbits(cand);
    return b > 0 && b <= 0x7FF0000000000000ll;
}

// 1 + index of the lowest set bit of m (0 for m = 0).
__host__ __device__ __forceinline__ int ffs64(long long m)
{
#ifdef __CUDA_ARCH__
    return __ffsll(m);
#else
    return __builtin_ffsll(m);
#endif
}

// Is t an integer multiple of the power of two p (p normal)? Equal to
// u = t / p; u == floor(u) in IEEE arithmetic for finite t.
__host__ __device__ __forceinline__ bool multiple_of_pow2(double t, double p)
{
    const long long tb = dbits(t) & 0x7FFFFFFFFFFFFFFFll;
    if (tb == 0) return true;
    const int et = (int)(tb >> 52);
    const long long m = (tb & ((1ll << 52) - 1)) | (et ? (1ll << 52) : 0ll);
    const int low = (et ? et : 1) - 1075 + (ffs64(m) - 1);   // exponent of t's lowest set bit
    return low >= (int)(dbits(p) >> 52) - 1023;
}

// The power-of-two step rule of the quantiser on bit patterns (all operands are
// non-negative doubles, whose bit patterns order like their values): drop to q
// when q < dt_old, double (once) when q >= 2 dt_old, 2 dt_old <= dt_max and
// t_new is a multiple of 2 dt_old, else keep; clamp to dt_max; 0 below dt_min.
// qb = pow2_floor_bits(cand); pos = dpositive(cand). dt_old in [2^-300, 2^300].
__host__ __device__ __forceinline__ double quantise_bits(long long qb, bool pos, double dt_old, double t_new,
                                                         double dt_max, double dt_min)
{
    if (!pos) return 0.0;
    const long long dto = dbits(dt_old), dt2 = dto + (1ll << 52), dmax = dbits(dt_max), dmin = dbits(dt_min);
    long long dt;
    if (qb < dto) {
        dt = qb;
    } else if (qb >= dt2 && dt2 <= dmax) {
        dt = multiple_of_pow2(t_new, dfrom(dt2)) ? dt2 : dto;
    } else {
        dt = dto;
    }
    if (dt > dmax) dt = dmax;
    if (dt < dmin) return 0.0;
    return dfrom(dt);
}

}  // namespace nb
