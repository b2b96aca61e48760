// Double-float ("df32") arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers, which carries about 48 significant bits.
//
// Why: GB300 runs FP64 instructions (and FP64<->FP32 conversions) on a narrow
// pipe of roughly 0.5 T lane-ops/s. A CSRC product needs one multiply-add per
// stored value, which would bound an FP64 product of a 211M-nnz matrix at about
// 0.42 ms, well above its HBM time. df32 keeps the doubles in memory. It splits
// them with integer instructions, multiplies and adds on the FP32 pipes with
// error-free transformations, and rebuilds doubles with integer instructions.
//
// Published methods used:
//  - TwoSum (Knuth, TAOCP vol. 2): s = a + b, err = (a - (s - v)) + (b - v), v = s - a.
//  - FastTwoSum (Dekker 1971): s = a + b, err = b - (s - a), for |a| >= |b|.
//  - TwoProduct with FMA: p = a*b, err = fma(a, b, -p).
// Explicit _rn intrinsics keep the compiler from contracting or reassociating
// these sequences.
#pragma once

#include <cstdint>

namespace csrc {

struct df32 {
  float hi, lo;
};

// Exponent window (biased FP64 exponent) in which the df32 result keeps its ~2^-46
// relative accuracy: magnitudes in [2^-50, 2^63). Inside it, products stay above
// 2^-100, so their error terms stay normal floats, and sums stay far below the FP32
// overflow threshold.
constexpr unsigned kDfExpMin = 1023u - 50u;
constexpr unsigned kDfExpMax = 1023u + 62u;

// Split an FP64 value into hi + lo using integer instructions only.
// hi = the value truncated to 24 significant bits. lo = the next 23 bits of the
// remainder (truncated), so |d - (hi + lo)| < 2^-46 |d|.
// With CHECK, *bad is set when d is neither zero nor inside [2^-50, 2^63).
// Doubles below 2^-103 keep only hi (lo = 0); below 2^-126 they become 0;
// at or above 2^128 they become +-inf (NaN stays NaN).
template <bool CHECK>
__device__ __forceinline__ df32 df_split(double d, unsigned* bad) {
  const unsigned L = (unsigned)__double2loint(d);
  const unsigned H = (unsigned)__double2hiint(d);
  const unsigned habs = H & 0x7fffffffu;
  const unsigned sign = H & 0x80000000u;
  const unsigned E = habs >> 20;
  // hi: rebias the exponent (1023 -> 127) and keep the top 23 mantissa bits
  const unsigned hi_mag = __funnelshift_l(L, habs - 0x38000000u, 3);
  // lo: 2^(e-23) * (1 + r/2^23) - 2^(e-23) = r * 2^(e-46), r = mantissa bits 28..6
  const unsigned base = (hi_mag & 0x7f800000u) - (23u << 23);
  const unsigned f1 = base | ((L >> 6) & 0x7fffffu);
  const float lo_mag = __fsub_rn(__uint_as_float(f1), __uint_as_float(base));
  df32 r;
  r.hi = __uint_as_float(hi_mag | sign);
  r.lo = __uint_as_float(__float_as_uint(lo_mag) | sign);
  if (CHECK) {
    if (E - kDfExpMin > kDfExpMax - kDfExpMin && (habs | L) != 0u) *bad = 1u;
  }
  if (E - 920u > 230u) {  // outside the exponents handled above (rare)
    if (E >= 897u && E < 920u) {
      r.lo = 0.0f;
    } else if (E < 897u) {
      r.hi = __uint_as_float(sign);
      r.lo = 0.0f;
    } else {
      const bool nan = (E == 2047u) && (((habs & 0xfffffu) | L) != 0u);
      r.hi = __uint_as_float(sign | (nan ? 0x7fc00000u : 0x7f800000u));
      r.lo = 0.0f;
    }
  }
  return r;
}

// (ah + al) * (bh + bl) ~= ph + pl (the al*bl term, < 2^-48 relative, is dropped).
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
  df32 p;
  p.hi = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p.hi);
  e = __fmaf_rn(a.hi, b.lo, e);
  p.lo = __fmaf_rn(a.lo, b.hi, e);
  return p;
}

// s += p with a renormalised result (TwoSum of the high parts, then FastTwoSum).
__device__ __forceinline__ void df_acc(df32& s, df32 p) {
  const float t = __fadd_rn(s.hi, p.hi);
  const float v = __fsub_rn(t, s.hi);
  float e = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, v)), __fsub_rn(p.hi, v));
  e = __fadd_rn(e, __fadd_rn(s.lo, p.lo));
  s.hi = __fadd_rn(t, e);
  s.lo = __fsub_rn(e, __fsub_rn(s.hi, t));
}

// s += p for a short run of terms (a thread's few pairs of one row): TwoSum of the
// high parts, error and low parts summed into s.lo without renormalising. The
// atomic flush that follows renormalises the high word.
__device__ __forceinline__ void df_acc_short(df32& s, df32 p) {
  const float t = __fadd_rn(s.hi, p.hi);
  const float v = __fsub_rn(t, s.hi);
  const float e = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, v)), __fsub_rn(p.hi, v));
  s.lo = __fadd_rn(s.lo, __fadd_rn(e, p.lo));
  s.hi = t;
}

// Error-compensated atomic accumulation of p into the pair of FP32 cells (*whi, *wlo).
// The atomic returns the old high word, so the rounding error of the high-word
// addition is recovered exactly (TwoSum) and sent to the low word with p.lo.
__device__ __forceinline__ void df_atomic_add(float* whi, float* wlo, df32 p) {
  const float old = atomicAdd(whi, p.hi);
  const float t = __fadd_rn(old, p.hi);
  const float v = __fsub_rn(t, old);
  const float e = __fadd_rn(__fsub_rn(old, __fsub_rn(t, v)), __fsub_rn(p.hi, v));
  atomicAdd(wlo, __fadd_rn(e, p.lo));
}

// Round hi + lo to a double using integer instructions (the common path).
// The FP32 pair is first renormalised (FastTwoSum). The low part is then
// aligned to the high part's 53-bit significand: bits below it are truncated,
// so the error is below one double ulp.
__device__ __forceinline__ double df_to_f64(df32 v) {
  float a = v.hi, b = v.lo;
  if (fabsf(a) < fabsf(b)) {
    const float t = a;
    a = b;
    b = t;
  }
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  const unsigned hb = __float_as_uint(s);
  const unsigned lb = __float_as_uint(e);
  const unsigned eh = (hb >> 23) & 0xffu;
  if (eh == 0u || eh == 0xffu) {
    // zero, subnormal, inf or NaN high part: rare; the slow pipe is fine here
    return (double)s + (double)e;
  }
  long long M = (long long)((hb & 0x7fffffu) | 0x800000u) << 29;  // in [2^52, 2^53)
  if ((lb & 0x7fffffffu) != 0u) {
    unsigned el = (lb >> 23) & 0xffu;
    unsigned ml = lb & 0x7fffffu;
    if (el == 0u) {
      el = 1u;  // subnormal low part
    } else {
      ml |= 0x800000u;
    }
    const int sh = (int)el - (int)eh + 29;  // low part in units of the double's last place
    long long lp = 0;
    if (sh >= 0) {
      lp = (long long)ml << sh;
    } else if (sh > -30) {
      lp = (long long)(ml >> (-sh));
    }
    M = ((hb ^ lb) & 0x80000000u) ? M - lp : M + lp;
  }
  int ex = (int)eh + 896;
  if (M >= (1LL << 53)) {
    M >>= 1;
    ++ex;
  } else if (M < (1LL << 52)) {
    M <<= 1;
    --ex;
  }
  const unsigned long long bits = ((unsigned long long)(hb >> 31) << 63) | ((unsigned long long)ex << 52) |
                                  ((unsigned long long)M & ((1ULL << 52) - 1ULL));
  return __longlong_as_double((long long)bits);
}

}  // namespace csrc
