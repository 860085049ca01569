// md_device.cuh -- small device helpers of libmd.so (sm_103a).
//
// GB300 runs FP64 at ~1/64 of the FP32 rate (measured: DFMA ~600 Gop/s,
// DADD/DMUL/DSETP and FP32<->FP64 conversions ~500-600 Gop/s for the whole
// GPU), so the helpers below keep the FP64 pipe for arithmetic that must be
// FP64 and do comparisons and conversions with integer instructions where
// that is exact.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "md_internal.cuh"

// |d| > h for a finite double d and a positive double h, as an integer
// compare of the bit patterns (IEEE doubles of one sign order like their
// bit patterns).  Avoids a DSETP on the FP64 pipe.
__device__ __forceinline__ bool md_abs_gt(double d, long long h_bits) {
  return (__double_as_longlong(d) & 0x7fffffffffffffffLL) > h_bits;
}

// r2 < c for r2 >= 0 and c > 0 by bit patterns (same ordering argument).
__device__ __forceinline__ bool md_lt_pos(double r2, long long c_bits) {
  return __double_as_longlong(r2) < c_bits;
}

// -x by flipping the sign bit with an integer instruction (off the FP64 pipe).
__device__ __forceinline__ double md_neg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}

// Minimum-image component: d - L*rint(d/L) for |d| < 3L/2, written as a
// conditional subtraction of +-L.  Identical to the rint form except when
// |d| is within one ulp of L/2, where either image is at distance L/2.
__device__ __forceinline__ double md_min_image(double d, double L, long long halfL_bits) {
  if (md_abs_gt(d, halfL_bits)) d = __dsub_rn(d, copysign(L, d));
  return d;
}

// Squared length with the fixed rounding order fma(dz,dz, fma(dy,dy, dx*dx)).
__device__ __forceinline__ double md_r2(double dx, double dy, double dz) {
  return __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
}

// Reciprocal 1/a for a > 0 in FP64: a hardware seed y0 (rcp.approx.ftz.f64,
// about 20 correct bits, off the FP64 pipe) refined with the cubic series
// 1/a = y0 / (1 - e) ~ y0 (1 + e + e^2), e = 1 - a y0, whose relative error
// is e^3 (Newton-Raphson and series refinement of reciprocals: Markstein,
// IBM J. Res. Dev. 34 (1990) 111).  Three FMAs on the FP64 pipe; the result
// is within a few ulps of the correctly rounded reciprocal.
__device__ __forceinline__ double md_rcp(double a) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
  const double e = __fma_rn(-a, y, 1.0);
  return __fma_rn(y, __fma_rn(e, e, e), y);
}

// 1/sqrt(a) for a > 0 in FP64: the rsqrt.approx.ftz.f64 seed y0 refined by
// the series (1 - e)^(-1/2) ~ 1 + e/2 + 3e^2/8 with e = 1 - a y0^2, whose
// relative error is O(e^3).  The seed has about 20 correct bits and one
// round leaves the result within 1 ulp of the correctly rounded value (the
// ulp test of md_eval_recip): five FP64-pipe operations.
__device__ __forceinline__ double md_rsqrt(double a) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
  const double e = __fma_rn(-a, y * y, 1.0);
  return __fma_rn(y * e, __fma_rn(0.375, e, 0.5), y);
}

// Owner of the unordered pair {i, j} in the half list: i owns it iff
// (i < j) equals (i + j even).  Each atom owns about half of its neighbors
// wherever it sits in the sorted order, so per-atom counts stay balanced
// (an index-ordered rule j > i gives counts from 0 to the full count).
__device__ __forceinline__ bool md_owns(int i, int j) {
  return (i < j) == (((i + j) & 1) == 0);
}

// Exact widening of a float to double with integer instructions (no FP64
// pipe).  Subnormal floats (|x| < 2^-126) become signed zero, which is the
// flush-to-zero convention of the FP32 arithmetic they come from.
__device__ __forceinline__ double md_widen(float x) {
  unsigned int u = __float_as_uint(x);
  unsigned long long s = (unsigned long long)(u >> 31) << 63;
  unsigned int e = (u >> 23) & 0xffu;
  if (e == 0) return __longlong_as_double((long long)s);
  unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
  unsigned long long de = (unsigned long long)(e == 0xffu ? 0x7ffu : e + 896u) << 52;
  return __longlong_as_double((long long)(s | de | m));
}

// Fixed-point force accumulators: a force component is held as a signed
// 64-bit integer count of 2^-MD_FIX_BITS units, so that sums of
// contributions are exact and independent of their order.  On GB300 integer
// atomics in shared memory run at ~5 per clock per SM, while FP64 ones go
// through the FP64 pipe (~1.6 per clock per SM) that the pair arithmetic
// needs; in global memory (L2) both kinds run off the SM's pipes.
#define MD_FIX_BITS 44
// Largest binary exponent e of a contribution 2^e <= |g| that may go to a
// fixed-point accumulator: |g| < 2^(MD_FIX_EMAX + 1) keeps the conversion a
// right shift.
#define MD_FIX_EMAX 7

// g rounded to the nearest multiple of 2^-MD_FIX_BITS (halves away from
// zero), as an integer count, using integer instructions only.  Returns
// false, leaving q unset, when the biased exponent of g is >= ex_lim (the
// caller's range limit, <= 1023 + MD_FIX_EMAX + 1; infinities and NaNs
// always fail).  Zeros and subnormals give 0.
__device__ __forceinline__ bool md_fix(double g, int ex_lim, long long& q) {
  const long long b = __double_as_longlong(g);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex >= ex_lim) return false;
  // |g| = m 2^(ex - 1075) with m = 2^52 + fraction (ex > 0), so the count is
  // m 2^(ex - 1075 + MD_FIX_BITS) = m >> sh, sh >= 1
  const int sh = 1075 - MD_FIX_BITS - ex;
  const unsigned long long m = ((unsigned long long)b & 0xfffffffffffffULL) | (1ULL << 52);
  const unsigned long long r = sh > 54 ? 0ULL : (m + (1ULL << (sh - 1))) >> sh;
  q = b < 0 ? -(long long)r : (long long)r;
  return true;
}

// An FP32 contribution g as a fixed-point count of 2^-MD_FIX_BITS units,
// with integer instructions only (the mixed form's force sums), for
// |g| < 2^(MD_FIX_EMAX + 1) (md_fix32_fits).  Every FP32 value with
// |g| >= 2^-21 is an exact multiple of 2^-44, so the count is exact there;
// smaller values are rounded toward minus infinity (error below 2^-44).
// |g| = m 2^(ex - 150) with m = 2^23 + fraction, so the count is
// m 2^(ex - 106) = (m << 28) >> (134 - ex): the sign goes onto m before the
// arithmetic right shift, and shr.s64 clamps shifts beyond 63 (|g| < 2^-56,
// and zeros and subnormals, whose exponent field is 0) to a sign fill, 0 or
// -1.
__device__ __forceinline__ long long md_fix32(float g) {
  static_assert(MD_FIX_BITS == 44 && MD_FIX_EMAX == 7, "shift constants below");
  const unsigned int b = __float_as_uint(g);
  const int m = (int)((b & 0x7fffffu) | 0x800000u);
  const int sg = (int)b >> 31;  // 0 or -1
  const long long ms = (long long)((m ^ sg) - sg) << 28;
  const unsigned int sh = 134u - ((b >> 23) & 0xffu);
  long long q;
  asm("shr.s64 %0, %1, %2;" : "=l"(q) : "l"(ms), "r"(sh));
  return q;
}

// All three FP32 contributions are below 2^(ex_lim - 127) in magnitude
// (ex_lim <= 127 + MD_FIX_EMAX + 1), so that md_fix32 applies; false for
// infinities and NaNs.
__device__ __forceinline__ bool md_fix32_fits(float gx, float gy, float gz, int ex_lim) {
  const unsigned int e = max(__float_as_uint(gx) & 0x7f800000u,
                             max(__float_as_uint(gy) & 0x7f800000u,
                                 __float_as_uint(gz) & 0x7f800000u));
  return e < ((unsigned int)ex_lim << 23);
}

// The value q * 2^-MD_FIX_BITS of a fixed-point count, exactly.  For
// |q| < 2^51 the double is assembled with integer instructions: |q| =
// 1.m * 2^p (p = 63 - clz), so the exponent field is p - 44 + 1023 and the
// mantissa the bits below the leading one, which fit in 52 bits whole.
// Larger counts take the conversion.
__device__ __forceinline__ double md_fold(long long q) {
  static_assert(MD_FIX_BITS == 44, "md_fold's exponent bias assumes 2^-44");
  if (q > -(1LL << 51) && q < (1LL << 51)) {
    if (q == 0) return 0.0;
    const unsigned long long sign = (unsigned long long)q & 0x8000000000000000ULL;
    const unsigned long long m = (unsigned long long)(q < 0 ? -q : q);
    const int lz = __clzll((long long)m);  // 13 .. 63
    const unsigned long long e = (unsigned long long)(63 - lz - MD_FIX_BITS + 1023);
    const unsigned long long mant = ((m << lz) << 1) >> 12;  // leading one shifted out
    return __longlong_as_double((long long)(sign | (e << 52) | mant));
  }
  return __dmul_rn(__ll2double_rn(q), 0x1p-44);
}

// f + the fixed-point count q (f + q 2^-44 rounded once); f is almost
// always +0 (it holds only contributions beyond the accumulators' range),
// and then the sum is the count's value itself with no FP64 operation.
__device__ __forceinline__ double md_fold_add(double f, long long q) {
  const double u = md_fold(q);
  return __double_as_longlong(f) == 0 ? u : __dadd_rn(f, u);
}

// Error-free sum (Knuth, TAOCP vol. 2, 4.2.2, "TwoSum"): s + err == a + b
// exactly, with s = fl(a + b).  Six FP32 additions.
__device__ __forceinline__ void md_two_sum(float a, float b, float& s, float& err) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float aa = __fsub_rn(s, bb);
  err = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}

// Accumulate term into the double-float accumulator (hi, lo).
__device__ __forceinline__ void md_acc2(float& hi, float& lo, float term) {
  float s, e;
  md_two_sum(hi, term, s, e);
  hi = s;
  lo = __fadd_rn(lo, e);
}

// Split of a position: hi = x rounded to the nearest multiple of the grid
// step 2^g.k, with every |x| < 2^24 2^g.k, and lo = fl32(x - hi)
// (|lo| <= 2^(g.k - 1)).  Differences of hi parts, and their shifts by the
// box edge (an FP32 value below 2^24 2^g.k, so on the same grid or a finer
// one), are then exact in FP32 whatever the coordinates' size: d = (hi_j -
// hi_i) + (lo_j - lo_i) keeps FP32's relative precision also for pairs
// across the periodic boundary (XGrid).
__device__ __forceinline__ float md_split_hi(double x, const XGrid& g) {
  // x = M 2^(e - 1075) (M the 53-bit significand): dropping the d = k + 1075
  // - e low bits of M, rounded to nearest (ties away from zero), leaves a
  // multiple of 2^k.  Integer operations on the bit pattern: the FP64 pipe
  // is the scarce one on this part.
  const long long b = __double_as_longlong(x);
  const long long sign = b & (long long)0x8000000000000000ULL;
  const int d = g.k + 1075 - (int)((b >> 52) & 0x7ff);
  long long h;
  if (d <= 0) {
    h = b;  // already on the grid
  } else if (d <= 52) {
    const long long r = 1LL << (d - 1);
    h = (b + r) & ~((r << 1) - 1);  // a carry into the exponent is the right value
  } else {
    h = d == 53 ? (sign | ((long long)(g.k + 1023) << 52)) : sign;  // +-2^k or +-0
  }
  // the FP32 pattern of h: exact while h has <= 24 significant bits (|x| <
  // 2^24 2^k); otherwise truncated, and lo takes the rest all the same
  const int eh = (int)((h >> 52) & 0x7ff);
  const unsigned int fb =
      eh == 0 ? 0u : ((unsigned int)(eh - 1023 + 127) << 23) | (unsigned int)((h >> 29) & 0x7fffff);
  return __uint_as_float((unsigned int)((unsigned long long)sign >> 32) | fb);
}
__device__ __forceinline__ void md_split(double x, const XGrid& g, float& hi, float& lo) {
  hi = md_split_hi(x, g);
  lo = __double2float_rn(__dsub_rn(x, md_widen(hi)));
}

// x as a fixed-point count X = x 2^F when that is exact and |x| < 2^(61 - F)
// (so |X| < 2^61); false otherwise.  Integer instructions only.  x = M
// 2^(e - 1075) with M the 53-bit significand: X = M 2^(e - 1075 + F), an
// integer iff e - 1075 + F >= 0 or the low 1075 - F - e bits of M are zero.
__device__ __forceinline__ bool md_xfix(double x, int F, long long& X) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) {  // zero (subnormals are never positions)
    X = 0;
    return (b & 0x7fffffffffffffffLL) == 0;
  }
  if (e - 1023 >= 61 - F) return false;  // |x| >= 2^(61 - F)
  const long long M = (b & 0xfffffffffffffLL) | (1LL << 52);
  const int sh = 1075 - F - e;
  long long m;
  if (sh <= 0) {
    m = M << (-sh);  // -sh <= 8: |x| < 2^(61 - F)
  } else {
    if (sh > 52 || (M & ((1LL << sh) - 1)) != 0) return false;
    m = M >> sh;
  }
  X = b < 0 ? -m : m;
  return true;
}

// Store the position p of atom i into its derived records: the double-float
// split (md_split; tag in hi.w) and, where xq is given (FP64 contexts), the
// fixed-point record, with MD_TAG_OFFGRID in the split's tag when some
// coordinate has no exact fixed-point form.  FP64 contexts keep only the hi
// parts of the split (lo = 0).  Returns the split.
__device__ __forceinline__ XSplit md_store_pos(const double4_32a& p, const XGrid& gr,
                                               XSplit* __restrict__ xs, XFix* __restrict__ xq,
                                               int64_t i, XSplit* __restrict__ xb = nullptr);

__device__ __forceinline__ int md_tag_of(const double4_32a& p) {
  return (int)__double_as_longlong(p.w);
}
__device__ __forceinline__ int md_type_of(const double4_32a& p) {
  return MD_TAG_TYPE(md_tag_of(p));
}
__device__ __forceinline__ double md_tag_bits(int tag) {
  return __longlong_as_double((long long)tag);
}

// 32-byte vector load through the read-only path (one sector).
__device__ __forceinline__ double4_32a md_ld4(const double4_32a* p) {
  double4_32a r;
  asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
      : "=d"(r.x), "=d"(r.y), "=d"(r.z), "=d"(r.w)
      : "l"(p));
  return r;
}

__device__ __forceinline__ XFix md_ld_xfix(const XFix* p) {
  XFix r;
  asm("ld.global.nc.v4.s64 {%0, %1, %2, %3}, [%4];"
      : "=l"(r.x), "=l"(r.y), "=l"(r.z), "=l"(r.w)
      : "l"(p));
  return r;
}

__device__ __forceinline__ XSplit md_ld_split(const XSplit* p) {
  XSplit r;
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(r.hi.x), "=f"(r.hi.y), "=f"(r.hi.z), "=f"(r.hi.w), "=f"(r.lo.x),
        "=f"(r.lo.y), "=f"(r.lo.z), "=f"(r.lo.w)
      : "l"(p));
  return r;
}

__device__ __forceinline__ XSplit md_store_pos(const double4_32a& p, const XGrid& gr,
                                               XSplit* __restrict__ xs, XFix* __restrict__ xq,
                                               int64_t i, XSplit* __restrict__ xb) {
  XSplit s;
  if (xq) {  // FP64 contexts read only the hi parts: no FP64 operation here
    s.hi.x = md_split_hi(p.x, gr);
    s.hi.y = md_split_hi(p.y, gr);
    s.hi.z = md_split_hi(p.z, gr);
    s.lo = make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    md_split(p.x, gr, s.hi.x, s.lo.x);
    md_split(p.y, gr, s.hi.y, s.lo.y);
    md_split(p.z, gr, s.hi.z, s.lo.z);
  }
  const int tag = md_tag_of(p);
  int stag = tag;
  if (xq) {  // FP64 contexts: the compacted kernel's fixed-point record
    XFix q;
    const int F = gr.rep[MD_TAG_REP(tag)].xfix;
    const bool on = md_xfix(p.x, F, q.x) & md_xfix(p.y, F, q.y) & md_xfix(p.z, F, q.z);
    q.w = (long long)(unsigned int)tag | ((long long)F << 32);
    xq[i] = q;
    if (!on) stag |= MD_TAG_OFFGRID;
  }
  s.hi.w = __int_as_float(stag);
  s.lo.w = 0.f;
  xs[i] = s;
  if (xb) xb[i] = s;
  return s;
}

// |x - x_build|^2 from the splits of the current and the build positions
// (FP32).  With both parts (mixed contexts) d = (hi - hi_b) + (lo - lo_b) is
// within ~1e-6 relative of the exact displacement.  With hi parts only (FP64
// contexts, lo = 0) each component of hi - hi_b is within one grid step 2^k
// of the exact one (each hi is within 2^(k-1) of its x), so the value
// returned is an upper bound: (|hi - hi_b| (1 + 2^-20) + 4 2^k)^2.
__device__ __forceinline__ float md_disp2(const XSplit& s, const XSplit& b, const XGrid& gr,
                                          bool hi_only) {
  const float dx = (s.hi.x - b.hi.x) + (s.lo.x - b.lo.x);
  const float dy = (s.hi.y - b.hi.y) + (s.lo.y - b.lo.y);
  const float dz = (s.hi.z - b.hi.z) + (s.lo.z - b.lo.z);
  const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
  if (!hi_only) return d2;
  const float step = __int_as_float((gr.k + 127) << 23);  // 2^k
  const float d = __fmaf_rn(sqrtf(d2), 1.f + 0x1p-20f, 4.f * step);
  return d * d;
}

// ---- the compacted FP64 kernel's integer path (XFix positions) --------------
//
// A pair's separation is D = X_j - X_i per axis (units 2^-F, |D| < 2^60
// for pairs closer than half the box).  The three |D| share one left shift
// sh that puts the largest at bit 60: A = |D| 2^sh < 2^61.  Products are
// then taken as the high 64 bits of 64 x 64-bit products (__umul64hi), whose
// truncation is below one unit of a result of 56 to 61 significant bits.

// |d| of a separation count.
__device__ __forceinline__ unsigned long long md_uabs(long long d) {
  return d < 0 ? (unsigned long long)(-d) : (unsigned long long)d;
}

// The common shift sh (>= 0) and the shifted magnitudes A = |D| 2^sh, and
// r^2 = (Dx^2 + Dy^2 + Dz^2) 2^-2F as a double, truncated: the sum of the
// three high products S is within 3 units below the exact sum 2^(2 sh - 64)
// (S ~ 2^56 or more for pairs near the cutoff), and S is truncated once
// more to 53 bits, so the result lies within 1.1 ulps below the exact r^2.
// Integer instructions only.
__device__ __forceinline__ double md_sep_r2(long long Dx, long long Dy, long long Dz, int F,
                                            unsigned long long& Ax, unsigned long long& Ay,
                                            unsigned long long& Az, int& sh) {
  Ax = md_uabs(Dx);
  Ay = md_uabs(Dy);
  Az = md_uabs(Dz);
  const unsigned long long am = Ax | Ay | Az;
  if (am == 0) {  // coincident atoms
    sh = 0;
    return 0.0;
  }
  sh = __clzll((long long)am) - 3;  // am < 2^61: sh >= 0, leading one to bit 60
  Ax <<= sh;
  Ay <<= sh;
  Az <<= sh;
  const unsigned long long S = __umul64hi(Ax, Ax) + __umul64hi(Ay, Ay) + __umul64hi(Az, Az);
  // r^2 = S 2^(64 - 2 sh - 2 F); S > 0 (its largest term is >= 2^56)
  const int lz = __clzll((long long)S);
  const unsigned long long m = (S << lz) >> 11;  // 53 bits, leading one at bit 52
  const long long e = 1150 - 2 * F - lz - 2 * sh;  // biased exponent of the result
  return __longlong_as_double(((e - 1) << 52) + (long long)m);
}

// The fixed-point count (units 2^-MD_FIX_BITS) of the contribution f d, with
// d = +-A 2^(-F - sh) (A and sh from md_sep_r2, neg: d < 0): the high 64
// bits H of the product of f's significand (at bit 63) and A, rounded to the
// nearest count.  Within one count of the exact f d 2^44 (the truncated low
// bits weigh below 2^-7 counts for any count in range).  False, leaving q
// unset, when |q| >= 2^qbits (the accumulators' range) or f is not finite.
// Integer instructions only.
__device__ __forceinline__ bool md_fix_prod(double f, unsigned long long A, bool neg, int sh,
                                            int F, int qbits, long long& q) {
  static_assert(MD_FIX_BITS == 44, "the exponent 978 below");
  const long long b = __double_as_longlong(f);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0x7ff) return false;
  if (e == 0) {
    q = 0;
    return true;
  }
  const unsigned long long Mn = ((unsigned long long)b << 11) | (1ULL << 63);
  const unsigned long long H = __umul64hi(Mn, A);  // < 2^61
  // |f d| 2^44 = Mn A 2^(e - 1042 - F - sh) = H 2^(e - 978 - F - sh) (+ the
  // low half)
  const int s = 978 + F + sh - e;
  if (s <= 0) return false;
  unsigned long long r = 0;
  if (s < 64) {
    r = (H + (1ULL << (s - 1))) >> s;
    if ((r >> qbits) != 0) return false;
  }
  q = ((b < 0) != neg) ? -(long long)r : (long long)r;
  return true;
}

// r^2 in FP64 from the position splits: the hi parts' difference and image
// shift are exact in FP32 (grid split, md_split), the lo parts' difference
// and the box's lo part are taken in FP64, so only the lo parts' own
// rounding (|x - hi - lo| <= 2^-25 grid step) remains: ~3e-12 relative to
// r^2 at a 168-wide box.  j's split is loaded again (volatile: the load
// stays on the rare path that calls this).
__device__ __forceinline__ double md_r2_split(const XSplit* pj, const XSplit& si, float hf0,
                                              float hf1, float hf2, float Lf0, float Lf1,
                                              float Lf2, float Ll0, float Ll1, float Ll2) {
  XSplit sj;
  asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(sj.hi.x), "=f"(sj.hi.y), "=f"(sj.hi.z), "=f"(sj.hi.w), "=f"(sj.lo.x),
                 "=f"(sj.lo.y), "=f"(sj.lo.z), "=f"(sj.lo.w)
               : "l"(pj));
  auto axis = [](float hj, float hi, float lj, float li, float hf, float Lf, float Ll) {
    float h = hj - hi;
    double l = __dsub_rn(md_widen(lj), md_widen(li));
    if (fabsf(h) > hf) {
      const float sg = copysignf(1.f, h);
      h -= sg * Lf;
      l = __dsub_rn(l, md_widen(sg * Ll));
    }
    return __dadd_rn(md_widen(h), l);
  };
  const double ex = axis(sj.hi.x, si.hi.x, sj.lo.x, si.lo.x, hf0, Lf0, Ll0);
  const double ey = axis(sj.hi.y, si.hi.y, sj.lo.y, si.lo.y, hf1, Lf1, Ll1);
  const double ez = axis(sj.hi.z, si.hi.z, sj.lo.z, si.lo.z, hf2, Lf2, Ll2);
  return md_r2(ex, ey, ez);
}

// Add NV values of each lane into the accumulators of the lane's replica:
// row `slot` of the replica's `spread` rows (acc + (rep * spread + slot) *
// MD_EV_STRIDE), which k_ev_fold sums afterwards -- spreading the warps'
// atomics over rows keeps them from queueing on one address.  Lanes with
// rep < 0 contribute nothing.  When the whole warp belongs to one replica
// (the common case) the warp reduces first and one lane issues the
// atomics.  All 32 lanes must call it.
template <int NV>
__device__ __forceinline__ void md_warp_add_rep(double (&v)[NV], int rep, double* acc,
                                                int spread, int slot) {
  const int lane = threadIdx.x & 31;
  const int r0 = __shfl_sync(0xffffffffu, rep, 0);
  const bool uniform = __all_sync(0xffffffffu, rep == r0 || rep < 0);
  if (uniform) {
#pragma unroll
    for (int c = 0; c < NV; c++) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], off);
    }
    if (lane == 0 && r0 >= 0) {
#pragma unroll
      for (int c = 0; c < NV; c++)
        atomicAdd(acc + ((int64_t)r0 * spread + slot) * MD_EV_STRIDE + c, v[c]);
    }
  } else if (rep >= 0) {
#pragma unroll
    for (int c = 0; c < NV; c++)
      atomicAdd(acc + ((int64_t)rep * spread + slot) * MD_EV_STRIDE + c, v[c]);
  }
}

// Block-wide sum of NV doubles into out[0..NV) of block's slot; all threads
// of the block must call it.  blockDim.x == MD_BLOCK.
template <int NV>
__device__ __forceinline__ void md_block_sum(double (&v)[NV], double* out_block) {
  __shared__ double red[MD_BLOCK / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NV; c++) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], off);
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < NV; c++) red[warp][c] = v[c];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < MD_BLOCK / 32; w++) s += red[w][threadIdx.x];
    out_block[threadIdx.x] = s;
  }
}
