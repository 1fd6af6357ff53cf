// df64.cuh -- double-float ("df64") arithmetic and complex helpers.
//
// GB300 issues FP32 instructions at a far higher rate than FP64 ones, so the
// library's FP64-class path keeps every quantity as an unevaluated sum of
// two floats, x = hi + lo with |lo| <= ulp(hi)/2 (48-bit significand), and
// computes with error-free transformations:
//   * TwoSum (Knuth, TAOCP vol. 2): s + e == a + b exactly;
//   * FastTwoSum (Dekker 1971): same when |a| >= |b|;
//   * TwoProd via FMA: p + e == a * b exactly;
//   * running sums kept as renormalised float pairs, fed with exact
//     products (the double-length accumulation of Dekker 1971).
// The `_rn` intrinsics keep the compiler from fusing or reordering these.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace tw {

struct __align__(8) dd { float hi, lo; };
struct __align__(16) cdd { dd re, im; };   // complex double-float, 16 bytes (float4 layout)
struct __align__(8) cf { float re, im; };  // complex float, 8 bytes
struct __align__(16) cd { double re, im; };  // complex double (set-up filters)

// ---------------------------------------------------------------- basics
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ dd dd_make(float hi, float lo) {
  dd r; fast_two_sum(hi, lo, r.hi, r.lo); return r;
}
__device__ __forceinline__ dd dd_zero() { dd r; r.hi = 0.f; r.lo = 0.f; return r; }
// the pair as it is (no renormalisation)
__device__ __forceinline__ dd dd_make_raw(float hi, float lo) { dd r; r.hi = hi; r.lo = lo; return r; }
__device__ __forceinline__ dd dd_neg(dd a) { a.hi = -a.hi; a.lo = -a.lo; return a; }

// sum with relative error O(2^-48) of |a| + |b|
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  dd r; fast_two_sum(s, e, r.hi, r.lo); return r;
}
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

// product with relative error O(2^-47)
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  dd r; fast_two_sum(p, e, r.hi, r.lo); return r;
}
__device__ __forceinline__ dd dd_mul_f(dd a, float b) {
  float p = __fmul_rn(a.hi, b);
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  dd r; fast_two_sum(p, e, r.hi, r.lo); return r;
}
// exact scaling by a power of two
__device__ __forceinline__ dd dd_scale2(dd a, float p2) { a.hi *= p2; a.lo *= p2; return a; }

// quotient a / b: float estimate refined once (Dekker's long division)
__device__ __forceinline__ dd dd_div(dd a, dd b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  dd r = dd_sub(a, dd_mul_f(b, q1));
  float q2 = __fdiv_rn(r.hi, b.hi);
  return dd_make(q1, q2);
}
// square root: float estimate x, one correction (a - x^2) / (2x)
__device__ __forceinline__ dd dd_sqrt(dd a) {
  if (a.hi <= 0.f) return dd_zero();
  float x = __fsqrt_rn(a.hi);
  float p = __fmul_rn(x, x);
  float pe = fmaf(x, x, -p);
  dd r = dd_sub(a, dd_make(p, pe));
  float c = __fdiv_rn(r.hi, __fmul_rn(2.f, x));
  return dd_make(x, c);
}

// ------------------------------------------------------- conversions
// IEEE double <-> df64.  These run at the edges of the library only.
__device__ __forceinline__ dd dd_from_double(double x) {
  dd r;
  r.hi = __double2float_rn(x);
  r.lo = __double2float_rn(x - (double)r.hi);
  return r;
}
__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

// ------------------------------------------------- accumulation
// value = s + t, renormalised after every step (|t| <= ulp(s)/2), so each
// step rounds at the 2^-48 level of the running sum; a float error term
// that is left to grow would instead lose O(k^1.5 u^2) over k terms.
struct dacc { float s, t; };
__device__ __forceinline__ dacc dacc_zero() { dacc a; a.s = 0.f; a.t = 0.f; return a; }
// A += a * b   (a sign is folded into the operands by the caller)
__device__ __forceinline__ void dacc_mac(dacc &A, dd a, dd b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);     // exact error of the leading product
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, r;
  two_sum(A.s, p, s, r);
  r = __fadd_rn(r, __fadd_rn(A.t, e));
  fast_two_sum(s, r, A.s, A.t);
}
__device__ __forceinline__ void dacc_add(dacc &A, dd a) {
  float s, r;
  two_sum(A.s, a.hi, s, r);
  r = __fadd_rn(r, __fadd_rn(A.t, a.lo));
  fast_two_sum(s, r, A.s, A.t);
}
__device__ __forceinline__ dd dacc_get(dacc A) { dd r; r.hi = A.s; r.lo = A.t; return r; }
// fold a partial sum into a double-float total and restart it
__device__ __forceinline__ void dacc_fold(dd &tot, dacc &A) {
  tot = dd_add(tot, dacc_get(A));
  A = dacc_zero();
}

// ------------------------------------------------------ complex df64
__device__ __forceinline__ cdd cdd_zero() { cdd z; z.re = dd_zero(); z.im = dd_zero(); return z; }
__device__ __forceinline__ cdd cdd_add(cdd a, cdd b) { cdd r; r.re = dd_add(a.re, b.re); r.im = dd_add(a.im, b.im); return r; }
__device__ __forceinline__ cdd cdd_sub(cdd a, cdd b) { cdd r; r.re = dd_sub(a.re, b.re); r.im = dd_sub(a.im, b.im); return r; }
__device__ __forceinline__ cdd cdd_conj(cdd a) { a.im = dd_neg(a.im); return a; }
// multiply by -i: (x + iy)(-i) = y - ix
__device__ __forceinline__ cdd cdd_mul_mi(cdd a) { cdd r; r.re = a.im; r.im = dd_neg(a.re); return r; }
__device__ __forceinline__ cdd cdd_mul_i(cdd a) { cdd r; r.re = dd_neg(a.im); r.im = a.re; return r; }
// a b + c d with relative error O(2^-47) of |a b| + |c d|: the two leading
// products and their errors are exact (TwoProd), the leading parts are added
// by TwoSum, and everything below them is gathered in one float before the
// single renormalisation
__device__ __forceinline__ dd dd_dot2(dd a, dd b, dd c, dd d) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float q = __fmul_rn(c.hi, d.hi);
  float f = fmaf(c.hi, d.hi, -q);
  f = fmaf(c.hi, d.lo, f);
  f = fmaf(c.lo, d.hi, f);
  float s, r;
  two_sum(p, q, s, r);
  r = __fadd_rn(r, __fadd_rn(e, f));
  dd o; fast_two_sum(s, r, o.hi, o.lo); return o;
}
__device__ __forceinline__ cdd cdd_mul(cdd a, cdd b) {
  cdd r;
  r.re = dd_dot2(a.re, b.re, dd_neg(a.im), b.im);
  r.im = dd_dot2(a.re, b.im, a.im, b.re);
  return r;
}
__device__ __forceinline__ cdd cdd_scale(cdd a, dd s) { cdd r; r.re = dd_mul(a.re, s); r.im = dd_mul(a.im, s); return r; }
__device__ __forceinline__ cdd cdd_scale2(cdd a, float p2) { a.re = dd_scale2(a.re, p2); a.im = dd_scale2(a.im, p2); return a; }

__device__ __forceinline__ cdd ld_cdd(const cdd *p) {
  float4 v = *reinterpret_cast<const float4 *>(p);
  cdd r; r.re.hi = v.x; r.re.lo = v.y; r.im.hi = v.z; r.im.lo = v.w; return r;
}
__device__ __forceinline__ void st_cdd(cdd *p, cdd a) {
  *reinterpret_cast<float4 *>(p) = make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo);
}

// ------------------------------------------------------- complex float
__device__ __forceinline__ cf cf_make(float r, float i) { cf z; z.re = r; z.im = i; return z; }
__device__ __forceinline__ cf cf_zero() { return cf_make(0.f, 0.f); }
__device__ __forceinline__ cf cf_add(cf a, cf b) { return cf_make(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ cf cf_sub(cf a, cf b) { return cf_make(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ cf cf_conj(cf a) { return cf_make(a.re, -a.im); }
__device__ __forceinline__ cf cf_mul_mi(cf a) { return cf_make(a.im, -a.re); }
__device__ __forceinline__ cf cf_mul_i(cf a) { return cf_make(-a.im, a.re); }
__device__ __forceinline__ cf cf_mul(cf a, cf b) {
  return cf_make(fmaf(a.re, b.re, -a.im * b.im), fmaf(a.re, b.im, a.im * b.re));
}

// --------------------------------------------- precision policies
// Each policy names a complex type, a real type and the operations the FFT
// engine needs, so one engine serves the df64 path and the FP32 path.
struct PolDD {
  typedef cdd cx;
  typedef dd re;
  static constexpr int occ = 3;   // CTAs of 256 threads per SM the FFT kernels aim for
  static constexpr int smem = 72 * 1024;   // shared-memory budget of one FFT CTA
  static __device__ __forceinline__ cx zero() { return cdd_zero(); }
  static __device__ __forceinline__ cx add(cx a, cx b) { return cdd_add(a, b); }
  static __device__ __forceinline__ cx sub(cx a, cx b) { return cdd_sub(a, b); }
  static __device__ __forceinline__ cx mul(cx a, cx b) { return cdd_mul(a, b); }
  static __device__ __forceinline__ cx conj(cx a) { return cdd_conj(a); }
  static __device__ __forceinline__ cx mul_mi(cx a) { return cdd_mul_mi(a); }
  static __device__ __forceinline__ cx mul_i(cx a) { return cdd_mul_i(a); }
  static __device__ __forceinline__ cx scale_re(cx a, re s) { return cdd_scale(a, s); }
  static __device__ __forceinline__ cx scale2(cx a, float p2) { return cdd_scale2(a, p2); }
  static __device__ __forceinline__ re re_add(re a, re b) { return dd_add(a, b); }
  static __device__ __forceinline__ re re_sub(re a, re b) { return dd_sub(a, b); }
  static __device__ __forceinline__ re re_neg(re a) { return dd_neg(a); }
  static __device__ __forceinline__ re re_mul(re a, re b) { return dd_mul(a, b); }
  static __device__ __forceinline__ re re_zero() { return dd_zero(); }
  static __device__ __forceinline__ cx make(re r, re i) { cx z; z.re = r; z.im = i; return z; }
  static __device__ __forceinline__ re real(cx a) { return a.re; }
  static __device__ __forceinline__ re imag(cx a) { return a.im; }
};
struct PolF {
  typedef cf cx;
  typedef float re;
  static constexpr int occ = 4;
  static constexpr int smem = 64 * 1024;
  static __device__ __forceinline__ cx zero() { return cf_zero(); }
  static __device__ __forceinline__ cx add(cx a, cx b) { return cf_add(a, b); }
  static __device__ __forceinline__ cx sub(cx a, cx b) { return cf_sub(a, b); }
  static __device__ __forceinline__ cx mul(cx a, cx b) { return cf_mul(a, b); }
  static __device__ __forceinline__ cx conj(cx a) { return cf_conj(a); }
  static __device__ __forceinline__ cx mul_mi(cx a) { return cf_mul_mi(a); }
  static __device__ __forceinline__ cx mul_i(cx a) { return cf_mul_i(a); }
  static __device__ __forceinline__ cx scale_re(cx a, re s) { return cf_make(a.re * s, a.im * s); }
  static __device__ __forceinline__ cx scale2(cx a, float p2) { return cf_make(a.re * p2, a.im * p2); }
  static __device__ __forceinline__ re re_add(re a, re b) { return a + b; }
  static __device__ __forceinline__ re re_sub(re a, re b) { return a - b; }
  static __device__ __forceinline__ re re_neg(re a) { return -a; }
  static __device__ __forceinline__ re re_mul(re a, re b) { return a * b; }
  static __device__ __forceinline__ re re_zero() { return 0.f; }
  static __device__ __forceinline__ cx make(re r, re i) { return cf_make(r, i); }
  static __device__ __forceinline__ re real(cx a) { return a.re; }
  static __device__ __forceinline__ re imag(cx a) { return a.im; }
};

// native FP64 policy: used at set-up, where accuracy matters and time does not
struct PolD {
  typedef cd cx;
  typedef double re;
  static constexpr int occ = 2;
  static constexpr int smem = 64 * 1024;
  static __device__ __forceinline__ cx make(re r, re i) { cx z; z.re = r; z.im = i; return z; }
  static __device__ __forceinline__ cx zero() { return make(0.0, 0.0); }
  static __device__ __forceinline__ cx add(cx a, cx b) { return make(a.re + b.re, a.im + b.im); }
  static __device__ __forceinline__ cx sub(cx a, cx b) { return make(a.re - b.re, a.im - b.im); }
  static __device__ __forceinline__ cx mul(cx a, cx b) {
    return make(fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re));
  }
  static __device__ __forceinline__ cx conj(cx a) { return make(a.re, -a.im); }
  static __device__ __forceinline__ cx mul_mi(cx a) { return make(a.im, -a.re); }
  static __device__ __forceinline__ cx mul_i(cx a) { return make(-a.im, a.re); }
  static __device__ __forceinline__ cx scale_re(cx a, re s) { return make(a.re * s, a.im * s); }
  static __device__ __forceinline__ cx scale2(cx a, float p2) { return make(a.re * p2, a.im * p2); }
  static __device__ __forceinline__ re re_add(re a, re b) { return a + b; }
  static __device__ __forceinline__ re re_sub(re a, re b) { return a - b; }
  static __device__ __forceinline__ re re_neg(re a) { return -a; }
  static __device__ __forceinline__ re re_mul(re a, re b) { return a * b; }
  static __device__ __forceinline__ re re_zero() { return 0.0; }
  static __device__ __forceinline__ re real(cx a) { return a.re; }
  static __device__ __forceinline__ re imag(cx a) { return a.im; }
};

// ----------------------------------- element loads/stores by format
// real scalars
__device__ __forceinline__ void ld_real(const double *p, dd &v) { v = dd_from_double(*p); }
__device__ __forceinline__ void ld_real(const dd *p, dd &v) {
  float2 t = *reinterpret_cast<const float2 *>(p); v.hi = t.x; v.lo = t.y;
}
__device__ __forceinline__ void ld_real(const float *p, float &v) { v = *p; }
__device__ __forceinline__ void ld_real(const double *p, float &v) { v = __double2float_rn(*p); }
__device__ __forceinline__ void st_real(double *p, dd v) { *p = dd_to_double(v); }
__device__ __forceinline__ void st_real(dd *p, dd v) {
  *reinterpret_cast<float2 *>(p) = make_float2(v.hi, v.lo);
}
__device__ __forceinline__ void st_real(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_real(double *p, float v) { *p = (double)v; }


// ------------------------------------------------ packed FP32 pairs
// Two independent FP32 lanes in one 64-bit register (add/sub/mul/fma.rn.f32x2):
// each lane rounds exactly like the scalar instruction, so a packed double-
// float sequence gives, lane by lane, the bits of the scalar one in half the
// instructions.  f2_make(lo, hi): lo is lane 0 (the lower address in memory).
struct f2 { unsigned long long v; };
__device__ __forceinline__ f2 f2_make(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 f2_split(f2 a) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a.v));
  return r;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) { f2 r; asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v)); return r; }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { f2 r; asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v)); return r; }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { f2 r; asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v)); return r; }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r; asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v)); return r;
}


// S + T += (ah + al)(bh + bl) lane by lane, exactly the steps of dacc_mac:
// bhn = -bh (so -(ah bh) is one rounded product and its error one FMA)
__device__ __forceinline__ void dacc_mac2(f2 &S, f2 &T, f2 ah, f2 al, f2 bh, f2 bhn, f2 bl) {
  const f2 pn = mul2(ah, bhn);
  f2 e = fma2(ah, bh, pn);
  e = fma2(ah, bl, e);
  e = fma2(al, bh, e);
  const f2 s = sub2(S, pn);
  const f2 bb = sub2(s, S);
  const f2 r = add2(sub2(sub2(S, sub2(s, bb)), add2(pn, bb)), add2(T, e));
  S = add2(s, r);
  T = sub2(r, sub2(S, s));
}
// (ah, al) = dd_add((ah, al), (bh, bl)) lane by lane
__device__ __forceinline__ void dd_add2(f2 &ah, f2 &al, f2 bh, f2 bl) {
  const f2 s = add2(ah, bh);
  const f2 bb = sub2(s, ah);
  f2 e = add2(sub2(ah, sub2(s, bb)), sub2(bh, bb));
  e = add2(e, add2(al, bl));
  ah = add2(s, e);
  al = sub2(e, sub2(ah, s));
}
}  // namespace tw
