// Device arithmetic helpers: complex numbers over float/double and double-float ("ff")
// numbers (an unevaluated sum hi + lo of two FP32 values, 48-bit significand).
//
// The ff operations follow the classical error-free transformations:
//   Knuth's TwoSum (exact a + b = s + e), Dekker's FastTwoSum (|a| >= |b|) and the
//   FMA-based TwoProduct (exact a * b = p + e with e = fma(a, b, -p)).
// They are used because the binary64 pipe of sm_103a runs at ~1/70 of the FP32 rate,
// so per-coefficient residual, correction and quadratic-form arithmetic is done in ff.
// This file must be compiled without fast-math (IEEE FP32 semantics are required).
#pragma once
#include <cuda_runtime.h>

namespace tdz {

#define TDZ_DEV __device__ __forceinline__

// ---------------------------------------------------------------------------- complex
template <class T>
struct cx {
  T r, i;
};
template <class T> TDZ_DEV cx<T> mk(T r, T i) { return cx<T>{r, i}; }
template <class T> TDZ_DEV cx<T> operator+(cx<T> a, cx<T> b) { return {a.r + b.r, a.i + b.i}; }
template <class T> TDZ_DEV cx<T> operator-(cx<T> a, cx<T> b) { return {a.r - b.r, a.i - b.i}; }
template <class T> TDZ_DEV cx<T> cmul(cx<T> a, cx<T> b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
// a - b*c
template <class T> TDZ_DEV cx<T> cmsub(cx<T> a, cx<T> b, cx<T> c) {
  return {a.r - b.r * c.r + b.i * c.i, a.i - b.r * c.i - b.i * c.r};
}
// a + b*c
template <class T> TDZ_DEV cx<T> cmadd(cx<T> a, cx<T> b, cx<T> c) {
  return {a.r + b.r * c.r - b.i * c.i, a.i + b.r * c.i + b.i * c.r};
}
template <class T> TDZ_DEV cx<T> crecip(cx<T> a) {
  T d = a.r * a.r + a.i * a.i;
  T s = T(1) / d;
  return {a.r * s, -a.i * s};
}
template <class T> TDZ_DEV cx<T> czero() { return {T(0), T(0)}; }
template <class T> TDZ_DEV T cnorm2(cx<T> a) { return a.r * a.r + a.i * a.i; }

// ---------------------------------------------------------------------------- double-float
struct ff {
  float h, l;
};
TDZ_DEV ff two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
TDZ_DEV ff fast_two_sum(float a, float b) {
  float s = a + b;
  float e = b - (s - a);
  return {s, e};
}
TDZ_DEV ff ff_add(ff a, ff b) {
  ff s = two_sum(a.h, b.h);
  float e = s.l + (a.l + b.l);
  return fast_two_sum(s.h, e);
}
TDZ_DEV ff ff_neg(ff a) { return {-a.h, -a.l}; }
TDZ_DEV ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
TDZ_DEV ff ff_mul(ff a, ff b) {
  float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return fast_two_sum(p, e);
}
TDZ_DEV ff ff_mulf(ff a, float b) {
  float p = a.h * b;
  float e = fmaf(a.h, b, -p);
  e = fmaf(a.l, b, e);
  return fast_two_sum(p, e);
}
TDZ_DEV ff ff_addf(ff a, float b) {
  ff s = two_sum(a.h, b);
  float e = s.l + a.l;
  return fast_two_sum(s.h, e);
}
TDZ_DEV float ff_f(ff a) { return a.h + a.l; }

// Dot2-style accumulator (Ogita, Rump, Oishi 2005): the running sum s is kept with a
// compensation c; each product is added as an exact TwoProduct pair.
struct ffacc {
  float s, c;
};
TDZ_DEV void acc_zero(ffacc& a) { a.s = 0.f; a.c = 0.f; }
// a += x * y  with x, y double-float numbers (lo*lo neglected)
TDZ_DEV void acc_mul(ffacc& a, ff x, ff y) {
  float p = x.h * y.h;
  float e = fmaf(x.h, y.h, -p);
  e = fmaf(x.h, y.l, e);
  e = fmaf(x.l, y.h, e);
  ff t = two_sum(a.s, p);
  a.s = t.h;
  a.c += t.l + e;
}
TDZ_DEV void acc_add(ffacc& a, ff x) {
  ff t = two_sum(a.s, x.h);
  a.s = t.h;
  a.c += t.l + x.l;
}
TDZ_DEV ff acc_get(const ffacc& a) { return fast_two_sum(a.s, a.c); }

// complex double-float
struct cff {
  ff r, i;
};
TDZ_DEV cff cff_add(cff a, cff b) { return {ff_add(a.r, b.r), ff_add(a.i, b.i)}; }
TDZ_DEV cff cff_addc(cff a, cx<float> b) { return {ff_addf(a.r, b.r), ff_addf(a.i, b.i)}; }

// ---------------------------------------------------------------------------- fx
// Double-float number with arithmetic operators, so that templated kernels written for float and
// double also instantiate in double-float (48-bit significand on the FP32 pipe). Conversions from
// double round to the nearest pair; in device code they cost binary64 operations, so kernels
// receive their constants already converted.
struct fx {
  float h, l;
  fx() = default;
  __host__ __device__ constexpr fx(float a, float b) : h(a), l(b) {}
  __host__ __device__ fx(int v) : h((float)v), l(0.f) {}
  __host__ __device__ fx(double v) : h((float)v), l((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
  __host__ __device__ explicit operator float() const { return h + l; }
};
TDZ_DEV fx to_fx(ff a) { return fx(a.h, a.l); }
TDZ_DEV ff to_ff(fx a) { return ff{a.h, a.l}; }
TDZ_DEV fx operator+(fx a, fx b) { return to_fx(ff_add(to_ff(a), to_ff(b))); }
TDZ_DEV fx operator-(fx a, fx b) { return to_fx(ff_add(to_ff(a), ff{-b.h, -b.l})); }
TDZ_DEV fx operator-(fx a) { return fx(-a.h, -a.l); }
TDZ_DEV fx operator*(fx a, fx b) { return to_fx(ff_mul(to_ff(a), to_ff(b))); }
TDZ_DEV fx& operator+=(fx& a, fx b) { return a = a + b; }
TDZ_DEV fx& operator-=(fx& a, fx b) { return a = a - b; }
TDZ_DEV fx& operator*=(fx& a, fx b) { return a = a * b; }
// a / b: FP32 quotient corrected once with the double-float remainder a - q b
TDZ_DEV fx operator/(fx a, fx b) {
  const float q0 = a.h / b.h;
  const ff r = ff_add(to_ff(a), ff_neg(ff_mulf(to_ff(b), q0)));
  const float q1 = r.h / b.h;
  return to_fx(fast_two_sum(q0, q1));
}
TDZ_DEV bool operator<(fx a, fx b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
// square root for templated kernels (float, double, fx)
TDZ_DEV float tsqrt(float a) { return sqrtf(a); }
TDZ_DEV double tsqrt(double a) { return ::sqrt(a); }
// sqrt(a), a >= 0: FP32 root s refined once with the double-float remainder a - s^2
TDZ_DEV fx tsqrt(fx a) {
  if (!(a.h > 0.f)) return fx(0.f, 0.f);
  const float s = sqrtf(a.h);
  const float p = s * s;
  const ff s2 = ff{p, fmaf(s, s, -p)};
  const ff r = ff_add(to_ff(a), ff_neg(s2));
  return to_fx(fast_two_sum(s, r.h / (2.f * s)));
}

// ---------------------------------------------------------------------------- packed FP32 pairs
// Two FP32 values in one 64-bit register, operated on by the f32x2 instructions of sm_100 and later
// (one instruction, two IEEE round-to-nearest results). A complex double-float number keeps its real
// and imaginary parts in the two lanes, so each step of a double-float operation on a complex number
// is one instruction instead of two; the results are bitwise those of the scalar operations above.
struct f2 {
  unsigned long long v;
};
TDZ_DEV f2 f2_pack(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
TDZ_DEV float2 f2_unpack(f2 a) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a.v));
  return r;
}
TDZ_DEV f2 f2_add(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
TDZ_DEV f2 f2_sub(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
TDZ_DEV f2 f2_mul(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
TDZ_DEV f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}

// complex double-float, packed: h = (re.h, im.h), l = (re.l, im.l)
struct pcff {
  f2 h, l;
};
// a real double-float factor as the packed broadcasts the products below take: x.h, -x.h, -x.l
struct pfac {
  f2 h, nh, nl;
};
TDZ_DEV pfac pfac_of(float h, float l) { return pfac{f2_pack(h, h), f2_pack(-h, -h), f2_pack(-l, -l)}; }
// a different real factor per lane: (h0 + l0) on lane 0, (h1 + l1) on lane 1
TDZ_DEV pfac pfac2_of(float h0, float l0, float h1, float l1) {
  return pfac{f2_pack(h0, h1), f2_pack(-h0, -h1), f2_pack(-l0, -l1)};
}
// the lanes exchanged: (im, re)
TDZ_DEV pcff pcff_swap(pcff a) {
  const float2 h = f2_unpack(a.h), l = f2_unpack(a.l);
  return pcff{f2_pack(h.y, h.x), f2_pack(l.y, l.x)};
}
// fast_two_sum on both lanes
TDZ_DEV pcff p_fast_two_sum(f2 a, f2 b) {
  const f2 s = f2_add(a, b);
  return pcff{s, f2_sub(b, f2_sub(s, a))};
}
// a + b (ff_add on both lanes)
TDZ_DEV pcff pcff_add(pcff a, pcff b) {
  const f2 s = f2_add(a.h, b.h);
  const f2 bb = f2_sub(s, a.h);
  const f2 e = f2_add(f2_sub(a.h, f2_sub(s, bb)), f2_sub(b.h, bb));
  return p_fast_two_sum(s, f2_add(e, f2_add(a.l, b.l)));
}
// x * y for a real factor x (ff_mul on both lanes; the error term is carried negated)
TDZ_DEV pcff pcff_scale(const pfac& x, pcff y) {
  const f2 p = f2_mul(x.h, y.h);
  f2 ne = f2_fma(x.nh, y.h, p);
  ne = f2_fma(x.nh, y.l, ne);
  ne = f2_fma(x.nl, y.h, ne);
  const f2 s = f2_sub(p, ne);  // fast_two_sum(p, e) with e = -ne
  return pcff{s, f2_sub(f2_sub(p, s), ne)};
}
// Dot2 accumulator of a complex sum, packed (acc_mul / acc_get on both lanes)
struct pacc {
  f2 s, c;
};
TDZ_DEV void pacc_zero(pacc& a) {
  a.s = f2_pack(0.f, 0.f);
  a.c = a.s;
}
// a += x * y (x real double-float, y complex double-float)
TDZ_DEV void pacc_mul(pacc& a, const pfac& x, pcff y) {
  const f2 p = f2_mul(x.h, y.h);
  f2 ne = f2_fma(x.nh, y.h, p);  // -(x.h y.h - p), exact
  ne = f2_fma(x.nh, y.l, ne);
  ne = f2_fma(x.nl, y.h, ne);
  const f2 s = f2_add(a.s, p);
  const f2 bb = f2_sub(s, a.s);
  const f2 t = f2_add(f2_sub(a.s, f2_sub(s, bb)), f2_sub(p, bb));
  a.s = s;
  a.c = f2_add(a.c, f2_sub(t, ne));
}
TDZ_DEV pcff pacc_get(const pacc& a) { return p_fast_two_sum(a.s, a.c); }

// ---------------------------------------------------------------------------- TF32 split
// x rounded to the nearest TF32 value (8 exponent bits, 10 stored significand bits: the low 13 bits
// of the FP32 pattern cleared after adding half of their weight, ties away from zero); x - tf32_hi(x)
// is exact in FP32 and at most 2^-11 |x|.
TDZ_DEV float tf32_hi(float x) { return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u); }

}  // namespace tdz
