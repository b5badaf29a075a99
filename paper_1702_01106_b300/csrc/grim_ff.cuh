// Float-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats (about 48 significant bits, rounding ~2^-47 of the operands), built
// from error-free transformations (Knuth's two-sum; the exact product error
// by FMA, as in Dekker's product).  On B300 a float-float operation costs
// 4-11 float32 instructions on a pipe 64 times wider than the float64 one,
// so face states and fluxes evaluated this way cost a fraction of their
// float64 time at an accuracy far below the solver tolerances.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>

namespace grim {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit ff(double d) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
  }
  __device__ __forceinline__ explicit ff(int i) : hi((float)i), lo(0.f) {}
};

// A compile-time constant in the working precision (for float-float: the
// pair of the nearest float and the float nearest to the remainder), so that
// literals cost no float64 conversion at run time.
template <typename T> __host__ __device__ constexpr T tconst(double x) { return T(x); }
template <> __host__ __device__ constexpr ff tconst<ff>(double x) {
  return ff(static_cast<float>(x), static_cast<float>(x - static_cast<double>(static_cast<float>(x))));
}
template <> __host__ __device__ constexpr double tconst<double>(double x) { return x; }
__device__ __forceinline__ double ff_join(ff a);
__device__ __forceinline__ double as_double(ff a) { return ff_join(a); }
__device__ __forceinline__ double as_double(double a) { return a; }

// s + e with |s| >= |e| (or s = 0): normalised pair.
__device__ __forceinline__ ff ff_quick(float s, float e) {
  const float h = s + e;
  return ff(h, e - (h - s));
}
// Exact sum a + b = s + err.
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = a + b;
  const float v = s - a;
  return ff(s, (a - (s - v)) + (b - v));
}

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
// The sum with the low parts added in plain float (Dekker's form): error
// within about 2^-47 (|x| + |y|), an absolute bound like float64's own
// rounding of a cancelling sum, at 11 float additions instead of the 20 of
// the relative-error form.
__device__ __forceinline__ ff operator+(ff x, ff y) {
  const ff s = ff_two_sum(x.hi, y.hi);
  return ff_quick(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ ff operator-(ff x, ff y) { return x + (-y); }
__device__ __forceinline__ ff operator*(ff x, ff y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return ff_quick(p, e);
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { a = a + b; return a; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { a = a - b; return a; }
__device__ __forceinline__ ff& operator*=(ff& a, ff b) { a = a * b; return a; }

__device__ __forceinline__ bool operator>(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(ff a, ff b) { return b > a; }

// The float64 and float forms stay visible beside the float-float overloads
// below.
using ::fabs;
using ::fmax;
using ::fmin;
using ::fma;

__device__ __forceinline__ ff fabs(ff a) { return (a.hi < 0.f || (a.hi == 0.f && a.lo < 0.f)) ? -a : a; }
__device__ __forceinline__ ff fmax(ff a, ff b) { return a > b ? a : b; }
__device__ __forceinline__ ff fmin(ff a, ff b) { return a > b ? b : a; }
__device__ __forceinline__ ff fma(ff a, ff b, ff c) { return a * b + c; }

// 1/y: the float reciprocal refined by one Newton step in float-float.
__device__ __forceinline__ ff nr_rcp(ff y) {
  const ff x(__frcp_rn(y.hi), 0.f);
  const ff one(1.f, 0.f);
  return x + x * (one - y * x);
}
// sqrt(a), a >= 0: the float root corrected by (a - s^2)/(2 s).
__device__ __forceinline__ ff sqr_root(ff a) {
  if (!(a.hi > 0.f)) return ff(0.f, 0.f);
  const float s = __fsqrt_rn(a.hi);
  const ff S(s, 0.f);
  const ff r = a - S * S;
  return ff_quick(s, r.hi * (0.5f / s));
}
// a^(-1/2), a > 0: the float estimate refined by one Newton step in
// float-float, y <- y + y (1 - (a y) y)/2 (a y first, so that y^2 cannot
// overflow for a small a).
__device__ __forceinline__ ff rsq(ff a) {
  const ff y(rsqrtf(a.hi), 0.f);
  const ff one(1.f, 0.f), half(0.5f, 0.f);
  return y + (y * half) * (one - (a * y) * y);
}

// A power of two s with s m in [1, 2) for a float m (s = 1 for m = 0; s and
// its inverse r kept normal floats), and a float-float value scaled by a
// power of two.  Used where the square of a small quantity (b^2 of a weak
// field) would leave the float range.
__device__ __forceinline__ void pow2_scale(float m, float& s, float& r) {
  int eb = m > 0.f ? (int)((__float_as_uint(m) >> 23) & 0xff) : 127;
  eb = eb < 1 ? 1 : (eb > 253 ? 253 : eb);
  s = __uint_as_float((unsigned)(254 - eb) << 23);
  r = __uint_as_float((unsigned)eb << 23);
}
__device__ __forceinline__ ff scale2(ff a, float s) { return ff(a.hi * s, a.lo * s); }

// Conversions by bit manipulation and float arithmetic (no float64 and no
// integer-to-float conversion instruction, which share the narrow float64
// pipe): a double split into its leading 24 significant bits (hi, truncated)
// and the float nearest to the remaining 29 (lo); a float widened exactly
// to double.  Values outside the normal float range take the float64 route.
// The float64 route, kept out of line so that the compiler cannot predicate
// its float64 instructions into the common path.
static __device__ __noinline__ ff ff_split_wide(double d) { return ff(d); }
__device__ __forceinline__ ff ff_split(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return ff(0.f, 0.f);
  // fast path for 2^-74 <= |d| < 2^100: every float below stays normal
  if (e < 1075 - 126 || e > 1023 + 100) return ff_split_wide(d);
  const unsigned sign = (unsigned)(b >> 63);
  const unsigned long long m = b & 0xfffffffffffffull;
  const float hi = __uint_as_float((sign << 31) | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(m >> 29));
  // the low 29 bits x = 64 xh + xl are worth x 2^(e - 1075): each part is
  // made exact as (2^23 + part) 2^k - 2^23 2^k from its bits, and one float
  // addition rounds their sum
  const unsigned x = (unsigned)(m & 0x1fffffffull);
  const unsigned eh = (unsigned)(e - 1069 + 150) << 23, el = (unsigned)(e - 1075 + 150) << 23;
  const float ph = __uint_as_float(eh | (x >> 6)) - __uint_as_float(eh);
  const float pl = __uint_as_float(el | (x & 63u)) - __uint_as_float(el);
  const float lo = ph + pl;
  return ff(hi, sign ? -lo : lo);
}
__device__ __forceinline__ double f_widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xff;
  if (ef == 0) return 0.0;  // zero or a float denormal (below 1e-38)
  const unsigned long long s = (unsigned long long)(u >> 31) << 63;
  const unsigned long long e = (unsigned long long)(ef - 127 + 1023) << 52;
  const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(s | e | m));
}
__device__ __forceinline__ double ff_join(ff a) { return f_widen(a.hi) + f_widen(a.lo); }

// Conversions for the float32 Jacobian by bit manipulation, without a branch
// and without the conversion instructions of the narrow float64 pipe:
// double to float with the significand truncated to 24 bits (magnitudes
// below the normal float range become signed zeros, above it infinities),
// and float to double exactly (float denormals become zero).
// Infinities stay infinite and NaNs stay NaN (a quiet NaN) both ways, so a
// float32 solve that overflowed is seen as such by the caller.
__device__ __forceinline__ float d2f_jac(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int ed = (int)((b >> 52) & 0x7ff);
  const int e = ed - 896;
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const unsigned long long md = b & 0xfffffffffffffull;
  const unsigned mag = (unsigned)e << 23 | (unsigned)(md >> 29);
  const unsigned special = sign | 0x7f800000u | (md != 0ull ? 0x400000u : 0u);  // inf or NaN
  const unsigned r = ed == 0x7ff ? special : (e < 1 ? sign : (e > 254 ? (sign | 0x7f800000u) : (sign | mag)));
  return __uint_as_float(r);
}
__device__ __forceinline__ double f2d_jac(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xff;
  const unsigned long long s = (unsigned long long)(u >> 31) << 63;
  const unsigned long long ed = ef == 0xffu ? 0x7ffull : (unsigned long long)(ef + 896);
  const unsigned long long v = s | ed << 52 | (unsigned long long)(u & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(ef == 0 ? s : v));
}

// Input in the working precision: float64 as is, float-float by the split,
// float (the float32 Jacobian's) by truncation.
template <typename T> __device__ __forceinline__ T from_double(double d);
template <> __device__ __forceinline__ double from_double<double>(double d) { return d; }
template <> __device__ __forceinline__ float from_double<float>(double d) { return d2f_jac(d); }
template <> __device__ __forceinline__ ff from_double<ff>(double d) { return ff_split(d); }

// Generalized minmod slope (Section 2.4.1) of vm, v0, vp in float-float, for
// the limited slopes of the mixed solver (sign tests on the leading parts).
__device__ __forceinline__ ff gm_slope(ff theta, ff vm, ff v0, ff vp) {
  const ff a = v0 - vm, c = vp - v0;
  if (!((a.hi > 0.f && c.hi > 0.f) || (a.hi < 0.f && c.hi < 0.f))) return ff(0.f, 0.f);
  const ff m = fmin(theta * fmin(fabs(a), fabs(c)), tconst<ff>(0.5) * fabs(a + c));
  return a.hi > 0.f ? m : -m;
}

// ---------------------------------------------------------------- paired lanes
// Two float-float values evaluated together (lane x and lane y: the left and
// right states of a face), on Blackwell's paired float32 instructions: FADD2,
// FMUL2 and FFMA2 act on both lanes of a float2 at once, so the same
// error-free transformations as ff above take one instruction stream for
// two values.  Square roots, reciprocals and comparisons act lane by lane.
struct ff2 {
  float2 hi, lo;
  ff2() = default;
  __host__ __device__ constexpr ff2(float hx, float hy, float lx, float ly) : hi{hx, hy}, lo{lx, ly} {}
  __device__ __forceinline__ ff2(float2 h, float2 l) : hi(h), lo(l) {}
  __device__ __forceinline__ ff2(ff a, ff b) : hi(make_float2(a.hi, b.hi)), lo(make_float2(a.lo, b.lo)) {}
  __device__ __forceinline__ explicit ff2(int i) : hi(make_float2((float)i, (float)i)), lo(make_float2(0.f, 0.f)) {}
  __device__ __forceinline__ ff x() const { return ff(hi.x, lo.x); }
  __device__ __forceinline__ ff y() const { return ff(hi.y, lo.y); }
};
template <> __host__ __device__ constexpr ff2 tconst<ff2>(double x) {
  return ff2(static_cast<float>(x), static_cast<float>(x), static_cast<float>(x - static_cast<double>(static_cast<float>(x))),
             static_cast<float>(x - static_cast<double>(static_cast<float>(x))));
}

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// s + e with |s| >= |e| in each lane: the normalised pairs (ff_quick).
__device__ __forceinline__ ff2 ff2_quick(float2 s, float2 e) {
  const float2 h = add2(s, e);
  return ff2(h, sub2(e, sub2(h, s)));
}
__device__ __forceinline__ ff2 operator-(ff2 a) { return ff2(neg2(a.hi), neg2(a.lo)); }
// Dekker's sum as for ff: Knuth's two-sum of the leading parts, the low
// parts added in plain float.
__device__ __forceinline__ ff2 operator+(ff2 x, ff2 y) {
  const float2 s = add2(x.hi, y.hi);
  const float2 v = sub2(s, x.hi);
  const float2 e = add2(sub2(x.hi, sub2(s, v)), sub2(y.hi, v));
  return ff2_quick(s, add2(e, add2(x.lo, y.lo)));
}
__device__ __forceinline__ ff2 operator-(ff2 x, ff2 y) { return x + (-y); }
__device__ __forceinline__ ff2 operator*(ff2 x, ff2 y) {
  const float2 p = mul2(x.hi, y.hi);
  float2 e = fma2(x.hi, y.hi, neg2(p));
  e = fma2(x.hi, y.lo, e);
  e = fma2(x.lo, y.hi, e);
  return ff2_quick(p, e);
}
__device__ __forceinline__ ff2& operator+=(ff2& a, ff2 b) { a = a + b; return a; }
__device__ __forceinline__ ff2& operator-=(ff2& a, ff2 b) { a = a - b; return a; }
__device__ __forceinline__ ff2& operator*=(ff2& a, ff2 b) { a = a * b; return a; }

__device__ __forceinline__ ff2 fmax(ff2 a, ff2 b) { return ff2(fmax(a.x(), b.x()), fmax(a.y(), b.y())); }
__device__ __forceinline__ ff2 fmin(ff2 a, ff2 b) { return ff2(fmin(a.x(), b.x()), fmin(a.y(), b.y())); }
__device__ __forceinline__ ff2 fabs(ff2 a) { return ff2(fabs(a.x()), fabs(a.y())); }
// Lane by lane: keep lane x where kx, lane y where ky, zero elsewhere.
__device__ __forceinline__ ff2 keep(ff2 a, bool kx, bool ky) {
  return ff2(make_float2(kx ? a.hi.x : 0.f, ky ? a.hi.y : 0.f), make_float2(kx ? a.lo.x : 0.f, ky ? a.lo.y : 0.f));
}
__device__ __forceinline__ ff2 scale2(ff2 a, float2 s) { return ff2(mul2(a.hi, s), mul2(a.lo, s)); }

// The generalized minmod of gm_slope above for two zones at once (lane x:
// vm, v0, vp of one zone, lane y of the other): the differences, the
// limiter's product and the sum on paired instructions, the sign tests and
// the minimum lane by lane.
__device__ __forceinline__ ff2 gm_slope2(ff theta, ff2 vm, ff2 v0, ff2 vp) {
  const ff2 a = v0 - vm, c = vp - v0;
  const bool kx = (a.hi.x > 0.f && c.hi.x > 0.f) || (a.hi.x < 0.f && c.hi.x < 0.f);
  const bool ky = (a.hi.y > 0.f && c.hi.y > 0.f) || (a.hi.y < 0.f && c.hi.y < 0.f);
  const ff2 m = fmin(ff2(theta, theta) * fmin(fabs(a), fabs(c)), tconst<ff2>(0.5) * fabs(a + c));
  const ff mx = m.x(), my = m.y();
  return keep(ff2(a.hi.x > 0.f ? mx : -mx, a.hi.y > 0.f ? my : -my), kx, ky);
}

// 1/y, sqrt(a) and a^(-1/2) as for ff, each lane's float estimate refined
// by the paired float-float step.
__device__ __forceinline__ ff2 nr_rcp(ff2 y) {
  const ff2 x(make_float2(__frcp_rn(y.hi.x), __frcp_rn(y.hi.y)), make_float2(0.f, 0.f));
  return x + x * (tconst<ff2>(1.0) - y * x);
}
__device__ __forceinline__ ff2 sqr_root(ff2 a) {
  const bool px = a.hi.x > 0.f, py = a.hi.y > 0.f;
  const float2 s = make_float2(px ? __fsqrt_rn(a.hi.x) : 1.f, py ? __fsqrt_rn(a.hi.y) : 1.f);
  const ff2 S(s, make_float2(0.f, 0.f));
  const ff2 r = a - S * S;
  return keep(ff2_quick(s, mul2(r.hi, make_float2(0.5f / s.x, 0.5f / s.y))), px, py);
}
__device__ __forceinline__ ff2 rsq(ff2 a) {
  const ff2 y(make_float2(rsqrtf(a.hi.x), rsqrtf(a.hi.y)), make_float2(0.f, 0.f));
  return y + (y * tconst<ff2>(0.5)) * (tconst<ff2>(1.0) - (a * y) * y);
}

}  // namespace grim
