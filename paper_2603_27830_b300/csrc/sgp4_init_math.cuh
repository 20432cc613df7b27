// Initialisation constants of near-Earth SGP4 as a function of the mean elements,
// (x^(2/3) as cbrt(x^2), x^3.5 as x^3 sqrt(x), one sincos per angle: the record
// build runs on B300's small FP64 unit, so its operation count is its cost),
// templated on the scalar: double for the record builder, Dual7<double> or
// Dual7<float> (value + derivatives with respect to the 7 elements) for the Jacobian
// the adjoint needs.  Equations of
// Spacetrack Report #3 as revised in 2006 (paper Sec. 2.1); readings: a0'' from
// n0'' by Kepler's third law, D4 with a0''^2.
#pragma once

#include <cmath>

#include "sgp4_device.cuh"

namespace sgp4 {

// Forward-mode dual number with 7 tangent directions (n0, e0, i0, RAAN0, argp0, M0, B*)
// over the scalar R: double for the FP64 paths, float for the Jacobians of the FP32
// adjoint (B300's FP32 lanes are 64 times its FP64 rate).
template <class R>
struct Dual7 {
  R v;
  R d[7];
};
using D7 = Dual7<double>;

// Scalar functions of R (the float versions are the accurate library ones, not the
// SFU intrinsics).
__device__ __forceinline__ double sc_sin(double x) { return ::sin(x); }
__device__ __forceinline__ float sc_sin(float x) { return ::sinf(x); }
__device__ __forceinline__ double sc_cos(double x) { return ::cos(x); }
__device__ __forceinline__ float sc_cos(float x) { return ::cosf(x); }
__device__ __forceinline__ double sc_sqrt(double x) { return ::sqrt(x); }
__device__ __forceinline__ float sc_sqrt(float x) { return ::sqrtf(x); }
__device__ __forceinline__ double sc_pow(double x, double p) { return ::pow(x, p); }
__device__ __forceinline__ float sc_pow(float x, float p) { return ::powf(x, p); }
__device__ __forceinline__ double sc_cbrt(double x) { return ::cbrt(x); }
__device__ __forceinline__ float sc_cbrt(float x) { return ::cbrtf(x); }
__device__ __forceinline__ double sc_rsqrt(double x) { return ::rsqrt(x); }
__device__ __forceinline__ float sc_rsqrt(float x) { return ::rsqrtf(x); }
__device__ __forceinline__ void sc_sincos(double x, double* s, double* c) { ::sincos(x, s, c); }
__device__ __forceinline__ void sc_sincos(float x, float* s, float* c) { ::sincosf(x, s, c); }

template <class R>
__device__ __forceinline__ Dual7<R> d7c(R x) {
  Dual7<R> r;
  r.v = x;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = R(0);
  return r;
}
template <class R>
__device__ __forceinline__ Dual7<R> d7var(R x, int k) {
  Dual7<R> r = d7c(x);
  r.d[k] = R(1);
  return r;
}
template <class R>
__device__ __forceinline__ Dual7<R> d7chain(const Dual7<R>& a, R val, R dfda) {
  Dual7<R> r;
  r.v = val;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = dfda * a.d[k];
  return r;
}
template <class R>
__device__ __forceinline__ Dual7<R> operator+(const Dual7<R>& a, const Dual7<R>& b) {
  Dual7<R> r; r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <class R>
__device__ __forceinline__ Dual7<R> operator-(const Dual7<R>& a, const Dual7<R>& b) {
  Dual7<R> r; r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <class R>
__device__ __forceinline__ Dual7<R> operator-(const Dual7<R>& a) {
  Dual7<R> r; r.v = -a.v;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = -a.d[k];
  return r;
}
template <class R>
__device__ __forceinline__ Dual7<R> operator*(const Dual7<R>& a, const Dual7<R>& b) {
  Dual7<R> r; r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <class R>
__device__ __forceinline__ Dual7<R> operator/(const Dual7<R>& a, const Dual7<R>& b) {
  Dual7<R> r; r.v = a.v / b.v;
  const R ib = R(1) / b.v;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <class R>
__device__ __forceinline__ Dual7<R> operator+(const Dual7<R>& a, double b) {
  Dual7<R> r = a; r.v += R(b); return r;
}
template <class R>
__device__ __forceinline__ Dual7<R> operator+(double a, const Dual7<R>& b) { return b + a; }
template <class R>
__device__ __forceinline__ Dual7<R> operator-(const Dual7<R>& a, double b) {
  Dual7<R> r = a; r.v -= R(b); return r;
}
template <class R>
__device__ __forceinline__ Dual7<R> operator-(double a, const Dual7<R>& b) { return -b + a; }
template <class R>
__device__ __forceinline__ Dual7<R> operator*(const Dual7<R>& a, double b) {
  return d7chain(a, a.v * R(b), R(b));
}
template <class R>
__device__ __forceinline__ Dual7<R> operator*(double a, const Dual7<R>& b) { return b * a; }
template <class R>
__device__ __forceinline__ Dual7<R> operator/(const Dual7<R>& a, double b) {
  return a * (1.0 / b);
}
template <class R>
__device__ __forceinline__ Dual7<R> operator/(double a, const Dual7<R>& b) {
  const R q = R(a) / b.v;
  return d7chain(b, q, -q / b.v);
}
template <class R>
__device__ __forceinline__ Dual7<R> sin(const Dual7<R>& a) {
  return d7chain(a, sc_sin(a.v), sc_cos(a.v));
}
template <class R>
__device__ __forceinline__ Dual7<R> cos(const Dual7<R>& a) {
  return d7chain(a, sc_cos(a.v), -sc_sin(a.v));
}
template <class R>
__device__ __forceinline__ Dual7<R> sqrt(const Dual7<R>& a) {
  const R s = sc_sqrt(a.v);
  return d7chain(a, s, R(0.5) / s);
}
template <class R>
__device__ __forceinline__ Dual7<R> rsqrt(const Dual7<R>& a) {
  const R r = sc_rsqrt(a.v);
  return d7chain(a, r, R(-0.5) * r * r * r);
}
template <class R>
__device__ __forceinline__ Dual7<R> pow(const Dual7<R>& a, double p) {
  const R y = sc_pow(a.v, R(p));
  return d7chain(a, y, R(p) * y / a.v);
}
template <class R>
__device__ __forceinline__ Dual7<R> fabs(const Dual7<R>& a) { return a.v < R(0) ? -a : a; }
template <class R>
__device__ __forceinline__ Dual7<R> cbrt(const Dual7<R>& a) {
  const R y = sc_cbrt(a.v);
  return d7chain(a, y, y / (R(3) * a.v));
}
template <class R>
__device__ __forceinline__ void sincos(const Dual7<R>& a, Dual7<R>* s, Dual7<R>* c) {
  R sv, cv;
  sc_sincos(a.v, &sv, &cv);
  *s = d7chain(a, sv, cv);
  *c = d7chain(a, cv, -sv);
}
template <class R>
__device__ __forceinline__ R val(const Dual7<R>& a) { return a.v; }
__device__ __forceinline__ double val(double a) { return a; }
// Exact float -> double with integer operations (normal floats and zero; the values
// passed are FP32 approximations of positive normal doubles).
__device__ __forceinline__ double f64_exact(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}

// Cube root of the positive doubles of the record build, (ke/n)^(2/3) = cbrt((ke/n)^2):
// an FP32 seed refined by two Newton steps y <- y - (y^3 - x) / (3 y^2) in FP64 with the
// reciprocal of 3 y^2 taken in FP32.  Each step multiplies the relative error by about
// that reciprocal's error (1e-7) and adds its square, so two steps take a 1e-7 seed to
// the last bits of a double.  Outside [1e-30, 1e30] the library's cbrt.  On B300 this
// is a dozen FP64-unit instructions; the record build is bound by that unit.
__device__ __forceinline__ double cbrt_pos(double x) {
  if (!(x > 1.0e-30 && x < 1.0e30)) return ::cbrt(x);
  double y = f64_exact(::cbrtf(f32_rn(x)));
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double y2 = y * y;
    const double r = f64_exact(1.0f / (3.0f * f32_rn(y2)));
    y = fma(-fma(y2, y, -x), r, y);
  }
  return y;
}
template <class R>
__device__ __forceinline__ Dual7<R> cbrt_pos(const Dual7<R>& a) { return cbrt(a); }

// Keep the double versions visible next to the dual overloads in this namespace.
using ::cbrt;
using ::cos;
using ::fabs;
using ::pow;
using ::rsqrt;
using ::sin;
using ::sincos;
using ::sqrt;

// The 33 record fields the propagation reads, plus C1 for the FP32 row.
template <class S>
struct InitFields {
  S n0pp, a0pp, e0, i0, raan0, argp0, m0;
  S mdot, argpdot, raandot, raan_cf, argp_cf, m_cf;
  S c1, bc4, bc5, d2, d3, d4, l2, l3, l4, l5;
  S eta, delm0, sinm0, xlcof, aycof;
  S cosi, sini, x3thm1, x1mth2, x7thm1;
  S raandot1;   // first-order node rate (for raan_cf), not a record field
  bool isimp;
};

// The computation comes in phases, so that the record-build kernel can run the two
// independent branches of it (drag terms; secular rates) in two warps:
//   init_spine   inclination terms, beta0, the un-Kozai'd mean motion and a0'' (in
//                parts: init_spine_a, the terms in n0 and e0 alone; init_spine_i, the
//                inclination terms; init_spine_b, the recovery, needing both);
//   init_angles  sin/cos of argp0 and M0 (independent of the spine);
//   init_drag    atmosphere, C1 .. C5, D2 .. L5 and the drag rates (spine, angles), in
//                three parts: init_drag_core (atmosphere, xi, eta, the C factors), then
//                init_drag_c (C3, C4, C5 and their terms) and init_drag_d (C1, D, L),
//                which are independent of each other;
//   init_rates   secular rates and the J3 coefficients (spine);
//   init_finish  the node drag term (drag and rates) and the element copies.
// Reciprocals and square roots are formed from a few rsqrt and divisions and reused (on
// B300 each FP64 division or square root is a chain of FP64-unit instructions, and the
// record build is bound by that chain).
template <class S>
struct InitSpine {
  S cosi, sini, th2, x3thm1, x1mth2, x7thm1, b2, rb, b, n0pp, a0pp, ia0pp;
};
template <class S>
struct InitAngles {
  S sinw, cosw, sinm, cosm;
};

// The spine's terms in n0 and e0 alone: n0 / ke, its reciprocal, a1 = (ke/n0)^(2/3) and
// beta0 (independent of the inclination, so a second warp can take them).
template <class S>
struct SpineA {
  S n0k, x1, a1, b2, rb, b;
};

// Valid elements only (the caller screens non-finite input, e0 outside [0,1), n0 <= 0).
template <class S>
__device__ __forceinline__ void init_spine_a(const S el[7], const Geo& g, SpineA<S>& sa) {
  const S n0 = el[0], e0 = el[1];
  sa.b2 = 1.0 - e0 * e0;
  sa.rb = rsqrt(sa.b2);                       // 1 / beta0
  sa.b = sa.b2 * sa.rb;
  sa.n0k = n0 * g.inv_xke;                    // n0 / ke = 1 / x1
  sa.x1 = 1.0 / sa.n0k;
  sa.a1 = cbrt_pos(sa.x1 * sa.x1);            // (ke / n0)^(2/3); 1 / a1^2 = a1 (n0 / ke)^2
}

// The inclination terms, then the Kozai -> Brouwer recovery (needs SpineA).
template <class S>
__device__ __forceinline__ void init_spine_i(const S el[7], InitSpine<S>& sp) {
  sincos(el[2], &sp.sini, &sp.cosi);
  sp.th2 = sp.cosi * sp.cosi;
  sp.x3thm1 = 3.0 * sp.th2 - 1.0;
  sp.x1mth2 = 1.0 - sp.th2;
  sp.x7thm1 = 7.0 * sp.th2 - 1.0;
}

template <class S>
__device__ __forceinline__ void init_spine_b(const S el[7], const Geo& g, const SpineA<S>& sa,
                                             InitSpine<S>& sp) {
  const S n0 = el[0];
  const double k2 = 0.5 * g.j2;
  sp.b2 = sa.b2; sp.rb = sa.rb; sp.b = sa.b;
  // Kozai -> Brouwer mean motion and semi-major axis.
  const S n0k = sa.n0k, a1 = sa.a1;
  const S c3b = 1.5 * k2 * sp.x3thm1 * (sp.rb * sp.rb * sp.rb);
  const S d1 = c3b * a1 * (n0k * n0k);
  const S a0 = a1 * (1.0 - d1 * (1.0 / 3.0) - d1 * d1 - (134.0 / 81.0) * d1 * d1 * d1);
  const S ia0 = 1.0 / a0;
  const S d0 = c3b * (ia0 * ia0);
  const S opd0 = 1.0 + d0;
  sp.n0pp = n0 / opd0;
  const S xpp = sa.x1 * opd0;                 // ke / n0''
  sp.a0pp = cbrt_pos(xpp * xpp);              // (ke / n0'')^(2/3)
  const S npk = sp.n0pp * g.inv_xke;
  sp.ia0pp = (sp.a0pp * sp.a0pp) * (npk * npk);   // 1 / a0'' = a0''^2 (n0'' / ke)^2
}

template <class S>
__device__ __forceinline__ void init_spine(const S el[7], const Geo& g, InitSpine<S>& sp) {
  SpineA<S> sa;
  init_spine_a(el, g, sa);
  init_spine_i(el, sp);
  init_spine_b(el, g, sa, sp);
}

template <class S>
__device__ __forceinline__ void init_angles(const S el[7], InitAngles<S>& an) {
  sincos(el[4], &an.sinw, &an.cosw);
  sincos(el[5], &an.sinm, &an.cosm);
}

// Atmosphere and the drag coefficients' common factors (spine).
template <class S>
struct DragCore {
  S ss, xi, eta, ipsi2, coef, coef1;
  bool isimp;
};

template <class S>
__device__ __forceinline__ void init_drag_core(const S el[7], const Geo& g,
                                               const InitSpine<S>& sp, DragCore<S>& dc) {
  const S e0 = el[1];
  const double inv_re = g.inv_re;
  const S a0pp = sp.a0pp;
  // Atmosphere: s and (q0 - s)^4 by perigee height.
  const S rp_er = a0pp * (1.0 - e0);
  const S hp = (rp_er - 1.0) * g.re;
  // Truncated drag: perigee below 220 km, and every deep-space orbit (period 2 pi / n0''
  // of 225 min or more).
  dc.isimp = val(rp_er) < 1.0 + 220.0 * inv_re || kTwoPi / val(sp.n0pp) >= 225.0;
  S s_km = 0.0 * hp + 78.0;
  if (val(hp) < 156.0) s_km = hp - 78.0;
  if (val(hp) < 98.0) s_km = 0.0 * hp + 20.0;
  const S qs = (120.0 - s_km) * inv_re;
  const S qs4 = qs * qs * qs * qs;
  dc.ss = 1.0 + s_km * inv_re;
  dc.xi = 1.0 / (a0pp - dc.ss);
  dc.eta = a0pp * e0 * dc.xi;
  const S psi2 = fabs(1.0 - dc.eta * dc.eta);
  const S rpsi = rsqrt(psi2);
  dc.ipsi2 = rpsi * rpsi;                              // 1 / psi2
  const S xi4 = dc.xi * dc.xi * dc.xi * dc.xi;
  dc.coef = qs4 * xi4;
  dc.coef1 = dc.coef * (dc.ipsi2 * dc.ipsi2 * dc.ipsi2 * rpsi);   // coef / psi2^3.5
}

// C3, C4, C5 and the drag terms built on them: argp_cf, m_cf, B* C4, B* C5 (spine,
// angles, core; none of them feeds the D and L coefficients).
template <class S>
__device__ __forceinline__ void init_drag_c(const S el[7], const Geo& g, const InitSpine<S>& sp,
                                            const InitAngles<S>& an, const DragCore<S>& dc,
                                            InitFields<S>& o) {
  const S e0 = el[1], bstar = el[6];
  const S a0pp = sp.a0pp, n0pp = sp.n0pp, b2 = sp.b2, x3thm1 = sp.x3thm1, x1mth2 = sp.x1mth2;
  const S eta = dc.eta, xi = dc.xi, ipsi2 = dc.ipsi2, coef = dc.coef, coef1 = dc.coef1;
  const S eta2 = eta * eta;
  const S eeta = e0 * eta;
  const S cos2w = 2.0 * an.cosw * an.cosw - 1.0;
  // C3 and the mean-anomaly drag term divide by e0 and by e0 eta; one reciprocal of e0
  // serves both (1 / eta = (a0'' - s) / (a0'' e0)).
  const bool e_big = val(e0) > 1.0e-4;
  const S ie0 = e_big ? 1.0 / e0 : 0.0 * e0;
  S C3 = 0.0 * e0;
  if (e_big) C3 = -2.0 * coef * xi * g.j3oj2 * n0pp * sp.sini * ie0;
  const S C4 = 2.0 * n0pp * coef1 * a0pp * b2 *
               (eta * (2.0 + 0.5 * eta2) + e0 * (0.5 + 2.0 * eta2) -
                g.j2 * xi * sp.ia0pp * ipsi2 *
                    (-3.0 * x3thm1 * (1.0 - 2.0 * eeta + eta2 * (1.5 - 0.5 * eeta)) +
                     0.75 * x1mth2 * (2.0 * eta2 - eeta * (1.0 + eta2)) * cos2w));
  const S C5 = 2.0 * coef1 * a0pp * b2 * (1.0 + 2.75 * (eta2 + eeta) + eeta * eta2);
  o.argp_cf = bstar * C3 * an.cosw;
  o.m_cf = 0.0 * e0;
  if (e_big) o.m_cf = -(2.0 / 3.0) * coef * bstar * (ie0 * ie0) * ((a0pp - dc.ss) * sp.ia0pp);
  o.bc4 = bstar * C4;
  o.bc5 = bstar * C5;
}

// C1 (through C2), the l2 and D / L coefficients, (1 + eta cos M0)^3, sin M0 (spine,
// angles, core).
template <class S>
__device__ __forceinline__ void init_drag_d(const S el[7], const Geo& g, const InitSpine<S>& sp,
                                            const InitAngles<S>& an, const DragCore<S>& dc,
                                            InitFields<S>& o) {
  const S e0 = el[1], bstar = el[6];
  const S a0pp = sp.a0pp, n0pp = sp.n0pp, x3thm1 = sp.x3thm1;
  const S eta = dc.eta, xi = dc.xi, ss = dc.ss;
  const S eta2 = eta * eta;
  const S eeta = e0 * eta;
  const S C2 = dc.coef1 * n0pp *
               (a0pp * (1.0 + 1.5 * eta2 + eeta * (4.0 + eta2)) +
                0.375 * g.j2 * xi * dc.ipsi2 * x3thm1 * (8.0 + 3.0 * eta2 * (8.0 + eta2)));
  const S C1 = bstar * C2;
  o.isimp = dc.isimp;
  o.l2 = 1.5 * C1;
  const S cm = 1.0 + eta * an.cosm;
  o.delm0 = cm * cm * cm;
  o.sinm0 = an.sinm;
  o.d2 = 0.0 * C1; o.d3 = o.d2; o.d4 = o.d2; o.l3 = o.d2; o.l4 = o.d2; o.l5 = o.d2;
  if (!dc.isimp) {
    const S c1sq = C1 * C1;
    o.d2 = 4.0 * a0pp * xi * c1sq;
    o.d3 = (4.0 / 3.0) * a0pp * xi * xi * (17.0 * a0pp + ss) * c1sq * C1;
    o.d4 = (2.0 / 3.0) * a0pp * a0pp * xi * xi * xi * (221.0 * a0pp + 31.0 * ss) * c1sq * c1sq;
    o.l3 = o.d2 + 2.0 * c1sq;
    o.l4 = 0.25 * (3.0 * o.d3 + 12.0 * C1 * o.d2 + 10.0 * c1sq * C1);
    o.l5 = 0.2 * (3.0 * o.d4 + 12.0 * C1 * o.d3 + 6.0 * o.d2 * o.d2 + 30.0 * c1sq * o.d2 +
                  15.0 * c1sq * c1sq);
  }
  o.c1 = C1;
  o.eta = eta;
}

template <class S>
__device__ __forceinline__ void init_drag(const S el[7], const Geo& g, const InitSpine<S>& sp,
                                          const InitAngles<S>& an, InitFields<S>& o) {
  DragCore<S> dc;
  init_drag_core(el, g, sp, dc);
  init_drag_c(el, g, sp, an, dc, o);
  init_drag_d(el, g, sp, an, dc, o);
}

template <class S>
__device__ __forceinline__ void init_rates(const Geo& g, const InitSpine<S>& sp,
                                           InitFields<S>& o) {
  const S n0pp = sp.n0pp, th2 = sp.th2, cosi = sp.cosi, sini = sp.sini, b = sp.b;
  const S pinv = sp.ia0pp * (sp.rb * sp.rb);  // 1 / (a0'' beta0^2)
  const S pinv2 = pinv * pinv;
  const S T1 = 1.5 * g.j2 * pinv2 * n0pp;
  const S T2 = 0.5 * T1 * g.j2 * pinv2;
  const S T3 = -0.46875 * g.j4 * pinv2 * pinv2 * n0pp;
  const S th4 = th2 * th2;
  o.mdot = n0pp + 0.5 * T1 * b * sp.x3thm1 + 0.0625 * T2 * b * (13.0 - 78.0 * th2 + 137.0 * th4);
  o.argpdot = -0.5 * T1 * (1.0 - 5.0 * th2) + 0.0625 * T2 * (7.0 - 114.0 * th2 + 395.0 * th4) +
              T3 * (3.0 - 36.0 * th2 + 49.0 * th4);
  o.raandot1 = -T1 * cosi;
  o.raandot = o.raandot1 + (0.5 * T2 * (4.0 - 19.0 * th2) + 2.0 * T3 * (3.0 - 7.0 * th2)) * cosi;

  S opc = 1.0 + cosi;
  if (::fabs((double)val(opc)) <= 1.5e-12) opc = 0.0 * opc + 1.5e-12;
  o.xlcof = -0.25 * g.j3oj2 * sini * (3.0 + 5.0 * cosi) / opc;
  o.aycof = -0.5 * g.j3oj2 * sini;
}

// raan_cf needs C1 (drag) and the first-order node rate (rates).
template <class S>
__device__ __forceinline__ void init_finish(const S el[7], const InitSpine<S>& sp,
                                            InitFields<S>& o) {
  o.raan_cf = 3.5 * sp.b2 * o.raandot1 * o.c1;
  o.n0pp = sp.n0pp; o.a0pp = sp.a0pp; o.e0 = el[1]; o.i0 = el[2]; o.raan0 = el[3];
  o.argp0 = el[4]; o.m0 = el[5];
  o.cosi = sp.cosi; o.sini = sp.sini; o.x3thm1 = sp.x3thm1; o.x1mth2 = sp.x1mth2;
  o.x7thm1 = sp.x7thm1;
}

// All phases in one thread (the dual-number Jacobians; the FP64 fallback paths).
template <class S>
__device__ __forceinline__ void init_fields(const S el[7], const Geo& g, InitFields<S>& o) {
  InitSpine<S> sp;
  InitAngles<S> an;
  init_spine(el, g, sp);
  init_angles(el, an);
  init_drag(el, g, sp, an, o);
  init_rates(g, sp, o);
  init_finish(el, sp, o);
}

}  // namespace sgp4
