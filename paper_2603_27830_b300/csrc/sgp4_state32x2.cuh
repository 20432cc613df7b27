// Two states of one satellite in one thread, in packed FP32 arithmetic (internal to
// the library).
//
// B300's FP32 instructions come in a packed form that applies one add, multiply or
// FMA to a pair of floats (__fadd2_rn, __fmul2_rn, __ffma2_rn: two lanes of work per
// issue slot, each lane rounded as its scalar instruction).  The FP32 propagation is
// bound by instruction issue, so a pair of states of the same satellite (two times) is
// computed together (the kernels run one or two pairs per thread): the time-dependent
// values are pairs, the record's fields are shared scalars, and every add, multiply
// and FMA of the state is one packed instruction for both.  Transcendentals (SFU), compares, selects and the integer work
// stay per state.  The arithmetic is that of state32 (same formulation, guard bands and
// status logic); the fusing of products into FMAs, the evaluation order of the drag
// polynomials (Horner form) and the truncation of the small rotations and of the cosine
// polynomial (each below 0.2 m) differ.  A record field enters a packed operation as a
// pair of equal halves, so the formulas are arranged to avoid most negated fields and
// multiplications by -1 (each is one more instruction per use); the few left are the
// exact product error of the phase, the negated a_xN, a_yN and sin RAAN reused several
// times, and two record fields.
#pragma once

#include "sgp4_device.cuh"

namespace sgp4 {
namespace x2 {

using F2 = float2;

__device__ __forceinline__ F2 S(float a) { return make_float2(a, a); }
__device__ __forceinline__ F2 add(F2 a, F2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ F2 mul(F2 a, F2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) { return __ffma2_rn(a, b, c); }
// a - b, one rounding per lane (the packed subtract)
__device__ __forceinline__ F2 sub(F2 a, F2 b) {
  F2 d;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\t"
      "mov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pd, pa, pb;\n\t"
      "mov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// x - rint(x) by the 1.5 * 2^23 rounding trick, lane by lane exact for |x| < 2^22.
__device__ __forceinline__ F2 wrap_rev(F2 x) {
  const F2 r = sub(add(x, S(kRoundMagic)), S(kRoundMagic));
  return sub(x, r);
}

// rsqrt_ftz per lane (its arguments are normal numbers outside the guard bands)
__device__ __forceinline__ F2 rsqrt(F2 x) { return make_float2(rsqrt_ftz(x.x), rsqrt_ftz(x.y)); }
// 1 / y for y > 0 as rsqrt(y)^2
__device__ __forceinline__ F2 rcp_pos(F2 y) {
  const F2 r = rsqrt(y);
  return mul(r, r);
}
__device__ __forceinline__ void sincos_sfu(F2 x, F2& s, F2& c) {
  __sincosf(x.x, &s.x, &c.x);
  __sincosf(x.y, &s.y, &c.y);
}

// (s, c) = (sin a, cos a) -> (sin(a + d), cos(a + d)) for the small short-period
// corrections.  Callers check |d| < 4e-3, where sin d = d within |d|^3/6 < 1.1e-8 and
// cos d = 1 - d^2/2 within d^4/24 < 1.1e-11 (0.1 m and 0.1 mm at 7,000 km).
__device__ __forceinline__ void rotate_small(F2& s, F2& c, F2 d) {
  const F2 cd = fma(S(-0.5f), mul(d, d), S(1.0f));
  const F2 s2 = fma(s, cd, mul(c, d));
  const F2 c2 = sub(mul(c, cd), mul(s, d));
  s = s2;
  c = c2;
}

__device__ __forceinline__ bool lt_abs(float x, float lim) { return fabsf(x) < lim; }

}  // namespace x2

// Two states of one record at times (th.x + tl.x) and (th.y + tl.y).  Returns the two
// status codes (or kRecomputeFP64) in code[0], code[1]; r and v as pairs.
__device__ __forceinline__ void state32x2(const Rec32& rc, const GeoF& g, float2 th, float2 tl,
                                          float2 r[3], float2 v[3], int code[2]) {
  using namespace x2;
  const int fatal = (rc.flags >> kFatalShift) & 0xff;
  const int code0 = fatal ? fatal : ((rc.flags & kFlagN0ppNonPos) ? 2 : 0);
  const F2 t = th;
  const F2 t2 = mul(t, t);

  // Secular drag polynomials (simplified-drag records carry zero drag terms).
  const F2 dargp = mul(S(rc.argpcf), t);
  const F2 mdf = mul(wrap_rev(fma(S(rc.mdr), t, S(rc.m0r))), S(kTwoPiF));
  const F2 cm = make_float2(__cosf(mdf.x), __cosf(mdf.y));
  const F2 c = fma(S(rc.eta), cm, S(1.0f));
  const F2 dm = mul(S(rc.mcf), sub(mul(mul(c, c), c), S(rc.delm0)));
  const F2 dd = add(dargp, dm);
  // tempa = 1 - C1 t - D2 t^2 - D3 t^3 - D4 t^4 and the t^2 .. t^5 mean-longitude
  // polynomial, both in Horner form
  F2 h = fma(S(rc.d4), t, S(rc.d3));
  h = fma(h, t, S(rc.d2));
  h = fma(h, t, S(rc.c1));
  const F2 tempa = sub(S(1.0f), mul(h, t));
  const F2 md = add(mdf, dd);
  const F2 sm = make_float2(__sinf(md.x), __sinf(md.y));
  const F2 tempe = fma(S(rc.bc5), sub(sm, S(rc.sinm0)), mul(S(rc.bc4), t));
  F2 hl = fma(S(rc.l5), t, S(rc.l4));
  hl = fma(hl, t, S(rc.l3));
  hl = fma(hl, t, S(rc.l2));
  const F2 templ = mul(hl, t2);
  const F2 a = mul(S(rc.a0pp), mul(tempa, tempa));
  F2 e = sub(S(rc.e0), tempe);
  // Status checks in the theory's order and the guard bands, per lane.
  bool g_e[2], f_e[2];
  {
    const float ev[2] = {e.x, e.y}, av[2] = {a.x, a.y};
    for (int l = 0; l < 2; ++l) {
      g_e[l] = !(fabsf(ev[l] - 1.0f) >= kGuardE) | !(fabsf(ev[l] + 0.001f) >= kGuardE) |
               !(av[l] > 1.0e-3f);
      f_e[l] = (ev[l] >= 1.0f) | (ev[l] < -0.001f);
    }
  }
  e = make_float2(fmaxf(e.x, 1.0e-6f), fmaxf(e.y, 1.0e-6f));
  const F2 ra = rsqrt(a);
  const F2 sa = mul(a, ra);
  const F2 ra3 = mul(mul(ra, ra), ra);

  // Phase of M + argp in revolutions; the n*t product as a double-float.
  F2 p = mul(S(rc.phidh), th);
  const F2 pe = fma(S(rc.phidh), th, mul(p, S(-1.0f)));     // exact rounding error of p
  const F2 s = fma(S(rc.phidh), tl, fma(S(rc.phidl), th, pe));
  p = wrap_rev(p);                                             // exact
  F2 y = wrap_rev(add(p, S(rc.phi0h)));
  y = add(y, add(s, S(rc.phi0l)));
  const F2 lrev = mul(S(rc.n0ppr), templ);
  const bool g_l[2] = {!x2::lt_abs(lrev.x, kGuardDragPhase), !x2::lt_abs(lrev.y, kGuardDragPhase)};
  y = add(y, wrap_rev(lrev));

  const F2 argp =
      mul(wrap_rev(fma(dd, S(-kInvTwoPiF), fma(S(rc.argpdr), t, S(rc.argp0r)))), S(kTwoPiF));
  const F2 raan =
      mul(wrap_rev(fma(S(rc.raancfr), t2, fma(S(rc.raandr), t, S(rc.raan0r)))), S(kTwoPiF));

  // Long-period periodics (J3).
  F2 sw, cw;
  sincos_sfu(argp, sw, cw);
  const F2 axn = mul(e, cw);
  const F2 q = rcp_pos(mul(a, sub(S(1.0f), mul(e, e))));
  const F2 ayn = fma(e, sw, mul(q, S(rc.aycof)));
  const F2 lpt = mul(mul(q, S(rc.xlcof)), axn);
  const bool g_lp[2] = {!x2::lt_abs(lpt.x, kGuardLongPeriod), !x2::lt_abs(lpt.y, kGuardLongPeriod)};
  const F2 U = mul(wrap_rev(fma(lpt, S(kInvTwoPiF), y)), S(kTwoPiF));
  const F2 eL2 = fma(axn, axn, mul(ayn, ayn));

  // Kepler: Newton from psi = U, warp-uniform step count from the e_L bound.
  F2 psi = U;
  const int K = __reduce_max_sync(__activemask(),
                                  max(newton_steps(eL2.x), newton_steps(eL2.y)));
  const F2 nayn = mul(ayn, S(-1.0f)), naxn = mul(axn, S(-1.0f));
  for (int k = 0; k < K; ++k) {
    F2 sp, cp;
    sincos_sfu(psi, sp, cp);
    const F2 f = sub(fma(axn, sp, fma(nayn, cp, U)), psi);
    const F2 fp = fma(naxn, cp, fma(nayn, sp, S(1.0f)));
    const F2 st = mul(f, rcp_pos(fp));
    psi = add(psi, make_float2(fminf(fmaxf(st.x, -0.95f), 0.95f),
                               fminf(fmaxf(st.y, -0.95f), 0.95f)));
  }
  // The final iterate's sin and cos from the SFU as well: their error (a few 1e-7 rad
  // for psi in [-1, 2 pi + 1]) goes into the along-track position, but the accurate
  // polynomial pair cost 4% of the kernel's time for 0.6 m of maximum error on the
  // Starlink-shaped set (8.9 -> 9.5 m over a day; catalogue 13.9 -> 16.0 m over seven).
  F2 sp, cp;
  sincos_sfu(psi, sp, cp);

  // Short-period preliminaries.
  const F2 ecosE = fma(axn, cp, mul(ayn, sp));
  const F2 esinE = fma(axn, sp, mul(nayn, cp));
  const F2 omel = sub(S(1.0f), eL2);
  const F2 pL = mul(a, omel);
  const bool g_p[2] = {!(fabsf(pL.x) >= kGuardP), !(fabsf(pL.y) >= kGuardP)};
  const bool f_p[2] = {pL.x < 0.0f, pL.y < 0.0f};
  const F2 rl = mul(a, sub(S(1.0f), ecosE));
  const F2 invr = rcp_pos(rl);
  const F2 rdotl = mul(mul(sa, esinE), invr);
  const F2 rpl = rsqrt(pL);
  const F2 rfdotl = mul(mul(pL, rpl), invr);
  const F2 betal = mul(omel, rsqrt(omel));
  const F2 w = mul(esinE, rcp_pos(add(betal, S(1.0f))));
  const F2 aor = mul(a, invr);
  const F2 sinu = mul(aor, fma(naxn, w, sub(sp, ayn)));
  const F2 cosu = mul(aor, fma(ayn, w, sub(cp, axn)));
  const F2 sin2u = mul(mul(cosu, sinu), S(2.0f));
  const F2 cos2u = fma(mul(sinu, sinu), S(-2.0f), S(1.0f));

  // Short-period periodics (J2).
  const F2 invp = mul(rpl, rpl);
  const F2 k = mul(S(g.half_j2), invp);
  const F2 kp = mul(k, invp);
  const F2 rk = fma(rl, fma(mul(kp, betal), S(-rc.x3thm1_15), S(1.0f)),
                    mul(mul(k, S(rc.half_x1mth2)), cos2u));
  const bool g_r[2] = {!(fabsf(rk.x - 1.0f) >= kGuardR), !(fabsf(rk.y - 1.0f) >= kGuardR)};
  const F2 nk = mul(ra3, k);
  const F2 rdotk = fma(mul(nk, S(-rc.x1mth2)), sin2u, rdotl);
  const F2 rfdotk = fma(nk, fma(S(rc.x1mth2), cos2u, S(rc.x3thm1_15)), rfdotl);

  // u_k, RAAN_k and i_k as small rotations of (sin, cos) pairs.
  const F2 du = mul(mul(kp, S(rc.x7thm1_m025)), sin2u);
  const F2 dO = mul(mul(kp, S(rc.c15cosi)), sin2u);
  const F2 di = mul(mul(kp, S(rc.c15cosisini)), cos2u);
  const bool g_d[2] = {
      !(fmaxf(fabsf(du.x), fmaxf(fabsf(dO.x), fabsf(di.x))) < 4.0e-3f),
      !(fmaxf(fabsf(du.y), fmaxf(fabsf(dO.y), fabsf(di.y))) < 4.0e-3f)};
  const F2 nrm = rsqrt(fma(sinu, sinu, mul(cosu, cosu)));
  F2 su = mul(sinu, nrm), cu = mul(cosu, nrm);
  x2::rotate_small(su, cu, du);
  F2 sO, cO;
  sincos_sfu(raan, sO, cO);
  x2::rotate_small(sO, cO, dO);
  F2 si = S(rc.sini), ci = S(rc.cosi);
  x2::rotate_small(si, ci, di);

  const F2 nsO = mul(sO, S(-1.0f));
  const F2 mx = mul(nsO, ci), my = mul(cO, ci), mz = si;
  const F2 ux = fma(mx, su, mul(cO, cu)), uy = fma(my, su, mul(sO, cu)), uz = mul(mz, su);
  const F2 vx = sub(mul(mx, cu), mul(cO, su));
  const F2 vy = fma(my, cu, mul(nsO, su));
  const F2 vz = mul(mz, cu);
  const F2 rs = mul(rk, S(g.re));
  r[0] = mul(rs, ux); r[1] = mul(rs, uy); r[2] = mul(rs, uz);
  const F2 vk = S(g.vkmps);
  v[0] = mul(fma(rdotk, ux, mul(rfdotk, vx)), vk);
  v[1] = mul(fma(rdotk, uy, mul(rfdotk, vy)), vk);
  v[2] = mul(fma(rdotk, uz, mul(rfdotk, vz)), vk);

  const float rkv[2] = {rk.x, rk.y};
  for (int l = 0; l < 2; ++l) {
    const bool need64 =
        g_e[l] | (!f_e[l] & (g_lp[l] | g_l[l] | g_p[l] | (!f_p[l] & (g_r[l] | g_d[l]))));
    int cd = f_e[l] ? 1 : (f_p[l] ? 4 : (rkv[l] < 1.0f ? 6 : 0));
    cd = need64 ? kRecomputeFP64 : cd;
    code[l] = code0 ? code0 : cd;
  }
}

}  // namespace sgp4
