// Forward pass of two states of one satellite in packed FP32, for the FP32 adjoint
// sweep (internal to the library).
//
// The FP32 adjoint recomputes each state forward and runs the reverse sweep of
// sgp4_sweep.cuh over it.  Like the FP32 propagation it is bound by instruction issue
// and by the traffic of its per-thread forward-value slot, so two states of the same
// satellite (consecutive times) run in one thread: every add, multiply and FMA is one
// packed instruction for both (__fadd2_rn, __fmul2_rn, __ffma2_rn and the packed
// subtract; transcendentals, compares and selects stay per state), and each forward
// value is one 8-byte word of the slot.  P2 is the pair type the generic reverse sweep
// runs on: its operators are the packed instructions without a rounding modifier, so
// that the code generator may fuse a product and a sum into one packed FMA, as it
// does for the scalar sweep.
//
// forward32x2 follows forward32 (same formulation, guard bands and status order, per
// state) except where the packed state of the propagation differs: the drag
// polynomials in Horner form and the small rotations with sin d = d (below 0.2 m).
// It never returns early for one state: a state outside the usable codes gets its
// code and garbage values, and its pair is swept state by state instead.
#pragma once

#include "sgp4_state32x2.cuh"
#include "sgp4_sweep.cuh"

namespace sgp4 {
namespace {

// A pair of FP32 values, one for each state of a packed pair.
struct P2 {
  float2 v;
  P2() = default;
  __device__ __forceinline__ P2(float a) : v(make_float2(a, a)) {}
  __device__ __forceinline__ explicit P2(float2 a) : v(a) {}
};

#define SGP4_P2_BINOP(NAME, OP)                                                        \
  __device__ __forceinline__ P2 NAME(P2 a, P2 b) {                                     \
    P2 d;                                                                              \
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"                                               \
        "mov.b64 pa, {%2, %3};\n\t"                                                    \
        "mov.b64 pb, {%4, %5};\n\t" OP " pd, pa, pb;\n\t"                              \
        "mov.b64 {%0, %1}, pd;\n\t}"                                                   \
        : "=f"(d.v.x), "=f"(d.v.y)                                                     \
        : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y));                             \
    return d;                                                                          \
  }
SGP4_P2_BINOP(operator+, "add.f32x2")
SGP4_P2_BINOP(operator-, "sub.f32x2")
SGP4_P2_BINOP(operator*, "mul.f32x2")
#undef SGP4_P2_BINOP

__device__ __forceinline__ P2 operator+(P2 a, float b) { return a + P2(b); }
__device__ __forceinline__ P2 operator+(float a, P2 b) { return P2(a) + b; }
__device__ __forceinline__ P2 operator-(P2 a, float b) { return a - P2(b); }
__device__ __forceinline__ P2 operator-(float a, P2 b) { return P2(a) - b; }
__device__ __forceinline__ P2 operator*(P2 a, float b) { return a * P2(b); }
__device__ __forceinline__ P2 operator*(float a, P2 b) { return P2(a) * b; }
__device__ __forceinline__ P2 operator-(P2 a) { return P2(0.0f) - a; }
__device__ __forceinline__ P2& operator+=(P2& a, P2 b) { return a = a + b; }
__device__ __forceinline__ P2 inv_pos(P2 x) { return P2(x2::rcp_pos(x.v)); }

// The packed sweep's slot: the forward values of Fwd, less four that its reverse sweep
// recomputes (1 - e^2, 1 + beta_L, 1 + eta cos M_DF and e_L cos E), so that the slot is
// 49 8-byte words (an odd count: conflict-free rows) and eight 64-thread blocks' slots
// fit in an SM's shared memory.
template <>
struct Fwd<P2> {
  P2 tt;
  P2 sMdf, cMdf, sMM, cMM;
  P2 tempa, templ, a, sqa, n, e, q, sw, cw, axn, ayn;
  P2 keep_e;
  P2 sp, cp, esinE, eL2, pL, rl, rdotl, sqp, rfdotl, betal, w, aor, As, Ac;
  P2 sinu, cosu, sin2u, cos2u, k, kp, fac, rk, nk, rdotk, rfdotk;
  P2 su, cu, sO, cO, si, ci;
  P2 pad;
};
__device__ __forceinline__ P2 fwd_om(const Fwd<P2>& f) { return P2(1.0f) - f.e * f.e; }
__device__ __forceinline__ P2 fwd_opb(const Fwd<P2>& f) { return P2(1.0f) + f.betal; }
__device__ __forceinline__ P2 fwd_ecosE(const Fwd<P2>& f) { return f.axn * f.cp + f.ayn * f.sp; }
__device__ __forceinline__ P2 fwd_c(const Fwd<P2>& f, const RevC<float>& rc) {
  return P2(1.0f) + rc.eta * f.cMdf;
}

// Per-state status of a packed forward pass where the second time is absent (an odd
// number of times): neither swept nor queued.
constexpr int kAbsentState = -2;

// Forward pass of the states at times (th.x + tl.x, th.y + tl.y) (minutes, split as in
// split_double) into the slot f; code[l] is state l's status, kRecomputeFP64 for a
// guard-band state (the order of the checks as in forward32).
__device__ __forceinline__ void forward32x2(const Rec32& rc, const GeoF& g, float2 th,
                                            float2 tl, Fwd<P2>& f, int code[2]) {
  using namespace x2;
  const int fatal = (rc.flags >> kFatalShift) & 0xff;
  const int code0 = fatal ? fatal : ((rc.flags & kFlagN0ppNonPos) ? 2 : 0);
  if (code0) {
    code[0] = code0;
    code[1] = code0;
    return;
  }
  const F2 t = th;
  f.tt = P2(t);
  const F2 t2 = mul(t, t);
  // tempa = 1 - C1 t - D2 t^2 - D3 t^3 - D4 t^4 and the mean-longitude drag polynomial
  // L2 t^2 + .. + L5 t^5, in Horner form (a simplified-drag record carries zero D, L3..L5
  // and B* C5 terms)
  F2 h = fma(S(rc.d4), t, S(rc.d3));
  h = fma(h, t, S(rc.d2));
  h = fma(h, t, S(rc.c1));
  const F2 tempa = sub(S(1.0f), mul(h, t));
  F2 hl = fma(S(rc.l5), t, S(rc.l4));
  hl = fma(hl, t, S(rc.l3));
  hl = fma(hl, t, S(rc.l2));
  const F2 templ = mul(hl, t2);
  F2 tempe = mul(S(rc.bc4), t);
  F2 dd = S(0.0f);
  if (!(rc.flags & kFlagIsimp)) {
    const F2 mdf = mul(wrap_rev(fma(S(rc.mdr), t, S(rc.m0r))), S(kTwoPiF));
    F2 s, c;
    sincos_sfu(mdf, s, c);
    f.sMdf = P2(s);
    f.cMdf = P2(c);
    const F2 cc = fma(S(rc.eta), c, S(1.0f));
    dd = fma(S(rc.mcf), sub(mul(mul(cc, cc), cc), S(rc.delm0)), mul(S(rc.argpcf), t));
    sincos_sfu(add(mdf, dd), s, c);
    f.sMM = P2(s);
    f.cMM = P2(c);
    tempe = fma(S(rc.bc5), sub(s, S(rc.sinm0)), tempe);
  }
  f.tempa = P2(tempa);
  f.templ = P2(templ);
  const F2 a = mul(S(rc.a0pp), mul(tempa, tempa));
  f.a = P2(a);
  const F2 e1 = sub(S(rc.e0), tempe);
  bool g_e[2], f_e[2];
  F2 e, keep;
  {
    const float ev[2] = {e1.x, e1.y}, av[2] = {a.x, a.y};
    float ek[2], kk[2];
    for (int l = 0; l < 2; ++l) {
      g_e[l] = !(fabsf(ev[l] - 1.0f) >= kGuardE && fabsf(ev[l] + 0.001f) >= kGuardE &&
                 av[l] > 1.0e-3f);
      f_e[l] = ev[l] >= 1.0f || ev[l] < -0.001f;
      kk[l] = ev[l] < 1.0e-6f ? 0.0f : 1.0f;
      ek[l] = fmaxf(ev[l], 1.0e-6f);
    }
    e = make_float2(ek[0], ek[1]);
    keep = make_float2(kk[0], kk[1]);
  }
  f.keep_e = P2(keep);
  f.e = P2(e);
  const F2 ra = rsqrt(a);
  f.sqa = P2(mul(a, ra));
  const F2 ra3 = mul(mul(ra, ra), ra);
  f.n = P2(mul(S(g.xke), ra3));

  // Phase of M + argp in revolutions: the n*t product as a double-float.
  F2 p = mul(S(rc.phidh), th);
  const F2 pe = fma(S(rc.phidh), th, mul(p, S(-1.0f)));     // exact rounding error of p
  const F2 s = fma(S(rc.phidh), tl, fma(S(rc.phidl), th, pe));
  p = wrap_rev(p);
  F2 y = wrap_rev(add(p, S(rc.phi0h)));
  y = add(y, add(s, S(rc.phi0l)));
  y = add(y, wrap_rev(mul(S(rc.n0ppr), templ)));
  const F2 argp =
      mul(wrap_rev(fma(dd, S(-kInvTwoPiF), fma(S(rc.argpdr), t, S(rc.argp0r)))), S(kTwoPiF));
  const F2 raan =
      mul(wrap_rev(fma(S(rc.raancfr), t2, fma(S(rc.raandr), t, S(rc.raan0r)))), S(kTwoPiF));

  // Long-period periodics (J3).
  F2 sw, cw;
  sincos_sfu(argp, sw, cw);
  f.sw = P2(sw);
  f.cw = P2(cw);
  const F2 axn = mul(e, cw);
  const F2 om = sub(S(1.0f), mul(e, e));
  const F2 q = rcp_pos(mul(a, om));
  const F2 ayn = fma(e, sw, mul(q, S(rc.aycof)));
  f.axn = P2(axn);
  f.q = P2(q);
  f.ayn = P2(ayn);
  const F2 lpt = mul(mul(q, S(rc.xlcof)), axn);
  const bool g_lp[2] = {!lt_abs(lpt.x, kGuardLongPeriod), !lt_abs(lpt.y, kGuardLongPeriod)};
  const F2 U = mul(wrap_rev(fma(lpt, S(kInvTwoPiF), y)), S(kTwoPiF));
  const F2 eL2 = fma(axn, axn, mul(ayn, ayn));
  f.eL2 = P2(eL2);

  // Kepler: Newton from psi = U, the step count of the pair's larger e_L.
  F2 psi = U;
  const int K = max(newton_steps(eL2.x), newton_steps(eL2.y));
  const F2 nayn = mul(ayn, S(-1.0f)), naxn = mul(axn, S(-1.0f));
  for (int k = 0; k < K; ++k) {
    F2 sp, cp;
    sincos_sfu(psi, sp, cp);
    const F2 fv = sub(fma(axn, sp, fma(nayn, cp, U)), psi);
    const F2 fp = fma(naxn, cp, fma(nayn, sp, S(1.0f)));
    const F2 st = mul(fv, rcp_pos(fp));
    psi = add(psi, make_float2(fminf(fmaxf(st.x, -0.95f), 0.95f),
                               fminf(fmaxf(st.y, -0.95f), 0.95f)));
  }
  F2 sp, cp;
  sincos_acc(psi.x, &sp.x, &cp.x);
  sincos_acc(psi.y, &sp.y, &cp.y);
  f.sp = P2(sp);
  f.cp = P2(cp);

  // Short-period preliminaries.
  const F2 ecosE = fma(axn, cp, mul(ayn, sp));
  const F2 esinE = fma(axn, sp, mul(nayn, cp));
  f.esinE = P2(esinE);
  const F2 omel = sub(S(1.0f), eL2);
  const F2 pL = mul(a, omel);
  f.pL = P2(pL);
  const bool g_p[2] = {!(fabsf(pL.x) >= kGuardP), !(fabsf(pL.y) >= kGuardP)};
  const bool f_p[2] = {pL.x < 0.0f, pL.y < 0.0f};
  const F2 rl = mul(a, sub(S(1.0f), ecosE));
  f.rl = P2(rl);
  const F2 invr = rcp_pos(rl);
  f.rdotl = P2(mul(mul(f.sqa.v, esinE), invr));
  const F2 rpl = rsqrt(pL);
  const F2 sqp = mul(pL, rpl);
  f.sqp = P2(sqp);
  const F2 rfdotl = mul(sqp, invr);
  f.rfdotl = P2(rfdotl);
  const F2 betal = mul(omel, rsqrt(omel));
  f.betal = P2(betal);
  const F2 opb = add(S(1.0f), betal);
  const F2 w = mul(esinE, rcp_pos(opb));
  f.w = P2(w);
  const F2 aor = mul(a, invr);
  f.aor = P2(aor);
  const F2 As = fma(naxn, w, sub(sp, ayn));
  const F2 Ac = fma(ayn, w, sub(cp, axn));
  f.As = P2(As);
  f.Ac = P2(Ac);
  const F2 sinu = mul(aor, As), cosu = mul(aor, Ac);
  f.sinu = P2(sinu);
  f.cosu = P2(cosu);
  const F2 sin2u = mul(mul(cosu, sinu), S(2.0f));
  const F2 cos2u = fma(mul(sinu, sinu), S(-2.0f), S(1.0f));
  f.sin2u = P2(sin2u);
  f.cos2u = P2(cos2u);

  // Short-period periodics (J2).
  const F2 invp = mul(rpl, rpl);
  const F2 k = mul(S(g.half_j2), invp);
  const F2 kp = mul(k, invp);
  f.k = P2(k);
  f.kp = P2(kp);
  const F2 fac = fma(mul(kp, betal), S(-rc.x3thm1_15), S(1.0f));
  f.fac = P2(fac);
  const F2 rk = fma(rl, fac, mul(mul(k, S(rc.half_x1mth2)), cos2u));
  f.rk = P2(rk);
  const bool g_r[2] = {!(fabsf(rk.x - 1.0f) >= kGuardR), !(fabsf(rk.y - 1.0f) >= kGuardR)};
  const F2 nk = mul(ra3, k);
  f.nk = P2(nk);
  f.rdotk = P2(fma(mul(nk, S(-rc.x1mth2)), sin2u, f.rdotl.v));
  f.rfdotk = P2(fma(nk, fma(S(rc.x1mth2), cos2u, S(rc.x3thm1_15)), rfdotl));

  // u_k, RAAN_k and i_k as small rotations of (sin, cos) pairs.
  const F2 du = mul(mul(kp, S(rc.x7thm1_m025)), sin2u);
  const F2 dO = mul(mul(kp, S(rc.c15cosi)), sin2u);
  const F2 di = mul(mul(kp, S(rc.c15cosisini)), cos2u);
  const bool g_d[2] = {
      !(fmaxf(fabsf(du.x), fmaxf(fabsf(dO.x), fabsf(di.x))) < 4.0e-3f),
      !(fmaxf(fabsf(du.y), fmaxf(fabsf(dO.y), fabsf(di.y))) < 4.0e-3f)};
  const F2 nrm = rsqrt(fma(sinu, sinu, mul(cosu, cosu)));
  F2 su = mul(sinu, nrm), cu = mul(cosu, nrm);
  rotate_small(su, cu, du);
  F2 sO, cO;
  sincos_sfu(raan, sO, cO);
  rotate_small(sO, cO, dO);
  F2 si = S(rc.sini), ci = S(rc.cosi);
  rotate_small(si, ci, di);
  f.su = P2(su); f.cu = P2(cu);
  f.sO = P2(sO); f.cO = P2(cO);
  f.si = P2(si); f.ci = P2(ci);

  const float rkv[2] = {rk.x, rk.y};
  for (int l = 0; l < 2; ++l) {
    int cd = rkv[l] < 1.0f ? 6 : 0;
    if (g_d[l]) cd = kRecomputeFP64;
    if (g_r[l]) cd = kRecomputeFP64;
    if (f_p[l]) cd = 4;
    if (g_p[l]) cd = kRecomputeFP64;
    if (g_lp[l]) cd = kRecomputeFP64;
    if (f_e[l]) cd = 1;
    if (g_e[l]) cd = kRecomputeFP64;
    code[l] = cd;
  }
}

}  // namespace
}  // namespace sgp4
