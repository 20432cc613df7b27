// Forward and reverse sweeps of one SGP4 state, shared by the adjoint, fit and
// Jacobian kernels (internal to the library).
//
// forward64 / forward32 recompute a state with the propagation kernels' formulations
// (FP32: the double-float n*t phase and the guard bands of state32) and keep the values
// the reverse sweep reads; reverse() turns output adjoints (g_r, g_v) into the adjoints
// of the 33 record fields, differentiating the Kepler solve at its root (implicit
// function theorem) and treating clamps and status decisions as constants (the
// derivative of the branch taken); init_jacobian gives d(field)/d(element) through
// sgp4init with dual numbers.
#pragma once

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "sgp4_device.cuh"
#include "sgp4_init_math.cuh"

namespace sgp4 {
namespace {

// Record fields, in Rec64 order.
enum AdjField {
  aN0pp, aA0pp, aE0, aI0, aRaan0, aArgp0, aM0, aMdot, aArgpdot, aRaandot, aRaanCf, aArgpCf,
  aMCf, aC1, aBC4, aBC5, aD2, aD3, aD4, aL2, aL3, aL4, aL5, aEta, aDelM0, aSinM0, aXlcof,
  aAycof, aCosi, aSini, aX3thm1, aX1mth2, aX7thm1, kNumAdj
};

constexpr int kAdjThreads = 128;
constexpr int kAdjWarps = kAdjThreads / 32;
// Resident blocks per SM asked of the register allocator for the FP32 fit step (one
// state per thread, its forward values in a 212-byte shared-memory slot per thread, 28 KB
// per block).  On B300 (sgp4_fit_step, 10,000 x 500, CUDA events): five blocks (96
// registers) 0.776 ms, six (80) 0.787, four (128) 0.780, three 0.853.  The packed adjoint
// and the Jacobian kernel choose their own.
constexpr int kAdjMinBlocksFP32 = 5;

// Values of the forward pass of one state that the reverse sweep reads (names as in
// the propagation: a, e, a_xN, a_yN, E, p_L, r, u and the short-period terms).  The
// FP32 kernels keep one per thread in shared memory (an odd number of 4-byte words, so
// that the 32 threads of a warp hit 32 different banks).
// The position and velocity unit vectors U, V and the rest of the output frame.
template <class T>
struct Frame {
  T mx, my, mz, Ux, Uy, Uz, Vx, Vy, Vz;
};

// Forward values that are cheap to recompute (the powers of t, the output frame): kept
// by the FP64 sweeps (registers; their time is the FP64 unit's), recomputed by the FP32
// ones (their time is the shared-memory traffic of the forward-value slot).
template <class T>
struct FwdKeep {};
template <>
struct FwdKeep<double> {
  double t2, t3, t4;
  Frame<double> fr;
};

template <class T>
struct Fwd : FwdKeep<T> {
  T tt;
  T sMdf, cMdf, c, sMM, cMM;   // sin/cos M_DF, 1 + eta cos M_DF, sin/cos(M_DF + dd)
  T tempa, templ, a, sqa, n, e, om, q, sw, cw, axn, ayn;
  T keep_e;                    // 0 where e was raised to 1e-6, else 1
  T sp, cp, ecosE, esinE, eL2, pL, rl, rdotl, sqp, rfdotl, betal, opb, w, aor, As, Ac;
  T sinu, cosu, sin2u, cos2u, k, kp, fac, rk, nk, rdotk, rfdotk;
  T su, cu, sO, cO, si, ci;
  T pad;
};
static_assert(sizeof(Fwd<float>) % 8 == 4, "odd word count for conflict-free rows");

// Forward values the reverse sweep reads through these accessors: kept in the slot by
// the scalar sweeps, recomputed from other slot values by the packed one (whose slot
// leaves them out).
template <class T>
__device__ __forceinline__ T fwd_om(const Fwd<T>& f) { return f.om; }
template <class T>
__device__ __forceinline__ T fwd_opb(const Fwd<T>& f) { return f.opb; }
template <class T>
__device__ __forceinline__ T fwd_ecosE(const Fwd<T>& f) { return f.ecosE; }
template <class T, class K>
__device__ __forceinline__ T fwd_c(const Fwd<T>& f, const K&) { return f.c; }

// Per-satellite constants of the reverse sweep.
template <class T>
struct RevC {
  T bc5, sinm0, mcf, delm0, eta, a0pp, xke, ixke, n0pp, xlcof, aycof;
  T x3thm1, x1mth2, x7thm1, cosi, sini, re, vk;
  bool isimp;
};

__device__ __forceinline__ RevC<double> rev_consts(const Rec64& rc, const Geo& g) {
  RevC<double> k;
  k.bc5 = rc.bc5; k.sinm0 = rc.sinm0; k.mcf = rc.m_cf; k.delm0 = rc.delm0; k.eta = rc.eta;
  k.a0pp = rc.a0pp; k.xke = g.xke; k.ixke = g.inv_xke; k.n0pp = rc.n0pp; k.xlcof = rc.xlcof;
  k.aycof = rc.aycof;
  k.x3thm1 = rc.x3thm1; k.x1mth2 = rc.x1mth2; k.x7thm1 = rc.x7thm1;
  k.cosi = rc.cosi; k.sini = rc.sini; k.re = g.re; k.vk = g.vkmps;
  k.isimp = rc.flags & kFlagIsimp;
  return k;
}

__device__ __forceinline__ RevC<float> rev_consts(const Rec32& rc, const GeoF& g) {
  RevC<float> k;
  k.bc5 = rc.bc5; k.sinm0 = rc.sinm0; k.mcf = rc.mcf; k.delm0 = rc.delm0; k.eta = rc.eta;
  k.a0pp = rc.a0pp; k.xke = g.xke; k.ixke = g.inv_xke; k.n0pp = rc.n0ppr * kTwoPiF;
  k.xlcof = rc.xlcof;
  k.aycof = rc.aycof; k.x3thm1 = rc.x3thm1_15 * (1.0f / 1.5f); k.x1mth2 = rc.x1mth2;
  k.x7thm1 = rc.x7thm1_m025 * -4.0f; k.cosi = rc.cosi; k.sini = rc.sini; k.re = g.re;
  k.vk = g.vkmps;
  k.isimp = rc.flags & kFlagIsimp;
  return k;
}

// Reciprocal of a positive quantity of the sweep (every divisor of the reverse sweep is
// positive on a usable state): FP32 through the flush-to-zero rsqrt (rcp_pos), FP64 a
// division.  Each reciprocal is taken once and reused.
__device__ __forceinline__ float inv_pos(float x) { return rcp_pos(x); }
__device__ __forceinline__ double inv_pos(double x) { return 1.0 / x; }

// The output frame from the forward values' (sin, cos) pairs.
template <class T>
__device__ __forceinline__ Frame<T> frame_of(const Fwd<T>& f) {
  Frame<T> r;
  r.mx = -f.sO * f.ci; r.my = f.cO * f.ci; r.mz = f.si;
  r.Ux = r.mx * f.su + f.cO * f.cu; r.Uy = r.my * f.su + f.sO * f.cu; r.Uz = r.mz * f.su;
  r.Vx = r.mx * f.cu - f.cO * f.su; r.Vy = r.my * f.cu - f.sO * f.su; r.Vz = r.mz * f.cu;
  return r;
}

// The frame and the powers of t of a state, kept (FP64) or recomputed (FP32).
template <class T>
__device__ __forceinline__ Frame<T> frame_get(const Fwd<T>& f) {
  if constexpr (std::is_same<T, double>::value) return f.fr;
  else return frame_of(f);
}
template <class T>
__device__ __forceinline__ void tpow_get(const Fwd<T>& f, T& t2, T& t3, T& t4) {
  if constexpr (std::is_same<T, double>::value) {
    t2 = f.t2; t3 = f.t3; t4 = f.t4;
  } else {
    t2 = f.tt * f.tt; t3 = t2 * f.tt; t4 = t3 * f.tt;
  }
}

// Forward pass of one state in FP64: the formulation of state64 (angle reduction by
// trunc, small rotations instead of atan2 and three sincos), keeping what the reverse
// sweep reads.  Returns the status code.
__device__ __forceinline__ int forward64(const Rec64& rc, const Geo& g, double t,
                                         Fwd<double>& f) {
  const int fatal = (rc.flags >> kFatalShift) & 0xff;
  if (fatal) return fatal;
  if (rc.flags & kFlagN0ppNonPos) return 2;
  const bool isimp = rc.flags & kFlagIsimp;
  const double mdf = rc.m0 + rc.mdot * t;
  const double argpdf = rc.argp0 + rc.argpdot * t;
  f.tt = t;
  const auto t2 = t * t, t3 = t2 * t, t4 = t3 * t;
  double raan = rc.raan0 + rc.raandot * t + rc.raan_cf * t2;
  double argp = argpdf;
  double tempa = 1.0 - rc.c1 * t;
  double tempe = rc.bc4 * t;
  double templ = rc.l2 * t2;
  f.sMdf = 0.0; f.cMdf = 0.0; f.c = 1.0; f.sMM = 0.0; f.cMM = 0.0;
  if (!isimp) {
    const double dargp = rc.argp_cf * t;
    sincos(wrap_2pi(mdf), &f.sMdf, &f.cMdf);
    f.c = 1.0 + rc.eta * f.cMdf;
    const double dd = dargp + rc.m_cf * (f.c * f.c * f.c - rc.delm0);
    argp = argpdf - dd;
    tempa = tempa - rc.d2 * t2 - rc.d3 * t3 - rc.d4 * t4;
    double sdd, cdd;
    sincos_small64(dd, sdd, cdd);
    f.sMM = f.sMdf * cdd + f.cMdf * sdd;
    f.cMM = f.cMdf * cdd - f.sMdf * sdd;
    tempe = tempe + rc.bc5 * (f.sMM - rc.sinm0);
    templ = templ + rc.l3 * t3 + t4 * (rc.l4 + t * rc.l5);
  }
  f.tempa = tempa;
  f.templ = templ;
  f.a = rc.a0pp * tempa * tempa;
  const double ra = rsqrt(f.a);
  f.sqa = f.a * ra;
  const double ia15 = ra * ra * ra;
  f.n = g.xke * ia15;
  const double e1 = rc.e0 - tempe;
  if (e1 >= 1.0 || e1 < -0.001) return 1;
  f.keep_e = e1 < 1.0e-6 ? 0.0 : 1.0;
  f.e = fmax(e1, 1.0e-6);
  raan = wrap_2pi(raan);
  argp = wrap_2pi(argp);
  const double mpa = mdf + argpdf + rc.n0pp * templ;   // M + argp (drag terms cancel)
  sincos(argp, &f.sw, &f.cw);
  f.axn = f.e * f.cw;
  f.om = 1.0 - f.e * f.e;
  f.q = 1.0 / (f.a * f.om);
  f.ayn = f.e * f.sw + f.q * rc.aycof;
  const double U = wrap_2pi(mpa + f.q * rc.xlcof * f.axn);
  f.eL2 = f.axn * f.axn + f.ayn * f.ayn;
  // sin, cos of the first iterate from sincos, of later ones by rotating the previous
  // pair by the step taken (Taylor for small steps): one FP64 sincos per state.
  double psi = U, sp, cp, step = 0.0;
  sincos(U, &sp, &cp);
  const int K = newton_steps64(f.eL2);
  for (int k = 0; k < K; ++k) {
    if (k > 0) rotate64(sp, cp, step);
    step = (U - f.ayn * cp + f.axn * sp - psi) / (1.0 - f.ayn * sp - f.axn * cp);
    step = fmin(fmax(step, -0.95), 0.95);
    psi += step;
    if (K == 10 && fabs(step) < 1.0e-12) break;
  }
  rotate64(sp, cp, step);
  f.sp = sp; f.cp = cp;
  f.ecosE = f.axn * cp + f.ayn * sp;
  f.esinE = f.axn * sp - f.ayn * cp;
  f.pL = f.a * (1.0 - f.eL2);
  if (f.pL < 0.0) return 4;
  f.rl = f.a * (1.0 - f.ecosE);
  const double invr = 1.0 / f.rl;
  f.rdotl = f.sqa * f.esinE * invr;
  const double rpl = rsqrt(f.pL);
  f.sqp = f.pL * rpl;
  f.rfdotl = f.sqp * invr;
  f.betal = sqrt(1.0 - f.eL2);
  f.opb = 1.0 + f.betal;
  f.w = f.esinE / f.opb;
  f.aor = f.a * invr;
  f.As = sp - f.ayn - f.axn * f.w;
  f.Ac = cp - f.axn + f.ayn * f.w;
  f.sinu = f.aor * f.As;
  f.cosu = f.aor * f.Ac;
  f.sin2u = 2.0 * f.cosu * f.sinu;
  f.cos2u = 1.0 - 2.0 * f.sinu * f.sinu;
  const double invp = rpl * rpl;
  f.k = 0.5 * g.j2 * invp;
  f.kp = f.k * invp;
  f.fac = 1.0 - 1.5 * f.kp * f.betal * rc.x3thm1;
  f.rk = f.rl * f.fac + 0.5 * f.k * rc.x1mth2 * f.cos2u;
  f.nk = ia15 * f.k;
  f.rdotk = f.rdotl - f.nk * rc.x1mth2 * f.sin2u;
  f.rfdotk = f.rfdotl + f.nk * (rc.x1mth2 * f.cos2u + 1.5 * rc.x3thm1);
  const double nrm = rsqrt(f.sinu * f.sinu + f.cosu * f.cosu);
  f.su = f.sinu * nrm; f.cu = f.cosu * nrm;
  rotate64(f.su, f.cu, -0.25 * f.kp * rc.x7thm1 * f.sin2u);
  sincos(raan, &f.sO, &f.cO);
  rotate64(f.sO, f.cO, 1.5 * f.kp * rc.cosi * f.sin2u);
  f.si = rc.sini; f.ci = rc.cosi;
  rotate64(f.si, f.ci, 1.5 * f.kp * rc.cosi * rc.sini * f.cos2u);
  f.t2 = t2; f.t3 = t3; f.t4 = t4;
  f.fr = frame_of(f);
  return f.rk < 1.0 ? 6 : 0;
}

// Forward pass of one state in FP32: the formulation and guard bands of state32
// (double-float n*t phase, bound-based Newton count, small rotations).  Returns the
// status code, or kRecomputeFP64 for a state inside a guard band.
__device__ __forceinline__ int forward32(const Rec32& rc, const GeoF& g, float th, float tl,
                                         Fwd<float>& f) {
  const int fatal = (rc.flags >> kFatalShift) & 0xff;
  if (fatal) return fatal;
  if (rc.flags & kFlagN0ppNonPos) return 2;
  const bool isimp = rc.flags & kFlagIsimp;
  const float t = th;
  f.tt = t;
  const auto t2 = t * t, t3 = t2 * t, t4 = t3 * t;
  float tempa = 1.0f - rc.c1 * t;
  float tempe = rc.bc4 * t;
  float templ = rc.l2 * t2;
  float dd = 0.0f;
  f.sMdf = 0.0f; f.cMdf = 0.0f; f.c = 1.0f; f.sMM = 0.0f; f.cMM = 0.0f;
  if (!isimp) {
    const float dargp = rc.argpcf * t;
    const float mdf = wrap_rev(fmaf(rc.mdr, t, rc.m0r)) * kTwoPiF;
    __sincosf(mdf, &f.sMdf, &f.cMdf);
    f.c = 1.0f + rc.eta * f.cMdf;
    dd = dargp + rc.mcf * (f.c * f.c * f.c - rc.delm0);
    tempa = tempa - rc.d2 * t2 - rc.d3 * t3 - rc.d4 * t4;
    __sincosf(mdf + dd, &f.sMM, &f.cMM);
    tempe = tempe + rc.bc5 * (f.sMM - rc.sinm0);
    templ = templ + rc.l3 * t3 + t4 * (rc.l4 + t * rc.l5);
  }
  f.tempa = tempa;
  f.templ = templ;
  f.a = rc.a0pp * tempa * tempa;
  const float e1 = rc.e0 - tempe;
  if (!(fabsf(e1 - 1.0f) >= kGuardE && fabsf(e1 + 0.001f) >= kGuardE && f.a > 1.0e-3f))
    return kRecomputeFP64;
  if (e1 >= 1.0f || e1 < -0.001f) return 1;
  f.keep_e = e1 < 1.0e-6f ? 0.0f : 1.0f;
  f.e = fmaxf(e1, 1.0e-6f);
  const float ra = rsqrt_ftz(f.a);
  f.sqa = f.a * ra;
  const float ra3 = ra * ra * ra;
  f.n = g.xke * ra3;

  float p = rc.phidh * th;
  const float pe = fmaf(rc.phidh, th, -p);
  const float s = fmaf(rc.phidh, tl, fmaf(rc.phidl, th, pe));
  p = p - round_magic(p);
  float y = wrap_rev(p + rc.phi0h);
  y += s + rc.phi0l;
  // The propagation also recomputes in FP64 the states whose drag phase n0'' templ
  // passes one revolution (kGuardDragPhase); the sweeps do not.  Those are orbits whose
  // drag polynomial of the semi-major axis has passed its minimum and which balloon (5
  // of the fitting workload's 10,000 satellites): sweeping their late states in FP64
  // made the FP32 adjoint 27% slower, so there the adjoint's, Jacobian's and fit's
  // FP32 forward values keep that term's FP32 rounding.
  y += wrap_rev(rc.n0ppr * templ);
  const float argp = wrap_rev(fmaf(rc.argpdr, t, rc.argp0r) - dd * kInvTwoPiF) * kTwoPiF;
  const float raan = wrap_rev(fmaf(rc.raancfr, t2, fmaf(rc.raandr, t, rc.raan0r))) * kTwoPiF;

  __sincosf(argp, &f.sw, &f.cw);
  f.axn = f.e * f.cw;
  f.om = 1.0f - f.e * f.e;
  f.q = rcp_pos(f.a * f.om);
  f.ayn = fmaf(f.e, f.sw, f.q * rc.aycof);
  const float lpt = f.q * rc.xlcof * f.axn;
  if (!(fabsf(lpt) < kGuardLongPeriod)) return kRecomputeFP64;
  const float U = wrap_rev(y + lpt * kInvTwoPiF) * kTwoPiF;
  f.eL2 = f.axn * f.axn + f.ayn * f.ayn;
  float psi = U;
  const int K = newton_steps(f.eL2);
  for (int k = 0; k < K; ++k) {
    float sp, cp;
    __sincosf(psi, &sp, &cp);
    const float fv = U - f.ayn * cp + f.axn * sp - psi;
    const float fp = 1.0f - f.ayn * sp - f.axn * cp;
    psi += fminf(fmaxf(fv * rcp_pos(fp), -0.95f), 0.95f);
  }
  sincos_acc(psi, &f.sp, &f.cp);
  f.ecosE = f.axn * f.cp + f.ayn * f.sp;
  f.esinE = f.axn * f.sp - f.ayn * f.cp;
  f.pL = f.a * (1.0f - f.eL2);
  if (!(fabsf(f.pL) >= kGuardP)) return kRecomputeFP64;
  if (f.pL < 0.0f) return 4;
  f.rl = f.a * (1.0f - f.ecosE);
  const float invr = rcp_pos(f.rl);
  f.rdotl = f.sqa * f.esinE * invr;
  const float rpl = rsqrt_ftz(f.pL);
  f.sqp = f.pL * rpl;
  f.rfdotl = f.sqp * invr;
  const float omel = 1.0f - f.eL2;
  f.betal = omel * rsqrt_ftz(omel);
  f.opb = 1.0f + f.betal;
  f.w = f.esinE * rcp_pos(f.opb);
  f.aor = f.a * invr;
  f.As = f.sp - f.ayn - f.axn * f.w;
  f.Ac = f.cp - f.axn + f.ayn * f.w;
  f.sinu = f.aor * f.As;
  f.cosu = f.aor * f.Ac;
  f.sin2u = 2.0f * f.cosu * f.sinu;
  f.cos2u = 1.0f - 2.0f * f.sinu * f.sinu;
  const float invp = rpl * rpl;
  f.k = g.half_j2 * invp;
  f.kp = f.k * invp;
  f.fac = fmaf(-f.kp * f.betal, rc.x3thm1_15, 1.0f);
  f.rk = f.rl * f.fac + f.k * rc.half_x1mth2 * f.cos2u;
  if (!(fabsf(f.rk - 1.0f) >= kGuardR)) return kRecomputeFP64;
  f.nk = ra3 * f.k;
  f.rdotk = f.rdotl - f.nk * rc.x1mth2 * f.sin2u;
  f.rfdotk = fmaf(f.nk, fmaf(rc.x1mth2, f.cos2u, rc.x3thm1_15), f.rfdotl);
  const float du = f.kp * rc.x7thm1_m025 * f.sin2u;
  const float dO = f.kp * rc.c15cosi * f.sin2u;
  const float di = f.kp * rc.c15cosisini * f.cos2u;
  if (!(fmaxf(fabsf(du), fmaxf(fabsf(dO), fabsf(di))) < 4.0e-3f)) return kRecomputeFP64;
  const float nrm = rsqrt_ftz(f.sinu * f.sinu + f.cosu * f.cosu);
  f.su = f.sinu * nrm; f.cu = f.cosu * nrm;
  rotate_small(f.su, f.cu, du);
  __sincosf(raan, &f.sO, &f.cO);
  rotate_small(f.sO, f.cO, dO);
  f.si = rc.sini; f.ci = rc.cosi;
  rotate_small(f.si, f.ci, di);
  return f.rk < 1.0f ? 6 : 0;
}

// Reverse sweep of one state: the adjoints of the 33 record fields, given the forward
// values f and the output adjoints gr (of r, km) and gv (of v, km/s).  Each field's
// adjoint goes to sink(field, value) as soon as it is final (fields that do not
// depend on the state, such as the drag terms of a simplified-drag record, are not
// passed), so that no array of 33 adjoints has to stay live through the sweep.
// T is the type of the state's values (double, float, or a packed pair of floats for
// two states), C that of the satellite's constants.
template <class T, class C, class Sink>
__device__ __forceinline__ void reverse(const Fwd<T>& f, const RevC<C>& rc, const T gr[3],
                                        const T gv[3], Sink&& sink) {
  const T one = T(1), two = T(2), half = T(0.5), c15 = T(1.5);
  const T re = rc.re, vk = rc.vk;
  T t2, t3, t4;
  tpow_get(f, t2, t3, t4);
  const Frame<T> fr = frame_get(f);
  // r = rk re U, v = vk (rdotk U + rfdotk V)
  const T Ubx = f.rk * re * gr[0] + vk * f.rdotk * gv[0];
  const T Uby = f.rk * re * gr[1] + vk * f.rdotk * gv[1];
  const T Ubz = f.rk * re * gr[2] + vk * f.rdotk * gv[2];
  const T Vbx = vk * f.rfdotk * gv[0], Vby = vk * f.rfdotk * gv[1], Vbz = vk * f.rfdotk * gv[2];
  const T rkb = re * (gr[0] * fr.Ux + gr[1] * fr.Uy + gr[2] * fr.Uz);
  const T rdotkb = vk * (gv[0] * fr.Ux + gv[1] * fr.Uy + gv[2] * fr.Uz);
  const T rfdotkb = vk * (gv[0] * fr.Vx + gv[1] * fr.Vy + gv[2] * fr.Vz);
  // U = M su + N cu, V = M cu - N su, M = (mx, my, mz), N = (cO, sO, 0)
  const T Mbx = Ubx * f.su + Vbx * f.cu, Mby = Uby * f.su + Vby * f.cu;
  const T Mbz = Ubz * f.su + Vbz * f.cu;
  const T Nbx = Ubx * f.cu - Vbx * f.su, Nby = Uby * f.cu - Vby * f.su;
  const T sub = Ubx * fr.mx + Uby * fr.my + Ubz * fr.mz - (Vbx * f.cO + Vby * f.sO);
  const T cub = Ubx * f.cO + Uby * f.sO + (Vbx * fr.mx + Vby * fr.my + Vbz * fr.mz);
  const T sOb = -Mbx * f.ci + Nby;
  const T cOb = Mby * f.ci + Nbx;
  const T cib = -Mbx * f.sO + Mby * f.cO;
  const T sib = Mbz;
  const T ukb = sub * f.cu - cub * f.su;       // (su, cu) = (sin u_k, cos u_k)
  const T raankb = sOb * f.cO - cOb * f.sO;
  const T ikb = sib * f.ci - cib * f.si;
  // rdot_k, rfdot_k
  const T nkb = -rdotkb * rc.x1mth2 * f.sin2u +
                rfdotkb * (rc.x1mth2 * f.cos2u + c15 * rc.x3thm1);
  T x1mth2b = -rdotkb * f.nk * f.sin2u + rfdotkb * f.nk * f.cos2u;
  T sin2ub = -rdotkb * f.nk * rc.x1mth2;
  T cos2ub = rfdotkb * f.nk * rc.x1mth2;
  T x3thm1b = rfdotkb * f.nk * c15;
  const T nb = nkb * f.k * rc.ixke;
  T kb = nkb * f.n * rc.ixke;
  // i_k = i0 + 1.5 kp cosi sini cos2u, RAAN_k = RAAN + 1.5 kp cosi sin2u,
  // u_k = u - 0.25 kp x7thm1 sin2u
  T kpb = ikb * c15 * rc.cosi * rc.sini * f.cos2u;
  T cosib = ikb * c15 * f.kp * rc.sini * f.cos2u;
  const T sinib = ikb * c15 * f.kp * rc.cosi * f.cos2u;
  cos2ub += ikb * c15 * f.kp * rc.cosi * rc.sini;
  kpb += raankb * c15 * rc.cosi * f.sin2u;
  cosib += raankb * c15 * f.kp * f.sin2u;
  sin2ub += raankb * c15 * f.kp * rc.cosi;
  kpb += -ukb * T(0.25) * rc.x7thm1 * f.sin2u;
  const T x7thm1b = -ukb * T(0.25) * f.kp * f.sin2u;
  sin2ub += -ukb * T(0.25) * f.kp * rc.x7thm1;
  // r_k = rl (1 - 1.5 kp betal x3thm1) + 0.5 k x1mth2 cos2u
  T rlb = rkb * f.fac;
  kpb += -rkb * f.rl * c15 * f.betal * rc.x3thm1;
  T betalb = -rkb * f.rl * c15 * f.kp * rc.x3thm1;
  x3thm1b += -rkb * f.rl * c15 * f.kp * f.betal;
  kb += rkb * half * rc.x1mth2 * f.cos2u;
  x1mth2b += rkb * half * f.k * f.cos2u;
  cos2ub += rkb * half * f.k * rc.x1mth2;
  // kp = k / pL, k = j2 / (2 pL)
  const T ipL = inv_pos(f.pL);
  kb += kpb * ipL;
  T pLb = -kpb * f.kp * ipL;
  pLb += -kb * f.k * ipL;
  // sin 2u, cos 2u, u = atan2(sin u, cos u)
  T sinub = two * f.cosu * sin2ub - T(4) * f.sinu * cos2ub;
  T cosub = two * f.sinu * sin2ub;
  const T iden = inv_pos(f.sinu * f.sinu + f.cosu * f.cosu);
  sinub += ukb * f.cosu * iden;
  cosub += -ukb * f.sinu * iden;
  // sin u = aor As, cos u = aor Ac
  const T aorb = sinub * f.As + cosub * f.Ac;
  const T Asb = sinub * f.aor, Acb = cosub * f.aor;
  T spb = Asb, cpb = Acb;
  T aynb = -Asb + Acb * f.w;
  T axnb = -Asb * f.w - Acb;
  const T wb = -Asb * f.axn + Acb * f.ayn;
  const T irl = inv_pos(f.rl), iopb = inv_pos(fwd_opb(f));
  T ab = aorb * irl;
  rlb += -aorb * f.aor * irl;
  T esinEb = wb * iopb;
  betalb += -wb * f.w * iopb;
  T eL2b = -betalb * half * inv_pos(f.betal);
  const T sqpb = rfdotkb * irl;
  rlb += -rfdotkb * f.rfdotl * irl;
  pLb += sqpb * half * inv_pos(f.sqp);
  const T sqab = rdotkb * f.esinE * irl;
  esinEb += rdotkb * f.sqa * irl;
  rlb += -rdotkb * f.rdotl * irl;
  ab += rlb * (one - fwd_ecosE(f));
  const T ecosEb = -rlb * f.a;
  ab += pLb * (one - f.eL2);
  eL2b += -pLb * f.a;
  axnb += two * f.axn * eL2b;
  aynb += two * f.ayn * eL2b;
  axnb += esinEb * f.sp;
  spb += esinEb * f.axn;
  aynb += -esinEb * f.cp;
  cpb += -esinEb * f.ayn;
  axnb += ecosEb * f.cp;
  cpb += ecosEb * f.axn;
  aynb += ecosEb * f.sp;
  spb += ecosEb * f.ayn;
  // Kepler at its root: psi - axn sin psi + ayn cos psi = U
  const T psib = spb * f.cp - cpb * f.sp;
  const T iD = inv_pos(one - f.axn * f.cp - f.ayn * f.sp);
  const T Ub = psib * iD;
  axnb += psib * f.sp * iD;
  aynb += -psib * f.cp * iD;
  // U = (M + argp) + q xlcof axn
  T qb = Ub * rc.xlcof * f.axn;
  sink(aXlcof, Ub * f.q * f.axn);
  axnb += Ub * f.q * rc.xlcof;
  // a_yN = e sin argp + q aycof
  T eb = aynb * f.sw;
  const T swb = aynb * f.e;
  qb += aynb * rc.aycof;
  sink(aAycof, aynb * f.q);
  // q = 1 / (a (1 - e^2))
  const T qab = -qb * f.q * f.q;
  ab += qab * fwd_om(f);
  eb += -two * f.e * (qab * f.a);
  // a_xN = e cos argp
  eb += axnb * f.cw;
  const T cwb = axnb * f.e;
  const T argpb = swb * f.cw - cwb * f.sw;
  // mpa = M_DF + argp_DF + n0'' templ, argp = argp_DF - dd, RAAN = RAAN_DF + raan_cf t^2
  const T mm2b = Ub;
  const T argp1b = Ub + argpb;
  sink(aN0pp, mm2b * f.templ);
  const T templb = mm2b * rc.n0pp;
  const T e1b = f.keep_e * eb;
  sink(aE0, e1b);
  const T tempeb = -e1b;
  ab += nb * T(-1.5) * f.n * inv_pos(f.a);
  ab += sqab * half * inv_pos(f.sqa);
  sink(aA0pp, ab * f.tempa * f.tempa);
  const T tempab = ab * rc.a0pp * two * f.tempa;
  T mdfb = mm2b, argpdfb = argp1b;
  if (!rc.isimp) {
    sink(aL3, templb * t3);
    sink(aL4, templb * t4);
    sink(aL5, templb * t4 * f.tt);
    sink(aBC5, tempeb * (f.sMM - rc.sinm0));
    const T sMMb = tempeb * rc.bc5;
    sink(aSinM0, -tempeb * rc.bc5);
    sink(aD2, -tempab * t2);
    sink(aD3, -tempab * t3);
    sink(aD4, -tempab * t4);
    // mm1 = M_DF + dd carries sin(mm1); argp = argp_DF - dd; dd = argp_cf t + dm
    const T mm1b = mm2b + sMMb * f.cMM;
    mdfb = mm1b;
    const T ddb = mm1b - argp1b;
    const T c = fwd_c(f, rc);
    sink(aMCf, ddb * (c * c * c - rc.delm0));
    const T cb = ddb * rc.mcf * T(3) * c * c;
    sink(aDelM0, -ddb * rc.mcf);
    sink(aEta, cb * f.cMdf);
    mdfb += -(cb * rc.eta) * f.sMdf;
    sink(aArgpCf, ddb * f.tt);
  }
  sink(aL2, templb * t2);
  sink(aBC4, tempeb * f.tt);
  sink(aC1, -tempab * f.tt);
  sink(aRaan0, raankb);
  sink(aRaandot, raankb * f.tt);
  sink(aRaanCf, raankb * t2);
  sink(aArgp0, argpdfb);
  sink(aArgpdot, argpdfb * f.tt);
  sink(aM0, mdfb);
  sink(aMdot, mdfb * f.tt);
  sink(aI0, ikb);
  sink(aCosi, cosib);
  sink(aSini, sinib);
  sink(aX3thm1, x3thm1b);
  sink(aX1mth2, x1mth2b);
  sink(aX7thm1, x7thm1b);
}

__device__ __forceinline__ bool usable(int code) { return code == 0 || code == 6; }

// FP64 forward and reverse sweeps of one state for the FP32 kernels (guard-band
// states), for the seed (g_r, g_v): writes the 33 field adjoints to bar (adds them to
// it with accumulate) and, if r and v are not null, the position (km) and velocity
// (km/s).  Out of line: rarely taken.
static __device__ __noinline__ int adjoint_fallback(RecordPtrs rp, Geo g, int64_t j, double t,
                                                    float gr0, float gr1, float gr2, float gv0,
                                                    float gv1, float gv2, float* bar, float* r,
                                                    float* v = nullptr, bool accumulate = false) {
  const Rec64 rc = load_rec64(rp, j);
  Fwd<double> f;
  const int code = forward64(rc, g, t, f);
  if (!usable(code)) return code;
  const RevC<double> k = rev_consts(rc, g);
  const double gr[3] = {gr0, gr1, gr2};
  const double gv[3] = {gv0, gv1, gv2};
  if (!accumulate)
    for (int q = 0; q < kNumAdj; ++q) bar[q] = 0.0f;
  reverse(f, k, gr, gv, [&](int q, double v) { bar[q] += (float)v; });
  const Frame<double> fr = frame_get(f);
  if (r) {
    r[0] = (float)(f.rk * g.re * fr.Ux);
    r[1] = (float)(f.rk * g.re * fr.Uy);
    r[2] = (float)(f.rk * g.re * fr.Uz);
  }
  if (v) {
    v[0] = (float)(g.vkmps * (f.rdotk * fr.Ux + f.rfdotk * fr.Vx));
    v[1] = (float)(g.vkmps * (f.rdotk * fr.Uy + f.rfdotk * fr.Vy));
    v[2] = (float)(g.vkmps * (f.rdotk * fr.Uz + f.rfdotk * fr.Vz));
  }
  return code;
}

// Warp sum of v by a shuffle tree in T; lane 0 stores it to part[idx][warp].
template <class T>
__device__ __forceinline__ void warp_partial(T v, int idx, T (*part)[kAdjWarps]) {
  for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) part[idx][threadIdx.x >> 5] = v;
}

// The record and the reverse-sweep constants of the block's satellite, in shared
// memory (every thread reads the same words: broadcasts).
template <class T>
struct SatShared {
  typename std::conditional<sizeof(T) == 4, Rec32, Rec64>::type rc;
  RevC<T> k;
};

template <class T>
__device__ __forceinline__ void load_sat(const RecordPtrs& rp, const Geo& g, const GeoF& gf,
                                         int64_t j, SatShared<T>& s) {
  if constexpr (sizeof(T) == 4) {
    s.rc = load_rec32(rp, j);
    s.k = rev_consts(s.rc, gf);
  } else {
    s.rc = load_rec64(rp, j);
    s.k = rev_consts(s.rc, g);
  }
}

// Forward values of one state: shared memory for FP32 (the reverse sweep then reads
// them from there instead of holding ~65 values in registers, which would leave two
// blocks per SM), registers for FP64 (whose kernels are bound by the FP64 unit).
template <class T>
struct FwdSlot {
  static constexpr int kRows = sizeof(T) == 4 ? kAdjThreads : 1;
};

// Compiler barrier between the forward and the reverse sweep: the reverse reloads the
// forward values from shared memory instead of keeping them live in registers.
__device__ __forceinline__ void reload_barrier() { asm volatile("" ::: "memory"); }

__device__ __forceinline__ bool elements_usable(const double e7[7]) {
  bool ok = true;
  for (int k = 0; k < 7; ++k) ok = ok && isfinite(e7[k]);
  return ok && e7[1] >= 0.0 && e7[1] < 1.0 && e7[0] > 0.0;
}

// Record-field Jacobian of sgp4init, d(field)/d(element), [kNumAdj][7] row-major, by
// dual numbers over R (false for unusable elements).  R = float serves the FP32
// sweeps: their field adjoints carry FP32 rounding already, and B300 runs FP32 dual
// arithmetic 64 times faster than FP64.  The branch decisions of the record build
// (simplified drag, s*, e0 > 1e-4) are then taken on FP32 values.
template <class R>
__device__ bool init_jacobian(const double e7[7], const Geo& g, R* J) {
  if (!elements_usable(e7)) return false;
  Dual7<R> x[7];
  for (int k = 0; k < 7; ++k) x[k] = d7var(R(e7[k]), k);
  InitFields<Dual7<R>> o;
  init_fields(x, g, o);
  const Dual7<R>* f[kNumAdj] = {&o.n0pp, &o.a0pp, &o.e0, &o.i0, &o.raan0, &o.argp0, &o.m0,
                                &o.mdot, &o.argpdot, &o.raandot, &o.raan_cf, &o.argp_cf,
                                &o.m_cf, &o.c1, &o.bc4, &o.bc5, &o.d2, &o.d3, &o.d4, &o.l2,
                                &o.l3, &o.l4, &o.l5, &o.eta, &o.delm0, &o.sinm0, &o.xlcof,
                                &o.aycof, &o.cosi, &o.sini, &o.x3thm1, &o.x1mth2, &o.x7thm1};
  for (int q = 0; q < kNumAdj; ++q)
    for (int k = 0; k < 7; ++k) J[q * 7 + k] = f[q]->d[k];
  return true;
}

}  // namespace
}  // namespace sgp4
