// Device-side SGP4 near-Earth theory for sm_103a: record layout, the FP64 state
// function and the mixed-precision FP32 state function.
//
// The theory is the one the paper implements (Sec. 2.1: Spacetrack Report #3 as
// revised in 2006, WGS-72); the error-code convention is Sec. 2.2 "Control Flow";
// one (satellite, time) state per thread is Sec. 2.2 "Vectorisation".  Symbols:
// n0'' (n0pp), a0'', xi, eta, C1..C5, D2..D4, a_xN, a_yN, U, psi = E + omega,
// e_L, p_L, r_k, u_k as in Spacetrack Report #3.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sgp4 {

// ---------------------------------------------------------------- record layout
// Structure of arrays inside one caller-owned arena:
//   [kNumF64 planes of double][kNumF32 planes of float][flags int32][epoch_day int32]
// each plane `stride` entries long, stride a multiple of 64 (256-byte planes).
enum F64Field {
  kN0pp, kA0pp, kE0, kI0, kRaan0, kArgp0, kM0, kBstar,
  kMdot, kArgpdot, kRaandot, kRaanCf, kArgpCf, kMCf,
  kC1, kBC4, kBC5, kD2, kD3, kD4, kL2, kL3, kL4, kL5,
  kEta, kDelM0, kSinM0, kXlcof, kAycof,
  kCosi, kSini, kX3thm1, kX1mth2, kX7thm1,
  kEpochFrac,
  kNumF64
};

// FP32-path planes.  Angles and their rates are stored in revolutions (x / 2 pi) so
// that the reduction mod one revolution is a subtraction of rint(x).  The mean
// argument of latitude phase (M0 + argp0) and its rate (Mdot + argpdot) are kept as
// unevaluated float sums hi + lo ("double-float").
enum F32Field {
  fPhi0H, fPhi0L, fPhiDH, fPhiDL,
  fM0r, fMdr, fArgp0r, fArgpdr, fRaan0r, fRaandr, fRaanCfr, fN0ppr,
  fA0pp, fE0, fC1, fBC4, fBC5, fD2, fD3, fD4, fL2, fL3, fL4, fL5,
  fEta, fDelM0, fSinM0, fArgpCf, fMCf, fXlcof, fAycof,
  fCosi, fSini, fX3thm1, fX1mth2, fX7thm1,
  kNumF32
};

// flags word
constexpr int kFlagIsimp = 1;        // perigee below 220 km: truncated drag terms
constexpr int kFlagN0ppNonPos = 2;   // n0'' <= 0 -> code 2 at every t
constexpr int kFatalShift = 8;       // bits 8..15: fatal input code (1 or 2)

__host__ __device__ inline int64_t record_stride(int64_t n) { return ((n + 63) / 64) * 64; }

__host__ __device__ inline size_t record_bytes(int64_t n) {
  const int64_t s = record_stride(n);
  return (size_t)s * (sizeof(double) * kNumF64 + sizeof(float) * kNumF32 + 2 * sizeof(int32_t));
}

struct RecordPtrs {
  double* f64;      // [kNumF64][stride]
  float* f32;       // [kNumF32][stride]
  int32_t* flags;   // [stride]
  int32_t* epoch_day;
  int64_t stride;
  int64_t n;
};

__host__ __device__ inline RecordPtrs record_ptrs(void* arena, int64_t n) {
  RecordPtrs p;
  p.stride = record_stride(n);
  p.n = n;
  char* base = static_cast<char*>(arena);
  p.f64 = reinterpret_cast<double*>(base);
  base += sizeof(double) * kNumF64 * p.stride;
  p.f32 = reinterpret_cast<float*>(base);
  base += sizeof(float) * kNumF32 * p.stride;
  p.flags = reinterpret_cast<int32_t*>(base);
  base += sizeof(int32_t) * p.stride;
  p.epoch_day = reinterpret_cast<int32_t*>(base);
  return p;
}

// Earth model, derived once on the host.
struct Geo {
  double xke;     // sqrt(mu) in Earth radii^1.5 per minute
  double j2;
  double j3oj2;   // J3/J2 (0 when J2 == 0)
  double j4;
  double re;      // km
  double vkmps;   // re * xke / 60: Earth radii per (1/xke min) -> km/s
};

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr float kInvTwoPiF = 0.159154943091895335769f;

// ============================================================== FP64 state
struct Rec64 {
  double n0pp, a0pp, e0, i0, raan0, argp0, m0;
  double mdot, argpdot, raandot, raan_cf, argp_cf, m_cf;
  double c1, bc4, bc5, d2, d3, d4, l2, l3, l4, l5;
  double eta, delm0, sinm0, xlcof, aycof;
  double cosi, sini, x3thm1, x1mth2, x7thm1;
  int flags;
};

__device__ __forceinline__ Rec64 load_rec64(const RecordPtrs& rp, int64_t j) {
  const double* __restrict__ f = rp.f64;
  const int64_t s = rp.stride;
  Rec64 r;
  r.n0pp = __ldg(f + kN0pp * s + j);
  r.a0pp = __ldg(f + kA0pp * s + j);
  r.e0 = __ldg(f + kE0 * s + j);
  r.i0 = __ldg(f + kI0 * s + j);
  r.raan0 = __ldg(f + kRaan0 * s + j);
  r.argp0 = __ldg(f + kArgp0 * s + j);
  r.m0 = __ldg(f + kM0 * s + j);
  r.mdot = __ldg(f + kMdot * s + j);
  r.argpdot = __ldg(f + kArgpdot * s + j);
  r.raandot = __ldg(f + kRaandot * s + j);
  r.raan_cf = __ldg(f + kRaanCf * s + j);
  r.argp_cf = __ldg(f + kArgpCf * s + j);
  r.m_cf = __ldg(f + kMCf * s + j);
  r.c1 = __ldg(f + kC1 * s + j);
  r.bc4 = __ldg(f + kBC4 * s + j);
  r.bc5 = __ldg(f + kBC5 * s + j);
  r.d2 = __ldg(f + kD2 * s + j);
  r.d3 = __ldg(f + kD3 * s + j);
  r.d4 = __ldg(f + kD4 * s + j);
  r.l2 = __ldg(f + kL2 * s + j);
  r.l3 = __ldg(f + kL3 * s + j);
  r.l4 = __ldg(f + kL4 * s + j);
  r.l5 = __ldg(f + kL5 * s + j);
  r.eta = __ldg(f + kEta * s + j);
  r.delm0 = __ldg(f + kDelM0 * s + j);
  r.sinm0 = __ldg(f + kSinM0 * s + j);
  r.xlcof = __ldg(f + kXlcof * s + j);
  r.aycof = __ldg(f + kAycof * s + j);
  r.cosi = __ldg(f + kCosi * s + j);
  r.sini = __ldg(f + kSini * s + j);
  r.x3thm1 = __ldg(f + kX3thm1 * s + j);
  r.x1mth2 = __ldg(f + kX1mth2 * s + j);
  r.x7thm1 = __ldg(f + kX7thm1 * s + j);
  r.flags = __ldg(rp.flags + j);
  return r;
}

// One state in FP64.  Returns the status code; r (km) and v (km/s) are written
// for codes 0 and 6 only.
__device__ __forceinline__ int state64(const Rec64& rc, const Geo& g, double t, double r[3],
                                       double v[3]) {
  const int fatal = (rc.flags >> kFatalShift) & 0xff;
  if (fatal) return fatal;
  const bool isimp = rc.flags & kFlagIsimp;

  // Secular gravity and drag (mean elements at t).
  const double mdf = rc.m0 + rc.mdot * t;
  const double argpdf = rc.argp0 + rc.argpdot * t;
  const double raandf = rc.raan0 + rc.raandot * t;
  const double t2 = t * t;
  double raan = raandf + rc.raan_cf * t2;
  double mm = mdf, argp = argpdf;
  double tempa = 1.0 - rc.c1 * t;
  double tempe = rc.bc4 * t;
  double templ = rc.l2 * t2;
  if (!isimp) {
    const double dargp = rc.argp_cf * t;
    const double c = 1.0 + rc.eta * cos(mdf);
    const double dm = rc.m_cf * (c * c * c - rc.delm0);
    mm = mdf + dargp + dm;
    argp = argpdf - dargp - dm;
    const double t3 = t2 * t, t4 = t3 * t;
    tempa = tempa - rc.d2 * t2 - rc.d3 * t3 - rc.d4 * t4;
    tempe = tempe + rc.bc5 * (sin(mm) - rc.sinm0);
    templ = templ + rc.l3 * t3 + t4 * (rc.l4 + t * rc.l5);
  }
  if (rc.flags & kFlagN0ppNonPos) return 2;
  const double a = rc.a0pp * tempa * tempa;
  const double n = g.xke / (a * sqrt(a));
  double e = rc.e0 - tempe;
  if (e >= 1.0 || e < -0.001) return 1;
  if (e < 1.0e-6) e = 1.0e-6;
  mm = mm + rc.n0pp * templ;
  double L = mm + argp + raan;
  raan = fmod(raan, kTwoPi);
  argp = fmod(argp, kTwoPi);
  L = fmod(L, kTwoPi);
  mm = fmod(L - argp - raan, kTwoPi);

  // Long-period periodics (J3).
  double sw, cw;
  sincos(argp, &sw, &cw);
  const double axn = e * cw;
  const double q = 1.0 / (a * (1.0 - e * e));
  const double ayn = e * sw + q * rc.aycof;
  const double xl = mm + argp + raan + q * rc.xlcof * axn;
  const double U = fmod(xl - raan, kTwoPi);

  // Kepler's equation, Newton with clamped steps; same stopping rule as the theory.
  double psi = U;
  for (int k = 0; k < 10; ++k) {
    double sp, cp;
    sincos(psi, &sp, &cp);
    double step = (U - ayn * cp + axn * sp - psi) / (1.0 - ayn * sp - axn * cp);
    step = fmin(fmax(step, -0.95), 0.95);
    psi += step;
    if (fabs(step) < 1.0e-12) break;
  }
  double sp, cp;
  sincos(psi, &sp, &cp);

  // Short-period preliminaries.
  const double ecosE = axn * cp + ayn * sp;
  const double esinE = axn * sp - ayn * cp;
  const double eL2 = axn * axn + ayn * ayn;
  const double pL = a * (1.0 - eL2);
  if (pL < 0.0) return 4;
  const double rl = a * (1.0 - ecosE);
  const double rdotl = sqrt(a) * esinE / rl;
  const double rfdotl = sqrt(pL) / rl;
  const double betal = sqrt(1.0 - eL2);
  const double w = esinE / (1.0 + betal);
  const double sinu = a / rl * (sp - ayn - axn * w);
  const double cosu = a / rl * (cp - axn + ayn * w);
  const double u = atan2(sinu, cosu);
  const double sin2u = 2.0 * cosu * sinu;
  const double cos2u = 1.0 - 2.0 * sinu * sinu;

  // Short-period periodics (J2).
  const double k = 0.5 * g.j2 / pL;
  const double kp = k / pL;
  const double rk = rl * (1.0 - 1.5 * kp * betal * rc.x3thm1) + 0.5 * k * rc.x1mth2 * cos2u;
  const double uk = u - 0.25 * kp * rc.x7thm1 * sin2u;
  const double raank = raan + 1.5 * kp * rc.cosi * sin2u;
  const double ik = rc.i0 + 1.5 * kp * rc.cosi * rc.sini * cos2u;
  const double rdotk = rdotl - n * k * rc.x1mth2 * sin2u / g.xke;
  const double rfdotk = rfdotl + n * k * (rc.x1mth2 * cos2u + 1.5 * rc.x3thm1) / g.xke;

  // Orientation and TEME output.
  double su, cu, sO, cO, si, ci;
  sincos(uk, &su, &cu);
  sincos(raank, &sO, &cO);
  sincos(ik, &si, &ci);
  const double mx = -sO * ci, my = cO * ci, mz = si;
  const double ux = mx * su + cO * cu, uy = my * su + sO * cu, uz = mz * su;
  const double vx = mx * cu - cO * su, vy = my * cu - sO * su, vz = mz * cu;
  const double rs = rk * g.re;
  r[0] = rs * ux; r[1] = rs * uy; r[2] = rs * uz;
  v[0] = (rdotk * ux + rfdotk * vx) * g.vkmps;
  v[1] = (rdotk * uy + rfdotk * vy) * g.vkmps;
  v[2] = (rdotk * uz + rfdotk * vz) * g.vkmps;
  return rk < 1.0 ? 6 : 0;
}

// Out-of-line FP64 recomputation of one state for the FP32 path's guard band
// (rarely taken; kept out of line so the FP32 kernel's registers stay small).
static __device__ __noinline__ int state64_fallback(RecordPtrs rp, Geo g, int64_t j, double t,
                                                    float r[3], float v[3]) {
  const Rec64 rc = load_rec64(rp, j);
  double r64[3], v64[3];
  const int code = state64(rc, g, t, r64, v64);
  for (int c = 0; c < 3; ++c) {
    r[c] = (float)r64[c];
    v[c] = (float)v64[c];
  }
  return code;
}

// ============================================================== FP32 state
struct GeoF {
  float xke, inv_xke, j2, re, vkmps;
};

struct Rec32 {
  float phi0h, phi0l, phidh, phidl;
  float m0r, mdr, argp0r, argpdr, raan0r, raandr, raancfr, n0ppr;
  float a0pp, e0, c1, bc4, bc5, d2, d3, d4, l2, l3, l4, l5;
  float eta, delm0, sinm0, argpcf, mcf, xlcof, aycof;
  float cosi, sini, x3thm1, x1mth2, x7thm1;
  int flags;
};

__device__ __forceinline__ Rec32 load_rec32(const RecordPtrs& rp, int64_t j) {
  const float* __restrict__ f = rp.f32;
  const int64_t s = rp.stride;
  Rec32 r;
#define SGP4_LD32(dst, fld) r.dst = __ldg(f + (fld) * s + j)
  SGP4_LD32(phi0h, fPhi0H); SGP4_LD32(phi0l, fPhi0L); SGP4_LD32(phidh, fPhiDH);
  SGP4_LD32(phidl, fPhiDL); SGP4_LD32(m0r, fM0r); SGP4_LD32(mdr, fMdr);
  SGP4_LD32(argp0r, fArgp0r); SGP4_LD32(argpdr, fArgpdr); SGP4_LD32(raan0r, fRaan0r);
  SGP4_LD32(raandr, fRaandr); SGP4_LD32(raancfr, fRaanCfr); SGP4_LD32(n0ppr, fN0ppr);
  SGP4_LD32(a0pp, fA0pp); SGP4_LD32(e0, fE0); SGP4_LD32(c1, fC1); SGP4_LD32(bc4, fBC4);
  SGP4_LD32(bc5, fBC5); SGP4_LD32(d2, fD2); SGP4_LD32(d3, fD3); SGP4_LD32(d4, fD4);
  SGP4_LD32(l2, fL2); SGP4_LD32(l3, fL3); SGP4_LD32(l4, fL4); SGP4_LD32(l5, fL5);
  SGP4_LD32(eta, fEta); SGP4_LD32(delm0, fDelM0); SGP4_LD32(sinm0, fSinM0);
  SGP4_LD32(argpcf, fArgpCf); SGP4_LD32(mcf, fMCf); SGP4_LD32(xlcof, fXlcof);
  SGP4_LD32(aycof, fAycof); SGP4_LD32(cosi, fCosi); SGP4_LD32(sini, fSini);
  SGP4_LD32(x3thm1, fX3thm1); SGP4_LD32(x1mth2, fX1mth2); SGP4_LD32(x7thm1, fX7thm1);
#undef SGP4_LD32
  r.flags = __ldg(rp.flags + j);
  return r;
}

// Reduce an angle in revolutions to [-1/2, 1/2].  Exact for |x| < 2^23.
__device__ __forceinline__ float wrap_rev(float x) { return x - rintf(x); }

// Rotate the unit vector (s, c) = (sin a, cos a) to (sin(a+d), cos(a+d)).  The
// corrections d of the short-period terms are O(J2/p_L^2) ~ 1e-3 rad, where a
// 5th/4th-order Taylor pair is exact to float precision; larger d (only for
// nearly degenerate orbits) takes the full sincosf.
__device__ __forceinline__ void rotate_small(float& s, float& c, float d) {
  float sd, cd;
  if (fabsf(d) < 0.05f) {
    const float d2 = d * d;
    sd = d * (1.0f - d2 * (1.0f / 6.0f) * (1.0f - d2 * 0.05f));
    cd = 1.0f - 0.5f * d2 * (1.0f - d2 * (1.0f / 12.0f));
  } else {
    sincosf(d, &sd, &cd);
  }
  const float s2 = s * cd + c * sd;
  const float c2 = c * cd - s * sd;
  s = s2;
  c = c2;
}

// Guard bands: a state whose FP32 value of e, p_L or r_k lies this close to a status
// threshold (or is not finite) is recomputed in FP64, so that the status equals the
// FP64 decision.  The FP32 errors of these quantities are ~1e-6 relative or less.
constexpr float kGuardE = 2.0e-5f;
constexpr float kGuardP = 2.0e-5f;
constexpr float kGuardR = 5.0e-5f;
constexpr int kRecomputeFP64 = -1;

// One state in FP32 with the n*t phase in double-float.  (th, tl) is tsince split as
// th + tl.  Returns the status code, or kRecomputeFP64 when the state must be
// recomputed by state64.
template <int K>
__device__ __forceinline__ int state32(const Rec32& rc, const GeoF& g, float th, float tl,
                                       float r[3], float v[3]) {
  const int fatal = (rc.flags >> kFatalShift) & 0xff;
  if (fatal) return fatal;
  if (rc.flags & kFlagN0ppNonPos) return 2;
  const bool isimp = rc.flags & kFlagIsimp;
  const float t = th;
  const float t2 = t * t;

  // Secular drag polynomials.
  float tempa = 1.0f - rc.c1 * t;
  float tempe = rc.bc4 * t;
  float templ = rc.l2 * t2;
  float dd = 0.0f;   // dargp + dM: moves M forward and argp back by the same angle
  if (!isimp) {
    const float dargp = rc.argpcf * t;
    const float mdf = wrap_rev(fmaf(rc.mdr, t, rc.m0r)) * kTwoPiF;
    const float c = 1.0f + rc.eta * cosf(mdf);
    const float dm = rc.mcf * (c * c * c - rc.delm0);
    dd = dargp + dm;
    const float t3 = t2 * t, t4 = t3 * t;
    tempa = tempa - rc.d2 * t2 - rc.d3 * t3 - rc.d4 * t4;
    tempe = tempe + rc.bc5 * (sinf(mdf + dd) - rc.sinm0);
    templ = templ + rc.l3 * t3 + t4 * (rc.l4 + t * rc.l5);
  }
  const float a = rc.a0pp * tempa * tempa;
  const float sa = sqrtf(a);
  const float n = g.xke / (a * sa);
  float e = rc.e0 - tempe;
  if (!(fabsf(e - 1.0f) >= kGuardE && fabsf(e + 0.001f) >= kGuardE)) return kRecomputeFP64;
  if (e >= 1.0f || e < -0.001f) return 1;
  if (e < 1.0e-6f) e = 1.0e-6f;

  // Phase of the mean argument of latitude, M + argp = M_DF + argp_DF + n0'' templ
  // (the drag corrections of M and argp cancel), in revolutions.  The n*t product is
  // evaluated as a double-float: (phidh + phidl) * (th + tl).
  float p = rc.phidh * th;
  const float pe = fmaf(rc.phidh, th, -p);            // exact rounding error of p
  const float s = fmaf(rc.phidh, tl, fmaf(rc.phidl, th, pe));
  p = p - rintf(p);                                    // exact
  float y = wrap_rev(p + rc.phi0h);
  y += s + rc.phi0l;
  y += wrap_rev(rc.n0ppr * templ);

  const float argp = wrap_rev(fmaf(rc.argpdr, t, rc.argp0r) - dd * kInvTwoPiF) * kTwoPiF;
  const float raan = wrap_rev(fmaf(rc.raancfr, t2, fmaf(rc.raandr, t, rc.raan0r))) * kTwoPiF;

  // Long-period periodics (J3).
  float sw, cw;
  sincosf(argp, &sw, &cw);
  const float axn = e * cw;
  const float q = 1.0f / (a * (1.0f - e * e));
  const float ayn = fmaf(e, sw, q * rc.aycof);
  const float U = wrap_rev(y + q * rc.xlcof * axn * kInvTwoPiF) * kTwoPiF;

  // Kepler: K Newton steps from psi = U, clamped to +-0.95.
  float psi = U;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float sp, cp;
    sincosf(psi, &sp, &cp);
    const float f = U - ayn * cp + axn * sp - psi;
    const float fp = 1.0f - ayn * sp - axn * cp;
    psi += fminf(fmaxf(__fdividef(f, fp), -0.95f), 0.95f);
  }
  float sp, cp;
  sincosf(psi, &sp, &cp);

  // Short-period preliminaries.
  const float ecosE = axn * cp + ayn * sp;
  const float esinE = axn * sp - ayn * cp;
  const float eL2 = axn * axn + ayn * ayn;
  const float pL = a * (1.0f - eL2);
  if (!(fabsf(pL) >= kGuardP)) return kRecomputeFP64;
  if (pL < 0.0f) return 4;
  const float rl = a * (1.0f - ecosE);
  const float invr = 1.0f / rl;
  const float rdotl = sa * esinE * invr;
  const float rfdotl = sqrtf(pL) * invr;
  const float betal = sqrtf(1.0f - eL2);
  const float w = esinE / (1.0f + betal);
  const float aor = a * invr;
  const float sinu = aor * (sp - ayn - axn * w);
  const float cosu = aor * (cp - axn + ayn * w);
  const float sin2u = 2.0f * cosu * sinu;
  const float cos2u = 1.0f - 2.0f * sinu * sinu;

  // Short-period periodics (J2).
  const float invp = 1.0f / pL;
  const float k = 0.5f * g.j2 * invp;
  const float kp = k * invp;
  const float rk = rl * (1.0f - 1.5f * kp * betal * rc.x3thm1) + 0.5f * k * rc.x1mth2 * cos2u;
  if (!(fabsf(rk - 1.0f) >= kGuardR)) return kRecomputeFP64;
  const float nk = n * k * g.inv_xke;
  const float rdotk = rdotl - nk * rc.x1mth2 * sin2u;
  const float rfdotk = rfdotl + nk * (rc.x1mth2 * cos2u + 1.5f * rc.x3thm1);

  // u_k, RAAN_k and i_k as small rotations of (sin, cos) pairs.
  const float nrm = rsqrtf(sinu * sinu + cosu * cosu);
  float su = sinu * nrm, cu = cosu * nrm;
  rotate_small(su, cu, -0.25f * kp * rc.x7thm1 * sin2u);
  float sO, cO;
  sincosf(raan, &sO, &cO);
  rotate_small(sO, cO, 1.5f * kp * rc.cosi * sin2u);
  float si = rc.sini, ci = rc.cosi;
  rotate_small(si, ci, 1.5f * kp * rc.cosi * rc.sini * cos2u);

  const float mx = -sO * ci, my = cO * ci, mz = si;
  const float ux = mx * su + cO * cu, uy = my * su + sO * cu, uz = mz * su;
  const float vx = mx * cu - cO * su, vy = my * cu - sO * su, vz = mz * cu;
  const float rs = rk * g.re;
  r[0] = rs * ux; r[1] = rs * uy; r[2] = rs * uz;
  v[0] = (rdotk * ux + rfdotk * vx) * g.vkmps;
  v[1] = (rdotk * uy + rfdotk * vy) * g.vkmps;
  v[2] = (rdotk * uz + rfdotk * vz) * g.vkmps;
  return rk < 1.0f ? 6 : 0;
}

}  // namespace sgp4
