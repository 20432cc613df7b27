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
//   [kNumF64 planes of double][stride rows of kF32Row floats][flags int32][epoch_day int32]
// planes are `stride` entries long, stride a multiple of 64 (256-byte planes).
enum F64Field {
  kN0pp, kA0pp, kE0, kI0, kRaan0, kArgp0, kM0, kBstar,
  kMdot, kArgpdot, kRaandot, kRaanCf, kArgpCf, kMCf,
  kC1, kBC4, kBC5, kD2, kD3, kD4, kL2, kL3, kL4, kL5,
  kEta, kDelM0, kSinM0, kXlcof, kAycof,
  kCosi, kSini, kX3thm1, kX1mth2, kX7thm1,
  kEpochFrac,
  // Deep space (period >= 225 min; written for deep-space records only): Greenwich
  // sidereal angle at the epoch, the lunar-solar secular rates, each body's long-period
  // amplitudes and mean anomaly at the epoch, the resonance amplitudes (one rev/day:
  // kDel1..3; two: kD2201..kD5433), the resonant longitude at the epoch and its rate
  // minus the mean motion.
  kGsto, kEdotLs, kIdotLs, kMdotLs, kArgpdotLs, kRaandotLs,
  kSunE2, kSunE3, kSunI2, kSunI3, kSunL2, kSunL3, kSunL4, kSunGh2, kSunGh3, kSunGh4,
  kSunH2, kSunH3, kSunM0,
  kMoonE2, kMoonE3, kMoonI2, kMoonI3, kMoonL2, kMoonL3, kMoonL4, kMoonGh2, kMoonGh3,
  kMoonGh4, kMoonH2, kMoonH3, kMoonM0,
  kDel1, kDel2, kDel3,
  kD2201, kD2211, kD3210, kD3222, kD4410, kD4422, kD5220, kD5232, kD5421, kD5433,
  kLambda0, kXfact,
  kNumF64
};
// Amplitudes of one body's long-period terms, in plane order from kSunE2 / kMoonE2.
constexpr int kBodyPlanes = kSunM0 - kSunE2 + 1;
static_assert(kMoonM0 - kMoonE2 + 1 == kBodyPlanes, "body plane blocks differ");

// FP32-path record: one 160-byte row of 40 floats per satellite (array of
// structures), read with ten 16-byte loads per state.  Angles and their rates are
// in revolutions (x / 2 pi) so that the reduction mod one revolution is a
// subtraction of rint(x).  The mean argument of latitude phase (M0 + argp0) and
// its rate (Mdot + argpdot) are unevaluated float sums hi + lo ("double-float").
// Slot fFlags holds the int32 flags word as raw bits.
enum F32Field {
  fPhi0H, fPhi0L, fPhiDH, fPhiDL,
  fM0r, fMdr, fArgp0r, fArgpdr, fRaan0r, fRaandr, fRaanCfr, fN0ppr,
  fA0pp, fE0, fC1, fBC4, fBC5, fD2, fD3, fD4, fL2, fL3, fL4, fL5,
  fEta, fDelM0, fSinM0, fArgpCf, fMCf, fXlcof, fAycof,
  fCosi, fSini, fX3thm1, fX1mth2, fX7thm1,   // fX3thm1 holds 1.5 (3 th^2 - 1), fX7thm1 holds
                                              // -0.25 (7 th^2 - 1): the factors they appear with
  fFlags,
  fHalfX1mth2, fC15Cosi, fC15CosiSini,        // 0.5 (1 - th^2), 1.5 cos i, 1.5 cos i sin i
  kNumF32Used
};
constexpr int kF32Row = 40;   // floats per satellite row (16-byte multiple)
static_assert(kNumF32Used <= kF32Row, "FP32 record row too small");

// flags word
constexpr int kFlagIsimp = 1;        // perigee below 220 km: truncated drag terms
constexpr int kFlagN0ppNonPos = 2;   // n0'' <= 0 -> code 2 at every t
constexpr int kFlagDeep = 4;         // deep space: FP64 deep-space state (the FP32 row's a0''
                                     // is NaN, which sends every FP32 state to FP64)
constexpr int kFlagRez1 = 16;        // deep space, one-revolution-per-day resonance
constexpr int kFlagRez2 = 32;        // deep space, two-revolutions-per-day resonance
constexpr int kFatalShift = 8;       // bits 8..15: fatal input code (1 or 2)

__host__ __device__ inline int64_t record_stride(int64_t n) { return ((n + 63) / 64) * 64; }

__host__ __device__ inline size_t record_bytes(int64_t n) {
  const int64_t s = record_stride(n);
  return (size_t)s * (sizeof(double) * kNumF64 + sizeof(float) * kF32Row + 2 * sizeof(int32_t));
}

struct RecordPtrs {
  double* f64;      // [kNumF64][stride]
  float* f32;       // [stride][kF32Row]
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
  base += sizeof(float) * kF32Row * p.stride;
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
  double inv_xke; // 1 / xke and 1 / re, taken once on the host (an FP64 division is a
  double inv_re;  // chain of FP64-unit instructions on B300)
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

// Angle reduction like C fmod(x, 2 pi) (sign kept), as x - 2 pi trunc(x / 2 pi): the
// same value to rounding, without fmod's iterative remainder on the FP64 unit.
__device__ __forceinline__ double wrap_2pi(double x) {
  return fma(-kTwoPi, trunc(x * (1.0 / kTwoPi)), x);
}

// sin d and cos d in FP64: 7th/6th-order Taylor pair for |d| < 1e-2 (truncation below
// 3e-18), the full sincos beyond.
__device__ __forceinline__ void sincos_small64(double d, double& sd, double& cd) {
  if (fabs(d) < 1.0e-2) {
    const double d2 = d * d;
    sd = d * (1.0 - d2 * (1.0 / 6.0) * (1.0 - d2 * (1.0 / 20.0) * (1.0 - d2 * (1.0 / 42.0))));
    cd = 1.0 - 0.5 * d2 * (1.0 - d2 * (1.0 / 12.0) * (1.0 - d2 * (1.0 / 30.0)));
  } else {
    sincos(d, &sd, &cd);
  }
}
// Rotate (s, c) = (sin a, cos a) to (sin(a+d), cos(a+d)) in FP64.
__device__ __forceinline__ void rotate64(double& s, double& c, double d) {
  double sd, cd;
  sincos_small64(d, sd, cd);
  const double s2 = s * cd + c * sd;
  const double c2 = c * cd - s * sd;
  s = s2;
  c = c2;
}

// Newton steps for Kepler's equation in FP64 from psi0 = U (same bound as the FP32
// path, target 1e-15 rad), thresholds on e_L^2: 1 step for e_L <= 1.26e-5, 2 for
// <= 0.0096, 3 for <= 0.129, 4 for <= 0.367, 5 for <= 0.5; beyond that the theory's
// rule (stop when a step is below 1e-12, at most 10 steps).
__device__ __forceinline__ int newton_steps64(double eL2) {
  return eL2 <= 1.5876e-10 ? 1 : eL2 <= 9.3e-5 ? 2 : eL2 <= 0.01664 ? 3 : eL2 <= 0.1347 ? 4
       : eL2 <= 0.25 ? 5 : 10;
}

// From the mean elements after all secular (and, in deep space, lunar-solar) terms to
// r, v: a (Earth radii), e, node, perigee, M + perigee (mpa), the J3 coefficients and
// the inclination's functions (x3thm1 = 3 cos^2 i - 1, x1mth2 = 1 - cos^2 i, x7thm1 =
// 7 cos^2 i - 1).
__device__ __forceinline__ int state64_tail(const Geo& g, double a, double e, double raan,
                                            double argp, double mpa, double xlcof,
                                            double aycof, double cosi, double sini,
                                            double x3thm1, double x1mth2, double x7thm1,
                                            double r[3], double v[3]) {
  // square roots and reciprocals through rsqrt (one FP64-unit sequence instead of a
  // square root and a division)
  const double ra = rsqrt(a);
  const double sa = a * ra;
  const double ia15 = ra * ra * ra;                    // n / ke

  // Long-period periodics (J3).
  double sw, cw;
  sincos(argp, &sw, &cw);
  const double axn = e * cw;
  const double q = 1.0 / (a * (1.0 - e * e));
  const double ayn = e * sw + q * aycof;
  const double U = wrap_2pi(mpa + q * xlcof * axn);
  const double eL2 = axn * axn + ayn * ayn;

  // Kepler's equation: Newton with clamped steps, count from the e_L bound.
  // sin, cos of the first iterate from sincos, of later ones by rotating the previous
  // pair by the step taken (Taylor for small steps): one FP64 sincos per state.
  double psi = U, sp, cp, step = 0.0;
  sincos(U, &sp, &cp);
  const int K = newton_steps64(eL2);
  for (int k = 0; k < K; ++k) {
    if (k > 0) rotate64(sp, cp, step);
    step = (U - ayn * cp + axn * sp - psi) / (1.0 - ayn * sp - axn * cp);
    step = fmin(fmax(step, -0.95), 0.95);
    psi += step;
    if (K == 10 && fabs(step) < 1.0e-12) break;
  }
  rotate64(sp, cp, step);      // sin, cos at the final iterate

  // Short-period preliminaries.
  const double ecosE = axn * cp + ayn * sp;
  const double esinE = axn * sp - ayn * cp;
  const double pL = a * (1.0 - eL2);
  if (pL < 0.0) return 4;
  const double rl = a * (1.0 - ecosE);
  const double invr = 1.0 / rl;
  const double rdotl = sa * esinE * invr;
  const double rpl = rsqrt(pL);
  const double spl = pL * rpl;
  const double rfdotl = spl * invr;
  const double betal = sqrt(1.0 - eL2);
  const double w = esinE / (1.0 + betal);
  const double aor = a * invr;
  const double sinu = aor * (sp - ayn - axn * w);
  const double cosu = aor * (cp - axn + ayn * w);
  const double sin2u = 2.0 * cosu * sinu;
  const double cos2u = 1.0 - 2.0 * sinu * sinu;

  // Short-period periodics (J2).
  const double invp = rpl * rpl;
  const double k = 0.5 * g.j2 * invp;
  const double kp = k * invp;
  const double rk = rl * (1.0 - 1.5 * kp * betal * x3thm1) + 0.5 * k * x1mth2 * cos2u;
  const double nk = ia15 * k;          // n k / ke
  const double rdotk = rdotl - nk * x1mth2 * sin2u;
  const double rfdotk = rfdotl + nk * (x1mth2 * cos2u + 1.5 * x3thm1);

  // u_k, RAAN_k and i_k as rotations of (sin, cos) pairs.
  const double nrm = rsqrt(sinu * sinu + cosu * cosu);
  double su = sinu * nrm, cu = cosu * nrm;
  rotate64(su, cu, -0.25 * kp * x7thm1 * sin2u);
  double sO, cO;
  sincos(raan, &sO, &cO);
  rotate64(sO, cO, 1.5 * kp * cosi * sin2u);
  double si = sini, ci = cosi;
  rotate64(si, ci, 1.5 * kp * cosi * sini * cos2u);

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

// One state in FP64.  Returns the status code; r (km) and v (km/s) are written
// for codes 0 and 6 only.  Same theory and status decisions as the FP32 path and the
// textbook form: atan2 and the sin/cos of u_k, RAAN_k, i_k are replaced by small
// rotations of (sin, cos) pairs by the short-period corrections.
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
  double argp = argpdf;
  double tempa = 1.0 - rc.c1 * t;
  double tempe = rc.bc4 * t;
  double templ = rc.l2 * t2;
  if (!isimp) {
    const double dargp = rc.argp_cf * t;
    double sm, cm;
    sincos(wrap_2pi(mdf), &sm, &cm);
    const double c = 1.0 + rc.eta * cm;
    const double dm = rc.m_cf * (c * c * c - rc.delm0);
    const double dd = dargp + dm;
    argp = argpdf - dd;
    const double t3 = t2 * t, t4 = t3 * t;
    tempa = tempa - rc.d2 * t2 - rc.d3 * t3 - rc.d4 * t4;
    double sdd, cdd;
    sincos_small64(dd, sdd, cdd);   // the drag shift dd is usually small
    tempe = tempe + rc.bc5 * (sm * cdd + cm * sdd - rc.sinm0);   // sin(M_DF + dd)
    templ = templ + rc.l3 * t3 + t4 * (rc.l4 + t * rc.l5);
  }
  if (rc.flags & kFlagN0ppNonPos) return 2;
  const double a = rc.a0pp * tempa * tempa;
  double e = rc.e0 - tempe;
  if (e >= 1.0 || e < -0.001) return 1;
  if (e < 1.0e-6) e = 1.0e-6;
  raan = wrap_2pi(raan);
  argp = wrap_2pi(argp);
  // M + argp: the drag corrections of M and argp cancel.
  const double mpa = mdf + argpdf + rc.n0pp * templ;
  return state64_tail(g, a, e, raan, argp, mpa, rc.xlcof, rc.aycof, rc.cosi, rc.sini,
                      rc.x3thm1, rc.x1mth2, rc.x7thm1, r, v);
}

// ============================================================== FP32 state
struct GeoF {
  float xke, inv_xke, j2, re, vkmps;
  float half_j2;
};

struct Rec32 {
  float phi0h, phi0l, phidh, phidl;
  float m0r, mdr, argp0r, argpdr, raan0r, raandr, raancfr, n0ppr;
  float a0pp, e0, c1, bc4, bc5, d2, d3, d4, l2, l3, l4, l5;
  float eta, delm0, sinm0, argpcf, mcf, xlcof, aycof;
  float cosi, sini, x3thm1_15, x1mth2, x7thm1_m025;
  float half_x1mth2, c15cosi, c15cosisini;
  int flags;
};

// Unpack ten float4 of one FP32 row.
__device__ __forceinline__ Rec32 unpack_rec32(const float4 q0, const float4 q1, const float4 q2,
                                              const float4 q3, const float4 q4, const float4 q5,
                                              const float4 q6, const float4 q7, const float4 q8,
                                              const float4 q9);

// Read-only path (__ldg): only for rows that no thread of the running kernel writes.
__device__ __forceinline__ Rec32 load_rec32(const RecordPtrs& rp, int64_t j) {
  const float4* __restrict__ row = reinterpret_cast<const float4*>(rp.f32 + j * kF32Row);
  return unpack_rec32(__ldg(row + 0), __ldg(row + 1), __ldg(row + 2), __ldg(row + 3),
                      __ldg(row + 4), __ldg(row + 5), __ldg(row + 6), __ldg(row + 7),
                      __ldg(row + 8), __ldg(row + 9));
}

// Coherent path: for a row the calling thread has just written (the record builder).
__device__ __forceinline__ Rec32 read_own_rec32(const float* row_f) {
  const float4* row = reinterpret_cast<const float4*>(row_f);
  return unpack_rec32(row[0], row[1], row[2], row[3], row[4], row[5], row[6], row[7], row[8],
                      row[9]);
}

__device__ __forceinline__ Rec32 unpack_rec32(const float4 q0, const float4 q1, const float4 q2,
                                              const float4 q3, const float4 q4, const float4 q5,
                                              const float4 q6, const float4 q7, const float4 q8,
                                              const float4 q9) {
  Rec32 r;
  r.phi0h = q0.x; r.phi0l = q0.y; r.phidh = q0.z; r.phidl = q0.w;
  r.m0r = q1.x; r.mdr = q1.y; r.argp0r = q1.z; r.argpdr = q1.w;
  r.raan0r = q2.x; r.raandr = q2.y; r.raancfr = q2.z; r.n0ppr = q2.w;
  r.a0pp = q3.x; r.e0 = q3.y; r.c1 = q3.z; r.bc4 = q3.w;
  r.bc5 = q4.x; r.d2 = q4.y; r.d3 = q4.z; r.d4 = q4.w;
  r.l2 = q5.x; r.l3 = q5.y; r.l4 = q5.z; r.l5 = q5.w;
  r.eta = q6.x; r.delm0 = q6.y; r.sinm0 = q6.z; r.argpcf = q6.w;
  r.mcf = q7.x; r.xlcof = q7.y; r.aycof = q7.z; r.cosi = q7.w;
  r.sini = q8.x; r.x3thm1_15 = q8.y; r.x1mth2 = q8.z; r.x7thm1_m025 = q8.w;
  r.flags = __float_as_int(q9.x);
  r.half_x1mth2 = q9.y; r.c15cosi = q9.z; r.c15cosisini = q9.w;
  return r;
}

// Round to the nearest integer (ties to even) for |x| < 2^22 without a rounding or
// conversion instruction: adding 1.5 * 2^23 leaves a float whose unit in the last
// place is 1, so the addition itself rounds.  On B300 the float<->int conversions and
// FRND share the small FP64 unit; these two adds run on the FMA pipe.
constexpr float kRoundMagic = 12582912.0f;   // 1.5 * 2^23
__device__ __forceinline__ float round_magic(float x) {
  return __fsub_rn(__fadd_rn(x, kRoundMagic), kRoundMagic);
}
// The same rounding, also returning the integer (from the bits of x + 1.5 * 2^23).
__device__ __forceinline__ float round_magic_int(float x, int& q) {
  const float y = __fadd_rn(x, kRoundMagic);
  q = __float_as_int(y) - __float_as_int(kRoundMagic);
  return __fsub_rn(y, kRoundMagic);
}
// Exact float of an integer with |i| < 2^22 (same trick in reverse).
__device__ __forceinline__ float int_to_float_small(int i) {
  return __fsub_rn(__int_as_float(__float_as_int(kRoundMagic) + i), kRoundMagic);
}

// SFU reciprocal square root with subnormal inputs flushed to zero.  Every argument in
// the FP32 states (a, a(1 - e^2), the Newton derivative, r_L, p_L, 1 - e_L^2, 1 + beta_L,
// sin^2 u + cos^2 u) is a normal number of order one on a state outside the guard
// bands, and guard-band states are recomputed in FP64, so the flush never changes a
// kept result.  rsqrtf's handling of subnormal inputs took 8% of the FP32 propagation
// kernel's time on B300 (about 3 more instructions per call).
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1 / y for y > 0 as rsqrt(y)^2 (one SFU operation and a multiply, ~2 ulp).  On B300
// the fast-divide intrinsic puts an instruction on the small FP64 unit (4 per state
// kept that unit 36% busy); every denominator of the FP32 path is positive.
__device__ __forceinline__ float rcp_pos(float y) {
  const float r = rsqrt_ftz(y);
  return r * r;
}

// Reduce an angle in revolutions to [-1/2, 1/2].  Exact for |x| < 2^22.
__device__ __forceinline__ float wrap_rev(float x) { return x - round_magic(x); }

// Split a double into float hi + lo with hi = t rounded to float and lo = the
// remainder rounded to float (so hi + lo carries ~48 significant bits), using only
// integer operations: B300's FP64 unit is a small fraction of the FP32 rate, and a
// conversion through it per state would be the kernel's busiest pipe.  IEEE 754
// binary64: hi keeps the top 24 bits of the 53-bit significand (round to nearest,
// ties to even), lo is the signed 29-bit remainder times 2^(exponent - 52).
// |t| < 2^-74 min (3e-21 s) is taken as zero; |t| >= 2^128 gives hi = +-inf.
__device__ __forceinline__ void split_double(double t, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(t);
  const unsigned w1 = (unsigned)(b >> 32), w0 = (unsigned)b;
  const int e = (int)((w1 >> 20) & 0x7ffu);
  const unsigned sign = w1 & 0x80000000u;
  if (e < 949) { hi = 0.0f; lo = 0.0f; return; }
  if (e > 1150) { hi = __uint_as_float(sign | 0x7f800000u); lo = 0.0f; return; }
  unsigned hs = (((w1 & 0xfffffu) | 0x100000u) << 3) | (w0 >> 29);   // 24-bit significand
  const unsigned rem = w0 & 0x1fffffffu;                                // low 29 bits
  const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (hs & 1u))) ? 1u : 0u;
  hs += up;   // a carry to 2^24 propagates into the exponent field below
  hi = __uint_as_float((sign | ((unsigned)(e - 896) << 23)) + (hs - 0x800000u));
  const int d = (int)rem - (up ? 0x20000000 : 0);                       // |d| <= 2^28
  // float(d) rounded once: d = dh * 2^12 + dl with both parts exact in float.
  const float fd = fmaf(int_to_float_small(d >> 12), 4096.0f, int_to_float_small(d & 4095));
  const float l = fd * __uint_as_float((unsigned)(e - 948) << 23);       // d * 2^(e-1075)
  lo = sign ? -l : l;
}

// double -> float rounded to nearest (ties to even) with integer operations only, for
// code that runs on B300's small FP64 unit, where a conversion instruction costs as
// much as a DFMA.  |x| below the smallest normal float (2^-126) gives a signed zero;
// beyond the float range +-inf; NaN stays NaN.
__device__ __forceinline__ float f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned w1 = (unsigned)(b >> 32), w0 = (unsigned)b;
  const int e = (int)((w1 >> 20) & 0x7ffu);
  const unsigned sign = w1 & 0x80000000u;
  if (e == 0x7ff)
    return __uint_as_float(sign | 0x7f800000u | (((w1 & 0xfffffu) | w0) ? 0x400000u : 0u));
  if (e < 897) return __uint_as_float(sign);
  if (e > 1150) return __uint_as_float(sign | 0x7f800000u);
  const unsigned m = ((w1 & 0xfffffu) << 3) | (w0 >> 29);   // top 23 fraction bits
  const unsigned rem = w0 & 0x1fffffffu;                     // the 29 bits dropped
  unsigned f = ((unsigned)(e - 896) << 23) + m;              // float exponent bias 127
  if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) f += 1u;   // carry is exact
  return __uint_as_float(sign | f);
}

// sin and cos of x, |x| <= 2^12, to ~1e-7 absolute: Cody-Waite reduction by pi/2
// with a two-part constant applied by FMA, then the Taylor series of sin (degree 9)
// and cos (degree 10) on [-pi/4, pi/4] (truncation below 2e-9), and the quadrant
// swap.  Used where an angle's error goes straight into the position (the final
// Kepler iterate and the node); elsewhere the SFU's __sincosf is accurate enough.
__device__ __forceinline__ void sincos_acc(float x, float* sp, float* cp) {
  int q;
  const float k = round_magic_int(x * 0.636619772367581343f, q);
  float r = fmaf(k, -1.57079637050628662f, x);
  r = fmaf(k, 4.37113900018624284e-8f, r);
  const float r2 = r * r;
  float ps = fmaf(r2, 2.75573192239858907e-6f, -1.98412698412698413e-4f);
  ps = fmaf(r2, ps, 8.33333333333333333e-3f);
  ps = fmaf(r2, ps, -1.66666666666666667e-1f);
  const float sn = fmaf(r * r2, ps, r);
  float pc = fmaf(r2, -2.75573192239858907e-7f, 2.48015873015873016e-5f);
  pc = fmaf(r2, pc, -1.38888888888888889e-3f);
  pc = fmaf(r2, pc, 4.16666666666666667e-2f);
  pc = fmaf(r2, pc, -0.5f);
  const float cs = fmaf(r2, pc, 1.0f);
  const float s0 = (q & 1) ? cs : sn;
  const float c0 = (q & 1) ? sn : cs;
  *sp = (q & 2) ? -s0 : s0;
  *cp = ((q + 1) & 2) ? -c0 : c0;
}

// Rotate the unit vector (s, c) = (sin a, cos a) to (sin(a+d), cos(a+d)).  The
// corrections d of the short-period terms are O(J2/p_L^2): below ~1e-3 rad for
// near-Earth orbits, where a 3rd/2nd-order Taylor pair is exact to float precision.
// |d| >= 4e-3 needs p_L < ~0.45 Earth radii (a perigee deep inside the Earth); the
// FP32 path hands such states to the FP64 recomputation instead.
__device__ __forceinline__ void rotate_small(float& s, float& c, float d) {
  // truncation d^5/120 and d^4/24 stay below 1e-11 for |d| < 4e-3 (callers check)
  const float d2 = d * d;
  const float sd = fmaf(d2 * (-1.0f / 6.0f), d, d);
  const float cd = fmaf(-0.5f, d2, 1.0f);
  const float s2 = s * cd + c * sd;
  const float c2 = c * cd - s * sd;
  s = s2;
  c = c2;
}

// Newton steps needed for Kepler's equation from psi0 = U: with |psi0 - psi*| <= e_L,
// f' >= 1 - e_L and |f''| <= e_L the error obeys err' <= e_L/(2(1-e_L)) err^2, which
// reaches 1e-8 rad after 1 step for e_L <= 0.0027, 2 for <= 0.093, 3 for <= 0.33 and
// 4 for <= 0.5; beyond that the theory's cap of 10 steps is used.
// The thresholds below are on e_L^2.
__device__ __forceinline__ int newton_steps(float eL2) {
  return eL2 <= 6.25e-6f ? 1 : eL2 <= 0.0081f ? 2 : eL2 <= 0.1089f ? 3 : eL2 <= 0.25f ? 4 : 10;
}

// Guard bands: a state whose FP32 value of e, p_L or r_k lies this close to a status
// threshold (or is not finite) is recomputed in FP64, so that the status equals the
// FP64 decision.  The FP32 errors of these quantities are ~1e-6 relative or less.
constexpr float kGuardE = 2.0e-5f;
constexpr float kGuardP = 2.0e-5f;
constexpr float kGuardR = 5.0e-5f;
// The long-period correction of U, q xlcof a_xN (rad), has the factor 1 / (1 + cos i)
// and grows without bound as the inclination nears 180 degrees; in FP32 its rounding
// error (~6e-8 of it) reaches the position once it exceeds a radian, so such states are
// recomputed in FP64 too (inclinations within a few hundredths of a degree of 180).
constexpr float kGuardLongPeriod = 1.0f;
// The drag part of the mean longitude, n0'' (L2 t^2 + .. + L5 t^5), is evaluated in FP32
// (in revolutions): its rounding error (a few 1e-7 of it) reaches the along-track
// position as it grows, and on records whose drag polynomial of the semi-major axis has
// passed its minimum (the mean orbit then balloons to millions of km) it reaches
// thousands of revolutions.  Past one revolution (about 13 m of along-track error at
// LEO radius) the state is recomputed in FP64: 3e-4 of the seven-day catalogue's
// states, 2e-4 of the element-fitting set's (its orbits with a perigee inside the
// atmosphere), none of the one-day Starlink-shaped set's.
constexpr float kGuardDragPhase = 1.0f;
constexpr int kRecomputeFP64 = -1;

// One state in FP32 with the n*t phase in double-float.  (th, tl) is tsince split as
// th + tl.  Returns the status code, or kRecomputeFP64 when the state must be
// recomputed by state64.  The status checks of the theory are evaluated as flags with a
// single exit at the end (states with a nonzero code compute on and are discarded):
// early returns cost every state divergence bookkeeping.
__device__ __forceinline__ int state32(const Rec32& rc, const GeoF& g, float th, float tl,
                                       float r[3], float v[3]) {
  const int fatal = (rc.flags >> kFatalShift) & 0xff;
  const int code0 = fatal ? fatal : ((rc.flags & kFlagN0ppNonPos) ? 2 : 0);
  const float t = th;
  const float t2 = t * t;

  // Secular drag polynomials.  Simplified-drag records carry zero d2..l5, bc5, argpcf
  // and mcf in the FP32 row, so the full form gives their truncated one without a
  // branch.
  const float dargp = rc.argpcf * t;
  const float mdf = wrap_rev(fmaf(rc.mdr, t, rc.m0r)) * kTwoPiF;
  const float c = 1.0f + rc.eta * __cosf(mdf);
  const float dm = rc.mcf * (c * c * c - rc.delm0);
  const float dd = dargp + dm;   // moves M forward and argp back by the same angle
  const float t3 = t2 * t, t4 = t3 * t;
  const float tempa = 1.0f - rc.c1 * t - rc.d2 * t2 - rc.d3 * t3 - rc.d4 * t4;
  const float tempe = rc.bc4 * t + rc.bc5 * (__sinf(mdf + dd) - rc.sinm0);
  const float templ = rc.l2 * t2 + rc.l3 * t3 + t4 * (rc.l4 + t * rc.l5);
  const float a = rc.a0pp * tempa * tempa;
  float e = rc.e0 - tempe;
  // Status checks in the theory's order (2, 1, 4, 6) and the guard bands around them,
  // as predicates combined at the end.
  const bool g_e = !(fabsf(e - 1.0f) >= kGuardE) | !(fabsf(e + 0.001f) >= kGuardE) |
                   !(a > 1.0e-3f);
  const bool f_e = (e >= 1.0f) | (e < -0.001f);
  e = fmaxf(e, 1.0e-6f);
  const float ra = rsqrt_ftz(a);
  const float sa = a * ra;
  const float ra3 = ra * ra * ra;           // n / ke = a^-1.5

  // Phase of the mean argument of latitude, M + argp = M_DF + argp_DF + n0'' templ
  // (the drag corrections of M and argp cancel), in revolutions.  The n*t product is
  // evaluated as a double-float: (phidh + phidl) * (th + tl).
  float p = rc.phidh * th;
  const float pe = fmaf(rc.phidh, th, -p);            // exact rounding error of p
  const float s = fmaf(rc.phidh, tl, fmaf(rc.phidl, th, pe));
  p = p - round_magic(p);                              // exact
  float y = wrap_rev(p + rc.phi0h);
  y += s + rc.phi0l;
  const float lrev = rc.n0ppr * templ;
  const bool g_l = !(fabsf(lrev) < kGuardDragPhase);
  y += wrap_rev(lrev);

  const float argp = wrap_rev(fmaf(rc.argpdr, t, rc.argp0r) - dd * kInvTwoPiF) * kTwoPiF;
  const float raan = wrap_rev(fmaf(rc.raancfr, t2, fmaf(rc.raandr, t, rc.raan0r))) * kTwoPiF;

  // Long-period periodics (J3).
  float sw, cw;
  __sincosf(argp, &sw, &cw);
  const float axn = e * cw;
  const float q = rcp_pos(a * (1.0f - e * e));
  const float ayn = fmaf(e, sw, q * rc.aycof);
  const float lpt = q * rc.xlcof * axn;
  const bool g_lp = !(fabsf(lpt) < kGuardLongPeriod);
  const float U = wrap_rev(y + lpt * kInvTwoPiF) * kTwoPiF;
  const float eL2 = axn * axn + ayn * ayn;

  // Kepler: Newton from psi = U, clamped to +-0.95, step count from the e_L bound.
  float psi = U;
  // The warp's largest step count, so that the loop is uniform across the warp (the
  // lanes of a warp are mostly one satellite at neighbouring times; extra steps only
  // refine a converged root).
  const int K = __reduce_max_sync(__activemask(), newton_steps(eL2));
  for (int k = 0; k < K; ++k) {
    float sp, cp;
    __sincosf(psi, &sp, &cp);
    const float f = U - ayn * cp + axn * sp - psi;
    const float fp = 1.0f - ayn * sp - axn * cp;
    psi += fminf(fmaxf(f * rcp_pos(fp), -0.95f), 0.95f);
  }
  float sp, cp;
  sincos_acc(psi, &sp, &cp);

  // Short-period preliminaries.
  const float ecosE = axn * cp + ayn * sp;
  const float esinE = axn * sp - ayn * cp;
  const float pL = a * (1.0f - eL2);
  const bool g_p = !(fabsf(pL) >= kGuardP);
  const bool f_p = pL < 0.0f;
  const float rl = a * (1.0f - ecosE);
  const float invr = rcp_pos(rl);
  const float rdotl = sa * esinE * invr;
  const float rpl = rsqrt_ftz(pL);
  const float rfdotl = pL * rpl * invr;
  const float omel = 1.0f - eL2;
  const float betal = omel * rsqrt_ftz(omel);
  const float w = esinE * rcp_pos(1.0f + betal);
  const float aor = a * invr;
  const float sinu = aor * (sp - ayn - axn * w);
  const float cosu = aor * (cp - axn + ayn * w);
  const float sin2u = 2.0f * cosu * sinu;
  const float cos2u = 1.0f - 2.0f * sinu * sinu;

  // Short-period periodics (J2).
  const float invp = rpl * rpl;
  const float k = g.half_j2 * invp;
  const float kp = k * invp;
  const float rk = rl * fmaf(-kp * betal, rc.x3thm1_15, 1.0f) + k * rc.half_x1mth2 * cos2u;
  const bool g_r = !(fabsf(rk - 1.0f) >= kGuardR);
  const float nk = ra3 * k;                 // n k / ke
  const float rdotk = rdotl - nk * rc.x1mth2 * sin2u;
  const float rfdotk = fmaf(nk, fmaf(rc.x1mth2, cos2u, rc.x3thm1_15), rfdotl);

  // u_k, RAAN_k and i_k as small rotations of (sin, cos) pairs.
  const float du = kp * rc.x7thm1_m025 * sin2u;
  const float dO = kp * rc.c15cosi * sin2u;
  const float di = kp * rc.c15cosisini * cos2u;
  const bool g_d = !(fmaxf(fabsf(du), fmaxf(fabsf(dO), fabsf(di))) < 4.0e-3f);
  const float nrm = rsqrt_ftz(sinu * sinu + cosu * cosu);
  float su = sinu * nrm, cu = cosu * nrm;
  rotate_small(su, cu, du);
  float sO, cO;
  __sincosf(raan, &sO, &cO);   // SFU: <= 3.6e-7 rad, a few metres at LEO radius
  rotate_small(sO, cO, dO);
  float si = rc.sini, ci = rc.cosi;
  rotate_small(si, ci, di);

  const float mx = -sO * ci, my = cO * ci, mz = si;
  const float ux = mx * su + cO * cu, uy = my * su + sO * cu, uz = mz * su;
  const float vx = mx * cu - cO * su, vy = my * cu - sO * su, vz = mz * cu;
  const float rs = rk * g.re;
  r[0] = rs * ux; r[1] = rs * uy; r[2] = rs * uz;
  v[0] = (rdotk * ux + rfdotk * vx) * g.vkmps;
  v[1] = (rdotk * uy + rfdotk * vy) * g.vkmps;
  v[2] = (rdotk * uz + rfdotk * vz) * g.vkmps;
  // A guard matters only while no earlier check has failed for certain.
  const bool need64 = g_e | (!f_e & (g_lp | g_l | g_p | (!f_p & (g_r | g_d))));
  int code = f_e ? 1 : (f_p ? 4 : (rk < 1.0f ? 6 : 0));
  code = need64 ? kRecomputeFP64 : code;
  return code0 ? code0 : code;
}

}  // namespace sgp4
