// Deep-space branch of SGP4 (SDP4) on sm_103a: the record constants and the FP64 state.
//
// Orbits with a period of 225 min or more take the deep-space branch of the 2006
// revision of Spacetrack Report #3 (the paper names it as future work, Sec. 6 and 7):
// the Sun's and Moon's perturbations from the quadrupole term of their tides (secular
// rates and long-period terms) and, near one and two revolutions per day, tesseral
// resonance integrated in the resonant longitude.  Deep-space states always run in
// FP64: the record builder makes the FP32 row's a0'' NaN, which every FP32 state
// sends to the FP64 recomputation (no test in the FP32 loops), and the FP64 states
// dispatch on the record's kFlagDeep.
//
// Readings (the CPU reference takes the same): the 2006 revision's "improved" mode
// (sidereal angle at the epoch from the IAU 1982 expression, no wrap of the node to
// [0, 2 pi) in the Lyddane form); the lunar-solar periodic terms applied absolutely;
// code 3 when the eccentricity after them leaves [0, 1], checked between codes 1 and
// 4; the resonance integrated for |tsince| <= 1e7 min, code 2 beyond that or for a
// non-finite tsince.
#pragma once

#include <cstdint>

#include "sgp4_device.cuh"

namespace sgp4 {
namespace deep {

// Sun and Moon: mean motion (rad/min), eccentricity, tide coefficient.
constexpr double kSunN = 1.19459e-5, kSunE = 0.01675, kSunC = 2.9864797e-6;
constexpr double kMoonN = 1.5835218e-4, kMoonE = 0.05490, kMoonC = 4.7968065e-7;
// sin and cos of the ecliptic's obliquity; cos and sin of the Sun's perigee argument.
constexpr double kSinObl = 0.39785416, kCosObl = 0.91744867;
constexpr double kCosPerSun = 0.1945905, kSinPerSun = -0.98088458;
constexpr double kEarthRot = 4.37526908801129966e-3;   // rad/min
// Tesseral terms of the one-revolution-per-day resonance: amplitudes of (2,2), (3,1),
// (3,3) and the phases in sin(k (lambda - phase)), k = 2, 1, 3.
constexpr double kQ22 = 1.7891679e-6, kQ31 = 2.1460748e-6, kQ33 = 2.2123015e-7;
constexpr double kPh22 = 2.8843198, kPh31 = 0.13130908, kPh33 = 0.37448087;
// ... and of the two-per-day resonance: amplitudes and argument phases of (2,2),
// (3,2), (4,4), (5,2), (5,4).
constexpr double kR22 = 1.7891679e-6, kR32 = 3.7393792e-7, kR44 = 7.3636953e-9;
constexpr double kR52 = 1.1428639e-7, kR54 = 2.1765803e-9;
constexpr double kG22 = 5.7686396, kG32 = 0.95240898, kG44 = 1.8014998;
constexpr double kG52 = 1.0508330, kG54 = 4.4108898;
constexpr double kStep = 720.0;     // resonance integrator step (min)
constexpr double kMaxT = 1.0e7;     // |tsince| the resonance integration covers (min)

}  // namespace deep

// Period 2 pi / n0'' of 225 min or more.
__host__ __device__ inline bool is_deep(double n0pp) { return kTwoPi / n0pp >= 225.0; }

// Resonance class from n0'' and e0: 1 for periods in (1200, 1800) min, 2 for mean
// motions in [8.26e-3, 9.24e-3] rad/min with e0 >= 0.5, else 0.
__host__ __device__ inline int resonance_class(double n0pp, double e0) {
  int c = 0;
  if (n0pp < 0.0052359877 && n0pp > 0.0034906585) c = 1;
  if (n0pp >= 8.26e-3 && n0pp <= 9.24e-3 && e0 >= 0.5) c = 2;
  return c;
}

// Greenwich mean sidereal angle (rad, [0, 2 pi)) at the Julian date day + frac: the
// IAU 1982 polynomial in Julian centuries from J2000, in seconds of time.
__device__ __forceinline__ double gmst_rad(int32_t day, double frac) {
  const double T = ((double)(day - 2451545) + frac) / 36525.0;
  const double sec = 67310.54841 + T * ((876600.0 * 3600.0 + 8640184.812866) +
                                        T * (0.093104 - 6.2e-6 * T));
  double th = fmod(sec * (kTwoPi / 86400.0), kTwoPi);
  return th < 0.0 ? th + kTwoPi : th;
}

// What the deep-space constants take from the near-Earth build.
struct DeepIn {
  double e0, i0, raan0, argp0, m0, n0pp, cosi, sini, mdot, argpdot, raandot, xke;
};

// One body's tide on the epoch orbit.  The body's orbit plane has inclination (cI, sI)
// to the equator; its perigee lies at the angle (cg, sg) from that plane's ascending
// node on the equator, which lies at (ch, sh) behind the satellite's node.  P, Q are
// the body's perigee direction and in-plane normal, first on the satellite's node
// axes (n: node line, m: in-plane normal to it, z: orbit normal), then on its perigee
// axes (x, y).  Writes the body's long-period amplitudes and mean anomaly at the epoch
// to planes [base, base + kBodyPlanes) and adds its secular rates (e, i, M, perigee,
// node) to rate[].
__device__ __forceinline__ void deep_body(double cg, double sg, double cI, double sI, double ch,
                                          double sh, double nb, double eb, double cb,
                                          double mb0, const DeepIn& in, double cw, double sw,
                                          bool near_equatorial, double* f, int64_t s,
                                          int64_t j, int base, double rate[5]) {
  const double ci = in.cosi, si = in.sini;
  const double Pn = cg * ch + sg * cI * sh;
  const double Qn = cg * cI * sh - sg * ch;
  const double Pe = sg * cI * ch - cg * sh;      // on the equatorial normal to the node line
  const double Qe = sg * sh + cg * cI * ch;
  const double Pm = ci * Pe + si * (sg * sI);
  const double Qm = ci * Qe + si * (cg * sI);
  const double Pz = ci * (sg * sI) - si * Pe;
  const double Qz = ci * (cg * sI) - si * Qe;
  const double Px = Pn * cw + Pm * sw, Py = Pm * cw - Pn * sw;
  const double Qx = Qn * cw + Qm * sw, Qy = Qm * cw - Qn * sw;

  const double e = in.e0, e2 = e * e, b2 = 1.0 - e2, beta = sqrt(b2);
  const double z31 = 12.0 * Px * Px - 3.0 * Py * Py;
  const double z32 = 24.0 * Px * Qx - 6.0 * Py * Qy;
  const double z33 = 12.0 * Qx * Qx - 3.0 * Qy * Qy;
  // P and Q keep their length in the orbit plane under the perigee rotation
  const double z1 = 6.0 * (Px * Px + Py * Py) + (2.0 * e2 + b2) * z31;
  const double z2 = 12.0 * (Px * Qx + Py * Qy) + (2.0 * e2 + b2) * z32;
  const double z3 = 6.0 * (Qx * Qx + Qy * Qy) + (2.0 * e2 + b2) * z33;
  const double z11 = Pz * (-6.0 * Pn - e2 * (24.0 * Px * cw + 6.0 * Py * sw));
  const double z13 = Qz * (-6.0 * Qn - e2 * (24.0 * Qx * cw + 6.0 * Qy * sw));
  const double z12 = -6.0 * (Pn * Qz + Qn * Pz) -
                     e2 * (24.0 * (Qx * Pz + Px * Qz) * cw + 6.0 * (Py * Qz + Qy * Pz) * sw);
  const double z21 = Pz * (6.0 * Pm + e2 * (24.0 * Px * sw - 6.0 * Py * cw));
  const double z23 = Qz * (6.0 * Qm + e2 * (24.0 * Qx * sw - 6.0 * Qy * cw));
  const double z22 = 6.0 * (Qm * Pz + Pm * Qz) +
                     e2 * (24.0 * (Qx * Pz + Px * Qz) * sw - 6.0 * (Qy * Pz + Py * Qz) * cw);

  const double s3 = cb / in.n0pp;
  const double s2 = -0.5 * s3 / beta;
  const double s4 = s3 * beta;
  const double s1 = -15.0 * e * s4;
  const double s5 = Px * Py + Qx * Qy;
  const double s6 = Qx * Py + Px * Qy;
  const double s7 = Qx * Qy - Px * Py;

  double* o = f + (int64_t)base * s + j;
  o[0 * s] = 2.0 * s1 * s6;                        // e: F2, F3
  o[1 * s] = 2.0 * s1 * s7;
  o[2 * s] = 2.0 * s2 * z12;                       // i
  o[3 * s] = 2.0 * s2 * (z13 - z11);
  o[4 * s] = -2.0 * s3 * z2;                       // M: F2, F3, sin f
  o[5 * s] = -2.0 * s3 * (z3 - z1);
  o[6 * s] = 2.0 * s3 * (21.0 + 9.0 * e2) * eb;
  o[7 * s] = 2.0 * s4 * z32;                       // perigee + cos i node
  o[8 * s] = 2.0 * s4 * (z33 - z31);
  o[9 * s] = -18.0 * s4 * eb;
  o[10 * s] = -2.0 * s2 * z22;                     // sin i node
  o[11 * s] = -2.0 * s2 * (z23 - z21);
  o[12 * s] = mb0;

  rate[0] += s1 * nb * s5;
  rate[1] += s2 * nb * (z11 + z13);
  rate[2] -= s3 * nb * (z1 + z3 - 14.0 - 6.0 * e2);
  const double gh = s4 * nb * (z31 + z33 - 6.0);
  if (near_equatorial) {
    rate[3] += gh;
  } else {
    const double node = -s2 * nb * (z21 + z23) / si;
    rate[4] += node;
    rate[3] += gh - ci * node;
  }
}

// Deep-space constants of record j (FP64 planes); returns the resonance class.
__device__ __forceinline__ int deep_record_init(const DeepIn& in, int32_t ep_day,
                                                double ep_frac, double* f, int64_t s,
                                                int64_t j) {
  using namespace deep;
  const double gsto = gmst_rad(ep_day, ep_frac);
  f[kGsto * s + j] = gsto;
  const double day = (double)(ep_day - 2415020) + ep_frac;   // from 1900 Jan 0.5

  // The Moon's orbit at the epoch: its node on the ecliptic regresses; inclination to
  // the equator cos I = cos(obl) cos(5.145 deg) - sin(obl) sin(5.145 deg) cos(node);
  // node on the equator (sin/cos hm); perigee argument from that node (gm).
  const double node_m = fmod(4.5236020 - 9.2422029e-4 * day, kTwoPi);
  double sn, cn;
  sincos(node_m, &sn, &cn);
  const double cIm = 0.91375164 - 0.03568096 * cn;
  const double sIm = sqrt(1.0 - cIm * cIm);
  const double shm = 0.089683511 * sn / sIm;
  const double chm = sqrt(1.0 - shm * shm);
  const double per_m = 5.8351514 + 0.0019443680 * day;
  const double gm =
      per_m + atan2(kSinObl * sn / sIm, chm * cn + kCosObl * shm * sn) - node_m;
  double sgm, cgm;
  sincos(gm, &sgm, &cgm);
  const double mb_moon = fmod(4.7199672 + 0.22997150 * day - per_m, kTwoPi);
  const double mb_sun = fmod(6.2565837 + 0.017201977 * day, kTwoPi);

  double sw, cw, sO, cO;
  sincos(in.argp0, &sw, &cw);
  sincos(in.raan0, &sO, &cO);
  const bool neq = in.i0 < 5.2359877e-2 || in.i0 > 3.14159265358979323846 - 5.2359877e-2;
  double rate[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // e, i, M, perigee, node
  deep_body(kCosPerSun, kSinPerSun, kCosObl, kSinObl, cO, sO, kSunN, kSunE, kSunC, mb_sun, in,
            cw, sw, neq, f, s, j, kSunE2, rate);
  deep_body(cgm, sgm, cIm, sIm, cO * chm + sO * shm, sO * chm - cO * shm, kMoonN, kMoonE, kMoonC,
            mb_moon, in, cw, sw, neq, f, s, j, kMoonE2, rate);
  f[kEdotLs * s + j] = rate[0];
  f[kIdotLs * s + j] = rate[1];
  f[kMdotLs * s + j] = rate[2];
  f[kArgpdotLs * s + j] = rate[3];
  f[kRaandotLs * s + j] = rate[4];

  const int rez = resonance_class(in.n0pp, in.e0);
  for (int k = kDel1; k <= kXfact; ++k) f[k * s + j] = 0.0;
  if (rez == 0) return 0;
  const double n = in.n0pp, e = in.e0, e2 = e * e, ci = in.cosi, si = in.sini;
  const double ainv = cbrt((n / in.xke) * (n / in.xke));      // 1 / a
  const double k2 = 3.0 * n * n * ainv * ainv;                 // 3 n^2 / a^2
  if (rez == 1) {
    // (l,m,p,q) = (3,1,1,0), (2,2,0,0), (3,3,0,0): Kaula's G_lpq(e) to e^4 and F_lmp(i)
    const double opc = 1.0 + ci;
    const double f311 = 0.9375 * si * si * (1.0 + 3.0 * ci) - 0.75 * opc;
    const double f220 = 0.75 * opc * opc;
    const double f330 = 1.875 * opc * opc * opc;
    f[kDel1 * s + j] = k2 * ainv * kQ31 * f311 * (1.0 + 2.0 * e2);
    f[kDel2 * s + j] = 2.0 * k2 * kQ22 * f220 * (1.0 + e2 * (-2.5 + 0.8125 * e2));
    f[kDel3 * s + j] = 3.0 * k2 * ainv * kQ33 * f330 * (1.0 + e2 * (-6.0 + 6.60937 * e2));
    f[kLambda0 * s + j] = fmod(in.m0 + in.raan0 + in.argp0 - gsto, kTwoPi);
    f[kXfact * s + j] = (in.mdot - n) + (in.argpdot + in.raandot - kEarthRot) + rate[2] +
                        rate[3] + rate[4];
    return 1;
  }
  // Two revolutions per day: G_lpq(e) as polynomial fits in e (e >= 0.5).
  const double e3 = e2 * e;
  const bool lo65 = e <= 0.65, lo70 = e < 0.7;
  const double g201 = -0.306 - 0.440 * (e - 0.64);
  const double g211 = lo65 ? 3.616 - 13.2470 * e + 16.2900 * e2
                           : -72.099 + 331.819 * e - 508.738 * e2 + 266.724 * e3;
  const double g310 = lo65 ? -19.302 + 117.3900 * e - 228.4190 * e2 + 156.5910 * e3
                           : -346.844 + 1582.851 * e - 2415.925 * e2 + 1246.113 * e3;
  const double g322 = lo65 ? -18.9068 + 109.7927 * e - 214.6334 * e2 + 146.5816 * e3
                           : -342.585 + 1554.908 * e - 2366.899 * e2 + 1215.972 * e3;
  const double g410 = lo65 ? -41.122 + 242.6940 * e - 471.0940 * e2 + 313.9530 * e3
                           : -1052.797 + 4758.686 * e - 7193.992 * e2 + 3651.957 * e3;
  const double g422 = lo65 ? -146.407 + 841.8800 * e - 1629.014 * e2 + 1083.4350 * e3
                           : -3581.690 + 16178.110 * e - 24462.770 * e2 + 12422.520 * e3;
  const double g520 = lo65    ? -532.114 + 3017.977 * e - 5740.032 * e2 + 3708.2760 * e3
                      : e > 0.715 ? -5149.66 + 29936.92 * e - 54087.36 * e2 + 31324.56 * e3
                                  : 1464.74 - 4664.75 * e + 3763.64 * e2;
  const double g533 = lo70 ? -919.22770 + 4988.6100 * e - 9064.7700 * e2 + 5542.21 * e3
                           : -37995.780 + 161616.52 * e - 229838.20 * e2 + 109377.94 * e3;
  const double g521 = lo70 ? -822.71072 + 4568.6173 * e - 8491.4146 * e2 + 5337.524 * e3
                           : -51752.104 + 218913.95 * e - 309468.16 * e2 + 146349.42 * e3;
  const double g532 = lo70 ? -853.66600 + 4690.2500 * e - 8624.7700 * e2 + 5341.4 * e3
                           : -40023.880 + 170470.89 * e - 242699.48 * e2 + 115605.82 * e3;
  // Kaula's F_lmp(i) of the ten terms.
  const double c2 = ci * ci, s2 = si * si;
  const double f220 = 0.75 * (1.0 + ci) * (1.0 + ci);
  const double f221 = 1.5 * s2;
  const double f321 = 1.875 * si * (1.0 - 2.0 * ci - 3.0 * c2);
  const double f322 = -1.875 * si * (1.0 + 2.0 * ci - 3.0 * c2);
  const double f441 = 35.0 * s2 * f220;
  const double f442 = 39.3750 * s2 * s2;
  const double f522 = 9.84375 * si * (s2 * (1.0 - 2.0 * ci - 5.0 * c2) +
                                      0.33333333 * (-2.0 + 4.0 * ci + 6.0 * c2));
  const double f523 = si * (4.92187512 * s2 * (-2.0 - 4.0 * ci + 10.0 * c2) +
                            6.56250012 * (1.0 + 2.0 * ci - 3.0 * c2));
  const double f542 = 29.53125 * si * (2.0 - 8.0 * ci + c2 * (-12.0 + 8.0 * ci + 10.0 * c2));
  const double f543 = 29.53125 * si * (-2.0 - 8.0 * ci + c2 * (12.0 + 8.0 * ci - 10.0 * c2));
  // dn/dt amplitude 3 n^2 (1/a)^l J_lm F G (l - 2p + q)
  const double k3 = k2 * ainv, k4 = k3 * ainv, k5 = k4 * ainv;
  f[kD2201 * s + j] = k2 * kR22 * f220 * g201;
  f[kD2211 * s + j] = k2 * kR22 * f221 * g211;
  f[kD3210 * s + j] = k3 * kR32 * f321 * g310;
  f[kD3222 * s + j] = k3 * kR32 * f322 * g322;
  f[kD4410 * s + j] = 2.0 * k4 * kR44 * f441 * g410;
  f[kD4422 * s + j] = 2.0 * k4 * kR44 * f442 * g422;
  f[kD5220 * s + j] = k5 * kR52 * f522 * g520;
  f[kD5232 * s + j] = k5 * kR52 * f523 * g532;
  f[kD5421 * s + j] = 2.0 * k5 * kR54 * f542 * g521;
  f[kD5433 * s + j] = 2.0 * k5 * kR54 * f543 * g533;
  f[kLambda0 * s + j] = fmod(in.m0 + 2.0 * (in.raan0 - gsto), kTwoPi);
  f[kXfact * s + j] = (in.mdot - n) + rate[2] + 2.0 * (in.raandot + rate[4] - kEarthRot);
  return 2;
}

// sin and cos of x - phase from those of x and of the phase.
__device__ __forceinline__ void shift(double sx, double cx, double sp, double cp, double& s,
                                      double& c) {
  s = sx * cp - cx * sp;
  c = cx * cp + sx * sp;
}

// sin and cos of the resonance terms' phases: [0, 3) the one-revolution-per-day terms'
// (phase31, 2 phase22, 3 phase33), [3, 8) the two-per-day terms' (g22 .. g54).
struct DeepPhases {
  double s[8], c[8];
};

__device__ __forceinline__ void deep_phase(int k, DeepPhases& p) {
  using namespace deep;
  const double ph[8] = {kPh31, 2.0 * kPh22, 3.0 * kPh33, kG22, kG32, kG44, kG52, kG54};
  sincos(ph[k], &p.s[k], &p.c[k]);
}

// One thread's resonance integration between states of one satellite: the last full
// step point (tc, lambda, n) of record j.  Continuing from it takes the same steps, so
// gives the same result, as starting from the epoch; like the revision's own cache it
// restarts at the epoch when t changes sign or moves back towards the epoch.
struct ResCache {
  int64_t j;
  double tc, lam, n;
  double ndot, dsum;   // the rates at that point
};

// Resonance: the resonant longitude lambda and mean motion n at t, fixed 720-min steps
// of the second-order Taylor series (dlambda/dt = n + xfact, dn/dt from the resonance
// terms, d2n/dt2 their derivative along lambda) from the epoch values or the cached step
// point, then a partial step.  The terms' sines come from one sincos of lambda (and of
// the perigee, which moves at its J2 rate in the two-per-day terms) per step and angle
// addition.  Returns false for a non-finite t or |t| > kMaxT.
__device__ __forceinline__ bool deep_resonance(const RecordPtrs& rp, int64_t j, int rez,
                                               double n0pp, double argp0, double argpdot,
                                               double t, double& n_out, double& lam_out,
                                               const DeepPhases& ph, ResCache& cache) {
  using namespace deep;
  if (!(fabs(t) <= kMaxT)) return false;
  const double* f = rp.f64;
  const int64_t s = rp.stride;
  const double xfact = __ldg(f + kXfact * s + j);
  double tc = 0.0, lam, n;
  // rates at the current step: ndot and sum of k amp cos(argument); `known`: they are
  // the cached ones of this step point
  double ndot = 0.0, dsum = 0.0;
  bool known = false;
  if (cache.j == j && cache.tc != 0.0 && t * cache.tc > 0.0 && fabs(t) >= fabs(cache.tc)) {
    tc = cache.tc;
    lam = cache.lam;
    n = cache.n;
    ndot = cache.ndot;
    dsum = cache.dsum;
    known = true;
  } else {
    lam = __ldg(f + kLambda0 * s + j);
    n = n0pp;
  }
  const double h = t > 0.0 ? kStep : -kStep;
  if (rez == 1) {
    const double d1 = __ldg(f + kDel1 * s + j), d2 = __ldg(f + kDel2 * s + j),
                 d3 = __ldg(f + kDel3 * s + j);
    for (;; known = false) {
      if (!known) {
        double s1, c1;
        sincos(lam, &s1, &c1);
        const double s2 = 2.0 * s1 * c1, c2 = c1 * c1 - s1 * s1;
        const double s3 = s2 * c1 + c2 * s1, c3 = c2 * c1 - s2 * s1;
        double a, b, x, y, u, w;
        shift(s1, c1, ph.s[0], ph.c[0], a, b);
        shift(s2, c2, ph.s[1], ph.c[1], x, y);
        shift(s3, c3, ph.s[2], ph.c[2], u, w);
        ndot = d1 * a + d2 * x + d3 * u;
        dsum = d1 * b + 2.0 * d2 * y + 3.0 * d3 * w;
      }
      const double ldot = n + xfact;
      if (!(fabs(t - tc) >= kStep)) {
        cache = ResCache{j, tc, lam, n, ndot, dsum};
        const double ft = t - tc;
        n_out = n + ndot * ft + dsum * ldot * (0.5 * ft * ft);
        lam_out = lam + ldot * ft + ndot * (0.5 * ft * ft);
        return true;
      }
      lam += ldot * h + ndot * (0.5 * h * h);
      n += ndot * h + dsum * ldot * (0.5 * h * h);
      tc += h;
    }
  }
  const double* d = f + kD2201 * s + j;   // ten planes kD2201 .. kD5433
  const double s22 = ph.s[3], c22 = ph.c[3], s32 = ph.s[4], c32 = ph.c[4];
  const double s44 = ph.s[5], c44 = ph.c[5], s52 = ph.s[6], c52 = ph.c[6];
  const double s54 = ph.s[7], c54 = ph.c[7];
  for (;; known = false) {
    const double ldot = n + xfact;
    if (!known) {
      double sl, cl, sw, cw;
      sincos(lam, &sl, &cl);
      sincos(argp0 + argpdot * tc, &sw, &cw);
      const double sl2 = 2.0 * sl * cl, cl2 = cl * cl - sl * sl;
      const double sw2 = 2.0 * sw * cw, cw2 = cw * cw - sw * sw;
      // sin, cos of lambda + w, lambda - w, lambda + 2w, 2 lambda + w, 2 lambda - w,
      // 2 lambda + 2 w
      const double slpw = sl * cw + cl * sw, clpw = cl * cw - sl * sw;
      const double slmw = sl * cw - cl * sw, clmw = cl * cw + sl * sw;
      const double slp2w = sl * cw2 + cl * sw2, clp2w = cl * cw2 - sl * sw2;
      const double s2lpw = sl2 * cw + cl2 * sw, c2lpw = cl2 * cw - sl2 * sw;
      const double s2lmw = sl2 * cw - cl2 * sw, c2lmw = cl2 * cw + sl2 * sw;
      const double s2lp2w = sl2 * cw2 + cl2 * sw2, c2lp2w = cl2 * cw2 - sl2 * sw2;
      double a, b;
      ndot = 0.0;
      dsum = 0.0;
      auto add = [&](int k, double sx, double cx, double sp, double cp, double weight) {
        shift(sx, cx, sp, cp, a, b);
        const double amp = __ldg(d + (int64_t)k * s);
        ndot = fma(amp, a, ndot);
        dsum = fma(amp * weight, b, dsum);
      };
      add(0, slp2w, clp2w, s22, c22, 1.0);     // 2w + lambda  (2,2,0,-1)
      add(1, sl, cl, s22, c22, 1.0);           // lambda       (2,2,1,1)
      add(2, slpw, clpw, s32, c32, 1.0);       // w + lambda   (3,2,1,0)
      add(3, slmw, clmw, s32, c32, 1.0);       // lambda - w   (3,2,2,2)
      add(4, s2lp2w, c2lp2w, s44, c44, 2.0);   // 2w + 2lambda (4,4,1,0)
      add(5, sl2, cl2, s44, c44, 2.0);         // 2 lambda     (4,4,2,2)
      add(6, slpw, clpw, s52, c52, 1.0);       // w + lambda   (5,2,2,0)
      add(7, slmw, clmw, s52, c52, 1.0);       // lambda - w   (5,2,3,2)
      add(8, s2lpw, c2lpw, s54, c54, 2.0);     // w + 2 lambda (5,4,2,1)
      add(9, s2lmw, c2lmw, s54, c54, 2.0);     // 2 lambda - w (5,4,3,3)
    }
    if (!(fabs(t - tc) >= kStep)) {
      cache = ResCache{j, tc, lam, n, ndot, dsum};
      const double ft = t - tc;
      n_out = n + ndot * ft + dsum * ldot * (0.5 * ft * ft);
      lam_out = lam + ldot * ft + ndot * (0.5 * ft * ft);
      return true;
    }
    lam += ldot * h + ndot * (0.5 * h * h);
    n += ndot * h + dsum * ldot * (0.5 * h * h);
    tc += h;
  }
}

// The Sun's and Moon's long-period terms at t added to (e, i, node, perigee, M): above
// 0.2 rad of perturbed inclination directly, below through the orbit normal's
// components (Lyddane), the node kept on the branch nearest its mean value.
__device__ __forceinline__ void deep_periodics(const RecordPtrs& rp, int64_t j, double t,
                                               double& e, double& inc, double& raan,
                                               double& argp, double& M) {
  using namespace deep;
  const double* f = rp.f64;
  const int64_t s = rp.stride;
  double pe = 0.0, pi = 0.0, pl = 0.0, pgh = 0.0, ph = 0.0;
  for (int b = 0; b < 2; ++b) {
    const double* o = f + (int64_t)(b ? kMoonE2 : kSunE2) * s + j;
    // true anomaly f = M + d, d = 2 e sin M (|d| <= 0.11): sin f, cos f by rotating
    // (sin M, cos M) by d, whose sine and cosine are Taylor series to d^11 and d^12
    // (truncation below 1e-22)
    const double mb = __ldg(o + 12 * s) + (b ? kMoonN : kSunN) * t;
    double sm, cm;
    sincos(mb, &sm, &cm);
    const double d = 2.0 * (b ? kMoonE : kSunE) * sm, d2 = d * d;
    const double sd =
        d * (1.0 - d2 * (1.0 / 6.0) * (1.0 - d2 * (1.0 / 20.0) * (1.0 - d2 * (1.0 / 42.0) *
             (1.0 - d2 * (1.0 / 72.0) * (1.0 - d2 * (1.0 / 110.0))))));
    const double cd =
        1.0 - d2 * 0.5 * (1.0 - d2 * (1.0 / 12.0) * (1.0 - d2 * (1.0 / 30.0) *
              (1.0 - d2 * (1.0 / 56.0) * (1.0 - d2 * (1.0 / 90.0) * (1.0 - d2 * (1.0 / 132.0))))));
    const double sf = sm * cd + cm * sd;
    const double cf = cm * cd - sm * sd;
    const double F2 = 0.5 * sf * sf - 0.25;
    const double F3 = -0.5 * sf * cf;
    pe += __ldg(o + 0 * s) * F2 + __ldg(o + 1 * s) * F3;
    pi += __ldg(o + 2 * s) * F2 + __ldg(o + 3 * s) * F3;
    pl += __ldg(o + 4 * s) * F2 + __ldg(o + 5 * s) * F3 + __ldg(o + 6 * s) * sf;
    pgh += __ldg(o + 7 * s) * F2 + __ldg(o + 8 * s) * F3 + __ldg(o + 9 * s) * sf;
    ph += __ldg(o + 10 * s) * F2 + __ldg(o + 11 * s) * F3;
  }
  inc += pi;
  e += pe;
  double si, ci;
  sincos(inc, &si, &ci);
  if (inc >= 0.2) {
    const double dnode = ph / si;
    argp += pgh - ci * dnode;
    raan += dnode;
    M += pl;
    return;
  }
  double so, co;
  sincos(raan, &so, &co);
  const double alpha = si * so + (ph * co + pi * ci * so);
  const double beta = si * co + (pi * ci * co - ph * so);
  raan = wrap_2pi(raan);
  const double L = M + argp + ci * raan + (pl + pgh - pi * raan * si);
  const double mean_node = raan;
  raan = atan2(alpha, beta);
  if (fabs(mean_node - raan) > 3.14159265358979323846)
    raan += raan < mean_node ? kTwoPi : -kTwoPi;
  M += pl;
  argp = L - M - ci * raan;
}

// One deep-space state in FP64 (record rc of row j): secular gravity and the truncated
// drag, the lunar-solar secular rates, the resonance, the lunar-solar periodics, then
// the near-Earth long- and short-period terms at the perturbed inclination.
#ifndef SGP4_DEEP_INLINE
#define SGP4_DEEP_INLINE __noinline__
#endif
static __device__ SGP4_DEEP_INLINE int state64_deep(const RecordPtrs rp, int64_t j, const Geo g,
                                             double t, double* r, double* v,
                                             const DeepPhases* ph, ResCache* cache) {
  const Rec64 rc = load_rec64(rp, j);
  const double* f = rp.f64;
  const int64_t s = rp.stride;
  double M = rc.m0 + rc.mdot * t;
  double argp = rc.argp0 + rc.argpdot * t;
  double raan = rc.raan0 + rc.raandot * t + rc.raan_cf * t * t;
  const double tempa = 1.0 - rc.c1 * t;
  const double tempe = rc.bc4 * t;
  const double templ = rc.l2 * t * t;
  double e = rc.e0 + __ldg(f + kEdotLs * s + j) * t;
  double inc = rc.i0 + __ldg(f + kIdotLs * s + j) * t;
  argp += __ldg(f + kArgpdotLs * s + j) * t;
  raan += __ldg(f + kRaandotLs * s + j) * t;
  M += __ldg(f + kMdotLs * s + j) * t;
  double n = rc.n0pp;
  const int rez = (rc.flags & kFlagRez1) ? 1 : (rc.flags & kFlagRez2) ? 2 : 0;
  if (rez) {
    double lam;
    if (!deep_resonance(rp, j, rez, rc.n0pp, rc.argp0, rc.argpdot, t, n, lam, *ph, *cache))
      return 2;
    const double theta = wrap_2pi(__ldg(f + kGsto * s + j) + t * deep::kEarthRot);
    M = rez == 1 ? lam - raan - argp + theta : lam - 2.0 * raan + 2.0 * theta;
  }
  if (n <= 0.0) return 2;
  const double a = cbrt((g.xke / n) * (g.xke / n)) * tempa * tempa;
  e -= tempe;
  if (e >= 1.0 || e < -0.001) return 1;
  if (e < 1.0e-6) e = 1.0e-6;
  M += rc.n0pp * templ;
  // mean angles reduced as in the near-Earth theory (the sign kept; wrap_2pi equals C
  // fmod to rounding without its iterative remainder)
  const double L = wrap_2pi(M + argp + raan);
  raan = wrap_2pi(raan);
  argp = wrap_2pi(argp);
  M = wrap_2pi(L - argp - raan);

  deep_periodics(rp, j, t, e, inc, raan, argp, M);
  if (inc < 0.0) {
    inc = -inc;
    raan += 3.14159265358979323846;
    argp -= 3.14159265358979323846;
  }
  if (e < 0.0 || e > 1.0) return 3;
  double si, ci;
  sincos(inc, &si, &ci);
  const double c2 = ci * ci;
  double opc = 1.0 + ci;
  if (fabs(opc) <= 1.5e-12) opc = 1.5e-12;
  const double xlcof = -0.25 * g.j3oj2 * si * (3.0 + 5.0 * ci) / opc;
  const double aycof = -0.5 * g.j3oj2 * si;
  double rr[3], vv[3];
  const int code = state64_tail(g, a, e, raan, argp, M + argp, xlcof, aycof, ci, si,
                                3.0 * c2 - 1.0, 1.0 - c2, 7.0 * c2 - 1.0, rr, vv);
  for (int c = 0; c < 3; ++c) {
    r[c] = rr[c];
    v[c] = vv[c];
  }
  return code;
}

// Any record in FP64: the deep-space state for deep-space records (phases computed
// here, no cache), else state64.
__device__ __forceinline__ int state64_any(const RecordPtrs& rp, int64_t j, const Rec64& rc,
                                           const Geo& g, double t, double r[3], double v[3]) {
  if (rc.flags & kFlagDeep) {
    DeepPhases ph;
    for (int k = 0; k < 8; ++k) deep_phase(k, ph);
    ResCache cache{-1, 0.0, 0.0, 0.0};
    return state64_deep(rp, j, g, t, r, v, &ph, &cache);
  }
  return state64(rc, g, t, r, v);
}

// Out-of-line FP64 recomputation of one guard-band (or deep-space) state: the record
// build's status at t = 0.
static __device__ __noinline__ int state64_fallback(RecordPtrs rp, Geo g, int64_t j, double t,
                                                    float r[3], float v[3]) {
  const Rec64 rc = load_rec64(rp, j);
  double r64[3], v64[3];
  const int code = state64_any(rp, j, rc, g, t, r64, v64);
  for (int c = 0; c < 3; ++c) {
    r[c] = (float)r64[c];
    v[c] = (float)v64[c];
  }
  return code;
}

}  // namespace sgp4
