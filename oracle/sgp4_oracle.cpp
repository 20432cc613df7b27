// SGP4 oracle (near-Earth and deep-space branches): TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, FP64 CPU restatement of the near-Earth SGP4 theory that the paper
// (Priestley & Handley, "jaxsgp4", Sec. 2.1) says it implements: the equations of
// Hoots & Roehrich, Spacetrack Report #3 (1980) as revised by Hoots et al. (2004) and
// Vallado et al. (AIAA 2006-6753), with the WGS-72 geopotential constants.
// Symbols follow Spacetrack Report #3: n0'' (un-Kozai'd mean motion), a0'', xi, eta,
// beta0, C1..C5, D2..D4, a_xN, a_yN, U, psi (= E + omega), e_L, p_L, r_k, u_k, ...
//
// Only tests, the smoke check and the CPU-baseline leg of the benchmark may load this
// library.  The GPU path shares no code, header or constant with it.
//
// The whole algorithm is written once, templated on the scalar type R: R = double
// gives the reference values, R = Dual (value + 7 partials) gives forward-mode
// derivatives with respect to (n0, e0, i0, RAAN0, argp0, M0, B*).  No blocking,
// fusion or reordering beyond the steps of the theory; every branch of the theory
// is an ordinary `if` on the value.
//
// Orbits with a period of 225 min or more take the deep-space branch of the same
// revision (SDP4: the report's deep-space section): lunar and solar perturbations
// and, near the one- and two-revolution-per-day commensurabilities, tesseral
// resonance.  The paper names this branch as future work (Sec. 6, 7); it is written
// here from the theory, in the same order.
//
// Readings of points the paper leaves open (the CUDA path takes the same ones):
//  * WGS-72 with ke computed from mu and the Earth radius (not the rounded
//    "WGS72old" ke literal).
//  * a0'' = (ke / n0'')^(2/3) (2006 revision), not a0/(1 - delta0) (1980 report).
//  * D4 carries a0''^2 (the dimensionally consistent form).
//  * Input validity (paper Sec. 2.2, "Control Flow": error codes instead of exits):
//    non-finite input or e0 outside [0,1) -> code 1, n0 <= 0 -> code 2, fatal for
//    the record.  Otherwise the init status is the status of the state at t = 0.
//  * Status precedence: first failing check in step order: 2, 1, 4, 6.  Codes
//    1, 2, 4 give r = v = NaN; code 6 (r_k < 1 Earth radius) keeps r, v.
//  * Kepler: Newton with the step clamped to +-0.95, stop when |dpsi| < 1e-12 or
//    after 10 steps; sin/cos are then taken at the final iterate.
//  * Angles reduced with C fmod (sign kept).
//  * Deep space: the "improved" operation mode of the 2006 revision (Greenwich
//    sidereal time at epoch from the IAU-82 formula, no wrap of the node into
//    [0, 2 pi) inside the Lyddane branch); the epoch is the record's own split
//    Julian date (epoch 0 when none is given); the lunar-solar periodic terms are
//    applied absolutely (their value at the epoch is not subtracted); the status
//    after the lunar-solar periodic terms is code 3 (e outside [0, 1]), checked
//    between codes 1 and 4.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>
#include <algorithm>

namespace oracle {

static const double kPi = 3.14159265358979323846;
static const double kTwoPi = 2.0 * kPi;

// ---------------------------------------------------------------- scalar types
// Forward-mode dual number with 7 tangent directions (the 7 mean elements).
struct Dual {
  double v;
  double d[7];
  Dual() : v(0.0) { for (double& x : d) x = 0.0; }
  Dual(double x) : v(x) { for (double& y : d) y = 0.0; }  // NOLINT: implicit constant
};

inline Dual make_var(double x, int k) { Dual r(x); r.d[k] = 1.0; return r; }
inline Dual chain(const Dual& a, double val, double dfda) {
  Dual r(val);
  for (int k = 0; k < 7; ++k) r.d[k] = dfda * a.d[k];
  return r;
}
inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r(a.v + b.v); for (int k = 0; k < 7; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r(a.v - b.v); for (int k = 0; k < 7; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
inline Dual operator-(const Dual& a) {
  Dual r(-a.v); for (int k = 0; k < 7; ++k) r.d[k] = -a.d[k]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r(a.v * b.v); for (int k = 0; k < 7; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v);
  for (int k = 0; k < 7; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
  return r;
}
inline Dual operator+(const Dual& a, double b) { return a + Dual(b); }
inline Dual operator+(double a, const Dual& b) { return Dual(a) + b; }
inline Dual operator-(const Dual& a, double b) { return a - Dual(b); }
inline Dual operator-(double a, const Dual& b) { return Dual(a) - b; }
inline Dual operator*(const Dual& a, double b) { return a * Dual(b); }
inline Dual operator*(double a, const Dual& b) { return Dual(a) * b; }
inline Dual operator/(const Dual& a, double b) { return a / Dual(b); }
inline Dual operator/(double a, const Dual& b) { return Dual(a) / b; }
inline bool operator<(const Dual& a, double b) { return a.v < b; }
inline bool operator>(const Dual& a, double b) { return a.v > b; }
inline bool operator<=(const Dual& a, double b) { return a.v <= b; }
inline bool operator>=(const Dual& a, double b) { return a.v >= b; }
inline Dual sin(const Dual& a) { return chain(a, std::sin(a.v), std::cos(a.v)); }
inline Dual cos(const Dual& a) { return chain(a, std::cos(a.v), -std::sin(a.v)); }
inline Dual sqrt(const Dual& a) { double s = std::sqrt(a.v); return chain(a, s, 0.5 / s); }
inline Dual pow(const Dual& a, double p) {
  return chain(a, std::pow(a.v, p), p * std::pow(a.v, p - 1.0)); }
inline Dual fabs(const Dual& a) { return a.v < 0.0 ? -a : a; }
inline Dual atan2(const Dual& y, const Dual& x) {
  Dual r(std::atan2(y.v, x.v));
  double den = x.v * x.v + y.v * y.v;
  for (int k = 0; k < 7; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) / den;
  return r;
}
// fmod by a constant: subtracting an integer multiple of c leaves derivatives unchanged.
inline Dual fmod(const Dual& a, double c) {
  Dual r = a; r.v = std::fmod(a.v, c); return r; }
inline double val(const Dual& a) { return a.v; }
inline double val(double a) { return a; }
inline bool finite_val(const Dual& a) { return std::isfinite(a.v); }
inline bool finite_val(double a) { return std::isfinite(a); }

using std::sin; using std::cos; using std::sqrt; using std::pow; using std::fabs;
using std::atan2; using std::fmod;

// ------------------------------------------------------------- geopotential
// Earth model (paper Sec. 2.1: WGS-72).  The tests zero J2..J4 for the two-body
// closed forms, so J3/J2 is defined as 0 when J2 == 0.
struct Geo {
  double mu;        // km^3/s^2
  double re;        // Earth equatorial radius, km
  double j2, j3, j4;
  double xke;       // sqrt(mu) in Earth radii^1.5 per minute
  double j3oj2;
};

inline Geo make_geo(const double c[5]) {
  Geo g;
  g.mu = c[0]; g.re = c[1]; g.j2 = c[2]; g.j3 = c[3]; g.j4 = c[4];
  g.xke = 60.0 / std::sqrt(g.re * g.re * g.re / g.mu);
  g.j3oj2 = (g.j2 != 0.0) ? g.j3 / g.j2 : 0.0;
  return g;
}

// ------------------------------------------------- deep-space theory constants
// Lunar-solar part (quadrupole tide of each body; report's deep-space section).  The
// tests may switch a body off (c = 0), make its orbit circular (e = 0) or scale the
// resonance amplitudes; the values below are the theory's.
struct DeepConsts {
  double n_sun, e_sun, c_sun;     // Sun: mean motion (rad/min), eccentricity, tide coefficient
  double n_moon, e_moon, c_moon;  // Moon: the same
  double res_scale;               // factor on every tesseral resonance amplitude
};

inline DeepConsts make_deep(const double* d) {
  DeepConsts c;
  c.n_sun = 1.19459e-5;   c.e_sun = 0.01675; c.c_sun = 2.9864797e-6;
  c.n_moon = 1.5835218e-4; c.e_moon = 0.05490; c.c_moon = 4.7968065e-7;
  c.res_scale = 1.0;
  if (d) {
    c.n_sun = d[0]; c.e_sun = d[1]; c.c_sun = d[2];
    c.n_moon = d[3]; c.e_moon = d[4]; c.c_moon = d[5]; c.res_scale = d[6];
  }
  return c;
}

// Orientation of the Sun's apparent orbit: sin and cos of the obliquity of the
// ecliptic, cos and sin of the argument of the Sun's perigee.
static const double kSinObl = 0.39785416, kCosObl = 0.91744867;
static const double kCosPerSun = 0.1945905, kSinPerSun = -0.98088458;
// Earth's rotation rate (rad/min).
static const double kEarthRot = 4.37526908801129966e-3;
// Tesseral harmonics in the resonance terms (Earth radii = 1): amplitudes of the
// (l, m) = (2,2), (3,1), (3,3) terms for one revolution per day and their phases
// (the resonant argument k lambda minus k times the phase, k = 1, 2, 3) ...
static const double kQ22 = 1.7891679e-6, kQ31 = 2.1460748e-6, kQ33 = 2.2123015e-7;
static const double kPhase31 = 0.13130908, kPhase22 = 2.8843198, kPhase33 = 0.37448087;
// ... and of the (2,2), (3,2), (4,4), (5,2), (5,4) terms for two revolutions per day,
// with the phase of each argument.
static const double kR22 = 1.7891679e-6, kR32 = 3.7393792e-7, kR44 = 7.3636953e-9;
static const double kR52 = 1.1428639e-7, kR54 = 2.1765803e-9;
static const double kG22 = 5.7686396, kG32 = 0.95240898, kG44 = 1.8014998;
static const double kG52 = 1.0508330, kG54 = 4.4108898;
// Resonance integrator: fixed step (min).
static const double kResStep = 720.0;

// Greenwich mean sidereal angle (rad, [0, 2 pi)) at the Julian date day + frac
// (IAU 1982 polynomial in Julian centuries from J2000, in seconds of time).
inline double gmst82(double day, double frac) {
  double T = ((day - 2451545.0) + frac) / 36525.0;
  double sec = 67310.54841 + (876600.0 * 3600.0 + 8640184.812866) * T + 0.093104 * T * T -
               6.2e-6 * T * T * T;
  double th = std::fmod(sec * (kTwoPi / 86400.0), kTwoPi);
  if (th < 0.0) th += kTwoPi;
  return th;
}

// Lunar-solar long-period terms of one body: amplitudes of the terms in
// F2 = sin^2 f / 2 - 1/4, F3 = -sin f cos f / 2 and sin f (f the body's true anomaly)
// in the eccentricity (e), inclination (i), mean anomaly (l), perigee + cos i node
// (gh) and sin i node (h); the body's mean motion, eccentricity and mean anomaly at
// the epoch.
template <class R>
struct LunarSolar {
  R e2, e3, i2, i3, l2, l3, l4, gh2, gh3, gh4, h2, h3;
  double n, ecc, M0;
};

// ---------------------------------------------------------- per-satellite record
// Constants of motion from the mean elements (Spacetrack Report #3, "initialization").
template <class R>
struct Rec {
  R n0, e0, i0, raan0, argp0, m0, bstar;   // mean elements (n0 Kozai, rad/min; angles rad)
  R n0pp, a0pp;                             // un-Kozai'd mean motion (rad/min), semi-major axis (ER)
  R cosi, sini, x3thm1, x1mth2, x7thm1;     // theta = cos i0 and its polynomials
  R beta0;                                  // sqrt(1 - e0^2)
  R s, xi, eta;                             // drag: s (ER), xi = 1/(a0''-s), eta = a0'' e0 xi
  R C1, C3, C4, C5, D2, D3, D4;
  R Mdot, argpdot, raandot;                 // secular rates (rad/min)
  R raan_cf, argp_cf, m_cf;                 // drag coefficients of Omega t^2, omega t and delta M
  R L2, L3, L4, L5;                         // mean-longitude polynomial coefficients
  R xlcof, aycof;                           // long-period J3 coefficients
  R delM0, sinM0;                           // (1 + eta cos M0)^3 and sin M0
  bool isimp;                               // perigee below 220 km: truncated drag
  int fatal;                                // 0, or 1/2 if the input elements are unusable
  // Deep space (period >= 225 min).
  bool deep;
  int irez;                                 // 0 none, 1 one rev/day, 2 two rev/day resonance
  double gsto;                              // Greenwich sidereal angle at epoch (rad)
  LunarSolar<R> sun, moon;                  // long-period coefficients of each body
  R edot, idot, mdot_ls, argpdot_ls, raandot_ls;   // lunar-solar secular rates (per min)
  R del1, del2, del3;                       // one-rev/day resonance amplitudes (rad/min^2)
  R d2201, d2211, d3210, d3222, d4410, d4422, d5220, d5232, d5421, d5433;  // two-rev/day
  R lambda0, xfact;                         // resonant longitude at epoch, its rate minus n
};

// ------------------------------------------------- deep space: initialisation
// Quadrupole tide of one body (Sun or Moon) on the satellite's epoch orbit.  The body
// moves on a fixed ellipse whose plane has inclination (cI, sI) to the equator, whose
// perigee lies at the angle (cg, sg) from that plane's ascending node on the equator,
// and whose node lies at the angle (ch, sh) behind the satellite's node.  a1..a6 are
// the components of the body's perigee direction P (odd) and of the in-plane normal Q
// (even) along the satellite's node line, the in-plane normal to it and the orbit
// normal; x1..x8 the same on the satellite's perigee axes.  The satellite's orbit is
// (e, n, i, w) at the epoch.  Returns the body's long-period coefficients and adds its
// secular rates to rc (the node terms are dropped within 3 deg of the equatorial
// planes, where the node is undefined).
template <class R>
LunarSolar<R> tide_terms(double cg, double sg, double cI, double sI, const R& ch, const R& sh,
                         double nb, double eb, double cb, double M0b, Rec<R>& rc,
                         const R& cosw, const R& sinw) {
  const R& ci = rc.cosi;
  const R& si = rc.sini;
  R a1 = cg * ch + sg * cI * sh;
  R a3 = -sg * ch + cg * cI * sh;
  R a7 = -cg * sh + sg * cI * ch;
  double a8 = sg * sI;
  R a9 = sg * sh + cg * cI * ch;
  double a10 = cg * sI;
  R a2 = ci * a7 + si * a8;
  R a4 = ci * a9 + si * a10;
  R a5 = -si * a7 + ci * a8;
  R a6 = -si * a9 + ci * a10;
  R x1 = a1 * cosw + a2 * sinw;
  R x2 = a3 * cosw + a4 * sinw;
  R x3 = -a1 * sinw + a2 * cosw;
  R x4 = -a3 * sinw + a4 * cosw;
  R x5 = a5 * sinw, x6 = a6 * sinw, x7 = a5 * cosw, x8 = a6 * cosw;

  R e = rc.e0;
  R e2 = e * e;
  R b2 = 1.0 - e2;
  R beta = sqrt(b2);
  R z31 = 12.0 * x1 * x1 - 3.0 * x3 * x3;
  R z32 = 24.0 * x1 * x2 - 6.0 * x3 * x4;
  R z33 = 12.0 * x2 * x2 - 3.0 * x4 * x4;
  R z1 = 2.0 * (3.0 * (a1 * a1 + a2 * a2) + z31 * e2) + b2 * z31;
  R z2 = 2.0 * (6.0 * (a1 * a3 + a2 * a4) + z32 * e2) + b2 * z32;
  R z3 = 2.0 * (3.0 * (a3 * a3 + a4 * a4) + z33 * e2) + b2 * z33;
  R z11 = -6.0 * a1 * a5 + e2 * (-24.0 * x1 * x7 - 6.0 * x3 * x5);
  R z12 = -6.0 * (a1 * a6 + a3 * a5) + e2 * (-24.0 * (x2 * x7 + x1 * x8) - 6.0 * (x3 * x6 + x4 * x5));
  R z13 = -6.0 * a3 * a6 + e2 * (-24.0 * x2 * x8 - 6.0 * x4 * x6);
  R z21 = 6.0 * a2 * a5 + e2 * (24.0 * x1 * x5 - 6.0 * x3 * x7);
  R z22 = 6.0 * (a4 * a5 + a2 * a6) + e2 * (24.0 * (x2 * x5 + x1 * x6) - 6.0 * (x4 * x7 + x3 * x8));
  R z23 = 6.0 * a4 * a6 + e2 * (24.0 * x2 * x6 - 6.0 * x4 * x8);

  R s3 = cb / rc.n0pp;
  R s2 = -0.5 * s3 / beta;
  R s4 = s3 * beta;
  R s1 = -15.0 * e * s4;
  R s5 = x1 * x3 + x2 * x4;
  R s6 = x2 * x3 + x1 * x4;
  R s7 = x2 * x4 - x1 * x3;

  LunarSolar<R> L;
  L.e2 = 2.0 * s1 * s6;
  L.e3 = 2.0 * s1 * s7;
  L.i2 = 2.0 * s2 * z12;
  L.i3 = 2.0 * s2 * (z13 - z11);
  L.l2 = -2.0 * s3 * z2;
  L.l3 = -2.0 * s3 * (z3 - z1);
  L.l4 = -2.0 * s3 * (-21.0 - 9.0 * e2) * eb;
  L.gh2 = 2.0 * s4 * z32;
  L.gh3 = 2.0 * s4 * (z33 - z31);
  L.gh4 = -18.0 * s4 * eb;
  L.h2 = -2.0 * s2 * z22;
  L.h3 = -2.0 * s2 * (z23 - z21);
  L.n = nb; L.ecc = eb; L.M0 = M0b;

  rc.edot = rc.edot + s1 * nb * s5;
  rc.idot = rc.idot + s2 * nb * (z11 + z13);
  rc.mdot_ls = rc.mdot_ls - nb * s3 * (z1 + z3 - 14.0 - 6.0 * e2);
  R gh = s4 * nb * (z31 + z33 - 6.0);
  bool near_equatorial = rc.i0 < 5.2359877e-2 || rc.i0 > kPi - 5.2359877e-2;
  if (near_equatorial) {
    rc.argpdot_ls = rc.argpdot_ls + gh;
  } else {
    R h = -nb * s2 * (z21 + z23) / si;   // node rate
    rc.raandot_ls = rc.raandot_ls + h;
    rc.argpdot_ls = rc.argpdot_ls + gh - ci * h;
  }
  return L;
}

// Deep-space constants of a record: Greenwich sidereal angle at the epoch, the
// Sun's and Moon's positions at the epoch, their tides, and the resonance terms.
// Needs n0'', the J2 secular rates and cos/sin i0 of the near-Earth initialisation.
template <class R>
void deep_init(const Geo& g, const DeepConsts& dc, double ep_day, double ep_frac, Rec<R>& rc) {
  rc.gsto = gmst82(ep_day, ep_frac);
  // Days from 1900 Jan 0.5 (JD 2415020.0).
  double day = (ep_day - 2415020.0) + ep_frac;

  // The Moon's orbit at the epoch: its ascending node on the ecliptic regresses; its
  // inclination to the equator follows from the obliquity and the 5.145 deg lunar
  // inclination (cos I = cos(obl) cos(i_M) - sin(obl) sin(i_M) cos node); its node on
  // the equator (sin/cos hm) and the argument of its perigee from that node.
  double node_m = std::fmod(4.5236020 - 9.2422029e-4 * day, kTwoPi);
  double stem = std::sin(node_m), ctem = std::cos(node_m);
  double cIm = 0.91375164 - 0.03568096 * ctem;
  double sIm = std::sqrt(1.0 - cIm * cIm);
  double shm = 0.089683511 * stem / sIm;
  double chm = std::sqrt(1.0 - shm * shm);
  double per_m = 5.8351514 + 0.0019443680 * day;      // longitude of the lunar perigee
  double arc = std::atan2(kSinObl * stem / sIm, chm * ctem + kCosObl * shm * stem);
  double gm = per_m + arc - node_m;
  double M0_moon = std::fmod(4.7199672 + 0.22997150 * day - per_m, kTwoPi);
  double M0_sun = std::fmod(6.2565837 + 0.017201977 * day, kTwoPi);

  rc.edot = R(0.0); rc.idot = R(0.0); rc.mdot_ls = R(0.0);
  rc.argpdot_ls = R(0.0); rc.raandot_ls = R(0.0);
  R cw = cos(rc.argp0), sw = sin(rc.argp0);
  R cO = cos(rc.raan0), sO = sin(rc.raan0);
  rc.sun = tide_terms(kCosPerSun, kSinPerSun, kCosObl, kSinObl, cO, sO, dc.n_sun, dc.e_sun,
                      dc.c_sun, M0_sun, rc, cw, sw);
  rc.moon = tide_terms(std::cos(gm), std::sin(gm), cIm, sIm, cO * chm + sO * shm,
                       sO * chm - cO * shm, dc.n_moon, dc.e_moon, dc.c_moon, M0_moon, rc, cw, sw);

  // Tesseral resonance: periods of 1200-1800 min (one revolution per day), or
  // 680-760 min with e >= 0.5 (two per day).
  rc.irez = 0;
  if (rc.n0pp < 0.0052359877 && rc.n0pp > 0.0034906585) rc.irez = 1;
  if (rc.n0pp >= 8.26e-3 && rc.n0pp <= 9.24e-3 && rc.e0 >= 0.5) rc.irez = 2;
  rc.del1 = R(0.0); rc.del2 = R(0.0); rc.del3 = R(0.0);
  rc.d2201 = R(0.0); rc.d2211 = R(0.0); rc.d3210 = R(0.0); rc.d3222 = R(0.0);
  rc.d4410 = R(0.0); rc.d4422 = R(0.0); rc.d5220 = R(0.0); rc.d5232 = R(0.0);
  rc.d5421 = R(0.0); rc.d5433 = R(0.0);
  rc.lambda0 = R(0.0); rc.xfact = R(0.0);
  if (rc.irez == 0) return;

  const R& n = rc.n0pp;
  const R& e = rc.e0;
  const R& ci = rc.cosi;
  const R& si = rc.sini;
  R e2 = e * e;
  R aonv = pow(n / g.xke, 2.0 / 3.0);     // 1 / a (Earth radii)
  // 3 n^2 / a^2: the factor of every dn/dt amplitude (times (1/a)^(l-2) below)
  R k = 3.0 * n * n * aonv * aonv * dc.res_scale;
  if (rc.irez == 1) {
    // Eccentricity functions G_lpq(e) and inclination functions F_lmp(i) of the
    // (l,m,p,q) = (3,1,1,0), (2,2,0,0), (3,3,0,0) terms.
    R g200 = 1.0 + e2 * (-2.5 + 0.8125 * e2);
    R g310 = 1.0 + 2.0 * e2;
    R g300 = 1.0 + e2 * (-6.0 + 6.60937 * e2);
    R opc = 1.0 + ci;
    R f220 = 0.75 * opc * opc;
    R f311 = 0.9375 * si * si * (1.0 + 3.0 * ci) - 0.75 * opc;
    R f330 = 1.875 * opc * opc * opc;
    rc.del1 = k * f311 * g310 * kQ31 * aonv;
    rc.del2 = 2.0 * k * f220 * g200 * kQ22;
    rc.del3 = 3.0 * k * f330 * g300 * kQ33 * aonv;
    rc.lambda0 = fmod(rc.m0 + rc.raan0 + rc.argp0 - rc.gsto, kTwoPi);
    rc.xfact = rc.Mdot + rc.argpdot + rc.raandot - kEarthRot + rc.mdot_ls + rc.argpdot_ls +
               rc.raandot_ls - rc.n0pp;
    return;
  }
  // Two revolutions per day: G_lpq(e) as fitted polynomials in e (they hold for the
  // e >= 0.5 of this class) ...
  R e3 = e2 * e;
  R g201 = -0.306 - (e - 0.64) * 0.440;
  R g211, g310, g322, g410, g422, g520, g521, g532, g533;
  if (e <= 0.65) {
    g211 = 3.616 - 13.2470 * e + 16.2900 * e2;
    g310 = -19.302 + 117.3900 * e - 228.4190 * e2 + 156.5910 * e3;
    g322 = -18.9068 + 109.7927 * e - 214.6334 * e2 + 146.5816 * e3;
    g410 = -41.122 + 242.6940 * e - 471.0940 * e2 + 313.9530 * e3;
    g422 = -146.407 + 841.8800 * e - 1629.014 * e2 + 1083.4350 * e3;
    g520 = -532.114 + 3017.977 * e - 5740.032 * e2 + 3708.2760 * e3;
  } else {
    g211 = -72.099 + 331.819 * e - 508.738 * e2 + 266.724 * e3;
    g310 = -346.844 + 1582.851 * e - 2415.925 * e2 + 1246.113 * e3;
    g322 = -342.585 + 1554.908 * e - 2366.899 * e2 + 1215.972 * e3;
    g410 = -1052.797 + 4758.686 * e - 7193.992 * e2 + 3651.957 * e3;
    g422 = -3581.690 + 16178.110 * e - 24462.770 * e2 + 12422.520 * e3;
    if (e > 0.715)
      g520 = -5149.66 + 29936.92 * e - 54087.36 * e2 + 31324.56 * e3;
    else
      g520 = 1464.74 - 4664.75 * e + 3763.64 * e2;
  }
  if (e < 0.7) {
    g533 = -919.22770 + 4988.6100 * e - 9064.7700 * e2 + 5542.21 * e3;
    g521 = -822.71072 + 4568.6173 * e - 8491.4146 * e2 + 5337.524 * e3;
    g532 = -853.66600 + 4690.2500 * e - 8624.7700 * e2 + 5341.4 * e3;
  } else {
    g533 = -37995.780 + 161616.52 * e - 229838.20 * e2 + 109377.94 * e3;
    g521 = -51752.104 + 218913.95 * e - 309468.16 * e2 + 146349.42 * e3;
    g532 = -40023.880 + 170470.89 * e - 242699.48 * e2 + 115605.82 * e3;
  }
  // ... and F_lmp(i) of the (l,m,p) = (2,2,0), (2,2,1), (3,2,1), (3,2,2), (4,4,1),
  // (4,4,2), (5,2,2), (5,2,3), (5,4,2), (5,4,3) terms.
  R ci2 = ci * ci;
  R si2 = si * si;
  R f220 = 0.75 * (1.0 + 2.0 * ci + ci2);
  R f221 = 1.5 * si2;
  R f321 = 1.875 * si * (1.0 - 2.0 * ci - 3.0 * ci2);
  R f322 = -1.875 * si * (1.0 + 2.0 * ci - 3.0 * ci2);
  R f441 = 35.0 * si2 * f220;
  R f442 = 39.3750 * si2 * si2;
  R f522 = 9.84375 * si * (si2 * (1.0 - 2.0 * ci - 5.0 * ci2) +
                           0.33333333 * (-2.0 + 4.0 * ci + 6.0 * ci2));
  R f523 = si * (4.92187512 * si2 * (-2.0 - 4.0 * ci + 10.0 * ci2) +
                 6.56250012 * (1.0 + 2.0 * ci - 3.0 * ci2));
  R f542 = 29.53125 * si * (2.0 - 8.0 * ci + ci2 * (-12.0 + 8.0 * ci + 10.0 * ci2));
  R f543 = 29.53125 * si * (-2.0 - 8.0 * ci + ci2 * (12.0 + 8.0 * ci - 10.0 * ci2));
  // dn/dt amplitude of term (l,m,p,q): 3 n^2 (1/a)^l F G J_lm (l - 2p + q), the last
  // factor being 1 for m = 2 and 2 for m = 4.
  R k3 = k * aonv, k4 = k3 * aonv, k5 = k4 * aonv;
  rc.d2201 = k * kR22 * f220 * g201;
  rc.d2211 = k * kR22 * f221 * g211;
  rc.d3210 = k3 * kR32 * f321 * g310;
  rc.d3222 = k3 * kR32 * f322 * g322;
  rc.d4410 = 2.0 * k4 * kR44 * f441 * g410;
  rc.d4422 = 2.0 * k4 * kR44 * f442 * g422;
  rc.d5220 = k5 * kR52 * f522 * g520;
  rc.d5232 = k5 * kR52 * f523 * g532;
  rc.d5421 = 2.0 * k5 * kR54 * f542 * g521;
  rc.d5433 = 2.0 * k5 * kR54 * f543 * g533;
  rc.lambda0 = fmod(rc.m0 + 2.0 * rc.raan0 - 2.0 * rc.gsto, kTwoPi);
  rc.xfact = rc.Mdot + rc.mdot_ls + 2.0 * (rc.raandot + rc.raandot_ls - kEarthRot) - rc.n0pp;
}

template <class R>
void sgp4_init_rec(const Geo& g, const DeepConsts& dc, const R el[7], double ep_day,
                   double ep_frac, Rec<R>& rc) {
  rc.n0 = el[0]; rc.e0 = el[1]; rc.i0 = el[2]; rc.raan0 = el[3];
  rc.argp0 = el[4]; rc.m0 = el[5]; rc.bstar = el[6];
  rc.fatal = 0;
  rc.deep = false;
  rc.irez = 0;
  for (int k = 0; k < 7; ++k)
    if (!finite_val(el[k])) rc.fatal = 1;
  if (rc.fatal == 0 && (rc.e0 < 0.0 || rc.e0 >= 1.0)) rc.fatal = 1;
  if (rc.fatal == 0 && rc.n0 <= 0.0) rc.fatal = 2;
  if (rc.fatal != 0) return;

  const double k2 = 0.5 * g.j2;           // k2 = J2/2 in Earth radii units

  // Recover the un-Kozai'd ("Brouwer") mean motion and semi-major axis.
  rc.cosi = cos(rc.i0);
  rc.sini = sin(rc.i0);
  R theta2 = rc.cosi * rc.cosi;
  rc.x3thm1 = 3.0 * theta2 - 1.0;
  rc.x1mth2 = 1.0 - theta2;
  rc.x7thm1 = 7.0 * theta2 - 1.0;
  R beta0sq = 1.0 - rc.e0 * rc.e0;
  rc.beta0 = sqrt(beta0sq);
  R beta0cube = beta0sq * rc.beta0;
  R a1 = pow(g.xke / rc.n0, 2.0 / 3.0);
  R delta1 = 1.5 * k2 * rc.x3thm1 / (a1 * a1 * beta0cube);
  R a0 = a1 * (1.0 - delta1 / 3.0 - delta1 * delta1 - (134.0 / 81.0) * delta1 * delta1 * delta1);
  R delta0 = 1.5 * k2 * rc.x3thm1 / (a0 * a0 * beta0cube);
  rc.n0pp = rc.n0 / (1.0 + delta0);
  rc.a0pp = pow(g.xke / rc.n0pp, 2.0 / 3.0);

  // Perigee-dependent atmosphere parameter s and (q0 - s)^4.
  R rp = rc.a0pp * (1.0 - rc.e0);              // perigee radius, ER
  R hp_km = (rp - 1.0) * g.re;                 // perigee height, km
  rc.isimp = rp < 1.0 + 220.0 / g.re;
  // Deep space: period 2 pi / n0'' of 225 min or more; its drag is always truncated.
  rc.deep = kTwoPi / rc.n0pp >= 225.0;
  if (rc.deep) rc.isimp = true;
  R s_km = R(78.0);
  if (hp_km < 156.0) s_km = hp_km - 78.0;
  if (hp_km < 98.0) s_km = R(20.0);
  R q0ms = (120.0 - s_km) / g.re;
  R q0ms4 = q0ms * q0ms * q0ms * q0ms;
  rc.s = 1.0 + s_km / g.re;

  rc.xi = 1.0 / (rc.a0pp - rc.s);
  rc.eta = rc.a0pp * rc.e0 * rc.xi;
  R eta2 = rc.eta * rc.eta;
  R e0eta = rc.e0 * rc.eta;
  R psi2 = fabs(1.0 - eta2);
  R xi4 = rc.xi * rc.xi * rc.xi * rc.xi;
  R coef = q0ms4 * xi4;
  R coef1 = coef / pow(psi2, 3.5);

  R C2 = coef1 * rc.n0pp *
         (rc.a0pp * (1.0 + 1.5 * eta2 + e0eta * (4.0 + eta2)) +
          0.375 * g.j2 * rc.xi / psi2 * rc.x3thm1 * (8.0 + 3.0 * eta2 * (8.0 + eta2)));
  rc.C1 = rc.bstar * C2;
  rc.C3 = R(0.0);
  if (rc.e0 > 1.0e-4)
    rc.C3 = -2.0 * coef * rc.xi * g.j3oj2 * rc.n0pp * rc.sini / rc.e0;
  rc.C4 = 2.0 * rc.n0pp * coef1 * rc.a0pp * beta0sq *
          (rc.eta * (2.0 + 0.5 * eta2) + rc.e0 * (0.5 + 2.0 * eta2) -
           g.j2 * rc.xi / (rc.a0pp * psi2) *
               (-3.0 * rc.x3thm1 * (1.0 - 2.0 * e0eta + eta2 * (1.5 - 0.5 * e0eta)) +
                0.75 * rc.x1mth2 * (2.0 * eta2 - e0eta * (1.0 + eta2)) * cos(2.0 * rc.argp0)));
  rc.C5 = 2.0 * coef1 * rc.a0pp * beta0sq * (1.0 + 2.75 * (eta2 + e0eta) + e0eta * eta2);

  // Secular rates from J2 (first and second order) and J4.
  R p0 = rc.a0pp * beta0sq;
  R pinv2 = 1.0 / (p0 * p0);
  R T1 = 1.5 * g.j2 * pinv2 * rc.n0pp;
  R T2 = 0.5 * T1 * g.j2 * pinv2;
  R T3 = -0.46875 * g.j4 * pinv2 * pinv2 * rc.n0pp;
  R theta4 = theta2 * theta2;
  rc.Mdot = rc.n0pp + 0.5 * T1 * rc.beta0 * rc.x3thm1 +
            0.0625 * T2 * rc.beta0 * (13.0 - 78.0 * theta2 + 137.0 * theta4);
  rc.argpdot = -0.5 * T1 * (1.0 - 5.0 * theta2) +
               0.0625 * T2 * (7.0 - 114.0 * theta2 + 395.0 * theta4) +
               T3 * (3.0 - 36.0 * theta2 + 49.0 * theta4);
  R raandot1 = -T1 * rc.cosi;
  rc.raandot = raandot1 + (0.5 * T2 * (4.0 - 19.0 * theta2) + 2.0 * T3 * (3.0 - 7.0 * theta2)) * rc.cosi;

  // Drag terms of the secular update.
  rc.raan_cf = 3.5 * beta0sq * raandot1 * rc.C1;
  rc.argp_cf = rc.bstar * rc.C3 * cos(rc.argp0);
  rc.m_cf = R(0.0);
  if (rc.e0 > 1.0e-4) rc.m_cf = -(2.0 / 3.0) * coef * rc.bstar / e0eta;
  rc.L2 = 1.5 * rc.C1;

  // Long-period (J3) coefficients; the (1 + cos i0) pole is guarded as in the theory.
  R one_p_cos = 1.0 + rc.cosi;
  if (fabs(one_p_cos) <= 1.5e-12) one_p_cos = R(1.5e-12);
  rc.xlcof = -0.25 * g.j3oj2 * rc.sini * (3.0 + 5.0 * rc.cosi) / one_p_cos;
  rc.aycof = -0.5 * g.j3oj2 * rc.sini;

  R c = 1.0 + rc.eta * cos(rc.m0);
  rc.delM0 = c * c * c;
  rc.sinM0 = sin(rc.m0);

  rc.D2 = R(0.0); rc.D3 = R(0.0); rc.D4 = R(0.0);
  rc.L3 = R(0.0); rc.L4 = R(0.0); rc.L5 = R(0.0);
  if (!rc.isimp) {
    R C1sq = rc.C1 * rc.C1;
    rc.D2 = 4.0 * rc.a0pp * rc.xi * C1sq;
    rc.D3 = (4.0 / 3.0) * rc.a0pp * rc.xi * rc.xi * (17.0 * rc.a0pp + rc.s) * C1sq * rc.C1;
    rc.D4 = (2.0 / 3.0) * rc.a0pp * rc.a0pp * rc.xi * rc.xi * rc.xi *
            (221.0 * rc.a0pp + 31.0 * rc.s) * C1sq * C1sq;
    rc.L3 = rc.D2 + 2.0 * C1sq;
    rc.L4 = 0.25 * (3.0 * rc.D3 + 12.0 * rc.C1 * rc.D2 + 10.0 * C1sq * rc.C1);
    rc.L5 = 0.2 * (3.0 * rc.D4 + 12.0 * rc.C1 * rc.D3 + 6.0 * rc.D2 * rc.D2 +
                   30.0 * C1sq * rc.D2 + 15.0 * C1sq * C1sq);
  }
  if (rc.deep) deep_init(g, dc, ep_day, ep_frac, rc);
}

// Mean (secularly updated) elements at tsince, before the periodic terms.
template <class R>
struct Mean {
  R a, e, n;          // semi-major axis (ER), eccentricity, mean motion (rad/min)
  R raan, argp, M;    // reduced mod 2 pi
  R i;                // inclination (i0 for near-Earth records)
  int code;           // 0, 1 or 2
};

// Tesseral resonance: the resonant longitude lambda and the mean motion n, integrated
// from the epoch to t with fixed steps of 720 min, each a second-order Taylor step
// (dlambda/dt = n + xfact, dn/dt from the resonance terms, d2n/dt2 from their
// derivative along lambda), and a final partial step to t.  In the two-per-day terms
// the perigee moves at its J2 secular rate.  The integration covers |t| <= kResMaxT
// (about 19 years); beyond that, or for a non-finite t, it returns false.
static const double kResMaxT = 1.0e7;

template <class R>
bool resonance(const Rec<R>& rc, double t, R& n_out, R& lambda_out) {
  if (!(std::fabs(t) <= kResMaxT)) return false;
  const double h = (t > 0.0) ? kResStep : -kResStep;
  double tc = 0.0;
  R lam = rc.lambda0;
  R n = rc.n0pp;
  for (;;) {
    R ldot = n + rc.xfact;
    R ndot, nddot;
    if (rc.irez == 1) {
      ndot = rc.del1 * sin(lam - kPhase31) + rc.del2 * sin(2.0 * (lam - kPhase22)) +
             rc.del3 * sin(3.0 * (lam - kPhase33));
      nddot = (rc.del1 * cos(lam - kPhase31) + 2.0 * rc.del2 * cos(2.0 * (lam - kPhase22)) +
               3.0 * rc.del3 * cos(3.0 * (lam - kPhase33))) * ldot;
    } else {
      R w = rc.argp0 + rc.argpdot * tc;
      R w2 = 2.0 * w;
      R l2 = 2.0 * lam;
      ndot = rc.d2201 * sin(w2 + lam - kG22) + rc.d2211 * sin(lam - kG22) +
             rc.d3210 * sin(w + lam - kG32) + rc.d3222 * sin(-w + lam - kG32) +
             rc.d4410 * sin(w2 + l2 - kG44) + rc.d4422 * sin(l2 - kG44) +
             rc.d5220 * sin(w + lam - kG52) + rc.d5232 * sin(-w + lam - kG52) +
             rc.d5421 * sin(w + l2 - kG54) + rc.d5433 * sin(-w + l2 - kG54);
      nddot = (rc.d2201 * cos(w2 + lam - kG22) + rc.d2211 * cos(lam - kG22) +
               rc.d3210 * cos(w + lam - kG32) + rc.d3222 * cos(-w + lam - kG32) +
               rc.d5220 * cos(w + lam - kG52) + rc.d5232 * cos(-w + lam - kG52) +
               2.0 * (rc.d4410 * cos(w2 + l2 - kG44) + rc.d4422 * cos(l2 - kG44) +
                      rc.d5421 * cos(w + l2 - kG54) + rc.d5433 * cos(-w + l2 - kG54))) * ldot;
    }
    if (std::fabs(t - tc) >= kResStep) {
      lam = lam + ldot * h + ndot * (0.5 * h * h);
      n = n + ndot * h + nddot * (0.5 * h * h);
      tc += h;
    } else {
      double ft = t - tc;
      n_out = n + ndot * ft + nddot * (0.5 * ft * ft);
      lambda_out = lam + ldot * ft + ndot * (0.5 * ft * ft);
      return true;
    }
  }
}

template <class R>
Mean<R> secular(const Geo& g, const Rec<R>& rc, double t) {
  Mean<R> m;
  m.code = 0;
  R M_df = rc.m0 + rc.Mdot * t;
  R argp_df = rc.argp0 + rc.argpdot * t;
  R raan_df = rc.raan0 + rc.raandot * t;
  R M = M_df;
  R argp = argp_df;
  double t2 = t * t;
  R raan = raan_df + rc.raan_cf * t2;
  R tempa = 1.0 - rc.C1 * t;
  R tempe = rc.bstar * rc.C4 * t;
  R templ = rc.L2 * t2;
  if (!rc.isimp) {
    R dargp = rc.argp_cf * t;
    R c = 1.0 + rc.eta * cos(M_df);
    R dM = rc.m_cf * (c * c * c - rc.delM0);
    M = M_df + dargp + dM;
    argp = argp_df - dargp - dM;
    double t3 = t2 * t, t4 = t3 * t;
    tempa = tempa - rc.D2 * t2 - rc.D3 * t3 - rc.D4 * t4;
    tempe = tempe + rc.bstar * rc.C5 * (sin(M) - rc.sinM0);
    templ = templ + rc.L3 * t3 + t4 * (rc.L4 + t * rc.L5);
  }
  R n = rc.n0pp;
  R e = rc.e0;
  m.i = rc.i0;
  if (rc.deep) {
    // Lunar-solar secular rates, then the resonance (mean motion and mean anomaly).
    e = e + rc.edot * t;
    m.i = m.i + rc.idot * t;
    argp = argp + rc.argpdot_ls * t;
    raan = raan + rc.raandot_ls * t;
    M = M + rc.mdot_ls * t;
    if (rc.irez != 0) {
      R lam;
      if (!resonance(rc, t, n, lam)) { m.code = 2; return m; }
      double theta = std::fmod(rc.gsto + t * kEarthRot, kTwoPi);
      if (rc.irez == 1)
        M = lam - raan - argp + theta;
      else
        M = lam - 2.0 * raan + 2.0 * theta;
    }
  }
  if (n <= 0.0) { m.code = 2; return m; }
  m.a = pow(g.xke / n, 2.0 / 3.0) * tempa * tempa;
  m.n = g.xke / pow(m.a, 1.5);
  m.e = e - tempe;
  if (m.e >= 1.0 || m.e < -0.001) { m.code = 1; return m; }
  if (m.e < 1.0e-6) m.e = R(1.0e-6);
  M = M + rc.n0pp * templ;
  R L = M + argp + raan;
  m.raan = fmod(raan, kTwoPi);
  m.argp = fmod(argp, kTwoPi);
  L = fmod(L, kTwoPi);
  m.M = fmod(L - m.argp - m.raan, kTwoPi);
  return m;
}

// Kepler's equation in the (a_xN, a_yN) form: find psi with
// psi - a_xN sin psi + a_yN cos psi = U.  Newton, step clamped to +-0.95.
template <class R>
R kepler(const R& U, const R& axn, const R& ayn, int* iters) {
  R psi = U;
  int k = 0;
  while (k < 10) {
    R sp = sin(psi), cp = cos(psi);
    R f = U - ayn * cp + axn * sp - psi;
    R fp = 1.0 - ayn * sp - axn * cp;
    R step = f / fp;
    if (step >= 0.95) step = R(0.95);
    else if (step <= -0.95) step = R(-0.95);
    psi = psi + step;
    ++k;
    if (fabs(val(step)) < 1.0e-12) break;
  }
  if (iters) *iters = k;
  return psi;
}

// Lunar-solar long-period terms at t added to the mean elements (e, i, node, perigee,
// mean anomaly).  Each body's true anomaly is taken to first order in its
// eccentricity.  Above 0.2 rad of (perturbed) inclination the node and perigee terms
// are applied directly; below, through the components of the orbit normal (Lyddane's
// form, which stays regular as sin i -> 0), with the node kept on the branch nearest
// its mean value.
template <class R>
void lunar_solar_periodics(const Rec<R>& rc, double t, R& e, R& inc, R& raan, R& argp, R& M) {
  R pe(0.0), pinc(0.0), pl(0.0), pgh(0.0), ph(0.0);
  const LunarSolar<R>* bodies[2] = {&rc.sun, &rc.moon};
  for (const LunarSolar<R>* b : bodies) {
    double Mb = b->M0 + b->n * t;
    double f = Mb + 2.0 * b->ecc * std::sin(Mb);
    double sf = std::sin(f), cf = std::cos(f);
    double F2 = 0.5 * sf * sf - 0.25;
    double F3 = -0.5 * sf * cf;
    pe = pe + b->e2 * F2 + b->e3 * F3;
    pinc = pinc + b->i2 * F2 + b->i3 * F3;
    pl = pl + b->l2 * F2 + b->l3 * F3 + b->l4 * sf;
    pgh = pgh + b->gh2 * F2 + b->gh3 * F3 + b->gh4 * sf;
    ph = ph + b->h2 * F2 + b->h3 * F3;
  }
  inc = inc + pinc;
  e = e + pe;
  R si = sin(inc), ci = cos(inc);
  if (inc >= 0.2) {
    R dnode = ph / si;
    argp = argp + (pgh - ci * dnode);
    raan = raan + dnode;
    M = M + pl;
    return;
  }
  R so = sin(raan), co = cos(raan);
  R alpha = si * so + (ph * co + pinc * ci * so);
  R beta = si * co + (-ph * so + pinc * ci * co);
  raan = fmod(raan, kTwoPi);
  R L = M + argp + ci * raan + (pl + pgh - pinc * raan * si);
  R mean_node = raan;
  raan = atan2(alpha, beta);
  if (fabs(mean_node - raan) > kPi) raan = (val(raan) < val(mean_node)) ? raan + kTwoPi : raan - kTwoPi;
  M = M + pl;
  argp = L - M - ci * raan;
}

// One state: position (km) and velocity (km/s) in TEME at tsince (min).
template <class R>
int sgp4_state(const Geo& g, const Rec<R>& rc, double t, R r[3], R v[3]) {
  if (rc.fatal) return rc.fatal;
  Mean<R> m = secular(g, rc, t);
  if (m.code) return m.code;

  // Deep space: lunar-solar periodics, then the inclination, its functions and the
  // J3 coefficients at the perturbed inclination.
  R ecc = m.e, inc = m.i, raan = m.raan, argp = m.argp, Mp = m.M;
  R cosi = rc.cosi, sini = rc.sini;
  R x3thm1 = rc.x3thm1, x1mth2 = rc.x1mth2, x7thm1 = rc.x7thm1;
  R xlcof = rc.xlcof, aycof = rc.aycof;
  if (rc.deep) {
    lunar_solar_periodics(rc, t, ecc, inc, raan, argp, Mp);
    if (inc < 0.0) { inc = -inc; raan = raan + kPi; argp = argp - kPi; }
    if (ecc < 0.0 || ecc > 1.0) return 3;
    cosi = cos(inc);
    sini = sin(inc);
    R c2 = cosi * cosi;
    x3thm1 = 3.0 * c2 - 1.0;
    x1mth2 = 1.0 - c2;
    x7thm1 = 7.0 * c2 - 1.0;
    R one_p_cos = 1.0 + cosi;
    if (fabs(one_p_cos) <= 1.5e-12) one_p_cos = R(1.5e-12);
    xlcof = -0.25 * g.j3oj2 * sini * (3.0 + 5.0 * cosi) / one_p_cos;
    aycof = -0.5 * g.j3oj2 * sini;
  }

  // Long-period periodics (J3).
  R axn = ecc * cos(argp);
  R q = 1.0 / (m.a * (1.0 - ecc * ecc));
  R ayn = ecc * sin(argp) + q * aycof;
  R LT = Mp + argp + raan + q * xlcof * axn;
  R U = fmod(LT - raan, kTwoPi);

  // Kepler's equation.
  R psi = kepler(U, axn, ayn, nullptr);
  R sp = sin(psi), cp = cos(psi);

  // Short-period preliminaries.
  R ecosE = axn * cp + ayn * sp;
  R esinE = axn * sp - ayn * cp;
  R eL2 = axn * axn + ayn * ayn;
  R pL = m.a * (1.0 - eL2);
  if (pL < 0.0) return 4;
  R rr = m.a * (1.0 - ecosE);
  R rdot = sqrt(m.a) * esinE / rr;
  R rfdot = sqrt(pL) / rr;
  R betaL = sqrt(1.0 - eL2);
  R w = esinE / (1.0 + betaL);
  R sinu = m.a / rr * (sp - ayn - axn * w);
  R cosu = m.a / rr * (cp - axn + ayn * w);
  R u = atan2(sinu, cosu);
  R sin2u = 2.0 * cosu * sinu;
  R cos2u = 1.0 - 2.0 * sinu * sinu;

  // Short-period periodics (J2).
  R k = 0.5 * g.j2 / pL;     // k2 / p_L
  R kp = k / pL;             // k2 / p_L^2
  R rk = rr * (1.0 - 1.5 * kp * betaL * x3thm1) + 0.5 * k * x1mth2 * cos2u;
  R uk = u - 0.25 * kp * x7thm1 * sin2u;
  R raank = raan + 1.5 * kp * cosi * sin2u;
  R ik = inc + 1.5 * kp * cosi * sini * cos2u;
  R rdotk = rdot - m.n * k * x1mth2 * sin2u / g.xke;
  R rfdotk = rfdot + m.n * k * (x1mth2 * cos2u + 1.5 * x3thm1) / g.xke;

  // Orientation vectors and TEME output.
  R su = sin(uk), cu = cos(uk);
  R sO = sin(raank), cO = cos(raank);
  R si = sin(ik), ci = cos(ik);
  R Mx = -sO * ci, My = cO * ci, Mz = si;
  R Nx = cO, Ny = sO;
  R Ux = Mx * su + Nx * cu, Uy = My * su + Ny * cu, Uz = Mz * su;
  R Vx = Mx * cu - Nx * su, Vy = My * cu - Ny * su, Vz = Mz * cu;
  double vscale = g.re * g.xke / 60.0;
  r[0] = rk * Ux * g.re; r[1] = rk * Uy * g.re; r[2] = rk * Uz * g.re;
  v[0] = (rdotk * Ux + rfdotk * Vx) * vscale;
  v[1] = (rdotk * Uy + rfdotk * Vy) * vscale;
  v[2] = (rdotk * Uz + rfdotk * Vz) * vscale;
  if (rk < 1.0) return 6;
  return 0;
}

// Status at t = 0 after a usable init (2006-revision practice).
template <class R>
int init_status(const Geo& g, const Rec<R>& rc) {
  if (rc.fatal) return rc.fatal;
  R r[3], v[3];
  return sgp4_state(g, rc, 0.0, r, v);
}

template <class F>
void parallel_for(int64_t n, int nthreads, F&& body) {
  if (nthreads <= 1 || n < 2) { body(int64_t(0), n); return; }
  nthreads = (int)std::min<int64_t>(nthreads, n);
  std::vector<std::thread> pool;
  int64_t chunk = (n + nthreads - 1) / nthreads;
  for (int k = 0; k < nthreads; ++k) {
    int64_t lo = k * chunk, hi = std::min<int64_t>(n, lo + chunk);
    if (lo >= hi) break;
    pool.emplace_back([=, &body] { body(lo, hi); });
  }
  for (auto& th : pool) th.join();
}

}  // namespace oracle

using namespace oracle;

static const double kNaN = std::numeric_limits<double>::quiet_NaN();

extern "C" {

int oracle_abi_version(void) { return 2; }

// Common arguments of the entry points below:
//   consts   [5]: mu (km^3/s^2), Earth radius (km), J2, J3, J4
//   dconsts  [7] or NULL: the deep-space constants of DeepConsts (NULL: the theory's)
//   el       [n][7]: n0 (rad/min), e0, i0, RAAN0, argp0, M0 (rad), B* (1/ER)
//   epoch    [n][2] or NULL: each record's epoch as a Julian date, integer day and
//            fraction (NULL: epoch 0); used by the deep-space terms only
static void init_one(const Geo& g, const DeepConsts& dc, const double* el, const double* epoch,
                     int64_t j, Rec<double>& rc) {
  double e7[7];
  for (int k = 0; k < 7; ++k) e7[k] = el[j * 7 + k];
  double d = epoch ? epoch[2 * j] : 0.0, f = epoch ? epoch[2 * j + 1] : 0.0;
  sgp4_init_rec(g, dc, e7, d, f, rc);
}

// Full propagation: tsince [T] (common grid) or [n][T] (per_sat_grid != 0), minutes.
// Outputs r, v [n][T][3] (km, km/s), status [n][T], init_status [n] (may be NULL).
void oracle_propagate(const double* consts, const double* dconsts, const double* el,
                      const double* epoch, int64_t n, const double* tsince, int64_t T,
                      int per_sat_grid, double* r, double* v, int32_t* status,
                      int32_t* init_stat, int nthreads) {
  const Geo g = make_geo(consts);
  const DeepConsts dc = make_deep(dconsts);
  parallel_for(n, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t j = lo; j < hi; ++j) {
      Rec<double> rc;
      init_one(g, dc, el, epoch, j, rc);
      if (init_stat) init_stat[j] = init_status(g, rc);
      const double* tj = per_sat_grid ? tsince + j * T : tsince;
      for (int64_t i = 0; i < T; ++i) {
        double rr[3], vv[3];
        int code = sgp4_state(g, rc, tj[i], rr, vv);
        int64_t o = (j * T + i);
        status[o] = code;
        bool keep = (code == 0 || code == 6);
        for (int c = 0; c < 3; ++c) {
          r[o * 3 + c] = keep ? rr[c] : kNaN;
          v[o * 3 + c] = keep ? vv[c] : kNaN;
        }
      }
    }
  });
}

// Record fields, one row of ORACLE_NREC values per satellite (names in oracle/__init__.py).
#define ORACLE_NREC 36
int oracle_nrec(void) { return ORACLE_NREC; }

void oracle_records(const double* consts, const double* dconsts, const double* el,
                    const double* epoch, int64_t n, double* out, int32_t* isimp,
                    int32_t* init_stat) {
  const Geo g = make_geo(consts);
  const DeepConsts dc = make_deep(dconsts);
  for (int64_t j = 0; j < n; ++j) {
    Rec<double> rc;
    init_one(g, dc, el, epoch, j, rc);
    double* o = out + j * ORACLE_NREC;
    for (int k = 0; k < ORACLE_NREC; ++k) o[k] = kNaN;
    if (init_stat) init_stat[j] = init_status(g, rc);
    if (isimp) isimp[j] = rc.fatal ? -1 : (rc.isimp ? 1 : 0);
    if (rc.fatal) continue;
    const double f[ORACLE_NREC] = {
        rc.n0pp, rc.a0pp, rc.cosi, rc.sini, rc.x3thm1, rc.x1mth2, rc.x7thm1, rc.beta0,
        rc.s, rc.xi, rc.eta, rc.C1, rc.C3, rc.C4, rc.C5, rc.D2, rc.D3, rc.D4,
        rc.Mdot, rc.argpdot, rc.raandot, rc.raan_cf, rc.argp_cf, rc.m_cf,
        rc.L2, rc.L3, rc.L4, rc.L5, rc.xlcof, rc.aycof, rc.delM0, rc.sinM0,
        rc.e0, rc.i0, rc.bstar, g.xke};
    for (int k = 0; k < ORACLE_NREC; ++k) o[k] = f[k];
  }
}

// Deep-space fields, one row of ORACLE_NDEEP values per satellite (names in
// oracle/__init__.py); deep[j] = -1 (unusable elements), 0 (near-Earth) or
// 1 + irez (deep space, irez = 0, 1, 2).
#define ORACLE_NDEEP 48
int oracle_ndeep(void) { return ORACLE_NDEEP; }

void oracle_deep_records(const double* consts, const double* dconsts, const double* el,
                         const double* epoch, int64_t n, double* out, int32_t* deep) {
  const Geo g = make_geo(consts);
  const DeepConsts dc = make_deep(dconsts);
  for (int64_t j = 0; j < n; ++j) {
    Rec<double> rc;
    init_one(g, dc, el, epoch, j, rc);
    double* o = out + j * ORACLE_NDEEP;
    for (int k = 0; k < ORACLE_NDEEP; ++k) o[k] = kNaN;
    deep[j] = rc.fatal ? -1 : (rc.deep ? 1 + rc.irez : 0);
    if (rc.fatal || !rc.deep) continue;
    const LunarSolar<double>& S = rc.sun;
    const LunarSolar<double>& L = rc.moon;
    const double f[ORACLE_NDEEP] = {
        rc.gsto, rc.edot, rc.idot, rc.mdot_ls, rc.argpdot_ls, rc.raandot_ls,
        S.e2, S.e3, S.i2, S.i3, S.l2, S.l3, S.l4, S.gh2, S.gh3, S.gh4, S.h2, S.h3, S.M0,
        L.e2, L.e3, L.i2, L.i3, L.l2, L.l3, L.l4, L.gh2, L.gh3, L.gh4, L.h2, L.h3, L.M0,
        rc.del1, rc.del2, rc.del3,
        rc.d2201, rc.d2211, rc.d3210, rc.d3222, rc.d4410, rc.d4422, rc.d5220, rc.d5232,
        rc.d5421, rc.d5433, rc.lambda0, rc.xfact, (double)rc.irez};
    for (int k = 0; k < ORACLE_NDEEP; ++k) o[k] = f[k];
  }
}

// Mean elements after the secular update (deep space: with the lunar-solar secular
// rates and the resonance, before the periodic terms): out [n][T][8] = (a ER, e,
// n rad/min, RAAN, argp, M reduced, code, i).
void oracle_mean(const double* consts, const double* dconsts, const double* el,
                 const double* epoch, int64_t n, const double* tsince, int64_t T, double* out) {
  const Geo g = make_geo(consts);
  const DeepConsts dc = make_deep(dconsts);
  for (int64_t j = 0; j < n; ++j) {
    Rec<double> rc;
    init_one(g, dc, el, epoch, j, rc);
    for (int64_t i = 0; i < T; ++i) {
      double* o = out + (j * T + i) * 8;
      for (int k = 0; k < 8; ++k) o[k] = kNaN;
      if (rc.fatal) { o[6] = rc.fatal; continue; }
      Mean<double> m = secular(g, rc, tsince[i]);
      o[6] = m.code;
      if (m.code) continue;
      o[0] = m.a; o[1] = m.e; o[2] = m.n; o[3] = m.raan; o[4] = m.argp; o[5] = m.M;
      o[7] = m.i;
    }
  }
}

// Deep-space elements after the lunar-solar periodic terms: out [n][T][6] = (e, i,
// RAAN, argp, M, code) for deep-space records (code 3 when e leaves [0, 1]); NaN and
// code -1 for near-Earth records.
void oracle_deep_periodics(const double* consts, const double* dconsts, const double* el,
                           const double* epoch, int64_t n, const double* tsince, int64_t T,
                           double* out) {
  const Geo g = make_geo(consts);
  const DeepConsts dc = make_deep(dconsts);
  for (int64_t j = 0; j < n; ++j) {
    Rec<double> rc;
    init_one(g, dc, el, epoch, j, rc);
    for (int64_t i = 0; i < T; ++i) {
      double* o = out + (j * T + i) * 6;
      for (int k = 0; k < 6; ++k) o[k] = kNaN;
      if (rc.fatal || !rc.deep) { o[5] = -1; continue; }
      Mean<double> m = secular(g, rc, tsince[i]);
      if (m.code) { o[5] = m.code; continue; }
      double e = m.e, inc = m.i, raan = m.raan, argp = m.argp, M = m.M;
      lunar_solar_periodics(rc, tsince[i], e, inc, raan, argp, M);
      o[0] = e; o[1] = inc; o[2] = raan; o[3] = argp; o[4] = M;
      o[5] = (e < 0.0 || e > 1.0) ? 3 : 0;
    }
  }
}

// Kepler solve exposed for the residual / bisection tests.
double oracle_kepler(double U, double axn, double ayn, int32_t* iters) {
  int k = 0;
  double psi = kepler<double>(U, axn, ayn, &k);
  if (iters) *iters = k;
  return psi;
}

// Greenwich mean sidereal angle (rad) at a split Julian date.
double oracle_gmst(double day, double frac) { return gmst82(day, frac); }

// Forward-mode Jacobian: dr, dv [n][T][3][7] = d(r,v)/d(n0, e0, i0, RAAN0, argp0, M0, B*).
// States whose status is not 0 or 6 get NaN.
void oracle_jacobian(const double* consts, const double* dconsts, const double* el,
                     const double* epoch, int64_t n, const double* tsince, int64_t T,
                     int per_sat_grid, double* dr, double* dv, int32_t* status, int nthreads) {
  const Geo g = make_geo(consts);
  const DeepConsts dc = make_deep(dconsts);
  parallel_for(n, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t j = lo; j < hi; ++j) {
      Dual e7[7];
      for (int k = 0; k < 7; ++k) e7[k] = make_var(el[j * 7 + k], k);
      double d = epoch ? epoch[2 * j] : 0.0, f = epoch ? epoch[2 * j + 1] : 0.0;
      Rec<Dual> rc;
      sgp4_init_rec(g, dc, e7, d, f, rc);
      const double* tj = per_sat_grid ? tsince + j * T : tsince;
      for (int64_t i = 0; i < T; ++i) {
        Dual rr[3], vv[3];
        int code = sgp4_state(g, rc, tj[i], rr, vv);
        int64_t o = j * T + i;
        if (status) status[o] = code;
        bool keep = (code == 0 || code == 6);
        for (int c = 0; c < 3; ++c)
          for (int k = 0; k < 7; ++k) {
            dr[(o * 3 + c) * 7 + k] = keep ? rr[c].d[k] : kNaN;
            dv[(o * 3 + c) * 7 + k] = keep ? vv[c].d[k] : kNaN;
          }
      }
    }
  });
}

}  // extern "C"
