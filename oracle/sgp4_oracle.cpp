// SGP4 near-Earth oracle: TEST INFRASTRUCTURE ONLY.
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
};

template <class R>
void sgp4_init_rec(const Geo& g, const R el[7], Rec<R>& rc) {
  rc.n0 = el[0]; rc.e0 = el[1]; rc.i0 = el[2]; rc.raan0 = el[3];
  rc.argp0 = el[4]; rc.m0 = el[5]; rc.bstar = el[6];
  rc.fatal = 0;
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
}

// Mean (secularly updated) elements at tsince, before the periodic terms.
template <class R>
struct Mean {
  R a, e, n;          // semi-major axis (ER), eccentricity, mean motion (rad/min)
  R raan, argp, M;    // reduced mod 2 pi
  int code;           // 0, 1 or 2
};

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
  if (rc.n0pp <= 0.0) { m.code = 2; return m; }
  m.a = pow(g.xke / rc.n0pp, 2.0 / 3.0) * tempa * tempa;
  m.n = g.xke / pow(m.a, 1.5);
  m.e = rc.e0 - tempe;
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

// One state: position (km) and velocity (km/s) in TEME at tsince (min).
template <class R>
int sgp4_state(const Geo& g, const Rec<R>& rc, double t, R r[3], R v[3]) {
  if (rc.fatal) return rc.fatal;
  Mean<R> m = secular(g, rc, t);
  if (m.code) return m.code;

  // Long-period periodics (J3).
  R axn = m.e * cos(m.argp);
  R q = 1.0 / (m.a * (1.0 - m.e * m.e));
  R ayn = m.e * sin(m.argp) + q * rc.aycof;
  R LT = m.M + m.argp + m.raan + q * rc.xlcof * axn;
  R U = fmod(LT - m.raan, kTwoPi);

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
  R rk = rr * (1.0 - 1.5 * kp * betaL * rc.x3thm1) + 0.5 * k * rc.x1mth2 * cos2u;
  R uk = u - 0.25 * kp * rc.x7thm1 * sin2u;
  R raank = m.raan + 1.5 * kp * rc.cosi * sin2u;
  R ik = rc.i0 + 1.5 * kp * rc.cosi * rc.sini * cos2u;
  R rdotk = rdot - m.n * k * rc.x1mth2 * sin2u / g.xke;
  R rfdotk = rfdot + m.n * k * (rc.x1mth2 * cos2u + 1.5 * rc.x3thm1) / g.xke;

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

int oracle_abi_version(void) { return 1; }

// Full propagation: elements [n][7] = (n0 rad/min, e0, i0, RAAN0, argp0, M0 rad, B* 1/ER);
// tsince [T] (common grid) or [n][T] (per_sat_grid != 0), minutes.
// Outputs r, v [n][T][3] (km, km/s), status [n][T], init_status [n] (may be NULL).
void oracle_propagate(const double* consts, const double* el, int64_t n, const double* tsince,
                      int64_t T, int per_sat_grid, double* r, double* v, int32_t* status,
                      int32_t* init_stat, int nthreads) {
  const Geo g = make_geo(consts);
  parallel_for(n, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t j = lo; j < hi; ++j) {
      double e7[7];
      for (int k = 0; k < 7; ++k) e7[k] = el[j * 7 + k];
      Rec<double> rc;
      sgp4_init_rec(g, e7, rc);
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

void oracle_records(const double* consts, const double* el, int64_t n, double* out,
                    int32_t* isimp, int32_t* init_stat) {
  const Geo g = make_geo(consts);
  for (int64_t j = 0; j < n; ++j) {
    double e7[7];
    for (int k = 0; k < 7; ++k) e7[k] = el[j * 7 + k];
    Rec<double> rc;
    sgp4_init_rec(g, e7, rc);
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

// Mean elements after the secular update: out [n][T][7] = (a ER, e, n rad/min,
// RAAN, argp, M reduced, code).
void oracle_mean(const double* consts, const double* el, int64_t n, const double* tsince,
                 int64_t T, double* out) {
  const Geo g = make_geo(consts);
  for (int64_t j = 0; j < n; ++j) {
    double e7[7];
    for (int k = 0; k < 7; ++k) e7[k] = el[j * 7 + k];
    Rec<double> rc;
    sgp4_init_rec(g, e7, rc);
    for (int64_t i = 0; i < T; ++i) {
      double* o = out + (j * T + i) * 7;
      for (int k = 0; k < 7; ++k) o[k] = kNaN;
      if (rc.fatal) { o[6] = rc.fatal; continue; }
      Mean<double> m = secular(g, rc, tsince[i]);
      o[6] = m.code;
      if (m.code) continue;
      o[0] = m.a; o[1] = m.e; o[2] = m.n; o[3] = m.raan; o[4] = m.argp; o[5] = m.M;
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

// Forward-mode Jacobian: dr, dv [n][T][3][7] = d(r,v)/d(n0, e0, i0, RAAN0, argp0, M0, B*).
// States whose status is not 0 or 6 get NaN.
void oracle_jacobian(const double* consts, const double* el, int64_t n, const double* tsince,
                     int64_t T, int per_sat_grid, double* dr, double* dv, int32_t* status,
                     int nthreads) {
  const Geo g = make_geo(consts);
  parallel_for(n, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t j = lo; j < hi; ++j) {
      Dual e7[7];
      for (int k = 0; k < 7; ++k) e7[k] = make_var(el[j * 7 + k], k);
      Rec<Dual> rc;
      sgp4_init_rec(g, e7, rc);
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
