// Adjoint (vector-Jacobian product) of the propagation with respect to the mean
// elements: given upstream gradients g_r, g_v of every state's r, v, it returns
//   g_el[j][k] = sum_t (dr_jt/del_jk) . g_r[j][t] + (dv_jt/del_jk) . g_v[j][t]
// for el = (n0, e0, i0, RAAN0, argp0, M0, B*), through propagation and sgp4init
// (the paper's differentiable propagator, Sec. 5).
//
// Two kernels:
//  * adjoint_prop_kernel: one block per satellite; each thread recomputes its
//    states forward and runs the hand-written reverse sweep of the propagation,
//    accumulating the adjoints of the 33 record fields the propagation reads (per
//    thread columns in shared memory, then a column sum).  The Kepler solve is
//    differentiated at its root (implicit function theorem), the clamps and
//    threshold decisions are constants of the sweep.
//  * adjoint_init_kernel: one thread per satellite pushes the 7 element directions
//    through sgp4init with dual numbers (the record build is per satellite, so
//    forward mode costs nothing next to the per-state sweep) and contracts the
//    record-field Jacobian with the accumulated field adjoints.
// States whose status is 1, 2 or 4 (NaN output) contribute nothing.
#include <cmath>
#include <cstdint>

#include "sgp4.h"
#include "sgp4_device.cuh"
#include "sgp4_init_math.cuh"
#include "sgp4_kernels.cuh"

namespace sgp4 {

namespace {

// Record fields, in Rec64 order.
enum AdjField {
  aN0pp, aA0pp, aE0, aI0, aRaan0, aArgp0, aM0, aMdot, aArgpdot, aRaandot, aRaanCf, aArgpCf,
  aMCf, aC1, aBC4, aBC5, aD2, aD3, aD4, aL2, aL3, aL4, aL5, aEta, aDelM0, aSinM0, aXlcof,
  aAycof, aCosi, aSini, aX3thm1, aX1mth2, aX7thm1, kNumAdj
};

constexpr int kAdjThreads = 128;

__device__ __forceinline__ void sc(double x, double& s, double& c) { sincos(x, &s, &c); }
__device__ __forceinline__ void sc(float x, float& s, float& c) { sincosf(x, &s, &c); }

// Forward recomputation and reverse sweep of one state in precision T.  Adds the
// adjoint of every record field into acc[f * kAdjThreads].  Returns the status.
template <class T>
__device__ int adjoint_state(const Rec64& rc, const Geo& g, double t, const T gr[3],
                             const T gv[3], double* acc, T* r_out = nullptr) {
  const int fatal = (rc.flags >> kFatalShift) & 0xff;
  if (fatal) return fatal;
  if (rc.flags & kFlagN0ppNonPos) return 2;
  const bool isimp = rc.flags & kFlagIsimp;
  const T one = T(1), two = T(2), half = T(0.5);

  // ------------------------------------------------------------------ forward
  // The angle sums (which grow as n t) in FP64; everything else in T.
  const double mdf_d = rc.m0 + rc.mdot * t;
  const double argpdf_d = rc.argp0 + rc.argpdot * t;
  const double t2d = t * t;
  const double raan1_d = rc.raan0 + rc.raandot * t + rc.raan_cf * t2d;
  const T tt = T(t), t2 = T(t2d), t3 = t2 * tt, t4 = t3 * tt;
  const T c1 = T(rc.c1), bc4 = T(rc.bc4), l2 = T(rc.l2);
  T tempa = one - c1 * tt;
  T tempe = bc4 * tt;
  T templ = l2 * t2;
  T sMdf = T(0), cMdf = T(0), c = one, dm = T(0), sMM = T(0), cMM = T(0);
  double mm1_d = mdf_d, argp1_d = argpdf_d;
  const T eta = T(rc.eta), mcf = T(rc.m_cf), delm0 = T(rc.delm0), bc5 = T(rc.bc5);
  const T d2 = T(rc.d2), d3 = T(rc.d3), d4 = T(rc.d4), l3 = T(rc.l3), l4 = T(rc.l4);
  const T l5 = T(rc.l5), sinm0 = T(rc.sinm0), argpcf = T(rc.argp_cf);
  if (!isimp) {
    const T dargp = argpcf * tt;
    sc(T(fmod(mdf_d, kTwoPi)), sMdf, cMdf);
    c = one + eta * cMdf;
    dm = mcf * (c * c * c - delm0);
    mm1_d = mdf_d + (double)dargp + (double)dm;
    argp1_d = argpdf_d - (double)dargp - (double)dm;
    tempa = tempa - d2 * t2 - d3 * t3 - d4 * t4;
    sc(T(fmod(mm1_d, kTwoPi)), sMM, cMM);
    tempe = tempe + bc5 * (sMM - sinm0);
    templ = templ + l3 * t3 + t4 * (l4 + tt * l5);
  }
  const T a0pp = T(rc.a0pp), e0 = T(rc.e0);
  const T a = a0pp * tempa * tempa;
  const T sqa = sqrt(a);
  const T xke = T(g.xke);
  const T n = xke / (a * sqa);
  const T e1 = e0 - tempe;
  if (e1 >= one || e1 < T(-0.001)) return 1;
  const bool clamped = e1 < T(1.0e-6);
  const T e = clamped ? T(1.0e-6) : e1;
  const double mm2_d = mm1_d + rc.n0pp * (double)templ;
  const T raan = T(fmod(raan1_d, kTwoPi));
  const T argp = T(fmod(argp1_d, kTwoPi));
  const T mpa = T(fmod(mm2_d + argp1_d, kTwoPi));   // M + argp (the node cancels in U)
  T sw, cw;
  sc(argp, sw, cw);
  const T axn = e * cw;
  const T om = one - e * e;
  const T qa = a * om;
  const T q = one / qa;
  const T aycof = T(rc.aycof), xlcof = T(rc.xlcof);
  const T ayn = e * sw + q * aycof;
  const T U = mpa + q * xlcof * axn;
  T psi = U;
  const T tol = sizeof(T) == 8 ? T(1.0e-12) : T(1.0e-6);
  for (int k = 0; k < 10; ++k) {
    T sp, cp;
    sc(psi, sp, cp);
    T step = (U - ayn * cp + axn * sp - psi) / (one - ayn * sp - axn * cp);
    step = fmin(fmax(step, T(-0.95)), T(0.95));
    psi += step;
    if (fabs(step) < tol) break;
  }
  T sp, cp;
  sc(psi, sp, cp);
  const T ecosE = axn * cp + ayn * sp;
  const T esinE = axn * sp - ayn * cp;
  const T eL2 = axn * axn + ayn * ayn;
  const T pL = a * (one - eL2);
  if (pL < T(0)) return 4;
  const T rl = a * (one - ecosE);
  const T rdotl = sqa * esinE / rl;
  const T sqp = sqrt(pL);
  const T rfdotl = sqp / rl;
  const T betal = sqrt(one - eL2);
  const T opb = one + betal;
  const T w = esinE / opb;
  const T aor = a / rl;
  const T As = sp - ayn - axn * w;
  const T Ac = cp - axn + ayn * w;
  const T sinu = aor * As, cosu = aor * Ac;
  const T u = atan2(sinu, cosu);
  const T sin2u = two * cosu * sinu;
  const T cos2u = one - two * sinu * sinu;
  const T j2 = T(g.j2);
  const T k = half * j2 / pL;
  const T kp = k / pL;
  const T x3thm1 = T(rc.x3thm1), x1mth2 = T(rc.x1mth2), x7thm1 = T(rc.x7thm1);
  const T cosi = T(rc.cosi), sini = T(rc.sini), i0 = T(rc.i0);
  const T fac = one - T(1.5) * kp * betal * x3thm1;
  const T rk = rl * fac + half * k * x1mth2 * cos2u;
  const T uk = u - T(0.25) * kp * x7thm1 * sin2u;
  const T raank = raan + T(1.5) * kp * cosi * sin2u;
  const T ik = i0 + T(1.5) * kp * cosi * sini * cos2u;
  const T nk = n * k / xke;
  const T rdotk = rdotl - nk * x1mth2 * sin2u;
  const T rfdotk = rfdotl + nk * (x1mth2 * cos2u + T(1.5) * x3thm1);
  T su, cu, sO, cO, si, ci;
  sc(uk, su, cu);
  sc(raank, sO, cO);
  sc(ik, si, ci);
  const T mx = -sO * ci, my = cO * ci, mz = si;
  const T Ux = mx * su + cO * cu, Uy = my * su + sO * cu, Uz = mz * su;
  const T Vx = mx * cu - cO * su, Vy = my * cu - sO * su, Vz = mz * cu;
  const int code = rk < one ? 6 : 0;
  if (r_out) {
    r_out[0] = rk * T(g.re) * Ux;
    r_out[1] = rk * T(g.re) * Uy;
    r_out[2] = rk * T(g.re) * Uz;
  }

  // ------------------------------------------------------------------ reverse
  const T re = T(g.re), vk = T(g.vkmps);
  const T Ubx = rk * re * gr[0] + vk * rdotk * gv[0];
  const T Uby = rk * re * gr[1] + vk * rdotk * gv[1];
  const T Ubz = rk * re * gr[2] + vk * rdotk * gv[2];
  const T Vbx = vk * rfdotk * gv[0], Vby = vk * rfdotk * gv[1], Vbz = vk * rfdotk * gv[2];
  const T rkb = re * (gr[0] * Ux + gr[1] * Uy + gr[2] * Uz);
  const T rdotkb = vk * (gv[0] * Ux + gv[1] * Uy + gv[2] * Uz);
  const T rfdotkb = vk * (gv[0] * Vx + gv[1] * Vy + gv[2] * Vz);
  // U = M su + N cu, V = M cu - N su, M = (mx, my, mz), N = (cO, sO, 0)
  const T Mbx = Ubx * su + Vbx * cu, Mby = Uby * su + Vby * cu, Mbz = Ubz * su + Vbz * cu;
  const T Nbx = Ubx * cu - Vbx * su, Nby = Uby * cu - Vby * su;
  const T sub = Ubx * mx + Uby * my + Ubz * mz - (Vbx * cO + Vby * sO);
  const T cub = Ubx * cO + Uby * sO + (Vbx * mx + Vby * my + Vbz * mz);
  const T sOb = -Mbx * ci + Nby;
  const T cOb = Mby * ci + Nbx;
  const T cib = -Mbx * sO + Mby * cO;
  const T sib = Mbz;
  const T ukb = sub * cu - cub * su;
  const T raankb = sOb * cO - cOb * sO;
  const T ikb = sib * ci - cib * si;
  // rdot_k, rfdot_k
  const T rdotlb = rdotkb, rfdotlb = rfdotkb;
  const T nkb = -rdotkb * x1mth2 * sin2u + rfdotkb * (x1mth2 * cos2u + T(1.5) * x3thm1);
  T x1mth2b = -rdotkb * nk * sin2u + rfdotkb * nk * cos2u;
  T sin2ub = -rdotkb * nk * x1mth2;
  T cos2ub = rfdotkb * nk * x1mth2;
  T x3thm1b = rfdotkb * nk * T(1.5);
  const T nb = nkb * k / xke;
  T kb = nkb * n / xke;
  // i_k, RAAN_k, u_k
  const T i0b = ikb;
  T kpb = ikb * T(1.5) * cosi * sini * cos2u;
  T cosib = ikb * T(1.5) * kp * sini * cos2u;
  const T sinib = ikb * T(1.5) * kp * cosi * cos2u;
  cos2ub += ikb * T(1.5) * kp * cosi * sini;
  const T raanb = raankb;
  kpb += raankb * T(1.5) * cosi * sin2u;
  cosib += raankb * T(1.5) * kp * sin2u;
  sin2ub += raankb * T(1.5) * kp * cosi;
  const T ub = ukb;
  kpb += -ukb * T(0.25) * x7thm1 * sin2u;
  const T x7thm1b = -ukb * T(0.25) * kp * sin2u;
  sin2ub += -ukb * T(0.25) * kp * x7thm1;
  // r_k
  T rlb = rkb * fac;
  kpb += -rkb * rl * T(1.5) * betal * x3thm1;
  T betalb = -rkb * rl * T(1.5) * kp * x3thm1;
  x3thm1b += -rkb * rl * T(1.5) * kp * betal;
  kb += rkb * half * x1mth2 * cos2u;
  x1mth2b += rkb * half * k * cos2u;
  cos2ub += rkb * half * k * x1mth2;
  // kp = k / pL, k = j2 / (2 pL)
  kb += kpb / pL;
  T pLb = -kpb * kp / pL;
  pLb += -kb * k / pL;
  // sin 2u, cos 2u, u = atan2(sin u, cos u)
  T sinub = two * cosu * sin2ub - T(4) * sinu * cos2ub;
  T cosub = two * sinu * sin2ub;
  const T den = sinu * sinu + cosu * cosu;
  sinub += ub * cosu / den;
  cosub += -ub * sinu / den;
  // sin u = aor As, cos u = aor Ac
  const T aorb = sinub * As + cosub * Ac;
  const T Asb = sinub * aor, Acb = cosub * aor;
  T spb = Asb, cpb = Acb;
  T aynb = -Asb + Acb * w;
  T axnb = -Asb * w - Acb;
  const T wb = -Asb * axn + Acb * ayn;
  T ab = aorb / rl;
  rlb += -aorb * aor / rl;
  T esinEb = wb / opb;
  betalb += -wb * w / opb;
  T eL2b = -betalb * half / betal;
  const T sqpb = rfdotlb / rl;
  rlb += -rfdotlb * rfdotl / rl;
  pLb += sqpb * half / sqp;
  T sqab = rdotlb * esinE / rl;
  esinEb += rdotlb * sqa / rl;
  rlb += -rdotlb * rdotl / rl;
  ab += rlb * (one - ecosE);
  const T ecosEb = -rlb * a;
  ab += pLb * (one - eL2);
  eL2b += -pLb * a;
  axnb += two * axn * eL2b;
  aynb += two * ayn * eL2b;
  axnb += esinEb * sp;
  spb += esinEb * axn;
  aynb += -esinEb * cp;
  cpb += -esinEb * ayn;
  axnb += ecosEb * cp;
  cpb += ecosEb * axn;
  aynb += ecosEb * sp;
  spb += ecosEb * ayn;
  // Kepler at its root: psi - axn sin psi + ayn cos psi = U
  const T psib = spb * cp - cpb * sp;
  const T D = one - axn * cp - ayn * sp;
  const T Ub = psib / D;
  axnb += psib * sp / D;
  aynb += -psib * cp / D;
  // U = (M + argp) + q xlcof axn
  const T mpab = Ub;
  T qb = Ub * xlcof * axn;
  const T xlcofb = Ub * q * axn;
  axnb += Ub * q * xlcof;
  // a_yN = e sin argp + q aycof
  T eb = aynb * sw;
  const T swb = aynb * e;
  qb += aynb * aycof;
  const T aycofb = aynb * q;
  // q = 1 / (a (1 - e^2))
  const T qab = -qb * q * q;
  ab += qab * om;
  eb += -two * e * (qab * a);
  // a_xN = e cos argp
  eb += axnb * cw;
  const T cwb = axnb * e;
  const T argpb = swb * cw - cwb * sw;
  // angles: mpa = mm2 + argp1, argp = argp1, raan = raan1 (mod 2 pi)
  const T mm2b = mpab;
  const T argp1b = mpab + argpb;
  const T raan1b = raanb;
  T mm1b = mm2b;
  const T n0ppb = mm2b * templ;
  const T templb = mm2b * T(rc.n0pp);
  const T e1b = clamped ? T(0) : eb;
  const T e0b = e1b;
  const T tempeb = -e1b;
  ab += nb * T(-1.5) * n / a;
  ab += sqab * half / sqa;
  const T a0ppb = ab * tempa * tempa;
  const T tempab = ab * a0pp * two * tempa;
  T mdfb, argpdfb;
  if (!isimp) {
    acc[aL3 * kAdjThreads] += (double)(templb * t3);
    acc[aL4 * kAdjThreads] += (double)(templb * t4);
    acc[aL5 * kAdjThreads] += (double)(templb * t4 * tt);
    acc[aBC5 * kAdjThreads] += (double)(tempeb * (sMM - sinm0));
    const T sMMb = tempeb * bc5;
    acc[aSinM0 * kAdjThreads] += (double)(-tempeb * bc5);
    acc[aD2 * kAdjThreads] += (double)(-tempab * t2);
    acc[aD3 * kAdjThreads] += (double)(-tempab * t3);
    acc[aD4 * kAdjThreads] += (double)(-tempab * t4);
    mm1b += sMMb * cMM;
    mdfb = mm1b;
    argpdfb = argp1b;
    const T dargpb = mm1b - argp1b;
    const T dmb = mm1b - argp1b;
    acc[aMCf * kAdjThreads] += (double)(dmb * (c * c * c - delm0));
    const T cb = dmb * mcf * T(3) * c * c;
    acc[aDelM0 * kAdjThreads] += (double)(-dmb * mcf);
    acc[aEta * kAdjThreads] += (double)(cb * cMdf);
    mdfb += -(cb * eta) * sMdf;
    acc[aArgpCf * kAdjThreads] += (double)(dargpb * tt);
  } else {
    mdfb = mm1b;
    argpdfb = argp1b;
  }
  acc[aL2 * kAdjThreads] += (double)(templb * t2);
  acc[aBC4 * kAdjThreads] += (double)(tempeb * tt);
  acc[aC1 * kAdjThreads] += (double)(-tempab * tt);
  acc[aRaan0 * kAdjThreads] += (double)raan1b;
  acc[aRaandot * kAdjThreads] += (double)raan1b * t;
  acc[aRaanCf * kAdjThreads] += (double)raan1b * t2d;
  acc[aArgp0 * kAdjThreads] += (double)argpdfb;
  acc[aArgpdot * kAdjThreads] += (double)argpdfb * t;
  acc[aM0 * kAdjThreads] += (double)mdfb;
  acc[aMdot * kAdjThreads] += (double)mdfb * t;
  acc[aN0pp * kAdjThreads] += (double)n0ppb;
  acc[aA0pp * kAdjThreads] += (double)a0ppb;
  acc[aE0 * kAdjThreads] += (double)e0b;
  acc[aI0 * kAdjThreads] += (double)i0b;
  acc[aXlcof * kAdjThreads] += (double)xlcofb;
  acc[aAycof * kAdjThreads] += (double)aycofb;
  acc[aCosi * kAdjThreads] += (double)cosib;
  acc[aSini * kAdjThreads] += (double)sinib;
  acc[aX3thm1 * kAdjThreads] += (double)x3thm1b;
  acc[aX1mth2 * kAdjThreads] += (double)x1mth2b;
  acc[aX7thm1 * kAdjThreads] += (double)x7thm1b;
  return code;
}

struct AdjArgs {
  RecordPtrs rp;
  Geo g;
  const double* tsince;
  int64_t T;
  int per_sat;
  const void* grad_r;
  const void* grad_v;
  double* field_bar;   // [n][kNumAdj], workspace
};

template <class T>
__global__ void __launch_bounds__(kAdjThreads) adjoint_prop_kernel(AdjArgs a) {
  __shared__ double acc[kNumAdj * kAdjThreads];
  const int tid = threadIdx.x;
  for (int f = 0; f < kNumAdj; ++f) acc[f * kAdjThreads + tid] = 0.0;
  const int64_t j = blockIdx.x;
  const Rec64 rc = load_rec64(a.rp, j);
  const T* gr = static_cast<const T*>(a.grad_r);
  const T* gv = static_cast<const T*>(a.grad_v);
  for (int64_t i = tid; i < a.T; i += kAdjThreads) {
    const int64_t s = j * a.T + i;
    const double t = a.per_sat ? a.tsince[s] : a.tsince[i];
    T g_r[3], g_v[3];
    for (int c = 0; c < 3; ++c) {
      g_r[c] = gr ? gr[s * 3 + c] : T(0);
      g_v[c] = gv ? gv[s * 3 + c] : T(0);
    }
    adjoint_state<T>(rc, a.g, t, g_r, g_v, acc + tid);
  }
  __syncthreads();
  if (tid < kNumAdj) {
    double sum = 0.0;
    for (int k = 0; k < kAdjThreads; ++k) sum += acc[tid * kAdjThreads + k];
    a.field_bar[j * kNumAdj + tid] = sum;
  }
}

__global__ void __launch_bounds__(64) adjoint_init_kernel(const double* __restrict__ el,
                                                          const double* __restrict__ field_bar,
                                                          int64_t n, Geo g,
                                                          double* __restrict__ grad) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double e7[7];
  bool ok = true;
  for (int k = 0; k < 7; ++k) {
    e7[k] = el[j * 7 + k];
    ok = ok && isfinite(e7[k]);
  }
  ok = ok && e7[1] >= 0.0 && e7[1] < 1.0 && e7[0] > 0.0;
  if (!ok) {
    for (int k = 0; k < 7; ++k) grad[j * 7 + k] = 0.0;
    return;
  }
  D7 x[7];
  for (int k = 0; k < 7; ++k) x[k] = d7var(e7[k], k);
  InitFields<D7> o;
  init_fields(x, g, o);
  const D7* f[kNumAdj] = {&o.n0pp, &o.a0pp, &o.e0, &o.i0, &o.raan0, &o.argp0, &o.m0,
                          &o.mdot, &o.argpdot, &o.raandot, &o.raan_cf, &o.argp_cf, &o.m_cf,
                          &o.c1, &o.bc4, &o.bc5, &o.d2, &o.d3, &o.d4, &o.l2, &o.l3, &o.l4,
                          &o.l5, &o.eta, &o.delm0, &o.sinm0, &o.xlcof, &o.aycof, &o.cosi,
                          &o.sini, &o.x3thm1, &o.x1mth2, &o.x7thm1};
  double out[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int q = 0; q < kNumAdj; ++q) {
    const double b = field_bar[j * kNumAdj + q];
    for (int k = 0; k < 7; ++k) out[k] += b * f[q]->d[k];
  }
  for (int k = 0; k < 7; ++k) grad[j * 7 + k] = out[k];
}

// Record-field Jacobian of sgp4init, d(field)/d(element), [kNumAdj][7], by dual
// numbers (false for unusable elements).
__device__ bool init_jacobian(const double e7[7], const Geo& g, double J[kNumAdj][7]) {
  bool ok = true;
  for (int k = 0; k < 7; ++k) ok = ok && isfinite(e7[k]);
  ok = ok && e7[1] >= 0.0 && e7[1] < 1.0 && e7[0] > 0.0;
  if (!ok) return false;
  D7 x[7];
  for (int k = 0; k < 7; ++k) x[k] = d7var(e7[k], k);
  InitFields<D7> o;
  init_fields(x, g, o);
  const D7* f[kNumAdj] = {&o.n0pp, &o.a0pp, &o.e0, &o.i0, &o.raan0, &o.argp0, &o.m0,
                          &o.mdot, &o.argpdot, &o.raandot, &o.raan_cf, &o.argp_cf, &o.m_cf,
                          &o.c1, &o.bc4, &o.bc5, &o.d2, &o.d3, &o.d4, &o.l2, &o.l3, &o.l4,
                          &o.l5, &o.eta, &o.delm0, &o.sinm0, &o.xlcof, &o.aycof, &o.cosi,
                          &o.sini, &o.x3thm1, &o.x1mth2, &o.x7thm1};
  for (int q = 0; q < kNumAdj; ++q)
    for (int k = 0; k < 7; ++k) J[q][k] = f[q]->d[k];
  return true;
}

struct FitArgs {
  RecordPtrs rp;
  Geo g;
  const double* el;      // [n][7]
  const double* tsince;
  int64_t T;
  int per_sat;
  const double* r_obs;   // [n][T][3]
  const double* lambda;  // [n] Levenberg-Marquardt damping
  double* el_out;        // [n][7]
  double* sse;           // [n] sum of squared position residuals at el (km^2)
};

// One Gauss-Newton / Levenberg-Marquardt step of batch least squares per satellite:
// residuals res_t = r_t(el) - r_obs_t over the states with finite output, the
// position Jacobian J_t = dr_t/del (three reverse sweeps per state, contracted with
// the init Jacobian), A = sum J_t^T J_t, b = sum J_t^T res_t, and the step
// delta = -(A + lambda diag A)^-1 b solved by Cholesky on the Jacobi-scaled matrix.
template <class T>
__global__ void __launch_bounds__(kAdjThreads) fit_step_kernel(FitArgs a) {
  __shared__ double acc[kNumAdj * kAdjThreads];
  __shared__ double Ji[kNumAdj][7];
  __shared__ double red[36][kAdjThreads / 32];
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  const int64_t j = blockIdx.x;
  double e7[7];
  for (int k = 0; k < 7; ++k) e7[k] = a.el[j * 7 + k];
  if (tid == 0) s_ok = init_jacobian(e7, a.g, Ji) ? 1 : 0;
  __syncthreads();
  if (!s_ok) {
    if (tid < 7) a.el_out[j * 7 + tid] = e7[tid];
    if (tid == 0) a.sse[j] = 0.0;
    return;
  }
  const Rec64 rc = load_rec64(a.rp, j);
  double A[28], b[7], sse = 0.0;
  for (int k = 0; k < 28; ++k) A[k] = 0.0;
  for (int k = 0; k < 7; ++k) b[k] = 0.0;
  const T zero3[3] = {T(0), T(0), T(0)};
  for (int64_t i = tid; i < a.T; i += kAdjThreads) {
    const int64_t s = j * a.T + i;
    const double t = a.per_sat ? a.tsince[s] : a.tsince[i];
    double Jt[3][7];
    T r[3];
    int code = 0;
    for (int c = 0; c < 3; ++c) {
      for (int f = 0; f < kNumAdj; ++f) acc[f * kAdjThreads + tid] = 0.0;
      T seed[3] = {T(0), T(0), T(0)};
      seed[c] = T(1);
      code = adjoint_state<T>(rc, a.g, t, seed, zero3, acc + tid, r);
      for (int k = 0; k < 7; ++k) {
        double v = 0.0;
        for (int f = 0; f < kNumAdj; ++f) v += acc[f * kAdjThreads + tid] * Ji[f][k];
        Jt[c][k] = v;
      }
    }
    if (code != 0 && code != 6) continue;
    double res[3];
    for (int c = 0; c < 3; ++c) res[c] = (double)r[c] - a.r_obs[s * 3 + c];
    if (!(isfinite(res[0]) && isfinite(res[1]) && isfinite(res[2]))) continue;
    sse += res[0] * res[0] + res[1] * res[1] + res[2] * res[2];
    int q = 0;
    for (int k = 0; k < 7; ++k) {
      b[k] += Jt[0][k] * res[0] + Jt[1][k] * res[1] + Jt[2][k] * res[2];
      for (int m = 0; m <= k; ++m, ++q)
        A[q] += Jt[0][k] * Jt[0][m] + Jt[1][k] * Jt[1][m] + Jt[2][k] * Jt[2][m];
    }
  }
  // Block reduction of the 28 + 7 + 1 sums (warp shuffles, then one value per warp).
  double vals[36];
  for (int k = 0; k < 28; ++k) vals[k] = A[k];
  for (int k = 0; k < 7; ++k) vals[28 + k] = b[k];
  vals[35] = sse;
  const int lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < 36; ++k) {
    double v = vals[k];
    for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (tid != 0) return;
  double S[36];
  for (int k = 0; k < 36; ++k) {
    double v = 0.0;
    for (int w = 0; w < kAdjThreads / 32; ++w) v += red[k][w];
    S[k] = v;
  }
  // Unpack A (lower triangle), Jacobi scaling, damping, Cholesky.
  double M[7][7], rhs[7], d[7];
  int q = 0;
  for (int k = 0; k < 7; ++k)
    for (int m = 0; m <= k; ++m, ++q) M[k][m] = M[m][k] = S[q];
  for (int k = 0; k < 7; ++k) d[k] = M[k][k] > 0.0 ? 1.0 / sqrt(M[k][k]) : 0.0;
  const double lam = a.lambda[j];
  for (int k = 0; k < 7; ++k) {
    for (int m = 0; m < 7; ++m) M[k][m] *= d[k] * d[m];
    M[k][k] = (d[k] > 0.0 ? M[k][k] : 1.0) * (1.0 + lam);
    rhs[k] = -S[28 + k] * d[k];
  }
  bool spd = true;
  for (int k = 0; k < 7 && spd; ++k) {
    for (int m = 0; m < k; ++m) M[k][k] -= M[k][m] * M[k][m];
    if (!(M[k][k] > 0.0)) { spd = false; break; }
    M[k][k] = sqrt(M[k][k]);
    for (int r2 = k + 1; r2 < 7; ++r2) {
      for (int m = 0; m < k; ++m) M[r2][k] -= M[r2][m] * M[k][m];
      M[r2][k] /= M[k][k];
    }
  }
  double x[7] = {0, 0, 0, 0, 0, 0, 0};
  if (spd) {
    for (int k = 0; k < 7; ++k) {            // forward substitution L y = rhs
      double v = rhs[k];
      for (int m = 0; m < k; ++m) v -= M[k][m] * x[m];
      x[k] = v / M[k][k];
    }
    for (int k = 6; k >= 0; --k) {           // back substitution L^T x = y
      double v = x[k];
      for (int m = k + 1; m < 7; ++m) v -= M[m][k] * x[m];
      x[k] = v / M[k][k];
    }
  }
  for (int k = 0; k < 7; ++k) a.el_out[j * 7 + k] = e7[k] + x[k] * d[k];
  a.sse[j] = S[35];
}

}  // namespace

cudaError_t launch_fit_step(const RecordPtrs& rp, const Geo& g, const double* el,
                            const double* tsince, int64_t T, int per_sat, bool fp32,
                            const double* r_obs, const double* lambda, double* el_out,
                            double* sse, cudaStream_t stream) {
  if (rp.n == 0) return cudaSuccess;
  FitArgs a;
  a.rp = rp;
  a.g = g;
  a.el = el;
  a.tsince = tsince;
  a.T = T;
  a.per_sat = per_sat;
  a.r_obs = r_obs;
  a.lambda = lambda;
  a.el_out = el_out;
  a.sse = sse;
  if (fp32) fit_step_kernel<float><<<(unsigned)rp.n, kAdjThreads, 0, stream>>>(a);
  else fit_step_kernel<double><<<(unsigned)rp.n, kAdjThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

size_t adjoint_workspace_bytes(int64_t n) {
  return n <= 0 ? 0 : (size_t)n * kNumAdj * sizeof(double);
}

cudaError_t launch_adjoint(const RecordPtrs& rp, const Geo& g, const double* el,
                           const double* tsince, int64_t T, int per_sat, bool fp32,
                           const void* grad_r, const void* grad_v, double* grad_el,
                           double* workspace, cudaStream_t stream) {
  if (rp.n == 0) return cudaSuccess;
  AdjArgs a;
  a.rp = rp;
  a.g = g;
  a.tsince = tsince;
  a.T = T;
  a.per_sat = per_sat;
  a.grad_r = grad_r;
  a.grad_v = grad_v;
  a.field_bar = workspace;
  if (fp32) adjoint_prop_kernel<float><<<(unsigned)rp.n, kAdjThreads, 0, stream>>>(a);
  else adjoint_prop_kernel<double><<<(unsigned)rp.n, kAdjThreads, 0, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int threads = 64;
  adjoint_init_kernel<<<(unsigned)((rp.n + threads - 1) / threads), threads, 0, stream>>>(
      el, workspace, rp.n, g, grad_el);
  return cudaGetLastError();
}

}  // namespace sgp4
