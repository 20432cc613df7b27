// Record builder: one thread per satellite computes the initialisation constants of
// near-Earth SGP4 (paper Sec. 2.1; Spacetrack Report #3 "initialization", 2006
// revision) in FP64 and writes them as structure-of-arrays planes, plus the FP32 /
// double-float row of the mixed-precision path and the init status.
#include <cmath>

#include "sgp4_device.cuh"
#include "sgp4_init_math.cuh"
#include "sgp4_kernels.cuh"

namespace sgp4 {

namespace {

// Satellites per 32-lane warp.  The record build is bound by B300's small FP64 unit,
// which works through the active lanes of a warp instruction; a Starlink-sized set
// (9,341) fills only half of the SM sub-partitions at 32 per warp, so fewer
// satellites per warp spread the same FP64 work over all of them.
#ifndef SGP4_INIT_LANES
#define SGP4_INIT_LANES 32
#endif

__global__ void __launch_bounds__(32) init_kernel(const double* __restrict__ el,
                                                   const int32_t* __restrict__ epoch_day,
                                                   const double* __restrict__ epoch_frac,
                                                   RecordPtrs rp, Geo g, GeoF gf,
                                                   int32_t* __restrict__ init_status) {
  if (threadIdx.x >= SGP4_INIT_LANES) return;
  const int64_t j = (int64_t)blockIdx.x * SGP4_INIT_LANES + threadIdx.x;
  if (j >= rp.n) return;
  const int64_t s = rp.stride;
  double* f = rp.f64;
  float* h = rp.f32 + j * kF32Row;   // this satellite's FP32 row

  const double n0 = el[j * 7 + 0], e0 = el[j * 7 + 1], i0 = el[j * 7 + 2];
  const double raan0 = el[j * 7 + 3], argp0 = el[j * 7 + 4], m0 = el[j * 7 + 5];
  const double bstar = el[j * 7 + 6];
  rp.epoch_day[j] = epoch_day ? epoch_day[j] : 0;
  f[kEpochFrac * s + j] = epoch_frac ? epoch_frac[j] : 0.0;

  // Input validity (fatal for the record): non-finite or e0 outside [0,1) -> 1,
  // n0 <= 0 -> 2.
  int fatal = 0;
  bool finite = isfinite(n0) && isfinite(e0) && isfinite(i0) && isfinite(raan0) &&
                isfinite(argp0) && isfinite(m0) && isfinite(bstar);
  if (!finite || e0 < 0.0 || e0 >= 1.0) fatal = 1;
  else if (n0 <= 0.0) fatal = 2;
  if (fatal) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int k = 0; k < kEpochFrac; ++k) f[k * s + j] = nan;
    for (int k = 0; k < kF32Row; ++k) h[k] = __int_as_float(0x7fc00000);
    h[fFlags] = __int_as_float(fatal << kFatalShift);
    rp.flags[j] = fatal << kFatalShift;
    init_status[j] = fatal;
    return;
  }

  InitFields<double> o;
  {
    const double e7[7] = {n0, e0, i0, raan0, argp0, m0, bstar};
    init_fields(e7, g, o);
  }
  const double n0pp = o.n0pp, a0pp = o.a0pp, mdot = o.mdot, argpdot = o.argpdot;
  const double raandot = o.raandot, raan_cf = o.raan_cf, argp_cf = o.argp_cf, m_cf = o.m_cf;
  const double C1 = o.c1, bc4 = o.bc4, bc5 = o.bc5, D2 = o.d2, D3 = o.d3, D4 = o.d4;
  const double L2 = o.l2, L3 = o.l3, L4 = o.l4, L5 = o.l5, eta = o.eta, delm0 = o.delm0;
  const double sinm0 = o.sinm0, xlcof = o.xlcof, aycof = o.aycof, cosi = o.cosi, sini = o.sini;
  const double x3thm1 = o.x3thm1, x1mth2 = o.x1mth2, x7thm1 = o.x7thm1;
  const bool isimp = o.isimp;

  // FP64 planes.
  f[kN0pp * s + j] = n0pp;     f[kA0pp * s + j] = a0pp;     f[kE0 * s + j] = e0;
  f[kI0 * s + j] = i0;         f[kRaan0 * s + j] = raan0;   f[kArgp0 * s + j] = argp0;
  f[kM0 * s + j] = m0;         f[kBstar * s + j] = bstar;   f[kMdot * s + j] = mdot;
  f[kArgpdot * s + j] = argpdot; f[kRaandot * s + j] = raandot; f[kRaanCf * s + j] = raan_cf;
  f[kArgpCf * s + j] = argp_cf;  f[kMCf * s + j] = m_cf;     f[kC1 * s + j] = C1;
  f[kBC4 * s + j] = bc4;       f[kBC5 * s + j] = bc5;       f[kD2 * s + j] = D2;
  f[kD3 * s + j] = D3;         f[kD4 * s + j] = D4;         f[kL2 * s + j] = L2;
  f[kL3 * s + j] = L3;         f[kL4 * s + j] = L4;         f[kL5 * s + j] = L5;
  f[kEta * s + j] = eta;       f[kDelM0 * s + j] = delm0;   f[kSinM0 * s + j] = sinm0;
  f[kXlcof * s + j] = xlcof;   f[kAycof * s + j] = aycof;   f[kCosi * s + j] = cosi;
  f[kSini * s + j] = sini;     f[kX3thm1 * s + j] = x3thm1; f[kX1mth2 * s + j] = x1mth2;
  f[kX7thm1 * s + j] = x7thm1;

  // FP32 row: angles in revolutions, the argument-of-latitude phase as double-float.
  // Conversions to float by integer operations (f32_rn, split_double): this kernel is
  // bound by the FP64 unit, where each conversion instruction would cost a DFMA.
  const double inv2pi = 1.0 / kTwoPi;
  double phi0 = (m0 + argp0) * inv2pi;
  phi0 -= floor(phi0);
  float hi, lo;
  split_double(phi0, hi, lo);
  h[fPhi0H] = hi; h[fPhi0L] = lo;
  split_double((mdot + argpdot) * inv2pi, hi, lo);
  h[fPhiDH] = hi; h[fPhiDL] = lo;
  double m0r = m0 * inv2pi;       m0r -= floor(m0r);
  double argp0r = argp0 * inv2pi; argp0r -= floor(argp0r);
  double raan0r = raan0 * inv2pi; raan0r -= floor(raan0r);
  h[fM0r] = f32_rn(m0r);
  h[fMdr] = f32_rn(mdot * inv2pi);
  h[fArgp0r] = f32_rn(argp0r);
  h[fArgpdr] = f32_rn(argpdot * inv2pi);
  h[fRaan0r] = f32_rn(raan0r);
  h[fRaandr] = f32_rn(raandot * inv2pi);
  h[fRaanCfr] = f32_rn(raan_cf * inv2pi);
  h[fN0ppr] = f32_rn(n0pp * inv2pi);
  h[fA0pp] = f32_rn(a0pp);   h[fE0] = f32_rn(e0);     h[fC1] = f32_rn(C1);
  h[fBC4] = f32_rn(bc4);     h[fBC5] = isimp ? 0.0f : f32_rn(bc5);   h[fD2] = f32_rn(D2);
  h[fD3] = f32_rn(D3);       h[fD4] = f32_rn(D4);     h[fL2] = f32_rn(L2);
  h[fL3] = f32_rn(L3);       h[fL4] = f32_rn(L4);     h[fL5] = f32_rn(L5);
  h[fEta] = f32_rn(eta);     h[fDelM0] = f32_rn(delm0); h[fSinM0] = f32_rn(sinm0);
  // Simplified-drag records (perigee below 220 km) drop the drag terms these three
  // carry: zero in the FP32 row, so that the FP32 state evaluates the drag block
  // unconditionally (no branch) and gets the theory's zero contributions.
  h[fArgpCf] = isimp ? 0.0f : f32_rn(argp_cf);
  h[fMCf] = isimp ? 0.0f : f32_rn(m_cf);
  h[fXlcof] = f32_rn(xlcof); h[fAycof] = f32_rn(aycof);
  h[fCosi] = f32_rn(cosi);   h[fSini] = f32_rn(sini);
  h[fX3thm1] = f32_rn(1.5 * x3thm1); h[fX1mth2] = f32_rn(x1mth2);
  h[fX7thm1] = f32_rn(-0.25 * x7thm1);
  h[fHalfX1mth2] = f32_rn(0.5 * x1mth2);
  h[fC15Cosi] = f32_rn(1.5 * cosi);
  h[fC15CosiSini] = f32_rn(1.5 * cosi * sini);

  int flags = 0;
  if (isimp) flags |= kFlagIsimp;
  if (n0pp <= 0.0) flags |= kFlagN0ppNonPos;
  rp.flags[j] = flags;
  h[fFlags] = __int_as_float(flags);
  for (int k = kNumF32Used; k < kF32Row; ++k) h[k] = 0.0f;

  // Init status: the status of the state at tsince = 0, from the FP32 state with
  // its FP64 recomputation inside the guard bands (so it equals the FP64 decision).
  {
    const Rec32 r32 = read_own_rec32(h);
    float r[3], v[3];
    const int code = state32(r32, gf, 0.0f, 0.0f, r, v);
    if (code != kRecomputeFP64) {
      init_status[j] = code;
      return;
    }
  }
  Rec64 rc;
  rc.n0pp = n0pp; rc.a0pp = a0pp; rc.e0 = e0; rc.i0 = i0; rc.raan0 = raan0; rc.argp0 = argp0;
  rc.m0 = m0; rc.mdot = mdot; rc.argpdot = argpdot; rc.raandot = raandot; rc.raan_cf = raan_cf;
  rc.argp_cf = argp_cf; rc.m_cf = m_cf; rc.c1 = C1; rc.bc4 = bc4; rc.bc5 = bc5; rc.d2 = D2;
  rc.d3 = D3; rc.d4 = D4; rc.l2 = L2; rc.l3 = L3; rc.l4 = L4; rc.l5 = L5; rc.eta = eta;
  rc.delm0 = delm0; rc.sinm0 = sinm0; rc.xlcof = xlcof; rc.aycof = aycof; rc.cosi = cosi;
  rc.sini = sini; rc.x3thm1 = x3thm1; rc.x1mth2 = x1mth2; rc.x7thm1 = x7thm1; rc.flags = flags;
  double r[3], v[3];
  init_status[j] = state64(rc, g, 0.0, r, v);
}

}  // namespace

cudaError_t launch_init(const double* el, const int32_t* epoch_day, const double* epoch_frac,
                        const RecordPtrs& rp, const Geo& g, int32_t* init_status,
                        cudaStream_t stream) {
  if (rp.n == 0) return cudaSuccess;
  const int threads = 32;
  const int64_t blocks = (rp.n + SGP4_INIT_LANES - 1) / SGP4_INIT_LANES;
  init_kernel<<<(unsigned)blocks, threads, 0, stream>>>(el, epoch_day, epoch_frac, rp, g,
                                                        geo_float(g), init_status);
  return cudaGetLastError();
}

}  // namespace sgp4
