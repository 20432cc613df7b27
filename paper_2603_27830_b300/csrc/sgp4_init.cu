// Record builder: one thread per satellite computes the initialisation constants of
// near-Earth SGP4 (paper Sec. 2.1; Spacetrack Report #3 "initialization", 2006
// revision) in FP64 and writes them as structure-of-arrays planes, plus the FP32 /
// double-float row of the mixed-precision path and the init status.
#include <cmath>

#include "sgp4_deep.cuh"
#include "sgp4_device.cuh"
#include "sgp4_init_math.cuh"
#include "sgp4_kernels.cuh"

#ifndef SGP4_INIT_SPLIT_BLOCKS
#define SGP4_INIT_SPLIT_BLOCKS 592
#endif

namespace sgp4 {

namespace {

// Named barrier `id` over `n` threads (a multiple of 32): arrive without waiting, or
// wait for all n.  Every thread of both warps of a block reaches them, whatever its
// satellite's state.
__device__ __forceinline__ void named_barrier_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_barrier_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// 32 satellites per block.  With kSplit, two warps share them: a lone warp on a
// sub-partition issues one FP64 instruction per ~64 cycles, so for small catalogues
// (fewer warps than sub-partitions) the record build takes as long as its longest chain
// of FP64 instructions.  The computation's two independent branches then run in
// different warps: warp 0 the spine (un-Kozai, a0'') and then the drag terms, warp 1 the
// sin/cos of argp0 and M0 and then the secular rates; they meet in shared memory.  For
// large catalogues the FP64 unit is saturated anyway and one warp does both branches
// (no duplicated loads and exchanges).
constexpr int kInitSats = 32;

template <bool kSplit>
__global__ void __launch_bounds__(kSplit ? 64 : 32) init_kernel(const double* __restrict__ el,
                                                   const int32_t* __restrict__ epoch_day,
                                                   const double* __restrict__ epoch_frac,
                                                   RecordPtrs rp, Geo g, GeoF gf,
                                                   int32_t* __restrict__ init_status) {
  __shared__ double sh_sp[12][kInitSats];     // InitSpine
  __shared__ double sh_an[4][kInitSats];      // InitAngles
  __shared__ double sh_x[2][kInitSats];       // C1 (drag), first-order node rate (rates)
  __shared__ double sh_dc[7][kInitSats];      // DragCore (warp 0 -> warp 1)
  __shared__ double sh_sa[6][kInitSats];      // SpineA (warp 1 -> warp 0)
  // A propagation launched after this build as its programmatic dependent may be
  // scheduled now; it waits for this grid's completion before reading the records.
  asm volatile("griddepcontrol.launch_dependents;");
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const bool w0 = !kSplit || w == 0;   // this thread runs the spine / drag branch
  const bool w1 = !kSplit || w == 1;   // this thread runs the angles / rates branch
  const int64_t j = (int64_t)blockIdx.x * kInitSats + lane;
  const bool live = j < rp.n;
  const int64_t s = rp.stride;
  double* f = rp.f64;
  float* h = rp.f32 + j * kF32Row;   // this satellite's FP32 row

  double e7[7] = {0, 0, 0, 0, 0, 0, 0};
  if (live)
    for (int k = 0; k < 7; ++k) e7[k] = el[j * 7 + k];
  const double n0 = e7[0], e0 = e7[1], i0 = e7[2], raan0 = e7[3], argp0 = e7[4], m0 = e7[5];
  const double bstar = e7[6];

  // Input validity (fatal for the record): non-finite or e0 outside [0,1) -> 1,
  // n0 <= 0 -> 2.
  int fatal = 0;
  bool finite = isfinite(n0) && isfinite(e0) && isfinite(i0) && isfinite(raan0) &&
                isfinite(argp0) && isfinite(m0) && isfinite(bstar);
  if (!finite || e0 < 0.0 || e0 >= 1.0) fatal = 1;
  else if (n0 <= 0.0) fatal = 2;
  const bool run = live && !fatal;

  if (live && w1) {
    rp.epoch_day[j] = epoch_day ? epoch_day[j] : 0;
    f[kEpochFrac * s + j] = epoch_frac ? epoch_frac[j] : 0.0;
  }
  if (live && fatal && w0) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int k = 0; k < kEpochFrac; ++k) f[k * s + j] = nan;
    for (int k = 0; k < kF32Row; ++k) h[k] = __int_as_float(0x7fc00000);
    h[fFlags] = __int_as_float(fatal << kFatalShift);
    rp.flags[j] = fatal << kFatalShift;
    init_status[j] = fatal;
  }

  // Phase 1: the spine (warp 0, its n0 / e0 terms from warp 1) and the angles (warp 1).
  InitSpine<double> sp;
  InitAngles<double> an;
  if constexpr (kSplit) {
    // warp 1: the spine's terms in n0 and e0, published on named barrier 2, then the
    // angles; warp 0: the inclination terms, then (barrier 2) the Kozai recovery
    SpineA<double> sa;
    if (w1) {
      if (run) {
        init_spine_a(e7, g, sa);
        sh_sa[0][lane] = sa.n0k; sh_sa[1][lane] = sa.x1; sh_sa[2][lane] = sa.a1;
        sh_sa[3][lane] = sa.b2;  sh_sa[4][lane] = sa.rb; sh_sa[5][lane] = sa.b;
      }
      __threadfence_block();
      named_barrier_arrive(2, 2 * kInitSats);
      if (run) init_angles(e7, an);
    } else {
      if (run) init_spine_i(e7, sp);
      named_barrier_sync(2, 2 * kInitSats);
      if (run) {
        sa.n0k = sh_sa[0][lane]; sa.x1 = sh_sa[1][lane]; sa.a1 = sh_sa[2][lane];
        sa.b2 = sh_sa[3][lane];  sa.rb = sh_sa[4][lane]; sa.b = sh_sa[5][lane];
        init_spine_b(e7, g, sa, sp);
      }
    }
  } else if (run) {
    init_spine(e7, g, sp);
    init_angles(e7, an);
  }
  if constexpr (kSplit) {
    if (run && w0) {
      const double v[12] = {sp.cosi, sp.sini, sp.th2, sp.x3thm1, sp.x1mth2, sp.x7thm1,
                            sp.b2, sp.rb, sp.b, sp.n0pp, sp.a0pp, sp.ia0pp};
      for (int k = 0; k < 12; ++k) sh_sp[k][lane] = v[k];
    }
    if (run && w1) {
      sh_an[0][lane] = an.sinw; sh_an[1][lane] = an.cosw;
      sh_an[2][lane] = an.sinm; sh_an[3][lane] = an.cosm;
    }
    __syncthreads();
  }
  if (kSplit && run) {
    if (w == 0) {
      an.sinw = sh_an[0][lane]; an.cosw = sh_an[1][lane];
      an.sinm = sh_an[2][lane]; an.cosm = sh_an[3][lane];
    } else {
      sp.cosi = sh_sp[0][lane]; sp.sini = sh_sp[1][lane]; sp.th2 = sh_sp[2][lane];
      sp.x3thm1 = sh_sp[3][lane]; sp.x1mth2 = sh_sp[4][lane]; sp.x7thm1 = sh_sp[5][lane];
      sp.b2 = sh_sp[6][lane]; sp.rb = sh_sp[7][lane]; sp.b = sh_sp[8][lane];
      sp.n0pp = sh_sp[9][lane]; sp.a0pp = sh_sp[10][lane]; sp.ia0pp = sh_sp[11][lane];
    }
  }

  // Phase 2: drag terms and secular rates, each branch writing its own fields to the
  // FP64 planes and the FP32 row.  Warp 0: the drag core (atmosphere, xi, eta, the C
  // factors), published through shared memory with a non-blocking arrival on named
  // barrier 1, then C1 and the D / L coefficients.  Warp 1: the secular rates, then
  // (after barrier 1) C3, C4, C5 and their terms, which nothing of warp 0's needs.
  // FP32 conversions by integer operations (f32_rn, split_double): an FP64-unit
  // conversion would cost as much as a DFMA.
  const double inv2pi = 1.0 / kTwoPi;
  InitFields<double> o = {};
  DragCore<double> dc = {};
  auto store_c = [&]() {   // C3 .. C5 terms (simplified drag: zero in the FP32 row)
    const bool isimp = dc.isimp;
    f[kArgpCf * s + j] = o.argp_cf; f[kMCf * s + j] = o.m_cf;
    f[kBC4 * s + j] = o.bc4;       f[kBC5 * s + j] = o.bc5;
    h[fBC4] = f32_rn(o.bc4);
    h[fBC5] = isimp ? 0.0f : f32_rn(o.bc5);
    h[fArgpCf] = isimp ? 0.0f : f32_rn(o.argp_cf);
    h[fMCf] = isimp ? 0.0f : f32_rn(o.m_cf);
  };
  if (w0) {
    if (run) init_drag_core(e7, g, sp, dc);
    if constexpr (kSplit) {
      if (run) {
        sh_dc[0][lane] = dc.ss;    sh_dc[1][lane] = dc.xi;    sh_dc[2][lane] = dc.eta;
        sh_dc[3][lane] = dc.ipsi2; sh_dc[4][lane] = dc.coef;  sh_dc[5][lane] = dc.coef1;
        sh_dc[6][lane] = dc.isimp ? 1.0 : 0.0;
      }
      __threadfence_block();
      named_barrier_arrive(1, 2 * kInitSats);
    }
    if (run) {
      if (!kSplit) {   // one warp: the C terms first (measured 6% faster than after)
        init_drag_c(e7, g, sp, an, dc, o);
        store_c();
      }
      init_drag_d(e7, g, sp, an, dc, o);
      if (kSplit) sh_x[0][lane] = o.c1;
      const bool isimp = dc.isimp;
      f[kN0pp * s + j] = sp.n0pp;  f[kA0pp * s + j] = sp.a0pp;  f[kE0 * s + j] = e0;
      f[kI0 * s + j] = i0;         f[kRaan0 * s + j] = raan0;   f[kArgp0 * s + j] = argp0;
      f[kM0 * s + j] = m0;         f[kBstar * s + j] = bstar;   f[kC1 * s + j] = o.c1;
      f[kD2 * s + j] = o.d2;       f[kD3 * s + j] = o.d3;       f[kD4 * s + j] = o.d4;
      f[kL2 * s + j] = o.l2;       f[kL3 * s + j] = o.l3;       f[kL4 * s + j] = o.l4;
      f[kL5 * s + j] = o.l5;       f[kEta * s + j] = o.eta;     f[kDelM0 * s + j] = o.delm0;
      f[kSinM0 * s + j] = o.sinm0; f[kCosi * s + j] = sp.cosi;  f[kSini * s + j] = sp.sini;
      f[kX3thm1 * s + j] = sp.x3thm1; f[kX1mth2 * s + j] = sp.x1mth2;
      f[kX7thm1 * s + j] = sp.x7thm1;
      h[fA0pp] = f32_rn(sp.a0pp); h[fE0] = f32_rn(e0);     h[fC1] = f32_rn(o.c1);
      h[fD2] = f32_rn(o.d2);     h[fD3] = f32_rn(o.d3);     h[fD4] = f32_rn(o.d4);
      h[fL2] = f32_rn(o.l2);     h[fL3] = f32_rn(o.l3);     h[fL4] = f32_rn(o.l4);
      h[fL5] = f32_rn(o.l5);     h[fEta] = f32_rn(o.eta);   h[fDelM0] = f32_rn(o.delm0);
      h[fSinM0] = f32_rn(o.sinm0);
      h[fCosi] = f32_rn(sp.cosi); h[fSini] = f32_rn(sp.sini);
      h[fX3thm1] = f32_rn(1.5 * sp.x3thm1); h[fX1mth2] = f32_rn(sp.x1mth2);
      h[fX7thm1] = f32_rn(-0.25 * sp.x7thm1);
      h[fHalfX1mth2] = f32_rn(0.5 * sp.x1mth2);
      h[fC15Cosi] = f32_rn(1.5 * sp.cosi);
      h[fC15CosiSini] = f32_rn(1.5 * sp.cosi * sp.sini);
      int flags = 0;
      if (isimp) flags |= kFlagIsimp;
      if (sp.n0pp <= 0.0) flags |= kFlagN0ppNonPos;
      if (is_deep(sp.n0pp)) {
        const int rez = resonance_class(sp.n0pp, e0);
        flags |= kFlagDeep | (rez == 1 ? kFlagRez1 : 0) | (rez == 2 ? kFlagRez2 : 0);
        h[fA0pp] = __int_as_float(0x7fc00000);   // NaN: every FP32 state goes to FP64
      }
      rp.flags[j] = flags;
      h[fFlags] = __int_as_float(flags);
      for (int k = kNumF32Used; k < kF32Row; ++k) h[k] = 0.0f;
    }
  }
  if (w1) {
    if (run) {
      init_rates(g, sp, o);
      if (kSplit) sh_x[1][lane] = o.raandot1;
      f[kMdot * s + j] = o.mdot;   f[kArgpdot * s + j] = o.argpdot;
      f[kRaandot * s + j] = o.raandot;
      f[kXlcof * s + j] = o.xlcof; f[kAycof * s + j] = o.aycof;
      // FP32 row: angles in revolutions, the argument-of-latitude phase as double-float.
      double phi0 = (m0 + argp0) * inv2pi;
      phi0 -= floor(phi0);
      float hi, lo;
      split_double(phi0, hi, lo);
      h[fPhi0H] = hi; h[fPhi0L] = lo;
      split_double((o.mdot + o.argpdot) * inv2pi, hi, lo);
      h[fPhiDH] = hi; h[fPhiDL] = lo;
      double m0r = m0 * inv2pi;       m0r -= floor(m0r);
      double argp0r = argp0 * inv2pi; argp0r -= floor(argp0r);
      double raan0r = raan0 * inv2pi; raan0r -= floor(raan0r);
      h[fM0r] = f32_rn(m0r);
      h[fMdr] = f32_rn(o.mdot * inv2pi);
      h[fArgp0r] = f32_rn(argp0r);
      h[fArgpdr] = f32_rn(o.argpdot * inv2pi);
      h[fRaan0r] = f32_rn(raan0r);
      h[fRaandr] = f32_rn(o.raandot * inv2pi);
      h[fN0ppr] = f32_rn(sp.n0pp * inv2pi);
      h[fXlcof] = f32_rn(o.xlcof); h[fAycof] = f32_rn(o.aycof);
    }
    if constexpr (kSplit) {
      named_barrier_sync(1, 2 * kInitSats);   // warp 0's drag core is in shared memory
      if (run) {
        dc.ss = sh_dc[0][lane];    dc.xi = sh_dc[1][lane];   dc.eta = sh_dc[2][lane];
        dc.ipsi2 = sh_dc[3][lane]; dc.coef = sh_dc[4][lane]; dc.coef1 = sh_dc[5][lane];
        dc.isimp = sh_dc[6][lane] != 0.0;
        init_drag_c(e7, g, sp, an, dc, o);
        store_c();
      }
    }
  }
  if constexpr (kSplit) __syncthreads();

  // Phase 3: the node drag term (C1 from the drag branch, the node rate from the rates
  // branch).
  if (run && w1) {
    const double raan_cf =
        kSplit ? 3.5 * sp.b2 * sh_x[1][lane] * sh_x[0][lane] : 3.5 * sp.b2 * o.raandot1 * o.c1;
    f[kRaanCf * s + j] = raan_cf;
    h[fRaanCfr] = f32_rn(raan_cf * inv2pi);
  }
  if constexpr (kSplit) __syncthreads();

  // Deep space: the lunar-solar and resonance constants, from the near-Earth fields
  // written above (the secular rates by warp 1, visible after the barrier).
  if (run && w0 && is_deep(sp.n0pp)) {
    const DeepIn in = {e0, i0, raan0, argp0, m0, sp.n0pp, sp.cosi, sp.sini,
                       f[kMdot * s + j], f[kArgpdot * s + j], f[kRaandot * s + j], g.xke};
    deep_record_init(in, rp.epoch_day[j], f[kEpochFrac * s + j], f, s, j);
  }

  // Init status: the status of the state at tsince = 0, from the FP32 state with its
  // FP64 recomputation inside the guard bands (so it equals the FP64 decision).
  if (run && w0) {
    const Rec32 r32 = read_own_rec32(h);
    float r[3], v[3];
    int code = state32(r32, gf, 0.0f, 0.0f, r, v);
    if (code == kRecomputeFP64) code = state64_fallback(rp, g, j, 0.0, r, v);
    init_status[j] = code;
  }
}

}  // namespace

cudaError_t launch_init(const double* el, const int32_t* epoch_day, const double* epoch_frac,
                        const RecordPtrs& rp, const Geo& g, int32_t* init_status,
                        cudaStream_t stream) {
  if (rp.n == 0) return cudaSuccess;
  const int64_t blocks = (rp.n + kInitSats - 1) / kInitSats;
  // Split while there is at most one block per sub-partition (4 x 148): below that the
  // FP64 unit idles between the dependent instructions of one warp.  Measured on B300:
  // 9341 satellites 33 -> 29 us, equal near 2e4, one warp faster from 3e4 (1e6: 0.84
  // against 0.90 ms).
  if (blocks <= SGP4_INIT_SPLIT_BLOCKS)
    init_kernel<true><<<(unsigned)blocks, 2 * kInitSats, 0, stream>>>(
        el, epoch_day, epoch_frac, rp, g, geo_float(g), init_status);
  else
    init_kernel<false><<<(unsigned)blocks, kInitSats, 0, stream>>>(
        el, epoch_day, epoch_frac, rp, g, geo_float(g), init_status);
  return cudaGetLastError();
}

}  // namespace sgp4
