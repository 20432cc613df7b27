// Propagation kernels: independent (satellite, time) states (paper Sec. 2.2,
// "Vectorisation": f(s, t) under a vmap over times composed with a vmap over
// satellites).  A thread takes a unit of states of one satellite that share the
// record: in FP32 four (the consecutive times 4i..4i+3 when T is a multiple of 4, else
// times i + k ceil(T/4)) as two pairs in packed arithmetic (run_range_x4, state32x2), or
// one pair (run_range_x2) for short grids whose units of four would be partly empty; in
// FP64 two (times i and i + ceil(T/2)) in turn on one load of the record, or one for
// problems that fit one wave (run_units64).  FP32 guard-band states are queued and
// recomputed in FP64 after the block's loop (fix_queued).
//   * a block walks a contiguous range of units, 128 per step, so consecutive steps of
//     a thread stay on one satellite and its record stays in L1 (FP32) or registers
//     (FP64);
//   * each thread stores its own r, v and status with streaming stores; a warp's
//     stores cover consecutive states, so L2 assembles them into full lines (on B300
//     this beat staging through shared memory with 16-byte stores by 3-6%).
// propagate_kernel: one problem, a persistent grid of one wave, each block owning
// one contiguous range.  batched_kernel: many problems ("requests") of uneven size
// in one persistent launch; blocks take fixed-size tiles of units from a global
// atomic counter, so uneven requests and uneven per-state cost balance themselves.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <type_traits>

#include "sgp4_deep.cuh"
#include "sgp4_device.cuh"
#include "sgp4_kernels.cuh"
#include "sgp4_state32x2.cuh"

namespace sgp4 {

namespace {

constexpr int kThreads = 128;
// Minimum resident 128-thread blocks per SM requested from the register allocator.
// FP32 (four states per thread): 4 blocks (128 registers); at 8 (64 registers) it
// spills heavily, 3 and 5 were slower.  The FP64 kernels are bound by the FP64 pipe
// and keep 4.
#ifndef SGP4_MIN_BLOCKS_FP32
#define SGP4_MIN_BLOCKS_FP32 4
#endif
// Programmatic dependent launch of the propagation kernels (see propagate_kernel).
#ifndef SGP4_PDL
#define SGP4_PDL 1
#endif
#ifndef SGP4_MIN_BLOCKS_FP64
#define SGP4_MIN_BLOCKS_FP64 4
#endif

// One problem's view: its time grid, its first record and its output base.
struct Range {
  const double* tsince;   // [T], or [n][T] when per_sat
  const int32_t* jd_day;  // absolute times [T] as Julian day + fraction, or null
  const double* jd_frac;
  int32_t jd0;            // with a split table of absolute times: the table's day origin
  int64_t T;
  int per_sat;
  int64_t sat0;           // record index of the problem's satellite 0
  void* r;                // output of the problem's state 0
  void* v;
  int32_t* status;
};

// a - b for double-floats (hi + lo, |lo| <= ulp(hi) / 2): Knuth's two-sum of the high
// parts, the low parts added, the sum renormalised.  On the FP32 pipes; the absolute-time
// path uses it instead of per-state FP64 arithmetic.
__device__ __forceinline__ void df_sub(float ah, float al, float bh, float bl, float& h,
                                       float& l) {
  const float s = ah - bh;
  const float v = s - ah;
  const float e = (ah - (s - v)) + (-bh - v);
  const float lo = e + (al - bl);
  h = s + lo;
  l = lo - (h - s);
}

// Minutes from day jd0 to the epoch of record rec, as float hi + lo (three FP64
// instructions, once per unit).
__device__ __forceinline__ void epoch_minutes(const RecordPtrs& rp, int64_t rec, int32_t jd0,
                                              float& h, float& l) {
  const double d = (double)(__ldg(rp.epoch_day + rec) - jd0);
  split_double(fma(1440.0, __ldg(rp.f64 + kEpochFrac * rp.stride + rec), 1440.0 * d), h, l);
}

// Guard-band states (kRecomputeFP64) are not recomputed inside the FP32 loops: a call
// of an out-of-line FP64 state there made the loops spill registers (7-13% of their
// time).  The loop queues the state's index in shared memory and marks its status;
// after the loop the block recomputes the queued states in FP64 (fix_queued).  A block
// that met more than the queue's capacity of them rescans its own units for the mark
// instead (one thread per unit, so a thread may then recompute several states in a row).
// The batched kernel's tiles hold kFixCap entries; the single-problem kernel's queue
// takes the dynamic shared memory its launch asks for beyond the time grid's split table
// (2,048 entries, or at least kFixCap on the longest split grids): a few blocks of the
// catalogue workload queue close to 300 states, and their rescans past a 256-entry queue
// had made the whole launch 55% longer.
constexpr int kFixCap = 256;
struct FixQueue {
  int64_t* idx;   // state index within the range, j * T + i
  int cap;        // entries idx holds
  int n;          // states queued (above cap: the queue overflowed)
};

__device__ __forceinline__ void queue_fix(FixQueue* fq, int32_t* status, int64_t idx) {
  const int slot = atomicAdd(&fq->n, 1);
  if (slot < fq->cap) fq->idx[slot] = idx;
  __stcs(status + idx, kRecomputeFP64);
}

// Index within the range of state k of unit u, or -1 where the unit has no state k:
// kSpu = 4 with consecutive times (4 i0 + k) or strided ones (i0 + k ceil(T/4)), kSpu = 2
// strided (i0 + k ceil(T/2)).
template <int kSpu, bool kCons>
struct UnitMap {
  int T, Tu;   // times, units per satellite
  __device__ int64_t operator()(int64_t u, int k) const {
    const int64_t j = u / Tu;
    const int i0 = (int)(u - j * Tu);
    const int i = kCons ? 4 * i0 + k : i0 + k * Tu;
    return i < T ? j * T + i : -1;
  }
};

// After the FP32 loop over units [ubeg, uend) of range rg and a __syncthreads: the
// queued guard-band states in FP64, their r, v (NaN for codes 1, 2, 4) and status.
// States of deep-space records are not queued (their FP32 row's a0'' NaN makes every one
// a guard-band state, which the loops drop): deep_pass_block computes them, which keeps
// the deep-space code and the call it needs out of the FP32 kernels (with it the
// headline kernel spilled).  The check below only serves a rescan.
// Adds the block's count to nfix (thread 0).  Inlined, FP64 state included: a kernel
// with no call at all ran 0.4-2.4% faster than one calling it out of line.
template <int kSpu, bool kCons>
__device__ __forceinline__ void fix_queued(const RecordPtrs& rp, const Geo& g, const Range& rg,
                                        const FixQueue* fq, int64_t ubeg, int64_t uend,
                                        unsigned long long& nfix) {
  const int n = fq->n;
  if (n == 0) return;
  const int T = (int)rg.T;
  const float q = __int_as_float(0x7fc00000);
  auto fix = [&](int64_t idx) {
    const int64_t j = idx / T;
    const int i = (int)(idx - j * T);
    const int64_t rec = rg.sat0 + j;
    double t;
    if (rg.jd_day) {
      const int dday = __ldg(rg.jd_day + i) - __ldg(rp.epoch_day + rec);
      const double dfrac = __ldg(rg.jd_frac + i) - __ldg(rp.f64 + kEpochFrac * rp.stride + rec);
      t = fma(1440.0, dfrac, (double)((long long)dday * 1440));
    } else {
      t = __ldg(rg.per_sat ? rg.tsince + j * T + i : rg.tsince + i);
    }
    // deep-space states are the deep-space pass's
    if (__ldg(rp.flags + rec) & kFlagDeep) return;
    float* gr = static_cast<float*>(rg.r) + idx * 3;
    float* gv = static_cast<float*>(rg.v) + idx * 3;
    const Rec64 rc = load_rec64(rp, rec);
    double r64[3], v64[3];
    const int cd = state64(rc, g, t, r64, v64);
    for (int c = 0; c < 3; ++c) {
      gr[c] = (float)r64[c];
      gv[c] = (float)v64[c];
    }
    if (cd != 0 && cd != 6) { gr[0] = q; gr[1] = q; gr[2] = q; gv[0] = q; gv[1] = q; gv[2] = q; }
    __stcs(rg.status + idx, cd);
  };
  if (n <= fq->cap) {
    for (int e = threadIdx.x; e < n; e += kThreads) fix(fq->idx[e]);
  } else {
    const UnitMap<kSpu, kCons> um{T, (T + kSpu - 1) / kSpu};
    for (int64_t u = ubeg + threadIdx.x; u < uend; u += kThreads)
      for (int k = 0; k < kSpu; ++k) {
        const int64_t idx = um(u, k);
        if (idx >= 0 && __ldcg(rg.status + idx) == kRecomputeFP64) fix(idx);
      }
  }
  if (threadIdx.x == 0) nfix += (unsigned long long)n;
}

// FP32, two states per thread (packed arithmetic, state32x2): unit u of [ubeg, uend)
// is satellite j = u / Th, times i0 = u % Th and i1 = i0 + Th (Th = ceil(T / 2); i1 does
// not exist for the last unit of an odd T), so both states share the record.
template <bool kJd>
__device__ __forceinline__ void run_range_x2(const RecordPtrs& rp, const GeoF& gf,
                                             const Range& rg, int64_t ubeg, int64_t uend,
                                             FixQueue* fq, const float2* split) {
  const int tid = threadIdx.x;
  const int T = (int)rg.T;            // <= INT32_MAX (checked by the API)
  const int Th = (T + 1) / 2;
  int64_t j = (ubeg + tid) / Th;
  int i0 = (int)((ubeg + tid) - j * Th);
  const int jstep = kThreads / Th, istep = kThreads - jstep * Th;
  for (int64_t u = ubeg + tid; u < uend; u += kThreads) {
    const int64_t rec = rg.sat0 + j;
    const int i1 = i0 + Th;
    const bool has1 = i1 < T;
    const int it[2] = {i0, has1 ? i1 : i0};
    auto tsince_at = [&](int i) -> double {
      if (rg.jd_day) {
        const int dday = __ldg(rg.jd_day + i) - __ldg(rp.epoch_day + rec);
        const double dfrac = __ldg(rg.jd_frac + i) - __ldg(rp.f64 + kEpochFrac * rp.stride + rec);
        return fma(1440.0, dfrac, (double)((long long)dday * 1440));
      }
      return __ldg(rg.per_sat ? rg.tsince + j * T + i : rg.tsince + i);
    };
    float2 th, tl;
    if (split) {
      const float2 a0 = split[it[0]], a1 = split[it[1]];
      th = make_float2(a0.x, a1.x);
      tl = make_float2(a0.y, a1.y);
      if constexpr (kJd) {   // table of minutes from day jd0: subtract the record's epoch
        float eh, el;
        epoch_minutes(rp, rec, rg.jd0, eh, el);
        df_sub(a0.x, a0.y, eh, el, th.x, tl.x);
        df_sub(a1.x, a1.y, eh, el, th.y, tl.y);
      }
    } else {
      split_double(tsince_at(it[0]), th.x, tl.x);
      split_double(tsince_at(it[1]), th.y, tl.y);
    }
    const Rec32 rc32 = load_rec32(rp, rec);
    float2 r2[3], v2[3];
    int code[2];
    state32x2(rc32, gf, th, tl, r2, v2, code);
    const float q = __int_as_float(0x7fc00000);
    // Common case, every present state valid (status 0 or 6): stores without per-lane
    // branches or NaN selects
    // (an absent second state repeats time i0, so its code equals the first state's)
    const bool fast = ((code[0] == 0) | (code[0] == 6)) & ((code[1] == 0) | (code[1] == 6));
    if (fast) {
      const int64_t idx = j * T + i0;
      float* gr = static_cast<float*>(rg.r) + idx * 3;
      float* gv = static_cast<float*>(rg.v) + idx * 3;
      const int o1 = Th * 3;   // state i1 = i0 + Th of the same satellite
      __stcs(gr + 0, r2[0].x); __stcs(gr + 1, r2[1].x); __stcs(gr + 2, r2[2].x);
      __stcs(gv + 0, v2[0].x); __stcs(gv + 1, v2[1].x); __stcs(gv + 2, v2[2].x);
      __stcs(rg.status + idx, code[0]);
      if (has1) {
        __stcs(gr + o1 + 0, r2[0].y); __stcs(gr + o1 + 1, r2[1].y); __stcs(gr + o1 + 2, r2[2].y);
        __stcs(gv + o1 + 0, v2[0].y); __stcs(gv + o1 + 1, v2[1].y); __stcs(gv + o1 + 2, v2[2].y);
        __stcs(rg.status + idx + Th, code[1]);
      }
    } else
    for (int l = 0; l < 2; ++l) {   // per lane: the last unit of an odd T, NaN outputs, FP64 recomputation
      if (l == 1 && !has1) break;
      const int64_t idx = j * T + it[l];
      float* gr = static_cast<float*>(rg.r) + idx * 3;
      float* gv = static_cast<float*>(rg.v) + idx * 3;
      const int cd = code[l];
      if (cd == kRecomputeFP64) {   // r, v and status written after the loop
        if (!(rc32.flags & kFlagDeep)) queue_fix(fq, rg.status, idx);   // deep: not ours
        continue;
      }
      {
        const bool bad = cd != 0 && cd != 6;
        const float rv[3] = {l ? r2[0].y : r2[0].x, l ? r2[1].y : r2[1].x, l ? r2[2].y : r2[2].x};
        const float vv[3] = {l ? v2[0].y : v2[0].x, l ? v2[1].y : v2[1].x, l ? v2[2].y : v2[2].x};
        __stcs(gr + 0, bad ? q : rv[0]); __stcs(gr + 1, bad ? q : rv[1]);
        __stcs(gr + 2, bad ? q : rv[2]);
        __stcs(gv + 0, bad ? q : vv[0]); __stcs(gv + 1, bad ? q : vv[1]);
        __stcs(gv + 2, bad ? q : vv[2]);
      }
      __stcs(rg.status + idx, cd);
    }
    // next unit of this thread: kThreads = jstep * Th + istep, so at most one wrap
    j += jstep;
    i0 += istep;
    if (i0 >= Th) {
      ++j;
      i0 -= Th;
    }
  }
}

// FP32, four states per thread: unit u is satellite j = u / Tq and times i0 + k Tq
// (k = 0..3, Tq = ceil(T / 4), the last ones absent past T), computed as two packed
// pairs (k = 0, 2) and (k = 1, 3) on one load of the record.  kPre (grids in minutes
// read per state, no split table): the next unit's four times are loaded while this
// unit computes (1 satellite x 1e7 times: 163 -> 126 us); a separate instantiation, as
// the prefetch's registers slow the split-table path.  kCons (T a multiple of 4,
// 16-byte aligned arrays; grids in minutes, or absolute times in the split table): the
// unit's times are the consecutive 4 i0 + k,
// so its r, v and status are 48, 48 and 16 contiguous bytes, written by seven 16-byte
// stores instead of 28 scalar ones, and its four times are two 16-byte loads (of the
// split table, or of the grid with kPre).
template <bool kPre, bool kJd, bool kCons = false>
__device__ __forceinline__ void run_range_x4(const RecordPtrs& rp, const GeoF& gf,
                                             const Range& rg, int64_t ubeg, int64_t uend,
                                             FixQueue* fq, const float2* split) {
  static_assert(!kCons || !(kJd && kPre), "absolute times take the split table");
  const int tid = threadIdx.x;
  const int T = (int)rg.T;
  const int Tq = (T + 3) / 4;
  int64_t j = (ubeg + tid) / Tq;
  int i0 = (int)((ubeg + tid) - j * Tq);
  const int jstep = kThreads / Tq, istep = kThreads - jstep * Tq;
  auto fetch = [&](int64_t jj, int ii0, double out[4]) {
    if constexpr (kCons) {   // four consecutive times: two 16-byte loads
      const double2* p = reinterpret_cast<const double2*>(
          rg.per_sat ? rg.tsince + jj * T + 4 * ii0 : rg.tsince + 4 * ii0);
      const double2 a = __ldg(p), b = __ldg(p + 1);
      out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = ii0 + k * Tq < T ? ii0 + k * Tq : ii0;
        out[k] = __ldg(rg.per_sat ? rg.tsince + jj * T + i : rg.tsince + i);
      }
    }
  };
  double tn[4] = {0.0, 0.0, 0.0, 0.0};
  if constexpr (kPre) {
    if (ubeg + tid < uend) fetch(j, i0, tn);
  }
  for (int64_t u = ubeg + tid; u < uend; u += kThreads) {
    const int64_t rec = rg.sat0 + j;
    int it[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = kCons ? 4 * i0 + k : i0 + k * Tq;
      it[k] = kCons || i < T ? i : i0;
    }
    const bool has3 = kCons || i0 + 3 * Tq < T;   // then all four exist
    double tc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) tc[k] = tn[k];
    if constexpr (kPre) {
      int64_t jn = j + jstep;
      int i0n = i0 + istep;
      if (i0n >= Tq) {
        ++jn;
        i0n -= Tq;
      }
      if (u + kThreads < uend) fetch(jn, i0n, tn);
    }
    auto tsince_at = [&](int i) -> double {
      if (rg.jd_day) {
        const int dday = __ldg(rg.jd_day + i) - __ldg(rp.epoch_day + rec);
        const double dfrac = __ldg(rg.jd_frac + i) - __ldg(rp.f64 + kEpochFrac * rp.stride + rec);
        return fma(1440.0, dfrac, (double)((long long)dday * 1440));
      }
      return __ldg(rg.per_sat ? rg.tsince + j * T + i : rg.tsince + i);
    };
    float th[4], tl[4];
    float eh = 0.0f, el = 0.0f;   // absolute times: the record's epoch from day jd0
    if (kJd && split) epoch_minutes(rp, rec, rg.jd0, eh, el);
    if constexpr (kCons && !kPre) {
      const float4* s4 = reinterpret_cast<const float4*>(split) + 2 * i0;
      const float4 a = s4[0], b = s4[1];
      th[0] = a.x; tl[0] = a.y; th[1] = a.z; tl[1] = a.w;
      th[2] = b.x; tl[2] = b.y; th[3] = b.z; tl[3] = b.w;
      if constexpr (kJd) {
#pragma unroll
        for (int k = 0; k < 4; ++k) df_sub(th[k], tl[k], eh, el, th[k], tl[k]);
      }
    } else
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (split) {
        const float2 a = split[it[k]];
        th[k] = a.x;
        tl[k] = a.y;
        if constexpr (kJd) df_sub(a.x, a.y, eh, el, th[k], tl[k]);
      } else {
        split_double(kPre ? tc[k] : tsince_at(it[k]), th[k], tl[k]);
      }
    }
    const Rec32 rc32 = load_rec32(rp, rec);
    float2 rA[3], vA[3], rB[3], vB[3];
    int cA[2], cB[2];
    state32x2(rc32, gf, make_float2(th[0], th[2]), make_float2(tl[0], tl[2]), rA, vA, cA);
    state32x2(rc32, gf, make_float2(th[1], th[3]), make_float2(tl[1], tl[3]), rB, vB, cB);
    auto ok = [](int c) { return (c == 0) | (c == 6); };
    const int64_t idx0 = j * T + (kCons ? 4 * i0 : i0);
    const int64_t kstride = kCons ? 1 : Tq;   // index step between the unit's states
    if (kCons && (ok(cA[0]) & ok(cA[1]) & ok(cB[0]) & ok(cB[1]))) {
      // states k = 0..3 are (A.x, B.x, A.y, B.y): 12 floats of r, 12 of v, 4 codes
      float4* gr = reinterpret_cast<float4*>(static_cast<float*>(rg.r) + idx0 * 3);
      float4* gv = reinterpret_cast<float4*>(static_cast<float*>(rg.v) + idx0 * 3);
      __stcs(gr + 0, make_float4(rA[0].x, rA[1].x, rA[2].x, rB[0].x));
      __stcs(gr + 1, make_float4(rB[1].x, rB[2].x, rA[0].y, rA[1].y));
      __stcs(gr + 2, make_float4(rA[2].y, rB[0].y, rB[1].y, rB[2].y));
      __stcs(gv + 0, make_float4(vA[0].x, vA[1].x, vA[2].x, vB[0].x));
      __stcs(gv + 1, make_float4(vB[1].x, vB[2].x, vA[0].y, vA[1].y));
      __stcs(gv + 2, make_float4(vA[2].y, vB[0].y, vB[1].y, vB[2].y));
      __stcs(reinterpret_cast<int4*>(rg.status + idx0), make_int4(cA[0], cB[0], cA[1], cB[1]));
    } else if (!kCons && (has3 & ok(cA[0]) & ok(cA[1]) & ok(cB[0]) & ok(cB[1]))) {
      // all four present and valid (status 0 or 6): stores without branches or selects
      float* gr = static_cast<float*>(rg.r) + idx0 * 3;
      float* gv = static_cast<float*>(rg.v) + idx0 * 3;
      const int o = Tq * 3;
      __stcs(gr + 0, rA[0].x); __stcs(gr + 1, rA[1].x); __stcs(gr + 2, rA[2].x);
      __stcs(gv + 0, vA[0].x); __stcs(gv + 1, vA[1].x); __stcs(gv + 2, vA[2].x);
      __stcs(gr + o + 0, rB[0].x); __stcs(gr + o + 1, rB[1].x); __stcs(gr + o + 2, rB[2].x);
      __stcs(gv + o + 0, vB[0].x); __stcs(gv + o + 1, vB[1].x); __stcs(gv + o + 2, vB[2].x);
      __stcs(gr + 2 * o + 0, rA[0].y); __stcs(gr + 2 * o + 1, rA[1].y); __stcs(gr + 2 * o + 2, rA[2].y);
      __stcs(gv + 2 * o + 0, vA[0].y); __stcs(gv + 2 * o + 1, vA[1].y); __stcs(gv + 2 * o + 2, vA[2].y);
      __stcs(gr + 3 * o + 0, rB[0].y); __stcs(gr + 3 * o + 1, rB[1].y); __stcs(gr + 3 * o + 2, rB[2].y);
      __stcs(gv + 3 * o + 0, vB[0].y); __stcs(gv + 3 * o + 1, vB[1].y); __stcs(gv + 3 * o + 2, vB[2].y);
      __stcs(rg.status + idx0, cA[0]);
      __stcs(rg.status + idx0 + Tq, cB[0]);
      __stcs(rg.status + idx0 + 2 * Tq, cA[1]);
      __stcs(rg.status + idx0 + 3 * Tq, cB[1]);
    } else {
      const float q = __int_as_float(0x7fc00000);
      for (int k = 0; k < 4; ++k) {
        if (!kCons && i0 + k * Tq >= T) break;
        // state k is lane k >> 1 of pair A (k even) or B (k odd), picked with selects:
        // a run-time index into the register arrays would put them in local memory
        const bool odd = k & 1, hi = k >= 2;
        auto pick = [&](const float2& a, const float2& b) {
          const float2 p = odd ? b : a;
          return hi ? p.y : p.x;
        };
        const int cd = odd ? (hi ? cB[1] : cB[0]) : (hi ? cA[1] : cA[0]);
        const int64_t idx = idx0 + k * kstride;
        if (cd == kRecomputeFP64) {   // r, v and status written after the loop
          if (!(rc32.flags & kFlagDeep)) queue_fix(fq, rg.status, idx);   // deep: not ours
          continue;
        }
        float* gr = static_cast<float*>(rg.r) + idx * 3;
        float* gv = static_cast<float*>(rg.v) + idx * 3;
        {
          const bool bad = cd != 0 && cd != 6;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            __stcs(gr + c, bad ? q : pick(rA[c], rB[c]));
            __stcs(gv + c, bad ? q : pick(vA[c], vB[c]));
          }
        }
        __stcs(rg.status + idx, cd);
      }
    }
    j += jstep;
    i0 += istep;
    if (i0 >= Tq) {
      ++j;
      i0 -= Tq;
    }
  }
}

// FP64, kSpu (1 or 2) states per thread: unit u is satellite j = u / Th and times
// i0 + l Th (Th = ceil(T / kSpu)), run in turn on one load of the record.  One state
// per thread for problems that fit one wave: the FP64 state is a long dependent chain
// on B300's FP64 unit (~15 us), so two in turn would double a small call's latency.
template <int kSpu>
__device__ __forceinline__ void run_units64(const RecordPtrs& rp, const Geo& g, const Range& rg,
                                            int64_t ubeg, int64_t uend) {
  const int tid = threadIdx.x;
  const int T = (int)rg.T;
  const int Th = (T + kSpu - 1) / kSpu;
  int64_t j = (ubeg + tid) / Th;
  int i0 = (int)((ubeg + tid) - j * Th);
  const int jstep = kThreads / Th, istep = kThreads - jstep * Th;
  int64_t cur = -1;
  Rec64 rc;
  const double q = __longlong_as_double(0x7ff8000000000000LL);
  for (int64_t u = ubeg + tid; u < uend; u += kThreads) {
    const int64_t rec = rg.sat0 + j;
    if (j != cur) {
      rc = load_rec64(rp, rec);
      cur = j;
    }
    for (int l = 0; l < kSpu; ++l) {
      const int i = i0 + l * Th;
      if (i >= T) break;
      double t;
      if (rg.jd_day) {
        const int dday = __ldg(rg.jd_day + i) - __ldg(rp.epoch_day + rec);
        const double dfrac = __ldg(rg.jd_frac + i) - __ldg(rp.f64 + kEpochFrac * rp.stride + rec);
        t = fma(1440.0, dfrac, (double)((long long)dday * 1440));
      } else {
        t = __ldg(rg.per_sat ? rg.tsince + j * T + i : rg.tsince + i);
      }
      if (rc.flags & kFlagDeep) continue;   // the deep-space pass's
      double r[3], v[3];
      const int code = state64(rc, g, t, r, v);
      const bool bad = code != 0 && code != 6;
      const int64_t idx = j * T + i;
      double* gr = static_cast<double*>(rg.r) + idx * 3;
      double* gv = static_cast<double*>(rg.v) + idx * 3;
      for (int c = 0; c < 3; ++c) {
        __stcs(gr + c, bad ? q : r[c]);
        __stcs(gv + c, bad ? q : v[c]);
      }
      __stcs(rg.status + idx, code);
    }
    // next unit of this thread: kThreads = jstep * Th + istep, so at most one wrap
    j += jstep;
    i0 += istep;
    if (i0 >= Th) {
      ++j;
      i0 -= Th;
    }
  }
}

// FP32 launches on a shared grid of at most this many times split the grid into float
// hi + lo once per block, into dynamic shared memory (48 KB at most: four resident
// blocks share an SM's 228 KB), instead of once per state (1,000 x 4,096: 55 -> 49 us).
constexpr int kSplitMaxT = 6144;

// kSpu: states per unit (FP32 2 or 4, FP64 1 or 2), chosen at launch; kPre: FP32
// four-state units with times read per state, prefetched (run_range_x4); kJd: FP32 with
// the split table of absolute times (each unit subtracts its record's epoch).  Separate
// instantiations keep each path free of the others' code.
template <typename Out>
static __device__ __noinline__ void deep_pass_block(const PropArgs a, int chunks, int64_t bid,
                                                    int64_t nblocks);

// The last `deep_blocks` blocks run the deep-space pass (deep_pass_block, work items of
// `deep_chunks` parts of the grid); the others propagate `chunk` units each.  Last, so
// that the propagation's blocks are the ones resident while the record build that this
// launch depends on runs (first, the pass's blocks held the SMs then: 2 us more on the
// Starlink-shaped step).
template <bool kFP32, int kSpu, bool kPre = false, bool kJd = false, bool kCons = false>
__global__ void __launch_bounds__(kThreads, kFP32 ? SGP4_MIN_BLOCKS_FP32 : SGP4_MIN_BLOCKS_FP64)
    propagate_kernel(PropArgs a, int64_t chunk, int deep_blocks, int deep_chunks) {
  // FP32: [t_count] split times when use_split, then the guard-band queue
  extern __shared__ __align__(16) float2 s_split[];
  __shared__ FixQueue s_fq;
#if SGP4_PDL
  // Launched as a programmatic dependent of the stream's previous kernel (the record
  // build, in a step): the blocks are scheduled while it runs and wait here, before
  // their first global access, until it has completed and its writes are visible.
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
  const int64_t prop_blocks = (int64_t)gridDim.x - deep_blocks;
  if ((int64_t)blockIdx.x >= prop_blocks) {
    deep_pass_block<std::conditional_t<kFP32, float, double>>(
        a, deep_chunks, (int64_t)blockIdx.x - prop_blocks, deep_blocks);
    return;
  }
  const int64_t total = a.rp.n * units_per_sat(a.t_count, kSpu);
  const int64_t beg = (int64_t)blockIdx.x * chunk;
  const int64_t end = min(total, beg + chunk);
  if (beg >= end) return;
  const bool use_split = kFP32 && !a.grid_per_sat && a.t_count <= kSplitMaxT;
  if (kFP32 && threadIdx.x == 0) {
    const int used = use_split ? (int)a.t_count : 0;
    s_fq.idx = reinterpret_cast<int64_t*>(s_split + used);
    unsigned dyn_bytes;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
    s_fq.cap = (int)(dyn_bytes / sizeof(int64_t)) - used;
    s_fq.n = 0;
  }
  const int32_t jd0 = a.jd_day ? __ldg(a.jd_day) : 0;
  if (use_split) {
    // minutes since epoch, or for absolute times minutes from the grid's first day (each
    // unit then subtracts its record's epoch in double-float arithmetic)
    for (int k = threadIdx.x; k < (int)a.t_count; k += kThreads) {
      const double t = a.jd_day ? fma(1440.0, __ldg(a.jd_frac + k),
                                      1440.0 * (double)(__ldg(a.jd_day + k) - jd0))
                                : __ldg(a.tsince + k);
      float h, l;
      split_double(t, h, l);
      s_split[k] = make_float2(h, l);
    }
  }
  if (kFP32) __syncthreads();   // the split table and the queue's count
  const GeoF gf = a.gf;
  Range rg;
  rg.tsince = a.tsince;
  rg.jd_day = a.jd_day;
  rg.jd_frac = a.jd_frac;
  rg.jd0 = jd0;
  rg.T = a.t_count;
  rg.per_sat = a.grid_per_sat;
  rg.sat0 = 0;
  rg.r = a.r;
  rg.v = a.v;
  rg.status = a.status;
  unsigned long long nfix = 0;
  const float2* split = use_split ? s_split : nullptr;
  if (kCons && !kPre && !use_split) return;   // (the launch takes this only with a split table)
  if constexpr (kFP32) {
    if constexpr (kSpu == 4) run_range_x4<kPre, kJd, kCons>(a.rp, gf, rg, beg, end, &s_fq, split);
    else run_range_x2<kJd>(a.rp, gf, rg, beg, end, &s_fq, split);
    __syncthreads();
    fix_queued<kSpu, kCons>(a.rp, a.g, rg, &s_fq, beg, end, nfix);
    if (a.fixups && nfix) atomicAdd(a.fixups, nfix);
  } else {
    run_units64<kSpu>(a.rp, a.g, rg, beg, end);
  }
}

// Persistent batched kernel: tiles of `tile_states` consecutive states of one
// request, numbered request by request (tile_start is the exclusive prefix sum of
// the tile counts); a block takes the next tile index from the counter until the
// tiles run out.  The counter is only incremented: no block ever waits on another.
template <bool kFP32>
__global__ void __launch_bounds__(kThreads, kFP32 ? SGP4_MIN_BLOCKS_FP32 : SGP4_MIN_BLOCKS_FP64)
    batched_kernel(BatchArgs a) {
  __shared__ unsigned long long s_tile;
  __shared__ int64_t s_fq_idx[kFixCap];
  __shared__ FixQueue s_fq;
  const GeoF gf = a.gf;
  const int64_t total_tiles = a.tile_start[a.n_req];
  unsigned long long nfix = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(a.counter, 1ULL);
      s_fq.idx = s_fq_idx;
      s_fq.cap = kFixCap;
      s_fq.n = 0;
    }
    __syncthreads();
    const int64_t tile = (int64_t)s_tile;
    __syncthreads();
    if (tile >= total_tiles) break;
    // Request owning the tile: the last q with tile_start[q] <= tile (requests with
    // no states have no tiles and are skipped by this rule).
    int lo = 0, hi = a.n_req - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(a.tile_start + mid) <= tile) lo = mid; else hi = mid - 1;
    }
    // A tile is tile_states / 4 units of four states (FP32) or tile_states / 2 units of
    // two (FP64); the request's tiles past this kernel's units are empty.
    const sgp4_request q = a.reqs[lo];
    const int spu = kFP32 ? 4 : 2;
    const int64_t units = q.n * units_per_sat(q.t_count, spu);
    const int64_t per_tile = a.tile_states / spu;
    const int64_t beg = (tile - __ldg(a.tile_start + lo)) * per_tile;
    const int64_t end = min(units, beg + per_tile);
    if (beg >= end) continue;
    Range rg;
    rg.tsince = a.tsince + q.t_offset;
    rg.jd_day = nullptr;
    rg.jd_frac = nullptr;
    rg.jd0 = 0;
    rg.T = q.t_count;
    rg.per_sat = 0;
    rg.sat0 = q.sat_offset;
    if (kFP32) {
      rg.r = static_cast<float*>(a.r) + q.out_offset * 3;
      rg.v = static_cast<float*>(a.v) + q.out_offset * 3;
    } else {
      rg.r = static_cast<double*>(a.r) + q.out_offset * 3;
      rg.v = static_cast<double*>(a.v) + q.out_offset * 3;
    }
    rg.status = a.status + q.out_offset;
    // (no prefetch: tiles are short, and it measured 1% slower on the 256-request batch)
    if constexpr (kFP32) {
      run_range_x4<false, false>(a.rp, gf, rg, beg, end, &s_fq, nullptr);
      __syncthreads();
      fix_queued<4, false>(a.rp, a.g, rg, &s_fq, beg, end, nfix);
      __syncthreads();   // the queue is reset with the next tile
    } else {
      run_units64<2>(a.rp, a.g, rg, beg, end);
    }
  }
  if (kFP32 && a.fixups && nfix) atomicAdd(a.fixups, nfix);
}

// Deep-space states of satellites [j0, j1) (at most kThreads) and times [i0, i1) of
// range rg, in FP64, by one block: the block gathers the slice's deep-space
// satellites in shared memory (none: it is done), then each thread takes a run of
// consecutive states (satellite-major), so that it carries its resonance integration
// from one time of a satellite to the next.  Outputs of type Out.
template <typename Out>
__device__ __forceinline__ void deep_slice(const RecordPtrs& rp, const Geo& g, const Range& rg,
                                           int64_t j0, int64_t j1, int i0, int i1, int* s_sel,
                                           int* s_key, int* s_n, const DeepPhases* ph) {
  if (threadIdx.x == 0) *s_n = 0;
  __syncthreads();
  const int64_t j = j0 + threadIdx.x;
  if (j < j1) {
    const int64_t rec = rg.sat0 + j;
    const int fl = __ldg(rp.flags + rec);
    if (fl & kFlagDeep) {
      // The branches of the deep-space state follow the record's class: the resonance
      // (none, one or two revolutions per day), the Lyddane form of the periodics (the
      // epoch inclination below 0.2 rad stands in for the perturbed one) and the
      // Newton step count (from e0).  B300's FP64 unit charges a warp instruction
      // whatever the number of its active lanes, so the block orders its satellites by
      // that class (then by index), and its warps take mostly uniform branches.
      const int rez = (fl & kFlagRez1) ? 1 : (fl & kFlagRez2) ? 2 : 0;
      const float inc = (float)__ldg(rp.f64 + kI0 * rp.stride + rec);
      const float e0 = (float)__ldg(rp.f64 + kE0 * rp.stride + rec);
      const float e2 = e0 * e0;
      const int eb = (e2 > 1.5876e-10f) + (e2 > 9.3e-5f) + (e2 > 0.01664f) + (e2 > 0.1347f) +
                     (e2 > 0.25f);
      const int key = ((rez * 2 + (inc < 0.2f ? 1 : 0)) * 8 + eb) * 256 + threadIdx.x;
      s_key[atomicAdd(s_n, 1)] = key;
    }
  }
  __syncthreads();
  const int nd = *s_n;
  if (threadIdx.x < nd) {   // rank of this entry among the block's keys (all distinct)
    const int mine = s_key[threadIdx.x];
    int rank = 0;
    for (int q = 0; q < nd; ++q) rank += s_key[q] < mine;
    s_sel[rank] = mine & 255;
  }
  __syncthreads();
  const int64_t T = rg.T;
  const int nt = i1 - i0;
  const Out q = (Out)__longlong_as_double(0x7ff8000000000000LL);
  const int64_t S = nt > 0 ? (int64_t)nd * nt : 0;
  const int64_t per = (S + kThreads - 1) / kThreads;
  const int64_t k0 = threadIdx.x * per, k1 = min(S, k0 + per);
  ResCache cache{-1, 0.0, 0.0, 0.0};
  for (int64_t k = k0; k < k1; ++k) {
    const int64_t jj = j0 + s_sel[k / nt];
    const int i = i0 + (int)(k % nt);
    const int64_t rec = rg.sat0 + jj;
    double t;
    if (rg.jd_day) {
      const int dday = __ldg(rg.jd_day + i) - __ldg(rp.epoch_day + rec);
      const double dfrac = __ldg(rg.jd_frac + i) - __ldg(rp.f64 + kEpochFrac * rp.stride + rec);
      t = fma(1440.0, dfrac, (double)((long long)dday * 1440));
    } else {
      t = __ldg(rg.per_sat ? rg.tsince + jj * T + i : rg.tsince + i);
    }
    double r64[3], v64[3];
    const int cd = state64_deep(rp, rec, g, t, r64, v64, ph, &cache);
    const bool keep = cd == 0 || cd == 6;
    const int64_t idx = jj * T + i;
    Out* gr = static_cast<Out*>(rg.r) + idx * 3;
    Out* gv = static_cast<Out*>(rg.v) + idx * 3;
    for (int c = 0; c < 3; ++c) {
      gr[c] = keep ? (Out)r64[c] : q;
      gv[c] = keep ? (Out)v64[c] : q;
    }
    rg.status[idx] = cd;
  }
  __syncthreads();
}

// The deep-space states of a single-problem call, in FP64, by the last `nblocks` blocks
// of its propagation launch (block `bid` of them; the other blocks propagate and leave
// deep-space states untouched).  Out of line: one copy for every instantiation of the
// propagation kernel, and none of its registers in the propagation's loops.  Without
// deep-space records the blocks read their satellites' flags and leave.
template <typename Out>
static __device__ __noinline__ void deep_pass_block(const PropArgs a, int chunks, int64_t bid,
                                                    int64_t nblocks) {
  __shared__ int s_sel[kThreads];
  __shared__ int s_key[kThreads];
  __shared__ int s_n;
  __shared__ DeepPhases s_ph;
  // Most record sets hold no deep-space record: each thread looks at its satellite of
  // every item of this block first, and the block leaves if none is one.
  {
    const int64_t n = a.rp.n;
    const int64_t items = (n + kThreads - 1) / kThreads * chunks;
    bool any = false;
#pragma unroll 8
    for (int64_t w = bid; w < items; w += nblocks) {
      const int64_t j = w / chunks * kThreads + threadIdx.x;
      any |= j < n && (__ldg(a.rp.flags + j) & kFlagDeep);
    }
    if (!__syncthreads_or(any)) return;
  }
  if (threadIdx.x < 8) deep_phase(threadIdx.x, s_ph);   // visible after deep_slice's barrier
  Range rg;
  rg.tsince = a.tsince;
  rg.jd_day = a.jd_day;
  rg.jd_frac = a.jd_frac;
  rg.jd0 = 0;
  rg.T = a.t_count;
  rg.per_sat = a.grid_per_sat;
  rg.sat0 = 0;
  rg.r = a.r;
  rg.v = a.v;
  rg.status = a.status;
  // work items: (slice of kThreads satellites, one of `chunks` parts of the grid)
  const int64_t n = a.rp.n;
  const int T = (int)a.t_count;
  const int per = (T + chunks - 1) / chunks;
  const int64_t items = (n + kThreads - 1) / kThreads * chunks;
  for (int64_t w = bid; w < items; w += nblocks) {
    const int64_t j0 = w / chunks * kThreads;
    const int i0 = (int)(w % chunks) * per;
    deep_slice<Out>(a.rp, a.g, rg, j0, min(n, j0 + kThreads), i0, min(T, i0 + per), s_sel,
                    s_key, &s_n, &s_ph);
  }
}

// The same after a batched launch, request by request.
template <bool kFP32>
__global__ void __launch_bounds__(kThreads, 4) deep_fix_batched_kernel(BatchArgs a) {
  __shared__ int s_sel[kThreads];
  __shared__ int s_key[kThreads];
  __shared__ int s_n;
  __shared__ DeepPhases s_ph;
  __shared__ sgp4_request s_req[kThreads];
  if (threadIdx.x < 8) deep_phase(threadIdx.x, s_ph);   // visible after deep_slice's barrier
  using Out = std::conditional_t<kFP32, float, double>;
  // The request table kThreads entries at a time through shared memory (one load each,
  // in parallel, instead of one dependent load per request per block); request k's
  // slices of kThreads satellites start at block k mod gridDim, so that the first slices
  // of the many small requests spread over the blocks instead of all going to block 0.
  for (int k0 = 0; k0 < a.n_req; k0 += kThreads) {
    const int nk = min(kThreads, a.n_req - k0);
    __syncthreads();   // the previous chunk's requests are no longer read
    if ((int)threadIdx.x < nk) s_req[threadIdx.x] = a.reqs[k0 + threadIdx.x];
    __syncthreads();
    for (int kk = 0; kk < nk; ++kk) {
      const sgp4_request q = s_req[kk];
      if (q.n == 0 || q.t_count == 0) continue;
      const int64_t first =
          ((int64_t)blockIdx.x + gridDim.x - (int64_t)((k0 + kk) % gridDim.x)) % gridDim.x;
      if (first * kThreads >= q.n) continue;
      Range rg;
      rg.tsince = a.tsince + q.t_offset;
      rg.jd_day = nullptr;
      rg.jd_frac = nullptr;
      rg.jd0 = 0;
      rg.T = q.t_count;
      rg.per_sat = 0;
      rg.sat0 = q.sat_offset;
      rg.r = static_cast<Out*>(a.r) + q.out_offset * 3;
      rg.v = static_cast<Out*>(a.v) + q.out_offset * 3;
      rg.status = a.status + q.out_offset;
      for (int64_t j0 = first * kThreads; j0 < q.n; j0 += (int64_t)gridDim.x * kThreads)
        deep_slice<Out>(a.rp, a.g, rg, j0, min(q.n, j0 + kThreads), 0, (int)q.t_count, s_sel,
                        s_key, &s_n, &s_ph);
    }
  }
}

template <typename K>
int blocks_per_sm_of(K kernel, size_t dyn_smem = 0) {
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, kThreads, dyn_smem) !=
      cudaSuccess)
    return 1;
  return bps > 0 ? bps : 1;
}

constexpr int kMaxDevices = 64;

// Resident blocks per SM of `kernel` on the current device, found once per device and
// cached in `cache` (zero = not yet known).  With `opt_in` the kernel's dynamic
// shared-memory limit is first raised to `dyn_smem`; that attribute belongs to the
// device, so it is set on each device the library launches on.
template <typename K>
cudaError_t device_bps(std::atomic<int> (&cache)[kMaxDevices], K kernel, size_t dyn_smem,
                       bool opt_in, int* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  int b = cache[dev].load(std::memory_order_acquire);
  if (b == 0) {
    if (opt_in) {
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)dyn_smem);
      if (e != cudaSuccess) return e;
    }
    b = blocks_per_sm_of(kernel, dyn_smem);
    cache[dev].store(b, std::memory_order_release);
  }
  *out = b;
  return cudaSuccess;
}

// The deep-space pass's share of a single-problem launch: work items of kThreads
// satellites x a part of the grid (parts of at least 32 times, as many as give
// SGP4_DEEP_ITEMS_PER_SM items per SM), taken round-robin by the launch's first blocks,
// SGP4_DEEP_BLOCKS_PER_SM per SM.  Measured on the 10,000 x 1,000 deep-space workload:
// 16 items per SM 19.0 ms, 4 items 22.4 (the last wave's items ran alone), 32 or 64
// items 19.9; one block per SM 22.2.  The pass runs in the propagation's own launch (its
// last blocks) rather than in a launch of its own, which cost every call about 2 us.
#ifndef SGP4_DEEP_ITEMS_PER_SM
#define SGP4_DEEP_ITEMS_PER_SM 16
#endif
#ifndef SGP4_DEEP_BLOCKS_PER_SM
#define SGP4_DEEP_BLOCKS_PER_SM 4
#endif
void deep_share(const PropArgs& a, int per_sm, int* chunks, int* blocks) {
  const int64_t slices = (a.rp.n + kThreads - 1) / kThreads;
  const int64_t sms = device_sm_count();
  const int64_t want = SGP4_DEEP_ITEMS_PER_SM * sms;
  *chunks = (int)std::max<int64_t>(
      1, std::min<int64_t>((a.t_count + 31) / 32, (want + slices - 1) / slices));
  *blocks = (int)std::min<int64_t>(slices * *chunks, per_sm * sms);
}

template <bool kFP32, int kSpu, bool kPre = false, bool kJd = false, bool kCons = false>
cudaError_t launch_spu(const PropArgs& a, cudaStream_t stream) {
  const int64_t total = a.rp.n * units_per_sat(a.t_count, kSpu);
  if (total == 0) return cudaSuccess;
  // FP32: the split table and the guard-band queue share the dynamic shared memory (an
  // opt-in above 48 KB): the grid's split times, then kFixQueueMin queue entries (the
  // queue takes what the table leaves, within kFP32Dyn bytes in all).  The resident
  // blocks per SM are found once with the largest size, so they hold for every launch.
  // A launch asks only for what its grid needs: the rest of the SM's 256 KB of L1 and
  // shared memory is then L1 cache, which a grid of one time per satellite (a 160-byte
  // record row read per state) needs (1e6 satellites x 1 time: 61 -> 41 us).
  constexpr size_t kFP32Dyn = (size_t)(kSplitMaxT + kFixCap) * sizeof(int64_t);
  constexpr int64_t kFixQueueMin = 2048;
  static_assert(sizeof(int64_t) == sizeof(float2), "queue entries reuse split slots");
  const int64_t split_t = (!a.grid_per_sat && a.t_count <= kSplitMaxT) ? a.t_count : 0;
  const size_t dyn = kFP32 ? std::min<size_t>(kFP32Dyn, (size_t)(split_t + kFixQueueMin) *
                                                            sizeof(int64_t))
                           : 0;
  static std::atomic<int> bps_dev[kMaxDevices];
  int bps = 0;
  const cudaError_t be = device_bps(bps_dev, propagate_kernel<kFP32, kSpu, kPre, kJd, kCons>,
                                    kFP32 ? kFP32Dyn : 0, kFP32, &bps);
  if (be != cudaSuccess) return be;
  const int64_t tiles = (total + kThreads - 1) / kThreads;
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)device_sm_count() * bps);
  const int64_t chunk = ((tiles + grid - 1) / grid) * kThreads;
  const int64_t blocks = (total + chunk - 1) / chunk;
  // The deep-space blocks: with an FP64 grid under nine tenths of a wave one per SM, so
  // that they are resident beside the propagation's blocks (in a launch of their own
  // before the propagation, the propagation's blocks were placed as theirs left and
  // piled onto the first SMs to free up; the FP64 kernel is bound by each SM's FP64
  // unit: 1e5 states 124 us instead of 96).
  const int64_t wave = (int64_t)device_sm_count() * bps;
  const bool full = blocks * 10 >= wave * 9;
  int deep_chunks = 1, deep_blocks = 0;
  deep_share(a, kFP32 || full ? SGP4_DEEP_BLOCKS_PER_SM : 1, &deep_chunks, &deep_blocks);
#if SGP4_PDL
  // A programmatic dependent's blocks are placed as the previous kernel's blocks leave
  // their SMs, so a grid of less than one wave can land several blocks on the first SMs
  // to free up; FP64 grids under nine tenths of a wave (the chunking leaves a wave-capped
  // grid a few blocks short) launch after the previous kernel has ended.  The FP32 kernel
  // keeps the overlap at every size (without it small calls took 1-2 us longer).
  const bool pdl = kFP32 || full || blocks == 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(blocks + deep_blocks));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, propagate_kernel<kFP32, kSpu, kPre, kJd, kCons>, a, chunk,
                            deep_blocks, deep_chunks);
#else
  propagate_kernel<kFP32, kSpu, kPre, kJd, kCons>
      <<<(unsigned)(blocks + deep_blocks), kThreads, dyn, stream>>>(a, chunk, deep_blocks,
                                                                   deep_chunks);
  return cudaGetLastError();
#endif
}

// FP32: four states per unit (on full units 0.94 of the time of two units of two) where
// partly empty units are rare: T a multiple of 4, or T >= 48 (at most 3 in 12 units;
// an absent state is computed anyway and a partly empty unit stores state by state).
// Other T take units of two, whose one possibly absent state is a predicated store
// (1e6 satellites x 10 times: 282 -> 130 us; x 1 time: 53 -> 41 us).
bool fp32_units_of_four(int64_t T) { return T % 4 == 0 || T >= 48; }

cudaError_t launch_fp32(const PropArgs& a, cudaStream_t stream) {
  const bool per_state = a.grid_per_sat || a.t_count > kSplitMaxT;   // no split table
  const bool jd_table = a.jd_day && !per_state;
  if (!fp32_units_of_four(a.t_count))
    return jd_table ? launch_spu<true, 2, false, true>(a, stream) : launch_spu<true, 2>(a, stream);
  if (jd_table) {
    const bool al = a.t_count % 4 == 0 && ((reinterpret_cast<uintptr_t>(a.r) |
                                            reinterpret_cast<uintptr_t>(a.v) |
                                            reinterpret_cast<uintptr_t>(a.status)) & 15) == 0;
    return al ? launch_spu<true, 4, false, true, true>(a, stream)
              : launch_spu<true, 4, false, true>(a, stream);
  }
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const bool cons = !a.jd_day && a.t_count % 4 == 0 && al16(a.r) && al16(a.v) &&
                    al16(a.status) && (!per_state || al16(a.tsince));
  if (per_state && !a.jd_day)
    return cons ? launch_spu<true, 4, true, false, true>(a, stream)
                : launch_spu<true, 4, true>(a, stream);
  if (cons) return launch_spu<true, 4, false, false, true>(a, stream);
  return launch_spu<true, 4>(a, stream);
}

// FP64: one state per thread while the two-state units would not fill one wave of the
// kernel (148 SMs x 4 blocks x 128 threads), two otherwise.
cudaError_t launch_fp64(const PropArgs& a, cudaStream_t stream) {
  static std::atomic<int> bps_dev[kMaxDevices];
  int bps = 0;
  const cudaError_t be = device_bps(bps_dev, propagate_kernel<false, 2>, 0, false, &bps);
  if (be != cudaSuccess) return be;
  const int64_t wave = (int64_t)device_sm_count() * bps * kThreads;
  return a.rp.n * units_per_sat(a.t_count, 2) < wave ? launch_spu<false, 1>(a, stream)
                                                     : launch_spu<false, 2>(a, stream);
}

template <bool kFP32>
int64_t grid_b(int64_t total_tiles, int grid_blocks) {
  static std::atomic<int> bps_dev[kMaxDevices];
  int bps = 1;
  if (device_bps(bps_dev, batched_kernel<kFP32>, 0, false, &bps) != cudaSuccess) bps = 1;
  int64_t grid = grid_blocks > 0 ? grid_blocks : (int64_t)device_sm_count() * bps;
  return std::max<int64_t>(1, std::min<int64_t>(grid, total_tiles));
}

}  // namespace

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

cudaError_t launch_propagate64(const PropArgs& a, cudaStream_t stream) {
  if (a.rp.n == 0 || a.t_count == 0) return cudaSuccess;
  return launch_fp64(a, stream);
}

cudaError_t launch_propagate32(const PropArgs& a, cudaStream_t stream) {
  if (a.rp.n == 0 || a.t_count == 0) return cudaSuccess;
  return launch_fp32(a, stream);
}

int64_t batched_grid(bool fp32, int64_t total_tiles, int grid_blocks) {
  return fp32 ? grid_b<true>(total_tiles, grid_blocks) : grid_b<false>(total_tiles, grid_blocks);
}

cudaError_t launch_batched(const BatchArgs& a, bool fp32, int64_t total_tiles, int64_t grid,
                           cudaStream_t stream) {
  if (total_tiles == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  // then the deep-space states the batched kernel left to deep_fix_batched_kernel
  const unsigned fix_grid = (unsigned)std::min<int64_t>(grid, 4 * (int64_t)device_sm_count());
  if (fp32) {
    batched_kernel<true><<<(unsigned)grid, kThreads, 0, stream>>>(a);
    deep_fix_batched_kernel<true><<<fix_grid, kThreads, 0, stream>>>(a);
  } else {
    batched_kernel<false><<<(unsigned)grid, kThreads, 0, stream>>>(a);
    deep_fix_batched_kernel<false><<<fix_grid, kThreads, 0, stream>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace sgp4
