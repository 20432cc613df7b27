// Adjoint (vector-Jacobian product) of the propagation with respect to the mean
// elements: given upstream gradients g_r, g_v of every state's r, v, it returns
//   g_el[j][k] = sum_t (dr_jt/del_jk) . g_r[j][t] + (dv_jt/del_jk) . g_v[j][t]
// for el = (n0, e0, i0, RAAN0, argp0, M0, B*), through propagation and sgp4init
// (the paper's differentiable propagator, Sec. 5).
//
// Kernels:
//  * adjoint_prop_kernel64 / adjoint_prop_kernel_x2: one block per satellite; each
//    thread recomputes its states forward (forward64, or forward32x2 for two
//    consecutive times in packed FP32: the same formulations as the propagation
//    kernels) and runs the hand-written reverse sweep of the propagation, giving the
//    adjoints of the 33 record fields the propagation reads.  A thread sums them over
//    its states in registers, the block over its threads, and the partial sums are
//    added in FP64.  The Kepler solve is differentiated at its root (implicit
//    function theorem); the clamps and threshold decisions are constants of the sweep.
//  * adjoint_init_kernel: one thread per satellite pushes the 7 element directions
//    through sgp4init with dual numbers (the record build is per satellite, so
//    forward mode costs little next to the per-state sweep; FP32 duals for the FP32
//    path) and contracts the record-field Jacobian with the accumulated adjoints.
//  * fit_jacobian_kernel + fit_step_kernel: one Levenberg-Marquardt step of batch
//    least squares per satellite (three reverse sweeps per state after one forward).
// States whose status is 1, 2 or 4 (NaN output) contribute nothing.
//
// The FP32 variants run every per-state operation in FP32 (with the double-float
// n*t phase of the FP32 propagation) and use FP64 only to add the warps' partial sums
// and for states inside the FP32 path's guard bands, which go through the FP64 sweep
// as in the propagation.  On B300 the FP64 unit retires a warp instruction per tens of
// cycles, so a handful of FP64 operations per state would bound the whole kernel.
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "sgp4.h"
#include "sgp4_device.cuh"
#include "sgp4_init_math.cuh"
#include "sgp4_kernels.cuh"
#include "sgp4_sweep.cuh"
#include "sgp4_sweep32x2.cuh"

namespace sgp4 {

namespace {

struct AdjArgs {
  RecordPtrs rp;
  Geo g;
  GeoF gf;
  const double* tsince;
  int64_t T;
  int per_sat;
  const void* grad_r;
  const void* grad_v;
  double* field_bar;   // [n][kNumAdj], workspace
};


// The FP64 sweep: the states of satellite j handled by this thread, forward and reverse,
// the field adjoints summed into acc.
__device__ __forceinline__ void prop_loop64(const AdjArgs& a, const SatShared<double>& sat,
                                            double (&acc)[kNumAdj], int64_t j) {
  const double* gr = static_cast<const double*>(a.grad_r);
  const double* gv = static_cast<const double*>(a.grad_v);
  Fwd<double> f;
  for (int64_t i = threadIdx.x; i < a.T; i += kAdjThreads) {
    const int64_t s = j * a.T + i;
    const double t = a.per_sat ? __ldg(a.tsince + s) : __ldg(a.tsince + i);
    double g_r[3], g_v[3];
    for (int c = 0; c < 3; ++c) {
      g_r[c] = gr ? gr[s * 3 + c] : 0.0;
      g_v[c] = gv ? gv[s * 3 + c] : 0.0;
    }
    if (usable(forward64(sat.rc, a.g, t, f)))
      reverse(f, sat.k, g_r, g_v, [&](int q, double v) { acc[q] += v; });
  }
}

__global__ void __launch_bounds__(kAdjThreads, 1) adjoint_prop_kernel64(AdjArgs a) {
  __shared__ double part[kNumAdj][kAdjWarps];
  __shared__ SatShared<double> sat;
  const int tid = threadIdx.x;
  const int64_t j = blockIdx.x;
  if (tid == 0) load_sat(a.rp, a.g, a.gf, j, sat);
  __syncthreads();
  if (sat.rc.flags & kFlagDeep) {   // deep-space records are not differentiated: zero
    if (tid < kNumAdj) a.field_bar[j * kNumAdj + tid] = 0.0;
    return;
  }
  double acc[kNumAdj];
#pragma unroll
  for (int q = 0; q < kNumAdj; ++q) acc[q] = 0.0;
  prop_loop64(a, sat, acc, j);
#pragma unroll
  for (int q = 0; q < kNumAdj; ++q) warp_partial(acc[q], q, part);
  __syncthreads();
  if (tid < kNumAdj) {
    double sum = 0.0;
    for (int w = 0; w < kAdjWarps; ++w) sum += part[tid][w];
    a.field_bar[j * kNumAdj + tid] = sum;
  }
}

// The FP32 sweep: two consecutive times of the satellite per thread in packed FP32
// (forward32x2 and the reverse sweep over P2), one block of kAdj2Threads per satellite.
// A pair whose two states are both usable is swept packed; the states of every other
// pair are queued (guard-band states for the FP64 sweep, usable ones for the scalar
// FP32 sweep) and swept one by one after the loop, so that a single call of either
// sweep in the loop does not cost the loop its registers.  With more than kAdjFixCap
// queued the block runs the packed forward over the satellite's pairs again to find
// them.  Each thread's slot holds its pair's forward values (49 8-byte words: an odd
// count, so the 16 threads of a half-warp's 8-byte accesses hit distinct bank pairs).
// Against the scalar FP32 sweep (one state per thread, 128 threads, 6 blocks per SM)
// it issues 570 instead of 906 instructions per state; the fitting workload's
// sgp4_adjoint (10,000 x 500) went 0.1925 -> 0.166 ms on B300.  The thread's 33 sums are
// kept as floats (the pair's two adjoints added first) rather than as pairs: 33
// registers fewer, so that eight blocks of 64 per SM fit in 128 registers each (the
// 49-word slot lets eight fit in shared memory): 0.166 ms, against 0.170 for pairs of
// sums at six blocks (168 registers), 0.186 for pairs at eight (spills in the loop) and
// 0.227 at four.
constexpr int kAdj2Threads = 64;
#ifndef SGP4_ADJ2_MIN_BLOCKS
#define SGP4_ADJ2_MIN_BLOCKS 8
#endif
constexpr int kAdj2MinBlocks = SGP4_ADJ2_MIN_BLOCKS;
constexpr int kAdjFixCap = 256;
constexpr int kQueueScalar = 1 << 30;   // queue entry: an FP32 state (else an FP64 one)
static_assert((sizeof(Fwd<P2>) / 8) % 2 == 1, "odd 8-byte word count for conflict-free rows");
static_assert(kNumAdj <= kAdj2Threads, "one column sum per thread");

struct AdjFixQueue {
  int i[kAdjFixCap];
  int n;   // states queued (above kAdjFixCap: the queue overflowed)
};

__device__ __forceinline__ double adj_time(const AdjArgs& a, int64_t j, int64_t i) {
  return a.per_sat ? __ldg(a.tsince + j * a.T + i) : __ldg(a.tsince + i);
}

// Past the capacity (or for an index the entry cannot hold) the block rescans its pairs
// after the loop anyway, so the count stops there: it stays within kAdjFixCap plus the
// block's threads, however many states a satellite has.
__device__ __forceinline__ void adj_enqueue(AdjFixQueue* fq, int64_t i, bool scalar) {
  if (i >= kQueueScalar || *reinterpret_cast<volatile int*>(&fq->n) > kAdjFixCap) {
    atomicMax(&fq->n, kAdjFixCap + 1);
    return;
  }
  const int slot = atomicAdd(&fq->n, 1);
  if (slot < kAdjFixCap) fq->i[slot] = (int)i | (scalar ? kQueueScalar : 0);
}

// One state of satellite j swept on its own, its field adjoints added to row: through
// the FP64 sweep (fp64) or the scalar FP32 one (which may still hand it to FP64).
__device__ __forceinline__ void adj_sweep_one(const AdjArgs& a, const SatShared<float>& sat,
                                              float* row, int64_t j, int64_t i, bool fp64) {
  const float* gr = static_cast<const float*>(a.grad_r);
  const float* gv = static_cast<const float*>(a.grad_v);
  const int64_t s = j * a.T + i;
  const double t = adj_time(a, j, i);
  float g_r[3], g_v[3];
  for (int c = 0; c < 3; ++c) {
    g_r[c] = gr ? gr[s * 3 + c] : 0.0f;
    g_v[c] = gv ? gv[s * 3 + c] : 0.0f;
  }
  if (!fp64) {
    Fwd<float> fl;
    float th, tl;
    split_double(t, th, tl);
    const int code = forward32(sat.rc, a.gf, th, tl, fl);
    if (code != kRecomputeFP64) {
      if (usable(code)) reverse(fl, sat.k, g_r, g_v, [&](int q, float v) { row[q] += v; });
      return;
    }
  }
  adjoint_fallback(a.rp, a.g, j, t, g_r[0], g_r[1], g_r[2], g_v[0], g_v[1], g_v[2], row,
                   nullptr, nullptr, true);
}

// The packed forward of pair p (times 2p, 2p + 1) into f; code[1] = kAbsentState past
// the last time.
// The times of pair p (the first one twice past the last time).
__device__ __forceinline__ void adj_pair_times(const AdjArgs& a, int64_t j, int64_t p,
                                               double& t0, double& t1) {
  t0 = adj_time(a, j, 2 * p);
  t1 = 2 * p + 1 < a.T ? adj_time(a, j, 2 * p + 1) : t0;
}

__device__ __forceinline__ void adj_forward_times(const AdjArgs& a, const SatShared<float>& sat,
                                                  int64_t p, double t0, double t1, Fwd<P2>& f,
                                                  int code[2]) {
  float2 th, tl;
  split_double(t0, th.x, tl.x);
  split_double(t1, th.y, tl.y);
  forward32x2(sat.rc, a.gf, th, tl, f, code);
  if (2 * p + 1 >= a.T) code[1] = kAbsentState;
}

__device__ __forceinline__ void adj_forward_pair(const AdjArgs& a, const SatShared<float>& sat,
                                                 int64_t j, int64_t p, Fwd<P2>& f, int code[2]) {
  double t0, t1;
  adj_pair_times(a, j, p, t0, t1);
  adj_forward_times(a, sat, p, t0, t1, f, code);
}

// After the loop (the thread's sums in its row, a __syncthreads behind): the queued
// states of satellite j swept one by one into the rows of the threads that take them.
__device__ __forceinline__ void adj_fix_queued2(const AdjArgs& a, const SatShared<float>& sat,
                                                const AdjFixQueue* fq, float* row, int64_t j) {
  const int n = fq->n;
  if (n == 0) return;
  if (n <= kAdjFixCap) {
    for (int e = threadIdx.x; e < n; e += kAdj2Threads) {
      const int v = fq->i[e];
      adj_sweep_one(a, sat, row, j, v & (kQueueScalar - 1), !(v & kQueueScalar));
    }
    return;
  }
  const int64_t npair = (a.T + 1) / 2;
  for (int64_t p = threadIdx.x; p < npair; p += kAdj2Threads) {
    Fwd<P2> fl;
    int code[2];
    adj_forward_pair(a, sat, j, p, fl, code);
    if (usable(code[0]) && usable(code[1])) continue;   // swept in the loop
    for (int l = 0; l < 2; ++l)
      if (code[l] == kRecomputeFP64 || usable(code[l]))
        adj_sweep_one(a, sat, row, j, 2 * p + l, code[l] == kRecomputeFP64);
  }
}

__global__ void __launch_bounds__(kAdj2Threads, kAdj2MinBlocks) adjoint_prop_kernel_x2(AdjArgs a) {
  __shared__ SatShared<float> sat;
  __shared__ Fwd<P2> sfwd[kAdj2Threads];
  __shared__ AdjFixQueue s_fq;
  const int tid = threadIdx.x;
  const int64_t j = blockIdx.x;
  if (tid == 0) {
    load_sat(a.rp, a.g, a.gf, j, sat);
    s_fq.n = 0;
  }
  __syncthreads();
  if (sat.rc.flags & kFlagDeep) {   // deep-space records are not differentiated: zero
    if (tid < kNumAdj) a.field_bar[j * kNumAdj + tid] = 0.0;
    return;
  }
  const float* gr = static_cast<const float*>(a.grad_r);
  const float* gv = static_cast<const float*>(a.grad_v);
  float acc[kNumAdj];
#pragma unroll
  for (int q = 0; q < kNumAdj; ++q) acc[q] = 0.0f;
  Fwd<P2>& f = sfwd[tid];
  const int64_t npair = (a.T + 1) / 2;
  double tn0 = 0.0, tn1 = 0.0;   // the times of the thread's next pair, loaded ahead
  if (tid < npair) adj_pair_times(a, j, tid, tn0, tn1);
  for (int64_t p = tid; p < npair; p += kAdj2Threads) {
    const double t0 = tn0, t1 = tn1;
    if (p + kAdj2Threads < npair) adj_pair_times(a, j, p + kAdj2Threads, tn0, tn1);
    // the pair's output adjoints first, so that their loads from memory overlap the
    // forward pass (the second state's are read only when it exists)
    const int64_t s = j * a.T + 2 * p;
    const int64_t s1 = 2 * p + 1 < a.T ? s + 1 : s;
    P2 g_r[3], g_v[3];
    for (int c = 0; c < 3; ++c) {
      g_r[c] = gr ? P2(make_float2(__ldcs(gr + s * 3 + c), __ldcs(gr + s1 * 3 + c))) : P2(0.0f);
      g_v[c] = gv ? P2(make_float2(__ldcs(gv + s * 3 + c), __ldcs(gv + s1 * 3 + c))) : P2(0.0f);
    }
    int code[2];
    adj_forward_times(a, sat, p, t0, t1, f, code);
    reload_barrier();
    if (usable(code[0]) && usable(code[1])) {
      reverse(f, sat.k, g_r, g_v, [&](int q, P2 v) { acc[q] += v.v.x + v.v.y; });
    } else {
      for (int l = 0; l < 2; ++l)
        if (code[l] == kRecomputeFP64 || usable(code[l]))
          adj_enqueue(&s_fq, 2 * p + l, code[l] != kRecomputeFP64);
    }
  }
  // Block sum through the slots, free now: each thread writes its 33 sums to its row
  // (where the queued states' sweeps add theirs), then thread c < 33 sums column c over
  // the rows (consecutive words of a row: conflict-free) in four interleaved parts,
  // added in FP64.
  float* row = reinterpret_cast<float*>(&sfwd[tid]);
#pragma unroll
  for (int q = 0; q < kNumAdj; ++q) row[q] = acc[q];
  __syncthreads();   // (also: every state queued)
  adj_fix_queued2(a, sat, &s_fq, row, j);
  __syncthreads();
  if (tid < kNumAdj) {
    float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int r = 0; r < kAdj2Threads; r += 4)
      for (int k = 0; k < 4; ++k) s4[k] += reinterpret_cast<const float*>(&sfwd[r + k])[tid];
    a.field_bar[j * kNumAdj + tid] =
        ((double)s4[0] + (double)s4[1]) + ((double)s4[2] + (double)s4[3]);
  }
}

// One thread per satellite: grad[j] = field_bar[j] . J (the init Jacobian over R).
template <class R>
__global__ void __launch_bounds__(64) adjoint_init_kernel(const double* __restrict__ el,
                                                          const double* __restrict__ field_bar,
                                                          int64_t n, Geo g,
                                                          double* __restrict__ grad) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double e7[7];
  for (int k = 0; k < 7; ++k) e7[k] = el[j * 7 + k];
  R J[kNumAdj * 7];
  if (!init_jacobian(e7, g, J)) {
    for (int k = 0; k < 7; ++k) grad[j * 7 + k] = 0.0;
    return;
  }
  R out[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
  for (int q = 0; q < kNumAdj; ++q) {
    const R b = R(field_bar[j * kNumAdj + q]);
    for (int k = 0; k < 7; ++k) out[k] += b * J[q * 7 + k];
  }
  for (int k = 0; k < 7; ++k) grad[j * 7 + k] = out[k];
}

// One thread per satellite: the init Jacobian of the fit step into the workspace.
template <class R>
__global__ void __launch_bounds__(64) fit_jacobian_kernel(const double* __restrict__ el,
                                                          int64_t n, Geo g, R* __restrict__ jac) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double e7[7];
  for (int k = 0; k < 7; ++k) e7[k] = el[j * 7 + k];
  if (!init_jacobian(e7, g, jac + j * kNumAdj * 7))
    for (int q = 0; q < kNumAdj * 7; ++q) jac[j * kNumAdj * 7 + q] = R(0);
}

struct FitArgs {
  RecordPtrs rp;
  Geo g;
  GeoF gf;
  const double* el;      // [n][7]
  const void* jac;       // [n][kNumAdj][7] of the kernel's T, fit_jacobian_kernel
  const double* tsince;
  int64_t T;
  int per_sat;
  const double* r_obs;   // [n][T][3]
  double* normal;        // [n][36] out: A lower triangle (28), b (7), sse, in FP64
};

// The states of satellite j handled by this thread: residuals, the rows of dr/del
// (the field adjoints of the seeds e_x, e_y, e_z contracted with the init Jacobian Ji)
// and their sums A += J_c^T J_c, b += J_c^T res_c, sse += |res|^2.
template <class T>
__device__ __forceinline__ void fit_loop(const FitArgs& a, const SatShared<T>& sat, Fwd<T>& f,
                                         const T (*Ji)[7], T (&A)[28], T (&b)[7], T& sse,
                                         int64_t j) {
  for (int64_t i = threadIdx.x; i < a.T; i += kAdjThreads) {
    const int64_t s = j * a.T + i;
    const double t = a.per_sat ? __ldg(a.tsince + s) : __ldg(a.tsince + i);
    int code;
    bool fell_back = false;
    T r[3];
    float* slot = reinterpret_cast<float*>(&f);   // fallback: 33 adjoints + position
    if constexpr (sizeof(T) == 4) {
      float th, tl;
      split_double(t, th, tl);
      code = forward32(sat.rc, a.gf, th, tl, f);
      reload_barrier();
      if (code == kRecomputeFP64) {
        code = adjoint_fallback(a.rp, a.g, j, t, 1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, slot,
                                slot + kNumAdj);
        reload_barrier();
        fell_back = true;
      }
    } else {
      code = forward64(sat.rc, a.g, t, f);
    }
    if (!usable(code)) continue;
    if (fell_back) {
      r[0] = T(slot[kNumAdj]); r[1] = T(slot[kNumAdj + 1]); r[2] = T(slot[kNumAdj + 2]);
    } else {
      const T rs = f.rk * sat.k.re;
      const Frame<T> fr = frame_get(f);
      r[0] = rs * fr.Ux; r[1] = rs * fr.Uy; r[2] = rs * fr.Uz;
    }
    T res[3];
    for (int c = 0; c < 3; ++c) res[c] = r[c] - T(a.r_obs[s * 3 + c]);
    if (!(isfinite(res[0]) && isfinite(res[1]) && isfinite(res[2]))) continue;
    sse += res[0] * res[0] + res[1] * res[1] + res[2] * res[2];
    // Not unrolled: one copy of the sweep keeps the kernel within the instruction
    // cache (the unrolled form ran 8% slower, stalled on instruction fetch).
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
      T Jc[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
      auto contract = [&](int q, T v) {
#pragma unroll
        for (int m = 0; m < 7; ++m) Jc[m] += v * Ji[q][m];
      };
      if (fell_back) {
        if (c > 0) {
          adjoint_fallback(a.rp, a.g, j, t, c == 1 ? 1.0f : 0.0f, c == 2 ? 1.0f : 0.0f, 0.0f,
                           0.0f, 0.0f, 0.0f, slot, nullptr);
          reload_barrier();
        }
        for (int q = 0; q < kNumAdj; ++q) contract(q, T(slot[q]));
      } else {
        const T zero3[3] = {T(0), T(0), T(0)};
        const T seed[3] = {T(c == 0), T(c == 1), T(c == 2)};
        reverse(f, sat.k, seed, zero3, contract);
      }
      int idx = 0;
#pragma unroll
      for (int m = 0; m < 7; ++m) {
        b[m] += Jc[m] * res[c];
#pragma unroll
        for (int l = 0; l <= m; ++l, ++idx) A[idx] += Jc[m] * Jc[l];
      }
    }
  }
}

// Normal equations of one Gauss-Newton / Levenberg-Marquardt step of batch least
// squares per satellite (one block each): residuals res_t = r_t(el) - r_obs_t over the
// states with finite output, the position Jacobian J_t = dr_t/del (one forward and
// three reverse sweeps per state, contracted with the init Jacobian), A = sum J_t^T
// J_t and b = sum J_t^T res_t.  Per-thread sums in T, warp sums by shuffles, the
// warps' sums in FP64.  fit_solve_kernel then takes the step.
template <class T>
__global__ void __launch_bounds__(kAdjThreads, sizeof(T) == 4 ? kAdjMinBlocksFP32 : 1)
    fit_step_kernel(FitArgs a) {
  __shared__ T Ji[kNumAdj][7];
  __shared__ T part[36][kAdjWarps];
  __shared__ int s_ok;
  __shared__ SatShared<T> sat;
  __shared__ Fwd<T> sfwd[FwdSlot<T>::kRows];
  const int tid = threadIdx.x;
  const int64_t j = blockIdx.x;
  if (tid == 0) {
    double e7[7];
    for (int k = 0; k < 7; ++k) e7[k] = a.el[j * 7 + k];
    s_ok = elements_usable(e7) ? 1 : 0;
    load_sat(a.rp, a.g, a.gf, j, sat);
  }
  for (int q = tid; q < kNumAdj * 7; q += kAdjThreads)
    (&Ji[0][0])[q] = static_cast<const T*>(a.jac)[j * kNumAdj * 7 + q];
  __syncthreads();
  if (!s_ok) return;   // fit_solve_kernel keeps the elements of unusable records
  if (sat.rc.flags & kFlagDeep) {
    // deep-space records are not fitted: zero normal equations leave their elements
    // unchanged, with zero residual
    if (tid < 36) a.normal[j * 36 + tid] = 0.0;
    return;
  }
  T A[28], b[7], sse = T(0);
#pragma unroll
  for (int q = 0; q < 28; ++q) A[q] = T(0);
#pragma unroll
  for (int q = 0; q < 7; ++q) b[q] = T(0);
  if constexpr (sizeof(T) == 4) {
    fit_loop(a, sat, sfwd[tid], Ji, A, b, sse, j);
  } else {
    Fwd<T> f;
    fit_loop(a, sat, f, Ji, A, b, sse, j);
  }
#pragma unroll
  for (int q = 0; q < 28; ++q) warp_partial(A[q], q, part);
#pragma unroll
  for (int q = 0; q < 7; ++q) warp_partial(b[q], 28 + q, part);
  warp_partial(sse, 35, part);
  __syncthreads();
  if (tid < 36) {
    double v = 0.0;
    for (int w = 0; w < kAdjWarps; ++w) v += (double)part[tid][w];
    a.normal[j * 36 + tid] = v;
  }
}

// One thread per satellite: the Levenberg-Marquardt step from the normal equations
// (A lower triangle, b, sse) of fit_step_kernel: Jacobi scaling, damping, Cholesky.
// A thread per satellite shares each FP64 warp instruction among 32 satellites (the
// FP64 unit charges per warp instruction).
__global__ void __launch_bounds__(64) fit_solve_kernel(const double* __restrict__ el,
                                                       const double* __restrict__ normal,
                                                       const double* __restrict__ lambda,
                                                       int64_t n, double* __restrict__ el_out,
                                                       double* __restrict__ sse) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double e7[7];
  for (int k = 0; k < 7; ++k) e7[k] = el[j * 7 + k];
  if (!elements_usable(e7)) {
    for (int k = 0; k < 7; ++k) el_out[j * 7 + k] = e7[k];
    sse[j] = 0.0;
    return;
  }
  const double* S = normal + j * 36;
  double M[7][7], rhs[7], d[7];
  int q = 0;
  for (int m = 0; m < 7; ++m)
    for (int l = 0; l <= m; ++l, ++q) M[m][l] = M[l][m] = S[q];
  for (int m = 0; m < 7; ++m) d[m] = M[m][m] > 0.0 ? 1.0 / sqrt(M[m][m]) : 0.0;
  const double lam = lambda[j];
  for (int m = 0; m < 7; ++m) {
    for (int l = 0; l < 7; ++l) M[m][l] *= d[m] * d[l];
    M[m][m] = (d[m] > 0.0 ? M[m][m] : 1.0) * (1.0 + lam);
    rhs[m] = -S[28 + m] * d[m];
  }
  bool spd = true;
  for (int m = 0; m < 7 && spd; ++m) {
    for (int l = 0; l < m; ++l) M[m][m] -= M[m][l] * M[m][l];
    if (!(M[m][m] > 0.0)) { spd = false; break; }
    M[m][m] = sqrt(M[m][m]);
    for (int r2 = m + 1; r2 < 7; ++r2) {
      for (int l = 0; l < m; ++l) M[r2][m] -= M[r2][l] * M[m][l];
      M[r2][m] /= M[m][m];
    }
  }
  double x[7] = {0, 0, 0, 0, 0, 0, 0};
  if (spd) {
    for (int m = 0; m < 7; ++m) {            // forward substitution L y = rhs
      double v = rhs[m];
      for (int l = 0; l < m; ++l) v -= M[m][l] * x[l];
      x[m] = v / M[m][m];
    }
    for (int m = 6; m >= 0; --m) {           // back substitution L^T x = y
      double v = x[m];
      for (int l = m + 1; l < 7; ++l) v -= M[l][m] * x[l];
      x[m] = v / M[m][m];
    }
  }
  for (int m = 0; m < 7; ++m) el_out[j * 7 + m] = e7[m] + x[m] * d[m];
  sse[j] = S[35];
}

}  // namespace

// Workspace: the init Jacobians [n][kNumAdj][7] (of the sweep's precision, in a
// double-sized slot) and the normal equations [n][36] (FP64).
size_t fit_workspace_bytes(int64_t n) {
  return n <= 0 ? 0 : (size_t)n * (kNumAdj * 7 + 36) * sizeof(double);
}

cudaError_t launch_fit_step(const RecordPtrs& rp, const Geo& g, const double* el,
                            const double* tsince, int64_t T, int per_sat, bool fp32,
                            const double* r_obs, const double* lambda, double* el_out,
                            double* sse, double* workspace, cudaStream_t stream) {
  if (rp.n == 0) return cudaSuccess;
  const int threads = 64;
  const unsigned blocks = (unsigned)((rp.n + threads - 1) / threads);
  double* normal = workspace + rp.n * kNumAdj * 7;
  if (fp32)
    fit_jacobian_kernel<float><<<blocks, threads, 0, stream>>>(
        el, rp.n, g, reinterpret_cast<float*>(workspace));
  else
    fit_jacobian_kernel<double><<<blocks, threads, 0, stream>>>(el, rp.n, g, workspace);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  FitArgs a;
  a.rp = rp;
  a.g = g;
  a.gf = geo_float(g);
  a.el = el;
  a.jac = workspace;
  a.tsince = tsince;
  a.T = T;
  a.per_sat = per_sat;
  a.r_obs = r_obs;
  a.normal = normal;
  if (fp32) fit_step_kernel<float><<<(unsigned)rp.n, kAdjThreads, 0, stream>>>(a);
  else fit_step_kernel<double><<<(unsigned)rp.n, kAdjThreads, 0, stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  fit_solve_kernel<<<blocks, threads, 0, stream>>>(el, normal, lambda, rp.n, el_out, sse);
  return cudaGetLastError();
}

cudaError_t launch_init_jacobian(const double* el, int64_t n, const Geo& g, bool fp32,
                                 void* out, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const int threads = 64;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (fp32)
    fit_jacobian_kernel<float><<<blocks, threads, 0, stream>>>(el, n, g, static_cast<float*>(out));
  else
    fit_jacobian_kernel<double><<<blocks, threads, 0, stream>>>(el, n, g,
                                                                 static_cast<double*>(out));
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
  a.gf = geo_float(g);
  a.tsince = tsince;
  a.T = T;
  a.per_sat = per_sat;
  a.grad_r = grad_r;
  a.grad_v = grad_v;
  a.field_bar = workspace;
  if (fp32) adjoint_prop_kernel_x2<<<(unsigned)rp.n, kAdj2Threads, 0, stream>>>(a);
  else adjoint_prop_kernel64<<<(unsigned)rp.n, kAdjThreads, 0, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int threads = 64;
  const unsigned blocks = (unsigned)((rp.n + threads - 1) / threads);
  if (fp32)
    adjoint_init_kernel<float><<<blocks, threads, 0, stream>>>(el, workspace, rp.n, g, grad_el);
  else
    adjoint_init_kernel<double><<<blocks, threads, 0, stream>>>(el, workspace, rp.n, g, grad_el);
  return cudaGetLastError();
}

}  // namespace sgp4
