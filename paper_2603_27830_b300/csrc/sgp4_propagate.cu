// Propagation kernels: one (satellite, time) state per thread (paper Sec. 2.2,
// "Vectorisation": f(s, t) under a vmap over times composed with a vmap over
// satellites), with
//   * a persistent grid of one wave, each block owning one contiguous range of the
//     flattened [n][T] state space, so consecutive iterations of a thread walk along
//     the time axis of the same satellite and its record stays in L1 (FP32) or in
//     registers (FP64);
//   * outputs staged in shared memory and written back with 16-byte streaming
//     stores ([n][T][3] is AoS per state, so a block's 128 states are 1.5 KB (FP32)
//     or 3 KB (FP64) of contiguous r, the same of v, and 512 B of status).
#include <algorithm>

#include "sgp4_device.cuh"
#include "sgp4_kernels.cuh"

namespace sgp4 {

namespace {

constexpr int kThreads = 128;
// Minimum resident 128-thread blocks per SM requested from the register allocator.
// The FP32 kernel is latency bound at low occupancy: on B300, 8 blocks (64
// registers) ran 5% (Starlink) to 15% (catalogue) faster than 4 blocks (128
// registers).  The FP64 kernel is bound by the FP64 pipe and keeps 4.
#ifndef SGP4_MIN_BLOCKS_FP32
#define SGP4_MIN_BLOCKS_FP32 8
#endif
#ifndef SGP4_MIN_BLOCKS_FP64
#define SGP4_MIN_BLOCKS_FP64 4
#endif

template <typename OutT>
__device__ __forceinline__ void nan_fill(OutT x[3]) {
  x[0] = x[1] = x[2] = OutT(__longlong_as_double(0x7ff8000000000000LL));
}

template <bool kFP32>
__global__ void __launch_bounds__(kThreads, kFP32 ? SGP4_MIN_BLOCKS_FP32 : SGP4_MIN_BLOCKS_FP64)
    propagate_kernel(PropArgs a, int64_t chunk) {
  using OutT = typename std::conditional<kFP32, float, double>::type;
  __shared__ __align__(16) OutT s_r[3 * kThreads];
  __shared__ __align__(16) OutT s_v[3 * kThreads];
  __shared__ __align__(16) int32_t s_st[kThreads];

  const int tid = threadIdx.x;
  const int64_t T = a.t_count;
  const int64_t total = a.rp.n * T;
  const int64_t beg = (int64_t)blockIdx.x * chunk;
  const int64_t end = min(total, beg + chunk);
  if (beg >= end) return;

  // (j, i) of this thread's first state; advanced incrementally afterwards.
  int64_t j = (beg + tid) / T;
  int64_t i = (beg + tid) - j * T;
  int64_t cur = -1;
  Rec64 rc64;
  GeoF gf;
  if (kFP32) {
    gf.xke = (float)a.g.xke;
    gf.inv_xke = (float)(1.0 / a.g.xke);
    gf.j2 = (float)a.g.j2;
    gf.re = (float)a.g.re;
    gf.vkmps = (float)a.g.vkmps;
  }
  unsigned long long nfix = 0;

  for (int64_t base = beg; base < end; base += kThreads) {
    const int64_t idx = base + tid;
    OutT rr[3], vv[3];
    int code = 0;
    if (idx < end) {
      if (!kFP32 && j != cur) {
        rc64 = load_rec64(a.rp, j);
        cur = j;
      }
      const double t = a.grid_per_sat ? __ldg(a.tsince + j * T + i) : __ldg(a.tsince + i);
      if (kFP32) {
        // The 160-byte FP32 row is re-read every state (ten 16-byte loads that L1
        // serves as broadcasts) instead of being held in registers across states.
        const Rec32 rc32 = load_rec32(a.rp, j);
        float th, tl;
        split_double(t, th, tl);
        float r32[3], v32[3];
        code = state32(rc32, gf, th, tl, r32, v32);
        if (code == kRecomputeFP64) {
          code = state64_fallback(a.rp, a.g, j, t, r32, v32);
          ++nfix;
        }
        for (int c = 0; c < 3; ++c) { rr[c] = (OutT)r32[c]; vv[c] = (OutT)v32[c]; }
      } else {
        double r64[3], v64[3];
        code = state64(rc64, a.g, t, r64, v64);
        for (int c = 0; c < 3; ++c) { rr[c] = (OutT)r64[c]; vv[c] = (OutT)v64[c]; }
      }
      if (code != 0 && code != 6) { nan_fill(rr); nan_fill(vv); }
    }
    s_r[3 * tid + 0] = rr[0]; s_r[3 * tid + 1] = rr[1]; s_r[3 * tid + 2] = rr[2];
    s_v[3 * tid + 0] = vv[0]; s_v[3 * tid + 1] = vv[1]; s_v[3 * tid + 2] = vv[2];
    s_st[tid] = code;
    __syncthreads();

    OutT* gr = static_cast<OutT*>(a.r) + base * 3;
    OutT* gv = static_cast<OutT*>(a.v) + base * 3;
    int32_t* gs = a.status + base;
    const int64_t cnt = min((int64_t)kThreads, end - base);
    if (cnt == kThreads) {
      constexpr int kVec = 3 * kThreads * (int)sizeof(OutT) / 16;
      constexpr int kVecSt = kThreads * 4 / 16;
      const int4* sr = reinterpret_cast<const int4*>(s_r);
      const int4* sv = reinterpret_cast<const int4*>(s_v);
      const int4* ss = reinterpret_cast<const int4*>(s_st);
      for (int k = tid; k < kVec; k += kThreads) {
        __stcs(reinterpret_cast<int4*>(gr) + k, sr[k]);
        __stcs(reinterpret_cast<int4*>(gv) + k, sv[k]);
      }
      if (tid < kVecSt) __stcs(reinterpret_cast<int4*>(gs) + tid, ss[tid]);
    } else {
      for (int k = tid; k < 3 * cnt; k += kThreads) { gr[k] = s_r[k]; gv[k] = s_v[k]; }
      if (tid < cnt) gs[tid] = s_st[tid];
    }
    __syncthreads();

    i += kThreads;
    if (i >= T) {
      const int64_t q = i / T;
      j += q;
      i -= q * T;
    }
  }
  if (kFP32 && a.fixups && nfix) atomicAdd(a.fixups, nfix);
}

template <bool kFP32>
cudaError_t launch(const PropArgs& a, cudaStream_t stream) {
  const int64_t total = a.rp.n * a.t_count;
  if (total == 0) return cudaSuccess;
  static int blocks_per_sm[2] = {0, 0};   // per precision; same kernel on every device
  int& bps = blocks_per_sm[kFP32 ? 1 : 0];
  if (bps == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, propagate_kernel<kFP32>,
                                                                  kThreads, 0);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
  }
  const int64_t tiles = (total + kThreads - 1) / kThreads;
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)device_sm_count() * bps);
  const int64_t chunk = ((tiles + grid - 1) / grid) * kThreads;
  const int64_t blocks = (total + chunk - 1) / chunk;
  propagate_kernel<kFP32><<<(unsigned)blocks, kThreads, 0, stream>>>(a, chunk);
  return cudaGetLastError();
}

}  // namespace

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

cudaError_t launch_propagate64(const PropArgs& a, cudaStream_t stream) {
  return launch<false>(a, stream);
}

cudaError_t launch_propagate32(const PropArgs& a, cudaStream_t stream) {
  return launch<true>(a, stream);
}

}  // namespace sgp4
