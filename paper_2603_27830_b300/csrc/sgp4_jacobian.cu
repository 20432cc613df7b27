// Per-state Jacobians of the TEME state (r, v) with respect to the mean elements
// (n0, e0, i0, RAAN0, argp0, M0, B*), through sgp4init and the propagation, and the
// propagation of an element covariance C to the state covariance J C J^T: the
// derivatives of the paper's differentiable propagator (Sec. 5) in the form
// conjunction screening uses.
//
// One block per satellite.  Each thread takes its states: one forward pass (kept in
// the thread's shared-memory slot on the FP32 path), then one reverse sweep per output
// component (six seeds e_rx .. e_vz), each contracted with the record-field Jacobian
// of sgp4init (computed once per satellite by launch_init_jacobian) into a row of
// J = d(r, v)/d(elements).  Guard-band states of the FP32 path use the FP64 sweep.
// States with status 1, 2 or 4 get NaN outputs, like their r and v.  Deep-space
// records are not differentiated: their states get status 5 and NaN outputs.
#include <cmath>
#include <cstdint>

#include "sgp4.h"
#include "sgp4_device.cuh"
#include "sgp4_kernels.cuh"
#include "sgp4_sweep.cuh"

namespace sgp4 {

namespace {

struct JacArgs {
  RecordPtrs rp;
  Geo g;
  GeoF gf;
  const double* el;       // [n][7]
  const void* jinit;      // [n][kNumAdj][7] of the kernel's T
  const double* tsince;
  int64_t T;
  int per_sat;
  JacOut out;
};

template <class T>
__device__ __forceinline__ void jac_loop(const JacArgs& a, const SatShared<T>& sat, Fwd<T>& f,
                                         const T (*Ji)[7], const T (*C)[7], int64_t j) {
  const T qnan = T(__longlong_as_double(0x7ff8000000000000LL));
  for (int64_t i = threadIdx.x; i < a.T; i += kAdjThreads) {
    const int64_t s = j * a.T + i;
    const double t = a.per_sat ? __ldg(a.tsince + s) : __ldg(a.tsince + i);
    int code;
    bool fell_back = false;
    float* slot = reinterpret_cast<float*>(&f);   // fallback: 33 adjoints, r, v
    if constexpr (sizeof(T) == 4) {
      float th, tl;
      split_double(t, th, tl);
      code = forward32(sat.rc, a.gf, th, tl, f);
      reload_barrier();
      if (code == kRecomputeFP64) {
        code = adjoint_fallback(a.rp, a.g, j, t, 1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, slot,
                                slot + kNumAdj, slot + kNumAdj + 3);
        reload_barrier();
        fell_back = true;
      }
    } else {
      code = forward64(sat.rc, a.g, t, f);
    }
    a.out.status[s] = code;
    T* r_out = static_cast<T*>(a.out.r);
    T* v_out = static_cast<T*>(a.out.v);
    T* jac = static_cast<T*>(a.out.jac);
    T* cov = static_cast<T*>(a.out.cov_out);
    if (!usable(code)) {
      for (int c = 0; c < 3; ++c) {
        if (r_out) r_out[s * 3 + c] = qnan;
        if (v_out) v_out[s * 3 + c] = qnan;
      }
      if (jac)
        for (int q = 0; q < 42; ++q) jac[s * 42 + q] = qnan;
      if (cov)
        for (int q = 0; q < 21; ++q) cov[s * 21 + q] = qnan;
      continue;
    }
    if (fell_back) {
      for (int c = 0; c < 3; ++c) {
        if (r_out) r_out[s * 3 + c] = T(slot[kNumAdj + c]);
        if (v_out) v_out[s * 3 + c] = T(slot[kNumAdj + 3 + c]);
      }
    } else {
      const T rs = f.rk * sat.k.re;
      const Frame<T> fr = frame_get(f);
      if (r_out) {
        r_out[s * 3 + 0] = rs * fr.Ux; r_out[s * 3 + 1] = rs * fr.Uy; r_out[s * 3 + 2] = rs * fr.Uz;
      }
      if (v_out) {
        const T vk = sat.k.vk;
        v_out[s * 3 + 0] = vk * (f.rdotk * fr.Ux + f.rfdotk * fr.Vx);
        v_out[s * 3 + 1] = vk * (f.rdotk * fr.Uy + f.rfdotk * fr.Vy);
        v_out[s * 3 + 2] = vk * (f.rdotk * fr.Uz + f.rfdotk * fr.Vz);
      }
    }
    if (!jac && !cov) continue;
    T J[6][7];
    // One sweep per output component; not unrolled (one copy of the sweep's code).
#pragma unroll 1
    for (int c = 0; c < 6; ++c) {
      T row[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
      auto contract = [&](int q, T val) {
#pragma unroll
        for (int m = 0; m < 7; ++m) row[m] += val * Ji[q][m];
      };
      if (fell_back) {
        if (c > 0) {
          adjoint_fallback(a.rp, a.g, j, t, c == 0 ? 1.0f : 0.0f, c == 1 ? 1.0f : 0.0f,
                           c == 2 ? 1.0f : 0.0f, c == 3 ? 1.0f : 0.0f, c == 4 ? 1.0f : 0.0f,
                           c == 5 ? 1.0f : 0.0f, slot, nullptr);
          reload_barrier();
        }
        for (int q = 0; q < kNumAdj; ++q) contract(q, T(slot[q]));
      } else {
        const T gr[3] = {T(c == 0), T(c == 1), T(c == 2)};
        const T gv[3] = {T(c == 3), T(c == 4), T(c == 5)};
        reverse(f, sat.k, gr, gv, contract);
      }
#pragma unroll
      for (int m = 0; m < 7; ++m) J[c][m] = row[m];
    }
    if (jac)
      for (int c = 0; c < 6; ++c)
        for (int m = 0; m < 7; ++m) jac[s * 42 + c * 7 + m] = J[c][m];
    if (cov) {
      // P = J C J^T, upper triangle row by row: P[p][q] = (J_p C) . J_q
      // J sits in local memory (the seed loop writes its rows at a run-time index); read
      // each row once into registers, the loops unrolled (5% on the FP32 kernel)
      T Jr[6][7];
#pragma unroll
      for (int p = 0; p < 6; ++p)
#pragma unroll
        for (int m = 0; m < 7; ++m) Jr[p][m] = J[p][m];
      int idx = 0;
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        T w[7];
#pragma unroll
        for (int l = 0; l < 7; ++l) {
          T acc = T(0);
#pragma unroll
          for (int m = 0; m < 7; ++m) acc += Jr[p][m] * C[m][l];
          w[l] = acc;
        }
#pragma unroll
        for (int q = p; q < 6; ++q, ++idx) {
          T acc = T(0);
#pragma unroll
          for (int l = 0; l < 7; ++l) acc += w[l] * Jr[q][l];
          cov[s * 21 + idx] = acc;
        }
      }
    }
  }
}

// Resident blocks per SM asked of the register allocator for the FP32 kernel: four, not
// the six of the other FP32 sweeps.  Each thread's 6 x 7 Jacobian sits in local memory
// (the seed loop writes its rows at a run-time index), and at six blocks that local
// memory (768 threads x 168 B) no longer fitted the L1 left beside the blocks' shared
// memory: sgp4_jacobian with covariance on 10,000 x 500 took 1.99 ms at six blocks,
// 1.84 at four, 1.98 at three and 1.90 at two (CUDA events, A/B on one box).
constexpr int kJacMinBlocksFP32 = 4;

template <class T>
__global__ void __launch_bounds__(kAdjThreads, sizeof(T) == 4 ? kJacMinBlocksFP32 : 1)
    jacobian_kernel(JacArgs a) {
  __shared__ T Ji[kNumAdj][7];
  __shared__ T C[7][7];
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
    if (sat.rc.flags & kFlagDeep) s_ok = 0;
  }
  for (int q = tid; q < kNumAdj * 7; q += kAdjThreads)
    (&Ji[0][0])[q] = static_cast<const T*>(a.jinit)[j * kNumAdj * 7 + q];
  if (a.out.cov && tid < 49) (&C[0][0])[tid] = T(a.out.cov[j * 49 + tid]);
  __syncthreads();
  if (!s_ok) {
    // unusable elements: the record's fatal status with NaN outputs, as propagation;
    // deep-space records (not differentiated here): status 5, NaN outputs
    const T qnan = T(__longlong_as_double(0x7ff8000000000000LL));
    const int fatal = (sat.rc.flags >> kFatalShift) & 0xff;
    const int code = (sat.rc.flags & kFlagDeep) ? 5 : fatal ? fatal : 1;
    for (int64_t i = tid; i < a.T; i += kAdjThreads) {
      const int64_t s = j * a.T + i;
      a.out.status[s] = code;
      for (int c = 0; c < 3; ++c) {
        if (a.out.r) static_cast<T*>(a.out.r)[s * 3 + c] = qnan;
        if (a.out.v) static_cast<T*>(a.out.v)[s * 3 + c] = qnan;
      }
      if (a.out.jac)
        for (int q = 0; q < 42; ++q) static_cast<T*>(a.out.jac)[s * 42 + q] = qnan;
      if (a.out.cov_out)
        for (int q = 0; q < 21; ++q) static_cast<T*>(a.out.cov_out)[s * 21 + q] = qnan;
    }
    return;
  }
  if constexpr (sizeof(T) == 4) {
    jac_loop(a, sat, sfwd[tid], Ji, C, j);
  } else {
    Fwd<T> f;
    jac_loop(a, sat, f, Ji, C, j);
  }
}

}  // namespace

size_t jacobian_workspace_bytes(int64_t n) {
  return n <= 0 ? 0 : (size_t)n * kNumAdj * 7 * sizeof(double);
}

cudaError_t launch_jacobian(const RecordPtrs& rp, const Geo& g, const double* el,
                            const double* tsince, int64_t T, int per_sat, bool fp32,
                            const JacOut& out, void* workspace, cudaStream_t stream) {
  if (rp.n == 0 || T == 0) return cudaSuccess;
  cudaError_t e = launch_init_jacobian(el, rp.n, g, fp32, workspace, stream);
  if (e != cudaSuccess) return e;
  JacArgs a;
  a.rp = rp;
  a.g = g;
  a.gf = geo_float(g);
  a.el = el;
  a.jinit = workspace;
  a.tsince = tsince;
  a.T = T;
  a.per_sat = per_sat;
  a.out = out;
  if (fp32) jacobian_kernel<float><<<(unsigned)rp.n, kAdjThreads, 0, stream>>>(a);
  else jacobian_kernel<double><<<(unsigned)rp.n, kAdjThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace sgp4
