// Host-side launch wrappers of the SGP4 kernels (internal to the library).
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "sgp4.h"
#include "sgp4_device.cuh"

namespace sgp4 {

cudaError_t launch_init(const double* el, const int32_t* epoch_day, const double* epoch_frac,
                        const RecordPtrs& rp, const Geo& g, int32_t* init_status,
                        cudaStream_t stream);

struct PropArgs {
  RecordPtrs rp;
  Geo g;
  GeoF gf;        // float copy of g, made on the host
  const double* tsince;
  const int32_t* jd_day = nullptr;   // absolute-time grid (Julian day + fraction), or null
  const double* jd_frac = nullptr;
  int64_t t_count;
  int grid_per_sat;
  void* r;
  void* v;
  int32_t* status;
  unsigned long long* fixups;
};

cudaError_t launch_propagate64(const PropArgs& a, cudaStream_t stream);
cudaError_t launch_propagate32(const PropArgs& a, cudaStream_t stream);

struct BatchArgs {
  RecordPtrs rp;
  Geo g;
  GeoF gf;
  const double* tsince;          // all requests' grids, concatenated
  const sgp4_request* reqs;      // [n_req], device
  const int64_t* tile_start;     // [n_req + 1], device: exclusive prefix of tile counts
  int32_t n_req;
  int64_t tile_states;
  unsigned long long* counter;   // next tile index (reset before every launch)
  void* r;
  void* v;
  int32_t* status;
  unsigned long long* fixups;
};

// Persistent grid of the batched kernel: grid_blocks if positive, else one full wave
// (SMs x resident blocks), at most one block per tile.  Queries the device: call it
// outside stream capture.
int64_t batched_grid(bool fp32, int64_t total_tiles, int grid_blocks);

// Resets the tile counter, then launches the persistent batched kernel on `grid` blocks.
cudaError_t launch_batched(const BatchArgs& a, bool fp32, int64_t total_tiles, int64_t grid,
                           cudaStream_t stream);

// Adjoint: field-adjoint workspace bytes and the two-kernel launch.
size_t adjoint_workspace_bytes(int64_t n);
cudaError_t launch_adjoint(const RecordPtrs& rp, const Geo& g, const double* el,
                           const double* tsince, int64_t T, int per_sat, bool fp32,
                           const void* grad_r, const void* grad_v, double* grad_el,
                           double* workspace, cudaStream_t stream);

// One batch-least-squares (Levenberg-Marquardt) step per satellite: the init-Jacobian
// workspace bytes and the two-kernel launch.
size_t fit_workspace_bytes(int64_t n);
cudaError_t launch_fit_step(const RecordPtrs& rp, const Geo& g, const double* el,
                            const double* tsince, int64_t T, int per_sat, bool fp32,
                            const double* r_obs, const double* lambda, double* el_out,
                            double* sse, double* workspace, cudaStream_t stream);

// Record-field Jacobian of sgp4init per satellite, [n][33][7] of float (fp32) or double.
cudaError_t launch_init_jacobian(const double* el, int64_t n, const Geo& g, bool fp32,
                                 void* out, cudaStream_t stream);

// Per-state Jacobians d(r, v)/d(elements) and covariance propagation.
struct JacOut {
  void* r;            // [n][T][3] or null
  void* v;            // [n][T][3] or null
  int32_t* status;    // [n][T]
  void* jac;          // [n][T][6][7] or null
  const double* cov;  // [n][7][7] element covariance, or null
  void* cov_out;      // [n][T][21] upper triangle of J C J^T, or null
};
size_t jacobian_workspace_bytes(int64_t n);
cudaError_t launch_jacobian(const RecordPtrs& rp, const Geo& g, const double* el,
                            const double* tsince, int64_t T, int per_sat, bool fp32,
                            const JacOut& out, void* workspace, cudaStream_t stream);

// Work tiles of one batched request (n satellites x t_count times): a tile is
// tile_states consecutive states' worth of units, walked in units of four states of
// one satellite by the FP32 kernel and of two by the FP64 kernel; the plan, built
// before the precision is known, gives each request the larger of the two counts (a
// kernel skips tiles past its own units).  tile_states is a multiple of 128.
__host__ __device__ inline int64_t units_per_sat(int64_t t_count, int states_per_unit) {
  return (t_count + states_per_unit - 1) / states_per_unit;
}
__host__ __device__ inline int64_t request_tiles(int64_t n, int64_t t_count, int64_t tile_states) {
  const int64_t u2 = n * units_per_sat(t_count, 2), p2 = tile_states / 2;
  const int64_t u4 = n * units_per_sat(t_count, 4), p4 = tile_states / 4;
  const int64_t t2 = (u2 + p2 - 1) / p2, t4 = (u4 + p4 - 1) / p4;
  return t2 > t4 ? t2 : t4;
}

// Earth model of the call's constants (host side, once per call).
inline Geo make_geo(const sgp4_consts& c) {
  Geo g;
  g.xke = 60.0 / std::sqrt(c.radius_km * c.radius_km * c.radius_km / c.mu_km3s2);
  g.j2 = c.j2;
  g.j3oj2 = (c.j2 != 0.0) ? c.j3 / c.j2 : 0.0;
  g.j4 = c.j4;
  g.re = c.radius_km;
  g.vkmps = c.radius_km * g.xke / 60.0;
  g.inv_xke = 1.0 / g.xke;
  g.inv_re = 1.0 / c.radius_km;
  return g;
}

// Float copy of the Earth model for the FP32 path (host side, once per call).
inline GeoF geo_float(const Geo& g) {
  GeoF gf;
  gf.xke = (float)g.xke;
  gf.inv_xke = (float)(1.0 / g.xke);
  gf.j2 = (float)g.j2;
  gf.re = (float)g.re;
  gf.vkmps = (float)g.vkmps;
  gf.half_j2 = (float)(0.5 * g.j2);
  return gf;
}

// SM count of the current device.
int device_sm_count();

}  // namespace sgp4
