// Host-side launch wrappers of the SGP4 kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sgp4_device.cuh"

namespace sgp4 {

cudaError_t launch_init(const double* el, const int32_t* epoch_day, const double* epoch_frac,
                        const RecordPtrs& rp, const Geo& g, int32_t* init_status,
                        cudaStream_t stream);

struct PropArgs {
  RecordPtrs rp;
  Geo g;
  const double* tsince;
  int64_t t_count;
  int grid_per_sat;
  void* r;
  void* v;
  int32_t* status;
  unsigned long long* fixups;
};

cudaError_t launch_propagate64(const PropArgs& a, cudaStream_t stream);
cudaError_t launch_propagate32(const PropArgs& a, cudaStream_t stream);

// SM count and resident blocks per SM for a kernel, cached per device.
int device_sm_count();

}  // namespace sgp4
