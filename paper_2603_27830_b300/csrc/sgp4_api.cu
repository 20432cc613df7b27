// extern "C" entry points declared in include/sgp4.h: host-side validation, then
// the kernel launches.  No device allocation happens here.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "sgp4.h"
#include "sgp4_device.cuh"
#include "sgp4_kernels.cuh"

namespace {

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

sgp4::Geo make_geo(const sgp4_consts& c) {
  sgp4::Geo g;
  g.xke = 60.0 / std::sqrt(c.radius_km * c.radius_km * c.radius_km / c.mu_km3s2);
  g.j2 = c.j2;
  g.j3oj2 = (c.j2 != 0.0) ? c.j3 / c.j2 : 0.0;
  g.j4 = c.j4;
  g.re = c.radius_km;
  g.vkmps = c.radius_km * g.xke / 60.0;
  return g;
}

bool consts_ok(const sgp4_consts& c) {
  return std::isfinite(c.mu_km3s2) && c.mu_km3s2 > 0 && std::isfinite(c.radius_km) &&
         c.radius_km > 0 && std::isfinite(c.j2) && std::isfinite(c.j3) && std::isfinite(c.j4);
}

bool records_ok(const sgp4_records* rec) {
  if (!rec || rec->n < 0) return false;
  if (rec->n > 0 && (!rec->arena || !aligned(rec->arena, 256))) return false;
  if (rec->stride != sgp4::record_stride(rec->n)) return false;
  return consts_ok(rec->consts);
}

}  // namespace

extern "C" {

int sgp4_version(void) { return 100; }

sgp4_consts sgp4_wgs72(void) {
  sgp4_consts c;
  c.mu_km3s2 = 398600.8;
  c.radius_km = 6378.135;
  c.j2 = 0.001082616;
  c.j3 = -0.00000253881;
  c.j4 = -0.00000165597;
  return c;
}

size_t sgp4_records_bytes(int64_t n) {
  if (n < 0) return 0;
  return sgp4::record_bytes(n);
}

sgp4_result sgp4_records_bind(void* arena, size_t bytes, int64_t n, const sgp4_consts* consts,
                              sgp4_records* out) {
  if (!out || n < 0) return SGP4_ERR_ARG;
  if (n > 0 && (!arena || !aligned(arena, 256))) return SGP4_ERR_ARG;
  if (n > ((int64_t)1 << 40)) return SGP4_ERR_ARG;
  const sgp4_consts c = consts ? *consts : sgp4_wgs72();
  if (!consts_ok(c)) return SGP4_ERR_ARG;
  if (bytes < sgp4::record_bytes(n)) return SGP4_ERR_OOM;
  out->arena = arena;
  out->n = n;
  out->stride = sgp4::record_stride(n);
  out->consts = c;
  return SGP4_OK;
}

sgp4_result sgp4_init(const double* elements, const int32_t* epoch_day, const double* epoch_frac,
                      int64_t n, const sgp4_records* records, int32_t* init_status,
                      void* stream) {
  if (!records_ok(records) || records->n != n) return SGP4_ERR_ARG;
  if (n == 0) return SGP4_OK;
  if (!elements || !init_status || !aligned(elements, 8)) return SGP4_ERR_ARG;
  const sgp4::RecordPtrs rp = sgp4::record_ptrs(records->arena, n);
  cudaError_t e = sgp4::launch_init(elements, epoch_day, epoch_frac, rp,
                                    make_geo(records->consts), init_status,
                                    static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SGP4_OK : SGP4_ERR_CUDA;
}

sgp4_result sgp4_propagate(const sgp4_records* records, const double* tsince, int64_t t_count,
                           int grid_per_sat, sgp4_precision precision, void* r, void* v,
                           int32_t* status, unsigned long long* fixups, void* stream) {
  if (!records_ok(records) || t_count < 0) return SGP4_ERR_ARG;
  if (precision != SGP4_FP64 && precision != SGP4_FP32) return SGP4_ERR_ARG;
  const int64_t n = records->n;
  if (n == 0 || t_count == 0) return SGP4_OK;
  if (n > INT64_MAX / 3 / t_count) return SGP4_ERR_ARG;
  if (!tsince || !r || !v || !status) return SGP4_ERR_ARG;
  if (!aligned(tsince, 8) || !aligned(r, 16) || !aligned(v, 16) || !aligned(status, 16))
    return SGP4_ERR_ARG;
  if (fixups && !aligned(fixups, 8)) return SGP4_ERR_ARG;
  sgp4::PropArgs a;
  a.rp = sgp4::record_ptrs(records->arena, n);
  a.g = make_geo(records->consts);
  a.tsince = tsince;
  a.t_count = t_count;
  a.grid_per_sat = grid_per_sat ? 1 : 0;
  a.r = r;
  a.v = v;
  a.status = status;
  a.fixups = fixups;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = precision == SGP4_FP64 ? sgp4::launch_propagate64(a, s)
                                         : sgp4::launch_propagate32(a, s);
  return e == cudaSuccess ? SGP4_OK : SGP4_ERR_CUDA;
}

}  // extern "C"
