// Batched propagation for callers that cannot allocate device memory.
//
// sgp4_propagate_batched needs a workspace from the caller for its tile counter, its
// tile prefix sums and its request table.  Some callers have no way to provide one:
// code that runs inside a host application which owns the device allocator and
// hands out only fixed buffers, flight or real-time software whose device memory is
// budgeted once at start-up, or a plug-in that must not grow a process's memory
// footprint after initialisation.  This entry point keeps that scratch in a
// fixed-size array inside the library instead (every GPU that loads the library
// holds it until the process exits) and otherwise runs the same batched kernel.
// The paper has no counterpart: it is a service feature of this library.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "sgp4.h"
#include "sgp4_device.cuh"
#include "sgp4_kernels.cuh"

namespace {

constexpr int32_t kMaxRequests = SGP4_STATIC_MAX_REQUESTS;
constexpr size_t kCounterBytes = 256;
constexpr size_t kTileStartBytes = ((sizeof(int64_t) * (kMaxRequests + 1) + 255) / 256) * 256;
constexpr size_t kRequestBytes = ((sizeof(sgp4_request) * kMaxRequests + 255) / 256) * 256;
constexpr size_t kScratchBytes = kCounterBytes + kTileStartBytes + kRequestBytes;

// Layout: [tile counter][tile_start, n + 1 entries][request table].  Shared by every
// call on a device; the prepare kernel rewrites tile_start and the launch resets the
// counter, so nothing of an earlier call is read.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// One block: tile count of every request, exclusive prefix sum into tile_start.
__global__ void __launch_bounds__(1024) prepare_static_kernel(int32_t n, int64_t tile_states) {
  __shared__ int64_t part[1024];
  const sgp4_request* reqs =
      reinterpret_cast<const sgp4_request*>(g_scratch + kCounterBytes + kTileStartBytes);
  int64_t* tile_start = reinterpret_cast<int64_t*>(g_scratch + kCounterBytes);
  const int k = threadIdx.x;
  int64_t tiles = 0;
  if (k < n) tiles = sgp4::request_tiles(reqs[k].n, reqs[k].t_count, tile_states);
  part[k] = tiles;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {   // inclusive scan (Hillis-Steele)
    const int64_t add = k >= off ? part[k - off] : 0;
    __syncthreads();
    part[k] += add;
    __syncthreads();
  }
  if (k < n) tile_start[k + 1] = part[k];
  if (k == 0) tile_start[0] = 0;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" sgp4_result sgp4_propagate_batched_static(
    const sgp4_request* requests, int32_t n_requests, int32_t tile_states,
    const sgp4_records* records, const double* tsince, int64_t tsince_len,
    sgp4_precision precision, void* r, void* v, int32_t* status, int64_t out_len, void* stream) {
  if (n_requests > kMaxRequests) return SGP4_ERR_OOM;   // beyond the static scratch
  if (n_requests < 0 || !records || records->n < 0) return SGP4_ERR_ARG;
  if (precision != SGP4_FP64 && precision != SGP4_FP32) return SGP4_ERR_ARG;
  if (tile_states <= 0 || tile_states % 128 != 0) return SGP4_ERR_ARG;
  if (records->n > 0 && (!records->arena || !aligned(records->arena, 256))) return SGP4_ERR_ARG;
  if (records->stride != sgp4::record_stride(records->n)) return SGP4_ERR_ARG;
  if (!(records->consts.mu_km3s2 > 0.0) || !(records->consts.radius_km > 0.0)) return SGP4_ERR_ARG;
  if (n_requests > 0 && !requests) return SGP4_ERR_ARG;
  if (tsince_len < 0 || out_len < 0) return SGP4_ERR_ARG;

  // The caller's table is copied once into this thread's own host array: the checks
  // below and the copy to the device both read that copy, so the device gets exactly
  // the table that was checked, and the copy's pageable source is staged before this
  // call returns even when the caller's table is page-locked.
  thread_local sgp4_request table[kMaxRequests];
  std::memcpy(table, requests, sizeof(sgp4_request) * (size_t)n_requests);

  // Host checks of the table without any buffer: bounds, overflow, and pairwise
  // non-overlap of the output ranges (at most 1024 requests).
  const int64_t kLimit = INT64_MAX / 4;
  int64_t total_tiles = 0;
  for (int32_t k = 0; k < n_requests; ++k) {
    const sgp4_request& q = table[k];
    if (q.n < 0 || q.t_count < 0 || q.sat_offset < 0 || q.t_offset < 0 || q.out_offset < 0)
      return SGP4_ERR_ARG;
    if (q.t_count > INT32_MAX) return SGP4_ERR_ARG;
    if (q.n > 0 && q.t_count > kLimit / 3 / q.n) return SGP4_ERR_ARG;
    const int64_t st = q.n * q.t_count;
    if (q.sat_offset > records->n - q.n || q.t_offset > tsince_len - q.t_count ||
        q.out_offset > out_len - st)
      return SGP4_ERR_ARG;
    total_tiles += sgp4::request_tiles(q.n, q.t_count, tile_states);
    if (st == 0) continue;
    for (int32_t m = 0; m < k; ++m) {
      const sgp4_request& p = table[m];
      const int64_t sp = p.n * p.t_count;
      if (sp > 0 && q.out_offset < p.out_offset + sp && p.out_offset < q.out_offset + st)
        return SGP4_ERR_ARG;
    }
  }
  if (total_tiles == 0) return SGP4_OK;
  if (!tsince || !r || !v || !status) return SGP4_ERR_ARG;
  if (!aligned(tsince, 8) || !aligned(r, 16) || !aligned(v, 16) || !aligned(status, 16))
    return SGP4_ERR_ARG;

  // A capture would record the copy from this thread's host table, which a graph
  // replay would read long after the call returned (and later calls rewrote it); it is
  // refused before any other CUDA call, so that nothing breaks the caller's capture.
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return SGP4_ERR_CUDA;
  }
  if (cap != cudaStreamCaptureStatusNone) return SGP4_ERR_ARG;

  // Device address of the scratch array, looked up once per device with that device
  // current (in host code the array's name is not a device address).
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SGP4_ERR_CUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return SGP4_ERR_CUDA;
      }
      g_addr[dev] = p;
    }
    base = g_addr[dev];
  }
  char* scratch = static_cast<char*>(base);

  // Request table into the scratch (the pageable copy is staged before return), then
  // the tile prefix sums on the device.
  cudaError_t e = cudaMemcpyAsync(scratch + kCounterBytes + kTileStartBytes, table,
                                  sizeof(sgp4_request) * (size_t)n_requests,
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return SGP4_ERR_CUDA;
  prepare_static_kernel<<<1, 1024, 0, s>>>(n_requests, tile_states);
  if (cudaGetLastError() != cudaSuccess) return SGP4_ERR_CUDA;

  sgp4::BatchArgs a;
  a.rp = sgp4::record_ptrs(records->arena, records->n);
  a.g = sgp4::make_geo(records->consts);
  a.gf = sgp4::geo_float(a.g);
  a.tsince = tsince;
  a.reqs = reinterpret_cast<const sgp4_request*>(scratch + kCounterBytes + kTileStartBytes);
  a.tile_start = reinterpret_cast<const int64_t*>(scratch + kCounterBytes);
  a.n_req = n_requests;
  a.tile_states = tile_states;
  a.counter = reinterpret_cast<unsigned long long*>(scratch);   // reset by launch_batched
  a.r = r;
  a.v = v;
  a.status = status;
  a.fixups = nullptr;
  const bool fp32 = precision == SGP4_FP32;
  const int64_t grid = sgp4::batched_grid(fp32, total_tiles, 0);
  e = sgp4::launch_batched(a, fp32, total_tiles, grid, s);
  return e == cudaSuccess ? SGP4_OK : SGP4_ERR_CUDA;
}
