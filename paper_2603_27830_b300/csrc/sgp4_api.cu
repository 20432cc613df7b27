// extern "C" entry points declared in include/sgp4.h: host-side validation, then
// the kernel launches.  No device allocation happens here.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <vector>

#include "sgp4.h"
#include "sgp4_device.cuh"
#include "sgp4_kernels.cuh"

namespace {

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

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

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Workspace layout of a batch: [tile counter, 256 B][tile_start int64 x (n+1)][requests].
size_t ws_tile_start_off() { return 256; }
size_t ws_reqs_off(int32_t n) { return 256 + round256(sizeof(int64_t) * ((size_t)n + 1)); }

bool mul_ok(int64_t a, int64_t b, int64_t limit) { return a == 0 || b <= limit / a; }

sgp4_result batch_args(const sgp4_batch_plan* plan, const sgp4_records* records,
                       const double* tsince, int64_t tsince_len, sgp4_precision precision,
                       void* r, void* v, int32_t* status, int64_t out_len,
                       unsigned long long* fixups, sgp4::BatchArgs* a) {
  if (!plan || !records_ok(records)) return SGP4_ERR_ARG;
  if (precision != SGP4_FP64 && precision != SGP4_FP32) return SGP4_ERR_ARG;
  if (plan->n_requests < 0 || plan->tile_states <= 0 || plan->tile_states % 128) return SGP4_ERR_ARG;
  if (plan->n_requests > 0 && !plan->workspace) return SGP4_ERR_ARG;
  if (records->n < plan->sats_needed || tsince_len < plan->tsince_needed ||
      out_len < plan->out_needed)
    return SGP4_ERR_ARG;
  if (plan->total_states > 0) {
    if (!tsince || !r || !v || !status) return SGP4_ERR_ARG;
    if (!aligned(tsince, 8) || !aligned(r, 16) || !aligned(v, 16) || !aligned(status, 16))
      return SGP4_ERR_ARG;
  }
  if (fixups && !aligned(fixups, 8)) return SGP4_ERR_ARG;
  char* ws = static_cast<char*>(plan->workspace);
  a->rp = sgp4::record_ptrs(records->arena, records->n);
  a->g = sgp4::make_geo(records->consts);
  a->gf = sgp4::geo_float(a->g);
  a->tsince = tsince;
  a->reqs = reinterpret_cast<const sgp4_request*>(ws + ws_reqs_off(plan->n_requests));
  a->tile_start = reinterpret_cast<const int64_t*>(ws + ws_tile_start_off());
  a->n_req = plan->n_requests;
  a->tile_states = plan->tile_states;
  a->counter = reinterpret_cast<unsigned long long*>(ws);
  a->r = r;
  a->v = v;
  a->status = status;
  a->fixups = fixups;
  return SGP4_OK;
}

struct BatchGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

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
                                    sgp4::make_geo(records->consts), init_status,
                                    static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SGP4_OK : SGP4_ERR_CUDA;
}

sgp4_result sgp4_propagate(const sgp4_records* records, const double* tsince, int64_t t_count,
                           int grid_per_sat, sgp4_precision precision, void* r, void* v,
                           int32_t* status, unsigned long long* fixups, void* stream) {
  if (!records_ok(records) || t_count < 0 || t_count > INT32_MAX) return SGP4_ERR_ARG;
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
  a.g = sgp4::make_geo(records->consts);
  a.gf = sgp4::geo_float(a.g);
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

sgp4_result sgp4_propagate_jd(const sgp4_records* records, const int32_t* jd_day,
                              const double* jd_frac, int64_t t_count, sgp4_precision precision,
                              void* r, void* v, int32_t* status, unsigned long long* fixups,
                              void* stream) {
  if (!records_ok(records) || t_count < 0 || t_count > INT32_MAX) return SGP4_ERR_ARG;
  if (precision != SGP4_FP64 && precision != SGP4_FP32) return SGP4_ERR_ARG;
  const int64_t n = records->n;
  if (n == 0 || t_count == 0) return SGP4_OK;
  if (n > INT64_MAX / 3 / t_count) return SGP4_ERR_ARG;
  if (!jd_day || !jd_frac || !r || !v || !status) return SGP4_ERR_ARG;
  if (!aligned(jd_day, 4) || !aligned(jd_frac, 8) || !aligned(r, 16) || !aligned(v, 16) ||
      !aligned(status, 16))
    return SGP4_ERR_ARG;
  if (fixups && !aligned(fixups, 8)) return SGP4_ERR_ARG;
  sgp4::PropArgs a;
  a.rp = sgp4::record_ptrs(records->arena, n);
  a.g = sgp4::make_geo(records->consts);
  a.gf = sgp4::geo_float(a.g);
  a.tsince = nullptr;
  a.jd_day = jd_day;
  a.jd_frac = jd_frac;
  a.t_count = t_count;
  a.grid_per_sat = 0;
  a.r = r;
  a.v = v;
  a.status = status;
  a.fixups = fixups;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = precision == SGP4_FP64 ? sgp4::launch_propagate64(a, s)
                                         : sgp4::launch_propagate32(a, s);
  return e == cudaSuccess ? SGP4_OK : SGP4_ERR_CUDA;
}

size_t sgp4_batch_workspace_bytes(int32_t n_requests) {
  if (n_requests < 0) return 0;
  return ws_reqs_off(n_requests) + round256(sizeof(sgp4_request) * (size_t)n_requests);
}

sgp4_result sgp4_batch_plan_init(const sgp4_request* requests, int32_t n_requests,
                                 int32_t tile_states, int32_t grid_blocks, void* workspace,
                                 size_t workspace_bytes, sgp4_batch_plan* plan, void* stream) {
  if (!plan || n_requests < 0 || grid_blocks < 0) return SGP4_ERR_ARG;
  if (tile_states <= 0 || tile_states % 128 != 0) return SGP4_ERR_ARG;
  if (n_requests > 0 && (!requests || !workspace || !aligned(workspace, 256))) return SGP4_ERR_ARG;
  if (n_requests > 0 && workspace_bytes < sgp4_batch_workspace_bytes(n_requests))
    return SGP4_ERR_OOM;
  // One host copy of the caller's table: the checks and the device copy read it, so
  // the device gets the table that was checked, and its pageable source is staged
  // before return even when the caller's table is page-locked.
  const std::vector<sgp4_request> table(requests, requests + n_requests);
  const int64_t kLimit = INT64_MAX / 4;
  std::vector<int64_t> tile_start((size_t)n_requests + 1, 0);
  std::vector<std::pair<int64_t, int64_t>> spans;
  spans.reserve((size_t)n_requests);
  int64_t sats = 0, ts = 0, outs = 0, total_states = 0;
  for (int32_t k = 0; k < n_requests; ++k) {
    const sgp4_request& q = table[(size_t)k];
    if (q.n < 0 || q.t_count < 0 || q.sat_offset < 0 || q.t_offset < 0 || q.out_offset < 0)
      return SGP4_ERR_ARG;
    if (q.t_count > INT32_MAX) return SGP4_ERR_ARG;
    if (q.sat_offset > kLimit - q.n || q.t_offset > kLimit - q.t_count) return SGP4_ERR_ARG;
    if (!mul_ok(q.n, q.t_count, kLimit / 3)) return SGP4_ERR_ARG;
    const int64_t st = q.n * q.t_count;
    if (q.out_offset > kLimit / 3 - st) return SGP4_ERR_ARG;
    sats = std::max(sats, q.sat_offset + q.n);
    ts = std::max(ts, q.t_offset + q.t_count);
    outs = std::max(outs, q.out_offset + st);
    total_states += st;
    if (total_states > kLimit) return SGP4_ERR_ARG;
    tile_start[(size_t)k + 1] = tile_start[(size_t)k] + sgp4::request_tiles(q.n, q.t_count, tile_states);
    if (st > 0) spans.emplace_back(q.out_offset, q.out_offset + st);
  }
  std::sort(spans.begin(), spans.end());
  for (size_t k = 1; k < spans.size(); ++k)
    if (spans[k].first < spans[k - 1].second) return SGP4_ERR_ARG;   // overlapping outputs
  plan->workspace = workspace;
  plan->n_requests = n_requests;
  plan->tile_states = tile_states;
  plan->grid_blocks = grid_blocks;
  plan->reserved = 0;
  plan->total_tiles = tile_start[(size_t)n_requests];
  plan->total_states = total_states;
  plan->sats_needed = sats;
  plan->tsince_needed = ts;
  plan->out_needed = outs;
  if (n_requests == 0) return SGP4_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  // Pageable sources: each copy returns once its source has been staged.
  cudaError_t e = cudaMemcpyAsync(ws + ws_tile_start_off(), tile_start.data(),
                                  sizeof(int64_t) * tile_start.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + ws_reqs_off(n_requests), table.data(),
                        sizeof(sgp4_request) * (size_t)n_requests, cudaMemcpyHostToDevice, s);
  return e == cudaSuccess ? SGP4_OK : SGP4_ERR_CUDA;
}

sgp4_result sgp4_propagate_batched(const sgp4_batch_plan* plan, const sgp4_records* records,
                                   const double* tsince, int64_t tsince_len,
                                   sgp4_precision precision, void* r, void* v, int32_t* status,
                                   int64_t out_len, unsigned long long* fixups, void* stream) {
  sgp4::BatchArgs a;
  const sgp4_result res = batch_args(plan, records, tsince, tsince_len, precision, r, v, status,
                                     out_len, fixups, &a);
  if (res != SGP4_OK) return res;
  if (plan->total_tiles == 0) return SGP4_OK;
  const bool fp32 = precision == SGP4_FP32;
  const int64_t grid = sgp4::batched_grid(fp32, plan->total_tiles, plan->grid_blocks);
  cudaError_t e = sgp4::launch_batched(a, fp32, plan->total_tiles, grid,
                                       static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SGP4_OK : SGP4_ERR_CUDA;
}

sgp4_result sgp4_batch_graph_create(const sgp4_batch_plan* plan, const sgp4_records* records,
                                    const double* tsince, int64_t tsince_len,
                                    sgp4_precision precision, void* r, void* v, int32_t* status,
                                    int64_t out_len, unsigned long long* fixups, void* stream,
                                    void** graph) {
  if (!graph || !stream) return SGP4_ERR_ARG;
  sgp4::BatchArgs a;
  const sgp4_result res = batch_args(plan, records, tsince, tsince_len, precision, r, v, status,
                                     out_len, fixups, &a);
  if (res != SGP4_OK) return res;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool fp32 = precision == SGP4_FP32;
  const int64_t grid = sgp4::batched_grid(fp32, plan->total_tiles, plan->grid_blocks);
  BatchGraph* bg = new BatchGraph();
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t le = sgp4::launch_batched(a, fp32, plan->total_tiles, grid, s);
    e = cudaStreamEndCapture(s, &bg->graph);
    if (e == cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&bg->exec, bg->graph, 0);
  if (e != cudaSuccess) {
    if (bg->graph) cudaGraphDestroy(bg->graph);
    delete bg;
    cudaGetLastError();
    return SGP4_ERR_CUDA;
  }
  *graph = bg;
  return SGP4_OK;
}

size_t sgp4_adjoint_workspace_bytes(int64_t n) { return sgp4::adjoint_workspace_bytes(n); }

sgp4_result sgp4_adjoint(const double* elements, const sgp4_records* records,
                         const double* tsince, int64_t t_count, int grid_per_sat,
                         sgp4_precision precision, const void* grad_r, const void* grad_v,
                         double* grad_elements, void* workspace, size_t workspace_bytes,
                         void* stream) {
  if (!records_ok(records) || t_count < 0) return SGP4_ERR_ARG;
  if (precision != SGP4_FP64 && precision != SGP4_FP32) return SGP4_ERR_ARG;
  const int64_t n = records->n;
  if (n == 0) return SGP4_OK;
  if (!elements || !grad_elements || !aligned(elements, 8) || !aligned(grad_elements, 8))
    return SGP4_ERR_ARG;
  if (t_count > 0 && (!tsince || !aligned(tsince, 8))) return SGP4_ERR_ARG;
  if (n > INT64_MAX / 3 / (t_count > 0 ? t_count : 1)) return SGP4_ERR_ARG;
  const size_t esz = precision == SGP4_FP32 ? 4 : 8;
  if ((grad_r && !aligned(grad_r, esz)) || (grad_v && !aligned(grad_v, esz)))
    return SGP4_ERR_ARG;
  if (!workspace || !aligned(workspace, 8)) return SGP4_ERR_ARG;
  if (workspace_bytes < sgp4::adjoint_workspace_bytes(n)) return SGP4_ERR_OOM;
  if (n > 0x7fffffffLL) return SGP4_ERR_ARG;   // one block per satellite
  cudaError_t e = sgp4::launch_adjoint(
      sgp4::record_ptrs(records->arena, n), sgp4::make_geo(records->consts), elements, tsince, t_count,
      grid_per_sat ? 1 : 0, precision == SGP4_FP32, t_count > 0 ? grad_r : nullptr,
      t_count > 0 ? grad_v : nullptr, grad_elements, static_cast<double*>(workspace),
      static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SGP4_OK : SGP4_ERR_CUDA;
}

size_t sgp4_fit_workspace_bytes(int64_t n) { return sgp4::fit_workspace_bytes(n); }

sgp4_result sgp4_fit_step(const double* elements, const sgp4_records* records,
                          const double* tsince, int64_t t_count, int grid_per_sat,
                          sgp4_precision precision, const double* r_obs, const double* lambda,
                          double* elements_out, double* sse, void* workspace,
                          size_t workspace_bytes, void* stream) {
  if (!records_ok(records) || t_count < 0) return SGP4_ERR_ARG;
  if (precision != SGP4_FP64 && precision != SGP4_FP32) return SGP4_ERR_ARG;
  const int64_t n = records->n;
  if (n == 0) return SGP4_OK;
  if (n > 0x7fffffffLL) return SGP4_ERR_ARG;
  if (n > INT64_MAX / 3 / (t_count > 0 ? t_count : 1)) return SGP4_ERR_ARG;
  const void* ptrs[] = {elements, lambda, elements_out, sse};
  for (const void* p : ptrs)
    if (!p || !aligned(p, 8)) return SGP4_ERR_ARG;
  if (elements_out == elements) return SGP4_ERR_ARG;
  if (t_count > 0 && (!tsince || !r_obs || !aligned(tsince, 8) || !aligned(r_obs, 8)))
    return SGP4_ERR_ARG;
  if (!workspace || !aligned(workspace, 8)) return SGP4_ERR_ARG;
  if (workspace_bytes < sgp4::fit_workspace_bytes(n)) return SGP4_ERR_OOM;
  cudaError_t e = sgp4::launch_fit_step(
      sgp4::record_ptrs(records->arena, n), sgp4::make_geo(records->consts), elements, tsince, t_count,
      grid_per_sat ? 1 : 0, precision == SGP4_FP32, r_obs, lambda, elements_out, sse,
      static_cast<double*>(workspace), static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SGP4_OK : SGP4_ERR_CUDA;
}

size_t sgp4_jacobian_workspace_bytes(int64_t n) { return sgp4::jacobian_workspace_bytes(n); }

sgp4_result sgp4_jacobian(const double* elements, const sgp4_records* records,
                          const double* tsince, int64_t t_count, int grid_per_sat,
                          sgp4_precision precision, void* r, void* v, int32_t* status, void* jac,
                          const double* cov, void* cov_out, void* workspace,
                          size_t workspace_bytes, void* stream) {
  if (!records_ok(records) || t_count < 0 || t_count > INT32_MAX) return SGP4_ERR_ARG;
  if (precision != SGP4_FP64 && precision != SGP4_FP32) return SGP4_ERR_ARG;
  const int64_t n = records->n;
  if (n == 0 || t_count == 0) return SGP4_OK;
  if (n > 0x7fffffffLL) return SGP4_ERR_ARG;   // one block per satellite
  if (n > INT64_MAX / 42 / t_count) return SGP4_ERR_ARG;
  if (!elements || !aligned(elements, 8) || !tsince || !aligned(tsince, 8)) return SGP4_ERR_ARG;
  if (!status || !aligned(status, 4)) return SGP4_ERR_ARG;
  const size_t esz = precision == SGP4_FP32 ? 4 : 8;
  const void* outs[] = {r, v, jac, cov_out};
  for (const void* p : outs)
    if (p && !aligned(p, esz)) return SGP4_ERR_ARG;
  if (cov_out && (!cov || !aligned(cov, 8))) return SGP4_ERR_ARG;
  if (!workspace || !aligned(workspace, 8)) return SGP4_ERR_ARG;
  if (workspace_bytes < sgp4::jacobian_workspace_bytes(n)) return SGP4_ERR_OOM;
  sgp4::JacOut out;
  out.r = r;
  out.v = v;
  out.status = status;
  out.jac = jac;
  out.cov = cov_out ? cov : nullptr;
  out.cov_out = cov_out;
  cudaError_t e = sgp4::launch_jacobian(
      sgp4::record_ptrs(records->arena, n), sgp4::make_geo(records->consts), elements, tsince, t_count,
      grid_per_sat ? 1 : 0, precision == SGP4_FP32, out, workspace,
      static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SGP4_OK : SGP4_ERR_CUDA;
}

sgp4_result sgp4_batch_graph_launch(void* graph, void* stream) {
  if (!graph) return SGP4_ERR_ARG;
  BatchGraph* bg = static_cast<BatchGraph*>(graph);
  cudaError_t e = cudaGraphLaunch(bg->exec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SGP4_OK : SGP4_ERR_CUDA;
}

sgp4_result sgp4_batch_graph_destroy(void* graph) {
  if (!graph) return SGP4_OK;
  BatchGraph* bg = static_cast<BatchGraph*>(graph);
  cudaError_t e1 = bg->exec ? cudaGraphExecDestroy(bg->exec) : cudaSuccess;
  cudaError_t e2 = bg->graph ? cudaGraphDestroy(bg->graph) : cudaSuccess;
  delete bg;
  return (e1 == cudaSuccess && e2 == cudaSuccess) ? SGP4_OK : SGP4_ERR_CUDA;
}

}  // extern "C"
