/*
 * sgp4.h -- C ABI of the B300 (sm_103a) SGP4 propagation library.
 *
 * The problem is the paper's f(s, t) -> (r, v), batched over satellites s and
 * times t (Priestley & Handley, "jaxsgp4", Sec. 2.2 "Vectorisation"): near-Earth
 * SGP4 (Spacetrack Report #3 equations as revised in 2006, WGS-72 constants,
 * Sec. 2.1), with invalid physical states flagged by integer codes instead of
 * aborting (Sec. 2.2 "Control Flow").  Records with a period of 225 min or more take
 * the same revision's deep-space branch (SDP4: the Sun's and Moon's perturbations and
 * tesseral resonance), which the paper names as future work (Sec. 6, 7); those
 * states are computed in FP64 in both precisions and depend on the record's epoch.
 *
 * Conventions for every entry point:
 *  - All array arguments are DEVICE pointers unless stated otherwise, owned by the
 *    caller, and must stay valid until the work queued on `stream` has finished.
 *    The library never allocates device memory in these calls.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    All calls are asynchronous with respect to the host.
 *  - Return value: SGP4_OK, or a negative sgp4_result.  Argument errors are
 *    detected on the host before any launch and leave all outputs untouched.
 *    SGP4_ERR_CUDA reports a failed launch (cudaGetLastError after the launch).
 *    Physical validity is never an API error: it is reported per record and per
 *    state in the int32 status arrays.
 *  - Units: mean motion in rad/min (Kozai, as in a TLE), angles in rad, B* in
 *    1/Earth radii, tsince in minutes from the record's epoch, r in km, v in km/s,
 *    TEME frame.
 *
 * Status codes (per record and per state):
 *   0  ok
 *   1  eccentricity out of range: input e0 outside [0,1) or a non-finite input
 *      element (fatal for the record), or mean e(t) >= 1 or < -0.001 after drag
 *   2  mean motion <= 0 (input n0 fatal for the record, or n0'' <= 0); deep space
 *      with resonance: also |tsince| > 1e7 min or a non-finite tsince (the resonance
 *      integration covers |tsince| <= 1e7 min)
 *   3  deep space: eccentricity outside [0, 1] after the lunar-solar periodic terms
 *   4  semi-latus rectum p_L < 0
 *   5  sgp4_jacobian only: a deep-space record, which it does not differentiate
 *   6  decayed: osculating radius below one Earth radius (r, v are still written)
 * Codes 1 to 5 write NaN to r and v.  The first failing check in this order wins:
 * 2, 1, 3, 4, 6.
 */
#ifndef SGP4_B300_SGP4_H
#define SGP4_B300_SGP4_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sgp4_result {
  SGP4_OK = 0,
  SGP4_ERR_ARG = -1,     /* bad size, NULL or misaligned pointer, bad enum        */
  SGP4_ERR_CUDA = -2,    /* a CUDA launch or runtime call failed                  */
  SGP4_ERR_OOM = -3,     /* a caller-provided buffer is too small                 */
  SGP4_ERR_TIMEOUT = -4  /* reserved for bounded device-side waits                */
} sgp4_result;

typedef enum sgp4_precision {
  SGP4_FP64 = 0,  /* every step in FP64; outputs double                            */
  SGP4_FP32 = 1   /* FP32 arithmetic with the n*t angle accumulation in double-float
                     and an FP64 recomputation of states near a status threshold;
                     outputs float                                                  */
} sgp4_precision;

enum {
  SGP4_STATUS_OK = 0,
  SGP4_STATUS_ECCENTRICITY = 1,
  SGP4_STATUS_MEAN_MOTION = 2,
  SGP4_STATUS_DEEP_ECCENTRICITY = 3,
  SGP4_STATUS_SEMI_LATUS = 4,
  SGP4_STATUS_NOT_DIFFERENTIATED = 5,
  SGP4_STATUS_DECAYED = 6
};

/* Earth model (paper Sec. 2.1: WGS-72).  ke is derived as 60/sqrt(R^3/mu). */
typedef struct sgp4_consts {
  double mu_km3s2;   /* gravitational parameter, km^3/s^2  */
  double radius_km;  /* equatorial radius, km              */
  double j2, j3, j4; /* zonal harmonics                    */
} sgp4_consts;

/* WGS-72: mu 398600.8, R 6378.135, J2 0.001082616, J3 -0.00000253881, J4 -0.00000165597. */
sgp4_consts sgp4_wgs72(void);

/*
 * Per-satellite records (the "initialisation" constants of Sec. 2.1 / Sec. 3.1:
 * un-Kozai'd mean motion, drag coefficients C1..C5, D2..D4, secular rates,
 * long-period coefficients).  Structure of arrays: one FP64 plane per field, one
 * FP32/double-float plane per field of the FP32 path, one int32 flag plane, each
 * padded to `stride` entries.  The struct is a plain value: `arena` is caller-owned
 * device memory of sgp4_records_bytes(n) bytes, 256-byte aligned.
 */
typedef struct sgp4_records {
  void* arena;        /* device memory written by sgp4_init                          */
  int64_t n;          /* number of satellites                                        */
  int64_t stride;     /* padded plane length (entries)                               */
  sgp4_consts consts; /* Earth model used by sgp4_init; propagation uses the same one */
} sgp4_records;

/* Bytes of arena needed for n satellites (0 if n < 0). */
size_t sgp4_records_bytes(int64_t n);

/*
 * Bind an arena to a record set.  Errors: SGP4_ERR_ARG if out is NULL, n < 0,
 * arena is NULL (n > 0) or not 256-byte aligned; SGP4_ERR_OOM if bytes is below
 * sgp4_records_bytes(n).  `consts` NULL selects WGS-72.
 */
sgp4_result sgp4_records_bind(void* arena, size_t bytes, int64_t n, const sgp4_consts* consts,
                              sgp4_records* out);

/*
 * sgp4_init: build the records from mean elements (paper Sec. 2.1, the
 * initialisation phase; Sec. 3.1 notes it is separate from propagation in the
 * C++ baseline).  One thread per satellite, FP64.
 *   elements     [n][7] double, row-major: n0 (rad/min, Kozai), e0, i0, RAAN0,
 *                argp0, M0 (rad), B* (1/Earth radii)
 *   epoch_day    [n] int32 and epoch_frac [n] double: epoch as Julian date split
 *                into an integer day and a fraction in [0, 1) (paper Sec. 6: a split
 *                epoch avoids the FP32 epoch rounding).  Both may be NULL (epoch 0).
 *                Stored in the records; sgp4_propagate_jd measures time from them;
 *                the deep-space terms of records with a period of 225 min or more
 *                (the Sun's and Moon's positions, the sidereal angle) depend on it.
 *   init_status  [n] int32 out: 1/2 for unusable input (fatal for the record),
 *                otherwise the status of the state at tsince = 0.
 * Errors: SGP4_ERR_ARG for NULL elements/records/init_status with n > 0, a record
 * set whose n differs from `n`, or elements not 8-byte aligned.
 */
sgp4_result sgp4_init(const double* elements, const int32_t* epoch_day, const double* epoch_frac,
                      int64_t n, const sgp4_records* records, int32_t* init_status,
                      void* stream);

/*
 * sgp4_propagate: r, v and status of every (satellite, time) state (paper
 * Sec. 2.2: f(s, t) -> (r, v) under vmap over satellites and times).
 *   tsince       [t_count] double (grid_per_sat == 0: one grid for all satellites)
 *                or [n][t_count] (grid_per_sat != 0), minutes since epoch
 *   precision    SGP4_FP64: r, v are double; SGP4_FP32: r, v are float
 *   r, v         [n][t_count][3], 16-byte aligned
 *   status       [n][t_count] int32, 16-byte aligned
 *   fixups       optional device counter (may be NULL): SGP4_FP32 adds the number
 *                of states recomputed in FP64 because a status threshold was
 *                within the FP32 guard band.  Ignored for SGP4_FP64.
 * Errors: SGP4_ERR_ARG for a bad precision, t_count < 0 or > INT32_MAX, NULL or
 * misaligned arrays when n * t_count > 0, or n * t_count * 3 overflowing int64.
 */
sgp4_result sgp4_propagate(const sgp4_records* records, const double* tsince, int64_t t_count,
                           int grid_per_sat, sgp4_precision precision, void* r, void* v,
                           int32_t* status, unsigned long long* fixups, void* stream);

/*
 * sgp4_propagate_jd: as sgp4_propagate, for absolute times shared by all satellites,
 * given as Julian dates split into day and fraction (paper Sec. 6 on epochs; the
 * theory propagates from each record's own epoch).  For record j and time i,
 *   tsince = 1440 ((jd_day[i] - epoch_day[j]) + (jd_frac[i] - epoch_frac[j])) minutes,
 * with the day difference taken in integers, evaluated on the device in FP64 (then
 * split into float hi + lo for the FP32 path).
 *   jd_day       [t_count] int32, 4-byte aligned; jd_frac [t_count] double, 8-byte aligned
 *   other arguments as in sgp4_propagate (outputs [n][t_count][3], [n][t_count])
 * |jd_day[i] - epoch_day[j]| must stay below 1,491,308 days (the int32 product by 1440).
 * Errors as sgp4_propagate.
 */
sgp4_result sgp4_propagate_jd(const sgp4_records* records, const int32_t* jd_day,
                              const double* jd_frac, int64_t t_count, sgp4_precision precision,
                              void* r, void* v, int32_t* status, unsigned long long* fixups,
                              void* stream);

/*
 * Batched propagation of many uneven problems in one persistent launch.  The paper
 * batches by composing vmaps over satellites and times (Sec. 2.2); a service
 * receives many such problems at once, each with its own satellites and grid.
 *
 * A request covers satellites [sat_offset, sat_offset + n) of one record set, the
 * grid tsince[t_offset, t_offset + t_count) (shared by its satellites), and writes
 * its n * t_count states, satellite-major, to the states
 * [out_offset, out_offset + n * t_count) of r, v ([states][3]) and status.
 * Output ranges of different requests must not overlap.
 */
typedef struct sgp4_request {
  int64_t sat_offset;
  int64_t n;
  int64_t t_offset;
  int64_t t_count;
  int64_t out_offset;
} sgp4_request;

/*
 * A prepared batch: host-side value whose tables live in the caller's workspace.
 * Fields are filled by sgp4_batch_plan_init; the *_needed fields are the minimum
 * sizes of records, tsince and outputs that sgp4_propagate_batched checks.
 */
typedef struct sgp4_batch_plan {
  void* workspace;        /* device, caller-owned, sgp4_batch_workspace_bytes(n) */
  int32_t n_requests;
  int32_t tile_states;    /* states per work tile, a multiple of 128 (the FP32
                             kernel walks a tile in units of four states of one
                             satellite, the FP64 kernel in units of two; each request
                             gets the larger of the two tile counts) */
  int32_t grid_blocks;    /* persistent grid size; 0 = one full wave on the device */
  int32_t reserved;
  int64_t total_tiles;
  int64_t total_states;
  int64_t sats_needed;    /* max over requests of sat_offset + n */
  int64_t tsince_needed;  /* max of t_offset + t_count */
  int64_t out_needed;     /* max of out_offset + n * t_count (states) */
} sgp4_batch_plan;

/* Device workspace bytes for a batch of n_requests (0 if n_requests < 0). */
size_t sgp4_batch_workspace_bytes(int32_t n_requests);

/*
 * Validate a HOST request table, derive the tiling and copy the tables to the
 * workspace (stream-ordered).  The call first takes its own pageable host copy of
 * `requests`, validates that copy and uploads it, so `requests` (pageable or
 * page-locked) may be reused as soon as the call returns.
 *   tile_states  states per tile, a positive multiple of 128 (chosen by the
 *                autotuner of the Python layer, e.g. 1024)
 *   grid_blocks  persistent grid size, 0 for one full wave
 * Errors: SGP4_ERR_ARG for a NULL plan/workspace/requests (n_requests > 0), a
 * negative size or offset, a t_count above INT32_MAX, a bad tile_states, overlapping
 * output ranges, or overflow; SGP4_ERR_OOM if workspace_bytes is too small; SGP4_ERR_CUDA if the copy
 * fails.
 */
sgp4_result sgp4_batch_plan_init(const sgp4_request* requests, int32_t n_requests,
                                 int32_t tile_states, int32_t grid_blocks, void* workspace,
                                 size_t workspace_bytes, sgp4_batch_plan* plan, void* stream);

/*
 * Propagate every request of the plan in one persistent kernel launch (preceded by
 * an 8-byte reset of the tile counter in the workspace).  Arguments as in
 * sgp4_propagate; tsince_len and out_len (states) are the sizes of tsince and of
 * r/v/status, checked against the plan.  Plans sharing a workspace must not run
 * concurrently.  Errors: SGP4_ERR_ARG as in sgp4_propagate, or a record set, grid
 * or output smaller than the plan needs.
 */
sgp4_result sgp4_propagate_batched(const sgp4_batch_plan* plan, const sgp4_records* records,
                                   const double* tsince, int64_t tsince_len,
                                   sgp4_precision precision, void* r, void* v, int32_t* status,
                                   int64_t out_len, unsigned long long* fixups, void* stream);

/*
 * Capture sgp4_propagate_batched with these arguments into a CUDA graph and
 * instantiate it; *graph receives an opaque handle.  `stream` must be a non-NULL
 * stream; it is used only for the capture.  Replaying the graph re-runs the batch
 * on the buffers given here.  Errors: those of sgp4_propagate_batched, SGP4_ERR_ARG
 * for a NULL stream or graph, SGP4_ERR_CUDA if capture or instantiation fails.
 */
sgp4_result sgp4_batch_graph_create(const sgp4_batch_plan* plan, const sgp4_records* records,
                                    const double* tsince, int64_t tsince_len,
                                    sgp4_precision precision, void* r, void* v, int32_t* status,
                                    int64_t out_len, unsigned long long* fixups, void* stream,
                                    void** graph);

/* Launch a graph made by sgp4_batch_graph_create on `stream`. */
sgp4_result sgp4_batch_graph_launch(void* graph, void* stream);

/* Destroy a graph made by sgp4_batch_graph_create (NULL is a no-op). */
sgp4_result sgp4_batch_graph_destroy(void* graph);

/*
 * Adjoint of the propagation (paper Sec. 5, "Differentiable Orbital Mechanics":
 * gradients of the state vectors with respect to the mean elements through the
 * initialisation and the propagation).  For upstream gradients g_r, g_v of every
 * state it returns, per satellite j and element k of (n0, e0, i0, RAAN0, argp0, M0,
 * B*):  grad[j][k] = sum_t dr_jt/del_jk . g_r[j][t] + dv_jt/del_jk . g_v[j][t].
 *   elements   [n][7] double, the elements the records were built from
 *   records    the record set built by sgp4_init from those elements
 *   tsince     as in sgp4_propagate ([t_count] or [n][t_count] with grid_per_sat)
 *   precision  SGP4_FP64: grad_r / grad_v are double and the sweep runs in FP64;
 *              SGP4_FP32: they are float and the sweep runs in FP32 (the n*t phase
 *              in double-float, states near a status threshold in FP64, as in
 *              sgp4_propagate); per-thread and per-warp sums in FP32, the sum over
 *              warps in FP64
 *   grad_r     [n][t_count][3] (may be NULL: zero); grad_v likewise
 *   grad_elements  [n][7] double out
 *   workspace  device, sgp4_adjoint_workspace_bytes(n) bytes, 8-byte aligned
 * States with status 1, 2 or 4 contribute nothing; records with unusable elements
 * and deep-space records (period 225 min or more, not differentiated) get a zero
 * gradient.  Errors: SGP4_ERR_ARG for NULL / misaligned arrays, a record
 * set of another size, bad precision or t_count < 0; SGP4_ERR_OOM for a small
 * workspace; SGP4_ERR_CUDA for a failed launch.
 */
size_t sgp4_adjoint_workspace_bytes(int64_t n);
sgp4_result sgp4_adjoint(const double* elements, const sgp4_records* records,
                         const double* tsince, int64_t t_count, int grid_per_sat,
                         sgp4_precision precision, const void* grad_r, const void* grad_v,
                         double* grad_elements, void* workspace, size_t workspace_bytes,
                         void* stream);

/*
 * One batch-least-squares step per satellite, fitting the mean elements to observed
 * positions with the gradients of sgp4_adjoint (paper Sec. 5 names gradient-based
 * orbit determination as the use of a differentiable SGP4).  For the states with
 * finite output, res_t = r_t(elements) - r_obs_t, J_t = dr_t/d(elements) (three
 * reverse sweeps per state), A = sum J^T J, b = sum J^T res; the step solves
 * (A' + lambda diag A') x = -b' on the Jacobi-scaled system (Cholesky) and returns
 * elements_out = elements + step (Levenberg-Marquardt with damping lambda[j]).
 *   elements      [n][7] double, the elements the records were built from
 *   r_obs         [n][t_count][3] double, observed TEME positions, km
 *   lambda        [n] double, damping (>= 0)
 *   elements_out  [n][7] double (may not alias elements)
 *   sse           [n] double out: sum of squared residuals at `elements`, km^2
 *   workspace     device, sgp4_fit_workspace_bytes(n) bytes, 8-byte aligned (holds
 *                 the Jacobian of sgp4init and the normal equations per satellite
 *                 during the call)
 * SGP4_FP32 runs the sweeps in FP32 as sgp4_adjoint does and forms A and b per thread
 * in FP32 (sums over warps in FP64); the Cholesky solve is FP64 in both precisions.
 * Unusable records and deep-space records (not fitted) keep their elements and get
 * sse 0.  Errors as sgp4_adjoint.
 */
size_t sgp4_fit_workspace_bytes(int64_t n);
sgp4_result sgp4_fit_step(const double* elements, const sgp4_records* records,
                          const double* tsince, int64_t t_count, int grid_per_sat,
                          sgp4_precision precision, const double* r_obs, const double* lambda,
                          double* elements_out, double* sse, void* workspace,
                          size_t workspace_bytes, void* stream);

/*
 * Per-state Jacobians of the TEME state with respect to the mean elements, through
 * sgp4init and the propagation (paper Sec. 5: derivatives of the propagator), and the
 * propagation of an element covariance to the state (P = J C J^T), the form used to
 * screen conjunctions.  For each state J = d(r_x, r_y, r_z, v_x, v_y, v_z) /
 * d(n0, e0, i0, RAAN0, argp0, M0, B*) (km and km/s per element unit), from one
 * forward pass and six reverse sweeps.
 *   elements, records, tsince, t_count, grid_per_sat, precision  as in sgp4_adjoint
 *   r, v        [n][t_count][3] out (may be NULL), float for SGP4_FP32, else double
 *   status      [n][t_count] int32 out (required), as sgp4_propagate
 *   jac         [n][t_count][6][7] out (may be NULL), precision's type
 *   cov         [n][7][7] double element covariance (read only if cov_out is given)
 *   cov_out     [n][t_count][21] out (may be NULL): upper triangle of P, row by row
 *               ((0,0), (0,1) .. (0,5), (1,1) .. (5,5)), precision's type
 *   workspace   device, sgp4_jacobian_workspace_bytes(n) bytes, 8-byte aligned
 * States with status 1, 2 or 4 get NaN in r, v, jac and cov_out; deep-space records
 * (period 225 min or more) are not differentiated: status 5 and NaN.  Errors:
 * SGP4_ERR_ARG for NULL elements / tsince / status, cov_out without cov, misaligned
 * arrays, a bad precision or sizes; SGP4_ERR_OOM for a small workspace; SGP4_ERR_CUDA
 * for a failed launch.
 */
size_t sgp4_jacobian_workspace_bytes(int64_t n);
sgp4_result sgp4_jacobian(const double* elements, const sgp4_records* records,
                          const double* tsince, int64_t t_count, int grid_per_sat,
                          sgp4_precision precision, void* r, void* v, int32_t* status, void* jac,
                          const double* cov, void* cov_out, void* workspace,
                          size_t workspace_bytes, void* stream);

/*
 * Batched propagation without any device allocation by the caller.  The paper has
 * no counterpart; this serves callers that cannot allocate device memory (a host
 * application that owns the allocator and hands out only fixed buffers, real-time
 * or flight software whose device memory is budgeted once at start-up, a plug-in
 * that must not grow its footprint after initialisation).  It runs the batched
 * kernel of sgp4_propagate_batched, with the tile counter, the tile prefix sums and
 * the request table in a fixed array inside the library: about 48 KB held on every
 * GPU that loads the library, until the process exits.
 *   requests     HOST table of n_requests <= SGP4_STATIC_MAX_REQUESTS requests
 *                (same meaning as for sgp4_batch_plan_init).  The call copies it
 *                into a per-thread host array, validates that copy and uploads it,
 *                so the table (pageable or page-locked) may be reused on return.
 *   tile_states  states per work tile, a positive multiple of 128
 *   other arguments as in sgp4_propagate_batched (no fixup counter)
 * The first call on a device looks up the array's device address with that device
 * current.  The call cannot be captured into a CUDA graph (its table copy reads a
 * host array that later calls rewrite): under an active stream capture it returns
 * SGP4_ERR_ARG and enqueues nothing; graphs use sgp4_batch_graph_*.  All calls on a device
 * share the array: two calls whose work overlaps on the GPU (different streams, or
 * different host threads) race and must be serialised by the caller.  Each call
 * rewrites the table and prefix sums and resets the counter before its launch.
 * Errors: SGP4_ERR_OOM if n_requests exceeds SGP4_STATIC_MAX_REQUESTS; SGP4_ERR_ARG
 * for bad or negative sizes (tsince_len, out_len included), offsets outside records /
 * tsince / outputs, overlapping outputs, a bad precision or tile size, NULL or
 * misaligned arrays, a stream under capture; SGP4_ERR_CUDA if the address lookup, the
 * capture query, the copy or a launch fails.
 * Calls no allocation routine.
 */
#define SGP4_STATIC_MAX_REQUESTS 1024
sgp4_result sgp4_propagate_batched_static(const sgp4_request* requests, int32_t n_requests,
                                          int32_t tile_states, const sgp4_records* records,
                                          const double* tsince, int64_t tsince_len,
                                          sgp4_precision precision, void* r, void* v,
                                          int32_t* status, int64_t out_len, void* stream);

/*
 * Two-line element sets (host functions; no device work).  The NORAD fixed-column
 * format: line 1 carries the catalogue number (five digits or "Alpha-5"), the epoch
 * (two-digit year, 57-99 -> 19xx, 00-56 -> 20xx, and day of year with fraction) and
 * B*; line 2 inclination, RAAN, eccentricity (implied leading point), argument of
 * perigee, mean anomaly (degrees) and mean motion (rev/day); each line ends with a
 * modulo-10 checksum of its first 68 columns ('-' counts 1).
 *
 * sgp4_tle_parse: one set into the units of sgp4_init.
 *   line1, line2   NUL-terminated lines of at least 69 columns (trailing CR/LF/blanks ok)
 *   elements       [7] out: n0 rad/min, e0, i0, RAAN0, argp0, M0 (rad), B* (1/Earth radii)
 *   epoch_day, epoch_frac  out: epoch as Julian date, integer day + fraction in [0, 1)
 *   satnum         out (may be NULL): catalogue number
 * Errors: SGP4_ERR_ARG for NULL pointers, short lines, wrong line numbers, a checksum
 * mismatch, different catalogue numbers on the two lines, or a malformed field.
 */
sgp4_result sgp4_tle_parse(const char* line1, const char* line2, double* elements,
                           int32_t* epoch_day, double* epoch_frac, int32_t* satnum);

/*
 * sgp4_tle_parse_text: every set in a text of two- or three-line sets (name lines and
 * blank lines are skipped), in order.  Stores at most `capacity` sets into elements
 * [capacity][7], epoch_day, epoch_frac and satnum (may be NULL); returns the number of
 * valid sets found (which may exceed capacity: call again with more room), or -1 for
 * bad arguments.  n_rejected (may be NULL) receives the number of sets or orphan
 * line-1s rejected.
 */
int64_t sgp4_tle_parse_text(const char* text, size_t len, int64_t capacity, double* elements,
                            int32_t* epoch_day, double* epoch_frac, int32_t* satnum,
                            int64_t* n_rejected);

/*
 * sgp4_tle_format: the set for elements (units of sgp4_init) and a split Julian epoch,
 * with first and second derivatives of the mean motion zero, at the format's
 * resolution (1e-4 deg, 1e-7 in e, 1e-8 rev/day, 1e-8 day in the epoch, 5 digits of B*).
 *   line1, line2   out: 70-byte buffers (69 columns + NUL)
 * Errors: SGP4_ERR_ARG for NULL pointers, satnum outside 0..99999, epoch_frac outside
 * [0, 1), an epoch outside 1957-2056, mean motion outside (0, 100) rev/day, e outside
 * [0, 1), inclination outside [0, 180] deg, or |B*| beyond the exponent digit.
 */
sgp4_result sgp4_tle_format(const double* elements, int32_t epoch_day, double epoch_frac,
                            int32_t satnum, char* line1, char* line2);

/*
 * CCSDS Orbit Mean-Elements Messages (OMM, CCSDS 502.0-B; host functions, no device
 * work) carrying SGP4 mean elements, in KVN ("KEYWORD = value [units]" lines) or XML.
 * Keywords read: EPOCH (UTC, ISO 8601 "YYYY-MM-DDThh:mm:ss[.f]" or
 * "YYYY-DDDThh:mm:ss[.f]", years 1583-9999), MEAN_MOTION (rev/day), ECCENTRICITY,
 * INCLINATION, RA_OF_ASC_NODE, ARG_OF_PERICENTER, MEAN_ANOMALY (deg), BSTAR (1/Earth
 * radii), NORAD_CAT_ID (optional); MEAN_ELEMENT_THEORY, REF_FRAME and TIME_SYSTEM, if
 * present, must be SGP4 (or SGP/SGP4), TEME and UTC.  Other keywords are skipped.
 *
 * sgp4_omm_parse_text: every message of a text, in order.  A text whose first
 * non-blank character is '<' is XML (one message per <omm> element), otherwise KVN
 * (a message starts at each CCSDS_OMM_VERS line).  Stores at most `capacity` messages
 * into elements [capacity][7] (units of sgp4_init), epoch_day, epoch_frac (Julian date
 * split as in sgp4_tle_parse) and satnum (may be NULL; -1 where NORAD_CAT_ID is
 * absent); returns the number of valid messages (which may exceed capacity: call again
 * with more room), or -1 for bad arguments.  n_rejected (may be NULL) receives the
 * number of messages rejected (a required keyword missing or malformed, another
 * theory, frame or time system).
 */
int64_t sgp4_omm_parse_text(const char* text, size_t len, int64_t capacity, double* elements,
                            int32_t* epoch_day, double* epoch_frac, int32_t* satnum,
                            int64_t* n_rejected);

/*
 * sgp4_omm_format: one KVN message (OMM 2.0 keywords) for elements (units of sgp4_init)
 * and a split Julian epoch, written NUL-terminated into buf[cap]: values with 17
 * significant digits, the epoch to the microsecond, zero mean-motion derivatives.
 *   satnum  catalogue number, or -1 to omit NORAD_CAT_ID
 *   name    OBJECT_NAME (may be NULL)
 * Errors: SGP4_ERR_ARG for NULL elements or buf, non-finite elements, epoch_frac
 * outside [0, 1), an epoch outside 1583-9999, a name with a line break, or a buffer
 * too small (about 700 bytes suffice).
 */
sgp4_result sgp4_omm_format(const double* elements, int32_t epoch_day, double epoch_frac,
                            int32_t satnum, const char* name, char* buf, size_t cap);

/* Library version (major*10000 + minor*100 + patch). */
int sgp4_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SGP4_B300_SGP4_H */
