/*
 * rsos.h -- C ABI of the GB300 RSOS multisurface sweep library (librsos.so).
 *
 * Kelling, Odor & Gemming, "Universality of (2+1)-dimensional restricted
 * solid-on-solid models" (arXiv:1605.02620):
 *   - model: deposition h -> h+1 at a site, accepted only if every
 *     nearest-neighbour height difference stays within N (Eq. 6), on a
 *     periodic L x L lattice from a flat start (section II);
 *   - many surfaces ("lanes") of one job share the sequence of selected sites
 *     and each lane acts on a selection only through its own random half mask
 *     (multisurface coding, section II);
 *   - double tiling: Tx x Ty tiles, each split into 2 x 2 sub-tiles, four sets
 *     updated in turn, tiling origin moved randomly after every sweep
 *     (section II); optionally the Tx(+1) x Ty(+1) tilings of the
 *     decomposition check (section III.C);
 *   - time in sweeps; one sweep is L^2 expected attempts per surface (1 MCS);
 *   - observable: squared interface width W^2 = <h^2> - <h>^2 (Eq. 2), at
 *     measurement times such as those of Eq. 10.
 * The random stream (Philox-4x32-10 keyed by the seed, counters built from
 * sweep, phase, tile, selection and lane word) is specified in the library's
 * design notes; results are a pure function of (params, t).
 *
 * Conventions for every call:
 *   - return value: RSOS_OK (0) or a negative RSOS_E* code; no C++ exception
 *     ever crosses this boundary;
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream);
 *   - device memory is owned by the library unless the caller passes its own
 *     buffer to rsos_init; host arrays are owned by the caller;
 *   - a handle is not thread-safe; distinct handles are independent;
 *   - after a CUDA error the handle is poisoned: every later call returns
 *     RSOS_ECUDA and rsos_last_cuda_error() gives the CUDA code.
 */
#ifndef RSOS_H
#define RSOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RSOS_OK 0
#define RSOS_EINVAL (-1)    /* invalid argument (sizes, ranges, NULL pointers)      */
#define RSOS_ENOMEM (-2)    /* device allocation failed or caller buffer too small  */
#define RSOS_ECUDA (-3)     /* a CUDA call failed (sticky for the handle)           */
#define RSOS_EOVERFLOW (-4) /* a sum does not fit int64 (W^2 is still valid)        */
#define RSOS_ETIMEOUT (-5)  /* a device-side wait gave up; the GPU stays usable     */
#define RSOS_EBUSY (-6)     /* the object is in use (e.g. a batch still running)    */
#define RSOS_ERANGE (-7)    /* capacity exhausted (series full, t limit reached)    */

typedef struct rsos_handle rsos_handle;
typedef struct rsos_batch rsos_batch;

/* Parameters of one job: S surfaces of one L x L lattice.
 *   L            periodic edge, up to 65536; with tiling 0 a multiple of the
 *                tile edge, with tiling 1 at least the base edges (see tiling).
 *   N            step bound of Eq. 6, 1 <= N <= 7 (coded in B = ceil(log2(2N+1))
 *                bits per site and surface).
 *   surfaces     S >= 1.  S == 1 runs the plain path (int32 heights, lane 0 of
 *                the stream); S > 1 the multisurface path with ceil(S/32)
 *                32-lane words per site and bit plane.  Lane j of any job is the
 *                same surface whatever S is.
 *   tile_x/y     DT tile edges (section II; 8 x 8 in the paper).  With
 *                tiling 0 the tiles are square, 2, 4, 8 or 16, dividing L;
 *                with tiling 1 they are the base edges Tx, Ty (2..30 each) of
 *                a (+1) tiling.  Part of the model: they change the
 *                dynamics.  0 means 8.
 *   phase_order  0: random permutation of the four sub-tile sets each sweep;
 *                1: fixed order 0,1,2,3.
 *   series_capacity  number of measurements the device series buffer holds
 *                (0 means 1024).
 *   engine       0 auto (the persistent engine for multisurface jobs on a
 *                regular tiling with at least 8 tile rows), 1 one launch per
 *                phase, 2 persistent dataflow kernel.  Every engine gives
 *                bit-identical results.
 *   seed         Philox key of the job.
 * Execution geometry of the persistent engine (no counterpart in the paper;
 * results are bit-identical for every choice; 0 = automatic, see
 * rsos_autotune):
 *   words_per_thread  32-lane words each thread holds: 1, 2 (uint64; needs
 *                an even number of words) or 4 (128-lane words, section II's
 *                SIMT groups of 128 realizations; needs whole groups of 128
 *                surfaces, 8 x 8 tiles and the persistent engine: engine 2,
 *                or engine 0 with L >= 64; RSOS_EINVAL otherwise).
 *   tiles_per_lane  tiles a lane runs per work item, 1..64; automatic: 2,
 *                more (up to 16 with 32-bit, 4 with 64-bit words) on large
 *                lattices while each phase keeps enough work items for every
 *                worker warp.
 *   phase_lag    slots between consecutive phase fronts of the ticket order,
 *                >= 2.
 *   tiling       0: regular tiles (above).  1: the (+1) tilings of the
 *                decomposition check (section III.C: 6(+1) x 10(+1)): along
 *                each axis the first L mod T of the L div T tiles are one
 *                site wider (needs L mod T <= L div T), every tile is halved
 *                into floor(w/2) and the rest, and the per-sweep origin is
 *                uniform over one period of the pattern (T if T divides L,
 *                else L).  With T even and dividing L it is the regular
 *                tiling, bit for bit.  Multisurface jobs (surfaces >= 2)
 *                only; engine 0 (auto) and 1 run one launch per phase,
 *                engine 2 the persistent engine, whose windows (the widest
 *                half of either axis plus halo) must fit a block (RSOS_EINVAL
 *                otherwise); the lattice rows hold T ceil(L / T) site records
 *                (T = tile_x). */
typedef struct {
    int32_t L;
    int32_t N;
    int32_t surfaces;
    int32_t tile_x;
    int32_t tile_y;
    int32_t phase_order;
    int32_t series_capacity;
    int32_t engine;
    uint64_t seed;
    int32_t words_per_thread;
    int32_t tiles_per_lane;
    int32_t phase_lag;
    int32_t tiling;
} rsos_params;

/* Bytes of device memory a job needs (lattice planes, h(0,0) per surface,
 * measurement scratch, series buffer).  Returns RSOS_EINVAL for invalid
 * params. */
int rsos_required_bytes(const rsos_params* params, size_t* bytes);

/* Autotuner of the execution geometry (no counterpart in the paper).  Times
 * candidate (words_per_thread, tiles_per_lane, phase_lag) settings of the
 * persistent engine for params' (L, N, surfaces, tile, phase order) on a
 * scratch job the library allocates and frees: `sweeps` timed sweeps after 3
 * warm-up sweeps each, CUDA events on stream.  Never changes the model (tile
 * size, N, seed): every candidate gives bit-identical results.  *tuned =
 * params with the fastest geometry filled in (fields already non-zero in
 * params are kept fixed); *us_per_sweep (nullable) = its time.  Results are
 * cached per device and (L, N, surfaces, tile, phase order, fixed fields):
 * a repeated call returns at once.  Jobs that do not use the persistent
 * engine are returned unchanged.  Synchronises the stream.  RSOS_EINVAL for
 * invalid params or sweeps < 1, RSOS_ENOMEM / RSOS_ECUDA as rsos_init. */
int rsos_autotune(const rsos_params* params, int32_t sweeps, rsos_params* tuned, double* us_per_sweep,
                  void* stream);

/* Create a job at time t = 0 with the flat initial condition (section II).
 *   dev_buf/dev_bytes  NULL/0: the library allocates the device memory from
 *                its stream-ordered pool on `stream` (no device-wide
 *                synchronisation; blocks released by rsos_free are reused)
 *                and later frees it; otherwise a caller-owned device buffer
 *                of at least rsos_required_bytes bytes, 256-byte aligned, that
 *                must outlive the handle (the library never frees it).
 *   stream       the allocation and the initialisation kernels are queued on
 *                it (asynchronous).  Later calls may use other streams: a
 *                call on a stream other than that of the handle's previous
 *                call first makes its stream wait for the earlier work.
 *   out          receives the handle (set to NULL on error).                  */
int rsos_init(const rsos_params* params, void* dev_buf, size_t dev_bytes, void* stream,
              rsos_handle** out);

/* Queue n_sweeps DT sweeps (t -> t + n_sweeps) on stream; asynchronous.  A
 * sweep is one pass of the double tiling (section II): the tiling origin is
 * drawn, then the four sub-tile sets are updated in turn, each active
 * sub-tile receiving 2a selections of Eq. 6 (L^2 expected attempts per
 * surface, one MCS).  At
 * every time in the measurement schedule (rsos_schedule) reached on the way,
 * exact sums are computed on the device and appended to the series buffer.
 * RSOS_ERANGE if t would exceed 2^32 - 1 or the series buffer would overflow. */
int rsos_sweep(rsos_handle* h, int64_t n_sweeps, void* stream);

/* Measure now (time t of the handle) and return per surface, into host
 * arrays of length S: sum_h = sum h, sum_h2 = sum h^2 (Eq. 2 numerators,
 * exact), w2 = W^2 (nullable), and *t_out = t (nullable).  Synchronises the
 * stream.  RSOS_EOVERFLOW if some sum does not fit int64 (then the affected
 * sums are set to INT64_MIN while w2 stays exact to double rounding). */
int rsos_width(rsos_handle* h, int64_t* sum_h, int64_t* sum_h2, double* w2, int64_t* t_out,
               void* stream);

/* Set the measurement schedule: ascending times (completed sweeps, Eq. 10 or
 * log-spaced); times <= the current t are ignored.  Copies the array.  A time
 * of 0 on a fresh handle records the flat start. */
int rsos_schedule(rsos_handle* h, const int64_t* times, int32_t n);

/* Copy the measured series to host arrays: times[cap], sum_h[cap*S],
 * sum_h2[cap*S], w2[cap*S] (row m = measurement m, column = surface; any of
 * the last three nullable).  *n_out receives the number of rows written
 * (min(cap, measurements so far)).  Synchronises the stream.
 * RSOS_EOVERFLOW as for rsos_width. */
int rsos_read_series(rsos_handle* h, int64_t* times, int64_t* sum_h, int64_t* sum_h2, double* w2,
                     int32_t cap, int32_t* n_out, void* stream);

/* Height-distribution moments (section III.C: skewness and kurtosis of the
 * heights in the steady state need the third and fourth central moments).
 * rsos_set_moments(h, 1): every later measurement (scheduled or rsos_moments)
 * also records sum h^3 and sum h^4 per surface, exactly; 0 returns to
 * sum h and sum h^2 only (the cheaper measurement).  RSOS_EINVAL for NULL or
 * on not 0/1. */
int rsos_set_moments(rsos_handle* h, int32_t on);

/* Measure now with moments: sums[S][8] (host, caller-owned) receives per
 * surface sum h^k for k = 1, 2, 3, 4, each as a two's-complement 128-bit
 * integer (low 64 bits, then high 64 bits); *t_out = t (nullable).
 * Synchronises the stream. */
int rsos_moments(rsos_handle* h, int64_t* sums, int64_t* t_out, void* stream);

/* The measured series with moments: times[cap] (nullable), sums[cap][S][8] as
 * for rsos_moments, has[cap] (nullable) = 1 where the row was measured with
 * moments on (elsewhere words 4..7 of each surface are 0).  *n_out receives
 * min(cap, measurements so far).  Synchronises the stream. */
int rsos_read_moments(rsos_handle* h, int64_t* times, int64_t* sums, int8_t* has, int32_t cap, int32_t* n_out,
                      void* stream);

/* Checkpoint / resume (no counterpart in the paper).  With counter-based
 * Philox a job's whole state is its parameters, t, the coded lattice (or the
 * heights of the plain path), h(0,0) per surface, the measurement schedule
 * and the measured series; a restored job continues bit-identically.
 * rsos_snapshot_bytes: size of the snapshot of h in bytes.
 * rsos_snapshot: write it into host_buf (caller-owned, >= that size;
 *   RSOS_ENOMEM if smaller); synchronises the stream.
 * rsos_restore: a new handle from a snapshot, like rsos_init (dev_buf /
 *   dev_bytes as there); RSOS_EINVAL if the bytes are not a snapshot of this
 *   format (checked before any device work).  Synchronises the stream. */
int rsos_snapshot_bytes(const rsos_handle* h, size_t* bytes);
int rsos_snapshot(rsos_handle* h, void* host_buf, size_t bytes, void* stream);
int rsos_restore(const void* host_buf, size_t bytes, void* dev_buf, size_t dev_bytes, void* stream,
                 rsos_handle** out);

/* Absolute heights of one surface at the current time into host_LxL
 * (row-major, x fastest, int64 [L*L]: heights pass 2^31 after long growth
 * runs, e.g. N = 4 beyond about 10^9 sweeps, and a checkpoint may restore any
 * height).  Synchronises the stream. */
int rsos_heights(rsos_handle* h, int32_t surface, int64_t* host_LxL, void* stream);

/* Fault-detection self-test of the persistent engine (no counterpart in the
 * paper).  Queues one launch whose every dependency wait can never be
 * satisfied (it asks for sweep t+2 before t+1 ran), so each wait expires after
 * budget_ns nanoseconds; checks that the launch reported the expiry, clears
 * the error word and returns RSOS_ETIMEOUT.  The lattice and t are untouched
 * and the handle stays usable.  RSOS_EINVAL unless the handle uses the
 * persistent engine.  Synchronises the stream. */
int rsos_selftest_timeout(rsos_handle* h, int64_t budget_ns, void* stream);

/* Number of CUDA kernels this handle has queued so far (initialisation,
 * sweeps, measurements); for accounting and benchmarks. */
int rsos_launches(const rsos_handle* h, int64_t* out);

/* Width measurement that allocates nothing (no counterpart in the paper).
 * For callers that cannot allocate device memory when they need a width:
 * code under a fixed memory budget handed out once (an arena owned by another
 * framework), real-time loops where an allocation would synchronise the
 * device, or jobs whose caller-owned buffer holds only the lattice.  Computes
 * the same exact per-surface sums as rsos_width for a multisurface lattice
 * (surfaces >= 2) given by device pointers:
 *   params  the job's parameters (as passed to rsos_init);
 *   planes  the coded lattice; in a caller-owned rsos_init buffer it starts at
 *           offset 0;
 *   h00     the surfaces' absolute heights of site (0,0) (int64 each); in a
 *           caller-owned buffer at offset B*L*L*ceil(S/32)*4 rounded up to a
 *           multiple of 256, B = ceil(log2(2N+1)) (with tiling 1, L*L there
 *           is L*T*ceil(L/T), T = tile_x: rows padded to whole column
 *           classes);
 *   sums    device output, surfaces x 4 int64: sum h (low, high 64 bits) and
 *           sum h^2 (low, high) as two's-complement 128-bit integers.
 * Queued on stream, asynchronous; calls no cudaMalloc or cudaFree.  Scratch is
 * one file-scope device array of RSOS_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library keeps until the process exits; lattices whose
 * measurement needs more (about 4*L*32*ceil(S/32) bytes plus per-column sums)
 * get RSOS_ERANGE.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) and keeps it for the life of the process,
 * so make that first call before any stream capture, and do not call it
 * again on a device after cudaDeviceReset (the array may then live at another
 * address).  Every call reuses the same array: calls that overlap on the GPU
 * (different streams or host threads) race and must be serialised by the
 * caller.  RSOS_EINVAL for invalid params, NULL pointers or a single-surface
 * job, RSOS_ECUDA if a CUDA call fails. */
#define RSOS_NOALLOC_SCRATCH_BYTES (8u << 20)
int rsos_width_noalloc(const rsos_params* params, const uint32_t* planes, const int64_t* h00, int64_t* sums,
                       void* stream);

/* Current time of the handle (completed sweeps). */
int rsos_time(const rsos_handle* h, int64_t* t_out);

/* Release the handle and the device memory it allocated (no counterpart in
 * the paper).  NULL-safe.
 * Stream-ordered: the memory goes back to the library's device memory pool
 * once the work last queued through the handle (on the stream of its most
 * recent call, which must still exist) has finished; neither the host nor
 * the device waits. */
int rsos_free(rsos_handle* h);

/* Static description of a status code. */
const char* rsos_strerror(int status);

/* 1 if this library is the bounds-checked build (RSOS_CHECKED: every record
 * a sweep kernel stages or writes back is tested against the lattice and
 * every shared-memory record against the block's dynamic shared memory; a
 * failed test is counted and the access skipped), else 0. */
int rsos_checked_build(void);

/* Out-of-range accesses counted for this job since rsos_init (always 0 in
 * the normal build, which does not test).  Synchronises the stream.
 * RSOS_EINVAL for NULL arguments, RSOS_ECUDA on a CUDA error. */
int rsos_bounds_errors(rsos_handle* h, uint32_t* count, void* stream);

/* Integer throughput of this GPU, measured (no counterpart in the paper: the
 * integer-pipe roofline of the sweep).  kind 0: 3-input logic (lop3, the
 * ALU pipe that runs the bit-sliced Eq. 6 test); 1: 32-bit multiply-add
 * (mad.lo, the FMA pipe of Philox and the site mapping); 2: Philox-4x32-10
 * blocks with precomputed round keys.  Runs `iters` iterations per thread of
 * a fixed instruction chain on 2048 threads per SM after a short warm-up,
 * timed with CUDA events on stream.  *per_s = 32-bit lane operations
 * (kinds 0, 1) or Philox blocks (kind 2) per second.  Synchronises the
 * stream.  RSOS_EINVAL for a bad kind, iters outside 1..2^30 or a NULL
 * per_s; RSOS_ECUDA on a CUDA error. */
int rsos_peak_int(int32_t kind, int64_t iters, double* per_s, void* stream);

/* CUDA error code behind the last RSOS_ECUDA of the handle (0 if none); with
 * h == NULL, the CUDA error of the last failed rsos_init on this thread. */
int rsos_last_cuda_error(const rsos_handle* h);

/* Advance several independent jobs together to their targets (t_target[i] >=
 * the job's time): multisurface jobs of equal N, word width and tile share one
 * persistent launch per class (the warps crowd onto as few jobs as keep them
 * busy), stopping at every scheduled measurement time on the way; other jobs
 * run through rsos_sweep.  Results are bit-identical to advancing each job
 * alone.  Synchronises the stream (the continuous-batching primitive of a
 * serving loop: admit and retire jobs between calls).  RSOS_EINVAL for a NULL
 * or repeated handle or a target before the job's time, RSOS_ETIMEOUT if a
 * device wait gave up. */
int rsos_advance(rsos_handle* const* jobs, const int64_t* t_target, int32_t n, void* stream);

/* ---------------------------------------------------------------------------
 * Batches: many independent jobs of different L and N advanced together by
 * one persistent dataflow kernel (captured in a CUDA graph), each to its own
 * final time.  Jobs never interact; every job's result is bit-identical to the
 * same job run alone.
 * ------------------------------------------------------------------------- */

/* Create a batch of n_jobs jobs (params[i], t_max[i] sweeps each) whose device
 * memory must fit hbm_budget bytes (0 = no limit).  Each job starts flat at
 * t = 0; its width is measured at t_max (and at the times of its schedule, if
 * set with rsos_batch_schedule).  Regular multisurface jobs share the
 * multi-job persistent launches; single-surface jobs and (+1) tilings run
 * through their own handles inside the batch.  RSOS_ENOMEM if the budget is
 * exceeded. */
int rsos_batch_create(const rsos_params* params, const int64_t* t_max, int32_t n_jobs,
                      size_t hbm_budget, rsos_batch** out);

/* Per-job measurement schedule (ascending times <= t_max[job]); optional. */
int rsos_batch_schedule(rsos_batch* b, int32_t job, const int64_t* times, int32_t n);

/* Queue the whole batch on stream (asynchronous).  A device wait that exceeds
 * its time limit ends the launch with RSOS_ETIMEOUT reported by
 * rsos_batch_poll. */
int rsos_batch_run(rsos_batch* b, void* stream);

/* Non-blocking: ids of jobs finished since the last poll into done_ids
 * (capacity cap), count into *n_done.  Returns RSOS_ETIMEOUT if the device
 * reported a wait that gave up, RSOS_EBUSY while work is in flight and no job
 * finished, else RSOS_OK. */
int rsos_batch_poll(rsos_batch* b, int32_t* done_ids, int32_t cap, int32_t* n_done);

/* Handle of job i of the batch (for rsos_width / rsos_read_series /
 * rsos_heights after the job finished).  Owned by the batch. */
int rsos_batch_job(rsos_batch* b, int32_t job, rsos_handle** out);

/* Synchronise and release the batch and all its jobs.  NULL-safe. */
int rsos_batch_free(rsos_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* RSOS_H */
