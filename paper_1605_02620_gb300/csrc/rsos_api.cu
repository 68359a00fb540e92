// C ABI of the RSOS multisurface sweep (declared in include/rsos.h).
//
// A handle owns one job: S surfaces of an L x L periodic lattice with step
// bound N (Eq. 6), DT tile T x T (section II), a Philox key, and its time t
// (completed sweeps).  rsos_sweep queues, per sweep, the four phase launches
// of the double tiling (section II), and after every scheduled time the exact
// width measurement of Eq. 2.  No exception crosses the ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/rsos.h"
#include "rsos_geometry.h"
#include "rsos_launch.h"

using rsos::JobDev;

struct rsos_handle {
    rsos_params p;
    bool plain;
    int SX, B, NW, NWT, S_pad;
    JobDev J;
    bool general;        // (+1) tiling of section III.C
    rsos::GenTiling G;   // its geometry (general only)
    unsigned char* base;
    size_t bytes;
    bool owns;
    int32_t* row0;
    int64_t* partial;
    int ncb;
    int64_t* rec;  // [cap + 1][S_pad][kRecWords]; the last row is rsos_width's scratch
    int cap;
    std::vector<int64_t> series_t;
    std::vector<char> series_mom;  // row m also holds sum h^3, sum h^4
    bool moments;                  // measurements record sum h^3, sum h^4 too
    int64_t t;
    std::vector<int64_t> sched;
    size_t sched_pos;
    int sticky;
    int cuda_err;
    size_t smem_budget;
    // persistent engine
    bool persist;
    int rows;  // tile rows of its items (L / T; L div Ty on a (+1) tiling)
    rsos::PersistPlan plan;
    unsigned long long* done;
    unsigned long long* ticket;
    unsigned int* err;
    long long budget_ns;
    int64_t launches;  // kernels queued by this handle
    // Stream of the handle's most recent work; a call on another stream first
    // waits for it (an event recorded on the old stream), so work queued
    // through the handle stays in order whatever streams the caller uses.
    cudaStream_t last_stream;
    cudaEvent_t switch_ev;
};

namespace {

constexpr int64_t kMaxSweeps = 0xFFFFFFFFll;

// int64 words per surface and measurement in the series buffer: sum h^k for
// k = 1..4 as 128-bit (lo, hi) pairs (k = 3, 4 only when moments are on).
constexpr int kRecWords = 8;

// CUDA error of the last failed rsos_init on this thread (no handle exists).
thread_local int g_init_cuda_err = 0;

struct Layout {
    size_t planes, h00, row0, partial, rec, persist, check, total;
    int ncb, S_pad, B, NW, T, cap;
    int nTc;    // class columns per row of the layout
    int CW, K;  // persistent engine: tiles per block, chunks per tile row
    int rows;   // persistent engine: tile rows (L / Ty)
    bool plain, persist_on;
};

// Tiles per lane and work item of the persistent engine (execution geometry
// only): params->tiles_per_lane if set, else RSOS_TILES_PER_LANE, else the
// automatic choice (rsos_geometry.h).
int persist_tiles_per_lane(const rsos_params* p, int NWP, int NWT, int rows, int nT)
{
    if (p->tiles_per_lane > 0) return p->tiles_per_lane;
    if (const char* env = std::getenv("RSOS_TILES_PER_LANE")) {
        const int v = std::atoi(env);
        if (v >= 1 && v <= 64) return v;
    }
    return rsos::auto_tiles_per_lane(NWP, NWT, rows, nT);
}

// Tiles per work item: one warp's 32 lanes over the lane-word groups of a
// tile, times the tiles per lane.
int persist_block_tiles(const rsos_params* p, int NWP, int NWT, int rows, int nT)
{
    const int cw = 32 / NWP;
    return (cw < 1 ? 1 : cw) * persist_tiles_per_lane(p, NWP, NWT, rows, nT);
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// 32-lane words per thread: 2 (uint64 registers) when the job has an even
// number of words and 2 bit planes, else 1.  With 3 or 4 planes a uint64
// window is 1.5-2x larger, so fewer warps fit an SM; one word per thread was
// measured faster there (L = 4096, 64 surfaces: 287 vs 305 us per sweep at
// N = 2, 420 vs 499 at N = 4), unless it would need more than 32 threads per
// tile.  params->words_per_thread, else RSOS_WORDS_PER_THREAD=1, overrides
// it (execution geometry only; results are identical); 4 (128-lane words,
// section II's widest multisurface word) only when asked for.
int words_per_thread(const rsos_params* p, int NW)
{
    if (p->words_per_thread == 1 || p->words_per_thread == 2 || p->words_per_thread == 4) return p->words_per_thread;
    if (const char* env = std::getenv("RSOS_WORDS_PER_THREAD"))
        if (std::atoi(env) == 1) return 1;
    if (NW % 2 != 0) return 1;
    if (rsos::bits_for_step(p->N) >= 3 && NW <= 32) return 1;
    return 2;
}

// Windows of the (+1)-tiling persistent engine (the widest half of either
// axis plus its halo, per thread of a block of kGenPersistWarps warps) fit a
// block's shared memory.
bool gen_persist_fits(const rsos_params* p)
{
    const int T = p->tile_x == 0 ? 8 : p->tile_x, Ty = p->tile_y == 0 ? 8 : p->tile_y;
    const rsos::GenTiling G = rsos::gen_tiling(p->L, T, Ty);
    const int NW = (p->surfaces + 31) / 32;
    const size_t per_thread =
        (size_t)(G.max_w + 2) * (G.max_h + 2) * rsos::bits_for_step(p->N) * 4 * (size_t)words_per_thread(p, NW);
    return per_thread * 32 * rsos::kGenPersistWarps <= 227 * 1024;
}

int validate(const rsos_params* p)
{
    if (!p) return RSOS_EINVAL;
    const int T = p->tile_x == 0 ? 8 : p->tile_x;
    const int Ty = p->tile_y == 0 ? 8 : p->tile_y;
    if (p->tiling == 1) {
        // (+1) tilings: multisurface jobs on the phase engine; halves of at
        // most 16 sites (the kernel's k / w by multiplication), and a window
        // of 32 threads within one block's shared memory.
        if (T > 30 || Ty > 30 || p->L > 65536) return RSOS_EINVAL;
        if (!rsos::gen_axis_valid(p->L, T) || !rsos::gen_axis_valid(p->L, Ty)) return RSOS_EINVAL;
        if (p->surfaces < 2) return RSOS_EINVAL;
        if (p->N < 1 || p->N > 7 || p->surfaces > (1 << 20)) return RSOS_EINVAL;
        if (p->words_per_thread < 0 || p->words_per_thread > 2) return RSOS_EINVAL;
        const rsos::GenTiling G = rsos::gen_tiling(p->L, T, Ty);
        const int NWc = (p->surfaces + 31) / 32;
        const size_t per_thread = (size_t)(G.max_w + 2) * (G.max_h + 2) * rsos::bits_for_step(p->N) * 4 *
                                  (size_t)words_per_thread(p, NWc);
        if (per_thread * 32 > 200 * 1024) return RSOS_EINVAL;
        if (p->engine == 2 && !gen_persist_fits(p)) return RSOS_EINVAL;
    } else {
        if (p->tiling != 0) return RSOS_EINVAL;
        if (T != Ty) return RSOS_EINVAL;
        if (T != 2 && T != 4 && T != 8 && T != 16) return RSOS_EINVAL;
        if (p->L < T || p->L > 65536 || p->L % T != 0) return RSOS_EINVAL;
    }
    if (p->N < 1 || p->N > 7) return RSOS_EINVAL;
    if (p->surfaces < 1 || p->surfaces > (1 << 20)) return RSOS_EINVAL;
    if (p->phase_order != 0 && p->phase_order != 1) return RSOS_EINVAL;
    if (p->series_capacity < 0 || p->series_capacity > (1 << 24)) return RSOS_EINVAL;
    if (p->engine < 0 || p->engine > 2) return RSOS_EINVAL;
    if (p->engine == 2 && p->surfaces == 1) return RSOS_EINVAL;  // plain path: phase engine only
    const int NW = (p->surfaces + 31) / 32;
    if (p->words_per_thread == 4) {
        // 128-lane words: the persistent engine on 8 x 8 tiles only (the
        // kernels instantiated for them), whole 128-lane groups
        if (T != 8 || NW % 4 != 0 || NW / 4 > 32 || p->surfaces < 2 || p->engine == 1) return RSOS_EINVAL;
        if (p->engine == 0 && p->L / T < 8) return RSOS_EINVAL;  // auto would pick the phase engine
    } else if (p->words_per_thread < 0 || p->words_per_thread > 2 || (p->words_per_thread == 2 && NW % 2 != 0)) {
        return RSOS_EINVAL;
    }
    if (p->tiles_per_lane < 0 || p->tiles_per_lane > 64) return RSOS_EINVAL;
    if (p->phase_lag < 0 || p->phase_lag == 1 || p->phase_lag > (1 << 20)) return RSOS_EINVAL;
    if (p->engine == 2) {
        const int NWT = words_per_thread(p, NW);
        if (NW / NWT > 32) return RSOS_EINVAL;
    }
    return RSOS_OK;
}

// Bytes of the coded lattice: int32 heights (plain), or L rows of T nTc
// site records (a (+1) tiling pads each row to whole class columns).
size_t lattice_bytes(const Layout& l, size_t L)
{
    return l.plain ? L * L * 4 : (size_t)l.B * L * (size_t)l.T * (size_t)l.nTc * l.NW * 4;
}

Layout layout_of(const rsos_params* p)
{
    Layout l;
    // Layout tile edge: column classes of the (x) tile edge; a (+1) tiling
    // keeps ceil(L / T) class columns per row (the last ones partly unused).
    l.T = p->tile_x == 0 ? 8 : p->tile_x;
    l.nTc = p->tiling == 1 ? rsos::gen_classes(p->L, l.T) : p->L / l.T;
    l.plain = p->surfaces == 1;
    l.B = rsos::bits_for_step(p->N);
    l.NW = (p->surfaces + 31) / 32;
    l.S_pad = l.plain ? 1 : l.NW * 32;
    l.cap = p->series_capacity == 0 ? 1024 : p->series_capacity;
    const size_t L = (size_t)p->L;
    JobDev J{};
    J.L = p->L;
    J.T = l.T;
    J.nT = l.nTc;
    J.NW = l.NW;
    l.ncb = rsos::measure_blocks(J, l.plain);
    l.planes = align256(lattice_bytes(l, L));
    l.h00 = align256((size_t)l.S_pad * 8);
    l.row0 = l.plain ? 0 : align256((size_t)l.S_pad * L * 4);
    l.partial = align256((size_t)l.ncb * l.S_pad * 6 * 8);  // moments need 6 words per entry
    l.rec = align256((size_t)(l.cap + 1) * l.S_pad * kRecWords * 8);
    // tiles per row and tile rows (a (+1) tiling: L div T of each axis)
    const int Ty = p->tile_y == 0 ? 8 : p->tile_y;
    const int nT = p->L / l.T;  // tiles per row (L div Tx on a (+1) tiling)
    l.rows = p->tiling == 1 ? p->L / Ty : nT;
    // Auto engine: the persistent dataflow engine for regular multisurface
    // jobs with at least 8 tile rows, one launch per phase otherwise.  On a
    // (+1) tiling the persistent engine runs only when asked for (engine 2):
    // its windows, sized for the widest half, leave 9 warps per SM (6(+1) x
    // 10(+1)), and at L = 9605 it measured 1.32 ms per sweep (4 tiles per
    // lane) against the phase engine's 1.28.
    l.persist_on = !l.plain && (p->engine == 2 || (p->engine == 0 && p->tiling == 0 && l.rows >= 8));
    if (l.persist_on && p->engine == 0) {
        // more lane-word groups than lanes of a warp: phase engine
        const int NWT = words_per_thread(p, l.NW);
        if (l.NW / NWT > 32) l.persist_on = false;
    }
    l.CW = l.K = 0;
    l.persist = 0;
    if (l.persist_on) {
        const int NWT = words_per_thread(p, l.NW);
        l.CW = persist_block_tiles(p, l.NW / NWT, NWT, l.rows, nT);
        l.K = (nT + l.CW - 1) / l.CW;
        l.persist = align256((size_t)4 * l.rows * 8) + 256;
    }
    l.check = 256;  // checked build: out-of-range access counter (last region)
    l.total = l.planes + l.h00 + l.row0 + l.partial + l.rec + l.persist + l.check;
    return l;
}

int fail_cuda(rsos_handle* h, cudaError_t e)
{
    if (e == cudaSuccess) return RSOS_OK;
    h->sticky = RSOS_ECUDA;
    h->cuda_err = (int)e;
    return RSOS_ECUDA;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Stream of a call on handle h: when it differs from the stream of the
// handle's previous work, the new stream waits for that work first.
cudaStream_t use_stream(rsos_handle* h, void* stream)
{
    const cudaStream_t s = as_stream(stream);
    if (s != h->last_stream) {
        cudaError_t e = cudaEventRecord(h->switch_ev, h->last_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->switch_ev, 0);
        // An old stream the caller has destroyed holds no more work of the
        // handle; clear the error so a later launch check does not see it.
        if (e != cudaSuccess) (void)cudaGetLastError();
        h->last_stream = s;
    }
    return s;
}

// Library-owned device memory comes from one stream-ordered pool per device
// (cudaMallocFromPoolAsync / cudaFreeAsync): creating and releasing a job
// never synchronises the device, so a serving loop can admit and retire jobs
// while others run.  Released blocks stay cached in the pool (up to a quarter
// of the device memory) for the next jobs.
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[kMaxPoolDevices] = {};

cudaError_t device_pool(cudaMemPool_t* out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            uint64_t keep = total_b / 4;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

// bytes of device memory, ordered on stream s, 256-byte aligned.
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = device_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e == cudaSuccess && (reinterpret_cast<uintptr_t>(*p) & 255u)) {
        cudaFreeAsync(*p, s);
        *p = nullptr;
        e = cudaErrorMisalignedAddress;
    }
    return e;
}

// Exact 128-bit (lo, hi) pair -> int64 with overflow flag.
bool fits64(int64_t lo, int64_t hi) { return hi == (lo < 0 ? -1 : 0); }

__int128 to128(int64_t lo, int64_t hi) { return ((__int128)hi << 64) | (__int128)(uint64_t)lo; }

// Eq. 2 from exact sums, evaluated around the integer part of the mean so the
// floating-point step only sees small numbers.
double width2_from_sums(__int128 sh, __int128 sh2, int64_t L)
{
    const __int128 area = (__int128)L * L;
    __int128 q = sh / area;
    if (sh % area < 0) q -= 1;
    const __int128 r = sh - q * area;  // 0 <= r < area
    const __int128 centred = sh2 - 2 * q * sh + q * q * area;  // sum (h - q)^2
    const double a = (double)area;
    const double m = (double)r / a;
    return (double)centred / a - m * m;
}

int measure_into(rsos_handle* h, int row, cudaStream_t s, bool moments)
{
    h->launches += h->plain ? 2 : 3;
    int64_t* dst = h->rec + (size_t)row * h->S_pad * kRecWords;
    return fail_cuda(h, moments ? rsos::launch_moments(h->J, h->plain, h->S_pad, h->row0, h->partial, h->ncb, dst, s)
                                : rsos::launch_measure(h->J, h->plain, h->S_pad, h->row0, h->partial, h->ncb, dst,
                                                       kRecWords, s));
}

int measure_due(rsos_handle* h, cudaStream_t s)
{
    while (h->sched_pos < h->sched.size() && h->sched[h->sched_pos] <= h->t) {
        if (h->sched[h->sched_pos] == h->t) {
            if ((int)h->series_t.size() >= h->cap) return RSOS_ERANGE;
            const int rc = measure_into(h, (int)h->series_t.size(), s, h->moments);
            if (rc) return rc;
            h->series_t.push_back(h->t);
            h->series_mom.push_back(h->moments ? 1 : 0);
        }
        ++h->sched_pos;
    }
    return RSOS_OK;
}

// One sweep on a (+1) tiling: the control draw over one period of the
// pattern, then one launch per phase.
int run_sweep_general(rsos_handle* h, cudaStream_t s)
{
    const uint32_t t = (uint32_t)h->t;
    const int L = h->J.L;
    const rsos::Control c =
        rsos::sweep_control(h->J.seed_lo, h->J.seed_hi, t, rsos::gen_period(L, h->p.tile_x),
                            rsos::gen_period(L, h->p.tile_y), h->p.phase_order);
    const rsos::GenOrigin o = rsos::gen_locate_origin_site(L, h->G, c.ox, c.oy);
    for (int p = 0; p < 4; ++p) {
        int n = 0;
        const cudaError_t e =
            rsos::launch_phase_general(h->J, h->G, h->NWT, t, p, c.perm[p], c.ox, c.oy, o, h->smem_budget, s, &n);
        h->launches += n;
        if (e != cudaSuccess) return fail_cuda(h, e);
    }
    h->t += 1;
    return RSOS_OK;
}

int run_sweep(rsos_handle* h, cudaStream_t s)
{
    if (h->general) return run_sweep_general(h, s);
    const uint32_t t = (uint32_t)h->t;
    const rsos::Control c = rsos::sweep_control(h->J.seed_lo, h->J.seed_hi, t, h->J.T, h->J.T,
                                                h->p.phase_order);
    const rsos::Origin00 o = rsos::locate_origin_site(h->J.L, h->J.T, c.ox, c.oy);
    for (int p = 0; p < 4; ++p) {
        cudaError_t e = h->plain
                            ? rsos::launch_phase_plain(h->J, h->SX, t, p, c.perm[p], c.ox, c.oy, h->smem_budget, s)
                            : rsos::launch_phase(h->J, h->SX, h->NWT, t, p, c.perm[p], c.ox, c.oy, o,
                                                 h->smem_budget, s);
        if (e != cudaSuccess) return fail_cuda(h, e);
        h->launches += 1;
    }
    h->t += 1;
    return RSOS_OK;
}

rsos::PersistArgs persist_args(const rsos_handle* h, uint32_t t0, int64_t n)
{
    rsos::PersistArgs A;
    A.J = h->J;
    A.G.L = h->J.L;
    A.G.T = h->J.T;
    A.G.nT = h->J.nT;
    A.G.K = h->plan.K;
    A.G.D = h->plan.D;
    A.G.phase_order = h->p.phase_order;
    A.G.seed_lo = h->J.seed_lo;
    A.G.seed_hi = h->J.seed_hi;
    A.done = h->done;
    A.ticket = h->ticket;
    A.err = h->err;
    A.t0 = t0;
    A.n_tickets = (unsigned long long)n * 4ull * (unsigned long long)h->J.nT * (unsigned long long)h->plan.K;
    A.CW = h->plan.CW;
    A.TPL = h->plan.CW / (32 / h->J.NWP);
    A.budget_ns = h->budget_ns;
    return A;
}

// The (+1)-tiling engine's arguments: the same fields over the tiling's rows.
rsos::GenPersistArgs gen_persist_args(const rsos_handle* h, uint32_t t0, int64_t n)
{
    const rsos::PersistArgs R = persist_args(h, t0, n);
    rsos::GenPersistArgs A;
    A.J = R.J;
    A.G = h->G;
    A.S.L = h->J.L;
    A.S.y = h->G.y;
    A.S.Px = rsos::gen_period(h->J.L, h->p.tile_x);
    A.S.Py = rsos::gen_period(h->J.L, h->p.tile_y);
    A.S.K = h->plan.K;
    A.S.D = h->plan.D;
    A.S.phase_order = h->p.phase_order;
    A.S.seed_lo = h->J.seed_lo;
    A.S.seed_hi = h->J.seed_hi;
    A.done = R.done;
    A.ticket = R.ticket;
    A.err = R.err;
    A.t0 = t0;
    A.n_tickets = (unsigned long long)n * 4ull * (unsigned long long)h->rows * (unsigned long long)h->plan.K;
    A.CW = R.CW;
    A.TPL = R.TPL;
    A.budget_ns = R.budget_ns;
    return A;
}

// One persistent launch of sweeps [t0, t0 + n) (after the ticket reset).
cudaError_t launch_job_persist(rsos_handle* h, uint32_t t0, int64_t n, cudaStream_t s)
{
    return h->general ? rsos::launch_gen_persist(h->p.N, h->NWT, gen_persist_args(h, t0, n), h->plan, s)
                      : rsos::launch_persist(h->J, h->SX, h->NWT, persist_args(h, t0, n), h->plan, s);
}

int run_persist_segment(rsos_handle* h, int64_t n, cudaStream_t s)
{
    // Tickets of one launch stay below 2^31: split very long segments.
    const int64_t per_sweep = 4ll * h->rows * h->plan.K;
    const int64_t max_sweeps = std::max<int64_t>(1, ((int64_t)1 << 31) / per_sweep);
    while (n > 0) {
        const int64_t m = std::min(n, max_sweeps);
        cudaError_t e = rsos::launch_zero(h->ticket, 8, s);
        if (e == cudaSuccess) e = launch_job_persist(h, (uint32_t)h->t, m, s);
        if (e != cudaSuccess) return fail_cuda(h, e);
        h->launches += 2;
        h->t += m;
        n -= m;
    }
    return RSOS_OK;
}

// Reads the persistent engine's error word (synchronises the stream).
int check_device_error(rsos_handle* h, cudaStream_t s)
{
    if (!h->persist) return RSOS_OK;
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, h->err, sizeof(v), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    if (v != 0) {
        h->sticky = RSOS_ETIMEOUT;
        return RSOS_ETIMEOUT;
    }
    return RSOS_OK;
}

void convert_row(const rsos_handle* h, const int64_t* rec_row, int64_t* sum_h, int64_t* sum_h2, double* w2,
                 bool* overflow)
{
    for (int j = 0; j < h->p.surfaces; ++j) {
        const int64_t* r = rec_row + (size_t)j * kRecWords;
        if (sum_h) {
            if (fits64(r[0], r[1])) sum_h[j] = r[0];
            else { sum_h[j] = INT64_MIN; *overflow = true; }
        }
        if (sum_h2) {
            if (fits64(r[2], r[3])) sum_h2[j] = r[2];
            else { sum_h2[j] = INT64_MIN; *overflow = true; }
        }
        if (w2) w2[j] = width2_from_sums(to128(r[0], r[1]), to128(r[2], r[3]), h->p.L);
    }
}

}  // namespace

namespace rsos {

cudaError_t launch_phase(const JobDev& J, int SX, int words_per_thread, uint32_t t, int p, int q, int ox, int oy,
                         const Origin00& o, size_t smem_budget, cudaStream_t s)
{
    switch (SX) {
        case 1: return launch_phase_s1(J, words_per_thread, t, p, q, ox, oy, o, smem_budget, s);
        case 2: return launch_phase_s2(J, words_per_thread, t, p, q, ox, oy, o, smem_budget, s);
        case 4: return launch_phase_s4(J, words_per_thread, t, p, q, ox, oy, o, smem_budget, s);
        case 8: return launch_phase_s8(J, words_per_thread, t, p, q, ox, oy, o, smem_budget, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_phase_plain(const JobDev& J, int SX, uint32_t t, int p, int q, int ox, int oy,
                               size_t smem_budget, cudaStream_t s)
{
    switch (SX) {
        case 1: return launch_phase_plain_s1(J, t, p, q, ox, oy, smem_budget, s);
        case 2: return launch_phase_plain_s2(J, t, p, q, ox, oy, smem_budget, s);
        case 4: return launch_phase_plain_s4(J, t, p, q, ox, oy, smem_budget, s);
        case 8: return launch_phase_plain_s8(J, t, p, q, ox, oy, smem_budget, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_persist(const JobDev& J, int SX, int words_per_thread, const PersistArgs& A, const PersistPlan& P,
                           cudaStream_t s)
{
    if (words_per_thread == 4) return SX == 4 ? launch_persist_w128(J, A, P, s) : cudaErrorInvalidValue;
    switch (SX) {
        case 1: return launch_persist_s1(J, words_per_thread, A, P, s);
        case 2: return launch_persist_s2(J, words_per_thread, A, P, s);
        case 4: return launch_persist_s4(J, words_per_thread, A, P, s);
        case 8: return launch_persist_s8(J, words_per_thread, A, P, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t plan_multi(int N, int SX, int words_per_thread, int* grid, int* block, size_t* smem)
{
    switch (SX) {
        case 1: return plan_multi_s1(N, words_per_thread, grid, block, smem);
        case 2: return plan_multi_s2(N, words_per_thread, grid, block, smem);
        case 4: return plan_multi_s4(N, words_per_thread, grid, block, smem);
        case 8: return plan_multi_s8(N, words_per_thread, grid, block, smem);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_multi(int N, int SX, int words_per_thread, const MultiArgs& M, int grid, int block, size_t smem,
                         cudaStream_t s)
{
    switch (SX) {
        case 1: return launch_multi_s1(N, words_per_thread, M, grid, block, smem, s);
        case 2: return launch_multi_s2(N, words_per_thread, M, grid, block, smem, s);
        case 4: return launch_multi_s4(N, words_per_thread, M, grid, block, smem, s);
        case 8: return launch_multi_s8(N, words_per_thread, M, grid, block, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t plan_persist(const JobDev& J, int SX, int words_per_thread, int block_tiles, int phase_lag,
                         PersistPlan* out)
{
    if (words_per_thread == 4)
        return SX == 4 ? plan_persist_w128(J, block_tiles, phase_lag, out) : cudaErrorInvalidValue;
    switch (SX) {
        case 1: return plan_persist_s1(J, words_per_thread, block_tiles, phase_lag, out);
        case 2: return plan_persist_s2(J, words_per_thread, block_tiles, phase_lag, out);
        case 4: return plan_persist_s4(J, words_per_thread, block_tiles, phase_lag, out);
        case 8: return plan_persist_s8(J, words_per_thread, block_tiles, phase_lag, out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rsos

extern "C" {

int rsos_required_bytes(const rsos_params* params, size_t* bytes)
{
    const int rc = validate(params);
    if (rc) return rc;
    if (!bytes) return RSOS_EINVAL;
    *bytes = layout_of(params).total;
    return RSOS_OK;
}

int rsos_init(const rsos_params* params, void* dev_buf, size_t dev_bytes, void* stream, rsos_handle** out)
{
    if (!out) return RSOS_EINVAL;
    *out = nullptr;
    const int rc = validate(params);
    if (rc) return rc;
    const Layout l = layout_of(params);
    if (dev_buf && (dev_bytes < l.total || (reinterpret_cast<uintptr_t>(dev_buf) & 255))) return RSOS_ENOMEM;
    rsos_handle* h = new (std::nothrow) rsos_handle();
    if (!h) return RSOS_ENOMEM;
    h->p = *params;
    h->general = params->tiling == 1;
    if (h->general) {
        h->p.tile_x = params->tile_x == 0 ? 8 : params->tile_x;
        h->p.tile_y = params->tile_y == 0 ? 8 : params->tile_y;
        h->G = rsos::gen_tiling(params->L, h->p.tile_x, h->p.tile_y);
    } else {
        h->p.tile_x = h->p.tile_y = l.T;
    }
    h->plain = l.plain;
    h->SX = l.T / 2;
    h->B = l.B;
    h->NW = l.NW;
    h->NWT = words_per_thread(params, l.NW);
    h->S_pad = l.S_pad;
    h->cap = l.cap;
    h->ncb = l.ncb;
    h->t = 0;
    h->sched_pos = 0;
    h->sticky = RSOS_OK;
    h->moments = false;
    h->cuda_err = 0;
    h->launches = l.persist_on ? 3 : 1;
    h->smem_budget = 113 * 1024;
    if (const char* env = std::getenv("RSOS_SMEM_BUDGET")) {
        const long v = std::atol(env);
        if (v >= 4096 && v <= 232448) h->smem_budget = (size_t)v;
    }
    h->bytes = l.total;
    h->last_stream = as_stream(stream);
    if (cudaEventCreateWithFlags(&h->switch_ev, cudaEventDisableTiming) != cudaSuccess) {
        g_init_cuda_err = (int)cudaGetLastError();
        delete h;
        return RSOS_ECUDA;
    }
    if (dev_buf) {
        h->base = static_cast<unsigned char*>(dev_buf);
        h->owns = false;
    } else {
        void* p = nullptr;
        const cudaError_t e = pool_alloc(&p, l.total, h->last_stream);
        if (e != cudaSuccess) {
            cudaEventDestroy(h->switch_ev);
            delete h;
            (void)cudaGetLastError();
            return RSOS_ENOMEM;
        }
        h->base = static_cast<unsigned char*>(p);
        h->owns = true;
    }
    unsigned char* cur = h->base;
    JobDev& J = h->J;
    J = JobDev{};
    if (h->plain) J.heights = reinterpret_cast<int32_t*>(cur);
    else J.planes = reinterpret_cast<uint32_t*>(cur);
    cur += l.planes;
    J.h00 = reinterpret_cast<int64_t*>(cur);
    cur += l.h00;
    h->row0 = l.row0 ? reinterpret_cast<int32_t*>(cur) : nullptr;
    cur += l.row0;
    h->partial = reinterpret_cast<int64_t*>(cur);
    cur += l.partial;
    h->rec = reinterpret_cast<int64_t*>(cur);
    cur += l.rec;
    h->persist = l.persist_on;
    h->done = nullptr;
    h->ticket = nullptr;
    h->err = nullptr;
    h->budget_ns = 1000000000ll;
    h->rows = l.rows;
    if (l.persist_on) {
        h->done = reinterpret_cast<unsigned long long*>(cur);
        cur += align256((size_t)4 * l.rows * 8);
        h->ticket = reinterpret_cast<unsigned long long*>(cur);
        h->err = reinterpret_cast<unsigned int*>(cur + 8);
    }
    J.L = params->L;
    J.T = l.T;
    J.nT = l.nTc;
    J.NW = l.NW;
    J.NWP = l.NW / h->NWT;
    J.N = params->N;
    J.B = l.B;
    J.phase_order = params->phase_order;
    J.seed_lo = (uint32_t)params->seed;
    J.seed_hi = (uint32_t)(params->seed >> 32);
    J.rk = rsos::philox_round_keys(J.seed_lo, J.seed_hi);
    J.bounds_err = reinterpret_cast<uint32_t*>(h->base + (l.total - l.check));
    cudaError_t e = cudaSuccess;
    if (l.persist_on) {
        e = h->general ? rsos::plan_gen_persist(J, h->G, h->NWT, l.CW, params->phase_lag, &h->plan)
                       : rsos::plan_persist(J, h->SX, h->NWT, l.CW, params->phase_lag, &h->plan);
        if (e == cudaSuccess && (h->plan.CW != l.CW || h->plan.K != l.K)) e = cudaErrorInvalidConfiguration;
        if (e == cudaSuccess) e = rsos::launch_zero(h->done, (size_t)4 * l.rows * 8, as_stream(stream));
        if (e == cudaSuccess) e = rsos::launch_zero(h->ticket, 16, as_stream(stream));
    }
    // Flat initial condition (section II): planes and h00 zero.
    if (e == cudaSuccess) e = rsos::launch_zero(h->base, l.planes + l.h00, as_stream(stream));
    if (e == cudaSuccess) e = rsos::launch_zero(J.bounds_err, l.check, as_stream(stream));
    if (e != cudaSuccess) {
        g_init_cuda_err = (int)e;
        (void)cudaGetLastError();
        if (h->owns) cudaFreeAsync(h->base, h->last_stream);
        cudaEventDestroy(h->switch_ev);
        delete h;
        return RSOS_ECUDA;
    }
    *out = h;
    return RSOS_OK;
}

int rsos_sweep(rsos_handle* h, int64_t n_sweeps, void* stream)
{
    if (!h || n_sweeps < 0) return RSOS_EINVAL;
    if (h->sticky) return h->sticky;
    if (h->t + n_sweeps > kMaxSweeps) return RSOS_ERANGE;
    // Capacity check before queueing anything.
    size_t due = 0;
    for (size_t k = h->sched_pos; k < h->sched.size() && h->sched[k] <= h->t + n_sweeps; ++k) ++due;
    if (h->series_t.size() + due > (size_t)h->cap) return RSOS_ERANGE;
    cudaStream_t s = use_stream(h, stream);
    int rc = measure_due(h, s);
    if (rc) return rc;
    const int64_t t_end = h->t + n_sweeps;
    while (h->t < t_end) {
        if (h->persist) {
            int64_t seg = t_end - h->t;
            if (h->sched_pos < h->sched.size() && h->sched[h->sched_pos] < t_end)
                seg = h->sched[h->sched_pos] - h->t;
            rc = run_persist_segment(h, seg, s);
        } else {
            rc = run_sweep(h, s);
        }
        if (rc) return rc;
        rc = measure_due(h, s);
        if (rc) return rc;
    }
    return RSOS_OK;
}

int rsos_checked_build(void)
{
#if defined(RSOS_CHECKED)
    return 1;
#else
    return 0;
#endif
}

int rsos_bounds_errors(rsos_handle* h, uint32_t* count, void* stream)
{
    if (!h || !count) return RSOS_EINVAL;
    cudaStream_t s = use_stream(h, stream);
    cudaError_t e = cudaMemcpyAsync(count, h->J.bounds_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return fail_cuda(h, e);
}

int rsos_selftest_timeout(rsos_handle* h, int64_t budget_ns, void* stream)
{
    if (!h || budget_ns <= 0) return RSOS_EINVAL;
    if (!h->persist) return RSOS_EINVAL;
    if (h->sticky) return h->sticky;
    cudaStream_t s = use_stream(h, stream);
    // Sweep t + 2 depends on sweep t + 1, which never runs: every wait of
    // this launch expires after budget_ns.
    const long long saved = h->budget_ns;
    h->budget_ns = budget_ns;
    cudaError_t e = rsos::launch_zero(h->ticket, 8, s);
    if (e == cudaSuccess) e = launch_job_persist(h, (uint32_t)(h->t + 2), 1, s);
    h->budget_ns = saved;
    if (e != cudaSuccess) return fail_cuda(h, e);
    unsigned int v = 0;
    e = cudaMemcpyAsync(&v, h->err, sizeof(v), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    // Clear the error word so the handle stays usable; nothing was written.
    e = rsos::launch_zero(h->ticket, 16, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    return v != 0 ? RSOS_ETIMEOUT : RSOS_OK;
}

int rsos_width(rsos_handle* h, int64_t* sum_h, int64_t* sum_h2, double* w2, int64_t* t_out, void* stream)
{
    if (!h || !sum_h || !sum_h2) return RSOS_EINVAL;
    if (h->sticky) return h->sticky;
    cudaStream_t s = use_stream(h, stream);
    int rc = check_device_error(h, s);
    if (rc) return rc;
    rc = measure_into(h, h->cap, s, false);
    if (rc) return rc;
    std::vector<int64_t> host((size_t)h->S_pad * kRecWords);
    cudaError_t e = cudaMemcpyAsync(host.data(), h->rec + (size_t)h->cap * h->S_pad * kRecWords, host.size() * 8,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    bool overflow = false;
    convert_row(h, host.data(), sum_h, sum_h2, w2, &overflow);
    if (t_out) *t_out = h->t;
    return overflow ? RSOS_EOVERFLOW : RSOS_OK;
}

int rsos_schedule(rsos_handle* h, const int64_t* times, int32_t n)
{
    if (!h || n < 0 || (n > 0 && !times)) return RSOS_EINVAL;
    for (int32_t k = 1; k < n; ++k)
        if (times[k] <= times[k - 1]) return RSOS_EINVAL;
    h->sched.assign(times, times + n);
    h->sched_pos = 0;
    while (h->sched_pos < h->sched.size() && h->sched[h->sched_pos] < h->t) ++h->sched_pos;
    return RSOS_OK;
}

int rsos_read_series(rsos_handle* h, int64_t* times, int64_t* sum_h, int64_t* sum_h2, double* w2, int32_t cap,
                     int32_t* n_out, void* stream)
{
    if (!h || cap < 0 || !n_out) return RSOS_EINVAL;
    if (h->sticky) return h->sticky;
    cudaStream_t s = use_stream(h, stream);
    const int rc = check_device_error(h, s);
    if (rc) return rc;
    const int n = std::min<int>(cap, (int)h->series_t.size());
    *n_out = n;
    if (n == 0) return RSOS_OK;
    std::vector<int64_t> host((size_t)n * h->S_pad * kRecWords);
    cudaError_t e = cudaMemcpyAsync(host.data(), h->rec, host.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    bool overflow = false;
    const int S = h->p.surfaces;
    for (int m = 0; m < n; ++m) {
        if (times) times[m] = h->series_t[m];
        convert_row(h, host.data() + (size_t)m * h->S_pad * kRecWords, sum_h ? sum_h + (size_t)m * S : nullptr,
                    sum_h2 ? sum_h2 + (size_t)m * S : nullptr, w2 ? w2 + (size_t)m * S : nullptr, &overflow);
    }
    return overflow ? RSOS_EOVERFLOW : RSOS_OK;
}

int rsos_set_moments(rsos_handle* h, int32_t on)
{
    if (!h || (on != 0 && on != 1)) return RSOS_EINVAL;
    h->moments = on != 0;
    return RSOS_OK;
}

int rsos_moments(rsos_handle* h, int64_t* sums, int64_t* t_out, void* stream)
{
    if (!h || !sums) return RSOS_EINVAL;
    if (h->sticky) return h->sticky;
    cudaStream_t s = use_stream(h, stream);
    int rc = check_device_error(h, s);
    if (rc) return rc;
    rc = measure_into(h, h->cap, s, true);
    if (rc) return rc;
    std::vector<int64_t> host((size_t)h->S_pad * kRecWords);
    cudaError_t e = cudaMemcpyAsync(host.data(), h->rec + (size_t)h->cap * h->S_pad * kRecWords, host.size() * 8,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    std::copy(host.begin(), host.begin() + (size_t)h->p.surfaces * kRecWords, sums);
    if (t_out) *t_out = h->t;
    return RSOS_OK;
}

int rsos_read_moments(rsos_handle* h, int64_t* times, int64_t* sums, int8_t* has, int32_t cap, int32_t* n_out,
                      void* stream)
{
    if (!h || cap < 0 || !n_out || !sums) return RSOS_EINVAL;
    if (h->sticky) return h->sticky;
    cudaStream_t s = use_stream(h, stream);
    const int rc = check_device_error(h, s);
    if (rc) return rc;
    const int n = std::min<int>(cap, (int)h->series_t.size());
    *n_out = n;
    if (n == 0) return RSOS_OK;
    std::vector<int64_t> host((size_t)n * h->S_pad * kRecWords);
    cudaError_t e = cudaMemcpyAsync(host.data(), h->rec, host.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    const int S = h->p.surfaces;
    for (int m = 0; m < n; ++m) {
        const bool mom = h->series_mom[m] != 0;
        if (times) times[m] = h->series_t[m];
        if (has) has[m] = mom ? 1 : 0;
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < kRecWords; ++k)
                sums[((size_t)m * S + j) * kRecWords + k] =
                    (mom || k < 4) ? host[((size_t)m * h->S_pad + j) * kRecWords + k] : 0;
    }
    return RSOS_OK;
}

int rsos_heights(rsos_handle* h, int32_t surface, int64_t* host_LxL, void* stream)
{
    if (!h || !host_LxL || surface < 0 || surface >= h->p.surfaces) return RSOS_EINVAL;
    if (h->sticky) return h->sticky;
    cudaStream_t s = use_stream(h, stream);
    const int rc = check_device_error(h, s);
    if (rc) return rc;
    const size_t n = (size_t)h->p.L * h->p.L;
    void* dev = nullptr;
    cudaError_t e = pool_alloc(&dev, n * 8, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return RSOS_ENOMEM;
    }
    e = rsos::launch_heights(h->J, h->plain, surface, h->row0, static_cast<int64_t*>(dev), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_LxL, dev, n * 8, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(dev, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return fail_cuda(h, e);
}

int rsos_launches(const rsos_handle* h, int64_t* out)
{
    if (!h || !out) return RSOS_EINVAL;
    *out = h->launches;
    return RSOS_OK;
}

int rsos_time(const rsos_handle* h, int64_t* t_out)
{
    if (!h || !t_out) return RSOS_EINVAL;
    *t_out = h->t;
    return RSOS_OK;
}

int rsos_free(rsos_handle* h)
{
    if (!h) return RSOS_OK;
    int rc = RSOS_OK;
    // Stream-ordered: the memory returns to the pool once the handle's last
    // queued work is done; the host does not wait and the device is not
    // synchronised.
    if (h->owns && cudaFreeAsync(h->base, h->last_stream) != cudaSuccess) rc = RSOS_ECUDA;
    if (cudaEventDestroy(h->switch_ev) != cudaSuccess) rc = RSOS_ECUDA;
    delete h;
    return rc;
}

const char* rsos_strerror(int status)
{
    switch (status) {
        case RSOS_OK: return "ok";
        case RSOS_EINVAL: return "invalid argument";
        case RSOS_ENOMEM: return "out of device memory or caller buffer too small/misaligned";
        case RSOS_ECUDA: return "CUDA error (handle poisoned)";
        case RSOS_EOVERFLOW: return "sum does not fit int64";
        case RSOS_ETIMEOUT: return "device wait timed out";
        case RSOS_EBUSY: return "busy";
        case RSOS_ERANGE: return "capacity or time limit exceeded";
        default: return "unknown status";
    }
}

int rsos_last_cuda_error(const rsos_handle* h) { return h ? h->cuda_err : g_init_cuda_err; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Multi-job execution (rsos_advance and batches).  Jobs are grouped into
// classes of equal (N, word width, tile edge); per round one multi-job
// persistent launch per class advances every member to its next stop (a
// measurement time or its target), then the members due for a measurement
// are measured.  Jobs outside the persistent engine run through rsos_sweep.
// ---------------------------------------------------------------------------
namespace {

struct BatchClass {
    int N, NWT, SX;
    std::vector<int> members;          // indices into MultiWork::jobs
    rsos::MultiJob* d_jobs;            // [rounds][members]
    unsigned long long* d_tickets;     // [members] tickets handed out, then [members] items finished
    unsigned int* d_first;             // 1
    unsigned int* d_exhausted;         // [members]
    unsigned int* d_err;               // 1
    int grid, block;
    size_t smem;
};

struct MultiWork {
    std::vector<rsos_handle*> jobs;
    std::vector<int64_t> target;
    std::vector<std::vector<int64_t>> stops;  // per job: ascending stop times, last = target
    std::vector<BatchClass> classes;
    std::vector<int> solo;
    size_t rounds = 0, per_round_jobs = 0;
    void* d_block = nullptr;           // class state
    void* d_tables = nullptr;          // job tables of all rounds
    rsos::MultiJob* h_jobs = nullptr;  // pinned staging of the job tables
    unsigned int* h_err = nullptr;     // pinned: error word of each class after its last launch
    // pooled: device buffers from the stream-ordered pool on `stream` and host
    // staging in the calling thread's cached pinned buffer (rsos_advance,
    // which synchronises the stream before it returns); otherwise plain
    // allocations that live as long as a batch.
    bool pooled = false;
    cudaStream_t stream = nullptr;
};

// Pinned host staging of rsos_advance, cached per thread and grown on demand:
// a call synchronises its stream before returning, so the next call on the
// same thread may reuse it.  Kept until the process exits.
struct PinnedCache {
    void* p = nullptr;
    size_t bytes = 0;
};
thread_local PinnedCache t_pinned;

void* pinned_scratch(size_t bytes)
{
    if (t_pinned.bytes < bytes) {
        if (t_pinned.p) cudaFreeHost(t_pinned.p);
        t_pinned.p = nullptr;
        t_pinned.bytes = 0;
        const size_t want = std::max<size_t>(bytes, 1 << 20);
        if (cudaHostAlloc(&t_pinned.p, want, cudaHostAllocDefault) != cudaSuccess) {
            t_pinned.p = nullptr;
            return nullptr;
        }
        t_pinned.bytes = want;
    }
    return t_pinned.p;
}

void multi_release(MultiWork& w)
{
    if (w.pooled) {
        if (w.d_tables) cudaFreeAsync(w.d_tables, w.stream);
        if (w.d_block) cudaFreeAsync(w.d_block, w.stream);
    } else {
        if (w.d_tables) cudaFree(w.d_tables);
        if (w.d_block) cudaFree(w.d_block);
        if (w.h_jobs) cudaFreeHost(w.h_jobs);
        if (w.h_err) cudaFreeHost(w.h_err);
    }
    w.d_tables = w.d_block = nullptr;
    w.h_jobs = nullptr;
    w.h_err = nullptr;
}

// Classes, launch plans, member order and all device / pinned buffers (no
// allocation happens later, so multi_enqueue can be captured in a graph).
// A job whose sweep holds at least twice as many work items as the GPU has
// worker warps keeps every warp busy alone: it runs through its own
// single-job persistent launches (one after another), and only the smaller
// jobs share the multi-job launches, where they run side by side.
bool fills_gpu(const rsos_handle* h)
{
    const int64_t items = 4ll * h->rows * h->plan.K;
    const int64_t workers = (int64_t)h->plan.grid * (h->plan.nthr / 32);
    return items >= 2 * workers;
}

int multi_prepare(MultiWork& w)
{
    for (size_t i = 0; i < w.jobs.size(); ++i) {
        rsos_handle* h = w.jobs[i];
        // the multi-job kernel runs regular tilings of 32- and 64-bit words
        if (!h->persist || h->general || fills_gpu(h) || h->NWT == 4) {
            w.solo.push_back((int)i);
            continue;
        }
        bool placed = false;
        for (BatchClass& c : w.classes)
            if (c.N == h->p.N && c.NWT == h->NWT && c.SX == h->SX) {
                c.members.push_back((int)i);
                placed = true;
                break;
            }
        if (!placed) {
            BatchClass c{};
            c.N = h->p.N;
            c.NWT = h->NWT;
            c.SX = h->SX;
            c.members.push_back((int)i);
            w.classes.push_back(c);
        }
    }
    // Members in decreasing lattice size (then target): the tail of a class is
    // many small jobs, which run side by side.
    for (BatchClass& c : w.classes)
        std::stable_sort(c.members.begin(), c.members.end(), [&](int x, int y) {
            const int64_t lx = w.jobs[x]->p.L, ly = w.jobs[y]->p.L;
            return lx != ly ? lx > ly : w.target[x] > w.target[y];
        });
    size_t dev_bytes = 0;
    for (BatchClass& c : w.classes) {
        if (rsos::plan_multi(c.N, c.SX, c.NWT, &c.grid, &c.block, &c.smem) != cudaSuccess) {
            (void)cudaGetLastError();
            return RSOS_ECUDA;
        }
        dev_bytes += align256(2 * c.members.size() * 8) + 256 + align256(c.members.size() * 4) + 256;
        w.per_round_jobs += c.members.size();
        for (int i : c.members) w.rounds = std::max(w.rounds, w.stops[i].size());
    }
    if (w.classes.empty()) return RSOS_OK;
    const size_t entries = w.per_round_jobs * w.rounds;
    if (w.pooled) {
        const size_t tables = align256(entries * sizeof(rsos::MultiJob));
        unsigned char* host = static_cast<unsigned char*>(pinned_scratch(tables + 256));
        if (!host || pool_alloc(&w.d_block, dev_bytes, w.stream) != cudaSuccess ||
            pool_alloc(&w.d_tables, entries * sizeof(rsos::MultiJob), w.stream) != cudaSuccess) {
            (void)cudaGetLastError();
            return RSOS_ENOMEM;
        }
        w.h_jobs = reinterpret_cast<rsos::MultiJob*>(host);
        w.h_err = reinterpret_cast<unsigned int*>(host + tables);
    } else {
        if (cudaMalloc(&w.d_block, dev_bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            w.d_block = nullptr;
            return RSOS_ENOMEM;
        }
        if (cudaMalloc(&w.d_tables, entries * sizeof(rsos::MultiJob)) != cudaSuccess ||
            cudaHostAlloc((void**)&w.h_jobs, entries * sizeof(rsos::MultiJob), cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void**)&w.h_err, w.classes.size() * sizeof(unsigned int), cudaHostAllocDefault) !=
                cudaSuccess) {
            (void)cudaGetLastError();
            return RSOS_ENOMEM;
        }
    }
    unsigned char* cur = static_cast<unsigned char*>(w.d_block);
    rsos::MultiJob* dj = static_cast<rsos::MultiJob*>(w.d_tables);
    for (size_t ci = 0; ci < w.classes.size(); ++ci) {
        BatchClass& c = w.classes[ci];
        const size_t m = c.members.size();
        c.d_tickets = reinterpret_cast<unsigned long long*>(cur);
        cur += align256(2 * m * 8);
        c.d_first = reinterpret_cast<unsigned int*>(cur);
        c.d_err = reinterpret_cast<unsigned int*>(cur + 8);
        cur += 256;
        c.d_exhausted = reinterpret_cast<unsigned int*>(cur);
        cur += align256(m * 4) + 256;
        c.d_jobs = dj;
        dj += m * w.rounds;
        w.h_err[ci] = 0;
    }
    return RSOS_OK;
}

// Completion event of a job; under stream capture it must become an external
// event node of the graph so that the host can query it after the launch.
cudaError_t record_done(cudaEvent_t ev, cudaStream_t s, bool capturing)
{
    return capturing ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal) : cudaEventRecord(ev, s);
}

// Queue all rounds on stream s (no allocation: capturable).  done (nullable)
// gets each job's completion event.
int multi_enqueue(MultiWork& w, cudaStream_t s, bool capturing, const std::vector<cudaEvent_t>* done)
{
    for (int i : w.solo) {
        rsos_handle* h = w.jobs[i];
        const int rc = rsos_sweep(h, w.target[i] - h->t, s);
        if (rc) return rc;
        if (done && record_done((*done)[i], s, capturing) != cudaSuccess) return RSOS_ECUDA;
    }
    if (w.classes.empty()) return RSOS_OK;
    for (const BatchClass& c : w.classes)
        for (int i : c.members) {
            rsos_handle* h = w.jobs[i];
            size_t due = 0;
            for (size_t k = h->sched_pos; k < h->sched.size() && h->sched[k] <= w.target[i]; ++k) ++due;
            if (h->series_t.size() + due > (size_t)h->cap) return RSOS_ERANGE;
        }
    for (BatchClass& c : w.classes)
        if (rsos::launch_zero(c.d_err, 4, s) != cudaSuccess) return RSOS_ECUDA;
    for (size_t r = 0; r < w.rounds; ++r) {
        size_t off = 0;
        for (size_t ci = 0; ci < w.classes.size(); ++ci) {
            BatchClass& c = w.classes[ci];
            rsos::MultiJob* row = w.h_jobs + r * w.per_round_jobs + off;
            off += c.members.size();
            bool any = false;
            for (size_t m = 0; m < c.members.size(); ++m) {
                const int i = c.members[m];
                rsos_handle* h = w.jobs[i];
                int64_t stop = h->t;
                if (r < w.stops[i].size()) stop = std::max<int64_t>(h->t, w.stops[i][r]);
                const int64_t per_sweep = 4ll * h->J.nT * h->plan.K;
                if ((stop - h->t) * per_sweep >= ((int64_t)1 << 31)) return RSOS_ERANGE;
                const rsos::PersistArgs a = persist_args(h, (uint32_t)h->t, stop - h->t);
                rsos::MultiJob& mj = row[m];
                mj.J = a.J;
                mj.G = a.G;
                mj.done = a.done;
                mj.ticket = c.d_tickets + m;
                mj.finished = c.d_tickets + c.members.size() + m;
                mj.n_tickets = a.n_tickets;
                // in-flight cap: two thirds of the tickets between an item and
                // its dependencies ((D - 2) slots of 4K items)
                mj.cap = (unsigned long long)std::max<int64_t>(32, (int64_t)(h->plan.D - 2) * 4 * h->plan.K * 2 / 3);
                mj.t0 = a.t0;
                mj.CW = a.CW;
                mj.TPL = a.TPL;
                mj.pad_ = 0;
                any |= a.n_tickets > 0;
                h->t = stop;
            }
            if (any) {
                rsos::MultiJob* dj = c.d_jobs + r * c.members.size();
                cudaError_t e =
                    cudaMemcpyAsync(dj, row, c.members.size() * sizeof(rsos::MultiJob), cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess) e = rsos::launch_zero(c.d_tickets, 2 * c.members.size() * 8, s);
                if (e == cudaSuccess) e = rsos::launch_zero(c.d_first, 4, s);
                if (e == cudaSuccess) e = rsos::launch_zero(c.d_exhausted, c.members.size() * 4, s);
                rsos::MultiArgs M;
                M.jobs = dj;
                M.n_jobs = (int)c.members.size();
                M.first = c.d_first;
                M.exhausted = c.d_exhausted;
                M.err = c.d_err;
                M.budget_ns = 1000000000ll;
                if (e == cudaSuccess) e = rsos::launch_multi(c.N, c.SX, c.NWT, M, c.grid, c.block, c.smem, s);
                if (e != cudaSuccess) return RSOS_ECUDA;
            }
            for (int i : c.members) {
                rsos_handle* h = w.jobs[i];
                if (any) h->launches += 5;
                const int rc = measure_due(h, s);
                if (rc) return rc;
            }
        }
        for (size_t ci = 0; ci < w.classes.size(); ++ci)
            for (int i : w.classes[ci].members)
                if (w.stops[i].size() == r + 1) {
                    if (cudaMemcpyAsync(&w.h_err[ci], w.classes[ci].d_err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
                        return RSOS_ECUDA;
                    if (done && record_done((*done)[i], s, capturing) != cudaSuccess) return RSOS_ECUDA;
                }
    }
    return RSOS_OK;
}

// Stops of job h on the way to target: its pending schedule times, then target.
std::vector<int64_t> stops_of(const rsos_handle* h, int64_t target)
{
    std::vector<int64_t> out;
    for (size_t k = h->sched_pos; k < h->sched.size(); ++k)
        if (h->sched[k] > h->t && h->sched[k] < target) out.push_back(h->sched[k]);
    out.push_back(target);
    return out;
}

}  // namespace

extern "C" int rsos_advance(rsos_handle* const* jobs, const int64_t* t_target, int32_t n, void* stream)
{
    if (!jobs || !t_target || n < 1) return RSOS_EINVAL;
    MultiWork w;
    for (int32_t i = 0; i < n; ++i) {
        rsos_handle* h = jobs[i];
        if (!h || t_target[i] < h->t || t_target[i] > kMaxSweeps) return RSOS_EINVAL;
        if (h->sticky) return h->sticky;
        for (int32_t k = 0; k < i; ++k)
            if (jobs[k] == h) return RSOS_EINVAL;
        w.jobs.push_back(h);
        w.target.push_back(t_target[i]);
        w.stops.push_back(stops_of(h, t_target[i]));
    }
    cudaStream_t s = as_stream(stream);
    for (rsos_handle* h : w.jobs) {
        use_stream(h, stream);
        const int rc = measure_due(h, s);  // a measurement due at the current time
        if (rc) return rc;
    }
    w.pooled = true;
    w.stream = s;
    int rc = multi_prepare(w);
    if (rc == RSOS_OK) rc = multi_enqueue(w, s, false, nullptr);
    cudaError_t e = cudaStreamSynchronize(s);
    if (rc == RSOS_OK && e != cudaSuccess) rc = RSOS_ECUDA;
    if (rc == RSOS_OK)
        for (size_t ci = 0; ci < w.classes.size(); ++ci)
            if (w.h_err[ci]) rc = RSOS_ETIMEOUT;
    if (rc == RSOS_ECUDA) g_init_cuda_err = (int)(e != cudaSuccess ? e : cudaGetLastError());
    multi_release(w);
    return rc;
}

// ---------------------------------------------------------------------------
// Batches (include/rsos.h): a MultiWork over jobs the batch owns, with each
// job's schedule as its stops, captured in one CUDA graph.
// ---------------------------------------------------------------------------
struct rsos_batch {
    MultiWork w;
    std::vector<int64_t> t_max;
    std::vector<std::vector<int64_t>> sched;
    std::vector<cudaEvent_t> done;
    std::vector<char> reported;
    bool prepared;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool queued;
    int status;
};

extern "C" {

int rsos_batch_free(rsos_batch* b);

int rsos_batch_create(const rsos_params* params, const int64_t* t_max, int32_t n_jobs, size_t hbm_budget,
                      rsos_batch** out)
{
    if (!out) return RSOS_EINVAL;
    *out = nullptr;
    if (!params || !t_max || n_jobs < 1) return RSOS_EINVAL;
    std::vector<rsos_params> ps(params, params + n_jobs);
    size_t total = 0;
    for (int32_t i = 0; i < n_jobs; ++i) {
        if (t_max[i] < 0 || t_max[i] > kMaxSweeps) return RSOS_EINVAL;
        // regular multisurface jobs join the multi-job persistent launches;
        // plain jobs and (+1) tilings run through their own handles
        if (ps[i].surfaces > 1 && ps[i].engine == 0 && ps[i].tiling == 0) {
            const int NW = (ps[i].surfaces + 31) / 32;
            if (NW / words_per_thread(&ps[i], NW) <= 32) ps[i].engine = 2;
        }
        size_t bytes = 0;
        const int rc = rsos_required_bytes(&ps[i], &bytes);
        if (rc) return rc;
        total += bytes;
    }
    if (hbm_budget && total > hbm_budget) return RSOS_ENOMEM;
    rsos_batch* b = new (std::nothrow) rsos_batch();
    if (!b) return RSOS_ENOMEM;
    b->prepared = false;
    b->graph = nullptr;
    b->exec = nullptr;
    b->queued = false;
    b->status = RSOS_OK;
    for (int32_t i = 0; i < n_jobs; ++i) {
        rsos_handle* h = nullptr;
        const int rc = rsos_init(&ps[i], nullptr, 0, nullptr, &h);
        if (rc) {
            rsos_batch_free(b);
            return rc;
        }
        b->w.jobs.push_back(h);
        b->w.target.push_back(t_max[i]);
        b->t_max.push_back(t_max[i]);
        b->sched.push_back(std::vector<int64_t>{t_max[i]});
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            rsos_batch_free(b);
            return RSOS_ECUDA;
        }
        b->done.push_back(ev);
        b->reported.push_back(0);
    }
    *out = b;
    return RSOS_OK;
}

int rsos_batch_schedule(rsos_batch* b, int32_t job, const int64_t* times, int32_t n)
{
    if (!b || job < 0 || job >= (int32_t)b->w.jobs.size() || b->queued) return RSOS_EINVAL;
    if (n < 0 || (n > 0 && !times)) return RSOS_EINVAL;
    std::vector<int64_t> s(times, times + n);
    for (size_t k = 0; k < s.size(); ++k) {
        if (s[k] < 0 || s[k] > b->t_max[job] || (k && s[k] <= s[k - 1])) return RSOS_EINVAL;
    }
    if (s.empty() || s.back() != b->t_max[job]) s.push_back(b->t_max[job]);
    b->sched[job] = s;
    return RSOS_OK;
}

int rsos_batch_run(rsos_batch* b, void* stream)
{
    if (!b) return RSOS_EINVAL;
    if (b->queued) return RSOS_EBUSY;
    cudaStream_t s = as_stream(stream);
    MultiWork& w = b->w;
    for (rsos_handle* h : w.jobs) use_stream(h, stream);  // before capture: no cross-stream waits inside
    int rc = RSOS_OK;
    if (!b->prepared) {
        w.stops.clear();
        for (size_t i = 0; i < w.jobs.size(); ++i) {
            rsos_handle* h = w.jobs[i];
            rc = rsos_schedule(h, b->sched[i].data(), (int32_t)b->sched[i].size());
            if (rc) return rc;
            std::vector<int64_t> st;
            for (int64_t v : b->sched[i])
                if (v > h->t) st.push_back(v);
            if (st.empty() || st.back() != b->t_max[i]) st.push_back(b->t_max[i]);
            w.stops.push_back(st);
        }
        rc = multi_prepare(w);
        if (rc) return rc;
        b->prepared = true;
    }
    // a measurement due at the start time (t = 0 in the schedule)
    for (rsos_handle* h : w.jobs) {
        rc = measure_due(h, s);
        if (rc) return rc;
    }
    const char* env = std::getenv("RSOS_BATCH_GRAPH");
    const bool use_graph = !(env && std::atoi(env) == 0) && s != nullptr;
    if (use_graph) {
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            g_init_cuda_err = (int)e;
            return RSOS_ECUDA;
        }
        rc = multi_enqueue(w, s, true, &b->done);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(s, &g);
        if (rc == RSOS_OK && e != cudaSuccess) rc = RSOS_ECUDA;
        if (rc == RSOS_OK) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (rc == RSOS_OK && e != cudaSuccess) rc = RSOS_ECUDA;
        b->graph = g;
        if (rc == RSOS_OK) e = cudaGraphLaunch(b->exec, s);
        if (rc == RSOS_OK && e != cudaSuccess) rc = RSOS_ECUDA;
        if (rc != RSOS_OK) {
            g_init_cuda_err = (int)(e != cudaSuccess ? e : cudaGetLastError());
            (void)cudaGetLastError();
        }
    } else {
        rc = multi_enqueue(w, s, false, &b->done);
    }
    if (rc) {
        b->status = rc;
        return rc;
    }
    b->queued = true;
    return RSOS_OK;
}

int rsos_batch_poll(rsos_batch* b, int32_t* done_ids, int32_t cap, int32_t* n_done)
{
    if (!b || !n_done || cap < 0 || (cap > 0 && !done_ids)) return RSOS_EINVAL;
    *n_done = 0;
    if (b->status) return b->status;
    if (!b->queued) return RSOS_EBUSY;
    bool pending = false;
    for (size_t i = 0; i < b->w.jobs.size(); ++i) {
        if (b->reported[i]) continue;
        const cudaError_t e = cudaEventQuery(b->done[i]);
        if (e == cudaSuccess) {
            for (size_t ci = 0; ci < b->w.classes.size(); ++ci)
                if (b->w.h_err && b->w.h_err[ci]) {
                    b->status = RSOS_ETIMEOUT;
                    return RSOS_ETIMEOUT;
                }
            if (*n_done < cap) {
                done_ids[(*n_done)++] = (int32_t)i;
                b->reported[i] = 1;
            } else {
                pending = true;
            }
        } else if (e == cudaErrorNotReady) {
            pending = true;
        } else {
            g_init_cuda_err = (int)e;
            b->status = RSOS_ECUDA;
            return RSOS_ECUDA;
        }
    }
    return (*n_done == 0 && pending) ? RSOS_EBUSY : RSOS_OK;
}

int rsos_batch_job(rsos_batch* b, int32_t job, rsos_handle** out)
{
    if (!b || !out || job < 0 || job >= (int32_t)b->w.jobs.size()) return RSOS_EINVAL;
    *out = b->w.jobs[job];
    return RSOS_OK;
}

int rsos_batch_free(rsos_batch* b)
{
    if (!b) return RSOS_OK;
    int rc = RSOS_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) rc = RSOS_ECUDA;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t ev : b->done) cudaEventDestroy(ev);
    multi_release(b->w);
    for (rsos_handle* h : b->w.jobs) {
        h->last_stream = nullptr;  // the device is idle: release without the run's stream
        const int r = rsos_free(h);
        if (r) rc = r;
    }
    delete b;
    return rc;
}

}  // extern "C"

// ---- Autotuner of the execution geometry --------------------------------
namespace {

using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int>;
std::mutex g_tune_mutex;
std::map<TuneKey, std::pair<rsos_params, double>> g_tune_cache;

// Microseconds per sweep of one geometry on a scratch job: 3 warm-up
// sweeps, then `sweeps` sweeps between CUDA events.
int time_geometry(const rsos_params& p, int sweeps, cudaStream_t s, double* us)
{
    rsos_handle* h = nullptr;
    int rc = rsos_init(&p, nullptr, 0, s, &h);
    if (rc) return rc;
    rc = rsos_sweep(h, 3, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (!rc && e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (!rc && e == cudaSuccess) rc = rsos_sweep(h, sweeps, s);
    if (!rc && e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const int rc_free = rsos_free(h);
    if (rc) return rc;
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return RSOS_ECUDA;
    }
    if (rc_free) return rc_free;
    *us = 1e3 * (double)ms / sweeps;
    return RSOS_OK;
}

}  // namespace

extern "C" int rsos_autotune(const rsos_params* params, int32_t sweeps, rsos_params* tuned, double* us_per_sweep,
                             void* stream)
{
    if (!params || !tuned || sweeps < 1) return RSOS_EINVAL;
    int rc = validate(params);
    if (rc) return rc;
    *tuned = *params;
    if (us_per_sweep) *us_per_sweep = 0.0;
    const Layout l = layout_of(params);
    // nothing to choose outside the regular persistent engine ((+1) tilings
    // keep the automatic geometry)
    if (!l.persist_on || params->tiling == 1) return RSOS_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return RSOS_ECUDA;
    }
    const TuneKey key{dev, params->L, params->N, params->surfaces, l.T, params->phase_order,
                      params->words_per_thread, params->tiles_per_lane, params->phase_lag};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *tuned = it->second.first;
            tuned->seed = params->seed;
            tuned->series_capacity = params->series_capacity;
            if (us_per_sweep) *us_per_sweep = it->second.second;
            return RSOS_OK;
        }
    }
    // Candidates: words per thread {1, 2}, work items of 32 / 64 / 128 tiles
    // and the automatic choice, the automatic phase lag and a shorter one;
    // fields set by the caller stay.
    std::vector<int> wpts, tpls_items, lags;
    if (params->words_per_thread) wpts = {params->words_per_thread};
    else {
        wpts = {1};
        if (l.NW % 2 == 0) wpts.push_back(2);
    }
    const int nT = params->L / l.T;
    if (params->phase_lag) lags = {params->phase_lag};
    else {
        lags = {0};
        if (nT / 6 >= 2) lags.push_back(nT / 6);
    }
    cudaStream_t s = as_stream(stream);
    rsos_params best = *params;
    double best_us = -1.0;
    for (int wpt : wpts) {
        const int NWP = l.NW / wpt;
        if (NWP > 32) continue;
        const int lanes_per_tile_group = std::max(1, 32 / NWP);
        std::vector<int> tpls;
        if (params->tiles_per_lane) tpls = {params->tiles_per_lane};
        else {
            for (int item : {32, 64, 128}) {
                const int v = std::max(1, item / lanes_per_tile_group);
                if (std::find(tpls.begin(), tpls.end(), v) == tpls.end() && v <= 64) tpls.push_back(v);
            }
            // and the automatic choice for this word width
            const int v = persist_tiles_per_lane(params, NWP, wpt, l.rows, nT);
            if (std::find(tpls.begin(), tpls.end(), v) == tpls.end()) tpls.push_back(v);
        }
        for (int tpl : tpls)
            for (int lag : lags) {
                rsos_params c = *params;
                c.words_per_thread = wpt;
                c.tiles_per_lane = tpl;
                c.phase_lag = lag;
                c.series_capacity = 1;
                if (validate(&c) != RSOS_OK || !layout_of(&c).persist_on) continue;
                double us = 0.0;
                rc = time_geometry(c, sweeps, s, &us);
                if (rc) return rc;
                if (best_us < 0.0 || us < best_us) {
                    best_us = us;
                    best = c;
                }
            }
    }
    best.seed = params->seed;
    best.series_capacity = params->series_capacity;
    *tuned = best;
    if (us_per_sweep) *us_per_sweep = best_us;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = {best, best_us};
    return RSOS_OK;
}

// ---- Checkpoint / resume -----------------------------------------------
// A snapshot is a host byte string: a fixed header, the schedule and series
// times, then the device state (coded lattice or heights, h00, measured
// series rows).  With counter-based Philox that is the whole state of a job:
// a restored job continues bit-identically.
namespace {

constexpr char kSnapMagic[8] = {'R', 'S', 'O', 'S', 'S', 'N', 'P', '1'};

struct SnapHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    rsos_params params;
    int64_t t;
    int32_t moments;
    int32_t n_series;
    int32_t n_sched;
    int32_t sched_pos;
    uint64_t lattice_bytes;
    uint64_t h00_bytes;
    uint64_t series_bytes;
};

size_t pad8(size_t v) { return (v + 7) & ~(size_t)7; }

size_t lattice_bytes_of(const rsos_handle* h)
{
    const size_t L = (size_t)h->p.L;
    // multisurface: L rows of T nT records (a (+1) tiling pads each row)
    return h->plain ? L * L * 4 : (size_t)h->B * L * (size_t)h->J.T * (size_t)h->J.nT * h->NW * 4;
}

size_t snapshot_size(const rsos_handle* h)
{
    const size_t n = h->series_t.size();
    return sizeof(SnapHeader) + 8 * h->sched.size() + 8 * n + pad8(n) + pad8(lattice_bytes_of(h)) +
           (size_t)h->S_pad * 8 + n * (size_t)h->S_pad * kRecWords * 8;
}

}  // namespace

extern "C" int rsos_snapshot_bytes(const rsos_handle* h, size_t* bytes)
{
    if (!h || !bytes) return RSOS_EINVAL;
    *bytes = snapshot_size(h);
    return RSOS_OK;
}

extern "C" int rsos_snapshot(rsos_handle* h, void* host_buf, size_t bytes, void* stream)
{
    if (!h || !host_buf) return RSOS_EINVAL;
    if (h->sticky) return h->sticky;
    if (bytes < snapshot_size(h)) return RSOS_ENOMEM;
    cudaStream_t s = use_stream(h, stream);
    int rc = check_device_error(h, s);
    if (rc) return rc;
    unsigned char* out = static_cast<unsigned char*>(host_buf);
    SnapHeader hd{};
    std::memcpy(hd.magic, kSnapMagic, 8);
    hd.version = 1;
    hd.header_bytes = sizeof(SnapHeader);
    hd.params = h->p;
    hd.t = h->t;
    hd.moments = h->moments ? 1 : 0;
    hd.n_series = (int32_t)h->series_t.size();
    hd.n_sched = (int32_t)h->sched.size();
    hd.sched_pos = (int32_t)h->sched_pos;
    hd.lattice_bytes = lattice_bytes_of(h);
    hd.h00_bytes = (uint64_t)h->S_pad * 8;
    hd.series_bytes = (uint64_t)hd.n_series * h->S_pad * kRecWords * 8;
    size_t off = 0;
    std::memcpy(out, &hd, sizeof(hd));
    off += sizeof(hd);
    std::memcpy(out + off, h->sched.data(), 8 * h->sched.size());
    off += 8 * h->sched.size();
    std::memcpy(out + off, h->series_t.data(), 8 * h->series_t.size());
    off += 8 * h->series_t.size();
    std::memset(out + off, 0, pad8(h->series_mom.size()));
    if (!h->series_mom.empty()) std::memcpy(out + off, h->series_mom.data(), h->series_mom.size());
    off += pad8(h->series_mom.size());
    const void* lattice = h->plain ? (const void*)h->J.heights : (const void*)h->J.planes;
    cudaError_t e = cudaMemcpyAsync(out + off, lattice, hd.lattice_bytes, cudaMemcpyDeviceToHost, s);
    off += pad8(hd.lattice_bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out + off, h->J.h00, hd.h00_bytes, cudaMemcpyDeviceToHost, s);
    off += hd.h00_bytes;
    if (e == cudaSuccess && hd.series_bytes)
        e = cudaMemcpyAsync(out + off, h->rec, hd.series_bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    return RSOS_OK;
}

extern "C" int rsos_restore(const void* host_buf, size_t bytes, void* dev_buf, size_t dev_bytes, void* stream,
                            rsos_handle** out)
{
    if (!out) return RSOS_EINVAL;
    *out = nullptr;
    if (!host_buf || bytes < sizeof(SnapHeader)) return RSOS_EINVAL;
    const unsigned char* in = static_cast<const unsigned char*>(host_buf);
    SnapHeader hd;
    std::memcpy(&hd, in, sizeof(hd));
    if (std::memcmp(hd.magic, kSnapMagic, 8) != 0 || hd.version != 1 || hd.header_bytes != sizeof(SnapHeader))
        return RSOS_EINVAL;
    if (validate(&hd.params) != RSOS_OK || hd.t < 0 || hd.t > kMaxSweeps || hd.n_series < 0 || hd.n_sched < 0 ||
        hd.sched_pos < 0 || hd.sched_pos > hd.n_sched || (hd.moments != 0 && hd.moments != 1))
        return RSOS_EINVAL;
    const Layout l = layout_of(&hd.params);
    const size_t L = (size_t)hd.params.L;
    const size_t lattice = lattice_bytes(l, L);
    const size_t n = (size_t)hd.n_series;
    if (hd.lattice_bytes != lattice || hd.h00_bytes != (size_t)l.S_pad * 8 || (int)n > l.cap ||
        hd.series_bytes != n * l.S_pad * kRecWords * 8)
        return RSOS_EINVAL;
    const size_t need = sizeof(SnapHeader) + 8 * (size_t)hd.n_sched + 8 * n + pad8(n) + pad8(lattice) +
                        hd.h00_bytes + hd.series_bytes;
    if (bytes < need) return RSOS_EINVAL;
    rsos_handle* h = nullptr;
    int rc = rsos_init(&hd.params, dev_buf, dev_bytes, stream, &h);
    if (rc) return rc;
    size_t off = sizeof(SnapHeader);
    h->sched.assign(reinterpret_cast<const int64_t*>(in + off), reinterpret_cast<const int64_t*>(in + off) + hd.n_sched);
    off += 8 * (size_t)hd.n_sched;
    h->sched_pos = (size_t)hd.sched_pos;
    h->series_t.assign(reinterpret_cast<const int64_t*>(in + off), reinterpret_cast<const int64_t*>(in + off) + n);
    off += 8 * n;
    h->series_mom.assign(in + off, in + off + n);
    off += pad8(n);
    h->t = hd.t;
    h->moments = hd.moments != 0;
    cudaStream_t s = as_stream(stream);
    void* lat = h->plain ? (void*)h->J.heights : (void*)h->J.planes;
    cudaError_t e = cudaMemcpyAsync(lat, in + off, lattice, cudaMemcpyHostToDevice, s);
    off += pad8(lattice);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->J.h00, in + off, hd.h00_bytes, cudaMemcpyHostToDevice, s);
    off += hd.h00_bytes;
    if (e == cudaSuccess && hd.series_bytes)
        e = cudaMemcpyAsync(h->rec, in + off, hd.series_bytes, cudaMemcpyHostToDevice, s);
    // The persistent engine counts completed items per (phase, tile row) from
    // t = 0: a job resumed at t has completed t sweeps of every row.
    std::vector<unsigned long long> done;
    if (e == cudaSuccess && h->persist) {
        done.assign((size_t)4 * h->rows, (unsigned long long)hd.t * (unsigned long long)h->plan.K);
        e = cudaMemcpyAsync(h->done, done.data(), done.size() * 8, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        rsos_free(h);
        return RSOS_ECUDA;
    }
    *out = h;
    return RSOS_OK;
}
