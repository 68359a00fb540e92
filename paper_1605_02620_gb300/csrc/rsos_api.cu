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
#include <new>
#include <vector>

#include "../../include/rsos.h"
#include "rsos_launch.h"

using rsos::JobDev;

struct rsos_handle {
    rsos_params p;
    bool plain;
    int SX, B, NW, NWT, S_pad;
    JobDev J;
    unsigned char* base;
    size_t bytes;
    bool owns;
    int32_t* row0;
    int64_t* partial;
    int ncb;
    int64_t* rec;  // [cap + 1][S_pad][4]; the last row is rsos_width's scratch
    int cap;
    std::vector<int64_t> series_t;
    int64_t t;
    std::vector<int64_t> sched;
    size_t sched_pos;
    int sticky;
    int cuda_err;
    size_t smem_budget;
    // persistent engine
    bool persist;
    rsos::PersistPlan plan;
    uint32_t* table;
    unsigned long long* done;
    unsigned long long* ticket;
    unsigned int* err;
    long long budget_ns;
    int64_t launches;  // kernels queued by this handle
};

namespace {

constexpr int64_t kMaxSweeps = 0xFFFFFFFFll;

// CUDA error of the last failed rsos_init on this thread (no handle exists).
thread_local int g_init_cuda_err = 0;

struct Layout {
    size_t planes, h00, row0, partial, rec, persist, total;
    int ncb, S_pad, B, NW, T, cap;
    int CW, K;  // persistent engine: tiles per block, chunks per tile row
    bool plain, persist_on;
};

// Tiles per lane and work item of the persistent engine (execution geometry
// only; RSOS_TILES_PER_LANE overrides the default of 2, the fastest measured
// for L = 4096, N = 1, 64 surfaces on GB300).
int persist_tiles_per_lane()
{
    if (const char* env = std::getenv("RSOS_TILES_PER_LANE")) {
        const int v = std::atoi(env);
        if (v >= 1 && v <= 64) return v;
    }
    return 2;
}

// Tiles per work item: one warp's 32 lanes over the lane-word groups of a
// tile, times the tiles per lane.
int persist_block_tiles(int NWP)
{
    const int cw = 32 / NWP;
    return (cw < 1 ? 1 : cw) * persist_tiles_per_lane();
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// 32-lane words per thread: 2 when the job has an even number of words
// (uint64 registers), else 1.  RSOS_WORDS_PER_THREAD=1 forces one word per
// thread (execution geometry only; results are identical).
int words_per_thread(int NW)
{
    if (const char* env = std::getenv("RSOS_WORDS_PER_THREAD"))
        if (std::atoi(env) == 1) return 1;
    return (NW % 2 == 0) ? 2 : 1;
}

int validate(const rsos_params* p)
{
    if (!p) return RSOS_EINVAL;
    const int T = p->tile_x == 0 ? 8 : p->tile_x;
    const int Ty = p->tile_y == 0 ? 8 : p->tile_y;
    if (T != Ty) return RSOS_EINVAL;
    if (T != 2 && T != 4 && T != 8 && T != 16) return RSOS_EINVAL;
    if (p->L < T || p->L > 65536 || p->L % T != 0) return RSOS_EINVAL;
    if (p->N < 1 || p->N > 7) return RSOS_EINVAL;
    if (p->surfaces < 1 || p->surfaces > (1 << 20)) return RSOS_EINVAL;
    if (p->phase_order != 0 && p->phase_order != 1) return RSOS_EINVAL;
    if (p->series_capacity < 0 || p->series_capacity > (1 << 24)) return RSOS_EINVAL;
    if (p->engine < 0 || p->engine > 2) return RSOS_EINVAL;
    if (p->engine == 2 && p->surfaces == 1) return RSOS_EINVAL;  // plain path: phase engine only
    if (p->engine == 2) {
        const int NW = (p->surfaces + 31) / 32, NWT = words_per_thread(NW);
        if (NW / NWT > 32) return RSOS_EINVAL;
    }
    return RSOS_OK;
}

Layout layout_of(const rsos_params* p)
{
    Layout l;
    l.T = p->tile_x == 0 ? 8 : p->tile_x;
    l.plain = p->surfaces == 1;
    l.B = rsos::bits_for_step(p->N);
    l.NW = (p->surfaces + 31) / 32;
    l.S_pad = l.plain ? 1 : l.NW * 32;
    l.cap = p->series_capacity == 0 ? 1024 : p->series_capacity;
    const size_t L = (size_t)p->L;
    JobDev J{};
    J.L = p->L;
    J.T = l.T;
    J.nT = p->L / l.T;
    J.NW = l.NW;
    l.ncb = rsos::measure_blocks(J, l.plain);
    l.planes = align256(l.plain ? L * L * 4 : (size_t)l.B * L * L * l.NW * 4);
    l.h00 = align256((size_t)l.S_pad * 8);
    l.row0 = l.plain ? 0 : align256((size_t)l.S_pad * L * 4);
    l.partial = align256((size_t)l.ncb * l.S_pad * 2 * 8);
    l.rec = align256((size_t)(l.cap + 1) * l.S_pad * 4 * 8);
    const int nT = p->L / l.T;
    // Auto engine: the persistent dataflow engine for multisurface jobs with
    // at least 8 tile rows, one launch per phase otherwise.
    l.persist_on = !l.plain && (p->engine == 2 || (p->engine == 0 && nT >= 8));
    if (l.persist_on && p->engine == 0) {
        // more lane-word groups than lanes of a warp: phase engine
        const int NWT = words_per_thread(l.NW);
        if (l.NW / NWT > 32) l.persist_on = false;
    }
    l.CW = l.K = 0;
    l.persist = 0;
    if (l.persist_on) {
        const int NWT = words_per_thread(l.NW);
        const int SX = l.T / 2;
        (void)SX;
        l.CW = persist_block_tiles(l.NW / NWT);
        l.K = (nT + l.CW - 1) / l.CW;
        l.persist = align256((size_t)4 * nT * 8) + align256((size_t)4 * nT * l.K * 4) + 256;
    }
    l.total = l.planes + l.h00 + l.row0 + l.partial + l.rec + l.persist;
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

int measure_into(rsos_handle* h, int row, cudaStream_t s)
{
    h->launches += h->plain ? 2 : 3;
    return fail_cuda(h, rsos::launch_measure(h->J, h->plain, h->S_pad, h->row0, h->partial, h->ncb,
                                             h->rec + (size_t)row * h->S_pad * 4, s));
}

int measure_due(rsos_handle* h, cudaStream_t s)
{
    while (h->sched_pos < h->sched.size() && h->sched[h->sched_pos] <= h->t) {
        if (h->sched[h->sched_pos] == h->t) {
            if ((int)h->series_t.size() >= h->cap) return RSOS_ERANGE;
            const int rc = measure_into(h, (int)h->series_t.size(), s);
            if (rc) return rc;
            h->series_t.push_back(h->t);
        }
        ++h->sched_pos;
    }
    return RSOS_OK;
}

int run_sweep(rsos_handle* h, cudaStream_t s)
{
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
    A.table = h->table;
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

int run_persist_segment(rsos_handle* h, int64_t n, cudaStream_t s)
{
    // Tickets of one launch stay below 2^31: split very long segments.
    const int64_t per_sweep = 4ll * h->J.nT * h->plan.K;
    const int64_t max_sweeps = std::max<int64_t>(1, ((int64_t)1 << 31) / per_sweep);
    while (n > 0) {
        const int64_t m = std::min(n, max_sweeps);
        cudaError_t e = rsos::launch_zero(h->ticket, 8, s);
        if (e == cudaSuccess)
            e = rsos::launch_persist(h->J, h->SX, h->NWT, persist_args(h, (uint32_t)h->t, m), h->plan, s);
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
        const int64_t* r = rec_row + (size_t)j * 4;
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
    switch (SX) {
        case 1: return launch_persist_s1(J, words_per_thread, A, P, s);
        case 2: return launch_persist_s2(J, words_per_thread, A, P, s);
        case 4: return launch_persist_s4(J, words_per_thread, A, P, s);
        case 8: return launch_persist_s8(J, words_per_thread, A, P, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t plan_persist(const JobDev& J, int SX, int words_per_thread, int block_tiles, PersistPlan* out)
{
    switch (SX) {
        case 1: return plan_persist_s1(J, words_per_thread, block_tiles, out);
        case 2: return plan_persist_s2(J, words_per_thread, block_tiles, out);
        case 4: return plan_persist_s4(J, words_per_thread, block_tiles, out);
        case 8: return plan_persist_s8(J, words_per_thread, block_tiles, out);
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
    h->p.tile_x = h->p.tile_y = l.T;
    h->plain = l.plain;
    h->SX = l.T / 2;
    h->B = l.B;
    h->NW = l.NW;
    h->NWT = words_per_thread(l.NW);
    h->S_pad = l.S_pad;
    h->cap = l.cap;
    h->ncb = l.ncb;
    h->t = 0;
    h->sched_pos = 0;
    h->sticky = RSOS_OK;
    h->cuda_err = 0;
    h->launches = l.persist_on ? 3 : 1;
    h->smem_budget = 113 * 1024;
    if (const char* env = std::getenv("RSOS_SMEM_BUDGET")) {
        const long v = std::atol(env);
        if (v >= 4096 && v <= 232448) h->smem_budget = (size_t)v;
    }
    h->bytes = l.total;
    if (dev_buf) {
        h->base = static_cast<unsigned char*>(dev_buf);
        h->owns = false;
    } else {
        void* p = nullptr;
        const cudaError_t e = cudaMalloc(&p, l.total);
        if (e != cudaSuccess) {
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
    h->table = nullptr;
    h->done = nullptr;
    h->ticket = nullptr;
    h->err = nullptr;
    h->budget_ns = 1000000000ll;
    if (l.persist_on) {
        const int nT = params->L / l.T;
        h->done = reinterpret_cast<unsigned long long*>(cur);
        cur += align256((size_t)4 * nT * 8);
        h->table = reinterpret_cast<uint32_t*>(cur);
        cur += align256((size_t)4 * nT * l.K * 4);
        h->ticket = reinterpret_cast<unsigned long long*>(cur);
        h->err = reinterpret_cast<unsigned int*>(cur + 8);
    }
    J.L = params->L;
    J.T = l.T;
    J.nT = params->L / l.T;
    J.NW = l.NW;
    J.NWP = l.NW / h->NWT;
    J.N = params->N;
    J.B = l.B;
    J.phase_order = params->phase_order;
    J.seed_lo = (uint32_t)params->seed;
    J.seed_hi = (uint32_t)(params->seed >> 32);
    J.rk = rsos::philox_round_keys(J.seed_lo, J.seed_hi);
    cudaError_t e = cudaSuccess;
    if (l.persist_on) {
        e = rsos::plan_persist(J, h->SX, h->NWT, l.CW, &h->plan);
        if (e == cudaSuccess && (h->plan.CW != l.CW || h->plan.K != l.K)) e = cudaErrorInvalidConfiguration;
        if (e == cudaSuccess) {
            std::vector<uint32_t> table((size_t)4 * J.nT * l.K);
            rsos::build_order_table(J.nT, l.K, h->plan.D, table.data());
            e = cudaMemcpyAsync(h->table, table.data(), table.size() * 4, cudaMemcpyHostToDevice, as_stream(stream));
            if (e == cudaSuccess) e = cudaStreamSynchronize(as_stream(stream));
        }
        if (e == cudaSuccess) e = rsos::launch_zero(h->done, (size_t)4 * J.nT * 8, as_stream(stream));
        if (e == cudaSuccess) e = rsos::launch_zero(h->ticket, 16, as_stream(stream));
    }
    // Flat initial condition (section II): planes and h00 zero.
    if (e == cudaSuccess) e = rsos::launch_zero(h->base, l.planes + l.h00, as_stream(stream));
    if (e != cudaSuccess) {
        g_init_cuda_err = (int)e;
        (void)cudaGetLastError();
        if (h->owns) cudaFree(h->base);
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
    cudaStream_t s = as_stream(stream);
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

int rsos_selftest_timeout(rsos_handle* h, int64_t budget_ns, void* stream)
{
    if (!h || budget_ns <= 0) return RSOS_EINVAL;
    if (!h->persist) return RSOS_EINVAL;
    if (h->sticky) return h->sticky;
    cudaStream_t s = as_stream(stream);
    // Sweep t + 2 depends on sweep t + 1, which never runs: every wait of
    // this launch expires after budget_ns.
    const long long saved = h->budget_ns;
    h->budget_ns = budget_ns;
    rsos::PersistArgs A = persist_args(h, (uint32_t)(h->t + 2), 1);
    h->budget_ns = saved;
    cudaError_t e = rsos::launch_zero(h->ticket, 8, s);
    if (e == cudaSuccess) e = rsos::launch_persist(h->J, h->SX, h->NWT, A, h->plan, s);
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
    cudaStream_t s = as_stream(stream);
    int rc = check_device_error(h, s);
    if (rc) return rc;
    rc = measure_into(h, h->cap, s);
    if (rc) return rc;
    std::vector<int64_t> host((size_t)h->S_pad * 4);
    cudaError_t e = cudaMemcpyAsync(host.data(), h->rec + (size_t)h->cap * h->S_pad * 4, host.size() * 8,
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
    cudaStream_t s = as_stream(stream);
    const int rc = check_device_error(h, s);
    if (rc) return rc;
    const int n = std::min<int>(cap, (int)h->series_t.size());
    *n_out = n;
    if (n == 0) return RSOS_OK;
    std::vector<int64_t> host((size_t)n * h->S_pad * 4);
    cudaError_t e = cudaMemcpyAsync(host.data(), h->rec, host.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(h, e);
    bool overflow = false;
    const int S = h->p.surfaces;
    for (int m = 0; m < n; ++m) {
        if (times) times[m] = h->series_t[m];
        convert_row(h, host.data() + (size_t)m * h->S_pad * 4, sum_h ? sum_h + (size_t)m * S : nullptr,
                    sum_h2 ? sum_h2 + (size_t)m * S : nullptr, w2 ? w2 + (size_t)m * S : nullptr, &overflow);
    }
    return overflow ? RSOS_EOVERFLOW : RSOS_OK;
}

int rsos_heights(rsos_handle* h, int32_t surface, int64_t* host_LxL, void* stream)
{
    if (!h || !host_LxL || surface < 0 || surface >= h->p.surfaces) return RSOS_EINVAL;
    if (h->sticky) return h->sticky;
    cudaStream_t s = as_stream(stream);
    const int rc = check_device_error(h, s);
    if (rc) return rc;
    const size_t n = (size_t)h->p.L * h->p.L;
    int64_t* dev = nullptr;
    cudaError_t e = cudaMalloc(&dev, n * 8);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return RSOS_ENOMEM;
    }
    e = rsos::launch_heights(h->J, h->plain, surface, h->row0, dev, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_LxL, dev, n * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dev);
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
    if (h->owns) {
        if (cudaDeviceSynchronize() != cudaSuccess) rc = RSOS_ECUDA;
        if (cudaFree(h->base) != cudaSuccess) rc = RSOS_ECUDA;
    }
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
