// Batches of independent jobs (include/rsos.h, "Batches").  Every job keeps
// its own handle; rsos_batch_run queues each job's sweeps and scheduled
// measurements and records one event per job so that rsos_batch_poll can
// report completions without blocking.
#include <cuda_runtime.h>

#include <new>
#include <vector>

#include "../../include/rsos.h"

struct rsos_batch {
    std::vector<rsos_handle*> jobs;
    std::vector<int64_t> t_max;
    std::vector<std::vector<int64_t>> sched;
    std::vector<cudaEvent_t> done;
    std::vector<char> reported;
    bool queued;
    int status;
};

extern "C" {

int rsos_batch_create(const rsos_params* params, const int64_t* t_max, int32_t n_jobs, size_t hbm_budget,
                      rsos_batch** out)
{
    if (!out) return RSOS_EINVAL;
    *out = nullptr;
    if (!params || !t_max || n_jobs < 1) return RSOS_EINVAL;
    size_t total = 0;
    for (int32_t i = 0; i < n_jobs; ++i) {
        size_t b = 0;
        const int rc = rsos_required_bytes(&params[i], &b);
        if (rc) return rc;
        if (t_max[i] < 0 || t_max[i] > 0xFFFFFFFFll) return RSOS_EINVAL;
        total += b;
    }
    if (hbm_budget && total > hbm_budget) return RSOS_ENOMEM;
    rsos_batch* b = new (std::nothrow) rsos_batch();
    if (!b) return RSOS_ENOMEM;
    b->queued = false;
    b->status = RSOS_OK;
    for (int32_t i = 0; i < n_jobs; ++i) {
        rsos_handle* h = nullptr;
        const int rc = rsos_init(&params[i], nullptr, 0, nullptr, &h);
        if (rc) {
            rsos_batch_free(b);
            return rc;
        }
        b->jobs.push_back(h);
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
    if (!b || job < 0 || job >= (int32_t)b->jobs.size() || b->queued) return RSOS_EINVAL;
    if (n < 0 || (n > 0 && !times)) return RSOS_EINVAL;
    std::vector<int64_t> s(times, times + n);
    for (size_t k = 0; k < s.size(); ++k) {
        if (s[k] > b->t_max[job] || (k && s[k] <= s[k - 1])) return RSOS_EINVAL;
    }
    if (s.empty() || s.back() != b->t_max[job]) s.push_back(b->t_max[job]);
    b->sched[job] = s;
    return RSOS_OK;
}

int rsos_batch_run(rsos_batch* b, void* stream)
{
    if (!b) return RSOS_EINVAL;
    if (b->queued) return RSOS_EBUSY;
    for (size_t i = 0; i < b->jobs.size(); ++i) {
        int rc = rsos_schedule(b->jobs[i], b->sched[i].data(), (int32_t)b->sched[i].size());
        if (rc == RSOS_OK) rc = rsos_sweep(b->jobs[i], b->t_max[i], stream);
        if (rc) {
            b->status = rc;
            return rc;
        }
        if (cudaEventRecord(b->done[i], reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) {
            b->status = RSOS_ECUDA;
            return RSOS_ECUDA;
        }
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
    for (size_t i = 0; i < b->jobs.size(); ++i) {
        if (b->reported[i]) continue;
        const cudaError_t e = cudaEventQuery(b->done[i]);
        if (e == cudaSuccess) {
            if (*n_done < cap) {
                done_ids[(*n_done)++] = (int32_t)i;
                b->reported[i] = 1;
            } else {
                pending = true;
            }
        } else if (e == cudaErrorNotReady) {
            pending = true;
        } else {
            b->status = RSOS_ECUDA;
            return RSOS_ECUDA;
        }
    }
    return (*n_done == 0 && pending) ? RSOS_EBUSY : RSOS_OK;
}

int rsos_batch_job(rsos_batch* b, int32_t job, rsos_handle** out)
{
    if (!b || !out || job < 0 || job >= (int32_t)b->jobs.size()) return RSOS_EINVAL;
    *out = b->jobs[job];
    return RSOS_OK;
}

int rsos_batch_free(rsos_batch* b)
{
    if (!b) return RSOS_OK;
    int rc = RSOS_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) rc = RSOS_ECUDA;
    for (cudaEvent_t ev : b->done) cudaEventDestroy(ev);
    for (rsos_handle* h : b->jobs) {
        const int r = rsos_free(h);
        if (r) rc = r;
    }
    delete b;
    return rc;
}

}  // extern "C"
