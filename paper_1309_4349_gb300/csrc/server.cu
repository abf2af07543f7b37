// server.cu -- serving form: a job server with continuous batching.
//
// Jobs (a lattice, a number of Monte Carlo steps, an optional histogram cadence)
// are submitted from any host thread.  One worker thread owns the GPU work:
//  - admission: queued jobs are admitted in arrival order while their device
//    memory fits the server's budget and the device's free memory; an admitted
//    job's lattice is placed on the device and stays resident until it finishes;
//  - rounds: every round advances each resident job by a quantum of steps in one
//    resident-kernel launch per launch shape (groups run on concurrent streams);
//    the quantum is sized so that every job's share takes about the same time;
//  - after each round, jobs that reached their step count are retired (results
//    copied to the host, memory freed) and newly arrived jobs join the next round.
// A job's result depends only on its parameters (the random numbers are keyed by
// seed, sweep, phase and site), never on the other jobs in a round.
#include <string.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>

#include "klmc_host.h"

namespace {

using Clock = std::chrono::steady_clock;

klmc_status fail(klmc_status s, const std::string &msg)
{
    klmc::set_last_error(msg.c_str());
    return s;
}

struct Job {
    uint64_t id = 0;
    klmc_params p;
    int64_t n_mcs = 0, hist_every = 0;
    uint32_t flags = 0;
    klmc_ctx *ctx = nullptr;
    int64_t done = 0;
    size_t bytes = 0;
    int32_t status = KLMC_EBUSY;
    double submit_s = 0, start_s = 0, finish_s = 0;
    int64_t n_hist = 0;
    long long *dhist = nullptr;  // device: sizes[cap], counts[cap], n
    int64_t hist_cap = 0;
    std::vector<int64_t> hist_sizes, hist_counts;
    std::vector<uint8_t> lattice;
    long long final_state[klmc::kStateSlots];
};

}  // namespace

struct klmc_server {
    size_t budget = 0, used = 0, peak = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Clock::time_point t0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    bool stop = false;
    uint64_t next_id = 1;
    std::deque<Job *> pending;
    std::vector<Job *> active;
    std::map<uint64_t, Job *> jobs;
    int64_t finished = 0, rounds = 0;
    double busy_s = 0.0;
    long long attempts = 0;
    // worker-owned device tables and streams
    klmc::SweepJob *djobs = nullptr;
    klmc::SweepCall *dcalls = nullptr;
    int *dmap = nullptr;
    int capacity = 0;
    std::map<std::pair<int, int>, std::pair<cudaStream_t, cudaEvent_t>> group_streams;
    cudaEvent_t fork = nullptr, round_done = nullptr;
    void *cluster_mem = nullptr;
    long long cluster_sites = 0;
    klmc::ClusterScratch cs;
    int sm_count = 152;
    std::string worker_error;
};

namespace {

double seconds(const klmc_server *s) { return std::chrono::duration<double>(Clock::now() - s->t0).count(); }

// Steps per round: about 4 ms of work for every job at the launch shape it runs
// with this round.
constexpr int kHelicalStreams = 8;  // streams for the helical jobs of a round

int64_t quantum(const Job *j, std::pair<int, int> shape)
{
    const klmc_ctx *c = j->ctx;
    const double t_mcs_us = klmc::host::model_mcs_us(c->p.Lx, c->p.Ly, shape.first, shape.second);
    int64_t q = (int64_t)(4000.0 / t_mcs_us);
    if (q < 1) q = 1;
    int64_t left = j->n_mcs - j->done;
    if (q > left) q = left;
    if (j->hist_every > 0) {
        const int64_t to_hist = j->hist_every - j->done % j->hist_every;
        if (q > to_hist) q = to_hist;
    }
    return q;
}

klmc_status ensure_tables(klmc_server *s, int n)
{
    if (n <= s->capacity) return KLMC_OK;
    int cap = s->capacity ? s->capacity : 64;
    while (cap < n) cap *= 2;
    if (s->djobs) cudaFreeAsync(s->djobs, s->stream);
    if (s->dcalls) cudaFreeAsync(s->dcalls, s->stream);
    if (s->dmap) cudaFreeAsync(s->dmap, s->stream);
    s->djobs = nullptr;
    s->dcalls = nullptr;
    s->dmap = nullptr;
    if (cudaMallocAsync(&s->djobs, sizeof(klmc::SweepJob) * (size_t)cap, s->stream) != cudaSuccess ||
        cudaMallocAsync(&s->dcalls, sizeof(klmc::SweepCall) * (size_t)cap, s->stream) != cudaSuccess ||
        cudaMallocAsync(&s->dmap, sizeof(int) * (size_t)cap, s->stream) != cudaSuccess)
        return fail(KLMC_ENOMEM, "server tables");
    s->capacity = cap;
    return KLMC_OK;
}

klmc_status ensure_cluster_scratch(klmc_server *s, long long N)
{
    if (N <= s->cluster_sites) return KLMC_OK;
    if (s->cluster_mem) cudaFreeAsync(s->cluster_mem, s->stream);
    s->cluster_mem = nullptr;
    const size_t bytes = klmc::cluster_scratch_bytes(N, N);
    if (cudaMallocAsync(&s->cluster_mem, bytes, s->stream) != cudaSuccess)
        return fail(KLMC_ENOMEM, "server cluster scratch");
    klmc::cluster_scratch_carve(s->cluster_mem, N, N, &s->cs);
    if (klmc::cluster_scratch_clear(s->cs, s->stream) != cudaSuccess)
        return fail(KLMC_ECUDA, "server cluster scratch clear");
    s->cluster_sites = N;
    return KLMC_OK;
}

void retire(klmc_server *s, Job *j, int32_t status)
{
    j->status = status;
    j->finish_s = seconds(s);
    if (j->ctx) {
        klmc::host::destroy(j->ctx);
        j->ctx = nullptr;
    }
    if (j->dhist) {
        cudaFreeAsync(j->dhist, s->stream);
        j->dhist = nullptr;
    }
    s->used -= j->bytes;
    s->finished += 1;
}

// Admits queued jobs while memory allows; returns the number admitted.
int admit(klmc_server *s)
{
    int n = 0;
    while (true) {
        Job *j = nullptr;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (s->pending.empty()) break;
            j = s->pending.front();
        }
        klmc_params p = j->p;
        p.stream = s->stream;  // the job's own allocator (alloc and free), if any, serves its lattice
        if (!p.alloc || !p.free) {
            p.alloc = nullptr;
            p.free = nullptr;
        }
        size_t need = klmc::host::device_bytes(&p);
        if (j->hist_every > 0) need += (size_t)(2 * ((long long)std::sqrt(2.0 * p.Lx * p.Ly) + 2) + 1) * 8;
        if (need > s->budget) {  // can never be admitted: fail it instead of blocking the queue
            std::lock_guard<std::mutex> lock(s->mu);
            s->pending.pop_front();
            j->status = KLMC_EINVAL;
            j->start_s = j->finish_s = seconds(s);
            s->finished += 1;
            s->done_cv.notify_all();
            continue;
        }
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        if (s->used + need > s->budget || need + (64u << 20) > free_b) break;  // wait for memory
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->pending.pop_front();
        }
        klmc_status st = klmc::host::create_async(&j->ctx, &p);
        if (st == KLMC_OK && j->ctx->helical && j->ctx->cluster < 0)
            st = fail(KLMC_EINVAL, "helical lattice whose bands are too thin for the resident sweep: it runs "
                                   "one launch per iteration, on its own handle");
        else if (st == KLMC_OK && j->ctx->cluster < 0)
            st = fail(KLMC_EINVAL, "lattice too large for the resident sweep");
        if (st != KLMC_OK) {
            if (j->ctx) klmc::host::destroy(j->ctx);
            j->ctx = nullptr;
            std::lock_guard<std::mutex> lock(s->mu);
            j->status = st;
            j->start_s = j->finish_s = seconds(s);
            s->finished += 1;
            s->done_cv.notify_all();
            continue;
        }
        if (j->hist_every > 0) {
            j->hist_cap = (int64_t)std::sqrt(2.0 * p.Lx * p.Ly) + 2;
            if (cudaMallocAsync(&j->dhist, (size_t)(2 * j->hist_cap + 1) * 8, s->stream) != cudaSuccess) {
                klmc::host::destroy(j->ctx);
                j->ctx = nullptr;
                std::lock_guard<std::mutex> lock(s->mu);
                j->status = KLMC_ENOMEM;
                s->finished += 1;
                s->done_cv.notify_all();
                continue;
            }
        }
        std::lock_guard<std::mutex> lock(s->mu);
        j->bytes = need;
        s->used += need;
        if (s->used > s->peak) s->peak = s->used;
        j->start_s = seconds(s);
        s->active.push_back(j);
        ++n;
    }
    return n;
}

klmc_status run_round(klmc_server *s)
{
    const int n = (int)s->active.size();
    klmc_status st = ensure_tables(s, n);
    if (st != KLMC_OK) return st;
    std::vector<klmc::SweepJob> hjobs(n);
    std::vector<klmc::SweepCall> hcalls(n);
    std::vector<int64_t> q(n);
    std::map<std::pair<int, int>, std::vector<int>> groups;
    // Periodic jobs share launches by shape; helical jobs run the resident helical
    // sweep, one launch each.
    std::vector<klmc_ctx *> ctxs;
    std::vector<int64_t> remaining;
    std::vector<int> periodic, helical;
    for (int i = 0; i < n; ++i) {
        if (s->active[i]->ctx->helical) {
            helical.push_back(i);
            continue;
        }
        periodic.push_back(i);
        ctxs.push_back(s->active[i]->ctx);
        remaining.push_back(s->active[i]->n_mcs - s->active[i]->done);
    }
    std::vector<std::pair<int, int>> pshapes, shapes(n);
    klmc::host::choose_shapes(ctxs, remaining, s->sm_count, true, &pshapes);
    for (size_t k = 0; k < periodic.size(); ++k) shapes[periodic[k]] = pshapes[k];
    for (int i : helical) shapes[i] = {s->active[i]->ctx->cluster, 512};
    for (int i = 0; i < n; ++i) {
        Job *j = s->active[i];
        q[i] = quantum(j, shapes[i]);
        hjobs[i] = j->ctx->job;
        hcalls[i].sweep0 = j->ctx->sweep;
        hcalls[i].n_mcs = q[i];
        hcalls[i].trace = nullptr;
        hcalls[i].trace_every = 0;
        if (!j->ctx->helical) groups[shapes[i]].push_back(i);
    }
    std::vector<int> hmap;
    hmap.reserve(n);
    for (auto &g : groups) {
        std::stable_sort(g.second.begin(), g.second.end(),
                         [&](int a, int b) { return s->active[a]->ctx->N > s->active[b]->ctx->N; });
        hmap.insert(hmap.end(), g.second.begin(), g.second.end());
    }
    cudaError_t e = cudaMemcpyAsync(s->djobs, hjobs.data(), sizeof(klmc::SweepJob) * (size_t)n,
                                    cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->dcalls, hcalls.data(), sizeof(klmc::SweepCall) * (size_t)n,
                            cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = hmap.empty() ? cudaSuccess
                         : cudaMemcpyAsync(s->dmap, hmap.data(), sizeof(int) * hmap.size(), cudaMemcpyHostToDevice,
                                           s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->fork, s->stream);
    // Helical jobs on a pool of kHelicalStreams streams (keys (-1 - k, 512)).
    for (size_t k = 0; k < helical.size() && e == cudaSuccess; ++k) {
        const int i = helical[k];
        const std::pair<int, int> key(-1 - (int)(k % kHelicalStreams), 512);
        auto it = s->group_streams.find(key);
        if (it == s->group_streams.end()) {
            cudaStream_t gs;
            cudaEvent_t ge;
            e = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ge, cudaEventDisableTiming);
            if (e != cudaSuccess) break;
            it = s->group_streams.emplace(key, std::make_pair(gs, ge)).first;
        }
        e = cudaStreamWaitEvent(it->second.first, s->fork, 0);
        if (e == cudaSuccess)
            e = klmc::launch_helical_resident(hjobs[i], hcalls[i], shapes[i].first, it->second.first);
        if (e == cudaSuccess) e = cudaEventRecord(it->second.second, it->second.first);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, it->second.second, 0);
    }
    int offset = 0;
    for (auto &g : groups) {
        if (e != cudaSuccess) break;
        auto it = s->group_streams.find(g.first);
        if (it == s->group_streams.end()) {
            cudaStream_t gs;
            cudaEvent_t ge;
            e = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ge, cudaEventDisableTiming);
            if (e != cudaSuccess) break;
            it = s->group_streams.emplace(g.first, std::make_pair(gs, ge)).first;
        }
        size_t smem = 0;
        for (int i : g.second) {
            const size_t b = klmc::resident_smem_bytes(s->active[i]->ctx->p.Lx, s->active[i]->ctx->p.Ly,
                                                       g.first.first);
            if (b > smem) smem = b;
        }
        e = cudaStreamWaitEvent(it->second.first, s->fork, 0);
        if (e == cudaSuccess)
            e = klmc::launch_resident_sweep(s->djobs, s->dcalls, s->dmap + offset, (int)g.second.size(),
                                            g.first.first, g.first.second, smem, it->second.first);
        if (e == cudaSuccess) e = cudaEventRecord(it->second.second, it->second.first);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, it->second.second, 0);
        offset += (int)g.second.size();
    }
    // Histograms at the cadence, final copies of finishing jobs.
    std::vector<Job *> finishing;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        Job *j = s->active[i];
        j->done += q[i];
        j->ctx->sweep += q[i];
        const bool last = j->done >= j->n_mcs;
        if (j->hist_every > 0 && (j->done % j->hist_every == 0 || last)) {
            klmc_status hs = ensure_cluster_scratch(s, j->ctx->N);
            if (hs != KLMC_OK) return hs;
            e = klmc::launch_cluster_histogram(j->ctx->lat, j->ctx->job.packing, j->ctx->p.Lx,
                                               j->ctx->p.Ly, j->ctx->pitch, j->ctx->p.geometry, 1, s->cs,
                                               j->dhist, j->dhist + j->hist_cap, j->hist_cap,
                                               j->dhist + 2 * j->hist_cap, s->stream, j->ctx->helical);
            j->n_hist += 1;
        }
        if (last) finishing.push_back(j);
    }
    if (e == cudaSuccess) e = cudaEventRecord(s->round_done, s->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(s->round_done);
    if (e != cudaSuccess) return fail(KLMC_ECUDA, std::string("server round: ") + cudaGetErrorString(e));
    s->rounds += 1;
    for (Job *j : finishing) {
        e = cudaMemcpy(j->final_state, j->ctx->state, sizeof(j->final_state), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && j->dhist) {
            long long nd = 0;
            e = cudaMemcpy(&nd, j->dhist + 2 * j->hist_cap, sizeof(nd), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && nd > 0 && nd <= j->hist_cap) {
                j->hist_sizes.resize((size_t)nd);
                j->hist_counts.resize((size_t)nd);
                e = cudaMemcpy(j->hist_sizes.data(), j->dhist, (size_t)nd * 8, cudaMemcpyDeviceToHost);
                if (e == cudaSuccess)
                    e = cudaMemcpy(j->hist_counts.data(), j->dhist + j->hist_cap, (size_t)nd * 8,
                                   cudaMemcpyDeviceToHost);
            }
        }
        if (e == cudaSuccess && (j->flags & KLMC_JOB_KEEP_LATTICE)) {
            j->lattice.resize((size_t)j->ctx->N);
            klmc_status ls = klmc_get_lattice(j->ctx, j->lattice.data(), j->ctx->N);
            if (ls != KLMC_OK) e = cudaErrorUnknown;
        }
        std::lock_guard<std::mutex> lock(s->mu);
        s->attempts += j->final_state[klmc::kAttempts];
        retire(s, j, e == cudaSuccess ? KLMC_OK : KLMC_ECUDA);
        s->done_cv.notify_all();
    }
    if (!finishing.empty()) {
        std::lock_guard<std::mutex> lock(s->mu);
        std::vector<Job *> keep;
        for (Job *j : s->active)
            if (j->status == KLMC_EBUSY) keep.push_back(j);
        s->active.swap(keep);
    }
    return e == cudaSuccess ? KLMC_OK : fail(KLMC_ECUDA, "server retire");
}

void worker_main(klmc_server *s)
{
    while (true) {
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->stop && s->pending.empty() && s->active.empty()) break;
            if (s->pending.empty() && s->active.empty()) {
                s->cv.wait_for(lock, std::chrono::milliseconds(50));
                continue;
            }
        }
        admit(s);
        if (s->active.empty()) {
            // Nothing fits right now (memory); wait briefly for retirements or a stop.
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv.wait_for(lock, std::chrono::milliseconds(2));
            continue;
        }
        const double t = seconds(s);
        klmc_status st = run_round(s);
        s->busy_s += seconds(s) - t;
        if (st != KLMC_OK) {
            std::lock_guard<std::mutex> lock(s->mu);
            s->worker_error = klmc_last_error();
            for (Job *j : s->active) retire(s, j, st);
            s->active.clear();
            s->done_cv.notify_all();
        }
    }
}

}  // namespace

extern "C" {

klmc_status klmc_server_create(klmc_server **out, size_t device_mem_budget, void *stream)
{
    if (!out) return fail(KLMC_EINVAL, "out is NULL");
    if (device_mem_budget == 0) return fail(KLMC_EINVAL, "device_mem_budget must be > 0");
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return fail(KLMC_ENODEV, "no CUDA device");
    klmc_server *s = new (std::nothrow) klmc_server();
    if (!s) return fail(KLMC_ENOMEM, "host allocation failed");
    s->budget = device_mem_budget;
    s->t0 = Clock::now();
    s->stream = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!s->stream) {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        s->own_stream = true;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->round_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        delete s;
        return fail(KLMC_ECUDA, std::string("server create: ") + cudaGetErrorString(e));
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev);
    s->worker = std::thread(worker_main, s);
    *out = s;
    return KLMC_OK;
}

klmc_status klmc_server_submit(klmc_server *s, const klmc_params *p, int64_t n_mcs, int64_t hist_every,
                               uint32_t flags, uint64_t *job_id)
{
    if (!s || !p || !job_id) return fail(KLMC_EINVAL, "NULL argument");
    if (n_mcs < 1) return fail(KLMC_EINVAL, "n_mcs must be >= 1");
    if (hist_every < 0) return fail(KLMC_EINVAL, "hist_every must be >= 0");
    if (p->Lx < 4 || p->Ly < 4) return fail(KLMC_EINVAL, "Lx and Ly must be >= 4");
    Job *j = new (std::nothrow) Job();
    if (!j) return fail(KLMC_ENOMEM, "host allocation failed");
    j->p = *p;
    j->n_mcs = n_mcs;
    j->hist_every = hist_every;
    j->flags = flags;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) {
            delete j;
            return fail(KLMC_ESTATE, "server is stopping");
        }
        j->id = s->next_id++;
        j->submit_s = seconds(s);
        s->jobs[j->id] = j;
        s->pending.push_back(j);
    }
    s->cv.notify_all();
    *job_id = j->id;
    return KLMC_OK;
}

klmc_status klmc_server_poll(klmc_server *s, uint64_t job_id, klmc_job_result *out)
{
    if (!s || !out) return fail(KLMC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(KLMC_EINVAL, "unknown job id");
    const Job *j = it->second;
    if (j->status == KLMC_EBUSY) return KLMC_EBUSY;
    out->status = j->status;
    out->reserved = 0;
    out->n_mcs = j->done;
    out->n_unlike = j->final_state[klmc::kNUnlike];
    out->attempts = j->final_state[klmc::kAttempts];
    out->unlike = j->final_state[klmc::kUnlike];
    out->draws = j->final_state[klmc::kDraws];
    out->accepts = j->final_state[klmc::kAccepts];
    out->submit_s = j->submit_s;
    out->start_s = j->start_s;
    out->finish_s = j->finish_s;
    out->n_histograms = j->n_hist;
    return KLMC_OK;
}

klmc_status klmc_server_job_lattice(klmc_server *s, uint64_t job_id, uint8_t *host_out, int64_t n)
{
    if (!s || !host_out) return fail(KLMC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(KLMC_EINVAL, "unknown job id");
    const Job *j = it->second;
    if (j->status == KLMC_EBUSY) return KLMC_EBUSY;
    if (j->lattice.empty()) return fail(KLMC_ESTATE, "job was not submitted with KLMC_JOB_KEEP_LATTICE");
    if (n != (int64_t)j->lattice.size()) return fail(KLMC_EINVAL, "n must equal Lx*Ly");
    memcpy(host_out, j->lattice.data(), (size_t)n);
    return KLMC_OK;
}

klmc_status klmc_server_job_histogram(klmc_server *s, uint64_t job_id, int64_t *sizes, int64_t *counts,
                                      int64_t capacity, int64_t *n_distinct)
{
    if (!s || !n_distinct) return fail(KLMC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(KLMC_EINVAL, "unknown job id");
    const Job *j = it->second;
    if (j->status == KLMC_EBUSY) return KLMC_EBUSY;
    const int64_t n = (int64_t)j->hist_sizes.size();
    *n_distinct = n;
    if (n > capacity) return fail(KLMC_ETRUNC, "capacity too small");
    for (int64_t k = 0; k < n; ++k) {
        sizes[k] = j->hist_sizes[(size_t)k];
        counts[k] = j->hist_counts[(size_t)k];
    }
    return KLMC_OK;
}

klmc_status klmc_server_release(klmc_server *s, uint64_t job_id)
{
    if (!s) return fail(KLMC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(KLMC_EINVAL, "unknown job id");
    if (it->second->status == KLMC_EBUSY) return fail(KLMC_EBUSY, "job still pending");
    delete it->second;
    s->jobs.erase(it);
    return KLMC_OK;
}

klmc_status klmc_server_get_stats(klmc_server *s, klmc_server_stats *out)
{
    if (!s || !out) return fail(KLMC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    out->submitted = (int64_t)(s->next_id - 1);
    out->finished = s->finished;
    out->queued = (int64_t)s->pending.size();
    out->resident = (int64_t)s->active.size();
    out->rounds = s->rounds;
    out->attempts = s->attempts;
    out->busy_s = s->busy_s;
    out->uptime_s = seconds(s);
    out->device_bytes = (int64_t)s->used;
    out->peak_device_bytes = (int64_t)s->peak;
    return KLMC_OK;
}

klmc_status klmc_server_drain(klmc_server *s, double timeout_s)
{
    if (!s) return fail(KLMC_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lock(s->mu);
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (s->finished < (int64_t)(s->next_id - 1)) {
        if (s->done_cv.wait_until(lock, deadline) == std::cv_status::timeout &&
            s->finished < (int64_t)(s->next_id - 1))
            return fail(KLMC_ETIMEOUT, "jobs still running at the deadline");
    }
    return KLMC_OK;
}

klmc_status klmc_server_destroy(klmc_server *s)
{
    if (!s) return KLMC_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaStreamSynchronize(s->stream);
    for (auto &kv : s->jobs) delete kv.second;
    if (s->djobs) cudaFreeAsync(s->djobs, s->stream);
    if (s->dcalls) cudaFreeAsync(s->dcalls, s->stream);
    if (s->dmap) cudaFreeAsync(s->dmap, s->stream);
    if (s->cluster_mem) cudaFreeAsync(s->cluster_mem, s->stream);
    cudaStreamSynchronize(s->stream);
    for (auto &g : s->group_streams) {
        cudaStreamDestroy(g.second.first);
        cudaEventDestroy(g.second.second);
    }
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->round_done) cudaEventDestroy(s->round_done);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return KLMC_OK;
}

}  // extern "C"
