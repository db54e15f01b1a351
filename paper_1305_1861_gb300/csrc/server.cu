// Served form: a request loop that admits counting jobs by device-memory footprint as they
// arrive and runs them concurrently (continuous batching).
//
// Each worker owns a context (its own memory pool, kept between jobs) and a stream. A job
// waits in FIFO order until a worker is idle AND its footprint estimate fits in what is left of
// the HBM budget; it then runs on that worker's stream, so jobs admitted while others are on
// the GPU overlap with them. A job whose estimate exceeds the whole budget is refused at submit
// time (TURTLE_E_BUSY). Results are exactly those of turtle_count on the same reads: nothing is
// shared between jobs except the device.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "turtle.h"
#include "host.h"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Ticket {
    turtle_job job{};
    uint64_t footprint = 0;
    bool done = false;
    int rc = 0;
    turtle_result res{};
    double t_submit = 0, t_start = 0, t_end = 0;
};

}  // namespace

struct turtle_server {
    int device = 0;
    uint64_t budget = 0, in_use = 0;
    turtle_params params{};
    std::vector<std::thread> workers;
    std::vector<turtle_ctx *> ctxs;
    std::vector<cudaStream_t> streams;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::unique_ptr<Ticket>> tickets;
    uint64_t next_id = 1;
    bool stop = false;
    turtle_server_stats stats{};
};

static void worker_loop(turtle_server *sv, int w) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        sv->cv_work.wait(lk, [&] {
            if (sv->stop) return true;
            if (sv->queue.empty()) return false;
            const Ticket *t = sv->tickets[sv->queue.front()].get();
            return sv->in_use + t->footprint <= sv->budget;  // admission by device-memory footprint
        });
        if (sv->stop) return;
        const uint64_t id = sv->queue.front();
        sv->queue.pop_front();
        Ticket *t = sv->tickets[id].get();
        sv->in_use += t->footprint;
        sv->stats.running++;
        if (sv->stats.running > sv->stats.peak_running) sv->stats.peak_running = sv->stats.running;
        if (sv->in_use > sv->stats.peak_admitted_bytes) sv->stats.peak_admitted_bytes = sv->in_use;
        t->t_start = now_ms();
        const turtle_job job = t->job;
        const bool more = !sv->queue.empty();
        lk.unlock();
        if (more) sv->cv_work.notify_one();  // the next job may fit beside this one
        turtle_reads r{job.bases, job.offsets, job.n_reads};
        turtle_result res{};
        const int rc = count_host_impl(sv->ctxs[w], &r, job.k, job.min_count, &sv->params, sv->streams[w], &res);
        lk.lock();
        t->res = res;
        t->rc = rc;
        t->t_end = now_ms();
        t->done = true;
        sv->in_use -= t->footprint;
        sv->stats.running--;
        sv->stats.completed++;
        if (rc) sv->stats.failed++;
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

extern "C" {

int turtle_server_create(int device, uint64_t hbm_budget_bytes, int max_concurrent, const turtle_params *params,
                         turtle_server **out) {
    if (!out || max_concurrent < 1 || max_concurrent > 64) return TURTLE_E_ARG;
    *out = nullptr;
    turtle_server *sv = new (std::nothrow) turtle_server();
    if (!sv) return TURTLE_E_NOMEM;
    sv->device = device;
    if (params) sv->params = *params;
    else turtle_params_default(&sv->params);
    if (sv->params.struct_size != sizeof(turtle_params)) turtle_params_default(&sv->params);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete sv;
        return TURTLE_E_NODEV;
    }
    if (!hbm_budget_bytes) {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        cudaGetLastError();
        hbm_budget_bytes = free_b / 2;
    }
    sv->budget = hbm_budget_bytes;
    sv->stats.budget_bytes = hbm_budget_bytes;
    for (int w = 0; w < max_concurrent; w++) {
        turtle_ctx *c = nullptr;
        int rc = turtle_ctx_create(device, &c);
        cudaStream_t st = nullptr;
        if (!rc && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = TURTLE_E_CUDA;
        if (rc) {
            if (c) turtle_ctx_destroy(c);
            cudaGetLastError();
            sv->stop = true;
            turtle_server_destroy(sv);
            return rc;
        }
        sv->ctxs.push_back(c);
        sv->streams.push_back(st);
    }
    for (int w = 0; w < max_concurrent; w++) sv->workers.emplace_back(worker_loop, sv, w);
    *out = sv;
    return TURTLE_OK;
}

int turtle_submit(turtle_server *sv, const turtle_job *job, uint64_t *ticket) {
    if (!sv || !job || !ticket || !job->offsets || (job->n_reads && !job->bases) || job->k < 1 || job->k > 64 ||
        job->min_count < 1)
        return TURTLE_E_ARG;
    *ticket = 0;
    const uint64_t n_bases = job->offsets[job->n_reads];
    const uint64_t fp = footprint_estimate(n_bases, job->n_reads, job->k, job->min_count, &sv->params);
    if (fp > sv->budget) return TURTLE_E_BUSY;  // could never be admitted
    auto t = std::make_unique<Ticket>();
    t->job = *job;
    t->footprint = fp;
    t->t_submit = now_ms();
    std::lock_guard<std::mutex> g(sv->mu);
    const uint64_t id = sv->next_id++;
    sv->tickets[id] = std::move(t);
    sv->queue.push_back(id);
    sv->stats.submitted++;
    if (sv->queue.size() > sv->stats.peak_queued) sv->stats.peak_queued = sv->queue.size();
    sv->cv_work.notify_one();
    *ticket = id;
    return TURTLE_OK;
}

int turtle_poll(turtle_server *sv, uint64_t ticket, int timeout_ms, turtle_result *out, turtle_job_times *times) {
    if (!sv || !out) return TURTLE_E_ARG;
    memset(out, 0, sizeof(*out));
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return TURTLE_E_ARG;
    Ticket *t = it->second.get();
    auto ready = [&] { return t->done; };
    if (timeout_ms < 0) sv->cv_done.wait(lk, ready);
    else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return TURTLE_E_TIMEOUT;
    const int rc = t->rc;
    *out = t->res;
    if (times) {
        times->queue_ms = t->t_start - t->t_submit;
        times->run_ms = t->t_end - t->t_start;
        times->total_ms = t->t_end - t->t_submit;
    }
    sv->tickets.erase(it);
    return rc;
}

int turtle_server_stats_get(turtle_server *sv, turtle_server_stats *st) {
    if (!sv || !st) return TURTLE_E_ARG;
    std::lock_guard<std::mutex> g(sv->mu);
    *st = sv->stats;
    st->queued = sv->queue.size();
    st->admitted_bytes = sv->in_use;
    return TURTLE_OK;
}

void turtle_server_destroy(turtle_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto &th : sv->workers) th.join();  // running jobs finish first
    for (auto &kv : sv->tickets) turtle_result_free(&kv.second->res);
    for (size_t w = 0; w < sv->ctxs.size(); w++) {
        turtle_ctx_destroy(sv->ctxs[w]);
        if (sv->streams[w]) cudaStreamDestroy(sv->streams[w]);
    }
    cudaGetLastError();
    delete sv;
}

}  // extern "C"
