// Served form: a request loop that admits counting jobs by device-memory footprint as they
// arrive and runs them with continuous batching.
//
// Several executor threads (default 2) share one queue and one HBM budget; each owns a context
// (device scratch) and a stream, so the batches they run overlap on the device. Whenever an
// executor is free it takes the oldest queued job whose footprint estimate fits what is left of
// the budget, plus every other queued job with the same k and min_count that still fits (up to
// max_batch jobs, and as many as the spare key bits can tag), and runs them as one batched
// pipeline: each stage is one launch for all of them. With params.batch_mixed (1, or 0 when the
// batched form's cost model expects it to pay) queued jobs of other k (at most 61) and the same
// min_count join the run as a mixed run. A run's results are split and copied to
// the host by the executor's copy-out thread while its next run executes. A job whose estimate
// exceeds the whole budget is refused at submit time (TURTLE_E_BUSY). Results are exactly those
// of turtle_count on the same reads.
#include <algorithm>
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

// One executor: a context, a stream and a copy-out thread of its own.
struct Executor {
    turtle_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::unique_ptr<BatchOutput> out;
    std::thread thread;
};

struct turtle_server {
    int device = 0;
    int max_batch = 1;
    uint64_t budget = 0, in_use = 0;
    turtle_params params{};
    std::vector<std::unique_ptr<Executor>> execs;
    uint64_t running_batches = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::unique_ptr<Ticket>> tickets;
    uint64_t next_id = 1;
    bool stop = false;
    turtle_server_stats stats{};
};

// A run has finished (or failed): hand each job its result, release its footprint.
static void finish(turtle_server *sv, const std::vector<uint64_t> &ids, const std::vector<uint64_t> &fps,
                   turtle_result *outs, int rc) {
    std::lock_guard<std::mutex> g(sv->mu);
    const double t = now_ms();
    for (size_t i = 0; i < ids.size(); i++) {
        Ticket *tk = sv->tickets[ids[i]].get();
        if (rc == TURTLE_OK) {
            tk->res = outs[i];
        } else {
            turtle_result_free(&outs[i]);
            memset(&tk->res, 0, sizeof(tk->res));
        }
        tk->rc = rc;
        tk->t_end = t;
        tk->done = true;
        sv->in_use -= fps[i];
        sv->stats.running--;
        sv->stats.completed++;
        if (rc) sv->stats.failed++;
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
}

static void executor_loop(turtle_server *sv, Executor *ex) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        sv->cv_work.wait(lk, [&] {
            if (sv->stop) return true;
            if (sv->queue.empty()) return false;
            return sv->in_use + sv->tickets[sv->queue.front()]->footprint <= sv->budget;  // admission
        });
        if (sv->stop) return;
        // continuous batching: the oldest job and the queued jobs that can share its pipeline (the same
        // k and min_count; in a mixed run any k <= MIXED_K_MAX with the same min_count)
        const turtle_job head = sv->tickets[sv->queue.front()]->job;
        auto pick = [&](bool mixed, size_t cap, std::vector<uint64_t> &ids, std::vector<uint64_t> &fps) {
            uint64_t room = sv->budget - sv->in_use;
            for (uint64_t id : sv->queue) {
                if (ids.size() >= cap) break;
                const Ticket *t = sv->tickets[id].get();
                const bool joins = mixed ? t->job.k <= MIXED_K_MAX && t->job.min_count == head.min_count
                                         : t->job.k == head.k && t->job.min_count == head.min_count;
                if ((ids.empty() || joins) && t->footprint <= room) {
                    room -= t->footprint;
                    ids.push_back(id);
                    fps.push_back(t->footprint);
                }
            }
        };
        std::vector<uint64_t> ids, fps;
        bool mixed = false;
        if (sv->params.batch_mixed != 2 && sv->params.compact == 0 && head.k <= MIXED_K_MAX) {
            pick(true, std::min<size_t>((size_t)sv->max_batch, 64), ids, fps);
            std::vector<turtle_job> js;
            std::vector<size_t> idx;
            bool several_k = false;
            for (uint64_t id : ids) {
                js.push_back(sv->tickets[id]->job);
                idx.push_back(idx.size());
                several_k |= js.back().k != head.k;
            }
            mixed = several_k && (sv->params.batch_mixed == 1 || mixed_runs_pay(js.data(), idx));
            if (!mixed) ids.clear(), fps.clear();
        }
        if (!mixed) pick(false, std::min<size_t>((size_t)sv->max_batch, batch_capacity(head.k)), ids, fps);
        for (uint64_t id : ids) sv->queue.erase(std::find(sv->queue.begin(), sv->queue.end(), id));
        const double t0 = now_ms();
        std::vector<turtle_job> jobs(ids.size());
        for (size_t i = 0; i < ids.size(); i++) {
            Ticket *t = sv->tickets[ids[i]].get();
            t->t_start = t0;
            jobs[i] = t->job;
            sv->in_use += fps[i];
        }
        sv->stats.running += ids.size();
        sv->stats.batches++;
        sv->running_batches++;
        if (sv->running_batches > sv->stats.peak_running_batches) sv->stats.peak_running_batches = sv->running_batches;
        if (ids.size() > sv->stats.largest_batch) sv->stats.largest_batch = ids.size();
        if (sv->stats.running > sv->stats.peak_running) sv->stats.peak_running = sv->stats.running;
        if (sv->in_use > sv->stats.peak_admitted_bytes) sv->stats.peak_admitted_bytes = sv->in_use;
        lk.unlock();
        std::shared_ptr<std::vector<turtle_result>> outs = std::make_shared<std::vector<turtle_result>>(ids.size());
        std::vector<size_t> idx(ids.size());
        for (size_t i = 0; i < idx.size(); i++) idx[i] = i;
        const int rc = batch_run_jobs(ex->ctx, jobs.data(), idx, &sv->params, ex->stream, outs->data(), *ex->out,
                                      [sv, ids, fps, outs](int r) { finish(sv, ids, fps, outs->data(), r); }, mixed);
        if (rc) finish(sv, ids, fps, outs->data(), rc);  // nothing was posted
        lk.lock();
        sv->running_batches--;  // this run's device work is done (its copy-out may still be running)
    }
}

extern "C" {

int turtle_server_create(int device, uint64_t hbm_budget_bytes, int max_batch, const turtle_params *params,
                         turtle_server **out) {
    return turtle_server_create_ex(device, hbm_budget_bytes, max_batch, 2, params, out);
}

int turtle_server_create_ex(int device, uint64_t hbm_budget_bytes, int max_batch, int executors,
                            const turtle_params *params, turtle_server **out) {
    if (!out || max_batch < 1 || max_batch > 64 || executors < 1 || executors > 16) return TURTLE_E_ARG;
    *out = nullptr;
    turtle_server *sv = new (std::nothrow) turtle_server();
    if (!sv) return TURTLE_E_NOMEM;
    sv->device = device;
    sv->max_batch = max_batch;
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
    sv->stats.executors = (uint64_t)executors;
    int rc = TURTLE_OK;
    for (int e = 0; e < executors && rc == TURTLE_OK; e++) {
        std::unique_ptr<Executor> ex(new (std::nothrow) Executor());
        if (!ex) {
            rc = TURTLE_E_NOMEM;
            break;
        }
        rc = turtle_ctx_create(device, &ex->ctx);
        if (!rc && cudaStreamCreateWithFlags(&ex->stream, cudaStreamNonBlocking) != cudaSuccess) rc = TURTLE_E_CUDA;
        if (!rc) {
            ex->out.reset(new (std::nothrow) BatchOutput());
            if (!ex->out || !ex->out->ok()) rc = TURTLE_E_CUDA;
        }
        sv->execs.push_back(std::move(ex));
    }
    if (rc) {
        cudaGetLastError();
        turtle_server_destroy(sv);
        return rc;
    }
    for (auto &ex : sv->execs) ex->thread = std::thread(executor_loop, sv, ex.get());
    *out = sv;
    return TURTLE_OK;
}

int turtle_submit(turtle_server *sv, const turtle_job *job, uint64_t *ticket) {
    if (!sv || !job || !ticket || !job->offsets || (job->n_reads && !job->bases) || job->k < 1 || job->k > 64 ||
        job->min_count < 1 || job->offsets[job->n_reads] < job->offsets[0])
        return TURTLE_E_ARG;
    *ticket = 0;
    const uint64_t n_bases = job->offsets[job->n_reads] - job->offsets[0];
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
        times->start_ms = t->t_start;
        times->end_ms = t->t_end;
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
    for (auto &ex : sv->execs)
        if (ex->thread.joinable()) ex->thread.join();  // running batches finish first
    for (auto &ex : sv->execs) {
        if (ex->out) ex->out->drain();  // and their copy-out
        ex->out.reset();
    }
    for (auto &kv : sv->tickets) turtle_result_free(&kv.second->res);
    for (auto &ex : sv->execs) {
        if (ex->ctx) turtle_ctx_destroy(ex->ctx);
        if (ex->stream) cudaStreamDestroy(ex->stream);
    }
    sv->execs.clear();
    cudaGetLastError();
    delete sv;
}

}  // extern "C"
