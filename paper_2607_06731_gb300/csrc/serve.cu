// Serving loop: many concurrent evolutionary runs submit one generation (a population to
// score against their resident dataset) at a time; requests are admitted by device-memory
// budget and packed into shared persistent launches (continuous batching).
//
// The paper sends a generation's genomes to the GPU once and returns one fitness per genome
// (Section 2.4) and batches populations so that device memory is never exceeded (Section
// 2.2); it reuses the memory of dead individuals instead of freeing it (Section 2.7). Here:
//   submit    copies the request's host arrays into pinned staging taken from a size-class
//             pool (buffers are recycled, never freed while the server lives) and queues it;
//   dispatch  one host thread admits queued requests in arrival order while their device
//             bytes fit the budget and a stream is free, packs all admitted requests into one
//             launch (one job per request; up to 64 jobs per persistent kernel), enqueues the
//             copies in, the scoring and the copies out on that stream and records an event;
//             requests arriving meanwhile go into the next launch on another stream, whose
//             copies and planning overlap the running one;
//   complete  the same thread polls the events, marks requests done with their latency and
//             returns their bytes to the budget.
// Every program's fitness is computed on its own with fixed-order sums and a fixed tile, so a
// request's results are the same bits alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.h"
#include "registry.h"

namespace beagle {
namespace {

using Clock = std::chrono::steady_clock;

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Pinned host buffers by power-of-two size class, recycled instead of freed.
class PinnedPool {
  public:
    ~PinnedPool() {
        for (auto &kv : free_)
            for (void *p : kv.second) cudaFreeHost(p);
    }
    void *get(size_t n, size_t *cls) {
        size_t c = 4096;
        while (c < n) c <<= 1;
        *cls = c;
        {
            std::lock_guard<std::mutex> lk(mu_);
            auto &v = free_[c];
            if (!v.empty()) {
                void *p = v.back();
                v.pop_back();
                return p;
            }
        }
        void *p = nullptr;
        if (cudaHostAlloc(&p, c, cudaHostAllocDefault) != cudaSuccess) return nullptr;
        return p;
    }
    void put(void *p, size_t cls) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu_);
        free_[cls].push_back(p);
    }

  private:
    std::mutex mu_;
    std::map<size_t, std::vector<void *>> free_;
};

struct Request {
    uint64_t ticket = 0;
    int32_t dataset = 0;
    int64_t P = 0, T = 0;        // programs, tokens
    int64_t N = 0;               // cases of the dataset
    void *host_in = nullptr;     // pinned: ops | consts | offsets | lengths
    size_t in_cls = 0, in_bytes = 0;
    size_t off_consts = 0, off_offs = 0, off_lens = 0;
    beagle_fitness *host_out = nullptr;   // pinned, P records
    size_t out_cls = 0;
    size_t dev_bytes = 0;        // admission charge: inputs + outputs + scoring scratch
    Clock::time_point t_submit, t_done;
    beagle_status status = BEAGLE_OK;
    std::string message;         // failure message, reported to the collecting thread
    bool done = false;
};

struct Batch {
    std::vector<std::shared_ptr<Request>> reqs;
    cudaStream_t stream = nullptr;
    cudaEvent_t event = nullptr;
    size_t bytes = 0;
    int slot = 0;
};

}  // namespace
}  // namespace beagle

using namespace beagle;

struct beagle_server {
    beagle_serve_config cfg;
    int device = 0;
    PinnedPool pinned;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<bool> slot_busy;
    std::vector<Batch> inflight;
    uint64_t next_ticket = 1;
    size_t bytes_in_use = 0, peak_bytes = 0;
    int64_t submitted = 0, completed = 0, rejected = 0, launches = 0;
    int64_t node_evals = 0;
    std::vector<double> latencies_us;
    Clock::time_point t_first, t_last;
    bool have_first = false;
    bool stop = false;
    std::thread worker;
    beagle_status fatal = BEAGLE_OK;
};

namespace beagle {
namespace {

void finish_request(beagle_server *s, const std::shared_ptr<Request> &r, beagle_status st) {
    r->status = st;
    if (st != BEAGLE_OK) r->message = beagle_last_error();
    r->done = true;
    r->t_done = Clock::now();
    s->pinned.put(r->host_in, r->in_cls);
    r->host_in = nullptr;
    if (st == BEAGLE_OK) {
        ++s->completed;
        s->node_evals += r->T * r->N;
        s->latencies_us.push_back(
            std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count());
        s->t_last = r->t_done;
    }
    hold_dataset(r->dataset, -1);
}

// Enqueue one batch on a free stream slot. Called with s->mu held.
beagle_status launch_batch(beagle_server *s, std::vector<std::shared_ptr<Request>> &reqs,
                           int slot) {
    Batch b;
    b.reqs = reqs;
    b.slot = slot;
    b.stream = s->streams[slot];
    b.event = s->events[slot];
    size_t total = 0;
    for (auto &r : reqs) total += up256(r->in_bytes) + up256(sizeof(beagle_fitness) * r->P);
    char *base = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&base), total, b.stream);
    if (e != cudaSuccess) return cuda_fail(e, "serve: device buffers");
    std::vector<JobRequest> jobs;
    char *cur = base;
    for (auto &r : reqs) {
        char *in = cur;
        cur += up256(r->in_bytes);
        beagle_fitness *out = reinterpret_cast<beagle_fitness *>(cur);
        cur += up256(sizeof(beagle_fitness) * r->P);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(in, r->host_in, r->in_bytes, cudaMemcpyHostToDevice, b.stream);
        jobs.push_back(JobRequest{reinterpret_cast<const uint8_t *>(in),
                                  reinterpret_cast<const int64_t *>(in + r->off_offs),
                                  reinterpret_cast<const int32_t *>(in + r->off_lens),
                                  reinterpret_cast<const float *>(in + r->off_consts), r->P,
                                  r->dataset, out, nullptr, nullptr});
    }
    beagle_status st = e == cudaSuccess ? BEAGLE_OK : cuda_fail(e, "serve: copy in");
    if (st == BEAGLE_OK) {
        Tune fixed;   // fixed shape: results independent of what else is in the launch
        fixed.cases = kCasesFp32;
        fixed.tile = tile_for(s->cfg.precision, kCasesFp32, 0);
        st = score_jobs(jobs.data(), static_cast<int>(jobs.size()), s->cfg.precision, b.stream,
                        &fixed);
    }
    for (size_t i = 0; st == BEAGLE_OK && i < reqs.size(); ++i) {
        e = cudaMemcpyAsync(reqs[i]->host_out, jobs[i].out,
                            sizeof(beagle_fitness) * reqs[i]->P, cudaMemcpyDeviceToHost,
                            b.stream);
        if (e != cudaSuccess) st = cuda_fail(e, "serve: copy out");
    }
    cudaFreeAsync(base, b.stream);
    if (st == BEAGLE_OK) {
        e = cudaEventRecord(b.event, b.stream);
        if (e != cudaSuccess) st = cuda_fail(e, "serve: event");
    }
    if (st != BEAGLE_OK) return st;
    for (auto &r : reqs) b.bytes += r->dev_bytes;
    s->slot_busy[slot] = true;
    ++s->launches;
    s->inflight.push_back(std::move(b));
    return BEAGLE_OK;
}

void worker_loop(beagle_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // 1. completions
        for (size_t i = 0; i < s->inflight.size();) {
            Batch &b = s->inflight[i];
            const cudaError_t q = cudaEventQuery(b.event);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            const beagle_status st = q == cudaSuccess ? BEAGLE_OK : cuda_fail(q, "serve: batch");
            for (auto &r : b.reqs) finish_request(s, r, st);
            s->bytes_in_use -= b.bytes;
            s->slot_busy[b.slot] = false;
            s->inflight.erase(s->inflight.begin() + static_cast<long>(i));
            s->cv_done.notify_all();
        }
        // 2. admission: arrival order, device-memory budget, a free stream slot
        int slot = -1;
        for (size_t k = 0; k < s->slot_busy.size(); ++k)
            if (!s->slot_busy[k]) { slot = static_cast<int>(k); break; }
        if (slot >= 0 && !s->queue.empty()) {
            std::vector<std::shared_ptr<Request>> take;
            size_t bytes = s->bytes_in_use;
            while (!s->queue.empty() && static_cast<int>(take.size()) < s->cfg.max_batch_jobs) {
                auto &r = s->queue.front();
                if (r->dev_bytes > static_cast<size_t>(s->cfg.hbm_budget_bytes)) {
                    ++s->rejected;   // can never fit: fail it instead of blocking the queue
                    finish_request(s, r, fail(BEAGLE_ERR_OOM, "request needs %zu device bytes, "
                                              "budget is %lld", r->dev_bytes,
                                              (long long)s->cfg.hbm_budget_bytes));
                    s->queue.pop_front();
                    s->cv_done.notify_all();
                    continue;
                }
                if (bytes + r->dev_bytes > static_cast<size_t>(s->cfg.hbm_budget_bytes)) break;
                bytes += r->dev_bytes;
                take.push_back(r);
                s->queue.pop_front();
            }
            if (!take.empty()) {
                s->bytes_in_use = bytes;
                s->peak_bytes = std::max(s->peak_bytes, bytes);
                const beagle_status st = launch_batch(s, take, slot);
                if (st != BEAGLE_OK) {
                    size_t b2 = 0;
                    for (auto &r : take) {
                        b2 += r->dev_bytes;
                        finish_request(s, r, st);
                    }
                    s->bytes_in_use -= b2;
                    s->cv_done.notify_all();
                }
                continue;   // look for more work / completions right away
            }
        }
        if (s->stop && s->queue.empty() && s->inflight.empty()) break;
        // 3. sleep until new work arrives or a short poll interval passes
        if (s->inflight.empty())
            s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

}  // namespace
}  // namespace beagle

extern "C" {

beagle_status beagle_serve_create(const beagle_serve_config *cfg, beagle_server **out) {
    if (!out) return fail(BEAGLE_ERR_ARG, "null server pointer");
    *out = nullptr;
    beagle_serve_config c{};
    if (cfg) c = *cfg;
    if (c.precision != BEAGLE_FP32_COMPENSATED && c.precision != BEAGLE_FP64)
        return fail(BEAGLE_ERR_ARG, "unknown precision %d", c.precision);
    if (c.max_inflight <= 0) c.max_inflight = 2;
    if (c.max_inflight > 8) return fail(BEAGLE_ERR_LIMIT, "max_inflight above 8");
    if (c.max_batch_jobs <= 0) c.max_batch_jobs = 64;
    if (c.max_batch_jobs > 1024) return fail(BEAGLE_ERR_LIMIT, "max_batch_jobs above 1024");
    if (c.hbm_budget_bytes <= 0) {
        size_t fr = 0, tot = 0;
        cudaError_t e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) return cuda_fail(e, "serve: memory info");
        c.hbm_budget_bytes = static_cast<int64_t>(fr / 2);
    }
    auto *s = new beagle_server();
    s->cfg = c;
    cudaGetDevice(&s->device);
    for (int i = 0; i < c.max_inflight; ++i) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            beagle_serve_destroy(s);
            return fail(BEAGLE_ERR_CUDA, "serve: stream or event creation failed");
        }
        s->streams.push_back(st);
        s->events.push_back(ev);
        s->slot_busy.push_back(false);
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return BEAGLE_OK;
}

beagle_status beagle_serve_submit(beagle_server *s, const beagle_request *req, uint64_t *ticket) {
    if (!s || !req || !ticket) return fail(BEAGLE_ERR_ARG, "null pointer argument");
    if (req->P < 0 || req->n_tokens < 0) return fail(BEAGLE_ERR_ARG, "negative size");
    if (req->P > 0 && (!req->programs || !req->offsets || !req->lengths || !req->consts))
        return fail(BEAGLE_ERR_ARG, "null program arrays");
    auto ds = find_dataset(req->dataset_id);
    if (!ds) return fail(BEAGLE_ERR_DATASET, "unknown dataset %d", req->dataset_id);
    if (ds->device != s->device) return fail(BEAGLE_ERR_DATASET, "dataset on another device");
    auto r = std::make_shared<Request>();
    r->dataset = req->dataset_id;
    r->P = req->P;
    r->T = req->n_tokens;
    r->N = ds->N;
    r->off_consts = up256(static_cast<size_t>(r->T));
    r->off_offs = r->off_consts + up256(4 * static_cast<size_t>(r->T));
    r->off_lens = r->off_offs + up256(8 * static_cast<size_t>(r->P));
    r->in_bytes = r->off_lens + 4 * static_cast<size_t>(r->P);
    r->host_in = s->pinned.get(r->in_bytes, &r->in_cls);
    r->host_out = static_cast<beagle_fitness *>(
        s->pinned.get(sizeof(beagle_fitness) * std::max<int64_t>(1, r->P), &r->out_cls));
    if (!r->host_in || !r->host_out) {
        s->pinned.put(r->host_in, r->in_cls);
        s->pinned.put(r->host_out, r->out_cls);
        return fail(BEAGLE_ERR_OOM, "serve: pinned staging");
    }
    char *h = static_cast<char *>(r->host_in);
    std::memcpy(h, req->programs, static_cast<size_t>(r->T));
    std::memcpy(h + r->off_consts, req->consts, 4 * static_cast<size_t>(r->T));
    std::memcpy(h + r->off_offs, req->offsets, 8 * static_cast<size_t>(r->P));
    std::memcpy(h + r->off_lens, req->lengths, 4 * static_cast<size_t>(r->P));
    const int64_t tiles = (ds->N + 511) / 512;
    r->dev_bytes = up256(r->in_bytes) + up256(sizeof(beagle_fitness) * r->P) +
                   up256(static_cast<size_t>(kNumFields) * 4 * tiles * r->P) +
                   up256(4 * static_cast<size_t>(r->P)) + 512;
    hold_dataset(r->dataset, +1);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        hold_dataset(r->dataset, -1);
        return fail(BEAGLE_ERR_BUSY, "server is shutting down");
    }
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    if (!s->have_first) {
        s->t_first = r->t_submit;
        s->have_first = true;
    }
    ++s->submitted;
    if (r->P == 0) {   // nothing to score
        finish_request(s, r, BEAGLE_OK);
    } else {
        s->queue.push_back(r);
        s->cv_work.notify_one();
    }
    s->all[r->ticket] = r;
    *ticket = r->ticket;
    return BEAGLE_OK;
}

static beagle_status collect(beagle_server *s, const std::shared_ptr<Request> &r,
                             beagle_fitness *host_out) {
    if (r->status == BEAGLE_OK && host_out && r->P > 0)
        std::memcpy(host_out, r->host_out, sizeof(beagle_fitness) * r->P);
    s->pinned.put(r->host_out, r->out_cls);
    r->host_out = nullptr;
    s->all.erase(r->ticket);
    if (r->status != BEAGLE_OK) return fail(r->status, "%s", r->message.c_str());
    return BEAGLE_OK;
}

beagle_status beagle_serve_poll(beagle_server *s, uint64_t ticket, beagle_fitness *host_out,
                                int32_t *done) {
    if (!s || !done) return fail(BEAGLE_ERR_ARG, "null pointer argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return fail(BEAGLE_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    auto r = it->second;
    *done = r->done ? 1 : 0;
    if (!r->done) return BEAGLE_OK;
    return collect(s, r, host_out);
}

beagle_status beagle_serve_wait(beagle_server *s, uint64_t ticket, beagle_fitness *host_out,
                                int64_t timeout_us) {
    if (!s) return fail(BEAGLE_ERR_ARG, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return fail(BEAGLE_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    auto r = it->second;
    const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    while (!r->done) {
        if (timeout_us >= 0) {
            if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done)
                return fail(BEAGLE_ERR_TIMEOUT, "ticket %llu not done within %lld us",
                            (unsigned long long)ticket, (long long)timeout_us);
        } else {
            s->cv_done.wait(lk);
        }
    }
    return collect(s, r, host_out);
}

beagle_status beagle_serve_stats(beagle_server *s, beagle_serve_counters *out) {
    if (!s || !out) return fail(BEAGLE_ERR_ARG, "null pointer argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof *out);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->queued = static_cast<int64_t>(s->queue.size());
    out->inflight_launches = static_cast<int64_t>(s->inflight.size());
    out->launches = s->launches;
    out->node_evals = s->node_evals;
    out->bytes_in_use = static_cast<int64_t>(s->bytes_in_use);
    out->peak_bytes = static_cast<int64_t>(s->peak_bytes);
    out->budget_bytes = s->cfg.hbm_budget_bytes;
    if (s->have_first && s->completed > 0) {
        const double sec = std::chrono::duration<double>(s->t_last - s->t_first).count();
        out->gpops = sec > 0 ? static_cast<double>(s->node_evals) / sec / 1e9 : 0.0;
    }
    if (!s->latencies_us.empty()) {
        std::vector<double> v = s->latencies_us;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) {
            const size_t i = static_cast<size_t>(f * static_cast<double>(v.size() - 1) + 0.5);
            return v[std::min(i, v.size() - 1)];
        };
        out->p50_us = q(0.50);
        out->p99_us = q(0.99);
        out->max_us = v.back();
    }
    return BEAGLE_OK;
}

beagle_status beagle_serve_destroy(beagle_server *s) {
    if (!s) return BEAGLE_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->all) {
        auto &r = kv.second;
        s->pinned.put(r->host_in, r->in_cls);
        s->pinned.put(r->host_out, r->out_cls);
    }
    for (auto st : s->streams) cudaStreamDestroy(st);
    for (auto ev : s->events) cudaEventDestroy(ev);
    delete s;
    return BEAGLE_OK;
}

}  // extern "C"
