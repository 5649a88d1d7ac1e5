// Serving loop: many concurrent evolutionary runs submit one generation (a population to
// score against their resident dataset) at a time, and requests are batched continuously on
// the device.
//
// The paper sends a generation's genomes to the GPU once and returns one fitness per genome
// ("Dividing Tasks Between CPU and GPU") and batches populations so that device memory is
// never exceeded ("Hardware Optimized"); it reuses the memory of dead individuals instead of
// freeing it ("CPU Optimizations"). Here:
//   submit    copies the request's host arrays into pinned staging taken from a size-class
//             pool (recycled, never freed while the server lives) and queues it;
//   admit     one serving thread takes queued requests in arrival order while their device
//             bytes fit the budget, copies each to the device and appends it as a job to the
//             running persistent kernel's queue (serve_kernels.cu) -- the kernel picks the new
//             job's work items up between those of the jobs it is already running, so a small
//             request does not wait for a large one to finish;
//   complete  the kernel raises a job's done flag in host memory once its last program is
//             merged; the fitness records are already in the request's pinned output buffer.
//             The thread retires the job, returns its bytes to the budget and admits more.
// The kernel exits when the host stops it (no work left) or after a bounded idle time, and is
// launched again when work arrives. Programs deeper than its 16-value stack (rare) are scored
// after a drain by the 32-value deep pass. Every program's fitness is computed on its own with
// fixed-order sums and a fixed tile, so a request's results are the same bits alone, in any
// mix, and through beagle_score.
#include <algorithm>
#include <atomic>
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
#include "serve.cuh"

namespace beagle {
namespace {

using Clock = std::chrono::steady_clock;

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

constexpr int kServeTile = 512;
constexpr uint64_t kIdleLimitNs = 50000000ull;   // the kernel exits after 50 ms without work

// Pinned host buffers by power-of-two size class, recycled instead of freed. Mapped into the
// device address space, so the kernel writes fitness records straight into them.
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
        if (cudaHostAlloc(&p, c, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess)
            return nullptr;
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
    std::shared_ptr<Dataset> ds;
    int64_t P = 0, T = 0;        // programs, tokens
    int64_t N = 0;               // cases of the dataset
    void *host_in = nullptr;     // pinned: ops | consts | offsets | lengths
    size_t in_cls = 0, in_bytes = 0;
    size_t off_consts = 0, off_offs = 0, off_lens = 0, off_order = 0;
    beagle_fitness *host_out = nullptr;   // pinned and mapped, P records (written by the GPU)
    size_t out_cls = 0;
    size_t dev_bytes = 0;        // admission charge: inputs and scoring scratch
    bool charged = false;        // dev_bytes counted in the server's bytes in use
    Clock::time_point t_submit, t_admit, t_done;
    beagle_status status = BEAGLE_OK;
    std::string message;
    bool done = false;
    // on the device
    char *dev = nullptr;
    int job = -1;
    int64_t tiles = 0;
    JobDev jd{};
    uint64_t gpu_start = 0, gpu_end = 0;   // %globaltimer stamps of the job
};

struct Timing {
    double queue_us, latency_us;
    uint64_t gpu_start, gpu_end;
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
    std::map<uint64_t, Timing> history;   // completed requests' timing (bounded)
    cudaStream_t kstream = nullptr, cstream = nullptr;
    cudaEvent_t kevent = nullptr;
    bool kernel_running = false;
    // the queue shared with the kernel
    ServeCtl *ctl = nullptr;        // mapped host memory
    ServeDone *dones = nullptr;     // mapped host memory [kServeMaxJobs]
    ServeJob *jobs = nullptr;       // device [kServeMaxJobs]
    ServeState *state = nullptr;    // device
    int njobs = 0;                  // jobs appended since the queue was last reset
    int lo = 0;                     // jobs before it are finished
    std::vector<std::shared_ptr<Request>> inflight;
    uint64_t next_ticket = 1;
    size_t bytes_in_use = 0, peak_bytes = 0;
    int64_t submitted = 0, completed = 0, rejected = 0, launches = 0, jobs_total = 0;
    int64_t node_evals = 0;
    std::vector<double> latencies_us;
    Clock::time_point t_first, t_last;
    bool have_first = false;
    bool stop = false;
    std::thread worker;
};

namespace beagle {
namespace {

void record_timing(beagle_server *s, const std::shared_ptr<Request> &r) {
    Timing tm;
    tm.queue_us = std::chrono::duration<double, std::micro>(r->t_admit - r->t_submit).count();
    tm.latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
    tm.gpu_start = r->gpu_start;
    tm.gpu_end = r->gpu_end;
    s->history[r->ticket] = tm;
    while (s->history.size() > 65536) s->history.erase(s->history.begin());
}

// Called with s->mu held.
void finish_request(beagle_server *s, const std::shared_ptr<Request> &r, beagle_status st) {
    r->status = st;
    if (st != BEAGLE_OK) r->message = beagle_last_error();
    r->done = true;
    r->t_done = Clock::now();
    if (r->t_admit.time_since_epoch().count() == 0) r->t_admit = r->t_done;
    s->pinned.put(r->host_in, r->in_cls);
    r->host_in = nullptr;
    if (r->dev) {
        cudaFreeAsync(r->dev, s->cstream);
        r->dev = nullptr;
    }
    if (r->charged) {
        s->bytes_in_use -= r->dev_bytes;
        r->charged = false;
    }
    if (st == BEAGLE_OK) {
        ++s->completed;
        s->node_evals += r->T * r->N;
        s->latencies_us.push_back(
            std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count());
        s->t_last = r->t_done;
        record_timing(s, r);
    }
    hold_dataset(r->dataset, -1);
    r->ds.reset();
    s->cv_done.notify_all();
}

// Device buffers, input copies and the job descriptor of an admitted request (serving thread,
// without the lock). Returns the job's descriptor in *out.
beagle_status stage_request(beagle_server *s, Request &r, ServeJob *out) {
    const int64_t tiles = (r.N + kServeTile - 1) / kServeTile;
    r.tiles = tiles;
    const size_t b_part = up256(static_cast<size_t>(kNumFields) * 4 * tiles * r.P);
    const size_t b_in = up256(r.in_bytes), b_td = up256(4 * static_cast<size_t>(r.P)),
                 b_flags = up256(static_cast<size_t>(r.P)),
                 b_deep = up256(4 * static_cast<size_t>(r.P)), b_cnt = 256;
    const size_t total = b_in + b_part + b_td + b_flags + b_deep + b_cnt;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&r.dev), total, s->cstream);
    if (e != cudaSuccess) {
        r.dev = nullptr;
        return fail(BEAGLE_ERR_OOM, "serve: device buffers: %s", cudaGetErrorString(e));
    }
    char *in = r.dev, *part = in + b_in, *td = part + b_part, *flags = td + b_td,
         *deep = flags + b_flags, *cnt = deep + b_deep;
    e = cudaMemcpyAsync(in, r.host_in, r.in_bytes, cudaMemcpyHostToDevice, s->cstream);
    if (e == cudaSuccess) e = cudaMemsetAsync(td, 0, b_td + b_flags, s->cstream);   // and flags
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, b_cnt, s->cstream);
    if (e != cudaSuccess) return cuda_fail(e, "serve: copy in");
    void *out_dev = nullptr;
    e = cudaHostGetDevicePointer(&out_dev, r.host_out, 0);
    if (e != cudaSuccess) return cuda_fail(e, "serve: mapped output");
    JobDev &J = r.jd;
    std::memset(&J, 0, sizeof J);
    J.ops = reinterpret_cast<const uint8_t *>(in);
    J.offs = reinterpret_cast<const int64_t *>(in + r.off_offs);
    J.lens = reinterpret_cast<const int32_t *>(in + r.off_lens);
    J.consts = reinterpret_cast<const float *>(in + r.off_consts);
    J.order = reinterpret_cast<const int32_t *>(in + r.off_order);
    J.out = static_cast<beagle_fitness *>(out_dev);
    J.partials = reinterpret_cast<uint32_t *>(part);
    const bool fp64 = s->cfg.precision == BEAGLE_FP64;
    J.tile_sy = fp64 ? r.ds->tile_sy64[0] : r.ds->tile_sy[0];   // 512-case tiles
    J.P = r.P;
    J.N = r.N;
    J.d = r.ds->d;
    J.rows = r.ds->rows;
    J.tiles = static_cast<int32_t>(tiles);
    J.ybar = r.ds->ybar;
    J.syy = fp64 ? r.ds->syy : r.ds->syy32;
    J.deep_list = reinterpret_cast<int32_t *>(deep);
    J.deep_count = reinterpret_cast<int32_t *>(cnt + 128);
    J.kind = kFitMse;
    // the early exit on invalid programs (the request's known-invalid flags, zeroed above)
    J.known_invalid = early_exit_enabled() ? reinterpret_cast<uint8_t *>(flags) : nullptr;
    std::memset(out, 0, sizeof *out);
    out->map = r.ds->map;
    out->dev = J;
    // programs per item: about 32 items per CTA of this request alone, 2-256 programs
    const int64_t work = r.P * tiles;
    const int grid = sm_count();
    out->group = plan_group(work, 31, grid);
    out->items = ((r.P + out->group - 1) / out->group) * tiles;
    out->tile_done = reinterpret_cast<int32_t *>(td);
    out->counters = reinterpret_cast<unsigned long long *>(cnt);
    return BEAGLE_OK;
}

// Launch the serving kernel on the kernel stream (s->mu held).
beagle_status launch_kernel(beagle_server *s) {
    ServeParams prm;
    std::memset(&prm, 0, sizeof prm);
    prm.jobs = s->jobs;
    void *ctl_dev = nullptr;
    cudaHostGetDevicePointer(&ctl_dev, s->ctl, 0);
    prm.ctl = static_cast<ServeCtl *>(ctl_dev);
    prm.state = s->state;
    prm.tile = kServeTile;
    prm.xbuf_floats = kServeRows * kServeTile;
    int32_t stall = 0;
    apply_wait_settings(&prm.wait_limit_ns, &stall);
    prm.idle_limit_ns = kIdleLimitNs;
    reinterpret_cast<volatile int32_t *>(&s->ctl->stop)[0] = 0;
    cudaError_t e = launch_serve(prm, s->cfg.precision, s->kstream);
    if (e == cudaSuccess) e = cudaEventRecord(s->kevent, s->kstream);
    if (e != cudaSuccess) return cuda_fail(e, "serve: kernel launch");
    s->kernel_running = true;
    ++s->launches;
    return BEAGLE_OK;
}

// Programs deeper than the serving kernel's stack: with the kernel stopped, the deep pass and
// the job's finalize on the kernel stream (s->mu held; rare).
beagle_status run_deep(beagle_server *s, Request &r) {
    LaunchParams<1> prm;
    std::memset(&prm, 0, sizeof prm);
    prm.maps[0] = r.ds->map;
    prm.jobs[0] = r.jd;
    char *hdr = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&hdr), kHdrBytes, s->kstream);
    if (e == cudaSuccess) e = cudaMemsetAsync(hdr, 0, kHdrBytes, s->kstream);
    if (e != cudaSuccess) return cuda_fail(e, "serve: deep pass scratch");
    prm.counter = reinterpret_cast<unsigned int *>(hdr + kHdrCounter);
    prm.error = reinterpret_cast<unsigned int *>(hdr + kHdrError);
    prm.njobs = 1;
    prm.tile = kServeTile;
    prm.group = 1;
    prm.xbuf_floats = r.ds->rows * kServeTile;
    int32_t stall = 0;
    apply_wait_settings(&prm.wait_limit_ns, &stall);
    e = launch_deep_and_finalize(prm, s->cfg.precision, s->kstream);
    cudaFreeAsync(hdr, s->kstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->kstream);
    if (e != cudaSuccess) return cuda_fail(e, "serve: deep pass");
    return BEAGLE_OK;
}

void reset_queue(beagle_server *s) {
    s->njobs = 0;
    s->lo = 0;
    reinterpret_cast<volatile int32_t *>(&s->ctl->njobs)[0] = 0;
    reinterpret_cast<volatile int32_t *>(&s->ctl->lo)[0] = 0;
    cudaMemsetAsync(s->state, 0, sizeof(ServeState), s->kstream);
    cudaStreamSynchronize(s->kstream);
}

void worker_loop(beagle_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle_since = Clock::now(), stop_since = Clock::now();
    while (true) {
        // 1. completions: the kernel raises a job's done flag after its last program
        bool deep_wait = false;
        for (size_t i = 0; i < s->inflight.size();) {
            auto r = s->inflight[i];
            const ServeDone *dn = &s->dones[r->job];
            if (reinterpret_cast<const volatile int32_t *>(&dn->state)[0] != 1) {
                ++i;
                continue;
            }
            std::atomic_thread_fence(std::memory_order_acquire);
            r->gpu_start = dn->t_start;
            r->gpu_end = dn->t_end;
            if (dn->deep > 0) {   // its deep programs still to score, with the kernel stopped
                if (s->kernel_running) {
                    deep_wait = true;
                    ++i;
                    continue;
                }
                const beagle_status st = run_deep(s, *r);
                finish_request(s, r, st);
            } else {
                finish_request(s, r, BEAGLE_OK);
            }
            s->inflight.erase(s->inflight.begin() + static_cast<long>(i));
        }
        // jobs before the oldest unfinished one need no more scanning by the kernel
        {
            int lo = s->njobs;
            for (auto &r : s->inflight) lo = std::min(lo, r->job);
            if (lo > s->lo) {
                s->lo = lo;
                reinterpret_cast<volatile int32_t *>(&s->ctl->lo)[0] = lo;
            }
        }
        // 2. the kernel's lifetime: it exits when stopped or idle
        if (s->kernel_running && cudaEventQuery(s->kevent) != cudaErrorNotReady) {
            s->kernel_running = false;
            ServeState st;
            if (cudaMemcpy(&st, s->state, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess ||
                st.error != 0u) {
                // a bounded wait ran out: fail the unfinished jobs and start a fresh queue
                const beagle_status bad = fail(BEAGLE_ERR_TIMEOUT, "serve: a device wait ran out");
                for (auto &r : s->inflight) finish_request(s, r, bad);
                s->inflight.clear();
                reset_queue(s);
            }
            continue;
        }
        if (deep_wait) {
            reinterpret_cast<volatile int32_t *>(&s->ctl->stop)[0] = 1;   // drain, then deep pass
        } else if (!s->kernel_running && s->inflight.empty() && s->njobs > 0 &&
                   (s->queue.empty() || s->njobs >= kServeMaxJobs)) {
            reset_queue(s);
        }
        // 3. admission: arrival order, device-memory budget, room in the job table
        std::vector<std::shared_ptr<Request>> take;
        size_t bytes = s->bytes_in_use;
        while (!deep_wait && !s->queue.empty() &&
               s->njobs + static_cast<int>(take.size()) < kServeMaxJobs &&
               static_cast<int>(take.size()) < s->cfg.max_batch_jobs) {
            auto &r = s->queue.front();
            if (r->dev_bytes > static_cast<size_t>(s->cfg.hbm_budget_bytes)) {
                ++s->rejected;   // can never fit: fail it instead of blocking the queue
                auto rr = r;
                s->queue.pop_front();
                finish_request(s, rr, fail(BEAGLE_ERR_OOM, "request needs %zu device bytes, "
                                           "budget is %lld", rr->dev_bytes,
                                           (long long)s->cfg.hbm_budget_bytes));
                continue;
            }
            if (bytes + r->dev_bytes > static_cast<size_t>(s->cfg.hbm_budget_bytes)) break;
            bytes += r->dev_bytes;
            r->charged = true;
            take.push_back(r);
            s->queue.pop_front();
        }
        if (!take.empty()) {
            s->bytes_in_use = bytes;
            s->peak_bytes = std::max(s->peak_bytes, bytes);
            const int first = s->njobs;
            s->njobs += static_cast<int>(take.size());   // reserve the table slots
            lk.unlock();
            std::vector<ServeJob> descs(take.size());
            std::vector<beagle_status> sts(take.size(), BEAGLE_OK);
            for (size_t i = 0; i < take.size(); ++i) {
                take[i]->t_admit = Clock::now();
                sts[i] = stage_request(s, *take[i], &descs[i]);
            }
            lk.lock();
            // the descriptors, then publication
            for (size_t i = 0; i < take.size(); ++i) {
                descs[i].claimed = 0;
                descs[i].done = s->dones + first + static_cast<int>(i);
                if (sts[i] != BEAGLE_OK) descs[i].items = 0;
                std::memset(s->dones + first + i, 0, sizeof(ServeDone));
            }
            cudaError_t e = cudaMemcpyAsync(s->jobs + first, descs.data(),
                                            sizeof(ServeJob) * descs.size(),
                                            cudaMemcpyHostToDevice, s->cstream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->cstream);
            for (size_t i = 0; i < take.size(); ++i) {
                auto &r = take[i];
                if (sts[i] == BEAGLE_OK && e != cudaSuccess) sts[i] = cuda_fail(e, "serve: job table");
                if (sts[i] != BEAGLE_OK) {
                    finish_request(s, r, sts[i]);
                    continue;
                }
                r->job = first + static_cast<int>(i);
                s->inflight.push_back(r);
                ++s->jobs_total;
            }
            std::atomic_thread_fence(std::memory_order_release);
            reinterpret_cast<volatile int32_t *>(&s->ctl->njobs)[0] = s->njobs;
            std::atomic_thread_fence(std::memory_order_seq_cst);
            idle_since = Clock::now();
        }
        // 4. a kernel for the published work
        if (!s->kernel_running && !deep_wait && !s->inflight.empty()) {
            const beagle_status st = launch_kernel(s);
            if (st != BEAGLE_OK) {
                for (auto &r : s->inflight) finish_request(s, r, st);
                s->inflight.clear();
                reset_queue(s);
            }
            continue;
        }
        // 5. no work left: let the kernel go (other work on this device needs its SMs)
        if (s->kernel_running && s->inflight.empty() && s->queue.empty())
            reinterpret_cast<volatile int32_t *>(&s->ctl->stop)[0] = 1;
        if (s->stop && s->queue.empty() && s->inflight.empty() && !s->kernel_running) break;
        if (s->stop && !s->kernel_running && Clock::now() - stop_since > std::chrono::seconds(30)) {
            // shutting down and the remaining jobs make no progress: fail them
            const beagle_status bad = fail(BEAGLE_ERR_TIMEOUT, "serve: shut down unfinished");
            for (auto &r : s->inflight) finish_request(s, r, bad);
            s->inflight.clear();
            while (!s->queue.empty()) {
                auto r = s->queue.front();
                s->queue.pop_front();
                finish_request(s, r, bad);
            }
            break;
        }
        if (!s->stop) stop_since = Clock::now();
        // 6. wait for work or poll the running jobs
        if (s->inflight.empty() && !s->kernel_running)
            s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
        (void)idle_since;
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
    if (c.max_inflight < 0 || c.max_inflight > 8) return fail(BEAGLE_ERR_LIMIT, "max_inflight above 8");
    if (c.max_batch_jobs <= 0) c.max_batch_jobs = 64;
    if (c.max_batch_jobs > 1024) return fail(BEAGLE_ERR_LIMIT, "max_batch_jobs above 1024");
    if (c.hbm_budget_bytes <= 0) {
        size_t fr = 0, tot = 0;
        cudaError_t e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) return cuda_fail(e, "serve: memory info");
        c.hbm_budget_bytes = static_cast<int64_t>(fr / 2);
    }
    const beagle_status ld = prepare_capture();   // pool settings, kernels loaded
    if (ld != BEAGLE_OK) return ld;
    cudaError_t e = load_serve_kernels();
    if (e != cudaSuccess) return cuda_fail(e, "serve: loading the serving kernel");
    auto *s = new beagle_server();
    s->cfg = c;
    cudaGetDevice(&s->device);
    e = cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->kevent, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void **>(&s->ctl), sizeof(ServeCtl),
                          cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void **>(&s->dones), sizeof(ServeDone) * kServeMaxJobs,
                          cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&s->jobs), sizeof(ServeJob) * kServeMaxJobs);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&s->state), sizeof(ServeState));
    if (e == cudaSuccess) e = cudaMemset(s->state, 0, sizeof(ServeState));
    if (e != cudaSuccess) {
        beagle_serve_destroy(s);
        return cuda_fail(e, "serve: creation");
    }
    std::memset(s->ctl, 0, sizeof(ServeCtl));
    std::memset(s->dones, 0, sizeof(ServeDone) * kServeMaxJobs);
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return BEAGLE_OK;
}

beagle_status beagle_serve_submit(beagle_server *s, const beagle_request *req, uint64_t *ticket) {
    if (!s || !req || !ticket) return fail(BEAGLE_ERR_ARG, "null pointer argument");
    if (req->P < 0 || req->n_tokens < 0) return fail(BEAGLE_ERR_ARG, "negative size");
    if (req->P > (int64_t(1) << 31) - 1) return fail(BEAGLE_ERR_LIMIT, "P >= 2^31");
    if (req->P > 0 && (!req->programs || !req->offsets || !req->lengths || !req->consts))
        return fail(BEAGLE_ERR_ARG, "null program arrays");
    auto ds = find_dataset(req->dataset_id);
    if (!ds) return fail(BEAGLE_ERR_DATASET, "unknown dataset %d", req->dataset_id);
    if (ds->device != s->device) return fail(BEAGLE_ERR_DATASET, "dataset on another device");
    if (ds->invalid_targets)
        return fail(BEAGLE_ERR_DATASET, "dataset %d holds invalid targets", req->dataset_id);
    auto r = std::make_shared<Request>();
    r->dataset = req->dataset_id;
    r->ds = ds;
    r->P = req->P;
    r->T = req->n_tokens;
    r->N = ds->N;
    r->off_consts = up256(static_cast<size_t>(r->T));
    r->off_offs = r->off_consts + up256(4 * static_cast<size_t>(r->T));
    r->off_lens = r->off_offs + up256(8 * static_cast<size_t>(r->P));
    r->off_order = r->off_lens + up256(4 * static_cast<size_t>(r->P));
    r->in_bytes = r->off_order + 4 * static_cast<size_t>(r->P);
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
    // Programs longest first (a counting sort of the lengths): the programs an item hands to
    // its warps then take similar times, and the short ones come last. Results do not depend
    // on the order.
    {
        std::vector<int64_t> start(kMaxLen + 2, 0);
        auto bucket = [](int32_t L) { return (L >= 1 && L <= kMaxLen) ? kMaxLen - L : kMaxLen + 1; };
        for (int64_t p = 0; p < r->P; ++p) ++start[bucket(req->lengths[p])];
        int64_t run = 0;
        for (auto &c : start) {
            const int64_t n = c;
            c = run;
            run += n;
        }
        int32_t *ord = reinterpret_cast<int32_t *>(h + r->off_order);
        for (int64_t p = 0; p < r->P; ++p) ord[start[bucket(req->lengths[p])]++] = static_cast<int32_t>(p);
    }
    const int64_t tiles = (ds->N + kServeTile - 1) / kServeTile;
    r->dev_bytes = up256(r->in_bytes) + up256(static_cast<size_t>(kNumFields) * 4 * tiles * r->P) +
                   2 * up256(4 * static_cast<size_t>(r->P)) + 256;
    hold_dataset(r->dataset, +1);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        hold_dataset(r->dataset, -1);
        s->pinned.put(r->host_in, r->in_cls);
        s->pinned.put(r->host_out, r->out_cls);
        return fail(BEAGLE_ERR_BUSY, "server is shutting down");
    }
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    if (!s->have_first) {
        s->t_first = r->t_submit;
        s->have_first = true;
    }
    ++s->submitted;
    s->all[r->ticket] = r;
    if (r->P == 0) {   // nothing to score
        finish_request(s, r, BEAGLE_OK);
    } else {
        s->queue.push_back(r);
        s->cv_work.notify_one();
    }
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

beagle_status beagle_serve_timing(beagle_server *s, uint64_t ticket, double *queue_us,
                                  double *latency_us, uint64_t *gpu_start_ns,
                                  uint64_t *gpu_end_ns) {
    if (!s) return fail(BEAGLE_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->history.find(ticket);
    if (it == s->history.end())
        return fail(BEAGLE_ERR_ARG, "ticket %llu has not completed (or is too old)",
                    (unsigned long long)ticket);
    if (queue_us) *queue_us = it->second.queue_us;
    if (latency_us) *latency_us = it->second.latency_us;
    if (gpu_start_ns) *gpu_start_ns = it->second.gpu_start;
    if (gpu_end_ns) *gpu_end_ns = it->second.gpu_end;
    return BEAGLE_OK;
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
    if (s->kstream) cudaStreamSynchronize(s->kstream);
    if (s->cstream) cudaStreamSynchronize(s->cstream);
    for (auto &kv : s->all) {
        auto &r = kv.second;
        s->pinned.put(r->host_in, r->in_cls);
        s->pinned.put(r->host_out, r->out_cls);
    }
    if (s->jobs) cudaFree(s->jobs);
    if (s->state) cudaFree(s->state);
    if (s->ctl) cudaFreeHost(s->ctl);
    if (s->dones) cudaFreeHost(s->dones);
    if (s->kevent) cudaEventDestroy(s->kevent);
    if (s->kstream) cudaStreamDestroy(s->kstream);
    if (s->cstream) cudaStreamDestroy(s->cstream);
    delete s;
    return BEAGLE_OK;
}

}  // extern "C"
