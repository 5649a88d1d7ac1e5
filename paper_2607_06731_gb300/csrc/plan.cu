// Launch planning: tile size, work-item size, scratch layout and the enqueue of one
// persistent scoring launch (plus finalize) per batch of up to kMaxJobs jobs.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.h"
#include "registry.h"

namespace beagle {

// Keep freed stream-ordered scratch in the device's default pool instead of returning it to
// the driver at every synchronisation, so repeated calls do not remap memory.
void keep_pool_memory(int dev) {
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    done.push_back(dev);
}

// Device-wait settings from the environment (read at every launch):
//   BEAGLE_WAIT_LIMIT_US  bound of every device wait in microseconds (default 4 s);
//   BEAGLE_TEST_STALL=1   test hook: the producer warp publishes no work, so the consumers'
//                         waits run out and every result of the launch carries FLAG_TIMEOUT.
void apply_wait_settings(uint64_t *limit_ns, int32_t *stall) {
    *limit_ns = 0;
    *stall = 0;
    if (const char *v = std::getenv("BEAGLE_WAIT_LIMIT_US")) {
        const long long us = std::atoll(v);
        if (us > 0) *limit_ns = static_cast<uint64_t>(us) * 1000ull;
    }
    if (const char *v = std::getenv("BEAGLE_TEST_STALL")) *stall = std::atoi(v) == 1 ? 1 : 0;
}

beagle_status prepare_capture() {
    int dev = 0;
    cudaGetDevice(&dev);
    keep_pool_memory(dev);
    const cudaError_t e = load_kernels();
    return e == cudaSuccess ? BEAGLE_OK : cuda_fail(e, "loading the scoring kernels");
}

namespace {

struct Planned {
    JobDev dev;
    const CUtensorMap *map;
    size_t part_bytes;
};

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// A launch is cut where the input rows change once it holds this many program-cases
// (P x N summed over its jobs): about 10^9 node evaluations at typical program lengths, a
// millisecond or more of GPU time, so the tail of a persistent launch is a small share.
constexpr int64_t kLaunchCases = int64_t(1) << 24;

template <int MAXJ>
beagle_status enqueue(const std::vector<Planned> &jobs, size_t b, size_t e, int precision,
                      int cases, int tile, int group, int nw, int grid, int xbuf_floats,
                      bool sort, cudaStream_t s) {
    LaunchParams<MAXJ> prm;
    std::memset(&prm, 0, sizeof prm);
    // header (work counters, error word, deep counts), the sort's totals, the known-invalid
    // flags, the sort's histograms, then per job: partials, the length order (when sorting)
    // and the list of programs deeper than the fast pass's stack
    size_t scratch = kHdrBytes;
    // (when sorting, also the packed-token buffer, its offsets and the packer results)
    auto pack_cap = [](int64_t P) {
        const int64_t c = P * kPackedPerProgram;
        return c < int64_t(0xfffffffe) ? c : int64_t(0xfffffffe);
    };
    for (size_t i = b; i < e; ++i) {
        scratch += up256(jobs[i].part_bytes) + up256(sizeof(int32_t) * jobs[i].dev.P);
        if (sort && !jobs[i].dev.order) {
            scratch += up256(sizeof(int32_t) * jobs[i].dev.P) +
                       up256(sizeof(uint2) * pack_cap(jobs[i].dev.P)) +
                       2 * up256(sizeof(uint32_t) * jobs[i].dev.P);
        }
    }
    // the length sort's counts: per-chunk histograms and per-job bucket totals (zeroed with the
    // header)
    int64_t nchunks = 0;
    int norder = 0;
    for (size_t i = b; i < e; ++i)
        if (sort && !jobs[i].dev.order) {
            nchunks += (jobs[i].dev.P + kOrderChunk - 1) / kOrderChunk;
            ++norder;
        }
    const size_t totals_bytes = up256(sizeof(int32_t) * (kMaxLen + 2) * norder);
    const size_t hist_bytes = up256(sizeof(int32_t) * (kMaxLen + 2) * nchunks);
    // each job's known-invalid flags (a byte per program, zeroed with the header)
    size_t flags_bytes = 0;
    for (size_t i = b; i < e; ++i) flags_bytes += up256(static_cast<size_t>(jobs[i].dev.P));
    scratch += totals_bytes + flags_bytes + hist_bytes;
    char *base = nullptr;
    cudaError_t err = cudaMallocAsync(reinterpret_cast<void **>(&base), scratch, s);
    if (err != cudaSuccess)
        return fail(BEAGLE_ERR_OOM, "scratch of %zu bytes: %s", scratch, cudaGetErrorString(err));
    err = cudaMemsetAsync(base, 0, kHdrBytes + totals_bytes + flags_bytes, s);
    if (err != cudaSuccess) {
        cudaFreeAsync(base, s);
        return cuda_fail(err, "scratch memset");
    }
    prm.counter = reinterpret_cast<unsigned int *>(base + kHdrCounter);
    prm.error = reinterpret_cast<unsigned int *>(base + kHdrError);
    char *cur = base + kHdrBytes;
    int32_t *order_totals = reinterpret_cast<int32_t *>(cur);
    cur += totals_bytes;
    uint8_t *flags = reinterpret_cast<uint8_t *>(cur);
    cur += flags_bytes;
    int32_t *order_hist = reinterpret_cast<int32_t *>(cur);
    cur += hist_bytes;
    int64_t items = 0;
    int nj = 0;
    OrderParams op;
    std::memset(&op, 0, sizeof op);
    for (size_t i = b; i < e; ++i, ++nj) {
        prm.maps[nj] = *jobs[i].map;
        prm.jobs[nj] = jobs[i].dev;
        prm.jobs[nj].known_invalid = early_exit_enabled() ? flags : nullptr;
        flags += up256(static_cast<size_t>(jobs[i].dev.P));
        if (MAXJ == 1) prm.jobs[nj].cases_run = case_counter(jobs[i].dev.P);
        prm.jobs[nj].partials = reinterpret_cast<uint32_t *>(cur);
        cur += up256(jobs[i].part_bytes);
        prm.jobs[nj].deep_list = reinterpret_cast<int32_t *>(cur);
        prm.jobs[nj].deep_count = reinterpret_cast<int32_t *>(base + kHdrDeep) + nj;
        cur += up256(sizeof(int32_t) * jobs[i].dev.P);
        if (sort && !jobs[i].dev.order) {
            int32_t *ord = reinterpret_cast<int32_t *>(cur);
            cur += up256(sizeof(int32_t) * jobs[i].dev.P);
            prm.jobs[nj].order = ord;
            uint2 *packed = reinterpret_cast<uint2 *>(cur);
            cur += up256(sizeof(uint2) * pack_cap(jobs[i].dev.P));
            uint32_t *poff = reinterpret_cast<uint32_t *>(cur);
            cur += up256(sizeof(uint32_t) * jobs[i].dev.P);
            uint32_t *pmeta = reinterpret_cast<uint32_t *>(cur);
            cur += up256(sizeof(uint32_t) * jobs[i].dev.P);
            prm.jobs[nj].packed = packed;
            prm.jobs[nj].poff = poff;
            prm.jobs[nj].pmeta = pmeta;
            op.lens[op.njobs] = jobs[i].dev.lens;
            op.order[op.njobs] = ord;
            op.poff[op.njobs] = poff;
            op.pcap[op.njobs] = pack_cap(jobs[i].dev.P);
            op.P[op.njobs] = jobs[i].dev.P;
            op.chunk0[op.njobs] = op.nchunks;
            op.nchunks += (jobs[i].dev.P + kOrderChunk - 1) / kOrderChunk;
            ++op.njobs;
        }
        prm.jobs[nj].groups = static_cast<int32_t>((jobs[i].dev.P + group - 1) / group);
        prm.jobs[nj].item0 = items;
        items += static_cast<int64_t>(prm.jobs[nj].groups) * prm.jobs[nj].tiles;
    }
    prm.njobs = nj;
    prm.total_items = items;
    prm.tile = tile;
    prm.group = group;
    prm.xbuf_floats = xbuf_floats;
    apply_wait_settings(&prm.wait_limit_ns, &prm.stall_producer);
    op.hist = order_hist;
    op.totals = order_totals;
    cudaError_t le = launch_length_order(op, s);
    if (le == cudaSuccess) le = launch_pack(prm, precision, s);
    if (le == cudaSuccess) {
        if constexpr (MAXJ == 1) le = launch_score(prm, precision, cases, nw, grid, s);
        else le = launch_score_batch(prm, precision, cases, nw, grid, s);
    }
    cudaFreeAsync(base, s);
    if (le != cudaSuccess) return cuda_fail(le, "scoring launch");
    return BEAGLE_OK;
}

}  // namespace

beagle_status score_jobs(const JobRequest *reqs, int n, int precision, cudaStream_t s,
                         const Tune *tune) {
    if (n < 0 || (n > 0 && !reqs)) return fail(BEAGLE_ERR_ARG, "bad job list");
    if (precision != BEAGLE_FP32_COMPENSATED && precision != BEAGLE_FP64)
        return fail(BEAGLE_ERR_ARG, "unknown precision %d", precision);
    int dev = 0;
    cudaGetDevice(&dev);
    keep_pool_memory(dev);
    std::vector<std::shared_ptr<Dataset>> keep;
    std::vector<Planned> jobs;
    for (int i = 0; i < n; ++i) {
        const JobRequest &r = reqs[i];
        if (r.P < 0) return fail(BEAGLE_ERR_ARG, "job %d: negative P", i);
        if (r.P > (int64_t(1) << 31) - 1) return fail(BEAGLE_ERR_LIMIT, "job %d: P >= 2^31", i);
        auto ds = find_dataset(r.dataset_id);
        if (!ds) return fail(BEAGLE_ERR_DATASET, "job %d: unknown dataset %d", i, r.dataset_id);
        if (ds->device != dev)
            return fail(BEAGLE_ERR_DATASET, "job %d: dataset %d lives on device %d, current is %d",
                        i, r.dataset_id, ds->device, dev);
        if (r.P == 0) continue;
        if (!r.programs || !r.offsets || !r.lengths || !r.consts ||
            (r.kind == kFitMse ? !r.out : !r.fit))
            return fail(BEAGLE_ERR_ARG, "job %d: null pointer argument", i);
        if (r.kind == kFitMse && ds->invalid_targets)
            return fail(BEAGLE_ERR_DATASET,
                        "job %d: dataset %d holds invalid targets; score it with "
                        "beagle_score_fit", i, r.dataset_id);
        Planned pj;
        std::memset(&pj, 0, sizeof pj);
        pj.dev.ops = r.programs;
        pj.dev.offs = r.offsets;
        pj.dev.lens = r.lengths;
        pj.dev.consts = r.consts;
        pj.dev.out = r.out;
        pj.dev.order = r.order;
        pj.dev.fout = r.fout;
        pj.dev.P = r.P;
        pj.dev.N = ds->N;
        pj.dev.d = ds->d;
        pj.dev.rows = ds->rows;
        pj.dev.ybar = ds->ybar;
        pj.dev.syy = precision == BEAGLE_FP64 ? ds->syy : ds->syy32;
        pj.dev.kind = r.kind;
        pj.dev.max_score = r.max_score;
        pj.dev.tax = r.tax;
        pj.dev.fit = r.fit;
        pj.map = &ds->map;
        keep.push_back(ds);
        jobs.push_back(pj);
    }
    if (jobs.empty()) return BEAGLE_OK;

    // Launches: jobs in ascending order of input rows (d + 2), up to kMaxJobs jobs each. A
    // launch's shared memory is sized by its widest dataset; where that would cost the launch
    // consumer warps (the shared-memory-stack paths) and it already holds enough work to fill
    // the GPU, the launch is cut where the rows change.
    std::vector<size_t> idx(jobs.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(),
                     [&](size_t a, size_t b) { return jobs[a].dev.rows < jobs[b].dev.rows; });
    const Tune cfg0 = tune ? *tune : current_tune();
    std::vector<size_t> cur;
    int64_t cur_cases = 0;   // sum of P x N of the launch being formed
    auto flush = [&]() -> beagle_status {
        if (cur.empty()) return BEAGLE_OK;
        std::vector<Planned> lj;
        std::vector<Dataset *> lds;
        int rows = 1;
        int64_t max_n = 1;
        for (size_t i : cur) {
            lj.push_back(jobs[i]);
            lds.push_back(keep[i].get());
            rows = std::max(rows, jobs[i].dev.rows);
            max_n = std::max(max_n, jobs[i].dev.N);
        }
        cur.clear();
        cur_cases = 0;
        // Launch shape: explicit tune, else the process-wide configuration, else the
        // autotuner's entry for this shape class, else automatic: tile 512 cases, 4 cases per
        // lane, as many consumer warps as shared memory allows, programs ordered by length.
        Tune cfg = cfg0;
        if (!tune && cfg.is_auto()) {
            Tune t;
            if (find_tuned(precision, rows, max_n, &t)) cfg = t;
        }
        if (cfg.tile && cfg.tile != 512 && cfg.tile != 256)
            return fail(BEAGLE_ERR_ARG, "tile must be 256 or 512");
        int cases = kCasesFp32;
        if (cfg.cases) {
            if (cfg.cases != 2 && cfg.cases != 4 && cfg.cases != 8)
                return fail(BEAGLE_ERR_ARG, "cases per lane must be 2, 4 or 8");
            cases = cfg.cases;
        }
        const int tile = tile_for(precision, cases, cfg.tile);
        const int xbuf_floats = rows * tile;
        const int grid = cfg.grid ? cfg.grid : sm_count();
        int nw = plan_warps(precision, cases, xbuf_floats, tile);
        if (cfg.warps) nw = std::min(nw, cfg.warps);
        if (nw < 1 || smem_bytes(precision, cases, xbuf_floats, tile, nw) > kSmemBudget)
            return fail(BEAGLE_ERR_LIMIT, "shared memory plan exceeds %zu bytes", kSmemBudget);
        const int which = tile == 512 ? 0 : 1;
        int64_t work = 0;
        for (size_t i = 0; i < lj.size(); ++i) {
            JobDev &J = lj[i].dev;
            J.tiles = static_cast<int32_t>((J.N + tile - 1) / tile);
            J.tile_sy = precision == BEAGLE_FP64 ? lds[i]->tile_sy64[which] : lds[i]->tile_sy[which];
            lj[i].part_bytes = static_cast<size_t>(J.kind == kFitMse ? static_cast<int>(kNumFields) : static_cast<int>(kNumFitFields)) *
                               J.tiles * J.P * sizeof(uint32_t);
            work += J.P * J.tiles;
        }
        int group = plan_group(work, nw, grid);
        if (cfg.group) group = cfg.group;
        // The length order and the packing kernel (programs packed and folded once per call)
        // pay for their launches only on launches of some size: smaller ones keep the caller's
        // order and pack per work item.
        int64_t pcases = 0;
        for (const Planned &pj : lj) pcases += pj.dev.P * pj.dev.N;
        const bool sort = cfg.unsorted == 2 || (cfg.unsorted == 0 && pcases >= kLaunchCases);
        if (lj.size() == 1)
            return enqueue<1>(lj, 0, 1, precision, cases, tile, group, nw, grid, xbuf_floats,
                              sort, s);
        return enqueue<kMaxJobs>(lj, 0, lj.size(), precision, cases, tile, group, nw, grid,
                                 xbuf_floats, sort, s);
    };
    // Consumer warps a launch would get with stage buffers for `rows` input rows (the shape a
    // launch takes without an autotuned entry): a wider dataset costs warps only on the paths
    // whose stacks live in shared memory; on the default path 31 warps fit up to d = 16.
    auto warps_for = [&](int rows) {
        const int cases = cfg0.cases ? cfg0.cases : kCasesFp32;
        const int tile = tile_for(precision, cases, cfg0.tile);
        int nw = plan_warps(precision, cases, rows * tile, tile);
        return cfg0.warps ? std::min(nw, cfg0.warps) : nw;
    };
    for (size_t i : idx) {
        if (!cur.empty() && (cur.size() == static_cast<size_t>(kMaxJobs) ||
                             (jobs[i].dev.rows != jobs[cur.back()].dev.rows &&
                              cur_cases >= kLaunchCases &&
                              warps_for(jobs[i].dev.rows) < warps_for(jobs[cur.back()].dev.rows)))) {
            const beagle_status st = flush();
            if (st != BEAGLE_OK) return st;
        }
        cur.push_back(i);
        cur_cases += jobs[i].dev.P * jobs[i].dev.N;
    }
    return flush();
}

static std::mutex g_tune_mu;
static Tune g_tune;
static std::vector<std::pair<TuneKey, Tune>> g_tuned;

TuneKey tune_key(int precision, int rows, int64_t max_n) {
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= max_n) ++lg;
    return TuneKey{precision, rows, lg};
}

bool find_tuned(int precision, int rows, int64_t max_n, Tune *out) {
    const TuneKey k = tune_key(precision, rows, max_n);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto &e : g_tuned)
        if (e.first == k) {
            *out = e.second;
            return true;
        }
    return false;
}

void store_tuned(int precision, int rows, int64_t max_n, const Tune &t) {
    const TuneKey k = tune_key(precision, rows, max_n);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &e : g_tuned)
        if (e.first == k) {
            e.second = t;
            return;
        }
    g_tuned.emplace_back(k, t);
}

void clear_tuned() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
}

Tune current_tune() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune;
}

void set_tune(const Tune &t) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune = t;
}

}  // namespace beagle

extern "C" beagle_status beagle_set_launch_config(const beagle_launch_config *cfg) {
    beagle::Tune t;
    if (cfg) {
        if (cfg->cases_per_lane && cfg->cases_per_lane != 2 && cfg->cases_per_lane != 4 &&
            cfg->cases_per_lane != 8)
            return beagle::fail(BEAGLE_ERR_ARG, "cases_per_lane must be 0, 2, 4 or 8");
        if (cfg->tile && cfg->tile != 512 && cfg->tile != 256)
            return beagle::fail(BEAGLE_ERR_ARG, "tile must be 0, 256 or 512");
        if (cfg->warps < 0 || cfg->warps > 31 || cfg->group < 0 || cfg->grid < 0)
            return beagle::fail(BEAGLE_ERR_ARG, "bad launch configuration");
        if (cfg->keep_order < 0 || cfg->keep_order > 2)
            return beagle::fail(BEAGLE_ERR_ARG, "keep_order must be 0, 1 or 2");
        t.cases = cfg->cases_per_lane;
        t.tile = cfg->tile;
        t.group = cfg->group;
        t.warps = cfg->warps;
        t.grid = cfg->grid;
        t.unsorted = cfg->keep_order;
    }
    beagle::set_tune(t);
    return BEAGLE_OK;
}

extern "C" beagle_status beagle_get_launch_config(beagle_launch_config *cfg) {
    if (!cfg) return beagle::fail(BEAGLE_ERR_ARG, "null pointer argument");
    const beagle::Tune t = beagle::current_tune();
    cfg->cases_per_lane = t.cases;
    cfg->tile = t.tile;
    cfg->group = t.group;
    cfg->warps = t.warps;
    cfg->grid = t.grid;
    cfg->keep_order = t.unsorted;
    return BEAGLE_OK;
}
