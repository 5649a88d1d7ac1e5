// Ragged batches: many (population, dataset) jobs in one persistent launch, a CUDA-graph plan
// that replays such a launch, and the autotuner that picks launch shapes by timing them.
#include <algorithm>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "registry.h"

namespace beagle {
namespace {

beagle_status to_requests(const beagle_job *jobs, int32_t n, std::vector<JobRequest> *out) {
    if (n < 0 || (n > 0 && !jobs)) return fail(BEAGLE_ERR_ARG, "bad job list");
    out->clear();
    for (int32_t i = 0; i < n; ++i) {
        const beagle_job &j = jobs[i];
        out->push_back(JobRequest{j.programs, j.offsets, j.lengths, j.consts, j.P, j.dataset_id,
                                  j.fitness_out, nullptr, nullptr});
    }
    return BEAGLE_OK;
}

}  // namespace
}  // namespace beagle

using namespace beagle;

struct beagle_batch_plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int32_t> held;   // dataset ids kept resident by this plan
};

extern "C" {

beagle_status beagle_score_batch(const beagle_job *jobs, int32_t n_jobs, int32_t precision,
                                 void *stream) {
    std::vector<JobRequest> reqs;
    beagle_status st = to_requests(jobs, n_jobs, &reqs);
    if (st != BEAGLE_OK) return st;
    return score_jobs(reqs.data(), n_jobs, precision, static_cast<cudaStream_t>(stream), nullptr);
}

beagle_status beagle_batch_plan_create(const beagle_job *jobs, int32_t n_jobs, int32_t precision,
                                       beagle_batch_plan **plan) {
    if (!plan) return fail(BEAGLE_ERR_ARG, "null plan pointer");
    *plan = nullptr;
    std::vector<JobRequest> reqs;
    beagle_status st = to_requests(jobs, n_jobs, &reqs);
    if (st != BEAGLE_OK) return st;
    auto *pl = new beagle_batch_plan();
    for (const auto &r : reqs) {
        st = hold_dataset(r.dataset_id, +1);
        if (st != BEAGLE_OK) {
            for (int32_t id : pl->held) hold_dataset(id, -1);
            delete pl;
            return st;
        }
        pl->held.push_back(r.dataset_id);
    }
    st = prepare_capture();
    if (st != BEAGLE_OK) {
        beagle_batch_plan_destroy(pl);
        return st;
    }
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        if (s) cudaStreamDestroy(s);
        beagle_batch_plan_destroy(pl);
        return cuda_fail(e, "batch plan: begin capture");
    }
    st = score_jobs(reqs.data(), n_jobs, precision, s, nullptr);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    cudaStreamDestroy(s);
    if (st != BEAGLE_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        beagle_batch_plan_destroy(pl);
        return st != BEAGLE_OK ? st : cuda_fail(e, "batch plan: end capture");
    }
    pl->graph = g;
    e = cudaGraphInstantiate(&pl->exec, g, 0);
    if (e != cudaSuccess) {
        beagle_batch_plan_destroy(pl);
        return cuda_fail(e, "batch plan: instantiate");
    }
    *plan = pl;
    return BEAGLE_OK;
}

beagle_status beagle_batch_plan_launch(beagle_batch_plan *plan, void *stream) {
    if (!plan || !plan->exec) return fail(BEAGLE_ERR_ARG, "null plan");
    cudaError_t e = cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "batch plan: launch");
    return BEAGLE_OK;
}

beagle_status beagle_batch_plan_destroy(beagle_batch_plan *plan) {
    if (!plan) return BEAGLE_OK;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    for (int32_t id : plan->held) hold_dataset(id, -1);
    delete plan;
    return BEAGLE_OK;
}

beagle_status beagle_autotune(const beagle_job *jobs, int32_t n_jobs, int32_t precision,
                              int32_t max_trials, void *stream, beagle_launch_config *best,
                              double *best_ms) {
    std::vector<JobRequest> reqs;
    beagle_status st = to_requests(jobs, n_jobs, &reqs);
    if (st != BEAGLE_OK) return st;
    if (n_jobs == 0) return fail(BEAGLE_ERR_ARG, "no jobs to tune on");
    int rows = 1;
    int64_t max_n = 1;
    for (const auto &r : reqs) {
        auto ds = find_dataset(r.dataset_id);
        if (!ds) return fail(BEAGLE_ERR_DATASET, "unknown dataset %d", r.dataset_id);
        rows = std::max(rows, ds->rows);
        max_n = std::max(max_n, ds->N);
    }
    // Candidates: cases per lane x tile x programs per item (0 = planner's choice).
    std::vector<Tune> cand;
    const int cases_list[3] = {4, 2, 8};
    const int tile_list[2] = {512, 256};
    const int group_list[2] = {0, 64};
    for (int c : cases_list)
        for (int t : tile_list)
            for (int g : group_list) {
                if (precision == BEAGLE_FP64 && c != 4) continue;   // one FP64 instantiation
                Tune tn;
                tn.cases = c;
                tn.tile = t;
                tn.group = g;
                cand.push_back(tn);
            }
    if (max_trials > 0 && static_cast<size_t>(max_trials) < cand.size()) cand.resize(max_trials);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double best_t = 1e300;
    Tune best_tune;
    for (const Tune &tn : cand) {
        st = score_jobs(reqs.data(), n_jobs, precision, s, &tn);   // warm-up (and validity)
        if (st == BEAGLE_ERR_LIMIT) {   // this shape does not fit (shared memory): skip it
            st = BEAGLE_OK;
            continue;
        }
        cudaEventRecord(a, s);
        for (int rep = 0; rep < 2 && st == BEAGLE_OK; ++rep)
            st = score_jobs(reqs.data(), n_jobs, precision, s, &tn);
        cudaEventRecord(b, s);
        if (st != BEAGLE_OK) break;
        if (cudaEventSynchronize(b) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms / 2.0 < best_t) {
            best_t = ms / 2.0;
            best_tune = tn;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != BEAGLE_OK) return st;
    if (best_t >= 1e300) return fail(BEAGLE_ERR_LIMIT, "no candidate launch shape fits");
    store_tuned(precision, rows, max_n, best_tune);
    if (best) {
        best->cases_per_lane = best_tune.cases;
        best->tile = best_tune.tile;
        best->group = best_tune.group;
        best->warps = best_tune.warps;
        best->grid = best_tune.grid;
        best->keep_order = best_tune.unsorted;
    }
    if (best_ms) *best_ms = best_t;
    return BEAGLE_OK;
}

beagle_status beagle_autotune_clear(void) {
    clear_tuned();
    return BEAGLE_OK;
}

}  // extern "C"
