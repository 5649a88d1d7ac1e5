// Host-side state shared by the C-ABI translation units.
#pragma once

#include <memory>

#include "common.cuh"

namespace beagle {

constexpr int kTileSizes[2] = {512, 256};    // cases per tile the kernels support

// A resident dataset: rows x_0..x_{d-1}, y, y - ybar, each padded to npad floats.
struct Dataset {
    int32_t id = 0;
    int device = 0;
    int64_t N = 0;
    int32_t d = 0, rows = 0;
    int64_t npad = 0;
    float *data = nullptr;                    // device [rows][npad]
    double *tile_sy[2] = {nullptr, nullptr};    // device, per tile size (512, 256): sums of
                                                // the stored fp32 values of y - ybar
    double *tile_sy64[2] = {nullptr, nullptr};  // same, of (double)y - ybar (FP64 path)
    CUtensorMap map;                          // box: 256 cases x rows
    double ybar = 0.0, syy = 0.0;
    double syy32 = 0.0;                         // sum of squares of the stored fp32 y - ybar
    bool invalid_targets = false;               // y may hold invalid targets (fit kinds only)
    int holds = 0;                            // serving runs that keep it resident
    ~Dataset();
};

std::shared_ptr<Dataset> find_dataset(int32_t id);
// Add delta (+1 / -1) to a dataset's hold count (held datasets cannot be released).
beagle_status hold_dataset(int32_t id, int delta);

// One (population, dataset) pair to score.
struct JobRequest {
    const uint8_t *programs;
    const int64_t *offsets;
    const int32_t *lengths;
    const float *consts;
    int64_t P;
    int32_t dataset_id;
    beagle_fitness *out;
    const int32_t *order;   // optional device permutation of [0, P), may be null
    void *fout;             // optional device [P][N] per-case outputs, may be null
    int32_t kind = 0;       // fitness kind (BEAGLE_FIT_*); MSE_R2 writes out, others fit
    int32_t max_score = 0;  // M of the paper's fitness functions
    double tax = 0.0;       // length tax per token (resolved: >= 0)
    beagle_fit_result *fit = nullptr;
};

// Launch-shape overrides (0 = choose automatically).
struct Tune {
    int group = 0;   // programs per work item
    int tile = 0;    // cases per tile (256 or 512)
    int grid = 0;    // CTAs
    int warps = 0;   // consumer warps per CTA (upper bound)
    int cases = 0;   // fitness cases per lane, FP32 path (2, 4, 8)
    int unsorted = 0;  // 0 automatic, 1 the caller's program order, 2 always the length order
    bool is_auto() const { return !group && !tile && !grid && !warps && !cases && !unsorted; }
};

// Process-wide launch configuration set with beagle_set_launch_config (all zero = automatic).
Tune current_tune();

// Autotuner results, keyed by shape class (precision, rows = d + 2, floor(log2(max N))).
struct TuneKey {
    int precision, rows, log2n;
    bool operator==(const TuneKey &o) const {
        return precision == o.precision && rows == o.rows && log2n == o.log2n;
    }
};
bool find_tuned(int precision, int rows, int64_t max_n, Tune *out);
void store_tuned(int precision, int rows, int64_t max_n, const Tune &t);
void clear_tuned();

// Everything a stream capture of score_jobs must not do the first time: set the memory pool's
// release threshold and load the kernels. Called before capturing.
void keep_pool_memory(int dev);
void apply_wait_settings(uint64_t *limit_ns, int32_t *stall);
beagle_status prepare_capture();

// Enqueue scoring of n jobs on stream s (one persistent launch per 64 jobs).
beagle_status score_jobs(const JobRequest *reqs, int n, int precision, cudaStream_t s,
                         const Tune *tune);

beagle_status fail(beagle_status code, const char *fmt, ...);
beagle_status cuda_fail(cudaError_t e, const char *what);
int sm_count();

}  // namespace beagle
