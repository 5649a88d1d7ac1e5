// Internal types shared by the host code and the kernels of libbeagle.
#pragma once

#include <cstdint>
#include <cuda.h>            // CUtensorMap (type only; the encoder is fetched at run time)
#include <cuda_runtime.h>

#include "../../include/beagle.h"

namespace beagle {

constexpr int kBox = 256;                         // cases per TMA box (box dims <= 256)
constexpr int kMaxRows = BEAGLE_MAX_VARS + 2;     // x_0..x_{d-1}, y, y - mean(y)
constexpr int kMaxDepth = BEAGLE_MAX_DEPTH;        // the paper's StackSize (32)
constexpr int kDepthFast = 16;                     // stack of the default scoring pass
// Scratch header of a launch: work counter, error word, one deep-program count per job.
constexpr size_t kHdrCounter = 0, kHdrError = 128, kHdrDeep = 256, kHdrBytes = 512;
constexpr int kMaxLen = BEAGLE_MAX_LENGTH;
constexpr int kMaxJobs = 64;                      // (population, dataset) pairs per launch

// Per-(program, tile) partial sums, stored field-major: field f of (tile t, program p) is
// partials[(f * tiles + t) * P + p] (a 32-bit word). Pairs are (hi, lo) fp32 compensated
// sums on the FP32 path and the two halves of an fp64 value on the FP64 path.
enum Field : int {
    kMean = 0,      // centring value m_t of the tile (fp32; the f value itself if constant)
    kSe2 = 1,       // sum (f - y)^2              (2 words)
    kSd = 3,        // sum (f - m_t)              (2 words)
    kSdd = 5,       // sum (f - m_t)^2            (2 words)
    kSdy = 7,       // sum (f - m_t) (y - ybar)   (2 words)
    kTileFlags = 9, // TF_* bits
    kMean64 = 10,   // FP64 path: second word of the fp64 centring value
    kNumFields = 11
};

// Per-(program, tile) partial sums of the paper's fitness functions (beagle_score_fit), same
// field-major layout. Correlation: the centred sums over the tile's valid pairs (both output
// and target valid), their count, c1 / c2 counts and the extremes of the valid outputs and
// targets (constancy is decided exactly from them); pairs are compensated fp32 pairs on the
// FP32 path, fp64 values on the FP64 path, scaled by 2^-kd (outputs) and 2^-ky (targets).
// Eq. 5 family and validation: the tile's integer score (two words) and c1 / c2.
enum FitField : int {
    kfMean = 0,      // centring value of the valid outputs (T: 1 or 2 words)
    kfN = 2,         // valid pairs
    kfC1 = 3,        // pairs with exactly one invalid member
    kfC2 = 4,        // pairs with both invalid
    kfSd = 5,        // sum (f - m) 2^-kd            (2 words)
    kfSdd = 7,       // sum ((f - m) 2^-kd)^2        (2 words)
    kfSdy = 9,       // sum (f - m) 2^-kd yc 2^-ky   (2 words)
    kfSy = 11,       // sum yc 2^-ky                 (2 words)
    kfSyy = 13,      // sum (yc 2^-ky)^2             (2 words)
    kfFmin = 15,     // smallest and largest valid output (T: 1 or 2 words each)
    kfFmax = 17,
    kfYmin = 19,     // smallest and largest valid target (fp32)
    kfYmax = 20,
    kfFlags = 21,    // TF_* bits | kd << 16 | ky << 24
    kNumFitFields = 22,
    kfScore = 5,     // Eq. 5 family / validation: int64 score of the tile (2 words)
};

// Fitness kinds of a job (include/beagle.h BEAGLE_FIT_*).
constexpr int kFitMse = BEAGLE_FIT_MSE_R2, kFitCorr = BEAGLE_FIT_CORRELATION,
              kFitStd = BEAGLE_FIT_STD, kFitStdHyper = BEAGLE_FIT_STD_HYPER,
              kFitValidate = BEAGLE_FIT_VALIDATE;

enum TileFlag : uint32_t {
    TF_INVALID = 1u,     // some case produced a non-finite value or |v| > 1e30
    TF_NONCONST = 2u,    // outputs in the tile are not all equal
    TF_MALFORMED = 4u,   // program failed the structural check
};

// One (population, dataset) pair of a launch.
struct JobDev {
    const uint8_t *ops;
    const int64_t *offs;
    const int32_t *lens;
    const float *consts;
    beagle_fitness *out;
    uint32_t *partials;      // [kNumFields][tiles][P]
    const double *tile_sy;   // [tiles] per-tile sum of the centred targets the kernel uses
    const int32_t *order;    // optional [P] permutation (programs in processing order)
    void *fout;              // optional [P][N] per-case outputs (float or double), else null
    int64_t P;
    int64_t N;
    int64_t item0;           // first global work item of this job
    int32_t d, rows, tiles, groups;
    double ybar, syy;
    int32_t *deep_list;      // [P] programs deeper than the fast pass's stack (or null)
    int32_t *deep_count;     // their number (device; zeroed before the launch)
    int32_t kind;            // fitness kind (kFit*); kFitMse writes out, the others fit
    int32_t max_score;       // M of the paper's fitness functions
    double tax;              // length tax per token
    beagle_fit_result *fit;  // [P] results of the paper's fitness functions
    // Programs packed once per call by the packing kernel (or null: each work item packs its
    // program itself): position q of the order holds its tokens at packed + poff[q] and its
    // packer result in pmeta[q] (kPackNone where it was not packed).
    uint2 *packed;
    const uint32_t *poff;
    uint32_t *pmeta;
    // Optional [P] flags, zero at launch: program p was found invalid on some tile (MSE kind
    // only). A later tile of p then stores the invalid flag without running it. Null: every
    // case of every tile runs (the early exits are off).
    uint8_t *known_invalid;
    // Optional [P] counters: the fitness cases each program's evaluation ran are added.
    int64_t *cases_run;
};

// Packer result of a pre-packed program: bits 0-15 the handler count, then the flags.
constexpr uint32_t kPackMalformed = 1u << 16;
constexpr uint32_t kPackDeep = 1u << 17;
constexpr uint32_t kPackConstBad = 1u << 18;
constexpr uint32_t kPackNone = 0xffffffffu;   // not packed (no room): the work item packs it
// Room in the packed-token buffer: this many tokens (8 bytes each) per program on average.
constexpr int64_t kPackedPerProgram = 136;

template <int MAXJ>
struct LaunchParams {
    CUtensorMap maps[MAXJ];  // X/y tile maps of each job's dataset
    JobDev jobs[MAXJ];
    int64_t total_items;
    unsigned int *counter;   // work counter (zero at launch)
    unsigned int *error;     // error word (0 = fine)
    int32_t njobs;
    int32_t tile;            // cases per tile: 256 or 512
    int32_t group;           // programs per work item
    int32_t xbuf_floats;     // floats per X stage buffer (max rows x tile)
    uint64_t wait_limit_ns;  // bound of every mbarrier wait (after it: error word, exit)
    int32_t stall_producer;  // test hook: the producer publishes nothing, so waits run out
    int32_t deep_pass;       // 1: this launch scores the jobs' deep lists (a 32-value stack)
};

// Error word bits
constexpr unsigned int kErrTimeoutFull = 1u;
constexpr unsigned int kErrTimeoutEmpty = 2u;

}  // namespace beagle
