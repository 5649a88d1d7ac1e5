// Internal types shared by the host code and the kernels of libbeagle.
#pragma once

#include <cstdint>
#include <cuda.h>            // CUtensorMap (type only; the encoder is fetched at run time)
#include <cuda_runtime.h>

#include "../../include/beagle.h"

namespace beagle {

constexpr int kBox = 256;                         // cases per TMA box (box dims <= 256)
constexpr int kMaxRows = BEAGLE_MAX_VARS + 2;     // x_0..x_{d-1}, y, y - mean(y)
constexpr int kMaxDepth = BEAGLE_MAX_DEPTH;
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
};

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
    int32_t pad_;
};

// Error word bits
constexpr unsigned int kErrTimeoutFull = 1u;
constexpr unsigned int kErrTimeoutEmpty = 2u;

}  // namespace beagle
