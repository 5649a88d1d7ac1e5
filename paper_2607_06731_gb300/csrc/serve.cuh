// Structures the serving loop (serve.cu) shares with its persistent kernel (serve_kernels.cu).
//
// Continuous batching on the device: one persistent kernel (a CTA per SM) takes work items
// from jobs the host keeps appending while it runs. The host writes a request's job -- inputs
// on the device, a descriptor in the job table -- and then raises `njobs` in host memory
// mapped into the device's address space. Each producer warp claims its next item from the
// active jobs in turn (round robin, one claim counter per job), so a job admitted while others
// run gets its share of the GPU at once. The warp that finishes the last tile of a program
// merges its tiles (the finalize step) at once; the warp that finishes the last (program,
// tile) unit of a job stamps the job's end and raises its done flag in mapped host memory,
// where the host's serving thread sees it.
#pragma once

#include "common.cuh"

namespace beagle {

constexpr int kServeMaxJobs = 8192;   // jobs per kernel lifetime (the table is append-only)
constexpr int kServeRows = kMaxRows;  // stage buffers sized for the widest dataset

// Host memory mapped into the device address space (written by the host, read by the device).
struct ServeCtl {
    int32_t njobs;                  // jobs in the table (raised after a job is written)
    int32_t lo;                     // every job before it is finished (its items all claimed)
    int32_t stop;                   // 1: exit once no published work is left
    int32_t pad_;
};

// One job's completion record, in mapped host memory (written by the device).
struct ServeDone {
    unsigned long long t_start;     // %globaltimer when its first unit started
    unsigned long long t_end;       // when its last unit ended
    int32_t deep;                   // programs deeper than the kernel's stack (not scored yet)
    int32_t state;                  // 1 once every unit is done (written last)
};

// Job descriptor in device memory (written by the host before the job is published).
struct alignas(128) ServeJob {   // 128-byte lines: no job shares a cache line with the next
    CUtensorMap map;                // X/y tiles of the job's dataset (box: 256 cases x rows)
    JobDev dev;                     // programs, partials, outputs (fitness in mapped host memory)
    unsigned long long claimed;     // work items claimed so far (zeroed; may pass items)
    int64_t items;                  // groups x tiles
    int32_t group;                  // programs per work item
    int32_t pad_;
    int32_t *tile_done;             // [P] tiles finished per program (zeroed)
    unsigned long long *counters;   // [0] units finished, [1] first start stamp (zeroed / max)
    ServeDone *done;                // the job's completion record (mapped host memory)
};

// Device-side state of the queue (device memory).
struct ServeState {
    unsigned int error;             // bounded-wait failures
    unsigned int pad_[3];
};

struct ServeParams {
    ServeJob *jobs;                 // device [kServeMaxJobs]
    ServeCtl *ctl;                  // mapped host memory
    ServeState *state;              // device
    int32_t tile;
    int32_t xbuf_floats;            // kServeRows x tile
    uint64_t wait_limit_ns;         // bound of the stage barriers' waits
    uint64_t idle_limit_ns;         // the kernel exits after this long without new work
};

// Launch the serving kernel (FP32-compensated or FP64 path) on stream s.
cudaError_t launch_serve(const ServeParams &prm, int precision, cudaStream_t s);
cudaError_t load_serve_kernels();

}  // namespace beagle
