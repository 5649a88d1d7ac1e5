// Launch entry points of the scoring kernels (host side).
#pragma once

#include "common.cuh"

namespace beagle {

constexpr int kWarpsFp32 = 15;   // consumer warps per CTA, FP32 path (plus one producer warp)
constexpr int kWarpsFp64 = 15;   // consumer warps per CTA, FP64 path
constexpr int kCasesFp32 = 2;    // fitness cases per lane per pass, FP32 path
constexpr int kCasesFp64 = 1;    // fitness cases per lane per pass, FP64 path

// Dynamic shared memory of one CTA for a launch with the given stage size and tile.
size_t smem_bytes(int precision, int xbuf_floats, int tile);

// Enqueue the persistent scoring kernel and the finalize kernel on stream s.
cudaError_t launch_score(const LaunchParams<1> &prm, int precision, int grid, cudaStream_t s);
// Opt-in CUDA-event timing of scoring-kernel launches (beagle_kernel_timing).
bool timing_enabled();
void timing_begin(cudaStream_t s, void **token);
void timing_end(cudaStream_t s, void *token);

cudaError_t launch_score_batch(const LaunchParams<kMaxJobs> &prm, int precision, int grid,
                               cudaStream_t s);

}  // namespace beagle
