// Launch entry points of the scoring kernels (host side).
#pragma once

#include "common.cuh"

namespace beagle {

constexpr int kMaxThreads = 1024;          // 31 consumer warps + 1 producer warp at most
constexpr int kCasesFp32 = 4;              // default fitness cases per lane, FP32 path (2, 4, 8)

// Programs per work item for work = sum of P x tiles over the launch: about 32 items per CTA,
// at least two programs per consumer warp (a smaller item leaves warps waiting for the next
// staged tile) and at most 256; a launch too small for that spreads its items over every CTA.
inline int plan_group(int64_t work, int nw, int grid) {
    int64_t lo = 2LL * nw;
    if (work < lo * grid) lo = work / grid > 1 ? work / grid : 1;
    const int64_t g = work / (32LL * grid);
    return static_cast<int>(g < lo ? lo : (g > 256 ? 256 : g));
}

// Cases per tile for a launch shape: 512 unless the caller asks for 256.
inline int tile_for(int /*precision*/, int /*cases*/, int requested) {
    return requested ? requested : 512;
}
constexpr int kCasesFp64 = 2;              // fitness cases per lane per pass, FP64 path
// Dynamic shared memory per CTA: 227 KB less room for the kernel's static work table.
constexpr size_t kSmemBudget = 225 * 1024;
// The persistent kernels take their SM's tensor memory whole, so they request at least this
// much shared memory: two CTAs of them never share an SM (the second's allocation would wait
// for the first to finish, and the SM it left idle would stay idle).
constexpr size_t kOneCtaPerSmSmem = 116 * 1024;
inline size_t one_cta_per_sm(size_t smem) { return smem > kOneCtaPerSmSmem ? smem : kOneCtaPerSmSmem; }

// Dynamic shared memory of one CTA with nw consumer warps and `cases` cases per lane.
size_t smem_bytes(int precision, int cases, int xbuf_floats, int tile, int nw);
// Most consumer warps whose shared memory fits in kSmemBudget (<= 31 for variants that fit
// in 64 registers per thread, else <= 15).
int plan_warps(int precision, int cases, int xbuf_floats, int tile);

// Enqueue the persistent scoring kernel (nw consumer warps + 1 producer per CTA) and the
// finalize kernel on stream s. `cases` (2, 4 or 8) selects the FP32 instantiation.
cudaError_t launch_score(const LaunchParams<1> &prm, int precision, int cases, int nw, int grid,
                         cudaStream_t s);
// Length-bucketed order of each job's programs (longest first), written to order[j].
// Where poff[j] is set, the same kernel gives each position of the order its offset in a
// packed-token buffer of pcap[j] tokens (each program its length + 1 tokens, in order; those
// that do not fit, and lengths outside [1, kMaxLen], get kPackNone).
// The sort runs over chunks of kOrderChunk programs: job j's chunks are chunk0[j] onward
// (nchunks over all jobs); hist holds nchunks x (kMaxLen + 2) counts and totals njobs x
// (kMaxLen + 2) counts, zeroed before the launch.
constexpr int64_t kOrderChunk = 4096;
struct OrderParams {
    const int32_t *lens[kMaxJobs];
    int32_t *order[kMaxJobs];
    uint32_t *poff[kMaxJobs];
    int64_t pcap[kMaxJobs];
    int64_t P[kMaxJobs];
    int64_t chunk0[kMaxJobs];
    int32_t *hist;
    int32_t *totals;
    int64_t nchunks;
    int32_t njobs;
};
cudaError_t launch_length_order(const OrderParams &prm, cudaStream_t s);
// Pack every program of the jobs that carry a packed-token buffer (JobDev::packed), once per
// call, for the fast pass's 16-value stack; programs deeper than that go to the deep lists.
// On the FP32 path constant subexpressions are folded first.
template <int MAXJ>
cudaError_t launch_pack(const LaunchParams<MAXJ> &prm, int precision, cudaStream_t s);

// Opt-in CUDA-event timing of scoring-kernel launches (beagle_kernel_timing).
bool timing_enabled();
// beagle_set_invalid_early_exit's setting, and beagle_count_cases' device array for a
// single-job launch of P programs (else null).
bool early_exit_enabled();
int64_t *case_counter(int64_t P);
void timing_begin(cudaStream_t s, void **token);
void timing_end(cudaStream_t s, void *token);

cudaError_t launch_score_batch(const LaunchParams<kMaxJobs> &prm, int precision, int cases,
                               int nw, int grid, cudaStream_t s);
// Load every scoring and finalize kernel instantiation (module loading is lazy), so that a
// later stream capture makes no loader calls.
cudaError_t load_kernels();
// The deep pass (32-value stack) over one job's deep list, then the finalize of every program
// of the job (the serving loop's path for programs deeper than its kernel's stack).
cudaError_t launch_deep_and_finalize(const LaunchParams<1> &prm, int precision, cudaStream_t s);

}  // namespace beagle
