// Length-bucketed work order: a counting sort of each job's programs by length, longest
// first, so that the programs a work item hands to its warps have similar lengths and the
// shortest programs come last (a small tail at the end of a persistent launch). With a
// packed-token buffer, each position of the order also gets its program's offset there.
//
// Two launches over chunks of kOrderChunk programs spread over the GPU: per-chunk histograms
// of the length buckets (bucket kMaxLen - L, lengths outside [1, kMaxLen] in the last bucket)
// with the job's bucket totals; then every chunk derives its range in each bucket (the
// bucket's start plus the counts of the job's earlier chunks) and scatters its programs,
// warps taking ranges of their own so that they never contend for a counter. The order among
// equal lengths is not fixed; results do not depend on it (every program's fitness is computed
// on its own).
#include "kernels.h"

namespace beagle {

namespace {

constexpr int kBuckets = kMaxLen + 2;
constexpr int kOrderThreads = 512;
constexpr int kOrderWarps = kOrderThreads / 32;

__device__ __forceinline__ int length_bucket(int32_t L) {
    return (L >= 1 && L <= kMaxLen) ? kMaxLen - L : kMaxLen + 1;
}

__device__ __forceinline__ int chunk_job(const OrderParams &prm, int64_t chunk) {
    int j = 0;
    while (j + 1 < prm.njobs && chunk >= prm.chunk0[j + 1]) ++j;
    return j;
}

__global__ void __launch_bounds__(kOrderThreads) order_hist_kernel(const __grid_constant__ OrderParams prm) {
    __shared__ int hist[kBuckets];
    const int64_t chunk = blockIdx.x;
    const int j = chunk_job(prm, chunk);
    const int64_t p0 = (chunk - prm.chunk0[j]) * kOrderChunk;
    const int64_t p1 = min(prm.P[j], p0 + kOrderChunk);
    for (int b = threadIdx.x; b < kBuckets; b += kOrderThreads) hist[b] = 0;
    __syncthreads();
    const int32_t *lens = prm.lens[j];
    for (int64_t p = p0 + threadIdx.x; p < p1; p += kOrderThreads)
        atomicAdd(&hist[length_bucket(lens[p])], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < kBuckets; b += kOrderThreads) {
        const int c = hist[b];
        prm.hist[chunk * kBuckets + b] = c;
        if (c) atomicAdd(&prm.totals[static_cast<int64_t>(j) * kBuckets + b], c);
    }
}

__global__ void __launch_bounds__(kOrderThreads) order_scatter_kernel(const __grid_constant__ OrderParams prm) {
    __shared__ int whist[kOrderWarps][kBuckets];
    __shared__ int start[kBuckets];
    __shared__ int base[kBuckets];
    __shared__ long long tok0[kBuckets];
    const int64_t chunk = blockIdx.x;
    const int j = chunk_job(prm, chunk);
    const int64_t c = chunk - prm.chunk0[j];
    const int64_t p0 = c * kOrderChunk;
    const int64_t p1 = min(prm.P[j], p0 + kOrderChunk);
    const int32_t *lens = prm.lens[j];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kOrderWarps * kBuckets; i += kOrderThreads)
        (&whist[0][0])[i] = 0;
    // the range of this chunk in each bucket: the counts of the job's earlier chunks
    for (int b = threadIdx.x; b < kBuckets; b += kOrderThreads) {
        int run = 0;
        for (int64_t k = 0; k < c; ++k) run += prm.hist[(prm.chunk0[j] + k) * kBuckets + b];
        base[b] = run;
    }
    if (threadIdx.x == 0) {
        int run = 0;
        long long toks = 0;
        const int *tot = prm.totals + static_cast<int64_t>(j) * kBuckets;
        for (int b = 0; b < kBuckets; ++b) {
            start[b] = run;
            tok0[b] = toks;
            run += tot[b];
            if (b < kMaxLen) toks += static_cast<long long>(tot[b]) * (kMaxLen - b + 1);
        }
    }
    __syncthreads();
    for (int64_t p = p0 + threadIdx.x; p < p1; p += kOrderThreads)
        atomicAdd(&whist[warp][length_bucket(lens[p])], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < kBuckets; b += kOrderThreads) {
        int run = start[b] + base[b];
        for (int w = 0; w < kOrderWarps; ++w) {
            const int k = whist[w][b];
            whist[w][b] = run;
            run += k;
        }
    }
    __syncthreads();
    int32_t *order = prm.order[j];
    uint32_t *poff = prm.poff[j];
    for (int64_t p = p0 + threadIdx.x; p < p1; p += kOrderThreads) {
        const int32_t L = lens[p];
        const int b = length_bucket(L);
        const int pos = atomicAdd(&whist[warp][b], 1);
        order[pos] = static_cast<int32_t>(p);
        if (poff) {
            const long long o = tok0[b] + static_cast<long long>(pos - start[b]) * (L + 1);
            poff[pos] = (b < kMaxLen && o + L + 1 <= prm.pcap[j]) ? static_cast<uint32_t>(o)
                                                                  : kPackNone;
        }
    }
}

}  // namespace

cudaError_t launch_length_order(const OrderParams &prm, cudaStream_t s) {
    if (prm.njobs <= 0 || prm.nchunks <= 0) return cudaSuccess;
    order_hist_kernel<<<static_cast<unsigned>(prm.nchunks), kOrderThreads, 0, s>>>(prm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    order_scatter_kernel<<<static_cast<unsigned>(prm.nchunks), kOrderThreads, 0, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace beagle
