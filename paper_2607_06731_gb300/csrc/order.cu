// Length-bucketed work order: a counting sort of each job's programs by length, longest
// first, so that the programs a work item hands to its warps have similar lengths and the
// shortest programs come last (a small tail at the end of a persistent launch).
#include "kernels.h"

namespace beagle {

namespace {

// One CTA per job: histogram of lengths (bucket kMaxLen + 1 - L, lengths outside [1, kMaxLen]
// in the last bucket), exclusive scan, scatter. The order among equal lengths is not fixed;
// results do not depend on it (every program's fitness is computed on its own). With a
// packed-token buffer, the scan also gives each bucket its first token, so a program's offset
// is its bucket's first token plus its rank in the bucket times its length + 1.
__global__ void __launch_bounds__(1024) length_order_kernel(const __grid_constant__ OrderParams prm) {
    constexpr int kBuckets = kMaxLen + 2;
    __shared__ int hist[kBuckets];
    __shared__ int start[kBuckets];
    __shared__ long long tok0[kBuckets];
    const int j = blockIdx.x;
    if (j >= prm.njobs) return;
    const int32_t *lens = prm.lens[j];
    int32_t *order = prm.order[j];
    uint32_t *poff = prm.poff[j];
    const int64_t P = prm.P[j];
    for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    auto bucket = [](int32_t L) {
        return (L >= 1 && L <= kMaxLen) ? kMaxLen - L : kMaxLen + 1;
    };
    for (int64_t p = threadIdx.x; p < P; p += blockDim.x) atomicAdd(&hist[bucket(lens[p])], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        long long toks = 0;
        for (int b = 0; b < kBuckets; ++b) {
            const int c = hist[b];
            hist[b] = run;
            start[b] = run;
            tok0[b] = toks;
            run += c;
            if (b < kMaxLen) toks += static_cast<long long>(c) * (kMaxLen - b + 1);
        }
    }
    __syncthreads();
    for (int64_t p = threadIdx.x; p < P; p += blockDim.x) {
        const int32_t L = lens[p];
        const int b = bucket(L);
        const int pos = atomicAdd(&hist[b], 1);
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
    if (prm.njobs <= 0) return cudaSuccess;
    length_order_kernel<<<prm.njobs, 1024, 0, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace beagle
