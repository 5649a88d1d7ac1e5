// Monte-Carlo ranking ("Monte-Carlo Ranking" in the overview, Table 2): a random sample of 100
// individuals estimates the population's percentiles, and one pass over the fitness array
// gives every individual its percentile group and breeding rights -- its number of children,
// whose expectation per group is Table 2's -- without sorting the population.
//
// One kernel: every CTA sorts the 100 sampled keys in shared memory (a rank sort: each of
// 100 threads counts the keys before its own) and takes the 10th, ..., 90th order statistics
// as thresholds; then a grid-stride pass over the population. Readings: higher keys are better
// (the caller's key is a field of the fitness records, negated for MSE-like fields); a NaN key
// ranks below every other; group g = the number of thresholds the key reaches (>=); children
// = floor(E_g) + 1 when u < E_g - floor(E_g), u a uniform number per individual that the
// caller draws.
#include <cmath>

#include "kernels.h"
#include "registry.h"

namespace beagle {
namespace {

__constant__ double kChildren[10] = {0.01, 0.03, 0.06, 0.15, 0.25, 0.5, 1.0, 1.5, 2.5, 4.0};

__device__ __forceinline__ double load_key(const char *base, int64_t stride, int64_t i, int neg) {
    const double v = *reinterpret_cast<const double *>(base + i * stride);
    return neg ? -v : v;
}

// a before b in ascending order with NaN first; ties broken by index (a stable rank)
__device__ __forceinline__ bool before(double a, int ia, double b, int ib) {
    const bool na = isnan(a), nb = isnan(b);
    if (na || nb) return na && (!nb || ia < ib);
    return a < b || (a == b && ia < ib);
}

__global__ void __launch_bounds__(256) rank_kernel(const char *key, int64_t stride, int neg,
                                                   int64_t P, const int64_t *sample,
                                                   const float *u, uint8_t *group,
                                                   int32_t *children) {
    __shared__ double s[100], sorted[100], thr[9];
    const int t = threadIdx.x;
    if (t < 100) {
        const int64_t i = sample[t];
        s[t] = (i >= 0 && i < P) ? load_key(key, stride, i, neg) : __longlong_as_double(0x7ff8000000000000ll);
    }
    __syncthreads();
    if (t < 100) {
        int r = 0;
        for (int j = 0; j < 100; ++j) r += before(s[j], j, s[t], t);
        sorted[r] = s[t];
    }
    __syncthreads();
    if (t < 9) thr[t] = sorted[10 * (t + 1)];
    __syncthreads();
    for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + t; p < P;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double k = load_key(key, stride, p, neg);
        int g = 0;
        if (!isnan(k)) {
#pragma unroll
            for (int q = 0; q < 9; ++q) g += (!isnan(thr[q]) && k >= thr[q]) ? 1 : 0;
        }
        const double e = kChildren[g], fl = floor(e);
        group[p] = static_cast<uint8_t>(g);
        children[p] = static_cast<int32_t>(fl) + (static_cast<double>(u[p]) < e - fl ? 1 : 0);
    }
}

}  // namespace
}  // namespace beagle

using namespace beagle;

extern "C" beagle_status beagle_rank(const double *key, int64_t key_stride_bytes, int32_t negate,
                                     int64_t P, const int64_t *sample, int32_t n_sample,
                                     const float *u, uint8_t *group_out, int32_t *children_out,
                                     void *stream) {
    if (P < 0 || n_sample != 100) return fail(BEAGLE_ERR_ARG, "P >= 0 and a sample of 100");
    if (P == 0) return BEAGLE_OK;
    if (!key || !sample || !u || !group_out || !children_out)
        return fail(BEAGLE_ERR_ARG, "null pointer argument");
    if (key_stride_bytes < 8 || key_stride_bytes % 8)
        return fail(BEAGLE_ERR_ARG, "key stride must be a positive multiple of 8 bytes");
    const int64_t blocks = std::min<int64_t>((P + 255) / 256, static_cast<int64_t>(sm_count()) * 8);
    rank_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const char *>(key), key_stride_bytes, negate != 0, P, sample, u,
        group_out, children_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rank kernel");
    return BEAGLE_OK;
}
