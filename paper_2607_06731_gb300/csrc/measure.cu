// Measurement support: per-operator throughput microbenchmark (roofline peak) and an
// opt-in CUDA-event timer around every scoring-kernel launch.
#include <algorithm>
#include <mutex>
#include <vector>

#include "kernels.h"
#include "registry.h"
#include "score.cuh"

namespace beagle {

// Each thread advances 8 independent chains v <- op(v) and keeps the same validity
// tracker as the interpreter (a NaN-propagating running max of |v|). The chains are
// contractive or bounded so the values stay in the operators' common ranges.
template <int OPC>
__global__ void __launch_bounds__(256) op_rate_kernel(float *sink, int iters, float seed) {
    using A = Arith<float>;
    float v[8], m = 0.0f;
    const float c = 1.0f + 1e-4f * seed;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = 0.5f + 0.01f * k + 1e-6f * threadIdx.x + seed;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float a = v[k];
            if constexpr (OPC == BEAGLE_OP_ADD) a = a + c * 1e-3f;
            else if constexpr (OPC == BEAGLE_OP_SUB) a = a - c * 1e-3f;
            else if constexpr (OPC == BEAGLE_OP_MUL) a = a * c;
            else if constexpr (OPC == BEAGLE_OP_PDIV) a = A::pdiv(c, a);   // divisor varies
            else if constexpr (OPC == BEAGLE_OP_SIN) a = A::sin_(a);
            else if constexpr (OPC == BEAGLE_OP_COS) a = A::cos_(a);
            else if constexpr (OPC == BEAGLE_OP_EXP) a = A::exp_(-a);
            else if constexpr (OPC == BEAGLE_OP_PLOG) a = A::plog(a) + 1.5f;
            else if constexpr (OPC == BEAGLE_OP_PSQRT) a = A::psqrt(a);
            else a = a * a;   // SQUARE
            m = A::track(m, a);
            v[k] = a;
        }
    }
    float s = m;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
    if (s == 12345.678f) sink[threadIdx.x] = s;   // keeps the chains live
}

// Dispatch cost: a threaded loop of the interpreter's dispatch sequence (mask the prefetched
// handler id, prefetch the next token from shared memory, indexed branch) over 256 tokens of
// eight one-instruction handlers, repeated. Each warp reports its cycles; the bounds check
// before the branch ends the loop after the last token.
#define BG_PROBE_DISPATCH                                                                  \
    "and.b32 h, %2, 7;\n\t"                                                                \
    "ld.shared.u32 %2, [%1];\n\t"                                                          \
    "add.u32 %1, %1, 4;\n\t"                                                               \
    "setp.ge.u32 pe, %1, %3;\n\t"                                                          \
    "@pe bra.uni END_%=;\n\t"                                                              \
    "brx.idx.uni h, TBL_%=;\n"

constexpr int kProbeTokens = 256;

__global__ void __launch_bounds__(1024) dispatch_probe_kernel(int reps, long long *cycles,
                                                              float *sink) {
    __shared__ uint32_t tok[32][kProbeTokens + 4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = lane; i < kProbeTokens + 4; i += 32)   // fixed pseudo-random handler ids
        tok[warp][i] = (static_cast<uint32_t>(i) * 2654435761u >> 13) & 7u;
    __syncwarp();
    float a = static_cast<float>(lane);
    const uint32_t base = smem_addr(&tok[warp][0]);
    const long long t0 = clock64();
    for (int r = 0; r < reps; ++r) {
        uint32_t nx = tok[warp][0];
        uint32_t pa = base + 4u;
        const uint32_t pend = base + 4u * kProbeTokens + 4u;
        asm volatile(
            "{\n\t.reg .b32 h;\n\t.reg .pred pe;\n\t"
            "TBL_%=: .branchtargets H0_%=, H1_%=, H2_%=, H3_%=, H4_%=, H5_%=, H6_%=, H7_%=;\n\t"
            BG_PROBE_DISPATCH
            "H0_%=:\n\tadd.f32 %0, %0, 0f3F800000;\n\t" BG_PROBE_DISPATCH
            "H1_%=:\n\tadd.f32 %0, %0, 0f40000000;\n\t" BG_PROBE_DISPATCH
            "H2_%=:\n\tmul.f32 %0, %0, 0f3F000000;\n\t" BG_PROBE_DISPATCH
            "H3_%=:\n\tadd.f32 %0, %0, 0fBF800000;\n\t" BG_PROBE_DISPATCH
            "H4_%=:\n\tadd.f32 %0, %0, 0f40400000;\n\t" BG_PROBE_DISPATCH
            "H5_%=:\n\tmul.f32 %0, %0, 0f3F400000;\n\t" BG_PROBE_DISPATCH
            "H6_%=:\n\tadd.f32 %0, %0, 0f40800000;\n\t" BG_PROBE_DISPATCH
            "H7_%=:\n\tmul.f32 %0, %0, 0f3F200000;\n\t" BG_PROBE_DISPATCH
            "END_%=:\n\t}"
            : "+f"(a), "+r"(pa), "+r"(nx)
            : "r"(pend)
            : "memory");
    }
    const long long t1 = clock64();
    if (lane == 0) cycles[blockIdx.x * 32 + warp] = t1 - t0;
    if (a == 12345.678f) sink[threadIdx.x] = a;
}
#undef BG_PROBE_DISPATCH

template <int OPC>
static double time_op(int blocks, int iters, cudaStream_t s, float *sink) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    op_rate_kernel<OPC><<<blocks, 256, 0, s>>>(sink, iters / 8, 0.0f);   // warm-up
    cudaEventRecord(a, s);
    op_rate_kernel<OPC><<<blocks, 256, 0, s>>>(sink, iters, 0.0f);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double evals = static_cast<double>(blocks) * 256.0 * 8.0 * iters;
    return evals / (ms * 1e-3);
}

// ---------------------------------------------------------------- kernel timer
namespace {
std::mutex g_tmu;
bool g_timing = false;
struct EvPair { cudaEvent_t a, b; };
std::vector<EvPair> g_events;
}

bool timing_enabled() {
    std::lock_guard<std::mutex> lk(g_tmu);
    return g_timing;
}

void timing_begin(cudaStream_t s, void **token) {
    EvPair p;
    cudaEventCreate(&p.a);
    cudaEventCreate(&p.b);
    cudaEventRecord(p.a, s);
    *token = new EvPair(p);
}

void timing_end(cudaStream_t s, void *token) {
    EvPair *p = static_cast<EvPair *>(token);
    cudaEventRecord(p->b, s);
    std::lock_guard<std::mutex> lk(g_tmu);
    g_events.push_back(*p);
    delete p;
}

}  // namespace beagle

using namespace beagle;

extern "C" {

beagle_status beagle_measure_op_rates(double *rates, int32_t n_rates, double seconds_hint,
                                      void *stream) {
    if (!rates || n_rates < BEAGLE_OP_SQUARE + 1)
        return fail(BEAGLE_ERR_ARG, "rates needs room for %d entries", BEAGLE_OP_SQUARE + 1);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *sink = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&sink), 256 * sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail(e, "measure_op_rates");
    const int blocks = sm_count() * 8;
    // About seconds_hint / 10 per operator at ~1e13 simple evaluations per second.
    const double hint = seconds_hint > 0 ? seconds_hint : 1.0;
    const int base = static_cast<int>(std::max(64.0, std::min(1e6, hint * 1e12 / (blocks * 2048.0))));
    for (int i = 0; i < n_rates; ++i) rates[i] = 0.0;
    rates[BEAGLE_OP_ADD] = time_op<BEAGLE_OP_ADD>(blocks, base, s, sink);
    rates[BEAGLE_OP_SUB] = time_op<BEAGLE_OP_SUB>(blocks, base, s, sink);
    rates[BEAGLE_OP_MUL] = time_op<BEAGLE_OP_MUL>(blocks, base, s, sink);
    rates[BEAGLE_OP_PDIV] = time_op<BEAGLE_OP_PDIV>(blocks, base / 4, s, sink);
    rates[BEAGLE_OP_SIN] = time_op<BEAGLE_OP_SIN>(blocks, base / 8, s, sink);
    rates[BEAGLE_OP_COS] = time_op<BEAGLE_OP_COS>(blocks, base / 8, s, sink);
    rates[BEAGLE_OP_EXP] = time_op<BEAGLE_OP_EXP>(blocks, base / 4, s, sink);
    rates[BEAGLE_OP_PLOG] = time_op<BEAGLE_OP_PLOG>(blocks, base / 8, s, sink);
    rates[BEAGLE_OP_PSQRT] = time_op<BEAGLE_OP_PSQRT>(blocks, base / 4, s, sink);
    rates[BEAGLE_OP_SQUARE] = time_op<BEAGLE_OP_SQUARE>(blocks, base, s, sink);
    // PLOG's chain carries one extra add: remove its cost (time per eval is additive).
    if (rates[BEAGLE_OP_PLOG] > 0 && rates[BEAGLE_OP_ADD] > 0) {
        const double t = 1.0 / rates[BEAGLE_OP_PLOG] - 1.0 / rates[BEAGLE_OP_ADD];
        if (t > 0) rates[BEAGLE_OP_PLOG] = 1.0 / t;
    }
    cudaFreeAsync(sink, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "measure_op_rates");
    return BEAGLE_OK;
}

beagle_status beagle_kernel_timing(int32_t enable) {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_timing = enable != 0;
    return BEAGLE_OK;
}

beagle_status beagle_kernel_time(double *total_ms, int64_t *launches) {
    std::vector<EvPair> ev;
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        ev.swap(g_events);
    }
    double tot = 0.0;
    beagle_status st = BEAGLE_OK;
    for (auto &p : ev) {
        cudaError_t e = cudaEventSynchronize(p.b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e != cudaSuccess && st == BEAGLE_OK) st = cuda_fail(e, "kernel_time");
        tot += ms;
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = static_cast<int64_t>(ev.size());
    return st;
}

}  // extern "C"

extern "C" beagle_status beagle_measure_dispatch(int32_t warps_per_sm,
                                                double *cycles_per_dispatch,
                                                double *dispatches_per_sm_cycle) {
    if (warps_per_sm < 1 || warps_per_sm > 32 || !cycles_per_dispatch ||
        !dispatches_per_sm_cycle)
        return fail(BEAGLE_ERR_ARG, "warps_per_sm must be 1-32 and outputs non-null");
    const int grid = sm_count();
    long long *cyc = nullptr;
    float *sink = nullptr;
    cudaError_t e = cudaMalloc(&cyc, sizeof(long long) * grid * 32);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float) * 1024);
    const int reps = 200;
    if (e == cudaSuccess) {
        dispatch_probe_kernel<<<grid, warps_per_sm * 32>>>(2, cyc, sink);   // warm-up
        dispatch_probe_kernel<<<grid, warps_per_sm * 32>>>(reps, cyc, sink);
        e = cudaDeviceSynchronize();
    }
    std::vector<long long> h(static_cast<size_t>(grid) * 32, 0);
    if (e == cudaSuccess)
        e = cudaMemcpy(h.data(), cyc, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost);
    cudaFree(cyc);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "dispatch probe");
    double sum = 0.0;
    long long mx = 1;
    for (int b = 0; b < grid; ++b)
        for (int w = 0; w < warps_per_sm; ++w) {
            sum += static_cast<double>(h[static_cast<size_t>(b) * 32 + w]);
            mx = std::max(mx, h[static_cast<size_t>(b) * 32 + w]);
        }
    const double per_warp = static_cast<double>(kProbeTokens - 1) * reps;
    *cycles_per_dispatch = sum / (static_cast<double>(grid) * warps_per_sm) / per_warp;
    *dispatches_per_sm_cycle = warps_per_sm * per_warp / static_cast<double>(mx);
    return BEAGLE_OK;
}
