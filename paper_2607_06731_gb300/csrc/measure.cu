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

// ---------------------------------------------------------------- early exit, case counts
namespace {
std::mutex g_emu;
bool g_early_exit = true;
int64_t *g_cases_run = nullptr;
int64_t g_cases_P = 0;
}

bool early_exit_enabled() {
    std::lock_guard<std::mutex> lk(g_emu);
    return g_early_exit;
}

int64_t *case_counter(int64_t P) {
    std::lock_guard<std::mutex> lk(g_emu);
    return g_cases_run && g_cases_P == P ? g_cases_run : nullptr;
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

beagle_status beagle_set_invalid_early_exit(int32_t enable) {
    std::lock_guard<std::mutex> lk(g_emu);
    g_early_exit = enable != 0;
    return BEAGLE_OK;
}

beagle_status beagle_count_cases(int64_t *cases_run, int64_t P) {
    if (cases_run && P <= 0) return fail(BEAGLE_ERR_ARG, "count_cases: P must be positive");
    std::lock_guard<std::mutex> lk(g_emu);
    g_cases_run = cases_run;
    g_cases_P = cases_run ? P : 0;
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
