// Host side of the C ABI (include/beagle.h): dataset registry, argument checks, launch
// planning and the host-buffer convenience call.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "registry.h"

namespace beagle {

static thread_local std::string g_err;

beagle_status fail(beagle_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

beagle_status cuda_fail(cudaError_t e, const char *what) {
    return fail(BEAGLE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------------ dataset registry
static std::mutex g_mu;
static std::unordered_map<int32_t, std::shared_ptr<Dataset>> g_sets;
static int32_t g_next_id = 1;

std::shared_ptr<Dataset> find_dataset(int32_t id) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_sets.find(id);
    return it == g_sets.end() ? nullptr : it->second;
}

beagle_status hold_dataset(int32_t id, int delta) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_sets.find(id);
    if (it == g_sets.end()) return fail(BEAGLE_ERR_DATASET, "unknown dataset %d", id);
    it->second->holds += delta;
    return BEAGLE_OK;
}

Dataset::~Dataset() {
    if (data) cudaFree(data);
    if (tile_sy[0]) cudaFree(tile_sy[0]);
    if (tile_sy[1]) cudaFree(tile_sy[1]);
    if (tile_sy64[0]) cudaFree(tile_sy64[0]);
    if (tile_sy64[1]) cudaFree(tile_sy64[1]);
}

// Neumaier-compensated fp64 accumulator.
struct Acc {
    double s = 0.0, c = 0.0;
    void add(double x) {
        const double t = s + x;
        c += std::fabs(s) >= std::fabs(x) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    double value() const { return s + c; }
};

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace beagle

using namespace beagle;

extern "C" {

const char *beagle_last_error(void) { return g_err.c_str(); }

int32_t beagle_version(void) { return 100; }

beagle_status beagle_upload_dataset(const float *X, const float *y, int64_t N, int32_t d,
                                    int32_t inputs_on_device, void *stream,
                                    int32_t *dataset_id) {
    return beagle_upload_dataset_ex(X, y, N, d, inputs_on_device, 0u, stream, dataset_id);
}

beagle_status beagle_upload_dataset_ex(const float *X, const float *y, int64_t N, int32_t d,
                                       int32_t inputs_on_device, uint32_t flags, void *stream,
                                       int32_t *dataset_id) {
    if (!X || !y || !dataset_id) return fail(BEAGLE_ERR_ARG, "null pointer argument");
    if (flags & ~BEAGLE_DATASET_INVALID_TARGETS) return fail(BEAGLE_ERR_ARG, "unknown flags");
    const bool allow_invalid = (flags & BEAGLE_DATASET_INVALID_TARGETS) != 0;
    if (N < 2) return fail(BEAGLE_ERR_ARG, "N must be >= 2 (got %lld)", (long long)N);
    if (d < 1 || d > BEAGLE_MAX_VARS)
        return fail(BEAGLE_ERR_LIMIT, "d must be in [1, %d] (got %d)", BEAGLE_MAX_VARS, d);
    if (N > (int64_t(1) << 31) - 1024)
        return fail(BEAGLE_ERR_LIMIT, "N above 2^31 - 1024 is not supported");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<float> hx(static_cast<size_t>(N) * d), hy(static_cast<size_t>(N));
    if (inputs_on_device) {
        cudaError_t e = cudaMemcpyAsync(hx.data(), X, hx.size() * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hy.data(), y, hy.size() * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "reading device dataset");
    } else {
        std::memcpy(hx.data(), X, hx.size() * 4);
        std::memcpy(hy.data(), y, hy.size() * 4);
    }
    for (size_t i = 0; i < hx.size(); ++i)
        if (!(std::fabs(static_cast<double>(hx[i])) <= 1e30))
            return fail(BEAGLE_ERR_DATASET, "X value %zu is non-finite or above 1e30", i);
    // Mean and sum of squares of the valid targets (all of them, unless invalid targets are
    // allowed).
    auto valid_y = [](float v) { return std::fabs(static_cast<double>(v)) <= 1e30; };
    Acc sy;
    int64_t nvalid = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (!valid_y(hy[i])) {
            if (allow_invalid) continue;
            return fail(BEAGLE_ERR_DATASET, "y value %lld is non-finite or above 1e30", (long long)i);
        }
        sy.add(hy[i]);
        ++nvalid;
    }
    const double ybar = nvalid ? sy.value() / static_cast<double>(nvalid) : 0.0;
    Acc syy;
    for (int64_t i = 0; i < N; ++i) {
        if (!valid_y(hy[i])) continue;
        const double c = static_cast<double>(hy[i]) - ybar;
        syy.add(c * c);
    }
    if (!allow_invalid && !(syy.value() > 0.0))
        return fail(BEAGLE_ERR_DATASET, "y is constant (S_yy = 0)");

    auto ds = std::make_shared<Dataset>();
    ds->N = N;
    ds->d = d;
    ds->rows = d + 2;
    ds->npad = (N + 63) / 64 * 64;
    ds->ybar = ybar;
    ds->syy = syy.value();
    ds->invalid_targets = allow_invalid;
    cudaGetDevice(&ds->device);
    const int64_t npad = ds->npad;
    std::vector<float> lay(static_cast<size_t>(ds->rows) * npad, 0.0f);
    for (int k = 0; k < d; ++k)
        std::memcpy(&lay[static_cast<size_t>(k) * npad], &hx[static_cast<size_t>(k) * N], N * 4);
    std::memcpy(&lay[static_cast<size_t>(d) * npad], hy.data(), N * 4);
    float *yc = &lay[static_cast<size_t>(d + 1) * npad];
    Acc syy32;
    for (int64_t i = 0; i < N; ++i) {
        if (!valid_y(hy[i])) {   // an invalid target: the centred row holds NaN there
            yc[i] = std::numeric_limits<float>::quiet_NaN();
            continue;
        }
        yc[i] = static_cast<float>(static_cast<double>(hy[i]) - ybar);
        syy32.add(static_cast<double>(yc[i]) * static_cast<double>(yc[i]));
    }
    // The FP32 path correlates outputs with these stored values, so its S_yy is theirs too
    // (1 - r^2 of an exact fit then stays at rounding level instead of 2^-24).
    ds->syy32 = syy32.value();
    // Per-tile sums of the stored centred targets, for the two tile sizes the kernels use.
    for (int which = 0; which < 2; ++which) {
        const int tile = kTileSizes[which];
        const int64_t T = (N + tile - 1) / tile;
        std::vector<double> ts(static_cast<size_t>(T)), ts64(static_cast<size_t>(T));
        for (int64_t t = 0; t < T; ++t) {
            Acc a, a64;
            for (int64_t i = t * tile; i < std::min(N, (t + 1) * tile); ++i) {
                if (!valid_y(hy[i])) continue;
                a.add(yc[i]);
                a64.add(static_cast<double>(hy[i]) - ybar);
            }
            ts[static_cast<size_t>(t)] = a.value();
            ts64[static_cast<size_t>(t)] = a64.value();
        }
        cudaError_t e = cudaMalloc(&ds->tile_sy[which], ts.size() * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMemcpy(ds->tile_sy[which], ts.data(), ts.size() * sizeof(double),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&ds->tile_sy64[which], ts64.size() * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMemcpy(ds->tile_sy64[which], ts64.data(), ts64.size() * sizeof(double),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(BEAGLE_ERR_OOM, "dataset upload: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaMalloc(&ds->data, lay.size() * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemcpy(ds->data, lay.data(), lay.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(BEAGLE_ERR_OOM, "dataset upload: %s", cudaGetErrorString(e));

    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(BEAGLE_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(N), static_cast<cuuint64_t>(ds->rows)};
    const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(npad) * sizeof(float)};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(kBox), static_cast<cuuint32_t>(ds->rows)};
    const cuuint32_t estride[2] = {1, 1};
    CUresult cr = enc(&ds->map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ds->data, gdim, gstride, box,
                      estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return fail(BEAGLE_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);

    std::lock_guard<std::mutex> lk(g_mu);
    ds->id = g_next_id++;
    g_sets[ds->id] = ds;
    *dataset_id = ds->id;
    return BEAGLE_OK;
}

beagle_status beagle_release_dataset(int32_t dataset_id) {
    std::shared_ptr<Dataset> ds;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_sets.find(dataset_id);
        if (it == g_sets.end()) return fail(BEAGLE_ERR_DATASET, "unknown dataset %d", dataset_id);
        if (it->second->holds > 0)
            return fail(BEAGLE_ERR_BUSY, "dataset %d is held by %d plan(s) or serving run(s)", dataset_id,
                        it->second->holds);
        ds = it->second;
        g_sets.erase(it);
    }
    cudaError_t e = cudaDeviceSynchronize();   // let enqueued work that reads it finish
    ds.reset();
    if (e != cudaSuccess) return cuda_fail(e, "release_dataset");
    return BEAGLE_OK;
}

beagle_status beagle_dataset_info(int32_t dataset_id, int64_t *N, int32_t *d, double *ybar,
                                  double *syy) {
    auto ds = find_dataset(dataset_id);
    if (!ds) return fail(BEAGLE_ERR_DATASET, "unknown dataset %d", dataset_id);
    if (N) *N = ds->N;
    if (d) *d = ds->d;
    if (ybar) *ybar = ds->ybar;
    if (syy) *syy = ds->syy;
    return BEAGLE_OK;
}

beagle_status beagle_validate_programs(const uint8_t *programs, const int64_t *offsets,
                                       const int32_t *lengths, int64_t P, int32_t d,
                                       int32_t max_depth, int64_t *first_bad) {
    return beagle_validate_programs_ex(programs, offsets, lengths, P, d, max_depth, nullptr, 0,
                                       first_bad);
}

beagle_status beagle_validate_programs_ex(const uint8_t *programs, const int64_t *offsets,
                                          const int32_t *lengths, int64_t P, int32_t d,
                                          int32_t max_depth, const uint8_t *allowed,
                                          int32_t n_allowed, int64_t *first_bad) {
    if (first_bad) *first_bad = -1;
    if (P < 0 || (P > 0 && (!programs || !offsets || !lengths)))
        return fail(BEAGLE_ERR_ARG, "bad arguments");
    if (n_allowed < 0 || (n_allowed > 0 && !allowed)) return fail(BEAGLE_ERR_ARG, "bad allowed list");
    // operator kind of a token for the whitelist: LOAD_k -> LOAD0, COPY/PASTE_k -> COPY0
    auto kind_of = [](int op) {
        if (op >= BEAGLE_OP_LOAD0 && op < BEAGLE_OP_LOAD0 + BEAGLE_MAX_VARS) return BEAGLE_OP_LOAD0;
        if ((op >= BEAGLE_OP_COPY0 && op < BEAGLE_OP_COPY0 + BEAGLE_MAX_REGS) ||
            (op >= BEAGLE_OP_PASTE0 && op < BEAGLE_OP_PASTE0 + BEAGLE_MAX_REGS))
            return BEAGLE_OP_COPY0;
        return op;
    };
    bool ok_kind[256];
    for (int k = 0; k < 256; ++k) ok_kind[k] = n_allowed == 0;
    for (int32_t i = 0; i < n_allowed; ++i) ok_kind[kind_of(allowed[i])] = true;
    for (int64_t p = 0; p < P; ++p) {
        const int32_t L = lengths[p];
        const char *why = nullptr;
        if (L < 1 || L > BEAGLE_MAX_LENGTH) why = "length out of [1, BEAGLE_MAX_LENGTH]";
        int depth = 0;
        bool full[BEAGLE_MAX_REGS] = {false};
        for (int32_t j = 0; !why && j < L; ++j) {
            const int op = programs[offsets[p] + j];
            int need = 0, delta = 0;
            if (op == BEAGLE_OP_CONST) delta = 1;
            else if (op >= BEAGLE_OP_LOAD0 && op < BEAGLE_OP_LOAD0 + BEAGLE_MAX_VARS) {
                if (op - BEAGLE_OP_LOAD0 >= d) why = "variable index >= d";
                delta = 1;
            } else if ((op >= BEAGLE_OP_ADD && op <= BEAGLE_OP_PDIV) || op == BEAGLE_OP_POW) {
                need = 2; delta = -1;
            } else if ((op >= BEAGLE_OP_SIN && op <= BEAGLE_OP_SQUARE) ||
                       (op >= BEAGLE_OP_SIGN && op <= BEAGLE_OP_TANH)) {
                need = 1;
            } else if (op == BEAGLE_OP_DUP) { need = 1; delta = 1; }
            else if (op == BEAGLE_OP_SWAP) need = 2;
            else if (op == BEAGLE_OP_DEL) { need = 1; delta = -1; }
            else if (op >= BEAGLE_OP_COPY0 && op < BEAGLE_OP_COPY0 + BEAGLE_MAX_REGS) {
                need = 1;
                if (full[op - BEAGLE_OP_COPY0]) why = "COPY into a variable that is still full";
                full[op - BEAGLE_OP_COPY0] = true;
            } else if (op >= BEAGLE_OP_PASTE0 && op < BEAGLE_OP_PASTE0 + BEAGLE_MAX_REGS) {
                delta = 1;
                if (!full[op - BEAGLE_OP_PASTE0]) why = "PASTE of an empty variable";
                full[op - BEAGLE_OP_PASTE0] = false;
            } else why = "unknown opcode";
            if (!why && !ok_kind[kind_of(op)]) why = "operator not in the allowed list";
            if (!why && depth < need) why = "stack underflow";
            depth += delta;
            if (!why && depth > max_depth) why = "stack deeper than max_depth";
        }
        for (int k = 0; !why && k < BEAGLE_MAX_REGS; ++k)
            if (full[k]) why = "COPY without a PASTE";
        if (!why && depth != 1) why = "program does not leave exactly one value";
        if (why) {
            if (first_bad) *first_bad = p;
            return fail(BEAGLE_ERR_PROGRAM, "program %lld: %s", (long long)p, why);
        }
    }
    return BEAGLE_OK;
}

beagle_status beagle_score(const uint8_t *programs, const int64_t *offsets,
                           const int32_t *lengths, const float *consts, int64_t P,
                           int32_t dataset_id, beagle_fitness *fitness_out,
                           int32_t precision, void *stream) {
    JobRequest req{programs, offsets, lengths, consts, P, dataset_id, fitness_out, nullptr,
                   nullptr};
    return score_jobs(&req, 1, precision, static_cast<cudaStream_t>(stream), nullptr);
}

beagle_status beagle_score_fit(const uint8_t *programs, const int64_t *offsets,
                               const int32_t *lengths, const float *consts, int64_t P,
                               int32_t dataset_id, const beagle_fit_config *cfg,
                               beagle_fit_result *fit_out, int32_t precision, void *stream) {
    if (!cfg) return fail(BEAGLE_ERR_ARG, "null fitness configuration");
    if (cfg->kind < BEAGLE_FIT_CORRELATION || cfg->kind > BEAGLE_FIT_VALIDATE)
        return fail(BEAGLE_ERR_ARG, "unknown fitness kind %d", cfg->kind);
    if (cfg->max_score < 1 || cfg->max_score > (1 << 22))
        return fail(BEAGLE_ERR_ARG, "max_score must be in [1, 2^22] (got %d)", cfg->max_score);
    auto ds = find_dataset(dataset_id);
    if (!ds) return fail(BEAGLE_ERR_DATASET, "unknown dataset %d", dataset_id);
    JobRequest req{programs, offsets, lengths, consts, P, dataset_id, nullptr, nullptr,
                   nullptr};
    req.kind = cfg->kind;
    req.max_score = cfg->max_score;
    req.tax = cfg->tax_per_token >= 0.0
                  ? cfg->tax_per_token
                  : static_cast<double>(cfg->max_score) * static_cast<double>(ds->N) / 85.0;
    req.fit = fit_out;
    return score_jobs(&req, 1, precision, static_cast<cudaStream_t>(stream), nullptr);
}

beagle_status beagle_eval(const uint8_t *programs, const int64_t *offsets,
                          const int32_t *lengths, const float *consts, int64_t P,
                          int32_t dataset_id, void *outputs, beagle_fitness *fitness_out,
                          int32_t precision, void *stream) {
    if (P > 0 && !outputs) return fail(BEAGLE_ERR_ARG, "outputs is null");
    JobRequest req{programs, offsets, lengths, consts, P, dataset_id, fitness_out, nullptr,
                   outputs};
    return score_jobs(&req, 1, precision, static_cast<cudaStream_t>(stream), nullptr);
}

beagle_status beagle_score_host(const uint8_t *programs, const int64_t *offsets,
                                const int32_t *lengths, const float *consts, int64_t P,
                                int64_t n_tokens, int32_t dataset_id,
                                beagle_fitness *fitness_out, int32_t precision, void *stream) {
    if (P < 0 || n_tokens < 0) return fail(BEAGLE_ERR_ARG, "negative size");
    if (P == 0) return BEAGLE_OK;
    if (!programs || !offsets || !lengths || !consts || !fitness_out)
        return fail(BEAGLE_ERR_ARG, "null pointer argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t b_ops = static_cast<size_t>(n_tokens), b_off = 8 * static_cast<size_t>(P),
                 b_len = 4 * static_cast<size_t>(P), b_cs = 4 * static_cast<size_t>(n_tokens),
                 b_out = sizeof(beagle_fitness) * static_cast<size_t>(P);
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t total = up(b_ops) + up(b_off) + up(b_len) + up(b_cs) + up(b_out);
    char *base = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&base), total, s);
    if (e != cudaSuccess) return fail(BEAGLE_ERR_OOM, "score_host: %s", cudaGetErrorString(e));
    char *d_ops = base, *d_off = d_ops + up(b_ops), *d_len = d_off + up(b_off),
         *d_cs = d_len + up(b_len), *d_out = d_cs + up(b_cs);
    e = cudaMemcpyAsync(d_ops, programs, b_ops, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, offsets, b_off, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_len, lengths, b_len, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_cs, consts, b_cs, cudaMemcpyHostToDevice, s);
    beagle_status st = BEAGLE_OK;
    if (e != cudaSuccess) st = cuda_fail(e, "score_host copy in");
    if (st == BEAGLE_OK)
        st = beagle_score(reinterpret_cast<uint8_t *>(d_ops), reinterpret_cast<int64_t *>(d_off),
                          reinterpret_cast<int32_t *>(d_len), reinterpret_cast<float *>(d_cs), P,
                          dataset_id, reinterpret_cast<beagle_fitness *>(d_out), precision, s);
    if (st == BEAGLE_OK) {
        e = cudaMemcpyAsync(fitness_out, d_out, b_out, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) st = cuda_fail(e, "score_host copy out");
    }
    cudaFreeAsync(base, s);
    e = cudaStreamSynchronize(s);
    if (st == BEAGLE_OK && e != cudaSuccess) st = cuda_fail(e, "score_host");
    return st;
}

}  // extern "C"
