// beagle_score_static: scoring that allocates no device memory.
//
// Some callers cannot allocate device memory while they score: a loop that must never
// block on the device (cudaMalloc and cudaFree may synchronise it), a process that reserves
// its whole device-memory budget up front, or code that runs while another component owns
// the allocator. For them the scoring kernel's scratch (work counter, error word and the
// per-(program, tile) partial sums) lives in a fixed array compiled into this library.
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "kernels.h"
#include "registry.h"

namespace beagle {
namespace {

// Held on every device that loads this part of the library, until the process exits.
__device__ __align__(256) unsigned char g_static_scratch[BEAGLE_STATIC_SCRATCH_BYTES];

std::mutex g_static_mu;
std::unordered_map<int, char *> g_static_addr;   // device ordinal -> device address

// Device address of g_static_scratch on device dev (which must be current). In host code
// the array's name is only a host-side stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress and cached.
beagle_status static_scratch_address(int dev, char **out) {
    std::lock_guard<std::mutex> lk(g_static_mu);
    auto it = g_static_addr.find(dev);
    if (it != g_static_addr.end()) {
        *out = it->second;
        return BEAGLE_OK;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "static scratch: cudaGetSymbolAddress");
    g_static_addr[dev] = static_cast<char *>(p);
    *out = static_cast<char *>(p);
    return BEAGLE_OK;
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace beagle

using namespace beagle;

extern "C" beagle_status beagle_score_static(const uint8_t *programs, const int64_t *offsets,
                                             const int32_t *lengths, const float *consts,
                                             int64_t P, int32_t dataset_id,
                                             beagle_fitness *fitness_out, int32_t precision,
                                             void *stream) {
    if (precision != BEAGLE_FP32_COMPENSATED && precision != BEAGLE_FP64)
        return fail(BEAGLE_ERR_ARG, "unknown precision %d", precision);
    if (P < 0) return fail(BEAGLE_ERR_ARG, "negative P");
    auto ds = find_dataset(dataset_id);
    if (!ds) return fail(BEAGLE_ERR_DATASET, "unknown dataset %d", dataset_id);
    int dev = 0;
    cudaGetDevice(&dev);
    if (ds->device != dev)
        return fail(BEAGLE_ERR_DATASET, "dataset %d lives on device %d, current is %d",
                    dataset_id, ds->device, dev);
    if (P == 0) return BEAGLE_OK;
    if (!programs || !offsets || !lengths || !consts || !fitness_out)
        return fail(BEAGLE_ERR_ARG, "null pointer argument");

    // A fixed launch shape, whatever beagle_set_launch_config or the autotuner chose: tiles
    // of 512 cases, 4 cases per lane on the FP32 path, as many consumer warps as shared
    // memory allows, programs in the caller's order (the length-bucketed order would need
    // scratch of its own). beagle_score with its automatic shape gives the same bits.
    if (P > (int64_t(1) << 31) - 1) return fail(BEAGLE_ERR_LIMIT, "P >= 2^31");
    const int tile = tile_for(precision, kCasesFp32, 512);
    const int64_t tiles = (ds->N + tile - 1) / tile;
    // 44 bytes per program and tile plus 4 per program (the list of programs deeper than the
    // fast pass's stack) after a 512-byte header; compared without forming the product,
    // which could wrap for huge P.
    const int64_t per_program = static_cast<int64_t>(kNumFields) * 4 * tiles + 4;
    const int64_t max_programs =
        (static_cast<int64_t>(BEAGLE_STATIC_SCRATCH_BYTES) - static_cast<int64_t>(kHdrBytes) -
         512) / per_program;
    if (P > max_programs)
        return fail(BEAGLE_ERR_LIMIT,
                    "static scratch holds at most %lld programs on %lld tiles of %d cases "
                    "(44 bytes per program and tile and 4 per program, limit %u bytes); got "
                    "P = %lld", (long long)max_programs, (long long)tiles, tile,
                    (unsigned)BEAGLE_STATIC_SCRATCH_BYTES, (long long)P);
    char *base = nullptr;
    beagle_status st = static_scratch_address(dev, &base);
    if (st != BEAGLE_OK) return st;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The array keeps the previous call's contents: the counters, error word and deep count
    // must start at zero (the partials and the deep list are written before they are read).
    cudaError_t e = cudaMemsetAsync(base, 0, kHdrBytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "static scratch: memset");

    const int grid = sm_count();
    const int64_t work = P * tiles;   // P < 2^31 and tiles < 2^22: no overflow
    const int xbuf_floats = ds->rows * tile;
    const int nw = plan_warps(precision, kCasesFp32, xbuf_floats, tile);
    if (nw < 1 || smem_bytes(precision, kCasesFp32, xbuf_floats, tile, nw) > kSmemBudget)
        return fail(BEAGLE_ERR_LIMIT, "shared memory plan exceeds %zu bytes", kSmemBudget);
    const int group = plan_group(work, nw, grid);

    LaunchParams<1> prm;
    std::memset(&prm, 0, sizeof prm);
    prm.maps[0] = ds->map;
    JobDev &J = prm.jobs[0];
    J.ops = programs;
    J.offs = offsets;
    J.lens = lengths;
    J.consts = consts;
    J.out = fitness_out;
    const size_t part_bytes = static_cast<size_t>(kNumFields) * 4 * tiles * P;
    J.partials = reinterpret_cast<uint32_t *>(base + kHdrBytes);
    J.deep_list = reinterpret_cast<int32_t *>(base + kHdrBytes + round256(part_bytes));
    J.deep_count = reinterpret_cast<int32_t *>(base + kHdrDeep);
    J.tile_sy = precision == BEAGLE_FP64 ? ds->tile_sy64[tile == 512 ? 0 : 1]
                                         : ds->tile_sy[tile == 512 ? 0 : 1];
    J.order = nullptr;
    J.fout = nullptr;
    J.P = P;
    J.N = ds->N;
    J.item0 = 0;
    J.d = ds->d;
    J.rows = ds->rows;
    J.tiles = static_cast<int32_t>(tiles);
    J.groups = static_cast<int32_t>((P + group - 1) / group);
    J.ybar = ds->ybar;
    J.syy = precision == BEAGLE_FP64 ? ds->syy : ds->syy32;
    prm.total_items = static_cast<int64_t>(J.groups) * tiles;
    prm.counter = reinterpret_cast<unsigned int *>(base + kHdrCounter);
    prm.error = reinterpret_cast<unsigned int *>(base + kHdrError);
    prm.njobs = 1;
    prm.tile = tile;
    prm.group = group;
    prm.xbuf_floats = xbuf_floats;
    apply_wait_settings(&prm.wait_limit_ns, &prm.stall_producer);
    e = launch_score(prm, precision, kCasesFp32, nw, grid, s);
    if (e != cudaSuccess) return cuda_fail(e, "static scoring launch");
    return BEAGLE_OK;
}
