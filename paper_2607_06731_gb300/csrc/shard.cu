// Population sharding by cost for several GPUs ("Hardware Optimized"): contiguous ranges of
// programs whose summed lengths are nearly equal (host code).
#include <vector>

#include "registry.h"

using namespace beagle;

extern "C" beagle_status beagle_shard_by_cost(const int32_t *lengths, int64_t P, int32_t n_shards,
                                              int64_t *bounds_out) {
    if (P < 0 || n_shards < 1 || !bounds_out || (P > 0 && !lengths))
        return fail(BEAGLE_ERR_ARG, "bad arguments");
    int64_t total = 0;
    for (int64_t p = 0; p < P; ++p) {
        if (lengths[p] < 0) return fail(BEAGLE_ERR_ARG, "negative length at %lld", (long long)p);
        total += lengths[p];
    }
    // shard k ends at the first program whose prefix cost reaches (k + 1) total / n_shards
    bounds_out[0] = 0;
    int64_t p = 0, acc = 0;
    for (int32_t k = 1; k < n_shards; ++k) {
        const long double target = static_cast<long double>(total) * k / n_shards;
        while (p < P && static_cast<long double>(acc) + lengths[p] / 2.0L <= target) acc += lengths[p++];
        bounds_out[k] = p;
    }
    bounds_out[n_shards] = P;
    return BEAGLE_OK;
}
