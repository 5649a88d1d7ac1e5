// Persistent scoring kernel and the fp64 finalize kernel (see score.cuh for the design).
#include <cstdio>

#include "score_device.cuh"

namespace beagle {
// Work layout of a launch, in shared memory: per job its first work item, programs to score
// and program groups; the launch's total items and programs per item. The fast pass copies
// them from the host's plan; the deep pass derives them from the deep-program counts the
// fast pass left in device memory (every CTA computes the same values).
template <int MAXJ>
struct WorkTable {
    int64_t item0[MAXJ];
    int64_t n[MAXJ];
    int32_t groups[MAXJ];
    int64_t total;
    int32_t group;
};

template <int MAXJ>
__device__ void build_work_table(const LaunchParams<MAXJ> &prm, WorkTable<MAXJ> &w) {
    int group = prm.group;
    if (prm.deep_pass) {
        int64_t work = 0;
        for (int j = 0; j < prm.njobs; ++j)
            work += static_cast<int64_t>(*prm.jobs[j].deep_count) * prm.jobs[j].tiles;
        const int64_t g = work / (32LL * gridDim.x);
        group = static_cast<int>(g < 1 ? 1 : (g > 256 ? 256 : g));
    }
    int64_t acc = 0;
    for (int j = 0; j < prm.njobs; ++j) {
        const JobDev &J = prm.jobs[j];
        const int64_t n = prm.deep_pass ? static_cast<int64_t>(*J.deep_count) : J.P;
        const int64_t groups = (n + group - 1) / group;
        w.item0[j] = acc;
        w.n[j] = n;
        w.groups[j] = static_cast<int32_t>(groups);
        acc += groups * J.tiles;
    }
    w.total = acc;
    w.group = group;
}

template <int MAXJ>
__device__ __forceinline__ int find_job(const WorkTable<MAXJ> &w, int njobs, int64_t item) {
    int j = 0;
    while (j + 1 < njobs && item >= w.item0[j + 1]) ++j;
    return j;
}

template <typename T, int K, int D, int MAXJ>
__global__ void __launch_bounds__(KernelThreads<T, K, D>::value, 1)
score_kernel(const __grid_constant__ LaunchParams<MAXJ> prm) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ WorkTable<MAXJ> work;
    using Lay = SmemLayout<T, K, D>;
    const int NW = static_cast<int>(blockDim.x / 32) - 1;   // consumer warps
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + 2;
    Slot *slots = reinterpret_cast<Slot *>(smem + 64);
    float *xbuf = reinterpret_cast<float *>(smem + Lay::xbuf_off());
    T *fbuf_all = reinterpret_cast<T *>(smem + Lay::fbuf_off(prm.xbuf_floats));
    uint2 *pbuf_all = reinterpret_cast<uint2 *>(smem + Lay::pbuf_off(prm.xbuf_floats, prm.tile, NW));
    T *stk_all = reinterpret_cast<T *>(smem + Lay::stack_off(prm.xbuf_floats, prm.tile, NW));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = prm.tile;
    const uint64_t limit = prm.wait_limit_ns ? prm.wait_limit_ns : kWaitLimitNs;
    constexpr bool kTmem = kTmemStackPath<T, K>;
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(smem + 32);
    if constexpr (kTmem) {
        if (warp == 0) tmem_alloc(tmem_base, tmem_columns(NW, D, K));
        tmem_fence_before_sync();
    }
    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&empty[0], NW);
        mbar_init(&empty[1], NW);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        build_work_table(prm, work);
    }
    __syncthreads();
    uint32_t tstk = 0;
    if constexpr (kTmem) {
        tmem_fence_after_sync();
        // lane quarter warp % 4 (TMEM lane field, bits 16-31), column slot warp / 4
        tstk = *tmem_base + (static_cast<uint32_t>(warp & 3) << 21) +
               static_cast<uint32_t>((warp >> 2) * tmem_cols_per_warp(D, K));
    }

    if (warp == NW) {
        // Producer: claim items, stage their X/y tile with TMA, publish the slot. (With the
        // test hook set it publishes nothing and issues no copy: the consumers' bounded waits
        // run out, set the error word and return.)
        if (lane == 0 && !prm.stall_producer) {
            int k = 0;
            for (;; ++k) {
                const int b = k & 1;
                if (k >= 2 && !mbar_wait(&empty[b], ((k >> 1) - 1) & 1, limit)) {
                    atomicOr(prm.error, kErrTimeoutEmpty);
                    break;
                }
                const int64_t item = static_cast<int64_t>(atomicAdd(prm.counter, 1u));
                Slot &s = slots[b];
                if (item >= work.total) {
                    s.job = -1;
                    mbar_arrive(&full[b]);
                    break;
                }
                const int j = find_job(work, prm.njobs, item);
                const JobDev &J = prm.jobs[j];
                const int64_t local = item - work.item0[j];
                const int t = static_cast<int>(local / work.groups[j]);
                const int g = static_cast<int>(local % work.groups[j]);
                s.job = j;
                s.tile = t;
                s.group = g;
                s.next = 0;
                const int boxes = tile / kBox;
                const uint32_t bytes = static_cast<uint32_t>(boxes * J.rows * kBox * sizeof(float));
                mbar_arrive_expect_tx(&full[b], bytes);
                float *dst = xbuf + static_cast<size_t>(b) * prm.xbuf_floats;
                for (int q = 0; q < boxes; ++q)
                    tma_load_2d(dst + q * J.rows * kBox, &prm.maps[j], t * tile + q * kBox, 0,
                                &full[b]);
            }
            // Let the copies this thread issued land before the CTA can exit: consumers
            // wait on every published slot, so only a timed-out run needs this wait.
            if (k >= 1) (void)mbar_wait(&full[(k - 1) & 1], ((k - 1) >> 1) & 1, limit);
        }
        return;
    }

    // Consumers
    T *fbuf = fbuf_all + static_cast<size_t>(warp) * tile;
    uint2 *pbuf = pbuf_all + static_cast<size_t>(warp) * (kMaxLen + 2);
    T *stk = stk_all + static_cast<size_t>(warp) * (Lay::stack_bytes_per_warp() / sizeof(T));
    for (int k = 0;; ++k) {
        const int b = k & 1;
        if (!mbar_wait(&full[b], (k >> 1) & 1, limit)) {
            if (lane == 0) atomicOr(prm.error, kErrTimeoutFull);
            break;
        }
        const volatile Slot *vs = &slots[b];
        Slot s;
        s.job = vs->job;
        s.tile = vs->tile;
        s.group = vs->group;
        if (s.job < 0) break;
        const JobDev &J = prm.jobs[s.job];
        const float *xs = xbuf + static_cast<size_t>(b) * prm.xbuf_floats;
        const int64_t p0 = static_cast<int64_t>(s.group) * work.group;
        const int64_t p1 = min(work.n[s.job], p0 + work.group);
        const int32_t *order = prm.deep_pass ? J.deep_list : J.order;
        for (;;) {
            int idx = 0;
            if (lane == 0) idx = atomicAdd(&slots[b].next, 1);
            idx = __shfl_sync(kFull, idx, 0);
            const int64_t q = p0 + idx;
            if (q >= p1) break;
            const int64_t p = order ? static_cast<int64_t>(order[q]) : q;
            process_program<T, K, D>(J, q, p, s.tile, tile, xs, pbuf, fbuf, stk, tstk, lane);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
    }
    if constexpr (kTmem) {
        // Every consumer warp gets here (the loop ends on the last slot or a timed-out wait);
        // the allocating warp frees the columns once all of them are done with TMEM.
        tmem_fence_before_sync();
        asm volatile("bar.sync 1, %0;" ::"r"(NW * 32) : "memory");
        if (warp == 0) {
            tmem_fence_after_sync();
            tmem_dealloc(*tmem_base, tmem_columns(NW, D, K));
        }
    }
}

// A group of finalize_group(tiles) lanes per program; blockIdx.x counts blocks of 256 groups'
// lanes (256 / g programs a block).
template <bool FP64, int MAXJ>
__global__ void finalize_kernel(const __grid_constant__ LaunchParams<MAXJ> prm) {
    const int jn = blockIdx.y;
    if (jn >= prm.njobs) return;
    const JobDev &J = prm.jobs[jn];
    if (J.kind != kFitMse) return;
    const int g = finalize_group(J.tiles);
    const int64_t p = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / g;
    // whole warps leave together (the group sums shuffle over the warp)
    const int64_t pw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31)) / g;
    if (pw >= J.P) return;
    finalize_mse_program<FP64>(J, p < J.P ? p : J.P - 1, prm.tile, *prm.error != 0u,
                               threadIdx.x & 31);
}

template <bool FP64, int MAXJ>
__global__ void fit_finalize_kernel(const __grid_constant__ LaunchParams<MAXJ> prm) {
    const int jn = blockIdx.y;
    if (jn >= prm.njobs) return;
    const JobDev &J = prm.jobs[jn];
    if (J.kind == kFitMse) return;
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= J.P) return;
    finalize_fit_program<FP64>(J, p, *prm.error != 0u);
}

// --------------------------------------------------------------------------- launchers
// Consumer warps of a kernel variant whose shared memory fits (nw_cap: the caller's bound).
template <typename T, int K, int D>
static int fit_warps(int xbuf_floats, int tile, int nw_cap) {
    int nw = KernelThreads<T, K, D>::value / 32 - 1;
    if (nw_cap > 0 && nw_cap < nw) nw = nw_cap;
    while (nw > 1 && SmemLayout<T, K, D>::total(xbuf_floats, tile, nw) > kSmemBudget) --nw;
    return nw;
}

template <typename T, int K, int D, int MAXJ>
static cudaError_t launch_pass(const LaunchParams<MAXJ> &prm, int nw, int grid,
                               cudaStream_t stream) {
    const size_t smem = one_cta_per_sm(SmemLayout<T, K, D>::total(prm.xbuf_floats, prm.tile, nw));
    auto kern = score_kernel<T, K, D, MAXJ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, (nw + 1) * 32, smem, stream>>>(prm);
    return cudaGetLastError();
}

// One scoring call: the fast pass (16-value stack) over every program, then -- when the jobs
// carry deep lists -- the deep pass (32-value stack; the 4-case path on FP32, whatever cases
// per lane the fast pass used: every path gives the same bits at a given tile) over the
// programs the fast pass found deeper, then the finalize kernels.
template <typename T, int K, int MAXJ>
static cudaError_t launch_impl(const LaunchParams<MAXJ> &prm, int nw, int grid,
                               cudaStream_t stream) {
    void *tok = nullptr;
    const bool timed = timing_enabled();
    if (timed) timing_begin(stream, &tok);
    cudaError_t e = launch_pass<T, K, kDepthFast, MAXJ>(prm, nw, grid, stream);
    bool deep = false;
    for (int j = 0; j < prm.njobs; ++j) deep |= prm.jobs[j].deep_list != nullptr;
    if (e == cudaSuccess && deep) {
        constexpr int KD = sizeof(T) == 4 ? 4 : K;
        LaunchParams<MAXJ> dp = prm;
        dp.deep_pass = 1;
        dp.counter = prm.counter + 1;   // the deep pass's own work counter (zeroed too)
        const int nwd = fit_warps<T, KD, kMaxDepth>(prm.xbuf_floats, prm.tile, 0);
        e = launch_pass<T, KD, kMaxDepth, MAXJ>(dp, nwd, grid, stream);
    }
    if (timed) timing_end(stream, tok);
    if (e != cudaSuccess) return e;
    int64_t maxP = 0;
    bool mse = false, fit = false;
    for (int j = 0; j < prm.njobs; ++j) {
        maxP = maxP > prm.jobs[j].P ? maxP : prm.jobs[j].P;
        (prm.jobs[j].kind == kFitMse ? mse : fit) = true;
    }
    if (maxP > 0) {
        dim3 fg(static_cast<unsigned>((maxP + 255) / 256), static_cast<unsigned>(prm.njobs));
        if (mse) {
            int gmax = 1;
            for (int j = 0; j < prm.njobs; ++j) gmax = max(gmax, finalize_group(prm.jobs[j].tiles));
            const dim3 fw(static_cast<unsigned>((maxP * gmax + 255) / 256), static_cast<unsigned>(prm.njobs));
            if (sizeof(T) == 8) finalize_kernel<true, MAXJ><<<fw, 256, 0, stream>>>(prm);
            else finalize_kernel<false, MAXJ><<<fw, 256, 0, stream>>>(prm);
            e = cudaGetLastError();
        }
        if (fit && e == cudaSuccess) {
            if (sizeof(T) == 8) fit_finalize_kernel<true, MAXJ><<<fg, 256, 0, stream>>>(prm);
            else fit_finalize_kernel<false, MAXJ><<<fg, 256, 0, stream>>>(prm);
            e = cudaGetLastError();
        }
    }
    return e;
}

size_t smem_bytes(int precision, int cases, int xbuf_floats, int tile, int nw) {
    if (precision == BEAGLE_FP64)
        return SmemLayout<double, kCasesFp64, kDepthFast>::total(xbuf_floats, tile, nw);
    switch (cases) {
    case 2: return SmemLayout<float, 2, kDepthFast>::total(xbuf_floats, tile, nw);
    case 8: return SmemLayout<float, 8, kDepthFast>::total(xbuf_floats, tile, nw);
    default: return SmemLayout<float, 4, kDepthFast>::total(xbuf_floats, tile, nw);
    }
}

int plan_warps(int precision, int cases, int xbuf_floats, int tile) {
    if (precision == BEAGLE_FP64)
        return fit_warps<double, kCasesFp64, kDepthFast>(xbuf_floats, tile, 0);
    switch (cases) {
    case 2: return fit_warps<float, 2, kDepthFast>(xbuf_floats, tile, 0);
    case 8: return fit_warps<float, 8, kDepthFast>(xbuf_floats, tile, 0);
    default: return fit_warps<float, 4, kDepthFast>(xbuf_floats, tile, 0);
    }
}

static int sm_count_dev() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

template <int MAXJ>
static cudaError_t launch_any(const LaunchParams<MAXJ> &prm, int precision, int cases, int nw,
                              int grid, cudaStream_t s) {
    if (precision == BEAGLE_FP64)
        return launch_impl<double, kCasesFp64, MAXJ>(prm, nw, grid, s);
    switch (cases) {
    case 2: return launch_impl<float, 2, MAXJ>(prm, nw, grid, s);
    case 8: return launch_impl<float, 8, MAXJ>(prm, nw, grid, s);
    default: return launch_impl<float, 4, MAXJ>(prm, nw, grid, s);
    }
}

template <typename T, int K, int MAXJ>
static cudaError_t load_one() {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, score_kernel<T, K, kDepthFast, MAXJ>);
    if (e == cudaSuccess)
        e = cudaFuncGetAttributes(&a, score_kernel<T, sizeof(T) == 4 ? 4 : K, kMaxDepth, MAXJ>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, finalize_kernel<sizeof(T) == 8, MAXJ>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, fit_finalize_kernel<sizeof(T) == 8, MAXJ>);
    return e;
}

cudaError_t load_kernels() {
    cudaError_t e = cudaSuccess;
    for (cudaError_t r : {load_one<float, 2, 1>(), load_one<float, 4, 1>(), load_one<float, 8, 1>(),
                          load_one<double, kCasesFp64, 1>(), load_one<float, 2, kMaxJobs>(),
                          load_one<float, 4, kMaxJobs>(), load_one<float, 8, kMaxJobs>(),
                          load_one<double, kCasesFp64, kMaxJobs>()})
        if (r != cudaSuccess) e = r;
    return e;
}

cudaError_t launch_score(const LaunchParams<1> &prm, int precision, int cases, int nw, int grid,
                         cudaStream_t s) {
    return launch_any<1>(prm, precision, cases, nw, grid, s);
}

cudaError_t launch_deep_and_finalize(const LaunchParams<1> &prm, int precision, cudaStream_t s) {
    LaunchParams<1> dp = prm;
    dp.deep_pass = 1;
    cudaError_t e;
    if (precision == BEAGLE_FP64) {
        const int nw = fit_warps<double, kCasesFp64, kMaxDepth>(prm.xbuf_floats, prm.tile, 0);
        e = launch_pass<double, kCasesFp64, kMaxDepth, 1>(dp, nw, sm_count_dev(), s);
        if (e == cudaSuccess) finalize_kernel<true, 1><<<dim3(static_cast<unsigned>((prm.jobs[0].P * finalize_group(prm.jobs[0].tiles) + 255) / 256), 1), 256, 0, s>>>(prm);
    } else {
        const int nw = fit_warps<float, 4, kMaxDepth>(prm.xbuf_floats, prm.tile, 0);
        e = launch_pass<float, 4, kMaxDepth, 1>(dp, nw, sm_count_dev(), s);
        if (e == cudaSuccess) finalize_kernel<false, 1><<<dim3(static_cast<unsigned>((prm.jobs[0].P * finalize_group(prm.jobs[0].tiles) + 255) / 256), 1), 256, 0, s>>>(prm);
    }
    return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t launch_score_batch(const LaunchParams<kMaxJobs> &prm, int precision, int cases,
                               int nw, int grid, cudaStream_t s) {
    return launch_any<kMaxJobs>(prm, precision, cases, nw, grid, s);
}

}  // namespace beagle
