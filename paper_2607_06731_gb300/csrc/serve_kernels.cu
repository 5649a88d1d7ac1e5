// Persistent serving kernel: continuous batching of scoring requests on the device.
//
// The scoring of a (program, case tile) unit is the one beagle_score runs (score_device.cuh:
// same packing, interpretation and tile statistics, same tile of 512 cases, the same fp64
// merge of the tiles in the same order), so a served program's fitness has the same bits as
// when it is scored alone. What differs is where the work comes from: producer warps claim
// items from a queue the host extends while the kernel runs (serve.cuh), and the per-program
// merge and the per-job completion are done in the kernel by the warp that finishes the last
// piece of work, so a small request that arrives while a large one runs is scored between
// the large one's items and completes first.
#include "registry.h"
#include "score_device.cuh"
#include "serve.cuh"

namespace beagle {
namespace {

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_sys(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.sys.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(int32_t *p, int v) {
    asm volatile("st.release.sys.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// The job's tensor map lives in global memory and was written by a copy before the job was
// published: order the tensor-map proxy's reads after that write.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *m) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
}

}  // namespace

template <typename T, int K>
__global__ void __launch_bounds__(KernelThreads<T, K, kDepthFast>::value, 1)
serve_kernel(const __grid_constant__ ServeParams prm) {
    constexpr int D = kDepthFast;
    extern __shared__ __align__(128) unsigned char smem[];
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
    }
    __syncthreads();
    uint32_t tstk = 0;
    if constexpr (kTmem) {
        tmem_fence_after_sync();
        tstk = *tmem_base + (static_cast<uint32_t>(warp & 3) << 21) +
               static_cast<uint32_t>((warp >> 2) * tmem_cols_per_warp(D, K));
    }

    if (warp == NW) {
        // Producer: claim the next item of the active jobs in turn (each job's own counter;
        // an exit leaves no claimed item behind), stage its tile, publish the slot. No work
        // for idle_limit_ns, or the host's stop flag with no work: exit.
        if (lane == 0) {
            int k = 0;
            unsigned rr = blockIdx.x;   // round-robin position over the active jobs
            for (;; ++k) {
                const int b = k & 1;
                if (k >= 2 && !mbar_wait(&empty[b], ((k >> 1) - 1) & 1, limit)) {
                    atomicOr(&prm.state->error, kErrTimeoutEmpty);
                    break;
                }
                Slot &s = slots[b];
                int job = -1;
                unsigned long long item = 0;
                const uint64_t t0 = global_ns();
                for (uint32_t spin = 0;; ++spin) {
                    const int nj = ld_acquire_sys(&prm.ctl->njobs);
                    const int lo = ld_acquire_sys(&prm.ctl->lo);
                    const int n = nj - lo;
                    for (int i = 0; i < n && job < 0; ++i) {
                        const int j = lo + static_cast<int>((rr + static_cast<unsigned>(i)) %
                                                            static_cast<unsigned>(n));
                        ServeJob &cj = prm.jobs[j];
                        const unsigned long long items =
                            static_cast<unsigned long long>(*reinterpret_cast<volatile const int64_t *>(&cj.items));
                        if (*reinterpret_cast<volatile unsigned long long *>(&cj.claimed) >= items)
                            continue;
                        const unsigned long long c = atomicAdd(&cj.claimed, 1ull);
                        if (c < items) {
                            job = j;
                            item = c;
                            rr += static_cast<unsigned>(i) + 1u;
                        }
                    }
                    if (job >= 0) break;
                    if (ld_acquire_sys(&prm.ctl->stop)) break;
                    if (global_ns() - t0 > prm.idle_limit_ns) break;
                    __nanosleep(spin < 64 ? 200 : 2000);
                }
                if (job < 0) {
                    s.job = -1;
                    mbar_arrive(&full[b]);
                    break;
                }
                ServeJob &SJ = prm.jobs[job];
                const int64_t local = static_cast<int64_t>(item);
                const int groups = static_cast<int>((SJ.dev.P + SJ.group - 1) / SJ.group);
                const int t = static_cast<int>(local / groups);
                const int g = static_cast<int>(local % groups);
                if (local == 0) SJ.counters[1] = global_ns();   // the job's first item
                s.job = job;
                s.tile = t;
                s.group = g;
                s.next = 0;
                const int rows = SJ.dev.rows;
                const int boxes = tile / kBox;
                const uint32_t bytes = static_cast<uint32_t>(boxes * rows * kBox * sizeof(float));
                tensormap_acquire(&SJ.map);
                mbar_arrive_expect_tx(&full[b], bytes);
                float *dst = xbuf + static_cast<size_t>(b) * prm.xbuf_floats;
                for (int q = 0; q < boxes; ++q)
                    tma_load_2d(dst + q * rows * kBox, &SJ.map, t * tile + q * kBox, 0, &full[b]);
            }
            if (k >= 1) (void)mbar_wait(&full[(k - 1) & 1], ((k - 1) >> 1) & 1, limit);
        }
        return;
    }

    // Consumers: score the programs of each staged item; the warp finishing a program's last
    // tile merges its tiles; the one finishing the job's last unit completes the job.
    T *fbuf = fbuf_all + static_cast<size_t>(warp) * tile;
    uint2 *pbuf = pbuf_all + static_cast<size_t>(warp) * (kMaxLen + 2);
    T *stk = stk_all + static_cast<size_t>(warp) * (Lay::stack_bytes_per_warp() / sizeof(T));
    for (int k = 0;; ++k) {
        const int b = k & 1;
        if (!mbar_wait(&full[b], (k >> 1) & 1, limit)) {
            if (lane == 0) atomicOr(&prm.state->error, kErrTimeoutFull);
            break;
        }
        const volatile Slot *vs = &slots[b];
        Slot s;
        s.job = vs->job;
        s.tile = vs->tile;
        s.group = vs->group;
        if (s.job < 0) break;
        ServeJob &SJ = prm.jobs[s.job];
        const JobDev &J = SJ.dev;
        const float *xs = xbuf + static_cast<size_t>(b) * prm.xbuf_floats;
        const int64_t p0 = static_cast<int64_t>(s.group) * SJ.group;
        const int64_t p1 = min(J.P, p0 + SJ.group);
        const unsigned long long units = static_cast<unsigned long long>(J.P) * J.tiles;
        for (;;) {
            int idx = 0;
            if (lane == 0) idx = atomicAdd(&slots[b].next, 1);
            idx = __shfl_sync(kFull, idx, 0);
            const int64_t q = p0 + idx;
            if (q >= p1) break;
            const int64_t p = J.order ? static_cast<int64_t>(J.order[q]) : q;
            const int deep = process_program<T, K, D>(J, q, p, s.tile, tile, xs, pbuf, fbuf, stk,
                                                      tstk, lane);
            // count the unit; the warp that completes the program's last tile merges them
            int last = 0;
            if (lane == 0) {
                __threadfence();   // this unit's partials before its count
                const int prev = atomicAdd(&SJ.tile_done[p], 1);
                last = (!deep && prev == J.tiles - 1) ? 1 : 0;
                if (last) __threadfence();
            }
            if (__shfl_sync(kFull, last, 0)) {
                __syncwarp();
                finalize_mse_program<sizeof(T) == 8>(J, p, tile, false, lane);
                __syncwarp();
            }
            if (lane == 0) {
                __threadfence();
                if (atomicAdd(&SJ.counters[0], 1ull) == units - 1) {
                    ServeDone *dn = SJ.done;
                    dn->t_start = SJ.counters[1];
                    dn->t_end = global_ns();
                    dn->deep = *reinterpret_cast<volatile int32_t *>(J.deep_count);
                    __threadfence_system();   // results and stamps before the flag
                    st_release_sys(&dn->state, 1);
                }
            }
            __syncwarp();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
    }
    if constexpr (kTmem) {
        tmem_fence_before_sync();
        asm volatile("bar.sync 1, %0;" ::"r"(NW * 32) : "memory");
        if (warp == 0) {
            tmem_fence_after_sync();
            tmem_dealloc(*tmem_base, tmem_columns(NW, D, K));
        }
    }
}

template <typename T, int K>
static cudaError_t launch_serve_impl(const ServeParams &prm, cudaStream_t s) {
    int nw = KernelThreads<T, K, kDepthFast>::value / 32 - 1;
    while (nw > 1 &&
           SmemLayout<T, K, kDepthFast>::total(prm.xbuf_floats, prm.tile, nw) > kSmemBudget)
        --nw;
    const size_t smem = one_cta_per_sm(SmemLayout<T, K, kDepthFast>::total(prm.xbuf_floats, prm.tile, nw));
    auto kern = serve_kernel<T, K>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<sm_count(), (nw + 1) * 32, smem, s>>>(prm);
    return cudaGetLastError();
}

cudaError_t launch_serve(const ServeParams &prm, int precision, cudaStream_t s) {
    if (precision == BEAGLE_FP64) return launch_serve_impl<double, kCasesFp64>(prm, s);
    return launch_serve_impl<float, kCasesFp32>(prm, s);
}

cudaError_t load_serve_kernels() {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, serve_kernel<float, kCasesFp32>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, serve_kernel<double, kCasesFp64>);
    return e;
}

}  // namespace beagle
