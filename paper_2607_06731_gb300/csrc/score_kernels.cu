// Persistent scoring kernel and the fp64 finalize kernel (see score.cuh for the design).
#include <cstdio>

#include "interp_ptx.cuh"
#include "interp_ptx8.cuh"
#include "kernels.h"
#include "score.cuh"

namespace beagle {

// Shared-memory layout of one CTA (dynamic), nw consumer warps:
//   [0, 64)        mbarriers: full[2], empty[2]
//   [64, 128)      slot descriptors (2 x Slot)
//   [128, ...)     X stage buffers: 2 x xbuf_floats fp32 (TMA destinations, 128-byte aligned)
//   ...            per-warp output buffers: nw x tile x T (none on the 8-case FP32 path)
//   ...            per-warp packed programs: nw x (kMaxLen + 2) x uint2
//   ...            per-warp value stacks: nw x (kMaxDepth - 1) rows x 32 K x T
struct Slot {
    int job;        // -1: no more work
    int tile;
    int group;
    int next;       // next program of the item (shared-memory counter)
};

// Tensor memory (TMEM): allocation of ncols columns (a power of two, 32..512) by one whole
// warp, the base address written to *dst in shared memory; the same warp frees it. The fences
// order TMEM accesses around the CTA barriers that publish the address and end its use.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_addr(dst)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// The 4-case FP32 path keeps its stack rows in tensor memory (64 columns a warp, the warp's
// 32-lane quarter of TMEM being warp % 4 and its column slot warp / 4); the other paths keep
// them in shared memory.
template <typename T, int K>
constexpr bool kTmemStackPath = sizeof(T) == 4 && K == 4;
constexpr int kTmemColsPerWarp = 64;
static_assert(4 * (kMaxDepth - 1) <= kTmemColsPerWarp, "a warp's stack rows fit its columns");
__host__ __device__ constexpr uint32_t tmem_columns(int nw) {   // power of two, 32..512
    const int need = (nw + 3) / 4 * kTmemColsPerWarp;
    return need <= 32 ? 32u : need <= 64 ? 64u : need <= 128 ? 128u : need <= 256 ? 256u : 512u;
}

template <typename T, int K>
struct SmemLayout {
    static constexpr size_t kStackRows = kMaxDepth - 1;
    static constexpr bool kTmemStack = kTmemStackPath<T, K>;
    static __host__ __device__ size_t xbuf_off() { return 128; }
    static __host__ __device__ size_t fbuf_off(int xbuf_floats) {
        return xbuf_off() + 2ull * xbuf_floats * sizeof(float);
    }
    static __host__ __device__ size_t pbuf_off(int xbuf_floats, int tile, int nw) {
        return fbuf_off(xbuf_floats) +
               (sizeof(T) == 4 && K == 8 ? 0 : static_cast<size_t>(nw) * tile * sizeof(T));
    }
    static __host__ __device__ size_t stack_off(int xbuf_floats, int tile, int nw) {
        return pbuf_off(xbuf_floats, tile, nw) + static_cast<size_t>(nw) * (kMaxLen + 2) * sizeof(uint2);
    }
    static __host__ __device__ size_t stack_bytes_per_warp() {
        return kTmemStack ? 0 : kStackRows * 32 * K * sizeof(T);
    }
    static __host__ __device__ size_t total(int xbuf_floats, int tile, int nw) {
        return stack_off(xbuf_floats, tile, nw) + static_cast<size_t>(nw) * stack_bytes_per_warp();
    }
};

// The 8-case FP32 path runs one 256-case tile per pass and keeps the outputs in registers;
// the other paths write them to the warp's shared-memory buffer.
template <typename T, int K>
constexpr bool kOutputsInRegs = sizeof(T) == 4 && K == 8;

// A tile's outputs in the order the statistics read them: lane l's values are the cases
// 128 h + 4 l + j (h over the tile's 128-case halves, j = 0..3), the order in which the 8-case
// path holds them, so every path forms the same sums in the same order.
template <typename T, int K>
struct TileValues {
    T r[kOutputsInRegs<T, K> ? 8 : 1];
    const T *buf;
    // values 4h..4h+3 of this lane (h a compile-time index on the register path)
    __device__ __forceinline__ void get4(int h, int lane, T (&v)[4]) const {
        if constexpr (kOutputsInRegs<T, K>) {
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = r[4 * h + j];
        } else if constexpr (sizeof(T) == 4) {
            const float4 q = *reinterpret_cast<const float4 *>(buf + h * 128 + lane * 4);
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else {
            const double2 *src = reinterpret_cast<const double2 *>(buf + h * 128 + lane * 4);
            const double2 a = src[0], b = src[1];
            v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
        }
    }
    // f(h, v) for every 128-case half of the tile that holds cases
    template <typename F>
    __device__ __forceinline__ void for_halves(int halves, int lane, F &&f) const {
        if constexpr (kOutputsInRegs<T, K>) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h < halves) {
                    T v[4];
                    get4(h, lane, v);
                    f(h, v);
                }
            }
        } else {
#pragma unroll 1
            for (int h = 0; h < halves; ++h) {
                T v[4];
                get4(h, lane, v);
                f(h, v);
            }
        }
    }
};

template <typename T, int K, int D>
__device__ __forceinline__ void process_program(const JobDev &J, int64_t p, int t, int tile,
                                                const float *xs, uint2 *pbuf, T *fbuf, T *stk,
                                                uint32_t tstk, int lane) {
    using Sum = typename SumOf<T>::type;
    constexpr bool kRegs = kOutputsInRegs<T, K>;
    constexpr int CH = 32 * K;
    const int64_t off = J.offs[p];
    const int L = J.lens[p];
    const Packed pk = pack_program<T, D>(J.ops + off, J.consts + off, L, J.d, pbuf, lane);
    if constexpr (sizeof(T) == 4 && K == 4) {
        // Bits 24-28 of each token: the handler id of the token after it (the 4-case
        // interpreter branches on it while it loads that token). Each round reads, then writes.
        for (int base = 0; base < pk.n; base += 32) {
            const int i = base + lane;
            const uint32_t nh = i < pk.n ? (pbuf[i + 1].x & 31u) : 0u;
            __syncwarp();
            if (i < pk.n) pbuf[i].x |= nh << 24;
            __syncwarp();
        }
    }

    const int64_t P = J.P;
    const int tiles = J.tiles;
    uint32_t *part = J.partials;
    auto field = [&](int f) -> uint32_t * {
        return part + (static_cast<int64_t>(f) * tiles + t) * P + p;
    };
    if (pk.malformed) {
        if (lane == 0) *field(kTileFlags) = TF_MALFORMED;
        return;
    }
    const int64_t tstart = static_cast<int64_t>(t) * tile;
    const int nval = static_cast<int>(min(static_cast<int64_t>(tile), J.N - tstart));
    const int rows = J.rows;

    TileValues<T, K> vals;
    vals.buf = fbuf;
    bool anybad = pk.const_bad;
    if constexpr (kRegs) {   // one pass: the whole 256-case tile
        bool bad[8];
        run_program_ptx8(smem_addr(pbuf), smem_addr(xs + lane * 4), smem_addr(stk + lane * 4),
                         vals.r, bad);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (bad[j] && (j >> 2) * 128 + lane * 4 + (j & 3) < nval) anybad = true;
    } else {
        for (int c0 = 0; c0 < nval; c0 += CH) {
            const float *xrow = xs + (c0 / kBox) * rows * kBox + (c0 % kBox) + lane * K;
            T f[K];
            bool bad[K];
            if constexpr (sizeof(T) == 4 && K == 4)
                run_program_ptx4(smem_addr(pbuf), smem_addr(xrow), tstk, f, bad);
            else
                run_program<T, K>(smem_addr(pbuf), pk.n, smem_addr(xrow),
                                  smem_addr(stk + lane * K), f, bad);
            sts_vec<T, K>(smem_addr(fbuf + c0 + lane * K), f);
#pragma unroll
            for (int j = 0; j < K; ++j)
                if (bad[j] && c0 + lane * K + j < nval) anybad = true;
        }
    }
    anybad = __any_sync(kFull, anybad);
    __syncwarp();
    const int halves = (nval + 127) / 128;
    if (J.fout) {   // per-case outputs requested (beagle_eval)
        T *dst = static_cast<T *>(J.fout) + p * J.N + tstart;
        vals.for_halves(halves, lane, [&](int h, const T (&v)[4]) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = h * 128 + lane * 4 + j;
                if (i < nval) dst[i] = v[j];
            }
        });
    }
    if (anybad) {
        if (lane == 0) *field(kTileFlags) = TF_INVALID;
        return;
    }

    // Tile statistics. Lane l's targets for half h are 4 consecutive floats. The general form
    // (FP64 path; FP32 when the one-pass sums overflow) takes two passes over the tile's
    // outputs: the tile mean first, then sums centred on it. Valid values reach 1e30, so on the
    // FP32 path each sum is taken over terms scaled by an exact power of two 2^-k (k = 0 unless
    // the tile holds values above 2^50); the finalize kernel multiplies back in fp64.
    const float *yrow = xs + J.d * kBox;          // target row
    const float *ycrow = xs + (J.d + 1) * kBox;   // centred-target row
    auto row4 = [&](const float *row, int h) {
        const int i = h * 128 + lane * 4;
        return *reinterpret_cast<const float4 *>(row + (i / kBox) * rows * kBox + (i % kBox));
    };
    auto elem = [](const float4 &v, int j) {
        return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
    };
    if constexpr (sizeof(T) == 4) {
        // One pass, around the mean m0 of the tile's first 128 outputs: the finalize merge
        // cancels about as little around m0 as around the tile mean. sum e^2 has positive terms
        // only and is a plain fp32 sum (relative error below 22 u: 16 terms a lane, then 5
        // pairwise steps); the centred sums are compensated. An overflow anywhere in these
        // unscaled sums leaves an infinity or a NaN in them; then the two-pass form below,
        // which scales the terms, runs instead (outputs or targets near 2^60 and above). The
        // outputs are all equal exactly when the sum of |f - f_0| is 0 (no flush to zero).
        float h0[4];
        vals.get4(0, lane, h0);
        const int n0 = min(nval, 128);
        float s0 = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (lane * 4 + j < n0) s0 += h0[j];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s0 += __shfl_xor_sync(kFull, s0, o);
        const float m0 = s0 / static_cast<float>(n0);
        const float fa = __shfl_sync(kFull, h0[0], 0);
        float se1 = 0.0f, ad = 0.0f;
        KahanF sd1, sdd1, sdy1;
        vals.for_halves(halves, lane, [&](int h, const T (&v)[4]) {
            const float4 y4 = row4(yrow, h);
            const float4 yc4 = row4(ycrow, h);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (h * 128 + lane * 4 + j < nval) {
                    const float fi = v[j];
                    const float e = fi - elem(y4, j);
                    se1 = fmaf(e, e, se1);
                    ad += fabsf(fi - fa);
                    const float dv = fi - m0;
                    sd1.add(dv);
                    sdd1.add_prod(dv, dv);
                    sdy1.add_prod(dv, elem(yc4, j));
                }
            }
        });
        const bool nc = __any_sync(kFull, ad != 0.0f);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) se1 += __shfl_xor_sync(kFull, se1, o);
        if (nc) {
            sd1.warp_allreduce();
            sdd1.warp_allreduce();
            sdy1.warp_allreduce();
        } else {
            sd1 = KahanF();
            sdd1 = KahanF();
            sdy1 = KahanF();
        }
        // Identical on every lane (the reductions are symmetric), so the branch is uniform.
        const float chk = se1 + (sd1.s + sd1.c) + (sdd1.s + sdd1.c) + (sdy1.s + sdy1.c);
        if (isfinite(chk)) {
            if (lane == 0) {
                uint32_t w[kNumFields];
                w[kMean] = __float_as_uint(nc ? m0 : fa);
                w[kMean64] = 0u;
                w[kSe2] = __float_as_uint(se1);
                w[kSe2 + 1] = 0u;
                put_pair(w + kSd, sd1);
                put_pair(w + kSdd, sdd1);
                put_pair(w + kSdy, sdy1);
                w[kTileFlags] = nc ? TF_NONCONST : 0u;
#pragma unroll
                for (int f = 0; f < kNumFields; ++f) *field(f) = w[f];
            }
            __syncwarp();
            return;
        }
    }
    T v0[4];
    vals.get4(0, 0, v0);
    const T f0 = __shfl_sync(kFull, v0[0], 0);
    Sum sf;
    bool nonconst = false;
    float emax = 0.0f, fmax_ = 0.0f, ymax = 0.0f;
    vals.for_halves(halves, lane, [&](int h, const T (&v)[4]) {
        const float4 y4 = row4(yrow, h);
        const float4 yc4 = row4(ycrow, h);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (h * 128 + lane * 4 + j < nval) {
                const T fi = v[j];
                sf.add(fi);
                nonconst |= (fi != f0);
                if constexpr (sizeof(T) == 4) {
                    emax = fmaxf(emax, fabsf(fi - elem(y4, j)));
                    fmax_ = fmaxf(fmax_, fabsf(fi));
                    ymax = fmaxf(ymax, fabsf(elem(yc4, j)));
                }
            }
        }
    });
    nonconst = __any_sync(kFull, nonconst);
    sf.warp_allreduce();
    int ke = 0, kd = 0, ky = 0;
    T se_scale = T(1), sd_scale = T(1), sy_scale = T(1);
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            emax = fmaxf(emax, __shfl_xor_sync(kFull, emax, o));
            fmax_ = fmaxf(fmax_, __shfl_xor_sync(kFull, fmax_, o));
            ymax = fmaxf(ymax, __shfl_xor_sync(kFull, ymax, o));
        }
        ke = scale_exponent(emax);
        kd = scale_exponent(2.0f * fmax_);
        ky = scale_exponent(ymax);
        se_scale = pow2f(-ke);
        sd_scale = pow2f(-kd);
        sy_scale = pow2f(-ky);
    }
    T m;
    if constexpr (sizeof(T) == 4) m = nonconst ? (sf.s + sf.c) / static_cast<float>(nval) : f0;
    else m = nonconst ? sf.s / static_cast<double>(nval) : f0;
    Sum se, sd, sdd, sdy;
    vals.for_halves(halves, lane, [&](int h, const T (&v)[4]) {
        const float4 y4 = row4(yrow, h);
        const float4 yc4 = row4(ycrow, h);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (h * 128 + lane * 4 + j < nval) {
                const T fi = v[j];
                const T e = (fi - static_cast<T>(elem(y4, j))) * se_scale;
                se.add_prod(e, e);
                if (nonconst) {
                    const T dv = (fi - m) * sd_scale;
                    sd.add(dv);
                    sdd.add_prod(dv, dv);
                    // FP32: the stored fp32 y - ybar; FP64: y - ybar formed in fp64.
                    const T yc = sizeof(T) == 4 ? static_cast<T>(elem(yc4, j))
                                                : static_cast<T>(elem(y4, j)) -
                                                      static_cast<T>(J.ybar);
                    sdy.add_prod(dv, yc * sy_scale);
                }
            }
        }
    });
    se.warp_allreduce();
    if (nonconst) {
        sd.warp_allreduce();
        sdd.warp_allreduce();
        sdy.warp_allreduce();
    }
    if (lane == 0) {
        uint32_t w[kNumFields];
        if constexpr (sizeof(T) == 4) {
            w[kMean] = __float_as_uint(m);
            w[kMean64] = 0u;
        } else {
            const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(m));
            w[kMean] = static_cast<uint32_t>(b);
            w[kMean64] = static_cast<uint32_t>(b >> 32);
        }
        put_pair(w + kSe2, se);
        put_pair(w + kSd, sd);
        put_pair(w + kSdd, sdd);
        put_pair(w + kSdy, sdy);
        w[kTileFlags] = (nonconst ? TF_NONCONST : 0u) | (static_cast<uint32_t>(ke) << 8) |
                        (static_cast<uint32_t>(kd) << 16) | (static_cast<uint32_t>(ky) << 24);
#pragma unroll
        for (int f = 0; f < kNumFields; ++f) *field(f) = w[f];
    }
    __syncwarp();
}

template <int MAXJ>
__device__ __forceinline__ int find_job(const LaunchParams<MAXJ> &prm, int64_t item) {
    int j = 0;
    while (j + 1 < prm.njobs && item >= prm.jobs[j + 1].item0) ++j;
    return j;
}

// Threads per CTA the kernel is compiled for (the register budget per thread follows from it).
// The 4-case FP32 path, its stack in tensor memory, gets 32 warps (64 registers a thread):
// more resident warps hide more of the dispatch latency (C2 population: 17 consumer warps
// 2,304 GPoPs, 27 at 72 registers 2,656, 31 at 64 registers 2,738); the 2-case path also
// fits 32 warps; the 8-case and FP64 paths get 16 warps (128 registers).
template <typename T, int K>
struct KernelThreads {
    static constexpr int value = sizeof(T) != 4 ? 512 : K == 2 ? 1024 : K == 4 ? 1024 : 512;
};

template <typename T, int K, int D, int MAXJ>
__global__ void __launch_bounds__(KernelThreads<T, K>::value, 1)
score_kernel(const __grid_constant__ LaunchParams<MAXJ> prm) {
    extern __shared__ __align__(128) unsigned char smem[];
    using Lay = SmemLayout<T, K>;
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
        if (warp == 0) tmem_alloc(tmem_base, tmem_columns(NW));
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
        // lane quarter warp % 4 (TMEM lane field, bits 16-31), column slot warp / 4
        tstk = *tmem_base + (static_cast<uint32_t>(warp & 3) << 21) +
               static_cast<uint32_t>((warp >> 2) * kTmemColsPerWarp);
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
                if (item >= prm.total_items) {
                    s.job = -1;
                    mbar_arrive(&full[b]);
                    break;
                }
                const int j = find_job(prm, item);
                const JobDev &J = prm.jobs[j];
                const int64_t local = item - J.item0;
                const int t = static_cast<int>(local / J.groups);
                const int g = static_cast<int>(local % J.groups);
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
        const int64_t p0 = static_cast<int64_t>(s.group) * prm.group;
        const int64_t p1 = min(J.P, p0 + prm.group);
        for (;;) {
            int idx = 0;
            if (lane == 0) idx = atomicAdd(&slots[b].next, 1);
            idx = __shfl_sync(kFull, idx, 0);
            const int64_t q = p0 + idx;
            if (q >= p1) break;
            const int64_t p = J.order ? static_cast<int64_t>(J.order[q]) : q;
            process_program<T, K, D>(J, p, s.tile, tile, xs, pbuf, fbuf, stk, tstk, lane);
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
            tmem_dealloc(*tmem_base, tmem_columns(NW));
        }
    }
}

// Finalize: merge each program's tiles in a fixed order in fp64 (Chan et al.'s pairwise
// update of centred sums), then MSE and 1 - r^2 (Eq. 1, squared).
template <bool FP64>
__device__ __forceinline__ double word_pair(const uint32_t *w0, const uint32_t *w1) {
    if constexpr (FP64) {
        return __longlong_as_double(static_cast<long long>(
            (static_cast<unsigned long long>(*w1) << 32) | *w0));
    } else {
        return static_cast<double>(__uint_as_float(*w0)) +
               static_cast<double>(__uint_as_float(*w1));
    }
}

template <bool FP64, int MAXJ>
__global__ void finalize_kernel(const __grid_constant__ LaunchParams<MAXJ> prm) {
    const int jn = blockIdx.y;
    if (jn >= prm.njobs) return;
    const JobDev &J = prm.jobs[jn];
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= J.P) return;
    const int T = J.tiles;
    const int64_t P = J.P;
    auto W = [&](int f, int t) { return J.partials + (static_cast<int64_t>(f) * T + t) * P + p; };
    beagle_fitness r;
    r.reserved = 0u;
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    uint32_t flags = 0u;
    if (*prm.error != 0u) {
        r.mse = r.one_minus_r2 = __longlong_as_double(0x7ff8000000000000ll);
        r.flags = BEAGLE_FLAG_TIMEOUT;
        J.out[p] = r;
        return;
    }
    bool nonconst = false, mdiff = false;
    double sse = 0.0, sumf = 0.0, m0 = 0.0;
    for (int t = 0; t < T; ++t) {
        const uint32_t tf = *W(kTileFlags, t);
        if (tf & TF_MALFORMED) flags |= BEAGLE_FLAG_MALFORMED;
        if (tf & TF_INVALID) flags |= BEAGLE_FLAG_INVALID;
    }
    if (flags) {
        r.mse = r.one_minus_r2 = inf;
        r.flags = flags;
        J.out[p] = r;
        return;
    }
    for (int t = 0; t < T; ++t) {
        const double n = static_cast<double>(min(static_cast<int64_t>(prm.tile),
                                                 J.N - static_cast<int64_t>(t) * prm.tile));
        const double m = FP64 ? word_pair<true>(W(kMean, t), W(kMean64, t))
                              : static_cast<double>(__uint_as_float(*W(kMean, t)));
        const uint32_t tf = *W(kTileFlags, t);
        const int ke = (tf >> 8) & 0xff, kd = (tf >> 16) & 0xff;
        sse += ldexp(word_pair<FP64>(W(kSe2, t), W(kSe2 + 1, t)), 2 * ke);
        sumf += n * m + ldexp(word_pair<FP64>(W(kSd, t), W(kSd + 1, t)), kd);
        nonconst |= (tf & TF_NONCONST) != 0u;
        if (t == 0) m0 = m;
        else mdiff |= (m != m0);
    }
    const double N = static_cast<double>(J.N);
    r.mse = sse / N;
    if (!nonconst && !mdiff) {
        r.one_minus_r2 = 1.0;
        r.flags = BEAGLE_FLAG_DEGENERATE;
        J.out[p] = r;
        return;
    }
    const double fbar = sumf / N;
    double sff = 0.0, sfy = 0.0;
    for (int t = 0; t < T; ++t) {
        const double n = static_cast<double>(min(static_cast<int64_t>(prm.tile),
                                                 J.N - static_cast<int64_t>(t) * prm.tile));
        const double m = FP64 ? word_pair<true>(W(kMean, t), W(kMean64, t))
                              : static_cast<double>(__uint_as_float(*W(kMean, t)));
        const uint32_t tf = *W(kTileFlags, t);
        const int kd = (tf >> 16) & 0xff, ky = (tf >> 24) & 0xff;
        const double dm = m - fbar;
        const double sd = ldexp(word_pair<FP64>(W(kSd, t), W(kSd + 1, t)), kd);
        sff += ldexp(word_pair<FP64>(W(kSdd, t), W(kSdd + 1, t)), 2 * kd) + 2.0 * dm * sd +
               n * dm * dm;
        sfy += ldexp(word_pair<FP64>(W(kSdy, t), W(kSdy + 1, t)), kd + ky) + dm * J.tile_sy[t];
    }
    if (!(sff > 0.0)) {
        r.one_minus_r2 = 1.0;
        r.flags = BEAGLE_FLAG_DEGENERATE;
    } else {
        const double rr = sfy / sqrt(sff * J.syy);
        r.one_minus_r2 = 1.0 - rr * rr;
        r.flags = 0u;
    }
    J.out[p] = r;
}

// --------------------------------------------------------------------------- launchers
template <typename T, int K, int D, int MAXJ>
static cudaError_t launch_impl(const LaunchParams<MAXJ> &prm, int nw, int grid,
                               cudaStream_t stream) {
    using Lay = SmemLayout<T, K>;
    const size_t smem = Lay::total(prm.xbuf_floats, prm.tile, nw);
    auto kern = score_kernel<T, K, D, MAXJ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    void *tok = nullptr;
    const bool timed = timing_enabled();
    if (timed) timing_begin(stream, &tok);
    kern<<<grid, (nw + 1) * 32, smem, stream>>>(prm);
    e = cudaGetLastError();
    if (timed) timing_end(stream, tok);
    if (e != cudaSuccess) return e;
    int64_t maxP = 0;
    for (int j = 0; j < prm.njobs; ++j) maxP = maxP > prm.jobs[j].P ? maxP : prm.jobs[j].P;
    if (maxP > 0) {
        dim3 fg(static_cast<unsigned>((maxP + 255) / 256), static_cast<unsigned>(prm.njobs));
        if (sizeof(T) == 8) finalize_kernel<true, MAXJ><<<fg, 256, 0, stream>>>(prm);
        else finalize_kernel<false, MAXJ><<<fg, 256, 0, stream>>>(prm);
        e = cudaGetLastError();
    }
    return e;
}

size_t smem_bytes(int precision, int cases, int xbuf_floats, int tile, int nw) {
    if (precision == BEAGLE_FP64)
        return SmemLayout<double, kCasesFp64>::total(xbuf_floats, tile, nw);
    switch (cases) {
    case 2: return SmemLayout<float, 2>::total(xbuf_floats, tile, nw);
    case 8: return SmemLayout<float, 8>::total(xbuf_floats, tile, nw);
    default: return SmemLayout<float, 4>::total(xbuf_floats, tile, nw);
    }
}

static int max_warps(int precision, int cases) {
    if (precision == BEAGLE_FP64) return KernelThreads<double, kCasesFp64>::value / 32 - 1;
    if (cases == 8) return KernelThreads<float, 8>::value / 32 - 1;
    if (cases == 2) return KernelThreads<float, 2>::value / 32 - 1;
    return KernelThreads<float, 4>::value / 32 - 1;
}

int plan_warps(int precision, int cases, int xbuf_floats, int tile) {
    int nw = max_warps(precision, cases);
    while (nw > 1 && smem_bytes(precision, cases, xbuf_floats, tile, nw) > kSmemBudget) --nw;
    return nw;
}

template <int MAXJ>
static cudaError_t launch_any(const LaunchParams<MAXJ> &prm, int precision, int cases, int nw,
                              int grid, cudaStream_t s) {
    if (precision == BEAGLE_FP64)
        return launch_impl<double, kCasesFp64, kMaxDepth, MAXJ>(prm, nw, grid, s);
    switch (cases) {
    case 2: return launch_impl<float, 2, kMaxDepth, MAXJ>(prm, nw, grid, s);
    case 8: return launch_impl<float, 8, kMaxDepth, MAXJ>(prm, nw, grid, s);
    default: return launch_impl<float, 4, kMaxDepth, MAXJ>(prm, nw, grid, s);
    }
}

template <typename T, int K, int MAXJ>
static cudaError_t load_one() {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, score_kernel<T, K, kMaxDepth, MAXJ>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, finalize_kernel<sizeof(T) == 8, MAXJ>);
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

cudaError_t launch_score_batch(const LaunchParams<kMaxJobs> &prm, int precision, int cases,
                               int nw, int grid, cudaStream_t s) {
    return launch_any<kMaxJobs>(prm, precision, cases, nw, grid, s);
}

}  // namespace beagle
