// Device code shared by the scoring kernels (score_kernels.cu) and the serving kernel
// (serve_kernels.cu): shared-memory layout, per-(program, tile) evaluation and tile
// statistics, and the per-program fp64 merge of the tiles (the finalize step).
#pragma once

#include "interp_ptx.cuh"
#include "interp_ptx8.cuh"
#include "kernels.h"
#include "score.cuh"

namespace beagle {

// Shared-memory layout of one CTA (dynamic), nw consumer warps:
//   [0, 64)        mbarriers: full[2], empty[2]
//   [64, 128)      slot descriptors (2 x Slot)
//   [128, ...)     X stage buffers: 2 x xbuf_floats fp32 (TMA destinations, 128-byte aligned)
//   ...            per-warp output buffers: nw x tile x T
//   ...            per-warp packed programs: nw x (kMaxLen + 2) x uint2
//   ...            per-warp value stacks: nw x (D - 1) rows x 32 K x T (none where the
//                  stack lives in tensor memory)
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

// The 4- and 8-case FP32 paths keep their stack rows in tensor memory (the warp's 32-lane
// quarter of TMEM being warp % 4 and its column slot warp / 4); the other paths keep them in
// shared memory.
template <typename T, int K>
constexpr bool kTmemStackPath = sizeof(T) == 4 && (K == 4 || K == 8);
// Columns a warp's stack takes: D - 1 rows of K columns, rounded to a power of two (4 cases:
// 64 for the 16-value fast pass, 128 for the 32-value deep pass; 8 cases: 128 for the fast
// pass, so 16 warps fill the 512 columns).
__host__ __device__ constexpr int tmem_cols_per_warp(int D, int K) {
    return K * (D - 1) <= 64 ? 64 : K * (D - 1) <= 128 ? 128 : 256;
}
static_assert(4 * (kDepthFast - 1) <= tmem_cols_per_warp(kDepthFast, 4), "rows fit the columns");
static_assert(4 * (kMaxDepth - 1) <= tmem_cols_per_warp(kMaxDepth, 4), "rows fit the columns");
static_assert(8 * (kDepthFast - 1) <= tmem_cols_per_warp(kDepthFast, 8), "rows fit the columns");
__host__ __device__ constexpr uint32_t tmem_columns(int nw, int D, int K) {   // power of two, 32..512
    const int need = (nw + 3) / 4 * tmem_cols_per_warp(D, K);
    return need <= 32 ? 32u : need <= 64 ? 64u : need <= 128 ? 128u : need <= 256 ? 256u : 512u;
}

template <typename T, int K, int D>
struct SmemLayout {
    static constexpr size_t kStackRows = D - 1;
    static constexpr bool kTmemStack = kTmemStackPath<T, K>;
    static __host__ __device__ size_t xbuf_off() { return 128; }
    static __host__ __device__ size_t fbuf_off(int xbuf_floats) {
        return xbuf_off() + 2ull * xbuf_floats * sizeof(float);
    }
    static __host__ __device__ size_t pbuf_off(int xbuf_floats, int tile, int nw) {
        return fbuf_off(xbuf_floats) + static_cast<size_t>(nw) * tile * sizeof(T);
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

// A tile's outputs, in the warp's shared-memory buffer in case order, read the way the
// statistics take them: lane l's values are the cases 128 h + 4 l + j (h over the tile's
// 128-case halves, j = 0..3), so every path forms the same sums in the same order.
template <typename T, int K>
struct TileValues {
    const T *buf;
    // values 4h..4h+3 of this lane
    __device__ __forceinline__ void get4(int h, int lane, T (&v)[4]) const {
        if constexpr (sizeof(T) == 4) {
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
#pragma unroll 1
        for (int h = 0; h < halves; ++h) {
            T v[4];
            get4(h, lane, v);
            f(h, v);
        }
    }
};

// ------------------------------------------------------------------ the paper's fitness
// Rows of the staged tile: lane l reads the 4 consecutive cases 128 h + 4 l .. + 3 of a row.
__device__ __forceinline__ float4 tile_row4(const float *row, int h, int lane, int rows) {
    const int i = h * 128 + lane * 4;
    return *reinterpret_cast<const float4 *>(row + (i / kBox) * rows * kBox + (i % kBox));
}
__device__ __forceinline__ float f4_elem(const float4 &v, int j) {
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

__device__ __forceinline__ long long warp_sum_i64(long long v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Eq. 5's per-case reward of a valid pair, in the path's precision, each operation rounded
// once (no contraction): q = min/max of the magnitudes, q^k (k = 1, 2, 3, 8), M q^k, minus
// M/11 when the two have opposite signs, rounded to nearest even.
__device__ __forceinline__ long long std_reward(float f, float y, int k, int M) {
    const float a = fabsf(f), b = fabsf(y);
    const float mx = fmaxf(a, b), mn = fminf(a, b);
    if (mx == 0.0f) return M;
    const float q = __fdiv_rn(mn, mx);
    float qk = q;
    if (k == 2) qk = __fmul_rn(q, q);
    else if (k == 3) qk = __fmul_rn(__fmul_rn(q, q), q);
    else if (k == 8) {
        const float q2 = __fmul_rn(q, q), q4 = __fmul_rn(q2, q2);
        qk = __fmul_rn(q4, q4);
    }
    const float Mf = static_cast<float>(M);
    float v = __fmul_rn(Mf, qk);
    if ((f < 0.0f && y > 0.0f) || (f > 0.0f && y < 0.0f)) v = __fsub_rn(v, __fdiv_rn(Mf, 11.0f));
    return static_cast<long long>(rintf(v));
}
__device__ __forceinline__ long long std_reward(double f, float yf, int k, int M) {
    const double y = static_cast<double>(yf);
    const double a = fabs(f), b = fabs(y);
    const double mx = fmax(a, b), mn = fmin(a, b);
    if (mx == 0.0) return M;
    const double q = __ddiv_rn(mn, mx);
    double qk = q;
    if (k == 2) qk = __dmul_rn(q, q);
    else if (k == 3) qk = __dmul_rn(__dmul_rn(q, q), q);
    else if (k == 8) {
        const double q2 = __dmul_rn(q, q), q4 = __dmul_rn(q2, q2);
        qk = __dmul_rn(q4, q4);
    }
    const double Md = static_cast<double>(M);
    double v = __dmul_rn(Md, qk);
    if ((f < 0.0 && y > 0.0) || (f > 0.0 && y < 0.0)) v = __dsub_rn(v, __ddiv_rn(Md, 11.0));
    return static_cast<long long>(rint(v));
}

template <typename T>
__device__ __forceinline__ void put_value(uint32_t *w, T v) {
    if constexpr (sizeof(T) == 4) {
        w[0] = __float_as_uint(v);
        w[1] = 0u;
    } else {
        const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
        w[0] = static_cast<uint32_t>(b);
        w[1] = static_cast<uint32_t>(b >> 32);
    }
}

// Tile statistics of the paper's fitness functions. Invalid cases arrive as NaN outputs (a
// valid value is never NaN); all_bad: a constant of the program is itself invalid, so every
// case is. Targets are valid when |y| <= 1e30 (NaN fails).
template <typename T, int K, typename Vals, typename FieldFn>
__device__ __forceinline__ void fit_tile_stats(const JobDev &J, int nval, bool all_bad,
                                            const Vals &vals, const float *xs, int lane,
                                            FieldFn field) {
    const int halves = (nval + 127) / 128;
    const int rows = J.rows;
    const float *yrow = xs + J.d * kBox;
    const float *ycrow = xs + (J.d + 1) * kBox;
    uint32_t c1 = 0, c2 = 0, n = 0;
    uint32_t w[kNumFitFields];
#pragma unroll
    for (int f = 0; f < kNumFitFields; ++f) w[f] = 0u;
    if (J.kind == kFitCorr) {
        using Sum = typename SumOf<T>::type;
        Sum sf;
        const T inf = static_cast<T>(INFINITY);
        T fabsmax = T(0), fmn = inf, fmx = -inf;
        float ymn = INFINITY, ymx = -INFINITY, ycmax = 0.0f;
        vals.for_halves(halves, lane, [&](int h, const T (&v)[4]) {
            const float4 y4 = tile_row4(yrow, h, lane, rows);
            const float4 yc4 = tile_row4(ycrow, h, lane, rows);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (h * 128 + lane * 4 + j < nval) {
                    const T fi = v[j];
                    const float yv = f4_elem(y4, j);
                    const bool fv = !all_bad && fi == fi, tv = fabsf(yv) <= 1e30f;
                    c1 += fv != tv;
                    c2 += !fv && !tv;
                    if (fv && tv) {
                        ++n;
                        sf.add(fi);
                        fabsmax = fmax(fabsmax, fabs(fi));
                        fmn = fmin(fmn, fi);
                        fmx = fmax(fmx, fi);
                        ymn = fminf(ymn, yv);
                        ymx = fmaxf(ymx, yv);
                        ycmax = fmaxf(ycmax, fabsf(f4_elem(yc4, j)));
                    }
                }
            }
        });
        n = __reduce_add_sync(kFull, n);
        c1 = __reduce_add_sync(kFull, c1);
        c2 = __reduce_add_sync(kFull, c2);
        sf.warp_allreduce();
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            fabsmax = fmax(fabsmax, __shfl_xor_sync(kFull, fabsmax, o));
            fmn = fmin(fmn, __shfl_xor_sync(kFull, fmn, o));
            fmx = fmax(fmx, __shfl_xor_sync(kFull, fmx, o));
            ymn = fminf(ymn, __shfl_xor_sync(kFull, ymn, o));
            ymx = fmaxf(ymx, __shfl_xor_sync(kFull, ymx, o));
            ycmax = fmaxf(ycmax, __shfl_xor_sync(kFull, ycmax, o));
        }
        T m = T(0);
        if constexpr (sizeof(T) == 4) m = n ? (sf.s + sf.c) / static_cast<float>(n) : 0.0f;
        else m = n ? sf.s / static_cast<double>(n) : 0.0;
        int kd = 0, ky = 0;
        T sds = T(1), sys = T(1);
        if constexpr (sizeof(T) == 4) {   // valid values reach 1e30: scale the fp32 sums
            kd = scale_exponent(2.0f * fabsmax);
            ky = scale_exponent(ycmax);
            sds = pow2f(-kd);
            sys = pow2f(-ky);
        }
        Sum sd, sdd, sdy, sy, syy;
        vals.for_halves(halves, lane, [&](int h, const T (&v)[4]) {
            const float4 y4 = tile_row4(yrow, h, lane, rows);
            const float4 yc4 = tile_row4(ycrow, h, lane, rows);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (h * 128 + lane * 4 + j < nval) {
                    const T fi = v[j];
                    const float yv = f4_elem(y4, j);
                    if (!all_bad && fi == fi && fabsf(yv) <= 1e30f) {
                        const T dv = (fi - m) * sds;
                        // FP32: the stored fp32 y - ybar; FP64: y - ybar formed in fp64
                        const T yc = (sizeof(T) == 4 ? static_cast<T>(f4_elem(yc4, j))
                                                     : static_cast<T>(yv) - static_cast<T>(J.ybar)) *
                                     sys;
                        sd.add(dv);
                        sdd.add_prod(dv, dv);
                        sdy.add_prod(dv, yc);
                        sy.add(yc);
                        syy.add_prod(yc, yc);
                    }
                }
            }
        });
        sd.warp_allreduce();
        sdd.warp_allreduce();
        sdy.warp_allreduce();
        sy.warp_allreduce();
        syy.warp_allreduce();
        if (lane == 0) {
            put_value<T>(w + kfMean, m);
            put_pair(w + kfSd, sd);
            put_pair(w + kfSdd, sdd);
            put_pair(w + kfSdy, sdy);
            put_pair(w + kfSy, sy);
            put_pair(w + kfSyy, syy);
            put_value<T>(w + kfFmin, fmn);
            put_value<T>(w + kfFmax, fmx);
            w[kfYmin] = __float_as_uint(ymn);
            w[kfYmax] = __float_as_uint(ymx);
            w[kfFlags] = (static_cast<uint32_t>(kd) << 16) | (static_cast<uint32_t>(ky) << 24);
        }
    } else {
        const int k = J.kind == kFitStd ? 1 : J.kind == kFitStd + 1 ? 2 :
                      J.kind == kFitStd + 2 ? 3 : 8;
        const int M = J.max_score;
        long long score = 0;
        vals.for_halves(halves, lane, [&](int h, const T (&v)[4]) {
            const float4 y4 = tile_row4(yrow, h, lane, rows);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (h * 128 + lane * 4 + j < nval) {
                    const T fi = v[j];
                    const float yv = f4_elem(y4, j);
                    const bool fv = !all_bad && fi == fi, tv = fabsf(yv) <= 1e30f;
                    c1 += fv != tv;
                    c2 += !fv && !tv;
                    if (J.kind == kFitValidate) {
                        if (fv && tv &&
                            fabs(static_cast<double>(fi) - static_cast<double>(yv)) <=
                                0.001 * fabs(static_cast<double>(yv)))
                            ++score;
                    } else if (fv && tv) {
                        score += std_reward(fi, yv, k, M);
                    } else {
                        score += (fv || tv) ? -M : M;
                    }
                }
            }
        });
        score = warp_sum_i64(score);
        c1 = __reduce_add_sync(kFull, c1);
        c2 = __reduce_add_sync(kFull, c2);
        if (lane == 0) {
            w[kfScore] = static_cast<uint32_t>(static_cast<unsigned long long>(score));
            w[kfScore + 1] = static_cast<uint32_t>(static_cast<unsigned long long>(score) >> 32);
        }
    }
    if (lane == 0) {
        w[kfN] = n;
        w[kfC1] = c1;
        w[kfC2] = c2;
#pragma unroll
        for (int f = 0; f < kNumFitFields; ++f) *field(f) = w[f];
    }
    __syncwarp();
}

// Score program p on tile t: the partials of (p, t) are written. Returns 1 instead when the
// program is deeper than this kernel's stack and was left to the deep pass (its partials are
// not written here), else 0. FIT: the job scores with the paper's fitness (J.kind != MSE); a
// compile-time flag, so the MSE code the hot loop runs carries none of the fitness branches.
template <typename T, int K, int D, bool FIT>
__device__ __forceinline__ int process_program_kind(const JobDev &J, int64_t q, int64_t p, int t,
                                                    int tile, const float *xs, uint2 *pbuf,
                                                    T *fbuf, T *stk, uint32_t tstk, int lane) {
    using Sum = typename SumOf<T>::type;
    constexpr int CH = 32 * K;
    constexpr bool kPtx = sizeof(T) == 4 && (K == 4 || K == 8);   // the inline-PTX loops
    // MSE / 1 - r^2 without per-case outputs: a tile with an invalid case is invalid whatever
    // its other cases hold (it stores only its flag). So no pass runs after the first that
    // finds one (nor any, for a folded constant that is invalid), and once some tile has found
    // the program invalid its later tiles store the flag without running it (the flag is
    // loaded here, its latency covered by the token copy below; L2, not L1, so that the other
    // SMs' stores are seen). The paper's fitness functions count invalid cases and run them all;
    // so does every launch whose flags array is null (beagle_set_invalid_early_exit(0)).
    const bool stop_at_invalid = !FIT && J.fout == nullptr && J.known_invalid != nullptr;
    const bool known_bad = stop_at_invalid && __ldcg(J.known_invalid + p) != 0;
    Packed pk;
    bool have = false;
    if constexpr (D == kDepthFast) {
        // Packed once for the call by the packing kernel: copy its tokens (the deep ones are
        // on the deep list already).
        if (J.packed) {
            const uint32_t m = J.pmeta[q];
            if (m != kPackNone) {
                pk.n = static_cast<int>(m & 0xffffu);
                pk.malformed = (m & kPackMalformed) != 0;
                pk.deep = (m & kPackDeep) != 0;
                pk.const_bad = (m & kPackConstBad) != 0;
                if (pk.deep && J.deep_list) return 1;
                if (!pk.malformed && !pk.deep) {
                    const uint2 *src = J.packed + J.poff[q];
                    for (int i = lane; i <= pk.n; i += 32) pbuf[i] = src[i];
                    __syncwarp();
                }
                have = true;
            }
        }
    }
    if (!have) {
        const int64_t off = J.offs[p];
        pk = pack_program<T, D>(J.ops + off, J.consts + off, J.lens[p], J.d, pbuf, lane);
        if (pk.deep) {
            // Deeper than this pass's stack: the deep pass scores it. The warp that meets the
            // program's first tile enqueues it once; without a deep list it cannot be scored.
            if (J.deep_list) {
                if (t == 0 && lane == 0) J.deep_list[atomicAdd(J.deep_count, 1)] = static_cast<int32_t>(p);
                return 1;
            }
        }
        if constexpr (kPtx) {
            // Bits 24-28 of each token: the handler id of the token after it (the inline-PTX
            // interpreters branch on it while they load that token). Each round reads, then
            // writes.
            for (int base = 0; base < pk.n; base += 32) {
                const int i = base + lane;
                const uint32_t nh = i < pk.n ? (pbuf[i + 1].x & 31u) : 0u;
                __syncwarp();
                if (i < pk.n) pbuf[i].x |= nh << 24;
                __syncwarp();
            }
        }
    }

    const int64_t P = J.P;
    const int tiles = J.tiles;
    uint32_t *part = J.partials;
    auto field = [&](int f) -> uint32_t * {
        return part + (static_cast<int64_t>(f) * tiles + t) * P + p;
    };
    if (pk.malformed || pk.deep) {
        if (lane == 0) *field(FIT ? kfFlags : kTileFlags) = TF_MALFORMED;
        return 0;
    }
    const int64_t tstart = static_cast<int64_t>(t) * tile;
    const int nval = static_cast<int>(min(static_cast<int64_t>(tile), J.N - tstart));
    const int rows = J.rows;

    TileValues<T, K> vals;
    vals.buf = fbuf;
    bool anybad = pk.const_bad || known_bad;
    int c_run = 0;   // cases the passes ran (a pass runs CH cases, the last one fewer)
    if constexpr (sizeof(T) == 4 && K == 8) {
        static_assert(CH == kBox, "a pass of the 8-case loop is one staged box");
        for (int c0 = 0; c0 < nval; c0 += CH) {
            if (stop_at_invalid && __any_sync(kFull, anybad)) break;
            c_run = c0 + CH;
            const float *xrow = xs + (c0 / kBox) * rows * kBox + lane * 4;
            float f[8];
            bool bad[8];
            run_program_ptx8(smem_addr(pbuf), smem_addr(xrow), tstk, f, bad);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (FIT && bad[j]) f[j] = __int_as_float(0x7fc00000);
                if (bad[j] && c0 + (j >> 2) * 128 + lane * 4 + (j & 3) < nval) anybad = true;
            }
            *reinterpret_cast<float4 *>(fbuf + c0 + lane * 4) = make_float4(f[0], f[1], f[2], f[3]);
            *reinterpret_cast<float4 *>(fbuf + c0 + 128 + lane * 4) = make_float4(f[4], f[5], f[6], f[7]);
        }
    } else {
        for (int c0 = 0; c0 < nval; c0 += CH) {
            if (stop_at_invalid && __any_sync(kFull, anybad)) break;
            c_run = c0 + CH;
            const float *xrow = xs + (c0 / kBox) * rows * kBox + (c0 % kBox) + lane * K;
            T f[K];
            bool bad[K];
            if constexpr (sizeof(T) == 4 && K == 4)
                run_program_ptx4(smem_addr(pbuf), smem_addr(xrow), tstk, f, bad);
            else
                run_program<T, K>(smem_addr(pbuf), pk.n, smem_addr(xrow),
                                  smem_addr(stk + lane * K), f, bad);
            if constexpr (FIT) {   // the paper's fitness: invalid cases become NaN
#pragma unroll
                for (int j = 0; j < K; ++j)
                    if (bad[j]) f[j] = static_cast<T>(__int_as_float(0x7fc00000));
            }
            sts_vec<T, K>(smem_addr(fbuf + c0 + lane * K), f);
#pragma unroll
            for (int j = 0; j < K; ++j)
                if (bad[j] && c0 + lane * K + j < nval) anybad = true;
        }
    }
    anybad = __any_sync(kFull, anybad);
    if (J.cases_run != nullptr && lane == 0)
        atomicAdd(reinterpret_cast<unsigned long long *>(J.cases_run + p),
                  static_cast<unsigned long long>(min(c_run, nval)));
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
    if constexpr (FIT) {
        fit_tile_stats<T, K>(J, nval, pk.const_bad, vals, xs, lane, field);
        return 0;
    }
    if (anybad) {
        if (lane == 0) {
            *field(kTileFlags) = TF_INVALID;
            if (stop_at_invalid && !known_bad) J.known_invalid[p] = 1;
        }
        return 0;
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
        // only and is a plain fp32 sum over each lane's pair half (8 terms, relative error below
        // 8 u), compensated beyond; the centred sums are compensated throughout. An overflow anywhere in these
        // unscaled sums leaves an infinity or a NaN in them; then the two-pass form below,
        // which scales the terms, runs instead (outputs or targets near 2^60 and above). The
        // outputs are all equal exactly when every f - f_0 is +0 or -0 (no flush to zero).
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
        // Lane pairs of cases (4l, 4l+1) and (4l+2, 4l+3) run through f32x2 instructions: each
        // half of every accumulator is its own sum, merged before the warp reduction. A case is
        // unlike case 0 when f - f_0 has a nonzero magnitude (an OR of its bits, sign masked).
        const float2 m02 = make_float2(m0, m0), fa2 = make_float2(fa, fa);
        float2 se2 = make_float2(0.0f, 0.0f);
        uint32_t dbits = 0u;
        KahanF2 sd2, sdd2, sdy2;
        auto pair_stats = [&](float2 f, float2 y, float2 yc, uint32_t kx, uint32_t ky) {
            const float2 e = sub2(f, y);
            se2 = __ffma2_rn(e, e, se2);
            const float2 d = sub2(f, fa2);
            dbits |= (__float_as_uint(d.x) & kx) | (__float_as_uint(d.y) & ky);
            const float2 dv = sub2(f, m02), dvn = sub2(m02, f);   // dvn = -dv exactly
            sd2.add(dv);
            sdd2.add_prod(dv, dvn, dv);
            sdy2.add_prod(dv, dvn, yc);
        };
        vals.for_halves(halves, lane, [&](int h, const T (&v)[4]) {
            const float4 y4 = row4(yrow, h);
            const float4 yc4 = row4(ycrow, h);
            if (h * 128 + 128 <= nval) {   // a full half (warp-uniform)
                pair_stats(make_float2(v[0], v[1]), make_float2(y4.x, y4.y),
                           make_float2(yc4.x, yc4.y), ~0u, ~0u);
                pair_stats(make_float2(v[2], v[3]), make_float2(y4.z, y4.w),
                           make_float2(yc4.z, yc4.w), ~0u, ~0u);
            } else {
                // The ragged half: a case past the end enters as f = y = m0, yc = 0 (every term
                // exactly 0) with its f - f_0 bits dropped.
                float f[4], y[4], yc[4];
                uint32_t keep[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool in = h * 128 + lane * 4 + j < nval;
                    f[j] = in ? v[j] : m0;
                    y[j] = in ? elem(y4, j) : m0;
                    yc[j] = in ? elem(yc4, j) : 0.0f;
                    keep[j] = in ? ~0u : 0u;
                }
                pair_stats(make_float2(f[0], f[1]), make_float2(y[0], y[1]),
                           make_float2(yc[0], yc[1]), keep[0], keep[1]);
                pair_stats(make_float2(f[2], f[3]), make_float2(y[2], y[3]),
                           make_float2(yc[2], yc[3]), keep[2], keep[3]);
            }
        });
        const bool nc = __any_sync(kFull, (dbits & 0x7fffffffu) != 0u);
        // The four sums (se, sd, sdd, sdy) over the warp by halving: after the step over lane
        // bit 4 each half of the warp holds two of them, after the step over bit 3 each group
        // of 8 lanes one (lanes 8g..8g+7 sum g), merged over its group in three more steps.
        KahanF q0, q1, q2, q3;
        q0.s = se2.x;
        q0.merge(se2.y, 0.0f);
        if (nc) {
            q1 = sd2.merged();
            q2 = sdd2.merged();
            q3 = sdy2.merged();
        }
        const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
        KahanF ka = hi16 ? q2 : q0, kb = hi16 ? q3 : q1;
        ka.merge(kf_shfl_xor(hi16 ? q0 : q2, 16));
        kb.merge(kf_shfl_xor(hi16 ? q1 : q3, 16));
        KahanF k = hi8 ? kb : ka;
        k.merge(kf_shfl_xor(hi8 ? ka : kb, 8));
#pragma unroll
        for (int o = 4; o >= 1; o >>= 1) k.merge(kf_shfl_xor(k, o));
        static_assert(kSd == kSe2 + 2 && kSdd == kSe2 + 4 && kSdy == kSe2 + 6,
                      "the sums' fields follow one another");
        if (__all_sync(kFull, isfinite(k.s + k.c))) {
            if ((lane & 7) == 0) {
                const int g = lane >> 3;
                *field(kSe2 + 2 * g) = __float_as_uint(k.s);
                *field(kSe2 + 2 * g + 1) = __float_as_uint(k.c);
            }
            if (lane == 0) {
                *field(kMean) = __float_as_uint(nc ? m0 : fa);
                *field(kMean64) = 0u;
                *field(kTileFlags) = nc ? TF_NONCONST : 0u;
            }
            __syncwarp();
            return 0;
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
    return 0;
}

// Threads per CTA the kernel is compiled for (the register budget per thread follows from it).
// The 4-case FP32 path, its stack in tensor memory, gets 32 warps (64 registers a thread):
// more resident warps hide more of the dispatch latency (C2 population: 17 consumer warps
// 2,304 GPoPs, 27 at 72 registers 2,656, 31 at 64 registers 2,738); the 2-case path also
// fits 32 warps; the 8-case and FP64 paths get 16 warps (128 registers).
// The deep pass (D = 32) of the 4-case path has 16 consumer warps: 128 tensor-memory columns
// each fill the 512 columns.
// q: the program's position in the work order, p its index.
template <typename T, int K, int D>
__device__ __forceinline__ int process_program(const JobDev &J, int64_t q, int64_t p, int t,
                                               int tile, const float *xs, uint2 *pbuf, T *fbuf,
                                               T *stk, uint32_t tstk, int lane) {
    if (J.kind == kFitMse)
        return process_program_kind<T, K, D, false>(J, q, p, t, tile, xs, pbuf, fbuf, stk, tstk, lane);
    return process_program_kind<T, K, D, true>(J, q, p, t, tile, xs, pbuf, fbuf, stk, tstk, lane);
}

template <typename T, int K, int D>
struct KernelThreads {
    // FP32 with the stack in TMEM: 4 cases, 16 values: 31 consumer warps (64 columns each);
    // 4 cases, 32 values, or 8 cases, 16 values: 16 warps (128 columns each)
    static constexpr int value = sizeof(T) != 4 ? 512 : (K == 4 && D > 16) ? 544 :
                                 K == 8 ? 544 : 1024;
};

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

// Sums over a group of g lanes (g a power of two, the group aligned), the same butterfly on
// every lane of the group: each level adds two values that commute, so every lane ends with
// the same bits, and the tree, hence the bits, depends only on g and on the lane each value
// started on.
__device__ __forceinline__ double group_sum_f64(double v, int g) {
    for (int o = g >> 1; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o, g);
    return v;
}
__device__ __forceinline__ float group_sum_f32(float v, int g) {
    for (int o = g >> 1; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o, g);
    return v;
}
// Lanes that merge one program's tiles: a power of two, at most 32 and at most the tile count
// rounded up (this GPU's fp64 rate is low: a warp's fp64 add takes 16 cycles, so few tiles are
// merged by few lanes).
__host__ __device__ __forceinline__ int finalize_group(int tiles) {
    int g = 1;
    while (g < 32 && g < tiles) g <<= 1;
    return g;
}

// One program's MSE and 1 - r^2 from its tile partials (tile: cases per tile; timed_out: the
// launch's error word was set), by a group of g = finalize_group(tiles) lanes of a warp (all 32
// lanes call it; r = lane % g): lane r takes tiles r, r + g, ..., then group sums. Two passes: the flags, sum of squared errors and output sum, then the sums centred on
// the program's mean. On the FP32 path each tile sum is a compensated pair (s, c): the s parts
// are added in fp64, the small c parts (about 2^-24 |s| each) in fp32, whose rounding adds
// about 2^-48 of the sum; an exponent k != 0 marks a tile whose terms were scaled by 2^-k.
// Few fp64 operations per tile: this GPU's fp64 rate is low. Lane 0 writes the result.
template <bool FP64>
__device__ __forceinline__ void finalize_mse_program(const JobDev &J, int64_t p, int tile,
                                                     bool timed_out, int lane) {
    const int T = J.tiles;
    const int g = finalize_group(T);
    const int rl = lane & (g - 1);
    const int64_t P = J.P;
    auto W = [&](int f, int t) { return J.partials + (static_cast<int64_t>(f) * T + t) * P + p; };
    beagle_fitness r;
    r.reserved = 0u;
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    if (timed_out) {
        r.mse = r.one_minus_r2 = __longlong_as_double(0x7ff8000000000000ll);
        r.flags = BEAGLE_FLAG_TIMEOUT;
        if (rl == 0) J.out[p] = r;
        return;
    }
    auto mean_of = [&](int t) {
        return FP64 ? word_pair<true>(W(kMean, t), W(kMean64, t))
                    : static_cast<double>(__uint_as_float(*W(kMean, t)));
    };
    const double m0 = mean_of(0);
    uint32_t flags = 0u;
    bool nonconst = false, mdiff = false;
    double sse = 0.0, sumf = 0.0;
    float sse_c = 0.0f, sumf_c = 0.0f;
    for (int t = rl; t < T; t += g) {
        const uint32_t tf = *W(kTileFlags, t);
        if (tf & TF_MALFORMED) flags |= BEAGLE_FLAG_MALFORMED;
        if (tf & TF_INVALID) flags |= BEAGLE_FLAG_INVALID;
        if (flags) continue;
        const double n = static_cast<double>(min(static_cast<int64_t>(tile),
                                                 J.N - static_cast<int64_t>(t) * tile));
        const double m = mean_of(t);
        const int ke = (tf >> 8) & 0xff, kd = (tf >> 16) & 0xff;
        if (FP64 || ke != 0) {
            sse += ldexp(word_pair<FP64>(W(kSe2, t), W(kSe2 + 1, t)), 2 * ke);
        } else {
            sse += static_cast<double>(__uint_as_float(*W(kSe2, t)));
            sse_c += __uint_as_float(*W(kSe2 + 1, t));
        }
        if (FP64 || kd != 0) {
            sumf += n * m + ldexp(word_pair<FP64>(W(kSd, t), W(kSd + 1, t)), kd);
        } else {
            sumf += n * m + static_cast<double>(__uint_as_float(*W(kSd, t)));
            sumf_c += __uint_as_float(*W(kSd + 1, t));
        }
        nonconst |= (tf & TF_NONCONST) != 0u;
        mdiff |= (m != m0);
    }
    for (int o = g >> 1; o >= 1; o >>= 1) {
        flags |= __shfl_xor_sync(kFull, flags, o, g);
        nonconst |= __shfl_xor_sync(kFull, nonconst ? 1 : 0, o, g) != 0;
        mdiff |= __shfl_xor_sync(kFull, mdiff ? 1 : 0, o, g) != 0;
    }
    if (flags) {
        r.mse = r.one_minus_r2 = inf;
        r.flags = flags;
        if (rl == 0) J.out[p] = r;
        return;
    }
    sse = group_sum_f64(sse, g) + static_cast<double>(group_sum_f32(sse_c, g));
    sumf = group_sum_f64(sumf, g) + static_cast<double>(group_sum_f32(sumf_c, g));
    const double N = static_cast<double>(J.N);
    r.mse = sse / N;
    if (!nonconst && !mdiff) {
        r.one_minus_r2 = 1.0;
        r.flags = BEAGLE_FLAG_DEGENERATE;
        if (rl == 0) J.out[p] = r;
        return;
    }
    const double fbar = sumf / N;
    double sff = 0.0, sfy = 0.0;
    float sff_c = 0.0f, sfy_c = 0.0f;
    for (int t = rl; t < T; t += g) {
        const double n = static_cast<double>(min(static_cast<int64_t>(tile),
                                                 J.N - static_cast<int64_t>(t) * tile));
        const double m = mean_of(t);
        const uint32_t tf = *W(kTileFlags, t);
        const int kd = (tf >> 16) & 0xff, ky = (tf >> 24) & 0xff;
        const double dm = m - fbar;
        double sd, sdd, sdy;
        if (FP64 || (kd | ky) != 0) {
            sd = ldexp(word_pair<FP64>(W(kSd, t), W(kSd + 1, t)), kd);
            sdd = ldexp(word_pair<FP64>(W(kSdd, t), W(kSdd + 1, t)), 2 * kd);
            sdy = ldexp(word_pair<FP64>(W(kSdy, t), W(kSdy + 1, t)), kd + ky);
        } else {
            sd = static_cast<double>(__uint_as_float(*W(kSd, t)));
            sdd = static_cast<double>(__uint_as_float(*W(kSdd, t)));
            sdy = static_cast<double>(__uint_as_float(*W(kSdy, t)));
            sff_c += __uint_as_float(*W(kSdd + 1, t)) +
                     2.0f * static_cast<float>(dm) * __uint_as_float(*W(kSd + 1, t));
            sfy_c += __uint_as_float(*W(kSdy + 1, t));
        }
        sff += sdd + 2.0 * dm * sd + n * dm * dm;
        sfy += sdy + dm * J.tile_sy[t];
    }
    sff = group_sum_f64(sff, g) + static_cast<double>(group_sum_f32(sff_c, g));
    sfy = group_sum_f64(sfy, g) + static_cast<double>(group_sum_f32(sfy_c, g));
    if (!(sff > 0.0)) {
        r.one_minus_r2 = 1.0;
        r.flags = BEAGLE_FLAG_DEGENERATE;
    } else {
        const double rr = sfy / sqrt(sff * J.syy);
        r.one_minus_r2 = 1.0 - rr * rr;
        r.flags = 0u;
    }
    if (rl == 0) J.out[p] = r;
}


// Finalize of the paper's fitness functions: per program, the tiles merged in a fixed order in
// fp64. Correlation: valid-pair count, c1, c2; the outputs' mean over the valid pairs from the
// tile means and sums, S_ff by Chan et al.'s update, the targets' sums centred on their own
// mean over the valid pairs; r (Eq. 1 over the valid pairs), then Eq. 2. Eq. 5 family and
// validation: the integer tile scores summed.
template <bool FP64>
__device__ __forceinline__ double fit_value(const uint32_t *w0, const uint32_t *w1) {
    if constexpr (FP64)
        return __longlong_as_double(static_cast<long long>(
            (static_cast<unsigned long long>(*w1) << 32) | *w0));
    else
        return static_cast<double>(__uint_as_float(*w0));
}

template <bool FP64>
__device__ __forceinline__ void finalize_fit_program(const JobDev &J, int64_t p, bool timed_out) {
    const int T = J.tiles;
    const int64_t P = J.P;
    auto W = [&](int f, int t) { return J.partials + (static_cast<int64_t>(f) * T + t) * P + p; };
    beagle_fit_result r;
    r.score = r.asr = r.r2 = r.taxed_score = 0.0;
    r.c1 = r.c2 = 0;
    r.flags = 0u;
    r.reserved = 0u;
    if (timed_out) {
        r.score = r.asr = r.r2 = r.taxed_score = __longlong_as_double(0x7ff8000000000000ll);
        r.flags = BEAGLE_FLAG_TIMEOUT;
        J.fit[p] = r;
        return;
    }
    bool malformed = false;
    long long c1 = 0, c2 = 0, n = 0;
    for (int t = 0; t < T; ++t) {
        if (*W(kfFlags, t) & TF_MALFORMED) malformed = true;
        n += *W(kfN, t);
        c1 += *W(kfC1, t);
        c2 += *W(kfC2, t);
    }
    if (malformed) {
        r.score = r.asr = r.taxed_score = -__longlong_as_double(0x7ff0000000000000ll);
        r.flags = BEAGLE_FLAG_MALFORMED;
        J.fit[p] = r;
        return;
    }
    const double M = static_cast<double>(J.max_score), N = static_cast<double>(J.N);
    double score;
    if (J.kind == kFitCorr) {
        // constancy over the valid pairs, exactly: every tile's extremes equal, and equal
        // across the tiles that hold valid pairs
        bool fconst = true, yconst = true, have = false;
        double f0 = 0.0;
        float y0 = 0.0f;
        for (int t = 0; t < T; ++t) {
            if (*W(kfN, t) == 0u) continue;
            const double fmn = fit_value<FP64>(W(kfFmin, t), W(kfFmin + 1, t));
            const double fmx = fit_value<FP64>(W(kfFmax, t), W(kfFmax + 1, t));
            const float ymn = __uint_as_float(*W(kfYmin, t)), ymx = __uint_as_float(*W(kfYmax, t));
            if (fmn != fmx) fconst = false;
            if (ymn != ymx) yconst = false;
            if (!have) {
                f0 = fmn;
                y0 = ymn;
                have = true;
            } else {
                if (fmn != f0) fconst = false;
                if (ymn != y0) yconst = false;
            }
        }
        double rr = 0.0;
        bool degenerate = true;
        if (n > 0 && !fconst && !yconst) {
            double sumf = 0.0;
            for (int t = 0; t < T; ++t) {
                const double nt = static_cast<double>(*W(kfN, t));
                if (nt == 0.0) continue;
                const int kd = (*W(kfFlags, t) >> 16) & 0xff;
                sumf += nt * fit_value<FP64>(W(kfMean, t), W(kfMean + 1, t)) +
                        ldexp(word_pair<FP64>(W(kfSd, t), W(kfSd + 1, t)), kd);
            }
            const double fbar = sumf / static_cast<double>(n);
            double sff = 0.0, sy = 0.0, syy = 0.0, sfy = 0.0;
            for (int t = 0; t < T; ++t) {
                const double nt = static_cast<double>(*W(kfN, t));
                if (nt == 0.0) continue;
                const uint32_t tf = *W(kfFlags, t);
                const int kd = (tf >> 16) & 0xff, ky = (tf >> 24) & 0xff;
                const double dm = fit_value<FP64>(W(kfMean, t), W(kfMean + 1, t)) - fbar;
                const double sd = ldexp(word_pair<FP64>(W(kfSd, t), W(kfSd + 1, t)), kd);
                const double syt = ldexp(word_pair<FP64>(W(kfSy, t), W(kfSy + 1, t)), ky);
                sff += ldexp(word_pair<FP64>(W(kfSdd, t), W(kfSdd + 1, t)), 2 * kd) +
                       2.0 * dm * sd + nt * dm * dm;
                sy += syt;
                syy += ldexp(word_pair<FP64>(W(kfSyy, t), W(kfSyy + 1, t)), 2 * ky);
                sfy += ldexp(word_pair<FP64>(W(kfSdy, t), W(kfSdy + 1, t)), kd + ky) + dm * syt;
            }
            syy -= sy * sy / static_cast<double>(n);   // centre on the valid pairs' mean
            if (sff > 0.0 && syy > 0.0) {
                rr = sfy / sqrt(sff * syy);
                degenerate = false;
            }
        }
        if (degenerate) r.flags |= BEAGLE_FLAG_DEGENERATE;
        const double r2 = rr * rr;
        r.r2 = r2;
        score = M * r2 * r2 * static_cast<double>(J.N - (c1 + c2)) - M * static_cast<double>(c1 - c2);
        r.asr = score / (M * N);
    } else {
        long long tot = 0;
        for (int t = 0; t < T; ++t)
            tot += static_cast<long long>((static_cast<unsigned long long>(*W(kfScore + 1, t)) << 32) |
                                          *W(kfScore, t));
        score = static_cast<double>(tot);
        if (J.kind == kFitValidate) {
            r.asr = score / N;
            if (tot == J.N) r.flags |= BEAGLE_FLAG_PERFECT;
        } else {
            r.asr = score / (M * N);
        }
    }
    r.score = score;
    r.c1 = c1;
    r.c2 = c2;
    r.taxed_score = score - J.tax * static_cast<double>(J.lens[p]);
    J.fit[p] = r;
}


}  // namespace beagle
