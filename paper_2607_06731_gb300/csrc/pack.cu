// The packing kernel: each program of a call translated into interpreter handlers once (the
// warp-cooperative packer of score.cuh: the program checked, leaves fused with the binary
// operator after them, the stack row of every handler), instead of once per case tile by
// every work item that meets it. Work items then copy the packed tokens into shared memory.
// On the FP32 path the kernel first folds constant subexpressions (below).
#include "kernels.h"
#include "score.cuh"

namespace beagle {

namespace {

// ------------------------------------------------------------------ constant folding
// An operator whose operands are all constants (leaves, or results of such operators) gives
// the same value on every fitness case: the packing kernel evaluates it once, with the very
// operations the interpreter would run (Arith<float>: the .rn adds and products, the same
// protected division, square root and log, the same sin, cos and CUDA functions), and the
// program carries the result as one constant. Every case's output keeps its bits; a folded
// value that fails the validity rule makes the program invalid, as it would on every case.
// FP32 path only: a folded double could not travel in the program's fp32 constants.
// Programs using DUP, SWAP, DEL or the COPY / PASTE registers are not folded.
__device__ __forceinline__ float fold_unary(int op, float a) {
    using A = Arith<float>;
    switch (op) {
    case OP_SIN: return A::sin_(a);
    case BEAGLE_OP_COS: return A::cos_(a);
    case BEAGLE_OP_EXP: return A::exp_(a);
    case BEAGLE_OP_PLOG: return A::plog(a);
    case BEAGLE_OP_PSQRT: return A::psqrt(a);
    case OP_SQUARE: return __fmul_rn(a, a);
    case OP_SIGN: return -a;
    case BEAGLE_OP_CUBE: return A::cube(a);
    case BEAGLE_OP_CBRT: return A::cbrt_(a);
    case BEAGLE_OP_TAN: return A::tan_(a);
    case BEAGLE_OP_ASIN: return A::asin_(a);
    case BEAGLE_OP_ACOS: return A::acos_(a);
    case BEAGLE_OP_ATAN: return A::atan_(a);
    default: return A::tanh_(a);
    }
}

__device__ __forceinline__ float fold_binary(int op, float a, float b) {   // a op b, b the top
    using A = Arith<float>;
    switch (op) {
    case OP_ADD: return __fadd_rn(a, b);
    case OP_SUB: return __fsub_rn(a, b);
    case OP_MUL: return __fmul_rn(a, b);
    case OP_PDIV: return A::pdiv(a, b);
    default: return A::pow_(a, b);
    }
}

// Per-warp shared-memory copy of a program being folded.
struct FoldBuf {
    uint8_t ops[kMaxLen + 32];
    uint8_t kill[kMaxLen + 32];
    uint8_t set[kMaxLen + 32];
    float cs[kMaxLen + 32];
    float nv[kMaxLen + 32];
};

__device__ __forceinline__ bool fold_unary_op(int op) {
    return (op >= OP_SIN && op <= OP_SQUARE) || (op >= OP_SIGN && op <= OP_TANH);
}
__device__ __forceinline__ bool fold_binary_op(int op) {
    return (op >= OP_ADD && op <= OP_PDIV) || op == OP_POW;
}

// Warp-cooperative folding of the program in fb (n tokens): passes of local rewrites, each
// pass replacing every "CONST unary" by one CONST and every "CONST CONST binary" by one
// CONST (in postfix the operands of an operator whose operands are all constants end up as
// adjacent CONSTs, so the passes fold every constant subexpression; the matches of one pass
// never share a token). Only programs of leaves, unary and binary operators that the packer
// would accept at a depth of at most kMaxDepth are folded, so a program is malformed exactly
// when it was (a deep one may become shallow and run in the fast pass: the same bits). Returns
// the new length, or -1 when nothing was folded; *bad: a constant or folded value fails the
// validity rule.
__device__ int warp_fold(FoldBuf &fb, int n, int d, int lane, bool *bad) {
    // the program's shape: operator classes, operands present, depth at most kMaxDepth, one
    // value left
    int depth = 0;
    bool ok = true;
    for (int base = 0; base < n; base += 32) {
        const int j = base + lane;
        const bool in = j < n;
        const int op = in ? fb.ops[j] : 0;
        const bool cst = op == OP_CONST, var = op >= OP_LOAD0 && op < OP_LOAD0 + BEAGLE_MAX_VARS;
        const bool un = fold_unary_op(op), bin = fold_binary_op(op);
        int delta = (cst || var) ? 1 : bin ? -1 : 0;
        if (!in) delta = 0;
        if (in && !(cst || un || bin || (var && op - OP_LOAD0 < d))) ok = false;
        int inc = delta;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += t;
        }
        const int after = depth + inc, before = after - delta;
        if (in && (before < (bin ? 2 : un ? 1 : 0) || after > kMaxDepth)) ok = false;
        depth = __shfl_sync(kFull, after, 31);
    }
    if (!__all_sync(kFull, ok) || depth != 1) return -1;
    bool any_fold = false, b = false;
    for (int base = 0; base < n; base += 32) {
        const int j = base + lane;
        if (j < n) {
            fb.kill[j] = 0;
            fb.set[j] = 0;
        }
    }
    __syncwarp();
    for (int pass = 0; pass < 32; ++pass) {
        // decisions (reads only), then the rewrite with compaction (which clears the flags)
        bool folded = false;
        for (int base = 0; base < n; base += 32) {
            const int j = base + lane;
            if (j < n) {
                const int op = fb.ops[j];
                if (j >= 1 && fold_unary_op(op) && fb.ops[j - 1] == OP_CONST) {
                    const float c = fb.cs[j - 1];
                    if (!(fabsf(c) <= Arith<float>::kBig)) b = true;
                    const float v = fold_unary(op, c);
                    if (!(fabsf(v) <= Arith<float>::kBig)) b = true;
                    fb.kill[j] = 1;
                    fb.set[j - 1] = 1;
                    fb.nv[j - 1] = v;
                    folded = true;
                } else if (j >= 2 && fold_binary_op(op) && fb.ops[j - 1] == OP_CONST &&
                           fb.ops[j - 2] == OP_CONST) {
                    const float c0 = fb.cs[j - 2], c1 = fb.cs[j - 1];
                    if (!(fabsf(c0) <= Arith<float>::kBig) || !(fabsf(c1) <= Arith<float>::kBig))
                        b = true;
                    const float v = fold_binary(op, c0, c1);
                    if (!(fabsf(v) <= Arith<float>::kBig)) b = true;
                    fb.kill[j] = 1;
                    fb.kill[j - 1] = 1;
                    fb.set[j - 2] = 1;
                    fb.nv[j - 2] = v;
                    folded = true;
                }
            }
        }
        __syncwarp();
        if (!__any_sync(kFull, folded)) break;
        any_fold = true;
        int out = 0;
        for (int base = 0; base < n; base += 32) {
            const int j = base + lane;
            const bool in = j < n;
            const bool keep = in && !fb.kill[j];
            const uint8_t op = in ? fb.ops[j] : 0;
            const float c = in ? (fb.set[j] ? fb.nv[j] : fb.cs[j]) : 0.0f;
            const unsigned m = __ballot_sync(kFull, keep);
            __syncwarp();
            if (in) {
                fb.kill[j] = 0;
                fb.set[j] = 0;
            }
            if (keep) {
                const int pos = out + __popc(m & ((1u << lane) - 1u));
                fb.ops[pos] = op;
                fb.cs[pos] = c;
            }
            out += __popc(m);
            __syncwarp();
        }
        n = out;
    }
    *bad = __any_sync(kFull, b);
    return any_fold ? n : -1;
}

// One warp per program (grid-stride over the positions of each job's order). The next
// handler's id goes into bits 24-28 of each token (the inline-PTX interpreters branch on it
// while they load that token); a program deeper than the fast pass's stack is appended to its
// job's deep list here, once.
// Packing: one warp per position (grid-stride). On the FP32 path the warp first copies the
// program into shared memory and folds it there.
template <typename T, int MAXJ>
__global__ void __launch_bounds__(256) pack_kernel(const __grid_constant__ LaunchParams<MAXJ> prm,
                                                   int fold) {
    __shared__ FoldBuf bufs[sizeof(T) == 4 ? 8 : 1];
    const int lane = threadIdx.x & 31;
    FoldBuf &fb = bufs[sizeof(T) == 4 ? (threadIdx.x >> 5) : 0];
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int j = 0; j < prm.njobs; ++j) {
        const JobDev &J = prm.jobs[j];
        if (!J.packed) continue;
        for (int64_t q = warp; q < J.P; q += nwarps) {
            const uint32_t off = J.poff[q];
            if (off == kPackNone) {
                if (lane == 0) J.pmeta[q] = kPackNone;
                continue;
            }
            const int64_t p = J.order[q];
            const int64_t o = J.offs[p];
            const int L = J.lens[p];
            uint2 *buf = J.packed + off;
            int lf = -1;
            bool fbad = false;
            if (sizeof(T) == 4 && fold && L >= 1 && L <= kMaxLen) {
                for (int i = lane; i < L; i += 32) {
                    fb.ops[i] = J.ops[o + i];
                    fb.cs[i] = J.consts[o + i];
                }
                __syncwarp();
                lf = warp_fold(fb, L, J.d, lane, &fbad);
            }
            // from the shared-memory copy (folded or not) on the FP32 path
            const bool copy = sizeof(T) == 4 && fold && L >= 1 && L <= kMaxLen;
            const Packed pk = copy
                ? pack_program<T, kDepthFast>(fb.ops, fb.cs, lf >= 0 ? lf : L, J.d, buf, lane)
                : pack_program<T, kDepthFast>(J.ops + o, J.consts + o, L, J.d, buf, lane);
            for (int base = 0; base < pk.n; base += 32) {
                const int k = base + lane;
                const uint32_t nh = k < pk.n ? (buf[k + 1].x & 31u) : 0u;
                __syncwarp();
                if (k < pk.n) buf[k].x |= nh << 24;
                __syncwarp();
            }
            if (lane == 0) {
                const bool cbad = pk.const_bad || fbad;
                J.pmeta[q] = static_cast<uint32_t>(pk.n) | (pk.malformed ? kPackMalformed : 0u) |
                             (pk.deep ? kPackDeep : 0u) | (cbad ? kPackConstBad : 0u);
                if (pk.deep && !pk.malformed && J.deep_list)
                    J.deep_list[atomicAdd(J.deep_count, 1)] = static_cast<int32_t>(p);
            }
            __syncwarp();
        }
    }
}

}  // namespace

template <int MAXJ>
cudaError_t launch_pack(const LaunchParams<MAXJ> &prm, int precision, cudaStream_t s) {
    int64_t total = 0;
    for (int j = 0; j < prm.njobs; ++j)
        if (prm.jobs[j].packed) total += prm.jobs[j].P;
    if (total == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // 8 warps a block, at most 8 blocks an SM: a warp per program while that fills the GPU
    const int64_t blocks = (total + 7) / 8;
    const int grid = static_cast<int>(blocks < 8LL * sms ? blocks : 8LL * sms);
    if (precision == BEAGLE_FP64) pack_kernel<double, MAXJ><<<grid, 256, 0, s>>>(prm, 0);
    else pack_kernel<float, MAXJ><<<grid, 256, 0, s>>>(prm, 1);
    return cudaGetLastError();
}

template cudaError_t launch_pack<1>(const LaunchParams<1> &, int, cudaStream_t);
template cudaError_t launch_pack<kMaxJobs>(const LaunchParams<kMaxJobs> &, int, cudaStream_t);

}  // namespace beagle
