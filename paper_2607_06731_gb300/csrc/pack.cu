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
struct FoldEnt {
    float v;
    bool pend;   // a constant not yet emitted (only the top of the stack can hold these)
};

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

// Fold program (ops, cs, L) into (fo, fc); returns its new length, or -1 to keep the program
// as it is: nothing to fold, a register (COPY / PASTE) program, or a structural fault (the
// packer then flags the original), so a program is malformed exactly when it was (a deep one
// may become shallow and run in the fast pass: the bits are the same). *bad is set when a
// constant or folded value fails the validity rule.
__device__ int fold_program(const uint8_t *ops, const float *cs, int L, uint8_t *fo, float *fc,
                            bool *bad) {
    FoldEnt st[kMaxDepth + 1];
    int sp = 0, out = 0, folded = 0;
    bool b = false;
    auto check = [&](float v) { if (!(fabsf(v) <= Arith<float>::kBig)) b = true; };
    auto flush = [&]() {   // emit the pending constants on top of the stack, bottom first
        int k = sp;
        while (k > 0 && st[k - 1].pend) --k;
        for (; k < sp; ++k) {
            fo[out] = static_cast<uint8_t>(OP_CONST);
            fc[out++] = st[k].v;
            st[k].pend = false;
        }
    };
    for (int j = 0; j < L; ++j) {
        const int op = ops[j];
        if (op == OP_CONST) {
            if (sp >= kMaxDepth) return -1;
            st[sp++] = FoldEnt{cs[j], true};
            check(cs[j]);
        } else if (op >= OP_LOAD0 && op < OP_LOAD0 + BEAGLE_MAX_VARS) {
            if (sp >= kMaxDepth) return -1;
            flush();
            fo[out] = static_cast<uint8_t>(op);
            fc[out++] = 0.0f;
            st[sp++] = FoldEnt{0.0f, false};
        } else if ((op >= OP_SIN && op <= OP_SQUARE) || (op >= OP_SIGN && op <= OP_TANH)) {
            if (sp < 1) return -1;
            if (st[sp - 1].pend) {
                const float v = fold_unary(op, st[sp - 1].v);
                check(v);
                st[sp - 1].v = v;
                ++folded;
            } else {
                fo[out] = static_cast<uint8_t>(op);
                fc[out++] = 0.0f;
            }
        } else if ((op >= OP_ADD && op <= OP_PDIV) || op == OP_POW) {
            if (sp < 2) return -1;
            if (st[sp - 2].pend && st[sp - 1].pend) {
                const float v = fold_binary(op, st[sp - 2].v, st[sp - 1].v);
                check(v);
                --sp;
                st[sp - 1].v = v;
                ++folded;
            } else {
                flush();
                fo[out] = static_cast<uint8_t>(op);
                fc[out++] = 0.0f;
                --sp;
                st[sp - 1] = FoldEnt{0.0f, false};
            }
        } else if (op == OP_DUP) {
            if (sp < 1 || sp >= kMaxDepth) return -1;
            if (st[sp - 1].pend) {
                st[sp] = st[sp - 1];
                ++sp;
                ++folded;
            } else {
                fo[out] = static_cast<uint8_t>(op);
                fc[out++] = 0.0f;
                st[sp++] = FoldEnt{0.0f, false};
            }
        } else if (op == OP_SWAP) {
            if (sp < 2) return -1;
            if (st[sp - 2].pend && st[sp - 1].pend) {
                const FoldEnt t = st[sp - 1];
                st[sp - 1] = st[sp - 2];
                st[sp - 2] = t;
                ++folded;
            } else {
                flush();
                fo[out] = static_cast<uint8_t>(op);
                fc[out++] = 0.0f;
            }
        } else if (op == OP_DEL) {
            if (sp < 1) return -1;
            if (st[sp - 1].pend) {
                --sp;
                ++folded;
            } else {
                fo[out] = static_cast<uint8_t>(op);
                fc[out++] = 0.0f;
                --sp;
            }
        } else {
            // COPY / PASTE (their depth rule counts the stack as the program writes it) and
            // unknown opcodes: the program is packed as it is
            return -1;
        }
    }
    if (sp != 1 || folded == 0) return -1;
    flush();
    *bad = b;
    return out;
}

// One warp per program (grid-stride over the positions of each job's order). The next
// handler's id goes into bits 24-28 of each token (the inline-PTX interpreters branch on it
// while they load that token); a program deeper than the fast pass's stack is appended to its
// job's deep list here, once.
template <typename T, int MAXJ>
__global__ void __launch_bounds__(256) pack_kernel(const __grid_constant__ LaunchParams<MAXJ> prm,
                                                   uint8_t *fold_ops, float *fold_cs) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int j = 0; j < prm.njobs; ++j) {
        const JobDev &J = prm.jobs[j];
        if (!J.packed) continue;
        const uint8_t *fops = fold_ops ? fold_ops + J.fold_base : nullptr;
        const float *fcs = fold_cs ? fold_cs + J.fold_base : nullptr;
        // 32 positions a warp at a time: each lane folds one program (FP32), then the warp
        // packs the 32 one after another
        for (int64_t q0 = warp * 32; q0 < J.P; q0 += nwarps * 32) {
            const int64_t ql = q0 + lane;
            int lf = -1;
            bool fbad = false;
            uint32_t offl = kPackNone;
            if (ql < J.P) offl = J.poff[ql];
            if constexpr (sizeof(T) == 4) {
                if (fops && offl != kPackNone) {
                    const int64_t p = J.order[ql];
                    const int64_t o = J.offs[p];
                    lf = fold_program(J.ops + o, J.consts + o, J.lens[p],
                                      fold_ops + J.fold_base + offl, fold_cs + J.fold_base + offl,
                                      &fbad);
                }
            }
            __syncwarp();
            const int n = static_cast<int>(min(static_cast<int64_t>(32), J.P - q0));
            for (int i = 0; i < n; ++i) {
                const int64_t q = q0 + i;
                const uint32_t off = __shfl_sync(kFull, offl, i);
                const int qlf = __shfl_sync(kFull, lf, i);
                const bool qbad = __shfl_sync(kFull, fbad ? 1 : 0, i) != 0;
                if (off == kPackNone) {
                    if (lane == 0) J.pmeta[q] = kPackNone;
                    continue;
                }
                const int64_t p = J.order[q];
                const int64_t o = J.offs[p];
                uint2 *buf = J.packed + off;
                const Packed pk =
                    qlf >= 0 ? pack_program<T, kDepthFast>(fops + off, fcs + off, qlf, J.d, buf, lane)
                             : pack_program<T, kDepthFast>(J.ops + o, J.consts + o, J.lens[p], J.d,
                                                           buf, lane);
                for (int base = 0; base < pk.n; base += 32) {
                    const int k = base + lane;
                    const uint32_t nh = k < pk.n ? (buf[k + 1].x & 31u) : 0u;
                    __syncwarp();
                    if (k < pk.n) buf[k].x |= nh << 24;
                    __syncwarp();
                }
                if (lane == 0) {
                    const bool cbad = pk.const_bad || qbad;
                    J.pmeta[q] = static_cast<uint32_t>(pk.n) | (pk.malformed ? kPackMalformed : 0u) |
                                 (pk.deep ? kPackDeep : 0u) | (cbad ? kPackConstBad : 0u);
                    if (pk.deep && !pk.malformed && J.deep_list)
                        J.deep_list[atomicAdd(J.deep_count, 1)] = static_cast<int32_t>(p);
                }
            }
        }
    }
}

}  // namespace

template <int MAXJ>
cudaError_t launch_pack(const LaunchParams<MAXJ> &prm, int precision, uint8_t *fold_ops,
                        float *fold_cs, cudaStream_t s) {
    int64_t total = 0;
    for (int j = 0; j < prm.njobs; ++j)
        if (prm.jobs[j].packed) total += prm.jobs[j].P;
    if (total == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // 8 warps a block, at most 8 blocks an SM: a warp per 32 programs while that fills the GPU
    const int64_t blocks = (total + 255) / 256;
    const int grid = static_cast<int>(blocks < 8LL * sms ? blocks : 8LL * sms);
    if (precision == BEAGLE_FP64) pack_kernel<double, MAXJ><<<grid, 256, 0, s>>>(prm, nullptr, nullptr);
    else pack_kernel<float, MAXJ><<<grid, 256, 0, s>>>(prm, fold_ops, fold_cs);
    return cudaGetLastError();
}

template cudaError_t launch_pack<1>(const LaunchParams<1> &, int, uint8_t *, float *,
                                    cudaStream_t);
template cudaError_t launch_pack<kMaxJobs>(const LaunchParams<kMaxJobs> &, int, uint8_t *,
                                           float *, cudaStream_t);

}  // namespace beagle
