// The packing kernel: each program of a call translated into interpreter handlers once (the
// warp-cooperative packer of score.cuh: the program checked, leaves fused with the binary
// operator after them, the stack row of every handler), instead of once per case tile by
// every work item that meets it. Work items then copy the packed tokens into shared memory.
#include "kernels.h"
#include "score.cuh"

namespace beagle {

namespace {

// One warp per program (grid-stride over the positions of each job's order). The next
// handler's id goes into bits 24-28 of each token (the inline-PTX interpreters branch on it
// while they load that token); a program deeper than the fast pass's stack is appended to its
// job's deep list here, once.
template <typename T, int MAXJ>
__global__ void __launch_bounds__(256) pack_kernel(const __grid_constant__ LaunchParams<MAXJ> prm) {
    const int lane = threadIdx.x & 31;
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
            uint2 *buf = J.packed + off;
            const Packed pk = pack_program<T, kDepthFast>(J.ops + o, J.consts + o, J.lens[p],
                                                          J.d, buf, lane);
            for (int base = 0; base < pk.n; base += 32) {
                const int i = base + lane;
                const uint32_t nh = i < pk.n ? (buf[i + 1].x & 31u) : 0u;
                __syncwarp();
                if (i < pk.n) buf[i].x |= nh << 24;
                __syncwarp();
            }
            if (lane == 0) {
                J.pmeta[q] = static_cast<uint32_t>(pk.n) | (pk.malformed ? kPackMalformed : 0u) |
                             (pk.deep ? kPackDeep : 0u) | (pk.const_bad ? kPackConstBad : 0u);
                if (pk.deep && !pk.malformed && J.deep_list)
                    J.deep_list[atomicAdd(J.deep_count, 1)] = static_cast<int32_t>(p);
            }
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
    if (precision == BEAGLE_FP64) pack_kernel<double, MAXJ><<<grid, 256, 0, s>>>(prm);
    else pack_kernel<float, MAXJ><<<grid, 256, 0, s>>>(prm);
    return cudaGetLastError();
}

template cudaError_t launch_pack<1>(const LaunchParams<1> &, int, cudaStream_t);
template cudaError_t launch_pack<kMaxJobs>(const LaunchParams<kMaxJobs> &, int, cudaStream_t);

}  // namespace beagle
