// lbm_noalloc.cu -- conserved totals of a population array, computed without
// allocating any memory (entry point lbm_totals_noalloc, declared in include/lbm.h).
//
// It is a variant of the FP64 reduction behind lbm_observables: that one keeps its
// per-block partial sums in device memory owned by a context; this one keeps them
// in a fixed-size array at file scope, so a caller that must not call cudaMalloc
// can still reduce a population array it owns.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbm {
void set_global_error(const std::string& msg);
}

namespace {

using lbm::Q;
using lbm::cx;
using lbm::cy;
using lbm::cz;

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 16384;             // partial-sum slots in the scratch array
constexpr long long kNodesPerBlock = 8192;    // nodes one block reduces
constexpr int kSlot = 8;                      // doubles per slot (5 used)
constexpr long long kMaxNodes = (long long)kMaxBlocks * kNodesPerBlock;   // 512^3

// Scratch of every call (1 MiB, held by each device that loads the library).
static __device__ __align__(256) double g_partials[kMaxBlocks * kSlot];

// Device address of g_partials, looked up once per device.
constexpr int kMaxDevices = 64;
double* g_partials_ptr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

// Sum of NV per-thread values over the block, written to out[0..NV): warp shuffles,
// then the warps of the block in index order (a fixed order: deterministic).
template <int NV>
__device__ inline void block_sum(double (&v)[NV], double* out) {
    __shared__ double sh[kThreads / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0;
        for (int w = 0; w < kThreads / 32; ++w) s += sh[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// Block b sums nodes [b * kNodesPerBlock, (b+1) * kNodesPerBlock) into slot b:
// sum f^r, sum f^b and the momentum sum_i c_i (f^r_i + f^b_i).
__global__ void partial_kernel(const float* __restrict__ f, long long n, double* partials) {
    double v[5] = {0, 0, 0, 0, 0};
    const long long n0 = (long long)blockIdx.x * kNodesPerBlock;
    const long long n1 = n0 + kNodesPerBlock < n ? n0 + kNodesPerBlock : n;
    for (long long m = n0 + threadIdx.x; m < n1; m += kThreads) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double a = f[(size_t)i * n + m];
            const double b = f[(size_t)(Q + i) * n + m];
            v[0] += a;
            v[1] += b;
            v[2] += cx(i) * (a + b);
            v[3] += cy(i) * (a + b);
            v[4] += cz(i) * (a + b);
        }
    }
    block_sum<5>(v, partials + (size_t)blockIdx.x * kSlot);
}

// One block adds the slots of this call in index order and writes the result.
__global__ void final_kernel(const double* partials, int nblocks, double* out) {
    double v[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] += partials[(size_t)b * kSlot + k];
    block_sum<5>(v, out);
}

}  // namespace

extern "C" lbm_status lbm_totals_noalloc(const float* pops, long long n_nodes, double* out,
                                         void* cuda_stream) {
    if (!pops || !out) {
        lbm::set_global_error("lbm_totals_noalloc: pops and out are required");
        return LBM_EINVAL;
    }
    if (n_nodes < 1 || n_nodes > kMaxNodes) {
        lbm::set_global_error("lbm_totals_noalloc: n_nodes must be in [1, " +
                              std::to_string(kMaxNodes) + "] (the size of its fixed scratch)");
        return LBM_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        lbm::set_global_error(std::string("lbm_totals_noalloc: no usable CUDA device: ") +
                              cudaGetErrorString(e));
        return LBM_ECUDA;
    }
    double* partials = nullptr;
    {
        // first call on this device (which is current): look up the scratch address
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_partials);
            if (e != cudaSuccess || !ptr) {
                lbm::set_global_error(std::string("lbm_totals_noalloc: cudaGetSymbolAddress: ") +
                                      cudaGetErrorString(e));
                return LBM_ECUDA;
            }
            g_partials_ptr[dev] = static_cast<double*>(ptr);
        }
        partials = g_partials_ptr[dev];
    }
    const int nblocks = (int)((n_nodes + kNodesPerBlock - 1) / kNodesPerBlock);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    partial_kernel<<<nblocks, kThreads, 0, s>>>(pops, n_nodes, partials);
    final_kernel<<<1, kThreads, 0, s>>>(partials, nblocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        lbm::set_global_error(std::string("lbm_totals_noalloc: launch: ") + cudaGetErrorString(e));
        return LBM_ECUDA;
    }
    return LBM_OK;
}
