// qm_noalloc.cu -- fused Philox -> normal moments without any allocation.
//
// Some callers cannot allocate device memory at the point where they need
// the moments: cudaMalloc can synchronise the device, which a latency-bound
// pipeline cannot afford; embedded runtimes plan all device memory up front
// and have no allocator to call; code that runs while a caching allocator
// holds its lock would deadlock on it.  For them this
// entry point keeps its reduction scratch in a file-scope device array that is
// part of the loaded module, so a call performs no cudaMalloc/cudaFree and no
// allocating library call.  The array (kMaxBlocks x 4 doubles = 512 KiB) lives
// on every device that loads the library until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "qm.h"
#include "qm_device.cuh"
#include "qm_host.h"

namespace qm {
namespace {

constexpr int kBlock = 256;
constexpr int kPerThread = 1024;                       // samples per thread
constexpr size_t kChunk = (size_t)kBlock * kPerThread;  // samples per block
constexpr int kMaxBlocks = 16384;                      // -> n <= 2^32

static __device__ __align__(256) double g_partials[kMaxBlocks * 4];

// Block b reduces samples [b kChunk, (b+1) kChunk) into g-scratch slot b,
// every slot it owns being overwritten (nothing needs clearing between calls).
__global__ void __launch_bounds__(kBlock)
k_moments_chunked(PhiloxKeys K, uint64_t blk0, size_t n, double* partials)
{
    const size_t first = (size_t)blockIdx.x * kChunk;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    float f1 = 0.f, f2 = 0.f, f3 = 0.f, f4 = 0.f;
    int cnt = 0;
    // thread t takes Philox blocks t, t + kBlock, ... of this chunk
    for (size_t b = threadIdx.x; b < kChunk / 4; b += kBlock) {
        const size_t i0 = first + b * 4;
        if (i0 >= n) break;
        const uint4 w = philox_block_keys(K, blk0 + first / 4 + b);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float x = (i0 + j < n) ? probit_grid24_tbl(ws[j] >> 8) : 0.0f;
            const float x2 = x * x;
            f1 += x;
            f2 += x2;
            f3 = __fmaf_rn(x2, x, f3);
            f4 = __fmaf_rn(x2, x2, f4);
        }
        if (++cnt == 16) {              // FP32 partials over 64 samples
            acc[0] += f1; acc[1] += f2; acc[2] += f3; acc[3] += f4;
            f1 = f2 = f3 = f4 = 0.f;
            cnt = 0;
        }
    }
    acc[0] += f1; acc[1] += f2; acc[2] += f3; acc[3] += f4;
    __shared__ double red[kBlock / 32][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) red[warp][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int wi = 0; wi < kBlock / 32; ++wi) v += red[wi][threadIdx.x];
        partials[(size_t)blockIdx.x * 4 + threadIdx.x] = v;
    }
}

// One warp per moment, fixed order over the nblocks slots.
__global__ void k_sum_slots(const double* partials, int nblocks, double* moments)
{
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= 4) return;
    double v = 0.0;
    for (int b = lane; b < nblocks; b += 32) v += partials[(size_t)b * 4 + k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) moments[k] = v;
}

// Device address of g_partials, looked up once per device with that device
// current (a host-side reference to g_partials is only a stand-in symbol).
double* scratch_address(qm_status* st)
{
    static std::mutex mu;
    static double* addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        *st = fail(QM_ERR_CUDA, "qm_sample_moments_noalloc: no current CUDA device");
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) {
            *st = fail(QM_ERR_CUDA, "qm_sample_moments_noalloc: cudaGetSymbolAddress: %s",
                       cudaGetErrorString(e));
            return nullptr;
        }
        addr[dev] = (double*)p;
    }
    *st = QM_OK;
    return addr[dev];
}

}  // namespace
}  // namespace qm

using namespace qm;

extern "C" qm_status qm_sample_moments_noalloc(uint64_t key, uint64_t ctr0, size_t n,
                                              double* moments4, void* stream)
{
    if (!moments4) return fail(QM_ERR_INVALID, "qm_sample_moments_noalloc: moments4 is NULL");
    if (ctr0 % 4 != 0) return fail(QM_ERR_INVALID, "qm_sample_moments_noalloc: ctr0 must be a multiple of 4");
    const size_t max_n = (size_t)kMaxBlocks * kChunk;
    if (n > max_n)
        return fail(QM_ERR_INVALID,
                    "qm_sample_moments_noalloc: n = %zu exceeds the static scratch limit of %zu samples",
                    n, max_n);
    qm_status st;
    double* scratch = scratch_address(&st);
    if (!scratch) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nblocks = n == 0 ? 0 : (int)((n + kChunk - 1) / kChunk);
    if (nblocks > 0) k_moments_chunked<<<nblocks, kBlock, 0, s>>>(philox_keys(key), ctr0 / 4, n, scratch);
    k_sum_slots<<<1, 128, 0, s>>>(scratch, nblocks, moments4);
    return check_launch("moments (no allocation)");
}
