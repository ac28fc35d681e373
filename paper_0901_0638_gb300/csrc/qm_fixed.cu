// qm_fixed.cu -- FP64 normal quantile from the exponential-coordinate segment
// table evaluated in 64-bit fixed point (QM_VAR_FIXED, the FP64 default); the
// method is described in qm_fx.cuh.  GB300 issues FP64 at about 1/62 of its
// FP32 rate; the integer pipes carry the segment polynomial, and one FP64 FMA
// per element remains.  A segment's 48 bytes sit in two arrays and arrive in
// one 256-bit and one 128-bit load (each lane gathers a random segment, and
// the L1 cost of a gather grows with the number of load instructions).
//
// Every 0 < u < 1 (subnormal u included) takes the same path: every binade
// e = -1 - E = 0 .. 1072 (x = 2d down to 2^-1073) has 64 segments.
// u = 1/2 gives +0, u = 0 gives -inf, u = 1 gives +inf, anything else NaN.
// This file holds the table (qm_fx_tables.h); fx_table_device() gives its
// device address to the kernels of other files.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "qm.h"
#include "qm_fx_tables.h"
#include "qm_host.h"

namespace qm {
namespace {

constexpr int kBlock = 128;

// Sixteen blocks of 128 per SM (32 registers, full occupancy): more warps to
// cover the latency of the table gathers (eight blocks measured 0.6 % faster
// than six, and sixteen blocks of 128 0.9 % faster than eight of 256).
template <int U>
__global__ void __launch_bounds__(kBlock, 16)
k_f64_fixed(const double* __restrict__ in, double* out, size_t n)
{
    const size_t nv = n / 2;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const double2* vin = reinterpret_cast<const double2*>(in);
    double2* vout = reinterpret_cast<double2*>(out);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride * U) {
        double2 a[U];
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (i + k * stride < nv) a[k] = __ldcs(vin + i + k * stride);
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (i + k * stride < nv)
                __stcs(vout + i + k * stride, make_double2(probit_fx(&fxt::SEG_FX, a[k].x), probit_fx(&fxt::SEG_FX, a[k].y)));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) out[n - 1] = probit_fx(&fxt::SEG_FX, in[n - 1]);
}

__global__ void __launch_bounds__(kBlock)
k_f64_fixed_scalar(const double* in, double* out, size_t n)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = probit_fx(&fxt::SEG_FX, in[i]);
}

template <class Kern>
int grid_of(Kern k, size_t items, int waves = 1)
{
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kBlock, 0) != cudaSuccess || bps < 1)
        bps = 1;
    const int sms = sm_count() > 0 ? sm_count() : 1;
    size_t g = (items + kBlock - 1) / kBlock;
    const size_t cap = (size_t)sms * bps * waves;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

// Launch on `s`; u and z are device arrays of n doubles (in place allowed).
qm_status launch_f64_fixed(const double* u, double* z, size_t n, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if ((uintptr_t)u % 16 == 0 && (uintptr_t)z % 16 == 0) {
        // one double2 per thread per pass over a grid of up to 64 x the
        // resident blocks (measured on the tail-stress mixture: 1, 4, 16, 64
        // waves give 188.0, 220.9, 229.7, 230.8 Gs/s; a plain device copy
        // also gains from more waves, 6494 -> 7061 GB/s)
        const int g = grid_of(k_f64_fixed<1>, n / 2, 64);
        k_f64_fixed<1><<<g, kBlock, 0, s>>>(u, z, n);
    } else {
        const int g = grid_of(k_f64_fixed_scalar, n, 16);
        k_f64_fixed_scalar<<<g, kBlock, 0, s>>>(u, z, n);
    }
    return check_launch("f64 fixed");
}

// Device address of the table on the current device (looked up once per
// device), for kernels compiled in other files.
const void* fx_table_device(qm_status* st)
{
    static std::mutex mu;
    static const void* addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        *st = fail(QM_ERR_CUDA, "fixed-point table: no current CUDA device");
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, fxt::SEG_FX) != cudaSuccess) {
            *st = fail(QM_ERR_CUDA, "fixed-point table: address lookup failed");
            return nullptr;
        }
        addr[dev] = p;
    }
    *st = QM_OK;
    return addr[dev];
}

}  // namespace qm
