// Device FMA-rate measurement (no counterpart in the paper): the roofline
// denominators of the ALU-bound force kernels.  Every thread of a grid that
// fills the device runs eight independent FMA chains, so the issue rate, not
// latency, bounds it; the result is written out so nothing is dead code.
#include "kernels.h"

namespace lqcd {
namespace {

constexpr int kChains = 8;
constexpr int kPeakBlock = 256;

template <typename R> __global__ void __launch_bounds__(kPeakBlock) fma_chains(R *out, int iters, R a, R b)
{
    R x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = R(threadIdx.x + c) * R(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    R s = R(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

} // namespace

cudaError_t measure_fma_rate(int precision, void *scratch, size_t scratch_bytes, double *tflops,
                             cudaStream_t st)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const bool f64 = precision == LQCD_F64;
    e = f64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chains<double>, kPeakBlock, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chains<float>, kPeakBlock, 0);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const size_t need = (size_t)blocks * kPeakBlock * (f64 ? 8 : 4);
    if (scratch == nullptr || scratch_bytes < need) return cudaErrorInvalidValue;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // calibrate on a short run, then time one run of about 20 ms
    int iters = 64;
    float ms = 0.f;
    for (int pass = 0; pass < 3 && e == cudaSuccess; ++pass) {
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (f64) fma_chains<double><<<(unsigned)blocks, kPeakBlock, 0, st>>>(static_cast<double *>(scratch), iters, 0.999999, 1e-7);
        else fma_chains<float><<<(unsigned)blocks, kPeakBlock, 0, st>>>(static_cast<float *>(scratch), iters, 0.9999f, 1e-4f);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess || pass == 2) break;
        const double scale = 20.0 / (ms > 1e-3f ? ms : 1e-3f);
        double next = iters * (scale < 1024.0 ? scale : 1024.0);
        if (next < 64) next = 64;
        if (next > (1 << 24)) next = 1 << 24;
        iters = (int)next;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * kChains * 16.0 * (double)iters * (double)blocks * kPeakBlock;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return cudaSuccess;
}

size_t fma_rate_scratch_bytes() { return (size_t)1 << 24; }

} // namespace lqcd
