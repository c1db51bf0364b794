// Gauge action S_G = (beta/3) sum_n sum_{34 loops P} c_P [3 - Re tr P_n]
// (paper Eq. 18_6_4_1, loops of Eq. 18_3_27_30) and the kinetic term
// K = (1/2) sum p^2 of the MD Hamiltonian, as deterministic FP64 reductions:
// every thread sums its sites in double, warps reduce by shuffles, blocks
// write one partial each to the caller's workspace, and one block adds the
// partials in a fixed order.  The grid is a fixed multiple of the SM count,
// so the summation order -- and the result, bit for bit -- is reproducible.
#include <cmath>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"
#include "su3.cuh"

namespace lqcd {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double warp_part[kBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_part[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (warp == 0) {
        s = lane < kBlock / 32 ? warp_part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s; // valid in thread 0
}

// U_{x,d} for d = +-(mu+1), and x advanced to x + hat(d).
template <typename R>
__device__ __forceinline__ Mat<R> walk(const R *__restrict__ links, const Geom &g, Coord &x, int d)
{
    if (d > 0) {
        const Mat<R> m = load_link(links, g.V, d - 1, index_of(g, x));
        step(g, x, d - 1, 1);
        return m;
    }
    step(g, x, -d - 1, -1);
    return dagger(load_link(links, g.V, -d - 1, index_of(g, x)));
}

template <typename R>
__global__ void __launch_bounds__(kBlock) action_partials(const ReduceArgs a, const LoopTable tab)
{
    const Geom g = make_geom(a.dims);
    const R *__restrict__ links = static_cast<const R *>(a.links);
    double acc = 0.0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < g.V;
         n += (int64_t)gridDim.x * blockDim.x) {
        const Coord x0 = coord_of(g, n);
        for (int l = 0; l < tab.count; ++l) {
            const Loop &lp = tab.l[l];
            Coord x = x0;
            Mat<R> m = walk(links, g, x, lp.d[0]);
            for (int j = 1; j < lp.len - 1; ++j) m = mul<N, N>(m, walk(links, g, x, lp.d[j]));
            const R retr = re_trace_mul<N, N>(m, walk(links, g, x, lp.d[lp.len - 1]));
            const double c = lp.cls == 0 ? a.c[0] : (lp.cls == 1 ? a.c[1] : a.c[2]);
            acc += c * (3.0 - (double)retr);
        }
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = s;
}

template <typename R> __global__ void __launch_bounds__(kBlock) kinetic_partials(const ReduceArgs a)
{
    const Geom g = make_geom(a.dims);
    const R *__restrict__ mom = static_cast<const R *>(a.mom);
    double acc = 0.0;
    const int64_t nlinks = 4 * g.V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlinks;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int mu = (int)(i / g.V);
        const int64_t n = i - mu * g.V;
        R p[8];
        load_algebra(mom, g.V, mu, n, p);
#pragma unroll
        for (int c = 0; c < 8; ++c) acc += 0.5 * (double)p[c] * (double)p[c];
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = s;
}

// One block of 1024 threads adds the partials in a fixed order and scales
// the total.
constexpr int kFinish = 1024;
__global__ void __launch_bounds__(kFinish) finish_sum(const double *partials, int count,
                                                      double scale, double *out)
{
    __shared__ double warp_part[kFinish / 32];
    double v = 0.0;
    for (int i = threadIdx.x; i < count; i += kFinish) v += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double s = warp_part[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) *out = scale * s;
    }
}

// Departure of the stored links from SU(3), in FP64 whatever the storage
// precision: with rows r0, r1 stored and r2 = conj(r0 x r1) rebuilt (so r2
// is orthogonal to both and det U = |r2|^2), U^dag U = 1 and det U = 1 hold
// exactly when |r0|^2 = |r1|^2 = 1 and <r0, r1> = 0; the measure is
// max(| |r0|^2 - 1 |, | |r1|^2 - 1 |, |<r0, r1>|, | |r2|^2 - 1 |) over links.
template <typename R> __global__ void __launch_bounds__(kBlock) unitarity_partials(const ReduceArgs a)
{
    const Geom g = make_geom(a.dims);
    const R *__restrict__ links = static_cast<const R *>(a.links);
    double worst = 0.0;
    const int64_t nlinks = 4 * g.V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlinks;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int mu = (int)(i / g.V);
        const int64_t n = i - mu * g.V;
        const Mat<R> u = load_link(links, g.V, mu, n);
        double n0 = 0.0, n1 = 0.0, cr = 0.0, ci = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double ar = u.re[0][j], ai = u.im[0][j], br = u.re[1][j], bi = u.im[1][j];
            n0 += ar * ar + ai * ai;
            n1 += br * br + bi * bi;
            cr += ar * br + ai * bi; // <r0, r1> = sum conj(a) b
            ci += ar * bi - ai * br;
        }
        const double c2 = cr * cr + ci * ci;
        const double d = fmax(fmax(fabs(n0 - 1.0), fabs(n1 - 1.0)),
                              fmax(sqrt(c2), fabs(n0 * n1 - c2 - 1.0)));
        worst = fmax(worst, d);
    }
    __shared__ double warp_part[kBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_down_sync(0xffffffffu, worst, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_part[warp] = worst;
    __syncthreads();
    if (warp == 0) {
        double m = lane < kBlock / 32 ? warp_part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        if (lane == 0) a.partials[blockIdx.x] = m;
    }
}

__global__ void __launch_bounds__(kFinish) finish_max(const double *partials, int count, double *out)
{
    __shared__ double warp_part[kFinish / 32];
    double v = 0.0;
    for (int i = threadIdx.x; i < count; i += kFinish) v = fmax(v, partials[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double m = warp_part[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        if (lane == 0) *out = m;
    }
}

// Library-held scratch of the allocation-free action entry point: one double
// per reduction block.  4096 doubles = 32 KiB, held by every device that
// loads the library until the process exits.
constexpr int kFixedPartials = 4096;
static __device__ __align__(256) double g_fixed_partials[kFixedPartials];

} // namespace

int reduction_blocks(int device)
{
    static std::mutex mu;
    static int cached[64] = {0};
    if (device < 0 || device >= 64) return 0;
    std::lock_guard<std::mutex> lk(mu);
    if (cached[device] == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
            sms <= 0)
            return 0;
        cached[device] = sms * 4;
    }
    return cached[device];
}

cudaError_t launch_action(const ReduceArgs &a, cudaStream_t st)
{
    if (a.precision == LQCD_F64)
        action_partials<double><<<a.blocks, kBlock, 0, st>>>(a, loop_table());
    else
        action_partials<float><<<a.blocks, kBlock, 0, st>>>(a, loop_table());
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finish_sum<<<1, kFinish, 0, st>>>(a.partials, a.blocks, a.scale, a.out);
    return cudaGetLastError();
}

cudaError_t launch_finish_sum(const double *partials, int count, double scale, double *out,
                              cudaStream_t st)
{
    finish_sum<<<1, kFinish, 0, st>>>(partials, count, scale, out);
    return cudaGetLastError();
}

cudaError_t launch_kinetic(const ReduceArgs &a, cudaStream_t st)
{
    if (a.precision == LQCD_F64)
        kinetic_partials<double><<<a.blocks, kBlock, 0, st>>>(a);
    else
        kinetic_partials<float><<<a.blocks, kBlock, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finish_sum<<<1, kFinish, 0, st>>>(a.partials, a.blocks, 1.0, a.out);
    return cudaGetLastError();
}

cudaError_t launch_unitarity(const ReduceArgs &a, cudaStream_t st)
{
    if (a.precision == LQCD_F64)
        unitarity_partials<double><<<a.blocks, kBlock, 0, st>>>(a);
    else
        unitarity_partials<float><<<a.blocks, kBlock, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finish_max<<<1, kFinish, 0, st>>>(a.partials, a.blocks, a.out);
    return cudaGetLastError();
}

// The 34 loops of Eq. 18_3_27_30 as direction sequences from n:
// plaquettes (mu, nu, -mu, -nu) for mu < nu, rectangles (mu, mu, nu, -mu,
// -mu, -nu) for mu != nu, cubes (mu, s nu, t r, -mu, -s nu, -t r) for
// mu < nu < r and s, t = +-1.
const LoopTable &loop_table()
{
    static LoopTable tab = [] {
        LoopTable t{};
        int n = 0;
        auto put = [&](int cls, std::initializer_list<int> d) {
            Loop &l = t.l[n++];
            l.cls = (int8_t)cls;
            l.len = (int8_t)d.size();
            int j = 0;
            for (int v : d) l.d[j++] = (int8_t)v;
        };
        for (int mu = 1; mu <= 4; ++mu)
            for (int nu = mu + 1; nu <= 4; ++nu) put(0, {mu, nu, -mu, -nu});
        for (int mu = 1; mu <= 4; ++mu)
            for (int nu = 1; nu <= 4; ++nu)
                if (nu != mu) put(1, {mu, mu, nu, -mu, -mu, -nu});
        for (int mu = 1; mu <= 4; ++mu)
            for (int nu = mu + 1; nu <= 4; ++nu)
                for (int r = nu + 1; r <= 4; ++r)
                    for (int s = 1; s >= -1; s -= 2)
                        for (int q = 1; q >= -1; q -= 2)
                            put(2, {mu, s * nu, q * r, -mu, -s * nu, -q * r});
        t.count = n;
        return t;
    }();
    return tab;
}

namespace {

// Device address of g_fixed_partials on `device`, looked up once per device
// (the device must be current).  Host code cannot use the symbol itself: on
// the host it names a host-side stand-in, not device memory.
cudaError_t fixed_partials_address(int device, double **out)
{
    static std::mutex mu;
    static double *addr[64] = {nullptr};
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (addr[device] == nullptr) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_fixed_partials);
        if (e != cudaSuccess) return e;
        if (p == nullptr) return cudaErrorInvalidSymbol;
        addr[device] = static_cast<double *>(p);
    }
    *out = addr[device];
    return cudaSuccess;
}

} // namespace

} // namespace lqcd

// Allocation-free variant of lqcd_gauge_action (declared in include/lqcd.h):
// the same argument checks and kernels, with the per-block partial sums kept
// in the fixed library-held array above instead of a caller workspace.
extern "C" int lqcd_gauge_action_noalloc(const lqcd_desc *desc, const void *links, double *action,
                                         void *stream)
{
    // NVTX range named after the entry point (no-op without a profiler)
    struct Range {
        Range() { nvtxRangePushA("lqcd_gauge_action_noalloc"); }
        ~Range() { nvtxRangePop(); }
    } const trace_range;
    int s = lqcd::check_desc(desc);
    if (s) return s;
    if ((s = lqcd::check_ptrs({links}))) return s;
    if (action == nullptr) return LQCD_ERR_ARG;
    if (((uintptr_t)action & 7u) != 0) return LQCD_ERR_ALIGN;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lqcd::cuda_status(e);
    const int blocks = lqcd::reduction_blocks(dev);
    if (blocks <= 0) return lqcd::cuda_status(cudaErrorInvalidDevice);
    if (blocks > lqcd::kFixedPartials) return LQCD_ERR_CAPACITY;
    double *partials = nullptr;
    e = lqcd::fixed_partials_address(dev, &partials);
    if (e != cudaSuccess) return lqcd::cuda_status(e);
    lqcd::ReduceArgs a{};
    for (int i = 0; i < 4; ++i) a.dims[i] = desc->dims[i];
    a.precision = desc->precision;
    a.links = links;
    a.c[0] = desc->c_plaq;
    a.c[1] = desc->c_rect;
    a.c[2] = desc->c_cube;
    a.scale = desc->beta / 3.0;
    a.partials = partials;
    a.blocks = blocks;
    a.out = action;
    return lqcd::cuda_status(lqcd::launch_action(a, static_cast<cudaStream_t>(stream)));
}
