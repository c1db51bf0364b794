// Molecular-dynamics steps and layout conversions, all streaming kernels
// (one thread per link or per 16-byte lane, grid-stride, coalesced 16-byte
// loads and stores of the structure-of-arrays planes).
//   momentum step  p^a += dt f^a                      (f = -dS/domega, Eq. 18_7_25_1)
//   link step      U <- exp(i dt sum_a p^a T_a) U     (left flow of Eq. 18_1_29_3)
//   links from omega  U = exp(i sum_a omega^a T_a)    (Eq. 18_1_29_3)
//   pack / unpack  full 3x3 complex <-> first two rows
#include "kernels.h"
#include "su3.cuh"

namespace lqcd {

namespace {

constexpr int kBlock = 256;

int64_t volume(const int dims[4])
{
    return (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
}

unsigned grid_for(int64_t items)
{
    int64_t g = (items + kBlock - 1) / kBlock;
    if (g < 1) g = 1;
    if (g > ((int64_t)1 << 30)) g = (int64_t)1 << 30;
    return (unsigned)g;
}

// Direction of link i of the link-major order (i = mu V + n, i < 4 V): three
// comparisons instead of a 64-bit division.
__device__ __forceinline__ int direction_of(int64_t i, int64_t V)
{
    return (int)(i >= V) + (int)(i >= 2 * V) + (int)(i >= 3 * V);
}

// p += dt f over 16-byte lanes of the algebra planes.
template <typename R>
__global__ void __launch_bounds__(kBlock) update_momenta(typename Vec<R>::type *__restrict__ p,
                                                         const typename Vec<R>::type *__restrict__ f,
                                                         int64_t lanes, R dt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < lanes;
         i += (int64_t)gridDim.x * blockDim.x) {
        auto a = p[i];
        const auto b = __ldg(f + i);
        if constexpr (Vec<R>::W == 4) {
            a.x = fma(dt, b.x, a.x);
            a.y = fma(dt, b.y, a.y);
            a.z = fma(dt, b.z, a.z);
            a.w = fma(dt, b.w, a.w);
        } else {
            a.x = fma(dt, b.x, a.x);
            a.y = fma(dt, b.y, a.y);
        }
        p[i] = a;
    }
}

// U <- exp(i dt P) U (FROM_UNIT: U = exp(i dt P)), rows 0 and 1 only, then
// Gram-Schmidt.  The link and algebra planes share the site index.
template <typename R, bool FROM_UNIT>
__global__ void __launch_bounds__(kBlock) update_links(R *__restrict__ links,
                                                       const R *__restrict__ mom, int64_t V, R dt)
{
    const int64_t nlinks = 4 * V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlinks;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int mu = direction_of(i, V);
        const int64_t n = i - mu * V;
        R p[8];
        load_algebra(mom, V, mu, n, p);
#pragma unroll
        for (int c = 0; c < 8; ++c) p[c] *= dt;
        const Mat<R> e = exp_i_hermitian(algebra_matrix(p));
        Mat<R> u;
        if constexpr (FROM_UNIT) {
            u = e;
        } else {
            const Mat<R> v = load_link(links, V, mu, n);
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    R re = R(0), im = R(0);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        re = fma(e.re[r][k], v.re[k][j], re);
                        re = fma(-e.im[r][k], v.im[k][j], re);
                        im = fma(e.re[r][k], v.im[k][j], im);
                        im = fma(e.im[r][k], v.re[k][j], im);
                    }
                    u.re[r][j] = re;
                    u.im[r][j] = im;
                }
        }
        reunitarise(u);
        store_link(links, V, mu, n, u);
    }
}

// The link step of update_links for one link of a batch of lattices: the
// persistent CTAs walk the concatenated link ranges.
struct LinkBatch {
    int n;
    int64_t total;
    int64_t begin[kMaxBatch + 1]; // first link of each lattice in the concatenation
    int64_t V[kMaxBatch];
    void *links[kMaxBatch];
    const void *mom[kMaxBatch];
};

template <typename R>
__global__ void __launch_bounds__(kBlock) update_links_batched(const __grid_constant__ LinkBatch B, R dt)
{
    int c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B.total;
         i += (int64_t)gridDim.x * blockDim.x) {
        while (c > 0 && i < B.begin[c]) --c;
        while (c + 1 < B.n && i >= B.begin[c + 1]) ++c;
        const int64_t V = B.V[c];
        const int64_t l = i - B.begin[c];
        const int mu = direction_of(l, V);
        const int64_t n = l - mu * V;
        R *links = static_cast<R *>(B.links[c]);
        R p[8];
        load_algebra(static_cast<const R *>(B.mom[c]), V, mu, n, p);
#pragma unroll
        for (int q = 0; q < 8; ++q) p[q] *= dt;
        const Mat<R> e = exp_i_hermitian(algebra_matrix(p));
        const Mat<R> v = load_link(links, V, mu, n);
        Mat<R> u;
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                R re = R(0), im = R(0);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    re = fma(e.re[r][k], v.re[k][j], re);
                    re = fma(-e.im[r][k], v.im[k][j], re);
                    im = fma(e.re[r][k], v.im[k][j], im);
                    im = fma(e.im[r][k], v.re[k][j], im);
                }
                u.re[r][j] = re;
                u.im[r][j] = im;
            }
        reunitarise(u);
        store_link(links, V, mu, n, u);
    }
}

// Chain rule through U = exp(X) U0, X = i W, W = omega.T (Eq. 18_1_29_3).
// A change d omega moves U by the left perturbation exp(i delta.T) with
// i delta.T = phi(ad_X)(i d omega.T), phi(z) = (e^z - 1)/z.  The force gives
// the left derivative dS/d delta^b = -f^b, so
//     dS/d omega^a = components of phi(-ad_X)(-i F),   F = f.T,
// since phi(ad_X) is orthogonal-adjoint to phi(-ad_X) on su(3).  Writing the
// series terms as -i H_n with Hermitian H_n:
//     H_0 = F,   H_n = -i [W, H_{n-1}] / (n+1),   A = sum_n H_n,
//     dS/d omega^a = -tr(lambda_a A)  (= -f^a at omega = 0).
// The series stops once (2 |W|_F)^n / (n+1)!, a bound on |H_n|/|F|, is below
// the working precision.
template <typename R>
__global__ void __launch_bounds__(kBlock) omega_gradient(const R *__restrict__ omega,
                                                         const R *__restrict__ force,
                                                         R *__restrict__ grad, int64_t V)
{
    constexpr int NMAX = sizeof(R) == 8 ? 40 : 24;
    const R eps = sizeof(R) == 8 ? R(1e-17) : R(1e-9);
    const int64_t nlinks = 4 * V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlinks;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int mu = direction_of(i, V);
        const int64_t n = i - mu * V;
        R w[8], f[8];
        load_algebra(omega, V, mu, n, w);
        load_algebra(force, V, mu, n, f);
        const Mat<R> W = algebra_matrix(w);
        Mat<R> h = algebra_matrix(f); // H_0 = F
        Mat<R> acc = h;
        R wn = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) wn += W.re[a][b] * W.re[a][b] + W.im[a][b] * W.im[a][b];
        const R bound = R(2) * sqrt(wn);
        R est = R(1);
        for (int k = 1; k <= NMAX; ++k) {
            const Mat<R> wh = mul<N, N>(W, h);
            const Mat<R> hw = mul<N, N>(h, W);
            const R inv = R(1) / R(k + 1);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    // H_k = -i (cr + i ci) / (k+1) with [W, H_{k-1}] = cr + i ci
                    const R cr = wh.re[a][b] - hw.re[a][b], ci = wh.im[a][b] - hw.im[a][b];
                    h.re[a][b] = ci * inv;
                    h.im[a][b] = -cr * inv;
                    acc.re[a][b] += h.re[a][b];
                    acc.im[a][b] += h.im[a][b];
                }
            est *= bound * inv;
            if (est < eps) break;
        }
        // dS/d omega^a = -tr(lambda_a A) (A Hermitian: real traces)
        R g[8];
        g[0] = -(acc.re[0][1] + acc.re[1][0]);
        g[1] = -(acc.im[1][0] - acc.im[0][1]);
        g[2] = -(acc.re[0][0] - acc.re[1][1]);
        g[3] = -(acc.re[0][2] + acc.re[2][0]);
        g[4] = -(acc.im[2][0] - acc.im[0][2]);
        g[5] = -(acc.re[1][2] + acc.re[2][1]);
        g[6] = -(acc.im[2][1] - acc.im[1][2]);
        g[7] = -R(0.57735026918962576451) * (acc.re[0][0] + acc.re[1][1] - R(2) * acc.re[2][2]);
        store_algebra(grad, V, mu, n, g);
    }
}

// Real r (0..NR-1) of item (n, mu) of a structure-of-arrays field with NR
// reals per item and W-wide lanes.
template <typename R, int NR>
__device__ __forceinline__ int64_t soa_index(int64_t V, int mu, int64_t n, int r)
{
    constexpr int W = Vec<R>::W;
    return (((int64_t)mu * (NR / W) + r / W) * V + n) * W + r % W;
}

// Precision conversion of a link (NR = 12) or algebra (NR = 8) field; the
// stored reals are converted one by one (FP32 -> FP64 exactly).
template <typename RS, typename RD, int NR>
__global__ void __launch_bounds__(kBlock) convert_field(const RS *__restrict__ src,
                                                        RD *__restrict__ dst, int64_t V)
{
    const int64_t nitems = 4 * V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nitems;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int mu = direction_of(i, V);
        const int64_t n = i - mu * V;
#pragma unroll
        for (int r = 0; r < NR; ++r)
            dst[soa_index<RD, NR>(V, mu, n, r)] = (RD)src[soa_index<RS, NR>(V, mu, n, r)];
    }
}

// full [V][4][3][3] (re, im) -> compact link layout (rows 0, 1)
template <typename R>
__global__ void __launch_bounds__(kBlock) pack(const R *__restrict__ full, R *__restrict__ links,
                                               int64_t V)
{
    const int64_t nlinks = 4 * V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlinks;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int mu = direction_of(i, V);
        const int64_t n = i - mu * V;
        const R *src = full + (n * 4 + mu) * 18;
        Mat<R> u;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                u.re[r][j] = src[(3 * r + j) * 2];
                u.im[r][j] = src[(3 * r + j) * 2 + 1];
            }
        store_link(links, V, mu, n, u);
    }
}

template <typename R>
__global__ void __launch_bounds__(kBlock) unpack(const R *__restrict__ links, R *__restrict__ full,
                                                 int64_t V)
{
    const int64_t nlinks = 4 * V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlinks;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int mu = direction_of(i, V);
        const int64_t n = i - mu * V;
        const Mat<R> u = load_link(links, V, mu, n);
        R *dst = full + (n * 4 + mu) * 18;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                dst[(3 * r + j) * 2] = u.re[r][j];
                dst[(3 * r + j) * 2 + 1] = u.im[r][j];
            }
    }
}

// Gram-Schmidt of rows 0 and 1 of every stored link in FP64 (row 2 is
// rebuilt on every load), rounded back to the storage precision.
template <typename R> __global__ void __launch_bounds__(kBlock) reunitarise_fp64(R *__restrict__ links, int64_t V)
{
    const int64_t nlinks = 4 * V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlinks;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int mu = direction_of(i, V);
        const int64_t n = i - mu * V;
        const Mat<R> u = load_link(links, V, mu, n);
        Mat<double> w;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                w.re[r][j] = (double)u.re[r][j];
                w.im[r][j] = (double)u.im[r][j];
            }
        reunitarise(w);
        Mat<R> v;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                v.re[r][j] = (R)w.re[r][j];
                v.im[r][j] = (R)w.im[r][j];
            }
        store_link(links, V, mu, n, v);
    }
}

// Word i of the counter-based SplitMix64 stream `seed` (Steele, Lea & Flood,
// "Fast splittable pseudorandom number generators", OOPSLA 2014):
// mix(seed + (i + 1) * golden gamma) with the published finaliser.
__device__ __forceinline__ uint64_t splitmix_word(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Standard normal j of stream `seed`: the Box-Muller transform (cosine
// branch) of words 2j and 2j+1 as 53-bit uniforms, u1 in (0, 1], u2 in [0, 1).
__device__ __forceinline__ double gaussian_of(uint64_t seed, uint64_t j)
{
    const uint64_t w1 = splitmix_word(seed, 2 * j), w2 = splitmix_word(seed, 2 * j + 1);
    const double u1 = ((double)(w1 >> 11) + 1.0) * 0x1p-53;
    const double u2 = (double)(w2 >> 11) * 0x1p-53;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
}

// p^a_{n,mu} = normal number (n*4 + mu)*8 + a of the stream, in FP64,
// rounded to the storage precision.
template <typename R>
__global__ void __launch_bounds__(kBlock) gaussian_momenta(R *__restrict__ mom, int64_t V, uint64_t seed)
{
    const int64_t nlinks = 4 * V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlinks;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int mu = direction_of(i, V);
        const int64_t n = i - mu * V;
        R p[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) p[a] = (R)gaussian_of(seed, (uint64_t)((n * 4 + mu) * 8 + a));
        store_algebra(mom, V, mu, n, p);
    }
}

} // namespace

cudaError_t launch_reunitarise(const MdArgs &a, cudaStream_t st)
{
    const int64_t V = volume(a.dims);
    if (a.precision == LQCD_F64)
        reunitarise_fp64<double><<<grid_for(4 * V), kBlock, 0, st>>>(static_cast<double *>(a.links), V);
    else
        reunitarise_fp64<float><<<grid_for(4 * V), kBlock, 0, st>>>(static_cast<float *>(a.links), V);
    return cudaGetLastError();
}

cudaError_t launch_gaussian_momenta(const MdArgs &a, cudaStream_t st)
{
    const int64_t V = volume(a.dims);
    if (a.precision == LQCD_F64)
        gaussian_momenta<double><<<grid_for(4 * V), kBlock, 0, st>>>(static_cast<double *>(a.mom_out), V, a.seed);
    else
        gaussian_momenta<float><<<grid_for(4 * V), kBlock, 0, st>>>(static_cast<float *>(a.mom_out), V, a.seed);
    return cudaGetLastError();
}

cudaError_t launch_update_momenta(const MdArgs &a, cudaStream_t st)
{
    const int64_t V = volume(a.dims);
    if (a.precision == LQCD_F64) {
        const int64_t lanes = 4 * 8 * V / 2;
        update_momenta<double><<<grid_for(lanes), kBlock, 0, st>>>(
            static_cast<double2 *>(a.mom_out), static_cast<const double2 *>(a.force), lanes, a.dt);
    } else {
        const int64_t lanes = 4 * 8 * V / 4;
        update_momenta<float><<<grid_for(lanes), kBlock, 0, st>>>(
            static_cast<float4 *>(a.mom_out), static_cast<const float4 *>(a.force), lanes,
            (float)a.dt);
    }
    return cudaGetLastError();
}

cudaError_t launch_update_links(const MdArgs &a, cudaStream_t st)
{
    const int64_t V = volume(a.dims);
    if (a.precision == LQCD_F64)
        update_links<double, false><<<grid_for(4 * V), kBlock, 0, st>>>(
            static_cast<double *>(a.links), static_cast<const double *>(a.mom), V, a.dt);
    else
        update_links<float, false><<<grid_for(4 * V), kBlock, 0, st>>>(
            static_cast<float *>(a.links), static_cast<const float *>(a.mom), V, (float)a.dt);
    return cudaGetLastError();
}

cudaError_t launch_update_links_batched(int precision, int n, const LinkStepItem *items, double dt,
                                        cudaStream_t st)
{
    if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
    LinkBatch B{};
    B.n = n;
    int64_t pos = 0;
    for (int c = 0; c < n; ++c) {
        B.begin[c] = pos;
        B.V[c] = items[c].V;
        B.links[c] = items[c].links;
        B.mom[c] = items[c].mom;
        pos += 4 * items[c].V;
    }
    B.begin[n] = pos;
    B.total = pos;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t grid = (pos + kBlock - 1) / kBlock;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    if (precision == LQCD_F64)
        update_links_batched<double><<<(unsigned)grid, kBlock, 0, st>>>(B, dt);
    else
        update_links_batched<float><<<(unsigned)grid, kBlock, 0, st>>>(B, (float)dt);
    return cudaGetLastError();
}

cudaError_t launch_links_from_omega(const MdArgs &a, cudaStream_t st)
{
    const int64_t V = volume(a.dims);
    if (a.precision == LQCD_F64)
        update_links<double, true><<<grid_for(4 * V), kBlock, 0, st>>>(
            static_cast<double *>(a.links), static_cast<const double *>(a.mom), V, 1.0);
    else
        update_links<float, true><<<grid_for(4 * V), kBlock, 0, st>>>(
            static_cast<float *>(a.links), static_cast<const float *>(a.mom), V, 1.0f);
    return cudaGetLastError();
}

cudaError_t launch_omega_gradient(const MdArgs &a, cudaStream_t st)
{
    const int64_t V = volume(a.dims);
    if (a.precision == LQCD_F64)
        omega_gradient<double><<<grid_for(4 * V), kBlock, 0, st>>>(
            static_cast<const double *>(a.mom), static_cast<const double *>(a.force),
            static_cast<double *>(a.mom_out), V);
    else
        omega_gradient<float><<<grid_for(4 * V), kBlock, 0, st>>>(
            static_cast<const float *>(a.mom), static_cast<const float *>(a.force),
            static_cast<float *>(a.mom_out), V);
    return cudaGetLastError();
}

template <int NR> static cudaError_t launch_convert_t(const MdArgs &a, int dst_precision,
                                                      cudaStream_t st)
{
    const int64_t V = volume(a.dims);
    const void *src = a.full_in;
    void *dst = a.full_out;
    const unsigned grid = grid_for(4 * V);
    if (a.precision == LQCD_F32 && dst_precision == LQCD_F64)
        convert_field<float, double, NR><<<grid, kBlock, 0, st>>>(static_cast<const float *>(src),
                                                                  static_cast<double *>(dst), V);
    else if (a.precision == LQCD_F64 && dst_precision == LQCD_F32)
        convert_field<double, float, NR><<<grid, kBlock, 0, st>>>(static_cast<const double *>(src),
                                                                  static_cast<float *>(dst), V);
    else if (a.precision == LQCD_F32)
        convert_field<float, float, NR><<<grid, kBlock, 0, st>>>(static_cast<const float *>(src),
                                                                 static_cast<float *>(dst), V);
    else
        convert_field<double, double, NR><<<grid, kBlock, 0, st>>>(
            static_cast<const double *>(src), static_cast<double *>(dst), V);
    return cudaGetLastError();
}

cudaError_t launch_convert(const MdArgs &a, int dst_precision, bool links, cudaStream_t st)
{
    return links ? launch_convert_t<12>(a, dst_precision, st) : launch_convert_t<8>(a, dst_precision, st);
}

cudaError_t launch_pack(const MdArgs &a, cudaStream_t st)
{
    const int64_t V = volume(a.dims);
    if (a.precision == LQCD_F64)
        pack<double><<<grid_for(4 * V), kBlock, 0, st>>>(static_cast<const double *>(a.full_in),
                                                          static_cast<double *>(a.links), V);
    else
        pack<float><<<grid_for(4 * V), kBlock, 0, st>>>(static_cast<const float *>(a.full_in),
                                                         static_cast<float *>(a.links), V);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const MdArgs &a, cudaStream_t st)
{
    const int64_t V = volume(a.dims);
    if (a.precision == LQCD_F64)
        unpack<double><<<grid_for(4 * V), kBlock, 0, st>>>(static_cast<const double *>(a.links),
                                                            static_cast<double *>(a.full_out), V);
    else
        unpack<float><<<grid_for(4 * V), kBlock, 0, st>>>(static_cast<const float *>(a.links),
                                                           static_cast<float *>(a.full_out), V);
    return cudaGetLastError();
}

} // namespace lqcd
