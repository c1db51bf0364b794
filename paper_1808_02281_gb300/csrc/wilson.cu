// Wilson fermion hopping term (Sec. III of the paper): the hopping operator
// calD of Eq. 18_7_17_4 applied to a spinor field, and the hopping-term force
// on every link, -i(B - C)_TA of Eqs. 18_1_29_19 to 18_7_17_30.
//
// Both are HBM-streaming kernels (a few hundred flops per 100-400 bytes), so
// the design is about bytes: spinors and links are read in 16-byte lanes,
// neighbours come from L1/L2 (a time slice of a 32^3 spinor field is 3 MB),
// and every (1 -+ gamma_mu) is applied as a spin projection to two colour
// vectors, so that each link multiplies two colour vectors instead of four.
#include "kernels.h"
#include "su3.cuh"

namespace lqcd {
namespace {

// ------------------------------------------------------------ gamma basis

// Euclidean gamma matrices of the chiral basis, gamma_mu acting along
// direction mu = x, y, z, t.  Each has one non-zero entry per row:
// gamma_mu[alpha][gperm(mu, alpha)] = i^gcode(mu, alpha):
//   gamma_x: columns 3 2 1 0, entries  i  i -i -i
//   gamma_y: columns 3 2 1 0, entries -1  1  1 -1
//   gamma_z: columns 2 3 0 1, entries  i -i -i  i
//   gamma_t: columns 2 3 0 1, entries  1  1  1  1
__host__ __device__ constexpr int gperm(int mu, int alpha) { return mu < 2 ? 3 - alpha : alpha ^ 2; }

__host__ __device__ constexpr int gcode(int mu, int alpha)
{
    return mu == 0   ? (alpha < 2 ? 1 : 3)
           : mu == 1 ? ((alpha == 0 || alpha == 3) ? 2 : 0)
           : mu == 2 ? ((alpha == 0 || alpha == 3) ? 1 : 3)
                     : 0;
}

// (re, im) = i^K (xr + i xi)
template <int K, typename R> __device__ __forceinline__ void times_ipow(R &re, R &im, R xr, R xi)
{
    constexpr int k = K & 3;
    if constexpr (k == 0) {
        re = xr;
        im = xi;
    } else if constexpr (k == 1) {
        re = -xi;
        im = xr;
    } else if constexpr (k == 2) {
        re = -xr;
        im = -xi;
    } else {
        re = xi;
        im = -xr;
    }
}

// A launch scalar in the kernel's precision (FP32 copies made on the host).
template <typename R> __device__ __forceinline__ R scalar_of(double d, float f)
{
    if constexpr (sizeof(R) == 8) return d;
    else return f;
}

template <typename R> struct Spinor {
    R re[4][3], im[4][3];
};
// Two colour vectors: the independent rows 0 and 1 of (1 + s gamma_mu) psi.
template <typename R> struct Half {
    R re[2][3], im[2][3];
};

// ------------------------------------------------------- site geometry

// Site coordinates and neighbour indices in type I: int whenever the site
// loops fit (2 V + a block below 2^31), so that the divisions of the site
// index and the neighbour offsets take 32-bit arithmetic (a 64-bit division
// is a long software sequence); the 16-byte lane addresses stay 64-bit.
// Measured at 32^3x64 FP32: hopping operator 0.176 -> 0.168 ms, force 0.281
// -> 0.246 ms (32-bit lane addresses as well were slower: 0.171, 0.289).
template <typename I> struct Sites {
    int L0, L1, L2, L3;
    I s1, s2, s3, V;
};

template <typename I> __device__ __forceinline__ Sites<I> make_sites(const int dims[4])
{
    Sites<I> g;
    g.L0 = dims[0];
    g.L1 = dims[1];
    g.L2 = dims[2];
    g.L3 = dims[3];
    g.s1 = dims[0];
    g.s2 = g.s1 * dims[1];
    g.s3 = g.s2 * dims[2];
    g.V = g.s3 * dims[3];
    return g;
}

// Coordinates of site n < 2^31 with the strides' division magic (three
// multiply-highs instead of three divisions by run-time values: hopping
// force 0.242 -> 0.234 ms at 32^3x64 FP32).
__device__ __forceinline__ Coord coord_fast(const Sites<int> &g, const DivMagic div[3], int n)
{
    Coord x;
    x.c3 = (int)div_by((unsigned)n, div[2]);
    int r = n - x.c3 * g.s3;
    x.c2 = (int)div_by((unsigned)r, div[1]);
    r -= x.c2 * g.s2;
    x.c1 = (int)div_by((unsigned)r, div[0]);
    x.c0 = r - x.c1 * g.s1;
    return x;
}

template <typename I> __device__ __forceinline__ Coord coord_in(const Sites<I> &g, I n)
{
    Coord x;
    x.c3 = (int)(n / g.s3);
    I r = n - x.c3 * g.s3;
    x.c2 = (int)(r / g.s2);
    r -= x.c2 * g.s2;
    x.c1 = (int)(r / g.s1);
    x.c0 = (int)(r - x.c1 * g.s1);
    return x;
}

// Index offset of the step s * hat(mu) (s = +-1), periodic.
template <typename I>
__device__ __forceinline__ I hop_offset(const Sites<I> &g, const Coord &x, int mu, int s)
{
    const int L = pick(mu, g.L0, g.L1, g.L2, g.L3);
    const int c = pick(mu, x.c0, x.c1, x.c2, x.c3);
    const I st = mu == 0 ? I(1) : (mu == 1 ? g.s1 : (mu == 2 ? g.s2 : g.s3));
    if (s > 0) return c + 1 == L ? (I)(1 - L) * st : st;
    return c == 0 ? (I)(L - 1) * st : -st;
}

// ------------------------------------------------------------ spinor I/O

template <typename R>
__device__ __forceinline__ Spinor<R> load_spinor(const R *__restrict__ x, int64_t V, int64_t n)
{
    using V4 = typename Vec<R>::type;
    constexpr int W = Vec<R>::W;
    const V4 *p = reinterpret_cast<const V4 *>(x) + n;
    R r[24];
#pragma unroll
    for (int q = 0; q < 24 / W; ++q) {
        const V4 v = __ldg(p + q * V);
        if constexpr (W == 4) {
            r[4 * q + 0] = v.x;
            r[4 * q + 1] = v.y;
            r[4 * q + 2] = v.z;
            r[4 * q + 3] = v.w;
        } else {
            r[2 * q + 0] = v.x;
            r[2 * q + 1] = v.y;
        }
    }
    Spinor<R> s;
#pragma unroll
    for (int al = 0; al < 4; ++al)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s.re[al][a] = r[2 * (3 * al + a)];
            s.im[al][a] = r[2 * (3 * al + a) + 1];
        }
    return s;
}

template <typename R>
__device__ __forceinline__ void store_spinor(R *__restrict__ x, int64_t V, int64_t n, const Spinor<R> &s)
{
    using V4 = typename Vec<R>::type;
    constexpr int W = Vec<R>::W;
    V4 *p = reinterpret_cast<V4 *>(x) + n;
    R r[24];
#pragma unroll
    for (int al = 0; al < 4; ++al)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            r[2 * (3 * al + a)] = s.re[al][a];
            r[2 * (3 * al + a) + 1] = s.im[al][a];
        }
#pragma unroll
    for (int q = 0; q < 24 / W; ++q) {
        V4 v;
        if constexpr (W == 4) v = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
        else v = make_double2(r[2 * q], r[2 * q + 1]);
        p[q * V] = v;
    }
}

// ------------------------------------------------ spin projection algebra

// Rows 0 and 1 of (1 + S gamma_MU) x.  Rows gperm(MU, 0) and gperm(MU, 1) of
// the same spinor are S i^gcode(MU, gperm) times them (gamma_MU^2 = 1), so
// these two colour vectors carry all of it.
template <int MU, int S, int AL, typename R>
__device__ __forceinline__ void project_row(Half<R> &h, const Spinor<R> &x)
{
    constexpr int p = gperm(MU, AL);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R tr, ti;
        times_ipow<gcode(MU, AL) + (S < 0 ? 2 : 0)>(tr, ti, x.re[p][a], x.im[p][a]);
        h.re[AL][a] = x.re[AL][a] + tr;
        h.im[AL][a] = x.im[AL][a] + ti;
    }
}

template <int MU, int S, typename R> __device__ __forceinline__ Half<R> project(const Spinor<R> &x)
{
    Half<R> h;
    project_row<MU, S, 0>(h, x);
    project_row<MU, S, 1>(h, x);
    return h;
}

// acc += (1 + S gamma_MU) applied form of the half spinor g: rows 0, 1 are g,
// row gperm(MU, alpha) is S i^gcode(MU, gperm(MU, alpha)) g_alpha.
template <int MU, int S, typename R>
__device__ __forceinline__ void accumulate(Spinor<R> &acc, const Half<R> &g)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R tr, ti;
        acc.re[0][a] += g.re[0][a];
        acc.im[0][a] += g.im[0][a];
        acc.re[1][a] += g.re[1][a];
        acc.im[1][a] += g.im[1][a];
        constexpr int p0 = gperm(MU, 0), p1 = gperm(MU, 1);
        times_ipow<gcode(MU, p0) + (S < 0 ? 2 : 0)>(tr, ti, g.re[0][a], g.im[0][a]);
        acc.re[p0][a] += tr;
        acc.im[p0][a] += ti;
        times_ipow<gcode(MU, p1) + (S < 0 ? 2 : 0)>(tr, ti, g.re[1][a], g.im[1][a]);
        acc.re[p1][a] += tr;
        acc.im[p1][a] += ti;
    }
}

// op(u) applied to both colour vectors of h (F = N: u, F = D: u^dagger).
template <int F, typename R> __device__ __forceinline__ Half<R> colour_mul(const Mat<R> &u, const Half<R> &h)
{
    Half<R> r;
#pragma unroll
    for (int al = 0; al < 2; ++al)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R re = R(0), im = R(0);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                re = fma(el_re<F>(u, a, b), h.re[al][b], re);
                re = fma(-el_im<F>(u, a, b), h.im[al][b], re);
                im = fma(el_re<F>(u, a, b), h.im[al][b], im);
                im = fma(el_im<F>(u, a, b), h.re[al][b], im);
            }
            r.re[al][a] = re;
            r.im[al][a] = im;
        }
    return r;
}

// m[b][a] += SIGN * sum_alpha p_alpha[b] conj(q_alpha[a]) over the two rows.
template <int SIGN, typename R>
__device__ __forceinline__ void outer_acc(Mat<R> &m, const Half<R> &p, const Half<R> &q)
{
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R re = m.re[b][a], im = m.im[b][a];
#pragma unroll
            for (int al = 0; al < 2; ++al) {
                // p * conj(q) = (pr qr + pi qi) + i (pi qr - pr qi)
                re = fma(R(SIGN) * p.re[al][b], q.re[al][a], re);
                re = fma(R(SIGN) * p.im[al][b], q.im[al][a], re);
                im = fma(R(SIGN) * p.im[al][b], q.re[al][a], im);
                im = fma(-R(SIGN) * p.re[al][b], q.im[al][a], im);
            }
            m.re[b][a] = re;
            m.im[b][a] = im;
        }
}

// ------------------------------------------------------- hopping operator

// acc += (1 - gamma_MU) U_{n,MU} x_{n+MU} + (1 + gamma_MU) U_{n-MU,MU}^dag x_{n-MU}
template <int MU, typename R, typename I>
__device__ __forceinline__ void hop(Spinor<R> &acc, const R *__restrict__ links,
                                    const R *__restrict__ x, const Sites<I> &g, const Coord &c, I n)
{
    const int64_t V = g.V;
    const int64_t nf = n + hop_offset(g, c, MU, 1);
    accumulate<MU, -1>(acc, colour_mul<N>(load_link(links, V, MU, n), project<MU, -1>(load_spinor(x, V, nf))));
    const int64_t nb = n + hop_offset(g, c, MU, -1);
    accumulate<MU, +1>(acc, colour_mul<D>(load_link(links, V, MU, nb), project<MU, +1>(load_spinor(x, V, nb))));
}

// The x hops from the lanes of the same warp, when a warp holds whole x
// rows (the x extent divides 32; lanes n and n +- x are then lanes of one
// row of L0 lanes, with periodic wrap inside the row).  Each lane projects
// its own spinor both ways, keeps (1 - gamma_x) x_n for lane n-1's forward
// hop and applies its own link's dagger to (1 + gamma_x) x_n for lane n+1's
// backward hop (U_{n,x} is the backward link of site n+x), so that lane n
// receives 2 x 12 reals by shuffles instead of loading two neighbour
// spinors and the backward link (15 of the 78 16-byte loads of a site).
template <typename R> __device__ __forceinline__ R shfl_row(R v, int src)
{
    return __shfl_sync(0xffffffffu, v, src);
}

template <typename R> __device__ __forceinline__ Half<R> shfl_half(const Half<R> &h, int src)
{
    Half<R> r;
#pragma unroll
    for (int al = 0; al < 2; ++al)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            r.re[al][a] = shfl_row(h.re[al][a], src);
            r.im[al][a] = shfl_row(h.im[al][a], src);
        }
    return r;
}

template <typename R>
__device__ __forceinline__ void hop_x_shuffled(Spinor<R> &acc, const R *__restrict__ links,
                                               const Spinor<R> &xn, int64_t V, int64_t n, int L0)
{
    const int lane = (int)(threadIdx.x & 31), m = L0 - 1;
    const int up = (lane & ~m) | ((lane + 1) & m), dn = (lane & ~m) | ((lane - 1) & m);
    const Mat<R> u = load_link(links, V, 0, n);
    const Half<R> fw = shfl_half(project<0, -1>(xn), up);                  // (1 - g_x) x_{n+x}
    const Half<R> bw = shfl_half(colour_mul<D>(u, project<0, +1>(xn)), dn); // U_{n-x}^dag (1 + g_x) x_{n-x}
    accumulate<0, -1>(acc, colour_mul<N>(u, fw));
    accumulate<0, +1>(acc, bw);
}

constexpr int kDslashBlock = 128;

// Register cap: 5 blocks (20 warps, 96 registers, a 64-byte spill) per SM in
// FP32: at 32^3x64 0.161 against 0.167 ms with 4 blocks (128 registers) and
// 0.245 ms with the uncapped 138 (12 warps) -- the kernel waits on loads, so
// warps in flight count more than the spill; FP64 is bound by the FP64 pipe
// and keeps its registers.
template <typename R> constexpr int dslash_min_blocks() { return sizeof(R) == 8 ? 1 : 5; }

// out_n = ca x_n + cb (calD x)_n, one thread per site.
// XSHFL: x hops by shuffles.
template <typename R, bool XSHFL, typename I>
__global__ void __launch_bounds__(kDslashBlock, dslash_min_blocks<R>())
    wilson_dslash(const __grid_constant__ WilsonArgs a)
{
    const Sites<I> g = make_sites<I>(a.dims);
    const int64_t V = g.V;
    const R *__restrict__ links = static_cast<const R *>(a.links);
    const R *__restrict__ x = static_cast<const R *>(a.x);
    R *__restrict__ out = static_cast<R *>(a.out);
    const R ca = scalar_of<R>(a.ca, a.fca), cb = scalar_of<R>(a.cb, a.fcb);
    const bool with_x = a.ca != 0.0;
    for (I n = (I)blockIdx.x * blockDim.x + threadIdx.x; n < g.V; n += (I)gridDim.x * blockDim.x) {
        Coord c;
        if constexpr (sizeof(I) == 4) c = coord_fast(g, a.div, n);
        else c = coord_in(g, n);
        Spinor<R> acc;
#pragma unroll
        for (int al = 0; al < 4; ++al)
#pragma unroll
            for (int b = 0; b < 3; ++b) acc.re[al][b] = acc.im[al][b] = R(0);
        if constexpr (XSHFL) {
            const Spinor<R> xn = load_spinor(x, V, (int64_t)n);
            hop_x_shuffled(acc, links, xn, V, (int64_t)n, g.L0);
        } else {
            hop<0>(acc, links, x, g, c, n);
        }
        hop<1>(acc, links, x, g, c, n);
        hop<2>(acc, links, x, g, c, n);
        hop<3>(acc, links, x, g, c, n);
        if (with_x) {
            const Spinor<R> xn = load_spinor(x, V, (int64_t)n);
#pragma unroll
            for (int al = 0; al < 4; ++al)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    acc.re[al][b] = fma(ca, xn.re[al][b], cb * acc.re[al][b]);
                    acc.im[al][b] = fma(ca, xn.im[al][b], cb * acc.im[al][b]);
                }
        } else {
#pragma unroll
            for (int al = 0; al < 4; ++al)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    acc.re[al][b] *= cb;
                    acc.im[al][b] *= cb;
                }
        }
        store_spinor(out, V, (int64_t)n, acc);
    }
}

// --------------------------------------------------- hopping-term force

// B - C on link (k, RHO), both as sums over the two independent spin rows:
//   B = sum_alpha (U chi_alpha) (x) psi_alpha^dag,  chi = (1 - g) X_{k+rho}, psi = (1 - g) Y_k
//   C = sum_alpha xi_alpha (x) (U eta_alpha)^dag,   xi = (1 + g) X_k,      eta = (1 + g) Y_{k+rho}
// (Eqs. 18_1_29_20_2 and 18_1_29_20_3 with (1 -+ g) Hermitian and
// (1 -+ g)^2 = 2 (1 -+ g), so the projector moves onto the other factor and
// the four spin rows fold into two.)
template <int RHO, typename R>
__device__ __forceinline__ Mat<R> b_minus_c(const R *__restrict__ links, const R *__restrict__ X,
                                            const R *__restrict__ Y, int64_t V, int64_t k, int64_t kp)
{
    const Mat<R> u = load_link(links, V, RHO, k);
    Mat<R> m;
    set_zero(m);
    outer_acc<1>(m, colour_mul<N>(u, project<RHO, -1>(load_spinor(X, V, kp))),
                 project<RHO, -1>(load_spinor(Y, V, k)));
    outer_acc<-1>(m, project<RHO, +1>(load_spinor(X, V, k)),
                  colour_mul<N>(u, project<RHO, +1>(load_spinor(Y, V, kp))));
    return m;
}

constexpr int kForceBlock = 128; // 32 sites x 4 directions, one direction per warp

template <typename R, typename I>
__global__ void __launch_bounds__(kForceBlock) wilson_hopping_force(const __grid_constant__ WilsonArgs a)
{
    const Sites<I> g = make_sites<I>(a.dims);
    const R *__restrict__ links = static_cast<const R *>(a.links);
    const R *__restrict__ X = static_cast<const R *>(a.x);
    const R *__restrict__ Y = static_cast<const R *>(a.y);
    const int rho = (int)(threadIdx.x >> 5);
    const I ks = (I)blockIdx.x * 32 + (I)(threadIdx.x & 31);
    if (ks >= g.V) return;
    Coord c;
    if constexpr (sizeof(I) == 4) c = coord_fast(g, a.div, ks);
    else c = coord_in(g, ks);
    const int64_t V = g.V, k = ks, kp = (int64_t)(ks + hop_offset(g, c, rho, 1));
    Mat<R> m;
    switch (rho) {
    case 0: m = b_minus_c<0>(links, X, Y, V, k, kp); break;
    case 1: m = b_minus_c<1>(links, X, Y, V, k, kp); break;
    case 2: m = b_minus_c<2>(links, X, Y, V, k, kp); break;
    default: m = b_minus_c<3>(links, X, Y, V, k, kp); break;
    }
    // f^i = coef * h^i,  h^i = -(tr(i T_i M) + c.c.) = Im tr(lambda_i M)
    R f[8];
    ta_components(m, -scalar_of<R>(a.coef, a.fcoef), f);
    if (a.force != nullptr) store_algebra(static_cast<R *>(a.force), V, rho, k, f);
    if (a.mom != nullptr) {
        R *mom = static_cast<R *>(a.mom);
        R p[8];
        load_algebra(mom, V, rho, k, p);
        const R dt = scalar_of<R>(a.dt, a.fdt);
#pragma unroll
        for (int q = 0; q < 8; ++q) p[q] = fma(dt, f[q], p[q]);
        store_algebra(mom, V, rho, k, p);
    }
}

unsigned blocks_for(int64_t items, int per_block)
{
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > ((int64_t)1 << 30)) b = (int64_t)1 << 30;
    return (unsigned)b;
}

// Site loops in int: n + grid stride stays below 2 V + a block.
bool sites_fit_int(int64_t V) { return 2 * V + 1024 < ((int64_t)1 << 31); }

// The launch copy of the arguments: FP32 scalars and the strides' division
// magic filled in.
WilsonArgs launch_args(WilsonArgs a)
{
    const int64_t s[3] = {a.dims[0], (int64_t)a.dims[0] * a.dims[1],
                          (int64_t)a.dims[0] * a.dims[1] * a.dims[2]};
    for (int i = 0; i < 3; ++i)
        a.div[i] = div_magic(s[i] < ((int64_t)1 << 31) ? (unsigned)s[i] : 1u);
    a.fca = (float)a.ca;
    a.fcb = (float)a.cb;
    a.fcoef = (float)a.coef;
    a.fdt = (float)a.dt;
    return a;
}

} // namespace

cudaError_t launch_wilson_dslash(const WilsonArgs &args, cudaStream_t st)
{
    const WilsonArgs a = launch_args(args);
    const int64_t V = (int64_t)a.dims[0] * a.dims[1] * a.dims[2] * a.dims[3];
    const unsigned grid = blocks_for(V, kDslashBlock);
    // shuffled x hops need whole x rows in every warp: L0 divides 32 (then
    // V is a multiple of L0 and every warp's first site starts a row), and a
    // grid-stride loop that never runs a warp past V with only part of it
    const int L0 = a.dims[0];
    const bool xshfl = L0 <= 32 && (32 % L0) == 0 && V % 32 == 0 &&
                       (int64_t)grid * kDslashBlock >= V;
    const bool i32 = sites_fit_int(V);
    if (a.precision == LQCD_F64) { // FP64-pipe bound; the shuffled form spills there
        if (i32) wilson_dslash<double, false, int><<<grid, kDslashBlock, 0, st>>>(a);
        else wilson_dslash<double, false, int64_t><<<grid, kDslashBlock, 0, st>>>(a);
    } else if (i32) {
        if (xshfl) wilson_dslash<float, true, int><<<grid, kDslashBlock, 0, st>>>(a);
        else wilson_dslash<float, false, int><<<grid, kDslashBlock, 0, st>>>(a);
    } else {
        if (xshfl) wilson_dslash<float, true, int64_t><<<grid, kDslashBlock, 0, st>>>(a);
        else wilson_dslash<float, false, int64_t><<<grid, kDslashBlock, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_wilson_hopping_force(const WilsonArgs &args, cudaStream_t st)
{
    const WilsonArgs a = launch_args(args);
    const int64_t V = (int64_t)a.dims[0] * a.dims[1] * a.dims[2] * a.dims[3];
    const unsigned grid = blocks_for(V, 32);
    const bool i32 = sites_fit_int(V);
    if (a.precision == LQCD_F64) {
        if (i32) wilson_hopping_force<double, int><<<grid, kForceBlock, 0, st>>>(a);
        else wilson_hopping_force<double, int64_t><<<grid, kForceBlock, 0, st>>>(a);
    } else {
        if (i32) wilson_hopping_force<float, int><<<grid, kForceBlock, 0, st>>>(a);
        else wilson_hopping_force<float, int64_t><<<grid, kForceBlock, 0, st>>>(a);
    }
    return cudaGetLastError();
}

} // namespace lqcd
