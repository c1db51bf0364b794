// Gauge force of the one-loop Symanzik action from plaquette-staple fields
// (paper Sec. II, Eq. 18_7_25_2; loops of Eq. 18_3_27_30), two kernels.
//
// Pass A (staple_fields) stores, for every link (x, mu) and every signed
// direction b perpendicular to mu, the plaquette staple
//     S^{(mu)}_b(x) = link(x+mu, b) U_mu(x+b)^dag link(x, b)^dag
// (the path x+mu -> x+mu+b -> x+b -> x): 24 "directions" per site instead
// of 4.  It is a product of three SU(3) matrices, so it is SU(3): its first
// two rows (which need only two rows of the first product) determine the
// third, conj(row0 x row1).  Planes are stored compact (two rows, the third
// rebuilt on load) or full (all 18 reals; the default schedule).
//
// Pass B (force_from_staples) builds every staple of the link (k, rho) from
// those fields.  With S = S^{(rho)} and A_b = link(k, b), B_b = link(k+rho, b),
// F = U_rho(k+rho), E = U_rho(k-rho), and the unitarity of the links:
//   plaquette            S_b(k)
//   rectangle, link first on the long side    F S_b(k+rho) S_b(k)
//   rectangle, link second on the long side   S_b(k) S_b(k-rho) E
//   rectangle along b    B_b S_b(k+b) A_b^dag
//   cube (a, b)          B_a S_b(k+a) S^{(a)}_b(k),  S^{(-c)}_b(k) = S^{(c)}_b(k-c)^dag
// (each equals the corresponding staple of the path form -- products of the
// same links -- once U U^dag = 1 is used for the link that the two staple
// factors share).  Summed with the loop coefficients and regrouped,
//   t = c_plaq sum_b S_b(k) + c_rect (F sum_b S_b(k+rho) S_b(k) + sum_b S_b(k) S_b(k-rho) E)
//     + sum_d B_d [ c_cube sum_{b perp d} S_b(k+d) S^{(d)}_b(k) + c_rect S_d(k+d) A_d^dag ],
// 51 SU(3) products per link in pass B and 12 (10 stored rows) per link in
// pass A, against 180 for the 48 staples walked one by one.  Every product
// of two SU(3) factors in pass B likewise forms two rows and takes its third
// from them, so the left factor's third row is never needed.
//
// The action comes out of pass B at no extra products: summing
// Re tr(U_{k,rho} t_{k,rho}) over links counts every loop once per link on it
// (L = 4 or 6 times) with its c_P, so with the plaquette staple sum Pl,
//   S_G = (beta/3) sum_links [ 3 (1.5 c_plaq + 3 c_rect + 4 c_cube)
//                              - Re tr(U t)/6 - (c_plaq/12) Re tr(U Pl) ]
// (Eq. 18_6_4_1), each link's share formed in the working precision from its
// two traces and summed in FP64.
//
// Work decomposition.  Both passes run in "virtual blocks" of 128 threads:
// the four warps of a block take the four directions of the same 32 sites
// (the planes around a site are read while they are in L1/L2, and each warp
// reads one plane per instruction, so a quarter-warp covers 8 consecutive
// sites of one 128-byte line).  A single lattice is launched with one CTA per
// virtual block; a batch of lattices of different extents runs as one
// persistent launch whose CTAs take the virtual blocks of all lattices from
// a work counter.  The
// action partial sum of a virtual block is the same in both, so a batched
// result equals the single-lattice result bit for bit.
#include <atomic>
#include <mutex>

#include "kernels.h"
#include "su3.cuh"

namespace lqcd {

namespace {

constexpr int kBlock = 128; // four warps: the four directions of 32 sites

__host__ __device__ __forceinline__ int64_t padded_sites(int64_t V) { return (V + 31) & ~(int64_t)31; }
__host__ __device__ __forceinline__ int64_t virtual_blocks(int64_t V) { return padded_sites(V) / 32; }

enum { SC_BETA6 = 0, SC_CPL, SC_CRT, SC_CCB, SC_ACT, SC_ACTPL, SC_DT };

template <typename R> __device__ __forceinline__ R scalar(const KernelScalars &s, int i)
{
    if constexpr (sizeof(R) == 4) return s.f[i];
    else return s.d[i];
}

// Storage of the 24 staple planes: compact (rows 0 and 1, 12 reals, the
// third row rebuilt on load) or full (all 18 reals, nothing rebuilt).  Both
// are cut into blocks of 32 consecutive sites: inside a block, 16-byte lane
// q (q < NW = 12/W compact, 18/W full) of the staple of site s is at
// q*512 + s*16 bytes, and for full FP32 staples the last two reals at
// NW*512 + s*8 -- 72 bytes per full staple in FP32, 144 in FP64, every
// access 16- or 8-byte aligned, and the lanes of one staple a constant 512
// bytes apart, so that a staple costs one address computation (plus one for
// the FP32 tail) however many lanes it has.  Plane P starts at
// P * plane_bytes, plane_bytes = the
// 32-site blocks of the lattice (V rounded up to 32) times the block size.
// Pass A writes them with evict-first stores: the 3.6 GB (at 32^3x64) would
// otherwise push the links that pass A re-reads out of L2.
constexpr int kStaplePlanes = 24;

template <typename R> struct FullBlock {
    using V4 = typename Vec<R>::type;
    static constexpr int W = Vec<R>::W;
    static constexpr int NW = 18 / W;        // whole 16-byte lanes per staple
    static constexpr int TAIL = 18 - NW * W; // reals in the FP32 tail (2)
    static constexpr int LANE = 32 * 16;     // bytes of one lane of a block
    static constexpr int BYTES = NW * LANE + TAIL * (int)sizeof(R) * 32;
    static_assert(NW * W + TAIL == 18, "a full staple holds 18 reals");
};

size_t full_plane_bytes(int64_t V, int precision)
{
    const size_t blk = precision == LQCD_F64 ? FullBlock<double>::BYTES : FullBlock<float>::BYTES;
    return (size_t)((V + 31) / 32) * blk;
}

// Compact planes: the first two rows (12 reals) of every staple, the third
// rebuilt on load, in the same 32-site blocks (lane q, q < 12/W, of site s at
// q*512 + s*16).
template <typename R> struct CompactBlock {
    using V4 = typename Vec<R>::type;
    static constexpr int W = Vec<R>::W;
    static constexpr int NW = 12 / W;
    static constexpr int LANE = 32 * 16;
    static constexpr int BYTES = NW * LANE;
};

template <typename R, bool FULL> struct Planes;

template <typename R> struct Planes<R, false> {
    using B = CompactBlock<R>;
    using V4 = typename B::V4;
    char *base;
    int64_t plane_bytes;
    using Ref = char *;

    __device__ __forceinline__ Ref at(int n) const
    {
        return base + (int64_t)(n >> 5) * B::BYTES + (n & 31) * 16;
    }

    __device__ __forceinline__ Mat<R> load(Ref r, int plane) const
    {
        const V4 *p = reinterpret_cast<const V4 *>(r + (int64_t)plane * plane_bytes);
        R x[12];
#pragma unroll
        for (int q = 0; q < B::NW; ++q) {
            const V4 v = __ldg(p + q * (B::LANE / 16));
            if constexpr (B::W == 4) {
                x[4 * q + 0] = v.x;
                x[4 * q + 1] = v.y;
                x[4 * q + 2] = v.z;
                x[4 * q + 3] = v.w;
            } else {
                x[2 * q + 0] = v.x;
                x[2 * q + 1] = v.y;
            }
        }
        Mat<R> u;
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                u.re[i][j] = x[6 * i + 2 * j];
                u.im[i][j] = x[6 * i + 2 * j + 1];
            }
        rebuild_row2(u);
        return u;
    }

    __device__ __forceinline__ void store(Ref r, int plane, const Mat<R> &u) const
    {
        V4 *p = reinterpret_cast<V4 *>(r + (int64_t)plane * plane_bytes);
        R x[12];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                x[6 * i + 2 * j] = u.re[i][j];
                x[6 * i + 2 * j + 1] = u.im[i][j];
            }
#pragma unroll
        for (int q = 0; q < B::NW; ++q) {
            V4 v;
            if constexpr (B::W == 4) v = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
            else v = make_double2(x[2 * q], x[2 * q + 1]);
            __stcs(p + q * (B::LANE / 16), v);
        }
    }
};

template <typename R> struct Planes<R, true> {
    using B = FullBlock<R>;
    using V4 = typename B::V4;
    char *base;          // plane 0
    int64_t plane_bytes;

    // The lane-0 and tail addresses of site n in plane 0.
    struct Ref {
        char *p;
        char *t;
    };

    __device__ __forceinline__ Ref at(int n) const
    {
        char *b = base + (int64_t)(n >> 5) * B::BYTES;
        const int s = n & 31;
        return Ref{b + s * 16, b + B::NW * B::LANE + s * 8};
    }

    __device__ __forceinline__ Mat<R> load(const Ref &r, int plane) const
    {
        const int64_t off = (int64_t)plane * plane_bytes;
        const V4 *p = reinterpret_cast<const V4 *>(r.p + off);
        R x[18];
#pragma unroll
        for (int q = 0; q < B::NW; ++q) {
            const V4 v = __ldg(p + q * (B::LANE / 16));
            if constexpr (B::W == 4) {
                x[4 * q + 0] = v.x;
                x[4 * q + 1] = v.y;
                x[4 * q + 2] = v.z;
                x[4 * q + 3] = v.w;
            } else {
                x[2 * q + 0] = v.x;
                x[2 * q + 1] = v.y;
            }
        }
        if constexpr (B::TAIL == 2) {
            const float2 t = __ldg(reinterpret_cast<const float2 *>(r.t + off));
            x[16] = t.x;
            x[17] = t.y;
        }
        Mat<R> u;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                u.re[i][j] = x[2 * (3 * i + j)];
                u.im[i][j] = x[2 * (3 * i + j) + 1];
            }
        return u;
    }

    __device__ __forceinline__ void store(const Ref &r, int plane, const Mat<R> &u) const
    {
        const int64_t off = (int64_t)plane * plane_bytes;
        V4 *p = reinterpret_cast<V4 *>(r.p + off);
        R x[18];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                x[2 * (3 * i + j)] = u.re[i][j];
                x[2 * (3 * i + j) + 1] = u.im[i][j];
            }
#pragma unroll
        for (int q = 0; q < B::NW; ++q) {
            V4 v;
            if constexpr (B::W == 4) v = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
            else v = make_double2(x[2 * q], x[2 * q + 1]);
            __stcs(p + q * (B::LANE / 16), v);
        }
        if constexpr (B::TAIL == 2) __stcs(reinterpret_cast<float2 *>(r.t + off), make_float2(x[16], x[17]));
    }
};

template <typename R, bool FULL> __device__ __forceinline__ Planes<R, FULL> planes_of(const SfLattice &L)
{
    if constexpr (FULL) {
        return Planes<R, true>{static_cast<char *>(L.staples), L.plane_bytes};
    } else {
        const int64_t V = (int64_t)L.dims[0] * L.dims[1] * L.dims[2] * L.dims[3];
        return Planes<R, false>{static_cast<char *>(L.staples),
                                ((V + 31) / 32) * CompactBlock<R>::BYTES};
    }
}

// Lattice geometry in 32-bit arithmetic: the staple-field algorithm runs only
// for V < 2^31 sites (its workspace, 1728 bytes a site in FP32, could not
// hold more), so site indices and neighbour offsets fit an int.
struct G32 {
    int L0, L1, L2, L3;
    int s1, s2, s3, V;
};

__device__ __forceinline__ G32 make_g32(const int dims[4])
{
    G32 g;
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

// Slots of SfLattice::div (the magic of each run-time divisor).
enum { DV_S1, DV_S2, DV_S3, DV_VOL, DV_SLICE, DV_MVOL, DV_MX, DV_MY, DV_NMX, DV_NMY, DV_NBX, DV_NBY };

__device__ __forceinline__ int divi(int n, const DivMagic &d) { return (int)div_by((unsigned)n, d); }

// Coordinates of site n (the divisions by the strides as multiply-highs).
__device__ __forceinline__ Coord coord32(const G32 &g, const DivMagic *dm, int n)
{
    Coord x;
    x.c3 = divi(n, dm[DV_S3]);
    int r = n - x.c3 * g.s3;
    x.c2 = divi(r, dm[DV_S2]);
    r -= x.c2 * g.s2;
    x.c1 = divi(r, dm[DV_S1]);
    x.c0 = r - x.c1 * g.s1;
    return x;
}

__device__ __forceinline__ int index32(const G32 &g, const Coord &x)
{
    return x.c0 + g.s1 * x.c1 + g.s2 * x.c2 + g.s3 * x.c3;
}

// Index offset of the step s * hat(mu) (s = +-1) from a site with
// coordinates x, periodic (the direction picked by a select chain, so that
// nothing is indexed at run time in per-thread storage).
__device__ __forceinline__ int step32(const G32 &g, const Coord &x, int mu, int s)
{
    const int L = pick(mu, g.L0, g.L1, g.L2, g.L3);
    const int c = pick(mu, x.c0, x.c1, x.c2, x.c3);
    const int st = pick(mu, 1, g.s1, g.s2, g.s3);
    if (s > 0) return c + 1 == L ? (1 - L) * st : st;
    return c == 0 ? (L - 1) * st : -st;
}

// Traversal order of pass B: the lattice is cut into spatial blocks of
// bx x by x bz sites that run over all t; blocks one after the other, inside
// a block t-slice by t-slice, inside a slice micro-tiles of mx x my x mz
// sites (x fastest within and between micro-tiles).  The staple planes of
// three neighbouring t-slices of one block then stay in L2 while the block
// is swept, and micro-tiles make y and z neighbours L1 hits.
struct Sweep {
    int bx, by, bz, mx, my, mz;
    int nbx, nby, nmx, nmy, mvol;
    int slice, vol;     // sites per block slice and per block
    const DivMagic *dm; // magic of vol, slice, mvol, mx, my, nmx, nmy, nbx, nby
};

__device__ __forceinline__ Sweep make_sweep(const SfLattice &L, const G32 &g)
{
    Sweep s;
    s.bx = L.sweep[0];
    s.by = L.sweep[1];
    s.bz = L.sweep[2];
    s.mx = L.micro[0];
    s.my = L.micro[1];
    s.mz = L.micro[2];
    s.nbx = L.counts[0];
    s.nby = L.counts[1];
    s.nmx = L.counts[2];
    s.nmy = L.counts[3];
    s.mvol = s.mx * s.my * s.mz;
    s.slice = s.bx * s.by * s.bz;
    s.vol = s.slice * g.L3;
    s.dm = L.div;
    return s;
}

__device__ __forceinline__ Coord swept_site(const Sweep &s, int j)
{
    const DivMagic *dm = s.dm;
    const int blk = divi(j, dm[DV_VOL]);
    const int r = j - blk * s.vol;
    Coord c;
    c.c3 = divi(r, dm[DV_SLICE]);
    const int r2 = r - c.c3 * s.slice;
    const int mt = divi(r2, dm[DV_MVOL]), w = r2 - mt * s.mvol;
    const int wq = divi(w, dm[DV_MX]), xin = w - wq * s.mx;
    const int zin = divi(wq, dm[DV_MY]), yin = wq - zin * s.my;
    const int mq = divi(mt, dm[DV_NMX]), mxi = mt - mq * s.nmx;
    const int mzi = divi(mq, dm[DV_NMY]), myi = mq - mzi * s.nmy;
    const int q = divi(blk, dm[DV_NBX]), bxi = blk - q * s.nbx;
    const int bzi = divi(q, dm[DV_NBY]), byi = q - bzi * s.nby;
    c.c0 = bxi * s.bx + mxi * s.mx + xin;
    c.c1 = byi * s.by + myi * s.my + yin;
    c.c2 = bzi * s.bz + mzi * s.mz + zin;
    return c;
}

// Sum over the block of one double per thread (result in thread 0); the
// trailing barrier lets the caller run it again in the next virtual block.
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double part[kBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) part[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (warp == 0) {
        s = lane < kBlock / 32 ? part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;
}

// block_sum over the four warps of row group `row` of a CTA of ROWS groups
// (named barrier 1 + row over its 128 threads; same order of summation).
template <int ROWS> __device__ __forceinline__ double group_sum(double v, int row)
{
    if constexpr (ROWS == 1) {
        return block_sum(v);
    } else {
        __shared__ double part[ROWS * kBlock / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) part[warp] = v;
        asm volatile("bar.sync %0, %1;" ::"r"(1 + row), "r"(kBlock) : "memory");
        double s = 0.0;
        if ((warp & 3) == 0) {
            s = lane < kBlock / 32 ? part[warp + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        }
        asm volatile("bar.sync %0, %1;" ::"r"(1 + row), "r"(kBlock) : "memory");
        return s;
    }
}

// Next virtual block for a persistent CTA of a batched launch, taken from a
// work counter: the blocks in flight stay a contiguous window of the sweep
// (as with hardware block scheduling), which keeps the L2 reuse of the
// traversal; a fixed stride per CTA would let the window spread out.
__device__ __forceinline__ int64_t next_virtual_block(unsigned long long *counter)
{
    __shared__ unsigned long long s_vb;
    if (threadIdx.x == 0) s_vb = atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t vb = (int64_t)s_vb;
    __syncthreads();
    return vb;
}

// The same queue with the next block claimed (by thread 0) when the current
// one starts and handed to the block when it ends, so that the atomic's
// latency overlaps the current block's work.
__device__ __forceinline__ unsigned long long claim_virtual_block(unsigned long long *counter)
{
    return threadIdx.x == 0 ? atomicAdd(counter, 1ull) : 0ull;
}

__device__ __forceinline__ int64_t publish_virtual_block(unsigned long long claimed)
{
    __shared__ unsigned long long s_vb;
    if (threadIdx.x == 0) s_vb = claimed;
    __syncthreads();
    const int64_t vb = (int64_t)s_vb;
    __syncthreads();
    return vb;
}

// Lattice of a batch that virtual block vb (global numbering) belongs to.
__device__ __forceinline__ int batch_entry(const SfBatch &B, int64_t vb)
{
    int c = 0;
    while (c + 1 < B.n && vb >= B.e[c + 1].vb_begin) ++c;
    return c;
}

// ---------------------------------------------------------------- pass A

// The six staples S^{(mu)}_b, b = +-nu (nu != mu), of the link (x, mu), x
// at coordinates c; stored at staple index sx of sf.
template <typename R, bool FULL>
__device__ __forceinline__ void site_staples(const R *__restrict__ links, const G32 &g, const Coord &c,
                                             int x, int mu, const Planes<R, FULL> &sf, int sx)
{
    const int64_t V = g.V;
    const int xm = x + step32(g, c, mu, 1); // x + mu
    const auto at = sf.at(sx);
#pragma unroll 1
    for (int iv = 0; iv < 3; ++iv) {
        const int nu = (mu + 1 + iv) & 3;
        const int vp = step32(g, c, nu, 1), vm = step32(g, c, nu, -1);
        // b = +nu:  U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
        // rows 0 and 1 of each staple (which need rows 0 and 1 of the first
        // product only); a full plane takes its third row from them, the
        // staple being a product of three SU(3) links
        Mat<R> t = mul<N, D>(load_link(links, V, nu, xm), load_link(links, V, mu, x + vp));
        Mat<R> up = mul_top2<N, D>(t, load_link(links, V, nu, x));
        if constexpr (FULL) rebuild_row2(up);
        sf.store(at, mu * 6 + 2 * iv, up);
        // b = -nu:  U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
        t = mul<D, D>(load_link(links, V, nu, xm + vm), load_link(links, V, mu, x + vm));
        Mat<R> dn = mul_top2<N, N>(t, load_link(links, V, nu, x + vm));
        if constexpr (FULL) rebuild_row2(dn);
        sf.store(at, mu * 6 + 2 * iv + 1, dn);
    }
}

// The 24 staples of the 32 sites of virtual block vb: thread = (site, mu).
template <typename R, bool FULL>
__device__ __forceinline__ void staples_block(const SfLattice &L, const G32 &g, int vb)
{
    const int mu = (int)(threadIdx.x >> 5);
    const int x = vb * 32 + (int)(threadIdx.x & 31);
    if (x >= g.V) return;
    site_staples<R, FULL>(static_cast<const R *>(L.links), g, coord32(g, L.div, x), x, mu,
                                planes_of<R, FULL>(L), x);
}

template <typename R, bool FULL>
__global__ void __launch_bounds__(kBlock) staple_fields(const __grid_constant__ SfLattice L)
{
    const G32 g = make_g32(L.dims);
    const int nvb = (int)virtual_blocks(g.V);
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) staples_block<R, FULL>(L, g, vb);
}

template <typename R, bool FULL>
__global__ void __launch_bounds__(kBlock) staple_fields_batched(const __grid_constant__ SfBatch B)
{
    for (int64_t vb = next_virtual_block(B.counter); vb < B.total;) {
        const unsigned long long next = claim_virtual_block(B.counter);
        const int c = batch_entry(B, vb);
        const SfLattice &L = B.e[c];
        staples_block<R, FULL>(L, make_g32(L.dims), (int)(vb - L.vb_begin));
        vb = publish_virtual_block(next);
    }
}

// ---------------------------------------------------------------- pass B

// Products of two SU(3) factors are accumulated as y += s * (a * op(b)) with
// the third row of the product rebuilt from its first two (mul_acc_su3: the
// third row of a is never rebuilt or loaded), or (DIRECT, full FP64 staples)
// as plain products accumulated in full, the sum scaled once: for FP64 that
// measured faster (114 vs 122 ms at 32^3x64: at the 255-register limit the
// extra temporaries spill); for FP32 the rebuilt form is faster (3.65 vs
// 3.75 ms).
template <int FB, bool DIRECT, typename R>
__device__ __forceinline__ void acc_su3(Mat<R> &y, const Mat<R> &a, const Mat<R> &b, R s)
{
    if constexpr (DIRECT) mul_acc<N, FB>(y, a, b); // s applied by the caller
    else mul_acc_su3<FB>(y, a, b, s);
}

// Where the staples of a site and of its neighbours are stored: in the
// lattice-wide staple field, the site index itself.
struct LatticeSites {
    const G32 *g;
    const Coord *c;
    int k;
    __device__ __forceinline__ int at0() const { return k; }
    __device__ __forceinline__ int nb(int mu, int s) const { return k + step32(*g, *c, mu, s); }
};

// The staples that start with link(k+rho, d), d = +-nu_d (NEG: minus):
//   t += B_d [ c_cube sum_{b perp rho, d} S_b(k+d) S^{(d)}_b(k) + c_rect S_d(k+d) A_d^dag ]
// (the orientation of the shared links fixed at compile time, so that each
// sign has one small loop body).
template <bool NEG, bool UNROLLQ, bool FULL, bool DIRECT, typename R, typename SI>
__device__ __forceinline__ void d_terms(Mat<R> &t, const R *__restrict__ links,
                                        const Planes<R, FULL> &sf, const SI &si, const G32 &g,
                                        const Coord &c, int rho, int k, int kp, int id, R c_rt,
                                        R c_cb)
{
    constexpr int FD = NEG ? D : N;
    const int64_t V = g.V;
    const int base = rho * 6;
    const int jd = 2 * id + (NEG ? 1 : 0);
    const int nud = (rho + 1 + id) & 3;
    const int kd = k + step32(g, c, nud, NEG ? -1 : 1); // k + d
    // S^{(d)}_b(k): plane nud*6 + j' at k, or (NEG) its dagger at k - nud = kd
    const auto at_d = sf.at(si.nb(nud, NEG ? -1 : 1));
    const auto at_2 = NEG ? at_d : sf.at(si.at0());
    Mat<R> y;
    set_zero(y);
    // the four signed b perpendicular to rho and d: two directions, two signs
#pragma unroll(UNROLLQ ? 2 : 1)
    for (int q = 0; q < 2; ++q) {
        const int ib = q == 0 ? (id == 0 ? 1 : 0) : (id == 2 ? 1 : 2);
        const int nub = (rho + 1 + ib) & 3;
        const int jp = 2 * ((nub - nud - 1) & 3);
        acc_su3<FD, DIRECT>(y, sf.load(at_d, base + 2 * ib),
                            sf.load(at_2, nud * 6 + jp), c_cb);
        acc_su3<FD, DIRECT>(y, sf.load(at_d, base + 2 * ib + 1),
                            sf.load(at_2, nud * 6 + jp + 1), c_cb);
    }
    Mat<R> r3 = sf.load(at_d, base + jd);
    if constexpr (DIRECT) {
        scale(y, c_cb);
        scale(r3, c_rt);
    }
    if constexpr (!NEG) {
        acc_su3<D, DIRECT>(y, r3, load_link(links, V, nud, k), c_rt); // A_d = U_nud(k)
        mul_acc<N, N>(t, load_link(links, V, nud, kp), y);         // B_d = U_nud(k+rho)
    } else {
        acc_su3<N, DIRECT>(y, r3, load_link(links, V, nud, kd), c_rt);  // A_d = U_nud(k-nud)^dag
        mul_acc<D, N>(t, load_link(links, V, nud, kp + (kd - k)), y);  // B_d = U_nud(k+rho-nud)^dag
    }
}

// Force (and the fused momentum step) on the link (k, rho), k at coordinates
// c, its staples found through si; returns its share of the action.
template <typename R, bool ACTION, bool UNROLLQ, bool FULL, bool DIRECT, typename SI>
__device__ __forceinline__ double force_link(const SfLattice &L, const KernelScalars &sc, const G32 &g,
                                             const Planes<R, FULL> &sf, const SI &si, const Coord &c,
                                             int k, int rho)
{
    const R *__restrict__ links = static_cast<const R *>(L.links);
    const int64_t V = g.V;
    const R c_pl = scalar<R>(sc, SC_CPL), c_rt = scalar<R>(sc, SC_CRT), c_cb = scalar<R>(sc, SC_CCB);
    const int kp = k + step32(g, c, rho, 1), km = k + step32(g, c, rho, -1);
    const int base = rho * 6;

    // plaquettes and the two rectangle chains along rho
    Mat<R> t;
    R tr_pl = R(0);
    {
        Mat<R> pl, p1, p2;
        set_zero(pl);
        set_zero(p1);
        set_zero(p2);
        const auto at_k = sf.at(si.at0()), at_p = sf.at(si.nb(rho, 1)), at_m = sf.at(si.nb(rho, -1));
#pragma unroll 1
        for (int jj = 0; jj < 6; ++jj) {
            const Mat<R> s = sf.load(at_k, base + jj);
            add_to(pl, s);
            acc_su3<N, DIRECT>(p1, sf.load(at_p, base + jj), s, c_rt);
            mul_acc<N, N>(p2, s, sf.load(at_m, base + jj));
        }
        if constexpr (ACTION) tr_pl = re_trace_mul<N, N>(load_link(links, V, rho, k), pl);
        t = pl;
        scale(t, c_pl);
        if constexpr (DIRECT) scale(p1, c_rt);
        mul_acc<N, N>(t, load_link(links, V, rho, kp), p1);
        scale(p2, c_rt);
        mul_acc<N, N>(t, p2, load_link(links, V, rho, km));
    }
    // cubes and the rectangles along d: positive, then negative d
#pragma unroll 1
    for (int id = 0; id < 3; ++id)
        d_terms<false, UNROLLQ, FULL, DIRECT>(t, links, sf, si, g, c, rho, k, kp, id, c_rt, c_cb);
#pragma unroll 1
    for (int id = 0; id < 3; ++id)
        d_terms<true, UNROLLQ, FULL, DIRECT>(t, links, sf, si, g, c, rho, k, kp, id, c_rt, c_cb);

    const Mat<R> m = mul<N, N>(load_link(links, V, rho, k), t);
    R f[8];
    ta_components(m, scalar<R>(sc, SC_BETA6), f);
    if (L.force != nullptr) store_algebra(static_cast<R *>(L.force), V, rho, k, f);
    if (L.mom != nullptr) {
        R *mom = static_cast<R *>(L.mom);
        R p[8];
        load_algebra(mom, V, rho, k, p);
        const R dt = scalar<R>(sc, SC_DT);
#pragma unroll
        for (int q = 0; q < 8; ++q) p[q] = fma(dt, f[q], p[q]);
        store_algebra(mom, V, rho, k, p);
    }
    if constexpr (ACTION) {
        const R tr_t = m.re[0][0] + m.re[1][1] + m.re[2][2];
        return (double)(scalar<R>(sc, SC_ACT) - tr_t * R(1.0 / 6.0) - scalar<R>(sc, SC_ACTPL) * tr_pl);
    }
    return 0.0;
}

// Force (and the fused momentum step) on the 128 links of virtual block vb
// of the sweep; returns the thread's share of the action (0 for a padding
// site).
template <typename R, bool ACTION, bool UNROLLQ, bool FULL, bool DIRECT>
__device__ __forceinline__ double force_block(const SfLattice &L, const KernelScalars &sc,
                                              const G32 &g, const Sweep &sw, int vb)
{
    const int rho = (int)((threadIdx.x >> 5) & 3);
    const int j = vb * 32 + (int)(threadIdx.x & 31);
    if (j >= g.V) return 0.0;
    const Coord c = swept_site(sw, j);
    const int k = index32(g, c);
    const LatticeSites si{&g, &c, k};
    return force_link<R, ACTION, UNROLLQ, FULL, DIRECT>(L, sc, g, planes_of<R, FULL>(L), si, c, k,
                                                        rho);
}

// Resident CTAs per SM the register allocation aims at: 4 (128 registers)
// unless the fused action asks for more registers (3) -- or DENSE forces 4.
template <typename R, bool ACTION, bool DENSE> constexpr int min_blocks()
{
    return sizeof(R) == 8 ? 2 : ((ACTION && !DENSE) ? 3 : 4);
}

// DIRECT products by default for full FP64 planes (see acc_su3).
template <typename R, bool FULL> constexpr bool direct_default() { return FULL && sizeof(R) == 8; }

// ROWS > 1: a CTA of ROWS groups of four warps on consecutive virtual
// blocks (y-neighbouring x rows of the sweep), so that the staples of a
// row's +-y neighbours are the own-row staples of another group of the CTA.
template <typename R, bool ACTION, bool UNROLLQ, bool DENSE = false, bool FULL = false,
          bool DIRECT = direct_default<R, FULL>(), int ROWS = 1>
__global__ void __launch_bounds__(ROWS * kBlock, (min_blocks<R, ACTION, DENSE>() / ROWS > 0
                                                       ? min_blocks<R, ACTION, DENSE>() / ROWS
                                                       : 1))
    force_from_staples(const __grid_constant__ SfLattice L, const __grid_constant__ KernelScalars sc)
{
    const G32 g = make_g32(L.dims);
    const Sweep sw = make_sweep(L, g);
    const int nvb = (int)virtual_blocks(g.V);
    const int row = ROWS == 1 ? 0 : (int)(threadIdx.x >> 7);
    for (int vb0 = blockIdx.x * ROWS; vb0 < nvb; vb0 += gridDim.x * ROWS) {
        const int vb = vb0 + row;
        double acc = 0.0;
        if (vb < nvb) acc = force_block<R, ACTION, UNROLLQ, FULL, DIRECT>(L, sc, g, sw, vb);
        if constexpr (ACTION) {
            const double s = group_sum<ROWS>(acc, row);
            if ((threadIdx.x & (kBlock - 1)) == 0 && vb < nvb) L.partials[vb] = s;
        }
    }
}

template <typename R, bool ACTION, bool UNROLLQ, bool DENSE = false, bool FULL = false,
          bool DIRECT = direct_default<R, FULL>()>
__global__ void __launch_bounds__(kBlock, (min_blocks<R, ACTION, DENSE>()))
    force_from_staples_batched(const __grid_constant__ SfBatch B,
                               const __grid_constant__ KernelScalars sc)
{
    for (int64_t vb = next_virtual_block(B.counter + 1); vb < B.total;) {
        const unsigned long long next = claim_virtual_block(B.counter + 1);
        const int c = batch_entry(B, vb);
        const SfLattice &L = B.e[c];
        const G32 g = make_g32(L.dims);
        const double acc = force_block<R, ACTION, UNROLLQ, FULL, DIRECT>(
            L, sc, g, make_sweep(L, g), (int)(vb - L.vb_begin));
        if constexpr (ACTION) {
            const double s = block_sum(acc);
            if (threadIdx.x == 0) L.partials[vb - L.vb_begin] = s;
        }
        vb = publish_virtual_block(next);
    }
}

// One block per lattice of a batch: its action from its partial sums, in the
// order and grouping of finish_sum, so batched and single results agree.
__global__ void __launch_bounds__(1024) finish_batched(const __grid_constant__ SfBatch B, double scale)
{
    const SfLattice &L = B.e[blockIdx.x];
    if (L.action == nullptr) return;
    const int count = (int)virtual_blocks((int64_t)L.dims[0] * L.dims[1] * L.dims[2] * L.dims[3]);
    __shared__ double warp_part[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < count; i += 1024) v += L.partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double s = warp_part[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) *L.action = scale * s;
    }
}

unsigned grid_of(int64_t items)
{
    if (items < 1) items = 1;
    if (items > ((int64_t)1 << 30)) items = (int64_t)1 << 30;
    return (unsigned)items;
}

// Pass-B schedules (same arithmetic, different traversal or occupancy):
//   0  micro-tiles 8x2x2, inner b loop rolled
//   1  micro-tiles 8x2x2, inner b loop unrolled
//   2  x rows (no micro-tiles), inner b loop rolled
//   3  x rows, registers capped for 4 CTAs/SM also with the fused action
//   4  x rows, staple planes stored full (18 reals, no row rebuilt on load),
//      spatial blocks up to 64x8x8 (full planes are 1.5x the bytes per site:
//      smaller blocks keep the sweep's working set in L2; 4.22 against
//      4.45 ms with 64x16x16 at 32^3x64 FP32)
//   5  as 4, registers capped for 4 CTAs/SM
//   6  as 4 with spatial blocks up to 64x16x16
//   7  as 5 in CTAs of two groups of four warps on consecutive virtual
//      blocks: with x extent 32 those are y-neighbouring x rows, and a row's
//      +-y staples are the other group's own staples (L1 hits)
//   8  as 7 with spatial blocks up to 64x16x8
// The process-wide choice per precision is set by lqcd_set_force_variant or
// lqcd_autotune_force; -1 means the default (default_variant).
constexpr int kSfVariants = 9;

// Built-in choice: full staples with the 4-CTA register cap in FP32 (at
// 32^3x64 3.42 ms against 3.45-3.46 ms for the two-row CTAs and 3.64-3.66
// for the others; at 32^4 1.73 against 1.75 ms), uncapped full staples in
// FP64 (110 against 128 ms with compact ones; two-row CTAs 110.2-110.3).
// The two-row CTAs won (3.54 against 3.67 ms at 32^3x64) while the sweep
// still divided by run-time extents; with multiply-high divisions the
// one-row CTA is ahead.  The dims are kept for shape-dependent choices.
int default_variant(int precision, const int dims[4])
{
    (void)dims;
    return precision == LQCD_F64 ? 4 : 5;
}

bool full_staples(int variant) { return variant >= 4; }

// Slot of a kernel instance in the occupancy cache of persistent_grid:
// kind (0 pass B, 1 pass B capped, 2 pass B full, 3 pass B full capped,
// 4 pass A compact, 5 pass A full) x precision x action x unrolled.
int grid_slot(int kind, bool f64, bool action, bool unrolled)
{
    return kind * 8 + (f64 ? 4 : 0) + (action ? 2 : 0) + (unrolled ? 1 : 0);
}
std::atomic<int> g_sf_variant[2] = {{-1}, {-1}};

// Largest divisor of L not above cap.
int block_extent(int L, int cap)
{
    for (int b = cap < L ? cap : L; b > 1; --b)
        if (L % b == 0) return b;
    return 1;
}

void set_traversal(SfLattice &L, int variant)
{
    const int cap_y = (variant == 4 || variant == 5 || variant == 7) ? 8 : 16;
    const int cap_z = (variant >= 4 && variant != 6) ? 8 : 16;
    L.sweep[0] = block_extent(L.dims[0], 64);
    L.sweep[1] = block_extent(L.dims[1], cap_y);
    L.sweep[2] = block_extent(L.dims[2], cap_z);
    if (variant >= 2) {
        L.micro[0] = L.sweep[0];
        L.micro[1] = L.micro[2] = 1;
    } else {
        L.micro[0] = block_extent(L.sweep[0], 8);
        L.micro[1] = L.sweep[1] % 2 == 0 ? 2 : 1;
        L.micro[2] = L.sweep[2] % 2 == 0 ? 2 : 1;
    }
    // the divisors of coord32 and swept_site (all below 2^31: V < 2^31)
    const int *d = L.dims;
    const int64_t slice = (int64_t)L.sweep[0] * L.sweep[1] * L.sweep[2];
    const int64_t dv[12] = {d[0],
                            (int64_t)d[0] * d[1],
                            (int64_t)d[0] * d[1] * d[2],
                            slice * d[3],
                            slice,
                            (int64_t)L.micro[0] * L.micro[1] * L.micro[2],
                            L.micro[0],
                            L.micro[1],
                            L.sweep[0] / L.micro[0],
                            L.sweep[1] / L.micro[1],
                            d[0] / L.sweep[0],
                            d[1] / L.sweep[1]};
    for (int i = 0; i < 12; ++i) L.div[i] = div_magic((unsigned)(dv[i] > 0 ? dv[i] : 1));
    L.counts[0] = (int)dv[DV_NBX];
    L.counts[1] = (int)dv[DV_NBY];
    L.counts[2] = (int)dv[DV_NMX];
    L.counts[3] = (int)dv[DV_NMY];
}

KernelScalars make_scalars(const ForceArgs &a)
{
    KernelScalars k;
    const double sc[7] = {a.beta / 6.0, a.c_plaq, a.c_rect, a.c_cube,
                          3.0 * (1.5 * a.c_plaq + 3.0 * a.c_rect + 4.0 * a.c_cube), a.c_plaq / 12.0,
                          a.dt};
    for (int i = 0; i < 7; ++i) {
        k.d[i] = sc[i];
        k.f[i] = (float)sc[i];
    }
    return k;
}

int resolve_variant(const ForceArgs &a)
{
    if (a.variant >= 0 && a.variant < kSfVariants) return a.variant;
    const int p = a.precision == LQCD_F64 ? 1 : 0;
    const int v = g_sf_variant[p].load();
    return v < 0 ? default_variant(a.precision, a.dims) : v;
}

// CTAs of a persistent launch: as many as are resident on the device at
// once (occupancy of the kernel times the SM count, cached per device).
template <typename K> unsigned persistent_grid(K kernel, int slot, int64_t work)
{
    static std::mutex mu;
    static int cached[64][48] = {{0}};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return grid_of(work);
    int resident = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (cached[dev][slot] == 0) {
            int sms = 0, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
            cached[dev][slot] = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
        }
        resident = cached[dev][slot];
    }
    return grid_of(work < resident ? work : resident);
}

template <typename R, bool ACTION>
cudaError_t launch_pass_b(const SfLattice &L, const KernelScalars &sc, int variant, cudaStream_t st)
{
    const int64_t V = (int64_t)L.dims[0] * L.dims[1] * L.dims[2] * L.dims[3];
    const unsigned grid = grid_of(virtual_blocks(V));
    if (variant == 1) force_from_staples<R, ACTION, true><<<grid, kBlock, 0, st>>>(L, sc);
    else if (variant == 3) force_from_staples<R, ACTION, false, true><<<grid, kBlock, 0, st>>>(L, sc);
    else if (variant == 4 || variant == 6)
        force_from_staples<R, ACTION, false, false, true><<<grid, kBlock, 0, st>>>(L, sc);

    else if (variant == 5)
        force_from_staples<R, ACTION, false, true, true><<<grid, kBlock, 0, st>>>(L, sc);
    else if (variant >= 7)
        force_from_staples<R, ACTION, false, true, true, direct_default<R, true>(), 2>
            <<<grid_of((virtual_blocks(V) + 1) / 2), 2 * kBlock, 0, st>>>(L, sc);
    else force_from_staples<R, ACTION, false><<<grid, kBlock, 0, st>>>(L, sc);
    return cudaGetLastError();
}

template <typename R, bool ACTION>
cudaError_t launch_pass_b_batched(const SfBatch &B, const KernelScalars &sc, int variant,
                                  cudaStream_t st)
{
    constexpr bool f64 = sizeof(R) == 8;
    if (variant == 1) {
        auto k = force_from_staples_batched<R, ACTION, true>;
        k<<<persistent_grid(k, grid_slot(0, f64, ACTION, true), B.total), kBlock, 0, st>>>(B, sc);
    } else if (variant == 3) {
        auto k = force_from_staples_batched<R, ACTION, false, true>;
        k<<<persistent_grid(k, grid_slot(1, f64, ACTION, false), B.total), kBlock, 0, st>>>(B, sc);
    } else if (variant == 4 || variant == 6) {
        auto k = force_from_staples_batched<R, ACTION, false, false, true>;
        k<<<persistent_grid(k, grid_slot(2, f64, ACTION, false), B.total), kBlock, 0, st>>>(B, sc);
    } else if (variant == 5 || variant >= 7) {
        auto k = force_from_staples_batched<R, ACTION, false, true, true>;
        k<<<persistent_grid(k, grid_slot(3, f64, ACTION, false), B.total), kBlock, 0, st>>>(B, sc);
    } else {
        auto k = force_from_staples_batched<R, ACTION, false>;
        k<<<persistent_grid(k, grid_slot(0, f64, ACTION, false), B.total), kBlock, 0, st>>>(B, sc);
    }
    return cudaGetLastError();
}

size_t round_up256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename R> cudaError_t launch_sf_t(const ForceArgs &a, cudaStream_t st)
{
    const int variant = resolve_variant(a);
    SfLattice L{};
    for (int i = 0; i < 4; ++i) L.dims[i] = a.dims[i];
    set_traversal(L, variant);
    L.plane_bytes = (int64_t)full_plane_bytes((int64_t)a.dims[0] * a.dims[1] * a.dims[2] * a.dims[3],
                                              a.precision);
    L.links = a.links;
    L.staples = a.staples;
    L.force = a.force;
    L.mom = a.mom;
    L.partials = a.partials;
    L.action = a.action;
    const KernelScalars sc = make_scalars(a);
    const int64_t nvb = virtual_blocks((int64_t)a.dims[0] * a.dims[1] * a.dims[2] * a.dims[3]);
    if (full_staples(variant)) staple_fields<R, true><<<grid_of(nvb), kBlock, 0, st>>>(L);
    else staple_fields<R, false><<<grid_of(nvb), kBlock, 0, st>>>(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.action != nullptr) {
        e = launch_pass_b<R, true>(L, sc, variant, st);
        if (e != cudaSuccess) return e;
        return launch_finish_sum(a.partials, (int)nvb, a.beta / 3.0, a.action, st);
    }
    return launch_pass_b<R, false>(L, sc, variant, st);
}

template <typename R>
cudaError_t launch_sf_batched_t(const ForceArgs &a, int n, const SfLattice *items,
                                unsigned long long *counter, cudaStream_t st)
{
    const int variant = resolve_variant(a);
    SfBatch B{};
    B.n = n;
    B.counter = counter;
    bool any_action = false;
    int64_t vb = 0;
    for (int c = 0; c < n; ++c) {
        B.e[c] = items[c];
        set_traversal(B.e[c], variant);
        B.e[c].plane_bytes = (int64_t)full_plane_bytes(
            (int64_t)items[c].dims[0] * items[c].dims[1] * items[c].dims[2] * items[c].dims[3],
            a.precision);
        B.e[c].vb_begin = vb;
        vb += virtual_blocks((int64_t)items[c].dims[0] * items[c].dims[1] * items[c].dims[2] *
                             items[c].dims[3]);
        any_action = any_action || items[c].action != nullptr;
    }
    B.total = vb;
    const KernelScalars sc = make_scalars(a);
    cudaError_t e = cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (full_staples(variant)) {
        auto ka = staple_fields_batched<R, true>;
        ka<<<persistent_grid(ka, grid_slot(5, sizeof(R) == 8, false, false), B.total), kBlock, 0, st>>>(B);
    } else {
        auto ka = staple_fields_batched<R, false>;
        ka<<<persistent_grid(ka, grid_slot(4, sizeof(R) == 8, false, false), B.total), kBlock, 0, st>>>(B);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (!any_action) return launch_pass_b_batched<R, false>(B, sc, variant, st);
    e = launch_pass_b_batched<R, true>(B, sc, variant, st);
    if (e != cudaSuccess) return e;
    finish_batched<<<n, 1024, 0, st>>>(B, a.beta / 3.0);
    return cudaGetLastError();
}

} // namespace

// Room for the 24 planes in the larger (full, 18-real, in blocks of 32
// sites) of the two storage forms, so that every schedule fits the same
// workspace.
size_t staple_field_bytes(const int dims[4], int precision)
{
    const int64_t V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
    return round_up256((size_t)kStaplePlanes * full_plane_bytes(V, precision));
}

bool staple_fields_supported(const int dims[4])
{
    return (int64_t)dims[0] * dims[1] * dims[2] * dims[3] < ((int64_t)1 << 31);
}

int staple_force_partials(const int dims[4])
{
    return (int)virtual_blocks((int64_t)dims[0] * dims[1] * dims[2] * dims[3]);
}

cudaError_t launch_force_staple_fields(const ForceArgs &a, cudaStream_t st)
{
    return a.precision == LQCD_F64 ? launch_sf_t<double>(a, st) : launch_sf_t<float>(a, st);
}

cudaError_t launch_force_staple_fields_batched(const ForceArgs &a, int n, const SfLattice *items,
                                               unsigned long long *counter, cudaStream_t st)
{
    if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
    return a.precision == LQCD_F64 ? launch_sf_batched_t<double>(a, n, items, counter, st)
                                   : launch_sf_batched_t<float>(a, n, items, counter, st);
}

int staple_force_variants() { return kSfVariants; }

int staple_force_variant(int precision, const int dims[4])
{
    const int p = precision == LQCD_F64 ? 1 : 0;
    const int v = g_sf_variant[p].load();
    return v < 0 ? default_variant(precision, dims) : v;
}

void set_staple_force_variant(int precision, int variant)
{
    g_sf_variant[precision == LQCD_F64 ? 1 : 0].store(variant);
}

} // namespace lqcd
