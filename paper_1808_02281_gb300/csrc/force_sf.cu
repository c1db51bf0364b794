// Gauge force of the one-loop Symanzik action from plaquette-staple fields
// (paper Sec. II, Eq. 18_7_25_2; loops of Eq. 18_3_27_30), two kernels.
//
// Pass A (staple_fields) stores, for every link (x, mu) and every signed
// direction b perpendicular to mu, the plaquette staple
//     S^{(mu)}_b(x) = link(x+mu, b) U_mu(x+b)^dag link(x, b)^dag
// (the path x+mu -> x+mu+b -> x+b -> x).  It is a product of three SU(3)
// matrices, so it is SU(3) and is stored in the compact two-row form, like a
// link: 24 "directions" per site instead of 4.
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
// pass A, against 180 for the 48 staples walked one by one.
//
// The action comes out of pass B at no extra products: summing
// Re tr(U_{k,rho} t_{k,rho}) over links counts every loop once per link on it
// (L = 4 or 6 times) with its c_P, so with the plaquette staple sum Pl,
//   S_G = (beta/3) sum_links [ 3 (1.5 c_plaq + 3 c_rect + 4 c_cube)
//                              - Re tr(U t)/6 - (c_plaq/12) Re tr(U Pl) ]
// (Eq. 18_6_4_1), each link's term formed in FP64 from its two traces.
#include <atomic>
#include <mutex>

#include "kernels.h"
#include "su3.cuh"

namespace lqcd {

namespace {

constexpr int kBlockA = 128; // four warps: the four directions of 32 sites
constexpr int kBlockB = 128; // four warps: the four directions of 32 sites

__host__ __device__ __forceinline__ int64_t padded_sites(int64_t V) { return (V + 31) & ~(int64_t)31; }

// ---------------------------------------------------------------- pass A

template <typename R>
__global__ void __launch_bounds__(kBlockA) staple_fields(const R *__restrict__ links,
                                                         R *__restrict__ sf, Geom g)
{
    // four warps per block: the four directions of 32 consecutive sites, so
    // the links around a site are read once from DRAM (a direction-major
    // order re-reads the neighbouring directions once per direction)
    const int64_t nthreads = 4 * padded_sites(g.V);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nthreads;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int mu = (int)((i >> 5) & 3);
        const int64_t x = ((i >> 7) << 5) | (i & 31);
        if (x >= g.V) continue;
        const Coord c = coord_of(g, x);
        const int64_t xm = x + disp(g, c, mu, 1); // x + mu
#pragma unroll 1
        for (int iv = 0; iv < 3; ++iv) {
            const int nu = (mu + 1 + iv) & 3;
            const int64_t vp = disp(g, c, nu, 1), vm = disp(g, c, nu, -1);
            // b = +nu:  U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
            Mat<R> t = mul<N, D>(load_link(links, g.V, nu, xm), load_link(links, g.V, mu, x + vp));
            store_link(sf, g.V, mu * 6 + 2 * iv, x, mul_top2<N, D>(t, load_link(links, g.V, nu, x)));
            // b = -nu:  U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
            t = mul<D, D>(load_link(links, g.V, nu, xm + vm), load_link(links, g.V, mu, x + vm));
            store_link(sf, g.V, mu * 6 + 2 * iv + 1, x,
                       mul_top2<N, N>(t, load_link(links, g.V, nu, x + vm)));
        }
    }
}

// ---------------------------------------------------------------- pass B

enum { SC_BETA6 = 0, SC_CPL, SC_CRT, SC_CCB, SC_ACT, SC_ACTPL, SC_DT };

template <typename R> __device__ __forceinline__ R scalar(const ForceArgs &a, int i)
{
    if constexpr (sizeof(R) == 4) return a.sc.f[i];
    else return a.sc.d[i];
}

// Traversal order of pass B: the lattice is cut into spatial blocks of
// bx x by x bz sites that run over all t; blocks one after the other, inside
// a block t-slice by t-slice, inside a slice micro-tiles of mx x my x mz
// sites (x fastest within and between micro-tiles), and the four links of a
// site next to each other.  The staple planes of three neighbouring t-slices
// of one block then stay in L2 while the block is swept, and a micro-tile
// makes the y and z neighbours of most sites in a thread block L1 hits.
struct Sweep {
    int bx, by, bz, mx, my, mz;
    int nbx, nby, nmx, nmy, mvol;
    int64_t slice, vol; // sites per block slice and per block
};

__device__ __forceinline__ Sweep make_sweep(const ForceArgs &a, const Geom &g)
{
    Sweep s;
    s.bx = a.sweep[0];
    s.by = a.sweep[1];
    s.bz = a.sweep[2];
    s.mx = a.micro[0];
    s.my = a.micro[1];
    s.mz = a.micro[2];
    s.nbx = g.L0 / s.bx;
    s.nby = g.L1 / s.by;
    s.nmx = s.bx / s.mx;
    s.nmy = s.by / s.my;
    s.mvol = s.mx * s.my * s.mz;
    s.slice = (int64_t)s.bx * s.by * s.bz;
    s.vol = s.slice * g.L3;
    return s;
}

__device__ __forceinline__ Coord swept_site(const Sweep &s, int64_t j)
{
    const int64_t blk = j / s.vol;
    const int64_t r = j - blk * s.vol;
    Coord c;
    c.c3 = (int)(r / s.slice);
    const int r2 = (int)(r - c.c3 * s.slice);
    const int mt = r2 / s.mvol, w = r2 - mt * s.mvol;
    const int xin = w % s.mx, yin = (w / s.mx) % s.my, zin = w / (s.mx * s.my);
    const int mxi = mt % s.nmx, myi = (mt / s.nmx) % s.nmy, mzi = mt / (s.nmx * s.nmy);
    const int bxi = (int)(blk % s.nbx);
    const int64_t q = blk / s.nbx;
    const int byi = (int)(q % s.nby);
    const int bzi = (int)(q / s.nby);
    c.c0 = bxi * s.bx + mxi * s.mx + xin;
    c.c1 = byi * s.by + myi * s.my + yin;
    c.c2 = bzi * s.bz + mzi * s.mz + zin;
    return c;
}

__device__ __forceinline__ double block_sum_b(double v)
{
    __shared__ double part[kBlockB / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) part[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (warp == 0) {
        s = lane < kBlockB / 32 ? part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

// The staples that start with link(k+rho, d), d = +-nu_d (NEG: minus):
//   t += B_d [ c_cube sum_{b perp rho, d} S_b(k+d) S^{(d)}_b(k) + c_rect S_d(k+d) A_d^dag ]
template <bool NEG, bool UNROLLQ, typename R>
__device__ __forceinline__ void d_terms(Mat<R> &t, const R *__restrict__ links,
                                        const R *__restrict__ sf, const Geom &g, const Coord &c,
                                        int rho, int64_t k, int64_t kp, int id, R c_rt, R c_cb)
{
    constexpr int FD = NEG ? D : N;
    const int base = rho * 6;
    const int jd = 2 * id + (NEG ? 1 : 0);
    const int nud = (rho + 1 + id) & 3;
    const int64_t kd = k + disp(g, c, nud, NEG ? -1 : 1); // k + d
    // S^{(d)}_b(k): plane nud*6 + j' at k, or (NEG) its dagger at k - nud = kd
    const int64_t site2 = NEG ? kd : k;
    Mat<R> y;
    set_zero(y);
    // the four signed b perpendicular to rho and d: two directions, two signs
#pragma unroll(UNROLLQ ? 2 : 1)
    for (int q = 0; q < 2; ++q) {
        const int ib = q == 0 ? (id == 0 ? 1 : 0) : (id == 2 ? 1 : 2);
        const int nub = (rho + 1 + ib) & 3;
        const int jp = 2 * ((nub - nud - 1) & 3);
        mul_acc<N, FD>(y, load_link(sf, g.V, base + 2 * ib, kd), load_link(sf, g.V, nud * 6 + jp, site2));
        mul_acc<N, FD>(y, load_link(sf, g.V, base + 2 * ib + 1, kd),
                       load_link(sf, g.V, nud * 6 + jp + 1, site2));
    }
    scale(y, c_cb);
    Mat<R> r3 = load_link(sf, g.V, base + jd, kd);
    scale(r3, c_rt);
    if constexpr (!NEG) {
        mul_acc<N, D>(y, r3, load_link(links, g.V, nud, k));  // A_d = U_nud(k)
        mul_acc<N, N>(t, load_link(links, g.V, nud, kp), y);  // B_d = U_nud(k+rho)
    } else {
        mul_acc<N, N>(y, r3, load_link(links, g.V, nud, kd)); // A_d = U_nud(k-nud)^dag
        mul_acc<D, N>(t, load_link(links, g.V, nud, kp + (kd - k)), y); // B_d = U_nud(k+rho-nud)^dag
    }
}

template <typename R, bool ACTION, bool UNROLLQ>
__global__ void __launch_bounds__(kBlockB, sizeof(R) == 4 ? (ACTION ? 3 : 4) : 2)
    force_from_staples(const ForceArgs a)
{
    const Geom g = make_geom(a.dims);
    const R *__restrict__ links = static_cast<const R *>(a.links);
    const R *__restrict__ sf = static_cast<const R *>(a.staples);
    const R c_pl = scalar<R>(a, SC_CPL), c_rt = scalar<R>(a, SC_CRT), c_cb = scalar<R>(a, SC_CCB);
    const R act_const = scalar<R>(a, SC_ACT), act_cpl = scalar<R>(a, SC_ACTPL);
    const Sweep sw = make_sweep(a, g);
    // sites padded to whole warps: thread i takes site ((i >> 7) << 5) | (i & 31)
    // and direction (i >> 5) & 3; padding sites are skipped
    const int64_t nthreads = 4 * padded_sites(g.V);
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nthreads;
         i += (int64_t)gridDim.x * blockDim.x) {
        if ((((i >> 7) << 5) | (i & 31)) >= g.V) continue;
        // the four warps of a thread block take the four directions of the
        // same 32 sites: the staple planes around a site are read while they
        // are in L1/L2 (a direction-major order re-reads them from DRAM once
        // per direction), and each warp reads one plane per instruction, so a
        // quarter-warp covers 8 consecutive sites of one 128-byte line
        const int rho = (int)((i >> 5) & 3);
        const Coord c = swept_site(sw, ((i >> 7) << 5) | (i & 31));
        const int64_t k = index_of(g, c);
        const int64_t kp = k + disp(g, c, rho, 1), km = k + disp(g, c, rho, -1);
        const int base = rho * 6;

        // plaquettes and the two rectangle chains along rho
        Mat<R> t;
        R tr_pl = R(0);
        {
            Mat<R> pl, p1, p2;
            set_zero(pl);
            set_zero(p1);
            set_zero(p2);
#pragma unroll 1
            for (int j = 0; j < 6; ++j) {
                const Mat<R> s = load_link(sf, g.V, base + j, k);
                add_to(pl, s);
                mul_acc<N, N>(p1, load_link(sf, g.V, base + j, kp), s);
                mul_acc<N, N>(p2, s, load_link(sf, g.V, base + j, km));
            }
            if constexpr (ACTION) tr_pl = re_trace_mul<N, N>(load_link(links, g.V, rho, k), pl);
            t = pl;
            scale(t, c_pl);
            scale(p1, c_rt);
            mul_acc<N, N>(t, load_link(links, g.V, rho, kp), p1);
            scale(p2, c_rt);
            mul_acc<N, N>(t, p2, load_link(links, g.V, rho, km));
        }

        // everything that starts with link(k+rho, d): cubes and the rectangle
        // along d; positive and negative d in two loops, each with one small
        // body (the orientation of the shared links is fixed at compile time)
#pragma unroll 1
        for (int id = 0; id < 3; ++id)
            d_terms<false, UNROLLQ>(t, links, sf, g, c, rho, k, kp, id, c_rt, c_cb);
#pragma unroll 1
        for (int id = 0; id < 3; ++id)
            d_terms<true, UNROLLQ>(t, links, sf, g, c, rho, k, kp, id, c_rt, c_cb);

        const Mat<R> u = load_link(links, g.V, rho, k);
        const Mat<R> m = mul<N, N>(u, t);
        R f[8];
        ta_components(m, scalar<R>(a, SC_BETA6), f);
        if (a.force != nullptr) store_algebra(static_cast<R *>(a.force), g.V, rho, k, f);
        if (a.mom != nullptr) {
            R *mom = static_cast<R *>(a.mom);
            R p[8];
            load_algebra(mom, g.V, rho, k, p);
            const R dt = scalar<R>(a, SC_DT);
#pragma unroll
            for (int q = 0; q < 8; ++q) p[q] = fma(dt, f[q], p[q]);
            store_algebra(mom, g.V, rho, k, p);
        }
        if constexpr (ACTION) {
            // this link's share of the action, formed in the working precision
            // (its rounding is that of the traces themselves) and summed in FP64
            const R tr_t = m.re[0][0] + m.re[1][1] + m.re[2][2];
            acc += (double)(act_const - tr_t * R(1.0 / 6.0) - act_cpl * tr_pl);
        }
    }
    if constexpr (ACTION) {
        const double s = block_sum_b(acc);
        if (threadIdx.x == 0) a.partials[blockIdx.x] = s;
    }
}

// ------------------------------------------------------ pass B, pipelined
//
// The same arithmetic as force_from_staples, with every operand streamed into
// shared memory by cp.async before it is needed.  Pass B has no reuse that a
// block could stage (the staples of one site fill 1152 B, so a halo'd tile
// does not fit), and its loads are scattered gathers that each thread issues
// for itself; the limiter is their latency.  Each thread therefore walks its
// 88 operands in 26 groups of at most 4 matrices and keeps NST groups in
// flight in a ring of shared-memory slots that only it reads: group g + NST-1
// is requested before group g is used.  Within a thread the ring needs no
// barrier: cp.async.wait_group orders the copies before the reads, and a slot
// is refilled only after the instructions that used its previous contents
// have issued.

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int NPEND> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory");
}

constexpr int kGroups = 26;

// Shared-memory ring of one thread: lane q of matrix m in stage st at
// base[((st * 4 + m) * LQ + q) * blockDim.x].
template <typename R> struct Ring {
    using V4 = typename Vec<R>::type;
    static constexpr int LQ = 12 / Vec<R>::W;
    V4 *base;

    __device__ __forceinline__ V4 *slot(int st, int m) const
    {
        return base + ((st * 4 + m) * LQ) * blockDim.x;
    }
    // request matrix `plane` (link or staple plane) at `site` into (st, m)
    __device__ __forceinline__ void fetch(int st, int m, const R *arr, int64_t V, int plane,
                                          int64_t site) const
    {
        const V4 *src = reinterpret_cast<const V4 *>(arr) + (int64_t)plane * LQ * V + site;
        V4 *dst = slot(st, m);
#pragma unroll
        for (int q = 0; q < LQ; ++q) cp_async16(dst + q * blockDim.x, src + q * V);
    }
    __device__ __forceinline__ Mat<R> read(int st, int m) const
    {
        const V4 *src = slot(st, m);
        R r[12];
#pragma unroll
        for (int q = 0; q < LQ; ++q) {
            const V4 v = src[q * blockDim.x];
            if constexpr (Vec<R>::W == 4) {
                r[4 * q + 0] = v.x;
                r[4 * q + 1] = v.y;
                r[4 * q + 2] = v.z;
                r[4 * q + 3] = v.w;
            } else {
                r[2 * q + 0] = v.x;
                r[2 * q + 1] = v.y;
            }
        }
        Mat<R> u;
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                u.re[i][j] = r[6 * i + 2 * j];
                u.im[i][j] = r[6 * i + 2 * j + 1];
            }
        rebuild_row2(u);
        return u;
    }
};

struct LinkSite {
    int rho;
    int64_t k, kp, km;
    Coord c;
};

// Request the operands of group g of link L into stage st (g past the end:
// an empty group, so that the group count stays uniform).
//   g 0..5   S_j(k), S_j(k+rho), S_j(k-rho)               (plaquettes, rectangle chains)
//   g 6      U_rho(k), U_rho(k+rho), U_rho(k-rho)
//   g 7..24  per d = 0..5: two cube groups (S^{(rho)}_b(k+d), S^{(d)}_b(k) for the two
//            signs of one b direction), then S_d(k+d), link(k, d), link(k+rho, d)
//   g 25     U_rho(k)
template <typename R>
__device__ __forceinline__ void issue_group(const Ring<R> &ring, int st, int g, const R *links,
                                            const R *sf, const Geom &gm, const LinkSite &L)
{
    if (g < kGroups) {
        const int64_t V = gm.V;
        const int base = L.rho * 6;
        if (g < 6) {
            ring.fetch(st, 0, sf, V, base + g, L.k);
            ring.fetch(st, 1, sf, V, base + g, L.kp);
            ring.fetch(st, 2, sf, V, base + g, L.km);
        } else if (g == 6) {
            ring.fetch(st, 0, links, V, L.rho, L.k);
            ring.fetch(st, 1, links, V, L.rho, L.kp);
            ring.fetch(st, 2, links, V, L.rho, L.km);
        } else if (g < 25) {
            const int h = g - 7;
            const int jd = h / 3, r = h - 3 * (h / 3);
            const int id = jd >> 1;
            const int nud = (L.rho + 1 + id) & 3;
            const bool neg = jd & 1;
            const int64_t kd = L.k + disp(gm, L.c, nud, neg ? -1 : 1);
            if (r < 2) {
                const int ib = r == 0 ? (id == 0 ? 1 : 0) : (id == 2 ? 1 : 2);
                const int nub = (L.rho + 1 + ib) & 3;
                const int jp = 2 * ((nub - nud - 1) & 3);
                const int64_t site2 = neg ? kd : L.k;
                ring.fetch(st, 0, sf, V, base + 2 * ib, kd);
                ring.fetch(st, 1, sf, V, nud * 6 + jp, site2);
                ring.fetch(st, 2, sf, V, base + 2 * ib + 1, kd);
                ring.fetch(st, 3, sf, V, nud * 6 + jp + 1, site2);
            } else {
                ring.fetch(st, 0, sf, V, base + jd, kd);
                ring.fetch(st, 1, links, V, nud, neg ? kd : L.k);
                ring.fetch(st, 2, links, V, nud, L.kp + (neg ? kd - L.k : 0));
            }
        } else {
            ring.fetch(st, 0, links, V, L.rho, L.k);
        }
    }
    cp_async_commit();
}

template <typename R, bool ACTION, int NST>
__global__ void __launch_bounds__(kBlockB, sizeof(R) == 4 ? 3 : 2)
    force_from_staples_async(const ForceArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Ring<R> ring{reinterpret_cast<typename Vec<R>::type *>(smem_raw) + threadIdx.x};
    const Geom g = make_geom(a.dims);
    const R *__restrict__ links = static_cast<const R *>(a.links);
    const R *__restrict__ sf = static_cast<const R *>(a.staples);
    const R c_pl = scalar<R>(a, SC_CPL), c_rt = scalar<R>(a, SC_CRT), c_cb = scalar<R>(a, SC_CCB);
    const R act_const = scalar<R>(a, SC_ACT), act_cpl = scalar<R>(a, SC_ACTPL);
    const Sweep sw = make_sweep(a, g);
    // sites padded to whole warps: thread i takes site ((i >> 7) << 5) | (i & 31)
    // and direction (i >> 5) & 3; padding sites are skipped
    const int64_t nthreads = 4 * padded_sites(g.V);
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nthreads;
         i += (int64_t)gridDim.x * blockDim.x) {
        if ((((i >> 7) << 5) | (i & 31)) >= g.V) continue;
        LinkSite L;
        L.rho = (int)((i >> 5) & 3);
        L.c = swept_site(sw, ((i >> 7) << 5) | (i & 31));
        L.k = index_of(g, L.c);
        L.kp = L.k + disp(g, L.c, L.rho, 1);
        L.km = L.k + disp(g, L.c, L.rho, -1);

        // prologue: NST - 1 groups in flight
#pragma unroll
        for (int q = 0; q < NST - 1; ++q) issue_group(ring, q, q, links, sf, g, L);
        int gi = 0;      // group being consumed
        int st = 0;      // its stage
        int st_next = NST - 1;
        auto advance = [&]() {
            issue_group(ring, st_next, gi + NST - 1, links, sf, g, L);
            st_next = st_next + 1 == NST ? 0 : st_next + 1;
            cp_async_wait<NST - 1>();
        };
        auto next = [&]() {
            ++gi;
            st = st + 1 == NST ? 0 : st + 1;
        };

        Mat<R> t;
        R tr_pl = R(0);
        {
            Mat<R> pl, p1, p2;
            set_zero(pl);
            set_zero(p1);
            set_zero(p2);
#pragma unroll 1
            for (int j = 0; j < 6; ++j) {
                advance();
                const Mat<R> s0 = ring.read(st, 0);
                add_to(pl, s0);
                mul_acc<N, N>(p1, ring.read(st, 1), s0);
                mul_acc<N, N>(p2, s0, ring.read(st, 2));
                next();
            }
            advance();
            if constexpr (ACTION) tr_pl = re_trace_mul<N, N>(ring.read(st, 0), pl);
            t = pl;
            scale(t, c_pl);
            scale(p1, c_rt);
            mul_acc<N, N>(t, ring.read(st, 1), p1);
            scale(p2, c_rt);
            mul_acc<N, N>(t, p2, ring.read(st, 2));
            next();
        }
#pragma unroll 1
        for (int jd = 0; jd < 6; ++jd) {
            const bool neg = jd & 1;
            Mat<R> y;
            set_zero(y);
#pragma unroll 1
            for (int r = 0; r < 2; ++r) {
                advance();
                if (!neg) {
                    mul_acc<N, N>(y, ring.read(st, 0), ring.read(st, 1));
                    mul_acc<N, N>(y, ring.read(st, 2), ring.read(st, 3));
                } else {
                    mul_acc<N, D>(y, ring.read(st, 0), ring.read(st, 1));
                    mul_acc<N, D>(y, ring.read(st, 2), ring.read(st, 3));
                }
                next();
            }
            advance();
            scale(y, c_cb);
            Mat<R> r3 = ring.read(st, 0);
            scale(r3, c_rt);
            if (!neg) {
                mul_acc<N, D>(y, r3, ring.read(st, 1));
                mul_acc<N, N>(t, ring.read(st, 2), y);
            } else {
                mul_acc<N, N>(y, r3, ring.read(st, 1));
                mul_acc<D, N>(t, ring.read(st, 2), y);
            }
            next();
        }
        advance();
        const Mat<R> m = mul<N, N>(ring.read(st, 0), t);
        next();

        R f[8];
        ta_components(m, scalar<R>(a, SC_BETA6), f);
        if (a.force != nullptr) store_algebra(static_cast<R *>(a.force), g.V, L.rho, L.k, f);
        if (a.mom != nullptr) {
            R *mom = static_cast<R *>(a.mom);
            R p[8];
            load_algebra(mom, g.V, L.rho, L.k, p);
            const R dt = scalar<R>(a, SC_DT);
#pragma unroll
            for (int q = 0; q < 8; ++q) p[q] = fma(dt, f[q], p[q]);
            store_algebra(mom, g.V, L.rho, L.k, p);
        }
        if constexpr (ACTION) {
            // this link's share of the action, formed in the working precision
            // (its rounding is that of the traces themselves) and summed in FP64
            const R tr_t = m.re[0][0] + m.re[1][1] + m.re[2][2];
            acc += (double)(act_const - tr_t * R(1.0 / 6.0) - act_cpl * tr_pl);
        }
    }
    if constexpr (ACTION) {
        const double s = block_sum_b(acc);
        if (threadIdx.x == 0) a.partials[blockIdx.x] = s;
    }
}

unsigned grid_of(int64_t items, int block)
{
    int64_t g = (items + block - 1) / block;
    if (g < 1) g = 1;
    if (g > ((int64_t)1 << 30)) g = (int64_t)1 << 30;
    return (unsigned)g;
}

} // namespace

size_t staple_field_bytes(const int dims[4], int precision)
{
    const int64_t V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
    const size_t real = precision == LQCD_F64 ? 8 : 4;
    return ((size_t)(24 * 12) * (size_t)V * real + 255) & ~(size_t)255;
}

int staple_force_partials(const int dims[4])
{
    const int64_t V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
    return (int)grid_of(4 * padded_sites(V), kBlockB);
}

// Dynamic shared memory of the pipelined pass B, and its once-per-device
// opt-in above the 48 KB default.
template <typename R, int NST> constexpr size_t async_smem_bytes()
{
    return (size_t)NST * 4 * (12 / Vec<R>::W) * kBlockB * 16;
}

template <typename R, bool ACTION, int NST>
static cudaError_t launch_async(const ForceArgs &a, unsigned grid, cudaStream_t st)
{
    constexpr size_t smem = async_smem_bytes<R, NST>();
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!done[dev]) {
            e = cudaFuncSetAttribute(force_from_staples_async<R, ACTION, NST>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            done[dev] = true;
        }
    }
    force_from_staples_async<R, ACTION, NST><<<grid, kBlockB, smem, st>>>(a);
    return cudaGetLastError();
}

// Largest divisor of L not above cap.
static int block_extent(int L, int cap)
{
    for (int b = cap < L ? cap : L; b > 1; --b)
        if (L % b == 0) return b;
    return 1;
}

// Pass-B variants (same arithmetic, different schedules):
//   0  micro-tiles 8x2x2, inner b loop rolled
//   1  micro-tiles 8x2x2, inner b loop unrolled
//   2  x rows (no micro-tiles), inner b loop rolled
//   3  micro-tiles 8x2x2, operands streamed through a cp.async ring
// The process-wide choice per precision is set by lqcd_set_force_variant or
// lqcd_autotune_force; -1 means the default.
constexpr int kSfVariants = 4;
constexpr int kSfDefault = 0;
static std::atomic<int> g_sf_variant[2] = {{-1}, {-1}};

template <typename R, bool ACTION>
static cudaError_t launch_pass_b(const ForceArgs &a, unsigned grid, cudaStream_t st)
{
    constexpr int NST = sizeof(R) == 4 ? 3 : 2;
    switch (a.variant) {
    case 1: force_from_staples<R, ACTION, true><<<grid, kBlockB, 0, st>>>(a); break;
    case 3: return launch_async<R, ACTION, NST>(a, grid, st);
    default: force_from_staples<R, ACTION, false><<<grid, kBlockB, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

template <typename R> static cudaError_t launch_sf_t(const ForceArgs &args, cudaStream_t st)
{
    ForceArgs a = args;
    const double sc[7] = {a.beta / 6.0, a.c_plaq, a.c_rect, a.c_cube,
                          3.0 * (1.5 * a.c_plaq + 3.0 * a.c_rect + 4.0 * a.c_cube), a.c_plaq / 12.0,
                          a.dt};
    for (int i = 0; i < 7; ++i) {
        a.sc.d[i] = sc[i];
        a.sc.f[i] = (float)sc[i];
    }
    a.sweep[0] = block_extent(a.dims[0], 64);
    a.sweep[1] = block_extent(a.dims[1], 16);
    a.sweep[2] = block_extent(a.dims[2], 16);
    if (a.variant == 2) {
        a.micro[0] = a.sweep[0];
        a.micro[1] = a.micro[2] = 1;
    } else {
        a.micro[0] = block_extent(a.sweep[0], 8);
        a.micro[1] = a.sweep[1] % 2 == 0 ? 2 : 1;
        a.micro[2] = a.sweep[2] % 2 == 0 ? 2 : 1;
    }
    const Geom g = make_geom(a.dims);
    staple_fields<R><<<grid_of(4 * padded_sites(g.V), kBlockA), kBlockA, 0, st>>>(
        static_cast<const R *>(a.links), static_cast<R *>(a.staples), g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned grid = grid_of(4 * padded_sites(g.V), kBlockB);
    if (a.action != nullptr) {
        e = launch_pass_b<R, true>(a, grid, st);
        if (e != cudaSuccess) return e;
        return launch_finish_sum(a.partials, (int)grid, a.beta / 3.0, a.action, st);
    }
    return launch_pass_b<R, false>(a, grid, st);
}

int staple_force_variants() { return kSfVariants; }

int staple_force_variant(int precision)
{
    const int v = g_sf_variant[precision == LQCD_F64 ? 1 : 0].load();
    return v < 0 ? kSfDefault : v;
}

void set_staple_force_variant(int precision, int variant)
{
    g_sf_variant[precision == LQCD_F64 ? 1 : 0].store(variant);
}

cudaError_t launch_force_staple_fields(const ForceArgs &args, cudaStream_t st)
{
    ForceArgs a = args;
    if (a.variant < 0 || a.variant >= kSfVariants) a.variant = staple_force_variant(a.precision);
    return a.precision == LQCD_F64 ? launch_sf_t<double>(a, st) : launch_sf_t<float>(a, st);
}

} // namespace lqcd
