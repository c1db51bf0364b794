// Gauge force of the one-loop Symanzik action (paper Sec. II, Eq. 18_7_25_2
// and the force algorithm after Eq. 18_6_6_13) on sm_103a.
//
// For the link (k, rho) the 48 staples are the loop remainders that run from
// k + rho back to k.  With a, b signed directions perpendicular to rho
// (6 choices each) they are, as direction sequences starting at k + rho:
//   plaquette   (b, -rho, -b)                       6
//   rectangle   (rho, b, -rho, -rho, -b)            6   link first on the long side
//               (b, -rho, -rho, -b, rho)            6   link second on the long side
//               (b, b, -rho, -b, -b)                6   long side along b
//   cube        (a, b, -rho, -a, -b),  a != +-b     24
// These are the forward and backward staples of Eq. 18_7_25_2 for every loop
// of Eq. 18_3_27_30 through the link, each occurrence once.  The force is
// f^a = 2 Re tr(i T_a G) with G = (beta/6) (U_{k,rho} t)_TA (Eqs. 18_6_6_11,
// 18_6_6_13), read off the Gell-Mann matrices (ta_components).
//
// Two kernels, one thread per link:
//   force_paths    walks the 48 staples of a per-direction table held in the
//                  kernel parameter (constant) bank: 180 matrix products.
//   force_factored regroups the staples by their shared end links,
//                  t = sum_b X_b A_b^dag + c_rect (sum_b K_b L_b^dag H_b^dag) E
//                  (names at factored_b), 134 matrix products; the two
//                  long-lived accumulators live in shared memory.
#include "kernels.h"
#include "su3.cuh"

namespace lqcd {

namespace {

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

// Epilogue shared by both kernels: f = components of (beta/6)(U t)_TA, then
// store f and/or apply the momentum step p += dt f.
template <typename R>
__device__ __forceinline__ void finish(const ForceArgs &a, const R *__restrict__ links,
                                       const Geom &g, int rho, int64_t n, const Mat<R> &t)
{
    const Mat<R> u = load_link(links, g.V, rho, n);
    const Mat<R> m = mul<N, N>(u, t);
    R f[8];
    ta_components(m, R(a.beta / 6.0), f);
    if (a.force != nullptr) store_algebra(static_cast<R *>(a.force), g.V, rho, n, f);
    if (a.mom != nullptr) {
        R *mom = static_cast<R *>(a.mom);
        R p[8];
        load_algebra(mom, g.V, rho, n, p);
        const R dt = R(a.dt);
#pragma unroll
        for (int i = 0; i < 8; ++i) p[i] = fma(dt, f[i], p[i]);
        store_algebra(mom, g.V, rho, n, p);
    }
}

// ------------------------------------------------------------ path table

template <typename R>
__global__ void __launch_bounds__(128) force_paths(const ForceArgs a, const StapleTable tab)
{
    const Geom g = make_geom(a.dims);
    const R *__restrict__ links = static_cast<const R *>(a.links);
    const int64_t nlinks = 4 * g.V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlinks;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int rho = (int)(i / g.V);
        const int64_t n = i - rho * g.V;
        Coord start = coord_of(g, n);
        step(g, start, rho, 1);
        Mat<R> t;
        set_zero(t);
        for (int s = 0; s < tab.count; ++s) {
            const Staple &st = tab.s[rho][s];
            Coord x = start;
            Mat<R> m = walk(links, g, x, st.d[0]);
            for (int j = 1; j < st.len; ++j) m = mul<N, N>(m, walk(links, g, x, st.d[j]));
            const R c = st.cls == 0 ? R(a.c_plaq) : (st.cls == 1 ? R(a.c_rect) : R(a.c_cube));
            axpy(t, c, m);
        }
        finish<R>(a, links, g, rho, n, t);
    }
}

// --------------------------------------------------------------- factored

// Shared-memory accumulator: element e of the calling thread's matrix at
// base[e * blockDim.x] (conflict-free: consecutive threads, consecutive words).
template <typename R> struct SmemMat {
    R *base;
    __device__ __forceinline__ Mat<R> load() const
    {
        Mat<R> m;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                m.re[i][j] = base[(2 * (3 * i + j)) * blockDim.x];
                m.im[i][j] = base[(2 * (3 * i + j) + 1) * blockDim.x];
            }
        return m;
    }
    __device__ __forceinline__ void store(const Mat<R> &m) const
    {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                base[(2 * (3 * i + j)) * blockDim.x] = m.re[i][j];
                base[(2 * (3 * i + j) + 1) * blockDim.x] = m.im[i][j];
            }
    }
    template <int FA, int FB>
    __device__ __forceinline__ void mul_acc(const Mat<R> &a, const Mat<R> &b) const
    {
        Mat<R> c = load();
        lqcd::mul_acc<FA, FB>(c, a, b);
        store(c);
    }
};

// Wrapped linear offsets from the link's site k = n along rho, along nu
// (the current b direction) and along the two directions perpendicular to
// both (the cube's a directions).
struct Offsets {
    int r_m1, r_p1, r_p2;
    int v_m2, v_m1, v_p1, v_p2;
    int a_m1[2], a_p1[2];
};

template <typename R> struct Links {
    const R *__restrict__ p;
    int64_t V;
    // U_mu at site, daggered when S < 0
    template <int S> __device__ __forceinline__ Mat<R> get(int mu, int64_t site) const
    {
        const Mat<R> m = load_link(p, V, mu, site);
        if constexpr (S > 0) return m;
        else return dagger(m);
    }
};

// One cube staple ending in A_b^dag (A_b^dag itself applied by the caller):
//   x += link(k+rho, a) link(k+rho+a, b) U_rho(k+a+b)^dag link(k+b, a)^dag
template <int SB, int SA, int J, typename R>
__device__ __forceinline__ void cube_term(Mat<R> &x, const Links<R> &L, int64_t n, int rho, int nu,
                                          int nua, const Offsets &o)
{
    const int ob1 = SB > 0 ? o.v_p1 : o.v_m1;       // k + b
    const int olb = SB > 0 ? 0 : o.v_m1;            // link(x, b) lives at x + olb
    const int oa1 = SA > 0 ? o.a_p1[J] : o.a_m1[J]; // k + a
    const int ola = SA > 0 ? 0 : o.a_m1[J];         // link(x, a) lives at x + ola
    Mat<R> t = mul<N, N>(L.template get<SA>(nua, n + o.r_p1 + ola),
                         L.template get<SB>(nu, n + o.r_p1 + oa1 + olb));
    t = mul<N, D>(t, L.template get<1>(rho, n + oa1 + ob1));
    mul_acc<N, D>(x, t, L.template get<SA>(nua, n + ob1 + ola));
}

// (Not inlined: a call boundary keeps the scheduler from hoisting the loads
// of both sign variants at once, which would spill.)
// All staples that end with A_b^dag = link(k, b)^dag, b = SB * nu, plus the
// b-term of the rectangles with the link second on the long side:
//   X_b = c_cube sum_a B_a Y_ab R_ab^dag M_ba^dag          (cubes)
//       + c_rect F G_b R'_b^dag R_b^dag                    (rectangle, link first)
//       + c_plaq K_b + c_rect B_b B2_b R2_b^dag A2_b^dag   (plaquette, rectangle along b)
//   t += X_b A_b^dag;   w += K_b L_b^dag H_b^dag,   K_b = B_b R_b^dag
// with B = link(k+rho, b), R = U_rho(k+b), F = U_rho(k+rho), G = link(k+2rho, b),
// R' = U_rho(k+rho+b), B2 = link(k+rho+b, b), R2 = U_rho(k+2b), A2 = link(k+b, b),
// L = U_rho(k-rho+b), H = link(k-rho, b), A = link(k, b), E = U_rho(k-rho).
template <int SB, typename R>
__device__ __noinline__ void factored_b(const SmemMat<R> &t, const SmemMat<R> &w,
                                           const Links<R> &L, int64_t n, int rho, int nu,
                                           int nua0, int nua1, const Offsets &o, R c_pl, R c_rt,
                                           R c_cb)
{
    const int ob1 = SB > 0 ? o.v_p1 : o.v_m1;
    const int ob2 = SB > 0 ? o.v_p2 : o.v_m2;
    const int olb = SB > 0 ? 0 : o.v_m1;
    const int obb = SB > 0 ? o.v_p1 : o.v_m2; // link(k+b, b) lives at k + obb
    Mat<R> x;
    set_zero(x);
    cube_term<SB, +1, 0>(x, L, n, rho, nu, nua0, o);
    cube_term<SB, -1, 0>(x, L, n, rho, nu, nua0, o);
    cube_term<SB, +1, 1>(x, L, n, rho, nu, nua1, o);
    cube_term<SB, -1, 1>(x, L, n, rho, nu, nua1, o);
    scale(x, c_cb);
    {
        // rectangle with the link first on the long side: F G R'^dag R^dag
        Mat<R> tmp = mul<N, N>(L.template get<1>(rho, n + o.r_p1),
                               L.template get<SB>(nu, n + o.r_p2 + olb));
        tmp = mul<N, D>(tmp, L.template get<1>(rho, n + o.r_p1 + ob1));
        scale(tmp, c_rt);
        mul_acc<N, D>(x, tmp, L.template get<1>(rho, n + ob1));
    }
    {
        // plaquette and the second rectangle class, through K = B R^dag
        const Mat<R> K =
            mul<N, D>(L.template get<SB>(nu, n + o.r_p1 + olb), L.template get<1>(rho, n + ob1));
        axpy(x, c_pl, K);
        const Mat<R> kl = mul<N, D>(K, L.template get<1>(rho, n + o.r_m1 + ob1));
        w.template mul_acc<N, D>(kl, L.template get<SB>(nu, n + o.r_m1 + olb));
    }
    {
        // rectangle along b: B B2 R2^dag A2^dag
        Mat<R> tmp = mul<N, N>(L.template get<SB>(nu, n + o.r_p1 + olb),
                               L.template get<SB>(nu, n + o.r_p1 + obb));
        tmp = mul<N, D>(tmp, L.template get<1>(rho, n + ob2));
        scale(tmp, c_rt);
        mul_acc<N, D>(x, tmp, L.template get<SB>(nu, n + obb));
    }
    t.template mul_acc<N, D>(x, L.template get<SB>(nu, n + olb));
}

template <typename R>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 3 : 2) force_factored(const ForceArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    R *smem = reinterpret_cast<R *>(smem_raw);
    const SmemMat<R> t{smem + threadIdx.x};
    const SmemMat<R> w{smem + 18 * blockDim.x + threadIdx.x};
    const Geom g = make_geom(a.dims);
    const Links<R> L{static_cast<const R *>(a.links), g.V};
    const R c_pl = R(a.c_plaq), c_rt = R(a.c_rect), c_cb = R(a.c_cube);
    const int64_t nlinks = 4 * g.V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlinks;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int rho = (int)(i / g.V);
        const int64_t n = i - rho * g.V;
        const Coord k = coord_of(g, n);
        Offsets o;
        o.r_m1 = (int)disp(g, k, rho, -1);
        o.r_p1 = (int)disp(g, k, rho, 1);
        o.r_p2 = (int)disp(g, k, rho, 2);
        Mat<R> z;
        set_zero(z);
        t.store(z);
        w.store(z);
#pragma unroll 1
        for (int j = 1; j < 4; ++j) {
            const int nu = (rho + j) & 3;
            // the two directions perpendicular to both rho and nu
            const int nua0 = (rho + (j == 1 ? 2 : 1)) & 3;
            const int nua1 = (rho + (j == 3 ? 2 : 3)) & 3;
            o.v_m2 = (int)disp(g, k, nu, -2);
            o.v_m1 = (int)disp(g, k, nu, -1);
            o.v_p1 = (int)disp(g, k, nu, 1);
            o.v_p2 = (int)disp(g, k, nu, 2);
            o.a_m1[0] = (int)disp(g, k, nua0, -1);
            o.a_p1[0] = (int)disp(g, k, nua0, 1);
            o.a_m1[1] = (int)disp(g, k, nua1, -1);
            o.a_p1[1] = (int)disp(g, k, nua1, 1);
            factored_b<+1>(t, w, L, n, rho, nu, nua0, nua1, o, c_pl, c_rt, c_cb);
            factored_b<-1>(t, w, L, n, rho, nu, nua0, nua1, o, c_pl, c_rt, c_cb);
        }
        // t += c_rect w E,  E = U_rho(k - rho)
        Mat<R> ww = w.load();
        scale(ww, c_rt);
        Mat<R> tt = t.load();
        mul_acc<N, N>(tt, ww, L.template get<1>(rho, n + o.r_m1));
        finish<R>(a, L.p, g, rho, n, tt);
    }
}

} // namespace

// ---------------------------------------------------------------- launch

template <typename R> static cudaError_t launch_force_t(const ForceArgs &a, cudaStream_t st)
{
    const int64_t V = (int64_t)a.dims[0] * a.dims[1] * a.dims[2] * a.dims[3];
    const int64_t nlinks = 4 * V;
    const int block = 128;
    int64_t grid = (nlinks + block - 1) / block;
    if (grid > (int64_t)1 << 30) grid = (int64_t)1 << 30;
    if (a.algo == LQCD_FORCE_PATHS) {
        force_paths<R><<<(unsigned)grid, block, 0, st>>>(a, staple_table());
    } else {
        const size_t smem = 2 * 18 * block * sizeof(R);
        force_factored<R><<<(unsigned)grid, block, smem, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_force(const ForceArgs &a, cudaStream_t st)
{
    return a.precision == LQCD_F64 ? launch_force_t<double>(a, st) : launch_force_t<float>(a, st);
}

// The per-direction staple table of the path kernel, built once on the host
// from the staple shapes listed at the top of this file.
const StapleTable &staple_table()
{
    static const StapleTable tab = [] {
        StapleTable t{};
        for (int rho = 0; rho < 4; ++rho) {
            const int r = rho + 1;
            int n = 0;
            auto put = [&](int cls, std::initializer_list<int> d) {
                Staple &s = t.s[rho][n++];
                s.cls = (int8_t)cls;
                s.len = (int8_t)d.size();
                int j = 0;
                for (int v : d) s.d[j++] = (int8_t)v;
            };
            for (int nu = 0; nu < 4; ++nu) {
                if (nu == rho) continue;
                for (int sb = 1; sb >= -1; sb -= 2) {
                    const int b = sb * (nu + 1);
                    put(0, {b, -r, -b});
                    put(1, {r, b, -r, -r, -b});
                    put(1, {b, -r, -r, -b, r});
                    put(1, {b, b, -r, -b, -b});
                    for (int nua = 0; nua < 4; ++nua) {
                        if (nua == rho || nua == nu) continue;
                        for (int sa = 1; sa >= -1; sa -= 2) {
                            const int aa = sa * (nua + 1);
                            put(2, {aa, b, -r, -aa, -b});
                        }
                    }
                }
            }
            t.count = n;
        }
        return t;
    }();
    return tab;
}

} // namespace lqcd
