// SU(3) / su(3) device algebra and the compact structure-of-arrays layout of
// links and algebra fields.  Shared by every kernel of liblqcd (never by the
// CPU oracle).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.h"

namespace lqcd {

// ---------------------------------------------------------------- types

template <typename R> struct Vec;  // 16-byte lane type of the SoA layout
template <> struct Vec<float> {
    using type = float4;
    static constexpr int W = 4;
};
template <> struct Vec<double> {
    using type = double2;
    static constexpr int W = 2;
};

// 3x3 complex matrix held in registers (split real / imaginary parts so that
// every product is plain FMA chains).
template <typename R> struct Mat {
    R re[3][3];
    R im[3][3];
};

template <typename R> __device__ __forceinline__ void set_zero(Mat<R> &m)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) m.re[i][j] = m.im[i][j] = R(0);
}

template <typename R> __device__ __forceinline__ void set_unit(Mat<R> &m)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            m.re[i][j] = (i == j) ? R(1) : R(0);
            m.im[i][j] = R(0);
        }
}

template <typename R> __device__ __forceinline__ Mat<R> dagger(const Mat<R> &a)
{
    Mat<R> r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            r.re[i][j] = a.re[j][i];
            r.im[i][j] = -a.im[j][i];
        }
    return r;
}

// Operand forms of a product: N = as is, D = daggered.
enum Form { N = 0, D = 1 };

// Element (i, j) of op(a), op = identity or dagger, as (re, im).
template <int F, typename R>
__device__ __forceinline__ R el_re(const Mat<R> &a, int i, int j)
{
    return F == N ? a.re[i][j] : a.re[j][i];
}
template <int F, typename R>
__device__ __forceinline__ R el_im(const Mat<R> &a, int i, int j)
{
    return F == N ? a.im[i][j] : -a.im[j][i];
}

// c = op_a(a) * op_b(b)
template <int FA, int FB, typename R>
__device__ __forceinline__ Mat<R> mul(const Mat<R> &a, const Mat<R> &b)
{
    Mat<R> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            R re = el_re<FA>(a, i, 0) * el_re<FB>(b, 0, j);
            R im = el_re<FA>(a, i, 0) * el_im<FB>(b, 0, j);
            re = fma(-el_im<FA>(a, i, 0), el_im<FB>(b, 0, j), re);
            im = fma(el_im<FA>(a, i, 0), el_re<FB>(b, 0, j), im);
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                re = fma(el_re<FA>(a, i, k), el_re<FB>(b, k, j), re);
                re = fma(-el_im<FA>(a, i, k), el_im<FB>(b, k, j), re);
                im = fma(el_re<FA>(a, i, k), el_im<FB>(b, k, j), im);
                im = fma(el_im<FA>(a, i, k), el_re<FB>(b, k, j), im);
            }
            c.re[i][j] = re;
            c.im[i][j] = im;
        }
    return c;
}

// Rows 0 and 1 of op_a(a) * op_b(b) (row 2 left zero): enough for a product
// that is stored in the compact two-row form.
template <int FA, int FB, typename R>
__device__ __forceinline__ Mat<R> mul_top2(const Mat<R> &a, const Mat<R> &b)
{
    Mat<R> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (i == 2) {
                c.re[i][j] = c.im[i][j] = R(0);
                continue;
            }
            R re = R(0), im = R(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                re = fma(el_re<FA>(a, i, k), el_re<FB>(b, k, j), re);
                re = fma(-el_im<FA>(a, i, k), el_im<FB>(b, k, j), re);
                im = fma(el_re<FA>(a, i, k), el_im<FB>(b, k, j), im);
                im = fma(el_im<FA>(a, i, k), el_re<FB>(b, k, j), im);
            }
            c.re[i][j] = re;
            c.im[i][j] = im;
        }
    return c;
}

template <typename R> __device__ __forceinline__ void add_to(Mat<R> &c, const Mat<R> &a)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            c.re[i][j] += a.re[i][j];
            c.im[i][j] += a.im[i][j];
        }
}

// c += op_a(a) * op_b(b)   (the accumulation is free: every term is an FMA)
template <int FA, int FB, typename R>
__device__ __forceinline__ void mul_acc(Mat<R> &c, const Mat<R> &a, const Mat<R> &b)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            R re = c.re[i][j], im = c.im[i][j];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                re = fma(el_re<FA>(a, i, k), el_re<FB>(b, k, j), re);
                re = fma(-el_im<FA>(a, i, k), el_im<FB>(b, k, j), re);
                im = fma(el_re<FA>(a, i, k), el_im<FB>(b, k, j), im);
                im = fma(el_im<FA>(a, i, k), el_re<FB>(b, k, j), im);
            }
            c.re[i][j] = re;
            c.im[i][j] = im;
        }
}

// c += s * a
template <typename R> __device__ __forceinline__ void axpy(Mat<R> &c, R s, const Mat<R> &a)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            c.re[i][j] = fma(s, a.re[i][j], c.re[i][j]);
            c.im[i][j] = fma(s, a.im[i][j], c.im[i][j]);
        }
}

template <typename R> __device__ __forceinline__ void scale(Mat<R> &c, R s)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            c.re[i][j] *= s;
            c.im[i][j] *= s;
        }
}

// Re tr(op_a(a) * op_b(b)) without forming the product.
template <int FA, int FB, typename R>
__device__ __forceinline__ R re_trace_mul(const Mat<R> &a, const Mat<R> &b)
{
    R s = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            s = fma(el_re<FA>(a, i, k), el_re<FB>(b, k, i), s);
            s = fma(-el_im<FA>(a, i, k), el_im<FB>(b, k, i), s);
        }
    return s;
}

// Row 2 of an SU(3) matrix from rows 0 and 1: row2 = conj(row0 x row1).
template <typename R> __device__ __forceinline__ void rebuild_row2(Mat<R> &u)
{
#define LQCD_CROSS(j, k, l)                                                                     \
    u.re[2][j] = (u.re[0][k] * u.re[1][l] - u.im[0][k] * u.im[1][l]) -                          \
                 (u.re[0][l] * u.re[1][k] - u.im[0][l] * u.im[1][k]);                           \
    u.im[2][j] = -((u.re[0][k] * u.im[1][l] + u.im[0][k] * u.re[1][l]) -                        \
                   (u.re[0][l] * u.im[1][k] + u.im[0][l] * u.re[1][k]));
    LQCD_CROSS(0, 1, 2)
    LQCD_CROSS(1, 2, 0)
    LQCD_CROSS(2, 0, 1)
#undef LQCD_CROSS
}

// y += s * (a * op_b(b)) for a, b in SU(3): rows 0 and 1 of the product
// come from rows 0 and 1 of a, and its third row is conj(row0 x row1) of the
// product (a product of SU(3) matrices is in SU(3)).  The third row of a is
// never read, so for a compact link or staple its rebuild is dead code:
// 96 instead of 132 flops per product.
template <int FB, typename R>
__device__ __forceinline__ void mul_acc_su3(Mat<R> &y, const Mat<R> &a, const Mat<R> &b,
                                            R s = R(1))
{
    Mat<R> p = mul_top2<N, FB>(a, b);
    rebuild_row2(p);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            y.re[i][j] = fma(s, p.re[i][j], y.re[i][j]);
            y.im[i][j] = fma(s, p.im[i][j], y.im[i][j]);
        }
}

// ------------------------------------------------------------- link I/O

// Link layout: real r of link (n, mu) at ((mu*(12/W) + r/W)*V + n)*W + r%W.
template <typename R>
__device__ __forceinline__ Mat<R> load_link(const R *__restrict__ links, int64_t V, int mu,
                                            int64_t n)
{
    using V4 = typename Vec<R>::type;
    constexpr int W = Vec<R>::W;
    const V4 *p = reinterpret_cast<const V4 *>(links) + (int64_t)mu * (12 / W) * V + n;
    R r[12];
#pragma unroll
    for (int q = 0; q < 12 / W; ++q) {
        V4 v = __ldg(p + q * V);
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

template <typename R>
__device__ __forceinline__ void store_link(R *__restrict__ links, int64_t V, int mu, int64_t n,
                                           const Mat<R> &u)
{
    using V4 = typename Vec<R>::type;
    constexpr int W = Vec<R>::W;
    V4 *p = reinterpret_cast<V4 *>(links) + (int64_t)mu * (12 / W) * V + n;
    R r[12];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            r[6 * i + 2 * j] = u.re[i][j];
            r[6 * i + 2 * j + 1] = u.im[i][j];
        }
#pragma unroll
    for (int q = 0; q < 12 / W; ++q) {
        V4 v;
        if constexpr (W == 4) {
            v = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
        } else {
            v = make_double2(r[2 * q], r[2 * q + 1]);
        }
        p[q * V] = v;
    }
}

// Algebra layout: component a of link (n, mu) at ((mu*(8/W) + a/W)*V + n)*W + a%W.
template <typename R>
__device__ __forceinline__ void load_algebra(const R *__restrict__ f, int64_t V, int mu, int64_t n,
                                             R a[8])
{
    using V4 = typename Vec<R>::type;
    constexpr int W = Vec<R>::W;
    const V4 *p = reinterpret_cast<const V4 *>(f) + (int64_t)mu * (8 / W) * V + n;
#pragma unroll
    for (int q = 0; q < 8 / W; ++q) {
        V4 v = __ldg(p + q * V);
        if constexpr (W == 4) {
            a[4 * q + 0] = v.x;
            a[4 * q + 1] = v.y;
            a[4 * q + 2] = v.z;
            a[4 * q + 3] = v.w;
        } else {
            a[2 * q + 0] = v.x;
            a[2 * q + 1] = v.y;
        }
    }
}

template <typename R>
__device__ __forceinline__ void store_algebra(R *__restrict__ f, int64_t V, int mu, int64_t n,
                                              const R a[8])
{
    using V4 = typename Vec<R>::type;
    constexpr int W = Vec<R>::W;
    V4 *p = reinterpret_cast<V4 *>(f) + (int64_t)mu * (8 / W) * V + n;
#pragma unroll
    for (int q = 0; q < 8 / W; ++q) {
        V4 v;
        if constexpr (W == 4) {
            v = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
        } else {
            v = make_double2(a[2 * q], a[2 * q + 1]);
        }
        p[q * V] = v;
    }
}

// ------------------------------------------------ su(3) <-> 3x3 matrices

// f^a = 2 Re tr(i T_a G) = -Im tr(lambda_a M) * s for G = s (M)_TA: the eight
// components of s times the traceless anti-Hermitian part of M, read off the
// Gell-Mann matrices (only the anti-Hermitian traceless part of M enters).
template <typename R>
__device__ __forceinline__ void ta_components(const Mat<R> &m, R s, R f[8])
{
    const R inv_sqrt3 = R(0.57735026918962576451);
    f[0] = -s * (m.im[0][1] + m.im[1][0]);
    f[1] = -s * (m.re[0][1] - m.re[1][0]);
    f[2] = -s * (m.im[0][0] - m.im[1][1]);
    f[3] = -s * (m.im[0][2] + m.im[2][0]);
    f[4] = -s * (m.re[0][2] - m.re[2][0]);
    f[5] = -s * (m.im[1][2] + m.im[2][1]);
    f[6] = -s * (m.re[1][2] - m.re[2][1]);
    f[7] = -s * inv_sqrt3 * (m.im[0][0] + m.im[1][1] - R(2) * m.im[2][2]);
}

// Q = sum_a p^a T_a (Hermitian, traceless) from the eight components.
template <typename R> __device__ __forceinline__ Mat<R> algebra_matrix(const R p[8])
{
    const R h = R(0.5);
    const R inv_sqrt3 = R(0.57735026918962576451);
    Mat<R> q;
    q.re[0][0] = h * (p[2] + inv_sqrt3 * p[7]);
    q.re[1][1] = h * (-p[2] + inv_sqrt3 * p[7]);
    q.re[2][2] = -inv_sqrt3 * p[7];
    q.im[0][0] = q.im[1][1] = q.im[2][2] = R(0);
    q.re[0][1] = q.re[1][0] = h * p[0];
    q.im[0][1] = -h * p[1];
    q.im[1][0] = h * p[1];
    q.re[0][2] = q.re[2][0] = h * p[3];
    q.im[0][2] = -h * p[4];
    q.im[2][0] = h * p[4];
    q.re[1][2] = q.re[2][1] = h * p[5];
    q.im[1][2] = -h * p[6];
    q.im[2][1] = h * p[6];
    return q;
}

// exp(i Q) for Hermitian traceless Q.  By the Cayley-Hamilton theorem
// Q^3 = c1 Q + c0 with c0 = det Q, c1 = tr(Q^2)/2, so every power
// Q^n = a_n + b_n Q + d_n Q^2 with (a, b, d)_{n+1} = (c0 d_n, a_n + c1 d_n, b_n),
// and exp(iQ) = f0 + f1 Q + f2 Q^2 with f = sum_n i^n/n! (a_n, b_n, d_n).
// Q is first scaled by 2^-s so that ||Q||_F <= 1; the series is then cut
// after NT terms (error < 1/(NT+1)!), and the result squared s times.
template <typename R> __device__ __forceinline__ Mat<R> exp_i_hermitian(Mat<R> q)
{
    constexpr int NT = sizeof(R) == 8 ? 19 : 12;
    Mat<R> q2 = mul<N, N>(q, q);
    R c1 = R(0.5) * (q2.re[0][0] + q2.re[1][1] + q2.re[2][2]);
    int s = 0;
    R scl = R(1);
    // ||Q||_F^2 = 2 c1
    while (R(2) * c1 * scl * scl > R(1) && s < 60) {
        scl *= R(0.5);
        ++s;
    }
    if (s > 0) {
        scale(q, scl);
        scale(q2, scl * scl);
        c1 *= scl * scl;
    }
    // c0 = det Q = tr(Q^3)/3 = Re tr(Q Q^2)/3
    R c0 = re_trace_mul<N, N>(q, q2) * R(1.0 / 3.0);
    // accumulate sum_n i^n/n! (a_n, b_n, d_n)
    R a = R(1), b = R(0), d = R(0);
    R f0r = R(1), f0i = R(0), f1r = R(0), f1i = R(0), f2r = R(0), f2i = R(0);
    R fact = R(1);
#pragma unroll
    for (int n = 1; n <= NT; ++n) {
        R an = c0 * d, bn = a + c1 * d, dn = b;
        a = an;
        b = bn;
        d = dn;
        fact *= R(1) / R(n);
        // i^n: n%4 = 0 -> 1, 1 -> i, 2 -> -1, 3 -> -i
        const int m = n & 3;
        const R sg = (m == 0 || m == 1) ? R(1) : R(-1);
        if (m == 0 || m == 2) {
            f0r += sg * fact * a;
            f1r += sg * fact * b;
            f2r += sg * fact * d;
        } else {
            f0i += sg * fact * a;
            f1i += sg * fact * b;
            f2i += sg * fact * d;
        }
    }
    Mat<R> e;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            // (f1r + i f1i) q + (f2r + i f2i) q2 (+ f0 on the diagonal)
            R re = f1r * q.re[i][j] - f1i * q.im[i][j] + f2r * q2.re[i][j] - f2i * q2.im[i][j];
            R im = f1r * q.im[i][j] + f1i * q.re[i][j] + f2r * q2.im[i][j] + f2i * q2.re[i][j];
            if (i == j) {
                re += f0r;
                im += f0i;
            }
            e.re[i][j] = re;
            e.im[i][j] = im;
        }
    for (int k = 0; k < s; ++k) e = mul<N, N>(e, e);
    return e;
}

// Row i scaled to unit length: u <- u + u c with c = 1/|u| - 1 written as
// -d / (r (1 + r)), d = |u|^2 - 1, r = |u|.  The plain form u <- u * (1/|u|)
// rounds the factor 1/|u| to a grid point next to 1, where the spacing is
// 2^-24 below 1 and 2^-23 above it, so that for rows that are already nearly
// normalised (every link step) FP32 rows came out longer on average
// (|u|^2 - 1 = +5e-8 over random SU(3) matrices: an action offset of about
// 1e-7 relative, 5 at 48^3x96).  Here the small correction c keeps its full
// relative precision and each entry is rounded once (FMA); in FP32 d is also
// formed without rounding bias: every square is split exactly into its
// rounded value and error by an FMA, the rounded values are added with
// their errors kept (two-sum), and 1 is subtracted from the leading part
// (exact for a sum within a factor 2 of 1).  The mean of |u|^2 - 1 is then
// below 1e-10 in FP32 (it was -1e-8 with d from a plain FP32 sum).
template <typename R> __device__ __forceinline__ void normalise_row(Mat<R> &u, int i)
{
    R d;
    if constexpr (sizeof(R) == 4) {
        R s = R(0), e = R(0);
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const R x = (j & 1) ? u.im[i][j >> 1] : u.re[i][j >> 1];
            const R p = __fmul_rn(x, x); // never contracted into an FMA
            const R pe = fma(x, x, -p);
            const R t = s + p;
            const R bb = t - s;
            e += ((s - (t - bb)) + (p - bb)) + pe;
            s = t;
        }
        d = (s - R(1)) + e;
    } else {
        R s = R(0);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            s = fma(u.re[i][j], u.re[i][j], s);
            s = fma(u.im[i][j], u.im[i][j], s);
        }
        d = s - R(1);
    }
    const R r = sqrt(R(1) + d);
    const R c = -d / (r * (R(1) + r));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        u.re[i][j] = fma(u.re[i][j], c, u.re[i][j]);
        u.im[i][j] = fma(u.im[i][j], c, u.im[i][j]);
    }
}

// Gram-Schmidt of rows 0 and 1, then row 2 = conj(row0 x row1).
template <typename R> __device__ __forceinline__ void reunitarise(Mat<R> &u)
{
    normalise_row(u, 0);
    // proj = <row0, row1> = sum conj(u0j) u1j
    R pr = R(0), pi = R(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        pr = fma(u.re[0][j], u.re[1][j], fma(u.im[0][j], u.im[1][j], pr));
        pi = fma(u.re[0][j], u.im[1][j], fma(-u.im[0][j], u.re[1][j], pi));
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        u.re[1][j] = fma(-pr, u.re[0][j], fma(pi, u.im[0][j], u.re[1][j]));
        u.im[1][j] = fma(-pr, u.im[0][j], fma(-pi, u.re[0][j], u.im[1][j]));
    }
    normalise_row(u, 1);
    rebuild_row2(u);
}

// ------------------------------------------------------------- geometry

// Periodic lattice, x fastest.  Extents and strides are scalar members and a
// direction is picked by a select chain, so that nothing is indexed at run
// time in per-thread storage (which would go to local memory).
struct Geom {
    int L0, L1, L2, L3;
    int64_t s1, s2, s3, V;
};

__host__ __device__ __forceinline__ Geom make_geom(const int dims[4])
{
    Geom g;
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

struct Coord {
    int c0, c1, c2, c3;
};

// n / d for n < 2^31 with the magic of d (kernels.h: DivMagic).
__device__ __forceinline__ unsigned div_by(unsigned n, const DivMagic &d)
{
    const unsigned t = __umulhi(d.m, n);
    return (t + ((n - t) >> d.sh1)) >> d.sh2;
}

__device__ __forceinline__ Coord coord_of(const Geom &g, int64_t n)
{
    Coord x;
    x.c3 = (int)(n / g.s3);
    int64_t r = n - x.c3 * g.s3;
    x.c2 = (int)(r / g.s2);
    r -= x.c2 * g.s2;
    x.c1 = (int)(r / g.s1);
    x.c0 = (int)(r - x.c1 * g.s1);
    return x;
}

__device__ __forceinline__ int pick(int mu, int a, int b, int c, int d)
{
    return mu == 0 ? a : (mu == 1 ? b : (mu == 2 ? c : d));
}

__device__ __forceinline__ int64_t pick64(int mu, int64_t a, int64_t b, int64_t c, int64_t d)
{
    return mu == 0 ? a : (mu == 1 ? b : (mu == 2 ? c : d));
}

__device__ __forceinline__ int64_t stride_of(const Geom &g, int mu)
{
    return pick64(mu, 1, g.s1, g.s2, g.s3);
}

// Linear-index offset of the displacement d * hat(mu), |d| <= 2, from a site
// whose mu-coordinate is c, with periodic wrap-around.
__device__ __forceinline__ int64_t disp(const Geom &g, const Coord &x, int mu, int d)
{
    const int L = pick(mu, g.L0, g.L1, g.L2, g.L3);
    const int c = pick(mu, x.c0, x.c1, x.c2, x.c3);
    int v = c + d;
    if (v >= L) v -= L;
    if (v >= L) v -= L;
    if (v < 0) v += L;
    if (v < 0) v += L;
    return (int64_t)(v - c) * stride_of(g, mu);
}

// One step x -> x + s * hat(mu) (s = +-1) on coordinates.
__device__ __forceinline__ void step(const Geom &g, Coord &x, int mu, int s)
{
    switch (mu) {
    case 0: x.c0 = x.c0 + s == g.L0 ? 0 : (x.c0 + s < 0 ? g.L0 - 1 : x.c0 + s); break;
    case 1: x.c1 = x.c1 + s == g.L1 ? 0 : (x.c1 + s < 0 ? g.L1 - 1 : x.c1 + s); break;
    case 2: x.c2 = x.c2 + s == g.L2 ? 0 : (x.c2 + s < 0 ? g.L2 - 1 : x.c2 + s); break;
    default: x.c3 = x.c3 + s == g.L3 ? 0 : (x.c3 + s < 0 ? g.L3 - 1 : x.c3 + s); break;
    }
}

__device__ __forceinline__ int64_t index_of(const Geom &g, const Coord &x)
{
    return (int64_t)x.c0 + g.s1 * x.c1 + g.s2 * x.c2 + g.s3 * x.c3;
}

} // namespace lqcd
