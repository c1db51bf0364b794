/*
 * Plain FP64 CPU oracle for the one-loop Symanzik improved gauge action, its
 * molecular-dynamics force and the MD momentum / link updates that use it
 * (D. Li, "The Calculation of Force in Lattice Quantum Chromodynamics",
 * Sec. II, Eqs. 18_3_27_30 ... 18_6_6_13), and the hopping operator of the
 * Wilson fermion matrix with its force on the links (Sec. III, Eqs. 18_7_17_4
 * and 18_1_29_19 ... 18_7_17_30).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA
 * library: only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or constant
 * with the CUDA sources.  It is deliberately slow: every quantity is the
 * paper's definition written out in its notation -- the action as the sum of
 * the 34 loop traces at every site, the force on each link as the derivative
 * of the loops through that link -- with C99 complex arithmetic, no blocking,
 * no fusion and no reordering beyond what the equations state.
 *
 * Conventions.
 *   - Directions are numbered 1..4 as in the paper (x, y, z, t).  A signed
 *     direction d is +mu or -mu.  Site n = (x, y, z, t), x fastest, periodic.
 *   - U[n][mu-1] is the 3x3 complex link U_{n,mu} on the link (n, n+mu);
 *     U_{n+mu,-mu} = U_{n,mu}^dagger  (Sec. II, text after Eq. 18_3_27_30).
 *   - T_a = lambda_a / 2 (Gell-Mann), tr(T_a T_b) = delta_ab / 2 (Eq. 18_1_29_3_0).
 *   - The force returned for link (k, rho) is the 8-vector
 *         f^a = -dS/domega^a_{k,rho} = 2 tr(T_a H_{k,rho}),
 *     where H = -sum_a T_a dS/domega^a = (beta/6) i (U t)_TA is the paper's
 *     Hermitian force (Eqs. 18_7_25_1, 18_7_25_2), and d/domega is the left
 *     Lie derivative U -> exp(i eps T_a) U (Eq. 18_7_26_1).
 *
 * Parity pins (checked by tests/test_oracle_pins.py, CPU only): unit
 * configuration, closed-form abelian fluxes, gauge invariance/covariance,
 * finite differences along all 8 generators, the Wilson-action limit against
 * an independent staple formula, uniform-link configurations against a
 * brute-force single-site sum, the identity of Eq. 18_6_6_13, the exponential
 * against scipy.linalg.expm, the reunitarisation against Gram-Schmidt (a QR
 * factorisation) on links that are not unitary, and leapfrog energy
 * conservation/reversibility; for Sec. III: the Clifford algebra of the gamma basis, the free-field
 * (unit-link) plane-wave spectrum of the hopping operator, its gamma_5
 * hermiticity, gauge covariance, and finite differences of
 * 2 Re Y^dag calD X along all 8 generators against the hopping force.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;
typedef struct { cplx m[3][3]; } mat3;

/* ---------------------------------------------------------------- geometry */

typedef struct { int L[4]; long V; } geom;

static geom make_geom(const int dims[4])
{
    geom g;
    g.V = 1;
    for (int i = 0; i < 4; ++i) { g.L[i] = dims[i]; g.V *= dims[i]; }
    return g;
}

static void coords(const geom *g, long n, int x[4])
{
    for (int i = 0; i < 4; ++i) { x[i] = (int)(n % g->L[i]); n /= g->L[i]; }
}

static long index_of(const geom *g, const int x[4])
{
    long n = 0;
    for (int i = 3; i >= 0; --i) n = n * g->L[i] + x[i];
    return n;
}

/* n + hat(d) for a signed direction d = +-mu, periodic in all four directions
 * (boundary conditions are not stated in the paper; periodic is assumed). */
static long step(const geom *g, long n, int d)
{
    int x[4];
    coords(g, n, x);
    int mu = abs(d) - 1;
    x[mu] += (d > 0) ? 1 : -1;
    x[mu] = (x[mu] % g->L[mu] + g->L[mu]) % g->L[mu];
    return index_of(g, x);
}

/* ----------------------------------------------------- 3x3 complex algebra */

static mat3 zero3(void) { mat3 r; memset(&r, 0, sizeof r); return r; }

static mat3 unit3(void)
{
    mat3 r = zero3();
    for (int i = 0; i < 3; ++i) r.m[i][i] = 1.0;
    return r;
}

static mat3 mul(mat3 a, mat3 b)
{
    mat3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx s = 0;
            for (int k = 0; k < 3; ++k) s += a.m[i][k] * b.m[k][j];
            r.m[i][j] = s;
        }
    return r;
}

static mat3 dagger(mat3 a)
{
    mat3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r.m[i][j] = conj(a.m[j][i]);
    return r;
}

static mat3 add(mat3 a, mat3 b)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) a.m[i][j] += b.m[i][j];
    return a;
}

static mat3 scale(cplx s, mat3 a)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) a.m[i][j] *= s;
    return a;
}

static cplx trace(mat3 a) { return a.m[0][0] + a.m[1][1] + a.m[2][2]; }

/* Traceless anti-Hermitian part, Eq. 18_6_6_11:
 *   B_TA = (B - B^dagger)/2 - tr(B - B^dagger)/6 * I. */
static mat3 traceless_antihermitian(mat3 b)
{
    mat3 d = add(b, scale(-1.0, dagger(b)));
    cplx tr = trace(d);
    mat3 r = scale(0.5, d);
    for (int i = 0; i < 3; ++i) r.m[i][i] -= tr / 6.0;
    return r;
}

/* The eight su(3) generators T_a = lambda_a / 2, normalised as in
 * Eq. 18_1_29_3_0.  a = 0..7 stands for the paper's i = 1..8. */
static mat3 generator(int a)
{
    mat3 l = zero3();
    switch (a) {
    case 0: l.m[0][1] = 1; l.m[1][0] = 1; break;
    case 1: l.m[0][1] = -I; l.m[1][0] = I; break;
    case 2: l.m[0][0] = 1; l.m[1][1] = -1; break;
    case 3: l.m[0][2] = 1; l.m[2][0] = 1; break;
    case 4: l.m[0][2] = -I; l.m[2][0] = I; break;
    case 5: l.m[1][2] = 1; l.m[2][1] = 1; break;
    case 6: l.m[1][2] = -I; l.m[2][1] = I; break;
    case 7:
        l.m[0][0] = 1.0 / sqrt(3.0);
        l.m[1][1] = 1.0 / sqrt(3.0);
        l.m[2][2] = -2.0 / sqrt(3.0);
        break;
    }
    return scale(0.5, l);
}

/* X = sum_a w^a T_a (Hermitian, traceless). */
static mat3 algebra_matrix(const double w[8])
{
    mat3 x = zero3();
    for (int a = 0; a < 8; ++a) x = add(x, scale(w[a], generator(a)));
    return x;
}

static double norm_inf(mat3 a)
{
    double best = 0.0;
    for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j) s += cabs(a.m[i][j]);
        if (s > best) best = s;
    }
    return best;
}

/* Matrix exponential by scaling and squaring of a truncated Taylor series:
 * exp(X) = (exp(X / 2^s))^(2^s), with ||X / 2^s|| <= 1/2 and 25 Taylor
 * terms, so the truncation error is below 0.5^26/26! ~ 4e-35 relative.
 * (Deliberately not the Cayley-Hamilton closed form used on the GPU.) */
static mat3 expm(mat3 x)
{
    int s = 0;
    double nrm = norm_inf(x);
    while (nrm > 0.5) { nrm *= 0.5; ++s; }
    mat3 y = scale(ldexp(1.0, -s), x);
    mat3 term = unit3(), sum = unit3();
    for (int k = 1; k <= 25; ++k) {
        term = scale(1.0 / k, mul(term, y));
        sum = add(sum, term);
    }
    for (int i = 0; i < s; ++i) sum = mul(sum, sum);
    return sum;
}

/* U = exp(i sum_a w^a T_a), Eq. 18_1_29_3. */
static mat3 exp_i_algebra(const double w[8])
{
    return expm(scale(I, algebra_matrix(w)));
}

/* Rows 0 and 1 orthonormalised by Gram-Schmidt, row 2 = conj(row0 x row1):
 * the nearest-by-construction SU(3) matrix used after a link update. */
static mat3 reunitarise(mat3 u)
{
    double n0 = 0;
    for (int j = 0; j < 3; ++j) n0 += creal(u.m[0][j] * conj(u.m[0][j]));
    n0 = 1.0 / sqrt(n0);
    for (int j = 0; j < 3; ++j) u.m[0][j] *= n0;
    cplx proj = 0;
    for (int j = 0; j < 3; ++j) proj += conj(u.m[0][j]) * u.m[1][j];
    for (int j = 0; j < 3; ++j) u.m[1][j] -= proj * u.m[0][j];
    double n1 = 0;
    for (int j = 0; j < 3; ++j) n1 += creal(u.m[1][j] * conj(u.m[1][j]));
    n1 = 1.0 / sqrt(n1);
    for (int j = 0; j < 3; ++j) u.m[1][j] *= n1;
    u.m[2][0] = conj(u.m[0][1] * u.m[1][2] - u.m[0][2] * u.m[1][1]);
    u.m[2][1] = conj(u.m[0][2] * u.m[1][0] - u.m[0][0] * u.m[1][2]);
    u.m[2][2] = conj(u.m[0][0] * u.m[1][1] - u.m[0][1] * u.m[1][0]);
    return u;
}

/* ----------------------------------------------------------- link field */

typedef struct {
    geom g;
    const cplx *U; /* [V][4][3][3] */
} field;

static mat3 get_link(const field *f, long n, int mu /* 1..4 */)
{
    mat3 r;
    memcpy(&r, f->U + ((size_t)n * 4 + (mu - 1)) * 9, sizeof r);
    return r;
}

/* U_{n,d} for a signed direction d: U_{n,-mu} = U_{n-mu,mu}^dagger. */
static mat3 link_dir(const field *f, long n, int d)
{
    if (d > 0) return get_link(f, n, d);
    return dagger(get_link(f, step(&f->g, n, d), -d));
}

/* -------------------------------------------------------------- 34 paths */

enum { CLS_PLAQ = 0, CLS_RECT = 1, CLS_CUBE = 2 };

typedef struct {
    int len;
    int d[6];
    int cls;
} path;

/* The 34 closed paths of Eq. 18_3_27_30 that begin and end at site n:
 *   6 plaquettes  (+mu, +nu, -mu, -nu)                 1 <= mu < nu <= 4
 *  12 rectangles  (+mu, +mu, +nu, -mu, -mu, -nu)       mu != nu
 *  16 cubes       (+mu, s nu, t rho, -mu, -s nu, -t rho)
 *                                                      mu < nu < rho, s,t = +-1
 * written as the direction sequences d_1..d_L of Eq. 18_6_6_3_0. */
static int build_paths(path p[34])
{
    int np = 0;
    for (int mu = 1; mu <= 4; ++mu)
        for (int nu = mu + 1; nu <= 4; ++nu) {
            path q = {4, {mu, nu, -mu, -nu, 0, 0}, CLS_PLAQ};
            p[np++] = q;
        }
    for (int mu = 1; mu <= 4; ++mu)
        for (int nu = 1; nu <= 4; ++nu) {
            if (nu == mu) continue;
            path q = {6, {mu, mu, nu, -mu, -mu, -nu}, CLS_RECT};
            p[np++] = q;
        }
    for (int mu = 1; mu <= 4; ++mu)
        for (int nu = mu + 1; nu <= 4; ++nu)
            for (int rho = nu + 1; rho <= 4; ++rho)
                for (int s = 1; s >= -1; s -= 2)
                    for (int t = 1; t >= -1; t -= 2) {
                        path q = {6, {mu, s * nu, t * rho, -mu, -s * nu, -t * rho}, CLS_CUBE};
                        p[np++] = q;
                    }
    return np;
}

/* Sites n_1..n_L visited by path p started at n (Eq. 18_6_6_3_0):
 * n_1 = n, n_{i+1} = n_i + hat(d_i). */
static void visit(const geom *g, const path *p, long n, long pos[6])
{
    pos[0] = n;
    for (int i = 1; i < p->len; ++i) pos[i] = step(g, pos[i - 1], p->d[i - 1]);
}

/* The path product P_n = U_{n_1,d_1} ... U_{n_L,d_L}. */
static mat3 path_product(const field *f, const path *p, long n)
{
    long pos[6];
    visit(&f->g, p, n, pos);
    mat3 m = unit3();
    for (int i = 0; i < p->len; ++i) m = mul(m, link_dir(f, pos[i], p->d[i]));
    return m;
}

/* -------------------------------------------------- coefficients (a1) */

/* alpha_s = -4 log(u0) / 3.06839 and the loop coefficients of
 * Eq. 18_3_27_30: c_plaq = 1, c_rect = -(1 + 0.4805 alpha_s) / (20 u0^2),
 * c_cube = -2 * 0.03325 alpha_s / u0^2 (the factor 2 is taken as printed). */
void oracle_coefficients(double u0, double c[3])
{
    double alpha_s = -4.0 * log(u0) / 3.06839;
    c[0] = 1.0;
    c[1] = -(1.0 + 0.4805 * alpha_s) / (20.0 * u0 * u0);
    c[2] = -(2.0 * 0.03325 * alpha_s) / (u0 * u0);
}

/* Exports the path table for the tests: d[34][6] (zero padded), len[34],
 * cls[34].  Returns the number of paths. */
int oracle_paths(int *d, int *len, int *cls)
{
    path p[34];
    int np = build_paths(p);
    for (int i = 0; i < np; ++i) {
        for (int j = 0; j < 6; ++j) d[i * 6 + j] = (j < p[i].len) ? p[i].d[j] : 0;
        len[i] = p[i].len;
        cls[i] = p[i].cls;
    }
    return np;
}

/* ------------------------------------------------------- action (a6) */

/* Neumaier-compensated running sum, so that the oracle's own rounding is
 * far below the tolerances it is used to check. */
typedef struct { double s, c; } ksum;
static void kadd(ksum *k, double x)
{
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else k->c += (x - t) + k->s;
    k->s = t;
}

/* Per-class sums  sum_n sum_{P in class} [3 - Re tr P_n]  (Eq. 18_6_4_1
 * without the factors beta/3 and c_P). out[0] plaquettes, out[1]
 * rectangles, out[2] cubes. */
void oracle_loop_sums(const int dims[4], const double *U, double out[3])
{
    field f = {make_geom(dims), (const cplx *)U};
    path p[34];
    int np = build_paths(p);
    ksum k[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int ip = 0; ip < np; ++ip)
        for (long n = 0; n < f.g.V; ++n)
            kadd(&k[p[ip].cls], 3.0 - creal(trace(path_product(&f, &p[ip], n))));
    for (int i = 0; i < 3; ++i) out[i] = k[i].s + k[i].c;
}

/* S_G = (beta/3) sum_{34 paths P} sum_n c_P [3 - Re tr P_n], Eq. 18_6_4_1. */
double oracle_gauge_action(const int dims[4], const double *U, double beta, const double c[3])
{
    double sums[3];
    oracle_loop_sums(dims, U, sums);
    ksum k = {0, 0};
    for (int i = 0; i < 3; ++i) kadd(&k, c[i] * sums[i]);
    return beta / 3.0 * (k.s + k.c);
}

/* The part of S_G made of the loops P_n that contain the link (k, rho) in
 * either orientation: the only part whose derivative along omega_{k,rho} is
 * non-zero (Eq. 18_7_26_1).  Used for cheap finite differences. */
double oracle_gauge_action_local(const int dims[4], const double *U, double beta,
                                 const double c[3], long k, int rho)
{
    field f = {make_geom(dims), (const cplx *)U};
    path p[34];
    int np = build_paths(p);
    long kr = step(&f.g, k, rho);
    ksum acc = {0, 0};
    for (int ip = 0; ip < np; ++ip)
        for (long n = 0; n < f.g.V; ++n) {
            long pos[6];
            visit(&f.g, &p[ip], n, pos);
            int hit = 0;
            for (int l = 0; l < p[ip].len; ++l) {
                if (p[ip].d[l] == rho && pos[l] == k) hit = 1;
                if (p[ip].d[l] == -rho && pos[l] == kr) hit = 1;
            }
            if (hit)
                kadd(&acc, c[p[ip].cls] * (3.0 - creal(trace(path_product(&f, &p[ip], n)))));
        }
    return beta / 3.0 * (acc.s + acc.c);
}

/* -------------------------------------------------------- force (a4, a5) */

/* What one loop through the link (k, rho) contributes to its derivative.
 * The loop P_n holds the link at position l (0-based), either as U_{k,rho}
 * itself (d_l = +rho, n_l = k) or as its inverse U_{k,rho}^dag = U_{k+rho,-rho}
 * (d_l = -rho, n_l = k + rho).  Write P_n = A U B or A U^dag B, with A the
 * factors before position l and B those after it.  Under the left
 * perturbation U -> exp(i eps T_a) U (Eqs. 18_7_26_1 to 18_7_26_3) the factor
 * becomes i T_a U, or U^dag (-i T_a), and the cyclic property of the trace
 * brings the link to the front:
 *   d/deps Re tr(A U B)     = Re tr(i T_a U (B A)),
 *   d/deps Re tr(A U^dag B) = Re tr(-i T_a B A U^dag) = Re tr(i T_a U (B A)^dag),
 * the last by Re tr M = Re tr M^dag.  Every loop through the link therefore
 * gives Re tr(i T_a U W); W = B A (forward) or (B A)^dag = A^dag B^dag
 * (backward) are the two staples of Eq. 18_7_25_2, returned here from the
 * sites pos[] that the loop visits. */
static mat3 staple(const field *f, const path *p, const long pos[6], int l, int forward)
{
    mat3 m = unit3();
    int L = p->len;
    if (forward) {
        for (int i = l + 1; i < L; ++i) m = mul(m, link_dir(f, pos[i], p->d[i]));
        for (int i = 0; i < l; ++i) m = mul(m, link_dir(f, pos[i], p->d[i]));
    } else {
        for (int i = l - 1; i >= 0; --i) m = mul(m, dagger(link_dir(f, pos[i], p->d[i])));
        for (int i = L - 1; i > l; --i) m = mul(m, dagger(link_dir(f, pos[i], p->d[i])));
    }
    return m;
}

/* f^a = 2 tr(T_a H) with H = (beta/6) i (U_{k,rho} t_{k,rho})_TA
 * (Eqs. 18_7_25_2, 18_6_6_11, 18_6_6_13). */
static void project(mat3 u, mat3 t, double beta, double out[8])
{
    mat3 h = scale(I * beta / 6.0, traceless_antihermitian(mul(u, t)));
    for (int a = 0; a < 8; ++a) out[a] = 2.0 * creal(trace(mul(generator(a), h)));
}

/* The force on the link (k, rho) from its definition, Eq. 18_7_25_1,
 *   H_{k,rho} = -sum_a T_a dS/domega^a_{k,rho},
 *   S = (beta/3) sum_P sum_n c_P [3 - Re tr P_n]                 (Eq. 18_6_4_1).
 * Only the loops through the link depend on omega_{k,rho}.  For a loop
 * shape P and a position l with d_l = +-rho exactly one start site puts the
 * link at position l:
 *   n = k - sum_{j<l} hat(d_j)             (d_l = +rho, Eq. 18_7_26_2),
 *   n = k + hat(rho) - sum_{j<l} hat(d_j)  (d_l = -rho, Eq. 18_7_26_3).
 * With the staples W of these loops (staple() above),
 *   -dS/domega^a = (beta/3) sum c_P Re tr(i T_a U W) = (beta/3) Re tr(i T_a U t),
 * t = sum c_P W, and the identity of Eq. 18_6_6_13,
 * sum_a T_a Re tr(i T_a B) = (1/2) i B_TA, gives H = (beta/6) i (U t)_TA. */
static void link_force(const field *f, const path p[34], int np, double beta, const double c[3],
                       long k, int rho, double out[8])
{
    mat3 t = zero3();
    for (int ip = 0; ip < np; ++ip)
        for (int l = 0; l < p[ip].len; ++l) {
            int dl = p[ip].d[l];
            if (dl != rho && dl != -rho) continue;
            long n = (dl == rho) ? k : step(&f->g, k, rho);
            for (int j = 0; j < l; ++j) n = step(&f->g, n, -p[ip].d[j]);
            long pos[6];
            visit(&f->g, &p[ip], n, pos);
            t = add(t, scale(c[p[ip].cls], staple(f, &p[ip], pos, l, dl == rho)));
        }
    project(get_link(f, k, rho), t, beta, out);
}

/* The force on every link, link by link.  Output f[V][4][8] (see project()). */
void oracle_gauge_force(const int dims[4], const double *U, double beta, const double c[3],
                        double *fout)
{
    field f = {make_geom(dims), (const cplx *)U};
    path p[34];
    int np = build_paths(p);
    for (long k = 0; k < f.g.V; ++k)
        for (int rho = 1; rho <= 4; ++rho)
            link_force(&f, p, np, beta, c, k, rho, fout + ((size_t)k * 4 + (rho - 1)) * 8);
}

/* The force on the single link (k, rho = 1..4). */
void oracle_gauge_force_link(const int dims[4], const double *U, double beta, const double c[3],
                             long k, int rho, double out[8])
{
    field f = {make_geom(dims), (const cplx *)U};
    path p[34];
    int np = build_paths(p);
    link_force(&f, p, np, beta, c, k, rho, out);
}

/* ---------------------------------------------------- exp map and MD (a7, a8) */

/* out[3][3] = exp(i sum_a w^a T_a), Eq. 18_1_29_3. */
void oracle_exp_i_algebra(const double w[8], double *out)
{
    mat3 u = exp_i_algebra(w);
    memcpy(out, &u, sizeof u);
}

/* Links from the 8 real parameters of every link: U_{n,mu} = exp(i omega.T)
 * (Eq. 18_1_29_3).  omega[V][4][8] -> U[V][4][3][3]. */
void oracle_links_from_omega(long nlinks, const double *omega, double *U)
{
    for (long i = 0; i < nlinks; ++i) {
        mat3 u = exp_i_algebra(omega + 8 * i);
        memcpy(U + 18 * i, &u, sizeof u);
    }
}

/* Momentum step of molecular dynamics: p^a += dt f^a, with f^a = -dS/domega^a
 * (the equation of motion that follows from H = sum p^2/2 + S_G and
 * Eq. 18_7_25_1). */
void oracle_md_update_momenta(long nlinks, double *p, const double *f, double dt)
{
    for (long i = 0; i < 8 * nlinks; ++i) p[i] += dt * f[i];
}

/* Link step of molecular dynamics: U <- exp(i dt sum_a p^a T_a) U, the flow
 * generated by the left parametrisation of Eq. 18_1_29_3, then
 * reunitarisation (Gram-Schmidt). */
void oracle_md_update_links(long nlinks, double *U, const double *p, double dt)
{
    for (long i = 0; i < nlinks; ++i) {
        double w[8];
        for (int a = 0; a < 8; ++a) w[a] = dt * p[8 * i + a];
        mat3 u;
        memcpy(&u, U + 18 * i, sizeof u);
        u = reunitarise(mul(exp_i_algebra(w), u));
        memcpy(U + 18 * i, &u, sizeof u);
    }
}

/* Kinetic term of the MD Hamiltonian, K = (1/2) sum p^a p^a. */
double oracle_kinetic_energy(long nlinks, const double *p)
{
    ksum k = {0, 0};
    for (long i = 0; i < 8 * nlinks; ++i) kadd(&k, 0.5 * p[i] * p[i]);
    return k.s + k.c;
}

/* Gauge transformation U'_{n,mu} = g_n U_{n,mu} g_{n+mu}^dagger, with
 * g[V][3][3].  The action is invariant because every P_n is a closed loop. */
void oracle_gauge_transform(const int dims[4], const double *U, const double *g, double *Uout)
{
    geom G = make_geom(dims);
    const cplx *gc = (const cplx *)g;
    for (long n = 0; n < G.V; ++n)
        for (int mu = 1; mu <= 4; ++mu) {
            mat3 u, gn, gm;
            memcpy(&u, (const cplx *)U + ((size_t)n * 4 + mu - 1) * 9, sizeof u);
            memcpy(&gn, gc + (size_t)n * 9, sizeof gn);
            memcpy(&gm, gc + (size_t)step(&G, n, mu) * 9, sizeof gm);
            mat3 r = mul(mul(gn, u), dagger(gm));
            memcpy((cplx *)Uout + ((size_t)n * 4 + mu - 1) * 9, &r, sizeof r);
        }
}

/* 2 tr(T_a H) read back as the Hermitian matrix H = sum_a f^a T_a (the
 * paper's force as a matrix, Eq. 18_7_25_1). */
void oracle_algebra_to_matrix(const double f[8], double *out)
{
    mat3 h = algebra_matrix(f);
    memcpy(out, &h, sizeof h);
}

/* B_TA of Eq. 18_6_6_11 for a test matrix b[3][3]. */
void oracle_traceless_antihermitian(const double *b, double *out)
{
    mat3 m;
    memcpy(&m, b, sizeof m);
    m = traceless_antihermitian(m);
    memcpy(out, &m, sizeof m);
}

/* The generator T_a (a = 0..7) as a 3x3 complex matrix, for the tests. */
void oracle_generator(int a, double *out)
{
    mat3 t = generator(a);
    memcpy(out, &t, sizeof t);
}

/* ===================================================== Wilson fermion (Sec. III)
 *
 * Spinor fields X[V][4][3] (Dirac index alpha, colour index a; complex).
 * The paper fixes no representation of the Euclidean gamma matrices; this
 * oracle takes the chiral basis below (Hermitian, gamma_mu^2 = 1,
 * {gamma_mu, gamma_nu} = 2 delta_{mu nu}, checked by the tests), with
 * gamma_1..gamma_4 acting along the directions x, y, z, t. */

typedef struct { cplx s[4][3]; } spinor;

/* gamma_mu for mu = 1..4, and gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 for
 * mu = 5 (written out as a product, not as a table). */
static void gamma_matrix(int mu, cplx g[4][4])
{
    memset(g, 0, 16 * sizeof(cplx));
    switch (mu) {
    case 1: g[0][3] = I;  g[1][2] = I;  g[2][1] = -I; g[3][0] = -I; break;
    case 2: g[0][3] = -1; g[1][2] = 1;  g[2][1] = 1;  g[3][0] = -1; break;
    case 3: g[0][2] = I;  g[1][3] = -I; g[2][0] = -I; g[3][1] = I;  break;
    case 4: g[0][2] = 1;  g[1][3] = 1;  g[2][0] = 1;  g[3][1] = 1;  break;
    case 5: {
        cplx a[4][4], b[4][4], p[4][4];
        gamma_matrix(1, a);
        for (int m = 2; m <= 4; ++m) {
            gamma_matrix(m, b);
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    cplx s = 0;
                    for (int k = 0; k < 4; ++k) s += a[i][k] * b[k][j];
                    p[i][j] = s;
                }
            memcpy(a, p, sizeof p);
        }
        memcpy(g, a, sizeof a);
        break;
    }
    }
}

/* (1 + sign * gamma_mu) acting on the Dirac index of x. */
static spinor spin_project(int mu, double sign, const spinor *x)
{
    cplx g[4][4];
    gamma_matrix(mu, g);
    spinor r;
    for (int al = 0; al < 4; ++al)
        for (int a = 0; a < 3; ++a) {
            cplx s = x->s[al][a];
            for (int be = 0; be < 4; ++be) s += sign * g[al][be] * x->s[be][a];
            r.s[al][a] = s;
        }
    return r;
}

/* u acting on the colour index of x. */
static spinor colour_mul(mat3 u, const spinor *x)
{
    spinor r;
    for (int al = 0; al < 4; ++al)
        for (int a = 0; a < 3; ++a) {
            cplx s = 0;
            for (int b = 0; b < 3; ++b) s += u.m[a][b] * x->s[al][b];
            r.s[al][a] = s;
        }
    return r;
}

static spinor get_spinor(const double *X, long n)
{
    spinor r;
    memcpy(&r, (const cplx *)X + (size_t)n * 12, sizeof r);
    return r;
}

/* The hopping part of the Wilson matrix, Eq. 18_7_17_4:
 *   (calD X)_n = sum_mu (1 - gamma_mu) U_{n,mu} X_{n+mu}
 *              + (1 + gamma_mu) U_{n,-mu} X_{n-mu},   U_{n,-mu} = U_{n-mu,mu}^dagger.
 * out[V][4][3]. */
static spinor hopping_site(const field *f, const double *X, long n)
{
    spinor acc;
    memset(&acc, 0, sizeof acc);
    for (int mu = 1; mu <= 4; ++mu) {
        spinor xf = get_spinor(X, step(&f->g, n, mu));
        spinor fw = spin_project(mu, -1.0, &xf);
        fw = colour_mul(link_dir(f, n, mu), &fw);
        spinor xb = get_spinor(X, step(&f->g, n, -mu));
        spinor bw = spin_project(mu, +1.0, &xb);
        bw = colour_mul(link_dir(f, n, -mu), &bw);
        for (int al = 0; al < 4; ++al)
            for (int a = 0; a < 3; ++a) acc.s[al][a] += fw.s[al][a] + bw.s[al][a];
    }
    return acc;
}

void oracle_wilson_hopping(const int dims[4], const double *U, const double *X, double *out)
{
    field f = {make_geom(dims), (const cplx *)U};
    for (long n = 0; n < f.g.V; ++n) {
        spinor acc = hopping_site(&f, X, n);
        memcpy((cplx *)out + (size_t)n * 12, &acc, sizeof acc);
    }
}

/* (calD X)_n at the single site n: out[4][3]. */
void oracle_wilson_hopping_site(const int dims[4], const double *U, const double *X, long n,
                                double *out)
{
    field f = {make_geom(dims), (const cplx *)U};
    spinor acc = hopping_site(&f, X, n);
    memcpy(out, &acc, sizeof acc);
}

/* The hopping-term force on link (k, rho) (rho = 1..4), Eqs. 18_1_29_20_1
 * to 18_7_17_30, literally:
 *   Z = (1 - gamma_rho) U_{k,rho} X_{k+rho},  B_{ba} = sum_alpha Z_{alpha b} conj(Y_{k, alpha a}),
 *   W = Y_{k+rho}^dagger (1 + gamma_rho) U_{k,rho}^dagger  (a row over alpha, a),
 *   C_{ba} = sum_alpha X_{k, alpha b} W_{alpha a},
 * and the 8 components of the paper's matrix -i (B - C)_TA = sum_i T_i h^i,
 *   h^i = -( tr(i T_i (B - C)) + c.c. ),
 * returned scaled: out[i] = coef * h^i.  With X = (D^dag D)^{-1} phi,
 * Y = D X and D = A - kappa calD, coef = kappa gives the hopping part of
 * -d/domega^i [phi^dag (D^dag D)^{-1} phi]  (Eqs. 18_6_24_0, 18_1_29_19). */
static void hopping_force_link(const field *f, const double *X, const double *Y, long k, int rho,
                               double coef, double out[8])
{
    long kp = step(&f->g, k, rho);
    mat3 u = get_link(f, k, rho);
    spinor xk = get_spinor(X, k), yk = get_spinor(Y, k);
    spinor xp = get_spinor(X, kp), yp = get_spinor(Y, kp);

    spinor ux = colour_mul(u, &xp);
    spinor z = spin_project(rho, -1.0, &ux);
    mat3 B = zero3();
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a)
            for (int al = 0; al < 4; ++al) B.m[b][a] += z.s[al][b] * conj(yk.s[al][a]);

    /* W_{alpha a} = sum_{beta, c} conj(Y_{beta c}) (1 + gamma)_{beta alpha} conj(U_{a c}) */
    cplx g[4][4];
    gamma_matrix(rho, g);
    cplx w[4][3];
    for (int al = 0; al < 4; ++al)
        for (int a = 0; a < 3; ++a) {
            cplx s = 0;
            for (int be = 0; be < 4; ++be) {
                cplx pg = (be == al ? 1.0 : 0.0) + g[be][al];
                for (int c = 0; c < 3; ++c) s += conj(yp.s[be][c]) * pg * conj(u.m[a][c]);
            }
            w[al][a] = s;
        }
    mat3 C = zero3();
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a)
            for (int al = 0; al < 4; ++al) C.m[b][a] += xk.s[al][b] * w[al][a];

    mat3 m = add(B, scale(-1.0, C));
    for (int i = 0; i < 8; ++i) {
        cplx tr = trace(mul(scale(I, generator(i)), m));
        out[i] = coef * (-(tr + conj(tr)));
    }
}

/* The hopping-term force on every link: out[V][4][8]. */
void oracle_wilson_hopping_force(const int dims[4], const double *U, const double *X,
                                 const double *Y, double coef, double *out)
{
    field f = {make_geom(dims), (const cplx *)U};
    for (long k = 0; k < f.g.V; ++k)
        for (int rho = 1; rho <= 4; ++rho)
            hopping_force_link(&f, X, Y, k, rho, coef, out + ((size_t)k * 4 + rho - 1) * 8);
}

/* The same on one link (k, rho = 1..4). */
void oracle_wilson_hopping_force_link(const int dims[4], const double *U, const double *X,
                                      const double *Y, double coef, long k, int rho, double out[8])
{
    field f = {make_geom(dims), (const cplx *)U};
    hopping_force_link(&f, X, Y, k, rho, coef, out);
}

/* gamma_mu (mu = 1..5) as a 4x4 complex matrix, for the tests. */
void oracle_gamma(int mu, double *out)
{
    cplx g[4][4];
    gamma_matrix(mu, g);
    memcpy(out, g, sizeof g);
}
