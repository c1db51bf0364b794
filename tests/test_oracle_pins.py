"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix
(no GPU).  Each test would fail on a plausible mistake in the oracle: a
dropped or mis-oriented loop, a wrong coefficient, a sign, a factor 2, a
transposed operand, a wrong generator."""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import oracle as O
from paper_1808_02281_gb300 import synth
from tests import helpers as H

DIMS4 = (4, 4, 4, 4)
BETA = 6.0


@pytest.fixture(scope="module")
def c1():
    """Workload 4^4: w_a ~ N(0, 0.5^2), seed 0, u0 = 0.87."""
    w = synth.WORKLOADS["4^4"]
    U = O.links_from_omega(synth.omega(w["dims"], w["sigma"], w["seed"]))
    c = O.coefficients(w["u0"])
    return U, c


@pytest.fixture(scope="module")
def c1_force(c1):
    U, c = c1
    return O.gauge_force(DIMS4, U, BETA, c)


def _hmat(f):
    """H = sum_a f^a lambda_a / 2 (numpy, textbook generators)."""
    return np.einsum("...a,aij->...ij", f, H.gell_mann() / 2)


# ------------------------------------------------------------ path table

def test_path_table_is_the_papers_enumeration():
    gold = H.read_paths()
    d, ln, cl = O.paths()
    names = ["plaq", "rect", "cube"]
    mine = sorted((names[c], tuple(int(v) for v in row[:n])) for row, n, c in zip(d, ln, cl))
    assert len(gold) == 34 and len(mine) == 34
    assert sorted(gold) == mine
    assert [sum(1 for k, _ in gold if k == n) for n in names] == [6, 12, 16]
    for _, seq in gold:  # every loop closes
        disp = np.zeros(4, int)
        for s in seq:
            disp[abs(s) - 1] += np.sign(s)
        assert not disp.any()


def test_48_staples_per_link():
    """Loop-link incidences per direction: 4*6 + 6*12 + 6*16 = 192 over the
    4 directions -> 48 staples per link (6 plaquette, 18 rectangle, 24 cube)."""
    counts = np.zeros((4, 3), int)
    for cls, seq in H.read_paths():
        for s in seq:
            counts[abs(s) - 1, ["plaq", "rect", "cube"].index(cls)] += 1
    assert (counts == [6, 18, 24]).all()


# --------------------------------------------------------- coefficients

def test_coefficients_tree_level():
    """u0 = 1: alpha_s = 0, so the action is the tree-level Luscher-Weisz
    action, c_rect = -1/20, c_cube = 0 (Eq. 18_3_27_30)."""
    np.testing.assert_allclose(O.coefficients(1.0), [1.0, -1.0 / 20.0, 0.0], atol=1e-16)


def test_coefficients_values():
    """alpha_s(0.87) = 0.18154415... from -4 ln(u0)/3.06839; the rectangle and
    cube coefficients then follow Eq. 18_3_27_30 with the printed 2 x 0.03325."""
    a = -4 * np.log(0.87) / 3.06839
    assert abs(a - 0.1815441549) < 1e-9
    c = O.coefficients(0.87)
    np.testing.assert_allclose(c, [1.0, -0.0718213744, -0.0159501735], atol=1e-10)


# ------------------------------------------------- special configurations

def test_unit_configuration_zero_action_and_force():
    V = 3 * 4 * 5 * 6
    dims = (3, 4, 5, 6)
    U = np.zeros((V, 4, 3, 3), complex)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    c = O.coefficients(0.87)
    assert O.gauge_action(dims, U, BETA, c) == 0.0
    assert not O.gauge_force(dims, U, BETA, c).any()


@pytest.mark.parametrize("dims,theta,phi,axes", [
    ((4, 4, 4, 4), np.pi / 2, 0.0, (0, 1, 2)),
    ((4, 4, 4, 4), np.pi / 2, np.pi / 2, (0, 1, 2)),
    ((4, 4, 4, 4), np.pi / 2, np.pi, (0, 1, 2)),
    ((8, 4, 3, 5), np.pi / 4, 3 * np.pi / 4, (0, 1, 2)),
    ((3, 5, 4, 6), 2 * np.pi / 5, -4 * np.pi / 5, (1, 3, 0)),
    ((4, 3, 6, 5), 2 * np.pi / 6, 2 * np.pi / 3, (2, 0, 3)),
])
def test_abelian_flux_closed_form(dims, theta, phi, axes):
    """Per-class loop sums equal the closed form derived from the loop shapes,
    which separates the three classes (and so the three coefficients)."""
    U = H.abelian_flux_links(dims, theta, phi, axes)
    V = int(np.prod(dims))
    np.testing.assert_allclose(O.loop_sums(dims, U), H.abelian_flux_class_sums(V, theta, phi),
                               rtol=1e-13, atol=1e-11)


def test_abelian_flux_worked_values():
    """S at beta = 6, u0 = 0.87 on 4^4 for three flux pairs."""
    c = O.coefficients(0.87)
    for (th, ph), want in [((np.pi / 2, 0.0), 599.1558292030),
                           ((np.pi / 2, np.pi / 2), 1263.6435689327),
                           ((np.pi / 2, np.pi), 2516.4920081496)]:
        S = O.gauge_action(DIMS4, H.abelian_flux_links(DIMS4, th, ph), BETA, c)
        assert abs(S - want) < 1e-9 * want


def test_uniform_links_brute_force():
    """U_{n,mu} = V_mu for all n: S/V is the single-site sum of the 34 loops
    (brute force over the golden table) and the force is the same on every site."""
    rng = np.random.default_rng(7)
    Vm = H.random_su3_numpy(rng, 4)
    dims = (3, 4, 3, 5)
    V = int(np.prod(dims))
    U = np.broadcast_to(Vm, (V, 4, 3, 3)).copy()
    c = O.coefficients(0.9)
    cm = {"plaq": c[0], "rect": c[1], "cube": c[2]}
    want = 0.0
    for cls, seq in H.read_paths():
        P = np.eye(3, dtype=complex)
        for s in seq:
            P = P @ (Vm[s - 1] if s > 0 else Vm[-s - 1].conj().T)
        want += cm[cls] * (3 - np.trace(P).real)
    want *= BETA / 3 * V
    assert abs(O.gauge_action(dims, U, BETA, c) - want) < 1e-12 * abs(want)
    f = O.gauge_force(dims, U, BETA, c)
    assert np.abs(f - f[0:1]).max() < 1e-13 * np.abs(f).max()


def test_wilson_limit_against_textbook_staples(c1):
    """c = (1, 0, 0) is the Wilson action S = (beta/3) sum_P (3 - Re tr P);
    its force f^a = (beta/3) Re tr(i T_a U Sigma), Sigma the 6 plaquette
    staples, written here independently of the oracle's TA projection."""
    U, _ = c1
    dims = DIMS4
    f = O.gauge_force(dims, U, BETA, np.array([1.0, 0.0, 0.0]))
    T = H.gell_mann() / 2
    V = int(np.prod(dims))
    X = H.site_coords(dims)

    def idx(x):
        x = [(x[i] % dims[i]) for i in range(4)]
        return x[0] + dims[0] * (x[1] + dims[1] * (x[2] + dims[2] * x[3]))

    dag = lambda m: m.conj().T
    for n in range(0, V, 17):
        x = X[n]
        for mu in range(4):
            e_mu = np.eye(4, dtype=int)[mu]
            S = np.zeros((3, 3), complex)
            for nu in range(4):
                if nu == mu:
                    continue
                e_nu = np.eye(4, dtype=int)[nu]
                S += U[idx(x + e_mu), nu] @ dag(U[idx(x + e_nu), mu]) @ dag(U[n, nu])
                S += dag(U[idx(x + e_mu - e_nu), nu]) @ dag(U[idx(x - e_nu), mu]) @ U[idx(x - e_nu), nu]
            want = np.array([BETA / 3 * np.trace(1j * T[a] @ U[n, mu] @ S).real for a in range(8)])
            np.testing.assert_allclose(f[n, mu], want, atol=1e-13)


# --------------------------------------------------- algebra and TA identity

def test_generators_are_gell_mann():
    T = np.stack([O.generator(a) for a in range(8)])
    np.testing.assert_allclose(T, H.gell_mann() / 2, atol=0)
    # normalisation of Eq. 18_1_29_3_0 and the textbook structure constants
    np.testing.assert_allclose(np.einsum("aij,bji->ab", T, T), np.eye(8) / 2, atol=1e-15)
    comm = lambda a, b: T[a] @ T[b] - T[b] @ T[a]
    np.testing.assert_allclose(comm(0, 1), 1j * T[2], atol=1e-15)          # f_123 = 1
    np.testing.assert_allclose(comm(3, 4), 0.5j * T[2] + np.sqrt(3) / 2 * 1j * T[7], atol=1e-15)


def test_ta_identity_eq_18_6_6_13():
    """sum_i T_i Re tr(i T_i B) = (1/2) i B_TA for any complex B, and B_TA is
    traceless anti-Hermitian with B - B_TA's anti-Hermitian part a multiple of 1."""
    rng = np.random.default_rng(3)
    T = H.gell_mann() / 2
    for _ in range(20):
        B = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        BTA = O.traceless_antihermitian(B)
        lhs = sum(T[i] * np.trace(1j * T[i] @ B).real for i in range(8))
        np.testing.assert_allclose(lhs, 0.5j * BTA, atol=1e-14)
        assert abs(np.trace(BTA)) < 1e-15
        np.testing.assert_allclose(BTA + BTA.conj().T, 0, atol=1e-15)
        R = (B - B.conj().T) / 2 - BTA
        np.testing.assert_allclose(R, R[0, 0] * np.eye(3), atol=1e-15)


def test_exponential_against_scipy():
    rng = np.random.default_rng(5)
    T = H.gell_mann() / 2
    for scale in (1e-3, 0.1, 0.5, 2.0, 10.0):
        w = scale * rng.standard_normal(8)
        E = O.exp_i_algebra(w)
        X = 1j * np.einsum("a,aij->ij", w, T)
        np.testing.assert_allclose(E, sla.expm(X), atol=1e-14 * max(1, scale))
        np.testing.assert_allclose(E @ E.conj().T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(E) - 1) < 1e-14
        np.testing.assert_allclose(E @ O.exp_i_algebra(-w), np.eye(3), atol=1e-14)


# ------------------------------------------------------------ the force

def test_force_link_equals_lattice_force(c1, c1_force):
    """The single-link entry point (used for sampled parity at full size)
    agrees with the whole-lattice one on links of every direction."""
    U, c = c1
    for n, mu in [(0, 0), (1, 1), (77, 2), (255, 3), (128, 0)]:
        np.testing.assert_allclose(O.gauge_force_link(DIMS4, U, BETA, c, n, mu),
                                   c1_force[n, mu], atol=1e-13)


def test_force_is_minus_the_gradient(c1, c1_force):
    """Central differences of S along exp(+-i eps T_a) U_{k,rho} for all 8
    generators on every link of the 4^4 lattice match -f^a (eps = 1e-4,
    O(eps^2) error)."""
    U, c = c1
    f = c1_force
    eps = 1e-4
    fmax = np.abs(f).max()
    links = range(U.shape[0] * 4)
    worst = 0.0
    for li in links:
        k, rho = divmod(int(li), 4)
        for a in range(8):
            w = np.zeros(8)
            w[a] = eps
            Up = U.copy()
            Up[k, rho] = O.exp_i_algebra(w) @ U[k, rho]
            Um = U.copy()
            Um[k, rho] = O.exp_i_algebra(-w) @ U[k, rho]
            fd = (O.gauge_action_local(DIMS4, Up, BETA, c, k, rho) -
                  O.gauge_action_local(DIMS4, Um, BETA, c, k, rho)) / (2 * eps)
            worst = max(worst, abs(fd + f[k, rho, a]))
    assert worst <= 1e-7 * fmax


def test_local_action_difference_equals_full(c1):
    U, c = c1
    rng = np.random.default_rng(11)
    for k, rho in [(5, 0), (200, 3)]:
        w = 0.05 * rng.standard_normal(8)
        U2 = U.copy()
        U2[k, rho] = O.exp_i_algebra(w) @ U[k, rho]
        d_full = O.gauge_action(DIMS4, U2, BETA, c) - O.gauge_action(DIMS4, U, BETA, c)
        d_loc = O.gauge_action_local(DIMS4, U2, BETA, c, k, rho) - \
            O.gauge_action_local(DIMS4, U, BETA, c, k, rho)
        assert abs(d_full - d_loc) < 1e-11 * max(1.0, abs(d_full))


def test_force_hermitian_traceless(c1, c1_force):
    """H = sum f^a T_a (the paper's force) is Hermitian and traceless, and the
    oracle's algebra read-back reproduces f (2 tr(T_a H) = f^a)."""
    T = H.gell_mann() / 2
    for f in c1_force.reshape(-1, 8)[::97]:
        Hm = O.algebra_to_matrix(f)
        np.testing.assert_allclose(Hm, Hm.conj().T, atol=1e-15)
        assert abs(np.trace(Hm)) < 1e-14
        np.testing.assert_allclose([2 * np.trace(T[a] @ Hm).real for a in range(8)], f, atol=1e-14)


def test_gauge_invariance_and_covariance(c1, c1_force):
    """U'_{n,mu} = g_n U g_{n+mu}^dag: S' = S and H' = g_n H g_n^dag."""
    U, c = c1
    g = O.links_from_omega(synth.gauge_parameters(DIMS4, seed=1).reshape(-1, 1, 8))[:, 0]
    U2 = O.gauge_transform(DIMS4, U, g)
    S1 = O.gauge_action(DIMS4, U, BETA, c)
    S2 = O.gauge_action(DIMS4, U2, BETA, c)
    assert abs(S2 - S1) <= 1e-13 * abs(S1)
    f2 = O.gauge_force(DIMS4, U2, BETA, c)
    H1 = _hmat(c1_force)
    H2 = _hmat(f2)
    rot = np.einsum("nij,nmjk,nlk->nmil", g, H1, g.conj())
    assert np.abs(H2 - rot).max() <= 1e-12 * np.abs(H1).max()


def test_abelian_flux_gauge_rotated(c1):
    """A random gauge rotation of the closed-form configuration keeps S."""
    dims = (4, 4, 4, 4)
    U = H.abelian_flux_links(dims, np.pi / 2, np.pi / 2)
    g = O.links_from_omega(synth.gauge_parameters(dims, seed=4).reshape(-1, 1, 8))[:, 0]
    c = O.coefficients(0.87)
    S = O.gauge_action(dims, O.gauge_transform(dims, U, g), BETA, c)
    assert abs(S - 1263.6435689327) < 1e-9 * S


def test_translation_invariance(c1, c1_force):
    U, c = c1
    shift = (1, 2, 3, 1)
    Ug = U.reshape(4, 4, 4, 4, 4, 3, 3)  # t, z, y, x, mu
    Us = np.roll(Ug, shift=(shift[3], shift[2], shift[1], shift[0]), axis=(0, 1, 2, 3)).reshape(U.shape)
    S1 = O.gauge_action(DIMS4, U, BETA, c)
    assert abs(O.gauge_action(DIMS4, Us, BETA, c) - S1) < 1e-13 * S1
    fs = O.gauge_force(DIMS4, Us, BETA, c).reshape(4, 4, 4, 4, 4, 8)
    fr = np.roll(c1_force.reshape(4, 4, 4, 4, 4, 8), shift=(shift[3], shift[2], shift[1], shift[0]),
                 axis=(0, 1, 2, 3))
    assert np.abs(fs - fr).max() < 1e-12


def test_axis_permutation_invariance(c1, c1_force):
    """Relabelling the axes x<->y (sites and link directions) maps S to S and
    the force on (n, x) to the force on (n', y)."""
    U, c = c1
    Ug = U.reshape(4, 4, 4, 4, 4, 3, 3)            # [t, z, y, x, mu]
    Up = np.swapaxes(Ug, 2, 3)[:, :, :, :, [1, 0, 2, 3]].reshape(U.shape)
    S1 = O.gauge_action(DIMS4, U, BETA, c)
    assert abs(O.gauge_action(DIMS4, Up, BETA, c) - S1) < 1e-13 * S1
    fp = O.gauge_force(DIMS4, Up, BETA, c).reshape(4, 4, 4, 4, 4, 8)
    want = np.swapaxes(c1_force.reshape(4, 4, 4, 4, 4, 8), 2, 3)[:, :, :, :, [1, 0, 2, 3]]
    assert np.abs(fp - want).max() < 1e-12


def test_complex_conjugation(c1, c1_force):
    """S(U*) = S(U); f^a(U*) = -f^a for real lambda_a, +f^a for imaginary."""
    U, c = c1
    S1 = O.gauge_action(DIMS4, U, BETA, c)
    assert abs(O.gauge_action(DIMS4, U.conj(), BETA, c) - S1) < 1e-13 * S1
    sign = np.array([-1, 1, -1, -1, 1, -1, 1, -1])
    fc = O.gauge_force(DIMS4, np.ascontiguousarray(U.conj()), BETA, c)
    assert np.abs(fc - sign * c1_force).max() < 1e-12


def test_force_linear_in_coefficients(c1):
    U, _ = c1
    parts = [O.gauge_force(DIMS4, U, BETA, e) for e in np.eye(3)]
    c = np.array([1.0, -0.07, -0.02])
    np.testing.assert_allclose(O.gauge_force(DIMS4, U, BETA, c),
                               sum(ci * p for ci, p in zip(c, parts)), atol=1e-13)


# -------------------------------------------------------------- MD steps

def test_md_link_update_is_left_exponential(c1):
    U, _ = c1
    p = synth.momenta(DIMS4, seed=9)
    dt = 0.05
    U2 = O.md_update_links(U, p, dt)
    T = H.gell_mann() / 2
    for n, mu in [(0, 0), (100, 2), (255, 3)]:
        X = 1j * dt * np.einsum("a,aij->ij", p[n, mu], T)
        np.testing.assert_allclose(U2[n, mu], sla.expm(X) @ U[n, mu], atol=1e-14)


def _gram_schmidt_by_qr(M):
    """Rows 0 and 1 of M orthonormalised in order, from LAPACK's Householder
    QR of the 3x2 matrix whose columns are those rows: M[:2].T = Q R, and with
    R's diagonal made positive real (Q -> Q D, R -> D* R, |D_ii| = 1) the
    columns of Q are the unique orthonormal pair in which row 0 is a positive
    multiple of q0 and row 1 has a positive component along q1 -- what
    Gram-Schmidt produces.  Returns [2, 3]."""
    q, r = np.linalg.qr(M[:2].T)
    d = np.diagonal(r)
    return (q * (d / np.abs(d))[None, :]).T


def _non_unitary_links(rng, n):
    """Three families of links that are not in SU(3): SU(3) matrices with row
    0 scaled and row 1 mixed with row 0, the same with row 1 scaled instead,
    and general complex Gaussian matrices."""
    base = H.random_su3_numpy(rng, n)
    a = base.copy()
    a[:, 0] *= rng.uniform(0.5, 1.5, size=(n, 1))
    a[:, 1] += (rng.normal(size=(n, 1)) + 1j * rng.normal(size=(n, 1))) * 0.3 * a[:, 0]
    b = base.copy()
    b[:, 1] *= rng.uniform(0.5, 1.5, size=(n, 1))
    b[:, 0] *= np.exp(1j * rng.uniform(0, 2 * np.pi, size=(n, 1)))
    c = rng.normal(size=(n, 3, 3)) + 1j * rng.normal(size=(n, 3, 3))
    return np.concatenate([a, b, c])


def _reunitarise(M):
    """The oracle's Gram-Schmidt alone: its link step with zero momenta
    multiplies by exp(0) = 1 (the series of the zero matrix is exactly the
    unit matrix) and reunitarises."""
    U = np.ascontiguousarray(M.reshape(-1, 1, 3, 3))
    return O.md_update_links(U, np.zeros((U.shape[0], 1, 8)), 0.3).reshape(-1, 3, 3)


def test_reunitarise_is_gram_schmidt_on_non_unitary_links():
    """The oracle's reunitarisation (after every link step; the paper fixes
    none) against the definition of Gram-Schmidt, pinned without retyping it:
    rows 0 and 1 equal LAPACK's QR factor with positive diagonal (a different
    algorithm for the same unique pair), and the result is in SU(3),
    U U^dag = 1 and det U = 1, which fixes row 2 given rows 0 and 1."""
    rng = np.random.default_rng(21)
    M = _non_unitary_links(rng, 40)
    G = _reunitarise(M)
    want = np.stack([_gram_schmidt_by_qr(m) for m in M])
    assert np.abs(G[:, :2] - want).max() < 1e-14
    eye = np.eye(3)
    assert np.abs(np.einsum("nij,nkj->nik", G, G.conj()) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(G) - 1).max() < 1e-14
    # already in SU(3): unchanged
    S = H.random_su3_numpy(rng, 8)
    assert np.abs(_reunitarise(S) - S).max() < 1e-14


def test_reunitarise_invariances():
    """Gram-Schmidt depends only on the ordered pair of subspaces
    span(r0) in span(r0, r1): scaling row 0 or row 1 by a positive number and
    adding any complex multiple of row 0 to row 1 leave the result unchanged.
    A phase e on row 0 multiplies row 0 of the result by e and row 2 by
    conj(e) (det U = 1), and leaves row 1 unchanged."""
    rng = np.random.default_rng(22)
    M = _non_unitary_links(rng, 20)
    G = _reunitarise(M)
    M2 = M.copy()
    M2[:, 0] *= 2.5
    M2[:, 1] = 0.4 * M2[:, 1] + (0.3 - 0.7j) * M2[:, 0]
    assert np.abs(_reunitarise(M2) - G).max() < 1e-13
    e = np.exp(0.9j)
    M3 = M.copy()
    M3[:, 0] *= e
    G3 = _reunitarise(M3)
    assert np.abs(G3[:, 0] - e * G[:, 0]).max() < 1e-13
    assert np.abs(G3[:, 1] - G[:, 1]).max() < 1e-13
    assert np.abs(G3[:, 2] - np.conj(e) * G[:, 2]).max() < 1e-13


def test_kinetic_energy():
    p = synth.momenta((2, 2, 2, 2), seed=4)
    assert abs(O.kinetic_energy(p) - 0.5 * np.sum(p * p)) < 1e-12


def test_leapfrog_reversible_and_second_order(c1):
    """Leapfrog built on the oracle's force: reversible to roundoff, and the
    energy violation falls as dt^2 -- which fails at once if the force had
    the wrong sign or scale (then dH would grow like dt)."""
    U, c = c1
    p = synth.momenta(DIMS4, seed=5)
    tau = 0.2
    dH = []
    for nsteps in (4, 8):
        dt = tau / nsteps
        U1, p1 = O.leapfrog(DIMS4, U, p, BETA, c, dt, nsteps)
        dH.append(O.hamiltonian(DIMS4, U1, p1, BETA, c) - O.hamiltonian(DIMS4, U, p, BETA, c))
        if nsteps == 4:
            U0, p0 = O.leapfrog(DIMS4, U1, -p1, BETA, c, dt, nsteps)
            assert np.abs(U0 - U).max() < 1e-11
            assert np.abs(-p0 - p).max() < 1e-10
    ratio = dH[0] / dH[1]
    assert 3.0 < ratio < 5.0, (dH, ratio)


def test_omelyan_reversible_and_second_order(c1):
    """The oracle's Omelyan integrator: reversible to roundoff, dH ~ dt^2, and
    smaller |dH| than leapfrog at the same step size."""
    U, c = c1
    p = synth.momenta(DIMS4, seed=5)
    tau = 0.2
    dH = []
    for nsteps in (2, 4):
        dt = tau / nsteps
        U1, p1 = O.omelyan(DIMS4, U, p, BETA, c, dt, nsteps)
        dH.append(O.hamiltonian(DIMS4, U1, p1, BETA, c) - O.hamiltonian(DIMS4, U, p, BETA, c))
        if nsteps == 2:
            U0, p0 = O.omelyan(DIMS4, U1, -p1, BETA, c, dt, nsteps)
            assert np.abs(U0 - U).max() < 1e-11
            assert np.abs(-p0 - p).max() < 1e-10
            Ul, pl = O.leapfrog(DIMS4, U, p, BETA, c, dt, nsteps)
            dH_lf = O.hamiltonian(DIMS4, Ul, pl, BETA, c) - O.hamiltonian(DIMS4, U, p, BETA, c)
            assert abs(dH[0]) < abs(dH_lf)
    ratio = dH[0] / dH[1]
    assert 3.0 < ratio < 5.0, (dH, ratio)
