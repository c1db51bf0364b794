"""Pins of the oracle's Wilson fermion part (Sec. III: the hopping operator
calD of Eq. 18_7_17_4 and the hopping-term force of Eqs. 18_1_29_19 to
18_7_17_30) against what the mathematics fixes, on the CPU.  A wrong sign of
a gamma matrix, a dropped complex conjugate, a transposed outer product, a
missing dagger or a wrong neighbour fails at least one of them."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1808_02281_gb300 import synth
from tests import helpers as H

DIMS = (4, 4, 4, 4)
V = 256


def _spinor(dims, seed):
    s = synth.spinor(dims, seed)
    return s[..., 0] + 1j * s[..., 1]


@pytest.fixture(scope="module")
def cfg():
    U = O.links_from_omega(synth.omega(DIMS, 0.5, 0))
    X = _spinor(DIMS, 11)
    Y = _spinor(DIMS, 12)
    return U, X, Y


def _unit_links(V):
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def test_gamma_clifford_algebra():
    """Hermitian, gamma_mu gamma_nu + gamma_nu gamma_mu = 2 delta, gamma_5
    Hermitian, squares to 1 and anticommutes with every gamma_mu."""
    g = [O.gamma(m) for m in range(1, 6)]
    one = np.eye(4)
    for a in range(5):
        np.testing.assert_array_equal(g[a], g[a].conj().T)
    for a in range(4):
        for b in range(4):
            np.testing.assert_allclose(g[a] @ g[b] + g[b] @ g[a], 2 * one * (a == b), atol=0)
        np.testing.assert_allclose(g[4] @ g[a] + g[a] @ g[4], 0, atol=0)
    np.testing.assert_allclose(g[4] @ g[4], one, atol=0)
    np.testing.assert_allclose(g[4], g[0] @ g[1] @ g[2] @ g[3], atol=0)


@pytest.mark.parametrize("k", [(1, 0, 0, 0), (0, 2, 1, 3), (1, 1, 1, 1), (3, 0, 2, 1)])
def test_free_field_plane_wave(k):
    """Unit links, X_n = exp(i p.n) u:  calD X = sum_mu [2 cos p_mu - 2 i
    sin p_mu gamma_mu] X  (forward (1 - gamma) e^{i p}, backward (1 + gamma)
    e^{-i p})."""
    dims = (4, 4, 6, 4)
    Vd = int(np.prod(dims))
    p = 2 * np.pi * np.array(k) / np.array(dims)
    pos = H.site_coords(dims)
    phase = np.exp(1j * pos @ p)
    rng = np.random.default_rng(5)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    X = phase[:, None, None] * u[None]
    got = O.wilson_hopping(dims, _unit_links(Vd), X)
    M = sum(2 * np.cos(p[m]) * np.eye(4) - 2j * np.sin(p[m]) * O.gamma(m + 1) for m in range(4))
    want = phase[:, None, None] * (M @ u)[None]
    assert np.abs(got - want).max() < 1e-13


def test_gamma5_hermiticity(cfg):
    """calD^dag = gamma_5 calD gamma_5:  Y^dag calD X = conj(X^dag g5 calD g5 Y)."""
    U, X, Y = cfg
    g5 = O.gamma(5)
    lhs = np.vdot(Y, O.wilson_hopping(DIMS, U, X))
    t = O.wilson_hopping(DIMS, U, np.einsum("ab,nbc->nac", g5, Y))
    rhs = np.conj(np.vdot(X, np.einsum("ab,nbc->nac", g5, t)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_hopping_gauge_covariant(cfg):
    """calD[U^g] (g X) = g calD[U] X  for U^g_{n,mu} = g_n U g_{n+mu}^dag."""
    U, X, _ = cfg
    g = O.links_from_omega(synth.gauge_parameters(DIMS, seed=1).reshape(-1, 1, 8))[:, 0]
    Ug = O.gauge_transform(DIMS, U, g)
    gX = np.einsum("nab,nsb->nsa", g, X)
    lhs = O.wilson_hopping(DIMS, Ug, gX)
    rhs = np.einsum("nab,nsb->nsa", g, O.wilson_hopping(DIMS, U, X))
    assert np.abs(lhs - rhs).max() < 1e-12


def test_hopping_neighbours_by_brute_force():
    """calD on a spinor supported on one site reaches exactly its 8
    neighbours, with (1 + gamma_mu) U_{m,mu}^dag ... at m = n - mu:
    (calD X)_{n-mu} carries (1 - gamma_mu) U_{n-mu,mu} X_n and
    (calD X)_{n+mu} carries (1 + gamma_mu) U_{n,mu}^dag X_n."""
    U = O.links_from_omega(synth.omega(DIMS, 0.7, 3))
    X = np.zeros((V, 4, 3), dtype=np.complex128)
    n = 1 + 4 * (2 + 4 * (3 + 4 * 1))
    X[n] = _spinor((1, 1, 1, 1), 7)[0]
    out = O.wilson_hopping(DIMS, U, X)
    coords = H.coords(DIMS, n)
    touched = set()
    for mu in range(4):
        g = O.gamma(mu + 1)
        fw = list(coords)
        fw[mu] = (fw[mu] - 1) % DIMS[mu]
        m = fw[0] + 4 * (fw[1] + 4 * (fw[2] + 4 * fw[3]))
        want = (np.eye(4) - g) @ (X[n] @ U[m, mu].T)
        np.testing.assert_allclose(out[m], want, atol=1e-14)
        bw = list(coords)
        bw[mu] = (bw[mu] + 1) % DIMS[mu]
        m2 = bw[0] + 4 * (bw[1] + 4 * (bw[2] + 4 * bw[3]))
        want = (np.eye(4) + g) @ (X[n] @ U[n, mu].conj())
        np.testing.assert_allclose(out[m2], want, atol=1e-14)
        touched |= {m, m2}
    rest = [i for i in range(V) if i not in touched]
    assert np.abs(out[rest]).max() == 0.0


def _phi(U, X, Y):
    """2 Re Y^dag calD X."""
    return 2.0 * np.vdot(Y, O.wilson_hopping(DIMS, U, X)).real


def test_hopping_force_is_minus_the_gradient(cfg):
    """h^i_{k,rho} = -d/deps 2 Re Y^dag calD[exp(i eps T_i) U_{k,rho}] X at 0
    (the left Lie derivative), by central differences on 96 links x 8."""
    U, X, Y = cfg
    h = O.wilson_hopping_force(DIMS, U, X, Y)
    eps = 1e-5
    links = synth.sample_links(V * 4, 96, seed=2)
    worst = 0.0
    for li in links:
        k, rho = divmod(int(li), 4)
        for a in range(8):
            d = []
            for s in (1, -1):
                Up = U.copy()
                Up[k, rho] = O.exp_i_algebra(s * eps * np.eye(8)[a]) @ U[k, rho]
                d.append(_phi(Up, X, Y))
            fd = -(d[0] - d[1]) / (2 * eps)
            worst = max(worst, abs(fd - h[k, rho, a]))
    assert worst < 1e-8 * np.abs(h).max(), worst


def test_hopping_force_link_and_scale(cfg):
    """The one-link and one-site forms equal the whole-lattice ones; coef
    scales the force."""
    U, X, Y = cfg
    D = O.wilson_hopping(DIMS, U, X)
    for n in (0, 37, 255):
        np.testing.assert_array_equal(O.wilson_hopping_site(DIMS, U, X, n), D[n])
    h = O.wilson_hopping_force(DIMS, U, X, Y)
    for li in synth.sample_links(V * 4, 16, seed=9):
        k, rho = divmod(int(li), 4)
        np.testing.assert_array_equal(O.wilson_hopping_force_link(DIMS, U, X, Y, 1.0, k, rho),
                                      h[k, rho])
    np.testing.assert_allclose(O.wilson_hopping_force(DIMS, U, X, Y, -0.125), -0.125 * h,
                               rtol=1e-15, atol=0)


def test_hopping_force_gauge_covariant(cfg):
    """Under U -> U^g, X -> g X, Y -> g Y the force matrix rotates at k:
    H'_{k,rho} = g_k H_{k,rho} g_k^dag (B and C both rotate that way)."""
    U, X, Y = cfg
    g = O.links_from_omega(synth.gauge_parameters(DIMS, seed=6).reshape(-1, 1, 8))[:, 0]
    Ug = O.gauge_transform(DIMS, U, g)
    gX = np.einsum("nab,nsb->nsa", g, X)
    gY = np.einsum("nab,nsb->nsa", g, Y)
    T = H.gell_mann() / 2
    H1 = np.einsum("nma,aij->nmij", O.wilson_hopping_force(DIMS, U, X, Y), T)
    H2 = np.einsum("nma,aij->nmij", O.wilson_hopping_force(DIMS, Ug, gX, gY), T)
    rot = np.einsum("nij,nmjk,nlk->nmil", g, H1, g.conj())
    assert np.abs(H2 - rot).max() < 1e-12 * np.abs(H1).max()


def test_hopping_force_swaps_under_adjoint(cfg):
    """Swapping X and Y conjugates Y^dag calD X into X^dag calD Y, whose real
    part equals Re Y^dag calD^dag X = Re Y^dag g5 calD g5 X: the force of
    (Y, X) equals the force of (g5 X, g5 Y)."""
    U, X, Y = cfg
    g5 = O.gamma(5)
    a = O.wilson_hopping_force(DIMS, U, Y, X)
    b = O.wilson_hopping_force(DIMS, U, np.einsum("ab,nbc->nac", g5, X),
                               np.einsum("ab,nbc->nac", g5, Y))
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_fermion_action_derivative_chain():
    """Eq. 18_6_24_0 end to end on a 3x2x2x2 lattice (288 unknowns):
    S_F(U) = phi^dag (D^dag D)^{-1} phi with D = 1 - kappa calD built densely
    from the oracle's calD, phi fixed.  At X = (D^dag D)^{-1} phi, Y = D X,
    -dS_F/domega^i_{k,rho} (central differences of a direct solve) equals
    kappa h^i(X, Y): the hopping force with coef = kappa."""
    dims = (3, 2, 2, 2)
    Vd = int(np.prod(dims))
    kappa = 0.12
    U0 = O.links_from_omega(synth.omega(dims, 0.6, 21))

    def dmat(U):
        n = Vd * 12
        cols = []
        for j in range(n):
            e = np.zeros(n, dtype=np.complex128)
            e[j] = 1.0
            cols.append(e - kappa * O.wilson_hopping(dims, U, e.reshape(Vd, 4, 3)).ravel())
        return np.stack(cols, axis=1)

    D0 = dmat(U0)
    X = _spinor(dims, 31)
    phi = D0.conj().T @ (D0 @ X.ravel())
    Y = (D0 @ X.ravel()).reshape(Vd, 4, 3)
    h = O.wilson_hopping_force(dims, U0, X, Y, kappa)

    def s_f(U):
        D = dmat(U)
        return np.vdot(phi, np.linalg.solve(D.conj().T @ D, phi)).real

    eps = 1e-5
    worst = 0.0
    for k, rho in [(0, 0), (5, 3), (17, 1), (23, 2)]:
        for a in range(8):
            d = []
            for sgn in (1, -1):
                U = U0.copy()
                U[k, rho] = O.exp_i_algebra(sgn * eps * np.eye(8)[a]) @ U0[k, rho]
                d.append(s_f(U))
            fd = -(d[0] - d[1]) / (2 * eps)
            worst = max(worst, abs(fd - h[k, rho, a]))
    assert worst < 1e-6 * np.abs(h).max(), worst
