"""Randomised properties of the oracle on lattices of random extents
(including the degenerate extents 1 and 2, where loops wrap onto themselves):
gauge covariance of the gauge and hopping forces, gauge invariance of the
action, and the force as the negative gradient of the action on a random
link.  CPU only."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_1808_02281_gb300 import synth  # noqa: E402
from tests import helpers as H  # noqa: E402

BETA = 6.0
T = H.gell_mann() / 2

dims_st = st.tuples(*[st.integers(min_value=1, max_value=4)] * 4)


def _gauge(dims, seed):
    return O.links_from_omega(synth.gauge_parameters(dims, seed=seed).reshape(-1, 1, 8))[:, 0]


@settings(max_examples=40, deadline=None)
@given(dims=dims_st, seed=st.integers(0, 10_000), u0=st.floats(0.8, 1.0))
def test_gauge_force_covariant_action_invariant(dims, seed, u0):
    U = O.links_from_omega(synth.omega(dims, 0.6, seed))
    c = O.coefficients(u0)
    g = _gauge(dims, seed + 1)
    Ug = O.gauge_transform(dims, U, g)
    S1, S2 = O.gauge_action(dims, U, BETA, c), O.gauge_action(dims, Ug, BETA, c)
    assert abs(S2 - S1) <= 1e-11 * max(1.0, abs(S1))
    F1 = np.einsum("nma,aij->nmij", O.gauge_force(dims, U, BETA, c), T)
    F2 = np.einsum("nma,aij->nmij", O.gauge_force(dims, Ug, BETA, c), T)
    rot = np.einsum("nij,nmjk,nlk->nmil", g, F1, g.conj())
    assert np.abs(F2 - rot).max() <= 1e-11 * max(1.0, np.abs(F1).max())


@settings(max_examples=40, deadline=None)
@given(dims=dims_st, seed=st.integers(0, 10_000))
def test_hopping_force_covariant(dims, seed):
    U = O.links_from_omega(synth.omega(dims, 0.6, seed))
    s1, s2 = synth.spinor(dims, seed + 2), synth.spinor(dims, seed + 3)
    X = s1[..., 0] + 1j * s1[..., 1]
    Y = s2[..., 0] + 1j * s2[..., 1]
    g = _gauge(dims, seed + 1)
    Ug = O.gauge_transform(dims, U, g)
    gX = np.einsum("nab,nsb->nsa", g, X)
    gY = np.einsum("nab,nsb->nsa", g, Y)
    H1 = np.einsum("nma,aij->nmij", O.wilson_hopping_force(dims, U, X, Y), T)
    H2 = np.einsum("nma,aij->nmij", O.wilson_hopping_force(dims, Ug, gX, gY), T)
    rot = np.einsum("nij,nmjk,nlk->nmil", g, H1, g.conj())
    assert np.abs(H2 - rot).max() <= 1e-11 * max(1.0, np.abs(H1).max())


@settings(max_examples=40, deadline=None)
@given(dims=dims_st, seed=st.integers(0, 10_000), pick=st.integers(0, 10**6),
       a=st.integers(0, 7))
def test_force_is_minus_gradient_on_a_random_link(dims, seed, pick, a):
    U = O.links_from_omega(synth.omega(dims, 0.6, seed))
    V = int(np.prod(dims))
    k, rho = divmod(pick % (4 * V), 4)
    c = O.coefficients(0.87)
    f = O.gauge_force_link(dims, U, BETA, c, k, rho)
    eps = 1e-4
    d = []
    for s in (1, -1):
        Up = U.copy()
        Up[k, rho] = O.exp_i_algebra(s * eps * np.eye(8)[a]) @ U[k, rho]
        d.append(O.gauge_action(dims, Up, BETA, c))
    fd = -(d[0] - d[1]) / (2 * eps)
    assert abs(fd - f[a]) <= 1e-6 * max(1.0, np.abs(f).max())
