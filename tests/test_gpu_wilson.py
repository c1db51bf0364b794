"""Parity of the Wilson hopping operator and the hopping-term force (Sec. III)
on the GPU, through the C ABI, with the FP64 CPU oracle.

Both sides read the same seeded links parameters and spinor normals; each
builds its links with its own exponential.

Tolerances (max over entries of |GPU - oracle| / max |oracle|):
  FP64 1e-12.  FP32 2e-5: every output entry is a sum of at most 8 (operator)
  or 24 (force) products of O(1) factors, each rounded at ~6e-8 relative, and
  the links carry their own FP32 exponential error (~1e-7); 2e-5 is ~30x the
  observed worst case, far below any algebra mistake (O(1) relative).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1808_02281_gb300 import build as B
from paper_1808_02281_gb300 import lqcd, synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-5}
KAPPA = 0.1315

CASES = [
    ((4, 4, 4, 4), 0.5),      # the 4^4 workload's spread
    ((3, 5, 4, 6), 0.4),      # ragged: V = 360, not a multiple of 32
    ((1, 2, 3, 4), 0.6),      # degenerate extents: x + mu = x and x + mu = x - mu
    ((8, 8, 8, 16), 0.3),     # 256 blocks of the force kernel
    ((6, 10, 6, 14), 0.15),   # near-unit links (the spread of the 16^3x32 workload)
    # x extent dividing 32: the operator's x hops by warp shuffles (FP32)
    ((32, 4, 2, 3), 0.4),     # one x row per warp
    ((16, 4, 4, 4), 0.4),     # two x rows per warp
]


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def _cplx(s):
    return s[..., 0] + 1j * s[..., 1]


_cache = {}


def _case(dims, sigma):
    key = (dims, sigma)
    if key not in _cache:
        omega = synth.omega(dims, sigma, 0)
        X = synth.spinor(dims, 11)
        Y = synth.spinor(dims, 12)
        U = O.links_from_omega(omega)
        _cache[key] = dict(omega=omega, X=X, Y=Y, U=U,
                           DX=O.wilson_hopping(dims, U, _cplx(X)),
                           h=O.wilson_hopping_force(dims, U, _cplx(X), _cplx(Y)))
    return _cache[key]


def _gpu(lat, c):
    U = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, c["omega"]))
    return U, lqcd.spinor_to_device(lat, c["X"]), lqcd.spinor_to_device(lat, c["Y"])


def _rel(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims,sigma", CASES)
def test_dslash_matches_oracle(dims, sigma, prec):
    c = _case(dims, sigma)
    lat = lqcd.Lattice(dims, prec)
    U, X, _ = _gpu(lat, c)
    got = lqcd.spinor_from_device(lqcd.wilson_dslash(lat, U, X, 0.0, 1.0))
    assert _rel(got, c["DX"]) <= TOL[prec]
    # D X = X - kappa calD X  (Eq. 18_7_17_2 without the clover term)
    got = lqcd.spinor_from_device(lqcd.wilson_dslash(lat, U, X, 1.0, -KAPPA))
    want = _cplx(c["X"]) - KAPPA * c["DX"]
    assert _rel(got, want) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims,sigma", CASES)
def test_hopping_force_matches_oracle(dims, sigma, prec):
    c = _case(dims, sigma)
    lat = lqcd.Lattice(dims, prec)
    U, X, Y = _gpu(lat, c)
    f = lqcd.algebra_from_device(lqcd.wilson_hopping_force(lat, U, X, Y, coef=1.0))
    assert _rel(f, c["h"]) <= TOL[prec]
    f = lqcd.algebra_from_device(lqcd.wilson_hopping_force(lat, U, X, Y, coef=-KAPPA))
    assert _rel(f, -KAPPA * c["h"]) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_hopping_force_momentum_step(prec):
    """mom += dt f fused, with and without storing f; f never touched when
    only the momenta are asked for."""
    dims, sigma = CASES[1]
    c = _case(dims, sigma)
    lat = lqcd.Lattice(dims, prec)
    U, X, Y = _gpu(lat, c)
    p0 = synth.momenta(dims, 5)
    dt = 0.037
    want = p0 + dt * KAPPA * c["h"]
    mom = lqcd.algebra_to_device(lat, p0)
    lqcd.wilson_hopping_force(lat, U, X, Y, coef=KAPPA, mom=mom, dt=dt)
    assert np.abs(lqcd.algebra_from_device(mom) - want).max() <= TOL[prec] * np.abs(want).max()
    mom = lqcd.algebra_to_device(lat, p0)
    f = torch.full(lat.algebra_shape, 7.0, dtype=lat.dtype, device="cuda")
    lqcd.wilson_hopping_force(lat, U, X, Y, coef=KAPPA, force=f, mom=mom, dt=dt)
    assert _rel(lqcd.algebra_from_device(f), KAPPA * c["h"]) <= TOL[prec]
    assert np.abs(lqcd.algebra_from_device(mom) - want).max() <= TOL[prec] * np.abs(want).max()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fermion_force_chain(prec):
    """Y = D X on the GPU, then the force with coef = kappa: the hopping part
    of -d/domega [phi^dag (D^dag D)^{-1} phi] for X = (D^dag D)^{-1} phi
    (Eqs. 18_6_24_0, 18_6_24_0_1), against the oracle's chain."""
    dims, sigma = CASES[0]
    c = _case(dims, sigma)
    lat = lqcd.Lattice(dims, prec)
    U, X, _ = _gpu(lat, c)
    Yg = lqcd.wilson_dslash(lat, U, X, 1.0, -KAPPA)
    f = lqcd.algebra_from_device(lqcd.wilson_hopping_force(lat, U, X, Yg, coef=KAPPA))
    Xo = _cplx(c["X"])
    Yo = Xo - KAPPA * c["DX"]
    want = O.wilson_hopping_force(dims, c["U"], Xo, Yo, KAPPA)
    assert _rel(f, want) <= TOL[prec]


def test_zero_spinors_give_zero():
    dims = (4, 4, 4, 4)
    lat = lqcd.Lattice(dims, "f32")
    U = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, synth.omega(dims, 0.5, 0)))
    Z = torch.zeros(lat.spinor_shape, dtype=lat.dtype, device="cuda")
    X = lqcd.spinor_to_device(lat, synth.spinor(dims, 11))
    assert float(lqcd.wilson_dslash(lat, U, Z, 1.0, -KAPPA).abs().max()) == 0.0
    assert float(lqcd.wilson_hopping_force(lat, U, X, Z).abs().max()) == 0.0
    assert float(lqcd.wilson_hopping_force(lat, U, Z, X).abs().max()) == 0.0


def _sampled_inputs(dims, sigma, sites, links):
    """Oracle-side links and spinors that hold the seeded values only where
    the sampled sites' operator and the sampled links' force read them (every
    other entry is zero and never read)."""
    V = int(np.prod(dims))
    P = H.site_coords(dims)
    L = np.array(dims)

    def idx(y):
        return int(y[0] + dims[0] * (y[1] + dims[1] * (y[2] + dims[2] * y[3])))

    need_u, need_x = set(), set()
    for n in sites:
        need_x.add(int(n))
        for mu in range(4):
            e = np.eye(4, dtype=np.int64)[mu]
            for s in (1, -1):
                m = idx((P[n] + s * e) % L)
                need_x.add(m)
                need_u.add(int(n) if s == 1 else m)
    for li in links:
        k, rho = divmod(int(li), 4)
        kp = idx((P[k] + np.eye(4, dtype=np.int64)[rho]) % L)
        need_u.add(k)
        need_x |= {k, kp}
    U = np.zeros((V, 4, 3, 3), np.complex128)
    nu = np.array(sorted(need_u))
    om = np.stack([synth.normals(0, 32, start=int(m) * 32) for m in nu]).reshape(-1, 4, 8)
    U[nu] = O.links_from_omega(sigma * om)
    X = np.zeros((V, 4, 3), np.complex128)
    Y = np.zeros((V, 4, 3), np.complex128)
    for m in sorted(need_x):
        X[m] = _cplx(synth.normals(11, 24, start=m * 24).reshape(4, 3, 2))
        Y[m] = _cplx(synth.normals(12, 24, start=m * 24).reshape(4, 3, 2))
    return U, X, Y


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_sampled_full_size(prec):
    """32^3x64, the benchmarked size and launch: 64 sampled sites of calD X
    and 64 sampled links of the force against the oracle one by one."""
    w = synth.WORKLOADS["32^3x64"]
    dims, sigma = w["dims"], w["sigma"]
    lat = lqcd.Lattice(dims, prec)
    V = lat.V
    U = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, synth.omega(dims, sigma, 0)))
    X = lqcd.spinor_to_device(lat, synth.spinor(dims, 11))
    Y = lqcd.spinor_to_device(lat, synth.spinor(dims, 12))
    sites = synth.sample_links(V, 64, seed=3)
    links = synth.sample_links(V * 4, 64, seed=2)
    DX = lqcd.wilson_dslash(lat, U, X, 0.0, 1.0)
    f = lqcd.wilson_hopping_force(lat, U, X, Y, coef=1.0)
    d_s = lqcd.spinor_from_device(DX)[sites]
    f_l = lqcd.algebra_from_device(f).reshape(-1, 8)[links]
    assert torch.isfinite(DX).all() and torch.isfinite(f).all()
    del U, X, Y, DX, f
    Uo, Xo, Yo = _sampled_inputs(dims, sigma, sites, links)
    want_d = np.stack([O.wilson_hopping_site(dims, Uo, Xo, int(n)) for n in sites])
    want_f = np.stack([O.wilson_hopping_force_link(dims, Uo, Xo, Yo, 1.0, int(li) // 4,
                                                   int(li) % 4) for li in links])
    assert _rel(d_s, want_d) <= TOL[prec]
    assert _rel(f_l, want_f) <= TOL[prec]


def _chiral_gamma5():
    """gamma_5 = gamma_x gamma_y gamma_z gamma_t of the library's chiral basis
    (the matrices the header writes out)."""
    gx = np.array([[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]])
    gy = np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]], dtype=complex)
    gz = np.array([[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]])
    gt = np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]], dtype=complex)
    return gx @ gy @ gz @ gt


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_gamma5_hermiticity_16x32(prec, tol):
    """On every site of the 16^3x32 workload: Y^dag calD X = conj(X^dag g5
    calD g5 Y) (calD^dag = g5 calD g5), with both sides from the GPU."""
    w = synth.WORKLOADS["16^3x32"]
    dims = w["dims"]
    lat = lqcd.Lattice(dims, prec)
    U = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, synth.omega(dims, w["sigma"], 0)))
    X = _cplx(synth.spinor(dims, 11))
    Y = _cplx(synth.spinor(dims, 12))
    g5 = _chiral_gamma5()
    DX = lqcd.spinor_from_device(lqcd.wilson_dslash(lat, U, lqcd.spinor_to_device(lat, X)))
    g5Y = np.einsum("ab,nbc->nac", g5, Y)
    Dg5Y = lqcd.spinor_from_device(lqcd.wilson_dslash(lat, U, lqcd.spinor_to_device(lat, g5Y)))
    lhs = np.vdot(Y, DX)
    rhs = np.conj(np.vdot(X, np.einsum("ab,nbc->nac", g5, Dg5Y)))
    scale = np.sqrt(np.vdot(Y, Y).real * np.vdot(DX, DX).real)
    assert abs(lhs - rhs) <= tol * scale


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_gauge_covariance_16x32(prec, tol):
    """16^3x32: under U -> g U g^dag (formed in numpy), X -> g X, Y -> g Y,
    calD X -> g calD X on every site and the force matrix rotates at k."""
    w = synth.WORKLOADS["16^3x32"]
    dims = w["dims"]
    lat = lqcd.Lattice(dims, prec)
    lat64 = lat.with_(precision="f64")
    U = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, synth.omega(dims, w["sigma"], 0)))
    full = lqcd.full_from_device(lqcd.unpack_links(lat, U))
    gl = lqcd.links_from_omega(lat64, lqcd.algebra_to_device(
        lat64, np.repeat(synth.gauge_parameters(dims, seed=1)[:, None, :], 4, axis=1)))
    g = lqcd.full_from_device(lqcd.unpack_links(lat64, gl))[:, 0]
    P = H.site_coords(dims)
    Ur = np.empty_like(full)
    for mu in range(4):
        sh = P.copy()
        sh[:, mu] = (sh[:, mu] + 1) % dims[mu]
        nb = sh[:, 0] + dims[0] * (sh[:, 1] + dims[1] * (sh[:, 2] + dims[2] * sh[:, 3]))
        Ur[:, mu] = g @ full[:, mu] @ np.conj(np.transpose(g[nb], (0, 2, 1)))
    U2 = lqcd.pack_links(lat, lqcd.full_to_device(lat, Ur))
    X = _cplx(synth.spinor(dims, 11))
    Y = _cplx(synth.spinor(dims, 12))
    gX = np.einsum("nab,nsb->nsa", g, X)
    gY = np.einsum("nab,nsb->nsa", g, Y)
    Xd, Yd = lqcd.spinor_to_device(lat, X), lqcd.spinor_to_device(lat, Y)
    gXd, gYd = lqcd.spinor_to_device(lat, gX), lqcd.spinor_to_device(lat, gY)
    D1 = lqcd.spinor_from_device(lqcd.wilson_dslash(lat, U, Xd))
    D2 = lqcd.spinor_from_device(lqcd.wilson_dslash(lat, U2, gXd))
    assert _rel(D2, np.einsum("nab,nsb->nsa", g, D1)) <= 4 * tol
    T = H.gell_mann() / 2
    F1 = np.einsum("nma,aij->nmij", lqcd.algebra_from_device(lqcd.wilson_hopping_force(lat, U, Xd, Yd)), T)
    F2 = np.einsum("nma,aij->nmij", lqcd.algebra_from_device(lqcd.wilson_hopping_force(lat, U2, gXd, gYd)), T)
    rot = np.einsum("nij,nmjk,nlk->nmil", g, F1, np.conj(g))
    assert np.abs(F2 - rot).max() <= 4 * tol * np.abs(F1).max()
