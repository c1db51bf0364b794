"""The differentiable action (forward = action kernel, backward = force
kernel and the exponential's chain rule), through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1808_02281_gb300 import build as B
from paper_1808_02281_gb300 import lqcd, synth
from paper_1808_02281_gb300.autograd import symanzik_action

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def _links(lat, sigma, seed=0):
    return lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, synth.omega(lat.dims, sigma, seed)))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gradient_at_zero_is_minus_force(prec):
    lat = lqcd.Lattice.symanzik((4, 4, 4, 6), 6.0, 0.87, prec)
    U0 = _links(lat, 0.4)
    om = torch.zeros(lat.algebra_shape, dtype=lat.dtype, device="cuda", requires_grad=True)
    S = symanzik_action(om, U0, lat)
    S.backward()
    f = lqcd.gauge_force(lat, U0)
    tol = 1e-13 if prec == "f64" else 1e-6
    assert torch.allclose(om.grad, -f, rtol=0, atol=tol * float(f.abs().max()))
    # the forward re-applies Gram-Schmidt to exp(0) U0 = U0: a rounding-level change
    tol_s = 1e-12 if prec == "f64" else 2e-5
    assert abs(float(S.item()) - float(lqcd.gauge_action(lat, U0).item())) < tol_s * abs(float(S.item()))


def test_gradcheck_fp64():
    """torch.autograd.gradcheck: numerical Jacobian of the action in omega
    (central differences through the forward kernels) against the backward."""
    lat = lqcd.Lattice.symanzik((2, 2, 2, 3), 6.0, 0.87, "f64")
    U0 = _links(lat, 0.5, seed=3)
    om = lqcd.algebra_to_device(lat, synth.omega(lat.dims, 0.3, seed=4)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda w: symanzik_action(w, U0, lat), (om,), eps=1e-6,
                                    atol=1e-7, rtol=1e-6)


def test_gradient_against_oracle_finite_differences():
    """At omega != 0 (4^4, FP64): dS/domega^a from the backward equals the
    central difference of the oracle's action of exp(i (omega +- eps e_a).T) U0."""
    dims = (4, 4, 4, 4)
    lat = lqcd.Lattice.symanzik(dims, 6.0, 0.87, "f64")
    w0 = synth.omega(dims, 0.5, 0)
    w = synth.omega(dims, 0.3, 7)
    U0 = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, w0))
    om = lqcd.algebra_to_device(lat, w).requires_grad_(True)
    symanzik_action(om, U0, lat).backward()
    g = lqcd.algebra_from_device(om.grad)
    U0_ref = O.links_from_omega(w0)
    Uw = np.einsum("nmij,nmjk->nmik", O.links_from_omega(w), U0_ref)   # exp(i w.T) U0
    c = O.coefficients(0.87)
    eps = 1e-4
    worst, scale = 0.0, np.abs(g).max()
    for li in synth.sample_links(lat.V * 4, 12, seed=8):
        n, mu = divmod(int(li), 4)
        for a in range(8):
            vals = []
            for sgn in (1, -1):
                wp = w[n, mu].copy()
                wp[a] += sgn * eps
                U = Uw.copy()
                U[n, mu] = O.exp_i_algebra(wp) @ U0_ref[n, mu]
                vals.append(O.gauge_action_local(dims, U, 6.0, c, n, mu))
            fd = (vals[0] - vals[1]) / (2 * eps)
            worst = max(worst, abs(fd - g[n, mu, a]))
    assert worst <= 1e-7 * scale


def test_finite_differences_full_size():
    """32^3x64, FP32 links in compact storage: the backward (FP32 force) along
    each of the 8 generators on 4096 random links (random signs) against the
    central difference, eps = 1e-4, of the FP64 action of the same links.
    Tolerance 1e-4 |g|_2 over the sampled links: the FP32 force is within
    2e-5 max|f| per link with errors that do not line up across links, so the
    signed sum errs by ~2e-5 (max|f| / rms|f|) |g|_2; the FD truncation
    (eps^2) and FP64 rounding of S (~1e-9 / eps) are far smaller."""
    w = synth.WORKLOADS["32^3x64"]
    dims = w["dims"]
    lat32 = lqcd.Lattice.symanzik(dims, w["beta"], w["u0"], "f32")
    lat64 = lat32.with_(precision="f64")
    U32 = _links(lat32, w["sigma"], w["seed"])
    om = torch.zeros(lat32.algebra_shape, dtype=torch.float32, device="cuda", requires_grad=True)
    symanzik_action(om, U32, lat32).backward()
    g = lqcd.algebra_from_device(om.grad)          # [V, 4, 8], = -force (FP32)
    # the same links in FP64 (exact promotion of the stored FP32 values)
    U64 = lqcd.pack_links(lat64, lqcd.unpack_links(lat32, U32).double())
    del U32
    links = synth.sample_links(lat32.V * 4, 4096, seed=2)
    signs = np.where(synth.words(11, 0, len(links)) & np.uint64(1), 1.0, -1.0)
    eps = 1e-4
    V = lat32.V
    for a in range(8):
        v = np.zeros((V, 4, 8))
        v.reshape(-1, 8)[links, a] = signs
        vd = lqcd.algebra_to_device(lat64, v)
        S = []
        for sgn in (1.0, -1.0):
            U = U64.clone()
            lqcd.md_update_links(lat64, U, vd, sgn * eps)
            S.append(float(lqcd.gauge_action(lat64, U).item()))
            del U
        fd = (S[0] - S[1]) / (2 * eps)
        want = float(np.sum(g.reshape(-1, 8)[links, a] * signs))
        scale = float(np.sqrt(np.sum(g.reshape(-1, 8)[links, a] ** 2)))
        assert abs(fd - want) <= 1e-4 * scale, (a, fd, want, scale)
