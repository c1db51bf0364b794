"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Both sides start from the same seeded algebra parameters omega and build
their links with their own exponential (the GPU: Cayley-Hamilton form; the
oracle: scaled Taylor series), so nothing but the seeded normals is shared.

Tolerances:
  force FP64  max_links |df| / max_links |f| <= 1e-12
  force FP32  max_links |df| / max_links |f| <= 2e-5
  action FP64 |dS| / |S| <= 1e-12
  action FP32 |dS| / |S| <= 2e-5  (per-loop FP32 trace error ~1e-6 absolute
              against loop terms 3 - Re tr P >= ~1e-2 at the smallest spread
              used, summed with random signs; the FP64 accumulation adds nothing)
  link exponential / link update: FP64 1e-13, FP32 2e-6 per entry (entries O(1))
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1808_02281_gb300 import build as B
from paper_1808_02281_gb300 import lqcd, synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL_F = {"f64": 1e-12, "f32": 2e-5}
TOL_S = {"f64": 1e-12, "f32": 2e-5}
TOL_U = {"f64": 1e-13, "f32": 2e-6}


@pytest.fixture(scope="session", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    lqcd._lib()


_cache = {}


def oracle_case(dims, sigma, u0, seed, beta=6.0):
    """Oracle links, coefficients, force and action for a seeded lattice."""
    key = (tuple(dims), sigma, u0, seed, beta)
    if key not in _cache:
        omega = synth.omega(dims, sigma, seed)
        U = O.links_from_omega(omega)
        c = O.coefficients(u0)
        _cache[key] = dict(omega=omega, U=U, c=c, f=O.gauge_force(dims, U, beta, c),
                           S=O.gauge_action(dims, U, beta, c))
    return _cache[key]


def gpu_links(lat, omega):
    return lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, omega))


def rel_force_err(f_gpu, f_ref):
    return np.abs(f_gpu - f_ref).max() / np.abs(f_ref).max()


CASES = [
    ((4, 4, 4, 4), 0.5, 0.87),       # the 4^4 workload
    ((16, 16, 16, 32), 0.15, 0.86),  # the 16^3x32 near-identity workload
    ((3, 4, 5, 6), 0.4, 0.9),        # odd extents, V = 360: ragged last block
    ((2, 3, 2, 5), 0.4, 0.87),       # extent 2: +-2 displacements coincide
    ((5, 1, 3, 2), 0.4, 0.87),       # extent 1 in one direction
    ((1, 1, 1, 1), 0.6, 0.87),       # a single site: every loop wraps onto itself
    ((8, 6, 12, 4), 0.4, 0.87),      # sweep blocks of 8x6x6: two z blocks, extents not powers of 2
    ((32, 3, 1, 3), 0.4, 0.87),      # x rows of 32: two-row CTAs pair y neighbours; 9 virtual
                                     # blocks, so the last two-row CTA has an idle group
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims,sigma,u0", CASES)
def test_links_from_omega(dims, sigma, u0, prec):
    ref = oracle_case(dims, sigma, u0, 0)
    lat = lqcd.Lattice.symanzik(dims, 6.0, u0, prec)
    U = lqcd.full_from_device(lqcd.unpack_links(lat, gpu_links(lat, ref["omega"])))
    assert np.abs(U - ref["U"]).max() < TOL_U[prec]


ALGOS = [lqcd.FORCE_PATHS, lqcd.FORCE_FACTORED, lqcd.FORCE_STAPLE_FIELDS]


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims,sigma,u0", CASES)
def test_force_parity(dims, sigma, u0, prec, algo):
    ref = oracle_case(dims, sigma, u0, 0)
    lat = lqcd.Lattice.symanzik(dims, 6.0, u0, prec, force_algo=algo)
    f = lqcd.algebra_from_device(lqcd.gauge_force(lat, gpu_links(lat, ref["omega"])))
    assert rel_force_err(f, ref["f"]) <= TOL_F[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims,sigma,u0", CASES)
def test_action_parity(dims, sigma, u0, prec):
    ref = oracle_case(dims, sigma, u0, 0)
    lat = lqcd.Lattice.symanzik(dims, 6.0, u0, prec)
    S = float(lqcd.gauge_action(lat, gpu_links(lat, ref["omega"])).item())
    assert abs(S - ref["S"]) <= TOL_S[prec] * abs(ref["S"])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_action_bitwise_reproducible(prec):
    dims = (8, 8, 8, 8)
    lat = lqcd.Lattice.symanzik(dims, 6.0, 0.87, prec)
    U = gpu_links(lat, synth.omega(dims, 0.3, 0))
    vals = {float(lqcd.gauge_action(lat, U).item()) for _ in range(3)}
    assert len(vals) == 1


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_abelian_flux_closed_form_gpu(prec):
    dims = (8, 4, 3, 5)
    th, ph = np.pi / 4, 3 * np.pi / 4
    lat = lqcd.Lattice.symanzik(dims, 6.0, 0.87, prec)
    U = lqcd.pack_links(lat, lqcd.full_to_device(lat, H.abelian_flux_links(dims, th, ph)))
    want = 6.0 / 3 * np.dot([lat.c_plaq, lat.c_rect, lat.c_cube],
                            H.abelian_flux_class_sums(lat.V, th, ph))
    S = float(lqcd.gauge_action(lat, U).item())
    assert abs(S - want) <= TOL_S[prec] * abs(want)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_unit_configuration_gpu(prec):
    dims = (3, 4, 5, 6)
    lat = lqcd.Lattice.symanzik(dims, 6.0, 0.87, prec)
    U = gpu_links(lat, np.zeros((lat.V, 4, 8)))
    assert float(lqcd.gauge_action(lat, U).item()) == 0.0
    assert not lqcd.algebra_from_device(lqcd.gauge_force(lat, U)).any()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_pack_unpack_roundtrip(prec):
    dims = (3, 4, 5, 6)
    ref = oracle_case(dims, 0.4, 0.9, 0)
    lat = lqcd.Lattice.symanzik(dims, 6.0, 0.9, prec)
    full = lqcd.full_to_device(lat, ref["U"])
    back = lqcd.full_from_device(lqcd.unpack_links(lat, lqcd.pack_links(lat, full)))
    assert np.abs(back - ref["U"]).max() < TOL_U[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_md_updates_parity(prec):
    dims = (4, 4, 4, 6)
    ref = oracle_case(dims, 0.4, 0.87, 0)
    lat = lqcd.Lattice.symanzik(dims, 6.0, 0.87, prec)
    p = synth.momenta(dims, seed=3)
    dt = 0.05
    # momentum step from the oracle's own force on both sides
    p_gpu = lqcd.algebra_to_device(lat, p)
    f_gpu = lqcd.algebra_to_device(lat, ref["f"])
    lqcd.md_update_momenta(lat, p_gpu, f_gpu, dt)
    p_ref = O.md_update_momenta(p, ref["f"], dt)
    tolp = 1e-14 if prec == "f64" else 2e-6
    assert np.abs(lqcd.algebra_from_device(p_gpu) - p_ref).max() <= tolp * np.abs(p_ref).max()
    # link step
    U_gpu = gpu_links(lat, ref["omega"])
    lqcd.md_update_links(lat, U_gpu, lqcd.algebra_to_device(lat, p), dt)
    U_ref = O.md_update_links(ref["U"], p, dt)
    assert np.abs(lqcd.full_from_device(lqcd.unpack_links(lat, U_gpu)) - U_ref).max() < 2 * TOL_U[prec]
    # kinetic energy
    K = float(lqcd.kinetic_energy(lat, lqcd.algebra_to_device(lat, p)).item())
    tolk = 1e-13 if prec == "f64" else 1e-6
    assert abs(K - O.kinetic_energy(p)) <= tolk * O.kinetic_energy(p)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims,sigma,u0", CASES)
def test_md_force_step_parity(dims, sigma, u0, prec, algo):
    """Force, fused momentum step and action from one call, against the
    oracle's force, momentum step and action."""
    ref = oracle_case(dims, sigma, u0, 0)
    lat = lqcd.Lattice.symanzik(dims, 6.0, u0, prec, force_algo=algo)
    U = gpu_links(lat, ref["omega"])
    p = synth.momenta(dims, seed=4)
    mom = lqcd.algebra_to_device(lat, p)
    force = lqcd.empty_algebra(lat)
    S = torch.empty((), dtype=torch.float64, device="cuda")
    lqcd.md_force_step(lat, U, force=force, mom=mom, dt=0.05, action=S)
    assert rel_force_err(lqcd.algebra_from_device(force), ref["f"]) <= TOL_F[prec]
    assert abs(float(S.item()) - ref["S"]) <= TOL_S[prec] * abs(ref["S"])
    p_ref = O.md_update_momenta(p, ref["f"], 0.05)
    tolp = 1e-12 if prec == "f64" else 2e-5
    assert np.abs(lqcd.algebra_from_device(mom) - p_ref).max() <= tolp * np.abs(p_ref).max()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims,sigma,u0", CASES)
def test_staple_field_variants_parity(dims, sigma, u0, prec):
    """Every schedule of the staple-field force gives the oracle's force and
    action (odd and degenerate extents included)."""
    ref = oracle_case(dims, sigma, u0, 0)
    lat = lqcd.Lattice.symanzik(dims, 6.0, u0, prec, force_algo=lqcd.FORCE_STAPLE_FIELDS)
    U = gpu_links(lat, ref["omega"])
    try:
        for v in range(lqcd.force_variant_count(lat)):
            lqcd.set_force_variant(lat, v)
            assert lqcd.get_force_variant(lat) == v
            force = lqcd.empty_algebra(lat)
            S = torch.empty((), dtype=torch.float64, device="cuda")
            lqcd.md_force_step(lat, U, force=force, action=S)
            assert rel_force_err(lqcd.algebra_from_device(force), ref["f"]) <= TOL_F[prec], v
            assert abs(float(S.item()) - ref["S"]) <= TOL_S[prec] * abs(ref["S"]), v
    finally:
        lqcd.set_force_variant(lat, -1)


def test_autotune_force():
    dims = (8, 8, 8, 16)
    lat = lqcd.Lattice.symanzik(dims, 6.0, 0.87, "f32", force_algo=lqcd.FORCE_STAPLE_FIELDS)
    U = gpu_links(lat, synth.omega(dims, 0.3, 0))
    try:
        best, ms = lqcd.autotune_force(lat, U, reps=2)
        assert 0 <= best < lqcd.force_variant_count(lat) == len(ms)
        assert all(t > 0 for t in ms) and ms[best] == min(ms)
        assert lqcd.get_force_variant(lat) == best
        with pytest.raises(lqcd.LqcdError):
            lqcd.set_force_variant(lat, len(ms))
    finally:
        lqcd.set_force_variant(lat, -1)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_staple_field_workspace_contract(prec):
    """STAPLE_FIELDS without a large enough workspace is an error; AUTO falls
    back to a workspace-free algorithm and gives the same force."""
    dims = (4, 4, 4, 6)
    lat = lqcd.Lattice.symanzik(dims, 6.0, 0.87, prec, force_algo=lqcd.FORCE_STAPLE_FIELDS)
    U = gpu_links(lat, synth.omega(dims, 0.3, 0))
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.gauge_force(lat, U, workspace=small)
    assert e.value.status == -4
    f_sf = lqcd.algebra_from_device(lqcd.gauge_force(lat, U))
    auto = lat.with_(force_algo=lqcd.FORCE_AUTO)
    f_auto_small = lqcd.algebra_from_device(lqcd.gauge_force(auto, U, workspace=small))
    assert rel_force_err(f_auto_small, f_sf) <= TOL_F[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("algo", [lqcd.FORCE_PATHS, lqcd.FORCE_FACTORED])
def test_fused_force_momentum_update(prec, algo):
    dims = (4, 6, 4, 8)
    lat = lqcd.Lattice.symanzik(dims, 6.0, 0.87, prec, force_algo=algo)
    U = gpu_links(lat, synth.omega(dims, 0.3, 0))
    p0 = lqcd.algebra_to_device(lat, synth.momenta(dims, seed=6))
    p_sep = p0.clone()
    lqcd.md_update_momenta(lat, p_sep, lqcd.gauge_force(lat, U), 0.07)
    p_fused = p0.clone()
    lqcd.gauge_force_update_momenta(lat, U, p_fused, 0.07)
    torch.testing.assert_close(p_fused, p_sep, rtol=0, atol=(1e-14 if prec == "f64" else 1e-6))


def _gauge_rotation(lat, seed):
    """g_n = exp(i v.T) built by the GPU exponential (links slot mu = 0)."""
    v = synth.gauge_parameters(lat.dims, seed)
    om = np.zeros((lat.V, 4, 8))
    om[:, 0] = v
    G = lqcd.full_from_device(lqcd.unpack_links(lat, gpu_links(lat, om)))[:, 0]
    return G


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gauge_invariance_gpu(prec):
    """16^3x32 workload: S is invariant and F covariant under a random gauge
    rotation (the rotated links are formed on the test side in numpy)."""
    w = synth.WORKLOADS["16^3x32"]
    dims = w["dims"]
    lat = lqcd.Lattice.symanzik(dims, w["beta"], w["u0"], prec)
    U = gpu_links(lat, synth.omega(dims, w["sigma"], w["seed"]))
    full = lqcd.full_from_device(lqcd.unpack_links(lat, U))
    g = _gauge_rotation(lat.with_(precision="f64"), seed=1)
    X = H.site_coords(dims)
    Ur = np.empty_like(full)
    for mu in range(4):
        shifted = X.copy()
        shifted[:, mu] = (shifted[:, mu] + 1) % dims[mu]
        nb = shifted[:, 0] + dims[0] * (shifted[:, 1] + dims[1] * (shifted[:, 2] + dims[2] * shifted[:, 3]))
        Ur[:, mu] = g @ full[:, mu] @ np.conj(np.transpose(g[nb], (0, 2, 1)))
    U2 = lqcd.pack_links(lat, lqcd.full_to_device(lat, Ur))
    S1 = float(lqcd.gauge_action(lat, U).item())
    S2 = float(lqcd.gauge_action(lat, U2).item())
    assert abs(S2 - S1) <= TOL_S[prec] * abs(S1)
    T = H.gell_mann() / 2
    F1 = np.einsum("nma,aij->nmij", lqcd.algebra_from_device(lqcd.gauge_force(lat, U)), T)
    F2 = np.einsum("nma,aij->nmij", lqcd.algebra_from_device(lqcd.gauge_force(lat, U2)), T)
    rot = np.einsum("nij,nmjk,nlk->nmil", g, F1, np.conj(g))
    assert np.abs(F2 - rot).max() <= 2 * TOL_F[prec] * np.abs(F1).max()


def _sampled_oracle(dims, sigma, u0, links, beta=6.0, seed=0):
    """Oracle force on sampled links, computed one by one from an oracle link
    field that holds exp(i omega.T) only where those links' staples reach
    (every other entry is never read)."""
    V = int(np.prod(dims))
    X = H.site_coords(dims)
    need = set()
    for li in links:
        n, rho = divmod(int(li), 4)
        x = X[n]
        for d in np.ndindex(5, 5, 5, 5):
            off = np.array(d) - 2
            if np.abs(off).sum() > 4:
                continue
            y = (x + off) % np.array(dims)
            m = y[0] + dims[0] * (y[1] + dims[1] * (y[2] + dims[2] * y[3]))
            need.add(int(m))
    need = np.array(sorted(need))
    U = np.zeros((V, 4, 3, 3), np.complex128)
    om = np.stack([synth.normals(seed, 32, start=int(m) * 32) for m in need]).reshape(-1, 4, 8)
    U[need] = O.links_from_omega(sigma * om)
    c = O.coefficients(u0)
    f = np.stack([O.gauge_force_link(dims, U, beta, c, int(li) // 4, int(li) % 4) for li in links])
    return f


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_force_sampled_full_size(prec):
    """32^3x64 (the benchmarked size) in the benchmarked launch configuration:
    sampled links against the oracle's per-link force (Eqs. 18_7_26_2/3)."""
    w = synth.WORKLOADS["32^3x64"]
    dims = w["dims"]
    lat = lqcd.Lattice.symanzik(dims, w["beta"], w["u0"], prec)
    links = synth.sample_links(lat.V * 4, 48, seed=2)
    U = gpu_links(lat, synth.omega(dims, w["sigma"], w["seed"]))
    f = lqcd.gauge_force(lat, U)
    fa = lqcd.algebra_from_device(f)
    f2 = lqcd.gauge_force(lat.with_(force_algo=lqcd.FORCE_FACTORED), U)
    fb = lqcd.algebra_from_device(f2)
    del U, f, f2
    got = fa.reshape(-1, 8)[links]
    want = _sampled_oracle(dims, w["sigma"], w["u0"], links)
    assert rel_force_err(got, want) <= TOL_F[prec]
    assert rel_force_err(fb.reshape(-1, 8)[links], want) <= TOL_F[prec]
    assert np.isfinite(fa).all()
    # every link: the two algorithms agree within twice the tolerance
    assert rel_force_err(fa, fb) <= 2 * TOL_F[prec]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_force_sampled_maximum_size(prec):
    """48^3x96 (42.5 M links, the largest workload), the staple-field force as
    the MD step uses it (full staple planes: in FP64 their offsets pass 2^31
    lanes, in FP32 the float2 region's do): sampled links against the oracle."""
    w = synth.WORKLOADS["48^3x96"]
    dims = w["dims"]
    lat = lqcd.Lattice.symanzik(dims, w["beta"], w["u0"], prec)
    links = synth.sample_links(lat.V * 4, 24, seed=2)
    U = gpu_links(lat, synth.omega(dims, w["sigma"], w["seed"]))
    fa = lqcd.algebra_from_device(lqcd.gauge_force(lat, U))
    del U
    torch.cuda.empty_cache()
    want = _sampled_oracle(dims, w["sigma"], w["u0"], links)
    assert rel_force_err(fa.reshape(-1, 8)[links], want) <= TOL_F[prec]
    assert np.isfinite(fa).all()
