"""MD trajectories on the GPU (leapfrog, Omelyan; FP32 and FP64; eager and
CUDA-graph) against the oracle's integrators and the integrators' own
invariants."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1808_02281_gb300 import build as B
from paper_1808_02281_gb300 import hmc, lqcd, synth

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def _state(prec, sigma=0.5, seed=0):
    return hmc.initial_state(DIMS, prec, sigma=sigma, u0=0.87, seed=seed)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 5e-5)])
@pytest.mark.parametrize("integrator", ["leapfrog", "omelyan"])
def test_trajectory_matches_oracle(prec, tol, integrator):
    st = _state(prec)
    w = synth.omega(DIMS, 0.5, 0)
    p = synth.momenta(DIMS, 1)
    U_ref, p_ref = O.links_from_omega(w), p
    c = O.coefficients(0.87)
    dt, n = 0.05, 3
    getattr(hmc, integrator)(st, dt, n)
    U_ref, p_ref = getattr(O, integrator)(DIMS, U_ref, p_ref, 6.0, c, dt, n)
    U = lqcd.full_from_device(lqcd.unpack_links(st.lat, st.links))
    pg = lqcd.algebra_from_device(st.mom)
    assert np.abs(U - U_ref).max() < tol
    assert np.abs(pg - p_ref).max() < tol * max(1.0, np.abs(p_ref).max())


@pytest.mark.parametrize("integrator", ["leapfrog", "omelyan"])
def test_reversibility_fp64(integrator):
    st = _state("f64")
    U0, p0 = st.links.clone(), st.mom.clone()
    run = hmc.INTEGRATORS[integrator]
    run(st, 0.05, 6)
    st.mom.neg_()
    run(st, 0.05, 6)
    st.mom.neg_()
    assert float((st.links - U0).abs().max()) < 1e-11
    assert float((st.mom - p0).abs().max()) < 1e-10


@pytest.mark.parametrize("integrator", ["leapfrog", "omelyan"])
def test_energy_violation_second_order(integrator):
    """dH ~ dt^2 (ratio 4 when dt halves) in FP64; matches the oracle's dH."""
    tau = 0.4
    dH = []
    for n in (4, 8):
        st = _state("f64")
        dH.append(hmc.trajectory(st, tau, tau / n, integrator))
    assert 3.0 < dH[0] / dH[1] < 5.0, dH
    w = synth.omega(DIMS, 0.5, 0)
    p = synth.momenta(DIMS, 1)
    U = O.links_from_omega(w)
    c = O.coefficients(0.87)
    U1, p1 = getattr(O, integrator)(DIMS, U, p, 6.0, c, tau / 8, 8)
    dH_ref = O.hamiltonian(DIMS, U1, p1, 6.0, c) - O.hamiltonian(DIMS, U, p, 6.0, c)
    assert abs(dH[1] - dH_ref) < 1e-9 * max(1.0, abs(O.hamiltonian(DIMS, U, p, 6.0, c)))


def test_fp32_dh_close_to_fp64():
    """The FP32 trajectory's dH, with the action of its FP32-stored links
    evaluated in FP64, tracks the FP64 trajectory's dH."""
    dims = (8, 8, 8, 8)
    out = {}
    for prec in ("f32", "f64"):
        st = hmc.initial_state(dims, prec, sigma=0.3, seed=2)
        out[prec] = hmc.trajectory(st, 0.5, 0.05, "omelyan", action_precision="f64")
    assert abs(out["f32"] - out["f64"]) < 2e-2 * max(1.0, abs(out["f64"])), out


def test_cuda_graph_replay_equals_eager():
    st = _state("f32", seed=4)
    eager = st.clone()
    hmc.omelyan(eager, 0.05, 5)
    g = hmc.GraphTrajectory(st, 0.05, 5, "omelyan")
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(st.links, eager.links)
    assert torch.equal(st.mom, eager.mom)


def test_convert_roundtrip():
    lat = lqcd.Lattice.symanzik(DIMS, 6.0, 0.87, "f32")
    U = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, synth.omega(DIMS, 0.5, 0)))
    U64 = lqcd.convert_links(lat, U, "f64")
    back = lqcd.convert_links(lat.with_(precision="f64"), U64, "f32")
    assert torch.equal(back, U)
    full32 = lqcd.unpack_links(lat, U).double()
    full64 = lqcd.unpack_links(lat.with_(precision="f64"), U64)
    assert float((full64[..., :2, :, :] - full32[..., :2, :, :]).abs().max()) == 0.0
    p = lqcd.algebra_to_device(lat, synth.momenta(DIMS, 3))
    p64 = lqcd.convert_algebra(lat, p, "f64")
    np.testing.assert_array_equal(lqcd.algebra_from_device(p64), lqcd.algebra_from_device(p))


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 1e-6)])
def test_gaussian_momenta_match_the_generator(prec, tol):
    """The GPU draws are the generator's: synth.momenta(dims, seed), the same
    SplitMix64 + Box-Muller definition evaluated in numpy (libm ulps apart)."""
    dims = (3, 5, 4, 6)
    lat = lqcd.Lattice(dims, prec)
    for seed in (0, 12345, 2**63 + 11):
        got = lqcd.algebra_from_device(lqcd.gaussian_momenta(lat, seed))
        want = synth.momenta(dims, seed % 2**64)
        assert np.abs(got - want).max() <= tol * max(1.0, np.abs(want).max())
    big = lqcd.algebra_from_device(lqcd.gaussian_momenta(lqcd.Lattice((16, 16, 16, 32), prec), 7))
    assert abs(big.mean()) < 3e-3 and abs(big.var() - 1.0) < 3e-3


def test_plaquette_against_oracle():
    st = _state("f64")
    U = O.links_from_omega(synth.omega(DIMS, 0.5, 0))
    sums = O.loop_sums(DIMS, U)
    want = 1.0 - sums[0] / (18.0 * 256)
    assert abs(hmc.plaquette(st) - want) < 1e-13
    unit = hmc.initial_state(DIMS, "f64", sigma=0.0)
    assert hmc.plaquette(unit) == 1.0


def test_metropolis_branches(monkeypatch):
    """Rejection restores the links bit for bit; acceptance keeps the
    integrated ones; the momenta are refreshed from the trajectory's stream."""
    cfg = hmc.HMCConfig(tau=0.2, dt=0.05, integrator="leapfrog", seed=9)
    st = _state("f64")
    U0 = st.links.clone()
    monkeypatch.setattr(hmc, "metropolis_uniform", lambda cfg, t: 1.0)
    rec = hmc.hmc_trajectory(st, cfg, 0)
    assert not rec["accepted"] and torch.equal(st.links, U0)
    monkeypatch.setattr(hmc, "metropolis_uniform", lambda cfg, t: 0.0)
    rec = hmc.hmc_trajectory(st, cfg, 0)
    assert rec["accepted"] and not torch.equal(st.links, U0)
    # the trajectory started from the refreshed momenta of stream word 0
    st2 = _state("f64")
    lqcd.gaussian_momenta(st2.lat, hmc.momentum_seed(cfg, 0), out=st2.mom)
    hmc.leapfrog(st2, 0.05, 4)
    assert torch.equal(st2.links, st.links)


def test_resume_from_checkpoint_is_bitwise(tmp_path):
    cfg = hmc.HMCConfig(tau=0.2, dt=0.05, integrator="omelyan", seed=3)
    st = _state("f64")
    full = list(hmc.run_hmc(st, cfg, 4))
    path = str(tmp_path / "run.ckpt")
    st2 = _state("f64")
    first = list(hmc.run_hmc(st2, cfg, 2, checkpoint=path))
    st3, cfg3, start = hmc.load_checkpoint(path)
    assert start == 2 and cfg3 == cfg
    rest = list(hmc.run_hmc(st3, cfg3, 2, start=start))
    assert torch.equal(st3.links, st.links) and torch.equal(st3.mom, st.mom)
    for a, b in zip(full, first + rest):
        assert a["dH"] == b["dH"] and a["accepted"] == b["accepted"] and a["action"] == b["action"]
    assert sum(r["accepted"] for r in full) >= 3    # small dt: nearly every trajectory accepted


def _perturbed(lat, U, scale0=1.0, mix=0.0):
    """The stored rows changed on the host: row 0 scaled, row 1 += mix * row 0."""
    full = lqcd.unpack_links(lat, U).clone()
    full[..., 0, :, :] *= scale0
    full[..., 1, :, :] += mix * full[..., 0, :, :]
    return lqcd.pack_links(lat, full)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-14), ("f32", 1e-6)])
def test_unitarity_deviation_closed_forms(prec, tol):
    st = _state(prec)
    lat = st.lat
    assert float(lqcd.unitarity_deviation(lat, st.links).item()) < tol
    s = 1.0 + 3e-3
    got = float(lqcd.unitarity_deviation(lat, _perturbed(lat, st.links, scale0=s)).item())
    assert abs(got - (s * s - 1.0)) < 10 * tol
    d = 2e-3
    got = float(lqcd.unitarity_deviation(lat, _perturbed(lat, st.links, mix=d)).item())
    assert abs(got - d) < 10 * tol


def test_reunitarise_matches_oracle_gram_schmidt():
    """FP64: the GPU's FP64 Gram-Schmidt of perturbed links equals the
    oracle's (its link step with zero momenta is exp(0) U, reunitarised)."""
    st = _state("f64")
    lat = st.lat
    P = _perturbed(lat, st.links, scale0=1.01, mix=0.02)
    full = lqcd.full_from_device(lqcd.unpack_links(lat, P))
    want = O.md_update_links(full, np.zeros((256, 4, 8)), 0.0)
    lqcd.reunitarise_links(lat, P)
    got = lqcd.full_from_device(lqcd.unpack_links(lat, P))
    assert np.abs(got - want).max() < 1e-14
    assert float(lqcd.unitarity_deviation(lat, P).item()) < 1e-14


def test_reunitarise_fp32_links_in_fp64():
    st = _state("f32")
    P = _perturbed(st.lat, st.links, scale0=1.01, mix=0.02)
    assert float(lqcd.unitarity_deviation(st.lat, P).item()) > 1e-2
    lqcd.reunitarise_links(st.lat, P)
    assert float(lqcd.unitarity_deviation(st.lat, P).item()) < 1e-6


def test_fp32_link_step_leaves_row_norms_unbiased():
    """The FP32 link step's Gram-Schmidt leaves no systematic departure of
    the stored row norms from 1: over a million rows the mean of |r|^2 - 1
    is below 2e-9 (rounding alone spreads single rows by ~5e-8; normalising
    with the factor 1/|r| rounded next to 1 gave a mean of +5e-8, an action
    offset of ~1e-7 relative that shows up as a constant FP32 - FP64 dH)."""
    dims = (16, 16, 16, 16)
    lat = lqcd.Lattice(dims, "f32")
    U = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, synth.omega(dims, 0.3, 3)))
    p = lqcd.algebra_to_device(lat, synth.momenta(dims, seed=4))
    for _ in range(3):
        lqcd.md_update_links(lat, U, p, 0.05)
    full = lqcd.full_from_device(lqcd.unpack_links(lat, U))
    for row in (0, 1):
        d = (np.abs(full[..., row, :]) ** 2).sum(-1) - 1.0
        assert np.abs(d).max() < 1e-6
        assert abs(d.mean()) < 2e-9, (row, d.mean(), d.std())


def test_same_start_study_small():
    """The same-start comparison on a small lattice: both runs start from the
    same Hamiltonian value, the FP32 error of dH is far below dH itself, and
    halving dt shrinks |dH| (same momenta for every dt)."""
    recs = list(hmc.same_start_study((8, 8, 8, 8), 0.5, [0.1, 0.05], "omelyan", seed=1, n_therm=4,
                                     therm_tau=0.3, therm_dt=0.05))
    therm = [r for r in recs if r["phase"] == "thermalise"]
    study = [r for r in recs if r["phase"] == "study"]
    assert len(therm) == 4 and len(study) == 2
    assert all(r["H0_equal"] for r in study)
    for r in study:
        assert r["abs_diff"] < 1e-3 * max(1.0, abs(r["dH_f64"])), r
    assert abs(study[1]["dH_f64"]) < abs(study[0]["dH_f64"])
