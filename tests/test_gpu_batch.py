"""Batches of lattices of uneven extents in one persistent launch per pass:
every lattice gets exactly its single-lattice result, and batch trajectories
(eager and CUDA-graph) equal the per-lattice ones."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1808_02281_gb300 import build as B
from paper_1808_02281_gb300 import hmc, lqcd, synth

pytestmark = pytest.mark.gpu

MIXED = [(4, 4, 4, 4), (3, 4, 5, 6), (8, 4, 6, 2), (2, 3, 2, 5), (5, 1, 3, 2), (6, 6, 6, 8)]


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def _single_step(bs, c, dt):
    lat = bs.params.with_(dims=bs.dims[c])
    U = bs.links[c]
    p = bs.mom[c].clone()
    f = lqcd.empty_algebra(lat)
    S = torch.empty((), dtype=torch.float64, device="cuda")
    lqcd.md_force_step(lat, U, force=f, mom=p, dt=dt, action=S)
    return f, p, S


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batched_force_step_equals_single(prec):
    """Bit-equal to the single-lattice call under every pass-B schedule."""
    bs = hmc.initial_batch(MIXED, prec, sigma=0.4, seed=3)
    n = len(MIXED)
    try:
        for v in range(lqcd.force_variant_count(bs.params)):
            lqcd.set_force_variant(bs.params, v)
            ref = [_single_step(bs, c, 0.07) for c in range(n)]
            force = [lqcd.empty_algebra(bs.params.with_(dims=d)) for d in bs.dims]
            mom = [p.clone() for p in bs.mom]
            actions = torch.empty(n, dtype=torch.float64, device="cuda")
            lqcd.md_force_step_batched(bs.params, bs.dims, bs.links, mom=mom, dt=0.07,
                                       force=force, actions=actions, workspace=bs.workspace)
            for c in range(n):
                assert torch.equal(force[c], ref[c][0]), (v, c)
                assert torch.equal(mom[c], ref[c][1]), (v, c)
                assert float(actions[c]) == float(ref[c][2]), (v, c)
    finally:
        lqcd.set_force_variant(bs.params, -1)


def test_batched_force_matches_oracle():
    bs = hmc.initial_batch(MIXED[:3], "f64", sigma=0.4, seed=5)
    force = [lqcd.empty_algebra(bs.params.with_(dims=d)) for d in bs.dims]
    actions = torch.empty(3, dtype=torch.float64, device="cuda")
    lqcd.md_force_step_batched(bs.params, bs.dims, bs.links, force=force, actions=actions,
                               workspace=bs.workspace)
    c_ref = O.coefficients(0.87)
    for c, dims in enumerate(bs.dims):
        U = O.links_from_omega(synth.omega(dims, 0.4, 5 + 2 * c))
        f_ref = O.gauge_force(dims, U, 6.0, c_ref)
        f = lqcd.algebra_from_device(force[c])
        assert np.abs(f - f_ref).max() <= 1e-12 * np.abs(f_ref).max()
        S_ref = O.gauge_action(dims, U, 6.0, c_ref)
        assert abs(float(actions[c]) - S_ref) <= 1e-12 * abs(S_ref)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batched_link_step_equals_single(prec):
    bs = hmc.initial_batch(MIXED, prec, sigma=0.4, seed=3)
    ref = []
    for c, d in enumerate(bs.dims):
        U = bs.links[c].clone()
        lqcd.md_update_links(bs.params.with_(dims=d), U, bs.mom[c], 0.05)
        ref.append(U)
    lqcd.md_update_links_batched(bs.params, bs.dims, bs.links, bs.mom, 0.05)
    for c in range(len(MIXED)):
        assert torch.equal(bs.links[c], ref[c]), c


def test_uneven_volume_workload():
    """The uneven-volume batch (4 each of 8^4, 12^3x24, 16^3x32, 24^3x48; FP32,
    w ~ N(0, 0.3^2), Gaussian momenta): one batched force step gives every
    lattice its single-lattice result."""
    bs = hmc.initial_batch(synth.BATCH_DIMS, "f32", sigma=0.3, seed=0)
    n = len(bs.dims)
    ref = [_single_step(bs, c, 0.05) for c in range(n)]
    mom = [p.clone() for p in bs.mom]
    actions = torch.empty(n, dtype=torch.float64, device="cuda")
    lqcd.md_force_step_batched(bs.params, bs.dims, bs.links, mom=mom, dt=0.05, actions=actions,
                               workspace=bs.workspace)
    for c in range(n):
        assert torch.equal(mom[c], ref[c][1]), c
        assert float(actions[c]) == float(ref[c][2]), c


def test_batch_trajectory_graph_equals_eager_and_single():
    dims = [(8, 8, 8, 8), (6, 6, 6, 12), (4, 4, 4, 4)]
    bs = hmc.initial_batch(dims, "f32", seed=9)
    eager = bs.clone()
    hmc.batch_leapfrog(eager, 0.05, 4)
    singles = []
    for c, d in enumerate(dims):
        st = hmc.MDState.create(bs.params.with_(dims=d), bs.links[c].clone(), bs.mom[c].clone())
        hmc.leapfrog(st, 0.05, 4)
        singles.append(st)
    g = hmc.GraphBatchTrajectory(bs, 0.05, 4, "leapfrog")
    g.replay()
    torch.cuda.synchronize()
    for c in range(len(dims)):
        assert torch.equal(bs.links[c], eager.links[c])
        assert torch.equal(bs.mom[c], eager.mom[c])
        assert torch.equal(eager.links[c], singles[c].links)
        assert torch.equal(eager.mom[c], singles[c].mom)


def test_batch_hmc_equals_single_runs():
    """Lattice c of a batch HMC run equals a single-lattice run with the
    settings lattice_config(cfg, c): same dH, same decisions, same links."""
    dims_list = MIXED[:3]
    cfg = hmc.HMCConfig(tau=0.2, dt=0.05, integrator="leapfrog", seed=11)
    bs = hmc.initial_batch(dims_list, "f64", sigma=0.4, seed=3)
    singles = []
    for c, d in enumerate(bs.dims):
        lat = bs.params.with_(dims=d)
        singles.append(hmc.MDState.create(lat, bs.links[c].clone(), bs.mom[c].clone()))
    recs = [r for step in hmc.run_hmc_batch(bs, cfg, 2) for r in step]
    for c, st in enumerate(singles):
        mine = list(hmc.run_hmc(st, hmc.lattice_config(cfg, c), 2))
        theirs = [r for r in recs if r["lattice"] == c]
        for a, b in zip(mine, theirs):
            assert a["dH"] == b["dH"] and a["accepted"] == b["accepted"], (c, a, b)
        assert torch.equal(st.links, bs.links[c]), c
