"""No entry point writes outside its buffers: every output, in-place buffer
and workspace is a view into a larger allocation whose margins hold a
sentinel, and the margins must be unchanged after the call (ragged and
regular lattices, both precisions, every force schedule, batches, Wilson
kernels).  Inputs are checked unchanged as well."""
import numpy as np
import pytest
import torch

from paper_1808_02281_gb300 import build as B
from paper_1808_02281_gb300 import lqcd, synth

pytestmark = pytest.mark.gpu

PAD_BYTES = 4096          # keeps the 256-byte alignment of workspaces
SENTINEL = -1.2345e30


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


class Padded:
    """A tensor of `shape` inside a sentinel-filled allocation."""

    def __init__(self, shape, dtype, fill=None):
        n = int(np.prod(shape))
        esize = torch.empty((), dtype=dtype).element_size()
        self.pad = PAD_BYTES // esize
        self.base = torch.empty(n + 2 * self.pad, dtype=dtype, device="cuda")
        if dtype == torch.uint8:
            self.base.fill_(0xA5)
        else:
            self.base.fill_(SENTINEL)
        self.view = self.base[self.pad:self.pad + n].view(shape)
        if fill is not None:
            self.view.copy_(fill)
        self.n = n

    def margins_intact(self):
        want = 0xA5 if self.base.dtype == torch.uint8 else SENTINEL
        lo = self.base[:self.pad]
        hi = self.base[self.pad + self.n:]
        return bool((lo == want).all()) and bool((hi == want).all())


def _lattice(dims, prec):
    w = synth.WORKLOADS["4^4"]
    lat = lqcd.Lattice.symanzik(dims, w["beta"], w["u0"], prec)
    omega = lqcd.algebra_to_device(lat, synth.omega(dims, 0.4, 0))
    return lat, omega


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("dims", [(3, 5, 4, 6), (8, 8, 8, 16)])
def test_gauge_entry_points_stay_in_bounds(dims, prec):
    lat, omega = _lattice(dims, prec)
    U = Padded(lat.link_shape, lat.dtype)
    lqcd.links_from_omega(lat, omega, out=U.view)
    assert U.margins_intact()
    links = U.view.clone()
    mom0 = lqcd.algebra_to_device(lat, synth.momenta(dims, 1))
    ws = Padded((lqcd.workspace_bytes(lat),), torch.uint8)
    for v in range(lqcd.force_variant_count(lat)):
        lqcd.set_force_variant(lat, v)
        try:
            f = Padded(lat.algebra_shape, lat.dtype)
            m = Padded(lat.algebra_shape, lat.dtype, fill=mom0)
            S = Padded((), torch.float64)
            lqcd.md_force_step(lat, links, force=f.view, mom=m.view, dt=0.03, action=S.view,
                               workspace=ws.view)
            torch.cuda.synchronize()
            assert f.margins_intact() and m.margins_intact() and S.margins_intact(), v
            assert ws.margins_intact(), v
        finally:
            lqcd.set_force_variant(lat, -1)
    assert torch.equal(links, U.view)
    for algo in (lqcd.FORCE_PATHS, lqcd.FORCE_FACTORED):
        f = Padded(lat.algebra_shape, lat.dtype)
        lqcd.gauge_force(lat.with_(force_algo=algo), links, out=f.view)
        assert f.margins_intact(), algo
    S = Padded((), torch.float64)
    lqcd.gauge_action(lat, links, out=S.view, workspace=ws.view)
    assert S.margins_intact() and ws.margins_intact()
    K = Padded((), torch.float64)
    lqcd.kinetic_energy(lat, mom0, out=K.view, workspace=ws.view)
    assert K.margins_intact() and ws.margins_intact()
    m = Padded(lat.algebra_shape, lat.dtype, fill=mom0)
    f0 = lqcd.gauge_force(lat, links)
    lqcd.md_update_momenta(lat, m.view, f0, 0.02)
    assert m.margins_intact()
    u = Padded(lat.link_shape, lat.dtype, fill=links)
    lqcd.md_update_links(lat, u.view, mom0, 0.02)
    assert u.margins_intact()
    lqcd.reunitarise_links(lat, u.view)
    assert u.margins_intact()
    dev = Padded((), torch.float64)
    lqcd.unitarity_deviation(lat, links, out=dev.view, workspace=ws.view)
    assert dev.margins_intact() and ws.margins_intact()
    m2 = Padded(lat.algebra_shape, lat.dtype)
    lqcd.gaussian_momenta(lat, 5, out=m2.view)
    assert m2.margins_intact()
    g = Padded(lat.algebra_shape, lat.dtype)
    lqcd.omega_gradient(lat, omega, f0, out=g.view)
    assert g.margins_intact()
    other = "f64" if prec == "f32" else "f32"
    lat2 = lat.with_(precision=other)
    c = Padded(lat2.link_shape, lat2.dtype)
    lqcd.convert_links(lat, links, other, out=c.view)
    assert c.margins_intact()
    c = Padded(lat2.algebra_shape, lat2.dtype)
    lqcd.convert_algebra(lat, mom0, other, out=c.view)
    assert c.margins_intact()
    full = Padded((lat.V, 4, 3, 3, 2), lat.dtype)
    lqcd.unpack_links(lat, links, out=full.view)
    assert full.margins_intact()
    back = Padded(lat.link_shape, lat.dtype)
    lqcd.pack_links(lat, full.view, out=back.view)
    assert back.margins_intact()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_wilson_entry_points_stay_in_bounds(prec):
    dims = (3, 5, 4, 6)
    lat, omega = _lattice(dims, prec)
    links = lqcd.links_from_omega(lat, omega)
    X = lqcd.spinor_to_device(lat, synth.spinor(dims, 11))
    X0 = X.clone()
    y = Padded(lat.spinor_shape, lat.dtype)
    lqcd.wilson_dslash(lat, links, X, 1.0, -0.13, out=y.view)
    assert y.margins_intact()
    f = Padded(lat.algebra_shape, lat.dtype)
    m = Padded(lat.algebra_shape, lat.dtype, fill=torch.zeros(lat.algebra_shape, dtype=lat.dtype))
    lqcd.wilson_hopping_force(lat, links, X, y.view, coef=0.13, force=f.view, mom=m.view, dt=0.1)
    assert f.margins_intact() and m.margins_intact()
    assert torch.equal(X, X0)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batched_entry_points_stay_in_bounds(prec):
    dims_list = [(3, 5, 4, 6), (4, 4, 4, 4), (2, 3, 2, 5)]
    params = lqcd.Lattice.symanzik(dims_list[0], 6.0, 0.87, prec)
    links, moms, forces, ups = [], [], [], []
    for c, d in enumerate(dims_list):
        lat = params.with_(dims=d)
        links.append(lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, synth.omega(d, 0.4, c))))
        moms.append(Padded(lat.algebra_shape, lat.dtype,
                           fill=lqcd.algebra_to_device(lat, synth.momenta(d, 10 + c))))
        forces.append(Padded(lat.algebra_shape, lat.dtype))
        ups.append(Padded(lat.link_shape, lat.dtype, fill=links[c]))
    ws = Padded((lqcd.workspace_bytes_batched(params, dims_list),), torch.uint8)
    acts = Padded((len(dims_list),), torch.float64)
    for v in range(lqcd.force_variant_count(params)):
        lqcd.set_force_variant(params, v)
        try:
            lqcd.md_force_step_batched(params, dims_list, links, mom=[m.view for m in moms],
                                       dt=0.01, force=[f.view for f in forces],
                                       actions=acts.view, workspace=ws.view)
            torch.cuda.synchronize()
            assert ws.margins_intact() and acts.margins_intact(), v
            assert all(m.margins_intact() for m in moms), v
            assert all(f.margins_intact() for f in forces), v
        finally:
            lqcd.set_force_variant(params, -1)
    lqcd.md_update_links_batched(params, dims_list, [u.view for u in ups], [m.view for m in moms], 0.01)
    assert all(u.margins_intact() for u in ups)
