"""The allocation-free action entry point, lqcd_gauge_action_noalloc.

Some callers cannot allocate device memory themselves (a host application
that owns all device memory through its own pool, or a loop with a fixed
memory budget); this entry point keeps its per-block partial sums in a fixed
array held by the library instead of a caller workspace.  The test calls it
through the C ABI, twice in a row, and compares each result with the
workspace-taking lqcd_gauge_action on the same links and stream: the two
run the same kernels with the same number of partial sums, so the values
must be bitwise equal (which also keeps them inside the action tolerances of
the parity tests).  It builds everything it needs itself, so it passes alone
in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1808_02281_gb300 import build as B
from paper_1808_02281_gb300 import lqcd, synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-5}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    return lqcd._lib()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims,sigma", [((4, 4, 4, 4), 0.5), ((3, 4, 5, 6), 0.4),
                                        ((16, 16, 16, 32), 0.15)])
def test_noalloc_action_matches_workspace_action(lib, dims, sigma, prec):
    lat = lqcd.Lattice.symanzik(dims, 6.0, 0.87, prec)
    links = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, synth.omega(dims, sigma, 0)))
    want = float(lqcd.gauge_action(lat, links).item())
    d = lat.desc()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):  # two calls in a row share the library's scratch
        out = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.lqcd_gauge_action_noalloc(ctypes.byref(d), ctypes.c_void_p(links.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, lib.lqcd_strerror(st)
        got = float(out.item())
        assert np.isfinite(got)
        assert got == want, (got, want)
        assert abs(got - want) <= TOL[prec] * abs(want)


def test_noalloc_rejects_bad_arguments(lib):
    """The same argument checks as lqcd_gauge_action (shared code): every
    rejected call returns its status and leaves the output untouched (it
    starts as NaN and must still be NaN)."""
    lat = lqcd.Lattice.symanzik((4, 4, 4, 4), 6.0, 0.87, "f32")
    links = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, synth.omega(lat.dims, 0.5, 0)))
    out = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    ws = lqcd.reduction_workspace(links.device)
    L, O = ctypes.c_void_p(links.data_ptr()), ctypes.c_void_p(out.data_ptr())

    def both(d, links_p=L, out_p=O):
        a = lib.lqcd_gauge_action_noalloc(d, links_p, out_p, None)
        b = lib.lqcd_gauge_action(d, links_p, out_p, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                  None)
        assert a == b, (a, b)
        return a

    assert both(None) == -1
    d = lat.desc()
    d.dims[2] = 0
    assert both(ctypes.byref(d)) == -2
    d = lat.desc()
    d.force_algo = 99
    assert both(ctypes.byref(d)) == -1
    d = lat.desc()
    d.precision = 7
    assert both(ctypes.byref(d)) == -1
    d = lat.desc()
    d.beta = float("inf")
    assert both(ctypes.byref(d)) == -1
    d = lat.desc()
    assert both(ctypes.byref(d), links_p=ctypes.c_void_p(links.data_ptr() + 4)) == -3
    assert both(ctypes.byref(d), out_p=ctypes.c_void_p(out.data_ptr() + 4)) == -3
    assert both(ctypes.byref(d), out_p=None) == -1
    torch.cuda.synchronize()
    assert np.isnan(float(out.item()))
