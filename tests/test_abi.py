"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/lqcd.h declares, and rejects bad arguments before touching
the device (so these calls never reach CUDA)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_1808_02281_gb300 import build as B
from paper_1808_02281_gb300 import lqcd

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "lqcd.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lqcd._lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lqcd_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("lqcd_gauge_action", "lqcd_gauge_force", "lqcd_md_update_momenta",
                 "lqcd_md_update_links"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_declares_every_export():
    assert set(declared_functions()) <= set(lqcd._EXPORTS)


def test_coefficients_match_oracle(lib):
    for u0 in (0.8, 0.86, 0.87, 0.95, 1.0):
        a, cp, cr, cc = lqcd.symanzik_coefficients(u0)
        np.testing.assert_allclose([cp, cr, cc], O.coefficients(u0), rtol=1e-15, atol=1e-17)
        assert abs(a - (-4 * np.log(u0) / 3.06839)) < 1e-15
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(lqcd.LqcdError):
            lqcd.symanzik_coefficients(bad)


def _desc(**kw):
    lat = lqcd.Lattice.symanzik((4, 4, 4, 4))
    d = lat.desc()
    for k, v in kw.items():
        if k == "dims":
            for i in range(4):
                d.dims[i] = v[i]
        else:
            setattr(d, k, v)
    return d


GOOD = ctypes.c_void_p(0x10000)      # aligned fake device pointers: never dereferenced,
GOOD2 = ctypes.c_void_p(0x20000)     # because every call below fails its argument check
MISALIGNED = ctypes.c_void_p(0x10008)


@pytest.mark.parametrize("kw,code", [
    (dict(dims=(0, 4, 4, 4)), -2),
    (dict(dims=(4, 4, -1, 4)), -2),
    (dict(dims=(1 << 20, 1 << 20, 1 << 20, 1 << 20)), -2),
    (dict(precision=7), -1),
    (dict(force_algo=9), -1),
    (dict(beta=float("nan")), -1),
    (dict(c_cube=float("inf")), -1),
])
def test_descriptor_rejected(lib, kw, code):
    d = _desc(**kw)
    assert lib.lqcd_gauge_force(ctypes.byref(d), GOOD, GOOD2, None, 0, None) == code
    assert lib.lqcd_md_update_links(ctypes.byref(d), GOOD, GOOD2, ctypes.c_double(0.1), None) == code
    assert lib.lqcd_workspace_bytes(ctypes.byref(d)) == 0


def test_pointer_checks(lib):
    d = _desc()
    assert lib.lqcd_gauge_force(None, GOOD, GOOD2, None, 0, None) == -1
    assert lib.lqcd_gauge_force(ctypes.byref(d), None, GOOD2, None, 0, None) == -1
    assert lib.lqcd_gauge_force(ctypes.byref(d), MISALIGNED, GOOD2, None, 0, None) == -3
    assert lib.lqcd_gauge_force(ctypes.byref(d), GOOD, MISALIGNED, None, 0, None) == -3
    assert lib.lqcd_gauge_force(ctypes.byref(d), GOOD, GOOD, None, 0, None) == -1   # aliasing
    assert lib.lqcd_md_update_momenta(ctypes.byref(d), GOOD, GOOD, ctypes.c_double(0.1), None) == -1
    assert lib.lqcd_md_update_momenta(ctypes.byref(d), GOOD, GOOD2, ctypes.c_double(float("nan")),
                                      None) == -1
    assert lib.lqcd_gauge_force_update_momenta(ctypes.byref(d), GOOD, GOOD,
                                               ctypes.c_double(0.1), None) == -1
    assert lib.lqcd_links_from_omega(ctypes.byref(d), GOOD, MISALIGNED, None) == -3
    assert lib.lqcd_pack_links(ctypes.byref(d), GOOD, GOOD, None) == -1
    assert lib.lqcd_unpack_links(ctypes.byref(d), None, GOOD, None) == -1
    assert lib.lqcd_gauge_action(ctypes.byref(d), GOOD, None, GOOD2, 4096, None) == -1
    assert lib.lqcd_kinetic_energy(ctypes.byref(d), MISALIGNED, GOOD2, GOOD, 4096, None) == -3


def test_wilson_argument_checks(lib):
    d = _desc()
    D = ctypes.c_double
    GOOD3 = ctypes.c_void_p(0x30000)
    GOOD4 = ctypes.c_void_p(0x40000)
    dslash = lib.lqcd_wilson_dslash
    assert dslash(None, GOOD, GOOD2, D(1), D(-0.1), GOOD3, None) == -1
    assert dslash(ctypes.byref(d), None, GOOD2, D(1), D(-0.1), GOOD3, None) == -1
    assert dslash(ctypes.byref(d), GOOD, MISALIGNED, D(1), D(-0.1), GOOD3, None) == -3
    assert dslash(ctypes.byref(d), GOOD, GOOD2, D(1), D(-0.1), GOOD2, None) == -1    # y == x
    assert dslash(ctypes.byref(d), GOOD, GOOD2, D(float("nan")), D(-0.1), GOOD3, None) == -1
    assert dslash(ctypes.byref(_desc(dims=(4, 0, 4, 4))), GOOD, GOOD2, D(1), D(1), GOOD3,
                  None) == -2
    force = lib.lqcd_wilson_hopping_force
    assert force(ctypes.byref(d), GOOD, GOOD2, GOOD3, D(0.1), None, None, D(0), None) == -1
    assert force(ctypes.byref(d), GOOD, GOOD2, None, D(0.1), GOOD4, None, D(0), None) == -1
    assert force(ctypes.byref(d), GOOD, GOOD2, GOOD3, D(0.1), MISALIGNED, None, D(0), None) == -3
    assert force(ctypes.byref(d), GOOD, GOOD2, GOOD3, D(0.1), None, MISALIGNED, D(0), None) == -3
    assert force(ctypes.byref(d), GOOD, GOOD2, GOOD3, D(0.1), GOOD4, GOOD4, D(0), None) == -1
    assert force(ctypes.byref(d), GOOD, GOOD2, GOOD3, D(0.1), GOOD2, None, D(0), None) == -1
    assert force(ctypes.byref(d), GOOD, GOOD2, GOOD3, D(float("inf")), GOOD4, None, D(0),
                 None) == -1


def test_unitarity_and_reunitarise_argument_checks(lib):
    d = _desc()
    assert lib.lqcd_unitarity_deviation(ctypes.byref(d), None, GOOD2, GOOD, 4096, None) == -1
    assert lib.lqcd_unitarity_deviation(ctypes.byref(d), GOOD, None, GOOD, 4096, None) == -1
    assert lib.lqcd_unitarity_deviation(ctypes.byref(d), MISALIGNED, GOOD2, GOOD, 4096, None) == -3
    assert lib.lqcd_unitarity_deviation(ctypes.byref(_desc(dims=(0, 4, 4, 4))), GOOD, GOOD2, GOOD,
                                        4096, None) == -2
    assert lib.lqcd_reunitarise_links(ctypes.byref(d), None, None) == -1
    assert lib.lqcd_reunitarise_links(ctypes.byref(d), MISALIGNED, None) == -3
    assert lib.lqcd_reunitarise_links(None, GOOD, None) == -1


def test_fma_rate_argument_checks(lib):
    out = ctypes.c_double()
    n = lib.lqcd_fma_rate_scratch_bytes()
    assert n >= 1 << 20
    assert lib.lqcd_measure_fma_rate(7, GOOD, n, ctypes.byref(out), None) == -1
    assert lib.lqcd_measure_fma_rate(0, GOOD, n, None, None) == -1
    assert lib.lqcd_measure_fma_rate(0, None, n, ctypes.byref(out), None) == -4
    assert lib.lqcd_measure_fma_rate(1, GOOD, n - 1, ctypes.byref(out), None) == -4
    assert lib.lqcd_measure_fma_rate(1, MISALIGNED, n, ctypes.byref(out), None) == -4


def test_spinor_marshalling_roundtrip():
    """Real r = 2*(3*alpha + a) + part of site n sits at ((r/W)*V + n)*W + r%W."""
    lat = lqcd.Lattice.symanzik((2, 3, 2, 2))
    x = np.arange(lat.V * 24, dtype=np.float64).reshape(lat.V, 4, 3, 2)
    for prec in ("f32", "f64"):
        L2 = lat.with_(precision=prec)
        t = lqcd.spinor_to_device(L2, x, device="cpu")
        assert tuple(t.shape) == L2.spinor_shape
        flat = t.numpy().ravel()
        W = L2.W
        for n, al, a, part in [(0, 0, 0, 0), (5, 2, 1, 1), (23, 3, 2, 1), (7, 1, 2, 0)]:
            r = 2 * (3 * al + a) + part
            assert flat[((r // W) * lat.V + n) * W + r % W] == x[n, al, a, part]
        back = lqcd.spinor_from_device(t)
        np.testing.assert_array_equal(back, x[..., 0] + 1j * x[..., 1])


def test_strerror(lib):
    assert lib.lqcd_strerror(0) == b"success"
    for code in range(-7, 0):
        assert lib.lqcd_strerror(code) not in (b"", b"unknown status")
    assert lib.lqcd_strerror(-99) == b"unknown status"
    assert lib.lqcd_version() == 1


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(lqcd, "_LIB", None)
    monkeypatch.setattr(lqcd, "LIB_PATH", "/nonexistent/liblqcd.so")
    with pytest.raises(RuntimeError, match="missing"):
        lqcd._lib()


def test_layout_marshalling_roundtrip():
    """The numpy <-> SoA reshapes used by the tests are inverse permutations
    and put component a of link (n, mu) where the header says."""
    lat = lqcd.Lattice.symanzik((2, 3, 2, 2))
    a = np.arange(lat.V * 32, dtype=np.float64).reshape(lat.V, 4, 8)
    for prec in ("f32", "f64"):
        L2 = lat.with_(precision=prec)
        t = lqcd.algebra_to_device(L2, a, device="cpu")
        flat = t.numpy().ravel()
        W = L2.W
        for n, mu, c in [(0, 0, 0), (5, 2, 7), (11, 3, 3)]:
            assert flat[((mu * (8 // W) + c // W) * lat.V + n) * W + c % W] == a[n, mu, c]
        np.testing.assert_array_equal(lqcd.algebra_from_device(t), a)


def test_batch_argument_checks(lib):
    d = _desc()
    refs = (lqcd.LatticeRef * 2)()
    for r in refs:
        for i in range(4):
            r.dims[i] = 4
        r.links = 0x10000
        r.mom = 0x20000
    assert lib.lqcd_md_force_step_batched(ctypes.byref(d), 0, refs, 0.1, GOOD, 1 << 30, None) == -1
    assert lib.lqcd_md_force_step_batched(ctypes.byref(d), 65, refs, 0.1, GOOD, 1 << 30, None) == -1
    refs[1].dims[2] = 0
    assert lib.lqcd_md_force_step_batched(ctypes.byref(d), 2, refs, 0.1, GOOD, 1 << 30, None) == -2
    refs[1].dims[2] = 4
    refs[1].mom = 0x20008
    assert lib.lqcd_md_force_step_batched(ctypes.byref(d), 2, refs, 0.1, GOOD, 1 << 30, None) == -3
    refs[1].mom = 0x20000
    dp = _desc(force_algo=1)
    assert lib.lqcd_md_force_step_batched(ctypes.byref(dp), 2, refs, 0.1, GOOD, 1 << 30, None) == -6
    assert lib.lqcd_md_force_step_batched(ctypes.byref(d), 2, refs, 0.1, GOOD, 16, None) == -4
    need = lib.lqcd_workspace_bytes_batched(ctypes.byref(d), 2, refs)
    assert need == 2 * lib.lqcd_workspace_bytes_batched(ctypes.byref(d), 1, refs) - 256
    assert need >= 2 * 24 * 12 * 256 * 4


def test_default_force_schedule(lib):
    """The built-in staple-field schedule (no lqcd_set_force_variant, no
    autotuning): full staples with the register cap in FP32, uncapped full
    staples in FP64, for every shape; a set choice overrides it, and -1
    restores it.  Host logic only (no CUDA call)."""
    cases = [((32, 32, 32, 64), "f32", 5), ((32, 32, 32, 32), "f32", 5),
             ((16, 16, 16, 32), "f32", 5), ((48, 48, 48, 96), "f32", 5),
             ((32, 32, 32, 64), "f64", 4), ((4, 4, 4, 4), "f64", 4)]
    for dims, prec, want in cases:
        lat = lqcd.Lattice.symanzik(dims, precision=prec)
        assert lqcd.force_variant_count(lat) == 9
        assert lqcd.get_force_variant(lat) == want, (dims, prec)
    lat = lqcd.Lattice.symanzik((16, 16, 16, 32))
    try:
        lqcd.set_force_variant(lat, 7)
        assert lqcd.get_force_variant(lqcd.Lattice.symanzik((32, 32, 32, 64))) == 7
        assert lqcd.get_force_variant(lqcd.Lattice.symanzik((32, 32, 32, 64), precision="f64")) == 4
    finally:
        lqcd.set_force_variant(lat, -1)
    assert lqcd.get_force_variant(lqcd.Lattice.symanzik((32, 32, 32, 64))) == 5
