"""Python face of the FP64 CPU oracle (``oracle/lqcd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the independent checker of the CUDA library.  Only
the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA path.

Array conventions (numpy, C order):
  links    complex128 [V, 4, 3, 3]  U_{n,mu}, site n = x + Lx*(y + Ly*(z + Lz*t))
  omega/p/f float64   [V, 4, 8]     algebra components along T_a = lambda_a/2
  spinors  complex128 [V, 4, 3]     X_{n, alpha a} (Dirac index alpha, colour a)
Everything follows D. Li, "The Calculation of Force in Lattice QCD", Sec. II
(gauge action and force) and Sec. III (Wilson hopping operator and its force).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lqcd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_dbl_p = ctypes.POINTER(ctypes.c_double)
_int_p = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc -O2 (no intrinsics, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def build_variant(source: str, path: str) -> str:
    """Compile C source text (a copy of the oracle) to `path` with the same
    flags as build(); used by the tests that plant mistakes in a copy."""
    src = path + ".c"
    with open(src, "w") as fh:
        fh.write(source)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", path, src, "-lm"],
                   check=True)
    return path


def _bind(L):
    L.oracle_coefficients.argtypes = [ctypes.c_double, _dbl_p]
    L.oracle_paths.argtypes = [_int_p, _int_p, _int_p]
    L.oracle_paths.restype = ctypes.c_int
    L.oracle_loop_sums.argtypes = [_int_p, _dbl_p, _dbl_p]
    L.oracle_gauge_action.argtypes = [_int_p, _dbl_p, ctypes.c_double, _dbl_p]
    L.oracle_gauge_action.restype = ctypes.c_double
    L.oracle_gauge_action_local.argtypes = [
        _int_p, _dbl_p, ctypes.c_double, _dbl_p, ctypes.c_long, ctypes.c_int]
    L.oracle_gauge_action_local.restype = ctypes.c_double
    L.oracle_gauge_force.argtypes = [_int_p, _dbl_p, ctypes.c_double, _dbl_p, _dbl_p]
    L.oracle_gauge_force_link.argtypes = [
        _int_p, _dbl_p, ctypes.c_double, _dbl_p, ctypes.c_long, ctypes.c_int, _dbl_p]
    L.oracle_exp_i_algebra.argtypes = [_dbl_p, _dbl_p]
    L.oracle_links_from_omega.argtypes = [ctypes.c_long, _dbl_p, _dbl_p]
    L.oracle_md_update_momenta.argtypes = [ctypes.c_long, _dbl_p, _dbl_p, ctypes.c_double]
    L.oracle_md_update_links.argtypes = [ctypes.c_long, _dbl_p, _dbl_p, ctypes.c_double]
    L.oracle_kinetic_energy.argtypes = [ctypes.c_long, _dbl_p]
    L.oracle_kinetic_energy.restype = ctypes.c_double
    L.oracle_gauge_transform.argtypes = [_int_p, _dbl_p, _dbl_p, _dbl_p]
    L.oracle_algebra_to_matrix.argtypes = [_dbl_p, _dbl_p]
    L.oracle_traceless_antihermitian.argtypes = [_dbl_p, _dbl_p]
    L.oracle_generator.argtypes = [ctypes.c_int, _dbl_p]
    L.oracle_gamma.argtypes = [ctypes.c_int, _dbl_p]
    L.oracle_wilson_hopping.argtypes = [_int_p, _dbl_p, _dbl_p, _dbl_p]
    L.oracle_wilson_hopping_site.argtypes = [_int_p, _dbl_p, _dbl_p, ctypes.c_long, _dbl_p]
    L.oracle_wilson_hopping_force.argtypes = [_int_p, _dbl_p, _dbl_p, _dbl_p, ctypes.c_double,
                                              _dbl_p]
    L.oracle_wilson_hopping_force_link.argtypes = [
        _int_p, _dbl_p, _dbl_p, _dbl_p, ctypes.c_double, ctypes.c_long, ctypes.c_int, _dbl_p]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Route every oracle call through another build of the oracle for the
    duration of the block (the tests that plant mistakes use it)."""
    global _lib
    saved = lib()
    _lib = _bind(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _d(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(_dbl_p)


def _dims(dims):
    arr = (ctypes.c_int * 4)(*[int(v) for v in dims])
    return arr


def _cplx(U) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.complex128)
    return U


def coefficients(u0: float) -> np.ndarray:
    """(c_plaq, c_rect, c_cube) of Eq. 18_3_27_30 for tadpole factor u0."""
    c = np.zeros(3)
    lib().oracle_coefficients(float(u0), _d(c))
    return c


def paths():
    """The 34 loops as (directions[34, 6] zero padded, lengths[34], classes[34])."""
    d = np.zeros((34, 6), dtype=np.intc)
    ln = np.zeros(34, dtype=np.intc)
    cl = np.zeros(34, dtype=np.intc)
    n = lib().oracle_paths(d.ctypes.data_as(_int_p), ln.ctypes.data_as(_int_p),
                           cl.ctypes.data_as(_int_p))
    return d[:n], ln[:n], cl[:n]


def loop_sums(dims, U) -> np.ndarray:
    """Per-class sums of 3 - Re tr P_n (plaquette, rectangle, cube)."""
    U = _cplx(U)
    out = np.zeros(3)
    lib().oracle_loop_sums(_dims(dims), _d(U.view(np.float64)), _d(out))
    return out


def gauge_action(dims, U, beta: float, c) -> float:
    """S_G of Eq. 18_6_4_1."""
    U = _cplx(U)
    c = np.ascontiguousarray(c, dtype=np.float64)
    return lib().oracle_gauge_action(_dims(dims), _d(U.view(np.float64)), float(beta), _d(c))


def gauge_action_local(dims, U, beta: float, c, site: int, rho: int) -> float:
    """The part of S_G from loops through link (site, rho); rho = 0..3."""
    U = _cplx(U)
    c = np.ascontiguousarray(c, dtype=np.float64)
    return lib().oracle_gauge_action_local(
        _dims(dims), _d(U.view(np.float64)), float(beta), _d(c), int(site), int(rho) + 1)


def gauge_force(dims, U, beta: float, c) -> np.ndarray:
    """f[V, 4, 8] = -dS/domega on every link (Eqs. 18_7_25_1 to 18_6_6_13)."""
    U = _cplx(U)
    c = np.ascontiguousarray(c, dtype=np.float64)
    V = U.shape[0]
    f = np.zeros((V, 4, 8))
    lib().oracle_gauge_force(_dims(dims), _d(U.view(np.float64)), float(beta), _d(c), _d(f))
    return f


def gauge_force_link(dims, U, beta: float, c, site: int, rho: int) -> np.ndarray:
    """f[8] on one link (start sites by Eqs. 18_7_26_2/3); rho = 0..3."""
    U = _cplx(U)
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = np.zeros(8)
    lib().oracle_gauge_force_link(_dims(dims), _d(U.view(np.float64)), float(beta), _d(c),
                                  int(site), int(rho) + 1, _d(out))
    return out


def gauge_force_links(dims, U, beta: float, c, sites, rhos) -> np.ndarray:
    """f[len(sites), 8] for a list of links, one by one."""
    return np.stack([gauge_force_link(dims, U, beta, c, s, r) for s, r in zip(sites, rhos)])


def exp_i_algebra(w) -> np.ndarray:
    """exp(i sum_a w^a T_a) as a 3x3 complex matrix (Eq. 18_1_29_3)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros((3, 3), dtype=np.complex128)
    lib().oracle_exp_i_algebra(_d(w), _d(out.view(np.float64)))
    return out


def links_from_omega(omega) -> np.ndarray:
    """U[V, 4, 3, 3] = exp(i omega.T) link by link; omega[V, 4, 8]."""
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    n = omega.size // 8
    U = np.zeros(omega.shape[:-1] + (3, 3), dtype=np.complex128)
    lib().oracle_links_from_omega(n, _d(omega), _d(U.view(np.float64)))
    return U


def md_update_momenta(p, f, dt: float) -> np.ndarray:
    p = np.array(p, dtype=np.float64, order="C", copy=True)
    f = np.ascontiguousarray(f, dtype=np.float64)
    lib().oracle_md_update_momenta(p.size // 8, _d(p), _d(f), float(dt))
    return p


def md_update_links(U, p, dt: float) -> np.ndarray:
    U = np.array(U, dtype=np.complex128, order="C", copy=True)
    p = np.ascontiguousarray(p, dtype=np.float64)
    lib().oracle_md_update_links(p.size // 8, _d(U.view(np.float64)), _d(p), float(dt))
    return U


def kinetic_energy(p) -> float:
    p = np.ascontiguousarray(p, dtype=np.float64)
    return lib().oracle_kinetic_energy(p.size // 8, _d(p))


def gauge_transform(dims, U, g) -> np.ndarray:
    """U'_{n,mu} = g_n U_{n,mu} g_{n+mu}^dagger; g[V, 3, 3]."""
    U = _cplx(U)
    g = _cplx(g)
    out = np.zeros_like(U)
    lib().oracle_gauge_transform(_dims(dims), _d(U.view(np.float64)), _d(g.view(np.float64)),
                                 _d(out.view(np.float64)))
    return out


def algebra_to_matrix(f) -> np.ndarray:
    """H = sum_a f^a T_a."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros((3, 3), dtype=np.complex128)
    lib().oracle_algebra_to_matrix(_d(f), _d(out.view(np.float64)))
    return out


def traceless_antihermitian(b) -> np.ndarray:
    b = _cplx(b)
    out = np.zeros((3, 3), dtype=np.complex128)
    lib().oracle_traceless_antihermitian(_d(b.view(np.float64)), _d(out.view(np.float64)))
    return out


def generator(a: int) -> np.ndarray:
    out = np.zeros((3, 3), dtype=np.complex128)
    lib().oracle_generator(int(a), _d(out.view(np.float64)))
    return out


def leapfrog(dims, U, p, beta: float, c, dt: float, nsteps: int):
    """Leapfrog trajectory built from the oracle's MD steps (used by the
    integrator pins): p(dt/2), [U(dt), p(dt)]*(n-1), U(dt), p(dt/2)."""
    p = md_update_momenta(p, gauge_force(dims, U, beta, c), dt / 2)
    for i in range(nsteps):
        U = md_update_links(U, p, dt)
        f = gauge_force(dims, U, beta, c)
        p = md_update_momenta(p, f, dt if i < nsteps - 1 else dt / 2)
    return U, p


OMELYAN_LAMBDA = 0.1931833275037836


def omelyan(dims, U, p, beta: float, c, dt: float, nsteps: int, lam: float = OMELYAN_LAMBDA):
    """Second-order minimum-norm integrator (Omelyan, Mryglod & Folk 2003)
    built from the oracle's MD steps: per step p(l dt) U(dt/2) p((1-2l) dt)
    U(dt/2) p(l dt), the last kick of a step merged with the first of the
    next.  (The paper names no integrator; this one is a test reference.)"""
    p = md_update_momenta(p, gauge_force(dims, U, beta, c), lam * dt)
    for i in range(nsteps):
        U = md_update_links(U, p, dt / 2)
        p = md_update_momenta(p, gauge_force(dims, U, beta, c), (1 - 2 * lam) * dt)
        U = md_update_links(U, p, dt / 2)
        p = md_update_momenta(p, gauge_force(dims, U, beta, c),
                              2 * lam * dt if i < nsteps - 1 else lam * dt)
    return U, p


def hamiltonian(dims, U, p, beta: float, c) -> float:
    return kinetic_energy(p) + gauge_action(dims, U, beta, c)


# ------------------------------------------------------ Wilson fermion (Sec. III)

def gamma(mu: int) -> np.ndarray:
    """gamma_mu (mu = 1..4, along x, y, z, t) and gamma_5 (mu = 5) of the
    oracle's chiral basis, 4x4 complex."""
    out = np.zeros((4, 4), dtype=np.complex128)
    lib().oracle_gamma(int(mu), _d(out.view(np.float64)))
    return out


def wilson_hopping(dims, U, X) -> np.ndarray:
    """calD X of Eq. 18_7_17_4; X, result complex [V, 4, 3]."""
    U = _cplx(U)
    X = _cplx(X)
    out = np.zeros_like(X)
    lib().oracle_wilson_hopping(_dims(dims), _d(U.view(np.float64)), _d(X.view(np.float64)),
                                _d(out.view(np.float64)))
    return out


def wilson_hopping_site(dims, U, X, site: int) -> np.ndarray:
    """(calD X)_site, complex [4, 3]."""
    U, X = _cplx(U), _cplx(X)
    out = np.zeros((4, 3), dtype=np.complex128)
    lib().oracle_wilson_hopping_site(_dims(dims), _d(U.view(np.float64)), _d(X.view(np.float64)),
                                     int(site), _d(out.view(np.float64)))
    return out


def wilson_hopping_force(dims, U, X, Y, coef: float = 1.0) -> np.ndarray:
    """coef * h[V, 4, 8], h^i = -(tr(i T_i (B - C)) + c.c.) on every link
    (Eqs. 18_1_29_20_1 to 18_7_17_30)."""
    U, X, Y = _cplx(U), _cplx(X), _cplx(Y)
    out = np.zeros((U.shape[0], 4, 8))
    lib().oracle_wilson_hopping_force(_dims(dims), _d(U.view(np.float64)),
                                      _d(X.view(np.float64)), _d(Y.view(np.float64)),
                                      float(coef), _d(out))
    return out


def wilson_hopping_force_link(dims, U, X, Y, coef: float, site: int, rho: int) -> np.ndarray:
    """The same on one link; rho = 0..3."""
    U, X, Y = _cplx(U), _cplx(X), _cplx(Y)
    out = np.zeros(8)
    lib().oracle_wilson_hopping_force_link(_dims(dims), _d(U.view(np.float64)),
                                           _d(X.view(np.float64)), _d(Y.view(np.float64)),
                                           float(coef), int(site), int(rho) + 1, _d(out))
    return out
