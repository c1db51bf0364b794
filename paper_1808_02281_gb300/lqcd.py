"""Thin Python binding of liblqcd (include/lqcd.h): argument marshalling only.

Every computation runs in the CUDA kernels of ``liblqcd.so``; torch supplies
device memory and the current CUDA stream.  There is no CPU fallback: if the
library is missing or a call fails, an exception is raised.

Tensor layouts (W = 4 for float32, 2 for float64; see include/lqcd.h):
  links    [4, 12 // W, V, W]   first two rows of every SU(3) link
  algebra  [4,  8 // W, V, W]   force, momenta, omega (components along T_a)
  full     [V, 4, 3, 3, 2]      complex 3x3 links as (re, im)
Helpers convert site-major numpy arrays [V, 4, 8] / complex [V, 4, 3, 3]
to and from these layouts (pure reshapes).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblqcd.so")

F32, F64 = 0, 1
FORCE_AUTO, FORCE_PATHS, FORCE_FACTORED, FORCE_STAPLE_FIELDS = 0, 1, 2, 3


class LqcdError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = _lib().lqcd_strerror(status).decode()
        if status == -5:
            msg += f" (cudaError {_lib().lqcd_last_cuda_error()})"
        super().__init__(f"{what}: {msg} [{status}]")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 4), ("precision", ctypes.c_int32),
                ("force_algo", ctypes.c_int32), ("beta", ctypes.c_double),
                ("c_plaq", ctypes.c_double), ("c_rect", ctypes.c_double),
                ("c_cube", ctypes.c_double)]


MAX_BATCH = 64


class LatticeRef(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 4), ("reserved", ctypes.c_int32 * 4),
                ("links", ctypes.c_void_p), ("mom", ctypes.c_void_p),
                ("force", ctypes.c_void_p), ("action", ctypes.c_void_p)]


_LIB = None
_EXPORTS = {
    "lqcd_symanzik_coefficients": (ctypes.c_int, [ctypes.c_double] + [ctypes.POINTER(ctypes.c_double)] * 4),
    "lqcd_links_from_omega": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lqcd_gauge_force": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_size_t, ctypes.c_void_p]),
    "lqcd_gauge_force_update_momenta": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p,
                                                       ctypes.c_double, ctypes.c_void_p]),
    "lqcd_md_force_step": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p]),
    "lqcd_gauge_action": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_size_t, ctypes.c_void_p]),
    "lqcd_gauge_action_noalloc": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p]),
    "lqcd_kinetic_energy": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_size_t, ctypes.c_void_p]),
    "lqcd_md_update_momenta": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_double, ctypes.c_void_p]),
    "lqcd_md_update_links": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_double, ctypes.c_void_p]),
    "lqcd_omega_gradient": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "lqcd_convert_links": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "lqcd_convert_algebra": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "lqcd_pack_links": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lqcd_unpack_links": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lqcd_wilson_dslash": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "lqcd_wilson_hopping_force": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]),
    "lqcd_unitarity_deviation": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "lqcd_reunitarise_links": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p]),
    "lqcd_gaussian_momenta": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_uint64, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    "lqcd_measure_fma_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                             ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "lqcd_fma_rate_scratch_bytes": (ctypes.c_size_t, []),
    "lqcd_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Desc)]),
    "lqcd_workspace_bytes_batched": (ctypes.c_size_t, [ctypes.POINTER(Desc), ctypes.c_int,
                                                       ctypes.POINTER(LatticeRef)]),
    "lqcd_md_force_step_batched": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_int, ctypes.POINTER(LatticeRef),
                                                  ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t,
                                                  ctypes.c_void_p]),
    "lqcd_md_update_links_batched": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_int,
                                                    ctypes.POINTER(LatticeRef), ctypes.c_double,
                                                    ctypes.c_void_p]),
    "lqcd_force_variant_count": (ctypes.c_int, [ctypes.POINTER(Desc)]),
    "lqcd_get_force_variant": (ctypes.c_int, [ctypes.POINTER(Desc)]),
    "lqcd_set_force_variant": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_int]),
    "lqcd_autotune_force": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "lqcd_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lqcd_last_cuda_error": (ctypes.c_int, []),
    "lqcd_version": (ctypes.c_int, []),
}


def _lib():
    """Load liblqcd.so; raise if it has not been built (no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1808_02281_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def library_path() -> str:
    _lib()
    return LIB_PATH


def symanzik_coefficients(u0: float):
    """(alpha_s, c_plaq, c_rect, c_cube) of Eq. 18_3_27_30 from u0."""
    out = [ctypes.c_double() for _ in range(4)]
    st = _lib().lqcd_symanzik_coefficients(float(u0), *[ctypes.byref(o) for o in out])
    if st:
        raise LqcdError(st, "lqcd_symanzik_coefficients")
    return tuple(o.value for o in out)


@dataclasses.dataclass
class Lattice:
    """A periodic lattice plus the action parameters (lqcd_desc)."""
    dims: tuple
    precision: str = "f32"   # "f32" or "f64"
    beta: float = 6.0
    c_plaq: float = 1.0
    c_rect: float = 0.0
    c_cube: float = 0.0
    force_algo: int = FORCE_AUTO

    @classmethod
    def symanzik(cls, dims, beta: float = 6.0, u0: float = 0.87, precision: str = "f32",
                 force_algo: int = FORCE_AUTO) -> "Lattice":
        _, cp, cr, cc = symanzik_coefficients(u0)
        return cls(tuple(int(d) for d in dims), precision, float(beta), cp, cr, cc, force_algo)

    @property
    def V(self) -> int:
        return int(np.prod(self.dims))

    @property
    def dtype(self):
        return torch.float32 if self.precision == "f32" else torch.float64

    @property
    def W(self) -> int:
        return 4 if self.precision == "f32" else 2

    @property
    def link_shape(self):
        return (4, 12 // self.W, self.V, self.W)

    @property
    def algebra_shape(self):
        return (4, 8 // self.W, self.V, self.W)

    @property
    def spinor_shape(self):
        return (24 // self.W, self.V, self.W)

    def desc(self) -> Desc:
        d = Desc()
        for i in range(4):
            d.dims[i] = int(self.dims[i])
        d.precision = F32 if self.precision == "f32" else F64
        d.force_algo = int(self.force_algo)
        d.beta = self.beta
        d.c_plaq, d.c_rect, d.c_cube = self.c_plaq, self.c_rect, self.c_cube
        return d

    def with_(self, **kw) -> "Lattice":
        return dataclasses.replace(self, **kw)


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(t: torch.Tensor, lat: Lattice, shape, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != lat.dtype:
        raise TypeError(f"{name} must be {lat.dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with shape {tuple(shape)}, got {tuple(t.shape)}")


def _call(name: str, *args):
    st = getattr(_lib(), name)(*args)
    if st:
        raise LqcdError(st, name)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def empty_links(lat: Lattice, device=None) -> torch.Tensor:
    return torch.empty(lat.link_shape, dtype=lat.dtype, device=device or "cuda")


def empty_algebra(lat: Lattice, device=None) -> torch.Tensor:
    return torch.empty(lat.algebra_shape, dtype=lat.dtype, device=device or "cuda")


def empty_spinor(lat: Lattice, device=None) -> torch.Tensor:
    return torch.empty(lat.spinor_shape, dtype=lat.dtype, device=device or "cuda")


def wilson_dslash(lat: Lattice, links: torch.Tensor, x: torch.Tensor, a: float = 0.0,
                  b: float = 1.0, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """y = a x + b calD x, calD the Wilson hopping operator (Eq. 18_7_17_4);
    a = 1, b = -kappa gives D x without the clover term."""
    _check(links, lat, lat.link_shape, "links")
    _check(x, lat, lat.spinor_shape, "x")
    out = empty_spinor(lat, x.device) if out is None else out
    _check(out, lat, lat.spinor_shape, "y")
    d = lat.desc()
    _call("lqcd_wilson_dslash", ctypes.byref(d), _ptr(links), _ptr(x), float(a), float(b),
          _ptr(out), _stream(stream))
    return out


def wilson_hopping_force(lat: Lattice, links: torch.Tensor, X: torch.Tensor, Y: torch.Tensor,
                         coef: float = 1.0, force: torch.Tensor | None = None,
                         mom: torch.Tensor | None = None, dt: float = 0.0, stream=None):
    """f = coef * h, h the components of -i(B - C)_TA (Eqs. 18_1_29_19 to
    18_7_17_30) on every link; stores f into ``force`` and/or applies
    mom += dt f.  With neither given, returns a new force tensor."""
    _check(links, lat, lat.link_shape, "links")
    _check(X, lat, lat.spinor_shape, "X")
    _check(Y, lat, lat.spinor_shape, "Y")
    if force is None and mom is None:
        force = empty_algebra(lat, links.device)
    for t, name in ((force, "force"), (mom, "mom")):
        if t is not None:
            _check(t, lat, lat.algebra_shape, name)
    d = lat.desc()
    _call("lqcd_wilson_hopping_force", ctypes.byref(d), _ptr(links), _ptr(X), _ptr(Y),
          float(coef), None if force is None else _ptr(force),
          None if mom is None else _ptr(mom), float(dt), _stream(stream))
    return force


def unitarity_deviation(lat: Lattice, links: torch.Tensor, out: torch.Tensor | None = None,
                        workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """max over links of the FP64 departure of the stored links from SU(3)
    (0-d float64 device tensor)."""
    _check(links, lat, lat.link_shape, "links")
    out = torch.empty((), dtype=torch.float64, device=links.device) if out is None else out
    ws = reduction_workspace(links.device) if workspace is None else workspace
    d = lat.desc()
    _call("lqcd_unitarity_deviation", ctypes.byref(d), _ptr(links), _ptr(out), _ptr(ws),
          ws.numel(), _stream(stream))
    return out


def reunitarise_links(lat: Lattice, links: torch.Tensor, stream=None) -> torch.Tensor:
    """Gram-Schmidt of every link in FP64, rounded to the storage precision (in place)."""
    _check(links, lat, lat.link_shape, "links")
    d = lat.desc()
    _call("lqcd_reunitarise_links", ctypes.byref(d), _ptr(links), _stream(stream))
    return links


def gaussian_momenta(lat: Lattice, seed: int, out: torch.Tensor | None = None,
                     device=None, stream=None) -> torch.Tensor:
    """p^a ~ N(0, 1) on every link from the counter-based stream `seed`
    (the same numbers as synth.momenta(dims, seed), drawn on the GPU)."""
    out = empty_algebra(lat, device) if out is None else out
    _check(out, lat, lat.algebra_shape, "mom")
    d = lat.desc()
    _call("lqcd_gaussian_momenta", ctypes.byref(d), ctypes.c_uint64(int(seed) & (2**64 - 1)),
          _ptr(out), _stream(stream))
    return out


def measure_fma_rate(precision: str = "f32", device=None, stream=None) -> float:
    """FMA issue rate of the device in TFLOP/s (FP32 or FP64; ~20 ms,
    synchronises)."""
    n = int(_lib().lqcd_fma_rate_scratch_bytes())
    scratch = torch.empty(n, dtype=torch.uint8, device=device or "cuda")
    out = ctypes.c_double()
    _call("lqcd_measure_fma_rate", F32 if precision == "f32" else F64, _ptr(scratch), n,
          ctypes.byref(out), _stream(stream))
    return out.value


def workspace_bytes(lat: Lattice) -> int:
    d = lat.desc()
    return int(_lib().lqcd_workspace_bytes(ctypes.byref(d)))


REDUCTION_WORKSPACE_BYTES = 1 << 16   # partial sums of up to 8192 reduction blocks


def reduction_workspace(device=None) -> torch.Tensor:
    """Workspace enough for the reductions alone (action, kinetic energy,
    unitarity check): one double per reduction block."""
    return torch.empty(REDUCTION_WORKSPACE_BYTES, dtype=torch.uint8, device=device or "cuda")


def make_workspace(lat: Lattice, device=None) -> torch.Tensor:
    n = max(workspace_bytes(lat), 256)
    return torch.empty(n, dtype=torch.uint8, device=device or "cuda")


def links_from_omega(lat: Lattice, omega: torch.Tensor, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    """U = exp(i omega.T) for every link (Eq. 18_1_29_3)."""
    _check(omega, lat, lat.algebra_shape, "omega")
    out = empty_links(lat, omega.device) if out is None else out
    _check(out, lat, lat.link_shape, "links")
    d = lat.desc()
    _call("lqcd_links_from_omega", ctypes.byref(d), _ptr(omega), _ptr(out), _stream(stream))
    return out


def gauge_force(lat: Lattice, links: torch.Tensor, out: torch.Tensor | None = None,
                workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """f^a = -dS/domega^a for every link (algebra layout).  Without a
    workspace one is allocated for the algorithms that use it."""
    _check(links, lat, lat.link_shape, "links")
    out = empty_algebra(lat, links.device) if out is None else out
    _check(out, lat, lat.algebra_shape, "force")
    ws = _workspace_for(lat, links.device, workspace)
    d = lat.desc()
    _call("lqcd_gauge_force", ctypes.byref(d), _ptr(links), _ptr(out),
          None if ws is None else _ptr(ws), 0 if ws is None else ws.numel(), _stream(stream))
    return out


def md_force_step(lat: Lattice, links: torch.Tensor, force: torch.Tensor | None = None,
                  mom: torch.Tensor | None = None, dt: float = 0.0,
                  action: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                  stream=None):
    """One force evaluation with optional fused consumers: store f, apply
    p += dt f, and/or write S_G (0-d float64 device tensor)."""
    _check(links, lat, lat.link_shape, "links")
    if force is not None:
        _check(force, lat, lat.algebra_shape, "force")
    if mom is not None:
        _check(mom, lat, lat.algebra_shape, "mom")
    if action is not None and (action.dtype != torch.float64 or not action.is_cuda):
        raise TypeError("action must be a float64 CUDA tensor")
    ws = make_workspace(lat, links.device) if workspace is None else workspace
    d = lat.desc()
    p = lambda t: None if t is None else _ptr(t)
    _call("lqcd_md_force_step", ctypes.byref(d), _ptr(links), p(force), p(mom), float(dt),
          p(action), _ptr(ws), ws.numel(), _stream(stream))
    return force, mom, action


def _workspace_for(lat: Lattice, device, workspace):
    if workspace is not None:
        return workspace
    if lat.force_algo in (FORCE_AUTO, FORCE_STAPLE_FIELDS):
        return make_workspace(lat, device)
    return None


def gauge_force_update_momenta(lat: Lattice, links: torch.Tensor, mom: torch.Tensor, dt: float,
                               stream=None) -> torch.Tensor:
    """mom += dt * f, the force never stored."""
    _check(links, lat, lat.link_shape, "links")
    _check(mom, lat, lat.algebra_shape, "mom")
    d = lat.desc()
    _call("lqcd_gauge_force_update_momenta", ctypes.byref(d), _ptr(links), _ptr(mom),
          float(dt), _stream(stream))
    return mom


def gauge_action(lat: Lattice, links: torch.Tensor, out: torch.Tensor | None = None,
                 workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """S_G (FP64, 0-d device tensor), Eq. 18_6_4_1."""
    _check(links, lat, lat.link_shape, "links")
    out = torch.empty((), dtype=torch.float64, device=links.device) if out is None else out
    ws = reduction_workspace(links.device) if workspace is None else workspace
    d = lat.desc()
    _call("lqcd_gauge_action", ctypes.byref(d), _ptr(links), _ptr(out), _ptr(ws), ws.numel(),
          _stream(stream))
    return out


def kinetic_energy(lat: Lattice, mom: torch.Tensor, out: torch.Tensor | None = None,
                   workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """K = sum p^2 / 2 (FP64, 0-d device tensor)."""
    _check(mom, lat, lat.algebra_shape, "mom")
    out = torch.empty((), dtype=torch.float64, device=mom.device) if out is None else out
    ws = reduction_workspace(mom.device) if workspace is None else workspace
    d = lat.desc()
    _call("lqcd_kinetic_energy", ctypes.byref(d), _ptr(mom), _ptr(out), _ptr(ws), ws.numel(),
          _stream(stream))
    return out


def md_update_momenta(lat: Lattice, mom: torch.Tensor, force: torch.Tensor, dt: float,
                      stream=None) -> torch.Tensor:
    _check(mom, lat, lat.algebra_shape, "mom")
    _check(force, lat, lat.algebra_shape, "force")
    d = lat.desc()
    _call("lqcd_md_update_momenta", ctypes.byref(d), _ptr(mom), _ptr(force), float(dt),
          _stream(stream))
    return mom


def md_update_links(lat: Lattice, links: torch.Tensor, mom: torch.Tensor, dt: float,
                    stream=None) -> torch.Tensor:
    _check(links, lat, lat.link_shape, "links")
    _check(mom, lat, lat.algebra_shape, "mom")
    d = lat.desc()
    _call("lqcd_md_update_links", ctypes.byref(d), _ptr(links), _ptr(mom), float(dt),
          _stream(stream))
    return links


def omega_gradient(lat: Lattice, omega: torch.Tensor, force: torch.Tensor,
                   out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """dS/domega for U = exp(i omega.T) U0, from the force at U."""
    _check(omega, lat, lat.algebra_shape, "omega")
    _check(force, lat, lat.algebra_shape, "force")
    out = empty_algebra(lat, omega.device) if out is None else out
    _check(out, lat, lat.algebra_shape, "grad")
    d = lat.desc()
    _call("lqcd_omega_gradient", ctypes.byref(d), _ptr(omega), _ptr(force), _ptr(out),
          _stream(stream))
    return out


def convert_links(lat: Lattice, links: torch.Tensor, precision: str,
                  out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The same links stored in another precision (into `out` or a new tensor)."""
    _check(links, lat, lat.link_shape, "links")
    dst_lat = lat.with_(precision=precision)
    out = empty_links(dst_lat, links.device) if out is None else out
    _check(out, dst_lat, dst_lat.link_shape, "out")
    d = lat.desc()
    _call("lqcd_convert_links", ctypes.byref(d), _ptr(links), F32 if precision == "f32" else F64,
          _ptr(out), _stream(stream))
    return out


def convert_algebra(lat: Lattice, field: torch.Tensor, precision: str,
                    out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The same algebra field (momenta, force) in another precision (into
    `out` or a new tensor)."""
    _check(field, lat, lat.algebra_shape, "field")
    dst_lat = lat.with_(precision=precision)
    out = empty_algebra(dst_lat, field.device) if out is None else out
    _check(out, dst_lat, dst_lat.algebra_shape, "out")
    d = lat.desc()
    _call("lqcd_convert_algebra", ctypes.byref(d), _ptr(field), F32 if precision == "f32" else F64,
          _ptr(out), _stream(stream))
    return out


def pack_links(lat: Lattice, full: torch.Tensor, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    _check(full, lat, (lat.V, 4, 3, 3, 2), "full")
    out = empty_links(lat, full.device) if out is None else out
    _check(out, lat, lat.link_shape, "links")
    d = lat.desc()
    _call("lqcd_pack_links", ctypes.byref(d), _ptr(full), _ptr(out), _stream(stream))
    return out


def unpack_links(lat: Lattice, links: torch.Tensor, out: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    _check(links, lat, lat.link_shape, "links")
    out = torch.empty((lat.V, 4, 3, 3, 2), dtype=lat.dtype, device=links.device) \
        if out is None else out
    _check(out, lat, (lat.V, 4, 3, 3, 2), "full")
    d = lat.desc()
    _call("lqcd_unpack_links", ctypes.byref(d), _ptr(links), _ptr(out), _stream(stream))
    return out


# ---------------------------------------------------------------- batches

def _batch_refs(params: Lattice, dims_list, links=None, mom=None, force=None, actions=None):
    n = len(dims_list)
    if not 1 <= n <= MAX_BATCH:
        raise ValueError(f"a batch holds 1..{MAX_BATCH} lattices")
    refs = (LatticeRef * n)()
    for c, dims in enumerate(dims_list):
        lat = params.with_(dims=tuple(int(d) for d in dims))
        for i in range(4):
            refs[c].dims[i] = int(dims[i])
        if links is not None:
            _check(links[c], lat, lat.link_shape, f"links[{c}]")
            refs[c].links = links[c].data_ptr()
        if mom is not None and mom[c] is not None:
            _check(mom[c], lat, lat.algebra_shape, f"mom[{c}]")
            refs[c].mom = mom[c].data_ptr()
        if force is not None and force[c] is not None:
            _check(force[c], lat, lat.algebra_shape, f"force[{c}]")
            refs[c].force = force[c].data_ptr()
        if actions is not None:
            refs[c].action = actions.data_ptr() + 8 * c
    return refs


def workspace_bytes_batched(params: Lattice, dims_list) -> int:
    refs = _batch_refs(params, dims_list)
    for r in refs:
        r.links = 16  # the size query checks pointers for presence only
    d = params.desc()
    return int(_lib().lqcd_workspace_bytes_batched(ctypes.byref(d), len(dims_list), refs))


def make_workspace_batched(params: Lattice, dims_list, device=None) -> torch.Tensor:
    n = max(workspace_bytes_batched(params, dims_list), 256)
    return torch.empty(n, dtype=torch.uint8, device=device or "cuda")


def md_force_step_batched(params: Lattice, dims_list, links, mom=None, dt: float = 0.0,
                          force=None, actions: torch.Tensor | None = None,
                          workspace: torch.Tensor | None = None, stream=None):
    """Force step of many lattices (extents dims_list, parameters of
    ``params``) in one launch per pass; actions: float64 device tensor [n]."""
    if actions is not None and (actions.dtype != torch.float64 or not actions.is_cuda
                                or actions.numel() != len(dims_list)):
        raise TypeError("actions must be a float64 CUDA tensor with one entry per lattice")
    refs = _batch_refs(params, dims_list, links, mom, force, actions)
    ws = make_workspace_batched(params, dims_list, links[0].device) if workspace is None else workspace
    d = params.desc()
    _call("lqcd_md_force_step_batched", ctypes.byref(d), len(dims_list), refs, float(dt), _ptr(ws),
          ws.numel(), _stream(stream))


def md_update_links_batched(params: Lattice, dims_list, links, mom, dt: float, stream=None):
    refs = _batch_refs(params, dims_list, links, mom)
    d = params.desc()
    _call("lqcd_md_update_links_batched", ctypes.byref(d), len(dims_list), refs, float(dt),
          _stream(stream))


def force_variant_count(lat: Lattice) -> int:
    d = lat.desc()
    n = _lib().lqcd_force_variant_count(ctypes.byref(d))
    if n < 0:
        raise LqcdError(n, "lqcd_force_variant_count")
    return n


def get_force_variant(lat: Lattice) -> int:
    d = lat.desc()
    return int(_lib().lqcd_get_force_variant(ctypes.byref(d)))


def set_force_variant(lat: Lattice, variant: int) -> None:
    d = lat.desc()
    _call("lqcd_set_force_variant", ctypes.byref(d), int(variant))


def autotune_force(lat: Lattice, links: torch.Tensor, reps: int = 3,
                   workspace: torch.Tensor | None = None, stream=None):
    """Time every force variant on these links and keep the fastest (the
    stream is synchronised).  Returns (best variant, [mean ms per variant])."""
    _check(links, lat, lat.link_shape, "links")
    n = force_variant_count(lat)
    scratch = empty_algebra(lat, links.device)
    ws = make_workspace(lat, links.device) if workspace is None else workspace
    best = ctypes.c_int(-1)
    ms = (ctypes.c_float * n)()
    d = lat.desc()
    _call("lqcd_autotune_force", ctypes.byref(d), _ptr(links), _ptr(scratch), _ptr(ws), ws.numel(),
          int(reps), _stream(stream), ctypes.byref(best), ms)
    return best.value, [ms[i] for i in range(n)]


# ----------------------------------------------------- layout marshalling

def algebra_to_device(lat: Lattice, a: np.ndarray, device="cuda", pin: bool = False) -> torch.Tensor:
    """Site-major [V, 4, 8] numpy -> algebra layout tensor (pure reshape)."""
    W = lat.W
    soa = np.ascontiguousarray(
        np.asarray(a).reshape(lat.V, 4, 8 // W, W).transpose(1, 2, 0, 3))
    t = torch.from_numpy(soa).to(lat.dtype)
    if pin:
        t = t.pin_memory()
    return t.to(device, non_blocking=pin)


def algebra_from_device(t: torch.Tensor) -> np.ndarray:
    """Algebra layout tensor -> site-major float64 numpy [V, 4, 8]."""
    a = t.detach().to("cpu", torch.float64).numpy()   # [4, 8/W, V, W]
    V = a.shape[2]
    return np.ascontiguousarray(a.transpose(2, 0, 1, 3).reshape(V, 4, 8))


def spinor_to_device(lat: Lattice, x: np.ndarray, device="cuda", pin: bool = False) -> torch.Tensor:
    """Spinor field, complex [V, 4, 3] or float [V, 4, 3, 2] (re, im) numpy
    -> spinor layout tensor [24/W, V, W] (pure reshape)."""
    x = np.asarray(x)
    if np.iscomplexobj(x):
        x = np.stack([x.real, x.imag], axis=-1)
    W = lat.W
    soa = np.ascontiguousarray(x.reshape(lat.V, 24 // W, W).transpose(1, 0, 2))
    t = torch.from_numpy(soa).to(lat.dtype)
    if pin:
        t = t.pin_memory()
    return t.to(device, non_blocking=pin)


def spinor_from_device(t: torch.Tensor) -> np.ndarray:
    """Spinor layout tensor -> complex128 numpy [V, 4, 3]."""
    a = t.detach().to("cpu", torch.float64).numpy()   # [24/W, V, W]
    V = a.shape[1]
    r = np.ascontiguousarray(a.transpose(1, 0, 2).reshape(V, 4, 3, 2))
    return r[..., 0] + 1j * r[..., 1]


def full_to_device(lat: Lattice, U: np.ndarray, device="cuda") -> torch.Tensor:
    """complex [V, 4, 3, 3] numpy -> full tensor [V, 4, 3, 3, 2]."""
    arr = np.ascontiguousarray(np.asarray(U, dtype=np.complex128)).view(np.float64)
    return torch.from_numpy(arr.reshape(lat.V, 4, 3, 3, 2)).to(device, lat.dtype)


def full_from_device(t: torch.Tensor) -> np.ndarray:
    """full tensor -> complex128 numpy [V, 4, 3, 3]."""
    a = t.detach().to("cpu", torch.float64).contiguous().numpy()
    return a[..., 0] + 1j * a[..., 1]
