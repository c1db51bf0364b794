"""Independent test-side constructions (numpy only): textbook Gell-Mann
matrices, closed-form abelian flux configurations, layout helpers.  Nothing
here calls the oracle or the CUDA library."""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_1..lambda_8 (textbook form)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return l


def read_paths():
    """The loops of the golden file as (class, tuple(directions))."""
    out = []
    with open(os.path.join(GOLDEN, "symanzik_paths.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            out.append((parts[0], tuple(int(v) for v in parts[1:])))
    return out


def coords(dims, n):
    x = []
    for L in dims:
        x.append(n % L)
        n //= L
    return x


def site_coords(dims) -> np.ndarray:
    """[V, 4] integer coordinates, x fastest."""
    V = int(np.prod(dims))
    n = np.arange(V)
    out = np.empty((V, 4), dtype=np.int64)
    for i, L in enumerate(dims):
        out[:, i] = n % L
        n = n // L
    return out


def abelian_flux_links(dims, theta, phi, axes=(0, 1, 2)) -> np.ndarray:
    """Diagonal links U_b(n) = exp(i theta n_a lam), U_c(n) = exp(i phi n_a lam),
    all other links unit, lam = diag(1, -1, 0); (a, b, c) = ``axes``.
    Every loop then equals exp(i Phi lam) with Phi = theta * (signed area
    projected on the (a, b) plane) + phi * (signed area on (a, c))."""
    a, b, c = axes
    V = int(np.prod(dims))
    x = site_coords(dims)[:, a].astype(np.float64)
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1
    for mu, ang in ((b, theta), (c, phi)):
        U[:, mu, 0, 0] = np.exp(1j * ang * x)
        U[:, mu, 1, 1] = np.exp(-1j * ang * x)
    return U


def abelian_flux_class_sums(V, theta, phi) -> np.ndarray:
    """Closed form of sum_n sum_{P in class} [3 - Re tr P_n] for the flux
    configuration above (plaquette, rectangle, cube), derived from the loop
    shapes of Eq. 18_3_27_30: 3 - Re tr exp(i Phi lam) = 2 (1 - cos Phi).
      plaquettes: the (a,b) and (a,c) plaquettes carry Phi = theta, phi;
      rectangles: four 2x1 loops carry +-2 theta and +-2 phi;
      cubes: 4 loops in the (a,b,c) cube carry +-theta +- phi, and the 8
             loops in (a,b,d), (a,c,d) carry +-theta, +-phi."""
    plaq = 2 * (1 - np.cos(theta)) + 2 * (1 - np.cos(phi))
    rect = 4 * (1 - np.cos(2 * theta)) + 4 * (1 - np.cos(2 * phi))
    cube = 4 * (2 - np.cos(theta + phi) - np.cos(theta - phi)) + \
        8 * (1 - np.cos(theta)) + 8 * (1 - np.cos(phi))
    return V * np.array([plaq, rect, cube])


def random_su3_numpy(rng, n) -> np.ndarray:
    """Haar-like random unitary matrices (QR of complex Gaussians), det fixed
    to 1: independent of any exponential."""
    z = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[:, None, None]


# Layout marshalling between the oracle's site-major arrays and the CUDA
# library's structure-of-arrays planes (pure reshapes, no arithmetic).

def algebra_to_soa(a: np.ndarray) -> np.ndarray:
    """[V, 4, 8] -> [4, 8, V]."""
    return np.ascontiguousarray(np.transpose(a, (1, 2, 0)))


def algebra_from_soa(a: np.ndarray) -> np.ndarray:
    """[4, 8, V] -> [V, 4, 8]."""
    return np.ascontiguousarray(np.transpose(a, (2, 0, 1)))
