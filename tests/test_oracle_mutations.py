"""The pins catch plausible mistakes: each case plants one mistake in a copy
of the oracle's C source (a sign, a dropped dagger, a transposed product, a
wrong loop shape, a wrong normalisation, a truncated series, a wrong
neighbour, ...), builds it, and runs a fast battery of the pins against it;
at least one pin must fail.  The unmutated oracle passes the same battery.
CPU only; the mistakes exist only in temporary copies."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import oracle as O
from paper_1808_02281_gb300 import synth
from tests import helpers as H

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "lqcd_oracle.c")
DIMS = (4, 3, 4, 3)
V = 144
BETA = 6.0
T = H.gell_mann() / 2


def _cplx(s):
    return s[..., 0] + 1j * s[..., 1]


def _fd_gauge(U, c, links, eps=1e-4):
    """max over links and generators of |-(S(+) - S(-))/2eps - f|, relative."""
    f = O.gauge_force(DIMS, U, BETA, c)
    worst = 0.0
    for li in links:
        k, rho = divmod(int(li), 4)
        for a in range(8):
            d = []
            for s in (1, -1):
                Up = U.copy()
                Up[k, rho] = sla.expm(1j * s * eps * T[a]) @ U[k, rho]
                d.append(O.gauge_action(DIMS, Up, BETA, c))
            worst = max(worst, abs(-(d[0] - d[1]) / (2 * eps) - f[k, rho, a]))
    return worst / max(np.abs(f).max(), 1e-300)


def _fd_wilson(U, X, Y, links, eps=1e-5):
    h = O.wilson_hopping_force(DIMS, U, X, Y)
    worst = 0.0
    for li in links:
        k, rho = divmod(int(li), 4)
        for a in range(8):
            d = []
            for s in (1, -1):
                Up = U.copy()
                Up[k, rho] = sla.expm(1j * s * eps * T[a]) @ U[k, rho]
                d.append(2 * np.vdot(Y, O.wilson_hopping(DIMS, Up, X)).real)
            worst = max(worst, abs(-(d[0] - d[1]) / (2 * eps) - h[k, rho, a]))
    return worst / max(np.abs(h).max(), 1e-300)


def battery():
    """Names of the pins that fail (empty: all pass)."""
    failed = []
    rng = np.random.default_rng(3)
    links = synth.sample_links(4 * V, 6, seed=5)

    c = O.coefficients(0.87)
    if abs(c[1] + 0.0718213744) > 1e-9 or abs(c[2] + 0.0159501735) > 1e-9 or c[0] != 1.0:
        failed.append("coefficients at u0 = 0.87")
    if np.abs(O.coefficients(1.0) - [1.0, -0.05, 0.0]).max() > 1e-15:
        failed.append("tree-level coefficients")

    unit = np.zeros((V, 4, 3, 3), complex)
    unit[..., 0, 0] = unit[..., 1, 1] = unit[..., 2, 2] = 1
    if O.gauge_action(DIMS, unit, BETA, c) != 0.0 or np.abs(O.gauge_force(DIMS, unit, BETA, c)).max() > 1e-14:
        failed.append("unit configuration")

    th, ph = 2 * np.pi / 4, 2 * 2 * np.pi / 4
    Uf = H.abelian_flux_links(DIMS, th, ph, axes=(0, 1, 3))
    want = H.abelian_flux_class_sums(V, th, ph)
    if np.abs(O.loop_sums(DIMS, Uf) - want).max() > 1e-9 * want.max():
        failed.append("abelian flux class sums")
    if abs(O.gauge_action(DIMS, Uf, BETA, c) - BETA / 3 * (c @ want)) > 1e-9 * abs(BETA / 3 * (c @ want)):
        failed.append("abelian flux action")

    Vm = H.random_su3_numpy(rng, 4)
    Uu = np.broadcast_to(Vm, (V, 4, 3, 3)).copy()
    cm = {"plaq": c[0], "rect": c[1], "cube": c[2]}
    su = 0.0
    for cls, seq in H.read_paths():
        Pm = np.eye(3, dtype=complex)
        for st in seq:
            Pm = Pm @ (Vm[st - 1] if st > 0 else Vm[-st - 1].conj().T)
        su += cm[cls] * (3 - np.trace(Pm).real)
    su *= BETA / 3 * V
    if abs(O.gauge_action(DIMS, Uu, BETA, c) - su) > 1e-12 * abs(su):
        failed.append("uniform links against the golden loop table")

    U = O.links_from_omega(synth.omega(DIMS, 0.5, 0))
    if _fd_gauge(U, c, links) > 1e-6:
        failed.append("gauge force = -grad S")
    f = O.gauge_force(DIMS, U, BETA, c)
    fl = np.stack([O.gauge_force_link(DIMS, U, BETA, c, int(li) // 4, int(li) % 4) for li in links])
    if np.abs(fl - f.reshape(-1, 8)[links]).max() > 1e-12 * np.abs(f).max():
        failed.append("per-link force = lattice algorithm")

    for _ in range(3):
        w = rng.normal(size=8)
        if np.abs(O.exp_i_algebra(w) - sla.expm(1j * np.einsum("a,aij->ij", w, T))).max() > 1e-13:
            failed.append("exponential vs expm")
            break

    M = rng.normal(size=(24, 1, 3, 3)) + 1j * rng.normal(size=(24, 1, 3, 3))
    G = O.md_update_links(M, np.zeros((24, 1, 8)), 0.3)[:, 0]
    q, r = np.linalg.qr(np.transpose(M[:, 0, :2], (0, 2, 1)))
    d = np.diagonal(r, axis1=1, axis2=2)
    want = np.transpose(q * (d / np.abs(d))[:, None, :], (0, 2, 1))
    if (np.abs(G[:, :2] - want).max() > 1e-13
            or np.abs(np.einsum("nij,nkj->nik", G, G.conj()) - np.eye(3)).max() > 1e-13
            or np.abs(np.linalg.det(G) - 1).max() > 1e-13):
        failed.append("reunitarisation = Gram-Schmidt (QR), in SU(3)")

    p = synth.momenta(DIMS, 7)
    dt = 0.07
    U1 = O.md_update_links(U, p, dt)
    P = np.einsum("nma,aij->nmij", p, T)
    E = np.stack([[sla.expm(1j * dt * P[n, m]) for m in range(4)] for n in range(3)])
    if np.abs(U1[:3] - np.einsum("nmij,nmjk->nmik", E, U[:3])).max() > 1e-12:
        failed.append("link step = exp(i dt p.T) U")
    f0 = O.gauge_force(DIMS, U, BETA, c)
    if np.abs(O.md_update_momenta(p, f0, dt) - (p + dt * f0)).max() > 1e-14:
        failed.append("momentum step")
    if abs(O.kinetic_energy(p) - 0.5 * np.sum(p * p)) > 1e-9:
        failed.append("kinetic energy")

    g = [O.gamma(m) for m in range(1, 5)]
    for a in range(4):
        for b in range(4):
            if np.abs(g[a] @ g[b] + g[b] @ g[a] - 2 * np.eye(4) * (a == b)).max() > 0:
                failed.append("Clifford algebra")
                break
    X = _cplx(synth.spinor(DIMS, 11))
    Y = _cplx(synth.spinor(DIMS, 12))
    k = np.array([1, 1, 2, 1])
    pw = 2 * np.pi * k / np.array(DIMS)
    phase = np.exp(1j * H.site_coords(DIMS) @ pw)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    M = sum(2 * np.cos(pw[m]) * np.eye(4) - 2j * np.sin(pw[m]) * g[m] for m in range(4))
    if np.abs(O.wilson_hopping(DIMS, unit, phase[:, None, None] * u[None])
              - phase[:, None, None] * (M @ u)[None]).max() > 1e-12:
        failed.append("hopping operator plane waves")
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    lhs = np.vdot(Y, O.wilson_hopping(DIMS, U, X))
    rhs = np.conj(np.vdot(X, g5 @ O.wilson_hopping(DIMS, U, np.einsum("ab,nbc->nac", g5, Y))))
    if abs(lhs - rhs) > 1e-12 * abs(lhs):
        failed.append("gamma_5 hermiticity")
    if _fd_wilson(U, X, Y, links) > 1e-7:
        failed.append("hopping force = -grad 2 Re Y^dag calD X")
    return failed


MUTATIONS = [
    ("c_rect: sign of the alpha_s term",
     "c[1] = -(1.0 + 0.4805 * alpha_s) / (20.0 * u0 * u0);",
     "c[1] = -(1.0 - 0.4805 * alpha_s) / (20.0 * u0 * u0);"),
    ("c_cube: the factor 2 dropped",
     "c[2] = -(2.0 * 0.03325 * alpha_s) / (u0 * u0);",
     "c[2] = -(0.03325 * alpha_s) / (u0 * u0);"),
    ("cube loop: last two steps swapped",
     "path q = {6, {mu, s * nu, t * rho, -mu, -s * nu, -t * rho}, CLS_CUBE};",
     "path q = {6, {mu, s * nu, t * rho, -mu, -t * rho, -s * nu}, CLS_CUBE};"),
    ("rectangle loop: last two steps swapped (a plaquette with a backtrack)",
     "path q = {6, {mu, mu, nu, -mu, -mu, -nu}, CLS_RECT};",
     "path q = {6, {mu, mu, nu, -mu, -nu, -mu}, CLS_RECT};"),
    ("backward staple: dagger dropped",
     "for (int i = l - 1; i >= 0; --i) m = mul(m, dagger(link_dir(f, pos[i], p->d[i])));",
     "for (int i = l - 1; i >= 0; --i) m = mul(m, link_dir(f, pos[i], p->d[i]));"),
    ("forward staple: factors in the wrong order",
     "for (int i = l + 1; i < L; ++i) m = mul(m, link_dir(f, pos[i], p->d[i]));",
     "for (int i = l + 1; i < L; ++i) m = mul(link_dir(f, pos[i], p->d[i]), m);"),
    ("projection: beta/3 instead of beta/6",
     "mat3 h = scale(I * beta / 6.0, traceless_antihermitian(mul(u, t)));",
     "mat3 h = scale(I * beta / 3.0, traceless_antihermitian(mul(u, t)));"),
    ("projection: t U instead of U t",
     "mat3 h = scale(I * beta / 6.0, traceless_antihermitian(mul(u, t)));",
     "mat3 h = scale(I * beta / 6.0, traceless_antihermitian(mul(t, u)));"),
    ("TA: Hermitian instead of anti-Hermitian part",
     "mat3 d = add(b, scale(-1.0, dagger(b)));",
     "mat3 d = add(b, dagger(b));"),
    ("generator lambda_2: sign",
     "case 1: l.m[0][1] = -I; l.m[1][0] = I; break;",
     "case 1: l.m[0][1] = I; l.m[1][0] = -I; break;"),
    ("exponential: series cut at 2 terms",
     "for (int k = 1; k <= 25; ++k) {",
     "for (int k = 1; k <= 2; ++k) {"),
    ("link step: exponential on the right",
     "u = reunitarise(mul(exp_i_algebra(w), u));",
     "u = reunitarise(mul(u, exp_i_algebra(w)));"),
    ("Gram-Schmidt: projection conjugated",
     "for (int j = 0; j < 3; ++j) proj += conj(u.m[0][j]) * u.m[1][j];",
     "for (int j = 0; j < 3; ++j) proj += u.m[0][j] * conj(u.m[1][j]);"),
    ("Gram-Schmidt: projection added instead of subtracted",
     "for (int j = 0; j < 3; ++j) u.m[1][j] -= proj * u.m[0][j];",
     "for (int j = 0; j < 3; ++j) u.m[1][j] += proj * u.m[0][j];"),
    ("Gram-Schmidt: row 1 not normalised",
     "n1 = 1.0 / sqrt(n1);",
     "n1 = 1.0;"),
    ("Gram-Schmidt: row 0 not normalised",
     "n0 = 1.0 / sqrt(n0);",
     "n0 = 1.0;"),
    ("Gram-Schmidt: row 2 without the complex conjugate",
     "u.m[2][1] = conj(u.m[0][2] * u.m[1][0] - u.m[0][0] * u.m[1][2]);",
     "u.m[2][1] = u.m[0][2] * u.m[1][0] - u.m[0][0] * u.m[1][2];"),
    ("momentum step: sign",
     "for (long i = 0; i < 8 * nlinks; ++i) p[i] += dt * f[i];",
     "for (long i = 0; i < 8 * nlinks; ++i) p[i] -= dt * f[i];"),
    ("kinetic energy: factor 1/2 dropped",
     "kadd(&k, 0.5 * p[i] * p[i]);",
     "kadd(&k, p[i] * p[i]);"),
    ("action: beta/6 instead of beta/3",
     "return beta / 3.0 * (k.s + k.c);",
     "return beta / 6.0 * (k.s + k.c);"),
    ("site index: t fastest instead of x",
     "for (int i = 3; i >= 0; --i) n = n * g->L[i] + x[i];",
     "for (int i = 0; i < 4; ++i) n = n * g->L[i] + x[i];"),
    ("gamma_3: two entries with the wrong sign",
     "case 3: g[0][2] = I;  g[1][3] = -I; g[2][0] = -I; g[3][1] = I;  break;",
     "case 3: g[0][2] = I;  g[1][3] = I; g[2][0] = -I; g[3][1] = -I;  break;"),
    ("hopping: (1 - gamma) on the backward hop",
     "spinor bw = spin_project(mu, +1.0, &xb);",
     "spinor bw = spin_project(mu, -1.0, &xb);"),
    ("hopping: backward link without dagger",
     "bw = colour_mul(link_dir(f, n, -mu), &bw);",
     "bw = colour_mul(get_link(f, step(&f->g, n, -mu), mu), &bw);"),
    ("hopping force: (1 + gamma) in B",
     "spinor z = spin_project(rho, -1.0, &ux);",
     "spinor z = spin_project(rho, +1.0, &ux);"),
    ("hopping force: B transposed",
     "B.m[b][a] += z.s[al][b] * conj(yk.s[al][a]);",
     "B.m[b][a] += z.s[al][a] * conj(yk.s[al][b]);"),
    ("hopping force: U instead of U^dag in C",
     "s += conj(yp.s[be][c]) * pg * conj(u.m[a][c]);",
     "s += conj(yp.s[be][c]) * pg * u.m[c][a];"),
    ("hopping force: complex conjugate dropped",
     "out[i] = coef * (-(tr + conj(tr)));",
     "out[i] = coef * (-(tr));"),
    ("hopping force: Y at k instead of k + rho",
     "spinor xp = get_spinor(X, kp), yp = get_spinor(Y, kp);",
     "spinor xp = get_spinor(X, kp), yp = get_spinor(Y, k);"),
]


def test_unmutated_oracle_passes_the_battery():
    assert battery() == []


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = O.build_variant(src.replace(old, new), str(tmp_path / "liboracle_mutant.so"))
    with O.using_library(path):
        failed = battery()
    assert failed, f"planted mistake not caught: {name}"
