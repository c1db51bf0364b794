"""Molecular-dynamics trajectories of the Symanzik gauge action (the HMC use
of the force, paper Sec. II) on liblqcd's kernels.

Integrators (the paper names none; both are standard symmetric splittings):
  leapfrog   p(dt/2) [U(dt) p(dt)]^(n-1) U(dt) p(dt/2)            n+1 forces
  omelyan    2nd-order minimum-norm (Omelyan, Mryglod & Folk, Comput. Phys.
             Commun. 151 (2003) 272), lambda = 0.1931833275037836:
             p(l dt) U(dt/2) p((1-2l) dt) U(dt/2) p(l dt) per step,   2n+1 forces
Every momentum kick is one lqcd_md_force_step (force and p += c f in one
pass, the force never stored); every drift one lqcd_md_update_links.

The Hamiltonian H = K + S is formed in FP64: K = sum p^2/2 from the stored
momenta, S from the action kernel, for FP32-stored links either in FP32
arithmetic or (``action_precision="f64"``) in FP64 arithmetic on the same
stored values.  A whole trajectory can be captured as one CUDA graph.

A full HMC run (``run_hmc``) adds to each trajectory the momentum refresh
(Gaussian momenta drawn on the GPU from a counter-based stream), the
Metropolis test accept with probability min(1, exp(-dH)) (the links are
restored on rejection), an optional FP64 reunitarisation of the links every
N trajectories, and a record per trajectory (dH, acceptance, action,
plaquette, the FP64 unitarity deviation of the links); ``save_checkpoint`` / ``load_checkpoint`` store and restore the
state so that a resumed run continues bit for bit.

``python -m paper_1808_02281_gb300.hmc`` runs the dH-versus-dt study;
``--same-start`` runs it from one thermalised start shared by the FP32 and
FP64 trajectories (same values), so that their dH difference is the error of
the FP32 arithmetic alone; ``--hmc N`` runs N HMC trajectories instead (JSON
line per trajectory).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import struct
import time

import torch

from . import lqcd, synth

OMELYAN_LAMBDA = 0.1931833275037836


@dataclasses.dataclass
class MDState:
    lat: lqcd.Lattice
    links: torch.Tensor
    mom: torch.Tensor
    workspace: torch.Tensor

    @classmethod
    def create(cls, lat: lqcd.Lattice, links: torch.Tensor, mom: torch.Tensor) -> "MDState":
        return cls(lat, links, mom, lqcd.make_workspace(lat, links.device))

    def clone(self) -> "MDState":
        return MDState(self.lat, self.links.clone(), self.mom.clone(), self.workspace)


def kick(st: MDState, coef: float) -> None:
    """p += coef * f(U)."""
    lqcd.md_force_step(st.lat, st.links, mom=st.mom, dt=coef, workspace=st.workspace)


def drift(st: MDState, coef: float) -> None:
    """U <- exp(i coef p.T) U."""
    lqcd.md_update_links(st.lat, st.links, st.mom, coef)


def leapfrog(st: MDState, dt: float, nsteps: int) -> None:
    kick(st, dt / 2)
    for i in range(nsteps):
        drift(st, dt)
        kick(st, dt if i < nsteps - 1 else dt / 2)


def omelyan(st: MDState, dt: float, nsteps: int, lam: float = OMELYAN_LAMBDA) -> None:
    kick(st, lam * dt)
    for i in range(nsteps):
        drift(st, dt / 2)
        kick(st, (1 - 2 * lam) * dt)
        drift(st, dt / 2)
        kick(st, 2 * lam * dt if i < nsteps - 1 else lam * dt)


INTEGRATORS = {"leapfrog": leapfrog, "omelyan": omelyan}


def force_evaluations(integrator: str, nsteps: int) -> int:
    return nsteps + 1 if integrator == "leapfrog" else 2 * nsteps + 1


def hamiltonian(st: MDState, action_precision: str | None = None) -> float:
    """H = K + S in FP64 (host float; synchronises)."""
    lat = st.lat
    K = lqcd.kinetic_energy(lat, st.mom, workspace=st.workspace)
    prec = action_precision or lat.precision
    if prec == lat.precision:
        S = lqcd.gauge_action(lat, st.links, workspace=st.workspace)
    else:
        lat2 = lat.with_(precision=prec)
        S = lqcd.gauge_action(lat2, lqcd.convert_links(lat, st.links, prec))
    return float(K.item()) + float(S.item())


def trajectory(st: MDState, tau: float, dt: float, integrator: str = "omelyan",
               action_precision: str | None = None) -> float:
    """Integrate one trajectory of length tau in place; return dH."""
    nsteps = max(1, int(round(tau / dt)))
    H0 = hamiltonian(st, action_precision)
    INTEGRATORS[integrator](st, tau / nsteps, nsteps)
    return hamiltonian(st, action_precision) - H0


class GraphTrajectory:
    """One trajectory (fixed dt and number of steps) captured as a CUDA graph
    on the tensors of ``st``; replay() integrates them in place."""

    def __init__(self, st: MDState, dt: float, nsteps: int, integrator: str = "omelyan"):
        self.st = st
        run = INTEGRATORS[integrator]
        # first launches (one-time device set-up of the library) outside capture
        scratch = st.clone()
        run(scratch, dt, 1)
        torch.cuda.synchronize()
        del scratch
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            run(st, dt, nsteps)

    def replay(self) -> None:
        self.graph.replay()


@dataclasses.dataclass
class BatchState:
    """Many lattices (uneven extents, one precision and action) advanced
    together: every kick and drift is one launch per pass for all of them."""
    params: lqcd.Lattice
    dims: list
    links: list
    mom: list
    workspace: torch.Tensor

    @classmethod
    def create(cls, params: lqcd.Lattice, dims, links, mom) -> "BatchState":
        dims = [tuple(d) for d in dims]
        return cls(params, dims, list(links), list(mom),
                   lqcd.make_workspace_batched(params, dims, links[0].device))

    def clone(self) -> "BatchState":
        return BatchState(self.params, self.dims, [u.clone() for u in self.links],
                          [p.clone() for p in self.mom], self.workspace)


def batch_kick(bs: BatchState, coef: float) -> None:
    lqcd.md_force_step_batched(bs.params, bs.dims, bs.links, mom=bs.mom, dt=coef,
                               workspace=bs.workspace)


def batch_drift(bs: BatchState, coef: float) -> None:
    lqcd.md_update_links_batched(bs.params, bs.dims, bs.links, bs.mom, coef)


def batch_leapfrog(bs: BatchState, dt: float, nsteps: int) -> None:
    batch_kick(bs, dt / 2)
    for i in range(nsteps):
        batch_drift(bs, dt)
        batch_kick(bs, dt if i < nsteps - 1 else dt / 2)


def batch_omelyan(bs: BatchState, dt: float, nsteps: int, lam: float = OMELYAN_LAMBDA) -> None:
    batch_kick(bs, lam * dt)
    for i in range(nsteps):
        batch_drift(bs, dt / 2)
        batch_kick(bs, (1 - 2 * lam) * dt)
        batch_drift(bs, dt / 2)
        batch_kick(bs, 2 * lam * dt if i < nsteps - 1 else lam * dt)


BATCH_INTEGRATORS = {"leapfrog": batch_leapfrog, "omelyan": batch_omelyan}


class GraphBatchTrajectory:
    """A batch trajectory captured as one CUDA graph (replay() advances the
    tensors of ``bs`` in place)."""

    def __init__(self, bs: BatchState, dt: float, nsteps: int, integrator: str = "leapfrog"):
        self.bs = bs
        run = BATCH_INTEGRATORS[integrator]
        scratch = bs.clone()
        run(scratch, dt, 1)
        torch.cuda.synchronize()
        del scratch
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            run(bs, dt, nsteps)

    def replay(self) -> None:
        self.graph.replay()


def initial_batch(dims_list, precision: str, sigma: float = 0.3, u0: float = 0.87,
                  beta: float = 6.0, seed: int = 0, device="cuda") -> BatchState:
    """One seeded lattice and momentum field per entry (seed + 2 * index)."""
    params = lqcd.Lattice.symanzik(dims_list[0], beta, u0, precision)
    links, mom = [], []
    for c, dims in enumerate(dims_list):
        lat = params.with_(dims=tuple(dims))
        links.append(lqcd.links_from_omega(
            lat, lqcd.algebra_to_device(lat, synth.omega(dims, sigma, seed + 2 * c), device)))
        mom.append(lqcd.algebra_to_device(lat, synth.momenta(dims, seed + 2 * c + 1), device))
    return BatchState.create(params, dims_list, links, mom)


def initial_state(dims, precision: str, sigma: float = 0.3, u0: float = 0.87,
                  beta: float = 6.0, seed: int = 0, device="cuda") -> MDState:
    """Links exp(i w.T), w ~ N(0, sigma^2) and Gaussian momenta, both from the
    seeded generator (the same draws for either precision)."""
    lat = lqcd.Lattice.symanzik(dims, beta, u0, precision)
    links = lqcd.links_from_omega(lat, lqcd.algebra_to_device(lat, synth.omega(dims, sigma, seed), device))
    mom = lqcd.algebra_to_device(lat, synth.momenta(dims, seed + 1), device)
    return MDState.create(lat, links, mom)


def dh_study(dims, tau: float, dts, integrator: str, precisions, seed: int = 0):
    """dH against dt for each precision; FP32 runs also report dH with the
    FP64 action of their stored links.  Yields one dict per (precision, dt)."""
    for prec in precisions:
        for dt in dts:
            st = initial_state(dims, prec, seed=seed)
            nsteps = max(1, int(round(tau / dt)))
            H0 = hamiltonian(st)
            H0_64 = hamiltonian(st, "f64") if prec == "f32" else H0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            INTEGRATORS[integrator](st, tau / nsteps, nsteps)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            rec = {"precision": prec, "dims": list(dims), "tau": tau, "dt": tau / nsteps,
                   "nsteps": nsteps, "integrator": integrator, "dH": hamiltonian(st) - H0,
                   "seconds": secs, "forces": force_evaluations(integrator, nsteps)}
            if prec == "f32":
                rec["dH_f64_action"] = hamiltonian(st, "f64") - H0_64
            yield rec
            del st
            torch.cuda.empty_cache()


def thermalise(st: MDState, n: int, tau: float, dt: float, integrator: str = "omelyan",
               seed: int = 0):
    """n molecular-dynamics trajectories with a momentum refresh before each
    and no accept/reject step: moves a synthetic start towards the typical
    configurations of the action, where the force is that of an equilibrium
    ensemble rather than of random links.  Momenta of trajectory t come from
    the counter-based stream word t of ``seed``.  Yields the trajectory's
    dH (in the state's own precision), then S and the plaquette after it."""
    nsteps = max(1, int(round(tau / dt)))
    for t in range(n):
        lqcd.gaussian_momenta(st.lat, _stream_word(seed, t), out=st.mom)
        H0 = hamiltonian(st)
        INTEGRATORS[integrator](st, tau / nsteps, nsteps)
        H1 = hamiltonian(st)
        S = float(lqcd.gauge_action(st.lat, st.links, workspace=st.workspace).item())
        yield {"trajectory": t, "dH": H1 - H0, "action": S, "plaquette": plaquette(st)}


def same_start_pair(links32: torch.Tensor, lat32: lqcd.Lattice, momentum_stream: int):
    """An FP32 state and an FP64 state that hold the same values: the FP32
    links and GPU-drawn FP32 momenta, and both promoted exactly to FP64."""
    mom32 = lqcd.gaussian_momenta(lat32, momentum_stream, device=links32.device)
    a = MDState.create(lat32, links32.clone(), mom32)
    lat64 = lat32.with_(precision="f64")
    b = MDState.create(lat64, lqcd.convert_links(lat32, links32, "f64"),
                       lqcd.convert_algebra(lat32, mom32, "f64"))
    return a, b


def same_start_study(dims, tau: float, dts, integrator: str = "omelyan", seed: int = 0,
                     n_therm: int = 100, therm_tau: float = 0.5, therm_dt: float = 0.025,
                     sigma: float = 0.3, u0: float = 0.87, beta: float = 6.0):
    """dH of FP32 and FP64 trajectories that start from the same state.

    The synthetic start (links exp(i w.T), w ~ N(0, sigma^2)) is first
    thermalised in FP32 (n_therm trajectories, see thermalise()) and
    reunitarised in FP64 (rounded to FP32); then for
    every dt one FP32 trajectory runs on the thermalised links with FP32
    momenta drawn on the GPU, and one FP64 trajectory on the same values
    promoted exactly.  H = K + S in FP64 in both (the FP32 run's action in
    FP64 arithmetic of its stored links), so H0 is the same number in both
    runs and dH_f32 - dH_f64 is the error of the FP32 arithmetic alone.
    Yields the thermalisation records, then one record per dt."""
    st = initial_state(dims, "f32", sigma, u0, beta, seed)
    for rec in thermalise(st, n_therm, therm_tau, therm_dt, integrator, seed + 101):
        rec["phase"] = "thermalise"
        yield rec
    # start from links that are in SU(3) to FP64 accuracy before rounding
    # (Gram-Schmidt in FP64, rounded to FP32), so that neither run starts
    # with a systematic departure that only the FP64 run would remove
    lqcd.reunitarise_links(st.lat, st.links)
    links32 = st.links.clone()
    lat32 = st.lat
    del st
    torch.cuda.empty_cache()
    for dt in dts:
        # the same momenta for every dt, so that dH(dt) follows one trajectory
        a, b = same_start_pair(links32, lat32, _stream_word(seed + 202, 0))
        nsteps = max(1, int(round(tau / dt)))
        rec = {"phase": "study", "dims": list(dims), "tau": tau, "dt": tau / nsteps, "nsteps": nsteps,
               "integrator": integrator, "forces": force_evaluations(integrator, nsteps)}
        H0a, H0b = hamiltonian(a, "f64"), hamiltonian(b)
        H0a_own = hamiltonian(a)
        rec["H0"] = H0b
        rec["H0_equal"] = H0a == H0b
        for name, stt in (("f32", a), ("f64", b)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            INTEGRATORS[integrator](stt, tau / nsteps, nsteps)
            torch.cuda.synchronize()
            rec[f"seconds_{name}"] = time.perf_counter() - t0
        rec["dH_f32"] = hamiltonian(a, "f64") - H0a
        rec["dH_f32_f32action"] = hamiltonian(a) - H0a_own
        rec["dH_f64"] = hamiltonian(b) - H0b
        rec["abs_diff"] = abs(rec["dH_f32"] - rec["dH_f64"])
        yield rec
        del a, b
        torch.cuda.empty_cache()


# ------------------------------------------------------------- HMC runs

def plaquette(st: MDState) -> float:
    """Average Re tr P / 3 over the 6V plaquettes, from the action kernel
    with Wilson coefficients: S_W = (beta/3) sum (3 - Re tr P)."""
    lat = st.lat.with_(c_plaq=1.0, c_rect=0.0, c_cube=0.0)
    S_w = float(lqcd.gauge_action(lat, st.links, workspace=st.workspace).item())
    return 1.0 - S_w / (6.0 * lat.beta * lat.V)


@dataclasses.dataclass
class HMCConfig:
    tau: float = 1.0
    dt: float = 0.05
    integrator: str = "omelyan"
    seed: int = 1
    action_precision: str | None = None   # "f64" for FP32 runs: Metropolis on the FP64 action
    reunitarise_every: int = 0            # > 0: FP64 Gram-Schmidt of the links every N trajectories


def _stream_word(seed: int, i: int) -> int:
    return int(synth.words(seed, i, 1)[0])


def momentum_seed(cfg: HMCConfig, trajectory: int) -> int:
    """Generator stream of the momenta of trajectory t: word t of stream seed."""
    return _stream_word(cfg.seed, trajectory)


def metropolis_uniform(cfg: HMCConfig, trajectory: int) -> float:
    """Uniform in [0, 1) of trajectory t: word t of stream seed + 1, top 53 bits."""
    return (_stream_word(cfg.seed + 1, trajectory) >> 11) * 2.0 ** -53


def hmc_trajectory(st: MDState, cfg: HMCConfig, trajectory: int) -> dict:
    """One HMC trajectory in place: refresh, integrate, Metropolis test."""
    t0 = time.perf_counter()
    lqcd.gaussian_momenta(st.lat, momentum_seed(cfg, trajectory), out=st.mom)
    saved = st.links.clone()
    nsteps = max(1, int(round(cfg.tau / cfg.dt)))
    H0 = hamiltonian(st, cfg.action_precision)
    INTEGRATORS[cfg.integrator](st, cfg.tau / nsteps, nsteps)
    H1 = hamiltonian(st, cfg.action_precision)
    dH = H1 - H0
    accept = metropolis_uniform(cfg, trajectory) < math.exp(min(0.0, -dH))
    if not accept:
        st.links.copy_(saved)
    del saved
    if cfg.reunitarise_every and (trajectory + 1) % cfg.reunitarise_every == 0:
        lqcd.reunitarise_links(st.lat, st.links)
    S = float(lqcd.gauge_action(st.lat, st.links, workspace=st.workspace).item())
    unitarity = float(lqcd.unitarity_deviation(st.lat, st.links, workspace=st.workspace).item())
    return {"trajectory": trajectory, "dH": dH, "accepted": bool(accept), "action": S,
            "plaquette": plaquette(st), "unitarity": unitarity, "nsteps": nsteps,
            "forces": force_evaluations(cfg.integrator, nsteps),
            "seconds": time.perf_counter() - t0}


def run_hmc(st: MDState, cfg: HMCConfig, n: int, start: int = 0, checkpoint: str | None = None,
            every: int = 0):
    """Trajectories start .. start+n-1 (yields one record each); with a
    checkpoint path, the state is saved after every `every` trajectories
    (and after the last)."""
    accepted = 0
    for i in range(n):
        t = start + i
        rec = hmc_trajectory(st, cfg, t)
        accepted += rec["accepted"]
        rec["acceptance"] = accepted / (i + 1)
        if checkpoint and ((every and (i + 1) % every == 0) or i == n - 1):
            save_checkpoint(checkpoint, st, cfg, next_trajectory=t + 1)
        yield rec


def batch_hamiltonians(bs: BatchState, action_precision: str | None = None) -> list:
    """H = K + S (FP64) of every lattice of the batch."""
    out = []
    for c, d in enumerate(bs.dims):
        lat = bs.params.with_(dims=d)
        st = MDState(lat, bs.links[c], bs.mom[c], bs.workspace)
        out.append(hamiltonian(st, action_precision))
    return out


def lattice_config(cfg: HMCConfig, c: int) -> HMCConfig:
    """Settings of lattice c of a batch run: its own generator streams
    (seed + 2c), so that lattice c of a batch run equals a single-lattice run
    with these settings."""
    return dataclasses.replace(cfg, seed=cfg.seed + 2 * c)


def batch_hmc_trajectory(bs: BatchState, cfg: HMCConfig, trajectory: int) -> list:
    """One HMC trajectory of every lattice of the batch: per-lattice
    momentum refresh, one batched integration (one launch per pass for all
    lattices), per-lattice Metropolis test and restore.  One record per
    lattice."""
    t0 = time.perf_counter()
    cfgs = [lattice_config(cfg, c) for c in range(len(bs.dims))]
    for c, d in enumerate(bs.dims):
        lqcd.gaussian_momenta(bs.params.with_(dims=d), momentum_seed(cfgs[c], trajectory),
                              out=bs.mom[c])
    saved = [u.clone() for u in bs.links]
    nsteps = max(1, int(round(cfg.tau / cfg.dt)))
    H0 = batch_hamiltonians(bs, cfg.action_precision)
    BATCH_INTEGRATORS[cfg.integrator](bs, cfg.tau / nsteps, nsteps)
    H1 = batch_hamiltonians(bs, cfg.action_precision)
    recs = []
    for c, d in enumerate(bs.dims):
        dH = H1[c] - H0[c]
        accept = metropolis_uniform(cfgs[c], trajectory) < math.exp(min(0.0, -dH))
        if not accept:
            bs.links[c].copy_(saved[c])
        recs.append({"trajectory": trajectory, "lattice": c, "dims": list(d), "dH": dH,
                     "accepted": bool(accept), "nsteps": nsteps})
    del saved
    secs = time.perf_counter() - t0
    for r in recs:
        r["seconds"] = secs
    return recs


def run_hmc_batch(bs: BatchState, cfg: HMCConfig, n: int, start: int = 0):
    """Trajectories start .. start+n-1 of every lattice; yields the list of
    per-lattice records of each trajectory."""
    for i in range(n):
        yield batch_hmc_trajectory(bs, cfg, start + i)


# ----------------------------------------------------------- checkpoints

_MAGIC = b"LQCDCKPT"
_VERSION = 1


def save_fields(path: str, meta: dict, fields: dict) -> None:
    """Binary checkpoint: magic, version, header length, a JSON header (meta
    and, per tensor, name, shape, dtype, byte offset and length), then the
    raw tensor bytes.  Written to a temporary file and renamed."""
    entries, blobs, off = [], [], 0
    for name, t in fields.items():
        a = t.detach().to("cpu").contiguous()
        b = a.numpy().tobytes()
        entries.append({"name": name, "shape": list(a.shape), "dtype": str(a.dtype).split(".")[-1],
                        "offset": off, "nbytes": len(b)})
        blobs.append(b)
        off += len(b)
    header = json.dumps({"meta": meta, "tensors": entries}).encode()
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as fh:
        fh.write(_MAGIC + struct.pack("<II", _VERSION, len(header)) + header)
        for b in blobs:
            fh.write(b)
    os.replace(tmp, path)


def load_fields(path: str, device="cpu"):
    """(meta, {name: tensor}) from a file written by save_fields."""
    with open(path, "rb") as fh:
        data = fh.read()
    if data[:8] != _MAGIC:
        raise ValueError(f"{path}: not a checkpoint")
    version, hlen = struct.unpack("<II", data[8:16])
    if version != _VERSION:
        raise ValueError(f"{path}: checkpoint version {version}, expected {_VERSION}")
    header = json.loads(data[16:16 + hlen])
    base = 16 + hlen
    out = {}
    for e in header["tensors"]:
        lo = base + e["offset"]
        if lo + e["nbytes"] > len(data):
            raise ValueError(f"{path}: truncated at tensor {e['name']}")
        dtype = getattr(torch, e["dtype"])
        t = torch.frombuffer(bytearray(data[lo:lo + e["nbytes"]]), dtype=dtype).reshape(e["shape"])
        out[e["name"]] = t.to(device)
    return header["meta"], out


def save_checkpoint(path: str, st: MDState, cfg: HMCConfig | None = None,
                    next_trajectory: int = 0) -> None:
    """Links, momenta, lattice parameters, HMC settings and the index of the
    next trajectory (which fixes the generator streams of the rest of the run)."""
    lat = st.lat
    meta = {"dims": list(lat.dims), "precision": lat.precision, "beta": lat.beta,
            "c_plaq": lat.c_plaq, "c_rect": lat.c_rect, "c_cube": lat.c_cube,
            "force_algo": lat.force_algo, "next_trajectory": next_trajectory,
            "hmc": dataclasses.asdict(cfg) if cfg is not None else None}
    save_fields(path, meta, {"links": st.links, "mom": st.mom})


def load_checkpoint(path: str, device="cuda"):
    """(MDState, HMCConfig or None, next trajectory) from save_checkpoint's file."""
    meta, f = load_fields(path, device)
    lat = lqcd.Lattice(tuple(meta["dims"]), meta["precision"], meta["beta"], meta["c_plaq"],
                       meta["c_rect"], meta["c_cube"], meta["force_algo"])
    cfg = HMCConfig(**meta["hmc"]) if meta.get("hmc") else None
    return MDState.create(lat, f["links"], f["mom"]), cfg, meta["next_trajectory"]


def main(argv=None):
    ap = argparse.ArgumentParser(description="dH against dt for FP32 and FP64 trajectories")
    ap.add_argument("--dims", type=int, nargs=4, default=[48, 48, 48, 96])
    ap.add_argument("--tau", type=float, default=1.0)
    ap.add_argument("--dts", type=float, nargs="+", default=[0.05, 0.025, 0.0125])
    ap.add_argument("--integrator", choices=sorted(INTEGRATORS), default="omelyan")
    ap.add_argument("--precisions", nargs="+", default=["f32", "f64"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--hmc", type=int, default=0, metavar="N",
                    help="run N HMC trajectories (first precision, first dt) instead of the study")
    ap.add_argument("--checkpoint", default=None, help="HMC: checkpoint file (resumed if present)")
    ap.add_argument("--same-start", action="store_true",
                    help="FP32 and FP64 trajectories from one thermalised start (same values)")
    ap.add_argument("--therm", type=int, default=100, help="same-start: thermalising trajectories")
    ap.add_argument("--therm-tau", type=float, default=0.5)
    ap.add_argument("--therm-dt", type=float, default=0.025)
    args = ap.parse_args(argv)
    from . import build
    build.build()
    if args.hmc:
        prec = args.precisions[0]
        cfg = HMCConfig(tau=args.tau, dt=args.dts[0], integrator=args.integrator,
                        seed=args.seed + 1, action_precision="f64" if prec == "f32" else None)
        start = 0
        if args.checkpoint and os.path.exists(args.checkpoint):
            st, saved_cfg, start = load_checkpoint(args.checkpoint)
            cfg = saved_cfg or cfg
        else:
            st = initial_state(tuple(args.dims), prec, seed=args.seed)
        for rec in run_hmc(st, cfg, args.hmc, start=start, checkpoint=args.checkpoint, every=1):
            print(json.dumps(rec), flush=True)
        return
    if args.same_start:
        for rec in same_start_study(tuple(args.dims), args.tau, args.dts, args.integrator,
                                    args.seed, args.therm, args.therm_tau, args.therm_dt):
            print(json.dumps(rec), flush=True)
        return
    for rec in dh_study(tuple(args.dims), args.tau, args.dts, args.integrator, args.precisions,
                        args.seed):
        print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main()
