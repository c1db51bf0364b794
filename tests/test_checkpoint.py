"""Checkpoint file format and the HMC generator streams, on the CPU."""
import numpy as np
import pytest
import torch

from paper_1808_02281_gb300 import hmc, synth


def test_fields_round_trip(tmp_path):
    p = str(tmp_path / "c.ckpt")
    a = torch.arange(4 * 3 * 10 * 4, dtype=torch.float32).reshape(4, 3, 10, 4) / 7
    b = torch.randn(4, 4, 10, 2, dtype=torch.float64)
    meta = {"dims": [2, 5, 1, 1], "precision": "f32", "next_trajectory": 17, "hmc": {"tau": 0.5}}
    hmc.save_fields(p, meta, {"links": a, "mom": b})
    m2, f = hmc.load_fields(p)
    assert m2 == meta
    assert f["links"].dtype == torch.float32 and torch.equal(f["links"], a)
    assert f["mom"].dtype == torch.float64 and torch.equal(f["mom"], b)


def test_fields_reject_bad_files(tmp_path):
    p = str(tmp_path / "c.ckpt")
    hmc.save_fields(p, {"x": 1}, {"t": torch.ones(100)})
    raw = open(p, "rb").read()
    bad = str(tmp_path / "bad.ckpt")
    open(bad, "wb").write(b"NOTACKPT" + raw[8:])
    with pytest.raises(ValueError, match="not a checkpoint"):
        hmc.load_fields(bad)
    open(bad, "wb").write(raw[:-8])
    with pytest.raises(ValueError, match="truncated"):
        hmc.load_fields(bad)
    open(bad, "wb").write(raw[:8] + (99).to_bytes(4, "little") + raw[12:])
    with pytest.raises(ValueError, match="version"):
        hmc.load_fields(bad)


def test_streams_are_counter_based():
    cfg = hmc.HMCConfig(seed=5)
    seeds = [hmc.momentum_seed(cfg, t) for t in range(4)]
    assert seeds == [int(w) for w in synth.words(5, 0, 4)]
    assert len(set(seeds)) == 4
    u = [hmc.metropolis_uniform(cfg, t) for t in range(1000)]
    assert all(0.0 <= x < 1.0 for x in u)
    assert abs(np.mean(u) - 0.5) < 0.05
    assert hmc.metropolis_uniform(cfg, 3) == (int(synth.words(6, 3, 1)[0]) >> 11) * 2.0 ** -53
