"""Checkpoint/resume of the MAID state and the per-iteration log (host side;
the bit-for-bit resume on the GPU is in test_gpu_checkpoint.py)."""
import json

import numpy as np
import torch

from paper_2502_09758_gb300 import adp, runtime


def _state():
    s = adp.adp_maid_state()
    for i, (name, typ) in enumerate(adp.adp_maid_state._fields_):
        setattr(s, name, (i + 1) * (0.1 + 1e-13) if typ is adp.ct.c_double else i + 1)
    return s


def test_checkpoint_round_trip_is_exact(tmp_path):
    s = _state()
    rng = np.random.default_rng(0)
    b = torch.from_numpy(rng.standard_normal((3, 5, 5)).astype(np.float32))
    x = torch.from_numpy(rng.standard_normal((3, 8, 6)))
    q = torch.from_numpy(rng.standard_normal((3, 8, 6)))
    p = tmp_path / "ck.npz"
    runtime.save_maid_checkpoint(p, s, b, x, q, workload="t", seed=3)
    s2, b2, x2, q2, meta = runtime.load_maid_checkpoint(p, device="cpu")
    for name, _ in adp.adp_maid_state._fields_:
        assert getattr(s2, name) == getattr(s, name), name
    assert b2.dtype == torch.float32 and x2.dtype == torch.float64
    assert torch.equal(b2, b) and torch.equal(x2, x) and torch.equal(q2, q)
    assert meta == {"workload": "t", "seed": 3}


def test_maid_log_records(tmp_path):
    s = _state()
    x_true = np.zeros((1, 2, 2))
    log = runtime.MaidLog(tmp_path / "run.jsonl", x_true=x_true)
    rec = log.record(s, True, 1.5, x=torch.full((1, 2, 2), 0.1, dtype=torch.float64))
    log.record(s, False, 2.0)
    log.close()
    lines = [json.loads(l) for l in open(tmp_path / "run.jsonl")]
    assert len(lines) == 2 and lines[0] == rec
    assert lines[0]["k"] == s.k and lines[0]["accepted"] and not lines[1]["accepted"]
    assert abs(lines[0]["psnr_x"] - 20.0) < 1e-9           # mse 0.01 against peak 1
