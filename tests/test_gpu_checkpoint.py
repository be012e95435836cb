"""Resume from a checkpoint reproduces the next MAID step bit for bit: the
state record, b, x~ and q saved after a step, reloaded, and stepped again give
exactly what the uninterrupted run gives (the engine's reductions run in a
fixed order)."""
import pytest
import torch

from paper_2502_09758_gb300 import adp, runtime, synth
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("prec", [adp.ADP_F32, adp.ADP_F64])
def test_resume_is_bit_exact(tmp_path, prec):
    inst = synth.make_instance("ck", 3, 48, 40, synth.motion_kernel(7, 5, 30), synth.motion_kernel(7, 5, 20), 0.02, 1)
    dt = torch.float32 if prec == adp.ADP_F32 else torch.float64
    y = torch.tensor(inst.y, dtype=dt, device="cuda")
    a = torch.tensor(inst.a, dtype=dt, device="cuda")
    prob = adp.Problem(adp.Params(3, 48, 40, 7, prec=prec), y, a)
    s = prob.maid_init(eps=1e-3, delta=1e-3, step=1e-2)
    b, x, q = a.clone(), y.clone(), torch.zeros_like(y)
    prob.maid_step(s, b, x, q)
    path = tmp_path / "step1.npz"
    runtime.save_maid_checkpoint(path, s, b, x, q)
    log = runtime.MaidLog(tmp_path / "run.jsonl", x_true=inst.x_true, b_true=inst.b_true)
    for _ in range(2):
        acc = prob.maid_step(s, b, x, q)
        log.record(s, acc, 0.0, b=b, x=x)
    log.close()
    s2, b2, x2, q2, _ = runtime.load_maid_checkpoint(path)
    for _ in range(2):
        prob.maid_step(s2, b2, x2, q2)
    assert torch.equal(b2, b) and torch.equal(x2, x) and torch.equal(q2, q)
    for name in ("k", "eps", "delta", "step", "loss", "ll_iters", "cg_iters", "trials", "accepted"):
        assert getattr(s2, name) == getattr(s, name), name
    prob.close()
