"""Batched MAID (adp_batch_*): many problems of uneven image and kernel size in
one cooperative launch, each on its own group of CTAs.  A problem's program
in a batch is the same as in a launch of its own, with fewer CTAs, so only the
order of the reduction sums differs: FP64 results must agree to rounding,
FP32 results to the FP32 parity tolerances.  The device-resident run (a CUDA
graph of several batched steps, state kept on the device) must reproduce the
same steps taken one call at a time.
"""
import numpy as np
import pytest
import torch

from paper_2502_09758_gb300 import adp, synth
from gpu_common import need_gpu, psnr, rel

pytestmark = pytest.mark.gpu

SHAPES = [(1, 40, 36, 5), (3, 64, 48, 7), (2, 33, 70, 9), (1, 96, 96, 15), (3, 50, 50, 3)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def make_set(prec, shapes=SHAPES):
    dt = torch.float32 if prec == adp.ADP_F32 else torch.float64
    out = []
    for k, (C, H, W, K) in enumerate(shapes):
        s = max(K / 5.0, 0.6)
        inst = synth.make_instance(f"b{k}", C, H, W, synth.gaussian_kernel(K, 1.2 * s), synth.gaussian_kernel(K, s),
                                   0.01, 10 + k)
        y = torch.tensor(inst.y, dtype=dt, device="cuda")
        a = torch.tensor(inst.a, dtype=dt, device="cuda")
        prob = adp.Problem(adp.Params(C, H, W, K, prec=prec), y, a)
        out.append((inst, prob, y, a))
    return out


def start(problems, **kw):
    states, bs, xs, qs = [], [], [], []
    for inst, prob, y, a in problems:
        states.append(prob.maid_init(eps=kw.get("eps", 1e-4), delta=kw.get("eps", 1e-4), step=kw.get("step", 1e-3),
                                     eps_stop=kw.get("eps_stop", 0.0)))
        bs.append(a.clone())
        xs.append(y.clone())
        qs.append(torch.zeros_like(y))
    return states, bs, xs, qs


def single_steps(problems, nsteps, stop_on_fail=True, **kw):
    states, bs, xs, qs = start(problems, **kw)
    logs = [[] for _ in problems]
    for i, (inst, prob, y, a) in enumerate(problems):
        for _ in range(nsteps):
            ok = prob.maid_step(states[i], bs[i], xs[i], qs[i])
            logs[i].append((ok, states[i].trials, states[i].ll_iters, states[i].cg_iters))
            if states[i].stopped or (stop_on_fail and not ok):
                break
    return states, bs, xs, logs


def n(t):
    return t.detach().double().cpu().numpy()


def test_batched_step_matches_single_launches_fp64():
    probs = make_set(adp.ADP_F64)
    s1, b1, x1, _ = single_steps(probs, 1)
    batch = adp.Batch([p for _, p, _, _ in probs])
    sizes = batch.group_sizes()
    assert all(g >= 1 for g in sizes) and sum(sizes) <= 152 * 4
    s2, b2, x2, q2 = start(probs)
    acc = batch.maid_step(s2, b2, x2, q2)
    for i in range(len(probs)):
        assert acc[i] == bool(s1[i].accepted)
        assert s2[i].trials == s1[i].trials
        assert abs(s2[i].ll_iters - s1[i].ll_iters) <= 1 and abs(s2[i].cg_iters - s1[i].cg_iters) <= 1
        assert s2[i].eps == s1[i].eps and s2[i].step == s1[i].step
        assert rel(n(b2[i]), n(b1[i])) <= 1e-9
        assert rel(n(x2[i]), n(x1[i])) <= 1e-8
    batch.close()


def test_batched_steps_fp32_with_rebalancing():
    probs = make_set(adp.ADP_F32)
    s1, b1, x1, _ = single_steps(probs, 3, stop_on_fail=False, eps=1e-3, step=1e-2)   # as the batch: 3 steps each
    batch = adp.Batch([p for _, p, _, _ in probs])
    s2, b2, x2, q2 = start(probs, eps=1e-3, step=1e-2)
    sizes0 = batch.group_sizes()
    for _ in range(3):
        batch.maid_step(s2, b2, x2, q2)
    sizes1 = batch.group_sizes()
    assert sum(sizes1) <= sum(sizes0) + len(probs)
    for i, (inst, _, _, _) in enumerate(probs):
        assert s2[i].k == s1[i].k
        assert rel(n(b2[i]), n(b1[i])) <= 1e-4
        assert rel(n(x2[i]), n(x1[i])) <= 1e-4
        assert abs(psnr(n(x2[i]), inst.x_true) - psnr(n(x1[i]), inst.x_true)) <= 0.05
    batch.close()


def test_graph_run_matches_step_by_step_fp64():
    probs = make_set(adp.ADP_F64, SHAPES[:3])
    nsteps = 4
    s1, b1, x1, logs = single_steps(probs, nsteps)
    batch = adp.Batch([p for _, p, _, _ in probs])
    s2, b2, x2, q2 = start(probs)
    totals = batch.maid_run_graph(s2, b2, x2, q2, nsteps)
    for i in range(len(probs)):
        assert s2[i].k == s1[i].k
        assert s2[i].eps == pytest.approx(s1[i].eps, rel=1e-12)
        assert rel(n(b2[i]), n(b1[i])) <= 1e-9
        assert rel(n(x2[i]), n(x1[i])) <= 1e-8
        fused, passes, ups, accepted = totals[i]
        assert ups == len(logs[i]) and accepted == sum(1 for l in logs[i] if l[0])
        assert abs(fused - sum(l[2] + l[3] for l in logs[i])) <= 2 * len(logs[i])
        assert passes > 0
    batch.close()


def test_graph_run_stops_each_problem_at_its_own_stop_rule():
    probs = make_set(adp.ADP_F64, SHAPES[:2])
    batch = adp.Batch([p for _, p, _, _ in probs])
    s, b, x, q = start(probs, eps=1e-4)
    s[1].eps_stop = 1e-4          # problem 1 has already reached its tolerance: no step runs
    b1_before = b[1].clone()
    totals = batch.maid_run_graph(s, b, x, q, 3)
    assert totals[1][2] == 0 and bool(s[1].stopped)
    assert torch.equal(b[1], b1_before)
    assert totals[0][2] == 3 and not s[0].stopped
    batch.close()


def test_batch_rejects_mixed_precisions():
    p32 = make_set(adp.ADP_F32, SHAPES[:1])[0][1]
    p64 = make_set(adp.ADP_F64, SHAPES[:1])[0][1]
    with pytest.raises(adp.AdpError) as e:
        adp.Batch([p32, p64])
    assert e.value.status == adp.ADP_EINVAL
