"""Host-side runtime around the library's calls: checkpoint/resume of the
MAID state, a per-iteration log, and the autotuners of the operator path and
of the direct path's launch shape.  Every step of the method runs in the
library (adp.py binds it); this module only stores, records and times those
calls."""
from __future__ import annotations

import numpy as np
import torch

from .adp import ADP_EINVAL, AdpError, adp_maid_state


def choose_operator_path(prob, b, x, iters=8, reps=2):
    """Autotune the operator path: time FISTA updates (adp_lower_solve with
    eps = 0, launches of ``iters`` and ``2 iters`` updates, so that the
    per-solve set-up cancels) on the direct path and, where the problem
    admits it, on the FFT path; keep the faster per update for later calls.
    Returns {"path": "direct" | "fft", "direct_ms": ..., "fft_ms": ...}
    (per update, best of ``reps``)."""
    per = {}
    for path in ("direct", "fft"):
        try:
            prob.set_fft(path == "fft")
        except AdpError as e:
            if e.status != ADP_EINVAL:
                raise
            continue
        per[path] = _fista_ms(prob, b, x, iters, reps)
    choice = min(per, key=per.get)
    prob.set_fft(choice == "fft")
    return {"path": choice, **{f"{k}_ms": v for k, v in per.items()}}


def _fista_ms(prob, b, x, iters, reps):
    """Per-update device time of FISTA (launches of iters and 2 iters updates
    with eps = 0, so that the per-solve set-up cancels), best of reps."""
    best = float("inf")
    for _ in range(reps):
        t = []
        for n in (iters, 2 * iters):
            xs = x.clone()
            prob.lower_solve(b, xs, 0.0, n)
            t.append(prob.last_kernel_ms())
        best = min(best, (t[1] - t[0]) / iters)
    return best


def launch_candidates(nstrips, nsm=152, max_ctas=512):
    """(grid, warps per CTA) shapes for the direct path's launch-shape
    autotuner: for 8, 6, 4 and 2 warps, the grid that gives every warp one
    strip (when it fits), one CTA per SM and the multiples of the SM count up
    to the strips' need.  Strips are 32 x MR pixels, dealt to warps in order,
    so a shape whose warp count divides the strips evenly leaves no warp idle
    in the last round."""
    out = []
    for nw in (8, 6, 4, 2):
        need = -(-nstrips // nw)
        grids = {min(nsm, need), min(need, max_ctas)}
        grids |= {k * nsm for k in (2, 3) if k * nsm <= min(need, max_ctas)}
        for g in sorted(grids):
            if g >= 1 and (g, nw) not in out:
                out.append((g, nw))
    return out


def choose_launch(prob, b, x, iters=8, reps=2, nsm=152):
    """Autotune the direct path's launch shape (adp_set_launch): time FISTA
    updates at the problem's own shape and at every candidate shape the device
    accepts, and keep the fastest.  Returns {"grid": ..., "nw": ...,
    "ms": {(grid, nw): per-update ms}}."""
    pr = prob.params
    mr = 8 if pr.prec == 1 else 4                    # strip rows: FP32 8, FP64 4
    nstrips = pr.C * (-(-pr.H // mr)) * (-(-pr.W // 32))
    start = (prob.grid_size(), prob.warps_per_cta())
    per = {}
    for g, nw in [start] + [c for c in launch_candidates(nstrips, nsm) if c != start]:
        try:
            prob.set_launch(g, nw)
        except AdpError as e:
            if e.status != ADP_EINVAL:
                raise
            continue
        per[(g, nw)] = _fista_ms(prob, b, x, iters, reps)
    choice = min(per, key=per.get) if per else start
    prob.set_launch(*choice)
    return {"grid": choice[0], "nw": choice[1], "ms": per}


def save_maid_checkpoint(path, state: adp_maid_state, b, x, q, **meta):
    """Everything Algorithm 2 carries from one upper iteration to the next,
    in one .npz: the state record (eps_k, delta_k, alpha_k, k, the constants
    and the last report), the kernel b, the lower-level iterate x~ and the CG
    warm start q, with their dtypes.  A later :func:`load_maid_checkpoint`
    and ``maid_step`` reproduce the next step bit for bit (the library's
    reductions run in a fixed order).  ``meta`` adds JSON-serialisable notes."""
    import json
    fields = {name: getattr(state, name) for name, _ in adp_maid_state._fields_}
    np.savez(path, state=json.dumps(fields), meta=json.dumps(meta),
             b=b.detach().cpu().numpy(), x=x.detach().cpu().numpy(), q=q.detach().cpu().numpy())


def load_maid_checkpoint(path, device="cuda"):
    """Returns (state, b, x, q, meta) from :func:`save_maid_checkpoint`, the
    images and kernel as contiguous tensors on ``device``."""
    import json
    with np.load(path) as f:
        fields = json.loads(str(f["state"]))
        meta = json.loads(str(f["meta"]))
        b, x, q = (torch.from_numpy(np.ascontiguousarray(f[k])).to(device) for k in ("b", "x", "q"))
    s = adp_maid_state()
    for name, _ in adp_maid_state._fields_:
        setattr(s, name, fields[name])
    return s, b, x, q, meta


class MaidLog:
    """One JSON record per upper iteration (k, eps_k, delta_k, alpha_k, the
    upper loss, ||z||, psi, lower-level and CG iterations, trials, accepted,
    stop rule, wall-clock ms; PSNR of x~ and b when the ground truth is given)
    appended to a .jsonl file."""

    def __init__(self, path, x_true=None, b_true=None):
        self.f = open(path, "a")
        self.x_true, self.b_true = x_true, b_true

    def record(self, state: adp_maid_state, accepted, wall_ms, b=None, x=None):
        import json
        rec = {"k": state.k, "eps": state.eps, "delta": state.delta, "step": state.step, "loss": state.loss,
               "znorm": state.znorm, "psi": state.psi, "ll_iters": state.ll_iters, "cg_iters": state.cg_iters,
               "trials": state.trials, "accepted": bool(accepted), "stopped": bool(state.stopped),
               "wall_ms": wall_ms}
        if self.x_true is not None and x is not None:
            mse = float(((x.detach().double().cpu().numpy() - self.x_true) ** 2).mean())
            rec["psnr_x"] = 10 * np.log10(1.0 / mse)
        if self.b_true is not None and b is not None:
            mse = float(((b.detach().double().cpu().numpy() - self.b_true) ** 2).mean())
            rec["psnr_b"] = 10 * np.log10(float(np.max(self.b_true)) ** 2 / mse)
        self.f.write(json.dumps(rec) + "\n")
        self.f.flush()
        return rec

    def close(self):
        self.f.close()
