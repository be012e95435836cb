"""Host-side runtime around the library's calls: checkpoint/resume of the
MAID state, a per-iteration log, and the operator-path autotuner.  Every step
of the method runs in the library (adp.py binds it); this module only stores,
records and times those calls."""
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
        best = float("inf")
        for _ in range(reps):
            t = []
            for n in (iters, 2 * iters):
                xs = x.clone()
                prob.lower_solve(b, xs, 0.0, n)
                t.append(prob.last_kernel_ms())
            best = min(best, (t[1] - t[0]) / iters)
        per[path] = best
    choice = min(per, key=per.get)
    prob.set_fft(choice == "fft")
    return {"path": choice, **{f"{k}_ms": v for k, v in per.items()}}


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
