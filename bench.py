#!/usr/bin/env python
"""Benchmark of the ADP-beta / MAID hot path on GB300.

One step = one MAID upper iteration (Algorithm 2) on the 256 x 256 RGB,
15 x 15 motion-blur workload: the lower-level FISTA solves, the upper loss,
the CG solve of the IFT hypergradient, the kernel-gradient correlation and the
backtracking trials with their re-solves, all inside one cooperative launch
of libadp.  Steps continue one MAID trajectory (paper defaults, Sec. 4.1);
W warm-up steps run first.

value: Mvalue*iter/s = (C*H*W values) x (FISTA + CG iterations executed in
the timed steps) / device time of those steps, summed over ranks (replicas).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MAID time-to-tolerance (s) vs plain FP32 GPU; Mpixel·iter/s of fused steps"
UNIT = "Mvalue·iter/s (values = C·H·W; iters = FISTA + CG iterations)"
WORKLOAD = "rgb256_k15_motion"
SM_COUNT, FP32_LANES = 152, 128
# MAID start for this workload (eps_0 = delta_0, alpha_0): the paper's 1e-2 / 0.1
# are sized for its own scaling; these were picked by a grid search over
# eps_0 in {1e-2, 1e-3, 1e-4} x alpha_0 in {1e-1, 1e-5, 1e-6, 1e-7} (every
# step accepted, least time), as the paper picks alpha and beta by grid search
EPS0, STEP0 = 1e-4, 1e-6


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and parts[1] and self.uuid not in parts[1] and parts[1] not in self.uuid:
                continue
            rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        mx = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_sample(inst, iters):
    """FP64 oracle (as it stands, single thread) running FISTA iterations of the
    lower level on the same workload: returns (Mvalue*iter/s, seconds)."""
    import oracle
    oracle.build()
    C, H, W = inst.shape
    P = oracle.Problem(C, H, W, inst.K, alpha=1e-2, reg_param=1e-2, beta=0.3)
    t = time.perf_counter()
    P.fista(inst.a, inst.y, inst.y, eps=0.0, max_iters=iters)
    dt = time.perf_counter() - t
    return C * H * W * iters / dt / 1e6, dt


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the host cores, bounded sample
    per step (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2502_09758_gb300 import synth
    inst = synth.rgb256_k15(0)
    per_step = 4
    for _ in range(args.warmup):
        oracle_sample(inst, 1)
    tot, units = 0.0, 0
    C, H, W = inst.shape
    for _ in range(args.steps):
        _, dt = oracle_sample(inst, per_step)
        tot += dt
        units += C * H * W * per_step
    val = units / tot / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "C": C, "H": H, "W": W, "K": inst.K},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} FISTA iterations of the FP64 oracle per step on the "
                                       f"{C}x{H}x{W}, K={inst.K} workload"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2502_09758_gb300 import adp, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    inst = synth.rgb256_k15(seed=rank)
    C, H, W = inst.shape
    K = inst.K
    N = C * H * W
    y = torch.tensor(inst.y, dtype=torch.float32, device=dev)
    a = torch.tensor(inst.a, dtype=torch.float32, device=dev)
    prob = adp.Problem(adp.Params(C, H, W, K, alpha=1e-2, reg_param=1e-2, beta=0.3), y, a)
    b, x = a.clone(), y.clone()
    q = torch.zeros_like(x)
    st = prob.maid_init(eps=EPS0, delta=EPS0, step=STEP0)
    for _ in range(args.warmup):
        prob.maid_step(st, b, x, q)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    props = torch.cuda.get_device_properties(dev)
    clk = Clocks(str(getattr(props, "uuid", "")) or None)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    step_ms, kern_ms, iters, passes, accepted = [], [], 0, 0, 0
    for _ in range(args.steps):
        flush.zero_()                       # L2 flush between timed steps (not timed)
        ev0.record()
        ok = prob.maid_step(st, b, x, q)
        ev1.record()
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        kern_ms.append(prob.last_kernel_ms())
        iters += st.ll_iters + st.cg_iters
        passes += prob.conv_passes_last()
        accepted += int(ok)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()

    tot_ms = sum(step_ms)
    units = N * iters
    if world > 1:
        t = torch.tensor([tot_ms, units], dtype=torch.float64, device=dev)
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        tot_ms_max, units_all = float(tmax[0]), float(t[1])
    else:
        tot_ms_max, units_all = tot_ms, float(units)
    value = units_all / (tot_ms_max / 1e3) / 1e6

    # end to end through the public API with host buffers: H2D of the step's
    # inputs (b, x~ warm start) from pinned memory, the call, D2H of b, x~, loss
    b_h = b.cpu().pin_memory()
    x_h = x.cpu().pin_memory()
    e2e_ms, e2e_units = 0.0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        b.copy_(b_h, non_blocking=True)
        x.copy_(x_h, non_blocking=True)
        prob.maid_step(st, b, x, q)
        b_h.copy_(b, non_blocking=True)
        x_h.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        _ = float(st.loss)
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_units += N * (st.ll_iters + st.cg_iters)
    esz = 4
    h2d = (C * K * K + N) * esz
    d2h = (C * K * K + N) * esz + 8

    pk = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    peak_tf = SM_COUNT * FP32_LANES * 2 * sm_max * 1e6 / 1e12
    flops = passes * 2.0 * K * K * N
    achieved = flops / (sum(kern_ms) / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "C": C, "H": H, "W": W, "K": K, "alpha": 1e-2, "huber": 1e-2,
                   "beta": 0.3, "maid_eps0": EPS0, "maid_step0": STEP0,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "maid": {"upper_iters_timed": args.steps, "accepted": accepted,
                 "fused_iters_per_step": iters / args.steps, "eps_end": st.eps,
                 "grid_ctas": prob.grid_size()},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": achieved / peak_tf, "traffic": None,
                     "kernel": "adp_kernel<float> (persistent MAID step)",
                     "peak_basis": f"152 SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz (max SM clock)"},
        "e2e": {"value": e2e_units / (e2e_ms / 1e3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt = oracle_sample(inst, args.cpu_iters)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{args.cpu_iters} FISTA iterations of the FP64 oracle on the "
                                          f"{C}x{H}x{W}, K={K} workload ({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-iters", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
