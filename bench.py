#!/usr/bin/env python3
"""Throughput benchmark of the ADER-DG hot path on GB300.

A step is one whole ADER-DG time step -- device CFL dt, space-time
predictor (Picard iterations), corrector (Rusanov faces, lift, update,
wave-speed maxima) -- over the 2D Euler isentropic vortex on 200 x 200
elements, N = 4 (1.0e6 DOFs, 4 variables), inputs resident in HBM.  The
metric is DOF-updates per second, a DOF being one spatial node of one
element advanced by one step (the paper's TDU convention, Sec. 3.1).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Between timed steps a 256 MiB buffer is written to flush L2 (129 MB); the
flush is outside the timed events.  Multi-GPU: one process per GPU
(torchrun), each GPU advances its own replica of the workload ("replicas
only": the path needs no collective); value = DOF-updates of all ranks /
max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s: FP64 plain vs FP32-batched at equal L2 error; p50/p99 solve latency"
UNIT = "DOF-updates/s"

WORKLOADS = {
    "euler2d_vortex_200x200_N4": dict(pde=2, dim=2, cells=(200, 200), N=4, lo=(0.0, 0.0), hi=(10.0, 10.0),
                                      params=(1.4,), ic="vortex"),
    "elastic3d_pulse_64^3_N3": dict(pde=3, dim=3, cells=(64, 64, 64), N=3, lo=(0.0,) * 3, hi=(1.0,) * 3,
                                    params=(1.0, 2.0, 1.0), ic="pulse"),
    "advection2d_sine_16x16_N3": dict(pde=1, dim=2, cells=(16, 16), N=3, lo=(0.0, 0.0), hi=(1.0, 1.0),
                                      params=(1.0, 1.0), ic="sine"),
}
DEFAULT_WORKLOAD = "euler2d_vortex_200x200_N4"

# ALU peaks of one GB300 from unit counts and the maximum SM clock (152 SMs,
# 2070 MHz): FP64 at 2 DFMA per clock per SM (the nominal 1.25 TFLOP/s),
# FP32 at 128 FFMA lanes per clock per SM.  The driver's peak file has no
# FP64/FP32 figures; bench.py also reports its own FMA-chain probe.
SMS, SM_MHZ = 152, 2070.0
FP64_PEAK_TFLOPS = SMS * SM_MHZ * 1e6 * 2 * 2 / 1e12
FP32_PEAK_TFLOPS = SMS * SM_MHZ * 1e6 * 128 * 2 / 1e12


def _initial_state(w, X):
    from paper_1808_03788_gb300 import inputs
    if w["ic"] == "vortex":
        return inputs.euler_vortex(X, lo=w["lo"], hi=w["hi"])
    if w["ic"] == "pulse":
        return inputs.elastic_pulse(X)
    return inputs.advection_sine(X, lo=w["lo"], hi=w["hi"])


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.lines: list[str] = []
        self.proc = None
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


def _gpu_id():
    try:
        import torch
        uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[0] if vis else None


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1808_03788_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(kernel: str, workload: str, precision: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources; otherwise None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        data = json.load(open(path))
    except Exception:
        return None
    rec = data.get("%s|%s|%s" % (kernel, workload, precision))
    if not rec or rec.get("source_hash") != _kernel_source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_throughput(w, steps: int):
    import numpy as np

    import oracle
    cfg = oracle.make_cfg(w["dim"], w["cells"], w["lo"], w["hi"], w["N"], w["pde"], w["params"])
    U = _initial_state(w, oracle.node_coords(cfg))
    dofs = oracle.n_elems(cfg) * (w["N"] + 1) ** w["dim"]
    t0 = time.perf_counter()
    for _ in range(steps):
        dt = oracle.cfl_dt(cfg, U)
        U = oracle.step(cfg, U, dt)
    el = time.perf_counter() - t0
    assert np.isfinite(U).all()
    return dofs * steps / el, el, oracle.threads()


def run_reference(args, w, rank, world):
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_throughput(w, 1)
    value, el, cores = oracle_throughput(w, args.steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(args, w, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d full ADER-DG steps of the whole mesh (plain FP64 C oracle, "
                                   "OpenMP over elements)" % args.steps},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(args, w, world):
    """The workload description both arms print (same keys and values)."""
    from paper_1808_03788_gb300 import inputs
    alpha = {1: 0.3001, 2: 0.1538, 3: 0.0936, 4: 0.0629, 5: 0.0451, 6: 0.0339, 7: 0.0265}[w["N"]]
    return {"workload": args.workload, "pde": {1: "advection", 2: "euler", 3: "elasticity"}[w["pde"]],
            "dim": w["dim"], "cells": list(w["cells"]), "N": w["N"], "nvar": inputs.nvar(w["pde"], w["dim"]),
            "dofs": int(w["dofs"]), "precision": args.precision, "picard_iters": w["N"] + 1,
            "cfl_alpha": alpha, "l2": "flushed: 256 MiB written between timed steps",
            "parallelism": "replicas" if world > 1 else "single-gpu"}


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------

def run_ours(args, w, rank, world):
    import numpy as np
    import torch

    import paper_1808_03788_gb300.aderdg as A

    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    prec = A.ADERDG_FP64 if args.precision == "fp64" else A.ADERDG_MIXED_FP32
    s = A.Solver(w["pde"], w["dim"], w["cells"], w["lo"], w["hi"], w["N"], w["params"], precision=prec,
                 stream=stream.cuda_stream)
    info = s.info()
    cfgd = _config(args, w, world)
    assert (info["cfl_alpha"], info["picard_iters"], info["dofs"]) == \
        (cfgd["cfl_alpha"], cfgd["picard_iters"], cfgd["dofs"]), (info, cfgd)
    X = s.node_coords(w["lo"], w["hi"])
    U0 = np.ascontiguousarray(_initial_state(w, X))
    dofs = info["dofs"]
    t_far = 1e30

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    s.set_state(U0)
    s.profile(True)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            s.step(t_far)
            s.profile_read()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

        clocks = ClockSampler(_gpu_id() if rank == 0 else None)
        if rank == 0:
            clocks.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        pred_ms, corr_ms = [], []
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            s.step(t_far)
            ev[k][1].record(stream)
            a, b = s.profile_read()
            pred_ms.append(a)
            corr_ms.append(b)
        torch.cuda.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = clocks.stop() if rank == 0 else None
    s.sync()
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * dofs * args.steps / (total_ms / 1e3)

    # ---- end to end through the public API with host buffers ------------------
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    host_in = torch.from_numpy(U0.copy()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    s.profile(False)
    e2e_ms = []
    with torch.cuda.stream(stream):
        for _ in range(2):
            s.set_state(host_in.numpy())
            s.step(t_far)
            s.get_state()
        for _ in range(e2e_steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.set_state(host_in.numpy())
            s.step(t_far)
            s.get_state(out=host_out.numpy(), check=True)  # into pinned host memory
            b.record(stream)
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))
    e2e_total = sum(e2e_ms)
    if world > 1:
        t = torch.tensor([e2e_total], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_total = float(t.item())
    state_bytes = U0.nbytes
    e2e = {"value": world * dofs * e2e_steps / (e2e_total / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
           "steps": e2e_steps, "api": "aderdg_set_state(HOST) + aderdg_step + aderdg_get_state(HOST)"}

    if rank != 0:
        s.close()
        return 0

    probe = {}
    for kind, name in ((0, "fp64"), (1, "fp32")):
        try:
            probe[name] = A.aderdg_peak_tflops(kind)
        except Exception as e:  # the probe is context only
            probe[name] = None
    pred_avg = statistics.mean(pred_ms)
    corr_avg = statistics.mean(corr_ms)
    if args.precision == "fp64":
        achieved = info["flops_predictor"] / (pred_avg / 1e3) / 1e12
        roofline = {"bound": "alu", "kernel": "k_predictor (FP64 DFMA pipe)", "achieved": achieved,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "peak_source": "derived: 152 SMs x 2 DFMA/clock x 2070 MHz (nominal 1.25 TFLOP/s); "
                                   "no FP64 figure in MEASURED_PEAKS.json",
                    "peak_probe_tflops": probe.get("fp64"),
                    "traffic": _traffic("k_predictor", args.workload, args.precision),
                    "algorithmic_flops_per_launch": info["flops_predictor"],
                    "launch_ms": pred_avg}
    else:
        achieved = info["flops_predictor"] / (pred_avg / 1e3) / 1e12
        roofline = {"bound": "alu", "kernel": "k_predictor (FP32 FFMA pipe)", "achieved": achieved,
                    "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                    "peak_source": "derived: 152 SMs x 128 FFMA lanes x 2070 MHz",
                    "peak_probe_tflops": probe.get("fp32"),
                    "traffic": _traffic("k_predictor", args.workload, args.precision),
                    "algorithmic_flops_per_launch": info["flops_predictor"],
                    "launch_ms": pred_avg}
    corr_gbs = info["bytes_corrector"] / (corr_avg / 1e3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    kernels = {
        "k_predictor": {"ms": pred_avg, "tflops": info["flops_predictor"] / (pred_avg / 1e3) / 1e12,
                        "gbs": info["bytes_predictor"] / (pred_avg / 1e3) / 1e9},
        "k_corrector": {"ms": corr_avg, "tflops": info["flops_corrector"] / (corr_avg / 1e3) / 1e12,
                        "gbs": corr_gbs, "hbm_frac": corr_gbs / hbm,
                        "hbm_peak_gbs": hbm},
    }

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, el, cores = oracle_throughput(w, args.cpu_steps)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d full ADER-DG steps of the whole %s mesh, plain FP64 C oracle, OpenMP over "
                         "elements (%.1f s)" % (args.cpu_steps, "x".join(map(str, w["cells"])), el)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": _config(args, w, world),
        "roofline": roofline,
        "kernels": kernels,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": 3 * args.steps,
    }
    print(json.dumps(line), flush=True)
    s.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    w = dict(WORKLOADS[args.workload])
    w["dofs"] = 1
    for c in w["cells"]:
        w["dofs"] *= c
    w["dofs"] *= (w["N"] + 1) ** w["dim"]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, w, rank, world)

    import torch
    if world > 1:
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    try:
        return run_ours(args, w, rank, world)
    finally:
        if world > 1:
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
