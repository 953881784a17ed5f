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
    # the seismic example's base grid (80^3, N = 3) with a synthetic
    # topography in place of the terrain data
    "diffuse3d_terrain_80^3_N3": dict(pde=4, dim=3, cells=(80, 80, 80), N=3, lo=(0.0,) * 3, hi=(1.0,) * 3,
                                      params=(), ic="terrain"),
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
    if w["ic"] == "terrain":
        return inputs.diffuse_terrain(X)
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
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "50"]
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
    """Hash of what the kernels are built from -- the CUDA/C++ sources and the
    public header with comments removed and whitespace collapsed, and the
    compiler flags of the build -- so that committed DRAM counters stay tied
    to the code they were taken on, not to its comments or layout."""
    import re

    from paper_1808_03788_gb300 import build as _b
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1808_03788_gb300", "csrc")
    files = [os.path.join(csrc, f) for f in sorted(os.listdir(csrc)) if f.endswith((".cu", ".cuh", ".h", ".cpp"))]
    files.append(os.path.join(ROOT, "include", "aderdg.h"))
    for path in files:
        src = open(path, encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())  # layout-independent
    flags = [f for f in _b.NVFLAGS + _b.CXXFLAGS if not os.path.isabs(f)]  # machine paths excluded
    h.update(" ".join(flags).encode())
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
    return {"workload": args.workload, "pde": {1: "advection", 2: "euler", 3: "elasticity", 4: "diffuse-interface elasticity"}[w["pde"]],
            "dim": w["dim"], "cells": list(w["cells"]), "N": w["N"], "nvar": inputs.nvar(w["pde"], w["dim"]),
            "dofs": int(w["dofs"]), "precision": args.precision, "picard_iters": w["N"] + 1,
            "cfl_alpha": alpha, "l2": "flushed: 256 MiB written between timed steps",
            "parallelism": "replicas" if world > 1 else "single-gpu"}


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------

def _max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time: every rank gets the max (barrier semantics
    of an all-reduce).  One process per GPU; the GPU path uses NCCL, the
    host tests gloo."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _time_single(A, torch, w, prec, stream, steps, warmup, flush, world, shapes=(0, 0), guess=0, picard=0):
    """Time `steps` device-CFL steps of one solve (L2 flushed between steps),
    with per-kernel CUDA events.  Returns the solver and the timings."""
    import numpy as np
    s = A.Solver(w["pde"], w["dim"], w["cells"], w["lo"], w["hi"], w["N"], w["params"], precision=prec,
                 stream=stream.cuda_stream, shapes=shapes, guess=guess, picard=picard)
    X = s.node_coords(w["lo"], w["hi"])
    U0 = np.ascontiguousarray(_initial_state(w, X))
    t_far = 1e30
    s.set_state(U0)
    s.profile(True)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.zero_()
            s.step(t_far)
            s.profile_read()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        pred_ms, corr_ms = [], []
        for k in range(steps):
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
    s.profile(False)
    return s, U0, step_ms, pred_ms, corr_ms


def _roofline(info, pred_avg, prec_name, probe, workload):
    achieved = info["flops_predictor"] / (pred_avg / 1e3) / 1e12
    if prec_name == "fp64":
        return {"bound": "alu", "kernel": "k_predictor (FP64 DFMA pipe)", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 2 DFMA/clock x 2070 MHz (nominal 1.25 TFLOP/s); "
                               "no FP64 figure in MEASURED_PEAKS.json",
                "peak_probe_tflops": probe.get("fp64"),
                "traffic": _traffic("k_predictor", workload, prec_name),
                "algorithmic_flops_per_launch": info["flops_predictor"], "launch_ms": pred_avg}
    return {"bound": "alu", "kernel": "k_predictor (FP32 FFMA pipe)", "achieved": achieved,
            "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
            "peak_source": "derived: 152 SMs x 128 FFMA lanes x 2070 MHz",
            "peak_probe_tflops": probe.get("fp32"),
            "traffic": _traffic("k_predictor", workload, prec_name),
            "algorithmic_flops_per_launch": info["flops_predictor"], "launch_ms": pred_avg}


def _hbm_peak_gbs():
    """Measured HBM copy bandwidth (MEASURED_PEAKS.json), else the 6.8 TB/s
    fallback of the profiling recipe."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0))
    except Exception:
        return 6800.0


def _kernels(info, pred_avg, corr_avg, hbm):
    corr_gbs = info["bytes_corrector"] / (corr_avg / 1e3) / 1e9
    return {
        "tile_shapes": {k: info[k] for k in ("pred_shape", "pred_threads", "pred_epb",
                                             "corr_shape", "corr_threads", "corr_epb")},
        "k_predictor": {"ms": pred_avg, "tflops": info["flops_predictor"] / (pred_avg / 1e3) / 1e12,
                        "gbs": info["bytes_predictor"] / (pred_avg / 1e3) / 1e9},
        "k_corrector": {"ms": corr_avg, "tflops": info["flops_corrector"] / (corr_avg / 1e3) / 1e12,
                        "gbs": corr_gbs, "hbm_frac": corr_gbs / hbm, "hbm_peak_gbs": hbm},
    }


def _guess_variants(A, torch, w, stream, flush, steps, warmup, shapes, l2_steps, probe, hbm, workload):
    """The initial guesses of Sec. 2.2 that cut the Picard iterations: the
    third-order guess with the paper's N-2 iterations, the CERK guess (a
    cubic, degree N-1 at N = 4) with max(1, N-3), and the extrapolation of
    the previous step's predictor with one.  Both precisions timed like the
    headline, and the L2 errors against the exact vortex after `l2_steps`
    steps next to the trivial guess's."""
    import numpy as np

    from paper_1808_03788_gb300 import inputs
    guesses = (("guess_order3", "third order (k1 = L(u), k2 = L(u + dt k1))", A.ADERDG_GUESS_ORDER3,
                max(1, w["N"] - 2)),
               ("guess_cerk", "CERK: cubic dense output of the classical fourth-order Runge-Kutta method",
                A.ADERDG_GUESS_CERK, max(1, w["N"] - 3)),
               ("guess_extrap", "extrapolation of the previous step's predictor", A.ADERDG_GUESS_EXTRAP, 1))
    out = {}
    for key, desc, guess, P in guesses:
        o = {"initial_guess": desc, "picard_iters": P}
        for name, prec in (("fp64", A.ADERDG_FP64), ("mixed", A.ADERDG_MIXED_FP32)):
            s, _, st, pr, co = _time_single(A, torch, w, prec, stream, steps, warmup, flush, 1, shapes, guess, P)
            info = s.info()
            s.close()
            p, c = statistics.mean(pr), statistics.mean(co)
            o[name] = {"value": info["dofs"] * steps / (sum(st) / 1e3), "ms_per_step": sum(st) / steps, "unit": UNIT,
                       "roofline": _roofline(info, p, name, probe, workload), "kernels": _kernels(info, p, c, hbm)}
        out[key] = o
    if w["ic"] == "vortex" and l2_steps > 0:
        _, wq = A.aderdg_gl_nodes(w["N"])
        wn = np.ones(1)
        for _ in range(w["dim"]):
            wn = np.kron(wq, wn)
        vol = np.prod([(w["hi"][d] - w["lo"][d]) / w["cells"][d] for d in range(w["dim"])])
        W = (vol * wn)[None, :, None]

        def err(prec, guess, picard):
            with A.Solver(w["pde"], w["dim"], w["cells"], w["lo"], w["hi"], w["N"], w["params"], precision=prec,
                          guess=guess, picard=picard) as s:
                X = s.node_coords(w["lo"], w["hi"])
                s.set_state(_initial_state(w, X))
                s.advance(1e30, max_steps=l2_steps)
                U, t, k = s.get_state()
            e = U - inputs.euler_vortex(X, t=t)
            return float(np.sqrt(np.sum(W * e * e, axis=(0, 1)))[0])

        trivial = err(A.ADERDG_FP64, 0, 0)
        for key, _, guess, P in guesses:
            out[key]["l2_steps"] = l2_steps
            out[key]["l2_err_vs_exact_rho_fp64_trivial"] = trivial
            out[key]["l2_err_vs_exact_rho_fp64"] = err(A.ADERDG_FP64, guess, P)
            out[key]["l2_err_vs_exact_rho_mixed"] = err(A.ADERDG_MIXED_FP32, guess, P)
    return out


LIMITER_CASES = ("vortex", "blast", "blast_sharp", "inclusion", "inclusion_unlimited", "vortex_mixed", "blast_mixed",
                 "blast_sharp_mixed")


def _limiter(A, torch, w, stream, flush, steps, warmup, cases=LIMITER_CASES, shapes=(0, 0)):
    """The a posteriori subcell limiter (Sec. 2.3) on the headline mesh, FP64:
    the vortex (smooth: detection only) and a blast (rho, p = 1 inside
    r = 2, 0.125 / 0.1 outside, tanh edge of width 0.3, centred in the box);
    and the path-conservative subcell scheme (eq. pde.nc.fv) on the
    diffuse-interface system: a soft inclusion (alpha 1 -> 0.3 across r = 2.5,
    tanh width 0.3, lambda = 2, mu = rho = 1) hit by two mirrored velocity
    boxes, limited and unlimited; the vortex and the blast again on the FP32
    path.  The blast_sharp cases keep the limited elements' subcell data
    between steps (limiter 2) and start from a blast with a sharp edge given
    as subcell averages (2 x 2 midpoint samples per subcell), FP64 and FP32
    path.  Each is timed like the headline, with the troubled elements of
    the last step."""
    import numpy as np

    from paper_1808_03788_gb300 import inputs
    out = {"precision": "fp64 (the *_mixed cases: the FP32 path)"}
    for name in cases:
        dim_pde = name.startswith("inclusion")
        pde, params = (A.ADERDG_PDE_DIFFUSE_ELASTICITY, ()) if dim_pde else (w["pde"], w["params"])
        lim = name != "inclusion_unlimited"
        sharp = name.startswith("blast_sharp")
        prec = A.ADERDG_MIXED_FP32 if name.endswith("_mixed") else A.ADERDG_FP64
        s = A.Solver(pde, w["dim"], w["cells"], w["lo"], w["hi"], w["N"], params, stream=stream.cuda_stream,
                     limiter=2 if sharp else int(lim), precision=prec, shapes=shapes)
        X = s.node_coords(w["lo"], w["hi"])
        x, y = X[..., 0], X[..., 1]
        avg = None
        if sharp:
            avg = inputs.subcell_means(inputs.euler_sharp_blast((5.0, 5.0), 2.0), w["cells"], w["lo"], w["hi"],
                                       w["N"], k=2)
        elif name.startswith("vortex"):
            U0 = inputs.euler_vortex(X, lo=w["lo"], hi=w["hi"])
        elif name.startswith("blast"):
            r = np.sqrt((x - 5.0) ** 2 + (y - 5.0) ** 2)
            rho = inputs.smooth_step(r, 2.0, 0.3, 1.0, 0.125)
            p = inputs.smooth_step(r, 2.0, 0.3, 1.0, 0.1)
            U0 = np.stack([rho, 0 * rho, 0 * rho, p / 0.4], axis=-1)
        else:
            alpha = inputs.smooth_step(np.sqrt((x - 5.0) ** 2 + (y - 5.0) ** 2), 2.5, 0.3, 0.3, 1.0)
            box = lambda a, b: np.where((a > 1.0) & (a < 3.0) & (b > 3.0) & (b < 6.0), 1.0, 0.0)
            z = 0 * x
            U0 = inputs.diffuse_pack(2, [z, z, z], [alpha * box(x, y), alpha * box(y, x)], alpha, 2.0, 1.0, 1.0)
        if sharp:
            s.set_subcell_state(avg)
        else:
            s.set_state(np.ascontiguousarray(U0))
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                flush.zero_()
                s.step(1e30)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                s.step(1e30)
                b.record(stream)
            torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        cnt = s.troubled()[1] if lim else 0
        info = s.info()
        s.close()
        out[name] = {"value": info["dofs"] * steps / (sum(ms) / 1e3), "ms_per_step": sum(ms) / steps,
                     "troubled_last_step": int(cnt), "elements": int(info["elements"]),
                     "tile_shapes": [info["pred_shape"], info["corr_shape"]]}
        if sharp:
            out[name]["subcell_data"] = "kept (limiter 2); initial state given as subcell averages"
    return out


def _equal_l2(A, w, steps):
    """Advance the FP64 and the mixed path `steps` CFL steps from the same
    initial state; relative L2 distance of the two and each one's L2 error
    against the exact translated vortex."""
    import numpy as np

    from paper_1808_03788_gb300 import inputs
    out = {}
    res = {}
    for name, prec in (("fp64", A.ADERDG_FP64), ("mixed", A.ADERDG_MIXED_FP32)):
        with A.Solver(w["pde"], w["dim"], w["cells"], w["lo"], w["hi"], w["N"], w["params"], precision=prec) as s:
            X = s.node_coords(w["lo"], w["hi"])
            s.set_state(_initial_state(w, X))
            s.advance(1e30, max_steps=steps)
            U, t, k = s.get_state()
            _, wq = A.aderdg_gl_nodes(w["N"])
            res[name] = (U, t, k, X, wq)
    U64, t64, k64, X, wq = res["fp64"]
    Umx, tmx, kmx, _, _ = res["mixed"]
    n = w["N"] + 1
    wn = np.ones(1)
    for _ in range(w["dim"]):
        wn = np.kron(wq, wn)
    vol = np.prod([(w["hi"][d] - w["lo"][d]) / w["cells"][d] for d in range(w["dim"])])
    W = (vol * wn)[None, :, None]
    l2 = lambda a: np.sqrt(np.sum(W * a * a, axis=(0, 1)))
    rel = float(np.max(l2(Umx - U64) / l2(U64)))
    out["steps"] = k64
    out["t"] = t64
    out["mixed_vs_fp64_rel_l2"] = rel
    if w["ic"] == "vortex":
        out["fp64_l2_err_vs_exact_rho"] = float(l2(U64 - inputs.euler_vortex(X, t=t64))[0])
        out["mixed_l2_err_vs_exact_rho"] = float(l2(Umx - inputs.euler_vortex(X, t=tmx))[0])
    out["equal_at_1e-6"] = rel <= 1e-6
    return out


def _end_time(A, torch, vortex_t_end=10.0, elastic_t_end=0.25, shapes=(0, 0)):
    """The configured end-time runs, FP64 and mixed from the same initial
    state: the 200^2 N = 4 vortex to t = 10 (its exact solution is the
    initial state again), with each path's L2 error of rho against the
    exact vortex and the mixed-vs-FP64 relative L2; and the 64^3 N = 3
    elastic pulse to t = 0.25, mixed against FP64 (no exact solution).
    Whole runs through aderdg_advance (graph-replayed steps)."""
    import numpy as np

    from paper_1808_03788_gb300 import inputs
    out = {}
    for key, wname, t_end in (("vortex_t10", "euler2d_vortex_200x200_N4", vortex_t_end),
                              ("elastic_t0.25", "elastic3d_pulse_64^3_N3", elastic_t_end)):
        if t_end <= 0:
            continue
        w = WORKLOADS[wname]
        res = {}
        for name, prec in (("fp64", A.ADERDG_FP64), ("mixed", A.ADERDG_MIXED_FP32)):
            with A.Solver(w["pde"], w["dim"], w["cells"], w["lo"], w["hi"], w["N"], w["params"], precision=prec,
                          shapes=shapes) as s:
                X = s.node_coords(w["lo"], w["hi"])
                s.set_state(np.ascontiguousarray(_initial_state(w, X)))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.advance(t_end)
                U, t, k = s.get_state()
                res[name] = (U, t, k, time.perf_counter() - t0)
        _, wq = A.aderdg_gl_nodes(w["N"])
        wn = np.ones(1)
        for _ in range(w["dim"]):
            wn = np.kron(wq, wn)
        vol = np.prod([(w["hi"][d] - w["lo"][d]) / w["cells"][d] for d in range(w["dim"])])
        W = (vol * wn)[None, :, None]
        l2 = lambda a: np.sqrt(np.sum(W * a * a, axis=(0, 1)))
        (U64, t64, k64, s64), (Umx, tmx, kmx, smx) = res["fp64"], res["mixed"]
        den = l2(U64)
        rel = l2(Umx - U64) / np.where(den > 0, den, 1.0)
        o = {"workload": wname, "t_end": t_end, "fp64": {"t": t64, "steps": k64, "wall_s": s64},
             "mixed": {"t": tmx, "steps": kmx, "wall_s": smx},
             "mixed_vs_fp64_rel_l2": float(np.max(rel)), "equal_at_1e-6": bool(np.max(rel) <= 1e-6)}
        if w["ic"] == "vortex":  # X: the node coordinates of the runs above
            o["fp64"]["l2_err_vs_exact_rho"] = float(l2(U64 - inputs.euler_vortex(X, t=t64))[0])
            o["mixed"]["l2_err_vs_exact_rho"] = float(l2(Umx - inputs.euler_vortex(X, t=tmx))[0])
        out[key] = o
    return out


def _partitioned(A, torch, w, stream, flush, steps, warmup, parts=(2, 2), shapes=(0, 0)):
    """The headline mesh split into parts blocks on this GPU (the
    distributed-memory step of Sec. 2.2: boundary predictor first, face
    traces exchanged while the interior predictor runs, one wave-speed
    reduction): ms per step next to the undivided solver's, both timed like
    the headline, and whether the two states are bitwise equal after the
    same steps."""
    import numpy as np
    out = {"parts": list(parts)}
    states = {}
    for name, prec in (("fp64", A.ADERDG_FP64), ("mixed", A.ADERDG_MIXED_FP32)):
        for kind in ("single", "partitioned"):
            extra = {"parts": parts} if kind == "partitioned" else {}
            cls = A.Partitioned if kind == "partitioned" else A.Solver
            with cls(w["pde"], w["dim"], w["cells"], w["lo"], w["hi"], w["N"], w["params"], precision=prec,
                     stream=stream.cuda_stream, shapes=shapes, **extra) as s:
                X = s.node_coords(w["lo"], w["hi"])
                s.set_state(np.ascontiguousarray(_initial_state(w, X)))
                with torch.cuda.stream(stream):
                    for _ in range(warmup):
                        flush.zero_()
                        s.step(1e30)
                    torch.cuda.synchronize()
                    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                          for _ in range(steps)]
                    for a, b in ev:
                        flush.zero_()
                        a.record(stream)
                        s.step(1e30)
                        b.record(stream)
                    torch.cuda.synchronize()
                ms = sum(a.elapsed_time(b) for a, b in ev) / steps
                states[(name, kind)] = s.get_state()[0]
                rec = {"ms_per_step": ms, "value": w["dofs"] / (ms / 1e3)}
                if kind == "partitioned":
                    rec.update(s.dd_info())
                out.setdefault(name, {})[kind] = rec
        out[name]["bitwise_equal"] = bool(np.array_equal(states[(name, "single")], states[(name, "partitioned")]))
    return out


def _elastic(A, torch, stream, flush, steps, shapes=(0, 0), workload="elastic3d_pulse_64^3_N3"):
    """A 3D elasticity workload -- the conservative system (64^3 elements,
    N = 3, 9 variables, Gaussian velocity pulse) or the diffuse-interface
    one (80^3, N = 3, 13 variables, synthetic topography): both paths, and
    how far apart they are after the timed steps."""
    import numpy as np
    w = dict(WORKLOADS[workload])
    out = {"workload": workload}
    states = {}
    for name, prec in (("fp64", A.ADERDG_FP64), ("mixed", A.ADERDG_MIXED_FP32)):
        s, _, st, pr, co = _time_single(A, torch, w, prec, stream, steps, 2, flush, 1, shapes)
        info = s.info()
        states[name] = s.get_state()[0]
        s.close()
        corr_gbs = info["bytes_corrector"] / (statistics.mean(co) / 1e3) / 1e9
        out[name] = {"value": info["dofs"] * steps / (sum(st) / 1e3), "ms_per_step": sum(st) / steps,
                     "predictor_ms": statistics.mean(pr), "corrector_ms": statistics.mean(co),
                     "predictor_tflops": info["flops_predictor"] / (statistics.mean(pr) / 1e3) / 1e12,
                     "corrector_gbs": corr_gbs, "corrector_hbm_frac": corr_gbs / _hbm_peak_gbs(),
                     "tile_shapes": [info["pred_shape"], info["corr_shape"]]}
    a, b = states["mixed"], states["fp64"]
    num = np.sqrt(np.sum((a - b) ** 2, axis=(0, 1)))
    den = np.sqrt(np.sum(b ** 2, axis=(0, 1)))
    out["mixed_vs_fp64_rel_l2"] = float(np.max(num[den > 0] / den[den > 0]))
    out["steps"] = steps + 2
    return out


def _batched(A, torch, steps, warmup, count, shapes=(0, 0)):
    """The batched workload: `count` independent 2D Euler vortex solves
    (meshes k^2, k in {32, ..., 256}; N in 2..6; eps in [1, 5]; centres in
    [3, 7]^2; seed 1808), FP32 predictor / FP64 update, one graph step each."""
    from paper_1808_03788_gb300 import inputs
    rec = inputs.batched_vortex_recipe(count)
    specs = [A.make_spec(2, 2, r["cells"], (0, 0), (10, 10), r["N"], (1.4,)) for r in rec]
    b = A.Batch(specs, precision=A.ADERDG_MIXED_FP32, torch_alloc=False, shapes=shapes)
    nodes = {N: A.aderdg_gl_nodes(N)[0] for N in range(2, 7)}
    for i, r in enumerate(rec):
        X = inputs.node_coords_torch(r["cells"], (0, 0), (10, 10), nodes[r["N"]])
        b.set_state(i, inputs.euler_vortex_torch(X, eps=r["eps"], center=r["center"]))
        del X
    info = b.info()
    t_far = [1e30] * count
    b.advance(t_far, max_steps=warmup)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    b.advance(None, max_steps=steps)
    t1.record()
    t1.synchronize()
    ms = t0.elapsed_time(t1)
    b.close()
    return {"value": info["dofs"] * steps / (ms / 1e3), "unit": UNIT, "solves": count,
            "dofs_per_step": info["dofs"], "groups": info["groups"], "steps": steps,
            "ms_per_step": ms / steps, "device_bytes": info["device_bytes"],
            "timing": "CUDA events around aderdg_batch_advance (graph-replayed, host check every 8 steps)",
            "dtype": "f32+f64"}


def _served(A, requests, rate, seed=1808, shapes=(0, 0)):
    """The served stream: the first `requests` of the seeded Poisson stream
    (mean `rate`/s, 50/50 2D Euler vortex / 3D elasticity pulse, run to
    t = 1), submitted at their arrival times to a continuous-batching server."""
    import numpy as np

    from paper_1808_03788_gb300 import inputs
    rec = inputs.served_stream_recipe(requests, rate, seed)
    if shapes == "auto":  # tune every (PDE, N) of the stream before it starts
        for key in sorted({(r["pde"], r["dim"], r["N"]) for r in rec}):
            sp = A.make_spec(key[0], key[1], (8,) * key[1], (0,) * key[1], (1,) * key[1], key[2],
                             (1.4,) if key[0] == 2 else (1.0, 2.0, 1.0))
            A.aderdg_autotune(sp, A.ADERDG_MIXED_FP32)
    srv = A.Server(precision=A.ADERDG_MIXED_FP32, shapes=shapes)
    prepared = []
    for r in rec:
        if r["pde"] == 2:
            spec = A.make_spec(2, 2, r["cells"], (0, 0), (10, 10), r["N"], (1.4,))
            x, _ = A.aderdg_gl_nodes(r["N"])
            X = inputs.node_coords_torch(r["cells"], (0, 0), (10, 10), x, device="cpu")
            u0 = inputs.euler_vortex_torch(X, eps=r["eps"], center=r["center"]).numpy()
        else:
            spec = A.make_spec(3, 3, r["cells"], (0, 0, 0), (1, 1, 1), r["N"], (1.0, 2.0, 1.0))
            x, _ = A.aderdg_gl_nodes(r["N"])
            X = inputs.node_coords_torch(r["cells"], (0,) * 3, (1,) * 3, x, device="cpu")
            u0 = inputs.elastic_pulse_torch(X, x0=r["x0"]).numpy()
        prepared.append((r["arrival"], spec, u0, r["t_end"], A.spec_size(spec) // A.nvar(r["pde"], r["dim"])))
    t0 = time.perf_counter()
    tickets = []
    for arr, spec, u0, t_end, dofs in prepared:
        delay = arr - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        tickets.append((srv.submit(spec, u0, t_end), dofs))
    results = {}
    while len(results) < len(tickets):
        for tk, dofs in tickets:
            if tk not in results:
                r = srv.poll(tk)
                if r is not None:
                    results[tk] = (r, dofs)
        time.sleep(0.001)
    makespan = time.perf_counter() - t0
    srv.close()
    lat = np.array([r["latency_s"] for r, _ in results.values()])
    work = sum(r["steps"] * d for r, d in results.values())
    ok = sum(1 for r, _ in results.values() if r["status"] == 0)
    return {"requests": len(tickets), "ok": ok, "rate_per_s": rate, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "latency_samples": int(lat.size),
            "p99_note": ("a tail estimate over %d samples" % lat.size) if lat.size >= 100 else
                        ("= the maximum of %d samples, not a tail estimate" % lat.size),
            "mean_queue_s":
                float(np.mean([r["queue_s"] for r, _ in results.values()])),
            "makespan_s": makespan, "dof_updates": work, "value": work / makespan, "unit": UNIT,
            "dtype": "f32+f64"}


def run_ours(args, w, rank, world):
    import numpy as np
    import torch

    import paper_1808_03788_gb300.aderdg as A

    stream = torch.cuda.Stream()
    prec = A.ADERDG_FP64 if args.precision == "fp64" else A.ADERDG_MIXED_FP32
    cfgd = _config(args, w, world)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    clocks = ClockSampler(_gpu_id() if rank == 0 else None)
    if rank == 0:
        clocks.start()
    if args.shapes == "auto":
        shapes = "auto"
    elif args.shapes == "default":
        shapes = (0, 0)
    else:  # explicit "predictor,corrector" shape indices
        shapes = tuple(int(x) for x in args.shapes.split(","))
    tune = {}
    if shapes == "auto":  # timed here, before anything is measured; handles then find the choice
        sp = A.make_spec(w["pde"], w["dim"], w["cells"], w["lo"], w["hi"], w["N"], w["params"])
        for name, pr in (("fp64", A.ADERDG_FP64), ("mixed", A.ADERDG_MIXED_FP32)):
            ch, ms = A.aderdg_autotune(sp, pr, force=True)
            tune[name] = {"chosen": list(ch), "predictor_ms": ms[:A.ADERDG_NUM_PRED_SHAPES],
                          "corrector_ms": ms[A.ADERDG_NUM_PRED_SHAPES:]}
    s, U0, step_ms, pred_ms, corr_ms = _time_single(A, torch, w, prec, stream, args.steps, args.warmup, flush, world,
                                                    shapes)
    clk = clocks.stop() if rank == 0 else None
    info = s.info()
    assert (info["cfl_alpha"], info["picard_iters"], info["dofs"]) == \
        (cfgd["cfl_alpha"], cfgd["picard_iters"], cfgd["dofs"]), (info, cfgd)
    dofs = info["dofs"]
    total_ms = _max_over_ranks(sum(step_ms), world)
    value = world * dofs * args.steps / (total_ms / 1e3)

    # ---- end to end through the public API with host buffers ------------------
    t_far = 1e30
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    host_in = torch.from_numpy(U0.copy()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
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
    s.close()
    e2e_total = _max_over_ranks(sum(e2e_ms), world)
    state_bytes = U0.nbytes
    e2e = {"value": world * dofs * e2e_steps / (e2e_total / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
           "steps": e2e_steps, "api": "aderdg_set_state(HOST) + aderdg_step + aderdg_get_state(HOST)"}

    if rank != 0:
        return 0

    probe = {}
    for kind, name in ((0, "fp64"), (1, "fp32")):
        try:
            probe[name] = None if args.no_probe else A.aderdg_peak_tflops(kind)
        except Exception:  # the probe is context only
            probe[name] = None
    hbm = _hbm_peak_gbs()
    pred_avg, corr_avg = statistics.mean(pred_ms), statistics.mean(corr_ms)
    roofline = _roofline(info, pred_avg, args.precision, probe, args.workload)
    kernels = _kernels(info, pred_avg, corr_avg, hbm)

    # ---- the rest of the metric: mixed at equal L2 error, batched, served ----------
    variants = {}
    if not args.no_variants:
        other = "mixed" if args.precision == "fp64" else "fp64"
        oprec = A.ADERDG_MIXED_FP32 if other == "mixed" else A.ADERDG_FP64
        s2, _, st2, pr2, co2 = _time_single(A, torch, w, oprec, stream, args.steps, args.warmup, flush, 1, shapes)
        i2 = s2.info()
        s2.close()
        p2, c2 = statistics.mean(pr2), statistics.mean(co2)
        variants[other] = {"value": dofs * args.steps / (sum(st2) / 1e3), "ms_per_step": sum(st2) / args.steps,
                           "unit": UNIT, "dtype": "f32+f64" if other == "mixed" else "f64",
                           "roofline": _roofline(i2, p2, other, probe, args.workload),
                           "kernels": _kernels(i2, p2, c2, hbm)}
        variants["equal_l2"] = _equal_l2(A, w, args.l2_steps)
        if args.end_time:
            variants["end_time"] = _end_time(A, torch, shapes=shapes)
        if args.dd_steps > 0:
            variants["partitioned"] = _partitioned(A, torch, w, stream, flush, args.dd_steps, args.warmup,
                                                   shapes=shapes)
        if args.limiter_steps > 0 and w["pde"] == 2:
            variants["limiter"] = _limiter(A, torch, w, stream, flush, args.limiter_steps, args.warmup,
                                           tuple(args.limiter_cases.split(",")), shapes)
        if args.guess_variant:
            variants.update(_guess_variants(A, torch, w, stream, flush, args.steps, args.warmup, shapes,
                                            args.l2_steps, probe, hbm, args.workload))
        if args.elastic_steps > 0 and args.workload != "elastic3d_pulse_64^3_N3":
            variants["elastic3d"] = _elastic(A, torch, stream, flush, args.elastic_steps, shapes)
        if args.diffuse_steps > 0 and args.workload != "diffuse3d_terrain_80^3_N3":
            variants["diffuse3d"] = _elastic(A, torch, stream, flush, args.diffuse_steps, shapes,
                                             "diffuse3d_terrain_80^3_N3")
        if args.batched_solves > 0:
            variants["batched"] = _batched(A, torch, args.batched_steps, args.batched_warmup, args.batched_solves,
                                           shapes)
        if args.served_requests > 0:
            variants["served"] = _served(A, args.served_requests, args.served_rate, shapes=shapes)
            sv = variants["served"]
            if args.served_scaled > 0 and sv["ok"] > 0:
                # the same stream at 80 % of the capacity the first run measured
                mean_work = sv["dof_updates"] / sv["requests"]
                rate = 0.8 * sv["value"] / mean_work
                variants["served_80pct"] = _served(A, args.served_scaled, rate, shapes=shapes)
                variants["served_80pct"]["rate_rule"] = "0.8 x measured DOF-updates/s / mean DOF-updates per request"

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        v, el, cores = oracle_throughput(w, args.cpu_steps)
        oracle.set_threads(1)
        try:
            v1, el1, _ = oracle_throughput(w, 1)
        finally:
            oracle.set_threads(0)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d full ADER-DG steps of the whole %s mesh, plain FP64 C oracle, OpenMP over "
                         "elements (%.1f s)" % (args.cpu_steps, "x".join(map(str, w["cells"])), el),
               "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                 "sample": "1 full step of the same mesh on one thread (%.1f s)" % el1}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": cfgd,
        "roofline": roofline,
        "kernels": kernels,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": 3 * args.steps,
        "autotune": tune or None,
        "variants": variants,
    }
    print(json.dumps(line), flush=True)
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
    ap.add_argument("--no-probe", action="store_true", help="skip the FMA peak probe")
    ap.add_argument("--no-variants", action="store_true",
                    help="only the headline path (no mixed/batched/served/equal-L2 runs)")
    ap.add_argument("--l2-steps", type=int, default=100)
    ap.add_argument("--elastic-steps", type=int, default=4)
    ap.add_argument("--limiter-steps", type=int, default=10,
                    help="timed steps of the subcell-limiter variant (0: skip)")
    ap.add_argument("--limiter-cases", default=",".join(LIMITER_CASES),
                    help="comma list of the limiter cases to time (%s)" % ",".join(LIMITER_CASES))
    ap.add_argument("--diffuse-steps", type=int, default=3,
                    help="timed steps of the 3D diffuse-interface variant (0: skip)")
    ap.add_argument("--batched-solves", type=int, default=256)
    ap.add_argument("--batched-steps", type=int, default=200, help="timed window of the batched workload")
    ap.add_argument("--batched-warmup", type=int, default=20)
    ap.add_argument("--served-requests", type=int, default=24)
    ap.add_argument("--served-rate", type=float, default=200.0)
    ap.add_argument("--served-scaled", type=int, default=12,
                    help="requests of a second served run at 80 %% of the measured capacity (0: skip)")
    ap.add_argument("--dd-steps", type=int, default=20,
                    help="timed steps of the partitioned (2 x 2 blocks) variant (0: skip)")
    ap.add_argument("--no-end-time", dest="end_time", action="store_false",
                    help="skip the configured end-time runs (vortex to t = 10, elastic pulse to t = 0.25)")
    ap.add_argument("--no-guess-variant", dest="guess_variant", action="store_false",
                    help="skip the initial-guess variants (third order, extrapolation)")
    ap.add_argument("--shapes", default="auto",
                    help="tile shapes of the kernels: auto (autotuned, default), default (shape 0) or "
                         "'P,C' (predictor and corrector shape indices)")
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
