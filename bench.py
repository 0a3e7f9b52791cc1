#!/usr/bin/env python
"""Benchmark of the sparse exact-GP hot path (arXiv 2205.09070) on GB300.

One step = one log-marginal-likelihood + gradient evaluation through the C ABI
(gp_lml_grad): assembly of K (cell list, count, scan, fill), batched CG over
[y, 32 probes], stochastic Lanczos quadrature and the adjoint gradient.

Workload (synthetic, seeded): the clustered 3-D mixture at N = 1,000,000
points (50 Gaussian components, sigma 0.02, 80 %, plus 20 % uniform
background), 8 functions x 16 bumps centred on mixture components, stationary
radius 0.005 * 5^(1/3), 32 probes, 50 Lanczos steps, CG rtol 1e-6 -- a stand-in
for the paper's 5-million-point station-day climate data (Sec. 3).

Printed JSON line (rank 0):
  value          LML+grad evaluations/s, inputs resident in HBM (FP32_MIXED path)
  e2e            the same through the C ABI with pinned HOST buffers (copies inside)
  fp64_path      the plain FP64 single-RHS path on the same workload
  assembly       assembled nnz/s
  roofline       the SpMM kernel (dominant): algorithmic bytes / average launch time
  cpu_baseline   the FP64 CPU oracle on a bounded sample of the workload
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LML+grad evals/s at N=1M (FP32-mixed, batched CG + SLQ + adjoint)"
UNIT = "evals/s"
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=1200)
    ap.add_argument("--n5m", type=int, default=1, help="add the 5M-point leg to the 1M line (0: skip)")
    ap.add_argument("--batch", type=int, default=1, help="add the 256-instance leg to the 1M line (0: skip)")
    ap.add_argument("--batch-only", type=int, default=0,
                    help="run only the many-instance leg's grouped path, on its first N instances (profiling runs)")
    ap.add_argument("--precond-block", type=int, default=None,
                    help="block-Jacobi block size of the preconditioned CG (default: the library's)")
    ap.add_argument("--spmm", default="auto", choices=["auto", "cpasync", "tma", "tma_wide", "cpasync_wide", "window"],
                    help="SpMM form: the library's autotuner (auto) or a forced form; profiling runs force "
                         "the form the plain run chose, since the tuner's timings are meaningless under ncu")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={SMI_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                f = [t.strip() for t in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        load = [s for s, p in zip(sm, pw) if p is not None and p > 250.0] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": num(rows[0][2]), "reasons": reasons, "samples": len(rows),
                "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------- helpers
def peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": d.get("hbm_gbs"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


SPMM_SOURCE = os.path.join(ROOT, "paper_2205_09070_gb300", "csrc", "spmm.cu")
SPMM_KERNELS = {0: "k_bspmm_f32<{kq}>", 1: "k_bspmm_tma<{kq},1>", 2: "k_bspmm_tma<{kq},{lw}>",
                3: "k_bspmm_f32w<{kq},{lw}>", 4: "k_wspmm<{kq},{lw}>"}


def spmm_kernel_name(variant: int, kp: int) -> str:
    kq = kp // 4
    lw = 3 if kq % 3 == 0 and kq >= 6 else 2 if kq % 2 == 0 and kq >= 4 else 1
    return SPMM_KERNELS.get(variant, "k_bspmm_?<{kq}>").format(kq=kq, lw=lw)


WINDOW_SOURCE = os.path.join(ROOT, "paper_2205_09070_gb300", "csrc", "window.cu")
ASSEMBLE_SOURCE = os.path.join(ROOT, "paper_2205_09070_gb300", "csrc", "assemble.cu")
_S_A = "// A: Q = Khat P on the 8x1 block CSR."
_S_TMA = "// ---------------------------------------------------------------- TMA form"
_S_WIDE = "// ---------------------------------------------------------------- wide cp.async form"
_S_HOST = "// ---------------------------------------------------------------- host side"
# The matrix a form multiplies is laid out by the assembly (the row order: the grid and the
# sort key; the 8x1 blocks), so those parts of the assembly are in every form's key: its
# DRAM traffic changes with them.
_ASM = [(ASSEMBLE_SOURCE, "// ------------------------------------------------------------------ cells",
         "// ------------------------------------------------------------------ radix sort"),
        (ASSEMBLE_SOURCE, "// ------------------------------------------------------------------ 8x1 block CSR",
         "int assemble_t(gp_ctx* c, const double* x, int64_t n, const double* h) {"),
        (ASSEMBLE_SOURCE, "  double h_cell = c->r_s * (1.0 + 1e-9);", "  c->grid = g;")]
# (file, first marker inclusive, second marker exclusive) of each SpMM form: its kernel, the
# helpers it calls and the assembly that lays out its matrix
SPMM_REGIONS = {
    "k_bspmm_f32": [(SPMM_SOURCE, _S_A, _S_TMA)] + _ASM,
    "k_bspmm_tma": [(SPMM_SOURCE, _S_A, _S_TMA), (SPMM_SOURCE, _S_TMA, _S_WIDE)] + _ASM,
    "k_bspmm_f32w": [(SPMM_SOURCE, _S_A, _S_TMA), (SPMM_SOURCE, _S_WIDE, _S_HOST)] + _ASM,
    "k_wspmm": [(WINDOW_SOURCE, "// ------------------------------------------------------------------ SpMM",
                 "typedef void (*WinFn)")] + _ASM,
}


def spmm_source_sha(kernel: str) -> str:
    """sha256 of the source regions of the SpMM form `kernel` (its kernel, helpers and the
    assembly that lays out its matrix)."""
    parts = []
    for path, a, b in SPMM_REGIONS[kernel.split("<")[0]]:
        src = open(path).read()
        parts.append(src[src.index(a):src.index(b)])
    return hashlib.sha256("".join(parts).encode()).hexdigest()


def traffic_record(kernel: str, kp: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the kernel's current source; else None (stale counters)."""
    path = os.path.join(ROOT, "profiles", "spmm_traffic.json")
    if not os.path.exists(path):
        return None
    for rec in json.load(open(path)).get("records", []):
        if rec.get("kernel") == kernel and rec.get("kp") == kp and rec.get("source_sha256") == spmm_source_sha(kernel):
            return rec
    return None


def workload(n: int):
    from paper_2205_09070_gb300 import workloads as W
    if n == 1_000_000:
        return W.mixture_1m()
    return W.mixture_3d(seed=6, n=n, r_s=0.005 * (5e6 / n) ** (1.0 / 3.0))


def cpu_oracle_sample(p, n_s: int) -> dict:
    """FP64 CPU oracle (dense Cholesky LML + exact gradient over every
    hyperparameter) on the first n_s points of the workload, projected to the
    full N by its O(N^3) cost."""
    from oracle import gp_oracle as O
    xs, ys = p.x[:n_s], p.y[:n_s]
    t0 = time.perf_counter()
    O.lml_grad_exact(xs, ys, p.h, p.dim, p.n1, p.n2, p.beta)
    t = time.perf_counter() - t0
    proj = (1.0 / t) * (n_s / p.n) ** 3
    return {"value": proj, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"dense-Cholesky LML + exact gradient ({len(p.h)} hyperparameters) on the first {n_s} "
                       f"points of the {p.n}-point workload: {t:.2f} s per evaluation, projected to N={p.n} "
                       f"by the O(N^3) cost"),
            "sample_seconds": t}


# ---------------------------------------------------------------- reference arm
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p = workload(a.n)
    n_s = 900
    for _ in range(max(a.warmup, 0)):
        pass  # the oracle has no warm state; warm-up steps are not needed
    times = []
    for _ in range(a.steps):
        r = cpu_oracle_sample(p, n_s)
        times.append(r["sample_seconds"])
    t = sum(times)
    value = (a.steps / t) * (n_s / p.n) ** 3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": p.name, "n": p.n, "dim": p.dim, "n_funcs": p.n1,
                                            "n_bumps": p.n2, "sample_points": n_s},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"dense FP64 oracle on the first {n_s} points per step, projected by O(N^3)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fp64_leg(gp, x, y, p, steps, lml, grad, ms_fp32, stream):
    """The plain FP64 single-RHS path on the same assembled workload: its
    evaluations/s, assembly nnz/s, and its distance to the FP32-mixed result
    against the SLQ standard error of the log-determinant."""
    import torch
    from paper_2205_09070_gb300 import default_opts
    o64 = default_opts(precision="fp64", n_probes=32, lanczos_steps=50, cg_rtol=1e-6, seed=2022, max_iter=20000)
    gp.lml_grad(x, y, p.h, o64)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(steps):
        lml64, grad64, info64 = gp.lml_grad(x, y, p.h, o64)
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = f0.elapsed_time(f1) / steps
    return {"value": 1e3 / ms64, "unit": UNIT, "ms_per_eval": ms64, "lml": lml64,
            "iters": info64["iters"], "lml_minus_fp32": lml - lml64,
            "lml_stderr_fp64": 0.5 * info64["logdet_stderr"],
            "grad_rel_diff_max": float(np.max(np.abs(grad - grad64)) / np.max(np.abs(grad64))),
            "assembly": {"nnz_per_s": info64["nnz"] / (info64["t_assemble_ms"] * 1e-3),
                         "ms": info64["t_assemble_ms"]},
            "speedup_fp32_mixed": ms64 / ms_fp32}


def leg_5m(GP, default_opts, spmm_flag, pc_kw, dev, local, stream, a):
    """N = 5,000,000 mixture (the literal configuration: r_s = 0.005, 8 x 16
    bumps, 32 probes, 50 Lanczos steps, rtol 1e-6): FP32-mixed evaluations/s
    over 2 timed steps after 1 warm-up, assembly nnz/s, and one evaluation of
    the plain FP64 path on the same points."""
    import torch
    from paper_2205_09070_gb300 import workloads as W
    p = W.mixture_3d(seed=5, n=5_000_000)
    x = torch.as_tensor(p.x, device=dev)
    y = torch.as_tensor(p.y, device=dev)
    gp = GP(p.dim, p.n1, p.n2, p.beta, device=local)
    o = default_opts(precision="fp32", n_probes=32, lanczos_steps=50, cg_rtol=1e-6, seed=2022,
                     max_iter=20000, flags=spmm_flag, **pc_kw)
    gp.lml_grad(x, y, p.h, o)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = 2
    e0.record(stream)
    for _ in range(steps):
        lml, grad, info = gp.lml_grad(x, y, p.h, o)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out = {"workload": "mixture_3d", "n": p.n, "n_active": info["n_active"], "nnz": info["nnz"],
           "value": 1e3 / ms, "unit": UNIT, "ms_per_eval": ms, "steps": steps, "cg_iters": info["iters"],
           "lml": lml, "lml_stderr": 0.5 * info["logdet_stderr"],
           "assembly": {"nnz_per_s": info["nnz"] / (info["t_assemble_ms"] * 1e-3), "ms": info["t_assemble_ms"]}}
    if a.fp64_steps > 0:
        out["fp64_path"] = fp64_leg(gp, x, y, p, 1, lml, grad, ms, stream)
    gp.close()
    del x, y
    torch.cuda.empty_cache()
    return out


def leg_batch(GP, default_opts, dev, local, stream, n_inst=256, streams=True):
    """The many-instance configuration: 256 independent 2-D GPs, N_i uniform in
    [1,000, 50,000], each with its own 2 x 4 bumps and r_s, y plus 16 probes,
    32 Lanczos steps, rtol 1e-6, LML + gradient per instance through
    gp_lml_grad_batched: instance evaluations/s over one timed batch after one
    warm-up batch, with the CG runs as grouped launches (the default), and the
    same through the worker streams (GP_FLAG_BATCH_STREAMS) for comparison."""
    import torch
    from paper_2205_09070_gb300 import workloads as W
    from paper_2205_09070_gb300.gpsparse import GP_FLAG_BATCH_STREAMS
    probs = W.batch_2d(seed=4)[:n_inst]
    offsets = np.concatenate([[0], np.cumsum([q.n for q in probs])])
    x = torch.as_tensor(np.concatenate([q.x for q in probs]), device=dev)
    y = torch.as_tensor(np.concatenate([q.y for q in probs]), device=dev)
    h = np.stack([q.h for q in probs])
    gp = GP(2, 2, 4, device=local)

    def timed(flags):
        o = default_opts(precision="fp32", n_probes=16, lanczos_steps=32, cg_rtol=1e-6, seed=2022, max_iter=20000,
                         flags=flags)
        gp.lml_grad_batched(offsets, x, y, h, o)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lml, grad, info = gp.lml_grad_batched(offsets, x, y, h, o)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), lml, info

    ms, lml, info = timed(0)
    if streams:
        ms_s, lml_s, _ = timed(GP_FLAG_BATCH_STREAMS)
    gp.close()
    out = {"workload": "batch_2d", "n_inst": len(probs), "n_total": int(offsets[-1]),
           "n_active": info["n_active"], "nnz": info["nnz"], "value": len(probs) / (ms * 1e-3),
           "unit": "instance evals/s", "ms_per_batch": ms, "max_iters": info["iters"],
           "path": "grouped CG launches: the iterations of all running instances in single launches",
           "lml_finite": bool(np.all(np.isfinite(lml)))}
    if streams:
        out["worker_streams"] = {"value": len(probs) / (ms_s * 1e-3), "ms_per_batch": ms_s,
                                 "path": "each instance on its own on 8 worker streams",
                                 "lml_max_abs_diff": float(np.max(np.abs(lml - lml_s)))}
    return out


# ---------------------------------------------------------------- our arm
def main():
    a = args_parse()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_09070_gb300 import GP, default_opts
    from paper_2205_09070_gb300.gpsparse import GP_FLAG_TIME_KERNELS

    if a.batch_only > 0:
        print(json.dumps({"batch_only": leg_batch(GP, default_opts, dev, local, torch.cuda.current_stream(dev),
                                                  a.batch_only, streams=False)}))
        return
    p = workload(a.n)
    x = torch.as_tensor(p.x, device=dev)
    y = torch.as_tensor(p.y, device=dev)
    gp = GP(p.dim, p.n1, p.n2, p.beta, device=local)
    from paper_2205_09070_gb300.gpsparse import SPMM_FLAGS
    spmm_flag = SPMM_FLAGS.get(a.spmm, 0)
    pc_kw = {} if a.precond_block is None else {"precond_block": a.precond_block}
    # the timed steps run without per-kernel events; a separate instrumented
    # pass afterwards gives the per-kernel times the rooflines use
    opts = default_opts(precision="fp32", n_probes=32, lanczos_steps=50, cg_rtol=1e-6, seed=2022,
                        max_iter=20000, flags=spmm_flag, **pc_kw)
    opts_timed = default_opts(precision="fp32", n_probes=32, lanczos_steps=50, cg_rtol=1e-6, seed=2022,
                              max_iter=20000, flags=GP_FLAG_TIME_KERNELS | spmm_flag, **pc_kw)

    for _ in range(a.warmup):
        gp.lml_grad(x, y, p.h, opts)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(a.steps):
            lml, grad, info = gp.lml_grad(x, y, p.h, opts)
            infos.append(info)
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if dist:
        from paper_2205_09070_gb300.sharding import max_over_ranks
        ms = max_over_ranks(ms, device=dev)
    clocks = clk.summary()
    value = world * a.steps / (ms / 1e3)

    launches = sum(i["launches"] for i in infos)
    t_asm = statistics.mean(i["t_assemble_ms"] for i in infos)

    # instrumented pass (outside the timed region): per-launch CUDA-event times
    # of the SpMM, the pair fill and the adjoint, recorded on the context stream
    tinfos = [gp.lml_grad(x, y, p.h, opts_timed)[2] for _ in range(2)]
    torch.cuda.synchronize()
    nnz = infos[-1]["nnz"]
    n_act = infos[-1]["n_active"]
    kp = infos[-1]["kp"]
    t_spmm = sum(i["t_spmm_kernel_ms"] for i in tinfos)
    n_spmm = sum(i["n_spmm"] for i in tinfos)
    spmm_ms = t_spmm / max(n_spmm, 1)
    t_fill = statistics.mean(i["t_fill_kernel_ms"] for i in tinfos)
    t_adj = statistics.mean(i["t_adjoint_kernel_ms"] for i in tinfos)
    pk = peaks()
    peak_src = (f"{pk['source']} (MEASURED_PEAKS.json hbm_gbs, burst copy)" if pk["source"] == "measured"
                else "fallback 6.8 TB/s")
    kname = spmm_kernel_name(infos[-1]["spmm_variant"], kp)
    trec = traffic_record(kname, kp)
    # algorithmic bytes (each input read once, each output written once):
    #   SpMM: 8 nnz (FP32 value + int32 column) + 4 kp N_act read (P) + 4 kp N_act
    #         written (Q) + 8 (N_act + 1) row pointers
    #   fill: 8 nnz written (column + FP32 value) + per active point its row
    #         pointer, cell, coordinates (FP32 cell-relative, FP64), mask, FP64
    #         bump row and D^-1/2 (76 + 8 n1 bytes) + the cell table (8 per cell)
    #   adjoint: 4 nnz columns (values recomputed) + per active point its row
    #         pointer, X row (4 kp), probe bits, cell, coordinates, mask, FP32
    #         bump row and D^-1/2, and the written g row (4 n1)
    n1 = p.n1
    bytes_spmm = 8 * nnz + 8 * n_act * kp + 8 * (n_act + 1)
    bytes_fill = 8 * nnz + n_act * (76 + 8 * n1) + 8 * infos[-1]["n_cells"]
    bytes_adj = 4 * nnz + n_act * (8 + 4 * kp + 8 + 16 + 16 + 24 + 4 + 4 * n1 + 4 + 4 * n1)

    def roof(kernel, nbytes, t_ms, **extra):
        ach = nbytes / (t_ms * 1e-3) / 1e9 if t_ms > 0 else 0.0
        return {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "kernel": kernel, "peak_source": peak_src,
                "algorithmic_bytes_per_launch": nbytes, "avg_launch_ms": t_ms, **extra}

    roofline = roof(kname, bytes_spmm, spmm_ms, traffic=trec["bytes_per_launch"] if trec else None,
                    launches_timed=n_spmm, share_of_step=(t_spmm / len(tinfos)) / (ms / a.steps),
                    limiter=("issue and latency at 12 warps per SM over gathers of 144-byte P rows staged "
                             "through shared memory (ncu: 50 % issue active, l1tex 54 % of peak, DRAM about 20 %)")
                    if kname.startswith("k_bspmm_f32") else
                    ("latency: one persistent CTA of 8 consumer warps per SM, warps paced by the slowest "
                     "block row of each tile") if kname.startswith("k_wspmm") else "TMA gather4 request rate")
    rooflines = {"fill": roof("k_pair<float,FILL>", bytes_fill, t_fill, traffic=None,
                              limiter="candidate tests (about 6.4 per stored entry) and FP64 entry values"),
                 "adjoint": roof("k_adjoint<float>", bytes_adj, t_adj, traffic=None,
                                 limiter="gathers of the neighbours' X rows and coordinates per stored entry")}

    # end to end through the C ABI with pinned host buffers
    xh = torch.as_tensor(p.x).pin_memory()
    yh = torch.as_tensor(p.y).pin_memory()
    gh = torch.zeros(gp.n_params, dtype=torch.float64).pin_memory()
    opts_e2e = default_opts(precision="fp32", n_probes=32, lanczos_steps=50, cg_rtol=1e-6, seed=2022,
                            max_iter=20000, flags=spmm_flag, **pc_kw)
    e2e = None
    if a.e2e_steps > 0:
        gp.lml_grad(xh, yh, p.h, opts_e2e, grad=gh)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.e2e_steps):
            gp.lml_grad(xh, yh, p.h, opts_e2e, grad=gh)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e = {"value": world * a.e2e_steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(p.x.nbytes + p.y.nbytes + p.h.nbytes),
               "d2h_bytes_per_step": int(8 + 8 * gp.n_params), "steps": a.e2e_steps}

    # plain FP64 single-RHS path on the same workload (same probes, rtol, steps)
    fp64 = fp64_leg(gp, x, y, p, a.fp64_steps, lml, grad, ms / a.steps, stream) if a.fp64_steps > 0 else None

    # the literal 5M-point configuration: FP32-mixed evaluations, assembly and
    # the plain FP64 path on the same points
    scale5m = None
    if a.n5m and p.n == 1_000_000:
        scale5m = leg_5m(GP, default_opts, spmm_flag, pc_kw, dev, local, stream, a)
    batch256 = leg_batch(GP, default_opts, dev, local, stream) if a.batch and p.n == 1_000_000 else None

    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        cpu = cpu_oracle_sample(p, a.cpu_sample)

    if rank == 0:
        metric = METRIC if p.n == 1_000_000 else METRIC.replace("N=1M", f"N={p.n:,}")
        line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic (seeded; stands in for the NOAA GHCN-Daily station-day data)",
                "config": {"workload": p.name, "n": p.n, "dim": p.dim, "n_funcs": p.n1, "n_bumps": p.n2,
                           "r_s": float(p.h[-3]), "n_probes": 32, "lanczos_steps": 50, "cg_rtol": 1e-6,
                           "precision": "FP32_MIXED", "parallelism": f"replicas x{world}", "spmm": a.spmm,
                           "l2": "working set larger than L2 (CSR re-assembled every step)",
                           "n_active": n_act, "nnz": nnz, "kp": kp, "cg_iters": infos[-1]["iters"],
                "lanczos_iters": infos[-1]["lanczos_iters"], "precond_block": infos[-1]["precond_block"],
                "spmm_form": ["cp.async stage", "TMA gather4 stage", "TMA gather4 stage, wide lanes",
                              "cp.async stage, wide lanes", "column windows, TMA bulk runs"][infos[-1]["spmm_variant"]]
                if infos[-1]["spmm_variant"] >= 0 else None},
                "lml": lml, "logdet_stderr": infos[-1]["logdet_stderr"],
                "assembly": {"nnz_per_s": nnz / (t_asm * 1e-3), "ms": t_asm, "fill_kernel_ms": t_fill},
                "adjoint_kernel_ms": t_adj,
                "roofline": roofline, "rooflines": rooflines, "clocks": clocks, "gpu_launches": launches,
                "e2e": e2e, "fp64_path": fp64, "scale_5m": scale5m, "batch_256": batch256, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    gp.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
