#!/usr/bin/env python3
"""Benchmark of the element-by-element (EbE) residual + Jacobi-PCG path on GB300.

Workload (default): the unit square with 2049 x 2049 nodes, P1 triangles split
SW-NE, interior nodes jittered by U[-0.2h, 0.2h] (seed 2), nu = 1,
f = (2 pi^2 + nu) sin(pi x) sin(pi y), Dirichlet 0 on x = 0 and y = 0,
homogeneous Neumann elsewhere: 4,198,401 nodes, 8,388,608 elements.

One step = one pass of the whole hot path on that input: element matrices
A_e = K_e + nu M_e (FP64, plus an FP32 copy), load vector and Jacobi diagonal,
then Jacobi-PCG from x0 = 0 to FP64 true relative residual 1e-8 with FP32
element matrices and vectors and FP64 reliable updates (the mixed-precision
solver).  The mesh partition (built once per mesh, like the paper's index
arrays) and the inputs are resident on the device before the timed region.

value = algorithmic bytes of the step (every kernel's minimum traffic: each
of the n_b^2 element matrix entries, connectivity index and node vector entry
counted once per pass; the library keeps only the n_b(n_b+1)/2 distinct
entries of the symmetric A_e, and reports that count too) / step time, in GB/s; the plain FP64 Jacobi-PCG of the same problem is
timed beside it ("plain_fp64").  The roofline object is the FP32 operator
application (patch kernel + halo fix-up) timed per launch with CUDA events on
its stream.  e2e repeats the step through the C ABI from pinned host buffers:
mesh, f and boundary sets in, solution out, including the partition build.

"batched" (skip with --no-batch): 256 independent squares (sides log-uniform
in [17, 513] nodes, seed 4) solved by the batched persistent solver in mixed
precision with an autotuned launch shape, against the same problems solved
one by one with ebe_solve (plain FP64 and mixed) and the batched FP64 solve.

"cube129" (skip with --no-cube): the 3D configuration, 129^3 nodes in 6 Kuhn
tetrahedra per cell, mixed-precision and plain FP64 solves to 1e-8 and the
operator rooflines.  "paper_experiment": the paper's own timed experiment
(Sec. 3, the 1025^2 square: element arrays and 124 Richardson / Chebyshev
iterations), beside the MATLAB times the paper quotes, as context.

"nu0" (skip with --no-nu0): the same 2049^2 workload with nu = 0, mixed and
plain FP64.  "square33" (skip with --no-small): the 33^2 square (2048
triangles, nu = 1, f = 1, Dirichlet 0), time to solution and per iteration.
"residual_variants_fp64" (skip with --no-variants): the FP64 residual with the
patch scatter against the node-centric, colour-by-colour and atomic ones.

"learned" (skip with --no-learned): the message-passing preconditioner trained
on 257^2 squares and deployed in flexible CG on 1025^2 and 2049^2, against
flexible CG with Jacobi and Jacobi-PCG (plain FP64 and mixed).

"summary", the line's last key, repeats every number of the metric in short
form: PCG time to 1e-8, mixed against plain FP64, per workload.

--impl reference times the FP64 CPU oracle (test infrastructure) on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EbE residual GB/s (% HBM peak); PCG time to FP64 rel. residual 1e-8 vs plain"


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=2049, help="nodes per side of the square")
    ap.add_argument("--nu", type=float, default=1.0)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip timing the comparison scatters")
    ap.add_argument("--no-nu0", action="store_true", help="skip the nu = 0 leg of the 2049^2 workload")
    ap.add_argument("--no-small", action="store_true", help="skip the 33^2 workload")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload (256 independent squares)")
    ap.add_argument("--batch-problems", type=int, default=256)
    ap.add_argument("--no-cube", action="store_true", help="skip the 129^3 tetrahedral workload")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip training the learned preconditioner (257^2) and deploying it (1025^2, 2049^2)")
    ap.add_argument("--profile-kernel", choices=["apply32", "residual64", "dw", "assemble", "vec", "cg", "small", "batch", "mpnn", "dw_cube"], default=None,
                    help="run a few launches of one kernel for an ncu capture (no JSON line)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- byte model
def bytes_model(dim: int, n_n: int, n_e: int, stored: bool = False):
    """Algorithmic bytes of each pass (each entry counted once per pass).

    Element: the n_b^2 entries of A_e (the method's n_b x n_b x n_e element
    arrays) + n_b int32 connectivity indices.  stored=True counts instead the
    n_b(n_b+1)/2 distinct entries of the symmetric A_e, which is what the
    library keeps and reads.
    Node vectors: every vector read or written by the pass, once.
    """
    nb = dim + 1
    na = nb * (nb + 1) // 2 if stored else nb * nb
    conn = 4 * nb * n_e
    m = {}
    # element matrices + load vector + Jacobi diagonal: coords (dim f64) + f (f64) in,
    # A64 + A32 out, b, d, dinv (f64) + b32, dinv32 (f32) out
    m["assemble_mixed"] = conn + n_n * 8 * (dim + 1) + n_e * na * (8 + 4) + n_n * (3 * 8 + 2 * 4)
    m["assemble_fp64"] = conn + n_n * 8 * (dim + 1) + n_e * na * 8 + n_n * 3 * 8
    m["residual64"] = conn + n_e * na * 8 + n_n * 3 * 8          # x, b in; r out
    m["residual32"] = conn + n_e * na * 4 + n_n * 3 * 4
    m["apply64"] = conn + n_e * na * 8 + n_n * 2 * 8             # p in; q out
    m["apply32"] = conn + n_e * na * 4 + n_n * 2 * 4
    # update (x, p, r, q, dinv in; x, r out) + direction (r, dinv, p in; p out)
    m["vec64"] = n_n * 8 * (7 + 4)
    m["vec_mixed"] = n_n * ((8 + 4 + 4 + 4 + 4) + (8 + 4) + (4 + 4 + 4) + 4)   # x FP64; r, p, q, dinv FP32
    # after a true residual: r.z and r.r (r64, dinv in; r32 out), then a direction step
    m["restart_mixed"] = n_n * ((8 + 4 + 4) + (4 + 4 + 4 + 4))
    m["restart64"] = n_n * ((8 + 8) + (8 + 8 + 8 + 8))
    # one iteration of the single-sync mixed solver (one pass): the operator's
    # element matrices and connectivity, and per node r, q, p, dinv (4 B) and
    # x (8 B) in, r, p, q (4 B) and x (8 B) out -- the direction the operator
    # applies is formed in registers, not read
    m["cg_mixed"] = conn + n_e * na * 4 + n_n * (4 * 4 + 8 + 3 * 4 + 8)
    # restart of the single-sync recurrence: r64, dinv in, r32 out
    m["cg_restart"] = n_n * (8 + 4 + 4)
    return m


def fp64_alu_model(nb: int, n_n: int, n_e: int, sms: int, mhz):
    """FP64-pipe ceiling of one FP64 residual (patch pass + fix-up).

    Operations on the FP64 pipe: the n_b x n_b local product (n_b^2 multiply
    or fused multiply-add instructions) and the n_b additions into the node
    sums per element, then r = b - sum and the r.r accumulation per node.
    GB300 issues two FP64 operations per SM and clock (1.25 TFLOP/s nominal
    counts an FMA as two flops).  Returns None when the clock is unknown."""
    if not mhz or not sms:
        return None
    ops = n_e * (nb * nb + nb) + 2 * n_n
    return {"ops_per_launch": int(ops), "peak_gops": round(2.0 * sms * float(mhz) * 1e6 / 1e9, 1)}


def step_bytes(m, info, mixed: bool, textbook: bool = False):
    """Algorithmic bytes of one step: element matrices, then the solve as it
    runs.  Mixed (single-sync solver): one pass per iteration plus one first
    pass per start of the recurrence (the initial one and every replacement),
    a restart and an FP64 true residual per check.  Textbook iteration
    (plain FP64, and the mixed arithmetic in that form, as the batched solver
    runs it): operator, update and direction per iteration, a true residual
    per check and a restart per replacement."""
    it, tr = info["iterations"], info["true_residuals"]
    if mixed and not textbook:
        return (m["assemble_mixed"] + (it + tr) * m["cg_mixed"] + tr * (m["residual64"] + m["cg_restart"]))
    if mixed:
        return (m["assemble_mixed"] + it * (m["apply32"] + m["vec_mixed"]) + tr * m["residual64"]
                + max(tr - 1, 0) * m["restart_mixed"])
    return m["assemble_fp64"] + it * (m["apply64"] + m["vec64"]) + tr * m["residual64"] + max(tr - 1, 0) * m["restart64"]


def solve_bytes(m, info, mixed: bool, textbook: bool = False):
    """step_bytes without the element-matrix generation."""
    return step_bytes(m, info, mixed, textbook) - m["assemble_mixed" if mixed else "assemble_fp64"]


# ----------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------------------- dist helpers
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_over_ranks(dist, device, seconds_or_ms, nbytes):
    """Whole-job figures of N replicas (one rank per GPU, each running the full
    workload): the slowest rank's time and the bytes of all ranks.  dist is
    torch.distributed (any backend) or None for a single process."""
    if dist is None:
        return seconds_or_ms, nbytes
    import torch
    t = torch.tensor([float(seconds_or_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    b = torch.tensor([float(nbytes)], dtype=torch.float64, device=device)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(t.item()), float(b.item())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_record(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, valid only
    while the kernel source is unchanged (source hash recorded beside it)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_1911_03973_gb300", "csrc", "k_patch.cu")
    if not os.path.exists(path):
        return None
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for line in open(path):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#") and f[0] == kernel and f[1] == digest:
            return float(f[2])
    return None


# ----------------------------------------------------------------------------- batched workload
def run_batch(args, dev, stream, profile=False):
    """Many independent problems: 256 squares with sides log-uniform in [17, 513]
    nodes, nu log-uniform in [1e-2, 10], 8 random Fourier modes of f, Dirichlet 0
    (seed 4).  The batched persistent solver (mixed precision, autotuned launch
    shape) against the same problems solved one by one with ebe_solve."""
    import torch
    import paper_1911_03973_gb300 as ebe
    from paper_1911_03973_gb300 import meshgen

    n_prob = 64 if profile else args.batch_problems
    probs = meshgen.config_batch(n_prob, seed=4)
    U = meshgen.batch_union(probs)
    n = int(U["node_off"][-1])
    with torch.cuda.stream(stream):
        h = ebe.ebe_create_batch(U["meshes"], device=dev.index, stream=stream.cuda_stream)
        ebe.ebe_set_problem_batch(h, U["nu"], U["f"], U["dirichlet"], U["g"], U["neumann"])
        ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        if profile:
            # one persistent launch of a few loop iterations (every problem stops at maxit)
            for _ in range(2):
                x.zero_()
                ebe.ebe_solve_batch(h, x, rtol=args.rtol, precision=ebe.EBE_PREC_MIXED, maxit=20)
            torch.cuda.synchronize()
            ebe.ebe_destroy(h)
            return None
        tune = ebe.ebe_batch_tune(h, ebe.EBE_PREC_MIXED, loops=40)

        def timed(prec, reps):
            best, res = None, None
            for _ in range(reps):
                x.zero_()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                infos, summ = ebe.ebe_solve_batch(h, x, rtol=args.rtol, precision=prec)
                ev1.record(stream)
                torch.cuda.synchronize()
                t = ev0.elapsed_time(ev1)
                if summ["n_converged"] != n_prob:
                    raise RuntimeError(f"batched solve: {n_prob - summ['n_converged']} problems did not converge")
                if best is None or t < best:
                    best, res = t, (infos, summ)
            return best, res

        ms_mixed, (infos, summ) = timed(ebe.EBE_PREC_MIXED, 3)
        ms_b64, (infos64, _) = timed(ebe.EBE_PREC_FP64, 1)
        ebe.ebe_destroy(h)
        # the same problems one by one (a handle per problem, as a user without batches would)
        handles = []
        for p in probs:
            hh = ebe.ebe_create(p["coords"], p["elems"], device=dev.index, stream=stream.cuda_stream)
            ebe.ebe_set_problem(hh, p["nu"], p["f"], p["dirichlet"], p["g"], p["neumann"])
            ebe.ebe_assemble(hh, ebe.EBE_STORE_MIXED)
            handles.append(hh)
        xs = [torch.zeros(p["coords"].shape[0], dtype=torch.float64, device=dev) for p in probs]
        seq = {}
        for name, prec in (("fp64", ebe.EBE_PREC_FP64), ("mixed", ebe.EBE_PREC_MIXED)):
            ebe.ebe_solve(handles[0], xs[0], rtol=args.rtol, precision=prec)     # graph capture outside the timing
            for v in xs:
                v.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for hh, v in zip(handles, xs):
                i = ebe.ebe_solve(hh, v, rtol=args.rtol, precision=prec)
                if i["status"] != "EBE_OK":
                    raise RuntimeError(f"sequential solve failed: {i}")
            ev1.record(stream)
            torch.cuda.synchronize()
            seq[name] = ev0.elapsed_time(ev1)
        for hh in handles:
            ebe.ebe_destroy(hh)
    byt = 0
    for p, i in zip(probs, infos):
        mk = bytes_model(p["coords"].shape[1], p["coords"].shape[0], p["elems"].shape[0])
        byt += solve_bytes(mk, i, True, textbook=True)     # the batched solver's textbook iteration
    its = [i["iterations"] for i in infos]
    return {
        "workload": f"batch{n_prob}_squares17-513_seed4", "n_problems": n_prob, "n_nodes": n,
        "n_elements": int(U["elem_off"][-1]), "solver": "one persistent cooperative launch, mixed precision",
        "ms_to_1e-8": round(ms_mixed, 2), "loops": summ["loops"], "iterations_max": max(its),
        "iterations_sum": sum(its), "shape": [summ["ctas_per_sm"], summ["tile_nodes"]],
        "phase_ms": {k: round(v, 2) for k, v in summ["phase_ms"].items()},
        "tuned_ms_per_loop": {f"{c}x{t}": round(ms, 4) for c, t, ms in tune["candidates"]},
        "gbs": round(byt / (ms_mixed / 1e3) / 1e9, 1),
        "batched_fp64_ms": round(ms_b64, 2),
        "sequential_fp64_ms": round(seq["fp64"], 2), "sequential_mixed_ms": round(seq["mixed"], 2),
        "speedup_vs_sequential_fp64": round(seq["fp64"] / ms_mixed, 3),
        "speedup_vs_sequential_mixed": round(seq["mixed"] / ms_mixed, 3),
    }


# ----------------------------------------------------------------------------- learned preconditioner
def run_cube(args, dev, stream):
    """The 3D configuration: the unit cube with 129^3 nodes, 6 Kuhn tetrahedra per
    cell (12,582,912 elements), nu = 0.5, f = 1 + 0.1 N(0,1) per node (seed 3),
    Dirichlet 0 on z = 0: mixed-precision and plain FP64 Jacobi-PCG to 1e-8
    (CUDA events around ebe_solve, element matrices assembled beforehand) and
    the per-launch times of the FP32 operator and the FP64 residual."""
    import torch
    import paper_1911_03973_gb300 as ebe
    from paper_1911_03973_gb300 import meshgen
    prob = meshgen.config_cube_noise(129, nu=0.5, seed=3)
    n_n, dim = prob["coords"].shape
    n_e = prob["elems"].shape[0]
    m = bytes_model(dim, n_n, n_e)
    out = {"workload": "cube129_kuhn_nu0.5_noise0.1_tet", "n_nodes": n_n, "n_elements": n_e, "n_b": dim + 1}
    with torch.cuda.stream(stream):
        h = ebe.ebe_create(prob["coords"], prob["elems"], device=dev.index, stream=stream.cuda_stream)
        ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
        ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
        x = torch.zeros(n_n, dtype=torch.float64, device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for key, prec in (("mixed", ebe.EBE_PREC_MIXED), ("plain_fp64", ebe.EBE_PREC_FP64)):
            times = []
            for rep_ in range(3):
                x.zero_()
                ev[0].record(stream)
                info = ebe.ebe_solve(h, x, rtol=args.rtol, precision=prec)
                ev[1].record(stream)
                ev[1].synchronize()
                if info["status"] != "EBE_OK":
                    raise RuntimeError(f"cube solve failed: {info}")
                if rep_ > 0:
                    times.append(ev[0].elapsed_time(ev[1]))
            out[key] = {"ms_to_1e-8": round(min(times), 2), "iterations": info["iterations"],
                        "true_residuals": info["true_residuals"], "rel_residual": info["rel_residual"]}
        out["speedup_vs_plain"] = round(out["plain_fp64"]["ms_to_1e-8"] / out["mixed"]["ms_to_1e-8"], 3)
        p32 = torch.rand(n_n, dtype=torch.float32, device=dev)
        q32 = torch.empty_like(p32)
        x64 = torch.rand(n_n, dtype=torch.float64, device=dev)
        r64 = torch.empty_like(x64)
        ebe.ebe_time_operator(h, p32, q32, True, 5)
        a32 = ebe.ebe_time_operator(h, p32, q32, True, 20)
        ebe.ebe_time_operator(h, x64, r64, False, 5)
        r64t = ebe.ebe_time_operator(h, x64, r64, False, 20)
        ebe.ebe_time_operator(h, x64, r64, False, 3, double_word=True)
        rdw = ebe.ebe_time_operator(h, x64, r64, False, 20, double_word=True)
        peak = peaks()[0]
        gdw = m["residual64"] / (sum(rdw) / 1e3) / 1e9
        g32 = m["apply32"] / (sum(a32) / 1e3) / 1e9
        g64 = m["residual64"] / (sum(r64t) / 1e3) / 1e9
        out["apply32"] = {"ms_per_launch": [round(a32[0], 5), round(a32[1], 5)], "bytes_per_launch": m["apply32"],
                          "gbs": round(g32, 1), "frac": round(g32 / peak, 4)}
        out["residual64"] = {"ms_per_launch": [round(r64t[0], 5), round(r64t[1], 5)],
                             "bytes_per_launch": m["residual64"], "gbs": round(g64, 1), "frac": round(g64 / peak, 4)}
        out["residual_dw"] = {"ms_per_launch": [round(rdw[0], 5), round(rdw[1], 5)],
                              "bytes_per_launch": m["residual64"], "gbs": round(gdw, 1), "frac": round(gdw / peak, 4)}
        ebe.ebe_time_cg_pass(h, reps=5)
        cgt = ebe.ebe_time_cg_pass(h, reps=40)
        gcg = m["cg_mixed"] / (sum(cgt) / 1e3) / 1e9
        out["cg_pass"] = {"ms_per_launch": [round(cgt[0], 5), round(cgt[1], 5)], "bytes_per_launch": m["cg_mixed"],
                          "gbs": round(gcg, 1), "frac": round(gcg / peak, 4)}
        ebe.ebe_destroy(h)
    return out


def _timed_solve(ebe, torch, h, x, stream, reps, **kw):
    """Best of `reps` timed ebe_solve calls from x0 = 0 (CUDA events on the
    handle's stream, one untimed call first); returns (ms, info)."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    x.zero_()
    ebe.ebe_solve(h, x, **kw)
    best, info = None, None
    for _ in range(reps):
        x.zero_()
        ev[0].record(stream)
        i = ebe.ebe_solve(h, x, **kw)
        ev[1].record(stream)
        ev[1].synchronize()
        if i["status"] != "EBE_OK":
            raise RuntimeError(f"solve failed: {i}")
        t = ev[0].elapsed_time(ev[1])
        if best is None or t < best:
            best, info = t, i
    return best, info


def run_pcg_leg(args, dev, stream, prob, reps=1):
    """Mixed-precision and plain FP64 Jacobi-PCG to FP64 rel. residual rtol on
    one problem, element matrices assembled beforehand (both stored):
    CUDA-event times of ebe_solve, iterations, speed-up of mixed over plain."""
    import torch
    import paper_1911_03973_gb300 as ebe
    n_n = prob["coords"].shape[0]
    with torch.cuda.stream(stream):
        h = ebe.ebe_create(prob["coords"], prob["elems"], device=dev.index, stream=stream.cuda_stream)
        ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
        ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
        x = torch.zeros(n_n, dtype=torch.float64, device=dev)
        out = {}
        for key, prec in (("mixed", ebe.EBE_PREC_MIXED), ("plain_fp64", ebe.EBE_PREC_FP64)):
            ms, info = _timed_solve(ebe, torch, h, x, stream, reps, rtol=args.rtol, precision=prec)
            out[key] = {"ms_to_1e-8": round(ms, 3), "iterations": info["iterations"],
                        "true_residuals": info["true_residuals"], "rel_residual": info["rel_residual"],
                        "us_per_iteration": round(1e3 * ms / max(info["iterations"], 1), 2)}
        out["speedup_vs_plain"] = round(out["plain_fp64"]["ms_to_1e-8"] / out["mixed"]["ms_to_1e-8"], 3)
        ebe.ebe_destroy(h)
    return out


def run_paper_experiment(dev, stream):
    """The paper's own timed experiment (Sec. 3), as context: the 1025^2 square,
    nu = 0, f = 1, u = 1 on the boundary; the element matrix arrays K_e, M_e and
    124 iterations of Richardson and of the three-level Chebyshev method with
    the spectral bounds of the structured mesh.  The paper quotes about 5 s per
    array and about 50 s per method in MATLAB on hardware it does not name."""
    import torch
    import paper_1911_03973_gb300 as ebe
    from paper_1911_03973_gb300 import meshgen
    n = 1025
    prob = meshgen.config_square_f1(n, nu=0.0, g_value=1.0)
    n_n, n_e, nb = prob["coords"].shape[0], prob["elems"].shape[0], prob["elems"].shape[1]
    lam1 = 8.0 * math.sin(math.pi / (2 * (n - 1))) ** 2          # bounds of the stencil spectrum
    lam2 = 8.0 * math.sin((n - 2) * math.pi / (2 * (n - 1))) ** 2
    out = {"workload": "square1025_f1_nu0_u1 (Sec. 3 experiment)", "n_nodes": n_n, "n_elements": n_e,
           "paper_matlab_s": {"K_e_array": 5.0, "M_e_array": 5.0, "124_iterations_per_method": 50.0}}
    with torch.cuda.stream(stream):
        h = ebe.ebe_create(prob["coords"], prob["elems"], device=dev.index, stream=stream.cuda_stream)
        ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
        K = torch.empty(n_e * nb * nb, dtype=torch.float64, device=dev)
        M = torch.empty_like(K)
        x = torch.zeros(n_n, dtype=torch.float64, device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

        def timed(fn, reps=3):
            fn()
            best = None
            for _ in range(reps):
                ev[0].record(stream)
                fn()
                ev[1].record(stream)
                ev[1].synchronize()
                t = ev[0].elapsed_time(ev[1])
                best = t if best is None else min(best, t)
            return round(best, 3)
        out["K_e_M_e_arrays_ms"] = timed(lambda: ebe.ebe_element_matrices(h, K, M))
        out["assemble_fp64_ms"] = timed(lambda: ebe.ebe_assemble(h, ebe.EBE_STORE_FP64))

        def rich():
            x.zero_()
            ebe.ebe_richardson(h, x, 124, 2.0 / (lam1 + lam2))

        def cheb2():
            x.zero_()
            ebe.ebe_chebyshev2_bounds(h, x, 124, lam1, lam2, 32)

        def cheb3():
            x.zero_()
            ebe.ebe_chebyshev3(h, x, 124, lam1, lam2)
        out["richardson_124_ms"] = timed(rich)
        out["chebyshev2_N32_124_ms"] = timed(cheb2)
        out["chebyshev3_124_ms"] = timed(cheb3)
        ebe.ebe_destroy(h)
    return out


def run_learned(args, dev, stream, profile=False):
    """Train the message-passing preconditioner on 257^2 jittered squares
    (random Fourier f, nu ~ U[0, 10]; 4 problems x 12 residual/error pairs
    from Jacobi-PCG, 1500 Adam steps), then solve unseen 1025^2 and 2049^2
    problems of the same kind with flexible CG + network, flexible CG +
    Jacobi, plain FP64 Jacobi-PCG and mixed-precision Jacobi-PCG."""
    import torch
    import paper_1911_03973_gb300 as ebe
    from paper_1911_03973_gb300 import learned

    def setup(n, seed):
        p = learned.training_problem(n, seed)
        h = ebe.ebe_create(p["coords"], p["elems"], device=dev.index, stream=stream.cuda_stream)
        ebe.ebe_set_problem(h, p["nu"], p["f"], p["dirichlet"], p["g"], p["neumann"])
        ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
        return p, h

    with torch.cuda.stream(stream):
        if profile:
            # three network applications on 1025^2 with seeded non-zero weights
            rng = np.random.Generator(np.random.PCG64(4))
            net = ebe.ebe_mpnn_create(dev.index, rng.normal(0, 0.1, ebe.ebe_mpnn_n_params()))
            p, h = setup(1025, 999)
            r = torch.rand(p["coords"].shape[0], dtype=torch.float64, device=dev)
            z = torch.empty_like(r)
            for _ in range(3):
                ebe.ebe_mpnn_apply(net, h, r, z)
            torch.cuda.synchronize()
            return None
        t0 = time.perf_counter()
        samples, keep = [], []
        for seed in range(4):
            p, h = setup(257, 100 + seed)
            keep.append(h)
            for r, e in learned.harvest(ebe, torch, h, p["coords"].shape[0], 12, dev):
                samples.append((h, r, e))
        t_harvest = time.perf_counter() - t0
        net = ebe.ebe_mpnn_create(dev.index)
        t0 = time.perf_counter()
        losses = learned.train(ebe, net, samples, steps=1500, lr=3e-3, seed=1)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        out = {"train": {"problems": "4 x 257^2 jittered, random Fourier f, nu ~ U[0,10]", "samples": len(samples),
                         "steps": 1500, "harvest_s": round(t_harvest, 1), "train_s": round(t_train, 2),
                         "loss_first64": round(float(np.mean(losses[:64])), 4),
                         "loss_last64": round(float(np.mean(losses[-64:])), 4)}}
        for n in (1025, 2049):
            p, h = setup(n, 999)
            nn = p["coords"].shape[0]

            def timed(fn):
                # the second of two calls: buffers, the mesh graph and CUDA
                # graphs of the solvers exist, as in a steady stream of solves
                x = torch.zeros(nn, dtype=torch.float64, device=dev)
                fn(x)
                x.zero_()
                torch.cuda.synchronize()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                info = fn(x)
                ev1.record(stream)
                torch.cuda.synchronize()
                return info, ev0.elapsed_time(ev1)

            ij, tj = timed(lambda x: ebe.ebe_solve_learned(h, None, x, rtol=args.rtol))
            il, tl = timed(lambda x: ebe.ebe_solve_learned(h, net, x, rtol=args.rtol))
            i0, t0n = timed(lambda x: ebe.ebe_solve_learned(h, net, x, rtol=args.rtol, race_iters=0))
            ip, tp = timed(lambda x: ebe.ebe_solve(h, x, rtol=args.rtol, precision=ebe.EBE_PREC_FP64))
            im, tm = timed(lambda x: ebe.ebe_solve(h, x, rtol=args.rtol, precision=ebe.EBE_PREC_MIXED))
            r = torch.rand(nn, dtype=torch.float64, device=dev)
            z = torch.empty_like(r)
            ebe.ebe_mpnn_apply(net, h, r, z)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(10):
                ebe.ebe_mpnn_apply(net, h, r, z)
            ev1.record(stream)
            torch.cuda.synchronize()
            out[f"square{n}"] = {
                "learned_fcg": {"ms": round(tl, 1), "iterations": il["iterations"], "fell_back": il["fell_back"],
                                "status": il["status"], "rule": "race of 16 Jacobi / 16 network iterations; a lost or undecided race or a slow window hands over to the mixed Jacobi-PCG"},
                "network_first": {"ms": round(t0n, 1), "iterations": i0["iterations"], "fell_back": i0["fell_back"],
                                  "rule": "network from the start, fallback rules only"},
                "jacobi_fcg": {"ms": round(tj, 1), "iterations": ij["iterations"]},
                "plain_fp64_pcg": {"ms": round(tp, 1), "iterations": ip["iterations"]},
                "mixed_pcg": {"ms": round(tm, 1), "iterations": im["iterations"]},
                "network_apply_ms": round(ev0.elapsed_time(ev1) / 10, 3)}
            ebe.ebe_destroy(h)
        for h in keep:
            ebe.ebe_destroy(h)
        ebe.ebe_mpnn_destroy(net)
    return out


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import paper_1911_03973_gb300 as ebe
    from paper_1911_03973_gb300 import build as ebe_build
    from paper_1911_03973_gb300 import meshgen

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
    if rank == 0:
        ebe_build.build()
    if dist:
        dist.barrier()
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    if args.profile_kernel == "small":
        # three mixed solves of the 33^2 square of the small configuration: one
        # launch of the one-CTA solver each
        p = meshgen.config_square_f1(33, nu=1.0)
        with torch.cuda.stream(stream):
            h = ebe.ebe_create(p["coords"], p["elems"], device=dev.index, stream=stream.cuda_stream)
            ebe.ebe_set_problem(h, p["nu"], p["f"], p["dirichlet"], p["g"], p["neumann"])
            ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
            x = torch.zeros(p["coords"].shape[0], dtype=torch.float64, device=dev)
            for _ in range(3):
                x.zero_()
                ebe.ebe_solve(h, x, rtol=1e-8, precision=ebe.EBE_PREC_MIXED)
            torch.cuda.synchronize()
            ebe.ebe_destroy(h)
        return None
    if args.profile_kernel == "batch":
        run_batch(args, dev, stream, profile=True)
        return None
    if args.profile_kernel == "mpnn":
        run_learned(args, dev, stream, profile=True)
        return None
    if args.profile_kernel == "dw_cube":
        # the double-word residual on the 129^3 tetrahedral workload
        prob = meshgen.config_cube_noise(129, nu=0.5, seed=3)
    else:
        prob = meshgen.config_square_jitter(args.n, nu=args.nu, seed=2)
    n_n, dim = prob["coords"].shape
    n_e = prob["elems"].shape[0]
    m = bytes_model(dim, n_n, n_e)
    m_stored = bytes_model(dim, n_n, n_e, stored=True)

    with torch.cuda.stream(stream):
        h = ebe.ebe_create(prob["coords"], prob["elems"], device=dev.index, stream=stream.cuda_stream)
        ebe.ebe_set_problem(h, prob["nu"], prob["f"], prob["dirichlet"], prob["g"], prob["neumann"])
        x = torch.zeros(n_n, dtype=torch.float64, device=dev)

        if args.profile_kernel:
            ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
            p32 = torch.rand(n_n, dtype=torch.float32, device=dev)
            q32 = torch.empty_like(p32)
            x64 = torch.rand(n_n, dtype=torch.float64, device=dev)
            r64 = torch.empty_like(x64)
            if args.profile_kernel == "vec":
                # three textbook mixed-precision CG iterations, launched one by one
                ebe.ebe_solve(h, x, rtol=1e-300, maxit=3, precision=ebe.EBE_PREC_MIXED_TEXTBOOK, chunk=1,
                              use_graph=False)
                torch.cuda.synchronize()
                return None
            if args.profile_kernel == "cg":
                # four single-sync passes (fresh pass + three iterations), launched one by one
                ebe.ebe_solve(h, x, rtol=1e-300, maxit=3, precision=ebe.EBE_PREC_MIXED, chunk=1, use_graph=False)
                torch.cuda.synchronize()
                return None
            for _ in range(3):
                if args.profile_kernel == "apply32":
                    ebe.ebe_apply(h, p32, q32)
                elif args.profile_kernel == "residual64":
                    ebe.ebe_residual(h, x64, r64)
                elif args.profile_kernel in ("dw", "dw_cube"):
                    ebe.ebe_residual(h, x64, r64, double_word=True)
                else:
                    ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
            torch.cuda.synchronize()
            return None

        def step(mixed=True):
            ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED if mixed else ebe.EBE_STORE_FP64)
            x.zero_()
            info = ebe.ebe_solve(h, x, rtol=args.rtol, precision=ebe.EBE_PREC_MIXED if mixed else ebe.EBE_PREC_FP64)
            if info["status"] != "EBE_OK":
                raise RuntimeError(f"solve failed: {info}")
            return info

        for _ in range(args.warmup):
            step()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = ebe.ebe_get_stats(h)["kernel_launches"]
        clocks = Clocks(dev.index)
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        infos = []
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        if dist:
            dist.barrier()
        ms_total = e0.elapsed_time(e1)
        launches = ebe.ebe_get_stats(h)["kernel_launches"] - l0
        bytes_total = sum(step_bytes(m, i, True) for i in infos)
        ms_total, bytes_total = reduce_over_ranks(dist, dev, ms_total, bytes_total)
        ms_step = ms_total / args.steps
        value = bytes_total / (ms_total / 1e3) / 1e9

        # plain FP64 Jacobi-PCG on the same problem ("vs plain")
        pinfo = []
        ms_plain = None
        if args.plain_steps > 0:
            ep0 = torch.cuda.Event(enable_timing=True)
            ep1 = torch.cuda.Event(enable_timing=True)
            step(mixed=False)
            ep0.record(stream)
            for _ in range(args.plain_steps):
                pinfo.append(step(mixed=False))
            ep1.record(stream)
            torch.cuda.synchronize()
            ms_plain = ep0.elapsed_time(ep1) / args.plain_steps
        # the same mixed-precision arithmetic in the textbook four-launch iteration
        ms_text, tinfo = None, None
        if args.plain_steps > 0:
            ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
            ms_text, tinfo = _timed_solve(ebe, torch, h, x, stream, 1, rtol=args.rtol,
                                          precision=ebe.EBE_PREC_MIXED_TEXTBOOK)

        # roofline: the solver's iteration (single-sync pass: patch + fix-up)
        # and the plain FP32 operator application, per-launch events on the stream
        ebe.ebe_assemble(h, ebe.EBE_STORE_MIXED)
        ebe.ebe_time_cg_pass(h, reps=5)
        ms_cg = ebe.ebe_time_cg_pass(h, reps=40)
        p32 = torch.rand(n_n, dtype=torch.float32, device=dev)
        q32 = torch.empty_like(p32)
        ms_patch, ms_fix = ebe.ebe_time_operator(h, p32, q32, apply=True, reps=20)
        x64 = torch.rand(n_n, dtype=torch.float64, device=dev)
        r64 = torch.empty_like(x64)
        ms_patch64, ms_fix64 = ebe.ebe_time_operator(h, x64, r64, apply=False, reps=20)
        ebe.ebe_time_operator(h, x64, r64, apply=False, reps=3, double_word=True)
        ms_dw = ebe.ebe_time_operator(h, x64, r64, apply=False, reps=20, double_word=True)
        variants = None
        if not args.no_variants:
            variants = {}
            for name in ("PATCH", "COLOUR", "NODE", "ATOMIC"):
                code = getattr(ebe, f"EBE_SCATTER_{name}")
                ebe.ebe_residual_variant(h, x64, r64, code)
                ev_a = torch.cuda.Event(enable_timing=True)
                ev_b = torch.cuda.Event(enable_timing=True)
                ev_a.record(stream)
                for _ in range(10):
                    ebe.ebe_residual_variant(h, x64, r64, code)
                ev_b.record(stream)
                torch.cuda.synchronize()
                t = ev_a.elapsed_time(ev_b) / 10
                variants[name.lower()] = {"ms": round(t, 4), "gbs": round(m["residual64"] / (t / 1e3) / 1e9, 1)}

    peak, peak_kind = peaks()
    ach = m["apply32"] / ((ms_patch + ms_fix) / 1e3) / 1e9
    ach_cg = m["cg_mixed"] / ((ms_cg[0] + ms_cg[1]) / 1e3) / 1e9
    ach64 = m["residual64"] / ((ms_patch64 + ms_fix64) / 1e3) / 1e9
    ach_dw = m["residual64"] / (sum(ms_dw) / 1e3) / 1e9
    alu64 = fp64_alu_model(dim + 1, n_n, n_e, torch.cuda.get_device_properties(dev).multi_processor_count,
                           clk.get("sm_mhz") or clk.get("sm_max_mhz"))
    if alu64 is not None:
        alu64["achieved_gops"] = round(alu64["ops_per_launch"] / ((ms_patch64 + ms_fix64) / 1e3) / 1e9, 1)
        alu64["frac"] = round(alu64["achieved_gops"] / alu64["peak_gops"], 4)
    trf = traffic_record("cg_pass")

    # e2e: the user's whole call sequence from pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        hc, he, hf = pin(prob["coords"]), pin(prob["elems"]), pin(prob["f"])
        hd, hg, hn = pin(prob["dirichlet"]), pin(prob["g"]), pin(prob["neumann"])
        hx = pin(np.zeros(n_n))
        h2d = hc.nbytes + he.nbytes + hf.nbytes + hd.nbytes + hg.nbytes + hn.nbytes + hx.nbytes
        d2h = hx.nbytes
        times, ebytes = [], 0
        parts = {"create": 0.0, "set_problem": 0.0, "assemble": 0.0, "solve_host": 0.0, "destroy": 0.0}
        for _ in range(args.e2e_steps):
            hx[:] = 0.0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h2 = ebe.ebe_create(hc, he, device=dev.index)
            t1 = time.perf_counter()
            ebe.ebe_set_problem(h2, prob["nu"], hf, hd, hg, hn)
            t2 = time.perf_counter()
            ebe.ebe_assemble(h2, ebe.EBE_STORE_MIXED)
            t3 = time.perf_counter()
            info = ebe.ebe_solve_host(h2, hx, rtol=args.rtol, precision=ebe.EBE_PREC_MIXED)
            t4 = time.perf_counter()
            ebe.ebe_destroy(h2)
            torch.cuda.synchronize()
            t5 = time.perf_counter()
            times.append(t5 - t0)
            for k, a, b in (("create", t0, t1), ("set_problem", t1, t2), ("assemble", t2, t3), ("solve_host", t3, t4),
                            ("destroy", t4, t5)):
                parts[k] += (b - a) * 1e3 / args.e2e_steps
            ebytes += step_bytes(m, info, True)
        e2e_s, ebytes = reduce_over_ranks(dist, dev, sum(times), float(ebytes))
        e2e = {"value": round(ebytes / e2e_s / 1e9, 2), "unit": "GB/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": round(1e3 * e2e_s / args.e2e_steps, 2),
               "includes": "ebe_create (host partition build) + ebe_set_problem + ebe_assemble + "
                           "ebe_solve_host + ebe_destroy",
               "ms_per_call": {k: round(v, 1) for k, v in parts.items()}}

    nu0 = None
    if rank == 0 and not args.no_nu0:
        nu0 = run_pcg_leg(args, dev, stream, meshgen.config_square_jitter(args.n, nu=0.0, seed=2))
        nu0 = {"workload": f"square{args.n}_jitter0.2_nu0_tri", **nu0}
    small = None
    if rank == 0 and not args.no_small:
        small = run_pcg_leg(args, dev, stream, meshgen.config_square_f1(33, nu=1.0), reps=5)
        small = {"workload": "square33_f1_nu1_dirichlet0 (2048 triangles)", **small}
    batched = None
    if not args.no_batch:
        batched = run_batch(args, dev, stream)
    learned_res = run_learned(args, dev, stream) if rank == 0 and not args.no_learned else None
    paper_exp = run_paper_experiment(dev, stream) if rank == 0 else None
    cube = run_cube(args, dev, stream) if rank == 0 and not args.no_cube else None

    cpu = cpu_par = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(prob, m, iters=40)
        cpu_par = oracle_parallel_sample(prob, m, iters=100)

    if rank != 0:
        return None
    info0 = infos[-1]
    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": workload_config(args, n_n, n_e, dim, world),
        "pcg": {"solver": "Jacobi-PCG, single-sync (two launches, one reduction per iteration), FP32 A_e/r/p/q, FP64 x, residual replacement by the double-word FP64 residual above 1e-6 |r0| and the FP64 one below, convergence confirmed in FP64",
                "ms_to_1e-8": round(ms_step, 2), "iterations": info0["iterations"],
                "true_residuals": info0["true_residuals"], "rel_residual": info0["rel_residual"],
                "plain_fp64_ms": round(ms_plain, 2) if ms_plain else None,
                "plain_fp64_iterations": pinfo[-1]["iterations"] if pinfo else None,
                "speedup_vs_plain": round(ms_plain / ms_step, 3) if ms_plain else None,
                "textbook_mixed_ms": round(ms_text, 2) if ms_text else None,
                "textbook_mixed_iterations": tinfo["iterations"] if tinfo else None},
        "roofline": {"bound": "hbm", "achieved": round(ach_cg, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(ach_cg / peak, 4), "traffic": trf,
                     "frac_of_nominal_8000": round(ach_cg / 8000.0, 4),
                     "kernel": "one iteration of the mixed solver: single-sync pass (k_cg_patch + k_cg_fixup)",
                     "ms_per_launch": [round(ms_cg[0], 5), round(ms_cg[1], 5)],
                     "bytes_per_launch": m["cg_mixed"], "peak_kind": peak_kind,
                     "stored_bytes_per_launch": m_stored["cg_mixed"],
                     "stored_gbs": round(m_stored["cg_mixed"] / ((ms_cg[0] + ms_cg[1]) / 1e3) / 1e9, 1)},
        "apply_fp32": {"gbs": round(ach, 1), "frac": round(ach / peak, 4),
                       "kernel": "FP32 operator application: patch pass + halo fix-up",
                       "ms_per_launch": [round(ms_patch, 5), round(ms_fix, 5)], "bytes_per_launch": m["apply32"],
                       "traffic": traffic_record("apply32"),
                       "stored_gbs": round(m_stored["apply32"] / ((ms_patch + ms_fix) / 1e3) / 1e9, 1)},
        "residual_fp64": {"gbs": round(ach64, 1), "frac": round(ach64 / peak, 4),
                          "ms_per_launch": [round(ms_patch64, 5), round(ms_fix64, 5)],
                          "bytes_per_launch": m["residual64"],
                          "stored_gbs": round(m_stored["residual64"] / ((ms_patch64 + ms_fix64) / 1e3) / 1e9, 1),
                          "fp64_pipe": alu64},
        "residual_dw": {"gbs": round(ach_dw, 1), "frac": round(ach_dw / peak, 4),
                        "kernel": "the FP64 residual in double-word FP32 arithmetic (EBE_F64_DW): patch + fix-up",
                        "ms_per_launch": [round(ms_dw[0], 5), round(ms_dw[1], 5)],
                        "bytes_per_launch": m["residual64"], "traffic": traffic_record("residual_dw")},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "cpu_baseline": cpu,
        "cpu_all_cores": cpu_par,
    }
    if nu0:
        line["nu0"] = nu0
    if small:
        line["square33"] = small
    if batched:
        line["batched"] = batched
    if learned_res:
        line["learned"] = learned_res
    if variants:
        line["residual_variants_fp64"] = variants
    if cube:
        line["cube129"] = cube
    if paper_exp:
        line["paper_experiment"] = paper_exp
    line["summary"] = summary_block(line, ms_plain, pinfo, peak)
    print(json.dumps(line), flush=True)
    return line


def summary_block(line, ms_plain, pinfo, peak):
    """Every number of the metric in a few hundred characters, as the line's
    last key: PCG time to 1e-8, mixed against plain FP64, per workload, the
    operators' HBM fractions and the comparison scatters."""
    pc = line["pcg"]
    r = line["roofline"]
    s = {"sq2049_nu1": {"mixed_ms": pc["ms_to_1e-8"], "it": pc["iterations"],
                        "plain_ms": round(ms_plain, 1) if ms_plain else None,
                        "plain_it": pinfo[-1]["iterations"] if pinfo else None, "x": pc["speedup_vs_plain"],
                        "textbook_mixed_ms": pc["textbook_mixed_ms"]}}
    for key, name in (("nu0", "sq2049_nu0"), ("square33", "sq33"), ("cube129", "cube129")):
        v = line.get(key)
        if v:
            s[name] = {"mixed_ms": v["mixed"]["ms_to_1e-8"], "it": v["mixed"]["iterations"],
                       "plain_ms": v["plain_fp64"]["ms_to_1e-8"], "plain_it": v["plain_fp64"]["iterations"],
                       "x": v["speedup_vs_plain"]}
    if "sq33" in s:
        s["sq33"].update({"us_per_it": line["square33"]["mixed"]["us_per_iteration"],
                          "plain_us_per_it": line["square33"]["plain_fp64"]["us_per_iteration"]})
    b = line.get("batched")
    if b:
        s["batch256"] = {"mixed_ms": b["ms_to_1e-8"], "batched_fp64_ms": b["batched_fp64_ms"],
                         "seq_fp64_ms": b["sequential_fp64_ms"], "x_vs_seq_fp64": b["speedup_vs_sequential_fp64"],
                         "gbs": b["gbs"], "frac": round(b["gbs"] / peak, 3)}
    lr = line.get("learned")
    if lr:
        s["learned"] = {k: {"fcg_net_ms": v["learned_fcg"]["ms"], "net_it": v["learned_fcg"]["iterations"],
                            "fell_back": v["learned_fcg"]["fell_back"], "plain_pcg_ms": v["plain_fp64_pcg"]["ms"],
                            "ratio_to_plain": round(v["learned_fcg"]["ms"] / v["plain_fp64_pcg"]["ms"], 3),
                            "mixed_pcg_ms": v["mixed_pcg"]["ms"],
                            "ratio_to_mixed": round(v["learned_fcg"]["ms"] / v["mixed_pcg"]["ms"], 3),
                            "net_first_ms": v["network_first"]["ms"]}
                        for k, v in lr.items() if k.startswith("square")}
    s["hbm_frac"] = {"cg_pass": r["frac"], "apply32": line["apply_fp32"]["frac"],
                     "residual64": line["residual_fp64"]["frac"], "residual_dw": line["residual_dw"]["frac"]}
    c = line.get("cube129")
    if c:
        s["hbm_frac"].update({"cube_cg_pass": c["cg_pass"]["frac"], "cube_apply32": c["apply32"]["frac"],
                              "cube_residual64": c["residual64"]["frac"], "cube_residual_dw": c["residual_dw"]["frac"]})
    v = line.get("residual_variants_fp64")
    if v:
        s["scatter_fp64_ms"] = {k: x["ms"] for k, x in v.items()}
    return s


def oracle_sample(prob, m, iters=10):
    """The FP64 oracle, single-threaded, on a bounded sample of the workload:
    element matrices + local systems of the full mesh, then `iters` Jacobi-PCG
    iterations.  Returns the cpu_baseline object (GB/s by the same byte model,
    FP64 passes)."""
    import oracle
    t0 = time.perf_counter()
    orc = oracle.Problem(prob)
    x, info = orc.pcg(rtol=1e-30, maxit=iters)
    dt = time.perf_counter() - t0
    nbytes = m["assemble_fp64"] + info["iterations"] * (m["apply64"] + m["vec64"]) + info["residual_evals"] * m["residual64"]
    return {"value": round(nbytes / dt / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "seconds": round(dt, 2),
            "sample": f"element matrices of all {orc.n_e} elements + {info['iterations']} FP64 Jacobi-PCG "
                      f"iterations ({info['residual_evals']} Algorithm-1 residuals), single thread"}


def oracle_parallel_sample(prob, m, iters=100):
    """The oracle's all-core timing build (OpenMP, colour-parallel element
    loop; colouring done before the clock starts) on the same kind of sample
    as oracle_sample: element arrays of the full mesh and `iters` FP64
    Jacobi-PCG iterations.  None where the host compiler has no OpenMP."""
    import oracle
    import oracle.parallel as oracle_parallel
    try:
        par = oracle_parallel.ParallelTiming(prob)
    except oracle.OracleError as e:
        return {"unavailable": str(e)}
    t0 = time.perf_counter()
    A, be = par.element_arrays()
    _, info = par.pcg(A, be, rtol=1e-30, maxit=iters)
    dt = time.perf_counter() - t0
    nbytes = m["assemble_fp64"] + info["iterations"] * (m["apply64"] + m["vec64"]) + info["residual_evals"] * m["residual64"]
    return {"value": round(nbytes / dt / 1e9, 3), "unit": "GB/s", "cores": par.threads, "nproc": os.cpu_count(),
            "kind": "oracle all-core timing build", "seconds": round(dt, 2), "colours": par.n_col,
            "sample": f"element matrices of all {par.n_e} elements + {info['iterations']} FP64 Jacobi-PCG iterations, "
                      f"OpenMP on {par.threads} threads, colour-parallel element loop"}


def workload_config(args, n_n: int, n_e: int, dim: int, world: int) -> dict:
    """The workload both arms report (the same dict for the same arguments)."""
    return {"workload": f"square{args.n}_jitter0.2_nu{args.nu:g}_tri", "n_nodes": n_n, "n_elements": n_e,
            "n_b": dim + 1, "rtol": args.rtol, "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (A_e FP64 + FP32 = %.0f MB)" % ((n_e * (dim + 1) * (dim + 2) // 2 * 12) / 1e6),
            "value_def": "algorithmic bytes of the step / step time"}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    from paper_1911_03973_gb300 import meshgen
    oracle.build()
    prob = meshgen.config_square_jitter(args.n, nu=args.nu, seed=2)
    n_n, dim = prob["coords"].shape
    m = bytes_model(dim, n_n, prob["elems"].shape[0])
    for _ in range(args.warmup):
        oracle_sample(prob, m, iters=2)
    samples = [oracle_sample(prob, m, iters=10) for _ in range(args.steps)]
    secs = sum(s["seconds"] for s in samples)
    val = sum(s["value"] * s["seconds"] for s in samples) / secs
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * secs / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, n_n, int(prob["elems"].shape[0]), dim, world),
            "cpu_baseline": {"value": round(val, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": samples[0]["sample"]},
            "e2e": {"value": round(val, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return line


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
