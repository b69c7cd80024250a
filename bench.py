"""Benchmark of the fused SLLBM step (GVUPS = vertex x velocity x population updates per second).

Default workload: the 1024x1024-vertex Taylor-Green vortex at order p = 4 (256x256 cells, D2Q25,
f and g populations), FP32 deviation storage, one fused kernel launch per step.  The state
(2 x 210 MB) is larger than the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload tgv256|riemann|sod|svi|tgv16] [--prec f32|bf16|f64]

Under torchrun every rank runs an independent replica on its own GPU (the method needs no
exchange between replicas); rank 0 prints one JSON line with the max-over-ranks time.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GVUPS (vertex x velocity x population updates/s), fused FP32 SLLBM step"
UNIT = "GVUPS"

# DRAM traffic (read + write bytes per launch) of the step kernel from an ncu capture, keyed by
# (kernel source digest, workload, precision); reported as null once the kernel source changes.
NCU_TRAFFIC = {
    # profiles/step_uniform_tgv256_p4_f32.md: 222.7 MB read + 173.6 MB written
    ("2bc27c161d73873e", "tgv256_p4", "f32"): 396.2e6,
    # profiles/step_mapped_svi512x256_p2_f32.md: 273.8 MB read + 78.4 MB written
    ("2bc27c161d73873e", "svi512x256_p2_mapped", "f32"): 352.2e6,
}


# Sources that decide what the two fused kernels of NCU_TRAFFIC do and how they are launched on
# which layout (kernels, shared device code, launch set-up, tables): a change to any of them
# voids the stored traffic.
MEASURED_SOURCES = ("api.cu", "kernels.h", "precompute.cu", "sllbm_internal.cuh", "step_gather.cu",
                    "step_mapped.cu", "step_uniform.cu", "tma.cuh")


def _kernel_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1910_13918_gb300", "csrc")
    for f in MEASURED_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def bytes_per_update(w, prec, kernel):
    """Algorithmic HBM bytes per update: the stored state read once and written once.  D2Q25
    FP32/BF16 storage keeps (f, g) pairs (the g slot zero with one population); FP64 and D2Q9
    keep the populations they have.  The fused mapped kernel also reads the 12-byte departure
    record of each (velocity, vertex), shared by the populations."""
    stored = (w.n_velocities * w.n_populations
              if prec == "f64" or w.velset == "d2q9" else 2 * w.n_velocities)
    elem = {"f32": 4, "bf16": 2, "f64": 8}[prec]
    b = 2 * stored * elem / (w.n_velocities * w.n_populations)
    if kernel == "mapped_fused":
        b += 12 / w.n_populations
    return b


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) < 9:
                continue
            for k, n in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float) -> float:
    """Max of a per-rank float over the default process group (identity without one).  The
    tensor lives on the GPU under NCCL and on the CPU under gloo."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _workload(name):
    from paper_1910_13918_gb300 import workloads as W
    return W.ALL[name]()


def _workload_desc(w):
    pops = "f and g populations" if w.n_populations == 2 else "f only (isothermal)"
    return (f"{w.name}: {w.nx}x{w.ny} vertices ({w.nx_cells}x{w.ny_cells} cells, p={w.order}), "
            f"{w.velset.upper()}, {pops}, dt={w.dt:.6g}, tau={w.tau:.6g}")


# -------------------------------------------------------------------------------------------------
# CPU oracle baseline (bounded sample of the same workload)
# -------------------------------------------------------------------------------------------------
class OracleSample:
    """The FP64 oracle on a bounded sample of a workload: one step for the first `rows` vertex
    rows.  Set-up (grid, the initial state where the sample's stencils reach) is done once; each
    timed step recomputes the departures, streams and collides, as the oracle's step does."""

    def __init__(self, w, rows=16):
        import numpy as np
        from oracle import sllbm as o
        self.o, self.w = o, w
        ax = o.Axis(w.nx_cells, w.order, w.x0, w.x1, w.bc_x == 0, w.nodes)
        ay = o.Axis(w.ny_cells, w.order, w.y0, w.y1, w.bc_y == 0, w.nodes)
        self.grid = grid = o.Grid(ax, ay, o.SineMap(w.map_a) if w.map_a else None)
        X, Y = grid.coords()
        self.verts = np.arange(min(rows, grid.ny) * grid.nx)
        self.q = q = w.n_velocities
        dep0 = o.Departures(grid, w.dt, self.verts, q=q)
        keys = []
        for i in range(q):
            for b in range(grid.p + 1):
                for a in range(grid.p + 1):
                    keys.append(ay.vertex_of(dep0.cy[i], b) * grid.nx + ax.vertex_of(dep0.cx[i], a))
        keys = np.unique(np.concatenate(keys))
        fields = [np.asarray(F).reshape(-1)[keys] for F in w.fields(X, Y)]
        f0, g0 = o.initial_state(*fields, w.cv, q)
        self.F = np.zeros((q, grid.ny * grid.nx))
        self.G = np.zeros((q, grid.ny * grid.nx))
        self.F[:, keys] = f0
        self.G[:, keys] = g0
        self.F = self.F.reshape(q, grid.ny, grid.nx)
        self.G = self.G.reshape(q, grid.ny, grid.nx)

    @property
    def n_vertices(self):
        return len(self.verts)

    def step_time(self):
        o, w = self.o, self.w
        t = time.perf_counter()
        dep = o.Departures(self.grid, w.dt, self.verts, q=self.q)
        fpre = o.stream(self.F, dep)
        gpre = o.stream(self.G, dep)
        o.collide(fpre, gpre, w.tau, w.cv, w.pr, w.isothermal)
        return time.perf_counter() - t


def cpu_baseline(w, rows=16, repeats=3):
    sample = OracleSample(w, rows)
    el = min(sample.step_time() for _ in range(repeats))
    nv = sample.n_vertices
    return {"value": nv * w.n_velocities * w.n_populations / el / 1e9, "unit": UNIT, "cores": 1,
            "kind": "oracle",
            "sample": f"one oracle step on the first {rows} vertex rows ({nv} vertices) of "
                      f"{w.name}, best of {repeats}: {el:.2f} s, numpy float64, one thread"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    w = _workload(args.workload)
    sample = OracleSample(w, rows=16)
    for _ in range(args.warmup):
        sample.step_time()
    times = [sample.step_time() for _ in range(args.steps)]
    nv = sample.n_vertices
    tot = sum(times)
    value = nv * w.n_velocities * w.n_populations * len(times) / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": _workload_desc(w), "sample_vertices": nv},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: one oracle step on the first 16 vertex rows "
                                       f"({nv} vertices) of {w.name}, numpy float64, one thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# -------------------------------------------------------------------------------------------------
# GPU arm
# -------------------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_1910_13918_gb300.sllbm import SLLBM
    w = _workload(args.workload)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = SLLBM.from_workload(w, prec=args.prec, stream=stream)
        s.precompute()
        x, y = (t.cpu().numpy() for t in s.coords())
        fields = w.fields(x, y)
        s.init(*fields)
        s.step(args.warmup)
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        m = s.moments()
    ms_max = max_over_ranks(ms)
    ms_step = ms_max / args.steps
    updates = w.updates_per_step

    # adjoint step (Pr = 1, thermal collision): lambda' -> S^T J_C^T lambda' on the library's
    # stream, at the moments of the state the forward run ended in; not part of `value`
    adjoint = None
    if not args.no_adjoint and not w.isothermal and w.pr == 1.0:
        with torch.cuda.stream(stream):
            mom = torch.stack([m["rho"], m["u"], m["v"], m["T"]]).contiguous()
            gen = torch.Generator(device="cuda").manual_seed(7)
            lam = torch.randn((2, 25, s.ny, s.nx), device="cuda", generator=gen)
            out = torch.empty_like(lam)
            for _ in range(3):
                s.adjoint_step(lam, out, mom)
            ka = 20
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(ka):
                s.adjoint_step(lam, out, mom)
                lam, out = out, lam
            a1.record(stream)
            torch.cuda.synchronize()
        ms_adj = max_over_ranks(a0.elapsed_time(a1)) / ka
        adjoint = {"ms_per_step": ms_adj, "value": updates * ws / (ms_adj * 1e-3) / 1e9, "unit": UNIT,
                   "steps": ka, "launches_per_step": 2 if w.map_a else 3,
                   "note": "sllbm_adjoint_step: pointwise J_C^T, then S^T as a pull over transposed stencils"}
    value = updates * args.steps * ws / (ms_max * 1e-3) / 1e9

    # end to end through the host-buffer entry point: copy state in, one step, copy state out
    e2e = None
    if not args.no_e2e:
        nb = s.state_bytes
        hin = torch.empty(nb, dtype=torch.uint8).pin_memory()
        hout = torch.empty(nb, dtype=torch.uint8).pin_memory()
        st = s.get_state()
        hin.copy_(st.view(torch.uint8).reshape(-1).cpu())
        a_in, a_out = hin.numpy(), hout.numpy()
        s.step_host(a_in, a_out, 1)
        k = max(3, min(args.steps, 20))
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(k):
            s.step_host(a_in, a_out, 1)
        el = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": updates * k * ws / el / 1e9, "unit": UNIT, "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb,
               "api": "sllbm_step_host (pinned host state in, 1 step, state out)"}

    if rank == 0:
        peaks, src = _peaks()
        alg_bytes = updates * bytes_per_update(w, args.prec, s.kernel_name)
        achieved = alg_bytes / (ms_step * 1e-3) / 1e9
        peak = float(peaks.get("hbm_gbs", 6800.0))
        traffic = NCU_TRAFFIC.get((_kernel_digest(), w.name, args.prec))
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"f32": "f32", "bf16": "f32 (bf16 storage)", "f64": "f64"}[args.prec],
            "data": "synthetic",
            "config": {"workload": _workload_desc(w), "kernel": s.kernel_name,
                       "n_vertices": w.n_vertices, "updates_per_step": updates,
                       "l2": "state 2 x %.0f MB > 129 MB L2, no flush" % (s.state_bytes / 1e6),
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"hbm_gbs of {src} peaks",
                         "algorithmic_bytes_per_launch": alg_bytes},
            "clocks": clocks,
            "e2e": e2e,
            "f_only_value": value / w.n_populations,   # the same time counted in f updates only
            "adjoint": adjoint,
            "gpu_launches": args.steps * s.launches_per_step,
            "mass_after": m["mass"],
        }
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tgv256")
    ap.add_argument("--prec", default="f32", choices=["f32", "bf16", "f64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
