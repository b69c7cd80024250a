"""Benchmark of the fused SLLBM step (GVUPS = vertex x velocity x population updates per second).

Headline workload: the 2D Riemann problem on 1024x1024 cells of order p = 3 (3073 x 3073 =
9,443,329 vertices, zero-gradient boundaries, D2Q25, f and g populations) with the quadrant
states of the paper's Table III, FP32 deviation storage, one fused kernel launch per step plus
the fix-up launch for the vertices next to the boundaries.  The state (2 x 1.89 GB) is far
larger than the 129 MB L2, so no flush is needed between steps.  Beside it the same line
carries the BF16-storage and plain FP64 forms of the step on the same grid, each with its error
against the FP64 oracle after one step (sampled vertices) and against the FP64 GPU step after
the whole run, the 1024x1024-vertex Taylor-Green vortex at p = 4 as a second grid, and the 3D
extension (D3Q125, the fused FP32 and the plain FP64 step) on the 128^3-vertex 3D Taylor-Green
vortex.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--repeats R] [--impl ours|reference]
                    [--workload riemann_paper|tgv256|riemann|sod|svi|tgv16] [--quick]

Each timed region is K steps between CUDA events on the library's stream (barrier and
synchronize on both sides); it is repeated R times (default 5) and the median is reported with
all R values.  Under torchrun every rank runs an independent replica on its own GPU (the method
needs no exchange between replicas); rank 0 prints one JSON line with the max-over-ranks times.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GVUPS (vertex x velocity x population updates/s), fused FP32 SLLBM step"
UNIT = "GVUPS"
SECONDARY = "tgv256"          # second grid of the line: the Taylor-Green vortex, p = 4

# DRAM traffic (read + write bytes per launch) of the step kernel from an ncu capture, keyed by
# (kernel source digest, workload, precision); reported as null once the kernel source changes.
NCU_TRAFFIC = {
    # 512^2-cell capture: 511.6 MB read + 429.2 MB written for 2,362,369 vertices, scaled by the
    # vertex count to the 3073^2 grid (a multi-pass capture of that grid exceeds the size rule)
    ("99a5f9bcc84ce154", "riemann1024_p3_tableIII", "f32"): 940.84e6 * 9443329 / 2362369,
    ("99a5f9bcc84ce154", "riemann512_p3_tableIII", "f32"): 940.84e6,
    # full-size capture: 219.5 MB read + 174.1 MB written
    ("99a5f9bcc84ce154", "tgv256_p4", "f32"): 393.62e6,
}

# Sources that decide what the fused kernels of NCU_TRAFFIC do and how they are launched on
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


def _barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def _workload(name):
    from paper_1910_13918_gb300 import workloads as W
    return W.ALL[name]()


def _workload_desc(w):
    pops = "f and g populations" if w.n_populations == 2 else "f only (isothermal)"
    states = " (Table III states)" if "states" in w.extra else ""
    return (f"{w.name}: {w.nx}x{w.ny} vertices ({w.nx_cells}x{w.ny_cells} cells, p={w.order}), "
            f"{w.velset.upper()}, {pops}{states}, dt={w.dt:.6g}, tau={w.tau:.6g}")


def sample_vertices(w, count=48, seed=2019):
    """Flat indices of the vertices whose one-step values are compared with the oracle: the four
    corners, the middle of each edge, vertices on and beside the lines where the initial fields
    jump (Riemann quadrants, Sod, shock), and seeded random vertices."""
    import numpy as np
    nx, ny = w.nx, w.ny
    pts = {(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1), (nx // 2, 0), (0, ny // 2),
           (nx - 1, ny // 2), (nx // 2, ny - 1)}
    split = w.extra.get("split", w.extra.get("x_shock", 0.5 if w.kind == "sod" else None))
    if split is not None:
        jx = int(round((split - w.x0) / (w.x1 - w.x0) * (nx - (0 if w.bc_x == 0 else 1))))
        jy = int(round((split - w.y0) / (w.y1 - w.y0) * (ny - (0 if w.bc_y == 0 else 1))))
        for dx in (-1, 0, 1):
            pts.add((min(max(jx + dx, 0), nx - 1), ny // 3))
            pts.add((nx // 3, min(max(jy + dx, 0), ny - 1)))
            pts.add((min(max(jx + dx, 0), nx - 1), min(max(jy + dx, 0), ny - 1)))
    rng = np.random.default_rng(seed)
    while len(pts) < count:
        pts.add((int(rng.integers(nx)), int(rng.integers(ny))))
    return np.array(sorted(y * nx + x for x, y in pts), dtype=np.int64)


def field_errors(gpu, ref, velocity_scale):
    """Max error per field (the tests' metric): rho and T pointwise relative; u and v relative to
    the larger of max |u_ref| and the workload's characteristic speed."""
    import numpy as np
    rho_g, u_g, v_g, t_g = (np.asarray(a, dtype=np.float64) for a in gpu)
    rho_r, u_r, v_r, t_r = (np.asarray(a, dtype=np.float64) for a in ref)
    umax = max(float(np.max(np.abs(u_r))), float(np.max(np.abs(v_r))), velocity_scale, 1e-12)
    return {"rho": float(np.max(np.abs(rho_g - rho_r) / np.abs(rho_r))),
            "u": float(np.max(np.abs(u_g - u_r)) / umax),
            "v": float(np.max(np.abs(v_g - v_r)) / umax),
            "T": float(np.max(np.abs(t_g - t_r) / np.abs(t_r)))}


# -------------------------------------------------------------------------------------------------
# CPU leg: the FP64 oracle on bounded samples of the same workload (timing, and the reference
# values of the sampled vertices after one step)
# -------------------------------------------------------------------------------------------------
class _Sparse:
    """Population field known on a sorted set of vertices, indexable like F[i, jy, jx]."""

    def __init__(self, nx, keys, values):
        self.nx, self.keys, self.values = nx, keys, values

    def __getitem__(self, idx):
        import numpy as np
        i, jy, jx = idx
        pos = np.searchsorted(self.keys, np.asarray(jy) * self.nx + np.asarray(jx))
        return self.values[i][pos]

    @property
    def dtype(self):
        return self.values.dtype

    @property
    def shape(self):
        return self.values.shape[:1]


class OracleSample:
    """The FP64 oracle on a bounded sample of a workload: one step at the vertices ``verts``.

    Set-up (grid, departure points -- built once, as the oracle's ``run`` does -- and the initial
    state where the sample's stencils reach) is untimed; a timed step is the oracle's stream of
    f and g plus its collision, on the sample."""

    def __init__(self, w, verts):
        import numpy as np
        from oracle import sllbm as o
        self.o, self.w = o, w
        ax = o.Axis(w.nx_cells, w.order, w.x0, w.x1, w.bc_x == 0, w.nodes)
        ay = o.Axis(w.ny_cells, w.order, w.y0, w.y1, w.bc_y == 0, w.nodes)
        grid = o.Grid(ax, ay, o.SineMap(w.map_a) if w.map_a else None)
        self.verts = np.asarray(verts)
        self.q = q = w.n_velocities
        self.dep = dep = o.Departures(grid, w.dt, self.verts, q=q)
        keys = []
        for i in range(q):
            for b in range(grid.p + 1):
                for a in range(grid.p + 1):
                    keys.append(ay.vertex_of(dep.cy[i], b) * grid.nx + ax.vertex_of(dep.cx[i], a))
        keys = np.unique(np.concatenate(keys))
        X, Y = grid.coords()
        fields = w.fields(X.reshape(-1)[keys], Y.reshape(-1)[keys])   # pointwise generators
        f0, g0 = o.initial_state(*fields, w.cv, q)
        self.F = _Sparse(grid.nx, keys, f0)
        self.G = _Sparse(grid.nx, keys, g0)

    @property
    def n_vertices(self):
        return len(self.verts)

    def step(self):
        o, w = self.o, self.w
        fpre = o.stream(self.F, self.dep)
        gpre = o.stream(self.G, self.dep)
        return o.collide(fpre, gpre, w.tau, w.cv, w.pr, w.isothermal)

    def step_time(self):
        t = time.perf_counter()
        self.step()
        return time.perf_counter() - t

    def macroscopic_after_step(self):
        f1, g1 = self.step()
        rho, u, th = self.o.macroscopic(f1, g1, self.w.cv)
        return rho, u[..., 0], u[..., 1], th


def _row_block(w, rows, row0=0):
    import numpy as np
    r0 = min(row0, w.ny - 1)
    r1 = min(r0 + rows, w.ny)
    return np.arange(r0 * w.nx, r1 * w.nx)


def _cpu_worker(w, rows, row0, barrier, queue):
    """One process of the all-core oracle timing: its own block of vertex rows, one step."""
    sample = OracleSample(w, _row_block(w, rows, row0))
    barrier.wait(timeout=600)
    t0 = time.perf_counter()
    sample.step()
    t1 = time.perf_counter()
    queue.put((sample.n_vertices, t0, t1))


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(w, rows=24, rows_per_core=16, repeats=3):
    """The oracle as it stands, timed on this host: one thread on the first ``rows`` vertex rows
    (best of ``repeats``), and one process per core on consecutive blocks of ``rows_per_core``
    rows each, all stepping at once (spawned processes: the parent already holds a CUDA
    context)."""
    import multiprocessing as mp
    sample = OracleSample(w, _row_block(w, rows))
    el = min(sample.step_time() for _ in range(repeats))
    nv = sample.n_vertices
    upd = w.n_velocities * w.n_populations
    out = {"value": nv * upd / el / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
           "cpu_model": _cpu_model(), "host_cores": os.cpu_count(),
           "sample": f"one oracle step (stream f, g + collide) on the first {rows} vertex rows "
                     f"({nv} vertices) of {w.name}, best of {repeats}: {el:.2f} s, numpy float64, "
                     f"one thread"}
    ncores = os.cpu_count() or 1
    rows = rows_per_core
    nproc = min(ncores, max(1, w.ny // rows))
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"           # one thread per process (the children inherit it)
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(nproc), ctx.Queue()
    procs = [ctx.Process(target=_cpu_worker, args=(w, rows, k * rows, barrier, queue))
             for k in range(nproc)]
    for p in procs:
        p.start()
    res, t_end = [], time.time() + 900
    while len(res) < nproc and time.time() < t_end:
        try:
            res.append(queue.get(timeout=1.0))
        except Exception:                   # queue.Empty: see whether a worker died
            if any(p.exitcode not in (None, 0) for p in procs):
                break
    for p in procs:
        p.join(timeout=5)
        if p.is_alive():
            p.terminate()
    if len(res) < nproc:
        out["all_cores"] = {"value": None, "unit": UNIT, "cores": nproc,
                            "unavailable": "a worker process failed or timed out"}
        return out
    nv_all = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    out["all_cores"] = {
        "value": nv_all * upd / wall / 1e9, "unit": UNIT, "cores": nproc,
        "sample": f"{nproc} processes, each one oracle step on its own block of {rows} vertex rows "
                  f"({nv_all} vertices in all), started together: {wall:.2f} s wall"}
    return out


def oracle_reference_at(w, verts):
    """Oracle (rho, u, v, theta) after one step from the unperturbed initial state at ``verts``."""
    return OracleSample(w, verts).macroscopic_after_step()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    w = _workload(args.workload)
    rows = 4
    sample = OracleSample(w, _row_block(w, rows))
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
                             "cpu_model": _cpu_model(),
                             "sample": f"each step: one oracle step (stream f, g + collide) on the "
                                       f"first {rows} vertex rows ({nv} vertices) of {w.name}, "
                                       f"numpy float64, one thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# -------------------------------------------------------------------------------------------------
# GPU arm
# -------------------------------------------------------------------------------------------------
def _event_pair():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def measure(w, prec, args, stream, verts, sampler=None, keep=False):
    """One precision form of the step on workload ``w``: the moments after one step at ``verts``
    (for the oracle comparison), then W warm-up steps and R timed regions of K steps each.
    Returns the per-repeat max-over-ranks times, the final moments and, if ``keep``, the context."""
    import torch
    from paper_1910_13918_gb300.sllbm import SLLBM
    with torch.cuda.stream(stream):
        s = SLLBM.from_workload(w, prec=prec, stream=stream)
        p0, p1 = _event_pair()
        torch.cuda.synchronize()
        p0.record(stream)
        s.precompute()   # departure tables / descriptors and vertex weights, FP64
        p1.record(stream)
        torch.cuda.synchronize()
        precompute_ms = p0.elapsed_time(p1)
        x, y = (t.cpu().numpy() for t in s.coords())
        s.init(*w.fields(x, y))
        del x, y
        s.step(1)
        m1 = s.moments(sums=False)
        idx = torch.as_tensor(verts, device=s.device)
        one_step = [m1[k].reshape(-1)[idx].double().cpu().numpy() for k in ("rho", "u", "v", "T")]
        del m1
        s.step(args.warmup)
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
            time.sleep(0.3)
        ms = []
        for _ in range(args.repeats):
            e0, e1 = _event_pair()
            _barrier()
            torch.cuda.synchronize()
            e0.record(stream)
            s.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            _barrier()
            ms.append(max_over_ranks(e0.elapsed_time(e1)))
        clocks = sampler.stop() if sampler else None
        with_moments = None
        if keep and w.velset != "d2q9":   # the same steps with the moments epilogue (D2Q25; 16 B a vertex)
            buf = torch.empty((4, s.ny, s.nx), dtype=torch.float32, device=s.device)
            e0, e1 = _event_pair()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                s.step_moments(buf)
            e1.record(stream)
            torch.cuda.synchronize()
            with_moments = max_over_ranks(e0.elapsed_time(e1)) / args.steps
            del buf
        mom = s.moments()
        final = torch.stack([mom["rho"], mom["u"], mom["v"], mom["T"]])
        info = {"kernel": s.kernel_name, "launches_per_step": s.launches_per_step,
                "state_bytes": s.state_bytes, "mass_after": mom["mass"], "nx": s.nx, "ny": s.ny,
                "precompute_ms": precompute_ms, "ms_per_step_with_moments": with_moments}
    if not keep:
        s.close()
        s = None
    return {"ms": ms, "one_step": one_step, "final": final, "info": info, "clocks": clocks, "ctx": s}


def _gpu_field_errors(final, ref, velocity_scale):
    """Max per-field error of a whole final field against the FP64 GPU step's (same metric)."""
    d = (final.double() - ref.double()).abs()
    umax = max(float(ref[1].abs().max()), float(ref[2].abs().max()), velocity_scale, 1e-12)
    return {"rho": float((d[0] / ref[0].double().abs()).max()), "u": float(d[1].max()) / umax,
            "v": float(d[2].max()) / umax, "T": float((d[3] / ref[3].double().abs()).max())}


def _summary(w, prec, r, args, ws, peak):
    ms_med = statistics.median(r["ms"])
    ms_step = ms_med / args.steps
    upd = w.updates_per_step
    alg = upd * bytes_per_update(w, prec, r["info"]["kernel"])
    achieved = alg / (ms_step * 1e-3) / 1e9
    out = {"ms_per_step": ms_step, "value": upd * ws / (ms_step * 1e-3) / 1e9, "unit": UNIT,
           "kernel": r["info"]["kernel"], "launches_per_step": r["info"]["launches_per_step"],
           "ms_per_region_repeats": r["ms"], "precompute_ms": r["info"]["precompute_ms"],
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak,
                        "bytes_per_update": bytes_per_update(w, prec, r["info"]["kernel"])}}
    wm = r["info"]["ms_per_step_with_moments"]
    if wm:
        out["with_moments_epilogue"] = {"ms_per_step": wm, "value": upd * ws / (wm * 1e-3) / 1e9,
                                        "unit": UNIT, "steps": args.steps,
                                        "note": "sllbm_step_moments: the step plus (rho, u, v, theta) "
                                                "of every vertex, 16 B a vertex more"}
    return out


def measure_grid(w, args, stream, ws, peak, sampler=None, precs=("f64", "f32", "bf16"), keep="f32"):
    """FP64 plain, FP32 and BF16-storage forms on one grid: timings, the sampled one-step values
    and, for FP32 and BF16, the whole-field error against the FP64 GPU step after the same run."""
    import torch
    verts = sample_vertices(w)
    res, out = {}, {}
    for prec in precs:
        res[prec] = measure(w, prec, args, stream, verts,
                            sampler=sampler if prec == keep else None, keep=(prec == keep))
        out[prec] = _summary(w, prec, res[prec], args, ws, peak)
        torch.cuda.empty_cache()
    nsteps = 1 + args.warmup + args.repeats * args.steps
    if "f64" in res:
        for prec in precs:
            if prec != "f64":
                out[prec]["err_vs_f64_gpu"] = {
                    "steps": nsteps,
                    "max_rel": _gpu_field_errors(res[prec]["final"], res["f64"]["final"],
                                                 w.velocity_scale)}
        if "f32" in out:
            out["speedup_f32_over_f64"] = out["f64"]["ms_per_step"] / out["f32"]["ms_per_step"]
        if "bf16" in out:
            out["speedup_bf16_over_f64"] = out["f64"]["ms_per_step"] / out["bf16"]["ms_per_step"]
    return verts, res, out


def measure_3d(args, stream, ws, peak, precs=("f64", "f32")):
    """The 3D extension (D3Q125, hexahedral cells) on the 3D Taylor-Green vortex: the plain FP64
    step and the sum-factorised FP32 step, W warm-up steps and R timed regions of K steps each,
    and the FP32 fields against the FP64 ones after the same run."""
    import numpy as np
    import torch
    from paper_1910_13918_gb300 import workloads as W
    from paper_1910_13918_gb300.sllbm import SLLBM3D, BC_PERIODIC
    w = W.tgv3d(cells=args.d3_cells)
    out, finals = {"workload": f"{w.name}: {w.shape[2]}^3 vertices ({w.cells[0]}^3 cells, p={w.order}), "
                               f"D3Q125, f and g, dt={w.dt:.6g}, tau={w.tau:.6g}",
                   "n_vertices": w.n_vertices, "updates_per_step": w.updates_per_step}, {}
    for prec in precs:
        with torch.cuda.stream(stream):
            s = SLLBM3D(cells=w.cells, order=w.order, box=w.box, bc=(BC_PERIODIC,) * 3, dt=w.dt,
                        tau=w.tau, cv=w.cv, prec=prec, stream=stream)
            s.precompute()
            kernel = s.kernel_name
            X, Y, Z = (t.cpu().numpy() for t in s.coords())
            s.init(*w.fields(X, Y, Z))
            del X, Y, Z
            s.step(args.warmup)
            ms = []
            for _ in range(args.repeats):
                e0, e1 = _event_pair()
                _barrier()
                torch.cuda.synchronize()
                e0.record(stream)
                s.step(args.steps)
                e1.record(stream)
                torch.cuda.synchronize()
                _barrier()
                ms.append(max_over_ranks(e0.elapsed_time(e1)))
            m = s.moments()
            finals[prec] = torch.stack([m[k] for k in ("rho", "u", "v", "w", "T")])
            s.close()
            torch.cuda.empty_cache()
        ms_step = statistics.median(ms) / args.steps
        bpu = 16.0 if prec == "f64" else 8.0
        achieved = w.updates_per_step * bpu / (ms_step * 1e-3) / 1e9
        out[prec] = {"ms_per_step": ms_step, "value": w.updates_per_step * ws / (ms_step * 1e-3) / 1e9,
                     "unit": UNIT, "kernel": kernel, "ms_per_region_repeats": ms,
                     "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                  "frac": achieved / peak, "bytes_per_update": bpu}}
    if "f64" not in finals:
        return out
    a, b = finals["f32"].double(), finals["f64"].double()
    umax = max(float(b[1].abs().max()), float(b[2].abs().max()), float(b[3].abs().max()), 1e-12)
    d = (a - b).abs()
    out["f32"]["err_vs_f64_gpu"] = {
        "steps": args.warmup + args.repeats * args.steps,
        "max_rel": {"rho": float((d[0] / b[0].abs()).max()), "u": float(d[1].max()) / umax,
                    "v": float(d[2].max()) / umax, "w": float(d[3].max()) / umax,
                    "T": float((d[4] / b[4].abs()).max())}}
    out["speedup_f32_over_f64"] = out["f64"]["ms_per_step"] / out["f32"]["ms_per_step"]
    return out


def adjoint_time(s, stream, ws, updates):
    """20 adjoint steps (S^T J_C^T) at the moments of the context's current state."""
    import torch
    with torch.cuda.stream(stream):
        m = s.moments(sums=False)
        mom = torch.stack([m["rho"], m["u"], m["v"], m["T"]]).contiguous()
        del m
        gen = torch.Generator(device="cuda").manual_seed(7)
        lam = torch.randn((2, 25, s.ny, s.nx), device="cuda", generator=gen)
        out = torch.empty_like(lam)
        for _ in range(3):
            s.adjoint_step(lam, out, mom)
        ka = 20
        a0, a1 = _event_pair()
        torch.cuda.synchronize()
        a0.record(stream)
        for _ in range(ka):
            s.adjoint_step(lam, out, mom)
            lam, out = out, lam
        a1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(a0.elapsed_time(a1)) / ka
    return {"ms_per_step": ms, "value": updates * ws / (ms * 1e-3) / 1e9, "unit": UNIT, "steps": ka,
            "note": "sllbm_adjoint_step: pointwise J_C^T into ghost-padded pairs, then S^T as a pull "
                    "over transposed stencils (TMA-staged on uniform grids)"}


def e2e_time(s, args, ws, updates):
    """End to end through the host-buffer entry point: state in from pinned host memory, one
    step, state out, every call."""
    import torch
    nb = s.state_bytes
    hin = torch.empty(nb, dtype=torch.uint8).pin_memory()
    hout = torch.empty(nb, dtype=torch.uint8).pin_memory()
    hin.copy_(s.get_state().view(torch.uint8).reshape(-1).cpu())
    a_in, a_out = hin.numpy(), hout.numpy()
    s.step_host(a_in, a_out, 1)
    k = max(3, min(args.steps, 20))
    groups = []
    for _ in range(3):   # median of three timed groups of k calls
        _barrier()
        t0 = time.perf_counter()
        for _ in range(k):
            s.step_host(a_in, a_out, 1)
        groups.append(max_over_ranks(time.perf_counter() - t0))
    el = statistics.median(groups)
    return {"value": updates * k * ws / el / 1e9, "unit": UNIT, "h2d_bytes_per_step": nb,
            "d2h_bytes_per_step": nb, "steps": k, "groups": 3,
            "ms_per_step_groups": [g / k * 1e3 for g in groups],
            "api": "sllbm_step_host (pinned host state in, 1 step, state out)"}


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if args.only_3d:   # the 3D entry alone (FP32 step only with --quick)
        peaks, _ = _peaks()
        out = measure_3d(args, torch.cuda.Stream(), ws, float(peaks.get("hbm_gbs", 6800.0)),
                         ("f32",) if args.quick else ("f64", "f32"))
        if rank == 0:
            print(json.dumps({"d3q125": out}))
        return 0
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    peaks, src = _peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    w = _workload(args.workload)
    stream = torch.cuda.Stream()
    sampler = ClockSampler(local)
    hp = args.prec if args.quick else "f32"   # precision of the headline form
    precs = (hp,) if args.quick else ("f64", "f32", "bf16")
    verts, res, forms = measure_grid(w, args, stream, ws, peak, sampler, precs, keep=hp)
    head = res[hp]
    s = head["ctx"]
    ms_med = statistics.median(head["ms"])
    ms_step = ms_med / args.steps
    updates = w.updates_per_step
    value = updates * args.steps * ws / (ms_med * 1e-3) / 1e9

    adjoint = None
    if not args.no_adjoint and not w.isothermal and w.pr == 1.0:
        adjoint = adjoint_time(s, stream, ws, updates)
        adjoint["launches_per_step"] = 2
    e2e = None if args.no_e2e else e2e_time(s, args, ws, updates)
    s.close()
    torch.cuda.empty_cache()

    secondary, one_step2 = None, None
    if not args.quick and args.workload != SECONDARY:
        w2 = _workload(SECONDARY)
        verts2, res2, forms2 = measure_grid(w2, args, stream, ws, peak)
        secondary = {"workload": _workload_desc(w2), "n_vertices": w2.n_vertices,
                     "updates_per_step": w2.updates_per_step, **forms2}
        secondary["f32"]["roofline"]["traffic"] = NCU_TRAFFIC.get((_kernel_digest(), w2.name, "f32"))
        one_step2 = {prec: res2[prec]["one_step"] for prec in precs}
        del res2

    three_d = None if (args.quick or args.no_3d) else measure_3d(args, stream, ws, peak)

    if rank == 0:
        alg_bytes = updates * bytes_per_update(w, hp, head["info"]["kernel"])
        achieved = alg_bytes / (ms_step * 1e-3) / 1e9
        traffic = NCU_TRAFFIC.get((_kernel_digest(), w.name, hp))
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": hp, "data": "synthetic",
            "config": {"workload": _workload_desc(w), "kernel": head["info"]["kernel"],
                       "n_vertices": w.n_vertices, "updates_per_step": updates,
                       "l2": "state 2 x %.0f MB > 129 MB L2, no flush" % (head["info"]["state_bytes"] / 1e6),
                       "timing": f"median of {args.repeats} timed regions of {args.steps} steps",
                       "ms_per_region_repeats": head["ms"],
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"hbm_gbs of {src} peaks (copy bandwidth)",
                         "algorithmic_bytes_per_launch": alg_bytes},
            "clocks": head["clocks"],
            "e2e": e2e,
            "f_only_value": value / w.n_populations,   # the same time counted in f updates only
            "forms": forms,
            "adjoint": adjoint,
            "gpu_launches": args.steps * head["info"]["launches_per_step"],
            "gpu_launches_note": "per timed region of the headline (each of the repeats)",
            "mass_after": head["info"]["mass_after"],
            "secondary": secondary,
            "d3q125": three_d,
        }
        if ws == 1 and not args.no_cpu_baseline:
            # the CPU leg: oracle timings, and the oracle's one-step values at the sampled
            # vertices against which every form's error is stated
            line["cpu_baseline"] = cpu_baseline(w)
            ref = oracle_reference_at(w, verts)
            for prec in precs:
                forms[prec]["err_vs_oracle_1step"] = {
                    "vertices": int(len(verts)),
                    "max_rel": field_errors(res[prec]["one_step"], ref, w.velocity_scale)}
            if secondary is not None:
                ref2 = oracle_reference_at(w2, verts2)
                for prec in precs:
                    secondary[prec]["err_vs_oracle_1step"] = {
                        "vertices": int(len(verts2)),
                        "max_rel": field_errors(one_step2[prec], ref2, w2.velocity_scale)}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--repeats", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="riemann_paper")
    ap.add_argument("--quick", action="store_true", help="one form (--prec) of the headline grid only")
    ap.add_argument("--prec", default="f32", choices=["f32", "bf16", "f64"],
                    help="the form timed with --quick")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3D (D3Q125) entry")
    ap.add_argument("--only-3d", action="store_true", help="the 3D (D3Q125) entry alone")
    ap.add_argument("--d3-cells", type=int, default=64, help="cells per axis of the 3D grid (p = 2)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.repeats < 1 or args.steps < 1:
        ap.error("at least one timed region of one step")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
