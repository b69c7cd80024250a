"""Full-size workloads on the GPU, in the launch configuration the benchmark times.

* one step: sampled vertices against the oracle, which evaluates the step only at those
  vertices (its initial state only where their stencils reach);
* long runs: the fused FP32 step against the plain FP64 GPU step (itself pinned to the oracle
  element by element in test_gpu_parity.py), plus size-independent properties.
"""
import numpy as np
import pytest
import torch

from paper_1910_13918_gb300 import workloads as W

from . import helpers as H

pytestmark = pytest.mark.gpu


def _sample(w, n=48, seed=11):
    rng = np.random.default_rng(seed)
    nx, ny = w.nx, w.ny
    pts = {(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1), (nx // 2, ny // 2), (1, ny // 3),
           (nx - 2, (2 * ny) // 3), (nx // 3, 1), (nx // 3, ny - 2)}
    for _ in range(n):
        pts.add((int(rng.integers(nx)), int(rng.integers(ny))))
    return np.array(sorted(iy * nx + ix for ix, iy in pts))


def _gpu(w, nsteps, prec):
    from paper_1910_13918_gb300.sllbm import SLLBM
    s = SLLBM.from_workload(w, prec=prec)
    s.precompute()
    x, y = (t.cpu().numpy() for t in s.coords())
    s.init(*w.fields(x, y, perturb=True))
    s.step(nsteps)
    return s


def _fields(s):
    m = s.moments()
    return tuple(m[k].cpu().numpy().reshape(-1) for k in ("rho", "u", "v", "T")), m


@pytest.mark.parametrize("name", ["tgv256", "sod", "riemann", "riemann_paper", "svi"])
def test_one_step_sampled_against_oracle(gpu_lib, name):
    w = W.ALL[name]()
    s = _gpu(w, 1, "f32")
    got, _ = _fields(s)
    verts = _sample(w)
    ref = H.oracle_step_at(w, verts)
    err = H.field_errors(tuple(a[verts] for a in got), ref, w.velocity_scale)
    assert max(err.values()) <= 1e-5, (name, s.kernel_name, err)


@pytest.mark.parametrize("name,nsteps", [("tgv256", 1000), ("riemann_paper", 200), ("svi", 200),
                                         ("sod", 300)])
def test_long_run_f32_against_f64(gpu_lib, name, nsteps):
    w = W.ALL[name]()
    a, ma = _fields(_gpu(w, nsteps, "f32"))
    b, mb = _fields(_gpu(w, nsteps, "f64"))
    err = H.field_errors(a, b, w.velocity_scale)
    assert max(err.values()) <= 1e-4, (name, err)
    assert abs(ma["mass"] / mb["mass"] - 1) < 1e-6


def test_riemann_table3_to_end_time_f32_against_f64(gpu_lib):
    """The 1024 x 1024-cell p = 3 grid with the Table III states to t = 0.3 (7447 steps), FP32
    against FP64, the FP64 mass and energy taken every 100 steps.  Over the whole field the FP32
    run follows the FP64 one to 1e-4 (L1, and at 99.9 % of the vertices); the largest pointwise
    differences, a few 1e-3, sit on the shock fronts, where the two runs place a discontinuity a
    fraction of a spacing apart.  The mass grows by what the zero-gradient boundaries let in
    (density 1 at speed 0.7276 through half of the left and half of the bottom edge)."""
    w = W.riemann_paper()
    runs = {}
    for prec in ("f32", "f64"):
        s = _gpu(w, 0, prec)
        log = []
        done = 0
        while done < w.steps:
            n = min(100, w.steps - done)
            s.step(n)
            done += n
            m = s.moments()
            log.append((done, m["mass"], m["energy"]))
        runs[prec] = (torch.stack([m[k].double() for k in ("rho", "u", "v", "T")]), log)
        s.close()
        torch.cuda.empty_cache()
    a, b = runs["f32"][0], runs["f64"][0]
    d = (a - b).abs()
    umax = max(float(b[1].abs().max()), float(b[2].abs().max()))
    scale = [b[0].abs(), umax, umax, b[3].abs()]
    for i, name in enumerate(("rho", "u", "v", "T")):
        l1 = float(d[i].sum() / (b[i].abs().sum() if i in (0, 3) else umax * b[i].numel()))
        rel = (d[i] / scale[i]).reshape(-1)
        p999 = float(torch.quantile(rel[::97], 0.999))
        print(f"riemann t = 0.3 {name}: L1 {l1:.2e}, 99.9 % {p999:.2e}, max {float(rel.max()):.2e}")
        assert l1 <= 1e-4 and p999 <= 1e-4, (name, l1, p999)
    for (n, m32, e32), (_, m64, e64) in zip(runs["f32"][1], runs["f64"][1]):
        assert abs(m32 / m64 - 1) < 2e-6 and abs(e32 / e64 - 1) < 2e-6, (n, m32, m64, e32, e64)
    m0 = 0.25 * sum(st[0] for st in W.RIEMANN_STATES_PAPER.values())
    t = w.steps * w.dt
    assert abs(runs["f64"][1][-1][1] / (m0 + 0.7276 * t) - 1) < 0.01, (runs["f64"][1][-1], m0, t)


def test_sod_long_run_f32_mass_tracks_f64(gpu_lib):
    """2000 steps of the Sod workload: the FP32 run keeps the FP64 run's mass (the interpolation
    reproduces constants exactly, so uniform regions do not drift) and its fields."""
    w = W.sod()
    n = 2000
    a, ma = _fields(_gpu(w, n, "f32"))
    b, mb = _fields(_gpu(w, n, "f64"))
    err = H.field_errors(a, b, w.velocity_scale)
    print("sod 2000 steps f32 vs f64:", err, "mass", ma["mass"] / mb["mass"] - 1)
    assert abs(ma["mass"] / mb["mass"] - 1) < 2e-6
    assert max(err.values()) < 1e-3, err


def test_tgv256_mass_and_energy_conserved(gpu_lib):
    w = W.tgv256()
    s = _gpu(w, 0, "f32")
    m0 = s.moments()
    s.step(500)
    m1 = s.moments()
    assert abs(m1["mass"] / m0["mass"] - 1) < 1e-6
    assert abs(m1["energy"] / m0["energy"] - 1) < 1e-5


def test_sod_full_run_matches_exact_solution(gpu_lib):
    """The Sod workload to t = 0.2 (13240 fused steps) against the exact Riemann solution."""
    from oracle import riemann
    w = W.sod()
    s = _gpu(w, w.steps, "f32")
    m = s.moments()
    x, _ = (t.cpu().numpy() for t in s.coords())
    rho = m["rho"].cpu().numpy()[0]
    re, _, _ = riemann.sample((1, 0, 1), (0.125, 0, 0.1), 1.4, (x[0] - 0.5) / 0.2)
    assert np.mean(np.abs(rho - re)) < 0.01, np.mean(np.abs(rho - re))


def test_riemann_baseline_states_leave_the_model_range(gpu_lib):
    """The four-quadrant states with the cold SW corner (T = 0.21 at |u| = 1.7) drive the
    temperature negative within a few steps, in FP32 and FP64 alike (the oracle does the same on
    a small grid: tests/test_oracle_physics.py)."""
    from paper_1910_13918_gb300.sllbm import SLLBMError
    w = W.riemann()
    for prec in ("f32", "f64"):
        s = _gpu(w, 0, prec)
        with pytest.raises(SLLBMError):
            for _ in range(10):
                s.step(1)
                s.moments(sums=False)


def test_svi_adjoint_against_central_differences(gpu_lib):
    """Shock-vortex workload (mapped grid, 200 steps, checkpoints every 20): the FP32 adjoint
    gradient of J = sum_{x > 1.5} A_v rho_v(t_end) w.r.t. the initial velocity, projected on 16
    seeded directions (N(0,1) x the vortex envelope), against central differences of the FP64
    forward step (eps = 1e-6 relative to the inflow speed)."""
    from paper_1910_13918_gb300.autograd import rollout
    from paper_1910_13918_gb300.sllbm import SLLBM
    w = W.svi()
    k = w.extra["checkpoint_every"]
    s = SLLBM.from_workload(w, prec="f32")
    s.precompute()
    x, y = (t.cpu().numpy() for t in s.coords())
    r, u, v, T = (torch.as_tensor(f, dtype=torch.float64, device="cuda") for f in w.fields(x, y))
    u.requires_grad_(True)
    v.requires_grad_(True)
    A = s.vertex_weights()
    mask = torch.as_tensor(x > w.extra["x_objective"], device="cuda")
    rho = rollout(s, u, v, r, T, w.steps, k)
    J = (A * mask * rho).sum()
    J.backward()
    du, dv = u.grad.cpu().numpy(), v.grad.cpu().numpy()
    # FP64 forward for the differences
    s64 = SLLBM.from_workload(w, prec="f64")
    s64.precompute()
    A64 = s64.vertex_weights().cpu().numpy()
    m64 = x > w.extra["x_objective"]
    rho0, u0, v0, T0 = w.fields(x, y)

    def J64(uu, vv):
        s64.init(rho0, uu, vv, T0)
        s64.step(w.steps)
        st = s64.get_state().cpu().numpy()
        return float(np.sum(A64 * m64 * st[0].sum(axis=0)))

    eps = 1e-6 * w.velocity_scale
    errs, ads = [], []
    for d1, d2 in W.svi_directions(w, x, y, 16):
        fd = (J64(u0 + eps * d1, v0 + eps * d2) - J64(u0 - eps * d1, v0 - eps * d2)) / (2 * eps)
        ad = float(np.sum(du * d1) + np.sum(dv * d2))
        errs.append(abs(fd - ad))
        ads.append(abs(ad))
    scale = max(ads)
    print("svi adjoint: max |AD| =", scale, "max |FD - AD| =", max(errs))
    assert scale > 1e-7, scale                      # a gradient well above FD round-off (~1e-9)
    # every direction within 1e-4 of the gradient's scale (the FP32 adjoint's rounding)
    for d, (e, ad) in enumerate(zip(errs, ads)):
        assert e <= 1e-4 * scale, (d, e, ad, scale)
