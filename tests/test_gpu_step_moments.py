"""The moments epilogue of the step kernels (sllbm_step_moments) against sllbm_moments.

BGK conserves mass, momentum and energy (Sec. II), so the moments each vertex's collision was
evaluated at are those of the state the step produces; the epilogue writes them from the fused,
fix-up, mapped and plain FP64 kernels without a second pass over the state.  Compared here with
the separate moments kernel (FP64 sums of the stored state) after the same step: to FP32
rounding for FP32 storage, to the precision of the FP32 output for the FP64 step, and to the
BF16 rounding of the stored state for BF16 storage.
"""
import numpy as np
import pytest

from . import helpers as H

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["tgv256", "riemann", "svi", "sod"])
@pytest.mark.parametrize("prec,tol", [("f32", 3e-6), ("f64", 1e-6), ("bf16", 3e-2)])
def test_step_moments_equal_the_moments_of_the_produced_state(name, prec, tol):
    import torch
    from paper_1910_13918_gb300.sllbm import SLLBM
    w = H.small_workloads()[name]
    s = SLLBM.from_workload(w, prec=prec)
    s.precompute()
    x, y = (t.cpu().numpy() for t in s.coords())
    s.init(*w.fields(x, y, perturb=True))
    s.step(3)
    buf = torch.full((4, s.ny, s.nx), float("nan"), dtype=torch.float32, device="cuda")
    s.step_moments(buf)
    m = s.moments()
    got = buf.double().cpu().numpy()
    ref = [m[k].double().cpu().numpy() for k in ("rho", "u", "v", "T")]
    assert np.all(np.isfinite(got)), "every vertex written (fused and fix-up kernels)"
    err = H.field_errors(got, ref, w.velocity_scale)
    assert max(err.values()) < tol, (s.kernel_name, err)


def test_step_moments_advances_like_step():
    """A step with the epilogue produces the same state as a plain step."""
    import torch
    from paper_1910_13918_gb300.sllbm import SLLBM
    w = H.small_workloads()["riemann"]
    states = []
    for with_moments in (False, True):
        s = SLLBM.from_workload(w, prec="f32")
        s.precompute()
        x, y = (t.cpu().numpy() for t in s.coords())
        s.init(*w.fields(x, y, perturb=True))
        if with_moments:
            buf = torch.empty((4, s.ny, s.nx), dtype=torch.float32, device="cuda")
            for _ in range(4):
                s.step_moments(buf)
        else:
            s.step(4)
        states.append(s.get_state().cpu().numpy())
    assert np.array_equal(states[0], states[1])
