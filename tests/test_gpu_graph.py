"""sllbm_step replays pairs of steps as a CUDA graph for calls of 4 or more steps on grids whose
state fits in 64 MB (all of these do).  The graph holds
the same launches with the same parameters as the direct steps, so the state after n steps taken
one call at a time (direct) and in one call (graph) must agree bit for bit.  Covered: the fused
uniform kernel with the fix-up gather on its side stream (zero-gradient grid), a periodic uniform
grid, the mapped kernel, the plain FP64 step, BF16 storage, the D2Q9 kernel; odd counts and a
start from the second state buffer; and the legacy default stream, which cannot be captured
(direct steps, same result)."""
import numpy as np
import pytest

from paper_1910_13918_gb300 import workloads as W

from . import helpers as H

pytestmark = pytest.mark.gpu


def _ctx(w, prec, stream):
    from paper_1910_13918_gb300.sllbm import SLLBM
    s = SLLBM.from_workload(w, prec=prec, stream=stream)
    s.precompute()
    x, y = (t.cpu().numpy() for t in s.coords())
    s.init(*w.fields(x, y, perturb=True))
    return s


CASES = {
    "riemann_f32": (lambda: H.small_workloads()["riemann"], "f32"),
    "tgv_f32": (lambda: W.tgv256().resized(6, 5), "f32"),
    "svi_f32": (lambda: H.small_workloads()["svi"], "f32"),
    "tgv_f64": (lambda: W.tgv256().resized(6, 5), "f64"),
    "riemann_bf16": (lambda: H.small_workloads()["riemann"], "bf16"),
    "d2q9_f32": (lambda: W.tgv_moving(velset="d2q9").resized(8, 8), "f32"),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("first,n", [(0, 9), (1, 6)])
def test_graph_steps_equal_direct_steps(gpu_lib, name, first, n):
    import torch
    make, prec = CASES[name]
    w = make()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a, b = _ctx(w, prec, stream), _ctx(w, prec, stream)
        for s in (a, b):
            if first:
                s.step(1)          # start the n steps from the second state buffer
        for _ in range(n):
            a.step(1)              # one step a call: direct launches
        b.step(n)                  # one call: graph replays (and direct steps for the odd one)
        b.step(5)
        for _ in range(5):
            a.step(1)
        sa, sb = (s.get_state().contiguous().view(torch.uint8).cpu().numpy() for s in (a, b))
    stream.synchronize()
    assert np.array_equal(sa, sb)


def test_default_stream_steps_directly(gpu_lib):
    import torch
    w = H.small_workloads()["riemann"]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        a = _ctx(w, "f32", side)
        a.step(7)
        ref = a.get_state().contiguous().view(torch.uint8).cpu().numpy()
    side.synchronize()
    legacy = torch.cuda.default_stream()
    b = _ctx(w, "f32", legacy)
    b.step(7)
    got = b.get_state().contiguous().view(torch.uint8).cpu().numpy()
    assert np.array_equal(ref, got)
