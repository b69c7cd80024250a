"""The bounded waits of the staging pipelines, on the GPU, without a fault.

The TMA-staged step kernels wait for their staged tiles on mbarriers with an iteration limit.
sllbm_selftest_bounded_wait runs that wait on an mbarrier nothing arrives on (no copy in flight)
and checks that it runs out, sets the error bit and returns; the context stays usable afterwards
(a step and its moments still work on the same device).
"""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports():
    from paper_1910_13918_gb300.sllbm import OK, load
    lib = load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.sllbm_selftest_bounded_wait(stream) == OK
    assert lib.sllbm_selftest_bounded_wait(stream) == OK   # and again: nothing left behind


def test_device_usable_after_the_selftest():
    from paper_1910_13918_gb300 import workloads as W
    from paper_1910_13918_gb300.sllbm import OK, SLLBM, load
    lib = load()
    assert lib.sllbm_selftest_bounded_wait(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == OK
    w = W.tgv16()
    s = SLLBM.from_workload(w, prec="f32")
    s.precompute()
    x, y = (t.cpu().numpy() for t in s.coords())
    s.init(*w.fields(x, y))
    s.step(3)
    m = s.moments()
    assert abs(m["mass"] / (2 * 3.141592653589793) ** 2 - 1) < 1e-6
