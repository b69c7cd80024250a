"""State in and out of the library (checkpoint / resume and the host-buffer step): the dense
[n_pop][25][ny][nx] layout round-trips exactly through the internal one, and the host-buffer step
equals set_state + step + get_state bit for bit (its copies are split into plane groups that
overlap the layout conversion)."""
import numpy as np
import pytest
import torch

from paper_1910_13918_gb300 import workloads as W

from . import helpers as H

pytestmark = pytest.mark.gpu

CASES = [("tgv256", "f32"), ("tgv256", "bf16"), ("tgv256", "f64"), ("svi", "f32"), ("sod", "f32")]


def _ctx(w, prec):
    from paper_1910_13918_gb300.sllbm import SLLBM
    s = SLLBM.from_workload(w, prec=prec)
    s.precompute()
    x, y = (t.cpu().numpy() for t in s.coords())
    s.init(*w.fields(x, y, perturb=True))
    return s


@pytest.mark.parametrize("name,prec", CASES + [("tgv_moving", "f32")])
def test_round_trip_and_host_step(gpu_lib, name, prec):
    w = W.tgv_moving(32) if name == "tgv_moving" else H.small_workloads()[name]
    s = _ctx(w, prec)
    s.step(3)
    st = s.get_state().clone()
    s.set_state(st)
    assert torch.equal(s.get_state(), st)
    # host-buffer step against the device path
    host_in = st.cpu().contiguous()
    a_in = host_in.view(torch.uint8).numpy().reshape(-1)
    a_out = np.empty_like(a_in)
    s.step_host(a_in, a_out, 2)
    s.set_state(st)
    s.step(2)
    dev = s.get_state().cpu().contiguous().view(torch.uint8).numpy().reshape(-1)
    assert np.array_equal(a_out, dev)
