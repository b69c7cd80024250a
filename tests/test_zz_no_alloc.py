"""sllbm_moments_noalloc, the allocation-free entry point, against sllbm_moments.

Some callers cannot allocate device memory at the point where they need the mass/energy
diagnostics: a framework whose caching allocator has reserved the device memory, a latency-bound
loop (cudaFree synchronises the device), or a fixed memory budget.  The allocation-free entry
point keeps its reduction scratch in a file-scope device array instead.  This file is collected
last so that a run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process (the first call looks up the array's device address).
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _noalloc(lib, state, nx, ny, cv, A):
    """One call; A None skips the sums (and passes no mass/energy buffer either)."""
    outs = [torch.empty((ny, nx), dtype=torch.float32, device="cuda") for _ in range(4)]
    me = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.sllbm_moments_noalloc(ctypes.c_void_p(state.data_ptr()), nx, ny, cv,
                                   ctypes.c_void_p(A.data_ptr()) if A is not None else None,
                                   *[ctypes.c_void_p(o.data_ptr()) for o in outs],
                                   ctypes.c_void_p(me.data_ptr()) if A is not None else None,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, outs, me.cpu().numpy()


def _check_fields(outs, ref, call):
    for name, got in zip(("rho", "u", "v", "T"), outs):
        np.testing.assert_allclose(got.cpu().numpy(), ref[name].cpu().numpy(), rtol=1e-6,
                                   atol=1e-7, err_msg=f"{name}, call {call}")


def test_moments_noalloc_matches_context_moments_on_two_calls():
    from paper_1910_13918_gb300 import workloads as W
    from paper_1910_13918_gb300.sllbm import SLLBM, load
    lib = load()
    w = W.svi().resized(40, 20, dt=0.01)
    s = SLLBM.from_workload(w, prec="f32")
    s.precompute()
    x, y = (t.cpu().numpy() for t in s.coords())
    s.init(*w.fields(x, y, perturb=True))
    A = s.vertex_weights()
    for call in range(2):          # two calls in a row, on two different states
        s.step(3)
        ref = s.moments()
        state = s.get_state()
        st, outs, me = _noalloc(lib, state, s.nx, s.ny, w.cv, A)
        assert st == 0, lib.sllbm_status_string(st)
        _check_fields(outs, ref, call)
        assert abs(me[0] / ref["mass"] - 1) < 1e-12 and abs(me[1] / ref["energy"] - 1) < 1e-12, \
            (call, me, ref["mass"], ref["energy"])


def test_moments_noalloc_fields_only_and_single_population():
    """Without vertex weights (no sums, no mass/energy buffer) on the two-population state, and
    on a one-population (C_v = 1, isothermal) state whose dense layout has 25 planes only."""
    from paper_1910_13918_gb300 import workloads as W
    from paper_1910_13918_gb300.sllbm import SLLBM, load
    lib = load()
    w = W.tgv16()
    s = SLLBM.from_workload(w, prec="f32")
    s.precompute()
    x, y = (t.cpu().numpy() for t in s.coords())
    s.init(*w.fields(x, y, perturb=True))
    s.step(2)
    st, outs, _ = _noalloc(lib, s.get_state(), s.nx, s.ny, w.cv, None)
    assert st == 0, lib.sllbm_status_string(st)
    _check_fields(outs, s.moments(), "A=NULL")

    wi = W.tgv_moving(points=32)
    assert wi.cv == 1.0 and wi.n_populations == 1
    si = SLLBM.from_workload(wi, prec="f32")
    si.precompute()
    xi, yi = (t.cpu().numpy() for t in si.coords())
    si.init(*wi.fields(xi, yi, perturb=True))
    si.step(3)
    state = si.get_state()
    assert state.shape[0] == 1
    A = si.vertex_weights()
    for call in range(2):
        ref = si.moments()
        st, outs, me = _noalloc(lib, state, si.nx, si.ny, 1.0, A)
        assert st == 0, lib.sllbm_status_string(st)
        _check_fields(outs, ref, f"C_v = 1, call {call}")
        assert abs(me[0] / ref["mass"] - 1) < 1e-12 and abs(me[1] / ref["energy"] - 1) < 1e-12
        si.step(1)
        state = si.get_state()


def test_moments_noalloc_rejects_oversized_grid_and_missing_sum_buffer():
    from paper_1910_13918_gb300.sllbm import ERR_ARG, ERR_UNSUPPORTED, load
    lib = load()
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    A = torch.zeros(4, dtype=torch.float64, device="cuda")
    me = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(nx, ny, a, m):
        return lib.sllbm_moments_noalloc(ctypes.c_void_p(dummy.data_ptr()), nx, ny, 2.5, a,
                                         None, None, None, None, m, stream)

    # all rejected on the host before anything is launched (the 4-float dummy is never read):
    # 4097 x 4097 vertices exceed the 16,777,216-vertex scratch; 2^20 x 2^20 vertices would wrap
    # a 32-bit block count; vertex weights without a buffer for the sums are an argument error
    assert call(4097, 4097, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(me.data_ptr())) == ERR_UNSUPPORTED
    assert call(1 << 20, 1 << 20, None, None) == ERR_UNSUPPORTED
    assert call(2, 2, ctypes.c_void_p(A.data_ptr()), None) == ERR_ARG
