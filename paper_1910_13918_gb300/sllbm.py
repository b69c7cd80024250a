"""Python binding of the SLLBM C ABI (``include/sllbm.h``) -- argument marshalling only.

Every step of the method runs in the CUDA library; this module passes device pointers of torch
CUDA tensors and the current CUDA stream through ``ctypes``.  There is no fallback: if the
library cannot be built or loaded, or CUDA is unavailable, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build
from . import workloads as _wl

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_STATE, ERR_NEWTON, ERR_UNSTABLE, ERR_UNSUPPORTED = range(8)
BC_PERIODIC, BC_ZERO_GRADIENT = 0, 1
NODES_GLC, NODES_EQUIDISTANT = 0, 1
MAP_IDENTITY, MAP_SINE = 0, 1
PREC_F32, PREC_BF16_STORE, PREC_F64_PLAIN = 0, 1, 2
VEL_D2Q25, VEL_D2Q9, VEL_D3Q125 = 0, 1, 2
VELSETS = {"d2q25": VEL_D2Q25, "d2q9": VEL_D2Q9}
PRECISIONS = {"f32": PREC_F32, "bf16": PREC_BF16_STORE, "f64": PREC_F64_PLAIN}

# every exported symbol of include/sllbm.h
EXPORTS = [
    "sllbm_create", "sllbm_destroy", "sllbm_set_stream", "sllbm_grid_info", "sllbm_state_bytes",
    "sllbm_vertex_coords", "sllbm_vertex_weights", "sllbm_precompute_departures",
    "sllbm_init_equilibrium", "sllbm_step", "sllbm_step_moments", "sllbm_step_host", "sllbm_moments", "sllbm_get_state",
    "sllbm_set_state", "sllbm_adjoint_step", "sllbm_init_equilibrium_vjp", "sllbm_step_kernel_name",
    "sllbm_launches_per_step", "sllbm_status_string", "sllbm_last_error", "sllbm_moments_noalloc",
    "sllbm_selftest_bounded_wait",
    "sllbm3d_create", "sllbm3d_destroy", "sllbm3d_grid_info", "sllbm3d_vertex_coords",
    "sllbm3d_precompute_departures", "sllbm3d_init_equilibrium", "sllbm3d_step", "sllbm3d_moments",
    "sllbm3d_get_state", "sllbm3d_set_state", "sllbm3d_last_error", "sllbm3d_step_kernel_name",
]


class GridDesc(ctypes.Structure):
    _fields_ = [("nx_cells", ctypes.c_int), ("ny_cells", ctypes.c_int), ("order", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double),
                ("y1", ctypes.c_double), ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
                ("nodes", ctypes.c_int), ("map", ctypes.c_int), ("map_param", ctypes.c_double * 4)]


class GridDesc3(ctypes.Structure):
    _fields_ = [("nx_cells", ctypes.c_int), ("ny_cells", ctypes.c_int), ("nz_cells", ctypes.c_int),
                ("order", ctypes.c_int), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double), ("z0", ctypes.c_double),
                ("z1", ctypes.c_double), ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
                ("bc_z", ctypes.c_int), ("nodes", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("velset", ctypes.c_int), ("dt", ctypes.c_double), ("tau", ctypes.c_double),
                ("cv", ctypes.c_double), ("T0", ctypes.c_double), ("prec", ctypes.c_int),
                ("pr", ctypes.c_double), ("isothermal", ctypes.c_int)]


class SLLBMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"SLLBM status {status}: {message}")
        self.status = status


_LIB = None


def load(path: str | None = None):
    """Build (if stale) and load the CUDA library.  Raises if that is impossible."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if path is None:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"SLLBM CUDA library missing at {path}")
    lib = ctypes.CDLL(path)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "sllbm_create": ([ctypes.POINTER(GridDesc), ctypes.POINTER(Params), P, ctypes.POINTER(P)], I),
        "sllbm_destroy": ([P], I),
        "sllbm_set_stream": ([P, P], I),
        "sllbm_grid_info": ([P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "sllbm_state_bytes": ([P, ctypes.POINTER(ctypes.c_size_t)], I),
        "sllbm_vertex_coords": ([P, V, V], I),
        "sllbm_vertex_weights": ([P, V], I),
        "sllbm_precompute_departures": ([P], I),
        "sllbm_init_equilibrium": ([P, V, V, V, V], I),
        "sllbm_step": ([P, I], I),
        "sllbm_step_moments": ([P, V], I),
        "sllbm_step_host": ([P, V, V, I], I),
        "sllbm_moments": ([P, V, V, V, V, ctypes.POINTER(D)], I),
        "sllbm_get_state": ([P, V], I),
        "sllbm_set_state": ([P, V], I),
        "sllbm_adjoint_step": ([P, V, V, V], I),
        "sllbm_init_equilibrium_vjp": ([P, V, V, V, V, V, V, V], I),
        "sllbm_step_kernel_name": ([P], ctypes.c_char_p),
        "sllbm_launches_per_step": ([P], I),
        "sllbm_status_string": ([I], ctypes.c_char_p),
        "sllbm_moments_noalloc": ([V, I, I, D, V, V, V, V, V, V, P], I),
        "sllbm_last_error": ([P], ctypes.c_char_p),
        "sllbm_selftest_bounded_wait": ([P], I),
        "sllbm3d_create": ([ctypes.POINTER(GridDesc3), ctypes.POINTER(Params), P, ctypes.POINTER(P)], I),
        "sllbm3d_destroy": ([P], I),
        "sllbm3d_grid_info": ([P] + [ctypes.POINTER(I)] * 4, I),
        "sllbm3d_vertex_coords": ([P, V, V, V], I),
        "sllbm3d_precompute_departures": ([P], I),
        "sllbm3d_init_equilibrium": ([P, V, V, V, V, V], I),
        "sllbm3d_step": ([P, I], I),
        "sllbm3d_moments": ([P, V, V, V, V, V], I),
        "sllbm3d_get_state": ([P, V], I),
        "sllbm3d_set_state": ([P, V], I),
        "sllbm3d_last_error": ([P], ctypes.c_char_p),
        "sllbm3d_step_kernel_name": ([P], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = lib
    return lib


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


class SLLBM:
    """One simulation context on the current CUDA device.

    ``grid`` and ``params`` are the plain fields of ``sllbm_grid_desc`` / ``sllbm_params``; use
    :meth:`from_workload` for the seeded workloads.
    """

    def __init__(self, *, nx_cells, ny_cells, order, x0, x1, y0, y1, bc_x, bc_y, dt, tau, cv,
                 prec="f32", nodes=NODES_GLC, map_kind=MAP_IDENTITY, map_a=0.0, pr=1.0,
                 isothermal=False, velset="d2q25", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("SLLBM needs a CUDA device; there is no CPU path")
        self.torch = torch
        self.lib = load()
        self.prec = prec
        g = GridDesc(nx_cells, ny_cells, order, x0, x1, y0, y1, bc_x, bc_y, nodes, map_kind,
                     (ctypes.c_double * 4)(map_a, 0.0, 0.0, 0.0))
        p = Params(VELSETS[velset], dt, tau, cv, 1.0, PRECISIONS[prec], pr, int(bool(isothermal)))
        self.nq = 9 if velset == "d2q9" else 25
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        self._check(self.lib.sllbm_create(ctypes.byref(g), ctypes.byref(p),
                                          ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(h)),
                    ctx=None)
        self.h = h
        nx, ny, npop = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.sllbm_grid_info(h, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(npop)))
        self.nx, self.ny, self.npop = nx.value, ny.value, npop.value
        self.n_vertices = self.nx * self.ny
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.state_dtype = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[prec]

    @classmethod
    def from_workload(cls, w: _wl.Workload, prec="f32", stream=None):
        return cls(nx_cells=w.nx_cells, ny_cells=w.ny_cells, order=w.order, x0=w.x0, x1=w.x1,
                   y0=w.y0, y1=w.y1, bc_x=w.bc_x, bc_y=w.bc_y, dt=w.dt, tau=w.tau, cv=w.cv,
                   prec=prec, nodes=NODES_GLC if w.nodes == "glc" else NODES_EQUIDISTANT,
                   map_kind=MAP_SINE if w.map_a else MAP_IDENTITY, map_a=w.map_a, pr=w.pr,
                   isothermal=w.isothermal, velset=w.velset, stream=stream)

    # -- plumbing -------------------------------------------------------------------------------
    def _check(self, status, ctx="self"):
        if status != OK:
            h = self.h if ctx == "self" else None
            msg = self.lib.sllbm_last_error(h).decode() if h else \
                self.lib.sllbm_status_string(status).decode()
            raise SLLBMError(status, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.sllbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vertex_tensor(self, dtype):
        return self.torch.empty((self.ny, self.nx), dtype=dtype, device=self.device)

    # -- API ------------------------------------------------------------------------------------
    @property
    def kernel_name(self):
        return self.lib.sllbm_step_kernel_name(self.h).decode()

    @property
    def launches_per_step(self):
        return int(self.lib.sllbm_launches_per_step(self.h))

    @property
    def state_bytes(self):
        b = ctypes.c_size_t()
        self._check(self.lib.sllbm_state_bytes(self.h, ctypes.byref(b)))
        return b.value

    def coords(self):
        x = self._vertex_tensor(self.torch.float64)
        y = self._vertex_tensor(self.torch.float64)
        self._check(self.lib.sllbm_vertex_coords(self.h, _ptr(x), _ptr(y)))
        return x, y

    def vertex_weights(self):
        A = self._vertex_tensor(self.torch.float64)
        self._check(self.lib.sllbm_vertex_weights(self.h, _ptr(A)))
        return A

    def precompute(self):
        self._check(self.lib.sllbm_precompute_departures(self.h))

    def init(self, rho, u, v, T):
        ts = [self.torch.as_tensor(a, dtype=self.torch.float64, device=self.device).contiguous()
              for a in (rho, u, v, T)]
        for t in ts:
            assert t.numel() == self.n_vertices
        self._check(self.lib.sllbm_init_equilibrium(self.h, *[_ptr(t) for t in ts]))
        self._init_inputs = ts

    def step(self, n=1):
        self._check(self.lib.sllbm_step(self.h, int(n)))

    def step_moments(self, buf4):
        """One step writing the (rho, u, v, theta) its collision used into a [4, ny, nx] float32
        tensor (the saved moments of the adjoint step)."""
        assert buf4.dtype == self.torch.float32 and buf4.is_contiguous() and buf4.numel() == 4 * self.n_vertices
        self._check(self.lib.sllbm_step_moments(self.h, _ptr(buf4)))

    def moments(self, sums=True):
        rho, u, v, T = (self._vertex_tensor(self.torch.float32) for _ in range(4))
        me = (ctypes.c_double * 2)()
        self._check(self.lib.sllbm_moments(self.h, _ptr(rho), _ptr(u), _ptr(v), _ptr(T),
                                           me if sums else None))
        out = {"rho": rho, "u": u, "v": v, "T": T}
        if sums:
            out["mass"], out["energy"] = me[0], me[1]
        return out

    def moments_into(self, buf4):
        """Write (rho, u, v, theta) into a [4, ny, nx] float32 tensor (no host sync of sums)."""
        n = self.n_vertices
        base = buf4.data_ptr()
        es = buf4.element_size()
        self._check(self.lib.sllbm_moments(self.h, ctypes.c_void_p(base), ctypes.c_void_p(base + n * es),
                                           ctypes.c_void_p(base + 2 * n * es),
                                           ctypes.c_void_p(base + 3 * n * es), None))

    def get_state(self, out=None):
        if out is None:
            out = self.torch.empty((self.npop, self.nq, self.ny, self.nx), dtype=self.state_dtype,
                                   device=self.device)
        self._check(self.lib.sllbm_get_state(self.h, _ptr(out)))
        return out

    def set_state(self, t):
        t = t.contiguous()
        assert t.numel() * t.element_size() == self.state_bytes
        self._check(self.lib.sllbm_set_state(self.h, _ptr(t)))

    def step_host(self, state_in: np.ndarray, state_out: np.ndarray, n=1):
        """Host-buffer step (copies in, n steps, copies out, synchronises)."""
        assert state_in.nbytes == self.state_bytes and state_out.nbytes == self.state_bytes
        self._check(self.lib.sllbm_step_host(self.h, ctypes.c_void_p(state_in.ctypes.data),
                                             ctypes.c_void_p(state_out.ctypes.data), int(n)))

    def adjoint_step(self, lam_in, lam_out, moments4):
        for t in (lam_in, lam_out):
            assert t.dtype == self.torch.float32 and t.is_contiguous() and t.numel() == 50 * self.n_vertices
        assert moments4.dtype == self.torch.float32 and moments4.numel() == 4 * self.n_vertices
        self._check(self.lib.sllbm_adjoint_step(self.h, _ptr(lam_in), _ptr(lam_out), _ptr(moments4)))

    def init_vjp(self, rho, u, v, T, lam0):
        ts = [self.torch.as_tensor(a, dtype=self.torch.float64, device=self.device).contiguous()
              for a in (rho, u, v, T)]
        du = self._vertex_tensor(self.torch.float32)
        dv = self._vertex_tensor(self.torch.float32)
        self._check(self.lib.sllbm_init_equilibrium_vjp(self.h, *[_ptr(t) for t in ts], _ptr(lam0),
                                                        _ptr(du), _ptr(dv)))
        return du, dv


class SLLBM3D:
    """The 3D extension (D3Q125, hexahedral cells) on the current CUDA device: the plain FP64 step
    (``prec="f64"``) or an FP32 step on deviation pairs (``prec="f32"``: sum-factorised and
    TMA-staged where the grid allows, else the one-launch gather step)."""

    def __init__(self, *, cells, order, box, bc, dt, tau, cv, isothermal=False,
                 nodes=NODES_GLC, prec="f64", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("SLLBM3D needs a CUDA device; there is no CPU path")
        self.torch = torch
        self.lib = load()
        (x0, x1), (y0, y1), (z0, z1) = box
        g = GridDesc3(*cells, order, x0, x1, y0, y1, z0, z1, *bc, nodes)
        if prec not in ("f32", "f64"):
            raise ValueError("3D precisions: f32 (fused FP32 step) or f64 (plain FP64 step)")
        self.prec = prec
        p = Params(VEL_D3Q125, dt, tau, cv, 1.0, PRECISIONS[prec], 1.0, int(bool(isothermal)))
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = self.lib.sllbm3d_create(ctypes.byref(g), ctypes.byref(p),
                                     ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(h))
        if st != OK:
            raise SLLBMError(st, self.lib.sllbm_status_string(st).decode())
        self.h = h
        n = [ctypes.c_int() for _ in range(4)]
        self._check(self.lib.sllbm3d_grid_info(h, *[ctypes.byref(x) for x in n]))
        self.nx, self.ny, self.nz, self.npop = (x.value for x in n)
        self.shape = (self.nz, self.ny, self.nx)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def _check(self, status):
        if status != OK:
            raise SLLBMError(status, self.lib.sllbm3d_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.sllbm3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _field(self):
        return self.torch.empty(self.shape, dtype=self.torch.float64, device=self.device)

    def coords(self):
        x, y, z = self._field(), self._field(), self._field()
        self._check(self.lib.sllbm3d_vertex_coords(self.h, _ptr(x), _ptr(y), _ptr(z)))
        return x, y, z

    def precompute(self):
        self._check(self.lib.sllbm3d_precompute_departures(self.h))

    @property
    def kernel_name(self):
        """The kernel sllbm3d_step uses: "stream3d", "gather_f32" or "plain_f64"."""
        return self.lib.sllbm3d_step_kernel_name(self.h).decode()

    def init(self, rho, u, v, w, T):
        ts = [self.torch.as_tensor(a, dtype=self.torch.float64, device=self.device).contiguous()
              for a in (rho, u, v, w, T)]
        for t in ts:
            assert t.numel() == self.nx * self.ny * self.nz
        self._check(self.lib.sllbm3d_init_equilibrium(self.h, *[_ptr(t) for t in ts]))
        self._init_inputs = ts

    def step(self, n=1):
        self._check(self.lib.sllbm3d_step(self.h, int(n)))

    def moments(self):
        out = {k: self._field() for k in ("rho", "u", "v", "w", "T")}
        self._check(self.lib.sllbm3d_moments(self.h, *[_ptr(out[k]) for k in ("rho", "u", "v", "w", "T")]))
        return out

    def get_state(self):
        out = self.torch.empty((self.npop, 125) + self.shape, dtype=self.torch.float64, device=self.device)
        self._check(self.lib.sllbm3d_get_state(self.h, _ptr(out)))
        return out

    def set_state(self, t):
        t = t.contiguous()
        assert t.dtype == self.torch.float64 and t.numel() == self.npop * 125 * self.nx * self.ny * self.nz
        self._check(self.lib.sllbm3d_set_state(self.h, _ptr(t)))
