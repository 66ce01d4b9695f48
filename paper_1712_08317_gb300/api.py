"""Thin Python layer over the C ABI: argument marshalling only.

Every step of the residual and the time step runs in libweno3.so (host
mesh builder + precompute, sm_103a kernels).  PyTorch provides device
memory and streams; numpy arrays carry host inputs.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _capi as capi

__all__ = ["Mesh", "Solver", "split_fp32", "params_struct", "probe_peak"]


PROBE_KINDS = {"ffma": 0, "ffma2": 1, "dfma": 2, "rcp": 3}


def probe_peak(kind: str, iters: int, stream=None):
    """Measured throughput of one SM pipe (weno_probe_peak): (operations per second, ops, ms)."""
    import torch
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream if stream is None else stream.cuda_stream)
    ops = C.c_double()
    ms = C.c_float()
    capi.check(capi.load().weno_probe_peak(PROBE_KINDS[kind], int(iters), st, C.byref(ops), C.byref(ms)))
    return ops.value / (ms.value * 1e-3), ops.value, ms.value


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Mesh:
    """Host mesh (topology, renumbering, stencils) owned by the library."""

    def __init__(self, nodes, cell_ptr, cell_nodes, bc="periodic", origin=(0.0, 0.0), extent=(1.0, 1.0), walls=(),
                 wall_from=(0.0, 0.0, 0.0, 0.0), inflow=(), _handle=None):
        self._lib = capi.load()
        if _handle is not None:
            self._h = _handle
        else:
            nodes = np.ascontiguousarray(nodes, dtype=np.float64)
            cell_ptr = np.ascontiguousarray(cell_ptr, dtype=np.int64)
            cell_nodes = np.ascontiguousarray(cell_nodes, dtype=np.int64)
            opts = capi.weno_mesh_opts()
            opts.bc = capi.WENO_BC_PERIODIC if bc == "periodic" else capi.WENO_BC_OUTFLOW
            opts.origin[0], opts.origin[1] = origin
            opts.extent[0], opts.extent[1] = extent
            opts.walls = sum(1 << int(w) for w in set(walls))
            for k in range(4):
                opts.wall_from[k] = float(wall_from[k])
            opts.inflow = sum(1 << int(w) for w in set(inflow))
            h = C.c_void_p()
            capi.check(self._lib.weno_mesh_create(_ptr(nodes), nodes.shape[0], _ptr(cell_ptr), _ptr(cell_nodes),
                                                  cell_ptr.shape[0] - 1, C.byref(opts), C.byref(h)))
            self._h = h
        self.info = self._info()
        self.perm = np.empty(self.info.n_cells, dtype=np.int64)
        capi.check(self._lib.weno_mesh_cell_permutation(self._h, _ptr(self.perm)))
        self.instance = np.empty(self.info.n_cells, dtype=np.int32)
        capi.check(self._lib.weno_mesh_cell_instance(self._h, _ptr(self.instance)))

    @classmethod
    def from_input(cls, mi):
        return cls(mi.nodes, mi.cell_ptr, mi.cell_nodes, mi.bc, mi.origin, mi.extent, getattr(mi, "walls", ()),
                   getattr(mi, "wall_from", (0.0, 0.0, 0.0, 0.0)), getattr(mi, "inflow", ()))

    @classmethod
    def concat(cls, meshes):
        arr = (C.c_void_p * len(meshes))(*[m._h for m in meshes])
        h = C.c_void_p()
        capi.check(capi.load().weno_mesh_concat(arr, len(meshes), C.byref(h)))
        return cls(None, None, None, _handle=h)

    def _info(self):
        info = capi.weno_mesh_info()
        capi.check(self._lib.weno_mesh_get_info(self._h, C.byref(info)))
        return info

    @property
    def n_cells(self):
        return int(self.info.n_cells)

    def weight_stats(self, **params):
        p = params_struct(**params)
        raw = np.empty(self.n_cells)
        opt = np.empty(self.n_cells)
        capi.check(self._lib.weno_mesh_weight_stats(self._h, C.byref(p), _ptr(raw), _ptr(opt)))
        return raw, opt

    def cell_tables(self, cell: int, **params):
        """Host FP64 run-time tables of one internal cell: dict(slot, grad_op, dg, gamma)."""
        p = params_struct(**params)
        slot = np.zeros(12, np.int32)
        gop = np.zeros((12, 4))
        dg = np.zeros((8, 2))
        gam = np.zeros(96)
        mg = np.zeros(2, np.int32)
        capi.check(self._lib.weno_mesh_cell_tables(self._h, C.byref(p), int(cell), _ptr(slot), _ptr(gop), _ptr(dg),
                                                   _ptr(gam), _ptr(mg)))
        M, G = int(mg[0]), int(mg[1])
        return {"M": M, "G": G, "slot": slot[:M].copy(), "grad_op": gop[:M].copy(), "dg": dg[:G].copy(),
                "gamma": gam[:G * M].reshape(G, M).copy()}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and getattr(self, "_lib", None) is not None:
            self._lib.weno_mesh_destroy(h)
            self._h = None


def params_struct(eqn="euler", precision="fp64", gas_gamma=1.4, adv=(1.0, 1.0), eps=1e-3, theta=3.0,
                  rcond=1e-12, optimize=True, linear=False, n_threads=0, characteristic=False, inflow_a=None,
                  inflow_b=None, inflow_line=(1.0, 0.0, 0.0, 0.0)):
    p = capi.weno_params()
    capi.load().weno_params_default(C.byref(p))
    p.eqn = capi.WENO_EQN_EULER if eqn == "euler" else capi.WENO_EQN_SCALAR
    p.precision = capi.WENO_FP64 if precision == "fp64" else capi.WENO_FP32C
    p.gas_gamma = gas_gamma
    p.adv[0], p.adv[1] = adv
    p.eps = eps
    p.theta = theta
    p.rcond = rcond
    p.optimize = int(bool(optimize))
    p.linear = int(bool(linear))
    p.n_threads = n_threads
    p.characteristic = int(bool(characteristic))
    for k in range(4):
        p.inflow_a[k] = 0.0 if inflow_a is None else float(inflow_a[k])
        p.inflow_b[k] = 0.0 if inflow_b is None else float(inflow_b[k])
        p.inflow_line[k] = float(inflow_line[k])
    return p


def split_fp32(W: np.ndarray):
    """FP64 values -> (hi, lo) float32 pair with hi + lo ~ W to ~2^-48 relative."""
    hi = W.astype(np.float32)
    lo = (W - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


class Solver:
    """Device tables + launches for one mesh (or a batch of instances)."""

    def __init__(self, mesh: Mesh, stream=None, **params):
        import torch
        self._torch = torch
        self._lib = capi.load()
        self.mesh = mesh
        self.params = dict(params)
        self.eqn = params.get("eqn", "euler")
        self.precision = params.get("precision", "fp64")
        self.nv = 4 if self.eqn == "euler" else 1
        self.dtype = torch.float64 if self.precision == "fp64" else torch.float32
        p = params_struct(**params)
        h = C.c_void_p()
        capi.check(self._lib.weno_solver_create(mesh._h, C.byref(p), self._stream(stream), C.byref(h)))
        self._h = h
        self.n_cells = mesh.n_cells
        self.n_instances = int(mesh.info.n_instances)

    def _stream(self, stream):
        if stream is None:
            return C.c_void_p(self._torch.cuda.current_stream().cuda_stream)
        return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))

    @staticmethod
    def _p(t):
        return None if t is None else C.c_void_p(t.data_ptr())

    def _check_state(self, U, lo):
        t = self._torch
        assert U.is_cuda and U.is_contiguous() and U.dtype == self.dtype and U.numel() == self.n_cells * self.nv
        if self.precision != "fp64":
            assert lo is not None and lo.is_cuda and lo.is_contiguous() and lo.dtype == t.float32 and lo.shape == U.shape

    # ----------------------------------------------------------- data marshalling
    def to_device(self, W: np.ndarray):
        """(nv, n_cells) FP64 values in input order -> device state (U, U_lo or None), internal order."""
        t = self._torch
        Wi = np.ascontiguousarray(np.asarray(W, dtype=np.float64)[:, self.mesh.perm].T)
        if self.precision == "fp64":
            return t.from_numpy(Wi).cuda(), None
        hi, lo = split_fp32(Wi)
        return t.from_numpy(hi).cuda(), t.from_numpy(lo).cuda()

    def to_host(self, U, U_lo=None) -> np.ndarray:
        """Device state -> (nv, n_cells) FP64 values in input order."""
        Wi = U.double().cpu().numpy().reshape(self.n_cells, self.nv)
        if U_lo is not None:
            Wi = Wi + U_lo.double().cpu().numpy().reshape(self.n_cells, self.nv)
        out = np.empty((self.nv, self.n_cells))
        out[:, self.mesh.perm] = Wi.T
        return out

    # ----------------------------------------------------------- calls
    def residual(self, U, U_lo=None, R=None, stream=None):
        self._check_state(U, U_lo)
        if R is None:
            R = self._torch.empty_like(U)
        capi.check(self._lib.weno_residual(self._h, self._p(U), self._p(U_lo), self._p(R), self._stream(stream)))
        return R

    def set_time(self, t: float, stream=None):
        capi.check(self._lib.weno_set_time(self._h, float(t), self._stream(stream)))

    def get_time(self, stream=None) -> np.ndarray:
        out = np.empty(self.n_instances)
        capi.check(self._lib.weno_get_time(self._h, _ptr(out), self._stream(stream)))
        return out

    def step(self, U, U_lo, dt: float, stream=None):
        self._check_state(U, U_lo)
        capi.check(self._lib.weno_step(self._h, self._p(U), self._p(U_lo), float(dt), self._stream(stream)))

    def step_instances(self, U, U_lo, dt_dev, stream=None):
        self._check_state(U, U_lo)
        assert dt_dev.is_cuda and dt_dev.dtype == self._torch.float64 and dt_dev.numel() == self.n_instances
        capi.check(self._lib.weno_step_instances(self._h, self._p(U), self._p(U_lo), self._p(dt_dev),
                                                 self._stream(stream)))

    def max_dt(self, U, U_lo=None, cfl=0.5, stream=None) -> np.ndarray:
        out = np.empty(self.n_instances)
        capi.check(self._lib.weno_max_dt(self._h, self._p(U), self._p(U_lo), float(cfl), _ptr(out),
                                         self._stream(stream)))
        return out

    def conservation(self, U, U_lo=None, stream=None) -> np.ndarray:
        out = np.empty(self.n_instances * self.nv)
        capi.check(self._lib.weno_conservation(self._h, self._p(U), self._p(U_lo), _ptr(out), self._stream(stream)))
        return out.reshape(self.n_instances, self.nv)

    def run_pass(self, which: int, U=None, U_lo=None, stream=None):
        """Launch one pass alone: 1 reconstruction, 2 face fluxes, 3 gather (profiling aid)."""
        capi.check(self._lib.weno_pass(self._h, int(which), self._p(U), self._p(U_lo), self._stream(stream)))

    def debug_stall(self, on: bool):
        """Testing aid: make the reconstruction's bounded waits run out (see weno_solver_debug_stall)."""
        capi.check(self._lib.weno_solver_debug_stall(self._h, 1 if on else 0))

    def check_instances(self, stream=None) -> np.ndarray:
        """Per-instance non-physical flags since the last check (cleared)."""
        out = np.zeros(self.n_instances, dtype=np.int32)
        capi.check(self._lib.weno_check_instances(self._h, _ptr(out), self._stream(stream)))
        return out

    def check(self, stream=None):
        capi.check(self._lib.weno_check(self._h, self._stream(stream)))

    def autotune(self, U, U_lo=None, stream=None):
        capi.check(self._lib.weno_autotune(self._h, self._p(U), self._p(U_lo), self._stream(stream)))

    def launch_config(self):
        cfg = np.zeros(6, dtype=np.int32)
        capi.check(self._lib.weno_solver_launch_config(self._h, _ptr(cfg)))
        return cfg

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and getattr(self, "_lib", None) is not None:
            self._lib.weno_solver_destroy(h)
            self._h = None
