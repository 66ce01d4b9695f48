"""weno_residual_static: the residual with its scratch in the library's fixed array.

It serves callers that may not allocate device memory once running (a
memory budget fixed at start-up, or a step loop that may not make allocation
calls).  Checked through the C ABI against weno_residual, on two calls in a
row, with another solver's call in between to show that leftover contents of
the shared array do not leak into a result.
"""
import ctypes

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1712_08317_gb300 import _capi  # noqa: E402
from paper_1712_08317_gb300.api import Mesh, Solver  # noqa: E402

TOL = 1e-11  # same relative bound as the FP64 parity tests; FP32C compared at FP32 rounding


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _static(sol, U, Ul, R):
    lib = _capi.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.weno_residual_static(sol._h, _p(U), _p(Ul), _p(R), stream)


def _regular(sol, U, Ul, R):
    lib = _capi.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.weno_residual(sol._h, _p(U), _p(Ul), _p(R), stream)


def _close(a, b, precision):
    scale = b.abs().max().item()
    tol = TOL if precision == "fp64" else 1e-6
    return (a - b).abs().max().item() <= tol * scale


def _density_ramp(x, y):
    """Density rising by 1e7 per unit length at temperature p / rho = 1, moving at (1, 0.5): the
    entropy field's indicators are ~1e11, so their sums of alpha leave the FP32 range and the
    characteristic path marks most cells for its FP64 fix-up."""
    rho = 1.0 + 1e7 * (x + 0.3 * y)
    one = np.ones_like(rho)
    return S.euler_prim_to_cons(rho, one, 0.5 * one, rho, 1.4)


@pytest.mark.parametrize("precision,characteristic,init", [
    ("fp64", False, "wave"), ("fp32c", False, "wave"), ("fp32c", True, "wave"), ("fp32c", True, "ramp")])
def test_static_scratch_residual_matches_weno_residual(precision, characteristic, init):
    mi = S.mesh_for_config(2, n=30, seed=5, kind="mixed")
    W = S.cell_average(mi, S.density_wave if init == "wave" else _density_ramp)
    sol = Solver(Mesh.from_input(mi), eqn="euler", precision=precision, characteristic=characteristic)
    U, Ul = sol.to_device(W)
    ref = torch.empty_like(U)
    assert _regular(sol, U, Ul, ref) == 0
    # a second solver on another mesh writes different contents into the shared array
    mi2 = S.mesh_for_config(3, n=20, seed=6, kind="tri")
    sol2 = Solver(Mesh.from_input(mi2), eqn="euler", precision=precision, characteristic=characteristic)
    U2, Ul2 = sol2.to_device(S.four_quadrant_average(mi2, 6))
    for _ in range(2):
        R = torch.full_like(U, float("nan"))
        assert _static(sol, U, Ul, R) == 0, _capi.load().weno_last_error()
        torch.cuda.synchronize()
        assert _close(R, ref, precision)
        if precision == "fp32c":  # the same kernels on the same inputs
            assert torch.equal(R, ref)
        R2 = torch.empty_like(U2)
        assert _static(sol2, U2, Ul2, R2) == 0
        torch.cuda.synchronize()
    sol.check()


def test_static_scratch_rejects_meshes_above_the_limit():
    mi = S.mesh_for_config(2, n=200, seed=1, kind="tri")   # 80,000 triangles, 120,000 faces
    mesh = Mesh.from_input(mi)
    need = (6 * mesh.info.n_tris * 4 + mesh.info.n_faces * 4) * 8
    assert need > 16 << 20
    sol = Solver(mesh, eqn="euler", precision="fp64")
    U, _ = sol.to_device(np.ones((4, mi.n_cells)) * np.array([[1.0], [0.1], [0.1], [2.5]]))
    R = torch.zeros_like(U)
    assert _static(sol, U, None, R) == _capi.WENO_EINVAL
    assert b"too large" in _capi.load().weno_last_error()
    assert torch.count_nonzero(R).item() == 0
