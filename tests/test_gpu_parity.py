"""CUDA path vs the FP64 CPU oracle, through the C ABI (needs a GB300)."""
import numpy as np
import pytest

import synthetic as S
from oracle import OracleMesh, OracleSolver, Params

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1712_08317_gb300 import _capi  # noqa: E402
from paper_1712_08317_gb300.api import Mesh, Solver  # noqa: E402

# sizes span many 256-thread blocks with a ragged tail
CASES = {
    "scalar-quad": dict(cfg=1, kind="quad", n=40, eqn="scalar", init=S.scalar_wave),
    "euler-tri": dict(cfg=2, kind="tri", n=24, eqn="euler", init=S.density_wave),
    "euler-mixed": dict(cfg=2, kind="mixed", n=30, eqn="euler", init=S.density_wave),
    "riemann-outflow": dict(cfg=3, kind="mixed", n=30, eqn="euler", init=None),
    "vortex-lowq": dict(cfg=5, kind=None, n=36, eqn="euler", init=S.isentropic_vortex),
    # reflective walls on the x = 1 and y = 0 sides (corner at (1, 0)), flow towards both
    "walls-mixed": dict(cfg=3, kind="mixed", n=26, eqn="euler", init="walls", walls=(1, 2)),
}


def _walls_flow(x, y, t=0.0):
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x) * np.cos(np.pi * y)
    u, v, p = 0.5 + 0 * x, -0.4 + 0 * x, 1.0 + 0.1 * np.cos(2 * np.pi * y)
    return np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)])

# FP64 bound: states, max over cells of |W_gpu - W_oracle|_inf / |W_oracle|_inf (per-cell relative);
# residuals, max over cells of |R_gpu - R_oracle| / max_cells |R_oracle| per variable
TOL_FP64 = 1e-11


def _case(name):
    c = CASES[name]
    if c["cfg"] == 5:
        mi = S.stretched_vortex_mesh(c["n"], seed=7)
    else:
        mi = S.mesh_for_config(c["cfg"], n=c["n"], seed=7, kind=c["kind"])
    mi.walls = c.get("walls", ())
    if c["init"] is None:
        W = S.four_quadrant_average(mi, seed=7)
    elif c["init"] == "walls":
        W = S.cell_average(mi, _walls_flow)
    else:
        W = S.cell_average(mi, c["init"])
    return mi, W, c["eqn"]


_oracles = {}


def _oracle(name, linear=False, characteristic=False, optimize=True):
    key = (name, linear, characteristic, optimize)
    if key not in _oracles:
        mi, W, eqn = _case(name)
        prm = Params(eqn=eqn, linear=linear, characteristic=characteristic, optimize=optimize)
        _oracles[key] = (mi, W, OracleSolver(OracleMesh.from_input(mi), prm))
    return _oracles[key]


def _rel(a, b):
    scale = np.abs(b).max(axis=1, keepdims=True)
    scale[scale == 0] = 1.0
    return float((np.abs(a - b) / scale).max())


def _flux_scale(osol, W):
    """Per cell and variable, the magnitude of the terms its residual sums: sum_f |F_f| / |Omega_i|.
    A residual is a cancelling sum of face fluxes, so its rounding (and any faithful difference
    between two implementations) is relative to this, not to |R_i|, which can be ~0 while the
    fluxes are O(1)."""
    F = osol.face_fluxes(W)
    S_ = np.zeros_like(W)
    np.add.at(S_, (slice(None), osol.fL), np.abs(F))
    inner = ~osol.boundary
    np.add.at(S_, (slice(None), osol.fR[inner]), np.abs(F[:, inner]))
    return S_ / osol.mesh.area[None, :]


def _rel_cell(a, b):
    return float((np.abs(a - b).max(axis=0) / np.abs(b).max(axis=0)).max())


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_residual_matches_oracle(name):
    mi, W, osol = _oracle(name)
    ref = osol.residual(W)
    sol = Solver(Mesh.from_input(mi), eqn=osol.params.eqn, precision="fp64")
    U, _ = sol.to_device(W)
    R = sol.to_host(sol.residual(U))
    sol.check()
    assert _rel(R, ref) < TOL_FP64
    # cell by cell: against the cell's own flux magnitudes, and against |R_i| where the residual is
    # not a near-total cancellation (|R_i| above 1% of the largest)
    d = np.abs(R - ref)
    assert float((d / _flux_scale(osol, W)).max()) < TOL_FP64
    big = np.abs(ref) > 1e-2 * np.abs(ref).max(axis=1, keepdims=True)
    assert float((d[big] / np.abs(ref[big])).max()) < 10 * TOL_FP64


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_ten_steps_match_oracle(name):
    mi, W, osol = _oracle(name)
    dt = osol.max_dt(W, 0.5)
    ref = W
    for _ in range(10):
        ref = osol.rk3_step(ref, dt)
    sol = Solver(Mesh.from_input(mi), eqn=osol.params.eqn, precision="fp64")
    U, _ = sol.to_device(W)
    for _ in range(10):
        sol.step(U, None, dt)
    torch.cuda.synchronize()
    sol.check()
    assert _rel_cell(sol.to_host(U), ref) < TOL_FP64


@pytest.mark.parametrize("name", ["scalar-quad", "euler-mixed"])
def test_linear_scheme_matches_oracle(name):
    mi, W, osol = _oracle(name, linear=True)
    ref = osol.residual(W)
    sol = Solver(Mesh.from_input(mi), eqn=osol.params.eqn, precision="fp64", linear=True)
    U, _ = sol.to_device(W)
    assert _rel(sol.to_host(sol.residual(U)), ref) < TOL_FP64


@pytest.mark.parametrize("name", ["euler-mixed", "vortex-lowq", "riemann-outflow", "scalar-quad", "euler-tri",
                                  "walls-mixed"])
def test_fp32c_tracks_the_oracle(name):
    """FP32 reconstruction / weights / flux with a compensated state: FP32-level agreement."""
    mi, W, osol = _oracle(name)
    ref_R = osol.residual(W)
    dt = osol.max_dt(W, 0.5)
    ref = W
    for _ in range(10):
        ref = osol.rk3_step(ref, dt)
    sol = Solver(Mesh.from_input(mi), eqn=osol.params.eqn, precision="fp32c")
    U, Ul = sol.to_device(W)
    R = sol.to_host(sol.residual(U, Ul))
    # the residual is a difference of O(1) fluxes divided by |Omega|: FP32 rounding of the
    # fluxes, amplified by the cancellation, bounds it
    assert _rel(R, ref_R) < 2e-3
    for _ in range(10):
        sol.step(U, Ul, dt)
    torch.cuda.synchronize()
    sol.check()
    assert _rel_cell(sol.to_host(U, Ul), ref) < 2e-6


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32c", 1e-12)])
def test_conservation_on_periodic_mesh(precision, tol):
    mi, W, osol = _oracle("vortex-lowq")
    sol = Solver(Mesh.from_input(mi), eqn="euler", precision=precision)
    U, Ul = sol.to_device(W)
    c0 = sol.conservation(U, Ul)[0]
    dt = sol.max_dt(U, Ul, 0.5)[0]
    for _ in range(20):
        sol.step(U, Ul, dt)
    c1 = sol.conservation(U, Ul)[0]
    assert np.abs(c1 - c0).max() <= tol * np.abs(c0).max()
    # the FP64 sums agree with the oracle's definition sum |Omega| W
    assert np.allclose(c0, osol.conservation(W), rtol=1e-12)


def test_max_dt_matches_oracle():
    for name in ("euler-mixed", "scalar-quad", "riemann-outflow"):
        mi, W, osol = _oracle(name)
        sol = Solver(Mesh.from_input(mi), eqn=osol.params.eqn, precision="fp64")
        U, _ = sol.to_device(W)
        assert sol.max_dt(U, None, 0.5)[0] == pytest.approx(osol.max_dt(W, 0.5), rel=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_batched_instances_equal_standalone_runs(precision):
    """One flattened launch over uneven instances with per-instance dt == separate solvers."""
    insts = [S.mesh_for_config(2, n=13, seed=1, kind="mixed"), S.mesh_for_config(3, n=17, seed=2, kind="tri"),
             S.mesh_for_config(2, n=9, seed=3, kind="quad")]
    inits = [S.cell_average(insts[0], S.density_wave), S.four_quadrant_average(insts[1], 2),
             S.cell_average(insts[2], S.density_wave)]
    meshes = [Mesh.from_input(m) for m in insts]
    singles = [Solver(m, eqn="euler", precision=precision) for m in meshes]
    states = [s.to_device(w) for s, w in zip(singles, inits)]
    dts = [s.max_dt(U, Ul, 0.4)[0] for s, (U, Ul) in zip(singles, states)]
    for s, (U, Ul), dt in zip(singles, states, dts):
        for _ in range(4):
            s.step(U, Ul, dt)
    big = Solver(Mesh.concat(meshes), eqn="euler", precision=precision)
    Wcat = np.concatenate(inits, axis=1)
    U, Ul = big.to_device(Wcat)
    dt_dev = torch.tensor(dts, dtype=torch.float64, device="cuda")
    for _ in range(4):
        big.step_instances(U, Ul, dt_dev)
    torch.cuda.synchronize()
    out = big.to_host(U, Ul)
    off = 0
    for s, (Ui, Uli), m in zip(singles, states, insts):
        ref = s.to_host(Ui, Uli)
        assert np.array_equal(out[:, off:off + m.n_cells], ref)
        off += m.n_cells


@pytest.mark.parametrize("characteristic", [False, True])
def test_batched_instances_with_walls_equal_standalone_runs(characteristic):
    """Instances with and without reflective walls in one launch == separate solvers (FP32C)."""
    a = S.mesh_for_config(3, n=11, seed=4, kind="mixed")
    a.walls = (0, 3)
    b = S.mesh_for_config(2, n=9, seed=5, kind="tri")
    insts = [a, b]
    inits = [S.cell_average(a, _walls_flow), S.cell_average(b, S.density_wave)]
    meshes = [Mesh.from_input(m) for m in insts]
    singles = [Solver(m, eqn="euler", precision="fp32c", characteristic=characteristic) for m in meshes]
    states = [s.to_device(w) for s, w in zip(singles, inits)]
    dts = [s.max_dt(U, Ul, 0.4)[0] for s, (U, Ul) in zip(singles, states)]
    for s, (U, Ul), dt in zip(singles, states, dts):
        for _ in range(3):
            s.step(U, Ul, dt)
    big = Solver(Mesh.concat(meshes), eqn="euler", precision="fp32c", characteristic=characteristic)
    U, Ul = big.to_device(np.concatenate(inits, axis=1))
    dt_dev = torch.tensor(dts, dtype=torch.float64, device="cuda")
    for _ in range(3):
        big.step_instances(U, Ul, dt_dev)
    torch.cuda.synchronize()
    out = big.to_host(U, Ul)
    off = 0
    for s, (Ui, Uli), m in zip(singles, states, insts):
        assert np.array_equal(out[:, off:off + m.n_cells], s.to_host(Ui, Uli))
        off += m.n_cells


def test_nonphysical_state_is_reported_and_cleared():
    mi, W, _ = _oracle("euler-mixed")
    sol = Solver(Mesh.from_input(mi), eqn="euler", precision="fp64")
    Wbad = W.copy()
    Wbad[0, 5] = -0.1
    U, _ = sol.to_device(Wbad)
    sol.residual(U)
    with pytest.raises(_capi.WenoError) as e:
        sol.check()
    assert e.value.code == _capi.WENO_ENONPHYS
    U, _ = sol.to_device(W)
    sol.residual(U)
    sol.check()


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_nonphysical_flags_name_the_instance(precision):
    mi, W, _ = _oracle("euler-mixed")
    m = Mesh.from_input(mi)
    big = Solver(Mesh.concat([m, m, m]), eqn="euler", precision=precision)
    Wcat = np.concatenate([W, W, W], axis=1)
    Wcat[3, W.shape[1] + 17] = -0.5       # negative energy in one cell of instance 1
    U, Ul = big.to_device(Wcat)
    big.residual(U, Ul)
    assert big.check_instances().tolist() == [0, 1, 0]
    assert big.check_instances().tolist() == [0, 0, 0]   # cleared
    big.residual(U, Ul)
    with pytest.raises(_capi.WenoError) as e:
        big.check()
    assert e.value.code == _capi.WENO_ENONPHYS and "1 of 3" in str(e.value)


@pytest.mark.parametrize("characteristic", [False, True])
def test_bounded_wait_reports_timeout_and_context_survives(characteristic):
    mi, W, _ = _oracle("euler-mixed")
    sol = Solver(Mesh.from_input(mi), eqn="euler", precision="fp32c", characteristic=characteristic)
    U, Ul = sol.to_device(W)
    R0 = sol.residual(U, Ul).clone()
    sol.check()
    sol.debug_stall(True)          # barriers expect an arrival nobody makes: every wait runs out (1 s)
    sol.residual(U, Ul)
    with pytest.raises(_capi.WenoError) as e:
        sol.check()
    assert e.value.code == _capi.WENO_ETIMEOUT
    sol.debug_stall(False)
    R1 = sol.residual(U, Ul)
    sol.check()
    assert torch.equal(R0, R1)     # the context is still usable and the results are unchanged
    sol64 = Solver(Mesh.from_input(mi), eqn="euler", precision="fp64")
    with pytest.raises(_capi.WenoError) as e:
        sol64.debug_stall(True)
    assert e.value.code == _capi.WENO_EINVAL


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_autotune_does_not_change_results(precision):
    mi, W, _ = _oracle("euler-mixed")
    sol = Solver(Mesh.from_input(mi), eqn="euler", precision=precision)
    U, Ul = sol.to_device(W)
    R0 = sol.residual(U, Ul).clone()
    sol.autotune(U, Ul)
    R1 = sol.residual(U, Ul)
    assert torch.equal(R0, R1)
    cfg = sol.launch_config()
    assert cfg[0] in (32, 64, 128, 256)


def test_invalid_arguments_return_codes():
    mi, W, _ = _oracle("euler-mixed")
    sol = Solver(Mesh.from_input(mi), eqn="euler", precision="fp32c")
    U, Ul = sol.to_device(W)
    lib = _capi.load()
    import ctypes
    # FP32C needs the compensation array
    assert lib.weno_step(sol._h, ctypes.c_void_p(U.data_ptr()), None, 0.1, None) == _capi.WENO_EINVAL
    assert lib.weno_step(sol._h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(Ul.data_ptr()), -1.0, None) == \
        _capi.WENO_EINVAL
    # characteristic variables are defined for the Euler equations only; theta < 1 and eps <= 0 are rejected
    mesh = Mesh.from_input(mi)
    for bad in (dict(eqn="scalar", characteristic=True), dict(theta=0.5), dict(eps=0.0)):
        with pytest.raises(_capi.WenoError) as e:
            Solver(mesh, precision="fp32c", **bad)
        assert e.value.code == _capi.WENO_EINVAL


EULER_CASES = [n for n in CASES if CASES[n]["eqn"] == "euler"]


@pytest.mark.parametrize("name", EULER_CASES)
def test_characteristic_fp64_residual_and_steps_match_oracle(name):
    """Characteristic-variable reconstruction (Section 4), FP64: residual and 10 RK3 steps."""
    mi, W, osol = _oracle(name, characteristic=True)
    sol = Solver(Mesh.from_input(mi), eqn="euler", precision="fp64", characteristic=True)
    U, _ = sol.to_device(W)
    assert _rel(sol.to_host(sol.residual(U)), osol.residual(W)) < TOL_FP64
    dt = osol.max_dt(W, 0.5)
    ref = W
    for _ in range(10):
        ref = osol.rk3_step(ref, dt)
    for _ in range(10):
        sol.step(U, None, dt)
    torch.cuda.synchronize()
    sol.check()
    assert _rel_cell(sol.to_host(U), ref) < TOL_FP64


@pytest.mark.parametrize("name", ["euler-mixed", "riemann-outflow", "vortex-lowq", "walls-mixed"])
def test_characteristic_fp32c_tracks_the_oracle(name):
    mi, W, osol = _oracle(name, characteristic=True)
    sol = Solver(Mesh.from_input(mi), eqn="euler", precision="fp32c", characteristic=True)
    U, Ul = sol.to_device(W)
    assert _rel(sol.to_host(sol.residual(U, Ul)), osol.residual(W)) < 2e-3
    dt = osol.max_dt(W, 0.5)
    ref = W
    for _ in range(10):
        ref = osol.rk3_step(ref, dt)
    for _ in range(10):
        sol.step(U, Ul, dt)
    torch.cuda.synchronize()
    sol.check()
    assert _rel_cell(sol.to_host(U, Ul), ref) < 2e-6


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32c", 1e-12)])
def test_characteristic_conserves_and_keeps_constant_states(precision, tol):
    mi, W, _ = _oracle("euler-mixed")
    sol = Solver(Mesh.from_input(mi), eqn="euler", precision=precision, characteristic=True)
    U, Ul = sol.to_device(W)
    c0 = sol.conservation(U, Ul)[0]
    dt = sol.max_dt(U, Ul, 0.5)[0]
    for _ in range(5):
        sol.step(U, Ul, dt)
    torch.cuda.synchronize()
    sol.check()
    c1 = sol.conservation(U, Ul)[0]
    assert np.abs(c1 - c0).max() <= tol * np.abs(c0).max()
    Wc = np.repeat(np.array([[1.2], [0.3], [-0.4], [2.9]]), W.shape[1], axis=1)
    U, Ul = sol.to_device(Wc)
    R = sol.to_host(sol.residual(U, Ul))
    assert np.abs(R).max() < (1e-12 if precision == "fp64" else 1e-4)  # face closure rounding only


def test_raw_linear_weights_on_the_low_quality_mesh_are_flagged_like_the_oracle():
    """Without Section 3.3 the weights on the aspect-ratio-10 vortex mesh are large enough that
    the very first reconstruction has negative pressure or density at some Gauss points: the
    oracle raises and both GPU precisions report WENO_ENONPHYS."""
    from oracle.scheme import NonPhysicalState
    mi, W, osol = _oracle("vortex-lowq", optimize=False)
    with pytest.raises(NonPhysicalState):
        osol.residual(W)
    for precision in ("fp64", "fp32c"):
        sol = Solver(Mesh.from_input(mi), eqn="euler", precision=precision, optimize=False)
        U, Ul = sol.to_device(W)
        sol.residual(U, Ul)
        with pytest.raises(_capi.WenoError) as e:
            sol.check()
        assert e.value.code == _capi.WENO_ENONPHYS


@pytest.mark.parametrize("name", ["euler-mixed", "scalar-quad", "riemann-outflow"])
def test_raw_linear_weights_match_oracle(name):
    """Section 3.3 switched off (raw minimum-norm weights, which reach large values on
    low-quality meshes): FP64 residual and FP32C tracking."""
    mi, W, osol = _oracle(name, optimize=False)
    ref = osol.residual(W)
    eqn = osol.params.eqn
    # the two sides' minimum-norm solves differ at rounding level; the raw weights multiply
    # that difference by their size (max |gamma| 552 raw vs 6.8 optimised on the split meshes)
    raw, opt = Mesh.from_input(mi).weight_stats()
    tol = TOL_FP64 * max(1.0, raw.max() / opt.max())
    sol = Solver(Mesh.from_input(mi), eqn=eqn, precision="fp64", optimize=False)
    U, _ = sol.to_device(W)
    assert _rel(sol.to_host(sol.residual(U)), ref) < tol
    s32 = Solver(Mesh.from_input(mi), eqn=eqn, precision="fp32c", optimize=False)
    U, Ul = s32.to_device(W)
    assert _rel(s32.to_host(s32.residual(U, Ul)), ref) < 2e-3



# ---------------------------------------------------------------- inflow sides, partial wall, moving state
def _inflow_case(kind="mixed", n=12):
    """A small double-Mach-like box: a Mach 2.5 shock at 60 degrees through (0.3, 0) running into
    gas at rest; bottom wall from x = 0.5, prescribed moving-shock state on the left, the rest of the
    bottom and the top, outflow on the right.  Within 10 steps the shock crosses top-side Gauss
    points, so the stage times decide some boundary states."""
    sh = S.moving_shock(2.5, 0.3, 0.0, 60.0)
    mi = S.tube_mesh(3 * n, n, (3.0, 1.0), kind, delta=0.1, seed=9, walls=(2,), wall_from=(0, 0, 0.5, 0),
                     inflow=(0, 2, 3))
    W = S.cell_average(mi, sh["f"])
    prm = dict(inflow_a=sh["post"], inflow_b=sh["pre"], inflow_line=sh["line"])
    return mi, W, prm


@pytest.mark.parametrize("characteristic", [False, True])
@pytest.mark.parametrize("kind", ["mixed", "quad"])
def test_inflow_fp64_residual_and_steps_match_oracle(kind, characteristic):
    mi, W, prm = _inflow_case(kind)
    osol = OracleSolver(OracleMesh.from_input(mi), Params(characteristic=characteristic, **prm))
    t0 = 0.013
    dt = osol.max_dt(W, 0.5)
    sol = Solver(Mesh.from_input(mi), eqn="euler", precision="fp64", characteristic=characteristic, **prm)
    assert sol.mesh.info.n_inflow == int(osol.mesh.face_inflow.sum())
    sol.set_time(t0)
    U, _ = sol.to_device(W)
    assert _rel(sol.to_host(sol.residual(U)), osol.residual(W, t=t0)) < TOL_FP64
    ref, t = W, t0
    for _ in range(10):
        ref = osol.rk3_step(ref, dt, t=t)
        t += dt
    for _ in range(10):
        sol.step(U, None, dt)
    torch.cuda.synchronize()
    sol.check()
    assert _rel_cell(sol.to_host(U), ref) < TOL_FP64
    assert sol.get_time()[0] == t
    # the boundary state did move: the same steps with the time frozen at t0 differ
    frozen = W
    for _ in range(10):
        frozen = osol.rk3_step(frozen, dt, t=t0)
    assert _rel_cell(frozen, ref) > 1e-3


@pytest.mark.parametrize("characteristic", [False, True])
def test_inflow_fp32c_tracks_the_oracle(characteristic):
    mi, W, prm = _inflow_case("mixed")
    osol = OracleSolver(OracleMesh.from_input(mi), Params(characteristic=characteristic, **prm))
    dt = osol.max_dt(W, 0.5)
    sol = Solver(Mesh.from_input(mi), eqn="euler", precision="fp32c", characteristic=characteristic, **prm)
    U, Ul = sol.to_device(W)
    assert _rel(sol.to_host(sol.residual(U, Ul)), osol.residual(W)) < 2e-3
    ref, t = W, 0.0
    for _ in range(10):
        ref = osol.rk3_step(ref, dt, t=t)
        t += dt
    for _ in range(10):
        sol.step(U, Ul, dt)
    torch.cuda.synchronize()
    sol.check()
    assert _rel_cell(sol.to_host(U, Ul), ref) < 2e-6


def test_batched_instances_with_inflow_keep_their_own_time():
    """An inflow instance batched with a periodic one, different dt per instance, equals standalone
    runs bit for bit (FP32C), and each instance's time advances by its own dt."""
    a, wa, prm = _inflow_case("mixed", n=8)
    b = S.mesh_for_config(2, n=9, seed=5, kind="tri")
    wb = S.cell_average(b, S.density_wave)
    meshes = [Mesh.from_input(a), Mesh.from_input(b)]
    singles = [Solver(m, eqn="euler", precision="fp32c", **prm) for m in meshes]
    states = [s.to_device(w) for s, w in zip(singles, (wa, wb))]
    dts = [s.max_dt(U, Ul, 0.4)[0] for s, (U, Ul) in zip(singles, states)]
    for s, (U, Ul), dt in zip(singles, states, dts):
        for _ in range(4):
            s.step(U, Ul, dt)
    big = Solver(Mesh.concat(meshes), eqn="euler", precision="fp32c", **prm)
    U, Ul = big.to_device(np.concatenate([wa, wb], axis=1))
    dt_dev = torch.tensor(dts, dtype=torch.float64, device="cuda")
    for _ in range(4):
        big.step_instances(U, Ul, dt_dev)
    torch.cuda.synchronize()
    out = big.to_host(U, Ul)
    assert np.array_equal(out[:, :a.n_cells], singles[0].to_host(*states[0]))
    assert np.array_equal(out[:, a.n_cells:], singles[1].to_host(*states[1]))
    t = big.get_time()
    assert t[0] == dts[0] + dts[0] + dts[0] + dts[0] and t[1] == dts[1] + dts[1] + dts[1] + dts[1]


@pytest.mark.parametrize("characteristic", [False, True])
@pytest.mark.parametrize("shape,size", [("ramp", 1e5), ("ramp", 1e7), ("step", 1e4), ("step", 1e5),
                                        ("rho_ramp", 1e5), ("rho_ramp", 1e7)])
def test_fp32c_weights_stay_finite_at_huge_indicators(shape, size, characteristic):
    """Section 3.4's alpha = gamma / (beta~ + eps)^2 with beta~ ~ gamma^2 beta^3: a steep pressure
    ramp makes every candidate's beta ~ 1e8-1e12, so (beta~ + eps)^2 overflows FP32 and every alpha
    of a group flushes to zero; a strong step puts such indicators next to smooth candidates.  In
    characteristic variables an isentropic-like pressure ramp projects to O(1) differences
    (dp / c^2), so an isothermal density ramp (p = rho, moving at Mach ~0.9: the entropy field
    carries (1 - 1/gamma) d rho) does the same there, and most cells take the FP64 fix-up.  The
    FP32C path (component-wise and characteristic) must still match the oracle (FP64) to FP32
    accuracy, with no NaN."""
    mi = S.mesh_for_config(3, n=14, seed=2, kind="mixed")
    om = OracleMesh.from_input(mi)
    cen = om.centroid
    rho, u, v = np.ones(len(cen)), np.zeros(len(cen)), np.zeros(len(cen))
    if shape == "ramp":
        p = 1.0 + size * (cen[:, 0] + 0.3 * cen[:, 1])
    elif shape == "step":
        p = np.where(cen[:, 0] + 0.3 * cen[:, 1] < 0.55, size, 1.0)
    else:
        rho = 1.0 + size * (cen[:, 0] + 0.3 * cen[:, 1])
        p, u, v = rho, u + 1.0, v + 0.5
    W = S.euler_prim_to_cons(rho, u, v, p, 1.4)
    ref = OracleSolver(om, Params(characteristic=characteristic)).residual(W)
    sol = Solver(Mesh.from_input(mi), eqn="euler", precision="fp32c", characteristic=characteristic)
    U, Ul = sol.to_device(W)
    Rd = sol.residual(U, Ul)
    assert bool(torch.isfinite(Rd).all())
    sol.check()
    assert _rel(sol.to_host(Rd), ref) < 2e-3
