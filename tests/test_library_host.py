"""The C-ABI library on the host: loads, exports include/weno3.h, host mesh logic vs the oracle.

No compute call touches a GPU here: mesh building and the FP64 precompute
diagnostics run on the host inside the library.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import synthetic as S
from oracle import OracleMesh, Params, precompute

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1712_08317_gb300 import _capi
    return _capi.load()


def test_library_exports_every_declared_symbol(lib):
    header = open(os.path.join(ROOT, "include", "weno3.h")).read()
    declared = set(re.findall(r"^(?:int|void|const char\*)\s+(weno_[a-z0-9_]+)\s*\(", header, re.M))
    assert len(declared) >= 18
    so = ctypes.CDLL(lib._name)
    for name in sorted(declared):
        assert hasattr(so, name), name
    from paper_1712_08317_gb300 import _capi
    assert declared == set(_capi.SIGNATURES), declared ^ set(_capi.SIGNATURES)


@pytest.mark.parametrize("cfg,kind,n", [(1, "quad", 9), (2, "tri", 8), (2, "mixed", 10), (3, "mixed", 10), (3, "tri", 7)])
def test_mesh_counts_and_permutation(cfg, kind, n):
    from paper_1712_08317_gb300.api import Mesh
    mi = S.mesh_for_config(cfg, n=n, seed=2, kind=kind)
    m = Mesh.from_input(mi)
    om = OracleMesh.from_input(mi)
    assert m.info.n_cells == mi.n_cells
    assert m.info.n_faces == om.n_faces
    assert m.info.n_boundary == int((om.face_R < 0).sum())
    assert sorted(m.perm.tolist()) == list(range(mi.n_cells))
    # internal order: quads first
    sizes = mi.cell_sizes()[m.perm]
    assert np.all(sizes[:m.info.n_quads] == 4) and np.all(sizes[m.info.n_quads:] == 3)


@pytest.mark.parametrize("cfg,kind", [(1, "quad"), (2, "tri"), (2, "mixed"), (3, "mixed")])
def test_host_precompute_matches_oracle_weights(cfg, kind):
    """The library's own FP64 precompute (Jacobi SVD, Green moments) vs the oracle's (pinv, midpoint rule)."""
    from paper_1712_08317_gb300.api import Mesh
    mi = S.mesh_for_config(cfg, n=9, seed=4, kind=kind)
    m = Mesh.from_input(mi)
    raw, opt = m.weight_stats()
    groups = precompute(OracleMesh.from_input(mi), Params())
    oraw = np.zeros(mi.n_cells)
    oopt = np.zeros(mi.n_cells)
    for t in groups:
        oraw[t.cells] = np.abs(t.gamma_raw).max(axis=(1, 2))
        oopt[t.cells] = np.abs(t.gamma).max(axis=(1, 2))
    assert np.allclose(raw, oraw[m.perm], rtol=1e-10, atol=1e-12)
    assert np.allclose(opt, oopt[m.perm], rtol=1e-10, atol=1e-12)


def test_batched_mesh_offsets():
    from paper_1712_08317_gb300.api import Mesh
    a = S.mesh_for_config(2, n=6, seed=1, kind="mixed")
    b = S.mesh_for_config(3, n=5, seed=2, kind="tri")
    ma, mb = Mesh.from_input(a), Mesh.from_input(b)
    m = Mesh.concat([ma, mb])
    assert m.info.n_instances == 2
    assert m.n_cells == a.n_cells + b.n_cells
    assert m.info.n_faces == ma.info.n_faces + mb.info.n_faces
    assert sorted(m.perm.tolist()) == list(range(m.n_cells))
    inst_of_input = np.empty(m.n_cells, int)
    inst_of_input[m.perm] = m.instance
    assert np.all(inst_of_input[:a.n_cells] == 0) and np.all(inst_of_input[a.n_cells:] == 1)
    raw, opt = m.weight_stats()
    ra, oa = ma.weight_stats()
    # same per-cell statistics as the standalone instance
    gid = np.empty(a.n_cells, int)
    gid[:] = -1
    for internal, inp in enumerate(m.perm):
        if inp < a.n_cells:
            gid[inp] = internal
    assert np.array_equal(opt[gid[ma.perm]], oa)


def _quad_mesh(nodes, cells, bc="outflow"):
    return dict(nodes=np.array(nodes, float), cell_ptr=np.arange(0, 4 * len(cells) + 1, 4),
                cell_nodes=np.array(cells).ravel(), bc=bc)


def test_invalid_meshes_are_rejected_with_codes():
    from paper_1712_08317_gb300 import _capi
    from paper_1712_08317_gb300.api import Mesh
    sq = [[0, 0], [1, 0], [1, 1], [0, 1], [0.4, 0.6]]
    with pytest.raises(_capi.WenoError) as e:   # non-convex quad (reflex at node 4)
        Mesh(**_quad_mesh(sq, [[0, 1, 4, 3]]))
    assert e.value.code == _capi.WENO_EMESH
    with pytest.raises(_capi.WenoError) as e:   # pentagon
        Mesh(np.array(sq, float), [0, 5], [0, 1, 2, 3, 4], "outflow")
    assert e.value.code == _capi.WENO_EMESH
    with pytest.raises(_capi.WenoError) as e:   # zero area
        Mesh(np.array([[0, 0], [1, 0], [2, 0]], float), [0, 3], [0, 1, 2], "outflow")
    assert e.value.code == _capi.WENO_EMESH
    mi = S.mesh_for_config(1, n=5)
    with pytest.raises(_capi.WenoError) as e:   # wrong period: boundaries do not pair
        Mesh(mi.nodes, mi.cell_ptr, mi.cell_nodes, "periodic", (0.0, 0.0), (2.5, 2.0))
    assert e.value.code == _capi.WENO_EPERIODIC
    with pytest.raises(_capi.WenoError) as e:
        Mesh(mi.nodes, mi.cell_ptr, np.where(mi.cell_nodes == 0, 10 ** 9, mi.cell_nodes), "periodic", (0, 0), (2, 2))
    assert e.value.code == _capi.WENO_EINVAL


def test_clockwise_cells_are_reoriented():
    from paper_1712_08317_gb300.api import Mesh
    mi = S.mesh_for_config(3, n=6, seed=3, kind="mixed")
    cn = mi.cell_nodes.copy()
    for c in range(0, mi.n_cells, 2):
        a, b = mi.cell_ptr[c], mi.cell_ptr[c + 1]
        cn[a:b] = cn[a:b][::-1]
    m1 = Mesh.from_input(mi)
    m2 = Mesh(mi.nodes, mi.cell_ptr, cn, mi.bc, mi.origin, mi.extent)
    assert np.array_equal(m1.perm, m2.perm)
    assert np.array_equal(m1.weight_stats()[1], m2.weight_stats()[1])


def test_wall_options_are_validated(lib):
    """Reflective walls name sides of an outflow box (bits 0-3); anything else is rejected."""
    from paper_1712_08317_gb300 import _capi
    from paper_1712_08317_gb300.api import Mesh
    mi = S.mesh_for_config(3, n=6, seed=1, kind="mixed")
    m = Mesh(mi.nodes, mi.cell_ptr, mi.cell_nodes, "outflow", (0.0, 0.0), (1.0, 1.0), walls=(0, 3))
    assert m.n_cells == mi.n_cells
    for bc, walls, extent in (("periodic", (1,), (1.0, 1.0)), ("outflow", (4,), (1.0, 1.0)),
                              ("outflow", (1,), (0.0, 1.0))):
        with pytest.raises(_capi.WenoError) as e:
            Mesh(mi.nodes, mi.cell_ptr, mi.cell_nodes, bc, (0.0, 0.0), extent, walls=walls)
        assert e.value.code == _capi.WENO_EINVAL


@pytest.mark.parametrize("kind", ["quad", "mixed", "tri"])
def test_inflow_faces_and_partial_walls_match_the_oracle(kind):
    """Inflow sides and walls starting part-way along a side classify the same faces as the oracle."""
    from paper_1712_08317_gb300.api import Mesh
    for walls, wall_from, inflow in (((2,), (0, 0, 0.25, 0), (0, 2, 3)), ((), (0, 0, 0, 0), (1,)),
                                     ((0, 2), (0.1, 0, 0.5, 0), (0, 1, 2, 3))):
        mi = S.tube_mesh(20, 6, (1.0, 0.3), kind, delta=0.1, seed=4, walls=walls, wall_from=wall_from, inflow=inflow)
        om = OracleMesh.from_input(mi)
        m = Mesh.from_input(mi)
        assert m.info.n_inflow == int(om.face_inflow.sum()) > 0
        assert m.info.n_boundary == int((om.face_R < 0).sum())


def test_inflow_options_are_validated(lib):
    from paper_1712_08317_gb300 import _capi
    from paper_1712_08317_gb300.api import Mesh
    mi = S.mesh_for_config(3, n=6, seed=1, kind="mixed")
    for bc, inflow, wall_from in (("periodic", (1,), (0, 0, 0, 0)), ("outflow", (5,), (0, 0, 0, 0)),
                                  ("outflow", (1,), (0, float("nan"), 0, 0))):
        with pytest.raises(_capi.WenoError) as e:
            Mesh(mi.nodes, mi.cell_ptr, mi.cell_nodes, bc, (0.0, 0.0), (1.0, 1.0), inflow=inflow, wall_from=wall_from)
        assert e.value.code == _capi.WENO_EINVAL


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_solver_create_rejects_theta_at_most_one(lib, theta):
    """The splitting of Section 3.4 needs theta > 1 (sigma- > 0); the check precedes any CUDA call."""
    from paper_1712_08317_gb300 import _capi
    from paper_1712_08317_gb300.api import Mesh, params_struct
    m = Mesh.from_input(S.mesh_for_config(1, n=6, seed=0))
    p = params_struct(theta=theta)
    h = ctypes.c_void_p()
    assert lib.weno_solver_create(m._h, ctypes.byref(p), None, ctypes.byref(h)) == _capi.WENO_EINVAL
    assert b"theta" in lib.weno_last_error()
    with pytest.raises(ValueError):
        Params(theta=theta)


def test_fp32c_solver_needs_eps_of_at_least_1e_15(lib):
    """FP32 nonlinear weights alpha = gamma / (beta~ + eps)^2 <= 1 / eps^2 must stay inside the FP32
    range: FP32C solvers reject eps < 1e-15 (before any CUDA call); FP64 solvers take any eps > 0."""
    from paper_1712_08317_gb300 import _capi
    from paper_1712_08317_gb300.api import Mesh, params_struct
    m = Mesh.from_input(S.mesh_for_config(1, n=6, seed=0))
    h = ctypes.c_void_p()
    p = params_struct(precision="fp32c", eps=1e-20)
    assert lib.weno_solver_create(m._h, ctypes.byref(p), None, ctypes.byref(h)) == _capi.WENO_EINVAL
    assert b"1e-15" in lib.weno_last_error()


def test_host_precompute_matches_oracle_on_row_triangles_with_walls():
    """The same comparison on rows of near-equilateral triangles (every node of valence 6 inside,
    half-width triangles on the sides) in a box with a partial wall and inflow sides, the double
    Mach reflection's boundary layout."""
    from paper_1712_08317_gb300.api import Mesh
    mi = S.tube_mesh(12, 8, (2.0, 1.0), "rowtri", walls=(2,), wall_from=(0, 0, 1.0 / 3.0, 0), inflow=(0, 2, 3))
    m = Mesh.from_input(mi)
    raw, opt = m.weight_stats()
    groups = precompute(OracleMesh.from_input(mi), Params())
    oraw = np.zeros(mi.n_cells)
    oopt = np.zeros(mi.n_cells)
    for t in groups:
        oraw[t.cells] = np.abs(t.gamma_raw).max(axis=(1, 2))
        oopt[t.cells] = np.abs(t.gamma).max(axis=(1, 2))
    assert np.allclose(raw, oraw[m.perm], rtol=1e-10, atol=1e-12)
    assert np.allclose(opt, oopt[m.perm], rtol=1e-10, atol=1e-12)
