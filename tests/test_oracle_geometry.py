"""Oracle geometry pinned to closed forms (Section 2 and Eq. 5)."""
import numpy as np
import pytest

import synthetic as S
from oracle.mesh import OracleMesh, polygon_area_centroid, polygon_average, GAUSS_A, GAUSS_B
from oracle.reconstruction import _polygon_monomial_averages


def test_unit_square_and_triangle_closed_forms():
    sq = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    a, c = polygon_area_centroid(sq)
    assert a == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(c, [0.5, 0.5], atol=1e-15)
    # avg x^2 = 1/3, avg xy = 1/4, avg y^2 = 1/3 on the unit square
    v = polygon_average(sq, lambda x, y: np.array([x * x, x * y, y * y]))
    assert np.allclose(v, [1 / 3, 1 / 4, 1 / 3], atol=1e-15)
    tri = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    a, c = polygon_area_centroid(tri)
    assert a == pytest.approx(0.5, abs=1e-15)
    assert np.allclose(c, [1 / 3, 1 / 3], atol=1e-15)
    # avg x^2 = 1/6, avg xy = 1/12 on the unit right triangle
    v = polygon_average(tri, lambda x, y: np.array([x * x, x * y]))
    assert np.allclose(v, [1 / 6, 1 / 12], atol=1e-15)


def test_monomial_averages_scaled_coordinates():
    # square [2,4]^2: centroid (3,3), area 4 -> s = 2, xi in [-1/2, 1/2]^2
    sq = np.array([[[2.0, 2.0], [4.0, 2.0], [4.0, 4.0], [2.0, 4.0]]])
    m = _polygon_monomial_averages(sq, np.array([4]), np.array([[3.0, 3.0]]), np.array([2.0]))
    # avg xi = 0, avg xi_x^2 = avg xi_y^2 = 1/12, avg xi_x xi_y = 0
    assert np.allclose(m[0], [0, 0, 1 / 12, 1 / 12, 0], atol=1e-15)


def test_edge_gauss_rule_is_exact_for_cubics():
    a = np.array([0.3, -1.2])
    b = np.array([2.1, 0.7])
    L = np.hypot(*(b - a))
    x1 = GAUSS_A * a + GAUSS_B * b
    x2 = GAUSS_B * a + GAUSS_A * b

    def f(p):
        return 1.0 + p[0] - 2 * p[1] + p[0] ** 3 - 3 * p[0] * p[1] ** 2

    # exact line integral by a fine composite Simpson rule on the cubic along the edge
    s = np.linspace(0.0, 1.0, 2001)
    pts = a[None] + s[:, None] * (b - a)[None]
    vals = f(pts.T)
    h = s[1] - s[0]
    exact = L * h / 3 * (vals[0] + vals[-1] + 4 * vals[1:-1:2].sum() + 2 * vals[2:-1:2].sum())
    assert L * 0.5 * (f(x1) + f(x2)) == pytest.approx(exact, rel=1e-13)


@pytest.mark.parametrize("kind", ["quad", "tri", "mixed"])
@pytest.mark.parametrize("bc_cfg", [2, 3])
def test_mesh_closure_and_counts(kind, bc_cfg):
    mi = S.mesh_for_config(bc_cfg, n=8, seed=3, kind=kind)
    m = OracleMesh.from_input(mi)
    assert m.area.min() > 0
    assert m.area.sum() == pytest.approx(mi.extent[0] * mi.extent[1], rel=1e-13)
    # every cell is closed: sum_p n_p |l_p| = 0 with outward normals
    acc = np.zeros((m.n_cells, 2))
    for f in range(m.n_faces):
        v = m.face_normal[f] * m.face_len[f]
        acc[m.face_L[f]] += v
        if m.face_R[f] >= 0:
            acc[m.face_R[f]] -= v
    assert np.abs(acc).max() < 1e-14
    n_edges_half = (3 * (m.cell_size == 3).sum() + 4 * (m.cell_size == 4).sum())
    n_bnd = int((m.face_R < 0).sum())
    assert 2 * m.n_faces - n_bnd == n_edges_half
    if mi.bc == "periodic":
        assert n_bnd == 0
        # torus: V - E + F = 0 with V = node classes
        assert len(np.unique(m.node_class)) - m.n_faces + m.n_cells == 0
    else:
        assert n_bnd == 4 * 8
        assert mi.n_nodes - m.n_faces + m.n_cells == 1


def test_cell_gauss_points_match_across_faces():
    mi = S.mesh_for_config(2, n=6, seed=1, kind="mixed")
    m = OracleMesh.from_input(mi)
    for f in range(m.n_faces):
        L, kL, R, kR = m.face_L[f], m.face_kL[f], m.face_R[f], m.face_kR[f]
        xl = m.cell_gauss[L, [2 * kL, 2 * kL + 1]]
        xr = m.cell_gauss[R, [2 * kR + 1, 2 * kR]] + m.face_shift[f]
        assert np.allclose(xl, xr, atol=1e-13)


@pytest.mark.parametrize("nx,ny", [(8, 5), (7, 6)])
def test_row_triangle_box(nx, ny):
    """Rows of near-equilateral triangles on a box: counter-clockwise, tiling the box exactly
    (areas sum to it), Euler's formula for a disc, 2 nx + 1 triangles per row, and boundary faces
    exactly on the box sides: nx on the bottom, nx or nx + 1 on the top (an odd top row holds
    nx + 2 nodes), one per row on each vertical side."""
    mi = S.tube_mesh(nx, ny, (2.0, 1.0), "rowtri")
    m = OracleMesh.from_input(mi)
    assert (m.cell_size == 3).all() and m.area.min() > 0
    assert m.area.sum() == pytest.approx(2.0, rel=1e-13)
    assert mi.n_nodes - m.n_faces + m.n_cells == 1
    assert m.n_cells == ny * (2 * nx + 1)
    top = nx if ny % 2 == 0 else nx + 1
    assert int((m.face_R < 0).sum()) == nx + top + 2 * ny
