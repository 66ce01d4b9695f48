"""Oracle nonlinear weights (Section 3.4) pinned by invariants and limiting cases."""
import dataclasses

import numpy as np

import synthetic as S
from oracle import OracleMesh, Params, precompute
from oracle.weno import gauss_values_group


def _case(kind="mixed", n=8, cfg=2, seed=4):
    mi = S.mesh_for_config(cfg, n=n, seed=seed, kind=kind)
    mesh = OracleMesh.from_input(mi)
    return mi, mesh, precompute(mesh, Params())


def test_constant_state_is_reproduced_exactly():
    """beta = 0 and sigma+ - sigma- = 1: R(x_G) = W for constant W (free-stream)."""
    mi, mesh, groups = _case()
    W = np.full((4, mesh.n_cells), 1.7)
    for t in groups:
        R = gauss_values_group(t, W, Params())
        assert np.abs(R - 1.7).max() < 1e-12  # rounding of sigma+- (|gamma| up to O(10))


def test_linear_data_is_reproduced_by_the_nonlinear_scheme():
    """All candidates agree at x_G for linear data, so any normalised weights give the exact value."""
    mi, mesh, groups = _case(cfg=3, kind="mixed")
    W = S.cell_average(mi, lambda x, y: (0.3 + 2.0 * x - 1.1 * y)[None], order=3)
    for t in groups:
        R = gauss_values_group(t, W, Params())[0]
        xG = mesh.cell_gauss[t.cells, :t.G]
        exact = 0.3 + 2.0 * xG[..., 0] - 1.1 * xG[..., 1]
        # interior cells whose candidates are all non-degenerate
        full = (t.members[..., 1] != t.cells[:, None]).all(-1)
        ghost = np.array([any(s[0] == 1 for s in mesh.slots[c]) for c in t.cells])
        sel = full & ~ghost
        assert sel.sum() > 10
        assert np.abs(R[sel] - exact[sel]).max() < 1e-12


def test_tiny_smoothness_reduces_to_the_linear_scheme():
    """beta << eps makes alpha proportional to gamma+-, so R -> sigma+ R+ - sigma- R- = sum gamma P."""
    mi, mesh, groups = _case()
    rng = np.random.default_rng(3)
    W = 1.0 + 1e-7 * rng.normal(size=(1, mesh.n_cells))
    for t in groups:
        R = gauss_values_group(t, W, Params())
        Rl = gauss_values_group(t, W, Params(linear=True))
        assert np.abs(R - Rl).max() < 1e-12


def test_splitting_is_identity_for_positive_weights():
    """With all gamma >= 0 the split weights equal gamma and R is the plain WENO combination."""
    mi, mesh, groups = _case(kind="quad", cfg=1)
    t = groups[0]
    pos = np.abs(t.gamma) + 0.01
    pos /= pos.sum(-1, keepdims=True)
    t2 = dataclasses.replace(t, gamma=pos)
    rng = np.random.default_rng(5)
    W = rng.normal(size=(1, mesh.n_cells))
    R = gauss_values_group(t2, W, Params())[0]
    # textbook WENO with the modified indicator and unsplit weights
    W0 = W[0, t.cells]
    dW = np.stack([W[0, t.members[..., 0]] - W0[:, None], W[0, t.members[..., 1]] - W0[:, None]], -1)
    g = np.einsum("nmab,nmb->nma", t.grad_op, dW)
    P = W0[:, None, None] + np.einsum("nma,nga->ngm", g, t.dG)
    beta = (t.area[:, None] * (g ** 2).sum(-1))[:, None, :]
    q = pos * beta
    a = pos / (beta * (1 + q + q * q) + Params().eps) ** 2
    ref = (a * P).sum(-1) / a.sum(-1)
    assert np.abs(R - ref).max() < 1e-12


def test_weights_approach_linear_weights_under_refinement():
    """delta+- -> gamma+- for smooth data: the nonlinear/linear gap shrinks with h (Section 3.4)."""
    gaps = []
    for n in (8, 16, 32):
        mi = S.mesh_for_config(1, n=n, seed=1)
        mesh = OracleMesh.from_input(mi)
        t = precompute(mesh, Params(eqn="scalar"))[0]
        W = S.cell_average(mi, S.scalar_wave)
        gap = gauss_values_group(t, W, Params()) - gauss_values_group(t, W, Params(linear=True))
        gaps.append(np.abs(gap).mean())
    assert gaps[0] > gaps[1] > gaps[2]
    assert gaps[1] / gaps[2] > 3.0


def test_discontinuity_gets_small_weights():
    """A jump inside some candidates' sub-stencils: the Gauss values stay within the local data range."""
    mi = S.mesh_for_config(3, n=16, seed=2, kind="mixed")
    mesh = OracleMesh.from_input(mi)
    groups = precompute(mesh, Params())
    W = np.where(mesh.centroid[:, 0] < 0.5, 1.0, 0.125)[None]
    over = []
    lin_over = []
    for t in groups:
        R = gauss_values_group(t, W, Params())[0]
        Rl = gauss_values_group(t, W, Params(linear=True))[0]
        over.append(np.maximum(R - 1.0, 0.125 - R).max())
        lin_over.append(np.maximum(Rl - 1.0, 0.125 - Rl).max())
    assert max(over) < 0.02 * 0.875
    assert max(lin_over) > 5 * max(over)
