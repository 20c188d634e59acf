"""Pins of the oracle's finite-element pieces against closed forms (CPU only).

Whitney edge elements reproduce constant fields exactly and map fields of
constant curl to discrete fields of the same constant curl, so the element
energies of such fields have closed forms; discrete gradients lie in the
kernel of K; loop sources are discretely divergence free; the observation
operator returns -B_z for a field of constant curl B.
"""
import numpy as np
import pytest

from oracle.fem import MU0, FEModel
from oracle.survey import loop_source, observation_operator
from paper_2605_19951_gb300 import inputs


@pytest.fixture(scope="module")
def fe3():
    xyz, tets = inputs.kuhn_box(3, 40.0, 1)
    # distort the interior vertices so that no tetrahedron is special
    rng = np.random.default_rng(7)
    lo, hi = xyz.min(0), xyz.max(0)
    inner = np.all((xyz > lo + 1) & (xyz < hi - 1), axis=1)
    xyz = xyz.copy()
    xyz[inner] += rng.uniform(-6, 6, size=(inner.sum(), 3))
    return FEModel(xyz, tets)


def _local_line_integrals(fe, field):
    """u_loc[t, i] = int along local edge i of field . dl (midpoint rule, exact for
    affine fields)."""
    from oracle.fem import LOCAL_EDGES
    X = fe.xyz[fe.tv]
    out = np.empty((X.shape[0], 6))
    for i, (a, b) in enumerate(LOCAL_EDGES):
        mid = 0.5 * (X[:, a] + X[:, b])
        out[:, i] = np.einsum("tk,tk->t", field(mid), X[:, b] - X[:, a])
    return out


def test_counts():
    n = 5
    xyz, tets = inputs.kuhn_box(n, 10.0, 2)
    fe = FEModel(xyz, tets)
    assert len(fe.edges) == 7 * n ** 3 + 9 * n ** 2 + 3 * n
    assert fe.N == 7 * n ** 3 - 9 * n ** 2 + 3 * n
    assert tets.shape[0] == 6 * n ** 3
    assert np.allclose(fe.vol.sum(), (n * 10.0) ** 3)


def test_mass_exact_for_constant_fields(fe3):
    E = np.array([0.3, -1.2, 0.7])
    u = _local_line_integrals(fe3, lambda x: np.broadcast_to(E, x.shape))
    energy = np.einsum("ti,tij,tj->t", u, fe3.Me1, u)
    assert np.allclose(energy, fe3.vol * (E @ E), rtol=1e-12)


def test_stiffness_exact_for_constant_curl(fe3):
    B = np.array([0.4, 0.9, -0.5])
    u = _local_line_integrals(fe3, lambda x: 0.5 * np.cross(B, x) + np.array([1.0, 2.0, 3.0]))
    energy = np.einsum("ti,tij,tj->t", u, fe3.Ke, u)
    assert np.allclose(energy, fe3.vol * (B @ B) / MU0, rtol=1e-11)


def test_stiffness_kills_gradients(fe3):
    rng = np.random.default_rng(3)
    phi = rng.standard_normal(fe3.xyz.shape[0])
    lo, hi = fe3.xyz.min(0), fe3.xyz.max(0)
    on_b = np.any((np.abs(fe3.xyz - lo) < 1e-9) | (np.abs(fe3.xyz - hi) < 1e-9), axis=1)
    phi[on_b] = 0.0
    u = fe3.gradient_matrix() @ phi
    r = fe3.K @ u
    assert np.abs(r).max() < 1e-10 * np.abs(fe3.K).max() * np.abs(u).max()


def test_mass_symmetric_positive_definite(fe3):
    sig = np.random.default_rng(4).uniform(1e-3, 1.0, fe3.tv.shape[0])
    M = fe3.mass(sig).toarray()
    assert np.allclose(M, M.T, atol=1e-14 * np.abs(M).max())
    assert np.linalg.eigvalsh(M).min() > 0


def test_loop_source_divergence_free():
    n, n_air = 6, 2
    xyz, tets = inputs.kuhn_box(n, 20.0, n_air)
    fe = FEModel(xyz, tets)
    loop = inputs.square_loop(n, n_air, 1, 2, 3)
    f = loop_source(fe, loop)
    assert set(np.unique(f)) <= {-1.0, 0.0, 1.0}
    assert np.count_nonzero(f) == len(loop)
    G = fe.gradient_matrix()
    # G^T f = 0: the discrete divergence of a closed loop current vanishes
    assert np.abs(G.T @ f).max() == 0.0
    # the loop runs counter-clockwise seen from +z: circulation of f along the
    # x-directed edges on the lower side is positive
    lower = [s for s in range(3)]
    for s in lower:
        e = fe.edge_id(int(loop[s]), int(loop[s + 1]))
        assert f[fe.dof[e]] == 1.0


def test_observation_constant_curl():
    n, n_air, h = 6, 2, 20.0
    xyz, tets = inputs.kuhn_box(n, h, n_air)
    fe = FEModel(xyz, tets)
    B = np.array([0.1, -0.3, 0.8])
    u = fe.interpolate(lambda x: 0.5 * np.cross(B, x))
    rx = np.array([[0.0, 0.0, 0.0],            # vertex
                   [h / 2, 0.0, 0.0],           # edge midpoint
                   [h / 3, -h / 4, 0.0],        # face interior
                   [-h, h, 0.0]])
    Q = observation_operator(fe, rx)
    assert np.allclose(Q @ u, -B[2], rtol=1e-12)


def test_observation_matches_element_curl():
    """Receiver inside a surface face: Q u = -(curl of the Whitney field)_z in
    either tetrahedron sharing the face (element curl, independent formula)."""
    n, n_air, h = 4, 2, 30.0
    xyz, tets = inputs.kuhn_box(n, h, n_air)
    fe = FEModel(xyz, tets)
    p = np.array([h * 0.3, h * 0.55, 0.0])
    Q = observation_operator(fe, p[None])
    u = np.random.default_rng(5).standard_normal(fe.N)
    X = fe.xyz[fe.tv]
    cen = X.mean(axis=1)
    found = 0
    for t in range(fe.tv.shape[0]):
        zs = X[t, :, 2]
        if np.sum(np.abs(zs) < 1e-9) != 3:
            continue
        face = X[t][np.abs(zs) < 1e-9][:, :2]
        a, b, c = face
        M = np.array([b - a, c - a]).T
        lam = np.linalg.solve(M, p[:2] - a)
        if lam.min() < 0 or lam.sum() > 1:
            continue
        ul = np.where(fe.tdof[t] >= 0, u[np.maximum(fe.tdof[t], 0)], 0.0)
        curl = (ul[:, None] * fe.curl[t]).sum(axis=0)
        assert np.isclose((Q @ u)[0], -curl[2], rtol=1e-11)
        found += 1
    assert found == 2 and cen is not None
