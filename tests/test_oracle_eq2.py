"""Pins of the Eq. 2 cost model in the oracle: mixed vertex areas (Meyer et al. 2003) and the
area-weighted feature-distance element costs.

* the mixed areas of a closed mesh partition its surface area;
* on regular polyhedra every vertex gets the same share;
* on an acute triangle each corner's share equals the area of its Voronoi cell piece, built
  directly from the circumcentre and the edge midpoints (shoelace formula), an independent
  construction of the cotangent formula;
* on an obtuse triangle the obtuse corner gets half, the others a quarter;
* with exactly copied features the relabelling has cost 0 and is the unique optimum.
"""
import numpy as np
import pytest

from oracle import exact as E
from oracle import problem as P
from synth import instances as I
from synth import meshes as M


def _surface(V, T):
    V = np.asarray(V, np.float64)
    return sum(0.5 * np.linalg.norm(np.cross(V[b] - V[a], V[c] - V[a])) for a, b, c in T)


@pytest.mark.parametrize("mesh", [M.tetrahedron(), M.icosahedron(), M.icosphere(2), M.torus(6, 9)])
def test_mixed_areas_partition_the_surface(mesh):
    a = P.mixed_areas(mesh.V, mesh.T)
    assert np.all(a > 0)
    assert a.sum() == pytest.approx(_surface(mesh.V, mesh.T), rel=1e-12)
    Y = M.deform_radial(mesh, np.random.default_rng(4)) if mesh.nt > 4 and mesh.nv < 300 else mesh
    assert P.mixed_areas(Y.V, Y.T).sum() == pytest.approx(_surface(Y.V, Y.T), rel=1e-12)


@pytest.mark.parametrize("mesh", [M.tetrahedron(), M.icosahedron()])
def test_regular_polyhedra_share_equally(mesh):
    a = P.mixed_areas(mesh.V, mesh.T)
    np.testing.assert_allclose(a, _surface(mesh.V, mesh.T) / mesh.nv, rtol=1e-12)


def _voronoi_piece(P0, P1, P2):
    """Area of the part of the triangle closer to P0 than to P1, P2 (acute triangle):
    the quadrilateral P0, mid(P0 P1), circumcentre, mid(P0 P2)."""
    a, b = P1 - P0, P2 - P0
    n = np.cross(a, b)
    # circumcentre of the triangle (standard vector formula)
    cc = P0 + (np.cross(n, a) * (b @ b) + np.cross(b, n) * (a @ a)) / (2.0 * (n @ n))
    quad = [P0, (P0 + P1) / 2, cc, (P0 + P2) / 2]
    # shoelace in the triangle's plane
    e1 = a / np.linalg.norm(a)
    e2 = np.cross(n / np.linalg.norm(n), e1)
    xy = [((q - P0) @ e1, (q - P0) @ e2) for q in quad]
    s = sum(x0 * y1 - x1 * y0 for (x0, y0), (x1, y1) in zip(xy, xy[1:] + xy[:1]))
    return abs(s) / 2.0


def test_acute_triangle_matches_voronoi_cells():
    V = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.4, 0.9, 0.2]])
    T = np.array([[0, 1, 2]])
    a = P.mixed_areas(V, T)
    for v in range(3):
        ref = _voronoi_piece(V[v], V[(v + 1) % 3], V[(v + 2) % 3])
        assert a[v] == pytest.approx(ref, rel=1e-12)
    assert a.sum() == pytest.approx(_surface(V, T), rel=1e-12)


def test_obtuse_triangle_split():
    V = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.3, 0.2, 0.0]])  # obtuse at vertex 2
    T = np.array([[0, 1, 2]])
    a = P.mixed_areas(V, T)
    area = _surface(V, T)
    np.testing.assert_allclose(a, [area / 4, area / 4, area / 2], rtol=1e-12)


def test_eq2_zero_noise_copy_has_unique_zero_optimum():
    inst = I.tet(seed=3, feat_noise=0.0)
    d = P.pair_euclid(inst.FX, inst.FY)
    prob = P.build_problem(inst.X.T, inst.Y.T, d, None, cost_model=1, VX=inst.X.V, VY=inst.Y.V)
    assert np.all(prob.cost >= 0)
    opt, x, nopt, _ = E.solve_exact(prob)
    assert opt == pytest.approx(0.0, abs=1e-15) and nopt == 1
    tt = (prob.vtype == P.TT) & (x == 1)
    assert np.all(inst.perm[prob.vm[tt]] == prob.vn[tt])
