"""Pins of the oracle's geometry and connectivity (closed surfaces, volumes, pairing)."""
import numpy as np
import pytest

from oracle.geometry import Geometry, inscribed_radius
from oracle.reference_element import ReferenceElement
from paper_1710_03887_gb300 import workloads as W


@pytest.fixture(scope="module")
def ref2():
    return ReferenceElement(2)


@pytest.mark.parametrize("jitter", [0.0, 0.15])
def test_kuhn_cube_volume_and_closed_surfaces(ref2, jitter):
    n = 3
    xyz, EToV = W.kuhn_cube(n, jitter=jitter, seed=1)
    g = Geometry(ref2, xyz, EToV)
    assert EToV.shape[0] == 6 * n ** 3
    assert g.volume.sum() == pytest.approx(8.0, rel=1e-13)           # [-1,1]^3
    # divergence theorem for a constant field: sum_f area_f n_f = 0
    closed = np.einsum("kf,kfi->ki", g.area, g.nrm)
    assert np.abs(closed).max() < 1e-14
    # boundary faces: 2 triangles per cell face on the 6 cube sides
    assert g.boundary.sum() == 12 * n ** 2
    assert np.all(g.J > 0)


def test_neighbours_are_consistent(ref2):
    xyz, EToV = W.kuhn_cube(3, jitter=0.1, seed=2)
    g = Geometry(ref2, xyz, EToV)
    K = g.K
    for k in range(K):
        for f in range(4):
            if g.boundary[k, f]:
                continue
            k2, f2 = g.EToE[k, f], g.EToF[k, f]
            assert g.EToE[k2, f2] == k and g.EToF[k2, f2] == f
            np.testing.assert_allclose(g.nrm[k2, f2], -g.nrm[k, f], atol=1e-14)
            assert g.area[k2, f2] == pytest.approx(g.area[k, f], rel=1e-13)
    # paired face nodes sit at the same physical point
    xf = g.x.reshape(-1, 3)
    np.testing.assert_allclose(xf[g.vmapP], xf[g.vmapM], atol=1e-13)


def test_periodic_pairing(ref2):
    xyz, EToV = W.kuhn_cube(2)
    g = Geometry(ref2, xyz, EToV, period=(2.0, 2.0, 2.0))
    assert not g.boundary.any()
    xf = g.x.reshape(-1, 3)
    d = xf[g.vmapP] - xf[g.vmapM]
    # paired nodes differ by a whole number of periods in each coordinate
    np.testing.assert_allclose(d / 2.0, np.round(d / 2.0), atol=1e-13)


def test_ball_boundary_on_sphere(ref2):
    xyz, EToV = W.ball(4, radius=1.0, jitter=0.1)
    g = Geometry(ref2, xyz, EToV)
    verts = g.verts
    fv = [(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)]
    for k, f in zip(*np.nonzero(g.boundary)):
        r = np.linalg.norm(verts[k, list(fv[f])], axis=1)
        np.testing.assert_allclose(r, 1.0, atol=1e-14)
    assert g.boundary.sum() == 12 * 4 ** 2
    # polyhedral ball: volume a little under 4/3 pi
    assert 3.4 < g.volume.sum() < 4.0 / 3.0 * np.pi


def test_inscribed_radius_regular_tet():
    # regular tetrahedron with edge a: r_in = a / sqrt(24)
    a = 2.0
    X = np.array([[-1.0, -1 / np.sqrt(3), -1 / np.sqrt(6)], [1.0, -1 / np.sqrt(3), -1 / np.sqrt(6)],
                  [0.0, 2 / np.sqrt(3), -1 / np.sqrt(6)], [0.0, 0.0, 3 / np.sqrt(6)]])
    g = Geometry(ReferenceElement(1), X, np.array([[0, 1, 2, 3]]))
    assert inscribed_radius(g)[0] == pytest.approx(a / np.sqrt(24.0), rel=1e-14)
    # Fscale = sJ / J with sJ = area / 2 and J = volume / (4/3)
    vol = a ** 3 / (6 * np.sqrt(2))
    area = np.sqrt(3) / 4 * a ** 2
    np.testing.assert_allclose(g.Fscale[0], (area / 2) / (vol * 3 / 4), rtol=1e-13)
