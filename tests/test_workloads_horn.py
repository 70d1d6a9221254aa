"""The horn-in-room workload (the two domain types of section 1.2, Table 1:
a room in front of the bell only, or a room enclosing the whole horn): a
lattice-mapped mesh of a flared horn and its room. Checked here against what
geometry alone fixes: exact volumes of the flat-walled room, convergence of
the horn's and the wall's volumes to the solids of revolution, the face tags
counted from the construction, the mirror symmetries, and free-stream
preservation of the oracle with every boundary kind of the workload."""
import numpy as np
import pytest

from oracle.euler_dg import CHARACTERISTIC, INFLOW_PULSE, SLIP_WALL, Gas
from oracle.euler_dg import Solver as OSolver
from oracle.geometry import Geometry
from oracle.reference_element import ReferenceElement
from paper_1710_03887_gb300 import workloads as W

SMALL = dict(m1=1, room_length=0.03, room_half=0.03, growth=1.8, horn_length=0.1, aspect=3.0)
ENCLOSED = dict(SMALL, behind=0.02)


def _volumes(p, xyz, EToV):
    g = Geometry(ReferenceElement(p), xyz, EToV)
    J = g.J.reshape(g.J.shape[0], -1)[:, 0]
    return g, J * 4.0 / 3.0


def test_profile_is_a_clamped_bessel_flare():
    x = np.array([0.0, 0.04, 0.5, 1.0])
    r = W.horn_radius(x)
    assert r[0] == r[1] == 0.006                       # the cylindrical bore
    assert r[2] == pytest.approx(0.006 * 0.55 ** -0.7)
    assert r[3] == pytest.approx(0.006 * 0.05 ** -0.7)
    assert np.all(np.diff(W.horn_radius(np.linspace(0, 1, 101))) >= 0)


@pytest.mark.parametrize("kw", [SMALL, ENCLOSED], ids=["bell-front", "enclosing"])
def test_tags_and_boundary_agree_with_the_oracle_connectivity(kw):
    xyz, EToV, tag, info = W.horn_in_room(**kw)
    g, vol = _volumes(1, xyz, EToV)
    assert np.array_equal(g.boundary, tag >= 0)
    m1 = kw["m1"]
    counts = np.bincount(tag[tag >= 0], minlength=3)
    assert counts[W.HORN_MOUTHPIECE] == 2 * (2 * m1) ** 2
    nh = info["planes"][1]
    inside = nh * 4 * (2 * m1) * 2                     # horn planes x perimeter cells x 2 triangles
    ring = ((2 * m1 + 2) ** 2 - (2 * m1) ** 2) * 2    # the bell rim / the wall's front end
    if info["type"] == "B":
        assert counts[W.HORN_WALL] == inside + ring
    else:
        outside = nh * 4 * (2 * m1 + 2) * 2            # the wall's outer surface
        cap = (2 * m1 + 2) ** 2 * 2 + 4 * (2 * m1 + 2) * 2
        assert counts[W.HORN_WALL] == inside + outside + ring + cap
    # the mouthpiece lies on x = 0 with outward normal -x; inner walls face away from the axis
    fx = g.x[:, g.ref.Fmask].mean(axis=2)              # face centroids [K, 4, 3]
    mouth = tag == W.HORN_MOUTHPIECE
    assert np.allclose(fx[mouth][:, 0], 0.0) and np.allclose(g.nrm[mouth][:, 0], -1.0)
    horn = info["horn_elements"][:, None] & (tag == W.HORN_WALL) & (fx[..., 0] < info["bell_x"] - 1e-12)
    assert np.all(np.einsum("fd,fd->f", g.nrm[horn][:, 1:], fx[horn][:, 1:]) > 0)
    if info["type"] == "A":                            # the wall's outer surface faces the axis
        out = ~info["horn_elements"][:, None] & (tag == W.HORN_WALL) & (fx[..., 0] > 1e-9) \
            & (fx[..., 0] < info["bell_x"] - 1e-12)
        assert out.any() and np.all(np.einsum("fd,fd->f", g.nrm[out][:, 1:], fx[out][:, 1:]) < 0)


@pytest.mark.parametrize("shape", ["box", "cylinder"])
def test_room_and_horn_volumes(shape):
    kw = dict(SMALL, shape=shape)
    xyz, EToV, tag, info = W.horn_in_room(**kw)
    _, vol = _volumes(1, xyz, EToV)
    assert np.all(vol > 0)
    room = vol[info["n_horn"]:].sum()
    L, h = kw["room_length"], kw["room_half"]
    if shape == "box":                                 # flat walls: exact
        assert room == pytest.approx((2 * h) ** 2 * L, rel=1e-12)
    else:                                              # inscribed polygon of the circle
        assert 0.95 * np.pi * h * h * L < room < np.pi * h * h * L
    # the horn's polygonal cross-sections converge to the disc at second order
    xs = np.linspace(0.0, kw["horn_length"], 20001)
    exact = np.pi * np.trapezoid(W.horn_radius(xs) ** 2, xs)
    errs = []
    for m1 in (1, 2, 4):
        xyz, EToV, _, info = W.horn_in_room(**dict(kw, m1=m1))
        _, vol = _volumes(1, xyz, EToV)
        errs.append(abs(vol[:info["n_horn"]].sum() - exact) / exact)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.02 and errs[1] / errs[2] > 3.0


def test_enclosing_room_volume_is_the_box_minus_the_solid():
    """Type A: flat outer walls, so the mesh volume is the box minus the
    horn's wall (thickness 0.002) and the mouthpiece cap; the polygonal
    annuli converge to the solid of revolution."""
    kw = dict(ENCLOSED)
    box = (2 * kw["room_half"]) ** 2 * (kw["room_length"] + kw["horn_length"] + kw["behind"])
    xs = np.linspace(0.0, kw["horn_length"], 20001)
    r = W.horn_radius(xs)
    solid = np.pi * np.trapezoid((r + 0.002) ** 2 - r * r, xs) + np.pi * (0.006 + 0.002) ** 2 * 0.002
    errs = []
    for m1 in (1, 2, 4):
        xyz, EToV, _, _ = W.horn_in_room(**dict(kw, m1=m1))
        _, vol = _volumes(1, xyz, EToV)
        assert np.all(vol > 0)
        errs.append(abs(box - vol.sum() - solid) / solid)
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.005


@pytest.mark.parametrize("kw", [SMALL, ENCLOSED], ids=["bell-front", "enclosing"])
def test_mirror_symmetries_of_the_mesh(kw):
    xyz, EToV, _, _ = W.horn_in_room(**dict(kw, m1=2))
    c = xyz[EToV].mean(axis=1)

    def canon(a):
        return a[np.lexsort(np.round(a, 12).T[::-1])]

    ref = canon(c)
    for M in (np.diag([1, -1, 1]), np.diag([1, 1, -1]), np.array([[1, 0, 0], [0, 0, 1], [0, 1, 0]])):
        assert np.allclose(canon(c @ M.T), ref, atol=1e-12)


@pytest.mark.parametrize("kw", [SMALL, ENCLOSED], ids=["bell-front", "enclosing"])
def test_rest_state_is_preserved_with_every_boundary_of_the_workload(kw):
    """Walls reflect a state at rest into itself, the characteristic
    condition returns the free stream, and the inflow pulse at t = 0 is the
    base state: the right-hand side vanishes to rounding."""
    xyz, EToV, tag, _ = W.horn_in_room(**kw)
    g = Geometry(ReferenceElement(2), xyz, EToV)
    gas = Gas(W.GAMMA, W.RHO0_SI, W.P0_SI)
    bc_id = np.where(tag < 0, 0, tag).astype(np.int64)
    orc = OSolver(g, gas, bc_id=bc_id, bc_mode={W.HORN_OUTER: CHARACTERISTIC,
                                                 W.HORN_WALL: SLIP_WALL,
                                                 W.HORN_MOUTHPIECE: INFLOW_PULSE})
    orc.inflow = (0.1, 2 * np.pi * 500.0)
    q = W.uniform_state(g.K, g.ref.Np, W.RHO0_SI, (0, 0, 0), W.P0_SI, W.GAMMA)
    r = orc.rhs(q, 0.0)
    scale = W.P0_SI * np.abs(g.Fscale).max()
    assert np.abs(r).max() <= 1e-12 * scale
    # a quarter period later the pulse drives the mouthpiece only
    r = orc.rhs(q, 0.25 * 2 * np.pi / orc.inflow[1])
    moved = np.abs(r).max(axis=(1, 2)) > 1e-9 * scale
    assert moved.any() and np.all(np.any(tag[moved] == W.HORN_MOUTHPIECE, axis=1))


def test_sensors_are_the_papers_positions():
    """The workload's sensors are the four of the paper's horn study (section
    3, Table 2; tests/golden/sensors_table2.txt) with the flare-room junction
    moved from x = 1.48 m to the workload's bell plane, and they keep the
    distances to the outer boundary that Table 2 lists (sensor 1: 1 cm below
    the top wall, sensor 2: 2 cm and sensor 3: 1 cm before the far wall),
    here measured on the mesh itself; each lies inside the mesh."""
    from pathlib import Path
    from oracle.euler_dg import Probes
    rows, junction = [], None
    for line in (Path(__file__).parent / "golden" / "sensors_table2.txt").read_text().splitlines():
        if line.startswith("# junction_x"):
            junction = float(line.split()[2])
        elif line.strip() and not line.startswith("#"):
            rows.append([float(v) for v in line.split()[1:]])
    paper = np.array(rows)
    xyz, EToV, _, info = W.horn_in_room(m1=1, growth=1.8)
    s = info["sensors"]
    np.testing.assert_allclose(s + [junction - info["bell_x"], 0.0, 0.0], paper, rtol=0, atol=1e-12)
    top, far = xyz[:, 1].max(), xyz[:, 0].max()
    assert top - s[0, 1] == pytest.approx(0.01, abs=1e-12)
    assert far - s[1, 0] == pytest.approx(0.02, abs=1e-12)
    assert far - s[2, 0] == pytest.approx(0.01, abs=1e-12)
    Probes(Geometry(ReferenceElement(1), xyz, EToV), s)


# ------------------------------------------------------------- the Table 1 shapes
# small versions of the outer shapes (horn 0.1 long): type B in front of the
# bell, type A enclosing the horn and reaching 0.03 behind its mouthpiece
SHAPES = {
    "B-half-sphere": dict(SMALL, shape="sphere"),
    "B-half-cone": dict(SMALL, shape="cone"),
    "A-sphere": dict(SMALL, shape="sphere", behind=0.03, growth=2.2),
    "A-cone": dict(SMALL, shape="cone", behind=0.03, room_half=0.06, growth=2.2),
    "A-scone": dict(SMALL, shape="scone", behind=0.03, room_half=0.06, growth=2.2),
}


def _shape_geometry(kw):
    """The exact outer surface of a shape: a function giving, for points
    [n, 3], the distance to the nearest piece of the surface, and the exact
    volume enclosed by the outer surface."""
    L, Rl, H, b = kw["horn_length"], kw["room_length"], kw["room_half"], kw.get("behind", 0.0)
    shape = kw["shape"]
    if shape == "sphere":
        if b > 0:
            xc, R = 0.5 * (L + Rl - b), 0.5 * (L + Rl + b)
            return (lambda p: np.abs(np.linalg.norm(p - [xc, 0, 0], axis=1) - R)), 4.0 / 3.0 * np.pi * R ** 3
        # the hemisphere: its sphere or its flat face in the bell plane
        return ((lambda p: np.minimum(np.abs(np.linalg.norm(p - [L, 0, 0], axis=1) - Rl),
                                      np.abs(p[:, 0] - L))), 2.0 / 3.0 * np.pi * Rl ** 3)
    if shape == "cone" and b == 0:
        # 45-degree cone: base disc in the bell plane, apex at L + Rl
        def dist(p):
            r = np.hypot(p[:, 1], p[:, 2])
            return np.minimum(np.abs((p[:, 0] - L) + r - Rl) / np.sqrt(2.0), np.abs(p[:, 0] - L))
        return dist, np.pi * Rl ** 3 / 3.0
    xa = -b
    k = H / (L + 0.01 - xa)
    rad1_0 = float(W.horn_radius(0.0)) + 0.002
    x_lo = xa + (rad1_0 + 0.5 * (k * (0.0 - xa) - rad1_0)) / k
    h_lo = x_lo - xa
    if shape == "cone":
        Hb = L + Rl - xa

        def dist(p):
            r = np.hypot(p[:, 1], p[:, 2])
            side = np.abs(r - k * (p[:, 0] - xa)) / np.sqrt(1 + k * k)
            return np.minimum(side, np.minimum(np.abs(p[:, 0] - x_lo), np.abs(p[:, 0] - L - Rl)))
        return dist, np.pi * k * k / 3.0 * (Hb ** 3 - h_lo ** 3)
    Rs = L + Rl - xa
    th = np.arctan(k)

    def dist(p):
        r = np.hypot(p[:, 1], p[:, 2])
        side = np.abs(r - k * (p[:, 0] - xa)) / np.sqrt(1 + k * k)
        sph = np.abs(np.linalg.norm(p - [xa, 0, 0], axis=1) - Rs)
        return np.minimum(np.minimum(side, sph), np.abs(p[:, 0] - x_lo))
    sector = 2.0 / 3.0 * np.pi * Rs ** 3 * (1.0 - np.cos(th))
    return dist, sector - np.pi * k * k / 3.0 * h_lo ** 3


def _tet_volumes(xyz, EToV):
    v = xyz[EToV]
    return np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0]) / 6.0


def _containing_tet(xyz, EToV, pt):
    """Index of a tetrahedron whose barycentric coordinates of pt are all >= -1e-12."""
    v = xyz[EToV]
    T = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
    lam = np.linalg.solve(T, (pt - v[:, 0])[..., None])[..., 0]
    ok = np.all(lam >= -1e-12, axis=1) & (lam.sum(axis=1) <= 1 + 1e-12)
    return np.nonzero(ok)[0]


def _solid_volume(kw):
    """Exact volume of the horn's solid parts in a type A domain: the wall
    (thickness 0.002 around the profile) and the cap behind the mouthpiece."""
    xs = np.linspace(0.0, kw["horn_length"], 20001)
    r = W.horn_radius(xs)
    return np.pi * np.trapezoid((r + 0.002) ** 2 - r * r, xs) + np.pi * (0.006 + 0.002) ** 2 * 0.002


@pytest.mark.parametrize("name", list(SHAPES))
def test_outer_boundary_lies_on_the_shape(name):
    """Every vertex of an outer (pass-through) face lies on the exact outer
    surface of the shape (sphere, cone, spherical cap or flat end)."""
    kw = SHAPES[name]
    xyz, EToV, tag, info = W.horn_in_room(**kw)
    assert info["name"] == name
    dist, _ = _shape_geometry(kw)
    fv = np.array([(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)])
    outer = EToV[:, fv][tag == W.HORN_OUTER].ravel()
    assert outer.size > 0
    assert dist(xyz[np.unique(outer)]).max() < 1e-12
    # and no vertex lies outside the shape's bounding radius
    scale = max(kw["room_length"], kw["room_half"]) + kw["horn_length"] + kw.get("behind", 0.0)
    assert np.abs(xyz).max() < 2 * scale


@pytest.mark.parametrize("name", list(SHAPES))
def test_shape_volumes_converge_to_the_solids(name):
    """The mesh's volume converges to the exact volume of the shape (minus
    the horn's solid parts for type A; the horn's interior for type B is
    counted apart) at second order in the lattice's angular resolution: the
    outer surface is an inscribed polyhedron."""
    kw = SHAPES[name]
    _, exact = _shape_geometry(kw)
    enclose = kw.get("behind", 0.0) > 0
    if enclose:
        exact = exact - _solid_volume(kw)
    errs, ms = [], []
    for m1, growth in ((1, kw["growth"]), (2, 1.5), (4, 1.25)):
        xyz, EToV, _, info = W.horn_in_room(**dict(kw, m1=m1, growth=growth))
        vol = _tet_volumes(xyz, EToV)
        assert np.all(vol > 0)
        v = vol.sum() if enclose else vol[info["n_horn"]:].sum()
        errs.append(abs(v - exact) / exact)
        ms.append(m1 + info["rings"])             # lattice half-width: angular resolution
    # second order: the error falls at least like 0.7 (m / m')^2 per step
    for i in range(2):
        assert errs[i] / errs[i + 1] > 0.7 * (ms[i + 1] / ms[i]) ** 2, (errs, ms)
    assert errs[2] < 0.005, errs


@pytest.mark.parametrize("name", list(SHAPES))
def test_shape_tags_symmetries_and_rest_state(name):
    """The face tags of the new shapes agree with the oracle's connectivity
    (every boundary face tagged, the mouthpiece and wall counts those of the
    horn), the mesh keeps the mirror symmetries, and a state at rest stays
    at rest with every boundary kind."""
    kw = SHAPES[name]
    xyz, EToV, tag, info = W.horn_in_room(**kw)
    g, vol = _volumes(1, xyz, EToV)
    assert np.all(vol > 0)
    assert np.array_equal(g.boundary, tag >= 0)
    counts = np.bincount(tag[tag >= 0], minlength=3)
    assert counts[W.HORN_MOUTHPIECE] == 2 * (2 * kw["m1"]) ** 2
    # the wall tags are those of the box of the same type (the horn is the same)
    _, _, tag_box, _ = W.horn_in_room(**dict(kw, shape="box", room_half=SMALL["room_half"]
                                             if info["type"] == "B" else kw["room_half"]))
    assert counts[W.HORN_WALL] == np.count_nonzero(tag_box == W.HORN_WALL)
    c = xyz[EToV].mean(axis=1)

    def canon(a):
        return a[np.lexsort(np.round(a, 12).T[::-1])]
    ref = canon(c)
    for M in (np.diag([1, -1, 1]), np.diag([1, 1, -1]), np.array([[1, 0, 0], [0, 0, 1], [0, 1, 0]])):
        assert np.allclose(canon(c @ M.T), ref, atol=1e-12)
    g2 = Geometry(ReferenceElement(2), xyz, EToV)
    gas = Gas(W.GAMMA, W.RHO0_SI, W.P0_SI)
    orc = OSolver(g2, gas, bc_id=np.where(tag < 0, 0, tag).astype(np.int64),
                  bc_mode={W.HORN_OUTER: CHARACTERISTIC, W.HORN_WALL: SLIP_WALL,
                           W.HORN_MOUTHPIECE: INFLOW_PULSE})
    orc.inflow = (0.1, 2 * np.pi * 500.0)
    q = W.uniform_state(g2.K, g2.ref.Np, W.RHO0_SI, (0, 0, 0), W.P0_SI, W.GAMMA)
    assert np.abs(orc.rhs(q, 0.0)).max() <= 1e-12 * W.P0_SI * np.abs(g2.Fscale).max()


@pytest.mark.parametrize("shape,behind", [("sphere", 0.0), ("cone", 0.0), ("sphere", 1.02),
                                          ("cone", 1.02), ("scone", 1.02)])
def test_full_size_shapes_hold_the_sensors(shape, behind):
    """At full size (coarse lattice) every shape contains the four sensors
    of Table 2 and reaches 1 cm past sensor 3 on the axis."""
    xyz, EToV, _, info = W.horn_in_room(shape=shape, behind=behind, m1=1, growth=1.8, aspect=8.0)
    s = info["sensors"]
    assert xyz[:, 0].max() - s[2, 0] == pytest.approx(0.01, abs=1e-12)
    assert np.all(_tet_volumes(xyz, EToV) > 0)
    for pt in s:
        assert _containing_tet(xyz, EToV, pt).size > 0
