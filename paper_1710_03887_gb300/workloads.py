"""Seeded synthetic workloads: tetrahedral meshes and initial states.

This module is the one place both the CUDA path and the CPU oracle take their
inputs from. It holds no arithmetic of the DG method itself: it only builds
vertex/element arrays and evaluates the initial condition at node positions
that the caller supplies.

Workloads (the paper's meshes are GMSH meshes of a trumpet in seven outer
domains, section 1.2 / Table 1; they are not available, so these synthetic
meshes stand in for them with matching element counts):

* ``kuhn_cube``: the cube [lo, hi]^3 cut into n^3 sub-cubes, each split into
  six tetrahedra along its main diagonal (Kuhn/Freudenthal split). The split is
  invariant under axis permutations and central inversion, which the symmetry
  tests rely on.
* ``ball``: the octant-mirrored lattice on [-1, 1]^3 pushed onto the ball of
  radius R by a radial map that is close to the identity at the centre and
  sends the lattice cube |x|_inf = 1 onto the sphere (see ``ball``). An
  optional seeded jitter of the interior lattice vertices (applied before the
  map) gives a quasi-uniform unstructured mesh.

Element vertex order follows the reference map of the solver: vertex 1 is the
image of (r,s,t) = (-1,-1,-1), vertex 2 of (1,-1,-1), vertex 3 of (-1,1,-1),
vertex 4 of (-1,-1,1). Every generated element is positively oriented.

The initial state is the acoustic pulse used throughout the paper's study in
its simplest form: flow at rest (section 2.2, Eq. 3) with a Gaussian pressure
bump, density following the isentropic relation (the adiabatic law of Eq. 6),
total energy from the ideal-gas law (Eq. 2).
"""
from __future__ import annotations

import numpy as np

# Six Kuhn tetrahedra of the unit cube: each is the chain 0 -> e_a -> e_a+e_b
# -> (1,1,1) for a permutation (a, b, c) of the axes.
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def kuhn_cube(n, lo=-1.0, hi=1.0, jitter=0.0, seed=0, mirrored=False):
    """Kuhn-split cube lattice.

    Returns ``(xyz, EToV)``: ``xyz`` float64 [(n+1)^3, 3], ``EToV`` int32
    [6 n^3, 4], positively oriented. ``jitter`` (fraction of the cell size)
    moves interior vertices by a seeded uniform offset in each coordinate.
    ``mirrored``: the split of each cell is reflected into the cell's octant
    (relative to the cube centre), so every cell's diagonal runs from its
    corner nearest the centre to the farthest one. The lattice stays
    conforming, gains the reflection symmetries of the cube, and no element
    has all four vertices on the cube surface.
    """
    n = int(n)
    if n < 1:
        raise ValueError("n must be >= 1")
    h = (hi - lo) / n
    g = np.arange(n + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    ijk = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    xyz = lo + h * ijk.astype(np.float64)

    def vid(q):
        return (q[:, 0] * (n + 1) + q[:, 1]) * (n + 1) + q[:, 2]

    c = np.arange(n)
    ci, cj, ck = np.meshgrid(c, c, c, indexing="ij")
    cell = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)
    if mirrored:
        # step direction per axis: away from the centre of the cube
        step = np.where(2 * cell + 1 >= n, 1, -1)
    else:
        step = np.ones_like(cell)
    start = cell + (step < 0)
    tets = []
    for perm in _PERMS:
        corner = start.copy()
        chain = [corner.copy()]
        for axis in perm:
            corner = corner.copy()
            corner[:, axis] += step[:, axis]
            chain.append(corner)
        tets.append(np.stack([vid(q) for q in chain], axis=1))
    # element order: cell-major (all six tets of a cell are consecutive)
    EToV = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int64)
    # orient positively: swap two vertices where the signed volume is negative
    v = xyz[EToV]
    det = np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0])
    neg = det < 0
    EToV[neg, 1], EToV[neg, 2] = EToV[neg, 2].copy(), EToV[neg, 1].copy()
    EToV = EToV.astype(np.int32)

    if jitter:
        rng = np.random.default_rng(seed)
        interior = np.all((ijk > 0) & (ijk < n), axis=1)
        off = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
        xyz = xyz + off * interior[:, None]
    _fix_orientation(xyz, EToV)
    return xyz, EToV


def _fix_orientation(xyz, EToV):
    v = xyz[EToV]
    d = np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]),
                  v[:, 3] - v[:, 0])
    if np.any(d <= 0):
        raise ValueError("mesh generator produced a non-positive element")


def periodic_vertex_classes(n):
    """Connectivity ids for the fully periodic Kuhn cube of ``kuhn_cube(n)``.

    Vertex (i, j, k) is identified with (i mod n, j mod n, k mod n); two faces
    are neighbours when their vertex-class triples agree.
    """
    g = np.arange(n + 1) % n
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    return ((I * n + J) * n + K).ravel().astype(np.int64)


def ball(n, radius=1.0, jitter=0.0, seed=0, sphere_from=1.0):
    """Ball of the given radius: ``kuhn_cube(n)`` on [-1,1]^3 mapped radially.

    A lattice point x with s = |x|_inf moves to  radius * x * g  with
    g = 1 - b (1 - |x|_inf / |x|_2)  and  b = min(1, s / sphere_from).
    Near the centre the map is close to the identity; every lattice cube
    |x|_inf = s >= sphere_from lands on the sphere of radius ``radius * s``.
    Along a ray the radial stretch is 1 - (1 - |x|_inf/|x|_2)(b + s b') >=
    1 - 2 (1 - 1/sqrt(3)) > 0.15, so the map keeps every cell positively
    oriented. With n = 32 this has 196,608 elements (the ~200k-element ball
    workload). With ``sphere_from = m / (n/2)`` the spheres of radius
    ``radius * m' / (n/2)``, m' >= m, are made of element faces (nested
    truncation radii).
    """
    if not (0.0 < sphere_from <= 1.0):
        raise ValueError("need 0 < sphere_from <= 1")
    xyz, EToV = kuhn_cube(n, -1.0, 1.0, jitter=jitter, seed=seed, mirrored=True)
    inf = np.max(np.abs(xyz), axis=1)
    two = np.linalg.norm(xyz, axis=1)
    ratio = np.where(two > 0, inf / np.where(two > 0, two, 1.0), 1.0)
    b = np.minimum(1.0, inf / sphere_from)
    g = 1.0 - b * (1.0 - ratio)
    xyz = radius * xyz * g[:, None]
    _fix_orientation(xyz, EToV)
    return xyz, EToV


def submesh(xyz, EToV, keep):
    """Restrict a mesh to the elements where ``keep`` is true (vertices renumbered)."""
    E = EToV[keep]
    used, inv = np.unique(E.ravel(), return_inverse=True)
    return xyz[used].copy(), inv.reshape(E.shape).astype(np.int32)


def morton_order(xyz, EToV, bits=10):
    """Permutation of the elements that sorts their centroids along the
    Morton (Z-order) curve of a 2^bits grid over the mesh's bounding box:
    consecutive elements are close in space, whatever order a mesh
    generator produced them in."""
    c = xyz[EToV].mean(axis=1)
    lo, hi = c.min(axis=0), c.max(axis=0)
    g = np.clip(((c - lo) / np.maximum(hi - lo, 1e-300) * (2 ** bits - 1)).round(), 0, 2 ** bits - 1)
    g = g.astype(np.uint64)
    code = np.zeros(len(c), dtype=np.uint64)
    for b in range(bits):
        for d in range(3):
            code |= ((g[:, d] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + d)
    return np.argsort(code, kind="stable")


def random_order(K, seed=0):
    """A seeded random permutation of K elements (no locality at all)."""
    return np.random.default_rng(seed).permutation(K)


def shuffle_vertices(xyz, EToV, seed=0):
    """The same mesh with each element's vertex list in a seeded random
    order, kept positively oriented (an odd permutation has its first two
    entries swapped back). Mesh generators list the vertices of shared faces
    in unrelated orders; the lattice generators here do not, so a shared
    face meets only some of the six vertex correspondences between its two
    sides. After this shuffle every correspondence occurs."""
    rng = np.random.default_rng(seed)
    E = np.array([row[rng.permutation(4)] for row in np.asarray(EToV)], dtype=np.int32)
    v = xyz[E]
    d = np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0])
    E[d < 0] = E[d < 0][:, [1, 0, 2, 3]]
    _fix_orientation(xyz, E)
    return E


def element_centroids(xyz, EToV):
    return xyz[EToV].mean(axis=1)


def gaussian_pulse_state(nodes, gamma, rho0, p0, amplitude, width,
                         center=(0.0, 0.0, 0.0)):
    """Conserved state [K, 5, Np] of a resting gas with a Gaussian pressure pulse.

    ``nodes`` is [K, Np, 3] (node positions of each element).
    p = p0 (1 + A exp(-|x - x_c|^2 / w^2)), rho = rho0 (p / p0)^(1/gamma),
    u = 0, E = p / (gamma - 1).
    """
    d = nodes - np.asarray(center, dtype=np.float64)
    r2 = np.einsum("kni,kni->kn", d, d)
    p = p0 * (1.0 + amplitude * np.exp(-r2 / (width * width)))
    rho = rho0 * (p / p0) ** (1.0 / gamma)
    q = np.zeros((nodes.shape[0], 5, nodes.shape[1]), dtype=np.float64)
    q[:, 0] = rho
    q[:, 4] = p / (gamma - 1.0)
    return q


def uniform_state(K, Np, rho, vel, p, gamma):
    """Conserved state [K, 5, Np] of a uniform flow."""
    q = np.empty((K, 5, Np), dtype=np.float64)
    u = np.asarray(vel, dtype=np.float64)
    q[:, 0] = rho
    q[:, 1:4] = (rho * u)[None, :, None]
    q[:, 4] = p / (gamma - 1.0) + 0.5 * rho * float(u @ u)
    return q


def random_smooth_state(nodes, gamma, rho0, p0, amplitude, seed=0):
    """Seeded smooth perturbation of all five fields (for parity tests).

    Each field gets a sum of three random plane waves of relative size
    ``amplitude``; velocities are scaled by the sound speed.
    """
    rng = np.random.default_rng(seed)
    c0 = np.sqrt(gamma * p0 / rho0)

    def field():
        f = np.zeros(nodes.shape[:2])
        for _ in range(3):
            k = rng.normal(size=3) * 2.0
            ph = rng.uniform(0, 2 * np.pi)
            f += np.sin(nodes @ k + ph) / 3.0
        return amplitude * f

    rho = rho0 * (1.0 + field())
    p = p0 * (1.0 + field())
    u = np.stack([c0 * field() for _ in range(3)], axis=1)  # [K,3,Np]
    q = np.empty((nodes.shape[0], 5, nodes.shape[1]))
    q[:, 0] = rho
    q[:, 1:4] = rho[:, None, :] * u
    q[:, 4] = p / (gamma - 1.0) + 0.5 * rho * np.sum(u * u, axis=1)
    return q


# SI air at rest, the default free stream of the solver's workloads
GAMMA = 1.4
RHO0_SI = 1.225
P0_SI = 101325.0


# ---------------------------------------------------------------- horn workload
# Boundary ids of ``horn_in_room``'s face tags
HORN_OUTER, HORN_WALL, HORN_MOUTHPIECE = 0, 1, 2


def horn_radius(x, bore=0.006, bell=0.06, x0=1.05, m=0.7):
    """Bessel-flared horn profile r(x) = bore (x0 - x)^-m, clamped to
    [bore, bell]: a short cylindrical bore (x < x0 - 1) and then the flare,
    r(1) = 0.0488 for the defaults. The horn's axis is the x axis and its
    mouthpiece the plane x = 0 (section 1.2 builds the paper's trumpet the same
    way: a straight bore, a flare, rotated about the axis)."""
    x = np.asarray(x, dtype=np.float64)
    r = bore * np.power(np.maximum(x0 - x, 1e-300), -m)
    return np.clip(r, bore, bell)


def _graded(h0, length, growth):
    """Positions 0 = y_0 < ... < y_n = length: the first spacing is exactly h0
    (a wall thickness, a cap), the following ones grow geometrically by about
    ``growth`` (scaled together so the last position is ``length``)."""
    if length <= h0:
        return np.array([0.0, length])
    if growth <= 1.0:
        n = max(1, int(round((length - h0) / h0)))
        return np.concatenate([[0.0], h0 + np.linspace(0.0, length - h0, n + 1)])
    n = max(1, int(np.ceil(np.log1p((length - h0) * (growth - 1.0) / (h0 * growth)) / np.log(growth))))
    rest = np.cumsum(h0 * growth ** np.arange(1, n + 1))
    return np.concatenate([[0.0, h0], h0 + rest * ((length - h0) / rest[-1])])


# the outer shapes of section 1.2 (Table 1) around the horn
HORN_SHAPES = ("box", "cylinder", "sphere", "cone", "scone")
_COS45 = np.sqrt(0.5)


def _outer_shape(shape, enclose, L, Rl, H, behind, rad1_0, sensor_dx=0.01):
    """Outer surface of a horn domain (section 1.2, Table 1). Returns a dict:

    x_lo, x_hi  the first and last lattice plane (the flat ends before any map)
    side(x)     outer radius of the lattice's last ring on each plane; a box
                or cylinder of that radius is meshed first
    radius      for the cylinder-based shapes, that constant radius
    cap_hi      None, or rho -> x of a curved right end (planes bent onto it)
    map         None, or (norm, xc, R, q): a radial map in the (x - xc, rho)
                half-plane, p -> p (1 - beta (1 - |p|_inf / |p|_n)),
                beta = (|p|_inf / R)^q, that takes the cylinder's side and
                flat ends onto a sphere (n = 2) or a 45-degree cone (n = 1)
                of radius R about (xc, 0, 0), and leaves points near the
                centre (and the plane x = xc) in place.

    Type B domains (``enclose`` False) start at the bell plane x = L; type A
    domains reach ``behind`` past the mouthpiece plane x = 0 on the axis.

    box, cylinder   flat ends at x = -behind (A) or L (B) and L + Rl; side H
                    (the box's square cross-section is blended in the caller)
    sphere     A: the ball through x = -behind and x = L + Rl on the axis
                  (centre (L + Rl - behind) / 2, radius (L + Rl + behind) / 2)
               B: the half-ball in front of the bell plane, centred on the
                  bell's centre, radius Rl (the rotated hemisphere)
    cone       A: apex on the axis at x = -behind, flat base at x = L + Rl,
                  side through radius H at x = L + sensor_dx (just above
                  sensor 1 of Table 2); the apex is cut off by a flat face
                  where the radius is halfway between the horn's outer
                  radius and the cone's radius at the mouthpiece plane
               B: base disc of radius Rl in the bell plane, apex on the axis
                  at x = L + Rl (a 45-degree side, facing the bell)
    scone      A: the spherical cone (sector): the A cone's apex, side and
                  cut, closed by the sphere about the apex through x = L + Rl
                  (it meets the side at a right angle)"""
    def const(R):
        return lambda x: np.full_like(np.asarray(x, dtype=np.float64), R)
    if shape in ("box", "cylinder"):
        return dict(x_lo=-behind if enclose else L, x_hi=L + Rl, side=const(H), radius=H,
                    cap_hi=None, map=None)
    if shape == "sphere":
        if enclose:
            xc, R = 0.5 * (L + Rl - behind), 0.5 * (L + Rl + behind)
            return dict(x_lo=xc - R, x_hi=xc + R, side=const(R), radius=R, cap_hi=None,
                        map=("l2", xc, R, 2.0))
        return dict(x_lo=L, x_hi=L + Rl, side=const(Rl), radius=Rl, cap_hi=None,
                    map=("l2", L, Rl, 2.0))
    if shape == "cone" and not enclose:
        return dict(x_lo=L, x_hi=L + Rl, side=const(Rl), radius=Rl, cap_hi=None,
                    map=("l1", L, Rl, 0.5))
    if shape in ("cone", "scone"):
        if not enclose:
            raise ValueError("the spherical cone is a type A domain (behind > 0)")
        xa = -behind
        k = H / (L + sensor_dx - xa)

        def side(x):
            return k * (np.asarray(x, dtype=np.float64) - xa)
        x_lo = xa + (rad1_0 + 0.5 * (float(side(0.0)) - rad1_0)) / k
        if shape == "cone":
            return dict(x_lo=x_lo, x_hi=L + Rl, side=side, radius=None, cap_hi=None, map=None)
        Rs = L + Rl - xa

        def cap_hi(rho):
            return xa + np.sqrt(np.maximum(Rs * Rs - rho * rho, 0.0))
        return dict(x_lo=x_lo, x_hi=xa + Rs / np.sqrt(1.0 + k * k), side=side, radius=None,
                    cap_hi=cap_hi, map=None)
    raise ValueError(f"shape must be one of {HORN_SHAPES}")


def _ring_offsets(width, n, first):
    """Offsets of rings 0..n from the inner radius across a gap of ``width``
    (per plane): geometric with first spacing ``first`` where the gap holds
    n such spacings, else uniform. Returns [planes, n + 1]."""
    width = np.asarray(width, dtype=np.float64)
    j = np.arange(n + 1, dtype=np.float64)
    out = np.empty(width.shape + (n + 1,))
    geo = width > n * first * (1.0 + 1e-12)
    out[~geo] = width[~geo, None] * j / n
    if np.any(geo):
        wg = width[geo]
        lo, hi = np.ones_like(wg) * (1.0 + 1e-12), np.full_like(wg, 4.0)
        while np.any(first * (hi ** n - 1.0) / (hi - 1.0) < wg):
            hi = np.where(first * (hi ** n - 1.0) / (hi - 1.0) < wg, 2.0 * hi, hi)
        for _ in range(200):                     # bisection for the growth factor
            mid = 0.5 * (lo + hi)
            big = first * (mid ** n - 1.0) / (mid - 1.0) > wg
            hi = np.where(big, mid, hi)
            lo = np.where(big, lo, mid)
        g = 0.5 * (lo + hi)
        out[geo] = first * (g[:, None] ** j - 1.0) / (g[:, None] - 1.0)
        out[geo] *= (wg / out[geo][:, -1])[:, None]
    return out


def horn_in_room(m1=3, room_length=1.02, room_half=1.0, shape="box", growth=1.12,
                 horn_length=1.0, wall=0.002, aspect=1.0, behind=0.0, profile=horn_radius):
    """A flared horn and the room around it, meshed without a mesh generator.

    Two domain types of section 1.2 (Table 1): with ``behind = 0`` the room
    lies in front of the bell only (type B, the bell-front domains: nothing
    behind the bell plane); with ``behind > 0`` the room encloses the whole
    horn and reaches ``behind`` past its mouthpiece plane (type A): the horn's
    wall (thickness ``wall``) and a cap of the same thickness behind the
    mouthpiece are solid.

    Logical lattice: planes ix along the axis, and a square lattice (i, j) in
    [-m, m]^2 across it. The inner block max(|i|, |j|) <= m1 maps onto the
    disc of radius r(x) = ``profile(x)`` (the horn's interior, continued
    behind the mouthpiece and in front of the bell with the end radii; the
    same square-to-disc blend as ``ball``); ring 1 onto the annulus of width
    ``wall`` around it (the wall, or on the bell plane its rim); rings 2..
    onto annuli whose widths grow by ``growth`` out to the room's side wall,
    blending from circles to the square of half-width ``room_half``
    (``shape="box"``) or staying circles of that radius (``"cylinder"``).
    Horn planes are spaced ``aspect`` times the local cross-section cell
    r(x)/m1; room planes grow from ``wall`` by ``growth`` away from the bell
    (and from the mouthpiece). Every kept cell is split into six tetrahedra
    (the Kuhn chains of ``kuhn_cube``, mirrored across the axis planes so
    the four quadrants are mirror images).

    Face tags: HORN_MOUTHPIECE on the horn's end disc at x = 0 (the inflow
    pulse of section 2.4), HORN_WALL on every face of the solid (the horn's
    inner and outer surfaces, the bell rim, the cap; slip walls, Eq. 4),
    HORN_OUTER on the room's outer boundary (pass-through).

    Returns ``(xyz, EToV, face_tag, info)``; ``info`` has the bell plane,
    element counts, and the sensor analogues of Table 2.
    """
    if shape not in HORN_SHAPES:
        raise ValueError(f"shape must be one of {HORN_SHAPES}")
    m1 = int(m1)
    if m1 < 1:
        raise ValueError("m1 must be >= 1")
    enclose = behind > 0.0
    rad1_0 = float(profile(np.asarray(0.0))) + wall
    spec = _outer_shape(shape, enclose, horn_length, room_length, room_half, behind, rad1_0)
    x_lo, x_hi, side, cap_hi = spec["x_lo"], spec["x_hi"], spec["side"], spec["cap_hi"]
    r_cyl = room_half if spec["radius"] is None else spec["radius"]
    if enclose and x_lo >= -2.0 * wall:
        raise ValueError("the domain must reach further behind the mouthpiece")
    # planes along the axis: behind the mouthpiece, along the horn, in front
    xh = [0.0]
    while xh[-1] < horn_length:
        xh.append(xh[-1] + aspect * float(profile(xh[-1])) / m1)
    xh = np.asarray(xh) * (horn_length / xh[-1])
    back = -_graded(wall, -x_lo, growth)[:0:-1] if enclose else np.zeros(0)
    i0 = len(back)                       # plane of the mouthpiece
    i1 = i0 + len(xh) - 1                # plane of the bell
    xs = np.concatenate([back, xh, horn_length + _graded(wall, x_hi - horn_length, growth)[1:]])
    NX = len(xs) - 1
    r_max = float(profile(np.asarray(horn_length)))
    if r_cyl <= r_max + 2 * wall:
        raise ValueError("the room must be wider than the bell and its rim")
    # ring fractions beyond the wall (from the bell's cross-section)
    rho = (r_max + wall) + _graded(wall, r_cyl - r_max - wall, growth)
    psi = (rho - rho[0]) / (rho[-1] - rho[0])          # 0 at ring 1 .. 1 at the side wall
    round_ = spec["radius"] is None                     # a side radius that changes along x
    if round_:
        # rings of a surface of revolution whose radius changes along the
        # axis: per plane, first spacing one wall thickness and geometric
        # growth out to the side (uniform where the gap is narrow)
        rad1_x = profile(np.clip(xs, 0.0, horn_length)) + wall
        gap = side(xs) - rad1_x
        if np.any(gap <= wall):
            raise ValueError("the outer surface comes too close to the horn")
        nr = len(_graded(wall, float(gap.max()), growth)) - 1
        ring_off = _ring_offsets(gap, nr, wall)            # [planes, nr + 1]
        m = m1 + 1 + nr
    else:
        m = m1 + len(rho)
    beta = 1.0 if shape == "box" else 0.0

    # vertex positions on the full logical lattice
    g = np.arange(-m, m + 1)
    IX, I, J = np.meshgrid(np.arange(NX + 1), g, g, indexing="ij")
    IX, I, J = IX.ravel(), I.ravel(), J.ravel()
    S = np.maximum(np.abs(I), np.abs(J))
    L2 = np.hypot(I, J).astype(np.float64)
    safe = np.where(L2 > 0, L2, 1.0)
    x = xs[IX]
    R = profile(np.clip(x, 0.0, horn_length))
    yz = np.zeros((IX.size, 2))
    inner = S <= m1
    v = np.stack([I, J], axis=1) / m1
    linf = S / m1
    gfac = 1.0 - linf * (1.0 - np.where(L2 > 0, S / safe, 1.0))
    yz[inner] = (R[:, None] * v * gfac[:, None])[inner]
    outer = ~inner
    rad1 = R + wall
    dir_c = np.stack([I, J], axis=1) / safe[:, None]
    if round_:
        kr = np.clip(S - m1 - 1, 0, nr)                 # ring index beyond the wall
        radk = rad1 + ring_off[IX, kr]
        yz_o = radk[:, None] * dir_c
    else:
        kr = np.clip(S - m1 - 1, 0, len(psi) - 1)
        radk = rad1 + (r_cyl - rad1) * psi[kr]
        bk = beta * psi[kr]
        dir_s = np.stack([I, J], axis=1) / np.where(S > 0, S, 1)[:, None]
        yz_o = radk[:, None] * ((1.0 - bk)[:, None] * dir_c + bk[:, None] * dir_s)
    yz[outer] = yz_o[outer]
    # a curved right end: the flat end plane is bent onto the end surface,
    # the bend fading out towards the bell plane (weight 0 there) so the
    # planes stay ordered along every lattice line; a point at radius rho of
    # a plane whose side radius is side(x) takes the bend of radius
    # rho s_hi / side(x) of the end plane, so the side itself does not move
    rr = np.hypot(yz[:, 0], yz[:, 1])
    if cap_hi is not None:
        s_hi = float(side(np.asarray(x_hi)))
        rhat = np.minimum(rr * s_hi / np.maximum(side(x), 1e-300), s_hi)
        b = cap_hi(rhat) - x_hi
        wgt = np.clip((x - horn_length) / (x_hi - horn_length), 0.0, 1.0) ** 2
        x = x + wgt * b
        rr = np.hypot(yz[:, 0], yz[:, 1])
    if spec["map"] is not None:
        # the cylinder onto the sphere or cone. In the (a, rho) half-plane
        # the map p -> p g, g = 1 - beta (1 - f), f = |p|_inf / |p|_n of
        # degree 0 and beta of degree q, has Jacobian g (1 - (1 + q) beta (1 - f)),
        # positive for q < 1 / (1 - 1/sqrt 2) - 1 (n = 2) or q < 1 (n = 1).
        # The horn (interior, wall, cap: rings up to the wall's outer one
        # between the cap's back and the bell) is held in place; its image
        # would move by at most |p|^3 / R^2 there.
        norm, xc, Rm, q = spec["map"]
        a = x - xc
        pinf = np.maximum(np.abs(a), rr)
        pn = np.hypot(a, rr) if norm == "l2" else np.abs(a) + rr
        f = np.where(pn > 0, pinf / np.where(pn > 0, pn, 1.0), 1.0)
        g = 1.0 - (pinf / Rm) ** q * (1.0 - f)
        if enclose:
            held = (S <= m1 + 1) & (x >= -wall - 1e-15) & (x <= horn_length + 1e-15)
            g = np.where(held, 1.0, g)
        x = xc + a * g
        yz = yz * g[:, None]
    xyz_all = np.column_stack([x, yz])

    # cells
    W = 2 * m + 1

    def vid(a, b, c):
        return (a * W + (b + m)) * W + (c + m)

    cx, ci, cj = np.meshgrid(np.arange(NX), np.arange(-m, m), np.arange(-m, m), indexing="ij")
    cx, ci, cj = cx.ravel(), ci.ravel(), cj.ravel()
    smax = np.maximum(np.maximum(np.abs(ci), np.abs(ci + 1)), np.maximum(np.abs(cj), np.abs(cj + 1)))
    in_horn = (cx >= i0) & (cx < i1)
    if enclose:
        solid = (in_horn & (smax == m1 + 1)) | ((cx == i0 - 1) & (smax <= m1 + 1))
        keep = ~solid
    else:
        keep = (cx >= i1) | (in_horn & (smax <= m1))
    cx, ci, cj = cx[keep], ci[keep], cj[keep]
    cells = np.stack([cx, ci, cj], axis=1)
    step = np.stack([np.ones_like(cx), np.where(ci >= 0, 1, -1), np.where(cj >= 0, 1, -1)], axis=1)
    start = cells + (step < 0)
    tets = []
    for perm in _PERMS:
        corner = start.copy()
        chain = [corner.copy()]
        for axis in perm:
            corner = corner.copy()
            corner[:, axis] += step[:, axis]
            chain.append(corner)
        tets.append(np.stack([vid(q[:, 0], q[:, 1], q[:, 2]) for q in chain], axis=1))
    EToV = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int64)
    tet_cx = np.repeat(cx, 6)
    # orientation from the logical lattice; the map must agree with it everywhere
    lat = np.column_stack([IX, I, J]).astype(np.float64)

    def signed(P):
        p = P[EToV]
        return np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])

    neg = signed(lat) < 0
    EToV[neg, 1], EToV[neg, 2] = EToV[neg, 2].copy(), EToV[neg, 1].copy()
    if np.any(signed(xyz_all) <= 0):
        raise ValueError("horn map folded a cell: lower growth or aspect")
    used, inv = np.unique(EToV.ravel(), return_inverse=True)
    EToV = inv.reshape(EToV.shape).astype(np.int32)
    xyz = xyz_all[used].copy()
    lix, ls = IX[used], S[used]

    # boundary faces (faces met once) and their tags
    fv = np.array([(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)])
    faces = np.sort(EToV[:, fv], axis=2).reshape(-1, 3).astype(np.int64)
    key = (faces[:, 0] * len(used) + faces[:, 1]) * len(used) + faces[:, 2]
    _, first, count = np.unique(key, return_inverse=True, return_counts=True)
    bnd = count[first] == 1
    fx, fs = lix[faces], ls[faces]
    fcx = np.repeat(tet_cx, 4)
    outer_f = np.all(fs == m, axis=1) | np.all(fx == NX, axis=1)
    if enclose:
        outer_f |= np.all(fx == 0, axis=1)
    else:
        outer_f |= np.all(fx == i1, axis=1) & (fs.max(axis=1) > m1 + 1)
    mouth = np.all(fx == i0, axis=1) & (fs.max(axis=1) <= m1) & (fcx >= i0)
    tag = np.full(faces.shape[0], -1, dtype=np.int8)
    tag[bnd] = HORN_WALL
    tag[bnd & outer_f] = HORN_OUTER
    tag[bnd & mouth] = HORN_MOUTHPIECE
    face_tag = tag.reshape(-1, 4)
    _fix_orientation(xyz, EToV)
    horn_cells = (cx >= i0) & (cx < i1) & (np.maximum(np.maximum(np.abs(ci), np.abs(ci + 1)),
                                                        np.maximum(np.abs(cj), np.abs(cj + 1))) <= m1)
    names = {("box", True): "A-cube", ("box", False): "B-half-cube", ("sphere", True): "A-sphere",
             ("sphere", False): "B-half-sphere", ("cone", True): "A-cone", ("cone", False): "B-half-cone",
             ("scone", True): "A-scone", ("cylinder", True): "A-cylinder",
             ("cylinder", False): "B-half-cylinder"}
    info = {
        "bell_x": horn_length,
        "bell_radius": r_max,
        "type": "A" if enclose else "B",
        "name": names[(shape, enclose)],
        "n_horn": int(6 * np.count_nonzero(horn_cells)),
        "n_room": int(EToV.shape[0] - 6 * np.count_nonzero(horn_cells)),
        "horn_elements": np.repeat(horn_cells, 6),
        "planes": (i0, i1 - i0, NX - i1),
        "rings": m - m1,
        # Table 2 positions relative to the bell and the room's walls
        "sensors": np.array([[horn_length + 0.01, room_half - 0.01, 0.0],
                             [horn_length + 1.00, 0.0, 0.0],
                             [horn_length + 1.01, 0.0, 0.0],
                             [horn_length + 0.37, 0.57, 0.0]]),
    }
    return xyz, EToV, face_tag, info
