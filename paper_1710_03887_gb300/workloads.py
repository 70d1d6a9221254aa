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
