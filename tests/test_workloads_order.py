"""Element-order helpers of the workload module (CPU): Morton and random
permutations are permutations; the Morton order keeps consecutive elements
close (as close as the lattice order, far closer than a random order) and
keeps the elements of one lattice cell together."""
import numpy as np

from paper_1710_03887_gb300 import workloads as W


def _mean_step(c, perm):
    return np.linalg.norm(np.diff(c[perm], axis=0), axis=1).mean()


def test_orders_are_permutations_with_the_expected_locality():
    xyz, EToV = W.ball(12, 1.0, jitter=0.1, seed=1)
    K = len(EToV)
    c = W.element_centroids(xyz, EToV)
    m = W.morton_order(xyz, EToV)
    r = W.random_order(K, 4)
    for p in (m, r):
        assert np.array_equal(np.sort(p), np.arange(K))
    assert np.array_equal(W.random_order(K, 4), r)            # seeded
    lattice, morton, rand = _mean_step(c, np.arange(K)), _mean_step(c, m), _mean_step(c, r)
    assert morton < 1.2 * lattice and rand > 4 * morton
    # a tile of 32 consecutive elements spans a small box in Morton order
    tiles = c[m][: (K // 32) * 32].reshape(-1, 32, 3)
    assert np.median(np.ptp(tiles, axis=1).max(axis=1)) < 0.5


def test_morton_order_of_a_permuted_mesh_restores_locality():
    xyz, EToV = W.kuhn_cube(6)
    perm = W.random_order(len(EToV), 2)
    shuffled = EToV[perm]
    c = W.element_centroids(xyz, shuffled)
    m = W.morton_order(xyz, shuffled)
    assert _mean_step(c, m) < 0.25 * _mean_step(c, np.arange(len(EToV)))


def test_shuffled_vertex_lists_keep_the_elements():
    """Each element keeps its four vertices, positively oriented, in a
    seeded order that differs from the lattice's for most elements."""
    xyz, EToV = W.kuhn_cube(3, jitter=0.1, seed=3)
    E = W.shuffle_vertices(xyz, EToV, seed=7)
    assert E.shape == EToV.shape and E.dtype == np.int32
    assert np.array_equal(np.sort(E, axis=1), np.sort(EToV, axis=1))
    v = xyz[E]
    vol = np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0])
    assert np.all(vol > 0)
    assert np.mean(np.any(E != EToV, axis=1)) > 0.8
    assert np.array_equal(W.shuffle_vertices(xyz, EToV, seed=7), E)      # seeded
