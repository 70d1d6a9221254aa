"""Host side of the C ABI (no GPU needed): symbols, operators, geometry, errors."""
import ctypes

import numpy as np
import pytest

from oracle.geometry import Geometry, inscribed_radius
from oracle.reference_element import ReferenceElement
from paper_1710_03887_gb300 import binding as B
from paper_1710_03887_gb300 import workloads as W


def test_library_exports_every_header_symbol():
    lib = B.load()
    names = B.header_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value
    # the binding declares every header function and nothing else
    assert sorted(B._SIGS) == sorted(names)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_reference_operators_match_oracle(p):
    L = B.reference_operators(p)
    R = ReferenceElement(p)
    for k in "rst":
        np.testing.assert_allclose(L[k], getattr(R, k), atol=1e-15)
    for k in ("Dr", "Ds", "Dt", "LIFT"):
        ref = getattr(R, k)
        np.testing.assert_allclose(L[k], ref, atol=1e-13 * np.abs(ref).max())
    np.testing.assert_array_equal(L["Fmask"], R.Fmask)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_modal_gauss_rules_match_the_oracle(p):
    """The library's own Gauss-Jacobi rules (Newton on the Jacobi recurrence)
    against the oracle's (a library routine), point by point: the collapsed
    products must be the same point sets for the discretisation to agree."""
    from oracle import modal_dg as MD
    vol, face = B.modal_quadrature(p)
    r, s, t, w = MD.tet_rule(2 * p)
    assert vol.shape == (len(w), 4) and len(w) == (p + 1) ** 3
    np.testing.assert_allclose(vol, np.stack([r, s, t, w], axis=1), rtol=0, atol=1e-14)
    u, v, wf = MD.tri_rule(2 * p + 1)
    assert face.shape == (len(wf), 3) and len(wf) == (p + 1) ** 2
    np.testing.assert_allclose(face, np.stack([u, v, wf], axis=1), rtol=0, atol=1e-14)
    with pytest.raises(B.DGError):
        B.modal_quadrature(9)


def test_unsupported_order_is_rejected():
    with pytest.raises(B.DGError) as e:
        B.Solver(7)
    assert e.value.code == B.DG_ERR_UNSUPPORTED


@pytest.mark.parametrize("jitter", [0.0, 0.12])
def test_geometry_and_connectivity_match_oracle(jitter):
    p = 2
    xyz, EToV = W.kuhn_cube(3, jitter=jitter, seed=3)
    S = B.Solver(p)
    S.upload_mesh(xyz, EToV)
    g = S.geometry()
    G = Geometry(ReferenceElement(p), xyz, EToV)
    np.testing.assert_allclose(g["J"], G.J, rtol=1e-14)
    np.testing.assert_allclose(g["drdx"], G.drdx, atol=1e-13)
    np.testing.assert_allclose(g["nrm"], G.nrm, atol=1e-14)
    np.testing.assert_allclose(g["sJ"], G.sJ, rtol=1e-13)
    np.testing.assert_array_equal(g["EToE"] < 0, G.boundary)
    inner = ~G.boundary
    np.testing.assert_array_equal(g["EToE"][inner], G.EToE[inner])
    np.testing.assert_array_equal(g["EToF"][inner], G.EToF[inner])
    np.testing.assert_array_equal(g["bc"][G.boundary], 0)
    np.testing.assert_allclose(S.node_coords(), G.x, atol=1e-15)


def _pairing_meshes():
    xyz, EToV = W.kuhn_cube(3, jitter=0.1, seed=4)
    yield "lattice", xyz, EToV, None
    yield "shuffled", xyz, W.shuffle_vertices(xyz, EToV, seed=1), None
    bx, bE = W.ball(4, 1.0, jitter=0.1, seed=2)
    yield "ball shuffled", bx, W.shuffle_vertices(bx, bE, seed=3), None
    yield "periodic shuffled", xyz, W.shuffle_vertices(xyz, EToV, seed=5), (2.0, 2.0, 2.0)


@pytest.mark.parametrize("p", [1, 3, 4])
def test_face_pairing_matches_the_oracle_for_every_orientation(p):
    """Each face node's partner as the stage kernels decode it (connection
    word + reference face-node tables) is the node the oracle pairs it with
    by coordinates; with shuffled vertex lists all six vertex
    correspondences between the sides of a face occur."""
    from ._cases import orientation_codes
    ref = ReferenceElement(p)
    for name, xyz, EToV, period in _pairing_meshes():
        vclass = W.periodic_vertex_classes(3) if period else None
        S = B.Solver(p)
        S.upload_mesh(xyz, EToV, vert_class=vclass)
        vol, fac = S.face_pairs()
        G = Geometry(ref, xyz, EToV, period=period)
        inner = ~G.boundary
        np.testing.assert_array_equal(vol[G.boundary], -1, err_msg=name)
        np.testing.assert_array_equal(vol[inner], G.vmapP[inner], err_msg=name)
        # the face-node position names the same node
        e2, f2 = G.EToE[inner], G.EToF[inner]
        np.testing.assert_array_equal(ref.Fmask[f2[:, None], fac[inner]], vol[inner] % ref.Np,
                                      err_msg=name)
        # the orientation codes of the tests' convention (uploaded with the
        # oracle's factors) give the same pairing as the library's own
        ids = EToV if period is None else vclass[EToV]              # vertices across the seam
        EToE = np.where(G.boundary, -1, G.EToE)
        codes = orientation_codes(ids, EToE, G.EToF)
        S2 = B.Solver(p)
        S2.upload_geometry(G.drdx, G.J, G.nrm, G.Fscale, EToE, G.EToF, codes)
        np.testing.assert_array_equal(S2.face_pairs()[0], vol, err_msg=name)
        if name != "lattice":
            assert set(codes[inner].tolist()) == set(range(6)), name


def test_one_and_two_element_meshes():
    """The degenerate meshes: one tetrahedron (four boundary faces) and two
    sharing a face, uploaded and paired as the oracle pairs them."""
    xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [1.0, 1.0, 1.0]])
    for EToV in (np.array([[0, 1, 2, 3]]), np.array([[0, 1, 2, 3], [2, 3, 1, 4]])):
        for p in (1, 4):
            S = B.Solver(p)
            S.upload_mesh(xyz, EToV)
            G = Geometry(ReferenceElement(p), xyz, EToV)
            vol, _ = S.face_pairs()
            np.testing.assert_array_equal(S.geometry()["EToE"] < 0, G.boundary)
            np.testing.assert_array_equal(np.where(G.boundary[:, :, None], -1, G.vmapP), vol)


def test_state_buffers_of_another_shape_or_type_are_refused():
    """The library reads and writes K * 5 * Np float64 values through the
    pointers it is given; the binding refuses any other buffer before the
    call (nothing reaches the library here, so no GPU is needed)."""
    import torch
    xyz, EToV = W.kuhn_cube(1)
    S = B.Solver(1)
    S.upload_mesh(xyz, EToV)
    K, Np = S.K, S.Np
    for bad in (np.zeros((K, Np, 5)), np.zeros((K - 1, 5, Np)), torch.zeros((K, 5, Np), dtype=torch.float32)):
        with pytest.raises(ValueError):
            S.set_state(bad)
    for bad in (np.zeros((K, 5, Np), dtype=np.float32), np.zeros((Np, 5, K)).T, np.zeros((K + 1, 5, Np)),
                torch.zeros((K, 5, Np), dtype=torch.float32)):
        with pytest.raises(ValueError):
            S.get_state(bad)
    with pytest.raises(ValueError):
        S.stable_dt(np.ones((K, 5, Np + 1)))
    # every other array argument: shape, element type, host or device
    bad_calls = [
        lambda: B.Solver(1).upload_mesh(xyz[:, :2], EToV),
        lambda: B.Solver(1).upload_mesh(xyz, EToV[:, :3]),
        lambda: B.Solver(1).upload_mesh(xyz, EToV, face_tag=np.zeros((K, 3))),
        lambda: B.Solver(1).upload_mesh(xyz, EToV, vert_class=np.zeros(len(xyz) - 1)),
        lambda: S.set_probes(np.zeros((2, 2))),
        lambda: S.read_probes(4, out=np.zeros((4, 3, 5))),
        lambda: S.upload_geometry(np.zeros((K, 9)), np.ones(K), np.zeros((K, 4, 3)), np.ones((K, 4)),
                                  np.zeros((K, 4)), np.zeros((K, 4)), np.zeros((K, 4))),
        lambda: S.set_trace_faces(np.arange(3), np.zeros(2)),
        lambda: S.mlp_loss_grad(torch.zeros((8, 12)), torch.zeros((8, 5))),          # host tensors
        lambda: S.mlp_forward(torch.zeros((8, 12)), torch.zeros((8, 5), dtype=torch.float64)),
    ]
    for call in bad_calls:
        with pytest.raises(ValueError):
            call()


def test_stable_dt_matches_oracle():
    from oracle.euler_dg import Gas, Solver
    xyz, EToV = W.kuhn_cube(3, jitter=0.1)
    S = B.Solver(3)
    S.upload_mesh(xyz, EToV)
    G = Geometry(ReferenceElement(3), xyz, EToV)
    q = W.gaussian_pulse_state(G.x, W.GAMMA, W.RHO0_SI, W.P0_SI, 0.1, 0.3)
    O = Solver(G, Gas(W.GAMMA, W.RHO0_SI, W.P0_SI))
    assert S.stable_dt(q, 0.5) == pytest.approx(O.stable_dt(q, 0.5), rel=1e-12)
    assert np.all(inscribed_radius(G) > 0)


def test_periodic_vertex_classes_close_the_box():
    xyz, EToV = W.kuhn_cube(3)
    S = B.Solver(1)
    S.upload_mesh(xyz, EToV, vert_class=W.periodic_vertex_classes(3))
    assert np.all(S.geometry()["EToE"] >= 0)


def test_mesh_errors():
    xyz, EToV = W.kuhn_cube(2)
    S = B.Solver(1)
    bad = EToV.copy()
    bad[3, [1, 2]] = bad[3, [2, 1]]                  # inverted element
    with pytest.raises(B.DGError) as e:
        S.upload_mesh(xyz, bad)
    assert e.value.code == B.DG_ERR_MESH
    dup = np.concatenate([EToV, EToV[:1]])           # a face shared by three elements
    with pytest.raises(B.DGError) as e:
        S.upload_mesh(xyz, dup)
    assert e.value.code == B.DG_ERR_MESH
    tags = np.full((EToV.shape[0], 4), -1, np.int8)  # boundary faces left untagged
    with pytest.raises(B.DGError) as e:
        S.upload_mesh(xyz, EToV, face_tag=tags)
    assert e.value.code == B.DG_ERR_MESH
    oob = EToV.copy()
    oob[0, 0] = 10 ** 6
    with pytest.raises(B.DGError):
        S.upload_mesh(xyz, oob)
    with pytest.raises(B.DGError):
        S.set_bc(9, B.DG_BC_CHARACTERISTIC)
    with pytest.raises(B.DGError):
        S.set_bc(0, 17)


def test_calls_out_of_order_fail_cleanly():
    S = B.Solver(1)
    with pytest.raises(B.DGError) as e:
        S.step(1, 1e-3)
    assert e.value.code == B.DG_ERR_ORDER
    lib = B.load()
    assert lib.dg_node_coords(S.h, None) == B.DG_ERR_ARG
    assert lib.dg_destroy(None) == B.DG_OK


def test_upload_geometry_round_trip_and_errors():
    """A mesh re-uploaded through its geometric factors (dg_upload_geometry)
    has the same geometry and stable time step; malformed factors are
    rejected, and calls that need vertices say so."""
    from paper_1710_03887_gb300 import workloads as W
    from ._cases import orientation_codes
    xyz, EToV = W.kuhn_cube(2, jitter=0.1, seed=2)
    S1 = B.Solver(2)
    S1.upload_mesh(xyz, EToV)
    g = S1.geometry()
    ori = orientation_codes(EToV, g["EToE"], g["EToF"])
    Fs = g["sJ"] / g["J"][:, None]
    S2 = B.Solver(2)
    S2.upload_geometry(g["drdx"], g["J"], g["nrm"], Fs, g["EToE"], g["EToF"], ori)
    g2 = S2.geometry()
    for k in ("J", "drdx", "nrm", "EToE", "EToF", "bc"):
        np.testing.assert_array_equal(g2[k], g[k])
    np.testing.assert_allclose(g2["sJ"], g["sJ"], rtol=1e-15)
    q = W.uniform_state(S1.K, S1.Np, 1.225, (0, 0, 0), 101325.0, 1.4)
    assert S2.stable_dt(q) == pytest.approx(S1.stable_dt(q), rel=1e-13)
    with pytest.raises(B.DGError) as ei:
        S2.node_coords()
    assert ei.value.code == B.DG_ERR_ORDER
    with pytest.raises(B.DGError) as ei:
        S2.set_probes([[0.0, 0.0, 0.0]])
    assert ei.value.code == B.DG_ERR_ORDER
    # malformed inputs
    e, f = np.argwhere(g["EToE"] >= 0)[0]
    bad = g["EToE"].copy()
    bad[e, f] = (bad[e, f] + 1) % S1.K
    with pytest.raises(B.DGError) as ei:
        S2.upload_geometry(g["drdx"], g["J"], g["nrm"], Fs, bad, g["EToF"], ori)
    assert ei.value.code == B.DG_ERR_MESH
    bad_o = ori.copy()
    bad_o[e, f] = (bad_o[e, f] + 1) % 6
    with pytest.raises(B.DGError) as ei:
        S2.upload_geometry(g["drdx"], g["J"], g["nrm"], Fs, g["EToE"], g["EToF"], bad_o)
    assert ei.value.code == B.DG_ERR_MESH
    bad_J = g["J"].copy()
    bad_J[3] = -1.0
    with pytest.raises(B.DGError) as ei:
        S2.upload_geometry(g["drdx"], bad_J, g["nrm"], Fs, g["EToE"], g["EToF"], ori)
    assert ei.value.code == B.DG_ERR_MESH
