"""Element partition and halo exchange on the CPU (no GPU).

* The plan: for every pair of ranks, the rows one sends are the rows the
  other receives (same global faces, same order); every cut face appears
  once on each side; the local meshes are valid meshes whose own elements
  keep their global neighbours and boundary tags.
* A partitioned run with two gloo ranks: each rank's local mesh (own
  elements and halo copies) is advanced by the float64 oracle stage by stage
  (in the test only: the library's stages run on the GPU), with the face
  traces of the cut faces exchanged before every stage through the
  library's plan and ``partition.exchange``. The stitched own states equal
  the single-domain oracle run to rounding, and the ranks' totals add up to
  the single-domain totals: the partition changes nothing but where an
  element is computed (Appendix A, Eq. 9: the domain is the union of the
  elements; Eq. 10 couples an element to its face neighbours only).
"""
import os
import socket
import sys

import numpy as np
import pytest

from paper_1710_03887_gb300 import partition as PT
from paper_1710_03887_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_face_neighbours_match_the_oracle_connectivity():
    from oracle.geometry import Geometry
    from oracle.reference_element import ReferenceElement
    xyz, EToV = W.kuhn_cube(3, jitter=0.1, seed=2)
    EToV = W.shuffle_vertices(xyz, EToV, seed=3)
    EToE, EToF = PT.face_neighbours(EToV)
    g = Geometry(ReferenceElement(1), xyz, EToV)
    assert np.array_equal(EToE < 0, g.boundary)
    # the two sides of a face name each other
    e, f = np.nonzero(EToE >= 0)
    assert np.array_equal(EToE[EToE[e, f], EToF[e, f]], e)
    assert np.array_equal(EToF[EToE[e, f], EToF[e, f]], f)
    # their vertex triples agree
    t1 = np.sort(EToV[e[:, None], PT.FACE_VERTS[f]], axis=1)
    t2 = np.sort(EToV[EToE[e, f][:, None], PT.FACE_VERTS[EToF[e, f]]], axis=1)
    assert np.array_equal(t1, t2)


@pytest.mark.parametrize("nparts", [2, 3, 5])
def test_plan_rows_match_between_ranks(nparts):
    xyz, EToV = W.kuhn_cube(6, jitter=0.1, seed=1)
    K = len(EToV)
    tag = np.where(PT.face_neighbours(EToV)[0] < 0, 0, -1).astype(np.int8)
    part = PT.partition_elements(xyz, EToV, nparts)
    sizes = np.bincount(part, minlength=nparts)
    assert sizes.sum() == K and sizes.max() - sizes.min() <= 1
    EToE, EToF = PT.face_neighbours(EToV)
    locs = [PT.local_mesh(xyz, EToV, part, r, face_tag=tag) for r in range(nparts)]
    ncut = 0
    for r, L in enumerate(locs):
        assert np.array_equal(L.l2g[:L.K_own], np.nonzero(part == r)[0])
        # own elements keep their global neighbours (through local ids) and tags
        gE, _ = PT.face_neighbours(L.EToV)
        own = L.l2g[:L.K_own]
        want = EToE[own]
        got = np.where(gE[:L.K_own] >= 0, L.l2g[np.maximum(gE[:L.K_own], 0)], -1)
        assert np.array_equal(got, want)
        assert np.array_equal(L.face_tag[:L.K_own], tag[own])
        # halo faces leading nowhere locally carry the halo tag
        hE, _ = PT.face_neighbours(L.EToV)
        lost = (hE[L.K_own:] < 0) & (EToE[L.l2g[L.K_own:]] >= 0)
        assert np.all(L.face_tag[L.K_own:][lost] == PT.HALO_TAG)
        # volumes stay positive (same vertex order)
        v = L.xyz[L.EToV]
        vol = np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0])
        assert np.all(vol > 0)
        for i, s in enumerate(L.peers):
            Ls = locs[s]
            j = Ls.peers.index(r)
            # rows r receives from s ...
            rr = slice(L.recv_off[i], L.recv_off[i + 1])
            recv = np.stack([L.l2g[L.recv_elem[rr]], L.recv_face[rr]], axis=1)
            # ... are the rows s sends to r, in the same order
            ss = slice(Ls.send_off[j], Ls.send_off[j + 1])
            send = np.stack([Ls.l2g[Ls.send_elem[ss]], Ls.send_face[ss]], axis=1)
            assert np.array_equal(recv, send)
            ncut += len(send)
            # and every such face is a face between the two parts
            g_e, g_f = send[:, 0], send[:, 1]
            assert np.all(part[g_e] == s) and np.all(part[EToE[g_e, g_f]] == r)
    e, f = np.nonzero(EToE >= 0)
    assert ncut == np.count_nonzero(part[e] != part[EToE[e, f]])


def test_partition_rejects_bad_counts():
    xyz, EToV = W.kuhn_cube(2)
    with pytest.raises(ValueError):
        PT.partition_elements(xyz, EToV, 0)
    with pytest.raises(ValueError):
        PT.partition_elements(xyz, EToV, len(EToV) + 1)


def _pack(L, q, Fmask):
    """Rows [n_send, 5, Nfp] of the own cut faces' traces (test-side packing)."""
    return np.ascontiguousarray(np.transpose(q[L.send_elem[:, None], :, Fmask[L.send_face]],
                                             (0, 2, 1)))


def _unpack(L, q, buf, Fmask):
    q[L.recv_elem[:, None], :, Fmask[L.recv_face]] = np.transpose(buf, (0, 2, 1))


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle.euler_dg import CHARACTERISTIC, FREESTREAM, LSRK_A, LSRK_B, LSRK_C, Gas, Solver
    from oracle.geometry import Geometry
    from oracle.reference_element import ReferenceElement
    from paper_1710_03887_gb300 import partition as PT
    from paper_1710_03887_gb300 import workloads as W
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        p, steps = 1, 20
        xyz, EToV = W.kuhn_cube(6)                          # configuration C1: 1296 elements
        gas = Gas(W.GAMMA, W.RHO0_SI, W.P0_SI)
        part = PT.partition_elements(xyz, EToV, world)
        L = PT.local_mesh(xyz, EToV, part, rank)
        ref = ReferenceElement(p)
        geom = Geometry(ref, L.xyz, L.EToV)
        bc_id = np.where(L.face_tag < 0, 0, L.face_tag).astype(np.int64)
        orc = Solver(geom, gas, bc_id=bc_id, bc_mode={0: CHARACTERISTIC, PT.HALO_TAG: FREESTREAM})
        # the C1 pulse on the local nodes; dt of the whole mesh (the same on every rank)
        q = W.gaussian_pulse_state(geom.x, W.GAMMA, W.RHO0_SI, W.P0_SI, 0.005, 0.15)
        full = Geometry(ref, xyz, EToV)
        dt = Solver(full, gas).stable_dt(W.gaussian_pulse_state(full.x, W.GAMMA, W.RHO0_SI,
                                                                 W.P0_SI, 0.005, 0.15), 0.5)
        send = torch.zeros((L.send_elem.size, 5, ref.Nfp), dtype=torch.float64)
        recv = torch.zeros((L.recv_elem.size, 5, ref.Nfp), dtype=torch.float64)
        res = np.zeros_like(q)
        t = 0.0
        for _ in range(steps):
            for k in range(5):
                send.copy_(torch.from_numpy(_pack(L, q, ref.Fmask)))
                PT.exchange(L, send, recv)
                _unpack(L, q, recv.numpy(), ref.Fmask)
                a, b, c = float(LSRK_A[k]), float(LSRK_B[k]), float(LSRK_C[k])
                res = a * res + dt * orc.rhs(q, t + c * dt)
                q = q + b * res
            t += dt
        own = q[:L.K_own]
        tot = torch.from_numpy(orc.totals(np.concatenate([own, np.zeros_like(q[L.K_own:])])))
        dist.all_reduce(tot)
        out.put((rank, L.l2g[:L.K_own], own, tot.numpy(), dt))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_domain_run():
    import torch.multiprocessing as mp
    from oracle.euler_dg import Gas, Solver
    from oracle.geometry import Geometry
    from oracle.reference_element import ReferenceElement
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in range(2)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    xyz, EToV = W.kuhn_cube(6)
    geom = Geometry(ReferenceElement(1), xyz, EToV)
    gas = Gas(W.GAMMA, W.RHO0_SI, W.P0_SI)
    orc = Solver(geom, gas)
    q0 = W.gaussian_pulse_state(geom.x, W.GAMMA, W.RHO0_SI, W.P0_SI, 0.005, 0.15)
    dt = res[0][4]
    assert dt == res[1][4] == orc.stable_dt(q0, 0.5)
    qo, _, _, _ = orc.run(q0, dt, 20)
    stitched = np.full_like(qo, np.nan)
    for _, ids, own, _, _ in res:
        stitched[ids] = own
    assert not np.isnan(stitched).any()                   # every element owned once
    err = np.abs(stitched - qo).max(axis=(0, 2)) / np.abs(qo - q0).max(axis=(0, 2))
    assert np.all(err < 1e-12), err
    for _, _, _, tot, _ in res:
        np.testing.assert_allclose(tot, orc.totals(qo), rtol=1e-13, atol=1e-13 * np.abs(tot).max())
