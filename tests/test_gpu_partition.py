"""The partitioned mesh on the GPU: contexts on ranks' local meshes (own
elements, then halo copies) with the face traces of cut faces exchanged
before every Runge-Kutta stage (dg_halo_pack / dg_halo_unpack /
dg_step_stages).

* One process, three emulated ranks on one GPU: every context packs, the
  test routes each rank's rows to its neighbours' receive buffers on the
  device (no kernel waits for another: the routing happens between launches),
  every context unpacks and advances one stage. The stitched own states
  equal the single-domain run to rounding: the partition changes which
  element of a face evaluates its flux (a face inside a tile is evaluated
  once, by its lower element; a face between tiles by both, each with its
  own normal), which moves results by an ulp: 1e-14 of each variable's
  largest value in float64, 1e-6 of the perturbation in the float32 forms.
  The ranks' totals and ledgers add up to the single-domain ones to
  rounding.
* Two processes on the same GPU with a gloo group: PartitionedSolver end to
  end (its exchange staged through host memory), the same check.
"""
import os
import socket
import sys

import numpy as np
import pytest

from paper_1710_03887_gb300 import binding as B
from paper_1710_03887_gb300 import partition as PT
from paper_1710_03887_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SI = dict(gamma=W.GAMMA, rho0=W.RHO0_SI, p0=W.P0_SI)
PRECS = {"fp64": B.DG_PREC_FP64, "f32": B.DG_PREC_F32, "f32_tc": B.DG_PREC_F32_TC}


def _mesh():
    xyz, EToV = W.kuhn_cube(6, jitter=0.1, seed=4)             # 1296 elements
    EToV = W.shuffle_vertices(xyz, EToV, seed=5)                  # every face orientation
    return xyz, EToV


def _close(stitched, q_ref, q0, prec):
    """Per variable: float64 to 1e-14 of max |q| (momentum: of rho0 c0 at
    least, the scale of its flux's rounding), float32 forms to 1e-6 of the
    perturbation from the free stream, max |q - (rho0, 0, E0)|."""
    d = np.abs(stitched - q_ref).max(axis=(0, 2))
    if prec == "fp64":
        scale = np.abs(q_ref).max(axis=(0, 2))
        scale[1:4] = np.maximum(scale[1:4], W.RHO0_SI * np.sqrt(W.GAMMA * W.P0_SI / W.RHO0_SI))
        return d / scale < 1e-14
    base = W.uniform_state(q_ref.shape[0], q_ref.shape[2], W.RHO0_SI, (0, 0, 0), W.P0_SI, W.GAMMA)
    return d / np.abs(q_ref - base).max(axis=(0, 2)) < 1e-6


def _single(p, prec, xyz, EToV, q0, dt, steps, dev, setup=None):
    import torch
    S = B.Solver(p, precision=PRECS[prec], **SI)
    S.set_stream(torch.cuda.current_stream(dev).cuda_stream)
    S.upload_mesh(xyz, EToV)
    if setup:
        setup(S)
    S.set_state(q0)
    S.step(steps, dt)
    q, _ = S.get_state()
    out = (q, S.totals(), S.boundary_flux())
    S.close()
    return out


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("p", [1, 3])
def test_emulated_ranks_reproduce_the_single_domain_run(cuda_device, p, prec):
    import torch
    xyz, EToV = _mesh()
    nranks, steps = 3, 6
    part = PT.partition_elements(xyz, EToV, nranks)
    locs = [PT.local_mesh(xyz, EToV, part, r) for r in range(nranks)]
    S0 = B.Solver(p, precision=PRECS[prec], **SI)
    S0.upload_mesh(xyz, EToV)
    nodes = S0.node_coords()
    q0 = W.gaussian_pulse_state(nodes, W.GAMMA, W.RHO0_SI, W.P0_SI, 0.05, 0.4, center=(0.2, -0.1, 0.1))
    dt = S0.stable_dt(q0, 0.5)
    S0.close()
    q_ref, tot_ref, led_ref = _single(p, prec, xyz, EToV, q0, dt, steps, cuda_device)
    stream = torch.cuda.current_stream(cuda_device).cuda_stream
    ctx, send, recv = [], [], []
    for L in locs:
        S = B.Solver(p, precision=PRECS[prec], **SI)
        S.set_stream(stream)
        S.upload_mesh(L.xyz, L.EToV, face_tag=L.face_tag)
        S.set_bc(PT.HALO_TAG, B.DG_BC_FREESTREAM)
        S.set_owned(L.K_own)
        S.set_halo(L.send_elem, L.send_face, L.recv_elem, L.recv_face)
        S.set_state(q0[L.l2g])
        tdt = getattr(torch, np.dtype(S.halo_dtype()).name)
        send.append(torch.empty((L.send_elem.size, 5, S.Nfp), dtype=tdt, device=cuda_device))
        recv.append(torch.empty((L.recv_elem.size, 5, S.Nfp), dtype=tdt, device=cuda_device))
        ctx.append(S)
    assert ctx[0].stage_index() == (0, 5)
    for _ in range(steps * 5):
        for S, b in zip(ctx, send):
            S.halo_pack(b)
        for r, L in enumerate(locs):
            for i, s in enumerate(L.peers):
                j = locs[s].peers.index(r)
                recv[r][L.recv_off[i]:L.recv_off[i + 1]].copy_(
                    send[s][locs[s].send_off[j]:locs[s].send_off[j + 1]])
        for S, b in zip(ctx, recv):
            S.halo_unpack(b)
        for S in ctx:
            S.step_stages(1, dt)
    assert ctx[0].stage_index() == (0, 5)
    stitched = np.full_like(q_ref, np.nan)
    tot, led = np.zeros(5), np.zeros(5)
    for S, L in zip(ctx, locs):
        q, t = S.get_state()
        assert t == pytest.approx(steps * dt, rel=1e-15)
        stitched[L.l2g[:L.K_own]] = q[:L.K_own]
        tot += S.totals()
        led += S.boundary_flux()
        S.close()
    assert not np.isnan(stitched).any()
    assert np.all(_close(stitched, q_ref, q0, prec)), np.abs(stitched - q_ref).max(axis=(0, 2))
    # totals: float64 sums in another order (per rank, then over the ranks);
    # in the float32 forms the summed states themselves differ by float32
    # ulps of the perturbation (~1e-3 of an energy perturbation of ~1e4 at
    # ~2.6e4 nodes): 1e-10 of the totals
    scale = np.abs(tot_ref).max()
    rt = 1e-13 if prec == "fp64" else 1e-10
    np.testing.assert_allclose(tot, tot_ref, rtol=rt, atol=rt * scale)
    np.testing.assert_allclose(led, led_ref, rtol=1e-9, atol=1e-13 * scale)


def test_partition_refusals(cuda_device):
    xyz, EToV = _mesh()
    part = PT.partition_elements(xyz, EToV, 2)
    L = PT.local_mesh(xyz, EToV, part, 0)
    S = B.Solver(2, **SI)
    S.upload_mesh(L.xyz, L.EToV, face_tag=L.face_tag)
    with pytest.raises(B.DGError):
        S.set_owned(0)
    with pytest.raises(B.DGError):
        S.set_owned(len(L.EToV) + 1)
    S.set_owned(L.K_own)
    with pytest.raises(B.DGError):                  # a halo face in the send list
        S.set_halo(L.recv_elem, L.recv_face, L.recv_elem, L.recv_face)
    with pytest.raises(B.DGError):                  # an own face in the receive list
        S.set_halo(L.send_elem, L.send_face, L.send_elem, L.send_face)
    S.set_halo(L.send_elem, L.send_face, L.recv_elem, L.recv_face)
    S.close()
    SM = B.Solver(2, precision=B.DG_PREC_MODAL, **SI)
    SM.upload_mesh(L.xyz, L.EToV, face_tag=L.face_tag)
    with pytest.raises(B.DGError):                  # the paper's face rule follows the numbering
        SM.set_owned(L.K_own)
    SM.close()
    # a step cannot start while one is in progress
    S2 = B.Solver(1, **SI)
    S2.upload_mesh(xyz, EToV)
    q0 = W.uniform_state(len(EToV), S2.Np, W.RHO0_SI, (0, 0, 0), W.P0_SI, W.GAMMA)
    S2.set_state(q0)
    S2.step_stages(2, 1e-6)
    assert S2.stage_index() == (2, 5)
    with pytest.raises(B.DGError):
        S2.step(1, 1e-6)
    S2.step_stages(3, 1e-6)
    S2.step(1, 1e-6)
    S2.set_state(q0)
    assert S2.stage_index() == (0, 5)
    S2.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1710_03887_gb300 import binding as B
    from paper_1710_03887_gb300 import partition as PT
    from paper_1710_03887_gb300 import workloads as W
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        dev = torch.device("cuda:0")
        torch.cuda.set_device(dev)
        xyz, EToV = _mesh()
        part = PT.partition_elements(xyz, EToV, world)
        L = PT.local_mesh(xyz, EToV, part, rank)
        PS = PT.PartitionedSolver(3, L, W.GAMMA, W.RHO0_SI, W.P0_SI, B.DG_PREC_F32, dev,
                                  host_staging=True)
        nodes = PS.S.node_coords()
        q0 = W.gaussian_pulse_state(nodes, W.GAMMA, W.RHO0_SI, W.P0_SI, 0.05, 0.4,
                                    center=(0.2, -0.1, 0.1))
        PS.set_state(q0)
        tot0 = PS.totals()
        PS.step(4, 2e-6)
        q, t = PS.own_state()
        out.put((rank, L.l2g[:L.K_own], q, t, tot0, PS.totals(), PS.boundary_flux()))
        PS.S.close()
    finally:
        dist.destroy_process_group()


def test_partitioned_solver_two_processes(cuda_device):
    import torch.multiprocessing as mp
    xyz, EToV = _mesh()
    S0 = B.Solver(3, precision=B.DG_PREC_F32, **SI)
    S0.upload_mesh(xyz, EToV)
    q0 = W.gaussian_pulse_state(S0.node_coords(), W.GAMMA, W.RHO0_SI, W.P0_SI, 0.05, 0.4,
                                center=(0.2, -0.1, 0.1))
    S0.close()
    q_ref, tot_ref, led_ref = _single(3, "f32", xyz, EToV, q0, 2e-6, 4, cuda_device)
    ctx = mp.get_context("spawn")
    qq = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, qq)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [qq.get(timeout=600) for _ in range(2)]
    for pr in procs:
        pr.join(120)
        assert pr.exitcode == 0
    stitched = np.full_like(q_ref, np.nan)
    for _, ids, q, t, _, tot, led in res:
        stitched[ids] = q
        assert t == pytest.approx(4 * 2e-6, rel=1e-15)
        scale = np.abs(tot_ref).max()
        np.testing.assert_allclose(tot, tot_ref, rtol=1e-10, atol=1e-10 * scale)
        np.testing.assert_allclose(led, led_ref, rtol=1e-9, atol=1e-13 * scale)
    assert np.all(_close(stitched, q_ref, q0, "f32")), np.abs(stitched - q_ref).max(axis=(0, 2))


def _emulated(p, prec, xyz, EToV, q0, dt, steps, dev, nranks=3, setup=None):
    """Stitched own states of emulated ranks (see the module docstring)."""
    import torch
    part = PT.partition_elements(xyz, EToV, nranks)
    locs = [PT.local_mesh(xyz, EToV, part, r) for r in range(nranks)]
    stream = torch.cuda.current_stream(dev).cuda_stream
    ctx, send, recv = [], [], []
    for L in locs:
        S = B.Solver(p, precision=PRECS[prec], **SI)
        S.set_stream(stream)
        S.upload_mesh(L.xyz, L.EToV, face_tag=L.face_tag)
        S.set_bc(PT.HALO_TAG, B.DG_BC_FREESTREAM)
        if setup:
            setup(S)
        S.set_owned(L.K_own)
        S.set_halo(L.send_elem, L.send_face, L.recv_elem, L.recv_face)
        S.set_state(q0[L.l2g])
        tdt = getattr(torch, np.dtype(S.halo_dtype()).name)
        send.append(torch.empty((L.send_elem.size, 5, S.Nfp), dtype=tdt, device=dev))
        recv.append(torch.empty((L.recv_elem.size, 5, S.Nfp), dtype=tdt, device=dev))
        ctx.append(S)
    for _ in range(steps * 5):
        for S, b in zip(ctx, send):
            S.halo_pack(b)
        for r, L in enumerate(locs):
            for i, s in enumerate(L.peers):
                j = locs[s].peers.index(r)
                recv[r][L.recv_off[i]:L.recv_off[i + 1]].copy_(
                    send[s][locs[s].send_off[j]:locs[s].send_off[j + 1]])
        for S, b in zip(ctx, recv):
            S.halo_unpack(b)
        for S in ctx:
            S.step_stages(1, dt)
    stitched = np.full_like(q0, np.nan)
    led = np.zeros(5)
    for S, L in zip(ctx, locs):
        q, _ = S.get_state()
        stitched[L.l2g[:L.K_own]] = q[:L.K_own]
        led += S.boundary_flux()
        S.close()
    return stitched, led


@pytest.mark.parametrize("prec", ["f32", "f32_tc"])
def test_emulated_ranks_with_the_learned_closure(cuda_device, prec):
    """The learned closure on every outer face (a seeded network; the memory
    of each outer-face node advanced by the rank that owns the face) under
    the partition: the stitched own states equal the single-domain run to
    rounding, and the ranks' ledgers add up to its ledger."""
    from oracle import mlp as OM
    xyz, EToV = _mesh()
    rng = np.random.default_rng(21)
    w = (OM.init_params(seed=21) + 0.05 * rng.normal(size=OM.N_PARAMS)).astype(np.float32)
    w[-5 - 64 * 5:] *= 0.2

    def setup(S):
        S.set_bc(0, B.DG_BC_LEARNED)
        S.set_bc_mlp(w, 1.0)
    S0 = B.Solver(3, precision=PRECS[prec], **SI)
    S0.upload_mesh(xyz, EToV)
    q0 = W.gaussian_pulse_state(S0.node_coords(), W.GAMMA, W.RHO0_SI, W.P0_SI, 0.05, 0.6,
                                center=(0.2, -0.1, 0.1))
    dt = S0.stable_dt(q0, 0.5)
    S0.close()
    steps = 6
    q_ref, _, led_ref = _single(3, prec, xyz, EToV, q0, dt, steps, cuda_device, setup)
    stitched, led = _emulated(3, prec, xyz, EToV, q0, dt, steps, cuda_device, setup=setup)
    assert not np.isnan(stitched).any()
    assert np.all(_close(stitched, q_ref, q0, prec)), np.abs(stitched - q_ref).max(axis=(0, 2))
    scale = np.abs(q_ref).max()
    np.testing.assert_allclose(led, led_ref, rtol=1e-9, atol=1e-13 * scale * len(EToV))
    # the closure is in play: the characteristic condition ends elsewhere
    q_char, _, _ = _single(3, prec, xyz, EToV, q0, dt, steps, cuda_device)
    base = W.uniform_state(q0.shape[0], q0.shape[2], W.RHO0_SI, (0, 0, 0), W.P0_SI, W.GAMMA)
    assert np.abs(q_char - q_ref).max() > 1e-4 * np.abs(q_ref - base).max()
