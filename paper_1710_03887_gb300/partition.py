"""Element partition of one mesh across ranks, and the halo exchange.

The DG discretisation couples an element to its face neighbours only, through
the surface term of Eq. 10, and the domain is a union of elements (Appendix
A, Eq. 9); so a mesh splits into element sets, one per rank (one GPU each),
that exchange, once per Runge-Kutta stage, the traces on the faces between
them (cut faces): 5 conserved values at each of the Nfp face nodes.

* ``partition_elements``: Morton slabs -- the elements sorted along the
  Morton curve of their centroids and cut into runs of near-equal length.
* ``local_mesh``: one rank's mesh: its own elements (in global order) followed
  by copies of the neighbours across its cut faces (halo elements), the
  face tags (faces of halo elements that lead nowhere locally get
  ``HALO_TAG``), and the exchange plan: per neighbour rank, the own faces whose
  traces it sends and the halo faces it receives into, both sorted by (global
  id of the element on the sending side, its face), so a receive row is the
  same face's send row on the neighbour.
* ``exchange``: moves the packed send rows to the neighbours and receives
  theirs (torch.distributed point-to-point: NCCL between GPUs, gloo on CPU).
* ``PartitionedSolver``: a library context on one rank's mesh that packs,
  exchanges and unpacks before every stage (dg_halo_pack, dg_halo_unpack,
  dg_step_stages) and reduces totals and the boundary ledger over the ranks.

Host logic only: every stage's arithmetic runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import workloads as W

# vertices of the four faces of a tetrahedron, in the library's face order
FACE_VERTS = np.array([(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)])
HALO_TAG = 7        # boundary id of halo faces that lead nowhere on this rank


def face_neighbours(EToV):
    """(EToE, EToF) [K, 4] from shared vertex triples; -1 on boundary faces.
    ValueError for a triple met more than twice (a non-manifold mesh)."""
    EToV = np.asarray(EToV, dtype=np.int64)
    K = EToV.shape[0]
    faces = np.sort(EToV[:, FACE_VERTS], axis=2).reshape(-1, 3)
    order = np.lexsort((faces[:, 2], faces[:, 1], faces[:, 0]))
    fs = faces[order]
    same = np.all(fs[1:] == fs[:-1], axis=1)
    if np.any(same[1:] & same[:-1]):
        raise ValueError("a face is shared by more than two elements")
    i = np.nonzero(same)[0]
    a, b = order[i], order[i + 1]
    EToE = np.full(K * 4, -1, dtype=np.int64)
    EToF = np.full(K * 4, -1, dtype=np.int64)
    EToE[a], EToF[a] = b // 4, b % 4
    EToE[b], EToF[b] = a // 4, a % 4
    return EToE.reshape(K, 4), EToF.reshape(K, 4)


def partition_elements(xyz, EToV, nparts):
    """Rank of every element: Morton slabs of near-equal size."""
    K = len(EToV)
    if not 1 <= nparts <= K:
        raise ValueError("need 1 <= nparts <= K")
    perm = W.morton_order(np.asarray(xyz), np.asarray(EToV))
    bounds = np.round(np.linspace(0, K, nparts + 1)).astype(np.int64)
    part = np.empty(K, dtype=np.int32)
    for r in range(nparts):
        part[perm[bounds[r]:bounds[r + 1]]] = r
    return part


@dataclass
class LocalMesh:
    rank: int
    xyz: np.ndarray            # local vertices
    EToV: np.ndarray           # [K_own + K_halo, 4] int32, own elements first
    face_tag: np.ndarray       # [K, 4] int8: -1 interior, else boundary id
    K_own: int
    l2g: np.ndarray            # global element id of each local element
    peers: list = field(default_factory=list)       # neighbour ranks, ascending
    send_elem: np.ndarray = None                    # own cut faces, peer by peer
    send_face: np.ndarray = None
    send_off: np.ndarray = None                     # [len(peers) + 1] row offsets
    recv_elem: np.ndarray = None                    # halo faces, peer by peer
    recv_face: np.ndarray = None
    recv_off: np.ndarray = None


def local_mesh(xyz, EToV, part, rank, face_tag=None, neighbours=None):
    """Rank ``rank``'s mesh and exchange plan (see the module docstring).
    ``neighbours`` = face_neighbours(EToV) if already computed."""
    xyz = np.asarray(xyz, dtype=np.float64)
    EToV = np.asarray(EToV)
    part = np.asarray(part)
    K = EToV.shape[0]
    EToE, EToF = face_neighbours(EToV) if neighbours is None else neighbours
    gtag = (np.where(EToE < 0, 0, -1) if face_tag is None else np.asarray(face_tag)).astype(np.int8)
    own = np.nonzero(part == rank)[0]
    if own.size == 0:
        raise ValueError(f"rank {rank} owns no element")
    nb = EToE[own]
    cut = (nb >= 0) & (part[np.maximum(nb, 0)] != rank)
    halo = np.unique(nb[cut])
    l2g = np.concatenate([own, halo])
    g2l = np.full(K, -1, dtype=np.int64)
    g2l[l2g] = np.arange(l2g.size)
    used, inv = np.unique(EToV[l2g].ravel(), return_inverse=True)
    lE = inv.reshape(-1, 4).astype(np.int32)
    tag = gtag[l2g].copy()
    # halo faces whose neighbour is not on this rank (and not a boundary)
    lnb = EToE[l2g]
    lost = (lnb >= 0) & (g2l[np.maximum(lnb, 0)] < 0)
    tag[lost] = HALO_TAG
    # exchange plan: own cut faces (send) and the matching halo faces (receive)
    oe, of = np.nonzero(cut)                 # own local index, face
    ge2 = nb[oe, of]                         # the neighbour (global) across each cut face
    gf2 = EToF[own[oe], of]                  # ... and its face number
    peer = part[ge2]
    peers = sorted(set(peer.tolist()))
    s_elem, s_face, r_elem, r_face = [], [], [], []
    s_off, r_off = [0], [0]
    for p in peers:
        # send: own faces towards p, sorted by (global own element, face)
        m = peer == p
        key = np.lexsort((of[m], own[oe[m]]))
        s_elem.append(oe[m][key])
        s_face.append(of[m][key])
        s_off.append(s_off[-1] + int(m.sum()))
        # receive: the halo elements of p across those faces, sorted by
        # (global halo element, its face) -- p's send order
        key = np.lexsort((gf2[m], ge2[m]))
        r_elem.append(g2l[ge2[m][key]])
        r_face.append(gf2[m][key])
        r_off.append(r_off[-1] + int(m.sum()))

    def cat(xs, dt):
        return np.concatenate(xs).astype(dt) if xs else np.zeros(0, dtype=dt)
    return LocalMesh(rank=rank, xyz=xyz[used], EToV=lE, face_tag=tag.astype(np.int8),
                     K_own=int(own.size), l2g=l2g, peers=peers,
                     send_elem=cat(s_elem, np.int32), send_face=cat(s_face, np.int8),
                     send_off=np.array(s_off, dtype=np.int64),
                     recv_elem=cat(r_elem, np.int32), recv_face=cat(r_face, np.int8),
                     recv_off=np.array(r_off, dtype=np.int64))


def exchange(local, send_buf, recv_buf, group=None):
    """Send each peer its rows of ``send_buf`` and receive its rows into
    ``recv_buf`` (torch tensors [rows, ...], CUDA with NCCL or CPU with gloo);
    returns when the received rows are usable on the current stream."""
    import torch.distributed as dist
    ops = []
    for i, p in enumerate(local.peers):
        s0, s1 = int(local.send_off[i]), int(local.send_off[i + 1])
        r0, r1 = int(local.recv_off[i]), int(local.recv_off[i + 1])
        ops.append(dist.P2POp(dist.isend, send_buf[s0:s1], p, group))
        ops.append(dist.P2POp(dist.irecv, recv_buf[r0:r1], p, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class PartitionedSolver:
    """One rank of a partitioned run: a library context on ``local`` (own
    elements and halo copies) whose stages are separated by halo exchanges.
    Needs CUDA and an initialised torch.distributed process group: NCCL moves
    the device buffers directly; with ``host_staging`` the packed rows go
    through host memory (for a CPU backend such as gloo)."""

    def __init__(self, order, local, gamma, rho0, p0, precision, device, group=None,
                 modes=None, host_staging=False):
        import torch
        from . import binding as B
        self.local = local
        self.group = group
        self.device = device
        self.S = B.Solver(order, gamma, rho0, p0, precision=precision)
        self.S.set_stream(torch.cuda.current_stream(device).cuda_stream)
        self.S.upload_mesh(local.xyz, local.EToV, face_tag=local.face_tag)
        self.S.set_bc(HALO_TAG, B.DG_BC_FREESTREAM)
        for ident, mode in (modes or {}).items():
            self.S.set_bc(ident, mode)
        self.S.set_owned(local.K_own)
        self.S.set_halo(local.send_elem, local.send_face, local.recv_elem, local.recv_face)
        tdt = getattr(torch, np.dtype(self.S.halo_dtype()).name)
        self.send = torch.empty((local.send_elem.size, 5, self.S.Nfp), dtype=tdt, device=device)
        self.recv = torch.empty((local.recv_elem.size, 5, self.S.Nfp), dtype=tdt, device=device)
        self.host_staging = host_staging
        if host_staging:
            self.send_h = torch.empty(self.send.shape, dtype=tdt).pin_memory()
            self.recv_h = torch.empty(self.recv.shape, dtype=tdt).pin_memory()

    def set_state(self, q, t=0.0):
        """q: this rank's local state [K_own + K_halo, 5, Np] (halo rows are
        overwritten by the first exchange)."""
        self.S.set_state(q, t)

    def exchange_halo(self):
        import torch
        self.S.halo_pack(self.send)
        if self.host_staging:
            self.send_h.copy_(self.send)              # synchronous: the rows are on the host
            exchange(self.local, self.send_h, self.recv_h, self.group)
            self.recv.copy_(self.recv_h)
        else:
            exchange(self.local, self.send, self.recv, self.group)
        self.S.halo_unpack(self.recv)

    def step(self, n, dt):
        _, nstage = self.S.stage_index()
        for _ in range(n * nstage):
            self.exchange_halo()
            self.S.step_stages(1, dt)

    def _allreduce(self, x):
        import torch
        import torch.distributed as dist
        t = torch.tensor(x, dtype=torch.float64,
                         device="cpu" if self.host_staging else self.device)
        dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

    def totals(self):
        """Conserved totals over all ranks (own elements only on each)."""
        return self._allreduce(self.S.totals())

    def boundary_flux(self):
        """Boundary ledger over all ranks."""
        return self._allreduce(self.S.boundary_flux())

    def own_state(self):
        """This rank's own elements' state [K_own, 5, Np] (float64, host)."""
        q, t = self.S.get_state()
        return q[:self.local.K_own], t
