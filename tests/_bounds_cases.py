"""Cases run on both builds of the library by tests/test_gpu_bounds_build.py.

One process loads one build (``DG_EULER_BUILD=debug`` selects the variant
with device bounds checks), so the test runs ``run_all`` in its own process
on the release build and ``main`` in a child process on the debug build.
The cases reach every index a kernel reads from the mesh tables:

* every arithmetic form, on a jittered cube whose vertex lists are shuffled
  (all six face orientations) with a last tile shorter than the others,
  every kind of outer face (characteristic, slip wall, inflow pulse) and
  probes;
* the learned closure in both float32 forms (its gather of outer-face
  traces and the stage kernels' boundary slots);
* a mesh split across two emulated ranks (halo pack and unpack, neighbour
  ids into halo copies).
"""
import numpy as np

from paper_1710_03887_gb300 import binding as B
from paper_1710_03887_gb300 import partition as PT
from paper_1710_03887_gb300 import workloads as W

SI = dict(gamma=W.GAMMA, rho0=W.RHO0_SI, p0=W.P0_SI)
PRECS = {"fp64": B.DG_PREC_FP64, "f32": B.DG_PREC_F32, "f32_tc": B.DG_PREC_F32_TC,
         "modal": B.DG_PREC_MODAL, "f32_tc1": B.DG_PREC_F32_TC1}
FORMS = [("fp64", 2), ("fp64", 3), ("f32", 3), ("f32", 4), ("f32_tc", 3), ("f32_tc", 4), ("f32_tc1", 3),
         ("modal", 2)]
PROBES = np.array([[0.1, 0.2, -0.3], [-0.5, 0.4, 0.6], [0.8, -0.7, 0.05]])


def mesh():
    """Jittered 3^3 cube (162 tets), vertex lists shuffled; boundary faces
    tagged 0, 1, 2 by the axis their outward direction is closest to."""
    xyz, EToV = W.kuhn_cube(3, jitter=0.12, seed=7)
    E = W.shuffle_vertices(xyz, EToV, seed=8)
    EToE, _ = PT.face_neighbours(E)
    tags = np.full(E.shape, -1, dtype=np.int8)
    for f, fv in enumerate(PT.FACE_VERTS):
        fc = xyz[E[:, fv]].mean(axis=1)          # on a cube face: one coordinate is +-1
        b = EToE[:, f] < 0
        tags[b, f] = np.argmax(np.abs(fc[b]), axis=1)
    return xyz, E, tags


def _solver(p, prec, xyz, E, tags, modes):
    S = B.Solver(p, precision=PRECS[prec], **SI)
    S.upload_mesh(xyz, E, face_tag=tags)
    for ident, mode in modes.items():
        S.set_bc(ident, mode)
    S.set_inflow(0.05, 2.0e4)
    return S


def _pulse(S):
    return W.gaussian_pulse_state(S.node_coords(), W.GAMMA, W.RHO0_SI, W.P0_SI, 0.05, 0.5,
                                  center=(0.3, -0.2, 0.1))


def _weights():
    rng = np.random.default_rng(3)
    return (0.05 * rng.standard_normal(B.DG_MLP_NPARAMS)).astype(np.float32)


def run_all(steps=3):
    """Arrays of every case, keyed by case."""
    xyz, E, tags = mesh()
    out = {}
    modes = {0: B.DG_BC_CHARACTERISTIC, 1: B.DG_BC_INFLOW_PULSE, 2: B.DG_BC_SLIP_WALL}
    for prec, p in FORMS:
        S = _solver(p, prec, xyz, E, tags, modes)
        q0 = _pulse(S)
        dt = S.stable_dt(q0, 0.5)
        S.set_state(q0)
        S.set_probes(PROBES, capacity=steps)
        S.step(steps, dt)
        q, _ = S.get_state()
        out[f"{prec}_p{p}_q"] = q
        out[f"{prec}_p{p}_probes"] = S.read_probes(steps)
        out[f"{prec}_p{p}_ledger"] = S.boundary_flux()
        S.sync()
        S.close()
    lmodes = {0: B.DG_BC_LEARNED, 1: B.DG_BC_CHARACTERISTIC, 2: B.DG_BC_SLIP_WALL}
    for prec in ("f32", "f32_tc"):
        S = _solver(3, prec, xyz, E, tags, lmodes)
        S.set_bc_mlp(_weights(), 1.0)
        q0 = _pulse(S)
        dt = S.stable_dt(q0, 0.5)
        S.set_state(q0)
        S.step(steps, dt)
        q, _ = S.get_state()
        out[f"learned_{prec}_q"] = q
        S.sync()
        S.close()
    out["partition_q"] = _partition(xyz, E, steps)
    return out


def _partition(xyz, E, steps):
    """Two emulated ranks (float32, p = 3): every stage packs, routes each
    rank's rows to the other's receive buffer on the device, unpacks and
    advances; the stitched own states."""
    import torch
    dev = torch.device("cuda:0")
    part = PT.partition_elements(xyz, E, 2)
    locs = [PT.local_mesh(xyz, E, part, r) for r in range(2)]
    ctx, send, recv = [], [], []
    S0 = B.Solver(3, precision=B.DG_PREC_F32, **SI)
    S0.upload_mesh(xyz, E)
    q0 = _pulse(S0)
    dt = S0.stable_dt(q0, 0.5)
    S0.close()
    stream = torch.cuda.current_stream(dev).cuda_stream
    for L in locs:
        S = B.Solver(3, precision=B.DG_PREC_F32, **SI)
        S.set_stream(stream)
        S.upload_mesh(L.xyz, L.EToV, face_tag=L.face_tag)
        S.set_bc(PT.HALO_TAG, B.DG_BC_FREESTREAM)
        S.set_owned(L.K_own)
        S.set_halo(L.send_elem, L.send_face, L.recv_elem, L.recv_face)
        S.set_state(q0[L.l2g])
        send.append(torch.empty((L.send_elem.size, 5, S.Nfp), dtype=torch.float32, device=dev))
        recv.append(torch.empty((L.recv_elem.size, 5, S.Nfp), dtype=torch.float32, device=dev))
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
    for S, L in zip(ctx, locs):
        q, _ = S.get_state()
        stitched[L.l2g[:L.K_own]] = q[:L.K_own]
        S.sync()
        S.close()
    return stitched


def selftest():
    """The debug build's failed-check path: a check that fails on purpose is
    reported as DG_ERR_BOUNDS by the next synchronising call, which clears
    it; the context then steps and synchronises cleanly. Returns the codes
    seen (the error's, then 0 for the clean step)."""
    xyz, E, tags = mesh()
    S = _solver(2, "f32", xyz, E, tags, {0: B.DG_BC_CHARACTERISTIC})
    q0 = _pulse(S)
    S.set_state(q0)
    S.bounds_selftest()
    codes = []
    try:
        S.sync()
        codes.append(0)
    except B.DGError as e:
        codes.append(e.code)
    S.step(1, S.stable_dt(q0, 0.5))
    S.sync()
    codes.append(0)
    S.close()
    return np.array(codes)


def main(path):
    """Child process (debug build): every case, the build flags and the
    self-test, saved to ``path``."""
    out = run_all()
    out["flags"] = np.array(B.build_flags())
    out["selftest"] = selftest()
    np.savez(path, **out)
