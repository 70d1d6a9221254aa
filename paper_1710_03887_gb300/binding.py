"""Python binding of the C ABI in include/dg_euler.h (argument marshalling only).

Every function of the header is exposed under the same name on ``lib`` (a
ctypes handle); ``Solver`` wraps a context for numpy / torch callers. Device
pointers may come from torch tensors (``tensor.data_ptr()``); the library
never holds on to them. There is no fallback: if the shared library cannot be
loaded the import of ``lib`` fails with the reason.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

import numpy as np

from . import build_lib

DG_OK = 0
DG_ERR_ARG = -1
DG_ERR_MESH = -2
DG_ERR_CUDA = -3
DG_ERR_ORDER = -4
DG_ERR_NONFINITE = -5
DG_ERR_UNSUPPORTED = -6
DG_ERR_TIMEOUT = -7
DG_ERR_BOUNDS = -8
DG_BUILD_BOUNDS_CHECKS = 1

DG_BC_FREESTREAM = 0
DG_BC_CHARACTERISTIC = 1
DG_BC_SLIP_WALL = 2
DG_BC_LEARNED = 3
DG_BC_INFLOW_PULSE = 4
DG_MLP_NPARAMS = 5317

DG_PREC_FP64 = 0
DG_PREC_F32 = 1
DG_PREC_F32_TC = 2
DG_PREC_MODAL = 3
DG_PREC_F32_TC1 = 4


class dg_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("rho0", C.c_double), ("p0", C.c_double),
                ("u0", C.c_double * 3), ("default_bc", C.c_int32), ("precision", C.c_int32)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_SIGS = {
    "dg_create": (C.c_int, [C.c_int, C.POINTER(dg_params), C.POINTER(_P)]),
    "dg_destroy": (C.c_int, [_P]),
    "dg_last_error": (C.c_char_p, [_P]),
    "dg_set_stream": (C.c_int, [_P, _P]),
    "dg_upload_mesh": (C.c_int, [_P, C.c_int64, _P, C.c_int64, _P, _P, _P]),
    "dg_set_bc": (C.c_int, [_P, C.c_int, C.c_int]),
    "dg_sizes": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "dg_node_coords": (C.c_int, [_P, _P]),
    "dg_get_geometry": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "dg_face_pairs": (C.c_int, [_P, _P, _P]),
    "dg_stable_dt": (C.c_int, [_P, _P, C.c_double, _D]),
    "dg_reference_operators": (C.c_int, [C.c_int, _P, _P, _P, _P, _P, _P]),
    "dg_set_state": (C.c_int, [_P, _P, C.c_double]),
    "dg_set_state_device": (C.c_int, [_P, _P, C.c_double]),
    "dg_get_state": (C.c_int, [_P, _P, _D]),
    "dg_get_state_device": (C.c_int, [_P, _P, _D]),
    "dg_step": (C.c_int, [_P, C.c_int, C.c_double]),
    "dg_eval_rhs": (C.c_int, [_P, _P]),
    "dg_set_probes": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "dg_read_probes": (C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_int)]),
    "dg_read_boundary_flux": (C.c_int, [_P, _P]),
    "dg_conserved_totals": (C.c_int, [_P, _P]),
    "dg_sync": (C.c_int, [_P]),
    "dg_build_flags": (C.c_int, [C.POINTER(C.c_int)]),
    "dg_bounds_selftest": (C.c_int, [_P]),
    "dg_set_kernel_timing": (C.c_int, [_P, C.c_int]),
    "dg_read_kernel_timing": (C.c_int, [_P, _D, C.POINTER(C.c_int64)]),
    "dg_weighted_totals_static": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int, _P, _P]),
    "dg_reference_mass": (C.c_int, [C.c_int, _P]),
    "dg_modal_quadrature": (C.c_int, [C.c_int, _P, _P, _P, _P]),
    "dg_modal_operators": (C.c_int, [C.c_int, _P, _P, _P, _P, _P]),
    "dg_set_bc_mlp": (C.c_int, [_P, _P, C.c_double]),
    "dg_get_bc_mlp": (C.c_int, [_P, _P]),
    "dg_set_trace_faces": (C.c_int, [_P, C.c_int64, _P, _P]),
    "dg_sample_traces": (C.c_int, [_P, _P, _P, _P]),
    "dg_upload_geometry": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "dg_set_inflow": (C.c_int, [_P, C.c_double, C.c_double]),
    "dg_mlp_loss_grad": (C.c_int, [_P, _P, _P, C.c_int64, _D, _P]),
    "dg_mlp_train": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int, C.c_double, _P]),
    "dg_mlp_forward": (C.c_int, [_P, _P, C.c_int64, _P]),
    "dg_set_owned": (C.c_int, [_P, C.c_int64]),
    "dg_set_halo": (C.c_int, [_P, C.c_int64, _P, _P, C.c_int64, _P, _P]),
    "dg_halo_pack": (C.c_int, [_P, _P]),
    "dg_halo_unpack": (C.c_int, [_P, _P]),
    "dg_step_stages": (C.c_int, [_P, C.c_int, C.c_double]),
    "dg_stage_index": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
}

_lib = None


def header_symbols():
    """Names of the functions declared in include/*.h."""
    import re
    names = []
    for h in sorted((Path(__file__).resolve().parent.parent / "include").glob("*.h")):
        text = h.read_text()
        names += re.findall(r"^\s*(?:int|const char\*)\s+(dg_\w+)\s*\(", text, flags=re.M)
    return names


def load(build=True):
    """Load (building first if needed) the shared library and declare signatures.
    With the environment variable DG_EULER_BUILD=debug the process loads the
    debug variant (device bounds checks; ``build_lib.build(debug=True)``)."""
    global _lib
    if _lib is not None:
        return _lib
    debug = os.environ.get("DG_EULER_BUILD", "") == "debug"
    if build:
        path = build_lib.build(debug=debug)
    else:
        path = build_lib.LIB_DEBUG if debug else build_lib.LIB
    if not Path(path).exists():
        raise OSError(f"{path} is missing: the CUDA library was not built")
    lib = C.CDLL(str(path))
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def build_flags():
    """dg_build_flags of the loaded library (DG_BUILD_BOUNDS_CHECKS for the
    debug build)."""
    f = C.c_int(0)
    rc = load().dg_build_flags(C.byref(f))
    if rc:
        raise DGError(rc, "dg_build_flags")
    return f.value


class DGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dg error {code}: {msg}")
        self.code = code


def _ptr(a):
    """Address of a numpy array (C-contiguous) or a torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _require(x, shape, dtype, name, device=False):
    """Refuse a buffer the library would read or write past, or misread:
    another shape (None matches any extent), element type or layout, or a
    host buffer where the library expects device memory (``device=True``)
    and the other way round. The C ABI sees only a pointer, so this is the
    last place a size can be checked."""
    if x is None:
        return
    got = tuple(x.shape)
    if len(got) != len(shape) or any(e is not None and g != e for g, e in zip(got, shape)):
        raise ValueError(f"{name}: expected shape {shape}, got {got}")
    if hasattr(x, "data_ptr"):                                  # torch tensor
        import torch
        ok = x.dtype == getattr(torch, np.dtype(dtype).name) and x.is_contiguous() \
            and bool(x.is_cuda) == device
    else:
        ok = x.dtype == dtype and x.flags.c_contiguous and not device
    if not ok:
        where = "device (CUDA)" if device else "host"
        raise ValueError(f"{name}: expected a C-contiguous {np.dtype(dtype).name} {where} buffer")


def reference_mass(order):
    """Mass matrix of the library's reference element (host only)."""
    lib = load()
    Np = (order + 1) * (order + 2) * (order + 3) // 6
    M = np.zeros((Np, Np))
    rc = lib.dg_reference_mass(order, _ptr(M))
    if rc != DG_OK:
        raise DGError(rc, "dg_reference_mass failed")
    return M


def reference_operators(order):
    """Library-built reference operators (host only): dict of numpy arrays."""
    lib = load()
    Np = (order + 1) * (order + 2) * (order + 3) // 6
    Nfp = (order + 1) * (order + 2) // 2
    rst = np.zeros((3, Np))
    Dr, Ds, Dt = (np.zeros((Np, Np)) for _ in range(3))
    LIFT = np.zeros((Np, 4 * Nfp))
    Fmask = np.zeros((4, Nfp), dtype=np.int32)
    rc = lib.dg_reference_operators(order, _ptr(rst), _ptr(Dr), _ptr(Ds), _ptr(Dt), _ptr(LIFT),
                                    _ptr(Fmask))
    if rc != DG_OK:
        raise DGError(rc, "dg_reference_operators failed")
    return dict(r=rst[0], s=rst[1], t=rst[2], Dr=Dr, Ds=Ds, Dt=Dt, LIFT=LIFT, Fmask=Fmask)


def modal_quadrature(order):
    """Gauss rules of the paper's discretisation (host only): volume points
    and weights [Nq, 4] (r, s, t, w), face points and weights [Nfq, 3] (u, v, w)."""
    lib = load()
    nq, nfq = C.c_int32(), C.c_int32()
    rc = lib.dg_modal_quadrature(order, None, None, C.byref(nq), C.byref(nfq))
    if rc != DG_OK:
        raise DGError(rc, "dg_modal_quadrature failed")
    vol, face = np.zeros((nq.value, 4)), np.zeros((nfq.value, 3))
    rc = lib.dg_modal_quadrature(order, _ptr(vol), _ptr(face), None, None)
    if rc != DG_OK:
        raise DGError(rc, "dg_modal_quadrature failed")
    return vol, face


def modal_operators(order):
    """Operators of the paper's discretisation on nodal values (host only):
    dict with Iq [Nq, Np], Sv [3, Np, Nq], Ifn [4, 7, Nfq, Nfp], Sf [4, 7, Np, Nfq], wf [Nfq]."""
    lib = load()
    Np = (order + 1) * (order + 2) * (order + 3) // 6
    Nfp = (order + 1) * (order + 2) // 2
    Nq, Nfq = (order + 1) ** 3, (order + 1) ** 2
    out = dict(Iq=np.zeros((Nq, Np)), Sv=np.zeros((3, Np, Nq)), Ifn=np.zeros((4, 7, Nfq, Nfp)),
               Sf=np.zeros((4, 7, Np, Nfq)), wf=np.zeros(Nfq))
    rc = lib.dg_modal_operators(order, *(_ptr(out[k]) for k in ("Iq", "Sv", "Ifn", "Sf", "wf")))
    if rc != DG_OK:
        raise DGError(rc, "dg_modal_operators failed")
    return out


class Solver:
    """One solver context (order p, free stream, float64)."""

    def __init__(self, order, gamma=1.4, rho0=1.225, p0=101325.0, u0=(0.0, 0.0, 0.0),
                 default_bc=DG_BC_CHARACTERISTIC, precision=DG_PREC_FP64):
        self.lib = load()
        prm = dg_params(gamma, rho0, p0, (C.c_double * 3)(*u0), default_bc, precision)
        h = _P()
        rc = self.lib.dg_create(order, C.byref(prm), C.byref(h))
        if rc != DG_OK:
            raise DGError(rc, "dg_create failed (order or parameters)")
        self.h = h
        self.order = order
        self.precision = precision
        self.K = 0
        self.Np = (order + 1) * (order + 2) * (order + 3) // 6
        self.Nfp = (order + 1) * (order + 2) // 2

    def _check(self, rc):
        if rc != DG_OK:
            raise DGError(rc, self.lib.dg_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.dg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle):
        self._check(self.lib.dg_set_stream(self.h, stream_handle))

    def upload_mesh(self, xyz, EToV, face_tag=None, vert_class=None):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        EToV = np.ascontiguousarray(EToV, dtype=np.int32)
        ft = None if face_tag is None else np.ascontiguousarray(face_tag, dtype=np.int8)
        vc = None if vert_class is None else np.ascontiguousarray(vert_class, dtype=np.int64)
        _require(xyz, (None, 3), np.float64, "xyz")
        _require(EToV, (None, 4), np.int32, "EToV")
        _require(ft, (EToV.shape[0], 4), np.int8, "face_tag")
        _require(vc, (xyz.shape[0],), np.int64, "vert_class")
        self._check(self.lib.dg_upload_mesh(self.h, xyz.shape[0], _ptr(xyz), EToV.shape[0],
                                            _ptr(EToV), _ptr(ft), _ptr(vc)))
        self.K = EToV.shape[0]

    def set_bc(self, bc_id, mode):
        self._check(self.lib.dg_set_bc(self.h, bc_id, mode))

    def set_inflow(self, amplitude, alpha):
        self._check(self.lib.dg_set_inflow(self.h, float(amplitude), float(alpha)))

    def node_coords(self):
        out = np.zeros((self.K, self.Np, 3))
        self._check(self.lib.dg_node_coords(self.h, _ptr(out)))
        return out

    def geometry(self):
        K = self.K
        g = dict(J=np.zeros(K), drdx=np.zeros((K, 3, 3)), nrm=np.zeros((K, 4, 3)),
                 sJ=np.zeros((K, 4)), EToE=np.zeros((K, 4), np.int32),
                 EToF=np.zeros((K, 4), np.int8), bc=np.zeros((K, 4), np.int8))
        self._check(self.lib.dg_get_geometry(self.h, *(_ptr(g[k]) for k in
                                                       ("J", "drdx", "nrm", "sJ", "EToE", "EToF", "bc"))))
        return g

    def face_pairs(self):
        """(vol_node [K,4,Nfp] int64, face_node [K,4,Nfp] int32): the other
        side's volume node (e2 * Np + n) and its face-node position for
        every face node, as the stage kernels decode them; -1 on boundary faces."""
        vol = np.zeros((self.K, 4, self.Nfp), dtype=np.int64)
        fac = np.zeros((self.K, 4, self.Nfp), dtype=np.int32)
        self._check(self.lib.dg_face_pairs(self.h, _ptr(vol), _ptr(fac)))
        return vol, fac

    def stable_dt(self, q, cfl=0.5):
        q = np.ascontiguousarray(q, dtype=np.float64)
        self._check_state_buffer(q, "stable_dt")
        dt = C.c_double()
        self._check(self.lib.dg_stable_dt(self.h, _ptr(q), cfl, C.byref(dt)))
        return dt.value

    def _check_state_buffer(self, x, name):
        """K * 5 * Np float64 values, on the host or (torch) on the GPU."""
        _require(x, (self.K, 5, self.Np), np.float64, name,
                 device=bool(getattr(x, "is_cuda", False)))

    def set_state(self, q, t=0.0):
        """q: numpy [K,5,Np] (host) or a torch tensor of that shape (CPU or CUDA), float64."""
        if hasattr(q, "data_ptr"):
            self._check_state_buffer(q, "set_state")
            fn = self.lib.dg_set_state_device if q.is_cuda else self.lib.dg_set_state
            self._check(fn(self.h, q.data_ptr(), t))
        else:
            qa = np.ascontiguousarray(q, dtype=np.float64)
            self._check_state_buffer(qa, "set_state")
            self._check(self.lib.dg_set_state(self.h, _ptr(qa), t))

    def get_state(self, out=None):
        """Copy the state into ``out`` (numpy, or a CPU or CUDA torch tensor,
        float64 [K,5,Np]) or a new array; returns (q, t)."""
        t = C.c_double()
        if out is None:
            out = np.zeros((self.K, 5, self.Np))
        self._check_state_buffer(out, "get_state")
        if hasattr(out, "is_cuda") and out.is_cuda:
            self._check(self.lib.dg_get_state_device(self.h, out.data_ptr(), C.byref(t)))
        elif hasattr(out, "data_ptr"):
            self._check(self.lib.dg_get_state(self.h, out.data_ptr(), C.byref(t)))
        else:
            self._check(self.lib.dg_get_state(self.h, _ptr(out), C.byref(t)))
        return out, t.value

    def step(self, n, dt):
        self._check(self.lib.dg_step(self.h, int(n), float(dt)))

    def eval_rhs(self):
        out = np.zeros((self.K, 5, self.Np))
        self._check(self.lib.dg_eval_rhs(self.h, _ptr(out)))
        return out

    def set_probes(self, xyz, capacity=1024):
        xyz = np.ascontiguousarray(np.atleast_2d(xyz), dtype=np.float64)
        _require(xyz, (None, 3), np.float64, "probe positions")
        self._check(self.lib.dg_set_probes(self.h, xyz.shape[0], _ptr(xyz), capacity))
        self.nprobe = xyz.shape[0]

    def read_probes(self, max_steps=1 << 30, out=None):
        n = getattr(self, "nprobe", 0)
        if out is None:
            cap = min(max_steps, 1 << 16)
            out = np.zeros((cap, max(n, 1), 5))
            max_steps = cap
        else:
            _require(out, (None, n, 5), np.float64, "read_probes out")
            max_steps = min(max_steps, out.shape[0])          # never more rows than out holds
        got = C.c_int()
        self._check(self.lib.dg_read_probes(self.h, max_steps, _ptr(out), C.byref(got)))
        return out[: got.value, :n]

    def boundary_flux(self):
        out = np.zeros(5)
        self._check(self.lib.dg_read_boundary_flux(self.h, _ptr(out)))
        return out

    def totals(self):
        out = np.zeros(5)
        self._check(self.lib.dg_conserved_totals(self.h, _ptr(out)))
        return out

    def sync(self):
        self._check(self.lib.dg_sync(self.h))

    def bounds_selftest(self):
        """Debug build: latch a failed bounds check on the device (no
        out-of-range access); the next synchronising call raises DG_ERR_BOUNDS."""
        self._check(self.lib.dg_bounds_selftest(self.h))

    # -- learned closure
    def set_bc_mlp(self, w, radius):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == DG_MLP_NPARAMS
        self._check(self.lib.dg_set_bc_mlp(self.h, _ptr(w), float(radius)))

    def get_bc_mlp(self):
        w = np.zeros(DG_MLP_NPARAMS, dtype=np.float32)
        self._check(self.lib.dg_get_bc_mlp(self.h, _ptr(w)))
        return w

    def upload_geometry(self, drdx, J, nrm, Fscale, EToE, EToF, orient, bc=None):
        """Mesh given by its geometric factors and connectivity (see the header)."""
        K = int(np.asarray(J).shape[0])
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (drdx, J, nrm, Fscale)]
        e2e = np.ascontiguousarray(EToE, dtype=np.int32)
        e2f = np.ascontiguousarray(EToF, dtype=np.int8)
        ori = np.ascontiguousarray(orient, dtype=np.int8)
        b = None if bc is None else np.ascontiguousarray(bc, dtype=np.int8)
        for x, shape, name in zip(a, ((K, 3, 3), (K,), (K, 4, 3), (K, 4)), ("drdx", "J", "nrm", "Fscale")):
            _require(x, shape, np.float64, name)
        _require(e2e, (K, 4), np.int32, "EToE")
        for x, name in ((e2f, "EToF"), (ori, "orient"), (b, "bc")):
            _require(x, (K, 4), np.int8, name)
        self._check(self.lib.dg_upload_geometry(self.h, K, *(_ptr(x) for x in a), _ptr(e2e), _ptr(e2f),
                                                _ptr(ori), None if b is None else _ptr(b)))
        self.K = K

    def set_trace_faces(self, elem, face):
        elem = np.ascontiguousarray(elem, dtype=np.int32).ravel()
        face = np.ascontiguousarray(face, dtype=np.int8).ravel()
        _require(face, elem.shape, np.int8, "trace face numbers")
        self._check(self.lib.dg_set_trace_faces(self.h, elem.size, _ptr(elem), _ptr(face)))
        self.ntrace = elem.size

    def sample_traces(self, X, Y, amp=None):
        """Fill device tensors X [ntrace*Nfp, 12], Y [ntrace*Nfp, 5] and, if
        given, amp [ntrace*Nfp] (float32)."""
        n = getattr(self, "ntrace", 0) * self.Nfp
        _require(X, (n, 12), np.float32, "X", device=True)
        _require(Y, (n, 5), np.float32, "Y", device=True)
        _require(amp, (n,), np.float32, "amp", device=True)
        self._check(self.lib.dg_sample_traces(self.h, X.data_ptr(), Y.data_ptr(),
                                              None if amp is None else amp.data_ptr()))

    @staticmethod
    def _samples(X, Y):
        _require(X, (None, 12), np.float32, "X", device=True)
        _require(Y, (X.shape[0], 5), np.float32, "Y", device=True)

    def mlp_loss_grad(self, X, Y):
        self._samples(X, Y)
        loss = C.c_double()
        grad = np.zeros(DG_MLP_NPARAMS, dtype=np.float32)
        self._check(self.lib.dg_mlp_loss_grad(self.h, X.data_ptr(), Y.data_ptr(), X.shape[0],
                                              C.byref(loss), _ptr(grad)))
        return loss.value, grad

    def mlp_train(self, X, Y, iters, lr):
        self._samples(X, Y)
        hist = np.zeros(max(iters, 1))
        self._check(self.lib.dg_mlp_train(self.h, X.data_ptr(), Y.data_ptr(), X.shape[0], int(iters),
                                          float(lr), _ptr(hist)))
        return hist[:iters]

    def mlp_forward(self, X, out):
        _require(X, (None, 12), np.float32, "X", device=True)
        _require(out, (X.shape[0], 5), np.float32, "out", device=True)
        self._check(self.lib.dg_mlp_forward(self.h, X.data_ptr(), X.shape[0], out.data_ptr()))

    # ---- partitioned meshes (own elements first, then halo copies)
    def set_owned(self, K_own):
        self._check(self.lib.dg_set_owned(self.h, int(K_own)))
        self.K_own = int(K_own)

    def set_halo(self, send_elem, send_face, recv_elem, recv_face):
        se = np.ascontiguousarray(send_elem, dtype=np.int32).ravel()
        sf = np.ascontiguousarray(send_face, dtype=np.int8).ravel()
        re_ = np.ascontiguousarray(recv_elem, dtype=np.int32).ravel()
        rf = np.ascontiguousarray(recv_face, dtype=np.int8).ravel()
        _require(sf, se.shape, np.int8, "send faces")
        _require(rf, re_.shape, np.int8, "receive faces")
        self._check(self.lib.dg_set_halo(self.h, se.size, _ptr(se), _ptr(sf), re_.size, _ptr(re_),
                                         _ptr(rf)))
        self.n_send, self.n_recv = se.size, re_.size

    def halo_dtype(self):
        """Element type of halo buffers: the state's own representation."""
        return (np.float32 if self.precision in (DG_PREC_F32, DG_PREC_F32_TC, DG_PREC_F32_TC1)
                else np.float64)

    def halo_pack(self, buf):
        """buf: CUDA tensor [n_send, 5, Nfp] of halo_dtype()."""
        _require(buf, (getattr(self, "n_send", 0), 5, self.Nfp), self.halo_dtype(), "send buffer",
                 device=True)
        self._check(self.lib.dg_halo_pack(self.h, buf.data_ptr()))

    def halo_unpack(self, buf):
        """buf: CUDA tensor [n_recv, 5, Nfp] of halo_dtype()."""
        _require(buf, (getattr(self, "n_recv", 0), 5, self.Nfp), self.halo_dtype(),
                 "receive buffer", device=True)
        self._check(self.lib.dg_halo_unpack(self.h, buf.data_ptr()))

    def step_stages(self, n, dt):
        self._check(self.lib.dg_step_stages(self.h, int(n), float(dt)))

    def stage_index(self):
        """(next stage, stages per step)."""
        k, n = C.c_int(), C.c_int()
        self._check(self.lib.dg_stage_index(self.h, C.byref(k), C.byref(n)))
        return k.value, n.value

    def set_kernel_timing(self, enable=True):
        self._check(self.lib.dg_set_kernel_timing(self.h, int(enable)))

    def read_kernel_timing(self):
        """(summed stage-kernel milliseconds, launches) since the last read."""
        ms = C.c_double()
        n = C.c_int64()
        self._check(self.lib.dg_read_kernel_timing(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value
