"""Python binding of the C ABI (include/mbs.h) with the same call names.

Only argument marshalling happens here; every step of the computation runs in
libmbs.so.  Complex blocks of nrhs vectors are passed column-major:

  * numpy arrays (host): shape (rows, nrhs) or (rows,), complex128; results
    come back as numpy arrays of the same form;
  * torch tensors (device): complex128 CUDA tensors of shape (rows, nrhs)
    whose transpose is contiguous (``torch.empty(nrhs, rows).T``), or 1-D;
    results come back as tensors of that layout on the same device.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

try:  # torch is only needed for device-resident arguments
    import torch
except Exception:  # pragma: no cover
    torch = None

PREC_FP64, PREC_MIXED, PREC_FP32 = L.PREC_FP64, L.PREC_MIXED, L.PREC_FP32


class MbsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{L.STATUS.get(status, status)}: {msg}")
        self.status = status


def _lib():
    return L.load()


def default_options(**kw) -> L.mbs_options:
    o = L.mbs_options()
    _lib().mbs_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _is_torch(a) -> bool:
    return torch is not None and isinstance(a, torch.Tensor)


class _Arg:
    """A complex (rows, nrhs) argument as a pointer the library can use."""

    def __init__(self, a, rows=None):
        if _is_torch(a):
            if a.dtype != torch.complex128:
                a = a.to(torch.complex128)
            t = a if a.dim() == 2 else a.reshape(-1, 1)
            if not t.T.is_contiguous():
                t = t.T.contiguous().T
            self.keep = t
            self.ptr = C.c_void_p(t.data_ptr())
            self.rows, self.nrhs = t.shape
            self.torch = True
        else:
            arr = np.asarray(a, dtype=np.complex128)
            self.was_1d = arr.ndim == 1
            t = arr.reshape(-1, 1) if arr.ndim == 1 else arr
            buf = np.ascontiguousarray(t.T)  # [nrhs][rows]
            self.keep = buf
            self.ptr = C.c_void_p(buf.ctypes.data)
            self.rows, self.nrhs = t.shape
            self.torch = False
        if rows and self.rows != rows:
            raise ValueError(f"expected {rows} rows, got {self.rows}")


def _out_like(arg: _Arg, rows: int):
    if arg.torch:
        dev = arg.keep.device
        pin = dev.type == "cpu" and arg.keep.is_pinned()
        t = torch.empty((arg.nrhs, rows), dtype=torch.complex128, device=dev, pin_memory=pin).T
        return t, C.c_void_p(t.data_ptr())
    buf = np.empty((arg.nrhs, rows), dtype=np.complex128)
    return buf, C.c_void_p(buf.ctypes.data)


def _ret(out, arg: _Arg):
    if arg.torch:
        return out
    res = out.T
    return res[:, 0] if getattr(arg, "was_1d", False) else res


def _soa(pts) -> np.ndarray:
    """(count, dim) points -> contiguous SoA float64 buffer (dim * count)."""
    return np.ascontiguousarray(np.asarray(pts, dtype=np.float64).T)


def shapes_bodies_from_workload(wl):
    """ctypes arrays of mbs_shape / mbs_body for an mbs_inputs.Workload."""
    keep = []
    shapes = (L.mbs_shape * len(wl.shapes))()
    for i, sh in enumerate(wl.shapes):
        x, y, z = _soa(sh.x), _soa(sh.y), _soa(sh.z)
        keep += [x, y, z]
        s = shapes[i]
        s.m, s.n, s.p = sh.m, sh.n, sh.p
        s.x = x.ctypes.data_as(C.POINTER(C.c_double))
        s.y = y.ctypes.data_as(C.POINTER(C.c_double))
        s.z = z.ctypes.data_as(C.POINTER(C.c_double))
        s.k, s.eps, s.proxy_radius = int(sh.k), float(sh.eps), float(sh.proxy_radius)
    bodies = (L.mbs_body * wl.T)()
    for t in range(wl.T):
        b = bodies[t]
        b.shape = int(wl.body_shape[t])
        for a in range(3):
            b.c[a] = float(wl.centres[t, a])
        R = wl.rots[t]
        for a in range(9):
            b.R[a] = float(R[a // 3, a % 3])
    return shapes, bodies, keep


class Context:
    """One solver context (mbs_ctx): dimension, wavenumber, options, and the
    device-resident scattering data after build_scattering_matrices."""

    def __init__(self, dim: int, kappa: float, options: L.mbs_options | None = None, **kw):
        self._h = C.c_void_p()
        opt = options if options is not None else default_options(**kw)
        self._check(_lib().mbs_create(dim, kappa, C.byref(opt), C.byref(self._h)))
        self.dim = dim
        self.kappa = kappa
        self.options = opt
        self.N = 0
        self.T = 0

    def _check(self, st):
        if st != L.MBS_OK:
            msg = _lib().mbs_last_error(self._h).decode() if self._h else ""
            raise MbsError(st, msg)

    def close(self):
        if self._h:
            _lib().mbs_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_options(self, **kw):
        for k, v in kw.items():
            setattr(self.options, k, v)
        self._check(_lib().mbs_set_options(self._h, C.byref(self.options)))

    def last_error(self) -> str:
        return _lib().mbs_last_error(self._h).decode()

    # ---- the paper's calls ------------------------------------------------
    def build_scattering_matrices(self, wl):
        shapes, bodies, keep = shapes_bodies_from_workload(wl)
        self._check(_lib().mbs_build_scattering_matrices(self._h, len(wl.shapes), shapes, wl.T,
                                                         bodies))
        N = C.c_int64()
        self._check(_lib().mbs_get_layout(self._h, C.byref(N), None, None))
        self.N = int(N.value)
        self.T = wl.T
        self.Mtot = int(sum(wl.shapes[s].m for s in wl.body_shape))
        self.Nm = int(sum(wl.shapes[s].n for s in wl.body_shape))
        return self

    def get_layout(self):
        N = C.c_int64()
        self._check(_lib().mbs_get_layout(self._h, C.byref(N), None, None))
        off = np.zeros(self.T + 1, dtype=np.int64)
        xyz = np.zeros(self.dim * N.value, dtype=np.float64)
        self._check(_lib().mbs_get_layout(self._h, C.byref(N), off.ctypes.data_as(C.POINTER(C.c_int64)),
                                          C.c_void_p(xyz.ctypes.data)))
        return int(N.value), off, xyz.reshape(self.dim, -1).T.copy()

    def get_shape(self, shape: int):
        k = C.c_int()
        self._check(_lib().mbs_get_shape(self._h, shape, C.byref(k), None, None, None))
        skel = np.zeros(k.value, dtype=np.int32)
        S = np.zeros((k.value, k.value), dtype=np.complex128, order="F")
        eps = C.c_double()
        self._check(_lib().mbs_get_shape(self._h, shape, C.byref(k),
                                         skel.ctypes.data_as(C.POINTER(C.c_int)),
                                         C.c_void_p(S.ctypes.data), C.byref(eps)))
        return {"k": k.value, "skel": skel.astype(np.int64), "S": np.array(S), "eps": eps.value}

    def get_shape_stats(self, shape: int):
        """Figures of one shape's build: rank_b (pivoted QR of B), rank_a_qr
        (pivoted QR of A), rank_a (singular values of A kept), the Jacobi
        sweeps of the SVD and s_norm (Frobenius norm of S)."""
        v = [C.c_int() for _ in range(4)]
        sn = C.c_double()
        self._check(_lib().mbs_get_shape_stats(self._h, shape, *[C.byref(x) for x in v], C.byref(sn)))
        out = dict(zip(("rank_b", "rank_a_qr", "rank_a", "sweeps"), (x.value for x in v)))
        out["s_norm"] = sn.value
        return out

    def rhs(self, v):
        a = _Arg(v, self.Mtot)
        out, p = _out_like(a, self.N)
        self._check(_lib().mbs_rhs(self._h, a.nrhs, a.ptr, p))
        return _ret(out, a)

    def apply_operator(self, q):
        a = _Arg(q, self.N)
        out, p = _out_like(a, self.N)
        self._check(_lib().mbs_apply_operator(self._h, a.nrhs, a.ptr, p))
        return _ret(out, a)

    def apply_G(self, q, precision: int = PREC_FP64):
        a = _Arg(q, self.N)
        out, p = _out_like(a, self.N)
        self._check(_lib().mbs_apply_G(self._h, precision, a.nrhs, a.ptr, p))
        return _ret(out, a)

    def solve(self, b, x0=None, raise_on_noconv: bool = True):
        a = _Arg(b, self.N)
        if x0 is None:
            if a.torch:
                dev = a.keep.device
                pin = dev.type == "cpu" and a.keep.is_pinned()
                x = torch.zeros((a.nrhs, self.N), dtype=torch.complex128, device=dev,
                                pin_memory=pin).T
                xp = C.c_void_p(x.data_ptr())
            else:
                x = np.zeros((a.nrhs, self.N), dtype=np.complex128)
                xp = C.c_void_p(x.ctypes.data)
        else:
            xa = _Arg(x0, self.N)
            x = xa.keep.clone() if xa.torch else xa.keep.copy()
            xp = C.c_void_p(x.data_ptr() if xa.torch else x.ctypes.data)
        info = L.mbs_solve_info()
        st = _lib().mbs_solve(self._h, a.nrhs, a.ptr, xp, C.byref(info))
        if st != L.MBS_OK and (raise_on_noconv or st != 5):
            self._check(st)
        info_d = {f: getattr(info, f) for f, _ in info._fields_}
        info_d["status"] = st
        return _ret(x, a), info_d

    def evaluate_field(self, pts, qhat):
        a = _Arg(qhat, self.N)
        if _is_torch(pts):
            P = pts.to(torch.float64)
            P = P if P.T.is_contiguous() else P.T.contiguous().T
            P = P.T
            pp = C.c_void_p(P.data_ptr())
            M = pts.shape[0]
        else:
            P = _soa(pts)
            pp = C.c_void_p(P.ctypes.data)
            M = np.asarray(pts).shape[0]
        out, p = _out_like(a, M)
        self._check(_lib().mbs_evaluate_field(self._h, a.nrhs, M, pp, a.ptr, p))
        return _ret(out, a)

    def reconstruct(self, v, qhat):
        """mbs_reconstruct: MFS source strengths of every body (sum of n x nrhs)
        from the boundary data v and the solved q_hat (Sec. 4.6)."""
        a = _Arg(v, self.Mtot)
        qa = _Arg(qhat, self.N)
        out, p = _out_like(a, self.Nm)
        self._check(_lib().mbs_reconstruct(self._h, a.nrhs, a.ptr, qa.ptr, p))
        return _ret(out, a)

    def evaluate_field_near(self, pts, qhat, qmfs):
        """mbs_evaluate_field_near: scattered field at targets anywhere outside
        the MFS curves, inside proxy surfaces included (Sec. 4.6)."""
        a = _Arg(qhat, self.N)
        ma = _Arg(qmfs, self.Nm)
        if _is_torch(pts):
            P = pts.to(torch.float64)
            P = P if P.T.is_contiguous() else P.T.contiguous().T
            P = P.T
            pp = C.c_void_p(P.data_ptr())
            M = pts.shape[0]
        else:
            P = _soa(pts)
            pp = C.c_void_p(P.ctypes.data)
            M = np.asarray(pts).shape[0]
        out, p = _out_like(a, M)
        self._check(_lib().mbs_evaluate_field_near(self._h, a.nrhs, M, pp, a.ptr, ma.ptr, p))
        return _ret(out, a)

    def inject_scattering(self, shape: int, skel, S, W=None):
        skel = np.ascontiguousarray(np.asarray(skel, dtype=np.int32))
        Sf = np.asfortranarray(np.asarray(S, dtype=np.complex128))
        Wf = None if W is None else np.asfortranarray(np.asarray(W, dtype=np.complex128))
        self._check(_lib().mbs_inject_scattering(
            self._h, shape, len(skel), skel.ctypes.data_as(C.POINTER(C.c_int)),
            C.c_void_p(Sf.ctypes.data), None if Wf is None else C.c_void_p(Wf.ctypes.data)))
        self._N = None  # the library rebuilds the layout on its next use

    @property
    def N(self) -> int:
        if self._N is None:
            n = C.c_int64()
            self._check(_lib().mbs_get_layout(self._h, C.byref(n), None, None))
            self._N = int(n.value)
        return self._N

    @N.setter
    def N(self, v):
        self._N = v


def apply_G_noalloc(dim: int, kappa: float, body_offsets, body, xw, q, y, stream=None) -> None:
    """mbs_apply_G_noalloc: y = G_hat q (FP64) with no device allocation.

    Every argument is a CUDA tensor owned by the caller: body_offsets (T+1,)
    int64, body (N,) int32, xw (dim, N) float64 SoA, q and y (N, nrhs)
    complex128 with column-major layout (``torch.empty(nrhs, N).T``).  The
    work is queued on `stream` (a torch.cuda.Stream or None)."""
    N = int(body.shape[0])
    T = int(body_offsets.shape[0]) - 1
    nrhs = int(q.shape[1]) if q.dim() == 2 else 1
    for t in (q, y):
        if not (t.dim() == 1 or t.T.is_contiguous()):
            raise ValueError("q and y must be column-major (rows, nrhs)")
    s = None if stream is None else C.c_void_p(stream.cuda_stream)
    st = _lib().mbs_apply_G_noalloc(dim, kappa, N, T, C.c_void_p(body_offsets.data_ptr()),
                                    C.c_void_p(body.data_ptr()), C.c_void_p(xw.data_ptr()), nrhs,
                                    C.c_void_p(q.data_ptr()), C.c_void_p(y.data_ptr()), s)
    if st != L.MBS_OK:
        raise MbsError(st, "mbs_apply_G_noalloc")


def launch_count() -> int:
    """Kernel launches issued by libmbs.so so far in this process."""
    return int(_lib().mbs_launch_count())


def _ctx_profile(self, enable: bool = True):
    self._check(_lib().mbs_profile(self._h, 1 if enable else 0))


def _ctx_kernel_times(self) -> dict:
    out = (C.c_double * 7)()
    self._check(_lib().mbs_kernel_times(self._h, out))
    return {"g32_ms": out[0], "g32_launches": int(out[1]), "g64_ms": out[2],
            "g64_launches": int(out[3]), "g32_path": int(out[4]), "g32_nsplit": int(out[5]),
            "sbuild_threads": int(out[6])}


Context.profile = _ctx_profile
Context.kernel_times = _ctx_kernel_times


def measure_peaks() -> dict:
    out = (C.c_double * 6)()
    st = _lib().mbs_measure_peaks(out)
    if st != L.MBS_OK:
        raise MbsError(st, "mbs_measure_peaks")
    return {"fp32_tflops": out[0], "fp64_tflops": out[1], "mufu_tops": out[2], "sms": int(out[3]),
            "clock_khz": int(out[4]), "fp32x2_tflops": out[5]}


class Server:
    """mbs_serve_*: continuous batching of independent solves."""

    def __init__(self, max_active: int = 4, hbm_budget: int = 0):
        self._h = C.c_void_p()
        st = _lib().mbs_serve_create(max_active, hbm_budget, C.byref(self._h))
        if st != L.MBS_OK:
            raise MbsError(st, "mbs_serve_create")
        self._keep = {}

    def set_policy(self, policy: int):
        """0: admit in arrival order; 1: shortest estimated work first."""
        st = _lib().mbs_serve_set_policy(self._h, policy)
        if st != L.MBS_OK:
            raise MbsError(st, "mbs_serve_set_policy")

    def submit(self, wl, v, tol: float = 1e-10, fp64: bool = False, max_iter: int = 0) -> int:
        shapes, bodies, keep = shapes_bodies_from_workload(wl)
        vb = np.ascontiguousarray(np.asarray(v, dtype=np.complex128).T)
        req = L.mbs_request()
        req.dim, req.kappa = wl.dim, wl.kappa
        req.nshapes, req.shapes = len(wl.shapes), shapes
        req.nbodies, req.bodies = wl.T, bodies
        req.nrhs = vb.shape[0]
        req.v = vb.ctypes.data_as(C.POINTER(C.c_double))
        req.tol = tol
        req.fp64 = 1 if fp64 else 0
        req.max_iter = max_iter
        rid = C.c_int64()
        st = _lib().mbs_serve_submit(self._h, C.byref(req), C.byref(rid))
        if st != L.MBS_OK:
            raise MbsError(st, "mbs_serve_submit")
        self._keep[rid.value] = vb.shape[0]
        return rid.value

    def poll(self, rid: int, want_solution: bool = False):
        res = L.mbs_request_result()
        st = _lib().mbs_serve_poll(self._h, rid, C.byref(res), None)
        if st != L.MBS_OK:
            raise MbsError(st, "mbs_serve_poll")
        d = {f: getattr(res, f) for f, _ in res._fields_}
        if want_solution and res.done == 1:
            nrhs = self._keep[rid]
            q = np.zeros((nrhs, res.N), dtype=np.complex128)
            _lib().mbs_serve_poll(self._h, rid, C.byref(res), C.c_void_p(q.ctypes.data))
            d["qhat"] = q.T
        return d

    def drain(self):
        _lib().mbs_serve_drain(self._h)

    def close(self):
        if self._h:
            _lib().mbs_serve_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
