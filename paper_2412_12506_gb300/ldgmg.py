"""Python binding of libldgmg (include/ldgmg.h, include/ldgmg_host.h).

Argument marshalling only: every computation runs in the C-ABI library
(CUDA kernels for sm_103a, host C++ for setup).  PyTorch supplies device
memory and streams.  Importing this module raises ImportError when the
library has not been built -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libldgmg.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"libldgmg.so not found at {LIB_PATH}; build it with "
                      "`python -m paper_2412_12506_gb300.build` (or __graft_entry__.build())")
_lib = ctypes.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, ETIMEOUT, EUNSUPPORTED = range(7)
JACOBI, SAI, GS = 0, 1, 2
FORM_B1, FORM_BT = 0, 1
FP64, FP32, BF16, FP16 = 0, 1, 2, 3
MAT_A, MAT_B, MAT_BT, MAT_D = 0, 1, 2, 3
_PREC = {"fp64": FP64, "fp32": FP32, "bf16": BF16, "fp16": FP16}
_FORM = {"B1": FORM_B1, "BT": FORM_BT}
_SMOOTHER = {"jacobi": JACOBI, "sai": SAI, "gs": GS}


class LdgmgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ldgmg status {status}: {msg}")
        self.status = status


class Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("periodic", ctypes.c_int)]


class SetupOpts(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("sai_level", ctypes.c_int), ("balance", ctypes.c_int),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("omega", ctypes.c_double),
                ("pre_form", ctypes.c_int), ("post_form", ctypes.c_int),
                ("vcycle_precision", ctypes.c_int), ("max_iter", ctypes.c_int), ("max_rhs", ctypes.c_int),
                ("outer_apply", ctypes.c_int), ("krylov", ctypes.c_int), ("restart", ctypes.c_int),
                ("zeta", ctypes.c_double)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("workers", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("simulate", ctypes.c_int), ("simulate_solve_s", ctypes.c_double), ("setup", SetupOpts),
                ("group_dofs", ctypes.c_size_t), ("group_max", ctypes.c_int), ("simulate_notconv_n", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("p", ctypes.c_int), ("stokes", ctypes.c_int),
                ("mu_host", ctypes.c_void_p), ("tau0", ctypes.c_double), ("taup", ctypes.c_double),
                ("rhs_host", ctypes.c_void_p), ("x_host", ctypes.c_void_p), ("tol", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("relres", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_end", ctypes.c_double),
                ("batch", ctypes.c_int), ("worker", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("builds", ctypes.c_uint64),
                ("evictions", ctypes.c_uint64), ("build_failures", ctypes.c_uint64),
                ("solve_calls", ctypes.c_uint64), ("max_batch_seen", ctypes.c_int),
                ("classes_resident", ctypes.c_int), ("bytes_resident", ctypes.c_size_t),
                ("bytes_peak", ctypes.c_size_t), ("hbm_budget", ctypes.c_size_t),
                ("precision_fallbacks", ctypes.c_uint64), ("group_calls", ctypes.c_uint64),
                ("group_requests", ctypes.c_uint64)]


_vp, _i, _i64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_P = ctypes.POINTER
_SIGS = {
    "ldgmg_default_opts": (None, [_P(SetupOpts)]),
    "ldgmg_assemble": (_i, [_P(Mesh), _i, _vp, _d, _P(_vp)]),
    "ldgmg_assemble_stokes": (_i, [_P(Mesh), _i, _vp, _i, _d, _d, _P(_vp)]),
    "ldgmg_op_info": (_i, [_vp, _P(_i64), _P(_i), _P(_i64)]),
    "ldgmg_op_fields": (_i, [_vp, _P(_i), _P(_i)]),
    "ldgmg_op_device_bytes": (_i, [_vp, _P(ctypes.c_size_t)]),
    "ldgmg_hier_device_bytes": (_i, [_vp, _P(ctypes.c_size_t)]),
    "ldgmg_hier_tuning": (_i, [_vp, _P(_i), _P(_d)]),
    "ldgmg_hier_tc_schedule": (_i, [_vp, _P(_i), _P(_i), _P(_d)]),
    "ldgmg_solve_history": (_i, [_vp, _i, _vp, _i, _P(_i)]),
    "ldgmg_apply": (_i, [_vp, _vp, _vp, _i, _vp]),
    "ldgmg_project_kernel": (_i, [_vp, _vp, _i, _vp]),
    "ldgmg_setup": (_i, [_vp, _P(SetupOpts), _vp, _P(_vp)]),
    "ldgmg_hier_info": (_i, [_vp, _i, _P(_i), _P(_i), _P(_i64), _P(_i), _P(_i64), _P(_i64)]),
    "ldgmg_vcycle": (_i, [_vp, _vp, _vp, _i, _vp]),
    "ldgmg_solve": (_i, [_vp, _vp, _d, _vp, _i, _P(_i), _P(_d), _vp]),
    "ldgmg_krylov_apply": (_i, [_vp, _i, _vp, _vp, _vp]),
    "ldgmg_level_apply": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
    "ldgmg_level_smooth": (_i, [_vp, _i, _i, _vp, _vp, _vp, _i, _vp]),
    "ldgmg_level_apply_batched": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp]),
    "ldgmg_level_restrict": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "ldgmg_level_prolong": (_i, [_vp, _i, _vp, _vp, _vp]),
    "ldgmg_bottom_solve": (_i, [_vp, _vp, _vp, _vp]),
    "ldgmg_export_level": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
    "ldgmg_op_free": (None, [_vp]),
    "ldgmg_hier_free": (None, [_vp]),
    "ldgmg_last_error": (ctypes.c_char_p, []),
    "ldgmg_kernel_launches": (ctypes.c_ulonglong, []),
    "ldgmg_selftest_bounded_wait": (_i, [_vp]),
    "ldgmg_project_kernel_noalloc": (_i, [_i64, _i, _vp, _vp]),
    "ldgmg_host_build": (_i, [_P(Mesh), _i, _vp, _d, _P(SetupOpts), _P(_vp)]),
    "ldgmg_host_build_stokes": (_i, [_P(Mesh), _i, _vp, _i, _d, _d, _P(SetupOpts), _P(_vp)]),
    "ldgmg_host_level_info": (_i, [_vp, _i, _P(_i), _P(_i), _P(_i64), _P(_i), _P(_i64), _P(_i64),
                                   _P(_i64)]),
    "ldgmg_host_export": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
    "ldgmg_host_colours": (_i, [_vp, _i, _vp, _P(_i)]),
    "ldgmg_host_tc_plan": (_i, [_i, _vp, _vp, _i, _i, _i, _i, _vp, _P(_i64), _vp, _vp, _vp]),
    "ldgmg_host_free": (None, [_vp]),
    "ldgmg_group_create": (_i, [_P(_vp)]),
    "ldgmg_group_free": (None, [_vp]),
    "ldgmg_solve_group": (_i, [_vp, _i, _P(_vp), _P(_vp), _P(_vp), _P(_d), _P(_i), _P(_d), _P(_i), _vp]),
    "ldgmg_group_cluster": (_i, [_vp, _P(_i)]),
    "ldgmg_server_create": (_i, [_P(ServerOpts), _P(_vp)]),
    "ldgmg_server_submit": (_i, [_vp, _P(Request), _P(ctypes.c_uint64)]),
    "ldgmg_server_wait": (_i, [_vp, ctypes.c_uint64, _P(Result)]),
    "ldgmg_server_get_stats": (_i, [_vp, _P(ServerStats)]),
    "ldgmg_server_clock": (_d, [_vp]),
    "ldgmg_server_destroy": (None, [_vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

EXPORTED = tuple(_SIGS)


def _check(status: int):
    if status != OK:
        raise LdgmgError(status, _lib.ldgmg_last_error().decode())


def kernel_launches() -> int:
    """Kernels enqueued by the library so far (ldgmg_kernel_launches)."""
    return int(_lib.ldgmg_kernel_launches())


def selftest_bounded_wait(stream=None) -> int:
    """ldgmg_selftest_bounded_wait: status of a device wait that must give up (ETIMEOUT)."""
    return int(_lib.ldgmg_selftest_bounded_wait(_stream(stream)))


NOALLOC_MAX_ELEMENTS = 16777216


def project_kernel_noalloc(v, N, b, offset=0, stream=None):
    """ldgmg_project_kernel_noalloc: subtract the mean of v[offset + e*b],
    e = 0..N-1, from those entries, in place, without any allocation in the
    library (include/ldgmg.h).  offset = 0 projects a scalar vector; a Stokes
    vector takes one call per field with offset = f * field_b.  v must be a
    contiguous CUDA float64 tensor long enough for the N strided entries: the
    C call cannot check its length, so this wrapper does."""
    import torch
    if not isinstance(v, torch.Tensor) or not v.is_cuda or v.dtype != torch.float64 or not v.is_contiguous():
        raise LdgmgError(EINVAL, "v must be a contiguous CUDA float64 tensor")
    N, b, offset = int(N), int(b), int(offset)
    if N > NOALLOC_MAX_ELEMENTS:
        # the library refuses the size before it touches v: let it say so
        _check(_lib.ldgmg_project_kernel_noalloc(N, b, _ptr(v), _stream(stream)))
    if N < 1 or b < 1 or offset < 0 or offset + (N - 1) * b + 1 > v.numel():
        raise LdgmgError(EINVAL, f"v has {v.numel()} entries; N = {N}, b = {b}, offset = {offset} "
                                 f"need {offset + (N - 1) * b + 1}")
    ptr = ctypes.c_void_p(v.data_ptr() + 8 * offset)
    _check(_lib.ldgmg_project_kernel_noalloc(N, b, ptr, _stream(stream)))
    return v


_OUTER = {"auto": 0, "fp64": 1, "df": 2}
_KRYLOV = {"auto": 0, "cg": 1, "gmres": 2, "fgmres": 3}
TAUP = 0.05   # default Stokes pressure-penalty scale (tau_p = taup h / min mu)


def make_opts(smoother="sai", sai_level=1, balance=True, nu1=3, nu2=3, omega=0.8, pre="B1", post="BT",
              precision="fp64", max_iter=200, max_rhs=1, outer="auto", krylov="auto", restart=50,
              zeta=0.0) -> SetupOpts:
    o = SetupOpts()
    _lib.ldgmg_default_opts(ctypes.byref(o))
    o.smoother = _SMOOTHER[smoother]
    o.sai_level = sai_level
    o.balance = int(bool(balance))
    o.nu1, o.nu2, o.omega = nu1, nu2, omega
    o.pre_form, o.post_form = _FORM[pre], _FORM[post]
    o.vcycle_precision = _PREC[precision]
    o.max_iter = max_iter
    o.max_rhs = max_rhs
    o.outer_apply = _OUTER[outer]
    o.krylov = _KRYLOV[krylov]
    o.restart = restart
    o.zeta = zeta
    return o


def _mu_ptr(mu):
    if mu is None:
        return None, None
    arr = np.ascontiguousarray(mu, dtype=np.float64)
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# host-side setup inspection (no GPU)
# ---------------------------------------------------------------------------

class HostHierarchy:
    """Host setup of ldgmg_setup without the device upload (include/ldgmg_host.h)."""

    def __init__(self, dim, n, p, mu=None, tau0=1.0, stokes=None, taup=TAUP, **opts):
        """stokes=None: scalar operator; stokes=0 / 1: Stokes standard / stress form."""
        keep, mp = _mu_ptr(mu)
        h = ctypes.c_void_p()
        o = make_opts(**opts)
        if stokes is None:
            _check(_lib.ldgmg_host_build(ctypes.byref(Mesh(dim, n, 1)), p, mp, tau0, ctypes.byref(o),
                                         ctypes.byref(h)))
        else:
            _check(_lib.ldgmg_host_build_stokes(ctypes.byref(Mesh(dim, n, 1)), p, mp, int(stokes), tau0, taup,
                                                ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.nlevels = self.info(0)["nlevels"]

    def info(self, level):
        nl, n, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        N, nA, nS, dA = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.ldgmg_host_level_info(self._h, level, ctypes.byref(nl), ctypes.byref(n), ctypes.byref(N),
                                          ctypes.byref(b), ctypes.byref(nA), ctypes.byref(nS),
                                          ctypes.byref(dA)))
        return dict(nlevels=nl.value, n=n.value, N=N.value, b=b.value, nnzb_A=nA.value, nnzb_S=nS.value,
                    distinct_A=dA.value)

    def export(self, level, which=MAT_A):
        inf = self.info(level)
        nnz = inf["nnzb_A"] if which == MAT_A else inf["nnzb_S"]
        N, b = inf["N"], inf["b"]
        rp = np.zeros(N + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        vals = np.zeros((nnz, b, b), np.float64)
        _check(_lib.ldgmg_host_export(self._h, level, which, rp.ctypes.data_as(_vp), col.ctypes.data_as(_vp),
                                      vals.ctypes.data_as(_vp)))
        return rp, col, vals

    def colours(self, level):
        """Colour of every element of a Gauss-Seidel level (ldgmg_host_colours)."""
        N = self.info(level)["N"]
        out = np.zeros(N, np.int32)
        nc = ctypes.c_int()
        _check(_lib.ldgmg_host_colours(self._h, level, out.ctypes.data_as(_vp), ctypes.byref(nc)))
        return out, nc.value

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.ldgmg_host_free(self._h)
            self._h = None


def host_tc_plan(n, row_ptr, col, rcap=64, precision="fp32", ctas=152, strip=8):
    """ldgmg_host_tc_plan: the cached tensor-core apply's schedule for a 2D
    block pattern.  Returns a dict (ctas, slots, strip, kmax, nloads, rec as an
    (n*n, 16) int32 array, seg, ld_elem)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    info = np.zeros(4, np.int32)
    nl = ctypes.c_int64()
    args = (n, rp.ctypes.data_as(_vp), cl.ctypes.data_as(_vp), rcap, _PREC[precision], ctas, strip,
            info.ctypes.data_as(_vp), ctypes.byref(nl))
    _check(_lib.ldgmg_host_tc_plan(*args, None, None, None))
    rec = np.zeros((n * n, 16), np.int32)
    seg = np.zeros(int(info[0]) + 1, np.int32)
    ld = np.zeros(max(nl.value, 1), np.int32)
    _check(_lib.ldgmg_host_tc_plan(*args, rec.ctypes.data_as(_vp), seg.ctypes.data_as(_vp),
                                   ld.ctypes.data_as(_vp)))
    return dict(ctas=int(info[0]), slots=int(info[1]), strip=int(info[2]), kmax=int(info[3]), nloads=nl.value,
                rec=rec, seg=seg, ld_elem=ld[:nl.value])


# ---------------------------------------------------------------------------
# device API
# ---------------------------------------------------------------------------

class Operator:
    """LDG operator A on the device: the scalar operator (ldgmg_assemble), or
    with stokes=0 / 1 the Stokes saddle-point operator in standard / stress
    form (ldgmg_assemble_stokes)."""

    def __init__(self, dim, n, p, mu=None, tau0=1.0, stokes=None, taup=TAUP):
        keep, mp = _mu_ptr(mu)
        h = ctypes.c_void_p()
        if stokes is None:
            _check(_lib.ldgmg_assemble(ctypes.byref(Mesh(dim, n, 1)), p, mp, tau0, ctypes.byref(h)))
        else:
            _check(_lib.ldgmg_assemble_stokes(ctypes.byref(Mesh(dim, n, 1)), p, mp, int(stokes), tau0, taup,
                                              ctypes.byref(h)))
        self._h = h
        N, b, nnz = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64()
        _check(_lib.ldgmg_op_info(h, ctypes.byref(N), ctypes.byref(b), ctypes.byref(nnz)))
        nf, bs = ctypes.c_int(), ctypes.c_int()
        _check(_lib.ldgmg_op_fields(h, ctypes.byref(nf), ctypes.byref(bs)))
        self.dim, self.n, self.p = dim, n, p
        self.N, self.b, self.nnzb = N.value, b.value, nnz.value
        self.nfields, self.field_b = nf.value, bs.value
        self.stokes = stokes
        self.size = self.N * self.b

    @property
    def device_bytes(self) -> int:
        v = ctypes.c_size_t()
        _check(_lib.ldgmg_op_device_bytes(self._h, ctypes.byref(v)))
        return v.value

    def _nrhs(self, t):
        n = t.numel() // self.size
        if n * self.size != t.numel():
            raise ValueError("vector length is not a multiple of N*b")
        return n

    def apply(self, x, y=None, stream=None):
        """y = A x; x holds one or several stacked vectors (shape (size,) or (nrhs, size))."""
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(_lib.ldgmg_apply(self._h, _ptr(x), _ptr(y), self._nrhs(x), _stream(stream)))
        return y

    def project_kernel(self, v, stream=None):
        _check(_lib.ldgmg_project_kernel(self._h, _ptr(v), self._nrhs(v), _stream(stream)))
        return v

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.ldgmg_op_free(self._h)
            self._h = None


class Hierarchy:
    """Multigrid hierarchy + smoothers + bottom solver (ldgmg_setup)."""

    def __init__(self, op: Operator, stream=None, **opts):
        self.op = op
        self.opts = opts
        o = make_opts(**opts)
        h = ctypes.c_void_p()
        _check(_lib.ldgmg_setup(op._h, ctypes.byref(o), _stream(stream), ctypes.byref(h)))
        self._h = h
        self.precision = opts.get("precision", "fp64")
        self.nlevels = self.info(0)["nlevels"]

    @property
    def device_bytes(self) -> int:
        v = ctypes.c_size_t()
        _check(_lib.ldgmg_hier_device_bytes(self._h, ctypes.byref(v)))
        return v.value

    def history(self, rhs=0):
        """Relative residual history of the last solve (ldgmg_solve_history)."""
        n = ctypes.c_int()
        _check(_lib.ldgmg_solve_history(self._h, rhs, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value)
        _check(_lib.ldgmg_solve_history(self._h, rhs, out.ctypes.data_as(_vp), n.value, ctypes.byref(n)))
        return out

    @property
    def tuning(self):
        """Autotuned tensor-core launch shape: (CTAs per SM, ms of the level-0 apply)."""
        c, t = ctypes.c_int(), ctypes.c_double()
        _check(_lib.ldgmg_hier_tuning(self._h, ctypes.byref(c), ctypes.byref(t)))
        return c.value, t.value

    @property
    def tc_schedule(self):
        """Cached tensor-core apply: (strip width or 0, x slots per CTA, x_j loads per row)."""
        L, S, lpr = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(_lib.ldgmg_hier_tc_schedule(self._h, ctypes.byref(L), ctypes.byref(S), ctypes.byref(lpr)))
        return L.value, S.value, lpr.value

    @property
    def vdtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    def info(self, level):
        nl, n, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        N, nA, nS = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.ldgmg_hier_info(self._h, level, ctypes.byref(nl), ctypes.byref(n), ctypes.byref(N),
                                    ctypes.byref(b), ctypes.byref(nA), ctypes.byref(nS)))
        return dict(nlevels=nl.value, n=n.value, N=N.value, b=b.value, nnzb_A=nA.value, nnzb_S=nS.value)

    def vcycle(self, b, x=None, stream=None):
        import torch
        if x is None:
            x = torch.empty_like(b)
        _check(_lib.ldgmg_vcycle(self._h, _ptr(b), _ptr(x), self.op._nrhs(b), _stream(stream)))
        return x

    def solve(self, rhs, tol=1e-10, x=None, stream=None, check=True):
        """Returns (x, iterations, true relative residual, status).  rhs/x may be
        CUDA or CPU tensors (host buffers are staged by the library).  With
        nrhs stacked right-hand sides (shape (nrhs, size)), iterations and
        residuals are lists."""
        import torch
        if x is None:
            x = torch.empty_like(rhs)
        nr = self.op._nrhs(rhs)
        it = (ctypes.c_int * nr)()
        rr = (ctypes.c_double * nr)()
        st = _lib.ldgmg_solve(self._h, _ptr(rhs), tol, _ptr(x), nr, it, rr, _stream(stream))
        if check and st not in (OK,):
            _check(st)
        if nr == 1:
            return x, it[0], rr[0], st
        return x, list(it), list(rr), st

    def krylov_apply(self, x, nrhs, y=None, stream=None):
        """y = A x with the outer CG's operator apply (ldgmg_krylov_apply); FP64
        vectors [element][rhs][mode], nrhs right-hand sides."""
        import torch
        if y is None:
            y = torch.empty_like(x)
        if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()) or \
                x.numel() != self.op.size * nrhs or y.shape != x.shape or y.dtype != x.dtype:
            raise ValueError("x, y must be contiguous CUDA float64 tensors of N*b*nrhs entries")
        _check(_lib.ldgmg_krylov_apply(self._h, nrhs, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def level_apply_batched(self, level, which, x, nrhs, y=None, stream=None):
        """y = M x for nrhs right-hand sides, float vectors [element][rhs][mode]."""
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(_lib.ldgmg_level_apply_batched(self._h, level, which, nrhs, _ptr(x), _ptr(y), _stream(stream)))
        return y

    # per-level entry points (vectors in the hierarchy's working dtype)
    def level_apply(self, level, which, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(_lib.ldgmg_level_apply(self._h, level, which, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def level_smooth(self, level, form, rhs, x_in=None, x_out=None, stream=None):
        import torch
        if x_out is None:
            x_out = torch.empty_like(rhs)
        xin = _ptr(x_in) if x_in is not None else None
        _check(_lib.ldgmg_level_smooth(self._h, level, _FORM[form], _ptr(rhs), xin, _ptr(x_out),
                                       int(x_in is None), _stream(stream)))
        return x_out

    def level_restrict(self, level, rhs, x, rc=None, stream=None):
        import torch
        if rc is None:
            inf = self.info(level + 1)
            rc = torch.empty(inf["N"] * inf["b"], dtype=rhs.dtype, device=rhs.device)
        _check(_lib.ldgmg_level_restrict(self._h, level, _ptr(rhs), _ptr(x), _ptr(rc), _stream(stream)))
        return rc

    def level_prolong(self, level, xc, x, stream=None):
        _check(_lib.ldgmg_level_prolong(self._h, level, _ptr(xc), _ptr(x), _stream(stream)))
        return x

    def bottom_solve(self, rhs, x=None, stream=None):
        import torch
        if x is None:
            x = torch.empty_like(rhs)
        _check(_lib.ldgmg_bottom_solve(self._h, _ptr(rhs), _ptr(x), _stream(stream)))
        return x

    def export_level(self, level, which=MAT_A):
        inf = self.info(level)
        nnz = inf["nnzb_A"] if which == MAT_A else inf["nnzb_S"]
        N, b = inf["N"], inf["b"]
        rp = np.zeros(N + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        vals = np.zeros((nnz, b, b), np.float64)
        _check(_lib.ldgmg_export_level(self._h, level, which, rp.ctypes.data_as(_vp), col.ctypes.data_as(_vp),
                                       vals.ctypes.data_as(_vp)))
        return rp, col, vals

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.ldgmg_hier_free(self._h)
            self._h = None


class Group:
    """Workspace of grouped solves (ldgmg_solve_group): many small problems,
    each on its own hierarchy, solved in one launch per cluster size."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(_lib.ldgmg_group_create(ctypes.byref(h)))
        self._h = h

    @staticmethod
    def cluster(hier) -> int:
        """CTAs per problem a grouped solve gives this hierarchy (0: not eligible)."""
        c = ctypes.c_int()
        _check(_lib.ldgmg_group_cluster(hier._h, ctypes.byref(c)))
        return c.value

    def solve(self, problems, stream=None, check=True):
        """problems: list of (hierarchy, rhs, x, tol); rhs / x FP64 tensors of
        N*b entries (CUDA or CPU).  Returns (iterations, relres, statuses) lists."""
        n = len(problems)
        hs = (_vp * n)(*[p[0]._h.value for p in problems])
        for hier, rhs, x, _ in problems:
            if rhs.numel() != hier.op.size or x.numel() != hier.op.size:
                raise ValueError("rhs and x must hold N*b entries of their hierarchy")
            if not (rhs.is_contiguous() and x.is_contiguous()) or rhs.element_size() != 8 or x.element_size() != 8:
                raise ValueError("rhs and x must be contiguous float64 tensors")
        bs = (_vp * n)(*[p[1].data_ptr() for p in problems])
        xs = (_vp * n)(*[p[2].data_ptr() for p in problems])
        tols = (_d * n)(*[float(p[3]) for p in problems])
        it = (_i * n)()
        rr = (_d * n)()
        stv = (_i * n)()
        st = _lib.ldgmg_solve_group(self._h, n, hs, bs, xs, tols, it, rr, stv, _stream(stream))
        if check and st != OK:
            _check(st)
        return list(it), list(rr), list(stv)

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.ldgmg_group_free(self._h)
            self._h = None


# ---------------------------------------------------------------------------
# serving engine (include/ldgmg_serve.h)
# ---------------------------------------------------------------------------

class Server:
    """Continuous-batching solve server (ldgmg_server_*).  submit() copies the
    inputs and returns a ticket; wait(ticket) returns (x, result dict)."""

    def __init__(self, workers=4, max_batch=32, hbm_budget=0, simulate=False, simulate_solve_s=0.0,
                 group_dofs=0, group_max=0, simulate_notconv_n=0, **opts):
        o = ServerOpts()
        o.hbm_budget, o.workers, o.max_batch = int(hbm_budget), workers, max_batch
        o.simulate, o.simulate_solve_s = int(bool(simulate)), simulate_solve_s
        o.group_dofs, o.group_max = int(group_dofs), int(group_max)
        o.simulate_notconv_n = int(simulate_notconv_n)
        o.setup = make_opts(**opts)
        h = ctypes.c_void_p()
        _check(_lib.ldgmg_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._live = {}

    def submit(self, dim, n, p, rhs, mu=None, stokes=None, tau0=1.0, taup=TAUP, tol=1e-10):
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        x = np.zeros_like(rhs)
        keep, mp = _mu_ptr(mu)
        q = Request(dim, n, p, -1 if stokes is None else int(stokes), mp, tau0, taup,
                    rhs.ctypes.data_as(_vp), x.ctypes.data_as(_vp), tol)
        t = ctypes.c_uint64()
        _check(_lib.ldgmg_server_submit(self._h, ctypes.byref(q), ctypes.byref(t)))
        self._live[t.value] = x
        return t.value

    def wait(self, ticket):
        r = Result()
        _check(_lib.ldgmg_server_wait(self._h, ticket, ctypes.byref(r)))
        x = self._live.pop(ticket)
        return x, {k: getattr(r, k) for k, _ in Result._fields_}

    def stats(self):
        s = ServerStats()
        _check(_lib.ldgmg_server_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def clock(self):
        return _lib.ldgmg_server_clock(self._h)

    def close(self):
        if getattr(self, "_h", None):
            _lib.ldgmg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()
