"""ctypes binding of include/tt_stochns.h (argument marshalling only).

Every computation runs in libttns.so on the GPU.  Importing this module does
not touch the GPU; `Context()` does, and raises if the library is missing or
no CUDA device is present.  Cores cross the boundary in the paper's shapes
(z1: n_t x r1, z2: r1 x n_xi x r2, z3: r2 x n_x) as numpy float64 arrays; the
binding converts to and from the library's layouts.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libttns.so")

TT_OK, TT_EINVAL, TT_ENOMEM, TT_ECUDA, TT_ENOCONV, TT_ERANK, TT_ENAN, TT_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
OP_FULL, OP_MEAN = 0, 1
PREC_LSC, PREC_LEARNED, PREC_PCD = 0, 1, 2
FP64, MIXED = 0, 1
ROUND_EXACT, ROUND_RANDOMIZED = 0, 1
F64 = 0
MAX_PICARD = 64

_P = C.c_void_p
_D = C.c_double
_I = C.c_int
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)


class ProblemDesc(C.Structure):
    _fields_ = [("n_nodes", _I), ("n_elem", _I), ("n_pnodes", _I), ("h", _D),
                ("xy", _DP), ("elem_q2", C.POINTER(C.c_longlong)), ("elem_q1", C.POINTER(C.c_longlong)),
                ("dirichlet", C.POINTER(C.c_ubyte)), ("inflow", _DP), ("m", _I), ("n_xi", _I),
                ("multi_index", C.POINTER(C.c_longlong)), ("nu", _DP), ("n_t", _I), ("tau", _D),
                ("tprofile", _DP)]


class SolverOpts(C.Structure):
    _fields_ = [("tol_picard", _D), ("tol_gmres", _D), ("eps_gmres", _D), ("eps_soln", _D),
                ("eps_conv", _D), ("tol_inner", _D), ("maxit_picard", _I), ("maxit_gmres", _I),
                ("maxit_inner", _I), ("precision", _I), ("learned", _P), ("init_u", _P), ("init_p", _P),
                ("rounding", _I), ("schur", _I)]


class PrecOpts(C.Structure):
    _fields_ = [("eps", _D), ("tol_inner", _D), ("maxit_inner", _I), ("net", _P)]


class TrainOpts(C.Structure):
    _fields_ = [("epochs", _I), ("batch", _I), ("lr", C.c_float), ("smooth_max", _I), ("omega", C.c_float)]


class GmresStats(C.Structure):
    _fields_ = [("its", _I), ("res0", _D), ("res", _D), ("inner_its", _I), ("fallbacks", _I)]


class PicardStats(C.Structure):
    _fields_ = [("picard_its", _I), ("stokes_its", _I), ("fnorm", _D),
                ("res", _D * (MAX_PICARD + 1)), ("gmres_its", _I * (MAX_PICARD + 1)),
                ("inner_its", _I * (MAX_PICARD + 1)), ("ranks", (_I * 4) * (MAX_PICARD + 1)),
                ("conv_ranks", (_I * 2) * (MAX_PICARD + 1)), ("fallbacks", _I * (MAX_PICARD + 1))]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FP = C.POINTER(C.c_float)


_SIGS = {
    "tt_ctx_create": (_I, [_P, ALLOC_FN, FREE_FN, _P, C.POINTER(_P)]),
    "tt_ctx_destroy": (_I, [_P]),
    "tt_last_error": (C.c_char_p, [_P]),
    "tt_ctx_launches": (C.c_longlong, [_P]),
    "tt_ctx_set_wait_limit": (_I, [_P, C.c_longlong]),
    "tt_ctx_profile": (_I, [_P, _I]),
    "tt_ctx_prof_read": (_I, [_P, _I, C.POINTER(C.c_longlong), _DP, _DP, _DP]),
    "tt_create": (_I, [_P, _I, _I, _I, _I, _I, _I, _I, _I, _P, _P, _P, _I, C.POINTER(_P)]),
    "tt_destroy": (_I, [_P]),
    "tt_shape": (_I, [_P, _IP, _IP, _IP, _IP, _IP]),
    "tt_capacity": (_I, [_P, _IP, _IP]),
    "tt_get_cores": (_I, [_P, _P, _P, _P, _P, _I]),
    "tt_round": (_I, [_P, _P, _D, C.POINTER(_P), _DP, _DP]),
    "tt_round_to": (_I, [_P, _P, _D, _P, _DP, _DP]),
    "tt_round_randomized": (_I, [_P, _P, _D, C.c_ulonglong, C.POINTER(_P), _DP, _DP, _IP]),
    "tt_dot": (_I, [_P, _P, _P, _DP]),
    "tt_norm": (_I, [_P, _P, _DP]),
    "tt_dot_noalloc": (_I, [_P, _P, _P, _DP]),
    "tt_axpby": (_I, [_P, _D, _P, _D, _P, _D, C.POINTER(_P)]),
    "tt_problem_create": (_I, [_P, C.POINTER(ProblemDesc), C.POINTER(_P)]),
    "tt_problem_destroy": (_I, [_P]),
    "tt_problem_sizes": (_I, [_P, _IP, _IP, _IP, _IP, _IP, _IP]),
    "tt_problem_matrix": (_I, [_P, _P, _I, _I, _IP, _IP, _IP, _IP, _IP, _DP]),
    "tt_rhs": (_I, [_P, _P, C.POINTER(_P), C.POINTER(_P)]),
    "tt_full_velocity": (_I, [_P, _P, _P, C.POINTER(_P)]),
    "tt_op_create": (_I, [_P, _P, _P, _I, C.POINTER(_P)]),
    "tt_op_destroy": (_I, [_P]),
    "tt_matvec": (_I, [_P, _P, _P, _P, _D, C.POINTER(_P), C.POINTER(_P)]),
    "tt_prec_create": (_I, [_P, _P, _I, C.POINTER(PrecOpts), C.POINTER(_P)]),
    "tt_prec_destroy": (_I, [_P]),
    "tt_prec_apply": (_I, [_P, _P, _P, _P, C.POINTER(_P), C.POINTER(_P), _IP, _IP]),
    "tt_net_create": (_I, [_P, _P, _I, _I, _FP, C.POINTER(_P)]),
    "tt_net_destroy": (_I, [_P]),
    "tt_net_info": (_I, [_P, _IP, _IP, _IP]),
    "tt_net_set_tensor_cores": (_I, [_P, _I]),
    "tt_net_get_params": (_I, [_P, _P, _FP]),
    "tt_net_apply": (_I, [_P, _P, _P, _DP, _I, _I, _DP]),
    "tt_net_loss_grad": (_I, [_P, _P, _P, _DP, _DP, _I, _I, _DP, _FP]),
    "tt_net_train": (_I, [_P, _P, _P, _DP, _I, _I, C.POINTER(TrainOpts), _DP]),
    "tt_residual": (_I, [_P, _P, _P, _P, _D, C.POINTER(_P), C.POINTER(_P), _DP]),
    "tt_gmres": (_I, [_P, _P, _P, C.POINTER(SolverOpts), _P, _P, _D, C.POINTER(_P), C.POINTER(_P),
                      C.POINTER(GmresStats)]),
    "picard_solve": (_I, [_P, _P, C.POINTER(SolverOpts), C.POINTER(_P), C.POINTER(_P),
                          C.POINTER(PicardStats)]),
    "picard_solve_batched": (_I, [_I, C.POINTER(_P), C.POINTER(SolverOpts), C.POINTER(_P), C.POINTER(_P),
                                  C.POINTER(PicardStats), _IP, _DP]),
}


class LibraryError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libttns error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libttns.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"GPU library not built: {path} (run paper_1906_06785_gb300.build)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


class Context:
    """A library context bound to a CUDA stream (torch's current stream by default)."""

    def __init__(self, stream=None, alloc=None, free=None):
        """alloc(bytes, stream) -> device pointer (int, 0 on failure) and
        free(ptr, bytes, stream): optional caller allocator for all device memory
        of the context (both or neither)."""
        self.lib = load()
        if stream is None:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device: the GPU library has no CPU fallback")
            stream = torch.cuda.current_stream().cuda_stream
        if (alloc is None) != (free is None):
            raise ValueError("give both alloc and free, or neither")
        if alloc is not None:
            self._cb = (ALLOC_FN(lambda n, st, u: alloc(n, st) or None),
                        FREE_FN(lambda p, n, st, u: free(p, n, st)))
        else:
            self._cb = (ALLOC_FN(), FREE_FN())
        h = _P()
        self._check(self.lib.tt_ctx_create(_P(stream), self._cb[0], self._cb[1], None, C.byref(h)), None)
        self.h = h

    def _check(self, code, h=True):
        if code != TT_OK:
            msg = self.lib.tt_last_error(self.h if h else None)
            raise LibraryError(code, msg.decode() if msg else "")

    def check(self, code, allow=()):
        if code != TT_OK and code not in allow:
            self._check(code)
        return code

    @property
    def launches(self):
        return int(self.lib.tt_ctx_launches(self.h))

    PROF_SLOTS = ("qr", "jacobi", "gemm", "spmm", "band_solve", "band_factor", "core", "assembly", "conv")

    def set_wait_limit(self, polls):
        """Polls a block makes at a grid barrier before giving up (TT_ETIMEOUT)."""
        self.check(self.lib.tt_ctx_set_wait_limit(self.h, int(polls)))

    def profile(self, enable=True):
        """Reset the per-kernel-class counters and turn event timing on or off."""
        self.check(self.lib.tt_ctx_profile(self.h, 1 if enable else 0))

    def prof_read(self):
        """{class: (launches, ms, flops, bytes)} since the last profile() call."""
        out = {}
        for i, name in enumerate(self.PROF_SLOTS):
            n = C.c_longlong(); ms = _D(); fl = _D(); by = _D()
            self.check(self.lib.tt_ctx_prof_read(self.h, i, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)))
            out[name] = (n.value, ms.value, fl.value, by.value)
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.tt_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- trains ------------------------------------------------------------
    def tt(self, z1, z2, z3, cap=(0, 0)):
        """New device train from cores in the paper's shapes (numpy); cap: rank
        capacities of its allocation (0: the ranks)."""
        z1 = np.asarray(z1, np.float64); z2 = np.asarray(z2, np.float64); z3 = np.asarray(z3, np.float64)
        n_t, r1 = z1.shape
        r1b, n_xi, r2 = z2.shape
        r2b, n_x = z3.shape
        if r1 != r1b or r2 != r2b:
            raise ValueError("inconsistent ranks")
        a1 = np.ascontiguousarray(z1.T)
        a2 = np.ascontiguousarray(z2)
        a3 = np.ascontiguousarray(z3.T)
        h = _P()
        self.check(self.lib.tt_create(self.h, n_t, n_xi, n_x, r1, r2, int(cap[0]), int(cap[1]), F64,
                                      a1.ctypes.data, a2.ctypes.data, a3.ctypes.data, 0, C.byref(h)))
        return TTHandle(self, h)

    def round(self, t, eps):
        out = _P(); nb = _D(); na = _D()
        self.check(self.lib.tt_round(self.h, t.h, eps, C.byref(out), C.byref(nb), C.byref(na)))
        return TTHandle(self, out), nb.value, na.value

    def round_randomized(self, t, eps, seed=1):
        """Randomized T_eps: (train, ||t||, ||T(t)||, sketch width)."""
        out = _P(); nb = _D(); na = _D(); sk = _I()
        self.check(self.lib.tt_round_randomized(self.h, t.h, eps, seed, C.byref(out), C.byref(nb), C.byref(na),
                                                C.byref(sk)))
        return TTHandle(self, out), nb.value, na.value, sk.value

    def round_to(self, t, eps, out):
        """T_eps(t) into the existing train `out`; returns (status, ||t||, ||T(t)||),
        status TT_ERANK when out's capacity cut a rank."""
        nb = _D(); na = _D()
        code = self.check(self.lib.tt_round_to(self.h, t.h, eps, out.h, C.byref(nb), C.byref(na)), allow=(TT_ERANK,))
        return code, nb.value, na.value

    def dot(self, a, b):
        out = _D()
        self.check(self.lib.tt_dot(self.h, a.h, b.h, C.byref(out)))
        return out.value

    def norm(self, a):
        out = _D()
        self.check(self.lib.tt_norm(self.h, a.h, C.byref(out)))
        return out.value

    def dot_noalloc(self, a, b):
        """<a, b> through the allocation-free entry point (static device scratch)."""
        out = _D()
        self.check(self.lib.tt_dot_noalloc(self.h, a.h, b.h, C.byref(out)))
        return out.value

    def axpby(self, alpha, a, beta, b, eps=0.0):
        out = _P()
        self.check(self.lib.tt_axpby(self.h, alpha, a.h, beta, b.h, eps, C.byref(out)))
        return TTHandle(self, out)

    # ---- problem -------------------------------------------------------------
    def problem(self, prob):
        return ProblemHandle(self, prob)


class TTHandle:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h

    def shape(self):
        v = [_I() for _ in range(5)]
        self.ctx.check(self.ctx.lib.tt_shape(self.h, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    @property
    def ranks(self):
        s = self.shape()
        return (s[3], s[4])

    @property
    def capacity(self):
        a, b = _I(), _I()
        self.ctx.check(self.ctx.lib.tt_capacity(self.h, C.byref(a), C.byref(b)))
        return (a.value, b.value)

    def cores(self):
        n_t, n_xi, n_x, r1, r2 = self.shape()
        a1 = np.empty((r1, n_t)); a2 = np.empty((r1, n_xi, r2)); a3 = np.empty((n_x, r2))
        self.ctx.check(self.ctx.lib.tt_get_cores(self.ctx.h, self.h, a1.ctypes.data, a2.ctypes.data,
                                                 a3.ctypes.data, 0))
        return a1.T.copy(), a2, a3.T.copy()

    def close(self):
        if self.h:
            self.ctx.lib.tt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def opts_from(tol, **over):
    """SolverOpts from a tolerance record; keyword overrides (precision=MIXED,
    learned=NetHandle, init=(u, p) TTHandles, ...)."""
    o = SolverOpts(tol_picard=tol.tol_picard, tol_gmres=tol.tol_gmres, eps_gmres=tol.eps_gmres,
                   eps_soln=tol.eps_soln, eps_conv=tol.eps_conv, tol_inner=tol.tol_inner,
                   maxit_picard=tol.maxit_picard, maxit_gmres=tol.maxit_gmres, maxit_inner=tol.maxit_inner,
                   precision=FP64)
    for k, v in over.items():
        if k == "learned":
            o.learned = v.h if v is not None else None
            o._net = v          # keep the network alive with the options
        elif k == "init":
            o.init_u, o.init_p = (v[0].h, v[1].h) if v is not None else (None, None)
            o._init = v
        else:
            setattr(o, k, v)
    return o


class ProblemHandle:
    """Device discretisation built from a `synth.Problem` (arrays copied by the library)."""

    def __init__(self, ctx, prob):
        self.ctx = ctx
        self.prob = prob
        m = prob.mesh
        self._keep = dict(
            xy=np.ascontiguousarray(m.xy, np.float64),
            q2=np.ascontiguousarray(m.elem_q2, np.int64),
            q1=np.ascontiguousarray(m.elem_q1, np.int64),
            dir=np.ascontiguousarray(m.dirichlet.astype(np.uint8)),
            inflow=np.ascontiguousarray(m.inflow, np.float64),
            mi=np.ascontiguousarray(prob.mi, np.int64),
            nu=np.ascontiguousarray(prob.nu, np.float64),
            tp=np.ascontiguousarray(prob.tprofile, np.float64))
        k = self._keep
        d = ProblemDesc(n_nodes=m.n_nodes, n_elem=m.n_elem, n_pnodes=m.n_pnodes, h=m.h,
                        xy=k["xy"].ctypes.data_as(_DP),
                        elem_q2=k["q2"].ctypes.data_as(C.POINTER(C.c_longlong)),
                        elem_q1=k["q1"].ctypes.data_as(C.POINTER(C.c_longlong)),
                        dirichlet=k["dir"].ctypes.data_as(C.POINTER(C.c_ubyte)),
                        inflow=k["inflow"].ctypes.data_as(_DP), m=prob.m, n_xi=prob.n_xi,
                        multi_index=k["mi"].ctypes.data_as(C.POINTER(C.c_longlong)),
                        nu=k["nu"].ctypes.data_as(_DP), n_t=prob.n_t, tau=prob.tau,
                        tprofile=k["tp"].ctypes.data_as(_DP))
        h = _P()
        ctx.check(ctx.lib.tt_problem_create(ctx.h, C.byref(d), C.byref(h)))
        self.h = h

    def sizes(self):
        v = [_I() for _ in range(6)]
        self.ctx.check(self.ctx.lib.tt_problem_sizes(self.h, *[C.byref(x) for x in v]))
        return dict(zip(("n_u", "n_p", "n_v", "n_xi", "n_t", "n_nodes"), (x.value for x in v)))

    def matrix(self, which, block=0):
        """(rowptr, col, vals, shape) of an assembled matrix (see tt_problem_matrix)."""
        nr, nc, nnz = _I(), _I(), _I()
        lib = self.ctx.lib
        self.ctx.check(lib.tt_problem_matrix(self.ctx.h, self.h, which, block, C.byref(nr), C.byref(nc),
                                             C.byref(nnz), None, None, None))
        rp = np.empty(nr.value + 1, np.int32); cl = np.empty(max(nnz.value, 1), np.int32)
        vals = np.empty(max(nnz.value, 1))
        self.ctx.check(lib.tt_problem_matrix(self.ctx.h, self.h, which, block, None, None, None,
                                             rp.ctypes.data_as(_IP), cl.ctypes.data_as(_IP),
                                             vals.ctypes.data_as(_DP)))
        return rp, cl[:nnz.value], vals[:nnz.value], (nr.value, nc.value)

    def rhs(self):
        a, b = _P(), _P()
        self.ctx.check(self.ctx.lib.tt_rhs(self.ctx.h, self.h, C.byref(a), C.byref(b)))
        return TTHandle(self.ctx, a), TTHandle(self.ctx, b)

    def full_velocity(self, u):
        w = _P()
        self.ctx.check(self.ctx.lib.tt_full_velocity(self.ctx.h, self.h, u.h, C.byref(w)))
        return TTHandle(self.ctx, w)

    def op(self, w=None, which=OP_FULL):
        h = _P()
        self.ctx.check(self.ctx.lib.tt_op_create(self.ctx.h, self.h, w.h if w is not None else None, which,
                                                 C.byref(h)))
        return OpHandle(self.ctx, h, which)

    def residual(self, u, p, eps):
        a, b, n = _P(), _P(), _D()
        self.ctx.check(self.ctx.lib.tt_residual(self.ctx.h, self.h, u.h, p.h, eps, C.byref(a), C.byref(b),
                                                C.byref(n)))
        return TTHandle(self.ctx, a), TTHandle(self.ctx, b), n.value

    def picard(self, opts):
        a, b = _P(), _P()
        st = PicardStats()
        code = self.ctx.check(self.ctx.lib.picard_solve(self.ctx.h, self.h, C.byref(opts), C.byref(a),
                                                        C.byref(b), C.byref(st)), allow=(TT_ENOCONV,))
        return TTHandle(self.ctx, a), TTHandle(self.ctx, b), st, code

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.tt_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class OpHandle:
    def __init__(self, ctx, h, which):
        self.ctx, self.h, self.which = ctx, h, which

    def matvec(self, u, p=None, eps=0.0):
        a, b = _P(), _P()
        self.ctx.check(self.ctx.lib.tt_matvec(self.ctx.h, self.h, u.h, p.h if p is not None else None, eps,
                                              C.byref(a), C.byref(b) if self.which == OP_FULL else None))
        if self.which == OP_FULL:
            return TTHandle(self.ctx, a), TTHandle(self.ctx, b)
        return TTHandle(self.ctx, a)

    def prec(self, au, ap, eps, tol_inner, maxit_inner, kind=PREC_LSC, net=None):
        """Apply the preconditioner of eq. (prec) once: (u, p, inner_its, fallbacks)."""
        pr = self.make_prec(kind, eps, tol_inner, maxit_inner, net)
        return pr.apply(au, ap)

    def make_prec(self, kind, eps, tol_inner, maxit_inner, net=None):
        o = PrecOpts(eps=eps, tol_inner=tol_inner, maxit_inner=maxit_inner, net=net.h if net is not None else None)
        h = _P()
        self.ctx.check(self.ctx.lib.tt_prec_create(self.ctx.h, self.h, kind, C.byref(o), C.byref(h)))
        return PrecHandle(self.ctx, h, self, net)

    def gmres(self, opts, bu, bp, bnorm=0.0, prec=None):
        a, b = _P(), _P()
        st = GmresStats()
        code = self.ctx.check(self.ctx.lib.tt_gmres(self.ctx.h, self.h, prec.h if prec is not None else None,
                                                    C.byref(opts), bu.h, bp.h, bnorm, C.byref(a), C.byref(b),
                                                    C.byref(st)), allow=(TT_ENOCONV,))
        return TTHandle(self.ctx, a), TTHandle(self.ctx, b), st, code

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.tt_op_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PrecHandle:
    def __init__(self, ctx, h, op, net):
        self.ctx, self.h, self.op, self.net = ctx, h, op, net

    def apply(self, au, ap):
        a, b, its, fb = _P(), _P(), _I(), _I()
        self.ctx.check(self.ctx.lib.tt_prec_apply(self.ctx.h, self.h, au.h, ap.h, C.byref(a), C.byref(b),
                                                  C.byref(its), C.byref(fb)))
        return TTHandle(self.ctx, a), TTHandle(self.ctx, b), its.value, fb.value

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.tt_prec_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _block(a):
    """(count, n_u) residual rows -> the library's n_u x count row-major block."""
    a = np.asarray(a, np.float64)
    return np.ascontiguousarray(a.T)


class NetHandle:
    """Learned mean-Oseen solve (tt_net_*): parameters flat FP32 in the library's
    layout (per layer W[out][in][3][3] then b[out])."""

    def __init__(self, problem, channels, depth, params):
        self.ctx = problem.ctx
        self.problem = problem
        p = np.ascontiguousarray(np.asarray(params, np.float32))
        h = _P()
        self.ctx.check(self.ctx.lib.tt_net_create(self.ctx.h, problem.h, channels, depth,
                                                  p.ctypes.data_as(_FP), C.byref(h)))
        self.h = h

    def set_tensor_cores(self, on):
        self.ctx.check(self.ctx.lib.tt_net_set_tensor_cores(self.h, 1 if on else 0))

    def info(self):
        n, nx, ny = _I(), _I(), _I()
        self.ctx.check(self.ctx.lib.tt_net_info(self.h, C.byref(n), C.byref(nx), C.byref(ny)))
        return n.value, nx.value, ny.value

    def params(self):
        out = np.empty(self.info()[0], np.float32)
        self.ctx.check(self.ctx.lib.tt_net_get_params(self.ctx.h, self.h, out.ctypes.data_as(_FP)))
        return out

    def apply(self, op, R):
        """Phi(r) for every row r of R (count, n_u) -> (count, n_u)."""
        A = _block(R)
        out = np.empty_like(A)
        self.ctx.check(self.ctx.lib.tt_net_apply(self.ctx.h, self.h, op.h, A.ctypes.data_as(_DP), A.shape[1], 0,
                                                 out.ctypes.data_as(_DP)))
        return out.T.copy()

    def loss_grad(self, op, R, T):
        A, Tb = _block(R), _block(T)
        loss = _D()
        g = np.empty(self.info()[0], np.float32)
        self.ctx.check(self.ctx.lib.tt_net_loss_grad(self.ctx.h, self.h, op.h, A.ctypes.data_as(_DP),
                                                     Tb.ctypes.data_as(_DP), A.shape[1], 0, C.byref(loss),
                                                     g.ctypes.data_as(_FP)))
        return loss.value, g

    def train(self, op, R, epochs, batch, lr, smooth_max=0, omega=2.0 / 3.0):
        A = _block(R)
        o = TrainOpts(epochs=epochs, batch=batch, lr=lr, smooth_max=smooth_max, omega=omega)
        losses = np.zeros(max(epochs, 1))
        self.ctx.check(self.ctx.lib.tt_net_train(self.ctx.h, self.h, op.h, A.ctypes.data_as(_DP), A.shape[1], 0,
                                                 C.byref(o), losses.ctypes.data_as(_DP)))
        return losses[:epochs]

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.tt_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def picard_batched(problems, opts):
    """Solve independent problems concurrently (picard_solve_batched).  `problems`:
    ProblemHandles on pairwise different contexts; `opts`: one SolverOpts per problem
    (or one for all).  Returns [(u, p, stats, status, seconds)] in input order."""
    n = len(problems)
    if n == 0:
        return []
    if isinstance(opts, SolverOpts):
        opts = [opts] * n
    lib = problems[0].ctx.lib
    probs = (_P * n)(*[pr.h for pr in problems])
    oarr = (SolverOpts * n)(*opts)
    U, Pp = (_P * n)(), (_P * n)()
    st = (PicardStats * n)()
    codes, secs = (_I * n)(), (_D * n)()
    code = lib.picard_solve_batched(n, probs, oarr, U, Pp, st, codes, secs)
    if code == TT_EINVAL and all(c == TT_OK for c in codes):
        problems[0].ctx._check(code)
    out = []
    for i, pr in enumerate(problems):
        u = TTHandle(pr.ctx, _P(U[i])) if U[i] else None
        p = TTHandle(pr.ctx, _P(Pp[i])) if Pp[i] else None
        out.append((u, p, st[i], codes[i], secs[i]))
    return out
