"""Python binding of librbicg.so (include/rbicg.h): argument marshalling only.

Every step of the solve runs in the CUDA library; PyTorch provides device memory and
streams.  Importing this module loads the library and raises if it is missing (there is no
CPU fallback).  Build it with `python -m paper_1010_0762_gb300.build`.

Names follow the C ABI: Solver.update_recycle / Solver.solve_pair / Solver.destroy wrap
rbicg_update_recycle / rbicg_solve_pair / rbicg_destroy; op_* wrap the component entry
points.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librbicg.so")

OK, NOT_CONVERGED, BREAKDOWN_RHO, BREAKDOWN_PQ, RECYCLE_EMPTY = 0, 1, 2, 3, 4
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NONFINITE, ERR_EIG = -1, -2, -3, -4, -5, -6
R64, C128 = 0, 1
FP64, FP32_REFINED = 0, 1


class Params(C.Structure):
    _fields_ = [("k", C.c_int), ("s", C.c_int), ("max_itn", C.c_int), ("tol", C.c_double),
                ("svd_tol", C.c_double), ("inner_tol", C.c_double), ("refine_max", C.c_int),
                ("precision", C.c_int), ("seed", C.c_uint64), ("setup_fp32", C.c_int),
                ("recycle", C.c_int), ("inner_svd_tol", C.c_double), ("guard", C.c_double),
                ("restarts", C.c_int), ("grid_blocks", C.c_int), ("refresh", C.c_int),
                ("setup_blocks", C.c_int), ("graphs", C.c_int)]


class CSRStruct(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("val", C.c_void_p), ("val_complex", C.c_int), ("has_shift", C.c_int),
                ("shift_re", C.c_double), ("shift_im", C.c_double)]


class Result(C.Structure):
    _fields_ = [("iters", C.c_int), ("cycles", C.c_int), ("recycle_dim", C.c_int), ("refine_steps", C.c_int),
                ("relres", C.c_double), ("relres_dual", C.c_double), ("true_relres", C.c_double),
                ("true_relres_dual", C.c_double), ("status", C.c_int), ("fallback", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class IrkaParams(C.Structure):
    _fields_ = [("r", C.c_int), ("max_steps", C.c_int), ("shift_tol", C.c_double), ("strategy", C.c_int),
                ("recycle_count", C.c_int), ("refresh_every", C.c_int), ("pool_tol", C.c_double),
                ("batched", C.c_int), ("conj_pairs", C.c_int)]


class IrkaResult(C.Structure):
    _fields_ = [("steps", C.c_int), ("converged", C.c_int), ("last_change", C.c_double), ("iters", C.c_int64),
                ("failed_solves", C.c_int), ("model_shifts", C.c_double * 64)]


class RBiCGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("rbicg status %d: %s" % (status, msg))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("librbicg.so not found at %s; build it with `python -m paper_1010_0762_gb300.build`"
                           % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    vp, i64, ci, cd = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "rbicg_default_params": (None, [C.POINTER(Params)]),
        "rbicg_create": (ci, [C.POINTER(Params), i64, ci, vp, C.POINTER(vp)]),
        "rbicg_update_recycle": (ci, [vp, C.POINTER(CSRStruct)]),
        "rbicg_solve_pair": (ci, [vp, C.POINTER(CSRStruct), vp, vp, vp, vp, C.POINTER(Result)]),
        "rbicg_solve_batch": (ci, [C.POINTER(vp), C.POINTER(C.POINTER(CSRStruct)), C.POINTER(vp), C.POINTER(vp),
                                   C.POINTER(vp), C.POINTER(vp), ci, C.POINTER(Result)]),
        "rbicg_export_recycle": (ci, [vp, vp, vp, C.POINTER(ci)]),
        "rbicg_import_recycle": (ci, [vp, vp, vp, ci]),
        "rbicg_reset": (ci, [vp]),
        "rbicg_set_refresh": (ci, [vp, ci]),
        "rbicg_residual_history": (ci, [vp, vp, ci, C.POINTER(ci)]),
        "rbicg_destroy": (ci, [vp]),
        "rbicg_last_error": (C.c_char_p, [vp]),
        "rbicg_launch_count": (i64, [vp]),
        "rbicg_profile": (ci, [vp, ci, C.POINTER(cd), C.POINTER(i64)]),
        "rbicg_profile_columns": (ci, [vp, C.POINTER(i64)]),
        "rbicg_profile_gram_pairs": (ci, [vp, C.POINTER(i64)]),
        "rbicg_op_dual_spmv_project": (ci, [C.POINTER(CSRStruct), ci, vp, vp, vp, vp, cd, cd, vp, vp, ci, ci,
                                            vp, vp, vp, vp, vp, vp, vp, vp]),
        "rbicg_op_gram": (ci, [ci, i64, vp, ci, ci, vp, ci, ci, ci, vp, vp]),
        "rbicg_op_eig_select": (ci, [ci, ci, vp, vp, ci, vp, vp, vp, C.POINTER(ci), vp]),
        "rbicg_op_svd": (ci, [ci, ci, vp, vp, vp, vp, vp]),
        "rbicg_autotune": (ci, [C.POINTER(Params), ci, C.POINTER(CSRStruct), ci, C.POINTER(ci), C.POINTER(cd)]),
        "rbicg_autotune_params": (ci, [C.POINTER(Params), ci, C.POINTER(CSRStruct), ci, C.POINTER(Params),
                                       C.POINTER(cd)]),
        "rbicg_engine_create": (ci, [vp, C.POINTER(vp)]),
        "rbicg_engine_submit": (ci, [vp, vp, C.POINTER(CSRStruct), vp, vp, vp, vp, i64]),
        "rbicg_engine_step": (ci, [vp, C.POINTER(ci)]),
        "rbicg_engine_poll": (ci, [vp, C.POINTER(i64), C.POINTER(Result), ci, C.POINTER(ci)]),
        "rbicg_engine_destroy": (ci, [vp]),
        "rbicg_bilinear_form": (ci, [C.POINTER(CSRStruct), ci, vp, vp, vp, vp, vp, vp]),
        "rbicg_irka_default_params": (None, [C.POINTER(IrkaParams)]),
        "rbicg_irka": (ci, [C.POINTER(Params), C.POINTER(IrkaParams), C.POINTER(CSRStruct), vp, vp, vp, vp,
                            vp, vp, vp, vp, vp, vp, C.POINTER(IrkaResult)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _check(st, handle=None):
    if st < 0:
        msg = lib.rbicg_last_error(handle)
        raise RBiCGError(st, msg.decode() if msg else "")
    return st


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def default_params(**kw):
    p = Params()
    lib.rbicg_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": FP64, "fp32_refined": FP32_REFINED}[v]
        setattr(p, k, v)
    return p


class Operator:
    """A sparse operator on the device: A (CSR) or, with `shift`, (shift I - A).

    Keeps the device tensors alive while the library may read them.
    """

    def __init__(self, row_ptr, col_idx, val, shift=None):
        self.row_ptr = row_ptr.contiguous()
        self.col_idx = col_idx.contiguous()
        self.val = val.contiguous()
        assert self.row_ptr.dtype == torch.int32 and self.col_idx.dtype == torch.int32
        assert self.val.dtype in (torch.float64, torch.complex128)
        self.n = self.row_ptr.numel() - 1
        self.shift = shift
        s = CSRStruct()
        s.n = self.n
        s.nnz = self.col_idx.numel()
        s.row_ptr = self.row_ptr.data_ptr()
        s.col_idx = self.col_idx.data_ptr() if self.col_idx.numel() else 0
        s.val = self.val.data_ptr() if self.val.numel() else 0
        s.val_complex = 1 if self.val.dtype == torch.complex128 else 0
        s.has_shift = 1 if shift is not None else 0
        if shift is not None:
            s.shift_re = float(np.real(shift))
            s.shift_im = float(np.imag(shift))
        self.struct = s

    @classmethod
    def from_csr(cls, A, device="cuda", shift=None):
        """From paper_1010_0762_gb300.inputs.CSR (or anything with row_ptr/col_idx/val arrays)."""
        val = np.asarray(A.val)
        vt = torch.complex128 if np.iscomplexobj(val) else torch.float64
        return cls(torch.as_tensor(np.asarray(A.row_ptr, dtype=np.int32), device=device),
                   torch.as_tensor(np.asarray(A.col_idx, dtype=np.int32), device=device),
                   torch.as_tensor(val, dtype=vt, device=device), shift=shift)


class Solver:
    """RBiCG solver for a sequence of dual systems of order n (rbicg_create)."""

    def __init__(self, n, dtype=R64, stream=None, **params):
        self.n = int(n)
        self.dtype = dtype
        self.params = default_params(**params)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib.rbicg_create(C.byref(self.params), self.n, dtype, _stream(self.stream), C.byref(h)))
        self.h = h
        self._op = None

    def update_recycle(self, op: Operator):
        self._op = op
        _check(lib.rbicg_update_recycle(self.h, C.byref(op.struct)), self.h)

    def solve_pair(self, op, b, bt, x, xt):
        """Solve A x = b, A^H xt = bt; x, xt hold the initial guesses and receive the solutions."""
        if op is not None:
            self._op = op
        r = Result()
        opp = C.byref(op.struct) if op is not None else None
        st = lib.rbicg_solve_pair(self.h, opp, _ptr(b), _ptr(bt), _ptr(x), _ptr(xt), C.byref(r))
        _check(st, self.h)
        return r.as_dict()

    def export_recycle(self):
        k = self.params.k
        dt = torch.complex128 if self.dtype == C128 else torch.float64
        U = torch.zeros(self.n, k, dtype=dt, device="cuda")
        Ut = torch.zeros(self.n, k, dtype=dt, device="cuda")
        p = C.c_int(0)
        _check(lib.rbicg_export_recycle(self.h, _ptr(U), _ptr(Ut), C.byref(p)), self.h)
        return U[:, :p.value].clone(), Ut[:, :p.value].clone()

    def import_recycle(self, U, Ut):
        U = U.contiguous(); Ut = Ut.contiguous()
        _check(lib.rbicg_import_recycle(self.h, _ptr(U), _ptr(Ut), U.shape[1]), self.h)

    def reset(self):
        _check(lib.rbicg_reset(self.h), self.h)

    def residual_history(self, max_count=132):
        """||r_m|| of the last solve's last iterations (oldest first)."""
        out = np.zeros(max_count)
        cnt = C.c_int(0)
        _check(lib.rbicg_residual_history(self.h, out.ctypes.data_as(C.c_void_p), max_count, C.byref(cnt)), self.h)
        return out[:cnt.value].copy()

    def set_refresh(self, refresh):
        _check(lib.rbicg_set_refresh(self.h, int(refresh)), self.h)
        self.params.refresh = int(refresh)

    def launch_count(self):
        return int(lib.rbicg_launch_count(self.h))

    def destroy(self):
        if getattr(self, "h", None):
            lib.rbicg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ------------------------------------------------------------------ component entry points
def autotune(op, dtype=None, trial_iters=60, **params):
    """Launch shape (blocks per iteration phase) for operator `op` by timed trials; returns
    (grid_blocks, microseconds per iteration).  Pass grid_blocks=... to Solver to use it."""
    p = default_params(**params)
    if dtype is None:
        dtype = C128 if op.val.dtype == torch.complex128 else R64
    g = C.c_int(0)
    us = C.c_double(0.0)
    _check(lib.rbicg_autotune(C.byref(p), dtype, C.byref(op.struct), int(trial_iters), C.byref(g), C.byref(us)))
    return g.value, us.value


def autotune_params(op, dtype=None, trial_iters=60, **params):
    """Launch knobs for operator `op` by timed trials (rbicg_autotune_params): returns a dict with
    grid_blocks, setup_blocks and graphs (pass them to Solver) and the time per recycled iteration."""
    p = default_params(**params)
    if dtype is None:
        dtype = C128 if op.val.dtype == torch.complex128 else R64
    out = Params()
    us = C.c_double(0.0)
    _check(lib.rbicg_autotune_params(C.byref(p), dtype, C.byref(op.struct), int(trial_iters), C.byref(out),
                                     C.byref(us)))
    return {"grid_blocks": out.grid_blocks, "setup_blocks": out.setup_blocks, "graphs": out.graphs,
            "us_per_iter": us.value}


class Engine:
    """Continuous batching (rbicg_engine_*): submit requests, step cycles, poll results."""

    def __init__(self, stream=None):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib.rbicg_engine_create(_stream(self.stream), C.byref(h)))
        self.h = h
        self._keep = {}   # tag -> tensors that must outlive the request

    def submit(self, solver, op, b, bt, x, xt, tag):
        if op is not None:
            solver._op = op
        opp = C.byref(op.struct) if op is not None else None
        st = lib.rbicg_engine_submit(self.h, solver.h, opp, _ptr(b), _ptr(bt), _ptr(x), _ptr(xt), int(tag))
        _check(st, solver.h)
        self._keep[int(tag)] = (op, b, bt, x, xt)

    def step(self):
        n = C.c_int(0)
        _check(lib.rbicg_engine_step(self.h, C.byref(n)))
        return n.value

    def poll(self, max_count=64):
        tags = (C.c_int64 * max_count)()
        res = (Result * max_count)()
        cnt = C.c_int(0)
        _check(lib.rbicg_engine_poll(self.h, tags, res, max_count, C.byref(cnt)))
        out = []
        for i in range(cnt.value):
            self._keep.pop(int(tags[i]), None)
            out.append((int(tags[i]), res[i].as_dict()))
        return out

    def close(self):
        if self.h:
            lib.rbicg_engine_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(solvers, ops, bs, bts, xs, xts):
    """Solve len(solvers) dual pairs together (rbicg_solve_batch): one launch per iteration phase
    for all of them; each solver keeps its own recycle space; results equal solving alone."""
    cnt = len(solvers)
    H = (C.c_void_p * cnt)(*[s_.h.value for s_ in solvers])
    As = (C.POINTER(CSRStruct) * cnt)(*[C.pointer(o.struct) if o is not None else None for o in ops])
    P = lambda ts: (C.c_void_p * cnt)(*[_ptr(t) for t in ts])
    out = (Result * cnt)()
    for s_, o in zip(solvers, ops):
        if o is not None:
            s_._op = o
    st = lib.rbicg_solve_batch(H, As, P(bs), P(bts), P(xs), P(xts), cnt, out)
    _check(st, solvers[0].h if cnt else None)
    return [out[i].as_dict() for i in range(cnt)]


def op_dual_spmv_project(op: Operator, r, rt, p_old, pt_old, beta, C_=None, Ct=None, Dc=None, stream=None):
    """Phase 1 of an iteration: returns (p, pt, z, zt, zeta, zetat)."""
    cx = r.dtype == torch.complex128
    dtype = C128 if cx else R64
    p = torch.empty_like(r); pt = torch.empty_like(r); z = torch.empty_like(r); zt = torch.empty_like(r)
    k = 0 if C_ is None else C_.shape[1]
    ldc = 0 if C_ is None else C_.stride(0)
    zeta = np.zeros(k, dtype=np.complex128 if cx else np.float64)
    zetat = np.zeros_like(zeta)
    dc = np.ascontiguousarray(Dc, dtype=np.float64) if k else np.zeros(1)
    st = lib.rbicg_op_dual_spmv_project(
        C.byref(op.struct), dtype, _ptr(r), _ptr(rt), _ptr(p_old), _ptr(pt_old), float(np.real(beta)),
        float(np.imag(beta)), _ptr(C_), _ptr(Ct), k, ldc, dc.ctypes.data_as(C.c_void_p), _ptr(p), _ptr(pt),
        _ptr(z), _ptr(zt), zeta.ctypes.data_as(C.c_void_p), zetat.ctypes.data_as(C.c_void_p), _stream(stream))
    _check(st)
    return p, pt, z, zt, zeta, zetat


def op_gram(X, Y, fp32=False, stream=None):
    """G = X^H Y for row-major device matrices X (n x mx), Y (n x my); returns numpy."""
    cx = X.dtype == torch.complex128
    G = np.zeros((X.shape[1], Y.shape[1]), dtype=np.complex128 if cx else np.float64)
    st = lib.rbicg_op_gram(C128 if cx else R64, X.shape[0], _ptr(X), X.shape[1], X.stride(0), _ptr(Y),
                           Y.shape[1], Y.stride(0), int(bool(fp32)), G.ctypes.data_as(C.c_void_p),
                           _stream(stream))
    _check(st)
    return G


def op_eig_select(L, R, k, complex_=None, stream=None):
    """Eigenvectors of L w = lambda R w for the k eigenvalues closest to 0 (R None: L w = lambda w)."""
    cx = np.iscomplexobj(L) or (R is not None and np.iscomplexobj(R)) if complex_ is None else complex_
    dt = np.complex128 if cx else np.float64
    m = L.shape[0]
    Lf = np.asfortranarray(L, dtype=dt)
    Rf = np.asfortranarray(R, dtype=dt) if R is not None else None
    W = np.zeros((m, k), dtype=dt, order="F")
    Wt = np.zeros((m, k), dtype=dt, order="F")
    lam = np.zeros(2 * k + 2)
    kk = C.c_int(0)
    st = lib.rbicg_op_eig_select(C128 if cx else R64, m, Lf.ctypes.data_as(C.c_void_p),
                                 Rf.ctypes.data_as(C.c_void_p) if Rf is not None else None, k,
                                 W.ctypes.data_as(C.c_void_p), Wt.ctypes.data_as(C.c_void_p),
                                 lam.ctypes.data_as(C.c_void_p), C.byref(kk), _stream(stream))
    _check(st)
    q = kk.value
    return W[:, :q], Wt[:, :q], lam[0:2 * q:2] + 1j * lam[1:2 * q:2]


def op_svd(S, stream=None):
    """S = M diag(sigma) N^H (one-sided Jacobi on the GPU); returns (M, sigma, N)."""
    cx = np.iscomplexobj(S)
    dt = np.complex128 if cx else np.float64
    k = S.shape[0]
    Sf = np.asfortranarray(S, dtype=dt)
    M = np.zeros((k, k), dtype=dt, order="F")
    N = np.zeros((k, k), dtype=dt, order="F")
    sig = np.zeros(k)
    st = lib.rbicg_op_svd(C128 if cx else R64, k, Sf.ctypes.data_as(C.c_void_p), M.ctypes.data_as(C.c_void_p),
                          sig.ctypes.data_as(C.c_void_p), N.ctypes.data_as(C.c_void_p), _stream(stream))
    _check(st)
    return M, sig, N


# ------------------------------------------------------------------ applications
def bilinear_form(op: Operator, u, w, x, xt, stream=None):
    """u^H Op^{-1} w from a solved pair Op x = w, Op^H xt = u (rbicg_bilinear_form): returns the
    primal estimate u^H x, the dual estimate xt^H w and the corrected u^H x + xt^H (w - Op x)."""
    dtype = C128 if x.dtype == torch.complex128 else R64
    out = np.zeros(6)
    _check(lib.rbicg_bilinear_form(C.byref(op.struct), dtype, _ptr(u), _ptr(w), _ptr(x), _ptr(xt),
                                   out.ctypes.data_as(C.c_void_p), _stream(stream)))
    z = out[0::2] + 1j * out[1::2]
    return (z if dtype == C128 else z.real)


def irka(op: Operator, b, c, shifts, stream=None, **kw):
    """IRKA (Algorithm 3) for G(s) = c^H (s I - A)^{-1} b with the library's RBiCG solves
    (rbicg_irka).  op: the real matrix A (no shift); b, c: real device vectors; shifts: the r
    initial shifts.  Keyword arguments set rbicg_irka_params fields (r is len(shifts)) and, with a
    solver_ prefix, rbicg_params fields of the solves (e.g. solver_k=16).  Returns a dict with the
    final shifts, the reduced model (Ar, Er, br, cr) of the last step, the shifts it interpolates at,
    per-solve iteration counts (steps x r) and the run's counters."""
    ip = IrkaParams()
    lib.rbicg_irka_default_params(C.byref(ip))
    sp = {}
    for k_, v in kw.items():
        if k_.startswith("solver_"):
            sp[k_[len("solver_"):]] = v
        else:
            setattr(ip, k_, v)
    r = len(shifts)
    ip.r = r
    p = default_params(**sp)
    sh = np.zeros(2 * r)
    sh[0::2] = np.real(shifts)
    sh[1::2] = np.imag(shifts)
    out = np.zeros(2 * r)
    Ar = np.zeros(2 * r * r); Er = np.zeros(2 * r * r); br = np.zeros(2 * r); cr = np.zeros(2 * r)
    its = np.zeros(ip.max_steps * r, dtype=np.int32)
    res = IrkaResult()
    f = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(lib.rbicg_irka(C.byref(p), C.byref(ip), C.byref(op.struct), _ptr(b), _ptr(c), f(sh), _stream(stream),
                          f(out), f(Ar), f(Er), f(br), f(cr), f(its), C.byref(res)))
    cx = lambda a: a[0::2] + 1j * a[1::2]
    ms = np.array(res.model_shifts[:2 * r])
    return {"shifts": cx(out), "Ar": cx(Ar).reshape(r, r, order="F"), "Er": cx(Er).reshape(r, r, order="F"),
            "br": cx(br), "cr": cx(cr), "model_shifts": cx(ms), "iters": its.reshape(ip.max_steps, r)[:res.steps],
            "steps": res.steps, "converged": bool(res.converged), "last_change": res.last_change,
            "total_iters": int(res.iters), "failed_solves": res.failed_solves}
