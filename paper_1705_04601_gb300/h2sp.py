"""Python binding of the h2sp C ABI (include/h2sp.h): argument marshalling only.

Every step of the method runs inside libh2sp.so.  PyTorch is used here only to
hold device memory (tensors whose data pointers are passed through) and to
name the current CUDA stream.  The functions keep the C names.

Vector layout: a block of ``nrhs`` FP64 columns of length n is a contiguous
tensor of shape (nrhs, n) (row r = column r, leading dimension n), or shape
(n,) for one column.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libh2sp.so")

H2SP_OK, H2SP_EINVAL, H2SP_ENOMEM, H2SP_ECUDA, H2SP_ESINGULAR = 0, -1, -2, -3, -4
H2SP_ESTATE, H2SP_ENOCONV, H2SP_ETIMEOUT, H2SP_EUNSUPPORTED = -5, -6, -7, -8
H2SP_FP64, H2SP_FP32, H2SP_FP64_CHOL, H2SP_FP32_CHOL, H2SP_BF16_CHOL, H2SP_BF16X3_CHOL = 0, 1, 2, 3, 7, 15
H2SP_SPARSIFY_FP32 = 1  # h2sp_opts.flags bit
H2SP_OP_UT, H2SP_OP_V, H2SP_OP_U, H2SP_OP_VT, H2SP_OP_S, H2SP_OP_H2, H2SP_OP_SINV = range(7)
H2SP_DIRECT, H2SP_IR, H2SP_GMRES = 0, 1, 2

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class Desc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("depth", ctypes.c_int32),
        ("level_ptr", _i32p), ("parent", _i32p), ("begin", _i64p), ("size", _i64p), ("rank", _i32p),
        ("far_ptr", _i64p), ("far_col", _i32p), ("near_ptr", _i64p), ("near_col", _i32p),
        ("leaf_basis_off", _i64p), ("transfer_off", _i64p), ("coupling_off", _i64p), ("near_off", _i64p),
        ("col_leaf_basis_off", _i64p), ("col_transfer_off", _i64p),
        ("leaf_basis", _vp), ("transfer", _vp), ("coupling", _vp), ("near_block", _vp),
        ("col_leaf_basis", _vp), ("col_transfer", _vp),
    ]


class Opts(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tol", ctypes.c_double), ("maxit", ctypes.c_int32),
                ("restart", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("status", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("depth", ctypes.c_int32), ("lstop", ctypes.c_int32), ("nnodes", ctypes.c_int32),
        ("nnzb", ctypes.c_int64), ("nnz", ctypes.c_int64), ("nsupernodes", ctypes.c_int32),
        ("nfront_levels", ctypes.c_int32), ("max_front", ctypes.c_int64), ("front_elems", ctypes.c_int64),
        ("factor_flops", ctypes.c_double), ("sparsify_flops", ctypes.c_double), ("factor_prec", ctypes.c_int32),
        ("plan_seconds", ctypes.c_double), ("sparsify_prec", ctypes.c_int32), ("nsys", ctypes.c_int32),
        ("factor_chol", ctypes.c_int32), ("chol_flops", ctypes.c_double), ("compensated_pivots", ctypes.c_int32),
    ]


class KernelTimes(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 16), ("timed", ctypes.c_int64 * 16), ("ms", ctypes.c_double * 16),
                ("work", ctypes.c_double * 16)]


KERNEL_CLASSES = ["gemm_update", "panel", "swap_trsm", "extend_add", "assemble", "transform", "householder",
                  "coupling", "solve", "h2_matvec", "apply", "vector", "gemm_inner"]

# name -> (restype, argtypes); every symbol of include/h2sp.h
SIGNATURES = {
    "h2sp_sparsify": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.POINTER(Opts), _vp, ctypes.POINTER(_vp)]),
    "h2sp_sparsify_analyzed": (ctypes.c_int, [_vp, ctypes.POINTER(Desc), ctypes.POINTER(Opts), _vp,
                                              ctypes.POINTER(_vp)]),
    "h2sp_analyze": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.POINTER(_vp)]),
    "h2sp_factor": (ctypes.c_int, [_vp, ctypes.c_int32, _vp]),
    "h2sp_refactor": (ctypes.c_int, [_vp, _vp]),
    "h2sp_solve": (ctypes.c_int, [_vp, ctypes.POINTER(SolveOpts), ctypes.c_int32, _vp, ctypes.c_int64, _vp,
                                  ctypes.c_int64, ctypes.POINTER(SolveInfo), _vp]),
    "h2sp_logdet": (ctypes.c_int, [_vp, _f64p, _i32p, _vp]),
    "h2sp_apply": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int64, _vp, ctypes.c_int64,
                                  _vp]),
    "h2sp_export_S": (ctypes.c_int, [_vp, _i64p, _i64p, _i32p, _i64p, _f64p, _vp]),
    "h2sp_export_Q": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _i64p, _f64p, _vp]),
    "h2sp_export_structure": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p, _i64p]),
    "h2sp_export_schedule": (ctypes.c_int, [_vp, _i32p, _i64p, _i64p, _i64p, _i64p, _i64p, _i32p]),
    "h2sp_export_near": (ctypes.c_int, [_vp, ctypes.c_int32, _i64p, _i32p, _i64p]),
    "h2sp_construct": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp)]),
    "h2sp_factor_ilut": (ctypes.c_int, [_vp, ctypes.c_double, _vp]),
    "h2sp_export_ilut": (ctypes.c_int, [_vp, _i32p, _i64p, _i32p, _f64p, _i64p, _i32p, _f64p, _i64p, _i64p]),
    "h2sp_h2_describe": (ctypes.c_int, [_vp, _vp]),
    "h2sp_h2_copy": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _i64p, _vp]),
    "h2sp_h2_destroy": (None, [_vp]),
    "h2sp_export_front": (ctypes.c_int, [_vp, ctypes.c_int32, _i64p, _i64p, _f64p, _vp]),
    "h2sp_measure_peak": (ctypes.c_int, [ctypes.c_int32, _f64p, _vp]),
    "h2sp_set_option": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int64]),
    "h2sp_solve_captured": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _vp, ctypes.c_int64,
                                           _vp, ctypes.c_int64, ctypes.c_void_p, _vp]),
    "h2sp_solve_host": (ctypes.c_int, [_vp, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_int32, _vp, ctypes.c_int64, _vp, ctypes.c_int64, ctypes.c_void_p,
                                       _vp]),
    "h2sp_query": (ctypes.c_int, [_vp, ctypes.POINTER(Stats)]),
    "h2sp_profile": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(KernelTimes)]),
    "h2sp_h2_matvec_static": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.c_int64, _vp, ctypes.c_int64, _vp]),
    "h2sp_destroy": (None, [_vp]),
    "h2sp_status_string": (ctypes.c_char_p, [ctypes.c_int32]),
    "h2sp_last_cuda_error": (ctypes.c_char_p, []),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libh2sp.so (built in-tree); fail loudly if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libh2sp.so is not built (run __graft_entry__.build() or "
                               "python -m paper_1705_04601_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class H2spError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.h2sp_status_string(status).decode()
        detail = L.h2sp_last_cuda_error().decode()
        super().__init__("%s: %s (%d)%s" % (where, msg, status, (": " + detail) if detail else ""))
        self.status = status


def _check(st: int, where: str):
    if st != H2SP_OK:
        raise H2spError(st, where)


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


def _stream(stream):
    if stream is None:
        import torch
        return _vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


class H2Input:
    """An H^2 matrix marshalled for the ABI: host structure arrays (kept alive
    here) and device copies of the numeric arrays (torch tensors on cuda),
    or ``device=None`` for h2sp_analyze (no numbers), or ``device="host"``
    for h2sp_solve_host: the numeric arrays stay in host memory (``host``:
    optional dict of page-locked torch tensors holding them)."""

    def __init__(self, h, device="cuda", nonblocking_from=None, host=None):
        self.h = h
        c = np.ascontiguousarray
        self.arrs = dict(
            level_ptr=c(h.level_ptr, np.int32), parent=c(h.parent, np.int32), begin=c(h.begin, np.int64),
            size=c(h.size, np.int64), rank=c(h.rank, np.int32), far_ptr=c(h.far_ptr, np.int64),
            far_col=c(h.far_col, np.int32), near_ptr=c(h.near_ptr, np.int64), near_col=c(h.near_col, np.int32),
            leaf_basis_off=c(h.leaf_basis_off, np.int64), transfer_off=c(h.transfer_off, np.int64),
            coupling_off=c(h.coupling_off, np.int64), near_off=c(h.near_off, np.int64),
        )
        if h.col_rank is not None:
            self.arrs["col_leaf_basis_off"] = c(h.col_leaf_basis_off, np.int64)
            self.arrs["col_transfer_off"] = c(h.col_transfer_off, np.int64)
        self.dev = {}
        self.host_ptrs = {}
        if device == "host":
            names = ["leaf_basis", "transfer", "coupling", "near_block"]
            if h.col_rank is not None:
                names += ["col_leaf_basis", "col_transfer"]
            self._keep = []
            for nm in names:
                if host is not None:
                    self.host_ptrs[nm] = host[nm].data_ptr()
                else:
                    a = c(getattr(h, nm), np.float64)
                    self._keep.append(a)
                    self.host_ptrs[nm] = a.ctypes.data
        elif device is not None:
            import torch
            names = ["leaf_basis", "transfer", "coupling", "near_block"]
            if h.col_rank is not None:
                names += ["col_leaf_basis", "col_transfer"]
            for nm in names:
                a = getattr(h, nm)
                src = nonblocking_from[nm] if nonblocking_from else torch.from_numpy(c(a, np.float64))
                t = torch.empty(max(a.size, 1), dtype=torch.float64, device=device)
                t[:a.size].copy_(src[:a.size] if nonblocking_from else src, non_blocking=bool(nonblocking_from))
                self.dev[nm] = t

    def desc(self) -> Desc:
        a = self.arrs
        d = Desc()
        d.n = int(self.h.n)
        d.depth = int(self.h.depth)
        for nm in ("level_ptr", "parent", "rank", "far_col", "near_col"):
            setattr(d, nm, _ptr(a[nm], ctypes.c_int32))
        for nm in ("begin", "size", "far_ptr", "near_ptr", "leaf_basis_off", "transfer_off", "coupling_off",
                   "near_off", "col_leaf_basis_off", "col_transfer_off"):
            setattr(d, nm, _ptr(a.get(nm), ctypes.c_int64))
        for nm in ("leaf_basis", "transfer", "coupling", "near_block", "col_leaf_basis", "col_transfer"):
            t = self.dev.get(nm)
            setattr(d, nm, t.data_ptr() if t is not None else self.host_ptrs.get(nm))
        return d


class ConstructDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("dim", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("level_ptr", _i32p), ("parent", _i32p), ("begin", _i64p), ("size", _i64p),
                ("box_lo", _f64p), ("box_hi", _f64p), ("far_ptr", _i64p), ("far_col", _i32p),
                ("near_ptr", _i64p), ("near_col", _i32p), ("points", _vp), ("kernel", ctypes.c_int32),
                ("diag", ctypes.c_double), ("order", ctypes.c_int32), ("tol", ctypes.c_double)]


KERNEL_IDS = {"log": 0, "inv": 1, "yukawa": 2, "gauss": 3}


class Constructed:
    """An H^2 matrix built on the GPU by h2sp_construct; owns its arrays.
    Serves as the input of h2sp_analyze / h2sp_sparsify (``desc()``)."""

    def __init__(self, ptr: _vp, n: int, depth: int, ncl: int):
        self.ptr = ptr
        self.n, self.depth, self.ncl = n, depth, ncl
        self.h = self  # the entry points read .h.n

    def desc(self) -> "Desc":
        d = Desc()
        _check(lib().h2sp_h2_describe(self.ptr, ctypes.byref(d)), "h2sp_h2_describe")
        return d

    def copy(self, which: int) -> np.ndarray:
        """Host copy of numeric array `which` (0 leaf_basis, 1 transfer, 2 coupling, 3 near_block)."""
        cnt = ctypes.c_int64(0)
        _check(lib().h2sp_h2_copy(self.ptr, int(which), None, ctypes.byref(cnt), _vp(None)), "h2sp_h2_copy")
        out = np.zeros(max(cnt.value, 1), np.float64)
        _check(lib().h2sp_h2_copy(self.ptr, int(which), _vp(out.ctypes.data), ctypes.byref(cnt), _vp(None)),
               "h2sp_h2_copy")
        return out[:cnt.value]

    def close(self):
        if self.ptr is not None and self.ptr.value:
            lib().h2sp_h2_destroy(self.ptr)
        self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def h2sp_construct(tree: dict, points, kernel: str, diag: float, order: int = 4, tol: float = 0.0,
                   stream=None) -> Constructed:
    """Build the H^2 matrix of `kernel` on the GPU.  `tree`: host arrays
    level_ptr, parent, begin, size, box_lo, box_hi (ncl x dim), far_ptr,
    far_col, near_ptr, near_col and the depth; `points`: a CUDA float64 tensor
    (n x dim) in tree order."""
    c = np.ascontiguousarray
    keep = dict(level_ptr=c(tree["level_ptr"], np.int32), parent=c(tree["parent"], np.int32),
                begin=c(tree["begin"], np.int64), size=c(tree["size"], np.int64),
                box_lo=c(tree["box_lo"], np.float64), box_hi=c(tree["box_hi"], np.float64),
                far_ptr=c(tree["far_ptr"], np.int64), far_col=c(tree["far_col"], np.int32),
                near_ptr=c(tree["near_ptr"], np.int64), near_col=c(tree["near_col"], np.int32))
    d = ConstructDesc()
    d.n = int(points.shape[0])
    d.dim = int(points.shape[1])
    d.depth = int(tree["depth"])
    for nm in ("level_ptr", "parent", "far_col", "near_col"):
        setattr(d, nm, _ptr(keep[nm], ctypes.c_int32))
    for nm in ("begin", "size", "far_ptr", "near_ptr"):
        setattr(d, nm, _ptr(keep[nm], ctypes.c_int64))
    for nm in ("box_lo", "box_hi"):
        setattr(d, nm, _ptr(keep[nm], ctypes.c_double))
    pts = points.contiguous()
    d.points = _vp(pts.data_ptr())
    d.kernel = KERNEL_IDS[kernel]
    d.diag = float(diag)
    d.order = int(order)
    d.tol = float(tol)
    out = _vp()
    _check(lib().h2sp_construct(ctypes.byref(d), _stream(stream), ctypes.byref(out)), "h2sp_construct")
    return Constructed(out, d.n, d.depth, int(keep["parent"].size))


class Handle:
    """Owns an h2sp handle; destroys it when closed or collected."""

    def __init__(self, ptr: _vp, inp: H2Input):
        self.ptr = ptr
        self.inp = inp   # the borrowed device arrays must outlive the handle

    def close(self):
        if self.ptr is not None and self.ptr.value:
            lib().h2sp_destroy(self.ptr)
        self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def h2sp_analyze(inp: H2Input) -> Handle:
    out = _vp()
    d = inp.desc()
    _check(lib().h2sp_analyze(ctypes.byref(d), ctypes.byref(out)), "h2sp_analyze")
    return Handle(out, inp)


def h2sp_sparsify(inp: H2Input, stream=None, flags: int = 0) -> Handle:
    out = _vp()
    d = inp.desc()
    o = Opts(int(flags))
    _check(lib().h2sp_sparsify(ctypes.byref(d), ctypes.byref(o), _stream(stream), ctypes.byref(out)),
           "h2sp_sparsify")
    return Handle(out, inp)


def h2sp_sparsify_analyzed(an: Handle, inp: H2Input, stream=None, flags: int = 0) -> Handle:
    """h2sp_sparsify with the host analysis of `an` (same structure, new numbers)."""
    out = _vp()
    d = inp.desc()
    o = Opts(int(flags))
    _check(lib().h2sp_sparsify_analyzed(an.ptr, ctypes.byref(d), ctypes.byref(o), _stream(stream),
                                        ctypes.byref(out)), "h2sp_sparsify_analyzed")
    return Handle(out, inp)


def h2sp_factor(h: Handle, prec: int = H2SP_FP64, stream=None):
    _check(lib().h2sp_factor(h.ptr, int(prec), _stream(stream)), "h2sp_factor")


def h2sp_refactor(h: Handle, stream=None):
    """Sparsify and factor again (graph replay) after new numbers were written into the input arrays."""
    _check(lib().h2sp_refactor(h.ptr, _stream(stream)), "h2sp_refactor")


def _cols(t, n):
    """(nrhs, leading dimension) of a (nrhs, n) or (n,) tensor; rows must be contiguous."""
    if t.dim() == 1:
        return 1, n
    if int(t.shape[1]) != n or (int(t.shape[1]) > 1 and int(t.stride(1)) != 1):
        raise ValueError("expected a (nrhs, n) tensor with contiguous rows")
    nrhs = int(t.shape[0])
    return nrhs, (n if nrhs == 1 else int(t.stride(0)))


def h2sp_solve(h: Handle, b, x, mode: int = H2SP_DIRECT, tol: float = 1e-10, maxit: int = 50, restart: int = 30,
               stream=None) -> SolveInfo:
    n = int(h.inp.h.n)
    nrhs, ldb = _cols(b, n)
    _, ldx = _cols(x, n)
    o = SolveOpts(int(mode), float(tol), int(maxit), int(restart))
    info = SolveInfo()
    st = lib().h2sp_solve(h.ptr, ctypes.byref(o), nrhs, _vp(b.data_ptr()), ldb, _vp(x.data_ptr()), ldx,
                          ctypes.byref(info), _stream(stream))
    if st not in (H2SP_OK, H2SP_ENOCONV):
        _check(st, "h2sp_solve")
    info.status = st
    return info


def h2sp_apply(h: Handle, op: int, x, y, stream=None):
    n = int(h.inp.h.n)
    nrhs, ldx = _cols(x, n)
    _, ldy = _cols(y, n)
    _check(lib().h2sp_apply(h.ptr, int(op), nrhs, _vp(x.data_ptr()), ldx, _vp(y.data_ptr()), ldy, _stream(stream)),
           "h2sp_apply")


def h2sp_solve_host(an, inp: H2Input, b_ptr: int, ldb: int, x_ptr: int, ldx: int, nrhs: int, flags: int = 0,
                    prec: int = H2SP_FP32, mode: int = H2SP_GMRES, tol: float = 1e-10, maxit: int = 60,
                    restart: int = 20, stream=None) -> SolveInfo:
    """The whole path from host memory (inp built with device="host"; b and x
    host arrays given by address and leading dimension, column-major)."""
    o = Opts(int(flags))
    so = SolveOpts(int(mode), float(tol), int(maxit), int(restart))
    info = SolveInfo()
    d = inp.desc()
    st = lib().h2sp_solve_host(an.ptr if an is not None else None, ctypes.byref(d), ctypes.byref(o), int(prec),
                               ctypes.byref(so), int(nrhs), _vp(b_ptr), int(ldb), _vp(x_ptr), int(ldx),
                               ctypes.byref(info), _stream(stream))
    if st not in (H2SP_OK, H2SP_ENOCONV):
        _check(st, "h2sp_solve_host")
    info.status = st
    return info


H2SP_OPTION_WAIT_POLLS, H2SP_OPTION_TEST_STALE_EPOCH = 1, 2
H2SP_OPTION_CHOL_TILES_PER_CTA, H2SP_OPTION_CHOL_PANEL_SMS, H2SP_OPTION_CHOL_LOOKAHEAD = 3, 4, 5
H2SP_OPTION_CHOL_WIDE = 6


def h2sp_set_option(h: Handle, option: int, value: int):
    _check(lib().h2sp_set_option(h.ptr, int(option), int(value)), "h2sp_set_option")


def h2sp_measure_peak(kind: int, stream=None) -> float:
    """Measured FMA rate of the current device in TFLOP/s (kind 0: FP64, 1: FP32)."""
    v = ctypes.c_double(0.0)
    _check(lib().h2sp_measure_peak(int(kind), ctypes.byref(v), _stream(stream)), "h2sp_measure_peak")
    return float(v.value)


def h2sp_solve_captured(h: Handle, b, x, steps: int, tol: float = 1e-10, stream=None) -> SolveInfo:
    """Fixed-step refinement replayed from a CUDA graph (captured on the first call)."""
    n = int(h.inp.h.n)
    nrhs, ldb = _cols(b, n)
    _, ldx = _cols(x, n)
    info = SolveInfo()
    st = lib().h2sp_solve_captured(h.ptr, int(steps), float(tol), nrhs, _vp(b.data_ptr()), ldb, _vp(x.data_ptr()), ldx,
                                   ctypes.byref(info), _stream(stream))
    if st not in (H2SP_OK, H2SP_ENOCONV):
        _check(st, "h2sp_solve_captured")
    info.status = st
    return info


def h2sp_logdet(h: Handle, stream=None):
    """(log|det A|, sign of det S) per independent system: two arrays of length nsys."""
    nsys = h2sp_query(h)["nsys"]
    ld = np.zeros(nsys, np.float64)
    sg = np.zeros(nsys, np.int32)
    _check(lib().h2sp_logdet(h.ptr, _ptr(ld, ctypes.c_double), _ptr(sg, ctypes.c_int32), _stream(stream)),
           "h2sp_logdet")
    return ld, sg


def h2sp_query(h: Handle) -> dict:
    st = Stats()
    _check(lib().h2sp_query(h.ptr, ctypes.byref(st)), "h2sp_query")
    return {name: getattr(st, name) for name, _ in Stats._fields_}


def h2sp_export_S(h: Handle, values: bool = True, stream=None) -> dict:
    q = h2sp_query(h)
    nn, nnzb, nnz = q["nnodes"], q["nnzb"], q["nnz"]
    ns = np.zeros(nn, np.int64)
    bp = np.zeros(nn + 1, np.int64)
    bc = np.zeros(max(nnzb, 1), np.int32)
    vo = np.zeros(max(nnzb, 1), np.int64)
    vals = np.zeros(max(nnz, 1), np.float64) if values else None
    _check(lib().h2sp_export_S(h.ptr, _ptr(ns, ctypes.c_int64), _ptr(bp, ctypes.c_int64), _ptr(bc, ctypes.c_int32),
                               _ptr(vo, ctypes.c_int64), _ptr(vals, ctypes.c_double) if values else None,
                               _stream(stream) if values else _vp(None)), "h2sp_export_S")
    return dict(node_size=ns, brow_ptr=bp, bcol_idx=bc[:nnzb], val_off=vo[:nnzb],
                vals=vals[:nnz] if values else None)


def h2sp_export_Q(h: Handle, cluster: int, col: bool = False, stream=None):
    m = ctypes.c_int64(0)
    _check(lib().h2sp_export_Q(h.ptr, int(cluster), int(col), ctypes.byref(m), None, _vp(None)), "h2sp_export_Q")
    if m.value == 0:
        return np.zeros((0, 0))
    q = np.zeros(m.value * m.value, np.float64)
    _check(lib().h2sp_export_Q(h.ptr, int(cluster), int(col), ctypes.byref(m), _ptr(q, ctypes.c_double),
                               _stream(stream)), "h2sp_export_Q")
    return q.reshape(m.value, m.value).T


def h2sp_export_front(h: Handle, k: int, stream=None):
    """(F, s): the factored front of supernode k as an f x f FP64 array and its supernode size."""
    f, sz = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().h2sp_export_front(h.ptr, int(k), ctypes.byref(f), ctypes.byref(sz), None, _vp(None)),
           "h2sp_export_front")
    v = np.zeros(max(f.value * f.value, 1), np.float64)
    _check(lib().h2sp_export_front(h.ptr, int(k), ctypes.byref(f), ctypes.byref(sz), _ptr(v, ctypes.c_double),
                                   _stream(stream)), "h2sp_export_front")
    return v[:f.value * f.value].reshape(f.value, f.value).T, int(sz.value)


def h2sp_export_structure(h: Handle) -> dict:
    q = h2sp_query(h)
    nn, nsn = q["nnodes"], q["nsupernodes"]
    nb = ctypes.c_int64(0)
    _check(lib().h2sp_export_structure(h.ptr, None, None, None, None, None, None, None, ctypes.byref(nb)),
           "h2sp_export_structure")
    out = dict(node_level=np.zeros(nn, np.int32), node_cluster=np.zeros(nn, np.int32), closure=np.zeros(nn, np.int32),
               order=np.zeros(nn, np.int32), sn_ptr=np.zeros(nsn + 1, np.int32), bnd_ptr=np.zeros(nsn + 1, np.int32),
               bnd=np.zeros(max(nb.value, 1), np.int32))
    _check(lib().h2sp_export_structure(h.ptr, *[_ptr(out[k], ctypes.c_int32) for k in
                                                ("node_level", "node_cluster", "closure", "order", "sn_ptr",
                                                 "bnd_ptr", "bnd")], ctypes.byref(nb)), "h2sp_export_structure")
    out["bnd"] = out["bnd"][:nb.value]
    return out


def h2sp_export_schedule(h: Handle, ncl: int) -> dict:
    """The device level schedule of h's structure: lstop, per cluster m, kp,
    off, xoff, per S node node_off (nnodes + 1) and node_cluster."""
    nn = h2sp_query(h)["nnodes"]
    out = dict(m=np.zeros(ncl, np.int64), kp=np.zeros(ncl, np.int64), off=np.zeros(ncl, np.int64),
               xoff=np.zeros(ncl, np.int64), node_off=np.zeros(nn + 1, np.int64), node_cluster=np.zeros(nn, np.int32))
    ls = ctypes.c_int32(0)
    _check(lib().h2sp_export_schedule(h.ptr, ctypes.byref(ls), *[_ptr(out[k], ctypes.c_int64) for k in
                                                                 ("m", "kp", "off", "xoff", "node_off")],
                                      _ptr(out["node_cluster"], ctypes.c_int32)), "h2sp_export_schedule")
    out["lstop"] = int(ls.value)
    return out


def h2sp_export_near(h: Handle, level: int, nrows: int) -> tuple:
    """(ptr, col): Near_level of the device level schedule as CSR over the
    level's nrows clusters."""
    nnz = ctypes.c_int64(0)
    _check(lib().h2sp_export_near(h.ptr, int(level), None, None, ctypes.byref(nnz)), "h2sp_export_near")
    ptr = np.zeros(nrows + 1, np.int64)
    col = np.zeros(max(nnz.value, 1), np.int32)
    _check(lib().h2sp_export_near(h.ptr, int(level), _ptr(ptr, ctypes.c_int64), _ptr(col, ctypes.c_int32),
                                  ctypes.byref(nnz)), "h2sp_export_near")
    return ptr, col[:nnz.value]


def h2sp_factor_ilut(h: Handle, tau: float, stream=None):
    """Threshold incomplete LU of S (ILUt, drop tolerance tau)."""
    _check(lib().h2sp_factor_ilut(h.ptr, float(tau), _stream(stream)), "h2sp_factor_ilut")


def h2sp_export_ilut(h: Handle) -> dict:
    """The incomplete factors: perm, and L / U as CSR in elimination order."""
    n = int(h.inp.h.n)
    nl, nu = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().h2sp_export_ilut(h.ptr, None, None, None, None, None, None, None, ctypes.byref(nl),
                                  ctypes.byref(nu)), "h2sp_export_ilut")
    out = dict(perm=np.zeros(n, np.int32), l_ptr=np.zeros(n + 1, np.int64), l_col=np.zeros(max(nl.value, 1), np.int32),
               l_val=np.zeros(max(nl.value, 1)), u_ptr=np.zeros(n + 1, np.int64),
               u_col=np.zeros(max(nu.value, 1), np.int32), u_val=np.zeros(max(nu.value, 1)))
    _check(lib().h2sp_export_ilut(h.ptr, _ptr(out["perm"], ctypes.c_int32), _ptr(out["l_ptr"], ctypes.c_int64),
                                  _ptr(out["l_col"], ctypes.c_int32), _ptr(out["l_val"], ctypes.c_double),
                                  _ptr(out["u_ptr"], ctypes.c_int64), _ptr(out["u_col"], ctypes.c_int32),
                                  _ptr(out["u_val"], ctypes.c_double), ctypes.byref(nl), ctypes.byref(nu)),
           "h2sp_export_ilut")
    for k, m in (("l_col", nl.value), ("l_val", nl.value), ("u_col", nu.value), ("u_val", nu.value)):
        out[k] = out[k][:m]
    return out


def h2sp_profile(h: Handle, timing: int = -1, reset: bool = False) -> dict:
    """Per-kernel-class counters: {class: {launches, timed, ms, work}}."""
    kt = KernelTimes()
    _check(lib().h2sp_profile(h.ptr, int(timing), int(bool(reset)), ctypes.byref(kt)), "h2sp_profile")
    return {nm: dict(launches=int(kt.launches[i]), timed=int(kt.timed[i]), ms=float(kt.ms[i]), work=float(kt.work[i]))
            for i, nm in enumerate(KERNEL_CLASSES)}


def h2sp_destroy(h: Handle):
    h.close()
