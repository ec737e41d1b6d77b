"""Thin Python binding of libbiharm_ext.so (ctypes).  Argument marshalling only.

Every name mirrors an ``ext_*`` entry point of ``include/biharm_ext.h``.  Arrays may be torch
tensors (CUDA or CPU, float32, contiguous) or numpy float32 arrays (host); shapes are [ny][nx].
There is no fallback: if the library is missing or fails to load, ``load()`` raises.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbiharm_ext.so")

BC = {"symmetric": 0, "periodic": 1, "dirichlet": 2}
DIR = {"out": 0, "in": 1}
PREC = {"fp32": 1, "mixed_bf16": 2, "mixed_fp16": 3}

EXT_OK, EXT_PENDING = 0, 1
EXT_EINVAL, EXT_ENOKNOWN, EXT_ENOMEM, EXT_EADMIT = -1, -2, -3, -4
EXT_ENOTCONV, EXT_EBREAKDOWN, EXT_ETIMEOUT, EXT_ECUDA = -5, -6, -7, -8
EXT_ENOTSUP, EXT_ENOTFOUND = -9, -10

EXPORTED = ["ext_options_default", "ext_create", "ext_solve", "ext_solve_batch", "ext_solve_multi",
            "ext_submit",
            "ext_poll", "ext_drain", "ext_destroy", "ext_strerror", "ext_last_error",
            "ext_apply_biharmonic", "ext_rhs", "ext_apply_preconditioner", "ext_solve_f64",
            "ext_profile_read", "ext_launch_count", "ext_apply_biharmonic_noalloc",
            "ext_noalloc_last_error", "ext_axis_basis", "ext_axis_slices", "ext_stencil_tile",
            "ext_axis_class_basis", "ext_solve3d", "ext_apply_biharmonic3d",
            "ext_apply_preconditioner3d"]
KERNEL_KINDS = ["setup", "stencil", "update", "true_residual", "prec_stage0", "prec_stage1",
                "prec_stage2", "prec_stage3", "output", "split", "prec_finish",
                "pq_finish", "low_fwd", "low_mid", "low_inv", "unfold", "fold"]


class ExtProblem(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("hx", C.c_double), ("hy", C.c_double),
                ("bc_x", C.c_int32), ("bc_y", C.c_int32), ("dir", C.c_int32)]


class ExtProblem3(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("hx", C.c_double),
                ("hy", C.c_double), ("hz", C.c_double), ("bc_x", C.c_int32), ("bc_y", C.c_int32),
                ("bc_z", C.c_int32), ("dir", C.c_int32)]


class ExtOptions(C.Structure):
    _fields_ = [("prec", C.c_int32), ("rtol", C.c_double), ("maxit", C.c_int32),
                ("true_res_every", C.c_int32), ("replace_factor", C.c_double),
                ("iters_per_launch", C.c_int32),
                ("hbm_budget", C.c_size_t), ("flexible", C.c_int32), ("max_slots", C.c_int32),
                ("profile", C.c_int32), ("autotune", C.c_int32), ("tile_y", C.c_int32),
                ("low_modes", C.c_int32), ("wait_cycles", C.c_int64), ("fold", C.c_int32)]


class ExtResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("relres_true", C.c_double),
                ("relres_rec", C.c_double), ("n_unknown", C.c_int32), ("n_known", C.c_int32),
                ("ms_queue", C.c_double), ("ms_solve", C.c_double), ("err_est", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ExtError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code}) {last_error()}")


_lib = None


def load():
    """Load the library (building it first if it is absent).  Raises if that fails."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        from . import build_ext
        build_ext.build()
    lib = C.CDLL(LIB_PATH)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    lib.ext_options_default.argtypes = [C.POINTER(ExtOptions)]
    lib.ext_options_default.restype = None
    lib.ext_create.argtypes = [C.POINTER(ExtOptions), P, C.POINTER(P)]
    lib.ext_create.restype = I
    lib.ext_solve.argtypes = [P, C.POINTER(ExtProblem), P, P, P, C.POINTER(ExtResult)]
    lib.ext_solve.restype = I
    lib.ext_solve_f64.argtypes = [P, C.POINTER(ExtProblem), P, P, P, C.POINTER(ExtResult)]
    lib.ext_solve_f64.restype = I
    lib.ext_solve_batch.argtypes = [P, I, C.POINTER(ExtProblem), C.POINTER(P), C.POINTER(P),
                                    C.POINTER(P), C.POINTER(ExtResult)]
    lib.ext_solve_batch.restype = I
    lib.ext_solve_multi.argtypes = [P, C.POINTER(ExtProblem), P, I, C.POINTER(P), C.POINTER(P),
                                    C.POINTER(ExtResult)]
    lib.ext_solve_multi.restype = I
    lib.ext_submit.argtypes = [P, C.POINTER(ExtProblem), P, P, P, C.POINTER(C.c_uint64)]
    lib.ext_submit.restype = I
    lib.ext_poll.argtypes = [P, C.c_uint64, C.POINTER(ExtResult)]
    lib.ext_poll.restype = I
    lib.ext_drain.argtypes = [P]
    lib.ext_drain.restype = I
    lib.ext_destroy.argtypes = [P]
    lib.ext_destroy.restype = None
    lib.ext_strerror.argtypes = [I]
    lib.ext_strerror.restype = C.c_char_p
    lib.ext_last_error.argtypes = []
    lib.ext_last_error.restype = C.c_char_p
    lib.ext_apply_biharmonic.argtypes = [P, C.POINTER(ExtProblem), P, P, P, C.POINTER(D)]
    lib.ext_apply_biharmonic.restype = I
    lib.ext_rhs.argtypes = [P, C.POINTER(ExtProblem), P, P, P]
    lib.ext_rhs.restype = I
    lib.ext_apply_preconditioner.argtypes = [P, C.POINTER(ExtProblem), P, P, P, C.POINTER(D)]
    lib.ext_apply_preconditioner.restype = I
    lib.ext_solve3d.argtypes = [P, C.POINTER(ExtProblem3), P, P, P, C.POINTER(ExtResult)]
    lib.ext_solve3d.restype = I
    lib.ext_apply_biharmonic3d.argtypes = [P, C.POINTER(ExtProblem3), P, P, P]
    lib.ext_apply_biharmonic3d.restype = I
    lib.ext_apply_preconditioner3d.argtypes = [P, C.POINTER(ExtProblem3), P, P, P, C.POINTER(D)]
    lib.ext_apply_preconditioner3d.restype = I
    lib.ext_profile_read.argtypes = [P, I, C.POINTER(D), C.POINTER(C.c_int64), I]
    lib.ext_profile_read.restype = I
    lib.ext_stencil_tile.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.ext_stencil_tile.restype = I
    lib.ext_launch_count.argtypes = [P]
    lib.ext_launch_count.restype = C.c_int64
    lib.ext_apply_biharmonic_noalloc.argtypes = [C.POINTER(ExtProblem), P, P, P, C.POINTER(D), P]
    lib.ext_apply_biharmonic_noalloc.restype = I
    lib.ext_noalloc_last_error.argtypes = []
    lib.ext_noalloc_last_error.restype = C.c_char_p
    lib.ext_axis_basis.argtypes = [C.c_int32, I, P, P]
    lib.ext_axis_basis.restype = I
    lib.ext_axis_class_basis.argtypes = [C.c_int32, I, C.c_int32, P, P]
    lib.ext_axis_class_basis.restype = I
    lib.ext_axis_slices.argtypes = [C.c_int32, I, C.c_int32, P, P]
    lib.ext_axis_slices.restype = I
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().ext_strerror(int(code)).decode()


def last_error() -> str:
    return load().ext_last_error().decode()


# ------------------------------------------------------------------------------------------------
# marshalling helpers
# ------------------------------------------------------------------------------------------------
def _ptr(a):
    """Raw data pointer of a contiguous float32/float64 torch tensor or numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("array must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def problem(nx, ny, bc_x="symmetric", bc_y=None, direction="out", hx=1.0, hy=None):
    bc_y = bc_x if bc_y is None else bc_y
    hy = hx if hy is None else hy
    return ExtProblem(int(nx), int(ny), float(hx), float(hy), BC[bc_x] if isinstance(bc_x, str)
                      else int(bc_x), BC[bc_y] if isinstance(bc_y, str) else int(bc_y),
                      DIR[direction] if isinstance(direction, str) else int(direction))


def problem3(nx, ny, nz, bc_x="periodic", bc_y=None, bc_z=None, direction="out", hx=1.0, hy=None,
             hz=None):
    """ExtProblem3 of an nz x ny x nx box (bc_y, bc_z default to bc_x; hy, hz to hx)."""
    bc_y = bc_x if bc_y is None else bc_y
    bc_z = bc_x if bc_z is None else bc_z
    hy = hx if hy is None else hy
    hz = hx if hz is None else hz
    code = lambda b: BC[b] if isinstance(b, str) else int(b)
    return ExtProblem3(int(nx), int(ny), int(nz), float(hx), float(hy), float(hz), code(bc_x),
                       code(bc_y), code(bc_z), DIR[direction] if isinstance(direction, str)
                       else int(direction))


def problem_of(p):
    """ExtProblem from a synth.Problem-like object."""
    return problem(p.nx, p.ny, p.bc_x, p.bc_y, p.direction, p.hx, p.hy)


def options(prec="fp32", rtol=1e-8, maxit=0, true_res_every=200, iters_per_launch=10,
            hbm_budget=0, flexible=0, max_slots=256, replace_factor=1e-2, profile=0,
            wait_cycles=0, autotune=1, tile_y=32, low_modes=None, fold=None):
    """ext_options with the library's defaults for every field not given (low_modes and fold:
    None keeps the library's default)."""
    o = ExtOptions()
    load().ext_options_default(C.byref(o))
    o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    o.rtol, o.maxit, o.true_res_every = float(rtol), int(maxit), int(true_res_every)
    o.replace_factor = float(replace_factor)
    o.iters_per_launch, o.hbm_budget = int(iters_per_launch), int(hbm_budget)
    o.flexible, o.max_slots, o.profile = int(flexible), int(max_slots), int(profile)
    o.wait_cycles = int(wait_cycles)
    o.autotune, o.tile_y = int(autotune), int(tile_y)
    if low_modes is not None:
        o.low_modes = int(low_modes)
    if fold is not None:
        o.fold = int(fold)
    return o


def _check(rc, what, ok=(EXT_OK,)):
    if rc not in ok:
        raise ExtError(rc, what)
    return rc


# ------------------------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ------------------------------------------------------------------------------------------------
def ext_create(opts=None, stream=None):
    """Returns an opaque context handle (int).  ``stream``: a torch.cuda.Stream, raw handle or None."""
    lib = load()
    h = C.c_void_p()
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    o = opts if opts is not None else options()
    _check(lib.ext_create(C.byref(o), s, C.byref(h)), "ext_create")
    return h.value


def ext_destroy(ctx):
    load().ext_destroy(ctx)


def ext_solve(ctx, prob, phi, f, out, check=True):
    """Solve one extension; returns the result as a dict (status may be a non-OK code if
    check=False)."""
    res = ExtResult()
    rc = load().ext_solve(ctx, C.byref(prob), _ptr(phi), _ptr(f), _ptr(out), C.byref(res))
    if check:
        _check(rc, "ext_solve")
    d = res.as_dict()
    d["rc"] = rc
    return d


def ext_solve_f64(ctx, prob, phi, f, out64, check=True):
    """As ext_solve with a float64 device output (f at known nodes, the FP64 iterate elsewhere)."""
    res = ExtResult()
    rc = load().ext_solve_f64(ctx, C.byref(prob), _ptr(phi), _ptr(f), _ptr(out64), C.byref(res))
    if check:
        _check(rc, "ext_solve_f64")
    d = res.as_dict()
    d["rc"] = rc
    return d


def ext_solve_batch(ctx, probs, phis, fs, outs, check=True):
    n = len(probs)
    PA = C.c_void_p * n
    parr = (ExtProblem * n)(*probs)
    res = (ExtResult * n)()
    rc = load().ext_solve_batch(ctx, n, parr, PA(*[_ptr(a) for a in phis]),
                                PA(*[_ptr(a) for a in fs]), PA(*[_ptr(a) for a in outs]), res)
    if check:
        _check(rc, "ext_solve_batch")
    return rc, [r.as_dict() for r in res]


def ext_solve_multi(ctx, prob, phi, fs, outs, check=True):
    """Several fields sharing one phi; returns (rc, [result dicts])."""
    n = len(fs)
    PA = C.c_void_p * n
    res = (ExtResult * n)()
    rc = load().ext_solve_multi(ctx, C.byref(prob), _ptr(phi), n, PA(*[_ptr(a) for a in fs]),
                                PA(*[_ptr(a) for a in outs]), res)
    if check:
        _check(rc, "ext_solve_multi")
    return rc, [r.as_dict() for r in res]


def ext_submit(ctx, prob, phi, f, out):
    t = C.c_uint64()
    _check(load().ext_submit(ctx, C.byref(prob), _ptr(phi), _ptr(f), _ptr(out), C.byref(t)),
           "ext_submit")
    return t.value


def ext_poll(ctx, ticket):
    res = ExtResult()
    rc = load().ext_poll(ctx, C.c_uint64(ticket), C.byref(res))
    d = res.as_dict()
    d["rc"] = rc
    return d


def ext_drain(ctx):
    return _check(load().ext_drain(ctx), "ext_drain")


def ext_apply_biharmonic(ctx, prob, phi, p, q):
    s = C.c_double()
    _check(load().ext_apply_biharmonic(ctx, C.byref(prob), _ptr(phi), _ptr(p), _ptr(q),
                                       C.byref(s)), "ext_apply_biharmonic")
    return s.value


def ext_rhs(ctx, prob, phi, f, b):
    _check(load().ext_rhs(ctx, C.byref(prob), _ptr(phi), _ptr(f), _ptr(b)), "ext_rhs")


def ext_apply_preconditioner(ctx, prob, phi, r, z):
    s = C.c_double()
    _check(load().ext_apply_preconditioner(ctx, C.byref(prob), _ptr(phi), _ptr(r), _ptr(z),
                                           C.byref(s)), "ext_apply_preconditioner")
    return s.value


def ext_solve3d(ctx, prob3, phi, f, out, check=True):
    """Solve one three-dimensional extension (device arrays [nz][ny][nx]); returns the result as
    a dict (status may be a non-OK code if check=False)."""
    res = ExtResult()
    rc = load().ext_solve3d(ctx, C.byref(prob3), _ptr(phi), _ptr(f), _ptr(out), C.byref(res))
    if check:
        _check(rc, "ext_solve3d")
    d = res.as_dict()
    d["rc"] = rc
    return d


def ext_apply_biharmonic3d(ctx, prob3, phi, p, q):
    _check(load().ext_apply_biharmonic3d(ctx, C.byref(prob3), _ptr(phi), _ptr(p), _ptr(q)),
           "ext_apply_biharmonic3d")


def ext_apply_preconditioner3d(ctx, prob3, phi, r, z):
    s = C.c_double()
    _check(load().ext_apply_preconditioner3d(ctx, C.byref(prob3), _ptr(phi), _ptr(r), _ptr(z),
                                             C.byref(s)), "ext_apply_preconditioner3d")
    return s.value


def _stream_of(stream, *arrays):
    """Raw stream handle: the given torch stream or handle; by default torch's current stream on
    the arrays' device (so the call is ordered after work the caller queued there), else NULL."""
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    for a in arrays:
        if getattr(a, "is_cuda", False):
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def ext_apply_biharmonic_noalloc(prob, phi, p, q, stream=None, check=True):
    """q = M L^2 p without any device allocation (fixed per-device scratch; see the header).
    Returns (rc, sum p.q).  Runs on ``stream`` (default: torch's current stream)."""
    s = C.c_double()
    st = _stream_of(stream, phi, p, q)
    rc = load().ext_apply_biharmonic_noalloc(C.byref(prob), _ptr(phi), _ptr(p), _ptr(q), C.byref(s), st)
    if check and rc != EXT_OK:
        raise ExtError(rc, "ext_apply_biharmonic_noalloc: " + load().ext_noalloc_last_error().decode())
    return rc, s.value


def ext_axis_basis(n, bc):
    """(Q, lam) of one axis's transform basis, computed by the library on the host (no GPU):
    Q[i, k] is the k-th orthonormal eigenvector of the axis's negative second difference at node i,
    lam[k] its eigenvalue (h = 1)."""
    Q = np.empty((int(n), int(n)), np.float64)
    lam = np.empty(int(n), np.float64)
    _check(load().ext_axis_basis(int(n), BC[bc] if isinstance(bc, str) else int(bc), _ptr(Q),
                                 _ptr(lam)), "ext_axis_basis")
    return Q, lam


def ext_axis_class_basis(n, bc, cls):
    """(Q, lam) of one mirror class (0 even, 1 odd) of an axis's basis, computed by the library on
    the host (no GPU): Q[i, j] (i, j < ceil(n/2)) is the class's j-th eigenvector at node i."""
    h = (int(n) + 1) // 2
    Q = np.empty((h, h), np.float64)
    lam = np.empty(h, np.float64)
    _check(load().ext_axis_class_basis(int(n), BC[bc] if isinstance(bc, str) else int(bc), int(cls),
                                       _ptr(Q), _ptr(lam)), "ext_axis_class_basis")
    return Q, lam


def ext_axis_slices(n, bc, type_="bf16"):
    """(codes, exps) of one axis's basis in tensor-core operand form, computed by the library on
    the host (no GPU): codes [2, 4, np, np] uint16 (Q then Q^T; four slices; FP16 or BF16 bit
    patterns of integers), exps [2, np, np // 128] int8 block exponents; np = n rounded up to 128."""
    np_ = (int(n) + 127) // 128 * 128
    codes = np.empty((2, 4, np_, np_), np.uint16)
    exps = np.empty((2, np_, np_ // 128), np.int8)
    t = {"fp16": 0, "bf16": 1}[type_] if isinstance(type_, str) else int(type_)
    _check(load().ext_axis_slices(int(n), BC[bc] if isinstance(bc, str) else int(bc), t,
                                  codes.ctypes.data, exps.ctypes.data), "ext_axis_slices")
    return codes, exps


def ext_profile_read(ctx, reset=True):
    """{kind: (total_ms, launches)} for a context created with profile=1."""
    n = len(KERNEL_KINDS)
    ms = (C.c_double * n)()
    cnt = (C.c_int64 * n)()
    _check(load().ext_profile_read(ctx, n, ms, cnt, int(reset)), "ext_profile_read")
    return {KERNEL_KINDS[i]: (ms[i], cnt[i]) for i in range(n)}


def ext_stencil_tile(ctx):
    """(tile_x, tile_y) of the stencil in the context's last solve."""
    tx, ty = C.c_int32(), C.c_int32()
    _check(load().ext_stencil_tile(ctx, C.byref(tx), C.byref(ty)), "ext_stencil_tile")
    return tx.value, ty.value


def ext_launch_count(ctx):
    return int(load().ext_launch_count(ctx))


@dataclass
class Extender:
    """Convenience wrapper owning one context."""
    prec: str = "fp32"
    rtol: float = 1e-8
    maxit: int = 0

    def __post_init__(self):
        self.ctx = ext_create(options(self.prec, self.rtol, self.maxit))

    def solve(self, prob, phi, f, out):
        return ext_solve(self.ctx, prob, phi, f, out)

    def close(self):
        if self.ctx:
            ext_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
