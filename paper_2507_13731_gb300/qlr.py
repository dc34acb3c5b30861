"""ctypes binding of libqlr.so: argument marshalling only.

Every computation runs in the CUDA library; this module turns torch tensors into the
`qlr_qmat` descriptors of include/qlr.h and raises `QlrError` on a non-zero return code.
PyTorch is used for device memory and streams only.

Quaternion matrices are torch tensors of logical shape (4, rows, cols) -- planes real, i, j, k
-- or (3, rows, cols) for a pure quaternion matrix (planes i, j, k; real part zero).  A tensor
whose last dimension is contiguous is row-major (the data matrix A); one whose middle dimension
is contiguous (e.g. from `empty_thin`) is column-major (Omega, Q, U, V and the sketches).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqlr.so")

# constants mirrored from include/qlr.h
OK, EINVAL, ESHAPE, ENOTPD, ENOCONV, ETIMEOUT, ECUDA, ENOMEM, EUNSUPPORTED = range(9)
F64, F32, BF16 = 0, 1, 2
ROW_MAJOR, COL_MAJOR = 0, 1
COMPUTE_AUTO, COMPUTE_F64, COMPUTE_F32, COMPUTE_TF32, COMPUTE_TF32X3, COMPUTE_BF16, COMPUTE_TF32_MIXED, \
    COMPUTE_TF32_RN = range(8)
COMPUTE_MIXED = COMPUTE_TF32_MIXED
OP_N, OP_H = 0, 1
ALG1, ALG2, ALG3, ALG4 = 1, 2, 3, 4
SIDE_AUTO, SIDE_X, SIDE_XH = -1, 0, 1
ORTH_CHOLQR2, ORTH_SCHOLQR3 = 0, 1
FLAG_QR_EVERY_PASS = 1
FLAG_NO_GRAPH = 2
PEAK_TF32_MMA, PEAK_BF16_MMA, PEAK_FP32_FMA, PEAK_FP64_FMA, PEAK_TF32_MMA_N64, PEAK_BF16_MMA_N64 = range(6)

_DT = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}
KID_NAMES = ["sketch_tc", "sketch_simt", "gram", "chol", "tri_inv", "apply", "jacobi", "refine", "misc", "series",
             "complete", "sketch_x3", "sketch_rn"]


class QlrError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {lib().qlr_strerror(code).decode()} (code {code})")


class QMatC(ctypes.Structure):
    _fields_ = [("plane", ctypes.c_void_p * 4), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("layout", ctypes.c_int32), ("dtype", ctypes.c_int32)]


class OptsC(ctypes.Structure):
    _fields_ = [("compute", ctypes.c_int32), ("side", ctypes.c_int32), ("orth", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class BatchStatsC(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("graph", ctypes.c_int32), ("tile_order", ctypes.c_int32),
                ("sketch_launches", ctypes.c_int32), ("tune_ms", ctypes.c_float * 16),
                ("launches_per_run", ctypes.c_int64), ("stage_k", ctypes.c_int32),
                ("col_block_max", ctypes.c_int32), ("ring_stages", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None


def lib():
    """Load libqlr.so; fails loudly if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2507_13731_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        Q = ctypes.POINTER(QMatC)
        O = ctypes.POINTER(OptsC)
        sig = {
            "qlr_create": (I, [ctypes.POINTER(P), I, P]),
            "qlr_destroy": (I, [P]),
            "qlr_set_stream": (I, [P, P]),
            "qlr_reserve": (I, [P, S]),
            "qlr_workspace_size": (S, [I64, I64, I, I, I, I, I]),
            "qlr_sync": (I, [P]),
            "qlr_strerror": (ctypes.c_char_p, [I]),
            "qlr_qsketch": (I, [P, I, Q, Q, Q, I]),
            "qlr_qgram": (I, [P, Q, P]),
            "qlr_qchol": (I, [P, I, P, P]),
            "qlr_cholqr": (I, [P, Q, Q, P, I]),
            "qlr_qtsvd": (I, [P, I, P, I, P, P, P, I]),
            "qlr_qrangefinder": (I, [P, Q, I, I, I, Q, O, Q, Q, P, ctypes.POINTER(I)]),
            "qlr_qsvd_lowrank": (I, [P, Q, I, I, I, I, Q, O, Q, P, Q]),
            "qlr_qblock_krylov": (I, [P, Q, I, I, I, Q, O, Q, P, Q]),
            "qlr_qbasis": (I, [P, Q, I, I, I, I, Q, O, Q, Q, P, ctypes.POINTER(I)]),
            "qlr_qsvd_lowrank_batched": (I, [P, I, Q, ctypes.POINTER(I), ctypes.POINTER(I), I, Q, O, Q,
                                             ctypes.POINTER(P), Q]),
            "qlr_residual_norm": (I, [P, Q, Q, I, Q, I, ctypes.POINTER(D)]),
            "qlr_qcomplete_update": (I, [P, Q, P, I64, Q, P, Q, I, Q]),
            "qlr_qcomplete": (I, [P, Q, P, I64, I, I, I, I, I, Q, O, Q, Q, P, Q]),
            "qlr_selftest_wait_timeout": (I, [P]),
            "qlr_set_timing": (I, [P, I]),
            "qlr_reset_stats": (I, [P]),
            "qlr_stats": (I, [P, I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(D)]),
            "qlr_qsketch_noalloc": (I, [P, I, Q, Q, Q, I, P]),
            "qlr_peak_probe": (I, [I, I, I64, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_float)]),
            "qlr_splitmix64": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64]),
            "qlr_gaussian_qmat_host": (I, [ctypes.c_uint64, I64, I64, I, P]),
            "qlr_fill_omega": (I, [P, ctypes.c_uint64, I, Q]),
            "qlr_batch_create": (I, [P, I, Q, ctypes.POINTER(I), ctypes.POINTER(I), I, Q, O, Q,
                                     ctypes.POINTER(P), Q, ctypes.POINTER(P)]),
            "qlr_batch_run": (I, [P]),
            "qlr_batch_info": (I, [P, ctypes.POINTER(BatchStatsC)]),
            "qlr_batch_destroy": (I, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, where: str) -> None:
    if rc != OK:
        raise QlrError(rc, where)


# ------------------------------------------------------------------------------------------
def empty_thin(rows: int, cols: int, dtype=torch.float32, device="cuda") -> torch.Tensor:
    """Column-major quaternion matrix storage: logical shape (4, rows, cols), rows contiguous."""
    return torch.empty(4, cols, rows, dtype=dtype, device=device).transpose(1, 2)


def to_thin(x: torch.Tensor) -> torch.Tensor:
    """Copy a (4, rows, cols) tensor into column-major storage on the same device."""
    out = empty_thin(x.shape[1], x.shape[2], x.dtype, x.device)
    out.copy_(x)
    return out


def qmat(t: torch.Tensor, layout: Optional[int] = None) -> QMatC:
    """Describe a quaternion tensor (4 or 3 planes) as a qlr_qmat.  `layout` forces ROW_MAJOR or
    COL_MAJOR (needed for degenerate 1-row / 1-column tensors); by default it is read from the
    strides."""
    if t.dim() != 3 or t.shape[0] not in (3, 4):
        raise ValueError("quaternion tensors have shape (4, rows, cols) or (3, rows, cols)")
    if t.dtype not in _DT:
        raise ValueError(f"unsupported dtype {t.dtype}")
    rows, cols = t.shape[1], t.shape[2]
    rs, cs = t.stride(1), t.stride(2)
    row_ok = (cs == 1 or cols <= 1) and (rs >= cols or rows <= 1)
    col_ok = (rs == 1 or rows <= 1) and (cs >= rows or cols <= 1)
    if layout is None:
        layout = ROW_MAJOR if (row_ok and cs == 1 and not (rs == 1 and col_ok)) else (COL_MAJOR if col_ok else ROW_MAJOR)
    if layout == ROW_MAJOR and not row_ok or layout == COL_MAJOR and not col_ok:
        raise ValueError("each plane must be row- or column-major with a unit stride")
    q = QMatC()
    q.rows, q.cols, q.dtype, q.layout = rows, cols, _DT[t.dtype], layout
    q.ld = max(rs if layout == ROW_MAJOR else cs, cols if layout == ROW_MAJOR else rows, 1)
    if layout == ROW_MAJOR and rows <= 1:
        q.ld = max(cols, 1)
    if layout == COL_MAJOR and cols <= 1:
        q.ld = max(rows, 1)
    off = 4 - t.shape[0]
    es = t.element_size()
    for c in range(4):
        q.plane[c] = None if c < off else t.data_ptr() + (c - off) * t.stride(0) * es
    return q


def _A(t):
    return qmat(t, ROW_MAJOR)


def _T(t):
    return qmat(t, COL_MAJOR)


def _opts(compute: int = COMPUTE_AUTO, side: int = SIDE_AUTO, orth: int = ORTH_CHOLQR2,
          qr_every_pass: bool = False) -> OptsC:
    return OptsC(compute, side, orth, FLAG_QR_EVERY_PASS if qr_every_pass else 0)


class Context:
    """A qlr context bound to a device and (by default) torch's current stream on it."""

    def __init__(self, device: int = 0, stream: Optional[torch.cuda.Stream] = None):
        self.device = device
        s = stream if stream is not None else torch.cuda.current_stream(device)
        self._stream = s
        h = ctypes.c_void_p()
        _check(lib().qlr_create(ctypes.byref(h), device, ctypes.c_void_p(s.cuda_stream)), "qlr_create")
        self.h = h

    def close(self) -> None:
        if getattr(self, "h", None):
            lib().qlr_destroy(self.h)
            self.h = None

    __del__ = close

    def set_stream(self, stream: torch.cuda.Stream) -> None:
        self._stream = stream
        _check(lib().qlr_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)), "qlr_set_stream")

    def reserve(self, nbytes: int) -> None:
        _check(lib().qlr_reserve(self.h, nbytes), "qlr_reserve")

    def sync(self) -> int:
        """Wait for the stream; return the device error code (0 if none)."""
        return lib().qlr_sync(self.h)

    def set_timing(self, on: bool) -> None:
        _check(lib().qlr_set_timing(self.h, 1 if on else 0), "qlr_set_timing")

    def reset_stats(self) -> None:
        _check(lib().qlr_reset_stats(self.h), "qlr_reset_stats")

    def stats(self) -> dict:
        """{kernel class: (launches, total ms)} since the last reset."""
        out = {}
        for kid, name in enumerate(KID_NAMES):
            n, ms = ctypes.c_int64(0), ctypes.c_double(0.0)
            _check(lib().qlr_stats(self.h, kid, ctypes.byref(n), ctypes.byref(ms)), "qlr_stats")
            out[name] = (n.value, ms.value)
        return out


def workspace_size(m, n, k, p, passes, algo=ALG2, compute=COMPUTE_AUTO) -> int:
    return lib().qlr_workspace_size(m, n, k, p, passes, algo, compute)


def qsketch(ctx: Context, op: int, A: torch.Tensor, X: torch.Tensor, Y: torch.Tensor, compute: int = COMPUTE_AUTO):
    a, x, y = _A(A), _T(X), _T(Y)
    _check(lib().qlr_qsketch(ctx.h, op, ctypes.byref(a), ctypes.byref(x), ctypes.byref(y), compute), "qlr_qsketch")
    return Y


def qsketch_noalloc(op: int, A: torch.Tensor, X: torch.Tensor, Y: torch.Tensor, compute: int,
                    stream: Optional[torch.cuda.Stream] = None, err: Optional[torch.Tensor] = None):
    """qlr_qsketch_noalloc: the tensor-core sketch product without a context and without any
    device allocation (scratch comes from the library's fixed device array); see include/qlr.h.
    A, X, Y (and err) must be on one CUDA device; the call runs on that device's `stream`
    (default: its current stream)."""
    devs = {t.device for t in (A, X, Y) + ((err,) if err is not None else ())}
    if len(devs) != 1 or next(iter(devs)).type != "cuda":
        raise ValueError("A, X, Y and err must be on one CUDA device")
    a, x, y = _A(A), _T(X), _T(Y)
    with torch.cuda.device(A.device):
        s = stream if stream is not None else torch.cuda.current_stream(A.device)
        ep = ctypes.c_void_p(err.data_ptr()) if err is not None else ctypes.c_void_p()
        _check(lib().qlr_qsketch_noalloc(ctypes.c_void_p(s.cuda_stream), op, ctypes.byref(a), ctypes.byref(x),
                                         ctypes.byref(y), compute, ep), "qlr_qsketch_noalloc")
    return Y


def qgram(ctx: Context, Y: torch.Tensor, G: torch.Tensor):
    y = _T(Y)
    _check(lib().qlr_qgram(ctx.h, ctypes.byref(y), ctypes.c_void_p(G.data_ptr())), "qlr_qgram")
    return G


def qchol(ctx: Context, G: torch.Tensor, R: torch.Tensor):
    _check(lib().qlr_qchol(ctx.h, G.shape[-1], ctypes.c_void_p(G.data_ptr()), ctypes.c_void_p(R.data_ptr())),
           "qlr_qchol")
    return R


def cholqr(ctx: Context, Y: torch.Tensor, Q: torch.Tensor, R: Optional[torch.Tensor] = None,
           orth: int = ORTH_CHOLQR2):
    y, q = _T(Y), _T(Q)
    rp = ctypes.c_void_p(R.data_ptr()) if R is not None else ctypes.c_void_p()
    _check(lib().qlr_cholqr(ctx.h, ctypes.byref(y), ctypes.byref(q), rp, orth), "qlr_cholqr")
    return Q, R


def qtsvd(ctx: Context, R: torch.Tensor, k: int, L: torch.Tensor, S: torch.Tensor, Rt: torch.Tensor, prec: int = F64):
    l = R.shape[-1]
    _check(lib().qlr_qtsvd(ctx.h, l, ctypes.c_void_p(R.data_ptr()), k, ctypes.c_void_p(L.data_ptr()),
                           ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(Rt.data_ptr()), prec), "qlr_qtsvd")
    return L, S, Rt


def qrangefinder(ctx: Context, A, k, p, passes, omega, Q1, Q2, R, compute=COMPUTE_AUTO, side=SIDE_AUTO,
                 orth=ORTH_CHOLQR2, qr_every_pass=False) -> int:
    a, om, q1, q2 = _A(A), _T(omega), _T(Q1), _T(Q2)
    o = _opts(compute, side, orth, qr_every_pass)
    used = ctypes.c_int(-1)
    _check(lib().qlr_qrangefinder(ctx.h, ctypes.byref(a), k, p, passes, ctypes.byref(om), ctypes.byref(o),
                                  ctypes.byref(q1), ctypes.byref(q2), ctypes.c_void_p(R.data_ptr()),
                                  ctypes.byref(used)), "qlr_qrangefinder")
    return used.value


def qsvd_lowrank(ctx: Context, A, k, p, passes, omega, U, S, V, algo=ALG2, compute=COMPUTE_AUTO, side=SIDE_AUTO,
                 orth=ORTH_CHOLQR2, qr_every_pass=False):
    a, om, u, v = _A(A), _T(omega), _T(U), _T(V)
    o = _opts(compute, side, orth, qr_every_pass)
    _check(lib().qlr_qsvd_lowrank(ctx.h, ctypes.byref(a), k, p, passes, algo, ctypes.byref(om), ctypes.byref(o),
                                  ctypes.byref(u), ctypes.c_void_p(S.data_ptr()), ctypes.byref(v)),
           "qlr_qsvd_lowrank")
    return U, S, V


def qbasis(ctx: Context, A, k, p, passes, omega, Q1, Q2, R, algo=ALG2, compute=COMPUTE_AUTO, side=SIDE_AUTO,
           orth=ORTH_CHOLQR2, qr_every_pass=False) -> int:
    """qlr_qbasis: the final bases Q1, Q2 and R of qsvd_lowrank's schedule (Q1: rows_fwd x L,
    Q2: rows_bwd x L, R: FP64 (4, L, L) storage); returns the side used."""
    a, om, q1, q2 = _A(A), _T(omega), _T(Q1), _T(Q2)
    o = _opts(compute, side, orth, qr_every_pass)
    used = ctypes.c_int(-1)
    _check(lib().qlr_qbasis(ctx.h, ctypes.byref(a), k, p, passes, algo, ctypes.byref(om), ctypes.byref(o),
                            ctypes.byref(q1), ctypes.byref(q2), ctypes.c_void_p(R.data_ptr()), ctypes.byref(used)),
           "qlr_qbasis")
    return used.value


def stacked_width(algo: int, l: int, passes: int) -> int:
    """Width L of the bases qbasis returns: l for Algorithms 1 and 2; the stacked Krylov width of
    Algorithms 3 and 4 ((v/2) l for even v, ((v-1)/2) l for odd v)."""
    if algo in (ALG3, ALG4):
        return (passes // 2 if passes % 2 == 0 else (passes - 1) // 2) * l
    return l


def qblock_krylov(ctx: Context, A, k, b, passes, omega, U, S, V, compute=COMPUTE_AUTO, side=SIDE_AUTO,
                  qr_every_pass=False):
    a, om, u, v = _A(A), _T(omega), _T(U), _T(V)
    o = _opts(compute, side, ORTH_CHOLQR2, qr_every_pass)
    _check(lib().qlr_qblock_krylov(ctx.h, ctypes.byref(a), k, b, passes, ctypes.byref(om), ctypes.byref(o),
                                   ctypes.byref(u), ctypes.c_void_p(S.data_ptr()), ctypes.byref(v)),
           "qlr_qblock_krylov")
    return U, S, V


def selftest_wait_timeout(ctx: Context) -> None:
    """Launch the failure-detection self test: a bounded device wait that times out, after which
    ctx.sync() returns ETIMEOUT once."""
    _check(lib().qlr_selftest_wait_timeout(ctx.h), "qlr_selftest_wait_timeout")


def _mask(mask: torch.Tensor, rows: int, cols: int):
    """Device uint8 observation mask (rows x cols, row-major, unit column stride): pointer, row stride."""
    if mask.dtype != torch.uint8 or mask.dim() != 2 or tuple(mask.shape) != (rows, cols):
        raise ValueError("the mask is a (rows, cols) uint8 tensor")
    if cols > 1 and mask.stride(1) != 1:
        raise ValueError("the mask must be row-major with a unit column stride")
    return ctypes.c_void_p(mask.data_ptr()), max(mask.stride(0) if rows > 1 else cols, cols, 1)


def complete_update(ctx: Context, M, mask, C, U=None, S=None, V=None, k: int = 0):
    """C = mask .* M + (1 - mask) .* U[:, :k] diag(S) V[:, :k]^H (eq. Step2); k = 0 gives P_Omega(M)."""
    m, c = _A(M), _A(C)
    mp, ml = _mask(mask, C.shape[1], C.shape[2])
    u = ctypes.byref(_T(U)) if U is not None else None
    v = ctypes.byref(_T(V)) if V is not None else None
    sp = ctypes.c_void_p(S.data_ptr()) if S is not None else None
    _check(lib().qlr_qcomplete_update(ctx.h, ctypes.byref(m), mp, ml, u, sp, v, k, ctypes.byref(c)),
           "qlr_qcomplete_update")
    return C


def complete(ctx: Context, M, mask, k, p, passes, iters, omega, C, U, S, V, algo=ALG2, compute=COMPUTE_AUTO,
             side=SIDE_AUTO, orth=ORTH_CHOLQR2):
    """Matrix completion by alternating updates (eqs. Step1, Step2) from C = P_Omega(M)."""
    m, c, om, u, v = _A(M), _A(C), _T(omega), _T(U), _T(V)
    mp, ml = _mask(mask, C.shape[1], C.shape[2])
    o = _opts(compute, side, orth)
    _check(lib().qlr_qcomplete(ctx.h, ctypes.byref(m), mp, ml, k, p, passes, algo, iters, ctypes.byref(om),
                               ctypes.byref(o), ctypes.byref(c), ctypes.byref(u), ctypes.c_void_p(S.data_ptr()),
                               ctypes.byref(v)), "qlr_qcomplete")
    return C, U, S, V


def qsvd_lowrank_batched(ctx: Context, As: Sequence[torch.Tensor], ks: Sequence[int], ps: Sequence[int], passes: int,
                         omegas, Us, Ss, Vs, compute=COMPUTE_AUTO):
    n = len(As)
    arrA = (QMatC * n)(*[_A(t) for t in As])
    arrO = (QMatC * n)(*[_T(t) for t in omegas])
    arrU = (QMatC * n)(*[_T(t) for t in Us])
    arrV = (QMatC * n)(*[_T(t) for t in Vs])
    kk = (ctypes.c_int * n)(*ks)
    pp = (ctypes.c_int * n)(*ps)
    sp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in Ss])
    o = _opts(compute, SIDE_X)
    _check(lib().qlr_qsvd_lowrank_batched(ctx.h, n, arrA, kk, pp, passes, arrO, ctypes.byref(o), arrU, sp, arrV),
           "qlr_qsvd_lowrank_batched")
    return Us, Ss, Vs


class Batch:
    """A batch plan: Algorithm 2 over many problems, planned (and autotuned, graph-captured) once,
    run many times on the context's stream.  The buffers passed here are the ones every run uses."""

    def __init__(self, ctx: Context, As, ks, ps, passes: int, omegas, Us, Ss, Vs, compute=COMPUTE_AUTO,
                 graph: bool = True, qr_every_pass: bool = False):
        n = len(As)
        self._keep = (As, omegas, Us, Ss, Vs)
        arrA = (QMatC * n)(*[_A(t) for t in As])
        arrO = (QMatC * n)(*[_T(t) for t in omegas])
        arrU = (QMatC * n)(*[_T(t) for t in Us])
        arrV = (QMatC * n)(*[_T(t) for t in Vs])
        kk = (ctypes.c_int * n)(*ks)
        pp = (ctypes.c_int * n)(*ps)
        sp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in Ss])
        o = _opts(compute, SIDE_X, ORTH_CHOLQR2, qr_every_pass)
        if not graph:
            o.flags |= FLAG_NO_GRAPH
        self.ctx = ctx
        self.h = ctypes.c_void_p()
        _check(lib().qlr_batch_create(ctx.h, n, arrA, kk, pp, passes, arrO, ctypes.byref(o), arrU, sp, arrV,
                                      ctypes.byref(self.h)), "qlr_batch_create")

    def run(self) -> None:
        _check(lib().qlr_batch_run(self.h), "qlr_batch_run")

    def info(self) -> dict:
        st = BatchStatsC()
        _check(lib().qlr_batch_info(self.h, ctypes.byref(st)), "qlr_batch_info")
        return {"lanes": st.lanes, "graph": bool(st.graph), "tile_order": st.tile_order,
                "sketch_launches": st.sketch_launches, "tune_ms": list(st.tune_ms),
                "launches_per_run": st.launches_per_run, "stage_k": st.stage_k,
                "col_block_max": st.col_block_max, "ring_stages": st.ring_stages}

    def close(self) -> None:
        if self.h:
            lib().qlr_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gaussian_qmat_host(seed: int, rows: int, cols: int, real_only: bool = False):
    """qlr_gaussian_qmat_host: the seeded Gaussian quaternion matrix (Def. 2) as a (4, rows, cols)
    float64 CPU tensor (column-major planes, as the library fills them)."""
    out = torch.zeros(4, cols, rows, dtype=torch.float64)
    _check(lib().qlr_gaussian_qmat_host(seed & 0xFFFFFFFFFFFFFFFF, rows, cols, 1 if real_only else 0,
                                        ctypes.c_void_p(out.data_ptr())), "qlr_gaussian_qmat_host")
    return out.transpose(1, 2)


def fill_omega(ctx: Context, seed: int, omega: torch.Tensor, real_only: bool = False) -> torch.Tensor:
    """qlr_fill_omega: write the seeded Gaussian test matrix into the column-major device tensor omega."""
    om = _T(omega)
    _check(lib().qlr_fill_omega(ctx.h, seed & 0xFFFFFFFFFFFFFFFF, 1 if real_only else 0, ctypes.byref(om)),
           "qlr_fill_omega")
    return omega


def splitmix64(seed: int, counter: int) -> int:
    return int(lib().qlr_splitmix64(seed & 0xFFFFFFFFFFFFFFFF, counter))


def peak_probe(kind: int, device: int = 0, iters: int = 1000):
    """qlr_peak_probe: (flops executed, milliseconds) of one throughput probe kernel."""
    f, t = ctypes.c_double(0.0), ctypes.c_float(0.0)
    _check(lib().qlr_peak_probe(kind, device, iters, ctypes.byref(f), ctypes.byref(t)), "qlr_peak_probe")
    return f.value, t.value


def measure_peak(kind: int, device: int = 0, target_ms: float = 40.0, reps: int = 3) -> float:
    """Dense peak in TFLOP/s of one probe: calibrate the iteration count on a short run so one
    launch takes about target_ms, then the best of `reps` launches."""
    mma = kind in (PEAK_TF32_MMA, PEAK_BF16_MMA, PEAK_TF32_MMA_N64, PEAK_BF16_MMA_N64)
    cap = 400000 if mma else 1 << 40
    iters = 2000 if mma else 20000
    f, ms = peak_probe(kind, device, iters)
    iters = int(min(cap, max(1, iters * target_ms / max(ms, 1e-3))))
    best = 0.0
    for _ in range(reps):
        f, ms = peak_probe(kind, device, iters)
        best = max(best, f / (ms * 1e-3) / 1e12)
    return best


def empty_rowmajor(rows: int, cols: int, planes: int = 4, dtype=torch.bfloat16, device="cuda") -> torch.Tensor:
    """Row-major quaternion storage (planes, rows, cols) whose row pitch is a multiple of 16 bytes, the
    tensor-core sketch's requirement (the pitch is padded, the view has exactly `cols` columns)."""
    esz = torch.empty(0, dtype=dtype).element_size()
    per = 16 // esz
    ld = (cols + per - 1) // per * per
    return torch.empty(planes, rows, ld, dtype=dtype, device=device)[:, :, :cols]


def residual_norm(ctx: Context, A, Q, side, start, iters=30) -> float:
    a, q, s = _A(A), _T(Q), _T(start)
    out = ctypes.c_double(0.0)
    _check(lib().qlr_residual_norm(ctx.h, ctypes.byref(a), ctypes.byref(q), side, ctypes.byref(s), iters,
                                   ctypes.byref(out)), "qlr_residual_norm")
    return out.value
