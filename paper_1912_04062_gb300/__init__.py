"""Python binding of libskeweig.so, the GB300 skew-symmetric eigensolver.

Argument marshalling only: every step of the solve runs in the CUDA library
(see ``include/skeweig.h`` for the contract of each entry point).  PyTorch
supplies device memory and the current stream.  Matrices are column-major
(Fortran-strided) float64 CUDA tensors; :func:`fortran` converts a tensor.

If the shared library is missing the import still works but every call raises
``RuntimeError`` -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libskeweig.so")

SKEW_OK = 0
SKEW_INFO_INVIT_BASE = 1000
SKEW_ERR_CUDA = 2001
SKEW_ERR_NOMEM = 2002
SKEW_ERR_DEVICE_TIMEOUT = 2003
SKEW_ERR_UNSUPPORTED = 2004
SKEW_ERR_NONFINITE = 2005
SKEW_ERR_WORKSPACE = 2006
SKEW_ERR_LAUNCH = 2007
SKEW_ERR_NOT_DEFINITE = 2008

SKEW_MODE_FP64 = 0
SKEW_MODE_MIXED_BF16X3 = 1
SKEW_MODE_MIXED_INT8 = 2
SKEW_MODE_MIXED_BF16X6 = 3
SKEW_MODE_MIXED_REFINED = 4

SKEW_FAULT_NOMEM = 1
SKEW_FAULT_INVIT_NOCONV = 2
SKEW_FAULT_TINY_WAIT = 4
SKEW_FAULT_NO_REFINE = 8
SKEW_QTRD_AUTO = 0
SKEW_QTRD_FP32 = 1
SKEW_QTRD_FP64 = 2
SKEW_QTRD_TC = 3
SKEW_QTRD_DF = 4
SKEW_TRIDIAG_AUTO = 0
SKEW_TRIDIAG_FULL = 1

# every entry point the header declares: name -> (restype, argtypes)
_i, _d, _p, _sz = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
SIGNATURES = {
    "skew_opts_default": (None, [_p]),
    "skew_eig_strerror": (ctypes.c_char_p, [_i]),
    "skew_last_cuda_error": (ctypes.c_char_p, []),
    "skew_eig": (_i, [_i, _p, _i, _i, _p, _p, _p, _p]),
    "skew_eig_workspace_size": (_sz, [_i, _i, _p]),
    "skew_eig_workspace_size_ex": (_sz, [_i, _i, _p, _i]),
    "skew_eig_ex": (_i, [_i, _p, _i, _i, _p, _p, _p, _i, _p, _p, _sz, _p, _p]),
    "skew_eig_host": (_i, [_i, _p, _i, _i, _p, _p, _p, _p, _p]),
    "skew_eig_batched_workspace_size": (_sz, [_i, _p, _p, _p]),
    "skew_eig_batched": (_i, [_i, _p, _p, _p, _p, _p, _p, _p, _p, _p]),
    "skew_eig_batched_ex": (_i, [_i, _p, _p, _p, _p, _p, _p, _p, _p, _p, _sz, _p, _p]),
    "skew_eig_profile": (_i, [_i, _p, _i, _i, _p, _p, _p, _i, _p, _p, _sz, _p, _p]),
    "skew_metrics_ws": (_sz, [_i, _i, _i]),
    "skew_eig_metrics": (_i, [_i, _p, _i, _i, _p, _p, _p, _i, _p, _i, _p, _p, _sz, _p]),
    "skew_launch_count": (ctypes.c_longlong, []),
    "skew_refine_stats": (_i, [_p, _p, _i]),
    "skew_refine_ws": (_sz, [_i]),
    "skew_refine": (_i, [_i, _p, _i, _p, _p, _p, _i, _i, _p, _sz, _p, _p]),
    "skew_refine_trace": (_i, [_p, _p, _i]),
    "skew_refine_slices": (_i, [_p, _p, _i]),
    "skew_kernel_timing": (_i, [_i]),
    "skew_kernel_timing_read": (_i, [_i, _p, _p, _p]),
    "skew_kernel_timing_dropped": (ctypes.c_longlong, []),
    "skew_release_memory": (None, []),
    "skew_kernel_timeline": (_i, [_i, _p, _p, _p]),
    "skew_gemm_bf16x3_ws": (_sz, [_i, _i, _i]),
    "skew_gemm_f64acc_ws": (_sz, [_i, _i, _i]),
    "skew_gemm_f64acc": (_i, [_i, _i, _i, _d, _p, ctypes.c_longlong, ctypes.c_longlong, _p, ctypes.c_longlong,
                              ctypes.c_longlong, _d, _p, _i, _p, _sz, _p, _p]),
    "skew_gemm_f64acc_ex": (_i, [_i, _i, _i, _d, _p, ctypes.c_longlong, ctypes.c_longlong, _p, ctypes.c_longlong,
                                 ctypes.c_longlong, _d, _p, _i, _i, _i, _p, _sz, _p, _p]),
    "skew_gemm_bf16x3": (_i, [_i, _i, _i, _d, _p, ctypes.c_longlong, ctypes.c_longlong, _p, ctypes.c_longlong,
                              ctypes.c_longlong, _d, _p, _i, _i, _i, _p, _sz, _p, _p]),
    "skew_band_reduce_ws": (_sz, [_i, _i]),
    "skew_band_reduce": (_i, [_i, _p, _i, _i, _p, _p, _sz, _p, _p]),
    "skew_band_pack": (_i, [_i, _i, _p, _i, _p, _i, _p]),
    "skew_chase_steps": (_i, [_i, _i]),
    "skew_chase_ws": (_sz, [_i, _i]),
    "skew_band_to_tridiag": (_i, [_i, _i, _p, _i, _p, _p, _p, _p, _sz, _p, _p]),
    "skew_tridiag_ws": (_sz, [_i, _i]),
    "skew_tridiag_eig": (_i, [_i, _p, _i, _p, _p, _i, _p, _sz, _p, _p]),
    "skew_tridiag_eig_noalloc": (_i, [_i, _p, _i, _p, _p, _i, _p, _p]),
    "skew_dmap": (_i, [_i, _i, _p, _i, _p, _p, _i, _p]),
    "skew_apply_qtrd": (_i, [_i, _i, _p, _p, _p, _i, _i, _p]),
    "skew_batched_set_config": (_i, [_p]),
    "skew_batched_get_config": (None, [_p]),
    "skew_batched_plan_create": (_i, [_i, _p, _p, _p, _p, _p, _p, _p, _p, _p, _sz, _p, _p, _p]),
    "skew_batched_plan_exec": (_i, [_p, _p]),
    "skew_batched_plan_tune": (_i, [_p, _p, _p, _p, _p, _i, _p]),
    "skew_batched_plan_get_config": (None, [_p, _p]),
    "skew_batched_plan_destroy": (None, [_p]),
    "skew_bse_workspace_size": (_sz, [_i, _i, _p]),
    "skew_bse_solve": (_i, [_i, _p, _p, _i, _p, _p, _i, _i, _p, _p, _p, _i, _p, _p, _sz, _p, _p]),
    "skew_apply_qtrd_f32_ws": (_sz, [_i, _i]),
    "skew_apply_qtrd_f32": (_i, [_i, _i, _p, _p, _p, _i, _i, _i, _p, _sz, _p, _p]),
    "skew_apply_qtrd_df": (_i, [_i, _i, _p, _p, _p, _i, _i, _p, _p]),
    "skew_qband_ws": (_sz, [_i, _i, _i]),
    "skew_apply_qband": (_i, [_i, _i, _p, _i, _p, _p, _i, _i, _p, _sz, _p]),
}


class skew_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("band", ctypes.c_int), ("check_finite", ctypes.c_int),
                ("fault", ctypes.c_int), ("refine_iters", ctypes.c_int), ("refine_rho", ctypes.c_int),
                ("qtrd", ctypes.c_int), ("tridiag", ctypes.c_int)]


class skew_batched_config(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int), ("smem_max_n", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


_lib = None


def lib():
    """Load libskeweig.so (raises RuntimeError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1912_04062_gb300/build.py "
                               "(or __graft_entry__.build()) first; there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class SkewError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        msg = lib().skew_eig_strerror(code).decode()
        if code == SKEW_ERR_CUDA:
            msg += " [" + lib().skew_last_cuda_error().decode() + "]"
        super().__init__(f"{where}: {msg} (code {code})")


def _check(code: int, where: str):
    if code != 0:
        raise SkewError(code, where)


def _torch():
    import torch
    return torch


def fortran(t):
    """Column-major (Fortran-strided) copy of a 2-D tensor, unless it already is."""
    if t.dim() == 2 and t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t
    return t.t().contiguous().t()


def fortran_empty(rows: int, cols: int, device="cuda"):
    torch = _torch()
    return torch.empty((cols, rows), dtype=torch.float64, device=device).t()


def _ptr(t):
    """Address of a CUDA tensor (None -> NULL) for an argument the C ABI takes
    as a DEVICE pointer.  A host tensor is refused: its address handed to a
    kernel would be dereferenced on the GPU."""
    if t is None:
        return ctypes.c_void_p(0)
    if not t.is_cuda:
        raise TypeError("expected a CUDA tensor for a device-pointer argument")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(t):
    """Address of a host tensor (None -> NULL) for the host-buffer entry point
    skew_eig_host."""
    if t is None:
        return ctypes.c_void_p(0)
    if t.is_cuda:
        raise TypeError("expected a host tensor for a host-pointer argument")
    return ctypes.c_void_p(t.data_ptr())


def _out(t, dtype, numel, what):
    """Device address of an output buffer of the given dtype holding at least
    `numel` elements (None -> NULL)."""
    if t is not None and (t.dtype != dtype or t.numel() < numel):
        raise TypeError(f"{what}: expected {dtype} with at least {numel} elements, got {t.dtype} {tuple(t.shape)}")
    return _ptr(t)


def _zbuf(Z, n, nev, what):
    """Device address of an eigenvector block: float64, n rows, at least nev
    columns, column-major (None -> NULL)."""
    torch = _torch()
    if Z is not None and (Z.dtype != torch.float64 or Z.dim() != 2 or Z.shape[0] != n or Z.shape[1] < nev
                          or (n > 1 and Z.stride(0) != 1)):
        raise TypeError(f"{what}: expected a column-major float64 {n} x {nev} tensor, got {Z.dtype} "
                        f"{tuple(Z.shape)} strides {tuple(Z.stride())}")
    return _ptr(Z)


def _ld(t):
    # one column: torch may keep any stride for the size-1 dimension, and the
    # leading dimension is then only required to cover the rows
    if t.dim() == 2 and t.shape[1] > 1:
        return max(1, t.stride(1))
    return max(1, t.shape[0])


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _as_device_f64(A):
    torch = _torch()
    if not (A.is_cuda and A.dtype == torch.float64):
        raise TypeError("expected a float64 CUDA tensor")
    return fortran(A)


@dataclass
class Options:
    mode: int = SKEW_MODE_FP64
    band: int = 64
    check_finite: int = 0
    fault: int = 0
    refine_iters: int = 0
    refine_rho: int = 0
    qtrd: int = 0
    tridiag: int = 0

    def c(self):
        o = skew_opts()
        lib().skew_opts_default(ctypes.byref(o))
        o.mode, o.band, o.check_finite, o.fault = self.mode, self.band, self.check_finite, self.fault
        o.refine_iters = self.refine_iters
        o.refine_rho = self.refine_rho
        o.qtrd = self.qtrd
        o.tridiag = self.tridiag
        return o


def skew_eig(A, nev: int, vectors: bool = True, stream=None):
    """Synchronous solve (device buffers).  Returns (lam, Z_re, Z_im)."""
    torch = _torch()
    A = _as_device_f64(A)
    n = A.shape[0]
    lam = torch.empty(max(nev, 1), dtype=torch.float64, device=A.device)
    Zr = fortran_empty(n, nev, A.device) if vectors else None
    Zi = fortran_empty(n, nev, A.device) if vectors else None
    code = lib().skew_eig(n, _ptr(A), _ld(A), nev, _ptr(lam), _ptr(Zr), _ptr(Zi), _stream(stream))
    _check(code, "skew_eig")
    return lam[:nev], Zr, Zi


def workspace_size(n: int, nev: int, opts: Options | None = None, vectors: bool = True) -> int:
    o = (opts or Options()).c()
    if vectors:
        return int(lib().skew_eig_workspace_size(n, nev, ctypes.byref(o)))
    return int(lib().skew_eig_workspace_size_ex(n, nev, ctypes.byref(o), 0))


def skew_eig_ex(A, nev: int, lam, Zr, Zi, workspace, d_info, opts: Options | None = None, stream=None) -> int:
    """Asynchronous solve into caller buffers; returns the launch status."""
    torch = _torch()
    A = _as_device_f64(A)
    n = A.shape[0]
    o = (opts or Options()).c()
    ldz = _ld(Zr) if Zr is not None else max(1, n)
    return lib().skew_eig_ex(n, _ptr(A), _ld(A), nev, _out(lam, torch.float64, nev, "lam"),
                             _zbuf(Zr, n, nev, "Zr"), _zbuf(Zi, n, nev, "Zi"), ldz, ctypes.byref(o),
                             _ptr(workspace), workspace.numel() * workspace.element_size(),
                             _out(d_info, torch.int32, 1, "d_info"), _stream(stream))


STAGES = ["ingest", "band_reduce", "band_pack", "chase", "tridiag", "dmap", "qtrd", "qband", "refine", "output"]


def skew_eig_profile(A, nev: int, lam, Zr, Zi, workspace, opts: Options | None = None, stream=None):
    """Synchronous solve into caller buffers with per-stage CUDA-event times.
    Returns (status, {stage: ms})."""
    torch = _torch()
    A = _as_device_f64(A)
    n = A.shape[0]
    o = (opts or Options()).c()
    ldz = _ld(Zr) if Zr is not None else max(1, n)
    ms = (ctypes.c_float * len(STAGES))()
    code = lib().skew_eig_profile(n, _ptr(A), _ld(A), nev, _out(lam, torch.float64, nev, "lam"),
                                  _zbuf(Zr, n, nev, "Zr"), _zbuf(Zi, n, nev, "Zi"), ldz, ctypes.byref(o),
                                  _ptr(workspace), workspace.numel() * workspace.element_size(), ms,
                                  _stream(stream))
    return code, dict(zip(STAGES, [float(x) for x in ms]))


def metrics(A, lam, Zr, Zi, cols=None, stream=None):
    """(residual, orthogonality, ||A||_F) over the columns `cols` (all if None)."""
    torch = _torch()
    A = _as_device_f64(A)
    n = A.shape[0]
    nev = Zr.shape[1]
    dcols = None
    ncols = nev
    if cols is not None:
        dcols = torch.as_tensor(cols, dtype=torch.int32, device=A.device)
        ncols = dcols.numel()
    ws = _ws(lib().skew_metrics_ws(n, nev, ncols), A.device)
    out = (ctypes.c_double * 3)()
    code = lib().skew_eig_metrics(n, _ptr(A), _ld(A), nev, _ptr(lam), _ptr(Zr), _ptr(Zi), _ld(Zr), _ptr(dcols),
                                  ncols, out, _ptr(ws), ws.numel(), _stream(stream))
    _check(code, "skew_eig_metrics")
    return float(out[0]), float(out[1]), float(out[2])


def gemm_bf16x3(A, B, C=None, alpha=1.0, beta=0.0, lower=False, planes=2, stream=None):
    """C = alpha * A @ B.T + beta * C on the tensor cores with BF16x3 splits
    (A: M x K, B: N x K float64 CUDA tensors of any strides; C Fortran-strided,
    returned).  lower=True: only the lower 128-tiles, C += alpha A B^T with a
    zero diagonal."""
    torch = _torch()
    M, K = A.shape
    N = B.shape[0]
    if C is None:
        C = fortran_empty(M, N, A.device)
        C.zero_()
    ws = _ws(lib().skew_gemm_bf16x3_ws(M, N, K), A.device)
    st = _status(A.device)
    code = lib().skew_gemm_bf16x3(M, N, K, alpha, _ptr(A), A.stride(0), A.stride(1), _ptr(B), B.stride(0),
                                  B.stride(1), beta, _ptr(C), _ld(C), 1 if lower else 0, planes, _ptr(ws), ws.numel(),
                                  _ptr(st), _stream(stream))
    _check(code, "skew_gemm_bf16x3")
    return C, st


def gemm_f64acc(A, B, C=None, alpha=1.0, beta=0.0, slices=8, lower=False, stream=None):
    """C = alpha * A @ B.T + beta * C to FP64 accuracy on the BF16 tensor cores
    (exact digit slices).  A: M x K, B: N x K float64 CUDA tensors.  slices < 8
    keeps fewer digit-slice products (error about 2^-7 slices); lower writes
    only the output tiles on or below the diagonal."""
    M, K = A.shape
    N = B.shape[0]
    if C is None:
        C = fortran_empty(M, N, A.device)
        C.zero_()
    ws = _ws(lib().skew_gemm_f64acc_ws(M, N, K), A.device)
    st = _status(A.device)
    if slices == 8 and not lower:
        code = lib().skew_gemm_f64acc(M, N, K, alpha, _ptr(A), A.stride(0), A.stride(1), _ptr(B), B.stride(0),
                                      B.stride(1), beta, _ptr(C), _ld(C), _ptr(ws), ws.numel(), _ptr(st),
                                      _stream(stream))
    else:
        code = lib().skew_gemm_f64acc_ex(M, N, K, alpha, _ptr(A), A.stride(0), A.stride(1), _ptr(B), B.stride(0),
                                         B.stride(1), beta, _ptr(C), _ld(C), int(slices), 1 if lower else 0,
                                         _ptr(ws), ws.numel(), _ptr(st), _stream(stream))
    _check(code, "skew_gemm_f64acc")
    return C, st


def refine_stats():
    """(iterations, [emax per iteration], [nclose per iteration]) of the most
    recent refinement in this process."""
    em = (ctypes.c_double * 8)()
    nc = (ctypes.c_int * 8)()
    it = lib().skew_refine_stats(em, nc, 8)
    return it, [float(x) for x in em[:it]], [int(x) for x in nc[:it]]


def refine(A, lam, Zr, Zi, iters=6, stream=None):
    """FP64 refinement of (lam, Zr + i Zi) in place (n even, nev = n/2)."""
    A = _as_device_f64(A)
    n = A.shape[0]
    ws = _ws(lib().skew_refine_ws(n), A.device)
    st = _status(A.device)
    code = lib().skew_refine(n, _ptr(A), _ld(A), _ptr(lam), _ptr(Zr), _ptr(Zi), _ld(Zr), iters, _ptr(ws),
                             ws.numel(), _ptr(st), _stream(stream))
    _check(code, "skew_refine")
    return lam, Zr, Zi


def refine_trace():
    rn = (ctypes.c_double * 8)()
    wh = (ctypes.c_longlong * 8)()
    it = lib().skew_refine_trace(rn, wh, 8)
    locs = [(int(w) & 0xFFFFF, (int(w) >> 20) & 0xFFFFF, (int(w) >> 40) & 1) for w in wh[:it]]
    return [float(x) for x in rn[:it]], locs


def refine_slices():
    """([Gram/projection slices per iteration], [update slices per iteration])
    of the most recent refinement in this process (8 = FP64-accurate)."""
    sl = (ctypes.c_int * 8)()
    su = (ctypes.c_int * 8)()
    it = lib().skew_refine_slices(sl, su, 8)
    return [int(x) for x in sl[:it]], [int(x) for x in su[:it]]


SKEW_KERNEL_OZAKI = 0
SKEW_KERNEL_SPLIT = 1
SKEW_KERNEL_OZAKI_REFINE = 2
SKEW_KERNEL_SLICE_SPLIT = 3
SKEW_KERNEL_PANEL_QR = 4
SKEW_KERNEL_GEMM_F64 = 5
SKEW_KERNEL_CHASE = 6
SKEW_KERNEL_BISECT = 7
SKEW_KERNEL_INVIT = 8
SKEW_KERNEL_QTRD = 9
SKEW_KERNEL_REFINE_AUX = 10
SKEW_KERNEL_OTHER = 11
KERNEL_KINDS = ["ozaki_product", "split_product", "ozaki_refine", "slice_split", "panel_qr", "gemm_f64",
                "chase", "bisect", "invit", "qtrd", "refine_aux", "other"]


def kernel_timing(enable: bool) -> None:
    """Switch per-launch event timing of the tensor-core product kernels on
    (clearing the record) or off."""
    lib().skew_kernel_timing(1 if enable else 0)


def kernel_timing_read(kind: int):
    """(total ms, algorithmic flops, launches) recorded for one kernel kind
    since timing was switched on.  Raises if any launch went unrecorded
    (the record pool was full), since the totals would then be short."""
    ms = ctypes.c_double()
    fl = ctypes.c_double()
    k = ctypes.c_longlong()
    code = lib().skew_kernel_timing_read(kind, ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(k))
    if code == -2:
        raise RuntimeError(f"kernel timing dropped {lib().skew_kernel_timing_dropped()} launches: "
                           "the per-kind totals are incomplete")
    _check(code, "skew_kernel_timing_read")
    return ms.value, fl.value, k.value



def kernel_timeline(cap=16384):
    """[(kind name, start ms, end ms)] of the timing records in launch order,
    relative to the first record's start (skew_kernel_timeline)."""
    kinds = (ctypes.c_int * cap)()
    t0 = (ctypes.c_double * cap)()
    t1 = (ctypes.c_double * cap)()
    cnt = lib().skew_kernel_timeline(cap, kinds, t0, t1)
    _check(min(cnt, 0), "skew_kernel_timeline")
    return [(KERNEL_KINDS[kinds[i]] if 0 <= kinds[i] < len(KERNEL_KINDS) else "?", t0[i], t1[i])
            for i in range(cnt)]

def _batch_arrays(As, nevs, vectors):
    torch = _torch()
    count = len(As)
    As = [_as_device_f64(A) for A in As]
    ns = [int(A.shape[0]) for A in As]
    lams = [torch.empty(max(nv, 1), dtype=torch.float64, device=A.device) for A, nv in zip(As, nevs)]
    Zr = [fortran_empty(n, nv, A.device) if vectors else None for A, n, nv in zip(As, ns, nevs)]
    Zi = [fortran_empty(n, nv, A.device) if vectors else None for A, n, nv in zip(As, ns, nevs)]
    IA = ctypes.c_int * max(count, 1)
    PA = ctypes.c_void_p * max(count, 1)
    c_n = IA(*ns)
    c_lda = IA(*[_ld(A) for A in As])
    c_nev = IA(*[int(v) for v in nevs])
    c_A = PA(*[A.data_ptr() for A in As])
    c_l = PA(*[t.data_ptr() for t in lams])
    c_zr = PA(*[z.data_ptr() for z in Zr]) if vectors else None
    c_zi = PA(*[z.data_ptr() for z in Zi]) if vectors else None
    return count, As, lams, Zr, Zi, (c_n, c_A, c_lda, c_nev, c_l, c_zr, c_zi)


def skew_eig_batched(As, nevs, vectors: bool = True, opts: Options | None = None, stream=None, info=False):
    """Solve many independent problems (list of float64 CUDA tensors A_b with
    nev_b each).  Returns lists (lam_b, Zr_b, Zi_b) [and the per-matrix status
    tensor when info=True]."""
    torch = _torch()
    count, As, lams, Zr, Zi, c = _batch_arrays(As, nevs, vectors)
    c_n, c_A, c_lda, c_nev, c_l, c_zr, c_zi = c
    o = (opts or Options()).c()
    nbytes = int(lib().skew_eig_batched_workspace_size(count, c_n, c_nev, ctypes.byref(o)))
    dev = As[0].device if As else torch.device("cuda")
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    d_info = torch.full((max(count, 1),), -1, dtype=torch.int32, device=dev)
    code = lib().skew_eig_batched_ex(count, c_n, c_A, c_lda, c_nev, c_l, c_zr, c_zi, ctypes.byref(o), _ptr(ws),
                                     ws.numel(), _ptr(d_info), _stream(stream))
    _check(code, "skew_eig_batched_ex")
    out = ([l[:nv] for l, nv in zip(lams, nevs)], Zr, Zi)
    return out + (d_info[:count],) if info else out


def bse_solve(A, B, nev: int, opts: Options | None = None, stream=None):
    """The Bethe-Salpeter eigenproblem H_BS = [[A, B], [-conj(B), -conj(A)]]
    (A Hermitian, B complex symmetric, h x h complex128 CUDA tensors) through
    skew_bse_solve (Sec. 3): the nev largest positive eigenvalues (descending)
    and psi (2h x nev complex128) with H_BS psi = psi diag(lam) and
    psi^H S psi = I.  Returns (lam, psi, status)."""
    torch = _torch()
    h = A.shape[0]
    dev = A.device
    Ar, Ai = fortran(A.real.contiguous()), fortran(A.imag.contiguous())
    Br, Bi = fortran(B.real.contiguous()), fortran(B.imag.contiguous())
    o = (opts or Options()).c()
    ws = _ws(lib().skew_bse_workspace_size(h, nev, ctypes.byref(o)), dev)
    lam = torch.empty(nev, dtype=torch.float64, device=dev)
    Pr, Pi = fortran_empty(2 * h, nev, dev), fortran_empty(2 * h, nev, dev)
    st = _status(dev)
    code = lib().skew_bse_solve(h, _ptr(Ar), _ptr(Ai), _ld(Ar), _ptr(Br), _ptr(Bi), _ld(Br), nev, _ptr(lam),
                                _ptr(Pr), _ptr(Pi), 2 * h, ctypes.byref(o), _ptr(ws), ws.numel(), _ptr(st),
                                _stream(stream))
    _check(code, "skew_bse_solve")
    return lam, torch.complex(Pr, Pi), st


def batched_set_config(ctas_per_sm: int, smem_max_n: int) -> None:
    """Process-wide launch configuration of the batched solve."""
    c = skew_batched_config(ctas_per_sm, smem_max_n)
    _check(lib().skew_batched_set_config(ctypes.byref(c)), "skew_batched_set_config")


def batched_get_config():
    c = skew_batched_config()
    lib().skew_batched_get_config(ctypes.byref(c))
    return int(c.ctas_per_sm), int(c.smem_max_n)


class BatchedPlan:
    """A batch of problems (orders <= 1024) prepared once and solved by one
    persistent launch per execute() (skew_batched_plan_*).  Holds its device
    buffers; execute() does no host synchronisation and can be captured in a
    CUDA graph."""

    def __init__(self, As, nevs, vectors: bool = True, config=None, stream=None):
        torch = _torch()
        self.count, self.As, lams, self.Zr, self.Zi, self._c = _batch_arrays(As, nevs, vectors)
        self.nevs = [int(v) for v in nevs]
        self.lams = lams
        c_n, c_A, c_lda, c_nev, c_l, c_zr, c_zi = self._c
        dev = self.As[0].device if self.As else torch.device("cuda")
        nbytes = int(lib().skew_eig_batched_workspace_size(self.count, c_n, c_nev, None))
        self.ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
        self.info = torch.zeros(max(self.count, 1), dtype=torch.int32, device=dev)
        cfg = skew_batched_config(*config) if config is not None else None
        self._plan = ctypes.c_void_p()
        code = lib().skew_batched_plan_create(self.count, c_n, c_A, c_lda, c_nev, c_l, c_zr, c_zi,
                                              ctypes.byref(cfg) if cfg is not None else None, _ptr(self.ws),
                                              self.ws.numel(), _ptr(self.info), _stream(stream),
                                              ctypes.byref(self._plan))
        _check(code, "skew_batched_plan_create")

    def execute(self, stream=None):
        _check(lib().skew_batched_plan_exec(self._plan, _stream(stream)), "skew_batched_plan_exec")

    def tune(self, stream=None):
        """Time every launch configuration on this batch; keep and return the
        fastest as (ctas_per_sm, smem_max_n) with the list of
        (ctas_per_sm, smem_max_n, ms) candidates."""
        cap = 64
        ca, cs = (ctypes.c_int * cap)(), (ctypes.c_int * cap)()
        cm = (ctypes.c_float * cap)()
        best = skew_batched_config()
        k = lib().skew_batched_plan_tune(self._plan, ctypes.byref(best), ca, cs, cm, cap, _stream(stream))
        if k < 0 or k > 10000:
            _check(k, "skew_batched_plan_tune")
        cands = [(int(ca[i]), int(cs[i]), float(cm[i])) for i in range(min(k, cap))]
        return (int(best.ctas_per_sm), int(best.smem_max_n)), cands

    def config(self):
        c = skew_batched_config()
        lib().skew_batched_plan_get_config(self._plan, ctypes.byref(c))
        return int(c.ctas_per_sm), int(c.smem_max_n)

    def results(self):
        return [l[:nv] for l, nv in zip(self.lams, self.nevs)], self.Zr, self.Zi

    def __del__(self):
        try:
            if self._plan:
                lib().skew_batched_plan_destroy(self._plan)
                self._plan = ctypes.c_void_p()
        except Exception:
            pass


def shard_lpt(sizes, world: int):
    """Partition batch members over `world` ranks by longest-processing-time on
    n^3 cost (largest first, each to the least-loaded rank, ties to the lowest
    rank).  Returns one sorted index list per rank; deterministic, so every
    rank computes the same partition without communication."""
    import heapq
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]) ** 3, i))
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]) ** 3, r))
    return [sorted(p) for p in parts]


def launch_count() -> int:
    return int(lib().skew_launch_count())


def skew_eig_host(A, nev: int, vectors: bool = True, opts: Options | None = None, stream=None):
    """Solve from host (ideally pinned) float64 tensors; returns host tensors."""
    torch = _torch()
    A = fortran(A.to(device="cpu", dtype=torch.float64))
    n = A.shape[0]
    pin = torch.cuda.is_available()
    lam = torch.empty(max(nev, 1), dtype=torch.float64, pin_memory=pin)
    Zr = torch.empty((nev, n), dtype=torch.float64, pin_memory=pin).t() if vectors else None
    Zi = torch.empty((nev, n), dtype=torch.float64, pin_memory=pin).t() if vectors else None
    o = (opts or Options()).c()
    code = lib().skew_eig_host(n, _hptr(A), _ld(A), nev, _hptr(lam), _hptr(Zr), _hptr(Zi), ctypes.byref(o),
                               _stream(stream))
    _check(code, "skew_eig_host")
    return lam[:nev], Zr, Zi


# ----------------------------------------------------------------- stages
def _status(device):
    torch = _torch()
    return torch.zeros(1, dtype=torch.int32, device=device)


def _ws(nbytes: int, device):
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def band_reduce(A, b: int = 64, stream=None):
    """Full-to-band reduction of skew A.  Returns (W, Tfac, status)."""
    torch = _torch()
    A = _as_device_f64(A)
    n = A.shape[0]
    W = fortran_empty(n, n, A.device)
    W.copy_(A)
    P = (n - 2) // b if n - 2 >= b else 0
    Tfac = torch.zeros(max(P, 1) * b * b, dtype=torch.float64, device=A.device)
    ws = _ws(lib().skew_band_reduce_ws(n, b), A.device)
    st = _status(A.device)
    code = lib().skew_band_reduce(n, _ptr(W), _ld(W), b, _ptr(Tfac), _ptr(ws), ws.numel(), _ptr(st), _stream(stream))
    _check(code, "skew_band_reduce")
    return W, Tfac, st


def band_pack(W, b: int = 64, stream=None):
    torch = _torch()
    n = W.shape[0]
    ldab = 2 * b + 1
    AB = torch.zeros((max(n, 1), ldab), dtype=torch.float64, device=W.device)  # row c = column c of AB
    _check(lib().skew_band_pack(n, b, _ptr(W), _ld(W), _ptr(AB), ldab, _stream(stream)), "skew_band_pack")
    return AB


def band_to_tridiag(AB, n: int, b: int = 64, stream=None):
    """Bulge chase on packed band AB (n rows of length 2b+1).  Returns
    (alpha, Vtrd, tautrd, status)."""
    torch = _torch()
    K = lib().skew_chase_steps(n, b)
    nsw = max(n - 2, 1)
    alpha = torch.zeros(max(n, 1), dtype=torch.float64, device=AB.device)
    Vtrd = torch.zeros(max(K, 1) * nsw * b, dtype=torch.float64, device=AB.device)
    tau = torch.zeros(max(K, 1) * nsw, dtype=torch.float64, device=AB.device)
    ws = _ws(lib().skew_chase_ws(n, b), AB.device)
    st = _status(AB.device)
    code = lib().skew_band_to_tridiag(n, b, _ptr(AB), 2 * b + 1, _ptr(alpha), _ptr(Vtrd), _ptr(tau), _ptr(ws),
                                      ws.numel(), _ptr(st), _stream(stream))
    _check(code, "skew_band_to_tridiag")
    return alpha[: max(n - 1, 0)], Vtrd, tau, st


def tridiag_eig(alpha, nev: int, vectors: bool = True, stream=None):
    """Eigenpairs of tridiag(alpha, 0, alpha): (lam desc, Q n x nev, status)."""
    torch = _torch()
    n = alpha.numel() + 1
    a = torch.zeros(n, dtype=torch.float64, device=alpha.device)
    a[: n - 1] = alpha
    lam = torch.empty(nev, dtype=torch.float64, device=alpha.device)
    Q = fortran_empty(n, nev, alpha.device) if vectors else None
    ws = _ws(lib().skew_tridiag_ws(n, nev), alpha.device)
    st = _status(alpha.device)
    code = lib().skew_tridiag_eig(n, _ptr(a), nev, _ptr(lam), _ptr(Q), n, _ptr(ws), ws.numel(), _ptr(st),
                                  _stream(stream))
    _check(code, "skew_tridiag_eig")
    return lam, Q, st


def tridiag_eig_noalloc(alpha, nev: int, vectors: bool = True, stream=None):
    """tridiag_eig through the entry point that allocates no device memory
    (its scratch is a static device array inside the library)."""
    torch = _torch()
    n = alpha.numel() + 1
    a = torch.zeros(n, dtype=torch.float64, device=alpha.device)
    a[: n - 1] = alpha
    lam = torch.empty(nev, dtype=torch.float64, device=alpha.device)
    Q = fortran_empty(n, nev, alpha.device) if vectors else None
    st = _status(alpha.device)
    code = lib().skew_tridiag_eig_noalloc(n, _ptr(a), nev, _ptr(lam), _ptr(Q), n, _ptr(st), _stream(stream))
    _check(code, "skew_tridiag_eig_noalloc")
    return lam, Q, st


def dmap(Q, stream=None):
    n, k = Q.shape
    Q = fortran(Q)
    X = fortran_empty(n, k, Q.device)
    Y = fortran_empty(n, k, Q.device)
    _check(lib().skew_dmap(n, k, _ptr(Q), _ld(Q), _ptr(X), _ptr(Y), n, _stream(stream)), "skew_dmap")
    return X, Y


def apply_qtrd(Vtrd, tau, Z, b: int = 64, stream=None):
    """Z <- Q_trd Z in place (Z Fortran-strided n x k)."""
    n, k = Z.shape
    _check(lib().skew_apply_qtrd(n, b, _ptr(Vtrd), _ptr(tau), _ptr(Z), _ld(Z), k, _stream(stream)), "skew_apply_qtrd")
    return Z


def apply_qtrd_f32(V32, tau32, Z, tensor: bool, b: int = 64, stream=None):
    """Z (float32, Fortran-strided n x k) <- Q_trd Z in place from FP32
    reflectors in the chase's slot layout (skew_apply_qtrd_f32); tensor
    selects the tcgen05 compact-WY form.  Returns the device status word."""
    n, k = Z.shape
    ws = _ws(lib().skew_apply_qtrd_f32_ws(n, 1 if tensor else 0), Z.device)
    st = _status(Z.device)
    _check(lib().skew_apply_qtrd_f32(n, b, _ptr(V32), _ptr(tau32), _ptr(Z), _ld(Z), k, 1 if tensor else 0,
                                     _ptr(ws), ws.numel(), _ptr(st), _stream(stream)), "skew_apply_qtrd_f32")
    return st


def apply_qtrd_df(Vtrd, tau, Z, b: int = 64, stream=None):
    """Z (float64, Fortran-strided n x k) <- Q_trd Z in place in double-float
    arithmetic (skew_apply_qtrd_df).  Returns the device status word."""
    n, k = Z.shape
    st = _status(Z.device)
    _check(lib().skew_apply_qtrd_df(n, b, _ptr(Vtrd), _ptr(tau), _ptr(Z), _ld(Z), k, _ptr(st), _stream(stream)),
           "skew_apply_qtrd_df")
    return st


def apply_qband(W, Tfac, Z, b: int = 64, stream=None):
    """Z <- Q_band Z in place."""
    n, k = Z.shape
    ws = _ws(lib().skew_qband_ws(n, b, k), Z.device)
    _check(lib().skew_apply_qband(n, b, _ptr(W), _ld(W), _ptr(Tfac), _ptr(Z), _ld(Z), k, _ptr(ws), ws.numel(),
                                  _stream(stream)), "skew_apply_qband")
    return Z


def strerror(code: int) -> str:
    return lib().skew_eig_strerror(code).decode()
