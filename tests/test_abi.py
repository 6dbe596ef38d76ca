"""The C-ABI library loads and exports every entry point include/skeweig.h
declares; host-side argument checks work without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "skeweig.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:long\s+long|\w+)\s*\*?\s*(skew_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def sk():
    from paper_1912_04062_gb300 import build
    build.build()
    import paper_1912_04062_gb300 as pkg
    pkg.lib()
    return pkg


def test_every_declared_symbol_is_exported(sk):
    names = _declared()
    assert len(names) >= 15
    L = ctypes.CDLL(sk.LIB_PATH)
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(sk.SIGNATURES), set(names) ^ set(sk.SIGNATURES)


def test_strerror_and_defaults(sk):
    L = sk.lib()
    for code in [0, -3, 1005, 2001, 2002, 2003, 2004, 2005, 2006, 2007, 9999]:
        assert L.skew_eig_strerror(code)
    o = sk.skew_opts()
    L.skew_opts_default(ctypes.byref(o))
    assert o.mode == 0 and o.band == 64


def test_argument_checks_are_host_side(sk):
    L = sk.lib()
    nul = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(16)  # never dereferenced: the checks fail first
    assert L.skew_eig(-1, fake, 1, 0, fake, nul, nul, nul) == -1
    assert L.skew_eig(4, nul, 4, 1, fake, nul, nul, nul) == -2
    assert L.skew_eig(4, fake, 3, 1, fake, nul, nul, nul) == -3
    assert L.skew_eig(4, fake, 4, 3, fake, nul, nul, nul) == -4
    assert L.skew_eig(5, fake, 5, 3, fake, nul, nul, nul) == -4
    assert L.skew_eig(4, fake, 4, 1, nul, nul, nul, nul) == -5
    assert L.skew_eig(4, fake, 4, 1, fake, fake, nul, nul) == -6
    # no-op cases
    assert L.skew_eig(0, nul, 1, 0, nul, nul, nul, nul) == 0
    assert L.skew_eig(1, fake, 1, 0, nul, nul, nul, nul) == 0
    assert L.skew_eig(9, fake, 9, 0, nul, nul, nul, nul) == 0
    # INT8 Ozaki mode is rejected before any device work
    o = sk.skew_opts()
    L.skew_opts_default(ctypes.byref(o))
    o.mode = sk.SKEW_MODE_MIXED_INT8
    assert L.skew_eig_ex(8, fake, 8, 2, fake, fake, fake, 8, ctypes.byref(o), fake, 1 << 20, fake, nul) == \
        sk.SKEW_ERR_UNSUPPORTED


def test_workspace_size_grows(sk):
    sizes = [sk.workspace_size(n, n // 2) for n in (64, 512, 4096)]
    assert sizes[0] < sizes[1] < sizes[2]
    # dominant terms: W (n^2), chase reflectors (~n^2), interleaved LU (4 n nev)
    n = 4096
    assert sizes[2] >= 8 * (2 * n * n)


def test_f64acc_ex_argument_checks_are_host_side(sk):
    L = sk.lib()
    nul = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(16)  # never dereferenced: the checks fail first

    def call(M=8, N=8, K=8, ldc=8, slices=8, lower=0):
        return L.skew_gemm_f64acc_ex(M, N, K, 1.0, fake, 8, 1, fake, 8, 1, 0.0, fake, ldc, slices, lower,
                                     fake, 1 << 20, fake, nul)
    assert call(M=-1) == -1
    assert call(N=-1) == -2
    assert call(K=0) == -3
    assert call(ldc=7) == -13
    assert call(slices=0) == -14
    assert call(slices=9) == -14
    assert call(lower=2) == -15
    # the error-name query is available without a failure
    assert L.skew_last_cuda_error()


def test_kernel_timing_switch_is_host_side(sk):
    L = sk.lib()
    assert L.skew_kernel_timing(1) == 0
    ms, fl, k = sk.kernel_timing_read(sk.SKEW_KERNEL_OZAKI)
    assert (ms, fl, k) == (0.0, 0.0, 0)
    assert L.skew_kernel_timing_read(12, None, None, None) == -1
    assert L.skew_kernel_timing_read(-1, None, None, None) == -1
    # no records yet: an empty timeline; a negative capacity is an argument error
    assert sk.kernel_timeline() == []
    assert L.skew_kernel_timeline(-1, None, None, None) == -1
    assert L.skew_kernel_timing_dropped() == 0
    assert L.skew_kernel_timing(0) == 0


def test_nomem_fault_fails_before_any_allocation(sk):
    # SKEW_FAULT_NOMEM: the allocating entry points report SKEW_ERR_NOMEM
    # before they touch the GPU, so this runs without one
    L = sk.lib()
    n, nev = 8, 4
    A = (ctypes.c_double * (n * n))()
    lam = (ctypes.c_double * nev)()
    Zr = (ctypes.c_double * (n * nev))()
    Zi = (ctypes.c_double * (n * nev))()
    o = sk.Options(fault=sk.SKEW_FAULT_NOMEM).c()
    nul = ctypes.c_void_p(0)
    assert L.skew_eig_host(n, A, n, nev, lam, Zr, Zi, ctypes.byref(o), nul) == sk.SKEW_ERR_NOMEM
    IA = ctypes.c_int * 2
    PA = ctypes.c_void_p * 2
    fake = PA(16, 16)
    assert L.skew_eig_batched(2, IA(4, 4), fake, IA(4, 4), IA(1, 1), fake, fake, fake, ctypes.byref(o),
                              nul) == sk.SKEW_ERR_NOMEM
    # argument errors still come first
    assert L.skew_eig_host(n, A, n - 1, nev, lam, Zr, Zi, ctypes.byref(o), nul) == -3
    # releasing the (empty) pools is a no-op without a GPU
    L.skew_release_memory()


def test_batched_argument_checks_are_host_side(sk):
    L = sk.lib()
    IA = ctypes.c_int * 2
    PA = ctypes.c_void_p * 2
    fake = PA(16, 16)
    nul = ctypes.c_void_p(0)

    def call(n=(4, 4), lda=(4, 4), nev=(1, 1), count=2, Zr=None, Zi=None):
        return L.skew_eig_batched(count, IA(*n), fake, IA(*lda), IA(*nev), fake, Zr, Zi, None, nul)
    assert call(count=-1) == -1
    assert call(n=(4, -1)) == -2
    assert call(lda=(4, 3)) == -4
    assert call(nev=(1, 3)) == -5
    assert call(Zr=fake, Zi=None) == -7
    assert L.skew_eig_batched(0, None, None, None, None, None, None, None, None, nul) == 0
    # workspace grows with the batch and covers the largest single solve
    small = sk.lib().skew_eig_batched_workspace_size(2, IA(40, 100), IA(20, 50), None)
    mid = sk.lib().skew_eig_batched_workspace_size(2, IA(40, 400), IA(20, 200), None)
    big = sk.lib().skew_eig_batched_workspace_size(2, IA(40, 2000), IA(20, 1000), None)
    assert 0 < small < mid < big
    # orders above the batched kernels' limit take the two-step solve's workspace
    assert big >= sk.workspace_size(2000, 1000)


def test_binding_constants_match_the_header(sk):
    # every SKEW_* integer constant of the header has the same value in the
    # Python binding (status codes, modes, fault hooks, kernel kinds)
    text = open(HEADER).read()
    consts = dict((k, int(v)) for k, v in re.findall(r"^#define\s+(SKEW_\w+)\s+(-?\d+)\b", text, flags=re.M))
    # enumerators of the mode enum
    consts.update((k, int(v)) for k, v in re.findall(r"^\s+(SKEW_MODE_\w+)\s*=\s*(\d+)", text, flags=re.M))
    assert len(consts) >= 30 and "SKEW_MODE_MIXED_REFINED" in consts
    missing = [k for k in consts if not hasattr(sk, k) and k not in ("SKEW_NSTAGES", "SKEW_KERNEL_KINDS")]
    assert not missing, missing
    for k, v in consts.items():
        if hasattr(sk, k):
            assert getattr(sk, k) == v, (k, getattr(sk, k), v)
    assert len(sk.STAGES) == consts["SKEW_NSTAGES"]
    assert len(sk.KERNEL_KINDS) == consts["SKEW_KERNEL_KINDS"]


def test_opts_struct_layout_matches_the_header(sk):
    # the ctypes mirror of skew_opts has the header's fields, in order, and
    # skew_opts_default fills it as documented (FP64 mode, b = 64 or 0)
    text = open(HEADER).read()
    body = re.search(r"typedef struct \{(.*?)\} skew_opts;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"int\s+(\w+)(\[\d+\])?\s*;", body)
    names = [f[0] for f in fields]
    assert names == [f[0] for f in sk.skew_opts._fields_]
    for (name, arr), (pname, ptype) in zip(fields, sk.skew_opts._fields_):
        n = int(arr[1:-1]) if arr else 1
        assert ctypes.sizeof(ptype) == n * ctypes.sizeof(ctypes.c_int), name
    o = sk.skew_opts()
    sk.lib().skew_opts_default(ctypes.byref(o))
    assert o.mode == sk.SKEW_MODE_FP64 and o.band in (0, 64) and o.fault == 0


def _prototypes():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"^\s*#.*$", "", text, flags=re.M)
    out = {}
    for m in re.finditer(r"([\w\s\*]+?)\b(skew_\w+)\s*\(([^)]*)\)\s*;", text):
        ret, name, params = m.group(1).strip(), m.group(2), m.group(3).strip()
        plist = [] if params in ("", "void") else [q.strip() for q in params.split(",")]
        out[name] = (ret, plist)
    return out


def _ctype_of(decl):
    d = " ".join(decl.replace("*", " * ").split())
    if "*" in d:
        return "ptr"
    base = re.sub(r"\b(const|unsigned)\b", "", d).split()
    t = " ".join(base[:-1]) if len(base) > 1 else base[0]
    return {"int": "int", "size_t": "size_t", "double": "double", "long long": "longlong", "void": "void",
            "long": "longlong"}[t]


def test_binding_signatures_match_the_prototypes(sk):
    # argument count and kind (pointer / int / size_t / double / long long) of
    # every ctypes declaration equal the header's prototype
    kind = {ctypes.c_void_p: "ptr", ctypes.c_char_p: "ptr", ctypes.c_int: "int", ctypes.c_size_t: "size_t",
            ctypes.c_double: "double", ctypes.c_longlong: "longlong", None: "void"}
    protos = _prototypes()
    assert set(protos) == set(sk.SIGNATURES)
    for name, (ret, params) in protos.items():
        restype, argtypes = sk.SIGNATURES[name]
        assert len(argtypes) == len(params), (name, len(argtypes), len(params))
        for a, decl in zip(argtypes, params):
            assert kind[a] == _ctype_of(decl), (name, decl, a)
        want_ret = "ptr" if "*" in ret else _ctype_of(ret + " x")
        assert kind[restype] == want_ret, (name, ret, restype)
