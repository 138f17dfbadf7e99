"""Thin ctypes binding of libed.so (include/ed.h), one Python function per C entry
point with the same name minus the ``ed_`` prefix.  Argument marshalling only:
every step of the computation runs in the library's CUDA kernels.

Device arrays are torch CUDA tensors (PyTorch provides device memory and
streams); the default stream argument is torch's current stream.  There is no
CPU fallback: importing this module without the built library raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libed.so")

ED_OK = 0
ED_F64, ED_F32, ED_C128, ED_C64 = 0, 1, 2, 3
ED_LANCZOS_F64, ED_LANCZOS_F32_MATVEC, ED_LANCZOS_RECOMPUTE, ED_LANCZOS_PUSH = 0, 1, 16, 32
ED_LANCZOS_REORTH = 64
ED_LANCZOS_VALUES_ONLY = 128

STATUS_NAMES = {
    0: "ED_OK", 1: "ED_ERR_INVALID_ARG", 2: "ED_ERR_NOT_A_GROUP", 3: "ED_ERR_BAD_CHARACTER",
    4: "ED_ERR_SYMMETRY_MISMATCH", 5: "ED_ERR_OOM", 6: "ED_ERR_CUDA", 7: "ED_ERR_INTERNAL",
    8: "ED_ERR_NOT_CONVERGED", 9: "ED_ERR_UNSUPPORTED", 10: "ED_ERR_TIMEOUT",
}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2308_16712_gb300.build.build() "
                      "(there is no fallback implementation)")

_lib = ctypes.CDLL(LIB_PATH)
_P = ctypes.c_void_p
_i32, _u64, _i64, _d = ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double


class Sector(ctypes.Structure):
    _fields_ = [("basis", ctypes.c_void_p), ("d_x", ctypes.c_void_p), ("d_y", ctypes.c_void_p)]


class TuneResult(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("search", ctypes.c_int), ("index", ctypes.c_int),
                ("ms_default", ctypes.c_double), ("ms_best", ctypes.c_double), ("variants_timed", ctypes.c_int)]


class LanczosInfo(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("matvecs", ctypes.c_int), ("ritz", ctypes.c_double),
                ("e0", ctypes.c_double), ("residual", ctypes.c_double),
                ("matvec_ms", ctypes.c_double)]


_SIGS = {
    "ed_status_string": (ctypes.c_char_p, [_i32]),
    "ed_release_cached_memory": (_i32, []),
    "ed_stream_status": (_i32, [_P]),
    "ed_basis_build": (_i32, [_i32, _i32, _i32, _i32, _P, _P, _P, ctypes.POINTER(_P)]),
    "ed_basis_size": (_i32, [_P, ctypes.POINTER(_u64)]),
    "ed_basis_count": (_i32, [_i32, _i32, _i32, _i32, _P, _P, _P, ctypes.POINTER(_u64)]),
    "ed_basis_states": (_i32, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "ed_basis_is_real": (_i32, [_P, ctypes.POINTER(_i32)]),
    "ed_basis_index": (_i32, [_P, _P, _P, _u64, _P]),
    "ed_basis_destroy": (None, [_P]),
    "ed_operator_create": (_i32, [_i32, _i32, _P, _P, _P, ctypes.POINTER(_P)]),
    "ed_operator_destroy": (None, [_P]),
    "ed_matvec": (_i32, [_P, _P, _P, _P, _i32, _i32, _P]),
    "ed_matvec_multi": (_i32, [_P, _P, _i32, _i32, _i32, _P]),
    "ed_lanczos": (_i32, [_P, _P, _P, _i32, _i32, ctypes.POINTER(_d), _P,
                          ctypes.POINTER(LanczosInfo), _P]),
    "ed_lanczos_eigs": (_i32, [_P, _P, _P, _i32, _i32, _i32, ctypes.POINTER(_d), _d, _P,
                               ctypes.POINTER(LanczosInfo), _P]),
    "ed_lanczos_block": (_i32, [_P, _P, _P, _i32, _i32, _i32, _i32, ctypes.POINTER(_d), ctypes.POINTER(_d), _P,
                                ctypes.POINTER(LanczosInfo), _P]),
    "ed_lanczos_multi": (_i32, [_P, _P, _i32, _i32, _i32, _i32, ctypes.POINTER(_d),
                                ctypes.POINTER(LanczosInfo), _P]),
    "ed_autotune": (_i32, [_P, _P, _P, _P, _i32, _i32, ctypes.POINTER(TuneResult), _P]),
    "ed_autotune_index": (_i32, [_P, _i32, _i32, _i32, _i32, _P, _P, _i32, _i32, ctypes.POINTER(TuneResult), _P]),
    "edx_tune_reset": (None, []),
    "ed_basis_count_noalloc": (_i32, [_i32, _i32, _i32, _i32, _P, _P, _P, ctypes.POINTER(_u64)]),
    "edx_launch_count": (ctypes.c_ulonglong, []),
    "edx_force_generic": (None, [_i32]),
    "edx_force_all_rotations": (None, [_i32]),
    "edx_index_policy": (None, [_i32]),
    "edx_inject_stall": (None, [_i32]),
    "edx_multi_policy": (None, [_i32]),
    "edx_lanczos_graph": (_i32, [_i32]),
    "edx_peak": (_d, [_i32, _P, _u64, ctypes.POINTER(_d), _P]),
    "edx_basis_bucket": (_i32, [_P, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_uint32)]),
    "edx_count_nnz": (_i32, [_P, _P, ctypes.POINTER(ctypes.c_ulonglong)]),
    "edx_force_prefix_search": (None, [_i32]),
    "edx_kernel_policy": (None, [_i32]),
    "edx_matvec_push": (_i32, [_P, _P, _P, _P, _i32, _P]),
    "edx_basis_hash": (_i32, [_P, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(_i32)]),
    "edx_basis_table": (_i32, [_P, ctypes.POINTER(_u64), ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(_i32)]),
    "edx_basis_factored": (_i32, [_P, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
}
for _name, (_res, _args) in _SIGS.items():
    if hasattr(_lib, _name):
        _f = getattr(_lib, _name)
        _f.restype = _res
        _f.argtypes = _args


class EDError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} "
                         f"({_lib.ed_status_string(status).decode()})")


def _check(st: int, where: str):
    if st != ED_OK:
        raise EDError(st, where)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _host(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class _DevArray:
    """__cuda_array_interface__ wrapper so torch can view library-owned memory."""

    def __init__(self, ptr: int, n: int, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}
        self._owner = owner


class Basis:
    """Owns an ed_basis handle."""

    def __init__(self, handle: ctypes.c_void_p, n_sites: int):
        self.handle = handle
        self.n_sites = n_sites

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.ed_basis_destroy(self.handle)
            self.handle = None


class Operator:
    """Owns an ed_operator handle."""

    def __init__(self, handle: ctypes.c_void_p, n_sites: int):
        self.handle = handle
        self.n_sites = n_sites

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.ed_operator_destroy(self.handle)
            self.handle = None


def release_cached_memory() -> None:
    """Return the device memory the library keeps cached for later calls."""
    _check(_lib.ed_release_cached_memory(), "ed_release_cached_memory")


def status_string(status: int) -> str:
    return _lib.ed_status_string(status).decode()


def stream_status(stream=None) -> int:
    """Synchronise the stream and return the device-detected status (0 = ok)."""
    return int(_lib.ed_stream_status(_stream(stream)))


def basis_build(n_sites: int, n_up: int, spin_inversion: int, perms, chars, stream=None) -> Basis:
    perms = _host(perms, np.int32).reshape(-1, n_sites)
    chars = _host(chars, np.float64).reshape(-1, 2)
    if len(perms) != len(chars):
        raise ValueError("perms and chars disagree on the group order")
    out = ctypes.c_void_p()
    _check(_lib.ed_basis_build(n_sites, n_up, spin_inversion, len(perms),
                               perms.ctypes.data_as(_P), chars.ctypes.data_as(_P), _stream(stream),
                               ctypes.byref(out)), "ed_basis_build")
    return Basis(out, n_sites)


def basis_count(n_sites: int, n_up: int, spin_inversion: int, perms, chars, stream=None) -> int:
    """Sector dimension from the enumeration's count pass (no basis kept)."""
    perms = _host(perms, np.int32).reshape(-1, n_sites)
    chars = _host(chars, np.float64).reshape(-1, 2)
    d = ctypes.c_uint64()
    _check(_lib.ed_basis_count(n_sites, n_up, spin_inversion, len(perms), perms.ctypes.data_as(_P),
                               chars.ctypes.data_as(_P), _stream(stream), ctypes.byref(d)),
           "ed_basis_count")
    return d.value


def basis_count_noalloc(n_sites: int, n_up: int, spin_inversion: int, perms, chars,
                        stream=None) -> int:
    """Sector dimension without any device allocation (fixed in-library scratch;
    overlapping calls race)."""
    perms = _host(perms, np.int32).reshape(-1, n_sites)
    chars = _host(chars, np.float64).reshape(-1, 2)
    d = ctypes.c_uint64()
    _check(_lib.ed_basis_count_noalloc(n_sites, n_up, spin_inversion, len(perms),
                                       perms.ctypes.data_as(_P), chars.ctypes.data_as(_P),
                                       _stream(stream), ctypes.byref(d)), "ed_basis_count_noalloc")
    return d.value


def basis_size(basis: Basis) -> int:
    d = ctypes.c_uint64()
    _check(_lib.ed_basis_size(basis.handle, ctypes.byref(d)), "ed_basis_size")
    return d.value


def basis_is_real(basis: Basis) -> bool:
    r = ctypes.c_int()
    _check(_lib.ed_basis_is_real(basis.handle, ctypes.byref(r)), "ed_basis_is_real")
    return bool(r.value)


def basis_states(basis: Basis):
    """(states, norms) as torch CUDA tensor views (int64 holding the uint64 bits,
    int16 holding the uint16 norms); valid while `basis` lives."""
    import torch
    s, n = ctypes.c_void_p(), ctypes.c_void_p()
    _check(_lib.ed_basis_states(basis.handle, ctypes.byref(s), ctypes.byref(n)), "ed_basis_states")
    dim = basis_size(basis)
    if dim == 0:
        dev = torch.device("cuda")
        return torch.empty(0, dtype=torch.int64, device=dev), torch.empty(0, dtype=torch.int16, device=dev)
    st = torch.as_tensor(_DevArray(s.value, dim, "<i8", basis), device="cuda")
    nm = torch.as_tensor(_DevArray(n.value, dim, "<i2", basis), device="cuda")
    return st, nm


def basis_index(basis: Basis, query, out=None, stream=None):
    """stateToIndex for an int64 CUDA tensor of states; returns int64 indices (-1 = absent)."""
    import torch
    q = query.contiguous()
    if out is None:
        out = torch.empty(q.numel(), dtype=torch.int64, device=q.device)
    _check(_lib.ed_basis_index(basis.handle, _ptr(q), _ptr(out), q.numel(), _stream(stream)),
           "ed_basis_index")
    return out


def operator_create(n_sites: int, sites, coeff, local) -> Operator:
    sites = _host(sites, np.int32).reshape(-1, 2)
    coeff = _host(coeff, np.float64).reshape(-1, 2)
    local = _host(local, np.float64).reshape(-1, 16, 2)
    out = ctypes.c_void_p()
    _check(_lib.ed_operator_create(n_sites, len(sites), coeff.ctypes.data_as(_P),
                                   sites.ctypes.data_as(_P), local.ctypes.data_as(_P),
                                   ctypes.byref(out)), "ed_operator_create")
    return Operator(out, n_sites)


_DTYPE_CODE = {"float64": ED_F64, "float32": ED_F32, "complex128": ED_C128, "complex64": ED_C64}


def matvec(op: Operator, basis: Basis, x, y, nvec: int = 1, stream=None):
    """y = H x (torch CUDA tensors of shape (dim,) or (dim, nvec), same dtype)."""
    if x.dtype != y.dtype:
        raise ValueError("x and y must share a dtype")
    code = _DTYPE_CODE[str(x.dtype).replace("torch.", "")]
    if not (x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x and y must be contiguous")
    _check(_lib.ed_matvec(op.handle, basis.handle, _ptr(x), _ptr(y), nvec, code, _stream(stream)),
           "ed_matvec")
    return y


def launch_count() -> int:
    """Kernel launches the library has issued since it was loaded (diagnostics)."""
    return int(_lib.edx_launch_count())


def force_generic(on: bool) -> None:
    """Testing aid: use the generic Benes group search even where the factored
    (rotation x coset) search applies.  Affects later launches and builds."""
    _lib.edx_force_generic(1 if on else 0)


def force_all_rotations(on: bool) -> None:
    """Test hook: the factored group search visits every rotation (no pruning
    to the tops of the longest runs of equal bits)."""
    _lib.edx_force_all_rotations(1 if on else 0)


def lanczos_graph(policy: int) -> int:
    """Test hook: single-sector Lanczos steps replayed from a CUDA graph (-1
    for sectors of at most 2^22 states, 0 never, 1 always); returns the
    previous policy."""
    return _lib.edx_lanczos_graph(policy)


INDEX_POLICIES = {"auto": 0, "hash": 1, "bucket": 2}


def index_policy(policy: str) -> None:
    """Test hook: the index later basis builds make -- "auto" (the bucketed
    index for large sectors), "hash" (always the hash index) or "bucket" (the
    bucketed index wherever its 64-bit entry can hold the key)."""
    _lib.edx_index_policy(INDEX_POLICIES[policy])


def basis_bucket(basis: Basis):
    """(present, log2 bucket count, stashed keys) of a basis's bucketed index."""
    bb, ns = _i32(0), ctypes.c_uint32(0)
    r = _lib.edx_basis_bucket(basis.handle, ctypes.byref(bb), ctypes.byref(ns))
    return bool(r == 1), bb.value, ns.value


PEAK_KINDS = {"int32_mix": 0, "fp64_fma": 1, "fp32_fma": 2, "gather32": 3}


def peak(kind: str, buf=None, stream=None):
    """Measured ceiling of this GPU (diagnostics): "int32_mix" integer ops/s of
    the group search's op mix (funnel shift, three-input logic, min, add),
    "fp64_fma" / "fp32_fma" fused multiply-adds per second, "gather32" random
    32-byte reads per second from the device tensor buf.  Returns (rate, ms)."""
    ms = _d(0.0)
    ptr = _ptr(buf) if buf is not None else ctypes.c_void_p(0)
    nbytes = buf.numel() * buf.element_size() if buf is not None else 0
    r = _lib.edx_peak(PEAK_KINDS[kind], ptr, nbytes, ctypes.byref(ms), _stream(stream))
    if r < 0:
        raise RuntimeError(f"edx_peak({kind}) failed")
    return r, ms.value


def _dtype_code(t):
    import torch
    return {torch.float64: ED_F64, torch.float32: ED_F32, torch.complex128: ED_C128,
            torch.complex64: ED_C64}[t.dtype]


def autotune(op: Operator, basis: Basis, x, y, nvec: int = 1, stream=None) -> dict:
    """ed_autotune: time the product variants for this basis on x (y is
    overwritten) and keep the fastest for later products."""
    r = TuneResult()
    _check(_lib.ed_autotune(op.handle, basis.handle, _ptr(x), _ptr(y), nvec, _dtype_code(x), ctypes.byref(r),
                            _stream(stream)), "ed_autotune")
    return {k: getattr(r, k) for k, _ in TuneResult._fields_}


def autotune_index(op: Operator, n_sites: int, n_up: int, spin_inversion: int, perms, chars, nvec: int = 1,
                   dtype: int = ED_F32, stream=None) -> dict:
    """ed_autotune_index: build the sector with each index, keep the faster one
    for later builds of sectors like it."""
    p = _host(perms, np.int32)
    c = _host(chars, np.float64)
    r = TuneResult()
    _check(_lib.ed_autotune_index(op.handle, n_sites, n_up, spin_inversion, p.shape[0],
                                  p.ctypes.data_as(_P), c.ctypes.data_as(_P), nvec, dtype, ctypes.byref(r),
                                  _stream(stream)), "ed_autotune_index")
    return {k: getattr(r, k) for k, _ in TuneResult._fields_}


def tune_reset() -> None:
    """Test hook: forget every tuned choice."""
    _lib.edx_tune_reset()


def multi_policy(policy: str) -> None:
    """Test hook: "auto", "batched" (always one launch) or "per_sector"."""
    _lib.edx_multi_policy({"auto": 0, "batched": 1, "per_sector": 2}[policy])


def inject_stall(on: bool) -> None:
    """Test hook: later batched launches wait on a gate that nothing opens
    (an injected producer stall); the bounded wait runs out and
    stream_status() returns ED_ERR_TIMEOUT (10)."""
    _lib.edx_inject_stall(1 if on else 0)


def count_nnz(op: Operator, basis: Basis) -> int:
    """Exact number of stored nonzeros of H in the sector (diagnostics)."""
    v = ctypes.c_ulonglong()
    if _lib.edx_count_nnz(op.handle, basis.handle, ctypes.byref(v)) != 0:
        raise RuntimeError("edx_count_nnz failed")
    return int(v.value)


def matvec_push(op: Operator, basis: Basis, x, y, stream=None):
    """Ablation: y = H x (one vector) by the transposed (push) form with atomic
    adds into y -- the paper's distributed product on one GPU.  The rounding
    of y depends on the order of the atomics, so repeated calls may differ in
    the last bits."""
    code = _DTYPE_CODE[str(x.dtype).replace("torch.", "")]
    if y.dtype != x.dtype or not (x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x and y must be contiguous with one dtype")
    _check(_lib.edx_matvec_push(op.handle, basis.handle, _ptr(x), _ptr(y), code, _stream(stream)),
           "edx_matvec_push")


KERNEL_POLICIES = {"auto": 0, "rowwise": 1, "term_parallel": 2}


def kernel_policy(policy: str) -> None:
    """Testing aid: which matvec kernel serves one vector (or a real block of 8)
    of an exchange-only operator: "auto" (one vector: term-parallel in single
    precision and for more than 32 sites, row-per-lane otherwise; blocks of 8
    vectors: term-parallel in fp32, row-per-lane in fp64), "rowwise" or
    "term_parallel" (both precisions).  Affects later launches."""
    _lib.edx_kernel_policy(KERNEL_POLICIES[policy])


def force_prefix_search(on: bool) -> None:
    """Testing aid: find indices through the prefix table and binary search even
    where the hash index exists.  Affects later launches."""
    _lib.edx_force_prefix_search(1 if on else 0)


def basis_hash(basis: Basis):
    """(hash index present, log2 buckets, largest bucket, 16-byte entries)."""
    hb, m, wd = _i32(), ctypes.c_uint32(), _i32()
    r = _lib.edx_basis_hash(basis.handle, ctypes.byref(hb), ctypes.byref(m), ctypes.byref(wd))
    return bool(r == 1), hb.value, m.value, bool(wd.value)


def basis_table(basis: Basis):
    """(prefix-table entries, largest bucket, probe steps of the index search)."""
    t, m, k = _u64(), ctypes.c_uint32(), _i32()
    _lib.edx_basis_table(basis.handle, ctypes.byref(t), ctypes.byref(m), ctypes.byref(k))
    return t.value, m.value, k.value


def basis_factored(basis: Basis):
    """(uses factored search, rotation order L, rotation step d, cosets)."""
    L, d, c = _i32(), _i32(), _i32()
    f = _lib.edx_basis_factored(basis.handle, ctypes.byref(L), ctypes.byref(d), ctypes.byref(c))
    return bool(f == 1), L.value, d.value, c.value


def matvec_multi(op: Operator, items, nvec: int = 1, stream=None):
    """y_s = H x_s for every (basis, x, y) in ``items`` in one launch; all x and y
    share one dtype."""
    items = list(items)
    if not items:
        return
    code = _DTYPE_CODE[str(items[0][1].dtype).replace("torch.", "")]
    arr = (Sector * len(items))()
    for k, (b, x, y) in enumerate(items):
        if x.dtype != items[0][1].dtype or y.dtype != x.dtype:
            raise ValueError("all x and y must share one dtype")
        if not (x.is_contiguous() and y.is_contiguous()):
            raise ValueError("x and y must be contiguous")
        arr[k] = Sector(b.handle, x.data_ptr() if x.numel() else None, y.data_ptr() if y.numel() else None)
    _check(_lib.ed_matvec_multi(op.handle, arr, len(items), nvec, code, _stream(stream)),
           "ed_matvec_multi")


@dataclass
class LanczosResult:
    e0: float
    steps: int
    matvecs: int
    ritz: float
    residual: float
    matvec_ms: float


def lanczos(op: Operator, basis: Basis, x0, steps: int, mode: int = ED_LANCZOS_F64, vec_out=None,
            stream=None) -> LanczosResult:
    e0 = ctypes.c_double()
    info = LanczosInfo()
    _check(_lib.ed_lanczos(op.handle, basis.handle, _ptr(x0), steps, mode, ctypes.byref(e0),
                           _ptr(vec_out) if vec_out is not None else None, ctypes.byref(info),
                           _stream(stream)), "ed_lanczos")
    return LanczosResult(e0.value, info.steps, info.matvecs, info.ritz, info.residual,
                         info.matvec_ms)


def lanczos_eigs(op: Operator, basis: Basis, x0, steps: int, n_eig: int, mode: int = ED_LANCZOS_F64,
                 vec_out=None, tol: float = 0.0, stream=None):
    """(lowest n_eig Ritz values as a list, LanczosResult of the lowest state);
    with tol > 0 an EDError (ED_ERR_NOT_CONVERGED) when the residual exceeds tol."""
    eigs = (ctypes.c_double * max(n_eig, 1))()
    info = LanczosInfo()
    _check(_lib.ed_lanczos_eigs(op.handle, basis.handle, _ptr(x0), steps, mode, n_eig, eigs, float(tol),
                                _ptr(vec_out) if vec_out is not None else None, ctypes.byref(info),
                                _stream(stream)), "ed_lanczos_eigs")
    return list(eigs[:n_eig]), LanczosResult(info.e0, info.steps, info.matvecs, info.ritz, info.residual,
                                             info.matvec_ms)


def lanczos_block(op: Operator, basis: Basis, x0, nvec: int, steps: int, mode: int = ED_LANCZOS_F32_MATVEC,
                  n_eig: int = 0, vec_out=None, stream=None):
    """Block Lanczos (ed_lanczos_block) from the [dim][nvec] fp64 start block x0:
    (lowest n_eig Ritz values as a list, LanczosResult with the refined energy)."""
    eigs = (ctypes.c_double * max(n_eig, 1))()
    e0 = _d(0.0)
    info = LanczosInfo()
    _check(_lib.ed_lanczos_block(op.handle, basis.handle, _ptr(x0), nvec, steps, mode, n_eig, eigs,
                                 ctypes.byref(e0), _ptr(vec_out) if vec_out is not None else None,
                                 ctypes.byref(info), _stream(stream)), "ed_lanczos_block")
    return list(eigs[:n_eig]), LanczosResult(info.e0, info.steps, info.matvecs, info.ritz, info.residual,
                                             info.matvec_ms)


def lanczos_multi(op: Operator, items, steps: int, mode: int = ED_LANCZOS_F64,
                  stream=None) -> list:
    """Lowest energy of every (basis, x0, vec_out or None) in ``items`` by one
    batched Lanczos run; x0 (and vec_out) are float64 for every sector, or
    complex128 for every sector."""
    items = list(items)
    if not items:
        return []
    code = _DTYPE_CODE[str(items[0][1].dtype).replace("torch.", "")]
    arr = (Sector * len(items))()
    for k, (b, x, v) in enumerate(items):
        if x.dtype != items[0][1].dtype or (v is not None and v.dtype != x.dtype):
            raise ValueError("all start and output vectors must share one dtype")
        if not x.is_contiguous() or (v is not None and not v.is_contiguous()):
            raise ValueError("vectors must be contiguous")
        arr[k] = Sector(b.handle, x.data_ptr(), v.data_ptr() if v is not None else None)
    e0 = (ctypes.c_double * len(items))()
    info = (LanczosInfo * len(items))()
    _check(_lib.ed_lanczos_multi(op.handle, arr, len(items), steps, mode, code, e0, info,
                                 _stream(stream)), "ed_lanczos_multi")
    return [LanczosResult(e0[k], info[k].steps, info[k].matvecs, info[k].ritz, info[k].residual,
                          info[k].matvec_ms) for k in range(len(items))]
