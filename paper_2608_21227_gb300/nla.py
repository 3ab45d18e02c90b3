"""Python binding of the C ABI in include/nla.h (argument marshalling only).

Every step of the computation runs in libnla.so's CUDA kernels; this module
only turns torch tensors into pointers, sizes and streams.  If the library
has not been built, every call raises: there is no CPU fallback.

Matrix convention: a 2-D CUDA tensor is handed to the library as the
column-major matrix it is in memory.  A Fortran-ordered (m, n) tensor (strides
(1, m)) is the m x n matrix itself; a C-contiguous (r, c) tensor is the
column-major c x r matrix A^T, which has the same singular values.  Either
way ``gesvd_vals(A)`` returns the singular values of A.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libnla.so")

F64, F32 = 0, 1
UPD_NATIVE, UPD_TF32, UPD_BF16, UPD_TF32X3, UPD_BF16X3 = 0, 1, 2, 3, 4
STATUS = {0: "NLA_OK", 1: "NLA_ERR_ARG", 2: "NLA_ERR_CUDA", 3: "NLA_ERR_CONFIG",
          4: "NLA_ERR_WORKSPACE", 5: "NLA_ERR_TIMEOUT", 6: "NLA_ERR_NOCONV", 7: "NLA_ERR_UNSUPPORTED"}


class NLAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Cfg(ctypes.Structure):
    _fields_ = [("band", ctypes.c_int), ("tile", ctypes.c_int), ("threads", ctypes.c_int),
                ("cols_per_block", ctypes.c_int), ("unroll", ctypes.c_int)]

    @classmethod
    def make(cls, band=0, tile=0, threads=0, cols_per_block=0, unroll=0):
        return cls(int(band), int(tile), int(threads), int(cols_per_block), int(unroll))

    def as_tuple(self):
        return (self.band, self.tile, self.threads, self.cols_per_block, self.unroll)


class Opts(ctypes.Structure):
    _fields_ = [("update", ctypes.c_int), ("cfg", ctypes.POINTER(Cfg)), ("preserve_a", ctypes.c_int)]


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_i = ctypes.c_int
_sz = ctypes.c_size_t
_psz = ctypes.POINTER(ctypes.c_size_t)
_popts = ctypes.POINTER(Opts)

_SIGNATURES = {
    "nla_gesvd_vals_workspace": [_i, _i, _i, _popts, _psz],
    "nla_gesvd_vals": [_i, _i, _i, _vp, _i, _vp, _vp, _sz, _vp, _popts, _vp],
    "nla_gesvd_vals_batched_workspace": [_i, _i, _i, _i, _psz],
    "nla_gesvd_vals_batched": [_i, _i, _vp, _vp, _vp, _vp, _vp, _i, _i, _vp, _sz, _vp, _popts, _vp],
    "nla_gebrd_band_workspace": [_i, _i, _i, _i, _popts, _psz],
    "nla_gebrd_band": [_i, _i, _i, _i, _vp, _i, _vp, _vp, _vp, _sz, _vp, _popts, _vp],
    "nla_band_extract": [_i, _i, _i, _vp, _i, _vp, _i, _vp],
    "nla_band2bd_workspace": [_i, _i, _i, _psz],
    "nla_band2bd": [_i, _i, _i, _vp, _i, _vp, _vp, _vp, _sz, _vp, _popts, _vp],
    "nla_bdsvd_vals_workspace": [_i, _psz],
    "nla_bdsvd_vals": [_i, _vp, _vp, _vp, _i, _vp, _sz, _vp, _vp],
    "nla_wait_selftest": [_i, _i, _vp, _vp],
}


def lib():
    """The loaded libnla.so.  Raises if the CUDA library was not built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libnla.so not built ({LIB_PATH} missing): run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            L.nla_last_error.restype = ctypes.c_char_p
            L.nla_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(st: int):
    if st != 0:
        raise NLAError(st, lib().nla_last_error().decode())


def _dtype_code(t) -> int:
    import torch

    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _stream_ptr(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _opts(update=UPD_NATIVE, cfg=None, preserve_a=False):
    o = Opts()
    o.update = int(update)
    o.preserve_a = int(bool(preserve_a))
    if cfg is not None:
        if not isinstance(cfg, Cfg):
            cfg = Cfg.make(*cfg) if isinstance(cfg, (tuple, list)) else Cfg.make(**cfg)
        o._cfg_keep = cfg  # keep alive
        o.cfg = ctypes.pointer(cfg)
    return o


def col_major_view(A):
    """(m, n, lda) of the column-major matrix a 2-D tensor holds in memory."""
    if A.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    r, c = A.shape
    s0, s1 = A.stride()
    if s0 == 1 and (s1 >= max(r, 1) or c <= 1):
        return r, c, max(s1, r, 1)  # Fortran order: the matrix itself
    if s1 == 1 and (s0 >= max(c, 1) or r <= 1):
        return c, r, max(s0, c, 1)  # C order: column-major A^T
    raise ValueError("tensor must have unit stride in one dimension")


def gesvd_vals_workspace(m, n, dtype_code, update=UPD_NATIVE, cfg=None, preserve_a=False) -> int:
    o = _opts(update, cfg, preserve_a)
    b = ctypes.c_size_t(0)
    _check(lib().nla_gesvd_vals_workspace(int(m), int(n), int(dtype_code), ctypes.byref(o), ctypes.byref(b)))
    return int(b.value)


def plan_cfg(m, n, dtype_code, side=0, update=UPD_NATIVE, cfg=None):
    """(band, tile, threads, cols_per_block, unroll) that gesvd_vals would use."""
    L = lib()
    L.nla_plan_cfg.argtypes = [_i, _i, _i, _popts, _i, ctypes.POINTER(Cfg)]
    L.nla_plan_cfg.restype = ctypes.c_int
    o = _opts(update, cfg)
    out = Cfg()
    _check(L.nla_plan_cfg(int(m), int(n), int(dtype_code), ctypes.byref(o), int(side), ctypes.byref(out)))
    return out.as_tuple()


def workspace(nbytes, device="cuda"):
    import torch

    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def gesvd_vals(A, update=UPD_NATIVE, cfg=None, preserve_a=False, work=None, S=None, info=None, stream=None):
    """Singular values (descending) of the matrix held by the CUDA tensor A.

    Returns (S, info): S has min(m, n) entries of A's dtype; info is a device
    int32 tensor (0 = success).  A is overwritten unless preserve_a.
    """
    import torch

    m, n, lda = col_major_view(A)
    dt = _dtype_code(A)
    o = _opts(update, cfg, preserve_a)
    need = ctypes.c_size_t(0)
    _check(lib().nla_gesvd_vals_workspace(m, n, dt, ctypes.byref(o), ctypes.byref(need)))
    if work is None or work.numel() < need.value:
        work = workspace(need.value, A.device)
    if S is None:
        S = torch.empty(min(m, n), dtype=A.dtype, device=A.device)
    if info is None:
        info = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib().nla_gesvd_vals(m, n, dt, _vp(A.data_ptr()), lda, _vp(S.data_ptr()), _vp(work.data_ptr()),
                                work.numel(), _vp(info.data_ptr()), ctypes.byref(o), _stream_ptr(stream)))
    return S, info


class Batch:
    """Device-side description of a batch of FP32 matrices for gesvd_vals_batched.

    ``mats`` is a list of CUDA float32 tensors; each is handed over as the
    column-major matrix it holds in memory (see col_major_view)."""

    def __init__(self, mats, device="cuda"):
        import torch

        views = [col_major_view(a) for a in mats]
        self.mats = mats
        self.m = torch.tensor([v[0] for v in views], dtype=torch.int32, device=device)
        self.n = torch.tensor([v[1] for v in views], dtype=torch.int32, device=device)
        self.lda = torch.tensor([v[2] for v in views], dtype=torch.int32, device=device)
        self.ptrs = torch.tensor([a.data_ptr() for a in mats], dtype=torch.int64, device=device)
        self.S = [torch.empty(min(v[0], v[1]), dtype=torch.float32, device=device) for v in views]
        self.sptrs = torch.tensor([s.data_ptr() for s in self.S], dtype=torch.int64, device=device)
        self.info = torch.zeros(len(mats), dtype=torch.int32, device=device)
        self.max_m = max([max(v[0], v[1]) for v in views] + [1])  # bounds max(m_i, n_i)
        self.max_n = max([min(v[0], v[1]) for v in views] + [1])  # bounds min(m_i, n_i)
        need = ctypes.c_size_t(0)
        _check(lib().nla_gesvd_vals_batched_workspace(len(mats), F32, self.max_m, self.max_n, ctypes.byref(need)))
        self.work = workspace(need.value, device)


def gesvd_vals_batched(batch, stream=None):
    """Singular values of every matrix of a Batch (one persistent launch); returns (list of S, info)."""
    _check(lib().nla_gesvd_vals_batched(len(batch.mats), F32, _vp(batch.m.data_ptr()), _vp(batch.n.data_ptr()),
                                        _vp(batch.lda.data_ptr()), _vp(batch.ptrs.data_ptr()),
                                        _vp(batch.sptrs.data_ptr()), batch.max_m, batch.max_n,
                                        _vp(batch.work.data_ptr()), batch.work.numel(), _vp(batch.info.data_ptr()),
                                        None, _stream_ptr(stream)))
    return batch.S, batch.info


def gebrd_band(A, band, update=UPD_NATIVE, cfg=None, work=None, stream=None):
    """Stage 1 in place on the column-major m x n matrix A (m >= n).  Returns (tauq, taup, info)."""
    import torch

    m, n, lda = col_major_view(A)
    dt = _dtype_code(A)
    o = _opts(update, cfg)
    need = ctypes.c_size_t(0)
    _check(lib().nla_gebrd_band_workspace(m, n, int(band), dt, ctypes.byref(o), ctypes.byref(need)))
    if work is None or work.numel() < need.value:
        work = workspace(need.value, A.device)
    nt = (n + band - 1) // band * band if n else 1
    tauq = torch.zeros(nt, dtype=A.dtype, device=A.device)
    taup = torch.zeros(nt, dtype=A.dtype, device=A.device)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib().nla_gebrd_band(m, n, int(band), dt, _vp(A.data_ptr()), lda, _vp(tauq.data_ptr()),
                                _vp(taup.data_ptr()), _vp(work.data_ptr()), work.numel(), _vp(info.data_ptr()),
                                ctypes.byref(o), _stream_ptr(stream)))
    return tauq, taup, info


def band_extract(A, band, stream=None):
    """Compact band storage (3*band+1 rows) of the leading n x n upper band of A."""
    import torch

    m, n, lda = col_major_view(A)
    n = min(m, n)
    ldab = 3 * band + 1
    ABt = torch.empty(n, ldab, dtype=A.dtype, device=A.device)  # column-major ldab x n
    _check(lib().nla_band_extract(n, int(band), _dtype_code(A), _vp(A.data_ptr()), lda, _vp(ABt.data_ptr()),
                                  ldab, _stream_ptr(stream)))
    return ABt


def band2bd(ABt, band, stream=None):
    """Bulge-chase the band storage ABt (tensor (n, ldab)) in place; returns (d, e, info) in FP64."""
    import torch

    n, ldab = ABt.shape
    need = ctypes.c_size_t(0)
    dt = _dtype_code(ABt)
    _check(lib().nla_band2bd_workspace(n, int(band), dt, ctypes.byref(need)))
    work = workspace(need.value, ABt.device)
    d = torch.empty(max(n, 1), dtype=torch.float64, device=ABt.device)
    e = torch.empty(max(n, 1), dtype=torch.float64, device=ABt.device)
    info = torch.zeros(1, dtype=torch.int32, device=ABt.device)
    _check(lib().nla_band2bd(n, int(band), dt, _vp(ABt.data_ptr()), ldab, _vp(d.data_ptr()), _vp(e.data_ptr()),
                             _vp(work.data_ptr()), work.numel(), _vp(info.data_ptr()), None, _stream_ptr(stream)))
    return d[:n], e[: max(n - 1, 0)], info


def wait_selftest(mode, budget_us, stream=None):
    """Run the failure-detection self-test (a bounded wait on something that never
    happens); returns the device info word (-NLA_ERR_TIMEOUT when the wait gave up)."""
    import torch

    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    _check(lib().nla_wait_selftest(int(mode), int(budget_us), _vp(info.data_ptr()), _stream_ptr(stream)))
    return info


def bdsvd_vals(d, e, dtype=None, stream=None):
    """Singular values (descending) of the upper bidiagonal (d, e) given as FP64 CUDA tensors."""
    import torch

    n = d.numel()
    dtype = dtype or torch.float64
    S = torch.empty(max(n, 1), dtype=dtype, device=d.device)
    info = torch.zeros(1, dtype=torch.int32, device=d.device)
    dt = F64 if dtype == torch.float64 else F32
    e_ptr = e.data_ptr() if e.numel() else d.data_ptr()
    need = ctypes.c_size_t(0)
    _check(lib().nla_bdsvd_vals_workspace(n, ctypes.byref(need)))
    work = workspace(need.value, d.device)
    _check(lib().nla_bdsvd_vals(n, _vp(d.data_ptr()), _vp(e_ptr), _vp(S.data_ptr()), dt, _vp(work.data_ptr()),
                                work.numel(), _vp(info.data_ptr()), _stream_ptr(stream)))
    return S[:n], info


class TraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int), ("total_ms", ctypes.c_double)]


def trace_enable(on=True):
    L = lib()
    L.nla_trace_enable.argtypes = [ctypes.c_int]
    _check(L.nla_trace_enable(int(bool(on))))


def trace_reset():
    lib().nla_trace_reset()


def trace_read():
    """{kernel class: (launches, total device ms)} since the last reset (synchronises)."""
    L = lib()
    L.nla_trace_read.argtypes = [ctypes.POINTER(TraceEntry), ctypes.c_int]
    L.nla_trace_read.restype = ctypes.c_int
    buf = (TraceEntry * 32)()
    k = L.nla_trace_read(buf, 32)
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(min(k, 32))}


def version() -> str:
    return lib().nla_version().decode()
