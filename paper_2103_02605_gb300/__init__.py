"""GB300-native f-circulant matrix-vector products without FFT.

Thin Python binding of the C ABI in ``include/fcirc.h`` / ``include/fcirc_plan.h``
(``_build/libfcirc.so``): argument marshalling only, every step of the
computation runs in the library's CUDA kernels.  PyTorch provides device
memory and streams.  If the shared library has not been built the calls
raise; there is no fallback path.

Tensors may live on the current CUDA device or in host memory.  With
device tensors the calls only enqueue work on ``stream`` (default: torch's
current stream).  With pageable host tensors they return when the results
are in place; with pinned host tensors only they are asynchronous like
``cudaMemcpyAsync`` -- synchronise ``stream`` before reading the outputs.

Method: Rosowski, "On Fast Computation of a Circulant Matrix-Vector Product"
(arXiv 2103.02605), Algorithm 1 / Theorem 1 (Section 2) and the
applications of Section 3.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

__all__ = [
    "FcircError", "library_path", "load",
    "fcirc_matvec", "fcirc_matvec_t", "fcirc_toeplitz_matvec", "fcirc_matvec_gf", "GF_P", "fcirc_matvec_ssa", "fcirc_matvec_noalloc", "APlan", "poly_mul_int", "bigint_mul",
    "fcirc_matvec_c64", "fcirc_matvec_backward", "fcirc_layer",
    "fcirc_matvec_batched", "batched_autotune", "BatchedGraph", "batched_partition", "batched_shard",
    "sync_status", "release", "set_checks",
    "nth_root", "node_twiddle", "leaf_param", "twiddle_from_factor",
    "prof_start", "prof_stop", "prof_report", "prof_launches", "prof_mul_probe",
    "PRIMES",
]

PRIMES = (998244353, 469762049, 167772161)
GF_P = (1 << 31) - 1   # the paper's field GF(p^2) = Z/pZ[sqrt 3]

_lock = threading.Lock()
_lib = None

_u32, _u64, _i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_vp = ctypes.c_void_p

_SIGNATURES = {
    "fcirc_matvec": ([_u32, _u32, _vp, _vp, _vp, _u64, _vp], _i32),
    "fcirc_matvec_noalloc": ([_u32, _u32, _vp, _vp, _vp, _u64, _vp], _i32),
    "fcirc_matvec_t": ([_u32, _u32, _vp, _vp, _vp, _u64, _vp], _i32),
    "fcirc_toeplitz_matvec": ([_u32, _vp, _vp, _vp, _u64, _vp], _i32),
    "fcirc_matvec_gf": ([_vp, _vp, _vp, _u32, _u32, _u64, _u64, _vp], _i32),
    "fcirc_matvec_ssa": ([_vp, _vp, _vp, _u32, _u32, _u64, _u64, _vp], _i32),
    "fcirc_aplan_create": ([_u32, _u32, _vp, _u64, _vp, ctypes.POINTER(_vp)], _i32),
    "fcirc_matvec_aplan": ([_vp, _vp, _vp, _vp], _i32),
    "fcirc_aplan_destroy": ([_vp], _i32),
    "poly_mul_int": ([_vp, _u64, _vp, _u64, _vp, _vp], _i32),
    "bigint_mul": ([_vp, _u64, _vp, _u64, _vp, _vp], _i32),
    "fcirc_matvec_c64": ([_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _u64, _u64, _vp], _i32),
    "fcirc_matvec_batched": ([_u32, _vp, _vp, _vp, _vp, _vp, _u32, _vp], _i32),
    "fcirc_batched_autotune": ([_u32, _vp, _vp, _vp, _vp, _vp, _u32, _vp, ctypes.POINTER(ctypes.c_int)], _i32),
    "fcirc_batched_config": ([ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], _i32),
    "fcirc_matvec_batched_graph": ([_u32, _vp, _vp, _vp, _vp, _vp, _u32, _u64, _vp, ctypes.POINTER(_vp)], _i32),
    "fcirc_graph_launch": ([_vp, _vp], _i32),
    "fcirc_graph_destroy": ([_vp], _i32),
    "fcirc_batched_partition": ([_vp, _u32, _u32, _u32, _vp, ctypes.POINTER(_u32), _vp], _i32),
    "fcirc_matvec_backward": ([_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _vp, _vp, _u64, _u64, _vp],
                              _i32),
    "fcirc_sync_status": ([_vp], _i32),
    "fcirc_error_string": ([_i32], ctypes.c_char_p),
    "fcirc_last_error": ([], ctypes.c_char_p),
    "fcirc_release": ([], _i32),
    "fcirc_set_checks": ([_i32], _i32),
    "fcirc_debug_fail_alloc": ([_i32], _i32),
    "fcirc_debug_spin_limit": ([ctypes.c_longlong], _i32),
    "fcirc_nth_root": ([_u32, _u32, _u32, ctypes.POINTER(_u32)], _i32),
    "fcirc_gf_nth_root": ([_u32, _u32, _u32, ctypes.POINTER(_u32), ctypes.POINTER(_u32)], _i32),
    "fcirc_node_twiddle": ([_u32, _u32, _u64, _u32, _u64, ctypes.POINTER(_u32), ctypes.POINTER(_u32)], _i32),
    "fcirc_leaf_param": ([_u32, _u32, _u64, _u64, ctypes.POINTER(_u32)], _i32),
    "fcirc_twiddle_from_factor": ([_u32, _u32, _u32, ctypes.POINTER(_u32), ctypes.POINTER(_u32)], _i32),
    "fcirc_prof_start": ([], _i32),
    "fcirc_prof_stop": ([], _i32),
    "fcirc_prof_report": ([ctypes.c_char_p, _u64], _i32),
    "fcirc_prof_launches": ([], _u64),
    "fcirc_prof_mul_probe": ([ctypes.c_int, _u32, _u32, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_double)], _i32),
}


class FcircError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


def library_path() -> str:
    return _build.LIB


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(
                    f"{path} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(path)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        L = load()
        name = L.fcirc_error_string(status).decode()
        detail = L.fcirc_last_error().decode()
        raise FcircError(status, f"{what}: {name} ({detail})")


def _stream_handle(stream, *tensors) -> int:
    import torch
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    if any(t.is_cuda for t in tensors):
        return int(torch.cuda.current_stream(tensors[0].device).cuda_stream)
    return 0


def _u32_tensor(t, name):
    import torch
    if t.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
        raise TypeError(f"{name} must be int32/uint32 holding residues, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _check_out(out, shape, dtypes, name="out"):
    """A caller's output tensor: one of `dtypes`, contiguous, of exactly
    `shape` (the library writes that many elements and no more)."""
    if out.dtype not in dtypes:
        raise TypeError(f"{name} must be one of {[str(d) for d in dtypes]}, got {out.dtype}")
    if not out.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(out.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(out.shape)}")
    return out


def _dtypes(*names):
    import torch
    return tuple(getattr(torch, n) for n in names if hasattr(torch, n))


# -- entry points --------------------------------------------------------------

def fcirc_matvec(p: int, f: int, a, x, out=None, stream=None):
    """c = A x over Z/pZ for the f-circulant A with row vector a (Definition 2,
    Algorithm 1).  a, x: 1-D int32/uint32 tensors of residues in [0, p),
    on the current CUDA device or on the host."""
    import torch
    _u32_tensor(a, "a")
    _u32_tensor(x, "x")
    if a.shape != x.shape or a.dim() != 1:
        raise ValueError("a and x must be 1-D of the same length")
    if out is None:
        out = torch.empty_like(a)
    _check_out(out, a.shape, _dtypes("int32", "uint32"))
    st = _stream_handle(stream, a, x, out)
    _check(load().fcirc_matvec(p, f % p, a.data_ptr(), x.data_ptr(), out.data_ptr(), a.numel(), st),
           "fcirc_matvec")
    return out


def fcirc_matvec_t(p: int, f: int, a, x, out=None, stream=None):
    """c = A^T x for the f-circulant A with row vector a (include/fcirc.h):
    the column convention, a(z) x(z) mod (z^n - f).  Same arguments as
    fcirc_matvec."""
    import torch
    _u32_tensor(a, "a")
    _u32_tensor(x, "x")
    if a.shape != x.shape or a.dim() != 1:
        raise ValueError("a and x must be 1-D of the same length")
    if out is None:
        out = torch.empty_like(a)
    _check_out(out, a.shape, _dtypes("int32", "uint32"))
    st = _stream_handle(stream, a, x, out)
    _check(load().fcirc_matvec_t(p, f % p, a.data_ptr(), x.data_ptr(), out.data_ptr(), a.numel(), st),
           "fcirc_matvec_t")
    return out


def fcirc_toeplitz_matvec(p: int, t, x, out=None, stream=None):
    """c = T x for the n x n Toeplitz matrix T[i][j] = t[j - i + n - 1]
    (t: 2n - 1 diagonals, lowest first), by Corollary 1's embedding into a
    power-of-two circulant (include/fcirc.h)."""
    import torch
    _u32_tensor(t, "t")
    _u32_tensor(x, "x")
    n = x.numel()
    if x.dim() != 1 or t.dim() != 1 or t.numel() != 2 * n - 1:
        raise ValueError("x must be 1-D of length n and t of length 2n - 1")
    if out is None:
        out = torch.empty_like(x)
    _check_out(out, x.shape, _dtypes("int32", "uint32"))
    st = _stream_handle(stream, t, x, out)
    _check(load().fcirc_toeplitz_matvec(p, t.data_ptr(), x.data_ptr(), out.data_ptr(), n, st),
           "fcirc_toeplitz_matvec")
    return out


def fcirc_matvec_gf(a, x, f=(1, 0), out=None, stream=None):
    """Batched f-circulant products over GF(p^2) = Z/pZ[sqrt 3], p = 2^31 - 1
    (the paper's field).  a, x: int32/uint32 tensors of shape (batch, n, 2)
    holding (re, im) = re + im sqrt 3; f = (f_re, f_im).  8 <= n <= 4096."""
    import torch
    for t, nm in ((a, "a"), (x, "x")):
        _u32_tensor(t, nm)
        if t.dim() != 3 or t.shape[2] != 2:
            raise ValueError(f"{nm} must have shape (batch, n, 2)")
    if a.shape != x.shape:
        raise ValueError("a and x must have the same shape")
    batch, n = a.shape[0], a.shape[1]
    if out is None:
        out = torch.empty_like(a)
    _check_out(out, a.shape, _dtypes("int32", "uint32"))
    st = _stream_handle(stream, a, x, out)
    _check(load().fcirc_matvec_gf(a.data_ptr(), x.data_ptr(), out.data_ptr(), int(f[0]) % GF_P, int(f[1]) % GF_P,
                                  n, batch, st), "fcirc_matvec_gf")
    return out


def fcirc_matvec_ssa(a, x, K: int, f_exp: int = 0, out=None, stream=None):
    """Batched f-circulant products over Z/(2^K + 1), f = 2^f_exp, K = 64 or
    128 (include/fcirc.h).  a, x: int64/uint64 tensors of shape
    (batch, n, K/64 + 1): K/64 little-endian words and a top word (value
    w + top 2^K, at most 2^K)."""
    import torch
    wpe = K // 64 + 1
    for t, nm in ((a, "a"), (x, "x")):
        if t.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)):
            raise TypeError(f"{nm} must be a 64-bit integer tensor")
        if t.dim() != 3 or t.shape[2] != wpe or not t.is_contiguous():
            raise ValueError(f"{nm} must be contiguous of shape (batch, n, {wpe})")
    if a.shape != x.shape:
        raise ValueError("a and x must have the same shape")
    if out is None:
        out = torch.empty_like(a)
    _check_out(out, a.shape, _dtypes("int64", "uint64"))
    st = _stream_handle(stream, a, x, out)
    _check(load().fcirc_matvec_ssa(a.data_ptr(), x.data_ptr(), out.data_ptr(), K, f_exp, a.shape[1], a.shape[0], st),
           "fcirc_matvec_ssa")
    return out


def fcirc_matvec_noalloc(p: int, f: int, a, x, out, stream=None):
    """fcirc_matvec for callers that cannot let the library allocate: a, x and
    out are device tensors (out preallocated), n <= 2^20; the library works
    in a fixed array it holds from load time (see include/fcirc.h)."""
    _u32_tensor(a, "a")
    _u32_tensor(x, "x")
    _u32_tensor(out, "out")
    if a.shape != x.shape or a.shape != out.shape or a.dim() != 1:
        raise ValueError("a, x and out must be 1-D of the same length")
    st = _stream_handle(stream, a, x, out)
    _check(load().fcirc_matvec_noalloc(p, f % p, a.data_ptr(), x.data_ptr(), out.data_ptr(), a.numel(), st),
           "fcirc_matvec_noalloc")
    return out


class APlan:
    """A fixed f-circulant matrix for many products (include/fcirc.h,
    fcirc_aplan_*): the row vector's tree of Algorithm 1 runs once here, and
    each ``matvec`` runs the vector's tree, the leaves and the recombination.
    ``a``: uint32 row vector (device or host tensor), values < p.  The plan
    owns n * 4 bytes of device memory until ``destroy`` (or garbage
    collection, or the end of a ``with`` block)."""

    def __init__(self, p: int, f: int, a, stream=None):
        _u32_tensor(a, "a")
        if a.dim() != 1:
            raise ValueError("a must be 1-D")
        self.p, self.f, self.n = p, f % p, a.numel()
        h = _vp()
        _check(load().fcirc_aplan_create(p, f % p, a.data_ptr(), a.numel(), _stream_handle(stream, a),
                                         ctypes.byref(h)), "fcirc_aplan_create")
        self._h = h

    def matvec(self, x, out=None, stream=None):
        import torch
        if self._h is None:
            raise ValueError("plan destroyed")
        _u32_tensor(x, "x")
        if x.dim() != 1 or x.numel() != self.n:
            raise ValueError(f"x must be 1-D of length {self.n}")
        if out is None:
            out = torch.empty_like(x)
        _check_out(out, x.shape, _dtypes("int32", "uint32"))
        st = _stream_handle(stream, x, out)
        _check(load().fcirc_matvec_aplan(self._h, x.data_ptr(), out.data_ptr(), st), "fcirc_matvec_aplan")
        return out

    def destroy(self):
        if getattr(self, "_h", None) is not None:
            _check(load().fcirc_aplan_destroy(self._h), "fcirc_aplan_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def poly_mul_int(P, Q, out=None, stream=None):
    """Exact product of integer polynomials with uint16 coefficients
    (Section 3.1).  P, Q: 1-D int16/uint16 tensors (bit patterns of uint16);
    returns int64 coefficients of length len(P) + len(Q) - 1."""
    import torch
    for t, nm in ((P, "P"), (Q, "Q")):
        if t.dtype not in (torch.int16, getattr(torch, "uint16", torch.int16)):
            raise TypeError(f"{nm} must be a 16-bit tensor, got {t.dtype}")
        if not t.is_contiguous() or t.dim() != 1:
            raise ValueError(f"{nm} must be 1-D contiguous")
    if P.numel() == 0 or Q.numel() == 0:
        raise ValueError("P and Q must not be empty")
    nout = P.numel() + Q.numel() - 1
    if out is None:
        out = torch.empty(nout, dtype=torch.int64, device=P.device)
    _check_out(out, (nout,), _dtypes("int64", "uint64"))
    st = _stream_handle(stream, P, Q, out)
    _check(load().poly_mul_int(P.data_ptr(), P.numel(), Q.data_ptr(), Q.numel(), out.data_ptr(), st),
           "poly_mul_int")
    return out


def bigint_mul(A, B, out=None, stream=None):
    """Product of two unsigned integers given as little-endian 16-bit limbs
    (Section 3.2).  A, B: 1-D int16/uint16 tensors; returns len(A) + len(B)
    limbs (int16 tensor holding the uint16 bit patterns)."""
    import torch
    for t, nm in ((A, "A"), (B, "B")):
        if t.dtype not in (torch.int16, getattr(torch, "uint16", torch.int16)):
            raise TypeError(f"{nm} must be a 16-bit tensor, got {t.dtype}")
        if not t.is_contiguous() or t.dim() != 1:
            raise ValueError(f"{nm} must be 1-D contiguous")
    if A.numel() == 0 or B.numel() == 0:
        raise ValueError("A and B must not be empty")
    if out is None:
        out = torch.empty(A.numel() + B.numel(), dtype=torch.int16, device=A.device)
    _check_out(out, (A.numel() + B.numel(),), _dtypes("int16", "uint16"))
    st = _stream_handle(stream, A, B, out)
    _check(load().bigint_mul(A.data_ptr(), A.numel(), B.data_ptr(), B.numel(), out.data_ptr(), st),
           "bigint_mul")
    return out


def _batched_args(f, offsets, a, x, out):
    import torch
    for t, nm, dt in ((f, "f", (torch.int32,)), (a, "a", (torch.int32,)), (x, "x", (torch.int32,)),
                      (offsets, "offsets", (torch.int64,))):
        if t.dtype not in dt + tuple(getattr(torch, u) for u in ("uint32", "uint64") if hasattr(torch, u)):
            raise TypeError(f"{nm}: unexpected dtype {t.dtype}")
        if not t.is_contiguous() or t.dim() != 1:
            raise ValueError(f"{nm} must be 1-D contiguous")
    if offsets.numel() != f.numel() + 1:
        raise ValueError("offsets must hold one more entry than f (count + 1)")
    if x.shape != a.shape:
        raise ValueError("a and x must have the same length")
    if out is None:
        out = torch.empty_like(a)
    return _check_out(out, a.shape, _dtypes("int32", "uint32"))


def fcirc_matvec_batched(p: int, f, offsets, a, x, out=None, stream=None):
    """Batched products c_i = A_i x_i over Z/pZ, instance i on
    [offsets[i], offsets[i+1]) of the packed a, x, out (int32/uint32 residues;
    offsets int64).  One persistent launch; see include/fcirc.h."""
    out = _batched_args(f, offsets, a, x, out)
    st = _stream_handle(stream, a, x, out)
    _check(load().fcirc_matvec_batched(p, f.data_ptr(), offsets.data_ptr(), a.data_ptr(), x.data_ptr(),
                                       out.data_ptr(), f.numel(), st), "fcirc_matvec_batched")
    return out


def batched_autotune(p: int, f, offsets, a, x, out=None, stream=None):
    """Times every launch configuration on these arguments and keeps the
    fastest for this batch shape; returns (index, ctas_per_sm, tile_log)."""
    out = _batched_args(f, offsets, a, x, out)
    st = _stream_handle(stream, a, x, out)
    ch = ctypes.c_int(-1)
    _check(load().fcirc_batched_autotune(p, f.data_ptr(), offsets.data_ptr(), a.data_ptr(), x.data_ptr(),
                                         out.data_ptr(), f.numel(), st, ctypes.byref(ch)), "fcirc_batched_autotune")
    cps, tl = ctypes.c_int(), ctypes.c_int()
    _check(load().fcirc_batched_config(ch.value, ctypes.byref(cps), ctypes.byref(tl)), "fcirc_batched_config")
    return ch.value, cps.value, tl.value


def batched_partition(offsets, nranks: int, rank: int):
    """The instances of `rank` when a batch is split over `nranks` ranks
    (include/fcirc.h, fcirc_batched_partition: longest processing time first
    on n log2 n, the same on every rank).  offsets: host uint64/int64
    sequence of count + 1 offsets.  Returns (members, loads): the ascending
    instance indices of `rank` (numpy uint32) and every rank's total cost
    (numpy float64).  Host only."""
    import numpy as np
    off = np.ascontiguousarray(np.asarray(offsets).astype(np.uint64, copy=False))
    if off.ndim != 1 or off.size < 1:
        raise ValueError("offsets must be a 1-D sequence of count + 1 entries")
    count = off.size - 1
    members = np.empty(max(count, 1), dtype=np.uint32)
    loads = np.empty(max(int(nranks), 1), dtype=np.float64)
    nm = _u32()
    _check(load().fcirc_batched_partition(off.ctypes.data, count, int(nranks), int(rank), members.ctypes.data,
                                          ctypes.byref(nm), loads.ctypes.data), "fcirc_batched_partition")
    return members[:nm.value].copy(), loads[:int(nranks)].copy()


def batched_shard(members, offsets, *arrays):
    """Packs the instances `members` of a batch back to back: returns the
    shard's offsets (uint64, len(members) + 1) and, for each packed array
    (instance i on [offsets[i], offsets[i+1])) or per-instance array (one
    entry per instance) given, the shard's copy.  Host (numpy) arrays."""
    import numpy as np
    off = np.asarray(offsets).astype(np.uint64, copy=False)
    members = np.asarray(members, dtype=np.int64)
    count = off.size - 1
    sizes = (off[1:] - off[:-1])[members]
    loc = np.zeros(members.size + 1, dtype=np.uint64)
    np.cumsum(sizes, out=loc[1:])
    total = int(off[-1])
    idx = None
    out = [loc]
    for arr in arrays:
        arr = np.asarray(arr)
        if arr.shape[0] == count and count != total:
            out.append(arr[members].copy())
            continue
        if arr.shape[0] != total:
            raise ValueError("an array is neither packed (offsets[-1] entries) nor per instance (count entries)")
        if idx is None:
            starts = off[:-1][members].astype(np.int64)
            idx = (np.repeat(starts - loc[:-1].astype(np.int64), sizes.astype(np.int64))
                   + np.arange(int(loc[-1]), dtype=np.int64))
        out.append(arr[idx].copy())
    return tuple(out)


class BatchedGraph:
    """The batched launch sequence captured into a CUDA graph for fixed device
    buffers (f, offsets, a, x, out); launch() replays it."""

    def __init__(self, p: int, f, offsets, a, x, out, total_n: int, stream=None):
        _batched_args(f, offsets, a, x, out)
        if total_n > a.numel():
            raise ValueError("total_n exceeds the packed arrays")
        st = _stream_handle(stream, a, x, out)
        h = _vp()
        _check(load().fcirc_matvec_batched_graph(p, f.data_ptr(), offsets.data_ptr(), a.data_ptr(), x.data_ptr(),
                                                 out.data_ptr(), f.numel(), total_n, st, ctypes.byref(h)),
               "fcirc_matvec_batched_graph")
        self._h = h
        self._keep = (f, offsets, a, x, out)

    def launch(self, stream=None):
        st = _stream_handle(stream, *self._keep[2:])
        _check(load().fcirc_graph_launch(self._h, st), "fcirc_graph_launch")

    def destroy(self):
        if self._h:
            load().fcirc_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _c64(t, name):
    import torch
    if t.dtype != torch.complex64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous complex64 tensor")
    return t


def fcirc_matvec_c64(a, x, f=1.0, out=None, stream=None):
    """Batched complex f-circulant product c = A x in FP32; a, x of shape
    (batch, n) or (n,), complex64."""
    import torch
    _c64(a, "a")
    _c64(x, "x")
    if a.shape != x.shape:
        raise ValueError("a and x must have the same shape")
    n = a.shape[-1]
    batch = a.numel() // n if n else 0
    if out is None:
        out = torch.empty_like(a)
    _c64(out, "out")
    if out.shape != a.shape:
        raise ValueError(f"out must have shape {tuple(a.shape)}")
    f = complex(f)
    st = _stream_handle(stream, a, x, out)
    _check(load().fcirc_matvec_c64(a.data_ptr(), x.data_ptr(), out.data_ptr(), f.real, f.imag, n, batch, st),
           "fcirc_matvec_c64")
    return out


def fcirc_matvec_backward(a, x, g, f=1.0, stream=None):
    """(grad_a, grad_x) of Re <g, A x> (PyTorch's complex convention)."""
    import torch
    for t, nm in ((a, "a"), (x, "x"), (g, "g")):
        _c64(t, nm)
    n = a.shape[-1]
    batch = a.numel() // n if n else 0
    ga = torch.empty_like(a)
    gx = torch.empty_like(x)
    f = complex(f)
    st = _stream_handle(stream, a, x, g)
    _check(load().fcirc_matvec_backward(a.data_ptr(), x.data_ptr(), g.data_ptr(), f.real, f.imag,
                                        ga.data_ptr(), gx.data_ptr(), n, batch, st), "fcirc_matvec_backward")
    return ga, gx


def _autograd_fn():
    import torch

    class FCircC64(torch.autograd.Function):
        """c = A x for f-circulant A with row vector a (complex FP32), with the
        hand-written adjoint as backward (see fcirc_matvec_backward)."""

        @staticmethod
        def forward(ctx, a, x, f):
            ctx.save_for_backward(a, x)
            ctx.f = f
            return fcirc_matvec_c64(a.contiguous(), x.contiguous(), f)

        @staticmethod
        def backward(ctx, g):
            a, x = ctx.saved_tensors
            ga, gx = fcirc_matvec_backward(a.contiguous(), x.contiguous(), g.contiguous(), ctx.f)
            return ga, gx, None

    return FCircC64


_FCIRC_FN = None


def fcirc_layer(a, x, f=1.0):
    """Differentiable complex f-circulant product (torch.autograd.Function)."""
    global _FCIRC_FN
    if _FCIRC_FN is None:
        _FCIRC_FN = _autograd_fn()
    return _FCIRC_FN.apply(a, x, complex(f))


def sync_status(stream=None) -> int:
    """Waits for the stream and returns the library's device status (0 = OK)."""
    import torch
    st = int(getattr(stream, "cuda_stream", stream)) if stream is not None else (
        int(torch.cuda.current_stream().cuda_stream) if torch.cuda.is_available() else 0)
    return int(load().fcirc_sync_status(st))


def set_checks(on: bool = True):
    """Input range checks before every product (include/fcirc.h,
    fcirc_set_checks); a violation shows up in sync_status()."""
    _check(load().fcirc_set_checks(1 if on else 0), "fcirc_set_checks")


def release():
    _check(load().fcirc_release(), "fcirc_release")


# -- launch tracing (include/fcirc_prof.h) ---------------------------------------

def prof_start():
    _check(load().fcirc_prof_start(), "fcirc_prof_start")


def prof_stop():
    _check(load().fcirc_prof_stop(), "fcirc_prof_stop")


def prof_report() -> dict:
    """{kernel name: (launches, total device ms)} since prof_start()."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().fcirc_prof_report(buf, len(buf)), "fcirc_prof_report")
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def prof_launches() -> int:
    return int(load().fcirc_prof_launches())


def prof_mul_probe(kind: int, ctas_per_sm: int = 4, iters: int = 4096):
    """(ms, multiplies per second) of the library's integer-multiply probe
    on the current device: kind 0 low-half, kind 1 high-half 32-bit
    multiplies (include/fcirc_prof.h)."""
    ms, rate = ctypes.c_double(), ctypes.c_double()
    _check(load().fcirc_prof_mul_probe(int(kind), int(ctas_per_sm), int(iters), ctypes.byref(ms),
                                       ctypes.byref(rate)), "fcirc_prof_mul_probe")
    return ms.value, rate.value


# -- host-side plan numbers (no GPU needed) -------------------------------------

def nth_root(p: int, f: int, log2k: int) -> int:
    r = _u32()
    _check(load().fcirc_nth_root(p, f, log2k, ctypes.byref(r)), "fcirc_nth_root")
    return r.value


def node_twiddle(p: int, f: int, n: int, level: int, j: int):
    s, si = _u32(), _u32()
    _check(load().fcirc_node_twiddle(p, f, n, level, j, ctypes.byref(s), ctypes.byref(si)),
           "fcirc_node_twiddle")
    return s.value, si.value


def leaf_param(p: int, f: int, n: int, j: int) -> int:
    v = _u32()
    _check(load().fcirc_leaf_param(p, f, n, j, ctypes.byref(v)), "fcirc_leaf_param")
    return v.value


def twiddle_from_factor(p: int, u: int, sigma: int):
    w, wp = _u32(), _u32()
    _check(load().fcirc_twiddle_from_factor(p, u, sigma, ctypes.byref(w), ctypes.byref(wp)),
           "fcirc_twiddle_from_factor")
    return w.value, wp.value
