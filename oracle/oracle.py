"""CPU oracle for the f-circulant product -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It loads ``fcirc_oracle.c`` (compiled
here with gcc + OpenMP) and exposes numpy-facing wrappers.  Nothing in it
shares code with the CUDA library, and the product never calls it.

Every routine is the plain dense definition (Definition 2 of the paper, the
row-vector convention of Section 1.2, schoolbook products for Section 3);
see the C file for the formulas.  Pins that tie each routine to something
other than itself live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fcirc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libfcirc_oracle.so")
_lock = threading.Lock()
_lib = None

u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
u16p = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
U32, U64 = ctypes.c_uint32, ctypes.c_uint64
F64 = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile the oracle shared object (host gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC",
                           "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_fcirc_matvec_mod.argtypes = [U32, U32, u32p, u32p, u32p, U64]
            L.oracle_fcirc_matvec_mod_rows.argtypes = [U32, U32, u32p, u32p, U64, u64p, U64, u32p]
            L.oracle_fcirc_matvec_t_mod.argtypes = [U32, U32, u32p, u32p, u32p, U64]
            L.oracle_toeplitz_matvec_mod.argtypes = [U32, u32p, u32p, u32p, U64]
            L.oracle_fcirc_matvec_gf.argtypes = [U32, U32, u32p, u32p, u32p, U64]
            L.oracle_fcirc_matvec_mod_batched.argtypes = [U32, u32p, u64p, u32p, u32p, u32p, U32]
            L.oracle_fcirc_matvec_c128.argtypes = [F64, F64, f64p, f64p, f64p, U64, U64]
            L.oracle_fcirc_grad_c128.argtypes = [F64, F64, f64p, f64p, f64p, f64p, f64p, U64, U64]
            L.oracle_poly_mul.argtypes = [u16p, U64, u16p, U64, i64p]
            L.oracle_poly_mul_coeffs.argtypes = [u16p, U64, u16p, U64, u64p, U64, i64p]
            L.oracle_bigint_mul.argtypes = [u16p, U64, u16p, U64, u16p]
            L.oracle_bigint_columns.argtypes = [u16p, U64, u16p, U64, u64p, U64, u64p]
            L.oracle_eval_u16_mod.argtypes = [u16p, U64, U64, U64]
            L.oracle_eval_u16_mod.restype = U64
            L.oracle_eval_i64_mod.argtypes = [i64p, U64, U64, U64]
            L.oracle_eval_i64_mod.restype = U64
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def _u32(v):
    return np.ascontiguousarray(v, dtype=np.uint32)


def _u16(v):
    return np.ascontiguousarray(v, dtype=np.uint16)


# -- f-circulant product mod p (Definition 2) --------------------------------

def fcirc_matvec_mod(p: int, f: int, a, x) -> np.ndarray:
    a, x = _u32(a), _u32(x)
    assert a.shape == x.shape and a.ndim == 1
    c = np.empty_like(a)
    lib().oracle_fcirc_matvec_mod(p, f % p, a, x, c, a.size)
    return c


def fcirc_matvec_t_mod(p: int, f: int, a, x) -> np.ndarray:
    """A^T x (column convention): a(z) x(z) mod (z^n - f), schoolbook."""
    a, x = _u32(a), _u32(x)
    assert a.shape == x.shape and a.ndim == 1
    c = np.empty_like(a)
    lib().oracle_fcirc_matvec_t_mod(p, f % p, a, x, c, a.size)
    return c


def toeplitz_matvec_mod(p: int, t, x) -> np.ndarray:
    """T x for T[i][j] = t[j - i + n - 1] (t: 2n - 1 diagonals), dense."""
    t, x = _u32(t), _u32(x)
    assert x.ndim == 1 and t.shape == (2 * x.size - 1,)
    c = np.empty_like(x)
    lib().oracle_toeplitz_matvec_mod(p, t, x, c, x.size)
    return c


GF_P = (1 << 31) - 1


def fcirc_matvec_gf(f, a, x) -> np.ndarray:
    """Over GF(p^2) = Z/pZ[sqrt 3], p = 2^31 - 1: a, x of shape (n, 2) or
    (batch, n, 2) holding (re, im); f = (f_re, f_im).  Dense definition."""
    a, x = _u32(a), _u32(x)
    assert a.shape == x.shape and a.shape[-1] == 2
    flat_a, flat_x = a.reshape(-1, a.shape[-2], 2), x.reshape(-1, x.shape[-2], 2)
    out = np.empty_like(flat_a)
    for b in range(flat_a.shape[0]):
        ab, xb = np.ascontiguousarray(flat_a[b]), np.ascontiguousarray(flat_x[b])
        cb = np.empty_like(ab)
        lib().oracle_fcirc_matvec_gf(int(f[0]) % GF_P, int(f[1]) % GF_P, ab.reshape(-1), xb.reshape(-1),
                                     cb.reshape(-1), ab.shape[0])
        out[b] = cb
    return out.reshape(a.shape)


def fcirc_matvec_ssa(K: int, f_exp: int, a, x) -> list:
    """Over Z/(2^K + 1) with f = 2^f_exp: c_i = sum_k a_k x_{(i+k) mod n}
    f^[i+k >= n] (Definition 2) in Python integers, for small n."""
    M = (1 << K) + 1
    f = pow(2, f_exp, M)
    n = len(a)
    out = []
    for i in range(n):
        s = 0
        for k in range(n):
            t = a[k] * x[(i + k) % n]
            s += t * f if i + k >= n else t
        out.append(s % M)
    return out


def fcirc_matvec_mod_rows(p: int, f: int, a, x, rows) -> np.ndarray:
    a, x = _u32(a), _u32(x)
    rows = np.ascontiguousarray(rows, dtype=np.uint64)
    out = np.empty(rows.size, dtype=np.uint32)
    lib().oracle_fcirc_matvec_mod_rows(p, f % p, a, x, a.size, rows, rows.size, out)
    return out


def fcirc_matvec_mod_batched(p: int, f, offsets, a, x) -> np.ndarray:
    a, x = _u32(a), _u32(x)
    f = _u32(f)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    c = np.empty_like(a)
    lib().oracle_fcirc_matvec_mod_batched(p, f, offsets, a, x, c, f.size)
    return c


# -- complex double (closing remark of Section 3.1) --------------------------

def _c2f(z):
    z = np.ascontiguousarray(z, dtype=np.complex128)
    return z.view(np.float64).reshape(-1).copy(), z.shape


def fcirc_matvec_c128(f: complex, a, x) -> np.ndarray:
    """a, x: complex arrays of shape (batch, n) or (n,)."""
    af, shape = _c2f(a)
    xf, _ = _c2f(x)
    n = shape[-1]
    batch = int(np.prod(shape[:-1])) if len(shape) > 1 else 1
    c = np.empty_like(af)
    lib().oracle_fcirc_matvec_c128(complex(f).real, complex(f).imag, af, xf, c, n, batch)
    return c.view(np.complex128).reshape(shape)


def fcirc_grad_c128(f: complex, a, x, g):
    """Returns (grad_a, grad_x) of L = Re <g, A x> (PyTorch convention)."""
    af, shape = _c2f(a)
    xf, _ = _c2f(x)
    gf, _ = _c2f(g)
    n = shape[-1]
    batch = int(np.prod(shape[:-1])) if len(shape) > 1 else 1
    ga = np.empty_like(af)
    gx = np.empty_like(af)
    lib().oracle_fcirc_grad_c128(complex(f).real, complex(f).imag, af, xf, gf, ga, gx, n, batch)
    return (ga.view(np.complex128).reshape(shape), gx.view(np.complex128).reshape(shape))


# -- polynomial and large-integer products (Section 3) -----------------------

def poly_mul(P, Q) -> np.ndarray:
    P, Q = _u16(P), _u16(Q)
    out = np.empty(P.size + Q.size - 1, dtype=np.int64)
    lib().oracle_poly_mul(P, P.size, Q, Q.size, out)
    return out


def poly_mul_coeffs(P, Q, idx) -> np.ndarray:
    P, Q = _u16(P), _u16(Q)
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.empty(idx.size, dtype=np.int64)
    lib().oracle_poly_mul_coeffs(P, P.size, Q, Q.size, idx, idx.size, out)
    return out


def bigint_mul(A, B) -> np.ndarray:
    A, B = _u16(A), _u16(B)
    out = np.empty(A.size + B.size, dtype=np.uint16)
    lib().oracle_bigint_mul(A, A.size, B, B.size, out)
    return out


def bigint_columns(A, B, idx) -> np.ndarray:
    A, B = _u16(A), _u16(B)
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.empty(idx.size, dtype=np.uint64)
    lib().oracle_bigint_columns(A, A.size, B, B.size, idx, idx.size, out)
    return out


def eval_u16_mod(coef, t: int, q: int) -> int:
    coef = _u16(coef)
    return int(lib().oracle_eval_u16_mod(coef, coef.size, t % q, q))


def eval_i64_mod(coef, t: int, q: int) -> int:
    coef = np.ascontiguousarray(coef, dtype=np.int64)
    return int(lib().oracle_eval_i64_mod(coef, coef.size, t % q, q))
