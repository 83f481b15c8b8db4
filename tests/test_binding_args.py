"""The Python binding rejects malformed arguments before it calls the
library: wrong dtypes, non-contiguous tensors, mismatched lengths and, for a
caller-supplied output, any shape other than the one the library writes
(a shorter one would be overrun).  CPU tensors, no GPU and no library call:
every case here raises before `load()` is reached."""
import pytest

torch = pytest.importorskip("torch")

import paper_2103_02605_gb300 as F  # noqa: E402

P1 = 998244353


def u32(n):
    return torch.zeros(n, dtype=torch.int32)


@pytest.fixture(autouse=True)
def no_library(monkeypatch):
    """Any call that got past the argument checks would load the library."""
    def refuse():
        raise AssertionError("argument checks let a malformed call through")
    monkeypatch.setattr(F, "load", refuse)


@pytest.mark.parametrize("fn", [F.fcirc_matvec, F.fcirc_matvec_t])
def test_matvec_outputs(fn):
    with pytest.raises(ValueError):
        fn(P1, 1, u32(8), u32(8), out=u32(7))                 # too short
    with pytest.raises(ValueError):
        fn(P1, 1, u32(8), u32(8), out=u32(16))                # too long
    with pytest.raises(TypeError):
        fn(P1, 1, u32(8), u32(8), out=torch.zeros(8, dtype=torch.int64))
    with pytest.raises(ValueError):
        fn(P1, 1, u32(8), u32(8), out=u32(16)[::2])           # not contiguous
    with pytest.raises(ValueError):
        fn(P1, 1, u32(8), u32(4))                             # a, x lengths differ
    with pytest.raises(TypeError):
        fn(P1, 1, torch.zeros(8), u32(8))                     # float residues


def test_toeplitz_outputs():
    with pytest.raises(ValueError):
        F.fcirc_toeplitz_matvec(P1, u32(15), u32(8), out=u32(15))
    with pytest.raises(ValueError):
        F.fcirc_toeplitz_matvec(P1, u32(14), u32(8))          # needs 2n - 1 diagonals


def test_gf_and_ssa_outputs():
    a = torch.zeros((3, 16, 2), dtype=torch.int32)
    with pytest.raises(ValueError):
        F.fcirc_matvec_gf(a, a, out=torch.zeros((3, 8, 2), dtype=torch.int32))
    s = torch.zeros((3, 16, 3), dtype=torch.int64)
    with pytest.raises(ValueError):
        F.fcirc_matvec_ssa(s, s, 128, 0, out=torch.zeros((3, 16, 2), dtype=torch.int64))
    with pytest.raises(TypeError):
        F.fcirc_matvec_ssa(s, s, 128, 0, out=torch.zeros((3, 16, 3), dtype=torch.int32))
    with pytest.raises(ValueError):
        F.fcirc_matvec_ssa(s, s, 64, 0)                       # K = 64 wants 2 words per element


def test_poly_and_bigint_outputs():
    P = torch.zeros(10, dtype=torch.int16)
    Q = torch.zeros(7, dtype=torch.int16)
    with pytest.raises(ValueError):
        F.poly_mul_int(P, Q, out=torch.zeros(15, dtype=torch.int64))   # needs 16
    with pytest.raises(TypeError):
        F.poly_mul_int(P, Q, out=torch.zeros(16, dtype=torch.int32))
    with pytest.raises(ValueError):
        F.poly_mul_int(P, torch.zeros(0, dtype=torch.int16))
    with pytest.raises(TypeError):
        F.poly_mul_int(P.to(torch.int32), Q)
    with pytest.raises(ValueError):
        F.bigint_mul(P, Q, out=torch.zeros(16, dtype=torch.int16))     # needs 17 limbs
    with pytest.raises(TypeError):
        F.bigint_mul(P, Q, out=torch.zeros(17, dtype=torch.int64))


def test_batched_arguments():
    f = u32(3)
    off = torch.tensor([0, 8, 16, 32], dtype=torch.int64)
    with pytest.raises(ValueError):
        F.fcirc_matvec_batched(P1, f, off, u32(32), u32(32), out=u32(31))
    with pytest.raises(ValueError):
        F.fcirc_matvec_batched(P1, u32(2), off, u32(32), u32(32))      # offsets is count + 1 long
    with pytest.raises(ValueError):
        F.fcirc_matvec_batched(P1, f, off, u32(32), u32(16))
    with pytest.raises(ValueError):
        F.BatchedGraph(P1, f, off, u32(32), u32(32), u32(32), 64)       # total_n beyond the arrays


def test_complex_outputs():
    a = torch.zeros((4, 16), dtype=torch.complex64)
    with pytest.raises(ValueError):
        F.fcirc_matvec_c64(a, a, out=torch.zeros((4, 8), dtype=torch.complex64))
    with pytest.raises(TypeError):
        F.fcirc_matvec_c64(a.to(torch.complex128), a)
