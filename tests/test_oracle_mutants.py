"""The pins must catch plausible mistakes in the oracle.  Each case below
compiles a temporary copy of oracle/fcirc_oracle.c with one planted mistake
(a dropped term, a wrong sign, a transposed operand, a missing conjugate ...)
and checks that at least one pin fails against it.  CPU only; the committed
oracle is never modified."""
import ctypes
import os
import subprocess
import tempfile

import pytest

import test_oracle_pins as pins
from oracle import oracle as O

SRC = os.path.join(os.path.dirname(O.__file__), "fcirc_oracle.c")

MUTANTS = {
    # f applied to the upper triangle instead of the lower one (complex path)
    "f_on_upper": ("return j >= i ? ld(a, j - i) : f * ld(a, n + j - i);",
                   "return j >= i ? f * ld(a, j - i) : ld(a, n + j - i);"),
    # diagonal term dropped (mod path)
    "drop_diagonal": ("for (uint64_t j = i; j < n; ++j)\n        upper",
                      "for (uint64_t j = i + 1; j < n; ++j)\n        upper"),
    # transposed operand in the wrapped part (mod path)
    "transposed_lower": ("lower = (lower + mulmod_u64(a[n + j - i], x[j], p)) % p;",
                         "lower = (lower + mulmod_u64(a[i - j], x[j], p)) % p;"),
    # f missing from the wrapped part (mod path)
    "drop_f": ("return (upper + mulmod_u64(f % p, lower, p)) % p;",
               "return (upper + lower) % p;"),
    # conjugate missing in the gradient of a
    "grad_a_no_conj": ("sa += conj(xik) * ld(gb, i);", "sa += xik * ld(gb, i);"),
    # wrap factor missing in the gradient of a
    "grad_a_no_f": ("cplx xik = idx >= n ? f * ld(xb, idx - n) : ld(xb, idx);",
                    "cplx xik = idx >= n ? ld(xb, idx - n) : ld(xb, idx);"),
    # gradient of x with A instead of A^H
    "grad_x_no_conj": ("sx += conj(fcirc_entry_c(f, ab, n, i, (uint64_t)k)) * ld(gb, i);",
                       "sx += fcirc_entry_c(f, ab, n, i, (uint64_t)k) * ld(gb, i);"),
    # column convention: f missing from the wrapped terms
    "t_drop_f": ("c[j] = (uint32_t)((direct + mulmod_u64(f % p, wrapped, p)) % p);",
                 "c[j] = (uint32_t)((direct + wrapped) % p);"),
    # column convention: wrapped terms indexed without the wrap
    "t_wrong_wrap": ("wrapped = (wrapped + mulmod_u64(a[m], x[j + n - m], p)) % p;",
                     "wrapped = (wrapped + mulmod_u64(a[m], x[m - j - 1], p)) % p;"),
    # Toeplitz: diagonal index mirrored
    "toeplitz_mirror": ("acc = (acc + mulmod_u64(t[j + n - 1 - i], x[j], p)) % p;",
                        "acc = (acc + mulmod_u64(t[i + n - 1 - j], x[j], p)) % p;"),
    # GF(p^2): 3 dropped from the sqrt 3 * sqrt 3 term
    "gf_no_three": ("*cr = (ar * br % GFP + 3 * (ai * bi % GFP)) % GFP;",
                    "*cr = (ar * br % GFP + (ai * bi % GFP)) % GFP;"),
    # GF(p^2): f missing from the wrapped terms
    "gf_drop_f": ("gf_mul(f_re, f_im, lr, li, &pr, &pi);", "pr = lr; pi = li;"),
    # off-by-one in the polynomial product window
    "poly_window": ("for (uint64_t i = lo; i <= hi; ++i)\n        s +=",
                    "for (uint64_t i = lo + 1; i <= hi; ++i)\n        s +="),
    # wrong carry width in the large-integer product
    "carry_width": ("carry = t >> 16;", "carry = t >> 15;"),
    # Horner step drops the point
    "eval_no_t": ("acc = (mulmod_u128(acc, t, q) + coef[k]) % q;",
                  "acc = (mulmod_u128(acc, t + 1, q) + coef[k]) % q;"),
}

PIN_CALLS = [
    lambda o: pins.test_layout_3x3_example_mod(o),
    lambda o: pins.test_layout_3x3_example_complex(o),
    lambda o: pins.test_identity_row(o, 8),
    lambda o: pins.test_shift_row(o, 7),
    lambda o: pins.test_f1_is_ordinary_circulant_fft(o, 32),
    lambda o: pins.test_general_f_by_diagonal_scaling_fft(o, 8, 2.0),
    lambda o: pins.test_transpose_is_polynomial_product_mod_xn_minus_f(o, 8),
    lambda o: pins.test_column_convention_is_the_transpose(o, 8),
    lambda o: pins.test_toeplitz_oracle(o, 6),
    lambda o: pins.test_gf_oracle_is_four_products_over_the_prime_field(o, 8),
    lambda o: pins.test_gf_oracle_shift_and_identity_rows(o, 5),
    lambda o: pins.test_algorithm1_bruteforce_equals_dense(o, 16, None),
    lambda o: pins.test_complex_gradients_finite_differences(o, 0.6 + 0.8j),
    lambda o: pins.test_complex_gradients_finite_differences(o, 2.0 - 0.5j),
    lambda o: pins.test_complex_adjoint_dot(o),
    lambda o: pins.test_poly_mul_vs_numpy_convolve(o, 13, 70),
    lambda o: pins.test_bigint_mul_vs_python_int(o, 64, 64),
    lambda o: pins.test_eval_mod_q(o),
]


def _compile_mutant(name, old, new, tmpdir):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = os.path.join(tmpdir, f"{name}.c")
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    so = os.path.join(tmpdir, f"lib{name}.so")
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                           "-o", so, path, "-lm"])
    return so


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, monkeypatch):
    old, new = MUTANTS[name]
    with tempfile.TemporaryDirectory() as d:
        so = _compile_mutant(name, old, new, d)
        real = O.lib()
        mutant = ctypes.CDLL(so)
        # same signatures as the real library
        for fn in dir(real):
            if fn.startswith("oracle_"):
                src_fn, dst_fn = getattr(real, fn), getattr(mutant, fn)
                dst_fn.argtypes = src_fn.argtypes
                dst_fn.restype = src_fn.restype
        monkeypatch.setattr(O, "_lib", mutant)
        caught = []
        for call in PIN_CALLS:
            try:
                call(O)
            except AssertionError:
                caught.append(call)
        assert caught, f"no pin caught mutant {name}"


def test_unmutated_oracle_passes_every_pin_call():
    """Control: the committed oracle passes all the pin calls used above, so a
    failure under a mutant is caused by the planted mistake."""
    for call in PIN_CALLS:
        call(O)


def _ssa_mutant_drop_f(K, f_exp, a, x):
    """The Z/(2^K + 1) oracle with the wrap factor f dropped."""
    M = (1 << K) + 1
    n = len(a)
    return [sum(a[k] * x[(i + k) % n] for k in range(n)) % M for i in range(n)]


def _ssa_mutant_wrong_index(K, f_exp, a, x):
    """The Z/(2^K + 1) oracle with the vector index mirrored."""
    M = (1 << K) + 1
    f = pow(2, f_exp, M)
    n = len(a)
    return [sum(a[k] * x[(i - k) % n] * (f if i + k >= n else 1) for k in range(n)) % M for i in range(n)]


@pytest.mark.parametrize("mutant", [_ssa_mutant_drop_f, _ssa_mutant_wrong_index])
def test_pins_catch_ssa_oracle_mutants(mutant):
    class Shim:
        fcirc_matvec_ssa = staticmethod(mutant)
    caught = False
    for call in (lambda o: pins.test_ssa_oracle_small_values_are_the_integer_product(o, 8),
                 lambda o: pins.test_ssa_oracle_identity_and_shift_rows(o, 64)):
        try:
            call(Shim)
        except AssertionError:
            caught = True
    assert caught
