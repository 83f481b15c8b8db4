"""The device arithmetic headers built for the host (tests/host_arith/
arith_host.cpp) and checked bit for bit against Python integers, without a
GPU:

* Z/(2^K + 1), K = 64, 128 (ssa.cuh, the branch-free normalisation, shift
  twiddles and the element 2^K): sums, differences, negation, products and
  products by 2^e, with the representation invariant (top word 1 only for
  2^K itself);
* GF(p^2), p = 2^31 - 1 (gfp2.hpp): the 32-bit Mersenne reduction of every
  x < 2^63 and the field operations;
* mod p (modarith.cuh): the Shoup product for any 32-bit operand, Montgomery
  reduction, and the leaf shift of the polynomial product: two sibling 2x2
  leaves and their first recombination level in the zero-cost form
  (bfly_rec_shift) against the shifted leaf's definition, (phi x1, x0) for
  the row (x0, x1), followed by the ordinary recombination."""
import os
import random
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("arith") / "arith_host")
    subprocess.run([cxx, "-O1", "-w", "-o", exe, os.path.join(HERE, "host_arith", "arith_host.cpp")], check=True)

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        res = out.stdout.split("\n")
        assert len(res) >= len(lines)
        return res[:len(lines)]
    return run


def _ssa_words(v, W):
    K = 64 * W
    if v == 1 << K:
        return [0] * W + [1]
    return [(v >> (64 * i)) & (2 ** 64 - 1) for i in range(W)] + [0]


@pytest.mark.parametrize("W", [1, 2])
def test_ssa_ring_ops(harness, W):
    rng = random.Random(11 + W)
    K = 64 * W
    M = (1 << K) + 1
    edge = [0, 1, 2, (1 << K) - 1, (1 << K) - 2, 1 << K, 1 << (K - 1)]
    if W == 2:
        edge += [(1 << 64) - 1, 1 << 64]
    vals = edge + [rng.randrange(1 << K) for _ in range(24)]
    lines, want = [], []
    for a in vals:
        for b in vals:
            for op, ref in (("add", (a + b) % M), ("sub", (a - b) % M), ("mul", (a * b) % M)):
                lines.append(f"ssa{W} {op} " + " ".join(f"{t:x}" for t in _ssa_words(a, W) + _ssa_words(b, W)))
                want.append(ref)
        lines.append(f"ssa{W} neg " + " ".join(f"{t:x}" for t in _ssa_words(a, W)))
        want.append((-a) % M)
        for e in sorted({0, 1, 63, 64, K - 1, K, K + 1, 2 * K - 1, rng.randrange(2 * K)}):
            lines.append(f"ssa{W} tw {e} " + " ".join(f"{t:x}" for t in _ssa_words(a, W)))
            want.append(a * pow(2, e, M) % M)
    for ln, w, o in zip(lines, want, harness(lines)):
        ws = [int(t, 16) for t in o.split()]
        got = sum(t << (64 * i) for i, t in enumerate(ws[:W])) + (ws[W] << K)
        assert got == w, ln
        assert ws[W] in (0, 1) and (ws[W] == 0 or not any(ws[:W])), ln   # 2^K only as (0, .., 0, 1)


def test_gf_mersenne_reduction_and_field_ops(harness):
    rng = random.Random(5)
    P = 2 ** 31 - 1
    xs = [0, 1, P - 1, P, P + 1, 2 ** 31, 2 ** 32 - 1, 2 ** 32, 2 ** 62, 2 ** 62 + 2 ** 33, 2 ** 63 - 1,
          P * P, 2 * P * P, (2 ** 31 - 1) * (2 ** 32 - 5)]   # red needs x < 2^63
    xs += [rng.randrange(2 ** 63) for _ in range(3000)] + [rng.randrange(2 ** 36) for _ in range(500)]
    lines = [f"gf red {x:x}" for x in xs]
    want = [str(x % P) for x in xs]
    vals = [0, 1, 2, P - 1, P - 2, 2 ** 30] + [rng.randrange(P) for _ in range(30)]
    for _ in range(3000):
        a, b, c, d = (rng.choice(vals) for _ in range(4))
        lines += [f"gf mul {a} {b} {c} {d}", f"gf add {a} {b} {c} {d}", f"gf sub {a} {b} {c} {d}",
                  f"gf neg {a} {b} 0 0"]
        want += [f"{(a * c + 3 * b * d) % P} {(a * d + b * c) % P}", f"{(a + c) % P} {(b + d) % P}",
                 f"{(a - c) % P} {(b - d) % P}", f"{(-a) % P} {(-b) % P}"]
    for ln, w, o in zip(lines, want, harness(lines)):
        assert o.strip() == w, ln


PRIMES = (998244353, 469762049, 167772161)


@pytest.mark.parametrize("p", PRIMES)
def test_shoup_and_montgomery(harness, p):
    rng = random.Random(p)
    lines, checks = [], []
    for _ in range(800):
        x, w = rng.randrange(2 ** 32), rng.randrange(p)
        lines.append(f"mod shoup {p} {x} {w}")
        checks.append(("shoup", x * w % p))
    pinv = pow(p, -1, 2 ** 32)
    for _ in range(800):
        t = rng.randrange(p * 2 ** 32)
        lines.append(f"mod redc {p} {t:x} {pinv}")
        checks.append(("redc", t * pow(2, -32, p) % p))
    for ln, (kind, ref), o in zip(lines, checks, harness(lines)):
        v = int(o)
        assert v % p == ref, ln
        assert (0 <= v < 2 * p) if kind == "shoup" else (0 < v <= 2 * p), ln


@pytest.mark.parametrize("p", PRIMES)
def test_leaf_shift_costs_no_multiplication(harness, p):
    """leaf2 on both sibling leaves, entries swapped, then bfly_rec on the
    entry-0 pair and bfly_rec_shift on the entry-1 pair equals the leaves of
    the row shifted by one place, (phi x1, x0), recombined the ordinary way
    (the halving deferred: (M1 + M2) s^-1, M1 - M2)."""
    rng = random.Random(p + 1)
    R1 = pow(2, -32, p)                     # the factor leaf2's Montgomery reduction leaves
    pinv = pow(p, -1, 2 ** 32)
    lines, want = [], []
    for _ in range(600):
        a = [rng.randrange(4 * p) for _ in range(4)]       # lazy inputs, as the tile holds them
        y = [rng.randrange(4 * p) for _ in range(4)]
        s = rng.randrange(1, p)
        si = pow(s, -1, p)

        def shifted_leaf(x0, x1, y0, y1, phi):
            r0, r1 = phi * x1 % p, x0 % p                  # the shifted row (phi x1, x0)
            return (r0 * y0 + r1 * y1) * R1 % p, (phi * r1 * y0 + r0 * y1) * R1 % p
        A = shifted_leaf(a[0], a[1], y[0], y[1], s)
        B = shifted_leaf(a[2], a[3], y[2], y[3], p - s)
        lo = [(A[k] + B[k]) * si % p for k in range(2)]
        hi = [(A[k] - B[k]) % p for k in range(2)]
        lines.append(f"mod leaf {p} " + " ".join(map(str, a + y)) + f" {s} {si} {pinv}")
        want.append(f"{lo[0]} {lo[1]} {hi[0]} {hi[1]}")
    for ln, w, o in zip(lines, want, harness(lines)):
        assert o.strip() == w, ln


@pytest.mark.parametrize("p", PRIMES + (2 ** 31 - 1, 7681, 17))
def test_barrett_products_of_the_plan_kernel(harness, p):
    """ModP (ring.hpp), the products and powers the batched plan kernel
    computes roots with: equal to exact integer arithmetic for random and
    edge operands, including (p - 1)^2, the largest product."""
    rng = random.Random(p + 7)
    ops = [(0, 0, 0), (1, 1, 1), (p - 1, p - 1, p - 2), (p - 1, 1, 2 ** 40 + 3), (p // 2, p - 2, 0)]
    ops += [(rng.randrange(p), rng.randrange(p), rng.randrange(2 ** 40)) for _ in range(600)]
    out = harness([f"mod barrett {p} {a} {b} {e}" for a, b, e in ops])
    for (a, b, e), o in zip(ops, out):
        m, pw = map(int, o.split())
        assert m == a * b % p and pw == pow(a, e, p), (a, b, e)


@pytest.mark.parametrize("p", PRIMES)
def test_roots_by_barrett_equal_the_plain_path(harness, p):
    """nth_root_2k_om with the Barrett reducer finds the same root (or the
    same absence of one) as with plain remainders, and the root is one:
    r^(2^k) = f."""
    v = ((p - 1) & -(p - 1)).bit_length() - 1
    g = next(g for g in range(2, p) if all(pow(g, (p - 1) // r, p) != 1 for r in (2, 3, 5, 7, 17)
                                              if (p - 1) % r == 0))
    Om = pow(g, (p - 1) >> v, p)
    rng = random.Random(p + 8)
    cases = [(1, 3), (p - 1, 1), (p - 1, v), (Om, v), (Om, 1)]
    cases += [(pow(rng.randrange(1, p), 2 ** k, p), k) for k in rng.choices(range(1, v), k=60)]
    cases += [(rng.randrange(1, p), rng.randrange(1, v)) for _ in range(60)]   # mostly no root
    out = harness([f"mod root {p} {f} {k} {Om} {v}" for f, k in cases])
    for (f, k), o in zip(cases, out):
        o1, r1, o2, r2 = map(int, o.split())
        assert (o1, r1) == (o2, r2), (f, k)
        if o1:
            assert pow(r1, 2 ** k, p) == f % p, (f, k)


@pytest.mark.parametrize("p", PRIMES + (7681, 17, 3))
def test_barrett_shoup_quotients(harness, p):
    """ModP's quotients (the batched kernel's twiddles and tile factors):
    floor(w 2^32 / p) and floor(w 2^64 / p) exactly, for every w in a random
    sample and at the edges 0, 1, p - 1."""
    rng = random.Random(p + 9)
    ws = sorted({0, 1, p - 1, p // 2} | {rng.randrange(p) for _ in range(500)})
    out = harness([f"mod bquot {p} {w}" for w in ws])
    for w, o in zip(ws, out):
        q32, hi, lo = map(int, o.split())
        assert q32 == (w << 32) // p, w
        assert (hi << 32) | lo == (w << 64) // p, w
