"""Shared-memory layouts of the register-staged kernels, checked exhaustively
on the CPU: every access pattern is a bijection onto the buffer (no two
threads' residues collide) and every warp access is free of bank conflicts.

The index formulas are restated from csrc/tile_dev.cuh (tphi, the 4096-residue
tile), csrc/kernels_fast.cu (cphi, one column per thread) and
csrc/kernels_col4.cu (c4_off and the store phase, four columns per thread).
Banks: 32 four-byte banks; a 128-bit access is served in four phases of
eight lanes, each of which must touch eight distinct 16-byte bank groups."""
from collections import Counter

import pytest


# -- 4096-residue tile -----------------------------------------------------------

def tphi(e):
    c = e >> 2
    r, col = c >> 3, c & 7
    g = (r & 3) ^ ((r & 8) >> 1)
    return (((r << 3) | (col ^ g)) << 2) | (e & 3)


def test_tile_layout_bijective():
    assert sorted(tphi(e) for e in range(4096)) == list(range(4096))


def test_tile_scalar_patterns_conflict_free():
    # stage A: residues tid + 256 j; stage B: 256 (tid >> 4) + 16 m + (tid & 15)
    for j in range(16):
        for w in range(8):
            lanes = range(32 * w, 32 * w + 32)
            assert len({tphi(t + 256 * j) % 32 for t in lanes}) == 32
            assert len({tphi(((t >> 4) << 8) + 16 * j + (t & 15)) % 32 for t in lanes}) == 32


def test_tile_vector_pattern_conflict_free():
    # stage C: residues 16 tid + 4 q read as 128-bit words
    for q in range(4):
        for t0 in range(0, 256, 8):
            groups = [(tphi(16 * t + 4 * q) // 4) % 8 for t in range(t0, t0 + 8)]
            assert len(set(groups)) == 8


# -- one column per thread (k_colfwd / k_colinv) -----------------------------------

def cphi(r, c):
    return ((r ^ ((r >> 4) & 7)) << 2) | c


@pytest.mark.parametrize("LF", [8, 9, 10, 11, 12])
def test_one_column_layout_conflict_free(LF):
    NT = (1 << LF) // 8
    NST = (LF + 3) // 4
    NL0 = LF - 4 * (NST - 1)
    for S in range(NST):
        NL = NL0 if S == 0 else 4
        D0 = 0 if S == 0 else NL0 + 4 * (S - 1)
        M, B, LST, LRB = 1 << NL, 16 >> NL, LF - D0 - NL, LF - D0
        words = set()
        for h in range(2 * B):
            for i in range(M):
                for w0 in range(0, NT, 32):
                    banks = []
                    for t in range(w0, min(w0 + 32, NT)):
                        gg = t + NT * h
                        col, g = gg & 3, gg >> 2
                        blk = g >> LST
                        row = (blk << LRB) + (g & ((1 << LST) - 1)) + (i << LST)
                        banks.append(cphi(row, col) % 32)
                        words.add(cphi(row, col))
                    assert len(set(banks)) == len(banks)
        assert words == set(range(4 << LF))


# -- four columns per thread (k_colfwd4 / k_colinv4) ---------------------------------

def c4_off16(LF, quad, row, LR=4):
    qs = ((quad & 3) << 1) | ((quad >> 2) & 1)
    return (quad << LF) + (row ^ ((row >> LR) & 7) ^ qs)


@pytest.mark.parametrize("LR", [3, 4])
@pytest.mark.parametrize("LF", [8, 9, 10, 11, 12])
def test_four_column_stages_conflict_free(LF, LR):
    """2^LR rows x 4 columns per thread, 4096 / 2^LR threads."""
    NT, ROWS = 4096 >> LR, 1 << LR
    NST = (LF + LR - 1) // LR
    NL0 = LF - LR * (NST - 1)
    for S in range(NST):
        NL = NL0 if S == 0 else LR
        D0 = 0 if S == 0 else NL0 + LR * (S - 1)
        M, B, LST, LRB, LGQ = 1 << NL, ROWS >> NL, LF - D0 - NL, LF - D0, LF - NL
        seen = set()
        for h in range(B):
            for i in range(M):
                for t0 in range(0, NT, 8):
                    groups = []
                    for t in range(t0, t0 + 8):
                        gg = t + NT * h
                        quad, g = gg >> LGQ, gg & ((1 << LGQ) - 1)
                        blk = g >> LST
                        row = (blk << LRB) + (g & ((1 << LST) - 1)) + (i << LST)
                        groups.append(c4_off16(LF, quad, row, LR) % 8)
                        seen.add(c4_off16(LF, quad, row, LR))
                    assert len(set(groups)) == 8
        assert seen == set(range(4096))


@pytest.mark.parametrize("LR", [3, 4])
@pytest.mark.parametrize("LF", [8, 9, 10, 11, 12])
@pytest.mark.parametrize("maxlcl", [0, 1, 2, 3])
def test_four_column_store_phase(LF, maxlcl, LR):
    """Each cluster rank's rows, every quad of the row segment: the words
    covered once for every cluster size, and -- for the two-CTA clusters the
    kernels are built with -- no two lanes of a phase in the same bank group
    of one CTA's shared memory."""
    NT, ROWS = 4096 >> LR, 1 << LR
    LNQ = 12 - LF
    LCL = min(0 if LNQ >= 3 else 3 - LNQ, maxlcl)
    LCQ, LRW = LNQ + LCL, LF - LCL
    RSTEP = NT >> LCQ
    cover = Counter()
    for rank in range(1 << LCL):
        for k in range(ROWS):
            for t0 in range(0, NT, 8):
                per_cta = {}
                for t in range(t0, t0 + 8):
                    cq = t & ((1 << LCQ) - 1)
                    row = (rank << LRW) + (t >> LCQ) + RSTEP * k
                    cover[(cq, row)] += 1
                    per_cta.setdefault(cq >> LNQ, []).append(c4_off16(LF, cq & ((1 << LNQ) - 1), row, LR) % 8)
                if maxlcl == 1:
                    for groups in per_cta.values():
                        assert len(set(groups)) == len(groups)
    assert len(cover) == (1 << LCQ) << LF and set(cover.values()) == {1}


def _c4_stage_owners(LF, S, LR=4):
    """16-byte slot -> thread of register stage S of a four-column pass (a
    thread writes back the slots it read)."""
    NT, ROWS = 4096 >> LR, 1 << LR
    NST = (LF + LR - 1) // LR
    NL0 = LF - LR * (NST - 1)
    NL = NL0 if S == 0 else LR
    D0 = 0 if S == 0 else NL0 + LR * (S - 1)
    M, B, LST, LRB, LGQ = 1 << NL, ROWS >> NL, LF - D0 - NL, LF - D0, LF - NL
    own = {}
    for t in range(NT):
        for h in range(B):
            gg = t + NT * h
            quad, g = gg >> LGQ, gg & ((1 << LGQ) - 1)
            blk = g >> LST
            for i in range(M):
                row = (blk << LRB) + (g & ((1 << LST) - 1)) + (i << LST)
                own[c4_off16(LF, quad, row, LR)] = t
    return own


@pytest.mark.parametrize("LF", [8, 9, 10, 11, 12])
def test_four_column_last_exchange_within_a_warp(LF):
    """The column passes synchronise the exchange between their last two
    register stages (either direction) with __syncwarp (kernels_col4.cu,
    c4_stage_sync): every slot is owned by threads of one warp in both
    stages; the earlier exchanges cross warps and keep CTA barriers."""
    NST = (LF + 3) // 4
    a, b = _c4_stage_owners(LF, NST - 2), _c4_stage_owners(LF, NST - 1)
    assert set(a) == set(b) == set(range(4096))
    assert all(a[k] // 32 == b[k] // 32 for k in a)
    if NST > 2:
        c = _c4_stage_owners(LF, NST - 3)
        assert any(c[k] // 32 != a[k] // 32 for k in a)


def test_tile_address_identities():
    """The tile kernel computes its shared-memory addresses from per-thread
    bases and compile-time terms; the identities behind that, for every
    thread and every unrolled index."""
    for tid in range(256):
        tA = tphi(tid)
        eb = ((tid >> 4) << 8) + (tid & 15)
        tB, tC = tphi(eb), tphi(16 * tid)
        for j in range(16):
            assert tphi(tid + 256 * j) == (tA ^ ((j & 1) << 4)) + (j << 8)
            assert tphi(eb + 16 * j) == (tB ^ ((((j >> 1) & 3) << 2) | ((j & 1) << 4))) + ((j >> 1) << 5)
        for q in range(4):
            assert tphi(16 * tid + 4 * q) == tC ^ (q << 2)


@pytest.mark.parametrize("LF", [8, 9, 10, 11, 12])
def test_four_column_address_identities(LF):
    """k_colfwd4 / k_colinv4 compute c4_off(quad, row0 + i 2^LST) as a
    per-group base plus compile-time terms; the identities behind that for
    every thread, group and row of every stage shape (2^4 rows per thread)."""
    LR = 4
    qs = lambda q: ((q & 3) << 1) | ((q >> 2) & 1)
    NST = (LF + LR - 1) // LR
    NL0 = LF - LR * (NST - 1)
    for S in range(NST):
        NL = NL0 if S == 0 else LR
        D0 = 0 if S == 0 else NL0 + LR * (S - 1)
        M, B, LST, LRB, LGQ = 1 << NL, 16 >> NL, LF - D0 - NL, LF - D0, LF - NL
        assert LST in (0, 4) or LST >= 7
        for t in range(256):
            for h in range(B):
                gg = t + 256 * h
                quad, g = gg >> LGQ, gg & ((1 << LGQ) - 1)
                row0 = ((g >> LST) << LRB) + (g & ((1 << LST) - 1))
                for i in range(M):
                    want = 4 * c4_off16(LF, quad, row0 + (i << LST), LR)
                    if LST >= 7:
                        got = (quad << (LF + 2)) + ((row0 ^ ((row0 >> 4) & 7) ^ qs(quad)) << 2) + (i << (LST + 2))
                    elif LST == 4:
                        got = (((quad << (LF + 2)) + ((row0 ^ qs(quad)) << 2)) ^ ((i & 7) << 2)) + (i << 6)
                    else:
                        kt = ((row0 >> 4) & 7) ^ qs(quad)
                        got = (quad << (LF + 2)) + (row0 << 2) + ((i ^ kt) << 2)
                    assert got == want


def test_tile_stage_b_c_exchanges_stay_in_a_half_warp():
    """The tile kernel's exchanges between stages B and C (tile_dev.cuh)
    synchronise with __syncwarp, not a CTA barrier: every shared-memory word
    thread tid reads or writes in those stages (stage B: residues
    256 (tid >> 4) + 16 m + (tid & 15); stage C: 16 tid .. 16 tid + 15, in
    tphi positions) lies in its block's 256 words [256 g, 256 g + 256),
    g = tid >> 4, and the 16 threads of block g lie in one warp."""
    for tid in range(256):
        g = tid >> 4
        words = {tphi(256 * g + 16 * m + (tid & 15)) for m in range(16)}
        words |= {tphi(16 * tid + q) for q in range(16)}
        assert all(256 * g <= w < 256 * g + 256 for w in words), tid
        assert (16 * g) // 32 == (16 * g + 15) // 32
    # and the blocks' words do not overlap: each is a permutation of its range
    for g in range(16):
        assert sorted(tphi(e) for e in range(256 * g, 256 * g + 256)) == list(range(256 * g, 256 * g + 256))


def _ilv_pos(i):
    """Python restatement of ilv_pos (kernels_mod.hpp): bits 2..12 of i
    rotated so that bit 12 (the tile's parity) becomes bit 2."""
    return (i & ~0x1FFF) | (((i >> 12) & 1) << 2) | ((i & 0xFFC) << 1) | (i & 3)


def test_tile_pair_interleave_is_a_permutation_of_each_pair_block():
    import numpy as np
    i = np.arange(1 << 16, dtype=np.int64)
    p = _ilv_pos(i)
    assert np.array_equal(np.sort(p), i)                   # a permutation
    assert np.array_equal(p >> 13, i >> 13)                # inside its 8192-word block
    # a column quad of rows 2t and 2t + 1 fills one aligned 32-byte sector
    for t in (0, 2, 6, 14):
        for q in (0, 1, 511, 1023):
            words = [_ilv_pos((t + r) * 4096 + 4 * q + c) for r in (0, 1) for c in range(4)]
            assert words == list(range(words[0], words[0] + 8)) and words[0] % 8 == 0


def test_interleave_address_identities_of_the_kernels():
    """The closed forms the kernels use instead of ilv_pos per element: the
    tile kernel's residue base + tid + 256 j at ilv_pos(base + tid) + 512 j,
    and the column passes' row pair k of rows row0.. (row0 a multiple of 16)
    at ilv_pos(origin) + 8192 k."""
    for base in (0, 4096, 8192, 3 * 4096, 4095 * 4096):
        for tid in range(256):
            b = _ilv_pos(base + tid)
            for j in range(16):
                assert _ilv_pos(base + tid + 256 * j) == b + 512 * j
    for pb_base in (0, 1 << 24):
        for quad in (0, 1, 7, 1023):
            for row0 in range(0, 4096, 16):
                o = pb_base + 4 * quad + (row0 << 12)
                for k in range(8):
                    for c in range(4):
                        assert _ilv_pos(o + ((row0 + 2 * k) << 12) - (row0 << 12) + c) == _ilv_pos(o) + 8192 * k + c
                        assert _ilv_pos(o + ((row0 + 2 * k + 1) << 12) - (row0 << 12) + c) == \
                            _ilv_pos(o) + 8192 * k + 4 + c


def test_forward_pass_tma_store_boxes():
    """The 12-level forward pass's TMA stores (kernels_col4.cu,
    fwd_tma_maps): shared-memory word 2048 k + 8 tid + 4 h + w of box k,
    written with thread tid's rows 16 tid + 2 k + h, column w of its quad,
    lands at the 5-D tensor {4, 2, 1024, 8, N / 65536} (strides 16, 32,
    32 KiB, 256 KiB bytes) coordinate (w, h, q, k, t0 + tid): that must be
    ilv_pos of the element's natural index, for every element of the CTA, and
    inside the array."""
    import numpy as np
    tid = np.arange(256, dtype=np.int64)[:, None, None, None]
    k = np.arange(8, dtype=np.int64)[None, :, None, None]
    h = np.arange(2, dtype=np.int64)[None, None, :, None]
    w = np.arange(4, dtype=np.int64)[None, None, None, :]
    for N, pbs in ((1 << 24, (0,)), (1 << 26, (0, 1, 3))):
        for pb in pbs:
            for cg in (0, 1, 2, 511, 1023):
                base = (pb << 24) + 4 * cg                    # c4_origin, l0 = log2(N) - 24
                q, t0 = (base & 4095) >> 2, base >> 16
                assert t0 + 256 <= N >> 16                    # the kernel's guard holds
                coord = w * 1 + h * 4 + q * 8 + k * 8192 + (t0 + tid) * 65536
                natural = base + ((16 * tid + 2 * k + h) << 12) + w
                assert np.array_equal(coord, _ilv_pos(natural))
                assert coord.min() >= 0 and coord.max() < N
                # shared memory: the eight boxes tile the 64 KB area exactly once
                smem = 2048 * k + 8 * tid + 4 * h + w
                assert np.array_equal(np.sort(smem.ravel()), np.arange(16384))


def _cpos(e):
    """Python restatement of cpos<T> for 8-byte elements (kernels_complex.cu)."""
    return e ^ (((e >> 4) & 7) | (((e >> 6) & 1) << 3))


@pytest.mark.parametrize("M", range(4, 13))
@pytest.mark.parametrize("swz", [True, False])
def test_complex_leaf_exchange_within_a_warp(M, swz):
    """The complex-layer kernels (and GF(p^2), Z/(2^K + 1), which keep the
    plain layout) synchronise the exchanges around their last stage with
    __syncwarp (kernels_complex.cu): every number the last stage (8
    contiguous numbers at 8 t) exchanges with the last register stage is
    held, in both, by threads of one warp; an instance's n / 8 threads are
    whole warps or lie inside one."""
    pos = _cpos if swz else (lambda e: e)
    N, NTI = 1 << M, (1 << M) // 8
    L = M - 1
    P = L - 2
    NST = (P + 2) // 3
    nl = (lambda s: P - 3 * (NST - 1) if s == 0 else 3)
    d0 = (lambda s: 0 if s == 0 else (P - 3 * (NST - 1)) + 3 * (s - 1))
    S = NST - 1
    NL, D0 = nl(S), d0(S)
    G, MM, LST, LRB = 8 >> NL, 1 << NL, M - D0 - NL, M - D0
    own = {}
    for t in range(NTI):
        for h in range(G):
            gg = t + NTI * h
            blk, off = gg >> LST, gg & ((1 << LST) - 1)
            for i in range(MM):
                own[pos((blk << LRB) + off + (i << LST))] = t
    assert sorted(own) == list(range(N))
    assert NTI % 32 == 0 or 32 % NTI == 0
    for t in range(NTI):
        for i in range(8):
            assert own[pos(8 * t + i)] // 32 == t // 32


def _complex_patterns(M):
    """Every shared-memory access of the complex kernels for n = 2^M, as one
    list of (instance, element) per warp instruction: the loads/stores
    e = t + (n/8) k, each register stage's accesses, and the last stage's
    8 contiguous numbers per thread (CShape in kernels_complex.cu)."""
    N = 1 << M
    L = M - 1
    NTI = N // 8
    CT = max(128, NTI)
    P = L - 2
    NST = (P + 2) // 3

    def nl(s):
        return P - 3 * (NST - 1) if s == 0 else 3

    def d0(s):
        return 0 if s == 0 else (P - 3 * (NST - 1)) + 3 * (s - 1)
    thr = [(tt // NTI, tt % NTI) for tt in range(CT)]
    out = [[(li, t + NTI * k) for li, t in thr] for k in range(8)]
    for S in range(NST):
        NL, D0 = nl(S), d0(S)
        LST, LRB = M - D0 - NL, M - D0
        for h in range(8 >> NL):
            for i in range(1 << NL):
                acc = []
                for li, t in thr:
                    gg = t + NTI * h
                    acc.append((li, ((gg >> LST) << LRB) + (gg & ((1 << LST) - 1)) + (i << LST)))
                out.append(acc)
    out += [[(li, 8 * t + i) for li, t in thr] for i in range(8)]
    return out


def _half_warp_wavefronts(acc, N, pos):
    """64-bit shared accesses: each half-warp takes one wavefront per distinct
    8-byte word in its busiest bank pair."""
    tot = 0
    for w in range(0, len(acc), 32):
        for hw in (0, 16):
            words = {}
            for li, e in acc[w + hw:w + hw + 16]:
                p = li * 2 * N + pos(e)
                words.setdefault(p % 16, set()).add(p)
            tot += max(len(v) for v in words.values())
    return tot


@pytest.mark.parametrize("M", range(3, 13))
def test_complex_layout_is_a_bijection_and_conflict_free(M):
    N = 1 << M
    assert sorted(_cpos(e) for e in range(N)) == list(range(N))
    assert all(_cpos(e) >> 4 == e >> 4 for e in range(N))
    pats = _complex_patterns(M)
    got = sum(_half_warp_wavefronts(a, N, _cpos) for a in pats)
    plain = sum(_half_warp_wavefronts(a, N, lambda e: e) for a in pats)
    ideal = sum(len(a) // 16 for a in pats)
    assert got <= plain
    if M >= 7:   # one instance per half-warp: every access conflict-free
        assert got == ideal
