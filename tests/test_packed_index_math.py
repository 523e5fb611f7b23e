"""Host checks of the word-level index arithmetic of the four-arm kernel's packed
per-trial form (design_stat_packed in csrc/sim_bayes4.cu).

The kernel forms its table indices and treatment codes from one word per trial
and look with byte permutations, dot products of packed bytes and multiply-mask
bit spreads.  These tests emulate those primitives (__byte_perm, __dp4a,
__umulhi) in Python from their documented definitions and check, over every
drop pattern and seeded random counts, that each word-level step equals the
plain per-treatment formula it replaces (the byte form, design_stat).  No GPU
and no oracle arithmetic involved: this pins the bit tricks, the GPU parity
tests pin the kernel's results.
"""
import itertools

import numpy as np

LOOKS = (10, 20, 40)          # the benchmark design's cumulative patients per arm
N1, N2, N3 = LOOKS
M = N1 + 1                    # first-look count values
S2 = (N1 + 1) + (N2 + 1)      # second-look codes
S3 = S2 + (N3 + 1)            # final-look codes
NT2 = S2 * (S2 + 1) * (S2 + 2) // 6
NT = S3 * (S3 + 1) * (S3 + 2) // 6


def byte_perm(x, y, s):
    """__byte_perm(x, y, s): result byte i is byte (nibble i of s) & 7 of the
    eight bytes {y:x} (x bytes 0-3, y bytes 4-7)."""
    b = [(x >> (8 * i)) & 0xFF for i in range(4)] + [(y >> (8 * i)) & 0xFF for i in range(4)]
    return sum(b[(s >> (4 * i)) & 7] << (8 * i) for i in range(4))


def dp4a(a, b, c=0):
    """Unsigned __dp4a: the dot product of the four byte pairs plus c."""
    return sum(((a >> (8 * i)) & 0xFF) * ((b >> (8 * i)) & 0xFF) for i in range(4)) + c


def umulhi(a, b):
    return (a * b) >> 32


def pack(bytes4):
    return sum((v & 0xFF) << (8 * i) for i, v in enumerate(bytes4))


def spread_sel(d):
    """The selector of the code permutation: 0x7654 with bit 2 of nibble i + 1
    cleared for each set bit i of d."""
    return ((d * 0x1240) & 0x4440) ^ 0x7654


def tri3(c):
    return c * (c + 1) * (c + 2) // 6


def tri2(b):
    return b * (b + 1) // 2


def test_byte_transpose_of_four_words():
    rng = np.random.default_rng(0)
    for _ in range(200):
        w = [int(v) for v in rng.integers(0, 2 ** 32, size=4)]
        t0, t1 = byte_perm(w[0], w[1], 0x5140), byte_perm(w[2], w[3], 0x5140)
        t2, t3 = byte_perm(w[0], w[1], 0x7362), byte_perm(w[2], w[3], 0x7362)
        out = [byte_perm(t0, t1, 0x5410), byte_perm(t0, t1, 0x7632),
               byte_perm(t2, t3, 0x5410), byte_perm(t2, t3, 0x7632)]
        for j in range(4):
            for a in range(4):
                assert (out[j] >> (8 * a)) & 0xFF == (w[a] >> (8 * j)) & 0xFF


def test_first_look_index_by_two_dot_products():
    w1hi, w1lo, m1sq = M | (1 << 8), (M << 16) | (1 << 24), M * M
    for x in itertools.product(range(M), repeat=4):
        p0 = pack(x)
        i1 = dp4a(p0, w1hi) * m1sq + dp4a(p0, w1lo)
        assert i1 == ((x[0] * M + x[1]) * M + x[2]) * M + x[3]


def test_second_look_codes_by_one_permutation():
    rng = np.random.default_rng(1)
    off1 = M * 0x01010100
    for drop1 in range(8):
        sel = spread_sel(drop1)
        for _ in range(50):
            x0 = [int(v) for v in rng.integers(0, N1 + 1, size=4)]
            x1 = [int(v) for v in rng.integers(0, N2 + 1, size=4)]
            t2 = byte_perm(pack(x0), pack(x1) + off1, sel)
            assert t2 & 0xFF == x1[0]
            for i in range(3):
                want = x0[i + 1] if (drop1 >> i) & 1 else (N1 + 1) + x1[i + 1]
                assert (t2 >> (8 * (i + 1))) & 0xFF == want


def test_final_codes_and_use_bits():
    rng = np.random.default_rng(2)
    off2 = S2 * 0x01010100
    for drop1, drop2 in itertools.product(range(8), range(8)):
        dd = drop1 | drop2
        for mask in range(8):
            x0 = [int(v) for v in rng.integers(0, N1 + 1, size=4)]
            x1 = [int(v) for v in rng.integers(0, N2 + 1, size=4)]
            x2 = [int(v) for v in rng.integers(0, N3 + 1, size=4)]
            t2 = byte_perm(pack(x0), pack(x1) + M * 0x01010100, spread_sel(drop1))
            t3 = byte_perm(t2, pack(x2) + off2, spread_sel(dd))
            assert t3 & 0xFF == x2[0]
            use = 7 & ~dd & mask
            v = ((t3 << 1) & 0xFEFEFE00) | ((use * 0x408100) & 0x01010100)
            for i in range(3):
                if (drop1 >> i) & 1:
                    code = x0[i + 1]
                elif (drop2 >> i) & 1:
                    code = (N1 + 1) + x1[i + 1]
                else:
                    code = S2 + x2[i + 1]
                assert (t3 >> (8 * (i + 1))) & 0xFF == code
                assert (v >> (8 * (i + 1))) & 0xFF == 2 * code + ((use >> i) & 1)


def test_sorted_second_look_entry_and_position_map():
    """The sorted-triple entry of the codes, its 3-bit field in the word table,
    and the map of the sorted positions' drop bits back to the treatments."""
    perm = [0] * 16
    for q in range(16):
        t0, t1 = q >> 2, q & 3
        t2 = 3 - t0 - t1
        if len({t0, t1, t2}) == 3 and max(t0, t1, t2) < 3 and min(t0, t1, t2) >= 0:
            m = 0
            for bits in range(8):
                out = ((bits & 1) << t0) | (((bits >> 1) & 1) << t1) | (((bits >> 2) & 1) << t2)
                m |= out << (3 * bits)
            perm[q] = m
    rng = np.random.default_rng(3)
    for _ in range(3000):
        codes = [int(v) for v in rng.integers(0, S2, size=3)]
        x10 = int(rng.integers(0, N2 + 1))
        t2 = pack([x10] + codes)
        v2 = ((t2 << 2) & 0xFCFCFC00) | 0x02010000
        u = sorted([(v2 >> 8) & 0xFF, (v2 >> 16) & 0xFF, v2 >> 24])
        c = [k >> 2 for k in u]
        assert c == sorted(codes)
        e2 = x10 * NT2 + tri3(u[2] >> 2) + tri2(u[1] >> 2) + (u[0] >> 2)
        assert 0 <= e2 < (N2 + 1) * NT2
        w2 = umulhi(e2, 0xCCCCCCCD) >> 3
        assert w2 == e2 // 10 and e2 - 10 * w2 < 10
        # the sorted positions' bits go to the treatments they came from
        pos_bits = int(rng.integers(0, 8))
        drop2 = (perm[((u[0] & 3) << 2) | (u[1] & 3)] >> (3 * pos_bits)) & 7
        want = 0
        for k in range(3):
            if (pos_bits >> k) & 1:
                want |= 1 << (u[k] & 3)
        assert drop2 == want


def test_final_table_index_and_division_by_ten_range():
    for c2 in range(S3):
        for c1 in range(c2 + 1):
            for c0 in range(c1 + 1):
                r = tri3(c2) + tri2(c1) + c0
                assert 0 <= r < NT
    # e2 / 10 by multiply-high for every index the table holds
    for e in range(0, (N2 + 1) * NT2, 7):
        assert umulhi(e, 0xCCCCCCCD) >> 3 == e // 10


def test_rejecting_counts_in_16_bit_halves():
    """Sums of the final counts of arms 0 and 2 (and 1 and 3) in the two halves
    of one word stay exact for 64 steps of 4 trials (the flush interval)."""
    rng = np.random.default_rng(4)
    a02 = a13 = 0
    want = [0, 0, 0, 0]
    for _ in range(64 * 4):
        x2 = [int(v) for v in rng.integers(0, 256, size=4)]
        p2 = pack(x2)
        a02 = (a02 + (p2 & 0x00FF00FF)) & 0xFFFFFFFF
        a13 = (a13 + byte_perm(p2, 0, 0x4341)) & 0xFFFFFFFF
        for a in range(4):
            want[a] += x2[a]
    assert [a02 & 0xFFFF, a13 & 0xFFFF, a02 >> 16, a13 >> 16] == want
