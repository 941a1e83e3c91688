"""Pins of the oracle's algebraic signature (Section 3.1):
sig^k(P) = sum_{i=0}^{l-1} p_i x^(k i), k = 1..4, in GF(2^16)."""
import random

import numpy as np
import pytest

import oracle
import workloads
from cases import edge_keys, five_symbol_collision, symbol_collision
from gfpoly import gmul, gpow, sig_by_polynomial, symbols


def comp(s, k):
    return (s >> (16 * (k - 1))) & 0xFFFF


def rand_key(rng, n, alphabet=None):
    if alphabet is None:
        return bytes(rng.randrange(256) for _ in range(n))
    return bytes(rng.choice(alphabet) for _ in range(n))


@pytest.mark.parametrize("method", ["tables", "horner"])
def test_special_cases(method):
    assert oracle.sig(b"", method) == 0
    # a single symbol has weight x^0 = 1 in every component
    assert oracle.sig(b"AB", method) == 0x4241424142414241           # little-endian pairing
    assert oracle.sig(b"A", method) == 0x0041004100410041            # odd byte is the low byte
    assert oracle.sig(b"\0\0", method) == 0
    # symbol i has weight x^(k i): "\0\0AB" -> 0x4241 * x^k
    s = oracle.sig(b"\0\0AB", method)
    for k in range(1, 5):
        assert comp(s, k) == gmul(0x4241, gpow(2, k))


@pytest.mark.parametrize("method", ["tables", "horner"])
def test_against_polynomial_definition(method):
    rng = random.Random(3)
    keys = edge_keys() + [rand_key(rng, n) for n in list(range(0, 40)) + [63, 64, 65, 127, 200, 511]]
    for key in keys:
        assert oracle.sig(key, method) == sig_by_polynomial(key), key


def test_worked_values_from_definition():
    # values of the definition computed by independent polynomial arithmetic, and the constants
    # worked out from the definition for these keys (the last one is the paper's example string)
    worked = {b"ABC": 0x46714059434D42C7, b"ABCD": 0x465D404F4346CAC7,
              b"Paul Sabatier University": 0x8FD210505191A40E}
    for key, value in worked.items():
        assert sig_by_polynomial(key) == value, key
        assert oracle.sig(key) == value, key
        assert oracle.sig(key, "horner") == value, key


def test_linearity():
    rng = random.Random(4)
    for n in (1, 2, 7, 16, 33, 256, 1001):
        a, b = rand_key(rng, n), rand_key(rng, n)
        x = bytes(p ^ q for p, q in zip(a, b))
        assert oracle.sig(x) == oracle.sig(a) ^ oracle.sig(b)


def test_concatenation_rule():
    # sig(A || B) = sig(A) + x^(k |A|) sig(B), |A| in symbols (A of even byte length)
    rng = random.Random(5)
    for la, lb in ((0, 5), (2, 3), (16, 16), (100, 37), (4096, 1000)):
        a, b = rand_key(rng, la), rand_key(rng, lb)
        sa, sb, sab = oracle.sig(a), oracle.sig(b), oracle.sig(a + b)
        for k in range(1, 5):
            assert comp(sab, k) == comp(sa, k) ^ oracle.gf_mul_tab(oracle.gf_pow_x(k * (la // 2)), comp(sb, k))


def test_odd_length_padding():
    # a key of odd length signs like the key with a zero byte appended
    rng = random.Random(6)
    for n in (1, 3, 17, 255):
        a = rand_key(rng, n)
        assert oracle.sig(a) == oracle.sig(a + b"\0")


def test_up_to_four_symbol_changes_always_detected():
    rng = random.Random(8)
    for trial in range(400):
        n = rng.randrange(8, 300)
        a = [rng.randrange(65536) for _ in range(n)]
        b = list(a)
        for pos in rng.sample(range(n), rng.randrange(1, 5)):
            b[pos] ^= rng.randrange(1, 65536)
        ka = b"".join(v.to_bytes(2, "little") for v in a)
        kb = b"".join(v.to_bytes(2, "little") for v in b)
        assert oracle.sig(ka) != oracle.sig(kb)


def test_vandermonde_no_four_symbol_collision_exhaustive_positions():
    # for every 4 positions among the first 12 symbols, the 4x4 matrix [x^(k i_j)]
    # is non-singular, so no non-zero change on those positions keeps sig^1..sig^4
    from itertools import combinations
    from gfpoly import solve
    for pos in combinations(range(12), 4):
        M = [[gpow(2, k * i) for i in pos] for k in range(1, 5)]
        # a non-singular system has the unique solution 0 for a zero right-hand side
        # and a solution for any right-hand side; check a random one round-trips
        rhs = [0x1234, 0x0F0F, 0xBEEF, 0x0001]
        d = solve(M, rhs)
        back = [0, 0, 0, 0]
        for k in range(4):
            for j in range(4):
                back[k] ^= gmul(M[k][j], d[j])
        assert back == rhs


def test_five_symbol_collision_is_tight():
    a, b = five_symbol_collision()
    assert a != b and len(a) == len(b)
    assert oracle.sig(a) == oracle.sig(b)
    assert sum(x != y for x, y in zip(symbols(a), symbols(b))) == 5


def test_beyond_field_order_wraps_exponent():
    # symbol index i >= 65535 has weight x^(k i mod 65535): a key of 65536 symbols
    # whose only non-zero symbols sit at i = 0 and i = 65535 has sig^k = 0.
    key = bytearray(2 * 65536)
    key[0] = 1
    key[2 * 65535] = 1
    assert oracle.sig(bytes(key)) == 0


def test_batch_matches_single():
    rng = random.Random(9)
    keys = edge_keys() + [rand_key(rng, rng.randrange(0, 600)) for _ in range(200)]
    import workloads
    rel = workloads.relation_from_keys(keys)
    for method in ("tables", "horner"):
        out = oracle.sig_batch(rel.arena, rel.off, method=method, nthreads=3)
        assert out.tolist() == [oracle.sig(k) for k in keys]


def test_two_component_signature_guarantee_and_tightness():
    """The paper's two-symbol signature (n = 2, Section 3.1): keys that differ
    in one or two symbols never share it (the 2x2 Vandermonde minors
    x^(i+j) (x^j - x^i) are non-zero for distinct positions), while a
    three-symbol difference can (constructed by solving the 2x3 system);
    the same pair still differs in the four-component signature here."""
    from gfpoly import gmul, gpow
    mask2 = oracle.component_mask(2)
    for i in range(40):
        for j in range(i + 1, 40):
            det = gmul(gpow(2, i), gpow(2, 2 * j)) ^ gmul(gpow(2, j), gpow(2, 2 * i))
            assert det != 0
    rng = random.Random(12)
    for _ in range(200):
        key = bytes(rng.randrange(256) for _ in range(2 * rng.randrange(2, 30)))
        ps = list(key)
        for pos in rng.sample(range(len(key) // 2), min(2, len(key) // 2)):
            ps[2 * pos] ^= rng.randrange(1, 256)
        other = bytes(ps)
        assert oracle.sig(key) & mask2 != oracle.sig(other) & mask2
    a, b = symbol_collision(2, 12, (0, 5, 11), seed=3)
    assert oracle.sig(a) & mask2 == oracle.sig(b) & mask2
    assert oracle.sig(a) != oracle.sig(b)
    assert oracle.component_mask(4) == (1 << 64) - 1


def test_cumulative_signatures_and_substring_rule():
    """Cumulative signatures (the signatures of a key's block prefixes): the
    last entry is the key's signature, and any substring starting on an even
    byte a follows from two prefixes by the concatenation rule,
    sig(P[a..b)) = x^(-k a/2) (sig(P[0..b)) + sig(P[0..a))), with the GF
    arithmetic taken from the textbook routines of gfpoly."""
    rng = random.Random(77)
    assert oracle.sig_prefixes(b"", 16) == [0]
    for _ in range(60):
        key = rand_key(rng, rng.randrange(1, 300))
        B = rng.choice([16, 32, 64, 256])
        C = oracle.sig_prefixes(key, B)
        assert len(C) == (len(key) + B - 1) // B
        assert C[-1] == oracle.sig(key)
        assert C[:-1] == [oracle.sig(key[:(j + 1) * B]) for j in range(len(C) - 1)]
        a = 2 * rng.randrange(0, len(key) // 2 + 1)
        b = rng.randrange(a, len(key) + 1)
        full, pre = oracle.sig(key[:b]), oracle.sig(key[:a])
        want = oracle.sig(key[a:b])
        got = 0
        for k in range(1, 5):
            d = comp(full, k) ^ comp(pre, k)
            got |= gmul(d, gpow(gpow(2, k * (a // 2)), 65534)) << (16 * (k - 1))
        assert got == want


def test_byte_symbol_signature_gf8():
    """The GF(2^8) signature (byte symbols): x is primitive under
    x^8+x^4+x^3+x^2+1 (order 255); tables = Horner = the polynomial definition;
    a single byte gives that byte in every component; keys of equal length
    under 255 bytes that differ in at most 4 bytes never collide, a constructed
    5-byte difference does, and past 255 bytes the exponent wraps (x^255 = 1),
    so equal changes at bytes 0 and 255 cancel."""
    from gfpoly import gmul8, gpow8, sig8_by_polynomial, solve8
    for p in (3, 5, 17):
        assert gpow8(2, 255 // p) != 1
    assert gpow8(2, 255) == 1
    rng = random.Random(88)
    assert oracle.sig8(b"") == 0
    for b in range(256):
        assert oracle.sig8(bytes([b])) == b * 0x01010101
    for _ in range(150):
        key = rand_key(rng, rng.randrange(0, 300))
        s = oracle.sig8(key)
        assert s == oracle.sig8(key, "horner") == sig8_by_polynomial(key)
    for _ in range(300):
        key = rand_key(rng, rng.randrange(4, 255))
        other = bytearray(key)
        for pos in rng.sample(range(len(key)), rng.randrange(1, 5)):
            other[pos] ^= rng.randrange(1, 256)
        assert oracle.sig8(bytes(other)) != oracle.sig8(key)
    pos = [2, 9, 40, 100, 200]
    M = [[gpow8(2, k * pos[j]) for j in range(4)] for k in range(1, 5)]
    d = solve8(M, [gpow8(2, k * pos[4]) for k in range(1, 5)]) + [1]
    key = rand_key(rng, 230)
    other = bytearray(key)
    for p_, dj in zip(pos, d):
        other[p_] ^= dj
    assert bytes(other) != key and oracle.sig8(bytes(other)) == oracle.sig8(key)
    key = rand_key(rng, 300)
    other = bytearray(key)
    other[0] ^= 0x5A
    other[255] ^= 0x5A
    assert oracle.sig8(bytes(other)) == oracle.sig8(key)
    batch_keys = [rand_key(rng, rng.randrange(0, 90)) for _ in range(200)]
    rel = workloads.relation_from_keys(batch_keys)
    assert oracle.sig8_batch(rel.arena, rel.off, nthreads=3).tolist() == [oracle.sig8(k) for k in batch_keys]
