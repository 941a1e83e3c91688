"""Pins of the oracle's GF(2^16) arithmetic (Section 3.1: XOR addition,
log/antilog multiplication, every non-zero element a power of alpha)."""
import random

import numpy as np

import oracle
from gfpoly import POLY, gmul, gpow


def test_x_is_primitive():
    # closed form: x has order 65535 = 3*5*17*257 iff x^65535 = 1 and x^(65535/p) != 1
    assert gpow(2, 65535) == 1
    for p in (3, 5, 17, 257):
        assert gpow(2, 65535 // p) != 1


def test_log_antilog_tables_are_inverse_bijections():
    log, alog = oracle.gf_tables()
    assert len(set(alog.tolist())) == 65535 and 0 not in set(alog.tolist())
    v = np.arange(1, 65536)
    assert np.array_equal(alog[log[v]], v.astype(np.uint16))
    assert alog[0] == 1 and alog[1] == 2 and alog[16] == (POLY ^ (1 << 16))


def test_products_agree_with_textbook_polynomial_product():
    rng = random.Random(1)
    for _ in range(3000):
        a, b = rng.randrange(65536), rng.randrange(65536)
        want = gmul(a, b)
        assert oracle.gf_mul_tab(a, b) == want
        assert oracle.gf_mul_shift(a, b) == want


def test_products_exhaustive_in_one_operand():
    b = 0xB7C3
    for a in range(0, 65536, 7):
        assert oracle.gf_mul_tab(a, b) == oracle.gf_mul_shift(a, b)
    assert oracle.gf_mul_tab(0, 5) == 0 and oracle.gf_mul_tab(1, 0xABCD) == 0xABCD


def test_field_axioms():
    rng = random.Random(2)
    for _ in range(500):
        a, b, c = (rng.randrange(65536) for _ in range(3))
        assert oracle.gf_mul_tab(a, b ^ c) == oracle.gf_mul_tab(a, b) ^ oracle.gf_mul_tab(a, c)
        assert oracle.gf_mul_tab(a, b) == oracle.gf_mul_tab(b, a)
    for e in (0, 1, 15, 16, 17, 1000, 65534, 65535, 65536, 10 ** 9):
        assert oracle.gf_pow_x(e) == gpow(2, e)
