"""Hand-made test inputs shared by the oracle tests and the GPU parity tests."""
import random

from gfpoly import gmul, gpow, solve, symbols


def symbol_collision(n_components: int, length_symbols: int, positions, seed: int = 7):
    """Two keys of equal length that differ in exactly n+1 symbols and have the
    same n-component signature.  The difference vector d (d_j at position i_j)
    must satisfy sum_j d_j x^(k i_j) = 0 for k = 1..n: n equations in n+1
    unknowns; fix the last d_j = 1 and solve the (Vandermonde) n x n system."""
    n = n_components
    rng = random.Random(seed)
    i = list(positions)
    assert len(i) == n + 1 and len(set(i)) == n + 1 and max(i) < length_symbols
    M = [[gpow(2, k * i[j]) for j in range(n)] for k in range(1, n + 1)]
    rhs = [gpow(2, k * i[n]) for k in range(1, n + 1)]
    d = solve(M, rhs) + [1]
    assert all(d), "degenerate solution"
    a = [rng.randrange(0x2020, 0x7E7E) for _ in range(length_symbols)]
    b = list(a)
    for pos, dj in zip(i, d):
        b[pos] ^= dj
    ka = b"".join(v.to_bytes(2, "little") for v in a)
    kb = b"".join(v.to_bytes(2, "little") for v in b)
    assert ka != kb and sum(x != y for x, y in zip(symbols(ka), symbols(kb))) == n + 1
    return ka, kb


def five_symbol_collision(length_symbols: int = 24, positions=(1, 4, 9, 15, 22), seed: int = 7):
    """Two keys of equal length that differ in exactly 5 symbols and have the
    same 4-component signature (symbol_collision with n = 4)."""
    return symbol_collision(4, length_symbols, positions, seed)


def edge_keys():
    """Keys that stress the symbol packing and the equality test."""
    ka, kb = five_symbol_collision()
    return [b"", b"", b"A", b"A\0", b"\0", b"\0\0", b"AB", b"AB", b"ABC", b"ABCD", b"Paul Sabatier University",
            b"\0" * 17, b"\xff" * 33, ka, kb, bytes(range(256)), bytes(range(255, -1, -1))]
