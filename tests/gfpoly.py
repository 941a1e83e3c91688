"""Textbook polynomial arithmetic over GF(2), for pinning the oracle.

Written independently of oracle/: elements of GF(2)[x] are Python ints (bit j =
coefficient of x^j); products are carry-less, remainders come from long
division.  Slow and only for small inputs."""

POLY = (1 << 16) | (1 << 12) | (1 << 3) | (1 << 1) | 1   # x^16 + x^12 + x^3 + x + 1


def clmul(a: int, b: int) -> int:
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        b >>= 1
    return r


def polymod(a: int, m: int = POLY) -> int:
    dm = m.bit_length() - 1
    while a and a.bit_length() - 1 >= dm:
        a ^= m << (a.bit_length() - 1 - dm)
    return a


def gmul(a: int, b: int) -> int:
    return polymod(clmul(a, b))


def gpow(a: int, e: int) -> int:
    r = 1
    while e:
        if e & 1:
            r = gmul(r, a)
        a = gmul(a, a)
        e >>= 1
    return r


def ginv(a: int) -> int:
    return gpow(a, 65534)


def symbols(key: bytes):
    """p_i = byte[2i] | byte[2i+1] << 8, zero high byte for an odd trailing byte."""
    b = bytes(key) + (b"\0" if len(key) % 2 else b"")
    return [b[2 * i] | (b[2 * i + 1] << 8) for i in range(len(b) // 2)]


def sig_by_polynomial(key: bytes) -> int:
    """Each component as one GF(2)[x] polynomial sum_i p_i(x) x^(k i), reduced once."""
    out = 0
    ps = symbols(key)
    for k in range(1, 5):
        big = 0
        for i, p in enumerate(ps):
            big ^= p << (k * i)
        out |= polymod(big) << (16 * (k - 1))
    return out


def solve(M, rhs):
    """Gaussian elimination over GF(2^16); M square list of lists."""
    n = len(M)
    A = [list(row) + [r] for row, r in zip(M, rhs)]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c])
        A[c], A[piv] = A[piv], A[c]
        inv = ginv(A[c][c])
        A[c] = [gmul(v, inv) for v in A[c]]
        for r in range(n):
            if r != c and A[r][c]:
                f = A[r][c]
                A[r] = [v ^ gmul(f, w) for v, w in zip(A[r], A[c])]
    return [A[r][n] for r in range(n)]


# ---- byte symbols: GF(2^8) with x^8 + x^4 + x^3 + x^2 + 1 -------------------

POLY8 = (1 << 8) | (1 << 4) | (1 << 3) | (1 << 2) | 1


def gmul8(a: int, b: int) -> int:
    return polymod(clmul(a, b), POLY8)


def gpow8(a: int, e: int) -> int:
    r = 1
    while e:
        if e & 1:
            r = gmul8(r, a)
        a = gmul8(a, a)
        e >>= 1
    return r


def sig8_by_polynomial(key: bytes) -> int:
    """Each component as one GF(2)[x] polynomial sum_i b_i(x) x^(k i), reduced once."""
    out = 0
    for k in range(1, 5):
        big = 0
        for i, b in enumerate(bytes(key)):
            big ^= b << (k * i)
        out |= polymod(big, POLY8) << (8 * (k - 1))
    return out


def solve8(M, rhs):
    """Gaussian elimination over GF(2^8): M x = rhs (M square, non-singular)."""
    n = len(M)
    A = [list(M[r]) + [rhs[r]] for r in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if A[r][c])
        A[c], A[p] = A[p], A[c]
        inv = gpow8(A[c][c], 254)
        A[c] = [gmul8(v, inv) for v in A[c]]
        for r in range(n):
            if r != c and A[r][c]:
                f = A[r][c]
                A[r] = [v ^ gmul8(f, w) for v, w in zip(A[r], A[c])]
    return [A[r][n] for r in range(n)]
