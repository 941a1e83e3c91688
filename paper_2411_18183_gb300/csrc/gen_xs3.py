"""Writes xs3_net.h: the bit-sliced Horner step of signature component 3 and
the map from its state to polynomial coordinates, as XOR networks.

Component 3 of Section 3.1 is sig^3 = sum_i p_i x^(3 i).  With the key read as
32-bit words v_t = p_{2t} | p_{2t+1} << 16 and D_b(y) = sum_t bit_b(v_t) y^t for
each bit position b,
    sig^3 = sum_b W_3(b) D_b(x^6),  W_3(b) = x^b (b < 16), x^(b - 13) (b >= 16).
x^6 = (x^3)^2, and theta = x^(3 * 2^9) = (x^3)^(2^9) is another Frobenius
conjugate of x^3, so D_b(x^6) = Frob^8(D_b(theta)) (Frob: squaring, of order
16 on GF(2^16)).  The kernel keeps the 32 elements D_b(theta) bit-sliced in 16
registers c_m (bit b of c_m = coordinate m of D_b(theta) in a basis B of
GF(2^16) over GF(2)), and Horner's rule over a 16-byte chunk,
    S <- S theta^4 + v3 theta^3 + v2 theta^2 + v1 theta + v0,
is a fixed GF(2)-linear map of (c, v0..v3): one XOR of a few inputs per
register.  Any invertible B gives the same signatures; the basis below was
found by a hill-climbing search over column operations (starting from the
powers of theta) for few XOR inputs, 13 three-input operations per chunk
against 12 for the x-step of components 1, 2 and 4.  At the end of a key,
poly coordinate i of D_b(x^6) is the XOR over m of A[i][m] c_m, A = Frob^8 B.

    python gen_xs3.py          # rewrites xs3_net.h next to this file
"""
from __future__ import annotations

import os
import random

POLY = 0x1100B          # x^16 + x^12 + x^3 + x + 1
EXP = 3 * 2 ** 9        # theta = x^EXP
BASIS = [1, 90, 7072, 48591, 4420, 51313, 25705, 17465, 27996, 15014, 31987, 24859, 8236, 11170, 32323, 31573]


def gmul(a: int, b: int) -> int:
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a & 0x10000:
            a ^= POLY
    return r


def gpow(a: int, e: int) -> int:
    r = 1
    e %= 65535
    while e:
        if e & 1:
            r = gmul(r, a)
        a = gmul(a, a)
        e >>= 1
    return r


def mat_cols(f) -> list[int]:
    """Columns (as 16-bit ints, poly coordinates) of the GF(2)-linear map f."""
    return [f(1 << j) for j in range(16)]


def mat_mul(A: list[int], B: list[int]) -> list[int]:
    """Columns of A @ B (both given by columns)."""
    def apply(cols, v):
        r = 0
        for j in range(16):
            if (v >> j) & 1:
                r ^= cols[j]
        return r
    return [apply(A, b) for b in B]


def mat_inv(cols: list[int]) -> list[int]:
    rows = [sum(((cols[j] >> i) & 1) << j for j in range(16)) | (1 << (16 + i)) for i in range(16)]
    for c in range(16):
        p = next(r for r in range(c, 16) if (rows[r] >> c) & 1)
        rows[c], rows[p] = rows[p], rows[c]
        for r in range(16):
            if r != c and (rows[r] >> c) & 1:
                rows[r] ^= rows[c]
    inv_rows = [rows[i] >> 16 for i in range(16)]
    return [sum(((inv_rows[i] >> j) & 1) << i for i in range(16)) for j in range(16)]


def apply(cols: list[int], v: int) -> int:
    r = 0
    for j in range(16):
        if (v >> j) & 1:
            r ^= cols[j]
    return r


def networks():
    theta = gpow(2, EXP)
    B = BASIS
    Binv = mat_inv(B)
    Mth = mat_cols(lambda v: gmul(theta, v))
    Mb = mat_mul(Binv, mat_mul(Mth, B))           # multiplication by theta in basis B
    inj = apply(Binv, 1)                          # the element 1 in basis B
    powers = [[1 << j for j in range(16)]]                 # Mb^0 .. Mb^4
    for _ in range(4):
        powers.append(mat_mul(Mb, powers[-1]))
    M4 = powers[4]
    # row i of the chunk step: state registers j with M4[i][j] = 1, words w with (Mb^w inj)[i] = 1
    step = []
    for i in range(16):
        terms = [f"c[{j}]" for j in range(16) if (M4[j] >> i) & 1]
        for w in range(4):
            if (apply(powers[w], inj) >> i) & 1:
                terms.append(f"v{w}")
        step.append(terms)
    F8 = mat_cols(lambda v: gpow(v, 2 ** 8) if v else 0)   # Frob^8 is linear
    A = mat_mul(F8, B)
    to_poly = [[f"c[{m}]" for m in range(16) if (A[m] >> i) & 1] for i in range(16)]
    return step, to_poly, Mb, inj, A


def check(step, to_poly, trials: int = 200) -> None:
    """Simulate both networks on random words and compare with a direct
    evaluation of sum_t (p_2t + x^3 p_2t+1) x^(6t) in GF(2^16)."""
    rng = random.Random(1)

    def run(terms, env):
        r = 0
        for t in terms:
            r ^= env[t]
        return r
    for _ in range(trials):
        nw = 4 * rng.randrange(1, 9)
        words = [rng.getrandbits(32) for _ in range(nw)]
        c = [0] * 16
        for ch in range(nw // 4 - 1, -1, -1):
            env = {f"c[{j}]": c[j] for j in range(16)}
            env.update({f"v{w}": words[4 * ch + w] for w in range(4)})
            c = [run(step[i], env) for i in range(16)]
        env = {f"c[{j}]": c[j] for j in range(16)}
        p = [run(to_poly[i], env) for i in range(16)]
        got = 0
        for i in range(16):
            lo, hi = p[i] & 0xFFFF, p[i] >> 16
            got ^= gmul(gpow(2, i), lo ^ gmul(hi, 8))
        want = 0
        for t, v in enumerate(words):
            want ^= gmul(gpow(2, 6 * t), (v & 0xFFFF) ^ gmul(v >> 16, 8))
        assert got == want, (got, want)


def xor_expr(terms) -> str:
    return " ^ ".join(terms) if terms else "0u"


def emit(step, to_poly) -> str:
    ops = sum(len(t) // 2 for t in step)                    # ceil((terms - 1) / 2) per register
    lines = [
        "// xs3_net.h -- written by gen_xs3.py; do not edit by hand.",
        "//",
        "// Bit-sliced Horner step of signature component 3 (sig^3 = sum_i p_i x^(3i),",
        f"// Section 3.1) over theta = x^{EXP}, in the basis of GF(2^16) given in",
        f"// gen_xs3.py, and the map of its state to polynomial coordinates of D_b(x^6).",
        f"// {ops} three-input XORs per 16-byte chunk.",
        "#pragma once",
        "",
        "namespace algsig {",
        "",
        "// S <- S theta^4 + v3 theta^3 + v2 theta^2 + v1 theta + v0 (v3 last in the key)",
        "__device__ __forceinline__ void xs3_chunk(uint32_t (&c)[16], uint32_t v0, uint32_t v1, uint32_t v2,",
        "                                          uint32_t v3) {",
    ]
    for i in range(16):
        lines.append(f"  const uint32_t n{i} = {xor_expr(step[i])};")
    lines.append("  " + " ".join(f"c[{i}] = n{i};" for i in range(8)))
    lines.append("  " + " ".join(f"c[{i}] = n{i};" for i in range(8, 16)))
    lines += [
        "}",
        "",
        "// p_i: bit b = coefficient of x^i in D_b(x^6)",
        "__device__ __forceinline__ void xs3_to_poly(const uint32_t (&c)[16], uint32_t (&p)[16]) {",
    ]
    for i in range(16):
        lines.append(f"  p[{i}] = {xor_expr(to_poly[i])};")
    lines += ["}", "", "}  // namespace algsig", ""]
    return "\n".join(lines)


def main() -> None:
    step, to_poly, *_ = networks()
    check(step, to_poly)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "xs3_net.h")
    with open(out, "w") as f:
        f.write(emit(step, to_poly))
    print(out)


if __name__ == "__main__":
    main()
