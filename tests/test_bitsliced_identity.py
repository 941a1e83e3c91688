"""The signature kernel's arithmetic for components 1, 2 and 4 (csrc/sigkey.cuh),
checked on the host against Section 3.1's definition with textbook GF(2^16)
products (gfpoly), not against the oracle.

The kernel reads a key as 32-bit words v_t = p_2t | p_2t+1 << 16 from the
start of the 32-byte block that holds its first byte (bytes before the key and
after its end zero; a key starting at an odd byte shifted down by one byte),
keeps for each bit b of a word the field element S_b = sum_t bit_b(v_t) x^t in
16 registers of 32 bits (register m holds coefficient m of every S_b), updates
them per 16-byte chunk, from the last chunk to the first, with the XOR network
of xs_chunk (S <- S x^4 + v3 x^3 + v2 x^2 + v1 x + v0), and finishes
component k in {1, 2, 4} as sum_m x^(2km) (lo16(c_m) + x^k hi16(c_m)) times
x^(-k s), s being the symbols before the key's start in its block.  The
network is taken from the kernel's source text and run here statement by
statement."""
import os
import random
import re

from gfpoly import gmul, gpow, ginv, sig_by_polynomial

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SIGKEY = os.path.join(ROOT, "paper_2411_18183_gb300", "csrc", "sigkey.cuh")
M32 = 0xFFFFFFFF


def chunk_network():
    """The body of xs_chunk as Python statements over c (a list) and v0..v3."""
    src = open(SIGKEY).read()
    m = re.search(r"void xs_chunk\(uint32_t \(&c\)\[16\], uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3\) \{(.*?)\n\}",
                  src, re.S)
    assert m, "xs_chunk not found"
    stmts = [s.strip() for s in m.group(1).replace("\n", " ").split(";") if s.strip()]
    out = []
    for s in stmts:
        s = re.sub(r"^const uint32_t\s+", "", s)
        assert re.fullmatch(r"[a-z0-9\[\]]+ = [a-z0-9\[\]\s^]+", s), s
        out.append(s)
    return compile("\n".join(out), "xs_chunk", "exec")


NET = chunk_network()


def bitsliced_state(words):
    c = [0] * 16
    for ch in range(len(words) // 4 - 1, -1, -1):
        env = {"c": c, "v0": words[4 * ch], "v1": words[4 * ch + 1], "v2": words[4 * ch + 2],
               "v3": words[4 * ch + 3]}
        exec(NET, {}, env)
        c = [x & M32 for x in env["c"]]
    return c


def finish(c, k, s):
    x = 2
    acc = 0
    for m in range(16):
        lo = c[m] & 0xFFFF
        hi = c[m] >> 16
        acc ^= gmul(gpow(x, 2 * k * m), lo ^ gmul(gpow(x, k), hi))
    return gmul(acc, ginv(gpow(x, k * s)))


def kernel_components(key: bytes, a: int):
    """Components 1, 2 and 4 of key placed at byte a (0..31) of its first block."""
    stream = bytes(a) + key
    if a & 1:
        stream = stream[1:]                          # the funnel shift of an odd start
    stream += bytes((-len(stream)) % 32 or 0)
    if not stream:
        stream = bytes(32)
    words = [int.from_bytes(stream[i:i + 4], "little") for i in range(0, len(stream), 4)]
    c = bitsliced_state(words)
    s = (a & ~1) // 2
    return {k: finish(c, k, s) for k in (1, 2, 4)}


def test_chunk_network_is_the_horner_step():
    """One network step equals S_b <- S_b x^4 + bit_b(v3) x^3 + ... + bit_b(v0), plane by plane."""
    rng = random.Random(3)
    for _ in range(200):
        c = [rng.getrandbits(32) for _ in range(16)]
        v = [rng.getrandbits(32) for _ in range(4)]
        env = {"c": list(c), "v0": v[0], "v1": v[1], "v2": v[2], "v3": v[3]}
        exec(NET, {}, env)
        for b in range(32):
            s_b = sum(((c[m] >> b) & 1) << m for m in range(16))
            want = gmul(s_b, 1 << 4) ^ sum(((v[w] >> b) & 1) << w for w in range(4))
            got = sum(((env["c"][m] >> b) & 1) << m for m in range(16))
            assert got == want, b


def test_components_one_two_four_match_the_definition():
    rng = random.Random(11)
    lengths = [0, 1, 2, 3, 15, 16, 17, 31, 32, 33, 63, 64, 65, 100, 255, 256, 257, 600, 1024, 1025]
    for it in range(240):
        n = lengths[it % len(lengths)] if it < 2 * len(lengths) else rng.randrange(0, 700)
        key = bytes(rng.randrange(256) for _ in range(n))
        a = rng.randrange(32)
        want = sig_by_polynomial(key)
        got = kernel_components(key, a)
        for k in (1, 2, 4):
            assert got[k] == (want >> (16 * (k - 1))) & 0xFFFF, (n, a, k)
