"""The component-3 network of the signature kernel (csrc/xs3_net.h) is what
csrc/gen_xs3.py writes, and that script's self-check holds: the bit-sliced
Horner step over theta = x^1536 in its basis, followed by the map back to
polynomial coordinates, gives sum_t (p_2t + x^3 p_2t+1) x^(6t) in GF(2^16)
for random words (so the header computes component 3 of Section 3.1)."""
import importlib.util
import os
import random

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2411_18183_gb300", "csrc")


def load_gen():
    spec = importlib.util.spec_from_file_location("gen_xs3", os.path.join(CSRC, "gen_xs3.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_header_is_the_generator_output():
    gen = load_gen()
    step, to_poly, *_ = gen.networks()
    with open(os.path.join(CSRC, "xs3_net.h")) as f:
        assert f.read() == gen.emit(step, to_poly)


def test_network_computes_component_three():
    gen = load_gen()
    step, to_poly, *_ = gen.networks()
    gen.check(step, to_poly, trials=300)


def test_network_against_an_independent_horner():
    """The same check with a textbook carry-less product and reduction
    written here, on keys of 1 to 12 chunks."""
    gen = load_gen()
    step, to_poly, *_ = gen.networks()
    P = 0x1100B

    def clmul(a, b):
        r = 0
        while b:
            if b & 1:
                r ^= a
            a <<= 1
            b >>= 1
        return r

    def mod(a):
        for bit in range(a.bit_length() - 1, 15, -1):
            if (a >> bit) & 1:
                a ^= P << (bit - 16)
        return a

    def run(terms, env):
        r = 0
        for t in terms:
            r ^= env[t]
        return r

    rng = random.Random(7)
    for _ in range(100):
        nw = 4 * rng.randrange(1, 13)
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
            got ^= (p[i] & 0xFFFF) << i ^ clmul(p[i] >> 16, 8) << i
        got = mod(got)
        # Horner in x^6 over the words' symbols: sum_t (lo + x^3 hi) x^(6t)
        want = 0
        for v in reversed(words):
            want = mod(clmul(want, 1 << 6) ^ (v & 0xFFFF) ^ clmul(v >> 16, 8))
        assert got == want
