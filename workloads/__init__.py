"""Seeded synthetic relations for the signature equi-join.

Holds no part of the method's arithmetic: it only produces key bytes, offsets
and ids, plus the ground truth of how they were made (which S rows copy which R
row).  The same (spec, seed) gives the same bytes on any machine.  Both the CPU
oracle and the CUDA path are fed from here.

The recipes stand in for the random tuples of the paper's experiments (Section
4.2: randomly generated tuples, string join attribute); the sizes and
distributions are the five workloads this package is measured on.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libgen.so")
_lock = threading.Lock()
_lib = None

ALPHABETS = {"printable": 0, "acgt": 1, "alnum": 2, "bytes": 3, "xml": 4}


class _Spec(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64), ("m", ctypes.c_uint64), ("n", ctypes.c_uint64),
        ("r_len_lo", ctypes.c_uint32), ("r_len_hi", ctypes.c_uint32),
        ("s_len_lo", ctypes.c_uint32), ("s_len_hi", ctypes.c_uint32),
        ("alphabet", ctypes.c_int32),
        ("frac_copy", ctypes.c_double), ("frac_near", ctypes.c_double),
        ("near_lo", ctypes.c_int32), ("near_hi", ctypes.c_int32),
        ("zipf_s", ctypes.c_double), ("dup_frac", ctypes.c_double),
        ("dup_lo", ctypes.c_int32), ("dup_hi", ctypes.c_int32),
    ]


@dataclasses.dataclass(frozen=True)
class JoinSpec:
    """Shape of one synthetic join R x S."""
    m: int                      # |R|
    n: int                      # |S|
    r_len: tuple                # R key length range, inclusive
    s_len: tuple                # fresh S key length range, inclusive
    alphabet: str = "printable"
    frac_copy: float = 0.0      # S rows that are exact copies of an R key
    frac_near: float = 0.0      # S rows that are near-duplicates of an R key
    near: tuple = (1, 6)        # changed byte positions of a near-duplicate
    zipf_s: float = 0.0         # partner choice: 0 uniform, else Zipf(s) over R rows
    dup_frac: float = 0.0       # distinct R keys that occur several times
    dup: tuple = (2, 8)         # total occurrences of such a key
    seed: int = 20081

    def scaled(self, m: int, n: int) -> "JoinSpec":
        return dataclasses.replace(self, m=m, n=n)


# The workloads.  Seeds follow 20081 + index of the workload.
CONFIGS = {
    # 10k x 100k, printable keys of 64-256 B, 30% of S copies a uniform R key, R unique
    "plain": JoinSpec(m=10_000, n=100_000, r_len=(64, 256), s_len=(64, 256), alphabet="printable",
                      frac_copy=0.30, seed=20081),
    # 1M x 10M, printable keys of 256-1024 B; 50% of S copies an R row chosen by Zipf(1.1);
    # 1% of distinct R keys occur 2-8 times
    "large": JoinSpec(m=1_000_000, n=10_000_000, r_len=(256, 1024), s_len=(256, 1024), alphabet="printable",
                      frac_copy=0.50, zipf_s=1.1, dup_frac=0.01, dup=(2, 8), seed=20082),
    # 100k x 1M, ACGT keys of 2048-8192 B; 40% exact copies, 40% near-duplicates (1-6 changed bytes)
    "collision": JoinSpec(m=100_000, n=1_000_000, r_len=(2048, 8192), s_len=(2048, 8192), alphabet="acgt",
                          frac_copy=0.40, frac_near=0.40, near=(1, 6), seed=20083),
}
# Profiling case: the shape of "large" at one fifth of the size (still larger than L2).
CONFIGS["medium"] = dataclasses.replace(CONFIGS["large"], m=200_000, n=2_000_000)


def _build_lib() -> None:
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp,
                           os.path.join(_HERE, "gen.c"), "-lm"])
    os.replace(tmp, _SO)


def build(device: bool = True) -> str:
    """Compile the host generator (gcc) and, with device=True, the device
    generator (nvcc, sm_103a)."""
    with _lock:
        _build_lib()
    if device:
        from . import device as _device
        _device.build()
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        srcs = [os.path.join(_HERE, f) for f in ("gen.c", "genrng.h")]
        if not os.path.exists(_SO) or os.path.getmtime(_SO) < max(os.path.getmtime(f) for f in srcs):
            _build_lib()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        lib.gen_plan.argtypes = [ctypes.POINTER(_Spec), P, P, P, P, P, P]
        lib.gen_plan.restype = ctypes.c_int
        lib.gen_fill_R.argtypes = [ctypes.POINTER(_Spec), P, P, P, ctypes.c_int]
        lib.gen_fill_S.argtypes = [ctypes.POINTER(_Spec), P, P, P, P, P, P, ctypes.c_int]
        lib.gen_key_bytes.argtypes = [ctypes.POINTER(_Spec), ctypes.c_uint64, ctypes.c_uint64, P, ctypes.c_uint64]
        lib.gen_perm_x.argtypes = [ctypes.c_uint64] * 4
        lib.gen_perm_x.restype = ctypes.c_uint64
        lib.gen_n_copy.argtypes = [ctypes.c_double, ctypes.c_uint64]
        lib.gen_n_copy.restype = ctypes.c_uint64
        _lib = lib
        return lib


def _cspec(sp: JoinSpec) -> _Spec:
    return _Spec(sp.seed, sp.m, sp.n, sp.r_len[0], sp.r_len[1], sp.s_len[0], sp.s_len[1],
                 ALPHABETS[sp.alphabet], sp.frac_copy, sp.frac_near, sp.near[0], sp.near[1],
                 sp.zipf_s, sp.dup_frac, sp.dup[0], sp.dup[1])


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclasses.dataclass
class Relation:
    """A packed relation: key i is arena[off[i]:off[i+1]], its id is ids[i].

    The arena array is padded to a multiple of 16 bytes plus 16 zero bytes, so
    every 16-byte aligned chunk that holds a key byte can be read whole."""
    arena: np.ndarray   # uint8
    off: np.ndarray     # uint64[n+1]
    ids: np.ndarray     # uint32[n]

    @property
    def n(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def nbytes(self) -> int:
        return int(self.off[-1] - self.off[0])

    def key(self, i: int) -> bytes:
        return bytes(self.arena[int(self.off[i]):int(self.off[i + 1])])

    def lengths(self) -> np.ndarray:
        return np.diff(self.off)


def padded_size(nbytes: int) -> int:
    return ((nbytes + 15) // 16) * 16 + 16


def relation_from_keys(keys, ids=None) -> Relation:
    """Pack a list of byte strings into a relation (for small hand-made cases)."""
    lens = np.array([len(k) for k in keys], dtype=np.uint64)
    off = np.zeros(len(keys) + 1, dtype=np.uint64)
    if len(keys):
        np.cumsum(lens, out=off[1:])
    arena = np.zeros(padded_size(int(off[-1])), dtype=np.uint8)
    pos = 0
    for k in keys:
        arena[pos:pos + len(k)] = np.frombuffer(bytes(k), dtype=np.uint8)
        pos += len(k)
    if ids is None:
        ids = np.arange(len(keys), dtype=np.uint32)
    return Relation(arena, off, np.asarray(ids, dtype=np.uint32))


@dataclasses.dataclass
class Workload:
    spec: JoinSpec
    R: Relation
    S: Relation
    r_mult: np.ndarray   # uint32[m]: R rows holding the same key as row r
    s_kind: np.ndarray   # uint8[n]: 0 fresh, 1 exact copy, 2 near-duplicate
    s_src: np.ndarray    # int64[n]: R row copied, or -1

    def expected_pairs(self) -> int:
        """Pair count implied by the construction: every exact copy of R row r
        joins every R row holding r's key.  (Fresh random keys and
        near-duplicates are assumed to join nothing; the oracle checks this.)"""
        src = self.s_src[self.s_kind == 1]
        return int(self.r_mult[src].astype(np.int64).sum())


def generate(spec: JoinSpec, nthreads: int | None = None, alloc=None) -> Workload:
    """Generate R and S for `spec`.

    `alloc(nbytes) -> np.ndarray[uint8]` may supply the arena buffers (for
    example views of pinned host memory); by default numpy allocates them."""
    lib = _load()
    cs = _cspec(spec)
    m, n = spec.m, spec.n
    if nthreads is None:
        nthreads = max(1, min(32, os.cpu_count() or 1))
    r_ident = np.empty(max(m, 1), dtype=np.uint64)
    r_len = np.empty(max(m, 1), dtype=np.uint32)
    r_mult = np.empty(max(m, 1), dtype=np.uint32)
    s_kind = np.empty(max(n, 1), dtype=np.uint8)
    s_src = np.empty(max(n, 1), dtype=np.int64)
    s_len = np.empty(max(n, 1), dtype=np.uint32)
    rc = lib.gen_plan(ctypes.byref(cs), _ptr(r_ident), _ptr(r_len), _ptr(r_mult),
                      _ptr(s_kind), _ptr(s_src), _ptr(s_len))
    if rc != 0:
        raise MemoryError("workload plan failed")
    offR = np.zeros(m + 1, dtype=np.uint64)
    np.cumsum(r_len[:m], out=offR[1:])
    offS = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(s_len[:n], out=offS[1:])

    def _arena(nb):
        size = padded_size(nb)
        if alloc is None:
            a = np.empty(size, dtype=np.uint8)
        else:
            a = alloc(size)
        a[nb:size] = 0
        return a

    aR = _arena(int(offR[-1]))
    aS = _arena(int(offS[-1]))
    lib.gen_fill_R(ctypes.byref(cs), _ptr(r_ident), _ptr(offR), _ptr(aR), nthreads)
    lib.gen_fill_S(ctypes.byref(cs), _ptr(s_kind), _ptr(s_src), _ptr(offS), _ptr(aS),
                   _ptr(offR), _ptr(aR), nthreads)
    R = Relation(aR, offR, np.arange(m, dtype=np.uint32))
    S = Relation(aS, offS, np.arange(n, dtype=np.uint32))
    return Workload(spec, R, S, r_mult[:m].copy(), s_kind[:n].copy(), s_src[:n].copy())


def key_bytes(spec: JoinSpec, rel: int, ident: int, length: int) -> bytes:
    lib = _load()
    cs = _cspec(spec)
    buf = np.zeros(max(length, 1), dtype=np.uint8)
    lib.gen_key_bytes(ctypes.byref(cs), rel, ident, _ptr(buf), length)
    return bytes(buf[:length])


def perm(seed: int, tag: int, n: int, x: int) -> int:
    return int(_load().gen_perm_x(seed, tag, n, x))


def n_copy(frac_copy: float, n: int) -> int:
    """S rows that copy an R key in a relation of n S rows (C llround, as the plan counts them)."""
    return int(_load().gen_n_copy(frac_copy, n))


# ----------------------------------------------------------------------------- batches of joins

@dataclasses.dataclass(frozen=True)
class BatchSpec:
    """Many independent joins of uneven sizes and key lengths (packed in one R
    and one S relation).  |R_j| is log-normal (median, sigma) clipped to
    r_range; |S_j| = s_factor |R_j|; each join draws one key-length band."""
    n_joins: int = 512
    r_median: float = 20_000
    sigma: float = 1.0
    r_range: tuple = (1_000, 1_000_000)
    s_factor: int = 10
    bands: tuple = ((32, 128), (256, 1024), (2048, 8192))
    frac_copy: float = 0.25
    alphabet: str = "printable"
    seed: int = 20084
    s_factor_range: tuple | None = None     # (lo, hi): |S_j| / |R_j| uniform per join instead of s_factor

    def scaled(self, factor: float, n_joins: int | None = None) -> "BatchSpec":
        """Relation sizes divided by `factor` (the shape is kept)."""
        return dataclasses.replace(self, r_median=self.r_median / factor,
                                   r_range=(max(1, int(self.r_range[0] / factor)), max(1, int(self.r_range[1] / factor))),
                                   n_joins=self.n_joins if n_joins is None else n_joins)

    def joins(self):
        """The JoinSpec of every join (pure function of the seed)."""
        rng = np.random.default_rng(self.seed)
        sizes = np.exp(rng.normal(np.log(self.r_median), self.sigma, self.n_joins))
        sizes = np.clip(np.rint(sizes), self.r_range[0], self.r_range[1]).astype(np.int64)
        bands = rng.integers(0, len(self.bands), self.n_joins)
        if self.s_factor_range is None:
            factors = [self.s_factor] * self.n_joins
        else:
            factors = rng.integers(self.s_factor_range[0], self.s_factor_range[1] + 1, self.n_joins).tolist()
        out = []
        for j in range(self.n_joins):
            lo, hi = self.bands[bands[j]]
            m = int(sizes[j])
            out.append(JoinSpec(m=m, n=int(factors[j]) * m, r_len=(lo, hi), s_len=(lo, hi), alphabet=self.alphabet,
                                frac_copy=self.frac_copy, seed=self.seed * 1_000_003 + j))
        return out


# Requests of the serving loop: |R| log-normal (median 50,000), |S| = 4-16 |R|,
# XML-like keys of 200-2000 bytes, 20% of S copies an R key.  The pool holds
# the distinct joins that requests ask for.
SERVE_SPEC = BatchSpec(n_joins=64, r_median=50_000, sigma=1.0, r_range=(1_000, 1_000_000), s_factor_range=(4, 16),
                       bands=((200, 2000),), frac_copy=0.20, alphabet="xml", seed=20085)
SERVE_RATE = 2000.0                 # mean arrivals per second (Poisson)
SERVE_BUDGET_BYTES = 120 * 10 ** 9  # admission bound on device memory


@dataclasses.dataclass
class BatchWorkload:
    spec: BatchSpec
    R: Relation
    S: Relation
    ranges: list          # (r_begin, r_end, s_begin, s_end) per join
    expected: list        # pair count implied by the construction, per join
    joins: list           # per-join Workload (views are not kept; for the oracle, see join_relations)

    def join_relations(self, j: int):
        """R and S of join j as stand-alone relations (ids = join-local rows)."""
        rb, re_, sb, se = self.ranges[j]
        def sub(rel, a, b):
            off = rel.off[a:b + 1]
            base = int(off[0])
            arena = rel.arena[base: int(off[-1])]
            pad = np.zeros(padded_size(arena.shape[0]), dtype=np.uint8)
            pad[: arena.shape[0]] = arena
            return Relation(pad, (off - np.uint64(base)).astype(np.uint64), np.arange(b - a, dtype=np.uint32))
        return sub(self.R, rb, re_), sub(self.S, sb, se)


def generate_batch(spec: BatchSpec, nthreads: int | None = None, alloc=None) -> BatchWorkload:
    """Generate every join and pack them into one R and one S relation."""
    specs = spec.joins()
    parts = [generate(js, nthreads=nthreads) for js in specs]
    mR = sum(p.R.n for p in parts)
    nS = sum(p.S.n for p in parts)
    bR = sum(p.R.nbytes for p in parts)
    bS = sum(p.S.nbytes for p in parts)

    def _arena(nb):
        size = padded_size(nb)
        a = np.empty(size, dtype=np.uint8) if alloc is None else alloc(size)
        a[nb:size] = 0
        return a

    aR, aS = _arena(bR), _arena(bS)
    offR = np.zeros(mR + 1, dtype=np.uint64)
    offS = np.zeros(nS + 1, dtype=np.uint64)
    ranges, expected = [], []
    r0 = s0 = 0
    pr = ps = 0
    for p in parts:
        aR[pr: pr + p.R.nbytes] = p.R.arena[: p.R.nbytes]
        aS[ps: ps + p.S.nbytes] = p.S.arena[: p.S.nbytes]
        offR[r0: r0 + p.R.n + 1] = p.R.off + np.uint64(pr)
        offS[s0: s0 + p.S.n + 1] = p.S.off + np.uint64(ps)
        ranges.append((r0, r0 + p.R.n, s0, s0 + p.S.n))
        expected.append(p.expected_pairs())
        r0 += p.R.n
        s0 += p.S.n
        pr += p.R.nbytes
        ps += p.S.nbytes
    R = Relation(aR, offR, np.arange(mR, dtype=np.uint32))
    S = Relation(aS, offS, np.arange(nS, dtype=np.uint32))
    return BatchWorkload(spec, R, S, ranges, expected, [])
