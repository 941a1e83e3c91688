"""CPU oracle for the algebraic-signature equi-join -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check in __graft_entry__ and bench.py's CPU-baseline /
reference arm may import this package.  The product path (the CUDA library and
its binding) never does, and this package never imports the product.

It wraps oracle.c, a plain C statement of:
  * GF(2^16) arithmetic with log/antilog tables and a shift-and-add product
    (Section 3.1 of the paper);
  * the 4-component algebraic signature sig^k(P) = sum_i p_i x^(k i), once by
    the table definition and once by Horner's rule (Section 3.1);
  * cumulative signatures (the signatures of a key's block prefixes), by
    definition from the signature routine, in Python;
  * the GF(2^8) byte-symbol signature (field polynomial x^8+x^4+x^3+x^2+1),
    by the table definition and by Horner's rule (Section 3.1's other symbol
    size);
  * the n-component signature (the first n of the four components) and the
    signature-only join of Figure 2 (pairs of equal signature and length, no
    byte comparison; not exact, kept to count collisions), in Python;
  * the prefix join T_L = {(r.id, s.id) : key(r)[:L] == key(s)[:L]} (the join
    on the keys' first L bytes that cumulative signatures serve), in Python;
  * the exact equi-join T = {(r.id, s.id) : key(r) == key(s)} by a nested loop,
    a simple hash join on full strings and a Grace (partitioned) hash join
    (Section 2; Figure 2 without the signature shortcut, since the result must
    be exact).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

POLY = 0x1100B          # x^16 + x^12 + x^3 + x + 1
ORDER = 65535


def _build_lib() -> None:
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp,
                           os.path.join(_HERE, "oracle.c")])
    os.replace(tmp, _SO)


def build() -> str:
    with _lock:
        _build_lib()
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        src = os.path.join(_HERE, "oracle.c")
        if not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
            _build_lib()
        lib = ctypes.CDLL(_SO)
        P, U64, U16 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint16
        lib.or_gf_init.restype = ctypes.c_int
        lib.or_gf_tables.argtypes = [P, P]
        lib.or_gf_mul_tab.argtypes = [U16, U16]
        lib.or_gf_mul_tab.restype = U16
        lib.or_gf_mul_shift.argtypes = [U16, U16]
        lib.or_gf_mul_shift.restype = U16
        lib.or_gf_pow_x.argtypes = [U64]
        lib.or_gf_pow_x.restype = U16
        lib.or_sig_tables.argtypes = [P, U64]
        lib.or_sig_tables.restype = U64
        lib.or_sig_horner.argtypes = [P, U64]
        lib.or_sig_horner.restype = U64
        lib.or_sig_batch.argtypes = [P, P, U64, P, ctypes.c_int, ctypes.c_int]
        lib.or_gf8_init.restype = ctypes.c_int
        lib.or_gf8_tables.argtypes = [P, P]
        lib.or_sig8_tables.argtypes = [P, U64]
        lib.or_sig8_tables.restype = U64
        lib.or_sig8_horner.argtypes = [P, U64]
        lib.or_sig8_horner.restype = U64
        lib.or_sig8_batch.argtypes = [P, P, U64, P, ctypes.c_int, ctypes.c_int]
        for f in (lib.or_join_nested, lib.or_join_simple):
            f.argtypes = [P, P, P, U64, P, P, P, U64, P, U64]
            f.restype = U64
        lib.or_join_grace.argtypes = [P, P, P, U64, P, P, P, U64, P, U64, ctypes.c_int, ctypes.c_int]
        lib.or_join_grace.restype = U64
        if not lib.or_gf_init():
            raise RuntimeError("oracle: x is not primitive under the field polynomial")
        if not lib.or_gf8_init():
            raise RuntimeError("oracle: x is not primitive under the GF(2^8) polynomial")
        _lib = lib
        return lib


def _buf(b: bytes):
    a = np.frombuffer(bytes(b) + b"\0", dtype=np.uint8)
    return a, a.ctypes.data


# ---------------------------------------------------------------- GF(2^16)

def gf_tables():
    """(log[65536], antilog[65535]) as uint16 arrays."""
    lib = _load()
    log = np.zeros(65536, dtype=np.uint16)
    alog = np.zeros(65535, dtype=np.uint16)
    lib.or_gf_tables(log.ctypes.data, alog.ctypes.data)
    return log, alog


def gf_mul_tab(a: int, b: int) -> int:
    return int(_load().or_gf_mul_tab(a, b))


def gf_mul_shift(a: int, b: int) -> int:
    return int(_load().or_gf_mul_shift(a, b))


def gf_pow_x(e: int) -> int:
    return int(_load().or_gf_pow_x(e))


# ---------------------------------------------------------------- signatures

def sig(key: bytes, method: str = "tables") -> int:
    """Packed 64-bit signature of one key: component k (1..4) in bits [16(k-1), 16k)."""
    lib = _load()
    arr, p = _buf(key)
    f = lib.or_sig_tables if method == "tables" else lib.or_sig_horner
    return int(f(p, len(key)))


def components(s: int):
    return tuple((s >> (16 * k)) & 0xFFFF for k in range(4))


POLY8 = 0x11D           # x^8 + x^4 + x^3 + x^2 + 1 (byte symbols)
ORDER8 = 255


def gf8_tables():
    """(log[256], antilog[255]) of GF(2^8) as uint8 arrays."""
    lib = _load()
    log = np.zeros(256, dtype=np.uint8)
    alog = np.zeros(255, dtype=np.uint8)
    lib.or_gf8_tables(log.ctypes.data, alog.ctypes.data)
    return log, alog


def sig8(key: bytes, method: str = "tables") -> int:
    """Signature over GF(2^8) with byte symbols (the paper's other symbol size):
    sig^k = sum_i b_i x^(k i), k = 1..4, component k in bits [8(k-1), 8k)."""
    lib = _load()
    arr, p = _buf(key)
    f = lib.or_sig8_tables if method == "tables" else lib.or_sig8_horner
    return int(f(p, len(key)))


def sig8_batch(arena: np.ndarray, off: np.ndarray, method: str = "tables", nthreads: int = 1) -> np.ndarray:
    lib = _load()
    n = off.shape[0] - 1
    out = np.zeros(max(n, 1), dtype=np.uint64)
    arena = np.ascontiguousarray(arena)
    off = np.ascontiguousarray(off, dtype=np.uint64)
    lib.or_sig8_batch(arena.ctypes.data, off.ctypes.data, n, out.ctypes.data, 0 if method == "tables" else 1, nthreads)
    return out[:n]


def component_mask(n_components: int) -> int:
    """Bits of the packed signature that hold components 1..n (Section 3.1: the
    n-symbol signature is the vector of the first n components)."""
    if n_components not in (1, 2, 3, 4):
        raise ValueError(n_components)
    return (1 << (16 * n_components)) - 1


def sig_batch(arena: np.ndarray, off: np.ndarray, method: str = "tables", nthreads: int = 1) -> np.ndarray:
    lib = _load()
    n = off.shape[0] - 1
    out = np.zeros(max(n, 1), dtype=np.uint64)
    arena = np.ascontiguousarray(arena)
    off = np.ascontiguousarray(off, dtype=np.uint64)
    lib.or_sig_batch(arena.ctypes.data, off.ctypes.data, n, out.ctypes.data,
                     0 if method == "tables" else 1, nthreads)
    return out[:n]


# ---------------------------------------------------------------- joins

def _rel_ptrs(rel):
    arena = np.ascontiguousarray(rel.arena)
    off = np.ascontiguousarray(rel.off, dtype=np.uint64)
    ids = np.ascontiguousarray(rel.ids, dtype=np.uint32)
    return (arena, off, ids), (arena.ctypes.data, off.ctypes.data, ids.ctypes.data, off.shape[0] - 1)


def _run_join(fn, R, S, extra=(), cap_hint=None):
    keepR, pr = _rel_ptrs(R)
    keepS, ps = _rel_ptrs(S)
    cap = cap_hint if cap_hint is not None else max(1024, ps[3])
    while True:
        out = np.zeros(2 * max(cap, 1), dtype=np.uint32)
        cnt = int(fn(*pr, *ps, out.ctypes.data, cap, *extra))
        if cnt <= cap:
            return sort_pairs(out[:2 * cnt].reshape(-1, 2))
        cap = cnt


def sort_pairs(pairs: np.ndarray) -> np.ndarray:
    """Sort (r_id, s_id) rows ascending, lexicographically, as uint32."""
    pairs = np.asarray(pairs, dtype=np.uint32).reshape(-1, 2)
    if pairs.shape[0] == 0:
        return pairs
    key = (pairs[:, 0].astype(np.uint64) << np.uint64(32)) | pairs[:, 1].astype(np.uint64)
    order = np.argsort(key, kind="stable")
    return pairs[order]


def join_nested(R, S) -> np.ndarray:
    return _run_join(_load().or_join_nested, R, S)


def join_simple(R, S) -> np.ndarray:
    return _run_join(_load().or_join_simple, R, S)


def join_grace(R, S, log2_parts: int = 8, nthreads: int = 4) -> np.ndarray:
    return _run_join(_load().or_join_grace, R, S, extra=(log2_parts, nthreads))


NO_ROW = 0xFFFFFFFF
MODES = {"inner": 0, "semi": 1, "anti": 2, "outer_s": 3}


def join_mode(R, S, mode: str) -> np.ndarray:
    """The join's output in one of the modes of the left/right/semi-join
    extensions (Section 5), by their plain definitions on the exact inner join
    T (R the build side, S the probe side):
      semi    = {(NO_ROW, s.id) : s has a partner in T}, anti = the S rows without one,
      outer_s = T plus the S anti rows (outer join preserving S);
      semi_r  = {(r.id, NO_ROW) : r has a partner in T}, anti_r = the R rows without one,
      outer_r = T plus the R anti rows (outer join preserving R).
    Sorted like sort_pairs."""
    T = join_simple(R, S)
    s_matched = set(T[:, 1].tolist())
    r_matched = set(T[:, 0].tolist())
    sids = [int(x) for x in S.ids]
    rids = [int(x) for x in R.ids]
    semi = [(NO_ROW, s) for s in sids if s in s_matched]
    anti = [(NO_ROW, s) for s in sids if s not in s_matched]
    semi_r = [(r, NO_ROW) for r in rids if r in r_matched]
    anti_r = [(r, NO_ROW) for r in rids if r not in r_matched]

    def arr(rows):
        return np.array(rows, dtype=np.uint32).reshape(-1, 2)
    if mode == "inner":
        out = T
    elif mode == "semi":
        out = arr(semi)
    elif mode == "anti":
        out = arr(anti)
    elif mode == "outer_s":
        out = np.concatenate([T, arr(anti)])
    elif mode == "semi_r":
        out = arr(semi_r)
    elif mode == "anti_r":
        out = arr(anti_r)
    elif mode == "outer_r":
        out = np.concatenate([T, arr(anti_r)])
    else:
        raise ValueError(mode)
    return sort_pairs(out)


def join_sig_only(R, S, n_components: int = 4, field: int = 16) -> np.ndarray:
    """The probe of Figure 2 as the paper states it (output on a signature
    match, Section 3.2): every (r.id, s.id) whose n-component signatures and
    key lengths are equal, with no byte comparison.  Plain definition: group R
    by (signature, length) and look every S key up.  field = 8 uses the byte
    symbol signatures (all four components).  Sorted like sort_pairs."""
    if field == 8:
        sR = sig8_batch(R.arena, R.off)
        sS = sig8_batch(S.arena, S.off)
    else:
        mask = np.uint64(component_mask(n_components))
        sR = sig_batch(R.arena, R.off) & mask
        sS = sig_batch(S.arena, S.off) & mask
    lR = np.diff(np.asarray(R.off, dtype=np.uint64))
    lS = np.diff(np.asarray(S.off, dtype=np.uint64))
    groups = {}
    for i in range(len(sR)):
        groups.setdefault((int(sR[i]), int(lR[i])), []).append(int(R.ids[i]))
    out = []
    for j in range(len(sS)):
        for rid in groups.get((int(sS[j]), int(lS[j])), ()):
            out.append((rid, int(S.ids[j])))
    return sort_pairs(np.array(out, dtype=np.uint32).reshape(-1, 2))


def join_prefix(R, S, prefix_len: int) -> np.ndarray:
    """The join on the keys' first prefix_len bytes, by its plain definition:
    every (r.id, s.id) with key(r)[:L] == key(s)[:L] as byte strings (so the
    truncated lengths are equal too).  Group R by its truncated key, look every
    S key up.  Sorted like sort_pairs."""
    L = int(prefix_len)
    groups = {}
    for i in range(len(R.off) - 1):
        k = bytes(R.arena[int(R.off[i]):int(R.off[i + 1])])[:L]
        groups.setdefault(k, []).append(int(R.ids[i]))
    out = []
    for j in range(len(S.off) - 1):
        k = bytes(S.arena[int(S.off[j]):int(S.off[j + 1])])[:L]
        for rid in groups.get(k, ()):
            out.append((rid, int(S.ids[j])))
    return sort_pairs(np.array(out, dtype=np.uint32).reshape(-1, 2))


def sig_prefixes(key: bytes, block_bytes: int) -> list:
    """Cumulative signatures by their definition: sig of the prefixes of
    block_bytes, 2 block_bytes, ... bytes (the last one the whole key; [0] for
    the empty key)."""
    key = bytes(key)
    if not key:
        return [0]
    nb = (len(key) + block_bytes - 1) // block_bytes
    return [sig(key[:min((j + 1) * block_bytes, len(key))]) for j in range(nb)]
