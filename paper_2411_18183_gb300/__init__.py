"""Python binding of libalgsig.so, the GB300 algebraic-signature equi-join.

Argument marshalling only: every step of the join runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the compiled library is missing, every call raises.

    import paper_2411_18183_gb300 as ag
    R = ag.DeviceRelation.from_host(arena, off, ids)      # or .from_tensors(...)
    sig = ag.sig_compute(R)                                # uint64 signatures (torch.int64 bits)
    pairs = ag.join(R, S)                                  # (cnt, 2) uint32 pairs as torch.int32 bits
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import torch

from . import build as _build_mod

LIB_PATH = _build_mod.LIB

AS_OK = 0
AS_ERR_INVALID = 1
AS_ERR_NOMEM = 2
AS_ERR_CAPACITY = 3
AS_ERR_TABLE_FULL = 4
AS_ERR_CUDA = 5
AS_ERR_UNSUPPORTED = 6

EXPORTS = ("as_last_error", "as_status_string", "as_version", "as_sig_compute", "as_sig_compute_n",
           "as_sig_shapes", "as_sig_compute_shape", "as_sig_compute_gf8",
           "as_sig_prefix_ws_bytes", "as_sig_prefix_offsets", "as_sig_prefixes", "as_join_table_bytes",
           "as_join_build", "as_join_probe_ws_bytes", "as_join_probe", "as_join_probe_sigs", "as_join_probe_mode", "as_join_ws_bytes", "as_join",
           "as_join_part_ws_bytes", "as_join_partitioned", "as_join_prefix_ws_bytes", "as_join_prefix", "as_baseline_ws_bytes", "as_baseline_join")


class AlgsigError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class Table(ctypes.Structure):
    """as_table of algsig.h: description of a built signature hash table."""
    _fields_ = [("slots", ctypes.c_void_p), ("sigR", ctypes.c_void_p), ("arenaR", ctypes.c_void_p),
                ("offR", ctypes.c_void_p), ("idR", ctypes.c_void_p), ("flags", ctypes.c_void_p),
                ("m", ctypes.c_uint64), ("cap", ctypes.c_uint64), ("log2cap", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("matched", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libalgsig.so (built by __graft_entry__.build() or paper_2411_18183_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libalgsig.so not built ({p}); run python -m paper_2411_18183_gb300.build")
        lib = ctypes.CDLL(p)
        P, U64, SZ, F, S = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_float, ctypes.c_int
        lib.as_last_error.restype = ctypes.c_char_p
        lib.as_status_string.restype = ctypes.c_char_p
        lib.as_status_string.argtypes = [S]
        lib.as_version.restype = S
        lib.as_sig_compute.argtypes = [P, P, U64, P, P]
        lib.as_sig_compute.restype = S
        lib.as_sig_compute_n.argtypes = [P, P, U64, S, P, P]
        lib.as_sig_compute_n.restype = S
        lib.as_sig_shapes.argtypes = [P, P, S]
        lib.as_sig_shapes.restype = S
        lib.as_sig_compute_shape.argtypes = [P, P, U64, S, S, P, P]
        lib.as_sig_compute_shape.restype = S
        lib.as_sig_compute_gf8.argtypes = [P, P, U64, P, P]
        lib.as_sig_compute_gf8.restype = S
        lib.as_sig_prefix_ws_bytes.argtypes = [U64]
        lib.as_sig_prefix_ws_bytes.restype = SZ
        lib.as_sig_prefix_offsets.argtypes = [P, U64, ctypes.c_uint32, P, P, SZ, P]
        lib.as_sig_prefix_offsets.restype = S
        lib.as_sig_prefixes.argtypes = [P, P, U64, ctypes.c_uint32, P, P, P]
        lib.as_sig_prefixes.restype = S
        lib.as_join_table_bytes.argtypes = [U64, F]
        lib.as_join_table_bytes.restype = SZ
        lib.as_join_ws_bytes.argtypes = [U64, U64, F]
        lib.as_join_ws_bytes.restype = SZ
        lib.as_join_probe_ws_bytes.argtypes = [U64]
        lib.as_join_probe_ws_bytes.restype = SZ
        lib.as_join_build.argtypes = [P, SZ, P, P, P, U64, P, F, ctypes.POINTER(Table), P]
        lib.as_join_build.restype = S
        lib.as_join_probe.argtypes = [ctypes.POINTER(Table), P, P, P, U64, P, P, SZ, P, U64, P, P, P]
        lib.as_join_probe.restype = S
        lib.as_join_probe_sigs.argtypes = [ctypes.POINTER(Table), P, P, P, U64, P, P, U64, P, P, P]
        lib.as_join_probe_sigs.restype = S
        lib.as_join_probe_mode.argtypes = [ctypes.POINTER(Table), P, P, P, U64, P, S, P, U64, P, P, P]
        lib.as_join_probe_mode.restype = S
        lib.as_join.argtypes = [P, P, P, U64, P, P, P, U64, F, P, SZ, P, U64, P, P, P]
        lib.as_join.restype = S
        lib.as_join_prefix_ws_bytes.argtypes = [U64, U64, F]
        lib.as_join_prefix_ws_bytes.restype = SZ
        lib.as_join_prefix.argtypes = [P, P, P, U64, P, P, P, U64, U64, F, P, SZ, P, U64, P, P, P]
        lib.as_join_prefix.restype = S
        lib.as_join_part_ws_bytes.argtypes = [U64, U64, F, ctypes.c_uint32]
        lib.as_join_part_ws_bytes.restype = SZ
        lib.as_join_partitioned.argtypes = [P, P, P, U64, P, P, P, U64, F, ctypes.c_uint32, P, SZ, P, U64, P, P, P]
        lib.as_join_partitioned.restype = S
        lib.as_baseline_ws_bytes.argtypes = [U64, U64, F]
        lib.as_baseline_ws_bytes.restype = SZ
        lib.as_baseline_join.argtypes = [P, P, P, U64, P, P, P, U64, F, S, P, SZ, P, U64, P, P, P]
        lib.as_baseline_join.restype = S
        if path is None:
            _lib = lib
        return lib


def _check(st: int, allow=()):
    if st != AS_OK and st not in allow:
        lib = load()
        raise AlgsigError(st, f"{lib.as_status_string(st).decode()}: {lib.as_last_error().decode()}")
    return st


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return t.data_ptr()


def _stream(stream) -> int | None:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


@dataclasses.dataclass
class DeviceRelation:
    """A relation resident in device memory: key i = arena[off[i]:off[i+1]].

    arena: uint8 (16-byte aligned, readable to the next 16-byte boundary past
    the last key byte); off: int64 tensor holding the uint64 offsets (n+1);
    ids: int32 tensor holding uint32 ids, or None for ids = row numbers."""
    arena: torch.Tensor
    off: torch.Tensor
    ids: torch.Tensor | None = None

    @property
    def n(self) -> int:
        return int(self.off.numel() - 1)

    @staticmethod
    def from_host(arena, off, ids=None, device="cuda", non_blocking=False) -> "DeviceRelation":
        """Copy numpy / torch host arrays to the device (allocating with torch)."""
        a = torch.as_tensor(arena).view(torch.uint8)
        o = torch.as_tensor(off).view(torch.int64)
        i = None if ids is None else torch.as_tensor(ids).view(torch.int32)
        pad = (-a.numel()) % 16
        if pad:
            a = torch.cat([a, torch.zeros(pad, dtype=torch.uint8)])
        return DeviceRelation(a.to(device, non_blocking=non_blocking), o.to(device, non_blocking=non_blocking),
                              None if i is None else i.to(device, non_blocking=non_blocking))


def version() -> int:
    return int(load().as_version())


def sig_shapes() -> list:
    """as_sig_shapes: the (warps per block, blocks in flight per key) launch shapes
    of the signature kernel; index 0 is the default."""
    lib = load()
    cnt = int(lib.as_sig_shapes(None, None, 0))
    w, d = (ctypes.c_int * cnt)(), (ctypes.c_int * cnt)()
    lib.as_sig_shapes(w, d, cnt)
    return [(int(w[i]), int(d[i])) for i in range(cnt)]


def sig_compute(rel: DeviceRelation, out: torch.Tensor | None = None, stream=None,
                n_components: int = 4, shape: int | None = None) -> torch.Tensor:
    """as_sig_compute (n_components = 4) or as_sig_compute_n (2: the paper's two-symbol
    signature, components 3 and 4 zero): uint64 signature of every key (as int64 bits).
    With `shape`, as_sig_compute_shape with that launch shape (see sig_shapes)."""
    lib = load()
    n = rel.n
    if out is None:
        out = torch.empty(max(n, 0), dtype=torch.int64, device=rel.arena.device)
    if shape is not None:
        _check(lib.as_sig_compute_shape(_ptr(rel.arena), _ptr(rel.off), n, n_components, shape, _ptr(out),
                                        _stream(stream)))
    elif n_components == 4:
        _check(lib.as_sig_compute(_ptr(rel.arena), _ptr(rel.off), n, _ptr(out), _stream(stream)))
    else:
        _check(lib.as_sig_compute_n(_ptr(rel.arena), _ptr(rel.off), n, n_components, _ptr(out), _stream(stream)))
    return out


def sig_compute_gf8(rel: DeviceRelation, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """as_sig_compute_gf8: byte-symbol signature over GF(2^8) of every key (int64 bits,
    component k in bits [8(k-1), 8k))."""
    lib = load()
    n = rel.n
    if out is None:
        out = torch.empty(max(n, 0), dtype=torch.int64, device=rel.arena.device)
    _check(lib.as_sig_compute_gf8(_ptr(rel.arena), _ptr(rel.off), n, _ptr(out), _stream(stream)))
    return out


def sig_prefixes(rel: DeviceRelation, block_bytes: int, stream=None):
    """as_sig_prefix_offsets + as_sig_prefixes: (pref_off int64[n+1], entries int64[total]);
    key i's cumulative signatures are entries[pref_off[i]:pref_off[i+1]] (prefixes of
    block_bytes, 2 * block_bytes, ... bytes, the last one the whole key).  Reads the
    total count back (synchronises the stream)."""
    lib = load()
    n = rel.n
    dev = rel.arena.device
    pref = torch.empty(n + 1, dtype=torch.int64, device=dev)
    ws = alloc_ws(int(lib.as_sig_prefix_ws_bytes(n)), dev)
    _check(lib.as_sig_prefix_offsets(_ptr(rel.off), n, block_bytes, _ptr(pref), _ptr(ws), ws.numel(),
                                     _stream(stream)))
    total = int(pref[n].item())
    out = torch.empty(max(total, 1), dtype=torch.int64, device=dev)
    _check(lib.as_sig_prefixes(_ptr(rel.arena), _ptr(rel.off), n, block_bytes, _ptr(pref), _ptr(out),
                               _stream(stream)))
    return pref, out[:total]


def join_table_bytes(m: int, load_factor: float = 0.5) -> int:
    return int(load().as_join_table_bytes(m, load_factor))


def join_ws_bytes(m: int, n: int, load_factor: float = 0.5) -> int:
    return int(load().as_join_ws_bytes(m, n, load_factor))


def join_probe_ws_bytes(n: int) -> int:
    return int(load().as_join_probe_ws_bytes(n))


def alloc_ws(nbytes: int, device="cuda") -> torch.Tensor:
    """Workspace buffer (256-byte aligned: torch's allocator aligns to 512)."""
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def join_build(R: DeviceRelation, ws: torch.Tensor, load_factor: float = 0.5, sigR: torch.Tensor | None = None,
               stream=None) -> Table:
    lib = load()
    t = Table()
    _check(lib.as_join_build(_ptr(ws), ws.numel(), _ptr(R.arena), _ptr(R.off), _ptr(R.ids), R.n, _ptr(sigR),
                             load_factor, ctypes.byref(t), _stream(stream)))
    return t


def join_probe(t: Table, S: DeviceRelation, pairs: torch.Tensor, count: torch.Tensor,
               sigS_out: torch.Tensor | None = None, ws: torch.Tensor | None = None, sync: bool = True,
               stream=None) -> int | None:
    """as_join_probe.  pairs: int32 tensor of 2*cap entries; count: int64 device scalar;
    ws: workspace of join_probe_ws_bytes(S.n) bytes when sigS_out is None.
    With sync=True returns the pair count (raises AlgsigError on capacity overflow)."""
    lib = load()
    cap = pairs.numel() // 2
    h = ctypes.c_uint64(0)
    _check(lib.as_join_probe(ctypes.byref(t), _ptr(S.arena), _ptr(S.off), _ptr(S.ids), S.n, _ptr(sigS_out),
                             _ptr(ws), 0 if ws is None else ws.numel(), _ptr(pairs), cap, _ptr(count),
                             ctypes.byref(h) if sync else None, _stream(stream)))
    return int(h.value) if sync else None


def join_probe_sigs(t: Table, S: DeviceRelation, sigS: torch.Tensor, pairs: torch.Tensor, count: torch.Tensor,
                    sync: bool = True, stream=None) -> int | None:
    """as_join_probe_sigs: the probe with S's signatures (int64[S.n], from sig_compute) given."""
    lib = load()
    cap = pairs.numel() // 2
    h = ctypes.c_uint64(0)
    _check(lib.as_join_probe_sigs(ctypes.byref(t), _ptr(S.arena), _ptr(S.off), _ptr(S.ids), S.n, _ptr(sigS),
                                  _ptr(pairs), cap, _ptr(count), ctypes.byref(h) if sync else None, _stream(stream)))
    return int(h.value) if sync else None


JOIN_MODES = {"inner": 0, "semi": 1, "anti": 2, "outer_s": 3, "sig_only": 4,
              "outer_r": 5, "semi_r": 6, "anti_r": 7}                # AS_JOIN_*
NO_ROW = 0xFFFFFFFF                                                  # AS_NO_ROW
ROWS_SCATTERED = 0xFFFFFFFFFFFFFFFF                                  # AS_ROWS_SCATTERED


def join_probe_mode(t: Table, S: DeviceRelation, sigS: torch.Tensor, pairs: torch.Tensor, count: torch.Tensor,
                    mode: str = "inner", sync: bool = True, stream=None) -> int | None:
    """as_join_probe_mode: inner pairs, or per-S-row (NO_ROW, s_id) records (semi, anti), or
    inner pairs plus the unmatched S rows (outer_s), or the R-side counterparts with per-R-row
    (r_id, NO_ROW) records (semi_r, anti_r, outer_r), or the signature-only pairs of the
    paper's probe without byte verification (sig_only; not exact)."""
    lib = load()
    cap = pairs.numel() // 2
    h = ctypes.c_uint64(0)
    _check(lib.as_join_probe_mode(ctypes.byref(t), _ptr(S.arena), _ptr(S.off), _ptr(S.ids), S.n, _ptr(sigS),
                                  JOIN_MODES[mode], _ptr(pairs), cap, _ptr(count), ctypes.byref(h) if sync else None,
                                  _stream(stream)))
    return int(h.value) if sync else None


PROBE_NOALLOC_MAX_KEYS = 1 << 20       # AS_PROBE_NOALLOC_MAX_KEYS


def join_probe_noalloc(t: Table, S: DeviceRelation, pairs: torch.Tensor, count: torch.Tensor, sync: bool = True,
                       stream=None) -> int | None:
    """as_join_probe_noalloc: as join_probe, with S's signatures in the library's fixed
    scratch (S.n <= PROBE_NOALLOC_MAX_KEYS); calls on one device must not overlap."""
    lib = load()
    f = lib.as_join_probe_noalloc
    if not getattr(lib, "_noalloc_ready", False):
        P, U64 = ctypes.c_void_p, ctypes.c_uint64
        f.argtypes = [ctypes.POINTER(Table), P, P, P, U64, P, U64, P, P, P]
        f.restype = ctypes.c_int
        lib._noalloc_ready = True
    cap = pairs.numel() // 2
    h = ctypes.c_uint64(0)
    _check(f(ctypes.byref(t), _ptr(S.arena), _ptr(S.off), _ptr(S.ids), S.n, _ptr(pairs),
                                     cap, _ptr(count), ctypes.byref(h) if sync else None, _stream(stream)))
    return int(h.value) if sync else None


def join_into(R: DeviceRelation, S: DeviceRelation, ws: torch.Tensor, pairs: torch.Tensor, count: torch.Tensor,
              load_factor: float = 0.5, sync: bool = True, stream=None, allow_capacity: bool = False):
    """as_join into caller buffers.  Returns (status, count) when sync, else (status, None)."""
    lib = load()
    cap = pairs.numel() // 2
    h = ctypes.c_uint64(0)
    st = lib.as_join(_ptr(R.arena), _ptr(R.off), _ptr(R.ids), R.n, _ptr(S.arena), _ptr(S.off), _ptr(S.ids), S.n,
                     load_factor, _ptr(ws), ws.numel(), _ptr(pairs), cap, _ptr(count),
                     ctypes.byref(h) if sync else None, _stream(stream))
    _check(st, allow=(AS_ERR_CAPACITY,) if allow_capacity else ())
    return st, (int(h.value) if sync else None)


def join(R: DeviceRelation, S: DeviceRelation, load_factor: float = 0.5, cap_pairs: int | None = None,
         stream=None) -> torch.Tensor:
    """The whole signature join.  Returns a (cnt, 2) int32 tensor of (r_id, s_id)
    pairs (uint32 bits) in unspecified order, retrying once with the exact
    size if the first guess of the capacity was too small."""
    dev = R.arena.device
    ws = alloc_ws(join_ws_bytes(R.n, S.n, load_factor), dev)
    cap = cap_pairs if cap_pairs is not None else max(1024, S.n)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    while True:
        pairs = torch.empty(2 * max(cap, 1), dtype=torch.int32, device=dev)
        st, cnt = join_into(R, S, ws, pairs, count, load_factor, sync=True, stream=stream, allow_capacity=True)
        if st == AS_OK:
            return pairs[:2 * cnt].view(-1, 2)
        cap = cnt


def join_prefix_ws_bytes(m: int, n: int, load_factor: float = 0.5) -> int:
    return int(load().as_join_prefix_ws_bytes(m, n, load_factor))


def join_prefix_into(R: DeviceRelation, S: DeviceRelation, prefix_len: int, ws: torch.Tensor, pairs: torch.Tensor,
                     count: torch.Tensor, load_factor: float = 0.5, sync: bool = True, stream=None,
                     allow_capacity: bool = False):
    """as_join_prefix (the join on the keys' first prefix_len bytes) into caller buffers."""
    lib = load()
    cap = pairs.numel() // 2
    h = ctypes.c_uint64(0)
    st = lib.as_join_prefix(_ptr(R.arena), _ptr(R.off), _ptr(R.ids), R.n, _ptr(S.arena), _ptr(S.off), _ptr(S.ids),
                            S.n, prefix_len, load_factor, _ptr(ws), ws.numel(), _ptr(pairs), cap, _ptr(count),
                            ctypes.byref(h) if sync else None, _stream(stream))
    _check(st, allow=(AS_ERR_CAPACITY,) if allow_capacity else ())
    return st, (int(h.value) if sync else None)


def join_prefix(R: DeviceRelation, S: DeviceRelation, prefix_len: int, load_factor: float = 0.5,
                cap_pairs: int | None = None, stream=None) -> torch.Tensor:
    """The join on the keys' first prefix_len bytes; (cnt, 2) int32 tensor of (r_id, s_id) pairs."""
    dev = R.arena.device
    ws = alloc_ws(join_prefix_ws_bytes(R.n, S.n, load_factor), dev)
    cap = cap_pairs if cap_pairs is not None else max(1024, S.n)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    while True:
        pairs = torch.empty(2 * max(cap, 1), dtype=torch.int32, device=dev)
        st, cnt = join_prefix_into(R, S, prefix_len, ws, pairs, count, load_factor, sync=True, stream=stream,
                                   allow_capacity=True)
        if st == AS_OK:
            return pairs[:2 * cnt].view(-1, 2)
        cap = cnt


PART_BITS_AUTO = 0xFFFFFFFF                                           # AS_PART_BITS_AUTO


def join_part_ws_bytes(m: int, n: int, load_factor: float = 0.5, part_bits: int = PART_BITS_AUTO) -> int:
    return int(load().as_join_part_ws_bytes(m, n, load_factor, part_bits))


def join_partitioned_into(R: DeviceRelation, S: DeviceRelation, ws: torch.Tensor, pairs: torch.Tensor,
                          count: torch.Tensor, load_factor: float = 0.5, part_bits: int = PART_BITS_AUTO,
                          sync: bool = True, stream=None, allow_capacity: bool = False):
    """as_join_partitioned (the radix-partitioned signature join) into caller buffers."""
    lib = load()
    cap = pairs.numel() // 2
    h = ctypes.c_uint64(0)
    st = lib.as_join_partitioned(_ptr(R.arena), _ptr(R.off), _ptr(R.ids), R.n, _ptr(S.arena), _ptr(S.off),
                                 _ptr(S.ids), S.n, load_factor, part_bits, _ptr(ws), ws.numel(), _ptr(pairs), cap,
                                 _ptr(count), ctypes.byref(h) if sync else None, _stream(stream))
    _check(st, allow=(AS_ERR_CAPACITY,) if allow_capacity else ())
    return st, (int(h.value) if sync else None)


def join_partitioned(R: DeviceRelation, S: DeviceRelation, load_factor: float = 0.5,
                     part_bits: int = PART_BITS_AUTO, cap_pairs: int | None = None, stream=None) -> torch.Tensor:
    """The radix-partitioned signature join; (cnt, 2) int32 tensor of (r_id, s_id) pairs."""
    dev = R.arena.device
    ws = alloc_ws(join_part_ws_bytes(R.n, S.n, load_factor, part_bits), dev)
    cap = cap_pairs if cap_pairs is not None else max(1024, S.n)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    while True:
        pairs = torch.empty(2 * max(cap, 1), dtype=torch.int32, device=dev)
        st, cnt = join_partitioned_into(R, S, ws, pairs, count, load_factor, part_bits, sync=True, stream=stream,
                                        allow_capacity=True)
        if st == AS_OK:
            return pairs[:2 * cnt].view(-1, 2)
        cap = cnt


def baseline_ws_bytes(m: int, n: int, load_factor: float = 0.5) -> int:
    return int(load().as_baseline_ws_bytes(m, n, load_factor))


def baseline_join_into(R: DeviceRelation, S: DeviceRelation, ws: torch.Tensor, pairs: torch.Tensor,
                       count: torch.Tensor, load_factor: float = 0.5, tagged: bool = False, sync: bool = True,
                       stream=None, allow_capacity: bool = False):
    """as_baseline_join (the full-string comparison join) into caller buffers."""
    lib = load()
    cap = pairs.numel() // 2
    h = ctypes.c_uint64(0)
    st = lib.as_baseline_join(_ptr(R.arena), _ptr(R.off), _ptr(R.ids), R.n, _ptr(S.arena), _ptr(S.off),
                              _ptr(S.ids), S.n, load_factor, 1 if tagged else 0, _ptr(ws), ws.numel(), _ptr(pairs),
                              cap, _ptr(count), ctypes.byref(h) if sync else None, _stream(stream))
    _check(st, allow=(AS_ERR_CAPACITY,) if allow_capacity else ())
    return st, (int(h.value) if sync else None)


def baseline_join(R: DeviceRelation, S: DeviceRelation, load_factor: float = 0.5, tagged: bool = False,
                  cap_pairs: int | None = None, stream=None) -> torch.Tensor:
    """The full-string comparison join; (cnt, 2) int32 tensor of (r_id, s_id) pairs."""
    dev = R.arena.device
    ws = alloc_ws(baseline_ws_bytes(R.n, S.n, load_factor), dev)
    cap = cap_pairs if cap_pairs is not None else max(1024, S.n)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    while True:
        pairs = torch.empty(2 * max(cap, 1), dtype=torch.int32, device=dev)
        st, cnt = baseline_join_into(R, S, ws, pairs, count, load_factor, tagged, sync=True, stream=stream,
                                     allow_capacity=True)
        if st == AS_OK:
            return pairs[:2 * cnt].view(-1, 2)
        cap = cnt


# ----------------------------------------------------------------------------- batches of joins

class JoinDesc(ctypes.Structure):
    """as_join_desc: join j's row ranges in the batch's R and S and its output region."""
    _fields_ = [("r_begin", ctypes.c_uint64), ("r_end", ctypes.c_uint64), ("s_begin", ctypes.c_uint64),
                ("s_end", ctypes.c_uint64), ("pair_offset", ctypes.c_uint64), ("pair_cap", ctypes.c_uint64)]


class Batch(ctypes.Structure):
    """as_batch: a prepared batch (device descriptors and workspace regions)."""
    _fields_ = [("descs", ctypes.c_void_p), ("slots", ctypes.c_void_p), ("sigR", ctypes.c_void_p),
                ("sigS", ctypes.c_void_p), ("flags", ctypes.c_void_p), ("n_joins", ctypes.c_uint64),
                ("slots_total", ctypes.c_uint64), ("mR", ctypes.c_uint64), ("nS", ctypes.c_uint64),
                ("r_first", ctypes.c_uint64), ("s_first", ctypes.c_uint64), ("sig_shape", ctypes.c_int32),
                ("reserved0", ctypes.c_int32)]


def _batch_lib():
    lib = load()
    if not getattr(lib, "_batch_ready", False):
        P, U64, SZ, F, S = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_float, ctypes.c_int
        D = ctypes.POINTER(JoinDesc)
        lib.as_join_batch_ws_bytes.argtypes = [D, S, U64, U64, F]
        lib.as_join_batch_ws_bytes.restype = SZ
        lib.as_join_batch_prepare.argtypes = [D, S, U64, U64, F, P, SZ, ctypes.POINTER(Batch), P]
        lib.as_join_batch_prepare.restype = S
        lib.as_join_batch_run.argtypes = [ctypes.POINTER(Batch), P, P, P, P, P, P, P, P, P]
        lib.as_join_batch_run.restype = S
        lib._batch_ready = True
    return lib


def make_descs(ranges, pair_caps) -> ctypes.Array:
    """ranges: iterable of (r_begin, r_end, s_begin, s_end); output regions laid out back to back."""
    ranges = list(ranges)
    arr = (JoinDesc * len(ranges))()
    off = 0
    for j, ((rb, re_, sb, se), cap) in enumerate(zip(ranges, pair_caps)):
        arr[j] = JoinDesc(int(rb), int(re_), int(sb), int(se), off, int(cap))
        off += int(cap)
    return arr


def total_pair_cap(descs) -> int:
    return max((d.pair_offset + d.pair_cap for d in descs), default=0)


def join_batch_ws_bytes(descs, mR: int, nS: int, load_factor: float = 0.5) -> int:
    return int(_batch_lib().as_join_batch_ws_bytes(descs, len(descs), mR, nS, load_factor))


def join_batch_prepare(descs, R: DeviceRelation, S: DeviceRelation, ws: torch.Tensor, load_factor: float = 0.5,
                       stream=None) -> Batch:
    b = Batch()
    _check(_batch_lib().as_join_batch_prepare(descs, len(descs), R.n, S.n, load_factor, _ptr(ws), ws.numel(),
                                              ctypes.byref(b), _stream(stream)))
    return b


def join_batch_run(b: Batch, R: DeviceRelation, S: DeviceRelation, pairs: torch.Tensor, counts: torch.Tensor,
                   stream=None) -> None:
    """Asynchronous (capturable in a CUDA graph)."""
    _check(_batch_lib().as_join_batch_run(ctypes.byref(b), _ptr(R.arena), _ptr(R.off), _ptr(R.ids), _ptr(S.arena),
                                          _ptr(S.off), _ptr(S.ids), _ptr(pairs), _ptr(counts), _stream(stream)))


def join_batch(R: DeviceRelation, S: DeviceRelation, ranges, pair_caps, load_factor: float = 0.5):
    """Run a batch once; returns a list of per-join (cnt, 2) int32 pair tensors (join-local ids
    unless the relations carry ids).  Raises if a join overflows its pair_cap."""
    descs = make_descs(ranges, pair_caps)
    dev = R.arena.device
    ws = alloc_ws(join_batch_ws_bytes(descs, R.n, S.n, load_factor), dev)
    b = join_batch_prepare(descs, R, S, ws, load_factor)
    pairs = torch.empty(2 * max(1, total_pair_cap(descs)), dtype=torch.int32, device=dev)
    counts = torch.zeros(len(descs), dtype=torch.int64, device=dev)
    join_batch_run(b, R, S, pairs, counts)
    cnt = counts.cpu().tolist()
    out = []
    for d, c in zip(descs, cnt):
        if c > d.pair_cap:
            raise AlgsigError(AS_ERR_CAPACITY, f"join overflowed its pair capacity ({c} > {d.pair_cap})")
        out.append(pairs[2 * d.pair_offset: 2 * (d.pair_offset + c)].view(-1, 2))
    return out
