"""The batch and serving workloads generated on the device (gen_dev.cu): the
same bytes as workloads.generate_batch, written straight into device memory,
so that a batch of hundreds of GB is generated wave by wave without a host
copy.  Covers the joins the device generator supports: distinct R keys,
uniform partners and no near-duplicates.

    plan = plan_batch(specs)              # every row's key identity and offset
    for j0, j1 in waves(plan, cap):       # runs of joins of at most cap key bytes
        w = fill_wave(plan, j0, j1)       # R and S of joins [j0, j1) on the device
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

from . import JoinSpec, ALPHABETS, n_copy

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libgendev.so")
_SRCS = ("gen_dev.cu", "genrng.h")
_lock = threading.Lock()
_lib = None


class GdJoin(ctypes.Structure):
    """gd_join of gen_dev.cu."""
    _fields_ = [("seed", ctypes.c_uint64), ("m", ctypes.c_uint64), ("n", ctypes.c_uint64),
                ("n_copy", ctypes.c_uint64), ("r_row0", ctypes.c_uint64), ("s_row0", ctypes.c_uint64),
                ("r_len_lo", ctypes.c_uint32), ("r_len_hi", ctypes.c_uint32),
                ("s_len_lo", ctypes.c_uint32), ("s_len_hi", ctypes.c_uint32),
                ("alphabet", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def build() -> str:
    """Compile libgendev.so for sm_103a (nvcc)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    subprocess.check_call([nvcc if os.path.exists(nvcc) else "nvcc", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-o", tmp,
                           os.path.join(_HERE, "gen_dev.cu")])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        srcs = [os.path.join(_HERE, f) for f in _SRCS]
        if not os.path.exists(_SO) or os.path.getmtime(_SO) < max(os.path.getmtime(f) for f in srcs):
            build()
        lib = ctypes.CDLL(_SO)
        P, U64, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        J = ctypes.POINTER(GdJoin)
        lib.gd_max_joins.restype = I
        lib.gd_plan.argtypes = [J, I, U64, U64, P, P, P, P, P]
        lib.gd_plan.restype = I
        lib.gd_fill.argtypes = [J, I, I, U64, P, P, P, U64, U64, P]
        lib.gd_fill.restype = I
        _lib = lib
        return lib


def supported(spec: JoinSpec) -> bool:
    """Whether the device generator makes this join (the host generator makes every join)."""
    return spec.dup_frac == 0 and spec.zipf_s == 0 and spec.frac_near == 0


def _table(specs, r0: int = 0, s0: int = 0):
    arr = (GdJoin * len(specs))()
    r, s = r0, s0
    for i, sp in enumerate(specs):
        arr[i] = GdJoin(sp.seed, sp.m, sp.n, n_copy(sp.frac_copy, sp.n), r, s, sp.r_len[0], sp.r_len[1],
                        sp.s_len[0], sp.s_len[1], ALPHABETS[sp.alphabet], 0)
        r += sp.m
        s += sp.n
    return arr


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"device generator: {what} failed (CUDA error {rc})")


@dataclasses.dataclass
class Plan:
    """Every row's key offset (prefix sums over all joins, int64 [rows + 1]) and
    identity, per side, on the device."""
    specs: list
    offR: object
    identR: object
    offS: object
    identS: object
    r_row0: list          # first R row of join j (len = joins + 1)
    s_row0: list

    def key_bytes(self, j0: int, j1: int) -> int:
        """R and S key bytes of joins [j0, j1)."""
        r = int(self.offR[self.r_row0[j1]]) - int(self.offR[self.r_row0[j0]])
        s = int(self.offS[self.s_row0[j1]]) - int(self.offS[self.s_row0[j0]])
        return r + s


def plan_batch(specs, device="cuda", stream=None) -> Plan:
    """Row plan of the joins `specs` (in order, packed back to back)."""
    import torch
    specs = list(specs)
    lib = _load()
    if not specs or len(specs) > lib.gd_max_joins():
        raise ValueError(f"1 to {lib.gd_max_joins()} joins per plan")
    if not all(supported(sp) for sp in specs) or len({sp.alphabet for sp in specs}) != 1:
        raise ValueError("the device generator makes joins with distinct R keys, uniform partners, no "
                         "near-duplicates and one alphabet")
    mR, nS = sum(sp.m for sp in specs), sum(sp.n for sp in specs)
    offR = torch.empty(mR + 1, dtype=torch.int64, device=device)
    offS = torch.empty(nS + 1, dtype=torch.int64, device=device)
    identR = torch.empty(max(mR, 1), dtype=torch.int64, device=device)
    identS = torch.empty(max(nS, 1), dtype=torch.int64, device=device)
    st = stream if stream is not None else torch.cuda.current_stream(device)
    _check(lib.gd_plan(_table(specs), len(specs), mR, nS, offR.data_ptr(), identR.data_ptr(), offS.data_ptr(),
                       identS.data_ptr(), ctypes.c_void_p(st.cuda_stream)), "plan")
    with torch.cuda.stream(st):
        torch.cumsum(offR, 0, out=offR)
        torch.cumsum(offS, 0, out=offS)
    st.synchronize()
    r_row0, s_row0 = [0], [0]
    for sp in specs:
        r_row0.append(r_row0[-1] + sp.m)
        s_row0.append(s_row0[-1] + sp.n)
    return Plan(specs, offR, identR, offS, identS, r_row0, s_row0)


def waves(plan: Plan, cap_bytes: int) -> list:
    """Consecutive runs [j0, j1) of joins whose R and S key bytes stay within
    cap_bytes (a join larger than the cap is a wave of its own)."""
    import torch
    jr = torch.tensor(plan.r_row0, dtype=torch.int64, device=plan.offR.device)
    js = torch.tensor(plan.s_row0, dtype=torch.int64, device=plan.offS.device)
    per = (plan.offR[jr].diff() + plan.offS[js].diff()).cpu().tolist()
    out, j0, acc = [], 0, 0
    for j, b in enumerate(per):
        if j > j0 and acc + b > cap_bytes:
            out.append((j0, j))
            j0, acc = j, 0
        acc += b
    out.append((j0, len(per)))
    return out


@dataclasses.dataclass
class Wave:
    """Joins [j0, j1) of a plan on the device: packed arenas (padded like the
    host generator's), offsets from 0, row ranges and expected pair counts."""
    j0: int
    j1: int
    arenaR: object
    offR: object
    arenaS: object
    offS: object
    ranges: list          # (r_begin, r_end, s_begin, s_end) per join, rows of the wave
    expected: list        # pairs per join: every S copy joins its one R row
    key_bytes: int

    @property
    def mR(self) -> int:
        return int(self.offR.numel() - 1)

    @property
    def nS(self) -> int:
        return int(self.offS.numel() - 1)


def fill_wave(plan: Plan, j0: int, j1: int, stream=None) -> Wave:
    """Generate the key bytes of joins [j0, j1) of the plan."""
    import torch
    lib = _load()
    specs = plan.specs[j0:j1]
    dev = plan.offR.device
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    table = _table(specs)
    sides = []
    for side, (off_all, ident_all, row0) in enumerate(((plan.offR, plan.identR, plan.r_row0),
                                                        (plan.offS, plan.identS, plan.s_row0))):
        a, b = row0[j0], row0[j1]
        with torch.cuda.stream(st):
            off = off_all[a: b + 1] - off_all[a]
        nbytes = int(off[-1])
        size = (nbytes + 15) // 16 * 16 + 16                 # the host generator's padding
        arena = torch.empty(size, dtype=torch.uint8, device=dev)
        ident = ident_all[a: b] if b > a else ident_all[:1]
        _check(lib.gd_fill(table, len(specs), side, b - a, off.data_ptr(), ident.data_ptr(), arena.data_ptr(),
                           size, nbytes, ctypes.c_void_p(st.cuda_stream)), "fill")
        sides.append((arena, off, nbytes))
    st.synchronize()
    ranges, r, s = [], 0, 0
    for sp in specs:
        ranges.append((r, r + sp.m, s, s + sp.n))
        r += sp.m
        s += sp.n
    expected = [n_copy(sp.frac_copy, sp.n) if sp.m > 0 else 0 for sp in specs]
    (aR, oR, bR), (aS, oS, bS) = sides
    return Wave(j0, j1, aR, oR, aS, oS, ranges, expected, bR + bS)
