"""Join of host-resident relations with the host-to-device copies overlapped.

R is copied whole and its table built; S is copied in chunks of rows into two
device buffers on a copy stream while the compute stream computes the
signatures of the previous chunk and probes the table with them, so the
transfer of S (the bulk of the bytes) runs under the join's kernels.  The
pairs of each chunk go to the chunk's own region of the device pair buffer
and are copied back to pinned host memory at the end.

A chunk's keys are copied as the 16-byte aligned span of the host arena that
holds them plus 16 bytes (the padding the kernels may read), and its offsets
stay absolute: the library is given the device buffer's address minus the
span's start as the arena base, so no offset is rewritten on the host.
"""
from __future__ import annotations

import numpy as np
import torch

from . import DeviceRelation, alloc_ws, join_build, join_probe_sigs, join_table_bytes, sig_compute


class _Shifted:
    """Stands for a device arena whose base lies `shift` bytes before a buffer
    (the buffer holds the arena bytes from `shift` on; offsets stay absolute)."""

    is_cuda = True

    def __init__(self, buf: torch.Tensor, shift: int):
        self._p = buf.data_ptr() - shift

    def is_contiguous(self) -> bool:
        return True

    def data_ptr(self) -> int:
        return self._p


class HostStreamJoin:
    """Reusable buffers and streams for joins of host relations given as pinned
    torch tensors (arena uint8, off int64, ids int32)."""

    def __init__(self, max_m: int, max_r_bytes: int, max_chunk_rows: int, max_chunk_bytes: int, cap_pairs: int,
                 max_chunks: int = 64, load_factor: float = 0.5):
        dev = "cuda"
        self.lf = load_factor
        self.rows = max_chunk_rows
        self.chunk_bytes = max_chunk_bytes
        self.R_arena = torch.empty(max_r_bytes + 64, dtype=torch.uint8, device=dev)
        self.R_off = torch.empty(max_m + 1, dtype=torch.int64, device=dev)
        self.R_ids = torch.empty(max(1, max_m), dtype=torch.int32, device=dev)
        self.ws = alloc_ws(join_table_bytes(max_m, load_factor))
        self.S_arena = [torch.empty(max_chunk_bytes + 64, dtype=torch.uint8, device=dev) for _ in range(2)]
        self.S_off = [torch.empty(max_chunk_rows + 1, dtype=torch.int64, device=dev) for _ in range(2)]
        self.S_ids = [torch.empty(max_chunk_rows, dtype=torch.int32, device=dev) for _ in range(2)]
        self.sigS = [torch.empty(max_chunk_rows, dtype=torch.int64, device=dev) for _ in range(2)]
        self.max_chunks = max_chunks
        self.cap = cap_pairs
        self.pairs = torch.empty(2 * cap_pairs, dtype=torch.int32, device=dev)
        self.counts = torch.zeros(max_chunks, dtype=torch.int64, device=dev)
        self.counts_host = torch.zeros(max_chunks, dtype=torch.int64).pin_memory()
        self.copy = torch.cuda.Stream()
        self.comp = torch.cuda.Stream()

    def chunks(self, off: np.ndarray):
        """Row cuts of S so that every chunk fits the buffers."""
        n = off.shape[0] - 1
        cuts = [0]
        while cuts[-1] < n:
            a = cuts[-1]
            b = min(n, a + self.rows)
            # shrink until the chunk's aligned byte span fits
            while b > a + 1 and (((int(off[b]) + 15) & ~15) + 16 - (int(off[a]) & ~15)) > self.chunk_bytes:
                b = a + max(1, (b - a) // 2)
            if (((int(off[b]) + 15) & ~15) + 16 - (int(off[a]) & ~15)) > self.chunk_bytes:
                raise ValueError("a key is longer than the chunk buffer")
            cuts.append(b)
        if len(cuts) - 1 > self.max_chunks:
            raise ValueError("too many chunks for the pair regions")
        return cuts

    def run(self, hR, hS, cuts, out_host: torch.Tensor):
        """Join host R = (arena, off, ids) with host S in the chunks `cuts`;
        returns the pair count and fills out_host (pinned int32[2 * cap]).
        Raises if a chunk's pairs overflow its region of the pair buffer."""
        m = hR[1].numel() - 1
        offS = hS[1]
        nch = len(cuts) - 1
        region = self.cap // max(1, nch)
        main = torch.cuda.current_stream()
        start = torch.cuda.Event()
        start.record(main)
        self.copy.wait_event(start)
        self.comp.wait_event(start)
        with torch.cuda.stream(self.copy):
            self.R_arena[: hR[0].numel()].copy_(hR[0], non_blocking=True)
            self.R_off[: m + 1].copy_(hR[1], non_blocking=True)
            self.R_ids[:m].copy_(hR[2], non_blocking=True)
        r_ready = torch.cuda.Event()
        r_ready.record(self.copy)
        self.comp.wait_event(r_ready)
        R = DeviceRelation(self.R_arena, self.R_off[: m + 1], self.R_ids[:m])
        table = join_build(R, self.ws, self.lf, stream=self.comp)
        free = [torch.cuda.Event() for _ in range(2)]
        for ev in free:
            ev.record(self.comp)
        for c in range(nch):
            a, b = cuts[c], cuts[c + 1]
            k = c & 1
            A0 = int(offS[a]) & ~15
            A1 = min(hS[0].numel(), ((int(offS[b]) + 15) & ~15) + 16)
            self.copy.wait_event(free[k])
            with torch.cuda.stream(self.copy):
                self.S_arena[k][: A1 - A0].copy_(hS[0][A0:A1], non_blocking=True)
                self.S_off[k][: b - a + 1].copy_(offS[a: b + 1], non_blocking=True)
                self.S_ids[k][: b - a].copy_(hS[2][a:b], non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(self.copy)
            self.comp.wait_event(ready)
            S = DeviceRelation(_Shifted(self.S_arena[k], A0), self.S_off[k][: b - a + 1], self.S_ids[k][: b - a])
            sig_compute(S, self.sigS[k][: b - a], stream=self.comp)
            join_probe_sigs(table, S, self.sigS[k][: b - a], self.pairs[2 * region * c: 2 * region * (c + 1)],
                            self.counts[c: c + 1], sync=False, stream=self.comp)
            free[k] = torch.cuda.Event()
            free[k].record(self.comp)
        with torch.cuda.stream(self.comp):
            self.counts_host[:nch].copy_(self.counts[:nch], non_blocking=True)
        self.comp.synchronize()
        counts = self.counts_host[:nch].tolist()
        if counts and max(counts) > region:
            raise RuntimeError(f"a chunk found {max(counts)} pairs, more than its region of {region}")
        total = 0
        with torch.cuda.stream(self.comp):
            for c, cnt in enumerate(counts):
                if cnt:
                    out_host[2 * total: 2 * (total + cnt)].copy_(self.pairs[2 * region * c: 2 * (region * c + cnt)],
                                                                  non_blocking=True)
                total += cnt
        self.comp.synchronize()
        main.wait_stream(self.comp)
        return total
