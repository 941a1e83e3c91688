"""Join of host relations with overlapped copies (stream.HostStreamJoin): the
pairs equal the oracle's, with S cut into many chunks, including chunks cut by
the byte budget and keys that start at odd offsets."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def host(rel):
    return (torch.from_numpy(rel.arena).pin_memory(), torch.from_numpy(rel.off.view(np.int64)).pin_memory(),
            torch.from_numpy(rel.ids.view(np.int32)).pin_memory())


@pytest.mark.parametrize("rows,chunk_bytes", [(997, 1 << 20), (5000, 64 << 10)])
def test_host_stream_join_matches_oracle(cuda, rows, chunk_bytes):
    from paper_2411_18183_gb300.stream import HostStreamJoin
    wl = workloads.generate(workloads.CONFIGS["large"].scaled(4000, 30_000))
    hR, hS = host(wl.R), host(wl.S)
    want = oracle.join_simple(wl.R, wl.S)
    sj = HostStreamJoin(max_m=wl.R.n, max_r_bytes=wl.R.arena.shape[0], max_chunk_rows=rows,
                        max_chunk_bytes=chunk_bytes, cap_pairs=512 * (len(want) + 1024), max_chunks=512)
    cuts = sj.chunks(wl.S.off)
    assert len(cuts) > 4
    out = torch.zeros(2 * sj.cap, dtype=torch.int32).pin_memory()
    for _ in range(2):                                  # buffers are reused across runs
        out.zero_()
        cnt = sj.run(hR, hS, cuts, out)
        got = oracle.sort_pairs(out[: 2 * cnt].numpy().view(np.uint32))
        assert np.array_equal(got, want)
