"""The synthetic generator: determinism and the stated shapes."""
import numpy as np

import workloads


def test_deterministic_and_seeded():
    spec = workloads.CONFIGS["plain"].scaled(300, 3000)
    a, b = workloads.generate(spec, nthreads=1), workloads.generate(spec, nthreads=5)
    assert np.array_equal(a.R.arena, b.R.arena) and np.array_equal(a.S.arena, b.S.arena)
    assert np.array_equal(a.S.off, b.S.off)
    c = workloads.generate(spec.__class__(**{**spec.__dict__, "seed": spec.seed + 1}))
    assert not np.array_equal(a.R.arena[:100], c.R.arena[:100])


def test_plain_shape():
    wl = workloads.generate(workloads.CONFIGS["plain"])
    for rel in (wl.R, wl.S):
        L = rel.lengths()
        assert L.min() >= 64 and L.max() <= 256
        body = rel.arena[: rel.nbytes]
        assert body.min() >= 0x20 and body.max() <= 0x7E
        assert rel.arena.shape[0] % 16 == 0 and rel.arena.shape[0] >= rel.nbytes + 16
    assert int((wl.s_kind == 1).sum()) == 30_000
    assert len({wl.R.key(i) for i in range(wl.R.n)}) == wl.R.n


def test_collision_near_duplicates():
    spec = workloads.CONFIGS["collision"].scaled(200, 2000)
    wl = workloads.generate(spec)
    assert int((wl.s_kind == 1).sum()) == 800 and int((wl.s_kind == 2).sum()) == 800
    assert set(np.unique(wl.S.arena[: wl.S.nbytes]).tolist()) <= set(b"ACGT")
    for j in np.nonzero(wl.s_kind == 2)[0][:100]:
        a = np.frombuffer(wl.S.key(j), dtype=np.uint8)
        b = np.frombuffer(wl.R.key(wl.s_src[j]), dtype=np.uint8)
        assert 1 <= int((a != b).sum()) <= 6


def test_large_duplicates_and_skew():
    spec = workloads.CONFIGS["large"].scaled(5000, 50_000)
    wl = workloads.generate(spec)
    assert int((wl.s_kind == 1).sum()) == 25_000
    L = wl.S.lengths()
    assert L.min() >= 256 and L.max() <= 1024
    counts = np.bincount(wl.s_src[wl.s_kind == 1], minlength=5000)
    assert counts.max() > 50 * counts.mean()          # Zipf head
    dup_rows = int((wl.r_mult > 1).sum())
    assert 0 < dup_rows < 0.2 * 5000


def test_perm_is_bijection():
    for n in (1, 2, 3, 17, 1000, 4097):
        vals = sorted(workloads.perm(99, 3, n, x) for x in range(n))
        assert vals == list(range(n))
