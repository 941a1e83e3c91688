"""GPU signatures (as_sig_compute through the C ABI) against the CPU oracle,
element by element, bit-exact."""
import random

import numpy as np
import pytest

import oracle
import workloads
from cases import edge_keys
from packing import interleave_gaps, relation_garbage_tail

pytestmark = pytest.mark.gpu


def gpu_sigs(ag, rel):
    R = ag.DeviceRelation.from_host(rel.arena, rel.off, rel.ids)
    return ag.sig_compute(R).cpu().numpy().view(np.uint64)


def check(ag, rel, nthreads=8):
    got = gpu_sigs(ag, rel)
    want = oracle.sig_batch(rel.arena, rel.off, nthreads=nthreads)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"{bad.size} mismatches, first at key {bad[:5].tolist()}"


def test_edge_keys_every_alignment(cuda):
    keys = edge_keys()
    for shift in range(16):
        check(cuda, relation_garbage_tail([b"#" * shift] + interleave_gaps(keys, seed=shift), seed=shift))


def test_all_short_lengths_all_alignments(cuda):
    rng = random.Random(11)
    keys = []
    for n in range(0, 80):
        for _ in range(16):
            keys.append(bytes(rng.randrange(256) for _ in range(n)))
    rng.shuffle(keys)
    check(cuda, relation_garbage_tail(interleave_gaps(keys, seed=1), seed=2))


def test_tile_boundaries(cuda):
    # lengths around multiples of the per-lane tile and of 32 tiles per round
    rng = random.Random(12)
    keys = []
    for base in (256, 512, 768, 8192, 8192 + 256):
        for d in (-17, -2, -1, 0, 1, 2, 15, 16, 17):
            keys.append(bytes(rng.randrange(256) for _ in range(base + d)))
    rng.shuffle(keys)
    check(cuda, relation_garbage_tail(interleave_gaps(keys, seed=3), seed=4))


def test_long_keys_many_rounds_and_exponent_wrap(cuda):
    rng = np.random.default_rng(13)
    keys = [rng.integers(0, 256, n, dtype=np.uint8).tobytes() for n in (1, 70_000, 131_069, 131_070, 131_071,
                                                                          200_001, 300_000)]
    check(cuda, relation_garbage_tail(interleave_gaps(keys, seed=5), seed=6), nthreads=8)


def test_plain_config_full(cuda):
    wl = workloads.generate(workloads.CONFIGS["plain"])
    check(cuda, wl.R)
    check(cuda, wl.S)


def test_collision_config_scaled(cuda):
    wl = workloads.generate(workloads.CONFIGS["collision"].scaled(1_000, 10_000))
    check(cuda, wl.S)


def test_large_config_scaled(cuda):
    wl = workloads.generate(workloads.CONFIGS["large"].scaled(10_000, 100_000))
    check(cuda, wl.S)


def test_two_component_signatures(cuda):
    """as_sig_compute_n with n = 2 (the paper's two-symbol signature): the first
    two components of the oracle's signature, bits 32..63 zero, at every
    alignment, over tile boundaries and on a scaled large-workload relation."""
    ag = cuda
    rng = random.Random(44)
    keys = edge_keys() + [bytes(rng.randrange(256) for _ in range(n)) for n in
                          list(range(0, 70)) + [255, 256, 257, 511, 512, 513, 4095, 4097, 9000]]
    rels = [relation_garbage_tail(interleave_gaps(keys, seed=s), seed=s) for s in range(3)]
    rels.append(workloads.generate(workloads.CONFIGS["large"].scaled(1000, 5000)).S)
    mask = np.uint64(oracle.component_mask(2))
    for rel in rels:
        D = ag.DeviceRelation.from_host(rel.arena, rel.off, rel.ids)
        got = ag.sig_compute(D, n_components=2).cpu().numpy().view(np.uint64)
        want = oracle.sig_batch(rel.arena, rel.off, nthreads=8) & mask
        assert np.array_equal(got, want)
    with pytest.raises(ag.AlgsigError):
        ag.sig_compute(ag.DeviceRelation.from_host(rels[0].arena, rels[0].off, rels[0].ids), n_components=3)


def test_every_launch_shape(cuda):
    """as_sig_compute_shape: each launch shape of the signature kernel gives the
    oracle's signatures, 4 and 2 components, on edge keys at every alignment,
    on lengths over the block and window boundaries and on a scaled relation of
    the large workload (one window per warp and several); an unknown shape is
    rejected."""
    ag = cuda
    rng = random.Random(45)
    keys = edge_keys() + [bytes(rng.randrange(256) for _ in range(n)) for n in
                          list(range(0, 70)) + [255, 256, 257, 511, 512, 513, 4095, 4097, 9000]]
    rels = [relation_garbage_tail([b"#" * s] + interleave_gaps(keys, seed=s), seed=s) for s in range(0, 16, 5)]
    rels.append(workloads.generate(workloads.CONFIGS["large"].scaled(2000, 60_000)).S)
    mask = np.uint64(oracle.component_mask(2))
    shapes = ag.sig_shapes()
    assert len(shapes) >= 2 and all(w > 0 and d > 0 for w, d in shapes)
    for rel in rels:
        D = ag.DeviceRelation.from_host(rel.arena, rel.off, rel.ids)
        want = oracle.sig_batch(rel.arena, rel.off, nthreads=8)
        for sh in range(len(shapes)):
            got = ag.sig_compute(D, shape=sh).cpu().numpy().view(np.uint64)
            bad = np.nonzero(got != want)[0]
            assert bad.size == 0, (shapes[sh], bad[:5].tolist())
            got2 = ag.sig_compute(D, shape=sh, n_components=2).cpu().numpy().view(np.uint64)
            assert np.array_equal(got2, want & mask), shapes[sh]
    D = ag.DeviceRelation.from_host(rels[0].arena, rels[0].off, rels[0].ids)
    for bad_shape in (-1, len(shapes)):
        with pytest.raises(ag.AlgsigError):
            ag.sig_compute(D, shape=bad_shape)


def test_mixed_length_runs_at_every_shape(cuda):
    """A relation above the size from which the warps' shares are cut by work
    (2^19 keys; a key counts its bytes + a fixed cost) whose key lengths change
    in runs (tens of thousands of 0-16-byte keys, two thousand of 4-8 KB,
    tens of thousands of 256-1024 bytes), so that the cuts fall inside and
    between runs of very different work per byte, garbage after the last key:
    every launch shape gives the oracle's signatures."""
    ag = cuda
    rng = np.random.default_rng(46)
    runs = [(80_000, 0, 16), (2_000, 4096, 8192), (80_000, 0, 16), (60_000, 256, 1024), (80_000, 1, 8),
            (2_000, 4096, 8192), (80_000, 0, 16), (60_000, 256, 1024), (80_000, 0, 16), (2_000, 4096, 8192)]
    lens = np.concatenate([rng.integers(lo, hi + 1, n) for n, lo, hi in runs]).astype(np.uint64)
    assert lens.size >= 1 << 19
    off = np.zeros(lens.size + 1, np.uint64)
    off[1:] = np.cumsum(lens)
    arena = rng.integers(0, 256, int(off[-1]) + 64, dtype=np.uint8)
    rel = workloads.Relation(arena, off, np.arange(lens.size, dtype=np.uint32))
    D = ag.DeviceRelation.from_host(rel.arena, rel.off, rel.ids)
    want = oracle.sig_batch(rel.arena, rel.off, nthreads=8)
    for sh in range(len(ag.sig_shapes())):
        got = ag.sig_compute(D, shape=sh).cpu().numpy().view(np.uint64)
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (sh, bad[:5].tolist())


@pytest.mark.parametrize("block_bytes", [16, 32, 48, 256, 4096])
def test_cumulative_signatures(cuda, block_bytes):
    """as_sig_prefix_offsets / as_sig_prefixes against the oracle's definition:
    the layout (an exclusive scan of max(1, ceil(len / B))) and every prefix
    signature, for keys of 0..100 bytes, around the 256- and 512-byte marks and
    longer, at every alignment, and on a scaled large-workload relation."""
    ag = cuda
    rng = random.Random(block_bytes)
    keys = [bytes(rng.randrange(256) for _ in range(n)) for n in
            list(range(0, 101)) + [255, 256, 257, 511, 512, 513, 1023, 5000, 20000]]
    rels = [relation_garbage_tail(interleave_gaps(keys, seed=s), seed=s) for s in range(2)]
    rels.append(workloads.generate(workloads.CONFIGS["large"].scaled(500, 3000)).S)
    for rel in rels:
        D = ag.DeviceRelation.from_host(rel.arena, rel.off, rel.ids)
        pref, out = ag.sig_prefixes(D, block_bytes)
        pref = pref.cpu().numpy()
        out = out.cpu().numpy().view(np.uint64)
        lens = np.diff(rel.off.astype(np.int64))
        cnt = np.maximum(1, (lens + block_bytes - 1) // block_bytes)
        assert np.array_equal(pref, np.concatenate([[0], np.cumsum(cnt)]))
        for i in range(rel.n):
            want = oracle.sig_prefixes(rel.key(i), block_bytes)
            assert out[pref[i]:pref[i + 1]].tolist() == want, (i, int(lens[i]))
    with pytest.raises(ag.AlgsigError):
        ag.sig_prefixes(ag.DeviceRelation.from_host(rels[0].arena, rels[0].off, rels[0].ids), 24)


def test_byte_symbol_signatures_gf8(cuda):
    """as_sig_compute_gf8 against the oracle's GF(2^8) definition: every
    alignment, every short length, keys past the 255-byte exponent wrap, and a
    scaled large-workload relation."""
    ag = cuda
    rng = random.Random(8)
    keys = edge_keys() + [bytes(rng.randrange(256) for _ in range(n)) for n in
                          list(range(0, 70)) + [254, 255, 256, 257, 511, 4097, 9000]]
    rels = [relation_garbage_tail(interleave_gaps(keys, seed=s), seed=s) for s in range(3)]
    rels.append(workloads.generate(workloads.CONFIGS["large"].scaled(1000, 5000)).S)
    for rel in rels:
        D = ag.DeviceRelation.from_host(rel.arena, rel.off, rel.ids)
        got = ag.sig_compute_gf8(D).cpu().numpy().view(np.uint64)
        want = oracle.sig8_batch(rel.arena, rel.off, nthreads=8)
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, f"{bad.size} mismatches, first at key {bad[:5].tolist()}"
