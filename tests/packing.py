"""Relations for the GPU parity tests whose keys start at every byte
alignment and are surrounded by non-zero bytes (neighbouring keys, garbage up
to the 16-byte boundary after the last key), so that every masking path of the
kernels is exercised."""
import random

import numpy as np

import workloads


def relation_garbage_tail(keys, seed=0, ids=None):
    rel = workloads.relation_from_keys(keys, ids)
    rng = random.Random(seed)
    end = int(rel.off[-1])
    for p in range(end, (end + 15) // 16 * 16):
        rel.arena[p] = rng.randrange(1, 256)
    return rel


def interleave_gaps(keys, seed=0):
    """(gap, key, gap, key, ...) with random garbage gaps of 0..16 bytes."""
    rng = random.Random(seed)
    out = []
    for k in keys:
        out.append(bytes(rng.randrange(1, 256) for _ in range(rng.randrange(0, 17))))
        out.append(bytes(k))
    return out
