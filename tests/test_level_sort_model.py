"""A model of the level-order sort of k_tree (csrc/prim.cu): a bitonic network over the keys
level * 2^14 + index, where thread work item p of stage (k, j) compares positions
i = 2p - (p mod j) and i + j, ascending when bit k of i is clear. CPU only.
"""
import numpy as np
import pytest


def bitonic_by_pairs(keys):
    key = keys.copy()
    P = len(key)
    k = 2
    while k <= P:
        j = k >> 1
        while j > 0:
            p = np.arange(P // 2)
            i = 2 * p - (p & (j - 1))
            a, b = key[i], key[i + j]
            swap = (a > b) == ((i & k) == 0)
            key[i] = np.where(swap, b, a)
            key[i + j] = np.where(swap, a, b)
            j >>= 1
        k <<= 1
    return key


@pytest.mark.parametrize("P", [1, 2, 4, 8, 64, 1024, 16384])
def test_pairs_cover_each_position_once(P):
    k = 2
    while k <= P:
        j = k >> 1
        while j > 0:
            p = np.arange(P // 2)
            i = 2 * p - (p & (j - 1))
            both = np.concatenate([i, i + j])
            assert np.array_equal(np.sort(both), np.arange(P)), (k, j)
            j >>= 1
        k <<= 1


@pytest.mark.parametrize("n", [1, 2, 3, 17, 600, 4097, 10002])
def test_sorts_level_index_keys(n):
    rng = np.random.default_rng(n)
    level = rng.integers(0, 200, n)
    P = 1
    while P < n:
        P <<= 1
    keys = np.full(P, 0xFFFFFFFF, np.uint64)
    keys[:n] = (level.astype(np.uint64) << np.uint64(14)) | np.arange(n, dtype=np.uint64)
    out = bitonic_by_pairs(keys)
    bylev = (out[:n] & np.uint64(0x3FFF)).astype(np.int64)
    assert np.array_equal(bylev, np.lexsort((np.arange(n), level)))
