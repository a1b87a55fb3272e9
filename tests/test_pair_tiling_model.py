"""A model of the symmetric pair tiling of k_pair_tiles (csrc/pair.cu): the mapping of a
linear CTA index to an upper-triangle tile pair (I, J), and the partial-sum slots the CTAs
write. CPU only.

The kernel finds the row I of tile pair tp with a float square root and then corrects it
with integer steps; CTA (I, J) writes its i-side sums into slot J of tile I's bodies and its
j-side sums into slot I of tile J's bodies (a diagonal CTA writes slot I once). The finish
pass adds the NT slots of every body, so each (tile, slot) must be written exactly once.
"""
import numpy as np
import pytest


def tile_pair(tp, NT):
    """(I, J) of upper-triangle tile pair tp: rows of length NT - I, float32 first guess."""
    b = np.float32(NT) + np.float32(0.5)
    disc = np.maximum(b * b - np.float32(2.0) * np.float32(tp), np.float32(0.0))
    i = int(np.floor(b - np.sqrt(disc, dtype=np.float32)))
    i = max(0, min(i, NT - 1))

    def start(r):
        return r * NT - (r * (r - 1)) // 2

    while i > 0 and start(i) > tp:
        i -= 1
    while i + 1 < NT and start(i + 1) <= tp:
        i += 1
    return i, i + (tp - start(i))


@pytest.mark.parametrize("NT", list(range(1, 130)) + [160, 200, 255, 256, 320, 321, 512])
def test_every_tile_pair_exactly_once(NT):
    seen = np.zeros((NT, NT), np.int32)
    for tp in range(NT * (NT + 1) // 2):
        I, J = tile_pair(tp, NT)
        assert 0 <= I <= J < NT, (tp, I, J)
        seen[I, J] += 1
    assert np.array_equal(seen, np.triu(np.ones((NT, NT), np.int32)))


@pytest.mark.parametrize("NT", [1, 2, 3, 7, 32, 79, 128])
def test_every_partial_slot_written_once(NT):
    writes = np.zeros((NT, NT), np.int32)   # [tile of the bodies, slot]
    for tp in range(NT * (NT + 1) // 2):
        I, J = tile_pair(tp, NT)
        if I == J:
            writes[I, I] += 1
        else:
            writes[I, J] += 1               # i-side sums of tile I's bodies
            writes[J, I] += 1               # j-side sums of tile J's bodies
    assert np.all(writes == 1)
