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


@pytest.mark.parametrize("NT", [1, 2, 3, 7, 32, 79, 128])
def test_each_tile_counted_to_nt_once_in_any_order(NT):
    """The on-chip reduction: every CTA counts itself in for tile I and (off the diagonal) tile
    J; the CTA whose increment returns NT - 1 sums that tile. In any completion order of the
    CTAs, every tile reaches NT exactly once, only after all its NT contributors have written,
    and every count is back at 0 at the end of the launch."""
    pairs = [tile_pair(tp, NT) for tp in range(NT * (NT + 1) // 2)]
    rng = np.random.default_rng(NT)
    for trial in range(5):
        order = rng.permutation(len(pairs)) if trial else np.arange(len(pairs))
        cnt = np.zeros(NT, np.int64)
        written = np.zeros((NT, NT), bool)  # [tile, slot]
        finished = np.zeros(NT, np.int64)
        for k in order:
            I, J = pairs[k]
            written[I, J if I != J else I] = True
            if I != J:
                written[J, I] = True
            for t in ([I] if I == J else [I, J]):
                old = cnt[t]
                cnt[t] += 1
                if old == NT - 1:
                    assert written[t].all()  # every slot of tile t is in place
                    finished[t] += 1
                    cnt[t] = 0
        assert np.all(finished == 1) and np.all(cnt == 0)


@pytest.mark.parametrize("W,n", [(1, 33), (1, 4096), (2, 4097), (2, 8192), (4, 8193), (4, 10240)])
def test_discarded_lines_are_the_tiles_slots(W, n):
    """finish_tile drops the L2 lines of tile t's NT x 4 runs of T doubles: every line it names
    is 128-byte aligned, lies inside the slot's partial buffer and belongs to tile t, and the
    lines of all tiles together cover the buffer once."""
    T = 32 * W
    npad = -(-n // T) * T
    NT = npad // T
    lines_per_run = T // 16
    covered = np.zeros(NT * 4 * npad // 16, np.int32)  # 128-byte lines of one slot's partials
    for t in range(NT):
        for l in range(NT * 4 * lines_per_run):
            run, line = divmod(l, lines_per_run)
            off = run * npad + t * T + 16 * line   # in doubles from the slot's base
            assert (off * 8) % 128 == 0
            assert 0 <= off and off + 16 <= NT * 4 * npad
            assert t * T <= off % npad < (t + 1) * T
            covered[off // 16] += 1
    assert np.all(covered == 1)


@pytest.mark.parametrize("W,n", [(1, 33), (1, 2050), (2, 4097), (4, 10002), (4, 10239)])
def test_finishing_pass_drops_only_its_blocks_lines(W, n):
    """k_pair_finish drops the L2 lines of a deferred slot's partials once its 64-thread block
    has read them: every line it names is 128-byte aligned, lies in the slot's partial buffer
    and holds only bodies of that block, and the blocks together cover each run's first npad
    bodies exactly once (no line is dropped twice or left behind)."""
    T, kBlock = 32 * W, 64
    npad = -(-n // T) * T
    NT = npad // T
    nblk = -(-npad // kBlock)
    lines_per_run = kBlock // 16
    covered = np.zeros(NT * 4 * npad // 16, np.int32)
    for b in range(nblk):
        b0 = b * kBlock
        for l in range(NT * 4 * lines_per_run):
            run, line = divmod(l, lines_per_run)
            if b0 + 16 * line >= npad:
                continue
            off = run * npad + b0 + 16 * line
            assert (off * 8) % 128 == 0
            assert 0 <= off and off + 16 <= NT * 4 * npad
            assert b0 <= off % npad and off % npad + 16 <= min(b0 + kBlock, npad)
            covered[off // 16] += 1
    assert np.all(covered == 1)
